"""GPU parity of the gradient pass (dmk_eval_grad) and of the differentiable
potential built on it.

Against the oracle's differentiated DMK on the same tree (FP64): the far
gradients differ by rounding only; the near gradients by the derivative of the
residual polynomial (fit to 1e-3 eps q(0)), within 2e-3 eps of their maximum;
the total within 1e-2 eps in rel-L2.  Against the direct-sum gradient (the
definition): 3 eps for the FP64 path.  The mixed path's far gradient carries
the single-precision Chebyshev coefficients through T_n' (up to p^2 larger than
T_n), so its bar against the direct sum is 3e-6 at eps = 1e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2308_00292_gb300 import inputs  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def dmk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_00292_gb300 import dmk as m
    m.lib()
    return m


def run_grad(dmk, x, q, y=None, **kw):
    with dmk.Plan(**kw) as plan:
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
        yd = None if y is None else torch.from_numpy(np.ascontiguousarray(y)).cuda()
        u, g = plan.eval_grad(xd, qd, yd)
        return u.cpu().numpy(), g.cpu().numpy()


CASES = {
    "uniform": lambda: inputs.uniform_cube(6000, seed=201),
    "clustered": lambda: inputs.clustered(8000, seed=202, nclusters=6),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_fp64_gradient_matches_oracle(dmk, oracle_mod, case, eps):
    x, q = CASES[case]()
    _, go, gf_o, gn_o = oracle_mod.dmk_grad(x, q, eps=eps, leaf_cap=60, parts=True)
    u, g = run_grad(dmk, x, q, eps=eps, leaf_cap=60, precision=0)
    _, gf = run_grad(dmk, x, q, eps=eps, leaf_cap=60, precision=0, flags=dmk.FLAG_FAR_ONLY)
    _, gn = run_grad(dmk, x, q, eps=eps, leaf_cap=60, precision=0, flags=dmk.FLAG_NEAR_ONLY)
    assert rel(gf, gf_o) < 1e-12
    assert np.abs(gn - gn_o).max() < 2e-3 * eps * np.abs(gn_o).max()
    assert rel(g, go) < 1e-2 * eps
    assert rel(g, oracle_mod.direct_grad(x, q)) < 3 * eps
    # the potentials of the gradient pass are those of the plain pass
    with dmk.Plan(eps, precision=0, leaf_cap=60) as plan:
        u0 = plan.eval(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()).cpu().numpy()
    assert np.array_equal(u, u0)


@pytest.mark.parametrize("case", sorted(CASES))
def test_mixed_gradient_matches_direct(dmk, oracle_mod, case):
    x, q = CASES[case]()
    _, g = run_grad(dmk, x, q, eps=1e-6, leaf_cap=60, precision=1)
    assert rel(g, oracle_mod.direct_grad(x, q)) < 3e-6


def test_gradient_separate_targets(dmk, oracle_mod):
    x, q = inputs.clustered(5000, seed=205, nclusters=4)
    y, _ = inputs.uniform_cube(700, seed=206)
    _, g = run_grad(dmk, x, q, y, eps=1e-9, leaf_cap=80, precision=0)
    assert rel(g, oracle_mod.direct_grad(x, q, y)) < 3e-9


def test_autograd_matches_direct_sums(dmk, oracle_mod):
    """L = sum_i w_i u_i: dL/drho = the potential of w (symmetric kernel),
    dL/dx_k = w_k grad u(x_k) + rho_k grad v(x_k) with v the potential of w."""
    x, q = inputs.uniform_cube(3000, seed=401)
    w = np.random.default_rng(402).standard_normal(len(x))
    plan = dmk.Plan(1e-9, precision=0, leaf_cap=80)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    qt = torch.from_numpy(q).cuda().requires_grad_(True)
    L = (torch.from_numpy(w).cuda() * dmk.potential(plan, xt, qt)).sum()
    L.backward()
    assert rel(qt.grad.cpu().numpy(), oracle_mod.direct(x, w)) < 3e-9
    gx_ref = w[:, None] * oracle_mod.direct_grad(x, q) + q[:, None] * oracle_mod.direct_grad(x, w)
    assert rel(xt.grad.cpu().numpy(), gx_ref) < 3e-9
    plan.close()


def test_autograd_central_differences(dmk):
    """Central differences (h = 1e-4) of L = sum_i w_i u_i in 64 random
    coordinates agree with the backward pass (FP64, eps 1e-9)."""
    x, q = inputs.uniform_cube(3000, seed=411)
    w = np.random.default_rng(412).standard_normal(len(x))
    wt = torch.from_numpy(w).cuda()
    qt = torch.from_numpy(q).cuda()
    plan = dmk.Plan(1e-9, precision=0, leaf_cap=80)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    (wt * dmk.potential(plan, xt, qt)).sum().backward()
    gx = xt.grad.cpu().numpy()
    rng = np.random.default_rng(413)
    pts, dims = rng.choice(len(x), 64, replace=False), rng.integers(0, 3, 64)
    h = 1e-4
    fd = []
    for i, d in zip(pts, dims):
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        lp = float((wt * plan.eval(torch.from_numpy(xp).cuda(), qt)).sum())
        lm = float((wt * plan.eval(torch.from_numpy(xm).cuda(), qt)).sum())
        fd.append((lp - lm) / (2 * h))
    ad = gx[pts, dims]
    assert np.linalg.norm(np.array(fd) - ad) < 1e-4 * np.linalg.norm(ad)
    plan.close()


def test_autograd_float32_inputs(dmk, oracle_mod):
    """The differentiable workload takes FP32 positions and charges: they are
    widened exactly at the boundary, the gradients come back in FP32 and match
    the direct sums of the widened inputs (mixed path, eps 1e-6)."""
    x32 = inputs.uniform_cube(4000, seed=421)[0].astype(np.float32)
    q32 = inputs.uniform_cube(4000, seed=422)[1].astype(np.float32)
    x, q = x32.astype(np.float64), q32.astype(np.float64)
    w = np.random.default_rng(423).standard_normal(len(x))
    plan = dmk.Plan(1e-6, precision=dmk.DMK_MIXED, leaf_cap=80)
    xt = torch.from_numpy(x32).cuda().requires_grad_(True)
    qt = torch.from_numpy(q32).cuda().requires_grad_(True)
    u = dmk.potential(plan, xt, qt)
    assert u.dtype == torch.float64
    (torch.from_numpy(w).cuda() * u).sum().backward()
    assert xt.grad.dtype == torch.float32 and qt.grad.dtype == torch.float32
    assert rel(u.detach().cpu().numpy(), oracle_mod.direct(x, q)) < 1e-6
    assert rel(qt.grad.cpu().numpy().astype(np.float64), oracle_mod.direct(x, w)) < 2e-6
    gx_ref = w[:, None] * oracle_mod.direct_grad(x, q) + q[:, None] * oracle_mod.direct_grad(x, w)
    assert rel(xt.grad.cpu().numpy().astype(np.float64), gx_ref) < 3e-6
    plan.close()


def test_autograd_separate_targets(dmk, oracle_mod):
    """Separate targets: dL/dy_j = rho_j grad v(y_j) at the sources and
    dL/dx_i = w_i grad u(x_i) at the targets, both formed by
    dmk_adjoint_combine (FP64, eps 1e-9)."""
    y, q = inputs.clustered(3000, seed=431, nclusters=3)
    x, _ = inputs.uniform_cube(800, seed=432)
    w = np.random.default_rng(433).standard_normal(len(x))
    plan = dmk.Plan(1e-9, precision=0, leaf_cap=80)
    yt = torch.from_numpy(y).cuda().requires_grad_(True)
    qt = torch.from_numpy(q).cuda().requires_grad_(True)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    (torch.from_numpy(w).cuda() * dmk.potential(plan, yt, qt, xt)).sum().backward()
    assert rel(qt.grad.cpu().numpy(), oracle_mod.direct(x, w, y)) < 3e-9
    assert rel(yt.grad.cpu().numpy(), q[:, None] * oracle_mod.direct_grad(x, w, y)) < 3e-9
    assert rel(xt.grad.cpu().numpy(), w[:, None] * oracle_mod.direct_grad(y, q, x)) < 3e-9
    plan.close()


def test_adjoint_combine_rows(dmk):
    """out_i = w1_i g1_i + w2_i g2_i, and each term alone, bit for bit."""
    rng = np.random.default_rng(441)
    n = 1001
    w1, w2 = rng.standard_normal(n), rng.standard_normal(n)
    g1, g2 = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    T = [torch.from_numpy(a).cuda() for a in (w1, g1, w2, g2)]
    both = dmk.adjoint_combine(*T).cpu().numpy()
    one = dmk.adjoint_combine(T[0], T[1]).cpu().numpy()
    assert np.array_equal(one, w1[:, None] * g1)
    assert np.allclose(both, w1[:, None] * g1 + w2[:, None] * g2, rtol=1e-15, atol=1e-15)
