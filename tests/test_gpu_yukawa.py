"""GPU parity of the Yukawa kernel exp(-lambda r)/r (Sec. 3.7) through the C ABI.

FP64 path against the oracle's DMK on the same tree: the far part (the
per-level weights and the root term are the same formulas, evaluated by two
independent codes) to 1e-10 relative, the near part within the residual
polynomial's fit (2e-2 eps of the mollifier), within 2e-1 eps, as is the total; and
against the direct Yukawa sum within eps.  Mixed precision against the direct
sum within 1e-6.  The unit-box map must carry lambda S, and what the path does
not support must be refused.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(dmk, x, q, y=None, **kw):
    with dmk.Plan(kernel=dmk.DMK_YUKAWA, **kw) as plan:
        return plan.eval(dev(x), dev(q), None if y is None else dev(y)).cpu().numpy()


CASES = {
    "uniform": lambda: inputs.uniform_cube(5000, seed=901),
    "clustered": lambda: inputs.clustered(6000, seed=902, nclusters=5),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("lam,eps,bar", [(1.0, 1e-6, 1.0), (10.0, 1e-6, 1.0), (10.0, 1e-9, 1.0), (40.0, 1e-9, 1.5)])
def test_fp64_matches_oracle(dmk, oracle_mod, case, lam, eps, bar):
    """Against the direct sum: within eps up to lambda S = 10; at lambda S = 40
    the residual kernels of the coarse levels (lambda R_l >= 10) keep tails of
    ~1e-5 S_l(0) beyond R_l and the method itself (the oracle) reaches 1.1 eps,
    so the bar there is 1.5 eps."""
    x, q = CASES[case]()
    p = dmk.Plan(kernel=dmk.DMK_YUKAWA, eps=eps, precision=0, lam=lam, flags=dmk.FLAG_HOST_ONLY).params()["p"]
    _, far, near = oracle_mod.dmk(x, q, eps=eps, leaf_cap=60, lam=lam, parts=True, p=p)
    uf = run(dmk, x, q, eps=eps, leaf_cap=60, precision=0, lam=lam, flags=dmk.FLAG_FAR_ONLY)
    un = run(dmk, x, q, eps=eps, leaf_cap=60, precision=0, lam=lam, flags=dmk.FLAG_NEAR_ONLY)
    u = run(dmk, x, q, eps=eps, leaf_cap=60, precision=0, lam=lam)
    assert rel(uf, far) < 1e-10
    assert rel(un, near) < 2e-1 * eps
    assert rel(u, far + near) < 2e-1 * eps
    assert rel(u, oracle_mod.direct(x, q, lam=lam)) < bar * eps


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("lam", [1.0, 10.0])
def test_mixed_matches_direct(dmk, oracle_mod, case, lam):
    x, q = CASES[case]()
    u = run(dmk, x, q, eps=1e-6, leaf_cap=60, precision=1, lam=lam)
    assert rel(u, oracle_mod.direct(x, q, lam=lam)) < 1e-6


def test_separate_targets(dmk, oracle_mod):
    x, q = inputs.uniform_cube(4000, seed=903)
    y = np.random.default_rng(904).random((1500, 3))
    u = run(dmk, x, q, y, eps=1e-6, leaf_cap=60, precision=1, lam=5.0)
    assert rel(u, oracle_mod.direct(x, q, y, lam=5.0)) < 1e-6


def test_lambda_scales_with_the_box(dmk):
    """(s x, lambda / s) maps to the same unit box with the same lambda S:
    potentials scale by 1/s."""
    x, q = inputs.clustered(5000, seed=905, nclusters=3)
    s = 16.0
    u1 = run(dmk, x, q, eps=1e-6, leaf_cap=60, precision=0, lam=8.0)
    u2 = run(dmk, s * x - 2.0, q, eps=1e-6, leaf_cap=60, precision=0, lam=8.0 / s)
    assert rel(s * u2, u1) < 1e-12


def test_table_cache_follows_lambda_s(dmk, oracle_mod):
    """One plan, two clouds of different extent: the second evaluation must use
    tables for its own lambda S."""
    x, q = inputs.uniform_cube(3000, seed=906)
    with dmk.Plan(kernel=dmk.DMK_YUKAWA, eps=1e-6, leaf_cap=60, precision=1, lam=6.0) as plan:
        u1 = plan.eval(dev(x), dev(q)).cpu().numpy()
        u2 = plan.eval(dev(3.0 * x), dev(q)).cpu().numpy()
    assert rel(u1, oracle_mod.direct(x, q, lam=6.0)) < 1e-6
    assert rel(u2, oracle_mod.direct(3.0 * x, q, lam=6.0)) < 1e-6


def test_unsupported_combinations(dmk):
    x, q = inputs.uniform_cube(500, seed=907)
    with dmk.Plan(kernel=dmk.DMK_YUKAWA, eps=1e-6, lam=2.0) as plan:
        with pytest.raises(dmk.DMKError) as e:
            plan.eval_grad(dev(x), dev(q))
        assert e.value.code == 2
        with pytest.raises(dmk.DMKError) as e:
            plan.eval_batch(dev(x), dev(q), [0, 200, 500])
        assert e.value.code == 2
        # a single-system batch is the plain evaluation
        u = plan.eval_batch(dev(x), dev(q), [0, 500]).cpu().numpy()
        assert np.all(np.isfinite(u))


def test_fp64_separate_targets_match_oracle(dmk, oracle_mod):
    x, q = inputs.clustered(4000, seed=908, nclusters=3)
    y = np.random.default_rng(909).random((1200, 3))
    u = run(dmk, x, q, y, eps=1e-9, leaf_cap=60, precision=0, lam=7.0)
    ref = oracle_mod.dmk(x, q, y, eps=1e-9, leaf_cap=60, lam=7.0)
    assert rel(u, ref) < 2e-1 * 1e-9
    assert rel(u, oracle_mod.direct(x, q, y, lam=7.0)) < 1e-9
