"""GPU parity of the 2D Laplace kernel log r (Sec. 3.7 at lambda = 0 in the
plane) through the C ABI: the FP64 pass against the oracle's 2D pass on the
same quad-tree (the two share the formulas, not the code; the residual's
smooth part is a Chebyshev fit within 1e-3 eps) within 1e-2 eps, and against
the direct sum within eps; separate targets, coincident points, the log S term
of the unit-box map, empty and one-point inputs, the host entry point, the
mixed-precision near field, and the options the 2D pass refuses.
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


def plan_p(dmk, eps):
    """The Chebyshev order the library takes (19 at the 1e-6 row in 2D)."""
    with dmk.Plan(kernel=dmk.DMK_LOG2D, dim=2, eps=eps, flags=dmk.FLAG_HOST_ONLY) as plan:
        return plan.params()["p"]


def run(dmk, x, q, y=None, **kw):
    with dmk.Plan(kernel=dmk.DMK_LOG2D, dim=2, **kw) as plan:
        return plan.eval(dev(x), dev(q), None if y is None else dev(y)).cpu().numpy()


CASES = {
    "disk": lambda: inputs.disk2d(3000, seed=821),
    "circle": lambda: inputs.circle2d(4000, seed=822),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("eps,leaf_cap", [(1e-6, 120), (1e-9, 160), (1e-6, 40)])
def test_matches_oracle_and_direct(dmk, oracle_mod, case, eps, leaf_cap):
    x, q = CASES[case]()
    u = run(dmk, x, q, eps=eps, leaf_cap=leaf_cap)
    ref = oracle_mod.dmk_log2d(x, q, eps=eps, leaf_cap=leaf_cap, p=plan_p(dmk, eps))
    assert rel(u, ref) < 1e-2 * eps
    assert rel(u, oracle_mod.direct_log2d(x, q)) < eps


def test_separate_targets_duplicates_and_scale(dmk, oracle_mod):
    x, q = inputs.circle2d(3000, seed=823)
    y = np.random.default_rng(824).uniform(-1.2, 1.2, size=(1300, 2))
    u = run(dmk, x, q, y, eps=1e-9, leaf_cap=100)
    assert rel(u, oracle_mod.direct_log2d(x, q, y)) < 1e-9
    assert rel(u, oracle_mod.dmk_log2d(x, q, y, eps=1e-9, leaf_cap=100)) < 1e-11
    xd = np.r_[x[:2000], x[:300]]
    qd = np.r_[q[:2000], q[:300]]
    u = run(dmk, xd, qd, eps=1e-9, leaf_cap=100)
    assert rel(u, oracle_mod.direct_log2d(xd, qd)) < 1e-9
    # a power-of-two scale maps to bitwise the same unit-box coordinates, so
    # only the log S term differs (a shift would round the coordinates)
    s = 0.125
    u1 = run(dmk, x, q, eps=1e-9, leaf_cap=100)
    u2 = run(dmk, s * x, q, eps=1e-9, leaf_cap=100)
    assert rel(u2 - np.log(s) * (q.sum() - q), u1) < 1e-13


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_close_pairs_across_scales(dmk, oracle_mod, eps):
    """Separations from 1e-3 down to 1e-150 at the corner of the unit box (the
    map keeps them: x - lo is exact there), so that t = r^2 / R^2 spans the
    residual kernel's table-driven log (t >= 2^-255) and its fallback below."""
    x, q = inputs.disk2d(2000, seed=827)
    x = x - x.min(axis=0) + 0.25
    seps = [1e-3, 1e-8, 1e-20, 1e-35, 1e-45, 1e-80, 1e-150]
    extra = [[0.0, 0.0]] + [[s, 0.0] for s in seps] + [[0.0, s] for s in seps[::2]]
    x = np.r_[x, np.array(extra)]
    q = np.r_[q, np.random.default_rng(828).uniform(-1, 1, len(extra))]
    u = run(dmk, x, q, eps=eps, leaf_cap=60)
    d = oracle_mod.direct_log2d(x, q)
    assert rel(u, d) < eps
    k = len(extra)
    assert np.max(np.abs(u[-k:] - d[-k:]) / np.abs(d[-k:])) < eps
    assert rel(u, oracle_mod.dmk_log2d(x, q, eps=eps, leaf_cap=60, p=plan_p(dmk, eps))) < 1e-2 * eps


def test_small_inputs_and_host_entry(dmk, oracle_mod):
    x, q = inputs.disk2d(2000, seed=825)
    with dmk.Plan(kernel=dmk.DMK_LOG2D, dim=2, eps=1e-6) as plan:
        ud = plan.eval(dev(x), dev(q)).cpu().numpy()
        uh = plan.eval_host(x, q)
        assert np.array_equal(ud, uh)
        assert plan.params()["leaf_cap"] == 120
        # one point: the far field's self term (the root window at r = 0)
        # cancels the removed S_L(0) to the method's accuracy, as in the oracle
        one = plan.eval(dev(x[:1]), dev(q[:1])).cpu().numpy()
        assert abs(one[0]) < 1e-6 * abs(q[0])
        p6 = plan_p(dmk, 1e-6)
        assert one == pytest.approx(oracle_mod.dmk_log2d(x[:1], q[:1], eps=1e-6, p=p6), abs=1e-12)
        two = plan.eval(dev(x[:2]), dev(q[:2])).cpu().numpy()
        r = np.linalg.norm(x[0] - x[1])
        assert two == pytest.approx([q[1] * np.log(r), q[0] * np.log(r)], abs=1e-6)
        assert two == pytest.approx(oracle_mod.dmk_log2d(x[:2], q[:2], eps=1e-6, p=p6), abs=1e-12)
        empty = plan.eval(dev(x[:0]), dev(q[:0]), dev(x[:5])).cpu().numpy()
        assert np.all(empty == 0.0)
    assert rel(ud, oracle_mod.direct_log2d(x, q)) < 1e-6


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("eps,leaf_cap", [(1e-6, 120), (1e-6, 40), (1e-7, 160)])
def test_mixed_near_field(dmk, oracle_mod, case, eps, leaf_cap):
    """The mixed path: FP32 residual pairs from hi/lo leaf-unit offsets, FP64
    far field and sums; within eps of the direct sum, and within a fraction of
    eps of the FP64 pass on the same tree."""
    x, q = CASES[case]()
    um = run(dmk, x, q, eps=eps, leaf_cap=leaf_cap, precision=dmk.DMK_MIXED)
    ud = run(dmk, x, q, eps=eps, leaf_cap=leaf_cap)
    assert rel(um, oracle_mod.direct_log2d(x, q)) < eps
    assert rel(um, ud) < 0.3 * eps
    ref = oracle_mod.dmk_log2d(x, q, eps=eps, leaf_cap=leaf_cap, p=plan_p(dmk, eps))
    assert rel(um, ref) < 0.3 * eps


def test_mixed_close_pairs(dmk, oracle_mod):
    """Separations from 1e-3 to 1e-150 on the mixed path: FP32 pairs down to
    r^2 = 2^-100 in leaf units, FP64 below, coincident points exact."""
    x, q = inputs.disk2d(2000, seed=829)
    x = x - x.min(axis=0) + 0.25
    seps = [1e-3, 1e-5, 1e-8, 1e-12, 1e-20, 1e-45, 1e-150]
    extra = [[0.0, 0.0], [0.0, 0.0]] + [[s, 0.0] for s in seps] + [[0.0, s] for s in seps[::2]]
    x = np.r_[x, np.array(extra)]
    q = np.r_[q, np.random.default_rng(830).uniform(-1, 1, len(extra))]
    um = run(dmk, x, q, eps=1e-6, leaf_cap=60, precision=dmk.DMK_MIXED)
    d = oracle_mod.direct_log2d(x, q)
    assert rel(um, d) < 1e-6
    k = len(extra)
    assert np.max(np.abs(um[-k:] - d[-k:]) / np.abs(d[-k:])) < 1e-6


def test_repeated_evaluations_identical(dmk):
    """The near field's queues and per-lane sums are added in a fixed order, so
    repeated evaluations agree bit for bit, on both paths."""
    x, q = inputs.circle2d(20000, seed=831)
    for prec, eps in ((dmk.DMK_FP64, 1e-8), (dmk.DMK_MIXED, 1e-6)):
        with dmk.Plan(kernel=dmk.DMK_LOG2D, dim=2, eps=eps, precision=prec, leaf_cap=120) as plan:
            xd, qd = dev(x), dev(q)
            u0 = plan.eval(xd, qd).cpu().numpy()
            for _ in range(4):
                assert np.array_equal(plan.eval(xd, qd).cpu().numpy(), u0)


def test_refused_options(dmk):
    x, q = inputs.disk2d(300, seed=826)
    for kw in (dict(precision=dmk.DMK_MIXED, eps=1e-8), dict(flags=dmk.FLAG_FAR_ONLY), dict(dim=3)):
        args = dict(kernel=dmk.DMK_LOG2D, dim=2, eps=1e-6)
        args.update(kw)
        with pytest.raises(dmk.DMKError) as e:
            dmk.Plan(**args)
        assert e.value.code == 2
    with dmk.Plan(kernel=dmk.DMK_LOG2D, dim=2, eps=1e-6) as plan:
        with pytest.raises(dmk.DMKError) as e:
            plan.eval_grad(dev(x), dev(q))
        assert e.value.code == 2
        with pytest.raises(dmk.DMKError) as e:
            plan.eval_batch(dev(x), dev(q), [0, 100, 300])
        assert e.value.code == 2


def _decode3(m):
    ix = iy = iz = 0
    for b in range(21):
        ix |= ((m >> (3 * b)) & 1) << b
        iy |= ((m >> (3 * b + 1)) & 1) << b
        iz |= ((m >> (3 * b + 2)) & 1) << b
    return ix, iy, iz


def test_tree_is_the_oracle_quadtree(dmk, oracle_mod):
    """The points lifted to z = 0 give, through the library's tree builder,
    the oracle's quad-tree: the same leaf level and cell for every point."""
    x, q = inputs.make("circle_disk2d", 6000, 827)
    with dmk.Plan(kernel=dmk.DMK_LOG2D, dim=2, eps=1e-6, leaf_cap=40) as plan:
        plan.eval(dev(x), dev(q))
        lev, cell = plan.tree()
    olev, oix, oiy, _ = oracle_mod.tree_log2d(x, leaf_cap=40)
    assert np.array_equal(lev, olev)
    d = np.array([_decode3(int(c)) for c in cell])
    assert np.array_equal(d[:, 0], oix) and np.array_equal(d[:, 1], oiy)
    assert np.all(d[:, 2] == 0)
