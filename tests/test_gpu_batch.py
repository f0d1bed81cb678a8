"""GPU parity of the batched evaluation (dmk_eval_batch): many independent
systems in one pass, through one forest.

Each system is its own problem: its tree must be the oracle's tree of that
system alone (bit-exact), its FP64 potentials the oracle's DMK of that system
(1e-2 eps, the single-system bar) and the direct sum within eps, and the mixed
path's within 1e-6 of the direct sum.  A batch must give what separate
evaluations of its systems give.
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


def run_batch(dmk, x, q, off, **kw):
    with dmk.Plan(**kw) as plan:
        u = plan.eval_batch(dev(x), dev(q), off).cpu().numpy()
        lev, cell = plan.tree()
        st = plan.stats()
    return u, lev, cell, st


def run_one(dmk, x, q, **kw):
    with dmk.Plan(**kw) as plan:
        return plan.eval(dev(x), dev(q)).cpu().numpy()


@pytest.fixture(scope="module")
def small_batch():
    # 14 systems of 100 .. 3000 points: some are a single leaf at leaf_cap 60,
    # others several levels deep; half uniform, half one Gaussian cluster
    return inputs.batch(14, seed=701, n_lo=100, n_hi=3000)


def test_forest_is_the_oracle_tree_of_every_system(dmk, oracle_mod, small_batch):
    x, q, off = small_batch
    _, lev, cell, st = run_batch(dmk, x, q, off, eps=1e-6, leaf_cap=60)
    assert st["n_points"] == off[-1]
    for s in range(len(off) - 1):
        a, b = off[s], off[s + 1]
        olev, ocell = oracle_mod.tree(x[a:b], eps=1e-6, leaf_cap=60)
        assert np.array_equal(lev[a:b], olev), s
        assert np.array_equal(cell[a:b], ocell), s


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_fp64_batch_matches_oracle_per_system(dmk, oracle_mod, small_batch, eps):
    x, q, off = small_batch
    u, _, _, _ = run_batch(dmk, x, q, off, eps=eps, leaf_cap=60, precision=0)
    for s in range(len(off) - 1):
        a, b = off[s], off[s + 1]
        ref = oracle_mod.dmk(x[a:b], q[a:b], eps=eps, leaf_cap=60)
        assert rel(u[a:b], ref) < 1e-2 * eps, s
        assert rel(u[a:b], oracle_mod.direct(x[a:b], q[a:b])) < eps, s


def test_mixed_batch_matches_direct_per_system(dmk, oracle_mod, small_batch):
    x, q, off = small_batch
    u, _, _, _ = run_batch(dmk, x, q, off, eps=1e-6, leaf_cap=60, precision=1)
    for s in range(len(off) - 1):
        a, b = off[s], off[s + 1]
        assert rel(u[a:b], oracle_mod.direct(x[a:b], q[a:b])) < 1e-6, s


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_separate_evaluations(dmk, small_batch, precision):
    """The forest holds each system's own tree and every kernel treats a box
    the same way whichever system it belongs to."""
    x, q, off = small_batch
    u, _, _, _ = run_batch(dmk, x, q, off, eps=1e-6, leaf_cap=60, precision=precision)
    for s in range(len(off) - 1):
        a, b = off[s], off[s + 1]
        one = run_one(dmk, x[a:b], q[a:b], eps=1e-6, leaf_cap=60, precision=precision)
        assert np.abs(u[a:b] - one).max() <= 1e-13 * np.abs(one).max(), s


def test_systems_do_not_see_each_other(dmk, small_batch):
    """Moving and recharging one system leaves every other system's potentials
    unchanged."""
    x, q, off = small_batch
    u0, _, _, _ = run_batch(dmk, x, q, off, eps=1e-6, leaf_cap=60, precision=1)
    x2, q2 = x.copy(), q.copy()
    a, b = off[3], off[4]
    x2[a:b] = 5.0 + 0.1 * x2[a:b]
    q2[a:b] = -3.0 * q2[a:b]
    u1, _, _, _ = run_batch(dmk, x2, q2, off, eps=1e-6, leaf_cap=60, precision=1)
    keep = np.ones(len(x), bool)
    keep[a:b] = False
    assert np.array_equal(u0[keep], u1[keep])
    # the moved system: same shape at 1/10 the size, charges times -3 (its unit
    # coordinates differ by the rounding of the move)
    assert rel(u1[a:b], -30.0 * u0[a:b]) < 2e-6


def test_edge_systems(dmk, oracle_mod):
    """Empty systems, one point, two points, coincident points, and a deep
    system next to single-leaf ones."""
    rng = np.random.default_rng(702)
    parts = [np.zeros((0, 3)), rng.random((1, 3)), rng.random((2, 3)), np.repeat(rng.random((1, 3)), 5, axis=0),
             np.zeros((0, 3)), inputs.clustered(4000, seed=703, nclusters=2)[0], rng.random((70, 3))]
    x = np.vstack(parts)
    q = rng.uniform(-1, 1, len(x))
    off = np.concatenate([[0], np.cumsum([len(p) for p in parts])])
    for precision, bar in ((0, 1e-6), (1, 1e-6)):
        u, _, _, _ = run_batch(dmk, x, q, off, eps=1e-6, leaf_cap=50, precision=precision)
        # a lone point, and points that all coincide, feel nothing: the smooth
        # far part at r = 0 and the residual's r = 0 correction cancel to the
        # method's precision
        for s in (1, 3):
            a, b = off[s], off[s + 1]
            assert np.abs(u[a:b]).max() < 1e-5 * np.abs(q[a:b]).sum(), (precision, s)
        for s in (2, 5, 6):
            a, b = off[s], off[s + 1]
            ref = oracle_mod.direct(x[a:b], q[a:b])
            assert rel(u[a:b], ref) < bar, (precision, s)


def test_single_system_batch_equals_eval(dmk, oracle_mod):
    x, q = inputs.uniform_cube(5000, seed=704)
    u, _, _, _ = run_batch(dmk, x, q, [0, len(x)], eps=1e-6, leaf_cap=80, precision=0)
    one = run_one(dmk, x, q, eps=1e-6, leaf_cap=80, precision=0)
    assert np.abs(u - one).max() <= 1e-13 * np.abs(one).max()


def test_invalid_offsets(dmk):
    x, q = inputs.uniform_cube(100, seed=705)
    with dmk.Plan(eps=1e-6) as plan:
        for bad in ([1, 100], [0, 60, 40, 100], [0]):
            with pytest.raises(dmk.DMKError) as e:
                plan.eval_batch(dev(x), dev(q), bad)
            assert e.value.code == 1
