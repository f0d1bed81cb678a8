"""The leaf-capacity autotuner (dmk_tune_leaf_cap).

The capacity n_s moves work between the near and the far field but leaves the
method's accuracy to p and nf (Table 1), so after tuning the evaluation must
still reach the direct sum within eps, and the plan must keep the fastest
candidate it measured.
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


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_plan_keeps_the_fastest_candidate_and_its_accuracy(dmk, oracle_mod, precision):
    x, q = inputs.clustered(20000, seed=611, nclusters=4)
    xd, qd = dev(x), dev(q)
    with dmk.Plan(eps=1e-6, precision=precision) as plan:
        cands = [40, 120, 300]
        best, times = plan.tune_leaf_cap(xd, qd, candidates=cands, reps=2)
        assert best in cands
        assert all(t > 0 for t in times.values())
        assert times[best] == min(times.values())
        assert plan.params()["leaf_cap"] == best
        u = plan.eval(xd, qd).cpu().numpy()
        # the next evaluation builds its tree with the tuned capacity
        assert plan.stats()["n_leaves"] > 0
    ref = oracle_mod.direct(x, q)
    assert rel(u, ref) < 1e-6


def test_default_candidates(dmk):
    x, q = inputs.uniform_cube(30000, seed=612)
    with dmk.Plan(eps=1e-6, precision=1) as plan:
        best, times = plan.tune_leaf_cap(dev(x), dev(q))
        assert best in (64, 100, 140, 200, 280, 400, 560)
        assert len(times) == 7 and times[best] == min(times.values())


def test_separate_targets(dmk, oracle_mod):
    x, q = inputs.uniform_cube(8000, seed=613)
    y = np.random.default_rng(614).random((3000, 3))
    with dmk.Plan(eps=1e-6, precision=1) as plan:
        best, _ = plan.tune_leaf_cap(dev(x), dev(q), dev(y), candidates=[50, 200], reps=1)
        u = plan.eval(dev(x), dev(q), dev(y)).cpu().numpy()
    assert best in (50, 200)
    assert rel(u, oracle_mod.direct(x, q, y)) < 1e-6


def test_invalid_candidates_leave_the_plan_unchanged(dmk):
    x, q = inputs.uniform_cube(1000, seed=615)
    with dmk.Plan(eps=1e-6, precision=1, leaf_cap=90) as plan:
        for bad in ([0, 100], [-5], [1 << 21]):
            with pytest.raises(dmk.DMKError) as e:
                plan.tune_leaf_cap(dev(x), dev(q), candidates=bad)
            assert e.value.code == 1
        with pytest.raises(dmk.DMKError):
            plan.tune_leaf_cap(dev(x), dev(q), candidates=[100], reps=1000)
        assert plan.params()["leaf_cap"] == 90


def test_batch_tuner(dmk, oracle_mod):
    x, q, off = inputs.batch(12, seed=616, n_lo=300, n_hi=4000)
    xd, qd = dev(x), dev(q)
    with dmk.Plan(eps=1e-6, precision=1) as plan:
        best, times = plan.tune_leaf_cap_batch(xd, qd, off, candidates=[30, 90, 250], reps=1)
        assert best in (30, 90, 250)
        assert times[best] == min(times.values())
        assert plan.params()["leaf_cap"] == best
        u = plan.eval_batch(xd, qd, off).cpu().numpy()
    for s in range(len(off) - 1):
        a, b = off[s], off[s + 1]
        assert rel(u[a:b], oracle_mod.direct(x[a:b], q[a:b])) < 1e-6, s
