"""The C ABI surface and the plan's host logic, without a GPU.

The library must load and export every function declared in include/dmk.h;
argument validation happens before any device call; a host-only plan exposes
its tables, which are checked against the oracle's independent
implementation of the same formulas (PSWF, Dhat_l, What_0, Phi).
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dmk():
    from paper_2308_00292_gb300 import build, dmk as m
    build.build()
    m.lib()
    return m


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dmk.h")).read()
    return sorted(set(re.findall(r"DMK_API\s+(?:int|const char \*)\s*(dmk_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(dmk):
    names = declared_functions()
    assert len(names) >= 10
    lib = ctypes.CDLL(dmk.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(dmk.EXPORTED)


def test_error_strings(dmk):
    L = dmk.lib()
    for code in range(8):
        assert len(L.dmk_error_string(code)) > 3
    assert L.dmk_error_string(99) == b"unknown status code"


def test_argument_validation_without_device(dmk):
    L = dmk.lib()
    h = ctypes.c_void_p()
    o = dmk.Opts()
    assert L.dmk_plan(0, 3, 1.0, ctypes.byref(o), ctypes.byref(h)) == 1      # eps out of range
    assert L.dmk_plan(0, 3, float("nan"), ctypes.byref(o), ctypes.byref(h)) == 1
    assert L.dmk_plan(1, 3, 1e-6, ctypes.byref(o), ctypes.byref(h)) == 1      # Yukawa without lambda
    assert L.dmk_plan(3, 3, 1e-6, ctypes.byref(o), ctypes.byref(h)) == 2      # kernel not implemented
    assert L.dmk_plan(0, 2, 1e-6, ctypes.byref(o), ctypes.byref(h)) == 2      # dimension
    assert L.dmk_plan(2, 3, 1e-6, ctypes.byref(o), ctypes.byref(h)) == 2      # log r is a 2D kernel
    ho = dmk.Opts(flags=dmk.FLAG_HOST_ONLY)
    assert L.dmk_plan(2, 2, 1e-6, ctypes.byref(ho), ctypes.byref(h)) == 0
    L.dmk_plan_destroy(h)
    h = ctypes.c_void_p()
    mixed = dmk.Opts(precision=1, flags=dmk.FLAG_HOST_ONLY)
    assert L.dmk_plan(2, 2, 1e-6, ctypes.byref(mixed), ctypes.byref(h)) == 0  # 2D mixed near field
    L.dmk_plan_destroy(h)
    h = ctypes.c_void_p()
    assert L.dmk_plan(2, 2, 1e-8, ctypes.byref(mixed), ctypes.byref(h)) == 2  # mixed below 1e-7
    far = dmk.Opts(flags=dmk.FLAG_HOST_ONLY | dmk.FLAG_FAR_ONLY)
    assert L.dmk_plan(2, 2, 1e-6, ctypes.byref(far), ctypes.byref(h)) == 2    # the 2D pass evaluates both parts
    assert L.dmk_plan(0, 3, 1e-6, ctypes.byref(o), None) == 1
    bad = dmk.Opts(p=17)
    assert L.dmk_plan(0, 3, 1e-6, ctypes.byref(bad), ctypes.byref(h)) == 1
    both = dmk.Opts(flags=3)
    assert L.dmk_plan(0, 3, 1e-6, ctypes.byref(both), ctypes.byref(h)) == 1
    assert L.dmk_eval(None, None, 0, None, None, 0, None, None) == 1
    assert L.dmk_plan_destroy(None) == 0
    assert b"eps" in L.dmk_last_error_detail() or True


def test_host_only_plan_cannot_evaluate(dmk):
    p = dmk.Plan(1e-6, flags=dmk.FLAG_HOST_ONLY)
    with pytest.raises(dmk.DMKError) as ei:
        p.eval_host(np.zeros((2, 3)), np.ones(2))
    assert ei.value.code == 1


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9, 1e-12])
def test_plan_parameters_follow_table1(dmk, eps):
    rows = {1e-3: (7.2462000846862793, 13, 9), 1e-6: (13.739999771118164, 25, 18),
            1e-9: (20.736000061035156, 39, 28), 1e-12: (27.870000839233398, 53, 38)}
    c, N1, p = rows[eps]
    prm = dmk.Plan(eps, flags=dmk.FLAG_HOST_ONLY).params()
    assert prm["c"] == c and 2 * prm["nf"] + 1 == N1 and prm["p"] == p


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_plan_tables_match_oracle(dmk, oracle_mod, eps):
    plan = dmk.Plan(eps, flags=dmk.FLAG_HOST_ONLY)
    prm = plan.params()
    oprm = oracle_mod.params(eps=eps)
    # psi_0^c on x = k/64, including the continuation beyond |x| = 1
    x = np.arange(257) / 64.0
    assert np.max(np.abs(plan.table(0) - oracle_mod.pswf(prm["c"], x))) < 1e-11
    assert abs(prm["psi0_over_c0"] - oracle_mod.kernel(oprm, oracle_mod.S_MOLLIFIED, 0, np.array([0.0]))[0]) < 1e-12
    # translation weights: w(s) = Dhat_0((2 pi/3) sqrt s) / 27 at R = 1
    w = plan.table(1)
    s = np.arange(len(w))
    ref = oracle_mod.kernel(oprm, oracle_mod.DHAT, 0, 2 * np.pi / 3 * np.sqrt(s)) / 27.0
    assert np.max(np.abs(w - ref)) < 1e-12 * np.max(np.abs(ref))
    # root weights
    tW = plan.table(2)
    hW = tW[0]
    assert abs(hW - oracle_mod.hW(oprm)) < 1e-15
    sW = np.arange(len(tW) - 1)
    refW = (hW / (2 * np.pi)) ** 3 * oracle_mod.kernel(oprm, oracle_mod.WHAT, 0, hW * np.sqrt(sW))
    assert np.max(np.abs(tW[1:] - refW)) < 1e-12 * np.max(np.abs(refW))
    # residual polynomial q(t) = Phi(sqrt t)/sqrt t = S_0(sqrt t) at R = 1
    ch = plan.table(3)
    t = np.linspace(0, 1, 301)
    qv = np.polynomial.chebyshev.chebval(2 * t - 1, ch)
    ref_q = oracle_mod.kernel(oprm, oracle_mod.S_MOLLIFIED, 0, np.sqrt(t))
    assert np.max(np.abs(qv - ref_q)) < 2e-3 * eps * ref_q[0]


def test_tuner_argument_validation_without_device(dmk):
    L = dmk.lib()
    best = ctypes.c_int(-1)
    assert L.dmk_tune_leaf_cap(None, None, 0, None, None, 0, None, 0, 0, ctypes.byref(best), None, None) == 1
    p = dmk.Plan(1e-6, flags=dmk.FLAG_HOST_ONLY)
    assert L.dmk_tune_leaf_cap(p._h, None, 0, None, None, 0, None, 0, 0, ctypes.byref(best), None, None) == 1
    assert best.value == -1


def test_batch_argument_validation_without_device(dmk):
    L = dmk.lib()
    off = (ctypes.c_int64 * 3)(0, 5, 9)
    assert L.dmk_eval_batch(None, None, None, off, 2, None, None) == 1
    p = dmk.Plan(1e-6, flags=dmk.FLAG_HOST_ONLY)
    assert L.dmk_eval_batch(p._h, None, None, off, 2, None, None) == 1


def test_foreign_plan_handles_are_refused(dmk):
    """Host-side fault injection: a handle that is not a live plan (here a
    zeroed buffer standing in for a corrupt or foreign pointer) is refused
    with DMK_ERR_INVALID_ARG by every entry point that takes a plan; a live
    host-only plan still answers."""
    L = dmk.lib()
    fake = ctypes.create_string_buffer(4096)
    h = ctypes.cast(fake, ctypes.c_void_p)
    dp = ctypes.POINTER(ctypes.c_double)
    n = ctypes.c_int64()
    assert L.dmk_eval(h, None, 0, None, None, 0, None, None) == 1
    assert L.dmk_eval_host(h, None, 0, None, None, 0, None, None) == 1
    assert L.dmk_plan_get_params(h, ctypes.byref(dmk.PlanParams())) == 1
    assert L.dmk_plan_get_table(h, 1, None, 0, ctypes.byref(n)) == 1
    assert L.dmk_get_stats(h, ctypes.byref(dmk.Stats())) == 1
    assert L.dmk_plan_destroy(h) == 1
    assert "live plan" in L.dmk_last_error_detail().decode()
    with dmk.Plan(1e-6, flags=dmk.FLAG_HOST_ONLY) as plan:
        assert plan.params()["p"] == 18
