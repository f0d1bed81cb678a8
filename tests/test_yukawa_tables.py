"""The library's Yukawa tables (host plan math, no device) against the oracle's
independent implementation of the same formulas (Sec. 3.7): translation
weights of every level, root weights, and the residual polynomials of the
mollified kernel, plus argument checks of the Yukawa plan.
"""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def dmk():
    from paper_2308_00292_gb300 import build, dmk as m
    build.build()
    m.lib()
    return m


def host_plan(dmk, eps, lam=1.0):
    return dmk.Plan(eps, flags=dmk.FLAG_HOST_ONLY, kernel=dmk.DMK_YUKAWA, lam=lam)


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
@pytest.mark.parametrize("lam_unit", [0.05, 3.0, 40.0])
def test_translation_weights(dmk, oracle_mod, eps, lam_unit):
    plan = host_plan(dmk, eps)
    prm = plan.params()
    op = oracle_mod.params(eps=eps, lam=lam_unit)
    nf = prm["nf"]
    s = np.arange(3 * nf * nf + 1)
    for level in (0, 2, 7):
        w = plan.yukawa_table(lam_unit, level, 0)
        h = oracle_mod.h(op, level)
        ref = (h / (2 * np.pi)) ** 3 * oracle_mod.kernel(op, oracle_mod.DHAT, level, h * np.sqrt(s))
        # relative to the weights' scale at small lambda (large lambda R makes
        # them tiny: psi far beyond 1)
        scale = np.abs(plan.yukawa_table(0.05, level, 0)).max()
        assert np.abs(w - ref).max() <= 1e-11 * max(np.abs(ref).max(), scale), level


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
@pytest.mark.parametrize("lam_unit", [0.05, 3.0, 40.0])
def test_root_weights(dmk, oracle_mod, eps, lam_unit):
    plan = host_plan(dmk, eps)
    n0 = plan.params()["n0"]
    op = oracle_mod.params(eps=eps, lam=lam_unit)
    hW = oracle_mod.hW(op)
    s = np.arange(3 * n0 * n0 + 1)
    ww = plan.yukawa_table(lam_unit, 0, 1)
    ref = (hW / (2 * np.pi)) ** 3 * oracle_mod.kernel(op, oracle_mod.WHAT, 0, hW * np.sqrt(s))
    scale = np.abs(plan.yukawa_table(0.05, 0, 1)).max()
    assert np.abs(ww - ref).max() <= 1e-11 * max(np.abs(ref).max(), scale)


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
@pytest.mark.parametrize("lam_unit", [0.05, 3.0, 40.0])
def test_residual_polynomials(dmk, oracle_mod, eps, lam_unit):
    """q_l(t) / R_l reproduces the oracle's mollified kernel S_l(r), r = R_l sqrt t,
    within the fit tolerance 2e-2 eps S_l(0) (or 2e-2 eps / R_l where lambda R_l
    is so large that the mollified kernel is negligible: the kernel then lies
    in the residual)."""
    plan = host_plan(dmk, eps)
    op = oracle_mod.params(eps=eps, lam=lam_unit)
    t = np.linspace(0.0, 1.0, 41)
    for level in (0, 3, 9):
        R = 2.0 ** -level
        mono = plan.yukawa_table(lam_unit, level, 2)
        q = np.polynomial.polynomial.polyval(2 * t - 1, mono) / R
        ref = oracle_mod.kernel(op, oracle_mod.S_MOLLIFIED, level, R * np.sqrt(t))
        assert np.abs(q - ref).max() <= 3e-2 * eps * max(abs(ref[0]), 1.0 / R), level


def test_yukawa_plan_arguments(dmk):
    L = dmk.lib()
    h = ctypes.c_void_p()
    for lam in (0.0, -1.0, float("nan"), float("inf")):
        o = dmk.Opts(kernel_param=lam, flags=dmk.FLAG_HOST_ONLY)
        assert L.dmk_plan(dmk.DMK_YUKAWA, 3, 1e-6, ctypes.byref(o), ctypes.byref(h)) == 1
    o = dmk.Opts(kernel_param=2.0, flags=dmk.FLAG_HOST_ONLY)
    assert L.dmk_plan(dmk.DMK_YUKAWA, 2, 1e-6, ctypes.byref(o), ctypes.byref(h)) == 2
    lap = dmk.Plan(1e-6, flags=dmk.FLAG_HOST_ONLY)
    with pytest.raises(dmk.DMKError):
        lap.yukawa_table(1.0, 0, 0)
