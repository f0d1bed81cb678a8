"""The library's 2D tables for log r (host plan math, no device) against the
oracle's independent implementation of the same formulas (Sec. 3.7 at
lambda = 0 in the plane): translation weights, root weights, and the
residual R_l(r) = log(r / R_l) + G(r^2 / R_l^2) with its value at r = 0.
"""
import numpy as np
import pytest

from numpy.polynomial import chebyshev


@pytest.fixture(scope="module")
def dmk():
    from paper_2308_00292_gb300 import build, dmk as m
    build.build()
    m.lib()
    return m


def plan(dmk, eps):
    return dmk.Plan(eps, flags=dmk.FLAG_HOST_ONLY, kernel=dmk.DMK_LOG2D, dim=2)


@pytest.mark.parametrize("eps", [1e-6, 1e-9, 1e-12])
def test_weights(dmk, oracle_mod, eps):
    pl = plan(dmk, eps)
    prm = pl.params()
    op = oracle_mod.params_log2d(eps=eps)
    nf = prm["nf"]
    s = np.arange(2 * nf * nf + 1)
    h = 2 * np.pi / 3
    ref = (h / (2 * np.pi)) ** 2 * oracle_mod.kernel_log2d(op, 3, 0, h * np.sqrt(s))
    w = pl.table(1)
    assert np.abs(w - ref).max() <= 1e-12 * np.abs(ref).max()
    # level independence: (h_l / 2 pi)^2 Dhat_l(h_l |m|) at level 5
    h5 = h * 32
    ref5 = (h5 / (2 * np.pi)) ** 2 * oracle_mod.kernel_log2d(op, 3, 5, h5 * np.sqrt(s))
    assert np.abs(w - ref5).max() <= 1e-12 * np.abs(ref).max()
    t2 = pl.table(2)
    hW, wW = t2[0], t2[1:]
    assert hW == pytest.approx(oracle_mod.hW_log2d(op), rel=1e-15)
    n0 = prm["n0"]
    assert n0 == oracle_mod.n0_log2d(op) and len(wW) == 2 * n0 * n0 + 1
    sW = np.arange(2 * n0 * n0 + 1)
    refW = (hW / (2 * np.pi)) ** 2 * oracle_mod.kernel_log2d(op, 4, 0, hW * np.sqrt(sW))
    assert np.abs(wW - refW).max() <= 1e-12 * np.abs(refW).max()


@pytest.mark.parametrize("eps", [1e-6, 1e-9, 1e-12])
def test_residual(dmk, oracle_mod, eps):
    pl = plan(dmk, eps)
    op = oracle_mod.params_log2d(eps=eps)
    g = pl.table(3)
    assert len(g) <= 64 and pl.params()["q_degree"] == len(g) - 1
    G0 = pl.table(4)[0]
    t = np.linspace(1e-6, 1.0, 57)
    lib = 0.5 * np.log(t) + chebyshev.chebval(2 * t - 1, g)
    ref = oracle_mod.kernel_log2d(op, 1, 0, np.sqrt(t))
    # the fit tolerance (1e-3 eps of max(1, |G|)) plus the rounding of two FP64
    # codes that reach |R| ~ 5
    bar = 5e-3 * eps + 4e-15 * max(1.0, np.abs(ref).max())
    assert np.abs(lib - ref).max() <= bar
    # scale-free: level 4 is the same function of r / R_4
    ref4 = oracle_mod.kernel_log2d(op, 1, 4, np.sqrt(t) / 16)
    assert np.abs(lib - ref4).max() <= bar
    # S_l(0) = log R_l - G(0)
    s0 = oracle_mod.kernel_log2d(op, 0, 3, np.zeros(1))[0]
    assert np.log(1 / 8) - G0 == pytest.approx(s0, abs=1e-12)
    assert chebyshev.chebval(-1.0, g) == pytest.approx(G0, abs=bar)


def test_mixed_plans(dmk):
    """The mixed path (FP32 residual pairs) is taken at eps >= 1e-7 with the FP64
    plan's tables, and refused below, where FP32 rounding reaches eps."""
    for eps in (1e-6, 1e-7):
        with dmk.Plan(eps, flags=dmk.FLAG_HOST_ONLY, kernel=dmk.DMK_LOG2D, dim=2,
                      precision=dmk.DMK_MIXED) as pm, plan(dmk, eps) as pd:
            a, b = pm.params(), pd.params()
            assert a["precision"] == dmk.DMK_MIXED
            assert all(a[k] == b[k] for k in ("p", "nf", "n0", "q_degree", "leaf_cap"))
    with pytest.raises(dmk.DMKError) as e:
        dmk.Plan(1e-8, flags=dmk.FLAG_HOST_ONLY, kernel=dmk.DMK_LOG2D, dim=2, precision=dmk.DMK_MIXED)
    assert e.value.code == 2


@pytest.mark.parametrize("eps", [1e-6, 1e-7])
def test_f32_series_cut(dmk, eps):
    """The FP32 near field's series for G: the Chebyshev coefficients cut where
    their tail sum stays below 1e-2 eps max(1, |G|), so that the cut G is
    within that bound of the full one everywhere on [-1, 1]."""
    with plan(dmk, eps) as pl:
        prm = pl.params()
        g = pl.table(3)
        d = prm["q_degree_f32"]
        assert 3 <= d <= prm["q_degree"]
        x = np.linspace(-1.0, 1.0, 1001)
        full = chebyshev.chebval(x, g)
        gmax = max(1.0, np.abs(full).max())
        assert np.abs(full - chebyshev.chebval(x, g[:d + 1])).max() <= 1e-2 * eps * gmax * (1 + 1e-9)
        if d < prm["q_degree"]:  # one more coefficient dropped would pass the bound
            assert np.abs(g[d:]).sum() > 1e-2 * eps * gmax


def test_table_log_method():
    """log t as the 2D near field forms it (Tang's table-driven method): t = m 2^e,
    F_k = 1 / (1 + (k + 1/2)/256) for the leading 8 fraction bits k of m,
    log m = -log F_k + log1p(m F_k - 1) with log1p by its Taylor series to degree
    5; against the library log over t in [2^-255, 1), to a few units of rounding
    of the result (the series remainder is below 5e-18)."""
    rng = np.random.default_rng(41)
    t = np.exp2(-rng.uniform(0.0, 255.0, 200000))
    t = np.r_[t, 1.0 - np.exp2(-np.arange(1, 53, dtype=float)), np.exp2(-np.arange(1, 256, dtype=float))]
    m, e = np.frexp(t)            # t = m 2^e, m in [1/2, 1)
    m, e = 2.0 * m, e - 1         # m in [1, 2)
    k = np.floor((m - 1.0) * 256.0).astype(int)
    F = 1.0 / (1.0 + (k + 0.5) / 256.0)
    r = m * F - 1.0               # (the kernel forms this with one FMA)
    assert np.all(np.abs(r) <= 2.0 ** -9 * (1 + 1e-12))
    h = ((((r * 0.2 - 0.25) * r + 1.0 / 3.0) * r - 0.5) * r + 1.0) * r   # log1p(r), degree 5
    got = e * np.log(2.0) + (-np.log(F) + h)
    ref = np.log(t)
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) < 8e-16
