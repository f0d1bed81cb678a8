"""Pins of the oracle's kernel splittings and their Fourier data.

Checked against the mathematics, not against the oracle itself: closed-form
Fourier transforms are compared with radial quadratures of the physical-space
kernels (App. A.2 eq. rbfft3d), the trapezoidal Fourier series of D_l and of
the windowed root kernel with the physical kernels they stand for
(eqs. differencekernelft2a, windowedkernel2), and the supports the splitting
promises (Sec. 3.6 properties (a)-(c)).
"""
import math

import numpy as np
import pytest


def radial_ft(f_of_r, k, rmax, n=4000):
    """4 pi int_0^rmax sin(kr)/(kr) f(r) r^2 dr by Gauss-Legendre (eq. rbfft3d)."""
    t, w = np.polynomial.legendre.leggauss(n)
    r = 0.5 * rmax * (t + 1.0)
    wr = 0.5 * rmax * w
    fr = f_of_r(r)
    out = []
    for kk in np.atleast_1d(k):
        s = np.sinc(kk * r / np.pi)  # sin(kr)/(kr)
        out.append(4.0 * np.pi * np.sum(wr * s * fr * r * r))
    return np.array(out)


@pytest.mark.parametrize("splitting", [0, 1])
@pytest.mark.parametrize("level", [0, 2])
def test_Dhat_matches_radial_transform(oracle_mod, splitting, level):
    """Dhat_l(k) (eqs. differencekernelft / differencekernelft3, incl. k = 0) equals
    the radial Fourier transform of D_l(r) = S_{l+1}(r) - S_l(r)."""
    prm = oracle_mod.params(eps=1e-6, splitting=splitting)
    R = 2.0 ** -level
    k = np.array([0.0, 0.5, 3.0, 10.0, 25.0, 60.0]) / R
    rmax = 1.5 * R if splitting == 0 else 2.0 * R
    num = radial_ft(lambda r: oracle_mod.kernel(prm, oracle_mod.D_DIFFERENCE, level, r), k, rmax)
    ana = oracle_mod.kernel(prm, oracle_mod.DHAT, level, k)
    scale = abs(ana[0])
    assert np.max(np.abs(num - ana)) < 1e-9 * scale


def _fourier_series_error(oracle_mod, prm, level, npts=3000, seed=0):
    h = oracle_mod.h(prm, level)
    R = 2.0 ** -level
    n = prm.nf
    m = np.arange(-n, n + 1)
    MX, MY, MZ = np.meshgrid(m, m, m, indexing="ij")
    km = h * np.sqrt(MX ** 2 + MY ** 2 + MZ ** 2).ravel()
    w = (h / (2 * np.pi)) ** 3 * oracle_mod.kernel(prm, oracle_mod.DHAT, level, km)
    rng = np.random.default_rng(seed)
    x = rng.uniform(-2 * R, 2 * R, size=(npts, 3))
    x[:100] = 0.0
    x[:100, 0] = np.linspace(0, 2 * R, 100)
    r = np.linalg.norm(x, axis=1)
    exact = oracle_mod.kernel(prm, oracle_mod.D_DIFFERENCE, level, r)
    approx = np.zeros(npts)
    for i0 in range(0, npts, 500):
        xs = x[i0:i0 + 500]
        ph = np.exp(1j * h * (np.outer(xs[:, 0], MX.ravel()) + np.outer(xs[:, 1], MY.ravel())
                              + np.outer(xs[:, 2], MZ.ravel())))
        approx[i0:i0 + 500] = (ph @ w).real
    d0 = oracle_mod.kernel(prm, oracle_mod.D_DIFFERENCE, level, np.array([0.0]))[0]
    return np.max(np.abs(approx - exact)) / abs(d0)


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_difference_kernel_fourier_series(oracle_mod, eps):
    """D_l(x) ~ sum_m w_{l,m} exp(i h_l m . x) for |x_i| <= 2 R_l (eq.
    differencekernelft2a) within eps, with Table 1's N1 and h_l = 2 pi/(3 R_l)."""
    prm = oracle_mod.params(eps=eps)
    assert 2 * prm.nf + 1 in (13, 25, 39, 53)
    for level in (0, 3):
        assert _fourier_series_error(oracle_mod, prm, level) < eps


def test_gaussian_difference_kernel_fourier_series(oracle_mod):
    prm = oracle_mod.params(eps=1e-6, splitting=1)
    assert _fourier_series_error(oracle_mod, prm, 1) < 1e-6


def _root_series(oracle_mod, prm, x):
    hW = oracle_mod.hW(prm)
    n = prm.n0
    m = np.arange(-n, n + 1)
    MX, MY, MZ = np.meshgrid(m, m, m, indexing="ij")
    km = hW * np.sqrt(MX ** 2 + MY ** 2 + MZ ** 2).ravel()
    w = (hW / (2 * np.pi)) ** 3 * oracle_mod.kernel(prm, oracle_mod.WHAT, 0, km)
    out = np.zeros(len(x))
    for i0 in range(0, len(x), 300):
        xs = x[i0:i0 + 300]
        ph = np.exp(1j * hW * (np.outer(xs[:, 0], MX.ravel()) + np.outer(xs[:, 1], MY.ravel())
                               + np.outer(xs[:, 2], MZ.ravel())))
        out[i0:i0 + 300] = (ph @ w).real
    return out


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_windowed_root_kernel_pswf(oracle_mod, eps):
    """W_0 = Phi_0(r)/r for r <= sqrt(3) (eq. kernelequivalence) from its Fourier
    series with the windowed transform What_0."""
    prm = oracle_mod.params(eps=eps)
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, size=(1500, 3))
    r = np.linalg.norm(x, axis=1)
    exact = oracle_mod.kernel(prm, oracle_mod.S_MOLLIFIED, 0, r)
    s0 = oracle_mod.kernel(prm, oracle_mod.S_MOLLIFIED, 0, np.array([0.0]))[0]
    assert np.max(np.abs(_root_series(oracle_mod, prm, x) - exact)) < eps * s0


def test_windowed_root_kernel_gaussian_closed_form(oracle_mod):
    """The Gaussian windowed kernel's Fourier series equals the closed form of
    Lemma trunc_lemma (eq. windowedkernel2), and erf(r/sigma)/r within erfc(b)."""
    from math import erf, sqrt
    prm = oracle_mod.params(eps=1e-6, splitting=1)
    sigma = 1.0 / prm.delta
    b = prm.gauss_b
    C = math.sqrt(3.0)
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, size=(800, 3))
    r = np.linalg.norm(x, axis=1)
    closed = np.array([erf(rr / sigma) / rr - 0.5 * (erf((b * sigma + C + rr) / sigma) / rr
                                                     - erf((b * sigma + C - rr) / sigma) / rr) for rr in r])
    series = _root_series(oracle_mod, prm, x)
    assert np.max(np.abs(series - closed)) < 1e-8 * np.max(np.abs(closed))
    mol = np.array([erf(rr / sigma) / rr for rr in r])
    assert np.max(np.abs(closed - mol) * r) <= math.erfc(b) * 1.01


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9, 1e-12])
def test_residual_compact_support(oracle_mod, eps):
    """R_L vanishes for r >= R_L (PSWF splitting, exact by construction of Phi)
    and equals 1/r - Phi(r/R_L)/r with Phi(1) = 1 (Sec. 3.6)."""
    prm = oracle_mod.params(eps=eps)
    for L in (0, 4):
        RL = 2.0 ** -L
        r = RL * np.linspace(1.0, 3.0, 7)
        assert np.all(oracle_mod.kernel(prm, oracle_mod.R_RESIDUAL, L, r) == 0.0)
        s = oracle_mod.kernel(prm, oracle_mod.S_MOLLIFIED, L, r)
        assert np.allclose(s * r, 1.0, rtol=0, atol=1e-13)
    # the mollified kernel at 0 is the self-interaction limit psi(0)/(c_0 R_L)
    lam0, c0, c2, _ = oracle_mod.pswf_constants(prm.c)
    s0 = oracle_mod.kernel(prm, oracle_mod.S_MOLLIFIED, 2, np.array([0.0, 1e-7]))
    assert abs(s0[0] - 4.0 / c0) < 1e-12 * s0[0]
    assert abs(s0[1] - s0[0]) < 1e-6 * s0[0]


def test_gaussian_splitting_is_ewald(oracle_mod):
    """Gaussian mollified kernel erf(r/sigma_l)/r with sigma_l = sigma_0 / 2^l
    (eqs. kerneldef, deltavalue); self-interaction limit 2/(sqrt(pi) sigma)
    (Sec. 3.1 remark); erfc(R_l/sigma_l) <= eps (support of R_l)."""
    from math import erf, erfc, pi, sqrt
    prm = oracle_mod.params(eps=1e-6, splitting=1)
    for l in (0, 3):
        sg = 2.0 ** -l / prm.delta
        r = np.array([0.01, 0.1, 0.3]) * 2.0 ** -l
        got = oracle_mod.kernel(prm, oracle_mod.S_MOLLIFIED, l, r)
        assert np.allclose(got, [erf(v / sg) / v for v in r], rtol=1e-14)
        assert abs(oracle_mod.kernel(prm, oracle_mod.S_MOLLIFIED, l, np.array([0.0]))[0]
                   - 2.0 / (sqrt(pi) * sg)) < 1e-12 / sg
        assert erfc(2.0 ** -l / sg) <= 1e-6
