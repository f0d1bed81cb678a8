"""Pins of the oracle's Yukawa kernel exp(-lambda r)/r (Sec. 3.7, the kernel
splitting done in Fourier space), against the mathematics: closed forms,
numerical integration of the defining transforms with a general-purpose
integrator, the Laplace limit lambda -> 0 (an independent code path with
physical-space closed forms), the Gaussian splitting (closed-form residual),
the direct sum within eps, and the scaling of lambda with the unit-box map.
"""
import numpy as np
import pytest

from paper_2308_00292_gb300 import inputs

integrate = pytest.importorskip("scipy.integrate")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_direct_two_points(oracle_mod):
    src = np.array([[0.1, 0.2, 0.3], [0.4, 0.6, 0.3]])
    rho = np.array([2.0, -3.0])
    r = 0.5
    u = oracle_mod.direct(src, rho, lam=4.0)
    assert u == pytest.approx([-3.0 * np.exp(-2.0) / r, 2.0 * np.exp(-2.0) / r], rel=1e-15)


def test_truncated_kernel_transform(oracle_mod):
    """What_0(k) / mollifier = 4 pi int_0^{R_t} exp(-lambda r) sin(k r) / k dr, the
    transform of the kernel truncated at R_t = 1 + sqrt 3 (the Gaussian split,
    whose mollifier at level 0 is exp(-(k^2 + lambda^2) sigma_0^2 / 4))."""
    lam = 2.5
    prm = oracle_mod.params(eps=1e-6, splitting=oracle_mod.GAUSSIAN, lam=lam)
    sg = 1.0 / prm.delta
    Rt = np.sqrt(3.0) + prm.gauss_b * sg
    for k in (0.0, 0.7, 3.3, 2 * np.pi / Rt, 11.0):
        got = oracle_mod.kernel(prm, oracle_mod.WHAT, 0, np.array([k]))[0]
        win = np.exp(-(k * k + lam * lam) * sg * sg / 4)
        if k == 0.0:
            tr = integrate.quad(lambda r: 4 * np.pi * np.exp(-lam * r) * r, 0, Rt, epsabs=0, epsrel=1e-13)[0]
        else:
            tr = integrate.quad(lambda r: 4 * np.pi * np.exp(-lam * r) * np.sin(k * r) / k, 0, Rt,
                                epsabs=0, epsrel=1e-13, limit=200)[0]
        assert got == pytest.approx(tr * win, rel=1e-11)


@pytest.mark.parametrize("lam", [0.3, 4.0])
def test_gaussian_residual_is_the_inverse_transform(oracle_mod, lam):
    """R_l(r) in closed form equals the radial inverse transform of
    4 pi (1 - exp(-(k^2 + lambda^2) sigma^2 / 4)) / (k^2 + lambda^2), computed as
    exp(-lambda r)/r minus the transform of the mollified part."""
    prm = oracle_mod.params(eps=1e-6, splitting=oracle_mod.GAUSSIAN, lam=lam)
    level = 2
    sg = 2.0 ** -level / prm.delta
    for r in (0.01, 0.07, 0.2):
        got = oracle_mod.kernel(prm, oracle_mod.R_RESIDUAL, level, np.array([r]))[0]
        f = lambda k: 2 / (np.pi * r) * np.exp(-(k * k + lam * lam) * sg * sg / 4) * k * np.sin(k * r) / (k * k + lam * lam)
        mol = integrate.quad(f, 0, 40 / sg, limit=400, epsabs=1e-14, epsrel=1e-12)[0]
        assert got == pytest.approx(np.exp(-lam * r) / r - mol, rel=1e-9, abs=1e-12 / r)


def test_pswf_mollifier_is_the_inverse_transform(oracle_mod):
    """S_l(r) = 2/(pi r) int_0^inf psi(sqrt(k^2 + lambda^2) R_l / c) k sin(k r) / (k^2 + lambda^2) dk.
    Its difference from the Laplace mollifier (lambda = 0, the closed form
    Phi(r/R)/r) is the integral of the difference of the integrands, which
    decays fast: checked with psi from the oracle and Simpson's rule on a fine
    grid."""
    lam, level = 1.5, 1
    prm = oracle_mod.params(eps=1e-6, lam=lam)
    p0 = oracle_mod.params(eps=1e-6)
    R, c = 2.0 ** -level, prm.c
    ks = np.linspace(1e-9, 8 * c / R, 80001)
    dpsi = (oracle_mod.pswf(c, np.sqrt(ks ** 2 + lam ** 2) * R / c) * ks / (ks ** 2 + lam ** 2)
            - oracle_mod.pswf(c, ks * R / c) / ks)
    for r in (0.0, 0.1, 0.3, 0.45):
        got = oracle_mod.kernel(prm, oracle_mod.S_MOLLIFIED, level, np.array([r]))[0]
        lap = oracle_mod.kernel(p0, oracle_mod.S_MOLLIFIED, level, np.array([r]))[0]
        g = dpsi * (ks if r == 0.0 else np.sin(ks * r) / r)
        ref = 2 / np.pi * integrate.simpson(g, x=ks)
        assert got - lap == pytest.approx(ref, rel=1e-7, abs=1e-12 * abs(lap))


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_laplace_limit(oracle_mod, eps):
    """lambda -> 0 reproduces the Laplace pass, whose splitting the oracle takes
    from the physical-space closed forms (Phi(r/R)/r, sin^2 windows): what
    remains is the physical O(lambda r) change of the kernel."""
    x, q = inputs.clustered(2500, seed=801, nclusters=3)
    lap = oracle_mod.dmk(x, q, eps=eps, leaf_cap=70)
    yuk = oracle_mod.dmk(x, q, eps=eps, leaf_cap=70, lam=1e-10)
    assert rel(yuk, lap) < 1e-2 * eps


@pytest.mark.parametrize("splitting", [0, 1])
@pytest.mark.parametrize("lam,eps", [(0.1, 1e-6), (1.0, 1e-9), (10.0, 1e-6), (30.0, 1e-9)])
def test_dmk_matches_direct(oracle_mod, splitting, lam, eps):
    x, q = inputs.uniform_cube(2000, seed=802)
    u = oracle_mod.dmk(x, q, eps=eps, leaf_cap=60, splitting=splitting, lam=lam)
    assert rel(u, oracle_mod.direct(x, q, lam=lam)) < eps


def test_dmk_clustered_matches_direct(oracle_mod):
    x, q = inputs.clustered(3000, seed=803, nclusters=4)
    u = oracle_mod.dmk(x, q, eps=1e-6, leaf_cap=60, lam=10.0)
    assert rel(u, oracle_mod.direct(x, q, lam=10.0)) < 1e-6


def test_lambda_scales_with_the_box(oracle_mod):
    """exp(-(lambda/s) |s x - s y|) / |s x - s y| = exp(-lambda |x - y|) / (s |x - y|):
    both clouds map to the same unit box with the same lambda S."""
    x, q = inputs.uniform_cube(1500, seed=804)
    s = 8.0
    u1 = oracle_mod.dmk(x, q, eps=1e-6, leaf_cap=60, lam=5.0)
    u2 = oracle_mod.dmk(s * x + 3.0, q, eps=1e-6, leaf_cap=60, lam=5.0 / s)
    assert rel(s * u2, u1) < 1e-12
