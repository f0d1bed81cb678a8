"""Pins of the oracle's prolate spheroidal wave function psi_0^c (App. A.5).

Each test checks the oracle against something other than itself: a library
routine (scipy's prolate angular function), the defining eigen-relation of
F_c evaluated by an independent quadrature here, analytic properties, and the
values the paper prints (Table 1, Fig. pswfgaussian).
"""
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TABLE1_C = [7.2462000846862793, 13.739999771118164, 20.736000061035156, 27.870000839233398]


@pytest.mark.parametrize("c", TABLE1_C[:3])
def test_pswf_matches_scipy_prolate_angular(oracle_mod, c):
    """S_00(c, x) / S_00(c, 0) from scipy equals psi_0^c(x) / psi_0^c(0)."""
    special = pytest.importorskip("scipy.special")
    x = np.linspace(0.0, 0.95, 20)
    ref = np.array([special.pro_ang1(0, 0, c, v)[0] for v in x])
    ref /= ref[0]
    got = oracle_mod.pswf(c, x)
    assert np.max(np.abs(got - ref)) < 1e-9


@pytest.mark.parametrize("c", TABLE1_C)
def test_pswf_eigen_relation(oracle_mod, c):
    """lambda_0 psi(x) = int_{-1}^{1} psi(t) exp(i c x t) dt (eq. pswfintegraloperator)
    for x in [-1, 1]: the oracle's Legendre series against a Gauss-Legendre
    quadrature of the operator done here."""
    t, w = np.polynomial.legendre.leggauss(300)
    psi_t = oracle_mod.pswf(c, t)
    lam0, c0, c2, chi0 = oracle_mod.pswf_constants(c)
    x = np.linspace(-1.0, 1.0, 41)
    lhs = lam0 * oracle_mod.pswf(c, x)
    rhs = (w[None, :] * psi_t[None, :] * np.cos(c * x[:, None] * t[None, :])).sum(axis=1)
    assert np.max(np.abs(lhs - rhs)) < 1e-13
    # the odd part of the operator vanishes on an even psi
    odd = (w[None, :] * psi_t[None, :] * np.sin(c * x[:, None] * t[None, :])).sum(axis=1)
    assert np.max(np.abs(odd)) < 1e-13


@pytest.mark.parametrize("c", TABLE1_C)
def test_pswf_shape_and_constants(oracle_mod, c):
    """psi_0 is even with no root in (-1, 1) (App. A.5); c_0 = lambda_0 psi(0)/2
    (Sec. 3.6, definition of c_0); c_0 and c_2 equal their integrals."""
    x = np.linspace(0.0, 1.0, 201)
    psi = oracle_mod.pswf(c, x)
    assert np.allclose(oracle_mod.pswf(c, -x), psi, rtol=0, atol=1e-15)
    assert np.all(psi > 0) and np.all(np.diff(psi) < 0)
    lam0, c0, c2, chi0 = oracle_mod.pswf_constants(c)
    assert abs(c0 - lam0 / 2.0) < 1e-14
    t, w = np.polynomial.legendre.leggauss(200)
    u = 0.5 * (t + 1.0)
    pu = oracle_mod.pswf(c, u)
    assert abs(0.5 * np.dot(w, pu) - c0) < 1e-14
    assert abs(0.5 * np.dot(w, u * u * pu) - c2) < 1e-14
    # the prolate eigenvalue chi_0 lies between c and c^2 for c > 1 (Sturm bound)
    assert c < chi0 + 1.0 and chi0 < c * c


def test_pswf_extension_off_interval(oracle_mod):
    """Off [-1, 1] the oracle uses the eigen-relation; near |x| = 1 it must join
    the Legendre series continuously (two different formulas)."""
    c = TABLE1_C[1]
    a = oracle_mod.pswf(c, np.array([1.0 - 1e-9, 1.0 + 1e-9]))
    assert abs(a[0] - a[1]) < 1e-11  # psi(0) = 1; both formulas agree to roundoff


def test_fig_pswfgaussian_value(oracle_mod):
    """Fig. pswfgaussian: at c = 16.893999... the scaled PSWF is stated to equal
    1e-6 at x = 1.  The standard psi_0^c (confirmed against scipy above) gives
    6.6e-7 there, so the caption is read as an order-of-magnitude statement."""
    rows = [l.split() for l in open(os.path.join(GOLD, "fig_pswfgaussian.txt")) if l[0] != "#"]
    c, x, val = (float(v) for v in rows[0])
    got = oracle_mod.pswf(c, [x])[0]
    assert 10 ** -0.5 * val < got < 10 ** 0.5 * val


def test_table1_c_gives_eps_decay(oracle_mod):
    """Table 1: c ~ log(1/eps) (eq. pswfcvalue); psi(1)/psi(0) decreases by
    about three decades per row."""
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_pswf_parameters.txt")) if l[0] != "#"]
    vals = []
    for r in rows:
        eps, logeps, c = float(r[0]), float(r[1]), float(r[2])
        assert abs(c - logeps) / logeps < 0.06
        vals.append(oracle_mod.pswf(c, [1.0])[0])
        assert vals[-1] < 1e3 * eps
    assert all(b < a * 1e-2 for a, b in zip(vals, vals[1:]))
