"""Pins of the oracle's gradients (the derivative of the potential in the
target position), against the mathematics: closed forms, central differences
of the potentials, and the direct sum within the method's precision.
"""
import numpy as np
import pytest

from paper_2308_00292_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_direct_grad_two_points(oracle_mod):
    """grad_x rho / |x - y| = rho (y - x) / |x - y|^3; coincident pairs skipped."""
    src = np.array([[0.1, 0.2, 0.3], [0.4, 0.6, 0.3]])
    rho = np.array([2.0, -3.0])
    g = oracle_mod.direct_grad(src, rho)
    d = src[1] - src[0]
    r3 = np.linalg.norm(d) ** 3
    assert np.allclose(g[0], -3.0 * d / r3, rtol=1e-15, atol=0)
    assert np.allclose(g[1], 2.0 * -d / r3, rtol=1e-15, atol=0)


def test_direct_grad_matches_central_differences(oracle_mod):
    """Targets at least 0.02 from every source, step 1e-5: the central
    difference is accurate to about (h / r)^2 < 1e-6."""
    x, q = inputs.uniform_cube(800, seed=301)
    t = np.random.default_rng(9301).random((60, 3))
    dmin = np.linalg.norm(t[:, None, :] - x[None, :, :], axis=2).min(axis=1)
    t = t[dmin > 0.02]
    assert len(t) >= 5
    g = oracle_mod.direct_grad(x, q, t)
    h = 1e-5
    fd = np.zeros_like(g)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd[:, d] = (oracle_mod.direct(x, q, t + e) - oracle_mod.direct(x, q, t - e)) / (2 * h)
    assert rel(g, fd) < 1e-5


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_dmk_grad_matches_direct(oracle_mod, eps):
    """The differentiated DMK pass reaches the direct-sum gradient to a few eps."""
    x, q = inputs.clustered(3000, seed=302, nclusters=3)
    _, g = oracle_mod.dmk_grad(x, q, eps=eps, leaf_cap=100)
    assert rel(g, oracle_mod.direct_grad(x, q)) < 3 * eps


def test_dmk_grad_is_the_derivative_of_the_dmk_potential(oracle_mod):
    """Moving a target inside its leaf changes neither the tree nor the unit box,
    so the DMK potential is smooth there and its central difference is the
    DMK gradient (far and near parts alike)."""
    x, q = inputs.uniform_cube(2000, seed=303)
    t = np.array([[0.31, 0.52, 0.47], [0.72, 0.18, 0.66], [0.5, 0.5, 0.5]])
    prm = oracle_mod.params(eps=1e-9, leaf_cap=80)
    _, g = oracle_mod.dmk_grad(x, q, t, prm=prm)
    h = 1e-6
    fd = np.zeros_like(g)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd[:, d] = (oracle_mod.dmk(x, q, t + e, prm=prm) - oracle_mod.dmk(x, q, t - e, prm=prm)) / (2 * h)
    assert rel(g, fd) < 1e-6


def test_dmk_grad_parts_add_up(oracle_mod):
    x, q = inputs.uniform_cube(1500, seed=304)
    pot, g, gf, gn = oracle_mod.dmk_grad(x, q, eps=1e-6, leaf_cap=60, parts=True)
    assert np.allclose(g, gf + gn, rtol=1e-14, atol=1e-14 * np.abs(g).max())
    assert rel(pot, oracle_mod.dmk(x, q, eps=1e-6, leaf_cap=60)) < 1e-14
