"""Pins of the oracle's direct sum (O1) and DMK pass (O2).

O1 is pinned by closed forms and an independent NumPy brute force.  O2 is
pinned against O1 (the definition, eq. discretesum) within eps, against the
paper's stage decomposition (eqs. farpotential / nearpotential: the far part
equals sum_j rho_j S_{L(j)}, the near part sum_j rho_j R_{L(j)} over pairs
within R_{L(j)}), against the Gaussian splitting (an independent splitting
of the same sum), and against invariances of 1/r.
"""
import numpy as np
import pytest

from paper_2308_00292_gb300 import inputs


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def brute_numpy(x, q, y=None):
    y = x if y is None else y
    d = np.linalg.norm(y[:, None, :] - x[None, :, :], axis=2)
    with np.errstate(divide="ignore"):
        k = np.where(d > 0, 1.0 / d, 0.0)
    return k @ q


# ---------------------------------------------------------------- O1 pins
def test_direct_two_points(oracle_mod):
    x = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.8]])
    u = oracle_mod.direct(x, np.array([2.0, -3.0]))
    assert np.allclose(u, [-3.0 / 0.5, 2.0 / 0.5], rtol=1e-15)


def test_direct_matches_numpy_and_skips_coincident(oracle_mod):
    x, q = inputs.uniform_cube(700, seed=11)
    x[5] = x[9]  # a coincident pair contributes nothing
    u = oracle_mod.direct(x, q)
    assert np.max(np.abs(u - brute_numpy(x, q))) < 1e-11
    y, _ = inputs.uniform_cube(300, seed=12)
    assert np.max(np.abs(oracle_mod.direct(x, q, y) - brute_numpy(x, q, y))) < 1e-11


def test_direct_lattice_symmetry(oracle_mod):
    """Centre of a symmetric cube of unit charges: 8 corners at distance sqrt(3)/2."""
    c = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float)
    x = np.vstack([c, [[0.5, 0.5, 0.5]]])
    q = np.r_[np.ones(8), 0.0]
    assert abs(oracle_mod.direct(x, q)[8] - 8 / (np.sqrt(3) / 2)) < 1e-13


# ---------------------------------------------------------------- O2 vs O1
@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
@pytest.mark.parametrize("dist", ["uniform", "clustered", "sphere"])
def test_dmk_matches_direct(oracle_mod, eps, dist):
    n = 2500
    if dist == "uniform":
        x, q = inputs.uniform_cube(n, seed=21)
    elif dist == "clustered":
        x, q = inputs.clustered(n, seed=22, nclusters=4)
    else:
        x, q = inputs.sphere(n, seed=23)
    u = oracle_mod.dmk(x, q, eps=eps, leaf_cap=60)
    assert rel_l2(u, oracle_mod.direct(x, q)) < eps


def test_dmk_separate_targets(oracle_mod):
    x, q = inputs.clustered(2000, seed=31, nclusters=3)
    y, _ = inputs.uniform_cube(900, seed=32)
    y[:10] = x[:10]  # targets coincident with sources
    u = oracle_mod.dmk(x, q, y, eps=1e-6, leaf_cap=50)
    assert rel_l2(u, oracle_mod.direct(x, q, y)) < 1e-6


def test_gaussian_splitting_agrees(oracle_mod):
    """Two independent splittings of the same sum agree within 2 eps (P8)."""
    x, q = inputs.clustered(1500, seed=41, nclusters=3)
    a = oracle_mod.dmk(x, q, eps=1e-6, leaf_cap=60, splitting=0)
    b = oracle_mod.dmk(x, q, eps=1e-6, leaf_cap=60, splitting=1)
    ref = oracle_mod.direct(x, q)
    assert rel_l2(a, b) < 2e-6
    assert rel_l2(b, ref) < 1e-6


# ---------------------------------------------------------------- stages
def test_stage_decomposition(oracle_mod):
    """far(x_i) = sum_j rho_j S_{L(j)}(|x_i - y_j|) (coincident pairs included at
    S(0)); near(x_i) = sum_j rho_j R_{L(j)}(r_ij) over 0 < r < R_{L(j)} minus the
    self terms rho_j S_{L(j)}(0) (eqs. farpotential, nearpotential, Step 5)."""
    x, q = inputs.clustered(1200, seed=51, nclusters=2)
    x[3] = x[4]
    prm = oracle_mod.params(eps=1e-9, leaf_cap=40)
    u, far, near = oracle_mod.dmk(x, q, prm=prm, parts=True)
    lev, _ = oracle_mod.tree(x, prm=prm)
    lo = x.min(axis=0)
    S = (x.max(axis=0) - lo).max()
    uu = (x - lo) / S
    d = np.linalg.norm(uu[:, None, :] - uu[None, :, :], axis=2)
    far_ref = np.zeros(len(x))
    near_ref = np.zeros(len(x))
    for L in np.unique(lev):
        js = np.where(lev == L)[0]
        dd = d[:, js].ravel()
        sk = oracle_mod.kernel(prm, oracle_mod.S_MOLLIFIED, int(L), dd).reshape(len(x), len(js))
        rk = np.zeros_like(dd)
        m = (dd > 0) & (dd < 2.0 ** -L)
        rk[m] = oracle_mod.kernel(prm, oracle_mod.R_RESIDUAL, int(L), dd[m])
        rk = rk.reshape(len(x), len(js))
        s0 = oracle_mod.kernel(prm, oracle_mod.S_MOLLIFIED, int(L), np.array([0.0]))[0]
        far_ref += sk @ q[js]
        near_ref += rk @ q[js] - ((d[:, js] == 0) * s0) @ q[js]
    far_ref /= S
    near_ref /= S
    assert rel_l2(far, far_ref) < 1e-9
    assert np.max(np.abs(near - near_ref)) < 1e-10 * np.max(np.abs(near_ref))


# ---------------------------------------------------------------- invariants
def test_linearity_in_charges(oracle_mod):
    x, q1 = inputs.uniform_cube(1500, seed=61)
    q2 = np.random.default_rng(62).standard_normal(1500)
    a = oracle_mod.dmk(x, 2.0 * q1 - 3.0 * q2, eps=1e-6, leaf_cap=60)
    b = 2.0 * oracle_mod.dmk(x, q1, eps=1e-6, leaf_cap=60) - 3.0 * oracle_mod.dmk(x, q2, eps=1e-6, leaf_cap=60)
    assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(a))


def test_scale_and_translation(oracle_mod):
    x, q = inputs.clustered(1500, seed=71, nclusters=3)
    u = oracle_mod.dmk(x, q, eps=1e-6, leaf_cap=60)
    # power-of-two scaling maps to the same unit box exactly: u scales by 1/4
    u4 = oracle_mod.dmk(4.0 * x, q, eps=1e-6, leaf_cap=60)
    assert np.max(np.abs(u4 - u / 4.0)) < 1e-14 * np.max(np.abs(u))
    # a translation changes the tree; agreement at the eps level
    ut = oracle_mod.dmk(x + np.array([0.3, -0.17, 5.0]), q, eps=1e-6, leaf_cap=60)
    assert rel_l2(ut, u) < 2e-6


def test_transposition(oracle_mod):
    """<phi, A_{X<-Y} rho> = <rho, A_{Y<-X} phi> for the symmetric kernel."""
    x, rho = inputs.clustered(900, seed=81, nclusters=2)
    y, phi = inputs.uniform_cube(700, seed=82)
    a = np.dot(phi, oracle_mod.dmk(x, rho, y, eps=1e-6, leaf_cap=40))
    b = np.dot(rho, oracle_mod.dmk(y, phi, x, eps=1e-6, leaf_cap=40))
    ref = np.dot(phi, oracle_mod.direct(x, rho, y))
    scale = np.linalg.norm(phi) * np.linalg.norm(oracle_mod.direct(x, rho, y))
    assert abs(a - b) < 2e-6 * scale and abs(a - ref) < 1e-6 * scale


def test_single_source(oracle_mod):
    x = np.array([[0.2, 0.3, 0.4]])
    y, _ = inputs.uniform_cube(400, seed=91)
    u = oracle_mod.dmk(x, np.array([1.5]), y, eps=1e-9, leaf_cap=30)
    assert rel_l2(u, 1.5 / np.linalg.norm(y - x, axis=1)) < 1e-9


# ---------------------------------------------------------------- adversarial
def test_all_points_in_one_leaf(oracle_mod):
    x, q = inputs.uniform_cube(200, seed=101)
    u = oracle_mod.dmk(x, q, eps=1e-6, leaf_cap=280)
    lev, _ = oracle_mod.tree(x, leaf_cap=280)
    assert np.all(lev == 0)
    assert rel_l2(u, oracle_mod.direct(x, q)) < 1e-6


def test_duplicates_and_faces(oracle_mod):
    x, q = inputs.uniform_cube(1500, seed=111)
    x[:40] = x[0]            # 40 coincident points (more than leaf_cap / 2)
    x[40:80, 0] = 1.0        # points on the max face
    x[80:120, 1] = 0.0       # points on the min face
    x[120:130] = [0.5, 0.5, 0.5]  # points on internal box corners
    u = oracle_mod.dmk(x, q, eps=1e-6, leaf_cap=30)
    assert rel_l2(u, oracle_mod.direct(x, q)) < 1e-6


def test_deep_cluster(oracle_mod):
    rng = np.random.default_rng(121)
    x = np.vstack([0.3 + 1e-5 * rng.standard_normal((600, 3)), rng.uniform(0, 1, (300, 3))])
    q = rng.uniform(-1, 1, 900)
    u = oracle_mod.dmk(x, q, eps=1e-6, leaf_cap=20)
    lev, _ = oracle_mod.tree(x, leaf_cap=20)
    assert lev.max() >= 14
    assert rel_l2(u, oracle_mod.direct(x, q)) < 1e-6


def test_tiny_inputs(oracle_mod):
    # one point: the far field carries rho S_0(0) ~ 3 rho, removed exactly by
    # the self correction, so the result is zero to eps * S_0(0)
    assert abs(oracle_mod.dmk(np.array([[0.1, 0.1, 0.1]]), np.array([1.0]), eps=1e-6)[0]) < 3e-6
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 2.0]])
    u = oracle_mod.dmk(x, np.array([1.0, 1.0]), eps=1e-9)
    assert np.allclose(u, 0.5, rtol=1e-9)


# ---------------------------------------------------------------- tree
def _adjacent(l1, c1, l2, c2):
    """closed cubes of (level, cell) share a point"""
    for d in range(3):
        a = c1[d] * 2.0 ** -l1, (c1[d] + 1) * 2.0 ** -l1
        b = c2[d] * 2.0 ** -l2, (c2[d] + 1) * 2.0 ** -l2
        if a[1] < b[0] or b[1] < a[0]:
            return False
    return True


def _decode(m, level):
    c = [0, 0, 0]
    for b in range(level):
        for d in range(3):
            c[d] |= ((int(m) >> (3 * b + d)) & 1) << b
    return c


def test_tree_level_restriction_and_capacity(oracle_mod):
    rng = np.random.default_rng(131)
    x = np.vstack([0.6 + 3e-4 * rng.standard_normal((1500, 3)), rng.uniform(0, 1, (300, 3))])
    cap = 25
    lev, cell, (bl, bc, bf) = oracle_mod.tree(x, leaf_cap=cap, with_boxes=True)
    leaves = [(int(l), _decode(c, l)) for l, c, f in zip(bl, bc, bf) if f]
    nonleaf = [(int(l), _decode(c, l)) for l, c, f in zip(bl, bc, bf) if not f]
    # every point lies in its leaf cell; leaves respect the capacity
    lo = x.min(axis=0)
    S = (x.max(axis=0) - lo).max()
    u = (x - lo) / S
    for i in range(0, len(x), 7):
        c = _decode(cell[i], lev[i])
        assert all(c[d] * 2.0 ** -lev[i] <= u[i, d] <= (c[d] + 1) * 2.0 ** -lev[i] for d in range(3))
    _, counts = np.unique(np.c_[lev, cell], axis=0, return_counts=True)
    assert counts.max() <= cap
    # level restriction: no leaf touches a non-leaf box two or more levels finer
    for (la, ca) in leaves:
        for (lb, cb) in nonleaf:
            if lb == la + 1:
                assert not _adjacent(la, ca, lb, cb)
    assert lev.max() - lev.min() >= 4
