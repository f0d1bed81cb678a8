"""CPU oracle for the discrete DMK evaluation pass (arXiv 2308.00292).

TEST INFRASTRUCTURE ONLY.  This package is loaded by the test suite, by the
smoke check and by the CPU-baseline leg of the benchmark -- never by the
product path.  It wraps ``liboracle.so``, a plain double-precision C
implementation written directly from the paper (see ``dmk_oracle.h``); it shares
no code with the CUDA library.

``build()`` compiles the library with gcc (OpenMP, no floating-point
contraction, so that the unit-box map is bit-identical on every host).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PSWF = 0
GAUSSIAN = 1


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "dmk_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("splitting", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("leaf_cap", ctypes.c_int),
        ("p", ctypes.c_int),
        ("nf", ctypes.c_int),
        ("n0", ctypes.c_int),
        ("c", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("gauss_b", ctypes.c_double),
        ("max_level", ctypes.c_int),
        ("nthreads", ctypes.c_int),
        ("lam", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.oracle_default_params.argtypes = [ctypes.POINTER(Params)]
            lib.oracle_default_params.restype = None
            lib.oracle_direct.argtypes = [dp, dp, i64, dp, i64, dp, ctypes.c_int]
            lib.oracle_direct.restype = None
            lib.oracle_direct_yukawa.argtypes = [dp, dp, i64, dp, i64, ctypes.c_double, dp, ctypes.c_int]
            lib.oracle_direct_yukawa.restype = None
            lib.oracle_dmk.argtypes = [ctypes.POINTER(Params), dp, dp, i64, dp, i64, dp, dp, dp]
            lib.oracle_dmk.restype = ctypes.c_int
            lib.oracle_direct_grad.argtypes = [dp, dp, i64, dp, i64, dp, ctypes.c_int]
            lib.oracle_direct_grad.restype = None
            lib.oracle_dmk_grad.argtypes = [ctypes.POINTER(Params), dp, dp, i64, dp, i64, dp, dp, dp, dp]
            lib.oracle_dmk_grad.restype = ctypes.c_int
            lib.oracle_tree.argtypes = [ctypes.POINTER(Params), dp, i64, dp, i64,
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int32), i64]
            lib.oracle_tree.restype = ctypes.c_int64
            lib.oracle_pswf.argtypes = [ctypes.c_double, dp, i64, dp]
            lib.oracle_pswf.restype = None
            lib.oracle_pswf_constants.argtypes = [ctypes.c_double, dp, dp, dp, dp]
            lib.oracle_pswf_constants.restype = None
            lib.oracle_kernel.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int, dp, i64, dp]
            lib.oracle_kernel.restype = None
            lib.oracle_h.argtypes = [ctypes.POINTER(Params), ctypes.c_int]
            lib.oracle_h.restype = ctypes.c_double
            lib.oracle_hW.argtypes = [ctypes.POINTER(Params)]
            lib.oracle_hW.restype = ctypes.c_double
            lib.oracle_direct_log2d.argtypes = [dp, dp, i64, dp, i64, dp, ctypes.c_int]
            lib.oracle_direct_log2d.restype = None
            lib.oracle_dmk_log2d.argtypes = [ctypes.POINTER(Params), dp, dp, i64, dp, i64, dp, dp, dp]
            lib.oracle_dmk_log2d.restype = ctypes.c_int
            lib.oracle_kernel_log2d.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int, dp, i64, dp]
            lib.oracle_kernel_log2d.restype = None
            lib.oracle_hW_log2d.argtypes = [ctypes.POINTER(Params)]
            lib.oracle_hW_log2d.restype = ctypes.c_double
            lib.oracle_n0_log2d.argtypes = [ctypes.POINTER(Params)]
            lib.oracle_n0_log2d.restype = ctypes.c_int
            lib.oracle_tree_log2d.argtypes = [ctypes.POINTER(Params), dp, i64, ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
            lib.oracle_tree_log2d.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.size == n
    return a


def params(eps=1e-6, splitting=PSWF, leaf_cap=280, nthreads=0, **kw) -> Params:
    """Method parameters with defaults filled from eps (Table 1 for PSWF)."""
    prm = Params()
    prm.splitting = splitting
    prm.eps = eps
    prm.leaf_cap = leaf_cap
    prm.nthreads = nthreads
    for k, v in kw.items():
        setattr(prm, k, v)
    _load().oracle_default_params(ctypes.byref(prm))
    return prm


def direct(src, rho, tgt=None, nthreads=0, lam=0.0) -> np.ndarray:
    """O1: u_i = sum_{j: y_j != x_i} rho_j K(|x_i - y_j|) (compensated sums),
    K(r) = 1/r, or exp(-lam r)/r (Yukawa) when lam > 0."""
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
    rho = _c64(rho, src.shape[0])
    tgt = src if tgt is None else np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(tgt.shape[0])
    if lam > 0.0:
        _load().oracle_direct_yukawa(_dp(src), _dp(rho), src.shape[0], _dp(tgt), tgt.shape[0], lam, _dp(out),
                                     nthreads)
    else:
        _load().oracle_direct(_dp(src), _dp(rho), src.shape[0], _dp(tgt), tgt.shape[0], _dp(out), nthreads)
    return out


def direct_grad(src, rho, tgt=None, nthreads=0) -> np.ndarray:
    """O1 gradient in the target position: sum_j rho_j (y_j - x_i) / |x_i - y_j|^3
    over y_j != x_i, as an (nt, 3) array."""
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
    rho = _c64(rho, src.shape[0])
    tgt = src if tgt is None else np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((tgt.shape[0], 3))
    _load().oracle_direct_grad(_dp(src), _dp(rho), src.shape[0], _dp(tgt), tgt.shape[0], _dp(out), nthreads)
    return out


def dmk_grad(src, rho, tgt=None, prm: Params | None = None, parts: bool = False, **kw):
    """O2 gradient of the potential at the targets, (nt, 3).

    Returns (pot, grad), or (pot, grad, grad_far, grad_near) if parts is True."""
    prm = prm if prm is not None else params(**kw)
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
    rho = _c64(rho, src.shape[0])
    tgt_a = src if tgt is None else np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, 3)
    nt = tgt_a.shape[0]
    pot = np.zeros(nt)
    g, gf, gn = np.zeros((nt, 3)), np.zeros((nt, 3)), np.zeros((nt, 3))
    rc = _load().oracle_dmk_grad(ctypes.byref(prm), _dp(src), _dp(rho), src.shape[0], _dp(tgt_a), nt,
                                 _dp(pot), _dp(g), _dp(gf), _dp(gn))
    if rc != 0:
        raise RuntimeError("oracle_dmk_grad failed with code %d" % rc)
    return (pot, g, gf, gn) if parts else (pot, g)


def dmk(src, rho, tgt=None, prm: Params | None = None, parts: bool = False, **kw):
    """O2: the plain DMK pass.  With tgt None every source is also a target.

    Returns the potentials, or (pot, far, near) if parts is True.
    """
    prm = prm if prm is not None else params(**kw)
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
    rho = _c64(rho, src.shape[0])
    same = tgt is None
    tgt_a = src if same else np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, 3)
    nt = tgt_a.shape[0]
    pot = np.zeros(nt)
    far = np.zeros(nt)
    near = np.zeros(nt)
    rc = _load().oracle_dmk(ctypes.byref(prm), _dp(src), _dp(rho), src.shape[0], _dp(tgt_a), nt,
                            _dp(pot), _dp(far), _dp(near))
    if rc != 0:
        raise RuntimeError("oracle_dmk failed with code %d" % rc)
    return (pot, far, near) if parts else pot


def tree(src, tgt=None, prm: Params | None = None, with_boxes: bool = False, **kw):
    """Leaf level and leaf Morton cell of every point (sources, then targets).

    With with_boxes, also returns (box_level, box_cell, box_leaf) ordered by
    level then Morton cell."""
    prm = prm if prm is not None else params(**kw)
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
    same = tgt is None
    tgt_a = src if same else np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, 3)
    n = src.shape[0] if same else src.shape[0] + tgt_a.shape[0]
    lev = np.zeros(max(n, 1), dtype=np.int32)
    cell = np.zeros(max(n, 1), dtype=np.int64)
    lib = _load()
    nb = lib.oracle_tree(ctypes.byref(prm), _dp(src), src.shape[0], _dp(tgt_a), tgt_a.shape[0],
                         lev.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                         cell.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), None, None, None, 0)
    if nb < 0:
        raise RuntimeError("oracle_tree failed with code %d" % nb)
    if not with_boxes:
        return lev[:n], cell[:n]
    bl = np.zeros(nb, dtype=np.int32)
    bc = np.zeros(nb, dtype=np.int64)
    bf = np.zeros(nb, dtype=np.int32)
    lib.oracle_tree(ctypes.byref(prm), _dp(src), src.shape[0], _dp(tgt_a), tgt_a.shape[0],
                    lev.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    cell.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                    bl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                    bf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), nb)
    return lev[:n], cell[:n], (bl, bc, bf)


def pswf(c: float, x) -> np.ndarray:
    """psi_0^c(x) normalised to psi(0) = 1."""
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    out = np.zeros_like(x)
    _load().oracle_pswf(c, _dp(x), x.size, _dp(out))
    return out


def pswf_constants(c: float):
    """(lambda_0, c_0, c_2, chi_0) for psi normalised to psi(0) = 1."""
    vals = [ctypes.c_double() for _ in range(4)]
    _load().oracle_pswf_constants(c, *[ctypes.byref(v) for v in vals])
    return tuple(v.value for v in vals)


S_MOLLIFIED, R_RESIDUAL, D_DIFFERENCE, DHAT, WHAT = range(5)


def kernel(prm: Params, what: int, level: int, r) -> np.ndarray:
    r = np.ascontiguousarray(np.atleast_1d(r), dtype=np.float64)
    out = np.zeros_like(r)
    _load().oracle_kernel(ctypes.byref(prm), what, level, _dp(r), r.size, _dp(out))
    return out


def h(prm: Params, level: int) -> float:
    return _load().oracle_h(ctypes.byref(prm), level)


def hW(prm: Params) -> float:
    return _load().oracle_hW(ctypes.byref(prm))


# ---- the 2D Laplace kernel log r (Sec. 3.7 at lambda = 0, in the plane) ----

def params_log2d(eps=1e-6, leaf_cap=120, nthreads=0, **kw) -> Params:
    """Parameters of the 2D pass; fields left at 0 are filled by the library
    (c, p, nf from Table 1, n0 from the 2D root window)."""
    prm = Params()
    prm.splitting = PSWF
    prm.eps = eps
    prm.leaf_cap = leaf_cap
    prm.nthreads = nthreads
    for k, v in kw.items():
        setattr(prm, k, v)
    return prm


def direct_log2d(src, rho, tgt=None, nthreads=0) -> np.ndarray:
    """O1 in the plane: u_i = sum_{j: y_j != x_i} rho_j log |x_i - y_j|."""
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 2)
    rho = _c64(rho, src.shape[0])
    tgt = src if tgt is None else np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, 2)
    out = np.zeros(tgt.shape[0])
    _load().oracle_direct_log2d(_dp(src), _dp(rho), src.shape[0], _dp(tgt), tgt.shape[0], _dp(out), nthreads)
    return out


def dmk_log2d(src, rho, tgt=None, prm: Params | None = None, parts: bool = False, **kw):
    """O2 in the plane for log r.  Returns the potentials (input units), or
    (pot, far, near) with the unit-box far and near parts if parts is True."""
    prm = prm if prm is not None else params_log2d(**kw)
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 2)
    rho = _c64(rho, src.shape[0])
    tgt_a = src if tgt is None else np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, 2)
    nt = tgt_a.shape[0]
    pot, far, near = np.zeros(nt), np.zeros(nt), np.zeros(nt)
    rc = _load().oracle_dmk_log2d(ctypes.byref(prm), _dp(src), _dp(rho), src.shape[0], _dp(tgt_a), nt,
                                  _dp(pot), _dp(far), _dp(near))
    if rc != 0:
        raise RuntimeError("oracle_dmk_log2d failed with code %d" % rc)
    return (pot, far, near) if parts else pot


def kernel_log2d(prm: Params, what: int, level: int, r) -> np.ndarray:
    """2D pieces: S_MOLLIFIED gives S_l(0) (r ignored), R_RESIDUAL R_l(r),
    DHAT Dhat_l(k), WHAT What_0(k)."""
    r = np.ascontiguousarray(np.atleast_1d(r), dtype=np.float64)
    out = np.zeros_like(r)
    _load().oracle_kernel_log2d(ctypes.byref(prm), what, level, _dp(r), r.size, _dp(out))
    return out


def hW_log2d(prm: Params) -> float:
    return _load().oracle_hW_log2d(ctypes.byref(prm))


def n0_log2d(prm: Params) -> int:
    return _load().oracle_n0_log2d(ctypes.byref(prm))


def tree_log2d(src, prm: Params | None = None, **kw):
    """The 2D quad-tree: per point (level, ix, iy) of its leaf, and the box count."""
    prm = prm if prm is not None else params_log2d(**kw)
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 2)
    n = src.shape[0]
    lev = np.zeros(max(n, 1), dtype=np.int32)
    ix = np.zeros(max(n, 1), dtype=np.int64)
    iy = np.zeros(max(n, 1), dtype=np.int64)
    nb = _load().oracle_tree_log2d(ctypes.byref(prm), _dp(src), n, lev.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   ix.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   iy.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if nb < 0:
        raise RuntimeError("oracle_tree_log2d failed with code %d" % nb)
    return lev[:n], ix[:n], iy[:n], nb
