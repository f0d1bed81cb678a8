"""ctypes binding of libdmk (``include/dmk.h``): argument marshalling only.

Every step of the evaluation runs in the library's CUDA kernels.  Device
arrays are passed as torch CUDA tensors (float64, contiguous, shape [n, 3] for
points) and evaluated with ``dmk_eval`` on torch's current stream; host arrays
(NumPy) go through ``dmk_eval_host``, which copies in and out.

If ``libdmk.so`` is missing this module raises on import of the library:
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdmk.so")

DMK_LAPLACE = 0
DMK_YUKAWA = 1
DMK_LOG2D = 2       # log r in the plane (dim 2, FP64)
DMK_FP64 = 0
DMK_MIXED = 1
FLAG_FAR_ONLY = 1
FLAG_NEAR_ONLY = 2
FLAG_HOST_ONLY = 4

ERRORS = {0: "DMK_OK", 1: "DMK_ERR_INVALID_ARG", 2: "DMK_ERR_UNSUPPORTED", 3: "DMK_ERR_OOM", 4: "DMK_ERR_CUDA",
          5: "DMK_ERR_TIMEOUT", 6: "DMK_ERR_DEPTH", 7: "DMK_ERR_INTERNAL"}

EXPORTED = ["dmk_plan", "dmk_eval", "dmk_eval_grad", "dmk_eval_host", "dmk_plan_destroy", "dmk_error_string",
            "dmk_last_error_detail", "dmk_plan_get_params", "dmk_plan_get_table", "dmk_get_stats", "dmk_get_tree",
            "dmk_direct_noalloc", "dmk_tune_leaf_cap", "dmk_eval_batch",
            "dmk_tune_leaf_cap_batch", "dmk_plan_get_yukawa_table", "dmk_adjoint_combine"]


class Opts(ctypes.Structure):
    _fields_ = [("leaf_cap", ctypes.c_int), ("precision", ctypes.c_int), ("kernel_param", ctypes.c_double),
                ("flags", ctypes.c_int), ("max_level", ctypes.c_int), ("p", ctypes.c_int), ("nf", ctypes.c_int)]


class PlanParams(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("c", ctypes.c_double), ("p", ctypes.c_int), ("nf", ctypes.c_int),
                ("n0", ctypes.c_int), ("leaf_cap", ctypes.c_int), ("max_level", ctypes.c_int),
                ("precision", ctypes.c_int), ("q_degree", ctypes.c_int), ("psi0_over_c0", ctypes.c_double),
                ("q_degree_f32", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_levels", ctypes.c_int32), ("n_boxes", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64), ("n_fout", ctypes.c_int64), ("n_fin", ctypes.c_int64),
                ("near_pairs", ctypes.c_int64), ("balance_rounds", ctypes.c_int32),
                ("t_tree_ms", ctypes.c_float), ("t_upward_ms", ctypes.c_float),
                ("t_downward_ms", ctypes.c_float), ("t_near_ms", ctypes.c_float), ("t_total_ms", ctypes.c_float),
                ("n_launches", ctypes.c_int64), ("near_pairs_inside", ctypes.c_int64),
                ("local_flops", ctypes.c_int64), ("t_local_ms", ctypes.c_float),
                ("t_incoming_ms", ctypes.c_float), ("incoming_reads", ctypes.c_int64),
                ("incoming_flops", ctypes.c_int64), ("t_planewave_ms", ctypes.c_float),
                ("near_pairs_screened", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DMKError(RuntimeError):
    def __init__(self, code, detail):
        super().__init__("%s: %s" % (ERRORS.get(code, code), detail))
        self.code = code


_lib = None
_lock = threading.Lock()


def lib():
    """Load libdmk.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise OSError("libdmk.so not built: run paper_2308_00292_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            vp, dp, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
            L.dmk_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(Opts),
                                   ctypes.POINTER(vp)]
            L.dmk_eval.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp]
            L.dmk_eval_grad.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp, vp]
            L.dmk_eval_batch.argtypes = [vp, vp, vp, ctypes.POINTER(i64), ctypes.c_int, vp, vp]
            L.dmk_plan_get_yukawa_table.argtypes = [vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, i64,
                                                    ctypes.POINTER(i64)]
            L.dmk_eval_host.argtypes = [vp, dp, i64, dp, dp, i64, dp, vp]
            L.dmk_plan_destroy.argtypes = [vp]
            L.dmk_error_string.argtypes = [ctypes.c_int]
            L.dmk_error_string.restype = ctypes.c_char_p
            L.dmk_last_error_detail.argtypes = []
            L.dmk_last_error_detail.restype = ctypes.c_char_p
            L.dmk_plan_get_params.argtypes = [vp, ctypes.POINTER(PlanParams)]
            L.dmk_plan_get_table.argtypes = [vp, ctypes.c_int, dp, i64, ctypes.POINTER(i64)]
            L.dmk_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
            L.dmk_get_tree.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64), i64]
            L.dmk_direct_noalloc.argtypes = [vp, i64, vp, vp, i64, vp, vp]
            L.dmk_adjoint_combine.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            L.dmk_tune_leaf_cap.argtypes = [vp, vp, i64, vp, vp, i64, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_float), vp]
            L.dmk_tune_leaf_cap_batch.argtypes = [vp, vp, vp, ctypes.POINTER(i64), ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float), vp]
            for name in EXPORTED:
                getattr(L, name).restype = getattr(L, name).restype or ctypes.c_int
            _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        detail = lib().dmk_last_error_detail().decode()
        raise DMKError(rc, detail)


def _dev(t, name, shape, device=None):
    """Raise ValueError unless t is a contiguous float64 CUDA tensor of the given
    shape (None entries match any size) on `device` (when given).  The library
    reads and writes exactly that many doubles through the raw pointer, so a
    wrong dtype, length or device would be an out-of-bounds access."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s must be a torch tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64:
        raise ValueError("%s must be float64, got %s" % (name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if device is not None and t.device != device:
        raise ValueError("%s is on %s, expected %s" % (name, t.device, device))
    if len(t.shape) != len(shape) or any(w is not None and w != g for w, g in zip(shape, t.shape)):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape),
                                                         tuple("*" if w is None else w for w in shape)))
    return t


class Plan:
    """A DMK plan: ``Plan(eps, precision=DMK_MIXED, leaf_cap=200)``."""

    def __init__(self, eps=1e-6, precision=DMK_FP64, leaf_cap=0, flags=0, max_level=0, p=0, nf=0, kernel=DMK_LAPLACE,
                 dim=3, lam=0.0):
        """lam: the Yukawa parameter (kernel DMK_YUKAWA, exp(-lam r)/r).
        kernel DMK_LOG2D takes dim=2: coordinates are (n, 2)."""
        self._h = ctypes.c_void_p()
        self._dim = dim
        o = Opts(leaf_cap, precision, float(lam), flags, max_level, p, nf)
        _check(lib().dmk_plan(kernel, dim, eps, ctypes.byref(o), ctypes.byref(self._h)))

    def close(self):
        if self._h:
            lib().dmk_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- eval
    def eval(self, sources, charges, targets=None, out=None, stream=None):
        """Potentials at the targets (every source when targets is None).

        torch CUDA tensors -> dmk_eval on the device (result is a tensor);
        NumPy arrays -> dmk_eval_host (result is an ndarray)."""
        if isinstance(sources, np.ndarray):
            return self.eval_host(sources, charges, targets, out)
        import torch
        _dev(sources, "sources", (None, self._dim))
        dev, ns = sources.device, sources.shape[0]
        _dev(charges, "charges", (ns,), dev)
        tgt = sources if targets is None else _dev(targets, "targets", (None, self._dim), dev)
        nt = tgt.shape[0]
        if out is None:
            out = torch.empty(nt, dtype=torch.float64, device=dev)
        _dev(out, "out", (nt,), dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        _check(lib().dmk_eval(self._h, sources.data_ptr(), ns, charges.data_ptr(), tgt.data_ptr(), nt,
                              out.data_ptr(), st))
        return out

    def eval_grad(self, sources, charges, targets=None, out=None, gout=None, stream=None):
        """Potentials and their gradients (n_tgt x 3) at the targets, torch CUDA tensors."""
        import torch
        _dev(sources, "sources", (None, self._dim))
        dev, ns = sources.device, sources.shape[0]
        _dev(charges, "charges", (ns,), dev)
        tgt = sources if targets is None else _dev(targets, "targets", (None, self._dim), dev)
        nt = tgt.shape[0]
        if out is None:
            out = torch.empty(nt, dtype=torch.float64, device=dev)
        if gout is None:
            gout = torch.empty(nt, 3, dtype=torch.float64, device=dev)
        _dev(out, "out", (nt,), dev)
        _dev(gout, "gout", (nt, 3), dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        _check(lib().dmk_eval_grad(self._h, sources.data_ptr(), ns, charges.data_ptr(), tgt.data_ptr(), nt,
                                   out.data_ptr(), gout.data_ptr(), st))
        return out, gout

    def eval_batch(self, points, charges, offsets, out=None, stream=None):
        """Potentials of independent systems: system s is points[offsets[s]:offsets[s+1]]
        (torch CUDA float64 tensors; offsets a host sequence of n_systems + 1 ints)."""
        import torch
        _dev(points, "points", (None, self._dim))
        dev, n = points.device, points.shape[0]
        _dev(charges, "charges", (n,), dev)
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        # the library validates the offsets themselves; the points must cover them
        if off.ndim != 1 or off.size < 1 or off.max() > n:
            raise ValueError("offsets must lie within the %d points" % n)
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=dev)
        _dev(out, "out", (n,), dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        _check(lib().dmk_eval_batch(self._h, points.data_ptr(), charges.data_ptr(),
                                    off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(off) - 1,
                                    out.data_ptr(), st))
        return out

    def tune_leaf_cap(self, sources, charges, targets=None, candidates=None, reps=0, stream=None):
        """Time the given problem at each candidate leaf capacity and keep the
        fastest in the plan; returns (best, {candidate: ms})."""
        import torch
        _dev(sources, "sources", (None, self._dim))
        dev = sources.device
        _dev(charges, "charges", (sources.shape[0],), dev)
        tgt = sources if targets is None else _dev(targets, "targets", (None, self._dim), dev)
        cand = None if candidates is None else (ctypes.c_int * len(candidates))(*candidates)
        ncand = 0 if candidates is None else len(candidates)
        times = (ctypes.c_float * (7 if candidates is None else max(ncand, 1)))()
        best = ctypes.c_int()
        st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        _check(lib().dmk_tune_leaf_cap(self._h, sources.data_ptr(), sources.shape[0], charges.data_ptr(),
                                       tgt.data_ptr(), tgt.shape[0], cand, ncand, reps, ctypes.byref(best),
                                       times, st))
        tried = list(candidates) if candidates is not None else [64, 100, 140, 200, 280, 400, 560]
        return best.value, dict(zip(tried, list(times)[:len(tried)]))

    def tune_leaf_cap_batch(self, points, charges, offsets, candidates=None, reps=0, stream=None):
        """tune_leaf_cap for a batch of systems (as in eval_batch)."""
        import torch
        _dev(points, "points", (None, self._dim))
        dev, n = points.device, points.shape[0]
        _dev(charges, "charges", (n,), dev)
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        if off.ndim != 1 or off.size < 1 or off.max() > n:
            raise ValueError("offsets must lie within the %d points" % n)
        cand = None if candidates is None else (ctypes.c_int * len(candidates))(*candidates)
        ncand = 0 if candidates is None else len(candidates)
        tried = list(candidates) if candidates is not None else [64, 100, 140, 200, 280, 400, 560]
        times = (ctypes.c_float * len(tried))()
        best = ctypes.c_int()
        st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        _check(lib().dmk_tune_leaf_cap_batch(self._h, points.data_ptr(), charges.data_ptr(),
                                             off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(off) - 1,
                                             cand, ncand, reps, ctypes.byref(best), times, st))
        return best.value, dict(zip(tried, list(times)))

    def eval_host(self, sources, charges, targets=None, out=None, stream=0):
        src = np.ascontiguousarray(sources, dtype=np.float64).reshape(-1, self._dim)
        q = np.ascontiguousarray(charges, dtype=np.float64).reshape(-1)
        if q.shape[0] != src.shape[0]:
            raise ValueError("charges has %d entries for %d sources" % (q.shape[0], src.shape[0]))
        tgt = src if targets is None else np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, self._dim)
        if out is None:
            out = np.empty(tgt.shape[0])
        if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
                and out.size == tgt.shape[0]):
            raise ValueError("out must be a contiguous float64 array of %d entries" % tgt.shape[0])
        dp = ctypes.POINTER(ctypes.c_double)
        _check(lib().dmk_eval_host(self._h, src.ctypes.data_as(dp), src.shape[0], q.ctypes.data_as(dp),
                                   tgt.ctypes.data_as(dp), tgt.shape[0], out.ctypes.data_as(dp), stream))
        return out

    # ---------------------------------------------------------------- introspection
    def params(self) -> dict:
        p = PlanParams()
        _check(lib().dmk_plan_get_params(self._h, ctypes.byref(p)))
        return {k: getattr(p, k) for k, _ in p._fields_}

    def yukawa_table(self, lambda_unit: float, level: int, which: int) -> np.ndarray:
        n = ctypes.c_int64()
        _check(lib().dmk_plan_get_yukawa_table(self._h, lambda_unit, level, which, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value)
        _check(lib().dmk_plan_get_yukawa_table(self._h, lambda_unit, level, which,
                                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value,
                                               ctypes.byref(n)))
        return out

    def table(self, which: int) -> np.ndarray:
        n = ctypes.c_int64()
        _check(lib().dmk_plan_get_table(self._h, which, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value)
        _check(lib().dmk_plan_get_table(self._h, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        n.value, ctypes.byref(n)))
        return out

    def stats(self) -> dict:
        s = Stats()
        _check(lib().dmk_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def tree(self):
        """(leaf_level, leaf_cell) of every point of the last evaluation."""
        n = self.stats()["n_points"]
        lev = np.zeros(n, dtype=np.int32)
        cell = np.zeros(n, dtype=np.int64)
        _check(lib().dmk_get_tree(self._h, lev.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  cell.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n))
        return lev, cell


def adjoint_combine(w1, g1, w2=None, g2=None, out=None, stream=None):
    """out_i = w1_i g1_i (+ w2_i g2_i) for n x 3 gradients, on the device
    (dmk_adjoint_combine); the terms take float64 CUDA tensors."""
    import torch
    n = g1.shape[0]
    _dev(g1, "g1", (n, 3))
    dev = g1.device
    _dev(w1, "w1", (n,), dev)
    if w2 is not None:
        _dev(w2, "w2", (n,), dev)
        _dev(g2, "g2", (n, 3), dev)
    if out is None:
        out = torch.empty(n, 3, dtype=torch.float64, device=dev)
    _dev(out, "out", (n, 3), dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    _check(lib().dmk_adjoint_combine(n, w1.data_ptr(), g1.data_ptr(), None if w2 is None else w2.data_ptr(),
                                     None if g2 is None else g2.data_ptr(), out.data_ptr(), st))
    return out


def potential(plan: Plan, sources, charges, targets=None):
    """Differentiable potentials: u_i = sum_{j : y_j != x_i} rho_j / |x_i - y_j| at the
    targets (every source when targets is None), with gradients with respect
    to the charges and to the source and target positions.

    The backward pass is two more evaluations of the same plan: the kernel is
    symmetric, so dL/drho_j = v(y_j) and dL/dy_j = rho_j grad v(y_j) for the
    potential v of charges dL/du at the targets, and dL/dx_i = dL/du_i grad u(x_i);
    the products run in the library (dmk_adjoint_combine).

    float32 inputs are widened to float64 at the boundary (exactly) and their
    gradients are returned in float32; the potentials are float64.
    """
    import torch

    def f64(t):
        return t.detach().to(torch.float64).contiguous()

    class _Potential(torch.autograd.Function):
        @staticmethod
        def forward(ctx, src, rho, tgt):
            same = tgt is None
            s64, r64 = f64(src), f64(rho)
            t64 = s64 if same else f64(tgt)
            need_pos = ctx.needs_input_grad[0] or (not same and ctx.needs_input_grad[2])
            if need_pos:
                u, gu = plan.eval_grad(s64, r64, None if same else t64)
            else:
                u = plan.eval(s64, r64, None if same else t64)
                gu = None
            ctx.same = same
            ctx.dtypes = (src.dtype, rho.dtype, None if same else tgt.dtype)
            ctx.save_for_backward(s64, r64, t64, gu if gu is not None else torch.empty(0, device=src.device))
            ctx.has_gu = gu is not None
            return u

        @staticmethod
        def backward(ctx, g):
            s64, r64, t64, gu = ctx.saved_tensors
            g = g.detach().to(torch.float64).contiguous()
            # the potential of charges g at the targets, and its gradient, at the sources
            if ctx.same:
                v, gv = plan.eval_grad(s64, g)
            else:
                v, gv = plan.eval_grad(t64, g, s64)
            d_rho = v.to(ctx.dtypes[1]) if ctx.needs_input_grad[1] else None
            d_src = d_tgt = None
            if ctx.needs_input_grad[0]:
                if ctx.same and ctx.has_gu:
                    d_src = adjoint_combine(r64, gv, g, gu)
                else:
                    d_src = adjoint_combine(r64, gv)
                d_src = d_src.to(ctx.dtypes[0])
            if not ctx.same and ctx.needs_input_grad[2] and ctx.has_gu:
                d_tgt = adjoint_combine(g, gu).to(ctx.dtypes[2])
            return d_src, d_rho, d_tgt

    return _Potential.apply(sources, charges, targets)
