"""dmk_direct_noalloc: the direct sum without any device allocation.

Some callers cannot let a library allocate device memory while they run:
applications that hand all device memory to their own pool, code recorded for
replay that must not call cudaMalloc, loops that cannot absorb the
synchronisation an allocation can cause.  dmk_direct_noalloc serves them with
the direct sum, using a fixed scratch array compiled into the library.

The entry point computes a plain definition (eq. discretesum with K = 1/r,
coincident pairs excluded), so it is checked element by element against the
oracle's compensated FP64 direct sum: |u_i - u_i^oracle| <= 1e-12 A_i with
A_i = sum_j |rho_j| / |x_i - y_j|, the rounding bound of a sum of at most a few
ten thousand FP64 terms.  Every case calls the entry point through the C ABI
twice in a row (the shared scratch keeps the previous call's contents) and
covers separate targets, targets that coincide with sources, n_tgt = 0,
n_src = 0 and the size limit.  This file runs after every other test, and it
passes alone in a fresh process too.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2308_00292_gb300 import inputs  # noqa: E402


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_00292_gb300 import dmk
    return dmk.lib()


def _call(lib, src, q, tgt, out):
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.dmk_direct_noalloc(src.data_ptr() if src.numel() else None, src.shape[0],
                                q.data_ptr() if q.numel() else None,
                                tgt.data_ptr() if tgt.numel() else None, tgt.shape[0],
                                out.data_ptr() if out.numel() else None, stream)
    torch.cuda.synchronize()
    return rc


def _check(oracle_mod, x, q, y, got):
    ref = oracle_mod.direct(x, q, y)
    bound = oracle_mod.direct(x, np.abs(q), y)  # A_i = sum |rho_j| / r_ij
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= 1e-12 * bound + 1e-300), float(np.max(np.abs(got - ref) / bound))


def _cases():
    x1, q1 = inputs.clustered(12000, seed=301, nclusters=5)
    x2, q2 = inputs.uniform_cube(7000, seed=302)
    y2, _ = inputs.uniform_cube(5000, seed=303)
    y2[:20] = x2[:20]            # targets on top of sources: their own terms drop out
    y2[20] = x2[100]
    return [(x1, q1, None), (x2, q2, y2)]


def test_direct_noalloc_matches_oracle_direct_sum(oracle_mod):
    lib = _lib()
    for x, q, y in _cases():
        xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
        yd = xd if y is None else torch.from_numpy(y).cuda()
        yy = x if y is None else y
        for _ in range(2):  # two calls in a row share the scratch
            out = torch.full((yd.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
            assert _call(lib, xd, qd, yd, out) == 0, lib.dmk_last_error_detail()
            _check(oracle_mod, x, q, yy, out.cpu().numpy())
        assert lib.dmk_last_error_detail() == b""


def test_direct_noalloc_empty_inputs(oracle_mod):
    lib = _lib()
    x, q = inputs.uniform_cube(300, seed=304)
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    # no targets: nothing is written
    sentinel = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    empty = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    assert _call(lib, xd, qd, empty, sentinel[:0]) == 0
    assert torch.all(sentinel == 7.0)
    # no sources: every potential is zero
    out = torch.full((300,), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(lib, empty, torch.empty(0, dtype=torch.float64, device="cuda"), xd, out) == 0
    assert torch.all(out == 0.0)
    # and a full call right after still matches the oracle
    out = torch.full((300,), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(lib, xd, qd, xd, out) == 0
    _check(oracle_mod, x, q, x, out.cpu().numpy())


def test_direct_noalloc_rejects_oversize():
    lib = _lib()
    x = torch.zeros((16385, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros(16385, dtype=torch.float64, device="cuda")
    out = torch.zeros(16385, dtype=torch.float64, device="cuda")
    rc = lib.dmk_direct_noalloc(x.data_ptr(), 16385, q.data_ptr(), x.data_ptr(), 16385, out.data_ptr(), None)
    assert rc == 1
    assert b"16384" in lib.dmk_last_error_detail()
    # the limit itself is accepted
    rc = lib.dmk_direct_noalloc(x.data_ptr(), 100, q.data_ptr(), x.data_ptr(), 16384, out.data_ptr(), None)
    torch.cuda.synchronize()
    assert rc == 0
