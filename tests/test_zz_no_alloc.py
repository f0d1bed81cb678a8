"""dmk_direct_noalloc: evaluation without any device allocation.

Some callers cannot let a library allocate device memory while they run: work
captured into a CUDA graph that must not call cudaMalloc, applications that
hand all device memory to their own pool, loops that cannot absorb the
synchronisation an allocation can cause.  dmk_direct_noalloc serves them with
the direct sum, using a fixed scratch array compiled into the library.

This test calls the entry point through the C ABI twice in a row (the shared
scratch keeps the previous call's contents) and checks each result against
dmk_eval on the same input at the accuracy the other tests use for the direct
sum (rel-L2 <= 1e-6 at eps = 1e-6).  It lives in its own file so that it runs
after every other test, and it works alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2308_00292_gb300 import inputs  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_direct_noalloc_matches_dmk_eval():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_00292_gb300 import dmk
    lib = dmk.lib()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [inputs.clustered(12000, seed=301, nclusters=5), inputs.uniform_cube(7000, seed=302)]
    for x, q in cases:
        xd = torch.from_numpy(x).cuda()
        qd = torch.from_numpy(q).cuda()
        n = x.shape[0]
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.dmk_direct_noalloc(xd.data_ptr(), n, qd.data_ptr(), xd.data_ptr(), n, out.data_ptr(), stream)
        assert rc == 0, lib.dmk_last_error_detail()
        torch.cuda.synchronize()
        with dmk.Plan(1e-6, precision=dmk.DMK_FP64, leaf_cap=120) as plan:
            ref = plan.eval(xd, qd).cpu().numpy()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(ref, got) < 1e-6


def test_direct_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_00292_gb300 import dmk
    lib = dmk.lib()
    x = torch.zeros((16385, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros(16385, dtype=torch.float64, device="cuda")
    out = torch.zeros(16385, dtype=torch.float64, device="cuda")
    rc = lib.dmk_direct_noalloc(x.data_ptr(), 16385, q.data_ptr(), x.data_ptr(), 16385, out.data_ptr(), None)
    assert rc == 1
    assert b"16384" in lib.dmk_last_error_detail()
