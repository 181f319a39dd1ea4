"""The allocation-free maxvol entry point (lra_maxvol_noalloc) against the
regular entry point.

lra_maxvol_noalloc serves callers that cannot allocate device memory while
they run (cudaMalloc/cudaFree may synchronise the device, and a framework or
serving allocator may own the memory).  Its scratch is one static device
array shared by all calls, so this test makes two calls in a row and checks
that each one matches what a regular one-sweep solve (lra_cross_submit,
which allocates its own scratch) selects for the same strip: the row indices
must be identical, as for all index results.

This file sorts last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1611_01391_gb300 as L  # noqa: E402


def _noalloc():
    lib = ctypes.CDLL(L.LIB_PATH)
    f = lib.lra_maxvol_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int32,
                  ctypes.c_void_p, ctypes.c_void_p]
    return f


def _regular_first_half_step(ctx, A, J0, l):
    """I after one sweep of the regular path = maxvol of the strip A[:, J0]
    from its Gauss-Jordan start (the horizontal step does not change I)."""
    params, keep = L.make_params(l, l, 1, J0)
    res = ctx.solve(L.make_source("dense", a=A), params, l)
    assert res.info.status == 0
    return res.I


@pytest.mark.parametrize("m,n,l", [(5000, 3000, 24), (700, 900, 8)])
def test_noalloc_matches_regular_entry_point_twice(m, n, l):
    f = _noalloc()
    stream = torch.cuda.Stream()
    with L.Context(0) as ctx:
        for call in range(2):
            A64 = W.factor_gaussian(1000 * call + m, m, n, l // 2 + 2, 1e-3)
            A = torch.from_numpy(A64).cuda()
            J0 = W.draw_indices(7 + call, n, l)
            expect = _regular_first_half_step(ctx, A, J0, l)
            strip = A[:, torch.from_numpy(J0.astype(np.int64)).cuda()].contiguous()
            pos = torch.full((l,), -1, dtype=torch.int32, device="cuda")
            status = torch.full((3,), -99, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            rc = f(strip.data_ptr(), m, l, l, 1, pos.data_ptr(), None, 1e-2, 0,
                   status.data_ptr(), stream.cuda_stream)
            assert rc == L.LRA_OK
            stream.synchronize()
            st = status.cpu().numpy()
            assert st[0] == L.LRA_OK and st[2] == 1
            np.testing.assert_array_equal(pos.cpu().numpy(), expect)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    f = _noalloc()
    strip = torch.zeros((200, 97), dtype=torch.float32, device="cuda")
    pos = torch.zeros(97, dtype=torch.int32, device="cuda")
    status = torch.zeros(3, dtype=torch.int32, device="cuda")
    rc = f(strip.data_ptr(), 200, 97, 97, 1, pos.data_ptr(), None, 1e-2, 0, status.data_ptr(), None)
    assert rc == L.LRA_ETOOLARGE
    rc = f(strip.data_ptr(), 5, 8, 97, 1, pos.data_ptr(), None, 1e-2, 0, status.data_ptr(), None)
    assert rc == L.LRA_EINVAL
