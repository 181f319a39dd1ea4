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

import oracle as O  # noqa: E402
import paper_1611_01391_gb300 as L  # noqa: E402
from tests._parity import separated  # noqa: E402


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


@pytest.mark.parametrize("m,l", [(6000, 24), (3000, 40), (2500, 96)])
def test_noalloc_warm_start_from_caller_inverse(m, l):
    """Warm start (Section 6.5: each half-step starts from the previous index
    set) with the caller's FP64 inverse of the cross S[pos, :]: the rows kept
    after the maxvol swaps are the FP64 oracle's (same FP32 entries) wherever
    every decision of the oracle's log is separated; otherwise they must at
    least be a dominant set (max |S S[pos, :]^{-1}| <= 1 + delta)."""
    f = _noalloc()
    delta = 1e-2
    S32 = W.factor_gaussian(31 * m + l, m, l, l, 1e-2).astype(np.float32)
    S64 = S32.astype(np.float64)
    pos0 = W.draw_indices(17 * m + l, m, l)
    xinv = np.linalg.inv(S64[pos0, :])
    trace = []
    ref = O.maxvol(S64, pos0, delta=delta, trace=trace)
    strip = torch.from_numpy(S32).cuda()
    pos = torch.from_numpy(np.asarray(pos0, np.int32)).cuda()
    xd = torch.from_numpy(np.ascontiguousarray(xinv)).cuda()
    status = torch.full((3,), -99, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = f(strip.data_ptr(), m, l, l, 1, pos.data_ptr(), xd.data_ptr(), delta, 0, status.data_ptr(), None)
    assert rc == L.LRA_OK
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    assert st[0] == L.LRA_OK and st[2] == 1
    got = pos.cpu().numpy()
    assert len(set(got.tolist())) == l
    if all(separated(d, delta) for d in trace):
        np.testing.assert_array_equal(got, np.asarray(ref.I))
        assert st[1] == ref.swaps
    else:
        B = np.linalg.solve(S64[got, :].T, S64.T).T
        assert np.abs(B).max() <= 1.0 + delta + 1e-9


def test_noalloc_rejects_sizes_beyond_its_scratch():
    f = _noalloc()
    strip = torch.zeros((200, 97), dtype=torch.float32, device="cuda")
    pos = torch.zeros(97, dtype=torch.int32, device="cuda")
    status = torch.zeros(3, dtype=torch.int32, device="cuda")
    rc = f(strip.data_ptr(), 200, 97, 97, 1, pos.data_ptr(), None, 1e-2, 0, status.data_ptr(), None)
    assert rc == L.LRA_ETOOLARGE
    rc = f(strip.data_ptr(), 5, 8, 97, 1, pos.data_ptr(), None, 1e-2, 0, status.data_ptr(), None)
    assert rc == L.LRA_EINVAL
