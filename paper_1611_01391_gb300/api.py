"""Convenience layer over the C ABI: builds the argument structs from torch
tensors / numpy arrays and runs submit -> wait -> fetch.  Argument
marshalling only; the solve itself runs in the library's kernels."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import (LRA_DENSE_F32, LRA_DENSE_F64, LRA_GEN_CAUCHY, LRA_GEN_GAUSS, LRA_GEN_INVDIST, LRA_PRE_AH,
               lra_batch_out, lra_batch_params, lra_cross_create, lra_cross_destroy,
               lra_cross_fetch_batch, lra_cross_fetch_cur, lra_cross_submit, lra_cross_submit_batch,
               lra_cross_wait, lra_cur_out, lra_info, lra_params, lra_preprocessed_recover, lra_source)

_KINDS = {"dense": None, "cauchy": LRA_GEN_CAUCHY, "gauss": LRA_GEN_GAUSS,
          "invdist": LRA_GEN_INVDIST}


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def make_source(kind: str, *, a=None, x=None, y=None, h: float = 0.0, d: int = 0, perm_rows=None,
                sign_rows=None, perm_cols=None, sign_cols=None, materialized: bool = False) -> lra_source:
    """Source descriptor from device tensors (kept alive by the caller).
    kind "preprocessed": M_bar = F M H for the stored FP32 a and the abridged
    Hadamard multipliers of depth d (int32 permutations, float32 +-1 signs);
    materialized: a already holds H_{m,d} M H_{n,d}."""
    import torch
    if kind == "preprocessed":
        if a.dtype != torch.float32 or not a.is_cuda or a.dim() != 2 or a.stride(1) != 1:
            raise ValueError("preprocessed source: row-major 2-D float32 CUDA tensor required")
        for t, dt in ((perm_rows, torch.int32), (sign_rows, torch.float32), (perm_cols, torch.int32),
                      (sign_cols, torch.float32)):
            if t is None or t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise ValueError("preprocessed source: int32 permutations and float32 signs on the device")
        return lra_source(LRA_PRE_AH, 0, a.shape[0], a.shape[1], a.data_ptr(), a.stride(0), None, None, 0.0,
                          d, perm_rows.data_ptr(), sign_rows.data_ptr(), perm_cols.data_ptr(), sign_cols.data_ptr(),
                          int(bool(materialized)))
    if kind == "dense":
        if a.dtype not in (torch.float32, torch.float64) or not a.is_cuda or a.dim() != 2:
            raise ValueError("dense source: 2-D float32/float64 CUDA tensor required")
        if a.stride(1) != 1:
            raise ValueError("dense source must be row-major")
        k = LRA_DENSE_F32 if a.dtype == torch.float32 else LRA_DENSE_F64
        return lra_source(k, 0, a.shape[0], a.shape[1], a.data_ptr(), a.stride(0), None, None, 0.0)
    kd = _KINDS[kind]
    if x.dtype != torch.float32 or y.dtype != torch.float32 or not x.is_cuda or not y.is_cuda:
        raise ValueError("generator points: float32 CUDA tensors required")
    if not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("generator points must be contiguous")
    dim = 1 if x.dim() == 1 else x.shape[1]
    return lra_source(kd, dim, x.shape[0], y.shape[0], None, 0, x.data_ptr(), y.data_ptr(), float(h))


@dataclass
class _HostArrays:
    J0: np.ndarray | None
    rows: np.ndarray | None
    cols: np.ndarray | None
    I0: np.ndarray | None = None


def make_params(k, l, sweeps, init_J, *, delta=1e-2, rank_tol=1e-6, tol=0.0, max_swaps=0,
                resid_rows=None, resid_cols=None, trace_cap=0, profile=False, full_residual=False,
                init_I=None, seed=0):
    """lra_params plus the host arrays it points to (keep both alive).
    init_J None: the library draws J from ``seed``; init_I: resume from a row set."""
    J0 = None if init_J is None else np.ascontiguousarray(init_J, dtype=np.int32)
    I0 = None if init_I is None else np.ascontiguousarray(init_I, dtype=np.int32)
    rows = None if resid_rows is None else np.ascontiguousarray(resid_rows, dtype=np.int32)
    cols = None if resid_cols is None else np.ascontiguousarray(resid_cols, dtype=np.int32)
    p = lra_params()
    p.k, p.l, p.sweeps, p.max_swaps = k, l, sweeps, max_swaps
    p.delta, p.rank_tol, p.tol = delta, rank_tol, tol
    p.init_J = None if J0 is None else J0.ctypes.data
    p.init_I = None if I0 is None else I0.ctypes.data
    p.seed = int(seed)
    if rows is not None:
        p.resid_q, p.resid_s = len(rows), len(cols)
        p.resid_rows, p.resid_cols = rows.ctypes.data, cols.ctypes.data
    p.trace_cap = trace_cap
    p.flags = (1 if profile else 0) | (2 if full_residual else 0)
    return p, _HostArrays(J0, rows, cols, I0)


@dataclass
class SolveResult:
    I: np.ndarray
    J: np.ndarray
    U: np.ndarray
    sigma: np.ndarray
    info: lra_info
    C: object = None
    R: object = None
    trace: np.ndarray | None = None
    trace_val: np.ndarray | None = None


class Context:
    """One library context (one device, one stream)."""

    def __init__(self, device=0, max_slots=64, mem_budget_bytes=0, stream=None, n_streams=1, max_grid=0):
        self.ctx = lra_cross_create(device, max_slots, mem_budget_bytes, stream, n_streams, max_grid)

    def close(self):
        if self.ctx:
            lra_cross_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, src, params):
        return lra_cross_submit(self.ctx, src, params)

    def fetch(self, job, l, m=None, n=None, want_strips=False, trace_cap=0, device=None):
        """Fetch I, J, U, sigma (host numpy) and optionally C, R as device tensors."""
        import torch
        info = lra_cross_wait(self.ctx, job)
        I = np.zeros(l, np.int32)
        J = np.zeros(l, np.int32)
        U = np.zeros((l, l), np.float64)
        sigma = np.zeros(l, np.float64)
        out = lra_cur_out()
        out.on_device = 0
        out.I, out.J, out.U, out.sigma = I.ctypes.data, J.ctypes.data, U.ctypes.data, sigma.ctypes.data
        C = R = None
        tr = tv = None
        if want_strips:
            C = torch.empty((m, l), dtype=torch.float32, device=device)
            R = torch.empty((l, n), dtype=torch.float32, device=device)
            out.C, out.R = C.data_ptr(), R.data_ptr()
        if trace_cap:
            tr = np.zeros((trace_cap, 4), np.int32)
            tv = np.zeros(trace_cap, np.float64)
            out.trace, out.trace_val = tr.ctypes.data, tv.ctypes.data
        lra_cross_fetch_cur(self.ctx, job, out)
        if tr is not None:
            tr, tv = tr[:info.trace_len], tv[:info.trace_len]
        return SolveResult(I, J, U, sigma, info, C, R, tr, tv)

    def solve(self, src, params, l, m=None, n=None, want_strips=False, trace_cap=0, device=None):
        job = self.submit(src, params)
        return self.fetch(job, l, m, n, want_strips, trace_cap, device)


@dataclass
class BatchResult:
    status: np.ndarray
    l: np.ndarray
    k_eff: np.ndarray
    swaps: np.ndarray
    I: np.ndarray
    J: np.ndarray
    U: np.ndarray
    sigma: np.ndarray
    est_err: np.ndarray
    info: lra_info
    trace_len: np.ndarray | None = None
    trace: np.ndarray | None = None
    trace_val: np.ndarray | None = None

    def block_trace(self, b):
        """Decision log of block b as rows (half_step, kind, i, j)."""
        n = int(self.trace_len[b])
        return self.trace[b, :n], self.trace_val[b, :n]


def make_batch_params(l_init, l_max, k_max, sweeps, tol, cand_J, sample_rows=None, sample_cols=None,
                      delta=1e-2, max_swaps=0, trace_cap=0):
    """lra_batch_params plus the host arrays it points to (keep both alive)."""
    cj = np.ascontiguousarray(cand_J, dtype=np.int32)
    sr = None if sample_rows is None else np.ascontiguousarray(sample_rows, dtype=np.int32)
    sc = None if sample_cols is None else np.ascontiguousarray(sample_cols, dtype=np.int32)
    p = lra_batch_params()
    p.l_init, p.l_max, p.k_max, p.sweeps, p.max_swaps = l_init, l_max, k_max, sweeps, max_swaps
    p.sample = 0 if sr is None else sr.shape[1]
    p.tol, p.delta = tol, delta
    p.cand_J = cj.ctypes.data
    if sr is not None:
        p.sample_rows, p.sample_cols = sr.ctypes.data, sc.ctypes.data
    p.flags = 0
    p.trace_cap = trace_cap
    return p, (cj, sr, sc)


def _batch_fetch(ctx, job, nb, l_max, trace_cap=0):
    info = lra_cross_wait(ctx, job)
    r = BatchResult(np.zeros(nb, np.int32), np.zeros(nb, np.int32), np.zeros(nb, np.int32),
                    np.zeros(nb, np.int32), np.zeros((nb, l_max), np.int32),
                    np.zeros((nb, l_max), np.int32), np.zeros((nb, l_max, l_max), np.float64),
                    np.zeros((nb, l_max), np.float32), np.zeros(nb, np.float64), info)
    out = lra_batch_out()
    out.on_device = 0
    out.status, out.l, out.k_eff, out.swaps = (r.status.ctypes.data, r.l.ctypes.data,
                                               r.k_eff.ctypes.data, r.swaps.ctypes.data)
    out.I, out.J, out.U = r.I.ctypes.data, r.J.ctypes.data, r.U.ctypes.data
    out.sigma, out.est_err = r.sigma.ctypes.data, r.est_err.ctypes.data
    if trace_cap:
        r.trace_len = np.zeros(nb, np.int32)
        r.trace = np.zeros((nb, trace_cap, 4), np.int32)
        r.trace_val = np.zeros((nb, trace_cap), np.float64)
        out.trace_len, out.trace, out.trace_val = (r.trace_len.ctypes.data, r.trace.ctypes.data,
                                                   r.trace_val.ctypes.data)
    lra_cross_fetch_batch(ctx, job, out)
    return r


def solve_batch(context, src, blocks, params, l_max):
    """Submit one batched launch and fetch every block's result (host arrays)."""
    blocks = np.ascontiguousarray(blocks, dtype=np.int64)
    job = lra_cross_submit_batch(context.ctx, src, blocks, params)
    return _batch_fetch(context.ctx, job, len(blocks), l_max, params.trace_cap)


def solve_preprocessed(context, pre, params, l, m, n, trace_cap=0, device=None):
    """C-A on M_bar = F M H (an LRA_PRE_AH source), then the LRA A U B of M
    it induces (Section 6.6): A = F^T Cbar / 2^d, B = Rbar H^T / 2^d, on the
    device.  Returns (SolveResult on M_bar with device strips C, R; A; B)."""
    import torch
    res = context.solve(pre, params, l, m, n, want_strips=True, trace_cap=trace_cap, device=device)
    A = torch.empty((m, l), dtype=torch.float32, device=res.C.device)
    B = torch.empty((l, n), dtype=torch.float32, device=res.C.device)
    stream = torch.cuda.current_stream(res.C.device).cuda_stream
    lra_preprocessed_recover(pre, res.C, res.R, A, B, stream)
    return res, A, B
