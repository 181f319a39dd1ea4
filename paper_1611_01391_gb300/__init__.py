"""GB300 cross-approximation (C-A) CUR library: thin Python binding.

Every step of a solve runs in the CUDA kernels of ``_lib/liblra_cross.so``;
this module only marshals arguments to the C ABI of ``include/lra_cross.h``
(same function names).  PyTorch supplies device memory and streams.  There is
no CPU path: importing fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

LIB_PATH = _build.LIB

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"CUDA library missing: {LIB_PATH}. Build it first "
        "(python -c 'import __graft_entry__ as g; g.build()').")

_lib = ctypes.CDLL(LIB_PATH)

# ---- enums ----------------------------------------------------------------
LRA_OK, LRA_PENDING = 0, 1
LRA_EINVAL, LRA_ENOMEM, LRA_EBUSY, LRA_ESINGULAR = -1, -2, -3, -4
LRA_ENONFINITE, LRA_ETIMEOUT, LRA_ECUDA, LRA_ENOTFOUND = -5, -6, -7, -8
LRA_ECANCELED, LRA_ETOOLARGE = -9, -10

LRA_DENSE_F32, LRA_DENSE_F64, LRA_GEN_CAUCHY, LRA_GEN_GAUSS, LRA_GEN_INVDIST, LRA_PRE_AH = range(6)
LRA_TRACE_GEPP, LRA_TRACE_SWAP, LRA_TRACE_STOP, LRA_TRACE_CAP = range(4)
LRA_STATE_RUNNING, LRA_STATE_DONE, LRA_STATE_FAILED = range(3)
LRA_FLAG_PROFILE = 1
LRA_FLAG_FULL_RESIDUAL = 2


# ---- structs (layout of include/lra_cross.h) ------------------------------
class lra_ctx_params(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_slots", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_uint64), ("stream", ctypes.c_void_p),
                ("n_streams", ctypes.c_int32), ("max_grid", ctypes.c_int32)]


class lra_source(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dim", ctypes.c_int32),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("a", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("h", ctypes.c_float),
                ("pre_d", ctypes.c_int32), ("pre_perm_rows", ctypes.c_void_p), ("pre_sign_rows", ctypes.c_void_p),
                ("pre_perm_cols", ctypes.c_void_p), ("pre_sign_cols", ctypes.c_void_p),
                ("pre_materialized", ctypes.c_int32)]


class lra_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("l", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("max_swaps", ctypes.c_int32), ("delta", ctypes.c_double),
                ("rank_tol", ctypes.c_double), ("tol", ctypes.c_double),
                ("init_J", ctypes.c_void_p), ("resid_q", ctypes.c_int64),
                ("resid_s", ctypes.c_int64), ("resid_rows", ctypes.c_void_p),
                ("resid_cols", ctypes.c_void_p), ("trace_cap", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("init_I", ctypes.c_void_p), ("seed", ctypes.c_uint64)]


class lra_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32),
                ("sweeps_done", ctypes.c_int32), ("k_eff", ctypes.c_int32),
                ("swaps_total", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("trace_len", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("est_rel_err", ctypes.c_double), ("est_mu", ctypes.c_double),
                ("est_var", ctypes.c_double), ("sigma_max", ctypes.c_double),
                ("gpu_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int32),
                ("maxvol_launches", ctypes.c_int32), ("maxvol_flops", ctypes.c_double),
                ("t_gather_ms", ctypes.c_double), ("t_maxvol_ms", ctypes.c_double),
                ("t_cross_ms", ctypes.c_double), ("t_resid_ms", ctypes.c_double),
                ("t_inverse_ms", ctypes.c_double), ("full_rel_err", ctypes.c_double),
                ("t_fullres_ms", ctypes.c_double)]


class lra_cur_out(ctypes.Structure):
    _fields_ = [("on_device", ctypes.c_int32), ("I", ctypes.c_void_p), ("J", ctypes.c_void_p),
                ("U", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("R", ctypes.c_void_p), ("trace", ctypes.c_void_p), ("trace_val", ctypes.c_void_p)]


class lra_cynical_params(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int32), ("q", ctypes.c_int32), ("outer_loops", ctypes.c_int32),
                ("inner_sweeps", ctypes.c_int32), ("delta", ctypes.c_double), ("rank_tol", ctypes.c_double),
                ("K", ctypes.c_void_p), ("L", ctypes.c_void_p)]


class lra_cynical_out(ctypes.Structure):
    _fields_ = [("I", ctypes.c_void_p), ("J", ctypes.c_void_p), ("U", ctypes.c_void_p),
                ("K", ctypes.c_void_p), ("L", ctypes.c_void_p)]


class lra_refine_params(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int32), ("l_new", ctypes.c_int32), ("rank_tol", ctypes.c_double),
                ("u_cols", ctypes.c_void_p), ("u_rows", ctypes.c_void_p), ("resid_q", ctypes.c_int64),
                ("resid_s", ctypes.c_int64), ("resid_rows", ctypes.c_void_p), ("resid_cols", ctypes.c_void_p)]


class lra_refine_out(ctypes.Structure):
    _fields_ = [("cols", ctypes.c_void_p), ("d", ctypes.c_void_p), ("rows", ctypes.c_void_p),
                ("dbar", ctypes.c_void_p), ("U", ctypes.c_void_p), ("p_cols", ctypes.c_void_p),
                ("p_rows", ctypes.c_void_p), ("est_rel_err", ctypes.c_void_p), ("k_eff", ctypes.c_void_p)]


class lra_block(ctypes.Structure):
    _fields_ = [("row0", ctypes.c_int64), ("m", ctypes.c_int64),
                ("col0", ctypes.c_int64), ("n", ctypes.c_int64)]


class lra_batch_params(ctypes.Structure):
    _fields_ = [("l_init", ctypes.c_int32), ("l_max", ctypes.c_int32), ("k_max", ctypes.c_int32),
                ("sweeps", ctypes.c_int32), ("max_swaps", ctypes.c_int32), ("sample", ctypes.c_int32),
                ("tol", ctypes.c_double), ("delta", ctypes.c_double),
                ("cand_J", ctypes.c_void_p), ("sample_rows", ctypes.c_void_p),
                ("sample_cols", ctypes.c_void_p), ("flags", ctypes.c_int32), ("trace_cap", ctypes.c_int32),
                ("cluster_mask", ctypes.c_int32), ("cutover_side", ctypes.c_int32), ("order", ctypes.c_int32)]


class lra_batch_out(ctypes.Structure):
    _fields_ = [("on_device", ctypes.c_int32), ("status", ctypes.c_void_p), ("l", ctypes.c_void_p),
                ("k_eff", ctypes.c_void_p), ("swaps", ctypes.c_void_p), ("I", ctypes.c_void_p),
                ("J", ctypes.c_void_p), ("U", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("est_err", ctypes.c_void_p), ("trace_len", ctypes.c_void_p), ("trace", ctypes.c_void_p),
                ("trace_val", ctypes.c_void_p)]


_ctx_p = ctypes.c_void_p
_job = ctypes.c_uint64


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_create = _sig("lra_cross_create", ctypes.c_int, ctypes.POINTER(_ctx_p), ctypes.POINTER(lra_ctx_params))
_destroy = _sig("lra_cross_destroy", ctypes.c_int, _ctx_p)
_submit = _sig("lra_cross_submit", ctypes.c_int, _ctx_p, ctypes.POINTER(lra_source),
               ctypes.POINTER(lra_params), ctypes.POINTER(_job))
_poll = _sig("lra_cross_poll", ctypes.c_int, _ctx_p, _job, ctypes.POINTER(lra_info))
_wait = _sig("lra_cross_wait", ctypes.c_int, _ctx_p, _job, ctypes.POINTER(lra_info))
_fetch = _sig("lra_cross_fetch_cur", ctypes.c_int, _ctx_p, _job, ctypes.POINTER(lra_cur_out))
_cancel = _sig("lra_cross_cancel", ctypes.c_int, _ctx_p, _job)
_footprint = _sig("lra_cross_footprint", ctypes.c_int, ctypes.POINTER(lra_source),
                  ctypes.POINTER(lra_params), ctypes.POINTER(ctypes.c_uint64))
_submit_batch = _sig("lra_cross_submit_batch", ctypes.c_int, _ctx_p, ctypes.POINTER(lra_source),
                     ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(lra_batch_params),
                     ctypes.POINTER(_job))
_fetch_batch = _sig("lra_cross_fetch_batch", ctypes.c_int, _ctx_p, _job, ctypes.POINTER(lra_batch_out))
_draw_columns = _sig("lra_draw_columns", ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                     ctypes.c_void_p)
_gather_entries = _sig("lra_gather_entries", ctypes.c_int, ctypes.POINTER(lra_source), ctypes.c_void_p,
                       ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p)
_maxvol_noalloc = _sig("lra_maxvol_noalloc", ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                       ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p)
_tune_batch = _sig("lra_cross_tune_batch", ctypes.c_int, _ctx_p, ctypes.POINTER(lra_source), ctypes.c_void_p,
                   ctypes.c_int32, ctypes.POINTER(lra_batch_params), ctypes.c_char_p,
                   ctypes.POINTER(lra_batch_params), ctypes.POINTER(ctypes.c_double),
                   ctypes.POINTER(ctypes.c_double))
_tuning_lookup = _sig("lra_batch_tuning_lookup", ctypes.c_int, ctypes.c_char_p, ctypes.c_char_p,
                      ctypes.POINTER(lra_source), ctypes.c_void_p, ctypes.c_int32,
                      ctypes.POINTER(lra_batch_params), ctypes.POINTER(lra_batch_params))
_cynical = _sig("lra_cross_cynical", ctypes.c_int, _ctx_p, ctypes.POINTER(lra_source),
                ctypes.POINTER(lra_cynical_params), ctypes.POINTER(lra_cynical_out))
_refine = _sig("lra_cross_refine", ctypes.c_int, _ctx_p, ctypes.POINTER(lra_source), ctypes.c_void_p,
               ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(lra_refine_params), ctypes.POINTER(lra_refine_out))
_pre_recover = _sig("lra_preprocessed_recover", ctypes.c_int, ctypes.POINTER(lra_source), ctypes.c_void_p,
                    ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_pre_materialize = _sig("lra_preprocess_materialize", ctypes.c_int, ctypes.POINTER(lra_source), ctypes.c_void_p,
                        ctypes.c_int64, ctypes.c_void_p)
class lra_rf_params(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int32), ("rank_tol", ctypes.c_double), ("resid_q", ctypes.c_int64),
                ("resid_s", ctypes.c_int64), ("resid_rows", ctypes.c_void_p), ("resid_cols", ctypes.c_void_p),
                ("mult_d", ctypes.c_int32), ("mult_sign", ctypes.c_void_p)]


class lra_rf_out(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p), ("V", ctypes.c_void_p), ("piv", ctypes.c_void_p), ("nrank", ctypes.c_void_p),
                ("est_rel_err", ctypes.c_void_p), ("gemm_mode", ctypes.c_void_p)]


class lra_lsr_params(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int32), ("shifted", ctypes.c_int32), ("mult_d", ctypes.c_int32),
                ("mult_sign", ctypes.c_void_p)]


class lra_lsr_out(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("rho", ctypes.c_void_p)]


_range_finder = _sig("lra_range_finder", ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(lra_source), ctypes.c_void_p,
                     ctypes.c_int32, ctypes.POINTER(lra_rf_params), ctypes.POINTER(lra_rf_out))
_dual_lsr = _sig("lra_dual_lsr", ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(lra_source), ctypes.c_void_p,
                 ctypes.c_int32, ctypes.POINTER(lra_lsr_params), ctypes.POINTER(lra_lsr_out))
_status_str = _sig("lra_status_str", ctypes.c_char_p, ctypes.c_int32)
_last_error = _sig("lra_cross_last_error", ctypes.c_char_p, _ctx_p)

EXPORTED = ["lra_cross_create", "lra_cross_destroy", "lra_cross_submit", "lra_cross_poll",
            "lra_cross_wait", "lra_cross_fetch_cur", "lra_cross_cancel", "lra_cross_footprint",
            "lra_status_str", "lra_cross_last_error", "lra_cross_submit_batch",
            "lra_cross_fetch_batch", "lra_draw_columns", "lra_gather_entries", "lra_maxvol_noalloc",
            "lra_cross_tune_batch", "lra_batch_tuning_lookup", "lra_cross_cynical", "lra_cross_refine",
            "lra_preprocessed_recover", "lra_preprocess_materialize", "lra_range_finder", "lra_dual_lsr"]


class LraError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{lra_status_str(code)} ({code}){': ' + msg if msg else ''}")
        self.code = code


def lra_status_str(code: int) -> str:
    return _status_str(int(code)).decode()


def lra_cross_last_error(ctx) -> str:
    return _last_error(ctx).decode()


def _check(code, ctx=None, ok=(LRA_OK,)):
    if code not in ok:
        raise LraError(code, lra_cross_last_error(ctx) if ctx else "")
    return code


# ---- the C ABI, one function per entry point --------------------------------
def lra_cross_create(device: int = 0, max_slots: int = 64, mem_budget_bytes: int = 0, stream=None,
                     n_streams: int = 1, max_grid: int = 0):
    p = lra_ctx_params(device, max_slots, mem_budget_bytes, stream or None, n_streams, max_grid)
    ctx = _ctx_p()
    _check(_create(ctypes.byref(ctx), ctypes.byref(p)))
    return ctx


def lra_cross_destroy(ctx) -> None:
    _check(_destroy(ctx))


def lra_cross_submit(ctx, src: lra_source, params: lra_params) -> int:
    job = _job()
    _check(_submit(ctx, ctypes.byref(src), ctypes.byref(params), ctypes.byref(job)), ctx)
    return job.value


def lra_cross_poll(ctx, job: int):
    info = lra_info()
    code = _poll(ctx, job, ctypes.byref(info))
    _check(code, ctx, ok=(LRA_OK, LRA_PENDING))
    return code, info


def lra_cross_wait(ctx, job: int) -> lra_info:
    info = lra_info()
    _check(_wait(ctx, job, ctypes.byref(info)), ctx)
    return info


def lra_cross_fetch_cur(ctx, job: int, out: lra_cur_out) -> int:
    return _check(_fetch(ctx, job, ctypes.byref(out)), ctx)


def lra_cross_cancel(ctx, job: int) -> None:
    _check(_cancel(ctx, job), ctx)


def lra_cross_submit_batch(ctx, src: lra_source, blocks, params: lra_batch_params) -> int:
    """blocks: int64 array (n_blocks x 4: row0, m, col0, n), C-contiguous."""
    job = _job()
    _check(_submit_batch(ctx, ctypes.byref(src), blocks.ctypes.data, len(blocks), ctypes.byref(params),
                         ctypes.byref(job)), ctx)
    return job.value


def lra_cross_fetch_batch(ctx, job: int, out: lra_batch_out) -> int:
    return _check(_fetch_batch(ctx, job, ctypes.byref(out)), ctx)


def lra_draw_columns(seed: int, n: int, l: int):
    """Initial column set drawn from a seed (host only), as numpy int32[l]."""
    import numpy as np
    out = np.zeros(l, np.int32)
    _check(_draw_columns(seed, n, l, out.ctypes.data))
    return out


def lra_gather_entries(src: lra_source, rows, cols, out, stream=None) -> None:
    """out[a, b] = M(rows[a], cols[b]) on the device (device int32 rows/cols,
    device float32 out of shape (len(rows), len(cols)))."""
    _check(_gather_entries(ctypes.byref(src), rows.data_ptr(), rows.numel(), cols.data_ptr(), cols.numel(),
                           out.data_ptr(), stream))


def lra_maxvol_noalloc(strip_ptr, N, l, row_stride, col_stride, pos_ptr, xinv_ptr, delta, max_swaps,
                       status_ptr, stream=None) -> int:
    """One maxvol half-step without device allocation (raw device pointers);
    returns the lra_status code."""
    return _maxvol_noalloc(strip_ptr, N, l, row_stride, col_stride, pos_ptr, xinv_ptr, delta, max_swaps,
                           status_ptr, stream)


def lra_range_finder(ctx, src: lra_source, J, r: int, U, V, rank_tol: float = 1e-6, resid_rows=None,
                     resid_cols=None, mult_d: int = 0, mult_sign=None):
    """Algorithm 5.1a with the sub-identity multiplier e_J (mult_d = 0) or
    the ASPH multiplier whose column t is mult_sign[t] times column J[t] of
    H_{n,mult_d}: U (m x r) and V (r x n) into the given float32 device
    tensors.  Returns a dict with piv, nrank, est_rel_err and gemm_mode."""
    import numpy as np
    Jh = np.ascontiguousarray(J, dtype=np.int32)
    p = lra_rf_params(r, rank_tol, 0, 0, None, None, mult_d, None)
    keep = []
    if mult_sign is not None:
        sg = np.ascontiguousarray(mult_sign, dtype=np.float32)
        keep.append(sg)
        p.mult_sign = sg.ctypes.data
    if resid_rows is not None:
        rr = np.ascontiguousarray(resid_rows, dtype=np.int32)
        rc = np.ascontiguousarray(resid_cols, dtype=np.int32)
        keep += [rr, rc]
        p.resid_q, p.resid_s, p.resid_rows, p.resid_cols = len(rr), len(rc), rr.ctypes.data, rc.ctypes.data
    piv = np.zeros(len(Jh), np.int32)
    nrank = np.zeros(1, np.int32)
    est = np.zeros(1)
    mode = np.zeros(1, np.int32)
    o = lra_rf_out(U.data_ptr(), V.data_ptr(), piv.ctypes.data, nrank.ctypes.data, est.ctypes.data, mode.ctypes.data)
    code = _range_finder(ctx, ctypes.byref(src), Jh.ctypes.data, len(Jh), ctypes.byref(p), ctypes.byref(o))
    res = {"piv": piv, "nrank": int(nrank[0]), "est_rel_err": float(est[0]), "gemm_mode": int(mode[0]),
           "status": int(code)}
    if code != LRA_OK and code != LRA_ESINGULAR:
        _check(code, ctx)
    return res


def lra_dual_lsr(ctx, W: lra_source, rows, passes: int = 3, shifted: bool = True, mult_d: int = 0,
                 mult_sign=None):
    """Algorithm 3.1 with a sub-identity multiplier (mult_d = 0: the kept
    rows) or the ASPH multiplier whose row t is mult_sign[t] times row
    rows[t] of H_{m,mult_d}: x (host FP64, n) and the sampled residual norm
    for W = (A | b)."""
    import numpy as np
    rh = np.ascontiguousarray(rows, dtype=np.int32)
    x = np.zeros(W.n - 1)
    rho = np.zeros(1)
    p = lra_lsr_params(passes, int(bool(shifted)), mult_d, None)
    sg = None
    if mult_sign is not None:
        sg = np.ascontiguousarray(mult_sign, dtype=np.float32)
        p.mult_sign = sg.ctypes.data
    o = lra_lsr_out(x.ctypes.data, rho.ctypes.data)
    _check(_dual_lsr(ctx, ctypes.byref(W), rh.ctypes.data, len(rh), ctypes.byref(p), ctypes.byref(o)), ctx)
    return x, float(rho[0])


def lra_preprocess_materialize(pre: lra_source, G, stream=None) -> None:
    """G = H_{m,d} M H_{n,d} on the device (torch float32 tensor, row-major)."""
    _check(_pre_materialize(ctypes.byref(pre), G.data_ptr(), G.stride(0), stream))


def lra_preprocessed_recover(pre: lra_source, Cbar, Rbar, A, B, stream=None) -> None:
    """A = F^T Cbar / 2^d, B = Rbar H^T / 2^d on the device (torch float32 tensors)."""
    _check(_pre_recover(ctypes.byref(pre), Cbar.data_ptr(), Rbar.data_ptr(), Cbar.shape[1], A.data_ptr(),
                        B.data_ptr(), stream))


def lra_cross_refine(ctx, src: lra_source, I, J, r: int, l_new: int, u_cols, u_rows, rank_tol: float = 1e-6,
                     resid_rows=None, resid_cols=None, scores: bool = False):
    """Section 7.2 refinement of the C-A CUR of (I, J): returns a dict with
    cols, d, rows, dbar, U (l_new x l_new), k_eff, est_rel_err and, with
    scores, the column and row scores p_cols (n), p_rows (m)."""
    import numpy as np
    Ih = np.ascontiguousarray(I, dtype=np.int32)
    Jh = np.ascontiguousarray(J, dtype=np.int32)
    uc = np.ascontiguousarray(u_cols, dtype=np.float64)
    ur = np.ascontiguousarray(u_rows, dtype=np.float64)
    p = lra_refine_params(r, l_new, rank_tol, uc.ctypes.data, ur.ctypes.data, 0, 0, None, None)
    keep = []
    if resid_rows is not None:
        rr = np.ascontiguousarray(resid_rows, dtype=np.int32)
        rc = np.ascontiguousarray(resid_cols, dtype=np.int32)
        keep += [rr, rc]
        p.resid_q, p.resid_s, p.resid_rows, p.resid_cols = len(rr), len(rc), rr.ctypes.data, rc.ctypes.data
    res = {"cols": np.zeros(l_new, np.int32), "d": np.zeros(l_new), "rows": np.zeros(l_new, np.int32),
           "dbar": np.zeros(l_new), "U": np.zeros((l_new, l_new)), "est_rel_err": np.zeros(1),
           "k_eff": np.zeros(1, np.int32)}
    if scores:
        res["p_cols"] = np.zeros(src.n)
        res["p_rows"] = np.zeros(src.m)
    o = lra_refine_out(res["cols"].ctypes.data, res["d"].ctypes.data, res["rows"].ctypes.data,
                       res["dbar"].ctypes.data, res["U"].ctypes.data,
                       res["p_cols"].ctypes.data if scores else None, res["p_rows"].ctypes.data if scores else None,
                       res["est_rel_err"].ctypes.data, res["k_eff"].ctypes.data)
    _check(_refine(ctx, ctypes.byref(src), Ih.ctypes.data, Jh.ctypes.data, len(Ih), ctypes.byref(p),
                   ctypes.byref(o)), ctx)
    res["est_rel_err"] = float(res["est_rel_err"][0])
    res["k_eff"] = int(res["k_eff"][0])
    return res


def lra_cross_cynical(ctx, src: lra_source, r: int, L, K=None, outer_loops: int = 1, inner_sweeps: int = 2,
                      delta: float = 1e-2, rank_tol: float = 1e-6):
    """Tests 3 (K given, outer_loops = 0) or Tests 4 (outer_loops >= 1):
    returns (I, J, U, K used, L used) as numpy arrays."""
    import numpy as np
    Lh = np.ascontiguousarray(L, dtype=np.int32)
    q = len(Lh)
    Kh = None if K is None else np.ascontiguousarray(K, dtype=np.int32)
    p = lra_cynical_params(r, q, outer_loops, inner_sweeps, delta, rank_tol,
                           None if Kh is None else Kh.ctypes.data, Lh.ctypes.data)
    I, J = np.zeros(r, np.int32), np.zeros(r, np.int32)
    U = np.zeros((r, r), np.float64)
    Ko, Lo = np.zeros(q, np.int32), np.zeros(q, np.int32)
    o = lra_cynical_out(I.ctypes.data, J.ctypes.data, U.ctypes.data, Ko.ctypes.data, Lo.ctypes.data)
    _check(_cynical(ctx, ctypes.byref(src), ctypes.byref(p), ctypes.byref(o)), ctx)
    return I, J, U, Ko, Lo


def lra_cross_tune_batch(ctx, src: lra_source, blocks, params: lra_batch_params, cache_path=None):
    """(tuned lra_batch_params, ms_default, ms_tuned); blocks as for submit_batch."""
    tuned = lra_batch_params()
    md, mt = ctypes.c_double(), ctypes.c_double()
    _check(_tune_batch(ctx, ctypes.byref(src), blocks.ctypes.data, len(blocks), ctypes.byref(params),
                       None if cache_path is None else str(cache_path).encode(), ctypes.byref(tuned),
                       ctypes.byref(md), ctypes.byref(mt)), ctx)
    return tuned, md.value, mt.value


def lra_batch_tuning_lookup(cache_path, gpu_name: str, src: lra_source, blocks, params: lra_batch_params):
    """The cached launch shape for this GPU and workload bucket, or None."""
    tuned = lra_batch_params()
    code = _tuning_lookup(str(cache_path).encode(), gpu_name.encode(), ctypes.byref(src), blocks.ctypes.data,
                          len(blocks), ctypes.byref(params), ctypes.byref(tuned))
    if code == LRA_ENOTFOUND:
        return None
    _check(code)
    return tuned


def lra_cross_footprint(src: lra_source, params: lra_params) -> int:
    b = ctypes.c_uint64()
    _check(_footprint(ctypes.byref(src), ctypes.byref(params), ctypes.byref(b)))
    return b.value


from .api import BatchResult, Context, SolveResult, make_params, make_source, solve_preprocessed  # noqa: E402

__all__ = EXPORTED + ["Context", "SolveResult", "BatchResult", "LraError", "make_params", "make_source",
                      "solve_preprocessed",
                      "lra_source", "lra_params", "lra_info", "lra_cur_out", "LIB_PATH"]
