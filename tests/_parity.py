"""Shared helpers of the GPU parity tests (no GPU needed to import)."""
from __future__ import annotations

import numpy as np

import oracle as O

# A decision is "separated" when its competing volume ratios differ by more
# than this relative amount: swapping row i into position j multiplies the
# volume by |B_ij|, so the candidates are the entries of |B| (GEPP: of the
# pivot column); the stop test compares max |B| with 1 + delta.
SEPARATION = 1e-6

# Truncation threshold of the nucleus on the device (FP32 entries); the FP64
# oracle's own default is 1e-12.  Input-matched comparisons (same entries,
# same decisions, same U) run the oracle at the device's threshold; the error
# bar is the pure-FP64 oracle at its default.
GPU_TAU = 1e-6


def separated(dec, delta):
    hs, kind, i, j, v1, v2 = dec
    if kind in (O.GEPP, O.SWAP):
        return v1 > 0 and (v1 - v2) / v1 > SEPARATION
    return abs(v1 - (1.0 + delta)) / (1.0 + delta) > SEPARATION


def compare_traces(gpu_trace, oracle_trace, delta):
    """Walk the two decision logs in order.  They must agree on every
    decision up to the first one where they differ, and that decision must be
    unseparated in the oracle's log (a genuine near-tie).  Returns
    (number of decisions compared, index of the first divergence or None)."""
    n = min(len(gpu_trace), len(oracle_trace))
    for idx in range(n):
        o = oracle_trace[idx]
        g = gpu_trace[idx]
        hs, kind, i, j = o[0], o[1], o[2], o[3]
        if kind in (O.GEPP, O.SWAP):
            same = (int(g[0]), int(g[1]), int(g[2]), int(g[3])) == (hs, kind, i, j)
        else:
            same = (int(g[0]), int(g[1])) == (hs, kind)
        if not same:
            assert not separated(o, delta), (
                f"decision {idx} differs although separated: oracle {o}, gpu {tuple(g)}")
            return idx, idx
    assert len(gpu_trace) == len(oracle_trace), (
        f"logs agree on {n} decisions but have lengths {len(gpu_trace)} vs {len(oracle_trace)}")
    return n, None


def rel_fro_error(A64, C, U, R):
    """||A - C U R||_F / ||A||_F in FP64 from the returned factors."""
    E = A64 - (np.asarray(C, np.float64) @ U) @ np.asarray(R, np.float64)
    return float(np.linalg.norm(E) / np.linalg.norm(A64))


def sampled_error(src64, C, U, R, rows, cols):
    return O.sampled_residual(src64, np.asarray(C, np.float64), U, np.asarray(R, np.float64),
                              rows, cols)["rel"]


def error_ok(err_gpu, err_oracle):
    """Within 1.05x of the FP64 oracle's error, or 1e-5 absolute."""
    return err_gpu <= max(1.05 * err_oracle, 1e-5)


class SubSource:
    """The block M[row0 : row0 + m, col0 : col0 + n] of an oracle source."""

    def __init__(self, src, row0, m, col0, n):
        self.src, self.row0, self.col0, self.m, self.n = src, int(row0), int(col0), int(m), int(n)

    def block(self, rows, cols):
        return self.src.block(self.row0 + np.asarray(rows), self.col0 + np.asarray(cols))


# Unit roundoff of the device's double-float arithmetic (an FP32 pair keeps
# about 48 significant bits).
U_DD = 2.0 ** -48


def check_nucleus(U_dev, sigma_dev, k_dev, X32, k, tau=GPU_TAU, sigma_rel=0.0):
    """The device's nucleus against the oracle's for the same cross: X32 holds
    the FP32 entries of M[I, J] at the device's own (I, J) (input-matched), so
    the only difference is the SVD's arithmetic (double-float on the device,
    FP64 here).  Backward-stable SVDs give |d sigma_j| <= c u sigma_1, and the
    truncated pseudo-inverse moves by at most about c u kappa_k |U| with
    kappa_k = sigma_1 / sigma_k; c = 64 l covers the l-term sums and the
    Jacobi sweeps.  sigma_rel: extra relative rounding of a sigma stored in
    lower precision (2^-24 for FP32 storage).  Returns (max |dU| / max |U|,
    bound)."""
    X = np.asarray(X32, np.float64)
    l = X.shape[0]
    U_ref, k_ref, s_ref = O.nucleus(X, k, tau)
    s_dev = np.asarray(sigma_dev, np.float64)[:l]
    c = 64.0 * l
    assert np.all(np.abs(s_dev - s_ref) <= c * U_DD * s_ref[0] + sigma_rel * s_ref), (s_dev, s_ref)
    # the kept rank: equal unless a singular value sits at the cut
    near_cut = np.any(np.abs(s_ref - tau * s_ref[0]) <= 1e-9 * s_ref[0])
    if not near_cut:
        assert k_dev == k_ref, (k_dev, k_ref)
    if k_dev != k_ref:
        return None, None
    kappa = s_ref[0] / s_ref[k_ref - 1] if k_ref > 0 else 1.0
    scale = float(np.abs(U_ref).max())
    bound = c * U_DD * kappa
    err = float(np.abs(np.asarray(U_dev) - U_ref).max()) / scale
    assert err <= bound, (err, bound, kappa)
    return err, bound
