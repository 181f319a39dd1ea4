"""Plain FP64 CPU oracle of the cross-approximation (C-A) CUR method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA
library and takes its inputs from the seeded generators in ``workloads``.

What it computes (Pan, Luan, Svadlenka, Zhao, "Superfast Low-Rank
Approximation and Least Squares Regression", arXiv:1611.01391):

* Section 6.5, Primitive Algorithm: given row and column index sets I, J of an
  m x n matrix M, the CUR generator is M[I, J]; its rank-k truncation is
  inverted (pseudo-inverse) into the nucleus U and the approximation is C U R
  with C = M[:, J], R = M[I, :].
* Section 6.5, C-A iterations (dual form of Remark rec-atnsr, starting with a
  vertical step): alternately fix a vertical strip M[:, J] and choose I inside
  it, then fix the horizontal strip M[I, :] and choose J inside it.  One sweep
  is one vertical plus one horizontal step (Section 12.2, Tests 2 and 4).
* The generator inside a strip is a square l x l submatrix of locally maximal
  volume (Section 12.2; the volume footnote of Section 6.5).  The sub-algorithm
  used here is square maxvol: start from the rows chosen by Gaussian
  elimination with partial pivoting on the very first strip, later from the
  previous index set; repeatedly swap in the entry of largest modulus of
  B = S X^{-1} while it exceeds 1 + delta.  Each swap of row i into position
  j multiplies |det X| by |B_ij| (a rank-one update of X), so volume grows
  monotonically and the loop terminates.
* Appendix F: a posteriori error estimate on a random q x s submatrix of the
  error matrix, with the observed mean and variance of its entries.

Readings where the paper is silent (documented with the design):
  |I| = |J| = l (square cross), truncation rank k <= l; delta = 1e-2 and a cap
  of 64 l swaps per half-step; exact ties go to the smaller row, then the
  smaller column; the nucleus keeps singular values > rank_tol * sigma_1,
  by default rank_tol = 1e-12 (entries in FP64); a caller comparing with a
  solver that gathers FP32 entries passes that solver's rank_tol (1e-6).

Entries are promoted to FP64 before any arithmetic.  Two source precisions
exist: ``fp64`` evaluates generator entries in FP64 (the error reference) and
``fp32`` evaluates them with FP32 operations in a fixed order (the entries a
FP32 gather sees, for pivot-by-pivot comparison).

Every decision is logged as (half_step, kind, i, j, v1, v2): v1 is the
winning |value| and v2 the runner-up (GEPP, SWAP), or v1 the final max |B|
(STOP, CAP).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GEPP, SWAP, STOP, CAP = 0, 1, 2, 3


class OracleSingular(RuntimeError):
    """The strip has no nonsingular l x l submatrix reachable by GEPP."""


# ---------------------------------------------------------------------------
# Sources: entry access to M (Section 1.1: the matrix is reachable entry by
# entry; a superfast method touches O((m + n) l) of its entries).
# ---------------------------------------------------------------------------

class Dense:
    """Stored matrix; entries are the stored values promoted to FP64."""

    def __init__(self, a):
        self.a = np.asarray(a)
        self.m, self.n = self.a.shape

    def block(self, rows, cols):
        return self.a[np.ix_(np.asarray(rows), np.asarray(cols))].astype(np.float64)


class _Points:
    def __init__(self, x, y, precision="fp64"):
        self.x = np.asarray(x, dtype=np.float32)
        self.y = np.asarray(y, dtype=np.float32)
        if self.x.ndim == 1:
            self.x = self.x[:, None]
            self.y = self.y[:, None]
        self.m, self.n = self.x.shape[0], self.y.shape[0]
        if precision not in ("fp32", "fp64"):
            raise ValueError(precision)
        self.precision = precision

    def _dist2(self, xs, ys):
        # |x - y|^2 summed coordinate by coordinate, left to right, one
        # rounding per operation in the chosen precision.
        acc = None
        for c in range(xs.shape[-1]):
            d = xs[..., c] - ys[..., c]
            sq = d * d
            acc = sq if acc is None else acc + sq
        return acc

    def _pair(self, rows, cols):
        xs = self.x[np.asarray(rows)][:, None, :]
        ys = self.y[np.asarray(cols)][None, :, :]
        if self.precision == "fp64":
            xs = xs.astype(np.float64)
            ys = ys.astype(np.float64)
        return xs, ys


class Cauchy(_Points):
    """a_ij = 1 / (x_i - y_j) on 1-D points."""

    def block(self, rows, cols):
        xs, ys = self._pair(rows, cols)
        d = xs[..., 0] - ys[..., 0]
        one = np.float32(1.0) if self.precision == "fp32" else 1.0
        return (one / d).astype(np.float64)


class Gauss(_Points):
    """a_ij = exp(-|x_i - y_j|^2 / h^2) on dim-D points."""

    def __init__(self, x, y, h, precision="fp64"):
        super().__init__(x, y, precision)
        self.h = h

    def block(self, rows, cols):
        xs, ys = self._pair(rows, cols)
        d2 = self._dist2(xs, ys)
        if self.precision == "fp32":
            h2 = np.float32(self.h) * np.float32(self.h)
            return np.exp(-(d2 / h2)).astype(np.float64)
        h2 = float(np.float32(self.h)) ** 2
        return np.exp(-(d2 / h2))


class InvDist(_Points):
    """a_ij = 1 / |x_i - y_j| on dim-D points."""

    def block(self, rows, cols):
        xs, ys = self._pair(rows, cols)
        d2 = self._dist2(xs, ys)
        one = np.float32(1.0) if self.precision == "fp32" else 1.0
        return (one / np.sqrt(d2)).astype(np.float64)


def columns(src, J):
    return src.block(np.arange(src.m), J)


def rows(src, I):
    return src.block(I, np.arange(src.n))


# ---------------------------------------------------------------------------
# Row selection inside a strip
# ---------------------------------------------------------------------------

def _runner_up(values, winner):
    """Largest entry of ``values`` other than position ``winner`` (0 if none)."""
    if values.size < 2:
        return 0.0
    rest = np.delete(values, winner)
    return float(rest.max())


def gepp_rows(S, trace=None, half_step=0, pivots=None, first=()):
    """Pivot rows of Gaussian elimination with partial pivoting on the N x l
    strip S: at step t take the free row of largest |entry| in column t of
    the Schur complement (smallest row on ties), then eliminate column t from
    the later columns of the free rows.  For the first len(first) steps only
    the rows listed in ``first`` are candidates (a previous index set kept
    and completed).  Returns the l pivot rows in order."""
    W = np.array(S, dtype=np.float64, copy=True)
    N, l = W.shape
    if N < l:
        raise ValueError("strip has fewer rows than columns")
    free = np.ones(N, dtype=bool)
    keep = np.zeros(N, dtype=bool)
    keep[list(first)] = True
    piv = []
    for t in range(l):
        cand = free & keep if t < len(first) else free
        mag = np.where(cand, np.abs(W[:, t]), -1.0)
        p = int(np.argmax(mag))
        v1 = float(mag[p])
        if trace is not None:
            v2 = max(_runner_up(mag, p), 0.0)
            trace.append((half_step, GEPP, p, t, v1, v2))
        if not v1 > 0.0:
            raise OracleSingular(f"zero pivot in column {t}")
        if pivots is not None:
            pivots.append(v1)
        piv.append(p)
        free[p] = False
        mult = W[free, t] / W[p, t]
        W[np.ix_(free, np.arange(t + 1, l))] -= np.outer(mult, W[p, t + 1:])
    return piv


@dataclass
class MaxvolResult:
    I: list
    swaps: int
    converged: bool
    max_b: float


def maxvol(S, I0, delta=1e-2, max_swaps=None, trace=None, half_step=0):
    """Square maxvol on the N x l strip S from initial row positions I0.

    B = S X^{-1} with X = S[I, :] (LU with partial pivoting through
    ``numpy.linalg.solve``).  While max |B_ij| > 1 + delta: put row i in
    position j of I and apply the rank-one update
        B <- B - B[:, j] (B[i, :] - e_j^T) / B_ij,
    which is B recomputed for the new X.  Ties in the argmax go to the
    smallest row, then the smallest column (row-major first maximum)."""
    S = np.asarray(S, dtype=np.float64)
    N, l = S.shape
    if max_swaps is None:
        max_swaps = 64 * l
    I = [int(i) for i in I0]
    X = S[I, :]
    B = np.linalg.solve(X.T, S.T).T
    swaps = 0
    while True:
        mag = np.abs(B).ravel()
        p = int(np.argmax(mag))
        v1 = float(mag[p])
        i, j = divmod(p, l)
        if v1 <= 1.0 + delta:
            if trace is not None:
                trace.append((half_step, STOP, i, j, v1, 0.0))
            return MaxvolResult(I, swaps, True, v1)
        if swaps >= max_swaps:
            if trace is not None:
                trace.append((half_step, CAP, i, j, v1, 0.0))
            return MaxvolResult(I, swaps, False, v1)
        if trace is not None:
            trace.append((half_step, SWAP, i, j, v1, _runner_up(mag, p)))
        pivot = B[i, j]
        r = B[i, :].copy()
        r[j] -= 1.0
        B = B - np.outer(B[:, j], r) / pivot
        B[i, :] = 0.0          # B[I, :] is the identity for the new X
        B[i, j] = 1.0
        I[j] = i
        swaps += 1


# ---------------------------------------------------------------------------
# Nucleus (Primitive Algorithm, stages 2-3) and error estimates
# ---------------------------------------------------------------------------

def nucleus(X, k, rank_tol=1e-12):
    """U = (X_k)^+ for the l x l CUR generator X: SVD X = P diag(sigma) Q^T,
    keep the k_eff = min(k, #{sigma_j > rank_tol sigma_1}) leading triplets,
    U = Q_k diag(1/sigma_k) P_k^T.  Returns (U, k_eff, sigma)."""
    X = np.asarray(X, dtype=np.float64)
    P, sigma, QT = np.linalg.svd(X)
    if not sigma[0] > 0.0:
        return np.zeros((X.shape[1], X.shape[0])), 0, sigma
    k_eff = int(min(k, np.count_nonzero(sigma > rank_tol * sigma[0])))
    U = (QT[:k_eff].T / sigma[:k_eff]) @ P[:, :k_eff].T
    return U, k_eff, sigma


def sampled_residual(src, C, U, R, sample_rows, sample_cols):
    """Appendix F: error matrix E = M - C U R restricted to the q x s
    submatrix (sample_rows, sample_cols).  Returns the relative Frobenius
    estimate sqrt(sum E^2 / sum M^2), the sums, and the observed mean
    mu_K = (1/K) sum E and variance sigma_K^2 = (1/K) sum (E - mu_K)^2."""
    sr = np.asarray(sample_rows)
    sc = np.asarray(sample_cols)
    A = src.block(sr, sc)
    E = A - (np.asarray(C)[sr] @ U) @ np.asarray(R)[:, sc]
    K = E.size
    sse = float(np.sum(E * E))
    ssa = float(np.sum(A * A))
    mu = float(np.sum(E)) / K
    var = float(np.sum((E - mu) ** 2)) / K
    rel = math.sqrt(sse / ssa) if ssa > 0 else math.inf
    return {"rel": rel, "sse": sse, "ssa": ssa, "mu": mu, "var": var, "K": K}


def full_residual(src, C, U, R, row_block=2048):
    """||M - C U R||_F / ||M||_F over all entries, in FP64 row blocks."""
    CU = np.asarray(C, dtype=np.float64) @ U
    R = np.asarray(R, dtype=np.float64)
    sse = 0.0
    ssa = 0.0
    cols = np.arange(src.n)
    for r0 in range(0, src.m, row_block):
        rr = np.arange(r0, min(src.m, r0 + row_block))
        A = src.block(rr, cols)
        E = A - CU[rr] @ R
        sse += float(np.sum(E * E))
        ssa += float(np.sum(A * A))
    return math.sqrt(sse / ssa), sse, ssa


# ---------------------------------------------------------------------------
# The C-A driver
# ---------------------------------------------------------------------------

@dataclass
class CrossResult:
    I: list
    J: list
    C: np.ndarray
    U: np.ndarray
    R: np.ndarray
    k_eff: int
    sigma: np.ndarray
    sweeps_done: int
    swaps: list = field(default_factory=list)
    converged: bool = True
    trace: list = field(default_factory=list)
    history: list = field(default_factory=list)
    estimate: dict | None = None


def cross_approximation(src, J0, k, sweeps, delta=1e-2, rank_tol=1e-12,
                        max_swaps=None, tol=0.0, sample_rows=None,
                        sample_cols=None, keep_trace=True, I0=None):
    """C-A iterations from the initial column set J0 (|J0| = l).

    Sweep s: C = M[:, J]; on the first sweep I = GEPP rows of C (or, when a
    row set I0 is given, I = I0: the iteration resumes from a previous
    (I, J), each step starting from the previous index set); I = maxvol of C
    from I; R = M[I, :]; J = maxvol of R^T from J.  After ``sweeps`` sweeps
    (or once the sampled estimate of the current CUR is <= tol, step 6 of
    the C-A iterations), C = M[:, J], R = M[I, :], U = (M[I, J]_k)^+."""
    J = [int(j) for j in J0]
    l = len(J)
    if not (1 <= k <= l):
        raise ValueError("need 1 <= k <= l")
    trace = [] if keep_trace else None
    swaps = []
    history = []
    converged = True
    I = None if I0 is None else [int(i) for i in I0]
    done = 0
    estimate = None
    for s in range(sweeps):
        C = columns(src, J)
        if s == 0 and I is None:
            I = gepp_rows(C, trace, half_step=2 * s)
        res = maxvol(C, I, delta, max_swaps, trace, half_step=2 * s)
        I = res.I
        swaps.append(res.swaps)
        converged &= res.converged
        R = rows(src, I)
        res = maxvol(R.T, J, delta, max_swaps, trace, half_step=2 * s + 1)
        J = res.I
        swaps.append(res.swaps)
        converged &= res.converged
        done = s + 1
        history.append((list(I), list(J)))
        if tol > 0.0 and sample_rows is not None:
            Cf = columns(src, J)
            U, _, _ = nucleus(src.block(I, J), k, rank_tol)
            estimate = sampled_residual(src, Cf, U, R, sample_rows, sample_cols)
            if estimate["rel"] <= tol:
                break
    C = columns(src, J)
    R = rows(src, I)
    U, k_eff, sigma = nucleus(src.block(I, J), k, rank_tol)
    if sample_rows is not None:
        estimate = sampled_residual(src, C, U, R, sample_rows, sample_cols)
    return CrossResult(I=I, J=J, C=C, U=U, R=R, k_eff=k_eff, sigma=sigma,
                       sweeps_done=done, swaps=swaps, converged=converged,
                       trace=trace if trace is not None else [],
                       history=history, estimate=estimate)


def cross_approximation_adaptive(src, J_cands, l_init, l_max, k_max, sweeps, tol,
                                 delta=1e-2, max_swaps=None, sample_rows=None,
                                 sample_cols=None, trace=None):
    """Rank-adaptive C-A for blocks whose rank is not known in advance (the
    far-field blocks of Section 9; the paper's HSS test finds the rank by a
    search, this is the growth rule read for it).

    The cross starts at l = l_init with the first candidate columns.  Each
    sweep is a vertical step (I = maxvol of M[:, J]) and a horizontal step
    (J = maxvol of M[I, :]^T).  Every strip starts from the previous index
    set: Gaussian elimination with partial pivoting whose pivots are
    restricted to that set (so B = S X^{-1} for the previous rows, with
    position t holding the pivot row of step t); the very first strip, and
    the rows a grown cross lacks, pivot freely.  After every sweep,
    k = #{sigma_j(M[I, J]) > tol sigma_1}:
      * k = l < k_max and l < l_max: the cross grows to min(l_max, 2 l) with
        the next unused candidate columns appended to J;
      * otherwise U = (M[I, J]_k)^+ with k_eff = min(k_max, k), and the
        iteration stops once k >= k_max, ``sweeps`` sweeps were made at this
        size, or the Appendix F estimate on (sample_rows, sample_cols), when
        given, is <= tol.

    With ``trace`` (a list), every decision is appended as (half_step, kind,
    i, j, v1, v2) with half-steps counted from 0 over the whole block.

    Returns (I, J, U, k_eff, sigma, l, swaps)."""
    J_cands = [int(j) for j in J_cands]
    l_cap = min(l_max, src.m, src.n)          # a cross cannot exceed the block
    J = J_cands[:min(l_init, l_cap)]
    l = len(J)
    I = []
    swaps = 0
    at_size = 0
    hs = 0
    while True:
        C = columns(src, J)
        start = gepp_rows(C, trace, hs, first=I)
        res = maxvol(C, start, delta, max_swaps, trace, hs)
        I = res.I
        swaps += res.swaps
        hs += 1
        RT = rows(src, I).T
        start = gepp_rows(RT, trace, hs, first=J)
        res = maxvol(RT, start, delta, max_swaps, trace, hs)
        J = res.I
        swaps += res.swaps
        hs += 1
        at_size += 1
        X = src.block(I, J)
        sigma = np.linalg.svd(X, compute_uv=False)
        k = int(np.count_nonzero(sigma > tol * sigma[0])) if sigma[0] > 0.0 else 0
        if k == l and k < k_max and l < l_cap:
            extra = [j for j in J_cands if j not in J][: min(l_cap, 2 * l) - l]
            if extra:
                J = J + extra
                l = len(J)
                at_size = 0
                continue
        U, k_eff, sigma = nucleus(X, k_max, tol)
        if k >= k_max or at_size >= sweeps:
            break
        if sample_rows is not None:
            est = sampled_residual(src, columns(src, J), U, rows(src, I), sample_rows, sample_cols)
            if est["rel"] <= tol:
                break
    return I, J, U, k_eff, sigma, l, swaps


# ---------------------------------------------------------------------------
# Cynical algorithms (Section 6.5) in the forms of Section 12.2, Tests 3 and 4
# ---------------------------------------------------------------------------

class _Sub:
    """The submatrix M[K, L] of a source, as a source of its own."""

    def __init__(self, src, K, L):
        self.src, self.K, self.L = src, np.asarray(K), np.asarray(L)
        self.m, self.n = len(self.K), len(self.L)

    def block(self, rows, cols):
        return self.src.block(self.K[np.asarray(rows)], self.L[np.asarray(cols)])


@dataclass
class CynicalResult:
    I: list
    J: list
    U: np.ndarray
    K: list
    L: list
    inner: CrossResult
    outer: CrossResult | None = None


def cynical(src, K, L, r, inner_sweeps=2, delta=1e-2, rank_tol=1e-12, max_swaps=None):
    """Tests 3 of Section 12.2, the Cynical algorithm of Section 6.5 with
    p x q = |K| x |L|: an r x r CUR generator of the submatrix M[K, L] with
    locally maximal volume, computed by C-A iterations inside that
    submatrix (maxvol over its rows, then over its columns, alternately,
    from its first r columns; the first vertical step starts from Gaussian
    elimination), is taken as the generator of M: I = K[I'], J = L[J'] and
    U = (M[I, J]_r)^+ (the inverse for a nonsingular generator, as in
    Tests 1).  Returns a CynicalResult."""
    K = [int(k) for k in K]
    L = [int(j) for j in L]
    if not (1 <= r <= min(len(K), len(L))):
        raise ValueError("need 1 <= r <= min(|K|, |L|)")
    sub = _Sub(src, K, L)
    inner = cross_approximation(sub, list(range(r)), k=r, sweeps=inner_sweeps, delta=delta,
                                rank_tol=rank_tol, max_swaps=max_swaps)
    I = [K[i] for i in inner.I]
    J = [L[j] for j in inner.J]
    return CynicalResult(I=I, J=J, U=inner.U, K=K, L=L, inner=inner)


def ca_cynical(src, L0, r, outer_loops=1, inner_sweeps=2, delta=1e-2, rank_tol=1e-12,
               max_swaps=None):
    """Tests 4 of Section 12.2: from the column set L0 (|L0| = q, 4 r in the
    paper) C-A loops with q x q generators (a vertical step: K' of locally
    maximal volume in M[:, L0]; a horizontal step: L' of locally maximal
    volume in M[K', :]), then Tests 3 on M[K', L'].  Returns a
    CynicalResult with the outer C-A run attached."""
    q = len(L0)
    outer = cross_approximation(src, L0, k=q, sweeps=outer_loops, delta=delta,
                                rank_tol=rank_tol, max_swaps=max_swaps)
    res = cynical(src, outer.I, outer.J, r, inner_sweeps, delta, rank_tol, max_swaps)
    res.outer = outer
    return res


# ---------------------------------------------------------------------------
# Refinement of a C-A CUR by leverage-score sampling (Section 7.2 and Remark
# resnrg: a crude LRA from C-A iterations, refined by the sampling of
# Algorithm 7.1; Appendix C, Algorithm C.1; Appendix D, Algorithm D.1)
# ---------------------------------------------------------------------------

def top_svd_of_cur(C, U, R, r):
    """Algorithm D.1 (Appendix D) for M ~ A W B with A = C, W = U, B = R:
    QR factorizations C = Q_c R_c and R^T = Q_r R_r, the SVD of the small
    core R_c U R_r^T = A S B^T, and the top-r triplets S = Q_c A_r,
    T = Q_r B_r.  Returns (S, sigma_r, T) with S m x r, T n x r."""
    C = np.asarray(C, np.float64)
    R = np.asarray(R, np.float64)
    Qc, Rc = np.linalg.qr(C)
    Qr, Rr = np.linalg.qr(R.T)
    A, sig, BT = np.linalg.svd(Rc @ np.asarray(U, np.float64) @ Rr.T)
    return Qc @ A[:, :r], sig[:r], Qr @ BT[:r].T


def sampling_scores(V):
    """Appendix C, eq. (smpl): for the rows v_i of V, p_i = v_i^T v_i / ||V||_F^2.
    With V the top-r singular vectors of a matrix (orthonormal columns) these
    are its SVD-based leverage scores with beta = 1, ||v_i||^2 / r (eq. levsc1)."""
    V = np.asarray(V, np.float64)
    w = np.sum(V * V, axis=1)
    return w / np.sum(w)


def exactly_sample(p, l, u):
    """Algorithm C.1 (Exactly(l) sampling and re-scaling) with its random
    choices given: draw t picks i_t, the smallest i whose cumulative score
    sum_{j <= i} p_j exceeds u_t (u_t uniform on [0, 1)), so that
    Probability(i_t = i) = p_i; the re-scaling is d_t = 1 / sqrt(l p_{i_t}).
    Returns (indices i_t, d_t)."""
    p = np.asarray(p, np.float64)
    cdf = np.cumsum(p)
    idx = []
    for t in range(l):
        i = int(np.searchsorted(cdf, u[t], side="right"))
        idx.append(min(i, len(p) - 1))
    idx = np.asarray(idx)
    return idx, 1.0 / np.sqrt(l * p[idx])


@dataclass
class RefineResult:
    cols: np.ndarray       # l sampled columns (with repeats)
    d: np.ndarray          # their re-scaling
    rows: np.ndarray       # k sampled rows
    dbar: np.ndarray       # their re-scaling
    U: np.ndarray          # l x k nucleus: C' U R' ~ M with C' = M[:, cols], R' = M[rows, :]
    p_cols: np.ndarray     # column scores (n)
    p_rows: np.ndarray     # row scores (m)
    sigma: np.ndarray      # top-r singular values of the C-A approximation


def refine_by_leverage(src, I, J, U, r, l, k, u_cols, u_rows, rank_tol=1e-12):
    """Section 7.2: take the C-A approximation M' = C U R (C = M[:, J],
    R = M[I, :]), compute its top-r SVD S Sigma T^T superfast (Algorithm
    D.1), the leverage scores with beta = 1 of its columns (rows of T) and
    of its rows (rows of S), and run Algorithm 7.1 with them: Exactly(l)
    columns and Exactly(k) rows (Algorithm C.1, random choices given as
    u_cols, u_rows), C' = M S_cols, R' = S_rows^T M, and the nucleus
    U' = D (Mk_r)^+ Dbar for Mk = Dbar M[rows, cols] D, truncated at rank r
    (the Primitive Algorithm's rank-r truncation of the generator)."""
    C = columns(src, J)
    R = rows(src, I)
    S, sig, T = top_svd_of_cur(C, U, R, r)
    p_cols = sampling_scores(T)
    p_rows = sampling_scores(S)
    cols, d = exactly_sample(p_cols, l, u_cols)
    rws, dbar = exactly_sample(p_rows, k, u_rows)
    Mk = dbar[:, None] * src.block(rws, cols) * d[None, :]
    Mp, _, _ = nucleus(Mk, r, rank_tol)
    Unew = d[:, None] * Mp * dbar[None, :]
    return RefineResult(cols=cols, d=d, rows=rws, dbar=dbar, U=Unew, p_cols=p_cols, p_rows=p_rows, sigma=sig)


# ---------------------------------------------------------------------------
# Pre-processing with abridged Hadamard multipliers (Section 8.1, family (i);
# recovery of an LRA with nonsingular multipliers, Section 6.6)
# ---------------------------------------------------------------------------

def abridged_hadamard(n, d):
    """The d-abridged Hadamard matrix H_{n,d}: the recursion
    H_{2s} = [[H_s, H_s], [H_s, -H_s]] run d times from H_{s0} = I_{s0},
    n = 2^d s0 (Section 8.1).  Dense, for small n."""
    if n % (1 << d):
        raise ValueError("2^d must divide n")
    H = np.eye(n >> d)
    for _ in range(d):
        H = np.block([[H, H], [H, -H]])
    return H


def aph_left(m, d, perm, sign):
    """Left multiplier F = D P H_{m,d} (rows permuted, then scaled by +-1):
    row i of F is sign[i] times row perm[i] of H_{m,d}."""
    return np.asarray(sign, np.float64)[:, None] * abridged_hadamard(m, d)[np.asarray(perm)]


def aph_right(n, d, perm, sign):
    """Right multiplier H = H_{n,d} P D: column j of H is sign[j] times
    column perm[j] of H_{n,d}."""
    return abridged_hadamard(n, d)[:, np.asarray(perm)] * np.asarray(sign, np.float64)[None, :]


def butterfly(vals, b, d):
    """Entry b of H_{2^d} applied along axis 0 of vals (indexed by the block
    p of the H_{n,d} recursion), summed in the order of the d recursive
    steps H_{2s} = [[H_s, H_s], [H_s, -H_s]] (Section 8.1; the order of
    the fast multiplication with at most 2dn additions): the innermost
    step combines the entries p that differ in bit 0, the next those that
    differ in bit 1, and so on; a step whose bit of b is 1 subtracts the
    second half.  b may be an array broadcast over the trailing axes.  The
    arithmetic is that of vals (float32 or float64), every step rounded."""
    vals = np.asarray(vals)
    if vals.dtype != np.float32:
        vals = vals.astype(np.float64)
    for k in range(d):
        sig = np.where((np.asarray(b) >> k) & 1, -1.0, 1.0).astype(vals.dtype)
        vals = vals[0::2] + sig * vals[1::2]
    return vals[0]


class Preprocessed:
    """The source M_bar = F M H for the multipliers of aph_left / aph_right,
    evaluated entry by entry from the 4^d entries of M each one combines:
    with x = pr[i] = b_i s_m + o_i and y = pc[j] = b_j s_n + o_j,
    M_bar[i, j] = sF[i] sH[j] sum_q (+-1) sum_p (+-1) M[p s_m + o_i, q s_n + o_j]:
    F applied first (the inner sums over p), then H (the outer sum over q),
    each in the order of the recursive steps (butterfly).  Precision "fp64":
    FP64 arithmetic on the entries of M; "fp32": the entries of M rounded to
    FP32 and every step of the butterfly rounded to FP32 (the fast product
    carried out in the arithmetic of an FP32 stored matrix)."""

    def __init__(self, src, d, perm_rows, sign_rows, perm_cols, sign_cols, precision="fp64"):
        self.src, self.d = src, int(d)
        self.m, self.n = src.m, src.n
        self.sm, self.sn = self.m >> d, self.n >> d
        if (self.sm << d) != self.m or (self.sn << d) != self.n:
            raise ValueError("2^d must divide m and n")
        self.pr, self.sr = np.asarray(perm_rows), np.asarray(sign_rows, np.float64)
        self.pc, self.sc = np.asarray(perm_cols), np.asarray(sign_cols, np.float64)
        self.precision = precision

    def block(self, rows, cols):
        rows, cols = np.asarray(rows), np.asarray(cols)
        D = 1 << self.d
        bc, oc = np.divmod(self.pc[cols], self.sn)
        ci = np.arange(D)[:, None] * self.sn + oc[None, :]          # D x len(cols): q s_n + o_j
        out = np.zeros((len(rows), len(cols)))
        dt = np.float32 if self.precision == "fp32" else np.float64
        for a, i in enumerate(rows):
            br, orow = divmod(int(self.pr[i]), self.sm)
            X = np.stack([self.src.block([p * self.sm + orow], ci.ravel()).reshape(ci.shape)
                          for p in range(D)]).astype(dt)            # X[p, q, c]
            inner = butterfly(X, br, self.d)                         # (F M)[., q s_n + o_j]
            out[a] = self.sr[i] * self.sc[cols] * butterfly(inner, bc, self.d).astype(np.float64)
        return out


def recover_lra(pre, Cbar, Rbar):
    """Section 6.6: from an LRA Cbar Ubar Rbar of M_bar = F M H with
    F F^T = 2^d I and H^T H = 2^d I, the induced LRA of M is
    (F^T Cbar / 2^d) Ubar (Rbar H^T / 2^d).  Returns (A, B), A = F^T Cbar / 2^d
    (m x l) and B = Rbar H^T / 2^d (l x n).  With H_{m,d} symmetric,
    F^T Cbar = H_{m,d} Y for Y[pr[i]] = sr[i] Cbar[i], and Rbar H^T = Z H_{n,d}
    for Z[:, pc[j]] = sc[j] Rbar[:, j]; both products in the butterfly order."""
    Cbar = np.asarray(Cbar, np.float64)
    Rbar = np.asarray(Rbar, np.float64)
    m, n, d = pre.m, pre.n, pre.d
    D, l = 1 << d, Cbar.shape[1]
    Y = np.empty_like(Cbar)
    Y[pre.pr] = pre.sr[:, None] * Cbar
    Y3 = Y.reshape(D, pre.sm, l)                                  # Y3[p, o] = Y[p s_m + o]
    A = np.stack([butterfly(Y3, b, d) for b in range(D)]).reshape(m, l) / D
    Z = np.empty_like(Rbar)
    Z[:, pre.pc] = Rbar * pre.sc[None, :]
    Z3 = Z.reshape(Rbar.shape[0], D, pre.sn).transpose(1, 0, 2)   # Z3[q, t, o] = Z[t, q s_n + o]
    B = np.stack([butterfly(Z3, b, d) for b in range(D)], axis=1).reshape(Rbar.shape[0], n) / D
    return A, B


# ---------------------------------------------------------------------------
# Initial column set from a seed (Section 12.2: the tests start from random
# columns), for callers that pass a seed instead of the columns
# ---------------------------------------------------------------------------

_MASK64 = (1 << 64) - 1


def splitmix64(state):
    """One step of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): returns
    (new state, output).  The state advances by the odd constant
    0x9E3779B97F4A7C15 (the 64-bit golden ratio); the output is the new state
    passed through two xor-shift-multiply rounds and a final xor-shift."""
    state = (state + 0x9E3779B97F4A7C15) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return state, z ^ (z >> 31)


def draw_columns(seed, n, l):
    """l distinct values of range(n) by Floyd's sampling algorithm (Bentley
    and Floyd, CACM 1987): for c = n - l, ..., n - 1 draw t uniform on
    [0, c] (here: the next SplitMix64 output mod (c + 1)) and take t, or c
    when t was already taken.  Returned in the order taken."""
    state = int(seed) & _MASK64
    taken = []
    seen = set()
    for c in range(n - l, n):
        state, r = splitmix64(state)
        t = r % (c + 1)
        v = c if t in seen else t
        seen.add(v)
        taken.append(v)
    return taken


def random_cross(src, I, J, k=None, rank_tol=0.0):
    """Section 12.2, Tests 1: CUR with given (random) I, J and U = W[I, J]^{-1}
    (k = l), or its rank-k truncated pseudo-inverse."""
    X = src.block(I, J)
    k = len(J) if k is None else k
    U, k_eff, sigma = nucleus(X, k, rank_tol)
    return columns(src, J), U, rows(src, I)
