"""Plain FP64 CPU oracle of the range finder (Algorithm 5.1a) and of the
superfast dual least squares regression (Algorithm 3.1 with sparse
orthogonal multipliers, Section 3 "Superfast dual LSR").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this module: only ``tests/`` and ``bench.py``'s CPU legs may use it.
It shares no code with the CUDA library.

What it computes (Pan, Luan, Svadlenka, Zhao, arXiv:1611.01391):

* Algorithm 5.1 (LRA via range finder), variant (a): for an m x n matrix M,
  a target rank r and an n x l multiplier H (r <= l <= n), Y = M H; FAILURE
  when the numerical rank of Y is below r; otherwise U = the r leftmost
  columns of the orthogonal factor of a rank-revealing QR factorisation of
  Y (here Businger-Golub QR with column pivoting, Golub & Van Loan 5.4.2)
  and V = U^+ M = U^T M (U has orthonormal columns), the LRA being U V.
* Sparse multipliers (Section 8.1 and Section 3's sub-identity recipe): a
  sub-identity multiplier picks columns J of M (Y = M[:, J]); an abridged
  scaled and permuted Hadamard (ASPH) multiplier takes l columns of
  H_{n,d} P D.
* Problem 3.1 (LSR): x = argmin ||A x - b||, minimum-norm solution A^+ b.
* Algorithm 3.1 with an orthogonal multiplier F (k x m, k < m): the solution
  of the k-row problem min ||F A x - F b||.  The superfast choice
  F = sqrt(m/k) (I_k | O) P samples k rows (the scale does not change the
  argmin); an ASPH multiplier takes k rows of P D H_{m,d}.
* The accuracy measure of the paper's LSR tables (Tables lsrRandom to
  lsrcoh): the relative residual norm ||A x - b|| / min_y ||A y - b||.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg

from .ca import abridged_hadamard


class RangeFinderFailure(ValueError):
    """Algorithm 5.1, stage 1: the numerical rank of M H is below r."""


@dataclass
class RangeFinderResult:
    U: np.ndarray        # m x r, orthonormal columns
    V: np.ndarray        # r x n, U^T M
    R: np.ndarray        # r x l: the leading rows of the pivoted QR's triangular factor
    piv: np.ndarray      # column order of the pivoted QR (indices into the l columns of Y)
    nrank: int           # numerical rank of Y


def asph_columns(n, d, perm, sign, l):
    """The n x l multiplier made of the first l columns of H_{n,d} P D
    (column j is sign[j] times column perm[j] of H_{n,d})."""
    H = abridged_hadamard(n, d)[:, np.asarray(perm)[:l]]
    return H * np.asarray(sign, np.float64)[None, :l]


def asph_rows(m, d, perm, sign, k):
    """The k x m multiplier made of the first k rows of D P H_{m,d}
    (row i is sign[i] times row perm[i] of H_{m,d})."""
    F = abridged_hadamard(m, d)[np.asarray(perm)[:k], :]
    return np.asarray(sign, np.float64)[:k, None] * F


def numerical_rank(Rdiag, rank_tol):
    """Number of diagonal entries of the pivoted triangular factor above
    rank_tol times the first (the pivoted QR orders them by size)."""
    a = np.abs(np.asarray(Rdiag, np.float64))
    if a.size == 0 or a[0] == 0.0:
        return 0
    return int(np.sum(a > rank_tol * a[0]))


def range_finder(M, H, r, rank_tol=1e-12):
    """Algorithm 5.1a.  M: dense m x n array (FP64 values); H: an n x l
    multiplier, or an integer index array J (the sub-identity multiplier
    whose columns are e_J, so that Y = M[:, J])."""
    M = np.asarray(M, np.float64)
    H = np.asarray(H)
    Y = M[:, H] if H.ndim == 1 else M @ H.astype(np.float64)
    Q, R, piv = scipy.linalg.qr(Y, mode="economic", pivoting=True)
    nr = numerical_rank(np.diag(R), rank_tol)
    if nr < r:
        raise RangeFinderFailure(f"numerical rank of M H is {nr} < r = {r}")
    U = Q[:, :r]
    V = U.T @ M
    return RangeFinderResult(U=U, V=V, R=R[:r], piv=piv, nrank=nr)


def lsr_solution(A, b):
    """Problem 3.1: the minimum-norm least squares solution A^+ b."""
    return np.linalg.lstsq(np.asarray(A, np.float64), np.asarray(b, np.float64), rcond=None)[0]


def dual_lsr(A, b, F):
    """Algorithm 3.1 with the multiplier F: the solution of min ||F A x - F b||.
    F: a k x m matrix, or an integer index array (the rows the sub-identity
    multiplier (I_k | O) P keeps; its scale sqrt(m/k) does not change the
    solution)."""
    A = np.asarray(A, np.float64)
    b = np.asarray(b, np.float64)
    F = np.asarray(F)
    if F.ndim == 1:
        return lsr_solution(A[F], b[F])
    F = F.astype(np.float64)
    return lsr_solution(F @ A, F @ b)


def relative_residual(A, b, x):
    """||A x - b|| / min_y ||A y - b|| (the measure of Tables lsrRandom to lsrcoh)."""
    A = np.asarray(A, np.float64)
    b = np.asarray(b, np.float64)
    best = np.linalg.norm(A @ lsr_solution(A, b) - b)
    return float(np.linalg.norm(A @ np.asarray(x, np.float64) - b) / best)
