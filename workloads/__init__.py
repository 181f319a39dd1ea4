"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and lays them out; it contains none of
the cross-approximation arithmetic.  Both the CPU oracle (``oracle/``) and the
GPU path (``paper_1611_01391_gb300``) consume what it produces, and neither one
is imported here.

Every generator takes an explicit integer seed and uses numpy's PCG64, whose
output stream is platform independent, so x86 and Arm hosts produce identical
bytes for identical seeds.

Workload families (sizes as in the named configurations):

* ``lowrank_svd``      -- A = U diag(s) V^T + E with Haar-orthogonal U, V
  (QR of a Gaussian matrix with the sign of diag(R) fixed positive), s_i = 1
  for i < r, E i.i.d. N(0, noise_std^2).  256 x 256, r = 8, noise variance
  1e-8 is the small dense FP64 case.  Inputs generated from an SVD follow the
  paper's tests of Section 11.1.
* ``factor_gaussian``  -- A = G1 G2^T / sqrt(r) + noise_std * N(0, 1), the
  perturbed factor-Gaussian family of Section 12.3 (stored FP32, 32768^2,
  r = 64, noise 1e-4 for the large stored case).
* ``tb_ranrc``         -- W = G1 G2 + 1e-10 G3 exactly as in Section 12.3
  (Table tb_ranrc).
* ``cauchy_points``    -- x_i ~ U[0,1], y_j ~ U[2,3] in FP32; the matrix
  a_ij = 1/(x_i - y_j) is never materialised.
* ``cloud_points``     -- points uniform in the unit cube (FP32, 3-D).
* ``draw_indices``     -- l distinct indices uniform without replacement:
  the random initial column set of Section 12.2 (Tests 1/2) and the random
  q x s error sample of Appendix F.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1611_01391


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    """n x n Haar-distributed orthogonal matrix: QR of a Gaussian matrix,
    columns re-signed so that diag(R) > 0."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def lowrank_svd(seed: int, m: int = 256, n: int = 256, r: int = 8,
                noise_std: float = 1e-4) -> np.ndarray:
    """FP64 m x n matrix U[:, :r] V[:, :r]^T + E (s_i = 1 for i < r)."""
    rng = rng_for(seed)
    u = haar_orthogonal(rng, m)[:, :r]
    v = haar_orthogonal(rng, n)[:, :r]
    e = rng.standard_normal((m, n)) * noise_std
    return u @ v.T + e


def factor_gaussian(seed: int, m: int, n: int, r: int, noise_std: float,
                    dtype=np.float32, row_block: int = 4096) -> np.ndarray:
    """m x n matrix G1 G2^T / sqrt(r) + noise_std * N(0,1), built in FP64 row
    blocks and stored in ``dtype`` (row-major)."""
    rng = rng_for(seed)
    g1 = rng.standard_normal((m, r))
    g2 = rng.standard_normal((n, r))
    out = np.empty((m, n), dtype=dtype)
    scale = 1.0 / np.sqrt(r)
    for r0 in range(0, m, row_block):
        r1 = min(m, r0 + row_block)
        blk = (g1[r0:r1] @ g2.T) * scale
        blk += noise_std * rng.standard_normal((r1 - r0, n))
        out[r0:r1] = blk.astype(dtype)
    return out


def tb_ranrc(seed: int, n: int, r: int) -> np.ndarray:
    """W = G1 G2 + 1e-10 G3 with G1 n x r, G2 r x n, G3 n x n Gaussian."""
    rng = rng_for(seed)
    g1 = rng.standard_normal((n, r))
    g2 = rng.standard_normal((r, n))
    g3 = rng.standard_normal((n, n))
    return g1 @ g2 + 1e-10 * g3


def cauchy_points(seed: int, m: int, n: int):
    """x in U[0,1] (m points) and y in U[2,3] (n points), FP32."""
    rng = rng_for(seed)
    x = rng.random(m, dtype=np.float32)
    y = (rng.random(n, dtype=np.float32) + np.float32(2.0)).astype(np.float32)
    return x, y


def cloud_points(seed: int, count: int, dim: int = 3, lo: float = 0.0,
                 hi: float = 1.0) -> np.ndarray:
    """count x dim FP32 points uniform in [lo, hi)^dim (point-major)."""
    rng = rng_for(seed)
    p = rng.random((count, dim), dtype=np.float32)
    return (np.float32(lo) + np.float32(hi - lo) * p).astype(np.float32)


def draw_indices(seed: int, n: int, l: int, sort: bool = False) -> np.ndarray:
    """l distinct indices in [0, n), uniform without replacement (int32)."""
    rng = rng_for(seed)
    idx = rng.choice(n, size=l, replace=False).astype(np.int32)
    return np.sort(idx) if sort else idx


def delta_matrix(m: int, n: int, i: int, j: int) -> np.ndarray:
    """The hard input of Appendix E: zeros except a single unit entry."""
    a = np.zeros((m, n))
    a[i, j] = 1.0
    return a
