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
* ``laplacian_single_layer`` -- class (i) of the paper's test inputs
  (Section 12.4, tb_Lp / tb_fh): the discretised single-layer Laplacian
  operator between the contours C(0,1) and C(0,2), normalised to unit
  spectral norm; the inputs on which plain C-A was reported to fail and
  pre-processing was applied.
* ``hadamard_multipliers`` -- the random permutations and +-1 scalings of
  the abridged scaled and permuted Hadamard multipliers (Section 8.1).
* ``lsr_problem``      -- the four input classes of the paper's LSR tests
  (Section 12, Tables lsrRandom, lsrill, lsrsemi, lsrcoh; recipes after
  AMT10): Gaussian A; ill-conditioned A = S diag(sigma) T^T with Haar S, T,
  leading singular values 10^4, 10^3, ..., 10^-9 and the rest 10^-10;
  semi-coherent A = [G 0; 0 D] with G Gaussian (m - n/2) x n/2 and D a
  random +-1 diagonal; coherent A = [D_n; 0]; b Gaussian (FP64).
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


def morton3(ix, iy, iz, bits):
    """Interleave the bits of three integer coordinate arrays (z-order)."""
    code = np.zeros(ix.shape, dtype=np.int64)
    for b in range(bits):
        code |= ((ix >> b) & 1).astype(np.int64) << (3 * b + 2)
        code |= ((iy >> b) & 1).astype(np.int64) << (3 * b + 1)
        code |= ((iz >> b) & 1).astype(np.int64) << (3 * b)
    return code


def octree_block_pairs(seed: int, npoints: int = 1 << 20, leaf: int = 2048, n_pairs: int = 4096,
                       eta: float = 1.0, depth: int = 6, min_size: int = 64):
    """Far-field blocks of the kernel 1/|x - y| on a point cloud (the
    multipole setting of Section 9).

    Points are uniform in [0,1)^3 and sorted in z-order at ``depth`` levels,
    so every octree box owns a contiguous range of the sorted array.  A box
    is split while it holds more than ``leaf`` points.  A pair (X, Y) of
    boxes of one level is admissible when max(diam X, diam Y) <= eta
    dist(X, Y) (diam = box diagonal, dist = distance between the boxes); the
    candidate blocks are the admissible pairs whose parents are not
    admissible (the interaction lists of the adaptive tree) with between
    ``min_size`` and ``leaf`` points on each side.  ``n_pairs`` of them are drawn without
    replacement.

    Returns (points (npoints x 3, FP32, sorted), blocks (n_pairs x 4 int64:
    row0, m, col0, n as ranges of the sorted point array))."""
    rng = rng_for(seed)
    pts = rng.random((npoints, 3), dtype=np.float32)
    cells = np.minimum((pts * (1 << depth)).astype(np.int64), (1 << depth) - 1)
    code = morton3(cells[:, 0], cells[:, 1], cells[:, 2], depth)
    order = np.argsort(code, kind="stable")
    pts = pts[order]
    code = code[order]

    def box_range(level, key):
        shift = 3 * (depth - level)
        lo = key << shift
        hi = (key + 1) << shift
        return int(np.searchsorted(code, lo, "left")), int(np.searchsorted(code, hi, "left"))

    def box_geom(level, key):
        w = 1.0 / (1 << level)
        ix = iy = iz = 0
        for b in range(level):
            ix |= ((key >> (3 * b + 2)) & 1) << b
            iy |= ((key >> (3 * b + 1)) & 1) << b
            iz |= ((key >> (3 * b)) & 1) << b
        return np.array([ix, iy, iz]) * w, w

    def admissible(g1, g2):
        (c1, w1), (c2, w2) = g1, g2
        gap = np.maximum(0.0, np.maximum(c1 - (c2 + w2), c2 - (c1 + w1)))
        dist = float(np.sqrt(np.sum(gap * gap)))
        diam = float(np.sqrt(3.0)) * max(w1, w2)
        return dist > 0.0 and diam <= eta * dist

    # adaptive tree: boxes per level that exist (and are split further)
    levels = {0: [0]}
    split = {}
    for level in range(0, depth):
        split[level] = []
        for key in levels[level]:
            a, b = box_range(level, key)
            if b - a > leaf:
                split[level].append(key)
        levels[level + 1] = [(k << 3) | c for k in split[level] for c in range(8)
                             if box_range(level + 1, (k << 3) | c)[1] > box_range(level + 1, (k << 3) | c)[0]]
    cands = []
    for level in range(1, depth + 1):
        boxes = levels.get(level, [])
        geo = {k: box_geom(level, k) for k in boxes}
        rng_ = {k: box_range(level, k) for k in boxes}
        parents = {}
        for k in boxes:
            parents.setdefault(k >> 3, []).append(k)
        pkeys = sorted(parents)
        pgeo = {p: box_geom(level - 1, p) for p in pkeys}
        for i, p in enumerate(pkeys):
            for q in pkeys:
                if admissible(pgeo[p], pgeo[q]):
                    continue  # handled at the parents' level
                for x in parents[p]:
                    for y in parents[q]:
                        if x == y or not admissible(geo[x], geo[y]):
                            continue
                        (a0, a1), (b0, b1) = rng_[x], rng_[y]
                        if min_size <= a1 - a0 <= leaf and min_size <= b1 - b0 <= leaf:
                            cands.append((a0, a1 - a0, b0, b1 - b0))
    cands = np.array(cands, dtype=np.int64)
    pick = rng.choice(len(cands), size=min(n_pairs, len(cands)), replace=False)
    return pts, cands[np.sort(pick)]


def block_candidates(seed: int, blocks: np.ndarray, l_max: int, q: int):
    """Per block: l_max distinct candidate columns (initial J and the columns
    added when the cross grows) and q sample rows / q sample columns for the
    Appendix F estimate, all local to the block, drawn without replacement."""
    rng = rng_for(seed)
    nb = len(blocks)
    jc = np.zeros((nb, l_max), np.int32)
    sr = np.zeros((nb, q), np.int32)
    sc = np.zeros((nb, q), np.int32)
    for b, (r0, m, c0, n) in enumerate(blocks):
        jc[b] = rng.choice(n, size=l_max, replace=False) if n >= l_max else np.resize(rng.permutation(n), l_max)
        sr[b] = np.sort(rng.choice(m, size=q, replace=False))
        sc[b] = np.sort(rng.choice(n, size=q, replace=False))
    return jc, sr, sc


def serving_requests(seed: int, count: int, min_side: int = 256, max_side: int = 16384,
                     ks=(8, 16, 32, 64), sweeps: int = 4, sample: int = 256):
    """A stream of independent LRA requests for the served form.

    Each request: generator uniform over {Cauchy 1/(x - y) with x ~ U[0,1],
    y ~ U[2,3]; Gaussian exp(-|x - y|^2 / 0.25) on points in U[0,1]^3;
    1/|x - y| between the clusters U[0,1]^3 and U[2,3]^3}, m and n
    log-uniform in [min_side, max_side], k uniform over ``ks``,
    l = min(96, ceil(1.5 k)), a random initial column set and a
    sample x sample error sample."""
    rng = rng_for(seed)
    reqs = []
    lo, hi = np.log(min_side), np.log(max_side)
    for _ in range(count):
        kind = ("cauchy", "gauss", "invdist")[int(rng.integers(0, 3))]
        m = int(np.exp(rng.uniform(lo, hi)))
        n = int(np.exp(rng.uniform(lo, hi)))
        k = int(ks[int(rng.integers(0, len(ks)))])
        l = min(96, int(np.ceil(1.5 * k)))
        if kind == "cauchy":
            x = rng.random(m, dtype=np.float32)
            y = (rng.random(n, dtype=np.float32) + np.float32(2.0)).astype(np.float32)
            h = 0.0
        elif kind == "gauss":
            x = rng.random((m, 3), dtype=np.float32)
            y = rng.random((n, 3), dtype=np.float32)
            h = 0.5
        else:
            x = rng.random((m, 3), dtype=np.float32)
            y = (rng.random((n, 3), dtype=np.float32) + np.float32(2.0)).astype(np.float32)
            h = 0.0
        J0 = rng.choice(n, size=l, replace=False).astype(np.int32)
        q = min(sample, m)
        s = min(sample, n)
        rows = np.sort(rng.choice(m, size=q, replace=False)).astype(np.int32)
        cols = np.sort(rng.choice(n, size=s, replace=False)).astype(np.int32)
        reqs.append(dict(kind=kind, m=m, n=n, k=k, l=l, sweeps=sweeps, x=x, y=y, h=h, J0=J0,
                         rows=rows, cols=cols))
    return reqs


def poisson_arrivals(seed: int, count: int, rate: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    rng = rng_for(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def delta_matrix(m: int, n: int, i: int, j: int) -> np.ndarray:
    """The hard input of Appendix E: zeros except a single unit entry."""
    a = np.zeros((m, n))
    a[i, j] = 1.0
    return a


def laplacian_single_layer(n: int, nodes: int = 8, row_block: int = 256) -> np.ndarray:
    """n x n FP64 matrix m_ij = c * integral over the arc j of the unit
    circle (angles 2 pi j / n .. 2 pi (j + 1) / n, arc-length measure) of
    log|x_i - y|, x_i = 2 exp(2 pi sqrt(-1) i / n) on the circle of radius 2,
    with c such that the spectral norm is 1.  Each arc integral by
    Gauss-Legendre quadrature with `nodes` points (the integrand is smooth:
    |x_i - y| >= 1)."""
    t, w = np.polynomial.legendre.leggauss(nodes)
    h = 2.0 * np.pi / n
    theta = (np.arange(n)[:, None] + (t[None, :] + 1.0) / 2.0) * h       # n arcs x nodes
    y = np.exp(1j * theta)
    x = 2.0 * np.exp(2j * np.pi * np.arange(n) / n)
    out = np.empty((n, n))
    for r0 in range(0, n, row_block):
        r1 = min(n, r0 + row_block)
        out[r0:r1] = (np.log(np.abs(x[r0:r1, None, None] - y[None, :, :])) @ w) * (h / 2.0)
    return out / np.linalg.norm(out, 2)


def hadamard_multipliers(seed: int, m: int, n: int):
    """Random permutations (int32) and +-1 scalings (float32) of the rows of
    F and the columns of H: (perm_rows, sign_rows, perm_cols, sign_cols)."""
    rng = rng_for(seed)
    pr = rng.permutation(m).astype(np.int32)
    sr = rng.choice(np.array([-1.0, 1.0], np.float32), m)
    pc = rng.permutation(n).astype(np.int32)
    sc = rng.choice(np.array([-1.0, 1.0], np.float32), n)
    return pr, sr, pc, sc


def lsr_problem(seed: int, kind: str, m: int, n: int):
    """(A, b) of one LSR test input (FP64): kind "gaussian", "ill",
    "semicoherent" or "coherent"."""
    rng = rng_for(seed)
    if kind == "gaussian":
        A = rng.standard_normal((m, n))
    elif kind == "ill":
        q, rr = np.linalg.qr(rng.standard_normal((m, n)))
        S = q * np.sign(np.diag(rr))[None, :]          # Haar on the m x n Stiefel manifold
        T = haar_orthogonal(rng, n)
        sig = np.full(n, 1e-10)
        lead = 10.0 ** np.arange(4, -10, -1)
        sig[:min(n, lead.size)] = lead[:n]
        A = (S * sig[None, :]) @ T.T
    elif kind == "semicoherent":
        h = n // 2
        A = np.zeros((m, n))
        A[:m - h, :h] = rng.standard_normal((m - h, h))
        A[m - h:, h:] = np.diag(rng.choice([-1.0, 1.0], n - h))
    elif kind == "coherent":
        A = np.zeros((m, n))
        A[:n, :n] = np.diag(rng.choice([-1.0, 1.0], n))
    else:
        raise ValueError(kind)
    b = rng.standard_normal(m)
    return A, b
