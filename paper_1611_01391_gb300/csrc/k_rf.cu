// The range finder of Algorithm 5.1a (LRA U V of M from Y = M H) and the
// superfast dual LSR of Algorithm 3.1 (the least squares problem of k
// sampled rows), both through tall-skinny factorisations in FP64:
//   * the Gram matrix Y^T Y of an N x k matrix, split over row chunks and
//     32 x 32 tiles of the Gram matrix (per-chunk partial sums, added in a
//     fixed order by the factorisation, so results are reproducible);
//   * the rank-revealing QR of Y as pivoted Cholesky of Y^T Y: diagonal
//     pivoting on the Schur complement picks, in exact arithmetic, the
//     columns of Businger-Golub QR with column pivoting (the largest
//     remaining column norm), and R_jj are that QR's diagonal;
//   * CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto 2014) for the
//     orthonormal factor, and shifted CholeskyQR3 (Fukaya, Kannan,
//     Nakatsukasa, Zhang, Yamamoto 2020) for the LSR, whose inputs can be
//     ill conditioned: leading passes on Y^T Y + s I, s = 11 (N k + k (k + 1))
//     u ||Y||_F^2, then two plain passes.
#include <cfloat>

#include "lra_internal.cuh"
#include "lra_kernels.h"

namespace lra {
namespace {

constexpr int kGt = 32;          // Gram tile
constexpr int kRowsBatch = 32;   // rows staged per step
constexpr int kSmallT = 1024;

// partials[chunk][a * k + c] = sum over the chunk's rows of Y[i][a] Y[i][c]
// for c >= a (upper triangle with the diagonal); Y element (i, c) at
// Y[i * si + c * st].  Block (tile pair, chunk): 32 x 32 threads, one
// entry each; 32 rows of both tiles' columns are staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(kGt * kGt) ts_gram_kernel(const T* __restrict__ Y, long long N, int k,
                                                            long long si, long long st, int nchunks,
                                                            double* __restrict__ partials,
                                                            const JobStatus* js) {
  if (js->status != LRA_OK) return;
  __shared__ double ya[kRowsBatch][kGt + 1], yb[kRowsBatch][kGt + 1];
  // tile pair (ta <= tb) from the linear block index
  const int nt = (k + kGt - 1) / kGt;
  int p = blockIdx.x, ta = 0;
  while (p >= nt - ta) {
    p -= nt - ta;
    ++ta;
  }
  const int tb = ta + p;
  const int chunk = blockIdx.y;
  const long long per = (N + nchunks - 1) / nchunks;
  const long long r0 = chunk * per, r1 = min(N, r0 + per);
  const int tx = threadIdx.x % kGt, ty = threadIdx.x / kGt;
  const int a = ta * kGt + ty, c = tb * kGt + tx;
  const int ca = ta * kGt + tx, cb = tb * kGt + tx;
  // thread (ty, tx) stages row base + ty, column tx of both tiles; the next
  // batch's two values are loaded while the current one is summed
  auto fetch = [&](long long base, T& va, T& vb) {
    const long long i = base + ty;
    va = (i < r1 && ca < k) ? Y[i * si + (long long)ca * st] : T(0);
    vb = (i < r1 && cb < k) ? Y[i * si + (long long)cb * st] : T(0);
  };
  double acc = 0.0;
  T va, vb;
  if (r0 < r1) fetch(r0, va, vb);
  for (long long base = r0; base < r1; base += kRowsBatch) {
    ya[ty][tx] = (double)va;
    yb[ty][tx] = (double)vb;
    __syncthreads();
    if (base + kRowsBatch < r1) fetch(base + kRowsBatch, va, vb);
#pragma unroll 8
    for (int t = 0; t < kRowsBatch; ++t) acc = fma(ya[t][ty], yb[t][tx], acc);
    __syncthreads();
  }
  if (a < k && c < k && c >= a) partials[(size_t)chunk * k * k + (size_t)a * k + c] = acc;
}

// One CTA: G = sum of the partials (fixed order), pivoted Cholesky
// G(piv, piv) = R^T R with the largest remaining diagonal as pivot (ties to
// the smaller column index), the numerical rank nr = #{R_jj > rank_tol R_00}
// (stopping there), and for r <= nr the l x r matrix Gm = P R_r^{-1}
// (row piv[s] of Gm is row s of R_r^{-1}, other rows zero), so that
// Y Gm = Y(:, piv[:r]) R_r^{-1}.  Below the target rank: LRA_ESINGULAR.
// No interchanges: G keeps the original order, step j writes row j of the
// factor as Rr[j][c] (column c of the original order) and updates the
// Schur complement of the columns not yet chosen; warp 0 finds each pivot
// with shuffles.  Shared memory: G (k x k) and Rr (k x k).
__global__ void __launch_bounds__(kSmallT) pchol_kernel(const double* __restrict__ partials, int nparts, int k,
                                                        int r, double rank_tol, double* __restrict__ Gm,
                                                        int* __restrict__ piv_out, JobStatus* js) {
  if (js->status != LRA_OK) return;
  extern __shared__ double pc_sm[];
  double* G = pc_sm;
  double* Rr = pc_sm + k * k;
  __shared__ int piv[kMaxL];
  __shared__ unsigned char done[kMaxL];
  __shared__ int p_s, nr_s;
  __shared__ double r00_s;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int a = e / k, c = e - a * k;
    double s = 0.0;
    if (c >= a)
      for (int b = 0; b < nparts; ++b) s += partials[(size_t)b * k * k + e];
    G[e] = s;
    Rr[e] = 0.0;
  }
  if (tid < k) {
    piv[tid] = tid;
    done[tid] = 0;
  }
  if (tid == 0) nr_s = k;
  __syncthreads();
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int a = e / k, c = e - a * k;
    if (c < a) G[e] = G[c * k + a];
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (tid < 32) {
      // the largest remaining diagonal, ties to the smaller column
      double best = -1.0;
      int bp = k;
      for (int q = lane; q < k; q += 32)
        if (!done[q] && G[q * k + q] > best) {
          best = G[q * k + q];
          bp = q;
        }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int op = __shfl_xor_sync(0xffffffffu, bp, off);
        if (ob > best || (ob == best && op < bp)) {
          best = ob;
          bp = op;
        }
      }
      if (lane == 0) {
        const double d = bp < k ? G[bp * k + bp] : 0.0;
        const double rjj = d > 0.0 ? sqrt(d) : 0.0;
        if (j == 0) r00_s = rjj;
        if (bp >= k || !(rjj > rank_tol * r00_s) || !(rjj > 0.0)) {
          nr_s = j;
        } else {
          Rr[j * k + bp] = rjj;
          piv[j] = bp;
          done[bp] = 1;
          p_s = bp;
        }
      }
    }
    __syncthreads();
    if (nr_s <= j) break;
    const int p = p_s;
    const double rjj = Rr[j * k + p];
    for (int c = tid; c < k; c += blockDim.x)
      if (!done[c]) Rr[j * k + c] = G[p * k + c] / rjj;
    __syncthreads();
    // Schur complement of the columns not chosen yet
    for (int e = tid; e < k * k; e += blockDim.x) {
      const int a = e / k, c = e - a * k;
      if (!done[a] && !done[c]) G[e] -= Rr[j * k + a] * Rr[j * k + c];
    }
    __syncthreads();
  }
  const int nr = nr_s;
  // the unchosen columns follow in their original order (a complete permutation)
  if (tid == 0) {
    js->k_eff = nr;
    int s = nr;
    for (int q = 0; q < k; ++q)
      if (!done[q]) piv[s++] = q;
  }
  __syncthreads();
  for (int q = tid; q < k; q += blockDim.x) piv_out[q] = piv[q];
  if (nr < r) {
    if (tid == 0) set_status(js, LRA_ESINGULAR);
    return;
  }
  // Gm = P R_r^{-1}: column t of R_r^{-1} by back substitution (thread t),
  // R[s][q] = Rr[s][piv[q]] (row s of the factor, pivoted column q)
  for (int e = tid; e < k * r; e += blockDim.x) Gm[e] = 0.0;
  __syncthreads();
  for (int t = tid; t < r; t += blockDim.x) {
    for (int s = t; s >= 0; --s) {
      double v = (s == t) ? 1.0 : 0.0;
      for (int q = s + 1; q <= t; ++q) v -= Rr[s * k + piv[q]] * Gm[(size_t)piv[q] * r + t];
      Gm[(size_t)piv[s] * r + t] = v / Rr[s * k + piv[s]];
    }
  }
}

// U[i][t] = sum_{c <= t} Q1[i][c] Linv[t][c] (Q1 R2^{-1} with R2 = L^T),
// rounded to FP32: the orthonormal factor of the second CholeskyQR pass.
__global__ void __launch_bounds__(256) rf_finish_kernel(const double* __restrict__ Q1, long long N, int r,
                                                        const double* __restrict__ Linv, float* __restrict__ U,
                                                        const JobStatus* js) {
  if (js->status != LRA_OK) return;
  extern __shared__ double Ls[];
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) Ls[e] = Linv[e];
  __syncthreads();
  const long long total = N * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / r;
    const int t = (int)(e - i * r);
    double acc = 0.0;
    for (int c = 0; c <= t; ++c) acc = fma(Q1[i * r + c], Ls[t * r + c], acc);
    U[e] = (float)acc;
  }
}

// FW[t][j] = W(rows[t], j) in FP64 for a stored FP32 or FP64 source.
__global__ void __launch_bounds__(256) gather_rows_f64_kernel(SourceDev s, const int* __restrict__ rows, int k,
                                                              double* __restrict__ FW) {
  const long long n = s.n, total = (long long)k * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / n, j = e - t * n;
    const long long i = __ldg(rows + t);
    FW[e] = s.kind == LRA_DENSE_F64 ? __ldg(static_cast<const double*>(s.a) + i * s.lda + j)
                                    : (double)__ldg(static_cast<const float*>(s.a) + i * s.lda + j);
  }
}

// Q[i][:] = W[i][:] R^{-1} (R upper k x k, given as its transpose Rt, lower,
// row j of Rt = column j of R), for a block of kTrsmRows rows per CTA held in
// shared memory, by panels of 32 columns: first every entry (i, j) of the
// panel subtracts sum_{c < j0} q_c R[c][j] (c in order, two rows per thread
// so that the FP64 pipe always has independent multiply-adds), then one warp
// per row solves the panel's triangle: lane t holds entry j0 + t, step s
// multiplies lane s's value by 1 / R_jj (formed beforehand) and the lanes
// t > s subtract R[j0 + s][j0 + t] times it.
constexpr int kTrsmRows = 16;

__global__ void __launch_bounds__(256) trsm_rows_kernel(const double* __restrict__ W, long long N, int k,
                                                        const double* __restrict__ Rt, double* __restrict__ Q,
                                                        const JobStatus* js) {
  if (js->status != LRA_OK) return;
  extern __shared__ double tr_sm[];
  double* Qs = tr_sm;                        // kTrsmRows x k
  double* rinv = Qs + (size_t)kTrsmRows * k; // k
  __shared__ double T[32][33];               // the panel's triangle of R: T[t][s] = R[j0 + s][j0 + t]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long i0 = (long long)blockIdx.x * kTrsmRows;
  const int nr = (int)min((long long)kTrsmRows, N - i0);
  for (int e = tid; e < nr * k; e += blockDim.x) Qs[e] = W[i0 * k + e];
  for (int j = tid; j < k; j += blockDim.x) rinv[j] = 1.0 / Rt[(size_t)j * k + j];
  for (int j0 = 0; j0 < k; j0 += 32) {
    const int w = min(32, k - j0);
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
      const int t = e >> 5, c = e & 31;
      T[t][c] = (t < w && c < t) ? Rt[(size_t)(j0 + t) * k + j0 + c] : 0.0;
    }
    __syncthreads();
    // the panel minus the part already solved: rows warp and warp + 8, column j0 + lane
    if (lane < w && j0 > 0) {
      const double* rt = Rt + (size_t)(j0 + lane) * k;
      for (int ib = warp; ib < nr; ib += 16) {
        const int ia = ib, ic = ib + 8;
        double xa = Qs[(size_t)ia * k + j0 + lane];
        double xc = ic < nr ? Qs[(size_t)ic * k + j0 + lane] : 0.0;
        const double* qa = Qs + (size_t)ia * k;
        const double* qc = Qs + (size_t)(ic < nr ? ic : ia) * k;
#pragma unroll 4
        for (int c = 0; c < j0; ++c) {
          const double r = __ldg(rt + c);
          xa = fma(-qa[c], r, xa);
          xc = fma(-qc[c], r, xc);
        }
        Qs[(size_t)ia * k + j0 + lane] = xa;
        if (ic < nr) Qs[(size_t)ic * k + j0 + lane] = xc;
      }
    }
    __syncthreads();
    // the triangle, one warp per row
    for (int ib = warp; ib < nr; ib += 8) {
      double x = lane < w ? Qs[(size_t)ib * k + j0 + lane] : 0.0;
      for (int s2 = 0; s2 < w; ++s2) {
        const double y = __shfl_sync(0xffffffffu, x * rinv[j0 + (lane < w ? lane : 0)], s2);
        if (lane == s2) Qs[(size_t)ib * k + j0 + s2] = y;
        if (lane > s2 && lane < w) x = fma(-T[lane][s2], y, x);
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nr * k; e += blockDim.x) Q[i0 * k + e] = Qs[e];
}

// Grid-wide barrier of a cooperative launch on a counter that only grows:
// the n-th barrier waits until the counter reaches n gridDim.x.  Thread 0 of
// each block arrives with a release add and polls with acquire loads,
// bounded by 2 s (LRA_ETIMEOUT); every thread returns the same verdict.
__device__ __forceinline__ bool coop_barrier(unsigned int* count, unsigned int target, JobStatus* js, int* flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    const unsigned long long t0 = globaltimer_ns();
    int ok = 1;
    for (unsigned int it = 1;; ++it) {
      if ((int)(ld_acquire_u32(count) - target) >= 0) break;
      if ((it & 63u) == 0 && globaltimer_ns() - t0 > kWaitNs) {
        set_status(js, LRA_ETIMEOUT);
        ok = 0;
        break;
      }
    }
    *flag = ok;
  }
  __syncthreads();
  return *flag != 0;
}

// Cooperative form of the FP64 Cholesky G + shift I = R^T R for k up to
// 1024, by panels of kCholP columns: G (upper triangle, from the partials)
// and R in global memory, two grid barriers per panel.  For the panel of
// rows j0 .. j1 - 1:
//   (A) every block factors the diagonal block itself (the same values
//       everywhere): for j = j0 .. j1 - 1, r_jj = sqrt(G_jj + shift) and
//       R[j][c] = G[j][c] / r_jj, then G[a][c] -= R[j][a] R[j][c] for the
//       block's rows a > j;
//   (B) one warp per column c >= j1 (over the whole grid) forms the panel's
//       rows of R there: lane i holds G[j0 + i][c]; step s divides lane s's
//       value by r_ss and the lanes i > s subtract R[s][j0 + i] times it;
//   (C) grid barrier; every block applies the panel to the trailing rows it
//       owns (a >= j1, a mod gridDim == blockIdx): G[a][c] -= R[s][a] R[s][c]
//       for s = j0 .. j1 - 1 in order; grid barrier.
// Every entry of G receives the same multiply-subtracts in the same order as
// in the column-by-column elimination (one multiply-subtract per earlier
// row, each from the row's final values), and every entry of R the same
// division, so the factor is the column-by-column one bit for bit.  A pivot
// d <= floor_rel G_jj (G_jj the column's squared norm before the
// elimination; floor_rel = 0: a non-positive pivot) is a numerically rank
// deficient column: LRA_ESINGULAR (every block sees the same value and
// stops).  Data written by other blocks is read past L1 (ld.global.cg).
constexpr int kCholP = 32;

__global__ void __launch_bounds__(256, 1) chol_coop_kernel(const double* __restrict__ partials, int nparts, int k,
                                                        double shift_rel, double floor_rel,
                                                        double* __restrict__ G, double* __restrict__ Gd,
                                                        double* __restrict__ R, double* __restrict__ Rt,
                                                        unsigned int* bar, JobStatus* js) {
  __shared__ double D[kCholP][kCholP + 1];   // the diagonal block (upper), then its rows of R
  __shared__ double rd[kCholP];              // the panel's r_jj
  __shared__ double ra[kCholP];              // R[j0 .. j1)[a] of the trailing row a
  __shared__ double red[8];
  __shared__ int flag;
  const int tid = threadIdx.x, nb = gridDim.x, b = blockIdx.x, lane = tid & 31, warp = tid >> 5;
  if (js->status != LRA_OK) return;
  for (long long e = (long long)b * blockDim.x + tid; e < (long long)k * k; e += (long long)nb * blockDim.x) {
    const int a = (int)(e / k), c = (int)(e - (long long)a * k);
    double s = 0.0;
    if (c >= a)
      for (int q = 0; q < nparts; ++q) s += partials[(size_t)q * k * k + e];
    G[e] = s;
    if (c == a) Gd[a] = s;
    R[e] = 0.0;
    Rt[e] = 0.0;
  }
  unsigned int nbar = 0;
  if (!coop_barrier(bar, ++nbar * nb, js, &flag)) return;
  // shift = shift_rel * trace(G), summed in a fixed order by every block
  double tr = 0.0;
  for (int a = tid; a < k; a += blockDim.x) tr += __ldcg(G + (size_t)a * k + a);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, off);
  if ((tid & 31) == 0) red[tid >> 5] = tr;
  __syncthreads();
  double trace = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) trace += red[w];
  const double shift = shift_rel * trace;
  for (int j0 = 0; j0 < k; j0 += kCholP) {
    const int j1 = min(j0 + kCholP, k), w = j1 - j0;
    // (A) the diagonal block
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int a = e / w, c = e - a * w;
      D[a][c] = c >= a ? __ldcg(G + (size_t)(j0 + a) * k + j0 + c) : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
      const double d = D[j][j] + shift;
      if (!(d > 0.0) || !(d > floor_rel * __ldcg(Gd + j0 + j))) {
        if (b == 0 && tid == 0) set_status(js, LRA_ESINGULAR);
        return;
      }
      const double rjj = sqrt(d);
      for (int c = j + 1 + tid; c < w; c += blockDim.x) D[j][c] = D[j][c] / rjj;
      if (tid == 0) rd[j] = rjj;
      __syncthreads();
      for (int e = tid; e < w * w; e += blockDim.x) {
        const int a = e / w, c = e - a * w;
        if (a > j && c >= a) D[a][c] -= D[j][a] * D[j][c];
      }
      __syncthreads();
    }
    if (b == 0)
      for (int e = tid; e < w * w; e += blockDim.x) {
        const int a = e / w, c = e - a * w;
        if (c >= a) {
          const double v = c == a ? rd[a] : D[a][c];
          R[(size_t)(j0 + a) * k + j0 + c] = v;
          Rt[(size_t)(j0 + c) * k + j0 + a] = v;
        }
      }
    // (B) the panel's rows of R in the columns c >= j1, one warp per column
    const int gw = b * (int)(blockDim.x >> 5) + warp, nw = nb * (int)(blockDim.x >> 5);
    for (int c = j1 + gw; c < k; c += nw) {
      double x = lane < w ? __ldcg(G + (size_t)(j0 + lane) * k + c) : 0.0;
      for (int s = 0; s < w; ++s) {
        double r = 0.0;
        if (lane == s) {
          r = x / rd[s];
          R[(size_t)(j0 + s) * k + c] = r;
          Rt[(size_t)c * k + j0 + s] = r;
        }
        r = __shfl_sync(0xffffffffu, r, s);
        if (lane > s && lane < w) x -= D[s][lane] * r;
      }
    }
    if (j1 >= k) break;
    // (C) the trailing rows this block owns
    if (!coop_barrier(bar, ++nbar * nb, js, &flag)) return;
    const int a_first = j1 + ((b - j1) % nb + nb) % nb;
    for (int a = a_first; a < k; a += nb) {
      __syncthreads();   // the previous row's ra read everywhere
      if (tid < w) ra[tid] = __ldcg(R + (size_t)(j0 + tid) * k + a);
      __syncthreads();
      for (int c = a + tid; c < k; c += blockDim.x) {
        double x = __ldcg(G + (size_t)a * k + c);
#pragma unroll
        for (int s = 0; s < kCholP; ++s)
          if (s < w) x -= ra[s] * __ldcg(R + (size_t)(j0 + s) * k + c);
        G[(size_t)a * k + c] = x;
      }
    }
    if (!coop_barrier(bar, ++nbar * nb, js, &flag)) return;
  }
}

// The least squares solution from the factors R_1 .. R_p of (FA | Fb) =
// Q R_p ... R_1 (upper, (n+1) x (n+1)): v = R_p ... R_1 e_n (the last column
// of the product, one thread per row for each factor), then x =
// (R_1)_nn^{-1} ... (R_p)_nn^{-1} v[:n] by back substitutions over blocks of
// 32 rows from the bottom: the block's rows take their products with the
// part already solved (one warp per row, lanes splitting the sum), then one
// warp solves the block's triangle, lane i holding row i and multiplying
// by the reciprocal of the diagonal (formed beforehand, in parallel).
// rho = |v[n]| is the residual norm of the sampled problem.
__global__ void __launch_bounds__(kSmallT) lsr_solve_kernel(const double* __restrict__ Rs, int p, int k,
                                                            double* __restrict__ v_out, double* __restrict__ x_out,
                                                            double* __restrict__ rho, const JobStatus* js) {
  if (js->status != LRA_OK) return;
  __shared__ double v[1024], tmp[1024];
  __shared__ double D[32][33], rest[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = k - 1;
  const size_t kk = (size_t)k * k;
  for (int a = tid; a < k; a += blockDim.x) v[a] = Rs[(size_t)a * k + n];   // R_1 e_n
  __syncthreads();
  for (int s = 1; s < p; ++s) {
    const double* Rm = Rs + s * kk;
    for (int a = tid; a < k; a += blockDim.x) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      int c = a;
      for (; c + 4 <= k; c += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(Rm[(size_t)a * k + c + u], v[c + u], acc[u]);
      }
      for (; c < k; ++c) acc[0] = fma(Rm[(size_t)a * k + c], v[c], acc[0]);
      tmp[a] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    __syncthreads();
    for (int a = tid; a < k; a += blockDim.x) v[a] = tmp[a];
    __syncthreads();
  }
  if (tid == 0) *rho = fabs(v[n]);
  for (int s = p - 1; s >= 0; --s) {
    const double* Rm = Rs + s * kk;
    for (int a = tid; a < n; a += blockDim.x) tmp[a] = 1.0 / Rm[(size_t)a * k + a];
    __syncthreads();
    for (int a1 = n; a1 > 0; a1 -= 32) {
      const int a0 = a1 > 32 ? a1 - 32 : 0, w = a1 - a0;
      if (warp < w) {
        const int a = a0 + warp;
        const double* row = Rm + (size_t)a * k;
        double t0 = 0.0, t1 = 0.0;
        int c = a1 + lane;
        for (; c + 32 < n; c += 64) {
          t0 = fma(row[c], v[c], t0);
          t1 = fma(row[c + 32], v[c + 32], t1);
        }
        if (c < n) t0 = fma(row[c], v[c], t0);
        double t = t0 + t1;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) rest[warp] = v[a] - t;
        if (lane < w) D[warp][lane] = row[a0 + lane];
      }
      __syncthreads();
      if (warp == 0) {
        double x = lane < w ? rest[lane] : 0.0;
        for (int j = w - 1; j >= 0; --j) {
          const double y = __shfl_sync(0xffffffffu, x * tmp[a0 + (lane < w ? lane : 0)], j);
          if (lane == j) v[a0 + j] = y;
          if (lane < j) x = fma(-D[lane][j], y, x);
        }
      }
      __syncthreads();
    }
  }
  for (int a = tid; a < n; a += blockDim.x) x_out[a] = v[a];
  for (int a = tid; a < k; a += blockDim.x) v_out[a] = v[a];
}

// ASPH multipliers (Section 8.1): Y[i][t] = sign[t] (M H_{n,d})[i][J[t]],
// with (b, o) = divmod(J[t], n / 2^d) the signed sum over q of
// M[i][q (n / 2^d) + o] in the order of the recursive Hadamard steps, in
// FP32 (the butterfly order of the pre-processed entries).
__global__ void __launch_bounds__(256) asph_cols_kernel(const float* __restrict__ M, long long lda, long long m,
                                                        long long sn, int d, const int* __restrict__ J,
                                                        const float* __restrict__ sign, int l,
                                                        float* __restrict__ Y) {
  const long long total = m * l;
  const int D = 1 << d;
  float stk[kMaxPreD + 1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / l;
    const int t = (int)(e - i * l);
    const long long y = __ldg(J + t);
    const long long b = y / sn, o = y - b * sn;
    const float* row = M + i * lda + o;
    float acc = 0.0f;
    for (int q = 0; q < D; ++q) acc = butterfly_push(stk, q, __ldg(row + q * sn), (unsigned)b);
    Y[e] = __ldg(sign + t) * acc;
  }
}

// FW[t][j] = sign[t] (H_{m,d} W)[rows[t]][j] in FP64: the signed sum over p
// of W[p (m / 2^d) + o][j], (b, o) = divmod(rows[t], m / 2^d), butterfly
// order; consecutive threads take consecutive j.
__global__ void __launch_bounds__(256) asph_rows_f64_kernel(SourceDev s, int d, long long sm,
                                                            const int* __restrict__ rows,
                                                            const float* __restrict__ sign, int k,
                                                            double* __restrict__ FW) {
  const long long n = s.n, total = (long long)k * n;
  const int D = 1 << d;
  double stk[kMaxPreD + 1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / n, j = e - t * n;
    const long long x = __ldg(rows + t);
    const long long b = x / sm, o = x - b * sm;
    double acc = 0.0;
    for (int p = 0; p < D; ++p) {
      const long long i = p * sm + o;
      const double v = s.kind == LRA_DENSE_F64 ? __ldg(static_cast<const double*>(s.a) + i * s.lda + j)
                                               : (double)__ldg(static_cast<const float*>(s.a) + i * s.lda + j);
      acc = butterfly_push(stk, p, v, (unsigned)b);
    }
    FW[e] = (double)__ldg(sign + t) * acc;
  }
}

int gram_chunks(long long N, int k) {
  const int nt = (k + kGt - 1) / kGt;
  const int pairs = nt * (nt + 1) / 2;
  long long ch = (2 * 152 + pairs - 1) / pairs;
  const long long max_by_rows = (N + 255) / 256;   // at least 256 rows per chunk
  if (ch > max_by_rows) ch = max_by_rows;
  if (ch < 1) ch = 1;
  if (ch > 256) ch = 256;
  return (int)ch;
}

}  // namespace

int ts_gram_chunks(long long N, int k) { return gram_chunks(N, k); }

cudaError_t launch_ts_gram_f32(const float* Y, long long N, int k, long long si, long long st, double* partials,
                               int nchunks, const JobStatus* js, cudaStream_t s) {
  const int nt = (k + kGt - 1) / kGt;
  ts_gram_kernel<float><<<dim3(nt * (nt + 1) / 2, nchunks), kGt * kGt, 0, s>>>(Y, N, k, si, st, nchunks, partials,
                                                                                js);
  return cudaGetLastError();
}

cudaError_t launch_ts_gram_f64(const double* Y, long long N, int k, double* partials, int nchunks,
                               const JobStatus* js, cudaStream_t s) {
  const int nt = (k + kGt - 1) / kGt;
  ts_gram_kernel<double><<<dim3(nt * (nt + 1) / 2, nchunks), kGt * kGt, 0, s>>>(Y, N, k, k, 1, nchunks, partials,
                                                                                 js);
  return cudaGetLastError();
}

cudaError_t launch_pchol(const double* partials, int nparts, int k, int r, double rank_tol, double* Gm, int* piv,
                         JobStatus* js, cudaStream_t s) {
  const size_t sm = sizeof(double) * 2 * k * k;
  cudaError_t e = smem_optin(reinterpret_cast<const void*>(pchol_kernel), (int)sm);
  if (e) return e;
  pchol_kernel<<<1, kSmallT, sm, s>>>(partials, nparts, k, r, rank_tol, Gm, piv, js);
  return cudaGetLastError();
}

cudaError_t launch_rf_finish(const double* Q1, long long N, int r, const double* Linv, float* U, const JobStatus* js,
                             int sms, cudaStream_t s) {
  long long g = (N * r + 255) / 256;
  if (g > (long long)sms * 8) g = (long long)sms * 8;
  rf_finish_kernel<<<(int)g, 256, sizeof(double) * r * r, s>>>(Q1, N, r, Linv, U, js);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows_f64(const SourceDev& src, const int* rows, int k, double* FW, int sms, cudaStream_t s) {
  long long g = ((long long)k * src.n + 255) / 256;
  if (g > (long long)sms * 8) g = (long long)sms * 8;
  gather_rows_f64_kernel<<<(int)g, 256, 0, s>>>(src, rows, k, FW);
  return cudaGetLastError();
}

cudaError_t launch_asph_cols(const float* M, long long lda, long long m, long long n, int d, const int* J,
                             const float* sign, int l, float* Y, int sms, cudaStream_t s) {
  long long g = (m * l + 255) / 256;
  if (g > (long long)sms * 8) g = (long long)sms * 8;
  asph_cols_kernel<<<(int)g, 256, 0, s>>>(M, lda, m, n >> d, d, J, sign, l, Y);
  return cudaGetLastError();
}

cudaError_t launch_asph_rows_f64(const SourceDev& src, int d, const int* rows, const float* sign, int k, double* FW,
                                 int sms, cudaStream_t s) {
  long long g = ((long long)k * src.n + 255) / 256;
  if (g > (long long)sms * 8) g = (long long)sms * 8;
  asph_rows_f64_kernel<<<(int)g, 256, 0, s>>>(src, d, src.m >> d, rows, sign, k, FW);
  return cudaGetLastError();
}

cudaError_t launch_chol_coop(const double* partials, int nparts, int k, double shift_rel, double floor_rel,
                             double* G, double* Gd, double* R, double* Rt, unsigned int* bar, JobStatus* js, int sms,
                             cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_coop_kernel, 256, 0);
  if (e) return e;
  int grid = sms * (per_sm > 0 ? 1 : 0);
  if (grid > k) grid = k;
  if (grid < 1) grid = 1;
  void* args[] = {(void*)&partials, (void*)&nparts, (void*)&k, (void*)&shift_rel, (void*)&floor_rel,
                  (void*)&G, (void*)&Gd, (void*)&R, (void*)&Rt, (void*)&bar, (void*)&js};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(chol_coop_kernel), dim3(grid), dim3(256), args, 0,
                                     s);
}

cudaError_t launch_trsm_rows(const double* W, long long N, int k, const double* Rt, double* Q, const JobStatus* js,
                             int sms, cudaStream_t s) {
  (void)sms;
  const size_t smem = sizeof(double) * ((size_t)kTrsmRows * k + k);
  cudaError_t e = smem_optin(reinterpret_cast<const void*>(trsm_rows_kernel), (int)smem);
  if (e) return e;
  trsm_rows_kernel<<<(int)((N + kTrsmRows - 1) / kTrsmRows), 256, smem, s>>>(W, N, k, Rt, Q, js);
  return cudaGetLastError();
}

cudaError_t launch_lsr_solve(const double* Rs, int p, int k, double* v, double* x, double* rho, const JobStatus* js,
                             cudaStream_t s) {
  lsr_solve_kernel<<<1, kSmallT, 0, s>>>(Rs, p, k, v, x, rho, js);
  return cudaGetLastError();
}

}  // namespace lra
