// Nucleus of the CUR approximation (Primitive Algorithm, stages 2-3 of
// Section 6.5): the l x l CUR generator X = M[I, J], its SVD, the rank-k
// truncation and U = (X_k)^+.
//
// The SVD (svd_dd.cuh) is QR with column pivoting followed by one-sided
// Jacobi on R^T, in double-float arithmetic; the left singular vectors of
// the kept triplets are X v_b / sigma_b.  X is first scaled by a power
// of two so that max |X| lies in [0.5, 1) (exact); sigma and U are scaled
// back.
#include <cooperative_groups.h>

#include <cfloat>

#include "lra_kernels.h"
#include "lra_internal.cuh"
#include "svd_dd.cuh"

namespace cg = cooperative_groups;

namespace lra {

constexpr int kNucThreads = 512;

__global__ void __launch_bounds__(kNucThreads, 1)
nucleus_kernel(const float* __restrict__ C, const int* __restrict__ I, int l, int k,
               double rank_tol, double* __restrict__ U, double* __restrict__ sigma_out,
               JobStatus* js) {
  if (js->status != LRA_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* W = reinterpret_cast<dd*>(smem_raw);           // column b at W + b*l
  dd* Z = W + (size_t)l * l;                          // column b at Z + b*l
  double* sig = reinterpret_cast<double*>(Z + (size_t)l * l);  // l
  dd* inv2 = reinterpret_cast<dd*>(sig + kMaxL);      // l
  SvdScratch* sc = reinterpret_cast<SvdScratch*>(inv2 + kMaxL);
  int* order = reinterpret_cast<int*>(sc + 1);        // l: order[rank] = column
  int* keff_s = order + kMaxL;
  int* scale_e = keff_s + 1;

  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) *scale_e = 0;
  __syncthreads();
  // power-of-two scale so that max |X| is in [0.5, 1)
  float amax = 0.0f;
  for (int e = tid; e < l * l; e += nthr) {
    const int a = e / l, b = e - a * l;
    amax = fmaxf(amax, fabsf(C[(size_t)__ldg(I + a) * l + b]));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
  if ((tid & 31) == 0 && amax > 0.0f) {
    int ex;
    frexpf(amax, &ex);
    atomicMax(scale_e, ex + 1024);  // offset keeps the stored value positive
  }
  __syncthreads();
  const int ex = *scale_e ? *scale_e - 1024 : 0;
  for (int e = tid; e < l * l; e += nthr) {
    const int a = e / l, b = e - a * l;             // X[a][b] = C[I[a]][b]
    W[(size_t)b * l + a] = dd_make(ldexpf(C[(size_t)__ldg(I + a) * l + b], -ex));
  }
  __syncthreads();
  svd_dd<kNucThreads>(W, Z, l, sc);
  jacobi_sigma<kNucThreads>(W, l, sig, order);
  if (tid == 0) {
    const double s1 = sig[order[0]];
    int ke = 0;
    if (s1 > 0.0)
      while (ke < k && ke < l && sig[order[ke]] > rank_tol * s1) ++ke;
    *keff_s = ke;
    js->k_eff = ke;
    js->sigma_max = ldexp(s1, ex);
  }
  for (int r = tid; r < l; r += nthr) {
    const double sb = sig[order[r]];
    inv2[r] = dd_from_double(sb > 0.0 ? 1.0 / (sb * sb) : 0.0);
    sigma_out[r] = ldexp(sb, ex);
  }
  __syncthreads();
  const int ke = *keff_s;
  left_vectors<kNucThreads>(W, Z, l, ke, order, inv2, sc->perm);
  nucleus_from_svd<kNucThreads>(W, Z, sc->perm, l, ke, order, inv2,
                                [&](int e, double v) { U[e] = ldexp(v, -ex); });
}

// X^{-1} of the cross X[a][b] = S[pos[a]][b] of an N x l strip (element
// (i, t) at strip[i*si + t*st]), by in-place Gauss-Jordan elimination with
// partial pivoting in FP64 (Golub & Van Loan, 3.4; l^3 FMAs).  Step t: the
// pivot is the largest |A[r][t]|, r >= t (smallest r on ties), rows t and p
// are swapped, column t is replaced by the column of the inverse it
// produces, and every other row is updated; the row swaps are undone as
// column swaps at the end.
//
// One thread-block cluster of 8 CTAs shares the FP64 work (GB300 issues
// FP64 at 1/64 of the FP32 rate, so one SM would be the bottleneck): CTA c
// owns columns [c w, c w + w), w = ceil(l / 8).  At step t the owner of
// column t picks the pivot, publishes p, 1/pivot and the multipliers (the
// column after the swap) in its shared memory, double-buffered by step
// parity; one cluster barrier; every CTA reads them through distributed
// shared memory and updates its own columns.  A zero pivot sets
// LRA_ESINGULAR, a non-finite entry LRA_ENONFINITE; every CTA takes the
// same exit, after a last cluster barrier.
constexpr int kInvCS = 8;    // CTAs per cluster
constexpr int kInvCT = 256;  // threads per CTA

struct InvPub {
  double f[2][kMaxL];        // multipliers of steps with parity 0 / 1
  double rp[2];              // 1 / pivot
  int p[2];                  // pivot row (-1: singular)
  int bad;                   // a non-finite entry in this CTA's columns
};

__global__ void __cluster_dims__(kInvCS, 1, 1) __launch_bounds__(kInvCT, 1)
cross_inverse_kernel(const float* __restrict__ strip, long long si, long long st,
                     const int* __restrict__ pos, int l, float2* __restrict__ xinv, JobStatus* js) {
  if (js->status != LRA_OK || js->stop) return;  // same value in every CTA of the cluster
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int w = (l + kInvCS - 1) / kInvCS;
  const int c0 = rank * w;
  const int nc = max(0, min(w, l - c0));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* A = reinterpret_cast<double*>(smem_raw);  // l x w, row-major: column c0 + cc at cc
  double* f = A + (size_t)l * w;                    // multipliers of the current step
  double* rowt = f + kMaxL;                         // scaled pivot row, own columns
  InvPub* pub = reinterpret_cast<InvPub*>(rowt + kMaxL);
  int* swaps = reinterpret_cast<int*>(pub + 1);     // row swapped with t at step t
  int* at = swaps + kMaxL;                          // column permutation of the result
  int* dest = at + kMaxL;

  int bad = 0;
  for (int e = tid; e < l * nc; e += kInvCT) {
    const int r = e / nc, cc = e - r * nc;
    const double v = (double)strip[(long long)__ldg(pos + r) * si + (long long)(c0 + cc) * st];
    if (!(fabs(v) <= DBL_MAX)) bad = 1;
    A[(size_t)r * w + cc] = v;
  }
  bad = __syncthreads_or(bad);
  if (tid == 0) pub->bad = bad;
  cl.sync();
  int any = 0;
  if (tid < kInvCS) any = *cl.map_shared_rank(&pub->bad, tid);
  any = __syncthreads_or(any);
  if (any) {
    if (rank == 0 && tid == 0) set_status(js, LRA_ENONFINITE);
    cl.sync();
    return;
  }
  for (int t = 0; t < l; ++t) {
    const int o = t / w, par = t & 1;
    if (rank == o) {
      const int ct = t - c0;
      if (tid < 32) {  // pivot: largest |A[r][t]|, r >= t, compared on IEEE bit patterns
        unsigned long long best = 0ull;
        int br = l;
        for (int r = t + tid; r < l; r += 32) {
          const unsigned long long k = abs_bits(A[(size_t)r * w + ct]);
          if (br == l || k > best) { best = k; br = r; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, off);
          const int orr = __shfl_down_sync(0xffffffffu, br, off);
          if (orr < l && (br == l || ob > best || (ob == best && orr < br))) { best = ob; br = orr; }
        }
        if (tid == 0) {
          const int pr = (best != 0ull && br < l) ? br : -1;
          pub->p[par] = pr;
          // one FP64 division for the whole step
          if (pr >= 0) pub->rp[par] = 1.0 / A[(size_t)pr * w + ct];
        }
      }
      __syncthreads();
      const int pr = pub->p[par];
      // multipliers: column t after the swap (row p holds the old row t)
      for (int r = tid; r < l; r += kInvCT) {
        const int rr = (r == pr) ? t : r;
        pub->f[par][r] = (r == t || pr < 0) ? 0.0 : A[(size_t)rr * w + ct];
      }
    }
    cl.sync();
    const InvPub* op = cl.map_shared_rank(pub, o);
    const int p = op->p[par];
    if (p < 0) {
      if (rank == 0 && tid == 0) set_status(js, LRA_ESINGULAR);
      cl.sync();
      return;
    }
    const double rp = op->rp[par];
    for (int r = tid; r < l; r += kInvCT) f[r] = op->f[par][r];
    if (tid == 0) swaps[t] = p;
    for (int cc = tid; cc < nc; cc += kInvCT) {
      const double x = A[(size_t)p * w + cc];
      if (p != t) A[(size_t)p * w + cc] = A[(size_t)t * w + cc];
      const double y = (c0 + cc == t) ? rp : x * rp;
      rowt[cc] = y;
      A[(size_t)t * w + cc] = y;
    }
    __syncthreads();
    for (int e = tid; e < l * nc; e += kInvCT) {
      const int r = e / nc, cc = e - r * nc;
      if (r == t) continue;
      const double a = (c0 + cc == t) ? 0.0 : A[(size_t)r * w + cc];
      A[(size_t)r * w + cc] = fma(-f[r], rowt[cc], a);
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first: result
  // column q is column at[q] of A
  if (tid == 0) {
    for (int q = 0; q < l; ++q) at[q] = q;
    for (int t = l - 1; t >= 0; --t) {
      const int p = swaps[t], x = at[t];
      at[t] = at[p];
      at[p] = x;
    }
    for (int q = 0; q < l; ++q) dest[at[q]] = q;
  }
  __syncthreads();
  for (int e = tid; e < l * nc; e += kInvCT) {
    const int r = e / nc, cc = e - r * nc;
    xinv[(size_t)r * l + dest[c0 + cc]] = split_double(A[(size_t)r * w + cc]);
  }
  cl.sync();  // no peer reads this CTA's shared memory after it exits
}

// The same elimination on one CTA of 512 threads (l <= 96, the matrix in
// shared memory), for contexts whose jobs overlap on the device: the cluster
// kernel is faster for one job but holds 8 SMs for it, this one one SM.
constexpr int kInvCtaT = 512;

__global__ void __launch_bounds__(kInvCtaT, 1)
cross_inverse_cta_kernel(const float* __restrict__ strip, long long si, long long st,
                     const int* __restrict__ pos, int l, float2* __restrict__ xinv, JobStatus* js) {
  if (js->status != LRA_OK || js->stop) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* A = reinterpret_cast<double*>(smem_raw);  // l x l, row-major
  double* f = A + (size_t)l * l;                    // column t before the step
  double* rowt = f + kMaxL;                         // pivot row after scaling
  double* recip = rowt + kMaxL;                     // 1 / pivot of the current step
  int* piv_row = reinterpret_cast<int*>(recip + 1);
  int* swaps = piv_row + 1;                         // row swapped with t at step t
  int* bad = swaps + kMaxL;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) *bad = 0;
  __syncthreads();
  for (int e = tid; e < l * l; e += nthr) {
    const int a = e / l, b = e - a * l;
    const double v = (double)strip[(long long)__ldg(pos + a) * si + (long long)b * st];
    if (!(fabs(v) <= DBL_MAX)) *bad = 1;
    A[e] = v;
  }
  __syncthreads();
  if (*bad) {
    if (tid == 0) set_status(js, LRA_ENONFINITE);
    return;
  }
  for (int t = 0; t < l; ++t) {
    if (tid < 32) {  // pivot: largest |A[r][t]|, r >= t, compared on IEEE bit patterns
      unsigned long long best = 0ull;
      int br = l;
      for (int r = t + tid; r < l; r += 32) {
        const unsigned long long k = abs_bits(A[(size_t)r * l + t]);
        if (br == l || k > best) { best = k; br = r; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, off);
        const int orr = __shfl_down_sync(0xffffffffu, br, off);
        if (orr < l && (br == l || ob > best || (ob == best && orr < br))) { best = ob; br = orr; }
      }
      if (tid == 0) {
        const int p = (best != 0ull && br < l) ? br : -1;
        *piv_row = p;
        swaps[t] = p;
        // one FP64 division for the whole step
        if (p >= 0) *recip = 1.0 / A[(size_t)p * l + t];
      }
    }
    __syncthreads();
    const int p = *piv_row;
    if (p < 0) {
      if (tid == 0) set_status(js, LRA_ESINGULAR);
      return;
    }
    const double rp = *recip;
    // multipliers f[r] = A[r][t] of the rows after the swap (row p will hold
    // the old row t), read before anything is written
    for (int r = tid; r < l; r += nthr) {
      const int rr = (r == p) ? t : r;
      f[r] = (r == t) ? 0.0 : A[(size_t)rr * l + t];
    }
    __syncthreads();
    // pivot row swapped into place and scaled by 1/pivot, its column t set to
    // 1/pivot
    for (int c = tid; c < l; c += nthr) {
      const double x = A[(size_t)p * l + c];
      if (p != t) A[(size_t)p * l + c] = A[(size_t)t * l + c];
      const double y = (c == t) ? rp : x * rp;
      rowt[c] = y;
      A[(size_t)t * l + c] = y;
    }
    __syncthreads();
    // A[r][c] -= f[r] rowt[c] for r != t, with A[r][t] starting from 0
    for (int e = tid; e < l * l; e += nthr) {
      const int r = e / l, c = e - r * l;
      if (r == t) continue;
      const double a = (c == t) ? 0.0 : A[e];
      A[e] = fma(-f[r], rowt[c], a);
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int t = l - 1; t >= 0; --t) {
    const int p = swaps[t];
    if (p != t)
      for (int r = tid; r < l; r += nthr) {
        const double x = A[(size_t)r * l + t];
        A[(size_t)r * l + t] = A[(size_t)r * l + p];
        A[(size_t)r * l + p] = x;
      }
    __syncthreads();
  }
  for (int e = tid; e < l * l; e += nthr) xinv[e] = split_double(A[e]);
}

// The same elimination for l <= 32 on one CTA.  At that size every step is
// a chain of latencies (an FP64 division is ~430 cycles on this part), so a
// step is cut to: the pivot, already reduced during the previous step's
// update (a shared-memory atomic max of packed (|value| as FP32, row) keys
// over the next column, smaller row on ties); one warp forms 1/pivot and the
// scaled pivot row; one barrier; one pass in which every thread writes its
// fixed entries of the next matrix from the current one (two buffers, so no
// entry is read after it is overwritten) and offers its entries of the next
// column as pivot candidates; a second barrier.  The arithmetic per entry is
// that of the cluster kernel.
constexpr int kInvSmallL = 32;
constexpr int kInvSmallT = 128;
constexpr int kInvSmallPer = (kInvSmallL * kInvSmallL + kInvSmallT - 1) / kInvSmallT;

__device__ __forceinline__ unsigned long long pivot_key(double v, int r) {
  // |v| rounded to FP32 orders the candidates; the low word prefers the
  // smaller row among equal keys
  return ((unsigned long long)__float_as_uint(fabsf((float)v)) << 32) | (unsigned)(0x7fffffff - r);
}

__global__ void __launch_bounds__(kInvSmallT, 1)
cross_inverse_small_kernel(const float* __restrict__ strip, long long si, long long st,
                           const int* __restrict__ pos, int l, float2* __restrict__ xinv, JobStatus* js) {
  if (js->status != LRA_OK || js->stop) return;
  __shared__ double buf[2][kInvSmallL * kInvSmallL];
  __shared__ double rowt[kInvSmallL];
  __shared__ unsigned long long pkey[2];
  __shared__ int p_s;
  __shared__ int swaps[kInvSmallL], at[kInvSmallL], dest[kInvSmallL];
  const int tid = threadIdx.x, lane = tid & 31;
  const int ll = l * l;
  // this thread's entries, fixed for all steps
  int er[kInvSmallPer], ec[kInvSmallPer];
#pragma unroll
  for (int k = 0; k < kInvSmallPer; ++k) {
    const int e = tid + k * kInvSmallT;
    er[k] = e < ll ? e / l : -1;
    ec[k] = e < ll ? e - (e / l) * l : 0;
  }
  if (tid < 2) pkey[tid] = 0ull;
  __syncthreads();
  int bad = 0;
#pragma unroll
  for (int k = 0; k < kInvSmallPer; ++k) {
    if (er[k] < 0) continue;
    const double v = (double)strip[(long long)__ldg(pos + er[k]) * si + (long long)ec[k] * st];
    if (!(fabs(v) <= DBL_MAX)) bad = 1;
    buf[0][er[k] * l + ec[k]] = v;
    if (ec[k] == 0) atomicMax(&pkey[0], pivot_key(v, er[k]));
  }
  if (__syncthreads_or(bad)) {
    if (tid == 0) set_status(js, LRA_ENONFINITE);
    return;
  }
  int cur = 0;
  for (int t = 0; t < l; ++t) {
    const double* A = buf[cur];
    if (tid < 32) {
      const unsigned long long key = pkey[t & 1];
      const int p = (key >> 32) != 0ull ? 0x7fffffff - (int)(unsigned)(key & 0xffffffffull) : -1;
      double rp = 0.0;
      if (lane == 0 && p >= 0) rp = 1.0 / A[p * l + t];
      rp = __shfl_sync(0xffffffffu, rp, 0);
      if (p >= 0 && lane < l) rowt[lane] = (lane == t) ? rp : A[p * l + lane] * rp;
      if (lane == 0) {
        p_s = p;
        swaps[t] = p;
        pkey[(t + 1) & 1] = 0ull;
      }
    }
    __syncthreads();
    const int p = p_s;
    if (p < 0) {
      if (tid == 0) set_status(js, LRA_ESINGULAR);
      return;
    }
    double* N = buf[cur ^ 1];
#pragma unroll
    for (int k = 0; k < kInvSmallPer; ++k) {
      const int r = er[k], c = ec[k];
      if (r < 0) continue;
      double v;
      if (r == t) {
        v = rowt[c];
      } else {
        const int rr = (r == p) ? t : r;  // row r after the swap is row rr before it
        const double a = (c == t) ? 0.0 : A[rr * l + c];
        v = fma(-A[rr * l + t], rowt[c], a);
      }
      N[r * l + c] = v;
      if (c == t + 1 && r > t) atomicMax(&pkey[(t + 1) & 1], pivot_key(v, r));
    }
    cur ^= 1;
    __syncthreads();
  }
  if (tid == 0) {
    for (int q = 0; q < l; ++q) at[q] = q;
    for (int t = l - 1; t >= 0; --t) {
      const int p = swaps[t], x = at[t];
      at[t] = at[p];
      at[p] = x;
    }
    for (int q = 0; q < l; ++q) dest[at[q]] = q;
  }
  __syncthreads();
  for (int e = tid; e < ll; e += kInvSmallT) {
    const int r = e / l, c = e - r * l;
    xinv[(size_t)r * l + dest[c]] = split_double(buf[cur][e]);
  }
}

cudaError_t launch_cross_inverse(const float* strip, long long si, long long st, const int* pos,
                                 int l, float2* xinv, JobStatus* js, cudaStream_t stream, bool one_sm) {
  if (l <= kInvSmallL) {
    cross_inverse_small_kernel<<<1, kInvSmallT, 0, stream>>>(strip, si, st, pos, l, xinv, js);
    return cudaGetLastError();
  }
  if (one_sm) {
    const size_t smem = ((size_t)l * l + 2 * kMaxL + 1) * sizeof(double) + (kMaxL + 2) * sizeof(int);
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(cross_inverse_cta_kernel), 227 * 1024);
    if (e) return e;
    cross_inverse_cta_kernel<<<1, kInvCtaT, smem, stream>>>(strip, si, st, pos, l, xinv, js);
    return cudaGetLastError();
  }
  const int w = (l + kInvCS - 1) / kInvCS;
  const size_t smem = ((size_t)l * w + 2 * kMaxL) * sizeof(double) + sizeof(InvPub) +
                      3 * kMaxL * sizeof(int);
  cross_inverse_kernel<<<kInvCS, kInvCT, smem, stream>>>(strip, si, st, pos, l, xinv, js);
  return cudaGetLastError();
}

cudaError_t launch_nucleus(const float* C, const int* I, int l, int k, double rank_tol,
                           double* U, double* sigma, JobStatus* js, cudaStream_t st) {
  const size_t smem = 2 * (size_t)l * l * sizeof(dd) + kMaxL * (sizeof(double) + sizeof(dd)) +
                      sizeof(SvdScratch) + (kMaxL + 2) * sizeof(int);
  const cudaError_t e = smem_optin(reinterpret_cast<const void*>(nucleus_kernel), 227 * 1024);
  if (e != cudaSuccess) return e;
  nucleus_kernel<<<1, kNucThreads, smem, st>>>(C, I, l, k, rank_tol, U, sigma, js);
  return cudaGetLastError();
}

}  // namespace lra
