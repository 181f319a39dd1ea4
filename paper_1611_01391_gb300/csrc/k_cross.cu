// Nucleus of the CUR approximation (Primitive Algorithm, stages 2-3 of
// Section 6.5): the l x l CUR generator X = M[I, J], its SVD, the rank-k
// truncation and U = (X_k)^+.
//
// The SVD (svd_dd.cuh) is QR with column pivoting followed by one-sided
// Jacobi on R^T, in double-float arithmetic.  X is first scaled by a power
// of two so that max |X| lies in [0.5, 1) (exact); sigma and U are scaled
// back.
#include <cfloat>

#include "lra_kernels.h"
#include "lra_internal.cuh"
#include "svd_dd.cuh"

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
  nucleus_from_svd<kNucThreads>(W, Z, sc->perm, l, ke, order, inv2,
                                [&](int e, double v) { U[e] = ldexp(v, -ex); });
}

// X^{-1} of the cross X[a][b] = S[pos[a]][b] of an N x l strip (element
// (i, t) at strip[i*si + t*st]), by in-place Gauss-Jordan elimination with
// partial pivoting in FP64 on one CTA (Golub & Van Loan, 3.4; l^3 FMAs
// against 1.5 l^3 for elimination on [X | I]).  Step t: the pivot is the
// largest |A[r][t]|, r >= t (smallest r on ties), rows t and p are swapped,
// column t is replaced by the column of the inverse it produces, and every
// other row is updated.  The row swaps are undone as column swaps at the
// end.  A zero pivot sets LRA_ESINGULAR, a non-finite entry LRA_ENONFINITE.
constexpr int kInvThreads = 512;

__global__ void __launch_bounds__(kInvThreads, 1)
cross_inverse_kernel(const float* __restrict__ strip, long long si, long long st,
                     const int* __restrict__ pos, int l, double* __restrict__ xinv, JobStatus* js) {
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
        const unsigned long long k =
            (unsigned long long)__double_as_longlong(A[(size_t)r * l + t]) & 0x7fffffffffffffffull;
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
  for (int e = tid; e < l * l; e += nthr) xinv[e] = A[e];
}

cudaError_t launch_cross_inverse(const float* strip, long long si, long long st, const int* pos,
                                 int l, double* xinv, JobStatus* js, cudaStream_t stream) {
  const size_t smem = ((size_t)l * l + 2 * kMaxL + 1) * sizeof(double) + (kMaxL + 2) * sizeof(int);
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(cross_inverse_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  cross_inverse_kernel<<<1, kInvThreads, smem, stream>>>(strip, si, st, pos, l, xinv, js);
  return cudaGetLastError();
}

cudaError_t launch_nucleus(const float* C, const int* I, int l, int k, double rank_tol,
                           double* U, double* sigma, JobStatus* js, cudaStream_t st) {
  const size_t smem = 2 * (size_t)l * l * sizeof(dd) + kMaxL * (sizeof(double) + sizeof(dd)) +
                      sizeof(SvdScratch) + (kMaxL + 2) * sizeof(int);
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(nucleus_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  nucleus_kernel<<<1, kNucThreads, smem, st>>>(C, I, l, k, rank_tol, U, sigma, js);
  return cudaGetLastError();
}

}  // namespace lra
