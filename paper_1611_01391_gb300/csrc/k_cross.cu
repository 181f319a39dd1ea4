// Nucleus of the CUR approximation (Primitive Algorithm, stages 2-3 of
// Section 6.5): the l x l CUR generator X = M[I, J], its SVD X = P S Q^T, the
// rank-k truncation and U = Q_k S_k^{-1} P_k^T.
//
// The SVD is the one-sided Jacobi method of Hestenes (1958), with the
// rotation of Rutishauser's symmetric Jacobi step (Golub & Van Loan,
// Algorithm 8.5.1) applied to column pairs: the columns of W = X V are
// orthogonalised in place, sigma_b = ||W[:, b]||, P[:, b] = W[:, b] / sigma_b
// and Q = V.  Pairs are visited in round-robin (circle) order so that the
// l/2 rotations of a round are independent; one warp handles one pair.
// Everything is FP64.
#include <cfloat>

#include "lra_kernels.h"
#include "lra_internal.cuh"

namespace lra {

constexpr int kNucThreads = 512;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__global__ void __launch_bounds__(kNucThreads, 1)
nucleus_kernel(const float* __restrict__ C, const int* __restrict__ I, int l, int k,
               double rank_tol, double* __restrict__ U, double* __restrict__ sigma_out,
               JobStatus* js) {
  if (js->status != LRA_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* W = reinterpret_cast<double*>(smem_raw);  // column b at W + b*l
  double* V = W + (size_t)l * l;                     // column b at V + b*l
  double* sig = V + (size_t)l * l;                   // l
  double* sig_sorted = sig + kMaxL;                  // l
  int* order = reinterpret_cast<int*>(sig_sorted + kMaxL);  // l: order[rank] = column
  int* rotated = order + kMaxL;
  int* keff_s = rotated + 1;

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;

  for (int e = tid; e < l * l; e += nthr) {
    const int a = e / l, b = e - a * l;             // X[a][b] = C[I[a]][b]
    W[(size_t)b * l + a] = (double)C[(size_t)__ldg(I + a) * l + b];
    V[(size_t)b * l + a] = (a == b) ? 1.0 : 0.0;
  }
  __syncthreads();

  // Pairs of a round are handled by groups of 8 lanes (4 pairs per warp), so
  // one FP64 instruction serves four rotations; the FP64 pipe is the limit.
  const int np = (l + 1) & ~1;                      // players incl. a dummy when l is odd
  const double tol = (double)l * DBL_EPSILON;
  const int gl = lane & 7;
  const int ngroups = nwarps * 4;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) *rotated = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int base = warp * 4; base < np / 2; base += ngroups) {
        const int slot = base + (lane >> 3);
        const int x0 = slot, x1 = np - 1 - slot;
        int p = (x0 == 0) ? 0 : ((x0 - 1 + round) % (np - 1)) + 1;
        int q = (x1 == 0) ? 0 : ((x1 - 1 + round) % (np - 1)) + 1;
        if (p > q) { const int t = p; p = q; q = t; }
        const bool act = slot < np / 2 && q < l;
        double* wp = W + (size_t)p * l;
        double* wq = W + (size_t)q * l;
        double al = 0.0, be = 0.0, ga = 0.0;
        if (act)
          for (int a = gl; a < l; a += 8) {
            const double u = wp[a], v = wq[a];
            al = fma(u, u, al);
            be = fma(v, v, be);
            ga = fma(u, v, ga);
          }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, off);
          be += __shfl_xor_sync(0xffffffffu, be, off);
          ga += __shfl_xor_sync(0xffffffffu, ga, off);
        }
        if (!act || al == 0.0 || be == 0.0 || ga * ga <= tol * tol * al * be) continue;
        // Rotation tangent t from the symmetric Jacobi step; an approximate t
        // (FP32) still gives an exactly orthogonal rotation because c and s
        // are formed from the same t in FP64: c = (1 + t^2)^{-1/2}, s = c t.
        const double zeta = (be - al) / (2.0 * ga);
        const float zf = (float)zeta;
        // |zeta| > 1e18 (columns of very different norms): t = 1/(2 zeta) to
        // FP32 accuracy, and zeta^2 would overflow FP32.
        const float tf = fabsf(zf) > 1e18f
                             ? 0.5f / zf
                             : (zf >= 0.0f ? 1.0f : -1.0f) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f)));
        const double t = (double)tf;
        const double x = fma(t, t, 1.0);
        double y = (double)rsqrtf((float)x);          // Newton-Raphson for x^{-1/2}
        y = y * fma(-0.5 * x * y, y, 1.5);
        y = y * fma(-0.5 * x * y, y, 1.5);
        const double c = y, s = y * t;
        double* vp = V + (size_t)p * l;
        double* vq = V + (size_t)q * l;
        for (int a = gl; a < l; a += 8) {
          const double u = wp[a], v = wq[a];
          wp[a] = fma(c, u, -s * v);
          wq[a] = fma(s, u, c * v);
          const double xx = vp[a], yy = vq[a];
          vp[a] = fma(c, xx, -s * yy);
          vq[a] = fma(s, xx, c * yy);
        }
        if (gl == 0) *rotated = 1;
      }
      __syncthreads();
    }
    if (*rotated == 0) break;
    __syncthreads();
  }

  // singular values, descending order (ties: smaller column first)
  for (int b = warp; b < l; b += nwarps) {
    double ss = 0.0;
    for (int a = lane; a < l; a += 32) ss = fma(W[(size_t)b * l + a], W[(size_t)b * l + a], ss);
    ss = warp_sum(ss);
    if (lane == 0) sig[b] = sqrt(ss);
  }
  __syncthreads();
  for (int b = tid; b < l; b += nthr) {
    int rank = 0;
    for (int c = 0; c < l; ++c)
      rank += (sig[c] > sig[b]) || (sig[c] == sig[b] && c < b);
    order[rank] = b;
    sig_sorted[rank] = sig[b];
  }
  __syncthreads();
  if (tid == 0) {
    const double s1 = sig_sorted[0];
    int ke = 0;
    if (s1 > 0.0)
      while (ke < k && ke < l && sig_sorted[ke] > rank_tol * s1) ++ke;
    *keff_s = ke;
    js->k_eff = ke;
    js->sigma_max = s1;
  }
  __syncthreads();
  const int ke = *keff_s;
  for (int b = tid; b < l; b += nthr) sigma_out[b] = sig_sorted[b];
  // U[p][q] = sum_r V[b_r][p] * W[b_r][q] / sigma_{b_r}^2  (P = W / sigma)
  for (int e = tid; e < l * l; e += nthr) {
    const int p = e / l, q = e - p * l;
    double acc = 0.0;
    for (int r = 0; r < ke; ++r) {
      const int b = order[r];
      const double s = sig[b];
      acc = fma(V[(size_t)b * l + p] / s, W[(size_t)b * l + q] / s, acc);
    }
    U[e] = acc;
  }
}

// X^{-1} of the cross X[a][b] = S[pos[a]][b] of an N x l strip (element
// (i, t) at strip[i*si + t*st]), by Gauss-Jordan elimination with partial
// pivoting on [X | I] in FP64 (one CTA).  Output row-major.  A zero pivot
// sets LRA_ESINGULAR, a non-finite entry LRA_ENONFINITE.
constexpr int kInvThreads = 512;

__global__ void __launch_bounds__(kInvThreads, 1)
cross_inverse_kernel(const float* __restrict__ strip, long long si, long long st,
                     const int* __restrict__ pos, int l, double* __restrict__ xinv, JobStatus* js) {
  if (js->status != LRA_OK || js->stop) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = 2 * l;
  double* A = reinterpret_cast<double*>(smem_raw);  // l x 2l, row-major
  double* f = A + (size_t)l * w;                    // column t before elimination
  double* recip = f + kMaxL;                        // 1 / pivot of the current step
  int* piv_row = reinterpret_cast<int*>(recip + 1);
  int* bad = piv_row + 1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) *bad = 0;
  __syncthreads();
  for (int e = tid; e < l * w; e += nthr) {
    const int a = e / w, b = e - a * w;
    double v;
    if (b < l) {
      v = (double)strip[(long long)__ldg(pos + a) * si + (long long)b * st];
      if (!(fabs(v) <= DBL_MAX)) *bad = 1;
    } else {
      v = (b - l == a) ? 1.0 : 0.0;
    }
    A[e] = v;
  }
  __syncthreads();
  if (*bad) {
    if (tid == 0) set_status(js, LRA_ENONFINITE);
    return;
  }
  // Columns < t of the left half are already unit columns, so step t only
  // touches columns t..2l-1 (width wt).  Magnitudes are compared on their
  // IEEE bit patterns (integer compares), and row t is scaled by the FP64
  // reciprocal of the pivot.
  for (int t = 0; t < l; ++t) {
    if (tid < 32) {  // pivot: largest |A[r][t]|, r >= t (smallest r on ties)
      unsigned long long best = 0ull;
      int br = l;
      for (int r = t + tid; r < l; r += 32) {
        const unsigned long long k =
            (unsigned long long)__double_as_longlong(A[(size_t)r * w + t]) & 0x7fffffffffffffffull;
        if (br == l || k > best) { best = k; br = r; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, off);
        const int orr = __shfl_down_sync(0xffffffffu, br, off);
        if (orr < l && (br == l || ob > best || (ob == best && orr < br))) { best = ob; br = orr; }
      }
      if (tid == 0) {
        *piv_row = (best != 0ull && br < l) ? br : -1;
        // one FP64 division for the whole step (all threads dividing would
        // occupy the FP64 pipe for thousands of cycles)
        if (br < l && best != 0ull) *recip = 1.0 / A[(size_t)br * w + t];
      }
    }
    __syncthreads();
    const int p = *piv_row;
    if (p < 0) {
      if (tid == 0) set_status(js, LRA_ESINGULAR);
      return;
    }
    if (p != t)
      for (int c = t + tid; c < w; c += nthr) {
        const double x = A[(size_t)t * w + c];
        A[(size_t)t * w + c] = A[(size_t)p * w + c];
        A[(size_t)p * w + c] = x;
      }
    __syncthreads();
    const double rp = *recip;
    for (int c = t + tid; c < w; c += nthr) A[(size_t)t * w + c] *= rp;
    for (int r = tid; r < l; r += nthr) f[r] = (r == t) ? 0.0 : A[(size_t)r * w + t];
    __syncthreads();
    const int wt = w - t;
    for (int e = tid; e < l * wt; e += nthr) {
      const int r = e / wt, c = t + (e - r * wt);
      if (r != t) A[(size_t)r * w + c] = fma(-f[r], A[(size_t)t * w + c], A[(size_t)r * w + c]);
    }
    __syncthreads();
  }
  for (int e = tid; e < l * l; e += nthr) {
    const int a = e / l, b = e - a * l;
    xinv[e] = A[(size_t)a * w + l + b];
  }
}

cudaError_t launch_cross_inverse(const float* strip, long long si, long long st, const int* pos,
                                 int l, double* xinv, JobStatus* js, cudaStream_t stream) {
  const size_t smem = ((size_t)l * 2 * l + kMaxL + 1) * sizeof(double) + 2 * sizeof(int);
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
  const size_t smem = (2 * (size_t)l * l + 2 * kMaxL) * sizeof(double) + (kMaxL + 2) * sizeof(int);
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
