// A posteriori error estimate of Appendix F: the error matrix E = M - C U R
// restricted to a random q x s submatrix (rows x cols), with
//   rel = sqrt(sum E^2 / sum M^2),  mu_K = (1/K) sum E,
//   sigma_K^2 = (1/K) sum (E - mu_K)^2,  K = q s.
// (C U) is formed for the sampled rows in FP64 and stored as an unevaluated
// FP32 pair hi + lo.  The length-l products (C U) R run in FP32 with the
// compensated dot product "Dot2" of Ogita, Rump & Oishi (SIAM J. Sci. Comput.
// 26(6), 2005): TwoProduct through an FMA and Knuth's TwoSum, which returns the
// dot product as accurately as if it were computed in twice the working
// precision.  Plain FP32 products would carry a rounding error of about
// sqrt(l) * 6e-8 * |M|, the size of the error being estimated on smooth
// generated matrices.  All sums over the sample are FP64, reduced in a fixed
// order, so the estimate is reproducible run to run.
#include "lra_kernels.h"
#include "lra_internal.cuh"

namespace lra {

constexpr int kTile = 32;

// cu = sum_p C[rows[a]][p] * U[p][t] in FP64, stored as CUq[a][t] = hi,
// CUq[q*l + a*l + t] = lo with hi = fp32(cu), lo = fp32(cu - hi).
__global__ void __launch_bounds__(256) cu_rows_kernel(const float* __restrict__ C,
                                                      const int* __restrict__ rows, int q, int l,
                                                      const double* __restrict__ U,
                                                      float* __restrict__ CUq,
                                                      const JobStatus* js) {
  if (js->status != LRA_OK) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= q * l) return;
  const int a = e / l, t = e - a * l;
  const float* crow = C + (size_t)__ldg(rows + a) * l;
  double acc = 0.0;
  for (int p = 0; p < l; ++p) acc = fma((double)__ldg(crow + p), __ldg(U + (size_t)p * l + t), acc);
  const float hi = (float)acc;
  CUq[e] = hi;
  CUq[(size_t)q * l + e] = (float)(acc - (double)hi);
}

// Error-free transformations (Knuth TwoSum; TwoProduct via FMA).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ void dot2_step(float x, float y, float& p, float& c) {
  const float h = __fmul_rn(x, y);
  const float r = fmaf(x, y, -h);
  float q;
  two_sum(p, h, p, q);
  c = __fadd_rn(c, __fadd_rn(q, r));
}

template <int KIND>
__global__ void __launch_bounds__(256) resid_tile_kernel(SourceDev s, const int* __restrict__ rows,
                                                         int q, const int* __restrict__ cols,
                                                         int sN, int l, const float* __restrict__ CUq,
                                                         const float* __restrict__ R,
                                                         double* __restrict__ partials,
                                                         const JobStatus* js) {
  if (js->status != LRA_OK) return;
  __shared__ float cu_t[kTile][kMaxL + 1];
  __shared__ float cl_t[kTile][kMaxL + 1];
  __shared__ float r_t[kMaxL][kTile + 1];
  __shared__ int ri[kTile], ci[kTile];
  __shared__ double red[3][8];
  const int a0 = blockIdx.y * kTile, b0 = blockIdx.x * kTile;
  const int tid = threadIdx.x;
  if (tid < kTile) {
    ri[tid] = (a0 + tid < q) ? __ldg(rows + a0 + tid) : -1;
    ci[tid] = (b0 + tid < sN) ? __ldg(cols + b0 + tid) : -1;
  }
  __syncthreads();
  for (int e = tid; e < kTile * l; e += blockDim.x) {
    const int a = e / l, t = e - a * l;
    cu_t[a][t] = (a0 + a < q) ? CUq[(size_t)(a0 + a) * l + t] : 0.0f;
    cl_t[a][t] = (a0 + a < q) ? CUq[(size_t)q * l + (size_t)(a0 + a) * l + t] : 0.0f;
  }
  for (int e = tid; e < kTile * l; e += blockDim.x) {
    const int t = e / kTile, b = e - t * kTile;
    r_t[t][b] = (ci[b] >= 0) ? __ldg(R + (size_t)t * s.n + ci[b]) : 0.0f;
  }
  __syncthreads();
  double sse = 0.0, ssa = 0.0, se = 0.0;
  for (int e = tid; e < kTile * kTile; e += blockDim.x) {
    const int a = e / kTile, b = e - a * kTile;
    if (ri[a] < 0 || ci[b] < 0) continue;
    float p = 0.0f, c = 0.0f;
    for (int t = 0; t < l; ++t) {
      const float rv = r_t[t][b];
      dot2_step(cu_t[a][t], rv, p, c);
      dot2_step(cl_t[a][t], rv, p, c);
    }
    const float m = entry<KIND>(s, ri[a], ci[b]);
    const double ev = ((double)m - (double)p) - (double)c;
    sse = fma(ev, ev, sse);
    ssa = fma((double)m, (double)m, ssa);
    se += ev;
  }
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sse += __shfl_xor_sync(0xffffffffu, sse, off);
    ssa += __shfl_xor_sync(0xffffffffu, ssa, off);
    se += __shfl_xor_sync(0xffffffffu, se, off);
  }
  if (lane == 0) {
    red[0][warp] = sse;
    red[1][warp] = ssa;
    red[2][warp] = se;
  }
  __syncthreads();
  if (tid < 3) {
    double acc = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += red[tid][w];
    partials[(size_t)(blockIdx.y * gridDim.x + blockIdx.x) * 3 + tid] = acc;
  }
}

__global__ void __launch_bounds__(256) resid_final_kernel(const double* __restrict__ partials,
                                                          int nblocks, long long K, JobStatus* js) {
  if (js->status != LRA_OK) return;
  __shared__ double red[3][256];
  const int tid = threadIdx.x;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int b = tid; b < nblocks; b += blockDim.x)
    for (int c = 0; c < 3; ++c) acc[c] += partials[(size_t)b * 3 + c];
  for (int c = 0; c < 3; ++c) red[c][tid] = acc[c];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int c = 0; c < 3; ++c) red[c][tid] += red[c][tid + w];
    __syncthreads();
  }
  if (tid == 0) {
    const double sse = red[0][0], ssa = red[1][0], se = red[2][0];
    const double mu = se / (double)K;
    js->est_sse = sse;
    js->est_ssa = ssa;
    js->est_rel = ssa > 0.0 ? sqrt(sse / ssa) : INFINITY;
    js->est_mu = mu;
    js->est_var = sse / (double)K - mu * mu;
  }
}

int sampled_residual_partials(int q, int sN) {
  return ((q + kTile - 1) / kTile) * ((sN + kTile - 1) / kTile);
}

cudaError_t launch_sampled_residual(const SourceDev& s, const int* rows, int q, const int* cols,
                                    int sN, int l, const float* C, const double* U, const float* R,
                                    float* CUq, double* partials, int max_partials, JobStatus* js,
                                    cudaStream_t st) {
  const int nb = sampled_residual_partials(q, sN);
  if (nb > max_partials) return cudaErrorInvalidValue;
  cu_rows_kernel<<<(q * l + 255) / 256, 256, 0, st>>>(C, rows, q, l, U, CUq, js);
  dim3 grid((sN + kTile - 1) / kTile, (q + kTile - 1) / kTile);
  LRA_DISPATCH_KIND_ALL(s.kind, (resid_tile_kernel<K><<<grid, 256, 0, st>>>(s, rows, q, cols, sN, l, CUq,
                                                                         R, partials, js)));
  resid_final_kernel<<<1, 256, 0, st>>>(partials, nb, (long long)q * sN, js);
  return cudaGetLastError();
}

__global__ void tol_check_kernel(JobStatus* js, double tol) {
  if (js->status == LRA_OK && js->est_rel <= tol) js->stop = 1;
}

cudaError_t launch_tol_check(JobStatus* js, double tol, cudaStream_t st) {
  tol_check_kernel<<<1, 1, 0, st>>>(js, tol);
  return cudaGetLastError();
}

}  // namespace lra
