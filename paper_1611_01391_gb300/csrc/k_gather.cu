// Strip gathers of the C-A iteration (Section 6.5): the vertical strip
// C = M[:, J] (m x l) and the horizontal strip R = M[I, :] (l x n), both FP32
// row-major.  For stored matrices these are memory gathers; for generators
// every entry is evaluated on the fly from the point coordinates.
#include "lra_kernels.h"
#include "lra_internal.cuh"

namespace lra {

// C[i*l + t] = M(i, J[t]).  Consecutive threads walk a row of C, so the
// stores are contiguous; for a stored M each row touches l scattered sectors.
template <int KIND>
__global__ void __launch_bounds__(256) gather_cols_kernel(SourceDev s, const int* __restrict__ J,
                                                          int l, float* __restrict__ C,
                                                          const JobStatus* js, int skip_on_stop) {
  if (js->status != LRA_OK || (skip_on_stop && js->stop)) return;
  __shared__ int Js[kMaxL];
  for (int t = threadIdx.x; t < l; t += blockDim.x) Js[t] = J[t];
  __syncthreads();
  const long long total = s.m * (long long)l;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (total < (1LL << 31)) {
    // 32-bit index arithmetic: a 64-bit division per entry would cost more
    // than the entry
    const unsigned int tot = (unsigned int)total, str = (unsigned int)stride, ul = (unsigned int)l;
    for (unsigned int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += str) {
      const unsigned int i = e / ul;
      C[e] = entry<KIND>(s, (long long)i, Js[e - i * ul]);
    }
    return;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += stride) {
    const long long i = e / l;
    const int t = (int)(e - i * l);
    C[e] = entry<KIND>(s, i, Js[t]);
  }
}

// R[t*n + j] = M(I[t], j).  Each thread produces four consecutive entries of
// one row; a stored FP32 row with 16-byte alignment is read with float4 loads.
template <int KIND>
__global__ void __launch_bounds__(256) gather_rows_kernel(SourceDev s, const int* __restrict__ I,
                                                          int l, float* __restrict__ R,
                                                          const JobStatus* js, int vec_ok) {
  if (js->status != LRA_OK || js->stop) return;
  const long long n = s.n;
  const long long nq = (n + 3) / 4;
  const long long total = nq * l;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const bool small = total < (1LL << 31) && nq < (1LL << 31);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += stride) {
    // 32-bit division where it fits (a 64-bit one costs more than the entries)
    const int t = small ? (int)((unsigned int)e / (unsigned int)nq) : (int)(e / nq);
    const long long j0 = (e - (long long)t * nq) * 4;
    const long long i = __ldg(I + t);
    float v[4];
    if constexpr (KIND == LRA_DENSE_F32) {
      const float* row = static_cast<const float*>(s.a) + i * s.lda;
      if (vec_ok && j0 + 3 < n) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(row + j0));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = (j0 + c < n) ? __ldg(row + j0 + c) : 0.0f;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = (j0 + c < n) ? entry<KIND>(s, i, j0 + c) : 0.0f;
    }
    float* out = R + (long long)t * n + j0;
    if (vec_ok && j0 + 3 < n) {
      *reinterpret_cast<float4*>(out) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
      for (int c = 0; c < 4 && j0 + c < n; ++c) out[c] = v[c];
    }
  }
}

// out[a*s + b] = M(rows[a], cols[b]): the FP32 entries every other kernel
// of the library sees.  An index outside M gives NaN and no access.
template <int KIND>
__global__ void __launch_bounds__(256) gather_entries_kernel(SourceDev src, const int* __restrict__ rows,
                                                             long long q, const int* __restrict__ cols,
                                                             long long s, float* __restrict__ out) {
  const long long total = q * s;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long a = e / s, b = e - a * s;
    const long long i = __ldg(rows + a), j = __ldg(cols + b);
    out[e] = (i >= 0 && i < src.m && j >= 0 && j < src.n) ? entry<KIND>(src, i, j) : __int_as_float(0x7fc00000);
  }
}

static int grid_for(long long work, int per_block, int sms) {
  long long g = (work + per_block - 1) / per_block;
  const long long cap = (long long)sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_gather_cols(const SourceDev& s, const int* J, int l, float* C,
                               const JobStatus* js, int skip_on_stop, int sms,
                               cudaStream_t st) {
  const int grid = grid_for(s.m * (long long)l, 256 * 4, sms);
  LRA_DISPATCH_KIND(s.kind, (gather_cols_kernel<K><<<grid, 256, 0, st>>>(s, J, l, C, js, skip_on_stop)));
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const SourceDev& s, const int* I, int l, float* R,
                               const JobStatus* js, int sms, cudaStream_t st) {
  const long long nq = (s.n + 3) / 4;
  const int grid = grid_for(nq * l, 256 * 2, sms);
  int vec_ok = (s.n % 4 == 0) && ((reinterpret_cast<uintptr_t>(R) & 15) == 0);
  if (s.kind == LRA_DENSE_F32)
    vec_ok = vec_ok && (s.lda % 4 == 0) && ((reinterpret_cast<uintptr_t>(s.a) & 15) == 0);
  LRA_DISPATCH_KIND(s.kind, (gather_rows_kernel<K><<<grid, 256, 0, st>>>(s, I, l, R, js, vec_ok)));
  return cudaGetLastError();
}

cudaError_t launch_gather_entries(const SourceDev& s, const int* rows, long long q, const int* cols,
                                  long long sN, float* out, cudaStream_t st) {
  const int grid = grid_for(q * sN, 256 * 4, 152);
  cudaError_t e = cudaSuccess;
  SourceDev sd = s;
  void* args[] = {&sd, const_cast<int**>(&rows), &q, const_cast<int**>(&cols), &sN, &out};
  // launched through its own return code: the runtime's last-error state is
  // left as the caller had it
  LRA_DISPATCH_KIND(s.kind, (e = cudaLaunchKernel(reinterpret_cast<const void*>(gather_entries_kernel<K>),
                                                   dim3(grid), dim3(256), args, 0, st)));
  return e;
}

}  // namespace lra
