// Strip gathers of the C-A iteration (Section 6.5): the vertical strip
// C = M[:, J] (m x l) and the horizontal strip R = M[I, :] (l x n), both FP32
// row-major.  For stored matrices these are memory gathers; for generators
// every entry is evaluated on the fly from the point coordinates.
#include "lra_kernels.h"
#include "lra_internal.cuh"
#include "tma.cuh"

#include <algorithm>

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
                                                          const JobStatus* js, int vec_ok, int skip_on_stop) {
  if (js->status != LRA_OK || (skip_on_stop && js->stop)) return;
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

// ---------------------------------------------------------------------------
// Stored FP32 M: C = M[:, J] with tiles moved by the Tensor Memory
// Accelerator.  A column gather from a row-major matrix reads one 32-byte
// sector per entry (unless columns share a sector), so the DRAM floor is
// m x (distinct sectors of J) x 32 bytes.  Each CTA
//   1. sorts J's sectors (j >> 3) and keeps each distinct one once: columns
//      that share a sector share its load;
//   2. streams row tiles of kColsTmaRows rows: per distinct sector one TMA box
//      of 8 FP32 x kColsTmaRows rows (the sector column of the tile), into a
//      ring of `stages` shared-memory buffers guarded by mbarriers.  The
//      tensor map asks for 64-byte L2 promotion: on GB300 a scattered
//      32-byte read costs 64 bytes of DRAM traffic with it, and 128 bytes
//      (a whole line) without it, for TMA boxes and plain loads alike
//      (measured on the stored 32768^2 matrix with l = 96: 195 MB against
//      390 MB per gather, 99.6 MB being the 32-byte sector floor);
//   3. transposes through shared memory: the tile's rows of C, contiguous in
//      C, are written with 16-byte stores, C[r][t] = box(slot[t])[r][J[t] & 7].
// Grid: one persistent CTA per SM over the row tiles.  Every mbarrier wait
// is bounded (2 s, then LRA_ETIMEOUT); the CTA waits for its copies in
// flight before it returns.
// ---------------------------------------------------------------------------

constexpr int kColsTmaRows = 16;       // rows per tile
constexpr int kColsTmaThreads = 256;
constexpr int kColsTmaMaxStages = 8;
constexpr int kColsTmaSmemBudget = 192 * 1024;

__global__ void __launch_bounds__(kColsTmaThreads, 1)
gather_cols_tma_kernel(const __grid_constant__ CUtensorMap tm, const int* __restrict__ J, int l, long long m,
                       float* __restrict__ C, JobStatus* js, int skip_on_stop, int stages) {
  if (js->status != LRA_OK || (skip_on_stop && js->stop)) return;
  extern __shared__ __align__(128) unsigned char csm[];
  __shared__ uint64_t full[kColsTmaMaxStages];
  __shared__ int sec[kMaxL], first[kMaxL], slot[kMaxL], off[kMaxL], secs[kMaxL];
  __shared__ int nsec_s;
  __shared__ int err;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* ring = reinterpret_cast<float*>(csm);
  // ---- distinct sectors of J, in increasing order
  if (tid == 0) {
    nsec_s = 0;
    err = 0;
  }
  for (int t = tid; t < l; t += kColsTmaThreads) {
    const int j = __ldg(J + t);
    sec[t] = j >> 3;
    off[t] = j & 7;
  }
  __syncthreads();
  for (int t = tid; t < l; t += kColsTmaThreads) {
    int f = 1;
    for (int u = 0; u < t; ++u) f &= (sec[u] != sec[t]);
    first[t] = f;
    if (f) atomicAdd(&nsec_s, 1);
  }
  __syncthreads();
  for (int t = tid; t < l; t += kColsTmaThreads) {
    int rank = 0;
    for (int u = 0; u < l; ++u) rank += (first[u] && sec[u] < sec[t]);
    slot[t] = rank;
    if (first[t]) secs[rank] = sec[t];
  }
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) tma::mbar_init(&full[s], 1);
    tma::mbar_fence_init();
  }
  __syncthreads();
  const int nsec = nsec_s;
  const int stage_floats = nsec * kColsTmaRows * 8;
  const uint32_t stage_bytes = (uint32_t)stage_floats * 4u;
  const long long ntiles = (m + kColsTmaRows - 1) / kColsTmaRows;
  const long long G = gridDim.x;
  // warp 0 fills stage `it % stages` with tile blockIdx.x + it G
  auto issue = [&](long long it) {
    const long long tile = blockIdx.x + it * G;
    if (tile >= ntiles) return;
    const int s = (int)(it % stages);
    if (lane == 0) tma::mbar_expect_tx(&full[s], stage_bytes);
    __syncwarp();
    float* dst = ring + (size_t)s * stage_floats;
    for (int k = lane; k < nsec; k += 32)
      tma::load_2d(dst + (size_t)k * kColsTmaRows * 8, &tm, secs[k] * 8, (int)(tile * kColsTmaRows), &full[s]);
  };
  if (warp == 0)
    for (int it = 0; it < stages; ++it) issue(it);
  const bool vec = (l & 3) == 0;
  long long it = 0;
  for (;; ++it) {
    const long long tile = blockIdx.x + it * G;
    if (tile >= ntiles) break;
    const int s = (int)(it % stages);
    const bool ok = tma::mbar_wait(&full[s], (uint32_t)((it / stages) & 1), &err);
    if (__syncthreads_or(!ok)) break;   // the whole CTA leaves together
    const float* st = ring + (size_t)s * stage_floats;
    const long long r0 = tile * kColsTmaRows;
    const int rows = (int)min((long long)kColsTmaRows, m - r0);
    const int count = rows * l;
    float* out = C + r0 * l;
    if (vec) {
      for (int e4 = tid * 4; e4 < count; e4 += kColsTmaThreads * 4) {
        float v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int e = e4 + c;
          const int r = e / l, t = e - r * l;
          v[c] = st[(slot[t] * kColsTmaRows + r) * 8 + off[t]];
        }
        *reinterpret_cast<float4*>(out + e4) = make_float4(v[0], v[1], v[2], v[3]);
      }
    } else {
      for (int e = tid; e < count; e += kColsTmaThreads) {
        const int r = e / l, t = e - r * l;
        out[e] = st[(slot[t] * kColsTmaRows + r) * 8 + off[t]];
      }
    }
    __syncthreads();   // every thread is done with stage s
    if (warp == 0) issue(it + stages);
  }
  // copies still in flight (an error ended the loop early): let them land
  if (warp == 0 && lane == 0) {
    for (long long k = it; k < it + stages; ++k) {
      if (blockIdx.x + k * G >= ntiles) break;
      tma::mbar_drain(&full[k % stages], (uint32_t)((k / stages) & 1));
    }
    if (err) set_status(js, LRA_ETIMEOUT);
  }
}

bool make_cols_map(TmaMap* map, const float* a, long long m, long long n, long long lda) {
  static_assert(sizeof(TmaMap) == sizeof(CUtensorMap), "TmaMap holds a CUtensorMap");
  if ((reinterpret_cast<uintptr_t>(a) & 15) != 0 || (lda & 3) != 0) return false;
  return tma::make_map_2d(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a, (uint64_t)n,
                          (uint64_t)m, (uint64_t)lda * 4, 8, kColsTmaRows, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_64B);
}

cudaError_t launch_gather_cols_tma(const TmaMap& map, const int* J, int l, long long m, float* C, JobStatus* js,
                                   int skip_on_stop, int sms, cudaStream_t st) {
  const size_t stage_max = (size_t)l * kColsTmaRows * 8 * sizeof(float);   // at most l distinct sectors
  int stages = (int)std::min<size_t>(kColsTmaMaxStages, kColsTmaSmemBudget / stage_max);
  if (stages < 2) stages = 2;
  const size_t smem = (size_t)stages * stage_max;
  cudaError_t e = smem_optin(reinterpret_cast<const void*>(gather_cols_tma_kernel), (int)smem);
  if (e) return e;
  const long long ntiles = (m + kColsTmaRows - 1) / kColsTmaRows;
  const int grid = (int)std::max<long long>(1, std::min<long long>(ntiles, sms));
  gather_cols_tma_kernel<<<grid, kColsTmaThreads, smem, st>>>(*reinterpret_cast<const CUtensorMap*>(&map), J, l,
                                                              m, C, js, skip_on_stop, stages);
  return cudaGetLastError();
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
  LRA_DISPATCH_KIND_ALL(s.kind, (gather_cols_kernel<K><<<grid, 256, 0, st>>>(s, J, l, C, js, skip_on_stop)));
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const SourceDev& s, const int* I, int l, float* R,
                               const JobStatus* js, int sms, cudaStream_t st, int skip_on_stop) {
  const long long nq = (s.n + 3) / 4;
  const int grid = grid_for(nq * l, 256 * 2, sms);
  int vec_ok = (s.n % 4 == 0) && ((reinterpret_cast<uintptr_t>(R) & 15) == 0);
  if (s.kind == LRA_DENSE_F32)
    vec_ok = vec_ok && (s.lda % 4 == 0) && ((reinterpret_cast<uintptr_t>(s.a) & 15) == 0);
  LRA_DISPATCH_KIND_ALL(s.kind, (gather_rows_kernel<K><<<grid, 256, 0, st>>>(s, I, l, R, js, vec_ok, skip_on_stop)));
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
  LRA_DISPATCH_KIND_ALL(s.kind, (e = cudaLaunchKernel(reinterpret_cast<const void*>(gather_entries_kernel<K>),
                                                   dim3(grid), dim3(256), args, 0, st)));
  return e;
}

}  // namespace lra
