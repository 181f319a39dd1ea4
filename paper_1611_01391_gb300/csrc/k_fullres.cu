// Full residual ||M - C U R||_F / ||M||_F of a CUR approximation of a stored
// FP32 matrix M on the tcgen05 tensor cores.  The paper avoids this check
// because it reads all m n entries (Appendix F explains the sampled
// alternative); it is the reference against which the rank-k error bound of
// Lemma 2.3 (letrnc) is compared.
//
// Method:
//   P = C U (m x l) is formed with a compensated FP32 dot product (Dot2 of
//   Ogita, Rump & Oishi on U's FP32 high part; the products with the low
//   part, 2^-24 of the sum, go into the compensation term), so P carries
//   about twice FP32 precision even when U has large entries.  Each row of P and each
//   column of R is scaled by a power of two into the FP16 range and split as
//       x = hi + lo * 2^-11,   hi = fp16(x),  lo = fp16((x - hi) * 2^11),
//   which keeps about 22 significant bits.  The product P R is then
//       D = Phi Rhi + 2^-11 (Phi Rlo + Plo Rhi)   (the Plo Rlo term, 2^-22
//   relative, is dropped), accumulated in FP32 in tensor memory by
//   tcgen05.mma kind::f16 (M = 128, N = 64, K = 16).  A plain FP32 or
//   split-BF16 product would carry errors of 1e-5 |M| or more, the size of
//   the residual being measured (1e-4 for the stored 32768^2 case).
//   The epilogue subtracts D from the TMA-loaded tile of M, squares and sums
//   in FP32 per tile and in FP64 across tiles; CUR itself is never written.
//
// Kernel structure (one CTA of 256 threads per SM, persistent):
//   warp 0 (one lane): TMA producer: P tiles once per work item, then per
//                      column tile the R^T tiles and the FP32 tile of M into a
//                      2-stage ring (128B-swizzled, as the MMA and the
//                      epilogue read them).
//   warp 1:            tensor-memory allocation (256 columns: two buffers of
//                      [D_hi | D_lo]) and, from one lane, the MMA issue.
//   warps 4..7:        epilogue: tcgen05.ld of D (lane = row), float4 reads
//                      of M from the swizzled stage, FP32 error, FP64 sums.
// Every mbarrier wait is bounded (2 s); a timeout sets LRA_ETIMEOUT and all
// roles leave their loops.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "lra_internal.cuh"
#include "lra_kernels.h"
#include "tma.cuh"

namespace lra {
namespace {

constexpr int kBM = 128;             // tile rows (MMA M)
constexpr int kBN = 64;              // tile columns (MMA N)
constexpr int kKBox = 64;            // FP16 elements per 128-byte swizzled row
constexpr int kStages = 2;
constexpr int kTilesPerItem = 64;    // column tiles per work item
constexpr int kFrThreads = 256;
constexpr float kLoScale = 2048.0f;  // lo parts are stored times 2^11
constexpr int kTmemCols = 256;

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ void dot2_acc(float x, float y, float& p, float& c) {
  const float h = __fmul_rn(x, y);
  const float r = fmaf(x, y, -h);
  float q;
  two_sum_f(p, h, p, q);
  c = __fadd_rn(c, __fadd_rn(q, r));
}

// U (FP64, l x l) -> FP32 hi/lo pair.
__global__ void split_u_kernel(const double* __restrict__ U, int ll, float* __restrict__ Uhi,
                               float* __restrict__ Ulo) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ll) return;
  const double u = U[e];
  const float hi = (float)u;
  Uhi[e] = hi;
  Ulo[e] = (float)(u - (double)hi);
}

// Scale exponent so that max |x 2^-e| <= 2^14 (FP16 max is 65504).
__device__ __forceinline__ int scale_exp(float amax) {
  if (!(amax > 0.0f)) return 0;
  int ex;
  frexpf(amax, &ex);  // amax = f 2^ex, f in [0.5, 1)
  return ex - 14;
}

__device__ __forceinline__ void split_store(float x, float inv_scale, __half* hi, __half* lo) {
  const float xs = x * inv_scale;  // exact: power-of-two scale
  const __half h = __float2half_rn(xs);
  *hi = h;
  *lo = __float2half_rn((xs - __half2float(h)) * kLoScale);
}

// One block of 128 threads per kPRows rows of P: P[i][t] = sum_q C[i][q]
// U[q][t] with U = Uhi + Ulo: Dot2 in FP32 on the Uhi products, the Ulo
// products (2^-24 of the sum) added into the compensation term with one FMA
// each (thread t keeps the sums of column t for the block's rows, so each
// entry of U it loads serves every row).  Then per row the max -> a
// power-of-two scale, FP16 hi/lo split, zero padding to kp.
constexpr int kPRows = 8;

__global__ void __launch_bounds__(128) split_p_kernel(const float* __restrict__ C,
                                                      const float* __restrict__ Uhi,
                                                      const float* __restrict__ Ulo, long long m,
                                                      int l, int kp, __half* __restrict__ Phi,
                                                      __half* __restrict__ Plo,
                                                      float* __restrict__ pscale,
                                                      const JobStatus* js) {
  if (js->status != LRA_OK) return;
  __shared__ float red[kPRows][4];
  __shared__ float crow[kPRows][kMaxL];
  const long long i0 = (long long)blockIdx.x * kPRows;
  const int nr = (int)min((long long)kPRows, m - i0);
  const int t = threadIdx.x;
  for (int e = t; e < kPRows * l; e += blockDim.x) {
    const int r = e / l, q = e - r * l;
    crow[r][q] = r < nr ? __ldg(C + (i0 + r) * l + q) : 0.0f;
  }
  __syncthreads();
  float val[kPRows];
#pragma unroll
  for (int r = 0; r < kPRows; ++r) val[r] = 0.0f;
  if (t < l) {
    float p[kPRows], c[kPRows];
#pragma unroll
    for (int r = 0; r < kPRows; ++r) p[r] = c[r] = 0.0f;
    for (int q = 0; q < l; ++q) {
      const float uh = __ldg(Uhi + (size_t)q * l + t), ul = __ldg(Ulo + (size_t)q * l + t);
#pragma unroll
      for (int r = 0; r < kPRows; ++r) {
        const float cv = crow[r][q];
        dot2_acc(cv, uh, p[r], c[r]);
        c[r] = fmaf(cv, ul, c[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < kPRows; ++r) val[r] = __fadd_rn(p[r], c[r]);
  }
#pragma unroll
  for (int r = 0; r < kPRows; ++r) {
    float amax = fabsf(val[r]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    if ((t & 31) == 0) red[r][t >> 5] = amax;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kPRows; ++r) {
    if (r >= nr) break;
    const float amax = fmaxf(fmaxf(red[r][0], red[r][1]), fmaxf(red[r][2], red[r][3]));
    const int ex = scale_exp(amax);
    const long long i = i0 + r;
    if (t < kp) {
      __half h = __float2half_rn(0.0f), lo = h;
      if (t < l) split_store(val[r], ldexpf(1.0f, -ex), &h, &lo);
      Phi[i * kp + t] = h;
      Plo[i * kp + t] = lo;
    }
    if (t == 0) pscale[i] = ldexpf(1.0f, ex);
  }
}

// One thread per row j of R^T (column j of R): scale, split, zero padding;
// the kp halves of a row are written as 16-byte groups of 8.
__global__ void __launch_bounds__(128) split_rt_kernel(const float* __restrict__ R, long long n,
                                                       int l, int kp, __half* __restrict__ RThi,
                                                       __half* __restrict__ RTlo,
                                                       float* __restrict__ rscale,
                                                       const JobStatus* js) {
  if (js->status != LRA_OK) return;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= n) return;
  float amax = 0.0f;
  for (int t = 0; t < l; ++t) amax = fmaxf(amax, fabsf(__ldg(R + (size_t)t * n + j)));
  const int ex = scale_exp(amax);
  const float inv = ldexpf(1.0f, -ex);
  uint4* hrow = reinterpret_cast<uint4*>(RThi + j * kp);
  uint4* lrow = reinterpret_cast<uint4*>(RTlo + j * kp);
  for (int t8 = 0; t8 < kp; t8 += 8) {
    __align__(16) __half h[8], lo[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t8 + u;
      h[u] = __float2half_rn(0.0f);
      lo[u] = h[u];
      if (t < l) split_store(__ldg(R + (size_t)t * n + j), inv, &h[u], &lo[u]);
    }
    hrow[t8 / 8] = *reinterpret_cast<const uint4*>(h);
    lrow[t8 / 8] = *reinterpret_cast<const uint4*>(lo);
  }
  rscale[j] = ldexpf(1.0f, ex);
}

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier, TMA, tcgen05
// ---------------------------------------------------------------------------

using namespace tma;

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row atoms 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D = F32, A = B = F16, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// the persistent residual kernel
// ---------------------------------------------------------------------------

struct FullresArgs {
  long long m, n;
  int kb;             // 64-element K boxes (kp / 64)
  int ksteps;         // MMA K steps of 16 (ceil(l / 16))
  int n_row_tiles, n_col_tiles, n_groups, n_items;
  const float* pscale;
  const float* rscale;
  double* partials;   // [grid][2]: sum E^2, sum M^2
  JobStatus* js;
};

struct __align__(8) FrBarriers {
  uint64_t p_full, p_empty;
  uint64_t full[kStages], r_empty[kStages], a_empty[kStages];
  uint64_t t_full[2], t_empty[2];
  uint32_t tmem_base;
  int err;
  double red[2][4];
};

__global__ void __launch_bounds__(kFrThreads, 1)
fullres_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmPhi,
               const __grid_constant__ CUtensorMap tmPlo, const __grid_constant__ CUtensorMap tmRhi,
               const __grid_constant__ CUtensorMap tmRlo, FullresArgs a) {
  if (a.js->status != LRA_OK) return;
  extern __shared__ __align__(1024) unsigned char fr_smem[];
  // 1024-byte aligned layout (swizzle atoms)
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(fr_smem) + 1023) & ~(uintptr_t)1023);
  const int kb = a.kb;
  const uint32_t p_bytes = (uint32_t)kb * kBM * 128;      // one of Phi / Plo
  const uint32_t r_bytes = (uint32_t)kb * kBN * 128;      // one of Rhi / Rlo
  const uint32_t a_bytes = kBM * kBN * 4;                 // FP32 tile of M
  unsigned char* sPhi = base;
  unsigned char* sPlo = sPhi + p_bytes;
  unsigned char* sStage = sPlo + p_bytes;
  const uint32_t stage_bytes = 2 * r_bytes + a_bytes;
  FrBarriers* fb = reinterpret_cast<FrBarriers*>(sStage + kStages * stage_bytes);
  volatile int* err = &fb->err;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&fb->p_full, 1);
    mbar_init(&fb->p_empty, 1);
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&fb->full[s], 1);
      mbar_init(&fb->r_empty[s], 1);
      mbar_init(&fb->a_empty[s], 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&fb->t_full[b], 1);
      mbar_init(&fb->t_empty[b], 4);
    }
    fb->err = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&fb->tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = fb->tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t g = 0, ic = 0, p_issued = 0;
      for (int item = blockIdx.x; item < a.n_items && !*err; item += gridDim.x, ++ic) {
        const int rb = item / a.n_groups, cg = item - rb * a.n_groups;
        if (!mbar_wait(&fb->p_empty, (ic & 1) ^ 1, err)) break;
        mbar_expect_tx(&fb->p_full, 2 * p_bytes);
        for (int k = 0; k < kb; ++k) {
          load_2d(sPhi + k * kBM * 128, &tmPhi, k * kKBox, rb * kBM, &fb->p_full);
          load_2d(sPlo + k * kBM * 128, &tmPlo, k * kKBox, rb * kBM, &fb->p_full);
        }
        ++p_issued;
        const int t0 = cg * kTilesPerItem, t1 = min(a.n_col_tiles, t0 + kTilesPerItem);
        for (int tile = t0; tile < t1; ++tile, ++g) {
          const uint32_t s = g % kStages, u = g / kStages;
          if (!mbar_wait(&fb->r_empty[s], (u & 1) ^ 1, err)) break;
          if (!mbar_wait(&fb->a_empty[s], (u & 1) ^ 1, err)) break;
          unsigned char* st = sStage + s * stage_bytes;
          mbar_expect_tx(&fb->full[s], stage_bytes);
          for (int k = 0; k < kb; ++k) {
            load_2d(st + k * kBN * 128, &tmRhi, k * kKBox, tile * kBN, &fb->full[s]);
            load_2d(st + r_bytes + k * kBN * 128, &tmRlo, k * kKBox, tile * kBN, &fb->full[s]);
          }
          for (int c = 0; c < 2; ++c)
            load_2d(st + 2 * r_bytes + c * kBM * 128, &tmA, tile * kBN + c * 32, rb * kBM,
                        &fb->full[s]);
        }
      }
      // leave no copy in flight: wait (bounded, even after an error) for the
      // last fills of every stage and of the P tiles
      for (int s = 0; s < kStages; ++s) {
        if ((uint32_t)s >= g) break;
        const uint32_t gg = g - 1 - s;
        mbar_drain(&fb->full[gg % kStages], (gg / kStages) & 1);
      }
      if (p_issued > 0) mbar_drain(&fb->p_full, (p_issued - 1) & 1);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t g = 0, ic = 0;
      for (int item = blockIdx.x; item < a.n_items && !*err; item += gridDim.x, ++ic) {
        const int rb = item / a.n_groups, cg = item - rb * a.n_groups;
        (void)rb;
        if (!mbar_wait(&fb->p_full, ic & 1, err)) break;
        tc_fence_after();
        const int t0 = cg * kTilesPerItem, t1 = min(a.n_col_tiles, t0 + kTilesPerItem);
        for (int tile = t0; tile < t1; ++tile, ++g) {
          const uint32_t s = g % kStages, u = g / kStages;
          const uint32_t b = g & 1, ub = g >> 1;
          if (!mbar_wait(&fb->full[s], u & 1, err)) break;
          if (!mbar_wait(&fb->t_empty[b], (ub & 1) ^ 1, err)) break;
          tc_fence_after();
          const uint32_t d_hi = tmem + b * 2 * kBN;
          const uint32_t d_lo = d_hi + kBN;
          const uint32_t st = smem_u32(sStage + s * stage_bytes);
          const uint32_t phi = smem_u32(sPhi), plo = smem_u32(sPlo);
          for (int ks = 0; ks < a.ksteps; ++ks) {
            const int k = ks >> 2;
            const uint32_t koff = (uint32_t)(ks & 3) * 32;
            const uint64_t ah = sw128_desc(phi + k * kBM * 128 + koff);
            const uint64_t al = sw128_desc(plo + k * kBM * 128 + koff);
            const uint64_t bh = sw128_desc(st + k * kBN * 128 + koff);
            const uint64_t bl = sw128_desc(st + r_bytes + k * kBN * 128 + koff);
            umma_f16(d_hi, ah, bh, ks > 0);
            umma_f16(d_lo, ah, bl, ks > 0);
            umma_f16(d_lo, al, bh, 1);
          }
          umma_commit(&fb->r_empty[s]);
          umma_commit(&fb->t_full[b]);
        }
        umma_commit(&fb->p_empty);
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 4;
    const int r = ew * 32 + lane;
    double acc_e = 0.0, acc_a = 0.0;
    uint32_t g = 0;
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
      const int rb = item / a.n_groups, cg = item - rb * a.n_groups;
      const long long row = (long long)rb * kBM + r;
      const float ps = row < a.m ? __ldg(a.pscale + row) : 0.0f;
      const int t0 = cg * kTilesPerItem, t1 = min(a.n_col_tiles, t0 + kTilesPerItem);
      bool ok = true;
      for (int tile = t0; tile < t1; ++tile, ++g) {
        const uint32_t s = g % kStages, u = g / kStages;
        const uint32_t b = g & 1, ub = g >> 1;
        // every lane waits; the outcome is made warp-uniform before the
        // .sync.aligned tensor-memory loads
        bool w = mbar_wait(&fb->t_full[b], ub & 1, err) && mbar_wait(&fb->full[s], u & 1, err);
        if (!__all_sync(0xffffffffu, w)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const unsigned char* sa = sStage + s * stage_bytes + 2 * r_bytes;
        float se = 0.0f, sa2 = 0.0f;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float dh[32], dl[32];
          const uint32_t lane_off = (uint32_t)(ew * 32) << 16;
          tmem_ld32(tmem + lane_off + b * 2 * kBN + half * 32, dh);
          tmem_ld32(tmem + lane_off + b * 2 * kBN + kBN + half * 32, dl);
          const unsigned char* arow = sa + half * kBM * 128 + r * 128;
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4) {
            const float4 av = *reinterpret_cast<const float4*>(arow + ((c4 ^ (r & 7)) << 4));
            const float am[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int j = c4 * 4 + q;
              const long long col = (long long)tile * kBN + half * 32 + j;
              const float rs = col < a.n ? __ldg(a.rscale + col) : 0.0f;
              const float v = fmaf(dl[j], 1.0f / kLoScale, dh[j]) * (ps * rs);
              const float e = am[q] - v;
              se = fmaf(e, e, se);
              sa2 = fmaf(am[q], am[q], sa2);
            }
          }
        }
        acc_e += (double)se;
        acc_a += (double)sa2;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&fb->t_empty[b]);
          mbar_arrive(&fb->a_empty[s]);
        }
      }
      if (!ok) break;
    }
    // epilogue block reduction (fixed order)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc_e += __shfl_xor_sync(0xffffffffu, acc_e, off);
      acc_a += __shfl_xor_sync(0xffffffffu, acc_a, off);
    }
    if (lane == 0) {
      fb->red[0][ew] = acc_e;
      fb->red[1][ew] = acc_a;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    a.partials[blockIdx.x * 2 + 0] = fb->red[0][0] + fb->red[0][1] + fb->red[0][2] + fb->red[0][3];
    a.partials[blockIdx.x * 2 + 1] = fb->red[1][0] + fb->red[1][1] + fb->red[1][2] + fb->red[1][3];
    if (fb->err) set_status(a.js, LRA_ETIMEOUT);
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

__global__ void fullres_final_kernel(const double* __restrict__ partials, int nblocks, JobStatus* js) {
  if (js->status != LRA_OK || threadIdx.x != 0) return;
  double se = 0.0, sa = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    se += partials[2 * b];
    sa += partials[2 * b + 1];
  }
  js->full_sse = se;
  js->full_ssa = sa;
  js->full_rel = sa > 0.0 ? sqrt(se / sa) : INFINITY;
}

bool make_map(CUtensorMap* map, CUtensorMapDataType dt, const void* gaddr, uint64_t inner,
              uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  return make_map_2d(map, dt, gaddr, inner, outer, row_bytes, box_inner, box_outer, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B);
}

}  // namespace

size_t fullres_workspace_bytes(long long m, long long n, int l, int grid) {
  const int kp = ((l + kKBox - 1) / kKBox) * kKBox;
  size_t b = 0;
  auto take = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
  take(sizeof(__half) * (size_t)m * kp);  // Phi
  take(sizeof(__half) * (size_t)m * kp);  // Plo
  take(sizeof(__half) * (size_t)n * kp);  // RThi
  take(sizeof(__half) * (size_t)n * kp);  // RTlo
  take(sizeof(float) * (size_t)m);        // pscale
  take(sizeof(float) * (size_t)n);        // rscale
  take(sizeof(float) * 2 * (size_t)l * l);  // Uhi, Ulo
  take(sizeof(double) * 2 * (size_t)grid);  // partials
  return b;
}

cudaError_t launch_full_residual(const float* A, long long lda, long long m, long long n, int l,
                                 const float* C, const double* U, const float* R, void* ws,
                                 int grid_cap, JobStatus* js, cudaStream_t st) {
  const int kp = ((l + kKBox - 1) / kKBox) * kKBox;
  unsigned char* w = static_cast<unsigned char*>(ws);
  auto take = [&](size_t x) {
    unsigned char* p = w;
    w += (x + 255) & ~(size_t)255;
    return p;
  };
  __half* Phi = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)m * kp));
  __half* Plo = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)m * kp));
  __half* RThi = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)n * kp));
  __half* RTlo = reinterpret_cast<__half*>(take(sizeof(__half) * (size_t)n * kp));
  float* pscale = reinterpret_cast<float*>(take(sizeof(float) * (size_t)m));
  float* rscale = reinterpret_cast<float*>(take(sizeof(float) * (size_t)n));
  float* Uhi = reinterpret_cast<float*>(take(sizeof(float) * 2 * (size_t)l * l));
  float* Ulo = Uhi + (size_t)l * l;
  double* partials = reinterpret_cast<double*>(take(sizeof(double) * 2 * (size_t)grid_cap));

  split_u_kernel<<<(l * l + 255) / 256, 256, 0, st>>>(U, l * l, Uhi, Ulo);
  split_p_kernel<<<(unsigned)((m + kPRows - 1) / kPRows), 128, 0, st>>>(C, Uhi, Ulo, m, l, kp, Phi, Plo, pscale, js);
  split_rt_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(R, n, l, kp, RThi, RTlo, rscale, js);
  cudaError_t e = cudaGetLastError();
  if (e) return e;

  CUtensorMap mA, mPhi, mPlo, mRhi, mRlo;
  if (!make_map(&mA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, n, m, lda * 4, 32, kBM) ||
      !make_map(&mPhi, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, Phi, kp, m, kp * 2, kKBox, kBM) ||
      !make_map(&mPlo, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, Plo, kp, m, kp * 2, kKBox, kBM) ||
      !make_map(&mRhi, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, RThi, kp, n, kp * 2, kKBox, kBN) ||
      !make_map(&mRlo, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, RTlo, kp, n, kp * 2, kKBox, kBN))
    return cudaErrorInvalidValue;

  FullresArgs a{};
  a.m = m;
  a.n = n;
  a.kb = kp / kKBox;
  a.ksteps = (l + 15) / 16;
  a.n_row_tiles = (int)((m + kBM - 1) / kBM);
  a.n_col_tiles = (int)((n + kBN - 1) / kBN);
  a.n_groups = (a.n_col_tiles + kTilesPerItem - 1) / kTilesPerItem;
  a.n_items = a.n_row_tiles * a.n_groups;
  a.pscale = pscale;
  a.rscale = rscale;
  a.partials = partials;
  a.js = js;
  const int grid = std::min(grid_cap, a.n_items);
  const size_t smem = 1024 + 2 * (size_t)a.kb * kBM * 128 +
                      kStages * (2 * (size_t)a.kb * kBN * 128 + kBM * kBN * 4) + sizeof(FrBarriers);
  if ((e = smem_optin(reinterpret_cast<const void*>(fullres_kernel), 227 * 1024))) return e;
  fullres_kernel<<<grid, kFrThreads, smem, st>>>(mA, mPhi, mPlo, mRhi, mRlo, a);
  fullres_final_kernel<<<1, 32, 0, st>>>(partials, grid, js);
  return cudaGetLastError();
}

}  // namespace lra
