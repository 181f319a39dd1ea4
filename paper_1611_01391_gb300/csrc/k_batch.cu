// Batched C-A over thousands of blocks of one generated matrix: the
// low-rank generators of the far-field (neutered) blocks of an HSS / FMM
// matrix, the "bottleneck stage" of Section 9, computed by C-A iterations
// (Section 6.5) in one persistent launch.
//
// Design:
//   * One CTA, or a thread-block cluster of 4 or 8 CTAs, solves one block at
//     a time and pulls the next block index from a device work queue (an
//     atomic counter), so uneven blocks balance themselves.  The strip of
//     the current half-step (up to 2048 rows x l <= 96 values, each a
//     double-float pair) is split across the cluster's shared memory and
//     never leaves the chip.
//   * Each decision: every CTA reduces its best candidate (packed
//     |value|/index key, warp shuffles), publishes it and that row in its
//     shared memory, one hardware cluster barrier, then every CTA reads the
//     four candidates through distributed shared memory and updates its rows.
//   * Every strip starts from Gauss-Jordan elimination with partial pivoting
//     whose pivots are restricted to the previous index set (the very first
//     strip, and the rows a grown cross lacks, pivot freely), and continues
//     with maxvol swaps.  The strip is held and updated in double-float
//     pairs (about 48 significant bits from FP32 instructions, as in the
//     plain maxvol): the crosses of a rank-adaptive block reach condition
//     numbers near 1 / tol = 1e6, where FP32 updates of B would carry errors
//     of 1e-1 and lose the pivot sequence, while pairs keep B accurate to
//     about 1e-8.  Candidates are ranked by the FP32 high part (ties: the
//     smaller row, then column); the stop test uses the whole pair.
//   * Rank adaptivity, after every sweep: the leader CTA takes the SVD of
//     the cross (QR with column pivoting, then one-sided Jacobi, double-float
//     arithmetic: an FP32 SVD cannot resolve singular values near
//     tol sigma_1 = 1e-6 sigma_1) and counts k = #{sigma_j > tol sigma_1}.
//     If k = l < k_max the cross grows (x2, up to l_max) with the block's
//     next candidate columns; otherwise U = (X_k)^+ (k_eff = min(k_max, k),
//     FP64) and the Appendix F estimate on a q x q sample are written, and
//     the block stops once k >= k_max, the estimate is <= tol, or the sweep
//     budget at this size is spent.
//   * The estimate uses compensated FP32 products and FP64 sums.
#include <cooperative_groups.h>

#include <cfloat>

#include "lra_internal.cuh"
#include "lra_kernels.h"
#include "dd_arith.cuh"
#include "svd_dd.cuh"

namespace cg = cooperative_groups;

namespace lra {
namespace {

constexpr int kBT = 256;                  // threads per CTA
constexpr int kStripFloats = (kMaxBatchSide / 4) * kMaxL;  // strip area per CTA (196 KB)
constexpr int kStripPairs = kStripFloats / 2;              // double-float entries it holds
constexpr int kMaxQ = 64;                 // sample size per side
constexpr int kDeferred = 1;              // status of a block left to a later pass (more CTAs)

// Shared memory of one CTA of a CS-CTA cluster.
template <int CS>
struct BatchSmemT {
  float B[kStripFloats];                  // strip chunk (kStripPairs pairs), row-major with stride l
  dd colj[kMaxBatchSide / CS];
  dd rrow[kMaxL];
  dd slot_row[2][kMaxL];                  // published candidate rows (read by peers)
  unsigned long long slot_key[2];
  int slot_nf[2];
  unsigned long long red_key[kBT / 32];
  int red_nf[kBT / 32];
  unsigned long long win_key;
  int win_nf;
  int pos[kMaxL];
  int Iset[kMaxL], Jset[kMaxL];
  unsigned char used[kMaxBatchSide / CS];
  int blk;
  int status;
  int swaps;
  int keff;
  int lnew;
  int grow, stop;
  double esum[2][kBT / 32];
};
// the nucleus (W, V, sigma, 1/sigma^2, order) and the estimate's operands
// reuse the strip area once the sweeps are over
static_assert(2 * kMaxL * kMaxL * sizeof(dd) + kMaxL * (sizeof(double) + sizeof(dd) + sizeof(int)) +
                      sizeof(SvdScratch) <= sizeof(float) * kStripFloats, "nucleus area");
static_assert(sizeof(float) * (2 * kMaxL * kMaxL + 4 * kMaxQ * kMaxL) <= sizeof(float) * kStripFloats,
              "estimate area");
static_assert(sizeof(BatchSmemT<1>) <= 227 * 1024, "one CTA's shared memory");

__device__ __forceinline__ unsigned long long pack_key(float v, int idx) {
  return ((unsigned long long)(__float_as_uint(v) & 0x7fffffffu) << 32) | (unsigned)(~idx);
}
__device__ __forceinline__ int key_idx(unsigned long long k) { return ~(int)(unsigned)(k & 0xffffffffu); }
__device__ __forceinline__ float key_val(unsigned long long k) { return __uint_as_float((unsigned)(k >> 32)); }

__device__ __forceinline__ void consider_f(unsigned long long& best, int& nf, float v, int idx) {
  if ((__float_as_uint(v) & 0x7fffffffu) >= 0x7f800000u) {
    nf = 1;
    return;
  }
  const unsigned long long k = pack_key(v, idx);
  if (k > best) best = k;
}

// CTA-wide reduction of (key, nf); result in s->win_key / s->win_nf.
template <typename S>
__device__ __forceinline__ void cta_reduce(S* s, unsigned long long key, int nf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_down_sync(0xffffffffu, key, off);
    nf |= __shfl_down_sync(0xffffffffu, nf, off);
    if (o > key) key = o;
  }
  if (lane == 0) {
    s->red_key[warp] = key;
    s->red_nf[warp] = nf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long k = 0ull;
    int f = 0;
    for (int w = 0; w < kBT / 32; ++w) {
      if (s->red_key[w] > k) k = s->red_key[w];
      f |= s->red_nf[w];
    }
    s->win_key = k;
    s->win_nf = f;
  }
  __syncthreads();
}

// One strip of the C-A iteration on the cluster: load the N x l strip
// (vertical: S[i][t] = M(row0 + i, col0 + other[t]); horizontal:
// S[j][t] = M(row0 + other[t], col0 + j)) as double-float pairs,
// Gauss-Jordan start, maxvol.  The start keeps the previous index set: for
// its first nfirst steps the pivot rows are restricted to the strip rows
// first[0 .. nfirst) (partial pivoting among them), later steps pivot over
// every free row; step t puts its pivot row in position t.  After l steps
// B = S X^{-1} with X the rows so chosen.  Returns false when the block
// failed (s->status set identically in all CTAs).  On return s->pos holds
// the selected strip rows.  With a decision log (trace != nullptr, written
// by the leader CTA's thread 0): every decision of this half-step as
// (half_step, kind, i, j) and its |value| in FP64, while *tlen < tcap.
template <int KIND, int CS>
__device__ bool half_step(const BatchArgs& a, cg::cluster_group& cl, BatchSmemT<CS>* s, bool vertical,
                          long long row0, long long col0, int N, int l, const int* other,
                          int nfirst, const int* first, int hs, int* trace, double* trace_v, int* tlen) {
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int rpc = (N + CS - 1) / CS;
  const int r0 = rank * rpc;
  const int nr = max(0, min(rpc, N - r0));
  dd* B = reinterpret_cast<dd*>(s->B);
  for (int e = tid; e < nr * l; e += kBT) {
    const int r = e / l, t = e - r * l;
    const long long g = r0 + r;
    B[e] = dd_make(vertical ? entry<KIND>(a.src, row0 + g, col0 + other[t])
                            : entry<KIND>(a.src, row0 + other[t], col0 + g));
  }
  for (int r = tid; r < nr; r += kBT) s->used[r] = 0;  // bit 0: pivoted, bit 1: in first
  __syncthreads();
  for (int t = tid; t < nfirst; t += kBT) {
    const int g = first[t];
    if (g >= r0 && g < r0 + nr) s->used[g - r0] = 2;
  }
  __syncthreads();

  unsigned long long mine = 0ull;
  int nf = 0;
  for (int r = tid; r < nr; r += kBT)
    if (nfirst == 0 || (s->used[r] & 2)) consider_f(mine, nf, B[r * l].hi, (r0 + r) * l);
  bool gepp = true;
  int step = 0, swaps = 0, buf = 0;
  bool ok = true;
  const bool log = trace != nullptr && rank == 0 && tid == 0;
  for (;;) {
    cta_reduce(s, mine, nf);
    const unsigned long long cb = s->win_key;
    if (tid == 0) {
      s->slot_key[buf] = cb;
      s->slot_nf[buf] = s->win_nf;
    }
    if (cb != 0ull && tid < l) {
      const int r = key_idx(cb) / l - r0;
      s->slot_row[buf][tid] = B[r * l + tid];
    }
    if (CS > 1) cl.sync(); else __syncthreads();
    unsigned long long win = 0ull;
    int wnf = 0, owner = 0;
    for (int p = 0; p < CS; ++p) {
      const unsigned long long k = *cl.map_shared_rank(&s->slot_key[buf], p);
      wnf |= *cl.map_shared_rank(&s->slot_nf[buf], p);
      if (k > win) {
        win = k;
        owner = p;
      }
    }
    const int idx = key_idx(win);
    const int istar = win == 0ull ? -1 : idx / l, jstar = win == 0ull ? 0 : idx - istar * l;
    // the winner's whole pair decides (the key ranks by its high part)
    const dd pv = win == 0ull ? dd_make(0.0f) : cl.map_shared_rank(&s->slot_row[buf][0], owner)[jstar];
    const double wv = fabs(dd_to_double(pv));
    int kind;
    if (wnf) {
      if (tid == 0) s->status = LRA_ENONFINITE;
      ok = false;
      break;
    }
    if (gepp) {
      if (win == 0ull || !(wv > 0.0)) {
        if (tid == 0) s->status = LRA_ESINGULAR;
        ok = false;
        break;
      }
      kind = LRA_TRACE_GEPP;
    } else if (wv <= 1.0 + a.delta) {
      kind = LRA_TRACE_STOP;
    } else if (swaps >= a.max_swaps) {
      kind = LRA_TRACE_CAP;
    } else {
      kind = LRA_TRACE_SWAP;
    }
    if (log && *tlen < a.trace_cap) {
      const int n = (*tlen)++;
      trace[4 * n + 0] = hs;
      trace[4 * n + 1] = kind;
      trace[4 * n + 2] = istar;
      trace[4 * n + 3] = jstar;
      trace_v[n] = wv;
    }
    if (kind == LRA_TRACE_STOP || kind == LRA_TRACE_CAP) break;
    if (tid < l) s->rrow[tid] = cl.map_shared_rank(&s->slot_row[buf][0], owner)[tid];
    for (int r = tid; r < nr; r += kBT) s->colj[r] = B[r * l + jstar];
    if (tid == 0) {
      if (gepp && istar >= r0 && istar < r0 + nr) s->used[istar - r0] |= 1;
      s->pos[jstar] = istar;
    }
    __syncthreads();
    // the update's row factor (B[i*, :] - e_j*^T) / B[i*, j*]
    if (tid < l) {
      dd rt = s->rrow[tid];
      if (tid == jstar) rt = dd_add(rt, dd_make(-1.0f));
      s->rrow[tid] = dd_div(rt, pv);
    }
    __syncthreads();
    const bool next_gepp = gepp && (step + 1 < l);
    const int next_col = step + 1;
    mine = 0ull;
    for (int e = tid; e < nr * l; e += kBT) {
      const int r = e / l, t = e - r * l;
      const int g = r0 + r;
      dd v;
      if (g == istar) {
        v = dd_make((t == jstar) ? 1.0f : 0.0f);   // the pivot row becomes e_j* exactly
        B[e] = v;
        if (!next_gepp) consider_f(mine, nf, v.hi, g * l + t);
      } else {
        v = dd_fnma(s->colj[r], s->rrow[t], B[e]);
        B[e] = v;
        if (next_gepp ? (t == next_col && !(s->used[r] & 1) && (next_col >= nfirst || (s->used[r] & 2)))
                      : true)
          consider_f(mine, nf, v.hi, g * l + t);
      }
    }
    if (gepp) {
      if (++step == l) gepp = false;
    } else {
      ++swaps;
    }
    buf ^= 1;
    __syncthreads();
  }
  if (tid == 0) {
    s->swaps += swaps;
    // work of this strip: every decision updates the N x l strip
    if (rank == 0) atomicAdd(&a.js->maxvol_flops, 2.0 * N * l * (double)(step + swaps));
  }
  cl.sync();  // peers finished reading this CTA's slots before they are reused
  return ok;
}

__device__ __forceinline__ void two_sum_b(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ void dot2_b(float x, float y, float& p, float& c) {
  const float h = __fmul_rn(x, y);
  const float r = fmaf(x, y, -h);
  float q;
  two_sum_b(p, h, p, q);
  c = __fadd_rn(c, __fadd_rn(q, r));
}

// Leader CTA, after every sweep: SVD of the cross X = M[I, J] (QR with
// column pivoting, then one-sided Jacobi, in double-float), the rank count
// k = #{sigma_j > tol sigma_1} and the decision to grow the cross (k = l <
// k_max, l below the block's cap, unused candidates left).  Unless it grows,
// the block's outputs are (re)written: I, J, sigma, k_eff = min(k_max, k),
// U = (X_k)^+ in FP64 and the Appendix F estimate; s->stop is set when
// k >= k_max or the estimate is <= tol.
template <int KIND, typename S>
__device__ void cross_step(const BatchArgs& a, S* s, int b, long long row0, long long col0,
                           long long n, int l, int lmax_b) {
  const int tid = threadIdx.x;
  dd* W = reinterpret_cast<dd*>(s->B);
  dd* Z = W + kMaxL * kMaxL;
  double* sig = reinterpret_cast<double*>(Z + kMaxL * kMaxL);
  dd* inv2 = reinterpret_cast<dd*>(sig + kMaxL);
  SvdScratch* sc = reinterpret_cast<SvdScratch*>(inv2 + kMaxL);
  int* order = reinterpret_cast<int*>(sc + 1);
  if (tid == 0) s->lnew = 0;
  __syncthreads();
  // X scaled by a power of two into [0.5, 1)
  float amax = 0.0f;
  for (int e = tid; e < l * l; e += kBT) {
    const int p = e / l, q = e - p * l;
    const float x = entry<KIND>(a.src, row0 + s->Iset[p], col0 + s->Jset[q]);
    amax = fmaxf(amax, fabsf(x));
    W[q * l + p] = dd_make(x);   // column q of X
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
  if ((tid & 31) == 0 && amax > 0.0f) {
    int ex;
    frexpf(amax, &ex);
    atomicMax(&s->lnew, ex + 1024);
  }
  __syncthreads();
  const int ex = s->lnew ? s->lnew - 1024 : 0;
  for (int e = tid; e < l * l; e += kBT) W[e].hi = ldexpf(W[e].hi, -ex);
  __syncthreads();
  svd_dd<kBT>(W, Z, l, sc);
  jacobi_sigma<kBT>(W, l, sig, order);
  if (tid == 0) {
    const double s1 = sig[order[0]];
    int k = 0;
    if (s1 > 0.0)
      while (k < l && sig[order[k]] > (double)a.tol * s1) ++k;
    int avail = 0;
    for (int c = 0; c < a.l_max; ++c) {
      const int j = a.jcand[(size_t)b * a.l_max + c];
      bool in = false;
      for (int t = 0; t < l; ++t) in |= (s->Jset[t] == j);
      avail += (!in && j < n);
    }
    s->grow = (k == l && k < a.k_max && l < lmax_b && avail > 0);
    s->keff = min(k, a.k_max);
    s->stop = (k >= a.k_max);
  }
  __syncthreads();
  if (s->grow) return;
  for (int t = tid; t < l; t += kBT) {
    a.out_I[(size_t)b * a.l_max + t] = s->Iset[t];
    a.out_J[(size_t)b * a.l_max + t] = s->Jset[t];
  }
  if (tid == 0) a.out_keff[b] = s->keff;
  float* sg_out = a.out_sigma + (size_t)b * a.l_max;
  for (int r = tid; r < l; r += kBT) {
    const double sb = sig[order[r]];
    inv2[r] = dd_from_double(sb > 0.0 ? 1.0 / (sb * sb) : 0.0);
    sg_out[r] = (float)ldexp(sb, ex);
  }
  __syncthreads();
  left_vectors<kBT>(W, Z, l, s->keff, order, inv2, sc->perm);
  double* Ub = a.out_U + (size_t)b * a.l_max * a.l_max;
  nucleus_from_svd<kBT>(W, Z, sc->perm, l, s->keff, order, inv2,
                        [&](int e, double v) { Ub[e] = ldexp(v, -ex); });
  __syncthreads();
  // Appendix F estimate on the q x q sample of this block
  const int q = a.q;
  if (q > 0) {
    float* Us = s->B;                      // U (l x l) back from global: hi part
    float* Usl = Us + kMaxL * kMaxL;       //   and lo part, U = hi + lo
    float* Cs = Usl + kMaxL * kMaxL;       // q x l: M(row0 + sr, col0 + J)
    float* Rs = Cs + kMaxQ * kMaxL;        // l x q: M(row0 + I, col0 + sc)
    float* CUh = Rs + kMaxL * kMaxQ;       // q x l: (C U) hi
    float* CUl = CUh + kMaxQ * kMaxL;      //        (C U) lo
    const int* sr = a.srow + (size_t)b * q;
    const int* scl = a.scol + (size_t)b * q;
    for (int e = tid; e < l * l; e += kBT) {
      const double u = Ub[e];
      const float hi = (float)u;
      Us[e] = hi;
      Usl[e] = (float)(u - (double)hi);
    }
    for (int e = tid; e < q * l; e += kBT) {
      const int i = e / l, t = e - i * l;
      Cs[e] = entry<KIND>(a.src, row0 + sr[i], col0 + s->Jset[t]);
      Rs[t * q + i] = entry<KIND>(a.src, row0 + s->Iset[t], col0 + scl[i]);
    }
    __syncthreads();
    for (int e = tid; e < q * l; e += kBT) {
      const int i = e / l, u = e - i * l;
      float p = 0.f, c = 0.f;
      for (int t = 0; t < l; ++t) {
        dot2_b(Cs[i * l + t], Us[t * l + u], p, c);
        c = __fmaf_rn(Cs[i * l + t], Usl[t * l + u], c);  // the lo part needs FP32 only
      }
      const float hi = __fadd_rn(p, c);
      CUh[e] = hi;
      CUl[e] = __fadd_rn(__fsub_rn(p, hi), c);  // rounding error of hi = p + c
    }
    __syncthreads();
    double se = 0.0, sa = 0.0;
    for (int e = tid; e < q * q; e += kBT) {
      const int i = e / q, j = e - i * q;
      float p = 0.f, c = 0.f;
      for (int u = 0; u < l; ++u) {
        dot2_b(CUh[i * l + u], Rs[u * q + j], p, c);
        dot2_b(CUl[i * l + u], Rs[u * q + j], p, c);
      }
      const float mv = entry<KIND>(a.src, row0 + sr[i], col0 + scl[j]);
      const double ev = ((double)mv - (double)p) - (double)c;
      se += ev * ev;
      sa += (double)mv * (double)mv;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      se += __shfl_xor_sync(0xffffffffu, se, off);
      sa += __shfl_xor_sync(0xffffffffu, sa, off);
    }
    if ((tid & 31) == 0) {  // fixed-order sum: reproducible bits
      s->esum[0][tid >> 5] = se;
      s->esum[1][tid >> 5] = sa;
    }
    __syncthreads();
    if (tid == 0) {
      double e2 = 0.0, a2 = 0.0;
      for (int w = 0; w < kBT / 32; ++w) {
        e2 += s->esum[0][w];
        a2 += s->esum[1][w];
      }
      const double est = a2 > 0.0 ? sqrt(e2 / a2) : 0.0;
      a.out_err[b] = est;
      if (est <= (double)a.tol) s->stop = 1;
    }
  }
  __syncthreads();
}

// A chain of passes over the blocks, with clusters of 1, 2, 4 or 8 CTAs
// (by default 1, 4, 8; the batch tuner picks the chain per workload).  The
// first pass takes every block; a block whose rank rule asks for a cross
// larger than its cluster can hold (l max(m, n) > CS kStripPairs), or, in
// the first pass, whose larger side exceeds the cut-over side, is left with
// status kDeferred and restarts from scratch in the next pass.  The last
// pass (CS = 8) holds every block (2048 x 96 pairs).  With one CTA a block
// needs no cluster barrier per decision and 152 blocks are in flight.  The
// decisions (argmax with the same tie-break over the whole strip) and the
// arithmetic per entry do not depend on the split, so a block's result is
// the same in any pass, chain or order.
static_assert(8 * kStripPairs >= kMaxBatchSide * kMaxL, "the 8-CTA pass holds every strip");
template <int KIND, int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kBT, 1) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char bsm[];
  BatchSmemT<CS>* s = reinterpret_cast<BatchSmemT<CS>*>(bsm);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const bool kFirst = a.pass_first != 0;
  constexpr bool kLast = (CS == 8);
  int* queue = a.queue + a.pass_idx;
  for (;;) {
    if (rank == 0 && tid == 0)  // a cancelled job takes no further block
      s->blk = (*(volatile const int*)&a.js->status != LRA_OK) ? a.n_blocks : atomicAdd(queue, 1);
    cl.sync();
    const int qpos = *cl.map_shared_rank(&s->blk, 0);
    if (qpos >= a.n_blocks) {
      cl.sync();  // nobody leaves while a peer may still read the leader's index
      break;
    }
    const int b = a.order ? a.order[qpos] : qpos;   // the queue's order of the blocks
    if (!kFirst && a.out_status[b] != kDeferred) {
      cl.sync();  // the leader may fetch the next index
      continue;
    }
    const long long row0 = a.blocks[4 * b + 0], m = a.blocks[4 * b + 1];
    const long long col0 = a.blocks[4 * b + 2], n = a.blocks[4 * b + 3];
    const int lmax_b = (int)min((long long)a.l_max, min(m, n));
    // largest cross whose strips fit this cluster's shared memory
    const int lcap = (int)min((long long)lmax_b, kStripPairs / ((max(m, n) + CS - 1) / CS));
    int l = min(a.l_init, lmax_b);
    bool deferred = !kLast && (l > lcap || (kFirst && a.cutover > 0 && max(m, n) > a.cutover));
    // decision log of this block (leader CTA, thread 0)
    int* btrace = a.trace_cap > 0 ? a.trace + (size_t)b * a.trace_cap * 4 : nullptr;
    double* btrace_v = a.trace_cap > 0 ? a.trace_v + (size_t)b * a.trace_cap : nullptr;
    int tlen = 0, hs = 0;
    for (int t = tid; t < l; t += kBT) s->Jset[t] = a.jcand[(size_t)b * a.l_max + t];
    if (tid == 0) {
      s->status = LRA_OK;
      s->swaps = 0;
    }
    __syncthreads();
    bool ok = true;
    int n_i = 0;       // rows of the previous I (none before the first sweep)
    int at_size = 0;   // sweeps at the current cross size
    while (!deferred) {
      ok = half_step<KIND, CS>(a, cl, s, true, row0, col0, (int)m, l, s->Jset, n_i, s->Iset, hs++, btrace,
                               btrace_v, &tlen);
      if (!ok) break;
      for (int t = tid; t < l; t += kBT) s->Iset[t] = s->pos[t];
      n_i = l;
      __syncthreads();
      ok = half_step<KIND, CS>(a, cl, s, false, row0, col0, (int)n, l, s->Iset, l, s->Jset, hs++, btrace,
                               btrace_v, &tlen);
      if (!ok) break;
      for (int t = tid; t < l; t += kBT) s->Jset[t] = s->pos[t];
      __syncthreads();
      ++at_size;
      if (rank == 0) cross_step<KIND>(a, s, b, row0, col0, n, l, lmax_b);
      cl.sync();
      const int grow = *cl.map_shared_rank(&s->grow, 0);
      const int stop = *cl.map_shared_rank(&s->stop, 0);
      if (grow) {
        if (!kLast && min(lmax_b, 2 * l) > lcap) {  // only a pass with more CTAs holds this cross
          deferred = true;
          break;
        }
        // append the next candidate columns that are not in J (same in every CTA)
        if (tid == 0) {
          const int l_new = min(lmax_b, 2 * l);
          int cnt = l;
          for (int c = 0; c < a.l_max && cnt < l_new; ++c) {
            const int j = a.jcand[(size_t)b * a.l_max + c];
            bool in = false;
            for (int t = 0; t < cnt; ++t) in |= (s->Jset[t] == j);
            if (!in && j < n) s->Jset[cnt++] = j;
          }
          s->lnew = cnt;
        }
        __syncthreads();
        l = s->lnew;
        at_size = 0;
        __syncthreads();
        continue;
      }
      if (stop || at_size >= a.sweeps) break;
    }
    if (rank == 0 && deferred) {
      if (tid == 0) a.out_status[b] = kDeferred;
    } else if (rank == 0) {
      if (tid == 0) {
        a.out_status[b] = ok ? (int)LRA_OK : s->status;
        a.out_l[b] = l;
        a.out_swaps[b] = s->swaps;
        if (a.trace_cap > 0) a.trace_len[b] = tlen;
        if (!ok) {
          a.out_keff[b] = 0;
          a.out_err[b] = 0.0;
        }
      }
      // defined contents past the l x l nucleus (and everywhere on failure)
      const int lu = ok ? l : 0;
      double* Ub = a.out_U + (size_t)b * a.l_max * a.l_max;
      for (int e = lu * lu + tid; e < a.l_max * a.l_max; e += kBT) Ub[e] = 0.0;
      for (int t = lu + tid; t < a.l_max; t += kBT) {
        a.out_sigma[(size_t)b * a.l_max + t] = 0.0f;
        a.out_I[(size_t)b * a.l_max + t] = -1;
        a.out_J[(size_t)b * a.l_max + t] = -1;
      }
    }
    cl.sync();  // block done: the leader may fetch the next block index
  }
}

}  // namespace

size_t batch_smem_bytes() { return sizeof(BatchSmemT<1>); }

template <int KIND, int CS>
static cudaError_t launch_pass(const BatchArgs& a, int sms, cudaStream_t st) {
  const size_t smem = sizeof(BatchSmemT<CS>);
  const cudaError_t e = smem_optin(reinterpret_cast<const void*>(batch_kernel<KIND, CS>), (int)smem);
  if (e) return e;
  batch_kernel<KIND, CS><<<(sms / CS) * CS, kBT, smem, st>>>(a);
  return cudaGetLastError();
}

// a.queue holds four zeroed counters, one per pass.  cluster_mask: bit c
// set = a pass with 2^c CTAs per cluster (the 8-CTA pass always runs last).
cudaError_t launch_batch(const BatchArgs& a0, int cluster_mask, int sms, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  BatchArgs a = a0;
  const int mask = (cluster_mask & 7) | 8;
  bool first = true;
  for (int c = 0; c < 4 && !e; ++c) {
    if (!(mask & (1 << c))) continue;
    a.pass_idx = c;
    a.pass_first = first ? 1 : 0;
    first = false;
    LRA_DISPATCH_KIND(a.src.kind, ({
      switch (c) {
        case 0: e = launch_pass<K, 1>(a, sms, st); break;
        case 1: e = launch_pass<K, 2>(a, sms, st); break;
        case 2: e = launch_pass<K, 4>(a, sms, st); break;
        default: e = launch_pass<K, 8>(a, sms, st); break;
      }
    }));
  }
  return e;
}

}  // namespace lra
