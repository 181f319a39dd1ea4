// Host runtime of the C ABI declared in include/lra_cross.h: contexts, job
// admission, per-job device memory and the launch sequence of one C-A solve
// (Section 6.5: C-A iterations, then the Primitive Algorithm's nucleus;
// Appendix F: sampled error estimate).
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "lra_internal.cuh"
#include "lra_kernels.h"

using namespace lra;

namespace {

struct Job {
  lra_job id = 0;
  SourceDev src{};
  int l = 0, k = 0, sweeps = 0, max_swaps = 0, trace_cap = 0, slot = -1;
  long long m = 0, n = 0, q = 0, s = 0;
  double delta = 0, rank_tol = 0, tol = 0;
  unsigned char* dmem = nullptr;
  size_t prefix = 0;  // bytes of dmem filled from the slot's staging at submit
  size_t bytes = 0;
  JobStatus* js = nullptr;
  GridBarrier* bar = nullptr;
  int *J = nullptr, *I = nullptr, *rows = nullptr, *cols = nullptr, *trace_i = nullptr;
  double *U = nullptr, *sigma = nullptr, *trace_v = nullptr, *partials = nullptr;
  float2 *xbuf0 = nullptr, *xbuf1 = nullptr;  // cross inverses as FP32 pairs
  float2* cand_rows = nullptr;
  float *C = nullptr, *R = nullptr, *CUq = nullptr;
  unsigned long long* win_ring = nullptr;
  int n_partials = 0;
  MaxvolPlan plan_col{}, plan_row{};
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  int launches = 0, maxvol_launches = 0;
  bool profile = false;
  bool full_res = false;
  bool resume = false;   // init_I given: the first vertical step warm-starts from it
  bool tma_cols = false;  // stored FP32 source: column gathers through TMA
  TmaMap col_map{};
  void* fr_ws = nullptr;
  std::vector<std::pair<int, cudaEvent_t>> prof;  // (kernel class, event after the launch)
  cudaStream_t stream = nullptr;  // the context stream this job runs on
  int stream_idx = -1;
  // batched jobs
  bool batch = false;
  int n_blocks = 0, b_lmax = 0, b_q = 0;
  long long* b_blocks = nullptr;
  int *b_jcand = nullptr, *b_srow = nullptr, *b_scol = nullptr, *b_queue = nullptr;
  int *b_status = nullptr, *b_l = nullptr, *b_keff = nullptr, *b_swaps = nullptr, *b_I = nullptr, *b_J = nullptr;
  double* b_U = nullptr;
  float* b_sigma = nullptr;
  double* b_err = nullptr;
  int b_tcap = 0;
  int *b_tlen = nullptr, *b_trace = nullptr;
  double* b_tval = nullptr;
};

enum { kClsGather = 0, kClsMaxvol = 1, kClsCross = 2, kClsResid = 3, kClsInverse = 4, kClsFullres = 5,
       kClsOther = 6 };

// Sub-buffer offsets of one job's single device allocation.
struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  }
};

}  // namespace

struct lra_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;           // streams[0]
  bool own_stream = false;
  std::vector<cudaStream_t> streams;       // jobs are spread over these
  std::vector<int> stream_load;            // active jobs per stream
  cudaStream_t ctrl = nullptr;             // cancellations run here, beside the jobs
  std::vector<cudaStream_t> copy_free;     // fetch copies: one stream per fetch in progress
  std::vector<cudaStream_t> copy_all;
  int* cancel_word = nullptr;              // pinned LRA_ECANCELED, copied over a job's status
  int sms = 0;
  int max_grid = 0;  // CTAs per maxvol launch at most
  size_t smem_optin = 0;
  int max_slots = 64;
  uint64_t budget = 0;
  uint64_t used_bytes = 0;
  JobStatus* pinned = nullptr;  // one result slot per job slot
  // pinned staging of each slot's submit-time inputs (status, barrier, J,
  // residual sample), copied to the device in one asynchronous copy
  std::vector<unsigned char*> stage;
  std::vector<size_t> stage_cap;
  // the jobs' device memory: a pool of this context that keeps what it has
  // (no return to the system at each synchronisation) and reuses a block
  // only once its free has run (no waits between the streams)
  cudaMemPool_t pool = nullptr;
  std::vector<int> free_slots;
  std::mutex mu;
  std::unordered_map<lra_job, Job*> jobs;
  lra_job next_id = 1;
  std::string last_error;
  cublasHandle_t blas = nullptr;   // the range finder's V = U^T M, created on first use
};

int lra::ctx_device(lra_ctx* ctx) { return ctx->device; }

void lra::set_ctx_error(lra_ctx* ctx, const char* msg) {
  std::lock_guard<std::mutex> lock(ctx->mu);
  ctx->last_error = msg;
}

cudaError_t lra::smem_optin(const void* func, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void*, int>, int>> done;  // (func, device) -> bytes
  std::lock_guard<std::mutex> lock(mu);
  for (auto& d : done)
    if (d.first.first == func && d.first.second == dev && d.second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (!e) done.push_back({{func, dev}, bytes});
  return e;
}

namespace {

lra_status fail(lra_ctx* ctx, lra_status code, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return code;
}

lra_status cuda_fail(lra_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? LRA_ENOMEM : LRA_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

lra_status validate_source(const lra_source* src, std::string* why) {
  if (!src) { *why = "null source"; return LRA_EINVAL; }
  if (src->kind < LRA_DENSE_F32 || src->kind > LRA_PRE_AH) { *why = "unknown source kind"; return LRA_EINVAL; }
  if (src->m < 1 || src->n < 1 || src->m > (1LL << 30) || src->n > (1LL << 30)) { *why = "bad matrix size"; return LRA_EINVAL; }
  if (src->kind == LRA_PRE_AH) {
    if (!src->a || src->lda < src->n) { *why = "pre-processed source needs a and lda >= n"; return LRA_EINVAL; }
    if (src->pre_d < 0 || src->pre_d > kMaxPreD) { *why = "pre_d must be in 0..10"; return LRA_EINVAL; }
    if ((src->m % (1LL << src->pre_d)) != 0 || (src->n % (1LL << src->pre_d)) != 0) {
      *why = "2^pre_d must divide m and n"; return LRA_EINVAL;
    }
    if (!src->pre_perm_rows || !src->pre_sign_rows || !src->pre_perm_cols || !src->pre_sign_cols) {
      *why = "pre-processed source needs its permutations and signs"; return LRA_EINVAL;
    }
  } else if (src->kind <= LRA_DENSE_F64) {
    if (!src->a || src->lda < src->n) { *why = "dense source needs a and lda >= n"; return LRA_EINVAL; }
  } else {
    if (!src->x || !src->y) { *why = "generator needs x and y"; return LRA_EINVAL; }
    if (src->kind != LRA_GEN_CAUCHY && (src->dim < 1 || src->dim > 3)) { *why = "dim must be 1..3"; return LRA_EINVAL; }
    if (src->kind == LRA_GEN_GAUSS && !(src->h > 0.0f)) { *why = "h must be > 0"; return LRA_EINVAL; }
  }
  return LRA_OK;
}

// Validation shared by submit and footprint.
lra_status validate(const lra_source* src, const lra_params* p, std::string* why) {
  if (!src || !p) { *why = "null argument"; return LRA_EINVAL; }
  const lra_status vs = validate_source(src, why);
  if (vs != LRA_OK) return vs;
  if (p->l < 1 || p->l > kMaxL) { *why = "l must be in 1..96"; return LRA_EINVAL; }
  if (p->k < 1 || p->k > p->l) { *why = "k must be in 1..l"; return LRA_EINVAL; }
  if (p->l > src->m || p->l > src->n) { *why = "l exceeds min(m, n)"; return LRA_EINVAL; }
  if (p->sweeps < 1 || p->sweeps > 1000) { *why = "sweeps must be in 1..1000"; return LRA_EINVAL; }
  if (!(p->delta > 0.0)) { *why = "delta must be > 0"; return LRA_EINVAL; }
  if (!(p->rank_tol >= 0.0)) { *why = "rank_tol must be >= 0"; return LRA_EINVAL; }
  if (p->resid_q < 0 || p->resid_s < 0 || (p->resid_q > 0) != (p->resid_s > 0)) { *why = "bad sample size"; return LRA_EINVAL; }
  if (p->resid_q > 0 && (!p->resid_rows || !p->resid_cols || p->resid_q > src->m || p->resid_s > src->n)) {
    *why = "bad sample index arrays"; return LRA_EINVAL;
  }
  if (p->tol > 0.0 && p->resid_q == 0) { *why = "tol needs a residual sample"; return LRA_EINVAL; }
  if (p->trace_cap < 0) { *why = "trace_cap must be >= 0"; return LRA_EINVAL; }
  if (p->flags & LRA_FLAG_FULL_RESIDUAL) {
    if (src->kind != LRA_DENSE_F32 || src->lda % 4 != 0 ||
        (reinterpret_cast<uintptr_t>(src->a) & 15) != 0) {
      *why = "full residual needs a dense FP32 source with lda % 4 == 0 and a 16-byte aligned base";
      return LRA_EINVAL;
    }
  }
  return LRA_OK;
}

size_t layout_bytes(const lra_source* src, const lra_params* p, Job* j) {
  const int l = p->l;
  const long long q = p->resid_q, s = p->resid_s;
  Layout L;
  // the inputs copied at submit come first, as one contiguous prefix
  const size_t o_js = L.take(sizeof(JobStatus));
  const size_t o_bar = L.take(sizeof(GridBarrier));
  const size_t o_J = L.take(sizeof(int) * l);
  const size_t o_rows = L.take(sizeof(int) * std::max<long long>(q, 1));
  const size_t o_cols = L.take(sizeof(int) * std::max<long long>(s, 1));
  const size_t o_ring = L.take(sizeof(unsigned long long) * kWinRing);
  const size_t o_I = L.take(sizeof(int) * l);
  const size_t prefix = L.off;
  const size_t o_x0 = L.take(sizeof(float2) * l * l);
  const size_t o_x1 = L.take(sizeof(float2) * l * l);
  const size_t o_U = L.take(sizeof(double) * l * l);
  const size_t o_sig = L.take(sizeof(double) * l);
  const size_t o_candr = L.take(sizeof(float2) * 2 * kMaxGrid * l);
  const size_t o_ti = L.take(sizeof(int) * 4 * std::max(p->trace_cap, 1));
  const size_t o_tv = L.take(sizeof(double) * std::max(p->trace_cap, 1));
  const int np = q > 0 ? sampled_residual_partials((int)q, (int)s) : 1;
  const size_t o_cuq = L.take(sizeof(float) * std::max<long long>(2 * q * l, 1));
  const size_t o_part = L.take(sizeof(double) * 3 * np);
  const size_t o_C = L.take(sizeof(float) * (size_t)src->m * l);
  const size_t o_R = L.take(sizeof(float) * (size_t)src->n * l);
  const bool fr = (p->flags & LRA_FLAG_FULL_RESIDUAL) != 0;
  const size_t o_fr = fr ? L.take(fullres_workspace_bytes(src->m, src->n, l, kMaxGrid)) : 0;
  if (j) {
    unsigned char* b = j->dmem;
    j->js = reinterpret_cast<JobStatus*>(b + o_js);
    j->bar = reinterpret_cast<GridBarrier*>(b + o_bar);
    j->J = reinterpret_cast<int*>(b + o_J);
    j->I = reinterpret_cast<int*>(b + o_I);
    j->xbuf0 = reinterpret_cast<float2*>(b + o_x0);
    j->xbuf1 = reinterpret_cast<float2*>(b + o_x1);
    j->U = reinterpret_cast<double*>(b + o_U);
    j->sigma = reinterpret_cast<double*>(b + o_sig);
    j->win_ring = reinterpret_cast<unsigned long long*>(b + o_ring);
    j->cand_rows = reinterpret_cast<float2*>(b + o_candr);
    j->trace_i = reinterpret_cast<int*>(b + o_ti);
    j->trace_v = reinterpret_cast<double*>(b + o_tv);
    j->rows = reinterpret_cast<int*>(b + o_rows);
    j->cols = reinterpret_cast<int*>(b + o_cols);
    j->CUq = reinterpret_cast<float*>(b + o_cuq);
    j->partials = reinterpret_cast<double*>(b + o_part);
    j->C = reinterpret_cast<float*>(b + o_C);
    j->R = reinterpret_cast<float*>(b + o_R);
    j->n_partials = np;
    j->fr_ws = fr ? (void*)(b + o_fr) : nullptr;
    j->prefix = prefix;
  }
  return L.off;
}

// Initial column set drawn from a seed (Section 12.2: the C-A tests start
// from a random set of columns).  Generator: SplitMix64 (Steele, Lea and
// Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
// state = seed, each draw adds 0x9E3779B97F4A7C15 to the state and mixes it.
// Sample: Floyd's algorithm (Bentley and Floyd, "A sample of brilliance",
// CACM 1987) for l distinct values of [0, n): for c = n - l ... n - 1 take
// t = draw mod (c + 1), then t if it is new, else c.  J0 lists the values in
// the order they were taken.
uint64_t splitmix64_next(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void draw_columns(uint64_t seed, long long n, int l, int32_t* out) {
  uint64_t state = seed;
  std::unordered_set<long long> taken;
  int cnt = 0;
  for (long long c = n - l; c < n; ++c) {
    const long long t = (long long)(splitmix64_next(&state) % (uint64_t)(c + 1));
    const long long v = taken.count(t) ? c : t;
    taken.insert(v);
    out[cnt++] = (int32_t)v;
  }
}

// count indices, each in [0, bound), no two equal.  Values up to 2^22 are
// marked in a per-thread stamp array (one generation number per call, so
// nothing is cleared between calls): O(count), which matters where a batch
// checks thousands of small index sets on the submitting thread.
bool distinct_in_range(const int32_t* v, long long count, long long bound) {
  for (long long i = 0; i < count; ++i)
    if (v[i] < 0 || v[i] >= bound) return false;
  long long vmax = -1;
  for (long long i = 0; i < count; ++i) vmax = std::max<long long>(vmax, v[i]);
  if (vmax < (1LL << 22)) {
    thread_local std::vector<uint32_t> stamp;
    thread_local uint32_t gen = 0;
    if ((long long)stamp.size() <= vmax) stamp.resize((size_t)vmax + 1, 0u);
    if (++gen == 0) {   // wrapped: start over
      std::fill(stamp.begin(), stamp.end(), 0u);
      gen = 1;
    }
    for (long long i = 0; i < count; ++i) {
      if (stamp[v[i]] == gen) return false;
      stamp[v[i]] = gen;
    }
    return true;
  }
  std::vector<int32_t> s(v, v + count);
  std::sort(s.begin(), s.end());
  return std::adjacent_find(s.begin(), s.end()) == s.end();
}

// Device memory goes back to the pool on the control stream behind the job's
// end: on the job's own stream the free would also wait for the jobs queued
// after it, and the pool could not hand the block to another job meanwhile.
void release_job(lra_ctx* ctx, Job* j) {
  if (j->dmem) {
    cudaStream_t fs = ctx->ctrl ? ctx->ctrl : j->stream;
    if (fs != j->stream && j->ev_end) cudaStreamWaitEvent(fs, j->ev_end, 0);
    cudaFreeAsync(j->dmem, fs);
  }
  if (j->stream_idx >= 0) ctx->stream_load[j->stream_idx]--;
  if (j->ev_start) cudaEventDestroy(j->ev_start);
  if (j->ev_end) cudaEventDestroy(j->ev_end);
  for (auto& pe : j->prof) cudaEventDestroy(pe.second);
  ctx->used_bytes -= j->bytes;
  if (j->slot >= 0) ctx->free_slots.push_back(j->slot);
  delete j;
}

// Enqueue the whole solve of one job on the context stream.
cudaError_t enqueue_solve(lra_ctx* ctx, Job* j, const lra_params* p) {
  cudaStream_t st = j->stream;
  cudaError_t e;
  JobStatus init{};
  init.status = LRA_OK;
  init.converged = 1;
  init.trace_cap = j->trace_cap;
  // status, grid barrier, J, the residual sample and the zeroed maxvol
  // candidate words: staged in the slot's pinned
  // buffer (free again only once this job is released) and sent in one copy
  if (ctx->stage_cap[j->slot] < j->prefix) {
    if (ctx->stage[j->slot]) cudaFreeHost(ctx->stage[j->slot]);
    ctx->stage[j->slot] = nullptr;
    ctx->stage_cap[j->slot] = 0;
    void* h = nullptr;
    if ((e = cudaMallocHost(&h, j->prefix))) return e;
    ctx->stage[j->slot] = static_cast<unsigned char*>(h);
    ctx->stage_cap[j->slot] = j->prefix;
  }
  unsigned char* hs = ctx->stage[j->slot];
  auto at = [&](const void* dev) { return hs + (static_cast<const unsigned char*>(dev) - j->dmem); };
  std::memset(hs, 0, j->prefix);
  std::memcpy(at(j->js), &init, sizeof(init));
  if (p->init_J) {
    std::memcpy(at(j->J), p->init_J, sizeof(int) * j->l);
  } else {
    std::vector<int32_t> J0(j->l);
    draw_columns(p->seed, j->n, j->l, J0.data());
    std::memcpy(at(j->J), J0.data(), sizeof(int) * j->l);
  }
  if (p->init_I) std::memcpy(at(j->I), p->init_I, sizeof(int) * j->l);
  if (j->q > 0) {
    std::memcpy(at(j->rows), p->resid_rows, sizeof(int) * j->q);
    std::memcpy(at(j->cols), p->resid_cols, sizeof(int) * j->s);
  }
  if ((e = cudaMemcpyAsync(j->dmem, hs, j->prefix, cudaMemcpyHostToDevice, st))) return e;
  MaxvolArgs col{};
  col.strip = j->C; col.N = j->m; col.l = j->l; col.si = j->l; col.st = 1;
  col.pos = j->I; col.win_ring = j->win_ring; col.cand_rows = j->cand_rows; col.bar = j->bar;
  col.js = j->js; col.trace_i = j->trace_i; col.trace_v = j->trace_v;
  col.delta = j->delta; col.max_swaps = j->max_swaps;
  MaxvolArgs row = col;
  row.strip = j->R; row.N = j->n; row.si = 1; row.st = j->n; row.pos = j->J;

  // after(cls, n): n kernels of class cls were just enqueued
  auto after = [&](int cls, int n) -> cudaError_t {
    j->launches += n;
    if (cls == kClsMaxvol) j->maxvol_launches += n;
    if (!j->profile) return cudaSuccess;
    cudaEvent_t ev;
    cudaError_t r = cudaEventCreate(&ev);
    if (r) return r;
    j->prof.emplace_back(cls, ev);
    return cudaEventRecord(ev, st);
  };
  // with several own streams the jobs overlap: the separate single-SM
  // inverse then leaves the other SMs to them.  With one stream the cross
  // inverse is on the critical path of the job: the maxvol grid computes it
  // itself when it fits on chip beside the strip (no separate launch).
  const bool one_sm = ctx->streams.size() > 1;
  const bool self_col = !one_sm && j->plan_col.stage_xinv;
  const bool self_row = !one_sm && j->plan_row.stage_xinv;
  col.self_inverse = self_col;
  row.self_inverse = self_row;
  // generator sources, one stream, no per-sweep tolerance test: the maxvol
  // launches evaluate their strips themselves (no gather launches and no
  // strip in HBM between half-steps); C and R are gathered once at the end
  const bool gen = j->src.kind >= LRA_GEN_CAUCHY && j->src.kind <= LRA_GEN_INVDIST && j->tol == 0.0 &&
                   self_col && self_row;
  // a fixed budget of sweeps: stop at a fixed point of the iteration
  col.fixed_point_exit = row.fixed_point_exit = j->tol == 0.0;
  col.total_half_steps = row.total_half_steps = 2 * j->sweeps;
  if (gen) {
    col.gen = 1;
    col.gen_idx = j->J;
    col.src = j->src;
    row.gen = 2;
    row.gen_idx = j->I;
    row.src = j->src;
  }
  // C = M[:, J]: through TMA tiles for a stored FP32 matrix, else entry by entry
  auto gather_c = [&](int skip_on_stop) -> cudaError_t {
    cudaError_t r = j->tma_cols
                        ? launch_gather_cols_tma(j->col_map, j->J, j->l, j->m, j->C, j->js, skip_on_stop, ctx->sms, st)
                        : launch_gather_cols(j->src, j->J, j->l, j->C, j->js, skip_on_stop, ctx->sms, st);
    return r ? r : after(kClsGather, 1);
  };
  if ((e = cudaEventRecord(j->ev_start, st))) return e;
  for (int sw = 0; sw < j->sweeps; ++sw) {
    if (!gen && (e = gather_c(1))) return e;
    // the very first vertical step starts from Gaussian elimination, unless
    // the caller resumes from its own row set (init_I): then it is a warm
    // start like every later one
    col.gepp = (sw == 0 && !j->resume);
    col.half_step = 2 * sw;
    col.xin = j->xbuf0;   // inverse of A[I, J] (vertical strip's cross)
    if (!col.gepp && !self_col) {
      if ((e = launch_cross_inverse(j->C, j->l, 1, j->I, j->l, j->xbuf0, j->js, st, !one_sm)) ||
          (e = after(kClsInverse, 1))) return e;
    }
    if ((e = launch_maxvol(col, j->plan_col, st)) || (e = after(kClsMaxvol, 1))) return e;
    if (!gen &&
        ((e = launch_gather_rows(j->src, j->I, j->l, j->R, j->js, ctx->sms, st)) || (e = after(kClsGather, 1))))
      return e;
    row.gepp = 0;
    row.half_step = 2 * sw + 1;
    row.xin = j->xbuf1;   // inverse of A[I, J]^T (horizontal strip's cross)
    if (!self_row && ((e = launch_cross_inverse(j->R, 1, j->n, j->J, j->l, j->xbuf1, j->js, st, !one_sm)) ||
                      (e = after(kClsInverse, 1)))) return e;
    row.count_sweep = 1;   // the sweep is counted by the row maxvol that completes it
    if ((e = launch_maxvol(row, j->plan_row, st)) || (e = after(kClsMaxvol, 1))) return e;
    if (j->tol > 0.0 && sw + 1 < j->sweeps) {
      if ((e = gather_c(1))) return e;
      if ((e = launch_nucleus(j->C, j->I, j->l, j->k, j->rank_tol, j->U, j->sigma, j->js, st, NucExtra(), !one_sm)) || (e = after(kClsCross, 1))) return e;
      if ((e = launch_sampled_residual(j->src, j->rows, (int)j->q, j->cols, (int)j->s, j->l, j->C, j->U,
                                       j->R, j->CUq, j->partials, j->n_partials, j->js, st)) ||
          (e = after(kClsResid, 3))) return e;
      if ((e = launch_tol_check(j->js, j->tol, st)) || (e = after(kClsOther, 1))) return e;
    }
  }
  // final strips for the returned CUR: C = M[:, J] (R = M[I, :] is current,
  // unless the strips were evaluated inside the maxvol launches)
  if ((e = gather_c(0))) return e;
  if (gen &&
      ((e = launch_gather_rows(j->src, j->I, j->l, j->R, j->js, ctx->sms, st, 0)) || (e = after(kClsGather, 1))))
    return e;
  if ((e = launch_nucleus(j->C, j->I, j->l, j->k, j->rank_tol, j->U, j->sigma, j->js, st, NucExtra(), !one_sm)) || (e = after(kClsCross, 1))) return e;
  if (j->full_res) {
    if ((e = launch_full_residual(static_cast<const float*>(j->src.a), j->src.lda, j->m, j->n, j->l, j->C,
                                  j->U, j->R, j->fr_ws, std::min(ctx->sms, kMaxGrid), j->js, st)) ||
        (e = after(kClsFullres, 5))) return e;
  }
  if (j->q > 0) {
    if ((e = launch_sampled_residual(j->src, j->rows, (int)j->q, j->cols, (int)j->s, j->l, j->C, j->U,
                                     j->R, j->CUq, j->partials, j->n_partials, j->js, st)) ||
        (e = after(kClsResid, 3))) return e;
  }
  if ((e = cudaMemcpyAsync(ctx->pinned + j->slot, j->js, sizeof(JobStatus), cudaMemcpyDeviceToHost, st))) return e;
  return cudaEventRecord(j->ev_end, st);
}

void fill_info(lra_ctx* ctx, Job* j, lra_info* out) {
  const JobStatus& h = ctx->pinned[j->slot];
  std::memset(out, 0, sizeof(*out));
  out->status = h.status;
  out->state = h.status == LRA_OK ? LRA_STATE_DONE : LRA_STATE_FAILED;
  out->sweeps_done = h.sweeps_done;
  out->k_eff = h.k_eff;
  out->swaps_total = h.swaps_total;
  out->converged = h.converged;
  out->trace_len = h.trace_len;
  out->est_rel_err = j->q > 0 ? h.est_rel : -1.0;
  out->est_mu = h.est_mu;
  out->est_var = h.est_var;
  out->sigma_max = h.sigma_max;
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, j->ev_start, j->ev_end) == cudaSuccess) out->gpu_ms = ms;
  out->kernel_launches = j->launches;
  out->maxvol_launches = j->maxvol_launches;
  out->maxvol_flops = h.maxvol_flops;
  double t[7] = {0, 0, 0, 0, 0, 0, 0};
  cudaEvent_t prev = j->ev_start;
  for (auto& pe : j->prof) {
    float d = 0.0f;
    if (cudaEventElapsedTime(&d, prev, pe.second) == cudaSuccess) t[pe.first] += d;
    prev = pe.second;
  }
  out->t_gather_ms = t[kClsGather];
  out->t_maxvol_ms = t[kClsMaxvol];
  out->t_cross_ms = t[kClsCross];
  out->t_resid_ms = t[kClsResid];
  out->t_inverse_ms = t[kClsInverse];
  out->t_fullres_ms = t[kClsFullres];
  out->full_rel_err = j->full_res ? h.full_rel : -1.0;
}

SourceDev make_src(const lra_source* src) {
  SourceDev d{};
  d.kind = src->kind;
  d.dim = src->kind == LRA_GEN_CAUCHY ? 1 : src->dim;
  d.m = src->m;
  d.n = src->n;
  d.a = src->a;
  d.lda = src->lda;
  d.x = src->x;
  d.y = src->y;
  d.h2 = src->h * src->h;
  if (src->kind == LRA_PRE_AH) {
    d.pre_d = src->pre_d;
    d.pre_mat = src->pre_materialized != 0;
    d.pre_sm = src->m >> src->pre_d;
    d.pre_sn = src->n >> src->pre_d;
    d.pre_pr = src->pre_perm_rows;
    d.pre_sr = src->pre_sign_rows;
    d.pre_pc = src->pre_perm_cols;
    d.pre_sc = src->pre_sign_cols;
  }
  return d;
}

// Least-loaded context stream for a new job (ties: lowest index).
void assign_stream(lra_ctx* ctx, Job* j) {
  size_t best = 0;
  for (size_t i = 1; i < ctx->streams.size(); ++i)
    if (ctx->stream_load[i] < ctx->stream_load[best]) best = i;
  j->stream_idx = (int)best;
  j->stream = ctx->streams[best];
  ctx->stream_load[best]++;
}

// A copy stream for one fetch (caller holds ctx->mu).  Fetches in
// progress on different threads each get their own, created on first need.
cudaStream_t take_copy_stream(lra_ctx* ctx) {
  if (!ctx->copy_free.empty()) {
    cudaStream_t s = ctx->copy_free.back();
    ctx->copy_free.pop_back();
    return s;
  }
  cudaStream_t s = nullptr;
  cudaSetDevice(ctx->device);
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) return ctx->ctrl;
  ctx->copy_all.push_back(s);
  return s;
}

void give_copy_stream(lra_ctx* ctx, cudaStream_t s) {
  if (s && s != ctx->ctrl) ctx->copy_free.push_back(s);
}

Job* find_job(lra_ctx* ctx, lra_job id) {
  auto it = ctx->jobs.find(id);
  return it == ctx->jobs.end() ? nullptr : it->second;
}

}  // namespace

extern "C" {

const char* lra_status_str(int32_t s) {
  switch (s) {
    case LRA_OK: return "ok";
    case LRA_PENDING: return "pending";
    case LRA_EINVAL: return "invalid argument";
    case LRA_ENOMEM: return "out of device memory";
    case LRA_EBUSY: return "admission refused (slots or memory budget)";
    case LRA_ESINGULAR: return "singular strip (no nonsingular l x l submatrix)";
    case LRA_ENONFINITE: return "non-finite matrix entry";
    case LRA_ETIMEOUT: return "device wait timed out";
    case LRA_ECUDA: return "CUDA error";
    case LRA_ENOTFOUND: return "unknown job";
    case LRA_ECANCELED: return "cancelled";
    case LRA_ETOOLARGE: return "strip too large for the on-chip working set";
    default: return "unknown status";
  }
}

const char* lra_cross_last_error(lra_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

lra_status lra_cross_create(lra_ctx** out, const lra_ctx_params* params) {
  if (!out || !params) return LRA_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return LRA_ECUDA;
  if (params->device < 0 || params->device >= ndev) return LRA_EINVAL;
  lra_ctx* ctx = new lra_ctx();
  ctx->device = params->device;
  ctx->max_slots = params->max_slots > 0 ? params->max_slots : 64;
  ctx->budget = params->mem_budget_bytes;
  cudaError_t e = cudaSetDevice(ctx->device);
  cudaDeviceProp prop{};
  if (!e) e = cudaGetDeviceProperties(&prop, ctx->device);
  if (e) { delete ctx; return LRA_ECUDA; }
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
  if (!coop) { delete ctx; return LRA_ECUDA; }
  ctx->sms = prop.multiProcessorCount;
  ctx->max_grid = params->max_grid > 0 ? std::min(params->max_grid, ctx->sms) : ctx->sms;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  if (params->stream) {
    ctx->stream = static_cast<cudaStream_t>(params->stream);
    ctx->streams.push_back(ctx->stream);
  } else {
    // own streams: jobs submitted while others run go to the least loaded
    // stream, so their kernels overlap on the device
    const int ns = std::max(1, std::min(32, params->n_streams));
    for (int i = 0; i < ns; ++i) {
      cudaStream_t s;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) {
        for (cudaStream_t t : ctx->streams) cudaStreamDestroy(t);
        delete ctx;
        return LRA_ECUDA;
      }
      ctx->streams.push_back(s);
    }
    ctx->stream = ctx->streams[0];
    ctx->own_stream = true;
  }
  ctx->stream_load.assign(ctx->streams.size(), 0);
  if (cudaMallocHost(&ctx->pinned, sizeof(JobStatus) * ctx->max_slots)) {
    if (ctx->own_stream)
      for (cudaStream_t t : ctx->streams) cudaStreamDestroy(t);
    delete ctx;
    return LRA_ENOMEM;
  }
  ctx->stage.assign(ctx->max_slots, nullptr);
  ctx->stage_cap.assign(ctx->max_slots, 0);
  cudaMemPoolProps pp{};
  pp.allocType = cudaMemAllocationTypePinned;
  pp.location.type = cudaMemLocationTypeDevice;
  pp.location.id = ctx->device;
  if (cudaMemPoolCreate(&ctx->pool, &pp)) {
    cudaFreeHost(ctx->pinned);
    if (ctx->own_stream)
      for (cudaStream_t t : ctx->streams) cudaStreamDestroy(t);
    delete ctx;
    return LRA_ECUDA;
  }
  uint64_t keep = ~0ULL;
  int no = 0;
  cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  for (int s = ctx->max_slots - 1; s >= 0; --s) ctx->free_slots.push_back(s);
  if (cudaStreamCreateWithFlags(&ctx->ctrl, cudaStreamNonBlocking)) ctx->ctrl = nullptr;
  if (cudaMallocHost(&ctx->cancel_word, sizeof(int))) ctx->cancel_word = nullptr;
  else *ctx->cancel_word = LRA_ECANCELED;
  *out = ctx;
  return LRA_OK;
}

lra_status lra_cross_destroy(lra_ctx* ctx) {
  if (!ctx) return LRA_EINVAL;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaSetDevice(ctx->device);
    for (cudaStream_t s : ctx->streams) cudaStreamSynchronize(s);
    for (auto& kv : ctx->jobs) release_job(ctx, kv.second);
    ctx->jobs.clear();
    for (cudaStream_t s : ctx->streams) cudaStreamSynchronize(s);
    if (ctx->own_stream)
      for (cudaStream_t s : ctx->streams) cudaStreamDestroy(s);
    if (ctx->ctrl) {
      cudaStreamSynchronize(ctx->ctrl);
      cudaStreamDestroy(ctx->ctrl);
    }
    for (cudaStream_t s : ctx->copy_all) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    if (ctx->cancel_word) cudaFreeHost(ctx->cancel_word);
    for (unsigned char* h : ctx->stage)
      if (h) cudaFreeHost(h);
    cudaFreeHost(ctx->pinned);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->blas) cublasDestroy(ctx->blas);
  }
  delete ctx;
  return LRA_OK;
}

lra_status lra_cross_footprint(const lra_source* src, const lra_params* params, uint64_t* bytes) {
  std::string why;
  lra_status s = validate(src, params, &why);
  if (s != LRA_OK) return s;
  if (!bytes) return LRA_EINVAL;
  *bytes = layout_bytes(src, params, nullptr);
  return LRA_OK;
}

lra_status lra_cross_submit(lra_ctx* ctx, const lra_source* src, const lra_params* p, lra_job* out) {
  if (!ctx || !out) return LRA_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  std::string why;
  lra_status s = validate(src, p, &why);
  if (s != LRA_OK) return fail(ctx, s, why);
  if (p->init_J && !distinct_in_range(p->init_J, p->l, src->n))
    return fail(ctx, LRA_EINVAL, "init_J must be l distinct columns");
  if (p->init_I && !distinct_in_range(p->init_I, p->l, src->m))
    return fail(ctx, LRA_EINVAL, "init_I must be l distinct rows");
  if (p->resid_q > 0 && (!distinct_in_range(p->resid_rows, p->resid_q, src->m) ||
                         !distinct_in_range(p->resid_cols, p->resid_s, src->n)))
    return fail(ctx, LRA_EINVAL, "residual sample indices must be distinct and in range");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e) return cuda_fail(ctx, e, "cudaSetDevice");

  Job* j = new Job();
  j->l = p->l; j->k = p->k; j->sweeps = p->sweeps;
  j->max_swaps = p->max_swaps > 0 ? p->max_swaps : 64 * p->l;
  j->trace_cap = p->trace_cap;
  j->profile = (p->flags & LRA_FLAG_PROFILE) != 0;
  j->full_res = (p->flags & LRA_FLAG_FULL_RESIDUAL) != 0;
  j->resume = p->init_I != nullptr;
  if (src->kind == LRA_DENSE_F32)
    j->tma_cols = make_cols_map(&j->col_map, static_cast<const float*>(src->a), src->m, src->n, src->lda);
  j->m = src->m; j->n = src->n; j->q = p->resid_q; j->s = p->resid_s;
  j->delta = p->delta; j->rank_tol = p->rank_tol; j->tol = p->tol;
  j->src = make_src(src);
  // at most max_grid CTAs, more only where the strip's chunks need them
  auto plan = [&](long long N, MaxvolPlan* pl) {
    return plan_maxvol(N, j->l, ctx->max_grid, ctx->smem_optin, pl) ||
           plan_maxvol(N, j->l, ctx->sms, ctx->smem_optin, pl);
  };
  if (!plan(j->m, &j->plan_col) || !plan(j->n, &j->plan_row)) {
    delete j;
    return fail(ctx, LRA_ETOOLARGE, "strip does not fit in the shared memory of the grid");
  }
  j->bytes = layout_bytes(src, p, nullptr);
  if ((int)ctx->jobs.size() >= ctx->max_slots || ctx->free_slots.empty() ||
      (ctx->budget && ctx->used_bytes + j->bytes > ctx->budget)) {
    delete j;
    return fail(ctx, LRA_EBUSY, "no free slot or memory budget exhausted");
  }
  assign_stream(ctx, j);
  if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&j->dmem), j->bytes, ctx->pool, j->stream))) {
    ctx->stream_load[j->stream_idx]--;
    delete j;
    return cuda_fail(ctx, e, "cudaMallocFromPoolAsync");
  }
  layout_bytes(src, p, j);
  j->slot = ctx->free_slots.back();
  ctx->free_slots.pop_back();
  ctx->used_bytes += j->bytes;
  if ((e = cudaEventCreate(&j->ev_start)) || (e = cudaEventCreate(&j->ev_end)) ||
      (e = enqueue_solve(ctx, j, p))) {
    cudaStreamSynchronize(j->stream);
    release_job(ctx, j);
    return cuda_fail(ctx, e, "enqueue");
  }
  j->id = ctx->next_id++;
  ctx->jobs[j->id] = j;
  *out = j->id;
  return LRA_OK;
}

lra_status lra_cross_poll(lra_ctx* ctx, lra_job id, lra_info* out) {
  if (!ctx || !out) return LRA_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  Job* j = find_job(ctx, id);
  if (!j) return fail(ctx, LRA_ENOTFOUND, "unknown job");
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaEventQuery(j->ev_end);
  if (e == cudaErrorNotReady) {
    std::memset(out, 0, sizeof(*out));
    out->state = LRA_STATE_RUNNING;
    out->status = LRA_PENDING;
    return LRA_PENDING;
  }
  if (e) return cuda_fail(ctx, e, "cudaEventQuery");
  fill_info(ctx, j, out);
  return LRA_OK;
}

lra_status lra_cross_wait(lra_ctx* ctx, lra_job id, lra_info* out) {
  if (!ctx || !out) return LRA_EINVAL;
  cudaEvent_t ev;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    Job* j = find_job(ctx, id);
    if (!j) return fail(ctx, LRA_ENOTFOUND, "unknown job");
    ev = j->ev_end;
    cudaSetDevice(ctx->device);
  }
  cudaError_t e = cudaEventSynchronize(ev);
  if (e) return cuda_fail(ctx, e, "cudaEventSynchronize");
  return lra_cross_poll(ctx, id, out);
}

lra_status lra_cross_fetch_cur(lra_ctx* ctx, lra_job id, const lra_cur_out* out) {
  if (!ctx || !out) return LRA_EINVAL;
  // Take the job out of the table under the lock, then wait for it with the
  // lock released: submit and poll from other threads proceed meanwhile.
  Job* j = nullptr;
  cudaStream_t cs = nullptr;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    j = find_job(ctx, id);
    if (!j) return fail(ctx, LRA_ENOTFOUND, "unknown job");
    if (j->batch) return fail(ctx, LRA_EINVAL, "batch job: use lra_cross_fetch_batch");
    ctx->jobs.erase(id);
    cs = take_copy_stream(ctx);
  }
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaEventSynchronize(j->ev_end);
  lra_status result = LRA_OK;
  std::string msg;
  if (e) {
    result = e == cudaErrorMemoryAllocation ? LRA_ENOMEM : LRA_ECUDA;
    msg = std::string("cudaEventSynchronize: ") + cudaGetErrorString(e);
  } else {
    const JobStatus& h = ctx->pinned[j->slot];   // the slot stays this job's until released
    result = (lra_status)h.status;
    if (result == LRA_OK) {
      const int l = j->l;
      struct Piece { void* dst; const void* src; size_t bytes; };
      const int tl = std::min(h.trace_len, j->trace_cap);
      Piece pieces[] = {
          {out->I, j->I, sizeof(int) * l},
          {out->J, j->J, sizeof(int) * l},
          {out->U, j->U, sizeof(double) * l * l},
          {out->sigma, j->sigma, sizeof(double) * l},
          {out->C, j->C, sizeof(float) * (size_t)j->m * l},
          {out->R, j->R, sizeof(float) * (size_t)j->n * l},
          {out->trace, j->trace_i, sizeof(int) * 4 * (size_t)tl},
          {out->trace_val, j->trace_v, sizeof(double) * (size_t)tl},
      };
      // the job has ended: the copies run on a copy stream of the context
      // that no other call uses meanwhile, so they wait for nothing else
      for (const Piece& pc : pieces) {
        if (e) break;
        if (!pc.dst || pc.bytes == 0) continue;
        e = cudaMemcpyAsync(pc.dst, pc.src, pc.bytes, cudaMemcpyDefault, cs);
      }
      if (!e) e = cudaStreamSynchronize(cs);
      if (e) {
        result = e == cudaErrorMemoryAllocation ? LRA_ENOMEM : LRA_ECUDA;
        msg = std::string("fetch copy: ") + cudaGetErrorString(e);
      }
    } else {
      msg = lra_status_str(result);
    }
  }
  std::lock_guard<std::mutex> lock(ctx->mu);
  give_copy_stream(ctx, cs);
  release_job(ctx, j);
  if (result != LRA_OK) fail(ctx, result, msg);
  return result;
}

lra_status lra_cross_cancel(lra_ctx* ctx, lra_job id) {
  if (!ctx) return LRA_EINVAL;
  Job* j = nullptr;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    j = find_job(ctx, id);
    if (!j) return fail(ctx, LRA_ENOTFOUND, "unknown job");
    ctx->jobs.erase(id);
    cudaSetDevice(ctx->device);
    // a job still running is marked cancelled: a copy engine writes
    // LRA_ECANCELED over its status word from the control stream, beside the
    // job's queued kernels, which then return at their start (kernels already
    // running finish)
    if (cudaEventQuery(j->ev_end) == cudaErrorNotReady && ctx->ctrl && ctx->cancel_word)
      cudaMemcpyAsync(&j->js->status, ctx->cancel_word, sizeof(int), cudaMemcpyHostToDevice, ctx->ctrl);
  }
  // wait for the job's stream work with the lock released
  cudaSetDevice(ctx->device);
  cudaEventSynchronize(j->ev_end);
  std::lock_guard<std::mutex> lock(ctx->mu);
  release_job(ctx, j);
  return LRA_OK;
}

// Algorithm 5.1a with a sub-identity multiplier (see the header).
lra_status lra_range_finder(lra_ctx* ctx, const lra_source* src, const int32_t* J, int32_t l,
                            const lra_rf_params* p, const lra_rf_out* out) {
  if (!ctx || !src || !J || !p || !out || !out->U || !out->V || !out->piv || !out->nrank) return LRA_EINVAL;
  std::string why;
  if (validate_source(src, &why) != LRA_OK) return fail(ctx, LRA_EINVAL, why);
  if (src->kind != LRA_DENSE_F32) return fail(ctx, LRA_EINVAL, "range finder: V = U^T M needs a stored FP32 matrix");
  const long long m = src->m, n = src->n;
  const int r = p->r, q = (int)p->resid_q, sN = (int)p->resid_s;
  if (l < 1 || l > kMaxL || l > n || l > m || r < 1 || r > l || !(p->rank_tol >= 0.0) || p->resid_q < 0 ||
      p->resid_s < 0 || (p->resid_q > 0) != (p->resid_s > 0) ||
      (p->resid_q > 0 && (!p->resid_rows || !p->resid_cols || p->resid_q > m || p->resid_s > n)))
    return fail(ctx, LRA_EINVAL, "range finder: bad sizes");
  if (!distinct_in_range(J, l, n)) return fail(ctx, LRA_EINVAL, "range finder: J must hold l distinct columns");
  const int md = p->mult_d;
  if (md < 0 || md > kMaxPreD || (n % (1LL << md)) != 0)
    return fail(ctx, LRA_EINVAL, "range finder: mult_d must be in 0..10 with 2^mult_d dividing n");
  if (md > 0 && p->mult_sign)
    for (int t = 0; t < l; ++t)
      if (p->mult_sign[t] != 1.0f && p->mult_sign[t] != -1.0f)
        return fail(ctx, LRA_EINVAL, "range finder: multiplier signs must be +1 or -1");
  if (q > 0 && (!distinct_in_range(p->resid_rows, q, m) || !distinct_in_range(p->resid_cols, sN, n)))
    return fail(ctx, LRA_EINVAL, "range finder: residual sample indices must be distinct and in range");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e) return cuda_fail(ctx, e, "cudaSetDevice");
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!ctx->blas && cublasCreate(&ctx->blas) != CUBLAS_STATUS_SUCCESS) {
      ctx->blas = nullptr;
      ctx->last_error = "range finder: cublasCreate failed";
      return LRA_ECUDA;
    }
  }
  const int nch = ts_gram_chunks(m, l), nch2 = ts_gram_chunks(m, r);
  const int nres = q > 0 ? sampled_residual_partials(q, sN) : 1;
  Layout lay;
  const size_t o_js = lay.take(sizeof(JobStatus)), o_J = lay.take(sizeof(int) * l);
  const size_t o_sr = lay.take(sizeof(int) * std::max(q, 1)), o_sc = lay.take(sizeof(int) * std::max(sN, 1));
  const size_t o_I = lay.take(sizeof(double) * r * r);   // identity nucleus for the estimate
  const size_t o_sg = lay.take(sizeof(float) * l);       // multiplier signs
  const size_t prefix = lay.off;
  const size_t o_Y = lay.take(sizeof(float) * (size_t)m * l);
  const size_t o_p1 = lay.take(sizeof(double) * (size_t)nch * l * l);
  const size_t o_Gm = lay.take(sizeof(double) * l * r), o_piv = lay.take(sizeof(int) * l);
  const size_t o_Q1 = lay.take(sizeof(double) * (size_t)m * r);
  const size_t o_p2 = lay.take(sizeof(double) * (size_t)nch2 * r * r), o_Li = lay.take(sizeof(double) * r * r);
  const size_t o_cuq = lay.take(sizeof(float) * std::max<size_t>(2 * (size_t)q * r, 1));
  const size_t o_pr = lay.take(sizeof(double) * 3 * nres);
  const size_t bytes = lay.off;
  cudaStream_t st = ctx->stream;
  unsigned char* b = nullptr;
  if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&b), bytes, ctx->pool, st)))
    return cuda_fail(ctx, e, "cudaMallocFromPoolAsync");
  auto P = [&](size_t o) { return b + o; };
  JobStatus* js = reinterpret_cast<JobStatus*>(P(o_js));
  int* dJ = reinterpret_cast<int*>(P(o_J));
  int *dsr = reinterpret_cast<int*>(P(o_sr)), *dsc = reinterpret_cast<int*>(P(o_sc));
  double* Ir = reinterpret_cast<double*>(P(o_I));
  float* Y = reinterpret_cast<float*>(P(o_Y));
  double *p1 = reinterpret_cast<double*>(P(o_p1)), *Gm = reinterpret_cast<double*>(P(o_Gm));
  int* dpiv = reinterpret_cast<int*>(P(o_piv));
  double *Q1 = reinterpret_cast<double*>(P(o_Q1)), *p2 = reinterpret_cast<double*>(P(o_p2));
  double* Linv = reinterpret_cast<double*>(P(o_Li));
  float* cuq = reinterpret_cast<float*>(P(o_cuq));
  double* rpart = reinterpret_cast<double*>(P(o_pr));
  std::vector<unsigned char> hs(prefix, 0);
  JobStatus init{};
  init.status = LRA_OK;
  std::memcpy(hs.data() + o_js, &init, sizeof(init));
  std::memcpy(hs.data() + o_J, J, sizeof(int) * l);
  if (q > 0) {
    std::memcpy(hs.data() + o_sr, p->resid_rows, sizeof(int) * q);
    std::memcpy(hs.data() + o_sc, p->resid_cols, sizeof(int) * sN);
  }
  for (int t = 0; t < r; ++t) {
    const double one = 1.0;
    std::memcpy(hs.data() + o_I + sizeof(double) * ((size_t)t * r + t), &one, sizeof(double));
  }
  for (int t = 0; t < l; ++t) {
    const float sg = (md > 0 && p->mult_sign) ? p->mult_sign[t] : 1.0f;
    std::memcpy(hs.data() + o_sg + sizeof(float) * t, &sg, sizeof(float));
  }
  const float* dsg = reinterpret_cast<const float*>(b + o_sg);
  const SourceDev sd = make_src(src);
  TmaMap cmap{};
  const bool tma = make_cols_map(&cmap, static_cast<const float*>(src->a), m, n, src->lda);
  JobStatus hjs{};
  std::vector<int> hpiv(l, 0);
  // Y = M[:, J]; rank-revealing QR of Y; Q1 = Y(:, piv[:r]) R_r^{-1} and its Gram
  if (!(e = cudaMemcpyAsync(b, hs.data(), prefix, cudaMemcpyHostToDevice, st)) &&
      !(e = md > 0 ? launch_asph_cols(static_cast<const float*>(src->a), src->lda, m, n, md, dJ, dsg, l, Y, ctx->sms,
                                      st)
          : tma   ? launch_gather_cols_tma(cmap, dJ, l, m, Y, js, 0, ctx->sms, st)
                  : launch_gather_cols(sd, dJ, l, Y, js, 0, ctx->sms, st)) &&
      !(e = launch_ts_gram_f32(Y, m, l, l, 1, p1, nch, js, st)) &&
      !(e = launch_pchol(p1, nch, l, r, p->rank_tol, Gm, dpiv, js, st)) &&
      !(e = launch_lev_project(Y, m, l, l, 1, Gm, r, Q1, nullptr, 0, js, st)) &&
      // CholeskyQR2: the orthonormal factor U = Q1 R2^{-1}
      !(e = launch_ts_gram_f64(Q1, m, r, p2, nch2, js, st)) && !(e = launch_lev_chol(p2, nch2, r, Linv, js, st)) &&
      !(e = launch_rf_finish(Q1, m, r, Linv, out->U, js, ctx->sms, st)) &&
      !(e = cudaMemcpyAsync(&hjs, js, sizeof(JobStatus), cudaMemcpyDeviceToHost, st)) &&
      !(e = cudaMemcpyAsync(hpiv.data(), dpiv, sizeof(int) * l, cudaMemcpyDeviceToHost, st)))
    e = cudaStreamSynchronize(st);
  if (e) {
    cudaFreeAsync(b, st);
    return cuda_fail(ctx, e, "range finder");
  }
  std::memcpy(out->piv, hpiv.data(), sizeof(int) * l);
  *out->nrank = hjs.k_eff;
  if (hjs.status != LRA_OK) {
    cudaFreeAsync(b, st);
    return fail(ctx, (lra_status)hjs.status,
                hjs.status == LRA_ESINGULAR ? "range finder: the numerical rank of M H is below r (FAILURE)"
                                            : "range finder: device status");
  }
  // V = U^T M: row-major V (r x n) is column-major n x r = M^c (n x m) (U^c)^T
  cublasSetStream(ctx->blas, st);
  const float one = 1.0f, zero = 0.0f;
  int mode = 1;
  cublasStatus_t bs = cublasGemmEx(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_T, (int)n, r, (int)m, &one, src->a, CUDA_R_32F,
                                   (int)src->lda, out->U, CUDA_R_32F, r, &zero, out->V, CUDA_R_32F, (int)n,
                                   CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT);
  if (bs != CUBLAS_STATUS_SUCCESS) {
    mode = 0;
    bs = cublasGemmEx(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_T, (int)n, r, (int)m, &one, src->a, CUDA_R_32F,
                      (int)src->lda, out->U, CUDA_R_32F, r, &zero, out->V, CUDA_R_32F, (int)n, CUBLAS_COMPUTE_32F,
                      CUBLAS_GEMM_DEFAULT);
  }
  if (bs != CUBLAS_STATUS_SUCCESS) {
    cudaFreeAsync(b, st);
    return fail(ctx, LRA_ECUDA, "range finder: cublasGemmEx failed");
  }
  if (out->gemm_mode) *out->gemm_mode = mode;
  // Appendix F estimate of U V: the CUR form with C = U, nucleus I_r, R = V
  if (q > 0 &&
      !(e = launch_sampled_residual(sd, dsr, q, dsc, sN, r, out->U, Ir, out->V, cuq, rpart, nres, js, st)) &&
      !(e = cudaMemcpyAsync(&hjs, js, sizeof(JobStatus), cudaMemcpyDeviceToHost, st)))
    e = cudaStreamSynchronize(st);
  else if (q == 0)
    e = cudaStreamSynchronize(st);
  cudaFreeAsync(b, st);
  if (e) return cuda_fail(ctx, e, "range finder");
  if (out->est_rel_err) *out->est_rel_err = q > 0 ? hjs.est_rel : -1.0;
  return LRA_OK;
}

// Algorithm 3.1 with a sub-identity multiplier (see the header).
lra_status lra_dual_lsr(lra_ctx* ctx, const lra_source* W, const int32_t* rows, int32_t k,
                        const lra_lsr_params* p, const lra_lsr_out* out) {
  if (!ctx || !W || !rows || !p || !out || !out->x) return LRA_EINVAL;
  std::string why;
  if (validate_source(W, &why) != LRA_OK) return fail(ctx, LRA_EINVAL, why);
  if (W->kind != LRA_DENSE_F64 && W->kind != LRA_DENSE_F32)
    return fail(ctx, LRA_EINVAL, "dual LSR: W = (A | b) must be a stored matrix");
  const long long m = W->m;
  const int kc = (int)W->n;   // n + 1 columns
  const int passes = p->passes;
  if (kc < 2 || kc > 1024 || k < kc || k > m || passes < 1 || passes > 4)
    return fail(ctx, LRA_EINVAL, "dual LSR: need 2 <= n + 1 <= 1024, n + 1 <= k <= m, 1..4 passes");
  if (!distinct_in_range(rows, k, m)) return fail(ctx, LRA_EINVAL, "dual LSR: rows must be distinct and in range");
  const int md = p->mult_d;
  if (md < 0 || md > kMaxPreD || (m % (1LL << md)) != 0)
    return fail(ctx, LRA_EINVAL, "dual LSR: mult_d must be in 0..10 with 2^mult_d dividing m");
  if (md > 0 && p->mult_sign)
    for (int t = 0; t < k; ++t)
      if (p->mult_sign[t] != 1.0f && p->mult_sign[t] != -1.0f)
        return fail(ctx, LRA_EINVAL, "dual LSR: multiplier signs must be +1 or -1");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e) return cuda_fail(ctx, e, "cudaSetDevice");
  const int nch = ts_gram_chunks(k, kc);
  const size_t kk = (size_t)kc * kc;
  Layout lay;
  const size_t o_js = lay.take(sizeof(JobStatus)), o_rows = lay.take(sizeof(int) * k);
  const size_t o_bar = lay.take(sizeof(unsigned int) * 4);   // grid-barrier counters, one per pass (zeroed)
  const size_t o_sg = lay.take(sizeof(float) * k);           // multiplier signs
  const size_t prefix = lay.off;
  const size_t o_W = lay.take(sizeof(double) * (size_t)k * kc), o_Qa = lay.take(sizeof(double) * (size_t)k * kc);
  const size_t o_p = lay.take(sizeof(double) * (size_t)nch * kk), o_G = lay.take(sizeof(double) * kk);
  const size_t o_Gd = lay.take(sizeof(double) * kc);
  const size_t o_Rt = lay.take(sizeof(double) * kk);
  const size_t o_R = lay.take(sizeof(double) * kk * passes);
  const size_t o_v = lay.take(sizeof(double) * kc), o_x = lay.take(sizeof(double) * kc);
  const size_t o_rho = lay.take(sizeof(double));
  const size_t bytes = lay.off;
  cudaStream_t st = ctx->stream;
  unsigned char* b = nullptr;
  if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&b), bytes, ctx->pool, st)))
    return cuda_fail(ctx, e, "cudaMallocFromPoolAsync");
  auto P = [&](size_t o) { return b + o; };
  JobStatus* js = reinterpret_cast<JobStatus*>(P(o_js));
  int* drows = reinterpret_cast<int*>(P(o_rows));
  double *FW = reinterpret_cast<double*>(P(o_W)), *Qa = reinterpret_cast<double*>(P(o_Qa));
  double *part = reinterpret_cast<double*>(P(o_p)), *G = reinterpret_cast<double*>(P(o_G));
  double* Gd = reinterpret_cast<double*>(P(o_Gd));
  double* Rs = reinterpret_cast<double*>(P(o_R));
  double* Rt = reinterpret_cast<double*>(P(o_Rt));
  double *dv = reinterpret_cast<double*>(P(o_v)), *dx = reinterpret_cast<double*>(P(o_x));
  double* drho = reinterpret_cast<double*>(P(o_rho));
  unsigned int* dbar = reinterpret_cast<unsigned int*>(P(o_bar));
  std::vector<unsigned char> hs(prefix, 0);
  JobStatus init{};
  init.status = LRA_OK;
  std::memcpy(hs.data() + o_js, &init, sizeof(init));
  std::memcpy(hs.data() + o_rows, rows, sizeof(int) * k);
  for (int t = 0; t < k; ++t) {
    const float sg = (md > 0 && p->mult_sign) ? p->mult_sign[t] : 1.0f;
    std::memcpy(hs.data() + o_sg + sizeof(float) * t, &sg, sizeof(float));
  }
  const SourceDev sd = make_src(W);
  // the shift of shifted CholeskyQR: 11 (k c + c (c + 1)) u, times ||F W||_F^2 on the device
  const double shift_rel = 11.0 * ((double)k * kc + (double)kc * (kc + 1)) * 0x1p-53;
  e = cudaMemcpyAsync(b, hs.data(), prefix, cudaMemcpyHostToDevice, st);
  if (!e)
    e = md > 0 ? launch_asph_rows_f64(sd, md, drows, reinterpret_cast<const float*>(P(o_sg)), k, FW, ctx->sms, st)
               : launch_gather_rows_f64(sd, drows, k, FW, ctx->sms, st);
  double *in = FW, *outq = Qa;
  for (int s = 0; s < passes && !e; ++s) {
    double* Rsp = Rs + s * kk;
    if ((e = launch_ts_gram_f64(in, k, kc, part, nch, js, st))) break;
    // the first passes - 2 passes (at least one) shifted, the last two plain;
    // in a plain pass a pivot at most 1e-3 s_rel times its column's squared
    // norm marks a numerically rank-deficient sample (after a shifted pass
    // the pivots stay near s_rel or above)
    const bool shift_here = p->shifted && s < std::max(1, passes - 2);
    if ((e = launch_chol_coop(part, nch, kc, shift_here ? shift_rel : 0.0, shift_here ? 0.0 : 1e-3 * shift_rel, G,
                              Gd, Rsp, Rt, dbar + s, js, ctx->sms, st)))
      break;
    if (s + 1 < passes) {
      if ((e = launch_trsm_rows(in, k, kc, Rt, outq, js, ctx->sms, st))) break;
      std::swap(in, outq);   // ping-pong: the gathered rows are not needed after the first pass
    }
  }
  JobStatus hjs{};
  std::vector<double> hx(kc, 0.0);
  double hrho = 0.0;
  if (!e && !(e = launch_lsr_solve(Rs, passes, kc, dv, dx, drho, js, st)) &&
      !(e = cudaMemcpyAsync(&hjs, js, sizeof(JobStatus), cudaMemcpyDeviceToHost, st)) &&
      !(e = cudaMemcpyAsync(hx.data(), dx, sizeof(double) * kc, cudaMemcpyDeviceToHost, st)) &&
      !(e = cudaMemcpyAsync(&hrho, drho, sizeof(double), cudaMemcpyDeviceToHost, st)))
    e = cudaStreamSynchronize(st);
  cudaFreeAsync(b, st);
  if (e) return cuda_fail(ctx, e, "dual LSR");
  if (hjs.status != LRA_OK)
    return fail(ctx, (lra_status)hjs.status,
                hjs.status == LRA_ESINGULAR ? "dual LSR: a Cholesky pivot is not positive" : "dual LSR: device status");
  std::memcpy(out->x, hx.data(), sizeof(double) * (kc - 1));
  if (out->rho) *out->rho = hrho;
  return LRA_OK;
}

lra_status lra_preprocess_materialize(const lra_source* pre, float* G, int64_t ldg, void* stream) {
  std::string why;
  if (validate_source(pre, &why) != LRA_OK || pre->kind != LRA_PRE_AH || pre->pre_materialized || pre->pre_d > 5 ||
      !G || ldg < pre->n)
    return LRA_EINVAL;
  const float* M = static_cast<const float*>(pre->a);
  // G must not overlap M (it is written while M is read)
  const char *g0 = reinterpret_cast<const char*>(G), *g1 = reinterpret_cast<const char*>(G + (pre->m - 1) * ldg + pre->n);
  const char *m0 = reinterpret_cast<const char*>(M), *m1 = reinterpret_cast<const char*>(M + (pre->m - 1) * pre->lda + pre->n);
  if (g0 < m1 && m0 < g1) return LRA_EINVAL;
  const cudaError_t e = launch_pre_materialize(M, pre->lda, G, ldg, pre->m, pre->n, pre->pre_d,
                                               static_cast<cudaStream_t>(stream));
  return e ? LRA_ECUDA : LRA_OK;
}

lra_status lra_preprocessed_recover(const lra_source* pre, const float* Cbar, const float* Rbar, int32_t l, float* A,
                                    float* B, void* stream) {
  std::string why;
  if (validate_source(pre, &why) != LRA_OK || pre->kind != LRA_PRE_AH) return LRA_EINVAL;
  if (!Cbar || !Rbar || !A || !B || l < 1 || l > kMaxL) return LRA_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* inv = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&inv), sizeof(int) * (size_t)(pre->m + pre->n), st);
  if (e) return e == cudaErrorMemoryAllocation ? LRA_ENOMEM : LRA_ECUDA;
  e = launch_pre_recover(make_src(pre), Cbar, Rbar, l, A, B, inv, st);
  cudaFreeAsync(inv, st);
  return e ? LRA_ECUDA : LRA_OK;
}

lra_status lra_draw_columns(uint64_t seed, int64_t n, int32_t l, int32_t* out) {
  if (!out || n < 1 || n > (1LL << 30) || l < 1 || l > n) return LRA_EINVAL;
  draw_columns(seed, n, l, out);
  return LRA_OK;
}

lra_status lra_gather_entries(const lra_source* src, const int32_t* rows, int64_t q, const int32_t* cols,
                              int64_t s, float* out, void* stream) {
  std::string why;
  if (validate_source(src, &why) != LRA_OK) return LRA_EINVAL;
  if (!rows || !cols || !out || q < 0 || s < 0 || q > (1LL << 30) || s > (1LL << 30)) return LRA_EINVAL;
  if (q == 0 || s == 0) return LRA_OK;
  const cudaError_t e = launch_gather_entries(make_src(src), rows, q, cols, s, out,
                                              static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? LRA_OK : (e == cudaErrorMemoryAllocation ? LRA_ENOMEM : LRA_ECUDA);
}

// Tests 3 / 4 of Section 12.2: one or two ordinary jobs of the context
// with the submatrix M[K, L] gathered between them (host orchestration).
lra_status lra_cross_cynical(lra_ctx* ctx, const lra_source* src, const lra_cynical_params* p,
                             const lra_cynical_out* out) {
  if (!ctx || !src || !p || !out || !out->I || !out->J || !out->U) return LRA_EINVAL;
  std::string why;
  if (validate_source(src, &why) != LRA_OK) return fail(ctx, LRA_EINVAL, why);
  const int q = p->q, r = p->r;
  if (q < 1 || q > kMaxL || q > src->m || q > src->n || r < 1 || r > q || p->inner_sweeps < 1 ||
      p->outer_loops < 0 || p->outer_loops > 1000 || !(p->delta > 0.0) || !(p->rank_tol >= 0.0) || !p->L ||
      (p->outer_loops == 0 && !p->K))
    return fail(ctx, LRA_EINVAL, "cynical: bad sizes or index sets");
  if (!distinct_in_range(p->L, q, src->n) || (p->outer_loops == 0 && !distinct_in_range(p->K, q, src->m)))
    return fail(ctx, LRA_EINVAL, "cynical: K and L must hold q distinct indices of M");
  std::vector<int32_t> K(q), L(q);
  lra_status st;
  if (p->outer_loops > 0) {
    // the outer C-A loops with q x q generators
    lra_params op{};
    op.k = q; op.l = q; op.sweeps = p->outer_loops; op.delta = p->delta; op.rank_tol = p->rank_tol;
    op.init_J = p->L;
    lra_job job = 0;
    if ((st = lra_cross_submit(ctx, src, &op, &job)) != LRA_OK) return st;
    lra_cur_out o{};
    std::vector<double> Uq((size_t)q * q);
    o.I = K.data(); o.J = L.data(); o.U = Uq.data();
    if ((st = lra_cross_fetch_cur(ctx, job, &o)) != LRA_OK) return st;
  } else {
    std::memcpy(K.data(), p->K, sizeof(int32_t) * q);
    std::memcpy(L.data(), p->L, sizeof(int32_t) * q);
  }
  // M[K, L] on the device (the entries every kernel sees)
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e) return cuda_fail(ctx, e, "cudaSetDevice");
  cudaStream_t sst = ctx->stream;
  unsigned char* buf = nullptr;
  // q <= 96: rows at 0, columns at 512, the q x q submatrix at 1024
  const size_t o_rows = 0, o_cols = 512, o_S = 1024;
  const size_t bytes = o_S + sizeof(float) * (size_t)q * q;
  if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&buf), bytes, ctx->pool, sst)))
    return cuda_fail(ctx, e, "cudaMallocFromPoolAsync");
  int32_t* rows = reinterpret_cast<int32_t*>(buf + o_rows);
  int32_t* cols = reinterpret_cast<int32_t*>(buf + o_cols);
  float* S = reinterpret_cast<float*>(buf + o_S);
  if (!(e = cudaMemcpyAsync(rows, K.data(), sizeof(int32_t) * q, cudaMemcpyHostToDevice, sst)) &&
      !(e = cudaMemcpyAsync(cols, L.data(), sizeof(int32_t) * q, cudaMemcpyHostToDevice, sst)) &&
      !(e = launch_gather_entries(make_src(src), rows, q, cols, q, S, sst)))
    e = cudaStreamSynchronize(sst);
  st = LRA_OK;
  if (e) {
    st = cuda_fail(ctx, e, "cynical: submatrix gather");
  } else {
    // the inner C-A iterations on the q x q submatrix, r x r generators
    lra_source ss{};
    ss.kind = LRA_DENSE_F32; ss.m = q; ss.n = q; ss.a = S; ss.lda = q;
    std::vector<int32_t> J0(r), Ii(r), Ji(r);
    for (int t = 0; t < r; ++t) J0[t] = t;
    lra_params ip{};
    ip.k = r; ip.l = r; ip.sweeps = p->inner_sweeps; ip.delta = p->delta; ip.rank_tol = p->rank_tol;
    ip.init_J = J0.data();
    lra_job job = 0;
    if ((st = lra_cross_submit(ctx, &ss, &ip, &job)) == LRA_OK) {
      lra_cur_out o{};
      o.I = Ii.data(); o.J = Ji.data(); o.U = out->U;
      if ((st = lra_cross_fetch_cur(ctx, job, &o)) == LRA_OK) {
        for (int t = 0; t < r; ++t) {
          out->I[t] = K[Ii[t]];
          out->J[t] = L[Ji[t]];
        }
        if (out->K) std::memcpy(out->K, K.data(), sizeof(int32_t) * q);
        if (out->L) std::memcpy(out->L, L.data(), sizeof(int32_t) * q);
      }
    }
  }
  cudaFreeAsync(buf, sst);
  return st;
}

// Section 7.2: refinement of the C-A CUR of (I, J) by leverage-score
// sampling (k_lev.cu: scores and Exactly(l) sampling; the strips, the
// nuclei and the Appendix F estimate through the solve's own kernels).
lra_status lra_cross_refine(lra_ctx* ctx, const lra_source* src, const int32_t* I, const int32_t* J, int32_t l,
                            const lra_refine_params* p, const lra_refine_out* out) {
  if (!ctx || !src || !I || !J || !p || !out || !out->cols || !out->d || !out->rows || !out->dbar || !out->U)
    return LRA_EINVAL;
  std::string why;
  if (validate_source(src, &why) != LRA_OK) return fail(ctx, LRA_EINVAL, why);
  const long long m = src->m, n = src->n;
  const int L2 = p->l_new;
  if (l < 1 || l > kMaxL || l > m || l > n || p->r < 1 || p->r > l || L2 < 1 || L2 > kMaxL || L2 > m || L2 > n ||
      !p->u_cols || !p->u_rows || !(p->rank_tol >= 0.0) || p->resid_q < 0 || p->resid_s < 0 ||
      (p->resid_q > 0) != (p->resid_s > 0) ||
      (p->resid_q > 0 && (!p->resid_rows || !p->resid_cols || p->resid_q > m || p->resid_s > n)))
    return fail(ctx, LRA_EINVAL, "refine: bad sizes");
  if (!distinct_in_range(I, l, m) || !distinct_in_range(J, l, n))
    return fail(ctx, LRA_EINVAL, "refine: I and J must hold l distinct indices of M");
  for (int t = 0; t < L2; ++t)
    if (!(p->u_cols[t] >= 0.0 && p->u_cols[t] < 1.0) || !(p->u_rows[t] >= 0.0 && p->u_rows[t] < 1.0))
      return fail(ctx, LRA_EINVAL, "refine: uniforms must lie in [0, 1)");
  if (p->resid_q > 0 && (!distinct_in_range(p->resid_rows, p->resid_q, m) ||
                         !distinct_in_range(p->resid_cols, p->resid_s, n)))
    return fail(ctx, LRA_EINVAL, "refine: residual sample indices must be distinct and in range");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e) return cuda_fail(ctx, e, "cudaSetDevice");
  const int r = p->r, q = (int)p->resid_q, sN = (int)p->resid_s;
  const int npm = lev_partials(m), npn = lev_partials(n);
  const int nres = q > 0 ? sampled_residual_partials(q, sN) : 1;
  Layout lay;
  const size_t o_js = lay.take(sizeof(JobStatus));
  const size_t o_I = lay.take(sizeof(int) * l), o_J = lay.take(sizeof(int) * l);
  const size_t o_u = lay.take(sizeof(double) * 2 * L2);
  const size_t o_sr = lay.take(sizeof(int) * std::max(q, 1)), o_sc = lay.take(sizeof(int) * std::max(sN, 1));
  const size_t prefix = lay.off;
  const size_t o_C = lay.take(sizeof(float) * (size_t)m * l), o_R = lay.take(sizeof(float) * (size_t)n * l);
  const size_t o_U = lay.take(sizeof(double) * l * l), o_sg = lay.take(sizeof(double) * l);
  const size_t o_P = lay.take(sizeof(double) * l * l), o_V = lay.take(sizeof(double) * l * l);
  const size_t o_G1 = lay.take(sizeof(double) * l * r), o_G2 = lay.take(sizeof(double) * l * r);
  const size_t o_Yc = lay.take(sizeof(double) * (size_t)m * r), o_Yr = lay.take(sizeof(double) * (size_t)n * r);
  const size_t o_pm = lay.take(sizeof(double) * (size_t)npm * r * r);
  const size_t o_pn = lay.take(sizeof(double) * (size_t)npn * r * r);
  const size_t o_Lc = lay.take(sizeof(double) * r * r), o_Lr = lay.take(sizeof(double) * r * r);
  const size_t o_wm = lay.take(sizeof(double) * m), o_wn = lay.take(sizeof(double) * n);
  const size_t o_sm = lay.take(sizeof(double) * m), o_sn = lay.take(sizeof(double) * n);
  const size_t o_ic = lay.take(sizeof(int) * L2), o_ir = lay.take(sizeof(int) * L2);
  const size_t o_d = lay.take(sizeof(double) * L2), o_db = lay.take(sizeof(double) * L2);
  const size_t o_C2 = lay.take(sizeof(float) * (size_t)m * L2), o_R2 = lay.take(sizeof(float) * (size_t)n * L2);
  const size_t o_U2 = lay.take(sizeof(double) * L2 * L2), o_sg2 = lay.take(sizeof(double) * L2);
  const size_t o_cuq = lay.take(sizeof(float) * std::max<size_t>(2 * (size_t)q * L2, 1));
  const size_t o_pr = lay.take(sizeof(double) * 3 * nres);
  const size_t bytes = lay.off;
  cudaStream_t st = ctx->stream;
  unsigned char* b = nullptr;
  if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&b), bytes, ctx->pool, st)))
    return cuda_fail(ctx, e, "cudaMallocFromPoolAsync");
  auto P = [&](size_t o) { return b + o; };
  JobStatus* js = reinterpret_cast<JobStatus*>(P(o_js));
  int *dI = reinterpret_cast<int*>(P(o_I)), *dJ = reinterpret_cast<int*>(P(o_J));
  double* du = reinterpret_cast<double*>(P(o_u));
  int *dsr = reinterpret_cast<int*>(P(o_sr)), *dsc = reinterpret_cast<int*>(P(o_sc));
  float *C = reinterpret_cast<float*>(P(o_C)), *R = reinterpret_cast<float*>(P(o_R));
  double *U = reinterpret_cast<double*>(P(o_U)), *sg = reinterpret_cast<double*>(P(o_sg));
  double *Pk = reinterpret_cast<double*>(P(o_P)), *Vk = reinterpret_cast<double*>(P(o_V));
  double *G1 = reinterpret_cast<double*>(P(o_G1)), *G2 = reinterpret_cast<double*>(P(o_G2));
  double *Yc = reinterpret_cast<double*>(P(o_Yc)), *Yr = reinterpret_cast<double*>(P(o_Yr));
  double *pm = reinterpret_cast<double*>(P(o_pm)), *pn = reinterpret_cast<double*>(P(o_pn));
  double *Lc = reinterpret_cast<double*>(P(o_Lc)), *Lr = reinterpret_cast<double*>(P(o_Lr));
  double *wm = reinterpret_cast<double*>(P(o_wm)), *wn = reinterpret_cast<double*>(P(o_wn));
  double *scm = reinterpret_cast<double*>(P(o_sm)), *scn = reinterpret_cast<double*>(P(o_sn));
  int *ic = reinterpret_cast<int*>(P(o_ic)), *ir = reinterpret_cast<int*>(P(o_ir));
  double *dd_ = reinterpret_cast<double*>(P(o_d)), *db = reinterpret_cast<double*>(P(o_db));
  float *C2 = reinterpret_cast<float*>(P(o_C2)), *R2 = reinterpret_cast<float*>(P(o_R2));
  double *U2 = reinterpret_cast<double*>(P(o_U2)), *sg2 = reinterpret_cast<double*>(P(o_sg2));
  float* cuq = reinterpret_cast<float*>(P(o_cuq));
  double* rpart = reinterpret_cast<double*>(P(o_pr));
  // the inputs, staged in host memory and sent in one copy
  std::vector<unsigned char> hs(prefix, 0);
  JobStatus init{};
  init.status = LRA_OK;
  std::memcpy(hs.data() + o_js, &init, sizeof(init));
  std::memcpy(hs.data() + o_I, I, sizeof(int) * l);
  std::memcpy(hs.data() + o_J, J, sizeof(int) * l);
  std::memcpy(hs.data() + o_u, p->u_cols, sizeof(double) * L2);
  std::memcpy(hs.data() + o_u + sizeof(double) * L2, p->u_rows, sizeof(double) * L2);
  if (q > 0) {
    std::memcpy(hs.data() + o_sr, p->resid_rows, sizeof(int) * q);
    std::memcpy(hs.data() + o_sc, p->resid_cols, sizeof(int) * sN);
  }
  const SourceDev sd = make_src(src);
  TmaMap cmap{};
  const bool tma = src->kind == LRA_DENSE_F32 &&
                   make_cols_map(&cmap, static_cast<const float*>(src->a), m, n, src->lda);
  auto gather_c = [&](const int* Jd, int ll, float* out_C) {
    return tma ? launch_gather_cols_tma(cmap, Jd, ll, m, out_C, js, 0, ctx->sms, st)
               : launch_gather_cols(sd, Jd, ll, out_C, js, 0, ctx->sms, st);
  };
  NucExtra vec;
  vec.Pk = Pk;
  vec.Vk = Vk;
  NucExtra scl;
  scl.rs = db;
  scl.cs = dd_;
  JobStatus hjs{};
  // phase 1: C = M[:, J], R = M[I, :], U = (X_r)^+ with the kept singular
  // vectors; the rank actually kept decides the dimension of the scores
  if (!(e = cudaMemcpyAsync(b, hs.data(), prefix, cudaMemcpyHostToDevice, st)) &&
      !(e = gather_c(dJ, l, C)) && !(e = launch_gather_rows(sd, dI, l, R, js, ctx->sms, st)) &&
      !(e = launch_nucleus(C, dI, l, r, p->rank_tol, U, sg, js, st, vec)) &&
      !(e = cudaMemcpyAsync(&hjs, js, sizeof(JobStatus), cudaMemcpyDeviceToHost, st)))
    e = cudaStreamSynchronize(st);
  const int rr = std::min(r, hjs.k_eff);
  if (!e && (hjs.status != LRA_OK || rr < 1)) {
    cudaFreeAsync(b, st);
    if (hjs.status != LRA_OK) return fail(ctx, (lra_status)hjs.status, "refine: device status");
    return fail(ctx, LRA_ESINGULAR, "refine: the C-A cross has rank 0");
  }
  // phase 2: H = C (U P_rr) and Z^T = R^T (U^T V_rr), their Gram matrices
  // and scores, the sampling, the refined strips and nucleus
  if (!e &&
      !(e = launch_lev_factors(U, Pk, Vk, l, rr, G1, G2, js, st)) &&
      !(e = launch_lev_project(C, m, l, l, 1, G1, rr, Yc, pm, npm, js, st)) &&
      !(e = launch_lev_project(R, n, l, 1, n, G2, rr, Yr, pn, npn, js, st)) &&
      !(e = launch_lev_chol(pm, npm, rr, Lc, js, st)) && !(e = launch_lev_chol(pn, npn, rr, Lr, js, st)) &&
      // Exactly(l_new) columns from the right scores, rows from the left ones
      !(e = launch_lev_scores_sample(Yr, n, rr, Lr, wn, du, L2, ic, dd_, scn, js, st)) &&
      !(e = launch_lev_scores_sample(Yc, m, rr, Lc, wm, du + L2, L2, ir, db, scm, js, st)) &&
      // C' = M[:, cols], R' = M[rows, :], U' = D (Dbar C'[rows, :] D)_rr^+ Dbar
      !(e = gather_c(ic, L2, C2)) && !(e = launch_gather_rows(sd, ir, L2, R2, js, ctx->sms, st)) &&
      !(e = launch_nucleus(C2, ir, L2, rr, p->rank_tol, U2, sg2, js, st, scl)) &&
      !(e = q > 0 ? launch_sampled_residual(sd, dsr, q, dsc, sN, L2, C2, U2, R2, cuq, rpart, nres, js, st)
                  : cudaSuccess) &&
      !(e = cudaMemcpyAsync(&hjs, js, sizeof(JobStatus), cudaMemcpyDeviceToHost, st)) &&
      !(e = cudaMemcpyAsync(out->cols, ic, sizeof(int) * L2, cudaMemcpyDeviceToHost, st)) &&
      !(e = cudaMemcpyAsync(out->d, dd_, sizeof(double) * L2, cudaMemcpyDeviceToHost, st)) &&
      !(e = cudaMemcpyAsync(out->rows, ir, sizeof(int) * L2, cudaMemcpyDeviceToHost, st)) &&
      !(e = cudaMemcpyAsync(out->dbar, db, sizeof(double) * L2, cudaMemcpyDeviceToHost, st)) &&
      !(e = cudaMemcpyAsync(out->U, U2, sizeof(double) * L2 * L2, cudaMemcpyDeviceToHost, st)) &&
      !(e = out->p_cols ? cudaMemcpyAsync(out->p_cols, scn, sizeof(double) * n, cudaMemcpyDeviceToHost, st)
                        : cudaSuccess) &&
      !(e = out->p_rows ? cudaMemcpyAsync(out->p_rows, scm, sizeof(double) * m, cudaMemcpyDeviceToHost, st)
                        : cudaSuccess))
    e = cudaStreamSynchronize(st);
  cudaFreeAsync(b, st);
  if (e) return cuda_fail(ctx, e, "refine");
  if (hjs.status != LRA_OK) return fail(ctx, (lra_status)hjs.status, "refine: device status");
  if (hjs.k_eff < 1) return fail(ctx, LRA_ESINGULAR, "refine: the sampled generator has rank 0");
  if (out->est_rel_err) *out->est_rel_err = q > 0 ? hjs.est_rel : -1.0;
  if (out->k_eff) *out->k_eff = rr;
  return LRA_OK;
}

static lra_status validate_batch(const lra_source* src, const lra_block* blocks, int32_t nb,
                                 const lra_batch_params* p, std::string* why) {
  if (!src || !blocks || !p) { *why = "null argument"; return LRA_EINVAL; }
  if (src->kind < LRA_DENSE_F32 || src->kind > LRA_GEN_INVDIST) { *why = "unknown source kind"; return LRA_EINVAL; }
  if (src->kind <= LRA_DENSE_F64 ? (!src->a || src->lda < src->n) : (!src->x || !src->y)) {
    *why = "source pointers"; return LRA_EINVAL;
  }
  if (src->kind == LRA_GEN_GAUSS || src->kind == LRA_GEN_INVDIST) {
    if (src->dim < 1 || src->dim > 3) { *why = "dim must be 1..3"; return LRA_EINVAL; }
  }
  if (nb < 1) { *why = "n_blocks must be >= 1"; return LRA_EINVAL; }
  if (p->l_max < 1 || p->l_max > kMaxL) { *why = "l_max must be in 1..96"; return LRA_EINVAL; }
  if (p->l_init < 1 || p->l_init > p->l_max) { *why = "l_init must be in 1..l_max"; return LRA_EINVAL; }
  if (p->k_max < 1 || p->k_max > p->l_max) { *why = "k_max must be in 1..l_max"; return LRA_EINVAL; }
  if (p->sweeps < 1 || p->sweeps > 100) { *why = "sweeps must be in 1..100"; return LRA_EINVAL; }
  if (p->sample < 0 || p->sample > 64) { *why = "sample must be in 0..64"; return LRA_EINVAL; }
  if (!(p->delta > 0.0) || !(p->tol >= 0.0)) { *why = "delta > 0 and tol >= 0 required"; return LRA_EINVAL; }
  if (p->trace_cap < 0 || p->trace_cap > (1 << 20)) { *why = "trace_cap must be in 0..2^20"; return LRA_EINVAL; }
  if (p->cluster_mask < 0 || p->cluster_mask > 15) { *why = "cluster_mask must be in 0..15"; return LRA_EINVAL; }
  if (p->cutover_side < 0) { *why = "cutover_side must be >= 0"; return LRA_EINVAL; }
  if (p->order != 0 && p->order != 1) { *why = "order must be 0 or 1"; return LRA_EINVAL; }
  if (!p->cand_J || (p->sample > 0 && (!p->sample_rows || !p->sample_cols))) {
    *why = "candidate / sample arrays required"; return LRA_EINVAL;
  }
  for (int32_t b = 0; b < nb; ++b) {
    const lra_block& k = blocks[b];
    if (k.m < 1 || k.n < 1 || k.m > kMaxBatchSide || k.n > kMaxBatchSide || k.row0 < 0 || k.col0 < 0 ||
        k.row0 + k.m > src->m || k.col0 + k.n > src->n) {
      *why = "block " + std::to_string(b) + " out of range (sides 1..2048 inside the source)";
      return LRA_EINVAL;
    }
    const long long lc = std::min<long long>(p->l_max, k.n);
    if (!distinct_in_range(p->cand_J + (size_t)b * p->l_max, lc, k.n)) {
      *why = "cand_J of block " + std::to_string(b) + " must hold distinct local columns";
      return LRA_EINVAL;
    }
    if (p->sample > 0 && (p->sample > k.m || p->sample > k.n ||
                          !distinct_in_range(p->sample_rows + (size_t)b * p->sample, p->sample, k.m) ||
                          !distinct_in_range(p->sample_cols + (size_t)b * p->sample, p->sample, k.n))) {
      *why = "sample indices of block " + std::to_string(b);
      return LRA_EINVAL;
    }
  }
  return LRA_OK;
}

lra_status lra_cross_submit_batch(lra_ctx* ctx, const lra_source* src, const lra_block* blocks,
                                  int32_t nb, const lra_batch_params* p, lra_job* out) {
  if (!ctx || !out) return LRA_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  std::string why;
  lra_status st = validate_batch(src, blocks, nb, p, &why);
  if (st != LRA_OK) return fail(ctx, st, why);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e) return cuda_fail(ctx, e, "cudaSetDevice");
  Job* j = new Job();
  j->batch = true;
  j->n_blocks = nb;
  j->b_lmax = p->l_max;
  j->b_q = p->sample;
  j->src = make_src(src);
  j->m = src->m;
  j->n = src->n;
  const size_t L = (size_t)p->l_max, q = (size_t)p->sample, NB = (size_t)nb;
  Layout lay;
  const size_t o_js = lay.take(sizeof(JobStatus));
  const size_t o_queue = lay.take(4 * sizeof(int));  // one work counter per pass
  const size_t o_blocks = lay.take(sizeof(long long) * 4 * NB);
  const size_t o_jc = lay.take(sizeof(int) * NB * L);
  const size_t o_sr = lay.take(sizeof(int) * NB * std::max<size_t>(q, 1));
  const size_t o_sc = lay.take(sizeof(int) * NB * std::max<size_t>(q, 1));
  const size_t o_st = lay.take(sizeof(int) * NB);
  const size_t o_l = lay.take(sizeof(int) * NB);
  const size_t o_ke = lay.take(sizeof(int) * NB);
  const size_t o_sw = lay.take(sizeof(int) * NB);
  const size_t o_I = lay.take(sizeof(int) * NB * L);
  const size_t o_J = lay.take(sizeof(int) * NB * L);
  const size_t o_U = lay.take(sizeof(double) * NB * L * L);
  const size_t o_sg = lay.take(sizeof(float) * NB * L);
  const size_t o_er = lay.take(sizeof(double) * NB);
  const size_t TC = (size_t)std::max(p->trace_cap, 0);
  const size_t o_tl = lay.take(sizeof(int) * NB);
  const size_t o_tr = lay.take(sizeof(int) * 4 * NB * std::max<size_t>(TC, 1));
  const size_t o_tv = lay.take(sizeof(double) * NB * std::max<size_t>(TC, 1));
  const size_t o_ord = lay.take(sizeof(int) * NB);
  j->bytes = lay.off;
  j->b_tcap = (int)TC;
  if ((int)ctx->jobs.size() >= ctx->max_slots || ctx->free_slots.empty() ||
      (ctx->budget && ctx->used_bytes + j->bytes > ctx->budget)) {
    delete j;
    return fail(ctx, LRA_EBUSY, "no free slot or memory budget exhausted");
  }
  assign_stream(ctx, j);
  if ((e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&j->dmem), j->bytes, ctx->pool, j->stream))) {
    ctx->stream_load[j->stream_idx]--;
    delete j;
    return cuda_fail(ctx, e, "cudaMallocFromPoolAsync");
  }
  unsigned char* base = j->dmem;
  j->js = reinterpret_cast<JobStatus*>(base + o_js);
  j->b_queue = reinterpret_cast<int*>(base + o_queue);
  j->b_blocks = reinterpret_cast<long long*>(base + o_blocks);
  j->b_jcand = reinterpret_cast<int*>(base + o_jc);
  j->b_srow = reinterpret_cast<int*>(base + o_sr);
  j->b_scol = reinterpret_cast<int*>(base + o_sc);
  j->b_status = reinterpret_cast<int*>(base + o_st);
  j->b_l = reinterpret_cast<int*>(base + o_l);
  j->b_keff = reinterpret_cast<int*>(base + o_ke);
  j->b_swaps = reinterpret_cast<int*>(base + o_sw);
  j->b_I = reinterpret_cast<int*>(base + o_I);
  j->b_J = reinterpret_cast<int*>(base + o_J);
  j->b_U = reinterpret_cast<double*>(base + o_U);
  j->b_sigma = reinterpret_cast<float*>(base + o_sg);
  j->b_err = reinterpret_cast<double*>(base + o_er);
  j->b_tlen = reinterpret_cast<int*>(base + o_tl);
  j->b_trace = reinterpret_cast<int*>(base + o_tr);
  j->b_tval = reinterpret_cast<double*>(base + o_tv);
  j->slot = ctx->free_slots.back();
  ctx->free_slots.pop_back();
  ctx->used_bytes += j->bytes;
  cudaStream_t s = j->stream;
  JobStatus init{};
  init.status = LRA_OK;
  init.converged = 1;
  BatchArgs a{};
  a.src = j->src;
  a.blocks = j->b_blocks;
  a.n_blocks = nb;
  a.jcand = j->b_jcand;
  a.srow = j->b_srow;
  a.scol = j->b_scol;
  a.q = p->sample;
  a.l_init = p->l_init;
  a.l_max = p->l_max;
  a.k_max = p->k_max;
  a.sweeps = p->sweeps;
  a.max_swaps = p->max_swaps > 0 ? p->max_swaps : 64 * p->l_max;
  a.tol = p->tol;
  a.delta = p->delta;
  a.trace_cap = (int)TC;
  a.cutover = p->cutover_side;
  // queue order: as given, or the largest blocks (m + n) first, so that the
  // long solves start early and the launch ends on short ones
  std::vector<int> ord;
  if (p->order == 1) {
    ord.resize(NB);
    for (int32_t b = 0; b < nb; ++b) ord[b] = b;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      return blocks[x].m + blocks[x].n > blocks[y].m + blocks[y].n;
    });
  }
  a.order = p->order == 1 ? reinterpret_cast<const int*>(base + o_ord) : nullptr;
  a.trace = j->b_trace;
  a.trace_v = j->b_tval;
  a.trace_len = j->b_tlen;
  a.queue = j->b_queue;
  a.out_status = j->b_status;
  a.out_l = j->b_l;
  a.out_keff = j->b_keff;
  a.out_swaps = j->b_swaps;
  a.out_I = j->b_I;
  a.out_J = j->b_J;
  a.out_U = j->b_U;
  a.out_sigma = j->b_sigma;
  a.out_err = j->b_err;
  a.js = j->js;
  static_assert(sizeof(lra_block) == 4 * sizeof(long long), "lra_block layout");
  if ((e = cudaEventCreate(&j->ev_start)) || (e = cudaEventCreate(&j->ev_end)) ||
      (e = cudaMemcpyAsync(j->js, &init, sizeof(init), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemsetAsync(j->b_queue, 0, 4 * sizeof(int), s)) ||
      (p->order == 1 && (e = cudaMemcpyAsync(base + o_ord, ord.data(), sizeof(int) * NB, cudaMemcpyHostToDevice, s))) ||
      (e = cudaMemsetAsync(j->b_tlen, 0, sizeof(int) * NB, s)) ||
      (e = cudaMemsetAsync(j->b_err, 0, sizeof(double) * NB, s)) ||
      (e = cudaMemsetAsync(j->b_keff, 0, sizeof(int) * NB, s)) ||
      (e = cudaMemcpyAsync(j->b_blocks, blocks, sizeof(lra_block) * NB, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(j->b_jcand, p->cand_J, sizeof(int) * NB * L, cudaMemcpyHostToDevice, s)) ||
      (q > 0 && ((e = cudaMemcpyAsync(j->b_srow, p->sample_rows, sizeof(int) * NB * q, cudaMemcpyHostToDevice, s)) ||
                 (e = cudaMemcpyAsync(j->b_scol, p->sample_cols, sizeof(int) * NB * q, cudaMemcpyHostToDevice, s)))) ||
      (e = cudaEventRecord(j->ev_start, s)) || (e = launch_batch(a, p->cluster_mask ? p->cluster_mask : kDefaultClusterMask, ctx->sms, s)) ||
      (e = cudaMemcpyAsync(ctx->pinned + j->slot, j->js, sizeof(JobStatus), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaEventRecord(j->ev_end, s))) {
    cudaStreamSynchronize(s);
    release_job(ctx, j);
    return cuda_fail(ctx, e, "batch enqueue");
  }
  j->launches = 1;
  j->id = ctx->next_id++;
  ctx->jobs[j->id] = j;
  *out = j->id;
  return LRA_OK;
}

lra_status lra_cross_fetch_batch(lra_ctx* ctx, lra_job id, const lra_batch_out* out) {
  if (!ctx || !out) return LRA_EINVAL;
  Job* j = nullptr;
  cudaStream_t cs = nullptr;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    j = find_job(ctx, id);
    if (!j) return fail(ctx, LRA_ENOTFOUND, "unknown job");
    if (!j->batch) return fail(ctx, LRA_EINVAL, "not a batch job: use lra_cross_fetch_cur");
    ctx->jobs.erase(id);
    cs = take_copy_stream(ctx);
  }
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaEventSynchronize(j->ev_end);
  lra_status result = e ? LRA_ECUDA : (lra_status)ctx->pinned[j->slot].status;
  if (!e) {
    const size_t NB = (size_t)j->n_blocks, L = (size_t)j->b_lmax;
    struct Piece { void* dst; const void* src; size_t bytes; };
    Piece pieces[] = {
        {out->status, j->b_status, sizeof(int) * NB}, {out->l, j->b_l, sizeof(int) * NB},
        {out->k_eff, j->b_keff, sizeof(int) * NB},    {out->swaps, j->b_swaps, sizeof(int) * NB},
        {out->I, j->b_I, sizeof(int) * NB * L},       {out->J, j->b_J, sizeof(int) * NB * L},
        {out->U, j->b_U, sizeof(double) * NB * L * L}, {out->sigma, j->b_sigma, sizeof(float) * NB * L},
        {out->est_err, j->b_err, sizeof(double) * NB},
        {out->trace_len, j->b_tlen, j->b_tcap ? sizeof(int) * NB : 0},
        {out->trace, j->b_trace, sizeof(int) * 4 * NB * (size_t)j->b_tcap},
        {out->trace_val, j->b_tval, sizeof(double) * NB * (size_t)j->b_tcap},
    };
    for (const Piece& pc : pieces) {
      if (e) break;
      if (!pc.dst || pc.bytes == 0) continue;
      e = cudaMemcpyAsync(pc.dst, pc.src, pc.bytes, cudaMemcpyDefault, cs);
    }
    if (!e) e = cudaStreamSynchronize(cs);
    if (e) result = LRA_ECUDA;
  }
  std::lock_guard<std::mutex> lock(ctx->mu);
  give_copy_stream(ctx, cs);
  release_job(ctx, j);
  if (e) return cuda_fail(ctx, e, "fetch");
  return result;
}

}  // extern "C"
