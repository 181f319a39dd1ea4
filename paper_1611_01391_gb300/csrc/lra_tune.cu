// Launch-shape tuner of the batched form: which cluster sizes the passes
// use, which blocks skip the one-CTA pass, and in which order the work queue
// hands out the blocks.  None of these changes a block's result (the
// decisions and the arithmetic per entry do not depend on the split), only
// the time; the tuner checks that on every candidate it runs.  The chosen
// shape is kept per GPU and workload bucket in a small JSON file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/lra_cross.h"
#include "lra_internal.cuh"
#include "lra_kernels.h"

namespace {

struct Shape {
  int mask, cutover, order;
};

long long pow2_at_least(long long v) {
  long long p = 1;
  while (p < v) p <<= 1;
  return p;
}

// <gpu name>|kind=<k>|lmax=<l>|kmax=<k>|blocks=<2^a>|median=<2^b>|max=<2^c>,
// with 2^a, 2^b, 2^c the powers of two at or above the block count, the
// median and the largest of the blocks' larger sides.
std::string bucket_key(const char* gpu, const lra_source* src, const lra_block* blocks, int nb,
                       const lra_batch_params* p) {
  std::vector<long long> side(nb);
  for (int b = 0; b < nb; ++b) side[b] = std::max(blocks[b].m, blocks[b].n);
  std::sort(side.begin(), side.end());
  std::string name;
  for (const char* c = gpu; *c; ++c) name += (*c == '"' || *c == '\\' || *c == '|') ? '_' : *c;
  std::ostringstream k;
  k << name << "|kind=" << src->kind << "|lmax=" << p->l_max << "|kmax=" << p->k_max
    << "|blocks=" << pow2_at_least(nb) << "|median=" << pow2_at_least(side[nb / 2])
    << "|max=" << pow2_at_least(side.back());
  return k.str();
}

// The cache: a JSON object with one entry per line,
//   "<key>": {"cluster_mask": M, "cutover_side": C, "order": O, "ms_default": D, "ms_tuned": T}
std::vector<std::string> cache_entries(const char* path) {
  std::vector<std::string> out;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line))
    if (line.find("\": {\"cluster_mask\":") != std::string::npos) out.push_back(line);
  return out;
}

bool cache_find(const char* path, const std::string& key, Shape* s) {
  const std::string head = "\"" + key + "\": {";
  for (const std::string& line : cache_entries(path)) {
    const size_t at = line.find(head);
    if (at == std::string::npos) continue;
    Shape t{};
    if (std::sscanf(line.c_str() + at + head.size(), "\"cluster_mask\": %d, \"cutover_side\": %d, \"order\": %d",
                    &t.mask, &t.cutover, &t.order) == 3) {
      *s = t;
      return true;
    }
  }
  return false;
}

bool cache_store(const char* path, const std::string& key, const Shape& s, double ms_def, double ms_best) {
  const std::string head = "\"" + key + "\": {";
  std::vector<std::string> keep;
  for (const std::string& line : cache_entries(path)) {
    if (line.find(head) != std::string::npos) continue;
    std::string t = line;
    while (!t.empty() && (t.back() == ',' || t.back() == ' ')) t.pop_back();
    keep.push_back(t);
  }
  char buf[256];
  std::snprintf(buf, sizeof(buf),
                "\"cluster_mask\": %d, \"cutover_side\": %d, \"order\": %d, \"ms_default\": %.4f, \"ms_tuned\": %.4f}",
                s.mask, s.cutover, s.order, ms_def, ms_best);
  keep.push_back("    " + head + buf);
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp);
    if (!f) return false;
    f << "{\n  \"lra_batch_tuning\": 1,\n  \"entries\": {\n";
    for (size_t i = 0; i < keep.size(); ++i) f << keep[i] << (i + 1 < keep.size() ? ",\n" : "\n");
    f << "  }\n}\n";
    if (!f) return false;
  }
  return std::rename(tmp.c_str(), path) == 0;
}

// The per-block outputs that decide equality between shapes.
struct Outputs {
  std::vector<int32_t> status, l, keff, I, J;
  std::vector<double> err;
};

lra_status run_shape(lra_ctx* ctx, const lra_source* src, const lra_block* blocks, int nb,
                     const lra_batch_params* p0, const Shape& sh, double* ms, Outputs* out) {
  lra_batch_params p = *p0;
  p.cluster_mask = sh.mask;
  p.cutover_side = sh.cutover;
  p.order = sh.order;
  p.trace_cap = 0;
  lra_job job = 0;
  lra_status st = lra_cross_submit_batch(ctx, src, blocks, nb, &p, &job);
  if (st != LRA_OK) return st;
  lra_info info{};
  st = lra_cross_wait(ctx, job, &info);
  if (st != LRA_OK) {
    lra_cross_cancel(ctx, job);
    return st;
  }
  *ms = info.gpu_ms;
  const size_t L = (size_t)p.l_max;
  out->status.assign(nb, 0);
  out->l.assign(nb, 0);
  out->keff.assign(nb, 0);
  out->I.assign(nb * L, 0);
  out->J.assign(nb * L, 0);
  out->err.assign(nb, 0.0);
  lra_batch_out o{};
  o.on_device = 0;
  o.status = out->status.data();
  o.l = out->l.data();
  o.k_eff = out->keff.data();
  o.I = out->I.data();
  o.J = out->J.data();
  o.est_err = out->err.data();
  return lra_cross_fetch_batch(ctx, job, &o);
}

bool same(const Outputs& a, const Outputs& b) {
  return a.status == b.status && a.l == b.l && a.keff == b.keff && a.I == b.I && a.J == b.J &&
         std::memcmp(a.err.data(), b.err.data(), sizeof(double) * a.err.size()) == 0;
}

}  // namespace

extern "C" {

lra_status lra_batch_tuning_lookup(const char* cache_path, const char* gpu_name, const lra_source* src,
                                   const lra_block* blocks, int32_t n_blocks, const lra_batch_params* params,
                                   lra_batch_params* tuned) {
  if (!cache_path || !gpu_name || !src || !blocks || n_blocks < 1 || !params || !tuned) return LRA_EINVAL;
  Shape s{};
  if (!cache_find(cache_path, bucket_key(gpu_name, src, blocks, n_blocks, params), &s)) return LRA_ENOTFOUND;
  *tuned = *params;
  tuned->cluster_mask = s.mask;
  tuned->cutover_side = s.cutover;
  tuned->order = s.order;
  return LRA_OK;
}

lra_status lra_cross_tune_batch(lra_ctx* ctx, const lra_source* src, const lra_block* blocks, int32_t n_blocks,
                                const lra_batch_params* params, const char* cache_path, lra_batch_params* tuned,
                                double* ms_default, double* ms_tuned) {
  if (!ctx || !src || !blocks || n_blocks < 1 || !params || !tuned) return LRA_EINVAL;
  if (ms_default) *ms_default = -1.0;
  if (ms_tuned) *ms_tuned = -1.0;
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, lra::ctx_device(ctx)) != cudaSuccess) return LRA_ECUDA;
  const std::string key = bucket_key(prop.name, src, blocks, n_blocks, params);
  Shape best{};
  if (cache_path && cache_find(cache_path, key, &best)) {
    *tuned = *params;
    tuned->cluster_mask = best.mask;
    tuned->cutover_side = best.cutover;
    tuned->order = best.order;
    return LRA_OK;
  }
  const Shape def{lra::kDefaultClusterMask, 0, 0};
  std::vector<Shape> cand;
  for (int mask : {def.mask, 1 | 2 | 8, 1 | 2 | 4 | 8, 1 | 8, 2 | 4 | 8})
    for (int cut : {0, 1024, 512})
      for (int ord : {0, 1}) cand.push_back(Shape{mask, cut, ord});
  Outputs ref, out;
  double t = 0.0, t_def = 0.0;
  // the default shape: a warm-up run, then the reference outputs and time
  lra_status st = run_shape(ctx, src, blocks, n_blocks, params, def, &t, &ref);
  if (st != LRA_OK) return st;
  double best_t = 1e300;
  for (const Shape& sh : cand) {
    double tmin = 1e300;
    for (int rep = 0; rep < 2; ++rep) {
      st = run_shape(ctx, src, blocks, n_blocks, params, sh, &t, &out);
      if (st != LRA_OK) return st;
      if (!same(ref, out)) {   // a shape changed a block's result: a bug, not a tuning outcome
        lra::set_ctx_error(ctx, "batch tuner: a launch shape changed per-block results");
        return LRA_ECUDA;
      }
      tmin = std::min(tmin, t);
    }
    if (sh.mask == def.mask && sh.cutover == def.cutover && sh.order == def.order) t_def = tmin;
    if (tmin < best_t) {
      best_t = tmin;
      best = sh;
    }
  }
  if (best_t >= 0.98 * t_def) {   // not a clear gain: keep the default shape
    best = def;
    best_t = t_def;
  }
  if (cache_path) cache_store(cache_path, key, best, t_def, best_t);
  *tuned = *params;
  tuned->cluster_mask = best.mask;
  tuned->cutover_side = best.cutover;
  tuned->order = best.order;
  if (ms_default) *ms_default = t_def;
  if (ms_tuned) *ms_tuned = best_t;
  return LRA_OK;
}

}  // extern "C"
