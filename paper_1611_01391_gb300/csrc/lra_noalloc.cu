// One maxvol half-step without any device memory allocation.
//
// Some callers cannot allocate device memory while they run: cudaMalloc and
// cudaFree may synchronise the whole device, and they fail or fragment the
// pool when another allocator (a framework's caching allocator, a serving
// process that reserves its memory up front) already owns most of the GPU.
// lra_maxvol_noalloc lets such callers run the same maxvol kernel as a full
// solve while passing only their own inputs and outputs.  The kernel's
// scratch (the candidate words, per-CTA candidate rows, the grid barrier, the status
// word) lives in a fixed static device array in this file instead of a
// per-job allocation.
#include <cuda_runtime.h>

#include <mutex>

#include "lra_internal.cuh"
#include "lra_kernels.h"

namespace lra {
namespace {

struct NoAllocScratch {
  JobStatus js;
  GridBarrier bar;
  int trace_i[4];
  double trace_v[1];
  unsigned long long win_ring[kWinRing];
  float2 cand_rows[2 * kMaxGrid * kMaxL];
  float2 xsplit[kMaxL * kMaxL];  // the caller's X^{-1} as FP32 pairs
};

// Static scratch: ~325 KB on every device that loads this library, held
// until the process exits.  Sized for l <= 96 and grids of <= 160 CTAs.
__device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
  void* scratch = nullptr;  // device address of g_noalloc_scratch
  int sms = 0;
  size_t smem_optin = 0;
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// First call on a device: resolve the device address of the static array
// (in host code its name is only a host-side stand-in) and the launch limits.
cudaError_t setup_device(int dev, DeviceSetup* out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.scratch) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int sms = 0, smem = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
    if ((e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    s.sms = sms;
    s.smem_optin = (size_t)smem;
    s.scratch = ptr;
  }
  *out = s;
  return cudaSuccess;
}

__global__ void noalloc_init_kernel(NoAllocScratch* s) {
  s->js = JobStatus{};
  s->js.status = LRA_OK;
  s->js.converged = 1;
  s->js.trace_cap = 0;
  s->bar.count = 0;
  s->bar.seq = 0;
  for (int i = 0; i < kWinRing; ++i) s->win_ring[i] = 0ull;
}

__global__ void noalloc_split_kernel(const double* __restrict__ xinv, int ll, NoAllocScratch* s) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ll; e += gridDim.x * blockDim.x)
    s->xsplit[e] = split_double(xinv[e]);
}

__global__ void noalloc_finish_kernel(const NoAllocScratch* s, int32_t* status_out) {
  status_out[0] = s->js.status;
  status_out[1] = s->js.swaps_total;
  status_out[2] = s->js.converged;
}

}  // namespace
}  // namespace lra

using namespace lra;

extern "C" lra_status lra_maxvol_noalloc(const float* strip, int64_t N, int32_t l,
                                         int64_t row_stride, int64_t col_stride, int32_t* pos,
                                         const double* xinv, double delta, int32_t max_swaps,
                                         int32_t* status_out, void* stream) {
  if (!strip || !pos || !status_out) return LRA_EINVAL;
  if (l < 1 || N < l || !(delta > 0.0)) return LRA_EINVAL;
  if (l > kMaxL) return LRA_ETOOLARGE;  // scratch holds rows of at most 96 entries
  // element (i, t) at strip[i*row_stride + t*col_stride]: both strides
  // positive and the N x l elements distinct (rows of l entries side by
  // side, or columns of N entries side by side), so that the kernel reads
  // only the N*l elements the caller described
  if (row_stride < 1 || col_stride < 1) return LRA_EINVAL;
  if (!(row_stride >= (int64_t)l * col_stride || col_stride >= N * row_stride)) return LRA_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LRA_ECUDA;
  DeviceSetup ds;
  if (setup_device(dev, &ds) != cudaSuccess) return LRA_ECUDA;
  MaxvolPlan plan;
  // the plan never exceeds 160 CTAs, the number of candidate rows in scratch
  if (!plan_maxvol(N, l, ds.sms, ds.smem_optin, &plan)) return LRA_ETOOLARGE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NoAllocScratch* s = static_cast<NoAllocScratch*>(ds.scratch);
  // Every launch is checked through its own return code, and the call
  // returns before enqueueing anything further when one fails.  The
  // runtime's last-error state is neither read nor cleared here, so an
  // error the caller left there stays the caller's.
  {
    void* args[] = {&s};
    if (cudaLaunchKernel(reinterpret_cast<const void*>(noalloc_init_kernel), dim3(1), dim3(1), args, 0, st))
      return LRA_ECUDA;
  }
  if (xinv) {
    int ll = l * l;
    void* args[] = {const_cast<double**>(&xinv), &ll, &s};
    if (cudaLaunchKernel(reinterpret_cast<const void*>(noalloc_split_kernel), dim3((ll + 255) / 256), dim3(256),
                         args, 0, st))
      return LRA_ECUDA;
  }
  MaxvolArgs a{};
  a.strip = strip;
  a.N = N;
  a.l = l;
  a.si = row_stride;
  a.st = col_stride;
  a.gepp = xinv ? 0 : 1;
  a.pos = pos;
  a.xin = xinv ? s->xsplit : nullptr;
  a.win_ring = s->win_ring;
  a.cand_rows = s->cand_rows;
  a.bar = &s->bar;
  a.js = &s->js;
  a.trace_i = s->trace_i;
  a.trace_v = s->trace_v;
  a.half_step = 0;
  a.delta = delta;
  a.max_swaps = max_swaps > 0 ? max_swaps : 64 * l;
  if (launch_maxvol(a, plan, st) != cudaSuccess) return LRA_ECUDA;
  {
    void* args[] = {&s, &status_out};
    if (cudaLaunchKernel(reinterpret_cast<const void*>(noalloc_finish_kernel), dim3(1), dim3(1), args, 0, st))
      return LRA_ECUDA;
  }
  return LRA_OK;
}
