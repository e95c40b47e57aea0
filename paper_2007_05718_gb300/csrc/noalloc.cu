// FP64 total energy of a dense population array without any allocation.
//
// Some callers cannot allocate device memory at the point where they want
// this number: code running while another framework owns the device memory
// pool, a real-time loop where allocation latency is not allowed, or a host
// process whose memory budget is fixed up front.  lb_rt_total_energy_noalloc
// gives them the same reduction as the library's energy-budget kernel
// (float32 sum over the directions of a site, FP64 sum over sites) with the
// per-block partial sums kept in a fixed file-scope device array instead of
// library-allocated scratch.
//
// The array is shared by every call on a device and keeps the last call's
// partials; each call overwrites exactly the slots it reads, so nothing has
// to be cleared, but two calls that run at the same time on the GPU (for
// example on two streams) race on it.
#include <mutex>
#include <string>

#include "lb_rt_internal.h"

namespace {

constexpr int kBlock = 256;                 // threads per block
constexpr int kSitesPerThread = 16;         // sites a thread reduces at most
constexpr int kMaxBlocks = 4096;            // partial slots in the static array
constexpr long long kMaxSites = (long long)kMaxBlocks * kBlock * kSitesPerThread;

// kMaxBlocks partial sums plus one result slot (read back for host outputs).
static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks + 1];

std::mutex g_setup_mutex;
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};  // device address of the array, per device

__global__ void k_partials(const float* __restrict__ pop, int ndir, long long sites,
                           double* __restrict__ partials) {
  __shared__ double sh[kBlock];
  double acc = 0.0;
  for (long long s = blockIdx.x * (long long)kBlock + threadIdx.x; s < sites;
       s += (long long)gridDim.x * kBlock) {
    float e = 0.f;
    for (int i = 0; i < ndir; ++i) e += pop[(size_t)i * sites + s];
    acc += (double)e;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void k_finish(const double* __restrict__ partials, int n, double* out) {
  __shared__ double sh[kBlock];
  double a = 0.0;
  for (int k = threadIdx.x; k < n; k += kBlock) a += partials[k];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int w = kBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

extern "C" lb_rt_status lb_rt_total_energy_noalloc(const float* pop, int ndir, long long sites,
                                                   double* out, int ptr_kind, void* stream) {
  auto bad = [](lb_rt_status st, const std::string& m) {
    lbrt::set_unbound_error("lb_rt_total_energy_noalloc: " + m);
    return st;
  };
  if (!pop || !out) return bad(LB_RT_EINVAL, "null pointer");
  if (ndir < 1 || sites < 1) return bad(LB_RT_EINVAL, "ndir and sites must be >= 1");
  if (ptr_kind != LB_RT_HOST && ptr_kind != LB_RT_DEVICE) return bad(LB_RT_EINVAL, "bad ptr_kind");
  if (sites > kMaxSites)
    return bad(LB_RT_EINVAL, std::to_string(sites) + " sites exceed the fixed scratch limit of " +
                                 std::to_string(kMaxSites));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bad(LB_RT_ECUDA, cudaGetErrorString(e));
  // the kernels dereference pop (and out for a device result): a host
  // pointer would fault on the GPU, so it is refused here
  auto device_reachable = [](const void* q) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
      (void)cudaGetLastError();
      return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
  };
  if (!device_reachable(pop)) return bad(LB_RT_EINVAL, "pop is not device or managed memory");
  if (ptr_kind == LB_RT_DEVICE && !device_reachable(out))
    return bad(LB_RT_EINVAL, "out is not device or managed memory (ptr_kind LB_RT_DEVICE)");
  if (dev < 0 || dev >= kMaxDevices) return bad(LB_RT_ECUDA, "device ordinal out of range");
  double* scratch = nullptr;
  {
    // set-up, once per device, with that device current: host code must use
    // the array's device address, never the host-side symbol
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return bad(LB_RT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long per_block = (long long)kBlock * kSitesPerThread;
  const int blocks = (int)((sites + per_block - 1) / per_block);  // 1 .. kMaxBlocks
  k_partials<<<blocks, kBlock, 0, s>>>(pop, ndir, sites, scratch);
  double* result = ptr_kind == LB_RT_DEVICE ? out : scratch + kMaxBlocks;
  k_finish<<<1, kBlock, 0, s>>>(scratch, blocks, result);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bad(LB_RT_ECUDA, cudaGetErrorString(e));
  if (ptr_kind == LB_RT_HOST) {
    e = cudaMemcpyAsync(out, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bad(LB_RT_ECUDA, cudaGetErrorString(e));
  }
  return LB_RT_OK;
}
