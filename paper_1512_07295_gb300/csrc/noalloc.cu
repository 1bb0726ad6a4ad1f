// pk_estimate_noalloc: the fused deconvolution / interlacing / shell-binning stage for callers that
// cannot allocate device memory and cannot hand the library a workspace.
//
// Some callers run where cudaMalloc is not an option: code inside a framework that owns all device
// memory and forbids allocation while its kernels run (plugins, custom operators of a graph runtime),
// services with a fixed, pre-reserved memory budget, and host callbacks that must not enter the
// allocator. This entry point keeps its scratch (per-slot window/phase tables, per-bin accumulators,
// weight sums) in a file-scope __device__ array of fixed size instead, so it allocates nothing; the
// caller still passes the transformed grids and the output arrays.
#include <mutex>

#include "host.cuh"

namespace pk {
namespace {

constexpr int kNoAllocMaxNg = 1024;
constexpr int kNoAllocMaxBins = 1024;
constexpr size_t kTablesBytes = size_t(3) * kNoAllocMaxNg * sizeof(double);
constexpr size_t kBinsBytes = size_t(kNoAllocMaxBins) * sizeof(double);
// tables | bin sums | bin |k| sums | bin counts | deterministic-mode scales | weight sums
constexpr size_t kScratchBytes = kTablesBytes + 4 * kBinsBytes + 256;

// One copy per GPU that loads the library, held until the process exits (about 56 KB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device. In host code the symbol is only a
// host-side stand-in, so the address is looked up (with that device current) on every call that is
// not being captured into a CUDA graph, which also picks up a new address after a device reset; a
// call under capture uses the address found by the device's last call outside capture (a capture may
// not start with the first call on a device).
pk_status noalloc_scratch(cudaStream_t s, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(PK_EINVAL, "device index %d out of range", dev);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress of the no-alloc scratch");
    g_noalloc_addr[dev] = p;
  } else if (!g_noalloc_addr[dev]) {
    return fail(PK_EINVAL, "pk_estimate_noalloc: make one call on device %d before capturing it into a graph", dev);
  }
  *out = g_noalloc_addr[dev];
  return PK_OK;
}

}  // namespace
}  // namespace pk

using namespace pk;

extern "C" pk_status pk_estimate_noalloc(const pk_config* cfg, const void* g1_dev, const void* g2_dev, double wsum, double w2sum,
                                         double* pk_dev, double* kmean_dev, int64_t* nmodes_dev, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (cfg->ng > kNoAllocMaxNg)
    return fail(PK_ESIZE, "pk_estimate_noalloc: ng = %d exceeds its fixed scratch limit of %d", cfg->ng, kNoAllocMaxNg);
  if (cfg->nbins > kNoAllocMaxBins)
    return fail(PK_ESIZE, "pk_estimate_noalloc: nbins = %d exceeds its fixed scratch limit of %d", cfg->nbins,
                kNoAllocMaxBins);
  if (!g1_dev || (cfg->interlace && !g2_dev) || !pk_dev || !kmean_dev || !nmodes_dev) return fail(PK_EINVAL, "bad pointers");
  if (!(wsum > 0.0) || !(w2sum > 0.0)) return fail(PK_EINVAL, "wsum and w2sum must be > 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* base = nullptr;
  if ((st = noalloc_scratch(s, &base)) != PK_OK) return st;
  char* b = static_cast<char*>(base);
  void* tables = b;
  double* bin_sum = reinterpret_cast<double*>(b + kTablesBytes);
  double* bin_k = reinterpret_cast<double*>(b + kTablesBytes + kBinsBytes);
  unsigned long long* bin_cnt = reinterpret_cast<unsigned long long*>(b + kTablesBytes + 2 * kBinsBytes);
  double* det_scale = reinterpret_cast<double*>(b + kTablesBytes + 3 * kBinsBytes);
  double* wsums = reinterpret_cast<double*>(b + kTablesBytes + 4 * kBinsBytes);
  // the scratch keeps the previous call's contents: clear the accumulators
  cudaError_t e = cudaMemsetAsync(bin_sum, 0, 3 * kBinsBytes, s);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  if ((e = launch_set_sums(wsums, wsum, w2sum, s)) != cudaSuccess) return cuda_fail(e, "set sums");
  EstimateArgs a;
  a.ng = cfg->ng;
  a.order = cfg->order;
  a.interlace = cfg->interlace;
  a.nbins = cfg->nbins;
  a.bin_lo2 = cfg->bin_lo2;
  a.bin_w2 = cfg->bin_w2;
  a.box = cfg->box;
  a.wsums = wsums;
  a.bin_sum = bin_sum;
  a.bin_k = bin_k;
  a.bin_cnt = bin_cnt;
  a.delta_out = nullptr;
  a.det_pass = cfg->prec == PK_FIXED64 ? 1 : 0;
  a.det_scale = det_scale;
  e = cfg->prec == PK_FP32 ? launch_estimate<float>(g1_dev, g2_dev, tables, a, s)
                           : launch_estimate<double>(g1_dev, g2_dev, tables, a, s);
  if (e != cudaSuccess) return cuda_fail(e, "estimate");
  e = launch_finalize(a, cfg->subtract_shot, pk_dev, kmean_dev, nmodes_dev, s);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "finalize");
}
