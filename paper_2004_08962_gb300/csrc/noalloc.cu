// hicu_conv_null_noalloc: the valid convolution of hicu_conv_null without a
// handle and without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they run
// the convolution, for example a host framework that has already reserved all
// free device memory for its own pool (cudaMalloc would fail), or a latency
// critical pipeline stage where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable.  The handle-based entry points own
// scratch that grows with cudaMalloc; this one uses a fixed scratch array
// compiled into the library instead.
//
// Scratch: one file-scope __device__ array (HICU_NOALLOC_SCRATCH_BYTES) holding
// the re-laid-out filter bank ([n][Ppad] complex64, Ppad = p rounded up to 16,
// at most HICU_NOALLOC_MAX_FILTER_WORDS entries) and the per-CTA partial sums of
// ||R||^2 (at most HICU_NOALLOC_MAX_PARTIALS CTAs).  Every GPU that loads the
// library keeps this array until the process exits.  Every call shares it and it
// keeps the last call's contents; every word a call reads is first written by
// that same call, so nothing has to start at zero.  Calls that overlap on the GPU
// (different streams, or several host threads) race on the array.
//
// Device address: host code cannot pass the array's name to a kernel (on the host
// it is only a stand-in symbol), so the first call on each device, with that
// device current, looks the address up with cudaGetSymbolAddress and caches it;
// that first call should come before any stream capture.  The cached address
// belongs to the device's context: a cudaDeviceReset between calls would leave
// it stale, so callers must not reset the device while they use this entry point.
//
// Shared memory: the convolution's halo tile takes 8*kz*(ky+3)*(kx+31) bytes;
// above 48 KB the call raises the kernel's dynamic shared-memory limit (a
// function attribute, no allocation), and a tile above the device's per-block
// opt-in maximum (227 KB on GB300) is refused with HICU_ERR_UNSUPPORTED.
#include <mutex>

#include "hicu_internal.cuh"

namespace {

constexpr size_t kFilterBytes = sizeof(float2) * (size_t)HICU_NOALLOC_MAX_FILTER_WORDS;
constexpr size_t kPartialBytes = sizeof(double) * (size_t)HICU_NOALLOC_MAX_PARTIALS;
static_assert(kFilterBytes + kPartialBytes == (size_t)HICU_NOALLOC_SCRATCH_BYTES, "scratch layout");
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[HICU_NOALLOC_SCRATCH_BYTES];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

hicu_status scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HICU_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return HICU_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return HICU_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HICU_OK;
}

}  // namespace

extern "C" hicu_status hicu_conv_null_noalloc(const hicu_geom* geom, const hicu_region* region,
                                              const float* x, const float* filters, int32_t p,
                                              float* R, double* objective, void* stream) {
  using namespace hicu;
  if (!x || !filters || (!R && !objective)) return HICU_ERR_ARG;
  if (p < 1 || p > 4096) return HICU_ERR_RANK;
  ConvGeom g;
  hicu_status s = make_conv_geom(nullptr, geom, region, &g);
  if (s) return s;
  const int Ppad = conv_ppad(p);
  dim3 grid, block;
  size_t smem = 0;
  conv_fp32_launch_shape(g, &grid, &block, &smem);
  const long long nblocks = (long long)grid.x * grid.y * grid.z;
  if ((long long)g.n * Ppad > HICU_NOALLOC_MAX_FILTER_WORDS || nblocks > HICU_NOALLOC_MAX_PARTIALS)
    return HICU_ERR_UNSUPPORTED;  // beyond the static scratch: use hicu_conv_null
  void* base = nullptr;
  s = scratch_for_current_device(&base);
  if (s) return s;
  if (smem > 48 * 1024) {
    // the halo tile needs the opt-in shared-memory size (a function attribute, no allocation)
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, (const void*)conv_fp32_kernel) != cudaSuccess) {
      cudaGetLastError();
      return HICU_ERR_CUDA;
    }
    if (smem + fa.sharedSizeBytes > (size_t)optin) return HICU_ERR_UNSUPPORTED;
    if (allow_max_dynamic_smem((const void*)conv_fp32_kernel) != cudaSuccess) return HICU_ERR_CUDA;
  }
  float2* fT = reinterpret_cast<float2*>(base);
  double* part = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kFilterBytes);
  cudaStream_t st = (cudaStream_t)stream;
  const long long tot = (long long)g.n * Ppad;
  int pblocks = (int)((tot + 255) / 256);
  if (pblocks > 4096) pblocks = 4096;
  prep_filters_kernel<<<pblocks, 256, 0, st>>>(g, reinterpret_cast<const float2*>(filters), p, fT, Ppad,
                                               nullptr, 0);
  conv_fp32_kernel<<<grid, block, smem, st>>>(g, full_view(geom, region, const_cast<float*>(x)), fT, p,
                                            Ppad, reinterpret_cast<float2*>(R), part);
  if (objective) sum_partials_kernel<<<1, 256, 0, st>>>(part, (int)nblocks, objective);
  if (cudaGetLastError() != cudaSuccess) return HICU_ERR_CUDA;
  return HICU_OK;
}
