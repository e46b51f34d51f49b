// Kernel masks K (Algorithm 1 takes the kernel mask as an input; the Discussion notes that
// circumscribing circular or spherical masks, instead of the rectangular box, improve SER).
//
// With a mask, a filter v holds the kernel values on the support of K only: n = C |K|
// coefficients ordered [c][support offset], the offsets in scan order (dx fastest).  The null
// space, the Gram matrix and the JL filters live on these n coefficients.  The convolutions keep
// the box layout [C][kz][ky][kx]: a support-layout bank is scattered into the box with zeros off
// the support (hicu_expand_filters), so the valid convolution and its adjoint are unchanged and
// the zero taps cost box-size work.  The Gram of the masked Hankel matrix H_K(x) is the box Gram
// restricted to the support's rows and columns, which the Gram's assembly step reads directly
// (the cell sums per lag are the same for any support).
//
// The mask itself is a small HOST array [kz][ky][kx] (nonzero = in the support).  Its two index
// maps go to the handle's workspace and are uploaded again only when the mask changes.
#include <cstring>

#include "hicu_internal.cuh"

namespace hicu {

namespace {

__global__ void support_scatter_kernel(int p, int C, int K, int nk, const int* __restrict__ inv,
                                       const float2* __restrict__ bank_sup, float2* __restrict__ bank_box) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  const long long tot = (long long)p * C * K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int kb = (int)(i % K);
    const long long fc = i / K;  // filter * C + coil
    const int j = inv[kb];
    bank_box[i] = j >= 0 ? bank_sup[fc * nk + j] : make_float2(0.f, 0.f);
  }
}

// bank_sup[k][c][j] = bank_box[k][c][sup[j]]: the support's coefficients of box-layout filters
__global__ void support_gather_kernel(int p, int C, int K, int nk, const int* __restrict__ sup,
                                      const float2* __restrict__ bank_box, float2* __restrict__ bank_sup) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  const long long tot = (long long)p * C * nk;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i % nk);
    const long long fc = i / nk;
    bank_sup[i] = bank_box[fc * K + sup[j]];
  }
}

}  // namespace

hicu_status launch_support_gather(hicu_handle* h, int p, int C, int K, int nk, const int* sup,
                                  const float2* bank_box, float2* bank_sup, cudaStream_t st) {
  const long long tot = (long long)p * C * nk;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 1024);
  launch_pdl(h, K_MISC, st, dim3(blocks), dim3(256), 0, support_gather_kernel, true, p, C, K, nk, sup, bank_box,
             bank_sup);
  return cuda_error(h, cudaGetLastError(), "support gather");
}

hicu_status support_maps(hicu_handle* h, const hicu_geom* geom, const uint8_t* kmask, const int** sup,
                         const int** inv, int* nk, cudaStream_t st) {
  if (!kmask) return set_error(h, HICU_ERR_ARG, "kernel mask: null pointer");
  const int K = geom->k[0] * geom->k[1] * geom->k[2];
  hicu_status s = HICU_OK;
  int* maps = (int*)ws_get(h, WS_SUP, sizeof(int) * 2 * (size_t)K, &s);
  if (s) return s;
  const bool same = (int)h->sup_mask.size() == K && std::memcmp(h->sup_mask.data(), kmask, K) == 0;
  if (!same) {
    std::vector<int> host(2 * (size_t)K, -1);
    int j = 0;
    for (int k = 0; k < K; ++k)
      if (kmask[k]) {
        host[j] = k;       // sup: support offset j -> box offset k
        host[K + k] = j;   // inv: box offset k -> support offset j
        ++j;
      }
    if (j == 0) return set_error(h, HICU_ERR_SHAPE, "kernel mask: empty support");
    // a pageable source: the call returns once the values are staged, so `host` may go
    if (cudaMemcpyAsync(maps, host.data(), sizeof(int) * 2 * (size_t)K, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return cuda_error(h, cudaGetLastError(), "kernel mask upload");
    h->sup_mask.assign(kmask, kmask + K);
    h->sup_nk = j;
  }
  *sup = maps;
  *inv = maps + K;
  *nk = h->sup_nk;
  return HICU_OK;
}

hicu_status launch_support_scatter(hicu_handle* h, int p, int C, int K, int nk, const int* inv,
                                   const float2* bank_sup, float2* bank_box, cudaStream_t st) {
  const long long tot = (long long)p * C * K;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 1024);
  launch_pdl(h, K_JL, st, dim3(blocks), dim3(256), 0, support_scatter_kernel, true, p, C, K, nk, inv, bank_sup,
             bank_box);
  return cuda_error(h, cudaGetLastError(), "support scatter");
}

}  // namespace hicu

using namespace hicu;

extern "C" int64_t hicu_support_length(const hicu_geom* geom, const uint8_t* kmask) {
  if (hicu_filter_length(geom) < 0 || !kmask) return -1;
  const int K = geom->k[0] * geom->k[1] * geom->k[2];
  int64_t nk = 0;
  for (int k = 0; k < K; ++k) nk += kmask[k] ? 1 : 0;
  return nk == 0 ? -1 : (int64_t)geom->ncoil * nk;
}

extern "C" hicu_status hicu_gram_support(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                         const uint8_t* kmask, const float* x, double* G, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!geom || !region || !x || !G) return set_error(h, HICU_ERR_ARG, "gram_support: null pointer");
  if (hicu_filter_length(geom) < 0) return set_error(h, HICU_ERR_SHAPE, "gram_support: invalid geometry");
  const int* sup = nullptr;
  const int* inv = nullptr;
  int nk = 0;
  cudaStream_t st = (cudaStream_t)stream;
  hicu_status s = support_maps(h, geom, kmask, &sup, &inv, &nk, st);
  if (s) return s;
  return run_gram(h, geom, region, x, G, st, sup, nk);
}

extern "C" hicu_status hicu_expand_filters(hicu_handle* h, const hicu_geom* geom, const uint8_t* kmask,
                                           const float* bank_sup, int32_t p, float* bank_box, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!geom || !bank_sup || !bank_box) return set_error(h, HICU_ERR_ARG, "expand_filters: null pointer");
  if (hicu_filter_length(geom) < 0) return set_error(h, HICU_ERR_SHAPE, "expand_filters: invalid geometry");
  if (p < 1) return set_error(h, HICU_ERR_RANK, "expand_filters: p must be at least 1");
  const int* sup = nullptr;
  const int* inv = nullptr;
  int nk = 0;
  cudaStream_t st = (cudaStream_t)stream;
  hicu_status s = support_maps(h, geom, kmask, &sup, &inv, &nk, st);
  if (s) return s;
  return launch_support_scatter(h, p, geom->ncoil, geom->k[0] * geom->k[1] * geom->k[2], nk, inv,
                                reinterpret_cast<const float2*>(bank_sup), reinterpret_cast<float2*>(bank_box), st);
}
