// Filter gradient and unobserved-entry projection: the two extra operations the
// differentiable wrappers of the convolutions need.
//
//  filter gradient : F_k[c, d] = sum_{o in V(S)} conj(x_c[o + d]) Rbar[o, k]
//                    = H(x)^H Rbar, the adjoint of v -> H(x) v in the filter variable
//                    (the filters are the unknowns of the annihilation relation of the
//                    Theory section; with Rbar = H(x) v it is the Gram product G v)
//  projection      : out = (1 - M) o x on S, 0 elsewhere (hard data consistency)
//
// The filter gradient is a contraction over all output positions for each of the
// n p filter coefficients.  A persistent grid of CTAs walks 32 x 4 position tiles;
// each CTA stages a tile of Rbar and, coil by coil, the input halo in shared memory
// and accumulates its share of the p x n coefficients in a shared-memory array
// (FP32; every coefficient has one owning thread, so there are no atomics).  Each CTA
// then writes its partial array and one more kernel sums the partials over CTAs in
// FP64 in a fixed order, so the result is deterministic.  Large p is done in chunks
// of filters so that the accumulator fits in shared memory.
#include <algorithm>

#include "hicu_internal.cuh"

namespace hicu {

constexpr int FG_TX = 32, FG_TY = 4, FG_NT = 128, FG_POS = FG_TX * FG_TY;
constexpr size_t FG_SMEM_TARGET = 100 * 1024;  // two CTAs per SM

static size_t fgrad_smem(const ConvGeom& g, int pk) {
  const size_t hsz = (size_t)g.kz * (FG_TY + g.ky - 1) * (FG_TX + g.kx - 1);
  return sizeof(float2) * ((size_t)pk * g.n + hsz + (size_t)FG_POS * pk);
}

__global__ void __launch_bounds__(FG_NT) fgrad_kernel(ConvGeom g, KView x, const float2* __restrict__ Rb, int p,
                                                      int k0, int pk, float2* __restrict__ partial) {
  extern __shared__ float2 fsm[];
  const int HX = FG_TX + g.kx - 1, HY = FG_TY + g.ky - 1;
  const int hsz = g.kz * HY * HX;
  float2* acc = fsm;                       // [pk][n]
  float2* halo = acc + (size_t)pk * g.n;   // [kz][HY][HX] of one coil
  float2* rt = halo + hsz;                 // [FG_POS][pk]
  const int tilesx = (g.sx + FG_TX - 1) / FG_TX, tilesy = (g.sy + FG_TY - 1) / FG_TY;
  const long long ntiles = (long long)tilesx * tilesy * g.sz;
  for (int i = threadIdx.x; i < pk * g.n; i += FG_NT) acc[i] = make_float2(0.f, 0.f);
  const int outs = pk * g.K;  // coefficients of one coil
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int bx = (int)(t % tilesx);
    const long long rest = t / tilesx;
    const int by = (int)(rest % tilesy), oz = (int)(rest / tilesy);
    const int ox0 = bx * FG_TX, oy0 = by * FG_TY;
    __syncthreads();  // the previous tile's readers are done with rt
    for (int i = threadIdx.x; i < FG_POS * pk; i += FG_NT) {
      const int pos = i / pk, kk = i - pos * pk;
      const int oxp = ox0 + (pos % FG_TX), oyp = oy0 + (pos / FG_TX);
      float2 v = make_float2(0.f, 0.f);  // positions past the valid range contribute nothing
      if (oxp < g.sx && oyp < g.sy) v = Rb[(((long long)oz * g.sy + oyp) * g.sx + oxp) * p + k0 + kk];
      rt[i] = v;
    }
    for (int c = 0; c < g.C; ++c) {
      __syncthreads();
      const float2* xc = x.p + (long long)c * x.sc;
      for (int i = threadIdx.x; i < hsz; i += FG_NT) {
        const int hx = i % HX;
        const int tt = i / HX;
        const int hy = tt % HY, hz = tt / HY;
        int ix = ox0 + hx, iy = oy0 + hy, iz = oz + hz;
        bool ok = true;
        if (g.cx) ix = wrap(ix, g.ex); else ok = ok && ix < g.ex;
        if (g.cy) iy = wrap(iy, g.ey); else ok = ok && iy < g.ey;
        if (g.cz) iz = wrap(iz, g.ez); else ok = ok && iz < g.ez;
        float2 v = make_float2(0.f, 0.f);
        if (ok) v = xc[(long long)(x.oz + iz) * x.sz + (long long)(x.oy + iy) * x.sy + (x.ox + ix)];
        halo[i] = v;
      }
      __syncthreads();
      for (int o = threadIdx.x; o < outs; o += FG_NT) {
        const int kk = o / g.K, d = o - kk * g.K;
        const int dx = d % g.kx, d2 = d / g.kx;
        const int dy = d2 % g.ky, dz = d2 / g.ky;
        float sr = 0.f, si = 0.f;
        for (int ty = 0; ty < FG_TY; ++ty) {
          const float2* hrow = halo + (dz * HY + ty + dy) * HX + dx;
          const float2* rrow = rt + (ty * FG_TX) * pk + kk;
#pragma unroll 8
          for (int tx = 0; tx < FG_TX; ++tx) {
            const float2 hv = hrow[tx], rv = rrow[tx * pk];  // conj(hv) * rv
            sr = fmaf(hv.x, rv.x, fmaf(hv.y, rv.y, sr));
            si = fmaf(hv.x, rv.y, fmaf(-hv.y, rv.x, si));
          }
        }
        float2& a = acc[(size_t)kk * g.n + (size_t)c * g.K + d];
        a.x += sr;
        a.y += si;
      }
    }
  }
  __syncthreads();
  float2* out = partial + (size_t)blockIdx.x * pk * g.n;
  for (int i = threadIdx.x; i < pk * g.n; i += FG_NT) out[i] = acc[i];
}

__global__ void fgrad_reduce_kernel(int nblk, int pk, int n, int k0, const float2* __restrict__ partial,
                                    float2* __restrict__ fbar) {
  const long long tot = (long long)pk * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int b = 0; b < nblk; ++b) {
      const float2 v = partial[(size_t)b * tot + i];
      sr += v.x;
      si += v.y;
    }
    const int kk = (int)(i / n), a = (int)(i % n);
    fbar[(long long)(k0 + kk) * n + a] = make_float2((float)sr, (float)si);
  }
}

__global__ void project_unobserved_kernel(int C, int nx, int ny, int nz, int ox, int oy, int oz, int ex, int ey,
                                          int ez, const uint8_t* __restrict__ mask, int mask_per_coil,
                                          const float2* x, float2* out) {
  const long long plane = (long long)nx * ny * nz;
  const long long tot = plane * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const long long v = i % plane;
    const int c = (int)(i / plane);
    const int ix = (int)(v % nx), iy = (int)((v / nx) % ny), iz = (int)(v / ((long long)nx * ny));
    bool keep = ix >= ox && ix < ox + ex && iy >= oy && iy < oy + ey && iz >= oz && iz < oz + ez;
    if (keep && mask) keep = mask[(mask_per_coil ? (long long)c * plane : 0) + v] == 0;
    out[i] = keep ? x[i] : make_float2(0.f, 0.f);
  }
}

}  // namespace hicu

using namespace hicu;

extern "C" hicu_status hicu_conv_null_filter_grad(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                                  const float* x, const float* Rbar, int32_t p, float* fbar,
                                                  void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!x || !Rbar || !fbar) return set_error(h, HICU_ERR_ARG, "conv_null_filter_grad: null pointer");
  if (p < 1 || p > 4096) return set_error(h, HICU_ERR_RANK, "conv_null_filter_grad: p out of range");
  ConvGeom g;
  hicu_status s = make_conv_geom(h, geom, region, &g);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int pk = p;
  while (pk > 1 && fgrad_smem(g, pk) > FG_SMEM_TARGET) --pk;
  const size_t smem = fgrad_smem(g, pk);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (smem > (size_t)optin)
    return set_error(h, HICU_ERR_UNSUPPORTED, "conv_null_filter_grad: filter length too large for one CTA");
  cudaError_t e = allow_max_dynamic_smem((const void*)fgrad_kernel);
  if (e != cudaSuccess) return cuda_error(h, e, "conv_null_filter_grad smem");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fgrad_kernel, FG_NT, smem);
  if (e != cudaSuccess || per_sm < 1) return set_error(h, HICU_ERR_CUDA, "conv_null_filter_grad: occupancy");
  const long long ntiles = (long long)((g.sx + FG_TX - 1) / FG_TX) * ((g.sy + FG_TY - 1) / FG_TY) * g.sz;
  const int nblk = (int)std::max<long long>(1, std::min<long long>(ntiles, (long long)h->num_sms * per_sm));
  float2* part = (float2*)ws_get(h, WS_FGRAD, sizeof(float2) * (size_t)nblk * pk * g.n, &s);
  if (s) return s;
  const KView xv = full_view(geom, region, const_cast<float*>(x));
  for (int k0 = 0; k0 < p; k0 += pk) {
    const int kc = std::min(pk, p - k0);
    HICU_LAUNCH(h, K_MISC, st,
                fgrad_kernel<<<nblk, FG_NT, fgrad_smem(g, kc), st>>>(g, xv, (const float2*)Rbar, p, k0, kc, part));
    const long long tot = (long long)kc * g.n;
    const int rb = (int)std::min<long long>((tot + 255) / 256, 1024);
    HICU_LAUNCH(h, K_MISC, st,
                fgrad_reduce_kernel<<<rb, 256, 0, st>>>(nblk, kc, g.n, k0, part, (float2*)fbar));
  }
  return cuda_error(h, cudaGetLastError(), "conv_null_filter_grad");
}

extern "C" hicu_status hicu_project_unobserved(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                               const uint8_t* mask, const float* x, float* out, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!x || !out) return set_error(h, HICU_ERR_ARG, "project_unobserved: null pointer");
  ConvGeom g;
  hicu_status s = make_conv_geom(h, geom, region, &g);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const long long tot = geom->dim[0] * geom->dim[1] * geom->dim[2] * (long long)geom->ncoil;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, (long long)h->num_sms * 16);
  HICU_LAUNCH(h, K_MISC, st,
              project_unobserved_kernel<<<blocks, 256, 0, st>>>(
                  geom->ncoil, (int)geom->dim[0], (int)geom->dim[1], (int)geom->dim[2], (int)region->off[0],
                  (int)region->off[1], (int)region->off[2], (int)region->ext[0], (int)region->ext[1],
                  (int)region->ext[2], mask, geom->mask_per_coil, (const float2*)x, (float2*)out));
  return cuda_error(h, cudaGetLastError(), "project_unobserved");
}
