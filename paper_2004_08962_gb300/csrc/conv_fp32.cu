// Plain complex-FP32 CUDA-core forms of the HICU convolutions.
//
//  conv    : R[o, k] = sum_{c,d} x_c[o + d] q_k[c, d]          (Theory: H(x) v is the
//            valid convolution of the k-space array with kernel v)
//  adjoint : g_c[u] = (1 - M[u]) sum_k sum_d conj(q_k[c, d]) R[u - d, k]
//            (Theory: the conjugate transpose of a valid convolution is a
//            convolution; hard data consistency zeroes observed entries)
//  update  : y <- y - eta g on unobserved entries, eta = ||g||^2 / ||H(g) Q~||^2
//            (Algorithm 1 step 8, exact line search)
//
// Each CTA owns a 32 x 4 tile of positions on one z-plane; the halo of the
// input it needs is staged in shared memory, filters are read through the
// read-only path in layouts where one 16-byte load serves two filters (conv)
// or two coils (adjoint).  Per-CTA partial sums of squared norms go to a
// partials array that a single-CTA kernel reduces in a fixed order, so every
// reduction is deterministic.
#include "hicu_internal.cuh"

namespace hicu {

int conv_ppad(int p) { return (p + 15) / 16 * 16; }
int adj_cpad(int C) {
  if (C <= 4) return 4;
  if (C <= 8) return 8;
  if (C <= 16) return 16;
  if (C <= 32) return 32;
  return 64;
}

// bank [p][n] -> fT [n][Ppad] (conv) and fA [K][Ppad][Cpad] (adjoint), zero padded.
__global__ void prep_filters_kernel(ConvGeom g, const float2* __restrict__ bank, int p,
                                    float2* __restrict__ fT, int Ppad, float2* __restrict__ fA,
                                    int Cpad) {
  const long long totT = (long long)g.n * Ppad;
  const long long totA = (long long)g.K * Ppad * Cpad;
  const long long tot = totT > totA ? totT : totA;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    if (fT && i < totT) {
      const int k = (int)(i % Ppad);
      const int a = (int)(i / Ppad);
      fT[i] = (k < p) ? bank[(long long)k * g.n + a] : make_float2(0.f, 0.f);
    }
    if (fA && i < totA) {
      const int c = (int)(i % Cpad);
      const long long t = i / Cpad;
      const int k = (int)(t % Ppad);
      const int kidx = (int)(t / Ppad);
      fA[i] = (k < p && c < g.C) ? bank[(long long)k * g.n + (long long)c * g.K + kidx]
                                 : make_float2(0.f, 0.f);
    }
  }
}

hicu_status launch_prep_filters(hicu_handle* h, const ConvGeom& g, const float2* bank, int p,
                                float2* fT, int Ppad, float2* fA, int Cpad, cudaStream_t st) {
  long long tot = (long long)g.n * Ppad;
  const long long totA = (long long)g.K * Ppad * Cpad;
  if (totA > tot) tot = totA;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  HICU_LAUNCH(h, K_MISC, st, prep_filters_kernel<<<blocks, 256, 0, st>>>(g, bank, p, fT, Ppad, fA, Cpad));
  return cuda_error(h, cudaGetLastError(), "prep_filters");
}

// ------------------------------------------------------------------ conv

constexpr int CTX = 32, CTY = 4, CNT = 128, CPT = 16;

__global__ void __launch_bounds__(CNT) conv_fp32_kernel(ConvGeom g, KView x,
                                                        const float2* __restrict__ fT, int p,
                                                        int Ppad, float2* __restrict__ R,
                                                        double* __restrict__ partial) {
  extern __shared__ float2 sh[];  // one coil's halo: [kz][HY][HX]
  __shared__ double red[CNT / 32];
  const int HX = CTX + g.kx - 1, HY = CTY + g.ky - 1;
  const int hsz = g.kz * HY * HX;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int ox0 = blockIdx.x * CTX, oy0 = blockIdx.y * CTY, oz = blockIdx.z;
  const int oxp = ox0 + tx, oyp = oy0 + ty;
  const bool valid = (oxp < g.sx) && (oyp < g.sy);
  float nrm = 0.f;  // FP32 per thread, FP64 across threads (FP64 is 1/58 of the FP32 rate)
  for (int kc = 0; kc < p; kc += CPT) {
    float acc[2 * CPT];
#pragma unroll
    for (int j = 0; j < 2 * CPT; ++j) acc[j] = 0.f;
    for (int c = 0; c < g.C; ++c) {
      __syncthreads();
      const float2* xc = x.p + (long long)c * x.sc;
      for (int i = threadIdx.x; i < hsz; i += CNT) {
        const int hx = i % HX;
        const int t = i / HX;
        const int hy = t % HY, hz = t / HY;
        int ix = ox0 + hx, iy = oy0 + hy, iz = oz + hz;
        bool ok = true;
        if (g.cx) ix = wrap(ix, g.ex); else ok = ok && ix < g.ex;
        if (g.cy) iy = wrap(iy, g.ey); else ok = ok && iy < g.ey;
        if (g.cz) iz = wrap(iz, g.ez); else ok = ok && iz < g.ez;
        float2 v = make_float2(0.f, 0.f);
        if (ok) v = xc[(long long)(x.oz + iz) * x.sz + (long long)(x.oy + iy) * x.sy + (x.ox + ix)];
        sh[i] = v;
      }
      __syncthreads();
      const float2* fc = fT + (long long)c * g.K * Ppad + kc;
      for (int dz = 0; dz < g.kz; ++dz) {
        for (int dy = 0; dy < g.ky; ++dy) {
          const float2* hrow = sh + (dz * HY + ty + dy) * HX + tx;
          const float2* frow = fc + (long long)((dz * g.ky + dy) * g.kx) * Ppad;
          for (int dx = 0; dx < g.kx; ++dx) {
            const float2 xv = hrow[dx];
            const float4* f4 = reinterpret_cast<const float4*>(frow + (long long)dx * Ppad);
#pragma unroll
            for (int j = 0; j < CPT / 2; ++j) {
              const float4 f = __ldg(f4 + j);
              acc[4 * j + 0] = fmaf(xv.x, f.x, fmaf(-xv.y, f.y, acc[4 * j + 0]));
              acc[4 * j + 1] = fmaf(xv.x, f.y, fmaf(xv.y, f.x, acc[4 * j + 1]));
              acc[4 * j + 2] = fmaf(xv.x, f.z, fmaf(-xv.y, f.w, acc[4 * j + 2]));
              acc[4 * j + 3] = fmaf(xv.x, f.w, fmaf(xv.y, f.z, acc[4 * j + 3]));
            }
          }
        }
      }
    }
    if (valid) {
      const long long o = ((long long)oz * g.sy + oyp) * g.sx + oxp;
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int k = kc + j;
        if (k < p) {
          const float2 v = make_float2(acc[2 * j], acc[2 * j + 1]);
          if (R) R[o * p + k] = v;
          nrm = fmaf(v.x, v.x, fmaf(v.y, v.y, nrm));
        }
      }
    }
  }
  const double t = block_sum<CNT>(nrm, red);
  if (threadIdx.x == 0)
    partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
}

void conv_fp32_launch_shape(const ConvGeom& g, dim3* grid, dim3* block, size_t* smem) {
  *grid = dim3((g.sx + CTX - 1) / CTX, (g.sy + CTY - 1) / CTY, g.sz);
  *block = dim3(CNT);
  *smem = sizeof(float2) * g.kz * (CTY + g.ky - 1) * (CTX + g.kx - 1);
}

hicu_status launch_conv_fp32(hicu_handle* h, const ConvGeom& g, KView x, const float2* fT, int p,
                             int Ppad, float2* R, double* partial, int* nblocks, cudaStream_t st) {
  dim3 grid((g.sx + CTX - 1) / CTX, (g.sy + CTY - 1) / CTY, g.sz);
  const size_t smem = sizeof(float2) * g.kz * (CTY + g.ky - 1) * (CTX + g.kx - 1);
  *nblocks = grid.x * grid.y * grid.z;
  if (partial == nullptr) return HICU_OK;  // sizing query
  if (smem > 48 * 1024) {
    const cudaError_t e = allow_max_dynamic_smem((const void*)conv_fp32_kernel);
    if (e != cudaSuccess) return cuda_error(h, e, "conv_fp32 smem");
  }
  HICU_LAUNCH(h, K_CONV, st, conv_fp32_kernel<<<grid, CNT, smem, st>>>(g, x, fT, p, Ppad, R, partial));
  return cuda_error(h, cudaGetLastError(), "conv_fp32");
}

// --------------------------------------------------------------- adjoint

constexpr int ATX = 32, ATY = 4, ANT = 128, APK = 8;

template <int CP>
__global__ void __launch_bounds__(ANT) adjoint_fp32_kernel(ConvGeom g,
                                                           const float2* __restrict__ R,
                                                           const float2* __restrict__ fA, int p,
                                                           int Ppad, MView m, KView gout,
                                                           double* __restrict__ partial) {
  extern __shared__ float2 sh[];  // [APK][HY][HX] slice of R around the tile
  __shared__ double red[ANT / 32];
  const int HX = ATX + g.kx - 1, HY = ATY + g.ky - 1;
  const int plane = HY * HX;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int ux0 = blockIdx.x * ATX, uy0 = blockIdx.y * ATY, uz = blockIdx.z;
  const int ux = ux0 + tx, uy = uy0 + ty;
  const bool valid = (ux < g.ex) && (uy < g.ey);
  float acc[2 * CP];
#pragma unroll
  for (int j = 0; j < 2 * CP; ++j) acc[j] = 0.f;

  for (int dz = 0; dz < g.kz; ++dz) {
    int oz = uz - dz;
    if (g.cz) oz = wrap(oz, g.ez);
    else if (oz < 0 || oz >= g.sz) continue;  // uniform over the CTA
    for (int kc = 0; kc < p; kc += APK) {
      __syncthreads();
      for (int i = threadIdx.x; i < APK * plane; i += ANT) {
        const int j = i / plane;
        const int t = i - j * plane;
        const int hy = t / HX, hx = t - (t / HX) * HX;
        const int k = kc + j;
        int ox = ux0 - (g.kx - 1) + hx, oy = uy0 - (g.ky - 1) + hy;
        bool ok = k < p;
        if (g.cx) ox = wrap(ox, g.ex); else ok = ok && ox >= 0 && ox < g.sx;
        if (g.cy) oy = wrap(oy, g.ey); else ok = ok && oy >= 0 && oy < g.sy;
        float2 v = make_float2(0.f, 0.f);
        if (ok) v = R[(((long long)oz * g.sy + oy) * g.sx + ox) * p + k];
        sh[i] = v;
      }
      __syncthreads();
      for (int dy = 0; dy < g.ky; ++dy) {
        for (int dx = 0; dx < g.kx; ++dx) {
          const float2* hp = sh + (ty + g.ky - 1 - dy) * HX + (tx + g.kx - 1 - dx);
          const float2* fb =
              fA + ((long long)((dz * g.ky + dy) * g.kx + dx) * Ppad + kc) * CP;
#pragma unroll 2
          for (int j = 0; j < APK; ++j) {
            const float2 r = hp[j * plane];
            const float4* f4 = reinterpret_cast<const float4*>(fb + j * CP);
#pragma unroll
            for (int c2 = 0; c2 < CP / 2; ++c2) {
              const float4 f = __ldg(f4 + c2);
              // acc[c] += conj(f_c) * r
              acc[4 * c2 + 0] = fmaf(f.x, r.x, fmaf(f.y, r.y, acc[4 * c2 + 0]));
              acc[4 * c2 + 1] = fmaf(f.x, r.y, fmaf(-f.y, r.x, acc[4 * c2 + 1]));
              acc[4 * c2 + 2] = fmaf(f.z, r.x, fmaf(f.w, r.y, acc[4 * c2 + 2]));
              acc[4 * c2 + 3] = fmaf(f.z, r.y, fmaf(-f.w, r.x, acc[4 * c2 + 3]));
            }
          }
        }
      }
    }
  }
  float nrm = 0.f;
  if (valid) {
    const long long mo = (long long)(m.oz + uz) * m.sz + (long long)(m.oy + uy) * m.sy + (m.ox + ux);
    const long long go = (long long)(gout.oz + uz) * gout.sz + (long long)(gout.oy + uy) * gout.sy +
                         (gout.ox + ux);
#pragma unroll
    for (int c = 0; c < CP; ++c) {
      if (c < g.C) {
        bool observed = false;
        if (m.p) observed = m.p[(long long)c * m.sc + mo] != 0;
        float2 v = make_float2(acc[2 * c], acc[2 * c + 1]);
        if (observed) v = make_float2(0.f, 0.f);
        gout.p[(long long)c * gout.sc + go] = v;
        nrm = fmaf(v.x, v.x, fmaf(v.y, v.y, nrm));
      }
    }
  }
  const double t = block_sum<ANT>((double)nrm, red);
  if (threadIdx.x == 0)
    partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
}

hicu_status launch_adjoint_fp32(hicu_handle* h, const ConvGeom& g, const float2* R,
                                const float2* fA, int p, int Ppad, int Cpad, MView m, KView gout,
                                double* partial, int* nblocks, cudaStream_t st) {
  dim3 grid((g.ex + ATX - 1) / ATX, (g.ey + ATY - 1) / ATY, g.ez);
  *nblocks = grid.x * grid.y * grid.z;
  if (partial == nullptr) return HICU_OK;
  const size_t smem = sizeof(float2) * APK * (ATY + g.ky - 1) * (ATX + g.kx - 1);
  switch (Cpad) {
    case 4: HICU_LAUNCH(h, K_ADJOINT, st, adjoint_fp32_kernel<4><<<grid, ANT, smem, st>>>(g, R, fA, p, Ppad, m, gout, partial)); break;
    case 8: HICU_LAUNCH(h, K_ADJOINT, st, adjoint_fp32_kernel<8><<<grid, ANT, smem, st>>>(g, R, fA, p, Ppad, m, gout, partial)); break;
    case 16: HICU_LAUNCH(h, K_ADJOINT, st, adjoint_fp32_kernel<16><<<grid, ANT, smem, st>>>(g, R, fA, p, Ppad, m, gout, partial)); break;
    case 32: HICU_LAUNCH(h, K_ADJOINT, st, adjoint_fp32_kernel<32><<<grid, ANT, smem, st>>>(g, R, fA, p, Ppad, m, gout, partial)); break;
    case 64: HICU_LAUNCH(h, K_ADJOINT, st, adjoint_fp32_kernel<64><<<grid, ANT, smem, st>>>(g, R, fA, p, Ppad, m, gout, partial)); break;
    default: return set_error(h, HICU_ERR_UNSUPPORTED, "adjoint: coil count above 64");
  }
  return cuda_error(h, cudaGetLastError(), "adjoint_fp32");
}

// ------------------------------------------------------------ reductions

__device__ double fixed_order_sum(const double* v, int n, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += v[i];
  return block_sum<256>(s, sh);
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double* out) {
  __shared__ double sh[8];
  const double s = fixed_order_sum(part, n, sh);
  if (threadIdx.x == 0) *out = s;
}

hicu_status launch_sum_partials(hicu_handle* h, const double* partial, int n, double* out,
                                cudaStream_t st) {
  HICU_LAUNCH(h, K_MISC, st, sum_partials_kernel<<<1, 256, 0, st>>>(partial, n, out));
  return cudaGetLastError() == cudaSuccess ? HICU_OK : HICU_ERR_CUDA;
}

// The descent step's finalisation and update in one launch: every CTA forms {eta, objective,
// ||g||^2, D} from the partial sums in the same fixed order (so all agree bitwise), CTA 0 stores
// them, and every CTA applies y <- y - eta g to its share of the unobserved entries.
__global__ void update_step_kernel(ConvGeom g, KView y, KView gb, MView m, const double* __restrict__ part,
                                   int n_obj, int n_g, int n_d, double* stats) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  __shared__ double sh[8];
  __shared__ double s_eta;
  const double obj = fixed_order_sum(part, n_obj, sh);
  const double gn2 = fixed_order_sum(part + n_obj, n_g, sh);
  const double D = fixed_order_sum(part + n_obj + n_g, n_d, sh);
  if (threadIdx.x == 0) {
    double eta = 0.0;
    if (D > 0.0 && gn2 > 0.0 && isfinite(D) && isfinite(gn2)) eta = gn2 / D;
    if (blockIdx.x == 0) {
      stats[0] = eta;
      stats[1] = obj;
      stats[2] = gn2;
      stats[3] = D;
    }
    s_eta = eta;
  }
  __syncthreads();
  const double eta = s_eta;
  if (eta == 0.0) return;
  const float e = (float)eta;
  const long long total = (long long)g.C * g.ez * g.ey * g.ex;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int ux = (int)(i % g.ex);
    long long t = i / g.ex;
    const int uy = (int)(t % g.ey);
    t /= g.ey;
    const int uz = (int)(t % g.ez);
    const int c = (int)(t / g.ez);
    if (m.p) {
      const long long mo = (long long)c * m.sc + (long long)(m.oz + uz) * m.sz +
                           (long long)(m.oy + uy) * m.sy + (m.ox + ux);
      if (m.p[mo]) continue;
    }
    const float2 gv = gb.p[(long long)c * gb.sc + (long long)(gb.oz + uz) * gb.sz +
                           (long long)(gb.oy + uy) * gb.sy + (gb.ox + ux)];
    float2* yp = y.p + (long long)c * y.sc + (long long)(y.oz + uz) * y.sz +
                 (long long)(y.oy + uy) * y.sy + (y.ox + ux);
    float2 yv = *yp;
    yv.x = fmaf(-e, gv.x, yv.x);
    yv.y = fmaf(-e, gv.y, yv.y);
    *yp = yv;
  }
}

hicu_status launch_update_step(hicu_handle* h, const ConvGeom& g, KView y, KView gb, MView m, const double* part,
                               int n_obj, int n_g, int n_d, double* stats, cudaStream_t st) {
  const long long total = (long long)g.C * g.ez * g.ey * g.ex;
  // one wave of CTAs (each forms eta once, then strides over its share)
  int blocks = (int)((total + 255) / 256);
  const int cap = 4 * (h->num_sms > 0 ? h->num_sms : 152);
  if (blocks > cap) blocks = cap;
  launch_pdl(h, K_MISC, st, dim3(blocks), dim3(256), 0, update_step_kernel, true, g, y, gb, m, part, n_obj, n_g,
             n_d, stats);
  return cudaGetLastError() == cudaSuccess ? HICU_OK : HICU_ERR_CUDA;
}


}  // namespace hicu
