// Soft data consistency and the l1 proximal step.
//
// Soft data consistency (Theory: the constraint f_1 = ||M o X - X0||^2 enters the cost with a
// multiplier lambda, Eq. 3).  The descent step then minimises
//   ||H(y) Q~||^2 + lambda ||M o (y - X0)||^2     over the entries of region S,
// with gradient g = sum_k H^H(H(y) q~_k) + lambda M o (y - X0) (factor 2 dropped: the exact line
// search absorbs it) and exact step eta = ||g||^2 / (||H(g) Q~||^2 + lambda ||M o g||^2).  The
// convolution and the unmasked adjoint are the hard-consistency kernels; soft_dc_kernel adds the
// data term to g and forms the per-CTA partial sums of lambda ||M o (y - X0)||^2, ||g||^2 and
// lambda ||M o g||^2, which the step's update kernel adds to the objective, the numerator and the
// denominator of the line search.
//
// l1 proximal step (Discussion: an l1 norm of a linear sparsifying transform of X adds a
// soft-thresholding after Algorithm 1 step 8).  The transform is the centred orthonormal inverse
// DFT of every coil over the image axes (x, y, and z unless z is a circular time axis), so the
// step is x <- T^H S_tau(T x), S_tau(w) = w max(0, 1 - tau / |w|).  The centring shifts are
// circular index shifts: in the other domain they are unit-modulus modulations, which commute with
// S_tau, so the step is the uncentred transform pair around the threshold.  The two FFTs are
// cuFFT's (a plan per handle, rebuilt only when the geometry changes); the threshold and the
// normalisation are one kernel between them.
#include <cufft.h>

#include "hicu_internal.cuh"

namespace hicu {

namespace {

__global__ void soft_dc_kernel(ConvGeom g, KView gb, KView y, KView x0, MView m, float lam, double lamd,
                               double* __restrict__ part_dc, double* __restrict__ part_g,
                               double* __restrict__ part_mg) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  __shared__ double sh[8];
  float s_dc = 0.f, s_g = 0.f, s_mg = 0.f;  // FP32 per thread, FP64 across threads
  const long long total = (long long)g.C * g.ez * g.ey * g.ex;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int ux = (int)(i % g.ex);
    long long t = i / g.ex;
    const int uy = (int)(t % g.ey);
    t /= g.ey;
    const int uz = (int)(t % g.ez);
    const int c = (int)(t / g.ez);
    float2* gp = gb.p + (long long)c * gb.sc + (long long)(gb.oz + uz) * gb.sz + (long long)(gb.oy + uy) * gb.sy +
                 (gb.ox + ux);
    float2 gv = *gp;
    const long long mo = (long long)c * m.sc + (long long)(m.oz + uz) * m.sz + (long long)(m.oy + uy) * m.sy +
                         (m.ox + ux);
    if (m.p && m.p[mo]) {
      const float2 yv = y.p[(long long)c * y.sc + (long long)(y.oz + uz) * y.sz + (long long)(y.oy + uy) * y.sy +
                            (y.ox + ux)];
      const float2 xv = x0.p[(long long)c * x0.sc + (long long)(x0.oz + uz) * x0.sz +
                             (long long)(x0.oy + uy) * x0.sy + (x0.ox + ux)];
      const float dr = yv.x - xv.x, di = yv.y - xv.y;
      s_dc = fmaf(dr, dr, fmaf(di, di, s_dc));
      gv.x = fmaf(lam, dr, gv.x);
      gv.y = fmaf(lam, di, gv.y);
      *gp = gv;
      s_mg = fmaf(gv.x, gv.x, fmaf(gv.y, gv.y, s_mg));
    }
    s_g = fmaf(gv.x, gv.x, fmaf(gv.y, gv.y, s_g));
  }
  const double b_dc = block_sum<256>((double)s_dc, sh);
  const double b_g = block_sum<256>((double)s_g, sh);
  const double b_mg = block_sum<256>((double)s_mg, sh);
  if (threadIdx.x == 0) {
    part_dc[blockIdx.x] = lamd * b_dc;
    part_g[blockIdx.x] = b_g;
    part_mg[blockIdx.x] = lamd * b_mg;
  }
}

// u <- u max(0, 1 - thr / |u|) * scale (thr and scale carry the unnormalised transforms' factors)
__global__ void l1_shrink_kernel(long long n, float2* __restrict__ u, float thr, float scale) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float2 v = u[i];
    const float a = hypotf(v.x, v.y);
    const float f = a > thr ? (1.f - thr / a) * scale : 0.f;
    v.x *= f;
    v.y *= f;
    u[i] = v;
  }
}

// observed samples restored after the l1 step under hard data consistency
__global__ void restore_observed_kernel(long long n, long long per_coil, float2* __restrict__ y,
                                        const float2* __restrict__ x0, const uint8_t* __restrict__ m, long long msc) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / per_coil, o = i % per_coil;
    if (m[c * msc + o]) y[i] = x0[i];
  }
}

int grid_for(hicu_handle* h, long long total) {
  long long blocks = (total + 255) / 256;
  const long long cap = 4 * (h->num_sms > 0 ? h->num_sms : 152);
  return (int)std::max(1ll, std::min(blocks, cap));
}

}  // namespace

hicu_status launch_soft_dc(hicu_handle* h, const ConvGeom& g, KView gb, KView y, KView x0, MView m, double lam,
                           double* part_dc, double* part_g, double* part_mg, int* nblocks, cudaStream_t st) {
  const int blocks = grid_for(h, (long long)g.C * g.ez * g.ey * g.ex);
  *nblocks = blocks;
  if (!part_dc) return HICU_OK;  // sizing query
  launch_pdl(h, K_MISC, st, dim3(blocks), dim3(256), 0, soft_dc_kernel, true, g, gb, y, x0, m, (float)lam, lam,
             part_dc, part_g, part_mg);
  return cuda_error(h, cudaGetLastError(), "soft data consistency");
}

hicu_status launch_restore_observed(hicu_handle* h, const hicu_geom* geom, float* y, const float* x0,
                                    const uint8_t* mask, cudaStream_t st) {
  const long long per_coil = geom->dim[0] * geom->dim[1] * geom->dim[2];
  const long long n = per_coil * geom->ncoil;
  launch_pdl(h, K_MISC, st, dim3(grid_for(h, n)), dim3(256), 0, restore_observed_kernel, true, n, per_coil,
             reinterpret_cast<float2*>(y), reinterpret_cast<const float2*>(x0), mask,
             geom->mask_per_coil ? per_coil : 0ll);
  return cuda_error(h, cudaGetLastError(), "restore observed");
}

void release_fft(hicu_handle* h) {
  if (h->fft_have) cufftDestroy((cufftHandle)h->fft_plan);
  h->fft_have = false;
}

hicu_status run_soft_threshold(hicu_handle* h, const hicu_geom* geom, float* x, double tau, cudaStream_t st) {
  // image axes (slowest first): z unless it is circular (time) or of length 1, y, x
  int n[3], rank = 0;
  long long batch = geom->ncoil, npix = 1;
  const long long nx = geom->dim[0], ny = geom->dim[1], nz = geom->dim[2];
  if (nz > 1 && !geom->circular[2]) n[rank++] = (int)nz;
  else batch *= nz;
  if (ny > 1) n[rank++] = (int)ny;
  if (nx > 1) n[rank++] = (int)nx;
  if (rank == 0) return set_error(h, HICU_ERR_SHAPE, "soft threshold: no image axis");
  for (int a = 0; a < rank; ++a) npix *= n[a];
  const long long key[5] = {rank, n[0], rank > 1 ? n[1] : 0, rank > 2 ? n[2] : 0, batch};
  bool same = h->fft_have;
  for (int a = 0; a < 5 && same; ++a) same = h->fft_key[a] == key[a];
  if (!same) {
    release_fft(h);
    cufftHandle plan;
    if (cufftPlanMany(&plan, rank, n, nullptr, 1, (int)npix, nullptr, 1, (int)npix, CUFFT_C2C, (int)batch) !=
        CUFFT_SUCCESS)
      return set_error(h, HICU_ERR_CUDA, "soft threshold: FFT plan");
    h->fft_plan = (int)plan;
    h->fft_have = true;
    for (int a = 0; a < 5; ++a) h->fft_key[a] = key[a];
  }
  const cufftHandle plan = (cufftHandle)h->fft_plan;
  if (cufftSetStream(plan, st) != CUFFT_SUCCESS) return set_error(h, HICU_ERR_CUDA, "soft threshold: FFT stream");
  cufftComplex* u = reinterpret_cast<cufftComplex*>(x);
  if (cufftExecC2C(plan, u, u, CUFFT_INVERSE) != CUFFT_SUCCESS)
    return set_error(h, HICU_ERR_CUDA, "soft threshold: inverse FFT");
  // unnormalised inverse: T x = u / sqrt(npix); threshold tau on T x is tau sqrt(npix) on u, and the
  // unnormalised forward transform of the result divided by npix is T^H S_tau(T x)
  const long long total = batch * npix;
  HICU_LAUNCH(h, K_MISC, st,
              l1_shrink_kernel<<<grid_for(h, total), 256, 0, st>>>(
                  total, reinterpret_cast<float2*>(x), (float)(tau * std::sqrt((double)npix)), (float)(1.0 / npix)));
  if (cufftExecC2C(plan, u, u, CUFFT_FORWARD) != CUFFT_SUCCESS)
    return set_error(h, HICU_ERR_CUDA, "soft threshold: forward FFT");
  return cuda_error(h, cudaGetLastError(), "soft threshold");
}

}  // namespace hicu

using namespace hicu;

extern "C" hicu_status hicu_soft_threshold(hicu_handle* h, const hicu_geom* geom, float* x, double tau,
                                           void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!geom || !x) return set_error(h, HICU_ERR_ARG, "soft_threshold: null pointer");
  if (hicu_filter_length(geom) < 0) return set_error(h, HICU_ERR_SHAPE, "soft_threshold: invalid geometry");
  if (!(tau >= 0.0) || !std::isfinite(tau)) return set_error(h, HICU_ERR_ARG, "soft_threshold: tau must be >= 0");
  if (tau == 0.0) return HICU_OK;
  return run_soft_threshold(h, geom, x, tau, (cudaStream_t)stream);
}
