// Randomized SVD of the Hankel matrix with a warm start (Theory: rSVD; Algorithm 1 step 2).
//
// The r principal right singular vectors V of H(x) on region S from l test vectors Omega (n x l):
// the previous outer iteration's V (warm start) followed by complex Gaussian columns.  One valid
// convolution with the l test vectors as filters and one filter gradient (the convolution's
// conjugate transpose) give Z = H^H (H Omega) = (H^H H) Omega: 2 l applications of H and H^H, H
// never formed.  The randomized SVD of H through H^H H in single-pass form, with a small shift nu
// for stability (Halko, Martinsson & Tropp 2011; Tropp, Yurtsever, Udell & Cevher 2017):
//     Y = Z + nu Omega,   T = Omega^H Y = R^H R (Cholesky),   K = Y R^{-1},
//     K^H K = U S U^H (its top r eigenpairs),   V = K U S^{-1/2},   lambda = S - nu,
// exact when rank(H) <= l.  The shift nu = 2^-17 ||Z||_F / sqrt(l) sits above the rounding of the
// FP32 convolution and filter gradient that form Z (a smaller one lets that rounding into the
// smallest directions of Omega^H Y).  The small dense steps run in FP64: the l x l Hermitian
// products (one warp per entry), the Cholesky factorisation (one CTA, right-looking), the
// triangular solve (a thread per coefficient), and the l x l eigenproblem by the principal-subspace
// solver (Householder tridiagonalisation).  J of Eq. 1 is trace(G) - sum(lambda), the trace being
// the energy of x over the windows of the kernel offsets.
#include <cmath>

#include "hicu_internal.cuh"

namespace hicu {

namespace {

// C[a][b] = sum_i conj(A[a][i]) B[b][i], A and B complex128 [l][n] (one warp per entry; C is
// Hermitian when A = B, and both triangles are formed so the result is exactly what was summed)
__global__ void rs_gram_kernel(int l, int n, const double2* __restrict__ A, const double2* __restrict__ B,
                               double2* __restrict__ C) {
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long long)l * l) return;
  const int a = (int)(warp / l), b = (int)(warp % l);
  const double2* pa = A + (long long)a * n;
  const double2* pb = B + (long long)b * n;
  double re = 0.0, im = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double2 u = pa[i], v = pb[i];
    re = fma(u.x, v.x, fma(u.y, v.y, re));
    im = fma(u.x, v.y, fma(-u.y, v.x, im));
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) C[warp] = make_double2(re, im);
}

// Z (complex64 [l][n] filter gradient) -> complex128, ||Z||_F^2 accumulated in *nrm (zeroed before)
__global__ void rs_widen_kernel(long long tot, const float2* __restrict__ Zf, double2* __restrict__ Z,
                                double* __restrict__ nrm) {
  __shared__ double sh[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = Zf[i];
    Z[i] = make_double2(v.x, v.y);
    s += (double)v.x * v.x + (double)v.y * v.y;
  }
  s = block_sum<256>(s, sh);
  if (threadIdx.x == 0) atomicAdd(nrm, s);
}

// Y = Z + nu Omega, nu = shift * sqrt(||Z||^2 / l) (nu written to *nu_out by thread 0)
__global__ void rs_shift_kernel(long long tot, int l, double shift, const double* __restrict__ nrm,
                                const double2* __restrict__ Omega, double2* __restrict__ Y, double* __restrict__ nu_out) {
  const double nu = shift * sqrt(*nrm / (double)l);
  if (blockIdx.x == 0 && threadIdx.x == 0) *nu_out = nu;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const double2 z = Y[i], o = Omega[i];
    Y[i] = make_double2(fma(nu, o.x, z.x), fma(nu, o.y, z.y));
  }
}

// T = R^H R in place (l x l row-major; the upper triangle becomes R, row j scaled by 1 / R[j][j]
// applied as it is formed).  Right-looking, one CTA; the lower triangle is left as it was.
// A diagonal that is not positive sets *err (HICU_ERR_NUMERIC) and stops.
__global__ void __launch_bounds__(1024) rs_cholesky_kernel(int l, double2* __restrict__ T, int* __restrict__ err) {
  __shared__ double s_d;
  for (int j = 0; j < l; ++j) {
    if (threadIdx.x == 0) {
      const double d = T[(long long)j * l + j].x;   // Hermitian: real diagonal
      s_d = d > 0.0 && isfinite(d) ? sqrt(d) : -1.0;
      if (s_d < 0.0) *err = HICU_ERR_NUMERIC;
    }
    __syncthreads();
    const double d = s_d;
    if (d < 0.0) return;
    const double inv = 1.0 / d;
    // row j of R: R[j][k] = T[j][k] / d for k > j, R[j][j] = d
    for (int k = j + threadIdx.x; k < l; k += blockDim.x) {
      double2 v = T[(long long)j * l + k];
      if (k == j) v = make_double2(d, 0.0);
      else v = make_double2(v.x * inv, v.y * inv);
      T[(long long)j * l + k] = v;
    }
    __syncthreads();
    // trailing update of the upper triangle: T[a][b] -= conj(R[j][a]) R[j][b], j < a <= b
    const long long m = l - j - 1;
    for (long long t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int a = j + 1 + (int)(t / m), b = j + 1 + (int)(t % m);
      if (b < a) continue;
      const double2 ra = T[(long long)j * l + a], rb = T[(long long)j * l + b];
      double2 v = T[(long long)a * l + b];
      v.x -= ra.x * rb.x + ra.y * rb.y;
      v.y -= ra.x * rb.y - ra.y * rb.x;
      T[(long long)a * l + b] = v;
    }
    __syncthreads();
  }
}

// K = Y R^{-1}, column by column (K R = Y, R upper): K[j][i] = (Y[j][i] - sum_{k<j} K[k][i] R[k][j]) / R[j][j];
// a thread per coefficient i, [l][n] layout (coalesced over i)
__global__ void rs_trsm_kernel(int l, int n, const double2* __restrict__ R, const double2* __restrict__ Y,
                               double2* __restrict__ K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = 0; j < l; ++j) {
    double2 acc = Y[(long long)j * n + i];
    for (int k = 0; k < j; ++k) {
      const double2 kk = K[(long long)k * n + i], rr = R[(long long)k * l + j];
      acc.x -= kk.x * rr.x - kk.y * rr.y;
      acc.y -= kk.x * rr.y + kk.y * rr.x;
    }
    const double inv = 1.0 / R[(long long)j * l + j].x;
    K[(long long)j * n + i] = make_double2(acc.x * inv, acc.y * inv);
  }
}

// V[j][i] = sum_k U[j][k] K[k][i] / sqrt(S[j]), eig_top[j] = S[j] - nu (at least 0)
__global__ void rs_lift_kernel(int r, int l, int n, const double2* __restrict__ U, const double2* __restrict__ K,
                               const double* __restrict__ S, const double* __restrict__ nu, double2* __restrict__ V,
                               double* __restrict__ eig_top) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < r && eig_top) eig_top[t] = fmax(S[t] - *nu, 0.0);
  if (t >= (long long)r * n) return;
  const int j = (int)(t / n), i = (int)(t % n);
  double re = 0.0, im = 0.0;
  for (int k = 0; k < l; ++k) {
    const double2 u = U[(long long)j * l + k], kk = K[(long long)k * n + i];
    re = fma(u.x, kk.x, fma(-u.y, kk.y, re));
    im = fma(u.x, kk.y, fma(u.y, kk.x, im));
  }
  const double s = S[j] > 0.0 ? 1.0 / sqrt(S[j]) : 0.0;
  V[t] = make_double2(re * s, im * s);
}

// trace of the Gram: sum over coils c and support offsets d of |x_c|^2 over the window W(d) (a CTA
// per (c, d)); *out gets the sum (zeroed before)
__global__ void rs_trace_kernel(ConvGeom g, KView x, const int* __restrict__ sup, int nk, double* __restrict__ out) {
  __shared__ double sh[8];
  const int c = blockIdx.x / nk, j = blockIdx.x % nk;
  const int kb = sup ? sup[j] : j;
  const int dx = kb % g.kx, dy = (kb / g.kx) % g.ky, dz = kb / (g.kx * g.ky);
  const float2* xc = x.p + (long long)c * x.sc;
  double s = 0.0;
  for (long long o = threadIdx.x; o < g.s; o += blockDim.x) {
    const int ox = (int)(o % g.sx), oy = (int)((o / g.sx) % g.sy), oz = (int)(o / ((long long)g.sx * g.sy));
    const int ix = g.cx ? wrap(ox + dx, g.ex) : ox + dx;
    const int iy = g.cy ? wrap(oy + dy, g.ey) : oy + dy;
    const int iz = g.cz ? wrap(oz + dz, g.ez) : oz + dz;
    const float2 v = xc[(long long)(x.oz + iz) * x.sz + (long long)(x.oy + iy) * x.sy + (x.ox + ix)];
    s += (double)v.x * v.x + (double)v.y * v.y;
  }
  s = block_sum<256>(s, sh);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

// C <- (C + C^H) / 2 (l x l row-major), so that the Cholesky factorisation and the eigen-solver see
// exactly Hermitian matrices (the FP32 filter gradient leaves Omega^H Z Hermitian only to rounding)
__global__ void rs_hermitize_kernel(int l, double2* __restrict__ C) {
  const long long tot = (long long)l * l;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t / l), b = (int)(t % l);
    if (b < a) continue;
    const double2 u = C[(long long)a * l + b], v = C[(long long)b * l + a];
    const double2 m = make_double2(0.5 * (u.x + v.x), 0.5 * (u.y - v.y));
    C[(long long)a * l + b] = m;
    C[(long long)b * l + a] = make_double2(m.x, -m.y);
  }
}

__global__ void rs_tail_kernel(int r, const double* __restrict__ trace, const double* __restrict__ eig,
                               double* __restrict__ tail) {
  double s = *trace;
  for (int j = 0; j < r; ++j) s -= eig[j];
  *tail = fmax(s, 0.0);
}

int cap_blocks(hicu_handle* h, long long tot, int per) {
  long long b = (tot + per - 1) / per;
  const long long cap = 8ll * (h->num_sms > 0 ? h->num_sms : 152);
  return (int)std::max(1ll, std::min(b, cap));
}

}  // namespace

hicu_status run_rsvd(hicu_handle* h, const hicu_geom* geom, const hicu_region* region, const uint8_t* kmask,
                     const float* x, int64_t r, int64_t l, const double* V_prev, int64_t r0, uint64_t seed,
                     uint64_t counter, double* V, double* eig_top, double* tail, cudaStream_t st) {
  ConvGeom g;
  hicu_status s = make_conv_geom(h, geom, region, &g);
  if (s) return s;
  const int* sup = nullptr;
  const int* inv = nullptr;
  int nk = g.K;
  if (kmask && (s = support_maps(h, geom, kmask, &sup, &inv, &nk, st))) return s;
  const int64_t n = (int64_t)g.C * nk, nbox = g.n;
  if (r < 1 || l <= r || l > n || r0 < 0 || r0 > l || (r0 > 0 && !V_prev))
    return set_error(h, HICU_ERR_RANK, "rsvd: need 1 <= r < l <= n and 0 <= r0 <= l");
  if (l > 4096) return set_error(h, HICU_ERR_UNSUPPORTED, "rsvd: at most 4096 test vectors");
  const size_t ln = (size_t)l * n;
  double2* Om = (double2*)ws_get(h, WS_RS_OMEGA, sizeof(double2) * ln, &s);
  if (s) return s;
  float2* bank = (float2*)ws_get(h, WS_RS_BANK, sizeof(float2) * (size_t)l * nbox, &s);
  if (s) return s;
  float2* Rc = (float2*)ws_get(h, WS_RS_R, sizeof(float2) * (size_t)g.s * l, &s);
  if (s) return s;
  double2* Y = (double2*)ws_get(h, WS_RS_Y, sizeof(double2) * ln, &s);
  if (s) return s;
  double2* K = (double2*)ws_get(h, WS_RS_K, sizeof(double2) * ln, &s);
  if (s) return s;
  double2* T = (double2*)ws_get(h, WS_RS_T, sizeof(double2) * (size_t)l * l, &s);
  if (s) return s;
  double2* U = (double2*)ws_get(h, WS_RS_U, sizeof(double2) * (size_t)r * l, &s);
  if (s) return s;
  double* sc = (double*)ws_get(h, WS_RS_SCAL, sizeof(double) * (size_t)(l + 8), &s);
  if (s) return s;
  double* S = sc;            // [r] eigenvalues of K^H K (ascending)
  double* nrm = sc + l;      // ||Z||^2
  double* nu = sc + l + 1;   // the shift
  double* trace = sc + l + 2;
  // Omega: warm-start rows, then complex Gaussian rows
  if ((s = launch_rsvd_omega(h, n, l, r0, V_prev, seed, counter, Om, st))) return s;
  // Z = H^H (H Omega): the test vectors as a filter bank in the convolutions' box layout
  if ((s = launch_to_c64(h, (const double*)Om, bank, (long long)ln, st))) return s;
  float2* boxbank = bank;
  float2* Zf = nullptr;
  if (kmask) {
    boxbank = (float2*)ws_get(h, WS_RS_BOX, sizeof(float2) * (size_t)l * nbox, &s);
    if (s) return s;
    if ((s = launch_support_scatter(h, (int)l, g.C, g.K, nk, inv, bank, boxbank, st))) return s;
  }
  if ((s = hicu_conv_null(h, geom, region, x, (const float*)boxbank, (int32_t)l, (float*)Rc, nullptr, HICU_FP32, st)))
    return s;
  if ((s = hicu_conv_null_filter_grad(h, geom, region, x, (const float*)Rc, (int32_t)l, (float*)boxbank, st)))
    return s;
  Zf = boxbank;
  if (kmask) {
    if ((s = launch_support_gather(h, (int)l, g.C, g.K, nk, sup, boxbank, bank, st))) return s;
    Zf = bank;
  }
  if (cudaMemsetAsync(sc + l, 0, sizeof(double) * 8, st) != cudaSuccess)
    return cuda_error(h, cudaGetLastError(), "rsvd: memset");
  HICU_LAUNCH(h, K_EIG, st, rs_widen_kernel<<<cap_blocks(h, (long long)ln, 256), 256, 0, st>>>((long long)ln, Zf, Y, nrm));
  HICU_LAUNCH(h, K_EIG, st,
              rs_shift_kernel<<<cap_blocks(h, (long long)ln, 256), 256, 0, st>>>((long long)ln, (int)l, 0x1.0p-17, nrm, Om,
                                                                                  Y, nu));
  // T = Omega^H Y, its Cholesky factor, K = Y R^-1, K^H K
  const long long warps = (long long)l * l;
  const int hb = cap_blocks(h, warps, 256);
  HICU_LAUNCH(h, K_EIG, st, rs_gram_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>((int)l, (int)n, Om, Y, T));
  HICU_LAUNCH(h, K_EIG, st, rs_hermitize_kernel<<<hb, 256, 0, st>>>((int)l, T));
  HICU_LAUNCH(h, K_EIG, st, rs_cholesky_kernel<<<1, 1024, 0, st>>>((int)l, T, h->dev_err));
  HICU_LAUNCH(h, K_EIG, st, rs_trsm_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>((int)l, (int)n, T, Y, K));
  HICU_LAUNCH(h, K_EIG, st, rs_gram_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>((int)l, (int)n, K, K, T));
  HICU_LAUNCH(h, K_EIG, st, rs_hermitize_kernel<<<hb, 256, 0, st>>>((int)l, T));
  if ((s = run_principal(h, l, r, (const double*)T, (double*)U, S, nullptr, nullptr, st))) return s;
  const long long rn = r * n;
  HICU_LAUNCH(h, K_EIG, st,
              rs_lift_kernel<<<(unsigned)((rn + 255) / 256), 256, 0, st>>>((int)r, (int)l, (int)n, U, K, S, nu,
                                                                           (double2*)V, eig_top));
  if (tail) {
    const KView xv = full_view(geom, region, const_cast<float*>(x));
    HICU_LAUNCH(h, K_EIG, st, rs_trace_kernel<<<(unsigned)(g.C * nk), 256, 0, st>>>(g, xv, sup, nk, trace));
    HICU_LAUNCH(h, K_EIG, st, rs_tail_kernel<<<1, 1, 0, st>>>((int)r, trace, eig_top, tail));
  }
  return cuda_error(h, cudaGetLastError(), "rsvd");
}

}  // namespace hicu

using namespace hicu;

extern "C" hicu_status hicu_principal_rsvd(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                           const uint8_t* kmask, const float* x, int64_t r, int64_t l,
                                           const double* V_prev, int64_t r0, uint64_t seed, uint64_t counter,
                                           double* V, double* eig_top, double* tail, void* stream) {
  if (!h) return HICU_ERR_ARG;
  if (!geom || !region || !x || !V || !eig_top) return set_error(h, HICU_ERR_ARG, "principal_rsvd: null pointer");
  if (hicu_filter_length(geom) < 0) return set_error(h, HICU_ERR_SHAPE, "principal_rsvd: invalid geometry");
  return run_rsvd(h, geom, region, kmask, x, r, l, V_prev, r0, seed, counter, V, eig_top, tail, (cudaStream_t)stream);
}
