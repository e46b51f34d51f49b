// Randomized SVD of the Hankel matrix with a warm start (Theory: rSVD; Algorithm 1 step 2).
//
// The r principal right singular vectors V of H(x) on region S from l test vectors Omega (n x l):
// the previous outer iteration's V (warm start) followed by complex Gaussian columns.  The sketch
// Z = H^H (H Omega) = G Omega is formed from the Gram G = H^H H of the region (the lag-form Gram
// kernels, double-word sums) and one n x n by n x l product in double-float arithmetic: H itself is
// never formed, and the Gram's cost does not grow with l as 2 l applications of H and H^H would.
// The randomized SVD of H through H^H H in single-pass form, with a small shift nu for stability
// (Halko, Martinsson & Tropp 2011; Tropp, Yurtsever, Udell & Cevher 2017):
//     Y = Z + nu Omega,   T = Omega^H Y = R^H R (Cholesky),   K = Y R^{-1},
//     K^H K = U S U^H (its top r eigenpairs),   V = K U S^{-1/2},   lambda = S - nu,
// exact when rank(H) <= l.  The shift is nu = 2^-17 ||Z||_F / sqrt(l).  The small dense steps:
// the l x l Hermitian products in FP64 (one warp per entry), the Cholesky factorisation in
// double-float (one CTA, right-looking; the matrix in shared memory when it fits), the triangular
// solve with a warp per coefficient (lanes over the sum), and the l x l eigenproblem by the
// principal-subspace solver (Householder tridiagonalisation).  J of Eq. 1 is trace(G) - sum(lambda).
#include <cmath>

#include "df.cuh"
#include "hicu_internal.cuh"

namespace hicu {

namespace {

// Y[k][i] = sum_j G[i][j] Omega[k][j] (G n x n row-major, Omega and Y [l][n], complex128):
// 32 x 32 outputs per CTA of 16 x 16 threads (2 x 2 each), tiles of 16 columns of G and Omega
// staged in shared memory as double-float, lazily normalised double-float accumulation
constexpr int GM_T = 32, GM_J = 16;
__global__ void __launch_bounds__(256) rs_gemm_kernel(int n, int l, const double2* __restrict__ G,
                                                      const double2* __restrict__ Om, double2* __restrict__ Y) {
  __shared__ float4 gs[GM_T][GM_J + 1], os[GM_T][GM_J + 1];  // +1: rows apart in different banks
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.x * GM_T, k0 = blockIdx.y * GM_T;
  cdf acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = c_zero();
  for (int j0 = 0; j0 < n; j0 += GM_J) {
    for (int e = threadIdx.x; e < GM_T * GM_J; e += 256) {
      const int rr = e / GM_J, cc = e - rr * GM_J, j = j0 + cc;
      const double2 gv = (i0 + rr < n && j < n) ? G[(long long)(i0 + rr) * n + j] : make_double2(0.0, 0.0);
      const double2 ov = (k0 + rr < l && j < n) ? Om[(long long)(k0 + rr) * n + j] : make_double2(0.0, 0.0);
      st4(&gs[rr][cc], c_from(gv));
      st4(&os[rr][cc], c_from(ov));
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < GM_J; ++jj) {
      const cdf g0 = ld4(&gs[tx][jj]), g1 = ld4(&gs[tx + 16][jj]);
      const cdf o0 = ld4(&os[ty][jj]), o1 = ld4(&os[ty + 16][jj]);
      c_acc_mul(acc[0][0], g0, o0);
      c_acc_mul(acc[0][1], g0, o1);
      c_acc_mul(acc[1][0], g1, o0);
      c_acc_mul(acc[1][1], g1, o1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + tx + 16 * a, k = k0 + ty + 16 * b;
      if (i < n && k < l) Y[(long long)k * n + i] = c_to(acc[a][b]);
    }
}

// ||Z||_F^2 accumulated in *nrm (zeroed before)
__global__ void rs_norm_kernel(long long tot, const double2* __restrict__ Z, double* __restrict__ nrm) {
  __shared__ double sh[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = Z[i];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  s = block_sum<256>(s, sh);
  if (threadIdx.x == 0) atomicAdd(nrm, s);
}

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

// T = R^H R (l x l row-major, Hermitian positive definite): on return the upper triangle of T
// holds R.  Right-looking, one CTA, in double-float on the FP32 pipe (the FP64 pipe of one SM is
// the slower one by far): W, the working copy, is shared memory when l^2 double-float entries fit
// (use_smem), else the workspace Wg.  A diagonal that is not positive sets *err
// (HICU_ERR_NUMERIC) and stops.
__global__ void __launch_bounds__(1024) rs_cholesky_kernel(int l, double2* __restrict__ T, float4* __restrict__ Wg,
                                                           int use_smem, int* __restrict__ err) {
  extern __shared__ float4 wsm[];
  __shared__ float4 s_d;  // (d, 1 / d) of the current column; d < 0 flags a failure
  float4* W = use_smem ? wsm : Wg;
  const long long ll = (long long)l * l;
  for (long long t = threadIdx.x; t < ll; t += blockDim.x) st4(&W[t], c_from(T[t]));
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    if (threadIdx.x == 0) {
      const dfl djj = ld4(&W[(long long)j * l + j]).re;  // Hermitian: real diagonal
      if (djj.hi > 0.f && isfinite(djj.hi)) {
        const dfl d = df_sqrt(djj), inv = df_rcp(d);
        s_d = make_float4(d.hi, d.lo, inv.hi, inv.lo);
      } else {
        s_d = make_float4(-1.f, 0.f, 0.f, 0.f);
        *err = HICU_ERR_NUMERIC;
      }
    }
    __syncthreads();
    const float4 dd = s_d;
    if (dd.x < 0.f) return;
    const dfl d = {dd.x, dd.y}, inv = {dd.z, dd.w};
    // row j of R: R[j][k] = W[j][k] / d for k > j, R[j][j] = d
    for (int k = j + threadIdx.x; k < l; k += blockDim.x) {
      cdf v = ld4(&W[(long long)j * l + k]);
      v = k == j ? cdf{d, {0.f, 0.f}} : cdf{df_mul(v.re, inv), df_mul(v.im, inv)};
      st4(&W[(long long)j * l + k], v);
    }
    __syncthreads();
    // trailing update of the upper triangle: W[a][b] -= conj(R[j][a]) R[j][b], j < a <= b
    const int m = l - j - 1;
    const long long mm = (long long)m * m;
    for (long long t = threadIdx.x; t < mm; t += blockDim.x) {
      const int a = j + 1 + (int)(t / m), b = j + 1 + (int)(t % m);
      if (b < a) continue;
      const cdf ra = ld4(&W[(long long)j * l + a]), rb = ld4(&W[(long long)j * l + b]);
      st4(&W[(long long)a * l + b], c_sub(ld4(&W[(long long)a * l + b]), c_mulc(ra, rb)));
    }
    __syncthreads();
  }
  for (long long t = threadIdx.x; t < ll; t += blockDim.x) {
    const int a = (int)(t / l), b = (int)(t % l);
    if (b >= a) T[t] = c_to(ld4(&W[t]));
  }
}

// K = Y R^{-1} (K R = Y, R upper; [l][n] layout): K[j][i] = (Y[j][i] - sum_{k<j} K[k][i] R[k][j]) /
// R[j][j], a warp per coefficient i, the lanes over the sum (a serial chain per coefficient would
// take l^2 / 2 dependent steps), the coefficient's K[.][i] kept in shared memory ([wpb][l])
__global__ void rs_trsm_kernel(int l, int n, const double2* __restrict__ R, const double2* __restrict__ Y,
                               double2* __restrict__ K) {
  extern __shared__ double2 ksm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long i = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= n) return;  // the whole warp
  double2* kc = ksm + (size_t)warp * l;
  for (int j = 0; j < l; ++j) {
    double re = 0.0, im = 0.0;
    for (int k = lane; k < j; k += 32) {
      const double2 kk = kc[k], rr = R[(long long)k * l + j];
      re = fma(kk.x, rr.x, fma(-kk.y, rr.y, re));
      im = fma(kk.x, rr.y, fma(kk.y, rr.x, im));
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    const double2 y = Y[(long long)j * n + i];
    const double inv = 1.0 / R[(long long)j * l + j].x;
    const double2 kv = make_double2((y.x - re) * inv, (y.y - im) * inv);
    if (lane == 0) {
      kc[j] = kv;
      K[(long long)j * n + i] = kv;
    }
    __syncwarp();
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

// trace of the Gram: the sum of its real diagonal (one CTA; *out written)
__global__ void rs_trace_kernel(int n, const double2* __restrict__ G, double* __restrict__ out) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += G[(long long)i * n + i].x;
  s = block_sum<256>(s, sh);
  if (threadIdx.x == 0) *out = s;
}

// C <- (C + C^H) / 2 (l x l row-major), so that the Cholesky factorisation and the eigen-solver see
// exactly Hermitian matrices (Omega^H Y is Hermitian only to the rounding of G Omega)
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
  const int64_t n = (int64_t)g.C * nk;
  if (r < 1 || l <= r || l > n || r0 < 0 || r0 > l || (r0 > 0 && !V_prev))
    return set_error(h, HICU_ERR_RANK, "rsvd: need 1 <= r < l <= n and 0 <= r0 <= l");
  if (l > 4096) return set_error(h, HICU_ERR_UNSUPPORTED, "rsvd: at most 4096 test vectors");
  const size_t ln = (size_t)l * n, ll = (size_t)l * l;
  double2* Om = (double2*)ws_get(h, WS_RS_OMEGA, sizeof(double2) * ln, &s);
  if (s) return s;
  double2* G = (double2*)ws_get(h, WS_RS_G, sizeof(double2) * (size_t)n * n, &s);
  if (s) return s;
  double2* Y = (double2*)ws_get(h, WS_RS_Y, sizeof(double2) * ln, &s);
  if (s) return s;
  double2* K = (double2*)ws_get(h, WS_RS_K, sizeof(double2) * ln, &s);
  if (s) return s;
  // T (l x l complex128) and the Cholesky factorisation's double-float working copy
  double2* T = (double2*)ws_get(h, WS_RS_T, sizeof(double2) * ll + sizeof(float4) * ll, &s);
  if (s) return s;
  float4* Wc = (float4*)(T + ll);
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
  // Z = H^H H Omega = G Omega, into Y
  if ((s = run_gram(h, geom, region, x, (double*)G, st, sup, kmask ? nk : 0))) return s;
  HICU_LAUNCH(h, K_EIG, st,
              rs_gemm_kernel<<<dim3((unsigned)((n + GM_T - 1) / GM_T), (unsigned)((l + GM_T - 1) / GM_T)), 256, 0,
                               st>>>((int)n, (int)l, G, Om, Y));
  if (cudaMemsetAsync(sc + l, 0, sizeof(double) * 8, st) != cudaSuccess)
    return cuda_error(h, cudaGetLastError(), "rsvd: memset");
  HICU_LAUNCH(h, K_EIG, st, rs_norm_kernel<<<cap_blocks(h, (long long)ln, 256), 256, 0, st>>>((long long)ln, Y, nrm));
  HICU_LAUNCH(h, K_EIG, st,
              rs_shift_kernel<<<cap_blocks(h, (long long)ln, 256), 256, 0, st>>>((long long)ln, (int)l, 0x1.0p-17, nrm, Om,
                                                                                  Y, nu));
  // T = Omega^H Y, its Cholesky factor, K = Y R^-1, K^H K
  const long long warps = (long long)l * l;
  const int hb = cap_blocks(h, warps, 256);
  HICU_LAUNCH(h, K_EIG, st, rs_gram_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>((int)l, (int)n, Om, Y, T));
  HICU_LAUNCH(h, K_EIG, st, rs_hermitize_kernel<<<hb, 256, 0, st>>>((int)l, T));
  {
    const size_t wbytes = sizeof(float4) * ll;
    const int use_smem = wbytes <= 200 * 1024;
    cudaError_t e0 = allow_max_dynamic_smem((const void*)rs_cholesky_kernel);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "rsvd cholesky smem");
    HICU_LAUNCH(h, K_EIG, st,
                rs_cholesky_kernel<<<1, 1024, use_smem ? wbytes : 0, st>>>((int)l, T, Wc, use_smem, h->dev_err));
  }
  {
    // warps per CTA: the coefficients' K[.][i] in shared memory, at most ~200 KB
    const size_t per_warp = sizeof(double2) * (size_t)l;
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / per_warp));
    cudaError_t e0 = allow_max_dynamic_smem((const void*)rs_trsm_kernel);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "rsvd trsm smem");
    HICU_LAUNCH(h, K_EIG, st,
                rs_trsm_kernel<<<(unsigned)((n + wpb - 1) / wpb), 32 * wpb, per_warp * wpb, st>>>((int)l, (int)n, T, Y,
                                                                                                    K));
  }
  HICU_LAUNCH(h, K_EIG, st, rs_gram_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>((int)l, (int)n, K, K, T));
  HICU_LAUNCH(h, K_EIG, st, rs_hermitize_kernel<<<hb, 256, 0, st>>>((int)l, T));
  if ((s = run_principal(h, l, r, (const double*)T, (double*)U, S, nullptr, nullptr, st))) return s;
  const long long rn = r * n;
  HICU_LAUNCH(h, K_EIG, st,
              rs_lift_kernel<<<(unsigned)((rn + 255) / 256), 256, 0, st>>>((int)r, (int)l, (int)n, U, K, S, nu,
                                                                           (double2*)V, eig_top));
  if (tail) {
    HICU_LAUNCH(h, K_EIG, st, rs_trace_kernel<<<1, 256, 0, st>>>((int)n, G, trace));
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
