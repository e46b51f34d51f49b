// JL compression of the null space (Algorithm 1 step 6; Theory, JL paragraph):
// Q~ = Q P with P i.i.d. zero-mean Gaussian of variance 1/p, drawn afresh for
// every descent step.  Projector form Q~ = Q Q^H P, and the same filters from the
// principal vectors V as Q~ = (I - V V^H) P.
//
// Random numbers: counter-based.  Element e of draw `counter` is Box-Muller on
// SplitMix64 outputs 2m+1 and 2m+2 of the stream started at `seed`, with
// m = counter*2^32 + e.  SplitMix64 is the generator of Steele, Lea & Flood
// (OOPSLA 2014): state advances by 0x9E3779B97F4A7C15 and each state is passed
// through the published 64-bit output mix.
#include "hicu_internal.cuh"

namespace hicu {

__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double jl_gauss(uint64_t seed, uint64_t counter, uint64_t e) {
  const uint64_t gamma = 0x9E3779B97F4A7C15ull;
  const uint64_t k0 = 2ull * ((counter << 32) + e);
  const uint64_t o1 = splitmix_mix(seed + (k0 + 1ull) * gamma);
  const uint64_t o2 = splitmix_mix(seed + (k0 + 2ull) * gamma);
  const double u1 = (double)((o1 >> 11) + 1ull) * 0x1.0p-53;  // (0, 1]
  const double u2 = (double)(o2 >> 11) * 0x1.0p-53;           // [0, 1)
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// P (rows x p, row-major) in float, from the caller's double matrix or drawn here; nsteps
// consecutive draws (counters counter, counter + 1, ...) one after another.
__global__ void jl_make_p_kernel(int rows, int p, int nsteps, const double* __restrict__ Pin, uint64_t seed,
                                 uint64_t counter, float* __restrict__ Pout) {
  const long long per = (long long)rows * p, tot = per * nsteps;
  const double scale = 1.0 / sqrt((double)p);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const long long t = i / per, e = i - t * per;
    const double v = Pin ? Pin[i] : jl_gauss(seed, counter + (uint64_t)t, (uint64_t)e) * scale;
    Pout[i] = (float)v;
  }
}

// complex128 -> complex64
__global__ void to_c64_kernel(const double2* __restrict__ in, float2* __restrict__ out, long long n) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}

// bank[k][a] = sum_j B[j][a] * W[j][k], B complex [m][n], W real [m][p] (nullspace mode)
__global__ void jl_combine_real_kernel(int n, int m, int p, const float2* __restrict__ B,
                                       const float* __restrict__ W, float2* __restrict__ bank) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (a >= n) return;
  float re = 0.f, im = 0.f;
  for (int j = 0; j < m; ++j) {
    const float2 b = B[(long long)j * n + a];
    const float w = __ldg(W + (long long)j * p + k);
    re = fmaf(b.x, w, re);
    im = fmaf(b.y, w, im);
  }
  bank[(long long)k * n + a] = make_float2(re, im);
}

// T[j][k] = sum_a conj(Q[j][a]) P[a][k]   (one warp per (j, k))
__global__ void jl_project_kernel(int n, int m, int p, const float2* __restrict__ Q,
                                  const float* __restrict__ P, float2* __restrict__ T) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m * p) return;
  const int j = warp / p, k = warp % p;
  float re = 0.f, im = 0.f;
  for (int a = lane; a < n; a += 32) {
    const float2 q = Q[(long long)j * n + a];
    const float w = P[(long long)a * p + k];
    re = fmaf(q.x, w, re);
    im = fmaf(-q.y, w, im);
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if (lane == 0) T[(long long)j * p + k] = make_float2(re, im);
}

// bank[k][a] = sum_j Q[j][a] T[j][k] (complex x complex)
__global__ void jl_combine_cplx_kernel(int n, int m, int p, const float2* __restrict__ Q,
                                       const float2* __restrict__ T, float2* __restrict__ bank) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (a >= n) return;
  float re = 0.f, im = 0.f;
  for (int j = 0; j < m; ++j) {
    const float2 q = Q[(long long)j * n + a];
    const float2 t = T[(long long)j * p + k];
    re = fmaf(q.x, t.x, fmaf(-q.y, t.y, re));
    im = fmaf(q.x, t.y, fmaf(q.y, t.x, im));
  }
  bank[(long long)k * n + a] = make_float2(re, im);
}

// bank[k][a] = P[a][k] - sum_j V[j][a] T[j][k]   (complement of the principal vectors V)
__global__ void jl_combine_compl_kernel(int n, int m, int p, const float2* __restrict__ V,
                                        const float2* __restrict__ T, const float* __restrict__ P,
                                        float2* __restrict__ bank) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (a >= n) return;
  float re = 0.f, im = 0.f;
  for (int j = 0; j < m; ++j) {
    const float2 q = V[(long long)j * n + a];
    const float2 t = T[(long long)j * p + k];
    re = fmaf(q.x, t.x, fmaf(-q.y, t.y, re));
    im = fmaf(q.x, t.y, fmaf(q.y, t.x, im));
  }
  bank[(long long)k * n + a] = make_float2(P[(long long)a * p + k] - re, -im);
}

// Complement form in one launch, one CTA per column k of P, the principal vectors V (complex64
// [m][n]) staged in shared memory: T_j = sum_a conj(V[j][a]) P[a][k] (a warp per j), then
// bank[k][a] = P[a][k] - sum_j V[j][a] T_j.  The same sums in the same order as
// jl_project_kernel + jl_combine_compl_kernel.  Dynamic shared memory: m n float2, n float, m float2.
constexpr int JLF_THREADS = 512;

__global__ void __launch_bounds__(JLF_THREADS) jl_compl_fused_kernel(int n, int m, int p, const float2* __restrict__ V,
                                                                     const float* __restrict__ P,
                                                                     float2* __restrict__ bank) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  extern __shared__ __align__(16) float2 jsm[];
  float2* Vs = jsm;                     // [m][n]
  float2* Ts = Vs + (size_t)m * n;      // [m]
  float* Ps = (float*)(Ts + m);         // [n]
  const int k = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    // 16-byte loads, eight in flight per thread (V is a workspace allocation: 256-byte aligned)
    const long long nv = (long long)m * n, n4 = nv / 2;
    const float4* V4 = reinterpret_cast<const float4*>(V);
    float4* Vs4 = reinterpret_cast<float4*>(Vs);
    long long i = tid;
    for (; i + 7 * JLF_THREADS < n4; i += 8 * JLF_THREADS) {
      float4 t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = V4[i + u * JLF_THREADS];
#pragma unroll
      for (int u = 0; u < 8; ++u) Vs4[i + u * JLF_THREADS] = t[u];
    }
    for (; i < n4; i += JLF_THREADS) Vs4[i] = V4[i];
    if ((nv & 1) && tid == 0) Vs[nv - 1] = V[nv - 1];
  }
  for (int a = tid; a < n; a += JLF_THREADS) Ps[a] = P[(long long)a * p + k];
  __syncthreads();
  for (int j = warp; j < m; j += JLF_THREADS / 32) {
    float re = 0.f, im = 0.f;
    for (int a = lane; a < n; a += 32) {
      const float2 q = Vs[(size_t)j * n + a];
      const float w = Ps[a];
      re = fmaf(q.x, w, re);
      im = fmaf(-q.y, w, im);
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) Ts[j] = make_float2(re, im);
  }
  __syncthreads();
  for (int a = tid; a < n; a += JLF_THREADS) {
    float re = 0.f, im = 0.f;
    for (int j = 0; j < m; ++j) {
      const float2 q = Vs[(size_t)j * n + a];
      const float2 t = Ts[j];
      re = fmaf(q.x, t.x, fmaf(-q.y, t.y, re));
      im = fmaf(q.x, t.y, fmaf(q.y, t.x, im));
    }
    bank[(long long)k * n + a] = make_float2(Ps[a] - re, -im);
  }
}

static size_t jl_fused_smem(int64_t n, int64_t m) { return sizeof(float2) * (size_t)(m * n + m) + sizeof(float) * (size_t)n; }

// on the side stream st (launch counted, not event-timed)
hicu_status jl_draw(hicu_handle* h, int64_t rows, int p, int nsteps, uint64_t seed, uint64_t counter, float* P,
                    cudaStream_t st) {
  const long long tot = rows * p * (long long)nsteps;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4 * h->num_sms) blocks = 4 * h->num_sms;
  HICU_LAUNCH_SIDE(h, K_JL, jl_make_p_kernel<<<blocks, 256, 0, st>>>((int)rows, p, nsteps, nullptr, seed, counter, P));
  return cuda_error(h, cudaGetLastError(), "jl draw");
}

namespace {
__global__ void jl_identity_kernel(int rows, float* __restrict__ P) {
  const long long tot = (long long)rows * rows;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x)
    P[i] = (i / rows == i % rows) ? 1.f : 0.f;
}
}  // namespace

namespace {
// bank[k][s n0 + i] += sum_j Q0[j][i] P2[s m0 + j][k]: the Q+ P2 part of [Q | Q+] P for the
// block-diagonal Q+ = blockdiag(Q0, ..., Q0)
__global__ void jl_qplus_add_kernel(int p, int n, int n0, int m0, const float2* __restrict__ Q0,
                                    const float* __restrict__ P2, float2* __restrict__ bank) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  const long long tot = (long long)p * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(idx / n), i = (int)(idx % n);
    const int s = i / n0, li = i % n0;
    float ar = 0.f, ai = 0.f;
    for (int j = 0; j < m0; ++j) {
      const float2 q = Q0[(long long)j * n0 + li];
      const float w = P2[(long long)(s * m0 + j) * p + k];
      ar = fmaf(q.x, w, ar);
      ai = fmaf(q.y, w, ai);
    }
    float2 b = bank[idx];
    b.x += ar;
    b.y += ai;
    bank[idx] = b;
  }
}
}  // namespace

hicu_status launch_jl_qplus(hicu_handle* h, int p, int64_t n, int n0, int m0, const float2* Q0f, const float* P2,
                            float* bank, cudaStream_t st) {
  const long long tot = (long long)p * n;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4 * h->num_sms) blocks = 4 * h->num_sms;
  launch_pdl(h, K_JL, st, dim3(blocks), dim3(256), 0, jl_qplus_add_kernel, true, p, (int)n, n0, m0, Q0f, P2,
             reinterpret_cast<float2*>(bank));
  return cuda_error(h, cudaGetLastError(), "jl qplus");
}

namespace {
// randomized-SVD test vectors Omega [l][n]: rows 0..r0-1 copied from V_prev, row r0 + b, entry a the
// complex Gaussian (z(2e) + i z(2e + 1)) / sqrt(2) of draw `counter`, e = a (l - r0) + b
__global__ void rsvd_omega_kernel(int n, int l, int r0, const double2* __restrict__ Vp, uint64_t seed,
                                  uint64_t counter, double2* __restrict__ Om) {
  const long long tot = (long long)l * n;
  const double s = 0.70710678118654752440;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(t / n), a = (int)(t % n);
    if (row < r0) {
      Om[t] = Vp[t];
    } else {
      const uint64_t e = (uint64_t)a * (uint64_t)(l - r0) + (uint64_t)(row - r0);
      Om[t] = make_double2(jl_gauss(seed, counter, 2ull * e) * s, jl_gauss(seed, counter, 2ull * e + 1ull) * s);
    }
  }
}
}  // namespace

hicu_status launch_rsvd_omega(hicu_handle* h, int64_t n, int64_t l, int64_t r0, const double* V_prev, uint64_t seed,
                              uint64_t counter, double2* Om, cudaStream_t st) {
  const long long tot = l * n;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 8 * h->num_sms) blocks = 8 * h->num_sms;
  HICU_LAUNCH(h, K_EIG, st, rsvd_omega_kernel<<<blocks, 256, 0, st>>>((int)n, (int)l, (int)r0,
                                                                      (const double2*)V_prev, seed, counter, Om));
  return cuda_error(h, cudaGetLastError(), "rsvd omega");
}

hicu_status jl_identity(hicu_handle* h, int64_t rows, float* P, cudaStream_t st) {
  const long long tot = rows * rows;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4 * h->num_sms) blocks = 4 * h->num_sms;
  HICU_LAUNCH(h, K_JL, st, jl_identity_kernel<<<blocks, 256, 0, st>>>((int)rows, P));
  return cuda_error(h, cudaGetLastError(), "jl identity");
}

hicu_status jl_convert_q(hicu_handle* h, int64_t n, int64_t nr, const double* Q, float2** Qf, cudaStream_t st) {
  hicu_status s = HICU_OK;
  *Qf = (float2*)ws_get(h, WS_QF, sizeof(float2) * nr * n, &s);
  if (s) return s;
  const long long tot = nr * n;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 2048) blocks = 2048;
  launch_pdl(h, K_JL, st, dim3(blocks), dim3(256), 0, to_c64_kernel, true, (const double2*)Q, *Qf, tot);
  return cuda_error(h, cudaGetLastError(), "jl convert");
}

hicu_status launch_jl_converted(hicu_handle* h, int64_t n, int64_t nr, int p, const float2* Qf, int mode,
                                const double* P, const float* Pdrawn, uint64_t seed, uint64_t counter,
                                float* bank, cudaStream_t st, bool pdl) {
  hicu_status s = HICU_OK;
  const int rows = (mode == HICU_JL_NULLSPACE) ? (int)nr : (int)n;
  const float* Pf = Pdrawn;
  if (!Pf) {
    float* Pw = (float*)ws_get(h, WS_P, sizeof(float) * rows * p, &s);
    if (s) return s;
    const long long tot = (long long)rows * p;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    HICU_LAUNCH(h, K_JL, st, jl_make_p_kernel<<<blocks, 256, 0, st>>>(rows, p, 1, P, seed, counter, Pw));
    Pf = Pw;
  }
  if (mode == HICU_JL_COMPLEMENT && nr > 0 && jl_fused_smem(n, nr) <= 200 * 1024) {
    const cudaError_t e0 = allow_max_dynamic_smem((const void*)jl_compl_fused_kernel);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "jl smem");
    launch_pdl(h, K_JL, st, dim3(p), dim3(JLF_THREADS), jl_fused_smem(n, nr), jl_compl_fused_kernel, pdl, (int)n,
               (int)nr, p, (const float2*)Qf, (const float*)Pf, (float2*)bank);
    return cuda_error(h, cudaGetLastError(), "jl_compress");
  }
  dim3 grid((unsigned)((n + 127) / 128), (unsigned)p);
  if (mode == HICU_JL_NULLSPACE) {
    HICU_LAUNCH(h, K_JL, st, jl_combine_real_kernel<<<grid, 128, 0, st>>>((int)n, (int)nr, p, Qf, Pf, (float2*)bank));
  } else {
    float2* T = (float2*)ws_get(h, WS_T, sizeof(float2) * nr * p, &s);
    if (s) return s;
    const long long warps = nr * p;
    HICU_LAUNCH(h, K_JL, st,
                jl_project_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>((int)n, (int)nr, p,
                                                                                        Qf, Pf, T));
    if (mode == HICU_JL_PROJECTOR)
      HICU_LAUNCH(h, K_JL, st,
                  jl_combine_cplx_kernel<<<grid, 128, 0, st>>>((int)n, (int)nr, p, Qf, T, (float2*)bank));
    else
      HICU_LAUNCH(h, K_JL, st,
                  jl_combine_compl_kernel<<<grid, 128, 0, st>>>((int)n, (int)nr, p, Qf, T, Pf, (float2*)bank));
  }
  return cuda_error(h, cudaGetLastError(), "jl_compress");
}

hicu_status launch_jl(hicu_handle* h, int64_t n, int64_t nr, int p, const double* Q, int mode,
                      const double* P, uint64_t seed, uint64_t counter, float* bank,
                      cudaStream_t st) {
  float2* Qf = nullptr;
  hicu_status s = jl_convert_q(h, n, nr, Q, &Qf, st);
  if (s) return s;
  return launch_jl_converted(h, n, nr, p, Qf, mode, P, nullptr, seed, counter, bank, st);
}

}  // namespace hicu
