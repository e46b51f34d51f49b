// Cyclic Jacobi inside one thread-block cluster (null-space step, Algorithm 1
// steps 2-3 in Gram form) for n <= 256: the same rotations, ordering and stopping
// rules as the grid-wide solver in eig.cu, on a different memory and arithmetic
// plan.
//
// A round of the grid-wide solver pays a grid barrier (~2 us) and L2 round trips,
// and its FP64 arithmetic runs at 1/58 of the FP32 rate.  Here the two ping-pong
// copies of A and the eigenvector matrix V live in the shared memory of the 16 CTAs
// of one cluster (row i in CTA i / rows; other CTAs' rows are reached through
// distributed shared memory), a round ends at the hardware cluster barrier, and
// the arithmetic is double-float: each real number is an unevaluated sum hi + lo
// of two FP32 numbers, added with Knuth's two-sum and multiplied with an FMA-based
// two-product (Dekker; the double-float formulas of Hida, Li and Bailey's QD
// library), which keeps ~2^-48 relative precision on the FP32 pipes.  Entries are
// pre-scaled by an exact power of two so that the largest is O(1).
//
// Round t: every CTA computes all n/2 rotations of the round (FP32 angle, made
// unitary to double-float precision by two Newton steps) from the current A, then
// one thread per upper pair-block (P <= Q) writes W_P^H A_PQ W_Q into the other A
// copy, together with its Hermitian mirror, and each CTA updates its own rows of
// V <- V W.  Convergence is tested after every sweep on all off-diagonal mass or on
// the coupling between the r largest diagonal entries and the rest.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "df.cuh"
#include "hicu_internal.cuh"

namespace cg = cooperative_groups;

namespace hicu {

constexpr int CL_THREADS = 512;
constexpr int CL_MAX_N = 256;
constexpr int CL_MAX_NP = CL_MAX_N / 2;
constexpr size_t CL_MAX_SMEM = 200 * 1024;

__device__ __forceinline__ cdf c_mul_e(cdf a, dfl ex, dfl ey) {  // a * e
  return {df_add(df_mul(a.re, ex), df_neg(df_mul(a.im, ey))), df_add(df_mul(a.re, ey), df_mul(a.im, ex))};
}
__device__ __forceinline__ cdf c_mul_ce(cdf a, dfl ex, dfl ey) {  // conj(e) * a
  return {df_add(df_mul(a.re, ex), df_mul(a.im, ey)), df_add(df_mul(a.im, ex), df_neg(df_mul(a.re, ey)))};
}
__device__ __forceinline__ cdf c_lin(dfl s, cdf a, dfl t, cdf b) {  // s a + t b, s and t real
  return {df_add(df_mul(s, a.re), df_mul(t, b.re)), df_add(df_mul(s, a.im), df_mul(t, b.im))};
}

// W = [[cs, sn], [-sn e, cs e]], e = ex + i ey (the convention of eig.cu)
struct RotDF {
  dfl cs, sn, ex, ey;
  int ident;
};

// 1 / sqrt(q) for q = 1 + O(1e-7): two Newton steps f <- f (3 - q f^2) / 2 from f = 1
__device__ __forceinline__ dfl df_rsqrt_near1(dfl q) {
  const dfl half = {0.5f, 0.f}, three_half = {1.5f, 0.f};
  dfl f = df_add(three_half, df_neg(df_mul(half, q)));
  f = df_mul(f, df_add(three_half, df_neg(df_mul(half, df_mul(q, df_mul(f, f))))));
  return f;
}

__device__ RotDF make_rot_df(dfl a, dfl c, cdf b) {
  RotDF R;
  const float bx = b.re.hi, by = b.im.hi;
  const float ab = hypotf(bx, by);
  const float thr = 1e-17f * sqrtf(fabsf(a.hi)) * sqrtf(fabsf(c.hi));
  if (!(ab > thr) || !(ab > 0.f)) {
    R.cs = {1.f, 0.f};
    R.sn = {0.f, 0.f};
    R.ex = {1.f, 0.f};
    R.ey = {0.f, 0.f};
    R.ident = 1;
    return R;
  }
  const float tau = df_add(c, df_neg(a)).hi / (2.f * ab);
  float t;
  if (fabsf(tau) > 1e18f) t = 0.5f / tau;
  else t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
  const float cs = rsqrtf(1.f + t * t);
  const dfl c0 = {cs, 0.f}, s0 = {t * cs, 0.f};
  dfl f = df_rsqrt_near1(df_add(df_mul(c0, c0), df_mul(s0, s0)));
  R.cs = df_mul(c0, f);
  R.sn = df_mul(s0, f);
  const dfl e0 = {bx / ab, 0.f}, e1 = {-by / ab, 0.f};
  f = df_rsqrt_near1(df_add(df_mul(e0, e0), df_mul(e1, e1)));
  R.ex = df_mul(e0, f);
  R.ey = df_mul(e1, f);
  R.ident = 0;
  return R;
}

// circle method: player 0 fixed, players 1..n-1 rotate by t each round
__device__ __forceinline__ void pair_cl(int n, int t, int i, int& p, int& q) {
  const int m = n - 1;
  int a = 0;
  if (i != 0) {
    a = i - 1 + t;
    a = a >= m ? a - m : a;
    a += 1;
  }
  int b = (n - 1 - i) - 1 + t;
  b = b >= m ? b - m : b;
  b += 1;
  p = a < b ? a : b;
  q = a < b ? b : a;
}

struct ClArgs {
  int n;      // padded size, a multiple of 2 x cluster size
  int nreal;  // n without the zero pad
  int r;
  int rows;   // rows per CTA
  const double2* A0;  // n x n FP64 start matrix
  const double2* V0;  // n x n FP64 start basis
  double2* Vout;      // n x n FP64 eigenvectors (columns); may alias V0
  double* diag;       // n FP64 diagonal at exit
  int* info;          // [0] sweeps, [1] converged, [3] mode
  unsigned long long* sweep_total;
  int max_sweeps;
  int mode;           // 0: all off-diagonal mass; 1: top-r / rest coupling
  double tol2;
};

__device__ __forceinline__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < CL_THREADS / 32; ++w) s += red[w];
  return s;
}

__device__ __forceinline__ double cta_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < CL_THREADS / 32; ++w) s = fmax(s, red[w]);
  return s;
}

__global__ void __launch_bounds__(CL_THREADS, 1) jacobi_cluster_kernel(ClArgs J) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int nct = (int)cluster.num_blocks();
  extern __shared__ float4 smem4[];
  // rotations and their index pairs, double-buffered by round parity: the V update of a round
  // runs during the next round's rotation phase
  __shared__ RotDF rot[2][CL_MAX_NP];
  __shared__ short pp[2][CL_MAX_NP], qq[2][CL_MAX_NP];
  __shared__ double dg[CL_MAX_N];
  __shared__ unsigned char top[CL_MAX_N];
  __shared__ double part[2];
  __shared__ double red[CL_THREADS / 32];
  const int n = J.n, np = n / 2, R = J.rows, tid = threadIdx.x;
  float4* Abuf0 = smem4;
  float4* Abuf1 = smem4 + (size_t)R * n;
  float4* Vloc = smem4 + 2 * (size_t)R * n;
  const int row0 = crank * R;

  // exact power-of-two scale that brings the largest entry of A near 1
  double amax = 0.0;
  for (int e = tid; e < R * n; e += CL_THREADS) {
    const double2 a = J.A0[(size_t)row0 * n + e];
    amax = fmax(amax, fmax(fabs(a.x), fabs(a.y)));
  }
  amax = cta_max(amax, red);
  if (tid == 0) part[0] = amax;
  cluster.sync();
  amax = 0.0;
  for (int c = 0; c < nct; ++c) amax = fmax(amax, cluster.map_shared_rank(part, c)[0]);
  int ex2 = 0;
  if (amax > 0.0 && amax <= 1.7e308) frexp(amax, &ex2);
  const double scale = ldexp(1.0, -ex2);

  for (int e = tid; e < R * n; e += CL_THREADS) {
    const double2 a = J.A0[(size_t)row0 * n + e];
    const dfl ar = df_from(a.x * scale), ai = df_from(a.y * scale);
    Abuf0[e] = make_float4(ar.hi, ar.lo, ai.hi, ai.lo);
    const double2 v = J.V0[(size_t)row0 * n + e];
    const dfl vr = df_from(v.x), vi = df_from(v.y);
    Vloc[e] = make_float4(vr.hi, vr.lo, vi.hi, vi.lo);
  }
  cluster.sync();  // every CTA has read `part` and holds its rows

  const int nblk = np * (np + 1) / 2;

  // V <- V W of round buffer `rb` on this CTA's rows, items k0, k0 + stride, ...
  auto v_update = [&](int rb, int k0, int stride) {
    for (int k = k0; k < R * np; k += stride) {
      const int rr = k / np, Q = k - (k / np) * np;
      if (rot[rb][Q].ident) continue;
      const RotDF wq = rot[rb][Q];
      float4* vp = Vloc + (size_t)rr * n + pp[rb][Q];
      float4* vq = Vloc + (size_t)rr * n + qq[rb][Q];
      const cdf v0 = ld4(vp), v1 = ld4(vq);
      const cdf u = c_mul_e(v1, wq.ex, wq.ey);
      st4(vp, c_lin(wq.cs, v0, df_neg(wq.sn), u));
      st4(vq, c_lin(wq.sn, v0, wq.cs, u));
    }
  };

  int cur = 0, sweeps = J.max_sweeps, converged = 0;
  int g = 0;      // rounds done (its parity selects the per-round buffers)
  int pend = -1;  // buffer of the round whose V update is still to be applied
  for (int sweep = 0; sweep < J.max_sweeps; ++sweep) {
    for (int t = 0; t < n - 1; ++t) {
      float4* Ac = cur ? Abuf1 : Abuf0;
      float4* An = cur ? Abuf0 : Abuf1;
      const int cb = g & 1;
      // phase 1: this round's rotations (threads < n/2), while the other threads apply the
      // previous round's rotations to V
      if (tid < np) {
        int p, q;
        pair_cl(n, t, tid, p, q);
        const float4* rp_ = cluster.map_shared_rank(Ac, p / R) + (size_t)(p % R) * n;
        const float4* rq_ = cluster.map_shared_rank(Ac, q / R) + (size_t)(q % R) * n;
        const cdf app = ld4(rp_ + p), apq = ld4(rp_ + q), aqq = ld4(rq_ + q);
        rot[cb][tid] = make_rot_df(app.re, aqq.re, apq);
        pp[cb][tid] = (short)p;
        qq[cb][tid] = (short)q;
      } else if (pend >= 0) {
        v_update(pend, tid - np, CL_THREADS - np);
      }
      __syncthreads();
      // phase 2: one thread per upper pair-block; blocks interleaved over the CTAs
      for (int b = tid * nct + crank; b < nblk; b += CL_THREADS * nct) {
        int Q = (int)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);
        while (Q * (Q + 1) / 2 > b) --Q;
        while ((Q + 1) * (Q + 2) / 2 <= b) ++Q;
        const int P = b - Q * (Q + 1) / 2;
        const int p1 = pp[cb][P], q1 = qq[cb][P], p2 = pp[cb][Q], q2 = qq[cb][Q];
        const float4* rp1 = cluster.map_shared_rank(Ac, p1 / R) + (size_t)(p1 % R) * n;
        const float4* rq1 = cluster.map_shared_rank(Ac, q1 / R) + (size_t)(q1 % R) * n;
        cdf b00 = ld4(rp1 + p2), b01 = ld4(rp1 + q2), b10 = ld4(rq1 + p2), b11 = ld4(rq1 + q2);
        const RotDF wp = rot[cb][P], wq = rot[cb][Q];
        if (!wq.ident) {  // M = A_blk W_Q
          const cdf u0 = c_mul_e(b01, wq.ex, wq.ey), u1 = c_mul_e(b11, wq.ex, wq.ey);
          const cdf m00 = c_lin(wq.cs, b00, df_neg(wq.sn), u0);
          const cdf m10 = c_lin(wq.cs, b10, df_neg(wq.sn), u1);
          b01 = c_lin(wq.sn, b00, wq.cs, u0);
          b11 = c_lin(wq.sn, b10, wq.cs, u1);
          b00 = m00;
          b10 = m10;
        }
        if (!wp.ident) {  // B = W_P^H M
          const cdf v0 = c_mul_ce(b10, wp.ex, wp.ey), v1 = c_mul_ce(b11, wp.ex, wp.ey);
          const cdf n00 = c_lin(wp.cs, b00, df_neg(wp.sn), v0);
          const cdf n01 = c_lin(wp.cs, b01, df_neg(wp.sn), v1);
          b10 = c_lin(wp.sn, b00, wp.cs, v0);
          b11 = c_lin(wp.sn, b01, wp.cs, v1);
          b00 = n00;
          b01 = n01;
        }
        float4* wp1 = cluster.map_shared_rank(An, p1 / R) + (size_t)(p1 % R) * n;
        float4* wq1 = cluster.map_shared_rank(An, q1 / R) + (size_t)(q1 % R) * n;
        if (P == Q) {  // diagonal entries of a Hermitian matrix are real
          b00.im = {0.f, 0.f};
          b11.im = {0.f, 0.f};
        } else {
          float4* wp2 = cluster.map_shared_rank(An, p2 / R) + (size_t)(p2 % R) * n;
          float4* wq2 = cluster.map_shared_rank(An, q2 / R) + (size_t)(q2 % R) * n;
          st4(wp2 + p1, c_conj(b00));
          st4(wp2 + q1, c_conj(b10));
          st4(wq2 + p1, c_conj(b01));
          st4(wq2 + q1, c_conj(b11));
        }
        st4(wp1 + p2, b00);
        st4(wp1 + q2, b01);
        st4(wq1 + p2, b10);
        st4(wq1 + q2, b11);
      }
      pend = cb;
      ++g;
      cluster.sync();
      cur ^= 1;
    }
    // convergence test on the current copy
    const float4* Ac = cur ? Abuf1 : Abuf0;
    if (J.mode == 1) {
      for (int i = tid; i < J.nreal; i += CL_THREADS)
        dg[i] = df_to(ld4(cluster.map_shared_rank(Ac, i / R) + (size_t)(i % R) * n + i).re);
      __syncthreads();
      for (int i = tid; i < J.nreal; i += CL_THREADS) {
        const double di = dg[i];
        int rk = 0;
        for (int j = 0; j < J.nreal; ++j) rk += (dg[j] > di) || (dg[j] == di && j < i);
        top[i] = rk < J.r ? 1 : 0;
      }
      __syncthreads();
    }
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < R * n; e += CL_THREADS) {
      const int rr = e / n, col = e - rr * n, i = row0 + rr;
      const cdf a = ld4(Ac + e);
      const double re = df_to(a.re), im = df_to(a.im);
      const double m2 = re * re + im * im;
      tot += m2;
      if (J.mode == 0) {
        if (i != col) off += m2;
      } else if (i < J.nreal && col < J.nreal && top[i] != top[col]) {
        off += m2;
      }
    }
    off = cta_sum(off, red);
    tot = cta_sum(tot, red);
    if (tid == 0) {
      part[0] = off;
      part[1] = tot;
    }
    cluster.sync();
    double o = 0.0, d = 0.0;
    for (int c = 0; c < nct; ++c) {
      const double* rp_ = cluster.map_shared_rank(part, c);
      o += rp_[0];
      d += rp_[1];
    }
    // every CTA reaches the same decision from the same partials; `part` is rewritten only
    // after the next sweep's cluster barriers, which all readers pass first
    if (o <= J.tol2 * d || !(o == o)) {
      sweeps = sweep + 1;
      converged = (o == o) ? 1 : 0;
      break;
    }
  }
  if (pend >= 0) v_update(pend, tid, CL_THREADS);  // the last round's rotations
  __syncthreads();
  const float4* Ac = cur ? Abuf1 : Abuf0;
  for (int e = tid; e < R * n; e += CL_THREADS) {
    const cdf v = ld4(Vloc + e);
    J.Vout[(size_t)row0 * n + e] = make_double2(df_to(v.re), df_to(v.im));
  }
  for (int rr = tid; rr < R; rr += CL_THREADS) {
    const int i = row0 + rr;
    J.diag[i] = df_to(ld4(Ac + (size_t)rr * n + i).re) / scale;
  }
  if (crank == 0 && tid == 0) {
    J.info[0] = sweeps;
    J.info[1] = converged;
    J.info[3] = J.mode;
    atomicAdd(J.sweep_total, (unsigned long long)sweeps);
  }
  cluster.sync();  // no CTA exits while another may still read its shared memory
}

// rank of each eigenvalue (ascending, ties by index) and the eigenvalue output
__global__ void cl_rank_kernel(int n, const double* __restrict__ diag, int* __restrict__ rank,
                               double* __restrict__ eig_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double li = diag[i];
  int r = 0;
  for (int j = 0; j < n; ++j) {
    const double lj = diag[j];
    r += (lj < li) || (lj == li && j < i);
  }
  rank[i] = r;
  if (eig_out) eig_out[r] = li;
}

static size_t cluster_smem(int npad, int nct) { return sizeof(float4) * 3 * (size_t)(npad / nct) * npad; }

static cudaLaunchConfig_t cluster_cfg(int nct, size_t smem, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nct;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(nct);
  cfg.blockDim = dim3(CL_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

int cluster_eig_npad(int64_t n, int nct) { return (int)((n + 2 * nct - 1) / (2 * nct) * (2 * nct)); }

int cluster_eig_ctas(int64_t n) {
  if (n < 2 || n > CL_MAX_N) return 0;
  // per n: 0 unknown, -1 unavailable, else the cluster size (host threads of a batch share it)
  static std::atomic<int> cached[CL_MAX_N + 1];
  static std::mutex mu;
  const int known = cached[n].load();
  if (known) return known > 0 ? known : 0;
  std::lock_guard<std::mutex> lock(mu);
  int found = -1;
  for (int nct : {16, 8}) {
    const int npad = cluster_eig_npad(n, nct);
    if (npad > CL_MAX_N) continue;
    const size_t smem = cluster_smem(npad, nct);
    if (smem > CL_MAX_SMEM) continue;
    if (nct > 8 && cudaFuncSetAttribute(jacobi_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                        1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (allow_max_dynamic_smem((const void*)jacobi_cluster_kernel) != cudaSuccess) continue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_cfg(nct, smem, 0, attr);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, jacobi_cluster_kernel, &cfg) == cudaSuccess && clusters >= 1) {
      found = nct;
      break;
    }
    cudaGetLastError();
  }
  cached[n].store(found);
  return found > 0 ? found : 0;
}

// Cluster Jacobi on A0 (npad x npad, zero-padded, already V0^H G V0 for a warm start) from
// the basis V0; writes the eigenvectors to Vout (may alias V0), eigvals and Q as run_nullspace.
hicu_status run_nullspace_cluster(hicu_handle* h, int n, int npad, int nct, int64_t r, const double2* A0,
                                  const double2* V0, double2* Vout, double* Q, double* eigvals, int flags,
                                  cudaStream_t st) {
  hicu_status s = HICU_OK;
  double* diag = (double*)ws_get(h, WS_EIG_PART, sizeof(double) * npad + 64, &s);
  if (s) return s;
  int* info = (int*)(diag + npad);
  int* rank = (int*)ws_get(h, WS_EIG_TMP, sizeof(int) * npad, &s);
  if (s) return s;
  cudaMemsetAsync(info, 0, 8 * sizeof(int), st);
  ClArgs J;
  J.n = npad;
  J.nreal = n;
  J.r = (int)r;
  J.rows = npad / nct;
  J.A0 = A0;
  J.V0 = V0;
  J.Vout = Vout;
  J.diag = diag;
  J.info = info;
  J.sweep_total = reinterpret_cast<unsigned long long*>(h->dev_err + 8);
  J.max_sweeps = 40;
  J.mode = (flags & 2) ? 1 : 0;
  J.tol2 = (flags & 2) ? 1e-16 : 1e-22;
  cudaLaunchAttribute attr[1];
  const size_t smem = cluster_smem(npad, nct);
  cudaError_t e = allow_max_dynamic_smem((const void*)jacobi_cluster_kernel);
  if (e != cudaSuccess) return cuda_error(h, e, "nullspace cluster smem");
  cudaLaunchConfig_t cfg = cluster_cfg(nct, smem, st, attr);
  HICU_LAUNCH(h, K_EIG, st, e = cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel, J));
  if (e != cudaSuccess) return cuda_error(h, e, "nullspace cluster launch");
  HICU_LAUNCH(h, K_MISC, st, cl_rank_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, diag, rank, eigvals));
  const long long nn = (long long)n * n;
  const int blocks = (int)std::min<long long>((nn + 255) / 256, 4096);
  HICU_LAUNCH(h, K_MISC, st,
              eig_gather_q_kernel<<<blocks, 256, 0, st>>>(n, npad, n - (int)r, Vout, rank, (double2*)Q));
  s = cuda_error(h, cudaGetLastError(), "nullspace cluster output");
  if (s) return s;
  h->eig_info = info;
  return HICU_OK;
}

}  // namespace hicu
