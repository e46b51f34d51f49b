// Principal subspace of the Gram matrix by Householder tridiagonalisation (Algorithm 1
// steps 2-3 in Gram form: V = the r principal right singular vectors of H, i.e. the
// eigenvectors of G = H^H H for its r largest eigenvalues; the null space is their
// orthogonal complement).
//
// Method (Golub & Van Loan, 4th ed., sections 8.3.1, 8.4.1 and 8.4.2):
//  1. G = Q_H T Q_H^H with T real symmetric tridiagonal: n - 1 Householder steps
//     H_k = I - tau_k v_k v_k^H, each making the part of column k below the
//     subdiagonal vanish with a real subdiagonal entry.  Every CTA forms v_k itself from its
//     copy of the pivot row k (G is Hermitian and kept in full), w = tau A v on its own rows,
//     one barrier, then the symmetric rank-2 update A <- A - v w^H - w v^H (w corrected by
//     -tau/2 (w^H v) v) of its own rows and, in every CTA, of the next pivot row.  n <= 416:
//     one 16-CTA cluster with the rows in shared memory (hardware cluster barrier); larger n:
//     a cooperative grid over all SMs (grid barrier on an arrival counter).
//  2. Eigenvalues of T by multisection on Sturm counts (the LDL^T pivot recurrence,
//     Kahan's form, which is backward stable): a CTA of 256 threads per eigenvalue, 256
//     points a round, two FP32 rounds then four double-float rounds.
//  3. Eigenvectors of T for the r largest eigenvalues by inverse iteration with a
//     pivoted tridiagonal LU; eigenvalues closer than 1e-10 ||T|| are solved one after
//     the other and orthogonalised against each other (modified Gram-Schmidt).
//  4. V = Q_H Z: the reflectors applied to each eigenvector in compact WY blocks of 32
//     (I - Y T Y^H per block, Schreiber & Van Loan), last block first; the WY factors are
//     built on a side stream during steps 2-3.
// Arithmetic: double-float (df.cuh, ~2^-48), because FP64 on this GPU is both slow and of
// long latency, and every stage here is a chain of dependent operations.  The input is
// pre-scaled by an exact power of two (largest entry O(1)); inputs and outputs are FP64.
// Accuracy: eigenvalues to ~1e-14 ||G|| (absolute), span(V) to ~1e-14 ||G|| / gap (the
// Davis-Kahan bound of a backward-stable method at this precision).
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "df.cuh"
#include "hicu_internal.cuh"

namespace cg = cooperative_groups;

namespace hicu {

constexpr int TD_THREADS = 512;

struct TdArgs {
  int n;
  float4* A;      // n x n row-major complex double-float (scaled G); rows updated in place when not
                  // held in shared memory
  float2* d;      // n   diagonal of T
  float2* e;      // n-1 subdiagonal of T
  float4* refl;   // n x n: row k holds v_k (v_k[0] = 1, length n-k-1)
  float4* tau;    // n-1
  float4* w;      // 2 n scratch (w0 = tau A v), by step parity
  float4* part;   // 2 gridDim.x partial sums w0^H v, by step parity
  float4* prow;   // 2 n: the next pivot row as stored, published by its owner, by step parity
  GridSync gs;
};

__device__ __forceinline__ float2 dpack(dfl a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ dfl dload(float2 a) { return {a.x, a.y}; }

// Householder scalars of the pivot row x (length m + 1; squares of x in xsq): tau, the inverse
// 1 / (x0 - beta) of v's leading entry before normalisation, beta; one warp.
__device__ __forceinline__ void td_scalars(int m, const float4* x, const float2* xsq, cdf& tau, cdf& scale,
                                            dfl& beta) {
  const int lane = threadIdx.x & 31;
  dfl t2 = df_f(0.f);
  for (int j = 2 + lane; j <= m; j += 32) t2 = df_add(t2, dload(xsq[j]));
  const dfl xn2 = df_warp_sum(t2);
  const cdf x0 = c_conj(ld4(&x[1]));
  tau = c_zero();
  scale = c_zero();
  beta = x0.re;
  if (!(xn2.hi == 0.f && x0.im.hi == 0.f)) {
    const dfl nrm = df_sqrt(df_add(df_add(df_mul(x0.re, x0.re), df_mul(x0.im, x0.im)), xn2));
    beta = x0.re.hi >= 0.f ? df_neg(nrm) : nrm;
    const dfl rb = df_rcp(beta);
    tau.re = df_sub(df_f(1.f), df_mul(x0.re, rb));  // (beta - x0.re) / beta
    tau.im = df_neg(df_mul(x0.im, rb));
    const cdf den = {df_sub(x0.re, beta), x0.im};
    const dfl dd = df_add(df_mul(den.re, den.re), df_mul(den.im, den.im));
    const dfl rd = df_rcp(dd);
    scale.re = df_mul(den.re, rd);
    scale.im = df_neg(df_mul(den.im, rd));
  }
}

// Grid barrier on a monotonic arrival counter: every CTA adds one (fire-and-forget, after a fence)
// and polls until the count reaches (epoch + 1) * G, one L2 round trip after the last arrival.
// Bounded like grid_sync: gives up after gs.timeout_ns (or another CTA's error), records
// HICU_ERR_TIMEOUT and returns false in every thread of the CTA.  gs.count starts at zero.
__device__ inline bool grid_sync_count(const GridSync& gs, unsigned& epoch) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = (epoch + 1u) * gs.nblocks;
    // arrival with release semantics at GPU scope (cumulative over the CTA's writes, which the
    // __syncthreads above made visible to this thread): one reduction, no separate fence
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gs.count) : "memory");
    unsigned long long t0 = 0;
    for (unsigned it = 0; ld_acquire_u32(gs.count) < target; ++it) {
      if ((it & 255u) == 255u) {
        const unsigned long long t = global_ns();
        if (t0 == 0) t0 = t;
        if (t - t0 > gs.timeout_ns || *((volatile int*)gs.err) != 0) {
          atomicExch(gs.err, (int)HICU_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  ++epoch;
  return s_ok != 0;
}

// One grid barrier per reflector.  Global row g is owned by CTA g mod G for the whole run and,
// with ROWS_IN_SMEM, held in that CTA's shared memory (local row g / G); it is updated in place by
// its owner only, except row k+1, the next pivot row: nobody writes it during step k, its owner
// publishes the stored values before the barrier, and every CTA forms its updated values from
// them and v, w, so the next Householder vector needs no second barrier.  w0, the partial sums
// and the published row alternate between two buffers: a CTA can start step k+1 while others
// still read step k's, but cannot reach step k+2 before every CTA has passed step k+1's barrier.
// Per step k (as in the one-cluster form below):
//   1. row sums s_i = sum_{j>=1} A_ij conj(x_{1+j}) of the own rows; w0_i = tau (A_i0 +
//      s_i / (x0 - beta)) to global memory and conj(w0_i) v_i to shared memory.  CTA barrier.
//   2. v; warp 0: the CTA's partial sum of conj(w0) v to global memory.  Grid barrier.
//   3. w0 and the published row prefetched, the G partial sums (every warp) -> alpha;
//      w = w0 + alpha v and the next pivot row x' = (stored row k+1) - conj(w) - w_0 conj(v)
//      with the squares of its entries.  CTA barrier.
//   4. warps 0..nw-2: rank-2 update of the own rows but row k+1; warp nw-1 meanwhile: the
//      Householder scalars of step k+1 from x'.  CTA barrier.
constexpr int TD_PF = 4;   // entries per thread prefetched after the barrier
constexpr int TD_SEG = 4;  // at most this many warps (segments) per row in the update

template <bool ROWS_IN_SMEM>
__global__ void __launch_bounds__(TD_THREADS) tridiag_kernel(const TdArgs a) {
  extern __shared__ float4 tsm[];
  const int n = a.n;
  const int G = gridDim.x, c = blockIdx.x;
  const int R = (n + G - 1) / G;  // rows per CTA
  float4* x = tsm;             // [n] current pivot row k: x[j] = A[k][k + j]
  float4* v = x + n;           // [n]
  float4* w = v + n;           // [n]
  float4* segp = w + n;        // [R][TD_SEG] partial row sums of the own rows (by local row, segment)
  float4* rows = segp + TD_SEG * R;  // [R][n] own rows (ROWS_IN_SMEM)
  float2* xsq = (float2*)(rows + (ROWS_IN_SMEM ? (size_t)R * n : 0));  // [n] squares of x
  __shared__ float4 hs[3];     // tau, 1 / (x0 - beta), beta of the current step
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = TD_THREADS / 32;
  auto row_of = [&](int g) -> float4* {
    return ROWS_IN_SMEM ? rows + (size_t)(g / G) * n : a.A + (size_t)g * n;
  };
  unsigned epoch = 0;
  if (ROWS_IN_SMEM)
    for (int idx = tid; idx < R * n; idx += TD_THREADS) {
      const int lr = idx / n, g = lr * G + c;
      if (g < n) rows[idx] = a.A[(size_t)g * n + (idx - lr * n)];
    }
  for (int j = tid; j < n; j += TD_THREADS) {
    const float4 xj = a.A[j];
    x[j] = xj;
    xsq[j] = dpack(df_add(df_mul({xj.x, xj.y}, {xj.x, xj.y}), df_mul({xj.z, xj.w}, {xj.z, xj.w})));
  }
  __syncthreads();
  if (warp == nw - 1) {
    cdf tau, scale;
    dfl beta;
    td_scalars(n - 1, x, xsq, tau, scale, beta);
    if (lane == 0) {
      st4(&hs[0], tau);
      st4(&hs[1], scale);
      hs[2] = make_float4(beta.hi, beta.lo, 0.f, 0.f);
    }
  }
  __syncthreads();
  // row sums of step 0 (later steps' sums are formed with the rank-2 update, phase 4)
  int S_prev = 1;
  {
    const int g0 = c >= 1 ? c : G;                          // the first own row with g >= 1
    const int nown0 = g0 <= n - 1 ? (n - 1 - g0) / G + 1 : 0;
    for (int q = warp; q < nown0; q += nw) {
      const int g = g0 + q * G;
      const float4* row = row_of(g) + 1;
      cdf y = c_zero();
      for (int j = 1 + lane; j < n - 1; j += 32) c_acc_mul(y, ld4(&row[j]), c_conj(ld4(&x[1 + j])));
      y = c_warp_sum(y);
      if (lane == 0) st4(&segp[(g / G) * TD_SEG], y);
    }
  }
  __syncthreads();
  for (int k = 0; k < n - 1; ++k) {
    const int m = n - k - 1;
    const int par = k & 1;
    const cdf tau = ld4(&hs[0]), scale = ld4(&hs[1]);
    const bool active = !(tau.re.hi == 0.f && tau.im.hi == 0.f);
    if (c == 0 && tid == 0) {
      a.d[k] = dpack(ld4(&x[0]).re);
      a.e[k] = dpack({hs[2].x, hs[2].y});
      st4(&a.tau[k], tau);
    }
    // --- the owner of row k+1 publishes it (stored values, columns k+1 ..)
    float4* pub = a.prow + par * n;
    if ((k + 1) % G == c) {
      const float4* src = row_of(k + 1) + (k + 1);
      for (int j = tid; j < m; j += TD_THREADS) pub[j] = src[j];
    }
    float4* wg = a.w + par * n;
    float4* pg = a.part + par * G;
    const int i0 = ((c - (k + 1)) % G + G) % G;  // first relative row owned by this CTA
    const int nown = i0 < m ? (m - 1 - i0) / G + 1 : 0;
    const int lrow0 = (k + 1 + i0) / G;           // its local row index
    // --- 1-2. warp 0: w0_i = tau (A_i0 + s_i / (x0 - beta)) of the own rows from their row sums
    // s_i (formed with the previous step's update) to global memory, and the CTA's partial sum of
    // conj(w0_i) v_i (v itself is formed after the barrier, under its loads)
    if (warp == 0) {
      cdf pc = c_zero();
      for (int q = lane; q < nown; q += 32) {
        const int i = i0 + q * G, lr = lrow0 + q;
        cdf y = ld4(&segp[lr * TD_SEG]);
        for (int sg = 1; sg < S_prev; ++sg) y = c_add(y, ld4(&segp[lr * TD_SEG + sg]));
        const float4* row = row_of(k + 1 + i) + (k + 1);
        const cdf w0 = c_mul(tau, c_add(ld4(&row[0]), c_mul(scale, y)));
        st4(&wg[i], w0);
        const cdf vi = i == 0 ? cdf{{1.f, 0.f}, {0.f, 0.f}} : c_mul(c_conj(ld4(&x[1 + i])), scale);
        pc = c_add(pc, c_mulc(w0, vi));
      }
      pc = c_warp_sum(pc);
      if (lane == 0) st4(&pg[c], pc);
    }
    if (!grid_sync_count(a.gs, epoch)) return;
    // --- 3. v (from the pivot row, before it is overwritten) while the other CTAs' w0, the
    // published row and the partial sums are loaded; then alpha, w, the next pivot row and its
    // squares
    float4 wpf[TD_PF], ppf[TD_PF], w00;
    if (warp * 32 < m) {
#pragma unroll
      for (int t = 0; t < TD_PF; ++t) {
        const int j = tid + t * TD_THREADS;
        if (j < m) {
          wpf[t] = __ldcg(&wg[j]);
          ppf[t] = __ldcg(&pub[j]);
        }
      }
      w00 = __ldcg(&wg[0]);
    }
    for (int j = tid; j < m; j += TD_THREADS) {
      const cdf vj = j == 0 ? cdf{{1.f, 0.f}, {0.f, 0.f}} : c_mul(c_conj(ld4(&x[1 + j])), scale);
      st4(&v[j], vj);
      if (c == 0) st4(&a.refl[(long long)k * n + j], vj);
    }
    __syncthreads();
    if (warp * 32 < m) {
      cdf sp = c_zero();
      for (int q = lane; q < G; q += 32) sp = c_add(sp, ld4(&pg[q]));
      const cdf ssum = c_warp_sum(sp);
      const cdf htau = {df_mul_f(tau.re, -0.5f), df_mul_f(tau.im, -0.5f)};
      const cdf alpha = c_mul(htau, ssum);
      const cdf w0c = c_add({{w00.x, w00.y}, {w00.z, w00.w}}, alpha);  // w_0 (v_0 = 1)
      auto form = [&](int j, const float4 wr, const float4 pr) {
        const cdf vj = ld4(&v[j]);
        const cdf wj = c_add({{wr.x, wr.y}, {wr.z, wr.w}}, c_mul(alpha, vj));
        st4(&w[j], wj);
        const cdf xj = c_sub({{pr.x, pr.y}, {pr.z, pr.w}}, c_add(c_conj(wj), c_mul(w0c, c_conj(vj))));
        st4(&x[j], xj);
        xsq[j] = dpack(df_add(df_mul(xj.re, xj.re), df_mul(xj.im, xj.im)));
      };
#pragma unroll
      for (int t = 0; t < TD_PF; ++t)
        if (tid + t * TD_THREADS < m) form(tid + t * TD_THREADS, wpf[t], ppf[t]);
      for (int j = tid + TD_PF * TD_THREADS; j < m; j += TD_THREADS) form(j, __ldcg(&wg[j]), __ldcg(&pub[j]));
    }
    __syncthreads();
    // --- 4. warps 0..nw-2: rank-2 update of the own rows but row k+1, each updated entry
    // (columns j >= 2) summed at once against conj(x') for the next step's row sums: S warps per
    // row, each over every S-th 32-column chunk; warp nw-1 meanwhile: the Householder scalars of
    // step k+1
    const int S = (nown > 0 && 2 * nown <= nw - 1) ? min(TD_SEG, (nw - 1) / nown) : 1;
    if (warp < nw - 1) {
      for (int t = warp; t < nown * S; t += nw - 1) {
        const int q = t / S, sg = t - q * S;
        const int i = i0 + q * G;
        if (i == 0) continue;
        // global row k+1+i = c + G (lrow0 + q): no division per entry
        float4* arow = (ROWS_IN_SMEM ? rows + (size_t)(lrow0 + q) * n : a.A + (size_t)(k + 1 + i) * n) + (k + 1);
        const cdf vi = ld4(&v[i]), wi = ld4(&w[i]);
        cdf y = c_zero();
        for (int j = 32 * sg + lane; j < m; j += 32 * S) {
          cdf acc = ld4(&arow[j]);
          if (active) {
            const cdf wj = ld4(&w[j]), vjj = ld4(&v[j]);
            df_acc_mul(acc.re, df_neg(vi.re), wj.re);
            df_acc_mul(acc.re, df_neg(vi.im), wj.im);
            df_acc_mul(acc.re, df_neg(wi.re), vjj.re);
            df_acc_mul(acc.re, df_neg(wi.im), vjj.im);
            df_acc_mul(acc.im, df_neg(vi.im), wj.re);
            df_acc_mul(acc.im, vi.re, wj.im);
            df_acc_mul(acc.im, df_neg(wi.im), vjj.re);
            df_acc_mul(acc.im, wi.re, vjj.im);
            acc = c_renorm(acc);
            st4(&arow[j], acc);
          }
          if (j >= 2) c_acc_mul(y, acc, c_conj(ld4(&x[j])));
        }
        y = c_warp_sum(y);
        if (lane == 0) st4(&segp[(lrow0 + q) * TD_SEG + sg], y);
      }
    } else if (k + 1 < n - 1) {
      cdf tau1, scale1;
      dfl beta1;
      td_scalars(m - 1, x, xsq, tau1, scale1, beta1);
      if (lane == 0) {
        st4(&hs[0], tau1);
        st4(&hs[1], scale1);
        hs[2] = make_float4(beta1.hi, beta1.lo, 0.f, 0.f);
      }
    }
    S_prev = S;
    __syncthreads();
  }
  if (c == 0 && tid == 0) a.d[n - 1] = dpack(ld4(&x[0]).re);
}

// ---------------------------------------------------------------- one-cluster form (n <= 416)
//
// The same steps inside one thread-block cluster of TDC_CTAS CTAs: global row g lives in the
// shared memory of CTA g mod TDC_CTAS (local row g / TDC_CTAS) for the whole run, and a step has
// one hardware cluster barrier.  Whatever other CTAs need is pushed into their shared memory by
// its producer before the barrier (remote stores, ordered by the barrier's release / acquire),
// so that after it every CTA reads locally: w0_i from the owner of row i, the CTAs' partial sums
// of conj(w0) v, and the stored row k+2 (the next step's pivot source) from its owner as it is
// updated.  Per step k, with v = conj(x_{1..m}) / (x0 - beta) (x the pivot row, v_0 = 1):
//   1. row sums s_i = sum_{j>=1} A_ij conj(x_{1+j}) of the own rows (a warp per row);
//      w0_i = tau (A_i0 + s_i / (x0 - beta)) pushed to every CTA.  CTA barrier.
//   2. v; the CTA's partial sum of conj(w0_i) v_i pushed to every CTA.  Cluster barrier.
//   3. alpha = -tau/2 sum conj(w0) v; w = w0 + alpha v; the next pivot row
//      x' = (stored row k+1) - conj(w) - w_0 conj(v) and the squares of its entries.  CTA barrier.
//   4. warps 0..nw-2: rank-2 update of the own rows but row k+1 (row k+2 pushed as it is
//      written); warp nw-1 meanwhile: the norm of x' and the Householder scalars of step k+1.
//      CTA barrier.
constexpr int TDC_CTAS = 16;
constexpr int TDC_THREADS = 512;
constexpr int TDC_MAX_N = 416;  // shared memory: R n + 7 n + R float4 and n float2 within 227 KB

struct TdcArgs {
  int n;
  const float4* A;  // n x n scaled double-float copy of G
  float2* d;
  float2* e;
  float4* refl;
  float4* tau;
};

__global__ void __launch_bounds__(TDC_THREADS, 1) tridiag_cluster_kernel(const TdcArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank(), nct = (int)cl.num_blocks();
  const int n = a.n;
  const int R = (n + nct - 1) / nct;
  extern __shared__ float4 csm[];
  float4* rows = csm;                // [R][n] own rows
  float4* x = rows + (size_t)R * n;  // [n] pivot row
  float4* v = x + n;                 // [n]
  float4* w = v + n;                 // [n]
  float4* w0all = w + n;             // [2][n] w0 of every trailing row (pushed by the owners), by step parity
  float4* pub = w0all + 2 * n;       // [2][n] the next pivot row as stored (pushed by its owner), by step parity
  float4* pcs = pub + 2 * n;         // [R] conj(w0_i) v_i of the own rows
  float2* xsq = (float2*)(pcs + R);  // [n] squares of the pivot row's entries (double-float)
  __shared__ float4 partall[2][TDC_CTAS];  // every CTA's partial sum of conj(w0) v, by step parity
  __shared__ float4 hs[3];                 // tau, 1 / (x0 - beta), beta of the current step
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = TDC_THREADS / 32;
  for (int idx = tid; idx < R * n; idx += TDC_THREADS) {
    const int lr = idx / n, j = idx - lr * n;
    const int g = lr * nct + crank;
    if (g < n) rows[idx] = a.A[(size_t)g * n + j];
  }
  for (int j = tid; j < n; j += TDC_THREADS) {
    const float4 xj = a.A[j];
    x[j] = xj;
    xsq[j] = dpack(df_add(df_mul({xj.x, xj.y}, {xj.x, xj.y}), df_mul({xj.z, xj.w}, {xj.z, xj.w})));
    if (j < n - 1) pub[j] = a.A[(size_t)n + 1 + j];  // row 1 from column 1: step 0's pivot source
  }
  __syncthreads();
  if (warp == nw - 1) {
    cdf tau, scale;
    dfl beta;
    td_scalars(n - 1, x, xsq, tau, scale, beta);
    if (lane == 0) {
      st4(&hs[0], tau);
      st4(&hs[1], scale);
      hs[2] = make_float4(beta.hi, beta.lo, 0.f, 0.f);
    }
  }
  cl.sync();  // every CTA running (remote stores below) and the step-0 scalars in place
  for (int k = 0; k < n - 1; ++k) {
    const int m = n - k - 1;  // m <= TDC_MAX_N - 1 < TDC_THREADS: one entry per thread below
    const int par = k & 1;
    const int lr0 = (k + 1 - crank + nct - 1) / nct;  // first own local row with g >= k+1
    const int nown = lr0 < R ? R - lr0 - ((R - 1) * nct + crank >= n ? 1 : 0) : 0;
    const cdf tau = ld4(&hs[0]), scale = ld4(&hs[1]);
    const bool active = !(tau.re.hi == 0.f && tau.im.hi == 0.f);
    if (crank == 0 && tid == 0) {
      a.d[k] = dpack(ld4(&x[0]).re);
      a.e[k] = dpack({hs[2].x, hs[2].y});
      st4(&a.tau[k], tau);
    }
    // --- 1. row sums against conj(x); w0 of the own rows pushed to every CTA
    for (int q = warp; q < nown; q += nw) {
      const int lr = lr0 + q, i = lr * nct + crank - (k + 1);
      const float4* row = rows + (size_t)lr * n + (k + 1);
      cdf y = c_zero();
      for (int j = 1 + lane; j < m; j += 32) c_acc_mul(y, ld4(&row[j]), c_conj(ld4(&x[1 + j])));
      y = c_warp_sum(y);  // the same in every lane
      const cdf w0 = c_mul(tau, c_add(ld4(&row[0]), c_mul(scale, y)));
      if (lane < nct) st4(cl.map_shared_rank(w0all, lane) + par * n + i, w0);
      if (lane == 0) {
        const cdf vi = i == 0 ? cdf{{1.f, 0.f}, {0.f, 0.f}} : c_mul(c_conj(ld4(&x[1 + i])), scale);
        st4(&pcs[q], c_mulc(w0, vi));
      }
    }
    __syncthreads();
    // --- 2. the CTA's partial sum pushed to every CTA; v after the cluster barrier is arrived at
    // (its entries are this thread's alone until step 3's CTA barrier)
    if (warp == 0) {
      const cdf pc = c_warp_sum(lane < nown ? ld4(&pcs[lane]) : c_zero());
      if (lane < nct) st4(cl.map_shared_rank(&partall[0][0], lane) + par * TDC_CTAS + crank, pc);
    }
    cl.barrier_arrive();
    cdf vt = c_zero();
    if (tid < m) {
      vt = tid == 0 ? cdf{{1.f, 0.f}, {0.f, 0.f}} : c_mul(c_conj(ld4(&x[1 + tid])), scale);
      st4(&v[tid], vt);
      if (crank == 0) st4(&a.refl[(long long)k * n + tid], vt);
    }
    cl.barrier_wait();
    // --- 3. alpha, w, the next pivot row and its squares (all local reads)
    if (warp * 32 < m) {  // only the warps that form entries need alpha
      const cdf ssum = c_warp_sum(lane < nct ? ld4(&partall[par][lane]) : c_zero());
      const cdf htau = {df_mul_f(tau.re, -0.5f), df_mul_f(tau.im, -0.5f)};
      const cdf alpha = c_mul(htau, ssum);
      if (tid < m) {
        const cdf wt = c_add(ld4(&w0all[par * n + tid]), c_mul(alpha, vt));
        const cdf w0 = c_add(ld4(&w0all[par * n]), alpha);  // w_0 (v_0 = 1)
        st4(&w[tid], wt);
        const cdf xt = c_sub(ld4(&pub[par * n + tid]), c_add(c_conj(wt), c_mul(w0, c_conj(vt))));
        st4(&x[tid], xt);
        xsq[tid] = dpack(df_add(df_mul(xt.re, xt.re), df_mul(xt.im, xt.im)));
      }
    }
    __syncthreads();
    // --- 4. rank-2 update (warps 0..nw-2) / Householder scalars of step k+1 (warp nw-1)
    if (warp < nw - 1) {
      if (active) {
        const int tot = nown * m;
        const float rm = 1.f / (float)m;
        float4* nxt = pub + (par ^ 1) * n;  // row k+2 from column k+2, for step k+1
        for (int idx = tid; idx < tot; idx += TDC_THREADS - 32) {
          const int q = (int)__fmul_rn((float)idx + 0.5f, rm);  // idx / m (exact: idx < 2^14, m <= 415)
          const int j = idx - q * m;
          const int lr = lr0 + q, i = lr * nct + crank - (k + 1);
          if (i == 0) continue;
          float4* aij = rows + (size_t)lr * n + (k + 1) + j;
          const cdf vi = ld4(&v[i]), wi = ld4(&w[i]), wj = ld4(&w[j]), vjj = ld4(&v[j]);
          cdf acc = ld4(aij);
          df_acc_mul(acc.re, df_neg(vi.re), wj.re);
          df_acc_mul(acc.re, df_neg(vi.im), wj.im);
          df_acc_mul(acc.re, df_neg(wi.re), vjj.re);
          df_acc_mul(acc.re, df_neg(wi.im), vjj.im);
          df_acc_mul(acc.im, df_neg(vi.im), wj.re);
          df_acc_mul(acc.im, vi.re, wj.im);
          df_acc_mul(acc.im, df_neg(wi.im), vjj.re);
          df_acc_mul(acc.im, wi.re, vjj.im);
          acc = c_renorm(acc);
          st4(aij, acc);
          if (i == 1 && j >= 1)
            for (int r = 0; r < nct; ++r) st4(cl.map_shared_rank(nxt, r) + (j - 1), acc);
        }
      } else {
        // no update: row k+2 as stored is the next pivot source
        for (int idx = tid; idx < nown * m; idx += TDC_THREADS - 32) {
          const int q = (int)__fmul_rn((float)idx + 0.5f, 1.f / (float)m);
          const int j = idx - q * m;
          const int lr = lr0 + q, i = lr * nct + crank - (k + 1);
          if (i != 1 || j < 1) continue;
          const float4 val = rows[(size_t)lr * n + (k + 1) + j];
          for (int r = 0; r < nct; ++r) cl.map_shared_rank(pub + (par ^ 1) * n, r)[j - 1] = val;
        }
      }
    } else if (k + 1 < n - 1) {
      cdf tau1, scale1;
      dfl beta1;
      td_scalars(m - 1, x, xsq, tau1, scale1, beta1);
      if (lane == 0) {
        st4(&hs[0], tau1);
        st4(&hs[1], scale1);
        hs[2] = make_float4(beta1.hi, beta1.lo, 0.f, 0.f);
      }
    }
    __syncthreads();
  }
  if (crank == 0 && tid == 0) a.d[n - 1] = dpack(ld4(&x[0]).re);
  cl.sync();  // no CTA leaves while others may still read or write its shared memory
}

static size_t tdc_smem(int n) {
  const int R = (n + TDC_CTAS - 1) / TDC_CTAS;
  return sizeof(float4) * ((size_t)R * n + 7 * (size_t)n + (size_t)R) + sizeof(float2) * (size_t)n;
}

static cudaLaunchConfig_t tdc_cfg(size_t smem, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = TDC_CTAS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(TDC_CTAS);
  cfg.blockDim = dim3(TDC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// whether this device runs the one-cluster form for n (cached per n; host threads of a batch
// share it)
static bool tdc_available(int n) {
  if (n < 2 || n > TDC_MAX_N) return false;
  static std::atomic<int> cached[TDC_MAX_N + 1];
  static std::mutex mu;
  const int known = cached[n].load();
  if (known) return known > 0;
  std::lock_guard<std::mutex> lock(mu);
  int ok = -1;
  const size_t smem = tdc_smem(n);
  if (cudaFuncSetAttribute(tridiag_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess &&
      allow_max_dynamic_smem((const void*)tridiag_cluster_kernel) == cudaSuccess) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tdc_cfg(smem, 0, attr);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, tridiag_cluster_kernel, &cfg) == cudaSuccess && clusters >= 1)
      ok = 1;
  }
  cudaGetLastError();
  cached[n].store(ok);
  return ok > 0;
}

// A = 2^-e G in double-float (the largest |Re|, |Im| of G in [2^(e-1), 2^e)); scale = 2^-e
__global__ void td_prep_kernel(long long nn, const double2* __restrict__ G, const unsigned long long* amax_bits,
                               double* scale_out, float4* __restrict__ A) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  const double amax = __longlong_as_double((long long)*amax_bits);
  int ex2 = 0;
  if (amax > 0.0 && amax <= 1.7e308) frexp(amax, &ex2);
  const double sc = ldexp(1.0, -ex2);
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = sc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const double2 g = G[i];
    st4(&A[i], c_from(make_double2(g.x * sc, g.y * sc)));
  }
}

// Gershgorin interval of T, its norm bound and the pivot floor; e2[i] = e[i]^2.
// info: [0] lo, [1] hi (double-float), [2] tnorm, [3] pivmin (float in .x)
__global__ void td_bounds_kernel(int n, const float2* __restrict__ d, const float2* __restrict__ e,
                                 float2* __restrict__ e2, float2* __restrict__ info) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  __shared__ float s_lo[256], s_hi[256], s_e2[256];
  float lo = 3e38f, hi = -3e38f, e2m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float el = i > 0 ? fabsf(e[i - 1].x) : 0.f, er = i < n - 1 ? fabsf(e[i].x) : 0.f;
    lo = fminf(lo, d[i].x - el - er);
    hi = fmaxf(hi, d[i].x + el + er);
    if (i < n - 1) {
      const dfl ei = dload(e[i]);
      e2[i] = dpack(df_mul(ei, ei));
      e2m = fmaxf(e2m, ei.hi * ei.hi);
    }
  }
  s_lo[threadIdx.x] = lo;
  s_hi[threadIdx.x] = hi;
  s_e2[threadIdx.x] = e2m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s_lo[threadIdx.x] = fminf(s_lo[threadIdx.x], s_lo[threadIdx.x + o]);
      s_hi[threadIdx.x] = fmaxf(s_hi[threadIdx.x], s_hi[threadIdx.x + o]);
      s_e2[threadIdx.x] = fmaxf(s_e2[threadIdx.x], s_e2[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // the bounds use the hi parts only: widen them by a relative 2^-20
    const float tn = fmaxf(fabsf(s_lo[0]), fabsf(s_hi[0]));
    const float pad = 0x1.0p-20f * tn + 1e-30f;
    const float pivmin = 1e-33f * fmaxf(1.f, s_e2[0]);
    info[0] = make_float2(s_lo[0] - pad, 0.f);
    info[1] = make_float2(s_hi[0] + pad, 0.f);
    info[2] = make_float2(tn, 0.f);
    info[3] = make_float2(pivmin, 0.f);
  }
}

// number of eigenvalues of T below x (Sturm count on the LDL^T pivots); d, e2 in shared memory
__device__ __forceinline__ int sturm_count(int n, const float2* d, const float2* e2, dfl x, float pivmin) {
  dfl q = df_sub(dload(d[0]), x);
  if (fabsf(q.hi) <= pivmin) q = {-pivmin, 0.f};
  int cnt = q.hi < 0.f;
  for (int i = 1; i < n; ++i) {
    q = df_sub(df_sub(dload(d[i]), x), df_mul(dload(e2[i - 1]), df_rcp(q)));
    if (fabsf(q.hi) <= pivmin) q = {-pivmin, 0.f};
    cnt += q.hi < 0.f;
  }
  return cnt;
}

// Eigenvalue t0 + blockIdx.x (ascending order), one CTA each: multisection with P = blockDim.x
// points a round (a multiple of 32, at most TB_THREADS) to an absolute width of 2^-46 ||T||:
// FP32 rounds from the Gershgorin interval while the bracket is wider than 2^-14 ||T||, then
// double-float rounds.  P follows the number of eigenvalues (bisection_points): the Sturm counts
// are long dependent chains, so a few eigenvalues want many points (fewer rounds) and many
// eigenvalues want few (the sweeps of all CTAs are issue-bound beyond ~8 warps per SM).
// Dynamic shared memory: d and e2 (2 n float2).
constexpr int TB_THREADS = 256;

__global__ void __launch_bounds__(TB_THREADS) td_bisect_kernel(int n, int t0, const float2* __restrict__ d,
                                                               const float2* __restrict__ e2,
                                                               const float2* __restrict__ info,
                                                               const double* __restrict__ scale,
                                                               float2* __restrict__ lam_scaled,
                                                               double* __restrict__ lam_out) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  extern __shared__ float2 bsm[];
  float2* sd = bsm;
  float2* se2 = bsm + n;
  __shared__ int wfirst[2][TB_THREADS / 32];
  const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = blockDim.x, nw = P >> 5;
  const int t = t0 + g;
  for (int i = tid; i < n; i += P) {
    sd[i] = d[i];
    if (i < n - 1) se2[i] = e2[i];
  }
  __syncthreads();
  const float tol = 0x1.0p-46f * info[2].x + info[3].x;
  const float pivmin = info[3].x;
  // the index of the first of the P points whose count exceeds t (P when none), from the warps'
  // ballots; the two buffers alternate by round, so one CTA barrier a round suffices
  int rnd = 0;
  auto first_above = [&](bool above_t) -> int {
    const unsigned above = __ballot_sync(0xffffffffu, above_t);
    if (lane == 0) wfirst[rnd & 1][warp] = above ? warp * 32 + __ffs(above) - 1 : P;
    __syncthreads();
    int first = P;
    for (int w = 0; w < nw; ++w) first = min(first, wfirst[rnd & 1][w]);
    ++rnd;
    return first;
  };
  // FP32 rounds first.  An FP32 Sturm count (reciprocal to ~2^-22) is exact for a matrix whose d
  // and e^2 differ from T's by a few ulps relatively, so its bracket holds the eigenvalue of T
  // within ~12 * 2^-24 ||T|| (Weyl); widened by 2^-16 ||T|| on each side it is handed to the
  // double-float rounds.
  float lo32 = info[0].x, hi32 = info[1].x;
  const float inv32 = 1.f / (float)(P + 1);
  for (int it = 0; it < 8 && hi32 - lo32 > 0x1.0p-14f * info[2].x; ++it) {
    const float step32 = (hi32 - lo32) * inv32;
    const float x32 = lo32 + step32 * (float)(tid + 1);
    float q = sd[0].x - x32;
    if (fabsf(q) <= pivmin) q = -pivmin;
    int cnt = q < 0.f;
    for (int i = 1; i < n; ++i) {
      q = (sd[i].x - x32) - se2[i - 1].x * rcp_approx(q);
      if (fabsf(q) <= pivmin) q = -pivmin;
      cnt += q < 0.f;
    }
    const int first = first_above(cnt > t);
    const float nlo = first == 0 ? lo32 : lo32 + step32 * (float)first;
    const float nhi = first == P ? hi32 : lo32 + step32 * (float)(first + 1);
    lo32 = nlo;
    hi32 = nhi;
  }
  const float pad = 0x1.0p-16f * info[2].x + pivmin;
  dfl lo = df_sub(df_f(lo32), df_f(pad)), hi = df_add(df_f(hi32), df_f(pad));
  const dfl inv = df_div(df_f(1.f), df_f((float)(P + 1)));
  for (int it = 0; it < 24 && df_sub(hi, lo).hi > tol; ++it) {
    const dfl step = df_mul(df_sub(hi, lo), inv);
    const int cnt = sturm_count(n, sd, se2, df_add(lo, df_mul_f(step, (float)(tid + 1))), pivmin);
    // the first point whose count exceeds t bounds the eigenvalue from above
    const int first = first_above(cnt > t);
    const dfl nlo = first == 0 ? lo : df_add(lo, df_mul_f(step, (float)first));
    const dfl nhi = first == P ? hi : df_add(lo, df_mul_f(step, (float)(first + 1)));
    lo = nlo;
    hi = nhi;
  }
  if (tid == 0) {
    const dfl l = df_mul_f(df_add(lo, hi), 0.5f);
    if (lam_scaled) lam_scaled[g] = dpack(l);
    if (lam_out) lam_out[g] = df_to(l) / *scale;
  }
}

// points a round for `count` eigenvalues: about 8 warps of Sturm chains per SM in all
static int bisection_points(int count, int num_sms) {
  const long long target = (long long)num_sms * 8 * 32;
  int P = TB_THREADS;
  while (P > 32 && (long long)count * P > target) P >>= 1;
  return P;
}

__device__ __forceinline__ float hash_unit(uint64_t t, uint64_t i) {
  uint64_t z = t * 0x9E3779B97F4A7C15ull + i * 0xBF58476D1CE4E5B9ull + 1ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(z >> 40) * 0x1.0p-24f * 2.f - 1.f;
}

// Eigenvectors of T for lam[0..r) (ascending) by inverse iteration; Z[j] (length n, real, unit).
// One warp per run of eigenvalues closer than 1e-10 ||T|| (the block of the run's first index
// does the work; the others leave): lane 0 runs the serial pivoted LU and the triangular
// solves in shared memory, the warp normalises and orthogonalises each new vector against the
// run's earlier ones (modified Gram-Schmidt).  The factors are stored for short serial chains:
// forward step (l_i, swap_i) in one float4; backward step x_i = z_i / u1_i - (u2_i / u1_i)
// x_{i+1} - (u3_i / u1_i) x_{i+2} with the three quotients in one float4 and a float2; the next
// step's factors are loaded one step ahead.  Shared memory: 6 n float2 (+ 2 n for copies of d and
// e when they fit, stage != 0).
__global__ void __launch_bounds__(32) td_inviter_kernel(int n, int r, const float2* __restrict__ d,
                                                        const float2* __restrict__ e,
                                                        const float2* __restrict__ lam,
                                                        const float2* __restrict__ info, float2* __restrict__ Z,
                                                        int stage) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  extern __shared__ __align__(16) float2 ism[];
  float4* fw = reinterpret_cast<float4*>(ism);  // [n] forward: (l.hi, l.lo, swap, 0)
  float4* bk = fw + n;                          // [n] backward: (u2/u1 .hi .lo, u3/u1 .hi .lo)
  float2* bi = reinterpret_cast<float2*>(bk + n);  // [n] 1 / u1
  float2* z = bi + n;                           // [n]
  float2* sd = stage ? z + n : nullptr;
  float2* se = stage ? sd + n : nullptr;
  const int j0 = blockIdx.x, lane = threadIdx.x;
  const float tnorm = info[2].x;
  const float ctol = 1e-10f * tnorm;
  if (j0 > 0 && df_sub(dload(lam[j0]), dload(lam[j0 - 1])).hi < ctol) return;  // not the first of its run
  int j1 = j0 + 1;
  while (j1 < r && df_sub(dload(lam[j1]), dload(lam[j1 - 1])).hi < ctol) ++j1;
  const float tiny = 0x1.0p-46f * tnorm + info[3].x;
  if (stage) {
    for (int i = lane; i < n; i += 32) {
      sd[i] = d[i];
      se[i] = i < n - 1 ? e[i] : make_float2(0.f, 0.f);
    }
    __syncwarp();
  }
  const float2* dd = stage ? sd : d;
  const float2* ee = stage ? se : e;
  for (int j = j0; j < j1; ++j) {
    const dfl lj = dload(lam[j]);
    if (lane == 0) {
      // pivoted LU of T - lj I
      dfl ca = df_sub(dload(dd[0]), lj), cc = dload(ee[0]);
      for (int i = 0; i < n - 1; ++i) {
        const dfl b = dload(ee[i]);
        const dfl na = df_sub(dload(dd[i + 1]), lj), nc = (i + 1 < n - 1) ? dload(ee[i + 1]) : df_f(0.f);
        if (fabsf(ca.hi) >= fabsf(b.hi)) {
          const dfl piv = fabsf(ca.hi) > tiny ? ca : df_f(ca.hi >= 0.f ? tiny : -tiny);
          const dfl pinv = df_rcp(piv);
          const dfl l = df_mul(b, pinv);
          const dfl q2 = df_mul(cc, pinv);
          fw[i] = make_float4(l.hi, l.lo, 0.f, 0.f);
          bk[i] = make_float4(q2.hi, q2.lo, 0.f, 0.f);
          bi[i] = dpack(pinv);
          ca = df_sub(na, df_mul(l, cc));
          cc = nc;
        } else {
          const dfl binv = df_rcp(b);
          const dfl l = df_mul(ca, binv);
          const dfl q2 = df_mul(na, binv), q3 = df_mul(nc, binv);
          fw[i] = make_float4(l.hi, l.lo, 1.f, 0.f);
          bk[i] = make_float4(q2.hi, q2.lo, q3.hi, q3.lo);
          bi[i] = dpack(binv);
          ca = df_sub(cc, df_mul(l, na));
          cc = df_neg(df_mul(l, nc));
        }
      }
      const dfl last = fabsf(ca.hi) > tiny ? ca : df_f(ca.hi >= 0.f ? tiny : -tiny);
      bk[n - 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      bi[n - 1] = dpack(df_rcp(last));
    }
    for (int i = lane; i < n; i += 32) z[i] = make_float2(hash_unit((uint64_t)(j + 1), (uint64_t)i), 0.f);
    __syncwarp();
    for (int iter = 0; iter < 3; ++iter) {
      if (lane == 0) {
        // forward: row swaps and L (factors and the next entry loaded a step ahead)
        dfl zi = dload(z[0]);
        float4 f = fw[0];
        float2 znx = n > 1 ? z[1] : make_float2(0.f, 0.f);
        for (int i = 0; i < n - 1; ++i) {
          const float4 fn = fw[i + 1 < n - 1 ? i + 1 : i];
          const float2 zn2 = z[i + 2 < n ? i + 2 : i + 1];
          dfl zn = dload(znx);
          if (f.z != 0.f) {
            const dfl t = zi;
            zi = zn;
            zn = t;
          }
          z[i] = dpack(zi);
          zi = df_sub(zn, df_mul({f.x, f.y}, zi));
          f = fn;
          znx = zn2;
        }
        z[n - 1] = dpack(zi);
        // back substitution: x_i = z_i / u1_i - q2_i x_{i+1} - q3_i x_{i+2}
        dfl x1 = df_f(0.f), x2 = df_f(0.f);  // x[i+1], x[i+2]
        float4 bq = bk[n - 1];
        float2 bz = z[n - 1], bu = bi[n - 1];
        for (int i = n - 1; i >= 0; --i) {
          const int ip = i > 0 ? i - 1 : 0;
          const float4 bqn = bk[ip];
          const float2 bzn = z[ip], bun = bi[ip];
          // off the chain: z_i / u1_i - q3_i x_{i+2}
          const dfl t = df_sub(df_mul(dload(bz), dload(bu)), df_mul({bq.z, bq.w}, x2));
          const dfl xi = df_sub(t, df_mul({bq.x, bq.y}, x1));
          z[i] = dpack(xi);
          x2 = x1;
          x1 = xi;
          bq = bqn;
          bz = bzn;
          bu = bun;
        }
      }
      __syncwarp();
      for (int q = j0; q < j; ++q) {  // modified Gram-Schmidt against the run's earlier vectors
        const float2* p = Z + (size_t)q * n;
        dfl dp = df_f(0.f);
        for (int i = lane; i < n; i += 32) dp = df_add(dp, df_mul(dload(p[i]), dload(z[i])));
        dp = df_warp_sum(dp);
        for (int i = lane; i < n; i += 32) z[i] = dpack(df_sub(dload(z[i]), df_mul(dp, dload(p[i]))));
        __syncwarp();
      }
      // scale by a power of two first (the solve can grow by ~1 / tiny), then normalise
      float mx = 0.f;
      for (int i = lane; i < n; i += 32) mx = fmaxf(mx, fabsf(z[i].x));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      int ex = 0;
      frexpf(mx, &ex);
      const float p2 = ldexpf(1.f, -ex);
      dfl nrm = df_f(0.f);
      for (int i = lane; i < n; i += 32) {
        const dfl zi = df_mul_f(dload(z[i]), p2);
        z[i] = dpack(zi);
        nrm = df_add(nrm, df_mul(zi, zi));
      }
      nrm = df_warp_sum(nrm);
      const dfl inv = nrm.hi > 0.f ? df_div(df_f(1.f), df_sqrt(nrm)) : df_f(0.f);
      for (int i = lane; i < n; i += 32) z[i] = dpack(df_mul(dload(z[i]), inv));
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) Z[(size_t)j * n + i] = z[i];
    __syncwarp();
  }
}

// Compact WY form of the back-transformation (Schreiber & Van Loan 1989): for a block of WY_B
// consecutive reflectors H_k0 ... H_k1-1 = I - Y T Y^H, with Y = [v_k0 .. v_k1-1] (v_k supported
// on the rows k+1 .. n-1) and T upper triangular: T_ii = tau_i, T[0:i, i] = -tau_i T[0:i, 0:i]
// (Y[:, 0:i]^H v_i).  One CTA per block builds T (into Tb) and a row-major copy of the block's
// reflectors Yt[block][g][j] (g = global row), used by the update u -= Y t.
constexpr int WY_B = 32;

__global__ void __launch_bounds__(256) td_wy_t_kernel(int n, const float4* __restrict__ refl,
                                                      const float4* __restrict__ tau, float4* __restrict__ Tb,
                                                      float4* __restrict__ Yt) {
  __shared__ float4 S[WY_B][WY_B + 1];  // S[i][j] = v_i^H v_j (i < j); rows padded against bank conflicts
  __shared__ float4 T[WY_B][WY_B + 1];
  const int blk = blockIdx.x, k0 = blk * WY_B, nb = min(WY_B, n - 1 - k0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // row-major copy: Yt[blk][g][j] = v_{k0+j}[g], zero where g <= k0 + j
  float4* Y = Yt + (size_t)blk * n * WY_B;
  for (int idx = threadIdx.x; idx < n * WY_B; idx += blockDim.x) {
    const int g = idx / WY_B, j = idx - g * WY_B;
    const int k = k0 + j;
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < nb && g > k) val = refl[(size_t)k * n + (g - k - 1)];
    Y[idx] = val;
  }
  __syncthreads();  // Y complete (global writes of this CTA are visible to it after the barrier)
  // S[i][j], i < j, one thread per pair over the rows g >= k0 + j + 1 of the row-major copy: for
  // a given g the threads read within one 512-byte row
  for (int pair = threadIdx.x; pair < WY_B * WY_B; pair += blockDim.x) {
    const int i = pair / WY_B, j = pair - i * WY_B;
    if (!(i < j && j < nb)) continue;
    // four lazily normalised chains (latency), combined at the end
    cdf a0 = c_zero(), a1 = c_zero(), a2 = c_zero(), a3 = c_zero();
    int g = k0 + j + 1;
    for (; g + 3 < n; g += 4) {
      const float4* y0 = Y + (size_t)g * WY_B;
      c_acc_mulc(a0, ld4(&y0[i]), ld4(&y0[j]));
      c_acc_mulc(a1, ld4(&y0[WY_B + i]), ld4(&y0[WY_B + j]));
      c_acc_mulc(a2, ld4(&y0[2 * WY_B + i]), ld4(&y0[2 * WY_B + j]));
      c_acc_mulc(a3, ld4(&y0[3 * WY_B + i]), ld4(&y0[3 * WY_B + j]));
    }
    for (; g < n; ++g) c_acc_mulc(a0, ld4(&Y[(size_t)g * WY_B + i]), ld4(&Y[(size_t)g * WY_B + j]));
    st4(&S[i][j], c_add(c_add(a0, a1), c_add(a2, a3)));
  }
  for (int idx = threadIdx.x; idx < WY_B * WY_B; idx += blockDim.x) T[idx / WY_B][idx % WY_B] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  // column recurrence, warp 0: column i from columns 0..i-1
  if (warp == 0) {
    for (int i = 0; i < nb; ++i) {
      const cdf ti = ld4(&tau[k0 + i]);
      // lane a < i: T[a][i] = -tau_i sum_{c=a}^{i-1} T[a][c] S[c][i]
      if (lane < i) {
        cdf a0 = c_zero(), a1 = c_zero(), a2 = c_zero(), a3 = c_zero();
        int c = lane;
        for (; c + 3 < i; c += 4) {
          c_acc_mul(a0, ld4(&T[lane][c]), ld4(&S[c][i]));
          c_acc_mul(a1, ld4(&T[lane][c + 1]), ld4(&S[c + 1][i]));
          c_acc_mul(a2, ld4(&T[lane][c + 2]), ld4(&S[c + 2][i]));
          c_acc_mul(a3, ld4(&T[lane][c + 3]), ld4(&S[c + 3][i]));
        }
        for (; c < i; ++c) c_acc_mul(a0, ld4(&T[lane][c]), ld4(&S[c][i]));
        const cdf acc = c_add(c_add(a0, a1), c_add(a2, a3));
        const cdf nt = {df_neg(ti.re), df_neg(ti.im)};
        st4(&T[lane][i], c_mul(nt, acc));
      }
      if (lane == 0) st4(&T[i][i], ti);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < WY_B * WY_B; idx += blockDim.x)
    Tb[(size_t)blk * WY_B * WY_B + idx] = T[idx / WY_B][idx % WY_B];
}

// V[j] = Q_H z_j applying the WY blocks last to first: u <- u - Y (T (Y^H u)).  One CTA per
// eigenvector, the vector in shared memory; written as complex128 rows of length n.  s = Y^H u
// with lane = reflector and the warps over rows (each row of the row-major copy is one 512-byte
// read), t = T s with a warp per row of T, and the update with a thread per row reading the
// reflectors column-major (consecutive rows are consecutive addresses).
constexpr int BX_THREADS = 256;

__global__ void __launch_bounds__(BX_THREADS, 2) td_backxform_wy_kernel(int n, int r, const float4* __restrict__ refl,
                                                                    const float4* __restrict__ Tb,
                                                                    const float4* __restrict__ Yt,
                                                                    const float2* __restrict__ Z,
                                                                    double2* __restrict__ V) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  constexpr int NW = BX_THREADS / 32;
  extern __shared__ float4 usm2[];
  __shared__ float4 part[NW][WY_B];
  __shared__ float4 sv[WY_B], tv[WY_B];
  const int j = blockIdx.x;
  if (j >= r) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float4* u = usm2;
  for (int i = tid; i < n; i += BX_THREADS) {
    const float2 zi = Z[(size_t)j * n + i];
    u[i] = make_float4(zi.x, zi.y, 0.f, 0.f);
  }
  __syncthreads();
  const int nblk = (n - 1 + WY_B - 1) / WY_B;
  for (int blk = nblk - 1; blk >= 0; --blk) {
    const int k0 = blk * WY_B, nb = min(WY_B, n - 1 - k0);
    const float4* Y = Yt + (size_t)blk * n * WY_B;  // zero where g <= k0 + lane
    // s = Y^H u
    {
      cdf acc = c_zero();
      int g = k0 + 1 + warp;
#pragma unroll 1
      for (; g + 3 * NW < n; g += 4 * NW) {
        const float4 y0 = Y[(size_t)g * WY_B + lane], y1 = Y[(size_t)(g + NW) * WY_B + lane];
        const float4 y2 = Y[(size_t)(g + 2 * NW) * WY_B + lane], y3 = Y[(size_t)(g + 3 * NW) * WY_B + lane];
        c_acc_mulc(acc, {{y0.x, y0.y}, {y0.z, y0.w}}, ld4(&u[g]));
        c_acc_mulc(acc, {{y1.x, y1.y}, {y1.z, y1.w}}, ld4(&u[g + NW]));
        c_acc_mulc(acc, {{y2.x, y2.y}, {y2.z, y2.w}}, ld4(&u[g + 2 * NW]));
        c_acc_mulc(acc, {{y3.x, y3.y}, {y3.z, y3.w}}, ld4(&u[g + 3 * NW]));
      }
      for (; g < n; g += NW) c_acc_mulc(acc, ld4(&Y[(size_t)g * WY_B + lane]), ld4(&u[g]));
      st4(&part[warp][lane], acc);
    }
    __syncthreads();
    if (warp == 0) {
      cdf sacc = ld4(&part[0][lane]);
#pragma unroll
      for (int w = 1; w < NW; ++w) sacc = c_add(sacc, ld4(&part[w][lane]));
      st4(&sv[lane], sacc);
    }
    __syncthreads();
    // t = T s (T upper triangular): warp per row, lanes over columns
    {
      const float4* Tblk = Tb + (size_t)blk * WY_B * WY_B;
      for (int i = warp; i < WY_B; i += NW) {
        cdf pr = c_zero();
        if (i < nb && lane >= i && lane < nb) pr = c_mul(ld4(&Tblk[i * WY_B + lane]), ld4(&sv[lane]));
        pr = c_warp_sum(pr);
        if (lane == 0) st4(&tv[i], pr);
      }
    }
    __syncthreads();
    // u[g] -= sum_c Y[g][c] t_c for the rows the block touches (Y[g][c] = v_{k0+c}[g], g > k0 + c)
    for (int g = k0 + 1 + tid; g < n; g += BX_THREADS) {
      const int cmax = min(nb, g - k0);
      cdf acc = c_zero();
      const float4* col = refl + (size_t)k0 * n + (g - k0 - 1);  // v_{k0+c}[g] = col[c (n - 1)]
      int c = 0;
#pragma unroll 1
      for (; c + 3 < cmax; c += 4) {
        const float4 y0 = col[(size_t)c * (n - 1)], y1 = col[(size_t)(c + 1) * (n - 1)];
        const float4 y2 = col[(size_t)(c + 2) * (n - 1)], y3 = col[(size_t)(c + 3) * (n - 1)];
        c_acc_mul(acc, {{y0.x, y0.y}, {y0.z, y0.w}}, ld4(&tv[c]));
        c_acc_mul(acc, {{y1.x, y1.y}, {y1.z, y1.w}}, ld4(&tv[c + 1]));
        c_acc_mul(acc, {{y2.x, y2.y}, {y2.z, y2.w}}, ld4(&tv[c + 2]));
        c_acc_mul(acc, {{y3.x, y3.y}, {y3.z, y3.w}}, ld4(&tv[c + 3]));
      }
      for (; c < cmax; ++c) c_acc_mul(acc, ld4(&col[(size_t)c * (n - 1)]), ld4(&tv[c]));
      st4(&u[g], c_sub(ld4(&u[g]), acc));
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += BX_THREADS) V[(size_t)j * n + i] = c_to(ld4(&u[i]));
}

// J = trace(G) - sum of the top r eigenvalues (the tail energy of Eq. 1); trace in FP64
__global__ void td_tail_kernel(int n, int r, const double2* __restrict__ G, const double* __restrict__ lam_top,
                               double* __restrict__ J) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += G[(size_t)i * n + i].x;
  for (int i = threadIdx.x; i < r; i += blockDim.x) s -= lam_top[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *J = fmax(red[0], 0.0);
}

static hicu_status launch_tridiag_grid(hicu_handle* h, int n, float4* A, float2* d, float2* e, float4* refl,
                                       float4* tau, float4* w, float4* part, float4* prow, cudaStream_t st) {
  TdArgs a;
  a.n = n;
  a.A = A;
  a.d = d;
  a.e = e;
  a.refl = refl;
  a.tau = tau;
  a.w = w;
  a.part = part;
  a.prow = prow;
  int grid = h->num_sms;
  // own rows in shared memory when they fit next to the three vectors
  const int R = (n + grid - 1) / grid;
  // x, v, w, the row sums and the squares of x; the own rows on top when they fit
  const size_t smem_vec = sizeof(float4) * (3 * (size_t)n + TD_SEG * (size_t)R) + sizeof(float2) * (size_t)n;
  const size_t smem_rows = smem_vec + sizeof(float4) * (size_t)R * n;
  const bool in_smem = smem_rows <= 200 * 1024;
  const void* kern = in_smem ? (const void*)tridiag_kernel<true> : (const void*)tridiag_kernel<false>;
  const size_t smem = in_smem ? smem_rows : smem_vec;
  {
    cudaError_t e0 = allow_max_dynamic_smem(kern);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "tridiag smem");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TD_THREADS, smem) != cudaSuccess || per_sm < 1)
      return set_error(h, HICU_ERR_CUDA, "principal subspace: occupancy query failed");
    grid = std::max(1, std::min(grid, h->num_sms * per_sm));
  }
  a.gs.count = h->dev_sync;
  a.gs.gen = h->dev_sync + 1;
  a.gs.err = h->dev_err;
  a.gs.nblocks = (unsigned)grid;
  a.gs.timeout_ns = 2000000000ull;  // 2 s per wait
  cudaMemsetAsync(h->dev_sync, 0, 2 * sizeof(unsigned), st);
  void* args[] = {&a};
  cudaError_t ce;
  if (h->coop_mu) {  // batch lane: cooperative launches of all lanes go in order to one stream
    std::lock_guard<std::mutex> lock(*h->coop_mu);
    ce = cudaEventRecord(h->coop_in, st);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h->coop_st, h->coop_in, 0);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(h->dev_sync, 0, 2 * sizeof(unsigned), h->coop_st);
    if (ce == cudaSuccess)
      HICU_LAUNCH(h, K_TRIDIAG, h->coop_st,
                  ce = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(TD_THREADS), args, smem, h->coop_st));
    if (ce == cudaSuccess) ce = cudaEventRecord(h->coop_out, h->coop_st);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, h->coop_out, 0);
  } else {
    HICU_LAUNCH(h, K_TRIDIAG, st, ce = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(TD_THREADS), args, smem, st));
  }
  if (ce != cudaSuccess) return cuda_error(h, ce, "principal subspace: tridiagonalisation launch");
  return HICU_OK;
}

// steps 2-4 and J, after the tridiagonalisation
static hicu_status finish_principal(hicu_handle* h, int n, int r, const double2* G, double* Vout, double* eig_top,
                                    double* eig_all, double* J, float2* d, float2* e, float2* e2, float2* lam,
                                    float2* info, float2* Z, float4* refl, float4* tau, double* scale,
                                    cudaStream_t st) {
  // the compact WY factors of the back-transformation need only the reflectors: build them on
  // the side stream while the eigenvalues and eigenvectors of T are computed
  const int nblk = (n - 1 + WY_B - 1) / WY_B;
  hicu_status sw = HICU_OK;
  float4* Tb = (float4*)ws_get(h, WS_EIG_WY, sizeof(float4) * (size_t)nblk * WY_B * (WY_B + (size_t)n), &sw);
  if (sw) return sw;
  float4* Yt = Tb + (size_t)nblk * WY_B * WY_B;
  if ((sw = ensure_side_stream(h))) return sw;
  {
    cudaError_t ce = cudaEventRecord(h->side_fork, st);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h->side_st, h->side_fork, 0);
    if (ce != cudaSuccess) return cuda_error(h, ce, "principal subspace: fork");
    HICU_LAUNCH_SIDE(h, K_EIG, td_wy_t_kernel<<<nblk, 256, 0, h->side_st>>>(n, refl, tau, Tb, Yt));
    ce = cudaEventRecord(h->side_join, h->side_st);
    if (ce != cudaSuccess) return cuda_error(h, ce, "principal subspace: join");
  }
  // 2. eigenvalues (top r; all n when requested)
  // the eigen-solver chain is stream-ordered (allow = false): as programmatic dependents the
  // waiting CTAs slowed it by 9 % at n = 1000 and gained nothing at n = 200
  launch_pdl(h, K_EIG, st, dim3(1), dim3(256), 0, td_bounds_kernel, false, n, (const float2*)d, (const float2*)e, e2,
             info);
  const size_t bsm_bytes = sizeof(float2) * 2 * (size_t)n;
  {
    cudaError_t e0 = allow_max_dynamic_smem((const void*)td_bisect_kernel);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "bisection smem");
  }
  const int nsm = h->num_sms > 0 ? h->num_sms : 148;
  launch_pdl(h, K_EIG, st, dim3(r), dim3(bisection_points(r, nsm)), bsm_bytes, td_bisect_kernel, false, n, n - r,
             (const float2*)d, (const float2*)e2, (const float2*)info, (const double*)scale, lam, eig_top);
  if (eig_all)
    HICU_LAUNCH(h, K_EIG, st,
                td_bisect_kernel<<<n, bisection_points(n, nsm), bsm_bytes, st>>>(n, 0, d, e2, info, scale, nullptr,
                                                                                 eig_all));
  // 3. eigenvectors of T, 4. back-transformation
  {
    const int stage = 8 * (size_t)n * sizeof(float2) <= 200 * 1024;
    const size_t ism = sizeof(float2) * (stage ? 8 : 6) * (size_t)n;
    cudaError_t e0 = allow_max_dynamic_smem((const void*)td_inviter_kernel);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "inverse iteration smem");
    launch_pdl(h, K_EIG, st, dim3(r), dim3(32), ism, td_inviter_kernel, false, n, r, (const float2*)d, (const float2*)e,
               (const float2*)lam, (const float2*)info, Z, stage);
  }
  {
    // apply the compact WY blocks, one CTA per eigenvector, once the factors are ready
    cudaError_t ce = cudaStreamWaitEvent(st, h->side_join, 0);
    if (ce != cudaSuccess) return cuda_error(h, ce, "principal subspace: wait");
    const size_t usm = sizeof(float4) * (size_t)n;
    cudaError_t e0 = allow_max_dynamic_smem((const void*)td_backxform_wy_kernel);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "backxform smem");
    HICU_LAUNCH(h, K_EIG, st,
                td_backxform_wy_kernel<<<r, BX_THREADS, usm, st>>>(n, r, refl, Tb, Yt, Z, (double2*)Vout));
  }
  if (J)
    launch_pdl(h, K_MISC, st, dim3(1), dim3(256), 0, td_tail_kernel, false, n, r, (const double2*)G,
               (const double*)eig_top, J);
  return cuda_error(h, cudaGetLastError(), "principal subspace");
}

hicu_status run_principal(hicu_handle* h, int64_t n64, int64_t r64, const double* Gd, double* Vout,
                          double* eig_top, double* eig_all, double* J, cudaStream_t st) {
  if (n64 < 2 || n64 > 4096) return set_error(h, HICU_ERR_SHAPE, "principal subspace: n must be in [2, 4096]");
  if (r64 <= 0 || r64 >= n64) return set_error(h, HICU_ERR_RANK, "principal subspace: rank must satisfy 0 < r < n");
  const int n = (int)n64, r = (int)r64;
  const long long nn = (long long)n * n;
  const double2* G = (const double2*)Gd;
  hicu_status s = HICU_OK;
  float4* A = (float4*)ws_get(h, WS_EIG_A0, sizeof(float4) * nn, &s);
  if (s) return s;
  float4* refl = (float4*)ws_get(h, WS_EIG_A1, sizeof(float4) * nn, &s);
  if (s) return s;
  // float4 units: tau (n), w (2n), part (2 nsm), prow (2n); float2 units: d, e, e2, lam (n each), info (4),
  // Z (r n); then amax bits and the scale (8 bytes each)
  const size_t nsm = (size_t)std::max(1, h->num_sms);
  const size_t f4 = (size_t)n + 2 * (size_t)n + 2 * nsm + 2 * (size_t)n;
  const size_t f2 = 4 * (size_t)n + 4 + (size_t)r * n;
  unsigned char* buf = (unsigned char*)ws_get(h, WS_EIG_V, 16 * f4 + 8 * f2 + 16, &s);
  if (s) return s;
  float4* tau = (float4*)buf;
  float4* w = tau + n;
  float4* part = w + 2 * n;
  float4* prow = part + 2 * nsm;
  float2* d = (float2*)(prow + 2 * n);
  float2* e = d + n;
  float2* e2 = e + n;
  float2* lam = e2 + n;
  float2* info = lam + n;
  float2* Z = info + 4;
  unsigned long long* amax_bits = (unsigned long long*)(Z + (size_t)r * n);
  double* scale = (double*)(amax_bits + 1);

  // scaled double-float copy of G
  const int eb = (int)std::min<long long>((nn + 255) / 256, (long long)h->num_sms * 8);
  cudaMemsetAsync(amax_bits, 0, sizeof(unsigned long long), st);
  HICU_LAUNCH(h, K_EIG, st, eig_absmax_kernel<<<eb, 256, 0, st>>>(nn, G, amax_bits));
  launch_pdl(h, K_EIG, st, dim3(eb), dim3(256), 0, td_prep_kernel, false, nn, G, (const unsigned long long*)amax_bits,
             scale, A);

  // 1. tridiagonalisation: one cluster for n <= 416, else cooperative over all SMs
  if (tdc_available(n)) {
    TdcArgs ca;
    ca.n = n;
    ca.A = A;
    ca.d = d;
    ca.e = e;
    ca.refl = refl;
    ca.tau = tau;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tdc_cfg(tdc_smem(n), st, attr);
    cudaError_t ce;
    HICU_LAUNCH(h, K_TRIDIAG, st, ce = cudaLaunchKernelEx(&cfg, tridiag_cluster_kernel, ca));
    if (ce != cudaSuccess) return cuda_error(h, ce, "principal subspace: cluster tridiagonalisation launch");
  } else {
    hicu_status s2 = launch_tridiag_grid(h, n, A, d, e, refl, tau, w, part, prow, st);
    if (s2) return s2;
  }
  return finish_principal(h, n, r, G, Vout, eig_top, eig_all, J, d, e, e2, lam, info, Z, refl, tau, scale, st);
}

}  // namespace hicu
