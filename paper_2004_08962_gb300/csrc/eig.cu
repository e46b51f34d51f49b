// Null-space step (Algorithm 1 steps 2-3 in Gram form): eigen-decomposition of
// the Hermitian n x n matrix G in FP64; Q = eigenvectors of the n - r smallest
// eigenvalues, the orthogonal complement of the r principal right singular
// vectors of H.
//
// Method: cyclic two-sided Jacobi with the round-robin (tournament) ordering,
// so each round rotates n/2 disjoint index pairs at once.  One round is
// A <- W^H A W with W block-diagonal (a 2x2 unitary per pair): every 2x2 block
// of the new matrix depends only on the matching old block and the two
// rotations, so a round is one fully parallel pass (ping-pong buffers) and the
// whole solve is one cooperative persistent kernel with one grid barrier per
// round.  Eigenvectors are accumulated in place (V <- V W).  Convergence is
// tested after every sweep on the off-diagonal mass.  A warm start seeds V with
// the previous call's eigenvectors and starts from V^H G V, which is nearly
// diagonal when G changed little (consecutive HICU iterations).
//
// Rotation for a pair with a = A_pp, c = A_qq, b = A_pq = |b| e^{i phi}:
// W = diag(1, e^{-i phi}) [[cs, sn], [-sn, cs]] with t = sn/cs the smaller root
// of t^2 + 2 tau t - 1 = 0, tau = (c - a) / (2|b|) (the symmetric Schur
// decomposition of Golub & Van Loan, after removing the phase of b).
#include <algorithm>

#include "hicu_internal.cuh"

namespace hicu {

struct Rot {
  double cs, sn, ex, ey;  // W = [[cs, sn], [-sn e, cs e]], e = ex + i ey
  int ident;              // 1: W = I (pair already decoupled)
};

// The rotation angle is computed in FP32 from the FP64 entries (an angle accurate to
// ~1e-7 leaves |A_pq| ~ 1e-7 |b|, so Jacobi still converges, with at worst a 1e-7
// linear rate near the end) and then made unitary to FP64 precision with two Newton
// steps for 1/sqrt(cs^2 + sn^2) and 1/|e|.  This keeps long FP64 sqrt/divide chains
// off the critical path of every round.  Pairs with |b| <= 1e-17 sqrt(|a c|) are left
// alone (the usual relative threshold, which protects tiny eigenvalues).
__device__ __forceinline__ Rot make_rot(double a, double c, double2 b) {
  Rot R;
  // the solver pre-scales A by a power of two to max |A_ij| < 1, so the FP32 conversions
  // below cannot overflow (entries below the FP32 range only ever mean |b| ~ 0)
  const float bx = (float)b.x, by = (float)b.y;
  const float ab = hypotf(bx, by);
  const float thr = 1e-17f * sqrtf(fabsf((float)a)) * sqrtf(fabsf((float)c));
  if (!(ab > thr) || !(ab > 0.f)) {
    R.cs = 1.0; R.sn = 0.0; R.ex = 1.0; R.ey = 0.0; R.ident = 1;
    return R;
  }
  const float tau = (float)(c - a) / (2.f * ab);
  float t;
  if (fabsf(tau) > 1e18f) t = 0.5f / tau;
  else t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
  const float cs = rsqrtf(1.f + t * t);
  double c64 = cs, s64 = (double)t * cs;
  double q = c64 * c64 + s64 * s64;
  double f = 1.5 - 0.5 * q;
  f = f * (1.5 - 0.5 * q * f * f);
  R.cs = c64 * f;
  R.sn = s64 * f;
  double x64 = bx / ab, y64 = -by / ab;
  q = x64 * x64 + y64 * y64;
  f = 1.5 - 0.5 * q;
  f = f * (1.5 - 0.5 * q * f * f);
  R.ex = x64 * f;
  R.ey = y64 * f;
  R.ident = 0;
  return R;
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 rscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

__device__ __forceinline__ void rot_entries(const Rot& R, double2& w00, double2& w01, double2& w10,
                                            double2& w11) {
  w00 = make_double2(R.cs, 0.0);
  w01 = make_double2(R.sn, 0.0);
  w10 = make_double2(-R.sn * R.ex, -R.sn * R.ey);
  w11 = make_double2(R.cs * R.ex, R.cs * R.ey);
}

// circle method: player 0 fixed, players 1..n-1 rotate by t each round
__device__ __forceinline__ void pair_of(int n, int t, int i, int& p, int& q) {
  const int m = n - 1;
  const int a = (i == 0) ? 0 : 1 + (i - 1 + t) % m;
  const int j = n - 1 - i;
  const int b = 1 + (j - 1 + t) % m;
  p = a < b ? a : b;
  q = a < b ? b : a;
}

struct JacArgs {
  int n;  // even (padded)
  double2* A0;
  double2* A1;
  double2* V;
  double* part;  // 2 doubles per CTA
  int* info;     // [0] sweeps, [1] converged, [2] buffer holding the result, [3] final mode
  int max_sweeps;
  double tol2;
  int mode;     // 0: stop when all off-diagonal mass is small; 1: stop when the coupling
                // between the r largest diagonal entries and the rest is small
  int nreal;    // n without the pad index
  int r;
  int* rankd;   // mode 1: descending rank of each diagonal entry (nreal ints)
  unsigned long long* sweep_total;  // running count of sweeps over all calls (tracing)
  GridSync gs;
};

__device__ double dyn_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += sh[i];
  return t;
}

// One warp owns one tile of JT x JT pair-blocks per round.  Pass 1: lane (b, c)
// writes column c of block b of W_P^H A_blk W_Q (all four inputs are loaded, so no
// lane diverges); pass 2: lane (b, r) updates row r of V on the block's column pair.
constexpr int JT = 4;
constexpr int JWARPS = 8;

__device__ __forceinline__ double2 cmul_e(double2 a, double ex, double ey) {  // a * e
  return make_double2(a.x * ex - a.y * ey, a.x * ey + a.y * ex);
}
__device__ __forceinline__ double2 cmul_ce(double2 a, double ex, double ey) {  // conj(e) * a
  return make_double2(a.x * ex + a.y * ey, a.y * ex - a.x * ey);
}
__device__ __forceinline__ double2 lin(double s, double2 a, double t, double2 b) {  // s a + t b
  return make_double2(fma(s, a.x, t * b.x), fma(s, a.y, t * b.y));
}

__global__ void __launch_bounds__(JWARPS * 32) jacobi_kernel(JacArgs J) {
  __shared__ Rot rp[JWARPS][JT], rq[JWARPS][JT];
  __shared__ double red[8];
  __shared__ int s_done;
  const int n = J.n, np = n / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntile = (np + JT - 1) / JT;
  const long long ntiles = (long long)ntile * ntile;
  // tiles interleaved CTA-fastest so that every SM gets work even when tiles < warps
  const long long gw = (long long)warp * gridDim.x + blockIdx.x;
  const long long nw = (long long)gridDim.x * JWARPS;
  int cur = 0;
  unsigned epoch = 0;  // grid barriers passed
  const int mode = J.mode;
  for (int sweep = 0; sweep < J.max_sweeps; ++sweep) {
    for (int t = 0; t < n - 1; ++t) {
      const double2* A = cur ? J.A1 : J.A0;
      double2* B = cur ? J.A0 : J.A1;
      for (long long tile = gw; tile < ntiles; tile += nw) {
        const int tp = (int)(tile / ntile), tq = (int)(tile % ntile);
        // this lane's block (i, j) and column/row `sub`; issue its loads before the rotations
        const int blk = lane >> 1, sub = lane & 1;
        const int i = blk / JT, j = blk % JT;
        const int P = tp * JT + i, Q = tq * JT + j;
        const bool valid = P < np && Q < np;
        // Hermitian: only blocks with P <= Q are transformed; each also writes its mirror
        const bool do_a = valid && (tp < tq || (tp == tq && i <= j));
        int p1 = 0, q1 = 0, p2 = 0, q2 = 0;
        double2 a00, a01, a10, a11, v0, v1;
        if (valid) {
          pair_of(n, t, P, p1, q1);
          pair_of(n, t, Q, p2, q2);
          if (do_a) {
            a00 = A[(long long)p1 * n + p2];
            a01 = A[(long long)p1 * n + q2];
            a10 = A[(long long)q1 * n + p2];
            a11 = A[(long long)q1 * n + q2];
          }
          const long long row = (long long)(sub ? q1 : p1) * n;
          v0 = J.V[row + p2];
          v1 = J.V[row + q2];
        }
        __syncwarp();
        if (lane < 2 * JT) {
          const int side = lane / JT, ii = lane % JT;
          const int PP = (side == 0 ? tp : tq) * JT + ii;
          if (PP < np) {
            int p, q;
            pair_of(n, t, PP, p, q);
            const Rot R = make_rot(A[(long long)p * n + p].x, A[(long long)q * n + q].x,
                                   A[(long long)p * n + q]);
            if (side == 0) rp[warp][ii] = R; else rq[warp][ii] = R;
          }
        }
        __syncwarp();
        if (valid) {
          const Rot wq = rq[warp][j];
          const Rot wp = rp[warp][i];
          if (do_a) {
          double2 b0, b1;
          if (wp.ident && wq.ident) {
            b0 = sub ? a01 : a00;
            b1 = sub ? a11 : a10;
          } else {
            // M = A_blk W_Q: m_r0 = cs a_r0 - sn (a_r1 e), m_r1 = sn a_r0 + cs (a_r1 e)
            const double2 u0 = cmul_e(a01, wq.ex, wq.ey), u1 = cmul_e(a11, wq.ex, wq.ey);
            double2 m0, m1;
            if (sub == 0) {
              m0 = lin(wq.cs, a00, -wq.sn, u0);
              m1 = lin(wq.cs, a10, -wq.sn, u1);
            } else {
              m0 = lin(wq.sn, a00, wq.cs, u0);
              m1 = lin(wq.sn, a10, wq.cs, u1);
            }
            // B = W_P^H M: b_0 = cs m0 - sn conj(e) m1, b_1 = sn m0 + cs conj(e) m1
            const double2 v = cmul_ce(m1, wp.ex, wp.ey);
            b0 = lin(wp.cs, m0, -wp.sn, v);
            b1 = lin(wp.sn, m0, wp.cs, v);
          }
          if (P == Q) {  // diagonal entries of a Hermitian matrix are real
            if (sub == 0) b0.y = 0.0; else b1.y = 0.0;
          }
          const int col = sub ? q2 : p2;
          B[(long long)p1 * n + col] = b0;
          B[(long long)q1 * n + col] = b1;
          if (P != Q) {
            B[(long long)col * n + p1] = make_double2(b0.x, -b0.y);
            B[(long long)col * n + q1] = make_double2(b1.x, -b1.y);
          }
          }
          // row `sub` (p1 or q1) of V on columns (p2, q2): V <- V W_Q
          if (!wq.ident) {
            const long long row = (long long)(sub ? q1 : p1) * n;
            const double2 u = cmul_e(v1, wq.ex, wq.ey);
            J.V[row + p2] = lin(wq.cs, v0, -wq.sn, u);
            J.V[row + q2] = lin(wq.sn, v0, wq.cs, u);
          }
        }
      }
      if (!grid_sync(J.gs, epoch)) return;
      cur ^= 1;
    }
    // convergence test: all off-diagonal mass (mode 0) or the coupling between the r
    // largest diagonal entries and the others (mode 1)
    {
      const double2* A = cur ? J.A1 : J.A0;
      if (mode == 1) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.nreal; i += gridDim.x * blockDim.x) {
          const double di = A[(long long)i * n + i].x;
          int rk = 0;
          for (int j = 0; j < J.nreal; ++j) {
            const double dj = A[(long long)j * n + j].x;
            rk += (dj > di) || (dj == di && j < i);
          }
          J.rankd[i] = rk;
        }
        if (!grid_sync(J.gs, epoch)) return;
      }
      double off = 0.0, tot = 0.0;
      for (int row = blockIdx.x; row < n; row += gridDim.x) {
        const bool top_row = (mode == 1 && row < J.nreal) ? (J.rankd[row] < J.r) : false;
        for (int col = threadIdx.x; col < n; col += blockDim.x) {
          const double2 v = A[(long long)row * n + col];
          const double m2 = v.x * v.x + v.y * v.y;
          tot += m2;
          if (mode == 0) {
            if (row != col) off += m2;
          } else if (row < J.nreal && col < J.nreal && top_row != (J.rankd[col] < J.r)) {
            off += m2;
          }
        }
      }
      const double so = dyn_block_sum(off, red);
      const double st = dyn_block_sum(tot, red);
      if (threadIdx.x == 0) {
        J.part[2 * blockIdx.x] = so;
        J.part[2 * blockIdx.x + 1] = st;
      }
      if (!grid_sync(J.gs, epoch)) return;
      if (threadIdx.x == 0) {
        double o = 0.0, d = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
          o += J.part[2 * b];
          d += J.part[2 * b + 1];
        }
        const int done = (o <= J.tol2 * d) ? 1 : 0;
        s_done = done || !(o == o);
        if (blockIdx.x == 0) {
          J.info[0] = sweep + 1;
          J.info[1] = done;
          J.info[2] = cur;
          J.info[3] = mode;
        }
      }
      __syncthreads();
      if (s_done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(J.sweep_total, (unsigned long long)(sweep + 1));
        return;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(J.sweep_total, (unsigned long long)J.max_sweeps);
}

// A (npad x npad) <- G (n x n, row-major) padded with zero rows and columns.  A zero
// pad row never couples (its rotations are the identity) and pad indices are excluded
// from the output ranking.
__global__ void eig_pad_kernel(int n, int npad, const double2* __restrict__ G, double2* __restrict__ A,
                               double2* __restrict__ V, int set_identity) {
  const long long nn = (long long)npad * npad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / npad), j = (int)(e % npad);
    double2 v = make_double2(0.0, 0.0);
    if (i < n && j < n) v = G[(long long)i * n + j];
    A[e] = v;
    if (set_identity) V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}

// C = op(X) Y, complex FP64, n x n row-major; op = identity or conjugate transpose.
__global__ void zgemm_kernel(int n, int conjT, const double2* __restrict__ X,
                             const double2* __restrict__ Y, double2* __restrict__ C) {
  __shared__ double2 sx[16][17], sy[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < n; k0 += 16) {
    const int kx = k0 + tx, ky = k0 + ty;
    double2 xv = make_double2(0.0, 0.0);
    if (row < n && kx < n) {
      if (conjT) {
        const double2 t = X[(long long)kx * n + row];
        xv = make_double2(t.x, -t.y);
      } else {
        xv = X[(long long)row * n + kx];
      }
    }
    sx[ty][tx] = xv;
    sy[ty][tx] = (ky < n && col < n) ? Y[(long long)ky * n + col] : make_double2(0.0, 0.0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = cadd(acc, cmul(sx[ty][k], sy[k][tx]));
    __syncthreads();
  }
  if (row < n && col < n) C[(long long)row * n + col] = acc;
}

__global__ void hermitize_kernel(int n, double2* A) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i > j) continue;
    const double2 a = A[(long long)i * n + j], b = A[(long long)j * n + i];
    const double2 m = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    A[(long long)i * n + j] = m;
    A[(long long)j * n + i] = make_double2(m.x, -m.y);
    if (i == j) A[(long long)i * n + i] = make_double2(m.x, 0.0);
  }
}

// largest |Re|, |Im| of A (non-negative doubles order like their bit patterns)
__global__ void eig_absmax_kernel(long long nn, const double2* __restrict__ A, unsigned long long* amax_bits) {
  double m = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 a = A[e];
    m = fmax(m, fmax(fabs(a.x), fabs(a.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(amax_bits, (unsigned long long)__double_as_longlong(m));
}

// A <- 2^-e A with 2^(e-1) <= max entry < 2^e: the Jacobi sums of squared entries then stay
// far from overflow and underflow whatever the scale of G (rotations are scale-invariant)
__global__ void eig_scale_kernel(long long nn, double2* __restrict__ A, const unsigned long long* amax_bits,
                                 double* scale_out) {
  const double amax = __longlong_as_double((long long)*amax_bits);
  int ex2 = 0;
  if (amax > 0.0 && amax <= 1.7e308) frexp(amax, &ex2);
  const double sc = ldexp(1.0, -ex2);
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = sc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 a = A[e];
    A[e] = make_double2(a.x * sc, a.y * sc);
  }
}

// rank of each eigenvalue (ascending, ties by index), eigenvalue output (undoing the scale)
__global__ void eig_rank_kernel(int n, int npad, const double2* A0, const double2* A1,
                                const int* __restrict__ info, const double* __restrict__ scale,
                                int* __restrict__ rank, double* __restrict__ eig_out) {
  const double2* A = info[2] ? A1 : A0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double li = A[(long long)i * npad + i].x;
  int r = 0;
  for (int j = 0; j < n; ++j) {
    const double lj = A[(long long)j * npad + j].x;
    r += (lj < li) || (lj == li && j < i);
  }
  rank[i] = r;
  if (eig_out) eig_out[r] = li / *scale;
}

// Q[rank_i][a] = V[a][i] for the nr smallest eigenvalues
__global__ void eig_gather_q_kernel(int n, int npad, int nr, const double2* __restrict__ V,
                                    const int* __restrict__ rank, double2* __restrict__ Q) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), a = (int)(e % n);
    const int r = rank[i];
    if (r < nr) Q[(long long)r * n + a] = V[(long long)a * npad + i];
  }
}

hicu_status run_nullspace(hicu_handle* h, int64_t n64, int64_t r, const double* G, double* Q,
                          double* eigvals, int flags, cudaStream_t st) {
  if (n64 < 2 || n64 > 4096) return set_error(h, HICU_ERR_SHAPE, "nullspace: n must be in [2, 4096]");
  if (r <= 0 || r >= n64) return set_error(h, HICU_ERR_RANK, "nullspace: rank must satisfy 0 < r < n");
  const int n = (int)n64;
  // one-cluster solver (shared-memory resident, double-float arithmetic, eig_cluster.cu) or the
  // grid-wide FP64 solver below
  if ((flags & HICU_NULLSPACE_GRID) && (flags & HICU_NULLSPACE_CLUSTER))
    return set_error(h, HICU_ERR_ARG, "nullspace: GRID and CLUSTER both requested");
  int nct = 0;
  if (flags & HICU_NULLSPACE_CLUSTER) {
    nct = cluster_eig_ctas(n);
    if (!nct) return set_error(h, HICU_ERR_UNSUPPORTED, "nullspace: no cluster solver for this n on this device");
  } else if (!(flags & HICU_NULLSPACE_GRID) && n <= h->auto_cluster_max) {
    nct = cluster_eig_ctas(n);
  }
  const int npad = nct ? cluster_eig_npad(n, nct) : (n + 1) / 2 * 2;
  const long long nn = (long long)npad * npad;
  hicu_status s = HICU_OK;
  double2* A0 = (double2*)ws_get(h, WS_EIG_A0, sizeof(double2) * nn, &s);
  if (s) return s;
  double2* A1 = (double2*)ws_get(h, WS_EIG_A1, sizeof(double2) * nn, &s);
  if (s) return s;
  double2* V = (double2*)ws_get(h, WS_EIG_V, sizeof(double2) * nn, &s);
  if (s) return s;
  double2* Vprev = (double2*)ws_get(h, WS_EIG_VPREV, sizeof(double2) * nn, &s);
  if (s) return s;
  int grid_blocks = 0;
  const int threads = JWARPS * 32;
  {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, threads, 0) != cudaSuccess ||
        per_sm < 1)
      return set_error(h, HICU_ERR_CUDA, "nullspace: occupancy query failed");
    const int ntile = (npad / 2 + JT - 1) / JT;
    const long long ntiles = (long long)ntile * ntile;
    grid_blocks = (int)std::min<long long>(ntiles, (long long)h->num_sms * std::min(per_sm, 1));
    if (grid_blocks < 1) grid_blocks = 1;
  }
  double* part = (double*)ws_get(h, WS_EIG_PART, sizeof(double) * 2 * grid_blocks + 128, &s);
  if (s) return s;
  int* info = (int*)(part + 2 * grid_blocks);                                  // 8 ints
  unsigned long long* amax_bits = (unsigned long long*)(part + 2 * grid_blocks + 4);
  double* scale = part + 2 * grid_blocks + 5;
  int* rank = (int*)ws_get(h, WS_EIG_TMP, sizeof(int) * 2 * npad, &s);
  if (s) return s;
  int* rankd = rank + npad;

  const bool use_warm = (flags & 1) && h->eig_have_v && h->eig_n == n && h->eig_npad == npad;
  int blocks = (int)std::min<long long>((nn + 255) / 256, 4096);
  if (!use_warm) {
    HICU_LAUNCH(h, K_MISC, st, eig_pad_kernel<<<blocks, 256, 0, st>>>(n, npad, (const double2*)G, A0, V, 1));
  } else {
    // A0 = Vprev^H (G Vprev); V = Vprev
    HICU_LAUNCH(h, K_MISC, st, eig_pad_kernel<<<blocks, 256, 0, st>>>(n, npad, (const double2*)G, A1, V, 0));
    dim3 gg((npad + 15) / 16, (npad + 15) / 16), bb(16, 16);
    // the pad columns of Vprev are pad unit vectors, so the product keeps the pad rows zero
    HICU_LAUNCH(h, K_MISC, st, zgemm_kernel<<<gg, bb, 0, st>>>(npad, 0, A1, Vprev, A0));  // A0 = A Vprev
    HICU_LAUNCH(h, K_MISC, st, zgemm_kernel<<<gg, bb, 0, st>>>(npad, 1, Vprev, A0, A1));  // A1 = Vprev^H A0
    HICU_LAUNCH(h, K_MISC, st, hermitize_kernel<<<blocks, 256, 0, st>>>(npad, A1));
    cudaMemcpyAsync(A0, A1, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(V, Vprev, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st);
  }
  s = cuda_error(h, cudaGetLastError(), "nullspace prep");
  if (s) return s;
  if (nct) {
    s = run_nullspace_cluster(h, n, npad, nct, r, A0, V, V, Q, eigvals, flags, st);
    if (s) return s;
    cudaMemcpyAsync(Vprev, V, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st);
    s = cuda_error(h, cudaGetLastError(), "nullspace output");
    if (s) return s;
    h->eig_have_v = true;
    h->eig_n = n;
    h->eig_npad = npad;
    return HICU_OK;
  }
  cudaMemsetAsync(h->dev_sync, 0, 2 * sizeof(unsigned), st);
  cudaMemsetAsync(info, 0, 8 * sizeof(int) + 16, st);  // info, amax bits
  {
    const int sb = (int)std::min<long long>((nn + 255) / 256, (long long)h->num_sms * 8);
    HICU_LAUNCH(h, K_MISC, st, eig_absmax_kernel<<<sb, 256, 0, st>>>(nn, A0, amax_bits));
    HICU_LAUNCH(h, K_MISC, st, eig_scale_kernel<<<sb, 256, 0, st>>>(nn, A0, amax_bits, scale));
  }
  JacArgs J;
  J.n = npad;
  J.A0 = A0;
  J.A1 = A1;
  J.V = V;
  J.part = part;
  J.info = info;
  J.max_sweeps = 40;
  // full decomposition: off-diagonal mass <= (1e-11 ||A||_F)^2.  Split criterion: coupling between
  // the top-r and the other diagonal entries <= (1e-8 ||A||_F)^2, which bounds the angle of the null
  // space by 1e-8 ||G|| / gap (the eigen-solve in FP32 changes the reconstruction by ~1e-6 NRMSE)
  J.tol2 = (flags & 2) ? 1e-16 : 1e-22;
  J.mode = (flags & 2) ? 1 : 0;
  J.nreal = n;
  J.r = (int)r;
  J.rankd = rankd;
  J.sweep_total = reinterpret_cast<unsigned long long*>(h->dev_err + 8);
  J.gs.count = h->dev_sync;
  J.gs.gen = h->dev_sync + 1;
  J.gs.err = h->dev_err;
  J.gs.nblocks = (unsigned)grid_blocks;
  J.gs.timeout_ns = 2000000000ull;  // 2 s per wait
  void* args[] = {&J};
  cudaError_t e;
  if (h->coop_mu) {  // batch lane: on the shared high-priority stream, in order
    std::lock_guard<std::mutex> lock(*h->coop_mu);
    e = cudaEventRecord(h->coop_in, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->coop_st, h->coop_in, 0);
    if (e == cudaSuccess)
      HICU_LAUNCH(h, K_EIG, h->coop_st,
                  e = cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(grid_blocks), dim3(threads),
                                                  args, 0, h->coop_st));
    if (e == cudaSuccess) e = cudaEventRecord(h->coop_out, h->coop_st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->coop_out, 0);
  } else {
    HICU_LAUNCH(h, K_EIG, st,
                e = cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(grid_blocks), dim3(threads),
                                                args, 0, st));
  }
  if (e != cudaSuccess) return cuda_error(h, e, "nullspace jacobi launch");
  HICU_LAUNCH(h, K_MISC, st, eig_rank_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, npad, A0, A1, info, scale, rank, eigvals));
  HICU_LAUNCH(h, K_MISC, st, eig_gather_q_kernel<<<blocks, 256, 0, st>>>(n, npad, n - (int)r, V, rank, (double2*)Q));
  cudaMemcpyAsync(Vprev, V, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st);
  s = cuda_error(h, cudaGetLastError(), "nullspace output");
  if (s) return s;
  h->eig_have_v = true;
  h->eig_n = n;
  h->eig_npad = npad;
  h->eig_info = info;
  return HICU_OK;
}

}  // namespace hicu
