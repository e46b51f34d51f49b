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
};

__device__ __forceinline__ Rot make_rot(double a, double c, double2 b) {
  Rot R;
  const double ab = hypot(b.x, b.y);
  if (!(ab > 0.0)) {
    R.cs = 1.0; R.sn = 0.0; R.ex = 1.0; R.ey = 0.0;
    return R;
  }
  const double tau = (c - a) / (2.0 * ab);
  double t;
  if (fabs(tau) > 1e150) t = 0.5 / tau;
  else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  const double cs = 1.0 / sqrt(1.0 + t * t);
  R.cs = cs;
  R.sn = t * cs;
  R.ex = b.x / ab;
  R.ey = -b.y / ab;
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
  int* info;     // [0] sweeps, [1] converged, [2] buffer holding the result
  int max_sweeps;
  double tol2;
  int T;  // tile side in pairs, blockDim.x == T*T
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

__global__ void __launch_bounds__(256) jacobi_kernel(JacArgs J) {
  __shared__ Rot rp[16], rq[16];
  __shared__ int ip[16], iq[16], jp[16], jq[16];
  __shared__ double red[8];
  __shared__ int s_done;
  const int n = J.n, np = n / 2, T = J.T;
  const int ntile = (np + T - 1) / T;
  const long long ntiles = (long long)ntile * ntile;
  int cur = 0;
  for (int sweep = 0; sweep < J.max_sweeps; ++sweep) {
    for (int t = 0; t < n - 1; ++t) {
      const double2* A = cur ? J.A1 : J.A0;
      double2* B = cur ? J.A0 : J.A1;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tp = (int)(tile / ntile), tq = (int)(tile % ntile);
        __syncthreads();
        if (threadIdx.x < 2 * T) {
          const int side = threadIdx.x / T, i = threadIdx.x % T;
          const int P = (side == 0 ? tp : tq) * T + i;
          if (P < np) {
            int p, q;
            pair_of(n, t, P, p, q);
            const Rot R = make_rot(A[(long long)p * n + p].x, A[(long long)q * n + q].x,
                                   A[(long long)p * n + q]);
            if (side == 0) { rp[i] = R; ip[i] = p; iq[i] = q; }
            else { rq[i] = R; jp[i] = p; jq[i] = q; }
          }
        }
        __syncthreads();
        const int i = threadIdx.x / T, j = threadIdx.x % T;
        const int P = tp * T + i, Q = tq * T + j;
        if (P < np && Q < np) {
          const int p1 = ip[i], q1 = iq[i], p2 = jp[j], q2 = jq[j];
          double2 u00, u01, u10, u11, w00, w01, w10, w11;
          rot_entries(rp[i], u00, u01, u10, u11);
          rot_entries(rq[j], w00, w01, w10, w11);
          const double2 a00 = A[(long long)p1 * n + p2], a01 = A[(long long)p1 * n + q2];
          const double2 a10 = A[(long long)q1 * n + p2], a11 = A[(long long)q1 * n + q2];
          // M = A_blk W_Q
          const double2 m00 = cadd(cmul(a00, w00), cmul(a01, w10));
          const double2 m01 = cadd(cmul(a00, w01), cmul(a01, w11));
          const double2 m10 = cadd(cmul(a10, w00), cmul(a11, w10));
          const double2 m11 = cadd(cmul(a10, w01), cmul(a11, w11));
          // B_blk = W_P^H M
          double2 b00 = cadd(cmulc(u00, m00), cmulc(u10, m10));
          double2 b01 = cadd(cmulc(u00, m01), cmulc(u10, m11));
          double2 b10 = cadd(cmulc(u01, m00), cmulc(u11, m10));
          double2 b11 = cadd(cmulc(u01, m01), cmulc(u11, m11));
          if (P == Q) {
            b01 = make_double2(0.0, 0.0);
            b10 = make_double2(0.0, 0.0);
            b00.y = 0.0;
            b11.y = 0.0;
          }
          B[(long long)p1 * n + p2] = b00;
          B[(long long)p1 * n + q2] = b01;
          B[(long long)q1 * n + p2] = b10;
          B[(long long)q1 * n + q2] = b11;
          // V <- V W on columns (p2, q2), rows p1 and q1
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            const long long row = (long long)(rr ? q1 : p1) * n;
            const double2 v0 = J.V[row + p2], v1 = J.V[row + q2];
            J.V[row + p2] = cadd(cmul(v0, w00), cmul(v1, w10));
            J.V[row + q2] = cadd(cmul(v0, w01), cmul(v1, w11));
          }
        }
      }
      if (!grid_sync(J.gs)) return;
      cur ^= 1;
    }
    // convergence test on the current matrix
    {
      const double2* A = cur ? J.A1 : J.A0;
      double off = 0.0, dia = 0.0;
      const long long nn = (long long)n * n;
      for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
           e += (long long)gridDim.x * blockDim.x) {
        const double2 v = A[e];
        const double m2 = v.x * v.x + v.y * v.y;
        if (e / n == e % n) dia += m2; else off += m2;
      }
      const double so = dyn_block_sum(off, red);
      const double sd = dyn_block_sum(dia, red);
      if (threadIdx.x == 0) {
        J.part[2 * blockIdx.x] = so;
        J.part[2 * blockIdx.x + 1] = sd;
      }
      if (!grid_sync(J.gs)) return;
      if (threadIdx.x == 0) {
        double o = 0.0, d = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
          o += J.part[2 * b];
          d += J.part[2 * b + 1];
        }
        const int done = (o <= J.tol2 * (o + d)) ? 1 : 0;
        s_done = done || !(o == o);
        if (blockIdx.x == 0) {
          J.info[0] = sweep + 1;
          J.info[1] = done;
          J.info[2] = cur;
        }
      }
      __syncthreads();
      if (s_done) return;
    }
  }
}

// A (npad x npad) <- G (n x n, row-major) padded with a zero row and column when n
// is odd.  A zero pad row never couples (its rotations are the identity) and the
// pad index is excluded from the output ranking.
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

// rank of each eigenvalue (ascending, ties by index), eigenvalue output
__global__ void eig_rank_kernel(int n, int npad, const double2* A0, const double2* A1,
                                const int* __restrict__ info, int* __restrict__ rank,
                                double* __restrict__ eig_out) {
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
  if (eig_out) eig_out[r] = li;
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
                          double* eigvals, int warm, cudaStream_t st) {
  if (n64 < 2 || n64 > 4096) return set_error(h, HICU_ERR_SHAPE, "nullspace: n must be in [2, 4096]");
  if (r <= 0 || r >= n64) return set_error(h, HICU_ERR_RANK, "nullspace: rank must satisfy 0 < r < n");
  const int n = (int)n64;
  const int npad = (n + 1) / 2 * 2;
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
  int T = (npad / 2 >= 12 * 16) ? 16 : 8;
  const int threads = T * T;
  {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, threads, 0) != cudaSuccess ||
        per_sm < 1)
      return set_error(h, HICU_ERR_CUDA, "nullspace: occupancy query failed");
    const int ntile = (npad / 2 + T - 1) / T;
    const long long ntiles = (long long)ntile * ntile;
    grid_blocks = (int)std::min<long long>(ntiles, (long long)h->num_sms * std::min(per_sm, 1));
    if (grid_blocks < 1) grid_blocks = 1;
  }
  double* part = (double*)ws_get(h, WS_EIG_PART, sizeof(double) * 2 * grid_blocks + 64, &s);
  if (s) return s;
  int* info = (int*)(part + 2 * grid_blocks);
  int* rank = (int*)ws_get(h, WS_EIG_TMP, sizeof(int) * npad, &s);
  if (s) return s;

  const bool use_warm = warm && h->eig_have_v && h->eig_n == n;
  int blocks = (int)std::min<long long>((nn + 255) / 256, 4096);
  if (!use_warm) {
    eig_pad_kernel<<<blocks, 256, 0, st>>>(n, npad, (const double2*)G, A0, V, 1);
  } else {
    // A0 = Vprev^H (G Vprev); V = Vprev
    eig_pad_kernel<<<blocks, 256, 0, st>>>(n, npad, (const double2*)G, A1, V, 0);
    dim3 gg((npad + 15) / 16, (npad + 15) / 16), bb(16, 16);
    // the pad column of Vprev is the pad unit vector, so the product keeps the pad row zero
    zgemm_kernel<<<gg, bb, 0, st>>>(npad, 0, A1, Vprev, A0);       // A0 = A Vprev
    zgemm_kernel<<<gg, bb, 0, st>>>(npad, 1, Vprev, A0, A1);       // A1 = Vprev^H A0
    hermitize_kernel<<<blocks, 256, 0, st>>>(npad, A1);
    cudaMemcpyAsync(A0, A1, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(V, Vprev, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st);
  }
  s = cuda_error(h, cudaGetLastError(), "nullspace prep");
  if (s) return s;
  cudaMemsetAsync(h->dev_sync, 0, 2 * sizeof(unsigned), st);
  cudaMemsetAsync(info, 0, 4 * sizeof(int), st);
  JacArgs J;
  J.n = npad;
  J.A0 = A0;
  J.A1 = A1;
  J.V = V;
  J.part = part;
  J.info = info;
  J.max_sweeps = 40;
  J.tol2 = 1e-26;
  J.T = T;
  J.gs.count = h->dev_sync;
  J.gs.gen = h->dev_sync + 1;
  J.gs.err = h->dev_err;
  J.gs.nblocks = (unsigned)grid_blocks;
  J.gs.timeout_ns = 2000000000ull;  // 2 s per wait
  void* args[] = {&J};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(grid_blocks),
                                              dim3(threads), args, 0, st);
  if (e != cudaSuccess) return cuda_error(h, e, "nullspace jacobi launch");
  eig_rank_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, npad, A0, A1, info, rank, eigvals);
  eig_gather_q_kernel<<<blocks, 256, 0, st>>>(n, npad, n - (int)r, V, rank, (double2*)Q);
  cudaMemcpyAsync(Vprev, V, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st);
  s = cuda_error(h, cudaGetLastError(), "nullspace output");
  if (s) return s;
  h->eig_have_v = true;
  h->eig_n = n;
  return HICU_OK;
}

}  // namespace hicu
