// Principal subspace of the Gram matrix by Householder tridiagonalisation (Algorithm 1
// steps 2-3 in Gram form: V = the r principal right singular vectors of H, i.e. the
// eigenvectors of G = H^H H for its r largest eigenvalues; the null space is their
// orthogonal complement).
//
// Method (Golub & Van Loan, 4th ed., sections 8.3.1, 8.4.1 and 8.4.2):
//  1. G = Q_H T Q_H^H with T real symmetric tridiagonal: n - 1 Householder steps
//     H_k = I - tau_k v_k v_k^H, each making the part of column k below the
//     subdiagonal vanish with a real subdiagonal entry.  One cooperative kernel;
//     every CTA forms v_k itself from row k (G is Hermitian and kept in full), then
//     w = tau A v on its own rows, one grid barrier, the symmetric rank-2 update
//     A <- A - v w^H - w v^H of its own rows (w corrected by -tau/2 (w^H v) v), and a
//     second barrier.
//  2. Eigenvalues of T by bisection on Sturm counts (the LDL^T pivot recurrence,
//     Kahan's form, which is backward stable), eight points per eigenvalue and round.
//  3. Eigenvectors of T for the r largest eigenvalues by inverse iteration with a
//     pivoted tridiagonal LU; eigenvalues closer than 1e-10 ||T|| are solved one after
//     the other and orthogonalised against each other (modified Gram-Schmidt).
//  4. V = Q_H Z: the reflectors applied to each eigenvector, last one first.
// The input is pre-scaled by an exact power of two, so no intermediate overflows or
// underflows whatever the scale of G.  Accuracy: eigenvalues to ~eps ||G|| (absolute),
// span(V) to ~eps ||G|| / gap (the Davis-Kahan bound of any backward-stable method).
#include <algorithm>

#include "hicu_internal.cuh"

namespace hicu {

constexpr int TD_THREADS = 256;
constexpr int BS_LANES = 8;  // bisection points per eigenvalue and round

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

struct TdArgs {
  int n;
  double2* A;      // n x n row-major, scaled copy of G (overwritten)
  double* d;       // n   diagonal of T
  double* e;       // n-1 subdiagonal of T
  double2* refl;   // n x n: row k holds v_k (v_k[0] = 1, length n-k-1)
  double2* tau;    // n-1
  double2* w;      // n   scratch (w0 = tau A v)
  double2* part;   // gridDim.x partial sums w0^H v
  GridSync gs;
};

__device__ inline double block_sum_bcast(double v, double* sh) {
  // sum over the CTA, result in every thread (two __syncthreads)
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(TD_THREADS) tridiag_kernel(const TdArgs a) {
  extern __shared__ double2 tsm[];
  double2* v = tsm;          // [n]
  double2* w = tsm + a.n;    // [n]
  __shared__ double red[TD_THREADS / 32];
  __shared__ double2 hh[2];  // tau, alpha
  __shared__ double hbeta;
  const int n = a.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = TD_THREADS / 32;
  const int G = gridDim.x, c = blockIdx.x;
  unsigned epoch = 0;
  for (int k = 0; k < n - 1; ++k) {
    const int m = n - k - 1;
    const double2* rowk = a.A + (long long)k * n + (k + 1);
    // --- the Householder vector of column k (every CTA, from row k)
    double s2 = 0.0;
    for (int j = tid; j < m; j += TD_THREADS) {
      const double2 x = zconj(rowk[j]);
      v[j] = x;
      if (j > 0) s2 += x.x * x.x + x.y * x.y;
    }
    const double xn2 = block_sum_bcast(s2, red);
    if (tid == 0) {
      const double2 x0 = v[0];
      double2 t = make_double2(0.0, 0.0), scale = make_double2(0.0, 0.0);
      double beta = x0.x;
      if (!(xn2 == 0.0 && x0.y == 0.0)) {
        beta = -copysign(sqrt(x0.x * x0.x + x0.y * x0.y + xn2), x0.x);
        t = make_double2((beta - x0.x) / beta, -x0.y / beta);
        const double2 den = make_double2(x0.x - beta, x0.y);  // v = x / (x0 - beta)
        const double dd = den.x * den.x + den.y * den.y;
        scale = make_double2(den.x / dd, -den.y / dd);
      }
      hh[0] = t;
      hh[1] = scale;
      hbeta = beta;
      if (c == 0) {
        a.d[k] = a.A[(long long)k * n + k].x;
        a.e[k] = beta;
        a.tau[k] = t;
      }
    }
    __syncthreads();
    const double2 tau = hh[0], scale = hh[1];
    const bool active = !(tau.x == 0.0 && tau.y == 0.0);
    for (int j = tid; j < m; j += TD_THREADS) {
      const double2 vj = j == 0 ? make_double2(1.0, 0.0) : (active ? zmul(v[j], scale) : make_double2(0.0, 0.0));
      v[j] = vj;
      if (c == 0) a.refl[(long long)k * n + j] = vj;
    }
    __syncthreads();
    // --- w0 = tau A v on this CTA's rows (row i of the trailing block is owned by CTA i mod G)
    double2 pp = make_double2(0.0, 0.0);
    if (active) {
      for (int i = c + G * warp; i < m; i += G * nw) {
        const double2* row = a.A + (long long)(k + 1 + i) * n + (k + 1);
        double2 y = make_double2(0.0, 0.0);
        for (int j = lane; j < m; j += 32) {
          const double2 aij = row[j], vj = v[j];
          y.x += aij.x * vj.x - aij.y * vj.y;
          y.y += aij.x * vj.y + aij.y * vj.x;
        }
        for (int o = 16; o > 0; o >>= 1) {
          y.x += __shfl_down_sync(0xffffffffu, y.x, o);
          y.y += __shfl_down_sync(0xffffffffu, y.y, o);
        }
        if (lane == 0) {
          const double2 w0 = zmul(tau, y);
          a.w[i] = w0;
          const double2 cv = zmul(zconj(w0), v[i]);
          pp.x += cv.x;
          pp.y += cv.y;
        }
      }
    }
    {
      const double px = block_sum_bcast(pp.x, red);
      const double py = block_sum_bcast(pp.y, red);
      if (tid == 0) a.part[c] = make_double2(px, py);
    }
    if (!grid_sync(a.gs, epoch)) return;
    // --- alpha = -tau/2 (w0^H v); w = w0 + alpha v; rank-2 update of this CTA's rows
    if (active) {
      double sx = 0.0, sy = 0.0;
      for (int q = tid; q < G; q += TD_THREADS) {
        const double2 pq = a.part[q];
        sx += pq.x;
        sy += pq.y;
      }
      sx = block_sum_bcast(sx, red);
      sy = block_sum_bcast(sy, red);
      const double2 alpha = zmul(make_double2(-0.5 * tau.x, -0.5 * tau.y), make_double2(sx, sy));
      for (int j = tid; j < m; j += TD_THREADS) {
        const double2 w0 = a.w[j], vj = v[j];
        w[j] = make_double2(w0.x + alpha.x * vj.x - alpha.y * vj.y, w0.y + alpha.x * vj.y + alpha.y * vj.x);
      }
      __syncthreads();
      for (int i = c + G * warp; i < m; i += G * nw) {
        double2* row = a.A + (long long)(k + 1 + i) * n + (k + 1);
        const double2 vi = v[i], wi = w[i];
        for (int j = lane; j < m; j += 32) {
          const double2 vj = v[j], wj = w[j];
          // A_ij -= v_i conj(w_j) + w_i conj(v_j)
          const double2 t1 = zmul(vi, zconj(wj)), t2 = zmul(wi, zconj(vj));
          double2 aij = row[j];
          aij.x -= t1.x + t2.x;
          aij.y -= t1.y + t2.y;
          row[j] = aij;
        }
      }
    }
    if (!grid_sync(a.gs, epoch)) return;
  }
  if (c == 0 && tid == 0) a.d[n - 1] = a.A[(long long)(n - 1) * n + (n - 1)].x;
}

// Gershgorin interval of T, its norm bound and the pivot floor: info[0..3] = lo, hi, tnorm, pivmin
__global__ void td_bounds_kernel(int n, const double* __restrict__ d, const double* __restrict__ e,
                                 double* __restrict__ info) {
  __shared__ double s_lo[256], s_hi[256], s_e2[256];
  double lo = 1e308, hi = -1e308, e2m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double el = i > 0 ? fabs(e[i - 1]) : 0.0, er = i < n - 1 ? fabs(e[i]) : 0.0;
    lo = fmin(lo, d[i] - el - er);
    hi = fmax(hi, d[i] + el + er);
    if (i < n - 1) e2m = fmax(e2m, e[i] * e[i]);
  }
  s_lo[threadIdx.x] = lo;
  s_hi[threadIdx.x] = hi;
  s_e2[threadIdx.x] = e2m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s_lo[threadIdx.x] = fmin(s_lo[threadIdx.x], s_lo[threadIdx.x + o]);
      s_hi[threadIdx.x] = fmax(s_hi[threadIdx.x], s_hi[threadIdx.x + o]);
      s_e2[threadIdx.x] = fmax(s_e2[threadIdx.x], s_e2[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tn = fmax(fabs(s_lo[0]), fabs(s_hi[0]));
    const double pivmin = 1e-290 * fmax(1.0, s_e2[0]);
    const double eps = 0x1.0p-52;
    info[0] = s_lo[0] - 4.0 * eps * tn - 2.0 * pivmin;
    info[1] = s_hi[0] + 4.0 * eps * tn + 2.0 * pivmin;
    info[2] = tn;
    info[3] = pivmin;
  }
}

// number of eigenvalues of T below x (Sturm count on the LDL^T pivots)
__device__ __forceinline__ int sturm_count(int n, const double* __restrict__ d, const double* __restrict__ e,
                                           double x, double pivmin) {
  double q = d[0] - x;
  if (fabs(q) <= pivmin) q = -pivmin;
  int cnt = q < 0.0;
  for (int i = 1; i < n; ++i) {
    const double ei = e[i - 1];
    q = (d[i] - x) - ei * ei / q;
    if (fabs(q) <= pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// Eigenvalue t0 + g (ascending order) for every group g of BS_LANES lanes: multisection to an
// absolute width of 2 eps ||T||.  lam_out[g] = eigenvalue / scale.
__global__ void td_bisect_kernel(int n, int t0, int count, const double* __restrict__ d, const double* __restrict__ e,
                                 const double* __restrict__ info, const double* __restrict__ scale,
                                 double* __restrict__ lam_scaled, double* __restrict__ lam_out) {
  const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / BS_LANES;
  const int sub = threadIdx.x % BS_LANES;
  const unsigned gmask = ((1u << BS_LANES) - 1u) << ((threadIdx.x & 31) / BS_LANES * BS_LANES);
  if (gid >= count) return;  // whole groups leave together (count is per group)
  const int t = t0 + gid;
  double lo = info[0], hi = info[1];
  const double tol = 2.0 * 0x1.0p-52 * info[2] + info[3];
  const double pivmin = info[3];
  for (int it = 0; it < 64 && hi - lo > tol; ++it) {
    const double step = (hi - lo) / (BS_LANES + 1);
    const double x = lo + step * (sub + 1);
    const int cnt = sturm_count(n, d, e, x, pivmin);
    // the first point whose count exceeds t bounds the eigenvalue from above
    const unsigned above = __ballot_sync(gmask, cnt > t) & gmask;
    const int first = above ? (__ffs(above) - 1) % BS_LANES : BS_LANES;
    const double nlo = first == 0 ? lo : lo + step * first;
    const double nhi = first == BS_LANES ? hi : lo + step * (first + 1);
    lo = nlo;
    hi = nhi;
  }
  if (sub == 0) {
    const double l = 0.5 * (lo + hi);
    if (lam_scaled) lam_scaled[gid] = l;
    if (lam_out) lam_out[gid] = l / *scale;
  }
}

__device__ __forceinline__ double hash_unit(uint64_t t, uint64_t i) {
  uint64_t z = t * 0x9E3779B97F4A7C15ull + i * 0xBF58476D1CE4E5B9ull + 1ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
}

// Eigenvectors of T for lam[0..r) (ascending) by inverse iteration; Z[j] (length n, real, unit).
// A thread owns a run of eigenvalues closer than 1e-10 ||T|| (the first of the run does the work)
// and orthogonalises each new vector against the earlier ones of its run.  work: 5 n doubles per
// thread (the pivoted LU of T - lam I).
__global__ void td_inviter_kernel(int n, int r, const double* __restrict__ d, const double* __restrict__ e,
                                  const double* __restrict__ lam, const double* __restrict__ info,
                                  double* __restrict__ work, double* __restrict__ Z) {
  const int j0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (j0 >= r) return;
  const double tnorm = info[2];
  const double ctol = 1e-10 * tnorm;
  if (j0 > 0 && lam[j0] - lam[j0 - 1] < ctol) return;  // not the first of its run
  int j1 = j0 + 1;
  while (j1 < r && lam[j1] - lam[j1 - 1] < ctol) ++j1;
  double* u1 = work + (size_t)j0 * 5 * n;
  double* u2 = u1 + n;
  double* u3 = u2 + n;
  double* lm = u3 + n;
  double* sw = lm + n;  // 1.0: rows i, i+1 swapped at step i
  const double tiny = 0x1.0p-52 * tnorm + info[3];
  for (int j = j0; j < j1; ++j) {
    const double lj = lam[j];
    // pivoted LU of T - lj I
    double ca = d[0] - lj, cc = n > 1 ? e[0] : 0.0;
    for (int i = 0; i < n - 1; ++i) {
      const double b = e[i];
      const double na = d[i + 1] - lj, nc = (i + 1 < n - 1) ? e[i + 1] : 0.0;
      if (fabs(ca) >= fabs(b)) {
        const double piv = fabs(ca) > tiny ? ca : (ca >= 0.0 ? tiny : -tiny);
        const double l = b / piv;
        lm[i] = l;
        sw[i] = 0.0;
        u1[i] = piv;
        u2[i] = cc;
        u3[i] = 0.0;
        ca = na - l * cc;
        cc = nc;
      } else {
        const double l = ca / b;
        lm[i] = l;
        sw[i] = 1.0;
        u1[i] = b;
        u2[i] = na;
        u3[i] = nc;
        ca = cc - l * na;
        cc = -l * nc;
      }
    }
    u1[n - 1] = fabs(ca) > tiny ? ca : (ca >= 0.0 ? tiny : -tiny);
    double* z = Z + (size_t)j * n;
    for (int i = 0; i < n; ++i) z[i] = hash_unit((uint64_t)(j + 1), (uint64_t)i);
    for (int iter = 0; iter < 3; ++iter) {
      // forward: row swaps and L
      for (int i = 0; i < n - 1; ++i) {
        double zi = z[i], zn = z[i + 1];
        if (sw[i] != 0.0) {
          const double t = zi;
          zi = zn;
          zn = t;
        }
        z[i] = zi;
        z[i + 1] = zn - lm[i] * zi;
      }
      // back substitution with U (diagonals u1, u2, u3)
      double x1 = 0.0, x2 = 0.0;  // x[i+1], x[i+2]
      double nrm = 0.0;
      for (int i = n - 1; i >= 0; --i) {
        double s = z[i];
        if (i + 1 < n) s -= u2[i] * x1;
        if (i + 2 < n) s -= u3[i] * x2;
        const double xi = s / u1[i];
        z[i] = xi;
        x2 = x1;
        x1 = xi;
      }
      for (int q = j0; q < j; ++q) {  // modified Gram-Schmidt against the run's earlier vectors
        const double* p = Z + (size_t)q * n;
        double dp = 0.0;
        for (int i = 0; i < n; ++i) dp += p[i] * z[i];
        for (int i = 0; i < n; ++i) z[i] -= dp * p[i];
      }
      for (int i = 0; i < n; ++i) nrm += z[i] * z[i];
      // scale by a power of two first (the solve can grow by ~1 / tiny), then normalise
      int ex = 0;
      frexp(sqrt(nrm), &ex);
      const double p2 = ldexp(1.0, -ex);
      nrm = 0.0;
      for (int i = 0; i < n; ++i) {
        z[i] *= p2;
        nrm += z[i] * z[i];
      }
      const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
      for (int i = 0; i < n; ++i) z[i] *= inv;
    }
  }
}

// V[j] = Q_H z_j = H_0 (H_1 (... H_{n-2} z_j)), one CTA per eigenvector, complex128 rows of length n
__global__ void __launch_bounds__(TD_THREADS) td_backxform_kernel(int n, int r, const double2* __restrict__ refl,
                                                                 const double2* __restrict__ tau,
                                                                 const double* __restrict__ Z,
                                                                 double2* __restrict__ V) {
  extern __shared__ double2 u[];
  __shared__ double red[TD_THREADS / 32];
  const int j = blockIdx.x;
  if (j >= r) return;
  for (int i = threadIdx.x; i < n; i += TD_THREADS) u[i] = make_double2(Z[(size_t)j * n + i], 0.0);
  __syncthreads();
  for (int k = n - 2; k >= 0; --k) {
    const int m = n - k - 1;
    const double2 tk = tau[k];
    if (tk.x == 0.0 && tk.y == 0.0) continue;
    const double2* vk = refl + (size_t)k * n;
    double sx = 0.0, sy = 0.0;
    for (int i = threadIdx.x; i < m; i += TD_THREADS) {
      const double2 vi = vk[i], ui = u[k + 1 + i];
      sx += vi.x * ui.x + vi.y * ui.y;  // conj(v) u
      sy += vi.x * ui.y - vi.y * ui.x;
    }
    sx = block_sum_bcast(sx, red);
    sy = block_sum_bcast(sy, red);
    const double2 ts = zmul(tk, make_double2(sx, sy));
    for (int i = threadIdx.x; i < m; i += TD_THREADS) {
      const double2 vi = vk[i];
      double2 ui = u[k + 1 + i];
      ui.x -= ts.x * vi.x - ts.y * vi.y;
      ui.y -= ts.x * vi.y + ts.y * vi.x;
      u[k + 1 + i] = ui;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += TD_THREADS) V[(size_t)j * n + i] = u[i];
}

// J = trace(G) - sum of the top r eigenvalues (the tail energy of Eq. 1); trace in FP64
__global__ void td_tail_kernel(int n, int r, const double2* __restrict__ G, const double* __restrict__ lam_top,
                               double* __restrict__ J) {
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

__global__ void td_copy_kernel(long long nn, const double2* __restrict__ in, double2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
    out[i] = in[i];
}

hicu_status run_principal(hicu_handle* h, int64_t n64, int64_t r64, const double* Gd, double* Vout,
                          double* eig_top, double* eig_all, double* J, cudaStream_t st) {
  if (n64 < 2 || n64 > 4096) return set_error(h, HICU_ERR_SHAPE, "principal subspace: n must be in [2, 4096]");
  if (r64 <= 0 || r64 >= n64) return set_error(h, HICU_ERR_RANK, "principal subspace: rank must satisfy 0 < r < n");
  const int n = (int)n64, r = (int)r64;
  const long long nn = (long long)n * n;
  const double2* G = (const double2*)Gd;
  hicu_status s = HICU_OK;
  double2* A = (double2*)ws_get(h, WS_EIG_A0, sizeof(double2) * nn, &s);
  if (s) return s;
  double2* refl = (double2*)ws_get(h, WS_EIG_A1, sizeof(double2) * nn, &s);
  if (s) return s;
  // small vectors: d, e, info(8), scale/amax(2), tau, w, part, lam (n), Z (r n), LU work (5 r n)
  const size_t nsm = (size_t)std::max(1, h->num_sms);
  const size_t small = (size_t)n * 2 + 16 + 2 * (size_t)n * 2 + nsm * 2 + (size_t)n;
  double* buf = (double*)ws_get(h, WS_EIG_V, sizeof(double) * (small + 6 * (size_t)r * n), &s);
  if (s) return s;
  double* d = buf;
  double* e = d + n;
  double* info = e + n;          // 8
  unsigned long long* amax_bits = (unsigned long long*)(info + 8);
  double* scale = info + 9;
  double2* tau = (double2*)(info + 16);
  double2* w = tau + n;
  double2* part = w + n;
  double* lam = (double*)(part + nsm);
  double* Z = lam + n;
  double* work = Z + (size_t)r * n;

  // scaled copy of G
  const int eb = (int)std::min<long long>((nn + 255) / 256, (long long)h->num_sms * 8);
  cudaMemsetAsync(amax_bits, 0, sizeof(unsigned long long), st);
  HICU_LAUNCH(h, K_EIG, st, td_copy_kernel<<<eb, 256, 0, st>>>(nn, G, A));
  HICU_LAUNCH(h, K_EIG, st, eig_absmax_kernel<<<eb, 256, 0, st>>>(nn, A, amax_bits));
  HICU_LAUNCH(h, K_EIG, st, eig_scale_kernel<<<eb, 256, 0, st>>>(nn, A, amax_bits, scale));

  // 1. tridiagonalisation (cooperative)
  TdArgs a;
  a.n = n;
  a.A = A;
  a.d = d;
  a.e = e;
  a.refl = refl;
  a.tau = tau;
  a.w = w;
  a.part = part;
  const size_t smem = sizeof(double2) * 2 * (size_t)n;
  int grid = std::min(h->num_sms, std::max(1, (n + 3) / 4));
  {
    static_assert(TD_THREADS == 256, "");
    cudaError_t e0 = allow_max_dynamic_smem((const void*)tridiag_kernel);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "tridiag smem");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_kernel, TD_THREADS, smem) != cudaSuccess ||
        per_sm < 1)
      return set_error(h, HICU_ERR_CUDA, "principal subspace: occupancy query failed");
    grid = std::min(grid, h->num_sms * per_sm);
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
      HICU_LAUNCH(h, K_EIG, h->coop_st,
                  ce = cudaLaunchCooperativeKernel((const void*)tridiag_kernel, dim3(grid), dim3(TD_THREADS), args,
                                                   smem, h->coop_st));
    if (ce == cudaSuccess) ce = cudaEventRecord(h->coop_out, h->coop_st);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, h->coop_out, 0);
  } else {
    HICU_LAUNCH(h, K_EIG, st,
                ce = cudaLaunchCooperativeKernel((const void*)tridiag_kernel, dim3(grid), dim3(TD_THREADS), args,
                                                 smem, st));
  }
  if (ce != cudaSuccess) return cuda_error(h, ce, "principal subspace: tridiagonalisation launch");

  // 2. eigenvalues (top r; all n when requested)
  HICU_LAUNCH(h, K_EIG, st, td_bounds_kernel<<<1, 256, 0, st>>>(n, d, e, info));
  {
    const int thr = 64;
    const int blocks = (r * BS_LANES + thr - 1) / thr;
    HICU_LAUNCH(h, K_EIG, st,
                td_bisect_kernel<<<blocks, thr, 0, st>>>(n, n - r, r, d, e, info, scale, lam, eig_top));
    if (eig_all) {
      const int ball = (n * BS_LANES + thr - 1) / thr;
      HICU_LAUNCH(h, K_EIG, st,
                  td_bisect_kernel<<<ball, thr, 0, st>>>(n, 0, n, d, e, info, scale, nullptr, eig_all));
    }
  }
  // 3. eigenvectors of T, 4. back-transformation
  HICU_LAUNCH(h, K_EIG, st, td_inviter_kernel<<<(r + 31) / 32, 32, 0, st>>>(n, r, d, e, lam, info, work, Z));
  {
    const size_t usm = sizeof(double2) * (size_t)n;
    cudaError_t e0 = allow_max_dynamic_smem((const void*)td_backxform_kernel);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "backxform smem");
    HICU_LAUNCH(h, K_EIG, st,
                td_backxform_kernel<<<r, TD_THREADS, usm, st>>>(n, r, refl, tau, Z, (double2*)Vout));
  }
  if (J) HICU_LAUNCH(h, K_MISC, st, td_tail_kernel<<<1, 256, 0, st>>>(n, r, G, eig_top, J));
  return cuda_error(h, cudaGetLastError(), "principal subspace");
}

}  // namespace hicu
