// Gram matrix G = H(x)^H H(x) of the multi-level Hankel matrix (Eq. 1; the
// Discussion names SVD of this Gram matrix as the alternative to rSVD),
// computed as multi-coil cross-correlation without forming H.
//
// Entry ((c1,d1),(c2,d2)) = sum_{u in W(d1)} conj(x_c1[u]) x_c2[u + delta],
// delta = d2 - d1, W(d) = {p + d : p a valid output}.  For one (c1, c2, delta)
// all windows W(d) are unions of the same few "cells": along each valid axis
// the cut points {0..k-1} and {L..L+k-1} (L = ext - k + 1) split the region
// into at most 2k-1 intervals; a circular axis is one cell.  So
//   1. gram_cells: one CTA per (task = (c1, c2, delta), row piece) forms the
//      products once per region point and sums them per cell, and
//   2. gram_assemble: each G entry adds the cells of its window.
// Hermitian symmetry halves the tasks: (c1 < c2) or (c1 == c2, delta >= 0).
//
// Accuracy: products of FP32 inputs are formed exactly (fmaf error term) and
// accumulated in double-word (float pair) arithmetic per thread, then summed
// across threads, cells and CTAs in double-float (df.cuh) in a fixed order
// (deterministic); only the finished entries are converted to FP64 (FP64
// arithmetic on this GPU is 1/58 of the FP32 rate).
#include <algorithm>
#include <vector>

#include "df.cuh"
#include "hicu_internal.cuh"

namespace hicu {

constexpr int GMAXCUT = 34;
constexpr int GMAXPIECE = 64;
constexpr int GXSLOT = 4;

struct GramParams {
  ConvGeom g;
  KView x;
  int ncx, ncy, ncz;
  int cutx[GMAXCUT], cuty[GMAXCUT], cutz[GMAXCUT];
  int npy, npz;
  int py0[GMAXPIECE], py1[GMAXPIECE], pyc[GMAXPIECE];
  int pz0[GMAXPIECE], pz1[GMAXPIECE], pzc[GMAXPIECE];
  int lx, ly, lz, nl, nlh, center;
  const int* sup;  // kernel mask: box offset of support offset j (nullptr: the whole box)
  int nk;          // offsets per coil in G's index (|K|, or kx ky kz)
};

// conj(a) b added to the double-word sums of its real and imaginary parts: per component the
// value is hi + lo.  Each real product is formed exactly (p plus its fma error term e), p enters
// the sum through a two-sum and the rounding errors of both go to lo; the sums are renormalised
// after every complex product.  The paired FP32 instructions of sm_100 and later (__fmul2_rn,
// __fadd2_rn, __ffma2_rn, two independent IEEE round-to-nearest operations each) carry the real and
// the imaginary sum together, which halves the instructions the kernels issue: the first pair of
// products is (ar br, ar bi), the second (ai bi, -ai br).  A difference x - y is formed as
// fma(y, -1, x), which rounds the same exact value once, and the error term as RN(p - a b) from the
// negated factor, which is -e exactly; so each component goes through the same rounded operations,
// in the same order, as a scalar two-sum accumulation, and the pairing does not change the sums.
__device__ __forceinline__ void dd_acc2(float2 a, float2 na, float2 b, float2& hi, float2& lo) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 p = __fmul2_rn(a, b);
  const float2 ne = __ffma2_rn(na, b, p);            // p - a b = -e, exact
  const float2 s = __fadd2_rn(hi, p);                // two-sum(hi, p) = s + err
  const float2 bb = __ffma2_rn(hi, m1, s);           // s - hi
  const float2 err = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, m1, s), m1, hi), __ffma2_rn(bb, m1, p));
  hi = s;
  lo = __fadd2_rn(lo, __ffma2_rn(ne, m1, err));      // lo + (err + e)
}

__device__ __forceinline__ void dd_renorm2(float2& hi, float2& lo) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 s = __fadd2_rn(hi, lo);
  lo = __ffma2_rn(__ffma2_rn(hi, m1, s), m1, lo);    // lo - (s - hi)
  hi = s;
}

__device__ __forceinline__ void cmac_dd2(float2 a, float2 b, float2& hi, float2& lo) {
  dd_acc2(make_float2(a.x, a.x), make_float2(-a.x, -a.x), b, hi, lo);
  dd_acc2(make_float2(a.y, -a.y), make_float2(-a.y, a.y), make_float2(b.y, b.x), hi, lo);
  dd_renorm2(hi, lo);
}

__host__ __device__ inline void decode_task(long long t, int C, int nl, int nlh, int center, int& c1,
                                            int& c2, int& l) {
  for (c1 = 0; c1 < C; ++c1) {
    const long long sz = nlh + (long long)(C - 1 - c1) * nl;
    if (t < sz) break;
    t -= sz;
  }
  if (t < nlh) {
    c2 = c1;
    l = center + (int)t;
  } else {
    t -= nlh;
    c2 = c1 + 1 + (int)(t / nl);
    l = (int)(t % nl);
  }
}

__host__ __device__ inline long long task_index(int c1, int c2, int l, int C, int nl, int nlh,
                                                int center) {
  const long long base =
      (long long)c1 * nlh + (long long)nl * ((long long)c1 * (C - 1) - (long long)c1 * (c1 - 1) / 2);
  if (c1 == c2) return base + (l - center);
  return base + nlh + (long long)(c2 - c1 - 1) * nl + l;
}

__global__ void __launch_bounds__(256) gram_cells_kernel(GramParams P, float4* __restrict__ part) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  __shared__ float4 vals[256 * GXSLOT];
  const ConvGeom& g = P.g;
  const long long task = blockIdx.x;
  const int piece = blockIdx.y;
  const int pyi = piece % P.npy, pzi = piece / P.npy;
  int c1, c2, l;
  decode_task(task, g.C, P.nl, P.nlh, P.center, c1, c2, l);
  const int ddx = l % P.lx - (g.kx - 1);
  const int ddy = (l / P.lx) % P.ly - (g.ky - 1);
  const int ddz = l / (P.lx * P.ly) - (g.kz - 1);
  const float2* xa = P.x.p + (long long)c1 * P.x.sc;
  const float2* xb = P.x.p + (long long)c2 * P.x.sc;
  const int nt = blockDim.x;

  float2 sh[GXSLOT], sl[GXSLOT];   // (re, im) double-word sums: hi, lo
  int bx[GXSLOT];
  bool bok[GXSLOT];
#pragma unroll
  for (int j = 0; j < GXSLOT; ++j) {
    sh[j] = sl[j] = make_float2(0.f, 0.f);
    const int xx = threadIdx.x + j * nt;
    int vx = xx + ddx;
    bool ok = xx < g.ex;
    if (g.cx) vx = wrap(vx, g.ex); else ok = ok && vx >= 0 && vx < g.ex;
    bx[j] = vx;
    bok[j] = ok;
  }
  for (int z = P.pz0[pzi]; z < P.pz1[pzi]; ++z) {
    int vz = z + ddz;
    if (g.cz) vz = wrap(vz, g.ez);
    else if (vz < 0 || vz >= g.ez) continue;
    for (int y = P.py0[pyi]; y < P.py1[pyi]; ++y) {
      int vy = y + ddy;
      if (g.cy) vy = wrap(vy, g.ey);
      else if (vy < 0 || vy >= g.ey) continue;
      const float2* arow = xa + (long long)(P.x.oz + z) * P.x.sz + (long long)(P.x.oy + y) * P.x.sy + P.x.ox;
      const float2* brow = xb + (long long)(P.x.oz + vz) * P.x.sz + (long long)(P.x.oy + vy) * P.x.sy + P.x.ox;
#pragma unroll
      for (int j = 0; j < GXSLOT; ++j) {
        if (bok[j]) {
          const float2 a = arow[threadIdx.x + j * nt];
          const float2 b = brow[bx[j]];
          cmac_dd2(a, b, sh[j], sl[j]);   // conj(a) * b = (ar br + ai bi) + i (ar bi - ai br)
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < GXSLOT; ++j) {
    const int xx = threadIdx.x + j * nt;
    if (xx < g.ex) vals[xx] = make_float4(sh[j].x, sl[j].x, sh[j].y, sl[j].y);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = nt >> 5;
  for (int ci = warp; ci < P.ncx; ci += nw) {
    cdf acc = c_zero();
    for (int xx = P.cutx[ci] + lane; xx < P.cutx[ci + 1]; xx += 32) {
      // zero-product cells (shifted sample outside S) were never written: skip them
      const int vx = xx + ddx;
      if (!g.cx && (vx < 0 || vx >= g.ex)) continue;
      acc = c_add(acc, ld4(&vals[xx]));
    }
    acc = c_warp_sum(acc);
    if (lane == 0) st4(&part[(task * (P.npy * P.npz) + piece) * P.ncx + ci], acc);
  }
}

// Row-streaming form for regions up to 256 positions wide: a CTA per (task, z piece), a thread
// per x position.  The CTA walks every row of its planes in order; a thread keeps one
// double-word accumulator for the y cell it is in and, when the row enters the next y cell,
// adds it into that cell's slot of a shared [y cell][x] buffer (its own column: no other thread
// writes it).  At the end the x cells of every y cell are summed (single-position x cells are
// copied, the interior cell by a warp reduction) into the same partial layout as
// gram_cells_kernel with one y piece per y cell.  The border rows, one-row cells, no longer cost a
// CTA and an x reduction each.  Dynamic shared memory: ncy * ex float4.
__global__ void gram_rows_kernel(GramParams P, float4* __restrict__ part) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  extern __shared__ float4 cellbuf[];  // [ncy][ex]
  const ConvGeom& g = P.g;
  const long long task = blockIdx.x;
  const int pzi = blockIdx.y;
  int c1, c2, l;
  decode_task(task, g.C, P.nl, P.nlh, P.center, c1, c2, l);
  const int ddx = l % P.lx - (g.kx - 1);
  const int ddy = (l / P.lx) % P.ly - (g.ky - 1);
  const int ddz = l / (P.lx * P.ly) - (g.kz - 1);
  const float2* xa = P.x.p + (long long)c1 * P.x.sc;
  const float2* xb = P.x.p + (long long)c2 * P.x.sc;
  const int xx = threadIdx.x;
  int vx = xx + ddx;
  bool ok = xx < g.ex;
  if (g.cx) vx = wrap(vx, g.ex);
  else ok = ok && vx >= 0 && vx < g.ex;
  if (xx < g.ex)
    for (int c = 0; c < P.ncy; ++c) cellbuf[c * g.ex + xx] = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 sh = make_float2(0.f, 0.f), sl = sh;   // (re, im) double-word sums: hi, lo
  int cell = -1;
  auto flush = [&]() {
    if (cell >= 0 && xx < g.ex) {
      float4* slot = &cellbuf[cell * g.ex + xx];
      const cdf sum = c_add(ld4(slot), cdf{{sh.x, sl.x}, {sh.y, sl.y}});
      st4(slot, sum);
    }
    sh = sl = make_float2(0.f, 0.f);
  };
  for (int z = P.pz0[pzi]; z < P.pz1[pzi]; ++z) {
    int vz = z + ddz;
    if (g.cz) vz = wrap(vz, g.ez);
    else if (vz < 0 || vz >= g.ez) continue;
    int cy = 0;
    for (int y = 0; y < g.ey; ++y) {
      while (P.cuty[cy + 1] <= y) ++cy;
      if (cy != cell) {
        flush();
        cell = cy;
      }
      int vy = y + ddy;
      if (g.cy) vy = wrap(vy, g.ey);
      else if (vy < 0 || vy >= g.ey) continue;
      if (ok) {
        const float2 a = xa[(long long)(P.x.oz + z) * P.x.sz + (long long)(P.x.oy + y) * P.x.sy + P.x.ox + xx];
        const float2 b = xb[(long long)(P.x.oz + vz) * P.x.sz + (long long)(P.x.oy + vy) * P.x.sy + P.x.ox + vx];
        cmac_dd2(a, b, sh, sl);   // conj(a) * b = (ar br + ai bi) + i (ar bi - ai br)
      }
    }
  }
  flush();
  __syncthreads();
  // x cells of every y cell
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const long long base = (task * (P.npy * P.npz) + (long long)pzi * P.npy) * P.ncx;
  for (int cyi = warp; cyi < P.ncy; cyi += nw) {
    const float4* row = cellbuf + cyi * g.ex;
    float4* out = part + base + (long long)cyi * P.ncx;
    for (int ci = 0; ci < P.ncx; ++ci) {
      const int x0 = P.cutx[ci], x1 = P.cutx[ci + 1];
      if (x1 - x0 == 1) {
        if (lane == 0) out[ci] = row[x0];
        continue;
      }
      cdf acc = c_zero();
      for (int x = x0 + lane; x < x1; x += 32) acc = c_add(acc, ld4(&row[x]));
      acc = c_warp_sum(acc);
      if (lane == 0) st4(&out[ci], acc);
    }
  }
}

// Lag-row form for regions up to 128 positions wide and kernels up to 5 wide in x and y: a CTA per
// (coil pair, y lag, z lag, z piece) and a thread per x position forms the products of one sample
// of coil c1 with the 2 kx - 1 samples of coil c2 at all x lags, so every loaded sample feeds
// 2 kx - 1 products and the row and index arithmetic is shared by them.  The y cells are split
// between two kinds of CTA (blockIdx.z): kind 0 sums the interior y cell, its rows spread over the
// CTA's row groups; kind 1 sums the single-row border cells, one row at a time per row group.  So
// every accumulator lives in registers for the whole CTA; the cells of x and the row groups are
// summed once at the end through shared memory.  The partial sums go to the same layout as
// gram_rows_kernel (y pieces = y cells), read by gram_assemble_kernel.
struct LagRowParams {
  int xw, rgroups;       // threads per row (= ex), row groups (blockDim = xw * rgroups rounded up to 32)
  int ly, nyz, cyz;      // y lags, y-z lags, centre y-z lag
  int y_lo, y_hi;        // interior y cell [y_lo, y_hi) (all rows for a circular y axis)
  int cy_int;            // its y cell index
  int nb;                // border rows (single-row y cells)
  int brow[2 * GMAXCUT]; // their rows
  int bcell[2 * GMAXCUT];// and y cell indices
};

__host__ __device__ inline void decode_task9(long long t, int C, int nyz, int cyz, int& c1, int& c2, int& lyz) {
  for (c1 = 0; c1 < C; ++c1) {
    const long long sz = (nyz - cyz) + (long long)(C - 1 - c1) * nyz;
    if (t < sz) break;
    t -= sz;
  }
  if (t < nyz - cyz) {
    c2 = c1;
    lyz = cyz + (int)t;
  } else {
    t -= nyz - cyz;
    c2 = c1 + 1 + (int)(t / nyz);
    lyz = (int)(t % nyz);
  }
}

// Three CTAs per SM (80 registers a thread; shared memory allows three CTAs of the knee-size case
// too): left to its own choice the compiler takes 99 registers, two CTAs fit, and the Gram of a
// 64 x 64 x 40 x 8 region takes 11 % longer.
template <int LX>
__global__ void __launch_bounds__(256, 3) gram_lagrow_kernel(GramParams P, LagRowParams Q, float4* __restrict__ part) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  extern __shared__ float4 red[];  // kind 0: [rgroups][LX][xw]; kind 1: [nb][LX][xw]
  const ConvGeom& g = P.g;
  const int kind = blockIdx.z;
  if (kind == 1 && Q.nb == 0) return;
  int c1, c2, lyz;
  decode_task9(blockIdx.x, g.C, Q.nyz, Q.cyz, c1, c2, lyz);
  const int pzi = blockIdx.y;
  const int ddy = lyz % Q.ly - (g.ky - 1);
  const int ddz = lyz / Q.ly - (g.kz - 1);
  const int x = threadIdx.x % Q.xw, rg = threadIdx.x / Q.xw;
  const bool active = rg < Q.rgroups;   // the block is rounded up to whole warps
  const float2* xa = P.x.p + (long long)c1 * P.x.sc + P.x.ox;
  const float2* xb = P.x.p + (long long)c2 * P.x.sc + P.x.ox;
  // x lags: the sample of coil c2 at x + j - (kx - 1).  A lag that leaves a non-circular region
  // reads a clamped sample instead: every cell that ends up in a Gram entry for lag j has all its
  // x + j - (kx - 1) inside the region, so those products only reach cells no entry reads.
  int bx[LX];
#pragma unroll
  for (int j = 0; j < LX; ++j) {
    int vx = x + j - (g.kx - 1);
    if (g.cx) vx = wrap(vx, g.ex);
    else vx = min(max(vx, 0), g.ex - 1);
    bx[j] = vx;
  }
  float2 sh[LX], sl[LX];   // (re, im) double-word sums of x lag j: hi, lo
  auto zero = [&]() {
#pragma unroll
    for (int j = 0; j < LX; ++j) sh[j] = sl[j] = make_float2(0.f, 0.f);
  };
  // one row pair: a = x_c1[z][y][x], b_j = x_c2[z + ddz][vy][x + j - (kx - 1)]
  auto row = [&](int z, int vz, int y, int vy) {
    const float2* ar = xa + (long long)(P.x.oz + z) * P.x.sz + (long long)(P.x.oy + y) * P.x.sy;
    const float2* br = xb + (long long)(P.x.oz + vz) * P.x.sz + (long long)(P.x.oy + vy) * P.x.sy;
    const float2 a = __ldg(ar + x);
    float2 b[LX];
#pragma unroll
    for (int j = 0; j < LX; ++j) b[j] = __ldg(br + bx[j]);
#pragma unroll
    for (int j = 0; j < LX; ++j) cmac_dd2(a, b[j], sh[j], sl[j]);   // conj(a) * b_j
  };
  auto shifted = [&](int v, int e, bool circ, int& out) -> bool {
    if (circ) { out = wrap(v, e); return true; }
    out = v;
    return v >= 0 && v < e;
  };
  const int z0 = P.pz0[pzi], z1 = P.pz1[pzi];
  if (!active) {
    // idle tail of the last warp: nothing to sum
  } else if (kind == 0) {
    zero();
    for (int z = z0; z < z1; ++z) {
      int vz;
      if (!shifted(z + ddz, g.ez, g.cz, vz)) continue;
      for (int y = Q.y_lo + rg; y < Q.y_hi; y += Q.rgroups) {
        int vy;
        if (!shifted(y + ddy, g.ey, g.cy, vy)) continue;
        row(z, vz, y, vy);
      }
    }
#pragma unroll
    for (int j = 0; j < LX; ++j) red[(rg * LX + j) * Q.xw + x] = make_float4(sh[j].x, sl[j].x, sh[j].y, sl[j].y);
  } else {
    for (int b = rg; b < Q.nb; b += Q.rgroups) {
      zero();
      const int y = Q.brow[b];
      int vy;
      if (shifted(y + ddy, g.ey, g.cy, vy)) {
        for (int z = z0; z < z1; ++z) {
          int vz;
          if (!shifted(z + ddz, g.ez, g.cz, vz)) continue;
          row(z, vz, y, vy);
        }
      }
#pragma unroll
      for (int j = 0; j < LX; ++j) red[(b * LX + j) * Q.xw + x] = make_float4(sh[j].x, sl[j].x, sh[j].y, sl[j].y);
    }
  }
  __syncthreads();
  // cells of x (and the row groups of kind 0): one warp per (set, lag).  Single-position cells
  // (the border columns) are copied lane by lane; only the wide cells take a warp reduction.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nsets = kind == 0 ? 1 : Q.nb;
  const int npieces = P.npy * P.npz;
  const bool diag_centre = (c1 == c2) && (lyz == Q.cyz);
  const int nsum = kind == 0 ? Q.rgroups : 1;
  for (int item = warp; item < nsets * LX; item += nw) {
    const int set = item / LX, j = item % LX;
    if (diag_centre && j < g.kx - 1) continue;   // lag with delta x < 0: its conjugate is stored
    const int l = j + (2 * g.kx - 1) * lyz;
    const long long task = task_index(c1, c2, l, g.C, P.nl, P.nlh, P.center);
    const int cy = kind == 0 ? Q.cy_int : Q.bcell[set];
    float4* out = part + (task * npieces + (long long)pzi * P.npy + cy) * P.ncx;
    const float4* src = red + (size_t)((kind == 0 ? 0 : set) * LX + j) * Q.xw;
    const size_t gstride = (size_t)LX * Q.xw;   // between row groups (kind 0)
    for (int ci = lane; ci < P.ncx; ci += 32) {
      const int x0 = P.cutx[ci];
      if (P.cutx[ci + 1] - x0 != 1) continue;
      cdf acc = ld4(&src[x0]);
      for (int r = 1; r < nsum; ++r) acc = c_add(acc, ld4(&src[r * gstride + x0]));
      st4(&out[ci], acc);
    }
    for (int ci = 0; ci < P.ncx; ++ci) {
      const int x0 = P.cutx[ci], x1 = P.cutx[ci + 1];
      if (x1 - x0 == 1) continue;
      cdf acc = c_zero();
      for (int xx = x0 + lane; xx < x1; xx += 32)
        for (int r = 0; r < nsum; ++r) acc = c_add(acc, ld4(&src[r * gstride + xx]));
      acc = c_warp_sum(acc);
      if (lane == 0) st4(&out[ci], acc);
    }
  }
}

__device__ __forceinline__ int cut_index(const int* cuts, int ncut, int v) {
  for (int i = 0; i < ncut; ++i)
    if (cuts[i] == v) return i;
  return -1;
}

__global__ void gram_assemble_kernel(GramParams P, const float4* __restrict__ part,
                                     double2* __restrict__ G) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  const ConvGeom& g = P.g;
  const int n = g.C * P.nk;   // G over the coefficients of the kernel mask's support
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int a = (int)(idx / n), b = (int)(idx % n);
  const int c1 = a / P.nk, c2 = b / P.nk;
  const int k1 = P.sup ? P.sup[a % P.nk] : a % P.nk, k2 = P.sup ? P.sup[b % P.nk] : b % P.nk;
  const int d1x = k1 % g.kx, d1y = (k1 / g.kx) % g.ky, d1z = k1 / (g.kx * g.ky);
  const int d2x = k2 % g.kx, d2y = (k2 / g.kx) % g.ky, d2z = k2 / (g.kx * g.ky);
  const int l = ((d2z - d1z + g.kz - 1) * P.ly + (d2y - d1y + g.ky - 1)) * P.lx + (d2x - d1x + g.kx - 1);
  const bool direct = (c1 < c2) || (c1 == c2 && l >= P.center);
  int tc1, tc2, tl, wx, wy, wz;
  if (direct) {
    tc1 = c1; tc2 = c2; tl = l; wx = d1x; wy = d1y; wz = d1z;
  } else {
    tc1 = c2; tc2 = c1; tl = P.nl - 1 - l; wx = d2x; wy = d2y; wz = d2z;
  }
  const long long task = task_index(tc1, tc2, tl, g.C, P.nl, P.nlh, P.center);
  int cx0 = 0, cx1 = 1, cy0 = 0, cy1 = 1, cz0 = 0, cz1 = 1;
  if (!g.cx) {
    cx0 = cut_index(P.cutx, P.ncx + 1, wx);
    cx1 = cut_index(P.cutx, P.ncx + 1, wx + g.ex - g.kx + 1);
  }
  if (!g.cy) {
    cy0 = cut_index(P.cuty, P.ncy + 1, wy);
    cy1 = cut_index(P.cuty, P.ncy + 1, wy + g.ey - g.ky + 1);
  }
  if (!g.cz) {
    cz0 = cut_index(P.cutz, P.ncz + 1, wz);
    cz1 = cut_index(P.cutz, P.ncz + 1, wz + g.ez - g.kz + 1);
  }
  if (cx0 < 0 || cx1 < 0 || cy0 < 0 || cy1 < 0 || cz0 < 0 || cz1 < 0) {
    G[idx] = make_double2(nan(""), nan(""));  // unreachable: window ends are always cut points
    return;
  }
  cdf acc = c_zero();
  const int npieces = P.npy * P.npz;
  for (int pz = 0; pz < P.npz; ++pz) {
    if (P.pzc[pz] < cz0 || P.pzc[pz] >= cz1) continue;
    for (int py = 0; py < P.npy; ++py) {
      if (P.pyc[py] < cy0 || P.pyc[py] >= cy1) continue;
      const float4* src = part + (task * npieces + (pz * P.npy + py)) * P.ncx;
      for (int cx = cx0; cx < cx1; ++cx) acc = c_add(acc, ld4(&src[cx]));
    }
  }
  const double sr = df_to(acc.re), si = df_to(acc.im);
  G[idx] = direct ? make_double2(sr, si) : make_double2(sr, -si);
}

// ------------------------------------------------------------------ host

static int build_cuts(int ext, int k, bool circular, int* cuts) {
  std::vector<int> v;
  if (circular) {
    v = {0, ext};
  } else {
    const int L = ext - k + 1;
    for (int i = 0; i < k; ++i) v.push_back(i);
    for (int i = 0; i < k; ++i) v.push_back(L + i);
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  for (size_t i = 0; i < v.size(); ++i) cuts[i] = v[i];
  return (int)v.size() - 1;  // number of cells
}

static int build_pieces(const int* cuts, int ncell, int* p0, int* p1, int* pc) {
  int total = cuts[ncell] - cuts[0];
  for (int len = std::max(8, (total + 31) / 32);; len *= 2) {
    int np = 0;
    bool fit = true;
    for (int c = 0; c < ncell && fit; ++c) {
      for (int s = cuts[c]; s < cuts[c + 1]; s += len) {
        if (np >= GMAXPIECE) { fit = false; break; }
        p0[np] = s;
        p1[np] = std::min(s + len, cuts[c + 1]);
        pc[np] = c;
        ++np;
      }
    }
    if (fit) return np;
  }
}

hicu_status run_gram(hicu_handle* h, const hicu_geom* geom, const hicu_region* reg, const float* x,
                     double* G, cudaStream_t st, const int* sup, int nk) {
  ConvGeom g;
  hicu_status s = make_conv_geom(h, geom, reg, &g);
  if (s) return s;
  if (g.kx > 16 || g.ky > 16 || g.kz > 16)
    return set_error(h, HICU_ERR_UNSUPPORTED, "gram: kernel extent above 16");
  if (g.ex > 256 * GXSLOT) return set_error(h, HICU_ERR_UNSUPPORTED, "gram: region x extent above 1024");
  GramParams P;
  P.g = g;
  P.sup = sup;
  P.nk = sup ? nk : g.K;
  P.x = full_view(geom, reg, const_cast<float*>(x));
  P.ncx = build_cuts(g.ex, g.kx, g.cx, P.cutx);
  P.ncy = build_cuts(g.ey, g.ky, g.cy, P.cuty);
  P.ncz = build_cuts(g.ez, g.kz, g.cz, P.cutz);
  P.npy = build_pieces(P.cuty, P.ncy, P.py0, P.py1, P.pyc);
  P.npz = build_pieces(P.cutz, P.ncz, P.pz0, P.pz1, P.pzc);
  P.lx = 2 * g.kx - 1;
  P.ly = 2 * g.ky - 1;
  P.lz = 2 * g.kz - 1;
  P.nl = P.lx * P.ly * P.lz;
  P.nlh = (P.nl + 1) / 2;
  P.center = (P.nl - 1) / 2;
  const long long ntasks = (long long)g.C * P.nlh + (long long)P.nl * ((long long)g.C * (g.C - 1) / 2);
  // row-streaming kernel when a thread per x position fits one CTA and the [y cell][x] buffer
  // fits shared memory; its y pieces are the y cells
  const size_t rows_smem = sizeof(float4) * (size_t)P.ncy * g.ex;
  const bool rows_form = g.ex <= 256 && rows_smem <= 96 * 1024;
  if (rows_form) {
    P.npy = P.ncy;
    for (int c = 0; c < P.ncy; ++c) {
      P.py0[c] = P.cuty[c];
      P.py1[c] = P.cuty[c + 1];
      P.pyc[c] = c;
    }
  }
  // lag-row form: every x lag of a (coil pair, y lag, z lag) task in one thread (kx, ky <= 5,
  // ex <= 128); the interior y cell and the single-row border cells of y go to two kinds of CTA
  LagRowParams Q;
  bool lagrow = rows_form && g.kx <= 5 && g.ky <= 5 && g.ex <= 128;
  if (lagrow) {
    Q.xw = g.ex;
    Q.rgroups = std::max(1, 256 / g.ex);
    Q.ly = P.ly;
    Q.nyz = P.ly * P.lz;
    Q.cyz = (Q.nyz - 1) / 2;
    int big = 0;
    for (int c = 0; c < P.ncy; ++c)
      if (P.cuty[c + 1] - P.cuty[c] > P.cuty[big + 1] - P.cuty[big]) big = c;
    Q.y_lo = P.cuty[big];
    Q.y_hi = P.cuty[big + 1];
    Q.cy_int = big;
    Q.nb = 0;
    for (int c = 0; c < P.ncy && lagrow; ++c) {
      if (c == big) continue;
      if (P.cuty[c + 1] - P.cuty[c] != 1 || Q.nb >= 2 * GMAXCUT) {
        lagrow = false;  // more than one multi-row y cell: the row-streaming form
        break;
      }
      Q.brow[Q.nb] = P.cuty[c];
      Q.bcell[Q.nb] = c;
      ++Q.nb;
    }
    if (sizeof(float4) * (size_t)std::max(Q.nb, Q.rgroups) * (2 * g.kx - 1) * Q.xw > 200 * 1024) lagrow = false;
  }
  const int npieces = P.npy * P.npz;
  float4* part = (float4*)ws_get(h, WS_GRAM_PART, sizeof(float4) * ntasks * npieces * P.ncx, &s);
  if (s) return s;
  if (lagrow) {
    const int LX = 2 * g.kx - 1;
    const long long ntask9 = (long long)g.C * (Q.nyz - Q.cyz) + (long long)Q.nyz * ((long long)g.C * (g.C - 1) / 2);
    const size_t smem = sizeof(float4) * (size_t)std::max(Q.nb, Q.rgroups) * LX * Q.xw;
    const int nt = (Q.xw * Q.rgroups + 31) / 32 * 32;
    const dim3 grid((unsigned)ntask9, (unsigned)P.npz, Q.nb > 0 ? 2u : 1u);
    const void* fn = LX == 9 ? (const void*)gram_lagrow_kernel<9> : LX == 7 ? (const void*)gram_lagrow_kernel<7>
                   : LX == 5 ? (const void*)gram_lagrow_kernel<5> : LX == 3 ? (const void*)gram_lagrow_kernel<3>
                   : (const void*)gram_lagrow_kernel<1>;
    const cudaError_t e0 = allow_max_dynamic_smem(fn);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "gram smem");
    switch (LX) {
      case 9: launch_pdl(h, K_GRAM, st, grid, dim3(nt), smem, gram_lagrow_kernel<9>, false, P, Q, part); break;
      case 7: launch_pdl(h, K_GRAM, st, grid, dim3(nt), smem, gram_lagrow_kernel<7>, false, P, Q, part); break;
      case 5: launch_pdl(h, K_GRAM, st, grid, dim3(nt), smem, gram_lagrow_kernel<5>, false, P, Q, part); break;
      case 3: launch_pdl(h, K_GRAM, st, grid, dim3(nt), smem, gram_lagrow_kernel<3>, false, P, Q, part); break;
      default: launch_pdl(h, K_GRAM, st, grid, dim3(nt), smem, gram_lagrow_kernel<1>, false, P, Q, part); break;
    }
    s = cuda_error(h, cudaGetLastError(), "gram_lagrow");
    if (s) return s;
    const long long nn = (long long)g.C * P.nk * g.C * P.nk;
    launch_pdl(h, K_GRAM, st, dim3((unsigned)((nn + 255) / 256)), dim3(256), 0, gram_assemble_kernel, false, P,
               (const float4*)part, (double2*)G);
    return cuda_error(h, cudaGetLastError(), "gram_assemble");
  }
  // stream-ordered (allow = false): as programmatic dependents, CTAs waiting beside the running
  // kernel slowed the Gram by 4-8 % on GB300
  if (rows_form) {
    const int nt = (g.ex + 31) / 32 * 32;
    const cudaError_t e0 = allow_max_dynamic_smem((const void*)gram_rows_kernel);
    if (e0 != cudaSuccess) return cuda_error(h, e0, "gram smem");
    launch_pdl(h, K_GRAM, st, dim3((unsigned)ntasks, (unsigned)P.npz), dim3(nt), rows_smem, gram_rows_kernel, false,
               P, part);
  } else {
    int nt = ((g.ex + GXSLOT - 1) / GXSLOT + 31) / 32 * 32;
    if (nt < 64) nt = 64;
    if (nt > 256) nt = 256;
    launch_pdl(h, K_GRAM, st, dim3((unsigned)ntasks, (unsigned)npieces), dim3(nt), 0, gram_cells_kernel, false, P,
               part);
  }
  s = cuda_error(h, cudaGetLastError(), "gram_cells");
  if (s) return s;
  const long long nn = (long long)g.C * P.nk * g.C * P.nk;
  launch_pdl(h, K_GRAM, st, dim3((unsigned)((nn + 255) / 256)), dim3(256), 0, gram_assemble_kernel, false, P,
             (const float4*)part, (double2*)G);
  return cuda_error(h, cudaGetLastError(), "gram_assemble");
}

}  // namespace hicu
