// Tensor-core (tcgen05, TMEM) split-BF16 forms of the HICU convolutions, 2D.
//
// Both operators are implicit GEMMs over the kernel offsets d (Theory: H(x) v is
// the valid convolution; its conjugate transpose is again a convolution):
//   conv    : R[o, k]   = sum_d sum_c  x_c[o + d] q_k[c, d]          K = 2C, N = 2p
//   adjoint : g_c[u]    = sum_d sum_k  conj(q_k[c, d]) R[u - d, k]   K = 2p, N = 2C
// Complex products run as real MMAs: the A row of a position is (re, im) of every
// channel, and B embeds each complex weight w as [[w.re, w.im], [-w.im, w.re]]
// (conv) or the conjugate embedding (adjoint).  Each FP32 value is split into
// bf16 hi + lo; the MMAs accumulate hi*hi + hi*lo + lo*hi in FP32 (the lo*lo
// term is below the FP32 accumulation error).
//
// Data path per CTA (128 threads, one M-tile = 128 consecutive positions):
//  * the input tile (rows of W positions plus the kernel halo) of every
//    (split, 4-channel chunk) plane is copied from a planar bf16 buffer
//    [split][chunk][Y][X][8] into shared memory with 1D bulk async copies, one
//    per row and plane, completing on an mbarrier;
//  * an offset d shifts the whole M-tile by dy*W + dx positions, i.e. the A
//    descriptor start moves by 16 bytes per position (no-swizzle K-major core
//    matrices are 8 positions x 16 bytes), so no im2col copy is ever made;
//  * one thread issues all MMAs of a K group into per-M-tile TMEM accumulators
//    and commits them to an mbarrier; K groups (pairs of chunks) stream through
//    one shared-memory buffer;
//  * epilogue: tcgen05.ld of each thread's accumulator row, then either R
//    (complex64 and/or split bf16 planes for the adjoint) with ||R||^2, or the
//    masked gradient g with ||g||^2.
// Every mbarrier wait is bounded (tc_ptx.cuh); a timeout skips the remaining
// work, records HICU_ERR_TIMEOUT and still releases TMEM.
#include <algorithm>

#include "hicu_internal.cuh"
#include "tc_ptx.cuh"

namespace hicu {

constexpr int TC_THREADS = 128;
constexpr int TC_SMEM_LIMIT = 220 * 1024;

struct TcParams {
  int kx, ky, K;       // kernel extent and offsets (2D)
  int X, Y;            // planar input extent (positions)
  int W;               // tile width in positions (<= 256)
  int Tx, Ty;          // outputs per tile row, output rows per CTA
  int ntx;             // tiles along x
  int org_x, org_y;    // input coordinate of the tile origin = output origin + (org_x, org_y)
  int chunks;          // 4-channel chunks of the A operand per split
  int groups;          // K groups (each = 2 chunks)
  int Npad;            // MMA N (multiple of 16)
  int Hpos;            // positions per shared-memory plane
  int nM;              // M tiles per CTA
  int tmem_cols;       // allocated TMEM columns (power of two >= nM * Npad)
  int conj_shift;      // 0: conv shift (dy*W + dx); 1: adjoint shift ((ky-1-dy)*W + (kx-1-dx))
  const uint4* ain;    // planar bf16 input, 16 bytes per (plane, position)
  const uint4* bw;     // B planes [group][d][split][2][Npad][8] bf16
  uint32_t bgroup_bytes;
  // outputs
  int mode;            // 0: conv (R and/or ||R||^2), 1: adjoint (masked g and ||g||^2)
  int ox_lim, oy_lim;  // valid output extent
  int p;               // conv: filters; adjoint: coils written
  float2* R;           // conv: complex64 [oy][ox][p] (nullable)
  uint4* Rs;           // conv: split planes of R [split][chunkR][oy_lim][ox_lim] (nullable)
  int chunksR;
  KView gout;          // adjoint: output view (region coordinates)
  MView m;             // adjoint: mask view
  double* partial;
  int* err;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// hi/lo split of 8 floats into two 16-byte bf16 words
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  float h[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    h[i] = __bfloat162float(__float2bfloat16_rn(v[i]));
    l[i] = v[i] - h[i];
  }
  hi = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]),
                  pack_bf16x2(h[6], h[7]));
  lo = make_uint4(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]), pack_bf16x2(l[4], l[5]),
                  pack_bf16x2(l[6], l[7]));
}

__global__ void __launch_bounds__(TC_THREADS, 1) tc_corr_kernel(const TcParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar_load, bar_mma;
  __shared__ uint32_t tslot;
  __shared__ double red[4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile_x = blockIdx.x % P.ntx, tile_y = blockIdx.x / P.ntx;
  const int x0 = tile_x * P.Tx, y0 = tile_y * P.Ty;  // output origin of the tile
  const int ix0 = x0 + P.org_x, iy0 = y0 + P.org_y;  // input origin (may be negative)
  const int rows = P.Ty + P.ky - 1;
  const uint32_t plane_bytes = (uint32_t)P.Hpos * 16u;
  unsigned char* sA = smem;                          // 4 planes: [split][2 chunks]
  unsigned char* sB = smem + 4 * plane_bytes;        // B of one K group

  if (tid == 0) {
    tc::mbar_init(&bar_load, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tslot, (uint32_t)P.tmem_cols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t taddr = tslot;

  // rows / columns of the input tile that exist in the planar buffer
  const int ry0 = max(0, -iy0), ry1 = min(rows, P.Y - iy0);
  const int cx0 = max(0, -ix0), cx1 = min(P.W, P.X - ix0);
  const bool full_tile = ry0 == 0 && ry1 == rows && cx0 == 0 && cx1 == P.W;

  bool ok = true;
  for (int grp = 0; grp < P.groups && ok; ++grp) {
    if (grp > 0) {
      tc::tc_fence_before();
      __syncthreads();  // previous group's MMAs are complete (bar_mma waited); buffer is free
    }
    // zero what the copies will not overwrite: missing rows/columns (adjoint halo) and the
    // padding chunk of an odd chunk count
    const bool pad_chunk = (2 * grp + 1 >= P.chunks);
    if (!full_tile || pad_chunk) {
      const int n16 = (int)(4 * plane_bytes / 16);
      uint4* z = reinterpret_cast<uint4*>(sA);
      for (int i = tid; i < n16; i += TC_THREADS) z[i] = make_uint4(0, 0, 0, 0);
      tc::fence_proxy_async_smem();
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t bytes = P.bgroup_bytes;
      const int ncopy = cx1 - cx0;
      int nplanes = 0;
      for (int cc = 0; cc < 2; ++cc)
        if (2 * grp + cc < P.chunks) ++nplanes;
      if (ry1 > ry0 && ncopy > 0) bytes += (uint32_t)(2 * nplanes * (ry1 - ry0) * ncopy * 16);
      tc::mbar_arrive_expect_tx(&bar_load, bytes);
      tc::bulk_g2s(sB, reinterpret_cast<const unsigned char*>(P.bw) + (size_t)grp * P.bgroup_bytes,
                   P.bgroup_bytes, &bar_load);
      if (ncopy > 0) {
        for (int s = 0; s < 2; ++s) {
          for (int cc = 0; cc < 2; ++cc) {
            const int j = 2 * grp + cc;
            if (j >= P.chunks) continue;
            const uint4* src_plane = P.ain + (size_t)(s * P.chunks + j) * P.Y * P.X;
            unsigned char* dst_plane = sA + (s * 2 + cc) * plane_bytes;
            for (int hy = ry0; hy < ry1; ++hy) {
              const uint4* src = src_plane + (size_t)(iy0 + hy) * P.X + (ix0 + cx0);
              tc::bulk_g2s(dst_plane + ((size_t)hy * P.W + cx0) * 16, src, (uint32_t)(ncopy * 16), &bar_load);
            }
          }
        }
      }
    }
    ok = tc::mbar_wait(&bar_load, grp & 1, P.err);
    ok = __syncthreads_and(ok);
    if (!ok) break;
    // one thread issues the group's MMAs for every M tile
    if (tid == 0) {
      tc::tc_fence_after();
      const uint32_t idesc = tc::idesc_bf16_f32(128, P.Npad);
      const uint32_t a_base = tc::smem_u32(sA), b_base = tc::smem_u32(sB);
      const uint32_t bsplit = 2u * P.Npad * 16u;  // one (d, split) B block: 2 chunk planes
      for (int mt = 0; mt < P.nM; ++mt) {
        const uint32_t dcol = taddr + (uint32_t)(mt * P.Npad);
        int first = (grp == 0);
        for (int dy = 0; dy < P.ky; ++dy) {
          for (int dx = 0; dx < P.kx; ++dx) {
            const int d = dy * P.kx + dx;
            const int shift = P.conj_shift ? (P.ky - 1 - dy) * P.W + (P.kx - 1 - dx) : dy * P.W + dx;
            const uint32_t apos = (uint32_t)(mt * 128 + shift) * 16u;
            const uint64_t a_hi = tc::smem_desc(a_base + apos, plane_bytes, 128);
            const uint64_t a_lo = tc::smem_desc(a_base + 2 * plane_bytes + apos, plane_bytes, 128);
            const uint32_t bd = b_base + (uint32_t)(d * 2) * bsplit;
            const uint64_t b_hi = tc::smem_desc(bd, P.Npad * 16u, 128);
            const uint64_t b_lo = tc::smem_desc(bd + bsplit, P.Npad * 16u, 128);
            tc::mma_bf16(dcol, a_hi, b_hi, idesc, first ? 0u : 1u);
            tc::mma_bf16(dcol, a_hi, b_lo, idesc, 1u);
            tc::mma_bf16(dcol, a_lo, b_hi, idesc, 1u);
            first = 0;
          }
        }
      }
      tc::mma_commit(&bar_mma);
    }
    ok = tc::mbar_wait(&bar_mma, grp & 1, P.err);
    ok = __syncthreads_and(ok);
    tc::tc_fence_after();
  }

  // epilogue: thread (warp, lane) owns accumulator row 32*warp + lane of every M tile.  Squared
  // norms are summed in FP32 per thread (at most a few hundred terms) and in FP64 across threads:
  // FP64 arithmetic runs at 1/58 of the FP32 rate on this part.
  float nrm = 0.f;
  if (ok) {
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    for (int mt = 0; mt < P.nM; ++mt) {
      const int mrow = mt * 128 + 32 * warp + lane;
      const int ly = mrow / P.W, lx = mrow - (mrow / P.W) * P.W;
      const int ox = x0 + lx, oy = y0 + ly;
      const bool valid = ly < P.Ty && lx < P.Tx && ox < P.ox_lim && oy < P.oy_lim;
      for (int c0 = 0; c0 < P.Npad; c0 += 16) {
        uint32_t r[16];
        tc::tmem_ld16(taddr + lane_base + (uint32_t)(mt * P.Npad + c0), r);
        tc::tmem_ld_wait();
        if (!valid) continue;
        if (P.mode == 0) {
          const long long o = (long long)oy * P.ox_lim + ox;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int k = c0 / 2 + q;
            if (k < P.p) {
              const float2 v = make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
              nrm = fmaf(v.x, v.x, fmaf(v.y, v.y, nrm));
              if (P.R) P.R[o * P.p + k] = v;
            }
          }
          if (P.Rs) {
            // two 4-filter chunks per 16 columns: split into bf16 planes for the adjoint
#pragma unroll
            for (int hc = 0; hc < 2; ++hc) {
              const int jr = c0 / 8 + hc;
              if (jr < P.chunksR) {
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                  const int k = jr * 4 + e / 2;
                  v[e] = (k < P.p) ? __uint_as_float(r[hc * 8 + e]) : 0.f;
                }
                uint4 hi, lo;
                split8(v, hi, lo);
                const size_t plane = (size_t)P.oy_lim * P.ox_lim;
                P.Rs[(size_t)jr * plane + o] = hi;
                P.Rs[(size_t)(P.chunksR + jr) * plane + o] = lo;
              }
            }
          }
        } else {
          const long long mo = (long long)(P.m.oz) * P.m.sz + (long long)(P.m.oy + oy) * P.m.sy + (P.m.ox + ox);
          const long long go = (long long)(P.gout.oz) * P.gout.sz + (long long)(P.gout.oy + oy) * P.gout.sy +
                               (P.gout.ox + ox);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int c = c0 / 2 + q;
            if (c < P.p) {
              float2 v = make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
              if (P.m.p && P.m.p[(long long)c * P.m.sc + mo]) v = make_float2(0.f, 0.f);
              P.gout.p[(long long)c * P.gout.sc + go] = v;
              nrm = fmaf(v.x, v.x, fmaf(v.y, v.y, nrm));
            }
          }
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)P.tmem_cols);
  double dn = (double)nrm;
  for (int o = 16; o > 0; o >>= 1) dn += __shfl_down_sync(0xffffffffu, dn, o);
  if (lane == 0) red[warp] = dn;
  __syncthreads();
  if (tid == 0) P.partial[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
}

// ------------------------------------------------------------- layout kernels

// region of a complex64 array -> planar split bf16 [split][chunk][ey][ex][8], chunk = 4 channels
__global__ void tc_split_input_kernel(int C, int ex, int ey, KView x, uint4* __restrict__ out) {
  const int chunks = C / 4;
  const long long plane = (long long)ex * ey;
  const long long tot = plane * chunks;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / plane);
    const long long pos = i - (long long)j * plane;
    const int ux = (int)(pos % ex), uy = (int)(pos / ex);
    float v[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 a = x.p[(long long)(4 * j + e) * x.sc + (long long)(x.oz) * x.sz + (long long)(x.oy + uy) * x.sy +
                           (x.ox + ux)];
      v[2 * e] = a.x;
      v[2 * e + 1] = a.y;
    }
    uint4 hi, lo;
    split8(v, hi, lo);
    out[(long long)j * plane + pos] = hi;
    out[(long long)(chunks + j) * plane + pos] = lo;
  }
}

// R complex64 [s][p] -> planar split bf16 [split][chunkR][s][8], chunk = 4 filters (zero padded)
__global__ void tc_split_r_kernel(long long npos, int p, const float2* __restrict__ R, uint4* __restrict__ out) {
  const int chunks = (p + 3) / 4;
  const long long tot = npos * chunks;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / npos);
    const long long pos = i - (long long)j * npos;
    float v[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 4 * j + e;
      const float2 a = (k < p) ? R[pos * p + k] : make_float2(0.f, 0.f);
      v[2 * e] = a.x;
      v[2 * e + 1] = a.y;
    }
    uint4 hi, lo;
    split8(v, hi, lo);
    out[(long long)j * npos + pos] = hi;
    out[(long long)(chunks + j) * npos + pos] = lo;
  }
}

// B planes [group][d][split][cc][Npad][8] from a bank [p][n] (n = C*K, filter order [c][ky][kx]).
// conv:    K index kk = 2c + t (t: re/im of x), N index = 2k + u:  [[f.re, f.im], [-f.im, f.re]]
// adjoint: K index kk = 2k + t (t: re/im of R), N index = 2c + u:  [[f.re, -f.im], [f.im, f.re]]
__global__ void tc_prep_b_kernel(int mode, int C, int K, int p, int groups, int Npad,
                                 const float2* __restrict__ bank, __nv_bfloat16* __restrict__ out) {
  const long long per_group = (long long)K * 2 * 2 * Npad * 8;
  const long long tot = per_group * groups;
  const int n = C * K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    long long t = i;
    const int e = (int)(t % 8); t /= 8;
    const int col = (int)(t % Npad); t /= Npad;
    const int cc = (int)(t % 2); t /= 2;
    const int split = (int)(t % 2); t /= 2;
    const int d = (int)(t % K); t /= K;
    const int grp = (int)t;
    const int kk = (grp * 2 + cc) * 8 + e;  // K index within the offset
    const int kin = kk >> 1, tin = kk & 1;  // input channel (coil or filter) and re/im
    const int kout = col >> 1, uout = col & 1;
    float w = 0.f;
    int coil, filt;
    if (mode == 0) { coil = kin; filt = kout; }
    else { coil = kout; filt = kin; }
    if (coil < C && filt < p && kout < (mode == 0 ? p : C)) {
      const float2 f = bank[(long long)filt * n + (long long)coil * K + d];
      if (mode == 0) w = (tin == 0) ? (uout == 0 ? f.x : f.y) : (uout == 0 ? -f.y : f.x);
      else w = (tin == 0) ? (uout == 0 ? f.x : -f.y) : (uout == 0 ? f.y : f.x);
    }
    const float hi = __bfloat162float(__float2bfloat16_rn(w));
    out[i] = __float2bfloat16_rn(split == 0 ? hi : w - hi);
  }
}

// ---------------------------------------------------------------- host side

struct TcPlan {
  TcParams P;
  size_t smem;
  int grid;
};

static int pow2_at_least(int v) {
  int p = 32;
  while (p < v) p <<= 1;
  return p;
}

// Tile plan for a valid correlation: output columns are split into the fewest tiles whose halo
// (Tx + kx - 1 positions) fits a 256-position row; the number of output rows per CTA (Ty) is the
// largest that still gives >= 148 CTAs, else the smallest that fills whole M tiles (most CTAs).
static bool tile_fits(const TcParams& P, int Ty, size_t b_bytes, int* Hpos_out, size_t* smem_out) {
  const int nM = (Ty * P.W + 127) / 128;
  if (nM * P.Npad > 512) return false;
  int Hpos = std::max((Ty + P.ky - 1) * P.W, nM * 128 + (P.ky - 1) * P.W + (P.kx - 1));
  Hpos = (Hpos + 7) / 8 * 8;
  const size_t smem = 4 * (size_t)Hpos * 16 + b_bytes;
  if (smem > (size_t)TC_SMEM_LIMIT) return false;
  *Hpos_out = Hpos;
  *smem_out = smem;
  return true;
}

static bool plan_tc(TcPlan* pl, int kx, int ky, int X, int Y, int ox_lim, int oy_lim, int org_x, int org_y,
                    int chunks, int Npad) {
  TcParams& P = pl->P;
  P.kx = kx;
  P.ky = ky;
  P.K = kx * ky;
  P.X = X;
  P.Y = Y;
  P.org_x = org_x;
  P.org_y = org_y;
  P.chunks = chunks;
  P.groups = (chunks + 1) / 2;
  P.Npad = Npad;
  const int maxTx = 256 - (kx - 1);
  P.ntx = (ox_lim + maxTx - 1) / maxTx;
  P.Tx = (ox_lim + P.ntx - 1) / P.ntx;
  P.W = P.Tx + kx - 1;
  const size_t b_bytes = (size_t)P.K * 2 * 2 * Npad * 16;
  P.bgroup_bytes = (uint32_t)b_bytes;
  const int tymax = std::min(oy_lim, 64);
  int chosen = 0, Hpos = 0;
  size_t smem = 0;
  for (int Ty = tymax; Ty >= 1; --Ty) {
    int hp;
    size_t sm;
    if (!tile_fits(P, Ty, b_bytes, &hp, &sm)) continue;
    if (P.ntx * ((oy_lim + Ty - 1) / Ty) >= 148) { chosen = Ty; Hpos = hp; smem = sm; break; }
  }
  if (chosen == 0) {
    const int ty_fill = std::max(1, std::min(tymax, (128 + P.W - 1) / P.W));
    for (int Ty = ty_fill; Ty >= 1; --Ty) {
      int hp;
      size_t sm;
      if (tile_fits(P, Ty, b_bytes, &hp, &sm)) { chosen = Ty; Hpos = hp; smem = sm; break; }
    }
  }
  if (chosen == 0) return false;
  P.Ty = chosen;
  P.nM = (P.Ty * P.W + 127) / 128;
  P.Hpos = Hpos;
  P.tmem_cols = pow2_at_least(P.nM * Npad);
  pl->smem = smem;
  pl->grid = P.ntx * ((oy_lim + P.Ty - 1) / P.Ty);
  P.ox_lim = ox_lim;
  P.oy_lim = oy_lim;
  return P.tmem_cols <= 512;
}

bool tc_supported(const ConvGeom& g) {
  return g.kz == 1 && g.ez == 1 && !g.cx && !g.cy && !g.cz && (g.C % 4) == 0 && g.kx <= 16 && g.ky <= 16;
}

hicu_status tc_prepare_input(hicu_handle* h, const ConvGeom& g, KView x, uint4* planar, cudaStream_t st) {
  const long long tot = (long long)g.ex * g.ey * (g.C / 4);
  int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  HICU_LAUNCH(h, K_MISC, st, tc_split_input_kernel<<<blocks, 256, 0, st>>>(g.C, g.ex, g.ey, x, planar));
  return cuda_error(h, cudaGetLastError(), "tc_split_input");
}

hicu_status tc_prepare_r(hicu_handle* h, const ConvGeom& g, const float2* R, int p, uint4* planar,
                         cudaStream_t st) {
  const long long tot = g.s * ((p + 3) / 4);
  int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  HICU_LAUNCH(h, K_MISC, st, tc_split_r_kernel<<<blocks, 256, 0, st>>>(g.s, p, R, planar));
  return cuda_error(h, cudaGetLastError(), "tc_split_r");
}

size_t tc_b_bytes(const ConvGeom& g, int p, int mode) {
  const int chunks = mode == 0 ? g.C / 4 : (p + 3) / 4;
  const int groups = (chunks + 1) / 2;
  const int Npad = mode == 0 ? (2 * p + 15) / 16 * 16 : (2 * g.C + 15) / 16 * 16;
  return (size_t)groups * g.K * 2 * 2 * Npad * 16;
}

hicu_status tc_prepare_weights(hicu_handle* h, const ConvGeom& g, const float2* bank, int p, int mode,
                               void* out, cudaStream_t st) {
  const int chunks = mode == 0 ? g.C / 4 : (p + 3) / 4;
  const int groups = (chunks + 1) / 2;
  const int Npad = mode == 0 ? (2 * p + 15) / 16 * 16 : (2 * g.C + 15) / 16 * 16;
  const long long tot = (long long)groups * g.K * 2 * 2 * Npad * 8;
  int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  HICU_LAUNCH(h, K_MISC, st,
              tc_prep_b_kernel<<<blocks, 256, 0, st>>>(mode, g.C, g.K, p, groups, Npad, bank,
                                                       (__nv_bfloat16*)out));
  return cuda_error(h, cudaGetLastError(), "tc_prep_b");
}

static hicu_status launch_plan(hicu_handle* h, TcPlan& pl, int cls, cudaStream_t st) {
  const cudaError_t e = allow_max_dynamic_smem((const void*)tc_corr_kernel);
  if (e != cudaSuccess) return cuda_error(h, e, "tc_corr smem");
  HICU_LAUNCH(h, cls, st, tc_corr_kernel<<<pl.grid, TC_THREADS, pl.smem, st>>>(pl.P));
  return cuda_error(h, cudaGetLastError(), "tc_corr");
}

// conv: x planar (region) -> R (complex64 and/or split planes), partial norms per CTA
hicu_status launch_conv_tc(hicu_handle* h, const ConvGeom& g, const uint4* xplanar, const void* bw, int p,
                           float2* R, uint4* Rs, double* partial, int* nblocks, cudaStream_t st) {
  TcPlan pl;
  const int Npad = (2 * p + 15) / 16 * 16;
  if (Npad > 256 || !plan_tc(&pl, g.kx, g.ky, g.ex, g.ey, g.sx, g.sy, 0, 0, g.C / 4, Npad))
    return set_error(h, HICU_ERR_UNSUPPORTED, "split-bf16 conv: tile does not fit shared memory");
  *nblocks = pl.grid;
  if (!partial) return HICU_OK;
  pl.P.conj_shift = 0;
  pl.P.ain = xplanar;
  pl.P.bw = (const uint4*)bw;
  pl.P.mode = 0;
  pl.P.p = p;
  pl.P.R = R;
  pl.P.Rs = Rs;
  pl.P.chunksR = (p + 3) / 4;
  pl.P.partial = partial;
  pl.P.err = h->dev_err;
  pl.P.m.p = nullptr;
  pl.P.gout.p = nullptr;
  return launch_plan(h, pl, K_CONV_TC, st);
}

// adjoint: split planes of R -> masked g (region view), partial norms per CTA
hicu_status launch_adjoint_tc(hicu_handle* h, const ConvGeom& g, const uint4* Rs, const void* bw, int p,
                              MView m, KView gout, double* partial, int* nblocks, cudaStream_t st) {
  TcPlan pl;
  const int Npad = (2 * g.C + 15) / 16 * 16;
  if (Npad > 256 ||
      !plan_tc(&pl, g.kx, g.ky, g.sx, g.sy, g.ex, g.ey, -(g.kx - 1), -(g.ky - 1), (p + 3) / 4, Npad))
    return set_error(h, HICU_ERR_UNSUPPORTED, "split-bf16 adjoint: tile does not fit shared memory");
  *nblocks = pl.grid;
  if (!partial) return HICU_OK;
  pl.P.conj_shift = 1;
  pl.P.ain = Rs;
  pl.P.bw = (const uint4*)bw;
  pl.P.mode = 1;
  pl.P.p = g.C;
  pl.P.R = nullptr;
  pl.P.Rs = nullptr;
  pl.P.chunksR = 0;
  pl.P.gout = gout;
  pl.P.m = m;
  pl.P.partial = partial;
  pl.P.err = h->dev_err;
  return launch_plan(h, pl, K_ADJOINT_TC, st);
}

}  // namespace hicu
