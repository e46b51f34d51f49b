// Tensor-core (tcgen05, TMEM) split-BF16 forms of the HICU convolutions, 2D and 3D.
//
// Both operators are implicit GEMMs over the kernel offsets d (Theory: H(x) v is
// the valid convolution; its conjugate transpose is again a convolution):
//   conv    : R[o, k]   = sum_d sum_c  x_c[o + d] q_k[c, d]
//   adjoint : g_c[u]    = sum_d sum_k  conj(q_k[c, d]) R[u - d, k]
// The adjoint is run as a correlation of R (origin shifted by -(k-1) per axis)
// with the flipped conjugate filters, so one kernel serves both.  Complex
// products run as real MMAs: an A row holds (re, im) of 8 input channels (one
// K = 16 step), and B embeds each complex weight w as [[w.re, w.im], [-w.im,
// w.re]].  Each FP32 value is split into bf16 hi + lo; B is stored as [B_hi |
// B_lo] along N, so two MMAs (A_hi and A_lo against [B_hi | B_lo]) form all
// four products in FP32 accumulators, summed in the epilogue.
//
// Streaming along the outer axis.  A problem is seen as planes (z) of rows (y)
// of positions (x); a 2D problem runs with its rows as planes.  One work unit
// is (8 output channels, a run of L output planes, Ty rows, one x tile).  The
// CTA walks the input planes v of the run once: input plane v contributes to
// output planes v - dz for every kernel offset dz, so one MMA multiplies the A
// tile of plane v with the weights of all kz offsets at once (N = 32 kz) and
// writes the kz output planes' accumulators, which sit side by side in a ring
// of TMEM slots.  This keeps N wide for small filter banks (p = 8 gives N =
// 160 for kz = 5) instead of re-reading the A tile once per z offset.
//
// Roles (192 threads): warp 0 lane 0 issues TMA tensor loads (5D tensor map,
// out-of-range boxes are zero-filled, which supplies the adjoint's halo) into a
// ring of shared-memory stages; warp 1 lane 0 issues the MMAs and commits each
// stage back to the producer and each finished output plane to the epilogue;
// warps 2-5 drain finished planes from TMEM (tcgen05.ld), zero the slot again
// (tcgen05.st; the whole ring is zeroed at the start, so every MMA accumulates),
// write R / the masked gradient and accumulate squared norms.  The filter bank of
// the unit's output-channel group stays resident in shared memory.  The grid is
// persistent (one CTA per SM, static unit schedule), so results are
// deterministic.  Every mbarrier wait is bounded (tc_ptx.cuh): on a timeout the
// role records HICU_ERR_TIMEOUT and stops, and TMEM is still released.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include <map>
#include <cstring>
#include "hicu_internal.cuh"
#include "tc_ptx.cuh"

namespace hicu {

constexpr int TC_THREADS = 192;
constexpr int TC_MAX_STAGES = 8;
constexpr int TC_SLOT_COLS = 32;               // 8 complex outputs x (re, im) x (hi, lo)
constexpr size_t TC_SMEM_LIMIT = 225 * 1024;   // dynamic shared memory used at most
constexpr size_t TC_BAR_BYTES = 1024;          // mbarriers at the start of dynamic smem

struct TcParams {
  // pseudo-3D geometry (a 2D problem has its rows as planes and one row per plane)
  int kx, ky, kz;
  int W, Tx, Ty, nM;        // row pitch (positions), outputs per row, rows per tile, M tiles
  int Wb, nbx;              // TMA box width and boxes per row (2 when a row exceeds 256 positions)
  int PA;                   // positions per shared-memory plane of a stage
  int ntx, nty, nzr, L;     // x tiles, y tiles, runs of L output planes
  int ogs, kgroups;         // output-channel groups of 8, K groups of 8 input channels
  int org_x, org_y, org_z;  // input coordinate = output coordinate + offset + org
  int Zin, circ_z;          // input planes; wrap modulo Zin when circ_z
  int ox_lim, oy_lim, oz_lim;
  int chunks_even;          // 4-channel planes per split in the input tensor
  int stages, rs;           // stage ring depth, accumulator slots per M tile
  int tmem_cols;
  uint32_t stage_bytes, b_bytes;
  long long units;
  const unsigned char* bw;  // B per output-channel group, b_bytes each
  int mode;                 // 0: conv (R, split R planes, norms); 1: adjoint (masked g, norm)
  int cout;                 // output channels: p (conv) or C (adjoint)
  float2* R;                // conv: complex64 [o][cout]
  uint4* Rs;                // conv: split planes [split][2 ogs][o][8]
  long long r_plane;        // positions per R plane (= valid outputs)
  float2* g;                // adjoint output, element c*g_sc + base + z*g_sz + y*g_sy + x
  long long g_sc, g_sz, g_sy, g_base;
  const uint8_t* m;         // adjoint mask (nullable), same addressing with its strides
  long long m_sc, m_sz, m_sy, m_base;
  uint4* gs;                // adjoint (nullable): g also as split input planes [split][gs_ce][o][8],
  long long gs_plane;       //   the layout of tc_split_input_kernel over the region
  int gs_ce;
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

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(tc::smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

struct Unit {
  int og, zr, ty, tx;
};

__device__ __forceinline__ Unit unit_of(const TcParams& P, long long u) {
  Unit U;
  U.tx = (int)(u % P.ntx);
  u /= P.ntx;
  U.ty = (int)(u % P.nty);
  u /= P.nty;
  U.zr = (int)(u % P.nzr);
  U.og = (int)(u / P.nzr);
  return U;
}

// The MMAs of one stage: for each of the NM M tiles, the kx offsets, each with the hi and the lo
// input planes, into the window of accumulator slots [d0, d0 + 32 n0) (and [0, 32 n1) where the
// ring wraps).  The single issuing thread is the kernel's critical path, so descriptors are formed
// once and advanced by adding to their address field (16-byte units; shared-memory addresses stay
// below 2^18, so the field never carries), and the loops are unrolled at compile time: in
// straight-line code an MMA of N = 160 issues about as fast as the tensor core completes it
// (about 80 cycles), while a loop with a branch per offset halves the issue rate.
struct StageWin {
  uint32_t d0, id0, id1, dstride;   // dstride: TMEM columns between the M tiles' rings
  uint64_t bw0, bw1, lo16, boff16;
};

template <int KX, int NM, bool WRAP>
__device__ __forceinline__ void stage_mmas(uint32_t taddr, uint64_t a_st, uint64_t b_st, const StageWin& w) {
#pragma unroll
  for (int mt = 0; mt < NM; ++mt) {
    const uint32_t dm = taddr + (uint32_t)mt * w.dstride;
    const uint64_t a_mt = a_st + (uint64_t)(mt * 128);
#pragma unroll
    for (int dx = 0; dx < KX; ++dx) {
      const uint64_t ah = a_mt + (uint64_t)dx, al = ah + w.lo16;
      const uint64_t bb = b_st + (uint64_t)dx * w.boff16;
      tc::mma_bf16_acc(dm + w.d0, ah, bb + w.bw0, w.id0);
      if (WRAP) tc::mma_bf16_acc(dm, ah, bb + w.bw1, w.id1);
      tc::mma_bf16_acc(dm + w.d0, al, bb + w.bw0, w.id0);
      if (WRAP) tc::mma_bf16_acc(dm, al, bb + w.bw1, w.id1);
    }
  }
}

template <int KX>
__device__ __forceinline__ void stage_mmas_kx(int nM, bool wrap, uint32_t taddr, uint64_t a_st, uint64_t b_st,
                                              const StageWin& w) {
  if (nM == 2) {
    if (wrap) stage_mmas<KX, 2, true>(taddr, a_st, b_st, w);
    else stage_mmas<KX, 2, false>(taddr, a_st, b_st, w);
  } else {
    if (wrap) stage_mmas<KX, 1, true>(taddr, a_st, b_st, w);
    else stage_mmas<KX, 1, false>(taddr, a_st, b_st, w);
  }
}

// the offsets of every M tile; kernel widths without an unrolled form take a loop
__device__ __forceinline__ void stage_mmas_any(int kx, int nM, bool wrap, uint32_t taddr, uint64_t a_st,
                                               uint64_t b_st, const StageWin& w) {
  switch (kx) {
    case 1: stage_mmas_kx<1>(nM, wrap, taddr, a_st, b_st, w); return;
    case 2: stage_mmas_kx<2>(nM, wrap, taddr, a_st, b_st, w); return;
    case 3: stage_mmas_kx<3>(nM, wrap, taddr, a_st, b_st, w); return;
    case 4: stage_mmas_kx<4>(nM, wrap, taddr, a_st, b_st, w); return;
    case 5: stage_mmas_kx<5>(nM, wrap, taddr, a_st, b_st, w); return;
    case 7: stage_mmas_kx<7>(nM, wrap, taddr, a_st, b_st, w); return;
    default: break;
  }
  for (int mt = 0; mt < nM; ++mt) {
    const uint32_t dm = taddr + (uint32_t)mt * w.dstride;
    const uint64_t a_mt = a_st + (uint64_t)(mt * 128);
    for (int dx = 0; dx < kx; ++dx) {
      const uint64_t ah = a_mt + (uint64_t)dx, al = ah + w.lo16;
      const uint64_t bb = b_st + (uint64_t)dx * w.boff16;
      tc::mma_bf16_acc(dm + w.d0, ah, bb + w.bw0, w.id0);
      if (wrap) tc::mma_bf16_acc(dm, ah, bb + w.bw1, w.id1);
      tc::mma_bf16_acc(dm + w.d0, al, bb + w.bw0, w.id0);
      if (wrap) tc::mma_bf16_acc(dm, al, bb + w.bw1, w.id1);
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_corr_kernel(const __grid_constant__ CUtensorMap amap, const TcParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // 128-byte aligned base (TMA destinations); the launch adds 128 bytes of slack
  unsigned char* smem = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  uint64_t* full = bars;                        // [stages]
  uint64_t* empty = bars + TC_MAX_STAGES;       // [stages]
  uint64_t* acc_full = bars + 2 * TC_MAX_STAGES;         // [rs]
  uint64_t* acc_empty = acc_full + 16;                   // [rs]
  uint64_t* bfull = acc_empty + 16;
  uint64_t* bfree = bfull + 1;
  uint64_t* done = bfree + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  double* red = reinterpret_cast<double*>(smem + 512);  // per-warp norm sums
  unsigned char* sB = smem + TC_BAR_BYTES;
  unsigned char* sA = sB + P.b_bytes;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < P.stages; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < P.rs; ++i) {
      tc::mbar_init(&acc_full[i], 1);
      tc::mbar_init(&acc_empty[i], 4);  // one arrival per epilogue warp
    }
    tc::mbar_init(bfull, 1);
    tc::mbar_init(bfree, 1);
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, (uint32_t)P.tmem_cols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t taddr = *tslot;
  // every accumulator slot starts at zero (and the epilogue zeroes each slot it drains), so that
  // every MMA accumulates: the epilogue warps clear their lane quarter of the allocation
  if (warp >= 2) {
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    for (int col = 0; col < P.tmem_cols; col += 16) tc::tmem_st16_zero(taddr + lane_base + (uint32_t)col);
    tc::tmem_st_wait();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  // programmatic dependent launch: the set-up above overlaps the previous kernel's tail; its
  // outputs (this kernel's inputs) are read only from here on
  pdl_wait();
  pdl_trigger();
  const int zspan = P.kz - 1;  // input planes beyond the last output plane of a run

  if (warp == 0) {
    // ------------------------------------------------------------- TMA producer
    if (lane == 0) {
      bool ok = true;
      // stage ring position and completed rounds (counters, not divisions: the roles' loops are on
      // the critical path and a 64-bit division costs about a hundred instructions)
      int s = 0;
      uint32_t round = 0;
      int prev_og = -1, j = 0;
      const uint32_t plane_b = (uint32_t)P.PA * 16u;
      const uint32_t a_tx = 4u * (uint32_t)P.nbx * (uint32_t)P.Ty * (uint32_t)P.Wb * 16u;
      for (long long u = blockIdx.x; u < P.units && ok; u += gridDim.x, ++j) {
        const Unit U = unit_of(P, u);
        if (U.og != prev_og) {
          if (j > 0) ok = tc::mbar_wait(bfree, (uint32_t)((j - 1) & 1), P.err);
          if (!ok) break;
          tc::mbar_arrive_expect_tx(bfull, P.b_bytes);
          tc::bulk_g2s(sB, P.bw + (size_t)U.og * P.b_bytes, P.b_bytes, bfull);
          prev_og = U.og;
        }
        const int zo_lo = U.zr * P.L, zo_hi = min(zo_lo + P.L, P.oz_lim);
        const int xin = U.tx * P.Tx + P.org_x;
        for (int v = zo_lo; v <= zo_hi - 1 + zspan && ok; ++v) {
          int zin = v + P.org_z;
          if (P.circ_z) zin = wrap(zin, P.Zin);
          for (int dy = 0; dy < P.ky && ok; ++dy) {
            const int yin = U.ty * P.Ty + dy + P.org_y;
            for (int kg = 0; kg < P.kgroups; ++kg) {
              if (round > 0) ok = tc::mbar_wait(&empty[s], (round - 1) & 1u, P.err);
              if (!ok) break;
              unsigned char* st = sA + (size_t)s * P.stage_bytes;
              tc::mbar_arrive_expect_tx(&full[s], a_tx);
#pragma unroll
              for (int sp = 0; sp < 2; ++sp)
#pragma unroll
                for (int cc = 0; cc < 2; ++cc)
                  for (int bx = 0; bx < P.nbx; ++bx)  // nbx > 1 only with one row per tile
                    tma_load_5d(st + (sp * 2 + cc) * plane_b + bx * P.Wb * 16, &amap, 0, xin + bx * P.Wb, yin,
                                zin, sp * P.chunks_even + 2 * kg + cc, &full[s]);
              if (++s == P.stages) {
                s = 0;
                ++round;
              }
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      bool ok = true;
      int s = 0, q0 = 0;
      uint32_t round = 0;
      int prev_og = -1, nb = 0;
      const uint32_t plane_b = (uint32_t)P.PA * 16u;
      const uint32_t lbo_b = 512u * (uint32_t)P.kz;   // cc0 -> cc1 core matrices of B
      const uint32_t boff = 1024u * (uint32_t)P.kz;   // B bytes per (kg, dy, dx)
      const uint32_t b_base = tc::smem_u32(sB);
      const uint64_t a_desc0 = tc::smem_desc(tc::smem_u32(sA), plane_b, 128);
      const uint64_t b_desc0 = tc::smem_desc(b_base, lbo_b, 128);
      const uint64_t stage16 = P.stage_bytes >> 4;
      StageWin w;
      w.lo16 = (2u * plane_b) >> 4;
      w.boff16 = boff >> 4;
      w.dstride = (uint32_t)(P.rs * TC_SLOT_COLS);
      for (long long u = blockIdx.x; u < P.units && ok; u += gridDim.x) {
        const Unit U = unit_of(P, u);
        if (U.og != prev_og) {
          ok = tc::mbar_wait(bfull, (uint32_t)(nb & 1), P.err);
          ++nb;
          prev_og = U.og;
          if (!ok) break;
        }
        const int zo_lo = U.zr * P.L, zo_hi = min(zo_lo + P.L, P.oz_lim);
        for (int v = zo_lo; v <= zo_hi - 1 + zspan && ok; ++v) {
          const int za = max(zo_lo, v - zspan), zb = min(zo_hi - 1, v);
          const int cnt = zb - za + 1;
          // output plane v starts here: its slot's previous plane must have been drained (and the
          // slot zeroed) by the epilogue before the first MMA accumulates into it
          const bool fresh = v <= zo_hi - 1;
          const int sa = (q0 + (za - zo_lo)) % P.rs;
          if (fresh) {
            const int qn = q0 + (v - zo_lo);
            if (qn >= P.rs) ok = tc::mbar_wait(&acc_empty[qn % P.rs], (uint32_t)(((qn / P.rs) - 1) & 1), P.err);
            if (!ok) break;
          }
          const int ba = P.kz - 1 - (v - za);  // B block of output plane za (blocks hold dz = kz-1-b)
          // the window's slots [sa, sa + cnt) as one MMA, or two where the ring wraps at rs
          const int n0 = min(cnt, P.rs - sa), n1 = cnt - n0;
          w.d0 = (uint32_t)(sa * TC_SLOT_COLS);
          w.id0 = tc::idesc_bf16_f32(128, TC_SLOT_COLS * n0);
          w.id1 = tc::idesc_bf16_f32(128, TC_SLOT_COLS * (n1 > 0 ? n1 : 1));
          w.bw0 = (uint64_t)ba * 32u;
          w.bw1 = (uint64_t)(ba + n0) * 32u;
          for (int dy = 0; dy < P.ky && ok; ++dy) {
            for (int kg = 0; kg < P.kgroups; ++kg) {
              ok = tc::mbar_wait(&full[s], round & 1u, P.err);
              if (!ok) break;
              tc::tc_fence_after();
              const uint64_t a_st = a_desc0 + (uint64_t)s * stage16;
              const uint64_t b_st = b_desc0 + (uint64_t)((kg * P.ky + dy) * P.kx) * w.boff16;
              stage_mmas_any(P.kx, P.nM, n1 > 0, taddr, a_st, b_st, w);
              tc::mma_commit(&empty[s]);
              if (++s == P.stages) {
                s = 0;
                ++round;
              }
            }
          }
          if (ok && v - zspan >= zo_lo) {
            const int qc = q0 + (v - zspan - zo_lo);  // output plane complete
            tc::mma_commit(&acc_full[qc % P.rs]);
          }
        }
        q0 += zo_hi - zo_lo;
        if (ok) tc::mma_commit(bfree);
      }
      tc::mma_commit(done);
      tc::mbar_wait(done, 0, P.err);
    }
  } else {
    // --------------------------------------------------------------------- epilogue
    const int quad = warp & 3;  // TMEM lanes 32*quad .. 32*quad + 31
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    double nrm_d = 0.0;
    bool ok = true;
    int q = 0;
    for (long long u = blockIdx.x; u < P.units && ok; u += gridDim.x) {
      const Unit U = unit_of(P, u);
      const int zo_lo = U.zr * P.L, zo_hi = min(zo_lo + P.L, P.oz_lim);
      for (int z = zo_lo; z < zo_hi; ++z, ++q) {
        const int slot = q % P.rs;
        ok = tc::mbar_wait(&acc_full[slot], (uint32_t)((q / P.rs) & 1), P.err);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        tc::tc_fence_after();
        uint32_t hi[2][16], lo[2][16];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          if (mt < P.nM) {
            const uint32_t col = taddr + lane_base + (uint32_t)((mt * P.rs + slot) * TC_SLOT_COLS);
            tc::tmem_ld16(col, hi[mt]);
            tc::tmem_ld16(col + 16u, lo[mt]);
          }
        }
        tc::tmem_ld_wait();
        // the slot back to zero for the next output plane that takes it
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          if (mt < P.nM) {
            const uint32_t col = taddr + lane_base + (uint32_t)((mt * P.rs + slot) * TC_SLOT_COLS);
            tc::tmem_st16_zero(col);
            tc::tmem_st16_zero(col + 16u);
          }
        }
        tc::tmem_st_wait();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[slot]);
        float nrm = 0.f;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          if (mt >= P.nM) continue;
          const int pos = mt * 128 + 32 * quad + lane;
          const int ly = pos / P.W, lx = pos - (pos / P.W) * P.W;
          const int ox = U.tx * P.Tx + lx, oy = U.ty * P.Ty + ly;
          if (!(ly < P.Ty && lx < P.Tx && ox < P.ox_lim && oy < P.oy_lim)) continue;
          float v[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(hi[mt][e]) + __uint_as_float(lo[mt][e]);
          if (P.mode == 0) {
            const long long o = ((long long)z * P.oy_lim + oy) * P.ox_lim + ox;
#pragma unroll
            for (int q2 = 0; q2 < 8; ++q2) {
              const int k = U.og * 8 + q2;
              if (k < P.cout) {
                nrm = fmaf(v[2 * q2], v[2 * q2], fmaf(v[2 * q2 + 1], v[2 * q2 + 1], nrm));
                if (P.R) P.R[o * P.cout + k] = make_float2(v[2 * q2], v[2 * q2 + 1]);
              } else {
                v[2 * q2] = 0.f;
                v[2 * q2 + 1] = 0.f;
              }
            }
            if (P.Rs) {
              const int nplanes = 2 * P.ogs;
#pragma unroll
              for (int hc = 0; hc < 2; ++hc) {
                float w8[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) w8[e] = v[8 * hc + e];
                uint4 h4, l4;
                split8(w8, h4, l4);
                const int jr = 2 * U.og + hc;
                P.Rs[(size_t)jr * P.r_plane + o] = h4;
                P.Rs[(size_t)(nplanes + jr) * P.r_plane + o] = l4;
              }
            }
          } else {
            const long long go = P.g_base + (long long)z * P.g_sz + (long long)oy * P.g_sy + ox;
            const long long mo = P.m_base + (long long)z * P.m_sz + (long long)oy * P.m_sy + ox;
            float vm[16];
#pragma unroll
            for (int q2 = 0; q2 < 8; ++q2) {
              const int c = U.og * 8 + q2;
              float2 w = make_float2(0.f, 0.f);
              if (c < P.cout) {
                w = make_float2(v[2 * q2], v[2 * q2 + 1]);
                if (P.m && P.m[(long long)c * P.m_sc + mo]) w = make_float2(0.f, 0.f);
                P.g[(long long)c * P.g_sc + go] = w;
                nrm = fmaf(w.x, w.x, fmaf(w.y, w.y, nrm));
              }
              vm[2 * q2] = w.x;
              vm[2 * q2 + 1] = w.y;
            }
            if (P.gs) {
              // the masked g of this position as the next convolution's split input (4 channels
              // per 16-byte word, hi and lo planes), in place of a separate split launch
              const long long o = ((long long)z * P.oy_lim + oy) * P.ox_lim + ox;
#pragma unroll
              for (int hc = 0; hc < 2; ++hc) {
                const int chunk = 2 * U.og + hc;
                if (chunk < P.gs_ce) {
                  float w8[8];
#pragma unroll
                  for (int e = 0; e < 8; ++e) w8[e] = vm[8 * hc + e];
                  uint4 h4, l4;
                  split8(w8, h4, l4);
                  P.gs[(size_t)chunk * P.gs_plane + o] = h4;
                  P.gs[(size_t)(P.gs_ce + chunk) * P.gs_plane + o] = l4;
                }
              }
            }
          }
        }
        nrm_d += (double)nrm;
      }
    }
    for (int o = 16; o > 0; o >>= 1) nrm_d += __shfl_down_sync(0xffffffffu, nrm_d, o);
    if (lane == 0) red[warp] = nrm_d;
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)P.tmem_cols);
  if (tid == 0) P.partial[blockIdx.x] = red[2] + red[3] + red[4] + red[5];
}

// ------------------------------------------------------------- layout kernels

// Region of a complex64 array -> planar split bf16 [split][chunk_even][ez][ey][ex][8],
// chunk = 4 channels; channels >= C (padding) are zero.
__global__ void tc_split_input_kernel(int C, int chunks_even, int ex, int ey, int ez, KView x,
                                      uint4* __restrict__ out) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  const long long plane = (long long)ex * ey * ez;
  const long long tot = plane * chunks_even;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / plane);
    const long long pos = i - (long long)j * plane;
    const int ux = (int)(pos % ex);
    const long long r = pos / ex;
    const int uy = (int)(r % ey), uz = (int)(r / ey);
    float v[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int c = 4 * j + e;
      float2 a = make_float2(0.f, 0.f);
      if (c < C)
        a = x.p[(long long)c * x.sc + (long long)(x.oz + uz) * x.sz + (long long)(x.oy + uy) * x.sy + (x.ox + ux)];
      v[2 * e] = a.x;
      v[2 * e + 1] = a.y;
    }
    uint4 hi, lo;
    split8(v, hi, lo);
    out[(long long)j * plane + pos] = hi;
    out[(long long)(chunks_even + j) * plane + pos] = lo;
  }
}

// R complex64 [s][p] -> planar split bf16 [split][chunk_even][s][8], chunk = 4 filters (zero padded)
__global__ void tc_split_r_kernel(long long npos, int p, int chunks_even, const float2* __restrict__ R,
                                  uint4* __restrict__ out) {
  const long long tot = npos * chunks_even;
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
    out[(long long)(chunks_even + j) * npos + pos] = lo;
  }
}

// B for the streamed correlation, per output-channel group og (8 outputs):
//   [og][kg][dy][dx][cc][blk][row][e]   (bf16), pseudo-3D offsets (dz, dy, dx)
// K index within the MMA step: cc*8 + e -> input channel 8 kg + 4 cc + e/2, t = e%2 (re/im);
// N row: blk b holds dz = kz-1-b, row = split*16 + 2 o + u (output channel 8 og + o, u = re/im).
// conv    (mode 0): weight of offset d = (dz, dy, dx) is f = bank[co][ci*K + d], embedding
//                   [[f.re, f.im], [-f.im, f.re]] (rows t, columns u);
// adjoint (mode 1): weight of shift d' is conj(bank[ci][co*K + (k-1-d')]), embedding
//                   [[f.re, -f.im], [f.im, f.re]].
// The pseudo-3D offset index is (dz*ky + dy)*kx + dx, which is the bank's [kz][ky][kx] order in
// 3D and its [ky][kx] order for a 2D problem run with rows as planes (ky = 1, kz = k_y).
struct PrepB {
  int mode, Cin, Cout, kgroups, ogs;
  long long tot;
  __nv_bfloat16* out;
};

// one element i of a B operand (see the layout above)
__device__ __forceinline__ __nv_bfloat16 prep_b_elem(const PrepB& q, int n, int kx, int ky, int kz,
                                                     const float2* __restrict__ bank, long long i) {
  const int K = kx * ky * kz;
  long long t = i;
  const int e = (int)(t % 8); t /= 8;
  const int row = (int)(t % 32); t /= 32;
  const int blk = (int)(t % kz); t /= kz;
  const int cc = (int)(t % 2); t /= 2;
  const int dx = (int)(t % kx); t /= kx;
  const int dy = (int)(t % ky); t /= ky;
  const int kg = (int)(t % q.kgroups); t /= q.kgroups;
  const int og = (int)t;
  const int dz = kz - 1 - blk;
  const int ci = 8 * kg + 4 * cc + e / 2, tin = e & 1;
  const int split = row >> 4, rr = row & 15;
  const int co = 8 * og + rr / 2, uout = rr & 1;
  float w = 0.f;
  if (ci < q.Cin && co < q.Cout) {
    if (q.mode == 0) {
      const float2 f = bank[(long long)co * n + (long long)ci * K + (dz * ky + dy) * kx + dx];
      w = (tin == 0) ? (uout == 0 ? f.x : f.y) : (uout == 0 ? -f.y : f.x);
    } else {
      const int d = ((kz - 1 - dz) * ky + (ky - 1 - dy)) * kx + (kx - 1 - dx);
      const float2 f = bank[(long long)ci * n + (long long)co * K + d];
      w = (tin == 0) ? (uout == 0 ? f.x : -f.y) : (uout == 0 ? f.y : f.x);
    }
  }
  const float hi = __bfloat162float(__float2bfloat16_rn(w));
  return __float2bfloat16_rn(split == 0 ? hi : w - hi);
}

// the B operands of the conv (q0) and of the adjoint (q1, tot = 0 when not wanted) in one launch
__global__ void tc_prep_b_kernel(PrepB q0, PrepB q1, int n, int kx, int ky, int kz, const float2* __restrict__ bank) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  const long long tot = q0.tot + q1.tot;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < q0.tot) q0.out[i] = prep_b_elem(q0, n, kx, ky, kz, bank, i);
    else q1.out[i - q0.tot] = prep_b_elem(q1, n, kx, ky, kz, bank, i - q0.tot);
  }
}

// The descent step's finalisation and update (as update_step_kernel) for the tensor-core path,
// a thread per (4-channel chunk, region position): y <- y - eta g on the unobserved entries (the
// observed ones are never written), and the updated y of the region written as the split input
// planes of the next step's convolution (the layout of tc_split_input_kernel), so that the next
// step needs no split launch of its own.
__global__ void update_step_planes_kernel(ConvGeom g, KView y, KView gb, MView m, const double* __restrict__ part,
                                          int n_obj, int n_g, int n_d, double* stats, uint4* __restrict__ planes,
                                          int chunks_even) {
  pdl_wait();  // programmatic dependent launch: inputs of the previous kernel
  pdl_trigger();
  __shared__ double sh[8];
  __shared__ double s_eta;
  const double obj = block_fixed_sum(part, n_obj, sh);
  const double gn2 = block_fixed_sum(part + n_obj, n_g, sh);
  const double D = block_fixed_sum(part + n_obj + n_g, n_d, sh);
  if (threadIdx.x == 0) {
    double eta = 0.0;
    if (D > 0.0 && gn2 > 0.0 && isfinite(D) && isfinite(gn2)) eta = gn2 / D;
    if (blockIdx.x == 0) {
      stats[0] = eta;
      stats[1] = obj;
      stats[2] = gn2;
      stats[3] = D;
    }
    s_eta = eta;
  }
  __syncthreads();
  const double eta = s_eta;
  const float e = (float)eta;
  const long long plane = (long long)g.ex * g.ey * g.ez;
  const long long tot = plane * chunks_even;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / plane);
    const long long pos = i - (long long)j * plane;
    const int ux = (int)(pos % g.ex);
    const long long r = pos / g.ex;
    const int uy = (int)(r % g.ey), uz = (int)(r / g.ey);
    float v[8];
#pragma unroll
    for (int e4 = 0; e4 < 4; ++e4) {
      const int c = 4 * j + e4;
      float2 a = make_float2(0.f, 0.f);
      if (c < g.C) {
        float2* yp = y.p + (long long)c * y.sc + (long long)(y.oz + uz) * y.sz + (long long)(y.oy + uy) * y.sy +
                     (y.ox + ux);
        a = *yp;
        const bool observed = m.p && m.p[(long long)c * m.sc + (long long)(m.oz + uz) * m.sz +
                                         (long long)(m.oy + uy) * m.sy + (m.ox + ux)];
        if (!observed && eta != 0.0) {
          const float2 gv = gb.p[(long long)c * gb.sc + (long long)(gb.oz + uz) * gb.sz +
                                 (long long)(gb.oy + uy) * gb.sy + (gb.ox + ux)];
          a.x = fmaf(-e, gv.x, a.x);
          a.y = fmaf(-e, gv.y, a.y);
          *yp = a;
        }
      }
      v[2 * e4] = a.x;
      v[2 * e4 + 1] = a.y;
    }
    uint4 hi, lo;
    split8(v, hi, lo);
    planes[(long long)j * plane + pos] = hi;
    planes[(long long)(chunks_even + j) * plane + pos] = lo;
  }
}

// ---------------------------------------------------------------- host side

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Pseudo-3D view of a problem: a 2D problem (kz = 1, one plane) runs with its rows as planes.
struct Pseudo {
  int kx, ky, kz;
  int circ;            // circular along the pseudo-z axis
  bool ok;             // a circular axis the kernel cannot wrap (x, or y of a 3D problem)
};

Pseudo pseudo_of(const ConvGeom& g) {
  Pseudo q;
  q.kx = g.kx;
  if (g.kz == 1 && g.ez == 1) {
    q.ky = 1;
    q.kz = g.ky;
    q.circ = g.cy;
    q.ok = !g.cx && !g.cz;
  } else {
    q.ky = g.ky;
    q.kz = g.kz;
    q.circ = g.cz;
    q.ok = !g.cx && !g.cy;
  }
  return q;
}

// extents of an array in pseudo-3D (x, y, z)
void pseudo_ext(const ConvGeom& g, int ax, int ay, int az, int* px, int* py, int* pz) {
  *px = ax;
  if (g.kz == 1 && g.ez == 1) {
    *py = 1;
    *pz = ay;
  } else {
    *py = ay;
    *pz = az;
  }
}

int chunks_even_of(int channels) { return 2 * ((channels + 7) / 8); }

struct TcPlan {
  TcParams P;
  size_t smem;
  int grid;
  int Xin, Yin;  // input extents (pseudo x, y)
};

// Tile plan.  x: the fewest tiles whose halo (Tx + kx - 1) fits 256 positions; y: as many rows
// as fill 256 positions (one row for a 2D problem); z: the run length L that minimises
// (units per CTA) x (planes each unit reads) over a persistent grid of num_sms CTAs.
bool plan_tc(TcPlan* pl, const ConvGeom& g, int mode, int p, int num_sms) {
  const Pseudo q = pseudo_of(g);
  if (!q.ok || q.kz > 8 || q.kx > 16) return false;
  TcParams& P = pl->P;
  P = TcParams{};
  P.kx = q.kx;
  P.ky = q.ky;
  P.kz = q.kz;
  P.circ_z = q.circ;
  P.mode = mode;
  const int Cin = mode == 0 ? g.C : p;
  P.cout = mode == 0 ? p : g.C;
  P.kgroups = (Cin + 7) / 8;
  P.ogs = (P.cout + 7) / 8;
  P.chunks_even = chunks_even_of(Cin);
  int ox, oy, oz, ix, iy, iz;
  if (mode == 0) {
    pseudo_ext(g, g.sx, g.sy, g.sz, &ox, &oy, &oz);
    pseudo_ext(g, g.ex, g.ey, g.ez, &ix, &iy, &iz);
    P.org_x = P.org_y = P.org_z = 0;
  } else {
    pseudo_ext(g, g.ex, g.ey, g.ez, &ox, &oy, &oz);
    pseudo_ext(g, g.sx, g.sy, g.sz, &ix, &iy, &iz);
    P.org_x = -(P.kx - 1);
    P.org_y = -(P.ky - 1);
    P.org_z = -(P.kz - 1);
  }
  P.ox_lim = ox;
  P.oy_lim = oy;
  P.oz_lim = oz;
  P.Zin = iz;
  pl->Xin = ix;
  pl->Yin = iy;
  // M rows are tile positions ly * W + lx; the valid ones (lx < Tx, ly < Ty) must fit 2 M tiles
  P.ntx = (ox + 255) / 256;
  P.Tx = (ox + P.ntx - 1) / P.ntx;
  P.W = P.Tx + P.kx - 1;
  P.Ty = 1;
  if (P.W <= 256) P.Ty = std::max(1, std::min(oy, (256 - P.Tx) / P.W + 1));
  P.nty = (oy + P.Ty - 1) / P.Ty;
  P.nM = ((P.Ty - 1) * P.W + P.Tx + 127) / 128;
  if (P.nM > 2) return false;
  P.nbx = P.W <= 256 ? 1 : 2;
  // One box keeps the row pitch W (a box of Ty rows lands as [Ty][W]).  A split row (Ty = 1):
  // TMA writes to shared memory start 128-byte aligned and the second box starts Wb positions
  // (16 bytes each) in, so Wb is a multiple of 8.
  P.Wb = P.nbx == 1 ? P.W : ((P.W + 1) / 2 + 7) / 8 * 8;
  P.PA = (std::max(P.nbx * P.Wb * P.Ty, P.nM * 128 + P.kx - 1) + 7) / 8 * 8;
  P.stage_bytes = (uint32_t)(4 * P.PA * 16);
  P.b_bytes = (uint32_t)((size_t)P.kgroups * P.kx * P.ky * P.kz * 1024);
  const size_t fixed = TC_BAR_BYTES + P.b_bytes + 128;
  if (fixed + 2 * (size_t)P.stage_bytes > TC_SMEM_LIMIT) return false;
  P.stages = (int)std::min<size_t>(TC_MAX_STAGES, (TC_SMEM_LIMIT - fixed) / P.stage_bytes);
  // the whole TMEM (one CTA per SM): a longer ring wraps fewer MMA windows
  P.rs = std::min(16, 512 / (TC_SLOT_COLS * P.nM));
  if (P.rs < P.kz || P.rs > 16) return false;
  int cols = 32;
  while (cols < P.nM * P.rs * TC_SLOT_COLS) cols <<= 1;
  P.tmem_cols = cols;
  // run length along z
  const long long per_z = (long long)P.ogs * P.nty * P.ntx;
  long long best_cost = -1;
  int bestL = 1;
  for (int L = 1; L <= oz; ++L) {
    const long long units = per_z * ((oz + L - 1) / L);
    const long long waves = (units + num_sms - 1) / num_sms;
    const long long cost = waves * (L + P.kz - 1);
    if (best_cost < 0 || cost <= best_cost) {
      best_cost = cost;
      bestL = L;
    }
  }
  P.L = bestL;
  P.nzr = (oz + P.L - 1) / P.L;
  P.units = per_z * P.nzr;
  pl->grid = (int)std::min<long long>(P.units, num_sms);
  // at least half the SM's shared memory, so that one CTA (and its TMEM ring) owns each SM
  pl->smem = std::max<size_t>(fixed + (size_t)P.stages * P.stage_bytes, 120 * 1024);
  return true;
}

bool encode_input_map(CUtensorMap* map, const void* base, int X, int Y, int Z, int planes, int W, int Ty) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[5] = {8, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)Z, (cuuint64_t)planes};
  const cuuint64_t strides[4] = {16, (cuuint64_t)16 * X, (cuuint64_t)16 * X * Y, (cuuint64_t)16 * X * Y * Z};
  const cuuint32_t box[5] = {8, (cuuint32_t)W, (cuuint32_t)Ty, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int device_sms(hicu_handle* h) { return h->num_sms > 0 ? h->num_sms : 148; }

// Plans and tensor maps are pure functions of their arguments; the descent loop asks for the same
// few again and again, so both are kept (process-wide, under a mutex; host threads of a batch
// share them).  A cached tensor map is keyed on its base address as well.
struct PlanKey {
  int v[16];
  bool operator<(const PlanKey& o) const { return std::memcmp(v, o.v, sizeof v) < 0; }
};
struct PlanEntry {
  bool ok;
  TcPlan plan;
};

bool plan_tc_cached(TcPlan* pl, const ConvGeom& g, int mode, int p, int num_sms) {
  static std::mutex mu;
  static std::map<PlanKey, PlanEntry> cache;
  PlanKey k;
  std::memset(k.v, 0, sizeof k.v);
  const int vals[16] = {g.C, g.kx, g.ky, g.kz, g.ex, g.ey, g.ez, g.sx, g.sy, g.sz, g.cx, g.cy, g.cz, mode, p, num_sms};
  std::memcpy(k.v, vals, sizeof vals);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(k);
    if (it != cache.end()) {
      if (it->second.ok) *pl = it->second.plan;
      return it->second.ok;
    }
  }
  PlanEntry e;
  e.ok = plan_tc(&e.plan, g, mode, p, num_sms);
  std::lock_guard<std::mutex> lock(mu);
  if (cache.size() > 4096) cache.clear();
  cache[k] = e;
  if (e.ok) *pl = e.plan;
  return e.ok;
}

struct MapKey {
  const void* base;
  int v[6];
  bool operator<(const MapKey& o) const {
    if (base != o.base) return base < o.base;
    return std::memcmp(v, o.v, sizeof v) < 0;
  }
};

bool encode_input_map_cached(CUtensorMap* map, const void* base, int X, int Y, int Z, int planes, int W, int Ty) {
  static std::mutex mu;
  static std::map<MapKey, CUtensorMap> cache;
  MapKey k;
  k.base = base;
  const int vals[6] = {X, Y, Z, planes, W, Ty};
  std::memcpy(k.v, vals, sizeof vals);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(k);
    if (it != cache.end()) {
      *map = it->second;
      return true;
    }
  }
  if (!encode_input_map(map, base, X, Y, Z, planes, W, Ty)) return false;
  std::lock_guard<std::mutex> lock(mu);
  if (cache.size() > 1024) cache.clear();
  cache[k] = *map;
  return true;
}

}  // namespace

bool tc_supported(const ConvGeom& g) {
  TcPlan a, b;
  return plan_tc_cached(&a, g, 0, 8, 152) && plan_tc_cached(&b, g, 1, 8, 152) && encode_fn() != nullptr;
}

bool tc_supported_p(const ConvGeom& g, int p) {
  TcPlan a, b;
  return plan_tc_cached(&a, g, 0, p, 152) && plan_tc_cached(&b, g, 1, p, 152) && encode_fn() != nullptr;
}

size_t tc_x_bytes(const ConvGeom& g) {
  return (size_t)16 * 2 * chunks_even_of(g.C) * g.ex * g.ey * g.ez;
}

size_t tc_r_bytes(const ConvGeom& g, int p) { return (size_t)16 * 2 * chunks_even_of(p) * g.s; }

size_t tc_b_bytes(const ConvGeom& g, int p, int mode) {
  const Pseudo q = pseudo_of(g);
  const int Cin = mode == 0 ? g.C : p, Cout = mode == 0 ? p : g.C;
  return (size_t)((Cout + 7) / 8) * ((Cin + 7) / 8) * q.kx * q.ky * q.kz * 1024;
}

hicu_status tc_prepare_input(hicu_handle* h, const ConvGeom& g, KView x, uint4* planar, cudaStream_t st) {
  const int ce = chunks_even_of(g.C);
  const long long tot = (long long)g.ex * g.ey * g.ez * ce;
  int blocks = (int)std::min<long long>((tot + 255) / 256, 8192);
  const cudaError_t e = launch_pdl(h, K_MISC, st, dim3(blocks), dim3(256), 0, tc_split_input_kernel, true, g.C, ce,
                                   g.ex, g.ey, g.ez, x, planar);
  return cuda_error(h, e != cudaSuccess ? e : cudaGetLastError(), "tc_split_input");
}

hicu_status launch_update_step_planes(hicu_handle* h, const ConvGeom& g, KView y, KView gb, MView m,
                                     const double* part, int n_obj, int n_g, int n_d, double* stats, uint4* planar,
                                     cudaStream_t st) {
  const int ce = chunks_even_of(g.C);
  const long long tot = (long long)g.ex * g.ey * g.ez * ce;
  int blocks = (int)((tot + 255) / 256);
  const int cap = 4 * (h->num_sms > 0 ? h->num_sms : 152);
  if (blocks > cap) blocks = cap;
  const cudaError_t e = launch_pdl(h, K_MISC, st, dim3(blocks), dim3(256), 0, update_step_planes_kernel, true, g,
                                   y, gb, m, part, n_obj, n_g, n_d, stats, planar, ce);
  return cuda_error(h, e != cudaSuccess ? e : cudaGetLastError(), "update");
}

hicu_status tc_prepare_r(hicu_handle* h, const ConvGeom& g, const float2* R, int p, uint4* planar,
                         cudaStream_t st) {
  const int ce = chunks_even_of(p);
  const long long tot = g.s * ce;
  int blocks = (int)std::min<long long>((tot + 255) / 256, 8192);
  HICU_LAUNCH(h, K_MISC, st, tc_split_r_kernel<<<blocks, 256, 0, st>>>(g.s, p, ce, R, planar));
  return cuda_error(h, cudaGetLastError(), "tc_split_r");
}

static PrepB prep_b_of(const ConvGeom& g, int p, int mode, void* out) {
  PrepB q;
  q.mode = mode;
  q.Cin = mode == 0 ? g.C : p;
  q.Cout = mode == 0 ? p : g.C;
  q.kgroups = (q.Cin + 7) / 8;
  q.ogs = (q.Cout + 7) / 8;
  q.tot = out ? (long long)tc_b_bytes(g, p, mode) / 2 : 0;
  q.out = (__nv_bfloat16*)out;
  return q;
}

hicu_status tc_prepare_weights(hicu_handle* h, const ConvGeom& g, const float2* bank, int p, void* out_conv,
                               void* out_adjoint, cudaStream_t st) {
  const Pseudo q = pseudo_of(g);
  const PrepB q0 = prep_b_of(g, p, 0, out_conv), q1 = prep_b_of(g, p, 1, out_adjoint);
  const long long tot = q0.tot + q1.tot;
  int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  const cudaError_t e = launch_pdl(h, K_MISC, st, dim3(blocks), dim3(256), 0, tc_prep_b_kernel, true, q0, q1, g.n,
                                   q.kx, q.ky, q.kz, bank);
  return cuda_error(h, e != cudaSuccess ? e : cudaGetLastError(), "tc_prep_b");
}

static hicu_status launch_plan(hicu_handle* h, TcPlan& pl, const void* in, int cls, cudaStream_t st) {
  CUtensorMap map;
  if (!encode_input_map_cached(&map, in, pl.Xin, pl.Yin, pl.P.Zin, 2 * pl.P.chunks_even, pl.P.Wb, pl.P.Ty))
    return set_error(h, HICU_ERR_CUDA, "split-bf16: tensor map encoding failed");
  const cudaError_t e = allow_max_dynamic_smem((const void*)tc_corr_kernel);
  if (e != cudaSuccess) return cuda_error(h, e, "tc_corr smem");
  const cudaError_t e2 = launch_pdl(h, cls, st, dim3(pl.grid), dim3(TC_THREADS), pl.smem, tc_corr_kernel, true, map,
                                    pl.P);
  return cuda_error(h, e2 != cudaSuccess ? e2 : cudaGetLastError(), "tc_corr");
}

// conv: x planar (region) -> R (complex64 and/or split planes), partial norms per CTA
hicu_status launch_conv_tc(hicu_handle* h, const ConvGeom& g, const uint4* xplanar, const void* bw, int p,
                           float2* R, uint4* Rs, double* partial, int* nblocks, cudaStream_t st) {
  TcPlan pl;
  if (!plan_tc_cached(&pl, g, 0, p, device_sms(h)))
    return set_error(h, HICU_ERR_UNSUPPORTED, "split-bf16 conv: geometry or filter bank does not fit the kernel");
  *nblocks = pl.grid;
  if (!partial) return HICU_OK;
  TcParams& P = pl.P;
  P.bw = (const unsigned char*)bw;
  P.R = R;
  P.Rs = Rs;
  P.r_plane = g.s;
  P.g = nullptr;
  P.m = nullptr;
  P.partial = partial;
  P.err = h->dev_err;
  return launch_plan(h, pl, xplanar, K_CONV_TC, st);
}

// adjoint: split planes of R -> masked g (region view), partial norms per CTA
hicu_status launch_adjoint_tc(hicu_handle* h, const ConvGeom& g, const uint4* Rs, const void* bw, int p,
                              MView m, KView gout, double* partial, int* nblocks, cudaStream_t st,
                              uint4* gsplit) {
  TcPlan pl;
  if (!plan_tc_cached(&pl, g, 1, p, device_sms(h)))
    return set_error(h, HICU_ERR_UNSUPPORTED,
                     "split-bf16 adjoint: geometry or filter bank does not fit the kernel");
  *nblocks = pl.grid;
  if (!partial) return HICU_OK;
  TcParams& P = pl.P;
  P.bw = (const unsigned char*)bw;
  P.R = nullptr;
  P.Rs = nullptr;
  P.g = gout.p;
  P.g_sc = gout.sc;
  P.m = m.p;
  P.m_sc = m.sc;
  const bool as2d = g.kz == 1 && g.ez == 1;
  // pseudo (z, y) strides: a 2D problem's rows are its planes
  P.g_sz = as2d ? gout.sy : gout.sz;
  P.g_sy = as2d ? 0 : gout.sy;
  P.g_base = (long long)gout.oz * gout.sz + (long long)gout.oy * gout.sy + gout.ox;
  P.m_sz = as2d ? m.sy : m.sz;
  P.m_sy = as2d ? 0 : m.sy;
  P.m_base = (long long)m.oz * m.sz + (long long)m.oy * m.sy + m.ox;
  P.gs = gsplit;
  P.gs_plane = (long long)g.ex * g.ey * g.ez;
  P.gs_ce = chunks_even_of(g.C);
  P.partial = partial;
  P.err = h->dev_err;
  return launch_plan(h, pl, Rs, K_ADJOINT_TC, st);
}

}  // namespace hicu
