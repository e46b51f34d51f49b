// Internal declarations shared by the libhicu translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <utility>
#include <string>
#include <vector>

#include "hicu.h"

namespace hicu {

// ------------------------------------------------------------------ views

// Read/write view of a complex64 k-space array.  Region coordinate (0,0,0)
// maps to element (c, oz, oy, ox); strides are in complex elements, x stride 1.
struct KView {
  float2* p;
  long long sc, sz, sy;
  int ox, oy, oz;
};

// Mask view: uint8, same addressing as KView with a coil stride (0 if shared).
struct MView {
  const uint8_t* p;  // nullptr = no mask
  long long sc, sz, sy;
  int ox, oy, oz;
};

// Geometry of one convolution problem on a region.
struct ConvGeom {
  int C;
  int kx, ky, kz, K;   // K = kx*ky*kz
  int n;               // C*K
  int ex, ey, ez;      // region extent
  int sx, sy, sz;      // valid-output extent
  int cx, cy, cz;      // circular flags
  long long s;         // sx*sy*sz
};

__host__ __device__ inline int wrap(int v, int m) {
  int r = v % m;
  return r < 0 ? r + m : r;
}

// ------------------------------------------------------------ reductions

template <int NT>
__device__ inline double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < NT / 32) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// Sum of v[0..n) by a CTA of 256 threads in a fixed order (the same in every CTA); thread 0 holds it.
__device__ inline double block_fixed_sum(const double* v, int n, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += v[i];
  return block_sum<256>(s, sh);
}

// ----------------------------------------------------- bounded grid barrier
// Used only inside cooperative launches (all CTAs co-resident).  Each wait
// gives up after `timeout_ns` and records HICU_ERR_TIMEOUT in *err.

struct GridSync {
  unsigned* count;
  unsigned* gen;
  int* err;
  unsigned nblocks;
  unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_acqrel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for cooperative kernels.  The count and generation words are zero at
// launch, so the k-th barrier (epoch k, counted by each CTA) completes when the generation
// reaches k + 1: arriving costs one atomic and waiting one acquire load per poll, with no
// extra round trip on the critical path.  The wait gives up after timeout_ns (or when
// another CTA recorded an error), records HICU_ERR_TIMEOUT and returns false in every thread
// of the CTA; the caller must then leave the kernel.
__device__ inline bool grid_sync(const GridSync& gs, unsigned& epoch) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = epoch + 1u;
    const unsigned old = atom_add_acqrel_u32(gs.count, 1u);
    if (old == gs.nblocks - 1) {
      *gs.count = 0u;
      st_release_u32(gs.gen, target);
    } else {
      unsigned long long t0 = 0;
      for (unsigned it = 0; ld_acquire_u32(gs.gen) != target; ++it) {
        if ((it & 255u) == 255u) {  // occasional checks keep them off the fast path
          const unsigned long long t = global_ns();
          if (t0 == 0) t0 = t;
          if (t - t0 > gs.timeout_ns || *((volatile int*)gs.err) != 0) {
            atomicExch(gs.err, (int)HICU_ERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  ++epoch;
  return s_ok != 0;
}

// Programmatic dependent launch: a kernel started with launch_pdl() may begin while the kernel
// before it on the stream is still running.  Such a kernel calls pdl_wait() before its first
// global-memory access (it returns once the preceding kernel has completed and its writes are
// visible; without the launch attribute it returns at once) and pdl_trigger() to let its own
// dependent start as early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------ host side

struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace hicu

// Launch a kernel through the handle's accounting (and event timing when its class is selected).
#define HICU_LAUNCH(h, cls, st, ...)  \
  do {                                 \
    hicu::prof_begin((h), (cls), (st)); \
    __VA_ARGS__;                       \
    hicu::prof_end((h), (cls), (st));   \
  } while (0)
// A launch on the side stream, concurrent with the caller's stream: counted, not event-timed (the
// class times add up the caller's stream; side work overlaps it).
#define HICU_LAUNCH_SIDE(h, cls, ...) \
  do {                                 \
    hicu::prof_count((h), (cls));      \
    __VA_ARGS__;                       \
  } while (0)

// The handle (opaque in the public header).
struct hicu_handle {
  int device = 0;
  int num_sms = 0;
  bool pdl = true;  // programmatic dependent launches (HICU_PDL=0 turns them off)
  std::string last_error;
  static constexpr int kSlots = 48;
  hicu::Workspace ws[kSlots];
  int* dev_err = nullptr;          // device error word
  unsigned* dev_sync = nullptr;    // grid-barrier words (count, gen)
  // warm-start state of the eigen-solver
  int64_t eig_n = 0;
  int eig_npad = 0;  // padded size of the stored eigenvectors (grid and cluster solvers pad differently)
  bool eig_have_v = false;
  int* eig_info = nullptr;  // device words of the last Jacobi run (sweeps, converged, buffer)
  // eigen-solver choice: largest n the size rule gives to the cluster solver
  int auto_cluster_max = HICU_NULLSPACE_CLUSTER_AUTO_MAX;
  // batch lanes: the cooperative (grid-barrier) launches of all lanes go to one shared
  // high-priority stream, in order, so that two of them never wait for each other's SMs and
  // their pending CTAs come first when SMs free up
  std::mutex* coop_mu = nullptr;     // guards the shared stream (owned by the batch parent)
  cudaStream_t coop_st = nullptr;    // shared stream (owned by the batch parent)
  cudaEvent_t coop_in = nullptr;     // this lane's work up to the launch
  cudaEvent_t coop_out = nullptr;    // the launch's completion
  std::mutex coop_mu_own;
  cudaStream_t coop_st_own = nullptr;
  // launch accounting and optional event timing of one kernel class
  int prof_class = -1;
  long long launches_all = 0;
  long long launches_class = 0;
  std::vector<cudaEvent_t> prof_events;
  size_t prof_used = 0;
  // side stream for work independent of the main chain inside one call (created on demand):
  // forked from and joined back to the caller's stream with events
  cudaStream_t side_st = nullptr;
  cudaEvent_t side_fork = nullptr;
  cudaEvent_t side_join = nullptr;
  cudaEvent_t draw_fork = nullptr;  // JL draws of an outer iteration
  cudaEvent_t draw_join = nullptr;
  // upload stream of hicu_reconstruct (created on demand): the part of a host input that the first
  // stages do not read, copied while they run
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_fork = nullptr;
  cudaEvent_t copy_join = nullptr;
  // l1 step (softdc.cu): the FFT plan (a cufftHandle) and the geometry key it was made for
  int fft_plan = 0;
  bool fft_have = false;
  long long fft_key[5] = {0, 0, 0, 0, 0};
  // kernel mask K (support.cu): host copy of the last mask whose maps sit in WS_SUP
  std::vector<uint8_t> sup_mask;
  int sup_nk = 0;
  // batch lanes (hicu_reconstruct_batched): one sub-handle and stream each, created on demand
  std::vector<hicu_handle*> lane_h;
  std::vector<cudaStream_t> lane_st;
  std::vector<cudaEvent_t> batch_ev;
};

namespace hicu {

enum Slot {
  WS_FT = 0,      // filters transposed for conv  [n][Ppad]
  WS_FA,          // filters transposed for adjoint [K][Ppad][Cpad]
  WS_PART,        // reduction partials (double)
  WS_STATS,       // internal stats double[8]
  WS_R,           // conv output R
  WS_G,           // gradient on the region
  WS_P,           // JL matrix
  WS_QF,          // Q in complex64
  WS_T,           // projector intermediate
  WS_BANK,        // filter bank [p][n]
  WS_GRAM_PART,   // Gram cell partial sums
  WS_EIG_A0,      // Jacobi ping
  WS_EIG_A1,      // Jacobi pong
  WS_EIG_V,       // eigenvectors
  WS_EIG_VPREV,   // previous eigenvectors (warm start)
  WS_EIG_PART,    // off-norm partials
  WS_EIG_TMP,     // GEMM temp for warm start
  WS_REC_G,       // reconstruct: Gram matrix
  WS_REC_Q,       // reconstruct: null basis
  WS_REC_EIG,     // reconstruct: eigenvalues
  WS_REC_X,       // reconstruct: staged x (host input)
  WS_REC_M,       // reconstruct: staged mask
  WS_REC_LOG,     // reconstruct: device log
  WS_REC_STATS,   // reconstruct: per-step stats
  WS_TC_X,        // split bf16 planes of the region input
  WS_TC_G,        // split bf16 planes of the gradient
  WS_TC_R,        // split bf16 planes of R
  WS_TC_BC,       // tensor-core B planes, conv
  WS_TC_BA,       // tensor-core B planes, adjoint
  WS_FGRAD,       // filter-gradient partials per CTA
  WS_EIG_WY,      // principal subspace: compact WY blocks of the back-transformation
  WS_REC_P,       // reconstruct: JL matrices of one outer iteration's descent steps
  WS_SUP,         // kernel mask maps: support offset -> box offset, box offset -> support offset or -1
  WS_BANK_SUP,    // reconstruct: filter bank on the support of K [p][C][|K|]
  WS_REC_X0,      // reconstruct: the observed data X0, kept for soft data consistency / the l1 step
  WS_QPLUS,       // reconstruct: the augmenting null vectors Q0 in complex64
  WS_RS_OMEGA,    // randomized SVD: test vectors [l][n] (complex128)
  WS_RS_G,        // randomized SVD: the Gram G of the region (n x n complex128)
  WS_RS_Y,        // randomized SVD: Y = Z + nu Omega
  WS_RS_K,        // randomized SVD: K = Y R^-1
  WS_RS_T,        // randomized SVD: l x l matrices
  WS_RS_U,        // randomized SVD: top eigenvectors of K^H K
  WS_RS_SCAL,     // randomized SVD: eigenvalues and scalars
  WS_COUNT
};
static_assert(WS_COUNT <= hicu_handle::kSlots, "workspace slots");

// Kernel classes for launch accounting / event timing (hicu_kernel_class in hicu.h).
enum KClass { K_GRAM = 0, K_EIG = 1, K_CONV = 2, K_ADJOINT = 3, K_JL = 4, K_MISC = 5, K_CONV_TC = 6,
              K_ADJOINT_TC = 7, K_TRIDIAG = 8 };
void prof_begin(hicu_handle* h, int cls, cudaStream_t st);
void prof_count(hicu_handle* h, int cls);
void prof_end(hicu_handle* h, int cls, cudaStream_t st);

// Launch through the handle's accounting as a programmatic dependent of the previous kernel on
// st (the kernel must call pdl_wait() before touching global memory).  allow = false, or the
// handle's switch off: an ordinary stream-ordered launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(hicu_handle* h, int cls, cudaStream_t st, dim3 grid, dim3 block, size_t smem,
                       void (*kernel)(KArgs...), bool allow, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (allow && h->pdl) ? 1 : 0;
  prof_begin(h, cls, st);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  prof_end(h, cls, st);
  return e;
}

// Raise a kernel's dynamic shared-memory cap to the device's opt-in maximum, once per
// kernel and device (thread-safe).  Never set per launch: host threads launching the same
// kernel with different sizes would race on the attribute.
cudaError_t allow_max_dynamic_smem(const void* kernel);
hicu_status set_error(hicu_handle* h, hicu_status s, const std::string& msg);
hicu_status cuda_error(hicu_handle* h, cudaError_t e, const char* where);
void* ws_get(hicu_handle* h, int slot, size_t bytes, hicu_status* st);

// Validation + device geometry.
hicu_status make_conv_geom(hicu_handle* h, const hicu_geom* g, const hicu_region* r,
                           ConvGeom* out);
KView full_view(const hicu_geom* g, const hicu_region* r, float* base);
MView mask_view(const hicu_geom* g, const hicu_region* r, const uint8_t* mask);

// Kernel launchers (stream = cudaStream_t).
hicu_status launch_prep_filters(hicu_handle* h, const ConvGeom& g, const float2* bank, int p,
                                float2* fT, int Ppad, float2* fA, int Cpad, cudaStream_t st);
int conv_ppad(int p);
int adj_cpad(int C);
hicu_status launch_conv_fp32(hicu_handle* h, const ConvGeom& g, KView x, const float2* fT, int p,
                             int Ppad, float2* R, double* partial, int* nblocks, cudaStream_t st);
// Launch shape of conv_fp32_kernel (grid, block, dynamic shared memory) for a geometry.
void conv_fp32_launch_shape(const ConvGeom& g, dim3* grid, dim3* block, size_t* smem);
__global__ void prep_filters_kernel(ConvGeom g, const float2* __restrict__ bank, int p,
                                    float2* __restrict__ fT, int Ppad, float2* __restrict__ fA,
                                    int Cpad);
__global__ void conv_fp32_kernel(ConvGeom g, KView x, const float2* __restrict__ fT, int p, int Ppad,
                                 float2* __restrict__ R, double* __restrict__ partial);
__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double* out);
hicu_status launch_adjoint_fp32(hicu_handle* h, const ConvGeom& g, const float2* R,
                                const float2* fA, int p, int Ppad, int Cpad, MView m, KView gout,
                                double* partial, int* nblocks, cudaStream_t st);
hicu_status launch_sum_partials(hicu_handle* h, const double* partial, int n, double* out,
                                cudaStream_t st);
// finalisation (stats = {eta, objective, ||g||^2, D} from the partials) and update in one launch
hicu_status launch_update_step(hicu_handle* h, const ConvGeom& g, KView y, KView gb, MView m, const double* part,
                               int n_obj, int n_g, int n_d, double* stats, cudaStream_t st);
// tensor-core (split-bf16) path: 2D and 3D, valid or circular along the outer axis
bool tc_supported(const ConvGeom& g);
size_t tc_b_bytes(const ConvGeom& g, int p, int mode);
size_t tc_x_bytes(const ConvGeom& g);          // split planes of a region input
size_t tc_r_bytes(const ConvGeom& g, int p);   // split planes of R
// B operands of the conv and / or the adjoint (nullptr: not wanted) from one filter bank, one launch
hicu_status tc_prepare_weights(hicu_handle* h, const ConvGeom& g, const float2* bank, int p, void* out_conv,
                               void* out_adjoint, cudaStream_t st);
hicu_status tc_prepare_input(hicu_handle* h, const ConvGeom& g, KView x, uint4* planar, cudaStream_t st);
// finalisation and update of a descent step that also writes the updated region of y as split
// input planes (the layout of tc_prepare_input)
hicu_status launch_update_step_planes(hicu_handle* h, const ConvGeom& g, KView y, KView gb, MView m,
                                     const double* part, int n_obj, int n_g, int n_d, double* stats, uint4* planar,
                                     cudaStream_t st);
hicu_status tc_prepare_r(hicu_handle* h, const ConvGeom& g, const float2* R, int p, uint4* planar,
                         cudaStream_t st);
hicu_status launch_conv_tc(hicu_handle* h, const ConvGeom& g, const uint4* xplanar, const void* bw, int p,
                           float2* R, uint4* Rs, double* partial, int* nblocks, cudaStream_t st);
// gsplit (nullable): also write the masked g as split input planes for the next convolution
hicu_status launch_adjoint_tc(hicu_handle* h, const ConvGeom& g, const uint4* Rs, const void* bw, int p,
                              MView m, KView gout, double* partial, int* nblocks, cudaStream_t st,
                              uint4* gsplit = nullptr);

hicu_status launch_jl(hicu_handle* h, int64_t n, int64_t nr, int p, const double* Q, int mode,
                      const double* P, uint64_t seed, uint64_t counter, float* bank,
                      cudaStream_t st);
// the same in two parts: Q (complex128 [nr][n]) to complex64 in the handle's workspace, then the
// compression from that copy (the reconstruction driver converts once per outer iteration)
hicu_status jl_convert_q(hicu_handle* h, int64_t n, int64_t nr, const double* Q, float2** Qf, cudaStream_t st);
// P: the caller's JL matrix (double, rows x p) or nullptr; Pdrawn: a float copy drawn beforehand
// (jl_draw) or nullptr, else P is drawn here from (seed, counter)
// pdl: the launch may overlap the previous kernel on st (false after a cross-stream wait)
hicu_status launch_jl_converted(hicu_handle* h, int64_t n, int64_t nr, int p, const float2* Qf, int mode,
                                const double* P, const float* Pdrawn, uint64_t seed, uint64_t counter,
                                float* bank, cudaStream_t st, bool pdl = false);
// JL matrices of nsteps consecutive draws (counters counter .. counter + nsteps - 1), each
// rows x p, into P (float, draw-major)
hicu_status jl_draw(hicu_handle* h, int64_t rows, int p, int nsteps, uint64_t seed, uint64_t counter, float* P,
                    cudaStream_t st);
// the rows x rows identity as a JL matrix (no compression: the exact gradient)
hicu_status jl_identity(hicu_handle* h, int64_t rows, float* P, cudaStream_t st);
// bank [p][n] += Q+ P2 for Q+ = blockdiag(Q0, ...): Q0f complex64 [m0][n0], P2 float [blocks m0][p]
hicu_status launch_jl_qplus(hicu_handle* h, int p, int64_t n, int n0, int m0, const float2* Q0f, const float* P2,
                            float* bank, cudaStream_t st);
// the handle's side stream and its events, created on first use
hicu_status ensure_side_stream(hicu_handle* h);
// planes_valid: the split planes of y on this region are current (TC path); keep_planes: the update
// leaves them current for the next step
hicu_status gd_step_filters(hicu_handle* h, const hicu_geom* geom, const hicu_region* region, float* y,
                            const uint8_t* mask, const float* filters, int32_t p, double* stats,
                            int32_t prec, cudaStream_t st,
                            bool planes_valid = false, bool keep_planes = false);

// sup (device, nk entries): the box offsets of a kernel mask's support; G is then (C nk) x (C nk)
// over the support's coefficients (nullptr: the whole box)
hicu_status run_gram(hicu_handle* h, const hicu_geom* geom, const hicu_region* reg, const float* x,
                     double* G, cudaStream_t st, const int* sup = nullptr, int nk = 0);
// kernel mask maps in the handle's workspace for a HOST mask [kz][ky][kx] (support.cu): *sup[nk]
// box offsets of the support, *inv[K] support index of each box offset or -1; re-uploaded only
// when the mask differs from the previous one
hicu_status support_maps(hicu_handle* h, const hicu_geom* geom, const uint8_t* kmask, const int** sup,
                         const int** inv, int* nk, cudaStream_t st);
// soft data consistency (softdc.cu): g += lambda M o (y - X0) on the region (gb), per-CTA partials of
// lambda ||M o (y - X0)||^2, ||g||^2 and lambda ||M o g||^2; part_dc == nullptr: sizing only
hicu_status launch_soft_dc(hicu_handle* h, const ConvGeom& g, KView gb, KView y, KView x0, MView m, double lam,
                           double* part_dc, double* part_g, double* part_mg, int* nblocks, cudaStream_t st);
// the l1 proximal step on the whole array (in place), and the restore of the observed samples
hicu_status run_soft_threshold(hicu_handle* h, const hicu_geom* geom, float* x, double tau, cudaStream_t st);
hicu_status launch_restore_observed(hicu_handle* h, const hicu_geom* geom, float* y, const float* x0,
                                    const uint8_t* mask, cudaStream_t st);
void release_fft(hicu_handle* h);
// one descent step with soft data consistency (abi.cu)
hicu_status gd_step_filters_soft(hicu_handle* h, const hicu_geom* geom, const hicu_region* region, float* y,
                                 const uint8_t* mask, const float* x0, double lam, const float* filters, int32_t p,
                                 double* stats, int32_t prec, cudaStream_t st);
// randomized SVD (rsvd.cu) and its helpers: test vectors (jl.cu), complex128 -> complex64 (jl.cu),
// box -> support coefficients (support.cu)
hicu_status run_rsvd(hicu_handle* h, const hicu_geom* geom, const hicu_region* region, const uint8_t* kmask,
                     const float* x, int64_t r, int64_t l, const double* V_prev, int64_t r0, uint64_t seed,
                     uint64_t counter, double* V, double* eig_top, double* tail, cudaStream_t st);
hicu_status launch_rsvd_omega(hicu_handle* h, int64_t n, int64_t l, int64_t r0, const double* V_prev, uint64_t seed,
                              uint64_t counter, double2* Om, cudaStream_t st);
hicu_status launch_support_gather(hicu_handle* h, int p, int C, int K, int nk, const int* sup,
                                  const float2* bank_box, float2* bank_sup, cudaStream_t st);
// bank_box[k][c][kbox] = bank_sup[k][c][inv[kbox]] (zero off the support)
hicu_status launch_support_scatter(hicu_handle* h, int p, int C, int K, int nk, const int* inv,
                                   const float2* bank_sup, float2* bank_box, cudaStream_t st);
// cluster Jacobi (eig_cluster.cu): cluster size for an n x n solve (0: use the grid solver),
// its padded size, and the solve itself on a prepared A0 / V0
int cluster_eig_ctas(int64_t n);
int cluster_eig_npad(int64_t n, int nct);
hicu_status run_nullspace_cluster(hicu_handle* h, int n, int npad, int nct, int64_t r, const double2* A0,
                                  const double2* V0, double2* Vout, double* Q, double* eigvals, int flags,
                                  cudaStream_t st);
__global__ void eig_gather_q_kernel(int n, int npad, int nr, const double2* __restrict__ V,
                                    const int* __restrict__ rank, double2* __restrict__ Q);
hicu_status run_nullspace(hicu_handle* h, int64_t n, int64_t r, const double* G, double* Q,
                          double* eigvals, int flags, cudaStream_t st);
// principal subspace by tridiagonalisation (eig_tridiag.cu): V [r][n], eig_top [r] ascending,
// eig_all [n] (nullable), J = trace(G) - sum(eig_top) (nullable)
hicu_status run_principal(hicu_handle* h, int64_t n, int64_t r, const double* G, double* V, double* eig_top,
                          double* eig_all, double* J, cudaStream_t st);
// shared with the Jacobi solver (eig.cu): largest |Re|, |Im| and the exact power-of-two pre-scale
__global__ void eig_absmax_kernel(long long nn, const double2* __restrict__ A, unsigned long long* amax_bits);
__global__ void eig_scale_kernel(long long nn, double2* __restrict__ A, const unsigned long long* amax_bits,
                                 double* scale_out);

}  // namespace hicu
