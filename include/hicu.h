/*
 * hicu.h - C ABI of libhicu, a GB300 (sm_103a) library for the hot path of
 * HICU, the calibrationless MRI reconstruction of Zhao, Potter & Ahmad
 * ("High-dimensional fast convolutional framework (HICU) for calibrationless
 * MRI", Magn. Reson. Med. 2021).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Complex numbers are interleaved (re, im) pairs: complex64 = 2 floats,
 *    complex128 = 2 doubles.
 *  - k-space x: complex64, shape [C][Nz][Ny][Nx] (x fastest, coil slowest).
 *    2D uses Nz = 1; 2D+t puts time in the Nz slot.  k-space is centred.
 *  - sampling mask M: uint8 (0 = unobserved, nonzero = observed), shape
 *    [Nz][Ny][Nx] shared by all coils, or [C][Nz][Ny][Nx] when
 *    geom.mask_per_coil = 1 (multi-shot channel stacks).
 *  - kernel support K is rectangular over all C coils (Theory section: a
 *    kernel of size Nc along the coil axis makes the convolution sum over
 *    coils), so n = C*kz*ky*kx.  A filter is n complex64 values ordered
 *    [C][kz][ky][kx]; a bank of p filters is [p][C][kz][ky][kx].
 *  - H(x) is the multi-level Hankel matrix of the Theory section; row p of
 *    H(x) is the patch x_c[p + d] over (c, d) in filter order, so H(x) v is
 *    the valid convolution of x with v (correlation form).  It is never
 *    formed.
 *  - region S = (off, ext) per axis (x, y, z), the centre-out region of
 *    Algorithm 1 step 4.  Valid outputs are the positions whose whole kernel
 *    footprint lies inside S, s = prod(ext - k + 1); an axis flagged circular
 *    wraps modulo ext and contributes ext outputs (2D+t time axis, Methods,
 *    Study II).  Nothing outside S is read or written.
 *  - R, the output of the convolution with a bank of p filters, is complex64
 *    [sz][sy][sx][p] (valid outputs in (z, y, x) order, filter fastest).
 *  - All data pointers are DEVICE pointers owned by the caller unless a call
 *    says otherwise; the library never frees them.  Scratch memory belongs to
 *    the handle, which grows it on demand with cudaMalloc.
 *  - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *    void*, NULL = legacy default stream) unless documented otherwise.  They
 *    return a hicu_status and never abort; hicu_last_error() gives the text.
 *  - Errors found on the device (a bounded wait that gave up, a non-finite
 *    value) are recorded in a device word of the handle and reported by
 *    hicu_check(), which synchronises the stream.
 *  - A handle belongs to the device that was current at hicu_create(); use
 *    it from one host thread at a time.
 */
#ifndef HICU_H_
#define HICU_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hicu_handle hicu_handle;

typedef enum {
  HICU_OK = 0,
  HICU_ERR_ARG = 1,         /* null pointer, bad enum or flag */
  HICU_ERR_SHAPE = 2,       /* geometry / region / layout inconsistent */
  HICU_ERR_RANK = 3,        /* r outside (0, n), p outside [1, n-r] */
  HICU_ERR_ALLOC = 4,       /* workspace allocation failed */
  HICU_ERR_CUDA = 5,        /* a CUDA runtime call or launch failed */
  HICU_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
  HICU_ERR_NUMERIC = 7,     /* non-finite value met on the device */
  HICU_ERR_UNSUPPORTED = 8  /* valid request this build does not handle */
} hicu_status;

typedef enum {
  HICU_FP32 = 0,        /* complex FP32 on CUDA cores (plain form) */
  HICU_SPLIT_BF16 = 1   /* tcgen05 tensor cores, hi+lo bf16 split, FP32 accumulate */
} hicu_prec;

typedef enum {
  HICU_JL_NULLSPACE = 0,  /* Q~ = Q P, P is (n-r) x p  (Algorithm 1 step 6) */
  HICU_JL_PROJECTOR = 1,  /* Q~ = Q (Q^H P), P is n x p: depends only on span(Q) */
  HICU_JL_COMPLEMENT = 2  /* Q~ = P - V (V^H P) from the r principal vectors V: the same
                             filters as HICU_JL_PROJECTOR (I - V V^H = Q Q^H), same draws of P */
} hicu_jl;

/* Kernel classes for launch accounting and event timing (hicu_profile_*). */
typedef enum {
  HICU_K_GRAM = 0,       /* Gram cross-correlation kernels */
  HICU_K_EIG = 1,        /* Jacobi eigen-solver */
  HICU_K_CONV = 2,       /* FP32 valid convolution */
  HICU_K_ADJOINT = 3,    /* FP32 masked adjoint */
  HICU_K_JL = 4,         /* JL draw and compression */
  HICU_K_MISC = 5,       /* layout, reductions, update, sorting */
  HICU_K_CONV_TC = 6,    /* tensor-core convolution */
  HICU_K_ADJOINT_TC = 7, /* tensor-core adjoint */
  HICU_K_TRIDIAG = 8     /* Householder tridiagonalisation (principal subspace) */
} hicu_kernel_class;

typedef struct {
  int64_t dim[3];        /* Nx, Ny, Nz */
  int32_t ncoil;         /* C (channels; shots stacked as channels count here) */
  int32_t k[3];          /* kernel extent kx, ky, kz (1 for an unused axis) */
  uint8_t circular[3];   /* per axis: 0 = valid convolution, 1 = circular */
  uint8_t mask_per_coil; /* 0: mask [Nz][Ny][Nx]; 1: mask [C][Nz][Ny][Nx] */
} hicu_geom;

typedef struct {
  int64_t off[3];        /* first index of S along x, y, z */
  int64_t ext[3];        /* extent of S along x, y, z */
} hicu_region;

/* One centre-out stage (Algorithm 1 steps 4-8 repeated `iters` times). */
typedef struct {
  hicu_region region;    /* S^(i) for the iterations of this stage */
  int32_t iters;         /* outer iterations in this stage */
  int32_t gd_steps;      /* G^(i): descent steps per outer iteration */
  int32_t p;             /* JL compression dimension */
} hicu_stage;

typedef struct {
  int64_t rank;              /* r */
  int32_t nstages;
  const hicu_stage* stages;  /* host array of nstages entries */
  uint64_t seed;             /* JL generator seed */
  int32_t jl;                /* hicu_jl */
  int32_t prec;              /* hicu_prec for the convolutions */
  int32_t gram_on_current;   /* 0: null space of H^(i-1) (Algorithm 1 step 2 as
                                printed, S^(0) := S^(1)); 1: use S^(i) */
  int32_t init;              /* 0: x^(0) = X0; 1: time-averaged along z (2D+t) */
  int32_t eig_solver;        /* null-space solver: 0 = HICU_NULLSPACE_TRIDIAG when jl is
                                HICU_JL_PROJECTOR (the principal vectors V, then
                                HICU_JL_COMPLEMENT filters), else Jacobi by size;
                                HICU_NULLSPACE_GRID or HICU_NULLSPACE_CLUSTER force
                                Jacobi (see hicu_nullspace); HICU_NULLSPACE_TRIDIAG
                                needs jl = HICU_JL_PROJECTOR */
  const uint8_t* kernel_mask;/* kernel mask K: HOST array [kz][ky][kx] of the box geom.k,
                                nonzero = in the support (Algorithm 1 input; Discussion:
                                circular or spherical masks); NULL = the whole box.  The
                                null space then has n = C |K| coefficients (see
                                hicu_gram_support) */
  double dc_weight;          /* lambda of the soft data-consistency cost lambda ||M o X - X0||^2
                                (Theory, Eq. 3); 0 = hard data consistency (observed samples
                                never move).  Steps as hicu_gd_step_soft */
  double l1_threshold;       /* tau of the l1 step hicu_soft_threshold after every descent step of
                                a stage whose region is the whole array (Discussion); 0 = off.
                                Under hard data consistency the observed samples are restored
                                after it */
  int32_t jl_exact;          /* 1: no JL compression (the stages' p are ignored): every descent step
                                uses the whole null space, Q~ = Q (HICU_JL_NULLSPACE, n - r
                                filters) or Q~ = I - V V^H (the principal-subspace route, n
                                filters; the same Q~ Q~^H = Q Q^H), i.e. the exact gradient of
                                ||H(y) Q||^2; 0: JL draws (Algorithm 1 step 6).  A bank
                                that large exceeds the split-BF16 adjoint's shared memory
                                (at most 64 filters of a 5 x 5 kernel, 8 of a 5 x 5 x 5):
                                HICU_ERR_UNSUPPORTED there, use HICU_FP32 */
  const double* qplus;       /* augmented null space [Q | Q+] of Algorithm 1 step 3 (Methods,
                                Study IV): Q0, complex128 [qplus_cols][n / qplus_blocks]
                                (DEVICE; row j a null vector of one channel group's Hankel
                                matrix, e.g. of the b0 scan: hicu_gram + hicu_nullspace), and
                                Q+ = blockdiag(Q0, ..., Q0) over qplus_blocks consecutive equal
                                groups of channels (the shots).  Each JL matrix gets
                                qplus_blocks * qplus_cols more rows, which multiply Q+
                                (Q~ = [Q | Q+] P).  NULL = no augmentation */
  int32_t qplus_cols;        /* columns of Q0 */
  int32_t qplus_blocks;      /* diagonal blocks of Q+ (must divide the channel count) */
  int32_t rsvd_cols;         /* eig_solver HICU_NULLSPACE_RSVD: test vectors l (0: min(n, r +
                                max(r/2, 8))); the previous iteration's r principal vectors are
                                the first r of them after the first outer iteration */
  uint64_t rsvd_seed;        /* its Gaussian test vectors: draw counter = outer iteration index */
} hicu_params;

/* Optional per-iteration log, HOST arrays (any may be NULL). */
typedef struct {
  double* J;          /* per outer iteration: sum of the n-r smallest eigenvalues (Eq. 1) */
  double* objective;  /* per descent step: ||H(y) Q~||_F^2 before the step */
  double* eta;        /* per descent step: exact line-search step size */
} hicu_log;

/* ---------------------------------------------------------------- handle */

/* Create a handle on the current CUDA device.  *out receives the handle. */
hicu_status hicu_create(hicu_handle** out);
/* Release the handle and its workspace (synchronises the device). */
hicu_status hicu_destroy(hicu_handle* h);
/* Text of the last error on this handle ("" if none).  Owned by the handle. */
const char* hicu_last_error(const hicu_handle* h);
/* Static name of a status code. */
const char* hicu_status_string(hicu_status s);
/* Synchronise `stream`, then report (and clear) any device-side error word. */
hicu_status hicu_check(hicu_handle* h, void* stream);

/*
 * Tracing: every kernel the library launches is counted; launches of one
 * selected class (hicu_kernel_class, -1 = none) are also bracketed by CUDA
 * events recorded on the launch stream, except launches on the handle's side
 * stream (work that overlaps the caller's stream: the JL draws of an outer
 * iteration, the compact-WY factors), which are counted but not timed, so that
 * the class times add up the caller's stream.  hicu_profile_select() resets the
 * counters; hicu_profile_read() synchronises on the last event and returns the
 * summed device time (ms) of the timed launches, their number, and the number
 * of launches of every class since the last select/read, then resets.
 */
hicu_status hicu_profile_select(hicu_handle* h, int32_t kernel_class);
hicu_status hicu_profile_read(hicu_handle* h, double* total_ms, int64_t* class_launches,
                              int64_t* all_launches);
/* Jacobi sweeps run by all hicu_nullspace calls since the last read (synchronises, resets). */
hicu_status hicu_profile_eig_sweeps(hicu_handle* h, int64_t* sweeps);

/* Filter length n = C*kx*ky*kz, or -1 for an invalid geometry. */
int64_t hicu_filter_length(const hicu_geom* geom);
/* Number of valid outputs s of region S, or -1 if S does not fit the geometry. */
int64_t hicu_num_outputs(const hicu_geom* geom, const hicu_region* region);

/* ------------------------------------------------------------ hot path */

/*
 * hicu_gram - G = H(x)^H H(x) on region S (Eq. 1: the eigenvalues of G are the
 * squared singular values of H; the Discussion names SVD of this Gram matrix
 * as the alternative to rSVD for Algorithm 1 step 2).
 *   x : complex64 k-space [C][Nz][Ny][Nx]
 *   G : complex128 n x n, row-major: G[a*n + b] = sum_p conj(h_p[a]) h_p[b]
 * Products of the FP32 inputs are formed exactly and accumulated in
 * double-word arithmetic; entries are computed by multi-coil cross-correlation
 * (one correlation per coil pair and lag), never from H itself.
 */
hicu_status hicu_gram(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                      const float* x, double* G, void* stream);

/* flags of hicu_nullspace */
#define HICU_NULLSPACE_WARM 1   /* start from the previous call's eigenvectors (same n) */
#define HICU_NULLSPACE_SPLIT 2  /* stop once the top-r / bottom n-r split has converged */
#define HICU_NULLSPACE_GRID 4    /* grid-wide FP64 solver */
#define HICU_NULLSPACE_CLUSTER 8 /* one-cluster double-float solver (n <= 256) */
/* without either flag: the cluster solver for n <= HICU_NULLSPACE_CLUSTER_AUTO_MAX, else the grid one */
#define HICU_NULLSPACE_CLUSTER_AUTO_MAX 128
/* hicu_params.eig_solver only: principal subspace by tridiagonalisation (hicu_principal_subspace) */
#define HICU_NULLSPACE_TRIDIAG 16
/* hicu_params.eig_solver only: principal vectors by randomized SVD with a warm start
   (hicu_principal_rsvd; no Gram matrix), needs jl = HICU_JL_PROJECTOR */
#define HICU_NULLSPACE_RSVD 32

/*
 * Kernel masks.  Algorithm 1 takes a {0,1} kernel mask K; a filter v lists the kernel values on
 * its support (Theory section), so n = C |K| coefficients ordered [c][support offset], the
 * offsets of the support in scan order of the box [kz][ky][kx] (dx fastest).  The Gram matrix,
 * null space and JL filters of a masked problem are of that length; the convolution calls take
 * filters in the box layout, zero off the support (hicu_expand_filters).  A mask is a HOST array
 * [kz][ky][kx] of uint8 (nonzero = in the support) over the box geom.k; the handle keeps its index
 * maps and uploads them again only when the mask changes.
 */

/* C |K| for the kernel mask, or -1 for an invalid geometry or an empty mask (host only). */
int64_t hicu_support_length(const hicu_geom* geom, const uint8_t* kmask);

/*
 * hicu_gram_support - G = H_K(x)^H H_K(x) for the masked Hankel matrix (columns (c, d) with d on
 * the support of K; Eq. 1 then holds for H_K).  The same cross-correlation sums as hicu_gram;
 * only the support's rows and columns are assembled.
 *   kmask : HOST [kz][ky][kx] kernel mask;  x : complex64 k-space (device)
 *   G     : complex128 (C |K|) x (C |K|) row-major (device)
 * HICU_ERR_SHAPE for an empty mask.
 */
hicu_status hicu_gram_support(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                              const uint8_t* kmask, const float* x, double* G, void* stream);

/*
 * hicu_expand_filters - bank_box[k][c][kz][ky][kx] = the coefficient of offset (kz, ky, kx) of
 * bank_sup[k][c][.] on the support of K, zero off the support: filters on a kernel mask in the
 * layout of the convolution calls.
 *   kmask    : HOST [kz][ky][kx] kernel mask
 *   bank_sup : complex64 [p][C |K|] (device);  bank_box : complex64 [p][C kz ky kx] (device)
 */
hicu_status hicu_expand_filters(hicu_handle* h, const hicu_geom* geom, const uint8_t* kmask,
                                const float* bank_sup, int32_t p, float* bank_box, void* stream);

/*
 * hicu_nullspace - eigen-decomposition of the Hermitian n x n matrix G and the
 * null-space basis Q spanned by the eigenvectors of its n-r smallest
 * eigenvalues (Algorithm 1 steps 2-3: Q is an orthonormal basis of the
 * orthogonal complement of the r principal right singular vectors of H).
 * Parallel cyclic Jacobi on the GPU, by one of two solvers:
 *   cluster: one thread-block cluster (16 or 8 SMs) holds the matrix in
 *     distributed shared memory and computes in double-float (FP32 pairs,
 *     ~2^-48 relative precision; inputs and outputs FP64).  n <= 256.  It
 *     leaves the other SMs free, so independent solves on separate streams run
 *     side by side.
 *   grid: one cooperative FP64 kernel over the whole GPU (bounded grid
 *     barriers; a barrier that times out sets the handle's device error word).
 * HICU_NULLSPACE_CLUSTER / HICU_NULLSPACE_GRID choose one (both: HICU_ERR_ARG;
 * CLUSTER for n > 256 or on a device that cannot run the cluster:
 * HICU_ERR_UNSUPPORTED); without either, n <= HICU_NULLSPACE_CLUSTER_AUTO_MAX
 * uses the cluster solver.
 *   G       : complex128 n x n row-major, Hermitian (only read)
 *   Q       : complex128 [(n-r)][n]: null vector j is Q[j*n .. j*n+n-1],
 *             ordered by ascending eigenvalue
 *   eigvals : double [n], ascending (nullable)
 *   flags   : HICU_NULLSPACE_WARM: start from V^H G V with V the previous
 *             call's eigenvectors (ignored if there is none of the same n
 *             and solver).
 *             HICU_NULLSPACE_SPLIT: stop as soon as the coupling between the
 *             r largest diagonal entries and the others is below 1e-8 ||G||_F
 *             (full decomposition: every off-diagonal entry, 1e-11 ||G||_F).  Q then spans
 *             the null space to within 1e-8 ||G|| / gap, but its vectors need not be
 *             individual eigenvectors and the n-r smallest eigvals are diagonal
 *             entries of a not fully diagonalised block (their sum, J of
 *             Eq. 1, is still exact).  Algorithm 1 step 3 needs only the span.
 * Eigenvectors are unique only up to a unit phase (and rotations inside
 * repeated eigenvalues).
 */
hicu_status hicu_nullspace(hicu_handle* h, int64_t n, int64_t r, const double* G, double* Q,
                           double* eigvals, int32_t flags, void* stream);

/*
 * hicu_principal_subspace - the r principal eigenvectors V of the Hermitian n x n
 * matrix G (Algorithm 1 step 2 in Gram form: the r principal right singular
 * vectors of H are the eigenvectors of G = H^H H for its r largest
 * eigenvalues; the null space of step 3 is their orthogonal complement, which
 * HICU_JL_COMPLEMENT uses without forming it).
 * Householder tridiagonalisation G = Q_H T Q_H^H (one barrier per reflector: a
 * 16-CTA cluster with the matrix in shared memory for n <= 416, else a
 * cooperative kernel over all SMs with a bounded grid barrier), multisection on
 * Sturm counts for the eigenvalues of T, inverse iteration for its r top
 * eigenvectors (eigenvalues closer than 1e-10 ||G|| are orthogonalised against
 * each other) and the reflectors applied to them in compact-WY blocks.
 * Double-float arithmetic (an unevaluated sum of two FP32 numbers, unit roundoff
 * 2^-48) on the FP32 pipes; the input is pre-scaled by a power of two; inputs and
 * outputs FP64.  Eigenvalues are accurate to ~1e-14 ||G|| (absolute) and span(V)
 * to ~1e-14 ||G|| / (lambda_r - lambda_{r+1}).
 *   n       : 2 .. 4096;  r : 1 .. n-1  (else HICU_ERR_SHAPE / HICU_ERR_RANK)
 *   G       : complex128 n x n row-major, Hermitian (only read)
 *   V       : complex128 [r][n]: row j is the eigenvector of eig_top[j]
 *   eig_top : double [r], the r largest eigenvalues, ascending
 *   eig_all : double [n], all eigenvalues ascending (nullable; costs one more
 *             bisection pass)
 *   tail    : device double, J = trace(G) - sum(eig_top), the tail energy of
 *             Eq. 1 (nullable)
 * All pointers are device pointers owned by the caller.  Scratch lives in the
 * handle.  Eigenvectors are unique only up to a unit phase (and rotations
 * inside repeated eigenvalues).
 */
hicu_status hicu_principal_subspace(hicu_handle* h, int64_t n, int64_t r, const double* G, double* V,
                                    double* eig_top, double* eig_all, double* tail, void* stream);

/*
 * hicu_principal_rsvd - the r principal right singular vectors of H(x) on S by randomized SVD
 * (Theory: rSVD; Algorithm 1 step 2), without an n x n eigendecomposition.  l test vectors Omega:
 * the r0 rows of V_prev (a warm start, e.g. the previous outer iteration's V), then complex
 * Gaussian vectors, entry a of vector r0 + b being (z(2e) + i z(2e + 1)) / sqrt(2),
 * e = a (l - r0) + b, z the counter-based generator of hicu_jl_compress with (seed, counter).
 * Z = H^H H Omega is formed as G Omega from the region's Gram G = H^H H (as hicu_gram, double-word
 * sums) in double-float arithmetic; then the single-pass randomized SVD of H through H^H H with a
 * stabilising shift nu = 2^-17 ||Z||_F / sqrt(l):
 *   Y = Z + nu Omega, Omega^H Y = R^H R (Cholesky), K = Y R^-1, V = the top r left singular
 *   vectors of K, eig_top = their squared singular values - nu.
 * Exact when rank(H) <= l.  The Cholesky factor is formed by one CTA in double-float (about
 * l^3 / 6 complex multiply-adds: tens of microseconds at l ~ 100, milliseconds at l in the
 * hundreds).  Workspace: n x n complex128 for G plus O(l n).
 *   kmask   : optional HOST kernel mask (NULL = the whole box); n = C |K| or C kx ky kz
 *   r, l    : 1 <= r < l <= min(n, 4096);  V_prev : complex128 [r0][n] (device), r0 <= l
 *   V       : complex128 [r][n] (device) row j the vector of eig_top[j] (ascending); may be V_prev
 *   tail    : optional device double, J = trace(H^H H) - sum(eig_top) (Eq. 1)
 * HICU_ERR_NUMERIC (via hicu_check) if the Cholesky factorisation meets a non-positive pivot.
 */
hicu_status hicu_principal_rsvd(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                const uint8_t* kmask, const float* x, int64_t r, int64_t l, const double* V_prev,
                                int64_t r0, uint64_t seed, uint64_t counter, double* V, double* eig_top,
                                double* tail, void* stream);

/*
 * hicu_nullspace_info - sweeps used by the last hicu_nullspace call on this
 * handle and how it converged: 0 = not within the sweep limit, 1 = full
 * decomposition, 2 = split criterion (synchronises the device).
 */
hicu_status hicu_nullspace_info(hicu_handle* h, int32_t* sweeps, int32_t* converged);

/*
 * hicu_jl_compress - Q~ = Q P with P i.i.d. N(0, 1/p) (Algorithm 1 step 6;
 * Theory, JL paragraph).
 *   Q       : complex128 [(nr)][n] null basis as returned by hicu_nullspace, or,
 *             with HICU_JL_COMPLEMENT, the nr = r principal vectors of
 *             hicu_principal_subspace
 *   mode    : HICU_JL_NULLSPACE (P is nr x p), HICU_JL_PROJECTOR (P is n x p,
 *             Q~ = Q (Q^H P)) or HICU_JL_COMPLEMENT (P is n x p, Q~ = P - V (V^H P))
 *   P       : optional float64 row-major P supplied by the caller (device);
 *             if NULL, P is drawn on the device: element (row, col) is
 *             z(seed, counter, row*p + col)/sqrt(p), z = Box-Muller on
 *             SplitMix64 outputs 2m+1, 2m+2 with m = counter*2^32 + row*p + col
 *   filters : complex64 [p][n] output bank
 */
hicu_status hicu_jl_compress(hicu_handle* h, int64_t n, int64_t nr, int32_t p, const double* Q,
                             int32_t mode, const double* P, uint64_t seed, uint64_t counter,
                             float* filters, void* stream);

/*
 * hicu_conv_null - R[:, k] = H(x) q~_k for the p filters (Theory: valid
 * convolution of the k-space array with each annihilating filter; Algorithm 1
 * step 7's inner term).
 *   x       : complex64 k-space, filters: complex64 [p][n]
 *   R       : complex64 [sz][sy][sx][p]
 *   objective : optional device double, receives ||R||_F^2
 */
hicu_status hicu_conv_null(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                           const float* x, const float* filters, int32_t p, float* R,
                           double* objective, int32_t prec, void* stream);

/*
 * hicu_conv_null_adjoint - g = (1 - M) o sum_k H^H(r_k) (Theory: the conjugate
 * transpose of a valid convolution is itself a convolution; hard data
 * consistency sets the gradient to zero at observed locations).
 *   R     : complex64 [sz][sy][sx][p];  mask: nullable (NULL = no projection)
 *   g     : complex64 [C][Nz][Ny][Nx]; every entry inside S is written,
 *           entries outside S are left untouched
 *   gnorm2: optional device double, receives ||g||^2
 */
hicu_status hicu_conv_null_adjoint(hicu_handle* h, const hicu_geom* geom,
                                   const hicu_region* region, const float* R,
                                   const float* filters, int32_t p, const uint8_t* mask,
                                   float* g, double* gnorm2, int32_t prec, void* stream);

/*
 * hicu_conv_null_filter_grad - F_k[c, d] = sum_{o in V(S)} conj(x_c[o + d]) Rbar[o, k],
 * i.e. F = H(x)^H Rbar: the adjoint of the convolution v -> H(x) v in the filter
 * variable (the annihilating filters of the Theory section are its unknowns), so
 * <H(x) v, Rbar> = <v, F>; with Rbar = H(x) v it is the Gram product (H^H H) v.
 * Used for gradients with respect to the filters.
 *   x     : complex64 k-space [C][Nz][Ny][Nx] (device), read on S as hicu_conv_null
 *   Rbar  : complex64 [sz][sy][sx][p] (device), hicu_conv_null's output layout
 *   fbar  : complex64 [p][n] (device), filter layout [p][C][kz][ky][kx]; fully written
 * Complex FP32 products, FP32 partial sums per CTA, FP64 sum over CTAs in a fixed
 * order (deterministic).  HICU_ERR_UNSUPPORTED if one filter's coefficients (n
 * complex values) and the staging tiles exceed a CTA's shared memory.
 */
hicu_status hicu_conv_null_filter_grad(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                       const float* x, const float* Rbar, int32_t p, float* fbar,
                                       void* stream);

/*
 * hicu_project_unobserved - out = (1 - M) o x on S and 0 outside S (the projection
 * of hard data consistency: only unobserved entries of the region move).
 *   mask : nullable (NULL = keep every entry of S); layout as the hicu_geom mask
 *   x, out : complex64 [C][Nz][Ny][Nx] (device); out may be x (in place)
 */
hicu_status hicu_project_unobserved(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                                    const uint8_t* mask, const float* x, float* out, void* stream);

/*
 * hicu_gd_step_filters - one descent step for a fixed filter bank Q~ with
 * exact line search (Algorithm 1 steps 7-8; Theory, ELS paragraph):
 *   g = (1 - M) o sum_k H^H(H(y) q~_k),  D = sum_k ||H(g) q~_k||^2,
 *   eta = ||g||^2 / D  (0 when g = 0 or D = 0),  y <- y - eta g.
 *   y     : complex64 k-space, updated in place; entries with M != 0 and
 *           entries outside S are never written
 *   stats : optional device double[4] = {eta, ||H(y)Q~||^2 before the step,
 *           ||g||^2, D}
 */
hicu_status hicu_gd_step_filters(hicu_handle* h, const hicu_geom* geom,
                                 const hicu_region* region, float* y, const uint8_t* mask,
                                 const float* filters, int32_t p, double* stats, int32_t prec,
                                 void* stream);

/*
 * hicu_gd_step_soft - one descent step on ||H(y) Q~||^2 + lambda ||M o y - X0||^2 with exact line
 * search: the soft data-consistency cost, f_1 with multiplier lambda (Theory, Eq. 3; Algorithm 1
 * steps 7-8).  Only entries of S move; observed ones move too.  On S:
 *   g   = sum_k H^H(H(y) q~_k) + lambda M o (y - X0)
 *   eta = ||g||^2 / (||H(g) Q~||^2 + lambda ||M o g||^2),   y <- y - eta g
 *   x0    : complex64 observed data X0, zero off the samples (device)
 *   lambda: >= 0 (0 gives the unconstrained step: no data term, every entry of S free)
 *   stats : optional device double[4] = {eta, objective before the step (both terms), ||g||^2,
 *           the denominator}
 * Other arguments as hicu_gd_step_filters.
 */
hicu_status hicu_gd_step_soft(hicu_handle* h, const hicu_geom* geom, const hicu_region* region, float* y,
                              const uint8_t* mask, const float* x0, double lambda, const float* filters,
                              int32_t p, double* stats, int32_t prec, void* stream);

/*
 * hicu_soft_threshold - the proximal step of tau ||T x||_1, x <- T^H S_tau(T x), in place on the
 * whole array (Discussion: an l1 norm of a linear sparsifying transform adds a soft-thresholding
 * after Algorithm 1 step 8).  T is the centred orthonormal inverse DFT of every coil over the image
 * axes (x, y, and z unless z is flagged circular: the time axis of 2D+t), i.e. the coil images;
 * S_tau(w) = w max(0, 1 - tau / |w|).  The two transforms are cuFFT's; the handle keeps the plan.
 *   x   : complex64 [C][Nz][Ny][Nx] (device), overwritten
 *   tau : >= 0 (0: no change)
 */
hicu_status hicu_soft_threshold(hicu_handle* h, const hicu_geom* geom, float* x, double tau, void* stream);

/*
 * hicu_gd_step - JL compression (hicu_jl_compress) followed by
 * hicu_gd_step_filters: Algorithm 1 steps 6-8 for one inner index j.
 */
hicu_status hicu_gd_step(hicu_handle* h, const hicu_geom* geom, const hicu_region* region,
                         float* y, const uint8_t* mask, const double* Q, int64_t nr, int32_t p,
                         int32_t jl_mode, uint64_t seed, uint64_t counter, const double* P,
                         double* stats, int32_t prec, void* stream);

/*
 * hicu_reconstruct - Algorithm 1 with centre-out stages: for every outer
 * iteration the Gram matrix and null space (hicu_gram, hicu_nullspace; region
 * chosen by params->gram_on_current), then G^(i) calls of hicu_gd_step with
 * JL counter = global step index (0, 1, 2, ...).  With params->kernel_mask the
 * Gram, null space and JL draws are over the C |K| coefficients of the mask's
 * support (hicu_gram_support) and each filter bank is placed in the box
 * (hicu_expand_filters) for the convolutions.
 *   x0, mask, x_out may be HOST or DEVICE pointers (detected per pointer);
 *   host buffers are staged through the handle's workspace with copies on
 *   `stream`, and the call then returns after x_out is written.  A host x0
 *   whose first stage covers only some z planes is uploaded in two parts:
 *   those planes on `stream`, the others on a copy stream of the handle
 *   while the first stages run; `stream` waits for that copy (an event)
 *   before any stage that reaches beyond the planes, before the output copy
 *   and before an error return, so synchronising `stream` covers it.  A
 *   circular z axis, params->init = 1, dc_weight > 0 and l1_threshold > 0
 *   upload x0 in one copy.  Host buffers must stay valid until `stream` has
 *   been synchronised.
 *   log: optional host log; when given, the call synchronises the stream.
 */
hicu_status hicu_reconstruct(hicu_handle* h, const hicu_geom* geom, const float* x0,
                             const uint8_t* mask, const hicu_params* params, float* x_out,
                             hicu_log* log, void* stream);

/* ------------------------------------------------------------- batches */

/* One independent reconstruction of a batch (arguments of hicu_reconstruct). */
typedef struct {
  hicu_geom geom;
  const float* x0;      /* host or device, as hicu_reconstruct */
  const uint8_t* mask;  /* host or device */
  hicu_params params;   /* params.stages must stay valid for the call */
  float* x_out;         /* host or device */
  hicu_log* log;        /* nullable */
} hicu_problem;

/* Per-problem outcome of hicu_reconstruct_batched. */
typedef struct {
  double start_ms;   /* GPU time from the start of the batch to the problem's first kernel */
  double end_ms;     /* ... to the completion of its last kernel (completion latency) */
  int32_t lane;      /* worker lane that ran it */
  int32_t status;    /* hicu_status of the problem */
  int64_t gd_steps;  /* descent steps it ran (sum of iters x gd_steps over its stages) */
} hicu_slice_report;

/*
 * hicu_batch_order - the order in which hicu_reconstruct_batched starts the
 * problems: descending estimated cost (longest first, so that the large
 * problems do not finish last), ties by index.  Host only; no GPU needed.
 *   order : int32 [nslices], a permutation of 0 .. nslices-1
 *   cost  : optional double [nslices], the estimate in floating-point
 *           operations (Gram, eigen-solver sweeps and convolutions of every
 *           stage)
 */
hicu_status hicu_batch_order(int32_t nslices, const hicu_problem* problems, int32_t* order, double* cost);

/*
 * hicu_reconstruct_batched - hicu_reconstruct for many independent problems of
 * uneven size (matrix size, coils, kernel, rank, schedule), run side by side.
 * There is no counterpart in the paper, which reconstructs slices one at a time.
 *   `lanes` worker lanes (0: min(nslices, 8)), each with its own stream,
 *   workspace and host thread, take problems from one queue in hicu_batch_order
 *   order.  Problems that take a Jacobi solver by size (eig_solver 0 with
 *   HICU_JL_NULLSPACE) use the cluster eigen-solver for n <= 256, which occupies
 *   16 SMs and leaves the others to the other lanes.  Cooperative launches
 *   (tridiagonalisation, grid Jacobi) of all lanes go, in order, to one shared
 *   high-priority stream: two grid-barrier kernels never wait for each other's
 *   SMs, and a pending one gets SMs first as they free up.
 *   Every problem gives the same result as hicu_reconstruct with the same
 *   params (and that eig_solver): lanes share no mutable state.
 *   The lanes start after the work already queued on `stream`; the call returns
 *   when every problem has finished (it synchronises the lanes, not `stream`).
 *   report : optional host array [nslices], indexed like `problems`
 * Returns HICU_OK or the first failing problem's status (in `problems` order);
 * the other problems still run.  hicu_last_error names the failing problem.
 */
hicu_status hicu_reconstruct_batched(hicu_handle* h, int32_t nslices, const hicu_problem* problems,
                                     int32_t lanes, hicu_slice_report* report, void* stream);

/* ------------------------------------------------------ allocation-free */

#define HICU_NOALLOC_MAX_FILTER_WORDS 131072 /* n * (p rounded up to 16), complex64 words */
#define HICU_NOALLOC_MAX_PARTIALS 65536      /* CTAs of the convolution grid:
                                                ceil(sx/32) * ceil(sy/4) * sz */
#define HICU_NOALLOC_SCRATCH_BYTES (8 * 131072 + 8 * 65536) /* 1.5 MiB static device array */

/*
 * hicu_conv_null_noalloc - the same convolution and ||R||^2 as hicu_conv_null
 * (FP32 form), for callers that cannot allocate device memory when they call
 * it: a host framework that already holds all free device memory in its own
 * pool, or a latency-critical stage that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree may cause.  The paper has no counterpart.
 *   No handle, no cudaMalloc/cudaFree, no allocating library call.  Scratch is
 *   one static device array of HICU_NOALLOC_SCRATCH_BYTES that every GPU
 *   loading the library keeps until the process exits.
 *   Limits: n * roundup(p, 16) <= HICU_NOALLOC_MAX_FILTER_WORDS,
 *   ceil(sx/32) * ceil(sy/4) * sz <= HICU_NOALLOC_MAX_PARTIALS, and the halo tile
 *   of 8*kz*(ky+3)*(kx+31) bytes within the device's per-block shared-memory
 *   opt-in maximum (227 KB on GB300); larger requests return HICU_ERR_UNSUPPORTED
 *   (use hicu_conv_null).  Other errors: HICU_ERR_ARG, HICU_ERR_RANK,
 *   HICU_ERR_SHAPE, HICU_ERR_CUDA (no error text without a handle).
 *   The first call on each device (with that device current) looks up the
 *   array's device address and keeps it; make that first call before any stream
 *   capture, and do not reset the device (cudaDeviceReset) between calls.
 *   All calls share the array and it keeps the previous call's contents; each
 *   call writes every word it reads, so nothing needs clearing.  Calls that
 *   overlap on the GPU (other streams or host threads) race on the array.
 *   Arguments as hicu_conv_null (device pointers; R and/or objective).
 */
hicu_status hicu_conv_null_noalloc(const hicu_geom* geom, const hicu_region* region, const float* x,
                                   const float* filters, int32_t p, float* R, double* objective,
                                   void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HICU_H_ */
