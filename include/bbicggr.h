/*
 * bbicggr.h -- C-ABI of the GB300 (sm_103a) preconditioned block BiCGGR solver for the
 * O(a)-improved (clover) Wilson-Dirac equation with multiple right-hand sides.
 *
 * The problem is A X = B (Tadano, Kuramashi, Sakurai, arXiv:0907.3261, Sec. 2, Eq. (1)):
 * A is the N x N clover Wilson-Dirac matrix on an Lx*Ly*Lz*Lt lattice, N = 12*V, V = Lx*Ly*Lz*Lt,
 * and X, B are N x L blocks of L right-hand sides ("source vectors").
 *
 * Conventions (the paper leaves A's structure to its Ref. [blockbicggr_app]; these are the
 * standard Sheikholeslami-Wohlert form in kappa normalisation, periodic boundaries):
 *   (A psi)(x) = A_D(x) psi(x) - kappa sum_mu [(1 - g_mu) U_mu(x) psi(x+mu)
 *                                             + (1 + g_mu) U_mu(x-mu)^H psi(x-mu)]
 *   A_D(x) = 1 - kappa c_SW sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x), sigma = (i/2)[g_mu, g_nu],
 *   F = (Q - Q^H)/(8i) with Q the four-leaf clover; chiral basis g_k = [[0,-i s_k],[i s_k,0]],
 *   g_t = [[0,1],[1,0]], g_5 = diag(1,1,-1,-1).
 *
 * Layouts (all complex128, real and imaginary parts interleaved, 16-byte aligned):
 *   site index        s = x + Lx*(y + Ly*(z + Lz*t))
 *   links             [V][4 mu][3][3]: U_mu(x), the link from x to x+mu, row-major; mu = x,y,z,t
 *   N x L blocks      [V][4 spin][3 colour][L]: element (row n, column i) at n*L + i, i.e. the
 *                     paper's N x L matrix stored row-major, right-hand sides innermost.
 *
 * Pointers: every buffer argument may be device memory or host memory (pageable or pinned); the
 * library finds out with cudaPointerGetAttributes.  Host buffers are staged through device
 * buffers owned by the context, with cudaMemcpyAsync on the given stream, and a call that was given
 * a host buffer synchronises the stream before it returns.  Device buffers must be 16-byte aligned.
 * Ownership: the caller owns every buffer it passes; the library never frees or keeps a pointer to
 * one after the call returns.  wd_create copies the links and derives the clover term into
 * context-owned device memory; solver workspace is allocated at the first call with a given L and
 * kept in the context until wd_destroy.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All device work of a call is
 * ordered on it.  A context must not be used from two host threads at once.
 * Errors: every entry point returns an int status (WD_OK = 0) and never aborts; wd_strerror gives
 * the code's name and wd_last_error() a one-line description of the last failure in this thread.
 */
#ifndef BBICGGR_H
#define BBICGGR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  WD_OK = 0,
  WD_EINVAL = 1,          /* bad argument: dims < 2 or too large, L outside [1, WD_LMAX], j < 0,
                             tol <= 0, NULL or misaligned pointer, a column of B that is zero */
  WD_ENOMEM = 2,          /* device or pinned-host allocation failed */
  WD_ECUDA = 3,           /* a CUDA runtime call failed; wd_last_error() has the CUDA message */
  WD_NOT_CONVERGED = 4,   /* maxit reached, or true residual above tol after max_restarts */
  WD_DIVERGED = 5,        /* max_i ||r_i|| / ||b_i|| exceeded opts.div_thresh (Sec. 3.3: 1e2) */
  WD_BREAKDOWN = 6        /* singular L x L system (rank loss, Sec. 4), Tr[W^H W] = 0, a
                             non-finite residual, or a singular clover block at wd_create */
};

#define WD_LMAX 16        /* largest number of right-hand sides per solve */

typedef struct wd_ctx wd_ctx;   /* opaque; owned by the library */
typedef struct wd_net wd_net;   /* opaque learned preconditioner; owned by the library */

/* Solver options.  Fill with bbicggr_default_opts() and change what you need. */
typedef struct {
  int maxit;              /* outer iterations, default 10000 (summed over restarts) */
  double div_thresh;      /* DIVERGED above this max relative recursive residual; default 1e2 */
  int max_restarts;       /* restarts from X when the true residual is above tol; default 3 */
  int precision;          /* 0: FP64 preconditioner (default); 1: FP32 preconditioner with FP32
                             accumulation -- the outer recurrences, the products W = AF and
                             Y = AG, the Gram matrices, the L x L solves and the true residual stay
                             FP64; 2: as 1, and the direction recurrences U = (P - zeta V) alpha,
                             P = R + U gamma, V = W + Y gamma and the Gram products in double-float
                             (FP32-pair, ~48-bit) arithmetic on the FP32 pipes, with the X and R
                             updates and column norms still FP64; 3: as 1 with the
                             preconditioner's blocks (its copy of U and the sweep iterates) stored
                             in BF16, arithmetic FP32; 4: double-float sweeps -- the operator
                             (links, A_D^{-1}, kappa) in FP32 and the spinors as FP32 pairs
                             (~48 bits), so M is linear to ~1e-13; 5: as 4, and the direction
                             recurrences in double-float as in 2.  In 1-5 the sweeps read 12-real
                             links (rows 0 and 1, row 2 rebuilt) when wd_link_reals says 12 */
  double* history;        /* optional host array: max_i ||r_i||/||b_i|| after every R update */
  int history_len;        /* capacity of history (entries beyond it are dropped) */
  int stall_window;       /* precision 1-5 only: when the max relative residual has not reached a new
                             minimum for this many iterations, or the low-precision run breaks
                             down or diverges, the solve starts over from X_0 with the FP64
                             preconditioner (block BiCGGR needs a fixed linear M, and the
                             rounding of a low-precision M can stall it near the critical kappa).  Default 16;
                             0 disables the fallback.  Costs one more N x L block of workspace */
  wd_net* net;            /* not NULL: M is this learned network instead of j-step Jacobi, with
                             its activations in FP32, or in BF16 with precision 3;
                             the stall rule above applies and its fallback is FP64 Jacobi with the
                             solve's j.  mvm_paper then counts the products with A only */
} bbicggr_opts;

/* Solve report.  rec_resid and true_resid, when not NULL, are caller-owned host arrays of L. */
typedef struct {
  int status;             /* same as the return value */
  int iters;              /* outer iterations k (summed over restarts) */
  int restarts;           /* restarts taken */
  long long mvm_paper;    /* #MVM as the paper counts it: L * sum over runs of 2(j+1)k + 1 */
  long long mvm_actual;   /* column-MVMs with a hopping term actually applied (the first Jacobi
                             sweep from G = 0 is site-local and not counted) */
  double max_rec_resid;   /* max_i ||r_i|| / ||b_i|| of the recursive residual at exit */
  double max_true_resid;  /* max_i ||b_i - A x_i|| / ||b_i|| at exit */
  double* rec_resid;      /* [L] or NULL */
  double* true_resid;     /* [L] or NULL */
  int history_count;      /* entries written to opts->history */
  double seconds;         /* wall time of the call (host clock, includes host<->device copies) */
  int fallbacks;          /* switches from the low-precision to the FP64 preconditioner (0 or 1) */
} bbicggr_info;

/* Build the operator A for the given links (Sec. 2; kappa and c_SW as in Sec. 3.1).
 * links: [V][4][3][3] complex128 (host or device); dims: {Lx, Ly, Lz, Lt}, each >= 2, V <= 2^26.
 * Copies the links, builds F_{mu nu} from the four-leaf clover, the two 6x6 chiral blocks of A_D per
 * site and their inverses (FP64), all in context-owned device memory.  *out is NULL on failure.
 * Returns WD_BREAKDOWN if some clover block is singular. */
int wd_create(wd_ctx** out, const void* links, const int dims[4], double kappa, double csw,
              void* stream);

/* Release everything the context owns.  NULL is a no-op. */
void wd_destroy(wd_ctx* ctx);

/* Y = A X for an N x L block (Sec. 2, Eq. (1)).  X and Y must not overlap.  1 <= L <= WD_LMAX. */
int wd_apply(wd_ctx* ctx, const void* X, void* Y, int L, void* stream);

/* G = M R, the j-step Jacobi preconditioner of Sec. 2 from the zero initial guess (Sec. 3.3):
 * G = sum_{i<j} (I - A_D^{-1} A)^i A_D^{-1} R for j >= 1 and G = R for j = 0.  Computed as j sweeps
 * G <- A_D^{-1}(R + kappa H G), H the hopping term.  `precision`: 0 = FP64 sweeps, 1 = FP32
 * sweeps, 3 = FP32 arithmetic on BF16-stored blocks (as in bbicggr_opts).  R and G must not
 * overlap. */
int jacobi_precond(wd_ctx* ctx, const void* R, void* G, int L, int j, int precision, void* stream);

/* jacobi_precond_noalloc: the same G = M R as jacobi_precond (FP64 sweeps), computed without
 * allocating any memory.  The paper has no counterpart; this exists for callers that cannot let a
 * library call cudaMalloc -- a framework whose caching allocator already owns the free device
 * memory, or a latency-bound loop that cannot pay for cudaMalloc/cudaFree and the device
 * synchronisation cudaFree implies.  jacobi_precond takes its ping-pong block from the context's
 * solver workspace (allocated on first use); this variant takes it from a file-scope device array
 * of 32 MiB.  wd_create loads that array on its device, so every GPU on which a context has been
 * created holds the 32 MiB from wd_create until the process exits (wd_create fails with
 * WD_ENOMEM if it cannot be loaded).
 *   Limits: 12*V*L <= 2,097,152 complex numbers (e.g. 8^3x16 with L <= 21, 16^3x32 does not fit);
 *   larger blocks return WD_EINVAL.  R and G must be device buffers (WD_EINVAL for host memory,
 *   which would need staging) and must not overlap.  The current device must be the context's
 *   device (WD_EINVAL otherwise).
 *   Set-up: every call looks up the array's device address on the current device
 *   (cudaGetSymbolAddress, which allocates nothing once wd_create has loaded the array).
 *   Sharing: every call on a device uses the same array, which keeps the last call's contents (the
 *   sweeps overwrite it before reading it, so nothing needs clearing).  Calls whose GPU work
 *   overlaps -- on different streams, or from different host threads -- race on the array. */
int jacobi_precond_noalloc(wd_ctx* ctx, const void* R, void* G, int L, int j, void* stream);

/* Preconditioned block BiCGGR (Sec. 2, algorithm box) with the j-step Jacobi preconditioner,
 * R~_0 = R_0 (Sec. 3.3).  X holds X_0 on entry (zero it for the paper's X_0 = 0) and the solution
 * on exit.  Iterates until max_i ||r_i||/||b_i|| <= tol on the recursive residual, checked after
 * every R update; then recomputes the true residual and restarts from X while it is above tol
 * (at most opts->max_restarts times).  On a non-OK return X holds the last iterate and info is
 * filled.  opts may be NULL (defaults); info may be NULL.  Every column of B must be non-zero. */
int bbicggr_solve(wd_ctx* ctx, const void* B, void* X, int L, int j, double tol,
                  const bbicggr_opts* opts, bbicggr_info* info, void* stream);

/* ---- Block updates of one outer iteration (Sec. 2, algorithm box), on caller-supplied N x L
 * device blocks of this context's lattice (complex128, 16-byte aligned, the layout above; host
 * buffers are WD_EINVAL).  They are the updates bbicggr_solve runs, exposed for tests and for
 * drivers that run the iteration themselves.  L x L matrices are host arrays of L*L complex128,
 * row-major (entry (a, b) at a*L + b); zeta is a host complex128 (re, im).  precision: 0 = FP64;
 * 1 = the products with the L x L matrix and the Gram products in double-float arithmetic (the
 * direction recurrences of bbicggr_opts.precision 2 and 5); the X and R updates and the column
 * norms are FP64 in both.  Each call synchronises the stream.  Output blocks must not overlap the
 * inputs (X and R are updated in place in bb_update_xr).
 *   bb_update_u:  U = (P - zeta V) alpha                         (S_k and U_k of the box)
 *   bb_update_xr: X <- X + zeta F + G,  R <- R - zeta W - Y,  rtr_new = R~_0^H R (new R),
 *                 rnorm2[i] = ||r_i||^2 (new R); rtr_new and rnorm2 may be NULL
 *   bb_update_pv: P = R + U gamma,  V = W + Y gamma,  rtv = R~_0^H V (new V); rtv may be NULL */
int bb_update_u(wd_ctx* ctx, const void* P, const void* V, void* U, int L, const double* zeta,
                const void* alpha, int precision, void* stream);
int bb_update_xr(wd_ctx* ctx, void* X, const void* F, const void* G, void* R, const void* W,
                 const void* Y, const void* Rt, int L, const double* zeta, void* rtr_new,
                 double* rnorm2, int precision, void* stream);
int bb_update_pv(wd_ctx* ctx, void* P, void* V, const void* R, const void* W, const void* U,
                 const void* Y, const void* Rt, int L, const void* gamma, void* rtv,
                 int precision, void* stream);

/* One solve of a batch (bbicggr_solve_batch).  B and X are device buffers; every job has its own
 * context (jobs may differ in lattice, kappa, c_SW, L, j and precision). */
typedef struct {
  wd_ctx* ctx;
  const void* B;          /* N x L, device */
  void* X;                /* X_0 in, solution out, device */
  int L;
  int j;
  double tol;
  bbicggr_opts opts;      /* every option is used, as in bbicggr_solve */
  bbicggr_info info;      /* filled on return; rec_resid / true_resid may point to host arrays */
} bbicggr_job;

/* Preconditioned block BiCGGR for several independent systems at once, with all control on the
 * device: every job is a branch of one CUDA graph.  A job's outer iteration is a conditional
 * while-node whose convergence test (the algorithm box's) runs in a kernel that sets the loop
 * condition; around it a second while-node runs one solve per pass and decides after each pass,
 * in a kernel, what bbicggr_solve decides on the host: start over from X_0 with the FP64 Jacobi
 * preconditioner when a low-precision or network run stalled, broke down or diverged (precision
 * fallback, opts.stall_window > 0), restart from X when the true residual is above tol (at most
 * opts.max_restarts times), or stop.  The host launches once and synchronises once.  Each job
 * reproduces bbicggr_solve on its own: the same iterations, restarts, fallbacks, residual
 * history and X.  info.mvm_actual is -1.  Returns WD_OK if every job converged, else the first
 * job's non-OK status; argument and CUDA errors return before any work. */
int bbicggr_solve_batch(bbicggr_job* jobs, int njobs, void* stream);

/* Copies the recursive residual R of the algorithm box (Sec. 2) as the last solve on ctx left it --
 * updated by R -= zeta W + Y every iteration, never recomputed from X -- to R (N x L, host or
 * device), so that a caller can measure how far it drifted from B - A X (the true residual,
 * Sec. 1).  L must be the last solve's; WD_EINVAL otherwise or before any solve.  Synchronises
 * the stream. */
int wd_copy_residual(wd_ctx* ctx, void* R, int L, void* stream);

void bbicggr_default_opts(bbicggr_opts* opts);
const char* wd_strerror(int code);
const char* wd_last_error(void);

/* ---- Learned preconditioner (the paper's future work on a better preconditioner, Sec. 4).
 * A network of `layers` gauge-covariant layers, linear in the spinor, channels
 * 1 -> hidden -> ... -> hidden -> 1 (hidden 1, 2 or 4):
 *   out_{c'}(x) = sum_{d=0..8} sum_c W[d][c'][c] (T_d psi_c)(x),   T_0 = 1,
 *   (T_{1+mu} psi)(x) = U_mu(x) psi(x+mu),  (T_{5+mu} psi)(x) = U_mu(x-mu)^H psi(x-mu),
 * W[d][c'][c] a complex 4x4 spin matrix.  Weights at the ABI: complex128, per layer
 * [9][C_out][C_in][4][4], layers concatenated (wd_net_num_weights complex numbers); stored as
 * complex64.  Activations FP32; inference may store them in BF16 instead (FP32 arithmetic either
 * way).  Training: loss = (1/L) sum_i ||N(r_i) - e_i||^2 / ||e_i||^2 over
 * pairs (r_i, e_i = A^{-1} r_i), gradient d loss / d conj(W), Adam on (Re W, Im W). */
int wd_net_create(wd_net** out, int layers, int hidden, const void* weights /* host or device */);
void wd_net_destroy(wd_net* net);
long long wd_net_num_weights(const wd_net* net);
int wd_net_set_weights(wd_net* net, const void* weights);   /* also resets the Adam state */
int wd_net_get_weights(const wd_net* net, void* out);       /* host or device, complex128 */
/* G = N(R) for device blocks R, G (N x L, complex128, site-major); bf16 = 1 stores the
 * activations in BF16 (0: FP32). */
int wd_net_apply(wd_ctx* ctx, wd_net* net, const void* R, void* G, int L, int bf16, void* stream);
/* Forward and backward pass on device blocks R, E: *loss (host, may be NULL) and the gradient
 * d loss / d conj(W), kept in the network for wd_net_adam_step and copied to `grad` (complex128,
 * host or device, may be NULL).  Synchronises the stream. */
int wd_net_loss_grad(wd_ctx* ctx, wd_net* net, const void* R, const void* E, int L, double* loss,
                     void* grad, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the gradient of the last loss_grad. */
int wd_net_adam_step(wd_net* net, double lr, void* stream);

/* Per-kernel instrumentation.  Every kernel launch of a context is counted per kernel class
 * (WD_K_*).  With timing on, each launch is also bracketed by two CUDA events recorded on the
 * launching stream, and the elapsed device times are summed when the call that launched them
 * returns.  wd_profile_read gives the launch count and summed milliseconds of one class since the
 * last wd_profile_reset; wd_profile_name its name. */
enum {
  WD_K_APPLY = 0,      /* dslash Y = A X */
  WD_K_RESID,          /* dslash R = B - A X */
  WD_K_JACOBI,         /* FP64 Jacobi sweep G <- A_D^{-1}(U + kappa H G) */
  WD_K_SITE_INV,       /* first Jacobi sweep G = A_D^{-1} U */
  WD_K_UPDATE_U,       /* U = (P - zeta V) alpha */
  WD_K_UPDATE_XR,      /* X += zeta F + G, R -= zeta W + Y, R~_0^H R, ||r_i||^2 */
  WD_K_UPDATE_PV,      /* P = R + U gamma, V = W + Y gamma, R~_0^H V */
  WD_K_GRAM,           /* standalone Gram product */
  WD_K_TRACE,          /* Tr[W^H R], Tr[W^H W] */
  WD_K_SOLVE_LL,       /* L x L LU solves */
  WD_K_COLNORM,        /* column norms */
  WD_K_COPY,           /* device-to-device block copies */
  WD_K_CONVERT,        /* FP64 <-> FP32 conversions of the FP32 preconditioner */
  WD_K_NET,            /* learned preconditioner G = N(R) (all its kernels) */
  WD_K_JACOBI_LP,      /* Jacobi sweep in FP32 arithmetic on FP32 or BF16 blocks, or in
                          double-float arithmetic */
  WD_K_COUNT
};
int wd_profile_enable(wd_ctx* ctx, int timing_on);
int wd_profile_reset(wd_ctx* ctx);
int wd_profile_read(const wd_ctx* ctx, int kernel_class, long long* launches, double* ms);
const char* wd_profile_name(int kernel_class);

/* Tile of the low-precision Jacobi sweep chosen by the autotuner for this L and storage
 * (precision 1: FP32 blocks, 3: BF16 blocks, 4: double-float sweeps, which take 1 or 2 RHS per
 * thread in 128-thread CTAs, staged 1 for the packed FP32x2 variant with 1 RHS per thread, and
 * staged 2 for the packed variant whose link and clover products are summed exactly on a fixed
 * grid per hop and per clover block -- offered only when every link has rows and columns of norm
 * at most 1, as unitary links do):
 * RHS per thread, threads per CTA, the minimum
 * resident CTAs per SM the kernel was compiled for (0: none; 8: at most 128 registers a thread),
 * and whether each direction's neighbour data is staged in shared memory (cp.async, two stages)
 * while the previous direction is computed.  The autotuner times every candidate tile once, at
 * the first preconditioner call with that L and storage, and keeps the fastest in the context.
 * WD_EINVAL until then.  Any output pointer may be NULL. */
int wd_tuned_tile(const wd_ctx* ctx, int L, int precision, int* rhs_per_thread, int* block,
                  int* min_blocks, int* staged);
/* Sets that tile by hand instead: rhs_per_thread 1 or 2 dividing L with block 64, 128 or 256,
 * min_blocks 0 (or, with block 64, 8, or 12 with one RHS per thread: at most 80 registers) and
 * staged 0; rhs_per_thread 0 with block 128 (the stencil of
 * every (site, rhs) pair split over two warps); or staged 1 with rhs_per_thread 2, block 64 and
 * min_blocks 0.  Double-float sweeps (precision 4): rhs_per_thread 1 or 2 with block 128,
 * min_blocks 0 and staged 0, or rhs_per_thread 1 with staged 1 or 2 (2: unitary links only). */
int wd_set_tile(wd_ctx* ctx, int L, int precision, int rhs_per_thread, int block, int min_blocks,
                int staged);

/* Link format of the low-precision sweeps: 12 (rows 0 and 1 of each FP32 link are read and row 2
 * is rebuilt as conj(row0 x row1), which holds for SU(3)) or 18 (all three rows read).  wd_create
 * picks 12 when every link's third row matches conj(row0 x row1) to 1e-6 per entry, else 18.
 * wd_set_link_reals(ctx, 18) forces the full format; asking for 12 with links that failed the
 * check is WD_EINVAL.  The FP64 path and the learned network always read 18 reals. */
int wd_link_reals(const wd_ctx* ctx, int* reals);
int wd_set_link_reals(wd_ctx* ctx, int reals);

/* Form of the FP64 stencil Y = A X, R = B - A X and of the FP64 Jacobi sweep (Eq. (1), Sec. 2),
 * which carry the outer method's products W = AF, Y = AG, the true residual and precision 0's
 * preconditioner.  1 (the default for links whose rows and columns have norm <= 1 + 1e-6, so
 * unitary links): the hopping sums run on the FP32 lanes, every operand cut exactly into three
 * FP32 numbers and the products summed exactly on fixed grids, so that the hopping term is
 * exact to ~2^-52 of its bound before one FP64 rounding; the site blocks, the spin projection
 * and the final combination stay FP64.  It is as accurate as FP64 arithmetic and about twice as
 * fast on GB300, whose FP64 pipe issues two lanes per clock per SM.  0: every operation on the
 * FP64 pipe.  Asking for 1 with other links is WD_EINVAL.  wd_get_apply_form returns the form
 * (-1 for a NULL ctx). */
int wd_set_apply_form(wd_ctx* ctx, int form);
int wd_get_apply_form(const wd_ctx* ctx);

/* ---- Domain decomposition across ranks (the paper picks the Jacobi preconditioner for its
 * parallelism, Sec. 2).  The lattice is cut into slabs along t; a rank's context is created with
 * wd_create on its slab extended by one t-slice on each side (dims {Lx, Ly, Lz, T + 2}, T >= 1
 * interior slices), the links of the extended slab filled from the neighbouring ranks (the
 * clover leaves reach one slice out).  Sites of the two halo slices are computed but not owned.
 * With a domain set:
 *   - every product with A and every Jacobi sweep that reads neighbours first fills the halo
 *     slices of its input block from the neighbouring ranks through `exchange`;
 *   - every Gram product, trace and column norm runs over the interior rows and is summed over
 *     the ranks through `allreduce`, so every rank solves the same L x L systems and takes the
 *     same convergence decisions;
 *   - bbicggr_solve takes B and X as blocks of the extended slab (their halo rows are ignored on
 *     entry; X's halo rows are overwritten) and must use precision 0 (FP64 Jacobi sweeps) and no
 *     network; wd_apply exchanges halos of a copy of X; jacobi_precond takes precision 0;
 *     bbicggr_solve_batch rejects the context; bb_update_* ignore the domain (all rows).
 * Both callbacks are called from the thread that called the library, with the stream drained.
 * They return 0 on success; anything else fails the call with WD_ECUDA. */
typedef struct {
  /* Halo exchange on host buffers of `bytes` each: send_lo is this rank's first interior slice
   * (the previous rank's upper halo), send_hi its last interior slice (the next rank's lower
   * halo); recv_lo receives the previous rank's last interior slice, recv_hi the next rank's
   * first (periodic in t). */
  int (*exchange)(const void* send_lo, const void* send_hi, void* recv_lo, void* recv_hi,
                  size_t bytes, void* user);
  /* Sum of n doubles over all ranks, in place in the host buffer `buf`; every rank must get the
   * same result. */
  int (*allreduce)(double* buf, int n, void* user);
  void* user;
} wd_domain;
/* Sets (dom not NULL, copied) or clears (NULL) the domain of a context.  WD_EINVAL if a callback
 * is NULL or the slab has fewer than 3 t-slices. */
int wd_set_domain(wd_ctx* ctx, const wd_domain* dom);

/* Lattice size and parameters of a context (for bindings): dims[4], V, kappa, c_SW. */
int wd_query(const wd_ctx* ctx, int dims[4], long long* volume, double* kappa, double* csw);

#ifdef __cplusplus
}
#endif
#endif /* BBICGGR_H */
