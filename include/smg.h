/*
 * smg.h -- C ABI of the GB300 structured-multigrid library (StructMG method,
 * arXiv 2506.21932): stencil Galerkin coarsening, dependence-preserving
 * Gauss-Seidel / ILU(0) smoothers, V-cycle preconditioned PCG / FGMRES.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid and vectors (Sec. 4.1, SG-DIA format): a structured grid of
 *   nx * ny * nz points; point (i,j,k) has linear index p = (i*ny + j)*nz + k
 *   (x slowest, z fastest).  A vector holds B values per point: v[p*B + r].
 * Matrices (Sec. 4.1, SG-DIA): for every point, one coefficient (B == 1) or
 *   one row-major BxB block (B == 3) per stencil offset, offsets in
 *   {-1,0,1}^3 (Sec. 4.2):
 *   A[((p*nstencil + e)*B + r)*B + c].  Coefficients whose neighbour lies off
 *   the grid must be 0 (zero padding).  The offset list may be given in any
 *   order but must contain the centre, no duplicates and be structurally
 *   symmetric; the library stores it in lexicographic order (dx slowest).
 * Memory: every pointer argument documented "device" is CUDA device memory
 *   owned by the caller; the library never frees or keeps it after the call
 *   returns (coefficients are copied at setup).  "host" pointers are ordinary
 *   host memory.  All work is enqueued on the caller's CUDA stream (a
 *   cudaStream_t passed as void*; NULL = legacy default stream) and the calls
 *   return after that work has completed unless stated otherwise.
 * Errors: every function returns an smg_status; nothing is thrown and no
 *   device trap is ever raised.  Device-side waits are bounded; a wait that
 *   runs out returns SMG_ETIMEOUT and leaves the context reusable.
 * Threads: one context must not be used from two threads at once.
 */
#ifndef SMG_H
#define SMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smg_ctx* smg_t;

typedef enum {
  SMG_OK = 0,
  SMG_EINVAL = 1,      /* bad argument: sizes, mask, options, off-grid coefficient != 0 */
  SMG_ENOMEM = 2,      /* device allocation failed */
  SMG_ECUDA = 3,       /* a CUDA runtime call failed */
  SMG_EBREAKDOWN = 4,  /* zero/negative pivot, zero diagonal, p^T A p <= 0 */
  SMG_ENOTCONV = 5,    /* tolerance not reached within maxit iterations */
  SMG_ENAN = 6,        /* non-finite residual */
  SMG_ETIMEOUT = 7     /* a bounded device-side wait ran out */
} smg_status;

enum { SMG_SMOOTHER_SGS = 0, SMG_SMOOTHER_ILU0 = 1, SMG_SMOOTHER_LGS = 2 };
enum { SMG_TRANSFER_FW27V = 0, SMG_TRANSFER_PC8C = 1, SMG_TRANSFER_C64C = 2, SMG_TRANSFER_C16C_XY = 3 };
enum { SMG_PREC_FP64 = 0, SMG_PREC_FP32 = 1, SMG_PREC_BF16 = 2 };
enum { SMG_KRYLOV_PCG = 0, SMG_KRYLOV_FPCG = 1, SMG_KRYLOV_FGMRES = 2 };

/* Solver options; an all-zero struct selects the defaults in brackets.
 *  smoother   [SGS]  symmetric lexicographic Gauss-Seidel (Sec. 4.4 GS-Forward
 *                    then GS-Backward) or ILU(0) on the matrix mask (Sec. 4.4
 *                    ILU formula; Sec. 4.2 ILU masks).  One pre- and one
 *                    post-smoothing step per level (Sec. 5.2); the first
 *                    pre-smoothing starts from zero (ZeroGuess, Table 8).
 *                    LGS: symmetric line Gauss-Seidel along z (Sec. 4.4 LGS):
 *                    each z-column is updated at once, its couplings to other
 *                    columns moved to the right-hand side and its tridiagonal
 *                    system solved exactly; columns in lexicographic (x, y)
 *                    order, then in reverse.  Requires block == 1, FP64,
 *                    relax_w 1 and nz <= 1024 (else SMG_EINVAL); a column
 *                    whose Thomas pivots are not all positive gives
 *                    SMG_EBREAKDOWN.
 *  transfer   [FW27V] vertex full weighting: coarse I on fine 2I+1, trilinear
 *                    P and R = P^T/8 (Table 2 pattern 3d27v); PC8C: cell
 *                    piecewise constant, R(I,u)=1 on u in 2I+{0,1}^3, P = R^T
 *                    (Table 2 pattern 3d8c); C64C: the same 3d8c restriction
 *                    with cell-centred trilinear interpolation, per dimension
 *                    3/4 from the fine cell's own coarse cell and 1/4 from
 *                    the next one on its side, coarse cells off the grid
 *                    dropped (Table 2 columns 3d8c / A / 3d64c; the Table 8
 *                    settings of rhd-3T and solid-3D).  R is not a multiple
 *                    of P^T, so the coarse operators and the V-cycle are
 *                    nonsymmetric: use FPCG or FGMRES (PCG is accepted; the
 *                    paper runs CG with it).  C16C_XY: 2-D semi-coarsening
 *                    (Table 8, weather): only x and y are halved, z is
 *                    kept; the 2 x 2 cell sum restricts and the cell-centred
 *                    bilinear interpolation of C64C acts in x and y (2d4c /
 *                    2d16c), so coarse grids keep whole z-columns for the
 *                    LGS smoother.  Coarsening stops when x or y is odd or
 *                    the smaller of them is below 8.
 *  precision  [FP64] storage and arithmetic of the hierarchy and V-cycle:
 *                    FP64, FP32, or BF16 values with one FP32 scale per row
 *                    and FP32 accumulation (not in the paper).  The Krylov
 *                    iteration, the outer residual and the coarsest solve stay
 *                    FP64.  BF16 requires block == 1.
 *  krylov     [PCG]  PCG, flexible PCG (Polak-Ribiere beta) or right-
 *                    preconditioned flexible GMRES(restart) (Sec. 5.2).
 *  restart    [30]   GMRES restart length, 1..64.
 *  relax_w    [1.0]  Gauss-Seidel weight w of the Sec. 4.4 formulas.
 *  max_levels [16]   cap on the number of levels (>= 1).
 *  spin_budget_ms [1000] bound on any single device-side wait, in ms.
 *  use_graph  [0]    1: capture each V-cycle in a CUDA graph and replay it.
 *  fuse_restrict [0] 1: the residual after pre-smoothing and its restriction
 *                    in one kernel on scalar levels with the full-weighting
 *                    or 3d8c restriction (fc = R (f - A u) without storing
 *                    the fine residual); 0: two kernels.  Same arithmetic in
 *                    the same order either way.  Off by default: the fine
 *                    residual is FP64-bound, and the fused pass's tile-edge
 *                    recomputation and lower occupancy cost more than the
 *                    fine-residual traffic it saves (measured on GB300).
 *  sweep_warps [0]   warps per 32-column strip of the point smoothers'
 *                    wavefront sweeps on 19/27-point levels: 1 one warp
 *                    does everything; 2 a helper warp loads the operands and
 *                    forms the early partial sums while the main warp only
 *                    finishes points (FP64 Gauss-Seidel with old values,
 *                    y extents above 384, and y extents above 256 except
 *                    for FP64 ILU(0), keep one); 0 the library's choice
 *                    (two where they apply).  Same arithmetic in the same
 *                    order either way. */
typedef struct {
  int smoother, transfer, precision, krylov, restart;
  double relax_w;
  int max_levels;
  int spin_budget_ms;
  int use_graph;
  int fuse_restrict;
  int sweep_warps;
} smg_options;

/* Build the hierarchy from the finest matrix (Sec. 4.2: only the finest A is
 * given).  Levels: halve every dimension while all are even and the smallest
 * is >= 8 (stride-2 full coarsening, Sec. 4.1 P2); with the x-y
 * semi-coarsening transfer only x and y, under the same rule for them.
 * Coarse operators: Galerkin A^C = R A^F P (Eq. 4) evaluated per coarse point
 * by influence chains (Eq. 5-10) derived once on the host from the (R, A, P)
 * patterns.  Smoother set-up per level; dense inverse of the coarsest level
 * by Gauss-Jordan elimination with partial pivoting (the paper does not
 * specify the coarsest solve; at most 8192 coarsest unknowns).
 *  out      host: receives the new context (NULL on failure).
 *  dims     host int[3] = {nx, ny, nz}, each >= 1 and <= 4096, ny <= 1024.
 *  nstencil number of offsets, 1..27;  offsets host int[nstencil][3].
 *  coeffs   device double, layout above; read during the call only.
 *  block    B = 1 or 3 (3 = three coupled unknowns per point, block GS).
 *  opt      host, may be NULL (all defaults).
 *  stream   cudaStream_t.
 * Errors: SMG_EINVAL (bad sizes/mask/options, nonzero off-grid coefficient),
 * SMG_ENOMEM, SMG_EBREAKDOWN (zero diagonal, ILU pivot <= 0, a line's Thomas
 * pivot <= 0, singular coarsest matrix), SMG_ECUDA, SMG_ETIMEOUT. */
int smg_setup(smg_t* out, const int dims[3], int nstencil, const int* offsets, const double* coeffs, int block,
              const smg_options* opt, void* stream);

/* One V(1,1)-cycle as preconditioner: z = M^{-1} r (Sec. 2, Fig. 1 V-cycle).
 *  r, z  device double [n*B]; may not alias.
 * Errors: SMG_EINVAL (NULL handle/pointers), SMG_ECUDA, SMG_ETIMEOUT. */
int smg_vcycle(smg_t h, const double* r, double* z, void* stream);

/* Profiled V-cycle: the same z = M^{-1} r as smg_vcycle (always run eagerly,
 * never from a captured graph), with a CUDA event recorded on the stream
 * after every stage, so the device time of each stage is measured without
 * host gaps.  Stage t (0 <= t < *count) ran on level levels[t]; stages[t] is
 * one of SMG_STAGE_* (PACK / UNPACK: vectors into and out of the sweeps'
 * skewed plane layout; POST_ADD: the unpack that adds the correction); ms[t]
 * its device time.  At most cap entries are
 * written (*count is the full number).  Synchronises the stream.  Not part
 * of the method: a measurement aid for the per-level cost of a cycle.
 * Errors: SMG_EINVAL (NULL or aliased pointers, cap < 0), SMG_ECUDA. */
enum { SMG_STAGE_PRE1 = 1, SMG_STAGE_PRE2 = 2, SMG_STAGE_RESIDUAL = 3, SMG_STAGE_RESTRICT = 4,
       SMG_STAGE_COARSE = 5, SMG_STAGE_PROLONG = 6, SMG_STAGE_POST_RESIDUAL = 7, SMG_STAGE_POST1 = 8,
       SMG_STAGE_POST2 = 9, SMG_STAGE_POST_ADD = 10, SMG_STAGE_CAST = 11, SMG_STAGE_LEARNED = 12,
       SMG_STAGE_PACK = 13, SMG_STAGE_UNPACK = 14 };
int smg_vcycle_profile(smg_t h, const double* r, double* z, int cap, int* count, int* levels, int* stages,
                       float* ms, void* stream);

/* Solve A x = b with the Krylov method of the options, preconditioned by one
 * V-cycle per iteration (Sec. 5.2), until ||r_k||_2 / ||b||_2 < tol (Table 8).
 *  b      device double [n*B];  x  device double [n*B]: initial guess in,
 *         solution out.
 *  tol    relative tolerance > 0;  maxit  >= 0 iterations.
 *  iters  host int*, may be NULL: iterations taken.
 *  relres host double*, may be NULL: TRUE relative residual ||b-Ax||/||b||
 *         recomputed in FP64 at exit.
 * Errors: SMG_ENOTCONV (iters = maxit), SMG_EBREAKDOWN (p^T A p <= 0 in CG),
 * SMG_ENAN, SMG_EINVAL, SMG_ECUDA, SMG_ETIMEOUT. */
int smg_solve(smg_t h, const double* b, double* x, double tol, int maxit, int* iters, double* relres, void* stream);

/* Hierarchy statistics (Eq. 2 complexities, Sec. 6.2).
 *  grid_complexity = sum_l n_l / n_0;  operator_complexity = sum_l n_l*ns_l /
 *  (n_0*ns_0) (SG-DIA storage counts every row as ns_l entries);
 *  vcycle_bytes = algorithmic HBM bytes of one V-cycle (each array touched
 *  once per kernel); setup_ms = device time of the last smg_setup. */
typedef struct {
  int levels;
  int dims[16][3];
  int nstencil[16];
  double grid_complexity, operator_complexity;
  double vcycle_bytes, vcycle_fp64_flops;
  double setup_ms;
  int precision, smoother, transfer, block;
} smg_stats_t;
int smg_stats(smg_t h, smg_stats_t* out);

void smg_destroy(smg_t h);
const char* smg_strerror(int status);

/* ---------------------------------------------------------------------------
 * Level-wise building blocks.  They run the same kernels as the V-cycle, one
 * at a time, on the hierarchy's own level data, for callers that compose
 * their own cycle and for parity testing.  Level 0 is the finest.
 * ------------------------------------------------------------------------- */

/* Number of levels, and dims / stencil (lexicographic offsets, int[27][3])
 * of level l.  Errors: SMG_EINVAL for a bad handle or level. */
int smg_level_count(smg_t h);
int smg_level_info(smg_t h, int l, int dims[3], int* nstencil, int* offsets);

/* Copy a level array into caller device memory `dst` of `bytes` bytes.
 * which: 0 A (double, layout above), 1 ILU(0) factors (double [n][ns]: unit-
 * lower L on lower offsets, U on centre and upper offsets), 2 inverse
 * diagonal (double: [n] for B == 1 / 1/u_pp for ILU, [n][B][B] for B == 3),
 * 3 low-precision matrix values ([n][ns] float for FP32, bf16 bits as
 * uint16 for BF16), 4 FP32 row scale of A [n], 5 low-precision ILU factors
 * ([n][ns] like 3: lower entries scaled by 6, upper by 7), 6 FP32 row scale of
 * L [n], 7 FP32 row scale of U [n], 8 FP32 inverse diagonal [n].
 * On levels whose ILU(0) sweeps read the skewed records, 5-8 are not kept
 * after set-up: the first request for one of them allocates and computes
 * all four on `stream` (SMG_ENOMEM if that allocation fails).
 * Returns SMG_EINVAL if the array does not exist on that level or bytes is
 * smaller than its size; writes the size to *needed if not NULL. */
int smg_level_copy(smg_t h, int l, int which, void* dst, size_t bytes, size_t* needed, void* stream);

/* Level operations (vectors are device arrays in the level's V-cycle
 * precision: double for FP64 hierarchies, float otherwise; B values/point).
 *  SMG_OP_SPMV         y = A x                               (x, -, y)
 *  SMG_OP_RESIDUAL     y = b - A x                           (x, b, y)
 *  SMG_OP_GS_FORWARD   x <- GS-Forward sweep on A x = b      (x, b, -) in place
 *  SMG_OP_GS_BACKWARD  x <- GS-Backward sweep                (x, b, -) in place
 *  SMG_OP_GS_ZERO      x <- GS-Forward from x = 0 (ZeroGuess) (x, b, -)
 *  SMG_OP_ILU_APPLY    y = U^{-1} L^{-1} b                    (-, b, y)
 *  SMG_OP_RESTRICT     y(level l+1) = R x(level l)           (x, -, y)
 *  SMG_OP_PROLONG_ADD  y(level l) += P x(level l+1)          (x, -, y)
 *  SMG_OP_COARSE_SOLVE y = A_c^{-1} b on the coarsest level (-, b, y), double
 *  SMG_OP_ILU_LOWER    y = L^{-1} b (unit lower solve only; y may equal b)
 *  SMG_OP_ILU_UPPER    y = U^{-1} b (upper solve only; y may equal b)
 *  SMG_OP_LGS_FORWARD  x <- forward line sweep on A x = b    (x, b, -) in place
 *  SMG_OP_LGS_BACKWARD x <- backward line sweep              (x, b, -) in place
 *  SMG_OP_LGS_ZERO     x <- forward line sweep from x = 0    (x, b, -)
 * A one-level hierarchy keeps its smoother data, so the sweeps are available
 * on level 0 even when it is also the coarsest level.
 * Errors: SMG_EINVAL (bad level/op/missing smoother data), SMG_ECUDA,
 * SMG_ETIMEOUT. */
enum {
  SMG_OP_SPMV = 0, SMG_OP_RESIDUAL = 1, SMG_OP_GS_FORWARD = 2, SMG_OP_GS_BACKWARD = 3, SMG_OP_GS_ZERO = 4,
  SMG_OP_ILU_APPLY = 5, SMG_OP_RESTRICT = 6, SMG_OP_PROLONG_ADD = 7, SMG_OP_COARSE_SOLVE = 8,
  SMG_OP_ILU_LOWER = 9, SMG_OP_ILU_UPPER = 10, SMG_OP_LGS_FORWARD = 11, SMG_OP_LGS_BACKWARD = 12,
  SMG_OP_LGS_ZERO = 13
};
int smg_level_apply(smg_t h, int l, int op, const void* x, const void* b, void* y, void* stream);

/* Warps per 32-column strip of the wavefront kernel that runs the point
 * sweep `op` (SMG_OP_GS_FORWARD / GS_BACKWARD / GS_ZERO / ILU_LOWER /
 * ILU_UPPER) of level l, in the V-cycle and in smg_level_apply: 2 the two-
 * warp kernel (option sweep_warps), 1 the one-warp warp-pipelined kernel,
 * 0 another kernel (or the level has no such sweep).  Host-only: reports the
 * choice the launch makes, launches nothing.  Errors: -SMG_EINVAL for a bad
 * handle, level or op. */
int smg_level_sweep_warps(smg_t h, int l, int op);

/* Number of CUDA kernels this library has enqueued since it was loaded (a
 * V-cycle replayed from a CUDA graph counts its kernels on every replay).
 * Host-only; never fails. */
long long smg_launch_count(void);

/* Failure-path self-test of the bounded device waits: launches one wait on a
 * device flag that nothing ever sets, with a budget of budget_ms (1..10000).
 * Returns SMG_ETIMEOUT when the wait ran out as designed (the context stays
 * usable), SMG_EINVAL for bad arguments, SMG_ECUDA on a CUDA failure. */
int smg_selftest_wait(smg_t h, int budget_ms, void* stream);

/* Replaces the bound of every device-side wait of the context's kernels
 * (smg_options.spin_budget_ms at set-up) by budget_ns nanoseconds, 0 <=
 * budget_ns <= 10 s.  With 0, a wait that is not satisfied at its first check
 * gives up at once: the kernels then take their abort path (error word set,
 * every CTA drains, bulk copies in flight are waited for with a fixed bound
 * of their own) and the call that launched them returns SMG_ETIMEOUT, after
 * which the context is unchanged and usable -- the failure path can be
 * exercised without a GPU fault.  A captured V-cycle graph is dropped (it
 * holds the old bound).  Host-only; SMG_EINVAL for a bad handle or budget. */
int smg_set_wait_budget_ns(smg_t h, long long budget_ns);

/* ---------------------------------------------------------------------------
 * Host-only symbolic derivation of influence chains (Sec. 4.3, Eq. 5-10).
 * Given R, A^F, P patterns as fine-grid offsets -- R and P relative to the
 * fine anchor of their coarse point, A relative to the fine point -- a chain
 * (r, a, q) links coarse point I to coarse neighbour I + dJ when
 * roff[r] + aoff[a] - poff[q] = 2*dJ (stride-2 coarsening).  dim = 2 or 3
 * (z components ignored/zero for 2).  Writes up to max_chains chains as
 * int[5] {r, a, q, dJ lexicographic index in {-1,0,1}^dim, 0} and returns the
 * total chain count, or -1 if a chain reaches a coarse offset outside
 * {-1,0,1}^dim or an argument is invalid.  No GPU is used.
 * ------------------------------------------------------------------------- */
int smg_derive_chains(int dim, int nr, const int* roff, int na, const int* aoff, int np, const int* poff,
                      int max_chains, int* chains);

/* Host-only: the Galerkin chain table the hierarchy set-up uses for one
 * transfer (SMG_TRANSFER_*) on a fine mask of nstencil offsets (int[3] each,
 * any order).  Returns the number of chains (Table 2 counts them: 1216 for
 * C64C on 19 points, 1728 on 27) and writes the coarse mask size to
 * *ncoarse if it is not NULL; -1 for an unknown transfer or a mask the
 * derivation rejects.  No GPU is used. */
int smg_rap_chain_count(int transfer, int nstencil, const int* offsets, int* ncoarse);

/* ---------------------------------------------------------------------------
 * Learned post-smoother (not in the paper).  A three-layer 3x3x3
 * convolutional network f (2 -> 16 -> 16 -> 1 channels, ReLU after the first
 * two layers, zero padding) maps the scaled residual and the log-coefficient
 * field to a correction.  Convolutions are implicit GEMMs on the tensor cores
 * with BF16 operands and FP32 accumulation.
 * Parameters: an FP32 device vector of smg_cnn_param_count() = 8241 values,
 * W1[16][2][3][3][3] b1[16] W2[16][16][3][3][3] b2[16] W3[1][16][3][3][3]
 * b3[1]; tap (a,b,c) multiplies the input at offset (a-1, b-1, c-1).
 * Volumes: FP32, grid layout of the matrices; in2 = two planes [2][n]
 * (channel 0, channel 1).  ws: caller-allocated device workspace of at least
 * smg_cnn_workspace_bytes(dims) bytes.  All calls are asynchronous on the
 * stream except smg_cnn_forward (synchronises).  Errors: SMG_EINVAL for bad
 * sizes, NULL pointers or a short workspace; SMG_ECUDA.
 * ------------------------------------------------------------------------- */
int smg_cnn_param_count(void);
int smg_cnn_workspace_bytes(const int dims[3], size_t* bytes);
/* out[n] = f(in2) */
int smg_cnn_forward(const int dims[3], const float* theta, const float* in2, float* out, void* ws, size_t ws_bytes,
                    void* stream);
/* loss += mean_p (f(in2)_p - target_p)^2 ; grad[8241] += d loss / d theta
 * (loss is one FP32 device scalar; both are accumulated, not overwritten). */
int smg_cnn_loss_grad(const int dims[3], const float* theta, const float* in2, const float* target, float* grad,
                      float* loss, void* ws, size_t ws_bytes, void* stream);
/* One Adam step (bias-corrected, step counts from 1) on n parameters with the
 * gradient multiplied by grad_scale. */
int smg_cnn_adam(int n, float* theta, float* m, float* v, const float* grad, int step, float lr, float beta1,
                 float beta2, float eps, float grad_scale, void* stream);
/* Attaches the network as a post-smoother of the finest level, applied after
 * every V-cycle: r' = r - A z, s = ||r'||_2 / sqrt(n),
 * delta = s * D^-1 f(r'/s, logk) with D the diagonal of A (the network
 * learns a correction relative to a Jacobi step), and z += delta only if
 * ||r' - A delta||_2 < ||r'||_2 (otherwise the plain V-cycle result is kept).  theta (FP32
 * [8241]) is packed at this call; logk (double [n], the log of the diffusion
 * coefficient) must stay valid while attached.  theta == NULL detaches.
 * The preconditioner is then nonlinear: the context's Krylov method must be
 * FPCG or FGMRES (SMG_EINVAL otherwise); one unknown per point only. */
int smg_set_learned_smoother(smg_t h, const float* theta, const double* logk, void* stream);
/* Where the attached network acts (not in the paper).  SMG_LEARNED_AFTER
 * (default): after the whole V-cycle, as above.  SMG_LEARNED_REPLACE: in
 * place of the finest level's post-smoothing: the V-cycle skips that
 * smoothing (also in smg_learned_sample, so the training pairs are the
 * residuals the coarse correction leaves), the correction is tested the same
 * way, and when it is rejected the skipped post-smoothing runs, so the
 * result is then exactly the plain V-cycle's (the decision is read back to
 * the host: one synchronisation per V-cycle).  FP64 hierarchies only.
 * Errors: SMG_EINVAL (NULL handle, bad mode, reduced-precision hierarchy). */
enum { SMG_LEARNED_AFTER = 0, SMG_LEARNED_REPLACE = 1 };
int smg_set_learned_mode(smg_t h, int mode);
/* One training pair for the post-smoother, built on the device from a known
 * error e0 (double [n], device): r0 = A e0, z = V-cycle(r0) (the plain one,
 * even when a network is attached), e1 = e0 - z (the exact error the V-cycle
 * leaves), r' = A e1, s = ||r'||_2 / sqrt(n); writes in2 = [r'/s ; logk]
 * (float [2][n]) and target = D e1 / s (float [n], D the diagonal of A: the
 * network output that would reproduce e1 exactly).  Synchronous on the
 * stream.  Errors: SMG_EINVAL (NULL pointer, B != 1), SMG_ECUDA, sweep
 * errors. */
int smg_learned_sample(smg_t h, const double* e0, const double* logk, float* in2, float* target, void* stream);
/* Loss and gradient of one training pair on this context's finest grid
 * (ws: smg_cnn_workspace_bytes of that grid).  kind SMG_LOSS_ERROR: the
 * error MSE of smg_cnn_loss_grad (target used).  kind SMG_LOSS_RESIDUAL:
 * the residual the correction leaves, loss += |A D^-1 y - in2[0..n)|^2 / n
 * with y = f(in2), A the finest matrix (FP64, assumed symmetric) and D its
 * diagonal (target unused): the quantity the acceptance test compares.
 * Both accumulate into grad and loss; asynchronous on the stream.
 * Errors: SMG_EINVAL (NULL pointer, B != 1, bad kind, short ws), SMG_ECUDA. */
enum { SMG_LOSS_ERROR = 0, SMG_LOSS_RESIDUAL = 1 };
int smg_learned_loss_grad(smg_t h, const float* theta, const float* in2, const float* target, int kind, float* grad,
                          float* loss, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * One Gauss-Seidel or ILU(0) triangular sweep that allocates no memory.
 * No counterpart in the paper: it exists for callers that cannot let a
 * library allocate device memory -- applications that own every byte of the
 * GPU through their own pool, fixed-budget real-time or embedded callers,
 * plug-ins whose host forbids cudaMalloc (it synchronises the device and
 * fragments the host's pool).  It needs no context: the caller passes the
 * matrix and vectors, and the sweep's scratch (progress counters per plane
 * and warp, plane ticket, error word: about 256 KB) is a fixed array in device memory
 * that every GPU which loads this library keeps until the process exits.
 *  op        SMG_OP_GS_FORWARD / SMG_OP_GS_BACKWARD / SMG_OP_GS_ZERO (u is
 *            the iterate, updated in place, b the right-hand side, dinv the
 *            inverse diagonal 1/a_pp), SMG_OP_ILU_LOWER (u = L^{-1} b, M the
 *            ILU(0) factors of smg_level_copy which 1, dinv unused, u may
 *            equal b), SMG_OP_ILU_UPPER (u = U^{-1} b, dinv = 1/u_pp, u may
 *            equal b).  The results equal smg_level_apply's for the same op.
 *  dims      host int[3]; nx <= 4096 (the scratch holds 16 counters per
 *            x-plane), ny <= 1024, nz <= 4096.
 *  nstencil, offsets  host; offsets in lexicographic order (dx slowest),
 *            unique, symmetric, with the centre (no reordered copy is made).
 *  M, dinv, b, u  device double, one value per point, layouts as above.
 *  relax_w   GS weight in (0, 2); 0 means 1.  spin_budget_ms: bound on any
 *            device-side wait (<= 0 means 1000).
 * FP64, one unknown per point.  The first call on a device looks up the
 * scratch's device address (cudaGetSymbolAddress) and caches it; make that
 * first call before capturing a stream.  All calls share the scratch and
 * each clears the part that must start at zero, so two calls that overlap
 * on the GPU (different streams, or threads without ordering) race and must
 * not be issued.  Calls no allocating routine.  Synchronises the stream.
 * Errors: SMG_EINVAL (sizes beyond the limits above, unsorted or invalid
 * offsets, bad op or pointers), SMG_ECUDA, SMG_ETIMEOUT.
 * ------------------------------------------------------------------------- */
int smg_sweep_noalloc(int op, const int dims[3], int nstencil, const int* offsets, const double* M,
                      const double* dinv, const double* b, double* u, double relax_w, int spin_budget_ms,
                      void* stream);

/* Library version string. */
const char* smg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SMG_H */
