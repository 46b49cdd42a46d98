/*
 * s3ttv.h - C ABI of a GB300 (sm_103a) solver for S3TTV hyperspectral
 * denoising and destriping (Takemoto, Naganuma, Ono, "Spatio-Spectral Structure
 * Tensor Total Variation for Hyperspectral Image Denoising and Destriping").
 *
 * The solver runs the preconditioned primal-dual splitting of Alg. 1 (Sec. III-C)
 * on Prob. (S3TTV_denoising) (Sec. III-B):
 *
 *     min_{u,s,t}  sum_l || P_l D D_s u ||_*
 *     s.t.  ||s||_1 <= alpha,  ||t||_1 <= beta,  D_v t = 0,
 *           ||u + s + t - v||_2 <= eps,  mu_min <= u <= mu_max,
 *
 * where D_v, D_h, D_s are forward differences with periodic boundaries along the
 * vertical (first), horizontal (second) and spectral (third) axes (Sec. II-A),
 * and P_l extracts the k x k x N3 block anchored at pixel l (eq. rewrite_Lu).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Cube layout: FP32, C-contiguous [N1][N2][N3], band fastest: element (i, j, b)
 *   is at offset (i*N2 + j)*N3 + b (a torch tensor of shape (N1, N2, N3)).
 * Blocks: one per anchor pixel l = p*N2 + q (all N1*N2 stride-1 windows, wrapped
 *   periodically as the footnote of Sec. III-A describes), covering pixels
 *   ((p+a) mod N1, (q+c) mod N2), a, c in [0, k).  A block matrix has k*k rows
 *   (row r = a*k + c) and 2*N3 columns in the order of eq. (SSST): column 2b holds
 *   D_v D_s, column 2b+1 holds D_h D_s of band b.  The block dual "Y" is stored
 *   [N1*N2][k*k][2*N3] in that order.
 * Pointers: unless an entry point says otherwise, a data pointer may point to
 *   device memory of the context's GPU or to host memory (pageable or pinned);
 *   the library asks the CUDA runtime which it is and stages host buffers through
 *   its own device workspace.  The caller owns every buffer it passes; the library
 *   never keeps a pointer past the call and never writes to an input.
 * Streams: all work runs on the context's stream; every entry point returns after
 *   that stream has finished the call's work (synchronous semantics).
 * Errors: each call returns an s3ttv_status; negative values are failures and
 *   leave the outputs untouched (argument errors are detected on the host before
 *   any launch).  s3ttv_last_error(ctx) gives a one-line description.  After
 *   S3TTV_ECUDA the context should be destroyed.  No C++ exception crosses the ABI.
 * Threads: a context must not be used by two host threads at the same time.
 */
#ifndef S3TTV_H
#define S3TTV_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct s3ttv_ctx s3ttv_ctx;

typedef enum s3ttv_status {
  S3TTV_OK = 0,            /* finished: the stop rule fired                          */
  S3TTV_MAXITER = 1,       /* finished: iteration cap reached first (results valid)  */
  S3TTV_EINVAL = -1,       /* invalid argument                                       */
  S3TTV_ENOMEM = -2,       /* device allocation failed                               */
  S3TTV_ECUDA = -3,        /* CUDA runtime error                                     */
  S3TTV_ENUMERIC = -4,     /* NaN or Inf appeared in the iterates                    */
  S3TTV_EUNSUPPORTED = -5, /* valid but outside what this library supports (see each call) */
  S3TTV_ESTATE = -6,       /* call made before s3ttv_setup                           */
  S3TTV_ETOOBIG = -7       /* input larger than an allocation-free entry point takes */
} s3ttv_status;

/* Per-call report.  Filled by the calls that take it (may be NULL). */
typedef struct s3ttv_info {
  int status;              /* the call's return value                                */
  int iters;               /* P-PDS passes completed by this call                    */
  int converged;           /* 1 if ||u+ - u|| / ||u|| < tol fired                    */
  int jacobi_nonconverged; /* blocks left with an unconverged eigen-solve (the FP32
                              sweep cap without the FP64 re-solve, or the re-solve's
                              own cap)                                              */
  double rel_change;       /* ||u+ - u||_2 / ||u||_2 of the last pass (eq. StopCri)  */
  double seconds;          /* host wall time of the call                             */
  double jacobi_sweeps;    /* mean eigen-solve sweeps per block and pass             */
  int jacobi_fallbacks;    /* blocks re-solved in FP64 after their FP32 eigen-solve
                              reached the sweep cap (S3TTV_OPT_FP64_FALLBACK)      */
  double first_order;      /* share of blocks and passes whose clip came from the
                              first-order update in the kept basis
                              (S3TTV_OPT_FIRST_ORDER)                              */
} s3ttv_info;

/* Step-size policies (option S3TTV_OPT_STEP_POLICY).
 * PAPER: eq. (stepsize_denoising) as printed: gamma_u = 1/(8L+1), L = N1*N2 blocks,
 *   gamma_s = 1, gamma_t = 1/3, gamma_Y = 1/4, gamma_y2 = 1/2, gamma_y3 = 1/3.
 * PC_EXACT: the same except gamma_u = 1/(8k^2+1), the exact column abs-sum of
 *   Lemma 1 (eq. Preconditioners) when every entry of D D_s u lies in k^2 blocks. */
enum { S3TTV_STEP_PAPER = 0, S3TTV_STEP_PC_EXACT = 1 };

/* Option keys for s3ttv_set_option. */
enum {
  S3TTV_OPT_STEP_POLICY = 1,       /* S3TTV_STEP_PAPER (default) or S3TTV_STEP_PC_EXACT  */
  S3TTV_OPT_CHECK_EVERY = 2,       /* passes between host reads of the stop flag (default 16) */
  S3TTV_OPT_JACOBI_MAX_SWEEPS = 3, /* sweep cap of the block eigen-solve (default 24, 1..64) */
  S3TTV_OPT_JACOBI_TOL = 4,        /* relative orthogonality tolerance: a sweep of a
                                      block eigen-solve in which no pair of rows was
                                      less orthogonal ends the solve (default 1e-4)       */
  S3TTV_OPT_PROFILE = 5,           /* 1: time each kernel class of every pass with CUDA
                                      events on the context stream (resets the totals);
                                      0: off (default)                                    */
  S3TTV_OPT_WARM_START = 6,        /* 1 (default): each block's eigen-solve starts from the
                                      eigenbasis it converged to in the previous pass
                                      (same result, fewer sweeps; 4 (k^2+1) k^2 bytes of
                                      workspace per block); 0: every pass starts cold     */
  S3TTV_OPT_TENSOR_CORES = 7,      /* block duals (Alg. 1 steps 8-11), k <= 5: 2 (default)
                                      forms the Gram Y'Y'^T and the product M Y' on tensor
                                      cores, each FP32 operand split into two TF32 parts and
                                      three of the four part products kept (FP32-level
                                      accuracy), every warp streaming one block of its own
                                      through double-buffered column chunks; 1: the same
                                      products with the four warps of a CTA sharing each
                                      block of a group of four; 0: the group form with FP32
                                      FMAs on CUDA cores                                  */
  S3TTV_OPT_LAYOUT = 8,            /* block matrices X_l: S3TTV_LAYOUT_PAPER (default) or
                                      S3TTV_LAYOUT_STACKED (below)                        */
  S3TTV_OPT_SPECTRAL_BOUNDARY = 9, /* D_s: S3TTV_SPECTRAL_PERIODIC (default, Sec. II-A)
                                      or S3TTV_SPECTRAL_OPEN (below)                      */
  S3TTV_OPT_REGULARIZER = 10,      /* the regularisation function of the problem:
                                      S3TTV_REG_S3TTV (default) or a comparison one (below) */
  S3TTV_OPT_AUTOTUNE = 11,         /* 1: the first s3ttv_iterate (or s3ttv_solve) of a
                                      problem shape with k <= 5 runs two passes, then one
                                      pass of every compiled block-dual form that fits
                                      (tensor or CUDA cores x CTAs per SM), twice each,
                                      timed with CUDA events, and keeps the fastest for
                                      the context (these are passes of the solve; the
                                      forms agree to FP32 rounding).  0 (default): the
                                      occupancy rule and S3TTV_OPT_TENSOR_CORES choose */
  S3TTV_OPT_HSSTV_OMEGA = 12,      /* HSSTV's weight omega of the first-order differences
                                      (default 0.05, (0, 2])                              */
  S3TTV_OPT_FP64_FALLBACK = 13,    /* 1 (default): a block whose FP32 eigen-solve reaches
                                      S3TTV_OPT_JACOBI_MAX_SWEEPS is re-solved in FP64 in
                                      the same pass (FP64 Gram and one-sided Jacobi,
                                      tolerance 1e-13, up to 80 sweeps; one extra launch
                                      per pass, which returns at once when no block is
                                      queued; up to 65,536 blocks per pass, the rest are
                                      applied as they stand and counted in
                                      jacobi_nonconverged); its warm-start rows start
                                      cold next pass.  0: such blocks are applied as
                                      they stand.  info.jacobi_fallbacks counts the
                                      re-solved blocks                                    */
  S3TTV_OPT_ALLOC_LIMIT = 14,      /* device bytes the context may hold (0, the default: no
                                      limit); an allocation past it fails with
                                      S3TTV_ENOMEM as a failed cudaMalloc would, and the
                                      context stays usable (host-side fault injection)    */
  S3TTV_OPT_NVTX = 15,             /* 1: NVTX ranges around each API call and each kernel
                                      class as a pass is enqueued (primal, l1-ball
                                      thresholds, block dual, dual, finalize), for
                                      profilers; 0 (default): none                        */
  S3TTV_OPT_JACOBI_POLISH_TOL = 16, /* relative orthogonality below which a pair of rows
                                      of the block eigen-solve is left as it is (0 <
                                      value <= S3TTV_OPT_JACOBI_TOL).  Every sweep
                                      rotates the pairs above it, but only a pair above
                                      the tolerance makes the solve run another sweep:
                                      a last sweep whose rotations stay below the
                                      tolerance tau moves a pair it already met by about
                                      n tau^2 at most.  0 (default): 2.5e-7, near the
                                      FP32 rounding of a row pair's dot product        */
  S3TTV_OPT_FIRST_ORDER = 17,      /* k <= 5, paper layout: a block whose stored
                                      eigen-rows W still nearly diagonalise this pass's
                                      Gram G takes its clip from the first-order
                                      (Daleckii-Krein) expansion of f(G) = min(1,
                                      G^-1/2) in that basis, B = W G W^T = D + O:
                                      M = W^T (f(D) + [f; d_i, d_j] o O) W, with no
                                      eigen-solve, when no eigenvalue can reach the kink
                                      at 1 (||O||_F < min |d_i - 1| / 4) and the bound
                                      on the neglected second-order term, ||O||_F^2
                                      times half the largest |f''| near the spectrum,
                                      is at most this value; the other blocks run the
                                      eigen-solve, which refreshes W.  Suggested 1e-6;
                                      0 (default): every warm block runs the
                                      eigen-solve                                     */
  S3TTV_OPT_BATCH_WORKLIST = 18    /* s3ttv_solve_batched with the streaming block-dual
                                      form (k <= 5, S3TTV or STV): 1 runs the block duals
                                      of every problem as one persistent launch per block
                                      side over a work list of all their blocks, between
                                      each pass's steps before and after them on the
                                      problems' own streams; 0 (default, faster: the
                                      problems' small kernels overlap their block duals):
                                      every problem's passes run on its own stream with
                                      its own block-dual launches                     */
};
/* Regularisers (option S3TTV_OPT_REGULARIZER).  Sec. IV runs its P-PDS-solvable
 * comparison methods by replacing S3TTV in Prob. (S3TTV_denoising) and solving
 * with the same P-PDS; five of them are built:
 *   S3TTV_REG_STV   sum_l || P_l D u ||_*: the nuclear norms of structure
 *                   tensors of first-order spatial differences (k^2 x 2N3
 *                   blocks, same block-dual path; the primal step has no D_s^T);
 *   S3TTV_REG_SSTV  || D D_s u ||_1: the dual is the cube pair (Y_v, Y_h) and
 *                   its conjugate prox is the clip to [-1, 1];
 *   S3TTV_REG_HSSTV1, S3TTV_REG_HSSTV2, S3TTV_REG_SSST: below.
 * Their step sizes are the exact Lemma 1 values of their operators
 * (STV: gamma_u = 1/(4k^2 + 1), gamma_Y = 1/2; SSTV: gamma_u = 1/9,
 * gamma_Y = 1/4; S3TTV_OPT_STEP_POLICY applies to S3TTV only).  With SSTV the
 * external "Y" state is [2][N1][N2][N3] (Y_v then Y_h) and s3ttv_block_dual
 * returns S3TTV_EUNSUPPORTED.  Changing the option drops the problem set up. */
enum {
  S3TTV_REG_S3TTV = 0,
  S3TTV_REG_STV = 1,
  S3TTV_REG_SSTV = 2,
  S3TTV_REG_HSSTV1 = 3,
  S3TTV_REG_HSSTV2 = 4,
  S3TTV_REG_SSST = 5
};
/* HSSTV (Hybrid SSTV): || (D_v D_s u, D_h D_s u, omega D_v u, omega D_h u) ||, the
 * l1 norm (S3TTV_REG_HSSTV1) or the l1,2 norm grouping each voxel's four entries
 * (S3TTV_REG_HSSTV2); the dual is four cubes ("Y" state [4][N1][N2][N3]) whose
 * conjugate prox clips each entry to [-1, 1] (l1) or scales each voxel's
 * 4-vector into the unit l2 ball (l1,2); gamma_u = 1/(9 + 4 omega), gamma_Y = 1/4
 * for all four parts (Lemma 1: row bounds 1/4 and 1/(2 omega)). */
/* SSST (spatio-spectral structure tensors): sum_l || P_l [D_v u, D_h u, D_s u] ||_*,
 * structure tensors of the first-order spatial and spectral differences, each a
 * k^2 x 3N3 block, row r the window pixel r, columns [v_1 h_1 s_1 ... v_N3 h_N3
 * s_N3]; the external "Y" state is [N1*N2][k*k][3*N3].  The blocks run on the
 * per-CTA path (FP32) for k <= 8, paper layout and periodic D_s only (other
 * settings return S3TTV_EUNSUPPORTED); gamma_u = 1/(6k^2 + 1), gamma_Y = 1/2
 * (Lemma 1: column abs-sums 6k^2, row abs-sums 2); s3ttv_block_dual returns
 * S3TTV_EUNSUPPORTED; s3ttv_objective evaluates the sum of nuclear norms. */
/* Block-matrix layouts (option S3TTV_OPT_LAYOUT).  PAPER is eq. (SSST): X_l is
 * k^2 x 2N3, row r the window pixel r = a k + c, columns [v_1 h_1 ... v_N3 h_N3].
 * STACKED is the (2k^2) x N3 matrix of the vertical and horizontal differences
 * stacked as rows (row 2r: D_v D_s u at pixel r, row 2r + 1: D_h D_s u; one
 * column per band).  The two hold the same entries but are different matrices
 * (different nuclear norms); the paper's Prob. (S3TTV_denoising) uses PAPER.
 * STACKED supports k <= 8 and runs every block on the per-CTA path (FP32).
 * The external block-dual layout ("Y" in s3ttv_get_state / s3ttv_set_state /
 * s3ttv_block_dual) follows: [N1*N2][k*k][2*N3] (PAPER) or [N1*N2][2*k*k][N3]
 * (STACKED).  Spectral boundary (option S3TTV_OPT_SPECTRAL_BOUNDARY): PERIODIC
 * wraps D_s from the last band to the first (the paper, Sec. II-A); OPEN stops
 * at the last band, so X_l has N3 - 1 band columns (the library keeps the
 * band-N3 column and its dual at zero).  With STACKED and OPEN, X_l is the
 * (2k^2) x (N3 - 1) matrix.  Changing either option drops the problem set up
 * (S3TTV_ESTATE until the next s3ttv_setup or s3ttv_solve); the step sizes are
 * those of the PAPER / PERIODIC operator (its column and row sums bound the
 * others'), so Theorem 1's condition still holds. */
enum { S3TTV_LAYOUT_PAPER = 0, S3TTV_LAYOUT_STACKED = 1 };
enum { S3TTV_SPECTRAL_PERIODIC = 0, S3TTV_SPECTRAL_OPEN = 1 };

/* Kernel classes reported by s3ttv_kernel_stats. */
enum {
  S3TTV_KERNEL_PRIMAL = 0,     /* steps 2-7 for u, arguments of steps 3-4           */
  S3TTV_KERNEL_L1_SEARCH = 1,  /* l1-ball thresholds of steps 3-4 (5 launches/pass) */
  S3TTV_KERNEL_BLOCK_DUAL = 2, /* steps 8-11: block duals and their singular values */
  S3TTV_KERNEL_DUAL = 3,       /* steps 3-4 finish, 12, 13                          */
  S3TTV_KERNEL_FINALIZE = 4,   /* step 14 scalar and the stop rule                  */
  S3TTV_KERNEL_CLASSES = 5
};

/* Which part of the solver state s3ttv_get_state / s3ttv_set_state address. */
enum {
  S3TTV_STATE_U = 0,   /* primal u,  cube                                     */
  S3TTV_STATE_S = 1,   /* primal s,  cube                                     */
  S3TTV_STATE_T = 2,   /* primal t,  cube                                     */
  S3TTV_STATE_Y2 = 3,  /* dual y2 (of D_v t = 0), cube                        */
  S3TTV_STATE_Y3 = 4,  /* dual y3 (of the l2 fidelity ball), cube             */
  S3TTV_STATE_Y = 5    /* block duals Y_1 .. Y_L, [N1*N2][k*k][2*N3]          */
};

/* Create a context on CUDA device `device`.  `stream` is a cudaStream_t to run on,
 * or NULL for a stream the context creates and owns.  Allocates nothing on the
 * device until a problem is set up.  Returns S3TTV_EINVAL if out is NULL or the
 * device does not exist, S3TTV_ECUDA on a runtime failure. */
int s3ttv_create(s3ttv_ctx **out, int device, void *stream);

/* Free the context and all its device workspace.  NULL is allowed. */
void s3ttv_destroy(s3ttv_ctx *ctx);

/* Static text for a status code. */
const char *s3ttv_strerror(int status);

/* Text of the last failure seen by this context ("" if none). */
const char *s3ttv_last_error(const s3ttv_ctx *ctx);

/* Set an option (keys above).  Takes effect at the next setup/iterate. */
int s3ttv_set_option(s3ttv_ctx *ctx, int key, double value);

/* Bytes of device workspace the context holds now. */
long long s3ttv_workspace_bytes(const s3ttv_ctx *ctx);

/* Number of kernels the passes of Alg. 1 (s3ttv_iterate, s3ttv_solve,
 * s3ttv_solve_batched) have launched on this context since it was created (10
 * per pass of each problem, plus one per problem and call). */
long long s3ttv_launch_count(const s3ttv_ctx *ctx);

/* With S3TTV_OPT_PROFILE on: total device milliseconds (ms[c]) and launches
 * (launches[c]) of each kernel class c < S3TTV_KERNEL_CLASSES accumulated by
 * s3ttv_iterate / s3ttv_solve since profiling was switched on.  Host arrays of
 * S3TTV_KERNEL_CLASSES entries; either may be NULL. */
int s3ttv_kernel_stats(const s3ttv_ctx *ctx, double *ms, long long *launches);

/* Solve Prob. (S3TTV_denoising) for the observation v with Alg. 1 (Sec. III-C).
 *
 * v        observed cube [N1][N2][N3] (host or device).
 * eps      radius of the l2 fidelity ball (eq. constraint_fidel), >= 0.
 * alpha    radius of the l1 ball of the sparse noise s (eq. constraint_sparse), >= 0.
 * beta     radius of the l1 ball of the stripe noise t (eq. constraint_stripe), >= 0.
 * mu_min, mu_max  box of u (eq. constraint_box), mu_min < mu_max.
 * k        block side (k x k x N3 blocks), 1 <= k <= min(N1, N2); this library supports k <= 16
 *          (k <= 5 on the tensor-core or CUDA-core per-warp path, 6..16, the paper's
 *          own 10 x 10 blocks included, on a per-CTA path in FP32; from k = 13 the
 *          two k^2 x k^2 matrices of each block live in an L2-resident global
 *          scratch of the context, and the FP64 re-solve of blocks at the sweep cap
 *          is not available) and N1 * N2 < 2^31, N1 * N2 * N3 < 2^33
 *          (S3TTV_EUNSUPPORTED otherwise).
 * max_iter iteration cap, >= 1.
 * tol      stop when ||u+ - u||_2 / ||u||_2 < tol (eq. StopCri_simulated), >= 0;
 *          0 runs exactly max_iter passes.
 * u        output clean cube (required); s, t: output sparse / stripe noise (NULL skips).
 * info     optional report.
 * Initial values: u = v, s = t = 0, every dual 0.  Requires N3 >= 2.
 * Returns S3TTV_OK, S3TTV_MAXITER, or a negative status. */
int s3ttv_solve(s3ttv_ctx *ctx, const float *v, int N1, int N2, int N3,
                float eps, float alpha, float beta, float mu_min, float mu_max,
                int k, int max_iter, float tol,
                float *u, float *s, float *t, s3ttv_info *info);

/* One problem of a batch for s3ttv_solve_batched: the arguments s3ttv_solve
 * takes for one cube (same meaning, layout and checks). */
typedef struct s3ttv_problem {
  const float *v;          /* observed cube [N1][N2][N3], host or device           */
  int N1, N2, N3;
  float eps, alpha, beta;  /* radii of the three constraint sets                   */
  float mu_min, mu_max;    /* box of u                                             */
  int k;                   /* block side                                           */
  float *u, *s, *t;        /* outputs (u required; s, t may be NULL), host or device */
} s3ttv_problem;

/* Solve n independent problems (cubes of different sizes and block sides) with
 * Alg. 1, each exactly as s3ttv_solve would solve it alone (the same passes, the
 * stop rule eq. StopCri_simulated applied to each problem on its own), but
 * concurrently: every problem has its own workspace and stream inside ctx
 * (created on first use, kept for later calls, released by s3ttv_destroy), and
 * one chunk of S3TTV_OPT_CHECK_EVERY passes (rounded up to even) of every
 * problem is recorded once as a CUDA graph and replayed, one graph launch per
 * chunk.  Options set on ctx apply to every problem (profiling excepted).  The
 * paper has no counterpart: it denoises one scene at a time.
 *
 * problems: n >= 1 descriptions; max_iter >= 1 and tol >= 0 as in s3ttv_solve.
 * infos: NULL or n reports; infos[i].status is problem i's result and
 * infos[i].seconds the time from the call's start until problem i was seen
 * stopped (the host reads the stop flags after each chunk, so to within one
 * chunk of passes; the whole call for a problem that ran to max_iter).
 * Returns S3TTV_OK when every problem's stop rule fired, S3TTV_MAXITER when
 * some problem reached max_iter first (all results valid), or the first
 * negative status (s3ttv_last_error names the problem); a problem whose setup
 * fails leaves its outputs unwritten. */
int s3ttv_solve_batched(s3ttv_ctx *ctx, int n, const s3ttv_problem *problems, int max_iter, float tol,
                        s3ttv_info *infos);

/* Stepping interface (the same solver, split so a caller can time passes,
 * inspect or replace the state).  s3ttv_setup loads a problem (same arguments and
 * checks as s3ttv_solve) and sets the initial values; s3ttv_iterate runs up to n
 * passes of Alg. 1, stopping early when the relative change drops below tol
 * (tol = 0: exactly n passes); info->iters counts the passes it ran. */
int s3ttv_setup(s3ttv_ctx *ctx, const float *v, int N1, int N2, int N3,
                float eps, float alpha, float beta, float mu_min, float mu_max, int k);
int s3ttv_iterate(s3ttv_ctx *ctx, int n, float tol, s3ttv_info *info);

/* Copy one state variable out of / into the context (after s3ttv_setup).
 * `which` is an S3TTV_STATE_* value; cubes have N1*N2*N3 floats, Y has
 * N1*N2*k*k*2*N3 floats in the layout described at the top.  Setting Y also
 * rebuilds the context's sum_l P_l^T Y_l.  Returns S3TTV_ESTATE before setup. */
int s3ttv_get_state(s3ttv_ctx *ctx, int which, float *dst);
int s3ttv_set_state(s3ttv_ctx *ctx, int which, const float *src);

/* Projection onto the l1 ball {x : ||x||_1 <= radius} (the prox of Alg. 1
 * steps 3-4; Sec. III-C), with the same threshold search the solver uses.
 * x, out: n floats (host or device; may alias).  radius >= 0.  tau_out (host,
 * may be NULL) receives the soft threshold (0 when ||x||_1 <= radius, +inf when
 * radius = 0).  n may be 0. */
int s3ttv_l1_ball(s3ttv_ctx *ctx, const float *x, float *out, long long n,
                  double radius, double *tau_out);

/* Block dual update of Alg. 1 steps 8-11 for every block, as the solver runs it:
 * Y_l <- Y'_l - gamma_Y prox_{gamma_Y^-1 ||.||_*}(Y'_l / gamma_Y) with
 * Y'_l = Y_l + gamma_Y P_l D D_s ubar, which by Moreau's identity
 * (eq. ProxConjugate) clips the singular values of Y'_l at 1; then
 * Z = sum_l P_l^T Y_l is returned split into Zv (column 2b parts) and Zh.
 * Y: [N1*N2][k*k][2*N3], updated in place; ubar: cube; Zv, Zh: output cubes.
 * All host or device.  info (may be NULL) reports jacobi_nonconverged and
 * jacobi_fallbacks (blocks re-solved in FP64, S3TTV_OPT_FP64_FALLBACK).
 * Uses the context's workspace (replaces any problem set up before).
 * S3TTV_EUNSUPPORTED with the SSTV, HSSTV or SSST regularisers. */
int s3ttv_block_dual(s3ttv_ctx *ctx, float *Y, const float *ubar, float *Zv, float *Zh,
                     int N1, int N2, int N3, int k, float gamma_Y, s3ttv_info *info);

/* The block-dual form S3TTV_OPT_AUTOTUNE chose: *tensor_cores 1 or 0 and
 * *ctas_per_sm (4 or 5), or *tensor_cores = -1 and *ctas_per_sm = 0 when none
 * has been chosen.  Host pointers, required. */
int s3ttv_tuned_form(const s3ttv_ctx *ctx, int *tensor_cores, int *ctas_per_sm);

/* Objective value S3TTV(u) = sum_l || P_l D D_s u ||_* of Prob.
 * (S3TTV_denoising) (eq. rewrite_Lu): the sum of the nuclear norms of the
 * k^2 x 2N3 structure tensors of all N1*N2 blocks.  u: cube (host or device);
 * value: host double.  Computed in FP64 (the block entries from the FP32 cube,
 * the Gram of each block and a one-sided Jacobi on its rows, sigma =
 * sqrt(eigenvalue)); an evaluation aid, far slower than a solver pass.
 * With S3TTV_OPT_REGULARIZER set to a comparison regulariser the value is that
 * regulariser's (STV, SSST: the same FP64 nuclear norms of their blocks; SSTV,
 * HSSTV: their l1 or l1,2 norms); the layout and spectral boundary options
 * apply as in the solver.
 * S3TTV_ENUMERIC if u is not finite or a block does not converge; k <= 12
 * (each block's FP64 k^2 x k^2 Gram in shared memory; k = 13..16, which the
 * solver takes, return S3TTV_EUNSUPPORTED here) and k <= 8 for the stacked
 * layout and SSST. */
int s3ttv_objective(s3ttv_ctx *ctx, const float *u, int N1, int N2, int N3, int k, double *value);

/* Quality of a restored cube u against a reference cube ref (both host or
 * device, same shape), the measures of Sec. IV-A:
 *   mpsnr     eq. (MPSNR), peak 1, averaged over the bands left after dropping
 *             the first and last `trim` (all bands if N3 <= 2 trim);
 *   mssim     eq. (MSSIM): SSIM [Wang et al. 2004] of each of those bands with
 *             the 11 x 11 Gaussian window of standard deviation 1.5 over every
 *             pixel whose window lies inside the image, C1 = 0.01^2,
 *             C2 = 0.03^2 (dynamic range 1); needs N1, N2 >= 11;
 *   sam_mean  eq. (2D_SAM) averaged over all pixels, radians (a pixel where one
 *             spectrum is zero counts pi/2, where both are zero 0);
 *   sam_map   the 2-D SAM itself, N1*N2 floats [N1][N2] (host or device).
 * Any output may be NULL (its work is skipped).  Sums in FP64. */
int s3ttv_quality(s3ttv_ctx *ctx, const float *u, const float *ref, int N1, int N2, int N3, int trim,
                  double *mpsnr, double *mssim, double *sam_mean, float *sam_map);

/* Allocation-free l1-ball projection.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, such as code whose
 * device memory is owned by an arena or pool it may not bypass, a plug-in whose
 * host forbids allocation after start-up, or a real-time loop that must not
 * touch the allocator.  It computes what s3ttv_l1_ball computes, with the same
 * kernels, needs no context and allocates nothing: its scratch (the threshold
 * search state and 2048 histogram bins, about 24 KB) is a fixed array in the
 * library's device memory, which every GPU that loads the library holds until
 * the process exits.
 *
 * x, out   DEVICE pointers to n floats on the current CUDA device, or managed
 *          memory (x and out may be the same buffer); host pointers and
 *          memory of another device are rejected with S3TTV_EINVAL (staging
 *          them would need an allocation).
 * n        0 <= n <= S3TTV_L1_STATIC_MAX_N (the bins count in 32 bits); larger
 *          n returns S3TTV_ETOOBIG before any work.
 * radius   >= 0, finite.  tau_out (host, may be NULL) receives the threshold.
 * stream   cudaStream_t to run on, NULL for the default stream; the call returns
 *          after that stream has finished its work.
 * The first call on a device looks up the device address of the scratch array
 * (cudaGetSymbolAddress, with that device current) and keeps it for the life of
 * the process; do not call this entry point on a device after
 * cudaDeviceReset of that device (the
 * module is reloaded there and the kept address goes stale).  Every call reuses the same array and clears it
 * first, so calls that overlap on the GPU (other streams or host threads using
 * the same device at the same time) race and must not be issued. */
#define S3TTV_L1_STATIC_MAX_N 4294967295LL
int s3ttv_l1_ball_static(const float *x, float *out, long long n, double radius, double *tau_out,
                         void *stream);

/* Radii of eq. (RadiusSet) (Sec. IV-A): alpha = rho N p_s / 2,
 * beta = rho 0.5 N p_t (1 - p_s) / 2, eps = rho sqrt(sigma^2 N (1 - p_s)), and
 * eps = 0.01 when sigma = 0 (the paper's choice for its stripe-only case).
 * All output pointers are host pointers and required. */
int s3ttv_radii(long long N, double sigma, double p_s, double p_t, double rho,
                double *eps, double *alpha, double *beta);

/* Step sizes (u, s, t, Y, y2, y3) of a policy for an N1 x N2 image and block k,
 * written to gammas[6] (host). */
int s3ttv_step_sizes(int N1, int N2, int k, int policy, double gammas[6]);

/* The FP32 arithmetic rate of a device, measured (the denominator of the ALU
 * roofline of the eigen-solve-bound block-dual kernels): every thread of a full
 * grid (8 CTAs of 256 threads per SM) runs 8 independent chains of FMAs, scalar
 * (packed = 0) or packed FP32x2 (packed = 1), sized until one launch takes
 * 20 ms; *tflops = 2 flops per lane FMA / the CUDA-event time of that launch.
 * Synchronous, on a stream of its own; changes no device setting.  tflops is a
 * host pointer.  S3TTV_EINVAL for a NULL pointer or packed not 0/1,
 * S3TTV_ECUDA when the device cannot run it. */
int s3ttv_fp32_peak(int device, int packed, double *tflops);

/* ---------------------------------------------------------------------------
 * Learned warm start.  The paper has no network: Alg. 1 starts from u = v,
 * s = t = 0.  These entry points train and run a small 3-D convolutional U-Net
 * that maps a noisy cube v to an estimate of (u, s, t); s3ttv_set_state then
 * starts the solver there, and the solver alone decides the result.
 *
 * Network: 3 levels of 32 / 64 / 128 channels, two 3 x 3 x 3 convolutions per
 * level (zero padding, bias, ReLU), 2 x 2 x 2 mean pooling, nearest upsampling,
 * skip connections by channel concatenation [upsampled, skip], and a
 * 1 x 1 x 1 head to three channels h; the prediction is (v + h0, h1, h2).
 * Weights are used in BF16 (FP32 master copies for Adam), activations are
 * stored in BF16, products accumulate in FP32.  Training minimises the mean
 * squared error over all voxels and the three outputs.
 *
 * Parameters: one flat FP32 vector of s3ttv_net_param_count() values: for each
 * convolution in network order (e1a 1->32, e1b 32->32, e2a 32->64, e2b 64->64,
 * ba 64->128, bb 128->128, d2a 192->64, d2b 64->64, d1a 96->32, d1b 32->32) the
 * weight w[out][tap][in], tap = 9 (dz+1) + 3 (dy+1) + (dx+1), then the bias
 * b[out]; last the head Wh[3][32] and bh[3].
 *
 * Volumes: B volumes of D x H x W voxels, C-contiguous [B][D][H][W]; a cube
 * [N1][N2][N3] is B = 1, D = N1, H = N2, W = N3.  D, H and W must be positive
 * multiples of 4 and B*D*H*W <= 2^26 (S3TTV_EUNSUPPORTED beyond).  Data
 * pointers may be host or device memory, as for the solver.  Every call returns
 * after the network's stream has finished; the network owns its workspace
 * (about 700 bytes per voxel, grown on demand).  Status codes as above;
 * S3TTV_ESTATE until parameters are set.
 * ------------------------------------------------------------------------- */
typedef struct s3ttv_net s3ttv_net;

/* Number of parameters (1,411,651). */
long long s3ttv_net_param_count(void);

/* Create a network on `device`, running on `cuda_stream` (NULL: its own). */
int s3ttv_net_create(s3ttv_net **out, int device, void *cuda_stream);
void s3ttv_net_destroy(s3ttv_net *net); /* NULL-safe */
const char *s3ttv_net_last_error(const s3ttv_net *net);

/* Load parameters (param_count floats) and reset the Adam state. */
int s3ttv_net_set_params(s3ttv_net *net, const float *theta);
/* Copy the current FP32 parameters out (param_count floats). */
int s3ttv_net_get_params(s3ttv_net *net, float *theta);

/* Prediction: u, s, t (B*D*H*W floats each) from v. */
int s3ttv_net_forward(s3ttv_net *net, const float *v, int B, int D, int H, int W,
                      float *u, float *s, float *t);

/* Loss (mean squared error of the prediction against u_ref, s_ref, t_ref; host
 * double, may be NULL) and its gradient with respect to every parameter
 * (param_count floats in the parameter order, may be NULL). */
int s3ttv_net_gradient(s3ttv_net *net, const float *v, const float *u_ref, const float *s_ref,
                       const float *t_ref, int B, int D, int H, int W, double *loss, float *grad);

/* One training step: the gradient as above, then one Adam update (beta1 0.9,
 * beta2 0.999, eps 1e-8, bias-corrected) with learning rate lr in [0, 1].
 * `loss` (may be NULL) receives the loss before the update. */
int s3ttv_net_train_step(s3ttv_net *net, const float *v, const float *u_ref, const float *s_ref,
                         const float *t_ref, int B, int D, int H, int W, float lr, double *loss);

#ifdef __cplusplus
}
#endif

#endif /* S3TTV_H */
