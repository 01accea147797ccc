/*
 * mm.h — C ABI of libmm, a single-GPU (GB300, sm_103a) maximum-likelihood CMB map-maker.
 *
 * The library solves (P^T N^-1 P) m = P^T N^-1 d by preconditioned conjugate gradients
 * (El Bouhargani et al., "MAPPRAISER", Sect. 2 and 3):
 *   P      pointing matrix, one row per time sample with the three weights (1, cos 2psi, sin 2psi)
 *          at the sample's sky pixel (Sect. 2, data model with a half-wave plate);
 *   N^-1   block-diagonal inverse-noise weights, one symmetric banded Toeplitz block per
 *          (detector, stationary interval) with half-bandwidth lambda (Eq. MADCAP);
 *   M_BD   block-Jacobi preconditioner (P^T diag(N^-1) P)^-1, one 3x3 block per pixel (Sect. 3.2);
 *   PCG    Algorithm 1 with x_0 = 0 and the stop rule ||r_k|| < eps ||b|| (Sect. 3.2).
 *
 * Conventions shared by every entry point
 *   - Status: every call returns an mm_status value and never throws across the ABI.  On error,
 *     mm_last_error() returns a message for the calling thread.
 *   - Ownership: mm_plan copies every input it is given (host or device memory) into plan-owned
 *     device memory and keeps no caller pointer after it returns.  Output buffers belong to the
 *     caller.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All
 *     calls except mm_plan / mm_plan_destroy / mm_pcg_solve are asynchronous on that stream.
 *   - Map vectors passed to mm_apply_A / mm_precond / mm_pcg_solve / mm_rhs are float64 device
 *     arrays in the plan's compacted pixel order, laid out [nrhs][n_obs][3] (I, Q, U per pixel).
 *     Time-domain vectors (mm_apply_P / mm_apply_Pt / mm_apply_Ninv) are float64 [N] device arrays
 *     in the sample order of the plan (blocks det-major, contiguous).
 *   - A plan is not thread-safe: calls on one plan must be serialised by the caller.
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_plan_s* mm_plan_t;
typedef struct mm_server_s* mm_server_t;
typedef int64_t mm_req_t;

typedef enum {
  MM_OK = 0,
  MM_EINVAL = 1,      /* invalid argument (sizes, pointers, pixel ids, non-finite band, ...) */
  MM_ENOMEM = 2,      /* device allocation failed */
  MM_ENOTSPD = 3,     /* a band's Fourier symbol is not positive, or no pixel survives excision */
  MM_EBREAKDOWN = 4,  /* <p, A p> <= 0 or not finite inside CG */
  MM_ENOTCONV = 5,    /* max_iter reached; the partial solution is returned */
  MM_ETIMEOUT = 6,    /* host-side deadline passed; the partial solution is returned */
  MM_EBUSY = 7,
  MM_ECUDA = 8        /* a CUDA runtime call failed */
} mm_status;

/* Arithmetic of the bulk operators P, N^-1, P^T (plan precision; a solve's opts->precision is
 * MM_FP64 or MM_FP32 and selects between the plan's FP64-class and FP32 operators).
 *   MM_FP64       FP64-class operators in IEEE FP64.
 *   MM_FP32       FP32 operators for the CG iterations; FP64-class operators in IEEE FP64.
 *   MM_DF64       FP64-class operators in double-float arithmetic: each value is a pair of FP32
 *                 numbers (hi + lo, a 48-bit significand) and the FFT runs on the FP32 pipes.
 *                 Normwise relative error of A x about 1e-14 instead of 1e-16.
 *   MM_FP32_DF64  FP32 operators for the CG iterations; FP64-class operators (right-hand side,
 *                 residual replacement, true residual) in double-float. */
enum { MM_FP64 = 0, MM_FP32 = 1, MM_DF64 = 2, MM_FP32_DF64 = 3 };
/* Algorithm of the block-Toeplitz product.
 *   MM_TPLZ_FFT     shared-memory overlap-save FFT tiles (every precision).
 *   MM_TPLZ_GEMM    the FP32 operators' N^-1 as banded Toeplitz-block GEMMs on the tensor cores
 *                   (tcgen05, 3xTF32, lambda <= 128, plans with FP32 operators); the FP64-class
 *                   operators keep the FFT tiles.
 *   MM_TPLZ_DIRECT  band sum by the definition (checks, tiny lambda).
 *   MM_TPLZ_AUTO    MM_TPLZ_GEMM where it measured faster than the FFT (FP32 operators, lambda up
 *                   to 64, the measured crossover), else MM_TPLZ_FFT. */
enum { MM_TPLZ_AUTO = 0, MM_TPLZ_FFT = 1, MM_TPLZ_GEMM = 2, MM_TPLZ_DIRECT = 3 };
/* Preconditioner: block-Jacobi, or the two-level a-posteriori A-DEF1 preconditioner built by
 * mm_deflation_build (Sect. 3.2, Eq. 2lvlDef). */
enum { MM_PREC_BD = 0, MM_PREC_2LVL_POST = 1 };

/*
 * Problem description (the map-making problem statement of Sect. 2 and 3).
 *   n_det, n_int   blocks are det-major: block b = det * n_int + interval, stored contiguously.
 *   block_len      HOST array [n_det * n_int] of samples per block (each >= 0); N = their sum.
 *   n_pix          number of global sky pixels; pix values must lie in [-1, n_pix).
 *   pix            [N] int32 global pixel per sample, -1 = flagged sample (a gap).
 *   psi            [N] float32 polarisation angle (radians); weights are (1, cos 2psi, sin 2psi).
 *   lambda         half-bandwidth: each block's first row has lambda + 1 coefficients c_0..c_lambda
 *                  (Eq. MADCAP keeps |t - t'| <= lambda).  0 <= lambda <= 12288.
 *   band           [n_det * n_int][lambda + 1] float64 first rows; every block's symbol
 *                  c_0 + 2 sum_k c_k cos(k w) must be positive (checked: MM_ENOTSPD).
 *   cond_max       pixels with fewer than 3 hits or cond_2 of their 3x3 block above cond_max are
 *                  excised together with their samples (Sect. 2.4); <= 0 selects 1e3.
 *   precision      MM_FP64, MM_FP32, MM_DF64 or MM_FP32_DF64 (above): arithmetic of mm_apply_A
 *                  (FP32 for MM_FP32 and MM_FP32_DF64) and of mm_rhs (the FP64-class operators).
 *   toeplitz_algo  MM_TPLZ_AUTO, MM_TPLZ_FFT, MM_TPLZ_GEMM or MM_TPLZ_DIRECT (above); MM_TPLZ_GEMM
 *                  needs lambda <= 128 and FP32 operators (MM_FP32 or MM_FP32_DF64), else MM_EINVAL.
 *   inputs_on_device  non-zero: pix, psi and band are device pointers; zero: host pointers.
 *   tile_steps     FP32 operators: overlap-save tiles walked by one CTA, which keeps the overlap
 *                  of consecutive tiles in shared memory (0 = chosen from the problem size).
 *   pt_sub         FP32 operators, the reduction of P^T: 0 = per-sample sums per pixel in shared
 *                  memory over the pixel windows; 4096, 8192 or 16384 = segment reduction over
 *                  pixel-sorted sub-windows of at most that many samples (runs of equal pixels
 *                  summed in registers; the plan stores the sorted order, 8 more bytes per sample).
 *                  Other values: MM_EINVAL.  mm_autotune times both forms.
 */
typedef struct {
  int32_t n_det;
  int32_t n_int;
  const int64_t* block_len;
  int64_t n_pix;
  const int32_t* pix;
  const float* psi;
  int32_t lambda;
  const double* band;
  double cond_max;
  int32_t precision;
  int32_t toeplitz_algo;
  int32_t inputs_on_device;
  int32_t tile_steps;
  int32_t pt_sub;
} mm_problem_desc;

/*
 * PCG options.
 *   tol            eps of the stop rule ||r|| < eps ||b|| (recursive residual of Algorithm 1).
 *   max_iter       cap on iterations (MM_ENOTCONV when reached).
 *   precond        MM_PREC_BD, or MM_PREC_2LVL_POST (needs mm_deflation_build on the plan).
 *   precision      MM_FP64: plain FP64 PCG.  MM_FP32: P, N^-1, P^T in FP32 with FP64 vectors,
 *                  dot products, alpha/beta and 3x3 blocks, and reliable updates: the recursive
 *                  residual is replaced by the FP64 true residual b - A x every `reliable_every`
 *                  iterations and before the solve is declared converged.
 *   reliable_every FP32 path only; <= 0 selects 50.
 *   check_every    iterations launched between host reads of the convergence flag (<= 0: 8).
 *   profile        0: each group of check_every iterations runs as one captured CUDA graph.
 *                  1: iterations are launched one by one and every Toeplitz-tile launch is
 *                  bracketed by CUDA events on the solve's stream (t_apply*_ms in mm_solve_info).
 *   deadline_us    host-side wall-clock limit in microseconds (<= 0: none) -> MM_ETIMEOUT.
 */
typedef struct {
  double tol;
  int32_t max_iter;
  int32_t precond;
  int32_t precision;
  int32_t reliable_every;
  int32_t check_every;
  int32_t profile;
  int64_t deadline_us;
} mm_solve_opts;

/* Per right-hand side outcome of a solve. */
typedef struct {
  int32_t status;        /* mm_status of this right-hand side */
  int32_t iters;         /* PCG iterations (A-applications inside the loop) */
  double rel_res;        /* final recursive ||r|| / ||b|| */
  double true_rel_res;   /* ||b - A x|| / ||b|| from an FP64 A-application after the solve */
  double t_ms;           /* wall time of the solve */
  int32_t n_true_res;    /* FP64 true-residual evaluations (FP32 path) */
  int32_t batch;         /* server: most requests that shared an A-application launch with it */
  double t_apply32_ms;   /* profile = 1: summed device time of the FP32 A-application launches */
  double t_apply64_ms;   /* profile = 1: same for the FP64 A-applications */
  int32_t n_apply32;     /* FP32 A-application launches (all columns in one launch) */
  int32_t n_apply64;     /* FP64 A-application launches */
  int64_t n_kernels;     /* kernels launched by the solve (its own, all columns) */
  double t_queue_ms;     /* server: time from mm_submit to admission (t_ms then runs to completion) */
  double t_unpoint32_ms; /* profile = 1: part of t_apply32_ms spent in the separate t = P x kernel */
  double t_point32_ms;   /* profile = 1: part of t_apply32_ms spent in the separate P^T kernel (0 when
                            the Toeplitz tiles scatter P^T themselves) */
} mm_solve_info;

/* Build a plan: validate, copy inputs, compact observed pixels, build and invert the 3x3 BD
 * blocks, excise ill-conditioned pixels, precompute the Toeplitz spectra.  Synchronous.
 * Sect. 3.1 (local pixel indexation, Toeplitz blocks), Sect. 2.4 and 3.2 (BD, excision). */
int mm_plan(const mm_problem_desc* desc, void* stream, mm_plan_t* out);

/* Sizes of a plan: n_obs kept pixels (map vectors hold 3 * n_obs values per right-hand side),
 * a device pointer to the [n_obs] compacted -> global pixel map (owned by the plan), the
 * number of samples and the plan's device footprint in bytes.  Any output may be NULL. */
int mm_plan_query(mm_plan_t plan, int64_t* n_obs, const int32_t** obs_to_global_dev,
                  int64_t* n_samples, size_t* bytes);

/* Release a plan and all its device memory.  NULL is a no-op. */
void mm_plan_destroy(mm_plan_t plan);

/* t = P~ x (un-pointing, Sect. 3.1): x [n_obs][3] -> t [N]; t = 0 at flagged/excised samples. */
int mm_apply_P(mm_plan_t plan, const double* x, double* t, void* stream);

/* y = P~^T t (pointing, Sect. 3.1): t [N] -> y [n_obs][3]; flagged/excised samples ignored. */
int mm_apply_Pt(mm_plan_t plan, const double* t, double* y, void* stream);

/* y = blockdiag_b T(c_b) t (stbmm, Sect. 3.1; Eq. MADCAP): t [N] -> y [N], FP64, no masking,
 * no wrap-around and no coupling across blocks. */
int mm_apply_Ninv(mm_plan_t plan, const double* t, double* y, void* stream);

/* b = P~^T N^-1 G d for nrhs data vectors: d [nrhs][N], float64 (d_is_fp32 = 0) or float32
 * (d_is_fp32 = 1), in device memory or in host memory (pinned or pageable); b [nrhs][n_obs][3]
 * device.  G zeroes flagged and excised samples of d.  A host d is copied by the library (on
 * double-float plans through two 64 MiB staging buffers of the plan, each chunk's copy overlapping
 * the previous chunk's conversion); the call then returns only after its work on the stream has
 * finished, so the host buffer may be reused at once.  With a device d the call is asynchronous. */
int mm_rhs(mm_plan_t plan, const void* d, int d_is_fp32, int nrhs, double* b, void* stream);

/* y = A x = P~^T N^-1 P~ x (Sect. 3.2, right to left) for nrhs vectors, in the plan's precision. */
int mm_apply_A(mm_plan_t plan, const double* x, double* y, int nrhs, void* stream);

/* Same as mm_apply_A, for callers that cannot allocate device memory (a fixed memory pool or
 * arena, a real-time loop, a host that accounts for all device memory itself).  The paper has
 * no counterpart: it is an interface choice of this library.  mm_apply_A grows plan-owned
 * working buffers with cudaMalloc on first use; this call instead uses one array of 32 MiB
 * compiled into the library, held by every GPU that loads it until the process exits, and calls
 * no cudaMalloc, cudaFree or other allocating routine.  Limits and rules:
 *   - nrhs * n_obs * 4 values of the plan's precision, twice (input and output), must fit in
 *     32 MiB (FP64: nrhs * n_obs <= 524,288; FP32: <= 1,048,576), else MM_EINVAL with a message;
 *   - FFT plans only (MM_TPLZ_DIRECT needs an N-sample buffer): MM_EINVAL otherwise;
 *   - the plan's own operator arithmetic, as mm_apply_A: FP32 on MM_FP32 and MM_FP32_DF64 plans,
 *     IEEE FP64 on MM_FP64 plans; MM_DF64 plans are refused with MM_EINVAL (their double-float
 *     operator needs an N-sample buffer), as are plans with templates;
 *   - every call shares the array and leaves its contents behind (each call clears what it
 *     accumulates), so calls whose GPU work overlaps (several streams or threads) race: the
 *     caller must serialise them;
 *   - the plan's device must be current; the first call on a device looks up the array's
 *     device address, so make it before any stream capture is under way on that device.
 * x, y: [nrhs][n_obs][3] float64 device arrays, as for mm_apply_A.  Asynchronous on stream. */
int mm_apply_A_noalloc(mm_plan_t plan, const double* x, double* y, int nrhs, void* stream);

/* z = M_BD r (block-Jacobi, Sect. 3.2) for nrhs vectors. */
int mm_precond(mm_plan_t plan, const double* r, double* z, int nrhs, void* stream);

/* Solve A x = b for nrhs independent right-hand sides by PCG (Algorithm 1), x_0 = 0.
 * b, x: [nrhs][n_obs][3] device.  info: HOST array [nrhs].  Blocks the calling thread until the
 * solve ends.  Returns the worst per-column status. */
int mm_pcg_solve(mm_plan_t plan, const double* b, double* x, int nrhs, const mm_solve_opts* opts,
                 mm_solve_info* info, void* stream);

/* Solve the map-making problem from the TOD: x = (P~^T N^-1 P~)^-1 P~^T N^-1 G d for nrhs data
 * vectors d [nrhs][N] (float64, or float32 with d_is_fp32; device memory, or host memory that the call
 * copies into a plan-owned device buffer grown on first use), by PCG (Algorithm 1) from
 * x_0 = 0 with the options of mm_pcg_solve.  With FP32 iterations (opts->precision MM_FP32) on an
 * MM_FP32_DF64 plan and the block-Jacobi preconditioner, the right-hand side is formed with the FP32
 * operators and every true residual is evaluated from the data as P~^T N^-1 G (d - P~ x) with the
 * double-float operator, so one FP64-class pass serves both the right-hand side's accuracy and the
 * final check (mm_rhs + mm_pcg_solve take two); the stop rule still requires the FP64-class true
 * residual below tol ||b||.  Any other combination runs mm_rhs (FP64-class b, written into x first)
 * and mm_pcg_solve.  x: [nrhs][n_obs][3] device; info: HOST [nrhs].  Blocks the calling thread.  The
 * paper's problem statement (Sect. 2): the TOD in, the map out. */
int mm_solve_tod(mm_plan_t plan, const void* d, int d_is_fp32, double* x, int nrhs, const mm_solve_opts* opts,
                 mm_solve_info* info, void* stream);

/* Autotuner of the FP32 A-application (an interface of this library; the paper has none).  Times
 * the plan's own FP32 A x (CUDA events on the plan's stream, median of a few runs, inputs of the
 * plan's size) over candidate configurations and keeps the fastest:
 *   1. FP32 overlap-save tiles walked per segment (1, 2, 4, ..., 32; a CTA keeps the overlap of
 *      consecutive tiles in shared memory, more segments keep more SMs busy); for lambda > 6144,
 *      also 65536-sample tiles split over 2-CTA clusters (more of each tile kept, but every CTA
 *      reads the whole tile);
 *   2. target samples per pixel-window group of P and P^T (8192 ... 65536);
 *   2b. the P^T reduction: per-sample shared-memory sums over the windows, or segment reduction
 *      over pixel-sorted sub-windows of at most 4096, 8192 or 16384 samples;
 *   3. block width for mm_block_cg_solve with block_width = 0: the widest of 1, 2, 4, ..., max_width
 *      whose device time per column of A X is within 2% of the best.
 * Every candidate's A x (of one filled input) is compared with the first candidate's; one that
 * differs by more than 1e-4 of the largest value is not chosen (n_rejected; max_rel_dev reports
 * the largest difference seen, FP32 rounding-order noise when all is well).
 * Results and every timing go to *out (HOST).  Rebuilds the plan's segments and windows (captured
 * solver graphs are captured again at the next solve).  Synchronous.  MM_EINVAL unless the plan
 * has FP32 operators with pixel windows (MM_FP32 or MM_FP32_DF64 FFT plan without templates). */
typedef struct {
  int32_t tile_steps;        /* chosen tiles per segment */
  int32_t win_samples;       /* chosen samples per window group */
  int32_t block_width;       /* chosen block width (columns per batched A X) */
  int32_t n_steps, n_win, n_width;
  int32_t steps_cand[8];
  double steps_ms[8];        /* one-column FP32 A x per candidate (ms) */
  int32_t win_cand[8];
  double win_ms[8];
  int32_t width_cand[8];
  double width_ms_per_col[8];
  double apply_ms;           /* one-column FP32 A x with the chosen configuration (ms) */
  int32_t big_tiles;         /* 1: 65536-sample tiles chosen, 0: timed and not chosen, -1: not a candidate */
  double big_tiles_ms;       /* their one-column FP32 A x (ms) when timed */
  double max_rel_dev;        /* largest relative difference of a candidate's A x from the first's */
  int32_t n_rejected;        /* candidates not chosen because their A x differed */
  int32_t seg_sub;           /* chosen P^T: sub-window samples of the segment reduction, 0 = windows */
  int32_t n_seg;
  int32_t seg_cand[4];       /* 0 = per-sample sums over the windows, else sub-window samples */
  double seg_ms[4];
} mm_tune_info;
int mm_autotune(mm_plan_t plan, int max_width, mm_tune_info* out, void* stream);

/* Solve A X = B for nrhs right-hand sides by block conjugate gradients: Algorithm 2 (Sect. 3.2)
 * in its block Orthomin form, applied with R_0 = [b_1 .. b_s] (s independent right-hand sides,
 * e.g. noise realisations, instead of one right-hand side split over subdomains):
 *   P_k = Z_k (Z_k^T A Z_k)^{-1/2} through a pivoted Cholesky factor (directions that became
 *   dependent are dropped; the paper leaves this case open), alpha_k = P_k^T R_{k-1},
 *   X_k = X_{k-1} + P_k alpha_k, R_k = R_{k-1} - A P_k alpha_k,
 *   Z_{k+1} = (I - P_k P_k^T A) M_BD R_k over the columns not yet converged.
 * The nrhs columns are solved in groups of block_width (0: min(nrhs, 64), or min(nrhs, the width
 * mm_autotune chose); at most 64), each group
 * sharing one batched A-application per iteration.  opts->precision selects FP32 or FP64
 * operators; the search blocks are FP32, X, R and the block_width x block_width matrices FP64.
 * A column stops when ||R_j|| < tol ||b_j||, confirmed by an FP64 true residual; columns above tol
 * restart from their true residual.  b, x: [nrhs][n_obs][3] device; info: HOST [nrhs]
 * (iters = block iterations to convergence).  With FP32 operators, a block that loses all its
 * directions away from a (re)start restarts from the FP64-class true residual (operator noise along
 * a null direction of a semi-definite A, as with templates); right after a restart that is a
 * breakdown.  Blocks the calling thread.  Returns the worst per-column status (MM_ENOTCONV after
 * opts->max_iter block iterations, MM_EBREAKDOWN). */
int mm_block_cg_solve(mm_plan_t plan, const double* b, double* x, int nrhs, int block_width,
                      const mm_solve_opts* opts, mm_solve_info* info, void* stream);

/* Variants of the enlarged CG recurrence (Sect. 3.2, ECG algorithm). */
enum { MM_ECG_ORTHOMIN = 0, MM_ECG_ORTHODIR = 1 };

/* Enlarged conjugate gradient for ONE right-hand side (Sect. 3.2, the ECG algorithm), x_0 = 0:
 * r_0 = b is split into t columns R_0 that sum to it (column i keeps the compacted pixels p with
 * floor(p t / n_obs) = i, all three Stokes parameters of a pixel together), Z_1 = M_BD R_0, and
 *   P_k = Z_k (Z_k^T A Z_k)^{-1/2} (pivoted Cholesky factor; dependent directions dropped),
 *   alpha_k = P_k^T R_{k-1}, X_k = X_{k-1} + P_k alpha_k, R_k = R_{k-1} - A P_k alpha_k,
 *   stop when ||sum_i R_k^(i)|| < tol ||b||, then
 *   MM_ECG_ORTHOMIN: Z_{k+1} = (I - P_k P_k^T A) M_BD R_k,
 *   MM_ECG_ORTHODIR: Z_{k+1} = (I - P_k P_k^T A - P_{k-1} P_{k-1}^T A) M_BD A P_k,
 * and x = sum_i X^(i).  Each iteration applies A to the whole t-column block at once (the batched
 * A X the paper names as the missing piece for ECG).  The stop is confirmed by an FP64-class true
 * residual ||b - A x||; above tol the recurrence restarts from it (at most 8 times).  The search
 * blocks are FP32, so the recursive residual can level off near 1e-7 ||b|| (Orthodir builds its
 * directions from A P_k and loses A-orthogonality in FP32): once below 1e-6 ||b||, a residual
 * ||sum_i R^(i)|| that has not halved in 10 block iterations also makes the solve check the true
 * residual and restart from it.
 *   t            enlarging factor, 1 <= t <= 64 (t = 1 is PCG).
 *   opts         tol, max_iter (block iterations), precision (MM_FP32: A on the search block in
 *                FP32; MM_FP64: the plan's FP64-class operator); precond must be MM_PREC_BD.
 * b, x: [n_obs][3] float64 device; info: HOST, one entry (iters = block iterations, batch = t).
 * Blocks the calling thread.  MM_ENOTCONV after max_iter iterations, MM_EBREAKDOWN when the block
 * loses all its directions on the first step from a (re)start or a norm is not finite (with FP32
 * search blocks a block that loses all its directions later restarts from the true residual, as
 * on semi-definite template systems); MM_EINVAL for bad arguments or a
 * MM_TPLZ_DIRECT plan. */
int mm_ecg_solve(mm_plan_t plan, const double* b, double* x, int t, int variant, const mm_solve_opts* opts,
                 mm_solve_info* info, void* stream);

/* Template map-making with diagonal weights (Sect. 2, Eq. genMapEstimator with the filtering operator
 * F_T = W - W T (T^T W T)^+ T^T W; the templates of Appendix A).  Attaches templates to a plan built
 * with lambda = 0, whose band rows c_0 = w_b are the diagonal weights W of each block; from then on
 * mm_apply_A, mm_rhs, mm_pcg_solve, mm_block_cg_solve, mm_ecg_solve and the deflation builders use
 * A = P~^T F_T P~ and b = P~^T F_T G d (the block-Jacobi preconditioner stays (P~^T W P~)^-1).
 * Templates per block (detector x stationary interval), one interval per block:
 *   n_poly    Legendre orders 0..n_poly-1 on x = 2 tau / (n - 1) - 1, scaled by sqrt((2k + 1) / n)
 *             (0..16);
 *   n_az      azimuth templates over the block's azimuth range [min, max] of its kept samples
 *             (0..64): az_interp = 0, bins (value 1 in bin floor((az - min) / (max - min) n_az));
 *             az_interp = 1, linear interpolation between n_az equally spaced nodes;
 *   n_hwp     harmonics cos(k phi), sin(k phi), k = 1..n_hwp, of the HWP angle phi (0..8).
 *   n_poly + n_az + 2 n_hwp must lie in [1, 64].
 *   az, hwp   [N] float32 per sample (host, or device with inputs_on_device); read during the call
 *             only (the caller keeps ownership; nothing keeps a pointer to them).
 * Setup: azimuth bins and interpolation fractions decided once in FP64 (every operator uses the
 * same ones), cos/sin of phi tabulated in FP32 and df64, each block's kernel T^T W T built in df64
 * (FP64-class) and pseudo-inverted (eigenvalues below 1e-12 of the largest dropped), and
 * M = P~^T W P~ per pixel.  The operators apply A x = M x - P~^T W T c with
 * c = (T^T W T)^+ T^T W P~ x in one fused kernel per application: FP32 for the FP32 (mixed-precision)
 * iterations, df64 for the FP64-class operator and b on every plan precision.  Plan memory grows by
 * about 25 B per sample (1 B bin, 8 + 16 B cos/sin of phi; + 12 B with interpolation; + 16 B of df64
 * pointing weights on plans that lack them) and 80 B per pixel.  Replaces previous templates.
 * Synchronous.  MM_EINVAL for a plan with lambda > 0, counts out of range or a block of 2^31 or
 * more samples; MM_ENOMEM when the tables do not fit; mm_apply_A_noalloc rejects such plans. */
typedef struct {
  int32_t n_poly;
  int32_t n_az;
  int32_t n_hwp;
  int32_t az_interp;
  const float* az;
  const float* hwp;
  int32_t inputs_on_device;
} mm_templates_desc;
int mm_templates_set(mm_plan_t plan, const mm_templates_desc* t, void* stream);

/* Noise weights estimated from the data (Sect. 2.2, how the weights are computed; the PSD model of
 * Eq. noisepowermodel with f_0 = 0).  For every block b of n_det * n_int (detector-major, block_len
 * HOST [n_det * n_int]):
 *   1. the averaged periodogram of its gap-masked TOD: max(1, floor(n / 32768)) segments of 32768
 *      samples (one zero-padded segment for a shorter block; a partial last segment is left out),
 *      P_k = |X_k|^2 / (kept samples of the segment), X the real DFT, averaged over segments;
 *   2. a Levenberg-Marquardt fit of log P_k by log(sigma^2 (1 + (f_knee / f_k)^alpha)) over
 *      k = 1..16384, f_k = k / 32768 cycles per sample, from a closed-form start (sigma^2 = mean of
 *      P_k over k >= 8192; a line through log(P_k / sigma^2 - 1) against log f_k over P_k > 3 sigma^2),
 *      steps bounded by 1 per parameter; without a 1/f excess (white noise) f_knee and alpha are
 *      not identifiable and any point of the flat valley may be returned;
 *   3. the first row of the block's inverse-noise Toeplitz matrix: 1/P on the 32768-point grid
 *      (1/P(0) := 0), inverse real DFT, Gaussian window N(0, lambda/2) over the lags, cut at lambda.
 *   pix, d   [N] device: int32 pixel (-1 = flagged sample) and float64 TOD.
 *   band     [n_det * n_int][lambda + 1] float64 device, written (zeros for a block without a kept
 *            sample); usable as mm_problem_desc.band.
 *   params   optional HOST [n_det * n_int][3]: log sigma^2, log f_knee (cycles per sample), alpha.
 * Transforms in FP32 (the tiles' shared-memory FFT), the fit with FP32 terms and FP64 sums.
 * Synchronous; allocates and frees its own scratch.  MM_EINVAL for bad sizes or lambda outside
 * [0, 12288]. */
int mm_estimate_bands(int32_t n_det, int32_t n_int, const int64_t* block_len, const int32_t* pix,
                      const double* d, int32_t lambda, double* band, double* params, void* stream);

/* Build the two-level a-posteriori deflation space of the plan (Sect. 3.2): m steps of the Lanczos
 * algorithm (Algorithm 3) on A (not M_BD A) from v_1 = b / ||b|| (x_0 = 0), storing A V_m; the
 * Ritz vectors of T_m = X Theta X^T give Z = V_m X and Z' = (A V_m) X (all m of them, as the paper
 * takes "all the precomputed vectors"); E = Z^T Z' and its pseudo-inverse (eigenvalues below
 * 1e-12 of the largest dropped).  b: [n_obs][3] float64 device; 1 <= m <= 64; precision selects
 * the FP32 or FP64 operator for the m A-applications.  Z, Z' are kept in FP32 on the plan and
 * replace any previous space.  Synchronous.  MM_EBREAKDOWN if b = 0. */
int mm_deflation_build(mm_plan_t plan, const double* b, int m, int precision, void* stream);

/* Build the two-level a-priori deflation space of the plan (Sect. 3.2, 2lvl a priori construction):
 * one column per stationary interval j (n_int of the plan; block b = det * n_int + j), whose total
 * intensity entry at pixel p is s_p^j / s_p, the fraction of p's kept samples that fall in interval
 * j (Q and U entries 0; the I rows are a partition of unity); then Z' = A Z, E = Z^T Z' and its
 * pseudo-inverse, as for mm_deflation_build, which it replaces.  precision selects the FP32 or
 * FP64-class operator for the n_int A-applications.  theta is left at 0.  Synchronous.
 * MM_EINVAL when n_int > 64.  The same MM_PREC_2LVL_POST solves and mm_deflation_apply use it. */
int mm_deflation_build_apriori(mm_plan_t plan, int precision, void* stream);

/* The plan's deflation space: *k columns; Z [k][n_obs][3] float64 device (may be NULL) and the
 * Ritz values theta [k] (HOST, may be NULL; 0 for an a-priori space).  *k = 0 when none was
 * built. */
int mm_deflation_get(mm_plan_t plan, int* k, double* Z, double* theta, void* stream);

/* z = M_2lvl r = M_BD (r - Z' E^-1 Z^T r) + Z E^-1 Z^T r (Eq. 2lvlDef0, applied right to left)
 * for nrhs vectors [nrhs][n_obs][3]; needs mm_deflation_build or mm_deflation_build_apriori.
 * Asynchronous on stream. */
int mm_deflation_apply(mm_plan_t plan, const double* r, double* z, int nrhs, void* stream);

/*
 * Serving: a request loop with continuous batching (an interface of this library; the paper has
 * none).  Requests wait in a queue and are admitted while fewer than max_slots are being planned or
 * run and the estimated device footprint of those stays within hbm_budget (a request is always
 * admitted when none is active).  Four planner threads build admitted requests' plans (pointing,
 * bands, spectra, block-Jacobi blocks), right-hand sides and PCG state on their own CUDA streams;
 * a server thread with one stream runs the iterations, one PCG iteration of every running request
 * per step; requests join between steps once planned and leave when they finish.  Their state
 * stays resident until then.
 *   FP32 requests (opts->precision MM_FP32): FP32 operators over pixel windows, P, N^-1 and P^T of
 *     all such requests in three shared launches per step (all their window groups, all their
 *     tile segments); right-hand side and residual replacement per request with the double-float
 *     FP64-class operators, as mm_pcg_solve on an MM_FP32_DF64 plan (the request's
 *     desc->precision is ignored).  A failed launch or copy ends the running requests with
 *     MM_ECUDA; the server goes on with the next ones.
 *   FP64-class requests (opts->precision MM_FP64): plain PCG with the plan's FP64-class operator in
 *     every iteration, in the arithmetic desc->precision selects (IEEE FP64 for MM_FP64 / MM_FP32,
 *     double-float for MM_DF64 / MM_FP32_DF64), one operator launch per request per step.
 */
/* Create a server (hbm_budget in bytes, 0 = 80% of the free device memory; max_slots >= 1). */
int mm_server_create(size_t hbm_budget, int max_slots, mm_server_t* out);
/* Queue a map-making solve.  desc and d are HOST memory (desc->inputs_on_device must be 0) and are
 * copied (by up to 8 threads) before the call returns; d is the TOD [N], float64 (d_is_fp32 = 0) or float32
 * (d_is_fp32 = 1).  opts->precision is MM_FP32 or MM_FP64 (above); opts->precond must be MM_PREC_BD;
 * MM_TPLZ_DIRECT plans are refused.  Non-blocking; *id identifies the request.  MM_EINVAL on bad
 * input (validated again at admission: a request that fails there finishes with that status). */
int mm_submit(mm_server_t server, const mm_problem_desc* desc, const void* d, int d_is_fp32,
              const mm_solve_opts* opts, mm_req_t* id);
/* MM_EBUSY while the request is queued or running; MM_OK (info filled) once it has finished. */
int mm_poll(mm_server_t server, mm_req_t id, mm_solve_info* info);
/* Wait up to timeout_us (< 0: forever) for the request, then copy its map into map_host
 * ([n_pix][3] float64 in global pixel order, 0 at unobserved or excised pixels; may be NULL) and
 * its info, and forget the request.  MM_ETIMEOUT if it did not finish in time (it keeps running);
 * otherwise the request's own status. */
int mm_wait(mm_server_t server, mm_req_t id, int64_t timeout_us, double* map_host, mm_solve_info* info);
/* Stop the server thread (running requests are abandoned) and free everything.  NULL is a no-op. */
void mm_server_destroy(mm_server_t server);

/* Message of the last failed call on this thread ("" if none). */
const char* mm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MM_H */
