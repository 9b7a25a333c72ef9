/*
 * asm.h -- C ABI of the GB300 sampler for the average spectrum method with
 * blocked modes sampling (K. Ghanem and E. Koch, "The Average Spectrum Method
 * for Analytic Continuation: Efficient Blocked Modes Sampling and Dependence on
 * Discretization Grid", arXiv:1912.01379).
 *
 * The library estimates the functional average of Eq. PI, discretised as
 * Eq. MCint: the mean of non-negative vectors fbar (fbar_n = A(omega_n) w_n,
 * Sec. V.B, Eq. Riemann) under the weight exp(-chi^2/2) of Eq. chi2, by Gibbs
 * moves along the right singular vectors of the whitened kernel restricted to
 * the blocks of a randomly chosen level (Sec. IV.B modes, IV.C blocked modes).
 *
 * Conventions for every call:
 *  - Return value: ASM_OK (0) or a negative ASM_ERR_* code; no exception or
 *    signal crosses this boundary.  asm_error_string() names the code.
 *  - Host arrays are plain C arrays owned by the caller; the library copies
 *    what it keeps during the call.  Matrices are row-major.
 *  - Device memory the caller passes (the workspace) stays owned by the caller
 *    and must stay allocated while the handle uses it.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  asm_sample is asynchronous on it; the result calls synchronise.
 *  - Handles are not thread-safe: one host thread at a time per handle.
 *  - All compute runs on the current CUDA device; there is no CPU fallback.
 */
#ifndef ASM_GB300_H
#define ASM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ASM_OK = 0,
    ASM_ERR_SHAPE = -1,      /* sizes or block partition inconsistent */
    ASM_ERR_NOT_SPD = -2,    /* covariance not symmetric positive definite */
    ASM_ERR_NONFINITE = -3,  /* NaN or Inf in an input */
    ASM_ERR_IMPROPER = -4,   /* a zero mode along which f >= 0 gives no bound */
    ASM_ERR_CUDA = -5,       /* a CUDA, cuBLAS or cuSOLVER call failed */
    ASM_ERR_STATE = -6,      /* call out of order (e.g. average before sample) */
    ASM_ERR_ARG = -7,        /* NULL or out-of-range argument */
    ASM_ERR_WORKSPACE = -8,  /* workspace missing, too small or misaligned */
    ASM_ERR_TOO_LARGE = -9,  /* a block or level exceeds a compiled limit */
    ASM_ERR_TIMEOUT = -10    /* a bounded device wait gave up; the run's results are invalid */
};

enum { ASM_FP64 = 0, ASM_MIXED = 1 };   /* precision of asm_sample */

/* asm_desc flags */
/* Test of the failure path (no counterpart in the paper): the record producer
 * of the sweep kernel withholds every move record and the consumers' bounded
 * waits give up after a few thousand polls instead of ~4M, so that a run ends
 * quickly with its timeouts counted and the result calls return
 * ASM_ERR_TIMEOUT; nothing is in flight when the kernel returns and the
 * context stays usable.  Never set in production. */
#define ASM_FLAG_TEST_STALL 0x80000000u

/* asm_sample flags */
#define ASM_SAMPLE_CONTINUE 1u   /* keep the chains of the previous call and go on */
#define ASM_SAMPLE_TIMING 2u     /* record CUDA events around every sweep-kernel launch */
#define ASM_SAMPLE_MOMENTS 4u    /* accumulate the snapshot moments asm_backward needs */
#define ASM_SAMPLE_REFRESH_FP64 8u  /* ASM_MIXED: refresh residuals on FP64 CUDA cores, not 3xTF32 tensor cores */
#define ASM_SAMPLE_STEP_TRACE 16u   /* record the step sizes of every sweep (asm_step_trace) */
#define ASM_SNAPSHOT_EVERY 8     /* kept sweeps between snapshots of all chains */

/* Environment variables the library reads (testing and tuning only; no result
 * depends on them, every chain does the same arithmetic under every launch
 * shape; values outside the ranges below are ignored):
 *   ASM_TEAM_LANES         8, 16 or 32: lanes per chain of a handle, read by
 *                          asm_setup (asm_tune replaces it);
 *   ASM_CONSUMERS_PER_CTA  1..7: chain warps per CTA of every sweep launch
 *                          (takes precedence over the heuristic and asm_tune);
 *   ASM_RING_DEPTH         2..48: stages of the move-record ring (default: as
 *                          many as shared memory holds, at most 48);
 *   ASM_RECORDS_PER_STAGE  1..8: consecutive move records per ring stage
 *                          (default 4: one barrier wait and release per stage);
 *   ASM_NO_U_STAGE         set: the block projections read U from global memory
 *                          instead of a shared-memory stage. */

typedef struct asm_problem asm_problem;  /* opaque, library-owned */

/* Problem description (Sec. II, Eq. likelihood and Eq. matrixeq; Sec. IV.C).
 *  M, N          number of data points (N_tau) and grid points (N_omega).
 *  K             M x N kernel acting on fbar: data mean = K fbar.
 *  G             M data (the mean gbar).
 *  C             M x M covariance of the data mean (symmetric positive definite).
 *  w             N Riemann weights (A = fbar / w); NULL means all ones.
 *  n_levels      number of partition levels (>= 1).
 *  level_nblocks blocks per level.
 *  block_start   concatenated start indices of the blocks of every level; each
 *                level starts at 0, starts increase, a block ends where the next
 *                one starts (the last one at N).  A level with one block is modes
 *                sampling; one-point blocks are components sampling.
 *  Kt, gt, d, V, U  optional given factors.  If all five are non-NULL, the
 *                library skips whitening and SVDs and uses them instead:
 *                Kt (M x N whitened kernel), gt (M whitened data) and, block
 *                after block in level order, d (n_b singular values, 0 marks a
 *                zero mode), V (n_b x n_b, mode-major: V[j*n_b+i] = component i
 *                of mode j) and U (min(M,n_b) x M, mode-major).  K, G, C are then
 *                unused unless C is also given, which the G-gradient of
 *                asm_backward needs.  This reproduces another implementation's modes.
 *  flags         0, or ASM_FLAG_TEST_STALL (tests of the failure path only).
 *  P, dK_dtheta, dw_dtheta  optional derivatives of the kernel and of the
 *                weights with respect to P grid-density (default-model)
 *                parameters; asm_backward then also returns the theta-gradient. */
typedef struct {
    int M, N;
    const double *K;
    const double *G;
    const double *C;
    const double *w;
    int n_levels;
    const int *level_nblocks;
    const int *block_start;
    const double *Kt, *gt, *d, *V, *U;
    uint32_t flags;
    int P;                      /* number of grid-density parameters theta (0: none) */
    const double *dK_dtheta;    /* P x M x N: dK/dtheta_p (row-major per p), or NULL */
    const double *dw_dtheta;    /* P x N: dw/dtheta_p, or NULL */
    /* Gamma prior prod_n fbar_n^(a_n - 1) (Eq. compat, Sec. V.C: sampling on this
     * grid what flat sampling on another grid gives; a_n = N rho(x_n) / (N' rho'(x_n))),
     * N values a_n >= 1, or NULL (flat).  Every move's draw from the fit's 1-D
     * conditional is then a proposal accepted with probability min(1, prior ratio)
     * (a Metropolis-Hastings step inside the Gibbs move, second uniform: word t mod 4
     * of ctr {t/4, s, q, problem xor 2^63}).  a_n < 1 is rejected (ASM_ERR_ARG): its
     * density diverges at 0 where clamped moves leave exact zeros. */
    const double *prior_shape;
} asm_desc;

/* Counters of the last asm_sample run (asm_status). */
typedef struct {
    int64_t chains, sweeps_done, kept_sweeps, precision;
    int64_t degenerate_moves;   /* interval of zero width: step 0 */
    int64_t zero_mode_moves;    /* flat draws along zero modes */
    int64_t tail_capped;        /* far-tail inverse-CDF solves that hit the cap */
    int64_t nonfinite_moves;    /* steps that came out NaN/Inf (then set to 0) */
    double max_resync_drift;    /* max |chi2_tracked - chi2_exact| / chi2_exact at refreshes */
    int64_t sweep_launches;     /* sweep-kernel launches since set-up of the chains */
    int64_t other_launches;     /* initial-state, refresh and reduction launches */
    int64_t timed_launches;     /* sweep launches timed with ASM_SAMPLE_TIMING */
    double sweep_kernel_ms;     /* summed event-timed duration of those launches */
    int64_t timeouts;           /* bounded device waits that gave up (0 in a valid run) */
    int64_t graph_replays;      /* refresh periods run as replays of the handle's CUDA graph */
    int64_t tc_refreshes;       /* residual refreshes run on the tensor cores (3xTF32) */
    int32_t team_lanes;         /* lanes per chain of the last sweep launch */
    int32_t consumers_per_cta;  /* chain warps per CTA of the last sweep launch */
    int32_t ctas;               /* CTAs of the last sweep launch (persistent) */
    int32_t work_items;         /* (problem, chain group) items of the last sweep launch */
    int32_t min_blocks;         /* CTAs per SM the last sweep launch's registers were budgeted for (1, 2) */
    int32_t reserved_;
    int64_t prior_rejections;   /* moves whose proposal the gamma prior rejected */
} asm_stats;

/* Set-up (Sec. IV: whitening C^{-1} = T^T T by Cholesky, K~ = T K, g~ = T G;
 * Sec. IV.B-C: SVD K~_b = U_b D_b V_b^T of every block of every level, in FP64
 * on the device).  Singular vectors get the sign that makes the largest
 * |component| of each V_j positive; d <= d_1 max(M,n_b) 2^-52 counts as a zero
 * mode, and so does d <= d_1 max(M,n_b) 2^-40 when V_j changes sign (below
 * that level U_j = K~ V_j / d_j is not resolvable in FP64 while the likelihood
 * is flat along V_j over its positivity interval).  On success *out receives a new handle (free with asm_destroy);
 * on failure *out is NULL and nothing stays allocated.  The environment variable
 * ASM_TEAM_LANES = 8, 16 or 32, read here, fixes the lanes per chain of the
 * handle's sweep launches (testing; other values are ignored, asm_tune overrides it). */
int asm_setup(const asm_desc *d, asm_problem **out);

/* Set-up of n independent problems as one batch handle (each problem as in
 * asm_setup; n >= 1, d points to n descriptors).  asm_sample on it runs every
 * problem's chains in the same persistent launches (work items = (problem,
 * chain group), costliest problems first); problem k keys its random numbers
 * with problem id P + k, P the handle's problem id (asm_set_stream_ids,
 * default 0), so problem k of a batch gives exactly what a single handle of
 * that problem gives with problem id P + k.  Results per problem:
 * asm_average_at.  Backward moments, chain states and checkpoints are for
 * single problems (ASM_ERR_ARG on a batch).  On failure nothing is kept. */
int asm_setup_batch(int n, const asm_desc *d, asm_problem **out);

/* Partition hierarchy of blocked modes sampling (Sec. IV.C and Fig. blocks):
 * level 0 is the whole grid (modes sampling); level l >= 1 splits the N grid
 * points into blocks of nominal width w_l = N / 2^l, boundaries at
 * round(k w_l + s_l) with s_l = w_l / 2 on even levels l >= 2 and 0 on odd
 * ones (the shift keeps every other level from having a boundary at the centre
 * of the grid); the last level has one point per block (components sampling).
 * Levels equal to the one above are left out.  Out: *n_levels (at most 33),
 * level_nblocks[l] (capacity 33), *total_blocks and, unless block_start is NULL,
 * the concatenated block starts of every level (capacity *total_blocks, so a
 * first call with block_start = NULL gives the size).  The result is a valid
 * asm_desc partition.  Host only; ASM_ERR_ARG for N < 1 or NULL outputs. */
int asm_partition_hierarchy(int N, int *n_levels, int *level_nblocks, int *block_start, int *total_blocks);

/* Number of problems of a handle (1 for asm_setup). */
int asm_problem_count(const asm_problem *p);

/* Autotuner of the sweep launch (no counterpart in the paper).  Times every
 * candidate shape -- lanes per chain S in {32, 16, 8} times chain warps per
 * CTA in {heuristic, 2, 3, 4, 5, 6, 7} times the register budget (kernels
 * compiled for one CTA per SM, up to 255 registers per thread, or for two,
 * 128), where it fits -- on one warm-up and three
 * timed sweeps of fresh trial chains in the caller's workspace (same layout
 * and size rule as asm_sample), and keeps the fastest for later asm_sample
 * calls on p.  The shape changes no result: every chain does the same
 * arithmetic in the same order under every shape.  The workspace's contents
 * are overwritten, so the next asm_sample must start fresh chains
 * (ASM_SAMPLE_CONTINUE then fails with ASM_ERR_STATE).  Synchronises
 * `stream`.  team_out / consumers_out / min_blocks_out (may be NULL) receive
 * the choice (consumers 0 = the built-in heuristic; min_blocks 1 or 2). */
int asm_tune(asm_problem *p, int chains, int precision, void *d_workspace, size_t workspace_bytes,
             void *stream, int *team_out, int *consumers_out, int *min_blocks_out);

/* Bytes of device workspace asm_sample needs for `chains` chains (per problem)
 * at `precision` (ASM_FP64 or ASM_MIXED); 0 for invalid arguments. */
size_t asm_workspace_bytes(const asm_problem *p, int chains, int precision);

/* Run burn_in + sweeps sweeps of `chains` independent chains (Sec. IV.C: every
 * sweep draws one level at random and moves every mode of every block of it
 * once, blocks left to right, modes in index order).  Each move draws the step
 * along its mode from the exact 1-D conditional, a Gaussian truncated to the
 * interval of Eq. modeLimits (flat for zero modes), by the inverse CDF of one
 * Philox4x64-10 uniform keyed by (seed, problem id, global chain id, sweep,
 * move); see asm_set_stream_ids.
 * Sweeps after burn-in are accumulated into FP64 sums of fbar and fbar^2.
 * precision: ASM_FP64 runs the chain state in FP64 with an FP64 residual
 * refresh every 64 sweeps; ASM_MIXED runs it in FP32 with FP64 accumulators and
 * refreshes r~ = g~ - K~ f every 64 sweeps as one tensor-core GEMM over all
 * chains in split precision (3xTF32: f_hi K_hi + f_hi K_lo + f_lo K_hi, FP32
 * accumulation; error ~2^-21 |K~||f| per term), the difference, chi^2 and the
 * drift in FP64 (ASM_SAMPLE_REFRESH_FP64: on FP64 CUDA cores instead).
 * flags: ASM_SAMPLE_CONTINUE continues the chains of the previous call on the
 * same workspace (same chains, seed and precision) without resetting the sums;
 * otherwise chains start from the flat default-model scale fit.
 * ASM_SAMPLE_TIMING records a CUDA event pair on `stream` around every sweep
 * launch; asm_status reports their summed duration.  Any other flag bit:
 * ASM_ERR_ARG.
 * Launches: one persistent sweep kernel per refresh period (64 sweeps) over
 * every (problem, chain group) work item, then the FP64 residual refresh.
 * Runs of whole periods replay a CUDA graph of (advance the sweep range,
 * sweep, refresh), instantiated on the first such call and kept in the handle
 * until the workspace, chain count, precision or launch shape changes; not
 * with ASM_SAMPLE_TIMING, ASM_SAMPLE_MOMENTS, or while `stream` is being
 * captured (then each launch is issued directly). 
 * d_workspace: device pointer, 256-byte aligned, >= asm_workspace_bytes(). */
int asm_sample(asm_problem *p, int chains, long burn_in, long sweeps, uint64_t seed,
               int precision, uint32_t flags, void *d_workspace, size_t workspace_bytes,
               void *stream);

/* Results of the last asm_sample (synchronises; ASM_ERR_TIMEOUT if a bounded
 * device wait of that run gave up).  Per grid point (N values,
 * any pointer may be NULL): mean_A = <fbar>/w, sem_A its standard error from
 * the spread of the independent chain means, ess = posterior variance of fbar
 * over sem^2, mean_fbar = <fbar>. */
int asm_average(asm_problem *p, double *mean_A, double *sem_A, double *ess, double *mean_fbar);

/* Vector-Jacobian products of <A> = <fbar>/w (synchronises; needs a run with
 * ASM_SAMPLE_MOMENTS).  With v (N) the cotangent of <A>:
 *  grad_G (M)      = v^T d<A>/dG = C^{-1} K Cov(fbar, fbar) (v/w): the derivative of
 *                    the posterior mean under exp(-chi^2/2) (Eq. likelihood) is the
 *                    posterior covariance with the gradient of -chi^2/2, which is
 *                    C^{-1}(K fbar - G), linear in fbar.
 *  grad_theta (P)  = Cov((v/w)^T fbar, s_p) - sum_n v_n <fbar_n> dw_n/dtheta_p / w_n^2,
 *                    s_p = (G - K fbar)^T C^{-1} (dK/dtheta_p) fbar (the flat measure on
 *                    fbar does not depend on theta).
 * Moments come from snapshots of all chains every ASM_SNAPSHOT_EVERY kept sweeps.
 * grad_G needs the covariance C (computed or given at set-up); grad_theta needs
 * P > 0; either pointer may be NULL. */
int asm_backward(asm_problem *p, const double *v, double *grad_G, double *grad_theta);

/* asm_average for problem k of a handle (k = 0 for a single problem). */
int asm_average_at(asm_problem *p, int k, double *mean_A, double *sem_A, double *ess, double *mean_fbar);

/* Monte Carlo error of <fbar> for problem k of a handle (synchronises), by
 * binning (Flyvbjerg and Petersen 1989; not in the paper): the kept sweeps of
 * every chain are cut into bins of 64 sweeps aligned to multiples of 64 in the
 * absolute sweep index (only bins wholly after the burn-in count), merged
 * pairwise over 8 levels (bins of 64 ... 8192 sweeps); at level l the squared
 * error of the grand mean is the variance of all chains' level-l bin means
 * over their number.  sem_fbar^2 (N) = the largest of these over the levels
 * with at least two bins per chain and of the squared spread of the chain
 * means (asm_average's error); ess (N) = posterior variance / sem_fbar^2.
 * A drift that all chains share (a common start not yet forgotten) raises the
 * binned error although it hides from the chain spread.  Optional outputs:
 * sigma2_levels (8 x N, NaN where a level has fewer than two bins in all) and
 * bins_per_chain (8).  Any argument but p may be NULL.  ASM_ERR_STATE before a
 * run with kept sweeps. */
int asm_mc_error(asm_problem *p, int k, double *ess, double *sem_fbar, double *sigma2_levels, int *bins_per_chain);

/* Current chain states (synchronises): f (chains x N, FP64 copy of fbar) and
 * chi2 (chains) = |r~|^2 of the residual the sampler tracks; either may be NULL. */
int asm_chain_state(asm_problem *p, double *f, double *chi2);

/* Counters of the last asm_sample (synchronises). */
int asm_status(asm_problem *p, asm_stats *out);

/* Allocation-free sampling.  The paper has no counterpart: this call exists
 * for callers that cannot allocate device memory themselves.  Examples: a
 * plug-in inside a host application that owns every byte of device memory
 * through its own pool (a cudaMalloc behind the pool's back breaks its
 * accounting and fails once the pool holds the memory), and service loops
 * that run under a fixed memory budget set at start-up, where an allocation
 * in the loop may fail, block or synchronise the device at an unpredictable
 * moment.
 * It runs the same sampling as asm_sample (fresh chains, burn_in + sweeps
 * sweeps; the mixed path always refreshes its residuals on the tensor cores)
 * and then the device part of asm_average, but its scratch (chain states,
 * residuals, sums and counters) lives in one library-owned static device
 * array of ASM_NOALLOC_SCRATCH_BYTES (64 MiB), which every GPU that loads the
 * library keeps until the process exits.  The call allocates and frees
 * nothing; a run whose asm_workspace_bytes(p, chains, precision) exceeds the
 * array is rejected with ASM_ERR_TOO_LARGE before any GPU work.
 * Outputs (caller-owned device buffers of N doubles, written asynchronously on
 * `stream`): d_mean_fbar = <fbar>, d_sem2_fbar = squared standard error of
 * <fbar> from the spread of the chain means, d_m2_fbar = <fbar^2>.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  Every call
 * shares the array and re-initialises what must start at zero, and the array
 * keeps the last call's contents: calls whose GPU work overlaps (other
 * streams, threads or handles on the same device) race on it and must be
 * serialised by the caller.  Until the next sampling call, asm_chain_state,
 * asm_status, asm_mc_error and asm_checkpoint of the handle read the array. */
#define ASM_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int asm_sample_noalloc(asm_problem *p, int chains, long burn_in, long sweeps, uint64_t seed,
                       int precision, double *d_mean_fbar, double *d_sem2_fbar, double *d_m2_fbar,
                       void *stream);

/* Measured arithmetic ceilings (no counterpart in the paper: the denominators
 * of the chain kernel's roofline).  Runs the chosen instruction mix on
 * register operands (the _SMEM kinds: V and R from shared memory as 16-byte
 * vectors, as the chain kernel reads them) on every SM at full occupancy with
 * eight independent streams per thread, growing the loop until one launch
 * takes about target_ms (0 < target_ms <= 2000), and returns the rate.
 *   ASM_CEIL_PASS_F32/_F64: elements per second of the fused pass of a move
 *     (Sec. IV.B): the update f + delta V (FMA), the clamp at 0 (max), the
 *     bound product x R (multiply) and the signed and unsigned integer minima
 *     of its bits (the two bound keys).
 *   ASM_CEIL_FFMA, _FMNMX, _IMNMX, _DFMA, _DMNMX, _I64MNMX: instructions per
 *     second of one operation alone (min/max kinds: of each minimum).
 * *sm_mhz (may be NULL) receives the SM clock during the launch, from
 * clock64() against the global timer; *ms (may be NULL) the launch time.
 * Allocates a few bytes of device memory and one stream, synchronises.
 * Returns ASM_ERR_ARG for an unknown kind or target. */
enum {
    ASM_CEIL_PASS_F32 = 0, ASM_CEIL_PASS_F32_SMEM = 1, ASM_CEIL_FFMA = 2, ASM_CEIL_FMNMX = 3,
    ASM_CEIL_IMNMX = 4, ASM_CEIL_PASS_F64 = 5, ASM_CEIL_PASS_F64_SMEM = 6, ASM_CEIL_DFMA = 7,
    ASM_CEIL_DMNMX = 8, ASM_CEIL_I64MNMX = 9, ASM_CEIL_KINDS = 10
};
int asm_measure_ceiling(int kind, double target_ms, double *ops_per_s, double *sm_mhz, double *ms);

/* Step sizes of the sampler (Sec. IV.D, Fig. MCsteps): delta[s] = the mean over
 * the chains of problem k of Delta_s = |f(s+1) - f(s)| / |f(s)|, f(s) the
 * chain's state before sweep s counted from the start of its chains, for the
 * first min(sweeps done, 4096, max_sweeps) sweeps; *n_sweeps receives that
 * count.  Recorded by every asm_sample that carries ASM_SAMPLE_STEP_TRACE
 * (sweeps run without the flag leave their entries at 0; the norms are summed
 * in the chain state's precision).  Synchronises.  The trace shows how far one
 * Monte Carlo step moves the model, the paper's measure of the efficiency of
 * components, modes and blocked modes sampling. */
int asm_step_trace(asm_problem *p, int k, double *delta, int max_sweeps, int *n_sweeps);

/* Identities that key the random numbers (Philox counter words): problem_id
 * (default 0) and the global id of local chain 0 (default 0).  Chains are
 * independent and keyed by their global id, so shards of one run placed on
 * several GPUs with chain_offset = first global chain of the shard reproduce
 * the unsharded run chain by chain (multi-GPU replicas: each GPU samples its
 * shard; the FP64 sums are added on the host).  Takes effect at the next
 * asm_sample that starts fresh chains. */
int asm_set_stream_ids(asm_problem *p, uint64_t problem_id, uint64_t chain_offset);

/* Checkpoint of the run state (synchronises): chain states, tracked residuals,
 * sums, bins of the Monte Carlo error, counters, the sweep count and the start
 * of the kept run, so that a restored run continues bit for bit (averages and
 * binned errors alike).  host_buf NULL: *bytes receives the size needed.
 * Otherwise *bytes is the buffer size on input and the bytes written on
 * output.  The blob is versioned; asm_restore accepts only the version this
 * library writes (ASM_ERR_ARG otherwise). */
int asm_checkpoint(asm_problem *p, void *host_buf, size_t *bytes);

/* Restore a checkpoint into d_workspace (>= asm_workspace_bytes for the
 * checkpoint's chains and precision) of a handle set up for the same problem;
 * the next asm_sample with ASM_SAMPLE_CONTINUE (same chains, seed, precision,
 * workspace) continues the run.  Synchronises `stream`. */
int asm_restore(asm_problem *p, const void *host_buf, size_t bytes, void *d_workspace,
                size_t workspace_bytes, void *stream);

/* Free the handle and its device memory (not the caller's workspace). */
void asm_destroy(asm_problem *p);

/* Static string naming an ASM_* code. */
const char *asm_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif
