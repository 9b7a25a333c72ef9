// asm_internal.h -- types shared by the host library and the sweep kernels.
// Not part of the public ABI (include/asm.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace asmgb {

// Rows of every block's mode data are padded to a multiple of this many
// elements so that any team size S <= 32 with 16-byte vectors stays in the row.
constexpr int kRowAlign = 128;
// Residual refresh period of the sweep loop (sweeps).
constexpr int kRefreshPeriod = 64;

// One block of one level, as the device sees it.  Offsets are in elements of
// the precision-specific arrays.
struct BlockDesc {
    int start;       // first grid point of the block
    int n;           // block width n_b
    int np;          // modes with a U column: min(M, n_b)
    int rs;          // row stride of V/R rows (multiple of kRowAlign)
    long long offV;  // V: n rows
    long long offR;  // R = -1/V (NaN where V is left out): n + 1 rows, the last all-NaN
    long long offd;  // d, invd: n values
    long long offU;  // Ut: np x M (mode-major); Um: M x np (grid-major)
    long long offRec;  // move records of the block: n records of recstride elements
    int recstride;     // elements per record (2 rs + 16)
    int usr;           // row stride of the staging copy of U (odd: conflict-free column reads)
    long long offUs;   // staging copy of U: np rows of usr elements, 16-byte aligned
};

// Device-side problem data in one precision T.
template <class T>
struct ProblemData {
    const T *V, *R;          // mode rows V and R = -1/V (NaN where V is left out of the bounds)
    const T *d, *invd;       // singular values and their reciprocals (0 for zero modes)
    const T *meta;           // per mode, 16 bytes: {d, 1/d} (FP32: {d, 1/d, 0, 0})
    const T *rec;            // per move j: {V_j, R_{j+1} (rs each), d_j, 1/d_j, |K~_b V_j|}
    const T *Ut, *Um;        // U in two layouts
    const T *Us;             // U mode-major with odd row stride, copied to shared memory per block visit
};

struct Counters {            // device counters, first bytes of the workspace
    unsigned long long degenerate, zero_mode, tail_capped, nonfinite;
    unsigned long long drift_bits;   // max relative chi2 drift, as ordered bits of a double
    unsigned long long timeouts;     // bounded waits that gave up (the launch then stopped early)
    unsigned long long prior_rejections;   // proposals the gamma prior rejected
    unsigned long long pad;
};

template <class T>
struct SweepParams {
    int M, N;
    int n_levels;
    const int *level_first;           // first block index of each level
    const int *level_nblocks;
    const BlockDesc *blocks;
    ProblemData<T> pd;
    T *F; int ldF;                    // chain states, chains x ldF
    T *R; int ldR;                    // tracked residuals, chains x ldR
    double *S1, *S2;                  // sums of f and f^2, chains x N
    // binning of the Monte Carlo error (every kBinSweeps sweeps): S1 at the last bin
    // boundary (chains x N), per chain and level the pending half of a bin pair and the
    // sums of the bin means and their squares (chains x kBinLevels x N), level-0 bins per chain
    double *S1p, *bpend, *bacc1, *bacc2;
    int *bcount;
    int chains;
    unsigned long long seed, problem_id;
    unsigned long long chain_offset;  // global id of local chain 0 (Philox key word)
    Counters *counters;
    // residual refresh / initial state of this problem (FP64)
    const double *KtT, *gt;           // whitened kernel (N x M) and data
    double *chi2;                     // chains
    double f0;                        // starting value of every fbar_n
    // whitened kernel split into TF32 high and low parts (M x ldK FP32 each) for
    // the tensor-core refresh of the mixed path
    const float *Khi, *Klo;
    int ldK;
    // reference state of the tensor-core refresh: the mean chain state fref (N,
    // FP32) and r_ref = g~ - K~ fref (M, FP64); the product is taken of f - fref
    float *fref;
    double *rref;
    // k-split of the tensor-core refresh: the grid points are cut into ksplit parts
    // whose FP32 partial products (ksplit x chains x ldR) are added in FP64 in part
    // order by the finishing kernel; ksplit = 1: no partials (nullptr)
    float *Dpart;
    int ksplit;
    // gamma prior: a_n - 1 per grid point (nullptr: flat)
    const T *prior_am1;
    // step-size trace (nullptr: off): sum over chains of |f(s+1) - f(s)| / |f(s)| for
    // the absolute sweeps s < trace_cap
    double *steptrace;
    int trace_cap;
    // FP32 chain state: the sums of f and f^2 over one launch's kept sweeps (FP32,
    // chains x ldF) where shared memory cannot hold them; added to S1, S2 per launch
    float *P1, *P2;
};

// What every problem of one launch shares: the CTA shape and the
// shared-memory plan (the union of the problems' needs).  The move records
// of a CTA's item flow through a ring of `depth` stages filled by one
// producer warp with bulk copies (TMA engine); `full` barriers signal a
// landed record, `empty` barriers collect the consumer warps' releases.
struct LaunchShape {
    int S;                            // lanes per chain (power of two, <= 32)
    int consumers;                    // consumer warps per CTA (the producer is one more)
    int depth;                        // stages in the ring
    int off_full, off_empty, off_stages;  // byte offsets in dynamic shared memory
    int stage_bytes;                  // bytes per stage (>= rps of the largest records)
    int rps;                          // move records per stage (consecutive moves of one block)
    int cpad;                         // shared-memory stride of the c/w buffers (>= max np)
    int mpad;                         // shared-memory stride of the residual (>= max M)
    int npad;                         // shared-memory sums of the kept sweeps per team (>= max N;
                                      // 0: the kept sweeps are added to the FP64 sums directly)
    int team_words;                   // shared-memory elements per team: 2 cpad + mpad + 8 S + 2 npad
    int n_items;                      // (problem, chain group) work items
    int minb;                         // register budget: 1 or 2 CTAs per SM
    int prior;                        // 1: kernels with the gamma prior's acceptance step
    int wait_limit;                   // polls before a bounded mbarrier wait gives up
    int stall;                        // test of the failure path: the producer issues no records
    // U of the visited block in shared memory (two stages filled by the producer with
    // one bulk copy per block visit; 0: the projections read U from global memory)
    int ubytes;                       // bytes per stage (blocks whose U is larger read global memory)
    int off_ubuf;                     // byte offset of the two stages
    int off_ubar;                     // byte offset of their full[2] and empty[2] barriers
};

// Per-launch control block in device memory: the work queue and the launch's
// sweep range.  Kept on the device so that one refresh period (advance the
// range, sweep, refresh) is a fixed sequence that a CUDA graph can replay.
struct RunCtrl {
    int queue;                        // next work item
    int pad_;
    long long sweep0, nsweeps;        // sweeps [sweep0, sweep0 + nsweeps)
    long long burn_in;                // absolute sweep index where accumulation starts
};

// A work item: problem index and chain group (consumers x 32/S chains).
struct WorkItem {
    int problem, group;
};

// Launchers (asm_sweep_{f32,f64}{,_m2}.cu).  kv: 16-byte vectors per lane.
// Persistent: `ctas` CTAs of (consumers + 1) warps pull work items from
// ctrl->queue (reset to 0 before the launch).  One problem (batch = false):
// its parameters p0 travel by value in the launch; several (batch = true):
// work item problems index the device array probs.  _m1 kernels budget the
// registers for one CTA per SM (up to 255 per thread), _m2 for two (128).
#define ASM_DECLARE_SWEEP_LAUNCHER(T, NAME)                                                                   \
    cudaError_t launch_sweeps_##NAME(const SweepParams<T> &p0, const SweepParams<T> *probs, const WorkItem *items, \
                                     RunCtrl *ctrl, const LaunchShape &shape, int kv, bool batch, int ctas,     \
                                     cudaStream_t s);                                                          \
    int sweep_ctas_per_sm_##NAME(const LaunchShape &shape, int kv, bool batch);
ASM_DECLARE_SWEEP_LAUNCHER(float, f32_m1)
ASM_DECLARE_SWEEP_LAUNCHER(float, f32_m2)
ASM_DECLARE_SWEEP_LAUNCHER(double, f64_m1)
ASM_DECLARE_SWEEP_LAUNCHER(double, f64_m2)
ASM_DECLARE_SWEEP_LAUNCHER(float, f32_prior)     // with the gamma prior, one CTA per SM
ASM_DECLARE_SWEEP_LAUNCHER(double, f64_prior)
#undef ASM_DECLARE_SWEEP_LAUNCHER
// Tensor-core residual refresh of the mixed path (asm_refresh_tc.cu): grid of
// (chain tiles of 128) x n_problems x (the largest k split) CTAs; max_bn = the
// largest refresh_tc_bn(M).
cudaError_t launch_refresh_tc(const SweepParams<float> *probs, int n_problems, int chains, int max_bn, int max_parts,
                              bool track_drift, cudaStream_t s);
int refresh_tc_bn(int M);                  // MMA N of a problem's M_tau tiles
int refresh_tc_ksplit(int chains, int N);  // parts of a problem's k range (a function of the problem)
// The FP64 combination of the k parts (problems with ksplit > 1): r~, chi^2, drift.
cudaError_t launch_refresh_finish(const SweepParams<float> *probs, int n_problems, int chains, bool track_drift,
                                  cudaStream_t s);
size_t refresh_tc_smem(int max_bn);        // dynamic shared memory of one CTA
constexpr int kRefreshTcLdK = 32;          // ldK is a multiple of this (one k-tile)
cudaError_t launch_split_k(const double *KtT, int M, int N, int ldK, float *Khi, float *Klo, cudaStream_t s);
// Reference state of every problem's tensor-core refresh: fref over tiles of 32
// grid points, then r_ref over tiles of 128 data points (two launches).
cudaError_t launch_refresh_ref(const SweepParams<float> *probs, int n_problems, int chains, int max_N, int max_M,
                               cudaStream_t s);
// Contractions of the backward pass (asm_moments.cu).  D: chains x ldD snapshot
// (centred); Sff (N x N, FP64) += D^T D; Y (chains x PM) = D Kth^T with Kth
// PM x N row-major (the whitened dK/dtheta of all parameters); Sq (chains x P)
// = the scores r~_q . (Y_q,p + kshift_p); y = L^{-T} K~ u for the G-product.
cudaError_t launch_gram(const float *D, int ldD, int chains, int N, double *Sff, cudaStream_t s);
cudaError_t launch_gram(const double *D, int ldD, int chains, int N, double *Sff, cudaStream_t s);
cudaError_t launch_kth_product(const float *D, int ldD, int chains, int N, const float *Kth, int PM, float *Y,
                               cudaStream_t s);
cudaError_t launch_kth_product(const double *D, int ldD, int chains, int N, const double *Kth, int PM, double *Y,
                               cudaStream_t s);
cudaError_t launch_scores(const float *R, int ldR, const float *Y, const double *kshift, int M, int chains, int P,
                          double *Sq, cudaStream_t s);
cudaError_t launch_scores(const double *R, int ldR, const double *Y, const double *kshift, int M, int chains, int P,
                          double *Sq, cudaStream_t s);
cudaError_t launch_vjp_G(const double *KtT, const double *L, const double *u, int M, int N, double *y,
                         cudaStream_t s);
// CTAs of the persistent kernel that fit one SM at this shape (shared memory included).
int sweep_ctas_per_sm_f32(const LaunchShape &shape, int kv, bool batch);
int sweep_ctas_per_sm_f64(const LaunchShape &shape, int kv, bool batch);
// Largest supported kv per precision.
// Polls of a bounded mbarrier wait before it gives up (each poll may suspend
// the thread briefly); a run that gives up counts a timeout and its results
// are reported as ASM_ERR_TIMEOUT.
constexpr int kWaitLimit = 1 << 22;
// Binning: bins of kBinSweeps kept sweeps aligned to multiples of kBinSweeps in
// the absolute sweep index (the refresh period), merged pairwise over kBinLevels
// levels (bins of 64 ... 8192 sweeps).
constexpr int kBinSweeps = 64;
constexpr int kBinLevels = 8;
// Sweeps from the chains' start whose step size the trace records.
constexpr int kStepTraceMax = 4096;
// Consumer warps per CTA: at most 7, so that a CTA (consumers + the producer)
// has at most 8 warps, two per SM sub-partition, and a thread may hold up to
// 255 registers (9 warps would put three on one sub-partition: 168).
constexpr int kMaxConsumers = 7;
// Deepest ring of move records (stages) a launch may use.
constexpr int kMaxRingDepth = 48;
// Move records per ring stage (one barrier wait and one release per stage).
constexpr int kRecordsPerStage = 4;
constexpr int kMaxKvF32 = 16;   // 64 floats per lane
constexpr int kMaxKvF64 = 32;   // 64 doubles per lane

}  // namespace asmgb
