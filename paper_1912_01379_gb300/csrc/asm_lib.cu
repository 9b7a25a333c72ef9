// asm_lib.cu -- C ABI (include/asm.h) of the GB300 average-spectrum sampler:
// set-up (whitening and block SVDs in FP64 on the device), the sweep loop with
// the periodic FP64 residual refresh, and the result reductions.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/asm.h"
#include "asm_internal.h"

using namespace asmgb;

namespace {

// ---------------------------------------------------------------------------
// small device kernels: initial state, residual refresh, result reduction
// ---------------------------------------------------------------------------
template <class T>
__global__ void init_kernel(T *F, int ldF, int N, double f0, double *S1, double *S2, int chains)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)chains * ldF;
    if (i < tot) {
        const int n = (int)(i % ldF);
        F[i] = n < N ? (T)f0 : T(0);
    }
    if (i < (long long)chains * N) {
        S1[i] = 0.0;
        S2[i] = 0.0;
    }
}

// r~ = g~ - K~ f in FP64 for every chain (one CTA per chain); chi2 = |r~|^2.
// Records the largest relative change of chi2 against the tracked residual.
template <class T>
__global__ void refresh_kernel(int M, int N, const double *__restrict__ KtT, const double *__restrict__ gt,
                               const T *__restrict__ F, int ldF, T *R, int ldR, double *chi2,
                               Counters *cnt, int track_drift)
{
    extern __shared__ double fs[];
    __shared__ double red_old[32], red_new[32];
    const int q = blockIdx.x;
    for (int n = threadIdx.x; n < N; n += blockDim.x) fs[n] = (double)F[(size_t)q * ldF + n];
    __syncthreads();
    double so = 0.0, sn = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        double a = gt[m];
        for (int n = 0; n < N; ++n) a -= KtT[(size_t)n * M + m] * fs[n];
        const double old = (double)R[(size_t)q * ldR + m];
        so += old * old;
        sn += a * a;
        R[(size_t)q * ldR + m] = (T)a;
    }
    for (int off = 16; off; off >>= 1) {
        so += __shfl_xor_sync(0xffffffffu, so, off);
        sn += __shfl_xor_sync(0xffffffffu, sn, off);
    }
    if ((threadIdx.x & 31) == 0) {
        red_old[threadIdx.x >> 5] = so;
        red_new[threadIdx.x >> 5] = sn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red_old[w]; b += red_new[w]; }
        if (chi2) chi2[q] = b;
        if (track_drift) {
            const double drift = fabs(a - b) / fmax(b, 1e-300);
            atomicMax(&cnt->drift_bits, (unsigned long long)__double_as_longlong(drift));
        }
    }
}

// The same refresh for every chain of every problem of a launch: CTA b handles
// chain b % chains of problem b / chains (parameters from the launch's table).
template <class T>
__global__ void refresh_all_kernel(const SweepParams<T> *__restrict__ probs, int chains, int track_drift)
{
    extern __shared__ double fs[];
    __shared__ double red_old[32], red_new[32];
    const SweepParams<T> &p = probs[blockIdx.x / chains];
    const int q = blockIdx.x % chains;
    const int M = p.M, N = p.N;
    for (int n = threadIdx.x; n < N; n += blockDim.x) fs[n] = (double)p.F[(size_t)q * p.ldF + n];
    __syncthreads();
    double so = 0.0, sn = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        double a = p.gt[m];
        for (int n = 0; n < N; ++n) a -= p.KtT[(size_t)n * M + m] * fs[n];
        const double old = (double)p.R[(size_t)q * p.ldR + m];
        so += old * old;
        sn += a * a;
        p.R[(size_t)q * p.ldR + m] = (T)a;
    }
    for (int off = 16; off; off >>= 1) {
        so += __shfl_xor_sync(0xffffffffu, so, off);
        sn += __shfl_xor_sync(0xffffffffu, sn, off);
    }
    if ((threadIdx.x & 31) == 0) {
        red_old[threadIdx.x >> 5] = so;
        red_new[threadIdx.x >> 5] = sn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red_old[w]; b += red_new[w]; }
        p.chi2[q] = b;
        if (track_drift) {
            const double drift = fabs(a - b) / fmax(b, 1e-300);
            atomicMax(&p.counters->drift_bits, (unsigned long long)__double_as_longlong(drift));
        }
    }
}

// Sets the launch's sweep range (advance = 0) or moves it on by its length
// (advance = 1), and resets the work queue.
__global__ void ctrl_kernel(RunCtrl *c, long long sweep0, long long nsweeps, long long burn_in, int advance)
{
    c->queue = 0;
    if (advance) {
        c->sweep0 += c->nsweeps;
    } else {
        c->sweep0 = sweep0;
        c->nsweeps = nsweeps;
        c->burn_in = burn_in;
    }
}

// Binning at a bin boundary (the end of a launch whose range ends at a multiple
// of kBinSweeps): CTA b handles chain b % chains of problem b / chains.  The sum
// of the last kBinSweeps sweeps is S1 - S1p; if the bin lies wholly after the
// burn-in its mean enters level 0, and pairs of level-k bin means merge into a
// level-(k+1) bin (level-k bin c, counted from 1, is the first of a pair when c
// is odd).  Sums of the bin means and their squares per level and grid point.
template <class T>
__global__ void bin_kernel(const SweepParams<T> *__restrict__ probs, int chains, const RunCtrl *ctrl)
{
    __shared__ int s_nb;
    const SweepParams<T> &p = probs[blockIdx.x / chains];
    const int q = blockIdx.x % chains;
    const long long s_end = ctrl->sweep0 + ctrl->nsweeps;
    const bool complete = s_end % kBinSweeps == 0 && s_end - kBinSweeps >= ctrl->burn_in;
    if (threadIdx.x == 0) s_nb = p.bcount[q] + (complete ? 1 : 0);
    __syncthreads();
    const int nb = s_nb;
    const int N = p.N;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const size_t i = (size_t)q * N + n;
        const double s1 = p.S1[i];
        double x = (s1 - p.S1p[i]) * (1.0 / kBinSweeps);
        p.S1p[i] = s1;
        if (!complete) continue;
        for (int k = 0; k < kBinLevels; ++k) {
            const size_t j = ((size_t)q * kBinLevels + k) * N + n;
            p.bacc1[j] += x;
            p.bacc2[j] += x * x;
            if (k + 1 == kBinLevels || ((nb >> k) & 1)) {
                if ((nb >> k) & 1) p.bpend[j] = x;
                break;
            }
            x = 0.5 * (p.bpend[j] + x);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && complete) p.bcount[q] = nb;
}

// Sums over chains, in chain order, of the binning sums of one problem:
// out[0][k][n] = sum of bin means, out[1][k][n] = sum of their squares.
__global__ void bin_reduce_kernel(const double *__restrict__ acc1, const double *__restrict__ acc2, int chains,
                                  int N, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // k * N + n
    if (i >= kBinLevels * N) return;
    double a = 0.0, b = 0.0;
    for (int q = 0; q < chains; ++q) {
        a += acc1[(size_t)q * kBinLevels * N + i];
        b += acc2[(size_t)q * kBinLevels * N + i];
    }
    out[i] = a;
    out[(size_t)kBinLevels * N + i] = b;
}

// FP32 state: the sums of the open 64-sweep block added to the FP64 sums now
// and cleared.  Used when a continuation starts a new burn-in: the kept run is
// broken, and the block's earlier kept sweeps must be in S1 before the next bin
// boundary, where the binning takes S1's growth over the bin as the bin's sum.
__global__ void fold_open_block_kernel(float *P1, float *P2, int ldP, double *S1, double *S2, int chains, int N)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)chains * N) return;
    const long long q = i / N, n = i % N;
    S1[i] += (double)P1[q * ldP + n];
    S2[i] += (double)P2[q * ldP + n];
    P1[q * ldP + n] = 0.f;
    P2[q * ldP + n] = 0.f;
}

// Per grid point: mean over chains and kept sweeps, the spread of the chain
// means (two passes) and the second moment.  P1, P2 (FP32 chain state; else
// null): the kept-sweep sums of a 64-sweep block still open, added here.
__global__ void reduce_kernel(const double *S1, const double *S2, const float *P1, const float *P2, int ldP,
                              int chains, int N, double kept, double *mean, double *semsq, double *m2)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    auto s1 = [&](int q) { return S1[(size_t)q * N + n] + (P1 ? (double)P1[(size_t)q * ldP + n] : 0.0); };
    double a = 0.0, b = 0.0;
    for (int q = 0; q < chains; ++q) {
        a += s1(q);
        b += S2[(size_t)q * N + n] + (P2 ? (double)P2[(size_t)q * ldP + n] : 0.0);
    }
    const double mu = a / (chains * kept);
    double v = 0.0;
    for (int q = 0; q < chains; ++q) {
        const double d = s1(q) / kept - mu;
        v += d * d;
    }
    mean[n] = mu;
    semsq[n] = chains > 1 ? v / ((double)(chains - 1) * chains) : NAN;
    m2[n] = b / (chains * kept);
}

// ---------------------------------------------------------------------------
// snapshot moments for the backward pass
// ---------------------------------------------------------------------------
// Sf[n] += sum over chains of f[q][n]
template <class T>
__global__ void colsum_kernel(const T *F, int ldF, int chains, int N, double *Sf)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double a = 0.0;
    for (int q = 0; q < chains; ++q) a += (double)F[(size_t)q * ldF + n];
    Sf[n] += a;
}

// shift[n] = mean over chains of f[q][n] (the centre of all later snapshots)
template <class T>
__global__ void shift_kernel(const T *F, int ldF, int chains, int N, double *shift)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double a = 0.0;
    for (int q = 0; q < chains; ++q) a += (double)F[(size_t)q * ldF + n];
    shift[n] = a / chains;
}

// D = F - shift (rows of chains, padding kept at zero)
template <class T>
__global__ void center_kernel(const T *F, int ldF, int chains, int N, const double *shift, T *D)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)chains * ldF) return;
    const int n = (int)(i % ldF);
    D[i] = n < N ? (T)((double)F[i] - shift[n]) : T(0);
}

// kshift[p*M + m] = (K~_theta_p shift)[m] in FP64
__global__ void kshift_kernel(const double *Kth, const double *shift, int M, int N, int P, double *kshift)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * P) return;
    const int pi = i / M, m = i - pi * M;
    double a = 0.0;
    for (int n = 0; n < N; ++n) a += Kth[((size_t)pi * M + m) * N + n] * shift[n];
    kshift[i] = a;
}

// Sfs[n*P + p] += sum_q f[q][n] s[q][p]; Ss[p] += sum_q s[q][p] (thread n < P also does Ss).
template <class T>
__global__ void fs_kernel(const T *F, int ldF, const double *Sq, int chains, int N, int P, double *Sfs,
                          double *Ss)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    for (int pi = 0; pi < P; ++pi) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < chains; ++q) {
            const double s = Sq[(size_t)q * P + pi];
            a += (double)F[(size_t)q * ldF + n] * s;
            b += s;
        }
        Sfs[(size_t)n * P + pi] += a;
        if (n == 0) Ss[pi] += b;
    }
}

// Backward: u = Cov(fbar) v' from the snapshot moments (v' = v / w).
// (the moments are of d = fbar - shift: the covariance is unchanged)
__global__ void vjp_cov_kernel(const double *Sff, const double *Sf, double ns, const double *vp, int N, double *u)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double mv = 0.0, a = 0.0;
    for (int k = 0; k < N; ++k) {
        mv += Sf[k] * vp[k];
        a += Sff[(size_t)k * N + n] * vp[k];
    }
    u[n] = a / ns - (Sf[n] / ns) * (mv / ns);
}

// Backward: g_theta[p] = Cov(v'^T fbar, s_p) - sum_n v_n <fbar_n> dw_pn / w_n^2.
__global__ void vjp_theta_kernel(const double *Sfs, const double *Ss, const double *Sf, const double *shift,
                                 double ns, const double *vp, const double *v, const double *w, const double *dw,
                                 int N, int P, double *g)
{
    const int pi = blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= P) return;
    double c = 0.0, m = 0.0, t = 0.0;
    for (int n = 0; n < N; ++n) {
        c += vp[n] * Sfs[(size_t)n * P + pi];
        m += vp[n] * Sf[n];
        t += v[n] * (Sf[n] / ns + shift[n]) * dw[(size_t)pi * N + n] / (w[n] * w[n]);
    }
    g[pi] = c / ns - (m / ns) * (Ss[pi] / ns) - t;
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int round_up_int(int x, int a) { return (x + a - 1) / a * a; }

struct WsLayout {
    size_t counters, F, R, S1, S2, chi2;
    size_t Sff, Sf, Sfs, Ss, Y, Sq;         // snapshot moments for the backward pass
    size_t shift, kshift, D;                // centring of the snapshots
    size_t S1p, bpend, bacc1, bacc2, bcount; // binning of the Monte Carlo error
    size_t fref, rref;                       // reference state of the tensor-core refresh
    size_t steptrace;                        // step-size trace (kStepTraceMax sweeps)
    size_t P1, P2;                           // FP32 path: kept-sweep sums of the open 64-sweep block (chains x ldF FP32)
    size_t Dpart;                            // FP32 path: k parts of the tensor-core refresh (ksplit x chains x ldR)
    int ksplit;
    size_t total;
    int ldF, ldR;
};

}  // namespace

// device buffers of one precision
struct PrecBuffers {
    void *V = nullptr, *R = nullptr, *d = nullptr, *invd = nullptr, *meta = nullptr,
         *rec = nullptr, *Ut = nullptr, *Um = nullptr, *Us = nullptr;
    void *prior_am1 = nullptr;   // a_n - 1 of the gamma prior (nullptr: flat)
};

struct asm_problem {
    int M = 0, N = 0, n_levels = 0, n_blocks = 0;
    std::vector<int> level_nblocks, level_first;
    std::vector<BlockDesc> blocks;
    std::vector<double> w;
    double f0 = 0.0;
    int max_nb = 0, max_np = 0;
    long long totV = 0, totR = 0, totd = 0, totU = 0, totRec = 0, totUs = 0;
    int max_rec = 0;   // largest record (elements)
    // device
    int *d_level_first = nullptr, *d_level_nblocks = nullptr;
    BlockDesc *d_blocks = nullptr;
    double *d_KtT = nullptr, *d_gt = nullptr;
    float *d_Khi = nullptr, *d_Klo = nullptr;   // K~ split into TF32 high/low parts (M x ldK)
    int ldK = 0;
    // backward pass
    int P = 0;
    double *d_L = nullptr;                 // Cholesky factor of C (M x M, column-major lower)
    double *d_Kth64 = nullptr;             // whitened dK/dtheta, P x M x N
    float *d_Kth32 = nullptr;
    double *d_w = nullptr, *d_dw = nullptr;   // weights and dw/dtheta (P x N)
    double *d_vjp = nullptr;               // scratch of asm_backward: v', v, u (N each), y (M), g (P)
    bool moments = false;
    long long nsnap = 0;                   // chain snapshots in the moments
    PrecBuffers b64, b32;
    // batch: one sub-handle per problem (empty for a single problem)
    std::vector<asm_problem *> kids;
    // run state
    void *ws_all = nullptr;   // the caller's workspace (header + every problem's section)
    void *ws = nullptr;       // this problem's section of it
    size_t ws_bytes = 0;
    int chains = 0, precision = -1, team = 32;
    long long sweeps_done = 0, kept = 0;
    long long kept_since = 0;   // every sweep from this one on has been accumulated
    unsigned long long seed = 0;
    unsigned long long problem_id = 0, chain_offset = 0;   // Philox identities of the run
    unsigned long long next_problem_id = 0, next_chain_offset = 0;
    cudaStream_t stream = nullptr;
    bool have_run = false;
    // launch shape chosen by asm_tune (0: the built-in heuristic)
    int tuned_consumers = 0;
    int tuned_minb = 0;   // CTAs per SM the registers are budgeted for (0: heuristic)
    // one refresh period (advance the range, sweep, refresh) as a CUDA graph
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    struct GraphKey {
        const void *ws_all = nullptr;
        int chains = 0, precision = -1, kv = 0, ctas = 0, S = 0, consumers = 0, depth = 0, n_items = 0, minb = 0,
            ubytes = 0, rps = 0, npad = 0;
        size_t refresh_smem = 0;
        unsigned long long seed = 0, problem_id = 0, chain_offset = 0;
        bool operator==(const GraphKey &o) const
        {
            return ws_all == o.ws_all && chains == o.chains && precision == o.precision && kv == o.kv &&
                   ctas == o.ctas && S == o.S && consumers == o.consumers && depth == o.depth &&
                   n_items == o.n_items && minb == o.minb && ubytes == o.ubytes && rps == o.rps && npad == o.npad &&
                   refresh_smem == o.refresh_smem &&
                   seed == o.seed &&
                   problem_id == o.problem_id && chain_offset == o.chain_offset;
        }
    } gkey;
    long long graph_replays = 0, tc_refreshes = 0;
    bool refresh_fp64 = false;   // mixed path: FP64 CUDA-core refresh instead of the tensor cores
    int last_team = 0, last_consumers = 0, last_ctas = 0, last_items = 0, last_minb = 0;   // last sweep launch
    bool no_graph = false;    // direct launches only (the allocation-free entry point)
    bool trace = false;       // ASM_SAMPLE_STEP_TRACE: the step-size trace of every sweep
    bool test_stall = false;  // ASM_FLAG_TEST_STALL: the failure path under test
    // launch bookkeeping
    long long sweep_launches = 0, other_launches = 0, timed_launches = 0;
    double timed_ms = 0.0;
    std::vector<cudaEvent_t> ev_pool;     // pairs (start, stop), reused
    size_t ev_used = 0;                   // events recorded and not yet read
    bool timing = false;
};

namespace {

WsLayout ws_layout(const asm_problem *p, int chains, int precision)
{
    WsLayout L{};
    const size_t es = precision == ASM_FP64 ? 8 : 4;
    L.ldF = round_up_int(p->N, 4);
    L.ldR = round_up_int(p->M, 4);
    size_t off = 0;
    L.counters = off; off = align_up(off + sizeof(Counters), 256);
    L.F = off; off = align_up(off + (size_t)chains * L.ldF * es, 256);
    L.R = off; off = align_up(off + (size_t)chains * L.ldR * es, 256);
    L.S1 = off; off = align_up(off + (size_t)chains * p->N * 8, 256);
    L.S2 = off; off = align_up(off + (size_t)chains * p->N * 8, 256);
    L.chi2 = off; off = align_up(off + (size_t)chains * 8, 256);
    const size_t N = (size_t)p->N, P = (size_t)p->P;
    L.Sff = off; off = align_up(off + N * N * 8, 256);
    L.Sf = off; off = align_up(off + N * 8, 256);
    L.Sfs = off; off = align_up(off + N * std::max<size_t>(P, 1) * 8, 256);
    L.Ss = off; off = align_up(off + std::max<size_t>(P, 1) * 8, 256);
    L.Y = off; off = align_up(off + (P ? (size_t)chains * P * p->M * es : 0), 256);
    L.Sq = off; off = align_up(off + (size_t)chains * std::max<size_t>(P, 1) * 8, 256);
    L.shift = off; off = align_up(off + N * 8, 256);
    L.kshift = off; off = align_up(off + (size_t)p->M * std::max<size_t>(P, 1) * 8, 256);
    L.D = off; off = align_up(off + (size_t)chains * L.ldF * es, 256);
    const size_t binned = (size_t)chains * kBinLevels * N * 8;
    L.S1p = off; off = align_up(off + (size_t)chains * N * 8, 256);
    L.bpend = off; off = align_up(off + binned, 256);
    L.bacc1 = off; off = align_up(off + binned, 256);
    L.bacc2 = off; off = align_up(off + binned, 256);
    L.bcount = off; off = align_up(off + (size_t)chains * 4, 256);
    L.fref = off; off = align_up(off + N * 4, 256);
    L.rref = off; off = align_up(off + (size_t)p->M * 8, 256);
    L.steptrace = off; off = align_up(off + (size_t)kStepTraceMax * 8, 256);
    L.P1 = off; off = align_up(off + (precision == ASM_FP64 ? 0 : (size_t)chains * L.ldF * 4), 256);
    L.P2 = off; off = align_up(off + (precision == ASM_FP64 ? 0 : (size_t)chains * L.ldF * 4), 256);
    L.ksplit = precision == ASM_FP64 ? 1 : refresh_tc_ksplit(chains, p->N);
    L.Dpart = off; off = align_up(off + (L.ksplit > 1 ? (size_t)L.ksplit * chains * L.ldR * 4 : 0), 256);
    L.total = off;
    return L;
}

// The problems a handle samples: itself, or every problem of a batch.
std::vector<asm_problem *> units_of(asm_problem *p)
{
    if (p->kids.empty()) return {p};
    return p->kids;
}
std::vector<const asm_problem *> units_of(const asm_problem *p)
{
    if (p->kids.empty()) return {p};
    return std::vector<const asm_problem *>(p->kids.begin(), p->kids.end());
}

// Workspace = header (launch control, work items, per-problem launch parameters)
// followed by one section per problem.
struct RunLayout {
    size_t ctrl, items, probs, header;
    std::vector<size_t> unit;   // offset of each problem's section
    size_t total;
};

RunLayout run_layout(const asm_problem *p, int chains, int precision)
{
    RunLayout R{};
    const auto us = units_of(p);
    const size_t nu = us.size();
    R.ctrl = 0;
    R.items = 256;
    R.probs = align_up(R.items + nu * (size_t)chains * sizeof(WorkItem), 256);
    R.header = align_up(R.probs + nu * sizeof(SweepParams<double>), 256);
    size_t off = R.header;
    for (const asm_problem *u : us) {
        R.unit.push_back(off);
        off = align_up(off + ws_layout(u, chains, precision).total, 256);
    }
    R.total = off;
    return R;
}

template <class T>
int upload(void **dst, const std::vector<T> &src)
{
    if (cudaMalloc(dst, std::max<size_t>(src.size(), 1) * sizeof(T)) != cudaSuccess) return ASM_ERR_CUDA;
    if (!src.empty() &&
        cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return ASM_ERR_CUDA;
    return ASM_OK;
}

void free_prec(PrecBuffers &b)
{
    void *ptrs[] = {b.V, b.R, b.d, b.invd, b.meta, b.rec, b.Ut, b.Um, b.Us, b.prior_am1};
    for (void *x : ptrs)
        if (x) cudaFree(x);
    b = PrecBuffers{};
}

// Per-block factors in host FP64 (mode-major), produced either by cuSOLVER or
// given by the caller.
struct HostFactors {
    std::vector<double> Kt, gt;            // M x N row-major, M
    std::vector<std::vector<double>> d;    // per block, n
    std::vector<std::vector<double>> V;    // per block, n x n mode-major
    std::vector<std::vector<double>> U;    // per block, np x M mode-major
    std::vector<std::vector<double>> dres; // per block, n: |K~_b V_j| for the residual update
};

// The residual moves by K~_b V_j delta whatever the draw of mode j was.  For a
// mode sampled flat (d = 0: numerically zero, or below the threshold of reading
// R2 with a sign-changing V_j) its small K~_b V_j is formed here in FP64, and U_j
// and dres_j are set to its direction and length, so that the exit update
// r~ -= U_b (dres delta) keeps the tracked residual equal to g~ - K~ f (the
// conditional means of weak modes are sensitive to a residual that misses it).
// Modes j >= np lie in the exact null space of the block: nothing to add.
void complete_residual_update(const asm_problem *p, HostFactors &hf)
{
    const int M = p->M, N = p->N;
    hf.dres.resize(p->blocks.size());
    for (size_t b = 0; b < p->blocks.size(); ++b) {
        const BlockDesc &B = p->blocks[b];
        std::vector<double> &dr = hf.dres[b];
        dr.assign(B.n, 0.0);
        for (int j = 0; j < B.np; ++j) {
            if (hf.d[b][j] > 0.0) {
                dr[j] = hf.d[b][j];
                continue;
            }
            const double *v = &hf.V[b][(size_t)j * B.n];
            std::vector<double> w(M, 0.0);
            double nrm2 = 0.0;
            for (int m = 0; m < M; ++m) {
                double a = 0.0;
                for (int i = 0; i < B.n; ++i) a += hf.Kt[(size_t)m * N + B.start + i] * v[i];
                w[m] = a;
                nrm2 += a * a;
            }
            const double nrm = std::sqrt(nrm2);
            dr[j] = nrm;
            for (int m = 0; m < M; ++m) hf.U[b][(size_t)j * M + m] = nrm > 0.0 ? w[m] / nrm : 0.0;
        }
    }
}

#define CK_CUDA(x) do { if ((x) != cudaSuccess) { rc = ASM_ERR_CUDA; goto done; } } while (0)
#define CK_CUBLAS(x) do { if ((x) != CUBLAS_STATUS_SUCCESS) { rc = ASM_ERR_CUDA; goto done; } } while (0)
#define CK_SOLVER(x) do { if ((x) != CUSOLVER_STATUS_SUCCESS) { rc = ASM_ERR_CUDA; goto done; } } while (0)

// Whitening (C = L L^T, K~ = L^{-1} K, g~ = L^{-1} G) and the SVD of every block,
// all in FP64 on the device (cuSOLVER potrf / gesvd, cuBLAS trsm / trsv).
int device_factorize(const asm_desc *ds, const asm_problem *p, HostFactors &hf, double **L_out)
{
    const int M = ds->M, N = ds->N;
    int rc = ASM_OK;
    cusolverDnHandle_t sh = nullptr;
    cublasHandle_t bh = nullptr;
    double *dC = nullptr, *dK = nullptr, *dG = nullptr, *dA = nullptr, *dS = nullptr, *dU = nullptr,
           *dVT = nullptr, *dwork = nullptr, *drwork = nullptr;
    int *dinfo = nullptr;
    int info = 0, lwork = 0;
    const double one = 1.0;
    std::vector<double> A, S, Uh, VTh;

    CK_SOLVER(cusolverDnCreate(&sh));
    CK_CUBLAS(cublasCreate(&bh));
    CK_CUDA(cudaMalloc(&dC, sizeof(double) * M * M));
    CK_CUDA(cudaMalloc(&dK, sizeof(double) * M * N));
    CK_CUDA(cudaMalloc(&dG, sizeof(double) * M));
    CK_CUDA(cudaMalloc(&dinfo, sizeof(int)));
    CK_CUDA(cudaMemcpy(dC, ds->C, sizeof(double) * M * M, cudaMemcpyHostToDevice));
    CK_CUDA(cudaMemcpy(dK, ds->K, sizeof(double) * M * N, cudaMemcpyHostToDevice));
    CK_CUDA(cudaMemcpy(dG, ds->G, sizeof(double) * M, cudaMemcpyHostToDevice));
    // Cholesky of the (symmetric) covariance: row-major and column-major agree
    CK_SOLVER(cusolverDnDpotrf_bufferSize(sh, CUBLAS_FILL_MODE_LOWER, M, dC, M, &lwork));
    CK_CUDA(cudaMalloc(&dwork, sizeof(double) * std::max(lwork, 1)));
    CK_SOLVER(cusolverDnDpotrf(sh, CUBLAS_FILL_MODE_LOWER, M, dC, M, dwork, lwork, dinfo));
    CK_CUDA(cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost));
    if (info != 0) { rc = ASM_ERR_NOT_SPD; goto done; }
    cudaFree(dwork); dwork = nullptr;
    // K row-major M x N is K^T column-major (N x M): solve X L^T = K^T, X = K~^T
    CK_CUBLAS(cublasDtrsm(bh, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT,
                          N, M, &one, dC, M, dK, N));
    CK_CUBLAS(cublasDtrsv(bh, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, M, dC, M, dG, 1));
    hf.Kt.resize((size_t)M * N);
    hf.gt.resize(M);
    CK_CUDA(cudaMemcpy(hf.Kt.data(), dK, sizeof(double) * M * N, cudaMemcpyDeviceToHost));
    CK_CUDA(cudaMemcpy(hf.gt.data(), dG, sizeof(double) * M, cudaMemcpyDeviceToHost));

    hf.d.resize(p->n_blocks);
    hf.V.resize(p->n_blocks);
    hf.U.resize(p->n_blocks);
    for (int b = 0; b < p->n_blocks; ++b) {
        const int s0 = p->blocks[b].start, n = p->blocks[b].n, np = std::min(M, n);
        const bool tall = M >= n;             // gesvd wants rows >= columns
        const int rm = tall ? M : n, cn = tall ? n : M;
        A.assign((size_t)rm * cn, 0.0);
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < n; ++j) {
                const double x = hf.Kt[(size_t)i * N + s0 + j];
                if (tall) A[i + (size_t)j * M] = x;     // A (M x n), column-major
                else A[j + (size_t)i * n] = x;          // A^T (n x M), column-major
            }
        CK_CUDA(cudaMalloc(&dA, sizeof(double) * rm * cn));
        CK_CUDA(cudaMalloc(&dS, sizeof(double) * cn));
        CK_CUDA(cudaMalloc(&dU, sizeof(double) * rm * (tall ? cn : rm)));
        CK_CUDA(cudaMalloc(&dVT, sizeof(double) * cn * cn));
        CK_CUDA(cudaMalloc(&drwork, sizeof(double) * std::max(cn, 2)));
        CK_CUDA(cudaMemcpy(dA, A.data(), sizeof(double) * rm * cn, cudaMemcpyHostToDevice));
        CK_SOLVER(cusolverDnDgesvd_bufferSize(sh, rm, cn, &lwork));
        CK_CUDA(cudaMalloc(&dwork, sizeof(double) * std::max(lwork, 1)));
        CK_SOLVER(cusolverDnDgesvd(sh, tall ? 'S' : 'A', 'A', rm, cn, dA, rm, dS, dU, rm, dVT, cn, dwork,
                                   lwork, drwork, dinfo));
        CK_CUDA(cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost));
        if (info != 0) { rc = ASM_ERR_CUDA; goto done; }
        S.resize(cn);
        Uh.resize((size_t)rm * (tall ? cn : rm));
        VTh.resize((size_t)cn * cn);
        CK_CUDA(cudaMemcpy(S.data(), dS, sizeof(double) * cn, cudaMemcpyDeviceToHost));
        CK_CUDA(cudaMemcpy(Uh.data(), dU, sizeof(double) * Uh.size(), cudaMemcpyDeviceToHost));
        CK_CUDA(cudaMemcpy(VTh.data(), dVT, sizeof(double) * VTh.size(), cudaMemcpyDeviceToHost));
        cudaFree(dA); cudaFree(dS); cudaFree(dU); cudaFree(dVT); cudaFree(dwork); cudaFree(drwork);
        dA = dS = dU = dVT = dwork = drwork = nullptr;

        std::vector<double> &d = hf.d[b], &V = hf.V[b], &U = hf.U[b];
        d.assign(n, 0.0);
        V.assign((size_t)n * n, 0.0);
        U.assign((size_t)np * M, 0.0);
        for (int j = 0; j < n; ++j) {
            for (int i = 0; i < n; ++i)
                V[(size_t)j * n + i] = tall ? VTh[j + (size_t)i * n] : Uh[i + (size_t)j * n];
            if (j < np) {
                d[j] = S[j];
                for (int m = 0; m < M; ++m) U[(size_t)j * M + m] = tall ? Uh[m + (size_t)j * M] : VTh[j + (size_t)m * M];
            }
        }
        // sign: the largest |component| of every V_j is positive (lowest index on ties).
        // Zero modes (flat on their interval): d <= d_1 max(M,n) 2^-52, and d up to
        // d_1 max(M,n) 2^-40 when V_j changes sign -- there U_j = K~ V_j / d_j is not
        // resolvable in FP64 (error ~ 2^-52 d_1 / d_j) while the likelihood is flat to
        // exp(-(d Delta)^2 / 2) over the positivity interval Delta.
        const double dmax = (double)std::max(M, n);
        const double thr0 = (np > 0 ? d[0] : 0.0) * dmax * 0x1p-52, thr = (np > 0 ? d[0] : 0.0) * dmax * 0x1p-40;
        for (int j = 0; j < n; ++j) {
            double *v = &V[(size_t)j * n];
            int imax = 0;
            for (int i = 1; i < n; ++i)
                if (std::fabs(v[i]) > std::fabs(v[imax])) imax = i;
            if (v[imax] < 0.0) {
                for (int i = 0; i < n; ++i) v[i] = -v[i];
                if (j < np)
                    for (int m = 0; m < M; ++m) U[(size_t)j * M + m] = -U[(size_t)j * M + m];
            }
            if (j < np && d[j] <= thr) {
                const double vm = std::fabs(v[imax]);
                bool pos = false, neg = false;
                for (int i = 0; i < n; ++i) {
                    if (std::fabs(v[i]) < 0x1p-40 * vm) continue;
                    pos = pos || v[i] > 0.0;
                    neg = neg || v[i] < 0.0;
                }
                if (d[j] <= thr0 || (pos && neg)) {
                    d[j] = 0.0;
                    for (int m = 0; m < M; ++m) U[(size_t)j * M + m] = 0.0;
                }
            }
        }
    }
done:
    if (rc == ASM_OK && L_out) {   // keep the Cholesky factor for the backward pass
        *L_out = dC;
        dC = nullptr;
    }
    if (dC) cudaFree(dC);
    if (dK) cudaFree(dK);
    if (dG) cudaFree(dG);
    if (dA) cudaFree(dA);
    if (dS) cudaFree(dS);
    if (dU) cudaFree(dU);
    if (dVT) cudaFree(dVT);
    if (dwork) cudaFree(dwork);
    if (drwork) cudaFree(drwork);
    if (dinfo) cudaFree(dinfo);
    if (bh) cublasDestroy(bh);
    if (sh) cusolverDnDestroy(sh);
    return rc;
}

// Cholesky factor of C on the device (column-major lower), for a problem whose
// factors were given but whose covariance is known.
int device_cholesky(const double *C, int M, double **L_out)
{
    cusolverDnHandle_t sh = nullptr;
    double *dC = nullptr, *dwork = nullptr;
    int *dinfo = nullptr;
    int rc = ASM_OK, lwork = 0, info = 0;
    CK_SOLVER(cusolverDnCreate(&sh));
    CK_CUDA(cudaMalloc(&dC, sizeof(double) * M * M));
    CK_CUDA(cudaMalloc(&dinfo, sizeof(int)));
    CK_CUDA(cudaMemcpy(dC, C, sizeof(double) * M * M, cudaMemcpyHostToDevice));
    CK_SOLVER(cusolverDnDpotrf_bufferSize(sh, CUBLAS_FILL_MODE_LOWER, M, dC, M, &lwork));
    CK_CUDA(cudaMalloc(&dwork, sizeof(double) * std::max(lwork, 1)));
    CK_SOLVER(cusolverDnDpotrf(sh, CUBLAS_FILL_MODE_LOWER, M, dC, M, dwork, lwork, dinfo));
    CK_CUDA(cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost));
    if (info != 0) rc = ASM_ERR_NOT_SPD;
done:
    if (rc == ASM_OK) {
        *L_out = dC;
        dC = nullptr;
    }
    if (dC) cudaFree(dC);
    if (dwork) cudaFree(dwork);
    if (dinfo) cudaFree(dinfo);
    if (sh) cusolverDnDestroy(sh);
    return rc;
}

// K~_theta_p = L^{-1} dK/dtheta_p for every parameter (same trsm as the kernel).
int whiten_dK(asm_problem *p, const double *dK)
{
    const int M = p->M, N = p->N, P = p->P;
    int rc = ASM_OK;
    const double one = 1.0;
    std::vector<float> h32;
    cublasHandle_t bh = nullptr;   // set-up only: the sampling and backward paths use no library
    CK_CUBLAS(cublasCreate(&bh));
    CK_CUDA(cudaMalloc(&p->d_Kth64, sizeof(double) * (size_t)P * M * N));
    CK_CUDA(cudaMalloc(&p->d_Kth32, sizeof(float) * (size_t)P * M * N));
    CK_CUDA(cudaMemcpy(p->d_Kth64, dK, sizeof(double) * (size_t)P * M * N, cudaMemcpyHostToDevice));
    for (int pi = 0; pi < P; ++pi)
        CK_CUBLAS(cublasDtrsm(bh, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T,
                              CUBLAS_DIAG_NON_UNIT, N, M, &one, p->d_L, M, p->d_Kth64 + (size_t)pi * M * N, N));
    {
        std::vector<double> h((size_t)P * M * N);
        CK_CUDA(cudaMemcpy(h.data(), p->d_Kth64, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
        h32.assign(h.begin(), h.end());
    }
    CK_CUDA(cudaMemcpy(p->d_Kth32, h32.data(), sizeof(float) * h32.size(), cudaMemcpyHostToDevice));
done:
    if (bh) cublasDestroy(bh);
    return rc;
}

// Host-side mode rows for one precision, then upload.
template <class T>
int build_precision(asm_problem *p, const HostFactors &hf, PrecBuffers &out)
{
    const int M = p->M;
    const T nan = std::numeric_limits<T>::quiet_NaN();
    constexpr int MW = 16 / sizeof(T);
    std::vector<T> V(p->totV, T(0)), R(p->totR, nan), d(p->totd, T(0)),
        invd(p->totd, T(0)), meta((size_t)p->totd * MW, T(0)), rec(std::max<long long>(p->totRec, 1), T(0)),
        Ut(std::max<long long>(p->totU, 1), T(0)),
        Um(std::max<long long>(p->totU, 1), T(0)),
        Us(p->totUs + 4, T(0));   // + 4: a copy rounded up to 16 bytes stays inside
    for (int b = 0; b < p->n_blocks; ++b) {
        const BlockDesc &B = p->blocks[b];
        const std::vector<double> &hd = hf.d[b], &hV = hf.V[b], &hU = hf.U[b];
        for (int j = 0; j < B.n; ++j) {
            const double *v = &hV[(size_t)j * B.n];
            double vmax = 0.0;
            for (int i = 0; i < B.n; ++i) vmax = std::max(vmax, std::fabs(v[i]));
            for (int i = 0; i < B.n; ++i) {
                V[B.offV + (size_t)j * B.rs + i] = (T)v[i];
                if (std::fabs(v[i]) < 0x1p-40 * vmax) continue;   // left out of the bounds
                R[B.offR + (size_t)j * B.rs + i] = (T)(-1.0 / v[i]);
            }
            d[B.offd + j] = (T)hd[j];
            invd[B.offd + j] = hd[j] > 0.0 ? (T)(1.0 / hd[j]) : T(0);
            meta[(size_t)(B.offd + j) * MW] = d[B.offd + j];
            meta[(size_t)(B.offd + j) * MW + 1] = invd[B.offd + j];
        }
        for (int j = 0; j < B.np; ++j)
            for (int m = 0; m < M; ++m) {
                Ut[B.offU + (size_t)j * M + m] = (T)hU[(size_t)j * M + m];
                Um[B.offU + (size_t)m * B.np + j] = (T)hU[(size_t)j * M + m];
                Us[B.offUs + (size_t)j * B.usr + m] = (T)hU[(size_t)j * M + m];
            }
        // move records: {V_j, R_{j+1}, d_j, 1/d_j, dres_j}
        for (int j = 0; j < B.n; ++j) {
            T *r = &rec[B.offRec + (size_t)j * B.recstride];
            for (int i = 0; i < B.rs; ++i) {
                r[i] = V[B.offV + (size_t)j * B.rs + i];
                r[B.rs + i] = R[B.offR + (size_t)(j + 1) * B.rs + i];
            }
            r[2 * B.rs] = d[B.offd + j];
            r[2 * B.rs + 1] = invd[B.offd + j];
            r[2 * B.rs + 2] = (T)hf.dres[b][j];
        }
    }
    int rc;
    if ((rc = upload(&out.V, V)) || (rc = upload(&out.R, R)) ||
        (rc = upload(&out.d, d)) || (rc = upload(&out.invd, invd)) || (rc = upload(&out.meta, meta)) || (rc = upload(&out.rec, rec)) ||
        (rc = upload(&out.Ut, Ut)) ||
        (rc = upload(&out.Um, Um)) || (rc = upload(&out.Us, Us)))
        return rc;
    return ASM_OK;
}

bool all_finite(const double *x, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

}  // namespace

namespace {

// Read the recorded event pairs (synchronises the stream) into the totals.
int drain_events(asm_problem *p)
{
    if (p->ev_used == 0) return ASM_OK;
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return ASM_ERR_CUDA;
    for (size_t i = 0; i + 1 < p->ev_used; i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->ev_pool[i], p->ev_pool[i + 1]) != cudaSuccess) return ASM_ERR_CUDA;
        p->timed_ms += ms;
        ++p->timed_launches;
    }
    p->ev_used = 0;
    return ASM_OK;
}

cudaEvent_t next_event(asm_problem *p)
{
    if (p->ev_used == p->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        p->ev_pool.push_back(e);
    }
    return p->ev_pool[p->ev_used++];
}

template <class T>
SweepParams<T> make_params(asm_problem *p, const PrecBuffers &b, const WsLayout &L, int chains)
{
    SweepParams<T> sp{};
    sp.M = p->M;
    sp.N = p->N;
    sp.n_levels = p->n_levels;
    sp.level_first = p->d_level_first;
    sp.level_nblocks = p->d_level_nblocks;
    sp.blocks = p->d_blocks;
    sp.pd.V = (const T *)b.V;
    sp.pd.R = (const T *)b.R;
    sp.pd.d = (const T *)b.d;
    sp.pd.invd = (const T *)b.invd;
    sp.pd.Ut = (const T *)b.Ut;
    sp.pd.Um = (const T *)b.Um;
    sp.pd.Us = (const T *)b.Us;
    char *ws = (char *)p->ws;
    sp.F = (T *)(ws + L.F);
    sp.ldF = L.ldF;
    sp.R = (T *)(ws + L.R);
    sp.ldR = L.ldR;
    sp.S1 = (double *)(ws + L.S1);
    sp.S2 = (double *)(ws + L.S2);
    sp.chains = chains;
    sp.seed = p->seed;
    sp.problem_id = p->problem_id;
    sp.chain_offset = p->chain_offset;
    sp.counters = (Counters *)(ws + L.counters);
    sp.pd.meta = (const T *)b.meta;
    sp.pd.rec = (const T *)b.rec;
    sp.KtT = p->d_KtT;
    sp.Khi = p->d_Khi;
    sp.Klo = p->d_Klo;
    sp.ldK = p->ldK;
    sp.prior_am1 = (const T *)b.prior_am1;
    sp.gt = p->d_gt;
    sp.chi2 = (double *)(ws + L.chi2);
    sp.S1p = (double *)(ws + L.S1p);
    sp.bpend = (double *)(ws + L.bpend);
    sp.bacc1 = (double *)(ws + L.bacc1);
    sp.bacc2 = (double *)(ws + L.bacc2);
    sp.bcount = (int *)(ws + L.bcount);
    sp.f0 = p->f0;
    sp.fref = (float *)(ws + L.fref);
    sp.rref = (double *)(ws + L.rref);
    sp.steptrace = p->trace ? (double *)(ws + L.steptrace) : nullptr;
    sp.P1 = sizeof(T) == 4 ? (float *)(ws + L.P1) : nullptr;
    sp.P2 = sizeof(T) == 4 ? (float *)(ws + L.P2) : nullptr;
    sp.ksplit = sizeof(T) == 4 ? L.ksplit : 1;
    sp.Dpart = sp.ksplit > 1 ? (float *)(ws + L.Dpart) : nullptr;
    sp.trace_cap = kStepTraceMax;
    return sp;
}

// Shared memory of the sweep kernel: per team c, w, r~ and the uniforms of a
// window of 4S moves (draws and prior acceptances); the ring's `full`
// and `empty` barriers and `depth` record stages.  Consumer warps per CTA:
// enough that the CTAs about cover the SMs once (all chains of an SM then
// share one ring), or the tuned count.  CTAs per SM: as many as the work
// needs and the registers allow (the persistent kernel queues the rest); the
// ring is as deep as the shared memory left to each of them.  For a batch the
// shape covers the largest problem.
int ctas_per_sm(int precision, const LaunchShape &sh, int kv, bool batch)
{
    if (precision == ASM_FP64)
        return sh.prior ? sweep_ctas_per_sm_f64_prior(sh, kv, batch)
               : sh.minb == 2 ? sweep_ctas_per_sm_f64_m2(sh, kv, batch) : sweep_ctas_per_sm_f64_m1(sh, kv, batch);
    return sh.prior ? sweep_ctas_per_sm_f32_prior(sh, kv, batch)
           : sh.minb == 2 ? sweep_ctas_per_sm_f32_m2(sh, kv, batch) : sweep_ctas_per_sm_f32_m1(sh, kv, batch);
}

template <class T>
bool plan_shape(LaunchShape &sh, int S, int max_rec, int max_np, int max_M, long long total_warps, int kv,
                bool batch, int want_consumers, int minb, bool prior, const std::vector<int> &ublk_bytes,
                int max_N_sum)
{
    sh.minb = prior ? 1 : minb;   // the prior's kernels exist for one CTA per SM
    sh.prior = prior ? 1 : 0;
    sh.wait_limit = kWaitLimit;
    sh.stall = 0;
    constexpr int kSMs = 152;
    constexpr int kMinRingRecords = 8;   // the U stages may not squeeze the ring below this many records
    const int TW = 32 / S;
    const int prec = sizeof(T) == 8 ? ASM_FP64 : ASM_MIXED;
    sh.S = S;
    sh.cpad = round_up_int(std::max(max_np, 1), 32);
    sh.mpad = round_up_int(std::max(max_M, 1), 32);
    sh.npad = 0;
    int consumers = want_consumers > 0
                        ? want_consumers
                        : (int)std::min<long long>(kMaxConsumers,
                                                   std::max<long long>(1, (total_warps + kSMs - 1) / kSMs));
    if (const char *e = std::getenv("ASM_CONSUMERS_PER_CTA")) {   // tuning override
        const int c = std::atoi(e);
        if (c >= 1 && c <= kMaxConsumers) consumers = c;
    }
    sh.rps = kRecordsPerStage;
    if (const char *e = std::getenv("ASM_RECORDS_PER_STAGE")) {   // tuning override
        const int r = std::atoi(e);
        if (r >= 1 && r <= 8) sh.rps = r;
    }
    // fewer records per stage where a ring of four stages would not fit (long records: FP64
    // state on large blocks)
    auto stage_of = [&](int rps) { return (int)align_up((size_t)rps * max_rec * sizeof(T), 128); };
    while (sh.rps > 1 && 4 * (size_t)stage_of(sh.rps) > 200 * 1024) --sh.rps;
    sh.stage_bytes = stage_of(sh.rps);
    const int kMinRing = std::max(2, (kMinRingRecords + sh.rps - 1) / sh.rps);
    // per-team state, then the ring's barriers (full, empty: 8 bytes per stage each), the
    // U stages' barriers (4 x 8 bytes, padded to 128) and the U stages
    constexpr int kBarBytes = 8 * kMaxRingDepth;
    auto words = [&](int npad) { return 2 * sh.cpad + sh.mpad + 8 * S + 2 * npad; };
    auto fixed = [&](int c) {
        return align_up((size_t)c * TW * words(sh.npad) * sizeof(T), 128) + 2 * kBarBytes + 128;
    };
    int max_depth = kMaxRingDepth;
    if (const char *e = std::getenv("ASM_RING_DEPTH")) {            // tuning override
        const int d = std::atoi(e);
        if (d >= 2 && d <= kMaxRingDepth) max_depth = d;
    }
    bool stage_u = std::getenv("ASM_NO_U_STAGE") == nullptr;       // tuning override
    for (; consumers >= 1; --consumers) {
        LaunchShape probe = sh;   // no dynamic shared memory: the register limit alone
        probe.consumers = consumers;
        probe.depth = 0;
        probe.off_stages = 0;
        probe.ubytes = 0;
        const int by_regs = std::max(1, ctas_per_sm(prec, probe, kv, batch));
        const long long ctas = (total_warps + consumers - 1) / consumers;
        const int per_sm = (int)std::min<long long>(by_regs, std::max<long long>(1, (ctas + kSMs - 1) / kSMs));
        const size_t budget = std::min<size_t>(220 * 1024 / per_sm, 227 * 1024);
        // FP32 chain state: the kept sweeps' sums of one launch (at most one refresh period)
        // in shared memory, added to the FP64 sums once per launch, where they fit
        sh.npad = 0;
        if (sizeof(T) == 4 && max_N_sum > 0 && std::getenv("ASM_NO_SMEM_SUMS") == nullptr) {
            sh.npad = round_up_int(max_N_sum, 32);
            if (fixed(consumers) + (size_t)kMinRing * sh.stage_bytes > budget) sh.npad = 0;
        }
        // U stages: as large as the largest block U that leaves room for a ring of kMinRing
        size_t ub = 0;
        if (stage_u) {
            const size_t room = budget > fixed(consumers) + (size_t)kMinRing * sh.stage_bytes
                                    ? (budget - fixed(consumers) - (size_t)kMinRing * sh.stage_bytes) / 2
                                    : 0;
            for (int b : ublk_bytes) {
                const size_t bb = align_up((size_t)b, 128);
                if (bb <= room && bb > ub) ub = bb;
            }
        }
        int depth = max_depth;
        while (depth > 2 && fixed(consumers) + 2 * ub + (size_t)depth * sh.stage_bytes > budget) --depth;
        if (fixed(consumers) + 2 * ub + (size_t)depth * sh.stage_bytes <= budget || consumers == 1) {
            if (fixed(consumers) + 2 * ub + (size_t)depth * sh.stage_bytes > 227 * 1024) return false;
            sh.consumers = consumers;
            sh.depth = depth;
            sh.ubytes = (int)ub;
            sh.team_words = words(sh.npad);
            sh.off_full = (int)align_up((size_t)consumers * TW * sh.team_words * sizeof(T), 128);
            sh.off_empty = sh.off_full + kBarBytes;
            sh.off_ubar = sh.off_full + 2 * kBarBytes;
            sh.off_ubuf = sh.off_ubar + 128;
            sh.off_stages = sh.off_ubuf + 2 * (int)ub;
            return true;
        }
    }
    return false;
}

int pick_kv(int max_nb, int vec, int S, int kmax)
{
    int need = (max_nb + vec * S - 1) / (vec * S);
    int kv = 1;
    while (kv < need) kv <<= 1;
    return kv <= kmax ? kv : -1;
}

// Snapshot of all chains into the moments of the backward pass (every
// ASM_SNAPSHOT_EVERY kept sweeps): Sff += F^T F, Sf += column sums of F and,
// with grid parameters, the scores s_p = r~ . (K~_theta_p f) into Sfs, Ss.
template <class T>
int moment_update(asm_problem *p, const WsLayout &L, int chains)
{
    char *ws = (char *)p->ws;
    const int N = p->N, M = p->M;
    const T *Fraw = (const T *)(ws + L.F);
    double *shift = (double *)(ws + L.shift);
    if (p->nsnap == 0) {   // centre every snapshot on the first one's mean (keeps FP32 GEMMs accurate)
        shift_kernel<T><<<(N + 127) / 128, 128, 0, p->stream>>>(Fraw, L.ldF, chains, N, shift);
        ++p->other_launches;
        if (p->P > 0) {
            kshift_kernel<<<(M * p->P + 127) / 128, 128, 0, p->stream>>>(p->d_Kth64, shift, M, N, p->P,
                                                                        (double *)(ws + L.kshift));
            ++p->other_launches;
        }
    }
    {
        const long long tot = (long long)chains * L.ldF;
        center_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, p->stream>>>(Fraw, L.ldF, chains, N, shift,
                                                                               (T *)(ws + L.D));
        ++p->other_launches;
    }
    const T *F = (const T *)(ws + L.D);
    // Sff += D^T D (FP32 partial sums over slices of chains in the mixed path, added in FP64)
    if (launch_gram(F, L.ldF, chains, N, (double *)(ws + L.Sff), p->stream) != cudaSuccess) return ASM_ERR_CUDA;
    colsum_kernel<T><<<(N + 127) / 128, 128, 0, p->stream>>>(F, L.ldF, chains, N, (double *)(ws + L.Sf));
    p->other_launches += 2;
    if (p->P > 0) {
        // Y = D K~_theta^T for every parameter at once, then the scores
        T *Y = (T *)(ws + L.Y);
        const T *Kth;
        if constexpr (sizeof(T) == 8) Kth = p->d_Kth64; else Kth = p->d_Kth32;
        if (launch_kth_product(F, L.ldF, chains, N, Kth, p->P * M, Y, p->stream) != cudaSuccess ||
            launch_scores((const T *)(ws + L.R), L.ldR, (const T *)Y, (const double *)(ws + L.kshift), M, chains,
                          p->P, (double *)(ws + L.Sq), p->stream) != cudaSuccess)
            return ASM_ERR_CUDA;
        p->other_launches += 2;
    }
    if (p->P > 0) {
        fs_kernel<T><<<(N + 127) / 128, 128, 0, p->stream>>>(F, L.ldF, (const double *)(ws + L.Sq), chains, N, p->P,
                                                             (double *)(ws + L.Sfs), (double *)(ws + L.Ss));
        ++p->other_launches;
    }
    if (cudaGetLastError() != cudaSuccess) return ASM_ERR_CUDA;
    p->nsnap += chains;
    return ASM_OK;
}

// Dynamic shared memory of a refresh kernel (one FP64 chain state).
template <class K>
int refresh_smem(K kernel, size_t bytes)
{
    if (bytes > 227 * 1024) return ASM_ERR_TOO_LARGE;
    if (bytes > 48 * 1024 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return ASM_ERR_CUDA;
    return ASM_OK;
}

void drop_graph(asm_problem *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->gkey = asm_problem::GraphKey{};
}

// Sweeps [s_begin, s_end) of every chain of every problem of handle h in
// persistent launches of the sweep kernel, one per refresh period (or
// snapshot interval), each followed where due by the FP64 refresh of all
// residuals.  Whole refresh periods are replays of one CUDA graph (advance
// the range, sweep, refresh) unless launches are timed, snapshots are taken
// or the caller's stream is being captured.
template <class T>
int run_all(asm_problem *h, int chains, long long s_begin, long long s_end, long long burn_abs)
{
    std::vector<asm_problem *> us = units_of(h);
    const RunLayout RL = run_layout(h, chains, h->precision);
    char *base = (char *)h->ws_all;
    std::vector<SweepParams<T>> probs;
    int max_rec = 0, max_np = 1, max_M = 1, max_nb = 1, max_N = 1;
    for (asm_problem *u : us) {
        const WsLayout L = ws_layout(u, chains, h->precision);
        probs.push_back(make_params<T>(u, sizeof(T) == 8 ? u->b64 : u->b32, L, chains));
        max_rec = std::max(max_rec, u->max_rec);
        max_np = std::max(max_np, u->max_np);
        max_M = std::max(max_M, u->M);
        max_nb = std::max(max_nb, u->max_nb);
        max_N = std::max(max_N, u->N);
    }
    // bytes of every block's U in its staging layout (np rows of usr elements, 16-byte multiple)
    std::vector<int> ublk;
    for (asm_problem *u : us)
        for (const BlockDesc &B : u->blocks)
            ublk.push_back((int)(((size_t)B.np * B.usr * sizeof(T) + 15) / 16 * 16));
    const int S = h->team;
    const int vec = 16 / (int)sizeof(T);
    const int kv = pick_kv(max_nb, vec, S, sizeof(T) == 8 ? kMaxKvF64 : kMaxKvF32);
    if (kv < 0) return ASM_ERR_TOO_LARGE;
    const int TW = 32 / S;
    const long long warps_per_unit = (chains + TW - 1) / TW;
    const bool batch = !h->kids.empty();
    const long long total_warps = warps_per_unit * (long long)us.size();
    // register budget: one CTA per SM (up to 255 registers) while one CTA of
    // consumers per SM holds every chain; two CTAs (128 registers) when there
    // are more chains than that, except for FP64 with wide blocks, whose chain
    // state would spill
    int minb = total_warps > 152LL * kMaxConsumers && !(sizeof(T) == 8 && kv >= 16) ? 2 : 1;
    if (h->tuned_minb) minb = h->tuned_minb;
    bool prior = false;   // any problem with a gamma prior: the kernels with the acceptance step
    for (asm_problem *u : us) prior = prior || (sizeof(T) == 8 ? u->b64.prior_am1 : u->b32.prior_am1) != nullptr;
    LaunchShape sh{};
    if (!plan_shape<T>(sh, S, max_rec, max_np, max_M, total_warps, kv, batch, h->tuned_consumers, minb, prior, ublk,
                       max_N))
        return ASM_ERR_TOO_LARGE;
    bool stall = h->test_stall;
    for (asm_problem *u : us) stall = stall || u->test_stall;
    if (stall) {   // failure-path test: no records, short waits
        sh.stall = 1;
        sh.wait_limit = 4096;
    }
    // work items, the costliest problems first (a longest-first queue)
    std::vector<int> order(us.size());
    for (size_t k = 0; k < us.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)us[a]->N * us[a]->max_nb > (long long)us[b]->N * us[b]->max_nb;
    });
    std::vector<WorkItem> items;
    const int groups = (int)((warps_per_unit + sh.consumers - 1) / sh.consumers);
    for (int k : order)
        for (int g = 0; g < groups; ++g) items.push_back(WorkItem{k, g});
    sh.n_items = (int)items.size();
    const int per_sm = ctas_per_sm(h->precision, sh, kv, batch);
    if (per_sm <= 0) return ASM_ERR_CUDA;
    const int ctas = (int)std::min<long long>(sh.n_items, 152LL * per_sm);
    h->last_team = sh.S;
    h->last_consumers = sh.consumers;
    h->last_ctas = ctas;
    h->last_items = sh.n_items;
    h->last_minb = sh.minb;
    const size_t rsmem = sizeof(double) * (size_t)max_N;
    if (const int rc = refresh_smem(refresh_all_kernel<T>, rsmem); rc != ASM_OK) return rc;
    // the mixed path refreshes on the tensor cores (3xTF32) unless asked for FP64 CUDA cores
    const bool tc = sizeof(T) == 4 && !h->refresh_fp64;
    int max_bn = 16, max_parts = 1;
    for (asm_problem *u : us) {
        max_bn = std::max(max_bn, refresh_tc_bn(u->M));
        if (tc) max_parts = std::max(max_parts, refresh_tc_ksplit(chains, u->N));
    }
    if (tc && refresh_tc_smem(max_bn) > 227 * 1024) return ASM_ERR_TOO_LARGE;
    SweepParams<T> *d_probs = (SweepParams<T> *)(base + RL.probs);
    WorkItem *d_items = (WorkItem *)(base + RL.items);
    RunCtrl *ctrl = (RunCtrl *)(base + RL.ctrl);
    if (cudaMemcpyAsync(d_probs, probs.data(), sizeof(SweepParams<T>) * probs.size(), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess)
        return ASM_ERR_CUDA;
    const unsigned n_refresh = (unsigned)(us.size() * chains);
    const SweepParams<T> &p0 = probs[0];   // a single problem's parameters travel by value
    auto sweep = [&](cudaStream_t st) {
        if constexpr (sizeof(T) == 8)
            return sh.prior ? launch_sweeps_f64_prior(p0, d_probs, d_items, ctrl, sh, kv, batch, ctas, st)
                   : sh.minb == 2 ? launch_sweeps_f64_m2(p0, d_probs, d_items, ctrl, sh, kv, batch, ctas, st)
                                  : launch_sweeps_f64_m1(p0, d_probs, d_items, ctrl, sh, kv, batch, ctas, st);
        else
            return sh.prior ? launch_sweeps_f32_prior(p0, d_probs, d_items, ctrl, sh, kv, batch, ctas, st)
                   : sh.minb == 2 ? launch_sweeps_f32_m2(p0, d_probs, d_items, ctrl, sh, kv, batch, ctas, st)
                                  : launch_sweeps_f32_m1(p0, d_probs, d_items, ctrl, sh, kv, batch, ctas, st);
    };
    auto binning = [&](cudaStream_t st) {
        bin_kernel<T><<<n_refresh, 128, 0, st>>>(d_probs, chains, ctrl);
        return cudaGetLastError();
    };
    // kernels of one refresh: reference state, tensor-core product and, with a k split, the
    // FP64 combination; or the FP64 CUDA-core refresh
    const int refresh_launches = tc ? (max_parts > 1 ? 4 : 3) : 1;
    auto refresh = [&](cudaStream_t st) {
        if constexpr (sizeof(T) == 4) {
            if (tc) {
                cudaError_t e = launch_refresh_ref(d_probs, (int)us.size(), chains, max_N, max_M, st);
                if (e == cudaSuccess) e = launch_refresh_tc(d_probs, (int)us.size(), chains, max_bn, max_parts, true, st);
                if (e == cudaSuccess && max_parts > 1) e = launch_refresh_finish(d_probs, (int)us.size(), chains, true, st);
                return e;
            }
        }
        refresh_all_kernel<T><<<n_refresh, 128, rsmem, st>>>(d_probs, chains, 1);
        return cudaGetLastError();
    };
    bool graphs = !h->timing && !h->moments && !h->no_graph && !h->trace;
    if (graphs) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) return ASM_ERR_CUDA;
        graphs = cs == cudaStreamCaptureStatusNone;
    }
    long long s = s_begin;
    while (s < s_end) {
        const long long whole = (s % kRefreshPeriod == 0) ? (s_end - s) / kRefreshPeriod : 0;
        if (graphs && whole >= 2) {
            asm_problem::GraphKey key;
            key.ws_all = h->ws_all;
            key.chains = chains;
            key.precision = h->precision;
            key.kv = kv;
            key.ctas = ctas;
            key.S = sh.S;
            key.consumers = sh.consumers;
            key.depth = sh.depth;
            key.n_items = sh.n_items;
            key.minb = sh.minb + 4 * sh.prior + 8 * sh.stall;
            key.ubytes = sh.ubytes;
            key.rps = sh.rps;
            key.npad = sh.npad;
            key.refresh_smem = tc ? refresh_tc_smem(max_bn) + 1 : rsmem;
            key.seed = p0.seed;   // by value in a single problem's launch
            key.problem_id = p0.problem_id;
            key.chain_offset = p0.chain_offset;
            if (!h->gexec || !(h->gkey == key)) {
                drop_graph(h);
                if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
                    return ASM_ERR_CUDA;
                if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                    return ASM_ERR_CUDA;
                ctrl_kernel<<<1, 1, 0, h->cap_stream>>>(ctrl, 0, 0, 0, 1);
                cudaError_t e = cudaGetLastError();
                if (e == cudaSuccess) e = sweep(h->cap_stream);
                if (e == cudaSuccess) e = binning(h->cap_stream);
                if (e == cudaSuccess) e = refresh(h->cap_stream);
                cudaGraph_t graph = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
                if (e == cudaSuccess && e2 == cudaSuccess)
                    e = cudaGraphInstantiate(&h->gexec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (e != cudaSuccess || e2 != cudaSuccess) {
                    h->gexec = nullptr;
                    return ASM_ERR_CUDA;
                }
                h->gkey = key;
            }
            // the first replay advances [s - P, s) to [s, s + P)
            ctrl_kernel<<<1, 1, 0, h->stream>>>(ctrl, s - kRefreshPeriod, kRefreshPeriod, burn_abs, 0);
            if (cudaGetLastError() != cudaSuccess) return ASM_ERR_CUDA;
            for (long long i = 0; i < whole; ++i)
                if (cudaGraphLaunch(h->gexec, h->stream) != cudaSuccess) return ASM_ERR_CUDA;
            h->sweep_launches += whole;
            h->other_launches += 1 + (2 + refresh_launches) * whole;   // per replay: range, binning, refresh
            h->graph_replays += whole;
            if (tc) h->tc_refreshes += whole;
            s += whole * kRefreshPeriod;
            continue;
        }
        long long seg = std::min<long long>(kRefreshPeriod - (s % kRefreshPeriod), s_end - s);
        if (h->moments) {   // also stop at the next snapshot of the kept sweeps
            const long long k = s < burn_abs ? -1 : (s - burn_abs) / ASM_SNAPSHOT_EVERY;
            const long long next = burn_abs + (k + 1) * ASM_SNAPSHOT_EVERY;
            seg = std::min(seg, next - s);
        }
        ctrl_kernel<<<1, 1, 0, h->stream>>>(ctrl, s, seg, burn_abs, 0);
        if (cudaGetLastError() != cudaSuccess) return ASM_ERR_CUDA;
        ++h->other_launches;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->timing) {
            if (h->ev_used + 2 > 4096 && drain_events(h) != ASM_OK) return ASM_ERR_CUDA;
            e0 = next_event(h);
            e1 = next_event(h);
            if (!e0 || !e1 || cudaEventRecord(e0, h->stream) != cudaSuccess) return ASM_ERR_CUDA;
        }
        if (sweep(h->stream) != cudaSuccess) return ASM_ERR_CUDA;
        if (h->timing && cudaEventRecord(e1, h->stream) != cudaSuccess) return ASM_ERR_CUDA;
        ++h->sweep_launches;
        s += seg;
        if (h->moments && s > burn_abs && (s - burn_abs) % ASM_SNAPSHOT_EVERY == 0) {
            const int rc = moment_update<T>(us[0], ws_layout(us[0], chains, h->precision), chains);
            if (rc != ASM_OK) return rc;
        }
        if (s % kRefreshPeriod == 0) {
            if (binning(h->stream) != cudaSuccess) return ASM_ERR_CUDA;
            if (refresh(h->stream) != cudaSuccess) return ASM_ERR_CUDA;
            h->other_launches += 1 + refresh_launches;
            if (tc) ++h->tc_refreshes;
        }
    }
    return ASM_OK;
}

template <class T>
int init_chains(asm_problem *p, const WsLayout &L, int chains)
{
    char *ws = (char *)p->ws;
    if (cudaMemsetAsync(ws + L.counters, 0, sizeof(Counters), p->stream) != cudaSuccess) return ASM_ERR_CUDA;
    const long long tot = (long long)chains * std::max(L.ldF, p->N);
    init_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, p->stream>>>(
        (T *)(ws + L.F), L.ldF, p->N, p->f0, (double *)(ws + L.S1), (double *)(ws + L.S2), chains);
    if (cudaGetLastError() != cudaSuccess) return ASM_ERR_CUDA;
    if (cudaMemsetAsync(ws + L.R, 0, (size_t)chains * L.ldR * sizeof(T), p->stream) != cudaSuccess)
        return ASM_ERR_CUDA;
    // snapshot moments of the backward pass start at zero
    if (cudaMemsetAsync(ws + L.Sff, 0, L.Y - L.Sff, p->stream) != cudaSuccess) return ASM_ERR_CUDA;
    // binning state starts empty
    if (cudaMemsetAsync(ws + L.S1p, 0, L.bcount + (size_t)chains * 4 - L.S1p, p->stream) != cudaSuccess)
        return ASM_ERR_CUDA;
    // and so does the step-size trace
    if (cudaMemsetAsync(ws + L.steptrace, 0, (size_t)kStepTraceMax * 8, p->stream) != cudaSuccess)
        return ASM_ERR_CUDA;
    // FP32 state: no 64-sweep block of kept sums open yet
    if (sizeof(T) == 4 && cudaMemsetAsync(ws + L.P1, 0, L.Dpart - L.P1, p->stream) != cudaSuccess)
        return ASM_ERR_CUDA;
    p->nsnap = 0;
    if (const int rc = refresh_smem(refresh_kernel<T>, sizeof(double) * p->N); rc != ASM_OK) return rc;
    refresh_kernel<T><<<chains, 128, sizeof(double) * p->N, p->stream>>>(
        p->M, p->N, p->d_KtT, p->d_gt, (const T *)(ws + L.F), L.ldF, (T *)(ws + L.R), L.ldR,
        (double *)(ws + L.chi2), (Counters *)(ws + L.counters), 0);
    if (cudaGetLastError() != cudaSuccess) return ASM_ERR_CUDA;
    p->other_launches += 2;
    return ASM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch of the allocation-free entry point: a fixed device array in this
// file.  Host code must not hand the symbol itself to a kernel (in host code
// it is a host-side stand-in); its device address is looked up once per device.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[ASM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on the
// first call per device, with that device current).
int noalloc_scratch(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return ASM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return ASM_ERR_CUDA;
        g_noalloc_addr[dev] = ptr;
    }
    *out = g_noalloc_addr[dev];
    return ASM_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *asm_error_string(int code)
{
    switch (code) {
    case ASM_OK: return "ok";
    case ASM_ERR_SHAPE: return "inconsistent sizes or block partition";
    case ASM_ERR_NOT_SPD: return "covariance is not symmetric positive definite";
    case ASM_ERR_NONFINITE: return "non-finite input";
    case ASM_ERR_IMPROPER: return "improper zero mode: f >= 0 does not bound a flat direction";
    case ASM_ERR_CUDA: return "CUDA, cuBLAS or cuSOLVER call failed";
    case ASM_ERR_STATE: return "call out of order";
    case ASM_ERR_ARG: return "invalid argument";
    case ASM_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case ASM_ERR_TOO_LARGE: return "size exceeds a compiled limit (register tile or static scratch)";
    case ASM_ERR_TIMEOUT: return "a bounded device wait gave up; results of that run are invalid";
    default: return "unknown error";
    }
}

int asm_setup(const asm_desc *ds, asm_problem **out)
{
    if (!ds || !out) return ASM_ERR_ARG;
    *out = nullptr;
    const int M = ds->M, N = ds->N;
    if (M < 1 || N < 1 || ds->n_levels < 1 || !ds->level_nblocks || !ds->block_start) return ASM_ERR_SHAPE;
    const bool given = ds->Kt && ds->gt && ds->d && ds->V && ds->U;
    if (!given && (!ds->K || !ds->G || !ds->C)) return ASM_ERR_ARG;
    // from here on every failure path releases what the handle holds with asm_destroy
    asm_problem *p = new (std::nothrow) asm_problem;
    if (!p) return ASM_ERR_ARG;
    p->M = M;
    p->N = N;
    p->n_levels = ds->n_levels;
    int nb = 0;
    for (int l = 0; l < ds->n_levels; ++l) {
        if (ds->level_nblocks[l] < 1) { asm_destroy(p); return ASM_ERR_SHAPE; }
        p->level_first.push_back(nb);
        p->level_nblocks.push_back(ds->level_nblocks[l]);
        nb += ds->level_nblocks[l];
    }
    p->n_blocks = nb;
    long long oV = 0, oR = 0, od = 0, oU = 0, oRec = 0, oUs = 0;
    for (int l = 0; l < ds->n_levels; ++l) {
        const int *st = ds->block_start + p->level_first[l];
        for (int b = 0; b < ds->level_nblocks[l]; ++b) {
            const int s0 = st[b], s1 = b + 1 < ds->level_nblocks[l] ? st[b + 1] : N;
            if ((b == 0 && s0 != 0) || s1 <= s0 || s1 > N) { asm_destroy(p); return ASM_ERR_SHAPE; }
            BlockDesc B{};
            B.start = s0;
            B.n = s1 - s0;
            B.np = std::min(M, B.n);
            B.rs = round_up_int(B.n, kRowAlign);
            B.offV = oV; oV += (long long)B.n * B.rs;
            B.offR = oR; oR += (long long)(B.n + 1) * B.rs;
            B.offd = od; od += B.n;
            B.offU = oU; oU += (long long)B.np * M;
            B.usr = M | 1;
            B.offUs = oUs; oUs += ((long long)B.np * B.usr + 3) / 4 * 4;   // 16-byte aligned in both precisions
            B.recstride = 2 * B.rs + 16;   // elements; 16 holds the mode data in both precisions
            B.offRec = oRec; oRec += (long long)B.n * B.recstride;
            p->max_rec = std::max(p->max_rec, B.recstride);
            p->blocks.push_back(B);
            p->max_nb = std::max(p->max_nb, B.n);
            p->max_np = std::max(p->max_np, B.np);
        }
    }
    p->totV = oV; p->totR = oR; p->totd = od; p->totU = oU; p->totRec = oRec; p->totUs = oUs;
    p->w.assign(N, 1.0);
    if (ds->w) {
        if (!all_finite(ds->w, N)) { asm_destroy(p); return ASM_ERR_NONFINITE; }
        for (int i = 0; i < N; ++i) p->w[i] = ds->w[i];
    }

    if (ds->flags & ~ASM_FLAG_TEST_STALL) { asm_destroy(p); return ASM_ERR_ARG; }
    p->test_stall = (ds->flags & ASM_FLAG_TEST_STALL) != 0;
    if (ds->P < 0 || (ds->P > 0 && (!ds->dK_dtheta || !ds->dw_dtheta))) { asm_destroy(p); return ASM_ERR_ARG; }
    p->P = ds->P;
    if (p->P > 0 && (!all_finite(ds->dK_dtheta, (size_t)p->P * M * N) || !all_finite(ds->dw_dtheta, (size_t)p->P * N))) {
        asm_destroy(p);
        return ASM_ERR_NONFINITE;
    }
    // gamma prior (Eq. compat): shapes a_n >= 1; all 1 is the flat measure
    std::vector<double> prior_am1;
    if (ds->prior_shape) {
        bool any = false;
        for (int n = 0; n < N; ++n) {
            const double a = ds->prior_shape[n];
            if (!std::isfinite(a)) { asm_destroy(p); return ASM_ERR_NONFINITE; }
            if (!(a >= 1.0)) { asm_destroy(p); return ASM_ERR_ARG; }
            any = any || a != 1.0;
        }
        if (any) {
            prior_am1.resize(N);
            for (int n = 0; n < N; ++n) prior_am1[n] = ds->prior_shape[n] - 1.0;
        }
    }
    HostFactors hf;
    int rc = ASM_OK;
    if (given) {
        if (!all_finite(ds->Kt, (size_t)M * N) || !all_finite(ds->gt, M)) { asm_destroy(p); return ASM_ERR_NONFINITE; }
        hf.Kt.assign(ds->Kt, ds->Kt + (size_t)M * N);
        hf.gt.assign(ds->gt, ds->gt + M);
        const double *dd = ds->d, *dv = ds->V, *du = ds->U;
        hf.d.resize(nb); hf.V.resize(nb); hf.U.resize(nb);
        for (int b = 0; b < nb; ++b) {
            const BlockDesc &B = p->blocks[b];
            hf.d[b].assign(dd, dd + B.n); dd += B.n;
            hf.V[b].assign(dv, dv + (size_t)B.n * B.n); dv += (size_t)B.n * B.n;
            hf.U[b].assign(du, du + (size_t)B.np * M); du += (size_t)B.np * M;
        }
    } else {
        if (!all_finite(ds->K, (size_t)M * N) || !all_finite(ds->G, M) || !all_finite(ds->C, (size_t)M * M)) {
            asm_destroy(p);
            return ASM_ERR_NONFINITE;
        }
        rc = device_factorize(ds, p, hf, &p->d_L);
        if (rc != ASM_OK) { asm_destroy(p); return rc; }
    }
    complete_residual_update(p, hf);
    if (given && ds->C) {
        if (!all_finite(ds->C, (size_t)M * M)) { asm_destroy(p); return ASM_ERR_NONFINITE; }
        rc = device_cholesky(ds->C, M, &p->d_L);
        if (rc != ASM_OK) { asm_destroy(p); return rc; }
    }
    if (p->P > 0) {
        if (!p->d_L) { asm_destroy(p); return ASM_ERR_ARG; }   // theta-gradients need C
        rc = whiten_dK(p, ds->dK_dtheta);
        if (rc != ASM_OK) { asm_destroy(p); return rc; }
    }
    {
        std::vector<double> dwv(ds->P > 0 ? ds->dw_dtheta : nullptr,
                                ds->P > 0 ? ds->dw_dtheta + (size_t)ds->P * N : nullptr);
        if (dwv.empty()) dwv.assign(1, 0.0);
        if ((rc = upload((void **)&p->d_w, p->w)) || (rc = upload((void **)&p->d_dw, dwv)) ||
            cudaMalloc(&p->d_vjp, sizeof(double) * (3 * (size_t)N + M + std::max(p->P, 1))) != cudaSuccess) {
            asm_destroy(p);
            return rc ? rc : ASM_ERR_CUDA;
        }
    }
    // properness: every zero mode must change sign (both bounds finite)
    for (int b = 0; b < nb; ++b) {
        const BlockDesc &B = p->blocks[b];
        for (int j = 0; j < B.n; ++j) {
            if (hf.d[b][j] > 0.0) continue;
            const double *v = &hf.V[b][(size_t)j * B.n];
            double vmax = 0.0;
            for (int i = 0; i < B.n; ++i) vmax = std::max(vmax, std::fabs(v[i]));
            bool pos = false, neg = false;
            for (int i = 0; i < B.n; ++i) {
                if (std::fabs(v[i]) < 0x1p-40 * vmax) continue;
                pos |= v[i] > 0.0;
                neg |= v[i] < 0.0;
            }
            if (!(pos && neg)) { asm_destroy(p); return ASM_ERR_IMPROPER; }
        }
    }
    // starting scale: s* = argmin_{s >= 0} |g~ - s K~ 1|^2 (flat default model)
    {
        double num = 0.0, den = 0.0;
        for (int i = 0; i < M; ++i) {
            double k = 0.0;
            for (int j = 0; j < N; ++j) k += hf.Kt[(size_t)i * N + j];
            num += k * hf.gt[i];
            den += k * k;
        }
        double s = den > 0.0 ? num / den : 0.0;
        if (!(s > 0.0) || !std::isfinite(s)) s = 1.0 / N;
        p->f0 = s;
    }
    std::vector<double> KtT((size_t)N * M);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < N; ++j) KtT[(size_t)j * M + i] = hf.Kt[(size_t)i * N + j];
    std::vector<int> lf(p->level_first), ln(p->level_nblocks);
    if ((rc = upload((void **)&p->d_KtT, KtT)) || (rc = upload((void **)&p->d_gt, hf.gt)) ||
        (rc = upload((void **)&p->d_level_first, lf)) || (rc = upload((void **)&p->d_level_nblocks, ln)) ||
        (rc = upload((void **)&p->d_blocks, p->blocks)) || (rc = build_precision<double>(p, hf, p->b64)) ||
        (rc = build_precision<float>(p, hf, p->b32))) {
        asm_destroy(p);
        return rc;
    }
    if (!prior_am1.empty()) {
        std::vector<float> am32(prior_am1.begin(), prior_am1.end());
        if ((rc = upload(&p->b64.prior_am1, prior_am1)) || (rc = upload(&p->b32.prior_am1, am32))) {
            asm_destroy(p);
            return rc;
        }
    }
    // K~ in TF32 high/low parts for the tensor-core refresh
    p->ldK = round_up_int(N, kRefreshTcLdK);
    const size_t nk = (size_t)M * p->ldK;
    if (cudaMalloc((void **)&p->d_Khi, nk * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&p->d_Klo, nk * sizeof(float)) != cudaSuccess ||
        launch_split_k(p->d_KtT, M, N, p->ldK, p->d_Khi, p->d_Klo, nullptr) != cudaSuccess ||
        cudaStreamSynchronize(nullptr) != cudaSuccess) {
        asm_destroy(p);
        return ASM_ERR_CUDA;
    }
    const char *team = std::getenv("ASM_TEAM_LANES");
    if (team) {
        const int t = std::atoi(team);
        if (t == 8 || t == 16 || t == 32) p->team = t;
    }
    *out = p;
    return ASM_OK;
}

size_t asm_workspace_bytes(const asm_problem *p, int chains, int precision)
{
    if (!p || chains < 1 || (precision != ASM_FP64 && precision != ASM_MIXED)) return 0;
    return run_layout(p, chains, precision).total;
}

int asm_partition_hierarchy(int N, int *n_levels, int *level_nblocks, int *block_start, int *total_blocks)
{
    if (N < 1 || !n_levels || !level_nblocks || !total_blocks) return ASM_ERR_ARG;
    std::vector<std::vector<int>> levels;
    levels.push_back({0});   // the whole grid: modes sampling
    int depth = 0;
    while ((1LL << depth) < N) ++depth;   // ceil(log2 N)
    for (int l = 1; l < depth; ++l) {
        const double w = (double)N / (double)(1LL << l);
        const double shift = (l % 2 == 0) ? 0.5 * w : 0.0;   // every other level, half a block
        std::vector<int> starts{0};
        for (long long k = 0;; ++k) {
            const double x = (double)k * w + shift;
            if (x >= (double)N) break;
            const int b = (int)std::floor(x + 0.5);
            if (b > starts.back() && b < N) starts.push_back(b);
        }
        if (starts != levels.back()) levels.push_back(starts);
    }
    if (N > 1) {   // one grid point per block: components sampling
        std::vector<int> starts(N);
        for (int n = 0; n < N; ++n) starts[n] = n;
        if (starts != levels.back()) levels.push_back(starts);
    }
    long long total = 0;
    for (const auto &l : levels) total += (long long)l.size();
    *n_levels = (int)levels.size();
    *total_blocks = (int)total;
    for (size_t l = 0; l < levels.size(); ++l) level_nblocks[l] = (int)levels[l].size();
    if (block_start) {
        long long o = 0;
        for (const auto &l : levels)
            for (int b : l) block_start[o++] = b;
    }
    return ASM_OK;
}

int asm_problem_count(const asm_problem *p)
{
    if (!p) return ASM_ERR_ARG;
    return p->kids.empty() ? 1 : (int)p->kids.size();
}

namespace {
// Point every problem of handle p at its section of the caller's workspace.
void bind_workspace(asm_problem *p, void *ws_all, size_t bytes, const RunLayout &RL, cudaStream_t stream)
{
    p->ws_all = ws_all;
    p->ws_bytes = bytes;
    p->stream = stream;
    const auto us = units_of(p);
    for (size_t k = 0; k < us.size(); ++k) {
        us[k]->ws_all = ws_all;
        us[k]->ws = (char *)ws_all + RL.unit[k];
        us[k]->ws_bytes = bytes;
        us[k]->stream = stream;
    }
}

// Fresh chains for every problem of handle p.
int start_chains(asm_problem *p, int chains, int precision, uint64_t seed, bool moments)
{
    const auto us = units_of(p);
    const bool batch = !p->kids.empty();
    p->moments = moments;
    p->chains = chains;
    p->precision = precision;
    p->seed = seed;
    p->problem_id = p->next_problem_id;
    p->chain_offset = p->next_chain_offset;
    p->sweeps_done = 0;
    p->kept = 0;
    p->sweep_launches = p->other_launches = p->timed_launches = 0;
    p->graph_replays = 0;
    p->tc_refreshes = 0;
    p->timed_ms = 0.0;
    for (size_t k = 0; k < us.size(); ++k) {
        asm_problem *u = us[k];
        if (batch) {
            u->moments = false;
            u->chains = chains;
            u->precision = precision;
            u->seed = seed;
            u->problem_id = p->problem_id + (unsigned long long)k;   // batch problem k: problem id P + k
            u->chain_offset = p->chain_offset;
            u->sweeps_done = 0;
            u->kept = 0;
            u->sweep_launches = u->other_launches = u->timed_launches = 0;
        }
        const WsLayout L = ws_layout(u, chains, precision);
        const int rc = precision == ASM_FP64 ? init_chains<double>(u, L, chains) : init_chains<float>(u, L, chains);
        if (rc != ASM_OK) return rc;
        u->have_run = true;
    }
    p->have_run = true;
    return ASM_OK;
}

// Sums the device counters of every problem of handle p (synchronises).
int read_counters_all(asm_problem *p, Counters *c)
{
    *c = Counters{};
    for (asm_problem *u : units_of(p)) {
        Counters cu{};
        if (cudaMemcpyAsync(&cu, u->ws, sizeof(cu), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
            cudaStreamSynchronize(p->stream) != cudaSuccess)
            return ASM_ERR_CUDA;
        c->degenerate += cu.degenerate;
        c->zero_mode += cu.zero_mode;
        c->tail_capped += cu.tail_capped;
        c->nonfinite += cu.nonfinite;
        c->timeouts += cu.timeouts;
        c->prior_rejections += cu.prior_rejections;
        c->drift_bits = std::max(c->drift_bits, cu.drift_bits);   // non-negative doubles order like their bits
    }
    return ASM_OK;
}

void finish_sweeps(asm_problem *p, long long s1, long long kept_add)
{
    p->sweeps_done = s1;
    p->kept += kept_add;
    if (!p->kids.empty())
        for (asm_problem *u : p->kids) {
            u->sweeps_done = s1;
            u->kept += kept_add;
        }
}
}  // namespace

int asm_sample(asm_problem *p, int chains, long burn_in, long sweeps, uint64_t seed, int precision,
               uint32_t flags, void *d_workspace, size_t workspace_bytes, void *stream)
{
    if (!p || chains < 1 || burn_in < 0 || sweeps < 0) return ASM_ERR_ARG;
    if (precision != ASM_FP64 && precision != ASM_MIXED) return ASM_ERR_ARG;
    if (flags & ~(ASM_SAMPLE_CONTINUE | ASM_SAMPLE_TIMING | ASM_SAMPLE_MOMENTS | ASM_SAMPLE_REFRESH_FP64 |
                  ASM_SAMPLE_STEP_TRACE))
        return ASM_ERR_ARG;
    const bool moments = (flags & ASM_SAMPLE_MOMENTS) != 0;
    if (moments && !p->kids.empty()) return ASM_ERR_ARG;   // backward moments: single problems
    const RunLayout RL = run_layout(p, chains, precision);
    if (!d_workspace || workspace_bytes < RL.total || ((uintptr_t)d_workspace & 255)) return ASM_ERR_WORKSPACE;
    const bool cont = (flags & ASM_SAMPLE_CONTINUE) != 0;
    if (cont && (!p->have_run || p->chains != chains || p->precision != precision || p->ws_all != d_workspace ||
                 p->seed != seed))
        return ASM_ERR_STATE;
    if (p->ev_used && drain_events(p) != ASM_OK) return ASM_ERR_CUDA;
    bind_workspace(p, d_workspace, workspace_bytes, RL, (cudaStream_t)stream);
    p->timing = (flags & ASM_SAMPLE_TIMING) != 0;
    p->refresh_fp64 = (flags & ASM_SAMPLE_REFRESH_FP64) != 0;
    p->trace = (flags & ASM_SAMPLE_STEP_TRACE) != 0;
    for (asm_problem *u : p->kids) u->trace = p->trace;
    int rc;
    if (!cont) {
        rc = start_chains(p, chains, precision, seed, moments);
        if (rc != ASM_OK) return rc;
    }
    const long long s0 = p->sweeps_done, s1 = s0 + burn_in + sweeps;
    if (cont && burn_in > 0 && precision == ASM_MIXED && s0 % kBinSweeps != 0) {
        // a new burn-in inside an open 64-sweep block: its earlier kept sweeps go to the FP64 sums now
        for (asm_problem *u : units_of(p)) {
            const WsLayout L = ws_layout(u, chains, precision);
            char *ws = (char *)u->ws;
            const long long tot = (long long)chains * u->N;
            fold_open_block_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, p->stream>>>(
                (float *)(ws + L.P1), (float *)(ws + L.P2), L.ldF, (double *)(ws + L.S1), (double *)(ws + L.S2),
                chains, u->N);
            ++u->other_launches;
        }
        if (cudaGetLastError() != cudaSuccess) return ASM_ERR_CUDA;
    }
    // first sweep of the unbroken run of kept sweeps: a continuation without burn-in
    // extends the previous one (bins may straddle the calls)
    long long burn_abs = s0 + burn_in;
    if (cont && burn_in == 0) burn_abs = std::min(burn_abs, p->kept_since);
    p->kept_since = burn_abs;
    rc = precision == ASM_FP64 ? run_all<double>(p, chains, s0, s1, burn_abs)
                               : run_all<float>(p, chains, s0, s1, burn_abs);
    if (rc != ASM_OK) return rc;
    finish_sweeps(p, s1, sweeps);
    return ASM_OK;
}

int asm_tune(asm_problem *p, int chains, int precision, void *d_workspace, size_t workspace_bytes, void *stream,
             int *team_out, int *consumers_out, int *min_blocks_out)
{
    if (!p || chains < 1 || (precision != ASM_FP64 && precision != ASM_MIXED)) return ASM_ERR_ARG;
    const RunLayout RL = run_layout(p, chains, precision);
    if (!d_workspace || workspace_bytes < RL.total || ((uintptr_t)d_workspace & 255)) return ASM_ERR_WORKSPACE;
    if (p->ev_used && drain_events(p) != ASM_OK) return ASM_ERR_CUDA;
    bind_workspace(p, d_workspace, workspace_bytes, RL, (cudaStream_t)stream);
    const int team0 = p->team, cons0 = p->tuned_consumers, minb0 = p->tuned_minb;
    const bool timing0 = p->timing;
    p->timing = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return ASM_ERR_CUDA;
    }
    int best_team = team0, best_cons = cons0, best_minb = minb0, rc = ASM_OK;
    float best = 0.f;
    bool any = false;
    const int teams[] = {32, 16, 8};
    const int conss[] = {0, 2, 3, 4, 5, 6, 7};   // 0: the built-in heuristic
    for (int trial = 0; trial < 3 * 7 * 2; ++trial) {
        const int S = teams[trial / 14], c = conss[(trial / 2) % 7], mb = 1 + trial % 2;
        {
            p->team = S;
            p->tuned_consumers = c;
            p->tuned_minb = mb;
            // fresh chains, one sweep to warm up, then the timed sweeps
            rc = start_chains(p, chains, precision, 0x74756e65ull, false);
            if (rc != ASM_OK) break;
            int r = precision == ASM_FP64 ? run_all<double>(p, chains, 0, 1, 0) : run_all<float>(p, chains, 0, 1, 0);
            if (r == ASM_ERR_TOO_LARGE) continue;   // this shape does not fit the problems
            if (r != ASM_OK) { rc = r; break; }
            if (cudaEventRecord(e0, p->stream) != cudaSuccess) { rc = ASM_ERR_CUDA; break; }
            r = precision == ASM_FP64 ? run_all<double>(p, chains, 1, 4, 0) : run_all<float>(p, chains, 1, 4, 0);
            if (r != ASM_OK) { rc = r; break; }
            float ms = 0.f;
            if (cudaEventRecord(e1, p->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = ASM_ERR_CUDA;
                break;
            }
            Counters c0{};
            if (read_counters_all(p, &c0) != ASM_OK) { rc = ASM_ERR_CUDA; break; }
            if (c0.timeouts) { rc = ASM_ERR_TIMEOUT; break; }
            if (!any || ms < best) {
                best = ms;
                best_team = S;
                best_cons = c;
                best_minb = mb;
                any = true;
            }
        }
        if (rc != ASM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->timing = timing0;
    // the workspace now holds trial chains: the next asm_sample starts afresh
    p->have_run = false;
    for (asm_problem *u : p->kids) u->have_run = false;
    if (rc != ASM_OK || !any) {
        p->team = team0;
        p->tuned_consumers = cons0;
        p->tuned_minb = minb0;
        return rc != ASM_OK ? rc : ASM_ERR_TOO_LARGE;
    }
    p->team = best_team;
    p->tuned_consumers = best_cons;
    p->tuned_minb = best_minb;
    if (team_out) *team_out = best_team;
    if (consumers_out) *consumers_out = best_cons;
    if (min_blocks_out) *min_blocks_out = best_minb;
    return ASM_OK;
}

namespace {
// Reads the run's device counters (synchronises the stream).
int read_counters(asm_problem *p, Counters *c)
{
    if (cudaMemcpyAsync(c, p->ws, sizeof(*c), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
        return ASM_ERR_CUDA;
    return ASM_OK;
}
}  // namespace

int asm_average_at(asm_problem *p, int k, double *mean_A, double *sem_A, double *ess, double *mean_fbar)
{
    if (!p || k < 0 || k >= asm_problem_count(p)) return ASM_ERR_ARG;
    if (p->kids.empty()) return asm_average(p, mean_A, sem_A, ess, mean_fbar);
    return asm_average(p->kids[(size_t)k], mean_A, sem_A, ess, mean_fbar);
}

int asm_average(asm_problem *p, double *mean_A, double *sem_A, double *ess, double *mean_fbar)
{
    if (!p) return ASM_ERR_ARG;
    if (!p->kids.empty()) return ASM_ERR_ARG;   // a batch: asm_average_at
    if (!p->have_run || p->kept < 1) return ASM_ERR_STATE;
    {
        Counters c{};
        const int rc0 = read_counters(p, &c);
        if (rc0 != ASM_OK) return rc0;
        if (c.timeouts) return ASM_ERR_TIMEOUT;
    }
    const WsLayout L = ws_layout(p, p->chains, p->precision);
    const int N = p->N;
    double *d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * 3 * N) != cudaSuccess) return ASM_ERR_CUDA;
    char *ws = (char *)p->ws;
    ++p->other_launches;
    const bool open32 = p->precision != ASM_FP64;   // FP32 state: sums of the open 64-sweep block
    reduce_kernel<<<(N + 127) / 128, 128, 0, p->stream>>>(
        (const double *)(ws + L.S1), (const double *)(ws + L.S2), open32 ? (const float *)(ws + L.P1) : nullptr,
        open32 ? (const float *)(ws + L.P2) : nullptr, L.ldF, p->chains, N, (double)p->kept, d, d + N, d + 2 * N);
    std::vector<double> h((size_t)3 * N);
    int rc = ASM_OK;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h.data(), d, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
        rc = ASM_ERR_CUDA;
    cudaFree(d);
    if (rc != ASM_OK) return rc;
    for (int n = 0; n < N; ++n) {
        const double mu = h[n], s2 = h[N + n], m2 = h[2 * N + n];
        const double var = std::max(m2 - mu * mu, 0.0);
        if (mean_fbar) mean_fbar[n] = mu;
        if (mean_A) mean_A[n] = mu / p->w[n];
        if (sem_A) sem_A[n] = std::sqrt(s2) / p->w[n];
        if (ess) ess[n] = s2 > 0.0 ? var / s2 : NAN;
    }
    return ASM_OK;
}

int asm_mc_error(asm_problem *p, int k, double *ess, double *sem_fbar, double *sigma2_levels, int *bins_per_chain)
{
    static_assert(kBinSweeps == kRefreshPeriod, "bins close at refresh boundaries");
    if (!p || k < 0 || k >= asm_problem_count(p)) return ASM_ERR_ARG;
    asm_problem *u = p->kids.empty() ? p : p->kids[(size_t)k];
    if (!p->have_run || !u->have_run || u->kept < 1) return ASM_ERR_STATE;
    {
        Counters c{};
        if (read_counters_all(p, &c) != ASM_OK) return ASM_ERR_CUDA;
        if (c.timeouts) return ASM_ERR_TIMEOUT;
    }
    const WsLayout L = ws_layout(u, u->chains, u->precision);
    const int N = u->N, chains = u->chains;
    const size_t nk = (size_t)kBinLevels * N;
    double *d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * (3 * (size_t)N + 2 * nk)) != cudaSuccess) return ASM_ERR_CUDA;
    const char *ws = (const char *)u->ws;
    const bool open32 = u->precision != ASM_FP64;
    reduce_kernel<<<(N + 127) / 128, 128, 0, p->stream>>>(
        (const double *)(ws + L.S1), (const double *)(ws + L.S2), open32 ? (const float *)(ws + L.P1) : nullptr,
        open32 ? (const float *)(ws + L.P2) : nullptr, L.ldF, chains, N, (double)u->kept, d, d + N, d + 2 * N);
    bin_reduce_kernel<<<(unsigned)((nk + 127) / 128), 128, 0, p->stream>>>(
        (const double *)(ws + L.bacc1), (const double *)(ws + L.bacc2), chains, N, d + 3 * N);
    p->other_launches += 2;
    std::vector<double> h(3 * (size_t)N + 2 * nk);
    int nb = 0;
    int rc = ASM_OK;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h.data(), d, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(&nb, ws + L.bcount, sizeof(int), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
        rc = ASM_ERR_CUDA;
    cudaFree(d);
    if (rc != ASM_OK) return rc;
    const double *A1 = h.data() + 3 * N, *A2 = A1 + nk;
    for (int l = 0; l < kBinLevels; ++l)
        if (bins_per_chain) bins_per_chain[l] = nb >> l;
    for (int n = 0; n < N; ++n) {
        const double mu = h[n], s2 = h[N + n], m2 = h[2 * N + n];
        const double var = std::max(m2 - mu * mu, 0.0);
        double best = s2;   // the spread of the chain means
        for (int l = 0; l < kBinLevels; ++l) {
            const long long c = nb >> l;                      // level-l bins per chain
            const double cnt = (double)c * chains;            // level-l bins in all
            double sig2 = NAN;
            if (cnt > 1.0) {
                const double m = A1[(size_t)l * N + n] / cnt;
                const double v = std::max(A2[(size_t)l * N + n] / cnt - m * m, 0.0) * cnt / (cnt - 1.0);
                sig2 = v / cnt;
                if (c >= 2) best = std::max(best, sig2);
            }
            if (sigma2_levels) sigma2_levels[(size_t)l * N + n] = sig2;
        }
        if (sem_fbar) sem_fbar[n] = std::sqrt(best);
        if (ess) ess[n] = best > 0.0 ? var / best : NAN;
    }
    return ASM_OK;
}

int asm_backward(asm_problem *p, const double *v, double *grad_G, double *grad_theta)
{
    if (!p || !v) return ASM_ERR_ARG;
    if (!p->kids.empty()) return ASM_ERR_ARG;
    if (!p->have_run || !p->moments || p->nsnap < 2) return ASM_ERR_STATE;
    if (grad_G && !p->d_L) return ASM_ERR_STATE;
    if (grad_theta && p->P == 0) return ASM_ERR_ARG;
    Counters c{};
    int rc = read_counters(p, &c);
    if (rc != ASM_OK) return rc;
    if (c.timeouts) return ASM_ERR_TIMEOUT;
    const int N = p->N, M = p->M;
    const WsLayout L = ws_layout(p, p->chains, p->precision);
    const char *ws = (const char *)p->ws;
    std::vector<double> hv(2 * (size_t)N);
    for (int n = 0; n < N; ++n) {
        hv[n] = v[n] / p->w[n];   // cotangent of fbar
        hv[N + n] = v[n];
    }
    double *d_vp = p->d_vjp, *d_v = p->d_vjp + N, *d_u = p->d_vjp + 2 * N, *d_y = p->d_vjp + 3 * N,
           *d_g = p->d_vjp + 3 * N + M;
    const double ns = (double)p->nsnap;
    if (cudaMemcpyAsync(d_vp, hv.data(), sizeof(double) * 2 * N, cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
        return ASM_ERR_CUDA;
    if (grad_G) {
        vjp_cov_kernel<<<(N + 127) / 128, 128, 0, p->stream>>>((const double *)(ws + L.Sff),
                                                               (const double *)(ws + L.Sf), ns, d_vp, N, d_u);
        // C^{-1} K u = L^{-T} (K~ u): hand-written product and triangular solve
        if (cudaGetLastError() != cudaSuccess || launch_vjp_G(p->d_KtT, p->d_L, d_u, M, N, d_y, p->stream) != cudaSuccess ||
            cudaMemcpyAsync(grad_G, d_y, sizeof(double) * M, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess)
            return ASM_ERR_CUDA;
    }
    if (grad_theta) {
        vjp_theta_kernel<<<(p->P + 31) / 32, 32, 0, p->stream>>>(
            (const double *)(ws + L.Sfs), (const double *)(ws + L.Ss), (const double *)(ws + L.Sf),
            (const double *)(ws + L.shift), ns, d_vp, d_v, p->d_w, p->d_dw, N, p->P, d_g);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(grad_theta, d_g, sizeof(double) * p->P, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess)
            return ASM_ERR_CUDA;
    }
    return cudaStreamSynchronize(p->stream) == cudaSuccess ? ASM_OK : ASM_ERR_CUDA;
}

int asm_chain_state(asm_problem *p, double *f, double *chi2)
{
    if (!p) return ASM_ERR_ARG;
    if (!p->kids.empty()) return ASM_ERR_ARG;
    if (!p->have_run) return ASM_ERR_STATE;
    {
        Counters c{};
        const int rc0 = read_counters(p, &c);
        if (rc0 != ASM_OK) return rc0;
        if (c.timeouts) return ASM_ERR_TIMEOUT;
    }
    const WsLayout L = ws_layout(p, p->chains, p->precision);
    const size_t es = p->precision == ASM_FP64 ? 8 : 4;
    const char *ws = (const char *)p->ws;
    std::vector<unsigned char> hF((size_t)p->chains * L.ldF * es), hR((size_t)p->chains * L.ldR * es);
    if (cudaMemcpyAsync(hF.data(), ws + L.F, hF.size(), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(hR.data(), ws + L.R, hR.size(), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
        return ASM_ERR_CUDA;
    for (int q = 0; q < p->chains; ++q) {
        if (f)
            for (int n = 0; n < p->N; ++n) {
                const size_t i = (size_t)q * L.ldF + n;
                f[(size_t)q * p->N + n] = es == 8 ? ((const double *)hF.data())[i] : ((const float *)hF.data())[i];
            }
        if (chi2) {
            double s = 0.0;
            for (int m = 0; m < p->M; ++m) {
                const size_t i = (size_t)q * L.ldR + m;
                const double r = es == 8 ? ((const double *)hR.data())[i] : ((const float *)hR.data())[i];
                s += r * r;
            }
            chi2[q] = s;
        }
    }
    return ASM_OK;
}

int asm_status(asm_problem *p, asm_stats *out)
{
    if (!p || !out) return ASM_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    if (!p->have_run) return ASM_ERR_STATE;
    if (drain_events(p) != ASM_OK) return ASM_ERR_CUDA;
    Counters c{};
    if (read_counters_all(p, &c) != ASM_OK) return ASM_ERR_CUDA;
    out->chains = p->chains;
    out->sweeps_done = p->sweeps_done;
    out->kept_sweeps = p->kept;
    out->precision = p->precision;
    out->degenerate_moves = (int64_t)c.degenerate;
    out->zero_mode_moves = (int64_t)c.zero_mode;
    out->tail_capped = (int64_t)c.tail_capped;
    out->nonfinite_moves = (int64_t)c.nonfinite;
    double drift;
    std::memcpy(&drift, &c.drift_bits, sizeof(drift));
    out->max_resync_drift = drift;
    out->sweep_launches = p->sweep_launches;
    out->other_launches = p->other_launches;
    if (!p->kids.empty())
        for (asm_problem *u : p->kids) out->other_launches += u->other_launches;
    out->timed_launches = p->timed_launches;
    out->sweep_kernel_ms = p->timed_ms;
    out->timeouts = (int64_t)c.timeouts;
    out->prior_rejections = (int64_t)c.prior_rejections;
    out->graph_replays = p->graph_replays;
    out->tc_refreshes = p->tc_refreshes;
    out->team_lanes = p->last_team;
    out->consumers_per_cta = p->last_consumers;
    out->ctas = p->last_ctas;
    out->work_items = p->last_items;
    out->min_blocks = p->last_minb;
    return ASM_OK;
}

int asm_sample_noalloc(asm_problem *p, int chains, long burn_in, long sweeps, uint64_t seed,
                       int precision, double *d_mean_fbar, double *d_sem2_fbar, double *d_m2_fbar,
                       void *stream)
{
    if (!p || chains < 1 || burn_in < 0 || sweeps < 1 || !d_mean_fbar || !d_sem2_fbar || !d_m2_fbar)
        return ASM_ERR_ARG;
    if (precision != ASM_FP64 && precision != ASM_MIXED) return ASM_ERR_ARG;
    if (!p->kids.empty()) return ASM_ERR_ARG;
    const RunLayout RL = run_layout(p, chains, precision);
    if (RL.total > ASM_NOALLOC_SCRATCH_BYTES) return ASM_ERR_TOO_LARGE;
    void *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != ASM_OK) return rc;
    if (p->ev_used && drain_events(p) != ASM_OK) return ASM_ERR_CUDA;
    bind_workspace(p, scratch, ASM_NOALLOC_SCRATCH_BYTES, RL, (cudaStream_t)stream);
    p->timing = false;
    p->refresh_fp64 = false;   // the mixed path refreshes on the tensor cores, whatever ran before
    p->trace = false;
    // counters, sums and residuals are zeroed and the chains re-started here
    rc = start_chains(p, chains, precision, seed, false);
    if (rc != ASM_OK) return rc;
    p->kept_since = burn_in;   // the kept run starts after this call's burn-in (checkpoints carry it)
    const long long s1 = (long long)burn_in + sweeps;
    p->no_graph = true;   // graph instantiation allocates
    rc = precision == ASM_FP64 ? run_all<double>(p, chains, 0, s1, burn_in) : run_all<float>(p, chains, 0, s1, burn_in);
    p->no_graph = false;
    if (rc != ASM_OK) return rc;
    finish_sweeps(p, s1, sweeps);
    const WsLayout L = ws_layout(p, chains, precision);
    const char *ws = (const char *)p->ws;
    const bool open32 = precision != ASM_FP64;
    reduce_kernel<<<(p->N + 127) / 128, 128, 0, p->stream>>>(
        (const double *)(ws + L.S1), (const double *)(ws + L.S2), open32 ? (const float *)(ws + L.P1) : nullptr,
        open32 ? (const float *)(ws + L.P2) : nullptr, L.ldF, chains, p->N, (double)sweeps, d_mean_fbar, d_sem2_fbar,
        d_m2_fbar);
    ++p->other_launches;
    return cudaGetLastError() == cudaSuccess ? ASM_OK : ASM_ERR_CUDA;
}

int asm_step_trace(asm_problem *p, int k, double *delta, int max_sweeps, int *n_sweeps)
{
    if (!p || !delta || !n_sweeps || max_sweeps < 0 || k < 0 || k >= asm_problem_count(p)) return ASM_ERR_ARG;
    asm_problem *u = p->kids.empty() ? p : p->kids[(size_t)k];
    if (!p->have_run || !u->have_run) return ASM_ERR_STATE;
    const int n = (int)std::min<long long>({u->sweeps_done, (long long)kStepTraceMax, (long long)max_sweeps});
    const WsLayout L = ws_layout(u, u->chains, u->precision);
    std::vector<double> h((size_t)std::max(n, 1));
    if (n > 0 && (cudaMemcpyAsync(h.data(), (const char *)u->ws + L.steptrace, sizeof(double) * n,
                                  cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
                  cudaStreamSynchronize(p->stream) != cudaSuccess))
        return ASM_ERR_CUDA;
    for (int s = 0; s < n; ++s) delta[s] = h[s] / u->chains;
    *n_sweeps = n;
    return ASM_OK;
}

int asm_set_stream_ids(asm_problem *p, uint64_t problem_id, uint64_t chain_offset)
{
    if (!p) return ASM_ERR_ARG;
    p->next_problem_id = problem_id;
    p->next_chain_offset = chain_offset;
    return ASM_OK;
}

namespace {
struct CheckpointHeader {
    uint64_t magic, version;
    int64_t M, N, chains, precision;
    uint64_t seed, problem_id, chain_offset;
    int64_t sweeps_done, kept, ws_bytes;
    int64_t kept_since;   // first sweep of the unbroken kept run (binning of a continuation)
};
constexpr uint64_t kCheckpointVersion = 4;
constexpr uint64_t kCheckpointMagic = 0x41534d434b505431ull;   // "ASMCKPT1"
}  // namespace

int asm_checkpoint(asm_problem *p, void *host_buf, size_t *bytes)
{
    if (!p || !bytes || !p->kids.empty()) return ASM_ERR_ARG;
    if (!p->have_run) return ASM_ERR_STATE;
    const WsLayout L = ws_layout(p, p->chains, p->precision);
    const size_t need = sizeof(CheckpointHeader) + L.total;
    if (!host_buf) {
        *bytes = need;
        return ASM_OK;
    }
    if (*bytes < need) return ASM_ERR_ARG;
    CheckpointHeader h{kCheckpointMagic, kCheckpointVersion, p->M, p->N, p->chains, p->precision, p->seed,
                       p->problem_id, p->chain_offset, p->sweeps_done, p->kept, (int64_t)L.total, p->kept_since};
    std::memcpy(host_buf, &h, sizeof(h));
    if (cudaMemcpyAsync((char *)host_buf + sizeof(h), p->ws, L.total, cudaMemcpyDeviceToHost, p->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
        return ASM_ERR_CUDA;
    *bytes = need;
    return ASM_OK;
}

int asm_restore(asm_problem *p, const void *host_buf, size_t bytes, void *d_workspace, size_t workspace_bytes,
                void *stream)
{
    if (!p || !host_buf || bytes < sizeof(CheckpointHeader) || !p->kids.empty()) return ASM_ERR_ARG;
    CheckpointHeader h;
    std::memcpy(&h, host_buf, sizeof(h));
    if (h.magic != kCheckpointMagic || h.version != kCheckpointVersion) return ASM_ERR_ARG;
    if (h.M != p->M || h.N != p->N) return ASM_ERR_SHAPE;
    if (h.precision != ASM_FP64 && h.precision != ASM_MIXED) return ASM_ERR_ARG;
    const WsLayout L = ws_layout(p, (int)h.chains, (int)h.precision);
    const RunLayout RL = run_layout(p, (int)h.chains, (int)h.precision);
    if ((int64_t)L.total != h.ws_bytes || bytes < sizeof(h) + L.total) return ASM_ERR_ARG;
    if (!d_workspace || workspace_bytes < RL.total || ((uintptr_t)d_workspace & 255)) return ASM_ERR_WORKSPACE;
    if (p->ev_used && drain_events(p) != ASM_OK) return ASM_ERR_CUDA;
    bind_workspace(p, d_workspace, workspace_bytes, RL, (cudaStream_t)stream);
    if (cudaMemcpyAsync(p->ws, (const char *)host_buf + sizeof(h), L.total, cudaMemcpyHostToDevice,
                        p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
        return ASM_ERR_CUDA;
    p->chains = (int)h.chains;
    p->precision = (int)h.precision;
    p->seed = h.seed;
    p->problem_id = p->next_problem_id = h.problem_id;
    p->chain_offset = p->next_chain_offset = h.chain_offset;
    p->sweeps_done = h.sweeps_done;
    p->kept = h.kept;
    p->kept_since = h.kept_since;
    p->sweep_launches = p->other_launches = p->timed_launches = 0;
    p->timed_ms = 0.0;
    p->timing = false;
    p->have_run = true;
    return ASM_OK;
}

int asm_setup_batch(int n, const asm_desc *d, asm_problem **out)
{
    if (!out || !d || n < 1) return ASM_ERR_ARG;
    *out = nullptr;
    asm_problem *b = new (std::nothrow) asm_problem;
    if (!b) return ASM_ERR_ARG;
    for (int k = 0; k < n; ++k) {
        asm_problem *u = nullptr;
        const int rc = asm_setup(&d[k], &u);
        if (rc != ASM_OK) {
            asm_destroy(b);
            return rc;
        }
        b->kids.push_back(u);
        b->M = std::max(b->M, u->M);
        b->N = std::max(b->N, u->N);
    }
    b->team = b->kids[0]->team;
    *out = b;
    return ASM_OK;
}

void asm_destroy(asm_problem *p)
{
    if (!p) return;
    for (asm_problem *u : p->kids) asm_destroy(u);
    p->kids.clear();
    void *ptrs[] = {p->d_level_first, p->d_level_nblocks, p->d_blocks, p->d_KtT, p->d_gt, p->d_Khi, p->d_Klo, p->d_L,
                    p->d_Kth64, p->d_Kth32, p->d_w, p->d_dw, p->d_vjp};
    for (void *x : ptrs)
        if (x) cudaFree(x);
    free_prec(p->b64);
    free_prec(p->b32);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    drop_graph(p);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    delete p;
}

}  // extern "C"
