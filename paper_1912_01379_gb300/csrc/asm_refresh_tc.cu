// Residual refresh of the mixed-precision path on the 5th-generation tensor
// cores: R~ = 1 g~^T - F K~^T for all chains of every problem of a launch, the
// product in split precision (3xTF32: A_hi K_hi + A_hi K_lo + A_lo K_hi, FP32
// accumulation in tensor memory), the difference from g~, chi^2 = |r~|^2 and the
// resync drift in FP64.
//
// Centring.  g~ and K~ f are large against their difference r~ when the data
// are accurate (|g~| ~ 1e2 .. 1e5 against |r~| ~ sqrt(M)), so an FP32
// accumulation of K~ f would leave an error of 2^-24 |g~| in r~.  The product
// is therefore taken of the centred states A = f - fref, with fref the mean
// chain state of the problem at this refresh, and r~ = r_ref - K~ A with
// r_ref = g~ - K~ fref formed in FP64 once per refresh: K~ A is of the size of
// the posterior spread, and its FP32 accumulation error shrinks with it.  The
// difference f - fref is formed exactly in FP64 before the split into TF32
// high and low parts.
//
// Split.  Both parts are rounded to the nearest TF32 value here, so that the
// MMA, which reads 10 mantissa bits of each operand, takes them exactly: a
// high part off by at most 2^-11 of x and a low part off by at most 2^-11 of
// the remainder, i.e. 2^-22 of x.  Left to the MMA's truncation the low part
// would lose up to 2^-21 of x.  With the dropped A_lo K_lo term each product
// K~_mn A_n then carries at most about 3 2^-22 of its size.
//
// One CTA of 128 threads owns 128 chains of one problem (the MMA's M = 128
// rows, one TMEM lane per chain) and one part of its grid points, and loops over
// the problem's M_tau tiles (N of the MMA, <= 256 columns of FP32 accumulator)
// and over the part's k-tiles of 32 grid points.  The parts (refresh_tc_ksplit:
// enough CTAs to cover the GPU, a function of the problem alone) keep each FP32
// accumulation short; with more than one, each CTA stores its FP32 product and
// refresh_finish_kernel adds the parts in FP64 in part order, so the result does
// not depend on which CTA finishes first.  Each k-tile is staged by all
// threads into shared memory in the canonical K-major layout without swizzle
// (core matrices of 8 rows x 16 bytes), A split into TF32 high and low parts on
// the way; K~ comes split from set-up.  Two stages alternate: thread 0 issues the 12 tcgen05.mma of a
// stage and commits them to the stage's mbarrier, which the threads wait on
// before staging into it again.  Waits are bounded (timeouts are counted).
#include "asm_sweep.cuh"

namespace asmgb {
namespace {

constexpr int kTcRows = 128;       // chains per CTA (MMA M)
constexpr int kTcBK = 32;          // grid points per k-tile: 128 bytes of FP32 per row
constexpr int kTcThreads = 128;
constexpr int kTcCols = 256;       // TMEM columns held by a CTA (>= the widest M_tau tile)
constexpr int kTcAtile = kTcRows * kTcBK * 4;   // bytes of one A (F) part per stage

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading byte offset (between
// core matrices along K), stride byte offset (between 8-row groups), descriptor
// version 1, no swizzle.
__device__ __forceinline__ unsigned long long umma_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    unsigned long long d = (unsigned long long)((saddr >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of kind::tf32: D in FP32, A and B TF32, both K-major,
// M = 128, N = n.
__device__ __forceinline__ unsigned tf32_idesc(int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned idesc,
                                          unsigned accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16])
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Nearest TF32 (10 explicit mantissa bits) of a finite float.
__device__ __forceinline__ float tf32_round(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Stages rows [row0, row0 + nrows) x columns [k0, k0 + 32) of a row-major FP32
// matrix (leading dimension ld, a multiple of 4; rows >= rows_valid and columns
// >= cols_valid read as 0) into the layout [row/8][k/4][row%8][k%4].  With
// `lo` the TF32 high part goes to hi and the remainder, rounded to TF32, to lo.
__device__ __forceinline__ void stage_rows(const float *__restrict__ src, int ld, int rows_valid, int cols_valid,
                                           int row0, int k0, int nrows, unsigned char *hi, unsigned char *lo)
{
    const int n4 = nrows * (kTcBK / 4);
    for (int e = threadIdx.x; e < n4; e += kTcThreads) {
        const int r8 = e & 7, kc = (e >> 3) & 7, rg = e >> 6;
        const int row = row0 + rg * 8 + r8;
        const int col = k0 + kc * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < rows_valid && col < cols_valid) {
            v = __ldg(reinterpret_cast<const float4 *>(src + (size_t)row * ld + col));
            if (col + 1 >= cols_valid) v.y = 0.f;
            if (col + 2 >= cols_valid) v.z = 0.f;
            if (col + 3 >= cols_valid) v.w = 0.f;
        }
        const int off = (rg * 8 + kc) * 128 + r8 * 16;
        if (lo) {
            const float4 h = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
            *reinterpret_cast<float4 *>(hi + off) = h;
            *reinterpret_cast<float4 *>(lo + off) = make_float4(tf32_round(v.x - h.x), tf32_round(v.y - h.y),
                                                                tf32_round(v.z - h.z), tf32_round(v.w - h.w));
        } else {
            *reinterpret_cast<float4 *>(hi + off) = v;
        }
    }
}

// The same layout for the centred chain states: rows of f - fref, the
// difference exact in FP64, split into TF32 high and low parts.
__device__ __forceinline__ void stage_centred(const float *__restrict__ F, int ld, const float *__restrict__ fref,
                                              int rows_valid, int cols_valid, int row0, int k0, unsigned char *hi,
                                              unsigned char *lo)
{
    const int n4 = kTcRows * (kTcBK / 4);
    for (int e = threadIdx.x; e < n4; e += kTcThreads) {
        const int r8 = e & 7, kc = (e >> 3) & 7, rg = e >> 6;
        const int row = row0 + rg * 8 + r8;
        const int col = k0 + kc * 4;
        float x[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
        if (row < rows_valid && col < cols_valid) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(F + (size_t)row * ld + col));
            x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (col + j < cols_valid) c[j] = fref[col + j];
                else x[j] = 0.f;
            }
        }
        float h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double d = (double)x[j] - (double)c[j];
            h[j] = tf32_round((float)d);
            l[j] = tf32_round((float)(d - (double)h[j]));
        }
        const int off = (rg * 8 + kc) * 128 + r8 * 16;
        *reinterpret_cast<float4 *>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
}

// Reference state of the refresh, in two steps over the whole GPU.
// fref = mean of the chain states (FP32): CTA (x, problem) takes 32 grid points,
// lane l point 32 x + l (coalesced rows), warp w the chains q = w mod 8 in order;
// the eight partial sums are added in warp order.
__global__ void refresh_fref_kernel(const SweepParams<float> *__restrict__ probs, int chains)
{
    __shared__ float part[8][32];
    const SweepParams<float> &p = probs[blockIdx.y];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + lane;
    if (blockIdx.x * 32 >= p.N) return;   // (uniform per CTA)
    float a = 0.f;
    if (n < p.N)
        for (int q = w; q < chains; q += 8) a += p.F[(size_t)q * p.ldF + n];
    part[w][lane] = a;
    __syncthreads();
    if (w == 0 && n < p.N) {
        float t = part[0][lane];
        for (int k = 1; k < 8; ++k) t += part[k][lane];
        p.fref[n] = t * (1.0f / (float)chains);
    }
}

// r_ref = g~ - K~ fref in FP64, one thread per data point.
__global__ void refresh_rref_kernel(const SweepParams<float> *__restrict__ probs)
{
    const SweepParams<float> &p = probs[blockIdx.y];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= p.M) return;
    double a = p.gt[m];
    for (int n = 0; n < p.N; ++n) a -= p.KtT[(size_t)n * p.M + m] * (double)p.fref[n];
    p.rref[m] = a;
}

__global__ void __launch_bounds__(kTcThreads, 1)
refresh_tc_kernel(const SweepParams<float> *__restrict__ probs, int chains, int stage_bytes, int track_drift)
{
    extern __shared__ unsigned char smem_dyn[];
    __shared__ unsigned long long bar[2];
    __shared__ unsigned s_tmem;
    const SweepParams<float> &p = probs[blockIdx.y];
    const int nparts = p.ksplit > 1 ? p.ksplit : 1;   // this problem's k parts
    if ((int)blockIdx.z >= nparts) return;            // (uniform per CTA, before any barrier)
    const int M = p.M, N = p.N;
    const int ntiles = (M + kTcCols - 1) / kTcCols;
    const int BN = ((M + ntiles - 1) / ntiles + 15) / 16 * 16;   // MMA N: a multiple of 16, <= 256
    const int nkt = (N + kTcBK - 1) / kTcBK;
    // this CTA's k-tiles [kt0, kt1) (every part holds at least one: nparts <= nkt)
    const int kt0 = (int)(((long long)blockIdx.z * nkt) / nparts);
    const int kt1 = (int)(((long long)(blockIdx.z + 1) * nkt) / nparts);
    const int warp = threadIdx.x >> 5;
    unsigned char *base = smem_dyn + ((1024 - (smem_addr(smem_dyn) & 1023)) & 1023);

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = s_tmem;
    const unsigned idesc = tf32_idesc(BN);
    const int row0 = blockIdx.x * kTcRows;
    const int q = row0 + threadIdx.x;   // this thread's chain = its TMEM lane
    const bool active = q < chains;
    double sum_old = 0.0, sum_new = 0.0;
    unsigned uses[2] = {0u, 0u};        // commits made to each stage's barrier
    int fail = 0;

    for (int mt = 0; mt < ntiles && !fail; ++mt) {
        const int m0 = mt * BN;
        for (int kt = kt0; kt < kt1; ++kt) {
            const int st = (kt - kt0) & 1;
            unsigned char *a_hi = base + (size_t)st * stage_bytes;
            unsigned char *a_lo = a_hi + kTcAtile;
            unsigned char *b_hi = a_lo + kTcAtile;
            unsigned char *b_lo = b_hi + (size_t)BN * kTcBK * 4;
            // the MMAs that last read this stage must have completed
            if (uses[st] && !mbar_wait(&bar[st], (uses[st] - 1u) & 1u, kWaitLimit)) fail = 1;
            if (__syncthreads_or(fail)) {
                fail = 1;
                break;
            }
            stage_centred(p.F, p.ldF, p.fref, chains, N, row0, kt * kTcBK, a_hi, a_lo);
            stage_rows(p.Khi, p.ldK, M, N, m0, kt * kTcBK, BN, b_hi, nullptr);
            stage_rows(p.Klo, p.ldK, M, N, m0, kt * kTcBK, BN, b_lo, nullptr);
            fence_proxy_async_smem();   // generic-proxy writes become visible to the tensor cores
            __syncthreads();
            if (threadIdx.x == 0) {
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < kTcBK / 8; ++ks) {   // K = 8 TF32 per MMA: two core matrices
                    const unsigned k_off = (unsigned)ks * 256u;
                    const unsigned long long dah = umma_desc(smem_addr(a_hi) + k_off, 128, 1024);
                    const unsigned long long dal = umma_desc(smem_addr(a_lo) + k_off, 128, 1024);
                    const unsigned long long dbh = umma_desc(smem_addr(b_hi) + k_off, 128, 1024);
                    const unsigned long long dbl = umma_desc(smem_addr(b_lo) + k_off, 128, 1024);
                    umma_tf32(tmem, dah, dbh, idesc, (kt > kt0 || ks > 0) ? 1u : 0u);
                    umma_tf32(tmem, dah, dbl, idesc, 1u);
                    umma_tf32(tmem, dal, dbh, idesc, 1u);
                }
                umma_commit(&bar[st]);
            }
            ++uses[st];
        }
        if (fail) break;
        // the last commit covers every MMA issued before it
        const int lst = (kt1 - kt0 - 1) & 1;
        if (!mbar_wait(&bar[lst], (uses[lst] - 1u) & 1u, kWaitLimit)) fail = 1;
        if (__syncthreads_or(fail)) {
            fail = 1;
            break;
        }
        tc_fence_after();
        const unsigned lane_base = tmem + ((unsigned)(warp * 32) << 16);
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + (unsigned)c0, v);
            if (active && nparts > 1) {   // this part's product, combined by refresh_finish_kernel
                float *Dq = p.Dpart + ((size_t)blockIdx.z * chains + q) * p.ldR;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int m = m0 + c0 + j;
                    if (m < M) Dq[m] = v[j];
                }
            } else if (active) {
                float *Rq = p.R + (size_t)q * p.ldR;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int m = m0 + c0 + j;
                    if (m < M) {
                        const double r = p.rref[m] - (double)v[j];
                        const double old = (double)Rq[m];
                        sum_old += old * old;
                        sum_new += r * r;
                        Rq[m] = (float)r;
                    }
                }
            }
        }
        // every lane is read before the next tile's MMAs overwrite the accumulator
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (fail) {
        // let the MMAs in flight finish before the CTA leaves (bounded), then count the timeout
        if (threadIdx.x == 0) {
            for (int s = 0; s < 2; ++s)
                if (uses[s]) mbar_wait(&bar[s], (uses[s] - 1u) & 1u, kWaitLimit);
            atomicAdd(&p.counters->timeouts, 1ull);
        }
    } else if (active && nparts == 1) {
        p.chi2[q] = sum_new;
        if (track_drift) {
            const double drift = fabs(sum_old - sum_new) / fmax(sum_new, 1e-300);
            atomicMax(&p.counters->drift_bits, (unsigned long long)__double_as_longlong(drift));
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// K~ (held transposed, N x M FP64) into TF32 high and low parts, M x ldK FP32
// each, zero beyond N.
__global__ void split_k_kernel(const double *__restrict__ KtT, int M, int N, int ldK, float *__restrict__ Khi,
                               float *__restrict__ Klo)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)M * ldK) return;
    const int m = (int)(i / ldK), n = (int)(i % ldK);
    const double x = n < N ? KtT[(size_t)n * M + m] : 0.0;
    const float h = tf32_round((float)x);
    Khi[i] = h;
    Klo[i] = tf32_round((float)(x - (double)h));
}

// r~ = r_ref - (sum over the k parts of their products, added in FP64 in part
// order), chi^2 and the drift, for the problems whose refresh is split over k:
// one warp per chain, the lanes over the data points.
__global__ void refresh_finish_kernel(const SweepParams<float> *__restrict__ probs, int chains, int track_drift)
{
    const SweepParams<float> &p = probs[blockIdx.y];
    if (p.ksplit <= 1) return;
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= chains) return;
    const size_t part = (size_t)chains * p.ldR;
    const float *Dq = p.Dpart + (size_t)q * p.ldR;
    float *Rq = p.R + (size_t)q * p.ldR;
    double sum_old = 0.0, sum_new = 0.0;
    for (int m = lane; m < p.M; m += 32) {
        double d = 0.0;
        for (int z = 0; z < p.ksplit; ++z) d += (double)Dq[z * part + m];
        const double r = p.rref[m] - d;
        const double old = (double)Rq[m];
        sum_old += old * old;
        sum_new += r * r;
        Rq[m] = (float)r;
    }
    for (int off = 16; off; off >>= 1) {
        sum_old += __shfl_xor_sync(0xffffffffu, sum_old, off);
        sum_new += __shfl_xor_sync(0xffffffffu, sum_new, off);
    }
    if (lane == 0) {
        p.chi2[q] = sum_new;
        if (track_drift) {
            const double drift = fabs(sum_old - sum_new) / fmax(sum_new, 1e-300);
            atomicMax(&p.counters->drift_bits, (unsigned long long)__double_as_longlong(drift));
        }
    }
}

}  // namespace

int refresh_tc_ksplit(int chains, int N)
{
    // enough CTAs to cover the GPU once, at least two k-tiles per part, at most 16 parts
    const int nkt = (N + kTcBK - 1) / kTcBK;
    const int tiles = (chains + kTcRows - 1) / kTcRows;
    int parts = (152 + tiles - 1) / tiles;
    parts = std::min(parts, std::max(1, nkt / 2));
    return std::max(1, std::min(parts, 16));
}

cudaError_t launch_refresh_finish(const SweepParams<float> *probs, int n_problems, int chains, bool track_drift,
                                  cudaStream_t s)
{
    const dim3 grid((unsigned)((chains + 3) / 4), (unsigned)n_problems);
    refresh_finish_kernel<<<grid, 128, 0, s>>>(probs, chains, track_drift ? 1 : 0);
    return cudaGetLastError();
}

int refresh_tc_bn(int M)
{
    const int ntiles = (M + kTcCols - 1) / kTcCols;
    return ((M + ntiles - 1) / ntiles + 15) / 16 * 16;
}

size_t refresh_tc_smem(int max_bn)
{
    return 2 * ((size_t)2 * kTcAtile + (size_t)2 * max_bn * kTcBK * 4) + 1024;
}

cudaError_t launch_refresh_tc(const SweepParams<float> *probs, int n_problems, int chains, int max_bn, int max_parts,
                              bool track_drift, cudaStream_t s)
{
    const int stage_bytes = 2 * kTcAtile + 2 * max_bn * kTcBK * 4;
    const size_t smem = refresh_tc_smem(max_bn);
    cudaError_t e = cudaFuncSetAttribute(refresh_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((chains + kTcRows - 1) / kTcRows), (unsigned)n_problems, (unsigned)max_parts);
    refresh_tc_kernel<<<grid, kTcThreads, smem, s>>>(probs, chains, stage_bytes, track_drift ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_refresh_ref(const SweepParams<float> *probs, int n_problems, int chains, int max_N, int max_M,
                               cudaStream_t s)
{
    refresh_fref_kernel<<<dim3((unsigned)((max_N + 31) / 32), (unsigned)n_problems), 256, 0, s>>>(probs, chains);
    refresh_rref_kernel<<<dim3((unsigned)((max_M + 127) / 128), (unsigned)n_problems), 128, 0, s>>>(probs);
    return cudaGetLastError();
}

cudaError_t launch_split_k(const double *KtT, int M, int N, int ldK, float *Khi, float *Klo, cudaStream_t s)
{
    const long long tot = (long long)M * ldK;
    split_k_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(KtT, M, N, ldK, Khi, Klo);
    return cudaGetLastError();
}

}  // namespace asmgb
