// asm_ceiling.cu -- measured arithmetic ceilings of the sweep kernel's
// instruction mix (the denominators of its roofline; no counterpart in the
// paper).
//
// Every move of blocked modes sampling (Sec. IV.B-C) runs, per element of the
// block, the fused pass of the chain kernel: the update f + delta V (one FMA),
// the clamp at zero (max), the bound product x R (multiply) and the two bound
// keys (signed and unsigned integer minima of the product's bits).  These
// kernels run that mix -- or one of its instructions alone -- on register
// operands at full occupancy, eight independent streams per thread, so that
// nothing but issue and pipe throughput limits them.  A variant reads V and R
// from shared memory as 16-byte vectors, as the chain kernel does.
#include <cuda_runtime.h>

#include "asm.h"

namespace {

constexpr int kThreads = 512;
constexpr int kStreams = 8;

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

template <class T> struct KeyOf;
template <> struct KeyOf<float> {
    using S = int;
    using U = unsigned;
    static __device__ __forceinline__ S bits(float x) { return __float_as_int(x); }
};
template <> struct KeyOf<double> {
    using S = long long;
    using U = unsigned long long;
    static __device__ __forceinline__ S bits(double x) { return __double_as_longlong(x); }
};

__device__ __forceinline__ float fmax_(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double fmax_(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float fmin_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double fmin_(double a, double b) { return fmin(a, b); }

// KIND 0: the pass (FMA, max, multiply, two integer minima) on registers;
// 1: the pass with V and R read from shared memory; 2: FMA only; 3: max and min only;
// 4: 32/64-bit signed and unsigned integer minima only.  clk[0..1] receives clock64() and
// the global timer (ns) of CTA 0, thread 0, before and after its loop.
template <class T, int KIND>
__global__ void __launch_bounds__(kThreads) ceiling_kernel(int iters, T delta, unsigned long long key,
                                                           unsigned long long *sink, long long *clk)
{
    using S = typename KeyOf<T>::S;
    using U = typename KeyOf<T>::U;
    // one row of V and R per CTA, read by every warp (as the chain kernel's
    // warps read the same move record)
    __shared__ __align__(16) T vs[32 * kStreams];
    __shared__ __align__(16) T rs[32 * kStreams];
    const int lane = threadIdx.x & 31;
    T f[kStreams], v[kStreams], r[kStreams];
    S lk[kStreams];
    U hk[kStreams];
#pragma unroll
    for (int i = 0; i < kStreams; ++i) {
        // operands from the runtime argument, so that none is a compile-time constant
        f[i] = T(1) + delta * T(0.004) * (T)(threadIdx.x + i);
        v[i] = delta * (T(2) - T(0.04) * (T)i);
        r[i] = T(-1) / v[i];
        lk[i] = (S)0;
        hk[i] = ~(U)0;
        if (threadIdx.x < 32) {
            vs[lane * kStreams + i] = v[i];
            rs[lane * kStreams + i] = r[i];
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[0] = clock64();
        clk[1] = (long long)globaltimer_ns();
    }
    for (int it = 0; it < iters; ++it) {
        if constexpr (KIND == 1) {
            // the chain kernel's operand path: 16-byte vectors of V and R per 16 bytes of elements
            constexpr int VEC = 16 / sizeof(T);
#pragma unroll
            for (int i = 0; i < kStreams; i += VEC) {
                if constexpr (VEC == 4) {
                    const float4 a = *reinterpret_cast<const float4 *>(&vs[lane * kStreams + i]);
                    const float4 b = *reinterpret_cast<const float4 *>(&rs[lane * kStreams + i]);
                    v[i] = a.x; v[i + 1] = a.y; v[i + 2] = a.z; v[i + 3] = a.w;
                    r[i] = b.x; r[i + 1] = b.y; r[i + 2] = b.z; r[i + 3] = b.w;
                } else {
                    const double2 a = *reinterpret_cast<const double2 *>(&vs[lane * kStreams + i]);
                    const double2 b = *reinterpret_cast<const double2 *>(&rs[lane * kStreams + i]);
                    v[i] = a.x; v[i + 1] = a.y;
                    r[i] = b.x; r[i + 1] = b.y;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kStreams; ++i) {
            if constexpr (KIND <= 1) {
                T x = fma(delta, v[i], f[i]);
                x = fmax_(x, T(0));
                f[i] = x;
                const S k = KeyOf<T>::bits(x * r[i]);
                lk[i] = k < lk[i] ? k : lk[i];
                hk[i] = (U)k < hk[i] ? (U)k : hk[i];
            } else if constexpr (KIND == 2) {
                f[i] = fma(delta, v[i], f[i]);
            } else if constexpr (KIND == 3) {
                // a maximum and a minimum, linked across the streams (neither is idempotent)
                f[i] = fmax_(f[i], v[i]);
                v[i] = fmin_(v[i], f[(i + 1) % kStreams]);
            } else {
                // signed and unsigned minima, linked across the streams so that
                // none of them folds away
                const S a = (S)hk[(i + 1) % kStreams];
                lk[i] = a < lk[i] ? a : lk[i];
                const U b = (U)lk[(i + 3) % kStreams];
                hk[i] = b < hk[i] ? b : hk[i];
            }
        }
        delta = -delta;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[2] = clock64();
        clk[3] = (long long)globaltimer_ns();
    }
    unsigned long long acc = 0;
#pragma unroll
    for (int i = 0; i < kStreams; ++i)
        acc ^= (unsigned long long)KeyOf<T>::bits(f[i]) ^ (unsigned long long)KeyOf<T>::bits(v[i]) ^
               (unsigned long long)lk[i] ^ (unsigned long long)hk[i];
    if (acc == key) sink[blockIdx.x] = acc;   // a runtime key: keeps every stream live
}

template <class T, int KIND>
cudaError_t run(int ctas, int iters, unsigned long long *sink, long long *clk, cudaStream_t s)
{
    ceiling_kernel<T, KIND><<<ctas, kThreads, 0, s>>>(iters, T(0.25), 0x5a5a5a5a5a5a5a5aull, sink, clk);
    return cudaGetLastError();
}

cudaError_t launch(int kind, int ctas, int iters, unsigned long long *sink, long long *clk, cudaStream_t s)
{
    switch (kind) {
    case ASM_CEIL_PASS_F32: return run<float, 0>(ctas, iters, sink, clk, s);
    case ASM_CEIL_PASS_F32_SMEM: return run<float, 1>(ctas, iters, sink, clk, s);
    case ASM_CEIL_FFMA: return run<float, 2>(ctas, iters, sink, clk, s);
    case ASM_CEIL_FMNMX: return run<float, 3>(ctas, iters, sink, clk, s);
    case ASM_CEIL_IMNMX: return run<float, 4>(ctas, iters, sink, clk, s);
    case ASM_CEIL_PASS_F64: return run<double, 0>(ctas, iters, sink, clk, s);
    case ASM_CEIL_PASS_F64_SMEM: return run<double, 1>(ctas, iters, sink, clk, s);
    case ASM_CEIL_DFMA: return run<double, 2>(ctas, iters, sink, clk, s);
    case ASM_CEIL_DMNMX: return run<double, 3>(ctas, iters, sink, clk, s);
    case ASM_CEIL_I64MNMX: return run<double, 4>(ctas, iters, sink, clk, s);
    default: return cudaErrorInvalidValue;
    }
}

// operations of one stream step: elements for the passes, instructions otherwise
double ops_per_step(int kind)
{
    return (kind == ASM_CEIL_FMNMX || kind == ASM_CEIL_DMNMX || kind == ASM_CEIL_IMNMX || kind == ASM_CEIL_I64MNMX)
               ? 2.0
               : 1.0;
}

}  // namespace

extern "C" int asm_measure_ceiling(int kind, double target_ms, double *ops_per_s, double *sm_mhz, double *ms_out)
{
    if (!ops_per_s || kind < 0 || kind >= ASM_CEIL_KINDS || !(target_ms > 0.0) || target_ms > 2000.0)
        return ASM_ERR_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return ASM_ERR_CUDA;
    const int ctas = sms * (per_sm / kThreads > 0 ? per_sm / kThreads : 1);
    unsigned long long *sink = nullptr;
    long long *clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    int rc = ASM_OK;
    long long hclk[4] = {0, 0, 0, 0};
    float ms = 0.f;
    int iters = 64;
    if (cudaMalloc(&sink, sizeof(unsigned long long) * ctas) != cudaSuccess ||
        cudaMalloc(&clk, sizeof(long long) * 4) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        rc = ASM_ERR_CUDA;
        goto done;
    }
    // warm up, then grow the loop until one launch takes about target_ms
    for (int pass = 0; pass < 8; ++pass) {
        if (cudaEventRecord(e0, s) != cudaSuccess || launch(kind, ctas, iters, sink, clk, s) != cudaSuccess ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = ASM_ERR_CUDA;
            goto done;
        }
        if (pass >= 1 && ms >= 0.7 * target_ms) break;
        const double grow = ms > 0.01f ? target_ms / ms : 64.0;
        const double next = (double)iters * (grow > 64.0 ? 64.0 : grow);
        iters = next > (double)(1 << 26) ? (1 << 26) : (int)next + 1;
    }
    if (cudaMemcpy(hclk, clk, sizeof(hclk), cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = ASM_ERR_CUDA;
        goto done;
    }
    *ops_per_s = (double)ctas * kThreads * kStreams * ops_per_step(kind) * (double)iters / (ms * 1e-3);
    if (sm_mhz) {
        const double dns = (double)(hclk[3] - hclk[1]);
        *sm_mhz = dns > 0 ? (double)(hclk[2] - hclk[0]) / dns * 1e3 : 0.0;
    }
    if (ms_out) *ms_out = ms;
done:
    if (sink) cudaFree(sink);
    if (clk) cudaFree(clk);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return rc;
}
