// asm_moments.cu -- the contractions of the backward pass, hand-written: the
// snapshot moments sum_q d_q d_q^T and the scores s_p(q) = r~_q . (K~_theta_p f_q)
// that the covariance identities of the gradients need, and the G-product
// C^{-1} K Cov(fbar) v' of the vector-Jacobian product.
//
// The gradients follow from the likelihood exp(-chi^2/2) of Eq. chi2 over the
// flat measure on fbar >= 0 (Eq. PI): d<fbar>/dG = Cov(fbar, fbar) K^T C^{-1}
// (the score of G is linear in fbar) and d<fbar>/dtheta_p = Cov(fbar, s_p)
// with s_p = (G - K fbar)^T C^{-1} (dK/dtheta_p) fbar, accumulated over
// snapshots of all chains.
//
// One tile kernel serves both products: out(i, j) = sum_k X(k, i) Y(k, j)
// over a 64 x 64 tile per CTA, k in slices of 16 staged in shared memory,
// accumulated in T registers (4 x 4 per thread).  Operands are strided views;
// the load order follows whichever of the operand's two strides is 1 so that
// global reads coalesce.
#include <cuda_runtime.h>

#include "asm_internal.h"

namespace asmgb {
namespace {

constexpr int kTile = 64;
constexpr int kSlice = 16;
constexpr int kThreads = 256;

__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

// Element (k, i) of an operand at ptr[k * sk + i * si]; zero outside k < K, i < I.
template <class T>
struct View {
    const T *ptr;
    long long sk, si;
    int K, I;
};

// Epilogues: add the tile into an FP64 matrix (atomically: several k-ranges
// may add into one tile), or store it.
struct AddF64 {
    double *out;
    long long ld;
    int I, J;
    template <class T>
    __device__ void operator()(int i, int j, T v) const
    {
        if (i < I && j < J) atomicAdd(out + (long long)i * ld + j, (double)v);
    }
};
template <class T>
struct StoreT {
    T *out;
    long long ld;
    int I, J;
    __device__ void operator()(int i, int j, T v) const
    {
        if (i < I && j < J) out[(long long)i * ld + j] = v;
    }
};

// Stage kSlice x kTile elements of a view into s[k][i]: consecutive threads
// take consecutive i (KFAST = false, si == 1) or consecutive k (KFAST = true, sk == 1).
template <class T, bool KFAST>
__device__ __forceinline__ void stage(const View<T> &v, int k0, int kend, int i0, T (*s)[kTile + 1])
{
#pragma unroll
    for (int r = 0; r < kSlice * kTile / kThreads; ++r) {
        const int e = threadIdx.x + kThreads * r;
        const int kk = KFAST ? (e & (kSlice - 1)) : (e / kTile);
        const int ii = KFAST ? (e / kSlice) : (e & (kTile - 1));
        const int k = k0 + kk, i = i0 + ii;
        s[kk][ii] = (k < kend && i < v.I) ? v.ptr[(long long)k * v.sk + (long long)i * v.si] : T(0);
    }
}

// out(i, j) = sum over k in [z * kslice, (z + 1) * kslice) of X(k, i) Y(k, j),
// z = blockIdx.z; tile (blockIdx.x, blockIdx.y).
template <class T, bool XK, bool YK, class Epi>
__global__ void __launch_bounds__(kThreads) tile_product_kernel(View<T> X, View<T> Y, int kslice, Epi epi)
{
    __shared__ T xs[kSlice][kTile + 1];
    __shared__ T ys[kSlice][kTile + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * kTile, j0 = blockIdx.y * kTile;
    const int kb = blockIdx.z * kslice;
    const int ke = min(X.K, kb + kslice);
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
    for (int k0 = kb; k0 < ke; k0 += kSlice) {
        stage<T, XK>(X, k0, ke, i0, xs);
        stage<T, YK>(Y, k0, ke, j0, ys);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kSlice; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                a[r] = xs[kk][ty * 4 + r];
                b[r] = ys[kk][tx * 4 + r];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma_(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) epi(i0 + ty * 4 + r, j0 + tx * 4 + c, acc[r][c]);
}

// Scores of every parameter: s[q][p] = r~_q . (Y[q][p M .. p M + M) + kshift_p),
// one warp per chain, FP64 sums.
template <class T>
__global__ void scores_kernel(const T *R, int ldR, const T *Y, long long ldY, const double *kshift, int M,
                              int chains, int P, double *Sq)
{
    const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= chains) return;
    for (int pi = 0; pi < P; ++pi) {
        double a = 0.0;
        for (int m = lane; m < M; m += 32)
            a += (double)R[q * ldR + m] * ((double)Y[q * ldY + (long long)pi * M + m] + kshift[(long long)pi * M + m]);
        for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) Sq[q * P + pi] = a;
    }
}

// y = K~ u (K~ given transposed, N x M), one thread per data point.
__global__ void kt_times_kernel(const double *KtT, const double *u, int M, int N, double *y)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double a = 0.0;
    for (int n = 0; n < N; ++n) a += KtT[(long long)n * M + m] * u[n];
    y[m] = a;
}

// Solve L^T g = y in place (L lower triangular, column-major M x M): back
// substitution by columns in one CTA.
__global__ void lt_solve_kernel(const double *L, int M, double *y)
{
    __shared__ double gi;
    for (int i = M - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            gi = y[i] / L[(long long)i * M + i];
            y[i] = gi;
        }
        __syncthreads();
        // L^T(k, i) = L(i, k), stored at column k: L[k * M + i]
        for (int k = threadIdx.x; k < i; k += blockDim.x) y[k] -= L[(long long)k * M + i] * gi;
        __syncthreads();
    }
}

template <class T>
cudaError_t gram_impl(const T *D, int ldD, int chains, int N, double *Sff, cudaStream_t s)
{
    // FP32 partial sums over slices of 256 chains, added into the FP64 moments
    const int kslice = 256;
    const View<T> v{D, ldD, 1, chains, N};
    const AddF64 epi{Sff, N, N, N};
    const dim3 grid((N + kTile - 1) / kTile, (N + kTile - 1) / kTile, (chains + kslice - 1) / kslice);
    tile_product_kernel<T, false, false, AddF64><<<grid, kThreads, 0, s>>>(v, v, kslice, epi);
    return cudaGetLastError();
}

template <class T>
cudaError_t kth_product_impl(const T *D, int ldD, int chains, int N, const T *Kth, int PM, T *Y, cudaStream_t s)
{
    // Y[q][j] = sum_n D[q][n] Kth[j][n]: X(k = n, i = q) = D[q ldD + n], Y(k = n, j) = Kth[j N + n]
    const View<T> x{D, 1, ldD, N, chains};
    const View<T> y{Kth, 1, N, N, PM};
    const StoreT<T> epi{Y, PM, chains, PM};
    const dim3 grid((chains + kTile - 1) / kTile, (PM + kTile - 1) / kTile, 1);
    tile_product_kernel<T, true, true, StoreT<T>><<<grid, kThreads, 0, s>>>(x, y, N, epi);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gram(const float *D, int ldD, int chains, int N, double *Sff, cudaStream_t s)
{
    return gram_impl<float>(D, ldD, chains, N, Sff, s);
}
cudaError_t launch_gram(const double *D, int ldD, int chains, int N, double *Sff, cudaStream_t s)
{
    return gram_impl<double>(D, ldD, chains, N, Sff, s);
}
cudaError_t launch_kth_product(const float *D, int ldD, int chains, int N, const float *Kth, int PM, float *Y,
                               cudaStream_t s)
{
    return kth_product_impl<float>(D, ldD, chains, N, Kth, PM, Y, s);
}
cudaError_t launch_kth_product(const double *D, int ldD, int chains, int N, const double *Kth, int PM, double *Y,
                               cudaStream_t s)
{
    return kth_product_impl<double>(D, ldD, chains, N, Kth, PM, Y, s);
}
template <class T>
static cudaError_t scores_impl(const T *R, int ldR, const T *Y, const double *kshift, int M, int chains, int P,
                               double *Sq, cudaStream_t s)
{
    scores_kernel<T><<<(unsigned)(((long long)chains * 32 + 255) / 256), 256, 0, s>>>(R, ldR, Y, (long long)P * M,
                                                                                     kshift, M, chains, P, Sq);
    return cudaGetLastError();
}
cudaError_t launch_scores(const float *R, int ldR, const float *Y, const double *kshift, int M, int chains, int P,
                          double *Sq, cudaStream_t s)
{
    return scores_impl<float>(R, ldR, Y, kshift, M, chains, P, Sq, s);
}
cudaError_t launch_scores(const double *R, int ldR, const double *Y, const double *kshift, int M, int chains, int P,
                          double *Sq, cudaStream_t s)
{
    return scores_impl<double>(R, ldR, Y, kshift, M, chains, P, Sq, s);
}
cudaError_t launch_vjp_G(const double *KtT, const double *L, const double *u, int M, int N, double *y, cudaStream_t s)
{
    kt_times_kernel<<<(M + 127) / 128, 128, 0, s>>>(KtT, u, M, N, y);
    lt_solve_kernel<<<1, 256, 0, s>>>(L, M, y);
    return cudaGetLastError();
}

}  // namespace asmgb
