// Grouped, batched GEMM whose shapes and pointers are read from device memory (GemmArgs), so that
// rank-dependent sizes decided on the GPU (truncation ranks) need no host round trip and the launch
// sequence is fixed (CUDA-graph capturable).  Column-major, op(A) is M x K, op(B) is K x N.
//
// Tiling: 64 x 64 output tile per CTA, K-step 16, 256 threads, 4 x 4 outputs per thread held in
// registers; operands staged through two shared-memory stages (the next K-step is fetched into registers
// while the current one is consumed), with loads coalesced along the contiguous index.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace tpcg {

constexpr int GBM = 64, GBN = 64, GBK = 16, GTHREADS = 256;

constexpr int GLOAD = (GBM * GBK) / GTHREADS;   // elements of each operand tile a thread moves per K-step

// global -> registers (bounds-checked; zero outside), coalesced along the contiguous index
template <typename T, bool TA>
__device__ __forceinline__ void gemm_fetch_a(T (&r)[GLOAD], const T* A, long long lda, int M, int K, int m0, int k0,
                                             int tid) {
#pragma unroll
    for (int q = 0; q < GLOAD; ++q) {
        const int e = tid + q * GTHREADS;
        int mm, kk;
        if (!TA) { mm = e % GBM; kk = e / GBM; }   // A[m + k lda]: contiguous in m
        else     { kk = e % GBK; mm = e / GBK; }   // A[k + m lda]: contiguous in k
        const int m = m0 + mm, k = k0 + kk;
        r[q] = (m < M && k < K) ? (TA ? A[k + (long long)m * lda] : A[m + (long long)k * lda]) : T(0);
    }
}

template <typename T, bool TA>
__device__ __forceinline__ void gemm_store_a(T (*As)[GBM + 1], const T (&r)[GLOAD], int tid) {
#pragma unroll
    for (int q = 0; q < GLOAD; ++q) {
        const int e = tid + q * GTHREADS;
        if (!TA) As[e / GBM][e % GBM] = r[q];
        else     As[e % GBK][e / GBK] = r[q];
    }
}

template <typename T, bool TB>
__device__ __forceinline__ void gemm_fetch_b(T (&r)[GLOAD], const T* B, long long ldb, int N, int K, int n0, int k0,
                                             int tid) {
#pragma unroll
    for (int q = 0; q < GLOAD; ++q) {
        const int e = tid + q * GTHREADS;
        int nn, kk;
        if (!TB) { kk = e % GBK; nn = e / GBK; }   // B[k + n ldb]: contiguous in k
        else     { nn = e % GBN; kk = e / GBN; }   // B[n + k ldb]: contiguous in n
        const int nI = n0 + nn, k = k0 + kk;
        r[q] = (nI < N && k < K) ? (TB ? B[nI + (long long)k * ldb] : B[k + (long long)nI * ldb]) : T(0);
    }
}

template <typename T, bool TB>
__device__ __forceinline__ void gemm_store_b(T (*Bs)[GBN + 1], const T (&r)[GLOAD], int tid) {
#pragma unroll
    for (int q = 0; q < GLOAD; ++q) {
        const int e = tid + q * GTHREADS;
        if (!TB) Bs[e % GBK][e / GBK] = r[q];
        else     Bs[e / GBN][e % GBN] = r[q];
    }
}

// grid: (ceil(Mmax/64), ceil(Nmax/64), ngroups_max * bmax).  count_dev (optional) caps the group count.
template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(GTHREADS) gemm_grouped_kernel(const GemmArgs* __restrict__ args,
                                                                const int* __restrict__ count_dev, int bmax,
                                                                int zmax) {
    // two shared-memory stages: the next K-step is fetched into registers while the current one is used
    __shared__ T As[2][GBK][GBM + 1];
    __shared__ T Bs[2][GBK][GBN + 1];
    const int gcount = count_dev != nullptr ? *count_dev : (zmax / bmax);
    for (int z = blockIdx.z; z < zmax; z += gridDim.z) {
    const int g = z / bmax;
    const int ib = z % bmax;
    if (g >= gcount) break;
    const GemmArgs a = args[g];
    if (a.acc ? (ib != 0) : (ib >= a.nbatch)) continue;
    const int M = a.M, N = a.N, K = a.K;
    const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
    if (m0 >= M || n0 >= N) continue;

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    const int nb = a.acc ? a.nbatch : 1;
    for (int b = 0; b < nb; ++b) {
        const int bi = a.acc ? b : ib;
        const T* A = static_cast<const T*>(a.A) + (long long)bi * a.sA;
        const T* B = static_cast<const T*>(a.B) + (long long)bi * a.sB;
        T ra[GLOAD], rb[GLOAD];
        gemm_fetch_a<T, TA>(ra, A, a.lda, M, K, m0, 0, tid);
        gemm_fetch_b<T, TB>(rb, B, a.ldb, N, K, n0, 0, tid);
        gemm_store_a<T, TA>(As[0], ra, tid);
        gemm_store_b<T, TB>(Bs[0], rb, tid);
        __syncthreads();
        int cur = 0;
        for (int k0 = 0; k0 < K; k0 += GBK) {
            const bool more = k0 + GBK < K;
            if (more) {
                gemm_fetch_a<T, TA>(ra, A, a.lda, M, K, m0, k0 + GBK, tid);
                gemm_fetch_b<T, TB>(rb, B, a.ldb, N, K, n0, k0 + GBK, tid);
            }
#pragma unroll
            for (int kk = 0; kk < GBK; ++kk) {
                T av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[cur][kk][tx + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[cur][kk][ty + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
            }
            if (more) {
                gemm_store_a<T, TA>(As[cur ^ 1], ra, tid);
                gemm_store_b<T, TB>(Bs[cur ^ 1], rb, tid);
            }
            __syncthreads();
            cur ^= 1;
        }
    }
    T* C = static_cast<T*>(a.C) + (a.acc ? 0LL : (long long)ib * a.sC);
    const T alpha = T(a.alpha), beta = T(a.beta);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + tx + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nI = n0 + ty + 16 * j;
            if (nI >= N) continue;
            T* c = C + m + (long long)nI * a.ldc;
            T v = alpha * acc[i][j];
            if (a.beta != 0.0) v += beta * (*c);
            *c = v;
        }
    }
    __syncthreads();
    }
}

// C = alpha * sum_{g < count} P_g + beta * C over an M x N column-major block (partials contiguous,
// stride M*N); M, N, count read from device.
template <typename T>
__global__ void reduce_partials_kernel(const T* __restrict__ P, const int* Mdev, const int* Ndev,
                                       const int* count_dev, T* __restrict__ C, long long ldc, double alpha,
                                       double beta) {
    const int M = *Mdev, N = *Ndev, cnt = *count_dev;
    const long long MN = (long long)M * N;
    if (ldc <= 0) ldc = M;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MN; e += (long long)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int g = 0; g < cnt; ++g) s += P[g * MN + e];
        const int m = (int)(e % M), nI = (int)(e / M);
        T* c = C + m + (long long)nI * ldc;
        T v = T(alpha) * s;
        if (beta != 0.0) v += T(beta) * (*c);
        *c = v;
    }
}

// CTA budget per SM of a grouped GEMM launch (0: one CTA per output tile and group, uncapped); set through
// tpcg_set_option
int gemm_ctas_per_sm();

// multiprocessors of the current device (queried once per device)
inline int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cache[dev] = v;
    }
    return cache[dev];
}

// FP32 groups on the tensor cores (gemm_tc.cu): same arguments, 3xTF32 products with FP32 accumulation
template <bool TA, bool TB>
int launch_gemm_tc(const GemmArgs* args, const int* count_dev, int ngroups_max, int bmax, int Mmax, int Nmax,
                   cudaStream_t st);
int tc_kind();        // TPCG_OPT_TC: 1 FP32 contractions on the tensor cores, 0 on the FP32 SIMT units
int tc_prepare();     // shared-memory opt-in of the tensor-core kernels on the current device
int tc_take_error();  // nonzero once a tensor-core kernel abandoned a wait (the flag is cleared)

template <typename T, bool TA, bool TB>
inline int launch_gemm(const GemmArgs* args, const int* count_dev, int ngroups_max, int bmax, int Mmax, int Nmax,
                       cudaStream_t st) {
    if (ngroups_max <= 0 || bmax <= 0 || Mmax <= 0 || Nmax <= 0) return TPCG_OK;
    if constexpr (sizeof(T) == 4) {
        if (tc_kind() == 1) return launch_gemm_tc<TA, TB>(args, count_dev, ngroups_max, bmax, Mmax, Nmax, st);
    }
    const long long zmax = (long long)ngroups_max * bmax;
    // the kernel strides over z, so the grid can be capped at a CTA budget per SM: argument lists sized for
    // the worst case (most groups empty at run time) then do not flood the CTA scheduler
    const long long gx = (Mmax + GBM - 1) / GBM, gy = (Nmax + GBN - 1) / GBN;
    const int per_sm = gemm_ctas_per_sm();
    const long long zcap = per_sm > 0 ? std::max(1LL, ((long long)per_sm * sm_count()) / std::max(1LL, gx * gy))
                                      : zmax;
    const long long gz = std::min(std::min(zmax, zcap), 65535LL);
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)gz);
    if (grid.y > 65535u || zmax > (1LL << 30)) {
        set_error("gemm grid too large");
        return TPCG_E_INVALID;
    }
    gemm_grouped_kernel<T, TA, TB><<<grid, GTHREADS, 0, st>>>(args, count_dev, bmax, (int)zmax);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}

}  // namespace tpcg
