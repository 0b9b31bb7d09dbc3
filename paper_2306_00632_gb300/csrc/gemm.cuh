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

// ------------------------------------------------------------------------------------------------------------
// FP32 variant with an 8 x 4 output block per thread: 128 threads per 64 x 64 tile, K-step 16.  Per K-step a thread
// reads its 8 rows of A and 4 columns of B as three 16-byte shared loads and issues 32 FMAs (the 4 x 4 kernel
// issues 8 scalar shared loads per 16 FMAs).  The tiles are staged through registers and two shared stages as in
// gemm_grouped_kernel; row stride 68 floats keeps the 16-byte reads aligned and spreads the strided stores.
// Same arguments, grid and results contract as gemm_grouped_kernel.
// ------------------------------------------------------------------------------------------------------------
constexpr int G8_THREADS = 128, G8_LD = GBM + 4, G8_LOAD = (GBM * GBK) / G8_THREADS;   // 8 elements per operand

template <bool TA>
__device__ __forceinline__ void g8_fetch_a(float (&r)[G8_LOAD], const float* A, long long lda, int M, int K, int m0,
                                           int k0, int tid) {
#pragma unroll
    for (int q = 0; q < G8_LOAD; ++q) {
        const int e = tid + q * G8_THREADS;
        int mm, kk;
        if (!TA) { mm = e % GBM; kk = e / GBM; }
        else     { kk = e % GBK; mm = e / GBK; }
        const int m = m0 + mm, k = k0 + kk;
        r[q] = (m < M && k < K) ? (TA ? A[k + (long long)m * lda] : A[m + (long long)k * lda]) : 0.f;
    }
}

template <bool TA>
__device__ __forceinline__ void g8_store_a(float* As, const float (&r)[G8_LOAD], int tid) {
#pragma unroll
    for (int q = 0; q < G8_LOAD; ++q) {
        const int e = tid + q * G8_THREADS;
        if (!TA) As[(e / GBM) * G8_LD + e % GBM] = r[q];
        else     As[(e % GBK) * G8_LD + e / GBK] = r[q];
    }
}

template <bool TB>
__device__ __forceinline__ void g8_fetch_b(float (&r)[G8_LOAD], const float* B, long long ldb, int N, int K, int n0,
                                           int k0, int tid) {
#pragma unroll
    for (int q = 0; q < G8_LOAD; ++q) {
        const int e = tid + q * G8_THREADS;
        int nn, kk;
        if (!TB) { kk = e % GBK; nn = e / GBK; }
        else     { nn = e % GBN; kk = e / GBN; }
        const int nI = n0 + nn, k = k0 + kk;
        r[q] = (nI < N && k < K) ? (TB ? B[nI + (long long)k * ldb] : B[k + (long long)nI * ldb]) : 0.f;
    }
}

template <bool TB>
__device__ __forceinline__ void g8_store_b(float* Bs, const float (&r)[G8_LOAD], int tid) {
#pragma unroll
    for (int q = 0; q < G8_LOAD; ++q) {
        const int e = tid + q * G8_THREADS;
        if (!TB) Bs[(e % GBK) * G8_LD + e / GBK] = r[q];
        else     Bs[(e / GBN) * G8_LD + e % GBN] = r[q];
    }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(G8_THREADS) gemm88_kernel(const GemmArgs* __restrict__ args,
                                                            const int* __restrict__ count_dev, int bmax, int zmax) {
    __shared__ __align__(16) float As[2][GBK * G8_LD];
    __shared__ __align__(16) float Bs[2][GBK * G8_LD];
    const int gcount = count_dev != nullptr ? *count_dev : (zmax / bmax);
    const int tid = threadIdx.x;
    const int tx = tid % 8, ty = tid / 8;   // rows 8 tx .. 8 tx + 7, columns 4 ty .. 4 ty + 3 of the tile
    for (int z = blockIdx.z; z < zmax; z += gridDim.z) {
        const int g = z / bmax;
        const int ib = z % bmax;
        if (g >= gcount) break;
        const GemmArgs a = args[g];
        if (a.acc ? (ib != 0) : (ib >= a.nbatch)) continue;
        const int M = a.M, N = a.N, K = a.K;
        const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
        if (m0 >= M || n0 >= N) continue;
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        const int nb = a.acc ? a.nbatch : 1;
        for (int b = 0; b < nb; ++b) {
            const int bi = a.acc ? b : ib;
            const float* A = static_cast<const float*>(a.A) + (long long)bi * a.sA;
            const float* B = static_cast<const float*>(a.B) + (long long)bi * a.sB;
            float ra[G8_LOAD], rb[G8_LOAD];
            g8_fetch_a<TA>(ra, A, a.lda, M, K, m0, 0, tid);
            g8_fetch_b<TB>(rb, B, a.ldb, N, K, n0, 0, tid);
            g8_store_a<TA>(As[0], ra, tid);
            g8_store_b<TB>(Bs[0], rb, tid);
            __syncthreads();
            int cur = 0;
            for (int k0 = 0; k0 < K; k0 += GBK) {
                const bool more = k0 + GBK < K;
                if (more) {
                    g8_fetch_a<TA>(ra, A, a.lda, M, K, m0, k0 + GBK, tid);
                    g8_fetch_b<TB>(rb, B, a.ldb, N, K, n0, k0 + GBK, tid);
                }
                const float* Ac = As[cur];
                const float* Bc = Bs[cur];
#pragma unroll
                for (int kk = 0; kk < GBK; ++kk) {
                    const float4 a0 = *reinterpret_cast<const float4*>(Ac + kk * G8_LD + 8 * tx);
                    const float4 a1 = *reinterpret_cast<const float4*>(Ac + kk * G8_LD + 8 * tx + 4);
                    const float4 b0 = *reinterpret_cast<const float4*>(Bc + kk * G8_LD + 4 * ty);
                    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float bv[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
                }
                if (more) {
                    g8_store_a<TA>(As[cur ^ 1], ra, tid);
                    g8_store_b<TB>(Bs[cur ^ 1], rb, tid);
                }
                __syncthreads();
                cur ^= 1;
            }
        }
        float* C = static_cast<float*>(a.C) + (a.acc ? 0LL : (long long)ib * a.sC);
        const float alpha = (float)a.alpha, beta = (float)a.beta;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nI = n0 + 4 * ty + j;
            if (nI >= N) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int m = m0 + 8 * tx + i;
                if (m >= M) continue;
                float* c = C + m + (long long)nI * a.ldc;
                float v = alpha * acc[i][j];
                if (a.beta != 0.0) v += beta * (*c);
                *c = v;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------------------------
// The same 8 x 4-per-thread FP32 tile with the operands copied global -> shared by cp.async (no staging
// registers) through GCP_STAGES shared stages: while a K-step is multiplied, the copies of the next
// GCP_STAGES - 1 are in flight.  Out-of-range elements are zero-filled by the copy itself (source size 0).
// ------------------------------------------------------------------------------------------------------------
constexpr int GCP_STAGES = 3;

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool pred) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    const int n = pred ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <bool TA, bool TB>
__device__ __forceinline__ void gcp_issue(float* As, float* Bs, const float* A, const float* B, long long lda,
                                          long long ldb, int M, int N, int K, int m0, int n0, int k0, int tid) {
#pragma unroll 2
    for (int q = 0; q < G8_LOAD; ++q) {
        const int e = tid + q * G8_THREADS;
        int mm, kk;
        if (!TA) { mm = e % GBM; kk = e / GBM; }
        else     { kk = e % GBK; mm = e / GBK; }
        const int m = m0 + mm, k = k0 + kk;
        const bool ok = m < M && k < K;
        const float* src = ok ? (TA ? A + k + (long long)m * lda : A + m + (long long)k * lda) : A;
        cp_async4(As + kk * G8_LD + mm, src, ok);
    }
#pragma unroll 2
    for (int q = 0; q < G8_LOAD; ++q) {
        const int e = tid + q * G8_THREADS;
        int nn, kk;
        if (!TB) { kk = e % GBK; nn = e / GBK; }
        else     { nn = e % GBN; kk = e / GBN; }
        const int nI = n0 + nn, k = k0 + kk;
        const bool ok = nI < N && k < K;
        const float* src = ok ? (TB ? B + nI + (long long)k * ldb : B + k + (long long)nI * ldb) : B;
        cp_async4(Bs + kk * G8_LD + nn, src, ok);
    }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(G8_THREADS) gemm_cpa_kernel(const GemmArgs* __restrict__ args,
                                                              const int* __restrict__ count_dev, int bmax, int zmax) {
    __shared__ __align__(16) float As[GCP_STAGES][GBK * G8_LD];
    __shared__ __align__(16) float Bs[GCP_STAGES][GBK * G8_LD];
    const int gcount = count_dev != nullptr ? *count_dev : (zmax / bmax);
    const int tid = threadIdx.x;
    const int tx = tid % 8, ty = tid / 8;   // rows 8 tx .. 8 tx + 7, columns 4 ty .. 4 ty + 3 of the tile
    for (int z = blockIdx.z; z < zmax; z += gridDim.z) {
        const int g = z / bmax;
        const int ib = z % bmax;
        if (g >= gcount) break;
        const GemmArgs a = args[g];
        if (a.acc ? (ib != 0) : (ib >= a.nbatch)) continue;
        const int M = a.M, N = a.N, K = a.K;
        const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
        if (m0 >= M || n0 >= N) continue;
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        const int nb = a.acc ? a.nbatch : 1;
        const int nk = (K + GBK - 1) / GBK;
        for (int b = 0; b < nb; ++b) {
            const int bi = a.acc ? b : ib;
            const float* A = static_cast<const float*>(a.A) + (long long)bi * a.sA;
            const float* B = static_cast<const float*>(a.B) + (long long)bi * a.sB;
#pragma unroll
            for (int st = 0; st < GCP_STAGES - 1; ++st) {   // prologue: the first stages (empty groups past K)
                if (st < nk) gcp_issue<TA, TB>(As[st], Bs[st], A, B, a.lda, a.ldb, M, N, K, m0, n0, st * GBK, tid);
                cp_async_commit();
            }
            for (int kt = 0; kt < nk; ++kt) {
                cp_async_wait<GCP_STAGES - 2>();   // this thread's copies of K-step kt have landed
                __syncthreads();                   // everyone's have, and everyone is done with K-step kt - 1
                const int nx = kt + GCP_STAGES - 1;
                if (nx < nk) {
                    const int sn = nx % GCP_STAGES;
                    gcp_issue<TA, TB>(As[sn], Bs[sn], A, B, a.lda, a.ldb, M, N, K, m0, n0, nx * GBK, tid);
                }
                cp_async_commit();
                const float* Ac = As[kt % GCP_STAGES];
                const float* Bc = Bs[kt % GCP_STAGES];
#pragma unroll
                for (int kk = 0; kk < GBK; ++kk) {
                    const float4 a0 = *reinterpret_cast<const float4*>(Ac + kk * G8_LD + 8 * tx);
                    const float4 a1 = *reinterpret_cast<const float4*>(Ac + kk * G8_LD + 8 * tx + 4);
                    const float4 b0 = *reinterpret_cast<const float4*>(Bc + kk * G8_LD + 4 * ty);
                    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float bv[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
                }
            }
            cp_async_wait<0>();
            __syncthreads();   // the stages are refilled by the next batch or tile
        }
        float* C = static_cast<float*>(a.C) + (a.acc ? 0LL : (long long)ib * a.sC);
        const float alpha = (float)a.alpha, beta = (float)a.beta;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nI = n0 + 4 * ty + j;
            if (nI >= N) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int m = m0 + 8 * tx + i;
                if (m >= M) continue;
                float* c = C + m + (long long)nI * a.ldc;
                float v = alpha * acc[i][j];
                if (a.beta != 0.0) v += beta * (*c);
                *c = v;
            }
        }
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
int gemm_kind();      // TPCG_OPT_GEMM_KIND: 1 the 8 x 4-per-thread FP32 kernel, 2 the same with cp.async stages, 0 the 4 x 4 one
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
    if constexpr (sizeof(T) == 4) {
        if (gemm_kind() >= 1) {   // 8 x 4 outputs per thread: half the threads per tile, same thread budget
            const long long zcap8 = per_sm > 0 ? std::max(1LL, ((long long)2 * per_sm * sm_count()) /
                                                                   std::max(1LL, gx * gy))
                                               : zmax;
            dim3 grid8((unsigned)gx, (unsigned)gy, (unsigned)std::min(std::min(zmax, zcap8), 65535LL));
            if (gemm_kind() == 2)
                gemm_cpa_kernel<TA, TB><<<grid8, G8_THREADS, 0, st>>>(args, count_dev, bmax, (int)zmax);
            else
                gemm88_kernel<TA, TB><<<grid8, G8_THREADS, 0, st>>>(args, count_dev, bmax, (int)zmax);
            TPCG_CHECK_LAUNCH();
            return TPCG_OK;
        }
    }
    gemm_grouped_kernel<T, TA, TB><<<grid, GTHREADS, 0, st>>>(args, count_dev, bmax, (int)zmax);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}

}  // namespace tpcg
