// FP32 grouped GEMM on the 5th-generation tensor cores (tcgen05), for the dense contractions of Alg. 1
// (Z formation, mode Grams, projections, Q S) and of the Tucker scalar products.
//
// Same contract as gemm_grouped_kernel (GemmArgs read from device memory, column-major, op(A) M x K,
// op(B) K x N, C = alpha op(A) op(B) + beta C, strided batches summed when acc = 1), computed as
//   * 128 x 128 output tiles, one CTA each, the FP32 accumulator in tensor memory (128 lanes x 128 columns);
//   * K in chunks of 32: every chunk of op(A) and op(B)^T is staged into shared memory in the K-major,
//     128-byte-swizzled layout that tcgen05.mma reads (row r of a tile holds 32 consecutive K values, 16-byte
//     chunk c stored at c ^ (r mod 8)), two stages deep so that staging overlaps the tensor-core work;
//   * FP32 accuracy from TF32 products by splitting each operand value x into hi = x (the tensor core uses
//     its TF32 part) and lo = x - tf32(x): A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo lo term is below
//     FP32 rounding), three kind::tf32 MMAs per 8-wide K step;
//   * one thread issues the MMAs and commits them to an mbarrier per stage; every wait on an mbarrier has an
//     iteration limit, after which the CTA records the failure, waits (bounded) for its MMAs, frees its tensor
//     memory and stops.
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "gemm.cuh"

namespace tpcg {

constexpr int TC_M = 128, TC_N = 128, TC_K = 32;       // tile and K chunk
constexpr int TC_THREADS = 256;
constexpr int TC_TILE_BYTES = TC_M * TC_K * 4;          // 16 KB per operand tile
constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;       // A hi, A lo, B hi, B lo
constexpr int TC_STAGES = 2;
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024;   // + alignment slack for the 1024-byte atoms
constexpr unsigned TC_TMEM_COLS = 128;
constexpr long long TC_SPIN_LIMIT = 1LL << 22;          // mbarrier polls before a wait is abandoned

__device__ int g_tc_error = 0;   // set when a wait was abandoned (read and cleared by tc_take_error)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; returns false when the limit was reached
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < TC_SPIN_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M = 128, N = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate));
}

// byte offset of element (row r, k) of a K-major 128-byte-swizzled tile of 32 FP32 per row
__device__ __forceinline__ uint32_t sw_off(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + ((k & 3) << 2));
}

__device__ __forceinline__ float tf32_lo(float x) {
    return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// stage rows [0, 128) x K values [k0, k0 + 32) of a column-major operand into the hi and lo tiles:
// element (r, k) is X[r + k ld] when rows are contiguous (ROWS), else X[k + r ld]; zero outside rows x kdim
template <bool ROWS>
__device__ __forceinline__ void stage_tile(unsigned char* hi, unsigned char* lo, const float* X, long long ld,
                                           int rows, int kdim, int r0, int k0, int tid) {
    if (ROWS) {   // consecutive threads take consecutive rows (coalesced), 16 K values each
        const int r = tid & 127, kb = (tid >> 7) * 16;
        const bool rin = r0 + r < rows;
        const float* src = X + (long long)(r0 + r);
#pragma unroll 4
        for (int j = 0; j < 16; ++j) {
            const int k = kb + j;
            const float x = (rin && k0 + k < kdim) ? src[(long long)(k0 + k) * ld] : 0.f;
            const uint32_t o = sw_off(r, k);
            *reinterpret_cast<float*>(hi + o) = x;
            *reinterpret_cast<float*>(lo + o) = tf32_lo(x);
        }
    } else {      // consecutive threads take consecutive K values (coalesced), 16 rows each
        const int k = tid & 31, rb = tid >> 5;
        const bool kin = k0 + k < kdim;
#pragma unroll 4
        for (int j = 0; j < 16; ++j) {
            const int r = rb + 8 * j;
            const float x = (kin && r0 + r < rows) ? X[(long long)(k0 + k) + (long long)(r0 + r) * ld] : 0.f;
            const uint32_t o = sw_off(r, k);
            *reinterpret_cast<float*>(hi + o) = x;
            *reinterpret_cast<float*>(lo + o) = tf32_lo(x);
        }
    }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(TC_THREADS, 1) gemm_tc_kernel(const GemmArgs* __restrict__ args,
                                                                const int* __restrict__ count_dev, int bmax,
                                                                int zmax) {
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) uint64_t mma_bar[TC_STAGES];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gcount = count_dev != nullptr ? *count_dev : (zmax / bmax);
    // work of this CTA: (m0, n0) and the groups / batch entries z = blockIdx.z, blockIdx.z + gridDim.z, ...
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * TC_N;
    bool any = false;
    for (int z = blockIdx.z; z < zmax && !any; z += gridDim.z) {
        const int g = z / bmax, ib = z % bmax;
        if (g >= gcount) break;
        const GemmArgs& a = args[g];
        if ((a.acc ? (ib == 0) : (ib < a.nbatch)) && m0 < a.M && n0 < a.N) any = true;
    }
    if (!any) return;   // uniform: nothing for this CTA (no barrier or tensor memory touched)
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mma_bar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    uint32_t uses[TC_STAGES] = {0, 0};     // commits issued per stage (mbarrier phase = uses - 1)
    bool failed = false;
    for (int z = blockIdx.z; z < zmax && !failed; z += gridDim.z) {
        const int g = z / bmax, ib = z % bmax;
        if (g >= gcount) break;
        const GemmArgs a = args[g];
        if (a.acc ? (ib != 0) : (ib >= a.nbatch)) continue;
        const int M = a.M, N = a.N, K = a.K;
        if (m0 >= M || n0 >= N) continue;
        const int nb = a.acc ? a.nbatch : 1;
        const int kchunks = (K + TC_K - 1) / TC_K;
        int c = 0;
        for (int b = 0; b < nb && !failed; ++b) {
            const int bi = a.acc ? b : ib;
            const float* A = static_cast<const float*>(a.A) + (long long)bi * a.sA;
            const float* B = static_cast<const float*>(a.B) + (long long)bi * a.sB;
            for (int kc = 0; kc < kchunks; ++kc, ++c) {
                // stages alternate over all chunks of this CTA; the stage used here was last used two chunks ago
                // (by this tile or the previous one): wait for those MMAs before overwriting its operands
                const int st = (int)((uses[0] + uses[1]) & 1u);
                if (uses[st] > 0) {
                    const bool ok = mbar_wait(smem_addr(&mma_bar[st]), (uses[st] - 1) & 1u);
                    if (__syncthreads_or(!ok)) { failed = true; break; }
                }
                unsigned char* base = smem + st * TC_STAGE_BYTES;
                const int k0 = kc * TC_K;
                // op(A)[m][k]: A[m + k lda] (TA = false) or A[k + m lda] (TA = true)
                stage_tile<!TA>(base, base + TC_TILE_BYTES, A, a.lda, M, K, m0, k0, tid);
                // op(B)^T[n][k] = op(B)[k][n]: B[k + n ldb] (TB = false) or B[n + k ldb] (TB = true)
                stage_tile<TB>(base + 2 * TC_TILE_BYTES, base + 3 * TC_TILE_BYTES, B, a.ldb, N, K, n0, k0, tid);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_addr(base);
                    const uint64_t ahi = smem_desc(sa), alo = smem_desc(sa + TC_TILE_BYTES);
                    const uint64_t bhi = smem_desc(sa + 2 * TC_TILE_BYTES), blo = smem_desc(sa + 3 * TC_TILE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TC_K / 8; ++kk) {   // 8 TF32 values = 32 bytes per step: +2 in 16-byte units
                        const uint64_t d = (uint64_t)(2 * kk);
                        mma_tf32(tmem, ahi + d, bhi + d, (c > 0 || kk > 0) ? 1u : 0u);
                        mma_tf32(tmem, ahi + d, blo + d, 1u);
                        mma_tf32(tmem, alo + d, bhi + d, 1u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_addr(&mma_bar[st]))
                                 : "memory");
                }
                ++uses[st];
            }
        }
        if (failed) break;
        // all MMAs of this tile done: the last commit covers every earlier one
        {
            const int last = (int)((uses[0] + uses[1] - 1) & 1u);
            const bool ok = mbar_wait(smem_addr(&mma_bar[last]), (uses[last] - 1) & 1u);
            if (__syncthreads_or(!ok)) { failed = true; break; }
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: warp w reads lanes 32 (w mod 4) .. + 31 (rows) and columns 64 (w / 4) .. + 63
        {
            const int row = 32 * (warp & 3) + lane;
            const int cbase = 64 * (warp >> 2);
            float* C = static_cast<float*>(a.C) + (a.acc ? 0LL : (long long)ib * a.sC);
            const float alpha = (float)a.alpha, beta = (float)a.beta;
            const int m = m0 + row;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(cbase + 32 * h);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (m < M) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int nI = n0 + cbase + 32 * h + j;
                        if (nI < N) {
                            float* cp = C + m + (long long)nI * a.ldc;
                            float v = alpha * __uint_as_float(r[j]);
                            if (beta != 0.f) v += beta * (*cp);
                            *cp = v;
                        }
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // the accumulator is read out before the next tile's first MMA overwrites it
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (failed) {
        if (tid == 0) {
            atomicExch(&g_tc_error, 1);
            s_fail = 1;
        }
        // wait, bounded, for every committed MMA of this CTA before the tensor memory is released
        for (int s = 0; s < TC_STAGES; ++s)
            if (uses[s] > 0) (void)mbar_wait(smem_addr(&mma_bar[s]), (uses[s] - 1) & 1u);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

// shared-memory opt-in of the four kernel variants on the current device (outside any stream capture)
int tc_prepare() {
    TPCG_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(gemm_tc_kernel<false, false>),
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    TPCG_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(gemm_tc_kernel<false, true>),
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    TPCG_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(gemm_tc_kernel<true, false>),
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    TPCG_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(gemm_tc_kernel<true, true>),
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    return TPCG_OK;
}

template <bool TA, bool TB>
int launch_gemm_tc(const GemmArgs* args, const int* count_dev, int ngroups_max, int bmax, int Mmax, int Nmax,
                   cudaStream_t st) {
    if (ngroups_max <= 0 || bmax <= 0 || Mmax <= 0 || Nmax <= 0) return TPCG_OK;
    const long long zmax = (long long)ngroups_max * bmax;
    const long long gx = (Mmax + TC_M - 1) / TC_M, gy = (Nmax + TC_N - 1) / TC_N;
    // one CTA per SM (shared memory); the kernel strides over the groups, so the grid is capped at the SMs
    const long long zcap = std::max(1LL, (long long)sm_count() / std::max(1LL, gx * gy));
    const long long gz = std::min(std::min(zmax, zcap), 65535LL);
    if (gy > 65535 || zmax > (1LL << 30)) {
        set_error("tensor-core gemm grid too large");
        return TPCG_E_INVALID;
    }
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)gz);
    gemm_tc_kernel<TA, TB><<<grid, TC_THREADS, TC_SMEM, st>>>(args, count_dev, bmax, (int)zmax);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}
template int launch_gemm_tc<false, false>(const GemmArgs*, const int*, int, int, int, int, cudaStream_t);
template int launch_gemm_tc<false, true>(const GemmArgs*, const int*, int, int, int, int, cudaStream_t);
template int launch_gemm_tc<true, false>(const GemmArgs*, const int*, int, int, int, int, cudaStream_t);
template int launch_gemm_tc<true, true>(const GemmArgs*, const int*, int, int, int, int, cudaStream_t);

int tc_take_error() {
    int h = 0;
    if (cudaMemcpyFromSymbol(&h, g_tc_error, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    void* addr = nullptr;
    if (h && cudaGetSymbolAddress(&addr, g_tc_error) == cudaSuccess && addr) sync_zero(addr, sizeof(int));
    cudaGetLastError();
    return h;
}

}  // namespace tpcg
