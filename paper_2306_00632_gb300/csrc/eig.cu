// Symmetric eigensolver for the mode Grams of ST-HOSVD (Alg. 1 step 3) on GB300.
//
// GB300's FP64 pipe runs at about 1/60 of its FP32 rate, so a one-CTA FP64 Jacobi spends tens of
// milliseconds on a 128 x 128 Gram.  Instead:
//   1. cyclic Jacobi in FP32, matrix and vectors in shared memory, round-robin pairs (M/2 disjoint
//      rotations per step, closed-form schedule), stopped at the FP32 rounding floor;
//   2. FP64 form: refinement of the eigenvectors by the iteration of Ogita and Aishima (2018), whose work
//      is four FP64 GEMMs per step spread over many SMs (split-K) plus elementwise kernels;
//      FP32 form: no refinement (the tail energies are measured on the projected slices instead).
#include <math.h>

#include "common.cuh"
#include "eig.cuh"
#include "gemm.cuh"

namespace tpcg {

// ----------------------------------------------------------------------------------------------------
// FP32 Jacobi.  G (M x M, ld M, type Tin) -> V (M x M float, ld M, global), lam (M float).
// Shared memory holds A and V when 2 M^2 floats fit, else A only (V in global), else neither.
// ----------------------------------------------------------------------------------------------------
template <typename Tin>
__global__ void __launch_bounds__(1024) jacobi32_kernel(const int* __restrict__ Mdev, const Tin* __restrict__ G,
                                                        float* __restrict__ Vg, float* __restrict__ Ag,
                                                        float* __restrict__ lam, int max_sweeps, int smem_mode) {
    const int M = *Mdev;
    extern __shared__ float sm[];
    float* A = (smem_mode >= 1) ? sm : Ag;
    float* V = (smem_mode >= 2) ? sm + (size_t)M * M : Vg;
    __shared__ float cs[2 * 520];
    __shared__ double red[64];
    __shared__ int s_done;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (M <= 0) return;
    const long long MM = (long long)M * M;
    for (long long e = tid; e < MM; e += nt) {
        A[e] = (float)G[e];
        V[e] = ((e % M) == (e / M)) ? 1.0f : 0.0f;
    }
    __syncthreads();
    const int Mp = (M + 1) & ~1;
    const int half = Mp / 2;
    const int P = Mp - 1;               // players 0..Mp-1 on the round-robin polygon
    // stop once ||offdiag||_F <= tol ||diag||_F (FP32 rounding floor of the rotations)
    const double tol = 4.0 * M * 6.0e-8;
    for (int sweep = 0; sweep < max_sweeps && M > 1; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (long long e = tid; e < MM; e += nt) {
            const int i = (int)(e % M), j = (int)(e / M);
            const double v = A[e];
            if (i == j) dia += v * v; else off += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_down_sync(0xffffffffu, off, o);
            dia += __shfl_down_sync(0xffffffffu, dia, o);
        }
        if ((tid & 31) == 0) { red[tid >> 5] = off; red[32 + (tid >> 5)] = dia; }
        __syncthreads();
        if (tid == 0) {
            double so = 0, sd = 0;
            for (int w = 0; w < (nt >> 5); ++w) { so += red[w]; sd += red[32 + w]; }
            s_done = (so <= tol * tol * sd || so == 0.0) ? 1 : 0;
        }
        __syncthreads();
        if (s_done) break;
        for (int step = 0; step < P; ++step) {
            // pair k of this step: (P, step) for k = 0, else ((step + k) mod P, (step - k) mod P)
            for (int k = tid; k < half; k += nt) {
                int a, b;
                if (k == 0) { a = P; b = step; } else { a = (step + k) % P; b = (step - k + P) % P; }
                const int p = a < b ? a : b, q = a < b ? b : a;
                float c = 1.0f, s = 0.0f;
                if (q < M) {
                    const float apq = A[p + (long long)q * M];
                    const float app = A[p + (long long)p * M], aqq = A[q + (long long)q * M];
                    if (fabsf(apq) > 1e-30f && fabsf(apq) > 1e-9f * sqrtf(fabsf(app * aqq))) {
                        const float th = (aqq - app) / (2.0f * apq);
                        const float t = (th >= 0.0f ? 1.0f : -1.0f) / (fabsf(th) + sqrtf(th * th + 1.0f));
                        c = rsqrtf(t * t + 1.0f);
                        s = t * c;
                    }
                }
                cs[2 * k] = c;
                cs[2 * k + 1] = s;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (long long e = tid; e < (long long)half * M; e += nt) {
                const int k = (int)(e / M), j = (int)(e % M);
                const float s = cs[2 * k + 1];
                if (s == 0.0f) continue;
                int a, b;
                if (k == 0) { a = P; b = step; } else { a = (step + k) % P; b = (step - k + P) % P; }
                const int p = a < b ? a : b, q = a < b ? b : a;
                const float c = cs[2 * k];
                const float apj = A[p + (long long)j * M], aqj = A[q + (long long)j * M];
                A[p + (long long)j * M] = c * apj - s * aqj;
                A[q + (long long)j * M] = s * apj + c * aqj;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (long long e = tid; e < (long long)half * M; e += nt) {
                const int k = (int)(e / M), i = (int)(e % M);
                const float s = cs[2 * k + 1];
                if (s == 0.0f) continue;
                int a, b;
                if (k == 0) { a = P; b = step; } else { a = (step + k) % P; b = (step - k + P) % P; }
                const int p = a < b ? a : b, q = a < b ? b : a;
                const float c = cs[2 * k];
                const float aip = A[i + (long long)p * M], aiq = A[i + (long long)q * M];
                A[i + (long long)p * M] = c * aip - s * aiq;
                A[i + (long long)q * M] = s * aip + c * aiq;
                const float vip = V[i + (long long)p * M], viq = V[i + (long long)q * M];
                V[i + (long long)p * M] = c * vip - s * viq;
                V[i + (long long)q * M] = s * vip + c * viq;
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < M; i += nt) lam[i] = A[i + (long long)i * M];
    if (smem_mode >= 2)
        for (long long e = tid; e < MM; e += nt) Vg[e] = V[e];
}

int jacobi32_smem_mode(int n, size_t* bytes) {
    const size_t nn = (size_t)n * n * sizeof(float);
    if (2 * nn <= 200 * 1024) { *bytes = 2 * nn; return 2; }
    if (nn <= 200 * 1024) { *bytes = nn; return 1; }
    *bytes = 0;
    return 0;
}

template <typename Tin>
int launch_jacobi32(const int* Mdev, const Tin* G, float* V, float* Ascratch, float* lam, int n, cudaStream_t st) {
    size_t bytes;
    const int mode = jacobi32_smem_mode(n, &bytes);
    static bool attr_set[2] = {false, false};
    const int ti = sizeof(Tin) == 8 ? 0 : 1;
    if (!attr_set[ti]) {
        cudaFuncSetAttribute(jacobi32_kernel<Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
        attr_set[ti] = true;
    }
    jacobi32_kernel<Tin><<<1, 1024, bytes, st>>>(Mdev, G, V, Ascratch, lam, 40, mode);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}
template int launch_jacobi32<double>(const int*, const double*, float*, float*, float*, int, cudaStream_t);
template int launch_jacobi32<float>(const int*, const float*, float*, float*, float*, int, cudaStream_t);

// ----------------------------------------------------------------------------------------------------
// FP64 refinement (Ogita & Aishima 2018).  For symmetric A and approximate eigenvectors X:
//   R = I - X^T X,  S = X^T A X,  lam_i = S_ii / (1 - R_ii),
//   delta = 2 (||S - diag(lam)||_F + ||A||_F ||R||_F),
//   E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)  if |lam_i - lam_j| > delta,  else R_ij / 2,
//   X <- X + X E.
// Work buffers (M x M doubles, ld M): X, XtX, AX, S, E; lam (M doubles).
// ----------------------------------------------------------------------------------------------------
__global__ void refine_plan_kernel(const int* __restrict__ Mdev, const double* A, double* X, double* XtX, double* AX,
                                   double* S, double* E, double* Xn, double* Part, GemmArgs* ga, int* counts,
                                   int nsplit) {
    if (threadIdx.x != 0) return;
    const int M = *Mdev;
    const long long MM = (long long)M * M;
    int ns = nsplit;
    if (ns > M) ns = M > 0 ? M : 1;
    const int chunk = M > 0 ? (M + ns - 1) / ns : 0;
    int used = 0;
    // groups [0, ns): XtX partials; [64, 64+ns): AX partials; [128, 128+ns): S partials; [192]: X E
    for (int g = 0; g < ns; ++g) {
        const int lo = g * chunk;
        int hi = lo + chunk;
        if (hi > M) hi = M;
        if (lo >= hi) break;
        GemmArgs a{};
        a.M = M; a.N = M; a.K = hi - lo; a.nbatch = 1; a.alpha = 1.0;
        a.A = X + lo; a.lda = M; a.B = X + lo; a.ldb = M;          // (X^T X): TN over rows lo..hi
        a.C = Part + (long long)used * MM; a.ldc = M;
        ga[g] = a;
        GemmArgs b{};
        b.M = M; b.N = M; b.K = hi - lo; b.nbatch = 1; b.alpha = 1.0;
        b.A = A + (long long)lo * M; b.lda = M; b.B = X + lo; b.ldb = M;   // A X: NN over k = lo..hi
        b.C = Part + (long long)(ns + used) * MM; b.ldc = M;
        ga[64 + g] = b;
        GemmArgs c{};
        c.M = M; c.N = M; c.K = hi - lo; c.nbatch = 1; c.alpha = 1.0;
        c.A = X + lo; c.lda = M; c.B = AX + lo; c.ldb = M;         // X^T (A X): TN
        c.C = Part + (long long)used * MM; c.ldc = M;
        ga[128 + g] = c;
        ++used;
    }
    GemmArgs d{};
    d.M = M; d.N = M; d.K = M; d.nbatch = 1; d.alpha = 1.0; d.beta = 1.0;
    d.A = X; d.lda = M; d.B = E; d.ldb = M; d.C = Xn; d.ldc = M;   // Xn (= X on entry) += X E
    ga[192] = d;
    counts[0] = used;
    counts[1] = M;
    counts[2] = M;
}

__global__ void refine_e_kernel(const int* __restrict__ Mdev, const double* __restrict__ A, const double* __restrict__ XtX,
                                const double* __restrict__ S, double* __restrict__ E, double* __restrict__ lam,
                                const double* __restrict__ X, double* __restrict__ Xn) {
    const int M = *Mdev;
    const long long MM = (long long)M * M;
    __shared__ double red[3][32];
    __shared__ double s_delta;
    // lam_i and the norms for delta (one CTA computes them; all CTAs recompute redundantly: M <= 1024)
    double sa = 0, ss = 0, sr = 0;
    for (long long e = threadIdx.x; e < MM; e += blockDim.x) {
        const int i = (int)(e % M), j = (int)(e / M);
        const double r = (i == j ? 1.0 : 0.0) - XtX[e];
        sa += A[e] * A[e];
        sr += r * r;
        if (i != j) ss += S[e] * S[e];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        sr += __shfl_down_sync(0xffffffffu, sr, o);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = sa; red[1][w] = ss; red[2][w] = sr; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, s = 0, r = 0;
        for (int q = 0; q < nw; ++q) { a += red[0][q]; s += red[1][q]; r += red[2][q]; }
        s_delta = 2.0 * (sqrt(s) + sqrt(a) * sqrt(r));
    }
    __syncthreads();
    const double delta = s_delta;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MM; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % M), j = (int)(e / M);
        const double rij = (i == j ? 1.0 : 0.0) - XtX[e];
        const double li = S[i + (long long)i * M] / (1.0 - (1.0 - XtX[i + (long long)i * M]));
        const double lj = S[j + (long long)j * M] / (1.0 - (1.0 - XtX[j + (long long)j * M]));
        double eij;
        if (i == j) eij = rij * 0.5;
        else if (fabs(li - lj) > delta) eij = (S[e] + lj * rij) / (lj - li);
        else eij = rij * 0.5;
        E[e] = eij;
        Xn[e] = X[e];
        if (i == j) lam[i] = li;
    }
}

__global__ void copy_f2d_kernel(const int* __restrict__ Mdev, const float* __restrict__ src, double* __restrict__ dst) {
    const int M = *Mdev;
    const long long MM = (long long)M * M;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MM; e += (long long)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

int refine_eig64(const int* Mdev, const double* A, const float* V32, int n, EigWork& w, int iters, cudaStream_t st) {
    const int nsplit = 32;
    copy_f2d_kernel<<<64, 256, 0, st>>>(Mdev, V32, w.X);
    TPCG_CHECK_LAUNCH();
    for (int it = 0; it < iters; ++it) {
        refine_plan_kernel<<<1, 32, 0, st>>>(Mdev, A, w.X, w.XtX, w.AX, w.S, w.E, w.Xn, w.Part, w.ga, w.counts, nsplit);
        TPCG_CHECK_LAUNCH();
        // X^T X
        TPCG_TRY((launch_gemm<double, true, false>(w.ga, w.counts, nsplit, 1, n, n, st)));
        reduce_partials_kernel<double><<<64, 256, 0, st>>>(w.Part, w.counts + 1, w.counts + 2, w.counts, w.XtX, 0, 1.0, 0.0);
        TPCG_CHECK_LAUNCH();
        // A X
        TPCG_TRY((launch_gemm<double, false, false>(w.ga + 64, w.counts, nsplit, 1, n, n, st)));
        reduce_partials_kernel<double><<<64, 256, 0, st>>>(w.Part + (size_t)nsplit * n * n, w.counts + 1, w.counts + 2,
                                                           w.counts, w.AX, 0, 1.0, 0.0);
        TPCG_CHECK_LAUNCH();
        // S = X^T (A X)
        TPCG_TRY((launch_gemm<double, true, false>(w.ga + 128, w.counts, nsplit, 1, n, n, st)));
        reduce_partials_kernel<double><<<64, 256, 0, st>>>(w.Part, w.counts + 1, w.counts + 2, w.counts, w.S, 0, 1.0, 0.0);
        TPCG_CHECK_LAUNCH();
        refine_e_kernel<<<32, 256, 0, st>>>(Mdev, A, w.XtX, w.S, w.E, w.lam, w.X, w.Xn);
        TPCG_CHECK_LAUNCH();
        // Xn = X + X E, then swap roles
        TPCG_TRY((launch_gemm<double, false, false>(w.ga + 192, nullptr, 1, 1, n, n, st)));
        double* t = w.X; w.X = w.Xn; w.Xn = t;
    }
    // final Rayleigh quotients of the refined vectors: lam_i = (X^T A X)_ii / (X^T X)_ii
    refine_plan_kernel<<<1, 32, 0, st>>>(Mdev, A, w.X, w.XtX, w.AX, w.S, w.E, w.Xn, w.Part, w.ga, w.counts, nsplit);
    TPCG_CHECK_LAUNCH();
    TPCG_TRY((launch_gemm<double, true, false>(w.ga, w.counts, nsplit, 1, n, n, st)));
    reduce_partials_kernel<double><<<64, 256, 0, st>>>(w.Part, w.counts + 1, w.counts + 2, w.counts, w.XtX, 0, 1.0, 0.0);
    TPCG_CHECK_LAUNCH();
    TPCG_TRY((launch_gemm<double, false, false>(w.ga + 64, w.counts, nsplit, 1, n, n, st)));
    reduce_partials_kernel<double><<<64, 256, 0, st>>>(w.Part + (size_t)nsplit * n * n, w.counts + 1, w.counts + 2,
                                                       w.counts, w.AX, 0, 1.0, 0.0);
    TPCG_CHECK_LAUNCH();
    TPCG_TRY((launch_gemm<double, true, false>(w.ga + 128, w.counts, nsplit, 1, n, n, st)));
    reduce_partials_kernel<double><<<64, 256, 0, st>>>(w.Part, w.counts + 1, w.counts + 2, w.counts, w.S, 0, 1.0, 0.0);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}

size_t eig_work_bytes(int n) {
    const size_t nn = (size_t)n * n;
    return nn * 8 * 6 + n * 8 + 64 * nn * 8 + 256 * sizeof(GemmArgs) + 64 + nn * 4 * 2 + n * 4 + n * 8 + n * 4;
}

int eig_work_alloc(EigWork* w, int n, std::vector<void*>* owned) {
    const size_t nn = (size_t)n * n;
    auto get = [&](void** p, size_t bytes) -> int {
        if (cudaMalloc(p, bytes < 16 ? 16 : bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("eig workspace: cudaMalloc failed");
            return TPCG_E_NOMEM;
        }
        owned->push_back(*p);
        return TPCG_OK;
    };
    TPCG_TRY(get((void**)&w->X, nn * 8));
    TPCG_TRY(get((void**)&w->Xn, nn * 8));
    TPCG_TRY(get((void**)&w->XtX, nn * 8));
    TPCG_TRY(get((void**)&w->AX, nn * 8));
    TPCG_TRY(get((void**)&w->S, nn * 8));
    TPCG_TRY(get((void**)&w->E, nn * 8));
    TPCG_TRY(get((void**)&w->lam, (size_t)n * 8));
    TPCG_TRY(get((void**)&w->Part, 64 * nn * 8));
    TPCG_TRY(get((void**)&w->ga, 256 * sizeof(GemmArgs)));
    TPCG_TRY(get((void**)&w->counts, 64));
    TPCG_TRY(get((void**)&w->V32, nn * 4));
    TPCG_TRY(get((void**)&w->A32, nn * 4));
    TPCG_TRY(get((void**)&w->lam32, (size_t)n * 4));
    TPCG_TRY(get((void**)&w->energy, (size_t)n * 8));
    TPCG_TRY(get((void**)&w->order, (size_t)n * 4));
    return TPCG_OK;
}

}  // namespace tpcg
