// Relative-tolerance truncation of a Tucker tensor (Alg. 1 with ST-HOSVD), device-driven.
//
//   step 1  QR of each factor Y_t (n x k_t).  When k_t >= n any orthonormal Q_t spanning R^n serves, so
//           Q_t = I and R_t = Y_t (no work); otherwise a Householder QR in one CTA per mode.
//   step 2  Z = sum_b scale_b G_b x_1 R_1^(b) x_2 R_2^(b) x_3 R_3^(b) over the core blocks b
//           (block-diagonal core): per block the middle mode on the small core, then mode 1, writing
//           the block's slab of a stacked matrix W; one fused GEMM over all blocks contracts mode 3.
//   step 3  ST-HOSVD of Z, modes 1, 2, 3 in order: Gram of the unfolding (split-K GEMM + ordered
//           reduction), Jacobi eigensolver, keep the smallest s_m whose discarded eigenvalues sum to
//           <= eps^2 ||Z||^2 / 3 (clipped by the rank cap), project Z x_m S_m^T.
//   step 4  new factors Q_t S_t, new core, descriptor of a plain tensor.
//
// Every shape is read from device memory (descriptor, RoundPlan, GemmArgs), so the host enqueues a fixed
// sequence of launches without synchronising.
#include <math.h>

#include <string>

#include "common.cuh"
#include "gemm.cuh"
#include "eig.cuh"
#include "kernels.cuh"

namespace tpcg {

// --------------------------------------------------------------------------------------------------
// Planner: descriptor -> plan and the GEMM arguments of step 2.
// gargs layout: [0, MAXB) middle-mode products, [MAXB, 2 MAXB) mode-1 products, [2 MAXB] fused mode 3.
// --------------------------------------------------------------------------------------------------
template <typename T>
__global__ void plan_round_kernel(const TuckerDesc* __restrict__ d, RoundPlan* plan, GemmArgs* ga, int n,
                                  int cap, double eps_host, const double* eps_dev, void* Rq0, void* Rq1,
                                  void* Rq2, const void* U0, const void* U1, const void* U2, T* T1, T* Wm,
                                  int* counts, long long t1cap, double* prof, int strict_mode, void* Zout) {
    if (threadIdx.x != 0) return;
    RoundPlan p;
    p.n = n;
    p.nblk = d->nblk;
    void* Rq[3] = {Rq0, Rq1, Rq2};
    const void* U[3] = {U0, U1, U2};
    for (int t = 0; t < 3; ++t) {
        p.k[t] = d->rank[t];
        p.useQ[t] = (p.k[t] < n) ? 1 : 0;
        p.kp[t] = p.k[t] < n ? p.k[t] : n;
        p.Rp[t] = p.useQ[t] ? (const void*)Rq[t] : U[t];
        p.ldR[t] = n;
        p.s[t] = 0;
        p.zdim[t] = p.kp[t];
    }
    p.cap = cap;
    p.eps = eps_dev ? *eps_dev : eps_host;
    p.norm2 = 0.0;
    p.discarded = 0.0;
    p.budget = 0.0;
    p.abs2 = 0.0;
    p.status = 0;
    // below eps ~ 1e-7 the budget eps^2 ||Z||^2 / 3 is under what an FP64 Gram resolves (the Gram squares the
    // singular values): the rule then keeps every direction it cannot certify as small enough
    p.strict = strict_mode >= 0 ? strict_mode : (p.eps < 1e-7 ? 1 : 0);
    p.kz3 = p.k[2];
    p.nsplit = 0;
    const int kp1 = p.kp[0], kp2 = p.kp[1];
    long long t1off = 0;
    for (int b = 0; b < p.nblk; ++b) {
        const BlockDesc& B = d->blk[b];
        const int r1 = B.r[0], r2 = B.r[1], r3 = B.r[2];
        // middle mode on the core: U_b[:, :, j3] (r1 x kp2) = G_b[:, :, j3] (r1 x r2) R_2b^T
        GemmArgs a{};
        a.M = r1; a.N = kp2; a.K = r2; a.nbatch = r3; a.acc = 0;
        a.A = B.core; a.lda = r1; a.sA = (long long)r1 * r2;
        a.B = static_cast<const T*>(p.Rp[1]) + (long long)B.off[1] * p.ldR[1]; a.ldb = p.ldR[1]; a.sB = 0;
        a.C = T1 + t1off; a.ldc = r1; a.sC = (long long)r1 * kp2;
        a.alpha = 1.0; a.beta = 0.0;
        if (r1 == 0 || r2 == 0 || r3 == 0) { a.M = 0; a.nbatch = 0; }
        ga[b] = a;
        // mode 1: V_b (kp1 x kp2 r3) = R_1b (kp1 x r1) U_b(1) (r1 x kp2 r3), scaled by the block scale
        GemmArgs c{};
        c.M = kp1; c.N = kp2 * r3; c.K = r1; c.nbatch = 1; c.acc = 0;
        c.A = static_cast<const T*>(p.Rp[0]) + (long long)B.off[0] * p.ldR[0]; c.lda = p.ldR[0]; c.sA = 0;
        c.B = T1 + t1off; c.ldb = r1; c.sB = 0;
        c.C = Wm + (long long)B.off[2] * kp1 * kp2; c.ldc = kp1; c.sC = 0;
        c.alpha = B.scale; c.beta = 0.0;
        if (r1 == 0 || r2 == 0 || r3 == 0) { c.M = 0; }
        ga[TPCG_MAX_BLOCKS + b] = c;
        t1off += (long long)r1 * kp2 * r3;
    }
    // fused mode 3: Z (kp1 kp2 x kp3) = W (kp1 kp2 x k3) R_3^T
    GemmArgs z{};
    z.M = kp1 * kp2; z.N = p.kp[2]; z.K = p.k[2]; z.nbatch = 1; z.acc = 0;
    z.A = Wm; z.lda = (long long)kp1 * kp2; z.sA = 0;
    z.B = p.Rp[2]; z.ldb = p.ldR[2]; z.sB = 0;
    z.C = Zout;
    z.ldc = (long long)kp1 * kp2; z.sC = 0;
    z.alpha = 1.0; z.beta = 0.0;
    ga[2 * TPCG_MAX_BLOCKS] = z;
    counts[0] = p.nblk;
    if (prof) {
        const double e = sizeof(T);
        const double M3 = (double)kp1 * kp2, K3 = p.k[2], N3 = p.kp[2];
        prof[2 * PK_ZGEMM] += 2.0 * M3 * N3 * K3;
        prof[2 * PK_ZGEMM + 1] += e * (M3 * K3 + N3 * K3 + M3 * N3);
        double fb = 0;
        for (int b = 0; b < p.nblk; ++b) {
            const BlockDesc& B = d->blk[b];
            fb += 2.0 * B.r[0] * kp2 * B.r[2] * B.r[1] + 2.0 * kp1 * kp2 * B.r[2] * B.r[0];
        }
        prof[2 * PK_ZBLK] += fb;
    }
    if (t1off > t1cap) {   // workspace too small for these blocks: produce nothing, flag the plan
        p.status = 1;
        counts[0] = 0;
        ga[2 * TPCG_MAX_BLOCKS].M = 0;
        for (int t = 0; t < 3; ++t) p.zdim[t] = 0;
    }
    *plan = p;
}

// --------------------------------------------------------------------------------------------------
// Householder QR of Y_t (n x k, k < n), one CTA per mode:  Y_t = Q_t R_t, Q_t n x k, R_t k x k.
// --------------------------------------------------------------------------------------------------
template <typename T>
__device__ T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = (lane < nw) ? red[lane] : T(0);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[32] = v;
    }
    __syncthreads();
    T r = red[32];
    __syncthreads();
    return r;
}

// Householder QR of Y (rows x k, column stride ld, k <= rows) by one CTA: A <- Y is the working copy; R (k x k,
// upper triangle, ld ldr) when R is non-null; Q = H_0 ... H_{k-1} [I; 0] (rows x k, ld ld).  tau holds k scalars
// and red 33 of shared memory.
template <typename T>
__device__ void householder_qr(const T* Y, T* A, T* R, T* Q, int rows, int k, long long ld, long long ldr, T* tau,
                               T* red, T* s_beta) {
    for (long long e = threadIdx.x; e < (long long)rows * k; e += blockDim.x) {
        const long long i = e % rows, c = e / rows;
        A[i + c * ld] = Y[i + c * ld];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < k; ++j) {
        // Householder vector of A[j:rows, j] (LAPACK larfg convention: v[0] = 1, R[j,j] = beta)
        T part = T(0);
        for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) part += A[i + j * ld] * A[i + j * ld];
        T sig = block_sum(part, red);
        const T alpha0 = A[j + j * ld];
        T beta, tj, scal;
        if (sig == T(0)) {
            tj = T(0); beta = alpha0; scal = T(0);
        } else {
            T nrm = sqrt(alpha0 * alpha0 + sig);
            beta = alpha0 >= T(0) ? -nrm : nrm;
            tj = (beta - alpha0) / beta;
            scal = T(1) / (alpha0 - beta);
        }
        for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) A[i + j * ld] *= scal;
        if (threadIdx.x == 0) { tau[j] = tj; *s_beta = beta; }
        __syncthreads();
        // apply H_j to the trailing columns, one warp per column
        if (tj != T(0)) {
            for (int c = j + 1 + wid; c < k; c += nw) {
                T* col = A + c * ld;
                const T* v = A + j * ld;
                T w = T(0);
                for (int i = j + lane; i < rows; i += 32) w += (i == j ? T(1) : v[i]) * col[i];
                for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                w *= tj;
                for (int i = j + lane; i < rows; i += 32) col[i] -= w * (i == j ? T(1) : v[i]);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) A[j + j * ld] = *s_beta;
        __syncthreads();
    }
    if (R) {
        for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x) {
            const int i = (int)(e % k), c = (int)(e / k);
            R[i + c * ldr] = (i <= c) ? A[i + c * ld] : T(0);
        }
    }
    // Q = H_0 H_1 ... H_{k-1} [I; 0], accumulated backwards
    for (long long e = threadIdx.x; e < (long long)rows * k; e += blockDim.x) {
        const int i = (int)(e % rows), c = (int)(e / rows);
        Q[i + (long long)c * ld] = (i == c) ? T(1) : T(0);
    }
    __syncthreads();
    for (int j = k - 1; j >= 0; --j) {
        const T tj = tau[j];
        if (tj != T(0)) {
            for (int c = j + wid; c < k; c += nw) {
                T* col = Q + c * ld;
                const T* v = A + j * ld;
                T w = T(0);
                for (int i = j + lane; i < rows; i += 32) w += (i == j ? T(1) : v[i]) * col[i];
                for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                w *= tj;
                for (int i = j + lane; i < rows; i += 32) col[i] -= w * (i == j ? T(1) : v[i]);
            }
        }
        __syncthreads();
    }
}

// Alg. 1 step 1: Y_t = Q_t R_t for the modes with k_t < n, one CTA per mode (n x k_t, ld n)
template <typename T>
__global__ void __launch_bounds__(1024) qr_kernel(const RoundPlan* __restrict__ plan, const T* Y0, const T* Y1,
                                                  const T* Y2, T* W0, T* W1, T* W2, T* R0, T* R1, T* R2, T* Q0,
                                                  T* Q1, T* Q2) {
    const int t = blockIdx.x;
    const RoundPlan& p = *plan;
    if (!p.useQ[t]) return;
    const int n = p.n, k = p.k[t];
    extern __shared__ unsigned char smem_raw[];
    T* tau = reinterpret_cast<T*>(smem_raw);      // k
    T* red = tau + n;                              // 33
    __shared__ T s_beta;
    householder_qr<T>(t == 0 ? Y0 : (t == 1 ? Y1 : Y2), t == 0 ? W0 : (t == 1 ? W1 : W2),
                      t == 0 ? R0 : (t == 1 ? R1 : R2), t == 0 ? Q0 : (t == 1 ? Q1 : Q2), n, k, n, n, tau, red,
                      &s_beta);
}

// --------------------------------------------------------------------------------------------------
// Gram of the mode-m unfolding of the working tensor (dims in plan.zdim): split into groups whose
// partial Grams are summed in a fixed order (deterministic).
//   m = 0: G = Z_(1) Z_(1)^T        (NT, K = d2 d3 split)
//   m = 1: G = sum_i3 Z_i3^T Z_i3   (TN, slices i3 grouped)
//   m = 2: G = Zmat^T Zmat          (TN, K = d1 d2 split)
// --------------------------------------------------------------------------------------------------
template <typename T>
__device__ void plan_gram(RoundPlan& p, GemmArgs* ga, const T* Zc, T* Part, int m, int nsplit_max, int min_k,
                          int* counts, double* prof) {
    const int d1 = p.zdim[0], d2 = p.zdim[1], d3 = p.zdim[2];
    const int M = p.zdim[m];
    int total = (m == 0) ? d2 * d3 : (m == 1 ? d3 : d1 * d2);
    if (prof) {
        prof[2 * PK_GRAM] += 2.0 * M * M * ((double)d1 * d2 * d3 / (M > 0 ? M : 1));
        prof[2 * PK_GRAM + 1] += sizeof(T) * ((double)d1 * d2 * d3 + (double)M * M);
    }
    int ns = total < nsplit_max ? total : nsplit_max;
    if (min_k > 0) {   // at least min_k of the reduction per group: fewer, longer groups (less partial traffic)
        const long long ktot = (long long)total * (m == 1 ? d1 : 1);
        const long long cap_k = ktot / min_k;
        if (cap_k < ns) ns = (int)cap_k;
    }
    if (ns < 1) ns = 1;
    if (M == 0 || total == 0) ns = 0;
    const int chunk = ns ? (total + ns - 1) / ns : 0;
    int used = 0;
    for (int g = 0; g < ns; ++g) {
        const int lo = g * chunk;
        int hi = lo + chunk;
        if (hi > total) hi = total;
        if (lo >= hi) break;
        GemmArgs a{};
        a.M = M; a.N = M; a.alpha = 1.0; a.beta = 0.0;
        a.C = Part + (long long)used * M * M; a.ldc = M; a.sC = 0;
        if (m == 0) {
            a.K = hi - lo; a.nbatch = 1; a.acc = 0;
            a.A = Zc + (long long)lo * d1; a.lda = d1; a.sA = 0;
            a.B = Zc + (long long)lo * d1; a.ldb = d1; a.sB = 0;
        } else if (m == 1) {
            a.K = d1; a.nbatch = hi - lo; a.acc = 1;
            a.A = Zc + (long long)lo * d1 * d2; a.lda = d1; a.sA = (long long)d1 * d2;
            a.B = Zc + (long long)lo * d1 * d2; a.ldb = d1; a.sB = (long long)d1 * d2;
        } else {
            a.K = hi - lo; a.nbatch = 1; a.acc = 0;
            a.A = Zc + lo; a.lda = (long long)d1 * d2; a.sA = 0;
            a.B = Zc + lo; a.ldb = (long long)d1 * d2; a.sB = 0;
        }
        ga[used++] = a;
    }
    p.nsplit = used;
    p.gm = m;
    p.gM = M;
    p.eM = M;
    p.rr = 0;
    counts[0] = used;
    counts[1] = M;
    counts[2] = M;
}

template <typename T>
__global__ void plan_gram_kernel(RoundPlan* plan, GemmArgs* ga, const T* Zc, T* Part, int m, int nsplit_max,
                                 int min_k, int* counts, double* prof) {
    if (threadIdx.x == 0) plan_gram<T>(*plan, ga, Zc, Part, m, nsplit_max, min_k, counts, prof);
}

// --------------------------------------------------------------------------------------------------
// Projection Z x_m S_m^T onto the s_m kept eigenvectors of mode m (the truncation rule itself runs in the
// eigensolver, eig.cu).
// --------------------------------------------------------------------------------------------------
__device__ void plan_projection(RoundPlan& p, GemmArgs* ga, const void* S, long long ldS, const void* Zc, void* Znext,
                                int m, int s) {
    const int d1 = p.zdim[0], d2 = p.zdim[1], d3 = p.zdim[2];
    GemmArgs a{};
    a.alpha = 1.0; a.beta = 0.0; a.nbatch = 1; a.acc = 0;
    if (m == 0) {        // S^T Z_(1)
        a.M = s; a.N = d2 * d3; a.K = d1;
        a.A = S; a.lda = ldS; a.B = Zc; a.ldb = d1 > 0 ? d1 : 1; a.C = Znext; a.ldc = s > 0 ? s : 1;
    } else if (m == 1) { // per slice: Z_i3 S
        a.M = d1; a.N = s; a.K = d2; a.nbatch = d3;
        a.A = Zc; a.lda = d1 > 0 ? d1 : 1; a.sA = (long long)d1 * d2;
        a.B = S; a.ldb = ldS; a.sB = 0;
        a.C = Znext; a.ldc = d1 > 0 ? d1 : 1; a.sC = (long long)d1 * s;
    } else {             // Zmat S
        a.M = d1 * d2; a.N = s; a.K = d3;
        a.A = Zc; a.lda = (long long)d1 * d2 > 0 ? (long long)d1 * d2 : 1; a.B = S; a.ldb = ldS; a.C = Znext;
        a.ldc = a.lda;
    }
    ga[0] = a;
}

// plan of the projection onto the kept eigenvectors (after the eigensolver set plan.s[m]) into gp; the working
// tensor's mode m shrinks to s_m, and for m < 2 the Gram of mode m + 1 of the projected tensor is planned into
// gg (a separate argument range: the projection's product runs first)
template <typename T>
__global__ void plan_proj_kernel(RoundPlan* plan, GemmArgs* gp, const T* S, const T* Zc, T* Znext, int m,
                                 GemmArgs* gg, T* Part, int nsplit_max, int min_k, int* counts, double* prof) {
    if (threadIdx.x != 0) return;
    RoundPlan& p = *plan;
    plan_projection(p, gp, S, p.n, Zc, Znext, m, p.s[m]);
    p.zdim[m] = p.s[m];
    if (m < 2) plan_gram<T>(p, gg, Znext, Part, m + 1, nsplit_max, min_k, counts, prof);
}

// --------------------------------------------------------------------------------------------------
// Rayleigh-Ritz reduction of a Gram G of order gM > RR_L (contexts with n > RR_L and a rank cap of at most
// RR_MAXCAP) to at most RR_L columns before the eigensolver:
//  1. pivoted Cholesky G = L L^T + S (diagonal pivoting, left-looking, one column per step) until the trace of
//     the Schur complement S is at most 1% (FP32) or 1e-8 (FP64) of this mode's truncation budget, or RR_L
//     columns;
//  2. Q = qr(L) (gM x rc), B = Q^T G Q (rc x rc) replaces G as the eigensolver's input, and the kept Ritz
//     vectors Q U are written back.
// The truncation rule is charged against trace(G).  For orthonormal kept vectors the discarded energy
// ||Z - S S^T Z||^2 = trace(G) - sum of the kept Ritz values exactly, so Alg. 1's bound holds.  The Ritz
// values of range(L) miss at most trace(S) of G's energy in total (Q^T G Q >= Q^T L L^T Q, whose trace is
// trace(G) - trace(S)), so the ranks are those of the exact rule up to that fraction of the budget.  When RR_L columns do
// not reach the 1% (slowly decaying spectra) the remainder counts as discarded and the rule keeps at most RR_L
// columns, more than the rank cap.  A Gram of order <= RR_L goes to the eigensolver unchanged.
// --------------------------------------------------------------------------------------------------
constexpr int RR_THREADS = 1024;

template <typename T>
__global__ void __launch_bounds__(RR_THREADS) rr_pchol_kernel(RoundPlan* plan, const T* __restrict__ G, T* Lf,
                                                               double* prof) {
    RoundPlan& p = *plan;
    const int M = p.gM, n = p.n, m = p.gm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = RR_THREADS / 32;
    extern __shared__ __align__(16) unsigned char rr_smem[];
    T* dg = reinterpret_cast<T*>(rr_smem);            // remaining diagonal (M entries; -1 once pivoted)
    T* prow = dg + n;                                   // row piv of L (RR_L entries)
    __shared__ T wbest[NW], wsum[NW];
    __shared__ int wbi[NW];
    __shared__ double s_tr, wtr[NW];
    if (M <= RR_L) {   // small Gram: the eigensolver takes it as it is
        if (tid == 0) { p.rr = 0; p.eM = M; }
        return;
    }
    double t = 0.0;
    for (int i = tid; i < M; i += RR_THREADS) {
        const T d = G[i + (long long)i * M];
        dg[i] = d;
        t += (double)d;
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) wtr[warp] = t;
    __syncthreads();
    if (tid == 0) {
        double tr = 0.0;
        for (int w = 0; w < NW; ++w) tr += wtr[w];   // fixed order: deterministic
        s_tr = tr;
        p.gtrace = tr;
        if (m == 0) {   // the budget of every mode comes from ||Z||^2 = trace of the first Gram
            p.norm2 = tr;
            p.budget = fmax(p.eps * p.eps * tr, p.abs2) / 3.0;
        }
    }
    __syncthreads();
    const double tr = s_tr;
    // FP32: 1% of the budget (the FP32 Gram resolves no finer); FP64: 1e-8 of it, which puts the Ritz vectors of
    // the kept directions within about 1e-4 eps of the eigenvectors (a direction u_j of eigenvalue lambda_j has
    // at most trace(S) / lambda_j of its square outside range(L))
    const T thr = (T)((sizeof(T) == 8 ? 1e-15 : 1e-9) * tr);
    const T stop_rem = (T)fmax((double)thr, (sizeof(T) == 8 ? 1e-8 : 1e-2) * p.budget);
    int rc = 0;
    for (int k = 0; k < RR_L; ++k) {
        // the largest remaining diagonal entry (ties: the lowest index) and the remaining trace
        T v = (T)-2, sm = (T)0;
        int bi = 0x7fffffff;
        for (int i = tid; i < M; i += RR_THREADS) {
            const T d = dg[i];
            if (d > v) { v = d; bi = i; }
            sm += d > (T)0 ? d : (T)0;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const T v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int b2 = __shfl_xor_sync(0xffffffffu, bi, o);
            sm += __shfl_xor_sync(0xffffffffu, sm, o);
            if (v2 > v || (v2 == v && b2 < bi)) { v = v2; bi = b2; }
        }
        if (lane == 0) { wbest[warp] = v; wbi[warp] = bi; wsum[warp] = sm; }
        __syncthreads();
        T dmax = (T)-2, rem = (T)0;
        int piv = 0;
        for (int w = 0; w < NW; ++w) {
            rem += wsum[w];
            if (wbest[w] > dmax || (wbest[w] == dmax && wbi[w] < piv)) { dmax = wbest[w]; piv = wbi[w]; }
        }
        // the same decision in every thread (a NaN stops the factorisation)
        if (!(dmax > thr) || !(rem > stop_rem)) break;
        for (int j = tid; j < k; j += RR_THREADS) prow[j] = Lf[piv + (long long)j * n];
        __syncthreads();
        const T r = sqrt(dmax);
        const T inv = (T)1 / r;
        for (int i = tid; i < M; i += RR_THREADS) {
            T l;
            if (i == piv) {
                l = r;
            } else if (dg[i] < (T)0) {   // pivoted earlier: its Schur complement row is zero
                l = (T)0;
            } else {
                T acc = G[i + (long long)piv * M];
                for (int j = 0; j < k; ++j) acc -= Lf[i + (long long)j * n] * prow[j];
                l = acc * inv;
            }
            Lf[i + (long long)k * n] = l;
            dg[i] = (i == piv) ? (T)-1 : (dg[i] < (T)0 ? dg[i] : dg[i] - l * l);
        }
        __syncthreads();
        rc = k + 1;
    }
    if (tid == 0) {
        p.rr = 1;
        p.eM = rc;
        if (prof) {   // Cholesky columns, QR of the basis, G Q, Q^T (G Q) and Q U (U counted as rc columns)
            const double mm = M, l = rc;
            prof[2 * PK_EIG] += mm * l * l + 4.0 * mm * l * l + 2.0 * mm * mm * l + 4.0 * mm * l * l;
            prof[2 * PK_EIG + 1] += sizeof(T) * (2.0 * mm * mm + 8.0 * mm * l);
        }
    }
}

// orthonormal basis Q (gM x eM, ld n) of the Cholesky columns by Householder QR; nothing when the Gram is small
template <typename T>
__global__ void __launch_bounds__(1024) rr_qr_kernel(const RoundPlan* __restrict__ plan, const T* Y, T* W, T* Q) {
    const RoundPlan& p = *plan;
    if (!p.rr) return;
    __shared__ T tau[RR_L];
    __shared__ T red[33];
    __shared__ T s_beta;
    householder_qr<T>(Y, W, nullptr, Q, p.gM, p.eM, p.n, 0, tau, red, &s_beta);
}

// the next product of the reduction (k = eM basis columns): 0: Y = G Q;  1: B = Q^T Y into the Gram's buffer
// (ld k); 2: Y = Q U (U = the eigensolver's kept vectors of B, in S, ld n)
template <typename T>
__global__ void rr_step_kernel(const RoundPlan* __restrict__ plan, GemmArgs* ga, T* G, const T* Q, T* Y, const T* S,
                               int m, int which) {
    if (threadIdx.x != 0) return;
    const RoundPlan& p = *plan;
    const int M = p.gM, k = p.eM;
    const bool on = p.rr && k > 0;
    GemmArgs a{};
    a.alpha = 1.0; a.beta = 0.0; a.nbatch = 1; a.acc = 0;
    if (which == 0) {
        a.M = on ? M : 0; a.N = k; a.K = M;
        a.A = G; a.lda = M > 0 ? M : 1; a.B = Q; a.ldb = p.n; a.C = Y; a.ldc = p.n;
    } else if (which == 1) {
        a.M = on ? k : 0; a.N = k; a.K = M;
        a.A = Q; a.lda = p.n; a.B = Y; a.ldb = p.n; a.C = G; a.ldc = k > 0 ? k : 1;
    } else {
        a.M = on ? M : 0; a.N = p.s[m]; a.K = k;
        a.A = Q; a.lda = p.n; a.B = S; a.ldb = p.n; a.C = Y; a.ldc = p.n;
    }
    ga[0] = a;
}

// S <- Y (the kept Ritz vectors, gM x s_m)
template <typename T>
__global__ void rr_copy_kernel(const RoundPlan* __restrict__ plan, const T* Y, T* S, int m) {
    const RoundPlan& p = *plan;
    if (!p.rr) return;
    const int M = p.gM, s = p.s[m], n = p.n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)M * s;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e % M, c = e / M;
        S[i + c * n] = Y[i + c * n];
    }
}

__global__ void rr_end_kernel(RoundPlan* plan) {
    if (threadIdx.x == 0) { plan->rr = 0; plan->eM = plan->gM; }
}

// --------------------------------------------------------------------------------------------------
// Step 4: factors Q_t S_t (or S_t when Q_t = I), new core, plain descriptor.
// --------------------------------------------------------------------------------------------------
template <typename T>
__global__ void plan_final_kernel(RoundPlan* plan, GemmArgs* ga, const T* Q0, const T* Q1, const T* Q2,
                                  const T* S0, const T* S1, const T* S2, T* U0, T* U1, T* U2, int* counts) {
    if (threadIdx.x != 0) return;
    RoundPlan& p = *plan;
    const T* Q[3] = {Q0, Q1, Q2};
    const T* S[3] = {S0, S1, S2};
    T* U[3] = {U0, U1, U2};
    for (int t = 0; t < 3; ++t) {
        GemmArgs a{};
        a.nbatch = 1; a.acc = 0; a.alpha = 1.0; a.beta = 0.0;
        a.M = p.n; a.N = p.s[t];
        if (p.useQ[t]) {
            a.K = p.k[t]; a.A = Q[t]; a.lda = p.n;
        } else {
            a.K = 0;  // handled by the copy kernel
            a.M = 0;
        }
        a.B = S[t]; a.ldb = p.n;
        a.C = U[t]; a.ldc = p.n;
        ga[t] = a;
    }
    counts[0] = 3;
}

template <typename T>
__global__ void final_copy_kernel(const RoundPlan* __restrict__ plan, const T* S0, const T* S1, const T* S2, T* U0,
                                  T* U1, T* U2, const T* Zfin, T* core, long long core_cap, TuckerDesc* d,
                                  double* info) {
    const RoundPlan& p = *plan;
    const int n = p.n;
    const T* S[3] = {S0, S1, S2};
    T* U[3] = {U0, U1, U2};
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long gs = (long long)gridDim.x * blockDim.x;
    for (int t = 0; t < 3; ++t) {
        if (p.useQ[t]) continue;
        const long long tot = (long long)n * p.s[t];
        for (long long e = gt; e < tot; e += gs) U[t][e] = S[t][e];
    }
    const long long cs = (long long)p.s[0] * p.s[1] * p.s[2];
    if (cs <= core_cap)
        for (long long e = gt; e < cs; e += gs) core[e] = Zfin[e];
    if (gt == 0) {
        d->nblk = 1;
        for (int t = 0; t < 3; ++t) {
            d->rank[t] = p.s[t];
            d->blk[0].off[t] = 0;
            d->blk[0].r[t] = p.s[t];
        }
        d->blk[0].core = core;
        d->blk[0].scale = 1.0;
        if (info) {
            info[0] = p.norm2;
            info[1] = p.discarded;
            info[2] = p.s[0];
            info[3] = p.s[1];
            info[4] = p.s[2];
            info[5] = p.status ? 2.0 : ((cs <= core_cap) ? 0.0 : 1.0);
        }
    }
}

// --------------------------------------------------------------------------------------------------
// Host driver
// --------------------------------------------------------------------------------------------------
// Alg. 1 steps 1-2 (planner, QR of the factors, Z formation) into c->Z0 and c->plan.
template <typename T>
int round_stage12(tpcg_ctx c, tucker_t* y, double eps, const double* eps_dev, int rc, cudaStream_t st,
                  int strict_mode = -1) {
    const int n = c->n;
    GemmArgs* ga = c->gargs;
    int* counts = reinterpret_cast<int*>(c->scal + 200);   // 8 ints of scratch in the scalar area
    T* Z0 = static_cast<T*>(c->Z0);
    T* Z1 = static_cast<T*>(c->Z1);
    plan_round_kernel<T><<<1, 32, 0, st>>>(static_cast<const TuckerDesc*>(y->desc), c->plan, ga, n, rc, eps, eps_dev,
                                           c->Rq[0], c->Rq[1], c->Rq[2], y->U[0], y->U[1], y->U[2],
                                           static_cast<T*>(c->T1), static_cast<T*>(c->Wm), counts,
                                           (long long)c->max_cols * c->n * c->rank_cap, prof_dev(), strict_mode, Z0);
    TPCG_CHECK_LAUNCH();
    // step 1: QR where k_t < n
    prof_begin(PK_QR, st);
    {
        size_t sm = (size_t)(n + 40) * sizeof(T);
        qr_kernel<T><<<3, 1024, sm, st>>>(c->plan, static_cast<const T*>(y->U[0]), static_cast<const T*>(y->U[1]),
                                          static_cast<const T*>(y->U[2]), static_cast<T*>(c->Yw[0]),
                                          static_cast<T*>(c->Yw[1]), static_cast<T*>(c->Yw[2]),
                                          static_cast<T*>(c->Rq[0]), static_cast<T*>(c->Rq[1]),
                                          static_cast<T*>(c->Rq[2]), static_cast<T*>(c->Qq[0]),
                                          static_cast<T*>(c->Qq[1]), static_cast<T*>(c->Qq[2]));
        TPCG_CHECK_LAUNCH();
    }
    prof_end(PK_QR, st);
    // step 2: Z formation
    const int rcap = c->rank_cap;
    prof_begin(PK_ZBLK, st);
    TPCG_TRY((launch_gemm<T, false, true>(ga, counts, TPCG_MAX_BLOCKS, rcap, rcap, n, st)));
    TPCG_TRY((launch_gemm<T, false, false>(ga + TPCG_MAX_BLOCKS, counts, TPCG_MAX_BLOCKS, 1, n, n * rcap, st)));
    prof_end(PK_ZBLK, st);
    prof_begin(PK_ZGEMM, st);
    TPCG_TRY((launch_gemm<T, false, true>(ga + 2 * TPCG_MAX_BLOCKS, nullptr, 1, 1, n * n, n, st)));
    prof_end(PK_ZGEMM, st);
    return TPCG_OK;
}

// Alg. 1 steps 3-4 (ST-HOSVD of c->Z0 under c->plan, new factors Q S and core) into y.
template <typename T>
int round_stage34(tpcg_ctx c, tucker_t* y, double* info_dev, cudaStream_t st) {
    const int n = c->n;
    GemmArgs* ga = c->gargs;
    int* counts = reinterpret_cast<int*>(c->scal + 200);
    T* Z0 = static_cast<T*>(c->Z0);
    T* Z1 = static_cast<T*>(c->Z1);
    const int rcap = c->rank_cap;
    // step 3: ST-HOSVD
    T* Zc = Z0;
    T* Zn = Z1;
    const int min_k = gram_min_k();
    GemmArgs* gproj = ga + MAX_SPLIT;   // projection arguments, apart from the next Gram's
    plan_gram_kernel<T><<<1, 32, 0, st>>>(c->plan, ga, Zc, static_cast<T*>(c->Part), 0, MAX_SPLIT, min_k, counts,
                                          prof_dev());
    TPCG_CHECK_LAUNCH();
    for (int m = 0; m < 3; ++m) {
        prof_begin(PK_GRAM, st);
        if (m == 0)
            TPCG_TRY((launch_gemm<T, false, true>(ga, counts, MAX_SPLIT, 1, n, n, st)));
        else
            TPCG_TRY((launch_gemm<T, true, false>(ga, counts, MAX_SPLIT, 1, n, n, st)));
        reduce_partials_kernel<T><<<64, 256, 0, st>>>(static_cast<T*>(c->Part), counts + 1, counts + 2, counts,
                                                      static_cast<T*>(c->Gm), 0, 1.0, 0.0);
        TPCG_CHECK_LAUNCH();
        prof_end(PK_GRAM, st);
        prof_begin(PK_EIG, st);
        T* Gm = static_cast<T*>(c->Gm);
        T* Sm = static_cast<T*>(c->S[m]);
        T* rY = static_cast<T*>(c->rrY);
        T* rQ = static_cast<T*>(c->rrQ);
        if (c->rr) {   // Grams above RR_L: Rayleigh-Ritz matrix Q^T G Q of a pivoted-Cholesky basis in place of G
            const size_t sm = ((size_t)n + RR_L) * sizeof(T);
            rr_pchol_kernel<T><<<1, RR_THREADS, sm, st>>>(c->plan, Gm, rY, prof_dev());
            TPCG_CHECK_LAUNCH();
            rr_qr_kernel<T><<<1, 1024, 0, st>>>(c->plan, rY, static_cast<T*>(c->rrW), rQ);
            TPCG_CHECK_LAUNCH();
            rr_step_kernel<T><<<1, 32, 0, st>>>(c->plan, ga, Gm, rQ, rY, Sm, m, 0);
            TPCG_CHECK_LAUNCH();
            TPCG_TRY((launch_gemm<T, false, false>(ga, nullptr, 1, 1, n, RR_L, st)));
            rr_step_kernel<T><<<1, 32, 0, st>>>(c->plan, ga, Gm, rQ, rY, Sm, m, 1);
            TPCG_CHECK_LAUNCH();
            TPCG_TRY((launch_gemm<T, true, false>(ga, nullptr, 1, 1, RR_L, RR_L, st)));
        }
        TPCG_TRY(launch_eig<T>(c->plan, Gm, c->eigw, Sm, c->evals, m, c->rr ? RR_L : n, st));
        if (c->rr) {   // kept Ritz vectors Q U back into S
            rr_step_kernel<T><<<1, 32, 0, st>>>(c->plan, ga, Gm, rQ, rY, Sm, m, 2);
            TPCG_CHECK_LAUNCH();
            TPCG_TRY((launch_gemm<T, false, false>(ga, nullptr, 1, 1, n, RR_L, st)));
            rr_copy_kernel<T><<<64, 256, 0, st>>>(c->plan, rY, Sm, m);
            TPCG_CHECK_LAUNCH();
            rr_end_kernel<<<1, 32, 0, st>>>(c->plan);
            TPCG_CHECK_LAUNCH();
        }
        prof_end(PK_EIG, st);
        prof_begin(PK_PROJ, st);
        plan_proj_kernel<T><<<1, 32, 0, st>>>(c->plan, gproj, static_cast<const T*>(c->S[m]), Zc, Zn, m, ga,
                                              static_cast<T*>(c->Part), MAX_SPLIT, min_k, counts, prof_dev());
        TPCG_CHECK_LAUNCH();
        if (m == 0)
            TPCG_TRY((launch_gemm<T, true, false>(gproj, nullptr, 1, 1, n, n * n, st)));
        else if (m == 1)
            TPCG_TRY((launch_gemm<T, false, false>(gproj, nullptr, 1, n, n, n, st)));
        else
            TPCG_TRY((launch_gemm<T, false, false>(gproj, nullptr, 1, 1, n * n, n, st)));
        prof_end(PK_PROJ, st);
        T* tmp = Zc; Zc = Zn; Zn = tmp;
    }
    // step 4
    plan_final_kernel<T><<<1, 32, 0, st>>>(c->plan, ga, static_cast<const T*>(c->Qq[0]),
                                           static_cast<const T*>(c->Qq[1]), static_cast<const T*>(c->Qq[2]),
                                           static_cast<const T*>(c->S[0]), static_cast<const T*>(c->S[1]),
                                           static_cast<const T*>(c->S[2]), static_cast<T*>(y->U[0]),
                                           static_cast<T*>(y->U[1]), static_cast<T*>(y->U[2]), counts);
    TPCG_CHECK_LAUNCH();
    TPCG_TRY((launch_gemm<T, false, false>(ga, counts, 3, 1, n, rcap, st)));
    final_copy_kernel<T><<<64, 256, 0, st>>>(c->plan, static_cast<const T*>(c->S[0]), static_cast<const T*>(c->S[1]),
                                             static_cast<const T*>(c->S[2]), static_cast<T*>(y->U[0]),
                                             static_cast<T*>(y->U[1]), static_cast<T*>(y->U[2]), Zc,
                                             static_cast<T*>(y->core), y->core_cap,
                                             static_cast<TuckerDesc*>(y->desc), info_dev);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}

template <typename T>
int round_impl(tpcg_ctx c, tucker_t* y, double eps, const double* eps_dev, int cap, double* info_dev,
               cudaStream_t st, int strict_mode) {
    const int rc = (cap > 0 && cap < c->rank_cap) ? cap : c->rank_cap;
    prof_begin(PK_ROUND, st);
    TPCG_TRY(round_stage12<T>(c, y, eps, eps_dev, rc, st, strict_mode));
    TPCG_TRY(round_stage34<T>(c, y, info_dev, st));
    prof_end(PK_ROUND, st);
    return TPCG_OK;
}

// round_impl captured once per (tensor, device tolerance, cap) into a CUDA graph and replayed: the ~30
// launches of a truncation become one graph launch, which matters when many solves share the host.  The
// launch sequence of a truncation does not depend on ranks (all sizes are read on the device), so the
// replay is exact.  Falls back to direct launches while profiling or on the legacy default stream.
template <typename T>
int round_cached(tpcg_ctx c, tucker_t* y, const double* eps_dev, int cap, cudaStream_t st, int strict_mode) {
    const int rc = (cap > 0 && cap < c->rank_cap) ? cap : c->rank_cap;
    if (prof_on() || !eps_dev || st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread)
        return round_impl<T>(c, y, 0.0, eps_dev, cap, nullptr, st, strict_mode);
    for (const auto& g : c->rgraphs)
        if (g.desc == y->desc && g.U0 == y->U[0] && g.eps_dev == eps_dev && g.rc == rc && g.strict == strict_mode) {
            TPCG_CUDA(cudaGraphLaunch(g.exec, st));
            g_launches.fetch_add(g.nkern, std::memory_order_relaxed);
            return TPCG_OK;
        }
    const long long k0 = t_launches;
    TPCG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int s = round_impl<T>(c, y, 0.0, eps_dev, rc, nullptr, st, strict_mode);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s != TPCG_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (s != TPCG_OK) return s;
        set_error(std::string("round_cached: stream capture failed: ") + cudaGetErrorString(e));
        return TPCG_E_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("round_cached: graph instantiation failed: ") + cudaGetErrorString(ei));
        return TPCG_E_CUDA;
    }
    c->rgraphs.push_back({y->desc, y->U[0], eps_dev, rc, strict_mode, exec, t_launches - k0});
    TPCG_CUDA(cudaGraphLaunch(exec, st));   // the kernels counted during capture run now
    return TPCG_OK;
}
template int round_cached<double>(tpcg_ctx, tucker_t*, const double*, int, cudaStream_t, int);
template int round_cached<float>(tpcg_ctx, tucker_t*, const double*, int, cudaStream_t, int);

// Mixed rounding: Alg. 1 steps 1-2 in FP64 (the Z formation carries the cancellation of a residual), then
// steps 3-4 in FP32 on the rounded Z.  y64 is an FP64 (block) tensor, out32 receives an FP32 plain tensor.
__global__ void demote_kernel(const RoundPlan* __restrict__ plan, const double* __restrict__ Z64, float* __restrict__ Z32,
                              const double* Q0, const double* Q1, const double* Q2, float* P0, float* P1, float* P2) {
    const RoundPlan& p = *plan;
    const long long nz = (long long)p.kp[0] * p.kp[1] * p.kp[2];
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x, gs = (long long)gridDim.x * blockDim.x;
    for (long long e = gt; e < nz; e += gs) Z32[e] = (float)Z64[e];
    const double* Q[3] = {Q0, Q1, Q2};
    float* P[3] = {P0, P1, P2};
    for (int t = 0; t < 3; ++t) {
        if (!p.useQ[t]) continue;
        const long long nq = (long long)p.n * p.k[t];
        for (long long e = gt; e < nq; e += gs) P[t][e] = (float)Q[t][e];
    }
}

__global__ void set_abs_kernel(RoundPlan* plan, double abs_tol) { plan->abs2 = abs_tol * abs_tol; }

int round_mixed(tpcg_ctx c64, tpcg_ctx c32, tucker_t* y64, tucker_t* out32, double eps, const double* eps_dev, int cap,
                double abs_tol, double* info_dev, cudaStream_t st) {
    const int rc = (cap > 0 && cap < c32->rank_cap) ? cap : c32->rank_cap;
    prof_begin(PK_ROUND, st);
    TPCG_TRY(round_stage12<double>(c64, y64, eps, eps_dev, rc, st));
    demote_kernel<<<256, 256, 0, st>>>(c64->plan, static_cast<const double*>(c64->Z0), static_cast<float*>(c32->Z0),
                                       static_cast<const double*>(c64->Qq[0]), static_cast<const double*>(c64->Qq[1]),
                                       static_cast<const double*>(c64->Qq[2]), static_cast<float*>(c32->Qq[0]),
                                       static_cast<float*>(c32->Qq[1]), static_cast<float*>(c32->Qq[2]));
    TPCG_CHECK_LAUNCH();
    TPCG_CUDA(cudaMemcpyAsync(c32->plan, c64->plan, sizeof(RoundPlan), cudaMemcpyDeviceToDevice, st));
    if (abs_tol > 0) {
        set_abs_kernel<<<1, 1, 0, st>>>(c32->plan, abs_tol);
        TPCG_CHECK_LAUNCH();
    }
    TPCG_TRY(round_stage34<float>(c32, out32, info_dev, st));
    prof_end(PK_ROUND, st);
    return TPCG_OK;
}

// Alg. 1 at tolerances below what one FP64 Gram resolves.  A mode Gram carries rounding errors of about
// eps_machine ||Z||^2, so for eps below ~1e-7 its smallest eigenvalues (the energies the budget
// eps^2 ||Z||^2 / 3 is about) are noise: a single pass then both keeps noise directions and may drop more than
// the budget.  Two passes resolve them:
//   A. Y_A = T(Y, EPS_RESOLVED): the part the Gram resolves (relative error <= EPS_RESOLVED);
//   B. E = Y - Y_A, rounded with the absolute budget (eps ||Y||)^2: E's own Grams resolve energies relative to
//      ||E||^2 <= EPS_RESOLVED^2 ||Y||^2, far below the budget;
//   Y~ = Y_A + T(E): ||Y - Y~|| = ||E - T(E)|| <= eps ||Y||, merged losslessly (QR of the joined factors, strict
//   rule at eps 0, then the rank cap).
// y is left unchanged; the result is written to out; E and F are scratch tensors of the context's capacity.
constexpr double EPS_RESOLVED = EPS_RESOLVED_PASS;

__global__ void save_norm2_kernel(const RoundPlan* __restrict__ plan, double* out) { *out = plan->norm2; }
__global__ void set_abs_rel_kernel(RoundPlan* plan, const double* __restrict__ eps_dev, double eps_host,
                                   const double* __restrict__ norm2) {
    const double e = eps_dev ? *eps_dev : eps_host;
    plan->abs2 = e * e * (*norm2);
}

int round_resolved(tpcg_ctx c, const tucker_t* y, tucker_t* out, double eps, const double* eps_dev, int cap,
                   double* norm2_slot, tucker_t* E, tucker_t* F, cudaStream_t st) {
    const int rc = (cap > 0 && cap < c->rank_cap) ? cap : c->rank_cap;
    TPCG_TRY(copy_tensor_impl<double>(y, out, c->n, out->cap, st));
    TPCG_TRY(round_impl<double>(c, out, EPS_RESOLVED, nullptr, rc, nullptr, st, 0));                  // A
    save_norm2_kernel<<<1, 1, 0, st>>>(c->plan, norm2_slot);                                           // ||Y||^2
    TPCG_CHECK_LAUNCH();
    TPCG_TRY(axpby_impl<double>(1.0, nullptr, y, -1.0, nullptr, out, E, nullptr, st));                  // E = Y - Y_A
    prof_begin(PK_ROUND, st);
    TPCG_TRY(round_stage12<double>(c, E, 0.0, nullptr, rc, st, 0));                                    // B
    set_abs_rel_kernel<<<1, 1, 0, st>>>(c->plan, eps_dev, eps, norm2_slot);
    TPCG_CHECK_LAUNCH();
    TPCG_TRY(round_stage34<double>(c, E, nullptr, st));
    prof_end(PK_ROUND, st);
    TPCG_TRY(axpby_impl<double>(1.0, nullptr, out, 1.0, nullptr, E, F, nullptr, st));                   // Y_A + T(E)
    TPCG_TRY(round_impl<double>(c, F, 0.0, nullptr, rc, nullptr, st, 1));                              // lossless
    return copy_tensor_impl<double>(F, out, c->n, out->cap, st);
}

// ||Z||^2 of the Z formed by round_stage12 (deterministic single-CTA reduction)
template <typename T>
__global__ void znorm2_kernel(const RoundPlan* __restrict__ plan, const T* __restrict__ Z, double* out) {
    const RoundPlan& p = *plan;
    const long long nz = (long long)p.kp[0] * p.kp[1] * p.kp[2];
    double acc = 0.0;
    for (long long e = threadIdx.x; e < nz; e += blockDim.x) acc += (double)Z[e] * (double)Z[e];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

// squared Frobenius norm of an unrounded tensor y (any block structure): Z formation of Alg. 1 in the
// working precision, then ||Z||^2 (exact: Q has orthonormal columns)
template <typename T>
int tensor_norm2(tpcg_ctx c, tucker_t* y, double* out_dev, cudaStream_t st) {
    TPCG_TRY(round_stage12<T>(c, y, 0.0, nullptr, c->rank_cap, st));
    znorm2_kernel<T><<<1, 1024, 0, st>>>(c->plan, static_cast<const T*>(c->Z0), out_dev);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}
template int tensor_norm2<double>(tpcg_ctx, tucker_t*, double*, cudaStream_t);
template int tensor_norm2<float>(tpcg_ctx, tucker_t*, double*, cudaStream_t);

template int round_impl<double>(tpcg_ctx, tucker_t*, double, const double*, int, double*, cudaStream_t, int);
template int round_impl<float>(tpcg_ctx, tucker_t*, double, const double*, int, double*, cudaStream_t, int);

}  // namespace tpcg
