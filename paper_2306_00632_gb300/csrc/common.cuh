// Internal types shared by the CUDA translation units of the TPCG library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/tpcg.h"

namespace tpcg {

// ------------------------------------------------------------------------------------ errors
void set_error(const std::string& msg);
// Host-to-device copies and zero fills that complete before the call returns, on a private non-blocking stream.
// cudaMemcpy / cudaMemset use the legacy default stream, which is not ordered with the non-blocking streams the
// solvers run on, and may return before the device write is done (pageable uploads, device memsets): a solve
// started right after them on another stream could read stale data or be overwritten by the late write.
int sync_to_device(void* dst, const void* src, size_t bytes);
int sync_zero(void* dst, size_t bytes);

// ------------------------------------------------------------------------------------ profiling
extern std::atomic<long long> g_launches;
extern thread_local long long t_launches;   // launches (or captured kernel nodes) issued by this thread
enum { PK_ZGEMM = 0, PK_ZBLK, PK_GRAM, PK_EIG, PK_PROJ, PK_QR, PK_APPLY, PK_FD, PK_DOT, PK_ROUND, PK_FINAL, PK_SWEEPS,
       PK_COUNT = 16 };
bool prof_on();
double* prof_dev();                       // device accumulators [kind*2] flops, [kind*2+1] bytes, or null
void prof_begin(int kind, cudaStream_t st);
void prof_end(int kind, cudaStream_t st);

#define TPCG_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ::tpcg::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
            return TPCG_E_CUDA;                                                           \
        }                                                                                 \
    } while (0)

#define TPCG_CHECK_LAUNCH()                                                               \
    do {                                                                                  \
        ::tpcg::g_launches.fetch_add(1, std::memory_order_relaxed);                       \
        ++::tpcg::t_launches;                                                             \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) {                                                          \
            ::tpcg::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));   \
            return TPCG_E_CUDA;                                                           \
        }                                                                                 \
    } while (0)

#define TPCG_TRY(expr)                   \
    do {                                 \
        int s_ = (expr);                 \
        if (s_ != TPCG_OK) return s_;    \
    } while (0)

// ------------------------------------------------------------------------------------ device descriptor
// Ranks and block list of a Tucker tensor, stored in tucker_t.desc.  Block b is scale_b * core_b placed
// at column offsets off[t] of the three factors (a block-diagonal core, Sec. 2.3).
struct BlockDesc {
    int off[3];
    int r[3];
    const void* core;   // dense r1 x r2 x r3 column-major
    double scale;
};
struct TuckerDesc {
    int nblk;
    int rank[3];        // factor columns in use
    int pad[4];
    BlockDesc blk[TPCG_MAX_BLOCKS];
};
static_assert(sizeof(TuckerDesc) <= TPCG_DESC_BYTES, "descriptor too large");

// ------------------------------------------------------------------------------------ grouped GEMM args
// C_g = alpha * op(A_g) op(B_g) + beta * C_g for every group g (column-major).  With nbatch > 1 and
// acc = 0 the group is a strided batch of independent products; with acc = 1 the products of the batch
// are summed into one C.  M, N or K = 0 makes the group a no-op (C untouched unless beta scaling is
// needed: then C = beta*C when K = 0).
struct GemmArgs {
    int M, N, K, nbatch;
    int acc, pad0;
    const void* A;
    long long lda, sA;
    const void* B;
    long long ldb, sB;
    void* C;
    long long ldc, sC;
    double alpha, beta;
};

// ------------------------------------------------------------------------------------ rounding plan
constexpr int MAX_SPLIT = 64;      // K-slices of a long Gram reduction

struct RoundPlan {
    int n, nblk;
    int k[3];          // columns of the input factors
    int kp[3];         // min(n, k): sizes of Z
    int useQ[3];       // 1 if a QR was needed (k < n), else Q = I
    int s[3];          // kept ranks
    int cap;
    int nsplit;        // groups of the current Gram
    int gm, gM;        // current Gram: mode and size
    int eM;            // order of the eigensolver's input: gM, or RR_L when the Gram goes through rr
    int rr;            // 1 while the current Gram is reduced by the Rayleigh-Ritz step (round.cu)
    double gtrace;     // trace of the current Gram when rr (the eigensolver's input is then Q^T G Q)
    int zdim[3];       // current dims of the working tensor
    double eps, budget, norm2, discarded;
    double abs2;       // absolute floor of the discarded energy (0: relative rule only)
    const void* Rp[3]; // R_t used to form Z (workspace R or the factor itself)
    long long ldR[3];
    int kz3;           // total K of the fused last-mode GEMM
    int status;
    int strict;        // FP64 rule: charge every discarded Gram eigenvalue its rounding uncertainty
};

// ------------------------------------------------------------------------------------ host objects
struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace tpcg

#include "eig.cuh"

constexpr int TPCG_CTX_TENSORS = 24;   // solver tensors of a context (allocated on first use)

struct tpcg_ctx_s {
    int n, max_cols, rank_cap, dtype;
    size_t elt;
    // rounding workspace
    void* Z0;            // n^3
    void* Z1;            // n^3
    void* Wm;            // n^2 * max_cols   (stacked mode-1/2 products, columns = fused K)
    void* T1;            // max_cols * n * rank_cap
    void* Rq[3];         // n * n            (R factors of the QR)
    void* Qq[3];         // n * n            (Q factors of the QR)
    void* Yw[3];         // n * n            (QR working copy)
    void* Gm;            // n * n            (Gram)
    void* Part;          // MAX_SPLIT * n * n (partials)
    void* S[3];          // n * n            (eigenvectors / kept singular vectors)
    double* evals;       // n
    tpcg::GemmArgs* gargs;   // device array of GEMM args (scratch for planners)
    tpcg::RoundPlan* plan;   // device
    double* scal;        // device scalars (256 doubles)
    double* dotw;        // small Gram matrices for dots: 3 * rank_cap * rank_cap * 2 + core temps
    void* dotT;          // rank_cap^3 * 2 temporaries for dot contractions
    void* fd[3][4];      // n * max_cols each: FD application scratch (gather, transform, scaled, back)
    tpcg::EigWork eigw;  // eigensolver work area
    // Rayleigh-Ritz reduction of Grams above RR_L (contexts with n > RR_L and rank_cap <= RR_MAXCAP; round.cu)
    int rr;              // 1 if this context uses it
    void* rrY;           // n x RR_L: pivoted-Cholesky columns, then G Q, then Q U
    void* rrQ;           // n x RR_L: orthonormal basis
    void* rrW;           // n x RR_L: QR working copy
    // TPCG iterate tensors (allocated on first solve)
    std::vector<void*> owned;
    tucker_t tens[TPCG_CTX_TENSORS];
    int have_tens;       // solver tensors allocated so far
    int tens_cap;
    tpcg_ctx_s* lo;      // FP32 companion of a mixed-precision context (else null)
    cudaEvent_t sync_ev; // event the solver's host waits poll
    unsigned char* hstage;   // pinned host staging for the solver's device-to-host reads (TPCG_HSTAGE_BYTES)
    cudaStream_t own_stream;   // created on first use by tpcg_solve_batch for NULL stream entries
    // captured roundings (CUDA graphs) of the solver tensors, keyed by tensor and tolerance source
    struct RoundGraph {
        const void* desc;
        const void* U0;
        const double* eps_dev;
        int rc;
        int strict;
        cudaGraphExec_t exec;
        long long nkern;
    };
    std::vector<RoundGraph> rgraphs;
    // per-iteration scalars of the last Alg. 5 run on this context (TPCG_HIST_COLS doubles per iteration)
    std::vector<double> hist;
};

namespace tpcg {
// FFT sizes of the chirp-z sine transforms of the preconditioner (dst.cu)
struct ChirpInfo {
    int L = 0, Mf = 0, logMf = 0;
};
}  // namespace tpcg

struct tpcg_problem_s {
    int n, p, R, RP, n1, n2, dtype;
    int k0, k1;          // Neumann flags of the two ends (App. B's sine variant)
    int rf[3];
    double lambda_min, lambda_max, norm_f;
    // host copies (double)
    std::vector<double> w, bands, f_core, f_U[3], lam, mu, v2u2, omega, alpha, w_val;
    std::vector<int> w_rowptr, w_col;
    // device copies in the compute dtype
    void* d_bands;       // R * 3 * (2p+1) * n
    double* d_w;         // R
    tucker_t f;          // rhs, plain with orthonormal factors
    void* d_f_store[5];  // owned buffers of f
    void* d_lam;         // n
    void* d_mu;          // n1
    int* d_wrow;         // n+1
    int* d_wcol;         // nnz
    void* d_wval;        // nnz
    int* d_wtrow;        // n1+1  (transpose CSR)
    int* d_wtcol;
    void* d_wtval;
    void* d_v2u2;        // n * n2
    void* d_dst;         // n1 x n1 sine matrix sqrt2 sin(j pi x_l)
    void* d_chirp;       // chirp-z tables of the FFT sine transforms (complex pairs), null if n1 > 1024
    tpcg::ChirpInfo chirp;
    double* d_omega;     // RP
    double* d_alpha;     // RP
    double* d_scal;      // problem scalars (lambda_min, ...)
    tpcg_problem_s* lo;  // FP32 companion of a mixed-precision problem (else null)
};
