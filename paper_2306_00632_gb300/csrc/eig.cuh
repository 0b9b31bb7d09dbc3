// Eigensolver of the mode Grams used by the ST-HOSVD step of the rounding (see eig.cu).
#pragma once

#include <vector>


namespace tpcg {

struct RoundPlan;

constexpr int SMAX_EIG = 1024;   // largest Gram (= n) the one-CTA eigensolver accepts
// Rayleigh-Ritz reduction of large Grams (round.cu): the largest basis (pivoted-Cholesky columns), and the
// largest rank cap of the contexts that use it
constexpr int RR_L = 128;
constexpr int RR_MAXCAP = RR_L - 16;

struct EigWork {
    void* Aw;        // n (n + 1) elements: the Gram when it does not fit shared memory
    void* Vw;        // n (n + 1) elements: the eigenvectors when they do not fit shared memory
};

size_t eig_work_bytes(int n);
// eigensolver of FP32 Grams up to 128 (TPCG_OPT_EIG): 1 pivoted Cholesky + one-sided Jacobi, 0 two-sided Jacobi
int eig_kind();
// shared-memory opt-ins of the eigensolver kernels on the current device (before any stream capture)
int eig_prepare();
int eig_work_alloc(EigWork* w, int n, std::vector<void*>* owned);

// Eigen-decomposition (Jacobi) of the plan's current Gram G (gM x gM, ld gM), truncation rule of mode m, kept
// eigenvectors (orthonormal) into S (ld n); plan.s[m], plan.discarded (and for m = 0 plan.norm2/budget)
// are updated on the device.
template <typename T>
int launch_eig(RoundPlan* plan, const T* G, EigWork& w, T* S, double* evals, int m, int n, cudaStream_t st);

}  // namespace tpcg
