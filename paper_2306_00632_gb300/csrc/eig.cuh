// Eigensolver pieces used by the ST-HOSVD step of the rounding (see eig.cu).
#pragma once

#include "common.cuh"

namespace tpcg {

// FP64 refinement work area (all M x M doubles with ld M, M <= n)
struct EigWork {
    double* X;
    double* Xn;
    double* XtX;
    double* AX;
    double* S;
    double* E;
    double* lam;       // n
    double* Part;      // 2 * 32 * n * n partial products
    GemmArgs* ga;      // 256 slots
    int* counts;       // 8 ints
    float* V32;        // n * n
    float* A32;        // n * n scratch when the matrix does not fit shared memory
    float* lam32;      // n
    double* energy;    // n slice energies (FP32 form)
    int* order;        // n kept/sorted slice indices
};

size_t eig_work_bytes(int n);
int eig_work_alloc(EigWork* w, int n, std::vector<void*>* owned);

template <typename Tin>
int launch_jacobi32(const int* Mdev, const Tin* G, float* V, float* Ascratch, float* lam, int n, cudaStream_t st);

int refine_eig64(const int* Mdev, const double* A, const float* V32, int n, EigWork& w, int iters, cudaStream_t st);

}  // namespace tpcg
