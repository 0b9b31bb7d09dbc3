// Host FP64 setup of a TPCG problem (App. A, App. B, Prop. 1): untimed, runs once per problem.
#pragma once

#include <vector>

#include "../../include/tpcg.h"

namespace tpcg {

struct HostProblem {
    int R = 0;                       // Kronecker terms of A~
    int rf[3] = {0, 0, 0};           // rhs ranks
    int n1 = 0, n2 = 0, RP = 0;      // App. B splitting, exponential-sum length
    int k0 = 0, k1 = 0;              // Neumann flags of the two ends (every direction)
    double lambda_min = 0, lambda_max = 0;
    std::vector<double> w;           // R weights
    std::vector<double> bands;       // [((j*3+t)*(2p+1)+d)*n + i] = K_t^j[i, i+d-p]
    std::vector<double> f_core;      // rf1 x rf2 x rf3
    std::vector<double> f_U[3];      // n x rf_t
    std::vector<double> lam;         // Lambda~ (n)
    std::vector<double> mu;          // n1
    std::vector<int> w_rowptr, w_col;
    std::vector<double> w_val;       // W (n x n1) in CSR
    std::vector<double> v2u2;        // n x n2
    std::vector<double> omega, alpha;
};

int host_setup(const tpcg_geometry& geo, int p, int n, HostProblem* out);
// elasticity (Sec. 5.3): out[3 i + j] = block A_ij with rhs component f_i and the shared FD tables
int host_elast_setup(const tpcg_geometry& geo, int p, int n, double lam, double mu, const double force[3],
                     HostProblem out[9]);

// pieces exposed for the exponential-sum search (also used by tests through the C ABI of the setup)
double expsum_error(const double* omega, const double* alpha, int R, double M, int npts);
int expsum_sinc(double M, double eps_prec, std::vector<double>* omega, std::vector<double>* alpha);
// best sums by the Remez exchange (expsum.cpp): the smallest R <= rmax with E_R(M) <= eps_prec / M, or -1
int expsum_best(double M, double eps_prec, int rmax, std::vector<double>* omega, std::vector<double>* alpha,
                double* E_out);
// which sums tpcg_setup uses: 1 best sums (default), 0 the sinc-quadrature search (tpcg_set_option)
int expsum_kind();

}  // namespace tpcg
