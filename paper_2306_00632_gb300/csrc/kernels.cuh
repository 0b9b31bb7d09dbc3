// Declarations of the templated device-side operations (one instantiation per compute dtype).
#pragma once

#include <initializer_list>

#include "common.cuh"

namespace tpcg {

// strict_mode: -1 automatic (the FP64 rule charges the Gram's rounding uncertainty when eps < 1e-7), 0 off, 1 on
template <typename T>
int round_impl(tpcg_ctx c, tucker_t* y, double eps, const double* eps_dev, int cap, double* info_dev,
               cudaStream_t st, int strict_mode = -1);
// FP64 Z formation, FP32 ST-HOSVD into out32; the discarded energy may also reach abs_tol^2 (absolute norm floor)
// round_impl(c, y, 0, eps_dev, cap) replayed from a per-context CUDA graph (captured on first use)
template <typename T>
int round_cached(tpcg_ctx c, tucker_t* y, const double* eps_dev, int cap, cudaStream_t st, int strict_mode = -1);
// FP64 Alg. 1 for eps below what one Gram resolves (two passes: the resolved part, then the remainder with the
// absolute budget); y unchanged, result in out, E and F scratch; norm2_slot: one device double of scratch
int round_resolved(tpcg_ctx c, const tucker_t* y, tucker_t* out, double eps, const double* eps_dev, int cap,
                   double* norm2_slot, tucker_t* E, tucker_t* F, cudaStream_t st);
int round_mixed(tpcg_ctx c64, tpcg_ctx c32, tucker_t* y64, tucker_t* out32, double eps, const double* eps_dev, int cap,
                double abs_tol, double* info_dev, cudaStream_t st);
// whether a context of this size, rank cap and dtype reduces its large Grams by Rayleigh-Ritz
int rr_kind();      // TPCG_OPT_RR
int gram_min_k();   // TPCG_OPT_GRAM_MIN_K
int round_rule();   // TPCG_OPT_ROUND_RULE: rule of tucker_round (-1 automatic, 0 plain, 1 strict, 2 resolved)
int resolved_kind();   // TPCG_OPT_RESOLVED: FP64 solves truncate x with round_resolved below its threshold
// The first pass of round_resolved rounds at EPS_RESOLVED_PASS, which one FP64 Gram pass resolves; solves take the
// resolved rule below RESOLVE_BELOW (one pass met the bound at 1e-7 on Alg. 5 iterates and broke it, 1.24 eps,
// at 6e-9)
constexpr double EPS_RESOLVED_PASS = 1e-7;
constexpr double RESOLVE_BELOW = 1e-8;
// FP32: every context with n > RR_L (the one-CTA FP32 Jacobi for larger Grams keeps its diagonal by rotation
// updates, whose drift spoils the trace-minus-kept rule); FP64: n > 256 (beyond the cluster eigensolver) with a
// rank cap that leaves the basis room
inline bool rr_context(int n, int rank_cap, int dtype) {
    return rr_kind() == 1 && (dtype == TPCG_F32 ? n > RR_L : (n > 256 && rank_cap <= RR_MAXCAP));
}
// ||y||^2 of any (block) tensor by the Z formation of Alg. 1
template <typename T>
int tensor_norm2(tpcg_ctx c, tucker_t* y, double* out_dev, cudaStream_t st);
// copy a plain FP32 tensor into an FP64 tensor (factors, core, descriptor)
int promote_tensor(const tucker_t* src32, tucker_t* dst64, cudaStream_t st);
// err: device int set to 1 when the product does not fit y (capacity or block limit).  Solvers pass a flag of
// their own context, so that solves sharing a problem never see each other's flags; null selects the problem's
// flag (standalone calls).
template <typename T>
int apply_impl(tpcg_problem pb, const tucker_t* x, tucker_t* y, bool residual, cudaStream_t st,
               const tucker_t* rhs = nullptr, int* err = nullptr);
// y <- y + sign A x with the new blocks appended to y's block list
template <typename T>
int apply_append_impl(tpcg_problem pb, const tucker_t* x, tucker_t* y, double sign, cudaStream_t st,
                      int* err = nullptr);
template <typename T>
int axpby_impl(double a, const double* a_dev, const tucker_t* x, double b, const double* b_dev, const tucker_t* y,
               tucker_t* z, int* err_dev, cudaStream_t st);
template <typename T>
int dot_impl(tpcg_ctx c, const tucker_t* x, const tucker_t* y, double* out_dev, cudaStream_t st);
// dot_impl replayed from a per-context CUDA graph keyed by (x, y, out)
template <typename T>
int dot_cached(tpcg_ctx c, const tucker_t* x, const tucker_t* y, double* out_dev, cudaStream_t st);
// <x, y> with its scratch in a fixed device array (no allocation; ranks <= dot_static_max_rank())
template <typename T>
int dot_static_impl(const tucker_t* x, const tucker_t* y, double* out_dev, cudaStream_t st);
int dot_static_max_rank();
// v = P~^-1 s (Alg. 4); wdir: direction weights c_t of a weighted Kronecker sum (null: all 1)
template <typename T>
int fd_impl(tpcg_problem pb, tpcg_ctx c, const tucker_t* s, tucker_t* v, cudaStream_t st, const double* wdir = nullptr);
template <typename T>
int copy_tensor_impl(const tucker_t* src, tucker_t* dst, int n, int cap, cudaStream_t st);

// chirp-z (Bluestein) FFT sine transforms of App. B (dst.cu): host tables for length n1 and degree p (complex
// pairs: twiddles, then forward and inverse pre/post chirps and filter spectra), and the batched transform of
// the columns c < mult rank_t of every mode t (kind 0: U_dft^T x, kind 1: U_dft x)
// Integer phase grid of App. B's sine matrix, 0-based l (point) and j (sinusoid):
//   U_dft[l, j] = sqrt2 sin(omega_j x_l + k0 pi/2) = sqrt2 sin(pi m / (4 D)),  m = (2 j + e)(2 l + c) + g,
// D = n_el, e = 2 - k0 - k1, c = 2 - 2 k0 (odd p: breakpoints without the Dirichlet ends) or 1 (even p: span
// midpoints), g = 2 k0 D.
struct SineGrid {
    long long D, e, c, g;
};
SineGrid sine_grid(int n1, int p, int k0, int k1);
int chirp_tables(int n1, int p, int k0, int k1, ChirpInfo* info, std::vector<double>* out);
template <typename T>
int launch_chirp(tpcg_problem pb, int kind, const TuckerDesc* sd, int mult, int rp_guard, int vcap, int maxcols,
                 const T* const* X, T* const* Y, int ldx, int ldy, cudaStream_t st);
int dst_kind();   // TPCG_OPT_DST: 1 FFT sine transforms, 0 dense sine matrix

int set_plain(tucker_t* t, int r1, int r2, int r3, cudaStream_t st);
int set_zero(tucker_t* t, cudaStream_t st);

// ---- Alg. 5 scalars: slots of ctx->scal (device doubles), parameters at scal + 100, update ops
enum {
    S_NF = 0, S_NR, S_ETA, S_RP, S_XI, S_OMEGA, S_EPS, S_EPSMIN, S_PXK, S_PXN, S_PP, S_V, S_DONE, S_ZQ, S_BETA,
    S_STOP, S_RR, S_BAD, S_TRIALS, S_ZN2, S_COUNT
};
enum { P_TOL = 0, P_EPS0, P_EPSMIN, P_ALPHA, P_DELTA, P_BT, P_COUNT };
enum { OP_INIT = 0, OP_OMEGA, OP_DT, OP_RES, OP_BETA, OP_XI };
// TPCG scalar updates (one thread each)
void launch_scalar(int op, double* s, const double* prm, cudaStream_t st);

// ---- solver helpers (api.cu)
int check_tensor(const tucker_t* t, int n, int dtype, const char* what);
// allocate the first `count` solver tensors of the context (n x max_cols factors, rank_cap^3 core)
int ensure_tensors(tpcg_ctx c, int count);
// wait on the host for the work enqueued on s: polls an event, yielding and then sleeping between polls
int host_wait(tpcg_ctx c, cudaStream_t s);
// device-to-host reads of small values through the context's pinned staging buffer, then one host_wait:
// copies into pageable memory would make the driver wait inside the copy call itself (spinning a core)
constexpr size_t TPCG_HSTAGE_BYTES = 4096;
struct D2H {
    void* dst;
    const void* src;
    size_t bytes;
};
int fetch(tpcg_ctx c, cudaStream_t s, const D2H* items, int count);
inline int fetch(tpcg_ctx c, cudaStream_t s, std::initializer_list<D2H> items) {
    return fetch(c, s, items.begin(), (int)items.size());
}

}  // namespace tpcg
