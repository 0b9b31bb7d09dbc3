// C ABI entry points: contexts, problems, Tucker operations and the TPCG driver (Alg. 5).
#include <math.h>
#include <cmath>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "gemm.cuh"
#include "kernels.cuh"
#include "setup.h"

namespace tpcg {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

static inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }
static inline size_t elt_of(int dtype) { return dtype == TPCG_F64 ? sizeof(double) : sizeof(float); }

static int dmalloc(void** p, size_t bytes, std::vector<void*>* owned) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        *p = nullptr;
        return TPCG_E_NOMEM;
    }
    if (owned) owned->push_back(*p);
    return TPCG_OK;
}

namespace {
// one private non-blocking stream per host thread for the blocking copies below (created on first use)
struct PrivStream {
    cudaStream_t s = nullptr;
    ~PrivStream() {
        if (s) cudaStreamDestroy(s);
    }
};
thread_local PrivStream t_priv;

int priv_stream(cudaStream_t* out) {
    if (!t_priv.s && cudaStreamCreateWithFlags(&t_priv.s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        t_priv.s = nullptr;
        set_error("cudaStreamCreateWithFlags failed");
        return TPCG_E_CUDA;
    }
    *out = t_priv.s;
    return TPCG_OK;
}
}  // namespace

int sync_to_device(void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return TPCG_OK;
    cudaStream_t s = nullptr;
    TPCG_TRY(priv_stream(&s));
    TPCG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    TPCG_CUDA(cudaStreamSynchronize(s));
    return TPCG_OK;
}

int sync_zero(void* dst, size_t bytes) {
    if (bytes == 0) return TPCG_OK;
    cudaStream_t s = nullptr;
    TPCG_TRY(priv_stream(&s));
    TPCG_CUDA(cudaMemsetAsync(dst, 0, bytes, s));
    TPCG_CUDA(cudaStreamSynchronize(s));
    return TPCG_OK;
}

// upload host doubles converted to the compute dtype
static int upload(void** dst, const double* src, size_t count, int dtype, std::vector<void*>* owned) {
    TPCG_TRY(dmalloc(dst, std::max<size_t>(count, 1) * elt_of(dtype), owned));
    if (count == 0) return TPCG_OK;
    if (dtype == TPCG_F64) {
        TPCG_TRY(sync_to_device(*dst, src, count * sizeof(double)));
    } else {
        std::vector<float> tmp(src, src + count);
        TPCG_TRY(sync_to_device(*dst, tmp.data(), count * sizeof(float)));
    }
    return TPCG_OK;
}

static int upload_int(int** dst, const int* src, size_t count, std::vector<void*>* owned) {
    TPCG_TRY(dmalloc(reinterpret_cast<void**>(dst), std::max<size_t>(count, 1) * sizeof(int), owned));
    if (count) TPCG_TRY(sync_to_device(*dst, src, count * sizeof(int)));
    return TPCG_OK;
}

// ------------------------------------------------------------------------------------ scalars of Alg. 5
// (slot layout in kernels.cuh)

__global__ void scalar_kernel(int op, double* s, const double* prm) {
    if (threadIdx.x != 0) return;
    switch (op) {
        case OP_INIT: {   // r_0 = f (x_0 = 0), s[S_RR] = <f, f>
            double nf = sqrt(fmax(s[S_RR], 0.0));
            s[S_NF] = nf;
            s[S_NR] = nf;
            s[S_ETA] = nf > 0 ? prm[P_BT] * prm[P_TOL] : 1.0;
            s[S_EPS] = prm[P_EPS0];
            s[S_EPSMIN] = prm[P_EPSMIN] > 0 ? prm[P_EPSMIN] : prm[P_TOL] * nf * 0.1;
            s[S_STOP] = (nf <= 0.0) ? 1.0 : 0.0;
            s[S_BAD] = isfinite(nf) ? 0.0 : 1.0;
            s[S_TRIALS] = 0.0;
            break;
        }
        case OP_OMEGA: {
            double xi = s[S_XI];
            if (!(xi > 0.0) || !isfinite(xi) || !isfinite(s[S_RP])) s[S_BAD] = 1.0;
            s[S_OMEGA] = s[S_RP] / xi;
            break;
        }
        case OP_DT: {     // Alg. 2: v = (Delta x~ . Delta x) / ||Delta x~||^2 with Delta x~ = omega p
            double den = s[S_OMEGA] * s[S_PP];
            double v = den != 0.0 ? (s[S_PXN] - s[S_PXK]) / den : 1.0;
            s[S_V] = v;
            s[S_TRIALS] += 1.0;
            if (fabs(v - 1.0) < prm[P_DELTA] || !isfinite(v)) {
                s[S_DONE] = 1.0;
            } else if (prm[P_ALPHA] * s[S_EPS] > s[S_EPSMIN]) {
                s[S_EPS] *= prm[P_ALPHA];
                s[S_DONE] = 0.0;
            } else {
                s[S_DONE] = 1.0;
            }
            break;
        }
        case OP_RES: {    // after r_{k+1}: ||r||, eta_{k+1} (eq. rel_tol_iterates), stopping test
            double nr = sqrt(fmax(s[S_RR], 0.0));
            s[S_NR] = nr;
            s[S_ETA] = nr > 0 ? fmin(prm[P_BT] * prm[P_TOL] * s[S_NF] / nr, 1.0) : 1.0;
            s[S_STOP] = (nr <= prm[P_TOL] * s[S_NF]) ? 1.0 : 0.0;
            if (!isfinite(nr)) s[S_BAD] = 1.0;
            break;
        }
        case OP_BETA: {
            s[S_BETA] = -s[S_ZQ] / s[S_XI];
            break;
        }
        case OP_XI: {
            if (!(s[S_XI] > 0.0) || !isfinite(s[S_XI])) s[S_BAD] = 1.0;
            break;
        }
    }
}

void launch_scalar(int op, double* s, const double* prm, cudaStream_t st) {
    scalar_kernel<<<1, 32, 0, st>>>(op, s, prm);
    g_launches.fetch_add(1, std::memory_order_relaxed);
}

// ------------------------------------------------------------------------------------ dispatch helpers
template <typename F>
static int by_dtype(int dtype, F&& f) {
    if (dtype == TPCG_F64) return f(double());
    if (dtype == TPCG_F32) return f(float());
    set_error("unknown dtype");
    return TPCG_E_INVALID;
}

int check_tensor(const tucker_t* t, int n, int dtype, const char* what) {
    if (!t || !t->desc || !t->U[0] || !t->U[1] || !t->U[2] || !t->core) {
        set_error(std::string(what) + ": null pointer in tucker_t");
        return TPCG_E_INVALID;
    }
    if (t->n != n || t->dtype != dtype || t->cap <= 0 || t->core_cap < 0) {
        set_error(std::string(what) + ": tucker_t has wrong n/dtype/cap");
        return TPCG_E_INVALID;
    }
    return TPCG_OK;
}

}  // namespace tpcg

using namespace tpcg;

// ======================================================================================= misc
extern "C" const char* tpcg_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* tpcg_version(void) { return "tpcg-gb300 0.1 (sm_103a)"; }

extern "C" void tpcg_params_default(tpcg_params* p) {
    p->tol = 1e-6;
    p->eps0 = 0.1;
    p->eps_min = 0.0;
    p->alpha = 0.5;
    p->delta = 1e-3;
    p->beta_trunc = 0.1;
    p->max_it = 500;
    p->rank_cap = 0;
    p->inner_tol = 2e-2;
    p->max_outer = 12;
    p->refine_keep = 3e-2;
}

// ======================================================================================= contexts
static size_t ctx_layout(int n, int max_cols, int rc, int dtype, size_t* sizes, bool rr) {
    const size_t e = elt_of(dtype);
    const size_t nn = (size_t)n * n;
    size_t i = 0;
    sizes[i++] = (size_t)n * nn * e;                         // Z0
    sizes[i++] = (size_t)n * nn * e;                         // Z1
    sizes[i++] = nn * (size_t)max_cols * e;                  // Wm
    sizes[i++] = (size_t)max_cols * n * rc * e;              // T1
    for (int t = 0; t < 9; ++t) sizes[i++] = nn * e;         // Rq, Qq, Yw
    sizes[i++] = nn * e;                                     // Gm
    sizes[i++] = (size_t)MAX_SPLIT * nn * e;                 // Part
    for (int t = 0; t < 3; ++t) sizes[i++] = nn * e;         // S
    sizes[i++] = (size_t)n * sizeof(double);                 // evals
    sizes[i++] = (2 * TPCG_MAX_BLOCKS + 64) * sizeof(GemmArgs);
    sizes[i++] = sizeof(RoundPlan);
    sizes[i++] = 256 * sizeof(double);                       // scal
    sizes[i++] = 3 * (size_t)rc * rc * e;                    // dotw
    sizes[i++] = 2 * (size_t)rc * rc * rc * e;               // dotT
    for (int t = 0; t < 12; ++t) sizes[i++] = (size_t)n * max_cols * e;   // fd scratch
    const size_t rrb = rr ? (size_t)n * RR_L * e : 0;
    for (int t = 0; t < 3; ++t) sizes[i++] = rrb;                         // rrY, rrQ, rrW
    size_t tot = eig_work_bytes(n);
    for (size_t j = 0; j < i; ++j) tot += (sizes[j] + 255) & ~(size_t)255;
    return tot;
}

// the solver tensors a context allocates on first use: 10 for a scalar solve, 17 for the FP64 level of a mixed
// solve (its FP64 fallback inner solve uses tensors 10..16), 21 for an elasticity solve
static size_t tens_bytes(int n, int max_cols, int rc, int dtype, int count = 10) {
    return count * ((3 * (size_t)n * max_cols + (size_t)rc * rc * rc) * elt_of(dtype) + TPCG_DESC_BYTES);
}

extern "C" size_t tpcg_ctx_bytes(int n, int max_cols, int rank_cap, int dtype) {
    size_t sizes[64];
    if (dtype == TPCG_MIXED)
        return ctx_layout(n, max_cols, rank_cap, TPCG_F64, sizes, rr_context(n, rank_cap, TPCG_F64)) +
               ctx_layout(n, max_cols, rank_cap, TPCG_F32, sizes, rr_context(n, rank_cap, TPCG_F32)) +
               tens_bytes(n, max_cols, rank_cap, TPCG_F64, 17) + tens_bytes(n, max_cols, rank_cap, TPCG_F32) +
               2 * eig_work_bytes(n);
    return ctx_layout(n, max_cols, rank_cap, dtype, sizes, rr_context(n, rank_cap, dtype)) +
           tens_bytes(n, max_cols, rank_cap, dtype) +
           eig_work_bytes(n);
}

extern "C" void tpcg_ctx_destroy(tpcg_ctx c) {
    if (!c) return;
    if (c->lo) tpcg_ctx_destroy(c->lo);
    if (c->sync_ev) cudaEventDestroy(c->sync_ev);
    if (c->hstage) cudaFreeHost(c->hstage);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    for (auto& g : c->rgraphs) cudaGraphExecDestroy(g.exec);
    for (void* p : c->owned) cudaFree(p);
    delete c;
}

extern "C" int tpcg_ctx_create(int n, int max_cols, int rank_cap, int dtype, tpcg_ctx* out) {
    if (dtype == TPCG_MIXED) {
        tpcg_ctx hi = nullptr, lo = nullptr;
        TPCG_TRY(tpcg_ctx_create(n, max_cols, rank_cap, TPCG_F64, &hi));
        int s = tpcg_ctx_create(n, max_cols, rank_cap, TPCG_F32, &lo);
        if (s != TPCG_OK) {
            tpcg_ctx_destroy(hi);
            return s;
        }
        hi->lo = lo;
        *out = hi;
        return TPCG_OK;
    }
    if (!out || n < 2 || n > 1024 || max_cols < 1 || rank_cap < 1 || rank_cap > n || rank_cap > 256 ||
        (dtype != TPCG_F64 && dtype != TPCG_F32)) {
        set_error("tpcg_ctx_create: invalid arguments (need 2 <= n <= 1024, 1 <= rank_cap <= min(n, 256))");
        return TPCG_E_INVALID;
    }
    // per-device launch attributes are settled here, outside any stream capture
    TPCG_TRY(eig_prepare());
    TPCG_TRY(tc_prepare());
    (void)sm_count();
    tpcg_ctx c = new tpcg_ctx_s();
    c->lo = nullptr;
    c->sync_ev = nullptr;
    c->hstage = nullptr;
    c->own_stream = nullptr;
    if (cudaEventCreateWithFlags(&c->sync_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        c->sync_ev = nullptr;
        set_error("tpcg_ctx_create: cudaEventCreateWithFlags failed");
        delete c;
        return TPCG_E_CUDA;
    }
    if (cudaHostAlloc(reinterpret_cast<void**>(&c->hstage), TPCG_HSTAGE_BYTES, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        c->hstage = nullptr;
        cudaEventDestroy(c->sync_ev);
        set_error("tpcg_ctx_create: cudaHostAlloc of the staging buffer failed");
        delete c;
        return TPCG_E_NOMEM;
    }
    c->n = n;
    c->max_cols = max_cols;
    c->rank_cap = rank_cap;
    c->dtype = dtype;
    c->elt = elt_of(dtype);
    c->have_tens = 0;
    c->tens_cap = 0;
    size_t sizes[64];
    c->rr = rr_context(n, rank_cap, dtype) ? 1 : 0;
    ctx_layout(n, max_cols, rank_cap, dtype, sizes, c->rr != 0);
    void** slots[64];
    int i = 0;
    slots[i++] = &c->Z0;
    slots[i++] = &c->Z1;
    slots[i++] = &c->Wm;
    slots[i++] = &c->T1;
    for (int t = 0; t < 3; ++t) slots[i++] = &c->Rq[t];
    for (int t = 0; t < 3; ++t) slots[i++] = &c->Qq[t];
    for (int t = 0; t < 3; ++t) slots[i++] = &c->Yw[t];
    slots[i++] = &c->Gm;
    slots[i++] = &c->Part;
    for (int t = 0; t < 3; ++t) slots[i++] = &c->S[t];
    slots[i++] = reinterpret_cast<void**>(&c->evals);
    slots[i++] = reinterpret_cast<void**>(&c->gargs);
    slots[i++] = reinterpret_cast<void**>(&c->plan);
    slots[i++] = reinterpret_cast<void**>(&c->scal);
    slots[i++] = reinterpret_cast<void**>(&c->dotw);
    slots[i++] = &c->dotT;
    for (int t = 0; t < 3; ++t)
        for (int q = 0; q < 4; ++q) slots[i++] = &c->fd[t][q];
    slots[i++] = &c->rrY;
    slots[i++] = &c->rrQ;
    slots[i++] = &c->rrW;
    for (int j = 0; j < i; ++j) {
        int s = dmalloc(slots[j], sizes[j], &c->owned);
        if (s != TPCG_OK) {
            tpcg_ctx_destroy(c);
            return s;
        }
    }
    {
        int s = eig_work_alloc(&c->eigw, n, &c->owned);
        if (s != TPCG_OK) {
            tpcg_ctx_destroy(c);
            return s;
        }
    }
    {
        const int s = sync_zero(c->scal, 256 * sizeof(double));
        if (s != TPCG_OK) {
            tpcg_ctx_destroy(c);
            return s;
        }
    }
    *out = c;
    return TPCG_OK;
}

// ======================================================================================= problems
static void host_orthonormalize_rhs(tpcg_problem pb) {
    // F_t = Q_t R_t (modified Gram-Schmidt, twice), core <- core x_t R_t: an exact change of basis.
    const int n = pb->n;
    std::vector<double> core = pb->f_core;
    int r[3] = {pb->rf[0], pb->rf[1], pb->rf[2]};
    for (int t = 0; t < 3; ++t) {
        const int k = r[t];
        std::vector<double>& F = pb->f_U[t];
        std::vector<double> Rm((size_t)k * k, 0.0);
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<double> Rp((size_t)k * k, 0.0);
            for (int j = 0; j < k; ++j) {
                double* fj = &F[(size_t)j * n];
                for (int i = 0; i < j; ++i) {
                    const double* fi = &F[(size_t)i * n];
                    double d = 0;
                    for (int q = 0; q < n; ++q) d += fi[q] * fj[q];
                    for (int q = 0; q < n; ++q) fj[q] -= d * fi[q];
                    Rp[i + (size_t)j * k] = d;
                }
                double nr = 0;
                for (int q = 0; q < n; ++q) nr += fj[q] * fj[q];
                nr = sqrt(nr);
                Rp[j + (size_t)j * k] = nr;
                if (nr > 0)
                    for (int q = 0; q < n; ++q) fj[q] /= nr;
            }
            if (pass == 0) {
                Rm = Rp;
            } else {   // R = Rp * Rm
                std::vector<double> Rn((size_t)k * k, 0.0);
                for (int i = 0; i < k; ++i)
                    for (int j = 0; j < k; ++j) {
                        double s = 0;
                        for (int q = 0; q < k; ++q) s += Rp[i + (size_t)q * k] * Rm[q + (size_t)j * k];
                        Rn[i + (size_t)j * k] = s;
                    }
                Rm = Rn;
            }
        }
        // core <- core x_t Rm
        std::vector<double> nc(core.size(), 0.0);
        int d[3] = {r[0], r[1], r[2]};
        for (int a = 0; a < d[0]; ++a)
            for (int b = 0; b < d[1]; ++b)
                for (int c = 0; c < d[2]; ++c) {
                    int idx[3] = {a, b, c};
                    double s = 0;
                    for (int q = 0; q < k; ++q) {
                        int jdx[3] = {a, b, c};
                        jdx[t] = q;
                        s += Rm[idx[t] + (size_t)q * k] * core[jdx[0] + (size_t)d[0] * (jdx[1] + (size_t)d[1] * jdx[2])];
                    }
                    nc[a + (size_t)d[0] * (b + (size_t)d[1] * c)] = s;
                }
        core = nc;
    }
    pb->f_core = core;
}

extern "C" void tpcg_problem_destroy(tpcg_problem pb) {
    if (!pb) return;
    if (pb->lo) tpcg_problem_destroy(pb->lo);
    void* ptrs[] = {pb->d_bands, pb->d_w, pb->d_lam, pb->d_mu, pb->d_wrow, pb->d_wcol, pb->d_wval, pb->d_wtrow,
                    pb->d_wtcol, pb->d_wtval, pb->d_v2u2, pb->d_dst, pb->d_chirp, pb->d_omega, pb->d_alpha, pb->d_scal,
                    pb->d_f_store[0], pb->d_f_store[1], pb->d_f_store[2], pb->d_f_store[3], pb->d_f_store[4]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete pb;
}

extern "C" int tpcg_problem_create(const tpcg_problem_arrays* a, tpcg_problem* out) {
    if (!a || !out) return TPCG_E_INVALID;
    if (a->dtype == TPCG_MIXED) {
        tpcg_problem_arrays b = *a;
        b.dtype = TPCG_F64;
        tpcg_problem hi = nullptr, lo = nullptr;
        TPCG_TRY(tpcg_problem_create(&b, &hi));
        b.dtype = TPCG_F32;
        int s = tpcg_problem_create(&b, &lo);
        if (s != TPCG_OK) {
            tpcg_problem_destroy(hi);
            return s;
        }
        hi->lo = lo;
        *out = hi;
        return TPCG_OK;
    }
    const int n = a->n, p = a->p;
    if (n < 2 || p < 1 || p > 5 || a->R < 1 || a->R > TPCG_MAX_BLOCKS - 1 || a->n1 < 1 || a->n2 < 0 ||
        a->n1 + a->n2 != n || a->RP < 1 || a->RP > TPCG_MAX_BLOCKS || (a->dtype != TPCG_F64 && a->dtype != TPCG_F32) ||
        !a->w || !a->bands || !a->f_core || !a->lam || !a->mu || !a->w_rowptr || !a->omega || !a->alpha ||
        a->lambda_min <= 0 || a->k0 < 0 || a->k0 > 1 || a->k1 < 0 || a->k1 > 1 || (a->k0 && a->k1)) {
        set_error("tpcg_problem_create: invalid arguments");
        return TPCG_E_INVALID;
    }
    for (int t = 0; t < 3; ++t)
        if (a->rf[t] < 1 || a->rf[t] > n || !a->f_U[t]) {
            set_error("tpcg_problem_create: invalid rhs");
            return TPCG_E_INVALID;
        }
    {   // every table must be finite: a NaN or Inf is refused here, before anything reaches the device
        const int bw = 2 * p + 1;
        const int nnz = a->w_rowptr[n];
        auto finite = [](const double* v, size_t cnt) {
            for (size_t i = 0; i < cnt; ++i)
                if (!std::isfinite(v[i])) return false;
            return true;
        };
        bool ok = nnz >= 0 && (nnz == 0 || a->w_val) && std::isfinite(a->lambda_min) &&
                  finite(a->w, a->R) && finite(a->bands, (size_t)a->R * 3 * bw * n) &&
                  finite(a->f_core, (size_t)a->rf[0] * a->rf[1] * a->rf[2]) && finite(a->lam, n) &&
                  finite(a->mu, a->n1) && finite(a->omega, a->RP) && finite(a->alpha, a->RP) &&
                  (nnz == 0 || finite(a->w_val, nnz)) && (a->n2 == 0 || !a->v2u2 || finite(a->v2u2, (size_t)n * a->n2));
        for (int t = 0; t < 3 && ok; ++t) ok = finite(a->f_U[t], (size_t)n * a->rf[t]);
        if (!ok) {
            set_error("tpcg_problem_create: a table holds a NaN or an Inf");
            return TPCG_E_INVALID;
        }
    }
    tpcg_problem pb = new tpcg_problem_s();
    pb->lo = nullptr;
    pb->d_chirp = nullptr;
    memset(pb->d_f_store, 0, sizeof(pb->d_f_store));
    pb->d_bands = pb->d_w = nullptr;
    pb->d_lam = pb->d_mu = pb->d_wval = pb->d_wtval = pb->d_v2u2 = pb->d_dst = nullptr;
    pb->d_wrow = pb->d_wcol = pb->d_wtrow = pb->d_wtcol = nullptr;
    pb->d_omega = pb->d_alpha = pb->d_scal = nullptr;
    pb->n = n; pb->p = p; pb->R = a->R; pb->RP = a->RP; pb->n1 = a->n1; pb->n2 = a->n2; pb->dtype = a->dtype;
    pb->k0 = a->k0; pb->k1 = a->k1;
    for (int t = 0; t < 3; ++t) pb->rf[t] = a->rf[t];
    pb->lambda_min = a->lambda_min;
    const int bw = 2 * p + 1;
    pb->w.assign(a->w, a->w + a->R);
    pb->bands.assign(a->bands, a->bands + (size_t)a->R * 3 * bw * n);
    pb->f_core.assign(a->f_core, a->f_core + (size_t)a->rf[0] * a->rf[1] * a->rf[2]);
    for (int t = 0; t < 3; ++t) pb->f_U[t].assign(a->f_U[t], a->f_U[t] + (size_t)n * a->rf[t]);
    pb->lam.assign(a->lam, a->lam + n);
    pb->mu.assign(a->mu, a->mu + a->n1);
    const int nnz = a->w_rowptr[n];
    pb->w_rowptr.assign(a->w_rowptr, a->w_rowptr + n + 1);
    pb->w_col.assign(a->w_col, a->w_col + nnz);
    pb->w_val.assign(a->w_val, a->w_val + nnz);
    pb->v2u2.assign(a->v2u2 ? a->v2u2 : a->lam, a->v2u2 ? a->v2u2 + (size_t)n * a->n2 : a->lam);
    pb->omega.assign(a->omega, a->omega + a->RP);
    pb->alpha.assign(a->alpha, a->alpha + a->RP);
    double lmax = 0;
    for (int i = 0; i < n; ++i) lmax = std::max(lmax, pb->lam[i]);
    pb->lambda_max = 3.0 * lmax;
    for (int e = 0; e < nnz; ++e)
        if (pb->w_col[e] < 0 || pb->w_col[e] >= a->n1) {
            delete pb;
            set_error("tpcg_problem_create: W column index out of range");
            return TPCG_E_INVALID;
        }
    host_orthonormalize_rhs(pb);
    double nf2 = 0;
    for (double v : pb->f_core) nf2 += v * v;
    pb->norm_f = sqrt(nf2);

    // W^T in CSR
    std::vector<int> trow(a->n1 + 1, 0), tcol(nnz);
    std::vector<double> tval(nnz);
    for (int e = 0; e < nnz; ++e) trow[pb->w_col[e] + 1]++;
    for (int l = 0; l < a->n1; ++l) trow[l + 1] += trow[l];
    {
        std::vector<int> fill(trow.begin(), trow.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int e = pb->w_rowptr[i]; e < pb->w_rowptr[i + 1]; ++e) {
                int l = pb->w_col[e];
                tcol[fill[l]] = i;
                tval[fill[l]] = pb->w_val[e];
                fill[l]++;
            }
    }
    // sine matrix U_dft[l, j] = sqrt2 sin(omega_j x_l + k0 pi/2) with the phase reduced exactly on its integer grid
    const int n1 = a->n1;
    const SineGrid sg = sine_grid(n1, p, a->k0, a->k1);
    std::vector<double> dst((size_t)n1 * n1);
    for (long long j = 0; j < n1; ++j)
        for (long long l = 0; l < n1; ++l) {
            const long long m = ((2 * j + sg.e) * (2 * l + sg.c) + sg.g) % (8 * sg.D);
            dst[l + j * n1] = sqrt(2.0) * sin(M_PI * (double)m / (4.0 * (double)sg.D));
        }
    std::vector<void*> owned;   // not used: problem buffers are tracked in the struct
    int s = TPCG_OK;
    auto fail = [&](int code) {
        tpcg_problem_destroy(pb);
        return code;
    };
    const int dt = a->dtype;
    if ((s = upload(&pb->d_bands, pb->bands.data(), pb->bands.size(), dt, nullptr))) return fail(s);
    if ((s = dmalloc(reinterpret_cast<void**>(&pb->d_w), a->R * sizeof(double), nullptr))) return fail(s);
    if ((s = sync_to_device(pb->d_w, pb->w.data(), a->R * sizeof(double)))) return fail(s);
    if ((s = upload(&pb->d_lam, pb->lam.data(), n, dt, nullptr))) return fail(s);
    if ((s = upload(&pb->d_mu, pb->mu.data(), n1, dt, nullptr))) return fail(s);
    if ((s = upload_int(&pb->d_wrow, pb->w_rowptr.data(), n + 1, nullptr))) return fail(s);
    if ((s = upload_int(&pb->d_wcol, pb->w_col.data(), nnz, nullptr))) return fail(s);
    if ((s = upload(&pb->d_wval, pb->w_val.data(), nnz, dt, nullptr))) return fail(s);
    if ((s = upload_int(&pb->d_wtrow, trow.data(), n1 + 1, nullptr))) return fail(s);
    if ((s = upload_int(&pb->d_wtcol, tcol.data(), nnz, nullptr))) return fail(s);
    if ((s = upload(&pb->d_wtval, tval.data(), nnz, dt, nullptr))) return fail(s);
    if ((s = upload(&pb->d_v2u2, pb->v2u2.data(), (size_t)n * a->n2, dt, nullptr))) return fail(s);
    if ((s = upload(&pb->d_dst, dst.data(), dst.size(), dt, nullptr))) return fail(s);
    if (n1 <= 1024) {   // FFT sine transforms (complex pairs in the compute dtype)
        std::vector<double> ct;
        if ((s = chirp_tables(n1, p, a->k0, a->k1, &pb->chirp, &ct))) return fail(s);
        if ((s = upload(&pb->d_chirp, ct.data(), ct.size(), dt, nullptr))) return fail(s);
    }
    if ((s = dmalloc(reinterpret_cast<void**>(&pb->d_omega), a->RP * sizeof(double), nullptr))) return fail(s);
    if ((s = dmalloc(reinterpret_cast<void**>(&pb->d_alpha), a->RP * sizeof(double), nullptr))) return fail(s);
    if ((s = sync_to_device(pb->d_omega, pb->omega.data(), a->RP * sizeof(double)))) return fail(s);
    if ((s = sync_to_device(pb->d_alpha, pb->alpha.data(), a->RP * sizeof(double)))) return fail(s);
    if ((s = dmalloc(reinterpret_cast<void**>(&pb->d_scal), 64 * sizeof(double), nullptr))) return fail(s);
    if ((s = sync_zero(pb->d_scal, 64 * sizeof(double)))) return fail(s);
    // rhs tensor
    tucker_t& f = pb->f;
    f.dtype = dt;
    f.n = n;
    f.cap = std::max(pb->rf[0], std::max(pb->rf[1], pb->rf[2]));
    f.core_cap = (long long)pb->rf[0] * pb->rf[1] * pb->rf[2];
    for (int t = 0; t < 3; ++t) {
        std::vector<double> padded((size_t)n * f.cap, 0.0);
        std::copy(pb->f_U[t].begin(), pb->f_U[t].end(), padded.begin());
        if ((s = upload(&pb->d_f_store[t], padded.data(), padded.size(), dt, nullptr))) return fail(s);
        f.U[t] = pb->d_f_store[t];
    }
    if ((s = upload(&pb->d_f_store[3], pb->f_core.data(), pb->f_core.size(), dt, nullptr))) return fail(s);
    f.core = pb->d_f_store[3];
    if ((s = dmalloc(&pb->d_f_store[4], TPCG_DESC_BYTES, nullptr))) return fail(s);
    f.desc = pb->d_f_store[4];
    // the descriptor kernel runs on this thread's private stream and only that stream is waited for: a
    // device-wide synchronisation would also wait for (and, while another thread captures a CUDA graph,
    // invalidate the capture of) the solves running concurrently
    cudaStream_t ps = nullptr;
    if ((s = priv_stream(&ps))) return fail(s);
    if ((s = set_plain(&f, pb->rf[0], pb->rf[1], pb->rf[2], ps))) return fail(s);
    if (cudaStreamSynchronize(ps) != cudaSuccess) {
        set_error("tpcg_problem_create: device error");
        return fail(TPCG_E_CUDA);
    }
    *out = pb;
    return TPCG_OK;
}

extern "C" int tpcg_setup(const tpcg_geometry* geo, int degree, int n, int dtype, tpcg_problem* out) {
    if (!geo || !out) return TPCG_E_INVALID;
    HostProblem hp;
    int s = host_setup(*geo, degree, n, &hp);
    if (s != TPCG_OK) return s;
    tpcg_problem_arrays a{};
    a.n = n; a.p = degree; a.R = hp.R; a.dtype = dtype;
    a.w = hp.w.data();
    a.bands = hp.bands.data();
    for (int t = 0; t < 3; ++t) { a.rf[t] = hp.rf[t]; a.f_U[t] = hp.f_U[t].data(); }
    a.f_core = hp.f_core.data();
    a.n1 = hp.n1; a.n2 = hp.n2; a.RP = hp.RP; a.w_nnz = (int)hp.w_val.size();
    a.lam = hp.lam.data(); a.mu = hp.mu.data();
    a.w_rowptr = hp.w_rowptr.data(); a.w_col = hp.w_col.data(); a.w_val = hp.w_val.data();
    a.v2u2 = hp.v2u2.empty() ? nullptr : hp.v2u2.data();
    a.omega = hp.omega.data(); a.alpha = hp.alpha.data(); a.lambda_min = hp.lambda_min;
    a.k0 = hp.k0; a.k1 = hp.k1;
    return tpcg_problem_create(&a, out);
}

extern "C" int tpcg_problem_get_info(tpcg_problem pb, tpcg_problem_info* o) {
    if (!pb || !o) return TPCG_E_INVALID;
    o->n = pb->n; o->p = pb->p; o->R = pb->R; o->RP = pb->RP; o->n1 = pb->n1; o->n2 = pb->n2; o->dtype = pb->dtype;
    for (int t = 0; t < 3; ++t) o->rf[t] = pb->rf[t];
    o->lambda_min = pb->lambda_min;
    o->lambda_max = pb->lambda_max;
    o->MP = pb->lambda_max / pb->lambda_min;
    o->norm_f = pb->norm_f;
    o->w_nnz = (int)pb->w_val.size();
    o->k0 = pb->k0;
    o->k1 = pb->k1;
    return TPCG_OK;
}

extern "C" int tpcg_problem_export_w(tpcg_problem pb, int* rowptr, int* col, double* val) {
    if (!pb) return TPCG_E_INVALID;
    if (rowptr) memcpy(rowptr, pb->w_rowptr.data(), pb->w_rowptr.size() * sizeof(int));
    if (col && !pb->w_col.empty()) memcpy(col, pb->w_col.data(), pb->w_col.size() * sizeof(int));
    if (val && !pb->w_val.empty()) memcpy(val, pb->w_val.data(), pb->w_val.size() * sizeof(double));
    return TPCG_OK;
}

extern "C" int tpcg_problem_export(tpcg_problem pb, double* w, double* bands, double* f_core, double* f_U0,
                                   double* f_U1, double* f_U2, double* lam, double* mu, double* v2u2, double* omega,
                                   double* alpha) {
    if (!pb) return TPCG_E_INVALID;
    auto cp = [](double* dst, const std::vector<double>& v) {
        if (dst && !v.empty()) memcpy(dst, v.data(), v.size() * sizeof(double));
    };
    cp(w, pb->w);
    cp(bands, pb->bands);
    cp(f_core, pb->f_core);
    cp(f_U0, pb->f_U[0]);
    cp(f_U1, pb->f_U[1]);
    cp(f_U2, pb->f_U[2]);
    cp(lam, pb->lam);
    cp(mu, pb->mu);
    if (pb->n2 > 0) cp(v2u2, pb->v2u2);
    cp(omega, pb->omega);
    cp(alpha, pb->alpha);
    return TPCG_OK;
}

// ======================================================================================= Tucker ops
extern "C" int tucker_set_plain(tucker_t* t, int r1, int r2, int r3, void* stream) {
    if (!t || !t->desc || r1 < 0 || r2 < 0 || r3 < 0 || r1 > t->cap || r2 > t->cap || r3 > t->cap ||
        (long long)r1 * r2 * r3 > t->core_cap) {
        set_error("tucker_set_plain: ranks exceed capacities");
        return TPCG_E_INVALID;
    }
    return set_plain(t, r1, r2, r3, S(stream));
}

extern "C" int tucker_get_ranks(const tucker_t* t, int* r3_out, int* nblk_out, void* stream) {
    if (!t || !t->desc) return TPCG_E_INVALID;
    int h[4];
    TPCG_CUDA(cudaMemcpyAsync(h, t->desc, sizeof(h), cudaMemcpyDeviceToHost, S(stream)));
    TPCG_CUDA(cudaStreamSynchronize(S(stream)));
    if (nblk_out) *nblk_out = h[0];
    if (r3_out)
        for (int q = 0; q < 3; ++q) r3_out[q] = h[1 + q];
    return TPCG_OK;
}

extern "C" int tucker_apply(tpcg_problem pb, const tucker_t* x, tucker_t* y, void* stream) {
    if (!pb) return TPCG_E_INVALID;
    TPCG_TRY(check_tensor(x, pb->n, pb->dtype, "tucker_apply x"));
    TPCG_TRY(check_tensor(y, pb->n, pb->dtype, "tucker_apply y"));
    return by_dtype(pb->dtype, [&](auto z) { return apply_impl<decltype(z)>(pb, x, y, false, S(stream)); });
}

extern "C" int tucker_residual(tpcg_problem pb, const tucker_t* x, tucker_t* y, void* stream) {
    if (!pb) return TPCG_E_INVALID;
    TPCG_TRY(check_tensor(x, pb->n, pb->dtype, "tucker_residual x"));
    TPCG_TRY(check_tensor(y, pb->n, pb->dtype, "tucker_residual y"));
    return by_dtype(pb->dtype, [&](auto z) { return apply_impl<decltype(z)>(pb, x, y, true, S(stream)); });
}

extern "C" int tucker_axpby(double a, const double* a_dev, const tucker_t* x, double b, const double* b_dev,
                            const tucker_t* y, tucker_t* z, void* stream) {
    if (!x || !y || !z) return TPCG_E_INVALID;
    TPCG_TRY(check_tensor(x, z->n, z->dtype, "tucker_axpby x"));
    TPCG_TRY(check_tensor(y, z->n, z->dtype, "tucker_axpby y"));
    TPCG_TRY(check_tensor(z, z->n, z->dtype, "tucker_axpby z"));
    if (z == x || z == y || z->desc == x->desc || z->desc == y->desc) {
        set_error("tucker_axpby: output must not alias an input");
        return TPCG_E_INVALID;
    }
    return by_dtype(z->dtype, [&](auto q) {
        return axpby_impl<decltype(q)>(a, a_dev, x, b, b_dev, y, z, nullptr, S(stream));
    });
}

// Outside a stream capture, the public scalar products read both descriptors (16 bytes each, synchronising
// the stream) and refuse a block tensor or a rank above the scratch limit with TPCG_E_INVALID.  Inside a
// capture nothing can be read back: the kernels then write NaN for such inputs.
static int check_dot_inputs(const tucker_t* x, const tucker_t* y, int max_rank, cudaStream_t st, const char* what) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    TPCG_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return TPCG_OK;
    int h[2][4];
    TPCG_CUDA(cudaMemcpyAsync(h[0], x->desc, sizeof(h[0]), cudaMemcpyDeviceToHost, st));
    TPCG_CUDA(cudaMemcpyAsync(h[1], y->desc, sizeof(h[1]), cudaMemcpyDeviceToHost, st));
    TPCG_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < 2; ++q) {
        if (h[q][0] != 1) {
            set_error(std::string(what) + ": " + (q ? "y" : "x") + " is not a plain tensor (" + std::to_string(h[q][0]) +
                      " core blocks); round it first");
            return TPCG_E_INVALID;
        }
        for (int t = 0; t < 3; ++t)
            if (h[q][1 + t] > max_rank) {
                set_error(std::string(what) + ": rank " + std::to_string(h[q][1 + t]) + " exceeds the limit " +
                          std::to_string(max_rank));
                return TPCG_E_INVALID;
            }
    }
    return TPCG_OK;
}

extern "C" int tucker_dot(tpcg_ctx c, const tucker_t* x, const tucker_t* y, double* out_dev, void* stream) {
    if (!c || !out_dev) return TPCG_E_INVALID;
    TPCG_TRY(check_tensor(x, c->n, c->dtype, "tucker_dot x"));
    TPCG_TRY(check_tensor(y, c->n, c->dtype, "tucker_dot y"));
    TPCG_TRY(check_dot_inputs(x, y, c->rank_cap, S(stream), "tucker_dot"));
    return by_dtype(c->dtype, [&](auto z) { return dot_impl<decltype(z)>(c, x, y, out_dev, S(stream)); });
}

extern "C" int tucker_dot_static(const tucker_t* x, const tucker_t* y, double* out_dev, void* stream) {
    if (!x || !y || !out_dev) {
        set_error("tucker_dot_static: null argument");
        return TPCG_E_INVALID;
    }
    TPCG_TRY(check_tensor(x, x->n, x->dtype, "tucker_dot_static x"));
    TPCG_TRY(check_tensor(y, x->n, x->dtype, "tucker_dot_static y"));
    if (x->dtype != TPCG_F64 && x->dtype != TPCG_F32) {
        set_error("tucker_dot_static: dtype must be TPCG_F64 or TPCG_F32");
        return TPCG_E_INVALID;
    }
    const int mr = dot_static_max_rank();
    if (x->cap > mr || y->cap > mr) {
        set_error("tucker_dot_static: tensor capacity " + std::to_string(std::max(x->cap, y->cap)) +
                  " exceeds the fixed scratch limit of rank " + std::to_string(mr));
        return TPCG_E_INVALID;
    }
    TPCG_TRY(check_dot_inputs(x, y, mr, S(stream), "tucker_dot_static"));
    return by_dtype(x->dtype, [&](auto z) { return dot_static_impl<decltype(z)>(x, y, out_dev, S(stream)); });
}

extern "C" int tucker_round(tpcg_ctx c, tucker_t* y, double eps, const double* eps_dev, int rank_cap,
                            double* info_dev, void* stream) {
    if (!c || (!eps_dev && !(eps >= 0.0))) return TPCG_E_INVALID;
    TPCG_TRY(check_tensor(y, c->n, c->dtype, "tucker_round y"));
    if (y->cap > c->max_cols) {
        set_error("tucker_round: tensor capacity exceeds the context's max_cols");
        return TPCG_E_INVALID;
    }
    return by_dtype(c->dtype, [&](auto z) {
        using T = decltype(z);
        const int rule = round_rule();
        if constexpr (sizeof(T) == 8) {
            if (rule == 2 && !eps_dev && eps < RESOLVE_BELOW && c->max_cols >= 3 * c->rank_cap) {
                TPCG_TRY(ensure_tensors(c, 3));
                const int rc = (rank_cap > 0 && rank_cap < c->rank_cap) ? rank_cap : c->rank_cap;
                TPCG_TRY(round_resolved(c, y, &c->tens[0], eps, nullptr, rc, c->scal + 143, &c->tens[1],
                                        &c->tens[2], S(stream)));
                int r3[3] = {0, 0, 0}, nb = 0;
                TPCG_TRY(tucker_get_ranks(&c->tens[0], r3, &nb, S(stream)));
                if (r3[0] > y->cap || r3[1] > y->cap || r3[2] > y->cap ||
                    (long long)r3[0] * r3[1] * r3[2] > y->core_cap) {
                    set_error("tucker_round: the resolved result does not fit the tensor's capacity");
                    return TPCG_E_INVALID;
                }
                return copy_tensor_impl<double>(&c->tens[0], y, c->n, y->cap, S(stream));
            }
        }
        return round_impl<T>(c, y, eps, eps_dev, rank_cap, info_dev, S(stream), rule == 2 ? -1 : rule);
    });
}

extern "C" int fd_precond_apply(tpcg_problem pb, tpcg_ctx c, const tucker_t* s, tucker_t* v, void* stream) {
    if (!pb || !c || pb->n != c->n || pb->dtype != c->dtype) return TPCG_E_INVALID;
    TPCG_TRY(check_tensor(s, pb->n, pb->dtype, "fd_precond_apply s"));
    TPCG_TRY(check_tensor(v, pb->n, pb->dtype, "fd_precond_apply v"));
    if (v->cap > c->max_cols) {
        set_error("fd_precond_apply: output capacity exceeds the context's max_cols");
        return TPCG_E_INVALID;
    }
    return by_dtype(pb->dtype, [&](auto z) { return fd_impl<decltype(z)>(pb, c, s, v, S(stream)); });
}

// ======================================================================================= TPCG (Alg. 5)
int tpcg::ensure_tensors(tpcg_ctx c, int count) {
    if (count > TPCG_CTX_TENSORS) {
        set_error("ensure_tensors: too many solver tensors requested");
        return TPCG_E_INVALID;
    }
    if (c->have_tens >= count) return TPCG_OK;
    const int n = c->n, cap = c->max_cols, rc = c->rank_cap;
    for (int i = c->have_tens; i < count; ++i) {
        tucker_t& t = c->tens[i];
        t.dtype = c->dtype;
        t.n = n;
        t.cap = cap;
        t.core_cap = (long long)rc * rc * rc;
        for (int q = 0; q < 3; ++q) TPCG_TRY(dmalloc(&t.U[q], (size_t)n * cap * c->elt, &c->owned));
        TPCG_TRY(dmalloc(&t.core, (size_t)t.core_cap * c->elt, &c->owned));
        TPCG_TRY(dmalloc(&t.desc, TPCG_DESC_BYTES, &c->owned));
        TPCG_TRY(sync_zero(t.desc, TPCG_DESC_BYTES));
        c->have_tens = i + 1;
    }
    return TPCG_OK;
}

// wait on the host for the work enqueued on s so far.  The thread polls an event: a few yields, then short
// sleeps.  Neither spinning in the driver (one core per waiting solver thread) nor a blocking-sync wait
// (woken through the driver's interrupt path, slow once tens of solver threads wait at once) shares the host
// cores as well when many solves run concurrently.
int tpcg::host_wait(tpcg_ctx c, cudaStream_t s) {
    TPCG_CUDA(cudaEventRecord(c->sync_ev, s));
    for (int it = 0;; ++it) {
        const cudaError_t e = cudaEventQuery(c->sync_ev);
        if (e == cudaSuccess) return TPCG_OK;
        if (e != cudaErrorNotReady) {
            cudaGetLastError();
            set_error(std::string("host_wait: ") + cudaGetErrorString(e));
            return TPCG_E_CUDA;
        }
        if (it < 16)
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int tpcg::fetch(tpcg_ctx c, cudaStream_t s, const D2H* items, int count) {
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        if (off + items[i].bytes > TPCG_HSTAGE_BYTES) {
            set_error("fetch: staging buffer too small");
            return TPCG_E_INVALID;
        }
        TPCG_CUDA(cudaMemcpyAsync(c->hstage + off, items[i].src, items[i].bytes, cudaMemcpyDeviceToHost, s));
        off += (items[i].bytes + 7) & ~(size_t)7;
    }
    TPCG_TRY(host_wait(c, s));
    off = 0;
    for (int i = 0; i < count; ++i) {
        memcpy(items[i].dst, c->hstage + off, items[i].bytes);
        off += (items[i].bytes + 7) & ~(size_t)7;
    }
    return TPCG_OK;
}

// ||f - A x|| / ||f|| of a solution x, in the working precision of the problem (no truncation)
template <typename T>
static int true_residual(tpcg_problem pb, tpcg_ctx c, const tucker_t* x, tucker_t* work, double* rel, cudaStream_t s) {
    TPCG_TRY(apply_impl<T>(pb, x, work, true, s, nullptr, reinterpret_cast<int*>(c->scal + 232)));
    double* d = c->scal + 130;
    TPCG_TRY(tensor_norm2<T>(c, work, d, s));
    double h = 0.0;
    TPCG_TRY(fetch(c, s, {{&h, d, sizeof(double)}}));
    *rel = pb->norm_f > 0 ? sqrt(std::max(h, 0.0)) / pb->norm_f : 0.0;
    return TPCG_OK;
}

// Alg. 5 for the right-hand side `rhs` (the problem's f~ unless given)
template <typename T>
static int solve_impl(tpcg_problem pb, tpcg_ctx c, const tpcg_params* prm, tucker_t* xout, tpcg_stats* st,
                      cudaStream_t s, const tucker_t* rhs = nullptr, int tbase = 0) {
    if (!rhs) rhs = &pb->f;
    TPCG_TRY(ensure_tensors(c, std::max(10, tbase + 9)));
    const int rc = (prm->rank_cap > 0 && prm->rank_cap < c->rank_cap) ? prm->rank_cap : c->rank_cap;
    double* sc = c->scal;
    double* dprm = c->scal + 100;
    double hp[P_COUNT] = {prm->tol, prm->eps0, prm->eps_min, prm->alpha, prm->delta, prm->beta_trunc};
    TPCG_CUDA(cudaMemcpyAsync(dprm, hp, sizeof(hp), cudaMemcpyHostToDevice, s));
    // capacity flags of the operator apply and of the preconditioner, read every iteration.  Both live in this
    // context: solves that share the problem never clear or raise each other's flags
    int* apply_err = reinterpret_cast<int*>(sc + 232);
    int* fd_err = reinterpret_cast<int*>(sc + 230);
    TPCG_CUDA(cudaMemsetAsync(apply_err, 0, sizeof(int), s));
    TPCG_CUDA(cudaMemsetAsync(fd_err, 0, sizeof(int), s));
    tucker_t* x = &c->tens[tbase + 0];
    tucker_t* r = &c->tens[tbase + 1];
    tucker_t* z = &c->tens[tbase + 2];
    tucker_t* p = &c->tens[tbase + 3];
    tucker_t* q = &c->tens[tbase + 4];
    tucker_t* big = &c->tens[tbase + 5];
    tucker_t* big2 = &c->tens[tbase + 6];
    tucker_t* rsE = &c->tens[tbase + 7];   // scratch of the resolved rule
    tucker_t* rsF = &c->tens[tbase + 8];
    double* eta = sc + S_ETA;
    // the FP64 rule's strict mode (reading R23) serves solves whose tolerance is below what the Gram resolves;
    // at tol >= 1e-8 Alg. 2's tolerance still falls to eps_min (about tol ||f~|| / 10), where strict mode would
    // keep Gram noise in x up to the rank cap, so those solves use the plain rule
    const int strict = prm->tol < 1e-8 ? -1 : 0;
    auto round_to = [&](tucker_t*& dst, const double* eps_dev) -> int {
        // round `big` in place, then make it the new `dst` (swap buffers)
        TPCG_TRY(round_cached<T>(c, big, eps_dev, rc, s, strict));
        std::swap(dst, big);
        return TPCG_OK;
    };
    // x_0 = 0, r_0 = f
    TPCG_TRY(set_zero(x, s));
    TPCG_TRY(copy_tensor_impl<T>(rhs, r, c->n, c->max_cols, s));
    TPCG_TRY(dot_cached<T>(c, r, r, sc + S_RR, s));
    launch_scalar(OP_INIT, sc, dprm, s);
    // z_0 = T(P^-1 r_0, eta_0), p_0 = z_0, q_0 = T(A p_0, eta_0), xi_0 = p_0 . q_0
    TPCG_TRY(fd_impl<T>(pb, c, r, big, s));
    TPCG_TRY(round_to(z, eta));
    TPCG_TRY(copy_tensor_impl<T>(z, p, c->n, c->max_cols, s));
    TPCG_TRY(apply_impl<T>(pb, p, big, false, s, nullptr, apply_err));
    TPCG_TRY(round_to(q, eta));
    TPCG_TRY(dot_cached<T>(c, p, q, sc + S_XI, s));
    launch_scalar(OP_XI, sc, dprm, s);
    double host[S_COUNT];
    int k = 0;
    int status = TPCG_OK;
    int trials_total = 0;
    double eps_now = prm->eps0;   // Alg. 2 tolerance on the host (fetched with each trial decision)
    const char* tr = getenv("TPCG_TRACE");
    const bool trace = tr && tr[0] == '1';
    c->hist.clear();
    int trials_prev = 0;
    for (;;) {
        int flags[2] = {0, 0};
        TPCG_TRY(fetch(c, s, {{host, sc, sizeof(host)}, {&flags[0], apply_err, sizeof(int)},
                              {&flags[1], fd_err, sizeof(int)}}));
        {   // the scalars after iteration k (the row of k = 0 holds the initial state)
            const double nf = host[S_NF] > 0 ? host[S_NF] : 1.0;
            const double row[TPCG_HIST_COLS] = {host[S_NR] / nf, k ? host[S_OMEGA] : 0.0, k ? host[S_BETA] : 0.0,
                                                host[S_XI], host[S_EPS], k ? host[S_V] : 1.0,
                                                (double)(trials_total - trials_prev), host[S_ETA]};
            c->hist.insert(c->hist.end(), row, row + TPCG_HIST_COLS);
            trials_prev = trials_total;
        }
        if (flags[0] || flags[1]) {
            set_error(std::string("tpcg_solve: an unrounded ") + (flags[0] ? "operator product" : "preconditioner output") +
                      " exceeded the context's max_cols or the block limit");
            status = TPCG_E_INVALID;
            break;
        }
        if (trace) {
            int rx[3], rr[3], rz[3], rp[3], rq[3], nb;
            tucker_get_ranks(x, rx, &nb, s);
            tucker_get_ranks(r, rr, &nb, s);
            tucker_get_ranks(z, rz, &nb, s);
            tucker_get_ranks(p, rp, &nb, s);
            tucker_get_ranks(q, rq, &nb, s);
            fprintf(stderr,
                    "tpcg k=%d res=%.3e eta=%.2e eps=%.2e v=%.4f omega=%.3e xi=%.3e trials=%d "
                    "rank x=(%d,%d,%d) r=(%d,%d,%d) z=(%d,%d,%d) p=(%d,%d,%d) q=(%d,%d,%d)\n",
                    k, host[S_NR] / host[S_NF], host[S_ETA], host[S_EPS], host[S_V], host[S_OMEGA], host[S_XI],
                    trials_total, rx[0], rx[1], rx[2], rr[0], rr[1], rr[2], rz[0], rz[1], rz[2], rp[0], rp[1], rp[2],
                    rq[0], rq[1], rq[2]);
        }
        if (host[S_BAD] != 0.0) { status = TPCG_E_BREAKDOWN; break; }
        if (host[S_STOP] != 0.0) break;
        if (k >= prm->max_it) { status = TPCG_E_NOT_CONVERGED; break; }
        // omega_k = r_k . p_k / xi_k
        TPCG_TRY(dot_cached<T>(c, r, p, sc + S_RP, s));
        launch_scalar(OP_OMEGA, sc, dprm, s);
        // dynamic truncation of x_k + omega_k p_k (Alg. 2)
        TPCG_TRY(dot_cached<T>(c, p, x, sc + S_PXK, s));
        TPCG_TRY(dot_cached<T>(c, p, p, sc + S_PP, s));
        TPCG_TRY(axpby_impl<T>(1.0, nullptr, x, 0.0, sc + S_OMEGA, p, big, nullptr, s));
        for (int trial = 0;; ++trial) {
            // below 1e-7 one FP64 Gram pass cannot resolve the budget: the resolved rule (two passes)
            bool resolved = false;
            if constexpr (sizeof(T) == 8)
                resolved = strict == 0 && resolved_kind() == 1 && eps_now < RESOLVE_BELOW &&
                           c->max_cols >= 3 * rc;
            if (resolved) {
                if constexpr (sizeof(T) == 8)
                    TPCG_TRY(round_resolved(c, big, big2, 0.0, sc + S_EPS, rc, sc + S_ZN2, rsE, rsF, s));
            } else {
                TPCG_TRY(copy_tensor_impl<T>(big, big2, c->n, c->max_cols, s));
                TPCG_TRY(round_cached<T>(c, big2, sc + S_EPS, rc, s, strict));
            }
            TPCG_TRY(dot_cached<T>(c, p, big2, sc + S_PXN, s));
            launch_scalar(OP_DT, sc, dprm, s);
            ++trials_total;
            double done;
            TPCG_TRY(fetch(c, s, {{&done, sc + S_DONE, sizeof(double)}, {&eps_now, sc + S_EPS, sizeof(double)}}));
            if (done != 0.0 || trial > 64) break;
        }
        std::swap(x, big2);
        // r_{k+1} = T(f - A x_{k+1}, eta_k); eta_{k+1}
        TPCG_TRY(apply_impl<T>(pb, x, big, true, s, rhs, apply_err));
        TPCG_TRY(round_to(r, eta));
        TPCG_TRY(dot_cached<T>(c, r, r, sc + S_RR, s));
        launch_scalar(OP_RES, sc, dprm, s);
        // z_{k+1} = T(P^-1 r_{k+1}, eta_{k+1});  beta_k = -z_{k+1} . q_k / xi_k
        TPCG_TRY(fd_impl<T>(pb, c, r, big, s));
        TPCG_TRY(round_to(z, eta));
        TPCG_TRY(dot_cached<T>(c, z, q, sc + S_ZQ, s));
        launch_scalar(OP_BETA, sc, dprm, s);
        // p_{k+1} = T(z_{k+1} + beta_k p_k, eta_{k+1})
        TPCG_TRY(axpby_impl<T>(1.0, nullptr, z, 0.0, sc + S_BETA, p, big, nullptr, s));
        TPCG_TRY(round_to(p, eta));
        // q_{k+1} = T(A p_{k+1}, eta_{k+1});  xi_{k+1} = p_{k+1} . q_{k+1}
        TPCG_TRY(apply_impl<T>(pb, p, big, false, s, nullptr, apply_err));
        TPCG_TRY(round_to(q, eta));
        TPCG_TRY(dot_cached<T>(c, p, q, sc + S_XI, s));
        launch_scalar(OP_XI, sc, dprm, s);
        ++k;
    }
    // copy x into the caller's tensor; measure its true residual (the problem's own rhs only)
    TPCG_TRY(copy_tensor_impl<T>(x, xout, c->n, xout->cap, s));
    double true_rel = -1.0;
    if (rhs == &pb->f) TPCG_TRY(true_residual<T>(pb, c, x, big, &true_rel, s));
    // (the internal tensors all have the same capacities, so their roles need no restoring)
    int rk[3] = {0, 0, 0};
    int nb = 0;
    TPCG_TRY(fetch(c, s, {{host, sc, sizeof(host)}}));
    TPCG_TRY(tucker_get_ranks(xout, rk, &nb, s));
    if (st) {
        st->iters = k;
        st->status = status;
        st->rel_res = host[S_NF] > 0 ? host[S_NR] / host[S_NF] : 0.0;
        for (int t = 0; t < 3; ++t) st->rank[t] = rk[t];
        const double n = c->n;
        st->mem_compression = ((double)rk[0] * rk[1] * rk[2] + n * (rk[0] + rk[1] + rk[2])) / (n * n * n) * 100.0;
        st->dt_trials = trials_total;
        st->max_rank_seen = std::max(rk[0], std::max(rk[1], rk[2]));
        st->outer_iters = 0;
        st->true_rel_res = true_rel;
    }
    return status;
}

// truncation tolerance of x + d in the mixed form: the correction d is kept to relative accuracy `keep`,
// eps = keep ||d|| / ||x + d|| (x and d plain)
__global__ void xeps_kernel(const double* dd, const double* xx, double keep, double* eps) {
    const double d = fmax(*dd, 0.0), x = fmax(*xx, 0.0);
    *eps = (d + x > 0.0) ? keep * sqrt(d / (d + x)) : 0.0;
}

// Mixed form: iterative refinement with FP64 residuals around FP32 Alg. 5 (see tpcg.h).  The outer loop
// carries the relaxation of Alg. 5 over to the refinement: the FP32 copy of the residual may lose
// beta tol ||f~|| / 2 in absolute terms, and the inner solve stops at the reduction the outer target needs.
// x stays plain: after each correction x <- T_rel(x + d, keep ||d|| / ||x + d||) in FP64, so every residual
// (and the stopping test) refers to the tensor that is returned.
static int solve_mixed(tpcg_problem pb, tpcg_ctx c, const tpcg_params* prm, tucker_t* xout, tpcg_stats* st,
                       cudaStream_t s) {
    tpcg_problem pb32 = pb->lo;
    tpcg_ctx c32 = c->lo;
    TPCG_TRY(ensure_tensors(c, 10));
    TPCG_TRY(ensure_tensors(c32, 10));
    const int rc = (prm->rank_cap > 0 && prm->rank_cap < c->rank_cap) ? prm->rank_cap : c->rank_cap;
    tucker_t* xacc = &c->tens[0];
    tucker_t* xsum = &c->tens[1];
    tucker_t* big = &c->tens[2];
    tucker_t* dco = &c->tens[3];
    tucker_t* r32 = &c32->tens[8];
    tucker_t* d32 = &c32->tens[9];
    const int max_outer = std::min(std::max(prm->max_outer, 1), 64);
    const double nf = pb->norm_f;
    const double abs_tol = 0.5 * prm->beta_trunc * prm->tol * nf;
    double* info = c->scal + 120;   // 6 doubles written by the rounding
    double* dd = c->scal + 140;
    double* xx = c->scal + 141;
    double* xeps = c->scal + 142;
    int* apply_err = reinterpret_cast<int*>(c->scal + 232);   // capacity flag of the FP64 residual (this context)
    TPCG_CUDA(cudaMemsetAsync(apply_err, 0, sizeof(int), s));
    const char* tr = getenv("TPCG_TRACE");
    const bool trace = tr && tr[0] == '1';
    TPCG_TRY(set_zero(xacc, s));
    tpcg_params in = *prm;
    in.rank_cap = rc;
    in.max_it = std::min(prm->max_it, 12);
    int status = TPCG_E_NOT_CONVERGED, outer = 0, inner_total = 0, trials = 0;
    double rel = 1.0;
    for (outer = 0; outer <= max_outer; ++outer) {
        // r = f - A x in FP64 (exact ||r|| from Z), truncated to 0.1 inner_tol (relative) or abs_tol in FP32
        TPCG_TRY(apply_impl<double>(pb, xacc, big, true, s, nullptr, apply_err));
        TPCG_TRY(round_mixed(c, c32, big, r32, 0.1 * prm->inner_tol, nullptr, rc, abs_tol, info, s));
        double h[6];
        int over = 0;
        TPCG_TRY(fetch(c, s, {{h, info, sizeof(h)}, {&over, apply_err, sizeof(int)}}));
        if (over) {
            set_error("tpcg_solve: the FP64 residual exceeded the context's max_cols or the block limit");
            status = TPCG_E_INVALID;
            break;
        }
        rel = nf > 0 ? sqrt(std::max(h[0], 0.0)) / nf : 0.0;
        if (trace) fprintf(stderr, "mixed outer=%d true_res=%.3e r-rank=(%g,%g,%g)\n", outer, rel, h[2], h[3], h[4]);
        if (!(rel == rel)) { status = TPCG_E_BREAKDOWN; break; }
        if (rel <= prm->tol) { status = TPCG_OK; break; }
        if (outer == max_outer) break;
        // inner tolerance: inner_tol, or the (looser) reduction that reaches tol from the current residual
        in.tol = std::min(0.5, std::max(prm->inner_tol, 0.5 * prm->tol / rel));
        in.eps_min = 0.1 * in.tol;
        tpcg_stats sin{};
        int si = solve_impl<float>(pb32, c32, &in, d32, &sin, s, r32);
        inner_total += sin.iters;
        trials += sin.dt_trials;
        if (trace) fprintf(stderr, "mixed inner tol=%.2e iters=%d status=%d\n", in.tol, sin.iters, si);
        if (si == TPCG_E_BREAKDOWN) {
            // the FP32 curvature p.q lost its sign (truncation noise at FP32 resolution): take this correction
            // from Alg. 5 in FP64 instead, on the FP64 residual truncated in FP64 (tensors 10..16 of the context)
            TPCG_TRY(round_impl<double>(c, big, 0.1 * prm->inner_tol, nullptr, rc, nullptr, s));
            tpcg_stats s64{};
            si = solve_impl<double>(pb, c, &in, dco, &s64, s, big, 10);
            inner_total += s64.iters;
            trials += s64.dt_trials;
            if (trace) fprintf(stderr, "mixed FP64 inner iters=%d status=%d\n", s64.iters, si);
            if (si != TPCG_OK && si != TPCG_E_NOT_CONVERGED) { status = si; break; }
        } else if (si != TPCG_OK && si != TPCG_E_NOT_CONVERGED) {
            status = si;
            break;
        } else {
            TPCG_TRY(promote_tensor(d32, dco, s));
        }
        // x <- T_rel(x + d, keep ||d|| / ||x + d||) in FP64
        TPCG_TRY(dot_impl<double>(c, dco, dco, dd, s));
        TPCG_TRY(dot_impl<double>(c, xacc, xacc, xx, s));
        xeps_kernel<<<1, 1, 0, s>>>(dd, xx, prm->refine_keep, xeps);
        TPCG_CHECK_LAUNCH();
        TPCG_TRY(axpby_impl<double>(1.0, nullptr, xacc, 1.0, nullptr, dco, xsum, nullptr, s));
        // keep ||d|| to relative accuracy refine_keep: its FP32 rounding noise is meant to be dropped (no strict
        // rule).  Once keep ||d|| / ||x + d|| is below what one FP64 Gram resolves, the resolved rule keeps d to
        // that accuracy instead of losing it in the Gram's rounding
        double dx[2];
        TPCG_TRY(fetch(c, s, {{dx, dd, 2 * sizeof(double)}}));
        const double d2 = std::max(dx[0], 0.0), x2 = std::max(dx[1], 0.0);
        const double xeps_host = d2 + x2 > 0.0 ? prm->refine_keep * sqrt(d2 / (d2 + x2)) : 0.0;
        if (resolved_kind() == 1 && xeps_host < RESOLVE_BELOW && c->max_cols >= 3 * rc) {
            TPCG_TRY(round_resolved(c, xsum, big, 0.0, xeps, rc, c->scal + 143, &c->tens[4], &c->tens[5], s));
            std::swap(xacc, big);
        } else {
            TPCG_TRY(round_impl<double>(c, xsum, 0.0, xeps, rc, nullptr, s, 0));
            std::swap(xacc, xsum);
        }
    }
    TPCG_TRY(copy_tensor_impl<double>(xacc, xout, c->n, xout->cap, s));
    int rk[3] = {0, 0, 0}, nb = 0;
    TPCG_TRY(tucker_get_ranks(xout, rk, &nb, s));
    if (st) {
        st->iters = inner_total;
        st->status = status;
        st->rel_res = rel;
        st->true_rel_res = rel;   // the FP64 residual of exactly the returned x
        st->outer_iters = outer;
        for (int t = 0; t < 3; ++t) st->rank[t] = rk[t];
        const double n = c->n;
        st->mem_compression = ((double)rk[0] * rk[1] * rk[2] + n * (rk[0] + rk[1] + rk[2])) / (n * n * n) * 100.0;
        st->dt_trials = trials;
        st->max_rank_seen = std::max(rk[0], std::max(rk[1], rk[2]));
    }
    return status;
}

extern "C" int tpcg_solve(tpcg_problem pb, tpcg_ctx c, const tpcg_params* prm, tucker_t* x, tpcg_stats* st,
                          void* stream) {
    if (!pb || !c || !prm || pb->n != c->n || pb->dtype != c->dtype || prm->tol <= 0 || prm->alpha <= 0 ||
        prm->alpha >= 1 || prm->max_it < 0) {
        set_error("tpcg_solve: invalid arguments");
        return TPCG_E_INVALID;
    }
    TPCG_TRY(check_tensor(x, pb->n, pb->dtype, "tpcg_solve x"));
    if (pb->lo || c->lo) {
        if (!pb->lo || !c->lo || pb->lo->n != c->lo->n) {
            set_error("tpcg_solve: the mixed form needs a TPCG_MIXED problem and a TPCG_MIXED context");
            return TPCG_E_INVALID;
        }
    }
    const int rfmax = std::max(pb->rf[0], std::max(pb->rf[1], pb->rf[2]));
    // residuals hold rhs columns + R rank_cap; in the mixed form the inner rhs is a residual of rank <= rank_cap
    const int rhs_cols = pb->lo ? std::max(rfmax, c->rank_cap) : rfmax;
    const int need = std::max(pb->R * c->rank_cap + rhs_cols, std::max(pb->RP * c->rank_cap, 2 * c->rank_cap));
    if (c->max_cols < need) {
        set_error("tpcg_solve: context max_cols " + std::to_string(c->max_cols) + " < required " +
                  std::to_string(need));
        return TPCG_E_INVALID;
    }
    if (pb->lo) return solve_mixed(pb, c, prm, x, st, S(stream));
    return by_dtype(pb->dtype, [&](auto z) { return solve_impl<decltype(z)>(pb, c, prm, x, st, S(stream)); });
}

extern "C" int tpcg_ctx_history(tpcg_ctx c, double* out, int max_rows, int* rows) {
    if (!c || !rows || max_rows < 0 || (max_rows > 0 && !out)) {
        set_error("tpcg_ctx_history: invalid arguments");
        return TPCG_E_INVALID;
    }
    const int have = (int)(c->hist.size() / TPCG_HIST_COLS);
    *rows = have;
    const int m = std::min(have, max_rows);
    if (m > 0) memcpy(out, c->hist.data(), (size_t)m * TPCG_HIST_COLS * sizeof(double));
    return TPCG_OK;
}

// Many independent solves at once: one host thread per solve, each on its own stream and context, so
// that their kernels overlap on the device (the eigensolver and QR kernels of one solve fill one SM each).
extern "C" int tpcg_ctx_stream(tpcg_ctx c, void** out) {
    if (!c || !out) return TPCG_E_INVALID;
    if (!c->own_stream && cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        c->own_stream = nullptr;
        cudaGetLastError();
        set_error("tpcg_ctx_stream: cudaStreamCreateWithFlags failed");
        return TPCG_E_CUDA;
    }
    *out = c->own_stream;
    return TPCG_OK;
}

extern "C" int tpcg_solve_batch(int count, const tpcg_problem* pbs, const tpcg_ctx* ctxs, const tpcg_params* prms,
                                tucker_t* xs, tpcg_stats* sts, void* const* streams, int* statuses) {
    if (count < 0 || (count > 0 && (!pbs || !ctxs || !prms || !xs || !streams || !statuses))) {
        set_error("tpcg_solve_batch: invalid arguments");
        return TPCG_E_INVALID;
    }
    for (int i = 0; i < count; ++i)
        for (int j = 0; j < i; ++j)
            if (ctxs[i] == ctxs[j] || (streams[i] && streams[i] == streams[j])) {
                set_error("tpcg_solve_batch: every solve needs its own context and its own stream (or NULL)");
                return TPCG_E_INVALID;
            }
    int dev = 0;
    TPCG_CUDA(cudaGetDevice(&dev));
    std::vector<std::thread> th;
    std::vector<std::string> errs(count);
    th.reserve(count);
    for (int i = 0; i < count; ++i) {
        th.emplace_back([&, i]() {
            if (cudaSetDevice(dev) != cudaSuccess) {
                statuses[i] = TPCG_E_CUDA;
                errs[i] = "cudaSetDevice failed in a solver thread";
                return;
            }
            // a NULL stream entry: the solve runs on its context's own stream (created once, kept with the
            // context so that its captured graphs keep launching on the same stream)
            if (!streams[i] && !ctxs[i]->own_stream &&
                cudaStreamCreateWithFlags(&ctxs[i]->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
                ctxs[i]->own_stream = nullptr;
                statuses[i] = TPCG_E_CUDA;
                errs[i] = "cudaStreamCreateWithFlags failed in a solver thread";
                return;
            }
            cudaStream_t st = streams[i] ? static_cast<cudaStream_t>(streams[i]) : ctxs[i]->own_stream;
            statuses[i] = tpcg_solve(pbs[i], ctxs[i], &prms[i], &xs[i], sts ? &sts[i] : nullptr, st);
            if (statuses[i] != TPCG_OK) errs[i] = tpcg_last_error();
            cudaStreamSynchronize(st);
        });
    }
    for (auto& t : th) t.join();
    for (int i = 0; i < count; ++i)
        if (statuses[i] != TPCG_OK && statuses[i] != TPCG_E_NOT_CONVERGED) {
            set_error("tpcg_solve_batch: solve " + std::to_string(i) + ": " + errs[i]);
            return statuses[i];
        }
    for (int i = 0; i < count; ++i)
        if (statuses[i] != TPCG_OK) return statuses[i];
    return TPCG_OK;
}
