// Tucker operations other than rounding: Kronecker-sum matvec (eq. tt_product) as a banded SpMM on the
// factors, Tucker sums (Sec. 2.3), scalar products (Sec. 2.3), the low-rank FD application (Alg. 4,
// App. B) and tensor copies.  Shapes come from the device descriptors.
#include <math.h>

#include <mutex>
#include <string>

#include "common.cuh"
#include "gemm.cuh"
#include "kernels.cuh"

namespace tpcg {

// --------------------------------------------------------------------------------------------------
// descriptors
// --------------------------------------------------------------------------------------------------
__global__ void set_plain_kernel(TuckerDesc* d, int r1, int r2, int r3, const void* core) {
    if (threadIdx.x != 0) return;
    d->nblk = 1;
    d->rank[0] = r1; d->rank[1] = r2; d->rank[2] = r3;
    d->blk[0].off[0] = d->blk[0].off[1] = d->blk[0].off[2] = 0;
    d->blk[0].r[0] = r1; d->blk[0].r[1] = r2; d->blk[0].r[2] = r3;
    d->blk[0].core = core;
    d->blk[0].scale = 1.0;
}

int set_plain(tucker_t* t, int r1, int r2, int r3, cudaStream_t st) {
    set_plain_kernel<<<1, 32, 0, st>>>(static_cast<TuckerDesc*>(t->desc), r1, r2, r3, t->core);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}

int set_zero(tucker_t* t, cudaStream_t st) { return set_plain(t, 0, 0, 0, st); }

// --------------------------------------------------------------------------------------------------
// y = A x  /  y = f - A x  (eq. tt_product): Y_t[:, base_t + j k_t + c] = K_t^j X_t[:, c];
// bands[((j*3 + t)*(2p+1) + d)*n + i] = K_t^j[i, i + d - p].  The extra "term" j = R copies F_t into the
// first columns for the residual.
// Grid: x = 128-row tiles, y = (term, chunk of APPLY_CB input columns), z = mode; a thread owns one row and
// keeps its 2p+1 band entries in registers across its chunk's columns (rows of X are reused from L1 by the
// neighbouring lanes).  Enough CTAs for the SMs at n = 512 (4 x 20 x 10 x 3 at k = 80, R = 19).
// --------------------------------------------------------------------------------------------------
constexpr int APPLY_CB = 8;

// output descriptor of the apply: blocks (f) + (j, b) for every term j and input block b
__device__ void apply_desc(const TuckerDesc* __restrict__ xd, const double* __restrict__ w, int R, double sign,
                           const TuckerDesc* fdsc, TuckerDesc* yd, int cap, int* err, double* prof, int n, int p,
                           int elt) {
    if (prof) {   // algorithmic work of the banded products: bands read once, X read, Y written
        double cols = (double)xd->rank[0] + xd->rank[1] + xd->rank[2];
        prof[2 * PK_APPLY] += 2.0 * (2 * p + 1) * (double)n * R * cols;
        prof[2 * PK_APPLY + 1] += (double)elt * ((double)R * 3 * (2 * p + 1) * n + (double)n * cols * (1.0 + R));
    }
    int nb = 0;
    int base[3] = {0, 0, 0};
    if (fdsc) {   // leading blocks: the rhs (residual) or y itself (append; fdsc == yd, nothing to copy)
        for (int t = 0; t < 3; ++t) base[t] = fdsc->rank[t];
        if (fdsc == yd)
            nb = fdsc->nblk;
        else
            for (int b = 0; b < fdsc->nblk; ++b) yd->blk[nb++] = fdsc->blk[b];
    }
    const int kx[3] = {xd->rank[0], xd->rank[1], xd->rank[2]};
    bool ok = (nb + R * xd->nblk <= TPCG_MAX_BLOCKS);
    for (int t = 0; t < 3; ++t) ok = ok && (base[t] + (long long)R * kx[t] <= cap);
    if (!ok) {
        if (err) *err = 1;
        yd->nblk = 0;
        yd->rank[0] = yd->rank[1] = yd->rank[2] = 0;
        return;
    }
    for (int j = 0; j < R; ++j)
        for (int b = 0; b < xd->nblk; ++b) {
            BlockDesc B = xd->blk[b];
            for (int t = 0; t < 3; ++t) B.off[t] += base[t] + j * kx[t];
            B.scale *= sign * w[j];
            yd->blk[nb++] = B;
        }
    yd->nblk = nb;
    for (int t = 0; t < 3; ++t) yd->rank[t] = base[t] + R * kx[t];
}

// yd: when non-null, block (0, 0, 0) also writes the output descriptor (only when yd is not read by this kernel,
// i.e. not for appends).  P (the degree) is a template parameter: the 2P+1 taps are unrolled, and row tiles
// that touch neither end of the band (all but the first and last) run without bounds checks.
template <typename T, int P>
__global__ void __launch_bounds__(128) apply_kernel(const T* __restrict__ bands, int n, int R, int nchunk,
                                                    const TuckerDesc* __restrict__ xd, const T* X0, const T* X1,
                                                    const T* X2, T* Y0, T* Y1, T* Y2, int cap,
                                                    const TuckerDesc* __restrict__ fd, const T* F0, const T* F1,
                                                    const T* F2, TuckerDesc* yd, const double* __restrict__ w,
                                                    double sign, int* err, double* prof) {
    constexpr int BW = 2 * P + 1;
    if (yd && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
        apply_desc(xd, w, R, sign, fd, yd, cap, err, prof, n, P, (int)sizeof(T));
    const int t = blockIdx.z, j = blockIdx.y / nchunk, chunk = blockIdx.y % nchunk;
    const int i0 = blockIdx.x * blockDim.x;
    const int i = i0 + threadIdx.x;
    const T* X = t == 0 ? X0 : (t == 1 ? X1 : X2);
    T* Y = t == 0 ? Y0 : (t == 1 ? Y1 : Y2);
    const int kx = xd->rank[t];
    const int base = fd ? fd->rank[t] : 0;
    const int c0 = chunk * APPLY_CB;
    if (j == R) {   // copy the rhs factor
        if (base > cap || i >= n) return;
        const T* F = t == 0 ? F0 : (t == 1 ? F1 : F2);
        for (int c = c0; c < base; c += nchunk * APPLY_CB)
            for (int q = c; q < c + APPLY_CB && q < base; ++q) Y[i + (long long)q * n] = F[i + (long long)q * n];
        return;
    }
    if (base + (long long)R * kx > cap) return;   // capacity violated: flagged by the descriptor
    if (c0 >= kx || i >= n) return;
    T band[BW];
    const T* bj = bands + ((long long)(j * 3 + t) * BW) * n;
#pragma unroll
    for (int d = 0; d < BW; ++d) band[d] = __ldg(bj + (long long)d * n + i);
    const bool interior = i0 >= P && i0 + (int)blockDim.x + P <= n;   // uniform over the block
    const long long col0 = base + (long long)j * kx;
    // columns c0, c0 + nchunk CB, ... (chunks stride over the columns when kx exceeds nchunk CB)
    for (int cb = c0; cb < kx; cb += nchunk * APPLY_CB) {
        const T* xr = X + (long long)cb * n + i - P;   // tap d of column cb + q at xr[d + q n]
        T* yr = Y + (col0 + cb) * n + i;
        if (interior && cb + APPLY_CB <= kx) {      // full chunk, no bounds: all loads in flight together
            T acc[APPLY_CB];
#pragma unroll
            for (int q = 0; q < APPLY_CB; ++q) {
                acc[q] = T(0);
#pragma unroll
                for (int d = 0; d < BW; ++d) acc[q] = fma(band[d], __ldg(xr + d + (long long)q * n), acc[q]);
            }
#pragma unroll
            for (int q = 0; q < APPLY_CB; ++q) yr[(long long)q * n] = acc[q];
        } else {
            for (int q = 0; q < APPLY_CB && cb + q < kx; ++q) {
                T acc = T(0);
#pragma unroll
                for (int d = 0; d < BW; ++d) {
                    const int ii = i + d - P;
                    if (ii >= 0 && ii < n) acc = fma(band[d], xr[d + (long long)q * n], acc);
                }
                yr[(long long)q * n] = acc;
            }
        }
    }
}

template <typename T>
static int launch_apply(int p, dim3 grid, cudaStream_t st, const T* bands, int n, int R, int nchunk,
                        const TuckerDesc* xd, const T* X0, const T* X1, const T* X2, T* Y0, T* Y1, T* Y2, int cap,
                        const TuckerDesc* fd, const T* F0, const T* F1, const T* F2, TuckerDesc* yd, const double* w,
                        double sign, int* err, double* prof) {
#define TPCG_APPLY_P(PP)                                                                                           \
    apply_kernel<T, PP><<<grid, 128, 0, st>>>(bands, n, R, nchunk, xd, X0, X1, X2, Y0, Y1, Y2, cap, fd, F0, F1, F2, \
                                              yd, w, sign, err, prof)
    switch (p) {
        case 1: TPCG_APPLY_P(1); break;
        case 2: TPCG_APPLY_P(2); break;
        case 3: TPCG_APPLY_P(3); break;
        case 4: TPCG_APPLY_P(4); break;
        case 5: TPCG_APPLY_P(5); break;
        default:
            set_error("apply: degree out of range (1..5)");
            return TPCG_E_INVALID;
    }
#undef TPCG_APPLY_P
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}

__global__ void apply_desc_kernel(const TuckerDesc* __restrict__ xd, const double* __restrict__ w, int R,
                                  double sign, const TuckerDesc* fdsc, TuckerDesc* yd, int cap,
                                  int* err, double* prof, int n, int p, int elt) {
    if (threadIdx.x != 0) return;
    apply_desc(xd, w, R, sign, fdsc, yd, cap, err, prof, n, p, elt);
}

// column chunks per term: enough to cover the largest input rank a y of this capacity can take (cap / R)
static inline int apply_chunks(int cap, int R) {
    const int kmax = std::max(1, cap / std::max(R, 1));
    return std::min(64, (kmax + APPLY_CB - 1) / APPLY_CB);
}

template <typename T>
int apply_impl(tpcg_problem pb, const tucker_t* x, tucker_t* y, bool residual, cudaStream_t st, const tucker_t* rhs,
               int* err) {
    const int n = pb->n;
    if (!err) err = reinterpret_cast<int*>(pb->d_scal + 60);
    const int nchunk = apply_chunks(y->cap, pb->R);
    dim3 grid((n + 127) / 128, (pb->R + (residual ? 1 : 0)) * nchunk, 3);
    const tucker_t* f = rhs ? rhs : &pb->f;
    prof_begin(PK_APPLY, st);
    TPCG_TRY(launch_apply<T>(pb->p, grid, st, static_cast<const T*>(pb->d_bands), n, pb->R, nchunk,
                             static_cast<const TuckerDesc*>(x->desc), static_cast<const T*>(x->U[0]),
                             static_cast<const T*>(x->U[1]), static_cast<const T*>(x->U[2]), static_cast<T*>(y->U[0]),
                             static_cast<T*>(y->U[1]), static_cast<T*>(y->U[2]), y->cap,
                             residual ? static_cast<const TuckerDesc*>(f->desc) : nullptr,
                             static_cast<const T*>(f->U[0]), static_cast<const T*>(f->U[1]),
                             static_cast<const T*>(f->U[2]), static_cast<TuckerDesc*>(y->desc), pb->d_w,
                             residual ? -1.0 : 1.0, err, prof_dev()));
    prof_end(PK_APPLY, st);
    return TPCG_OK;
}
// y <- y + sign A x: the R new blocks and their factor columns are appended after y's own (block sums of
// operators, e.g. y_i = sum_j A_ij x_j of the elasticity system)
template <typename T>
int apply_append_impl(tpcg_problem pb, const tucker_t* x, tucker_t* y, double sign, cudaStream_t st, int* err) {
    const int n = pb->n;
    if (!err) err = reinterpret_cast<int*>(pb->d_scal + 60);
    const int nchunk = apply_chunks(y->cap, pb->R);
    dim3 grid((n + 127) / 128, pb->R * nchunk, 3);
    prof_begin(PK_APPLY, st);
    // y's descriptor is read by every block (its old ranks are the column base): it is updated afterwards
    TPCG_TRY(launch_apply<T>(pb->p, grid, st, static_cast<const T*>(pb->d_bands), n, pb->R, nchunk,
                             static_cast<const TuckerDesc*>(x->desc), static_cast<const T*>(x->U[0]),
                             static_cast<const T*>(x->U[1]), static_cast<const T*>(x->U[2]), static_cast<T*>(y->U[0]),
                             static_cast<T*>(y->U[1]), static_cast<T*>(y->U[2]), y->cap,
                             static_cast<const TuckerDesc*>(y->desc), nullptr, nullptr, nullptr, nullptr, nullptr,
                             0.0, nullptr, nullptr));
    apply_desc_kernel<<<1, 32, 0, st>>>(static_cast<const TuckerDesc*>(x->desc), pb->d_w, pb->R, sign,
                                        static_cast<const TuckerDesc*>(y->desc), static_cast<TuckerDesc*>(y->desc),
                                        y->cap, err, prof_dev(), n, pb->p, (int)sizeof(T));
    TPCG_CHECK_LAUNCH();
    prof_end(PK_APPLY, st);
    return TPCG_OK;
}
template int apply_append_impl<double>(tpcg_problem, const tucker_t*, tucker_t*, double, cudaStream_t, int*);
template int apply_append_impl<float>(tpcg_problem, const tucker_t*, tucker_t*, double, cudaStream_t, int*);

template int apply_impl<double>(tpcg_problem, const tucker_t*, tucker_t*, bool, cudaStream_t, const tucker_t*, int*);
template int apply_impl<float>(tpcg_problem, const tucker_t*, tucker_t*, bool, cudaStream_t, const tucker_t*, int*);

// --------------------------------------------------------------------------------------------------
// z = a x + b y: concatenated factors, block lists shifted and scaled (Sec. 2.3, sum).
// --------------------------------------------------------------------------------------------------
template <typename T>
__global__ void concat_kernel(const TuckerDesc* __restrict__ xd, const T* X0, const T* X1, const T* X2,
                              const TuckerDesc* __restrict__ yd, const T* Y0, const T* Y1, const T* Y2, T* Z0,
                              T* Z1, T* Z2, int n, int cap) {
    const int t = blockIdx.z;
    const T* X = t == 0 ? X0 : (t == 1 ? X1 : X2);
    const T* Y = t == 0 ? Y0 : (t == 1 ? Y1 : Y2);
    T* Z = t == 0 ? Z0 : (t == 1 ? Z1 : Z2);
    const int kx = xd->rank[t], ky = yd->rank[t];
    if (kx + ky > cap) return;
    const long long tx = (long long)n * kx, ty = (long long)n * ky;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tx + ty;
         e += (long long)gridDim.x * blockDim.x)
        Z[e] = e < tx ? X[e] : Y[e - tx];
}

__global__ void axpby_desc_kernel(const TuckerDesc* __restrict__ xd, double a, const double* a_dev,
                                  const TuckerDesc* __restrict__ yd, double b, const double* b_dev, TuckerDesc* zd,
                                  int cap, int* err) {
    if (threadIdx.x != 0) return;
    const double av = a_dev ? *a_dev : a;
    const double bv = b_dev ? *b_dev : b;
    bool ok = xd->nblk + yd->nblk <= TPCG_MAX_BLOCKS;
    for (int t = 0; t < 3; ++t) ok = ok && (xd->rank[t] + yd->rank[t] <= cap);
    if (!ok) {
        if (err) *err = 1;
        zd->nblk = 0;
        zd->rank[0] = zd->rank[1] = zd->rank[2] = 0;
        return;
    }
    int nb = 0;
    for (int i = 0; i < xd->nblk; ++i) {
        BlockDesc B = xd->blk[i];
        B.scale *= av;
        zd->blk[nb++] = B;
    }
    for (int i = 0; i < yd->nblk; ++i) {
        BlockDesc B = yd->blk[i];
        for (int t = 0; t < 3; ++t) B.off[t] += xd->rank[t];
        B.scale *= bv;
        zd->blk[nb++] = B;
    }
    zd->nblk = nb;
    for (int t = 0; t < 3; ++t) zd->rank[t] = xd->rank[t] + yd->rank[t];
}

template <typename T>
int axpby_impl(double a, const double* a_dev, const tucker_t* x, double b, const double* b_dev, const tucker_t* y,
               tucker_t* z, int* err_dev, cudaStream_t st) {
    const int n = z->n;
    dim3 grid(64, 1, 3);
    concat_kernel<T><<<grid, 256, 0, st>>>(static_cast<const TuckerDesc*>(x->desc), static_cast<const T*>(x->U[0]),
                                           static_cast<const T*>(x->U[1]), static_cast<const T*>(x->U[2]),
                                           static_cast<const TuckerDesc*>(y->desc), static_cast<const T*>(y->U[0]),
                                           static_cast<const T*>(y->U[1]), static_cast<const T*>(y->U[2]),
                                           static_cast<T*>(z->U[0]), static_cast<T*>(z->U[1]),
                                           static_cast<T*>(z->U[2]), n, z->cap);
    TPCG_CHECK_LAUNCH();
    axpby_desc_kernel<<<1, 32, 0, st>>>(static_cast<const TuckerDesc*>(x->desc), a, a_dev,
                                        static_cast<const TuckerDesc*>(y->desc), b, b_dev,
                                        static_cast<TuckerDesc*>(z->desc), z->cap, err_dev);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}
template int axpby_impl<double>(double, const double*, const tucker_t*, double, const double*, const tucker_t*,
                                tucker_t*, int*, cudaStream_t);
template int axpby_impl<float>(double, const double*, const tucker_t*, double, const double*, const tucker_t*,
                               tucker_t*, int*, cudaStream_t);

// --------------------------------------------------------------------------------------------------
// <x, y> = vec(G_x)^T vec(G_y x_1 W_1 x_2 W_2 x_3 W_3), W_t = X_t^T Y_t (Sec. 2.3), both plain.
// ctx scratch: dotw (3 W_t, rank_cap^2 each, as T), dotT (two rank_cap^3 buffers).
// gargs slots used: [0..2] W_t, [3] mode 1, [4] mode 2, [5] mode 3.
// --------------------------------------------------------------------------------------------------
template <typename T>
__global__ void plan_dot_kernel(const TuckerDesc* __restrict__ xd, const T* X0, const T* X1, const T* X2,
                                const TuckerDesc* __restrict__ yd, const T* Y0, const T* Y1, const T* Y2, int n,
                                int rc, T* Wb, T* Ta, T* Tb, GemmArgs* ga, int* counts) {
    if (threadIdx.x != 0) return;
    const T* X[3] = {X0, X1, X2};
    const T* Y[3] = {Y0, Y1, Y2};
    int r[3], s[3];
    bool bad = xd->nblk != 1 || yd->nblk != 1;
    for (int t = 0; t < 3; ++t) {
        r[t] = xd->rank[t];
        s[t] = yd->rank[t];
        bad = bad || r[t] > rc || s[t] > rc;
    }
    counts[1] = bad ? 1 : 0;
    if (bad)
        for (int t = 0; t < 3; ++t) r[t] = s[t] = 0;
    const long long rc2 = (long long)rc * rc;
    for (int t = 0; t < 3; ++t) {
        GemmArgs a{};
        a.M = r[t]; a.N = s[t]; a.K = n; a.nbatch = 1; a.acc = 0; a.alpha = 1.0; a.beta = 0.0;
        a.A = X[t]; a.lda = n; a.B = Y[t]; a.ldb = n; a.C = Wb + t * rc2; a.ldc = r[t] > 0 ? r[t] : 1;
        ga[t] = a;
    }
    const void* Gy = yd->blk[0].core;
    // mode 1: Ta (r1 x s2 s3) = W_1 (r1 x s1) G_y(1)
    GemmArgs m1{};
    m1.M = r[0]; m1.N = s[1] * s[2]; m1.K = s[0]; m1.nbatch = 1; m1.alpha = yd->blk[0].scale; m1.beta = 0.0;
    m1.A = Wb; m1.lda = r[0] > 0 ? r[0] : 1; m1.B = Gy; m1.ldb = s[0] > 0 ? s[0] : 1; m1.C = Ta; m1.ldc = m1.lda;
    ga[3] = m1;
    // mode 2 per slice i3: Tb[:, :, i3] (r1 x r2) = Ta[:, :, i3] (r1 x s2) W_2^T
    GemmArgs m2{};
    m2.M = r[0]; m2.N = r[1]; m2.K = s[1]; m2.nbatch = s[2]; m2.alpha = 1.0; m2.beta = 0.0;
    m2.A = Ta; m2.lda = m1.lda; m2.sA = (long long)r[0] * s[1];
    m2.B = Wb + rc2; m2.ldb = r[1] > 0 ? r[1] : 1;
    m2.C = Tb; m2.ldc = m1.lda; m2.sC = (long long)r[0] * r[1];
    ga[4] = m2;
    // mode 3: Ta (r1 r2 x r3) = Tb (r1 r2 x s3) W_3^T
    GemmArgs m3{};
    m3.M = r[0] * r[1]; m3.N = r[2]; m3.K = s[2]; m3.nbatch = 1; m3.alpha = 1.0; m3.beta = 0.0;
    m3.A = Tb; m3.lda = m3.M > 0 ? m3.M : 1; m3.B = Wb + 2 * rc2; m3.ldb = r[2] > 0 ? r[2] : 1;
    m3.C = Ta; m3.ldc = m3.lda;
    ga[5] = m3;
    counts[0] = 3;
}

template <typename T>
__global__ void dot_finish_kernel(const TuckerDesc* __restrict__ xd, const T* Ta, double* out, const int* bad) {
    __shared__ double red[32];
    if (*bad) {
        if (threadIdx.x == 0) *out = nan("");
        return;
    }
    const long long tot = (long long)xd->rank[0] * xd->rank[1] * xd->rank[2];
    const T* Gx = static_cast<const T*>(xd->blk[0].core);
    double s = 0.0;
    for (long long e = threadIdx.x; e < tot; e += blockDim.x) s += (double)Gx[e] * (double)Ta[e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        *out = v * xd->blk[0].scale;
    }
}

template <typename T>
int dot_impl(tpcg_ctx c, const tucker_t* x, const tucker_t* y, double* out_dev, cudaStream_t st) {
    const int n = c->n, rc = c->rank_cap;
    GemmArgs* ga = c->gargs + 2 * TPCG_MAX_BLOCKS + 8;   // disjoint from the rounding slots
    int* counts = reinterpret_cast<int*>(c->scal + 210);
    T* Wb = reinterpret_cast<T*>(c->dotw);
    T* Ta = static_cast<T*>(c->dotT);
    T* Tb = Ta + (long long)rc * rc * rc;
    prof_begin(PK_DOT, st);
    plan_dot_kernel<T><<<1, 32, 0, st>>>(static_cast<const TuckerDesc*>(x->desc), static_cast<const T*>(x->U[0]),
                                         static_cast<const T*>(x->U[1]), static_cast<const T*>(x->U[2]),
                                         static_cast<const TuckerDesc*>(y->desc), static_cast<const T*>(y->U[0]),
                                         static_cast<const T*>(y->U[1]), static_cast<const T*>(y->U[2]), n, rc, Wb,
                                         Ta, Tb, ga, counts);
    TPCG_CHECK_LAUNCH();
    TPCG_TRY((launch_gemm<T, true, false>(ga, counts, 3, 1, rc, rc, st)));
    TPCG_TRY((launch_gemm<T, false, false>(ga + 3, nullptr, 1, 1, rc, rc * rc, st)));
    TPCG_TRY((launch_gemm<T, false, true>(ga + 4, nullptr, 1, rc, rc, rc, st)));
    TPCG_TRY((launch_gemm<T, false, true>(ga + 5, nullptr, 1, 1, rc * rc, rc, st)));
    dot_finish_kernel<T><<<1, 1024, 0, st>>>(static_cast<const TuckerDesc*>(x->desc), Ta, out_dev, counts + 1);
    TPCG_CHECK_LAUNCH();
    prof_end(PK_DOT, st);
    return TPCG_OK;
}
template int dot_impl<double>(tpcg_ctx, const tucker_t*, const tucker_t*, double*, cudaStream_t);
template int dot_impl<float>(tpcg_ctx, const tucker_t*, const tucker_t*, double*, cudaStream_t);

// dot_impl replayed from a per-context CUDA graph keyed by (x, y, out), as round_cached
template <typename T>
int dot_cached(tpcg_ctx c, const tucker_t* x, const tucker_t* y, double* out_dev, cudaStream_t st) {
    if (prof_on() || st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread)
        return dot_impl<T>(c, x, y, out_dev, st);
    for (const auto& g : c->rgraphs)
        if (g.rc == -1 && g.desc == x->desc && g.U0 == y->desc && g.eps_dev == out_dev) {
            TPCG_CUDA(cudaGraphLaunch(g.exec, st));
            g_launches.fetch_add(g.nkern, std::memory_order_relaxed);
            return TPCG_OK;
        }
    const long long k0 = t_launches;
    TPCG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int s = dot_impl<T>(c, x, y, out_dev, st);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s != TPCG_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (s != TPCG_OK) return s;
        set_error(std::string("dot_cached: stream capture failed: ") + cudaGetErrorString(e));
        return TPCG_E_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("dot_cached: graph instantiation failed: ") + cudaGetErrorString(ei));
        return TPCG_E_CUDA;
    }
    c->rgraphs.push_back({x->desc, y->desc, out_dev, -1, 0, exec, t_launches - k0});
    TPCG_CUDA(cudaGraphLaunch(exec, st));
    return TPCG_OK;
}
template int dot_cached<double>(tpcg_ctx, const tucker_t*, const tucker_t*, double*, cudaStream_t);
template int dot_cached<float>(tpcg_ctx, const tucker_t*, const tucker_t*, double*, cudaStream_t);


// --------------------------------------------------------------------------------------------------
// The same dot with no allocation at all, for callers that cannot call cudaMalloc: code that runs while
// someone else's stream capture is open (an allocation there breaks the capture), allocator or driver
// callbacks, and hosts that size every device buffer up front and forbid growth.  The scratch of the
// context-based dot (GEMM argument slots, the three cross-Grams W_t, the two contraction buffers) lives
// in one fixed device array of this file, sized for ranks <= DOT_STATIC_MAX_RANK in FP64.  Nothing in it
// has to start at zero: every buffer is written (beta = 0) before it is read.  Concurrent calls share
// the array, so calls whose executions overlap on the device race.
// --------------------------------------------------------------------------------------------------
constexpr int DOT_STATIC_MAX_RANK = 64;
constexpr size_t DOT_STATIC_ARGS_OFF = 0;
constexpr size_t DOT_STATIC_CNT_OFF = ((6 * sizeof(GemmArgs) + 255) / 256) * 256;
constexpr size_t DOT_STATIC_W_OFF = DOT_STATIC_CNT_OFF + 256;
constexpr size_t DOT_STATIC_T_OFF =
    DOT_STATIC_W_OFF + ((3 * (size_t)DOT_STATIC_MAX_RANK * DOT_STATIC_MAX_RANK * sizeof(double) + 255) / 256) * 256;
constexpr size_t DOT_STATIC_BYTES =
    DOT_STATIC_T_OFF + 2 * (size_t)DOT_STATIC_MAX_RANK * DOT_STATIC_MAX_RANK * DOT_STATIC_MAX_RANK * sizeof(double);

static __device__ __align__(256) unsigned char g_dot_scratch[DOT_STATIC_BYTES];

// address of g_dot_scratch on the current device, looked up once per device (the first call on a device
// does this set-up; make it before any stream capture that will contain the call)
static int dot_static_scratch(unsigned char** out) {
    static std::mutex mu;
    static void* addr[64] = {};
    int dev = 0;
    TPCG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("tucker_dot_static: device ordinal out of range");
        return TPCG_E_INVALID;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_dot_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error(std::string("tucker_dot_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return TPCG_E_CUDA;
        }
        addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(addr[dev]);
    return TPCG_OK;
}

int dot_static_max_rank() { return DOT_STATIC_MAX_RANK; }

template <typename T>
int dot_static_impl(const tucker_t* x, const tucker_t* y, double* out_dev, cudaStream_t st) {
    unsigned char* base = nullptr;
    TPCG_TRY(dot_static_scratch(&base));
    const int n = x->n, rc = DOT_STATIC_MAX_RANK;
    GemmArgs* ga = reinterpret_cast<GemmArgs*>(base + DOT_STATIC_ARGS_OFF);
    int* counts = reinterpret_cast<int*>(base + DOT_STATIC_CNT_OFF);
    T* Wb = reinterpret_cast<T*>(base + DOT_STATIC_W_OFF);
    T* Ta = reinterpret_cast<T*>(base + DOT_STATIC_T_OFF);
    T* Tb = Ta + (long long)rc * rc * rc;
    plan_dot_kernel<T><<<1, 32, 0, st>>>(static_cast<const TuckerDesc*>(x->desc), static_cast<const T*>(x->U[0]),
                                         static_cast<const T*>(x->U[1]), static_cast<const T*>(x->U[2]),
                                         static_cast<const TuckerDesc*>(y->desc), static_cast<const T*>(y->U[0]),
                                         static_cast<const T*>(y->U[1]), static_cast<const T*>(y->U[2]), n, rc, Wb,
                                         Ta, Tb, ga, counts);
    TPCG_CHECK_LAUNCH();
    TPCG_TRY((launch_gemm<T, true, false>(ga, counts, 3, 1, rc, rc, st)));
    TPCG_TRY((launch_gemm<T, false, false>(ga + 3, nullptr, 1, 1, rc, rc * rc, st)));
    TPCG_TRY((launch_gemm<T, false, true>(ga + 4, nullptr, 1, rc, rc, rc, st)));
    TPCG_TRY((launch_gemm<T, false, true>(ga + 5, nullptr, 1, 1, rc * rc, rc, st)));
    dot_finish_kernel<T><<<1, 1024, 0, st>>>(static_cast<const TuckerDesc*>(x->desc), Ta, out_dev, counts + 1);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}
template int dot_static_impl<double>(const tucker_t*, const tucker_t*, double*, cudaStream_t);
template int dot_static_impl<float>(const tucker_t*, const tucker_t*, double*, cudaStream_t);

// --------------------------------------------------------------------------------------------------
// FD preconditioner, Alg. 4 with U~ = [W U_dft diag(1/mu) | V2 U2] (App. B):
//   u_t = U_dft^T (W^T S_t),  z2_t = (V2U2)^T S_t
//   for j < RP:  E_t[:, j r + c] = D_(t,j)[:n1] u_t[:, c] / mu^2,  E2_t = D_(t,j)[n1:] z2_t
//   V_t = W (U_dft E_t) + V2U2 E2_t;  core superdiag(omega / lambda_min) (x) G_s.
// ctx->fd[t][0..3] scratch buffers (n x max_cols each): T, u|z2, E|E2, A.
// gargs slots (offset 2*MAXB + 16): [0..2] u_t, [3..5] z2_t, [6..8] A_t, [9..11] V_t += V2U2 E2_t.
// --------------------------------------------------------------------------------------------------
template <typename T>
__global__ void fd_gather_kernel(const TuckerDesc* __restrict__ sd, const T* S0, const T* S1, const T* S2,
                                 const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ val,
                                 int n, int n1, T* B0, T* B1, T* B2) {
    const int t = blockIdx.z;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (l >= n1 || c >= sd->rank[t]) return;
    const T* S = t == 0 ? S0 : (t == 1 ? S1 : S2);
    T* B = t == 0 ? B0 : (t == 1 ? B1 : B2);
    T acc = T(0);
    for (int e = rp[l]; e < rp[l + 1]; ++e) acc = fma(val[e], S[ci[e] + (long long)c * n], acc);
    B[l + (long long)c * n1] = acc;
}

template <typename T>
__global__ void plan_fd_kernel(const TuckerDesc* __restrict__ sd, const T* S0, const T* S1, const T* S2, int n,
                               int n1, int n2, int RP, const T* dst, const T* v2u2, T* Tb0, T* Tb1, T* Tb2, T* Ub0,
                               T* Ub1, T* Ub2, T* Eb0, T* Eb1, T* Eb2, T* Ab0, T* Ab1, T* Ab2, T* V0, T* V1, T* V2,
                               GemmArgs* ga, int* counts, int vcap, int* err) {
    if (threadIdx.x != 0) return;
    const T* S[3] = {S0, S1, S2};
    T* Tb[3] = {Tb0, Tb1, Tb2};
    T* Ub[3] = {Ub0, Ub1, Ub2};
    T* Eb[3] = {Eb0, Eb1, Eb2};
    T* Ab[3] = {Ab0, Ab1, Ab2};
    T* V[3] = {V0, V1, V2};
    for (int t = 0; t < 3; ++t) {
        int r = sd->rank[t];
        int cols = RP * r;
        if (cols > vcap) {   // output capacity exceeded: flag and turn every product of this mode off
            if (err) *err = 1;
            r = 0;
            cols = 0;
        }
        // u_t (n1 x r) = dst^T T_t
        GemmArgs a{};
        a.M = n1; a.N = r; a.K = n1; a.nbatch = 1; a.alpha = 1.0;
        a.A = dst; a.lda = n1; a.B = Tb[t]; a.ldb = n1; a.C = Ub[t]; a.ldc = n1;
        ga[t] = a;
        // z2_t (n2 x r) = v2u2^T S_t, stored after u_t
        GemmArgs b{};
        b.M = n2; b.N = r; b.K = n; b.nbatch = 1; b.alpha = 1.0;
        b.A = v2u2; b.lda = n; b.B = S[t]; b.ldb = n; b.C = Ub[t] + (long long)n1 * r; b.ldc = n2 > 0 ? n2 : 1;
        ga[3 + t] = b;
        // A_t (n1 x RP r) = dst E_t
        GemmArgs c{};
        c.M = n1; c.N = cols; c.K = n1; c.nbatch = 1; c.alpha = 1.0;
        c.A = dst; c.lda = n1; c.B = Eb[t]; c.ldb = n1; c.C = Ab[t]; c.ldc = n1;
        ga[6 + t] = c;
        // V_t += v2u2 E2_t   (E2_t stored after E_t)
        GemmArgs d{};
        d.M = n; d.N = cols; d.K = n2; d.nbatch = 1; d.alpha = 1.0; d.beta = 1.0;
        d.A = v2u2; d.lda = n; d.B = Eb[t] + (long long)n1 * cols; d.ldb = n2 > 0 ? n2 : 1; d.C = V[t]; d.ldc = n;
        if (n2 == 0) d.M = 0;
        ga[9 + t] = d;
    }
    counts[0] = 3;
}

// E_(t,j) = D_(t,j) Z_t: grid x = 128-row tiles, y = (term j, group of FD_CG input columns), z = mode; a thread
// computes its row's factor exp(-alpha_j c_t lambda_l / lambda_min) / mu_l^2 once (in the compute precision) and
// scales that row of its group's columns (coalesced along the rows, the group's loads in flight together)
constexpr int FD_CG = 16;

template <typename T>
__global__ void __launch_bounds__(128) fd_scale_kernel(const TuckerDesc* __restrict__ sd, const T* __restrict__ U0,
                                                       const T* __restrict__ U1, const T* __restrict__ U2,
                                                       const T* __restrict__ lam, const T* __restrict__ mu,
                                                       const double* __restrict__ alpha, double lmin, double c0,
                                                       double c1, double c2, int n1, int n2, int RP, int ncg,
                                                       T* __restrict__ E0, T* __restrict__ E1, T* __restrict__ E2,
                                                       int vcap) {
    const int t = blockIdx.z, j = blockIdx.y / ncg, cg = blockIdx.y % ncg;
    const int r = sd->rank[t];
    const int n = n1 + n2;
    if (j >= RP || RP * r > vcap) return;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const T* __restrict__ U = t == 0 ? U0 : (t == 1 ? U1 : U2);
    T* __restrict__ E = t == 0 ? E0 : (t == 1 ? E1 : E2);
    const long long cols = (long long)RP * r;
    // direction weight c_t (1 for the Poisson operator; mu + (lambda + mu) delta_ti for elasticity block i)
    const T aj = (T)(alpha[j] * (t == 0 ? c0 : (t == 1 ? c1 : c2)) / lmin);
    const T dl = exp(-aj * lam[l]);
    for (int cb = cg * FD_CG; cb < r; cb += ncg * FD_CG) {
        const int ce = cb + FD_CG < r ? cb + FD_CG : r;
        if (l < n1) {
            const T m = mu[l];
            const T f = dl / (m * m);
#pragma unroll 4
            for (int c = cb; c < ce; ++c) E[l + (long long)(j * r + c) * n1] = f * U[l + (long long)c * n1];
        } else {
            const int q = l - n1;
#pragma unroll 4
            for (int c = cb; c < ce; ++c)
                E[(long long)n1 * cols + q + (long long)(j * r + c) * n2] = dl * U[(long long)n1 * r + q + (long long)c * n2];
        }
    }
}

// z2_t (n2 x r) = v2u2^T S_t (n2 <= 3 rows, K = n): one warp per output entry, fixed-order shuffle reduction
template <typename T>
__global__ void fd_v2_kernel(const TuckerDesc* __restrict__ sd, const T* __restrict__ v2u2, const T* S0,
                             const T* S1, const T* S2, T* Ub0, T* Ub1, T* Ub2, int n, int n1, int n2, int RP,
                             int vcap) {
    const int t = blockIdx.z;
    const int r = sd->rank[t];
    if (RP * r > vcap) return;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= n2 * r) return;
    const int q = w % n2, c = w / n2;
    const T* S = t == 0 ? S0 : (t == 1 ? S1 : S2);
    T* Ub = t == 0 ? Ub0 : (t == 1 ? Ub1 : Ub2);
    T acc = T(0);
    for (int i = lane; i < n; i += 32) acc = fma(v2u2[i + (long long)q * n], S[i + (long long)c * n], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) Ub[(long long)n1 * r + q + (long long)c * n2] = acc;
}

template <typename T>
__global__ void fd_scatter_kernel(const TuckerDesc* __restrict__ sd, const T* A0, const T* A1, const T* A2,
                                  const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ val,
                                  int n, int n1, int RP, T* V0, T* V1, T* V2, int vcap) {
    const int t = blockIdx.z;
    const int r = sd->rank[t];
    const int col = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= RP * r || RP * r > vcap || i >= n) return;
    const T* A = t == 0 ? A0 : (t == 1 ? A1 : A2);
    T* V = t == 0 ? V0 : (t == 1 ? V1 : V2);
    T acc = T(0);
    for (int e = rp[i]; e < rp[i + 1]; ++e) acc = fma(val[e], A[ci[e] + (long long)col * n1], acc);
    V[i + (long long)col * n] = acc;
}

__global__ void fd_desc_kernel(const TuckerDesc* __restrict__ sd, const double* __restrict__ omega, double lmin,
                               int RP, TuckerDesc* vd, int vcap, int* err, double* prof, int n, int n1, int n2, int p,
                               int elt) {
    if (threadIdx.x != 0) return;
    if (prof) {   // algorithmic work of Alg. 4 per input column: W^T gather, sine transforms, R_P scalings, W scatter
        const double cols = (double)sd->rank[0] + sd->rank[1] + sd->rank[2];
        const double lg = n1 > 1 ? log2((double)n1) : 1.0;
        prof[2 * PK_FD] += (1.0 + RP) * cols * (5.0 * n1 * lg + 4.0 * (p + 1) * n + 2.0 * (double)n * n2);
        prof[2 * PK_FD + 1] += (double)elt * (double)n * cols * (2.0 + 2.0 * RP);
    }
    bool ok = RP * sd->nblk <= TPCG_MAX_BLOCKS;
    for (int t = 0; t < 3; ++t) ok = ok && (RP * sd->rank[t] <= vcap);
    if (!ok) {
        if (err) *err = 1;
        vd->nblk = 0;
        vd->rank[0] = vd->rank[1] = vd->rank[2] = 0;
        return;
    }
    int nb = 0;
    for (int j = 0; j < RP; ++j)
        for (int b = 0; b < sd->nblk; ++b) {
            BlockDesc B = sd->blk[b];
            for (int t = 0; t < 3; ++t) B.off[t] += j * sd->rank[t];
            B.scale *= omega[j] / lmin;
            vd->blk[nb++] = B;
        }
    vd->nblk = nb;
    for (int t = 0; t < 3; ++t) vd->rank[t] = RP * sd->rank[t];
}

template <typename T>
int fd_impl(tpcg_problem pb, tpcg_ctx c, const tucker_t* s, tucker_t* v, cudaStream_t st, const double* wdir) {
    const double cw[3] = {wdir ? wdir[0] : 1.0, wdir ? wdir[1] : 1.0, wdir ? wdir[2] : 1.0};
    // weighted spectrum sum_t c_t lambda_t: its minimum is (sum_t c_t) / 3 times the unweighted lambda_min
    const double lmin = pb->lambda_min * (cw[0] + cw[1] + cw[2]) / 3.0;
    const int n = pb->n, n1 = pb->n1, n2 = pb->n2, RP = pb->RP;
    const int rc = c->rank_cap;
    GemmArgs* ga = c->gargs + 2 * TPCG_MAX_BLOCKS + 16;
    int* counts = reinterpret_cast<int*>(c->scal + 220);
    int* err = reinterpret_cast<int*>(c->scal + 230);
    T* buf[3][4];
    for (int t = 0; t < 3; ++t)
        for (int q = 0; q < 4; ++q) buf[t][q] = static_cast<T*>(c->fd[t][q]);
    const TuckerDesc* sd = static_cast<const TuckerDesc*>(s->desc);
    prof_begin(PK_FD, st);
    dim3 g1((n1 + 127) / 128, rc, 3);
    fd_gather_kernel<T><<<g1, 128, 0, st>>>(sd, static_cast<const T*>(s->U[0]), static_cast<const T*>(s->U[1]),
                                            static_cast<const T*>(s->U[2]), pb->d_wtrow, pb->d_wtcol,
                                            static_cast<const T*>(pb->d_wtval), n, n1, buf[0][0], buf[1][0],
                                            buf[2][0]);
    TPCG_CHECK_LAUNCH();
    plan_fd_kernel<T><<<1, 32, 0, st>>>(sd, static_cast<const T*>(s->U[0]), static_cast<const T*>(s->U[1]),
                                        static_cast<const T*>(s->U[2]), n, n1, n2, RP,
                                        static_cast<const T*>(pb->d_dst), static_cast<const T*>(pb->d_v2u2),
                                        buf[0][0], buf[1][0], buf[2][0], buf[0][1], buf[1][1], buf[2][1], buf[0][2],
                                        buf[1][2], buf[2][2], buf[0][3], buf[1][3], buf[2][3],
                                        static_cast<T*>(v->U[0]), static_cast<T*>(v->U[1]),
                                        static_cast<T*>(v->U[2]), ga, counts, v->cap, err);
    TPCG_CHECK_LAUNCH();
    const bool fft = pb->d_chirp != nullptr && dst_kind() == 1;
    const T* fx[3] = {buf[0][0], buf[1][0], buf[2][0]};
    T* fy[3] = {buf[0][1], buf[1][1], buf[2][1]};
    if (fft)   // u_t = U_dft^T T_t by FFTs
        TPCG_TRY(launch_chirp<T>(pb, 0, sd, 1, RP, v->cap, rc, fx, fy, n1, n1, st));
    else
        TPCG_TRY((launch_gemm<T, true, false>(ga, counts, 3, 1, n1, rc, st)));
    if (n2 > 0) {
        fd_v2_kernel<T><<<dim3((n2 * rc + 7) / 8, 1, 3), 256, 0, st>>>(
            sd, static_cast<const T*>(pb->d_v2u2), static_cast<const T*>(s->U[0]), static_cast<const T*>(s->U[1]),
            static_cast<const T*>(s->U[2]), buf[0][1], buf[1][1], buf[2][1], n, n1, n2, RP, v->cap);
        TPCG_CHECK_LAUNCH();
    }
    const int ncg = (rc + FD_CG - 1) / FD_CG;
    dim3 g2((n + 127) / 128, RP * ncg, 3);
    fd_scale_kernel<T><<<g2, 128, 0, st>>>(sd, buf[0][1], buf[1][1], buf[2][1], static_cast<const T*>(pb->d_lam),
                                           static_cast<const T*>(pb->d_mu), pb->d_alpha, lmin, cw[0], cw[1], cw[2], n1, n2, RP,
                                           ncg, buf[0][2], buf[1][2], buf[2][2], v->cap);
    TPCG_CHECK_LAUNCH();
    const T* ex[3] = {buf[0][2], buf[1][2], buf[2][2]};
    T* ey[3] = {buf[0][3], buf[1][3], buf[2][3]};
    if (fft)   // A_t = U_dft E_t by FFTs
        TPCG_TRY(launch_chirp<T>(pb, 1, sd, RP, RP, v->cap, RP * rc, ex, ey, n1, n1, st));
    else
        TPCG_TRY((launch_gemm<T, false, false>(ga + 6, counts, 3, 1, n1, RP * rc, st)));
    dim3 g3((n + 127) / 128, RP * rc, 3);
    fd_scatter_kernel<T><<<g3, 128, 0, st>>>(sd, buf[0][3], buf[1][3], buf[2][3], pb->d_wrow, pb->d_wcol,
                                             static_cast<const T*>(pb->d_wval), n, n1, RP, static_cast<T*>(v->U[0]),
                                             static_cast<T*>(v->U[1]), static_cast<T*>(v->U[2]), v->cap);
    TPCG_CHECK_LAUNCH();
    if (n2 > 0) TPCG_TRY((launch_gemm<T, false, false>(ga + 9, counts, 3, 1, n, RP * rc, st)));
    fd_desc_kernel<<<1, 32, 0, st>>>(sd, pb->d_omega, lmin, RP, static_cast<TuckerDesc*>(v->desc), v->cap,
                                     err, prof_dev(), n, n1, n2, pb->p, (int)sizeof(T));
    TPCG_CHECK_LAUNCH();
    prof_end(PK_FD, st);
    return TPCG_OK;
}
template int fd_impl<double>(tpcg_problem, tpcg_ctx, const tucker_t*, tucker_t*, cudaStream_t, const double*);
template int fd_impl<float>(tpcg_problem, tpcg_ctx, const tucker_t*, tucker_t*, cudaStream_t, const double*);

// --------------------------------------------------------------------------------------------------
// copies
// --------------------------------------------------------------------------------------------------
template <typename T>
__global__ void copy_factors_kernel(const TuckerDesc* __restrict__ sd, const T* S0, const T* S1, const T* S2, T* D0,
                                    T* D1, T* D2, int n, int cap) {
    const int t = blockIdx.z;
    const int k = sd->rank[t];
    if (k > cap) return;
    const T* S = t == 0 ? S0 : (t == 1 ? S1 : S2);
    T* D = t == 0 ? D0 : (t == 1 ? D1 : D2);
    const long long tot = (long long)n * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
        D[e] = S[e];
}

// plain source: copy its core into dst's core as well and point the descriptor at it
template <typename T>
__global__ void copy_core_kernel(const TuckerDesc* __restrict__ sd, TuckerDesc* dd, T* dcore, long long ccap) {
    __shared__ int plain;
    if (threadIdx.x == 0) plain = (sd->nblk == 1);
    __syncthreads();
    if (plain) {
        const BlockDesc& B = sd->blk[0];
        const long long tot = (long long)B.r[0] * B.r[1] * B.r[2];
        const T* src = static_cast<const T*>(B.core);
        if (tot <= ccap)
            for (long long e = threadIdx.x; e < tot; e += blockDim.x) dcore[e] = src[e];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nb = sd->nblk;
        dd->nblk = nb;
        for (int t = 0; t < 3; ++t) dd->rank[t] = sd->rank[t];
        for (int b = 0; b < nb; ++b) dd->blk[b] = sd->blk[b];
        if (plain) dd->blk[0].core = dcore;
    }
}

template <typename T>
int copy_tensor_impl(const tucker_t* src, tucker_t* dst, int n, int cap, cudaStream_t st) {
    dim3 grid(64, 1, 3);
    copy_factors_kernel<T><<<grid, 256, 0, st>>>(static_cast<const TuckerDesc*>(src->desc),
                                                 static_cast<const T*>(src->U[0]), static_cast<const T*>(src->U[1]),
                                                 static_cast<const T*>(src->U[2]), static_cast<T*>(dst->U[0]),
                                                 static_cast<T*>(dst->U[1]), static_cast<T*>(dst->U[2]), n, cap);
    TPCG_CHECK_LAUNCH();
    copy_core_kernel<T><<<1, 1024, 0, st>>>(static_cast<const TuckerDesc*>(src->desc),
                                            static_cast<TuckerDesc*>(dst->desc), static_cast<T*>(dst->core),
                                            dst->core_cap);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}
template int copy_tensor_impl<double>(const tucker_t*, tucker_t*, int, int, cudaStream_t);
template int copy_tensor_impl<float>(const tucker_t*, tucker_t*, int, int, cudaStream_t);

// FP32 plain tensor -> FP64 tensor
__global__ void promote_kernel(const TuckerDesc* __restrict__ sd, const float* S0, const float* S1, const float* S2,
                               const float* Sc, double* D0, double* D1, double* D2, double* Dc, TuckerDesc* dd, int n,
                               int cap, long long ccap) {
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x, gs = (long long)gridDim.x * blockDim.x;
    const float* S[3] = {S0, S1, S2};
    double* D[3] = {D0, D1, D2};
    const int r[3] = {sd->rank[0], sd->rank[1], sd->rank[2]};
    const bool ok = sd->nblk == 1 && r[0] <= cap && r[1] <= cap && r[2] <= cap &&
                    (long long)r[0] * r[1] * r[2] <= ccap;
    if (!ok) {
        if (gt == 0) { dd->nblk = 0; dd->rank[0] = dd->rank[1] = dd->rank[2] = 0; }
        return;
    }
    for (int t = 0; t < 3; ++t)
        for (long long e = gt; e < (long long)n * r[t]; e += gs) D[t][e] = (double)S[t][e];
    const float* core = static_cast<const float*>(sd->blk[0].core);
    const double sc = sd->blk[0].scale;
    for (long long e = gt; e < (long long)r[0] * r[1] * r[2]; e += gs) Dc[e] = sc * (double)core[e];
    if (gt == 0) {
        dd->nblk = 1;
        for (int t = 0; t < 3; ++t) {
            dd->rank[t] = r[t];
            dd->blk[0].off[t] = 0;
            dd->blk[0].r[t] = r[t];
        }
        dd->blk[0].core = Dc;
        dd->blk[0].scale = 1.0;
    }
}

int promote_tensor(const tucker_t* src32, tucker_t* dst64, cudaStream_t st) {
    promote_kernel<<<128, 256, 0, st>>>(static_cast<const TuckerDesc*>(src32->desc), static_cast<const float*>(src32->U[0]),
                                        static_cast<const float*>(src32->U[1]), static_cast<const float*>(src32->U[2]),
                                        nullptr, static_cast<double*>(dst64->U[0]), static_cast<double*>(dst64->U[1]),
                                        static_cast<double*>(dst64->U[2]), static_cast<double*>(dst64->core),
                                        static_cast<TuckerDesc*>(dst64->desc), dst64->n, dst64->cap, dst64->core_cap);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}

}  // namespace tpcg
