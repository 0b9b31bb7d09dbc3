// Sine transforms of the fast-diagonalization preconditioner (Alg. 4 with the eigenvector basis of App. B)
// by FFTs: O(n1 log n1) per column instead of the dense n1 x n1 product.
//
// App. B writes the eigenvector block as U_dft[l, j] = sqrt2 sin(omega_j x_l + k0 pi/2) on the interpolation
// points, omega_j = (j - k0/2 - k1/2) pi with the Neumann flags k0, k1 of the two ends: for two Dirichlet ends
// DST-I (odd degree) or DST-II (even degree), with a Neumann end the half-shifted sine and cosine variants.
// Alg. 4 applies U_dft^T (forward) and U_dft (inverse).  On the integer grid of sine_grid (kernels.cuh), with
// 0-based indices q (input) and o (output), every one of them is
//     y_o = sqrt2 Im( sum_q x_q exp(i pi (4 q o + a q + b o + g) / (4 D)) ),
// (a, b) = (2e, 2c) forward and (2c, 2e) inverse, g = e c + 2 k0 D (for two Dirichlet ends: D = n1 + 1 and
// (4, 4, 4) for odd degree; D = n1 and (4, 2, 2) forward, (2, 4, 2) inverse for even degree).  Any length n1
// (126 = 2 3^2 7 or 510 = 2 3 5 17 in the benchmark sizes) is handled by Bluestein's chirp-z identity
// 2 q o = q^2 + o^2 - (o - q)^2:
//     y_o = Im( post_o  sum_q (x_q pre_q) h_(o - q) ),   pre_q = e(a q + 2 q^2), post_o = sqrt2 e(b o + g + 2 o^2),
//     h_k = e(-2 k^2),  e(m) = exp(i pi m / (4 D)),
// a linear convolution evaluated with power-of-two FFTs of size Mf >= 2 n1 - 1 in shared memory: a
// decimation-in-frequency FFT (natural order in, bit-reversed out), the product with the precomputed spectrum
// of h (stored bit-reversed, 1 / Mf folded in), and a decimation-in-time inverse FFT (bit-reversed in,
// natural out).  All phases are integers m reduced modulo 8 D before one FP64 sin/cos on the host, so the
// tables are exact to FP64 rounding.
#include <math.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace tpcg {

static int bit_reverse(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r = (r << 1) | ((i >> b) & 1);
    return r;
}

SineGrid sine_grid(int n1, int p, int k0, int k1) {
    SineGrid g;
    const bool odd = (p % 2) == 1;
    g.D = odd ? n1 + 1 - k0 - k1 : n1;   // n_el
    g.e = 2 - k0 - k1;
    g.c = odd ? 2 - 2 * k0 : 1;
    g.g = 2 * k0 * g.D;
    return g;
}

// host tables in complex double pairs: [tw (Mf/2)] [pre_0 (L)] [post_0 (L)] [hs_0 (Mf)] [pre_1] [post_1] [hs_1]
int chirp_tables(int n1, int p, int k0, int k1, ChirpInfo* info, std::vector<double>* out) {
    if (n1 < 1 || n1 > 4096) {
        set_error("chirp_tables: n1 out of range");
        return TPCG_E_INVALID;
    }
    const int L = n1;
    int Mf = 1, logm = 0;
    while (Mf < 2 * L - 1) { Mf *= 2; ++logm; }
    if (Mf < 2) { Mf = 2; logm = 1; }
    const SineGrid sg = sine_grid(n1, p, k0, k1);
    const long long D = sg.D;
    const long long per = 8 * D;
    auto phase = [&](long long m, double* re, double* im) {
        long long r = m % per;
        if (r < 0) r += per;
        const double ang = M_PI * (double)r / (4.0 * (double)D);
        *re = cos(ang);
        *im = sin(ang);
    };
    info->L = L;
    info->Mf = Mf;
    info->logMf = logm;
    const size_t total = (size_t)Mf / 2 + 2 * ((size_t)2 * L + Mf);
    out->assign(2 * total, 0.0);
    double* o = out->data();
    for (int k = 0; k < Mf / 2; ++k) {   // tw_k = exp(-2 pi i k / Mf)
        const double ang = -2.0 * M_PI * (double)k / (double)Mf;
        o[2 * k] = cos(ang);
        o[2 * k + 1] = sin(ang);
    }
    size_t off = (size_t)Mf / 2;
    for (int kind = 0; kind < 2; ++kind) {
        const long long a4 = kind == 0 ? 2 * sg.e : 2 * sg.c;
        const long long b4 = kind == 0 ? 2 * sg.c : 2 * sg.e;
        const long long g4 = sg.e * sg.c + sg.g;
        for (long long q = 0; q < L; ++q) phase(a4 * q + 2 * q * q, &o[2 * (off + q)], &o[2 * (off + q) + 1]);
        off += L;
        for (long long q = 0; q < L; ++q) {
            double re, im;
            phase(b4 * q + g4 + 2 * q * q, &re, &im);
            o[2 * (off + q)] = sqrt(2.0) * re;
            o[2 * (off + q) + 1] = sqrt(2.0) * im;
        }
        off += L;
        // spectrum of the wrapped filter h_k (k = 0..L-1 at k, k = -(L-1)..-1 at Mf + k), direct DFT in FP64
        std::vector<double> hr(Mf, 0.0), hi(Mf, 0.0);
        for (long long k = 0; k < L; ++k) {
            phase(-2 * k * k, &hr[k], &hi[k]);
            if (k > 0) { hr[Mf - k] = hr[k]; hi[Mf - k] = hi[k]; }
        }
        for (int m = 0; m < Mf; ++m) {
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < Mf; ++k) {
                if (hr[k] == 0.0 && hi[k] == 0.0) continue;
                const long long km = ((long long)k * m) % Mf;
                const double ang = -2.0 * M_PI * (double)km / (double)Mf;
                const double c = cos(ang), s = sin(ang);
                sr += hr[k] * c - hi[k] * s;
                si += hr[k] * s + hi[k] * c;
            }
            const int pos = bit_reverse(m, logm);   // the forward FFT leaves element m at position bitrev(m)
            o[2 * (off + pos)] = sr / Mf;
            o[2 * (off + pos) + 1] = si / Mf;
        }
        off += Mf;
    }
    return TPCG_OK;
}

template <typename T>
struct cplx;
template <>
struct cplx<float> { using type = float2; };
template <>
struct cplx<double> { using type = double2; };

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {   // a * conj(b)
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}

constexpr int CHIRP_THREADS = 256;

// Y[:, c] = transform(X[:, c]) for the columns c < mult * rank_t of mode t = blockIdx.z, cpb columns per CTA.
// Modes whose output would exceed vcap columns produce nothing (the preconditioner reports that case).
template <typename T>
__global__ void __launch_bounds__(CHIRP_THREADS) chirp_dst_kernel(
    const TuckerDesc* __restrict__ sd, int mult, int rp_guard, int vcap, int L, int Mf, int cpb,
    const typename cplx<T>::type* __restrict__ tw, const typename cplx<T>::type* __restrict__ pre,
    const typename cplx<T>::type* __restrict__ post, const typename cplx<T>::type* __restrict__ hsb, const T* X0,
    const T* X1, const T* X2, T* Y0, T* Y1, T* Y2, int ldx, int ldy) {
    using C = typename cplx<T>::type;
    const int t = blockIdx.z;
    const int r = sd->rank[t];
    if ((long long)rp_guard * r > vcap) return;
    const int cols = mult * r;
    const int col0 = blockIdx.x * cpb;
    if (col0 >= cols) return;
    const int nc = min(cpb, cols - col0);
    const T* X = t == 0 ? X0 : (t == 1 ? X1 : X2);
    T* Y = t == 0 ? Y0 : (t == 1 ? Y1 : Y2);
    extern __shared__ __align__(16) unsigned char chirp_smem[];
    C* tws = reinterpret_cast<C*>(chirp_smem);     // Mf / 2 twiddles
    C* buf = tws + Mf / 2;                         // nc columns of Mf
    const int tid = threadIdx.x;
    for (int k = tid; k < Mf / 2; k += CHIRP_THREADS) tws[k] = tw[k];
    for (int e = tid; e < nc * Mf; e += CHIRP_THREADS) {
        const int c = e / Mf, q = e - c * Mf;
        C v;
        v.x = T(0);
        v.y = T(0);
        if (q < L) {
            const T x = X[q + (long long)(col0 + c) * ldx];
            const C pq = pre[q];
            v.x = x * pq.x;
            v.y = x * pq.y;
        }
        buf[e] = v;
    }
    __syncthreads();
    const int halfn = Mf / 2;
    // forward FFT, decimation in frequency: natural order in, bit-reversed order out
    for (int h = halfn; h >= 1; h >>= 1) {
        const int tstride = halfn / h;   // Mf / (2 h)
        for (int b = tid; b < nc * halfn; b += CHIRP_THREADS) {
            const int c = b / halfn, j = b - c * halfn;
            const int i = j & (h - 1), k0 = (j - i) * 2;
            C* col = buf + c * Mf;
            const C u = col[k0 + i], v = col[k0 + i + h];
            C s, d;
            s.x = u.x + v.x; s.y = u.y + v.y;
            d.x = u.x - v.x; d.y = u.y - v.y;
            col[k0 + i] = s;
            col[k0 + i + h] = cmul(d, tws[i * tstride]);
        }
        __syncthreads();
    }
    // product with the filter spectrum (bit-reversed like the data, 1 / Mf included)
    for (int e = tid; e < nc * Mf; e += CHIRP_THREADS) {
        const int q = e % Mf;
        buf[e] = cmul(buf[e], hsb[q]);
    }
    __syncthreads();
    // inverse FFT, decimation in time: bit-reversed order in, natural order out (conjugate twiddles)
    for (int h = 1; h < Mf; h <<= 1) {
        const int tstride = halfn / h;
        for (int b = tid; b < nc * halfn; b += CHIRP_THREADS) {
            const int c = b / halfn, j = b - c * halfn;
            const int i = j & (h - 1), k0 = (j - i) * 2;
            C* col = buf + c * Mf;
            const C tt = cmulc(col[k0 + i + h], tws[i * tstride]);
            const C u = col[k0 + i];
            C s, d;
            s.x = u.x + tt.x; s.y = u.y + tt.y;
            d.x = u.x - tt.x; d.y = u.y - tt.y;
            col[k0 + i] = s;
            col[k0 + i + h] = d;
        }
        __syncthreads();
    }
    for (int e = tid; e < nc * L; e += CHIRP_THREADS) {
        const int c = e / L, o = e - c * L;
        const C po = post[o], v = buf[c * Mf + o];
        Y[o + (long long)(col0 + c) * ldy] = po.x * v.y + po.y * v.x;   // Im(post_o v)
    }
}

// columns per CTA: two FFT lengths' worth of data at most (at least one column)
static int chirp_cpb(int Mf) { return std::max(1, std::min(8, 2048 / Mf)); }

template <typename T>
int launch_chirp(tpcg_problem pb, int kind, const TuckerDesc* sd, int mult, int rp_guard, int vcap, int maxcols,
                 const T* const* X, T* const* Y, int ldx, int ldy, cudaStream_t st) {
    using C = typename cplx<T>::type;
    const ChirpInfo& ci = pb->chirp;
    const int L = ci.L, Mf = ci.Mf;
    const C* base = static_cast<const C*>(pb->d_chirp);
    const C* tw = base;
    const C* pre = base + Mf / 2 + (size_t)kind * (2 * L + Mf);
    const C* post = pre + L;
    const C* hsb = post + L;
    const int cpb = chirp_cpb(Mf);
    const size_t smem = ((size_t)Mf / 2 + (size_t)cpb * Mf) * sizeof(C);
    if (maxcols <= 0) return TPCG_OK;
    dim3 grid((maxcols + cpb - 1) / cpb, 1, 3);
    chirp_dst_kernel<T><<<grid, CHIRP_THREADS, smem, st>>>(sd, mult, rp_guard, vcap, L, Mf, cpb, tw, pre, post, hsb,
                                                          X[0], X[1], X[2], Y[0], Y[1], Y[2], ldx, ldy);
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}
template int launch_chirp<double>(tpcg_problem, int, const TuckerDesc*, int, int, int, int, const double* const*,
                                  double* const*, int, int, cudaStream_t);
template int launch_chirp<float>(tpcg_problem, int, const TuckerDesc*, int, int, int, int, const float* const*,
                                 float* const*, int, int, cudaStream_t);

}  // namespace tpcg
