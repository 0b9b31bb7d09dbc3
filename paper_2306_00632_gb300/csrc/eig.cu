// Symmetric eigensolver for the mode Grams of ST-HOSVD (Alg. 1 step 3): cyclic Jacobi in one CTA.
//
// Jacobi is used (rather than tridiagonalisation + bisection) because on a positive semi-definite Gram it
// resolves the small eigenvalues to high relative accuracy when rotations stop at
// |a_pq| <= eps sqrt(a_pp a_qq) (Demmel & Veselic): the tails of the truncation rule are then sums of
// accurate small eigenvalues, so tight tolerances do not keep rounding noise.
//
//   * A (and V when both fit) in shared memory with leading dimension M + 1 (rows and columns read
//     without bank conflicts); otherwise in global memory (L2 resident);
//   * round-robin ordering: step s pairs (P, s) and ((s + k) mod P, (s - k) mod P), P = M' - 1, so M'/2
//     disjoint rotations run in parallel; the pairs and rotations of a step are computed once into shared
//     memory, then each thread applies both rotations to 2 x 2 blocks of A (upper blocks, mirrored) and
//     one rotation to rows of V (2 barriers per step);
//   * sweeps until no rotation is needed (or a sweep cap), then eigenvalues sorted decreasingly, the
//     truncation rule (clamped tail sums), and the kept eigenvectors written to S (ld n).
#include <math.h>

#include <mutex>
#include <string>

#include <cooperative_groups.h>

#include "common.cuh"
#include "eig.cuh"

namespace tpcg {

// key of the decreasing rank-counting sorts: a NaN eigenvalue sorts last, so that the ranks of any input
// (including NaN data) form a permutation and every index written through them stays in range
__device__ __forceinline__ double sort_key(double v) { return v == v ? v : -INFINITY; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Truncation rule of ST-HOSVD for mode m on the decreasingly sorted eigenvalues lam[0..M): the smallest s whose
// discarded energy is <= budget, then the cap; updates p.s[m] and p.discarded.  FP64: sum of the clamped
// discarded eigenvalues (conservative; accurate thanks to Jacobi's relative accuracy).  FP32: trace minus the
// kept eigenvalues (unbiased; the clamped FP32 small eigenvalues are noise-dominated).  One thread.
// threads of the one-CTA eigensolver (512 was measured slower alone and no faster with 16-32 solves at once)
constexpr int EIG_THREADS = 1024;

// relative rotation threshold of the Jacobi sweeps: diagonal entries converge to relative accuracy ~tau^2 and
// eigenvectors to angles ~tau times the eigenvalue ratio over the gap; the thresholds keep the FP64 vectors at
// parity level (1e-12) and the FP32 ones well inside FP32 truncation accuracy (3e-5)
template <typename T>
__host__ __device__ constexpr double jacobi_tau() { return sizeof(T) == 8 ? 1e-12 : 3e-5; }
// one-sided Jacobi (FP32): a pair is orthogonal once |a_p . a_q| <= HJ_TAU |a_p| |a_q|.  The normalised columns
// are then eigenvectors orthonormal to about HJ_TAU; the FP32 dot product itself resolves about 4e-7 at 128 rows.
constexpr float HJ_TAU = 2e-6f;
// a sweep whose rotations all had |a_p . a_q| <= HJ_TAU_LAST |a_p| |a_q| is the last one: cyclic Jacobi converges
// quadratically, so the sweep after it would only meet products near HJ_TAU_LAST^2 ~ HJ_TAU
constexpr float HJ_TAU_LAST = 1.5e-3f;

// Energy of the Gram outside the Rayleigh-Ritz subspace (trace(G) minus the Ritz values; 0 when the
// eigensolver's input is the Gram itself).  The FP32 rule (trace minus kept) counts it implicitly.
__device__ __forceinline__ double rr_remainder(const RoundPlan& p, const double* lam, int M, double trace) {
    if (!p.rr) return 0.0;
    double all = 0.0;
    for (int i = 0; i < M; ++i) all += lam[i] > 0.0 ? lam[i] : 0.0;
    return trace - all > 0.0 ? trace - all : 0.0;
}

// trace the truncation rule works with: the input's own, or the Gram's when the input is the Rayleigh-Ritz
// matrix Q^T G Q
__device__ __forceinline__ double rule_trace(const RoundPlan& p, double own) { return p.rr ? p.gtrace : own; }

template <typename T>
__device__ int truncation_rule(RoundPlan& p, const double* lam, int M, double trace, int m) {
    int s = M;
    if (sizeof(T) == 8) {
        // each eigenvalue of an FP64 Gram is known only to about eps trace (the Gram squares the singular
        // values, so sigma_i below sqrt(eps) sigma_max is unresolved).  In strict mode (tolerances below what
        // the Gram resolves) a direction is discarded only if its clamped eigenvalue plus that uncertainty
        // still fits the budget, so the truncation stays lossless instead of dropping directions whose energy
        // it cannot see; otherwise the clamped eigenvalues are used as they are.
        const double unc = p.strict ? 4.0 * 2.220446049250313e-16 * trace : 0.0;
        double tail = rr_remainder(p, lam, M, trace);
        for (int i = M - 1; i >= 0; --i) {
            const double li = (lam[i] > 0.0 ? lam[i] : 0.0) + unc;
            if (tail + li <= p.budget) { tail += li; s = i; } else break;
        }
    } else {
        double cum = 0.0;
        for (int q = 0; q <= M; ++q) {
            const double tail = trace - cum;
            if (tail <= p.budget) { s = q; break; }
            if (q < M) cum += lam[q];
        }
    }
    if (s == 0 && trace > 0.0 && p.norm2 > 0.0) s = 1;
    if (p.cap > 0 && s > p.cap) s = p.cap;
    double disc = 0.0;
    if (sizeof(T) == 8) {
        disc = rr_remainder(p, lam, M, trace);
        for (int i = s; i < M; ++i) disc += lam[i] > 0.0 ? lam[i] : 0.0;
    } else {
        double cum = 0.0;
        for (int i = 0; i < s; ++i) cum += lam[i];
        disc = trace - cum > 0.0 ? trace - cum : 0.0;
    }
    p.discarded += disc;
    p.s[m] = s;
    return s;
}

// SM: A and V both in shared memory (known at compile time, so the step loop uses shared-memory accesses
// rather than generic ones); otherwise a_smem / v_smem choose per matrix at run time.
template <typename T, bool SM>
__global__ void __launch_bounds__(EIG_THREADS) jacobi_eig_kernel(RoundPlan* plan, const T* __restrict__ G, T* __restrict__ Ag,
                                                          T* __restrict__ Vg, T* __restrict__ S, double* evals, int m,
                                                          int a_smem, int v_smem, int max_sweeps, double* prof) {
    RoundPlan& p = *plan;
    const int M = p.eM;
    const int n = p.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    extern __shared__ unsigned char smem_raw[];
    T* sbase = reinterpret_cast<T*>(smem_raw);
    const int ld = M + 1;
    T* A = SM ? sbase : (a_smem ? sbase : Ag);
    T* V = SM ? sbase + M * ld : (v_smem ? sbase + (long long)M * ld : Vg);
    __shared__ T cs[2 * 512];
    __shared__ short pq[2 * 512];
    __shared__ double lam[SMAX_EIG];
    __shared__ short ord[SMAX_EIG];
    __shared__ int s_rot, s_keep;
    __shared__ double s_tr;
    if (M <= 0) {
        if (tid == 0) {
            p.s[m] = 0;
            if (m == 0) { p.norm2 = 0; p.budget = 0; }
        }
        return;
    }
    for (int j = 0; j < M; ++j)
        for (int i = tid; i < M; i += nt) {
            A[i + j * ld] = G[i + (long long)j * M];
            V[i + j * ld] = (i == j) ? T(1) : T(0);
        }
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < M; ++i) t += (double)G[i + (long long)i * M];
        s_tr = t;
        if (m == 0) {
            p.norm2 = rule_trace(p, t);
            p.budget = fmax(p.eps * p.eps * p.norm2, p.abs2) / 3.0;
        }
    }
    __syncthreads();
    const int Mp = (M + 1) & ~1;
    const int half = Mp / 2;
    const int P = Mp - 1;
    // rotate only when a_pq is above the relative threshold and, in FP32, the absolute floor eps trace (entries
    // below it are rounding noise of the Gram itself).  FP64 has no absolute floor: with one, the block of
    // eigenvalues below eps trace stayed unrotated, its diagonal entries read as energies the truncation could
    // not discard, and the iterates of Alg. 5 kept those directions (mode ranks 43 instead of 27-33 on a
    // 48^3 problem).  The relative threshold tau need not reach
    // machine precision: once |a_pq| <= tau sqrt(a_pp a_qq) every diagonal entry is its eigenvalue to relative
    // accuracy ~tau^2, and the truncation rule only ever uses trace - sum(kept diagonal), which is the exact
    // discarded energy of the current orthonormal basis whatever the remaining off-diagonal mass.
    const T epsr = (T)jacobi_tau<T>();
    const T epsa = (T)((sizeof(T) == 8 ? 0.0 : 1.2e-7) * s_tr);
    const int nblk = half * (half + 1) / 2;   // 2 x 2 blocks (a <= b) of the pair partition
    // blocks of this thread (q = tid + j nt), decoded once when there are at most 4 per thread
    constexpr int NBREG = 4;   // 2 x 2 blocks per thread decoded once (enough up to M = 180 at 1024 threads)
    int ab[NBREG];
    const bool reg_blocks = nblk <= NBREG * nt;
    if (reg_blocks) {
#pragma unroll
        for (int j = 0; j < NBREG; ++j) {
            const int q = tid + j * nt;
            ab[j] = -1;
            if (q < nblk) {
                int bb = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
                while ((bb + 1) * (bb + 2) / 2 <= q) ++bb;
                while (bb * (bb + 1) / 2 > q) --bb;
                ab[j] = (q - bb * (bb + 1) / 2) | (bb << 16);
            }
        }
    }
    // V update: a warp (or a multiple of warps) per pair, consecutive rows across the lanes
    const int vtpp = max(32, (nt / half) & ~31);
    const int vk0 = tid / vtpp, vi0 = tid % vtpp, vkstep = nt / vtpp > 0 ? nt / vtpp : 1;
    // A <- J_a^T A J_b on the 2 x 2 block (pair a rows, pair b columns), mirrored for a < b
    auto update_block = [&](int a, int b) {
        const T sa = cs[2 * a + 1], sb = cs[2 * b + 1];
        if (sa == T(0) && sb == T(0)) return;
        const T ca = cs[2 * a], cb = cs[2 * b];
        const int pa = pq[2 * a], qa = pq[2 * a + 1], pb = pq[2 * b], qb = pq[2 * b + 1];
        if (qa < 0 || qb < 0) {
            // one side is the padding index: a single row/column pair (M odd)
            if (qa < 0 && qb < 0) return;
            if (qa < 0) {   // rotate columns pb, qb of row pa (and mirror)
                const T x = A[pa + pb * ld], y = A[pa + qb * ld];
                const T xn = cb * x - sb * y, yn = sb * x + cb * y;
                A[pa + pb * ld] = xn; A[pa + qb * ld] = yn;
                A[pb + pa * ld] = xn; A[qb + pa * ld] = yn;
            } else {        // rotate rows pa, qa of column pb (and mirror)
                const T x = A[pa + pb * ld], y = A[qa + pb * ld];
                const T xn = ca * x - sa * y, yn = sa * x + ca * y;
                A[pa + pb * ld] = xn; A[qa + pb * ld] = yn;
                A[pb + pa * ld] = xn; A[pb + qa * ld] = yn;
            }
            return;
        }
        const int cpb = pb * ld, cqb = qb * ld;
        const T x00 = A[pa + cpb], x01 = A[pa + cqb];
        const T x10 = A[qa + cpb], x11 = A[qa + cqb];
        // rows: J_a^T X
        const T r00 = ca * x00 - sa * x10, r01 = ca * x01 - sa * x11;
        const T r10 = sa * x00 + ca * x10, r11 = sa * x01 + ca * x11;
        // columns: (J_a^T X) J_b
        T y00 = cb * r00 - sb * r01, y01 = sb * r00 + cb * r01;
        T y10 = cb * r10 - sb * r11, y11 = sb * r10 + cb * r11;
        if (a == b) { y01 = T(0); y10 = T(0); }   // the rotated pair is annihilated
        A[pa + cpb] = y00; A[pa + cqb] = y01;
        A[qa + cpb] = y10; A[qa + cqb] = y11;
        if (a != b) {
            const int cpa = pa * ld, cqa = qa * ld;
            A[pb + cpa] = y00; A[qb + cpa] = y01;
            A[pb + cqa] = y10; A[qb + cqa] = y11;
        }
    };
    int nsweeps = 0;
    for (int sweep = 0; sweep < max_sweeps && M > 1; ++sweep) {
        ++nsweeps;
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int step = 0; step < P; ++step) {
            for (int k = tid; k < half; k += nt) {
                int a, b;
                if (k == 0) {
                    a = P; b = step;
                } else {   // (step + k) mod P and (step - k) mod P, with 0 < k < P and 0 <= step < P
                    a = step + k; if (a >= P) a -= P;
                    b = step - k; if (b < 0) b += P;
                }
                const int pi = a < b ? a : b, qi = a < b ? b : a;
                T c = T(1), s = T(0);
                if (qi < M) {
                    const T apq = A[pi + qi * ld];
                    const T app = A[pi + pi * ld], aqq = A[qi + qi * ld];
                    if (fabs(apq) > epsr * sqrt(fabs(app * aqq)) && fabs(apq) > epsa) {
                        const T th = (aqq - app) / (T(2) * apq);
                        const T t = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
                        c = T(1) / sqrt(t * t + T(1));
                        s = t * c;
                        s_rot = 1;
                    }
                }
                cs[2 * k] = c;
                cs[2 * k + 1] = s;
                pq[2 * k] = (short)pi;
                pq[2 * k + 1] = (short)(qi < M ? qi : -1);
            }
            __syncthreads();
            if (reg_blocks) {
#pragma unroll
                for (int j = 0; j < NBREG; ++j)
                    if (ab[j] >= 0) update_block(ab[j] & 0xffff, ab[j] >> 16);
            } else {
                for (int q = tid; q < nblk; q += nt) {
                    // q -> (a, b) with a <= b: b = largest with b (b + 1) / 2 <= q
                    int bb = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
                    while ((bb + 1) * (bb + 2) / 2 <= q) ++bb;
                    while (bb * (bb + 1) / 2 > q) --bb;
                    update_block(q - bb * (bb + 1) / 2, bb);
                }
            }
            // V <- V J
            for (int k = vk0; k < half; k += vkstep) {
                const T s = cs[2 * k + 1];
                if (s == T(0) || pq[2 * k + 1] < 0) continue;
                const T c = cs[2 * k];
                T* Vp = V + pq[2 * k] * ld;
                T* Vq = V + pq[2 * k + 1] * ld;
                for (int i = vi0; i < M; i += vtpp) {
                    const T vip = Vp[i], viq = Vq[i];
                    Vp[i] = c * vip - s * viq;
                    Vq[i] = s * vip + c * viq;
                }
            }
            __syncthreads();
        }
        if (!s_rot) break;
        __syncthreads();
    }
    // eigenvalues sorted decreasingly (rank counting)
    for (int i = tid; i < M; i += nt) {
        const double li = sort_key((double)A[i + (long long)i * ld]);
        int rk = 0;
        for (int j = 0; j < M; ++j) {
            const double lj = sort_key((double)A[j + (long long)j * ld]);
            if (lj > li || (lj == li && j < i)) ++rk;
        }
        ord[rk] = (short)i;
        lam[rk] = li;
    }
    __syncthreads();
    if (tid == 0) {
        const int s = truncation_rule<T>(p, lam, M, rule_trace(p, s_tr), m);
        s_keep = s;
        for (int i = 0; i < M; ++i) evals[i] = lam[i];
        if (prof) {   // algorithmic work: the dense symmetric eigen-decomposition count 9 M^3; Gram in, S out
            prof[2 * PK_EIG] += 9.0 * (double)M * M * M;
            prof[2 * PK_EIG + 1] += (double)sizeof(T) * ((double)M * M + (double)M * s);
            prof[2 * PK_SWEEPS] += nsweeps;       // Jacobi sweeps, and the number of Grams
            prof[2 * PK_SWEEPS + 1] += 1.0;
        }
    }
    __syncthreads();
    const int s = s_keep;
    for (int c = 0; c < s; ++c)
        for (int i = tid; i < M; i += nt) S[i + (long long)c * n] = V[i + (long long)ord[c] * ld];
}

// ------------------------------------------------------------------------------------------------------------
// Cluster-parallel cyclic Jacobi: one cluster of CJ_C CTAs per Gram, for n' <= CJ_MAXM.
//
// The M' players (matrix indices; M' = M rounded up to a multiple of 4 CJ_C, the extra ones dummies that
// never rotate) sit in h = M'/2 pair slots, top[k] / bot[k].  CTA c owns slots [c ppc, (c+1) ppc) and keeps
// the full COLUMNS of A and V of its 2 ppc players in shared memory (A is symmetric, so a column holds the
// row as well).  One step of a sweep:
//   1. each CTA computes the rotations of its own pairs (a_pp, a_qq, a_pq are in its columns) and writes them
//      into every CTA's rotation table through distributed shared memory; cluster barrier;
//   2. each CTA applies all h row rotations to its columns, then the column rotations of its own pairs to A
//      and V (both columns are local), and zeroes the annihilated a_pq;
//   3. the circle method moves every player one slot around the ring (top[0] fixed).  Inside a CTA this is a
//      relabelling of buffers; at a CTA boundary one top column moves right and one bottom column moves left,
//      pushed into the neighbour's landing buffers; cluster barrier; landing columns are copied into the
//      freed buffers.
// M'-1 steps make a sweep in which every pair meets once.  The FP64 arithmetic of a step is split over the
// cluster's SMs, which is what matters on a part whose FP64 rate is 1/64 of FP32.
// ------------------------------------------------------------------------------------------------------------
constexpr int CJ_C = 8;          // CTAs per cluster (portable size)
constexpr int CJ_THREADS = 256;
constexpr int CJ_MAXM = 256;     // largest padded Gram
constexpr int CJ_MAXPPC = CJ_MAXM / (2 * CJ_C);

static inline int cj_padded(int M) { return ((M + 4 * CJ_C - 1) / (4 * CJ_C)) * (4 * CJ_C); }

template <typename T>
__global__ void __cluster_dims__(CJ_C, 1, 1) __launch_bounds__(CJ_THREADS)
    cjacobi_eig_kernel(RoundPlan* plan, const T* __restrict__ G, T* __restrict__ S, double* evals, int m,
                       int max_sweeps, double* prof) {
    namespace cgx = cooperative_groups;
    cgx::cluster_group cluster = cgx::this_cluster();
    const int crank = (int)cluster.block_rank();
    RoundPlan& p = *plan;
    const int M = p.eM;
    const int n = p.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (M <= 1) {   // uniform across the cluster: nothing to rotate
        if (crank == 0 && tid == 0) {
            double t = M == 1 ? (double)G[0] : 0.0;
            if (m == 0) { p.norm2 = rule_trace(p, t); p.budget = fmax(p.eps * p.eps * p.norm2, p.abs2) / 3.0; }
            double lam1[1] = {t};
            const int s = truncation_rule<T>(p, lam1, M, rule_trace(p, t), m);
            if (M == 1) evals[0] = t;
            if (s > 0) S[0] = T(1);
        }
        return;
    }
    const int Mp = ((M + 4 * CJ_C - 1) / (4 * CJ_C)) * (4 * CJ_C);
    const int h = Mp / 2, ppc = h / CJ_C, lo = crank * ppc;
    const int ncol = 2 * ppc;
    const int ld = Mp + 1;
    extern __shared__ unsigned char smem_raw[];
    T* sA = reinterpret_cast<T*>(smem_raw);            // (ncol + 2) columns: slot buffers, landing top, landing bot
    T* sV = sA + (size_t)(ncol + 2) * ld;
    const int LT = ncol, LB = ncol + 1;
    __shared__ T csv[2 * (CJ_MAXM / 2)];
    __shared__ short pqv[2 * (CJ_MAXM / 2)];
    __shared__ short tix[CJ_MAXPPC], bix[CJ_MAXPPC], topP[CJ_MAXPPC], botP[CJ_MAXPPC];
    __shared__ short inP[2];                           // players arriving in the landing buffers (top, bot)
    __shared__ int flags[CJ_C];
    __shared__ int s_rot, s_keep;
    __shared__ double lam_all[CJ_MAXM];                // CTA 0: eigenvalue of each player
    __shared__ double lam[CJ_MAXM];
    __shared__ short rank_of[CJ_MAXM];
    __shared__ double s_tr;
    // initial slots: top[k] = 2k, bot[k] = 2k + 1; buffers 0..ppc-1 top, ppc..2ppc-1 bottom
    if (tid < ppc) {
        tix[tid] = (short)tid;
        bix[tid] = (short)(ppc + tid);
        topP[tid] = (short)(2 * (lo + tid));
        botP[tid] = (short)(2 * (lo + tid) + 1);
    }
    __syncthreads();
    for (int w = tid; w < ncol * Mp; w += nt) {
        const int j = w / Mp, i = w % Mp;
        const int P = j < ppc ? topP[j] : botP[j - ppc];
        const int b = j < ppc ? tix[j] : bix[j - ppc];
        sA[b * ld + i] = (P < M && i < M) ? G[i + (long long)P * M] : T(0);
        sV[b * ld + i] = (i == P) ? T(1) : T(0);
    }
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < M; ++i) t += (double)G[i + (long long)i * M];
        s_tr = t;
        if (m == 0 && crank == 0) {
            p.norm2 = rule_trace(p, t);
            p.budget = fmax(p.eps * p.eps * p.norm2, p.abs2) / 3.0;
        }
    }
    __syncthreads();
    const T epsr = (T)jacobi_tau<T>();
    const T epsa = (T)((sizeof(T) == 8 ? 0.0 : 1.2e-7) * s_tr);   // FP64: relative threshold only (see above)
    cluster.sync();   // every CTA initialised before any remote write
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int step = 0; step < Mp - 1; ++step) {
            // 1. rotations of the own pairs, broadcast to every CTA's table
            if (tid < ppc) {
                const int k = lo + tid;
                const int Pt = topP[tid], Pb = botP[tid];
                const int pi = Pt < Pb ? Pt : Pb, qi = Pt < Pb ? Pb : Pt;
                const int bp = Pt < Pb ? tix[tid] : bix[tid], bq = Pt < Pb ? bix[tid] : tix[tid];
                T c = T(1), sn = T(0);
                if (qi < M) {
                    const T apq = sA[bq * ld + pi];
                    const T app = sA[bp * ld + pi], aqq = sA[bq * ld + qi];
                    if (fabs(apq) > epsr * sqrt(fabs(app * aqq)) && fabs(apq) > epsa) {
                        const T th = (aqq - app) / (T(2) * apq);
                        const T t = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
                        c = T(1) / sqrt(t * t + T(1));
                        sn = t * c;
                        s_rot = 1;
                    }
                }
                for (int r = 0; r < CJ_C; ++r) {
                    T* rcs = cluster.map_shared_rank(csv, r);
                    short* rpq = cluster.map_shared_rank(pqv, r);
                    rcs[2 * k] = c;
                    rcs[2 * k + 1] = sn;
                    rpq[2 * k] = (short)pi;
                    rpq[2 * k + 1] = (short)(qi < M ? qi : -1);
                }
            }
            cluster.sync();
            // 2a. row rotations (all pairs) on the local columns; lanes run over columns (conflict-free rows)
            for (int w = tid; w < h * ncol; w += nt) {
                const int j = w % ncol, k = w / ncol;
                const T sn = csv[2 * k + 1];
                if (sn == T(0)) continue;
                const T c = csv[2 * k];
                const int pi = pqv[2 * k], qi = pqv[2 * k + 1];
                T* col = sA + (j < ppc ? tix[j] : bix[j - ppc]) * ld;
                const T x = col[pi], y = col[qi];
                col[pi] = c * x - sn * y;
                col[qi] = sn * x + c * y;
            }
            __syncthreads();
            // 2b. column rotations of the own pairs, A and V
            for (int w = tid; w < ppc * Mp; w += nt) {
                const int kk = w / Mp, i = w % Mp;
                const int k = lo + kk;
                const T sn = csv[2 * k + 1];
                if (sn == T(0)) continue;
                const T c = csv[2 * k];
                const bool topfirst = topP[kk] < botP[kk];
                const int bp = topfirst ? tix[kk] : bix[kk], bq = topfirst ? bix[kk] : tix[kk];
                T* Ap = sA + bp * ld;
                T* Aq = sA + bq * ld;
                const T x = Ap[i], y = Aq[i];
                Ap[i] = c * x - sn * y;
                Aq[i] = sn * x + c * y;
                T* Vp = sV + bp * ld;
                T* Vq = sV + bq * ld;
                const T vx = Vp[i], vy = Vq[i];
                Vp[i] = c * vx - sn * vy;
                Vq[i] = sn * vx + c * vy;
            }
            __syncthreads();
            if (tid < ppc) {   // the rotated pair is annihilated
                const int k = lo + tid;
                if (csv[2 * k + 1] != T(0)) {
                    const int pi = pqv[2 * k], qi = pqv[2 * k + 1];
                    const bool topfirst = topP[tid] < botP[tid];
                    const int bp = topfirst ? tix[tid] : bix[tid], bq = topfirst ? bix[tid] : tix[tid];
                    sA[bq * ld + pi] = T(0);
                    sA[bp * ld + qi] = T(0);
                }
            }
            __syncthreads();
            // 3. ring move: push the boundary columns into the neighbours' landing buffers
            const bool send_right = crank < CJ_C - 1, send_left = crank > 0;
            if (send_right) {   // top of the last own slot -> landing top of crank + 1
                T* rA = cluster.map_shared_rank(sA, crank + 1) + LT * ld;
                T* rV = cluster.map_shared_rank(sV, crank + 1) + LT * ld;
                const T* a = sA + tix[ppc - 1] * ld;
                const T* v = sV + tix[ppc - 1] * ld;
                for (int i = tid; i < Mp; i += nt) { rA[i] = a[i]; rV[i] = v[i]; }
                if (tid == 0) cluster.map_shared_rank(inP, crank + 1)[0] = topP[ppc - 1];
            }
            if (send_left) {    // bottom of the first own slot -> landing bottom of crank - 1
                T* rA = cluster.map_shared_rank(sA, crank - 1) + LB * ld;
                T* rV = cluster.map_shared_rank(sV, crank - 1) + LB * ld;
                const T* a = sA + bix[0] * ld;
                const T* v = sV + bix[0] * ld;
                for (int i = tid; i < Mp; i += nt) { rA[i] = a[i]; rV[i] = v[i]; }
                if (tid == 0) cluster.map_shared_rank(inP, crank - 1)[1] = botP[0];
            }
            cluster.sync();
            // relabel (one thread), then copy the landing columns into the freed buffers
            __shared__ short fill_top, fill_bot;   // buffers that receive the landing columns (-1: none)
            if (tid == 0) {
                short nt_[CJ_MAXPPC], nb_[CJ_MAXPPC], ntp[CJ_MAXPPC], nbp[CJ_MAXPPC];
                short ftop = -1, fbot = -1;
                // tops: slot kk takes slot kk-1's top; slot 0 keeps it (CTA 0), takes the landing (others)
                for (int kk = 1; kk < ppc; ++kk) { nt_[kk] = tix[kk - 1]; ntp[kk] = topP[kk - 1]; }
                // bottoms: slot kk takes slot kk+1's bottom
                for (int kk = 0; kk + 1 < ppc; ++kk) { nb_[kk] = bix[kk + 1]; nbp[kk] = botP[kk + 1]; }
                if (crank == 0) {
                    nt_[0] = tix[0]; ntp[0] = topP[0];
                    nt_[1] = bix[0]; ntp[1] = botP[0];   // bot[0] -> top[1]
                    for (int kk = 2; kk < ppc; ++kk) { nt_[kk] = tix[kk - 1]; ntp[kk] = topP[kk - 1]; }
                } else {
                    nt_[0] = bix[0]; ntp[0] = inP[0];     // freed bottom buffer receives the landing top
                    ftop = bix[0];
                }
                if (crank == CJ_C - 1) {
                    nb_[ppc - 1] = tix[ppc - 1]; nbp[ppc - 1] = topP[ppc - 1];   // top[h-1] -> bot[h-1]
                } else {
                    nb_[ppc - 1] = tix[ppc - 1]; nbp[ppc - 1] = inP[1];   // freed top buffer receives the landing bottom
                    fbot = tix[ppc - 1];
                }
                for (int kk = 0; kk < ppc; ++kk) {
                    tix[kk] = nt_[kk]; topP[kk] = ntp[kk];
                    bix[kk] = nb_[kk]; botP[kk] = nbp[kk];
                }
                fill_top = ftop;
                fill_bot = fbot;
            }
            __syncthreads();
            if (fill_top >= 0)
                for (int i = tid; i < Mp; i += nt) {
                    sA[fill_top * ld + i] = sA[LT * ld + i];
                    sV[fill_top * ld + i] = sV[LT * ld + i];
                }
            if (fill_bot >= 0)
                for (int i = tid; i < Mp; i += nt) {
                    sA[fill_bot * ld + i] = sA[LB * ld + i];
                    sV[fill_bot * ld + i] = sV[LB * ld + i];
                }
            __syncthreads();
        }
        // sweep end: did any CTA rotate?  (every CTA writes its flag into every CTA, then reads locally)
        if (tid < CJ_C) cluster.map_shared_rank(flags, tid)[crank] = s_rot;
        cluster.sync();
        int any = 0;
        for (int r = 0; r < CJ_C; ++r) any |= flags[r];
        cluster.sync();   // flags read before the next sweep may overwrite them
        if (!any) break;
    }
    // eigenvalues of the real players into CTA 0
    for (int j = tid; j < ncol; j += nt) {
        const int P = j < ppc ? topP[j] : botP[j - ppc];
        const int b = j < ppc ? tix[j] : bix[j - ppc];
        if (P < M) cluster.map_shared_rank(lam_all, 0)[P] = (double)sA[b * ld + P];
    }
    cluster.sync();
    if (crank == 0) {
        // decreasing order by rank counting (ties by index), then the truncation rule
        for (int i = tid; i < M; i += nt) {
            const double li = sort_key(lam_all[i]);
            int rk = 0;
            for (int j = 0; j < M; ++j) {
                const double lj = sort_key(lam_all[j]);
                if (lj > li || (lj == li && j < i)) ++rk;
            }
            lam[rk] = li;
            rank_of[i] = (short)rk;
        }
        __syncthreads();
        if (tid == 0) {
            const int s = truncation_rule<T>(p, lam, M, rule_trace(p, s_tr), m);
            s_keep = s;
            for (int i = 0; i < M; ++i) evals[i] = lam[i];
            if (prof) {
                prof[2 * PK_EIG] += 9.0 * (double)M * M * M;
                prof[2 * PK_EIG + 1] += (double)sizeof(T) * ((double)M * M + (double)M * s);
            }
        }
        __syncthreads();
        for (int r = 1; r < CJ_C; ++r) {
            short* rr = cluster.map_shared_rank(rank_of, r);
            for (int i = tid; i < M; i += nt) rr[i] = rank_of[i];
            if (tid == 0) cluster.map_shared_rank(&s_keep, r)[0] = s_keep;
        }
    }
    cluster.sync();
    // kept eigenvectors: column rank_of[P] of S receives V's column of player P
    const int s = s_keep;
    for (int w = tid; w < ncol * M; w += nt) {
        const int j = w / M, i = w % M;
        const int P = j < ppc ? topP[j] : botP[j - ppc];
        if (P >= M) continue;
        const int rk = rank_of[P];
        if (rk < s) S[i + (long long)rk * n] = sV[(j < ppc ? tix[j] : bix[j - ppc]) * ld + i];
    }
    cluster.sync();   // no CTA leaves while another may still address its shared memory
}

// Dynamic shared-memory opt-in of a kernel, once per (kernel slot, device): cudaFuncSetAttribute is a host call
// that takes driver locks, so it stays off the per-launch path that many solver threads share.
static int smem_optin(const void* func, int slot, int bytes) {
    static std::mutex mu;
    static bool done[8][64] = {};
    int dev = 0;
    TPCG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) dev = 63;
    std::lock_guard<std::mutex> lock(mu);
    if (!done[slot][dev]) {
        TPCG_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        done[slot][dev] = true;
    }
    return TPCG_OK;
}

// FP64 Grams up to CJ_MAXM go to the cluster kernel (FP64 arithmetic bound); FP32 Grams stay on one CTA
template <typename T>
static bool use_cluster_eig(int n) {
    return sizeof(T) == 8 && n >= 2 && cj_padded(n) <= CJ_MAXM;
}

// ------------------------------------------------------------------------------------------------------------
// FP32 Grams up to JV_MAXM with A and V resident in shared memory: the cyclic Jacobi of jacobi_eig_kernel (same
// pair order, thresholds and rotation formula; the truncation rule is shared) arranged for fewer instructions
// and no idle warps per step:
//  - the thread that computes a pair's rotation also writes the rotated 2 x 2 diagonal block
//    (a_pp - t a_pq, a_qq + t a_pq, zero coupling), so the update phase has only the half (half - 1) / 2
//    off-diagonal blocks: two per thread at M = 128, the same for every warp;
//  - V <- V J of step s runs beside the rotations of step s + 1 (V is not read by them), on the warps that
//    compute no rotation; the rotations are double-buffered by step parity;
//  - each pair's rotation is packed as float2 (c, s) and its indices as int4 (p, q, p ld, q ld); the 2 x 2
//    products and the V update use paired FP32 FMAs (__ffma2_rn / __fmul2_rn); V's columns are 16-byte
//    aligned, one float4 of a column per lane.
// ------------------------------------------------------------------------------------------------------------
constexpr int JV_MAXM = 128;   // a V column is at most 32 float4 (one per lane)

static inline size_t jv_smem_bytes(int n) {
    const size_t a = ((size_t)n * (n + 1) + 3) & ~(size_t)3;
    return (a + (size_t)n * ((n + 3) & ~3)) * sizeof(float);
}

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

__global__ void __launch_bounds__(EIG_THREADS) jacobi_eig_v_kernel(RoundPlan* plan, const float* __restrict__ G,
                                                                   float* __restrict__ S, double* evals, int m,
                                                                   int max_sweeps, double* prof) {
    RoundPlan& p = *plan;
    const int M = p.eM;
    const int n = p.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    extern __shared__ __align__(16) unsigned char jv_smem[];
    const int ld = M + 1;
    const int ldv = (M + 3) & ~3;
    float* A = reinterpret_cast<float*>(jv_smem);
    float* V = A + ((M * ld + 3) & ~3);
    __shared__ float2 cs[2][JV_MAXM / 2];
    __shared__ int4 pinfo[2][JV_MAXM / 2];
    __shared__ double lam[JV_MAXM];
    __shared__ short ord[JV_MAXM];
    __shared__ int s_rot, s_keep;
    __shared__ double s_tr;
    if (M <= 0) {
        if (tid == 0) {
            p.s[m] = 0;
            if (m == 0) { p.norm2 = 0; p.budget = 0; }
        }
        return;
    }
    for (int e = tid; e < M * M; e += nt) {
        const int i = e % M, j = e / M;
        A[i + j * ld] = G[e];
    }
    for (int e = tid; e < M * ldv; e += nt) {   // V = I, padding rows zero (they stay zero under rotations)
        const int i = e % ldv, j = e / ldv;
        V[e] = (i == j) ? 1.f : 0.f;
    }
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < M; ++i) t += (double)G[i + (long long)i * M];
        s_tr = t;
        if (m == 0) {
            p.norm2 = rule_trace(p, t);
            p.budget = fmax(p.eps * p.eps * p.norm2, p.abs2) / 3.0;
        }
    }
    __syncthreads();
    const int Mp = (M + 1) & ~1;
    const int half = Mp / 2;
    const int P = Mp - 1;
    const float epsr = (float)jacobi_tau<float>();
    const float epsa = (float)(1.2e-7 * s_tr);
    // off-diagonal blocks (a < b) of this thread: q = tid + j nt, q = b (b - 1) / 2 + a
    const int nblk = half * (half - 1) / 2;
    constexpr int NBREG = 2;   // nblk <= 2016 <= 2 x 1024 for M <= 128
    int ab[NBREG];
#pragma unroll
    for (int j = 0; j < NBREG; ++j) {
        const int q = tid + j * nt;
        ab[j] = -1;
        if (q < nblk) {
            int bb = (int)((1.0f + sqrtf(8.0f * (float)q + 1.0f)) * 0.5f);
            while (bb * (bb - 1) / 2 > q) --bb;
            while ((bb + 1) * bb / 2 <= q) ++bb;
            ab[j] = (q - bb * (bb - 1) / 2) | (bb << 16);
        }
    }
    // roles in the first phase of a step: the last `half` threads compute rotations, the warps below them
    // rotate V by the previous step's rotations
    const int krot = tid - (nt - half);
    const int warp = tid >> 5, lane = tid & 31;
    const int nvw = (nt - half) >> 5;
    const bool vlane = 4 * lane < M;
    // V <- V J for the rotations in buffer b (one warp per pair of columns, four rows per lane)
    auto update_v = [&](int b) {
        for (int k = warp; k < half; k += nvw) {
            const float2 r = cs[b][k];
            const int4 pk = pinfo[b][k];
            if (r.y == 0.f || pk.y < 0 || !vlane) continue;
            float4* Vp = reinterpret_cast<float4*>(V + pk.x * ldv) + lane;
            float4* Vq = reinterpret_cast<float4*>(V + pk.y * ldv) + lane;
            const float4 vp = *Vp, vq = *Vq;
            const float2 c2 = f2(r.x, r.x), s2 = f2(r.y, r.y), ms2 = f2(-r.y, -r.y);
            const float2 p01 = __ffma2_rn(c2, f2(vp.x, vp.y), __fmul2_rn(ms2, f2(vq.x, vq.y)));
            const float2 p23 = __ffma2_rn(c2, f2(vp.z, vp.w), __fmul2_rn(ms2, f2(vq.z, vq.w)));
            const float2 q01 = __ffma2_rn(s2, f2(vp.x, vp.y), __fmul2_rn(c2, f2(vq.x, vq.y)));
            const float2 q23 = __ffma2_rn(s2, f2(vp.z, vp.w), __fmul2_rn(c2, f2(vq.z, vq.w)));
            *Vp = make_float4(p01.x, p01.y, p23.x, p23.y);
            *Vq = make_float4(q01.x, q01.y, q23.x, q23.y);
        }
    };
    // A <- J_a^T A J_b on the off-diagonal 2 x 2 block (pair a rows, pair b columns, a < b) and its mirror
    auto update_block = [&](const float2* csb, const int4* pib, int a, int b) {
        const float2 ra = csb[a], rb = csb[b];
        if (ra.y == 0.f && rb.y == 0.f) return;
        const int4 ia = pib[a], ib = pib[b];
        const float ca = ra.x, sa = ra.y, cb = rb.x, sb = rb.y;
        const int pa = ia.x, qa = ia.y, pb = ib.x, qb = ib.y;
        if (qa < 0 || qb < 0) {   // one side is the padding index (M odd): a single row / column pair
            if (qa < 0 && qb < 0) return;
            if (qa < 0) {   // rotate columns pb, qb of row pa (and mirror)
                const float x = A[pa + ib.z], y = A[pa + ib.w];
                const float xn = cb * x - sb * y, yn = sb * x + cb * y;
                A[pa + ib.z] = xn; A[pa + ib.w] = yn;
                A[pb + ia.z] = xn; A[qb + ia.z] = yn;
            } else {        // rotate rows pa, qa of column pb (and mirror)
                const float x = A[pa + ib.z], y = A[qa + ib.z];
                const float xn = ca * x - sa * y, yn = sa * x + ca * y;
                A[pa + ib.z] = xn; A[qa + ib.z] = yn;
                A[pb + ia.z] = xn; A[pb + ia.w] = yn;
            }
            return;
        }
        const int cpb = ib.z, cqb = ib.w;
        const float2 X0 = f2(A[pa + cpb], A[pa + cqb]);   // row pa: columns pb, qb
        const float2 X1 = f2(A[qa + cpb], A[qa + cqb]);   // row qa
        // rows: J_a^T X
        const float2 R0 = __ffma2_rn(f2(ca, ca), X0, __fmul2_rn(f2(-sa, -sa), X1));
        const float2 R1 = __ffma2_rn(f2(sa, sa), X0, __fmul2_rn(f2(ca, ca), X1));
        // columns: (J_a^T X) J_b, on (r00, r10) and (r01, r11)
        const float2 C0 = f2(R0.x, R1.x), C1 = f2(R0.y, R1.y);
        const float2 Y0 = __ffma2_rn(f2(cb, cb), C0, __fmul2_rn(f2(-sb, -sb), C1));   // (y00, y10)
        const float2 Y1 = __ffma2_rn(f2(sb, sb), C0, __fmul2_rn(f2(cb, cb), C1));     // (y01, y11)
        A[pa + cpb] = Y0.x; A[pa + cqb] = Y1.x;
        A[qa + cpb] = Y0.y; A[qa + cqb] = Y1.y;
        const int cpa = ia.z, cqa = ia.w;
        A[pb + cpa] = Y0.x; A[qb + cpa] = Y1.x;
        A[pb + cqa] = Y0.y; A[qb + cqa] = Y1.y;
    };
    int nsweeps = 0;
    int g = 0;   // steps done: the rotations of step g are in buffer g & 1
    for (int sweep = 0; sweep < max_sweeps && M > 1; ++sweep) {
        ++nsweeps;
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int step = 0; step < P; ++step, ++g) {
            const int cur = g & 1;
            // phase 1: rotations of this step (and their diagonal blocks); V by the previous step's rotations
            if (krot >= 0) {
                const int k = krot;
                int a, b;
                if (k == 0) {
                    a = P; b = step;
                } else {   // (step + k) mod P and (step - k) mod P, with 0 < k < P and 0 <= step < P
                    a = step + k; if (a >= P) a -= P;
                    b = step - k; if (b < 0) b += P;
                }
                const int pi = a < b ? a : b, qi = a < b ? b : a;
                float c = 1.f, s = 0.f;
                if (qi < M) {
                    const float apq = A[pi + qi * ld];
                    const float app = A[pi + pi * ld], aqq = A[qi + qi * ld];
                    if (fabsf(apq) > epsr * sqrtf(fabsf(app * aqq)) && fabsf(apq) > epsa) {
                        const float th = (aqq - app) / (2.f * apq);
                        const float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
                        c = 1.f / sqrtf(t * t + 1.f);
                        s = t * c;
                        A[pi + pi * ld] = app - t * apq;   // the rotated diagonal block: coupling annihilated
                        A[qi + qi * ld] = aqq + t * apq;
                        A[pi + qi * ld] = 0.f;
                        A[qi + pi * ld] = 0.f;
                        s_rot = 1;
                    }
                }
                cs[cur][k] = f2(c, s);
                pinfo[cur][k] = qi < M ? make_int4(pi, qi, pi * ld, qi * ld) : make_int4(pi, -1, pi * ld, 0);
            } else if (warp < nvw && g > 0) {
                update_v(cur ^ 1);
            }
            __syncthreads();
            // phase 2: the off-diagonal blocks
#pragma unroll
            for (int j = 0; j < NBREG; ++j)
                if (ab[j] >= 0) update_block(cs[cur], pinfo[cur], ab[j] & 0xffff, ab[j] >> 16);
            __syncthreads();
        }
        if (!s_rot) break;
        __syncthreads();
    }
    if (g > 0) {   // V by the last step's rotations
        if (warp < nvw) update_v((g - 1) & 1);
        __syncthreads();
    }
    // eigenvalues sorted decreasingly (rank counting)
    for (int i = tid; i < M; i += nt) {
        const double li = sort_key((double)A[i + i * ld]);
        int rk = 0;
        for (int j = 0; j < M; ++j) {
            const double lj = sort_key((double)A[j + j * ld]);
            if (lj > li || (lj == li && j < i)) ++rk;
        }
        ord[rk] = (short)i;
        lam[rk] = li;
    }
    __syncthreads();
    if (tid == 0) {
        const int s = truncation_rule<float>(p, lam, M, rule_trace(p, s_tr), m);
        s_keep = s;
        for (int i = 0; i < M; ++i) evals[i] = lam[i];
        if (prof) {   // algorithmic work: the dense symmetric eigen-decomposition count 9 M^3; Gram in, S out
            prof[2 * PK_EIG] += 9.0 * (double)M * M * M;
            prof[2 * PK_EIG + 1] += (double)sizeof(float) * ((double)M * M + (double)M * s);
            prof[2 * PK_SWEEPS] += nsweeps;
            prof[2 * PK_SWEEPS + 1] += 1.0;
        }
    }
    __syncthreads();
    const int s = s_keep;
    for (int c = 0; c < s; ++c)
        for (int i = tid; i < M; i += nt) S[i + (long long)c * n] = V[i + ord[c] * ldv];
}

// ------------------------------------------------------------------------------------------------------------
// FP32 Grams up to HJ_MAXM: pivoted Cholesky, then one-sided (Hestenes) Jacobi on the Cholesky factor.
//
//  1. G = sum_k l_k l_k^T by the outer-product Cholesky with diagonal pivoting (pivots chosen by index, no
//     row swaps, so L = [l_1 .. l_rc] satisfies G = L L^T in G's own index order), with G held in registers
//     (32 entries per thread).  It stops once the remaining diagonal (the trace of the Schur complement) is
//     at most 1% of this mode's truncation budget, or every remaining pivot is below 1e-9 trace(G): the
//     remainder is then energy the truncation discards anyway, and the truncation rule (trace minus kept
//     eigenvalues) counts it.  The pivoted Cholesky of G = Z Z^T is the column-pivoted QR of Z^T (L = R^T up
//     to the row order), the preconditioning step of Drmac and Veselic's one-sided Jacobi SVD, after which few
//     sweeps are needed.
//  2. One-sided Jacobi makes the columns of L mutually orthogonal by plane rotations from the right:
//     L J = U Sigma, so the normalised columns are eigenvectors of G and their squared norms its
//     eigenvalues; no rotation matrix is accumulated.  Pair (a_p, a_q) with alpha = |a_p|^2, beta = |a_q|^2,
//     gamma = a_p . a_q rotates when gamma^2 > tau^2 alpha beta: zeta = (beta - alpha) / (2 gamma),
//     t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), a_p <- c a_p - s a_q, a_q <- s a_p + c a_q, and the
//     norms follow as alpha - t gamma, beta + t gamma (recomputed exactly at every sweep start).  Sweeps end
//     when none rotates, or after a sweep whose rotations were all below HJ_TAU_LAST (quadratic convergence
//     leaves the next sweep's products near HJ_TAU).
//  3. The columns are the players of a round-robin tournament (circle method, one fixed player) on 8 NWA
//     players, NWA in {2, 4, 8, 16} the fewest warps whose ring holds the rc columns of L: four pair slots per
//     warp, every lane holding four rows of each of its warp's eight columns in registers.  A step computes
//     the four pair products of a warp with one packed butterfly (each lane ends with the full gamma of one
//     slot), rotates in registers, then moves every column but the fixed one to the next position of the
//     ring: inside a warp this is a register move, and only the two columns at a warp's ends cross to the
//     neighbouring warps, through double-buffered shared memory (one barrier per step).
// ------------------------------------------------------------------------------------------------------------
constexpr int HJ_WARPS = 16;
constexpr int HJ_THREADS = 32 * HJ_WARPS;
constexpr int HJ_SLOTS = 4;                                  // pair slots per warp
constexpr int HJ_PLAYERS = 2 * HJ_SLOTS * HJ_WARPS;          // columns of the largest ring (128)
constexpr int HJ_MAXM = 128;                                 // rows: four per lane
static_assert(HJ_PLAYERS == HJ_MAXM, "ring and row layout");

static inline size_t hj_smem_bytes() {
    return ((size_t)HJ_MAXM * HJ_MAXM + (size_t)2 * 2 * HJ_WARPS * HJ_MAXM) * sizeof(float);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

__global__ void __launch_bounds__(HJ_THREADS) hestenes_eig_kernel(RoundPlan* plan, const float* __restrict__ G,
                                                                  float* __restrict__ S, double* evals, int m,
                                                                  int max_sweeps, float tau, double* prof) {
    RoundPlan& p = *plan;
    const int M = p.eM;
    const int n = p.n;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char hj_smem[];
    float* L = reinterpret_cast<float*>(hj_smem);            // factor columns, then the rotated columns; ld 128
    float* X = L + HJ_MAXM * HJ_MAXM;                        // ring exchange [buffer][direction][warp][row]
    __shared__ float dg[HJ_MAXM];
    __shared__ float wbest[HJ_WARPS], wsum[HJ_WARPS];
    __shared__ int wbi[HJ_WARPS];
    __shared__ float xa[2][2][HJ_WARPS];
    __shared__ double lam[HJ_PLAYERS];                        // squared column norms, by column
    __shared__ double lsort[HJ_PLAYERS];                      // the same, decreasing
    __shared__ short ord[HJ_PLAYERS];
    __shared__ int s_keep;
    __shared__ double s_tr;
    if (M <= 0) {
        if (tid == 0) {
            p.s[m] = 0;
            if (m == 0) { p.norm2 = 0; p.budget = 0; }
        }
        return;
    }
    // G in registers: entry (i, j) with j = warp + 16 a, i = lane + 32 b
    float Ar[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int j = warp + 16 * a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = lane + 32 * b;
            Ar[a][b] = (i < M && j < M) ? G[i + (long long)j * M] : 0.f;
        }
    }
    for (int e = tid; e < HJ_MAXM * HJ_MAXM / 4; e += HJ_THREADS)
        reinterpret_cast<float4*>(L)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = tid; i < HJ_MAXM; i += HJ_THREADS) dg[i] = (i < M) ? G[i + (long long)i * M] : -1.f;
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < M; ++i) t += (double)G[i + (long long)i * M];
        s_tr = t;
        if (m == 0) {
            p.norm2 = rule_trace(p, t);
            p.budget = fmax(p.eps * p.eps * p.norm2, p.abs2) / 3.0;
        }
    }
    __syncthreads();
    const float tr = (float)s_tr;
    // ---- 1. pivoted Cholesky, G = sum_k l_k l_k^T, until the Schur complement is negligible for this mode
    const float thr = 1e-9f * tr;
    const float stop_rem = fmaxf(thr, 0.01f * (float)p.budget);
    int rc = 0;
    for (int k = 0; k < M; ++k) {
        {   // the largest remaining diagonal entry (ties: the lowest index) and the remaining trace
            const int i = warp * 8 + (lane & 7);
            float v = lane < 8 ? dg[i] : -2.f;
            float sm = lane < 8 ? fmaxf(dg[i], 0.f) : 0.f;
            int bi = i;
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                const float v2 = __shfl_xor_sync(FULL, v, o);
                const int b2 = __shfl_xor_sync(FULL, bi, o);
                sm += __shfl_xor_sync(FULL, sm, o);
                if (v2 > v || (v2 == v && b2 < bi)) { v = v2; bi = b2; }
            }
            if (lane == 0) { wbest[warp] = v; wbi[warp] = bi; wsum[warp] = sm; }
        }
        __syncthreads();
        float dmax = -2.f, rem = 0.f;
        int piv = 0;
        for (int w = 0; w < HJ_WARPS; ++w) {
            rem += wsum[w];
            if (wbest[w] > dmax) { dmax = wbest[w]; piv = wbi[w]; }
        }
        // the same decision in every thread (a NaN stops the factorisation)
        if (!(dmax > thr) || !(rem > stop_rem)) break;
        const float r = sqrtf(dmax);
        if (warp == (piv & 15)) {   // the warp holding column piv writes l_k = G_k[:, piv] / sqrt(d_piv)
            const int ap = piv >> 4;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float a = 0.f;
#pragma unroll
                for (int q = 0; q < 8; ++q) a = (q == ap) ? Ar[q][b] : a;
                const int i = lane + 32 * b;
                if (i < M) L[i + k * HJ_MAXM] = (i == piv) ? r : a / r;
            }
        }
        __syncthreads();
        const float* lk = L + k * HJ_MAXM;
        float li[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) li[b] = lk[lane + 32 * b];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int j = warp + 16 * a;
            const float lj = lk[j];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int i = lane + 32 * b;
                const float v = (i == piv || j == piv) ? 0.f : fmaf(-li[b], lj, Ar[a][b]);
                Ar[a][b] = v;
                if (i == j && i < M) dg[i] = (i == piv) ? -1.f : v;
            }
        }
        __syncthreads();
        rc = k + 1;
    }
    // ---- 2. one-sided Jacobi on the rc columns of L: a ring of 8 NWA players
    const int NWA = rc <= 16 ? 2 : (rc <= 32 ? 4 : (rc <= 64 ? 8 : 16));
    const int H = HJ_SLOTS * NWA;                  // pair slots; slot k starts with columns k and H + k
    const int P = 2 * H;
    const bool active = warp < NWA;
    float T[HJ_SLOTS][4], B[HJ_SLOTS][4], aT[HJ_SLOTS], aB[HJ_SLOTS];
#pragma unroll
    for (int j = 0; j < HJ_SLOTS; ++j) {
        const int k = HJ_SLOTS * warp + j;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f), b = t;
        if (active) {
            t = ld4(L + k * HJ_MAXM + 4 * lane);
            b = ld4(L + (H + k) * HJ_MAXM + 4 * lane);
        }
        T[j][0] = t.x; T[j][1] = t.y; T[j][2] = t.z; T[j][3] = t.w;
        B[j][0] = b.x; B[j][1] = b.y; B[j][2] = b.z; B[j][3] = b.w;
        aT[j] = 0.f;
        aB[j] = 0.f;
    }
    const int pj = (lane >> 3) & 3;         // the slot whose rotation this lane computes
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
    const float floor_g = 1e-12f * tr;      // products below this are rounding noise of the factor
    const float tau2 = tau * tau;
    const float taul2 = HJ_TAU_LAST * HJ_TAU_LAST;
    int nsweeps = 0, buf = 0;
    for (int sweep = 0; sweep < max_sweeps && rc > 1; ++sweep) {
        ++nsweeps;
#pragma unroll
        for (int j = 0; j < HJ_SLOTS; ++j) {   // exact squared norms
            float st = 0.f, sb = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) { st = fmaf(T[j][q], T[j][q], st); sb = fmaf(B[j][q], B[j][q], sb); }
            aT[j] = warp_sum(st);
            aB[j] = warp_sum(sb);
        }
        int rot = 0, big = 0;
        for (int step = 0; step < P - 1; ++step) {
            if (active) {
                float g[HJ_SLOTS];
#pragma unroll
                for (int j = 0; j < HJ_SLOTS; ++j) {
                    float acc = 0.f;
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc = fmaf(T[j][q], B[j][q], acc);
                    g[j] = acc;
                }
                // packed butterfly: after it, every lane holds the full product of slot pj
                const float x0 = __shfl_xor_sync(FULL, b4 ? g[0] : g[2], 16);
                const float x1 = __shfl_xor_sync(FULL, b4 ? g[1] : g[3], 16);
                const float u0 = (b4 ? g[2] : g[0]) + x0;
                const float u1 = (b4 ? g[3] : g[1]) + x1;
                const float y = __shfl_xor_sync(FULL, b3 ? u0 : u1, 8);
                float gm = (b3 ? u1 : u0) + y;
                gm += __shfl_xor_sync(FULL, gm, 4);
                gm += __shfl_xor_sync(FULL, gm, 2);
                gm += __shfl_xor_sync(FULL, gm, 1);
                const float al = pj == 0 ? aT[0] : pj == 1 ? aT[1] : pj == 2 ? aT[2] : aT[3];
                const float be = pj == 0 ? aB[0] : pj == 1 ? aB[1] : pj == 2 ? aB[2] : aB[3];
                float c = 1.f, s = 0.f, tg = 0.f;
                if (gm * gm > tau2 * al * be && fabsf(gm) > floor_g) {
                    const float zeta = (be - al) * __frcp_rn(2.f * gm);
                    const float t = copysignf(__frcp_rn(fabsf(zeta) + __fsqrt_rn(fmaf(zeta, zeta, 1.f))), zeta);
                    c = __frsqrt_rn(fmaf(t, t, 1.f));
                    s = c * t;
                    tg = t * gm;
                    rot = 1;
                    if (gm * gm > taul2 * al * be) big = 1;
                }
#pragma unroll
                for (int j = 0; j < HJ_SLOTS; ++j) {
                    const float cj = __shfl_sync(FULL, c, 8 * j), sj = __shfl_sync(FULL, s, 8 * j);
                    const float tgj = __shfl_sync(FULL, tg, 8 * j);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float tp = T[j][q], bq = B[j][q];
                        T[j][q] = fmaf(cj, tp, -sj * bq);
                        B[j][q] = fmaf(sj, tp, cj * bq);
                    }
                    aT[j] -= tgj;
                    aB[j] += tgj;
                }
                // ring move: top[k] -> top[k+1] (top[0] fixed), top[H-1] -> bottom[H-1], bottom[k] -> bottom[k-1],
                // bottom[0] -> top[1]; the two columns at a warp's ends go through shared memory
                float* xt = X + ((buf * 2 + 0) * HJ_WARPS) * HJ_MAXM;
                float* xb = X + ((buf * 2 + 1) * HJ_WARPS) * HJ_MAXM;
                if (warp < NWA - 1) {
                    st4(xt + warp * HJ_MAXM + 4 * lane, T[HJ_SLOTS - 1]);
                    if (lane == 0) xa[buf][0][warp] = aT[HJ_SLOTS - 1];
                }
                if (warp > 0) {
                    st4(xb + warp * HJ_MAXM + 4 * lane, B[0]);
                    if (lane == 0) xa[buf][1][warp] = aB[0];
                }
            }
            __syncthreads();
            if (active) {
                const float* xt = X + ((buf * 2 + 0) * HJ_WARPS) * HJ_MAXM;
                const float* xb = X + ((buf * 2 + 1) * HJ_WARPS) * HJ_MAXM;
                float oB0[4], oT3[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) { oB0[q] = B[0][q]; oT3[q] = T[HJ_SLOTS - 1][q]; }
                const float oaB0 = aB[0], oaT3 = aT[HJ_SLOTS - 1];
#pragma unroll
                for (int j = 0; j < HJ_SLOTS - 1; ++j) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) B[j][q] = B[j + 1][q];
                    aB[j] = aB[j + 1];
                }
                if (warp == NWA - 1) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) B[HJ_SLOTS - 1][q] = oT3[q];
                    aB[HJ_SLOTS - 1] = oaT3;
                } else {
                    const float4 v = ld4(xb + (warp + 1) * HJ_MAXM + 4 * lane);
                    B[HJ_SLOTS - 1][0] = v.x; B[HJ_SLOTS - 1][1] = v.y;
                    B[HJ_SLOTS - 1][2] = v.z; B[HJ_SLOTS - 1][3] = v.w;
                    aB[HJ_SLOTS - 1] = xa[buf][1][warp + 1];
                }
#pragma unroll
                for (int j = HJ_SLOTS - 1; j >= 2; --j) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) T[j][q] = T[j - 1][q];
                    aT[j] = aT[j - 1];
                }
                if (warp == 0) {   // top[0] stays; bottom[0] enters the top row at slot 1
#pragma unroll
                    for (int q = 0; q < 4; ++q) T[1][q] = oB0[q];
                    aT[1] = oaB0;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) T[1][q] = T[0][q];
                    aT[1] = aT[0];
                    const float4 v = ld4(xt + (warp - 1) * HJ_MAXM + 4 * lane);
                    T[0][0] = v.x; T[0][1] = v.y; T[0][2] = v.z; T[0][3] = v.w;
                    aT[0] = xa[buf][0][warp - 1];
                }
            }
            buf ^= 1;
        }
        if (!__syncthreads_or(rot)) break;
        if (!__syncthreads_or(big)) break;   // only small rotations this sweep: converged to about HJ_TAU
    }
    // ---- 3. eigenvalues (exact squared norms), decreasing order, truncation rule, normalised kept columns
    __syncthreads();
    float* C = L;   // the rotated columns, ld HJ_MAXM (L is no longer needed)
    if (active) {
#pragma unroll
        for (int j = 0; j < HJ_SLOTS; ++j) {
            const int k = HJ_SLOTS * warp + j;
            st4(C + k * HJ_MAXM + 4 * lane, T[j]);
            st4(C + (H + k) * HJ_MAXM + 4 * lane, B[j]);
            float st = 0.f, sb = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) { st = fmaf(T[j][q], T[j][q], st); sb = fmaf(B[j][q], B[j][q], sb); }
            st = warp_sum(st);
            sb = warp_sum(sb);
            if (lane == 0) { lam[k] = (double)st; lam[H + k] = (double)sb; }
        }
    }
    __syncthreads();
    for (int i = tid; i < HJ_PLAYERS; i += HJ_THREADS) {
        if (i < P) {
            const double li = sort_key(lam[i]);
            int rk = 0;
            for (int j = 0; j < P; ++j) {
                const double lj = sort_key(lam[j]);
                if (lj > li || (lj == li && j < i)) ++rk;
            }
            ord[rk] = (short)i;
            lsort[rk] = lam[i];
        } else {
            lsort[i] = 0.0;   // eigenvalues past the ring: zero (the Cholesky remainder is discarded energy)
        }
    }
    __syncthreads();
    if (tid == 0) {
        int s = truncation_rule<float>(p, lsort, M, rule_trace(p, s_tr), m);
        while (s > 0 && !(lsort[s - 1] > 0.0)) --s;   // a zero column is never kept (its energy is already
        p.s[m] = s;                                   // counted as discarded)
        s_keep = s;
        for (int i = 0; i < M; ++i) evals[i] = lsort[i];
        if (prof) {
            prof[2 * PK_EIG] += 9.0 * (double)M * M * M;
            prof[2 * PK_EIG + 1] += (double)sizeof(float) * ((double)M * M + (double)M * s);
            prof[2 * PK_SWEEPS] += nsweeps;
            prof[2 * PK_SWEEPS + 1] += 1.0;
        }
    }
    __syncthreads();
    const int s = s_keep;
    for (int c = warp; c < s; c += HJ_WARPS) {
        const int col = ord[c];
        const float inv = (float)(1.0 / sqrt(lam[col]));
        for (int i = lane; i < M; i += 32) S[i + (long long)c * n] = C[i + col * HJ_MAXM] * inv;
    }
}

// shared-memory layout: A (M (M+1)) and V (M (M+1)) when both fit, else A only, else neither
static size_t jacobi_smem_plan(int n, size_t elt, int* a_smem, int* v_smem) {
    const size_t limit = 190 * 1024;   // leaves room for the ~20 KB of static shared memory
    const size_t one = (size_t)n * (n + 1) * elt;
    if (2 * one <= limit) { *a_smem = 1; *v_smem = 1; return 2 * one; }
    if (one <= limit) { *a_smem = 1; *v_smem = 0; return one; }
    *a_smem = 0; *v_smem = 0;
    return 0;
}

template <typename T>
int launch_eig(RoundPlan* plan, const T* G, EigWork& w, T* S, double* evals, int m, int n, cudaStream_t st) {
    if (use_cluster_eig<T>(n)) {
        const int Mp = cj_padded(n);
        const size_t bytes = 2 * (size_t)(2 * (Mp / (2 * CJ_C)) + 2) * (Mp + 1) * sizeof(T);
        TPCG_TRY(smem_optin(reinterpret_cast<const void*>(cjacobi_eig_kernel<T>), sizeof(T) == 8 ? 0 : 1, 200 * 1024));
        cjacobi_eig_kernel<T><<<CJ_C, CJ_THREADS, bytes, st>>>(plan, G, S, evals, m, 20, prof_dev());
        TPCG_CHECK_LAUNCH();
        return TPCG_OK;
    }
    if constexpr (sizeof(T) == 4) {
        if (n <= HJ_MAXM && eig_kind() == 1) {   // FP32 Grams up to 128: pivoted Cholesky + one-sided Jacobi
            TPCG_TRY(smem_optin(reinterpret_cast<const void*>(hestenes_eig_kernel), 7, (int)hj_smem_bytes()));
            hestenes_eig_kernel<<<1, HJ_THREADS, hj_smem_bytes(), st>>>(plan, G, S, evals, m, 30, HJ_TAU,
                                                                        prof_dev());
            TPCG_CHECK_LAUNCH();
            return TPCG_OK;
        }
        if (n <= JV_MAXM) {   // FP32 Grams up to 128: packed rotations, vectorised V update
            TPCG_TRY(smem_optin(reinterpret_cast<const void*>(jacobi_eig_v_kernel), 6, 190 * 1024));
            jacobi_eig_v_kernel<<<1, EIG_THREADS, jv_smem_bytes(n), st>>>(plan, G, S, evals, m, 20, prof_dev());
            TPCG_CHECK_LAUNCH();
            return TPCG_OK;
        }
    }
    int a_smem = 0, v_smem = 0;
    const size_t bytes = jacobi_smem_plan(n, sizeof(T), &a_smem, &v_smem);
    T* Aw = reinterpret_cast<T*>(w.Aw);
    T* Vw = reinterpret_cast<T*>(w.Vw);
    if (a_smem && v_smem) {
        TPCG_TRY(smem_optin(reinterpret_cast<const void*>(jacobi_eig_kernel<T, true>), sizeof(T) == 8 ? 4 : 5,
                            190 * 1024));
        jacobi_eig_kernel<T, true><<<1, EIG_THREADS, bytes, st>>>(plan, G, Aw, Vw, S, evals, m, 1, 1, 20,
                                                                 prof_dev());
    } else {
        TPCG_TRY(smem_optin(reinterpret_cast<const void*>(jacobi_eig_kernel<T, false>), sizeof(T) == 8 ? 2 : 3,
                            190 * 1024));
        jacobi_eig_kernel<T, false><<<1, EIG_THREADS, bytes, st>>>(plan, G, Aw, Vw, S, evals, m, a_smem, v_smem, 20,
                                                                  prof_dev());
    }
    TPCG_CHECK_LAUNCH();
    return TPCG_OK;
}
int eig_prepare() {
    TPCG_TRY(smem_optin(reinterpret_cast<const void*>(cjacobi_eig_kernel<double>), 0, 200 * 1024));
    TPCG_TRY(smem_optin(reinterpret_cast<const void*>(cjacobi_eig_kernel<float>), 1, 200 * 1024));
    TPCG_TRY(smem_optin(reinterpret_cast<const void*>(jacobi_eig_kernel<double, false>), 2, 190 * 1024));
    TPCG_TRY(smem_optin(reinterpret_cast<const void*>(jacobi_eig_kernel<float, false>), 3, 190 * 1024));
    TPCG_TRY(smem_optin(reinterpret_cast<const void*>(jacobi_eig_kernel<double, true>), 4, 190 * 1024));
    TPCG_TRY(smem_optin(reinterpret_cast<const void*>(jacobi_eig_kernel<float, true>), 5, 190 * 1024));
    TPCG_TRY(smem_optin(reinterpret_cast<const void*>(jacobi_eig_v_kernel), 6, 190 * 1024));
    TPCG_TRY(smem_optin(reinterpret_cast<const void*>(hestenes_eig_kernel), 7, (int)hj_smem_bytes()));
    return TPCG_OK;
}

template int launch_eig<double>(RoundPlan*, const double*, EigWork&, double*, double*, int, int, cudaStream_t);
template int launch_eig<float>(RoundPlan*, const float*, EigWork&, float*, double*, int, int, cudaStream_t);

size_t eig_work_bytes(int n) { return 2 * (size_t)n * (n + 1) * sizeof(double); }

int eig_work_alloc(EigWork* w, int n, std::vector<void*>* owned) {
    if (n > SMAX_EIG) {
        set_error("eigensolver supports n <= " + std::to_string(SMAX_EIG));
        return TPCG_E_INVALID;
    }
    for (void** p : {&w->Aw, &w->Vw}) {
        if (cudaMalloc(p, (size_t)n * (n + 1) * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            set_error("eig workspace: cudaMalloc failed");
            return TPCG_E_NOMEM;
        }
        owned->push_back(*p);
    }
    return TPCG_OK;
}

}  // namespace tpcg
