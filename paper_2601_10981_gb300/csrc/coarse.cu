// Coarse propagator G in the augmented POD space and the parareal update of
// eq. (formula4), swept over the subintervals in order (Algorithm 2 and the remark after
// it: U^k_{n+1} needs U^k_n).
//
// For V = [R, d] with d~ = U - R R^T U and d = d~ / ||d~|| (eqs. (eqaug), (eq12)), the
// bordered reduced matrices of eq. (eq13) are
// assembled from the level-2 Galerkin blocks R^T R, R^T L R (computed once per
// subinterval by the POD update) and the border terms R^T d~, R^T L d~, (L^T d~)^T R,
// d~^T L d~.  Because G is affine and both G terms of eq. (formula4) use the same space,
//     G(U) - G(P U') = V Phi^Lc Mv^{-1} V^T (U - U'),   Phi = (Mv + dT Lv)^{-1} Mv,
// so the forcing cancels and one reduced propagation of the difference suffices.
//
// The whole sweep is one persistent cooperative launch (one CTA per SM, each owning a
// fixed contiguous range of grid points).  Per subinterval, three grid-wide barriers:
//   A  R^T U, R^T U', U.U
//   C  d~ = U - R (R^T U)                       ; R^T d~, d~.d~, d~.(U - U')
//   D  L d~, L^T d~ at owned points             ; R^T L d~, R^T L^T d~, d~.L d~
//   E  reduced solve, repeated by every CTA on identical inputs (no barrier)
//   F  U^k_{n+1} = F_n + R g + d~ g_d at owned points (read back by the next A)
// Sums over points: per-CTA partials (fixed thread and warp order), then every CTA adds
// the partials of all CTAs in CTA order, so all CTAs hold bit-identical values and the
// result does not depend on scheduling.  Each dot product over the basis is taken by one
// warp per column with coalesced reads of the column.
#include "pr_internal.cuh"

#include <algorithm>
#include <math.h>

namespace pr {

constexpr int CS_THREADS = 256;

// Block-sum nq (<= MAXQ) values, write the chunk partial, and let the last CTA of the
// batch item add the chunk partials in chunk order into out[q].
template <int MAXQ>
__device__ __forceinline__ void chunk_reduce(double (&acc)[MAXQ], int nq, double* part, int chunks,
                                             int c, unsigned* counter, double* const* outs) {
    __shared__ double red[MAXQ * 8];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
        if (q < nq) {
            double v = acc[q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0) red[q * 8 + warp] = v;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += red[q * 8 + w];
        part[(size_t)c * MAXQ + q] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atom_add_acq_rel_u32(counter, 1u) == (unsigned)chunks - 1u);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        double s = 0.0;
        for (int cc = 0; cc < chunks; ++cc) s += part[(size_t)cc * MAXQ + q];
        *outs[q] = s;
    }
    if (threadIdx.x == 0) st_relaxed_u32(counter, 0u);
}

// Small dense solves of iteration 0 (one CTA, FP64), K <= CS_MAXK.
constexpr int CS_MAXK = 33;

// LU with partial pivoting of the K x K matrix A (ld CS_MAXK) in shared memory; piv[K].
__device__ void lu_factor(double* A, int K, int* piv) {
    __shared__ int s_p;
    for (int j = 0; j < K; ++j) {
        if (threadIdx.x == 0) {
            int p = j;
            double best = fabs(A[j * CS_MAXK + j]);
            for (int i = j + 1; i < K; ++i) {
                const double v = fabs(A[i * CS_MAXK + j]);
                if (v > best) { best = v; p = i; }
            }
            piv[j] = p;
            s_p = p;
        }
        __syncthreads();
        const int p = s_p;
        if (p != j) {
            for (int c = threadIdx.x; c < K; c += blockDim.x) {
                const double t = A[j * CS_MAXK + c];
                A[j * CS_MAXK + c] = A[p * CS_MAXK + c];
                A[p * CS_MAXK + c] = t;
            }
        }
        __syncthreads();
        const double piv_v = A[j * CS_MAXK + j];
        for (int i = j + 1 + threadIdx.x; i < K; i += blockDim.x) {
            const double l = (piv_v != 0.0) ? A[i * CS_MAXK + j] / piv_v : 0.0;
            A[i * CS_MAXK + j] = l;
            for (int c = j + 1; c < K; ++c) A[i * CS_MAXK + c] -= l * A[j * CS_MAXK + c];
        }
        __syncthreads();
    }
}

// Solve LU x = b in place for column vector x (ld stride between entries), by one thread.
__device__ void lu_solve_col(const double* A, int K, const int* piv, double* x, int stride) {
    for (int j = 0; j < K; ++j) {
        const int p = piv[j];
        if (p != j) {
            const double t = x[j * stride];
            x[j * stride] = x[p * stride];
            x[p * stride] = t;
        }
    }
    for (int i = 0; i < K; ++i) {
        double s = x[i * stride];
        for (int k = 0; k < i; ++k) s -= A[i * CS_MAXK + k] * x[k * stride];
        x[i * stride] = s;
    }
    for (int i = K - 1; i >= 0; --i) {
        double s = x[i * stride];
        for (int k = i + 1; k < K; ++k) s -= A[i * CS_MAXK + k] * x[k * stride];
        const double d = A[i * CS_MAXK + i];
        x[i * stride] = (d != 0.0) ? s / d : 0.0;
    }
}

// ------------------------------------------------------------------------------------
// Persistent coarse sweep.
constexpr int CSW_THREADS = 512;
constexpr int CSW_WARPS = CSW_THREADS / 32;
constexpr int CSW_MAXM = 32;                  // level-2 dimension supported
constexpr int CSW_MAXK = CSW_MAXM + 1;        // with the augmentation direction
constexpr int CSW_MAXQ = 3 * CSW_MAXM + 3;    // reductions per stage
constexpr int CSW_LDA = 2 * CSW_MAXK + 1;     // [Ac | Mv | b]
constexpr int CSW_MAX_GRID = 1024;

size_t coarse_part_doubles(long long, int) { return (size_t)2 * CSW_MAXQ * CSW_MAX_GRID; }

struct CswShared {
    double RU[CSW_MAXM], RUp[CSW_MAXM], RD[CSW_MAXM], RL[CSW_MAXM], RLt[CSW_MAXM];
    double UU, DD, DdU, DLD;   // DdU = d~ . (U - U')
    // time-dependent flows: R^T D d~, R^T A_q d~ and d~.D d~, d~.A_q d~
    double RPD[CSW_MAXM], RPA0[CSW_MAXM], RPA1[CSW_MAXM];
    double PDD, PDA0, PDA1;
    double c0, c1;
    double red[CSW_WARPS * 3];
    double g[CSW_MAXK];
    double A[CSW_MAXK * CSW_LDA];
    double prow[CSW_LDA];
    double mult[CSW_MAXK];
    double x[CSW_MAXK], y[CSW_MAXK];
    double inv_piv;
    int piv;
};

// Deterministic CTA sum of nq (<= 3) per-thread values; thread 0 writes part[q][cta].
__device__ __forceinline__ void csw_block_sums(const double* v, int nq, CswShared& sh, double* part,
                                               int G) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < nq; ++q) {
        double x = v[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) sh.red[q * CSW_WARPS + warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        double s = 0.0;
        for (int w = 0; w < CSW_WARPS; ++w) s += sh.red[threadIdx.x * CSW_WARPS + w];
        part[(size_t)threadIdx.x * G + blockIdx.x] = s;
    }
}

// Per-CTA partials of R_i . x0 (quantity q0 + i) and, if x1, R_i . x1 (quantity q1 + i)
// over the owned points, one warp per column, four independent chains per lane.
__device__ __forceinline__ void csw_dots(const double* R, long long Ng, int m, const double* x0,
                                         int q0, const double* x1, int q1, long long lo, long long hi,
                                         double* part, int G) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < m; i += CSW_WARPS) {
        const double* r = R + (size_t)i * Ng;
        double s0[4] = {0.0, 0.0, 0.0, 0.0}, s1[4] = {0.0, 0.0, 0.0, 0.0};
        long long p = lo + lane;
        for (; p + 96 < hi; p += 128) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double rv = r[p + 32 * u];
                s0[u] += rv * x0[p + 32 * u];
                if (x1) s1[u] += rv * x1[p + 32 * u];
            }
        }
        for (int u = 0; p < hi; p += 32, ++u) {
            const double rv = r[p];
            s0[u & 3] += rv * x0[p];
            if (x1) s1[u & 3] += rv * x1[p];
        }
        double a0 = (s0[0] + s0[1]) + (s0[2] + s0[3]);
        double a1 = (s1[0] + s1[1]) + (s1[2] + s1[3]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a0 += __shfl_down_sync(0xffffffffu, a0, off);
            a1 += __shfl_down_sync(0xffffffffu, a1, off);
        }
        if (lane == 0) {
            part[(size_t)(q0 + i) * G + blockIdx.x] = a0;
            if (x1) part[(size_t)(q1 + i) * G + blockIdx.x] = a1;
        }
    }
}

// Sum the partials of all CTAs, in CTA order, for quantities 0..nq-1; out(q) receives
// the value.  Every CTA computes the same sums.
template <typename Out>
__device__ __forceinline__ void csw_reduce(const double* part, int nq, int G, Out&& out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; q < nq; q += CSW_WARPS) {
        double s = 0.0;
        for (int c = lane; c < G; c += 32) s += part[(size_t)q * G + c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) out(q, s);
    }
    __syncthreads();
}

// Reduced solve of one subinterval (all threads of the CTA, FP64): Gauss-Jordan with
// partial pivoting on [Ac | Mv | b], Ac = Mv + dT Lv, b = V^T (U - U'), which gives
// T = Ac^{-1} Mv and y = Ac^{-1} b = T Mv^{-1} b; then x = T^{Lc-1} y = Phi^Lc Mv^{-1} b.
__device__ void csw_small(CswShared& sh, const CoarseSweepArgs& a, int m, const double* Mr,
                          const double* Lr) {
    const double nd = sqrt(fmax(sh.DD, 0.0));
    const bool aug = nd > 0.0 && nd > a.aug_tol * sqrt(fmax(sh.UU, 0.0));
    const int K = aug ? m + 1 : m;
    const int nc = 2 * K + 1;
    const double dT = a.dT;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int i = e / K, j = e - i * K;
        double mv, lv;
        if (i < m && j < m) {
            mv = Mr[(size_t)i * a.ldM + j];
            lv = Lr[(size_t)i * a.ldM + j];
        } else if (i < m) {      // column m: R^T d, R^T L d
            mv = sh.RD[i] / nd;
            lv = sh.RL[i] / nd;
        } else if (j < m) {      // row m: d^T R, (L^T d)^T R
            mv = sh.RD[j] / nd;
            lv = sh.RLt[j] / nd;
        } else {
            mv = sh.DD / (nd * nd);
            lv = sh.DLD / (nd * nd);
        }
        sh.A[i * CSW_LDA + j] = mv + dT * lv;
        sh.A[i * CSW_LDA + K + j] = mv;
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        sh.A[i * CSW_LDA + 2 * K] = (i < m) ? sh.RU[i] - sh.RUp[i] : sh.DdU / nd;
    __syncthreads();
    for (int j = 0; j < K; ++j) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            double best = -1.0;
            int bi = j;
            for (int i = j + lane; i < K; i += 32) {
                const double v = fabs(sh.A[i * CSW_LDA + j]);
                if (v > best) { best = v; bi = i; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) {
                sh.piv = bi;
                const double pv = sh.A[bi * CSW_LDA + j];
                sh.inv_piv = (pv != 0.0) ? 1.0 / pv : 0.0;
            }
        }
        __syncthreads();
        const int pr = sh.piv;
        if (pr != j) {
            for (int c = j + threadIdx.x; c < nc; c += blockDim.x) {
                const double t = sh.A[j * CSW_LDA + c];
                sh.A[j * CSW_LDA + c] = sh.A[pr * CSW_LDA + c];
                sh.A[pr * CSW_LDA + c] = t;
            }
        }
        __syncthreads();
        for (int c = j + 1 + threadIdx.x; c < nc; c += blockDim.x) sh.prow[c] = sh.A[j * CSW_LDA + c] * sh.inv_piv;
        for (int i = threadIdx.x; i < K; i += blockDim.x) sh.mult[i] = sh.A[i * CSW_LDA + j];
        __syncthreads();
        const int w = nc - j - 1;
        for (int e = threadIdx.x; e < K * w; e += blockDim.x) {
            const int i = e / w, c = j + 1 + (e - i * w);
            sh.A[i * CSW_LDA + c] = (i == j) ? sh.prow[c] : sh.A[i * CSW_LDA + c] - sh.mult[i] * sh.prow[c];
        }
        __syncthreads();
    }
    // x = y, then Lc - 1 products with T
    for (int i = threadIdx.x; i < K; i += blockDim.x) sh.x[i] = sh.A[i * CSW_LDA + 2 * K];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = 1; l < a.Lc; ++l) {
        for (int i = warp; i < K; i += CSW_WARPS) {
            double s = (lane < K) ? sh.A[i * CSW_LDA + K + lane] * sh.x[lane] : 0.0;
            if (lane + 32 < K) s += sh.A[i * CSW_LDA + K + lane + 32] * sh.x[lane + 32];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) sh.y[i] = s;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += blockDim.x) sh.x[i] = sh.y[i];
        __syncthreads();
    }
    for (int i = threadIdx.x; i <= m; i += blockDim.x) {
        double v = 0.0;
        if (i < m) v = sh.x[i];
        else if (aug) v = sh.x[m] / nd;
        sh.g[i] = v;
    }
    __syncthreads();
}

// Gauss-Jordan with partial pivoting on the K x nc matrix sh.A (columns K.. are
// right-hand sides); afterwards those columns hold Ac^{-1} times them.
__device__ void csw_gauss_jordan(CswShared& sh, int K, int nc) {
    for (int j = 0; j < K; ++j) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            double best = -1.0;
            int bi = j;
            for (int i = j + lane; i < K; i += 32) {
                const double v = fabs(sh.A[i * CSW_LDA + j]);
                if (v > best) { best = v; bi = i; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) {
                sh.piv = bi;
                const double pv = sh.A[bi * CSW_LDA + j];
                sh.inv_piv = (pv != 0.0) ? 1.0 / pv : 0.0;
            }
        }
        __syncthreads();
        const int pr = sh.piv;
        if (pr != j) {
            for (int c = j + threadIdx.x; c < nc; c += blockDim.x) {
                const double t = sh.A[j * CSW_LDA + c];
                sh.A[j * CSW_LDA + c] = sh.A[pr * CSW_LDA + c];
                sh.A[pr * CSW_LDA + c] = t;
            }
        }
        __syncthreads();
        for (int c = j + 1 + threadIdx.x; c < nc; c += blockDim.x) sh.prow[c] = sh.A[j * CSW_LDA + c] * sh.inv_piv;
        for (int i = threadIdx.x; i < K; i += blockDim.x) sh.mult[i] = sh.A[i * CSW_LDA + j];
        __syncthreads();
        const int w = nc - j - 1;
        for (int e = threadIdx.x; e < K * w; e += blockDim.x) {
            const int i = e / w, c = j + 1 + (e - i * w);
            sh.A[i * CSW_LDA + c] = (i == j) ? sh.prow[c] : sh.A[i * CSW_LDA + c] - sh.mult[i] * sh.prow[c];
        }
        __syncthreads();
    }
}

// Reduced propagation for a time-dependent flow: the matrices change with the coarse
// time, so each of the Lc steps solves (Mv + dT Lv(t_l)) x_l = Mv x_{l-1}, started from
// x_1 = Ac(t_1)^{-1} b, b = V^T (U - U') (the same vector as Phi_1 Mv^{-1} b).
__device__ void csw_small_tdep(CswShared& sh, const CoarseSweepArgs& a, int m, const double* Mr,
                               const double* Lr, double t_n) {
    const double nd = sqrt(fmax(sh.DD, 0.0));
    const bool aug = a.augment && nd > 0.0 && nd > a.aug_tol * sqrt(fmax(sh.UU, 0.0));
    const int K = aug ? m + 1 : m;
    const double dT = a.dT;
    const long long PL = (long long)a.ldM * a.ldM;
    // Mv in the x slot area: keep it in sh.y? use the RHS column for b, Mv read from Mr
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        sh.x[i] = (i < m) ? sh.RU[i] - sh.RUp[i] : sh.DdU / nd;
    __syncthreads();
    auto mv = [&](int i, int j) -> double {
        if (i < m && j < m) return Mr[(size_t)i * a.ldM + j];
        if (i < m) return sh.RD[i] / nd;
        if (j < m) return sh.RD[j] / nd;
        return sh.DD / (nd * nd);
    };
    for (int l = 1; l <= a.Lc; ++l) {
        if (threadIdx.x == 0) {
            double q0, q1;
            flow_coeffs(a.kind, a.w, t_n + l * dT, q0, q1);
            sh.c0 = q0;
            sh.c1 = q1;
        }
        __syncthreads();
        const double q0 = sh.c0, q1 = sh.c1;
        for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
            const int i = e / K, j = e - i * K;
            double lv;
            if (i < m && j < m) {
                const size_t o = (size_t)i * a.ldM + j;
                lv = Lr[o] + q0 * Lr[PL + o] + q1 * Lr[2 * PL + o];
            } else if (i < m) {     // column m: R^T L d
                lv = (sh.RPD[i] + q0 * sh.RPA0[i] + q1 * sh.RPA1[i]) / nd;
            } else if (j < m) {     // row m: (L^T d)^T R, advection pieces antisymmetric
                lv = (sh.RPD[j] - q0 * sh.RPA0[j] - q1 * sh.RPA1[j]) / nd;
            } else {
                lv = (sh.PDD + q0 * sh.PDA0 + q1 * sh.PDA1) / (nd * nd);
            }
            sh.A[i * CSW_LDA + j] = mv(i, j) + dT * lv;
        }
        // right-hand side: b at the first step, then Mv x
        for (int i = threadIdx.x; i < K; i += blockDim.x) {
            double r;
            if (l == 1) r = sh.x[i];
            else {
                r = 0.0;
                for (int j = 0; j < K; ++j) r += mv(i, j) * sh.x[j];
            }
            sh.A[i * CSW_LDA + K] = r;
        }
        __syncthreads();
        csw_gauss_jordan(sh, K, K + 1);
        for (int i = threadIdx.x; i < K; i += blockDim.x) sh.x[i] = sh.A[i * CSW_LDA + K];
        __syncthreads();
    }
    for (int i = threadIdx.x; i <= m; i += blockDim.x) {
        double v = 0.0;
        if (i < m) v = sh.x[i];
        else if (aug) v = sh.x[m] / nd;
        sh.g[i] = v;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CSW_THREADS, 1) coarse_sweep_kernel(CoarseSweepArgs a) {
    __shared__ CswShared sh;
    const int G = gridDim.x;
    const long long Ng = a.g.Ng;
    const long long CH = (Ng + G - 1) / G;
    const long long lo = min(Ng, (long long)blockIdx.x * CH), hi = min(Ng, lo + CH);
    int buf = 0;
    auto part = [&]() { return a.part + (size_t)buf * CSW_MAXQ * G; };
    auto barrier = [&]() -> bool { return group_barrier(a.bar, (unsigned)G, a.spin_limit, a.err); };
    const int n_ = a.g.n;
    const long long n2 = (long long)n_ * n_;
    const int n2i = n_ * n_;
    const double inv2h = 0.5 / a.g.h, epsh2 = a.g.eps / (a.g.h * a.g.h);

    for (int t = 0; t < a.count; ++t) {
        const long long n = a.n0 + t;
        const double* U = a.U + n * a.sU;
        const double* Up = a.Up + n * a.sUp;
        const double* F = a.F + n * a.sF;
        double* out = a.out + n * a.sOut;
        const double* R = a.R + n * a.sR;
        const double* Mr = a.Mr + n * a.sM;
        const double* Lr = a.Lr + n * a.sML;
        const double t_n = a.t0 + n * a.DeltaT;
        int m = a.m[n * a.sm];
        if (m > a.maxm || m < 0) {
            if (threadIdx.x == 0) record_error(a.err, DERR_BREAKDOWN);
            m = max(0, min(m, a.maxm));
        }
        // ---- A: R^T U, R^T U', U.U
        {
            double v[1] = {0.0};
            for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) v[0] += U[p] * U[p];
            csw_block_sums(v, 1, sh, part() + (size_t)(2 * m) * G, G);
            csw_dots(R, Ng, m, U, 0, Up, m, lo, hi, part(), G);
            if (!barrier()) return;
            csw_reduce(part(), 2 * m + 1, G, [&](int q, double s) {
                if (q < m) sh.RU[q] = s;
                else if (q < 2 * m) sh.RUp[q - m] = s;
                else sh.UU = s;
            });
            buf ^= 1;
        }
        if (!a.augment) {
            // plain coarse space: no augmentation direction
            if (threadIdx.x == 0) {
                sh.DD = 0.0;
                sh.DdU = 0.0;
                sh.DLD = 0.0;
            }
            __syncthreads();
            if (a.tdep) csw_small_tdep(sh, a, m, Mr, Lr, t_n);
            else csw_small(sh, a, m, Mr, Lr);
            for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                double s = F[p];
                for (int i = 0; i < m; ++i) s += R[(size_t)i * Ng + p] * sh.g[i];
                out[p] = s;
            }
            continue;
        }
        // ---- C: d~ = U - R (R^T U) ; R^T d~, d~.d~, d~.(U - U').  One projection: the
        //         Galerkin space span{R, d~} = span{R, U} does not depend on how much of R
        //         is taken out of U, and the mass-matrix column R^T d~ carries whatever
        //         rounding leaves in span R (at most ~eps ||U|| / ||d~|| of d~ / ||d~||).
        {
            double v[2] = {0.0, 0.0};
            for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
                const double u = U[p];
                double d = u;
                for (int i = 0; i < m; ++i) d -= sh.RU[i] * R[(size_t)i * Ng + p];
                a.d[p] = d;
                v[0] += d * d;
                v[1] += d * (u - Up[p]);
            }
            csw_block_sums(v, 2, sh, part() + (size_t)m * G, G);
            __syncthreads();
            csw_dots(R, Ng, m, a.d, 0, nullptr, 0, lo, hi, part(), G);
            if (!barrier()) return;
            csw_reduce(part(), m + 2, G, [&](int q, double s) {
                if (q < m) sh.RD[q] = s;
                else if (q == m) sh.DD = s;
                else sh.DdU = s;
            });
            buf ^= 1;
        }
        // ---- D: L d~, L^T d~ (an analytic b_d does not depend on x_d, so L^T flips the
        //         advection; a stored perturbation is read at the neighbours) ;
        //         R^T L d~, R^T L^T d~, d~.L d~.  Time-dependent flows: the pieces D d~,
        //         A0 d~, A1 d~ and their projections instead, combined per coarse step.
        if (a.tdep) {
            const double* tab0 = a.g.tab;
            const double* tab1 = a.g.tab + (size_t)TAB_B1 * n_;
            const double* d = a.d;
            double v[3] = {0.0, 0.0, 0.0};
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                // 32-bit index arithmetic (n^3 < 2^31): 64-bit division costs ~70 instructions
                const int i32 = (int)i, z = i32 / n2i, rz = i32 - z * n2i, y = rz / n_, x = rz - y * n_;
                const long long base = i - x, rowb = i - (long long)y * n_, plb = i - (long long)z * n2;
                const double uc = d[i];
                const double uxp = d[base + (x + 1 == n_ ? 0 : x + 1)], uxm = d[base + (x == 0 ? n_ - 1 : x - 1)];
                const double uyp = d[rowb + (long long)(y + 1 == n_ ? 0 : y + 1) * n_];
                const double uym = d[rowb + (long long)(y == 0 ? n_ - 1 : y - 1) * n_];
                const double uzp = d[plb + (long long)(z + 1 == n_ ? 0 : z + 1) * n2];
                const double uzm = d[plb + (long long)(z == 0 ? n_ - 1 : z - 1) * n2];
                const double dx = uxp - uxm, dy = uyp - uym, dz = uzp - uzm;
                const double pd = -epsh2 * ((uxp + uxm) + (uyp + uym) + (uzp + uzm) - 6.0 * uc);
                const double a0 = ((tab0[TXY * n_ + y] + tab0[TXZ * n_ + z]) * dx +
                                   (tab0[TYX * n_ + x] + tab0[TYZ * n_ + z]) * dy +
                                   (tab0[TZX * n_ + x] + tab0[TZY * n_ + y]) * dz) * inv2h;
                const double a1 = ((tab1[TXY * n_ + y] + tab1[TXZ * n_ + z]) * dx +
                                   (tab1[TYX * n_ + x] + tab1[TYZ * n_ + z]) * dy +
                                   (tab1[TZX * n_ + x] + tab1[TZY * n_ + y]) * dz) * inv2h;
                a.Ld[i] = pd;
                a.Ltd[i] = a0;
                a.A1d[i] = a1;
                v[0] += uc * pd;
                v[1] += uc * a0;
                v[2] += uc * a1;
            }
            csw_block_sums(v, 3, sh, part() + (size_t)(3 * m) * G, G);
            __syncthreads();
            csw_dots(R, Ng, m, a.Ld, 0, a.Ltd, m, lo, hi, part(), G);
            csw_dots(R, Ng, m, a.A1d, 2 * m, nullptr, 0, lo, hi, part(), G);
            if (!barrier()) return;
            csw_reduce(part(), 3 * m + 3, G, [&](int q, double s) {
                if (q < m) sh.RPD[q] = s;
                else if (q < 2 * m) sh.RPA0[q - m] = s;
                else if (q < 3 * m) sh.RPA1[q - 2 * m] = s;
                else if (q == 3 * m) sh.PDD = s;
                else if (q == 3 * m + 1) sh.PDA0 = s;
                else sh.PDA1 = s;
            });
            buf ^= 1;
        } else
        {
            const double* tab = a.g.tab;
            const double* d = a.d;
            double v[1] = {0.0};
            for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                // 32-bit index arithmetic (n^3 < 2^31): 64-bit division costs ~70 instructions
                const int i32 = (int)i, z = i32 / n2i, rz = i32 - z * n2i, y = rz / n_, x = rz - y * n_;
                const long long base = i - x, rowb = i - (long long)y * n_, plb = i - (long long)z * n2;
                const double uc = d[i];
                const double uxp = d[base + (x + 1 == n_ ? 0 : x + 1)], uxm = d[base + (x == 0 ? n_ - 1 : x - 1)];
                const double uyp = d[rowb + (long long)(y + 1 == n_ ? 0 : y + 1) * n_];
                const double uym = d[rowb + (long long)(y == 0 ? n_ - 1 : y - 1) * n_];
                const double uzp = d[plb + (long long)(z + 1 == n_ ? 0 : z + 1) * n2];
                const double uzm = d[plb + (long long)(z == 0 ? n_ - 1 : z - 1) * n2];
                const double bx = tab[TXY * n_ + y] + tab[TXZ * n_ + z];
                const double by = tab[TYX * n_ + x] + tab[TYZ * n_ + z];
                const double bz = tab[TZX * n_ + x] + tab[TZY * n_ + y];
                const double dif = epsh2 * ((uxp + uxm) + (uyp + uym) + (uzp + uzm) - 6.0 * uc);
                double adv, advt;   // (b . grad d)_i and the advection part of (L^T d)_i
                if (!a.g.pert) {
                    adv = (bx * (uxp - uxm) + by * (uyp - uym) + bz * (uzp - uzm)) * inv2h;
                    advt = -adv;
                } else {
                    // a stored perturbation varies along every axis: column i of the
                    // advection matrix holds +B_d(x_{i-e_d})/(2h) and -B_d(x_{i+e_d})/(2h)
                    const double* P = a.g.pert;
                    const long long ixp = base + (x + 1 == n_ ? 0 : x + 1), ixm = base + (x == 0 ? n_ - 1 : x - 1);
                    const long long iyp = rowb + (long long)(y + 1 == n_ ? 0 : y + 1) * n_;
                    const long long iym = rowb + (long long)(y == 0 ? n_ - 1 : y - 1) * n_;
                    const long long izp = plb + (long long)(z + 1 == n_ ? 0 : z + 1) * n2;
                    const long long izm = plb + (long long)(z == 0 ? n_ - 1 : z - 1) * n2;
                    adv = ((bx + P[i]) * (uxp - uxm) + (by + P[Ng + i]) * (uyp - uym) +
                           (bz + P[2 * Ng + i]) * (uzp - uzm)) * inv2h;
                    advt = (((bx + P[ixm]) * uxm - (bx + P[ixp]) * uxp) +
                            ((by + P[Ng + iym]) * uym - (by + P[Ng + iyp]) * uyp) +
                            ((bz + P[2 * Ng + izm]) * uzm - (bz + P[2 * Ng + izp]) * uzp)) * inv2h;
                }
                const double Ld = adv - dif;
                a.Ld[i] = Ld;
                a.Ltd[i] = advt - dif;
                v[0] += uc * Ld;
            }
            csw_block_sums(v, 1, sh, part() + (size_t)(2 * m) * G, G);
            __syncthreads();
            csw_dots(R, Ng, m, a.Ld, 0, a.Ltd, m, lo, hi, part(), G);
            if (!barrier()) return;
            csw_reduce(part(), 2 * m + 1, G, [&](int q, double s) {
                if (q < m) sh.RL[q] = s;
                else if (q < 2 * m) sh.RLt[q - m] = s;
                else sh.DLD = s;
            });
            buf ^= 1;
        }
        // ---- E: reduced solve ; F: U^k_{n+1} = F_n + R g + d~ g_d
        if (a.tdep) csw_small_tdep(sh, a, m, Mr, Lr, t_n);
        else csw_small(sh, a, m, Mr, Lr);
        for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
            double s = F[p] + a.d[p] * sh.g[m];
            for (int i = 0; i < m; ++i) s += R[(size_t)i * Ng + p] * sh.g[i];
            out[p] = s;
        }
        // out is read back at the same points by the same threads (next stage A) and by
        // other threads of this CTA only after the __syncthreads in csw_block_sums
    }
}

int coarse_sweep_grid() {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, coarse_sweep_kernel, CSW_THREADS, 0);
    return std::min(CSW_MAX_GRID, std::max(1, std::min(occ, 1) * sms));
}

int coarse_max_m() { return CSW_MAXM; }

cudaError_t launch_coarse_sweep(CoarseSweepArgs a, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    if (a.maxm > CSW_MAXM) return cudaErrorInvalidValue;
    const int grid = coarse_sweep_grid();
    void* args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)coarse_sweep_kernel, dim3(grid), dim3(CSW_THREADS),
                                                args, 0, st);
    ++g_launch_count;
    return e;
}

// ------------------------------------------------------------------------------------
// Iteration 0 in reduced coordinates: beta_0 = M0^{-1} p0, then N*Lc implicit Euler
// steps (M0 + dT L0) beta_l = M0 beta_{l-1} + dT q0; beta at the end of subinterval n is
// stored in beta[n*ldb .. ] (n = 0..N-1 gives U^0_{n+1}).
__global__ void g0_kernel(const double* M0, const double* L0, const double* p0, const double* q0,
                          const int* m0p, int ld, int N, int Lc, double dT, double* beta, int ldb,
                          int* err, G0Tdep td) {
    __shared__ double Mv[CS_MAXK * CS_MAXK];
    __shared__ double Ac[CS_MAXK * CS_MAXK];
    __shared__ double T[CS_MAXK * CS_MAXK];
    __shared__ double w[CS_MAXK], x[CS_MAXK], y[CS_MAXK];
    __shared__ int piv[CS_MAXK];
    __shared__ double s_c[2];
    const int K = *m0p;
    if (K <= 0 || K > CS_MAXK) {
        if (K > CS_MAXK && threadIdx.x == 0) record_error(err, DERR_BREAKDOWN);
        return;
    }
    if (td.tdep) {
        // L(t) = D + c0(t) A0 + c1(t) A1 and f(t) = f + c0(t) g0 + c1(t) g1: assemble and
        // factor at every coarse time t = T0 + l dT
        const size_t PL = (size_t)ld * ld;
        for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
            const int i = e / K, j = e - i * K;
            Mv[i * CS_MAXK + j] = M0[(size_t)i * ld + j];
            T[i * CS_MAXK + j] = M0[(size_t)i * ld + j];   // Mv, kept for the right-hand side
        }
        for (int i = threadIdx.x; i < K; i += blockDim.x) x[i] = p0[i];
        __syncthreads();
        lu_factor(Mv, K, piv);
        if (threadIdx.x == 0) lu_solve_col(Mv, K, piv, x, 1);   // beta_0 = M0^{-1} V0^T u_hat0
        __syncthreads();
        for (int n = 0; n < N; ++n) {
            for (int l = 1; l <= Lc; ++l) {
                if (threadIdx.x == 0) {
                    double c0, c1;
                    flow_coeffs(td.kind, td.w, td.T0 + ((double)n * Lc + l) * dT, c0, c1);
                    s_c[0] = c0;
                    s_c[1] = c1;
                }
                __syncthreads();
                const double c0 = s_c[0], c1 = s_c[1];
                for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
                    const int i = e / K, j = e - i * K;
                    const size_t o = (size_t)i * ld + j;
                    Ac[i * CS_MAXK + j] = T[i * CS_MAXK + j] + dT * (L0[o] + c0 * L0[PL + o] + c1 * L0[2 * PL + o]);
                }
                for (int i = threadIdx.x; i < K; i += blockDim.x) {
                    double r = dT * ((q0 ? q0[i] : 0.0) + c0 * td.qg[i] + c1 * td.qg[ld + i]);
                    for (int j = 0; j < K; ++j) r += T[i * CS_MAXK + j] * x[j];
                    y[i] = r;
                }
                __syncthreads();
                lu_factor(Ac, K, piv);
                if (threadIdx.x == 0) lu_solve_col(Ac, K, piv, y, 1);
                __syncthreads();
                for (int i = threadIdx.x; i < K; i += blockDim.x) x[i] = y[i];
                __syncthreads();
            }
            for (int i = threadIdx.x; i < K; i += blockDim.x) beta[(size_t)n * ldb + i] = x[i];
        }
        return;
    }
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int i = e / K, j = e - i * K;
        Mv[i * CS_MAXK + j] = M0[(size_t)i * ld + j];
        Ac[i * CS_MAXK + j] = M0[(size_t)i * ld + j] + dT * L0[(size_t)i * ld + j];
        T[i * CS_MAXK + j] = M0[(size_t)i * ld + j];
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        w[i] = q0 ? dT * q0[i] : 0.0;
        x[i] = p0[i];
    }
    __syncthreads();
    lu_factor(Ac, K, piv);
    for (int c = threadIdx.x; c <= K; c += blockDim.x) {
        if (c < K) lu_solve_col(Ac, K, piv, T + c, CS_MAXK);
        else lu_solve_col(Ac, K, piv, w, 1);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int i = e / K, j = e - i * K;
        Ac[i * CS_MAXK + j] = Mv[i * CS_MAXK + j];
    }
    __syncthreads();
    lu_factor(Ac, K, piv);
    if (threadIdx.x == 0) lu_solve_col(Ac, K, piv, x, 1);
    __syncthreads();
    for (int n = 0; n < N; ++n) {
        for (int l = 0; l < Lc; ++l) {
            for (int i = threadIdx.x; i < K; i += blockDim.x) {
                double s = w[i];
                for (int j = 0; j < K; ++j) s += T[i * CS_MAXK + j] * x[j];
                y[i] = s;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < K; i += blockDim.x) x[i] = y[i];
            __syncthreads();
        }
        for (int i = threadIdx.x; i < K; i += blockDim.x) beta[(size_t)n * ldb + i] = x[i];
    }
}

cudaError_t launch_g0(const double* M0, const double* L0, const double* p0, const double* q0,
                      const int* m0, int ld, int N, int Lc, double dT, double* beta, int ldb,
                      int* err, const G0Tdep& td, cudaStream_t st) {
    g0_kernel<<<1, 128, 0, st>>>(M0, L0, p0, q0, m0, ld, N, Lc, dT, beta, ldb, err, td);
    ++g_launch_count;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(CS_THREADS) norms_kernel(const double* A, const double* Bv,
                                                          const double* Rf, long long Ng, long long CH,
                                                          int chunks, double* part, unsigned* counter,
                                                          double* out) {
    const int n = blockIdx.y, c = blockIdx.x;
    const double* a = A + (size_t)n * Ng;
    const double* b = Bv + (size_t)n * Ng;
    const double* r = Rf ? Rf + (size_t)n * Ng : nullptr;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long p_lo = (long long)c * CH, p_hi = min(Ng, p_lo + CH);
    for (long long p = p_lo + threadIdx.x; p < p_hi; p += blockDim.x) {
        const double av = a[p];
        const double d = av - b[p];
        acc[0] += d * d;
        acc[1] += av * av;
        if (r) {
            const double rv = r[p];
            acc[2] += (av - rv) * (av - rv);
            acc[3] += rv * rv;
        }
    }
    double* outs[4] = {out + 4 * n, out + 4 * n + 1, out + 4 * n + 2, out + 4 * n + 3};
    chunk_reduce<4>(acc, 4, part + (size_t)n * chunks * 4, chunks, c, counter + n, outs);
}

size_t norms_part_doubles(long long Ng, int cnt) { return (size_t)gram_chunks(Ng) * 4 * cnt; }

cudaError_t launch_norms(const double* a, const double* b, const double* r, long long Ng, int cnt,
                         double* part, unsigned* counter, double* out, cudaStream_t st) {
    if (cnt <= 0) return cudaSuccess;
    const int chunks = gram_chunks(Ng);
    const long long CH = (Ng + chunks - 1) / chunks;
    norms_kernel<<<dim3(chunks, cnt), CS_THREADS, 0, st>>>(a, b, r, Ng, CH, chunks, part, counter, out);
    ++g_launch_count;
    return cudaGetLastError();
}

__global__ void nonfinite_kernel(const double* x, long long count, int* flag) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        if (!isfinite(x[i])) { atomicOr(flag, 1); return; }
    }
}

cudaError_t launch_nonfinite(const double* x, long long count, int* flag, cudaStream_t st) {
    nonfinite_kernel<<<608, 256, 0, st>>>(x, count, flag);
    ++g_launch_count;
    return cudaGetLastError();
}

} // namespace pr
