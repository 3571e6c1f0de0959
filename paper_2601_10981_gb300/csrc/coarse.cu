// Coarse propagator G in the augmented POD space and the parareal update of
// eq. (formula4), for one subinterval at a time (the sweep over n is sequential,
// Algorithm 2 and the remark after it).
//
// For V = [R, d] with d~ = U - R R^T U orthogonalised once more against R and
// d = d~ / ||d~|| (eqs. (eqaug), (eq12)), the bordered reduced matrices of eq. (eq13) are
// assembled from the level-2 Galerkin blocks R^T R, R^T L R (computed once per
// subinterval by the POD update) and the border terms R^T d~, R^T L d~, (L^T d~)^T R,
// d~^T L d~.  Because G is affine and both G terms of eq. (formula4) use the same space,
//     G(U) - G(P U') = V Phi^Lc Mv^{-1} V^T (U - U'),   Phi = (Mv + dT Lv)^{-1} Mv,
// so the forcing cancels and one reduced propagation of the difference suffices.
//
// Passes over the grid (each a kernel; reductions are chunk partials summed in chunk
// order by the last CTA, so results do not depend on scheduling):
//   1  gram:     R^T U, R^T U'
//   2  resid:    d~ = U - R c                       ; R^T d~, U.U
//   3  reorth:   d~ -= R c2                         ; R^T d~, d~.d~, d~.U, d~.U'
//   4  Ld:       L d~, L^T d~                       ; d~.L d~
//   5  gram:     R^T L d~, R^T L^T d~
//   6  small:    reduced solve (one CTA, FP64)
//   7  update:   U^k_{n+1} = F_n + R g + d~ g_d
#include "pr_internal.cuh"

#include <algorithm>
#include <math.h>

namespace pr {

constexpr int CS_THREADS = 256;
constexpr int CS_MAXQ = 36;   // m + 3 <= 36  ->  level-2 dimension <= 33 in the coarse sweep

// Offsets into the `dots` scratch (doubles).  maxm = largest level-2 dimension.
struct DotsLayout {
    int RU, RL, RD, RD2, UU, DD, DU, DUp, DLD, total;
    __host__ __device__ DotsLayout(int maxm) {
        RU = 0;                   // [maxm][2]: R^T U, R^T U'
        RL = RU + 2 * maxm;       // [maxm][2]: R^T L d~, R^T L^T d~
        RD = RL + 2 * maxm;       // [maxm]:    R^T d~ (first pass)
        RD2 = RD + maxm;          // [maxm]:    R^T d~ (after re-orthogonalisation)
        UU = RD2 + maxm;
        DD = UU + 1;
        DU = DD + 1;
        DUp = DU + 1;
        DLD = DUp + 1;
        total = DLD + 1;
    }
};

size_t coarse_part_doubles(long long Ng, int maxm) {
    return (size_t)gram_chunks(Ng) * (size_t)std::max(CS_MAXQ, 2 * maxm + 2) + 64;
}

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

// Pointer/count descriptors for the two gram passes, written on the device so that the
// level-2 dimension m can stay on the device.
struct CsDesc {
    const void* colsR[64];
    const void* colsUU[2];
    const void* colsL[2];
    int m;
    int two;
};

__global__ void cs_prepare_kernel(CsDesc* desc, const void* R, const int* m_ptr, int maxm,
                                  long long Ng, int esize, const double* U, const double* Up,
                                  const double* Ld, const double* Ltd) {
    if (threadIdx.x != 0) return;
    const int m = min(*m_ptr, maxm);
    for (int i = 0; i < m; ++i) desc->colsR[i] = reinterpret_cast<const char*>(R) + (size_t)i * Ng * esize;
    desc->colsUU[0] = U;
    desc->colsUU[1] = Up;
    desc->colsL[0] = Ld;
    desc->colsL[1] = Ltd;
    desc->m = m;
    desc->two = 2;
}

template <typename KT>
__global__ void __launch_bounds__(CS_THREADS) cs_resid_kernel(CoarseArgs a, const CsDesc* desc,
                                                              long long CH, int chunks) {
    const int m = desc->m;
    const DotsLayout L(a.maxm);
    const double* c = a.dots + L.RU;  // [i*2 + 0] = R^T U
    __shared__ double sc[CS_MAXQ];
    for (int i = threadIdx.x; i < m; i += blockDim.x) sc[i] = c[2 * i];
    __syncthreads();
    const KT* R = reinterpret_cast<const KT*>(a.R);
    double acc[CS_MAXQ];
#pragma unroll
    for (int q = 0; q < CS_MAXQ; ++q) acc[q] = 0.0;
    double uu = 0.0;
    const long long p_lo = (long long)blockIdx.x * CH, p_hi = min(a.g.Ng, p_lo + CH);
    for (long long p = p_lo + threadIdx.x; p < p_hi; p += blockDim.x) {
        const double u = a.U[p];
        double rv[CS_MAXQ];
        double d = u;
#pragma unroll
        for (int i = 0; i < CS_MAXQ - 3; ++i) {
            if (i < m) {
                rv[i] = (double)R[(size_t)i * a.g.Ng + p];
                d -= rv[i] * sc[i];
            }
        }
        a.d[p] = d;
#pragma unroll
        for (int i = 0; i < CS_MAXQ - 3; ++i)
            if (i < m) acc[i] += rv[i] * d;
        uu += u * u;
    }
    // outputs: R^T d~ -> RD[0..m), U.U -> UU (slot m)
#pragma unroll
    for (int q = 0; q < CS_MAXQ; ++q)
        if (q == m) acc[q] = uu;
    double* outs[CS_MAXQ];
    for (int i = 0; i < CS_MAXQ; ++i) outs[i] = a.dots + L.RD + min(i, a.maxm - 1);
    outs[m] = a.dots + L.UU;
    chunk_reduce<CS_MAXQ>(acc, m + 1, a.part, chunks, blockIdx.x, a.counter + 0, outs);
}

template <typename KT>
__global__ void __launch_bounds__(CS_THREADS) cs_reorth_kernel(CoarseArgs a, const CsDesc* desc,
                                                               long long CH, int chunks) {
    const int m = desc->m;
    const DotsLayout L(a.maxm);
    __shared__ double sc[CS_MAXQ];
    for (int i = threadIdx.x; i < m; i += blockDim.x) sc[i] = a.dots[L.RD + i];
    __syncthreads();
    const KT* R = reinterpret_cast<const KT*>(a.R);
    double acc[CS_MAXQ];
#pragma unroll
    for (int q = 0; q < CS_MAXQ; ++q) acc[q] = 0.0;
    double dd = 0.0, du = 0.0, dup = 0.0;
    const long long p_lo = (long long)blockIdx.x * CH, p_hi = min(a.g.Ng, p_lo + CH);
    for (long long p = p_lo + threadIdx.x; p < p_hi; p += blockDim.x) {
        double rv[CS_MAXQ];
        double d = a.d[p];
#pragma unroll
        for (int i = 0; i < CS_MAXQ - 3; ++i) {
            if (i < m) {
                rv[i] = (double)R[(size_t)i * a.g.Ng + p];
                d -= rv[i] * sc[i];
            }
        }
        a.d[p] = d;
#pragma unroll
        for (int i = 0; i < CS_MAXQ - 3; ++i)
            if (i < m) acc[i] += rv[i] * d;
        dd += d * d;
        du += d * a.U[p];
        dup += d * a.Up[p];
    }
#pragma unroll
    for (int q = 0; q < CS_MAXQ; ++q) {
        if (q == m) acc[q] = dd;
        if (q == m + 1) acc[q] = du;
        if (q == m + 2) acc[q] = dup;
    }
    double* outs[CS_MAXQ];
    for (int i = 0; i < CS_MAXQ; ++i) outs[i] = a.dots + L.RD2 + min(i, a.maxm - 1);
    outs[m] = a.dots + L.DD;
    outs[m + 1] = a.dots + L.DU;
    outs[m + 2] = a.dots + L.DUp;
    chunk_reduce<CS_MAXQ>(acc, m + 3, a.part, chunks, blockIdx.x, a.counter + 1, outs);
}

// L d~ and L^T d~ (b_d independent of x_d: L^T flips the advection sign), and d~.L d~.
__global__ void __launch_bounds__(CS_THREADS) cs_Ld_kernel(CoarseArgs a, long long CH, int chunks) {
    const int n = a.g.n;
    const long long n2 = (long long)n * n;
    const double* tab = a.g.tab;
    const double inv2h = 0.5 / a.g.h, epsh2 = a.g.eps / (a.g.h * a.g.h);
    double acc[1] = {0.0};
    const long long p_lo = (long long)blockIdx.x * CH, p_hi = min(a.g.Ng, p_lo + CH);
    for (long long i = p_lo + threadIdx.x; i < p_hi; i += blockDim.x) {
        const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / n2);
        const long long base = i - x;
        const long long rowb = i - (long long)y * n;
        const long long plb = i - (long long)z * n2;
        const double* d = a.d;
        const double uc = d[i];
        const double uxp = d[base + (x + 1 == n ? 0 : x + 1)], uxm = d[base + (x == 0 ? n - 1 : x - 1)];
        const double uyp = d[rowb + (long long)(y + 1 == n ? 0 : y + 1) * n];
        const double uym = d[rowb + (long long)(y == 0 ? n - 1 : y - 1) * n];
        const double uzp = d[plb + (long long)(z + 1 == n ? 0 : z + 1) * n2];
        const double uzm = d[plb + (long long)(z == 0 ? n - 1 : z - 1) * n2];
        const double bx = tab[TXY * n + y] + tab[TXZ * n + z];
        const double by = tab[TYX * n + x] + tab[TYZ * n + z];
        const double bz = tab[TZX * n + x] + tab[TZY * n + y];
        const double adv = (bx * (uxp - uxm) + by * (uyp - uym) + bz * (uzp - uzm)) * inv2h;
        const double dif = epsh2 * ((uxp + uxm) + (uyp + uym) + (uzp + uzm) - 6.0 * uc);
        const double Ld = adv - dif;
        a.Ld[i] = Ld;
        a.Ltd[i] = -adv - dif;
        acc[0] += uc * Ld;
    }
    double* outs[1] = {a.dots + DotsLayout(a.maxm).DLD};
    chunk_reduce<1>(acc, 1, a.part, chunks, blockIdx.x, a.counter + 2, outs);
}

// Reduced solve (one CTA, FP64).  K = m + aug <= 33 (CS_MAXQ - 3).
constexpr int CS_MAXK = CS_MAXQ - 3;

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

__global__ void cs_small_kernel(CoarseArgs a, const CsDesc* desc) {
    __shared__ double Mv[CS_MAXK * CS_MAXK];
    __shared__ double Ac[CS_MAXK * CS_MAXK];
    __shared__ double T[CS_MAXK * CS_MAXK];
    __shared__ double x[CS_MAXK], y[CS_MAXK];
    __shared__ int piv[CS_MAXK];
    __shared__ int s_K;
    __shared__ double s_nd;
    const int m = desc->m;
    const DotsLayout L(a.maxm);
    const double* D = a.dots;
    if (threadIdx.x == 0) {
        const double dd = D[L.DD], uu = D[L.UU];
        const double nd = sqrt(fmax(dd, 0.0));
        const bool aug = nd > a.aug_tol * sqrt(fmax(uu, 0.0)) && nd > 0.0;
        s_K = aug ? m + 1 : m;
        s_nd = aug ? nd : 0.0;
    }
    __syncthreads();
    const int K = s_K;
    const double nd = s_nd;
    const double dT = a.dT;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int i = e / K, j = e - i * K;
        double mv, lv;
        if (i < m && j < m) {
            mv = a.Mr[(size_t)i * a.maxm + j];
            lv = a.Lr[(size_t)i * a.maxm + j];
        } else if (i < m) {          // column m: R^T d, R^T L d
            mv = D[L.RD2 + i] / nd;
            lv = D[L.RL + 2 * i + 0] / nd;
        } else if (j < m) {          // row m: d^T R, d^T L R = (L^T d)^T R
            mv = D[L.RD2 + j] / nd;
            lv = D[L.RL + 2 * j + 1] / nd;
        } else {
            mv = D[L.DD] / (nd * nd);
            lv = D[L.DLD] / (nd * nd);
        }
        Mv[i * CS_MAXK + j] = mv;
        Ac[i * CS_MAXK + j] = mv + dT * lv;
        T[i * CS_MAXK + j] = mv;  // right-hand sides of Ac T = Mv
    }
    // projection of the difference: V^T (U - U')
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        x[i] = (i < m) ? D[L.RU + 2 * i] - D[L.RU + 2 * i + 1] : (D[L.DU] - D[L.DUp]) / nd;
    __syncthreads();
    lu_factor(Ac, K, piv);
    for (int c = threadIdx.x; c < K; c += blockDim.x) lu_solve_col(Ac, K, piv, T + c, CS_MAXK);
    __syncthreads();
    // Mv x0 = V^T (U - U'): factor Mv (Ac is no longer needed)
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int i = e / K, j = e - i * K;
        Ac[i * CS_MAXK + j] = Mv[i * CS_MAXK + j];
    }
    __syncthreads();
    lu_factor(Ac, K, piv);
    if (threadIdx.x == 0) lu_solve_col(Ac, K, piv, x, 1);
    __syncthreads();
    for (int l = 0; l < a.Lc; ++l) {
        for (int i = threadIdx.x; i < K; i += blockDim.x) {
            double s = 0.0;
            for (int j = 0; j < K; ++j) s += T[i * CS_MAXK + j] * x[j];
            y[i] = s;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += blockDim.x) x[i] = y[i];
        __syncthreads();
    }
    for (int i = threadIdx.x; i <= a.maxm; i += blockDim.x) {
        double v = 0.0;
        if (i < m) v = x[i];
        else if (i == m && K == m + 1) v = x[m] / nd;
        a.coef[i] = v;
    }
}

template <typename KT>
__global__ void __launch_bounds__(CS_THREADS) cs_update_kernel(CoarseArgs a, const CsDesc* desc) {
    const int m = desc->m;
    __shared__ double g[CS_MAXK + 1];
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = a.coef[i];
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.g.Ng) return;
    const KT* R = reinterpret_cast<const KT*>(a.R);
    double s = a.F[p] + a.d[p] * g[m];
    for (int i = 0; i < m; ++i) s += (double)R[(size_t)i * a.g.Ng + p] * g[i];
    a.out[p] = s;
}

cudaError_t launch_coarse_update(const CoarseArgs& a, bool r_f32, cudaStream_t st) {
    if (a.maxm > CS_MAXK - 1) return cudaErrorInvalidValue;
    const int chunks = gram_chunks(a.g.Ng);
    long long CH = (a.g.Ng + chunks - 1) / chunks;
    const DotsLayout L(a.maxm);
    const int esize = r_f32 ? 4 : 8;
    // descriptors live right after the dot products in the dots scratch
    CsDesc* desc = reinterpret_cast<CsDesc*>(a.dots + ((L.total + 7) / 8) * 8);
    cs_prepare_kernel<<<1, 32, 0, st>>>(desc, a.R, a.m_ptr, a.maxm, a.g.Ng, esize, a.U, a.Up, a.Ld, a.Ltd);
    ++g_launch_count;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // pass 1: R^T [U, U']
    GramArgs ga{};
    ga.colsA = desc->colsR;
    ga.colsB = desc->colsUU;
    ga.KA = &desc->m;
    ga.KB = &desc->two;
    ga.ldcols = 0;
    ga.Ng = a.g.Ng;
    ga.B = 1;
    ga.maxKA = a.maxm;
    ga.maxKB = 2;
    ga.sym = false;
    ga.part = a.part;
    ga.counter = a.counter + 3;
    ga.G = a.dots + L.RU;
    ga.ldG = 2;
    ga.ldG_b = 0;
    e = launch_gram(ga, r_f32, false, st);
    if (e != cudaSuccess) return e;
    // passes 2, 3
    if (r_f32) cs_resid_kernel<float><<<chunks, CS_THREADS, 0, st>>>(a, desc, CH, chunks);
    else cs_resid_kernel<double><<<chunks, CS_THREADS, 0, st>>>(a, desc, CH, chunks);
    ++g_launch_count;
    if (r_f32) cs_reorth_kernel<float><<<chunks, CS_THREADS, 0, st>>>(a, desc, CH, chunks);
    else cs_reorth_kernel<double><<<chunks, CS_THREADS, 0, st>>>(a, desc, CH, chunks);
    ++g_launch_count;
    // pass 4
    cs_Ld_kernel<<<chunks, CS_THREADS, 0, st>>>(a, CH, chunks);
    ++g_launch_count;
    // pass 5: R^T [L d~, L^T d~]
    ga.colsB = desc->colsL;
    ga.G = a.dots + L.RL;
    ga.counter = a.counter + 4;
    e = launch_gram(ga, r_f32, false, st);
    if (e != cudaSuccess) return e;
    // pass 6, 7
    cs_small_kernel<<<1, 128, 0, st>>>(a, desc);
    ++g_launch_count;
    const unsigned blocks = (unsigned)((a.g.Ng + CS_THREADS - 1) / CS_THREADS);
    if (r_f32) cs_update_kernel<float><<<blocks, CS_THREADS, 0, st>>>(a, desc);
    else cs_update_kernel<double><<<blocks, CS_THREADS, 0, st>>>(a, desc);
    ++g_launch_count;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Iteration 0 in reduced coordinates: beta_0 = M0^{-1} p0, then N*Lc implicit Euler
// steps (M0 + dT L0) beta_l = M0 beta_{l-1} + dT q0; beta at the end of subinterval n is
// stored in beta[n*ldb .. ] (n = 0..N-1 gives U^0_{n+1}).
__global__ void g0_kernel(const double* M0, const double* L0, const double* p0, const double* q0,
                          const int* m0p, int ld, int N, int Lc, double dT, double* beta, int ldb,
                          int* err) {
    __shared__ double Mv[CS_MAXK * CS_MAXK];
    __shared__ double Ac[CS_MAXK * CS_MAXK];
    __shared__ double T[CS_MAXK * CS_MAXK];
    __shared__ double w[CS_MAXK], x[CS_MAXK], y[CS_MAXK];
    __shared__ int piv[CS_MAXK];
    const int K = *m0p;
    if (K <= 0 || K > CS_MAXK) {
        if (K > CS_MAXK && threadIdx.x == 0) record_error(err, DERR_BREAKDOWN);
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
                      int* err, cudaStream_t st) {
    g0_kernel<<<1, 128, 0, st>>>(M0, L0, p0, q0, m0, ld, N, Lc, dT, beta, ldb, err);
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
