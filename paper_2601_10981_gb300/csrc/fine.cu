// Fine propagator F of the adaptive parareal method (Algorithm 2, fine sweep):
// batched implicit Euler, eq. (semi-dis-eq)/(algform) with M = I on the periodic FD grid,
//     (I + dt L_h) u_j = u_{j-1} + dt f,
// one BiCGStab solve per step, all active subintervals in one persistent cooperative
// launch.
//
// Design (GB300): the grid is split into groups of G co-resident CTAs; a group owns one
// subinterval at a time and marches it through all S steps, synchronising only its own
// CTAs with a bounded acquire/release barrier (no grid-wide sync, no host round trip).
// Each CTA owns a contiguous range of grid rows (one row = n points along x), so loads
// are coalesced along x and the 7-point neighbours of a row are mostly L1/L2 hits.
//
// Each step is solved for the increment delta = u_j - u_{j-1} ("delta form"):
//     (I + dt L) delta = dt (f - L u_{j-1}),   delta_0 = 0,
// which generates the same Krylov iterates as BiCGStab on the paper's system started
// from u_{j-1}.  The state u stays FP64; delta and the Krylov vectors are KT (double in
// the FP64 mode, float in the FP32 mode).  The residual of the state is formed in FP64.
// Stopping rule: ||r|| <= tol ||u_{j-1} + dt f||.
//
// BiCGStab phases (van der Vorst 1992), each followed by a group barrier:
//   setup : u_{j-1} = u_{j-2} + delta (fused), r = rhat = dt (f - L u_{j-1});  <r,r>, <b,b>
//   ph1   : p = r + beta (p' - omega v'),  v = A p;                  <rhat, v>
//   ph2   : s = r - alpha v,               t = A s;        <t,s>, <t,t>, <s,s>
//   ph3   : delta += alpha p + omega s,    r = s - omega t;      <rhat,r>, <r,r>
// p and s are recomputed at the 6 neighbours instead of being stored, p/v alternate
// between two buffers so that neighbours read the previous iterate.
#include "pr_internal.cuh"

#include <algorithm>
#include <math.h>

namespace pr {

// ------------------------------------------------------------------------------------
// Velocity tables (six 1-D tables, see Grid).
__global__ void tables_kernel(int kind, double A, double B, double C, int k, double b0,
                              double b1, double b2, int n, double L, double* tab) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = i * (L / n);
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (kind == PR_FLOW_ABC) {
        v[TXY] = C * cos(x);  // b_x = A sin z + C cos y
        v[TXZ] = A * sin(x);
        v[TYX] = B * sin(x);  // b_y = B sin x + A cos z
        v[TYZ] = A * cos(x);
        v[TZX] = B * cos(x);  // b_z = C sin y + B cos x
        v[TZY] = C * sin(x);
    } else if (kind == PR_FLOW_KOLMOGOROV) {
        v[TXY] = sin((double)k * x);  // b = (sin k y, 0, 0)
    } else {
        v[TXY] = b0;
        v[TYX] = b1;
        v[TZX] = b2;
    }
    for (int t = 0; t < 6; ++t) tab[t * n + i] = v[t];
}

cudaError_t launch_tables(const pr_flow& flow, int n, double L, double* tab, cudaStream_t st) {
    tables_kernel<<<(n + 127) / 128, 128, 0, st>>>(flow.kind, flow.A, flow.B, flow.C, flow.k,
                                                   flow.b[0], flow.b[1], flow.b[2], n, L, tab);
    ++g_launch_count;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// out = L u or L^T u on whole grid functions.  Every supported velocity has b_d
// independent of x_d, so b_d(x +- e_d) = b_d(x) and L^T only flips the advection sign.
template <typename TI, typename TO>
__global__ void apply_L_kernel(Grid g, const void* const* in_cols, void* const* out_cols,
                               const int* count, int ldcols, bool transpose) {
    const int b = blockIdx.z, c = blockIdx.y;
    if (c >= count[b]) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.Ng) return;
    const TI* in = (const TI*)in_cols[(size_t)b * ldcols + c];
    TO* out = (TO*)out_cols[(size_t)b * ldcols + c];
    const int n = g.n;
    const long long n2 = (long long)n * n;
    const int x = (int)(i % n);
    const int y = (int)((i / n) % n);
    const int z = (int)(i / n2);
    const long long base = i - x;
    const long long ixp = base + (x + 1 == n ? 0 : x + 1), ixm = base + (x == 0 ? n - 1 : x - 1);
    const long long rowb = i - (long long)y * n;
    const long long iyp = rowb + (long long)(y + 1 == n ? 0 : y + 1) * n;
    const long long iym = rowb + (long long)(y == 0 ? n - 1 : y - 1) * n;
    const long long plb = i - (long long)z * n2;
    const long long izp = plb + (long long)(z + 1 == n ? 0 : z + 1) * n2;
    const long long izm = plb + (long long)(z == 0 ? n - 1 : z - 1) * n2;
    const double* tab = g.tab;
    const double bx = tab[TXY * n + y] + tab[TXZ * n + z];
    const double by = tab[TYX * n + x] + tab[TYZ * n + z];
    const double bz = tab[TZX * n + x] + tab[TZY * n + y];
    const double u0 = (double)in[i];
    const double uxp = (double)in[ixp], uxm = (double)in[ixm];
    const double uyp = (double)in[iyp], uym = (double)in[iym];
    const double uzp = (double)in[izp], uzm = (double)in[izm];
    double adv = bx * (uxp - uxm) + by * (uyp - uym) + bz * (uzp - uzm);
    if (transpose) adv = -adv;
    const double lap = (uxp + uxm) + (uyp + uym) + (uzp + uzm) - 6.0 * u0;
    out[i] = (TO)(adv * (0.5 / g.h) - g.eps * lap / (g.h * g.h));
}

cudaError_t launch_apply_L(const Grid& g, const void* const* in_cols, void* const* out_cols,
                           const int* count, int ldcols, int max_count, int B, bool in_f32,
                           bool out_f32, bool transpose, cudaStream_t st) {
    if (max_count <= 0 || B <= 0) return cudaSuccess;
    dim3 grid((unsigned)((g.Ng + 255) / 256), (unsigned)max_count, (unsigned)B);
    if (in_f32 && out_f32)
        apply_L_kernel<float, float><<<grid, 256, 0, st>>>(g, in_cols, out_cols, count, ldcols, transpose);
    else if (in_f32)
        apply_L_kernel<float, double><<<grid, 256, 0, st>>>(g, in_cols, out_cols, count, ldcols, transpose);
    else if (out_f32)
        apply_L_kernel<double, float><<<grid, 256, 0, st>>>(g, in_cols, out_cols, count, ldcols, transpose);
    else
        apply_L_kernel<double, double><<<grid, 256, 0, st>>>(g, in_cols, out_cols, count, ldcols, transpose);
    ++g_launch_count;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Fine sweep kernel.

// Per-thread partial sums: KT = float accumulates 16 points in float, then in double.
template <typename KT, int NQ>
struct Acc {
    double d[NQ];
    KT f[NQ];
    int c;
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < NQ; ++q) { d[q] = 0.0; f[q] = (KT)0; }
        c = 0;
    }
    __device__ __forceinline__ void flush() {
#pragma unroll
        for (int q = 0; q < NQ; ++q) { d[q] += (double)f[q]; f[q] = (KT)0; }
        c = 0;
    }
    __device__ __forceinline__ void tick() {
        if (++c == 16) flush();
    }
};

struct Nbr {
    long long c, xp, xm, yp, ym, zp, zm;
    int x, y, z;
};

__device__ __forceinline__ Nbr neighbours(int x, int y, int z, int n, long long n2) {
    Nbr o;
    o.x = x; o.y = y; o.z = z;
    const long long row = (long long)z * n2 + (long long)y * n;
    o.c = row + x;
    o.xp = row + (x + 1 == n ? 0 : x + 1);
    o.xm = row + (x == 0 ? n - 1 : x - 1);
    o.yp = (long long)z * n2 + (long long)(y + 1 == n ? 0 : y + 1) * n + x;
    o.ym = (long long)z * n2 + (long long)(y == 0 ? n - 1 : y - 1) * n + x;
    o.zp = (long long)(z + 1 == n ? 0 : z + 1) * n2 + (long long)y * n + x;
    o.zm = (long long)(z == 0 ? n - 1 : z - 1) * n2 + (long long)y * n + x;
    return o;
}

template <typename KT>
struct FineShared {
    double red[4 * 32];
    double sums[4];
};

// Sum of the per-CTA partials of a group for quantities 0..nq-1 (fixed order, read by
// warp 0, lane 0 result broadcast through shared memory).
__device__ __forceinline__ void group_sums(const double* part, int grid, int g0, int G, int nq,
                                           double* out_sums) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int q = 0; q < nq; ++q) {
            double s = 0.0;
            for (int i = lane; i < G; i += 32) s += part[(size_t)q * grid + g0 + i];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (lane == 0) out_sums[q] = s;
        }
    }
    __syncthreads();
}

template <typename KT>
__global__ void __launch_bounds__(256) fine_kernel(FineArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ FineShared<KT> sh;

    const int G = a.G;
    const int g = blockIdx.x / G;
    const int q = blockIdx.x % G;
    const int grid = gridDim.x;
    const int n = a.g.n;
    const long long n2 = (long long)n * n;
    const long long Ng = a.g.Ng;
    const int rows_pass = blockDim.x / n;
    const int tx = threadIdx.x % n;
    const int ty = threadIdx.x / n;
    const long long nrows = n2;
    const long long r_lo = nrows * q / G, r_hi = nrows * (q + 1) / G;

    // shared tables: unscaled FP64 velocity (setup) and dt/(2h)-scaled KT (Krylov)
    double* tabd = reinterpret_cast<double*>(smem_raw);
    KT* tabk = reinterpret_cast<KT*>(tabd + 6 * n);
    for (int i = threadIdx.x; i < 6 * n; i += blockDim.x) {
        const double v = a.g.tab[i];
        tabd[i] = v;
        tabk[i] = (KT)(v * a.dt * 0.5 / a.g.h);
    }
    __syncthreads();

    const double h = a.g.h, eps = a.g.eps, dt = a.dt;
    const double inv2h = 0.5 / h, epsh2 = eps / (h * h);
    const KT c1 = (KT)(dt * eps / (h * h));
    const KT c0 = (KT)(1.0 + 6.0 * dt * eps / (h * h));

    KT* W = reinterpret_cast<KT*>(a.ws) + (size_t)g * FINE_NVEC * Ng;
    KT* delta = W;
    KT* r = W + Ng;
    KT* rh = W + 2 * Ng;
    KT* pbuf[2] = {W + 3 * Ng, W + 4 * Ng};
    KT* vbuf[2] = {W + 5 * Ng, W + 6 * Ng};
    KT* t = W + 7 * Ng;
    double* ust = a.ust + (size_t)g * 2 * Ng;
    unsigned* bar = a.bar + 2 * g;
    double* part = a.part;  // [2][4][grid]
    const int g0 = g * G;
    int ph = 0;  // reduction phase counter (partials double-buffered on ph & 1)

    // A applied at a point given the 7 values of the operand.
    auto applyA = [&](const Nbr& o, KT vc, KT vxp, KT vxm, KT vyp, KT vym, KT vzp, KT vzm) -> KT {
        const KT ax = tabk[TXY * n + o.y] + tabk[TXZ * n + o.z];
        const KT ay = tabk[TYX * n + o.x] + tabk[TYZ * n + o.z];
        const KT az = tabk[TZX * n + o.x] + tabk[TZY * n + o.y];
        return c0 * vc + (ax - c1) * vxp - (ax + c1) * vxm + (ay - c1) * vyp - (ay + c1) * vym +
               (az - c1) * vzp - (az + c1) * vzm;
    };

    for (int b = g; b < a.B; b += a.numGroups) {
        const double* u_in = a.u_in + (size_t)b * Ng;
        KT* snap_b = a.snap ? reinterpret_cast<KT*>(a.snap) + (size_t)b * a.n_snap * Ng : nullptr;
        long long its_total = 0;
        int its_max = 0;
        int status = 0;
        bool dvalid = false;

        for (int j = 1; j <= a.S; ++j) {
            // ---------------- setup: u_{j-1} = u_{j-2} + delta ; r = dt (f - L u_{j-1})
            const double* P = (j <= 2) ? u_in : ust + (size_t)((j - 2) & 1) * Ng;
            double* Wt = (j >= 2) ? ust + (size_t)((j - 1) & 1) * Ng : nullptr;
            const bool use_d = (j >= 2) && dvalid;
            KT* snap_j = nullptr;
            if (snap_b && (j - 1) % a.dM == 0 && (j - 1) / a.dM < a.n_snap)
                snap_j = snap_b + (size_t)((j - 1) / a.dM) * Ng;
            {
                Acc<KT, 2> acc;
                acc.init();
                if (ty < rows_pass) {
                    for (long long rr = r_lo + ty; rr < r_hi; rr += rows_pass) {
                        const int z = (int)(rr / n), y = (int)(rr % n);
                        const Nbr o = neighbours(tx, y, z, n, n2);
                        auto cur = [&](long long i) -> double {
                            return use_d ? P[i] + (double)delta[i] : P[i];
                        };
                        const double uc = cur(o.c);
                        const double uxp = cur(o.xp), uxm = cur(o.xm);
                        const double uyp = cur(o.yp), uym = cur(o.ym);
                        const double uzp = cur(o.zp), uzm = cur(o.zm);
                        if (Wt) Wt[o.c] = uc;
                        if (snap_j) snap_j[o.c] = (KT)uc;
                        const double bx = tabd[TXY * n + y] + tabd[TXZ * n + z];
                        const double by = tabd[TYX * n + tx] + tabd[TYZ * n + z];
                        const double bz = tabd[TZX * n + tx] + tabd[TZY * n + y];
                        const double adv = bx * (uxp - uxm) + by * (uyp - uym) + bz * (uzp - uzm);
                        const double lap = (uxp + uxm) + (uyp + uym) + (uzp + uzm) - 6.0 * uc;
                        const double Lu = adv * inv2h - epsh2 * lap;
                        const double fi = a.f ? a.f[o.c] : 0.0;
                        const KT rk = (KT)(dt * (fi - Lu));
                        r[o.c] = rk;
                        rh[o.c] = rk;
                        const double bi = uc + dt * fi;
                        acc.f[0] += rk * rk;
                        acc.f[1] += (KT)(bi * bi);
                        acc.tick();
                    }
                }
                acc.flush();
                block_sum<2>(acc.d, sh.red);
                if (threadIdx.x == 0) {
                    part[(size_t)((ph & 1) * 4 + 0) * grid + blockIdx.x] = acc.d[0];
                    part[(size_t)((ph & 1) * 4 + 1) * grid + blockIdx.x] = acc.d[1];
                }
            }
            if (!group_barrier(bar, G, a.spin_limit, a.err)) return;
            group_sums(part + (size_t)(ph & 1) * 4 * grid, grid, g0, G, 2, sh.sums);
            ++ph;
            const double rr0 = sh.sums[0], bb = sh.sums[1];
            const double thr = a.tol * sqrt(bb);
            bool conv = sqrt(rr0) <= thr;
            if (!isfinite(rr0) || !isfinite(bb)) { status = DERR_NONFINITE; conv = true; }
            double rho = rr0, alpha = 1.0, omega = 1.0, beta = 0.0;
            int it = 0;
            while (!conv) {
                ++it;
                // ---------------- ph1: p = r + beta (p' - omega v'), v = A p
                KT* pn = pbuf[it & 1];
                KT* po = pbuf[(it - 1) & 1];
                KT* vn = vbuf[it & 1];
                KT* vo = vbuf[(it - 1) & 1];
                {
                    const KT bk = (KT)beta, ok = (KT)omega;
                    const bool first = (it == 1);
                    Acc<KT, 1> acc;
                    acc.init();
                    if (ty < rows_pass) {
                        for (long long rr = r_lo + ty; rr < r_hi; rr += rows_pass) {
                            const int z = (int)(rr / n), y = (int)(rr % n);
                            const Nbr o = neighbours(tx, y, z, n, n2);
                            auto pv = [&](long long i) -> KT {
                                return first ? r[i] : r[i] + bk * (po[i] - ok * vo[i]);
                            };
                            const KT pc = pv(o.c);
                            const KT av = applyA(o, pc, pv(o.xp), pv(o.xm), pv(o.yp), pv(o.ym),
                                                 pv(o.zp), pv(o.zm));
                            pn[o.c] = pc;
                            vn[o.c] = av;
                            acc.f[0] += rh[o.c] * av;
                            acc.tick();
                        }
                    }
                    acc.flush();
                    block_sum<1>(acc.d, sh.red);
                    if (threadIdx.x == 0) part[(size_t)((ph & 1) * 4) * grid + blockIdx.x] = acc.d[0];
                }
                if (!group_barrier(bar, G, a.spin_limit, a.err)) return;
                group_sums(part + (size_t)(ph & 1) * 4 * grid, grid, g0, G, 1, sh.sums);
                ++ph;
                const double rv = sh.sums[0];
                if (rv == 0.0 || !isfinite(rv)) {
                    status = isfinite(rv) ? DERR_BREAKDOWN : DERR_NONFINITE;
                    --it;
                    break;
                }
                alpha = rho / rv;
                // ---------------- ph2: s = r - alpha v, t = A s
                {
                    const KT al = (KT)alpha;
                    Acc<KT, 3> acc;
                    acc.init();
                    if (ty < rows_pass) {
                        for (long long rr = r_lo + ty; rr < r_hi; rr += rows_pass) {
                            const int z = (int)(rr / n), y = (int)(rr % n);
                            const Nbr o = neighbours(tx, y, z, n, n2);
                            auto sv = [&](long long i) -> KT { return r[i] - al * vn[i]; };
                            const KT sc = sv(o.c);
                            const KT tv = applyA(o, sc, sv(o.xp), sv(o.xm), sv(o.yp), sv(o.ym),
                                                 sv(o.zp), sv(o.zm));
                            t[o.c] = tv;
                            acc.f[0] += tv * sc;
                            acc.f[1] += tv * tv;
                            acc.f[2] += sc * sc;
                            acc.tick();
                        }
                    }
                    acc.flush();
                    block_sum<3>(acc.d, sh.red);
                    if (threadIdx.x == 0) {
                        for (int qq = 0; qq < 3; ++qq)
                            part[(size_t)((ph & 1) * 4 + qq) * grid + blockIdx.x] = acc.d[qq];
                    }
                }
                if (!group_barrier(bar, G, a.spin_limit, a.err)) return;
                group_sums(part + (size_t)(ph & 1) * 4 * grid, grid, g0, G, 3, sh.sums);
                ++ph;
                const double ts = sh.sums[0], tt = sh.sums[1], ss = sh.sums[2];
                const bool half = sqrt(ss) <= thr;
                if (!half) {
                    if (tt == 0.0 || !isfinite(tt)) {
                        status = isfinite(tt) ? DERR_BREAKDOWN : DERR_NONFINITE;
                        omega = 0.0;
                    } else {
                        omega = ts / tt;
                        if (omega == 0.0) status = DERR_BREAKDOWN;
                    }
                }
                // ---------------- ph3: delta += alpha p + omega s ; r = s - omega t
                {
                    const KT al = (KT)alpha, om = (KT)omega;
                    const bool first = (it == 1);
                    const bool upd_r = !half && status == 0;
                    Acc<KT, 2> acc;
                    acc.init();
                    if (ty < rows_pass) {
                        for (long long rr = r_lo + ty; rr < r_hi; rr += rows_pass) {
                            const long long i = (rr / n) * n2 + (rr % n) * n + tx;
                            const KT dold = first ? (KT)0 : delta[i];
                            const KT pc = pn[i];
                            if (half || status != 0) {
                                delta[i] = dold + al * pc;
                            } else {
                                const KT sc = r[i] - al * vn[i];
                                delta[i] = dold + al * pc + om * sc;
                                const KT rn = sc - om * t[i];
                                r[i] = rn;
                                acc.f[0] += rh[i] * rn;
                                acc.f[1] += rn * rn;
                                acc.tick();
                            }
                        }
                    }
                    acc.flush();
                    block_sum<2>(acc.d, sh.red);
                    if (threadIdx.x == 0 && upd_r) {
                        part[(size_t)((ph & 1) * 4 + 0) * grid + blockIdx.x] = acc.d[0];
                        part[(size_t)((ph & 1) * 4 + 1) * grid + blockIdx.x] = acc.d[1];
                    }
                    if (!group_barrier(bar, G, a.spin_limit, a.err)) return;
                    if (half || status != 0) break;
                    group_sums(part + (size_t)(ph & 1) * 4 * grid, grid, g0, G, 2, sh.sums);
                    ++ph;
                }
                const double rho_new = sh.sums[0], rr1 = sh.sums[1];
                if (!isfinite(rr1)) { status = DERR_NONFINITE; break; }
                if (sqrt(rr1) <= thr) break;
                if (rho_new == 0.0) { status = DERR_BREAKDOWN; break; }
                if (it >= a.maxit) { status = DERR_NOT_CONVERGED; break; }
                beta = (rho_new / rho) * (alpha / omega);
                rho = rho_new;
            }
            dvalid = it > 0;
            its_total += it;
            its_max = max(its_max, it);
            if (status != 0) {
                // keep marching (the caller reports the status); a non-finite state
                // would only propagate, so the remaining steps are skipped
                if (status == DERR_NONFINITE) break;
            }
        }
        // ---------------- final: u_S = u_{S-1} + delta ; snapshot of u_S
        {
            const int S = a.S;
            const double* P = (S >= 2) ? ust + (size_t)((S - 1) & 1) * Ng : u_in;
            KT* snap_S = (snap_b && S % a.dM == 0 && S / a.dM < a.n_snap)
                             ? snap_b + (size_t)(S / a.dM) * Ng : nullptr;
            double* out = a.u_out + (size_t)b * Ng;
            if (ty < rows_pass) {
                for (long long rr = r_lo + ty; rr < r_hi; rr += rows_pass) {
                    const long long i = (rr / n) * n2 + (rr % n) * n + tx;
                    const double u = dvalid ? P[i] + (double)delta[i] : P[i];
                    out[i] = u;
                    if (snap_S) snap_S[i] = (KT)u;
                }
            }
        }
        if (q == 0 && threadIdx.x == 0) {
            a.status[b] = status;
            a.its_total[b] = (int)its_total;
            a.its_max[b] = its_max;
        }
        // The next subinterval's first setup reads only its own input state and writes
        // r/rhat, which no CTA of this group reads before the next barrier.
    }
}

int fine_block_threads(int n) {
    const int rows = n >= 256 ? 1 : 256 / n;
    return n * rows;
}

static size_t fine_smem(int n, bool fp32) {
    return (size_t)6 * n * sizeof(double) + (size_t)6 * n * (fp32 ? sizeof(float) : sizeof(double));
}

int fine_max_ctas(int n, bool fp32, int ctas_per_sm) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = fine_block_threads(n);
    const size_t smem = fine_smem(n, fp32);
    if (fp32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fine_kernel<float>, threads, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fine_kernel<double>, threads, smem);
    if (ctas_per_sm > 0) occ = std::min(occ, ctas_per_sm);
    return std::max(1, occ) * std::max(1, sms);
}

cudaError_t launch_fine(FineArgs a, bool fp32, int ctas_per_sm, int max_groups, cudaStream_t st) {
    if (a.B <= 0) return cudaSuccess;
    const int n = a.g.n;
    if (n > 256 || n < 4) return cudaErrorInvalidValue;
    const int max_ctas = fine_max_ctas(n, fp32, ctas_per_sm);
    const long long rows = (long long)n * n;
    int G = a.G;
    if (G <= 0) G = (int)std::max<long long>(1, std::min<long long>(rows, max_ctas / a.B));
    G = (int)std::min<long long>(G, std::min<long long>(rows, max_ctas));
    int groups = std::min(a.B, std::max(1, max_ctas / G));
    groups = std::min(groups, max_groups);
    a.G = G;
    a.numGroups = groups;
    const int grid = G * groups;
    const int threads = fine_block_threads(n);
    const size_t smem = fine_smem(n, fp32);
    void* args[] = {&a};
    cudaError_t e;
    if (fp32)
        e = cudaLaunchCooperativeKernel((const void*)fine_kernel<float>, dim3(grid), dim3(threads),
                                        args, smem, st);
    else
        e = cudaLaunchCooperativeKernel((const void*)fine_kernel<double>, dim3(grid), dim3(threads),
                                        args, smem, st);
    ++g_launch_count;
    return e;
}

} // namespace pr
