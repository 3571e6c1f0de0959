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
// from u_{j-1}.  delta and the Krylov vectors are KT (double in the FP64 mode, float in
// the FP32 mode).  The FP64 mode keeps the state u in FP64.  The FP32 mode keeps it as an
// unevaluated sum hi + lo of two floats (8 bytes, ~48 significant bits) and runs on the
// FP32 pipe only: GB300 issues FP64 arithmetic at 1/64 of the FP32 rate, so an FP64
// residual stencil would cost more than all of the FP32 Krylov work.  Its residual uses
// differences of neighbouring hi parts, which are exact when the neighbours are within a
// factor of two (Sterbenz), so r keeps FP32 accuracy relative to the differences.
// Snapshots are written in FP64 in both modes: the POD criterion keeps modes down to
// lambda/lambda_1 ~ 1e-12, which FP32-rounded snapshots cannot resolve.
// The FP32 mode starts BiCGStab from the previous step's increment (linear extrapolation
// in time; r = dt (f - L (u_{j-1} + delta_{j-1})) - delta_{j-1}), which halves the
// iterations per step at its 1e-9 tolerance; the FP64 mode starts from 0.
// Stopping rule: ||r|| <= tol ||u_{j-1} + dt f||.
//
// BiCGStab phases (van der Vorst 1992), each followed by a group barrier:
//   setup : u_{j-1} = u_{j-2} + delta (fused), r = rhat = dt (f - L u_{j-1});  <r,r>, <b,b>
//   ph1   : p = r + beta (p' - omega v'),  v = A p;                  <rhat, v>
//   ph2   : s = r - alpha v,               t = A s;        <t,s>, <t,t>, <s,s>
//   ph3   : delta += alpha p + omega s,    r = s - omega t;      <rhat,r>, <r,r>
// p and s are recomputed at the 6 neighbours instead of being stored, p/v alternate
// between two buffers so that neighbours read the previous iterate.
// The persistent fine-sweep kernel (implicit Euler with BiCGStab per step, or explicit
// RK4), shared by the translation units that instantiate it for each Krylov type.
#pragma once
#include "df.cuh"
#include "pr_internal.cuh"

#include <algorithm>
#include <math.h>
#include <type_traits>

namespace pr {

enum FineMode { FINE_MODE_IMPLICIT = 0, FINE_MODE_IMPLICIT_TD = 1, FINE_MODE_RK4 = 2, FINE_MODE_IMPLICIT_PERT = 3 };

// ------------------------------------------------------------------------------------
// Fine sweep kernel.
//
// Ownership: the n^3 points of a subinterval are cut into NY columns of TY rows (y); a
// column has n tile-planes (z).  The NY * n tile-planes, column by column, are split into
// G contiguous ranges of equal length, one per CTA of the group, so any G balances the
// work: a CTA owns the tail of one column and the head of the next, each a tile (y0, a
// range of planes).  Stencil phases march a tile plane by plane through a shared-memory
// ring of planes: the operand of the stencil (u, p or s) is computed once per plane, with
// one halo row on each side in y, and the 6 neighbours of a point come from the ring
// (x +- 1 wraps inside the row, z +- 1 from the adjacent slots).  Global traffic per point
// and phase is one load per input vector (plus the 2/TY halo rows and the 2 halo planes of
// each tile) and one store per output.

// Per-thread partial sums in two levels: runs of 16 ticks accumulate in f, the runs in
// s, both in KT.  The FP32 mode thus keeps its dot products off GB300's narrow FP64 pipe
// (a double flush per run cost a conversion and an addition there); cta_sum then gives
// the CTA total in double.
template <typename KT, int NQ>
struct Acc {
    double d[NQ];   // CTA total, valid in thread 0 after cta_sum
    KT s[NQ];
    KT f[NQ];
    int c;
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < NQ; ++q) { d[q] = 0.0; s[q] = (KT)0; f[q] = (KT)0; }
        c = 0;
    }
    __device__ __forceinline__ void flush() {
#pragma unroll
        for (int q = 0; q < NQ; ++q) { s[q] += f[q]; f[q] = (KT)0; }
        c = 0;
    }
    __device__ __forceinline__ void tick() {
        if (++c == 16) flush();
    }
};

// CTA sum of the per-thread partials acc.s into acc.d (thread 0, fixed order).  With
// KT = float the in-warp tree runs in float and only the warp totals are added in double.
template <typename KT, int NQ>
__device__ __forceinline__ void cta_sum(Acc<KT, NQ>& acc, double* red) {
    if constexpr (std::is_same<KT, double>::value) {
        double v[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = acc.s[q];
        block_sum<NQ>(v, red);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc.d[q] = v[q];
        }
    } else {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int nwarps = (blockDim.x + 31) >> 5;
        float w[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            w[q] = acc.s[q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) w[q] += __shfl_down_sync(0xffffffffu, w[q], off);
        }
        __syncthreads();
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) red[q * 32 + warp] = (double)w[q];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                double t = 0.0;
                for (int i = 0; i < nwarps; ++i) t += red[q * 32 + i];
                acc.d[q] = t;
            }
        }
    }
}

struct FineShared {
    double red[4 * 32];
    double sums[4];
    // BiCGStab scalars and decisions, written by thread 0 after each group reduction:
    // GB300 runs FP64 divisions and square roots on its narrow FP64 pipe, so they are
    // taken once per CTA instead of once per thread
    double thr, rho, alpha, omega, beta;
    int status, flag;
    double c0, c1;   // time coefficients of a time-dependent flow at the current step
};

// Sum of the per-CTA partials of a group for quantities 0..nq-1 (fixed order, read by
// warp 0); thread 0 then runs post(sums), and the results reach every thread through
// shared memory.
template <typename Post>
__device__ __forceinline__ void group_sums(const double* part, int grid, int g0, int G, int nq,
                                           double* out_sums, Post&& post) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int q = 0; q < nq; ++q) {
            double s = 0.0;
            for (int i = lane; i < G; i += 32) s += part[(size_t)q * grid + g0 + i];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (lane == 0) out_sums[q] = s;
        }
        if (lane == 0) post(out_sums);
    }
    __syncthreads();
}

// Tile t (= the y-block column t) of a CTA that owns tile-planes [p_lo, p_hi): rows
// y0 .. y0 + TY - 1, planes zlo .. zhi - 1 (non-empty for p_lo / n <= t < ceil(p_hi / n)).
struct TileGeom {
    int n, TY, p_lo, p_hi;
    __device__ __forceinline__ void tile(int t, int& y0, int& zlo, int& zhi) const {
        y0 = t * TY;
        zlo = max(p_lo - t * n, 0);
        zhi = min(p_hi - t * n, n);
    }
};

// W consecutive points along x handled by one thread (W = 4: 16-byte vector accesses).
template <typename T, int W>
struct Vec {
    T v[W];
};
template <typename T, int W>
__device__ __forceinline__ Vec<T, W> vload(const T* p) {
    Vec<T, W> o;
    if constexpr (W == 4 && sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        o.v[0] = q.x; o.v[1] = q.y; o.v[2] = q.z; o.v[3] = q.w;
    } else if constexpr (W == 4 && std::is_same<T, float2>::value) {
        const float4 q0 = *reinterpret_cast<const float4*>(p);
        const float4 q1 = *reinterpret_cast<const float4*>(p + 2);
        o.v[0] = make_float2(q0.x, q0.y); o.v[1] = make_float2(q0.z, q0.w);
        o.v[2] = make_float2(q1.x, q1.y); o.v[3] = make_float2(q1.z, q1.w);
    } else if constexpr (W == 4 && sizeof(T) == 8) {
        const double2 q0 = *reinterpret_cast<const double2*>(p);
        const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
        o.v[0] = q0.x; o.v[1] = q0.y; o.v[2] = q1.x; o.v[3] = q1.y;
    } else {
#pragma unroll
        for (int e = 0; e < W; ++e) o.v[e] = p[e];
    }
    return o;
}
template <typename T, int W>
__device__ __forceinline__ void vstore(T* p, const Vec<T, W>& o) {
    if constexpr (W == 4 && sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o.v[0], o.v[1], o.v[2], o.v[3]);
    } else if constexpr (W == 4 && std::is_same<T, float2>::value) {
        *reinterpret_cast<float4*>(p) = make_float4(o.v[0].x, o.v[0].y, o.v[1].x, o.v[1].y);
        *reinterpret_cast<float4*>(p + 2) = make_float4(o.v[2].x, o.v[2].y, o.v[3].x, o.v[3].y);
    } else if constexpr (W == 4 && sizeof(T) == 8) {
        *reinterpret_cast<double2*>(p) = make_double2(o.v[0], o.v[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(o.v[2], o.v[3]);
    } else {
#pragma unroll
        for (int e = 0; e < W; ++e) p[e] = o.v[e];
    }
}

// Planes per barrier of the stencil march and slots of its shared-memory ring.  Two
// planes per barrier halve the barriers but cost registers (spills) and expose the
// owned-point loads of the second plane: 110 ms against 102 ms for the 64^3 Kolmogorov
// sweep, so one plane per barrier stays.
constexpr int FINE_PLANES = 1;
constexpr int FINE_SLOTS = 2 * FINE_PLANES + 2;

// Double-float state of the FP32 mode: u = hi + lo with |lo| <= ulp(hi) / 2.
__device__ __forceinline__ float2 df_split(double u) {
    const float hi = __double2float_rn(u);
    return make_float2(hi, __double2float_rn(u - (double)hi));
}
__device__ __forceinline__ double df_value(float2 u) { return (double)u.x + (double)u.y; }
// (hi, lo) + d: TwoSum of hi and d (Knuth), then the renormalising FastTwoSum
__device__ __forceinline__ float2 df_add(float2 u, float d) {
    const float s = __fadd_rn(u.x, d);
    const float bb = __fsub_rn(s, u.x);
    const float e = __fadd_rn(__fsub_rn(u.x, __fsub_rn(s, bb)), __fsub_rn(d, bb));
    const float lo = __fadd_rn(u.y, e);
    const float hi = __fadd_rn(s, lo);
    return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
}

// snapshot value of the float-pair state: bits moved, one FP64 addition
__device__ __forceinline__ double df_value_bits(float hi, float lo) { return df_to_double(hi, lo); }

// Operand of the FP32-mode setup march: the float pair of the state, stored in the ring
// as two float planes (hi, then lo at a fixed offset), so that the stencil reads the hi
// neighbours with float loads.
template <int W> struct HiLo { Vec<float, W> hi, lo; };
template <typename T> struct is_hilo : std::false_type {};
template <int W> struct is_hilo<HiLo<W>> : std::true_type {};
// Asynchronous global -> shared copy of B bytes (4, 8 or 16; both addresses aligned to
// B), one commit group, and the wait for all but the newest n groups.
template <int B>
__device__ __forceinline__ void cp_async_b(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (B == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_newest() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// FP32-mode pointwise update phase: planes of its six inputs staged per thread in shared
// memory (over the idle ring), FINE_PH3_SLOTS - 1 planes ahead.  Two slots fit inside the
// setup ring, so the shared-memory footprint (and the L1 left beside it) is unchanged;
// measured on the 64^3 sweep: 2 slots 62.9 ms, 3 slots 63.5 ms, 4 slots 65.1 ms.
constexpr int FINE_PH3_SLOTS = 2;

// The FP32-mode implicit setup ring: the stencil operand op (one float) and the state
// u = hi + lo, in three planes.
template <int W> struct OpHiLo { Vec<float, W> op, hi, lo; };
template <typename T> struct is_ophilo : std::false_type {};
template <int W> struct is_ophilo<OpHiLo<W>> : std::true_type {};
// Owned-point inputs of the FP32-mode implicit setup: forcing and the initial increment.
// The stored velocity perturbation at W points (empty unless P).
template <typename KT, int W, bool P> struct PertV { Vec<KT, W> x, y, z; };
template <typename KT, int W> struct PertV<KT, W, false> {};
template <typename KT, int W, bool P> struct OwnFD { Vec<KT, W> f, d; PertV<KT, W, P> b; };
template <typename KT, int W, bool P> struct OwnH { Vec<KT, W> h; PertV<KT, W, P> b; };

// Raw inputs of the stencil operand, loaded one plane ahead (software pipelining).
template <typename ST, typename KT, int W> struct RawSetup { Vec<ST, W> u; Vec<KT, W> d; };
template <typename KT, int W> struct RawP { Vec<KT, W> r, p, v; };
template <typename KT, int W> struct RawS { Vec<KT, W> r, v; };
template <typename ST, typename KT, int W> struct RawF { Vec<ST, W> u; Vec<KT, W> d; };
template <typename KT, int W> struct RawP2 { Vec<KT, W> d, p; };
template <typename KT, int W> struct Raw6 { Vec<KT, W> d, p, r, v, t, h; };
struct NoOwn {};
// The 7-point values of W consecutive points: centre and the x, y, z neighbours.
template <typename T, int W> struct Nb7 { Vec<T, W> c, xp, xm, yp, ym, zp, zm; };

// KT: Krylov type.  W: points per thread along x.  KF: ring rows each thread fills per
// plane (ceil((TY+2)/RP)).  KS: owned rows per thread per plane (TY/RP).
// MODE: FINE_MODE_IMPLICIT (steady flow), FINE_MODE_IMPLICIT_TD (time-dependent flow:
// tables rebuilt per step), FINE_MODE_RK4 (explicit RK4, either flow) or
// FINE_MODE_IMPLICIT_PERT (steady flow plus a stored per-point velocity perturbation,
// three more loads per point and stencil).  Each mode is its own instantiation, so that
// no path's register allocation burdens another.
template <typename KT, int W, int KF, int KS, int MODE>
__global__ void __launch_bounds__(256, 2) fine_kernel(FineArgs a) {
    constexpr bool RK = MODE == FINE_MODE_RK4;
    constexpr bool PT = MODE == FINE_MODE_IMPLICIT_PERT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ FineShared sh;

    const int G = a.G;
    const int g = blockIdx.x / G;
    const int q = blockIdx.x % G;
    const int grid = gridDim.x;
    const int n = a.g.n;
    const int n2 = n * n;
    const long long Ng = a.g.Ng;
    const int lanes = n / W;                 // threads per row
    const int RP = a.RP;                     // rows per pass of the CTA (divides TY)
    // the CTA is rounded up to whole warps; threads past lanes * RP only join the
    // reductions and barriers
    const bool active = threadIdx.x < lanes * RP;
    const int lx = threadIdx.x % lanes;
    const int ty = active ? threadIdx.x / lanes : RP + a.TY + 2;
    const int x0 = lx * W;
    const int TY = a.TY, RW = a.TY + 2;
    const int TPN = a.NY * n;   // tile-planes of a subinterval (G <= TPN)
    const int p_lo = (int)((long long)TPN * q / G), p_hi = (int)((long long)TPN * (q + 1) / G);
    const TileGeom geo{n, a.TY, p_lo, p_hi};
    const int t_lo = p_lo / n, t_hi = (p_hi + n - 1) / n;
    const int xl = (x0 == 0) ? n - 1 : x0 - 1;   // left neighbour of the first point
    const int xr = (x0 + W == n) ? 0 : x0 + W;   // right neighbour of the last point

    // velocity tables (FP64, and scaled by dt/(2h) in KT), forcing tables of the
    // time-dependent flows (GX, GY, GZ combined for the current step), then the ring
    double* tabd = reinterpret_cast<double*>(smem_raw);
    KT* tabk = reinterpret_cast<KT*>(tabd + 6 * n);
    double* ftd = reinterpret_cast<double*>(smem_raw + (size_t)6 * n * (sizeof(double) + sizeof(KT)));
    KT* ftk = reinterpret_cast<KT*>(ftd + 3 * n);
    unsigned char* ring_raw = smem_raw + (((size_t)9 * n * (sizeof(double) + sizeof(KT)) + 31) / 32) * 32;
    double* ringd = reinterpret_cast<double*>(ring_raw);
    KT* ringk = reinterpret_cast<KT*>(ring_raw);
    constexpr bool DF = std::is_same<KT, float>::value;   // double-float state
    // float offset of the lo planes of the FP32-mode setup ring (the ring's upper half)
    const int ring_lo = FINE_SLOTS * (a.TY + 2) * n;
    (void)ringd;
    // per-job constants (a launch can hold subintervals of several problems on the same
    // grid, see FineJob); set by load_job
    const double h = a.g.h;
    const double inv2h = 0.5 / h;
    double dt = 0.0, epsh2 = 0.0;
    KT c1 = (KT)0, c0 = (KT)1;
    const KT* bpk = nullptr;   // stored velocity perturbation (FINE_MODE_IMPLICIT_PERT)
    KT kp = (KT)0;             // its Krylov scale dt / (2h)
    (void)bpk;
    (void)kp;

    KT* Wk = reinterpret_cast<KT*>(a.ws) + (size_t)g * FINE_NVEC * Ng;
    KT* delta = Wk;
    KT* r = Wk + Ng;
    KT* rh = Wk + 2 * Ng;
    KT* p0 = Wk + 3 * Ng;
    KT* p1 = Wk + 4 * Ng;
    KT* v0 = Wk + 5 * Ng;
    KT* v1 = Wk + 6 * Ng;
    KT* t = Wk + 7 * Ng;
    double* ust = a.ust + (size_t)g * 2 * Ng;
    unsigned* bar = a.bar + 2 * g;
    double* part = a.part;  // [2][4][grid]
    const int g0 = g * G;
    int ph = 0;

    // Velocity terms: b_x = T_xy[y] + T_xz[z], b_y = T_yx[x] + T_yz[z], b_z = T_zx[x] + T_zy[y],
    // pre-scaled by dt/(2h) for the Krylov operator.  x-terms per thread, y-terms per owned
    // row slot (set per tile), z-terms per plane.
    KT ky_x[W], kz_x[W];
    int cur_job = -1;
    auto load_job = [&](int jb) {
        const FineJob& J = a.jobs[jb];
        __syncthreads();   // nobody reads the previous job's tables any more
        for (int i = threadIdx.x; i < 6 * n; i += blockDim.x) {
            const double v = J.tab[i];
            tabd[i] = v;
            tabk[i] = (KT)(v * J.dt * 0.5 / h);
        }
        __syncthreads();
        dt = J.dt;
        if constexpr (PT) {
            bpk = reinterpret_cast<const KT*>(J.pert);
            kp = (KT)(J.dt * 0.5 / h);
        }
        epsh2 = J.eps / (h * h);
        c1 = (KT)(dt * J.eps / (h * h));
        c0 = (KT)(1.0 + 6.0 * dt * J.eps / (h * h));
#pragma unroll
        for (int e = 0; e < W; ++e) {
            ky_x[e] = tabk[TYX * n + x0 + e];
            kz_x[e] = tabk[TZX * n + x0 + e];
        }
        cur_job = jb;
    };
    // Time-dependent flows: the tables of b(t_new) = c0 b^0 + c1 b^1 and of the forcing
    // part c0 g^0 + c1 g^1 for the step ending at t_new (the implicit step evaluates L and
    // f at the new time).  Every reader of the previous tables has passed a barrier.
    auto step_tables = [&](const FineJob& J, double t_new) {
        if (threadIdx.x == 0) {
            double q0, q1;
            flow_coeffs(J.kind, J.w, t_new, q0, q1);
            sh.c0 = q0;
            sh.c1 = q1;
        }
        __syncthreads();
        const double q0 = sh.c0, q1 = sh.c1;
        const double* T1 = J.tab + (size_t)TAB_B1 * n;
        const double* Gt = J.tab + (size_t)TAB_G * n;
        for (int i = threadIdx.x; i < 6 * n; i += blockDim.x) {
            const double v = q0 * J.tab[i] + q1 * T1[i];
            tabd[i] = v;
            tabk[i] = (KT)(v * dt * 0.5 / h);
        }
        for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
            const double v = J.no_forcing ? 0.0 : q0 * Gt[i] + q1 * Gt[3 * n + i];
            ftd[i] = v;
            ftk[i] = (KT)v;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < W; ++e) {
            ky_x[e] = tabk[TYX * n + x0 + e];
            kz_x[e] = tabk[TZX * n + x0 + e];
        }
    };
    KT kx_y[KS], kz_y[KS];
    KT kx_z = 0, ky_z = 0;
    auto tile_terms = [&](int y0) {
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int y = min(y0 + ty + k * RP, n - 1);
            kx_y[k] = tabk[TXY * n + y];
            kz_y[k] = tabk[TZY * n + y];
        }
    };
    auto plane_terms = [&](int z) {
        kx_z = tabk[TXZ * n + z];
        ky_z = tabk[TYZ * n + z];
    };

    // The x +- 1 neighbours of the W points: shifts of the centre vector plus one edge
    // value on each side read from the ring row.
    auto shift = [&](const auto* row, const auto& c, auto& xp, auto& xm) {
#pragma unroll
        for (int e = 0; e < W - 1; ++e) {
            xp.v[e] = c.v[e + 1];
            xm.v[e + 1] = c.v[e];
        }
        xp.v[W - 1] = row[xr];
        xm.v[0] = row[xl];
    };

    // ---- tile march for stencil phases (ring of FINE_SLOTS planes, one barrier per
    // FINE_PLANES planes):
    //   load(i) -> Raw            inputs of the operand at the W points from index i
    //   opnd(Raw) -> Vec          operand values written into the ring
    //   own(i) -> Own             inputs the output needs at owned points
    //   out(i, k, y, Own, rowc, rowzp, rowzm)   per owned W points (k: row slot); rowc is
    //                             the ring row of the points, rowzp / rowzm the rows above /
    //                             below in z; rowc +- n are the y neighbours
    // Plane p lives in slot (p - zlo + 1) mod FINE_SLOTS.  A round at z commits planes
    // z+1 .. z+np (np <= PL), then the barrier, then the stencils of planes z .. z+np-1
    // read planes z-1 .. z+np.  A thread that runs ahead can only reach the commits of
    // the next round, planes z+np+1 .. z+2np, whose slots differ from those of z-1 .. z+np
    // as long as 2 PL + 2 <= FINE_SLOTS; the next barrier stops it there.
    //   pipe                       true: prefetch the next round's first plane during the
    //                              stencils; false: load each plane just before committing
    //                              it (fewer live registers)
    auto march = [&](bool pipe, auto* ring, auto&& load, auto&& opnd, auto&& own, auto&& out) {
        using Raw = decltype(load(0));
        using Own = decltype(own(0));
        constexpr int PL = FINE_PLANES, NSL = FINE_SLOTS;
        for (int tt = t_lo; tt < t_hi; ++tt) {
            int y0, zlo, zhi;
            geo.tile(tt, y0, zlo, zhi);
            tile_terms(y0);
            int fidx[KF];
#pragma unroll
            for (int k = 0; k < KF; ++k) {
                const int rr = ty + k * RP;
                int y = y0 + rr - 1;
                y = (y < 0) ? y + n : (y >= n ? y - n : y);
                fidx[k] = (rr < RW) ? y * n + x0 : -1;   // in-plane offset, -1: no row
            }
            Raw pre[KF];
            Own opre[KS];
            auto prefetch = [&](int zp) {
                const int zz = (zp < 0) ? zp + n : (zp >= n ? zp - n : zp);
#pragma unroll
                for (int k = 0; k < KF; ++k)
                    if (fidx[k] >= 0) pre[k] = load(zz * n2 + fidx[k]);
            };
            auto own_of = [&](int z, Own (&dst)[KS]) {
#pragma unroll
                for (int k = 0; k < KS; ++k)
                    if (ty + k * RP < TY) dst[k] = own(z * n2 + (y0 + ty + k * RP) * n + x0);
            };
            auto slot = [&](int p) { return (p - zlo + 1) % NSL; };
            auto commit = [&](int sl) {
#pragma unroll
                for (int k = 0; k < KF; ++k) {
                    const int rr = ty + k * RP;
                    if (fidx[k] < 0) continue;
                    auto* dst = ring + (sl * RW + rr) * n + x0;
                    const auto val = opnd(pre[k]);
                    if constexpr (is_hilo<std::decay_t<decltype(val)>>::value) {
                        vstore(dst, val.hi);
                        vstore(dst + ring_lo, val.lo);
                    } else if constexpr (is_ophilo<std::decay_t<decltype(val)>>::value) {
                        vstore(dst, val.op);
                        vstore(dst + ring_lo, val.hi);
                        vstore(dst + 2 * ring_lo, val.lo);
                    } else {
                        vstore(dst, val);
                    }
                }
            };
            prefetch(zlo - 1);
            commit(0);
            prefetch(zlo);
            commit(1);
            if (pipe) {
                prefetch(zlo + 1);
                own_of(zlo, opre);
            }
            for (int z = zlo; z < zhi; z += PL) {
                const int np = min(PL, zhi - z);
#pragma unroll
                for (int q = 1; q <= PL; ++q) {
                    if (q > np) break;
                    if (!pipe || q > 1) prefetch(z + q);
                    commit(slot(z + q));
                }
                __syncthreads();
                Own cur[PL][KS];
                if (pipe) {
#pragma unroll
                    for (int k = 0; k < KS; ++k) cur[0][k] = opre[k];
#pragma unroll
                    for (int q = 1; q < PL; ++q)
                        if (q < np) own_of(z + q, cur[q]);
                    if (z + np < zhi) {
                        prefetch(z + np + 1);
                        own_of(z + np, opre);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < PL; ++q)
                        if (q < np) own_of(z + q, cur[q]);
                }
#pragma unroll
                for (int q = 0; q < PL; ++q) {
                    if (q >= np) break;
                    const int zq = z + q;
                    const int sc = slot(zq), sp = slot(zq + 1), sm = slot(zq - 1);
                    plane_terms(zq);
#pragma unroll
                    for (int k = 0; k < KS; ++k) {
                        const int rr = ty + k * RP;
                        if (rr >= TY) continue;
                        out(zq * n2 + (y0 + rr) * n + x0, k, y0 + rr, cur[q][k], ring + (sc * RW + rr + 1) * n,
                            ring + (sp * RW + rr + 1) * n, ring + (sm * RW + rr + 1) * n);
                    }
                }
            }
            __syncthreads();   // the next tile's prologue rewrites slots 0 and 1
        }
    };
    // ---- pointwise loop over owned points, one plane of KS rows at a time
    auto owned = [&](auto&& load, auto&& fn) {
        using Raw = decltype(load(0));
        for (int tt = t_lo; tt < t_hi; ++tt) {
            int y0, zlo, zhi;
            geo.tile(tt, y0, zlo, zhi);
            for (int z = zlo; z < zhi; ++z) {
                Raw v[KS];
#pragma unroll
                for (int k = 0; k < KS; ++k)
                    if (ty + k * RP < TY) v[k] = load(z * n2 + (y0 + ty + k * RP) * n + x0);
#pragma unroll
                for (int k = 0; k < KS; ++k)
                    if (ty + k * RP < TY) fn(z * n2 + (y0 + ty + k * RP) * n + x0, v[k]);
            }
        }
    };
    // The 7-point operand values of the W points from ring rows (vector loads).
    auto nb7 = [&](const auto* rowc, const auto* rowzp, const auto* rowzm) {
        using T = std::remove_const_t<std::remove_pointer_t<decltype(rowc)>>;
        Nb7<T, W> o;
        o.c = vload<T, W>(rowc + x0);
        shift(rowc, o.c, o.xp, o.xm);
        o.yp = vload<T, W>(rowc + n + x0);
        o.ym = vload<T, W>(rowc - n + x0);
        o.zp = vload<T, W>(rowzp + x0);
        o.zm = vload<T, W>(rowzm + x0);
        return o;
    };
    // The stored perturbation at the W points from index i (FINE_MODE_IMPLICIT_PERT).  It is
    // loaded where the stencil uses it, not one plane ahead with the other owned-point
    // inputs: its 3 W registers held across the march made the instantiation spill.
    auto load_pert = [&](int i) -> PertV<KT, W, PT> {
        PertV<KT, W, PT> o;
        if constexpr (PT) {
            o.x = vload<KT, W>(bpk + i);
            o.y = vload<KT, W>(bpk + Ng + i);
            o.z = vload<KT, W>(bpk + 2 * Ng + i);
        }
        return o;
    };
    // A = I + dt L at the W points of row slot k (pb: the perturbation there)
    auto applyA = [&](int k, const Vec<KT, W>& c, const Vec<KT, W>& xp, const Vec<KT, W>& xm,
                      const Vec<KT, W>& yp, const Vec<KT, W>& ym, const Vec<KT, W>& zp,
                      const Vec<KT, W>& zm, const PertV<KT, W, PT>& pb) -> Vec<KT, W> {
        Vec<KT, W> o;
#pragma unroll
        for (int e = 0; e < W; ++e) {
            KT ax = kx_y[k] + kx_z;
            KT ay = ky_x[e] + ky_z;
            KT az = kz_x[e] + kz_y[k];
            if constexpr (PT) {
                ax += kp * pb.x.v[e];
                ay += kp * pb.y.v[e];
                az += kp * pb.z.v[e];
            }
            o.v[e] = c0 * c.v[e] + (ax - c1) * xp.v[e] - (ax + c1) * xm.v[e] + (ay - c1) * yp.v[e] -
                     (ay + c1) * ym.v[e] + (az - c1) * zp.v[e] - (az + c1) * zm.v[e];
        }
        return o;
    };
    using VK = Vec<KT, W>;
    using VD = Vec<double, W>;

    for (int b = g; b < a.B; b += a.numGroups) {
        // job of item b and its index lb within the job
        int jb = 0, lb = b;
        while (jb + 1 < a.njobs && lb >= a.jobs[jb].B) lb -= a.jobs[jb++].B;
        if (jb != cur_job) load_job(jb);
        const FineJob& J = a.jobs[jb];
        const int S = J.S, dM = J.dM, n_snap = J.n_snap;
        const double* u_in = J.u_in + (size_t)lb * Ng;
        double* snap_b = J.snap ? reinterpret_cast<double*>(J.snap) + (size_t)lb * n_snap * Ng : nullptr;
        long long its_total = 0;
        int its_max = 0;
        bool dvalid = false;
        __syncthreads();
        if (threadIdx.x == 0) sh.status = 0;

        const bool tdep = RK ? (J.tdep != 0) : (MODE == FINE_MODE_IMPLICIT_TD);
        const double t_item = J.t0 + lb * J.DeltaT;   // start of this subinterval
        if constexpr (RK) {
            // ---------------- explicit alternative: classical RK4 on u' = f(t) - L(t) u.
            // Stage s is the residual pass of the implicit setup on the operand
            // v_s = u + a_s kappa_{s-1}: kappa_s = dt (f(t_s) - L(t_s) v_s), a = 0, 1/2,
            // 1/2, 1 at t_s = t, t + dt/2, t + dt/2, t + dt; the last stage forms
            // u_new = u + (kappa_1 + 2 kappa_2 + 2 kappa_3 + kappa_4) / 6 at owned points.
            KT* kap[3] = {delta, r, rh};
            const KT dtf = (KT)dt;
            for (int j = 1; j <= S; ++j) {
                const double tj = t_item + (j - 1) * dt;
                const double* Pd = (j == 1) ? u_in : ust + (size_t)((j - 1) & 1) * Ng;   // u_{j-1}
                double* Wd = (j == S) ? nullptr : ust + (size_t)(j & 1) * Ng;            // u_j
                double* outS = (j == S) ? J.u_out + (size_t)lb * Ng : nullptr;
                double* snap_prev = (snap_b && (j - 1) % dM == 0 && (j - 1) / dM < n_snap)
                                        ? snap_b + (size_t)((j - 1) / dM) * Ng : nullptr;
                double* snap_new = (j == S && snap_b && S % dM == 0 && S / dM < n_snap)
                                       ? snap_b + (size_t)(S / dM) * Ng : nullptr;
                for (int stg = 0; stg < 4; ++stg) {
                    const double ts = tj + (stg == 0 ? 0.0 : (stg == 3 ? dt : 0.5 * dt));
                    const KT ca = (KT)(stg == 0 ? 0.0 : (stg == 3 ? 1.0 : 0.5));
                    if (tdep) step_tables(J, ts);
                    const KT* kin = stg ? kap[stg - 1] : nullptr;
                    KT* kout = stg < 3 ? kap[stg] : nullptr;
                    const bool last = stg == 3;
                    if constexpr (!DF) {
                        const double* fp = J.f;
                        march(false, ringd,
                              [&](int i) -> RawSetup<double, KT, W> {
                                  RawSetup<double, KT, W> o;
                                  o.u = vload<double, W>(Pd + i);
                                  if (kin) o.d = vload<KT, W>(kin + i);
                                  else {
#pragma unroll
                                      for (int e = 0; e < W; ++e) o.d.v[e] = (KT)0;
                                  }
                                  return o;
                              },
                              [&](const RawSetup<double, KT, W>& v) -> VD {
                                  VD o;
#pragma unroll
                                  for (int e = 0; e < W; ++e) o.v[e] = v.u.v[e] + (double)ca * (double)v.d.v[e];
                                  return o;
                              },
                              [&](int) -> NoOwn { return NoOwn{}; },
                              [&](int i, int, int y, const NoOwn&, const double* rowc, const double* rowzp,
                                  const double* rowzm) {
                                  const int z = i / n2;
                                  const double bx = tabd[TXY * n + y] + tabd[TXZ * n + z];
                                  const double byz = tabd[TYZ * n + z], bzy = tabd[TZY * n + y];
#pragma unroll 1
                                  for (int e = 0; e < W; ++e) {
                                      const int x = x0 + e;
                                      const int xp = (e == W - 1) ? xr : x + 1;
                                      const int xm = (e == 0) ? xl : x - 1;
                                      const double c = rowc[x];
                                      const double uxp = rowc[xp], uxm = rowc[xm];
                                      const double uyp = rowc[n + x], uym = rowc[x - n];
                                      const double uzp = rowzp[x], uzm = rowzm[x];
                                      const double by = tabd[TYX * n + x] + byz;
                                      const double bz = tabd[TZX * n + x] + bzy;
                                      const double adv = bx * (uxp - uxm) + by * (uyp - uym) + bz * (uzp - uzm);
                                      const double lap = (uxp + uxm) + (uyp + uym) + (uzp + uzm) - 6.0 * c;
                                      double fi = fp ? fp[i + e] : 0.0;
                                      if (tdep) fi += ftd[x] + ftd[n + y] + ftd[2 * n + z];
                                      const double kp = dt * (fi - (adv * inv2h - epsh2 * lap));
                                      if (stg == 0 && snap_prev) snap_prev[i + e] = c;
                                      if (!last) {
                                          kout[i + e] = (KT)kp;
                                      } else {
                                          const double un = Pd[i + e] +
                                              ((double)kap[0][i + e] + 2.0 * (double)kap[1][i + e] +
                                               2.0 * (double)kap[2][i + e] + kp) / 6.0;
                                          if (Wd) Wd[i + e] = un;
                                          if (outS) outS[i + e] = un;
                                          if (snap_new) snap_new[i + e] = un;
                                      }
                                  }
                              });
                    } else {
                        const float2* Pf = (j == 1) ? nullptr : reinterpret_cast<const float2*>(Pd);
                        float2* Wf = reinterpret_cast<float2*>(Wd);
                        const float* ff = J.f32;
                        float* ringh = reinterpret_cast<float*>(ring_raw);
                        march(true, ringh,
                              [&](int i) -> RawSetup<float2, KT, W> {
                                  RawSetup<float2, KT, W> o;
                                  if (Pf) o.u = vload<float2, W>(Pf + i);
                                  else {
                                      const VD ud = vload<double, W>(u_in + i);
#pragma unroll
                                      for (int e = 0; e < W; ++e) o.u.v[e] = df_split(ud.v[e]);
                                  }
                                  if (kin) o.d = vload<KT, W>(kin + i);
                                  else {
#pragma unroll
                                      for (int e = 0; e < W; ++e) o.d.v[e] = (KT)0;
                                  }
                                  return o;
                              },
                              [&](const RawSetup<float2, KT, W>& v) -> HiLo<W> {
                                  HiLo<W> o;
#pragma unroll
                                  for (int e = 0; e < W; ++e) {
                                      const float2 u = df_add(v.u.v[e], ca * v.d.v[e]);
                                      o.hi.v[e] = u.x;
                                      o.lo.v[e] = u.y;
                                  }
                                  return o;
                              },
                              [&](int i) -> VK {
                                  VK fo;
                                  if (ff) fo = vload<KT, W>(ff + i);
                                  else {
#pragma unroll
                                      for (int e = 0; e < W; ++e) fo.v[e] = (KT)0;
                                  }
                                  return fo;
                              },
                              [&](int i, int k, int yy, const VK& fv0, const float* rowc, const float* rowzp,
                                  const float* rowzm) {
                                  const auto q = nb7(rowc, rowzp, rowzm);
                                  VK fv = fv0;
                                  if (tdep) {
                                      const KT fyz = ftk[n + yy] + ftk[2 * n + i / n2];
#pragma unroll
                                      for (int e = 0; e < W; ++e) fv.v[e] += ftk[x0 + e] + fyz;
                                  }
                                  const KT ax = kx_y[k] + kx_z;
                                  VK kv;
#pragma unroll
                                  for (int e = 0; e < W; ++e) {
                                      const float c = q.c.v[e];
                                      const KT ay = ky_x[e] + ky_z;
                                      const KT az = kz_x[e] + kz_y[k];
                                      const KT dx = __fsub_rn(q.xp.v[e], q.xm.v[e]);
                                      const KT dy = __fsub_rn(q.yp.v[e], q.ym.v[e]);
                                      const KT dz = __fsub_rn(q.zp.v[e], q.zm.v[e]);
                                      const KT sx = __fsub_rn(__fsub_rn(q.xp.v[e], c), __fsub_rn(c, q.xm.v[e]));
                                      const KT sy = __fsub_rn(__fsub_rn(q.yp.v[e], c), __fsub_rn(c, q.ym.v[e]));
                                      const KT sz = __fsub_rn(__fsub_rn(q.zp.v[e], c), __fsub_rn(c, q.zm.v[e]));
                                      kv.v[e] = dtf * fv.v[e] - (ax * dx + ay * dy + az * dz) + c1 * ((sx + sy) + sz);
                                  }
                                  if (stg == 0 && snap_prev) {
                                      const VK clo = vload<float, W>(rowc + ring_lo + x0);
                                      VD sd;
#pragma unroll
                                      for (int e = 0; e < W; ++e) sd.v[e] = df_value_bits(q.c.v[e], clo.v[e]);
                                      vstore(snap_prev + i, sd);
                                  }
                                  if (!last) {
                                      vstore(kout + i, kv);
                                      return;
                                  }
                                  // u_new = u + (k1 + 2 k2 + 2 k3 + k4) / 6, the state as a float pair
                                  Vec<float2, W> u2;
                                  if (Pf) u2 = vload<float2, W>(Pf + i);
                                  else {
                                      const VD ud = vload<double, W>(u_in + i);
#pragma unroll
                                      for (int e = 0; e < W; ++e) u2.v[e] = df_split(ud.v[e]);
                                  }
                                  const VK k1 = vload<KT, W>(kap[0] + i), k2 = vload<KT, W>(kap[1] + i);
                                  const VK k3 = vload<KT, W>(kap[2] + i);
#pragma unroll
                                  for (int e = 0; e < W; ++e)
                                      u2.v[e] = df_add(u2.v[e], (k1.v[e] + 2.0f * k2.v[e] + 2.0f * k3.v[e] + kv.v[e]) *
                                                                    (1.0f / 6.0f));
                                  if (Wf) vstore(Wf + i, u2);
                                  if (outS || snap_new) {
                                      VD ud;
#pragma unroll
                                      for (int e = 0; e < W; ++e) ud.v[e] = df_value_bits(u2.v[e].x, u2.v[e].y);
                                      if (outS) vstore(outS + i, ud);
                                      if (snap_new) vstore(snap_new + i, ud);
                                  }
                              });
                    }
                    if (!group_barrier(bar, G, a.spin_limit, a.err)) return;
                }
            }
        } else {
        for (int j = 1; j <= S; ++j) {
            if (tdep) step_tables(J, t_item + j * dt);
            // ---------------- setup: u_{j-1} = u_{j-2} + delta ; r = rhat = dt (f - L u_{j-1})
            const double* P = (j <= 2) ? u_in : ust + (size_t)((j - 2) & 1) * Ng;
            double* Wt = (j >= 2) ? ust + (size_t)((j - 1) & 1) * Ng : nullptr;
            const bool use_d = (j >= 2) && dvalid;
            // FP32 mode: BiCGStab starts from the previous increment (the FP64 mode starts
            // from 0, i.e. from u_{j-1}, like the plain definition)
            const bool xg = DF && use_d;
            double* snap_j = nullptr;
            if (snap_b && (j - 1) % dM == 0 && (j - 1) / dM < n_snap)
                snap_j = snap_b + (size_t)((j - 1) / dM) * Ng;
            const double* fp = J.f;
            Acc<KT, 2> acc;
            acc.init();
            if constexpr (!DF) {
                march(false, ringd,
                      [&](int i) -> RawSetup<double, KT, W> {
                          RawSetup<double, KT, W> o;
                          o.u = vload<double, W>(P + i);
                          if (use_d) o.d = vload<KT, W>(delta + i);
                          else {
#pragma unroll
                              for (int e = 0; e < W; ++e) o.d.v[e] = (KT)0;
                          }
                          return o;
                      },
                      [&](const RawSetup<double, KT, W>& v) -> VD {
                          VD o;
#pragma unroll
                          for (int e = 0; e < W; ++e) o.v[e] = v.u.v[e] + (double)v.d.v[e];
                          return o;
                      },
                      [&](int) -> NoOwn { return NoOwn{}; },
                      [&](int i, int, int y, const NoOwn&, const double* rowc, const double* rowzp,
                          const double* rowzm) {
                          const int z = i / n2;
                          const double bx = tabd[TXY * n + y] + tabd[TXZ * n + z];
                          const double byz = tabd[TYZ * n + z], bzy = tabd[TZY * n + y];
                          // one point at a time: the FP64 stencil of all W points at once
                          // would raise the register count of the whole kernel
#pragma unroll 1
                          for (int e = 0; e < W; ++e) {
                              const int x = x0 + e;
                              const int xp = (e == W - 1) ? xr : x + 1;
                              const int xm = (e == 0) ? xl : x - 1;
                              const double c = rowc[x];
                              const double uxp = rowc[xp], uxm = rowc[xm];
                              const double uyp = rowc[n + x], uym = rowc[x - n];
                              const double uzp = rowzp[x], uzm = rowzm[x];
                              double bxe = bx;
                              double by = tabd[TYX * n + x] + byz;
                              double bz = tabd[TZX * n + x] + bzy;
                              if constexpr (PT) {
                                  const double* bpd = reinterpret_cast<const double*>(bpk);
                                  bxe += bpd[i + e];
                                  by += bpd[Ng + i + e];
                                  bz += bpd[2 * Ng + i + e];
                              }
                              const double adv = bxe * (uxp - uxm) + by * (uyp - uym) + bz * (uzp - uzm);
                              const double lap = (uxp + uxm) + (uyp + uym) + (uzp + uzm) - 6.0 * c;
                              const double Lu = adv * inv2h - epsh2 * lap;
                              double fi = fp ? fp[i + e] : 0.0;
                              if (tdep) fi += ftd[x] + ftd[n + y] + ftd[2 * n + z];
                              const KT rk = (KT)(dt * (fi - Lu));
                              if (Wt) Wt[i + e] = c;
                              if (snap_j) snap_j[i + e] = c;
                              r[i + e] = rk;
                              rh[i + e] = rk;
                              const double bi = c + dt * fi;
                              acc.f[0] += rk * rk;
                              acc.f[1] += (KT)(bi * bi);
                          }
                          acc.tick();
                      });
            } else {
                // double-float state: the same residual, FP32 arithmetic only
                const float2* Pf = (j <= 2) ? nullptr : reinterpret_cast<const float2*>(P);
                float2* Wf = reinterpret_cast<float2*>(Wt);
                const float* ff = J.f32;
                const KT dtf = (KT)dt;
                // residual from a one-float operand (exact neighbour differences, Sterbenz);
                // the neglected dt L of its rounding is ~1e-7 of dt L(u), at the level of
                // the solver tolerance; lo enters the state update and the snapshots.
                // Initial guess: the previous increment (xg), i.e. the operand
                // u_{j-1} + delta and r = dt (f - L (u_{j-1} + delta)) - delta; else 0.
                float* ringh = reinterpret_cast<float*>(ring_raw);
                march(true, ringh,
                      [&](int i) -> RawSetup<float2, KT, W> {
                          RawSetup<float2, KT, W> o;
                          if (Pf) o.u = vload<float2, W>(Pf + i);
                          else {
                              const VD ud = vload<double, W>(u_in + i);
#pragma unroll
                              for (int e = 0; e < W; ++e) o.u.v[e] = df_split(ud.v[e]);
                          }
                          if (use_d) o.d = vload<KT, W>(delta + i);
                          else {
#pragma unroll
                              for (int e = 0; e < W; ++e) o.d.v[e] = (KT)0;
                          }
                          return o;
                      },
                      [&](const RawSetup<float2, KT, W>& v) -> OpHiLo<W> {
                          OpHiLo<W> o;
#pragma unroll
                          for (int e = 0; e < W; ++e) {
                              const float2 u = df_add(v.u.v[e], v.d.v[e]);
                              o.hi.v[e] = u.x;
                              o.lo.v[e] = u.y;
                              // u.x + (u.y + d): within ulp(op) / 2 of u_{j-1} + delta
                              o.op.v[e] = xg ? u.x + (u.y + v.d.v[e]) : u.x;
                          }
                          return o;
                      },
                      [&](int i) -> OwnFD<KT, W, PT> {
                          OwnFD<KT, W, PT> o;
                          if (ff) o.f = vload<KT, W>(ff + i);
                          else {
#pragma unroll
                              for (int e = 0; e < W; ++e) o.f.v[e] = (KT)0;
                          }
                          if (xg) o.d = vload<KT, W>(delta + i);
                          else {
#pragma unroll
                              for (int e = 0; e < W; ++e) o.d.v[e] = (KT)0;
                          }
                          return o;
                      },
                      [&](int i, int k, int yy, const OwnFD<KT, W, PT>& ow, const float* rowc, const float* rowzp,
                          const float* rowzm) {
                          const auto q = nb7(rowc, rowzp, rowzm);
                          const VK chi = vload<float, W>(rowc + ring_lo + x0);
                          const VK clo = vload<float, W>(rowc + 2 * ring_lo + x0);
                          const PertV<KT, W, PT> pbv = load_pert(i);
                          (void)pbv;
                          VK fv = ow.f;
                          if (tdep) {
                              const KT fyz = ftk[n + yy] + ftk[2 * n + i / n2];
#pragma unroll
                              for (int e = 0; e < W; ++e) fv.v[e] += ftk[x0 + e] + fyz;
                          }
                          VK rv;
#pragma unroll
                          for (int e = 0; e < W; ++e) {
                              const float c = q.c.v[e];
                              KT ax = kx_y[k] + kx_z;
                              KT ay = ky_x[e] + ky_z;
                              KT az = kz_x[e] + kz_y[k];
                              if constexpr (PT) {
                                  ax += kp * pbv.x.v[e];
                                  ay += kp * pbv.y.v[e];
                                  az += kp * pbv.z.v[e];
                              }
                              const KT dx = __fsub_rn(q.xp.v[e], q.xm.v[e]);
                              const KT dy = __fsub_rn(q.yp.v[e], q.ym.v[e]);
                              const KT dz = __fsub_rn(q.zp.v[e], q.zm.v[e]);
                              const KT sx = __fsub_rn(__fsub_rn(q.xp.v[e], c), __fsub_rn(c, q.xm.v[e]));
                              const KT sy = __fsub_rn(__fsub_rn(q.yp.v[e], c), __fsub_rn(c, q.ym.v[e]));
                              const KT sz = __fsub_rn(__fsub_rn(q.zp.v[e], c), __fsub_rn(c, q.zm.v[e]));
                              const KT lap = (sx + sy) + sz;
                              // r = dt (f - L op) - delta: dt b.grad(op) = a . (2h grad op),
                              // dt eps lap / h^2 = c1 lap
                              const KT rk = (dtf * fv.v[e] - (ax * dx + ay * dy + az * dz) + c1 * lap) - ow.d.v[e];
                              rv.v[e] = rk;
                              const KT bi = chi.v[e] + dtf * fv.v[e];
                              acc.f[0] += rk * rk;
                              acc.f[1] += bi * bi;
                          }
                          vstore(r + i, rv);
                          vstore(rh + i, rv);
                          if (Wf) {
                              Vec<float2, W> u2;
#pragma unroll
                              for (int e = 0; e < W; ++e) u2.v[e] = make_float2(chi.v[e], clo.v[e]);
                              vstore(Wf + i, u2);
                          }
                          if (snap_j) {
                              VD sd;
#pragma unroll
                              for (int e = 0; e < W; ++e) sd.v[e] = df_value_bits(chi.v[e], clo.v[e]);
                              vstore(snap_j + i, sd);
                          }
                          acc.tick();
                      });
            }
            {
                acc.flush();
                cta_sum<KT, 2>(acc, sh.red);
                if (threadIdx.x == 0) {
                    part[(size_t)((ph & 1) * 4 + 0) * grid + blockIdx.x] = acc.d[0];
                    part[(size_t)((ph & 1) * 4 + 1) * grid + blockIdx.x] = acc.d[1];
                }
            }
            if (!group_barrier(bar, G, a.spin_limit, a.err)) return;
            group_sums(part + (size_t)(ph & 1) * 4 * grid, grid, g0, G, 2, sh.sums, [&](const double* s) {
                const double rr0 = s[0], bb = s[1];
                sh.thr = J.tol * sqrt(bb);
                int conv = sqrt(rr0) <= sh.thr;
                if (!isfinite(rr0) || !isfinite(bb)) { sh.status = DERR_NONFINITE; conv = 1; }
                sh.flag = conv;
                sh.rho = rr0;
                sh.alpha = 1.0;
                sh.omega = 1.0;
                sh.beta = 0.0;
            });
            ++ph;
            const bool conv = sh.flag != 0;
            int it = 0;
            while (!conv) {
                ++it;
                // ---------------- ph1: p = r + beta (p' - omega v'), v = A p
                KT* pn = (it & 1) ? p1 : p0;
                KT* po = (it & 1) ? p0 : p1;
                KT* vn = (it & 1) ? v1 : v0;
                KT* vo = (it & 1) ? v0 : v1;
                {
                    const KT bk = (KT)sh.beta, ok = (KT)sh.omega;
                    const bool first = (it == 1);
                    Acc<KT, 1> acc;
                    acc.init();
                    march(true, ringk,
                          [&](int i) -> RawP<KT, W> {
                              RawP<KT, W> o;
                              o.r = vload<KT, W>(r + i);
                              if (!first) {
                                  o.p = vload<KT, W>(po + i);
                                  o.v = vload<KT, W>(vo + i);
                              } else {
#pragma unroll
                                  for (int e = 0; e < W; ++e) { o.p.v[e] = (KT)0; o.v.v[e] = (KT)0; }
                              }
                              return o;
                          },
                          [&](const RawP<KT, W>& v) -> VK {
                              VK o;
#pragma unroll
                              for (int e = 0; e < W; ++e) o.v[e] = v.r.v[e] + bk * (v.p.v[e] - ok * v.v.v[e]);
                              return o;
                          },
                          [&](int i) -> OwnH<KT, W, PT> { return {vload<KT, W>(rh + i), {}}; },
                          [&](int i, int k, int, const OwnH<KT, W, PT>& ow, const KT* rowc, const KT* rowzp,
                              const KT* rowzm) {
                              const VK& rhv = ow.h;
                              const auto q7 = nb7(rowc, rowzp, rowzm);
                              const VK av = applyA(k, q7.c, q7.xp, q7.xm, q7.yp, q7.ym, q7.zp, q7.zm, load_pert(i));
                              vstore(pn + i, q7.c);
                              vstore(vn + i, av);
#pragma unroll
                              for (int e = 0; e < W; ++e) acc.f[0] += rhv.v[e] * av.v[e];
                              acc.tick();
                          });
                    acc.flush();
                    cta_sum<KT, 1>(acc, sh.red);
                    if (threadIdx.x == 0) part[(size_t)((ph & 1) * 4) * grid + blockIdx.x] = acc.d[0];
                }
                if (!group_barrier(bar, G, a.spin_limit, a.err)) return;
                group_sums(part + (size_t)(ph & 1) * 4 * grid, grid, g0, G, 1, sh.sums, [&](const double* s) {
                    const double rv = s[0];
                    if (rv == 0.0 || !isfinite(rv)) {
                        sh.status = isfinite(rv) ? DERR_BREAKDOWN : DERR_NONFINITE;
                        sh.flag = 1;
                    } else {
                        sh.alpha = sh.rho / rv;
                        sh.flag = 0;
                    }
                });
                ++ph;
                if (sh.flag) {
                    --it;
                    break;
                }
                // ---------------- ph2: s = r - alpha v, t = A s
                {
                    const KT al = (KT)sh.alpha;
                    Acc<KT, 3> acc;
                    acc.init();
                    march(true, ringk,
                          [&](int i) -> RawS<KT, W> { return {vload<KT, W>(r + i), vload<KT, W>(vn + i)}; },
                          [&](const RawS<KT, W>& v) -> VK {
                              VK o;
#pragma unroll
                              for (int e = 0; e < W; ++e) o.v[e] = v.r.v[e] - al * v.v.v[e];
                              return o;
                          },
                          [&](int) -> NoOwn { return NoOwn{}; },
                          [&](int i, int k, int, const NoOwn&, const KT* rowc, const KT* rowzp,
                              const KT* rowzm) {
                              const auto q7 = nb7(rowc, rowzp, rowzm);
                              const VK tv = applyA(k, q7.c, q7.xp, q7.xm, q7.yp, q7.ym, q7.zp, q7.zm, load_pert(i));
                              vstore(t + i, tv);
#pragma unroll
                              for (int e = 0; e < W; ++e) {
                                  acc.f[0] += tv.v[e] * q7.c.v[e];
                                  acc.f[1] += tv.v[e] * tv.v[e];
                                  acc.f[2] += q7.c.v[e] * q7.c.v[e];
                              }
                              acc.tick();
                          });
                    acc.flush();
                    cta_sum<KT, 3>(acc, sh.red);
                    if (threadIdx.x == 0) {
                        for (int qq = 0; qq < 3; ++qq)
                            part[(size_t)((ph & 1) * 4 + qq) * grid + blockIdx.x] = acc.d[qq];
                    }
                }
                if (!group_barrier(bar, G, a.spin_limit, a.err)) return;
                group_sums(part + (size_t)(ph & 1) * 4 * grid, grid, g0, G, 3, sh.sums, [&](const double* s) {
                    const double ts = s[0], tt2 = s[1], ss = s[2];
                    const int half = sqrt(ss) <= sh.thr;
                    if (!half) {
                        if (tt2 == 0.0 || !isfinite(tt2)) {
                            sh.status = isfinite(tt2) ? DERR_BREAKDOWN : DERR_NONFINITE;
                            sh.omega = 0.0;
                        } else {
                            sh.omega = ts / tt2;
                            if (sh.omega == 0.0) sh.status = DERR_BREAKDOWN;
                        }
                    }
                    sh.flag = half;
                });
                ++ph;
                const bool half = sh.flag != 0;
                // ---------------- ph3: delta += alpha p + omega s ; r = s - omega t
                {
                    const KT al = (KT)sh.alpha, om = (KT)sh.omega;
                    const bool first = (it == 1) && !xg;   // delta holds the initial guess
                    const bool upd_r = !half && sh.status == 0;
                    Acc<KT, 2> acc;
                    acc.init();
                    // the update of the owned points from their six inputs
                    auto p3_fn = [&](int i, const Raw6<KT, W>& v) {
                        VK dn, rn;
#pragma unroll
                        for (int e = 0; e < W; ++e) {
                            const KT sc_ = v.r.v[e] - al * v.v.v[e];
                            dn.v[e] = v.d.v[e] + al * v.p.v[e] + om * sc_;
                            rn.v[e] = sc_ - om * v.t.v[e];
                            acc.f[0] += v.h.v[e] * rn.v[e];
                            acc.f[1] += rn.v[e] * rn.v[e];
                        }
                        vstore(delta + i, dn);
                        vstore(r + i, rn);
                        acc.tick();
                    };
                    bool staged3 = false;
                    if constexpr (DF && KS == 1) {
                        if (upd_r) {
                            // inputs of plane z staged by cp.async while planes z-2, z-1 are
                            // updated; each thread reads back only what it copied, so no
                            // barrier is needed; layout [slot][input][thread][W] (no bank
                            // conflicts).  The ring is idle in this phase.
                            staged3 = true;
                            constexpr int NS = FINE_PH3_SLOTS;
                            float* stg = reinterpret_cast<float*>(ring_raw);
                            const int nthr = blockDim.x;
                            const bool act = ty < TY;
                            auto sad = [&](int sl, int q) { return stg + ((size_t)(sl * 6 + q) * nthr + threadIdx.x) * W; };
                            for (int tt = t_lo; tt < t_hi; ++tt) {
                                int y0, zlo, zhi;
                                geo.tile(tt, y0, zlo, zhi);
                                const int rowoff = (y0 + ty) * n + x0;
                                auto issue = [&](int z, int sl) {
                                    if (act && z < zhi) {
                                        const long long i = (long long)z * n2 + rowoff;
                                        if (!first) cp_async_b<4 * W>(sad(sl, 0), delta + i);
                                        cp_async_b<4 * W>(sad(sl, 1), pn + i);
                                        cp_async_b<4 * W>(sad(sl, 2), r + i);
                                        cp_async_b<4 * W>(sad(sl, 3), vn + i);
                                        cp_async_b<4 * W>(sad(sl, 4), t + i);
                                        cp_async_b<4 * W>(sad(sl, 5), rh + i);
                                    }
                                    cp_async_commit_group();
                                };
#pragma unroll
                                for (int d = 0; d < NS - 1; ++d) issue(zlo + d, d);
                                int sl = 0;
                                for (int z = zlo; z < zhi; ++z) {
                                    // refill the slot of plane z - 1 (read last iteration)
                                    issue(z + NS - 1, sl == 0 ? NS - 1 : sl - 1);
                                    cp_async_wait_newest<NS - 1>();
                                    if (act) {
                                        Raw6<KT, W> v;
                                        if (!first) v.d = vload<float, W>(sad(sl, 0));
                                        else {
#pragma unroll
                                            for (int e = 0; e < W; ++e) v.d.v[e] = 0.0f;
                                        }
                                        v.p = vload<float, W>(sad(sl, 1));
                                        v.r = vload<float, W>(sad(sl, 2));
                                        v.v = vload<float, W>(sad(sl, 3));
                                        v.t = vload<float, W>(sad(sl, 4));
                                        v.h = vload<float, W>(sad(sl, 5));
                                        p3_fn(z * n2 + rowoff, v);
                                    }
                                    sl = (sl + 1 == NS) ? 0 : sl + 1;
                                }
                                cp_async_wait_newest<0>();
                            }
                        }
                    }
                    if (upd_r && !staged3) {
                        owned([&](int i) -> Raw6<KT, W> {
                                  Raw6<KT, W> o;
                                  if (!first) o.d = vload<KT, W>(delta + i);
                                  else {
#pragma unroll
                                      for (int e = 0; e < W; ++e) o.d.v[e] = (KT)0;
                                  }
                                  o.p = vload<KT, W>(pn + i);
                                  o.r = vload<KT, W>(r + i);
                                  o.v = vload<KT, W>(vn + i);
                                  o.t = vload<KT, W>(t + i);
                                  o.h = vload<KT, W>(rh + i);
                                  return o;
                              },
                              p3_fn);
                    } else if (!upd_r) {
                        owned([&](int i) -> RawP2<KT, W> {
                                  RawP2<KT, W> o;
                                  if (!first) o.d = vload<KT, W>(delta + i);
                                  else {
#pragma unroll
                                      for (int e = 0; e < W; ++e) o.d.v[e] = (KT)0;
                                  }
                                  o.p = vload<KT, W>(pn + i);
                                  return o;
                              },
                              [&](int i, const RawP2<KT, W>& v) {
                                  VK dn;
#pragma unroll
                                  for (int e = 0; e < W; ++e) dn.v[e] = v.d.v[e] + al * v.p.v[e];
                                  vstore(delta + i, dn);
                              });
                    }
                    acc.flush();
                    cta_sum<KT, 2>(acc, sh.red);
                    if (threadIdx.x == 0 && upd_r) {
                        part[(size_t)((ph & 1) * 4 + 0) * grid + blockIdx.x] = acc.d[0];
                        part[(size_t)((ph & 1) * 4 + 1) * grid + blockIdx.x] = acc.d[1];
                    }
                    if (!group_barrier(bar, G, a.spin_limit, a.err)) return;
                    if (!upd_r) break;
                    group_sums(part + (size_t)(ph & 1) * 4 * grid, grid, g0, G, 2, sh.sums, [&](const double* s) {
                        const double rho_new = s[0], rr1 = s[1];
                        int stop = 1;
                        if (!isfinite(rr1)) sh.status = DERR_NONFINITE;
                        else if (sqrt(rr1) <= sh.thr) {}
                        else if (rho_new == 0.0) sh.status = DERR_BREAKDOWN;
                        else if (it >= J.maxit) sh.status = DERR_NOT_CONVERGED;
                        else {
                            sh.beta = (rho_new / sh.rho) * (sh.alpha / sh.omega);
                            sh.rho = rho_new;
                            stop = 0;
                        }
                        sh.flag = stop;
                    });
                    ++ph;
                }
                if (sh.flag) break;
            }
            dvalid = it > 0 || xg;
            its_total += it;
            its_max = max(its_max, it);
            // a non-finite state would only propagate: skip the remaining steps
            if (sh.status == DERR_NONFINITE) break;
        }
        // ---------------- final: u_S = u_{S-1} + delta ; snapshot of u_S
        {
            const double* P = (S >= 2) ? ust + (size_t)((S - 1) & 1) * Ng : u_in;
            double* snap_S = (snap_b && S % dM == 0 && S / dM < n_snap)
                                 ? snap_b + (size_t)(S / dM) * Ng : nullptr;
            double* outp = J.u_out + (size_t)lb * Ng;
            const bool dv = dvalid;
            if constexpr (!DF) {
                owned([&](int i) -> RawF<double, KT, W> {
                          RawF<double, KT, W> o;
                          o.u = vload<double, W>(P + i);
                          if (dv) o.d = vload<KT, W>(delta + i);
                          else {
#pragma unroll
                              for (int e = 0; e < W; ++e) o.d.v[e] = (KT)0;
                          }
                          return o;
                      },
                      [&](int i, const RawF<double, KT, W>& v) {
                          VD u;
#pragma unroll
                          for (int e = 0; e < W; ++e) u.v[e] = v.u.v[e] + (double)v.d.v[e];
                          vstore(outp + i, u);
                          if (snap_S) vstore(snap_S + i, u);
                      });
            } else {
                const float2* Pf = (S >= 2) ? reinterpret_cast<const float2*>(P) : nullptr;
                owned([&](int i) -> RawF<float2, KT, W> {
                          RawF<float2, KT, W> o;
                          if (Pf) o.u = vload<float2, W>(Pf + i);
                          else {
                              const VD ud = vload<double, W>(u_in + i);
#pragma unroll
                              for (int e = 0; e < W; ++e) o.u.v[e] = df_split(ud.v[e]);
                          }
                          if (dv) o.d = vload<KT, W>(delta + i);
                          else {
#pragma unroll
                              for (int e = 0; e < W; ++e) o.d.v[e] = (KT)0;
                          }
                          return o;
                      },
                      [&](int i, const RawF<float2, KT, W>& v) {
                          VD u;
#pragma unroll
                          for (int e = 0; e < W; ++e) u.v[e] = df_value(df_add(v.u.v[e], v.d.v[e]));
                          vstore(outp + i, u);
                          if (snap_S) vstore(snap_S + i, u);
                      });
            }
        }
        }   // implicit Euler
        if (q == 0 && threadIdx.x == 0) {
            J.status[lb] = sh.status;
            J.its_total[lb] = (int)its_total;
            J.its_max[lb] = its_max;
        }
        // The next subinterval's first setup reads only its own input state (and the
        // ring), and writes r/rhat at owned points, which no CTA of this group reads
        // before the next barrier.
    }
}

// ------------------------------------------------------------------------------------
// Launch geometry.  W = 4 points per thread when n % 4 == 0, else 1.  A row has n/W
// lanes.  CTAs of at most 128 threads (RP rows a pass, one owned row a thread) when the
// tile keeps at least 8 rows: the kernel is latency-bound at 128 registers a thread, and
// small CTAs (4 an SM) let the groups of a launch fill nearly every CTA slot (64^3, 64
// subintervals: 9 CTAs a subinterval, 576 of 608 slots, where 256-thread CTAs fill 256 of
// 304; the fine sweep 63.1 -> 58.3 ms).  Otherwise RP is the largest divisor of n with
// RP * n/W <= 256 and a tile has TY = KS * RP rows (KS in {1, 2}), its FINE_SLOTS-plane
// ring (8 bytes a point) within 64 KB.
struct FineGeom {
    int W, lanes, RP, TY, KS, KF, threads;
    size_t smem;
};

inline FineGeom fine_geom(int n, bool fp32) {
    FineGeom g{};
    g.W = (n % 4 == 0) ? 4 : 1;
    g.lanes = n / g.W;
    int rp128 = 1;
    for (int rp = 1; rp <= n; ++rp)
        if (n % rp == 0 && rp * g.lanes <= 128) rp128 = rp;
    g.RP = 1;
    for (int rp = 1; rp <= n; ++rp)
        if (n % rp == 0 && rp * g.lanes <= 256) g.RP = rp;
    g.KS = 1;
    if (rp128 >= 8) {
        g.RP = rp128;
    } else if (n % (2 * g.RP) == 0 && 2 * g.RP <= 16 &&
               (size_t)FINE_SLOTS * (2 * g.RP + 2) * n * 8 <= 64 * 1024) {
        g.KS = 2;
    }
    g.TY = g.KS * g.RP;
    g.KF = (g.TY + 2 + g.RP - 1) / g.RP;
    g.threads = (g.lanes * g.RP + 31) / 32 * 32;   // whole warps (full-mask shuffles)
    const size_t tabs = ((size_t)9 * n * (sizeof(double) + (fp32 ? sizeof(float) : sizeof(double))) + 31) / 32 * 32;
    // ring: 8 bytes a point (FP64 value, or the float pair of the FP32 mode's RK4 stages),
    // 12 in the FP32 mode's implicit setup (operand, hi, lo)
    const size_t ring = (size_t)FINE_SLOTS * (g.TY + 2) * n * (fp32 ? 12 : 8);
    // FP32 mode, one owned row a thread: the pointwise phase stages FINE_PH3_SLOTS planes of
    // six float inputs per thread over the ring
    const size_t ph3 = (fp32 && g.KS == 1) ? (size_t)FINE_PH3_SLOTS * 6 * g.threads * g.W * sizeof(float) : 0;
    g.smem = tabs + std::max(ring, ph3);
    return g;
}


using FineFn = void (*)(FineArgs);
// The instantiation for W points per thread, ring rows KF / owned rows KS and MODE, or
// nullptr (defined in fine_f32.cu and fine_f64.cu).
FineFn fine_fn_f32(int W, int KF, int KS, int mode);
FineFn fine_fn_f64(int W, int KF, int KS, int mode);
FineFn fine_fn_pert(bool fp32, int W, int KF, int KS);   // FINE_MODE_IMPLICIT_PERT (fine_pert.cu)

}  // namespace pr
