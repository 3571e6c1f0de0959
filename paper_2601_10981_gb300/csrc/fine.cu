// Host side of the fine propagator and the whole-grid operator kernels: velocity and
// forcing tables, L u for the Galerkin blocks, the launch of the persistent fine sweep
// (the kernel itself is in fine_kernel.cuh, instantiated by fine_f32.cu / fine_f64.cu).
#include "fine_kernel.cuh"


#include <algorithm>
#include <math.h>
#include <type_traits>

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

// Table buffer of a context: b^0, b^1, g^0, g^1 and a zero block (layout in pr_internal.cuh).
// Eq. (koleq): b^0 = (cos y, cos z, cos x), b^1 = (sin z, sin x, sin y), c = (1, cos t);
// g^0 = -cos y, g^1 = -sin z.  Sec. 4.2 (A = B = C = 1, phase p = sin wt):
// sin(a + p) = cos p sin a + sin p cos a and cos(a + p) = cos p cos a - sin p sin a give
// b^0 = the steady ABC field, b^1 = (cos z - sin y, cos x - sin z, cos y - sin x),
// c = (cos p, sin p); g^0 = -sin z - cos y, g^1 = -cos z + sin y.
__global__ void flow_tables_kernel(int kind, double A, double B, double C, int k, double b0,
                                   double b1, double b2, int n, double L, double* tab) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = i * (L / n);
    double v0[6] = {0, 0, 0, 0, 0, 0}, v1[6] = {0, 0, 0, 0, 0, 0};
    double g0[3] = {0, 0, 0}, g1[3] = {0, 0, 0};   // GX, GY, GZ
    const double sx = sin(x), cx = cos(x);
    if (kind == PR_FLOW_ABC) {
        v0[TXY] = C * cx;
        v0[TXZ] = A * sx;
        v0[TYX] = B * sx;
        v0[TYZ] = A * cx;
        v0[TZX] = B * cx;
        v0[TZY] = C * sx;
    } else if (kind == PR_FLOW_KOLMOGOROV) {
        v0[TXY] = sin((double)k * x);
    } else if (kind == PR_FLOW_CONST) {
        v0[TXY] = b0;
        v0[TYX] = b1;
        v0[TZX] = b2;
    } else if (kind == PR_FLOW_PAPER_KOLMOGOROV) {
        v0[TXY] = cx;   // b_x: cos y + sin z cos t
        v1[TXZ] = sx;
        v0[TYZ] = cx;   // b_y: cos z + sin x cos t
        v1[TYX] = sx;
        v0[TZX] = cx;   // b_z: cos x + sin y cos t
        v1[TZY] = sx;
        g0[1] = -cx;    // f: -cos y - sin z cos t
        g1[2] = -sx;
    } else if (kind == PR_FLOW_PAPER_ABC) {
        v0[TXZ] = sx;  v0[TXY] = cx;  v1[TXZ] = cx;  v1[TXY] = -sx;   // b_x
        v0[TYX] = sx;  v0[TYZ] = cx;  v1[TYX] = cx;  v1[TYZ] = -sx;   // b_y
        v0[TZY] = sx;  v0[TZX] = cx;  v1[TZY] = cx;  v1[TZX] = -sx;   // b_z
        g0[2] = -sx;  g0[1] = -cx;  g1[2] = -cx;  g1[1] = sx;         // f
    }
    for (int t = 0; t < 6; ++t) {
        tab[t * n + i] = v0[t];
        tab[(TAB_B1 + t) * n + i] = v1[t];
        tab[(TAB_ZERO + t) * n + i] = 0.0;
    }
    for (int t = 0; t < 3; ++t) {
        tab[(TAB_G + t) * n + i] = g0[t];
        tab[(TAB_G + 3 + t) * n + i] = g1[t];
    }
}

cudaError_t launch_flow_tables(const pr_flow& flow, int n, double L, double* tab, cudaStream_t st) {
    flow_tables_kernel<<<(n + 127) / 128, 128, 0, st>>>(flow.kind, flow.A, flow.B, flow.C, flow.k,
                                                        flow.b[0], flow.b[1], flow.b[2], n, L, tab);
    ++g_launch_count;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Grid transfers of the Parareal-II comparator (restriction by injection, trilinear
// prolongation on the periodic grid).
__global__ void restrict_diff_kernel(const double* U, const double* Up, int n, int c, double* out_c) {
    const int nc = n / c;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nc3 = (long long)nc * nc * nc;
    if (i >= nc3) return;
    const int x = (int)(i % nc), y = (int)((i / nc) % nc), z = (int)(i / ((long long)nc * nc));
    const long long f = ((long long)z * c * n + (long long)y * c) * n + (long long)x * c;
    out_c[i] = Up ? U[f] - Up[f] : U[f];
}

__global__ void prolong_add_kernel(const double* xc, long long sxc, int n, int c, const double* F, long long sF,
                                   double* out, long long sout) {
    const int nc = n / c;
    const int b = blockIdx.y;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n3 = (long long)n * n * n;
    if (i >= n3) return;
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((long long)n * n));
    const double* X = xc + (size_t)b * sxc;
    // the coarse cell and the offsets inside it along each axis
    const int x0 = x / c, y0 = y / c, z0 = z / c;
    const int x1 = (x0 + 1) % nc, y1 = (y0 + 1) % nc, z1 = (z0 + 1) % nc;
    const double wx = (double)(x - x0 * c) / c, wy = (double)(y - y0 * c) / c, wz = (double)(z - z0 * c) / c;
    auto at = [&](int zz, int yy, int xx) { return X[((long long)zz * nc + yy) * nc + xx]; };
    // tensor-product (trilinear) interpolation: along x, then y, then z
    const double a00 = (1.0 - wx) * at(z0, y0, x0) + wx * at(z0, y0, x1);
    const double a01 = (1.0 - wx) * at(z0, y1, x0) + wx * at(z0, y1, x1);
    const double a10 = (1.0 - wx) * at(z1, y0, x0) + wx * at(z1, y0, x1);
    const double a11 = (1.0 - wx) * at(z1, y1, x0) + wx * at(z1, y1, x1);
    const double b0 = (1.0 - wy) * a00 + wy * a01;
    const double b1 = (1.0 - wy) * a10 + wy * a11;
    const double v = (1.0 - wz) * b0 + wz * b1;
    out[(size_t)b * sout + i] = (F ? F[(size_t)b * sF + i] : 0.0) + v;
}

cudaError_t launch_restrict_diff(const double* U, const double* Up, int n, int c, double* out_c,
                                 cudaStream_t st) {
    const long long nc3 = (long long)(n / c) * (n / c) * (n / c);
    restrict_diff_kernel<<<(unsigned)((nc3 + 255) / 256), 256, 0, st>>>(U, Up, n, c, out_c);
    ++g_launch_count;
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(const double* xc, long long sxc, int n, int c, const double* F, long long sF,
                               double* out, long long sout, int B, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    const long long n3 = (long long)n * n * n;
    prolong_add_kernel<<<dim3((unsigned)((n3 + 255) / 256), (unsigned)B), 256, 0, st>>>(xc, sxc, n, c, F, sF, out,
                                                                                       sout);
    ++g_launch_count;
    return cudaGetLastError();
}

// g^q(x, y, z) = GX_q[x] + GY_q[y] + GZ_q[z] as grid functions (the forcing pieces of a
// time-dependent flow, for their projections onto V0).
__global__ void g_fields_kernel(const double* tab, int n, double* g0, double* g1) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n3 = (long long)n * n * n;
    if (i >= n3) return;
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((long long)n * n));
    const double* G = tab + (size_t)TAB_G * n;
    g0[i] = G[x] + G[n + y] + G[2 * n + z];
    g1[i] = G[3 * n + x] + G[4 * n + y] + G[5 * n + z];
}

cudaError_t launch_g_fields(const double* tab, int n, double* g0, double* g1, cudaStream_t st) {
    const long long n3 = (long long)n * n * n;
    g_fields_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, st>>>(tab, n, g0, g1);
    ++g_launch_count;
    return cudaGetLastError();
}

cudaError_t launch_tables(const pr_flow& flow, int n, double L, double* tab, cudaStream_t st) {
    tables_kernel<<<(n + 127) / 128, 128, 0, st>>>(flow.kind, flow.A, flow.B, flow.C, flow.k,
                                                   flow.b[0], flow.b[1], flow.b[2], n, L, tab);
    ++g_launch_count;
    return cudaGetLastError();
}

__global__ void to_float_kernel(const double* in, float* out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

cudaError_t launch_to_float(const double* in, float* out, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    to_float_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
    ++g_launch_count;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// out = L u or L^T u on whole grid functions.  Every supported velocity has b_d
// independent of x_d, so b_d(x +- e_d) = b_d(x) and L^T only flips the advection sign.
// One thread per point runs over all columns of its batch item: the neighbour offsets and
// the velocity terms are formed once (32-bit index arithmetic, no FP64 division), each
// column costs its seven loads and a dozen FP64 operations.
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) apply_L_kernel(Grid g, const void* const* in_cols, void* const* out_cols,
                                                      const int* count, int ldcols, bool transpose,
                                                      double inv2h, double epsh2) {
    const int b = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int)g.Ng) return;
    const int n = g.n, n2 = n * n;
    const int z = i / n2;
    const int rem = i - z * n2;
    const int y = rem / n;
    const int x = rem - y * n;
    const int ixp = i + (x + 1 == n ? 1 - n : 1), ixm = i + (x == 0 ? n - 1 : -1);
    const int iyp = i + (y + 1 == n ? n - n2 : n), iym = i + (y == 0 ? n2 - n : -n);
    const int izp = i + (z + 1 == n ? n2 - (int)g.Ng : n2), izm = i + (z == 0 ? (int)g.Ng - n2 : -n2);
    const double* tab = g.tab;
    const double bx = tab[TXY * n + y] + tab[TXZ * n + z];
    const double by = tab[TYX * n + x] + tab[TYZ * n + z];
    const double bz = tab[TZX * n + x] + tab[TZY * n + y];
    // Row i of the advection part holds +-b_d(x_i)/(2h) at i +- e_d.  L^T: column i holds
    // +b_d(x_{i-e_d})/(2h) at i - e_d and -b_d(x_{i+e_d})/(2h) at i + e_d; the analytic
    // b_d does not vary along x_d, a stored perturbation does.
    double cxp, cxm, cyp, cym, czp, czm;   // advection coefficients of u at the neighbours
    if (!g.pert) {
        const double sg = transpose ? -inv2h : inv2h;
        cxp = sg * bx, cyp = sg * by, czp = sg * bz;
        cxm = -cxp, cym = -cyp, czm = -czp;
    } else if (!transpose) {
        const long long N = g.Ng;
        cxp = inv2h * (bx + g.pert[i]);
        cyp = inv2h * (by + g.pert[N + i]);
        czp = inv2h * (bz + g.pert[2 * N + i]);
        cxm = -cxp, cym = -cyp, czm = -czp;
    } else {
        const long long N = g.Ng;
        cxp = -inv2h * (bx + g.pert[ixp]), cxm = inv2h * (bx + g.pert[ixm]);
        cyp = -inv2h * (by + g.pert[N + iyp]), cym = inv2h * (by + g.pert[N + iym]);
        czp = -inv2h * (bz + g.pert[2 * N + izp]), czm = inv2h * (bz + g.pert[2 * N + izm]);
    }
    const int cnt = count[b];
    for (int c = 0; c < cnt; ++c) {
        const TI* in = (const TI*)in_cols[(size_t)b * ldcols + c];
        TO* out = (TO*)out_cols[(size_t)b * ldcols + c];
        const double u0 = (double)in[i];
        const double uxp = (double)in[ixp], uxm = (double)in[ixm];
        const double uyp = (double)in[iyp], uym = (double)in[iym];
        const double uzp = (double)in[izp], uzm = (double)in[izm];
        double adv;
        if (!(transpose && g.pert))   // cd_m = -cd_p: differences first, exact for close values
            adv = cxp * (uxp - uxm) + cyp * (uyp - uym) + czp * (uzp - uzm);
        else
            adv = (cxp * uxp + cxm * uxm) + (cyp * uyp + cym * uym) + (czp * uzp + czm * uzm);
        const double lap = (uxp + uxm) + (uyp + uym) + (uzp + uzm) - 6.0 * u0;
        out[i] = (TO)(adv - epsh2 * lap);
    }
}

// FP32 mode: L u of FP64 columns in double-float arithmetic on the FP32 pipe (GB300 runs
// FP64 at 1/64 of the FP32 rate).  L u at a point is the weighted sum of the seven stencil
// values; the weights (formed in FP64 once per point) and the values are split into float
// pairs by moving bits, and the sum is taken with error-free products and TwoSums
// (df_mac), ~1e-15 relative to the sum of the terms' magnitudes.
__global__ void __launch_bounds__(256) apply_L_df_kernel(Grid g, const void* const* in_cols, void* const* out_cols,
                                                         const int* count, int ldcols, double inv2h, double epsh2) {
    const int b = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int)g.Ng) return;
    const int n = g.n, n2 = n * n;
    const int z = i / n2;
    const int rem = i - z * n2;
    const int y = rem / n;
    const int x = rem - y * n;
    int nb[7];
    nb[0] = i;
    nb[1] = i + (x + 1 == n ? 1 - n : 1);
    nb[2] = i + (x == 0 ? n - 1 : -1);
    nb[3] = i + (y + 1 == n ? n - n2 : n);
    nb[4] = i + (y == 0 ? n2 - n : -n);
    nb[5] = i + (z + 1 == n ? n2 - (int)g.Ng : n2);
    nb[6] = i + (z == 0 ? (int)g.Ng - n2 : -n2);
    const double* tab = g.tab;
    double bx = tab[TXY * n + y] + tab[TXZ * n + z];
    double by = tab[TYX * n + x] + tab[TYZ * n + z];
    double bz = tab[TZX * n + x] + tab[TZY * n + y];
    if (g.pert) {
        bx += g.pert[i];
        by += g.pert[g.Ng + i];
        bz += g.pert[2 * g.Ng + i];
    }
    const double ax = inv2h * bx, ay = inv2h * by, az = inv2h * bz;
    const double wd[7] = {6.0 * epsh2, ax - epsh2, -ax - epsh2, ay - epsh2, -ay - epsh2, az - epsh2, -az - epsh2};
    float2 w[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) w[k] = d2df_bits(wd[k]);
    const int cnt = count[b];
    for (int c = 0; c < cnt; ++c) {
        const double* in = (const double*)in_cols[(size_t)b * ldcols + c];
        double* out = (double*)out_cols[(size_t)b * ldcols + c];
        double u[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) u[k] = in[nb[k]];
        float sh = 0.0f, sl = 0.0f;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const float2 v = d2df_bits(u[k]);
            df_mac(sh, sl, w[k].x, w[k].y, v.x, v.y);
        }
        out[i] = df_to_double(sh, sl);
    }
}

cudaError_t launch_apply_L_df(const Grid& g, const void* const* in_cols, void* const* out_cols, const int* count,
                              int ldcols, int max_count, int B, cudaStream_t st) {
    if (max_count <= 0 || B <= 0) return cudaSuccess;
    if (g.Ng > (1LL << 30)) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((g.Ng + 255) / 256), (unsigned)B);
    apply_L_df_kernel<<<grid, 256, 0, st>>>(g, in_cols, out_cols, count, ldcols, 0.5 / g.h, g.eps / (g.h * g.h));
    ++g_launch_count;
    return cudaGetLastError();
}

cudaError_t launch_apply_L(const Grid& g, const void* const* in_cols, void* const* out_cols,
                           const int* count, int ldcols, int max_count, int B, bool in_f32,
                           bool out_f32, bool transpose, cudaStream_t st) {
    if (max_count <= 0 || B <= 0) return cudaSuccess;
    if (g.Ng > (1LL << 30)) return cudaErrorInvalidValue;   // 32-bit point indices
    dim3 grid((unsigned)((g.Ng + 255) / 256), (unsigned)B);
    const double inv2h = 0.5 / g.h, epsh2 = g.eps / (g.h * g.h);
    if (in_f32 && out_f32)
        apply_L_kernel<float, float><<<grid, 256, 0, st>>>(g, in_cols, out_cols, count, ldcols, transpose, inv2h, epsh2);
    else if (in_f32)
        apply_L_kernel<float, double><<<grid, 256, 0, st>>>(g, in_cols, out_cols, count, ldcols, transpose, inv2h, epsh2);
    else if (out_f32)
        apply_L_kernel<double, float><<<grid, 256, 0, st>>>(g, in_cols, out_cols, count, ldcols, transpose, inv2h, epsh2);
    else
        apply_L_kernel<double, double><<<grid, 256, 0, st>>>(g, in_cols, out_cols, count, ldcols, transpose, inv2h,
                                                             epsh2);
    ++g_launch_count;
    return cudaGetLastError();
}

int fine_block_threads(int n) { return fine_geom(n, true).threads; }
int fine_tile_rows(int n) { return fine_geom(n, true).TY; }

static FineFn fine_select(int n, bool fp32, int mode = FINE_MODE_IMPLICIT) {
    const FineGeom g = fine_geom(n, fp32);
    return fp32 ? fine_fn_f32(g.W, g.KF, g.KS, mode) : fine_fn_f64(g.W, g.KF, g.KS, mode);
}

int fine_max_ctas(int n, bool fp32, int ctas_per_sm) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const FineGeom geo = fine_geom(n, fp32);
    FineFn fn = fine_select(n, fp32);
    if (!fn) return 1;
    if (geo.smem > 48 * 1024)
        cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, geo.threads, geo.smem);
    if (ctas_per_sm > 0) occ = std::min(occ, ctas_per_sm);
    return std::max(1, occ) * std::max(1, sms);
}

cudaError_t launch_fine(FineArgs a, bool fp32, int ctas_per_sm, int max_groups, cudaStream_t st) {
    if (a.B <= 0) return cudaSuccess;
    const int n = a.g.n;
    if (n > 256 || n < 4) return cudaErrorInvalidValue;
    const bool rk = a.jobs[0].rk4 != 0;
    const bool pt = a.jobs[0].pert != nullptr;
    bool td = false;
    for (int j = 0; j < a.njobs; ++j) {
        if ((a.jobs[j].rk4 != 0) != rk) return cudaErrorInvalidValue;   // one integrator per launch
        if ((a.jobs[j].pert != nullptr) != pt) return cudaErrorInvalidValue;   // one stencil kind
        td = td || a.jobs[j].tdep != 0;
    }
    // the perturbation is a steady field of the implicit propagator
    if (pt && (rk || td)) return cudaErrorInvalidValue;
    const int mode = rk ? FINE_MODE_RK4
                        : (td ? FINE_MODE_IMPLICIT_TD : (pt ? FINE_MODE_IMPLICIT_PERT : FINE_MODE_IMPLICIT));
    FineFn fn = fine_select(n, fp32, mode);
    if (!fn) return cudaErrorInvalidValue;
    if (mode != FINE_MODE_IMPLICIT) {   // fine_max_ctas configured the steady instantiation
        const FineGeom g2 = fine_geom(n, fp32);
        if (g2.smem > 48 * 1024)
            cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g2.smem);
    }
    const FineGeom geo = fine_geom(n, fp32);
    const int max_ctas = fine_max_ctas(n, fp32, ctas_per_sm);
    a.TY = geo.TY;
    a.RP = geo.RP;
    a.NY = n / a.TY;
    // CTAs per subinterval: as many as fit beside the other active subintervals (the
    // tile-planes split evenly over any count), at most one tile-plane each
    int G = a.G;
    if (G <= 0) G = std::max(1, max_ctas / a.B);
    G = std::min(std::min(G, max_ctas), a.NY * n);
    int groups = std::min(a.B, std::max(1, max_ctas / G));
    groups = std::min(groups, max_groups);
    a.G = G;
    a.numGroups = groups;
    const int grid = G * groups;
    void* args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(geo.threads), args, geo.smem, st);
    ++g_launch_count;
    return e;
}

} // namespace pr
