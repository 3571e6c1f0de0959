// Internal declarations shared by the CUDA translation units of the parareal library.
// Device utilities (bounded barriers, deterministic block reductions), kernel parameter
// structs and the host-side launchers the context code calls.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/parareal.h"

namespace pr {

// ---------------------------------------------------------------------------------
// Error codes recorded by kernels into a device int (first error wins).
enum DevErr : int {
    DERR_OK = 0,
    DERR_NOT_CONVERGED = PR_ERR_NOT_CONVERGED,
    DERR_BREAKDOWN = PR_ERR_BREAKDOWN,
    DERR_TIMEOUT = PR_ERR_TIMEOUT,
    DERR_NONFINITE = PR_ERR_NONFINITE,
};

extern long long g_launch_count;   // kernels launched by this library (host counter)

// ---------------------------------------------------------------------------------
// The FD operator of eq. (eq1): (L u)_i = sum_d b_d(i)(u_{i+e_d}-u_{i-e_d})/(2h)
//                                        - eps sum_d (u_{i+e_d}-2u_i+u_{i-e_d})/h^2.
// Velocity: b_x = tab[0][y] + tab[1][z], b_y = tab[2][x] + tab[3][z],
//           b_z = tab[4][x] + tab[5][y]   (six 1-D tables of n doubles, device).
struct Grid {
    int n;
    long long Ng;      // n^3
    double h;
    double eps;
    const double* tab; // 6*n
    const double* pert; // stored velocity perturbation [3][Ng] (b'_x, b'_y, b'_z), or nullptr
};

enum TabIdx { TXY = 0, TXZ = 1, TYX = 2, TYZ = 3, TZX = 4, TZY = 5 };

// Time-dependent flows (Sec. 4) are separable: b(x, t) = c0(t) b^0(x) + c1(t) b^1(x) and
// f(x, t) = f_given(x) + c0(t) g^0(x) + c1(t) g^1(x), each b^q with the six 1-D tables
// above and each g^q = GX[x] + GY[y] + GZ[z].  A context's table buffer holds
// [b^0 (6n) | b^1 (6n) | g^0, g^1 (2 x 3n) | zeros (6n)]; steady flows have b^0 = b,
// b^1 = 0, g = 0, c = (1, 0).
constexpr int TAB_B1 = 6, TAB_G = 12, TAB_ZERO = 18, TAB_TOTAL = 24;   // offsets in units of n
__host__ __device__ inline bool flow_time_dependent(int kind) {
    return kind == PR_FLOW_PAPER_KOLMOGOROV || kind == PR_FLOW_PAPER_ABC;
}
// c0(t), c1(t) of the flow (and of its forcing)
__device__ inline void flow_coeffs(int kind, double w, double t, double& c0, double& c1) {
    if (kind == PR_FLOW_PAPER_KOLMOGOROV) {
        c0 = 1.0;
        c1 = cos(t);
    } else if (kind == PR_FLOW_PAPER_ABC) {
        const double ph = sin(w * t);
        c0 = cos(ph);
        c1 = sin(ph);
    } else {
        c0 = 1.0;
        c1 = 0.0;
    }
}
// All TAB_TOTAL * n table entries of a flow (see above).
cudaError_t launch_flow_tables(const pr_flow& flow, int n, double L, double* tab, cudaStream_t st);
// Parareal-II transfers between the grid of n^3 points and the one coarsened by c:
// out_c = R (U - Up) by injection (Up may be nullptr), and out = F + P x_c by trilinear
// interpolation on the periodic grid (F may be nullptr); B items, item strides sF, sC.
cudaError_t launch_restrict_diff(const double* U, const double* Up, int n, int c, double* out_c,
                                 cudaStream_t st);
cudaError_t launch_prolong_add(const double* xc, long long sxc, int n, int c, const double* F, long long sF,
                               double* out, long long sout, int B, cudaStream_t st);
// The forcing pieces g^0, g^1 of a table buffer as grid functions.
cudaError_t launch_g_fields(const double* tab, int n, double* g0, double* g1, cudaStream_t st);

// ---------------------------------------------------------------------------------
// Memory-model helpers (PTX acquire/release at gpu scope).
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u32(unsigned* p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void record_error(int* err, int code) {
    atomicCAS(err, 0, code);
}

// Barrier of `count` co-resident CTAs on bar[0] (arrivals) / bar[1] (generation).
// Thread 0 arrives with release semantics and polls the generation with acquire
// semantics at most `spin_limit` times; on time-out it records DERR_TIMEOUT and the
// whole CTA gets `false` (the caller returns).  Every CTA of the group must call it the
// same number of times.
__device__ __forceinline__ bool group_barrier(unsigned* bar, unsigned count,
                                              long long spin_limit, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen = ld_acquire_u32(bar + 1);
        unsigned arrived = atom_add_acq_rel_u32(bar, 1u);
        if (arrived == count - 1) {
            st_relaxed_u32(bar, 0u);
            st_release_u32(bar + 1, gen + 1u);
        } else {
            long long spins = 0;
            while (ld_acquire_u32(bar + 1) == gen) {
                if (spins >= spin_limit) {
                    ok = 0;
                    record_error(err, DERR_TIMEOUT);
                    break;
                }
                ++spins;
                __nanosleep(64);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Deterministic block sum of NQ doubles per thread; the result is valid in thread 0
// (returned in-place in v[] of thread 0).  Fixed shuffle tree, then warp sums added in
// warp order.  `red` must hold NQ * 32 doubles of shared memory.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) red[q * 32 + warp] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += red[q * 32 + w];
            v[q] = s;
        }
    }
}

// ---------------------------------------------------------------------------------
// Fine sweep (a batch of independent implicit-Euler runs, one per subinterval).
// One problem in a fine launch: B consecutive subintervals that share grid size, Krylov
// type and tile geometry with the other jobs of the launch but have their own flow,
// diffusion, step, forcing, buffers and tolerance.
struct FineJob {
    const double* tab;  // velocity tables [6][n]; time-dependent flows: the whole table
                        // buffer [b^0 | b^1 | g^0, g^1 | 0] (TAB_TOTAL x n)
    int tdep;           // time-dependent flow: tables rebuilt at every step
    int rk4;            // explicit classical RK4 instead of implicit Euler + BiCGStab
    int no_forcing;     // homogeneous propagation: the flow's forcing pieces are left out
    int kind;           // pr_flow_kind (time coefficients)
    double w;
    double t0, DeltaT;  // item lb of the job starts at t0 + lb DeltaT
    double eps;
    double dt;          // fine step
    int S;              // fine steps
    int dM, n_snap;     // snapshot stride / count (n_snap = 0: none)
    const double* f;    // forcing [Ng] or nullptr
    const float* f32;   // the same rounded to float (FP32 mode), nullptr without forcing
    const double* u_in; // [B][Ng]
    double* u_out;      // [B][Ng]
    void* snap;         // [B][n_snap][Ng] doubles, or nullptr
    double tol;
    int maxit;
    int* status;        // [B] per-subinterval error code
    int* its_total;     // [B]
    int* its_max;       // [B]
    int B;
    const void* pert;   // stored velocity perturbation [3][Ng] in the Krylov type (float in
                        // the FP32 mode, double in FP64), unscaled, or nullptr
};
constexpr int FINE_MAX_JOBS = 16;

struct FineArgs {
    Grid g;             // n, Ng, h (the per-job flow and eps are in jobs[])
    int njobs;
    FineJob jobs[FINE_MAX_JOBS];
    int B;              // subintervals in this launch: the sum of jobs[].B
    void* ws;           // [numGroups][NVEC][Ng] of KT
    double* ust;        // [numGroups][2][Ng]
    double* part;       // [numGroups][2][4][n]
    unsigned* bar;      // [numGroups][2]
    int G;              // CTAs per group
    int numGroups;
    int TY, NY;         // a subinterval: NY columns of TY rows, n tile-planes each
    int RP;             // rows per pass of a CTA (threads = n/W lanes x RP, rounded to warps)
    long long spin_limit;
    int* err;           // launch-wide error code
};
constexpr int FINE_NVEC = 8; // delta, r, rhat, p0, p1, v0, v1, t

// Launch the persistent fine sweep.  Chooses numGroups = min(B, grid / G) and G from
// the occupancy unless a.G > 0.  Returns the CUDA error of the launch.
cudaError_t launch_fine(FineArgs a, bool fp32, int ctas_per_sm, int max_groups,
                        cudaStream_t st);
// Largest number of co-resident CTAs of the fine kernel for this grid size.
int fine_max_ctas(int n, bool fp32, int ctas_per_sm);
int fine_tile_rows(int n);
int fine_block_threads(int n);

// out[i] = (float)in[i], i < n
cudaError_t launch_to_float(const double* in, float* out, long long n, cudaStream_t st);

cudaError_t launch_tables(const pr_flow& flow, int n, double L, double* tab,
                          cudaStream_t st);
// out[c] = L u[c] (transpose: L^T) for columns c < count[b] of each batch item b;
// columns given as pointer arrays in_cols[b*ldcols + c], out_cols[...]; TI/TO = float
// or double selected by the flags.
// FP32 mode: L u of FP64 columns in double-float arithmetic (no transpose).
cudaError_t launch_apply_L_df(const Grid& g, const void* const* in_cols, void* const* out_cols, const int* count,
                              int ldcols, int max_count, int B, cudaStream_t st);
cudaError_t launch_apply_L(const Grid& g, const void* const* in_cols,
                           void* const* out_cols, const int* count, int ldcols,
                           int max_count, int B, bool in_f32, bool out_f32, bool transpose,
                           cudaStream_t st);

// ---------------------------------------------------------------------------------
// Batched cross Gram  G[b] = A_b^T B_b  (A_b: KA[b] columns, B_b: KB[b] columns of Ng
// points each, column pointer arrays), accumulated in FP64 (FP32 inputs: FP32 over
// 32-point blocks, FP64 above).  sym: A_b == B_b and only the upper triangle is formed,
// then mirrored.  Output G[b*ldG_b + i*ldG + j], i < KA, j < KB.  Chunk partials are
// summed in a fixed order by the last CTA of each batch item (deterministic).
struct GramArgs {
    const void* const* colsA; // [B][ldcols]
    const void* const* colsB;
    const int* KA;            // [B] (device)
    const int* KB;            // [B]
    int ldcols;
    long long Ng;
    int B;
    int maxKA, maxKB;
    bool sym;
    double* part;             // [B][chunks][maxKA*maxKB]
    unsigned* counter;        // [B], zero on entry, left zero on exit
    double* G;                // [B][ldG_b]
    int ldG;                  // row stride
    long long ldG_b;          // batch stride
    double scaleB;            // unused (1.0)
    bool df;                  // FP64 operands in double-float arithmetic (FP32 mode)
    // [B][ldcols] block index of each column, or null.  With sym and df, output tiles whose
    // rows and columns all lie in one block are not computed but set to the identity: the
    // caller asserts that every block has orthonormal columns (Cholesky-QR'd bases).
    const int* colblk;
};
int gram_chunks(long long Ng);
size_t gram_part_doubles(long long Ng, int B, int maxKA, int maxKB);
cudaError_t launch_gram(const GramArgs& a, bool a_f32, bool b_f32, cudaStream_t st);
// Symmetric Gram W^T W of up to 64 FP64 columns on the tensor cores (tcgen05, error-free
// BF16 digits, FP64-accurate; gram_tc.cu; up to 32 columns the narrow, exactly summed
// form when the partial buffer holds two chunks of the other Gram kernels per unit).  colmax: device scratch of B x ld (ld >= maxKA)
// 64-bit words; err: device error flag (PR_ERR_TIMEOUT if a wait on an mbarrier gives up
// after spin_limit polls; the MMAs in flight are then waited for, with the default bound,
// and the tensor memory freed).
cudaError_t launch_gram_tc(const GramArgs& a, unsigned long long* colmax, int ld, int* err, long long spin_limit,
                           cudaStream_t st);
int gram_tc_max_cols();
// M_b = I_{m[b]} for b < B (row stride ld, batch stride ld_b).
cudaError_t launch_identity(double* M, int ld, long long ld_b, const int* m, int B, cudaStream_t st);

// Tall-skinny multiply: Out_b[:, j] = sum_i In_b[:, i] C_b[i][j], i < KIN[b], j < KOUT[b];
// inputs as column pointers, output contiguous columns out + b*ld_out_b + j*Ng.
struct TsmmArgs {
    const void* const* colsIn; // [B][ldcols]
    const int* KIN;            // [B]
    const int* KOUT;           // [B]
    int ldcols;
    const double* C;           // [B][ldC_b]: C[i*ldC + j]
    int ldC;
    long long ldC_b;
    void* out;
    long long ld_out_b;        // elements between batch items
    long long Ng;
    int B;
    int maxKIN, maxKOUT;
    bool df;                   // FP64 in and out, double-float arithmetic (FP32 mode)
};
cudaError_t launch_tsmm(const TsmmArgs& a, bool in_f32, bool out_f32, cudaStream_t st);

// Batched symmetric eigenproblem (cyclic Jacobi, FP64) + POD selection (Algorithm 1):
// G[b] (K[b] x K[b], row stride ldG, batch stride ldG_b) -> lam[b][0..K) descending,
// m[b] (criterion with gamma, tau, cap), C[b] = Y[:, :m] diag(lam^-1/2) stored
// C[b*ldC_b + i*ldC + j].
struct EigArgs {
    const double* G; int ldG; long long ldG_b;
    const int* K;
    int maxK;
    int B;
    double gamma, tau;
    int cap;
    double* lam;               // [B][maxK]
    int* m;                    // [B]
    double* C; int ldC; long long ldC_b;
    int* err;
};
cudaError_t launch_eig_pod(const EigArgs& a, cudaStream_t st);

// Batched Cholesky of Gram matrices and X = L^{-T}: G[b] (m[b] x m[b]) -> X[b].
cudaError_t launch_chol_inv(const double* G, int ldG, long long ldG_b, const int* m, int maxm,
                            int B, double* X, int ldX, long long ldX_b, int* err,
                            cudaStream_t st);

// Fill column pointer arrays: for batch b, cols[b*ld + ...] = concatenation of nb blocks
// (block j: base pointer bases[b*nb + j], count cnt[b*nb + j] read on the device,
// column stride Ng elements of esize bytes); K[b] = total; blk[b*ld + k] (if not null) =
// the block of column k.
cudaError_t launch_assemble_cols(const void* const* bases, const int* const* cnt_ptrs,
                                 int nb, int B, long long Ng, int esize, const void** cols,
                                 int ld, int* K, int* blk, cudaStream_t st);

// ---------------------------------------------------------------------------------
// Coarse sweep pieces (one subinterval, sequential in n).
// Persistent coarse sweep over subintervals n = n0 .. n0+count-1, in order: item n reads
// U^k_n = U + n*sU (for n > n0 the output of item n-1 when sU == sOut and
// out == U + sU), U^{k-1}_n, F_n, its level-2 basis (m[n*sm] FP64 columns of stride Ng)
// and Galerkin blocks, and writes U^k_{n+1} = out + n*sOut.
struct CoarseSweepArgs {
    Grid g;
    long long n0;
    int count;
    const double* U;  long long sU;
    const double* Up; long long sUp;
    const double* F;  long long sF;
    double* out;      long long sOut;
    const double* R;  long long sR;
    const int* m;     long long sm;
    const double* Mr;       // R^T R, m x m with leading dimension ldM, stride sM per item
    const double* Lr;       // R^T L R (steady flows) or the pieces R^T D R, R^T A0 R,
                            // R^T A1 R (time-dependent), ldM x ldM each, ldM^2 apart,
                            // stride sML per item
    long long sM, sML;
    int ldM;
    // time-dependent flows: L(t) = D + c0(t) A0 + c1(t) A1 with D = -eps Lap_h and the
    // advection pieces A_q = b^q . grad_h (antisymmetric); coarse step l of item n ends at
    // t0 + n DeltaT + l dT
    int tdep, kind;
    double w, t0, DeltaT;
    double* A1d;            // scratch [Ng] (A1 d~)
    int maxm;               // <= coarse_max_m()
    double dT;
    int Lc;
    double aug_tol;
    int augment;            // 0: plain coarse space R (no d~ stages, no augmentation)
    double* d;              // scratch [Ng] each
    double* Ld;
    double* Ltd;
    double* part;           // coarse_part_doubles()
    unsigned* bar;          // [2], bar[0] zero at launch
    long long spin_limit;
    int* err;
};
cudaError_t launch_coarse_sweep(CoarseSweepArgs a, cudaStream_t st);
int coarse_max_m();
size_t coarse_part_doubles(long long Ng, int maxm);

// Iteration 0: beta_n = reduced coordinates of U^0_n, n = 1..N (G_0 in V0), from
// M0 = V0^T V0, L0 = V0^T L V0, p0 = V0^T u_hat0, q0 = V0^T f.
// Time-dependent flows in iteration 0: L0 holds the pieces V0^T D V0, V0^T A0 V0,
// V0^T A1 V0 (ld^2 apart) and qg the projections V0^T g^0, V0^T g^1 (ld apart).
struct G0Tdep {
    int tdep, kind;
    double w, T0;
    const double* qg;
};
cudaError_t launch_g0(const double* M0, const double* L0, const double* p0, const double* q0,
                      const int* m0, int ld, int N, int Lc, double dT, double* beta, int ldb,
                      int* err, const G0Tdep& td, cudaStream_t st);

// Convergence: for n < cnt: out[n*4 + 0..3] = ||a_n-b_n||^2, ||a_n||^2, ||a_n-r_n||^2,
// ||r_n||^2 (r may be null: last two zero).
cudaError_t launch_norms(const double* a, const double* b, const double* r, long long Ng,
                         int cnt, double* part, unsigned* counter, double* out,
                         cudaStream_t st);
size_t norms_part_doubles(long long Ng, int cnt);

// Operator on caller buffers with its scratch in a static device array (noalloc.cu).
cudaError_t apply_L_noalloc(int n, double L, const pr_flow& flow, const double* d_pert, double eps,
                            const double* d_in,
                            double* d_out, int count, bool transpose, cudaStream_t st);
int noalloc_max_n();
int noalloc_max_count();
size_t noalloc_scratch_bytes();

// Scan for NaN/Inf: sets *flag = 1 if any of the first `count` doubles is not finite.
cudaError_t launch_nonfinite(const double* x, long long count, int* flag, cudaStream_t st);

} // namespace pr
