// Context and C ABI of the adaptive-parareal library (include/parareal.h).
//
// The host side only orchestrates: every step of Algorithm 2 runs in the kernels of
// fine.cu, pod.cu and coarse.cu, enqueued on one stream without host round trips inside
// a phase.  The host reads device results only in pr_check / pr_sync / pr_get_*.
#include "pr_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace pr {
long long g_launch_count = 0;
}

using namespace pr;

namespace {

int steps_for(double span, double dt) {
    const double q = span / dt;
    const double r = std::nearbyint(q);
    if (std::fabs(q - r) < 1e-9 * std::max(1.0, q)) return (int)r;
    return (int)std::ceil(q);
}

struct Bump {
    size_t off = 0;
    char* base = nullptr;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) / 256 * 256;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

}  // namespace

struct pr_ctx {
    // problem
    int n = 0;
    double L = 0, h = 0;
    long long Ng = 0;
    pr_flow flow{};
    double eps = 0, T = 0;
    int N = 0;
    double pod_tol = 0;
    pr_opts o{};
    // derived
    double DeltaT = 0, dt = 0, T0 = 0, dT = 0;
    int S = 0, S0 = 0, Lc = 0, dM = 0, ns = 0, ns0 = 0, nsmax = 0;
    double gamma1 = 0, gamma3 = 0, tau = 0, tau1 = 1e-13, lin_tol = 0;
    bool fp32 = false;
    int esz = 8;         // POD bases are FP64 in both modes (the augmentation needs them exact)
    int wave = 0;        // > 0: the iteration streams in waves of this many subintervals
    int wave_lo = 0, wave_hi = 0;   // subintervals whose snapshots the store holds
    int r2_lo = 0, r2_hi = 0;       // wave mode: subintervals whose level-2 bases are held
    int mcap0 = 0, mcap1 = 0, w2 = 0, mcap2 = 0, mscr = 0, maxK = 0, ldcols = 0;
    int groups_max = 1;
    int max_ctas = 1;
    bool has_f = false;
    bool tdep = false;   // time-dependent flow of Sec. 4 (tables and Galerkin pieces per time)
    std::vector<double> pert_host;   // stored velocity perturbation [3][Ng] (empty: none)
    // device
    cudaStream_t st = nullptr;
    bool own_ws = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_ready = false;
    double* tab = nullptr;
    double* u0 = nullptr;
    double* f = nullptr;
    float* f32 = nullptr;   // forcing rounded to float (FP32-mode fine sweep)
    double* Ubuf[2] = {nullptr, nullptr};
    int cur = 0;  // Ubuf[cur] holds the latest iterate
    double* Fend = nullptr;
    char* snap = nullptr;
    char* R1[2] = {nullptr, nullptr};
    int* m1[2] = {nullptr, nullptr};
    char* R1t = nullptr;           // wave mode: level-1 bases of the current wave
    int* m1t = nullptr;
    int r1cur = 0;  // R1[r1cur]: level-1 bases of the latest pod update
    char* V0 = nullptr;
    int* m0 = nullptr;
    char* R2 = nullptr;
    int* m2 = nullptr;
    int* mop = nullptr;            // POD dimensions of pr_op_pod
    char* LR = nullptr;
    char* scr[1] = {nullptr};
    double* Mr = nullptr;
    double* Lr = nullptr;
    double* M0 = nullptr;
    double* L0 = nullptr;
    double* p0 = nullptr;
    double* q0 = nullptr;
    double* pert = nullptr;       // stored velocity perturbation [3][Ng], FP64
    float* pert32 = nullptr;      // the same in float (FP32-mode Krylov operator)
    double* pertc = nullptr;      // injected onto the Parareal-II coarse grid [3][Ngc]
    float* pertc32 = nullptr;
    double* qg = nullptr;         // V0^T g^0, V0^T g^1 (time-dependent flows)
    double* gq = nullptr;         // g^0, g^1 as grid functions (time-dependent flows)
    double* cA1 = nullptr;        // coarse-sweep scratch A1 d~
    // Parareal-II: the grid coarsened by 2, its tables, forcing, fine-kernel workspace,
    // the restricted input, the coarse output and iteration 0's coarse trajectory
    int nc = 0;
    long long Ngc = 0;
    double* tabc = nullptr;
    double* fc = nullptr;
    float* fc32 = nullptr;
    void* fwsc = nullptr;
    double* ustc = nullptr;
    double* fpartc = nullptr;
    unsigned* fbarc = nullptr;
    int max_ctas_c = 1;
    double* xc = nullptr;
    double* yc = nullptr;
    double* trajc = nullptr;
    double* beta = nullptr;
    double* gout = nullptr;
    double* lam = nullptr;
    double* Cm = nullptr;
    double* X = nullptr;
    double* gpart = nullptr;
    size_t gpart_n = 0;
    unsigned long long* colmax = nullptr;   // [N + 1][64] column maxima of the tensor-core Gram
    unsigned* counters = nullptr;  // [N + 64]
    const void** colsA = nullptr;
    const void** colsB = nullptr;
    int* colblk = nullptr;         // [N + 1][ldcols] block of each colsA column (level 2)
    const void** bases = nullptr;  // [N][4]
    const int** cntp = nullptr;    // [N][4]
    int* KA = nullptr;
    int* KB = nullptr;
    int* ones = nullptr;           // [N+1] = 1
    int* cnst = nullptr;           // [0] = ns, [1] = ns0, [2] = op m, [3] = 1
    void* fws = nullptr;
    size_t fws_bytes = 0;
    double* ust = nullptr;
    double* fpart = nullptr;
    unsigned* fbar = nullptr;
    int* fstatus = nullptr;
    int* fits = nullptr;
    int* fitsmax = nullptr;
    int* derr = nullptr;
    int* nonfin = nullptr;
    double* cd = nullptr;
    double* cLd = nullptr;
    double* cLtd = nullptr;
    double* cpart = nullptr;
    double* npart = nullptr;
    double* nout = nullptr;
    double* ref = nullptr;        // owned cudaMalloc
    // state
    int k_done = -1;   // -1: nothing, 0: iteration 0, k: iteration k complete
    int phase = 0;     // for k_done+1: 0 none, 1 fine done, 2 pod done
    bool initial_set = false;
    bool checked = true;
    std::vector<double> last_inc, last_err;
    std::string err;
    cudaEvent_t ev[8] = {};
    bool ev_ready = false;
    std::vector<cudaEvent_t> fev;   // pairs around the fine launches of the last fine sweep
    int fev_used = 0;
};

namespace {

pr_status fail(pr_ctx* c, pr_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

pr_status cuda_fail(pr_ctx* c, cudaError_t e, const char* where) {
    return fail(c, PR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PR_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);     \
    } while (0)

// Assign (base != null) or size (base == null) the workspace.
size_t plan(pr_ctx* c, char* base) {
    Bump b;
    b.base = base;
    const long long Ng = c->Ng;
    const int N = c->N;
    c->tab = b.take<double>((size_t)TAB_TOTAL * c->n);
    c->u0 = b.take<double>(Ng);
    c->f = b.take<double>(Ng);
    c->f32 = b.take<float>(Ng);
    c->Ubuf[0] = b.take<double>((size_t)(N + 1) * Ng);
    c->Ubuf[1] = b.take<double>((size_t)(N + 1) * Ng);
    c->Fend = b.take<double>((size_t)N * Ng);
    // wave mode: the snapshot store, the level-2 bases, POD scratch and fine workspace
    // hold one wave; the level-1 bases keep one generation (updated in place after each
    // wave's level 2) plus the current wave's
    const int NB = c->wave > 0 ? std::min(c->wave, N) : N;
    c->snap = b.take<char>((size_t)std::max(NB, 1) * c->nsmax * Ng * sizeof(double));
    for (int i = 0; i < (c->wave > 0 ? 1 : 2); ++i) {
        c->R1[i] = b.take<char>((size_t)N * c->mcap1 * Ng * c->esz);
        c->m1[i] = b.take<int>(N);
    }
    if (c->wave > 0) {
        c->R1t = b.take<char>((size_t)NB * c->mcap1 * Ng * c->esz);
        c->m1t = b.take<int>(NB);
    }
    c->V0 = b.take<char>((size_t)c->mcap0 * Ng * c->esz);
    c->m0 = b.take<int>(1);
    c->R2 = b.take<char>((size_t)NB * c->mcap2 * Ng * c->esz);
    c->m2 = b.take<int>(N + 1);
    c->mop = b.take<int>(N + 1);
    c->LR = b.take<char>((size_t)NB * c->mscr * Ng * c->esz);
    c->scr[0] = b.take<char>((size_t)NB * c->mscr * Ng * c->esz);
    c->Mr = b.take<double>((size_t)(N + 1) * c->mcap2 * c->mcap2);
    // Galerkin blocks of L: R^T L R (steady flows) or the pieces R^T D R, R^T A0 R, R^T A1 R
    c->Lr = b.take<double>((size_t)(N + 1) * 3 * c->mcap2 * c->mcap2);
    c->M0 = b.take<double>((size_t)c->mcap0 * c->mcap0);
    c->L0 = b.take<double>((size_t)3 * c->mcap0 * c->mcap0);
    c->p0 = b.take<double>(c->mcap0);
    c->q0 = b.take<double>(c->mcap0);
    c->qg = b.take<double>((size_t)2 * c->mcap0);
    c->gq = c->tdep ? b.take<double>((size_t)2 * Ng) : nullptr;
    const bool pt = !c->pert_host.empty();
    c->pert = pt ? b.take<double>((size_t)3 * Ng) : nullptr;
    c->pert32 = pt && c->fp32 ? b.take<float>((size_t)3 * Ng) : nullptr;
    const bool pt2 = pt && c->o.method == PR_METHOD_PARAREAL_II;
    c->pertc = pt2 ? b.take<double>((size_t)3 * c->Ngc) : nullptr;
    c->pertc32 = pt2 && c->fp32 ? b.take<float>((size_t)3 * c->Ngc) : nullptr;
    c->cA1 = b.take<double>(Ng);
    if (c->o.method == PR_METHOD_PARAREAL_II) {
        const long long Ngc = c->Ngc;
        const size_t kesz2 = c->fp32 ? sizeof(float) : sizeof(double);
        c->tabc = b.take<double>((size_t)TAB_TOTAL * c->nc);
        c->fc = b.take<double>(Ngc);
        c->fc32 = b.take<float>(Ngc);
        c->fwsc = b.take<char>(std::max((size_t)FINE_NVEC * Ngc * kesz2, (size_t)FINE_NVEC * Ngc * sizeof(double)));
        c->ustc = b.take<double>((size_t)2 * Ngc);
        c->fpartc = b.take<double>((size_t)8 * c->max_ctas_c);
        c->fbarc = b.take<unsigned>(2);
        c->xc = b.take<double>(Ngc);
        c->yc = b.take<double>(Ngc);
        c->trajc = b.take<double>((size_t)(N + 1) * Ngc);
    }
    c->beta = b.take<double>((size_t)N * c->mcap0);
    c->gout = b.take<double>((size_t)N * c->maxK * c->maxK);
    c->lam = b.take<double>((size_t)N * c->maxK);
    c->Cm = b.take<double>((size_t)N * c->maxK * c->maxK);
    c->X = b.take<double>((size_t)N * c->mscr * c->mscr);
    c->gpart_n = gram_part_doubles(Ng, NB + 1, c->maxK, c->maxK);
    c->gpart = b.take<double>(c->gpart_n);
    c->colmax = b.take<unsigned long long>((size_t)(N + 1) * gram_tc_max_cols());
    c->counters = b.take<unsigned>((size_t)N + 64);
    c->colsA = b.take<const void*>((size_t)(N + 1) * c->ldcols);
    c->colsB = b.take<const void*>((size_t)(N + 1) * c->ldcols);
    c->colblk = b.take<int>((size_t)(N + 1) * c->ldcols);
    c->bases = b.take<const void*>((size_t)(N + 1) * 4);
    c->cntp = b.take<const int*>((size_t)(N + 1) * 4);
    c->KA = b.take<int>(N + 1);
    c->KB = b.take<int>(N + 1);
    c->ones = b.take<int>(N + 1);
    c->cnst = b.take<int>(8);
    const size_t kesz = c->fp32 ? sizeof(float) : sizeof(double);  // Krylov vectors
    c->fws_bytes = std::max((size_t)c->groups_max * FINE_NVEC * Ng * kesz,
                            (size_t)FINE_NVEC * Ng * sizeof(double));
    c->fws = b.take<char>(c->fws_bytes);
    c->ust = b.take<double>((size_t)c->groups_max * 2 * Ng);
    c->fpart = b.take<double>((size_t)8 * c->max_ctas);
    c->fbar = b.take<unsigned>((size_t)2 * c->groups_max);
    c->fstatus = b.take<int>(N + 1);
    c->fits = b.take<int>(N + 1);
    c->fitsmax = b.take<int>(N + 1);
    c->derr = b.take<int>(1);
    c->nonfin = b.take<int>(1);
    c->cd = b.take<double>(Ng);
    c->cLd = b.take<double>(Ng);
    c->cLtd = b.take<double>(Ng);
    c->cpart = b.take<double>(coarse_part_doubles(Ng, c->mcap2));
    c->npart = b.take<double>(norms_part_doubles(Ng, N + 1));
    c->nout = b.take<double>((size_t)4 * (N + 1));
    return b.off + 256;
}

Grid grid_of(const pr_ctx* c) {
    Grid g;
    g.n = c->n;
    g.Ng = c->Ng;
    g.h = c->h;
    g.eps = c->eps;
    g.tab = c->tab;
    g.pert = c->pert;
    return g;
}

pr_status init_ws(pr_ctx* c) {
    plan(c, c->ws);
    cudaStream_t st = c->st;
    PR_CUDA(cudaMemsetAsync(c->counters, 0, sizeof(unsigned) * ((size_t)c->N + 64), st));
    PR_CUDA(cudaMemsetAsync(c->derr, 0, sizeof(int), st));
    PR_CUDA(cudaMemsetAsync(c->fstatus, 0, sizeof(int) * ((size_t)c->N + 1), st));
    PR_CUDA(cudaMemsetAsync(c->fits, 0, sizeof(int) * ((size_t)c->N + 1), st));
    PR_CUDA(cudaMemsetAsync(c->fitsmax, 0, sizeof(int) * ((size_t)c->N + 1), st));
    PR_CUDA(cudaMemsetAsync(c->m1[0], 0, sizeof(int) * c->N, st));
    if (c->m1[1]) PR_CUDA(cudaMemsetAsync(c->m1[1], 0, sizeof(int) * c->N, st));
    PR_CUDA(cudaMemsetAsync(c->m2, 0, sizeof(int) * ((size_t)c->N + 1), st));
    PR_CUDA(cudaMemsetAsync(c->f, 0, sizeof(double) * c->Ng, st));
    PR_CUDA(cudaMemsetAsync(c->f32, 0, sizeof(float) * c->Ng, st));
    std::vector<int> ones(c->N + 1, 1);
    PR_CUDA(cudaMemcpy(c->ones, ones.data(), sizeof(int) * ones.size(), cudaMemcpyHostToDevice));
    int cn[8] = {c->ns, c->ns0, 0, 1, 0, 0, 0, 0};
    PR_CUDA(cudaMemcpy(c->cnst, cn, sizeof(cn), cudaMemcpyHostToDevice));
    PR_CUDA(launch_flow_tables(c->flow, c->n, c->L, c->tab, st));
    if (c->o.method == PR_METHOD_PARAREAL_II) {
        PR_CUDA(launch_flow_tables(c->flow, c->nc, c->L, c->tabc, st));
        PR_CUDA(cudaMemsetAsync(c->fc, 0, sizeof(double) * c->Ngc, st));
        PR_CUDA(cudaMemsetAsync(c->fc32, 0, sizeof(float) * c->Ngc, st));
    }
    if (c->tdep) PR_CUDA(launch_g_fields(c->tab, c->n, c->gq, c->gq + c->Ng, st));
    if (c->pert) {
        PR_CUDA(cudaMemcpy(c->pert, c->pert_host.data(), sizeof(double) * 3 * c->Ng, cudaMemcpyHostToDevice));
        if (c->pert32) PR_CUDA(launch_to_float(c->pert, c->pert32, 3 * c->Ng, st));
        if (c->pertc) {
            // injection onto the coarse grid (the restriction of the coarse propagator)
            const int n = c->n, nc = c->nc;
            std::vector<double> pc((size_t)3 * c->Ngc);
            for (int d = 0; d < 3; ++d)
                for (int z = 0; z < nc; ++z)
                    for (int y = 0; y < nc; ++y)
                        for (int x = 0; x < nc; ++x)
                            pc[(size_t)d * c->Ngc + ((size_t)z * nc + y) * nc + x] =
                                c->pert_host[(size_t)d * c->Ng + ((size_t)(2 * z) * n + 2 * y) * n + 2 * x];
            PR_CUDA(cudaMemcpy(c->pertc, pc.data(), sizeof(double) * pc.size(), cudaMemcpyHostToDevice));
            if (c->pertc32) PR_CUDA(launch_to_float(c->pertc, c->pertc32, 3 * c->Ngc, st));
        }
    }
    if (!c->ev_ready) {
        for (auto& e : c->ev) PR_CUDA(cudaEventCreate(&e));
        c->ev_ready = true;
    }
    c->ws_ready = true;
    return PR_OK;
}

pr_status ensure_ws(pr_ctx* c) {
    if (c->ws_ready) return PR_OK;
    if (!c->ws) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, c->ws_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PR_ERR_OOM, "cudaMalloc of " + std::to_string(c->ws_bytes) +
                                           " bytes failed: " + cudaGetErrorString(e));
        }
        c->ws = (char*)p;
        c->own_ws = true;
    }
    return init_ws(c);
}

// Host-built block descriptors (bases/counts) for B batch items, nb blocks each, uploaded
// and expanded on the device into column pointer arrays.
pr_status upload_blocks(pr_ctx* c, const std::vector<const void*>& bases,
                        const std::vector<const int*>& cnts, int nb, int B, const void** cols,
                        int* K, int esize, int* blk = nullptr) {
    PR_CUDA(cudaMemcpyAsync(c->bases, bases.data(), sizeof(void*) * bases.size(),
                            cudaMemcpyHostToDevice, c->st));
    PR_CUDA(cudaMemcpyAsync(c->cntp, cnts.data(), sizeof(int*) * cnts.size(),
                            cudaMemcpyHostToDevice, c->st));
    // pageable async copies are staged before returning and stream-ordered, so the host
    // vectors may go out of scope and the next upload cannot overtake this expansion
    PR_CUDA(launch_assemble_cols(c->bases, c->cntp, nb, B, c->Ng, esize, cols, c->ldcols, K, blk, c->st));
    return PR_OK;
}

// Column pointer arrays for B contiguous blocks base + b*bstride (count cnt[b] or the
// same device int for all when cnt_stride = 0).
pr_status cols_contig(pr_ctx* c, const char* base, size_t bstride_bytes, const int* cnt, int cnt_stride,
                      int B, const void** cols, int* K, int esize) {
    std::vector<const void*> bs(B);
    std::vector<const int*> cs(B);
    for (int b = 0; b < B; ++b) {
        bs[b] = base + (size_t)b * bstride_bytes;
        cs[b] = cnt + (size_t)b * cnt_stride;
    }
    return upload_blocks(c, bs, cs, 1, B, cols, K, esize);
}

// POD_Mode + one Cholesky-QR pass on B batch items whose snapshot columns are already in
// (c->colsA, c->KA).  Result: dest + b*dest_bstride (columns of Ng), dims m_dest[b].
// ortho_blocks: the snapshot columns are blocks of orthonormal bases (c->colblk says
// which); the FP32 mode then takes their diagonal Gram blocks as the identity.
// Symmetric Grams of the FP32 mode: on the tensor cores (error-free BF16 digit products,
// FP64-accurate; gram_tc.cu) for 55..64 columns, which the double-float kernel does not
// take (gram_mode PR_GRAM_AUTO), for every width up to 64 (PR_GRAM_TENSOR), or never
// (PR_GRAM_DF); every other Gram runs in double-float or FP64.
// k_exact: every item has maxKA columns (a snapshot window), not a cap on a POD dimension
// that lives on the device; the automatic choice of the tensor cores needs the column
// count (a Gram of 4 columns under a cap of 32 is faster in double-float).
cudaError_t gram_auto(pr_ctx* c, const GramArgs& ga, bool in_f32, bool k_exact) {
    const int mode = c->o.gram_mode;
    const bool fits = c->fp32 && !in_f32 && ga.sym && ga.colblk == nullptr && ga.maxKA <= gram_tc_max_cols() &&
                      ga.B <= (c->wave > 0 ? c->wave : c->N) + 1;
    // measured crossovers against the double-float kernel (64 items x 262,144 points, wall
    // time incl. the column-maximum pass): the narrow tensor form (<= 32 columns) wins from
    // 20 columns (20: 2.7 vs 3.0 ms, 32: 3.3 vs 6.9 ms; 16: 2.1 vs 1.9), the wide one
    // (33..64) beyond the double-float kernel's 384 output tiles a pass (55 columns)
    const bool narrow = ga.maxKA >= 20 && ga.maxKA <= 32;
    const bool wide = ga.maxKA > 54;
    if (fits && (mode == PR_GRAM_TENSOR || (mode == PR_GRAM_AUTO && k_exact && (narrow || wide))))
        return launch_gram_tc(ga, c->colmax, gram_tc_max_cols(), c->derr, c->o.spin_limit, c->st);
    return launch_gram(ga, in_f32, in_f32, c->st);
}

pr_status pod_pipeline(pr_ctx* c, int B, int maxK, double gamma, double tau, bool in_f32, int cap,
                       int mmax, char* dest, size_t dest_bstride_elems, int* m_dest,
                       bool ortho_blocks = false, bool k_exact = true) {
    const bool f32 = false;  // bases and their Grams are FP64
    cudaStream_t st = c->st;
    // Gram W^T W
    GramArgs ga{};
    ga.colsA = c->colsA;
    ga.colsB = c->colsA;
    ga.KA = c->KA;
    ga.KB = c->KA;
    ga.ldcols = c->ldcols;
    ga.Ng = c->Ng;
    ga.B = B;
    ga.maxKA = maxK;
    ga.maxKB = maxK;
    ga.sym = true;
    ga.part = c->gpart;
    ga.counter = c->counters;
    ga.G = c->gout;
    ga.ldG = maxK;
    ga.ldG_b = (long long)maxK * maxK;
    ga.df = c->fp32;   // FP32 mode: double-float Grams and projections on the FP32 pipe
    // the bases leave Cholesky QR orthonormal to ~1e-15, far below the FP32 mode's accuracy
    ga.colblk = (c->fp32 && ortho_blocks && !in_f32) ? c->colblk : nullptr;
    PR_CUDA(gram_auto(c, ga, in_f32, k_exact));
    // eigenpairs + dimension + C = Y_m Lambda_m^{-1/2}
    EigArgs ea{};
    ea.G = c->gout;
    ea.ldG = maxK;
    ea.ldG_b = (long long)maxK * maxK;
    ea.K = c->KA;
    ea.maxK = maxK;
    ea.B = B;
    ea.gamma = gamma;
    ea.tau = tau;
    ea.cap = cap > 0 ? std::min(cap, mmax) : mmax;
    ea.lam = c->lam;
    ea.m = m_dest;
    ea.C = c->Cm;
    ea.ldC = mmax;
    ea.ldC_b = (long long)maxK * mmax;
    ea.err = c->derr;
    PR_CUDA(launch_eig_pod(ea, st));
    // R0 = W C -> scr[0]
    TsmmArgs ta{};
    ta.colsIn = c->colsA;
    ta.KIN = c->KA;
    ta.KOUT = m_dest;
    ta.ldcols = c->ldcols;
    ta.C = c->Cm;
    ta.ldC = mmax;
    ta.ldC_b = (long long)maxK * mmax;
    ta.out = c->scr[0];
    ta.ld_out_b = (long long)mmax * c->Ng;
    ta.Ng = c->Ng;
    ta.B = B;
    ta.maxKIN = maxK;
    ta.maxKOUT = mmax;
    ta.df = c->fp32;
    PR_CUDA(launch_tsmm(ta, in_f32, f32, st));
    // one Cholesky QR pass (reading R7): scr[0] -> dest
    pr_status s = cols_contig(c, c->scr[0], (size_t)mmax * c->Ng * c->esz, m_dest, 1, B, c->colsB, c->KB, c->esz);
    if (s != PR_OK) return s;
    GramArgs gb = ga;
    gb.colblk = nullptr;
    gb.colsA = c->colsB;
    gb.colsB = c->colsB;
    gb.KA = c->KB;
    gb.KB = c->KB;
    gb.maxKA = mmax;
    gb.maxKB = mmax;
    gb.ldG = mmax;
    gb.ldG_b = (long long)mmax * mmax;
    PR_CUDA(gram_auto(c, gb, f32, false));   // m_dest columns per item, mmax a cap
    PR_CUDA(launch_chol_inv(c->gout, mmax, (long long)mmax * mmax, m_dest, mmax, B, c->X, mmax,
                            (long long)mmax * mmax, c->derr, st));
    TsmmArgs tb = ta;
    tb.colsIn = c->colsB;
    tb.KIN = c->KB;
    tb.KOUT = m_dest;
    tb.C = c->X;
    tb.ldC = mmax;
    tb.ldC_b = (long long)mmax * mmax;
    tb.maxKIN = mmax;
    tb.out = dest;
    tb.ld_out_b = (long long)dest_bstride_elems;
    PR_CUDA(launch_tsmm(tb, f32, f32, st));
    return PR_OK;
}

// Galerkin blocks of B bases (dest columns, counts m[b]): M = R^T R, L = R^T L_h R
// into Mo/Lo + b*mmax*mmax (ld mmax).
// Galerkin blocks of B bases R (eqs. (eq8)/(eq00)): Mo = R^T R and, with item stride
// 3 mmax^2 in Lo, R^T L R (steady flows) or the pieces R^T D R, R^T A0 R, R^T A1 R
// (time-dependent flows, L(t) = D + c0(t) A0 + c1(t) A1, D = -eps Lap_h).
pr_status galerkin(pr_ctx* c, char* R, size_t bstride_elems, const int* m, int B, int mmax, double* Mo,
                   double* Lo, bool orthonormal = false) {
    const bool f32 = false;
    pr_status s = cols_contig(c, R, bstride_elems * c->esz, m, 1, B, c->colsA, c->KA, c->esz);
    if (s != PR_OK) return s;
    s = cols_contig(c, c->LR, (size_t)mmax * c->Ng * c->esz, m, 1, B, c->colsB, c->KB, c->esz);
    if (s != PR_OK) return s;
    GramArgs ga{};
    ga.colsA = c->colsA;
    ga.colsB = c->colsA;
    ga.KA = c->KA;
    ga.KB = c->KA;
    ga.ldcols = c->ldcols;
    ga.Ng = c->Ng;
    ga.B = B;
    ga.maxKA = mmax;
    ga.maxKB = mmax;
    ga.sym = true;
    ga.part = c->gpart;
    ga.counter = c->counters;
    ga.G = Mo;
    ga.ldG = mmax;
    ga.ldG_b = (long long)mmax * mmax;
    ga.df = c->fp32;
    if (c->fp32 && orthonormal)
        // FP32 mode: the bases come out of a Cholesky-QR pass (orthonormal to ~1e-15), so
        // their mass matrix V^T V is the identity to that level; the FP64 mode forms it
        PR_CUDA(launch_identity(Mo, mmax, (long long)mmax * mmax, m, B, c->st));
    else
        PR_CUDA(launch_gram(ga, f32, f32, c->st));
    const Grid g = grid_of(c);
    Grid pieces[3] = {g, g, g};
    int np = 1;
    if (c->tdep) {
        pieces[0].tab = c->tab + (size_t)TAB_ZERO * c->n;   // D: no advection
        pieces[1].eps = 0.0;                                 // A0
        pieces[2].eps = 0.0;                                 // A1
        pieces[2].tab = c->tab + (size_t)TAB_B1 * c->n;
        np = 3;
    }
    ga.sym = false;
    ga.colsB = c->colsB;
    ga.KB = c->KB;
    ga.ldG_b = (long long)3 * mmax * mmax;
    for (int q = 0; q < np; ++q) {
        if (c->fp32)   // FP32 mode: double-float on the FP32 pipe
            PR_CUDA(launch_apply_L_df(pieces[q], c->colsA, (void* const*)c->colsB, c->KA, c->ldcols, mmax, B, c->st));
        else
            PR_CUDA(launch_apply_L(pieces[q], c->colsA, (void* const*)c->colsB, c->KA, c->ldcols, mmax, B, f32, f32,
                                   false, c->st));
        ga.G = Lo + (size_t)q * mmax * mmax;
        PR_CUDA(launch_gram(ga, f32, f32, c->st));
    }
    return PR_OK;
}

// Fine propagation of B subintervals; item b starts at t0 + b * DeltaT.
pr_status run_fine(pr_ctx* c, const double* u_in, double* u_out, char* snap, int B, int steps,
                   int n_snap, int stat_off, bool force_fp64, double t0, double DeltaT) {
    const bool f32 = c->fp32 && !force_fp64;
    FineArgs a{};
    a.g = grid_of(c);
    a.njobs = 1;
    FineJob& J = a.jobs[0];
    J.tab = c->tab;
    J.tdep = c->tdep ? 1 : 0;
    J.rk4 = c->o.fine == PR_FINE_RK4 ? 1 : 0;
    J.kind = c->flow.kind;
    J.w = c->flow.w;
    J.t0 = t0;
    J.DeltaT = DeltaT;
    J.eps = c->eps;
    J.dt = c->dt;
    J.S = steps;
    J.dM = c->dM;
    J.n_snap = snap ? n_snap : 0;
    J.f = c->has_f ? c->f : nullptr;
    J.f32 = c->has_f ? c->f32 : nullptr;
    J.u_in = u_in;
    J.u_out = u_out;
    J.snap = snap;
    J.tol = force_fp64 ? std::min(c->lin_tol, 1e-14) : c->lin_tol;
    J.maxit = c->o.lin_maxit;
    J.status = c->fstatus + stat_off;
    J.its_total = c->fits + stat_off;
    J.its_max = c->fitsmax + stat_off;
    J.B = B;
    J.pert = c->pert ? (f32 ? (const void*)c->pert32 : (const void*)c->pert) : nullptr;
    a.B = B;
    a.ws = c->fws;
    a.ust = c->ust;
    a.part = c->fpart;
    a.bar = c->fbar;
    a.G = c->o.group_ctas;
    a.spin_limit = c->o.spin_limit;
    a.err = c->derr;
    int max_groups = force_fp64 && c->fp32 ? 1 : c->groups_max;
    PR_CUDA(cudaMemsetAsync(c->fbar, 0, sizeof(unsigned) * 2 * c->groups_max, c->st));
    PR_CUDA(launch_fine(a, f32, c->o.ctas_per_sm, max_groups, c->st));
    return PR_OK;
}

// Parareal-II: implicit Euler with step dT on the grid coarsened by 2, one item, from
// x_in at time t0 for `steps` steps (with or without the forcing), snapshots every dM.
pr_status run_coarse_grid(pr_ctx* c, const double* x_in, double* y_out, double* snap, int steps, int n_snap,
                          int dM, double t0, bool with_forcing) {
    FineArgs a{};
    a.g.n = c->nc;
    a.g.Ng = c->Ngc;
    a.g.h = c->L / c->nc;
    a.g.eps = c->eps;
    a.g.tab = c->tabc;
    a.g.pert = c->pertc;
    a.njobs = 1;
    FineJob& J = a.jobs[0];
    J.tab = c->tabc;
    J.tdep = c->tdep ? 1 : 0;
    J.rk4 = 0;
    J.no_forcing = with_forcing ? 0 : 1;
    J.kind = c->flow.kind;
    J.w = c->flow.w;
    J.t0 = t0;
    J.DeltaT = 0.0;
    J.eps = c->eps;
    J.dt = c->dT;
    J.S = steps;
    J.dM = dM;
    J.n_snap = snap ? n_snap : 0;
    J.f = (with_forcing && c->has_f) ? c->fc : nullptr;
    J.f32 = (with_forcing && c->has_f) ? c->fc32 : nullptr;
    J.u_in = x_in;
    J.u_out = y_out;
    J.snap = snap;
    J.tol = c->lin_tol;
    J.maxit = c->o.lin_maxit;
    J.status = c->fstatus + c->N;
    J.its_total = c->fits + c->N;
    J.its_max = c->fitsmax + c->N;
    J.B = 1;
    J.pert = c->pertc ? (c->fp32 ? (const void*)c->pertc32 : (const void*)c->pertc) : nullptr;
    a.B = 1;
    a.ws = c->fwsc;
    a.ust = c->ustc;
    a.part = c->fpartc;
    a.bar = c->fbarc;
    a.G = 0;
    a.spin_limit = c->o.spin_limit;
    a.err = c->derr;
    PR_CUDA(cudaMemsetAsync(c->fbarc, 0, sizeof(unsigned) * 2, c->st));
    PR_CUDA(launch_fine(a, c->fp32, c->o.ctas_per_sm, 1, c->st));
    return PR_OK;
}

pr_status read_device_errors(pr_ctx* c) {
    int e = 0;
    PR_CUDA(cudaMemcpyAsync(&e, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    std::vector<int> stat(c->N + 1);
    PR_CUDA(cudaMemcpyAsync(stat.data(), c->fstatus, sizeof(int) * (c->N + 1), cudaMemcpyDeviceToHost,
                            c->st));
    PR_CUDA(cudaStreamSynchronize(c->st));
    if (e != 0) {
        PR_CUDA(cudaMemsetAsync(c->derr, 0, sizeof(int), c->st));
        return fail(c, (pr_status)e,
                    e == PR_ERR_TIMEOUT ? "in-kernel barrier exceeded its spin limit"
                                        : "a kernel recorded an error (Cholesky pivot or eigen size)");
    }
    for (int n = 0; n <= c->N; ++n) {
        if (stat[n] != 0) {
            PR_CUDA(cudaMemsetAsync(c->fstatus, 0, sizeof(int) * (c->N + 1), c->st));
            return fail(c, (pr_status)stat[n],
                        "fine propagator on subinterval " + std::to_string(n) + ": " +
                            pr_status_string((pr_status)stat[n]));
        }
    }
    return PR_OK;
}

pr_status check_finite_host(const double* x, long long n) {
    for (long long i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return PR_ERR_NONFINITE;
    return PR_OK;
}

// The blocks of eq. (W^k_n) for subinterval n: left neighbour (m_l = 1), this
// subinterval, previous iteration (p = 1; V0 at k = 1, reading R8), as (base, count).
struct L2Blocks {
    const void* base[3];
    const int* cnt[3];
};

// Level-2 POD (eq. (W^k_n)) and the Galerkin matrices of the result for subintervals
// n_lo .. n_hi-1 into R2 (item n at R2 + (n - n_lo) mcap2 columns), m2 + n, Mr/Lr at n;
// blocks(n) gives the level-1 blocks of n.
template <typename BlocksOf>
pr_status level2_range(pr_ctx* c, int n_lo, int n_hi, char* R2, BlocksOf blocks) {
    const int B2 = n_hi - n_lo;
    if (B2 <= 0) return PR_OK;
    const long long Ng = c->Ng;
    std::vector<const void*> bs;
    std::vector<const int*> cs;
    for (int n = n_lo; n < n_hi; ++n) {
        const L2Blocks q = blocks(n);
        for (int j = 0; j < 3; ++j) {
            bs.push_back(q.base[j]);
            cs.push_back(q.cnt[j]);
        }
    }
    pr_status s = upload_blocks(c, bs, cs, 3, B2, c->colsA, c->KA, c->esz, c->colblk);
    if (s != PR_OK) return s;
    s = pod_pipeline(c, B2, c->w2, c->gamma3, c->tau, false, c->o.m_cap, c->mcap2, R2, (size_t)c->mcap2 * Ng,
                     c->m2 + n_lo, true, false);
    if (s != PR_OK) return s;
    return galerkin(c, R2, (size_t)c->mcap2 * Ng, c->m2 + n_lo, B2, c->mcap2,
                    c->Mr + (size_t)n_lo * c->mcap2 * c->mcap2, c->Lr + (size_t)n_lo * 3 * c->mcap2 * c->mcap2, true);
}

// run_fine bracketed by a pair of the context's fine-launch events (pr_get_fine_ms).
pr_status run_fine_timed(pr_ctx* c, const double* u_in, double* u_out, char* snap, int B, int n_snap, int stat_off,
                         double t0) {
    if ((int)c->fev.size() < c->fev_used + 2) {
        for (int i = 0; i < 2; ++i) {
            cudaEvent_t e;
            PR_CUDA(cudaEventCreate(&e));
            c->fev.push_back(e);
        }
    }
    PR_CUDA(cudaEventRecord(c->fev[c->fev_used], c->st));
    pr_status s = run_fine(c, u_in, u_out, snap, B, c->S, n_snap, stat_off, false, t0, c->DeltaT);
    if (s != PR_OK) return s;
    PR_CUDA(cudaEventRecord(c->fev[c->fev_used + 1], c->st));
    c->fev_used += 2;
    return PR_OK;
}

// Level-1 POD of B snapshot windows (stride ns grid functions) into dest (stride mcap1).
pr_status level1(pr_ctx* c, const char* snap, int B, char* dest, int* m_dest) {
    const long long Ng = c->Ng;
    pr_status s = cols_contig(c, snap, (size_t)c->ns * Ng * sizeof(double), c->cnst + 0, 0, B, c->colsA, c->KA,
                              sizeof(double));
    if (s != PR_OK) return s;
    return pod_pipeline(c, B, c->ns, c->gamma1, c->tau1, false, c->o.m_cap, c->mcap1, dest, (size_t)c->mcap1 * Ng,
                        m_dest);
}

CoarseSweepArgs coarse_args(pr_ctx* c) {
    CoarseSweepArgs a{};
    a.g = grid_of(c);
    a.tdep = c->tdep ? 1 : 0;
    a.kind = c->flow.kind;
    a.w = c->flow.w;
    a.t0 = c->T0;
    a.DeltaT = c->DeltaT;
    a.A1d = c->cA1;
    a.ldM = c->mcap2;
    a.maxm = c->mcap2;
    a.dT = c->dT;
    a.Lc = c->Lc;
    a.aug_tol = c->o.aug_tol;
    a.augment = 1;
    a.d = c->cd;
    a.Ld = c->cLd;
    a.Ltd = c->cLtd;
    a.part = c->cpart;
    a.bar = c->counters + c->N + 16;
    a.spin_limit = c->o.spin_limit;
    a.err = c->derr;
    return a;
}

// The sequential augmented coarse sweep of eq. (formula4) over n = n_lo .. n_hi-1 of
// iteration k: U^k_{n+1} = G(U^k_n) + F_n - G(P U^{k-1}_n) into Ubuf[1 - cur], with the
// level-2 bases of item n at R2 + (n - n_lo) mcap2 columns.
pr_status coarse_range(pr_ctx* c, int n_lo, int n_hi, const char* R2) {
    if (n_hi <= n_lo) return PR_OK;
    const long long Ng = c->Ng;
    CoarseSweepArgs a = coarse_args(c);
    a.n0 = n_lo;
    a.count = n_hi - n_lo;
    a.U = c->Ubuf[1 - c->cur];
    a.sU = Ng;
    a.Up = c->Ubuf[c->cur];
    a.sUp = Ng;
    a.F = c->Fend;
    a.sF = Ng;
    a.out = c->Ubuf[1 - c->cur] + Ng;
    a.sOut = Ng;
    a.sR = (long long)c->mcap2 * Ng;
    a.R = reinterpret_cast<const double*>(R2) - (size_t)n_lo * a.sR;   // item n at a.R + n sR
    a.m = c->m2;
    a.sm = 1;
    a.Mr = c->Mr;
    a.Lr = c->Lr;
    a.sM = (long long)c->mcap2 * c->mcap2;
    a.sML = (long long)3 * c->mcap2 * c->mcap2;
    PR_CUDA(cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), c->st));
    PR_CUDA(launch_coarse_sweep(a, c->st));
    return PR_OK;
}

// Wave mode: iteration k streamed over waves of subintervals n = k-1, k, ... in order.
// For each wave: the fine sweep with its snapshots; the level-1 POD into the wave's
// bases; the level-2 POD and Galerkin matrices of the wave's subintervals n >= k (left
// neighbour: the wave's, or the one the previous wave committed; previous-iteration
// block: the committed basis of iteration k-1, or V0 at k = 1); the coarse sweep over the
// same subintervals, which continues from U^k_n that the previous wave's sweep wrote;
// then the wave's level-1 bases replace the committed ones.  Every step sees exactly the
// inputs it has in the single-launch form, in the same order.
pr_status wave_sweep(pr_ctx* c, int k) {
    const long long Ng = c->Ng;
    const int N = c->N, W = c->wave;
    const size_t bstride = (size_t)c->mcap1 * Ng * c->esz;
    const double* Uold = c->Ubuf[c->cur];
    double* Unew = c->Ubuf[1 - c->cur];
    c->fev_used = 0;
    // U^k_n = U^{k-1}_n for n < k (reading R10)
    PR_CUDA(cudaMemcpyAsync(Unew, Uold, sizeof(double) * (size_t)k * Ng, cudaMemcpyDeviceToDevice, c->st));
    for (int a = k - 1; a < N; a += W) {
        const int nb = std::min(W, N - a);
        pr_status s = run_fine_timed(c, Uold + (size_t)a * Ng, c->Fend + (size_t)a * Ng, c->snap, nb, c->ns, a,
                                     c->T0 + a * c->DeltaT);
        if (s != PR_OK) return s;
        c->wave_lo = a;
        c->wave_hi = a + nb;
        if (a == k - 1)   // U^k_k = F_{k-1} (reading R10)
            PR_CUDA(cudaMemcpyAsync(Unew + (size_t)k * Ng, c->Fend + (size_t)(k - 1) * Ng, sizeof(double) * Ng,
                                    cudaMemcpyDeviceToDevice, c->st));
        s = level1(c, c->snap, nb, c->R1t, c->m1t);
        if (s != PR_OK) return s;
        const int n_lo = std::max(a, k), n_hi = a + nb;
        s = level2_range(c, n_lo, n_hi, c->R2, [&](int n) {
            L2Blocks q{};
            if (c->o.m_l >= 1) {
                const bool in_wave = n - 1 >= a;
                q.base[0] = in_wave ? c->R1t + (size_t)(n - 1 - a) * bstride : c->R1[0] + (size_t)(n - 1) * bstride;
                q.cnt[0] = in_wave ? c->m1t + (n - 1 - a) : c->m1[0] + (n - 1);
            }
            q.base[1] = c->R1t + (size_t)(n - a) * bstride;
            q.cnt[1] = c->m1t + (n - a);
            if (c->o.p >= 1) {
                q.base[2] = k == 1 ? (const void*)c->V0 : (const void*)(c->R1[0] + (size_t)n * bstride);
                q.cnt[2] = k == 1 ? c->m0 : c->m1[0] + n;
            }
            return q;
        });
        if (s != PR_OK) return s;
        s = coarse_range(c, n_lo, n_hi, c->R2);
        if (s != PR_OK) return s;
        PR_CUDA(cudaMemcpyAsync(c->R1[0] + (size_t)a * bstride, c->R1t, (size_t)nb * bstride, cudaMemcpyDeviceToDevice,
                                c->st));
        PR_CUDA(cudaMemcpyAsync(c->m1[0] + a, c->m1t, sizeof(int) * nb, cudaMemcpyDeviceToDevice, c->st));
        c->r2_lo = n_lo;
        c->r2_hi = n_hi;
    }
    return PR_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

void pr_opts_init(pr_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->m_l = 1;
    o->p = 1;
    o->precision = PR_FP64;
    o->lin_maxit = 200;
    o->aug_tol = 1e-12;
    o->spin_limit = 1LL << 22;
    o->method = PR_METHOD_ADAPTIVE;
    o->fine = PR_FINE_IMPLICIT_EULER;
    o->wave = 0;
    o->gram_mode = PR_GRAM_AUTO;
}

const char* pr_status_string(pr_status s) {
    switch (s) {
        case PR_OK: return "ok";
        case PR_ERR_INVALID_ARG: return "invalid argument";
        case PR_ERR_OOM: return "out of device memory";
        case PR_ERR_CUDA: return "CUDA error";
        case PR_ERR_NOT_CONVERGED: return "BiCGStab did not converge";
        case PR_ERR_BREAKDOWN: return "breakdown";
        case PR_ERR_TIMEOUT: return "in-kernel barrier timed out";
        case PR_ERR_NONFINITE: return "non-finite value";
        case PR_ERR_STATE: return "phase called out of order";
        case PR_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* pr_last_error(const pr_ctx* c) { return c ? c->err.c_str() : "null context"; }

long long pr_launch_count(void) { return g_launch_count; }

pr_status pr_create(const pr_grid* grid, const pr_flow* flow, double eps, double T, int n_sub,
                    double dt_fine, double pod_tol, const pr_opts* opts, pr_ctx** out) {
    if (!out) return PR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid || !flow) return PR_ERR_INVALID_ARG;
    if (grid->n < 4 || grid->n > 256) return PR_ERR_UNSUPPORTED;
    if (!(eps > 0) || !(T > 0) || n_sub < 1 || !(dt_fine > 0) || !(pod_tol >= 0 && pod_tol < 1))
        return PR_ERR_INVALID_ARG;
    if (flow->kind < PR_FLOW_ABC || flow->kind > PR_FLOW_PAPER_ABC) return PR_ERR_INVALID_ARG;
    if (flow->kind == PR_FLOW_PAPER_ABC && !std::isfinite(flow->w)) return PR_ERR_INVALID_ARG;
    pr_opts o;
    if (opts) o = *opts; else pr_opts_init(&o);
    if (o.m_l < 0 || o.m_l > 1 || o.p < 0 || o.p > 1) return PR_ERR_UNSUPPORTED;
    if (o.precision != PR_FP64 && o.precision != PR_FP32) return PR_ERR_INVALID_ARG;
    if (o.method != PR_METHOD_ADAPTIVE && o.method != PR_METHOD_PARAREAL_I && o.method != PR_METHOD_PARAREAL_II)
        return PR_ERR_INVALID_ARG;
    if (o.method == PR_METHOD_PARAREAL_II && (grid->n % 2 != 0 || grid->n / 2 < 4)) return PR_ERR_UNSUPPORTED;
    if (o.fine != PR_FINE_IMPLICIT_EULER && o.fine != PR_FINE_RK4) return PR_ERR_INVALID_ARG;
    if (o.lin_maxit <= 0) o.lin_maxit = 200;
    if (o.spin_limit < 0) o.spin_limit = 1LL << 22;
    if (o.aug_tol <= 0) o.aug_tol = 1e-12;
    if (o.wave < 0) return PR_ERR_INVALID_ARG;
    if (o.gram_mode < PR_GRAM_AUTO || o.gram_mode > PR_GRAM_TENSOR) return PR_ERR_INVALID_ARG;
    if (o.wave > 0 && o.method != PR_METHOD_ADAPTIVE) return PR_ERR_UNSUPPORTED;   // waves stream Algorithm 2
    pr_ctx* c = new pr_ctx();
    c->n = grid->n;
    c->L = grid->L > 0 ? grid->L : 2.0 * M_PI;
    c->h = c->L / c->n;
    c->Ng = (long long)c->n * c->n * c->n;
    c->flow = *flow;
    c->flow.pert = nullptr;   // the caller's array is copied below, never kept
    c->tdep = flow_time_dependent(flow->kind);
    if (flow->pert) {
        if (c->tdep || o.fine == PR_FINE_RK4) {
            delete c;
            return PR_ERR_UNSUPPORTED;   // the perturbation is a steady field of the implicit path
        }
        const size_t np = (size_t)3 * grid->n * grid->n * grid->n;
        c->pert_host.assign(flow->pert, flow->pert + np);
        for (double v : c->pert_host)
            if (!std::isfinite(v)) {
                delete c;
                return PR_ERR_INVALID_ARG;
            }
    }
    c->eps = eps;
    c->T = T;
    c->N = n_sub;
    c->pod_tol = pod_tol;
    c->o = o;
    c->fp32 = o.precision == PR_FP32;
    c->esz = 8;  // POD bases are FP64 in both modes (the augmentation needs them exact)
    c->wave = (o.wave > 0 && o.wave < n_sub) ? o.wave : 0;
    c->DeltaT = T / n_sub;
    c->S = steps_for(c->DeltaT, dt_fine);
    c->dt = c->DeltaT / c->S;
    c->T0 = o.T0 > 0 ? o.T0 : c->DeltaT;
    c->S0 = steps_for(c->T0, c->dt);
    const double dT = o.dT > 0 ? o.dT : c->DeltaT / 10.0;
    c->Lc = steps_for(c->DeltaT, dT);
    c->dT = c->DeltaT / c->Lc;
    if (o.n_snap > 0) {
        if (o.n_snap < 2) { delete c; return PR_ERR_INVALID_ARG; }
        c->dM = std::max(1, c->S / (o.n_snap - 1));
    } else {
        c->dM = 5;
    }
    c->ns = c->S / c->dM + 1;
    c->ns0 = c->S0 / c->dM + 1;
    if (o.n_snap > 0) {
        c->ns = std::min(c->ns, o.n_snap);
        c->ns0 = std::min(c->ns0, o.n_snap);
    }
    c->nsmax = std::max(c->ns, c->ns0);
    c->gamma1 = 1.0 - pod_tol;
    c->gamma3 = 1.0 - (o.pod_tol3 > 0 ? o.pod_tol3 : pod_tol * 4e-3);
    c->tau = o.rank_tau > 0 ? o.rank_tau : 1e-13;
    c->lin_tol = o.lin_tol > 0 ? o.lin_tol : (c->fp32 ? 1e-9 : 1e-14);
    const int cap = o.m_cap;
    c->mcap0 = cap > 0 ? std::min(cap, c->ns0) : c->ns0;
    c->mcap1 = cap > 0 ? std::min(cap, c->ns) : c->ns;
    c->w2 = (o.m_l + 1) * c->mcap1 + o.p * std::max(c->mcap1, c->mcap0);
    c->mcap2 = cap > 0 ? std::min(cap, c->w2) : c->w2;
    c->mscr = std::max(c->mcap0, std::max(c->mcap1, c->mcap2));
    c->maxK = std::max(c->nsmax, c->w2);
    c->ldcols = c->maxK + 2;
    c->has_f = false;
    if (c->mcap2 > 32 || c->mcap0 > 33 || (o.method == PR_METHOD_PARAREAL_I && c->mcap0 > coarse_max_m())) {
        delete c;
        return PR_ERR_UNSUPPORTED;  // reduced systems are solved in one CTA (<= 33 unknowns)
    }
    if (c->maxK > 96) {
        delete c;
        return PR_ERR_UNSUPPORTED;  // Gram eigenproblems up to 96 x 96 (one CTA each)
    }
    if (o.method == PR_METHOD_PARAREAL_II) {
        c->nc = c->n / 2;
        c->Ngc = (long long)c->nc * c->nc * c->nc;
        c->max_ctas_c = std::max(fine_max_ctas(c->nc, c->fp32, o.ctas_per_sm), fine_max_ctas(c->nc, false, o.ctas_per_sm));
    }
    c->max_ctas = fine_max_ctas(c->n, c->fp32, o.ctas_per_sm);
    c->max_ctas = std::max(c->max_ctas, fine_max_ctas(c->n, false, o.ctas_per_sm));
    c->groups_max = std::max(1, std::min(c->wave > 0 ? c->wave : c->N, c->max_ctas));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        delete c;
        return PR_ERR_CUDA;
    }
    c->ws_bytes = plan(c, nullptr);
    *out = c;
    return PR_OK;
}

void pr_destroy(pr_ctx* c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    if (c->own_ws && c->ws) cudaFree(c->ws);
    if (c->ref) cudaFree(c->ref);
    if (c->ev_ready)
        for (auto& e : c->ev) cudaEventDestroy(e);
    for (auto& e : c->fev) cudaEventDestroy(e);
    delete c;
}

pr_status pr_get_sizes(const pr_ctx* c, int* S, int* S0, int* dM, int* n_s, int* n_s0, int* Lc,
                       double* dt_eff, double* DeltaT) {
    if (!c) return PR_ERR_INVALID_ARG;
    if (S) *S = c->S;
    if (S0) *S0 = c->S0;
    if (dM) *dM = c->dM;
    if (n_s) *n_s = c->ns;
    if (n_s0) *n_s0 = c->ns0;
    if (Lc) *Lc = c->Lc;
    if (dt_eff) *dt_eff = c->dt;
    if (DeltaT) *DeltaT = c->DeltaT;
    return PR_OK;
}

size_t pr_workspace_bytes(const pr_ctx* c) { return c ? c->ws_bytes : 0; }

pr_status pr_bind_workspace(pr_ctx* c, void* p, size_t bytes) {
    if (!c || !p) return PR_ERR_INVALID_ARG;
    if (bytes < c->ws_bytes) return fail(c, PR_ERR_OOM, "bound workspace smaller than pr_workspace_bytes");
    if ((reinterpret_cast<uintptr_t>(p) & 255) != 0) return fail(c, PR_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (c->own_ws && c->ws) cudaFree(c->ws);
    c->own_ws = false;
    c->ws = (char*)p;
    c->ws_ready = false;
    c->k_done = -1;
    c->phase = 0;
    c->initial_set = false;
    return init_ws(c);
}

pr_status pr_set_stream(pr_ctx* c, void* s) {
    if (!c) return PR_ERR_INVALID_ARG;
    c->st = (cudaStream_t)s;
    return PR_OK;
}

pr_status pr_set_initial(pr_ctx* c, const double* u0, const double* f) {
    if (!c || !u0) return PR_ERR_INVALID_ARG;
    if (check_finite_host(u0, c->Ng) != PR_OK || (f && check_finite_host(f, c->Ng) != PR_OK))
        return fail(c, PR_ERR_NONFINITE, "initial state or forcing holds NaN/Inf");
    pr_status s = ensure_ws(c);
    if (s != PR_OK) return s;
    PR_CUDA(cudaMemcpyAsync(c->u0, u0, sizeof(double) * c->Ng, cudaMemcpyHostToDevice, c->st));
    if (f) PR_CUDA(cudaMemcpyAsync(c->f, f, sizeof(double) * c->Ng, cudaMemcpyHostToDevice, c->st));
    else PR_CUDA(cudaMemsetAsync(c->f, 0, sizeof(double) * c->Ng, c->st));
    PR_CUDA(launch_to_float(c->f, c->f32, c->Ng, c->st));
    if (c->o.method == PR_METHOD_PARAREAL_II) {   // the forcing at the coarse points
        PR_CUDA(launch_restrict_diff(c->f, nullptr, c->n, 2, c->fc, c->st));
        PR_CUDA(launch_to_float(c->fc, c->fc32, c->Ngc, c->st));
    }
    PR_CUDA(cudaStreamSynchronize(c->st));
    c->has_f = f != nullptr;
    c->initial_set = true;
    c->k_done = -1;
    c->phase = 0;
    return PR_OK;
}

pr_status pr_iteration0(pr_ctx* c) {
    if (!c) return PR_ERR_INVALID_ARG;
    if (!c->initial_set) return fail(c, PR_ERR_STATE, "pr_set_initial first");
    pr_status s;
    const long long Ng = c->Ng;
    double* U = c->Ubuf[0];
    c->cur = 0;
    if (c->o.method == PR_METHOD_PARAREAL_II) {
        // u_hat0 = F(0, T0, u0); the coarse trajectory x_{n+1} = G_c(x_n) from x_0 = R u_hat0
        // (R P = I), U^0_n = P x_n
        s = run_fine(c, c->u0, U, nullptr, 1, c->S0, 0, 0, false, 0.0, 0.0);
        if (s != PR_OK) return s;
        PR_CUDA(launch_restrict_diff(U, nullptr, c->n, 2, c->xc, c->st));
        s = run_coarse_grid(c, c->xc, c->yc, c->trajc, c->N * c->Lc, c->N + 1, c->Lc, c->T0, true);
        if (s != PR_OK) return s;
        PR_CUDA(launch_prolong_add(c->trajc + c->Ngc, c->Ngc, c->n, 2, nullptr, 0, U + Ng, Ng, c->N, c->st));
        c->r1cur = 0;
        c->k_done = 0;
        c->phase = 0;
        c->checked = true;
        return PR_OK;
    }
    // fine propagator on [0, T0] with snapshots (slot 0 of the snapshot store)
    s = run_fine(c, c->u0, U, c->snap, 1, c->S0, c->ns0, 0, false, 0.0, 0.0);
    if (s != PR_OK) return s;
    // V0 = POD_Mode(W, gamma1)
    s = cols_contig(c, c->snap, 0, c->cnst + 1, 0, 1, c->colsA, c->KA, sizeof(double));
    if (s != PR_OK) return s;
    s = pod_pipeline(c, 1, c->ns0, c->gamma1, c->tau1, false, c->o.m_cap, c->mcap0, c->V0,
                     (size_t)c->mcap0 * Ng, c->m0);
    if (s != PR_OK) return s;

    // Galerkin matrices of V0 and projections of u_hat0, f
    s = galerkin(c, c->V0, (size_t)c->mcap0 * Ng, c->m0, 1, c->mcap0, c->M0, c->L0);
    if (s != PR_OK) return s;
    {
        // p0 = V0^T u_hat0, q0 = V0^T f : gram of V0 columns against [u_hat0, f]
        std::vector<const void*> bs = {U, c->f};
        PR_CUDA(cudaMemcpyAsync(c->colsB, bs.data(), sizeof(void*) * 2, cudaMemcpyHostToDevice, c->st));
        PR_CUDA(cudaStreamSynchronize(c->st));
        GramArgs ga{};
        ga.colsA = c->colsA;  // V0 columns from galerkin()
        ga.colsB = c->colsB;
        ga.KA = c->KA;
        ga.KB = c->cnst + 3;  // 1 column
        ga.ldcols = 0;
        ga.Ng = Ng;
        ga.B = 1;
        ga.maxKA = c->mcap0;
        ga.maxKB = 1;
        ga.part = c->gpart;
        ga.counter = c->counters;
        ga.G = c->p0;
        ga.ldG = 1;
        ga.ldG_b = 0;
        PR_CUDA(launch_gram(ga, false, false, c->st));
        if (c->has_f) {
            ga.colsB = c->colsB + 1;
            ga.G = c->q0;
            PR_CUDA(launch_gram(ga, false, false, c->st));
        }
        if (c->tdep) {
            // qg = V0^T g^0, V0^T g^1: the time-dependent forcing pieces
            std::vector<const void*> gs = {c->gq, c->gq + Ng};
            PR_CUDA(cudaMemcpyAsync(c->colsB + 2, gs.data(), sizeof(void*) * 2, cudaMemcpyHostToDevice, c->st));
            PR_CUDA(cudaStreamSynchronize(c->st));
            for (int q = 0; q < 2; ++q) {
                ga.colsB = c->colsB + 2 + q;
                ga.G = c->qg + (size_t)q * c->mcap0;
                PR_CUDA(launch_gram(ga, false, false, c->st));
            }
        }
    }
    G0Tdep td{};
    td.tdep = c->tdep ? 1 : 0;
    td.kind = c->flow.kind;
    td.w = c->flow.w;
    td.T0 = c->T0;
    td.qg = c->qg;
    PR_CUDA(launch_g0(c->M0, c->L0, c->p0, c->has_f ? c->q0 : nullptr, c->m0, c->mcap0, c->N, c->Lc, c->dT,
                      c->beta, c->mcap0, c->derr, td, c->st));
    // U^0_{n+1} = V0 beta_n
    s = cols_contig(c, c->V0, 0, c->m0, 0, c->N, c->colsA, c->KA, c->esz);
    if (s != PR_OK) return s;
    TsmmArgs ta{};
    ta.colsIn = c->colsA;
    ta.KIN = c->KA;
    ta.KOUT = c->ones;
    ta.ldcols = c->ldcols;
    ta.C = c->beta;
    ta.ldC = 1;
    ta.ldC_b = c->mcap0;
    ta.out = U + Ng;
    ta.ld_out_b = Ng;
    ta.Ng = Ng;
    ta.B = c->N;
    ta.maxKIN = c->mcap0;
    ta.maxKOUT = 1;
    PR_CUDA(launch_tsmm(ta, false, false, c->st));
    c->r1cur = 0;
    c->k_done = 0;
    c->phase = 0;
    c->checked = true;
    return PR_OK;
}

pr_status pr_fine_sweep(pr_ctx* c, int k) {
    if (!c) return PR_ERR_INVALID_ARG;
    if (k < 1 || k > c->N) return fail(c, PR_ERR_INVALID_ARG, "k out of range");
    if (c->k_done != k - 1 || c->phase != 0) return fail(c, PR_ERR_STATE, "pr_fine_sweep out of order");
    const long long Ng = c->Ng;
    const int B = c->N - k + 1;
    const double* Uprev = c->Ubuf[c->cur];
    const bool plain = c->o.method != PR_METHOD_ADAPTIVE;   // no snapshots needed
    if (c->wave > 0) {
        pr_status s = wave_sweep(c, k);
        if (s != PR_OK) return s;
        c->phase = 1;
        return PR_OK;
    }
    c->fev_used = 0;
    pr_status s = run_fine_timed(c, Uprev + (size_t)(k - 1) * Ng, c->Fend + (size_t)(k - 1) * Ng,
                                 plain ? nullptr : c->snap + (size_t)(k - 1) * c->ns * Ng * c->esz, B, c->ns,
                                 k - 1, c->T0 + (k - 1) * c->DeltaT);
    if (s != PR_OK) return s;
    c->phase = 1;
    return PR_OK;
}

pr_status pr_fine_sweep_batch(pr_ctx* const* ctxs, const int* ks, int count) {
    if (!ctxs || !ks || count < 1) return PR_ERR_INVALID_ARG;
    if (count > FINE_MAX_JOBS) return fail(ctxs[0], PR_ERR_INVALID_ARG, "more contexts than one fine launch holds");
    pr_ctx* owner = nullptr;
    for (int i = 0; i < count; ++i) {
        pr_ctx* c = ctxs[i];
        if (!c) return PR_ERR_INVALID_ARG;
        const int k = ks[i];
        if (k < 1 || k > c->N) return fail(c, PR_ERR_INVALID_ARG, "k out of range");
        if (c->k_done != k - 1 || c->phase != 0) return fail(c, PR_ERR_STATE, "pr_fine_sweep_batch out of order");
        if (!c->ws_ready) return fail(c, PR_ERR_STATE, "workspace not initialised (pr_set_initial first)");
        if (c->wave > 0) return fail(c, PR_ERR_UNSUPPORTED, "pr_fine_sweep_batch: contexts in wave mode sweep alone");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return fail(c, PR_ERR_INVALID_ARG, "a context appears twice");
        if (owner && (c->n != owner->n || c->L != owner->L || c->fp32 != owner->fp32 ||
                      c->o.fine != owner->o.fine || (c->pert != nullptr) != (owner->pert != nullptr)))
            return fail(c, PR_ERR_INVALID_ARG,
                        "batched contexts need the same grid, precision, fine integrator and stencil kind "
                        "(with or without a stored perturbation)");
        if (!owner || c->groups_max > owner->groups_max) owner = c;
    }
    FineArgs a{};
    a.g = grid_of(owner);
    a.njobs = count;
    a.B = 0;
    for (int i = 0; i < count; ++i) {
        pr_ctx* c = ctxs[i];
        const int k = ks[i];
        const long long Ng = c->Ng;
        FineJob& J = a.jobs[i];
        J.tab = c->tab;
        J.tdep = c->tdep ? 1 : 0;
        J.rk4 = c->o.fine == PR_FINE_RK4 ? 1 : 0;
        J.kind = c->flow.kind;
        J.w = c->flow.w;
        J.t0 = c->T0 + (k - 1) * c->DeltaT;
        J.DeltaT = c->DeltaT;
        J.eps = c->eps;
        J.dt = c->dt;
        J.S = c->S;
        J.dM = c->dM;
        const bool plain = c->o.method != PR_METHOD_ADAPTIVE;
        J.n_snap = plain ? 0 : c->ns;
        J.f = c->has_f ? c->f : nullptr;
        J.f32 = c->has_f ? c->f32 : nullptr;
        J.u_in = c->Ubuf[c->cur] + (size_t)(k - 1) * Ng;
        J.u_out = c->Fend + (size_t)(k - 1) * Ng;
        J.snap = plain ? nullptr : c->snap + (size_t)(k - 1) * c->ns * Ng * c->esz;
        J.tol = c->lin_tol;
        J.maxit = c->o.lin_maxit;
        J.status = c->fstatus + (k - 1);
        J.its_total = c->fits + (k - 1);
        J.its_max = c->fitsmax + (k - 1);
        J.B = c->N - k + 1;
        J.pert = c->pert ? (c->fp32 ? (const void*)c->pert32 : (const void*)c->pert) : nullptr;
        a.B += J.B;
    }
    a.ws = owner->fws;
    a.ust = owner->ust;
    a.part = owner->fpart;
    a.bar = owner->fbar;
    a.G = owner->o.group_ctas;
    a.spin_limit = owner->o.spin_limit;
    a.err = owner->derr;
    // order: each context's earlier work -> the launch on the owner's stream -> each
    // context's later work
    for (int i = 0; i < count; ++i) {
        pr_ctx* c = ctxs[i];
        if (c == owner) continue;
        PR_CUDA(cudaEventRecord(c->ev[7], c->st));
        PR_CUDA(cudaStreamWaitEvent(owner->st, c->ev[7], 0));
    }
    {
        pr_ctx* c = owner;
        PR_CUDA(cudaMemsetAsync(c->fbar, 0, sizeof(unsigned) * 2 * c->groups_max, c->st));
        PR_CUDA(launch_fine(a, c->fp32, c->o.ctas_per_sm, c->groups_max, c->st));
        PR_CUDA(cudaEventRecord(c->ev[7], c->st));
    }
    for (int i = 0; i < count; ++i) {
        pr_ctx* c = ctxs[i];
        if (c == owner) continue;
        PR_CUDA(cudaStreamWaitEvent(c->st, owner->ev[7], 0));
    }
    for (int i = 0; i < count; ++i) ctxs[i]->phase = 1;
    return PR_OK;
}

pr_status pr_tune_fine(pr_ctx* c, int steps, int* best_group_ctas, double* best_ms) {
    if (!c || !best_group_ctas) return PR_ERR_INVALID_ARG;
    if (c->k_done < 0 || c->phase != 0 || !c->ws_ready)
        return fail(c, PR_ERR_STATE, "pr_tune_fine needs iteration 0 done and no phase in progress");
    steps = std::max(1, std::min(steps, c->S));
    const int NY = c->n / fine_tile_rows(c->n);
    const int maxc = fine_max_ctas(c->n, c->fp32, c->o.ctas_per_sm);
    const double* u_in = c->Ubuf[c->cur];
    const int B = c->N;
    double best = 1e300;
    int bestG = 0;
    // candidates: the even split of every CTA slot over the subintervals, then whole
    // multiples of the y-block columns
    std::vector<int> cand{std::max(1, maxc / B)};
    for (int z = 1; NY * z <= maxc && z <= c->n; z *= 2)
        if (NY * z != cand[0]) cand.push_back(NY * z);
    for (int Gc : cand) {
        c->o.group_ctas = Gc;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {   // the first run warms up
            PR_CUDA(cudaEventRecord(c->ev[0], c->st));
            pr_status s = run_fine(c, u_in, c->Fend, nullptr, B, steps, 0, 0, false, c->T0, c->DeltaT);
            if (s != PR_OK) return s;
            PR_CUDA(cudaEventRecord(c->ev[1], c->st));
        }
        PR_CUDA(cudaEventSynchronize(c->ev[1]));
        PR_CUDA(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        if (ms < best) {
            best = ms;
            bestG = c->o.group_ctas;
        }
    }
    c->o.group_ctas = bestG;
    // the tuning sweeps leave no state behind: statuses and counts are cleared, F_n is
    // rewritten by the next fine sweep
    PR_CUDA(cudaMemsetAsync(c->fstatus, 0, sizeof(int) * (c->N + 1), c->st));
    PR_CUDA(cudaMemsetAsync(c->fits, 0, sizeof(int) * (c->N + 1), c->st));
    PR_CUDA(cudaMemsetAsync(c->fitsmax, 0, sizeof(int) * (c->N + 1), c->st));
    pr_status s = read_device_errors(c);
    if (s != PR_OK) return s;
    *best_group_ctas = bestG;
    if (best_ms) *best_ms = best;
    return PR_OK;
}

pr_status pr_pod_update(pr_ctx* c, int k) {
    if (!c) return PR_ERR_INVALID_ARG;
    if (c->k_done != k - 1 || c->phase != 1) return fail(c, PR_ERR_STATE, "pr_pod_update out of order");
    if (c->o.method != PR_METHOD_ADAPTIVE || c->wave > 0) {
        // plain parareal: no POD bases; wave mode: done wave by wave in pr_fine_sweep
        c->phase = 2;
        return PR_OK;
    }
    const long long Ng = c->Ng;
    const int N = c->N;
    pr_status s;
    // level 1: n = k-1 .. N-1 into R1[nw] (the other buffer)
    const int nw = 1 - c->r1cur;
    const size_t bstride = (size_t)c->mcap1 * Ng * c->esz;
    s = level1(c, c->snap + (size_t)(k - 1) * c->ns * Ng * sizeof(double), N - k + 1,
               c->R1[nw] + (size_t)(k - 1) * bstride, c->m1[nw] + (k - 1));
    if (s != PR_OK) return s;
    // level 2: n = k .. N-1 (left neighbour(s), this subinterval, previous iteration)
    s = level2_range(c, k, N, c->R2 + (size_t)k * c->mcap2 * Ng * c->esz, [&](int n) {
        L2Blocks q{};
        if (c->o.m_l >= 1) {
            q.base[0] = c->R1[nw] + (size_t)(n - 1) * bstride;
            q.cnt[0] = c->m1[nw] + (n - 1);
        }
        q.base[1] = c->R1[nw] + (size_t)n * bstride;
        q.cnt[1] = c->m1[nw] + n;
        if (c->o.p >= 1) {
            q.base[2] = k == 1 ? (const void*)c->V0 : (const void*)(c->R1[1 - nw] + (size_t)n * bstride);
            q.cnt[2] = k == 1 ? c->m0 : c->m1[1 - nw] + n;
        }
        return q;
    });
    if (s != PR_OK) return s;
    c->r1cur = nw;
    c->phase = 2;
    return PR_OK;
}

pr_status pr_coarse_sweep(pr_ctx* c, int k) {
    if (!c) return PR_ERR_INVALID_ARG;
    if (c->k_done != k - 1 || c->phase != 2) return fail(c, PR_ERR_STATE, "pr_coarse_sweep out of order");
    const long long Ng = c->Ng;
    const double* Uold = c->Ubuf[c->cur];
    double* Unew = c->Ubuf[1 - c->cur];
    if (c->wave > 0) {   // the sweep ran wave by wave inside pr_fine_sweep
        c->cur = 1 - c->cur;
        c->k_done = k;
        c->phase = 0;
        c->checked = false;
        return PR_OK;
    }
    PR_CUDA(cudaMemcpyAsync(Unew, Uold, sizeof(double) * (size_t)k * Ng, cudaMemcpyDeviceToDevice, c->st));
    PR_CUDA(cudaMemcpyAsync(Unew + (size_t)k * Ng, c->Fend + (size_t)(k - 1) * Ng, sizeof(double) * Ng,
                            cudaMemcpyDeviceToDevice, c->st));
    if (c->o.method == PR_METHOD_PARAREAL_II) {
        // U^k_{n+1} = F_n + P Phi_c R (U^k_n - U^{k-1}_n): G is affine, so the forcing
        // cancels and the coarse propagation of the difference is homogeneous
        for (int n = k; n < c->N; ++n) {
            PR_CUDA(launch_restrict_diff(Unew + (size_t)n * Ng, Uold + (size_t)n * Ng, c->n, 2, c->xc, c->st));
            pr_status s = run_coarse_grid(c, c->xc, c->yc, nullptr, c->Lc, 0, 1, c->T0 + n * c->DeltaT, false);
            if (s != PR_OK) return s;
            PR_CUDA(launch_prolong_add(c->yc, 0, c->n, 2, c->Fend + (size_t)n * Ng, 0, Unew + (size_t)(n + 1) * Ng,
                                       0, 1, c->st));
        }
        c->cur = 1 - c->cur;
        c->k_done = k;
        c->phase = 0;
        c->checked = false;
        return PR_OK;
    }
    if (c->o.method == PR_METHOD_ADAPTIVE) {
        pr_status s = coarse_range(c, k, c->N, c->R2 + (size_t)k * c->mcap2 * Ng * c->esz);
        if (s != PR_OK) return s;
        c->cur = 1 - c->cur;
        c->k_done = k;
        c->phase = 0;
        c->checked = false;
        return PR_OK;
    }
    // Parareal-I: G in the fixed space V0, no augmentation
    CoarseSweepArgs a = coarse_args(c);
    a.n0 = k;
    a.count = c->N - k;
    a.U = Unew;
    a.sU = Ng;
    a.Up = Uold;
    a.sUp = Ng;
    a.F = c->Fend;
    a.sF = Ng;
    a.out = Unew + Ng;
    a.sOut = Ng;
    a.R = reinterpret_cast<const double*>(c->V0);
    a.sR = 0;
    a.m = c->m0;
    a.sm = 0;
    a.Mr = c->M0;
    a.Lr = c->L0;
    a.sM = 0;
    a.sML = 0;
    a.ldM = c->mcap0;
    a.maxm = c->mcap0;
    a.augment = 0;
    PR_CUDA(cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), c->st));
    PR_CUDA(launch_coarse_sweep(a, c->st));
    c->cur = 1 - c->cur;
    c->k_done = k;
    c->phase = 0;
    c->checked = false;
    return PR_OK;
}

pr_status pr_check(pr_ctx* c, int k, double* max_inc, double* max_err) {
    if (!c) return PR_ERR_INVALID_ARG;
    if (c->k_done != k || k < 1) return fail(c, PR_ERR_STATE, "pr_check needs pr_coarse_sweep(k) first");
    const long long Ng = c->Ng;
    const int cnt = c->N + 1;
    PR_CUDA(launch_norms(c->Ubuf[c->cur], c->Ubuf[1 - c->cur], c->ref, Ng, cnt, c->npart, c->counters + 0,
                         c->nout, c->st));
    std::vector<double> h(4 * cnt);
    PR_CUDA(cudaMemcpyAsync(h.data(), c->nout, sizeof(double) * 4 * cnt, cudaMemcpyDeviceToHost, c->st));
    PR_CUDA(cudaStreamSynchronize(c->st));
    pr_status s = read_device_errors(c);
    if (s != PR_OK) return s;
    c->last_inc.assign(cnt, 0.0);
    c->last_err.assign(cnt, -1.0);
    double mi = 0.0, me = c->ref ? 0.0 : -1.0;
    bool finite = true;
    for (int n = 0; n < cnt; ++n) {
        const double d2 = h[4 * n], a2 = h[4 * n + 1];
        const double inc = a2 > 0 ? std::sqrt(d2 / a2) : std::sqrt(d2);
        c->last_inc[n] = inc;
        mi = std::max(mi, inc);
        if (!std::isfinite(inc)) finite = false;
        if (c->ref) {
            const double e2 = h[4 * n + 2], r2 = h[4 * n + 3];
            const double err = r2 > 0 ? std::sqrt(e2 / r2) : std::sqrt(e2);
            c->last_err[n] = err;
            me = std::max(me, err);
        }
    }
    c->checked = true;
    if (max_inc) *max_inc = mi;
    if (max_err) *max_err = me;
    if (!finite) return fail(c, PR_ERR_NONFINITE, "non-finite interface state");
    return PR_OK;
}

pr_status pr_sync(pr_ctx* c) {
    if (!c) return PR_ERR_INVALID_ARG;
    PR_CUDA(cudaStreamSynchronize(c->st));
    if (!c->ws_ready) return PR_OK;
    return read_device_errors(c);
}

static pr_status alloc_ref(pr_ctx* c) {
    if (c->ref) return PR_OK;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(double) * (size_t)(c->N + 1) * c->Ng);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PR_ERR_OOM, "reference allocation failed");
    }
    c->ref = (double*)p;
    return PR_OK;
}

pr_status pr_set_reference(pr_ctx* c, const double* U, int on_device) {
    if (!c || !U) return PR_ERR_INVALID_ARG;
    pr_status s = ensure_ws(c);
    if (s != PR_OK) return s;
    s = alloc_ref(c);
    if (s != PR_OK) return s;
    PR_CUDA(cudaMemcpyAsync(c->ref, U, sizeof(double) * (size_t)(c->N + 1) * c->Ng,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
    PR_CUDA(cudaStreamSynchronize(c->st));
    return PR_OK;
}

pr_status pr_compute_reference(pr_ctx* c, int fp64) {
    if (!c) return PR_ERR_INVALID_ARG;
    if (!c->initial_set) return fail(c, PR_ERR_STATE, "pr_set_initial first");
    pr_status s = alloc_ref(c);
    if (s != PR_OK) return s;
    const long long Ng = c->Ng;
    const bool force = fp64 != 0;
    s = run_fine(c, c->u0, c->ref, nullptr, 1, c->S0, 0, c->N, force, 0.0, 0.0);
    if (s != PR_OK) return s;
    for (int n = 0; n < c->N; ++n) {
        s = run_fine(c, c->ref + (size_t)n * Ng, c->ref + (size_t)(n + 1) * Ng, nullptr, 1, c->S, 0, c->N,
                     force, c->T0 + n * c->DeltaT, c->DeltaT);
        if (s != PR_OK) return s;
    }
    return pr_sync(c);
}

pr_status pr_solve(pr_ctx* c, double tol, int k_max, const double* ref, pr_report* rep) {
    if (!c) return PR_ERR_INVALID_ARG;
    if (!c->initial_set) return fail(c, PR_ERR_STATE, "pr_set_initial first");
    pr_status s;
    if (ref) {
        s = pr_set_reference(c, ref, 0);
        if (s != PR_OK) return s;
    }
    pr_report R;
    std::memset(&R, 0, sizeof(R));
    R.max_err = -1.0;
    const int kmax = (k_max <= 0) ? c->N : std::min(k_max, c->N);
    cudaEvent_t* ev = c->ev;
    PR_CUDA(cudaEventRecord(ev[0], c->st));
    if (c->k_done < 0) {
        s = pr_iteration0(c);
        if (s != PR_OK) return s;
    }
    PR_CUDA(cudaEventRecord(ev[1], c->st));
    PR_CUDA(cudaEventSynchronize(ev[1]));
    float ms = 0;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    R.t_iter0 = ms * 1e-3;
    R.t_total = R.t_iter0;
    long long its_sum = 0, steps_sum = 0;
    for (int k = c->k_done + 1; k <= kmax; ++k) {
        PR_CUDA(cudaEventRecord(ev[2], c->st));
        if ((s = pr_fine_sweep(c, k)) != PR_OK) return s;
        PR_CUDA(cudaEventRecord(ev[3], c->st));
        if ((s = pr_pod_update(c, k)) != PR_OK) return s;
        PR_CUDA(cudaEventRecord(ev[4], c->st));
        if ((s = pr_coarse_sweep(c, k)) != PR_OK) return s;
        PR_CUDA(cudaEventRecord(ev[5], c->st));
        double mi = 0, me = -1;
        if ((s = pr_check(c, k, &mi, &me)) != PR_OK) return s;
        PR_CUDA(cudaEventRecord(ev[6], c->st));
        PR_CUDA(cudaEventSynchronize(ev[6]));
        float a, b2, d, e2;
        cudaEventElapsedTime(&a, ev[2], ev[3]);
        cudaEventElapsedTime(&b2, ev[3], ev[4]);
        cudaEventElapsedTime(&d, ev[4], ev[5]);
        cudaEventElapsedTime(&e2, ev[5], ev[6]);
        R.t_fine += a * 1e-3;
        R.t_pod += b2 * 1e-3;
        R.t_coarse += d * 1e-3;
        R.t_check += e2 * 1e-3;
        R.t_total += (a + b2 + d + e2) * 1e-3;
        R.k = k;
        R.max_inc = mi;
        R.max_err = me;
        const int B = c->N - k + 1;
        R.fine_dof_steps += (double)B * c->S * (double)c->Ng;
        std::vector<int> tot(c->N + 1), mx(c->N + 1);
        PR_CUDA(cudaMemcpy(tot.data(), c->fits, sizeof(int) * (c->N + 1), cudaMemcpyDeviceToHost));
        PR_CUDA(cudaMemcpy(mx.data(), c->fitsmax, sizeof(int) * (c->N + 1), cudaMemcpyDeviceToHost));
        for (int n = k - 1; n < c->N; ++n) {
            its_sum += tot[n];
            R.lin_iters_max = std::max(R.lin_iters_max, mx[n]);
        }
        steps_sum += (long long)B * c->S;
        const double crit = c->ref ? me : mi;
        if (crit <= tol) {
            R.converged = 1;
            break;
        }
    }
    R.lin_iters_mean = steps_sum ? (double)its_sum / steps_sum : 0.0;
    {
        int m0 = 0;
        std::vector<int> m1(c->N), m2(c->N);
        PR_CUDA(cudaMemcpy(&m0, c->m0, sizeof(int), cudaMemcpyDeviceToHost));
        PR_CUDA(cudaMemcpy(m1.data(), c->m1[c->r1cur], sizeof(int) * c->N, cudaMemcpyDeviceToHost));
        PR_CUDA(cudaMemcpy(m2.data(), c->m2, sizeof(int) * c->N, cudaMemcpyDeviceToHost));
        R.m0 = m0;
        for (int n = std::max(0, R.k - 1); n < c->N; ++n) R.m1_max = std::max(R.m1_max, m1[n]);
        for (int n = std::max(1, R.k); n < c->N; ++n) R.m2_max = std::max(R.m2_max, m2[n]);
    }
    if (rep) *rep = R;
    return PR_OK;
}

pr_status pr_get_interface(pr_ctx* c, int n, double* out) {
    if (!c || !out || n < 0 || n > c->N) return PR_ERR_INVALID_ARG;
    if (c->k_done < 0) return fail(c, PR_ERR_STATE, "no iterate yet");
    PR_CUDA(cudaMemcpyAsync(out, c->Ubuf[c->cur] + (size_t)n * c->Ng, sizeof(double) * c->Ng,
                            cudaMemcpyDeviceToHost, c->st));
    PR_CUDA(cudaStreamSynchronize(c->st));
    return PR_OK;
}

pr_status pr_get_interfaces(pr_ctx* c, double* out) {
    if (!c || !out) return PR_ERR_INVALID_ARG;
    if (c->k_done < 0) return fail(c, PR_ERR_STATE, "no iterate yet");
    PR_CUDA(cudaMemcpyAsync(out, c->Ubuf[c->cur], sizeof(double) * (size_t)(c->N + 1) * c->Ng,
                            cudaMemcpyDeviceToHost, c->st));
    PR_CUDA(cudaStreamSynchronize(c->st));
    return PR_OK;
}

pr_status pr_set_interfaces(pr_ctx* c, const double* U, int k_done) {
    if (!c || !U || k_done < 0 || k_done >= c->N) return PR_ERR_INVALID_ARG;
    if (c->k_done < 0) return fail(c, PR_ERR_STATE, "iteration 0 must have run (V0 is part of the state)");
    if (k_done >= 1 && c->k_done < 1)
        return fail(c, PR_ERR_STATE, "level-1 bases of iteration k_done are not available");
    PR_CUDA(cudaMemcpyAsync(c->Ubuf[c->cur], U, sizeof(double) * (size_t)(c->N + 1) * c->Ng,
                            cudaMemcpyHostToDevice, c->st));
    c->k_done = k_done;
    c->phase = 0;
    return PR_OK;
}

pr_status pr_get_diagnostics(pr_ctx* c, double* inc, double* err, int* m0, int* m1, int* m2) {
    if (!c) return PR_ERR_INVALID_ARG;
    PR_CUDA(cudaStreamSynchronize(c->st));
    const int cnt = c->N + 1;
    if (inc) for (int n = 0; n < cnt; ++n) inc[n] = n < (int)c->last_inc.size() ? c->last_inc[n] : 0.0;
    if (err) for (int n = 0; n < cnt; ++n) err[n] = n < (int)c->last_err.size() ? c->last_err[n] : -1.0;
    if (!c->ws_ready) return PR_OK;
    if (m0) PR_CUDA(cudaMemcpy(m0, c->m0, sizeof(int), cudaMemcpyDeviceToHost));
    if (m1) PR_CUDA(cudaMemcpy(m1, c->m1[c->r1cur], sizeof(int) * c->N, cudaMemcpyDeviceToHost));
    if (m2) PR_CUDA(cudaMemcpy(m2, c->m2, sizeof(int) * c->N, cudaMemcpyDeviceToHost));
    return PR_OK;
}

pr_status pr_get_fine_ms(pr_ctx* c, double* ms, int* launches) {
    if (!c || !ms) return PR_ERR_INVALID_ARG;
    if (c->fev_used == 0) return fail(c, PR_ERR_STATE, "no fine sweep timed yet");
    PR_CUDA(cudaEventSynchronize(c->fev[c->fev_used - 1]));
    double t = 0.0;
    for (int i = 0; i < c->fev_used; i += 2) {
        float a = 0.f;
        PR_CUDA(cudaEventElapsedTime(&a, c->fev[i], c->fev[i + 1]));
        t += a;
    }
    *ms = t;
    if (launches) *launches = c->fev_used / 2;
    return PR_OK;
}

pr_status pr_get_lin_stats(pr_ctx* c, int* total, int* mx) {
    if (!c) return PR_ERR_INVALID_ARG;
    PR_CUDA(cudaStreamSynchronize(c->st));
    if (total) PR_CUDA(cudaMemcpy(total, c->fits, sizeof(int) * c->N, cudaMemcpyDeviceToHost));
    if (mx) PR_CUDA(cudaMemcpy(mx, c->fitsmax, sizeof(int) * c->N, cudaMemcpyDeviceToHost));
    return PR_OK;
}

pr_status pr_rewind(pr_ctx* c) {
    if (!c) return PR_ERR_INVALID_ARG;
    if (c->k_done < 1 || c->phase != 0) return fail(c, PR_ERR_STATE, "no completed iteration to undo");
    // wave mode keeps one generation of level-1 bases: iteration k >= 2 replaced those of
    // k-1 in place; iteration 1 used V0 instead, so it can be repeated
    if (c->wave > 0 && c->k_done > 1)
        return fail(c, PR_ERR_STATE, "wave mode can only undo iteration 1 (the level-1 bases of k-1 are replaced)");
    PR_CUDA(cudaStreamSynchronize(c->st));
    c->cur = 1 - c->cur;
    if (c->o.method == PR_METHOD_ADAPTIVE && c->wave == 0) c->r1cur = 1 - c->r1cur;
    c->k_done -= 1;
    c->phase = 0;
    return PR_OK;
}

pr_status pr_get_fine_end(pr_ctx* c, int n, double* out) {
    if (!c || !out || n < 0 || n >= c->N) return PR_ERR_INVALID_ARG;
    if (!c->ws_ready) return fail(c, PR_ERR_STATE, "no workspace");
    PR_CUDA(cudaMemcpyAsync(out, c->Fend + (size_t)n * c->Ng, sizeof(double) * c->Ng,
                            cudaMemcpyDeviceToHost, c->st));
    PR_CUDA(cudaStreamSynchronize(c->st));
    return PR_OK;
}

pr_status pr_get_snapshots(pr_ctx* c, int n, void* out) {
    if (!c || !out || n < 0 || n >= c->N) return PR_ERR_INVALID_ARG;
    if (!c->ws_ready) return fail(c, PR_ERR_STATE, "no workspace");
    const size_t per = (size_t)c->ns * c->Ng * sizeof(double);
    size_t slot = (size_t)n;
    if (c->wave > 0) {   // the store holds the last wave only
        if (n < c->wave_lo || n >= c->wave_hi)
            return fail(c, PR_ERR_STATE, "wave mode: the snapshots of this subinterval are not resident");
        slot = (size_t)(n - c->wave_lo);
    }
    PR_CUDA(cudaMemcpyAsync(out, c->snap + slot * per, per, cudaMemcpyDeviceToHost, c->st));
    PR_CUDA(cudaStreamSynchronize(c->st));
    return PR_OK;
}

pr_status pr_get_basis(pr_ctx* c, int level, int n, void* out, int* m_out) {
    if (!c || !m_out || level < 0 || level > 2) return PR_ERR_INVALID_ARG;
    if (level > 0 && (n < 0 || n >= c->N)) return PR_ERR_INVALID_ARG;
    if (!c->ws_ready) return fail(c, PR_ERR_STATE, "no workspace");
    const size_t col = (size_t)c->Ng * c->esz;
    const char* base;
    const int* mp;
    if (level == 0) { base = c->V0; mp = c->m0; }
    else if (level == 1) { base = c->R1[c->r1cur] + (size_t)n * c->mcap1 * col; mp = c->m1[c->r1cur] + n; }
    else if (c->wave > 0) {   // the last wave's level-2 bases only
        if (n < c->r2_lo || n >= c->r2_hi)
            return fail(c, PR_ERR_STATE, "wave mode: the level-2 basis of this subinterval is not resident");
        base = c->R2 + (size_t)(n - c->r2_lo) * c->mcap2 * col;
        mp = c->m2 + n;
    } else { base = c->R2 + (size_t)n * c->mcap2 * col; mp = c->m2 + n; }
    int m = 0;
    PR_CUDA(cudaMemcpyAsync(&m, mp, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    PR_CUDA(cudaStreamSynchronize(c->st));
    *m_out = m;
    if (out && m > 0) {
        PR_CUDA(cudaMemcpyAsync(out, base, (size_t)m * col, cudaMemcpyDeviceToHost, c->st));
        PR_CUDA(cudaStreamSynchronize(c->st));
    }
    return PR_OK;
}

// ---------------------------------------------------------------------------------
pr_status pr_op_apply_L(pr_ctx* c, const double* d_in, double* d_out, int count, int transpose) {
    if (!c || !d_in || !d_out || count < 0) return PR_ERR_INVALID_ARG;
    if (c->tdep) return fail(c, PR_ERR_UNSUPPORTED, "pr_op_apply_L: time-dependent flows need a time");
    pr_status s = ensure_ws(c);
    if (s != PR_OK) return s;
    Grid g = grid_of(c);
    for (int c0 = 0; c0 < count; c0 += c->N + 1) {
        const int B = std::min(count - c0, c->N + 1);
        std::vector<const void*> in(B), out(B);
        for (int b = 0; b < B; ++b) {
            in[b] = d_in + (size_t)(c0 + b) * c->Ng;
            out[b] = d_out + (size_t)(c0 + b) * c->Ng;
        }
        PR_CUDA(cudaMemcpyAsync(c->colsA, in.data(), sizeof(void*) * B, cudaMemcpyHostToDevice, c->st));
        PR_CUDA(cudaMemcpyAsync(c->colsB, out.data(), sizeof(void*) * B, cudaMemcpyHostToDevice, c->st));
        PR_CUDA(launch_apply_L(g, c->colsA, (void* const*)c->colsB, c->ones, 1, 1, B, false, false,
                               transpose != 0, c->st));
        PR_CUDA(cudaStreamSynchronize(c->st));
    }
    return PR_OK;
}

pr_status pr_op_apply_L_df(pr_ctx* c, const double* d_in, double* d_out, int count) {
    if (!c || !d_in || !d_out || count < 0) return PR_ERR_INVALID_ARG;
    if (c->tdep) return fail(c, PR_ERR_UNSUPPORTED, "pr_op_apply_L_df: time-dependent flows need a time");
    pr_status s = ensure_ws(c);
    if (s != PR_OK) return s;
    Grid g = grid_of(c);
    for (int c0 = 0; c0 < count; c0 += c->N + 1) {
        const int B = std::min(count - c0, c->N + 1);
        std::vector<const void*> in(B), out(B);
        for (int b = 0; b < B; ++b) {
            in[b] = d_in + (size_t)(c0 + b) * c->Ng;
            out[b] = d_out + (size_t)(c0 + b) * c->Ng;
        }
        PR_CUDA(cudaMemcpyAsync(c->colsA, in.data(), sizeof(void*) * B, cudaMemcpyHostToDevice, c->st));
        PR_CUDA(cudaMemcpyAsync(c->colsB, out.data(), sizeof(void*) * B, cudaMemcpyHostToDevice, c->st));
        PR_CUDA(launch_apply_L_df(g, c->colsA, (void* const*)c->colsB, c->ones, 1, 1, B, c->st));
        PR_CUDA(cudaStreamSynchronize(c->st));
    }
    return PR_OK;
}

pr_status pr_op_fine(pr_ctx* c, const double* d_in, double* d_out, void* d_snap, int B, double t0,
                     int steps, int dM, int n_snap) {
    if (!c || !d_in || !d_out || B < 1 || B > c->N || steps < 1) return PR_ERR_INVALID_ARG;
    if (n_snap < 0 || (n_snap > 0 && (!d_snap || dM < 1))) return PR_ERR_INVALID_ARG;
    pr_status s = ensure_ws(c);
    if (s != PR_OK) return s;
    const int saved = c->dM;
    c->dM = dM > 0 ? dM : 1;
    s = run_fine(c, d_in, d_out, (char*)d_snap, B, steps, n_snap, 0, false, t0, 0.0);
    c->dM = saved;
    if (s != PR_OK) return s;
    return pr_sync(c);
}

pr_status pr_op_pod(pr_ctx* c, const void* d_W, int w_f32, int n_cols, int B, double gamma, int cap,
                    void* d_R, int* m_out) {
    if (!c || !d_W || !d_R || !m_out || B < 1 || B > c->N || n_cols < 1) return PR_ERR_INVALID_ARG;
    if (n_cols > c->maxK || !(gamma > 0 && gamma <= 1)) return PR_ERR_INVALID_ARG;
    if (c->wave > 0 && B > c->wave) return fail(c, PR_ERR_INVALID_ARG, "wave mode: B above the wave size");
    const int mmax = cap > 0 ? std::min(cap, n_cols) : n_cols;
    if (mmax > c->mscr) return fail(c, PR_ERR_INVALID_ARG, "POD dimension above the context's cap");
    pr_status s = ensure_ws(c);
    if (s != PR_OK) return s;
    int nc = n_cols;
    PR_CUDA(cudaMemcpy(c->cnst + 2, &nc, sizeof(int), cudaMemcpyHostToDevice));
    const int wes = w_f32 ? 4 : 8;
    s = cols_contig(c, (const char*)d_W, (size_t)n_cols * c->Ng * wes, c->cnst + 2, 0, B, c->colsA, c->KA, wes);
    if (s != PR_OK) return s;
    s = pod_pipeline(c, B, n_cols, gamma, w_f32 ? 1e-6 : c->tau1, w_f32 != 0, cap, mmax, (char*)d_R,
                     (size_t)mmax * c->Ng, c->mop);
    if (s != PR_OK) return s;
    PR_CUDA(cudaMemcpyAsync(m_out, c->mop, sizeof(int) * B, cudaMemcpyDeviceToHost, c->st));
    return pr_sync(c);
}

pr_status pr_op_gram(pr_ctx* c, const double* d_W, int n_cols, int B, double* d_G, int tensor) {
    if (!c || !d_W || !d_G || B < 1 || n_cols < 1) return PR_ERR_INVALID_ARG;
    const int bmax = (c->wave > 0 ? c->wave : c->N) + 1;   // partial sums: gram_part_doubles(Ng, bmax, ...)
    if (B > bmax || n_cols > c->maxK) return fail(c, PR_ERR_INVALID_ARG, "pr_op_gram: B or n_cols above the context's sizes");
    if (tensor < 0 || tensor > 2) return fail(c, PR_ERR_INVALID_ARG, "pr_op_gram: tensor must be 0, 1 or 2");
    if (tensor == 1 && n_cols > gram_tc_max_cols())
        return fail(c, PR_ERR_INVALID_ARG, "pr_op_gram: the tensor-core Gram takes at most 64 columns");
    pr_status s = ensure_ws(c);
    if (s != PR_OK) return s;
    int nc = n_cols;
    PR_CUDA(cudaMemcpyAsync(c->cnst + 2, &nc, sizeof(int), cudaMemcpyHostToDevice, c->st));
    s = cols_contig(c, (const char*)d_W, (size_t)n_cols * c->Ng * sizeof(double), c->cnst + 2, 0, B, c->colsA, c->KA,
                    sizeof(double));
    if (s != PR_OK) return s;
    GramArgs ga{};
    ga.colsA = c->colsA;
    ga.colsB = c->colsA;
    ga.KA = c->KA;
    ga.KB = c->KA;
    ga.ldcols = c->ldcols;
    ga.Ng = c->Ng;
    ga.B = B;
    ga.maxKA = n_cols;
    ga.maxKB = n_cols;
    ga.sym = true;
    ga.part = c->gpart;
    ga.counter = c->counters;
    ga.G = d_G;
    ga.ldG = n_cols;
    ga.ldG_b = (long long)n_cols * n_cols;
    ga.df = (tensor == 2);
    if (tensor == 1) PR_CUDA(launch_gram_tc(ga, c->colmax, gram_tc_max_cols(), c->derr, c->o.spin_limit, c->st));
    else PR_CUDA(launch_gram(ga, false, false, c->st));
    return pr_sync(c);
}

pr_status pr_op_coarse_update(pr_ctx* c, const void* d_R, int m, const double* d_U, const double* d_Uprev,
                              const double* d_F, double* d_out) {
    if (!c || !d_R || !d_U || !d_Uprev || !d_F || !d_out || m < 0) return PR_ERR_INVALID_ARG;
    if (m > c->mcap2) return fail(c, PR_ERR_INVALID_ARG, "m above the context's level-2 cap");
    if (c->tdep) return fail(c, PR_ERR_UNSUPPORTED, "pr_op_coarse_update: time-dependent flows need a time");
    pr_status s = ensure_ws(c);
    if (s != PR_OK) return s;
    PR_CUDA(cudaMemcpy(c->m2 + c->N, &m, sizeof(int), cudaMemcpyHostToDevice));
    double* Mr = c->Mr + (size_t)c->N * c->mcap2 * c->mcap2;
    double* Lr = c->Lr + (size_t)c->N * 3 * c->mcap2 * c->mcap2;
    if (m > 0) {
        s = galerkin(c, (char*)d_R, (size_t)c->mcap2 * c->Ng, c->m2 + c->N, 1, c->mcap2, Mr, Lr);
        if (s != PR_OK) return s;
    }
    CoarseSweepArgs a = coarse_args(c);
    a.n0 = 0;
    a.count = 1;
    a.U = d_U;
    a.Up = d_Uprev;
    a.F = d_F;
    a.out = d_out;
    a.R = reinterpret_cast<const double*>(d_R);
    a.m = c->m2 + c->N;
    a.Mr = Mr;
    a.Lr = Lr;
    PR_CUDA(cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), c->st));
    PR_CUDA(launch_coarse_sweep(a, c->st));
    return pr_sync(c);
}

pr_status pr_op_apply_L_noalloc(pr_ctx* c, const double* d_in, double* d_out, int count, int transpose) {
    if (!c || !d_in || !d_out || count < 0) return fail(c, PR_ERR_INVALID_ARG, "null pointer or negative count");
    if (c->tdep) return fail(c, PR_ERR_UNSUPPORTED, "pr_op_apply_L_noalloc: time-dependent flows need a time");
    if (c->n > pr::noalloc_max_n())
        return fail(c, PR_ERR_INVALID_ARG, "pr_op_apply_L_noalloc: n above its static scratch (n <= " +
                                               std::to_string(pr::noalloc_max_n()) + ")");
    if (count > pr::noalloc_max_count())
        return fail(c, PR_ERR_INVALID_ARG, "pr_op_apply_L_noalloc: more than " +
                                               std::to_string(pr::noalloc_max_count()) +
                                               " grid functions in one call");
    if (!c->pert_host.empty() && !c->ws_ready)
        return fail(c, PR_ERR_UNSUPPORTED,
                    "pr_op_apply_L_noalloc: a stored velocity perturbation lives in the workspace "
                    "(bind it and call pr_set_initial first)");
    PR_CUDA(pr::apply_L_noalloc(c->n, c->L, c->flow, c->pert, c->eps, d_in, d_out, count, transpose != 0, c->st));
    PR_CUDA(cudaStreamSynchronize(c->st));
    return PR_OK;
}

}  // extern "C"
