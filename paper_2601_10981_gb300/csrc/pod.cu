// POD of snapshot matrices (Algorithm 1, POD_Mode, and the two-level POD of Case II):
//   Gram W^T M W (M = I)           -> gram_kernel     (batched, split over points)
//   eigenpairs, rank r, dimension m -> eig_pod_kernel  (cyclic Jacobi, FP64, one CTA/matrix)
//   R = W Y_m Lambda_m^{-1/2}       -> tsmm_kernel     (tall-skinny multiply)
//   Cholesky-QR re-orthonormalisation -> gram + chol_inv_kernel + tsmm, one pass
// The Gram and projection stream every snapshot once per use; the small dense steps stay
// in FP64 because their stability needs it (Gram-based POD squares the conditioning).
#include "df.cuh"
#include "pr_internal.cuh"

#include <algorithm>
#include <math.h>

namespace pr {

constexpr int GRAM_THREADS = 256;
constexpr int GRAM_SUB = 32;

int gram_chunks(long long Ng) {
    long long ch = (Ng / 128 + 31) / 32 * 32;
    ch = std::max<long long>(256, std::min<long long>(16384, ch));
    return (int)((Ng + ch - 1) / ch);
}
static long long gram_chunk_len(long long Ng) {
    const int c = gram_chunks(Ng);
    long long ch = (Ng + c - 1) / c;
    return (ch + GRAM_SUB - 1) / GRAM_SUB * GRAM_SUB;
}
size_t gram_part_doubles(long long Ng, int B, int maxKA, int maxKB) {
    return (size_t)B * gram_chunks(Ng) * (size_t)maxKA * maxKB;
}

// Output o of a batch item -> (i, j).  Non-symmetric: row-major KA x KB.  Symmetric:
// the upper triangle i <= j enumerated row by row.
__device__ __forceinline__ void out_index(int o, int KA, int KB, bool sym, int& i, int& j) {
    if (!sym) {
        i = o / KB;
        j = o - i * KB;
        return;
    }
    // rows i have KA - i entries; find i with cumulative count
    int rem = o, row = 0, len = KA;
    while (rem >= len) { rem -= len; ++row; --len; }
    i = row;
    j = row + rem;
}

// The last CTA of batch item b to finish adds the chunk partials in chunk order (a fixed
// order: the result does not depend on scheduling) and writes G (both triangles if sym).
__device__ void gram_finish(const GramArgs& a, int b, int chunks, int KA, int KB, int nout) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned ticket = atom_add_acq_rel_u32(a.counter + b, 1u);
        s_last = (ticket == (unsigned)chunks - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const size_t outsz = (size_t)a.maxKA * a.maxKB;
    const double* bpart = a.part + (size_t)b * chunks * outsz;
    double* Gb = a.G + (size_t)b * a.ldG_b;
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        int i, j;
        out_index(o, KA, KB, a.sym, i, j);
        // in chunk order (reproducible), the loads in batches of 16 independent ones (a
        // chain of dependent loads here held the item's last CTA for tens of microseconds)
        const double* src = bpart + (size_t)i * a.maxKB + j;
        double s = 0.0;
        int cc = 0;
        for (; cc + 16 <= chunks; cc += 16) {
            double v[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = src[(size_t)(cc + e) * outsz];
#pragma unroll
            for (int e = 0; e < 16; ++e) s += v[e];
        }
        for (; cc < chunks; ++cc) s += src[(size_t)cc * outsz];
        Gb[(size_t)i * a.ldG + j] = s;
        if (a.sym) Gb[(size_t)j * a.ldG + i] = s;
    }
    if (threadIdx.x == 0) st_relaxed_u32(a.counter + b, 0u);
}

template <typename TA, typename TB, typename TACC, int MAXO>
__global__ void __launch_bounds__(GRAM_THREADS) gram_kernel(GramArgs a, long long CH, int chunks) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.y, c = blockIdx.x;
    const int KA = a.KA[b];
    const int KB = a.sym ? KA : a.KB[b];
    const int nout = a.sym ? KA * (KA + 1) / 2 : KA * KB;
    const long long p_lo = (long long)c * CH;
    const long long p_hi = min(a.Ng, p_lo + CH);
    const int lda = KA + 1, ldb = KB + 1;
    TACC* sA = reinterpret_cast<TACC*>(smem_raw);
    TACC* sB = a.sym ? sA : sA + GRAM_SUB * lda;
    const void* const* colsA = a.colsA + (size_t)b * a.ldcols;
    const void* const* colsB = (a.sym ? a.colsA : a.colsB) + (size_t)b * a.ldcols;

    int oi[MAXO], oj[MAXO];
    double acc64[MAXO];
    TACC acc[MAXO];
#pragma unroll
    for (int k = 0; k < MAXO; ++k) {
        const int o = threadIdx.x + k * GRAM_THREADS;
        int i = 0, j = 0;
        if (o < nout) out_index(o, KA, KB, a.sym, i, j);
        oi[k] = (o < nout) ? i : -1;
        oj[k] = j;
        acc64[k] = 0.0;
        acc[k] = (TACC)0;
    }
    for (long long p0 = p_lo; p0 < p_hi; p0 += GRAM_SUB) {
        __syncthreads();
        for (int e = threadIdx.x; e < GRAM_SUB * KA; e += GRAM_THREADS) {
            const int col = e / GRAM_SUB, pp = e - col * GRAM_SUB;
            const long long p = p0 + pp;
            sA[pp * lda + col] = (p < p_hi) ? (TACC)(reinterpret_cast<const TA*>(colsA[col])[p]) : (TACC)0;
        }
        if (!a.sym) {
            for (int e = threadIdx.x; e < GRAM_SUB * KB; e += GRAM_THREADS) {
                const int col = e / GRAM_SUB, pp = e - col * GRAM_SUB;
                const long long p = p0 + pp;
                sB[pp * ldb + col] = (p < p_hi) ? (TACC)(reinterpret_cast<const TB*>(colsB[col])[p]) : (TACC)0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < MAXO; ++k) {
            if (oi[k] >= 0) {
                const TACC* pa = sA + oi[k];
                const TACC* pb = sB + oj[k];
                TACC s = acc[k];
#pragma unroll 8
                for (int pp = 0; pp < GRAM_SUB; ++pp) s += pa[pp * lda] * pb[pp * ldb];
                acc[k] = s;
            }
        }
        if (sizeof(TACC) == 4) {
#pragma unroll
            for (int k = 0; k < MAXO; ++k) { acc64[k] += (double)acc[k]; acc[k] = (TACC)0; }
        }
    }
    const size_t outsz = (size_t)a.maxKA * a.maxKB;
    double* mypart = a.part + ((size_t)b * chunks + c) * outsz;
#pragma unroll
    for (int k = 0; k < MAXO; ++k) {
        if (oi[k] >= 0) {
            const double v = (sizeof(TACC) == 4) ? acc64[k] : (double)acc[k];
            mypart[(size_t)oi[k] * a.maxKB + oj[k]] = v;
        }
    }
    gram_finish(a, b, chunks, KA, KB, nout);
}


// ------------------------------------------------------------------------------------
// Gram of FP64 columns in double-float arithmetic (FP32 mode).  The FP64 Gram of the
// snapshots runs at the FP64 rate (1/64 of FP32 on GB300); here each staged value is
// split into a float pair (d2df_bits) and every product-sum is an error-free df_mac2 on
// the FP32 pipe, two rows per packed instruction.  Row partials fold into a df
// accumulator every SUB rows (64 or 128), so the chunk sums keep ~1e-15 relative accuracy (the
// POD needs the Gram to ~1e-13 of its norm).
//   load      cp.async of the next block of SUB rows of every column (raw FP64)
//             while the current block is reduced
//   convert   raw -> column-major float planes hi, lo (quads of four rows XOR-swizzled by
//             column so that the 16-byte reads of neighbouring tiles hit different banks)
//   compute   one thread per 2 x 2 output tile and row group: the CTA has ntiles x P
//             threads, group g takes the row quads g, g + P, ...; the groups' FP64 sums
//             meet in shared memory at the end of the chunk.
// SUB rows per staged block: 128 for CTAs of 256 threads or more, 64 below (measured on
// the 64^3 workload: CholQR Grams 1.12 -> 0.88 and 1.48 -> 1.33 ms, Galerkin 2.53 -> 2.38,
// level-2 2.37 -> 2.25 with 128 rows; a 160-thread level-1 Gram took 6.83 ms with 64 rows
// and 7.00 with 128); a column plane holds SUB + 4 floats.
constexpr int GDF_MAXTHR = 384;
constexpr int GDF_MAXTILES = 2048;   // tiles of one item (2 x 2 each): up to 126 columns (sym)

template <int SUB>
__device__ __forceinline__ int gdf_pos(int col, int r) {
    return col * (SUB + 4) + ((((r >> 2) ^ ((col >> 3) & 1)) << 2) | (r & 3));
}
__host__ __device__ __forceinline__ int gdf_cols(int K) { return (K + 1) & ~1; }
__host__ __device__ __forceinline__ int gdf_tiles(int KA, int KB, bool sym) {
    const int nbA = (KA + 1) / 2, nbB = (KB + 1) / 2;
    return sym ? nbA * (nbA + 1) / 2 : nbA * nbB;
}
// 8-byte asynchronous global -> shared copy; src_bytes = 0 fills zeros without reading
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <int SUB>
__global__ void __launch_bounds__(GDF_MAXTHR, 2) gram_df_kernel(GramArgs a, long long CH, int chunks) {
    constexpr int GDF_SUB = SUB, GDF_LDP = SUB + 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int b = blockIdx.y, c = blockIdx.x;
    const int KA = a.KA[b];
    const int KB = a.sym ? KA : a.KB[b];
    const int nout = a.sym ? KA * (KA + 1) / 2 : KA * KB;
    const long long p_lo = (long long)c * CH;
    const long long p_hi = min(a.Ng, p_lo + CH);
    const int ncA = gdf_cols(a.maxKA), ncB = a.sym ? 0 : gdf_cols(a.maxKB);
    const int plA = ncA * GDF_LDP, plB = ncB * GDF_LDP;
    double* rawA = reinterpret_cast<double*>(smem_raw);             // [ncA][GDF_SUB]
    double* rawB = rawA + (size_t)ncA * GDF_SUB;                     // [ncB][GDF_SUB]
    float* sA = reinterpret_cast<float*>(rawB + (size_t)ncB * GDF_SUB);   // planes hi, lo
    float* sB = a.sym ? sA : sA + 2 * plA;
    const int plb = a.sym ? plA : plB;
    const void* const* colsA = a.colsA + (size_t)b * a.ldcols;
    const void* const* colsB = (a.sym ? a.colsA : a.colsB) + (size_t)b * a.ldcols;

    const int nbA = (KA + 1) / 2, nbB = (KB + 1) / 2;
    int ntiles_all = gdf_tiles(KA, KB, a.sym);
    const size_t outsz = (size_t)a.maxKA * a.maxKB;
    double* mypart = a.part + ((size_t)b * chunks + c) * outsz;
    // Blocks with orthonormal columns: a tile inside one diagonal block is the identity
    // (written here: 1 on the diagonal from chunk 0, 0 elsewhere); the remaining tiles
    // are listed in order and shared out as usual.  The list is built nthr tiles a round.
    __shared__ short s_tile[GDF_MAXTILES];
    __shared__ int s_wcnt[GDF_MAXTHR / 32 + 1];
    const bool compact = a.sym && a.colblk != nullptr;
    if (compact) {
        const int* blk = a.colblk + (size_t)b * a.ldcols;
        int base = 0;
        for (int t0 = 0; t0 < ntiles_all; t0 += nthr) {
            const int t = t0 + tid;
            bool need = false;
            if (t < ntiles_all) {
                int bi, bj;
                out_index(t, nbA, nbB, true, bi, bj);
                const int i0 = 2 * bi, j0 = 2 * bj, q = blk[i0];
                const bool same =
                    (i0 + 1 >= KA || blk[i0 + 1] == q) && blk[j0] == q && (j0 + 1 >= KA || blk[j0 + 1] == q);
                need = !same;
                if (same) {
                    for (int r = 0; r < 2; ++r)
                        for (int s2 = 0; s2 < 2; ++s2) {
                            const int i = i0 + r, j = j0 + s2;
                            if (i < KA && j < KA && i <= j)
                                mypart[(size_t)i * a.maxKB + j] = (i == j && c == 0) ? 1.0 : 0.0;
                        }
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, need);
            const int lane = tid & 31, warp = tid >> 5, nw = (nthr + 31) >> 5;
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int off = 0, tot = 0;
            for (int w = 0; w < nw; ++w) {
                const int cw = s_wcnt[w];
                off += (w < warp) ? cw : 0;
                tot += cw;
            }
            if (need) s_tile[base + off + __popc(bal & ((1u << lane) - 1u))] = (short)t;
            base += tot;
            __syncthreads();
        }
        ntiles_all = base;
    }
    // passes of at most nthr tiles (more than one only for items wider than the launch's
    // threads cover; each pass streams the chunk again)
    for (int t_base = 0; t_base < ntiles_all; t_base += nthr) {
        const int ntiles = min(nthr, ntiles_all - t_base);
        const int P = max(1, nthr / ntiles);
        const int grp = tid / ntiles;
        const bool active = grp < P;
        int ti = 0, tj = 0;
        if (active) {
            int bi, bj;
            const int t = t_base + tid - grp * ntiles;
            out_index(compact ? (int)s_tile[t] : t, nbA, nbB, a.sym, bi, bj);
            ti = 2 * bi;
            tj = 2 * bj;
        }
        f2p sh[2][2], sl[2][2], Ah[2][2], Al[2][2];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int q = 0; q < 2; ++q) sh[r][q] = sl[r][q] = Ah[r][q] = Al[r][q] = 0ull;
        auto load = [&](double* raw, int ncols, int K, const void* const* cols, long long p0) {
            for (int e = tid; e < ncols * GDF_SUB; e += nthr) {
                const int col = e / GDF_SUB, r = e - col * GDF_SUB;
                const long long p = p0 + r;
                const bool ok = col < K && p < p_hi;
                const double* src = ok ? reinterpret_cast<const double*>(cols[col]) + p : reinterpret_cast<const double*>(a.part);
                cp_async8(raw + e, src, ok ? 8 : 0);
            }
        };
        auto convert = [&](const double* raw, float* dst, int pl, int ncols) {
            for (int e = tid; e < ncols * GDF_SUB; e += nthr) {
                const int col = e / GDF_SUB, r = e - col * GDF_SUB;
                const float2 v = d2df_bits(raw[e]);
                const int o = gdf_pos<SUB>(col, r);
                dst[o] = v.x;
                dst[pl + o] = v.y;
            }
        };
        auto quad = [&](const float* pln, int col, int q) {
            return *reinterpret_cast<const ulonglong2*>(pln + col * GDF_LDP + ((q ^ ((col >> 3) & 1)) << 2));
        };
        // the item's own column counts (the buffers are laid out for the launch's largest):
        // a POD window under a cap of 48 columns that holds 12 costs 12 columns of copies and
        // conversions, not 48 (the tiles only read columns < gdf_cols(K))
        const int kA = gdf_cols(KA), kB = a.sym ? 0 : gdf_cols(KB);
        load(rawA, kA, KA, colsA, p_lo);
        if (!a.sym) load(rawB, kB, KB, colsB, p_lo);
        cp_async_commit();
        int nblk = 0;
        for (long long p0 = p_lo; p0 < p_hi; p0 += GDF_SUB) {
            cp_async_wait_all();
            __syncthreads();   // this block's rows landed; every thread is done with the planes
            convert(rawA, sA, plA, kA);
            if (!a.sym) convert(rawB, sB, plB, kB);
            __syncthreads();   // planes ready, raw buffers free
            if (p0 + GDF_SUB < p_hi) {
                load(rawA, kA, KA, colsA, p0 + GDF_SUB);
                if (!a.sym) load(rawB, kB, KB, colsB, p0 + GDF_SUB);
            }
            cp_async_commit();
            if (active) {
#pragma unroll 1
                for (int q = grp; q < GDF_SUB / 4; q += P) {
                    ulonglong2 bh[2], bl[2];
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2) {
                        bh[s2] = quad(sB, tj + s2, q);
                        bl[s2] = quad(sB + plb, tj + s2, q);
                    }
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const ulonglong2 ah = quad(sA, ti + r, q), al = quad(sA + plA, ti + r, q);
                        const f2p nx = neg2(ah.x), ny = neg2(ah.y);
#pragma unroll
                        for (int s2 = 0; s2 < 2; ++s2) {
                            df_mac2(sh[r][s2], sl[r][s2], ah.x, nx, al.x, bh[s2].x, bl[s2].x);
                            df_mac2(sh[r][s2], sl[r][s2], ah.y, ny, al.y, bh[s2].y, bl[s2].y);
                        }
                    }
                }
            }
            if (++nblk == P) {   // SUB rows a thread since the last fold
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2) {
                        df_add2(Ah[r][s2], Al[r][s2], sh[r][s2], sl[r][s2]);
                        sh[r][s2] = sl[r][s2] = 0ull;
                    }
                nblk = 0;
            }
        }
        cp_async_wait_all();   // the last (empty) group
        double acc[2][2];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                df_add2(Ah[r][s2], Al[r][s2], sh[r][s2], sl[r][s2]);
                const float2 h = upk2(Ah[r][s2]), l = upk2(Al[r][s2]);
                acc[r][s2] = df_to_double(h.x, l.x) + df_to_double(h.y, l.y);   // even + odd rows
            }
        // groups > 0 hand their sums to group 0 through shared memory
        double* sacc = reinterpret_cast<double*>(smem_raw);
        if (P > 1) {
            __syncthreads();
            if (active && grp > 0) {
                double* d = sacc + ((size_t)(grp - 1) * ntiles + (tid - grp * ntiles)) * 4;
                d[0] = acc[0][0];
                d[1] = acc[0][1];
                d[2] = acc[1][0];
                d[3] = acc[1][1];
            }
            __syncthreads();
            if (active && grp == 0) {
                for (int gg = 1; gg < P; ++gg) {
                    const double* d = sacc + ((size_t)(gg - 1) * ntiles + tid) * 4;
                    acc[0][0] += d[0];
                    acc[0][1] += d[1];
                    acc[1][0] += d[2];
                    acc[1][1] += d[3];
                }
            }
        }
        if (active && grp == 0) {
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    const int i = ti + r, j = tj + s2;
                    if (i < KA && j < KB && (!a.sym || i <= j)) mypart[(size_t)i * a.maxKB + j] = acc[r][s2];
                }
        }
        __syncthreads();   // the group sums are read: the buffers are free for the next pass
    }
    gram_finish(a, b, chunks, KA, KB, nout);
}

// Threads of gram_df_kernel: every tile of the largest batch item once, times the row
// groups that fit in 256 threads, or two groups when one would leave a single group and
// two still fit the launch bound (128 < tiles <= 192: the 33-column level-1 Gram, 6.83 ->
// 6.60 ms on the 64^3 workload); 0 when the df kernel does not apply.
static int gram_df_threads(const GramArgs& a) {
    const int tiles = gdf_tiles(a.maxKA, a.maxKB, a.sym);
    if (tiles <= 0 || tiles > GDF_MAXTILES) return 0;
    if (tiles > GDF_MAXTHR) return GDF_MAXTHR;   // wider items take several passes
    const int P = (tiles > 128 && 2 * tiles <= GDF_MAXTHR) ? 2 : std::max(1, 256 / tiles);
    return (tiles * P + 31) / 32 * 32;
}
// Shared memory of gram_df_kernel: raw blocks and float planes, at least the group sums.
static size_t gram_df_smem(const GramArgs& a, int threads, int sub) {
    const size_t cols = (size_t)gdf_cols(a.maxKA) + (a.sym ? 0 : gdf_cols(a.maxKB));
    const size_t stage = cols * sub * sizeof(double) + cols * 2 * (sub + 4) * sizeof(float);
    const size_t sums = (size_t)threads * 4 * sizeof(double);
    return std::max(stage, sums);
}
template <typename TA, typename TB, typename TACC>
static cudaError_t gram_dispatch(const GramArgs& a, cudaStream_t st) {
    const int chunks = gram_chunks(a.Ng);
    const long long CH = gram_chunk_len(a.Ng);
    const int nout = a.sym ? a.maxKA * (a.maxKA + 1) / 2 : a.maxKA * a.maxKB;
    const int need = (nout + GRAM_THREADS - 1) / GRAM_THREADS;
    const size_t smem = (size_t)GRAM_SUB * ((a.maxKA + 1) + (a.sym ? 0 : a.maxKB + 1)) * sizeof(TACC);
    dim3 grid(chunks, a.B);
    if (need <= 2)
        gram_kernel<TA, TB, TACC, 2><<<grid, GRAM_THREADS, smem, st>>>(a, CH, chunks);
    else if (need <= 4)
        gram_kernel<TA, TB, TACC, 4><<<grid, GRAM_THREADS, smem, st>>>(a, CH, chunks);
    else if (need <= 10)
        gram_kernel<TA, TB, TACC, 10><<<grid, GRAM_THREADS, smem, st>>>(a, CH, chunks);
    else if (need <= 20)
        gram_kernel<TA, TB, TACC, 20><<<grid, GRAM_THREADS, smem, st>>>(a, CH, chunks);
    else if (need <= 40)
        gram_kernel<TA, TB, TACC, 40><<<grid, GRAM_THREADS, smem, st>>>(a, CH, chunks);
    else
        return cudaErrorInvalidValue;
    ++g_launch_count;
    return cudaGetLastError();
}

cudaError_t launch_gram(const GramArgs& a, bool a_f32, bool b_f32, cudaStream_t st) {
    if (a.B <= 0 || a.maxKA <= 0 || (!a.sym && a.maxKB <= 0)) return cudaSuccess;
    if (a.df && !a_f32 && !b_f32) {
        const int thr = gram_df_threads(a);
        int sub = thr >= 256 ? 128 : 64;
        size_t smem = thr > 0 ? gram_df_smem(a, thr, sub) : 0;
        if (smem > 160 * 1024 && sub == 128) {
            sub = 64;
            smem = gram_df_smem(a, thr, sub);
        }
        if (thr > 0 && smem <= 160 * 1024) {
            const int chunks = gram_chunks(a.Ng);
            const long long CH = gram_chunk_len(a.Ng);
            const void* fn = sub == 128 ? (const void*)gram_df_kernel<128> : (const void*)gram_df_kernel<64>;
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (sub == 128)
                gram_df_kernel<128><<<dim3(chunks, a.B), thr, smem, st>>>(a, CH, chunks);
            else
                gram_df_kernel<64><<<dim3(chunks, a.B), thr, smem, st>>>(a, CH, chunks);
            ++g_launch_count;
            return cudaGetLastError();
        }
    }
    // FP32 accumulation only when both operands are FP32.
    if (a_f32 && (b_f32 || a.sym)) return gram_dispatch<float, float, float>(a, st);
    if (a_f32) return gram_dispatch<float, double, double>(a, st);
    if (b_f32) return gram_dispatch<double, float, double>(a, st);
    return gram_dispatch<double, double, double>(a, st);
}

// ------------------------------------------------------------------------------------
// Out_b = In_b C_b.  One thread per point; a block of J outputs (J a multiple of 4, the
// smallest that covers the remaining columns) is accumulated with compile-time trip
// counts, so no predicated-off multiply-adds are issued.  C sits in shared memory with
// rows padded to a multiple of 4 by zeros.
template <typename TI, typename TO, typename TC, int J>
__device__ __forceinline__ void tsmm_block(const void* const* cols, int KIN, const TC* sC, int KP,
                                           int j0, int jn, long long p, long long Ng, TO* out) {
    TC acc[J];
#pragma unroll
    for (int jj = 0; jj < J; ++jj) acc[jj] = (TC)0;
    for (int i = 0; i < KIN; ++i) {
        const TC x = (TC)(reinterpret_cast<const TI*>(cols[i])[p]);
        const TC* crow = sC + (size_t)i * KP + j0;
#pragma unroll
        for (int jj = 0; jj < J; ++jj) acc[jj] += x * crow[jj];
    }
#pragma unroll
    for (int jj = 0; jj < J; ++jj)
        if (jj < jn) out[(size_t)(j0 + jj) * Ng + p] = (TO)acc[jj];
}

template <typename TI, typename TO, typename TC>
__global__ void __launch_bounds__(256) tsmm_kernel(TsmmArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC* sC = reinterpret_cast<TC*>(smem_raw);
    const int b = blockIdx.y;
    const int KIN = a.KIN[b], KOUT = a.KOUT[b];
    if (KOUT <= 0) return;
    const int KP = (KOUT + 3) / 4 * 4;
    const double* Cb = a.C + (size_t)b * a.ldC_b;
    for (int e = threadIdx.x; e < KIN * KP; e += blockDim.x) {
        const int i = e / KP, j = e - i * KP;
        sC[e] = (j < KOUT) ? (TC)Cb[(size_t)i * a.ldC + j] : (TC)0;
    }
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.Ng) return;
    const void* const* cols = a.colsIn + (size_t)b * a.ldcols;
    TO* out = reinterpret_cast<TO*>(a.out) + (size_t)b * a.ld_out_b;
    for (int j0 = 0; j0 < KOUT; j0 += 32) {
        const int jn = min(32, KOUT - j0);
        switch ((jn + 3) / 4) {
        case 1: tsmm_block<TI, TO, TC, 4>(cols, KIN, sC, KP, j0, jn, p, a.Ng, out); break;
        case 2: tsmm_block<TI, TO, TC, 8>(cols, KIN, sC, KP, j0, jn, p, a.Ng, out); break;
        case 3: tsmm_block<TI, TO, TC, 12>(cols, KIN, sC, KP, j0, jn, p, a.Ng, out); break;
        case 4: tsmm_block<TI, TO, TC, 16>(cols, KIN, sC, KP, j0, jn, p, a.Ng, out); break;
        case 5: tsmm_block<TI, TO, TC, 20>(cols, KIN, sC, KP, j0, jn, p, a.Ng, out); break;
        case 6: tsmm_block<TI, TO, TC, 24>(cols, KIN, sC, KP, j0, jn, p, a.Ng, out); break;
        case 7: tsmm_block<TI, TO, TC, 28>(cols, KIN, sC, KP, j0, jn, p, a.Ng, out); break;
        default: tsmm_block<TI, TO, TC, 32>(cols, KIN, sC, KP, j0, jn, p, a.Ng, out); break;
        }
    }
}

// Out_b = In_b C_b with FP64 input and output in double-float arithmetic (FP32 mode):
// one thread per point, blocks of J <= 16 outputs.  C sits in shared memory as float-pair
// planes hi, lo (rows padded to a multiple of 4, read as warp-wide broadcasts); each input
// is split once per block (d2df_bits) and broadcast into both lanes of a packed pair, so
// one df_mac2 serves two outputs.  The inputs travel by cp.async in groups of TSMM_TG into
// the thread's own shared-memory slots, one group ahead (no registers held, no barrier:
// each thread reads back only its own copies).
constexpr int TSMM_TG = 8;
template <int J>
__device__ __forceinline__ void tsmm_df_block(const void* const* cols, int KIN, const float* sC, int pl, int KP,
                                              int j0, int jn, long long p, long long Ng, double* out,
                                              double* stg, int nthr) {
    constexpr int H = J / 2;
    f2p sh[H], sl[H];
#pragma unroll
    for (int h = 0; h < H; ++h) sh[h] = sl[h] = 0ull;
    // stg: this thread's slots, [slot][k][thread] (thread-contiguous: no bank conflicts)
    auto slot_of = [&](int sl2, int k) { return stg + (size_t)(sl2 * TSMM_TG + k) * nthr; };
    auto issue = [&](int g, int sl2) {
#pragma unroll
        for (int k = 0; k < TSMM_TG; ++k) {
            const int i = g * TSMM_TG + k;
            if (i < KIN) cp_async8(slot_of(sl2, k), reinterpret_cast<const double*>(cols[i]) + p, 8);
        }
        cp_async_commit();
    };
    const int ng = (KIN + TSMM_TG - 1) / TSMM_TG;
    issue(0, 0);
    for (int g = 0; g < ng; ++g) {
        issue(g + 1, (g + 1) & 1);   // the slot of group g - 1, read in the previous pass
        cp_async_wait1();            // group g landed
#pragma unroll 2
        for (int k = 0; k < TSMM_TG; ++k) {
            const int i = g * TSMM_TG + k;
            if (i >= KIN) break;
            const float2 x = d2df_bits(*slot_of(g & 1, k));
            const f2p xh = pk2(x.x, x.x), nxh = pk2(-x.x, -x.x), xl = pk2(x.y, x.y);
            const float* row = sC + (size_t)i * KP + j0;
#pragma unroll
            for (int h4 = 0; h4 < J / 4; ++h4) {
                const ulonglong2 ch = *reinterpret_cast<const ulonglong2*>(row + 4 * h4);
                const ulonglong2 cl = *reinterpret_cast<const ulonglong2*>(row + pl + 4 * h4);
                df_mac2(sh[2 * h4], sl[2 * h4], xh, nxh, xl, ch.x, cl.x);
                df_mac2(sh[2 * h4 + 1], sl[2 * h4 + 1], xh, nxh, xl, ch.y, cl.y);
            }
        }
    }
    cp_async_wait_all();
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const float2 vh = upk2(sh[h]), vl = upk2(sl[h]);
        if (2 * h < jn) out[(size_t)(j0 + 2 * h) * Ng + p] = df_to_double(vh.x, vl.x);
        if (2 * h + 1 < jn) out[(size_t)(j0 + 2 * h + 1) * Ng + p] = df_to_double(vh.y, vl.y);
    }
}

__global__ void __launch_bounds__(256) tsmm_df_kernel(TsmmArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sC = reinterpret_cast<float*>(smem_raw);
    const int b = blockIdx.y;
    const int KIN = a.KIN[b], KOUT = a.KOUT[b];
    if (KOUT <= 0) return;
    const int KP = (KOUT + 3) / 4 * 4;
    const int pl = a.maxKIN * ((a.maxKOUT + 3) / 4 * 4);   // floats per plane
    const double* Cb = a.C + (size_t)b * a.ldC_b;
    for (int e = threadIdx.x; e < KIN * KP; e += blockDim.x) {
        const int i = e / KP, j = e - i * KP;
        const float2 v = (j < KOUT) ? d2df_bits(Cb[(size_t)i * a.ldC + j]) : make_float2(0.0f, 0.0f);
        sC[e] = v.x;
        sC[pl + e] = v.y;
    }
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.Ng) return;
    const void* const* cols = a.colsIn + (size_t)b * a.ldcols;
    double* out = reinterpret_cast<double*>(a.out) + (size_t)b * a.ld_out_b;
    // per-thread input slots after the C planes (16-byte aligned)
    double* stg = reinterpret_cast<double*>(smem_raw + ((size_t)2 * pl * sizeof(float) + 15) / 16 * 16) + threadIdx.x;
    const int nthr = blockDim.x;
    for (int j0 = 0; j0 < KOUT; j0 += 16) {
        const int jn = min(16, KOUT - j0);
        switch ((jn + 3) / 4) {
        case 1: tsmm_df_block<4>(cols, KIN, sC, pl, KP, j0, jn, p, a.Ng, out, stg, nthr); break;
        case 2: tsmm_df_block<8>(cols, KIN, sC, pl, KP, j0, jn, p, a.Ng, out, stg, nthr); break;
        case 3: tsmm_df_block<12>(cols, KIN, sC, pl, KP, j0, jn, p, a.Ng, out, stg, nthr); break;
        default: tsmm_df_block<16>(cols, KIN, sC, pl, KP, j0, jn, p, a.Ng, out, stg, nthr); break;
        }
    }
}

cudaError_t launch_tsmm(const TsmmArgs& a, bool in_f32, bool out_f32, cudaStream_t st) {
    if (a.B <= 0 || a.maxKOUT <= 0) return cudaSuccess;
    dim3 grid((unsigned)((a.Ng + 255) / 256), a.B);
    const size_t cells = (size_t)a.maxKIN * ((a.maxKOUT + 3) / 4 * 4);
    if (a.df && !in_f32 && !out_f32) {
        const size_t smem = (2 * cells * sizeof(float) + 15) / 16 * 16 + (size_t)2 * TSMM_TG * 256 * sizeof(double);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute((const void*)tsmm_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        tsmm_df_kernel<<<grid, 256, smem, st>>>(a);
    } else if (in_f32 && out_f32) {
        tsmm_kernel<float, float, float><<<grid, 256, cells * sizeof(float), st>>>(a);
    } else if (!in_f32 && out_f32) {
        // FP64 input (snapshots): accumulate in FP64 and round only the output, the
        // combinations of nearly parallel snapshots that give trailing modes cancel
        tsmm_kernel<double, float, double><<<grid, 256, cells * sizeof(double), st>>>(a);
    } else if (in_f32) {
        tsmm_kernel<float, double, double><<<grid, 256, cells * sizeof(double), st>>>(a);
    } else {
        tsmm_kernel<double, double, double><<<grid, 256, cells * sizeof(double), st>>>(a);
    }
    ++g_launch_count;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Batched symmetric eigensolver (parallel cyclic Jacobi, round-robin pairing) + POD
// selection of Algorithm 1.
constexpr int EIG_THREADS = 256;
constexpr int EIG_MAX_SWEEPS = 40;

__device__ __forceinline__ void rr_pair(int r, int i, int Kp, int& p, int& q) {
    const int M = Kp - 1;
    if (i == 0) {
        p = M;
        q = r;
    } else {
        p = (r + i) % M;
        q = (r - i + M) % M;
    }
}

__global__ void __launch_bounds__(EIG_THREADS) eig_pod_kernel(EigArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.x;
    const int K = a.K[b];
    double* lam_out = a.lam + (size_t)b * a.maxK;
    double* Cb = a.C + (size_t)b * a.ldC_b;
    if (K <= 0) {
        if (threadIdx.x == 0) a.m[b] = 0;
        return;
    }
    const int Kp = K + (K & 1);
    const int ld = Kp + 1;   // odd stride in doubles: row and column sweeps hit distinct banks
    double* A = reinterpret_cast<double*>(smem_raw);
    double* V = A + (size_t)Kp * ld;
    double* cs = V + (size_t)Kp * ld;           // [Kp/2][2]
    double* lam = cs + Kp;                       // [Kp]
    int* perm = reinterpret_cast<int*>(lam + Kp);  // [Kp]
    int* pq = perm + Kp;                         // [Kp/2][2]: the round's pairs
    __shared__ double red[32];
    __shared__ int s_stop;
    __shared__ double s_prev;   // ||off||_F^2 before the previous sweep
    const double* Gb = a.G + (size_t)b * a.ldG_b;
    for (int e = threadIdx.x; e < Kp * Kp; e += blockDim.x) {
        const int i = e / Kp, j = e - i * Kp;
        A[i * ld + j] = (i < K && j < K) ? Gb[(size_t)i * a.ldG + j] : 0.0;
        V[i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int npair = Kp / 2;
    // fixed thread -> (pair, first row) map of the rotation updates: no divisions per element
    const int ti = threadIdx.x % npair, kst = blockDim.x / npair;
    const int tk0 = threadIdx.x / npair;
    for (int sweep = 0; sweep < EIG_MAX_SWEEPS; ++sweep) {
        // convergence: off-diagonal Frobenius norm against the whole matrix
        double off = 0.0, tot = 0.0;
        for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
            const int i = e / K, j = e - i * K;
            const double v = A[i * ld + j];
            tot += v * v;
            if (i != j) off += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_down_sync(0xffffffffu, off, o);
            tot += __shfl_down_sync(0xffffffffu, tot, o);
        }
        if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = off; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double so = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) so += red[w];
            red[31] = so;
        }
        __syncthreads();
        const double offsum = red[31];
        __syncthreads();
        if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = tot; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double st = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) st += red[w];
            // converged when the off-diagonal part is at the rounding level of the Gram
            // matrix itself, ||off||_F <= K eps ||A||_F: a tighter bound sits below the
            // noise of the rotations (fused multiply-adds) and would never be met.  The
            // rotations' own noise can also sit just above that bound, so a sweep that no
            // longer cuts ||off|| four-fold within 16 times of it ends the iteration too
            // (past the quadratic phase further sweeps only reshuffle rounding noise)
            const double tolK = (double)K * 2.220446049250313e-16;
            const bool stalled = sweep > 0 && offsum <= 256.0 * tolK * tolK * st && offsum * 16.0 >= s_prev;
            s_stop = (offsum <= tolK * tolK * st) || st == 0.0 || stalled;
            s_prev = offsum;
        }
        __syncthreads();
        if (s_stop) break;
        for (int r = 0; r < Kp - 1; ++r) {
            for (int i = threadIdx.x; i < npair; i += blockDim.x) {
                int p, q;
                rr_pair(r, i, Kp, p, q);
                double c = 1.0, s = 0.0;
                if (p < K && q < K) {
                    const double apq = A[p * ld + q];
                    const double app = A[p * ld + p], aqq = A[q * ld + q];
                    if (apq != 0.0 && fabs(apq) > 1e-300) {
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = tt * c;
                    }
                }
                cs[2 * i] = c;
                cs[2 * i + 1] = s;
                pq[2 * i] = p;
                pq[2 * i + 1] = q;
            }
            __syncthreads();
            const bool upd = tk0 < kst && cs[2 * ti + 1] != 0.0;
            const double c = cs[2 * ti], s = cs[2 * ti + 1];
            const int p = pq[2 * ti], q = pq[2 * ti + 1];
            if (upd) {
                // A <- A J, V <- V J (columns p, q)
                for (int k = tk0; k < Kp; k += kst) {
                    const double akp = A[k * ld + p], akq = A[k * ld + q];
                    A[k * ld + p] = c * akp - s * akq;
                    A[k * ld + q] = s * akp + c * akq;
                    const double vkp = V[k * ld + p], vkq = V[k * ld + q];
                    V[k * ld + p] = c * vkp - s * vkq;
                    V[k * ld + q] = s * vkp + c * vkq;
                }
            }
            __syncthreads();
            if (upd) {
                // A <- J^T A (rows p, q)
                for (int k = tk0; k < Kp; k += kst) {
                    const double apk = A[p * ld + k], aqk = A[q * ld + k];
                    A[p * ld + k] = c * apk - s * aqk;
                    A[q * ld + k] = s * apk + c * aqk;
                }
            }
            __syncthreads();
        }
    }
    // eigenvalues, descending order (ties by index)
    for (int i = threadIdx.x; i < K; i += blockDim.x) lam[i] = A[i * ld + i];
    __syncthreads();
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        int rank = 0;
        const double li = lam[i];
        for (int j = 0; j < K; ++j) {
            const double lj = lam[j];
            rank += (lj > li) || (lj == li && j < i);
        }
        perm[rank] = i;
    }
    __syncthreads();
    __shared__ int s_m;
    if (threadIdx.x == 0) {
        const double l1 = lam[perm[0]];
        int m = 0;
        if (l1 > 0.0) {
            int r = 0;
            for (int i = 0; i < K; ++i) r += lam[perm[i]] > a.tau * l1;
            double total = 0.0;
            for (int i = 0; i < r; ++i) total += sqrt(lam[perm[i]]);
            double cum = 0.0;
            m = r;
            for (int i = 0; i < r; ++i) {
                cum += sqrt(lam[perm[i]]);
                if (cum >= a.gamma * total) { m = i + 1; break; }
            }
            if (a.cap > 0) m = min(m, a.cap);
            m = min(m, r);
        }
        s_m = m;
        a.m[b] = m;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.maxK; i += blockDim.x) lam_out[i] = (i < K) ? lam[perm[i]] : 0.0;
    const int m = s_m;
    for (int e = threadIdx.x; e < K * m; e += blockDim.x) {
        const int i = e / m, j = e - i * m;
        const int src = perm[j];
        Cb[(size_t)i * a.ldC + j] = V[i * ld + src] / sqrt(lam[src]);
    }
}

cudaError_t launch_eig_pod(const EigArgs& a, cudaStream_t st) {
    if (a.B <= 0) return cudaSuccess;
    const int Kp = a.maxK + (a.maxK & 1);
    const size_t smem = (size_t)2 * Kp * (Kp + 1) * sizeof(double) + (size_t)2 * Kp * sizeof(double) +
                        (size_t)2 * Kp * sizeof(int) + 16;
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaFuncSetAttribute(eig_pod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = smem;
    }
    eig_pod_kernel<<<a.B, EIG_THREADS, smem, st>>>(a);
    ++g_launch_count;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Cholesky G = L L^T (FP64) and X = L^{-T}, one CTA per matrix.
__global__ void chol_inv_kernel(const double* G, int ldG, long long ldG_b, const int* mp, int maxm,
                                double* X, int ldX, long long ldX_b, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.x;
    const int m = mp[b];
    if (m <= 0) return;
    double* L = reinterpret_cast<double*>(smem_raw);   // [maxm][maxm]
    double* Li = L + (size_t)maxm * maxm;                // [maxm][maxm]
    __shared__ int s_bad;
    const double* Gb = G + (size_t)b * ldG_b;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e - i * m;
        L[i * maxm + j] = (j <= i) ? Gb[(size_t)i * ldG + j] : 0.0;
    }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (threadIdx.x == 0) {
            double d = L[j * maxm + j];
            for (int k = 0; k < j; ++k) d -= L[j * maxm + k] * L[j * maxm + k];
            if (!(d > 0.0)) { s_bad = 1; d = 1.0; }
            L[j * maxm + j] = sqrt(d);
        }
        __syncthreads();
        const double ljj = L[j * maxm + j];
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
            double s = L[i * maxm + j];
            for (int k = 0; k < j; ++k) s -= L[i * maxm + k] * L[j * maxm + k];
            L[i * maxm + j] = s / ljj;
        }
        __syncthreads();
    }
    // columns of L^{-1} by forward substitution
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        for (int i = 0; i < m; ++i) {
            if (i < c) { Li[i * maxm + c] = 0.0; continue; }
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) s -= L[i * maxm + k] * Li[k * maxm + c];
            Li[i * maxm + c] = s / L[i * maxm + i];
        }
    }
    __syncthreads();
    double* Xb = X + (size_t)b * ldX_b;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e - i * m;
        Xb[(size_t)i * ldX + j] = s_bad ? (i == j ? 1.0 : 0.0) : Li[j * maxm + i];
    }
    if (threadIdx.x == 0 && s_bad) record_error(err, DERR_BREAKDOWN);
}

cudaError_t launch_chol_inv(const double* G, int ldG, long long ldG_b, const int* m, int maxm,
                            int B, double* X, int ldX, long long ldX_b, int* err,
                            cudaStream_t st) {
    if (B <= 0 || maxm <= 0) return cudaSuccess;
    const size_t smem = (size_t)2 * maxm * maxm * sizeof(double);
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = smem;
    }
    chol_inv_kernel<<<B, 128, smem, st>>>(G, ldG, ldG_b, m, maxm, X, ldX, ldX_b, err);
    ++g_launch_count;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// M_b = I_{m[b]} (the Galerkin mass matrix V^T V of an orthonormal basis, M = I).
__global__ void identity_kernel(double* M, int ld, long long ld_b, const int* m) {
    const int b = blockIdx.x, mb = m[b];
    double* Mb = M + (size_t)b * ld_b;
    for (int e = threadIdx.x; e < mb * mb; e += blockDim.x) {
        const int i = e / mb, j = e - i * mb;
        Mb[(size_t)i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
}

cudaError_t launch_identity(double* M, int ld, long long ld_b, const int* m, int B, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    identity_kernel<<<B, 256, 0, st>>>(M, ld, ld_b, m);
    ++g_launch_count;
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
__global__ void assemble_cols_kernel(const void* const* bases, const int* const* cnt_ptrs, int nb,
                                     long long Ng, int esize, const void** cols, int ld, int* K,
                                     int* blk) {
    const int b = blockIdx.x;
    if (threadIdx.x != 0) return;
    int k = 0;
    for (int j = 0; j < nb; ++j) {
        const char* base = reinterpret_cast<const char*>(bases[(size_t)b * nb + j]);
        const int* cp = cnt_ptrs[(size_t)b * nb + j];
        const int c = (base && cp) ? *cp : 0;
        for (int i = 0; i < c && k < ld; ++i) {
            if (blk) blk[(size_t)b * ld + k] = j;
            cols[(size_t)b * ld + k++] = base + (size_t)i * Ng * esize;
        }
    }
    K[b] = k;
}

cudaError_t launch_assemble_cols(const void* const* bases, const int* const* cnt_ptrs, int nb, int B,
                                 long long Ng, int esize, const void** cols, int ld, int* K, int* blk,
                                 cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    assemble_cols_kernel<<<B, 32, 0, st>>>(bases, cnt_ptrs, nb, Ng, esize, cols, ld, K, blk);
    ++g_launch_count;
    return cudaGetLastError();
}

} // namespace pr
