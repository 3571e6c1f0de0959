// Gram matrix G = W^T W of FP64 columns on GB300's fifth-generation tensor cores
// (tcgen05.mma, BF16 operands, FP32 accumulation in tensor memory), with FP64 accuracy.
//
// Step 1 of POD_Mode (Algorithm 1) forms the Gram matrix of the snapshots; its trailing
// eigenvalues (down to 1e-13 of the largest) decide the POD dimension, so the Gram must
// be as accurate as an FP64 one (~1e-15 relative).  A BF16 or TF32 product is not.  Here
// every FP64 value is cut, error-free, into integer digits that BF16 holds exactly, and
// the tensor core multiplies digits:
//
//   column i is aligned to its largest magnitude, 2^(e_i - 2) > max_p |W[p, i]|, and each
//   value is written as  W[p, i] = 2^e_i * sum_{s=1..8} d_s(p, i) 2^(-7 s)  (+ < 2^(e_i-56))
//   with balanced digits d_s in [-64, 63] (the value truncated to 2^-53 of the column's
//   largest magnitude; the headroom bit keeps the top digit from carrying out);
//   G[i, j] = 2^(e_i + e_j) * sum_{s,t} 2^(-7 (s + t)) sum_p d_s(p, i) d_t(p, j).
//
// A digit product is an integer of at most 2^12 in magnitude, so a sum of 4096 of them
// is an integer below 2^24 and exact in the FP32 accumulator.  Products of equal weight
// (equal s + t) share an accumulator: with the two slices s, s+1 (s odd) stacked as the
// 128 rows of the MMA's A operand and slice t as its B operand, the accumulator of tile c
// collects, in its top 64 lanes, the products with s + t = c and, in its bottom 64 lanes,
// those with s + t = c + 1, from at most four (s, t) pairs each.  Every 1024 points
// (4 x 1024 x 2^12 = 2^24) the eight tiles (c = 2..9, all pairs with s + t <= 9; the
// dropped ones weigh below 2^-58 of a leading product) are read back with tcgen05.ld and
// added into FP64 accumulators with their weights, which are powers of two.  The only
// roundings are those FP64 additions and the 56-bit truncation of each value, so the
// result has the accuracy of an FP64 Gram.
//
// Work split: a persistent grid, one CTA per SM (the eight tiles fill the SM's 512 TMEM
// columns); a CTA takes work units (batch item, chunk of points) in turn and, per stage
// of 64 points, its 128 threads load the FP64 values, cut them into digits and store them
// in shared memory in the canonical K-major layout of the MMA operands (8 x 16-byte core
// matrices, no swizzle), then one thread issues the 80 MMAs of the stage and commits
// them to an mbarrier.  Every wait on the mbarrier is bounded: on time-out the kernel
// records PR_ERR_TIMEOUT, waits (bounded) for its MMAs in flight, frees its tensor memory
// and returns.  Column maxima come from a pre-pass (colmax_kernel).
#include "pr_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <stdint.h>

namespace pr {

namespace {

constexpr int TC_THREADS = 256;   // 8 warps: two cover each tensor-memory lane quarter
constexpr int TC_N = 64;             // columns handled (K <= 64)
constexpr int TC_PTS = 64;           // points per shared-memory stage
constexpr int TC_SLICES = 8;         // digits per value
constexpr int TC_TILES = 8;          // accumulator tiles c = 2..9
constexpr int TC_STAGES_PER_DRAIN = 16;   // 16 x 64 = 1024 points per accumulation
constexpr int TC_TMEM_COLS = TC_TILES * TC_N;   // 512: all of an SM's tensor memory
// operand layout: core matrix (8 rows x 8 BF16 = 128 B) of slice s, row group g (rows
// 8g..8g+7, i.e. columns of W), K group kg (points 8kg..8kg+7) at
// ((s * 8 + g) * 8 + kg) * 128 bytes; LBO (next core matrix along K) = 128 B, SBO (next
// 8-row group) = 1024 B
constexpr int TC_LBO = 128;
constexpr int TC_SBO = 1024;
constexpr int TC_STAGE_BYTES = TC_SLICES * 8 * TC_SBO;   // 64 KiB
static_assert(2 * TC_STAGE_BYTES >= TC_N * TC_N * (int)sizeof(double), "the stage buffers hold the half sums");
constexpr long long TC_SPIN_LIMIT = 1LL << 24;   // polls of an mbarrier (~1 s with the sleeps)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// UMMA shared-memory matrix descriptor (K-major, no swizzle): start address, leading
// (K) and stride (M/N) byte offsets, each >> 4; descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t umma_desc(unsigned saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(TC_LBO >> 4) << 16) |
           ((uint64_t)(TC_SBO >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and
// 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr unsigned TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TC_N >> 3) << 17) |
                              ((unsigned)(128 >> 4) << 24);

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, uint64_t adesc, uint64_t bdesc, unsigned accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accum));
}

__device__ __forceinline__ void mma_commit(unsigned mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Bounded wait for phase `parity` of the mbarrier (non-blocking test, short sleeps: about
// a second at most); false on time-out.
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
    for (long long it = 0; it < TC_SPIN_LIMIT; ++it) {
        unsigned ok = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it >= 64) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}

// Fixed-point value of x in units of 2^(e - 56) (|x| < 2^(e - 2), so |result| < 2^54),
// truncated toward zero, from the bits of x (integer operations only).
__device__ __forceinline__ long long fixed56(double x, int e) {
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0) return 0;   // zero or subnormal (below 2^-1022)
    const long long mant = (bits & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll;
    const int sh = ex - 1019 - e;   // x * 2^(56 - e) = mant * 2^sh, sh <= 1
    long long y;
    if (sh >= 0) y = mant << sh;
    else y = (sh <= -63) ? 0 : (mant >> (-sh));
    return bits < 0 ? -y : y;
}

// Balanced base-128 digits of y (|y| < 2^54): y = sum_{s=1..8} d_s 128^(8-s),
// d_s in [-64, 63].  The low 28 bits of y give the four lower digits (and a carry of 0 or
// 1 into the high part), the high part the four upper ones, all in 32-bit integers.  (The
// seven lower steps leave |y| < 2^54 / 128^7 + 1/2 < 33, so the top digit takes what is
// left without a carry.)  The kernel runs these steps for 8 values in lockstep.

// two small integers (|a|, |b| <= 64, exact in BF16) as a packed BF16 pair, a in the low half
__device__ __forceinline__ unsigned pack_bf16x2(int a, int b) {
    const __nv_bfloat162 p = __floats2bfloat162_rn((float)a, (float)b);
    return *reinterpret_cast<const unsigned*>(&p);
}

}  // namespace

// colmax[b * ld + i] = bit pattern of max_p |W_b[p, i]| (non-negative doubles order like
// their bit patterns), by atomicMax from each CTA's chunk; the buffer starts at zero.
__global__ void __launch_bounds__(256) colmax_kernel(GramArgs a, long long CH, unsigned long long* colmax,
                                                     int ld) {
    const int b = blockIdx.y;
    const int K = a.KA[b];
    const long long p_lo = (long long)blockIdx.x * CH, p_hi = min(a.Ng, p_lo + CH);
    const void* const* cols = a.colsA + (size_t)b * a.ldcols;
    __shared__ unsigned long long red[8];
    for (int i = 0; i < K; ++i) {
        const double* c = reinterpret_cast<const double*>(cols[i]);
        unsigned long long m = 0ull;
        for (long long p = p_lo + threadIdx.x; p < p_hi; p += blockDim.x) {
            const unsigned long long v = (unsigned long long)__double_as_longlong(fabs(c[p]));
            m = v > m ? v : m;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
            m = o > m ? o : m;
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0ull;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = red[w] > t ? red[w] : t;
            if (t) atomicMax(colmax + (size_t)b * ld + i, t);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) gram_tc_kernel(GramArgs a, long long CH, int chunks,
                                                                const unsigned long long* colmax, int ld,
                                                                int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_mbar[2];
    __shared__ unsigned s_tmem;
    __shared__ int s_e[TC_N];
    __shared__ int s_last;
    unsigned char* stages = smem_raw;   // two stages of TC_STAGE_BYTES, 1024-aligned
    double* sacc = reinterpret_cast<double*>(smem_raw);   // reused for the bottom-half sums
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned mbar0 = smem_u32(&s_mbar[0]);
    const unsigned stage_s = smem_u32(stages);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0 + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    unsigned parity[2] = {0u, 0u};
    bool pending[2] = {false, false};   // a commit on this stage buffer not yet waited for
    bool failed = false;
    // wait for the MMAs that read stage buffer q (all threads; one vote decides)
    auto wait_buf = [&](int q) -> bool {
        if (!pending[q]) return true;
        const bool ok = mbar_wait(mbar0 + 8u * q, parity[q]);
        parity[q] ^= 1u;
        pending[q] = false;
        return __syncthreads_or(ok ? 0 : 1) == 0;
    };
    // drain rows: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its lane = accumulator
    // row r) and the 32 columns 32 (w / 4) .. + 31; rows r < 64 hold the products with
    // s + t = c (top), rows r >= 64 those with s + t = c + 1 (bottom)
    const int row = 32 * (warp & 3) + lane;
    const int cbase = 32 * (warp >> 2);
    const bool top = row < 64;
    const int irow = top ? row : row - 64;
    // tiles c0 = 0..3 and 4..7 fold into exact 46-bit integers H, Lo (weights 2^(7(3-c0)),
    // 2^(7(7-c0))), worth H 2^(-7(5+d)) + Lo 2^(-7(9+d)) with d = 0 (top) or 1 (bottom)
    const double wH = ldexp(1.0, -7 * (5 + (top ? 0 : 1)));
    const double wL = ldexp(1.0, -7 * (9 + (top ? 0 : 1)));
    double acc[32];
    int prevK = TC_N;   // rows [K, prevK) of the stage buffers may hold another item's digits

    const int units = a.B * chunks;
    for (int u = blockIdx.x; u < units && !failed; u += gridDim.x) {
        const int b = u / chunks, chunk = u - b * chunks;
        const int K = a.KA[b];
        const long long p_lo = (long long)chunk * CH, p_hi = min(a.Ng, p_lo + CH);
        const void* const* cols = a.colsA + (size_t)b * a.ldcols;
        if (tid < TC_N) {
            const unsigned long long m = (tid < K) ? colmax[(size_t)b * ld + tid] : 0ull;
            // 2^(e - 2) > max |W[:, i]|:  e = unbiased exponent of the maximum + 3
            s_e[tid] = m ? (int)((m >> 52) & 0x7FF) - 1023 + 3 : 0;
        }
        if (K < prevK) {   // zero the digit rows of columns K .. prevK - 1 in both buffers
            const int nrow = prevK - K;
            for (int e = tid; e < 2 * TC_SLICES * nrow * 8; e += TC_THREADS) {
                const int bufq = e / (TC_SLICES * nrow * 8);
                const int r = e - bufq * TC_SLICES * nrow * 8;
                const int sl = r / (nrow * 8), rest = r - sl * nrow * 8;
                const int col = K + rest / 8, kg = rest & 7;
                *reinterpret_cast<uint4*>(stages + bufq * TC_STAGE_BYTES +
                                          ((sl * 8 + (col >> 3)) * 8 + kg) * 128 + (col & 7) * 16) =
                    make_uint4(0u, 0u, 0u, 0u);
            }
        }
        prevK = K;
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0.0;
        __syncthreads();
        int nst = 0, si = 0;   // stages since the last drain; stage counter of the unit
        for (long long p0 = p_lo; p0 < p_hi; p0 += TC_PTS, ++si) {
            const int q = si & 1;
            unsigned char* stage = stages + q * TC_STAGE_BYTES;
            // ---- this thread's items of the stage (one column and 8 consecutive points
            //      each; item it -> row rho = it & 7 of row group it >> 6, K group
            //      (it >> 3) & 7, so that 8 consecutive threads fill one 128-byte core-
            //      matrix row): all their loads are issued before anything waits
            double xr[2][8];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int it = tid + r * TC_THREADS;
                const int col = ((it >> 6) << 3) | (it & 7), kg = (it >> 3) & 7;
                const long long pb = p0 + kg * 8;
#pragma unroll
                for (int k = 0; k < 8; ++k) xr[r][k] = 0.0;
                if (col < K) {
                    const double* c = reinterpret_cast<const double*>(cols[col]);
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (pb + k < p_hi) xr[r][k] = c[pb + k];
                }
            }
            if (!wait_buf(q)) {   // the MMAs that read this buffer two stages ago
                failed = true;
                break;
            }
            // ---- digits into the stage buffer (columns >= K stay zero): the 8 points of an
            //      item are cut in lockstep, digit by digit (8 independent chains), and each
            //      slice's 16-byte core-matrix row is stored as soon as it is complete
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int it = tid + r * TC_THREADS;
                const int col = ((it >> 6) << 3) | (it & 7), kg = (it >> 3) & 7;
                if (col >= K) continue;
                const int e = s_e[col];
                int lo[8], hi[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const long long y = fixed56(xr[r][k], e);
                    lo[k] = (int)(y & 0xFFFFFFFll);
                    hi[k] = (int)(y >> 28);
                }
                unsigned char* rowp = stage + ((col >> 3) * 8 + kg) * 128 + (col & 7) * 16;
#pragma unroll
                for (int sl = TC_SLICES - 1; sl >= 0; --sl) {
                    int d[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        int& v = (sl >= TC_SLICES / 2) ? lo[k] : hi[k];
                        d[k] = ((v + 64) & 127) - 64;
                        v = (v - d[k]) >> 7;
                        if (sl == TC_SLICES / 2) hi[k] += lo[k];   // the carry out of the low half
                    }
                    *reinterpret_cast<uint4*>(rowp + sl * 8 * TC_SBO) =
                        make_uint4(pack_bf16x2(d[0], d[1]), pack_bf16x2(d[2], d[3]), pack_bf16x2(d[4], d[5]),
                                   pack_bf16x2(d[6], d[7]));
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            // ---- 4 K-steps of 16 points x 20 (s, t) pairs, committed to this buffer's mbarrier
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned sb = stage_s + q * TC_STAGE_BYTES;
                const unsigned first = (nst == 0) ? 0u : 1u;   // 0: the window's first write of a tile
#pragma unroll
                for (int k = 0; k < TC_PTS / 16; ++k) {
#pragma unroll
                    for (int sa = 0; sa < TC_SLICES; sa += 2) {   // A: slices sa, sa + 1 (0-based)
#pragma unroll
                        for (int t = 0; t < TC_TILES; ++t) {      // B: slice t; tile c0 = sa + t
                            if (sa + t >= TC_TILES) continue;
                            const int c0 = sa + t;
                            // the first pair into tile c0 in issue order is (sa = 0, t = c0) for
                            // c0 < 8; it overwrites the tile at the window's first K-step
                            const unsigned acc = (k == 0 && sa == 0) ? first : 1u;
                            mma_bf16(tmem + (unsigned)(c0 * TC_N),
                                     umma_desc(sb + (sa * 8) * TC_SBO + (2 * k) * TC_LBO),
                                     umma_desc(sb + (t * 8) * TC_SBO + (2 * k) * TC_LBO), acc);
                        }
                    }
                }
                mma_commit(mbar0 + 8u * q);
            }
            pending[q] = true;
            ++nst;
            if (nst == TC_STAGES_PER_DRAIN || p0 + TC_PTS >= p_hi) {
                // ---- drain: every MMA so far has completed once both buffers are waited for
                if (!wait_buf(q) || !wait_buf(q ^ 1)) {
                    failed = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned lane_base = tmem + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)cbase;
#pragma unroll
                for (int j0 = 0; j0 < 32; j0 += 16) {
                    long long H[16], Lo[16];
#pragma unroll
                    for (int e2 = 0; e2 < 16; ++e2) H[e2] = Lo[e2] = 0ll;
#pragma unroll
                    for (int c0 = 0; c0 < TC_TILES; ++c0) {
                        float v[16];
                        tmem_ld16(lane_base + (unsigned)(c0 * TC_N + j0), v);
#pragma unroll
                        for (int e2 = 0; e2 < 16; ++e2) {
                            const long long x = (long long)__float2int_rn(v[e2]);   // an exact integer
                            if (c0 < 4) H[e2] += x << (7 * (3 - c0));
                            else Lo[e2] += x << (7 * (7 - c0));
                        }
                    }
#pragma unroll
                    for (int e2 = 0; e2 < 16; ++e2)
                        acc[j0 + e2] = fma((double)H[e2], wH, fma((double)Lo[e2], wL, acc[j0 + e2]));
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
                nst = 0;
            }
        }
        if (failed) break;
        // ---- the unit's partial Gram: top + bottom halves, scaled by 2^(e_i + e_j)
        __syncthreads();   // every MMA of the unit completed (drained): the buffers are free
        if (!top) {
#pragma unroll
            for (int j = 0; j < 32; ++j) sacc[irow * TC_N + cbase + j] = acc[j];
        }
        __syncthreads();
        const size_t outsz = (size_t)a.maxKA * a.maxKB;
        double* mypart = a.part + ((size_t)b * chunks + chunk) * outsz;
        if (top && irow < K) {
            const int ei = s_e[irow];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int jj = cbase + j;
                if (jj >= irow && jj < K)
                    mypart[(size_t)irow * a.maxKB + jj] = ldexp(acc[j] + sacc[irow * TC_N + jj], ei + s_e[jj]);
            }
        }
        // the last unit of item b sums the chunk partials in chunk order
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned ticket = atom_add_acq_rel_u32(a.counter + b, 1u);
            s_last = (ticket == (unsigned)chunks - 1u);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            const double* bpart = a.part + (size_t)b * chunks * outsz;
            double* Gb = a.G + (size_t)b * a.ldG_b;
            for (int o = tid; o < K * K; o += TC_THREADS) {
                const int i = o / K, j = o - i * K;
                if (j < i) continue;
                double sum = 0.0;
                for (int cc = 0; cc < chunks; ++cc) sum += bpart[(size_t)cc * outsz + (size_t)i * a.maxKB + j];
                Gb[(size_t)i * a.ldG + j] = sum;
                Gb[(size_t)j * a.ldG + i] = sum;
            }
            if (tid == 0) st_relaxed_u32(a.counter + b, 0u);
        }
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) record_error(err, DERR_TIMEOUT);
        // MMAs may still be running: wait once more (bounded) on both buffers before the
        // tensor memory is released
        for (int q = 0; q < 2; ++q)
            if (pending[q]) mbar_wait(mbar0 + 8u * q, parity[q]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

int gram_tc_max_cols() { return TC_N; }

cudaError_t launch_gram_tc(const GramArgs& a, unsigned long long* colmax, int ld, int* err, cudaStream_t st) {
    if (!a.sym || a.maxKA > TC_N || a.maxKA <= 0 || !colmax || !err || ld < a.maxKA) return cudaErrorInvalidValue;
    if (a.B <= 0) return cudaSuccess;
    // the chunks of the other Gram kernels, so that the partial buffer (gram_part_doubles)
    // fits; any chunk length works for this kernel
    const int chunks = gram_chunks(a.Ng);
    const long long CH = ((a.Ng + chunks - 1) / chunks + TC_PTS - 1) / TC_PTS * TC_PTS;
    cudaError_t e = cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * (size_t)a.B * ld, st);
    if (e != cudaSuccess) return e;
    colmax_kernel<<<dim3(chunks, a.B), 256, 0, st>>>(a, CH, colmax, ld);
    ++g_launch_count;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one CTA an SM: the tiles take all 512 tensor-memory columns, and the two stage
    // buffers (128 KiB of shared memory) keep a second CTA off the SM
    const size_t smem = 2 * TC_STAGE_BYTES;
    e = cudaFuncSetAttribute((const void*)gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(sms, a.B * chunks));
    gram_tc_kernel<<<grid, TC_THREADS, smem, st>>>(a, CH, chunks, colmax, ld, err);
    ++g_launch_count;
    return cudaGetLastError();
}

}  // namespace pr
