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
// Two forms share the digit scheme: the wide one described here (up to 64 columns,
// gram_tc_kernel) and a narrow, warp-specialised one for up to 32 columns
// (gram_tc32_kernel, described at its definition), which sums exactly and rounds once.
//
// Wide form.  Work split: a persistent grid, one CTA per SM (the eight tiles fill the SM's 512 TMEM
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
// a second at most with the default limit); false on time-out.
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity, long long limit = TC_SPIN_LIMIT) {
    for (long long it = 0; it <= limit; ++it) {
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

__device__ __forceinline__ void tmem_ld8(unsigned taddr, float (&v)[8]) {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[e]);
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
// Eight columns at a time, two points a load where the columns are 16-byte aligned (eight
// independent 16-byte loads in flight per thread), per-warp maxima in shared memory, one
// barrier and one atomic per column and CTA.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long x, unsigned long long y) {
    return x > y ? x : y;
}
__global__ void __launch_bounds__(256) colmax_kernel(GramArgs a, long long CH, unsigned long long* colmax,
                                                     int ld) {
    const int b = blockIdx.y;
    const int K = a.KA[b];
    const long long p_lo = (long long)blockIdx.x * CH, p_hi = min(a.Ng, p_lo + CH);
    const void* const* cols = a.colsA + (size_t)b * a.ldcols;
    __shared__ unsigned long long red[8][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i0 = 0; i0 < K; i0 += 8) {
        const double* c[8];
        unsigned long long m[8];
        bool al = (p_lo & 1) == 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {   // columns past K read column i0 again (never stored)
            c[j] = reinterpret_cast<const double*>(cols[i0 + j < K ? i0 + j : i0]);
            m[j] = 0ull;
            al = al && ((reinterpret_cast<uintptr_t>(c[j]) & 15u) == 0);
        }
        long long p = p_lo + (al ? 2 * (long long)threadIdx.x : (long long)threadIdx.x);
        if (al) {
            for (; p + 1 < p_hi; p += 2 * (long long)blockDim.x) {
                double2 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = *reinterpret_cast<const double2*>(c[j] + p);
#pragma unroll
                for (int j = 0; j < 8; ++j) m[j] = umax64(m[j], umax64(abs_bits(v[j].x), abs_bits(v[j].y)));
            }
        }
        // the remaining single points (an odd tail, or every point of unaligned columns)
        for (; p < p_hi; p += (al ? 2 * (long long)blockDim.x : (long long)blockDim.x)) {
#pragma unroll
            for (int j = 0; j < 8; ++j) m[j] = umax64(m[j], abs_bits(c[j][p]));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) m[j] = umax64(m[j], __shfl_xor_sync(0xffffffffu, m[j], off));
            if (lane == 0 && i0 + j < K) red[warp][i0 + j] = m[j];
        }
    }
    __syncthreads();
    if (threadIdx.x < K) {
        unsigned long long t = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = umax64(t, red[w][threadIdx.x]);
        if (t) atomicMax(colmax + (size_t)b * ld + threadIdx.x, t);
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) gram_tc_kernel(GramArgs a, long long CH, int chunks,
                                                                const unsigned long long* colmax, int ld,
                                                                int* err, long long limit) {
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
        const bool ok = mbar_wait(mbar0 + 8u * q, parity[q], limit);
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
                // chunk order (reproducible), loads in batches of 16 independent ones
                const double* src = bpart + (size_t)i * a.maxKB + j;
                double sum = 0.0;
                int cc = 0;
                for (; cc + 16 <= chunks; cc += 16) {
                    double v[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] = src[(size_t)(cc + e) * outsz];
#pragma unroll
                    for (int e = 0; e < 16; ++e) sum += v[e];
                }
                for (; cc < chunks; ++cc) sum += src[(size_t)cc * outsz];
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

namespace {

// ---------------------------------------------------------------------------------------
// Narrow form, K <= 32 columns: one M = 128 x N = 256 x K = 16 MMA per 16 points.
//
// The digit rows of a stage are slice s (0 = most significant) x 32 columns, 256 rows in
// all.  A is rows 0..127 (slices 0..3), B all 256 rows (slices 0..7), so one MMA forms
// every product D_s^T D_t with s <= 3: accumulator lane 32 s + i, column 32 t + j holds
// P_st[i, j] = sum_p d_s(p, i) d_t(p, j).  The Gram needs the pairs with min(s, t) <= 3
// (the pairs with both s, t >= 4 weigh below 2^-58 of 2^(e_i + e_j); the wide form above
// drops more); those with s >= 4 are transposes of computed ones, P_st = P_ts^T, so
//   G = sum_{s<=3, t} w_st P_st + (sum_{s<=3, t>=4} w_st P_st)^T,  w_st = 2^(-7 (s+t+2)).
// Each accumulator position takes one digit product a point, so a window of 4096 points
// stays below 2^24 (exact in FP32); the tensor memory holds two windows (2 x 256 columns)
// and the MMAs of one run while the other is read back.
//
// Warp roles: warps 0-7 load the FP64 values (one stage ahead, in registers), cut them
// into digits, store them into a ring of four shared-memory stages, and read back the
// accumulators of finished windows; warp 8 issues the MMAs (one thread) and owns the
// tensor memory.  They meet only at mbarriers (stage full / stage free / window done /
// window read), every wait bounded.  Read-back is integer: each (s, i, j) folds its eight
// tiles into two exact 64-bit integers H (t <= 3) and L (t >= 4), kept in shared memory
// over the windows of a work unit; at the unit's end the 12 terms of each output are
// summed exactly in 128-bit integers and stored as the unit's partial; the last unit of
// an item adds the partials (exact) and rounds once to FP64.  The result is the exactly
// rounded value of the digit sum: reproducible bit for bit, whatever the chunking.
constexpr int N2_PROD = 256;                     // producer threads (warps 0-7)
constexpr int N2_THREADS = N2_PROD + 32;         // + the MMA warp
constexpr int N2_COLS = 32;
constexpr int N2_PTS = 64;                       // points per stage
constexpr int N2_NS = 3;                         // stages in the digit ring
constexpr int N2_DEPTH = 3;                      // stages of FP64 values in flight (cp.async)
constexpr int N2_STG_BYTES = N2_PTS * N2_COLS * 8;   // 16 KiB of FP64 values a stage
constexpr int N2_STAGE_BYTES = TC_SLICES * N2_COLS * N2_PTS * 2;   // 32 KiB
constexpr int N2_WIN = 4096;                     // points per accumulation window (2^12)
constexpr int N2_TMEM_COLS = 512;                // two windows of 256 FP32 columns
constexpr int N2_XP = 33;                        // 64-bit row pitch of the exchange arrays
constexpr int N2_XWORDS = 4 * 32 * N2_XP;        // per array (H or L)
constexpr int N2_SMEM = N2_NS * N2_STAGE_BYTES + (N2_DEPTH + 1) * N2_STG_BYTES + 2 * N2_XWORDS * 8;
static_assert(N2_SMEM + 256 <= 227 * 1024, "shared memory of the narrow form");
constexpr unsigned N2_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(256 >> 3) << 17) |
                              ((unsigned)(128 >> 4) << 24);
// B = sum_{k=0..7} 64 * 128^k: z = y + B has the unsigned base-128 digits u_k = d_k + 64
constexpr unsigned long long N2_BIAS = 0x0081020408102040ull;

__device__ __forceinline__ unsigned long long shr64_clamp(unsigned long long x, unsigned r) {
    unsigned long long y;
    asm("shr.b64 %0, %1, %2;" : "=l"(y) : "l"(x), "r"(r));   // r >= 64 gives 0
    return y;
}

// Digit field bp of z (bits bp .. bp + 6 of the 56-bit z = zh:zl) for two points, packed
// as a BF16 pair of the digits u - 64: the halves hold 128 + u (bits 0x4300 | u), and one
// packed BF16 subtraction of 192 leaves u - 64 exactly.
template <int BP>
__device__ __forceinline__ unsigned digit_pair(unsigned zla, unsigned zha, unsigned zlb, unsigned zhb) {
    unsigned fa, fb16;
    if constexpr (BP + 7 <= 32) {
        fa = zla >> BP;
        fb16 = (BP <= 16) ? (zlb << (16 - BP)) : (zlb >> (BP - 16));
    } else if constexpr (BP >= 32) {
        fa = zha >> (BP - 32);
        fb16 = (BP - 32 <= 16) ? (zhb << (16 - (BP - 32))) : (zhb >> (BP - 32 - 16));
    } else {
        fa = __funnelshift_r(zla, zha, BP);
        fb16 = __funnelshift_r(zlb, zhb, BP) << 16;
    }
    const unsigned w = (fa & 0x7Fu) | (fb16 & 0x7F0000u) | 0x43004300u;
    __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&w);
    const unsigned c192 = 0x43404340u;
    v = __hsub2(v, *reinterpret_cast<const __nv_bfloat162*>(&c192));
    return *reinterpret_cast<const unsigned*>(&v);
}

// z = 2^(56 - e) x truncated toward zero, plus the bias, as two 32-bit words; ce = e + 1020.
// Zero and subnormal x take the effective exponent 1 (no implicit bit).
__device__ __forceinline__ void cut56(double x, int ce, unsigned& zl, unsigned& zh) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
    const unsigned exf = hi & 0x7FF00000u;
    const unsigned imp = min(exf, 0x100000u);
    const int exe = (int)(max(exf, 0x100000u) >> 20);
    const unsigned long long m = ((unsigned long long)((hi & 0xFFFFFu) | imp) << 32) | lo;
    const unsigned long long y = shr64_clamp(m << 1, (unsigned)(ce - exe));   // ce >= exe
    const unsigned long long sg = (unsigned long long)(long long)((int)hi >> 31);
    const unsigned long long z = (N2_BIAS - sg) + (y ^ sg);
    zl = (unsigned)z;
    zh = (unsigned)(z >> 32);
}

// Bounded mbarrier wait that also gives up once another thread has recorded a failure.
// try_wait suspends the thread (at most ~1 us a try, by its time hint) instead of
// spinning, so waiting warps leave the issue slots to the others; `limit` tries (the
// context's spin limit, 2^22 ~ a few seconds by default).  limit 0: one non-blocking
// test, so that a wait not already complete gives up at once.
__device__ __forceinline__ bool mbar_wait_f(unsigned mbar, unsigned parity, volatile int* fail, long long limit) {
    if (limit == 0) {
        if (mbar_wait(mbar, parity, 0)) return true;
        *fail = 1;
        return false;
    }
    for (long long it = 0; it <= limit; ++it) {
        unsigned ok = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 15) == 15 && *fail) return false;
    }
    *fail = 1;
    return false;
}
__device__ __forceinline__ void mbar_arrive(unsigned mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void prod_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ void mma_n256(unsigned tmem_d, uint64_t desc, unsigned accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %1, %2, p;\n\t}\n" ::"r"(tmem_d),
        "l"(desc), "r"(N2_IDESC), "r"(accum));
}

// the exponent e of a column (2^(e - 2) > max |W[:, i]|) from its column-maximum bits
__device__ __forceinline__ int col_exp(unsigned long long m) {
    return m ? (int)((m >> 52) & 0x7FF) - 1023 + 3 : 0;
}

// 2^sc * S, rounded once to the nearest double (ties to even)
__device__ __forceinline__ double i128_to_double(__int128 S, int sc) {
    if (S == 0) return 0.0;
    const bool neg = S < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-S) : (unsigned __int128)S;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    unsigned long long v = lo;
    int sh = 0;
    if (hi != 0) {
        sh = 64 - __clzll((long long)hi);   // 1..64: the bits above the low word
        const unsigned long long rest = sh == 64 ? lo : (lo << (64 - sh));
        v = (sh == 64 ? hi : ((hi << (64 - sh)) | (lo >> sh))) | (rest != 0 ? 1ull : 0ull);   // sticky bit
    }
    const double d = __ull2double_rn(v);
    // times 2^(sh + sc) in two exact power-of-two factors (each exponent within the normal range)
    const int k = sh + sc, k1 = max(-1022, min(1023, k / 2)), k2 = max(-1022, min(1023, k - k / 2));
    const double f1 = __longlong_as_double((long long)(k1 + 1023) << 52);
    const double f2 = __longlong_as_double((long long)(k2 + 1023) << 52);
    return (neg ? -d : d) * f1 * f2;
}

}  // namespace

// 9 warps: three share one SM sub-partition's 16K registers, so at most 168 a thread
__global__ void __launch_bounds__(N2_THREADS, 1) gram_tc32_kernel(GramArgs a, long long U, int chunks,
                                                                  const unsigned long long* colmax, int ld,
                                                                  int* err, long long limit) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_bar[2 * N2_NS + 5];
    __shared__ unsigned s_tmem;
    __shared__ volatile int s_fail;
    __shared__ int s_last;
    unsigned char* stg = smem_raw + N2_NS * N2_STAGE_BYTES;   // FP64 staging ring, N2_DEPTH + 1 slots
    long long* sH = reinterpret_cast<long long*>(stg + (N2_DEPTH + 1) * N2_STG_BYTES);
    long long* sL = sH + N2_XWORDS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned full0 = smem_u32(&s_bar[0]);            // [N2_NS], 256 arrivals
    const unsigned empty0 = smem_u32(&s_bar[N2_NS]);       // [N2_NS], MMA commit
    const unsigned tfull0 = smem_u32(&s_bar[2 * N2_NS]);   // [2], MMA commit
    const unsigned tempty0 = tfull0 + 16;                  // [2], 256 arrivals
    const unsigned done = tfull0 + 32;                     // MMA commit at exit
    const unsigned stage_s = smem_u32(smem_raw);

    if (tid == 0) {
        for (int q = 0; q < N2_NS; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8u * q), "r"(N2_PROD) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8u * q) : "memory");
        }
        for (int h = 0; h < 2; ++h) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tfull0 + 8u * h) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tempty0 + 8u * h), "r"(N2_PROD) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    // zero the stage ring once (digit rows of columns >= K then only ever hold digits of
    // earlier items, which reach no output read back)
    for (int e = tid; e < N2_NS * N2_STAGE_BYTES / 16; e += N2_THREADS)
        reinterpret_cast<uint4*>(smem_raw)[e] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(N2_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    const int units = a.B * chunks;
    auto unit_lo = [&](int u) -> long long { return (long long)(u % chunks) * U; };
    auto unit_hi = [&](int u) -> long long { return min(a.Ng, (long long)(u % chunks) * U + U); };

    if (warp == 8) {
        // ---------------- MMA issue (one thread) ----------------
        if (lane == 0) {
            int gs = 0, gw = 0;
            bool bad = false;
            for (int u = blockIdx.x; u < units; u += gridDim.x) {
                const long long lo = unit_lo(u), hi = unit_hi(u);
                for (long long w0 = lo; w0 < hi; w0 += N2_WIN, ++gw) {
                    const long long w1 = min(hi, w0 + N2_WIN);
                    const int h = gw & 1;
                    if (!bad && !mbar_wait_f(tempty0 + 8u * h, ((gw >> 1) & 1) ^ 1, &s_fail, limit)) bad = true;
                    const unsigned td = tmem + (unsigned)(h * 256);
                    for (long long p0 = w0; p0 < w1; p0 += N2_PTS, ++gs) {
                        const int q = gs % N2_NS;
                        if (!bad && !mbar_wait_f(full0 + 8u * q, (gs / N2_NS) & 1, &s_fail, limit)) bad = true;
                        if (!bad) {
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const unsigned sb = stage_s + q * N2_STAGE_BYTES;
#pragma unroll
                            for (int k = 0; k < N2_PTS / 16; ++k)
                                mma_n256(td, umma_desc(sb + k * 2 * TC_LBO), (p0 == w0 && k == 0) ? 0u : 1u);
                        }
                        mma_commit(empty0 + 8u * q);
                    }
                    mma_commit(tfull0 + 8u * h);
                }
            }
            mma_commit(done);
            mbar_wait(done, 0);   // every MMA of this CTA has completed (bounded; also after a failure)
        }
        __syncwarp();
    } else {
        // ---------------- producers / read-back (warps 0-7) ----------------
        const int col = ((tid >> 6) << 3) | (tid & 7), kg = (tid >> 3) & 7;
        const int qd = warp & 3, ch = warp >> 2;   // read-back: lane quarter (slice s) and column half
        bool bad = false;
        int gw = 0;
        // one pending read-back: window pw of unit pu (its first / last window?)
        int pu = -1, pw = 0;
        bool pfirst = false, plast = false;

        // Position in the CTA's sequence of stages, with the unit's values kept in registers
        // (no divisions per stage): unit u (item b, K columns, points lo .. hi), stage at p0,
        // and this thread's column pointer (null for col >= K).
        struct Pos {
            int u, b, K;
            long long lo, hi, p0;
            const double* c;
        };
        auto set_unit = [&](Pos& P, int u) {
            P.u = u;
            if (u >= units) return;
            P.b = u / chunks;
            P.K = a.KA[P.b];
            P.lo = (long long)(u - P.b * chunks) * U;
            P.hi = min(a.Ng, P.lo + U);
            P.p0 = P.lo;
            P.c = col < P.K ? reinterpret_cast<const double*>(a.colsA[(size_t)P.b * a.ldcols + col]) : nullptr;
        };
        auto advance = [&](Pos& P) {
            P.p0 += N2_PTS;
            if (P.p0 >= P.hi) set_unit(P, P.u + gridDim.x);
        };
        // this thread's 8 values of a stage (column col, points kg * 8 ..), copied by cp.async
        // into its own 16-byte chunks of a staging slot: chunk k (points 2k, 2k + 1) at
        // (k * 256 + tid) * 16, so that a warp's reads hit distinct banks; points past the
        // unit are zero-filled (source size 0 reads nothing).  Columns >= K are neither
        // copied nor cut: their digit rows reach no output that is read back.
        const unsigned stg_s = smem_u32(stg) + (unsigned)tid * 16u;
        auto issue = [&](const Pos& P, int slot) {
            if (P.c == nullptr) return;
            const long long pb = P.p0 + kg * 8;
            const unsigned d0 = stg_s + (unsigned)(slot * N2_STG_BYTES);
            if (pb + 8 <= P.hi && ((reinterpret_cast<uintptr_t>(P.c) & 15u) == 0)) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + (unsigned)(k * 256 * 16)),
                                 "l"(P.c + pb + 2 * k)
                                 : "memory");
                return;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {   // 8-byte copies (ragged tail or 8-byte aligned columns)
                const bool v = pb + k < P.hi;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d0 + (unsigned)((k >> 1) * 256 * 16 + (k & 1) * 8)),
                             "l"(v ? P.c + pb + k : P.c), "r"(v ? 8u : 0u)
                             : "memory");
            }
        };

        auto readback = [&]() {
            const int h = pw & 1;
            if (!bad && !mbar_wait_f(tfull0 + 8u * h, (pw >> 1) & 1, &s_fail, limit)) bad = true;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned base = tmem + ((unsigned)(32 * qd) << 16) + (unsigned)(h * 256 + 16 * ch);
            long long* hrow = sH + (qd * 32 + lane) * N2_XP + 16 * ch;
            long long* lrow = sL + (qd * 32 + lane) * N2_XP + 16 * ch;
#pragma unroll 1
            for (int j0 = 0; j0 < 16; j0 += 8) {   // two passes of 8 columns (fewer live registers)
                long long H[8], L[8];
#pragma unroll
                for (int e2 = 0; e2 < 8; ++e2) H[e2] = L[e2] = 0ll;
#pragma unroll
                for (int t = 0; t < TC_SLICES; ++t) {
                    float v[8];
                    tmem_ld8(base + (unsigned)(t * 32 + j0), v);
#pragma unroll
                    for (int e2 = 0; e2 < 8; ++e2) {
                        const long long x = (long long)__float2int_rn(v[e2]);   // an exact integer
                        if (t < 4) H[e2] += x << (7 * (3 - t));
                        else L[e2] += x << (7 * (7 - t));
                    }
                }
#pragma unroll
                for (int e2 = 0; e2 < 8; ++e2) {
                    hrow[j0 + e2] = pfirst ? H[e2] : hrow[j0 + e2] + H[e2];
                    lrow[j0 + e2] = pfirst ? L[e2] : lrow[j0 + e2] + L[e2];
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(tempty0 + 8u * h);
            if (!plast) return;
            // ---- the unit's partial: 12 exact terms per output (i <= j), in 128-bit integers
            prod_sync();
            const int b = pu / chunks, chunk = pu - b * chunks;
            const int K = a.KA[b];
            const int mk = a.maxKA;
            __int128* mypart =
                reinterpret_cast<__int128*>(a.part) + ((size_t)b * chunks + chunk) * (size_t)mk * mk;
            for (int o = tid; o < K * K; o += N2_PROD) {
                const int i = o / K, j = o - i * K;
                if (j < i) continue;
                __int128 S = 0;
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    S += ((__int128)sH[(s * 32 + i) * N2_XP + j]) << (7 * (7 - s));
                    S += ((__int128)(sL[(s * 32 + i) * N2_XP + j] + sL[(s * 32 + j) * N2_XP + i])) << (7 * (3 - s));
                }
                mypart[(size_t)i * mk + j] = S;
            }
            __threadfence();
            prod_sync();
            if (tid == 0) {
                const unsigned ticket = atom_add_acq_rel_u32(a.counter + b, 1u);
                s_last = (ticket == (unsigned)chunks - 1u);
            }
            prod_sync();
            if (s_last) {
                __threadfence();
                const __int128* bpart = reinterpret_cast<const __int128*>(a.part) + (size_t)b * chunks * mk * mk;
                double* Gb = a.G + (size_t)b * a.ldG_b;
                for (int o = tid; o < K * K; o += N2_PROD) {
                    const int i = o / K, j = o - i * K;
                    if (j < i) continue;
                    // the chunk partials in batches of 16 independent loads (a chain of
                    // dependent loads here held the CTA for tens of microseconds)
                    const __int128* src = bpart + (size_t)i * mk + j;
                    const size_t cs = (size_t)mk * mk;
                    __int128 S = 0;
                    int cc = 0;
                    for (; cc + 16 <= chunks; cc += 16) {
                        __int128 v[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[e] = src[(size_t)(cc + e) * cs];
#pragma unroll
                        for (int e = 0; e < 16; ++e) S += v[e];
                    }
                    for (; cc < chunks; ++cc) S += src[(size_t)cc * cs];
                    const int sc = col_exp(colmax[(size_t)b * ld + i]) + col_exp(colmax[(size_t)b * ld + j]) - 84;
                    const double g = i128_to_double(S, sc);
                    Gb[(size_t)i * a.ldG + j] = g;
                    Gb[(size_t)j * a.ldG + i] = g;
                }
                if (tid == 0) st_relaxed_u32(a.counter + b, 0u);
            }
            prod_sync();
        };

        // the stages in order; the copies run N2_DEPTH stages ahead of the digit cut
        Pos P, I;
        set_unit(P, blockIdx.x);
        I = P;
        for (int d = 0; d < N2_DEPTH; ++d) {
            if (I.u < units) {
                issue(I, d);
                advance(I);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        int ce = 0;
        int q = 0, slot = 0;             // digit stage gs % N2_NS, staging slot gs % (N2_DEPTH + 1)
        unsigned eph = 1u;               // parity to wait for on the digit stage's free barrier
        while (P.u < units) {
            if (I.u < units) {
                issue(I, slot == 0 ? N2_DEPTH : slot - 1);   // slot (gs + N2_DEPTH) % (N2_DEPTH + 1)
                advance(I);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            if (P.p0 == P.lo)   // a new unit: this thread's column exponent
                ce = col_exp(P.c ? colmax[(size_t)P.b * ld + col] : 0ull) + 1020;
            asm volatile("cp.async.wait_group %0;" ::"n"(N2_DEPTH) : "memory");   // this stage's copies
            if (!bad && !mbar_wait_f(empty0 + 8u * q, eph, &s_fail, limit)) bad = true;
            if (P.c) {
                double xc[8];
                const unsigned char* sp = stg + (size_t)slot * N2_STG_BYTES + (size_t)tid * 16;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const double2 v = *reinterpret_cast<const double2*>(sp + k * 256 * 16);
                    xc[2 * k] = v.x;
                    xc[2 * k + 1] = v.y;
                }
                unsigned zl[8], zh[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) cut56(xc[k], ce, zl[k], zh[k]);
                // slice s holds digit k = 7 - s (bits 7k .. 7k + 6 of z); row 32 s + col, K group kg
                unsigned char* rowp = smem_raw + q * N2_STAGE_BYTES + ((col >> 3) * 8 + kg) * 128 + (col & 7) * 16;
#define N2_SLICE(S)                                                                                        \
    *reinterpret_cast<uint4*>(rowp + (S) * 4 * 1024) =                                                     \
        make_uint4(digit_pair<7 * (7 - (S))>(zl[0], zh[0], zl[1], zh[1]),                                  \
                   digit_pair<7 * (7 - (S))>(zl[2], zh[2], zl[3], zh[3]),                                  \
                   digit_pair<7 * (7 - (S))>(zl[4], zh[4], zl[5], zh[5]),                                  \
                   digit_pair<7 * (7 - (S))>(zl[6], zh[6], zl[7], zh[7]));
                N2_SLICE(0) N2_SLICE(1) N2_SLICE(2) N2_SLICE(3) N2_SLICE(4) N2_SLICE(5) N2_SLICE(6) N2_SLICE(7)
#undef N2_SLICE
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            mbar_arrive(full0 + 8u * q);
            // the end of a window: read back the previous one, this one becomes pending
            const long long wend = min(P.hi, P.lo + (((P.p0 - P.lo) >> 12) + 1) * N2_WIN);
            if (P.p0 + N2_PTS >= wend) {
                if (pu >= 0) readback();
                pu = P.u;
                pw = gw;
                pfirst = (P.p0 - P.lo) < N2_WIN;
                plast = (wend == P.hi);
                ++gw;
            }
            if (++q == N2_NS) {
                q = 0;
                eph ^= 1u;
            }
            slot = (slot == N2_DEPTH) ? 0 : slot + 1;
            advance(P);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (pu >= 0) readback();
    }
    if (s_fail && tid == 0) record_error(err, DERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 8) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N2_TMEM_COLS)
                     : "memory");
    }
}

int gram_tc_max_cols() { return TC_N; }

cudaError_t launch_gram_tc(const GramArgs& a, unsigned long long* colmax, int ld, int* err, long long spin_limit,
                           cudaStream_t st) {
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
    if (a.maxKA <= N2_COLS && chunks >= 2) {
        // narrow form: units of U points (at least two per partial slot of the other Gram
        // kernels, since a unit's partial is K x K 128-bit integers)
        const int ctc = chunks / 2;
        const long long U2 = ((a.Ng + ctc - 1) / ctc + N2_PTS - 1) / N2_PTS * N2_PTS;
        const int chunks2 = (int)((a.Ng + U2 - 1) / U2);
        e = cudaFuncSetAttribute((const void*)gram_tc32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 N2_SMEM);
        if (e != cudaSuccess) return e;
        const int grid2 = std::max(1, std::min(sms, a.B * chunks2));
        gram_tc32_kernel<<<grid2, N2_THREADS, N2_SMEM, st>>>(a, U2, chunks2, colmax, ld, err, spin_limit);
        ++g_launch_count;
        return cudaGetLastError();
    }
    const int grid = std::max(1, std::min(sms, a.B * chunks));
    gram_tc_kernel<<<grid, TC_THREADS, smem, st>>>(a, CH, chunks, colmax, ld, err, spin_limit);
    ++g_launch_count;
    return cudaGetLastError();
}

}  // namespace pr
