// pr_op_apply_L_noalloc: the operator L_h (or L_h^T) on caller buffers without any device
// allocation.
//
// Some callers cannot call cudaMalloc at all: code running while another framework owns
// the whole device memory budget (a caching allocator holding every free byte, a fixed
// memory plan in an inference server), code on a thread that must not block on the
// allocator's implicit synchronisation, or hosts that forbid late allocations after
// start-up.  pr_op_apply_L needs the context workspace (velocity tables and column
// pointer lists); this variant keeps that scratch in one file-scope __device__ array of
// NOALLOC_SCRATCH_BYTES (13 568) bytes instead, which every GPU that loads the library
// holds until the process exits.  Limits: n <= 256 and at most 64 grid functions per call.
//
// The array is shared by all calls on a device and keeps the last call's contents; every
// call rewrites all of it that it reads, so nothing needs clearing.  Two calls whose work
// overlaps on the GPU (different streams, no ordering) race on it.  The device address of
// the array is looked up with cudaGetSymbolAddress on the first call on each device, with
// that device current, and kept for the life of the process; do not use the library
// across a cudaDeviceReset, which would leave the kept address stale.
#include "pr_internal.cuh"

#include <algorithm>
#include <mutex>
#include <vector>

namespace pr {

constexpr int NOALLOC_MAX_N = 256;       // velocity tables: 6 x n doubles
constexpr int NOALLOC_MAX_COLS = 64;     // grid functions per call
constexpr size_t NOALLOC_TAB_BYTES = (size_t)6 * NOALLOC_MAX_N * sizeof(double);
constexpr size_t NOALLOC_PTR_BYTES = (size_t)NOALLOC_MAX_COLS * sizeof(void*);
constexpr size_t NOALLOC_SCRATCH_BYTES =
    NOALLOC_TAB_BYTES + 2 * NOALLOC_PTR_BYTES + NOALLOC_MAX_COLS * sizeof(int);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

__global__ void noalloc_fill_counts(int* counts, int cnt) {
    const int i = threadIdx.x;
    if (i < NOALLOC_MAX_COLS) counts[i] = (i < cnt) ? 1 : 0;
}

namespace {
std::mutex g_noalloc_mu;
std::vector<unsigned char*> g_noalloc_addr;  // per device, set up on first use
}

// Device address of the scratch array on the current device (looked up once per device).
static cudaError_t noalloc_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if ((int)g_noalloc_addr.size() <= dev) g_noalloc_addr.resize(dev + 1, nullptr);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

int noalloc_max_n() { return NOALLOC_MAX_N; }
int noalloc_max_count() { return NOALLOC_MAX_COLS; }
size_t noalloc_scratch_bytes() { return NOALLOC_SCRATCH_BYTES; }

cudaError_t apply_L_noalloc(int n, double L, const pr_flow& flow, const double* d_pert, double eps,
                            const double* d_in, double* d_out, int count, bool transpose, cudaStream_t st) {
    if (n > NOALLOC_MAX_N || count > NOALLOC_MAX_COLS) return cudaErrorInvalidValue;
    if (count <= 0) return cudaSuccess;
    unsigned char* base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return e;
    double* tab = reinterpret_cast<double*>(base);
    void** in_ptrs = reinterpret_cast<void**>(base + NOALLOC_TAB_BYTES);
    void** out_ptrs = reinterpret_cast<void**>(base + NOALLOC_TAB_BYTES + NOALLOC_PTR_BYTES);
    int* counts = reinterpret_cast<int*>(base + NOALLOC_TAB_BYTES + 2 * NOALLOC_PTR_BYTES);
    e = launch_tables(flow, n, L, tab, st);
    if (e != cudaSuccess) return e;
    Grid g;
    g.n = n;
    g.Ng = (long long)n * n * n;
    g.h = L / n;
    g.eps = eps;
    g.tab = tab;
    g.pert = d_pert;
    void* hin[NOALLOC_MAX_COLS];
    void* hout[NOALLOC_MAX_COLS];
    for (int i = 0; i < count; ++i) {
        hin[i] = const_cast<double*>(d_in) + (size_t)i * g.Ng;
        hout[i] = d_out + (size_t)i * g.Ng;
    }
    // pageable async copies are staged before returning and ordered on the stream
    e = cudaMemcpyAsync(in_ptrs, hin, sizeof(void*) * count, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(out_ptrs, hout, sizeof(void*) * count, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    noalloc_fill_counts<<<1, NOALLOC_MAX_COLS, 0, st>>>(counts, count);
    ++g_launch_count;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one column per batch item: count[b] = 1 for b < count
    return launch_apply_L(g, (const void* const*)in_ptrs, (void* const*)out_ptrs, counts, 1, 1, count,
                          false, false, transpose, st);
}

}  // namespace pr
