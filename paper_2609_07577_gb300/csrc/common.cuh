// Internal helpers shared by the CUDA translation units of libsnnmap.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

namespace snn {

// ---------------------------------------------------------------------------
// Device status word bits (set by kernels with atomicOr, read by the host).
enum : int32_t {
    ST_INVALID = 1,     // input breaks the documented layout
    ST_INFEASIBLE = 2,  // one neuron alone breaks Delta or Phi
    ST_CAPACITY = 4,    // an internal buffer bound was exceeded (never expected)
    ST_TIMEOUT = 8,     // a bounded device wait ran out
    ST_BADSTATE = 16,   // refinement started from a state breaking a limit
};

// Host-side error carrier.
struct Status {
    int code = 0;
    std::string msg;
    bool ok() const { return code == 0; }
};

#define SNN_CUDA(call)                                                           \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            return ::snn::Status{e_ == cudaErrorMemoryAllocation ? 3 : 5,        \
                                 std::string(#call) + ": " + cudaGetErrorString(e_)}; \
        }                                                                        \
    } while (0)

#define SNN_TRY(expr)                         \
    do {                                      \
        ::snn::Status s_ = (expr);            \
        if (!s_.ok()) return s_;              \
    } while (0)

constexpr unsigned FULL = 0xffffffffu;

// Every kernel launch of the library goes through SNN_L, which counts it
// (process-wide, reported by snnmap_launch_count).
void note_launch();
int64_t launch_count();
#define SNN_L (void)::snn::note_launch(),

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// 64-bit finalizer (splitmix64) used for hyperedge content hashes and
// hash-table probing; only ever compared for equality, never for results.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline int bits_for(uint64_t maxval)
{
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
}

// ---------------------------------------------------------------------------
// One level of the hierarchy, all arrays in device memory (structure of
// arrays). Hyperedge a has pins hpins[hoff[a] .. hoff[a+1]): the source
// first, then its distinct destination super-nodes in ascending order.
// vinc lists the hyperedges incident to each vertex, with bit 31 set when
// the vertex is the hyperedge's source.
struct Level {
    int32_t V = 0, E = 0;
    int64_t P = 0;
    int64_t* hoff = nullptr;
    int32_t* hpins = nullptr;
    int64_t* hw = nullptr;
    int32_t* hk = nullptr;
    uint8_t* hsd = nullptr;
    int64_t* voff = nullptr;
    int32_t* vinc = nullptr;
    int32_t* vsize = nullptr;
    int32_t* vinpins = nullptr;
    int32_t* vincnt = nullptr;
    int32_t* vinint = nullptr;
    int32_t* cid = nullptr;      // map to the next level (own allocation, always kept)
    int32_t maxlen = 0;          // longest hyperedge
    void* block = nullptr;       // single allocation holding every array but cid
    size_t bytes = 0;
    bool resident = false;       // arrays in memory (else only sizes and cid)
};

constexpr uint32_t SRC_BIT = 0x80000000u;

// Carves several arrays out of one device allocation.
struct Carver {
    size_t total = 0;
    std::vector<std::pair<void**, size_t>> items;
    template <typename T>
    void add(T** p, int64_t n)
    {
        size_t b = (size_t)(n > 0 ? n : 1) * sizeof(T);
        b = (b + 255) & ~(size_t)255;
        items.push_back({(void**)p, b});
        total += b;
    }
    void assign(void* base)
    {
        char* c = (char*)base;
        for (auto& it : items) {
            *it.first = c;
            c += it.second;
        }
    }
};

// Device memory of a handle: stream-ordered allocations from one memory pool
// per device that keeps freed blocks for reuse across stream
// synchronizations. (The default pool hands unused memory back to the CUDA driver
// at every synchronization, so each level's and each refinement round's
// arrays would be mapped afresh.) The pool is trimmed to nothing when the
// last live handle is freed (pool_handles(-1) returns 0).
cudaError_t dev_malloc(void** p, size_t bytes, cudaStream_t s);
template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes, cudaStream_t s)
{
    return dev_malloc((void**)p, bytes, s);
}
// adds `delta` (+1 at handle creation, -1 at its release) to the count of
// live handles and returns the new count; at 0 the pools are trimmed
int pool_handles(int delta);

// Bump allocator for temporaries of one step. Memory stays reserved across
// steps and grows (stream-ordered) when a step needs more.
struct Arena {
    std::vector<void*> chunks;
    std::vector<size_t> sizes;
    size_t used = 0;      // in the last chunk
    size_t peak = 0;      // sum needed by the largest step
    size_t step_total = 0;
    cudaStream_t stream = 0;

    Status reserve(size_t bytes);
    Status take(size_t bytes, void** out);
    template <typename T>
    Status alloc(T** p, int64_t n)
    {
        void* v = nullptr;
        SNN_TRY(take((size_t)(n > 0 ? n : 1) * sizeof(T), &v));
        *p = (T*)v;
        return Status{};
    }
    // position of the bump pointer; rewind(m) hands back everything taken
    // after mark() returned m (chunks added since are freed, stream-ordered)
    struct Mark {
        size_t nchunks, used, step_total;
    };
    Mark mark() const { return Mark{chunks.size(), used, step_total}; }
    void rewind(const Mark& m);
    void reset();              // forget this step's allocations (stream-ordered)
    void release();            // free everything
    size_t held() const;
};

// ---------------------------------------------------------------------------
// Primitives (prims.cu).

// out[i] = sum of in[0..i) (exclusive); *total (device, may be null) = sum.
Status scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* total,
                                 Arena& ar, cudaStream_t s);
Status scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                          Arena& ar, cudaStream_t s);
Status scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total,
                          Arena& ar, cudaStream_t s);
// inclusive sum scans
Status scan_inclusive_i64(const int64_t* in, int64_t* out, int64_t n, Arena& ar, cudaStream_t s);
Status scan_inclusive_i32(const int32_t* in, int32_t* out, int64_t n, Arena& ar, cudaStream_t s);
// inclusive max scan
Status scan_inclusive_max_i32(const int32_t* in, int32_t* out, int64_t n, Arena& ar,
                              cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs over key bits [0, end_bit).
// Sorted data ends in (keys, vals); the *_alt buffers are scratch of size n.
Status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                        int64_t n, int end_bit, Arena& ar, cudaStream_t s);

// Small fills.
Status fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s);
Status fill_i64(int64_t* p, int64_t v, int64_t n, cudaStream_t s);
Status iota_i32(int32_t* p, int64_t n, cudaStream_t s);

// Grid size for grid-stride loops over n items.
inline int grid_for(int64_t n, int threads, int cap = 152 * 32)
{
    int64_t g = ceil_div(n > 0 ? n : 1, threads);
    return (int)(g < cap ? g : cap);
}

// Lanes per hyperedge for the kernels that spread one hyperedge's pins over a
// group of lanes: the mean hyperedge size (pins per hyperedge) rounded up to
// a power of two in [4, 32], so that short hyperedges do not leave most of a
// warp idle. Groups are aligned within their warp.
inline int hedge_lanes(int64_t P, int64_t E)
{
    int64_t m = E > 0 ? (P + E - 1) / E : 32;
    int g = 4;
    while (g < 32 && g < m) g <<= 1;
    return g;
}

// launches kern<G> (G of 4, 8, 16, 32 lanes per hyperedge) with enough
// threads for n hyperedges
#define SNN_HEDGE_LAUNCH(G, kern, n, s, ...)                                                     \
    do {                                                                                         \
        switch (G) {                                                                             \
        case 4:                                                                                  \
            SNN_L kern<4><<<::snn::grid_for((int64_t)(n) * 4, 256), 256, 0, s>>>(__VA_ARGS__);     \
            break;                                                                               \
        case 8:                                                                                  \
            SNN_L kern<8><<<::snn::grid_for((int64_t)(n) * 8, 256), 256, 0, s>>>(__VA_ARGS__);     \
            break;                                                                               \
        case 16:                                                                                 \
            SNN_L kern<16><<<::snn::grid_for((int64_t)(n) * 16, 256), 256, 0, s>>>(__VA_ARGS__);   \
            break;                                                                               \
        default:                                                                                 \
            SNN_L kern<32><<<::snn::grid_for((int64_t)(n) * 32, 256), 256, 0, s>>>(__VA_ARGS__);   \
        }                                                                                        \
    } while (0)

}  // namespace snn
