// Device-wide primitives: scratch arena, prefix scans and a stable LSD radix
// sort. Everything here is deterministic (no atomics on values whose order
// matters, no spin waits): reduce-then-scan for scans, and for the sort a
// per-tile digit histogram, a scan of the digit-major histogram table and a
// stable scatter whose in-tile ranks come from warp match_any groups.
#include "common.cuh"

#include <atomic>
#include <climits>
#include <mutex>

namespace snn {

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Pool-backed device allocations

namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};
int g_live_handles = 0;
}  // namespace

static cudaError_t pool_of(int dev, cudaMemPool_t* out)
{
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps pr{};
        pr.allocType = cudaMemAllocationTypePinned;
        pr.handleTypes = cudaMemHandleTypeNone;
        pr.location.type = cudaMemLocationTypeDevice;
        pr.location.id = dev;
        cudaMemPool_t p = nullptr;
        cudaError_t e = cudaMemPoolCreate(&p, &pr);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        // handles on other streams (the batched and served forms) reuse
        // freed blocks only once their frees are known complete: no wait is
        // ever inserted between their streams
        int no = 0;
        if (e == cudaSuccess)
            e = cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowInternalDependencies, &no);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pools[dev] = p;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

cudaError_t dev_malloc(void** p, size_t bytes, cudaStream_t s)
{
    int dev = -1;
    cudaError_t e = cudaStreamGetDevice(s, &dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = nullptr;
    e = pool_of(dev, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

int pool_handles(int delta)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    g_live_handles += delta;
    if (g_live_handles < 0) g_live_handles = 0;
    if (g_live_handles == 0)
        for (cudaMemPool_t p : g_pools)
            if (p) cudaMemPoolTrimTo(p, 0);
    return g_live_handles;
}

// ---------------------------------------------------------------------------
// Arena

Status Arena::reserve(size_t bytes)
{
    if (!chunks.empty() && sizes.back() >= bytes && chunks.size() == 1) return Status{};
    release();
    void* p = nullptr;
    SNN_CUDA(dev_malloc(&p, bytes, stream));
    chunks.push_back(p);
    sizes.push_back(bytes);
    used = 0;
    return Status{};
}

Status Arena::take(size_t bytes, void** out)
{
    bytes = (bytes + 255) & ~(size_t)255;
    step_total += bytes;
    if (chunks.empty() || used + bytes > sizes.back()) {
        size_t want = bytes;
        if (chunks.empty() && peak > want) want = peak;
        if (want < ((size_t)64 << 20)) want = (size_t)64 << 20;
        void* p = nullptr;
        SNN_CUDA(dev_malloc(&p, want, stream));
        chunks.push_back(p);
        sizes.push_back(want);
        used = 0;
    }
    *out = (char*)chunks.back() + used;
    used += bytes;
    return Status{};
}

void Arena::reset()
{
    if (step_total > peak) peak = step_total;
    if (chunks.size() > 1) {
        // consolidate: next step gets one chunk as large as this step needed
        for (void* p : chunks) cudaFreeAsync(p, stream);
        chunks.clear();
        sizes.clear();
        void* p = nullptr;
        size_t want = peak + ((size_t)16 << 20);
        if (dev_malloc(&p, want, stream) == cudaSuccess) {
            chunks.push_back(p);
            sizes.push_back(want);
        }
    }
    used = 0;
    step_total = 0;
}

void Arena::rewind(const Mark& m)
{
    if (step_total > peak) peak = step_total;
    while (chunks.size() > m.nchunks && !chunks.empty()) {
        cudaFreeAsync(chunks.back(), stream);
        chunks.pop_back();
        sizes.pop_back();
    }
    used = m.used;
    step_total = m.step_total;
}

void Arena::release()
{
    for (void* p : chunks) cudaFreeAsync(p, stream);
    chunks.clear();
    sizes.clear();
    used = 0;
}

size_t Arena::held() const
{
    size_t t = 0;
    for (size_t s : sizes) t += s;
    return t;
}

// ---------------------------------------------------------------------------
// Fills

template <typename T>
__global__ void k_fill(T* p, T v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_iota(int32_t* p, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

Status fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s)
{
    if (n <= 0) return Status{};
    SNN_L k_fill<int32_t><<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
    SNN_CUDA(cudaGetLastError());
    return Status{};
}

Status fill_i64(int64_t* p, int64_t v, int64_t n, cudaStream_t s)
{
    if (n <= 0) return Status{};
    SNN_L k_fill<int64_t><<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
    SNN_CUDA(cudaGetLastError());
    return Status{};
}

Status iota_i32(int32_t* p, int64_t n, cudaStream_t s)
{
    if (n <= 0) return Status{};
    SNN_L k_iota<<<grid_for(n, 256), 256, 0, s>>>(p, n);
    SNN_CUDA(cudaGetLastError());
    return Status{};
}

// ---------------------------------------------------------------------------
// Scans

constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

template <typename T>
struct OpSum {
    __device__ static T id() { return (T)0; }
    __device__ T operator()(T a, T b) const { return a + b; }
};

template <typename T>
struct OpMax {
    __device__ static T id() { return sizeof(T) == 8 ? (T)LLONG_MIN : (T)INT_MIN; }
    __device__ T operator()(T a, T b) const { return a > b ? a : b; }
};

template <typename T, typename Op>
__device__ T block_reduce(T v, T* sh)
{
    Op op;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(FULL, v, o));
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < SC_THREADS / 32 ? sh[lane] : Op::id();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(FULL, v, o));
    }
    return v;
}

// exclusive scan of one value per thread across the block; sh holds >= 64 T
template <typename T, typename Op>
__device__ T block_exclusive(T v, T* sh)
{
    Op op;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc = op(t, inc);
    }
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T wi = lane < SC_THREADS / 32 ? sh[lane] : Op::id();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi = op(t, wi);
        }
        T ex = __shfl_up_sync(FULL, wi, 1);
        if (lane == 0) ex = Op::id();
        if (lane < SC_THREADS / 32) sh[32 + lane] = ex;
    }
    __syncthreads();
    T warp_ex = sh[32 + warp];
    T exl = __shfl_up_sync(FULL, inc, 1);
    if (lane == 0) exl = Op::id();
    T r = op(warp_ex, exl);
    __syncthreads();
    return r;
}

template <typename Tin, typename T, typename Op>
__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce(const Tin* in, int64_t n, T* bsum)
{
    __shared__ T sh[SC_THREADS / 32];
    Op op;
    T acc = Op::id();
    int64_t base = (int64_t)blockIdx.x * SC_TILE;
    for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS) {
        int64_t j = base + i;
        if (j < n) acc = op(acc, (T)in[j]);
    }
    acc = block_reduce<T, Op>(acc, sh);
    if (threadIdx.x == 0) bsum[blockIdx.x] = acc;
}

template <typename Tin, typename T, typename Op, bool INCL>
__global__ void __launch_bounds__(SC_THREADS)
    k_scan_tile(const Tin* in, int64_t n, T* out, const T* boff, T* total)
{
    __shared__ T tile[SC_TILE];
    __shared__ T sh[64];
    Op op;
    int64_t base = (int64_t)blockIdx.x * SC_TILE;
    for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS) {
        int64_t j = base + i;
        tile[i] = j < n ? (T)in[j] : Op::id();
    }
    __syncthreads();
    T v[SC_ITEMS];
    T run = Op::id();
#pragma unroll
    for (int k = 0; k < SC_ITEMS; k++) {
        v[k] = tile[threadIdx.x * SC_ITEMS + k];
        run = op(run, v[k]);
    }
    T ex = block_exclusive<T, Op>(run, sh);
    T acc = op(boff ? boff[blockIdx.x] : Op::id(), ex);
#pragma unroll
    for (int k = 0; k < SC_ITEMS; k++) {
        if (INCL) {
            acc = op(acc, v[k]);
            tile[threadIdx.x * SC_ITEMS + k] = acc;
        } else {
            tile[threadIdx.x * SC_ITEMS + k] = acc;
            acc = op(acc, v[k]);
        }
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == SC_THREADS - 1) *total = acc;
    __syncthreads();
    for (int i = threadIdx.x; i < SC_TILE; i += SC_THREADS) {
        int64_t j = base + i;
        if (j < n) out[j] = tile[i];
    }
}

template <typename T, typename Op>
__global__ void k_set_identity(T* p)
{
    *p = Op::id();
}

template <typename Tin, typename T, typename Op, bool INCL>
static Status scan_impl(const Tin* in, T* out, int64_t n, T* total, Arena& ar, cudaStream_t s)
{
    if (n <= 0) {
        if (total) {
            SNN_L k_set_identity<T, Op><<<1, 1, 0, s>>>(total);
            SNN_CUDA(cudaGetLastError());
        }
        return Status{};
    }
    int64_t nb = ceil_div(n, SC_TILE);
    if (nb == 1) {
        SNN_L k_scan_tile<Tin, T, Op, INCL><<<1, SC_THREADS, 0, s>>>(in, n, out, nullptr, total);
        SNN_CUDA(cudaGetLastError());
        return Status{};
    }
    T* bsum = nullptr;
    SNN_TRY(ar.alloc(&bsum, nb));
    SNN_L k_scan_reduce<Tin, T, Op><<<(unsigned)nb, SC_THREADS, 0, s>>>(in, n, bsum);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY((scan_impl<T, T, Op, false>(bsum, bsum, nb, nullptr, ar, s)));
    SNN_L k_scan_tile<Tin, T, Op, INCL><<<(unsigned)nb, SC_THREADS, 0, s>>>(in, n, out, bsum, total);
    SNN_CUDA(cudaGetLastError());
    return Status{};
}

Status scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* total,
                                 Arena& ar, cudaStream_t s)
{
    return scan_impl<int32_t, int64_t, OpSum<int64_t>, false>(in, out, n, total, ar, s);
}

Status scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, Arena& ar,
                          cudaStream_t s)
{
    return scan_impl<int64_t, int64_t, OpSum<int64_t>, false>(in, out, n, total, ar, s);
}

Status scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total, Arena& ar,
                          cudaStream_t s)
{
    return scan_impl<int32_t, int32_t, OpSum<int32_t>, false>(in, out, n, total, ar, s);
}

Status scan_inclusive_i64(const int64_t* in, int64_t* out, int64_t n, Arena& ar, cudaStream_t s)
{
    return scan_impl<int64_t, int64_t, OpSum<int64_t>, true>(in, out, n, nullptr, ar, s);
}

Status scan_inclusive_i32(const int32_t* in, int32_t* out, int64_t n, Arena& ar, cudaStream_t s)
{
    return scan_impl<int32_t, int32_t, OpSum<int32_t>, true>(in, out, n, nullptr, ar, s);
}

Status scan_inclusive_max_i32(const int32_t* in, int32_t* out, int64_t n, Arena& ar,
                              cudaStream_t s)
{
    return scan_impl<int32_t, int32_t, OpMax<int32_t>, true>(in, out, n, nullptr, ar, s);
}

// ---------------------------------------------------------------------------
// Radix sort: 8-bit digits, tiles of 4096 keys (8 warps x 16 rounds of 32).

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

__global__ void __launch_bounds__(RS_THREADS)
    k_rs_upsweep(const uint64_t* keys, int64_t n, int shift, uint32_t* counts, int nblk)
{
    __shared__ uint32_t hist[256];
    for (int i = threadIdx.x; i < 256; i += RS_THREADS) hist[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        int64_t j = base + i;
        if (j < n) atomicAdd(&hist[(keys[j] >> shift) & 255], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += RS_THREADS) counts[(int64_t)i * nblk + blockIdx.x] = hist[i];
}

__global__ void __launch_bounds__(RS_THREADS)
    k_rs_downsweep(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                   int64_t n, int shift, const uint32_t* offs, int nblk)
{
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t boff[256];
    __shared__ uint32_t tmp[RS_WARPS][32];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    for (int i = threadIdx.x; i < 256; i += RS_THREADS) boff[i] = offs[(int64_t)i * nblk + blockIdx.x];
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (32 * RS_ROUNDS);
    uint64_t k[RS_ROUNDS];
    uint32_t rank[RS_ROUNDS];
    unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t j = base + r * 32 + lane;
        bool valid = j < n;
        k[r] = valid ? kin[j] : 0;
        uint32_t d = valid ? (uint32_t)((k[r] >> shift) & 255) : 256u;
        unsigned peers = __match_any_sync(FULL, d);
        int leader = __ffs(peers) - 1;
        if (lane == leader && valid) {
            uint32_t c = wcnt[warp][d];
            tmp[warp][lane] = c;
            wcnt[warp][d] = c + __popc(peers);
        }
        __syncwarp();
        rank[r] = valid ? tmp[warp][leader] + __popc(peers & lt) : 0;
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps per digit, plus the block's global offset
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
        uint32_t acc = boff[d];
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = wcnt[w][d];
            wcnt[w][d] = acc;
            acc += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t j = base + r * 32 + lane;
        if (j < n) {
            uint32_t d = (uint32_t)((k[r] >> shift) & 255);
            uint32_t pos = wcnt[warp][d] + rank[r];
            kout[pos] = k[r];
            vout[pos] = vin[j];
        }
    }
}

Status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                        int64_t n, int end_bit, Arena& ar, cudaStream_t s)
{
    if (n <= 1 || end_bit <= 0) return Status{};
    if (n >= ((int64_t)1 << 32)) return Status{1, "radix sort: too many items"};
    int nblk = (int)ceil_div(n, RS_TILE);
    uint32_t* counts = nullptr;
    SNN_TRY(ar.alloc(&counts, (int64_t)256 * nblk));
    int passes = (end_bit + 7) / 8;
    uint64_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        SNN_L k_rs_upsweep<<<nblk, RS_THREADS, 0, s>>>(ki, n, shift, counts, nblk);
        SNN_CUDA(cudaGetLastError());
        SNN_TRY((scan_impl<uint32_t, uint32_t, OpSum<uint32_t>, false>(counts, counts,
                                                                      (int64_t)256 * nblk,
                                                                      nullptr, ar, s)));
        SNN_L k_rs_downsweep<<<nblk, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n, shift, counts, nblk);
        SNN_CUDA(cudaGetLastError());
        uint64_t* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
    }
    if (ki != keys) {
        SNN_CUDA(cudaMemcpyAsync(keys, ki, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        SNN_CUDA(cudaMemcpyAsync(vals, vi, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    return Status{};
}

}  // namespace snn
