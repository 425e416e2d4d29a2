// Segmented sort of small uint32 key lists, one list per hyperedge, followed
// by a per-hyperedge epilogue. Hyperedges are split into size buckets once
// per level (by pin count L):
//   T:  L <= 16      one thread, keys in a local array (insertion sort)
//   B0: L <= 32      one warp, keys in registers (shuffle bitonic network)
//   B1: L <= 256     one warp, keys in a per-warp shared-memory slice
//   B2: L <= 16384   one block of 512 threads, keys in dynamic shared memory
//   B3: larger       one block of 1024 threads, keys in a global scratch slice
// Each kernel walks its bucket's list with a grid-stride loop whose bound is
// read on the device, so no host synchronization is needed to launch them.
// Sorted keys are padded with 0xffffffff, which no key may equal.
//
// A Job supplies:
//   __device__ int len(int32_t a)                number of keys of hyperedge a
//   __device__ uint32_t load(int32_t a, int i)   key i (0 <= i < len)
//   __device__ void finish(int32_t a, const uint32_t* s, int n)
//        run by one full warp on the n sorted keys s[0..n)
//   __device__ void finish_thread(int32_t a, const uint32_t* s, int n, int st)
//                                                   (key i at s[i * st])
//        the same, run by a single thread
#pragma once
#include "common.cuh"

namespace snn {

constexpr int SEG_T_CAP = 16;
constexpr int SEG_B1_CAP = 256;
constexpr int SEG_B2_CAP = 16384;
constexpr int SEG_B2_THREADS = 512;
constexpr int SEG_B3_THREADS = 1024;
constexpr int SEG_B3_BLOCKS = 16;
constexpr uint32_t KEY_PAD = 0xffffffffu;

// Per-level bucket lists of hyperedge ids: one array of E ids holding the
// buckets (T, B0, B1, B2, B3) back to back; meta (device int32[10]) =
// start[5], count[5].
struct SegBuckets {
    int32_t* list = nullptr;
    int32_t* meta = nullptr;
    int64_t b3_cap = 0;        // power of two >= longest hyperedge if any is in B3
};

__device__ __forceinline__ uint32_t warp_bitonic32(uint32_t v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            uint32_t o = __shfl_xor_sync(FULL, v, j);
            bool up = (lane & k) == 0;
            bool lower = (lane & j) == 0;
            uint32_t mn = v < o ? v : o, mx = v < o ? o : v;
            v = (lower == up) ? mn : mx;
        }
    }
    return v;
}

__device__ __forceinline__ int pow2_at_least(int n, int lo)
{
    int p = lo;
    while (p < n) p <<= 1;
    return p;
}

// bitonic sort of s[0..N) (N a power of two) by one warp
__device__ __forceinline__ void warp_bitonic_smem(uint32_t* s, int N)
{
    int lane = threadIdx.x & 31;
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < N; i += 32) {
                int ixj = i ^ j;
                if (ixj > i) {
                    uint32_t a = s[i], b = s[ixj];
                    bool asc = (i & k) == 0;
                    if ((a > b) == asc) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// bitonic sort of s[0..N) by the whole block (s in shared or global memory)
__device__ __forceinline__ void block_bitonic(uint32_t* s, int N)
{
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    uint32_t a = s[i], b = s[ixj];
                    bool asc = (i & k) == 0;
                    if ((a > b) == asc) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

enum : int { SEG_BT = 0, SEG_BB0 = 1, SEG_BB1 = 2, SEG_BB2 = 3, SEG_BB3 = 4, SEG_NB = 5 };

// One thread per list of at most SEG_T_CAP keys: the keys are sorted in
// registers by a fully unrolled bitonic network (padding sorts last) and
// handed to the epilogue through shared memory, slot i of thread t at
// i * blockDim + t so that a warp's lanes touch consecutive banks.
template <class Job>
__global__ void __launch_bounds__(256) k_seg_t(Job job, const int32_t* __restrict__ lists,
                                               const int32_t* __restrict__ meta)
{
    __shared__ uint32_t sk[SEG_T_CAP * 256];
    const int32_t* list = lists + meta[SEG_BT];
    int n = meta[SEG_NB + SEG_BT];
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        int idx = base + threadIdx.x;
        if (idx >= n) continue;
        int32_t a = list[idx];
        int L = job.len(a);
        uint32_t k[SEG_T_CAP];
#pragma unroll
        for (int i = 0; i < SEG_T_CAP; i++) k[i] = i < L ? job.load(a, i) : KEY_PAD;
#pragma unroll
        for (int w = 2; w <= SEG_T_CAP; w <<= 1) {
#pragma unroll
            for (int j = w >> 1; j > 0; j >>= 1) {
#pragma unroll
                for (int i = 0; i < SEG_T_CAP; i++) {
                    int l = i ^ j;
                    if (l > i) {
                        bool up = (i & w) == 0;
                        uint32_t x = k[i], y = k[l];
                        if ((x > y) == up) {
                            k[i] = y;
                            k[l] = x;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < SEG_T_CAP; i++) sk[i * 256 + threadIdx.x] = k[i];
        job.finish_thread(a, sk + threadIdx.x, L, 256);
    }
}

template <class Job>
__global__ void __launch_bounds__(256) k_seg_b0(Job job, const int32_t* __restrict__ lists,
                                                const int32_t* __restrict__ meta)
{
    __shared__ uint32_t buf[8][32];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t* list = lists + meta[SEG_BB0];
    int n = meta[SEG_NB + SEG_BB0];
    for (int idx = blockIdx.x * 8 + warp; idx < n; idx += gridDim.x * 8) {
        int32_t a = list[idx];
        int L = job.len(a);
        uint32_t v = lane < L ? job.load(a, lane) : KEY_PAD;
        v = warp_bitonic32(v);
        buf[warp][lane] = v;
        __syncwarp();
        job.finish(a, buf[warp], L);
        __syncwarp();
    }
}

template <class Job>
__global__ void __launch_bounds__(256) k_seg_b1(Job job, const int32_t* __restrict__ lists,
                                                const int32_t* __restrict__ meta)
{
    __shared__ uint32_t buf[8][SEG_B1_CAP];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t* list = lists + meta[SEG_BB1];
    int n = meta[SEG_NB + SEG_BB1];
    uint32_t* s = buf[warp];
    for (int idx = blockIdx.x * 8 + warp; idx < n; idx += gridDim.x * 8) {
        int32_t a = list[idx];
        int L = job.len(a);
        int N = pow2_at_least(L, 32);
        for (int i = lane; i < N; i += 32) s[i] = i < L ? job.load(a, i) : KEY_PAD;
        __syncwarp();
        warp_bitonic_smem(s, N);
        job.finish(a, s, L);
        __syncwarp();
    }
}

// B2 (shared memory) and B3 (global scratch, gscratch != nullptr)
template <class Job>
__global__ void k_seg_big(Job job, const int32_t* __restrict__ lists,
                          const int32_t* __restrict__ meta, int bucket, uint32_t* gscratch,
                          int64_t cap)
{
    extern __shared__ uint32_t sbuf[];
    uint32_t* s = gscratch ? gscratch + (int64_t)blockIdx.x * cap : sbuf;
    const int32_t* list = lists + meta[bucket];
    int n = meta[SEG_NB + bucket];
    for (int idx = blockIdx.x; idx < n; idx += gridDim.x) {
        int32_t a = list[idx];
        int L = job.len(a);
        int N = pow2_at_least(L, 32);
        for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = i < L ? job.load(a, i) : KEY_PAD;
        __syncthreads();
        block_bitonic(s, N);
        if (threadIdx.x < 32) job.finish(a, s, L);
        __syncthreads();
    }
}

// Builds the bucket lists of a level (device-only; list holds E ids, meta 8
// ints, both caller-allocated).
// Also adds sum |e|(|e|-1) over the level's hyperedges to *w2 (device).
Status seg_classify(const int64_t* hoff, int32_t E, int32_t maxlen, SegBuckets& b, Arena& ar,
                    cudaStream_t s, int64_t* w2);

// Grid sizes for the four bucket kernels.
inline int seg_grid_small(int32_t E) { return grid_for((int64_t)E * 32, 256, 152 * 16); }
inline int seg_grid_big(int32_t E) { return grid_for(E, 1, 152 * 2); }

template <class Job>
Status seg_run(const Job& job, const SegBuckets& b, int32_t E, Arena& ar, cudaStream_t s)
{
    if (E <= 0) return Status{};
    SNN_L k_seg_t<Job><<<grid_for(E, 256, 152 * 16), 256, 0, s>>>(job, b.list, b.meta);
    SNN_CUDA(cudaGetLastError());
    SNN_L k_seg_b0<Job><<<seg_grid_small(E), 256, 0, s>>>(job, b.list, b.meta);
    SNN_CUDA(cudaGetLastError());
    SNN_L k_seg_b1<Job><<<seg_grid_small(E), 256, 0, s>>>(job, b.list, b.meta);
    SNN_CUDA(cudaGetLastError());
    {
        size_t smem = SEG_B2_CAP * sizeof(uint32_t);
        SNN_CUDA(cudaFuncSetAttribute(k_seg_big<Job>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        SNN_L k_seg_big<Job><<<seg_grid_big(E), SEG_B2_THREADS, smem, s>>>(job, b.list, b.meta,
                                                                            SEG_BB2, nullptr, 0);
        SNN_CUDA(cudaGetLastError());
    }
    if (b.b3_cap > 0) {
        uint32_t* g = nullptr;
        SNN_TRY(ar.alloc(&g, (int64_t)SEG_B3_BLOCKS * b.b3_cap));
        SNN_L k_seg_big<Job><<<SEG_B3_BLOCKS, SEG_B3_THREADS, 0, s>>>(job, b.list, b.meta, SEG_BB3,
                                                                       g, b.b3_cap);
        SNN_CUDA(cudaGetLastError());
    }
    return Status{};
}

}  // namespace snn
