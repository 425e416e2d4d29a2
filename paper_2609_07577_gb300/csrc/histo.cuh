// Open-addressing integer histograms keyed by a vertex or partition id, used
// per vertex by the neighbour histogram (coarsening) and the partition
// connection histogram (refinement gains).
#pragma once
#include "common.cuh"

namespace snn {

// (s1, m1) beats (s2, m2): larger value, ties to the lower id; id < 0 = none
__device__ __forceinline__ bool better(int64_t s1, int32_t m1, int64_t s2, int32_t m2)
{
    if (m1 < 0) return false;
    if (m2 < 0) return true;
    return s1 > s2 || (s1 == s2 && m1 < m2);
}

// Table slots: key (-1 empty), summed weight, summed shared-inbound count;
// `used` lists occupied slots in insertion order.
template <typename S>
struct Table {
    int32_t* key;
    S* sc;
    uint32_t* ov;
    int32_t* used;
    int32_t* nfill;
    uint32_t mask;   // capacity - 1

    // returns false if the table is full
    __device__ __forceinline__ bool add(int32_t m, S w, uint32_t o) const
    {
        uint32_t slot = hash32((uint32_t)m) & mask;
        for (uint32_t probe = 0; probe <= mask; probe++) {
            int32_t k = *(volatile int32_t*)&key[slot];
            if (k == -1) {
                int32_t prev = atomicCAS(&key[slot], -1, m);
                if (prev == -1) {
                    int32_t u = atomicAdd(nfill, 1);
                    if ((uint32_t)u <= mask) used[u] = (int32_t)slot;
                    k = m;
                } else {
                    k = prev;
                }
            }
            if (k == m) {
                atomicAdd(&sc[slot], w);
                if (o) atomicAdd(&ov[slot], o);
                return true;
            }
            slot = (slot + 1) & mask;
        }
        return false;
    }
};

// One incidence's segment: elements [b, b+len) of some per-hyperedge array,
// with the hyperedge's weight w, multiplicity k, whether the visiting vertex
// is a destination (nd), and the hyperedge's selfdst flag (sd).
template <typename S>
struct Seg {
    int64_t b;
    int32_t len;
    S w;
    uint32_t k;
    int nd, sd;
};

// Visits, with one warp, the elements of the segments of incidences
// [i0, ve) of a vertex, 32 incidences at a time taken every `stride`. The
// segments of a chunk are flattened into one range so that all 32 lanes
// work on consecutive elements. V::seg(i) gives incidence i's segment;
// V::elem(seg, off) handles element `off` of it and returns false if the
// table is full. Returns false as soon as an element fails or the table
// holds more than `limit` keys (checked once per chunk).
template <typename S, class Vis>
__device__ bool warp_flat_visit(Vis& vis, int64_t i0, int64_t ve, int64_t stride,
                                const int32_t* nfill, int32_t limit)
{
    int lane = threadIdx.x & 31;
    for (int64_t ib = i0; ib < ve; ib += stride) {
        int64_t i = ib + lane;
        Seg<S> sg{0, 0, 0, 0, 0, 0};
        if (i < ve) sg = vis.seg(i);
        int32_t pre = sg.len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t2 = __shfl_up_sync(FULL, pre, o);
            if (lane >= o) pre += t2;
        }
        int32_t total = __shfl_sync(FULL, pre, 31);
        pre -= sg.len;
        bool ok = true;
        for (int32_t vbase = 0; vbase < total; vbase += 32) {
            int32_t v = vbase + lane;
            int32_t lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                int32_t c = lo + step;
                int32_t pc = __shfl_sync(FULL, pre, c & 31);
                if (c < 32 && pc <= v) lo = c;
            }
            Seg<S> t;
            t.b = __shfl_sync(FULL, sg.b, lo);
            t.len = __shfl_sync(FULL, sg.len, lo);
            t.w = __shfl_sync(FULL, sg.w, lo);
            t.k = __shfl_sync(FULL, sg.k, lo);
            t.nd = __shfl_sync(FULL, sg.nd, lo);
            t.sd = __shfl_sync(FULL, sg.sd, lo);
            int32_t pt = __shfl_sync(FULL, pre, lo);
            if (v < total) {
                if (!vis.elem(t, v - pt)) ok = false;
            }
        }
        __syncwarp();
        if (!__all_sync(FULL, ok) || *(volatile const int32_t*)nfill > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void warp_argmax(int64_t& bs, int32_t& bm, uint32_t& bo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int64_t s2 = __shfl_xor_sync(FULL, bs, o);
        int32_t m2 = __shfl_xor_sync(FULL, bm, o);
        uint32_t o2 = __shfl_xor_sync(FULL, bo, o);
        if (better(s2, m2, bs, bm)) {
            bs = s2;
            bm = m2;
            bo = o2;
        }
    }
}

// table carving: a warp slice or a block table from raw memory
template <typename S>
__device__ __forceinline__ Table<S> carve_table(unsigned char* base, int32_t cap, int32_t* nfill)
{
    Table<S> t;
    t.key = (int32_t*)base;
    t.sc = (S*)(base + (size_t)cap * sizeof(int32_t));
    t.ov = (uint32_t*)(base + (size_t)cap * (sizeof(int32_t) + sizeof(S)));
    t.used = (int32_t*)(base + (size_t)cap * (2 * sizeof(int32_t) + sizeof(S)));
    t.nfill = nfill;
    t.mask = (uint32_t)(cap - 1);
    return t;
}

template <typename S>
__host__ __device__ constexpr size_t table_bytes(int64_t cap)
{
    return (size_t)cap * (3 * sizeof(int32_t) + sizeof(S));
}

}  // namespace snn

namespace snn {

template <typename S>
__global__ void k_init_tables(unsigned char* g, int blocks, int64_t cap)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < blocks * cap;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = i / cap, j = i - b * cap;
        Table<S> t = carve_table<S>(g + (size_t)b * table_bytes<S>(cap), (int32_t)cap, nullptr);
        t.key[j] = -1;
        t.sc[j] = 0;
        t.ov[j] = 0;
    }
}

// global-memory tables for the block tier: key -1, sums 0
template <typename S>
inline Status init_global_tables(unsigned char* g, int blocks, int64_t cap, cudaStream_t s)
{
    SNN_L k_init_tables<S><<<grid_for(blocks * cap, 256), 256, 0, s>>>(g, blocks, cap);
    SNN_CUDA(cudaGetLastError());
    return Status{};
}

}  // namespace snn
