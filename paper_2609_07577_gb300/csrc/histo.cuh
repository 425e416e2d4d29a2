// Per-vertex integer histograms keyed by a vertex id (coarsening: score and
// shared inbound count per neighbour) or a partition id (refinement:
// connection weight and inbound overlap per adjacent partition), followed by
// an argmax over the keys. Sums are integer atomics, so results do not
// depend on the order of updates.
//
// Vertices are first binned by their work (total length of the segments
// their incidences contribute), which bounds their number of distinct keys:
//   warp tier   work <= 3/4 of a 512-slot table: one warp, shared memory;
//               cannot overflow.
//   block tier  work <= 2^16: one 256-thread block, 2048-slot shared table;
//               a vertex with more than 1536 distinct keys is handed on.
//   big tier    work <= 2^22 or hand-overs: one 512-thread block per SM with
//               a 16384-slot shared table; overflow is handed on.
//   split tier  the rest: the incidences are cut into items of about 16384
//               elements processed by warps all over the GPU, all adding into
//               one global-memory table per vertex sized to twice its bound
//               of distinct keys (so it cannot overflow); one block per
//               vertex then reduces the table.
// Every tier visits a chunk of 32 incidences at a time with their segments
// flattened into one range, so all 32 lanes load consecutive elements even
// when segments are short.
//
// A Policy supplies:
//   typedef S (score type), struct Acc (per-thread sums, with add(Acc) and
//   __device__ Acc reduce over a warp)
//   int32_t V (vertices), key space bound `keys`
//   static constexpr bool kOptimistic               try the warp tier even when the
//                                                   bound exceeds its table (few keys expected)
//   __device__ bool skip(n)                         n needs no histogram (result
//                                                   written by write(n, 0, -1, 0, Acc()))
//   __device__ int64_t seg_len(int64_t i)           segment length of incidence i
//   __device__ int64_t vb(n), ve(n)                 incidence range of vertex n
//   __device__ Seg<S> seg(int64_t i, Acc&)          segment of incidence i
//   __device__ bool elem(n, const Seg<S>&, off, const Table<S>&, Acc&)
//   __device__ void consider(n, key, int64 sc, uint32 ov, const Acc& total,
//                            int64_t& best, int32_t& bkey, uint32_t& bov)
//   __device__ void write(n, best, bkey, bov, const Acc& total)
#pragma once
#include "common.cuh"
#include "histo_tiers.cuh"

#include <algorithm>
#include <type_traits>

namespace snn {

// (s1, m1) beats (s2, m2): larger value, ties to the lower id; id < 0 = none
__device__ __forceinline__ bool better(int64_t s1, int32_t m1, int64_t s2, int32_t m2)
{
    if (m1 < 0) return false;
    if (m2 < 0) return true;
    return s1 > s2 || (s1 == s2 && m1 < m2);
}

// Open-addressing slots: key (-1 empty), summed weight, summed overlap.
template <typename S>
struct Table {
    int32_t* key;
    S* sc;
    uint32_t* ov;
    uint32_t mask;     // capacity - 1
    uint32_t probes;   // probe limit of add()

    // returns false if m finds no slot within the probe limit (tables that
    // must never fail use the full capacity as the limit)
    __device__ __forceinline__ bool add(int32_t m, S w, uint32_t o) const
    {
        return try_add(m, w, o, probes);
    }

    // returns false if m has no slot within the first max_probes probed
    __device__ __forceinline__ bool try_add(int32_t m, S w, uint32_t o, uint32_t max_probes) const
    {
        uint32_t slot = hash32((uint32_t)m) & mask;
        for (uint32_t probe = 0; probe < max_probes; probe++) {
            int32_t k = *(volatile int32_t*)&key[slot];
            if (k == -1) {
                int32_t prev = atomicCAS(&key[slot], -1, m);
                k = prev == -1 ? m : prev;
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

template <typename S>
__host__ __device__ constexpr size_t slot_bytes()
{
    return 2 * sizeof(int32_t) + sizeof(S);
}

template <typename S>
__device__ __forceinline__ Table<S> carve_table(unsigned char* base, int64_t cap)
{
    Table<S> t;
    t.key = (int32_t*)base;
    t.sc = (S*)(base + (size_t)cap * sizeof(int32_t));
    t.ov = (uint32_t*)(base + (size_t)cap * (sizeof(int32_t) + sizeof(S)));
    t.mask = (uint32_t)(cap - 1);
    t.probes = (uint32_t)cap;
    return t;
}

// One incidence's segment: elements [b, b+len) of a per-hyperedge array,
// with the hyperedge's weight w, multiplicity k, whether the visiting vertex
// is one of its destinations (nd) and its selfdst flag (sd).
template <typename S>
struct Seg {
    int64_t b;
    int32_t len;
    S w;
    uint32_t k;
    int nd, sd;
};

// One warp visits incidences [i0, ve) of vertex n, 32 at a time every
// `stride`, flattening their segments. Returns false if an insert failed.
template <typename S, class Pol, class Tb>
__device__ bool warp_visit(const Pol& pol, int32_t n, int64_t i0, int64_t ve, int64_t stride,
                           const Tb& t, typename Pol::Acc& acc)
{
    int lane = threadIdx.x & 31;
    bool ok = true;
    for (int64_t ib = i0; ib < ve; ib += stride) {
        int64_t i = ib + lane;
        Seg<S> sg{0, 0, 0, 0, 0, 0};
        if (i < ve) sg = pol.seg(i, acc);
        int32_t pre = sg.len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t2 = __shfl_up_sync(FULL, pre, o);
            if (lane >= o) pre += t2;
        }
        int32_t total = __shfl_sync(FULL, pre, 31);
        pre -= sg.len;
        for (int32_t vbase = 0; vbase < total; vbase += 32) {
            int32_t v = vbase + lane;
            int32_t lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                int32_t c = lo + step;
                int32_t pc = __shfl_sync(FULL, pre, c & 31);
                if (c < 32 && pc <= v) lo = c;
            }
            Seg<S> g;
            g.b = __shfl_sync(FULL, sg.b, lo);
            g.len = __shfl_sync(FULL, sg.len, lo);
            g.w = __shfl_sync(FULL, sg.w, lo);
            g.k = __shfl_sync(FULL, sg.k, lo);
            g.nd = __shfl_sync(FULL, sg.nd, lo);
            g.sd = __shfl_sync(FULL, sg.sd, lo);
            int32_t pt = __shfl_sync(FULL, pre, lo);
            if (v < total && !pol.elem(n, g, v - pt, t, acc)) ok = false;
        }
    }
    return __all_sync(FULL, ok);
}

template <typename S>
__device__ __forceinline__ void clear_slots(const Table<S>& t, int64_t from, int64_t to,
                                            int64_t stride)
{
    for (int64_t i = from; i < to; i += stride) {
        t.key[i] = -1;
        t.sc[i] = 0;
        t.ov[i] = 0;
    }
}

// best over slots [from, to) by `stride`, resetting them
template <typename S, class Pol>
__device__ void scan_slots(const Pol& pol, int32_t n, const Table<S>& t, int64_t from, int64_t to,
                           int64_t stride, const typename Pol::Acc& tot, int64_t& bs, int32_t& bk,
                           uint32_t& bo)
{
    for (int64_t i = from; i < to; i += stride) {
        int32_t k = t.key[i];
        if (k < 0) continue;
        int64_t s = (int64_t)t.sc[i];
        uint32_t o = t.ov[i];
        t.key[i] = -1;
        t.sc[i] = 0;
        t.ov[i] = 0;
        pol.consider(n, k, s, o, tot, bs, bk, bo);
    }
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

constexpr int HT_WARPS = 8;
constexpr int HT_WCAP = 512;            // warp table slots
constexpr int HT_WLOAD = HT_WCAP * 3 / 4;
constexpr int HT_BTHREADS = 256;
constexpr int HT_BCAP = 2048;           // block table slots
constexpr int HT_GTHREADS = 512;        // big-block tier
constexpr int64_t HT_CHUNK = 1024;      // incidences per split-tier work item
enum : int { HT_TIER_WARP = 0, HT_TIER_BLOCK = 1, HT_TIER_BIG = 2, HT_TIER_SPLIT = 3, HT_NTIER = 4 };
// counters of run_histogram: per-tier vertex counts, then the summed work and
// the number of vertices given a histogram (not skipped)
// and the next list positions the block and big tiers hand out (dynamic
// scheduling: a block takes the next vertex when it is done with one)
enum : int {
    HT_CNT_WORK = HT_NTIER, HT_CNT_VERTS = HT_NTIER + 1, HT_CNT_NEXT = HT_NTIER + 2,
    HT_NCNT = HT_NTIER + 2 + HT_NTIER
};

template <typename S>
__host__ __device__ constexpr int big_cap()
{
    return sizeof(S) == 4 ? 16384 : 8192;
}

__host__ __device__ inline int64_t pow2_ceil(int64_t x)
{
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Work of each vertex: total segment length over its incidences, or -1 when
// the policy decides it without a histogram. One thread per vertex tests
// skip() and lists the vertices to count (warp-aggregated appends); then one
// warp per listed vertex sums its segments. Rounds that evaluate few
// vertices pay a thread, not a warp, per skipped vertex, while full passes
// keep a warp per vertex.
template <class Pol>
__global__ void __launch_bounds__(256) k_ht_skip(Pol pol, int64_t* work, int32_t* todo, int32_t* ntodo)
{
    int lane = threadIdx.x & 31;
    unsigned lt = lanemask_lt();
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < pol.V;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t n = base + threadIdx.x;
        bool count = false;
        if (n < pol.V) {
            if (pol.skip((int32_t)n)) work[n] = -1;
            else count = true;
        }
        unsigned m = __ballot_sync(FULL, count);
        if (!m) continue;
        int leader = __ffs(m) - 1;
        int32_t pos = 0;
        if (lane == leader) pos = atomicAdd(ntodo, __popc(m));
        pos = __shfl_sync(FULL, pos, leader);
        if (count) todo[pos + __popc(m & lt)] = (int32_t)n;
    }
}

template <class Pol>
__global__ void __launch_bounds__(256)
    k_ht_work(Pol pol, int64_t* work, const int32_t* __restrict__ todo, const int32_t* __restrict__ ntodo)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t nt = *ntodo;
    for (int64_t idx = gw; idx < nt; idx += nw) {
        int32_t n = todo[idx];
        int64_t w = 0;
        for (int64_t i = pol.vb(n) + lane; i < pol.ve(n); i += 32) w += pol.seg_len(i);
        w = warp_sum(w);
        if (lane == 0) work[n] = w;
    }
}

// lists: tier t's vertices at lists + t*V; cnt[t] their number; the split
// tier also records each vertex's table capacity
template <class Pol>
__device__ __forceinline__ void ht_push(const Pol& pol, int tier, int32_t n, int64_t work,
                                        int32_t* lists, int64_t* cnt, int64_t* scap)
{
    int64_t p = (int64_t)atomicAdd((unsigned long long*)&cnt[tier], 1ull);
    lists[(int64_t)tier * pol.V + p] = n;
    if (tier == HT_TIER_SPLIT) {
        int64_t bound = work < pol.keys ? work : pol.keys;
        scap[p] = pow2_ceil(2 * (bound > 16 ? bound : 16));
    }
}

template <class Pol>
__global__ void __launch_bounds__(256)
    k_ht_classify(Pol pol, const int64_t* __restrict__ workv, int32_t* lists, int64_t* cnt,
                  int64_t* scap, HtTiers tiers)
{
    int lane = threadIdx.x & 31;
    unsigned lt = lanemask_lt();
    int64_t wsum = 0, vsum = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < pol.V;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t n = base + threadIdx.x;
        int tier = -1;
        int64_t work = 0;
        if (n < pol.V) {
            work = workv[n];
            if (work <= 0) {
                // skipped, or nothing to count: the empty table's result
                // (no key, zero sums) without a histogram
                pol.write((int32_t)n, 0, -1, 0, typename Pol::Acc());
            } else {
                wsum += work;
                vsum++;
                int64_t bound = work < pol.keys ? work : pol.keys;
                if (bound <= HT_WLOAD) tier = work <= tiers.wwork ? HT_TIER_WARP : HT_TIER_SPLIT;
                else if (Pol::kOptimistic && work <= tiers.wwork) tier = HT_TIER_WARP;
                else if (work <= tiers.bwork) tier = HT_TIER_BLOCK;
                else if (work <= tiers.gwork) tier = HT_TIER_BIG;
                else tier = HT_TIER_SPLIT;
            }
        }
        for (int t = 0; t < HT_NTIER; t++) {
            unsigned m = __ballot_sync(FULL, tier == t);
            if (!m) continue;
            int leader = __ffs(m) - 1;
            int64_t pos = 0;
            if (lane == leader) pos = (int64_t)atomicAdd((unsigned long long*)&cnt[t], (unsigned long long)__popc(m));
            pos = __shfl_sync(FULL, pos, leader);
            if (tier == t) {
                int64_t p = pos + __popc(m & lt);
                lists[(int64_t)t * pol.V + p] = (int32_t)n;
                if (t == HT_TIER_SPLIT) {
                    int64_t bound = work < pol.keys ? work : pol.keys;
                    scap[p] = pow2_ceil(2 * (bound > 16 ? bound : 16));
                }
            }
        }
    }
    wsum = warp_sum(wsum);
    vsum = warp_sum(vsum);
    if (lane == 0 && vsum) {
        atomicAdd((unsigned long long*)&cnt[HT_CNT_WORK], (unsigned long long)wsum);
        atomicAdd((unsigned long long*)&cnt[HT_CNT_VERTS], (unsigned long long)vsum);
    }
}

template <class Pol>
__global__ void __launch_bounds__(HT_WARPS * 32)
    k_ht_warp(Pol pol, int32_t* lists, int64_t* cnt, const int64_t* __restrict__ workv,
              int64_t* scap)
{
    using S = typename Pol::S;
    using Acc = typename Pol::Acc;
    extern __shared__ __align__(16) unsigned char ht_dyn[];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t* list = lists + (int64_t)HT_TIER_WARP * pol.V;
    int64_t nl = cnt[HT_TIER_WARP];
    int64_t gw = blockIdx.x * (int64_t)HT_WARPS + warp, nw = (int64_t)gridDim.x * HT_WARPS;
    Table<S> full = carve_table<S>(ht_dyn + (size_t)warp * HT_WCAP * slot_bytes<S>(), HT_WCAP);
    clear_slots(full, lane, HT_WCAP, 32);
    __syncwarp();
    for (int64_t idx = gw; idx < nl; idx += nw) {
        int32_t n = list[idx];
        int64_t vb = pol.vb(n), ve = pol.ve(n);
        Acc acc;
        int64_t work = workv[n];
        int64_t bound = work < pol.keys ? work : pol.keys;
        int64_t cap = pow2_ceil(2 * (bound > 8 ? bound : 8));
        if (cap > HT_WCAP) cap = HT_WCAP;
        Table<S> t = full;
        t.mask = (uint32_t)(cap - 1);
        // a vertex whose bound fits the table cannot overflow it; others
        // (policies that expect few keys) try it and move on if it fills
        bool sure = bound <= HT_WLOAD;
        t.probes = sure ? (uint32_t)cap : 32u;
        bool ok = warp_visit<S>(pol, n, vb, ve, 32, t, acc);
        __syncwarp();
        if (!ok) {
            clear_slots(t, lane, cap, 32);
            if (lane == 0) ht_push(pol, HT_TIER_BLOCK, n, work, lists, cnt, scap);
            __syncwarp();
            continue;
        }
        Acc tot = Pol::warp_reduce(acc);
        int64_t bs = 0;
        int32_t bk = -1;
        uint32_t bo = 0;
        scan_slots<S>(pol, n, t, lane, cap, 32, tot, bs, bk, bo);
        warp_argmax(bs, bk, bo);
        if (lane == 0) pol.write(n, bs, bk, bo, tot);
        __syncwarp();
    }
}

// A policy may split elem into load (the element's global reads, giving an
// Item) and put (the table update), declaring `struct Item`; the block tiers
// then keep several elements' loads in flight per thread.
template <class P, class = void>
struct has_item : std::false_type {};
template <class P>
struct has_item<P, std::void_t<typename P::Item>> : std::true_type {};

// the last index lo in [from, n) with spre[lo] <= v (spre non-decreasing,
// spre[from] <= v): one probe while v stays in the same segment, a binary
// search when it moved on
__device__ __forceinline__ int32_t seg_find(const int32_t* spre, int32_t n, int32_t from, int32_t v)
{
    if (from + 1 >= n || spre[from + 1] > v) return from;
    int32_t lo = from + 1, hi = n - 1;
    while (lo < hi) {
        int32_t mid = (lo + hi + 1) >> 1;
        if (spre[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Block-wide visit of incidences [vb, ve): tiles of blockDim incidences, one
// per thread, segment lengths scanned across the block, then every thread
// takes elements v = tid, tid + blockDim, ... of the tile's flattened range
// and finds its segment in shared memory (the elements of a thread are
// increasing, so its search resumes where the previous one ended).
template <typename S, class Pol, int T>
__device__ bool block_visit(const Pol& pol, int32_t n, int64_t vb, int64_t ve, const Table<S>& t,
                            typename Pol::Acc& acc, Seg<S>* sseg, int32_t* spre, int32_t* swarp,
                            int* sfail)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = T / 32;
    bool ok = true;
    for (int64_t tile = vb; tile < ve; tile += T) {
        int64_t i = tile + threadIdx.x;
        Seg<S> sg{0, 0, 0, 0, 0, 0};
        if (i < ve) sg = pol.seg(i, acc);
        int32_t inc = sg.len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t2 = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += t2;
        }
        if (lane == 31) swarp[warp] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t run = 0;
            for (int w = 0; w < nw; w++) {
                int32_t c = swarp[w];
                swarp[w] = run;
                run += c;
            }
            swarp[nw] = run;
        }
        __syncthreads();
        spre[threadIdx.x] = swarp[warp] + inc - sg.len;
        sseg[threadIdx.x] = sg;
        int32_t total = swarp[nw];
        __syncthreads();
        int32_t lo = 0;
        if constexpr (has_item<Pol>::value) {
            constexpr int U = 4;
            for (int32_t v0 = threadIdx.x; v0 < total && ok; v0 += U * T) {
                typename Pol::Item it[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    int32_t v = v0 + u * T;
                    if (v < total) {
                        lo = seg_find(spre, T, lo, v);
                        it[u] = pol.load(n, sseg[lo], v - spre[lo]);
                    } else {
                        it[u] = Pol::none();
                    }
                }
#pragma unroll
                for (int u = 0; u < U; u++) ok = pol.put(n, it[u], t, acc) && ok;
            }
        } else {
            for (int32_t v = threadIdx.x; v < total; v += T) {
                lo = seg_find(spre, T, lo, v);
                if (!pol.elem(n, sseg[lo], v - spre[lo], t, acc)) {
                    ok = false;
                    break;
                }
            }
        }
        if (!ok) *sfail = 1;
        __syncthreads();
        if (*sfail) break;
    }
    return *sfail == 0;
}

// Block (T threads) per vertex with a CAP-slot shared table; vertices whose
// keys do not fit are pushed to tier `next`.
template <class Pol, int T, int CAP, int TIER, int NEXT>
__global__ void __launch_bounds__(T)
    k_ht_block(Pol pol, int32_t* lists, int64_t* cnt, int64_t* scap, const int64_t* __restrict__ workv)
{
    using S = typename Pol::S;
    using Acc = typename Pol::Acc;
    extern __shared__ __align__(16) unsigned char ht_dyn[];
    __shared__ __align__(16) unsigned char sseg_raw[sizeof(Seg<S>) * T];
    __shared__ int32_t spre[T];
    __shared__ int32_t swarp[T / 32 + 1];
    __shared__ int sfail;
    __shared__ __align__(16) unsigned char wacc_raw[sizeof(Acc) * (T / 32)];
    __shared__ int64_t rs[T / 32];
    __shared__ int32_t rk[T / 32];
    __shared__ uint32_t ro[T / 32];
    Seg<S>* sseg = (Seg<S>*)sseg_raw;
    Acc* wacc = (Acc*)wacc_raw;
    const int nwarps = T / 32;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Table<S> t = carve_table<S>(ht_dyn, CAP);
    t.probes = 64;   // a vertex that clusters the table this much moves on
    clear_slots(t, threadIdx.x, CAP, T);
    const int32_t* list = lists + (int64_t)TIER * pol.V;
    int64_t nl = cnt[TIER];
    __shared__ int64_t snext;
    for (;;) {
        if (threadIdx.x == 0) {
            snext = (int64_t)atomicAdd((unsigned long long*)&cnt[HT_CNT_NEXT + TIER], 1ull);
            sfail = 0;
        }
        __syncthreads();
        int64_t idx = snext;
        if (idx >= nl) break;
        int32_t n = list[idx];
        int64_t vb = pol.vb(n), ve = pol.ve(n);
        Acc acc;
        bool ok = block_visit<S, Pol, T>(pol, n, vb, ve, t, acc, sseg, spre, swarp, &sfail);
        Acc wa = Pol::warp_reduce(acc);
        if (lane == 0) wacc[warp] = wa;
        __syncthreads();
        if (!ok) {
            clear_slots(t, threadIdx.x, CAP, T);
            if (threadIdx.x == 0) ht_push(pol, NEXT, n, workv[n], lists, cnt, scap);
            __syncthreads();
            continue;
        }
        Acc tot = wacc[0];
        for (int w = 1; w < nwarps; w++) tot.add(wacc[w]);
        int64_t bs = 0;
        int32_t bk = -1;
        uint32_t bo = 0;
        scan_slots<S>(pol, n, t, threadIdx.x, CAP, T, tot, bs, bk, bo);
        warp_argmax(bs, bk, bo);
        if (lane == 0) {
            rs[warp] = bs;
            rk[warp] = bk;
            ro[warp] = bo;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nwarps; w++)
                if (better(rs[w], rk[w], bs, bk)) {
                    bs = rs[w];
                    bk = rk[w];
                    bo = ro[w];
                }
            pol.write(n, bs, bk, bo, tot);
        }
        __syncthreads();
    }
}

// Split tier. The incidences of the split vertices are laid out flat
// (vertex j owns flat positions [od[j], od[j+1])) and cut into work items of
// about `item` elements: an item starts at a vertex's first incidence or
// where the running element count crosses a multiple of `item`. The item
// size is chosen so that the items outnumber the resident warps.

__device__ __forceinline__ int64_t find_owner(const int64_t* od, int64_t ns, int64_t f)
{
    int64_t lo = 0, hi = ns - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (od[mid] <= f) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// degree, table capacity (twice the key bound, at most twice `limit` when
// limit > 0) and total work of the split vertices
template <class Pol>
__global__ void k_ht_split_deg(Pol pol, const int32_t* __restrict__ slist, int64_t ns, int64_t* deg,
                               const int64_t* __restrict__ workv, int64_t* total_work,
                               int64_t* scap, int64_t limit)
{
    int64_t w = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ns;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = slist[j];
        deg[j] = pol.ve(n) - pol.vb(n);
        int64_t work = workv[n];
        w += work;
        int64_t bound = work < pol.keys ? work : pol.keys;
        if (limit > 0 && bound > limit) bound = limit;
        scap[j] = pow2_ceil(2 * (bound > 16 ? bound : 16));
    }
    w = warp_sum(w);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd((unsigned long long*)total_work, (unsigned long long)w);
}

template <class Pol>
__global__ void k_ht_split_len(Pol pol, const int32_t* __restrict__ slist, int64_t ns,
                               const int64_t* __restrict__ od, int64_t D, int64_t* len)
{
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < D;
         f += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = find_owner(od, ns, f);
        len[f] = pol.seg_len(pol.vb(slist[j]) + (f - od[j]));
    }
}

static __global__ void k_ht_split_starts(int64_t ns, const int64_t* __restrict__ od, int64_t D,
                                  const int64_t* __restrict__ x, const int64_t* __restrict__ len,
                                  int32_t* start, int64_t item)
{
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < D;
         f += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = find_owner(od, ns, f);
        int64_t base = x[od[j]];
        int s = 0;
        if (f == od[j]) s = 1;
        else {
            int64_t b0 = (x[f - 1] - base) / item, b1 = (x[f] - base) / item;
            s = b1 != b0;
        }
        start[f] = s;
    }
}

static __global__ void k_ht_split_items(int64_t D, const int32_t* __restrict__ start,
                                 const int32_t* __restrict__ pos, int64_t* item_f0)
{
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < D;
         f += (int64_t)gridDim.x * blockDim.x)
        if (start[f]) item_f0[pos[f]] = f;
}

// adds the used slots of a warp-private table into the global table g and
// clears them
template <typename S>
__device__ bool flush_private(const Table<S>& p, int64_t cap, const Table<S>& g)
{
    int lane = threadIdx.x & 31;
    bool ok = true;
    for (int64_t i = lane; i < cap; i += 32) {
        int32_t k = p.key[i];
        if (k < 0) continue;
        if (!g.add(k, p.sc[i], p.ov[i])) ok = false;
        p.key[i] = -1;
        p.sc[i] = 0;
        p.ov[i] = 0;
    }
    __syncwarp();
    return __all_sync(FULL, ok);
}

// Items of vertices with few possible keys (table capacity <= HT_WCAP) are
// counted in a warp-private shared table first and flushed once per item,
// so many warps working for one vertex do not all hit the same few global
// slots; other items add straight into the global table.
template <class Pol>
__global__ void __launch_bounds__(HT_WARPS * 32)
    k_ht_split_visit(Pol pol, const int32_t* __restrict__ slist, int64_t ns,
                     const int64_t* __restrict__ od, int64_t D,
                     const int64_t* __restrict__ item_f0, int64_t nitems,
                     const int64_t* __restrict__ toff, const int64_t* __restrict__ scap,
                     unsigned char* pool, typename Pol::Acc* gacc, int32_t* ovf, uint32_t probes)
{
    using S = typename Pol::S;
    using Acc = typename Pol::Acc;
    extern __shared__ __align__(16) unsigned char ht_dyn[];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Table<S> priv = carve_table<S>(ht_dyn + (size_t)warp * HT_WCAP * slot_bytes<S>(), HT_WCAP);
    clear_slots(priv, lane, HT_WCAP, 32);
    __syncwarp();
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = gw; it < nitems; it += nw) {
        int64_t f0 = item_f0[it];
        int64_t f1 = it + 1 < nitems ? item_f0[it + 1] : D;
        int64_t j = find_owner(od, ns, f0);
        if (f1 > od[j + 1]) f1 = od[j + 1];
        int32_t n = slist[j];
        int64_t vb = pol.vb(n) + (f0 - od[j]);
        int64_t ve = pol.vb(n) + (f1 - od[j]);
        Table<S> g = carve_table<S>(pool + toff[j] * slot_bytes<S>(), scap[j]);
        if (probes) g.probes = probes;
        Acc acc;
        bool ok;
        if (scap[j] <= HT_WCAP) {
            Table<S> p = priv;
            p.mask = (uint32_t)(scap[j] - 1);
            p.probes = (uint32_t)scap[j];
            ok = warp_visit<S>(pol, n, vb, ve, 32, p, acc);
            ok = flush_private(p, scap[j], g) && ok;
        } else {
            ok = warp_visit<S>(pol, n, vb, ve, 32, g, acc);
        }
        if (!ok && lane == 0) ovf[j] = 1;
        Acc wa = Pol::warp_reduce(acc);
        if (lane == 0) wa.atomic_into(&gacc[j]);
    }
}

template <class Pol>
__global__ void __launch_bounds__(1024)
    k_ht_split_scan(Pol pol, const int32_t* __restrict__ slist, int64_t ns,
                    const int64_t* __restrict__ toff, const int64_t* __restrict__ scap,
                    unsigned char* pool, const typename Pol::Acc* gacc,
                    const int32_t* __restrict__ ovf)
{
    using S = typename Pol::S;
    __shared__ int64_t rs[32];
    __shared__ int32_t rk[32];
    __shared__ uint32_t ro[32];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int nwarps = blockDim.x >> 5;
    for (int64_t j = blockIdx.x; j < ns; j += gridDim.x) {
        if (ovf[j]) continue;   // redone with a larger table
        int32_t n = slist[j];
        Table<S> t = carve_table<S>(pool + toff[j] * slot_bytes<S>(), scap[j]);
        typename Pol::Acc tot = gacc[j];
        int64_t bs = 0;
        int32_t bk = -1;
        uint32_t bo = 0;
        scan_slots<S>(pol, n, t, threadIdx.x, scap[j], blockDim.x, tot, bs, bk, bo);
        warp_argmax(bs, bk, bo);
        if (lane == 0) {
            rs[warp] = bs;
            rk[warp] = bk;
            ro[warp] = bo;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nwarps; w++)
                if (better(rs[w], rk[w], bs, bk)) {
                    bs = rs[w];
                    bk = rk[w];
                    bo = ro[w];
                }
            pol.write(n, bs, bk, bo, tot);
        }
        __syncthreads();
    }
}

static __global__ void k_ht_collect_ovf(const int32_t* __restrict__ slist, int64_t ns,
                                        const int32_t* __restrict__ ovf, int32_t* out, int64_t* cnt)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ns;
         j += (int64_t)gridDim.x * blockDim.x)
        if (ovf[j]) out[atomicAdd((unsigned long long*)cnt, 1ull)] = slist[j];
}

template <typename S>
__global__ void k_ht_pool_clear(unsigned char* pool, const int64_t* __restrict__ toff,
                                const int64_t* __restrict__ scap, int64_t ns)
{
    for (int64_t j = blockIdx.x; j < ns; j += gridDim.x) {
        Table<S> t = carve_table<S>(pool + toff[j] * slot_bytes<S>(), scap[j]);
        clear_slots(t, threadIdx.x, scap[j], blockDim.x);
    }
}

template <typename K>
inline Status set_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024)
        SNN_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return Status{};
}

constexpr int64_t HT_SPLIT_CAP = 1 << 16;

// Split tier for the vertices slist[0..ns). limit > 0 caps the tables and
// appends the vertices that overflowed to `again` at the device counter
// *nagain (the caller clears it; h_cnt[0] receives its new value);
// limit == 0 sizes every table to its exact bound, which cannot overflow.
template <class Pol>
Status run_split(const Pol& pol, Arena& ar, cudaStream_t s, const int32_t* sl, int64_t ns,
                 const int64_t* workv, int64_t limit, int32_t* again, int64_t* nagain,
                 int64_t* h_cnt)
{
    using S = typename Pol::S;
    int64_t *toff, *deg, *od, *tot, *scap;
    int32_t* ovf;
    SNN_TRY(ar.alloc(&toff, ns + 1));
    SNN_TRY(ar.alloc(&deg, ns));
    SNN_TRY(ar.alloc(&od, ns + 1));
    SNN_TRY(ar.alloc(&tot, 4));
    SNN_TRY(ar.alloc(&scap, ns));
    SNN_TRY(ar.alloc(&ovf, ns));
    SNN_CUDA(cudaMemsetAsync(tot, 0, 4 * sizeof(int64_t), s));
    SNN_CUDA(cudaMemsetAsync(ovf, 0, (size_t)ns * sizeof(int32_t), s));
    SNN_L k_ht_split_deg<Pol><<<grid_for(ns, 256), 256, 0, s>>>(pol, sl, ns, deg, workv, tot + 2, scap,
                                                              limit);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(scan_exclusive_i64(scap, toff, ns, tot, ar, s));
    SNN_TRY(scan_exclusive_i64(deg, od, ns, od + ns, ar, s));
    SNN_CUDA(cudaMemcpyAsync(h_cnt, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaMemcpyAsync(h_cnt + 1, od + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaMemcpyAsync(h_cnt + 2, tot + 2, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    int64_t slots = h_cnt[0], D = h_cnt[1];
    int64_t item = pow2_ceil(h_cnt[2] / (152 * 64 * 2) + 1);
    item = item < 1024 ? 1024 : (item > 16384 ? 16384 : item);
    int64_t *len, *x, *item_f0;
    int32_t *start, *pos;
    SNN_TRY(ar.alloc(&len, D));
    SNN_TRY(ar.alloc(&x, D));
    SNN_TRY(ar.alloc(&start, D));
    SNN_TRY(ar.alloc(&pos, D));
    SNN_TRY(ar.alloc(&item_f0, D));
    SNN_L k_ht_split_len<Pol><<<grid_for(D, 256), 256, 0, s>>>(pol, sl, ns, od, D, len);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(scan_exclusive_i64(len, x, D, nullptr, ar, s));
    SNN_L k_ht_split_starts<<<grid_for(D, 256), 256, 0, s>>>(ns, od, D, x, len, start, item);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(scan_exclusive_i32(start, pos, D, (int32_t*)(tot + 1), ar, s));
    SNN_L k_ht_split_items<<<grid_for(D, 256), 256, 0, s>>>(D, start, pos, item_f0);
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaMemcpyAsync(h_cnt, tot + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    int64_t items = h_cnt[0];
    unsigned char* pool;
    typename Pol::Acc* gacc;
    SNN_TRY(ar.alloc(&pool, slots * (int64_t)slot_bytes<S>()));
    SNN_TRY(ar.alloc(&gacc, ns));
    SNN_CUDA(cudaMemsetAsync(gacc, 0, (size_t)ns * sizeof(typename Pol::Acc), s));
    SNN_L k_ht_pool_clear<S><<<(int)std::min<int64_t>(ns, 152 * 8), 256, 0, s>>>(pool, toff, scap, ns);
    SNN_CUDA(cudaGetLastError());
    size_t wsm = (size_t)HT_WARPS * HT_WCAP * slot_bytes<S>();
    SNN_TRY(set_smem(k_ht_split_visit<Pol>, wsm));
    SNN_L k_ht_split_visit<Pol><<<(int)std::min<int64_t>(ceil_div(items, HT_WARPS), 152 * 8),
                                  HT_WARPS * 32, wsm, s>>>(pol, sl, ns, od, D, item_f0, items, toff,
                                                           scap, pool, gacc, ovf,
                                                           limit > 0 ? 256u : 0u);
    SNN_CUDA(cudaGetLastError());
    SNN_L k_ht_split_scan<Pol><<<(int)std::min<int64_t>(ns, 152 * 4), 1024, 0, s>>>(pol, sl, ns, toff,
                                                                                    scap, pool, gacc, ovf);
    SNN_CUDA(cudaGetLastError());
    if (limit > 0) {
        SNN_L k_ht_collect_ovf<<<grid_for(ns, 256), 256, 0, s>>>(sl, ns, ovf, again, nagain);
        SNN_CUDA(cudaGetLastError());
        SNN_CUDA(cudaMemcpyAsync(h_cnt, nagain, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SNN_CUDA(cudaStreamSynchronize(s));
    }
    return Status{};
}

// table capacity of each split-tier vertex (as k_ht_split_deg sizes it)
template <class Pol>
__global__ void k_ht_split_caps(Pol pol, const int32_t* __restrict__ slist, int64_t ns,
                                const int64_t* __restrict__ workv, int64_t limit, int64_t* caps)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ns;
         j += (int64_t)gridDim.x * blockDim.x) {
        int64_t work = workv[slist[j]];
        int64_t bound = work < pol.keys ? work : pol.keys;
        if (limit > 0 && bound > limit) bound = limit;
        caps[j] = pow2_ceil(2 * (bound > 16 ? bound : 16));
    }
}

// cuts[c] .. cuts[c+1]: consecutive runs of slist whose tables hold at most
// pool_slots slots together (a single larger vertex forms its own run)
template <class Pol>
Status split_cuts(const Pol& pol, Arena& ar, cudaStream_t s, const int32_t* sl, int64_t ns,
                  const int64_t* workv, int64_t limit, int64_t pool_slots,
                  std::vector<int64_t>& cuts)
{
    cuts.assign(1, 0);
    if (ns <= 0) return Status{};
    Arena::Mark m = ar.mark();
    int64_t *caps, *pre;
    SNN_TRY(ar.alloc(&caps, ns));
    SNN_TRY(ar.alloc(&pre, ns));
    SNN_L k_ht_split_caps<Pol><<<grid_for(ns, 256), 256, 0, s>>>(pol, sl, ns, workv, limit, caps);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(scan_inclusive_i64(caps, pre, ns, ar, s));
    std::vector<int64_t> hp((size_t)ns);
    SNN_CUDA(cudaMemcpyAsync(hp.data(), pre, (size_t)ns * 8, cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    ar.rewind(m);
    int64_t start = 0;
    while (start < ns) {
        int64_t base = start > 0 ? hp[(size_t)start - 1] : 0;
        int64_t j = std::upper_bound(hp.begin() + start, hp.end(), base + pool_slots) - hp.begin();
        if (j <= start) j = start + 1;
        cuts.push_back(j);
        start = j;
    }
    return Status{};
}

// Host driver: work, classification and the warp, block and big-block tiers
// run without host synchronization; the split tier follows reads of its
// sizes. d_cnt: >= HT_NTIER device int64; h_cnt: a pinned host int64[>=3];
// status: device word. d_cnt: >= HT_NCNT device int64 (per-tier counts, summed
// work, vertices histogrammed).
template <class Pol>
Status run_histogram(const Pol& pol, Arena& ar, cudaStream_t s, int64_t* d_cnt, int64_t* h_cnt,
                     int64_t* status, const HtTiers& tiers = HtTiers{})
{
    using S = typename Pol::S;
    int32_t V = pol.V;
    if (V <= 0) return Status{};
    int32_t* lists;
    int64_t *scap, *workv;
    SNN_TRY(ar.alloc(&lists, (int64_t)HT_NTIER * V));
    SNN_TRY(ar.alloc(&scap, V));
    SNN_TRY(ar.alloc(&workv, V));
    SNN_CUDA(cudaMemsetAsync(d_cnt, 0, HT_NCNT * sizeof(int64_t), s));
    int32_t *todo, *ntodo;
    SNN_TRY(ar.alloc(&todo, V));
    SNN_TRY(ar.alloc(&ntodo, 1));
    SNN_CUDA(cudaMemsetAsync(ntodo, 0, sizeof(int32_t), s));
    SNN_L k_ht_skip<Pol><<<grid_for(V, 256), 256, 0, s>>>(pol, workv, todo, ntodo);
    SNN_L k_ht_work<Pol><<<grid_for((int64_t)V * 32, 256), 256, 0, s>>>(pol, workv, todo, ntodo);
    SNN_CUDA(cudaGetLastError());
    SNN_L k_ht_classify<Pol><<<grid_for(V, 256), 256, 0, s>>>(pol, workv, lists, d_cnt, scap, tiers);
    SNN_CUDA(cudaGetLastError());
    size_t wsm = (size_t)HT_WARPS * HT_WCAP * slot_bytes<S>();
    size_t bsm = (size_t)HT_BCAP * slot_bytes<S>();
    size_t gsm = (size_t)big_cap<S>() * slot_bytes<S>();
    auto kb = k_ht_block<Pol, HT_BTHREADS, HT_BCAP, HT_TIER_BLOCK, HT_TIER_BIG>;
    auto kg = k_ht_block<Pol, HT_GTHREADS, big_cap<S>(), HT_TIER_BIG, HT_TIER_SPLIT>;
    // set on every call: the attribute is per device, and handles on other
    // host threads may reach this point concurrently
    SNN_TRY(set_smem(k_ht_warp<Pol>, wsm));
    SNN_TRY(set_smem(kb, bsm));
    SNN_TRY(set_smem(kg, gsm));
    SNN_L k_ht_warp<Pol><<<(int)std::min<int64_t>(ceil_div(V, HT_WARPS), 152 * 8), HT_WARPS * 32, wsm,
                           s>>>(pol, lists, d_cnt, workv, scap);
    SNN_CUDA(cudaGetLastError());
    SNN_L kb<<<(int)std::min<int64_t>(V, 152 * 8), HT_BTHREADS, bsm, s>>>(pol, lists, d_cnt, scap, workv);
    SNN_CUDA(cudaGetLastError());
    SNN_L kg<<<152, HT_GTHREADS, gsm, s>>>(pol, lists, d_cnt, scap, workv);
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaMemcpyAsync(h_cnt, d_cnt + HT_TIER_SPLIT, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    int64_t ns = h_cnt[0];
    if (ns == 0) return Status{};
    const int32_t* sl = lists + (int64_t)HT_TIER_SPLIT * V;
    // first pass with tables capped at 2 * HT_SPLIT_CAP slots; vertices that
    // overflow them are redone with tables sized to their exact key bound
    // Both passes run over chunks of vertices whose tables fit in a pool of
    // max(64 MiB, 4 bytes per pin of the level), so the scratch of this tier
    // stays bounded whatever the degree distribution; chunks are cut from
    // the vertices' actual table sizes.
    int32_t* again;
    int64_t* nagain;
    SNN_TRY(ar.alloc(&again, ns));
    SNN_TRY(ar.alloc(&nagain, 1));
    SNN_CUDA(cudaMemsetAsync(nagain, 0, sizeof(int64_t), s));
    const int64_t pool_slots =
        std::max<int64_t>((int64_t)64 << 20, 4 * pol.L.P) / (int64_t)slot_bytes<S>();
    std::vector<int64_t> cuts;
    SNN_TRY(split_cuts(pol, ar, s, sl, ns, workv, HT_SPLIT_CAP, pool_slots, cuts));
    h_cnt[0] = 0;
    for (size_t c = 0; c + 1 < cuts.size(); c++) {
        Arena::Mark m = ar.mark();
        SNN_TRY(run_split(pol, ar, s, sl + cuts[c], cuts[c + 1] - cuts[c], workv, HT_SPLIT_CAP,
                          again, nagain, h_cnt));
        ar.rewind(m);
    }
    int64_t n2 = h_cnt[0];
    if (n2 == 0) return Status{};
    SNN_TRY(split_cuts(pol, ar, s, again, n2, workv, 0, pool_slots, cuts));
    for (size_t c = 0; c + 1 < cuts.size(); c++) {
        Arena::Mark m = ar.mark();
        SNN_TRY(run_split(pol, ar, s, again + cuts[c], cuts[c + 1] - cuts[c], workv, 0, nullptr,
                          nullptr, h_cnt));
        ar.rewind(m);
    }
    return Status{};
}

}  // namespace snn
