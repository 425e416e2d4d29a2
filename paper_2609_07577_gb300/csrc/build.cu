// Level 0 of the hierarchy (the SNN hypergraph of Sec. 2) and the per-level
// helpers every stage shares: size buckets, incidence lists, level memory.
#include "internal.cuh"

#include <nvtx3/nvToolsExt.h>

namespace snn {

// ---------------------------------------------------------------------------
// scalars

Status read_scalars(snnmap_hgraph* h)
{
    SNN_CUDA(cudaMemcpyAsync(h->h_scal, h->d_scal, SC_COUNT * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, h->stream));
    SNN_CUDA(cudaStreamSynchronize(h->stream));
    if (!h->prof_pend.empty()) prof_collect(h);
    return Status{};
}

// ---------------------------------------------------------------------------
// profiler

const char* const kStageNames[PS_N] = {"build",    "affinity",  "match",  "contract",
                                       "incidence", "pincount", "gains",  "sortmoves",
                                       "replay",   "validity",  "apply",  "save",
                                       "rows",     "cross"};

static cudaEvent_t prof_event(snnmap_hgraph* h)
{
    if (!h->prof_pool.empty()) {
        cudaEvent_t e = h->prof_pool.back();
        h->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Every stage scope is also an NVTX range named after the stage (a start/end
// pair, so scopes that replace one another need not nest), which timeline
// and kernel profilers show around the stage's launches; with no tool
// attached the calls return at once.
ProfScope::ProfScope(snnmap_hgraph* h_, int stage_) : h(h_), stage(stage_)
{
    range = nvtxRangeStartA(kStageNames[stage]);
    if (!h->prof_on) return;
    a = prof_event(h);
    b = prof_event(h);
    if (a && b) cudaEventRecord(a, h->stream);
}

ProfScope::~ProfScope()
{
    nvtxRangeEnd(range);
    if (!h->prof_on || !a || !b) return;
    cudaEventRecord(b, h->stream);
    h->prof_pend.push_back({stage, a, b});
}

void prof_collect(snnmap_hgraph* h)
{
    for (auto& p : h->prof_pend) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            h->prof_ms[p.stage] += ms;
            h->prof_calls[p.stage] += 1;
        } else {
            cudaGetLastError();
        }
        h->prof_pool.push_back(p.a);
        h->prof_pool.push_back(p.b);
    }
    h->prof_pend.clear();
}

void prof_release(snnmap_hgraph* h)
{
    cudaStreamSynchronize(h->stream);
    prof_collect(h);
    for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
    h->prof_pool.clear();
}

Status zero_scalars(snnmap_hgraph* h)
{
    SNN_CUDA(cudaMemsetAsync(h->d_scal, 0, SC_COUNT * sizeof(int64_t), h->stream));
    return Status{};
}

// ---------------------------------------------------------------------------
// level memory

Status level_alloc(snnmap_hgraph* h, Level& L, LevelExtra& X, int32_t V, int32_t E, int64_t P)
{
    Carver c;
    L.V = V;
    L.E = E;
    L.P = P;
    c.add(&L.hoff, (int64_t)E + 1);
    c.add(&L.hpins, P);
    c.add(&L.hw, E);
    c.add(&L.hk, E);
    c.add(&L.hsd, E);
    c.add(&L.voff, (int64_t)V + 1);
    c.add(&L.vinc, P);
    c.add(&L.vsize, V);
    c.add(&L.vinpins, V);
    c.add(&L.vincnt, V);
    c.add(&L.vinint, V);
    c.add(&X.seg.list, E);
    c.add(&X.seg.meta, 2 * SEG_NB);
    void* p = nullptr;
    SNN_CUDA(dev_malloc(&p, c.total, h->stream));
    c.assign(p);
    L.block = p;
    L.bytes = c.total;
    if (!L.cid) SNN_CUDA(dev_malloc((void**)&L.cid, (size_t)(V > 0 ? V : 1) * 4, h->stream));
    L.resident = true;
    return Status{};
}

int64_t held_bytes(const snnmap_hgraph* h)
{
    int64_t t = (int64_t)h->scratch.held() + (int64_t)h->cap_v * 20;
    if (h->dense.C) t += h->dense.cap * (h->dense.Kp * 8 + 20);
    if (h->mat.S) t += h->mat.cap * 16;
    for (auto& L : h->levels) t += (int64_t)L.bytes + 4 * (int64_t)L.V;
    return t;
}

void note_bytes(snnmap_hgraph* h)
{
    int64_t b = held_bytes(h);
    if (b > h->peak_bytes) h->peak_bytes = b;
}

void level_free(snnmap_hgraph* h, Level& L)
{
    if (L.block) cudaFreeAsync(L.block, h->stream);
    if (L.cid) cudaFreeAsync(L.cid, h->stream);
    L = Level{};
}

void level_release(snnmap_hgraph* h, Level& L)
{
    if (!L.resident) return;
    if (L.block) cudaFreeAsync(L.block, h->stream);
    int32_t* cid = L.cid;
    Level k;
    k.V = L.V;
    k.E = L.E;
    k.P = L.P;
    k.maxlen = L.maxlen;
    k.cid = cid;
    L = k;
}

// ---------------------------------------------------------------------------
// size buckets

__device__ __forceinline__ int seg_bucket(int64_t len)
{
    return len <= SEG_T_CAP ? SEG_BT
         : len <= 32 ? SEG_BB0 : (len <= SEG_B1_CAP ? SEG_BB1 : (len <= SEG_B2_CAP ? SEG_BB2 : SEG_BB3));
}

// bucket flags packed two per int64 (pa: T, B0; pb: B1, B2; pc: B3)
__global__ void k_seg_flags(const int64_t* __restrict__ hoff, int32_t E, int64_t* pa, int64_t* pb,
                            int64_t* pc, int64_t* w2)
{
    int64_t acc = 0;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < E;
         a += (int64_t)gridDim.x * blockDim.x) {
        int64_t len = hoff[a + 1] - hoff[a];
        int b = seg_bucket(len);
        pa[a] = (int64_t)(b == SEG_BT) | ((int64_t)(b == SEG_BB0) << 32);
        pb[a] = (int64_t)(b == SEG_BB1) | ((int64_t)(b == SEG_BB2) << 32);
        pc[a] = (int64_t)(b == SEG_BB3);
        acc += len * (len - 1);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd((unsigned long long*)w2, (unsigned long long)acc);
}

__global__ void k_seg_meta(const int64_t* tot, int32_t* meta)
{
    int32_t c[SEG_NB] = {(int32_t)(tot[0] & 0xffffffff), (int32_t)(tot[0] >> 32),
                         (int32_t)(tot[1] & 0xffffffff), (int32_t)(tot[1] >> 32),
                         (int32_t)(tot[2] & 0xffffffff)};
    int32_t run = 0;
    for (int b = 0; b < SEG_NB; b++) {
        meta[b] = run;
        meta[SEG_NB + b] = c[b];
        run += c[b];
    }
}

__global__ void k_seg_scatter(const int64_t* __restrict__ hoff, int32_t E,
                              const int64_t* __restrict__ pa, const int64_t* __restrict__ pb,
                              const int64_t* __restrict__ pc, const int32_t* __restrict__ meta,
                              int32_t* list)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < E;
         a += (int64_t)gridDim.x * blockDim.x) {
        int b = seg_bucket(hoff[a + 1] - hoff[a]);
        int64_t pos = b == SEG_BT ? (pa[a] & 0xffffffff)
                    : b == SEG_BB0 ? (pa[a] >> 32)
                    : b == SEG_BB1 ? (pb[a] & 0xffffffff)
                    : b == SEG_BB2 ? (pb[a] >> 32)
                                   : (pc[a] & 0xffffffff);
        list[meta[b] + pos] = (int32_t)a;
    }
}

Status seg_classify(const int64_t* hoff, int32_t E, int32_t maxlen, SegBuckets& b, Arena& ar,
                    cudaStream_t s, int64_t* w2)
{
    int64_t *pa, *pb, *pc, *tot;
    SNN_TRY(ar.alloc(&pa, E));
    SNN_TRY(ar.alloc(&pb, E));
    SNN_TRY(ar.alloc(&pc, E));
    SNN_TRY(ar.alloc(&tot, 3));
    b.b3_cap = 0;
    if (maxlen > SEG_B2_CAP) {
        int64_t c = SEG_B2_CAP;
        while (c < maxlen) c <<= 1;
        b.b3_cap = c;
    }
    if (E > 0) {
        SNN_L k_seg_flags<<<grid_for(E, 256), 256, 0, s>>>(hoff, E, pa, pb, pc, w2);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(scan_exclusive_i64(pa, pa, E, tot, ar, s));
    SNN_TRY(scan_exclusive_i64(pb, pb, E, tot + 1, ar, s));
    SNN_TRY(scan_exclusive_i64(pc, pc, E, tot + 2, ar, s));
    SNN_L k_seg_meta<<<1, 1, 0, s>>>(tot, b.meta);
    SNN_CUDA(cudaGetLastError());
    if (E > 0) {
        SNN_L k_seg_scatter<<<grid_for(E, 256), 256, 0, s>>>(hoff, E, pa, pb, pc, b.meta, b.list);
        SNN_CUDA(cudaGetLastError());
    }
    return Status{};
}

// ---------------------------------------------------------------------------
// incidence lists: degree count, scan, scatter with the source bit

// Lanes of a warp holding the same vertex add their count once (consecutive
// hyperedges of a coarse level share most of their super-nodes); the loop
// runs over whole warps so the match covers all 32 lanes.
__global__ void k_count_deg(const int32_t* __restrict__ pins, int64_t P, int32_t* deg)
{
    int lane = threadIdx.x & 31;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < P;
         base += stride) {
        int64_t j = base + lane;
        int32_t q = j < P ? pins[j] : -1;
        unsigned same = __match_any_sync(FULL, q);
        if (q >= 0 && lane == __ffs(same) - 1) atomicAdd(&deg[q], __popc(same));
    }
}

// a group of G lanes per hyperedge
template <int G>
__global__ void k_csc_fill(const int64_t* __restrict__ hoff, const int32_t* __restrict__ pins,
                           int32_t E, const int64_t* __restrict__ voff, int32_t* cursor,
                           int32_t* vinc)
{
    int lane = threadIdx.x & (G - 1);
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) / G;
    for (int64_t a = gw; a < E; a += nw) {
        int64_t b = hoff[a], e = hoff[a + 1];
        for (int64_t j = b + lane; j < e; j += G) {
            int32_t q = pins[j];
            int32_t slot = atomicAdd(&cursor[q], 1);
            vinc[voff[q] + slot] = (int32_t)((uint32_t)a | (j == b ? SRC_BIT : 0u));
        }
    }
}

Status build_incidence(snnmap_hgraph* h, Level& L)
{
    ProfScope prof(h, PS_INCIDENCE);
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    int32_t *deg, *cursor;
    SNN_TRY(ar.alloc(&deg, L.V));
    SNN_TRY(ar.alloc(&cursor, L.V));
    if (L.V > 0) {
        SNN_CUDA(cudaMemsetAsync(deg, 0, (size_t)L.V * sizeof(int32_t), s));
        SNN_CUDA(cudaMemsetAsync(cursor, 0, (size_t)L.V * sizeof(int32_t), s));
    }
    if (L.P > 0) {
        SNN_L k_count_deg<<<grid_for(L.P, 256), 256, 0, s>>>(L.hpins, L.P, deg);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(scan_exclusive_i32_to_i64(deg, L.voff, L.V, L.voff + L.V, ar, s));
    if (L.E > 0) {
        SNN_HEDGE_LAUNCH(hedge_lanes(L.P, L.E), k_csc_fill, L.E, s, L.hoff, L.hpins, L.E, L.voff,
                         cursor, L.vinc);
        SNN_CUDA(cudaGetLastError());
    }
    return Status{};
}

// ---------------------------------------------------------------------------
// S0: validation, copy, canonical destination order, vertex state

__global__ void k_in_hedges(const int64_t* __restrict__ off, const int32_t* __restrict__ w,
                            int32_t E, int32_t* kept, int64_t* klen, int64_t* scal)
{
    int32_t bad = 0;
    int64_t mx = 0, wsum = 0;
    int32_t zero = 0;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < E;
         a += (int64_t)gridDim.x * blockDim.x) {
        int64_t len = off[a + 1] - off[a];
        if (len < 1 || len > 0x7fffffff || w[a] < 0) bad = 1;
        int k = len >= 2 ? 1 : 0;
        if (k && w[a] == 0) zero = 1;
        kept[a] = k;
        klen[a] = k ? len : 0;
        if (len > mx) mx = len;
        wsum += w[a] > 0 ? w[a] : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int64_t m2 = __shfl_xor_sync(FULL, mx, o);
        mx = m2 > mx ? m2 : mx;
        wsum += __shfl_xor_sync(FULL, wsum, o);
        bad |= __shfl_xor_sync(FULL, bad, o);
        zero |= __shfl_xor_sync(FULL, zero, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr((int*)&scal[SC_STATUS], ST_INVALID);
        if (zero) atomicOr((int*)&scal[SC_E], 1);
        atomicMax((unsigned long long*)&scal[SC_C], (unsigned long long)mx);
        atomicAdd((unsigned long long*)&scal[SC_D], (unsigned long long)wsum);
    }
}

__global__ void k_in_pins(const int32_t* __restrict__ pins, int64_t P, int32_t V, int64_t* scal)
{
    int bad = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t q = pins[j];
        if (q < 0 || q >= V) bad = 1;
    }
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicOr((int*)&scal[SC_STATUS], ST_INVALID);
}

__global__ void k_copy_hedges(const int64_t* __restrict__ off, const int32_t* __restrict__ pins,
                              const int32_t* __restrict__ w, int32_t E,
                              const int32_t* __restrict__ kept, const int32_t* __restrict__ newid,
                              const int64_t* __restrict__ newoff, Level L)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = gw; a < E; a += nw) {
        if (!kept[a]) continue;
        int32_t e = newid[a];
        int64_t src = off[a], dst = newoff[a], len = off[a + 1] - off[a];
        for (int64_t j = lane; j < len; j += 32) L.hpins[dst + j] = pins[src + j];
        if (lane == 0) {
            L.hoff[e] = dst;
            L.hw[e] = w[a];
            L.hk[e] = 1;
            L.hsd[e] = 0;
        }
    }
}

__global__ void k_set_last_off(int64_t* hoff, int32_t E, const int64_t* P)
{
    hoff[E] = *P;
}

// Sorts each hyperedge's destinations in place and flags repeated
// destinations and the source listed as a destination.
struct BuildCheckJob {
    const int64_t* hoff;
    int32_t* pins;
    int64_t* scal;
    __device__ int len(int32_t a) const { return (int)(hoff[a + 1] - hoff[a] - 1); }
    __device__ uint32_t load(int32_t a, int i) const { return (uint32_t)pins[hoff[a] + 1 + i]; }
    __device__ void finish(int32_t a, const uint32_t* s, int n) const
    {
        int lane = threadIdx.x & 31;
        int64_t base = hoff[a];
        uint32_t src = (uint32_t)pins[base];
        int bad = 0;
        for (int c = 0; c < n; c += 32) {
            int i = c + lane;
            if (i < n) {
                uint32_t v = s[i];
                if ((i > 0 && s[i - 1] == v) || v == src) bad = 1;
                pins[base + 1 + i] = (int32_t)v;
            }
        }
        if (__any_sync(FULL, bad) && lane == 0) atomicOr((int*)&scal[SC_STATUS], ST_INVALID);
    }
    __device__ void finish_thread(int32_t a, const uint32_t* s, int n, int st) const
    {
        int64_t base = hoff[a];
        uint32_t src = (uint32_t)pins[base];
        int bad = 0;
        for (int i = 0; i < n; i++) {
            if ((i > 0 && s[(i - 1) * st] == s[(i) * st]) || s[(i) * st] == src) bad = 1;
            pins[base + 1 + i] = (int32_t)s[(i) * st];
        }
        if (bad) atomicOr((int*)&scal[SC_STATUS], ST_INVALID);
    }
};

__global__ void k_count_inpins(const int64_t* __restrict__ hoff, const int32_t* __restrict__ pins,
                               int32_t E, int32_t* inpins)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = gw; a < E; a += nw) {
        for (int64_t j = hoff[a] + 1 + lane; j < hoff[a + 1]; j += 32) atomicAdd(&inpins[pins[j]], 1);
    }
}

__global__ void k_vertex_init(Level L, int32_t delta, int32_t phi, int64_t* scal)
{
    int bad = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < L.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t ip = L.vinpins[n];
        L.vsize[n] = 1;
        L.vincnt[n] = ip;
        L.vinint[n] = 0;
        if (ip > phi || ip > delta) bad = 1;
    }
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0)
        atomicOr((int*)&scal[SC_STATUS], ST_INFEASIBLE);
}

Status build_level0(snnmap_hgraph* h, int32_t V, int32_t E, const int64_t* d_off,
                    const int32_t* d_pins, const int32_t* d_w)
{
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    int64_t ends[2] = {0, 0};
    SNN_CUDA(cudaMemcpyAsync(&ends[0], d_off, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaMemcpyAsync(&ends[1], d_off + E, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (ends[0] != 0 || ends[1] < E) return Status{SNNMAP_ERR_INVALID, "offsets: first must be 0 and every hyperedge needs a pin"};
    int64_t Pin = ends[1];
    SNN_TRY(zero_scalars(h));
    int32_t *kept, *newid;
    int64_t *klen, *newoff;
    SNN_TRY(ar.alloc(&kept, E));
    SNN_TRY(ar.alloc(&newid, E));
    SNN_TRY(ar.alloc(&klen, E));
    SNN_TRY(ar.alloc(&newoff, E));
    if (E > 0) {
        SNN_L k_in_hedges<<<grid_for(E, 256), 256, 0, s>>>(d_off, d_w, E, kept, klen, h->d_scal);
        SNN_CUDA(cudaGetLastError());
    }
    if (Pin > 0) {
        SNN_L k_in_pins<<<grid_for(Pin, 256), 256, 0, s>>>(d_pins, Pin, V, h->d_scal);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(scan_exclusive_i32(kept, newid, E, (int32_t*)(h->d_scal + SC_A), ar, s));
    SNN_TRY(scan_exclusive_i64(klen, newoff, E, h->d_scal + SC_B, ar, s));
    SNN_TRY(read_scalars(h));
    if (h->h_scal[SC_STATUS] & ST_INVALID)
        return Status{SNNMAP_ERR_INVALID, "hyperedge without pins, negative weight or pin id out of range"};
    int32_t E0 = (int32_t)(h->h_scal[SC_A] & 0xffffffff);
    int64_t P0 = h->h_scal[SC_B];
    int32_t maxlen = (int32_t)h->h_scal[SC_C];
    h->wide = (uint64_t)h->h_scal[SC_D] >= 0xffffffffull;
    h->wsum = h->h_scal[SC_D];
    h->wzero = h->h_scal[SC_E] != 0;

    h->levels.emplace_back();
    h->extra.emplace_back();
    Level& L = h->levels.back();
    LevelExtra& X = h->extra.back();
    SNN_TRY(level_alloc(h, L, X, V, E0, P0));
    L.maxlen = maxlen;
    if (E > 0) {
        SNN_L k_copy_hedges<<<grid_for((int64_t)E * 32, 256), 256, 0, s>>>(d_off, d_pins, d_w, E, kept,
                                                                      newid, newoff, L);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_L k_set_last_off<<<1, 1, 0, s>>>(L.hoff, E0, h->d_scal + SC_B);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(seg_classify(L.hoff, E0, maxlen, X.seg, ar, s, h->d_scal + SC_W2));
    BuildCheckJob job{L.hoff, L.hpins, h->d_scal};
    {
        ProfScope prof(h, PS_BUILD);
        SNN_TRY(seg_run(job, X.seg, E0, ar, s));
    }
    if (V > 0) SNN_CUDA(cudaMemsetAsync(L.vinpins, 0, (size_t)V * sizeof(int32_t), s));
    if (E0 > 0) {
        SNN_L k_count_inpins<<<grid_for((int64_t)E0 * 32, 256), 256, 0, s>>>(L.hoff, L.hpins, E0, L.vinpins);
        SNN_CUDA(cudaGetLastError());
    }
    if (V > 0) {
        SNN_L k_vertex_init<<<grid_for(V, 256), 256, 0, s>>>(L, h->prm.delta, h->prm.phi, h->d_scal);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(build_incidence(h, L));
    SNN_TRY(read_scalars(h));
    X.pair_terms = h->h_scal[SC_W2];
    h->scratch.reset();
    if (h->h_scal[SC_STATUS] & ST_INVALID)
        return Status{SNNMAP_ERR_INVALID, "repeated destination or source listed as a destination"};
    if (h->h_scal[SC_STATUS] & ST_INFEASIBLE)
        return Status{SNNMAP_ERR_INFEASIBLE, "a neuron alone exceeds Delta or Phi"};
    return Status{};
}

}  // namespace snn
