// Coarsening (Sec. 4.1): neighbour histogram and candidate (Eq.
// neigh_histogram), then the matching of Eq. matching over the candidate
// pseudo-forest.
//
// Histogram. For vertex n, every pin m != n of every hyperedge a incident to
// n adds omega(a) to score(n, m) and, when n and m are both destinations of a,
// k(a) (original axons merged into a) to their shared inbound count. The
// table is an open-addressing hash table keyed by m: one per warp in shared
// memory for ordinary vertices; vertices whose distinct neighbours overflow
// it are redone by a block with a larger shared table, and those overflowing
// that by a block with a table in global scratch. Sums are integer atomics,
// so the result does not depend on the order of updates. The pins of up to
// 32 incident hyperedges are flattened into one virtual range so all 32
// lanes load consecutive pins even when hyperedges are short.
//
// Candidate. Among neighbours m that keep the merged super-node within
// Omega, Phi and Delta (merged inbound set = in_count(n) + in_count(m) -
// shared), the highest score wins, ties to the lower id.
//
// Matching. Two-cycles of the candidate graph match. Every other vertex x
// with children (vertices whose candidate is x) has a best child bc(x) (max
// score, ties to the lower id). Linking x to its parent p = cand(x) whenever
// bc(p) = x and neither is a root splits the forest into chains; Eq.
// matching then matches a vertex to its parent exactly when it sits at an
// odd distance from the top of its chain, and a vertex that is not matched
// to its parent takes its best child. Distances come from a bounded walk,
// with pointer jumping for chains longer than the walk.
#include "histo.cuh"
#include "internal.cuh"

#include <algorithm>
#include <memory>

namespace snn {

constexpr int MATCH_WALK = 64;

// Neighbour histogram policy: for vertex n, every pin m != n of every
// incident hyperedge a adds omega(a) to m's score and, when n and m are both
// destinations of a, k(a) to their shared inbound count. The best neighbour
// keeping the merged super-node within Omega, Phi and Delta wins.
template <typename S_>
struct AffPol {
    using S = S_;
    static constexpr bool kOptimistic = false;
    struct Acc {
        __device__ Acc() {}
        __device__ void add(const Acc&) {}
        __device__ void atomic_into(Acc*) const {}
    };
    static __device__ Acc warp_reduce(const Acc& a) { return a; }

    Level L;
    int32_t V;
    int64_t keys;
    int32_t omega, delta, phi;
    int32_t* cand;
    int64_t* cscore;
    int32_t* cov;
    const int32_t* vmin;   // smallest size and inbound pins over the level's vertices
    bool prefilter;        // some pair can break Omega or Phi (else elem skips the test)
    const uint8_t* only = nullptr;   // if set, the vertices evaluated (others untouched)
    const int4* vst;       // (size, inbound pins, inbound axons) per vertex

    // n cannot merge even with the smallest vertex: no candidate
    __device__ bool skip(int32_t n) const
    {
        if (only && !only[n]) return true;
        return (int64_t)L.vsize[n] + vmin[0] > omega || (int64_t)L.vinpins[n] + vmin[1] > phi;
    }
    __device__ int64_t vb(int32_t n) const { return L.voff[n]; }
    __device__ int64_t ve(int32_t n) const { return L.voff[n + 1]; }
    __device__ int64_t seg_len(int64_t i) const
    {
        int32_t a = (int32_t)((uint32_t)L.vinc[i] & ~SRC_BIT);
        return L.hoff[a + 1] - L.hoff[a];
    }
    __device__ Seg<S> seg(int64_t i, Acc&) const
    {
        uint32_t inc = (uint32_t)L.vinc[i];
        int32_t a = (int32_t)(inc & ~SRC_BIT);
        Seg<S> g;
        g.sd = L.hsd[a];
        g.nd = !(inc & SRC_BIT) || g.sd;
        g.b = L.hoff[a];
        g.len = (int32_t)(L.hoff[a + 1] - g.b);
        g.w = (S)L.hw[a];
        g.k = (uint32_t)L.hk[a];
        return g;
    }
    // one element: neighbour m (-1: nothing to add), weight, shared count
    struct Item {
        int32_t m;
        S w;
        uint32_t o;
    };
    static __device__ Item none() { return Item{-1, 0, 0u}; }
    __device__ Item load(int32_t n, const Seg<S>& g, int32_t off) const
    {
        Item it;
        it.m = L.hpins[g.b + off];
        it.w = g.w;
        int md = off != 0 || g.sd;   // pin 0 is the source
        it.o = (g.nd && md) ? g.k : 0u;
        // a neighbour whose size or inbound pins alone break Omega or Phi
        // with n can never be the candidate: leave it out of the table
        if (it.m == n) {
            it.m = -1;
        } else if (prefilter) {
            int4 a = vst[n], b = vst[it.m];
            if ((int64_t)a.x + b.x > omega || (int64_t)a.y + b.y > phi) it.m = -1;
        }
        return it;
    }
    template <class Tb>
    __device__ bool put(int32_t, const Item& it, const Tb& t, Acc&) const
    {
        return it.m < 0 || t.add(it.m, it.w, it.o);
    }
    template <class Tb>
    __device__ bool elem(int32_t n, const Seg<S>& g, int32_t off, const Tb& t, Acc& acc) const
    {
        return put(n, load(n, g, off), t, acc);
    }
    __device__ void consider(int32_t n, int32_t m, int64_t s, uint32_t o, const Acc&, int64_t& bs,
                             int32_t& bk, uint32_t& bo) const
    {
        int4 a = vst[n], b = vst[m];
        bool valid = (int64_t)a.x + b.x <= omega && (int64_t)a.y + b.y <= phi &&
                     (int64_t)a.z + b.z - (int64_t)o <= delta;
        if (valid && better(s, m, bs, bk)) {
            bs = s;
            bk = m;
            bo = o;
        }
    }
    __device__ void write(int32_t n, int64_t bs, int32_t bk, uint32_t bo, const Acc&) const
    {
        if (only && !only[n]) return;
        cand[n] = bk;
        cscore[n] = bk < 0 ? 0 : bs;
        cov[n] = bk < 0 ? 0 : (int32_t)bo;
    }
};

// (size, inbound pins, inbound axons) of every vertex in one 16-byte entry, so
// a neighbour's state is one gather in the histograms' hot loops
__global__ void k_pack_state(Level L, int4* vst)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < L.V;
         n += (int64_t)gridDim.x * blockDim.x)
        vst[n] = make_int4(L.vsize[n], L.vinpins[n], L.vincnt[n], 0);
}

// ---------------------------------------------------------------------------
// matching

__global__ void k_count_cand(int32_t V, const int32_t* __restrict__ cand, int64_t* scal)
{
    int c = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        c += cand[n] >= 0;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)&scal[SC_A], (unsigned long long)c);
}

__global__ void k_child_best_score(int32_t V, const int32_t* __restrict__ cand,
                                   const int64_t* __restrict__ cscore, int64_t* bestsc)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = cand[n];
        if (c >= 0) atomicMax((long long*)&bestsc[c], (long long)cscore[n]);
    }
}

__global__ void k_child_best_id(int32_t V, const int32_t* __restrict__ cand,
                                const int64_t* __restrict__ cscore,
                                const int64_t* __restrict__ bestsc, int32_t* bc)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = cand[n];
        if (c >= 0 && cscore[n] == bestsc[c]) atomicMin(&bc[c], (int32_t)n);
    }
}

__device__ __forceinline__ bool is_root(const int32_t* cand, int32_t n)
{
    int32_t c = cand[n];
    return c >= 0 && cand[c] == n;
}

// link(n) = parent when n is its parent's best child and neither is a root
__global__ void k_link(int32_t V, const int32_t* __restrict__ cand, const int32_t* __restrict__ bc,
                       int32_t* link)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = cand[n];
        int32_t lk = -1;
        if (c >= 0 && cand[c] != (int32_t)n && !is_root(cand, c) && bc[c] == (int32_t)n) lk = c;
        link[n] = lk;
    }
}

// parity of the distance to the chain top, by a walk of at most MATCH_WALK
// links; longer chains are left to pointer jumping (par = 2)
__global__ void k_walk(int32_t V, const int32_t* __restrict__ link, uint8_t* par, int64_t* scal)
{
    int c = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = (int32_t)n;
        int d = 0;
        while (d < MATCH_WALK && link[x] >= 0) {
            x = link[x];
            d++;
        }
        if (link[x] >= 0) {
            par[n] = 2;
            c++;
        } else {
            par[n] = (uint8_t)(d & 1);
        }
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)&scal[SC_B], (unsigned long long)c);
}

// pointer jumping over all vertices (fallback): nxt/pj hold the current
// jump target and the parity of the distance covered so far
__global__ void k_jump_init(int32_t V, const int32_t* __restrict__ link, int32_t* nxt, uint8_t* pj)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        nxt[n] = link[n];
        pj[n] = link[n] >= 0 ? 1 : 0;
    }
}

__global__ void k_jump(int32_t V, const int32_t* __restrict__ nxt, const uint8_t* __restrict__ pj,
                       int32_t* nxt2, uint8_t* pj2, int64_t* scal)
{
    int c = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = nxt[n];
        if (x >= 0) {
            nxt2[n] = nxt[x];
            pj2[n] = pj[n] ^ pj[x];
            c += nxt[x] >= 0;
        } else {
            nxt2[n] = -1;
            pj2[n] = pj[n];
        }
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)&scal[SC_B], (unsigned long long)c);
}

__global__ void k_jump_done(int32_t V, const uint8_t* __restrict__ pj, uint8_t* par)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        if (par[n] == 2) par[n] = pj[n];
}

// Eq. matching: matched to the parent at odd distance (or in a root
// two-cycle), otherwise to the best child if any
__global__ void k_match_finish(int32_t V, const int32_t* __restrict__ cand,
                               const int32_t* __restrict__ bc, const uint8_t* __restrict__ par,
                               int32_t* match, int64_t* scal)
{
    int c = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t cn = cand[n];
        int32_t m = -1;
        if (cn >= 0 && (cand[cn] == (int32_t)n || par[n] == 1)) m = cn;
        else if (bc[n] != 0x7fffffff) m = bc[n];
        match[n] = m;
        c += m > (int32_t)n;
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)&scal[SC_C], (unsigned long long)c);
}

// ---------------------------------------------------------------------------

// vm[0], vm[1]: smallest size and inbound pins; vm[2], vm[3]: largest
__global__ void k_level_min(Level L, int32_t* vm)
{
    int32_t ms = 0x7fffffff, mi = 0x7fffffff, xs = 0, xi = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < L.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        ms = min(ms, L.vsize[n]);
        mi = min(mi, L.vinpins[n]);
        xs = max(xs, L.vsize[n]);
        xi = max(xi, L.vinpins[n]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ms = min(ms, __shfl_xor_sync(FULL, ms, o));
        mi = min(mi, __shfl_xor_sync(FULL, mi, o));
        xs = max(xs, __shfl_xor_sync(FULL, xs, o));
        xi = max(xi, __shfl_xor_sync(FULL, xi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&vm[0], ms);
        atomicMin(&vm[1], mi);
        atomicMax(&vm[2], xs);
        atomicMax(&vm[3], xi);
    }
}

template <typename S>
static Status affinity(snnmap_hgraph* h, Level& L)
{
    int32_t* vmin;
    SNN_TRY(h->scratch.alloc(&vmin, 4));
    SNN_TRY(fill_i32(vmin, 0x7fffffff, 2, h->stream));
    SNN_CUDA(cudaMemsetAsync(vmin + 2, 0, 2 * sizeof(int32_t), h->stream));
    SNN_L k_level_min<<<grid_for(L.V, 256), 256, 0, h->stream>>>(L, vmin);
    SNN_CUDA(cudaGetLastError());
    int32_t vm[4];
    SNN_CUDA(cudaMemcpyAsync(vm, vmin, sizeof(vm), cudaMemcpyDeviceToHost, h->stream));
    SNN_CUDA(cudaStreamSynchronize(h->stream));
    int4* vst;
    SNN_TRY(h->scratch.alloc(&vst, L.V));
    SNN_L k_pack_state<<<grid_for(L.V, 256), 256, 0, h->stream>>>(L, vst);
    SNN_CUDA(cudaGetLastError());
    AffPol<S> pol;
    pol.vst = vst;
    pol.vmin = vmin;
    pol.prefilter = 2 * (int64_t)vm[2] > h->prm.omega || 2 * (int64_t)vm[3] > h->prm.phi;
    pol.L = L;
    pol.V = L.V;
    pol.keys = L.V;
    pol.omega = h->prm.omega;
    pol.delta = h->prm.delta;
    pol.phi = h->prm.phi;
    pol.cand = h->cand;
    pol.cscore = h->cscore;
    pol.cov = h->cov;
    int64_t* cnt;
    SNN_TRY(h->scratch.alloc(&cnt, HT_NCNT));
    if (L.V <= 0) SNN_CUDA(cudaMemsetAsync(cnt, 0, HT_NCNT * sizeof(int64_t), h->stream));
    SNN_TRY(run_histogram(pol, h->scratch, h->stream, cnt, h->h_scal + 12, h->d_scal, h->tiers));
    // the counters reach the level record after the matching's synchronization
    SNN_CUDA(cudaMemcpyAsync(h->h_tier, cnt, HT_NCNT * sizeof(int64_t), cudaMemcpyDeviceToHost,
                             h->stream));
    h->extra.back().carried = 0;
    h->tier_level = (int32_t)h->extra.size() - 1;
    h->tier_form = 1;
    return Status{};
}

void tier_fold(snnmap_hgraph* h)
{
    static_assert(HT_NCNT <= TIER_SLOTS, "counter set larger than its slot in h_tier");
    int32_t l = h->tier_level;
    if (l < 0) return;
    h->tier_level = -1;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess || l >= (int32_t)h->extra.size()) return;
    LevelExtra& X = h->extra[l];
    const int64_t* a = h->h_tier;
    const int64_t* b = h->h_tier + TIER_SLOTS;
    int64_t blk = a[HT_TIER_BLOCK] + a[HT_TIER_BIG], glb = a[HT_TIER_SPLIT], wk = a[HT_CNT_WORK];
    int64_t nf = a[HT_CNT_VERTS];
    if (h->tier_form == 2) {   // carried: new super-nodes' lists, then the full histograms
        blk += b[HT_TIER_BLOCK] + b[HT_TIER_BIG];
        glb += b[HT_TIER_SPLIT];
        wk += b[HT_CNT_WORK];
        nf = b[HT_CNT_VERTS];
    }
    X.n_block = (int32_t)blk;
    X.n_global = (int32_t)glb;
    X.n_full = (int32_t)nf;
    X.hist_work = wk;
}


// ---------------------------------------------------------------------------
// Candidates carried through a contraction.
//
// After level l is contracted, a vertex x of level l + 1 is either the
// super-node of a matched pair (NEW) or the image of an unmatched vertex n.
// For two unmatched vertices every hyperedge holding both maps onto one of
// the same omega, k and destination roles (a hyperedge vanishes only when all
// its pins share one super-node; duplicates that merge hold both as well),
// and their sizes and inbound counts are unchanged: their score, shared count
// and validity carry over. With c = cand(n) at level l:
//   c = -1 (NONE): no unmatched neighbour is valid; only new super-nodes
//       adjacent to x can be x's candidate.
//   c unmatched (KEEP): cid(c) stays the best unmatched neighbour with the
//       same score; a new super-node beats it only by Eq. neigh_histogram's
//       order (larger score, ties to the lower id).
//   c matched (MERGED), w = cid(c): score(x, w) >= score(n, c), and w's id is
//       below that of every unmatched neighbour of equal score (cid keeps the
//       order of representatives, and min(c, match(c)) <= c), so if w is
//       valid the best valid new super-node is the candidate; if the best one
//       is not w, x is evaluated in full.
// Scores towards new super-nodes come from the hyperedges holding one: each
// such hyperedge's list of new super-nodes (with destination roles) is the
// segment x visits, so this histogram does sum_a |a| |new(a)| updates
// instead of sum_a |a| (|a| - 1). New super-nodes and rejected MERGED vertices
// then get the full histogram.

enum : uint8_t { AK_NONE = 0, AK_KEEP = 1, AK_MERGED = 2, AK_NEW = 3 };
constexpr uint32_t NOT_DEST = 0x80000000u;

__global__ void k_ac_prep(int32_t V, const int32_t* __restrict__ cid,
                          const int32_t* __restrict__ match, const int32_t* __restrict__ cand,
                          const int64_t* __restrict__ cscore, const int32_t* __restrict__ cov,
                          AffCarry ac)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = cid[n];
        if (match[n] >= 0) {
            ac.kind[x] = AK_NEW;
            ac.full[x] = 1;
            continue;
        }
        int32_t c = cand[n];
        uint8_t k = AK_NONE;
        int32_t ic = -1;
        if (c >= 0) {
            ic = cid[c];
            k = match[c] >= 0 ? AK_MERGED : AK_KEEP;
        }
        ac.kind[x] = k;
        ac.full[x] = 0;
        ac.cand[x] = ic;
        ac.score[x] = k == AK_KEEP ? cscore[n] : 0;
        ac.ov[x] = k == AK_KEEP ? cov[n] : 0;
    }
}

// per hyperedge: its number of new super-nodes; work[0] += (|a| - cnt) cnt.
// A group of G lanes per hyperedge; each warp takes 32 / G consecutive
// hyperedges per step, so the group sums run with the whole warp.
template <int G>
__global__ void __launch_bounds__(256)
    k_ac_count(Level L, const uint8_t* __restrict__ kind, int32_t* lcnt, int64_t* work)
{
    constexpr int PER = 32 / G;
    int lane = threadIdx.x & (G - 1);
    int grp = (threadIdx.x & 31) / G;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t acc = 0;
    for (int64_t base = warp * PER; base < L.E; base += nwarp * PER) {
        int64_t a = base + grp;
        int c = 0;
        int64_t len = 0;
        if (a < L.E) {
            int64_t b = L.hoff[a], e = L.hoff[a + 1];
            len = e - b;
            for (int64_t j = b + lane; j < e; j += G) c += kind[L.hpins[j]] == AK_NEW;
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
        if (lane == 0 && a < L.E) {
            lcnt[a] = c;
            acc += (len - c) * (int64_t)c;
        }
    }
    if (lane == 0 && acc) atomicAdd((unsigned long long*)work, (unsigned long long)acc);
}

// the lists: new super-nodes of each hyperedge in pin order, bit 31 set for
// a source that is not also a destination
__global__ void __launch_bounds__(256)
    k_ac_fill(Level L, const uint8_t* __restrict__ kind, const int64_t* __restrict__ loff,
              uint32_t* lpins)
{
    int lane = threadIdx.x & 31;
    unsigned lt = lanemask_lt();
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = gw; a < L.E; a += nw) {
        int64_t b = L.hoff[a], e = L.hoff[a + 1];
        int64_t o = loff[a];
        if (loff[a + 1] == o) continue;
        int sd = L.hsd[a];
        for (int64_t cb = b; cb < e; cb += 32) {
            int64_t j = cb + lane;
            int32_t m = j < e ? L.hpins[j] : 0;
            bool nw_ = j < e && kind[m] == AK_NEW;
            unsigned mk = __ballot_sync(FULL, nw_);
            if (nw_)
                lpins[o + __popc(mk & lt)] = (uint32_t)m | ((j != b || sd) ? 0u : NOT_DEST);
            o += __popc(mk);
        }
    }
}

// work[0] += incidence segment lengths of the NEW vertices (what their full
// histograms cost); MERGED vertices mostly keep the new super-node their
// candidate merged into (k_ac_check), so they are left out of the estimate
__global__ void __launch_bounds__(256)
    k_ac_fullwork(Level L, const uint8_t* __restrict__ kind, int64_t* work)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t acc = 0;
    for (int64_t base = gw * 32; base < L.V; base += nw * 32) {
        int64_t n = base + lane;
        unsigned mem = __ballot_sync(FULL, n < L.V && kind[n] == AK_NEW);
        while (mem) {
            int src = __ffs(mem) - 1;
            mem &= mem - 1;
            int32_t m = (int32_t)__shfl_sync(FULL, (int32_t)n, src);
            for (int64_t i = L.voff[m] + lane; i < L.voff[m + 1]; i += 32) {
                int32_t a = (int32_t)((uint32_t)L.vinc[i] & ~SRC_BIT);
                acc += L.hoff[a + 1] - L.hoff[a];
            }
        }
    }
    acc = warp_sum(acc);
    if (lane == 0 && acc) atomicAdd((unsigned long long*)work, (unsigned long long)acc);
}

// MERGED vertices whose best valid new super-node is not w = cand (full
// flag 2): w's validity decides between keeping that result (0) and a full
// histogram (1). ov(x, w) sums k over the hyperedges in which both are
// destinations (w found by binary search among the sorted destinations).
__global__ void __launch_bounds__(256)
    k_ac_check(Level L, AffCarry ac, int32_t omega, int32_t delta, int32_t phi)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < L.V; base += nw * 32) {
        int64_t n = base + lane;
        bool f = n < L.V && ac.full[n] == 2;
        unsigned mem = __ballot_sync(FULL, f);
        while (mem) {
            int src = __ffs(mem) - 1;
            mem &= mem - 1;
            int32_t x = (int32_t)__shfl_sync(FULL, (int32_t)n, src);
            int32_t w = ac.cand[x];
            int64_t ov = 0;
            for (int64_t i = L.voff[x] + lane; i < L.voff[x + 1]; i += 32) {
                uint32_t inc = (uint32_t)L.vinc[i];
                int32_t a = (int32_t)(inc & ~SRC_BIT);
                int sd = L.hsd[a];
                if ((inc & SRC_BIT) && !sd) continue;   // x is not a destination of a
                int64_t b = L.hoff[a], e = L.hoff[a + 1];
                bool wd;
                if (L.hpins[b] == w) {
                    wd = sd != 0;
                } else {
                    int64_t lo = b + 1, hi = e;
                    while (lo < hi) {
                        int64_t mid = (lo + hi) >> 1;
                        if (L.hpins[mid] < w) lo = mid + 1;
                        else hi = mid;
                    }
                    wd = lo < e && L.hpins[lo] == w;
                }
                if (wd) ov += L.hk[a];
            }
            ov = warp_sum(ov);
            if (lane == 0) {
                bool valid = (int64_t)L.vsize[x] + L.vsize[w] <= omega &&
                             (int64_t)L.vinpins[x] + L.vinpins[w] <= phi &&
                             (int64_t)L.vincnt[x] + L.vincnt[w] - ov <= delta;
                ac.full[x] = valid ? 0 : 1;
            }
        }
    }
}

// Histogram of each carried vertex over the new super-nodes of its
// hyperedges, combined with its carried candidate.
template <typename S_>
struct AffNewPol {
    using S = S_;
    static constexpr bool kOptimistic = false;
    struct Acc {
        __device__ Acc() {}
        __device__ void add(const Acc&) {}
        __device__ void atomic_into(Acc*) const {}
    };
    static __device__ Acc warp_reduce(const Acc& a) { return a; }

    Level L;
    int32_t V;
    int64_t keys;
    int32_t omega, delta, phi;
    const int64_t* loff;
    const uint32_t* lpins;
    AffCarry ac;
    bool prefilter;
    const int4* vst;   // (size, inbound pins, inbound axons) per vertex
    int32_t* cand;
    int64_t* cscore;
    int32_t* cov;

    __device__ bool skip(int32_t n) const { return ac.kind[n] == AK_NEW; }
    __device__ int64_t vb(int32_t n) const { return L.voff[n]; }
    __device__ int64_t ve(int32_t n) const { return L.voff[n + 1]; }
    __device__ int64_t seg_len(int64_t i) const
    {
        int32_t a = (int32_t)((uint32_t)L.vinc[i] & ~SRC_BIT);
        return loff[a + 1] - loff[a];
    }
    __device__ Seg<S> seg(int64_t i, Acc&) const
    {
        uint32_t inc = (uint32_t)L.vinc[i];
        int32_t a = (int32_t)(inc & ~SRC_BIT);
        Seg<S> g;
        g.sd = L.hsd[a];
        g.nd = !(inc & SRC_BIT) || g.sd;
        g.b = loff[a];
        g.len = (int32_t)(loff[a + 1] - g.b);
        g.w = (S)L.hw[a];
        g.k = (uint32_t)L.hk[a];
        return g;
    }
    struct Item {
        int32_t m;
        S w;
        uint32_t o;
    };
    static __device__ Item none() { return Item{-1, 0, 0u}; }
    __device__ Item load(int32_t n, const Seg<S>& g, int32_t off) const
    {
        uint32_t e = lpins[g.b + off];
        Item it;
        it.m = (int32_t)(e & ~NOT_DEST);
        it.w = g.w;
        it.o = (g.nd && !(e & NOT_DEST)) ? g.k : 0u;
        if (prefilter) {
            int4 a = vst[n], b = vst[it.m];
            if ((int64_t)a.x + b.x > omega || (int64_t)a.y + b.y > phi) it.m = -1;
        }
        return it;
    }
    template <class Tb>
    __device__ bool put(int32_t, const Item& it, const Tb& t, Acc&) const
    {
        return it.m < 0 || t.add(it.m, it.w, it.o);
    }
    template <class Tb>
    __device__ bool elem(int32_t n, const Seg<S>& g, int32_t off, const Tb& t, Acc& acc) const
    {
        return put(n, load(n, g, off), t, acc);
    }
    __device__ void consider(int32_t n, int32_t m, int64_t s, uint32_t o, const Acc&, int64_t& bs,
                             int32_t& bk, uint32_t& bo) const
    {
        int4 a = vst[n], b = vst[m];
        bool valid = (int64_t)a.x + b.x <= omega && (int64_t)a.y + b.y <= phi &&
                     (int64_t)a.z + b.z - (int64_t)o <= delta;
        if (valid && better(s, m, bs, bk)) {
            bs = s;
            bk = m;
            bo = o;
        }
    }
    __device__ void write(int32_t n, int64_t bs, int32_t bk, uint32_t bo, const Acc&) const
    {
        uint8_t k = ac.kind[n];
        if (k == AK_NEW) return;
        if (k == AK_KEEP && better(ac.score[n], ac.cand[n], bs, bk)) {
            bs = ac.score[n];
            bk = ac.cand[n];
            bo = (uint32_t)ac.ov[n];
        } else if (k == AK_MERGED && bk != ac.cand[n]) {
            // w = cand is not the best valid new super-node: either it is
            // invalid (full histogram) or another one beats it (then that one
            // is the candidate); k_ac_check decides by w's validity
            ac.full[n] = bk < 0 ? 1 : 2;
            if (bk < 0) return;
        }
        cand[n] = bk;
        cscore[n] = bk < 0 ? 0 : bs;
        cov[n] = bk < 0 ? 0 : (int32_t)bo;
    }
};

void aff_carry_free(snnmap_hgraph* h)
{
    AffCarry& C = h->icar;
    for (void* p : {(void*)C.cand, (void*)C.score, (void*)C.ov, (void*)C.kind, (void*)C.full})
        if (p) cudaFreeAsync(p, h->stream);
    C = AffCarry{};
}

Status aff_carry(snnmap_hgraph* h, int32_t src)
{
    AffCarry& C = h->icar;
    C.level = -1;
    if (h->coarsen_mode == 1 || h->levels.size() != (size_t)src + 2) return Status{};
    const Level& F = h->levels[src];
    if (C.cap < h->levels[src + 1].V) {
        aff_carry_free(h);
        size_t n = (size_t)(h->cap_v > 0 ? h->cap_v : 1);
        cudaStream_t s = h->stream;
        bool ok = dev_malloc(&C.cand, n * 4, s) == cudaSuccess &&
                  dev_malloc(&C.score, n * 8, s) == cudaSuccess &&
                  dev_malloc(&C.ov, n * 4, s) == cudaSuccess &&
                  dev_malloc(&C.kind, n, s) == cudaSuccess &&
                  dev_malloc(&C.full, n, s) == cudaSuccess;
        if (!ok) {
            // no room: the next levels take full histograms
            cudaGetLastError();
            aff_carry_free(h);
            return Status{};
        }
        C.cap = (int64_t)n;
    }
    if (F.V > 0) {
        SNN_L k_ac_prep<<<grid_for(F.V, 256), 256, 0, h->stream>>>(F.V, F.cid, h->match, h->cand,
                                                                  h->cscore, h->cov, C);
        SNN_CUDA(cudaGetLastError());
    }
    C.level = src + 1;
    return Status{};
}

// S1 on a level whose candidates were carried: *done false when the full
// histogram is expected to be cheaper (nothing written then)
template <typename S>
static Status affinity_carried(snnmap_hgraph* h, Level& L, bool* done)
{
    *done = false;
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    AffCarry& C = h->icar;
    int64_t E = L.E;
    int32_t *vmin, *lcnt;
    int64_t *work, *loff;
    SNN_TRY(ar.alloc(&vmin, 4));
    SNN_TRY(ar.alloc(&work, 4));
    SNN_TRY(ar.alloc(&lcnt, E));
    SNN_TRY(ar.alloc(&loff, E + 1));
    SNN_TRY(fill_i32(vmin, 0x7fffffff, 2, s));
    SNN_CUDA(cudaMemsetAsync(vmin + 2, 0, 2 * sizeof(int32_t), s));
    SNN_CUDA(cudaMemsetAsync(work, 0, 4 * sizeof(int64_t), s));
    SNN_L k_level_min<<<grid_for(L.V, 256), 256, 0, s>>>(L, vmin);
    if (E > 0) SNN_HEDGE_LAUNCH(hedge_lanes(L.P, E), k_ac_count, E, s, L, C.kind, lcnt, work);
    SNN_L k_ac_fullwork<<<grid_for(L.V, 256), 256, 0, s>>>(L, C.kind, work + 1);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(scan_exclusive_i32_to_i64(lcnt, loff, E, loff + E, ar, s));
    int64_t hv[3];
    int32_t vm[4];
    SNN_CUDA(cudaMemcpyAsync(vm, vmin, sizeof(vm), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaMemcpyAsync(hv, work, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaMemcpyAsync(hv + 2, loff + E, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    // carried work: the new super-nodes' lists and the new super-nodes' full
    // histograms (plus those of the few MERGED vertices whose super-node no
    // longer suits them)
    int64_t full_work = h->extra.back().pair_terms + L.P;
    if (h->coarsen_mode != 2 && 4 * (hv[0] + hv[1]) >= 3 * full_work) return Status{};
    uint32_t* lpins;
    SNN_TRY(ar.alloc(&lpins, hv[2]));
    if (E > 0 && hv[2] > 0)
        SNN_L k_ac_fill<<<grid_for(E * 32, 256), 256, 0, s>>>(L, C.kind, loff, lpins);
    SNN_CUDA(cudaGetLastError());
    bool prefilter = 2 * (int64_t)vm[2] > h->prm.omega || 2 * (int64_t)vm[3] > h->prm.phi;
    int4* vst;
    SNN_TRY(ar.alloc(&vst, L.V));
    SNN_L k_pack_state<<<grid_for(L.V, 256), 256, 0, s>>>(L, vst);
    SNN_CUDA(cudaGetLastError());
    int64_t* cnt;
    SNN_TRY(ar.alloc(&cnt, HT_NCNT));
    if (L.V <= 0) SNN_CUDA(cudaMemsetAsync(cnt, 0, HT_NCNT * sizeof(int64_t), s));
    {
        AffNewPol<S> pol;
        pol.L = L;
        pol.V = L.V;
        pol.keys = h->last_pairs > 0 ? h->last_pairs : 1;
        pol.omega = h->prm.omega;
        pol.delta = h->prm.delta;
        pol.phi = h->prm.phi;
        pol.loff = loff;
        pol.lpins = lpins;
        pol.ac = C;
        pol.prefilter = prefilter;
        pol.vst = vst;
        pol.cand = h->cand;
        pol.cscore = h->cscore;
        pol.cov = h->cov;
        SNN_TRY(run_histogram(pol, ar, s, cnt, h->h_scal + 12, h->d_scal, h->tiers));
        SNN_CUDA(cudaMemcpyAsync(h->h_tier, cnt, HT_NCNT * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    }
    SNN_L k_ac_check<<<grid_for(L.V, 256), 256, 0, s>>>(L, C, h->prm.omega, h->prm.delta,
                                                        h->prm.phi);
    SNN_CUDA(cudaGetLastError());
    {
        AffPol<S> pol;
        pol.vmin = vmin;
        pol.prefilter = prefilter;
        pol.only = C.full;
        pol.vst = vst;
        pol.L = L;
        pol.V = L.V;
        pol.keys = L.V;
        pol.omega = h->prm.omega;
        pol.delta = h->prm.delta;
        pol.phi = h->prm.phi;
        pol.cand = h->cand;
        pol.cscore = h->cscore;
        pol.cov = h->cov;
        SNN_TRY(run_histogram(pol, ar, s, cnt, h->h_scal + 12, h->d_scal, h->tiers));
        SNN_CUDA(cudaMemcpyAsync(h->h_tier + TIER_SLOTS, cnt, HT_NCNT * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
    }
    h->extra.back().carried = 1;
    h->tier_level = (int32_t)h->extra.size() - 1;
    h->tier_form = 2;
    *done = true;
    return Status{};
}

Status coarsen_level(snnmap_hgraph* h, int32_t* n_cand, int32_t* n_pairs)
{
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    Level& L = h->levels.back();
    int32_t V = L.V;
    *n_cand = 0;
    *n_pairs = 0;
    h->have_matching = false;
    SNN_TRY(zero_scalars(h));
    if (V == 0) return Status{};
    {
        ProfScope prof(h, PS_AFFINITY);
        bool done = false;
        int32_t lev = (int32_t)h->levels.size() - 1;
        SNN_TRY(mat_affinity(h, lev, &done));
        if (!done && h->icar.level == lev) {
            if (h->wide) SNN_TRY(affinity_carried<unsigned long long>(h, L, &done));
            else SNN_TRY(affinity_carried<uint32_t>(h, L, &done));
        }
        if (done) {
        } else if (h->wide) {
            SNN_TRY(affinity<unsigned long long>(h, L));
        } else {
            SNN_TRY(affinity<uint32_t>(h, L));
        }
    }
    int g = grid_for(V, 256);
    std::unique_ptr<ProfScope> prof(new ProfScope(h, PS_MATCH));
    SNN_L k_count_cand<<<g, 256, 0, s>>>(V, h->cand, h->d_scal);
    SNN_CUDA(cudaGetLastError());
    int64_t* bestsc;
    int32_t *bc, *link, *nxt, *nxt2;
    uint8_t *par, *pj, *pj2;
    SNN_TRY(ar.alloc(&bestsc, V));
    SNN_TRY(ar.alloc(&bc, V));
    SNN_TRY(ar.alloc(&link, V));
    SNN_TRY(ar.alloc(&par, V));
    SNN_TRY(fill_i64(bestsc, INT64_MIN, V, s));
    SNN_TRY(fill_i32(bc, 0x7fffffff, V, s));
    SNN_L k_child_best_score<<<g, 256, 0, s>>>(V, h->cand, h->cscore, bestsc);
    SNN_L k_child_best_id<<<g, 256, 0, s>>>(V, h->cand, h->cscore, bestsc, bc);
    SNN_L k_link<<<g, 256, 0, s>>>(V, h->cand, bc, link);
    SNN_L k_walk<<<g, 256, 0, s>>>(V, link, par, h->d_scal);
    SNN_CUDA(cudaGetLastError());
    prof.reset();
    SNN_TRY(read_scalars(h));
    *n_cand = (int32_t)h->h_scal[SC_A];
    int64_t unresolved = h->h_scal[SC_B];
    if (*n_cand == 0) return Status{};
    if (unresolved > 0) {
        SNN_TRY(ar.alloc(&nxt, V));
        SNN_TRY(ar.alloc(&nxt2, V));
        SNN_TRY(ar.alloc(&pj, V));
        SNN_TRY(ar.alloc(&pj2, V));
        SNN_L k_jump_init<<<g, 256, 0, s>>>(V, link, nxt, pj);
        SNN_CUDA(cudaGetLastError());
        for (int it = 0; it < 40; it++) {
            SNN_TRY(zero_scalars(h));
            SNN_L k_jump<<<g, 256, 0, s>>>(V, nxt, pj, nxt2, pj2, h->d_scal);
            SNN_CUDA(cudaGetLastError());
            std::swap(nxt, nxt2);
            std::swap(pj, pj2);
            SNN_TRY(read_scalars(h));
            if (h->h_scal[SC_B] == 0) break;
        }
        SNN_L k_jump_done<<<g, 256, 0, s>>>(V, pj, par);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(zero_scalars(h));
    prof.reset(new ProfScope(h, PS_MATCH));
    SNN_L k_match_finish<<<g, 256, 0, s>>>(V, h->cand, bc, par, h->match, h->d_scal);
    SNN_CUDA(cudaGetLastError());
    prof.reset();
    SNN_TRY(read_scalars(h));
    *n_pairs = (int32_t)h->h_scal[SC_C];
    h->have_matching = true;
    h->last_pairs = *n_pairs;
    return Status{};
}

// Eq. matching over any candidate pseudo-forest, for callers outside
// coarsening: the same kernels as coarsen_level, with its own scalars. A
// vertex without a candidate may still have children (never so in
// coarsening, where validity is symmetric); it then tops its chain at even
// distance and takes its best child, as the equation's second case says.
Status match_forest(int32_t V, const int32_t* cand, const int64_t* cscore, int32_t* match,
                    int64_t* d_scal, Arena& ar, cudaStream_t s, int64_t* n_pairs)
{
    *n_pairs = 0;
    if (V <= 0) return Status{};
    int g = grid_for(V, 256);
    int64_t h_scal[SC_COUNT];
    int64_t* bestsc;
    int32_t *bc, *link, *nxt, *nxt2;
    uint8_t *par, *pj, *pj2;
    SNN_TRY(ar.alloc(&bestsc, V));
    SNN_TRY(ar.alloc(&bc, V));
    SNN_TRY(ar.alloc(&link, V));
    SNN_TRY(ar.alloc(&par, V));
    SNN_CUDA(cudaMemsetAsync(d_scal, 0, SC_COUNT * sizeof(int64_t), s));
    SNN_TRY(fill_i64(bestsc, INT64_MIN, V, s));
    SNN_TRY(fill_i32(bc, 0x7fffffff, V, s));
    SNN_L k_child_best_score<<<g, 256, 0, s>>>(V, cand, cscore, bestsc);
    SNN_L k_child_best_id<<<g, 256, 0, s>>>(V, cand, cscore, bestsc, bc);
    SNN_L k_link<<<g, 256, 0, s>>>(V, cand, bc, link);
    SNN_L k_walk<<<g, 256, 0, s>>>(V, link, par, d_scal);
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaMemcpyAsync(h_scal, d_scal, sizeof(h_scal), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (h_scal[SC_B] > 0) {
        SNN_TRY(ar.alloc(&nxt, V));
        SNN_TRY(ar.alloc(&nxt2, V));
        SNN_TRY(ar.alloc(&pj, V));
        SNN_TRY(ar.alloc(&pj2, V));
        SNN_L k_jump_init<<<g, 256, 0, s>>>(V, link, nxt, pj);
        SNN_CUDA(cudaGetLastError());
        for (int it = 0; it < 40; it++) {
            SNN_CUDA(cudaMemsetAsync(d_scal, 0, SC_COUNT * sizeof(int64_t), s));
            SNN_L k_jump<<<g, 256, 0, s>>>(V, nxt, pj, nxt2, pj2, d_scal);
            SNN_CUDA(cudaGetLastError());
            std::swap(nxt, nxt2);
            std::swap(pj, pj2);
            SNN_CUDA(cudaMemcpyAsync(h_scal, d_scal, sizeof(h_scal), cudaMemcpyDeviceToHost, s));
            SNN_CUDA(cudaStreamSynchronize(s));
            if (h_scal[SC_B] == 0) break;
        }
        SNN_L k_jump_done<<<g, 256, 0, s>>>(V, pj, par);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_CUDA(cudaMemsetAsync(d_scal, 0, SC_COUNT * sizeof(int64_t), s));
    SNN_L k_match_finish<<<g, 256, 0, s>>>(V, cand, bc, par, match, d_scal);
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaMemcpyAsync(h_scal, d_scal, sizeof(h_scal), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    *n_pairs = h_scal[SC_C];
    return Status{};
}

}  // namespace snn
