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

constexpr int AFF_WARPS = 8;
constexpr int AFF_T = 512;                 // slots per warp table
constexpr int AFF_LOAD = AFF_T * 3 / 4;    // distinct neighbours before a warp gives up
constexpr int AFF_BT = 8192;               // slots of the block shared table
constexpr int AFF_BLOAD = AFF_BT * 3 / 4;
constexpr int AFF_BTHREADS = 256;
constexpr int MATCH_WALK = 64;

// neighbour terms of vertex n: pins of its incident hyperedges
template <typename S>
struct AffVis {
    const Level& L;
    int32_t n;
    const Table<S>& t;
    __device__ Seg<S> seg(int64_t i) const
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
    __device__ bool elem(const Seg<S>& g, int32_t off) const
    {
        int32_t m = L.hpins[g.b + off];
        if (m == n) return true;
        int md = off != 0 || g.sd;   // pin 0 is the source
        return t.add(m, g.w, (g.nd && md) ? g.k : 0u);
    }
};

// Best valid neighbour among the table's used slots [u0, nused) taken every
// `stride`; resets those slots. Per-thread result.
template <typename S>
__device__ void scan_table(const Level& L, int32_t n, const Table<S>& t, int32_t u0, int32_t nused,
                           int32_t stride, int32_t omega, int32_t delta, int32_t phi,
                           int64_t& bs, int32_t& bm, uint32_t& bo)
{
    int64_t sz = L.vsize[n], ip = L.vinpins[n], ic = L.vincnt[n];
    for (int32_t u = u0; u < nused; u += stride) {
        int32_t slot = t.used[u];
        int32_t m = t.key[slot];
        int64_t s = (int64_t)t.sc[slot];
        uint32_t o = t.ov[slot];
        t.key[slot] = -1;
        t.sc[slot] = 0;
        t.ov[slot] = 0;
        bool valid = sz + L.vsize[m] <= omega && ip + L.vinpins[m] <= phi &&
                     ic + L.vincnt[m] - (int64_t)o <= delta;
        if (valid && better(s, m, bs, bm)) {
            bs = s;
            bm = m;
            bo = o;
        }
    }
}

template <typename S>
__global__ void __launch_bounds__(AFF_WARPS * 32)
    k_aff_warp(Level L, int32_t omega, int32_t delta, int32_t phi, int32_t* cand, int64_t* cscore,
               int32_t* cov, int32_t* heavy, int64_t* scal)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ int32_t nfill[AFF_WARPS];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Table<S> t = carve_table<S>(smem_raw + (size_t)warp * table_bytes<S>(AFF_T), AFF_T, &nfill[warp]);
    for (int i = lane; i < AFF_T; i += 32) {
        t.key[i] = -1;
        t.sc[i] = 0;
        t.ov[i] = 0;
    }
    int64_t gw = blockIdx.x * (int64_t)AFF_WARPS + warp;
    int64_t nw = (int64_t)gridDim.x * AFF_WARPS;
    for (int64_t n = gw; n < L.V; n += nw) {
        if (lane == 0) nfill[warp] = 0;
        __syncwarp();
        AffVis<S> vis{L, (int32_t)n, t};
        bool ok = warp_flat_visit<S>(vis, L.voff[n], L.voff[n + 1], 32, &nfill[warp], AFF_LOAD);
        __syncwarp();
        int32_t nused = nfill[warp];
        if (!ok || nused > AFF_T) {
            // reset the whole table and hand the vertex to the block tier
            for (int i = lane; i < AFF_T; i += 32) {
                t.key[i] = -1;
                t.sc[i] = 0;
                t.ov[i] = 0;
            }
            if (lane == 0) {
                int32_t pos = atomicAdd((int*)&scal[SC_E], 1);
                heavy[pos] = (int32_t)n;
            }
            __syncwarp();
            continue;
        }
        int64_t bs = 0;
        int32_t bm = -1;
        uint32_t bo = 0;
        scan_table<S>(L, (int32_t)n, t, lane, nused, 32, omega, delta, phi, bs, bm, bo);
        warp_argmax(bs, bm, bo);
        if (lane == 0) {
            cand[n] = bm;
            cscore[n] = bm < 0 ? 0 : bs;
            cov[n] = bm < 0 ? 0 : (int32_t)bo;
        }
        __syncwarp();
    }
}

// Block tier: one block per listed vertex. Shared table (gtab == nullptr) or
// a per-block slice of a global table of `cap` slots (key -1 / zero sums on
// entry; every vertex resets what it used). Vertices overflowing the shared
// table are appended to `next`.
template <typename S>
__global__ void __launch_bounds__(AFF_BTHREADS)
    k_aff_block(Level L, int32_t omega, int32_t delta, int32_t phi, int32_t* cand,
                int64_t* cscore, int32_t* cov, const int32_t* list, const int64_t* count_slot,
                int32_t* next, int64_t* next_slot, unsigned char* gtab, int64_t cap)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ int32_t nfill;
    __shared__ int sh_fail;
    __shared__ int64_t rs[AFF_BTHREADS / 32];
    __shared__ int32_t rm[AFF_BTHREADS / 32];
    __shared__ uint32_t ro[AFF_BTHREADS / 32];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = AFF_BTHREADS / 32;
    int64_t tcap = gtab ? cap : AFF_BT;
    int32_t limit = gtab ? (int32_t)(cap - 1) : AFF_BLOAD;
    Table<S> t = carve_table<S>(gtab ? gtab + (size_t)blockIdx.x * table_bytes<S>(cap) : smem_raw,
                                (int32_t)tcap, &nfill);
    if (!gtab) {
        for (int i = threadIdx.x; i < AFF_BT; i += AFF_BTHREADS) {
            t.key[i] = -1;
            t.sc[i] = 0;
            t.ov[i] = 0;
        }
    }
    int32_t cnt = (int32_t)*count_slot;
    for (int32_t idx = blockIdx.x; idx < cnt; idx += gridDim.x) {
        int32_t n = list[idx];
        if (threadIdx.x == 0) {
            nfill = 0;
            sh_fail = 0;
        }
        __syncthreads();
        AffVis<S> vis{L, n, t};
        bool ok = warp_flat_visit<S>(vis, L.voff[n] + 32 * warp, L.voff[n + 1], 32 * nwarps,
                                     &nfill, limit);
        if (!ok) atomicOr(&sh_fail, 1);
        __syncthreads();
        int32_t nused = nfill;
        if (sh_fail || nused > limit) {
            for (int64_t i = threadIdx.x; i < tcap; i += AFF_BTHREADS) {
                t.key[i] = -1;
                t.sc[i] = 0;
                t.ov[i] = 0;
            }
            if (threadIdx.x == 0 && next) {
                int32_t pos = atomicAdd((int*)next_slot, 1);
                next[pos] = n;
            }
            __syncthreads();
            continue;
        }
        int64_t bs = 0;
        int32_t bm = -1;
        uint32_t bo = 0;
        scan_table<S>(L, n, t, threadIdx.x, nused, AFF_BTHREADS, omega, delta, phi, bs, bm, bo);
        warp_argmax(bs, bm, bo);
        if (lane == 0) {
            rs[warp] = bs;
            rm[warp] = bm;
            ro[warp] = bo;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nwarps; w++)
                if (better(rs[w], rm[w], bs, bm)) {
                    bs = rs[w];
                    bm = rm[w];
                    bo = ro[w];
                }
            cand[n] = bm;
            cscore[n] = bm < 0 ? 0 : bs;
            cov[n] = bm < 0 ? 0 : (int32_t)bo;
        }
        __syncthreads();
    }
}

template <typename S>
constexpr size_t aff_warp_smem()
{
    return (size_t)AFF_WARPS * table_bytes<S>(AFF_T);
}

template <typename S>
constexpr size_t aff_block_smem()
{
    return table_bytes<S>(AFF_BT);
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

template <typename S>
static Status affinity(snnmap_hgraph* h, Level& L)
{
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    const snnmap_params& p = h->prm;
    int32_t V = L.V;
    int32_t *heavy, *heavy2;
    SNN_TRY(ar.alloc(&heavy, V));
    SNN_TRY(ar.alloc(&heavy2, V));
    static bool attrs = false;
    if (!attrs) {
        SNN_CUDA(cudaFuncSetAttribute(k_aff_warp<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)aff_warp_smem<S>()));
        SNN_CUDA(cudaFuncSetAttribute(k_aff_block<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)aff_block_smem<S>()));
        attrs = true;
    }
    int grid = (int)std::min<int64_t>(ceil_div(V, AFF_WARPS), 152 * 3 * 8);
    SNN_L k_aff_warp<S><<<grid, AFF_WARPS * 32, aff_warp_smem<S>(), s>>>(
        L, p.omega, p.delta, p.phi, h->cand, h->cscore, h->cov, heavy, h->d_scal);
    SNN_CUDA(cudaGetLastError());
    SNN_L k_aff_block<S><<<152, AFF_BTHREADS, aff_block_smem<S>(), s>>>(
        L, p.omega, p.delta, p.phi, h->cand, h->cscore, h->cov, heavy, h->d_scal + SC_E, heavy2,
        h->d_scal + SC_F, nullptr, 0);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(read_scalars(h));
    int64_t n2 = h->h_scal[SC_F];
    if (n2 > 0) {
        int64_t cap = 1024;
        while (cap < 2 * (int64_t)V) cap <<= 1;
        int64_t per = (int64_t)table_bytes<S>(cap);
        int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(16, ((int64_t)1 << 30) / per));
        if (blocks > n2) blocks = (int)n2;
        unsigned char* gtab;
        SNN_TRY(ar.alloc(&gtab, blocks * per));
        SNN_TRY(init_global_tables<S>(gtab, blocks, cap, s));
        SNN_L k_aff_block<S><<<blocks, AFF_BTHREADS, 0, s>>>(
            L, p.omega, p.delta, p.phi, h->cand, h->cscore, h->cov, heavy2, h->d_scal + SC_F,
            nullptr, nullptr, gtab, cap);
        SNN_CUDA(cudaGetLastError());
    }
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
        if (h->wide) {
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

}  // namespace snn
