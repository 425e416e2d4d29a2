// Contraction (Sec. 4.1: each level's hypergraph is materialized from its
// predecessor while every super-node carries its constrained state).
//
// 1. Coarse ids: a vertex represents its pair if it is unmatched or the
//    lower id of the pair; cid = rank of the representative (exclusive scan).
// 2. Super-node state: size, inbound pins and internal axons add up over the
//    members; the size of the merged inbound set is the paper's
//    in_count(n) + in_count(m) - shared(n, m), the shared count being the
//    candidate overlap of the pair. A level rebuilt through composed maps
//    (no matching at hand) recomputes it from the coarse level as internal
//    axons + the k of every coarse hyperedge the super-node is a
//    destination of.
// 3. Per hyperedge (segmented sort): s' = cid(source), destinations mapped
//    through cid, sorted, made unique; s' among them sets selfdst and is
//    removed. A hyperedge left with no destination is dropped and its
//    multiplicity k moves into the source super-node's internal count.
// 4. Duplicate hyperedges (same s', selfdst, destination list) merge: a
//    stable radix sort on (s', 32-bit content hash) brings candidates
//    together, an exact comparison of the contents decides, and the first
//    of each equal group becomes the coarse hyperedge; omega and k add up.
// 5. Compaction into the next level's arrays, then its incidence lists.
//
// The same routine (build_coarse) materializes any level l from a resident
// level j < l through the composed map cid_{l-1} o ... o cid_j: the image of
// an axon does not depend on the order of the merges, so a level whose
// arrays were released to save memory is rebuilt exactly.
#include "internal.cuh"

#include <memory>

namespace snn {

__global__ void k_rep_flags(int32_t V, const int32_t* __restrict__ match, int32_t* isrep)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = match[n];
        isrep[n] = (m < 0 || (int32_t)n < m) ? 1 : 0;
    }
}

struct NextState {
    int32_t *size, *inpins, *inint;
};

__global__ void k_cid_map(int32_t V, const int32_t* __restrict__ match,
                          const int32_t* __restrict__ repidx, int32_t* cid)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = match[n];
        cid[n] = repidx[(m < 0 || (int32_t)n < m) ? (int32_t)n : m];
    }
}

// member sums per coarse vertex
__global__ void k_sum_state(Level S, const int32_t* __restrict__ map, NextState ns)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < S.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = map[n];
        atomicAdd(&ns.size[u], S.vsize[n]);
        atomicAdd(&ns.inpins[u], S.vinpins[n]);
        if (S.vinint[n]) atomicAdd(&ns.inint[u], S.vinint[n]);
    }
}

// in_count += k(a) for every destination of every hyperedge a (vincnt must
// hold the internal counts on entry)
__global__ void k_in_count(Level N)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = gw; a < N.E; a += nw) {
        int64_t b = N.hoff[a], e = N.hoff[a + 1];
        int32_t k = N.hk[a];
        for (int64_t j = b + 1 + lane; j < e; j += 32) atomicAdd(&N.vincnt[N.hpins[j]], k);
        if (lane == 0 && N.hsd[a]) atomicAdd(&N.vincnt[N.hpins[b]], k);
    }
}

// in_count of the next level straight from a matching: an unmatched vertex
// keeps its count; a pair's super-node has in_count(n) + in_count(m) -
// shared(n, m), the shared count being the candidate overlap of the member
// whose candidate is the other (pairs are matched along candidate arcs)
__global__ void k_in_count_pairs(Level S, const int32_t* __restrict__ map,
                                 const int32_t* __restrict__ match, const int32_t* __restrict__ cand,
                                 const int32_t* __restrict__ cov, int32_t* incnt_next)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < S.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = match[n];
        if (m < 0) {
            incnt_next[map[n]] = S.vincnt[n];
        } else if ((int32_t)n < m) {
            int32_t ov = cand[n] == m ? cov[n] : cov[m];
            incnt_next[map[n]] = S.vincnt[n] + S.vincnt[m] - ov;
        }
    }
}

__global__ void k_compose(int64_t n, int32_t* c, const int32_t* __restrict__ next)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        c[i] = next[c[i]];
}

// Remaps one hyperedge's destinations through cid; output at the same
// offsets in tpins (source first), length tlen (0: dropped).
struct ContractJob {
    const int64_t* hoff;
    const int32_t* hpins;
    const uint8_t* hsd;
    const int32_t* hk;
    const int32_t* cid;
    int32_t* tpins;
    int32_t* tlen;
    uint8_t* tsd;
    uint32_t* thash;
    int32_t* inint_next;     // may be null (nothing recorded for dropped hyperedges)
    bool discard_self = false;   // G_P: a destination in the source's part is discarded
                                 // without marking selfdst
    __device__ int len(int32_t a) const { return (int)(hoff[a + 1] - hoff[a] - 1); }
    __device__ uint32_t load(int32_t a, int i) const
    {
        return (uint32_t)cid[hpins[hoff[a] + 1 + i]];
    }
    __device__ void finish(int32_t a, const uint32_t* s, int n) const
    {
        int lane = threadIdx.x & 31;
        int64_t base = hoff[a];
        uint32_t sp = (uint32_t)cid[hpins[base]];
        int cnt = 0;
        int sd = discard_self ? 0 : hsd[a];
        uint64_t hsum = 0;
        unsigned lt = lanemask_lt();
        for (int c = 0; c < n; c += 32) {
            int i = c + lane;
            bool valid = i < n;
            uint32_t v = valid ? s[i] : KEY_PAD;
            bool isnew = valid && (i == 0 || s[i - 1] != v);
            bool self = valid && v == sp;
            bool keep = isnew && !self;
            unsigned mk = __ballot_sync(FULL, keep);
            if (keep) {
                tpins[base + 1 + cnt + __popc(mk & lt)] = (int32_t)v;
                hsum += mix64(v);
            }
            cnt += __popc(mk);
            if (__any_sync(FULL, self) && !discard_self) sd = 1;
        }
        hsum = warp_sum(hsum);
        if (lane == 0) {
            tpins[base] = (int32_t)sp;
            if (cnt == 0) {
                tlen[a] = 0;
                if (sd && inint_next) atomicAdd(&inint_next[sp], hk[a]);
            } else {
                tlen[a] = 1 + cnt;
                tsd[a] = (uint8_t)sd;
                uint64_t hh = hsum + mix64(0x5bd1e995ull + (uint64_t)sd) + mix64((uint64_t)cnt << 1);
                thash[a] = (uint32_t)(hh ^ (hh >> 32));
            }
        }
    }
    __device__ void finish_thread(int32_t a, const uint32_t* s, int n, int st) const
    {
        int64_t base = hoff[a];
        uint32_t sp = (uint32_t)cid[hpins[base]];
        int cnt = 0, sd = discard_self ? 0 : hsd[a];
        uint64_t hsum = 0;
        for (int i = 0; i < n; i++) {
            uint32_t v = s[(i) * st];
            if (i > 0 && s[(i - 1) * st] == v) continue;
            if (v == sp) {
                if (!discard_self) sd = 1;
                continue;
            }
            tpins[base + 1 + cnt++] = (int32_t)v;
            hsum += mix64(v);
        }
        tpins[base] = (int32_t)sp;
        if (cnt == 0) {
            tlen[a] = 0;
            if (sd && inint_next) atomicAdd(&inint_next[sp], hk[a]);
        } else {
            tlen[a] = 1 + cnt;
            tsd[a] = (uint8_t)sd;
            uint64_t hh = hsum + mix64(0x5bd1e995ull + (uint64_t)sd) + mix64((uint64_t)cnt << 1);
            thash[a] = (uint32_t)(hh ^ (hh >> 32));
        }
    }
};

__global__ void k_dedup_keys(int32_t E, const int32_t* __restrict__ tlen,
                             const int64_t* __restrict__ hoff, const int32_t* __restrict__ tpins,
                             const uint32_t* __restrict__ thash, uint64_t dropped_hi,
                             uint64_t* keys, uint32_t* vals)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < E;
         a += (int64_t)gridDim.x * blockDim.x) {
        uint64_t hi = tlen[a] > 0 ? (uint64_t)(uint32_t)tpins[hoff[a]] : dropped_hi;
        keys[a] = (hi << 32) | (tlen[a] > 0 ? thash[a] : 0u);
        vals[a] = (uint32_t)a;
    }
}

__global__ void k_run_heads(int32_t E, const uint64_t* __restrict__ keys, int32_t* headpos)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x)
        headpos[i] = (i == 0 || keys[i] != keys[i - 1]) ? (int32_t)i : 0;
}

__device__ __forceinline__ bool same_content(int32_t a, int32_t b, const int64_t* hoff,
                                             const int32_t* tpins, const int32_t* tlen,
                                             const uint8_t* tsd)
{
    if (tlen[a] != tlen[b] || tsd[a] != tsd[b]) return false;
    const int32_t* pa = tpins + hoff[a];
    const int32_t* pb = tpins + hoff[b];
    for (int32_t i = 0; i < tlen[a]; i++)
        if (pa[i] != pb[i]) return false;
    return true;
}

// rep[i] = first position j of i's run (equal keys) whose content equals i's
__global__ void k_dedup_rep(int32_t E, const uint64_t* __restrict__ keys,
                            const uint32_t* __restrict__ vals, const int32_t* __restrict__ runstart,
                            const int64_t* __restrict__ hoff, const int32_t* __restrict__ tpins,
                            const int32_t* __restrict__ tlen, const uint8_t* __restrict__ tsd,
                            int32_t* rep, int32_t* head)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = (int32_t)vals[i];
        if (tlen[a] == 0) {
            rep[i] = -1;
            head[i] = 0;
            continue;
        }
        int32_t j = runstart[i];
        while (j < i && !same_content((int32_t)vals[j], a, hoff, tpins, tlen, tsd)) j++;
        rep[i] = j;
        head[i] = j == i ? 1 : 0;
    }
}

__global__ void k_dedup_accum(int32_t E, const uint32_t* __restrict__ vals,
                              const int32_t* __restrict__ rep, const int32_t* __restrict__ gidh,
                              const int32_t* __restrict__ tlen, const int64_t* __restrict__ hw,
                              const int32_t* __restrict__ hk, int64_t* tw, int32_t* tk,
                              int64_t* newlen, int32_t* gid)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = rep[i];
        if (r < 0) {
            gid[i] = -1;
            continue;
        }
        int32_t g = gidh[r];
        int32_t a = (int32_t)vals[i];
        gid[i] = g;
        atomicAdd((unsigned long long*)&tw[g], (unsigned long long)hw[a]);
        atomicAdd(&tk[g], hk[a]);
        if (r == i) newlen[g] = tlen[a];
    }
}

// a group of G lanes per hyperedge
template <int G>
__global__ void k_dedup_emit(int32_t E, const uint32_t* __restrict__ vals,
                             const int32_t* __restrict__ rep, const int32_t* __restrict__ gid,
                             const int64_t* __restrict__ hoff, const int32_t* __restrict__ tpins,
                             const int32_t* __restrict__ tlen, const uint8_t* __restrict__ tsd,
                             const int64_t* __restrict__ tw, const int32_t* __restrict__ tk,
                             const int64_t* __restrict__ newoff, Level N)
{
    int lane = threadIdx.x & (G - 1);
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) / G;
    for (int64_t i = gw; i < E; i += nw) {
        if (rep[i] != (int32_t)i) continue;
        int32_t a = (int32_t)vals[i];
        int32_t g = gid[i];
        int64_t dst = newoff[g], src = hoff[a];
        int32_t len = tlen[a];
        for (int32_t j = lane; j < len; j += G) N.hpins[dst + j] = tpins[src + j];
        if (lane == 0) {
            N.hoff[g] = dst;
            N.hsd[g] = tsd[a];
            N.hw[g] = tw[g];
            N.hk[g] = tk[g];
        }
    }
}

__global__ void k_set_off_end(int64_t* hoff, int32_t E, int64_t P) { hoff[E] = P; }

// Materializes levels[dst] from the resident levels[src] through `map`
// (int32[V(src)] into the new level's ids); *d_V2 (device) is its vertex
// count. If levels[dst] already records sizes (a released level being
// rebuilt), the rebuilt sizes must match them.
Status build_coarse(snnmap_hgraph* h, int32_t src, const int32_t* map, const int64_t* d_V2,
                    int32_t dst, const int32_t* match, const int32_t* cand, const int32_t* cov)
{
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    Level& L = h->levels[src];
    LevelExtra& X = h->extra[src];
    int32_t V = L.V, E = L.E;
    SNN_TRY(zero_scalars(h));
    std::unique_ptr<ProfScope> prof(new ProfScope(h, PS_CONTRACT));
    NextState ns;
    SNN_TRY(ar.alloc(&ns.size, V));
    SNN_TRY(ar.alloc(&ns.inpins, V));
    SNN_TRY(ar.alloc(&ns.inint, V));
    if (V > 0) {
        SNN_CUDA(cudaMemsetAsync(ns.size, 0, (size_t)V * 4, s));
        SNN_CUDA(cudaMemsetAsync(ns.inpins, 0, (size_t)V * 4, s));
        SNN_CUDA(cudaMemsetAsync(ns.inint, 0, (size_t)V * 4, s));
        SNN_L k_sum_state<<<grid_for(V, 256), 256, 0, s>>>(L, map, ns);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_CUDA(cudaMemcpyAsync(h->d_scal + SC_A, d_V2, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));

    // per-hyperedge remap, sort, unique
    int32_t *tpins, *tlen;
    uint8_t* tsd;
    uint32_t* thash;
    SNN_TRY(ar.alloc(&tpins, L.P));
    SNN_TRY(ar.alloc(&tlen, E));
    SNN_TRY(ar.alloc(&tsd, E));
    SNN_TRY(ar.alloc(&thash, E));
    ContractJob job{L.hoff, L.hpins, L.hsd, L.hk, map, tpins, tlen, tsd, thash, ns.inint};
    SNN_TRY(seg_run(job, X.seg, E, ar, s));

    // duplicate hyperedges
    uint64_t *keys, *keys2;
    uint32_t *vals, *vals2;
    int32_t *headpos, *runstart, *rep, *head, *gidh, *gid, *tk;
    int64_t *tw, *newlen, *newoff;
    SNN_TRY(ar.alloc(&keys, E));
    SNN_TRY(ar.alloc(&keys2, E));
    SNN_TRY(ar.alloc(&vals, E));
    SNN_TRY(ar.alloc(&vals2, E));
    SNN_TRY(ar.alloc(&headpos, E));
    SNN_TRY(ar.alloc(&runstart, E));
    SNN_TRY(ar.alloc(&rep, E));
    SNN_TRY(ar.alloc(&head, E));
    SNN_TRY(ar.alloc(&gidh, E));
    SNN_TRY(ar.alloc(&gid, E));
    SNN_TRY(ar.alloc(&tk, E));
    SNN_TRY(ar.alloc(&tw, E));
    SNN_TRY(ar.alloc(&newlen, E));
    SNN_TRY(ar.alloc(&newoff, E));
    int ge = grid_for(E, 256);
    int hibits = bits_for((uint64_t)V);
    if (E > 0) {
        SNN_L k_dedup_keys<<<ge, 256, 0, s>>>(E, tlen, L.hoff, tpins, thash, (uint64_t)V, keys, vals);
        SNN_CUDA(cudaGetLastError());
        SNN_TRY(radix_sort_pairs(keys, vals, keys2, vals2, E, 32 + hibits, ar, s));
        SNN_L k_run_heads<<<ge, 256, 0, s>>>(E, keys, headpos);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(scan_inclusive_max_i32(headpos, runstart, E, ar, s));
    if (E > 0) {
        SNN_L k_dedup_rep<<<ge, 256, 0, s>>>(E, keys, vals, runstart, L.hoff, tpins, tlen, tsd, rep, head);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(scan_exclusive_i32(head, gidh, E, (int32_t*)(h->d_scal + SC_B), ar, s));
    if (E > 0) {
        SNN_CUDA(cudaMemsetAsync(tw, 0, (size_t)E * sizeof(int64_t), s));
        SNN_CUDA(cudaMemsetAsync(tk, 0, (size_t)E * sizeof(int32_t), s));
        SNN_CUDA(cudaMemsetAsync(newlen, 0, (size_t)E * sizeof(int64_t), s));
        SNN_L k_dedup_accum<<<ge, 256, 0, s>>>(E, vals, rep, gidh, tlen, L.hw, L.hk, tw, tk, newlen, gid);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(scan_exclusive_i64(newlen, newoff, E, h->d_scal + SC_C, ar, s));
    prof.reset();
    SNN_TRY(read_scalars(h));
    int32_t V2 = (int32_t)h->h_scal[SC_A];
    int32_t E2 = (int32_t)(h->h_scal[SC_B] & 0xffffffff);
    int64_t P2 = h->h_scal[SC_C];

    Level& N = h->levels[dst];
    LevelExtra& NX = h->extra[dst];
    if (N.E != 0 || N.P != 0 || N.V != 0) {
        if (N.V != V2 || N.E != E2 || N.P != P2)
            return Status{SNNMAP_ERR_CUDA, "rebuilt level differs from the released one"};
    }
    SNN_TRY(level_alloc(h, N, NX, V2, E2, P2));
    N.maxlen = L.maxlen;
    prof.reset(new ProfScope(h, PS_CONTRACT));
    if (V2 > 0) {
        SNN_CUDA(cudaMemcpyAsync(N.vsize, ns.size, (size_t)V2 * 4, cudaMemcpyDeviceToDevice, s));
        SNN_CUDA(cudaMemcpyAsync(N.vinpins, ns.inpins, (size_t)V2 * 4, cudaMemcpyDeviceToDevice, s));
        SNN_CUDA(cudaMemcpyAsync(N.vinint, ns.inint, (size_t)V2 * 4, cudaMemcpyDeviceToDevice, s));
        if (!match)
            SNN_CUDA(cudaMemcpyAsync(N.vincnt, ns.inint, (size_t)V2 * 4, cudaMemcpyDeviceToDevice, s));
    }
    if (match && V > 0) {
        SNN_L k_in_count_pairs<<<grid_for(V, 256), 256, 0, s>>>(L, map, match, cand, cov, N.vincnt);
        SNN_CUDA(cudaGetLastError());
    }
    if (E > 0) {
        SNN_HEDGE_LAUNCH(hedge_lanes(L.P, L.E), k_dedup_emit, E, s, E, vals, rep, gid, L.hoff, tpins,
                         tlen, tsd, tw, tk, newoff, N);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_L k_set_off_end<<<1, 1, 0, s>>>(N.hoff, E2, P2);
    SNN_CUDA(cudaGetLastError());
    if (E2 > 0 && !match) {
        SNN_L k_in_count<<<grid_for((int64_t)E2 * 32, 256), 256, 0, s>>>(N);
        SNN_CUDA(cudaGetLastError());
    }
    prof.reset();
    SNN_TRY(build_incidence(h, N));
    SNN_CUDA(cudaMemsetAsync(h->d_scal + SC_W2, 0, sizeof(int64_t), s));
    SNN_TRY(seg_classify(N.hoff, E2, N.maxlen, NX.seg, ar, s, h->d_scal + SC_W2));
    SNN_TRY(read_scalars(h));
    NX.pair_terms = h->h_scal[SC_W2];
    ar.reset();
    return Status{};
}

Status contract_level(snnmap_hgraph* h)
{
    if (!h->have_matching || h->last_pairs <= 0) return Status{SNNMAP_ERR_STATE, "no matching to contract"};
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    int32_t src = (int32_t)h->levels.size() - 1;
    Level& L = h->levels[src];
    int32_t V = L.V;
    int32_t *isrep, *repidx;
    int64_t* d_V2;
    SNN_TRY(ar.alloc(&isrep, V));
    SNN_TRY(ar.alloc(&repidx, V));
    SNN_TRY(ar.alloc(&d_V2, 1));
    SNN_CUDA(cudaMemsetAsync(d_V2, 0, sizeof(int64_t), s));
    {
        ProfScope prof(h, PS_CONTRACT);
        SNN_L k_rep_flags<<<grid_for(V, 256), 256, 0, s>>>(V, h->match, isrep);
        SNN_CUDA(cudaGetLastError());
        SNN_TRY(scan_exclusive_i32(isrep, repidx, V, (int32_t*)d_V2, ar, s));
        SNN_L k_cid_map<<<grid_for(V, 256), 256, 0, s>>>(V, h->match, repidx, L.cid);
        SNN_CUDA(cudaGetLastError());
    }
    h->levels.emplace_back();
    h->extra.emplace_back();
    SNN_TRY(build_coarse(h, src, h->levels[src].cid, d_V2, src + 1, h->match, h->cand, h->cov));
    h->have_matching = false;
    ProfScope prof(h, PS_AFFINITY);
    if (h->mat.level == src) SNN_TRY(mat_descend(h, src));
    if (h->mat.level != src + 1) SNN_TRY(aff_carry(h, src));
    return Status{};
}

// ---------------------------------------------------------------------------
// G_P (Sec. 3, Partitioning Definition): the image of every axon under rho,
// the source's partition as source, the other partitions of its pins as
// destinations (a destination in the source's partition is discarded, which
// breaks the self-cycle); axons with equal images merge and eta sums their
// omega. An axon whose pins all share one partition keeps no destination:
// it is left out of A and its omega reported as internal weight.

__global__ void k_gp_internal(int32_t E, const int32_t* __restrict__ tlen,
                              const int64_t* __restrict__ hw, int64_t* out)
{
    int64_t w = 0;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < E;
         a += (int64_t)gridDim.x * blockDim.x)
        if (tlen[a] == 0) w += hw[a];
    w = warp_sum(w);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd((unsigned long long*)out, (unsigned long long)w);
}

void gp_free(snnmap_hgraph* h)
{
    GpOut& G = h->gp;
    for (void* p : {(void*)G.hoff, (void*)G.hpins, (void*)G.eta, (void*)G.axons, (void*)G.hsd})
        if (p) cudaFreeAsync(p, h->stream);
    G = GpOut{};
}

Status emit_gp(snnmap_hgraph* h, int32_t K, const int32_t* rho)
{
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    gp_free(h);
    SNN_TRY(ensure_resident(h, 0));
    Level& L = h->levels[0];
    LevelExtra& X = h->extra[0];
    int32_t E = L.E;
    SNN_TRY(zero_scalars(h));
    int32_t *tpins, *tlen;
    uint8_t* tsd;
    uint32_t* thash;
    SNN_TRY(ar.alloc(&tpins, L.P));
    SNN_TRY(ar.alloc(&tlen, E));
    SNN_TRY(ar.alloc(&tsd, E));
    SNN_TRY(ar.alloc(&thash, E));
    ContractJob job{L.hoff, L.hpins, L.hsd, L.hk, rho, tpins, tlen, tsd, thash, nullptr, true};
    SNN_TRY(seg_run(job, X.seg, E, ar, s));

    uint64_t *keys, *keys2;
    uint32_t *vals, *vals2;
    int32_t *headpos, *runstart, *rep, *head, *gidh, *gid, *tk;
    int64_t *tw, *newlen, *newoff;
    SNN_TRY(ar.alloc(&keys, E));
    SNN_TRY(ar.alloc(&keys2, E));
    SNN_TRY(ar.alloc(&vals, E));
    SNN_TRY(ar.alloc(&vals2, E));
    SNN_TRY(ar.alloc(&headpos, E));
    SNN_TRY(ar.alloc(&runstart, E));
    SNN_TRY(ar.alloc(&rep, E));
    SNN_TRY(ar.alloc(&head, E));
    SNN_TRY(ar.alloc(&gidh, E));
    SNN_TRY(ar.alloc(&gid, E));
    SNN_TRY(ar.alloc(&tk, E));
    SNN_TRY(ar.alloc(&tw, E));
    SNN_TRY(ar.alloc(&newlen, E));
    SNN_TRY(ar.alloc(&newoff, E));
    int ge = grid_for(E, 256);
    if (E > 0) {
        SNN_L k_gp_internal<<<ge, 256, 0, s>>>(E, tlen, L.hw, h->d_scal + SC_D);
        SNN_L k_dedup_keys<<<ge, 256, 0, s>>>(E, tlen, L.hoff, tpins, thash, (uint64_t)K, keys, vals);
        SNN_CUDA(cudaGetLastError());
        SNN_TRY(radix_sort_pairs(keys, vals, keys2, vals2, E, 32 + bits_for((uint64_t)K), ar, s));
        SNN_L k_run_heads<<<ge, 256, 0, s>>>(E, keys, headpos);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(scan_inclusive_max_i32(headpos, runstart, E, ar, s));
    if (E > 0) {
        SNN_L k_dedup_rep<<<ge, 256, 0, s>>>(E, keys, vals, runstart, L.hoff, tpins, tlen, tsd, rep, head);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(scan_exclusive_i32(head, gidh, E, (int32_t*)(h->d_scal + SC_B), ar, s));
    if (E > 0) {
        SNN_CUDA(cudaMemsetAsync(tw, 0, (size_t)E * sizeof(int64_t), s));
        SNN_CUDA(cudaMemsetAsync(tk, 0, (size_t)E * sizeof(int32_t), s));
        SNN_CUDA(cudaMemsetAsync(newlen, 0, (size_t)E * sizeof(int64_t), s));
        SNN_L k_dedup_accum<<<ge, 256, 0, s>>>(E, vals, rep, gidh, tlen, L.hw, L.hk, tw, tk, newlen, gid);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(scan_exclusive_i64(newlen, newoff, E, h->d_scal + SC_C, ar, s));
    SNN_TRY(read_scalars(h));
    int32_t E2 = (int32_t)(h->h_scal[SC_B] & 0xffffffff);
    int64_t P2 = h->h_scal[SC_C];
    GpOut& G = h->gp;
    SNN_CUDA(dev_malloc(&G.hoff, ((size_t)E2 + 1) * 8, s));
    SNN_CUDA(dev_malloc(&G.hpins, (size_t)(P2 > 0 ? P2 : 1) * 4, s));
    SNN_CUDA(dev_malloc(&G.eta, (size_t)(E2 > 0 ? E2 : 1) * 8, s));
    SNN_CUDA(dev_malloc(&G.axons, (size_t)(E2 > 0 ? E2 : 1) * 4, s));
    SNN_CUDA(dev_malloc(&G.hsd, (size_t)(E2 > 0 ? E2 : 1), s));
    G.E = E2;
    G.P = P2;
    G.K = K;
    G.internal = h->h_scal[SC_D];
    Level N;
    N.hoff = G.hoff;
    N.hpins = G.hpins;
    N.hsd = G.hsd;
    N.hw = G.eta;
    N.hk = G.axons;
    if (E > 0) {
        SNN_HEDGE_LAUNCH(hedge_lanes(L.P, L.E), k_dedup_emit, E, s, E, vals, rep, gid, L.hoff, tpins,
                         tlen, tsd, tw, tk, newoff, N);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_L k_set_off_end<<<1, 1, 0, s>>>(G.hoff, E2, P2);
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaStreamSynchronize(s));
    ar.reset();
    return Status{};
}

// Intermediate levels (neither level 0 nor the coarsest) stay resident when
// their index is a multiple of keep_stride; the stride doubles while their
// bytes exceed the budget. Released levels keep their sizes and cid map.
void thin_levels(snnmap_hgraph* h)
{
    int32_t top = (int32_t)h->levels.size() - 1;
    auto held = [&]() {
        int64_t b = 0;
        for (int32_t i = 1; i < top; i++)
            if (h->levels[i].resident) b += (int64_t)h->levels[i].bytes;
        return b;
    };
    for (;;) {
        for (int32_t i = 1; i < top; i++)
            if (h->levels[i].resident && i % h->keep_stride != 0) level_release(h, h->levels[i]);
        if (held() <= h->level_budget || h->keep_stride >= (1 << 30)) break;
        h->keep_stride *= 2;
    }
}

// The level's arrays back in memory: rebuilt from the nearest resident level
// below through the composed cid maps.
Status ensure_resident(snnmap_hgraph* h, int32_t l)
{
    if (h->levels[l].resident) return Status{};
    int32_t j = l - 1;
    while (j > 0 && !h->levels[j].resident) j--;
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    const Level& S = h->levels[j];
    int32_t* c;
    int64_t* d_V2;
    SNN_TRY(ar.alloc(&c, S.V));
    SNN_TRY(ar.alloc(&d_V2, 1));
    if (S.V > 0)
        SNN_CUDA(cudaMemcpyAsync(c, S.cid, (size_t)S.V * 4, cudaMemcpyDeviceToDevice, s));
    for (int32_t m = j + 1; m < l; m++) {
        SNN_L k_compose<<<grid_for(S.V, 256), 256, 0, s>>>(S.V, c, h->levels[m].cid);
        SNN_CUDA(cudaGetLastError());
    }
    int64_t v2 = h->levels[l].V;
    SNN_CUDA(cudaMemcpyAsync(d_V2, &v2, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    return build_coarse(h, j, c, d_V2, l);
}

}  // namespace snn
