// Contraction (Sec. 4.1: each level's hypergraph is materialized from its
// predecessor while every super-node carries its constrained state).
//
// 1. Coarse ids: a vertex represents its pair if it is unmatched or the
//    lower id of the pair; cid = rank of the representative (exclusive scan).
// 2. Super-node state: size, inbound pins and internal axons add up; the
//    merged inbound set has in_count(n) + in_count(m) - shared(n, m).
// 3. Per hyperedge (segmented sort): s' = cid(source), destinations mapped
//    through cid, sorted, made unique; s' among them sets selfdst and is
//    removed. A hyperedge left with no destination is dropped and its
//    multiplicity k moves into the source super-node's internal count.
// 4. Duplicate hyperedges (same s', selfdst, destination list) merge: a
//    stable radix sort on (s', 32-bit content hash) brings candidates
//    together, an exact comparison of the contents decides, and the first
//    of each equal group becomes the coarse hyperedge; omega and k add up.
// 5. Compaction into the next level's arrays, then its incidence lists.
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
    int32_t *size, *inpins, *incnt, *inint;
};

__global__ void k_cid_state(Level L, const int32_t* __restrict__ match,
                            const int32_t* __restrict__ cand, const int32_t* __restrict__ cov,
                            const int32_t* __restrict__ repidx, NextState ns)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < L.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = match[n];
        if (!(m < 0 || (int32_t)n < m)) continue;
        int32_t c = repidx[n];
        L.cid[n] = c;
        if (m < 0) {
            ns.size[c] = L.vsize[n];
            ns.inpins[c] = L.vinpins[n];
            ns.incnt[c] = L.vincnt[n];
            ns.inint[c] = L.vinint[n];
        } else {
            L.cid[m] = c;
            int32_t ov = cand[n] == m ? cov[n] : cov[m];
            ns.size[c] = L.vsize[n] + L.vsize[m];
            ns.inpins[c] = L.vinpins[n] + L.vinpins[m];
            ns.incnt[c] = L.vincnt[n] + L.vincnt[m] - ov;
            ns.inint[c] = L.vinint[n] + L.vinint[m];
        }
    }
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
    int32_t* inint_next;
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
        int sd = hsd[a];
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
            if (__any_sync(FULL, self)) sd = 1;
        }
        hsum = warp_sum(hsum);
        if (lane == 0) {
            tpins[base] = (int32_t)sp;
            if (cnt == 0) {
                tlen[a] = 0;
                if (sd) atomicAdd(&inint_next[sp], hk[a]);
            } else {
                tlen[a] = 1 + cnt;
                tsd[a] = (uint8_t)sd;
                uint64_t hh = hsum + mix64(0x5bd1e995ull + (uint64_t)sd) + mix64((uint64_t)cnt << 1);
                thash[a] = (uint32_t)(hh ^ (hh >> 32));
            }
        }
    }
    __device__ void finish_thread(int32_t a, const uint32_t* s, int n) const
    {
        int64_t base = hoff[a];
        uint32_t sp = (uint32_t)cid[hpins[base]];
        int cnt = 0, sd = hsd[a];
        uint64_t hsum = 0;
        for (int i = 0; i < n; i++) {
            uint32_t v = s[i];
            if (i > 0 && s[i - 1] == v) continue;
            if (v == sp) {
                sd = 1;
                continue;
            }
            tpins[base + 1 + cnt++] = (int32_t)v;
            hsum += mix64(v);
        }
        tpins[base] = (int32_t)sp;
        if (cnt == 0) {
            tlen[a] = 0;
            if (sd) atomicAdd(&inint_next[sp], hk[a]);
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

__global__ void k_dedup_emit(int32_t E, const uint32_t* __restrict__ vals,
                             const int32_t* __restrict__ rep, const int32_t* __restrict__ gid,
                             const int64_t* __restrict__ hoff, const int32_t* __restrict__ tpins,
                             const int32_t* __restrict__ tlen, const uint8_t* __restrict__ tsd,
                             const int64_t* __restrict__ tw, const int32_t* __restrict__ tk,
                             const int64_t* __restrict__ newoff, Level N)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < E; i += nw) {
        if (rep[i] != (int32_t)i) continue;
        int32_t a = (int32_t)vals[i];
        int32_t g = gid[i];
        int64_t dst = newoff[g], src = hoff[a];
        int32_t len = tlen[a];
        for (int32_t j = lane; j < len; j += 32) N.hpins[dst + j] = tpins[src + j];
        if (lane == 0) {
            N.hoff[g] = dst;
            N.hsd[g] = tsd[a];
            N.hw[g] = tw[g];
            N.hk[g] = tk[g];
        }
    }
}

__global__ void k_set_off_end(int64_t* hoff, int32_t E, int64_t P) { hoff[E] = P; }

Status contract_level(snnmap_hgraph* h)
{
    if (!h->have_matching || h->last_pairs <= 0) return Status{SNNMAP_ERR_STATE, "no matching to contract"};
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    Level& L = h->levels.back();
    LevelExtra& X = h->extra.back();
    int32_t V = L.V, E = L.E;
    int g = grid_for(V, 256);
    SNN_TRY(zero_scalars(h));
    std::unique_ptr<ProfScope> prof(new ProfScope(h, PS_CONTRACT));

    // 1-2. coarse ids and super-node state
    int32_t *isrep, *repidx;
    NextState ns;
    SNN_TRY(ar.alloc(&isrep, V));
    SNN_TRY(ar.alloc(&repidx, V));
    SNN_TRY(ar.alloc(&ns.size, V));
    SNN_TRY(ar.alloc(&ns.inpins, V));
    SNN_TRY(ar.alloc(&ns.incnt, V));
    SNN_TRY(ar.alloc(&ns.inint, V));
    SNN_L k_rep_flags<<<g, 256, 0, s>>>(V, h->match, isrep);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(scan_exclusive_i32(isrep, repidx, V, (int32_t*)(h->d_scal + SC_A), ar, s));
    SNN_L k_cid_state<<<g, 256, 0, s>>>(L, h->match, h->cand, h->cov, repidx, ns);
    SNN_CUDA(cudaGetLastError());

    // 3. per-hyperedge remap, sort, unique
    int32_t *tpins, *tlen;
    uint8_t* tsd;
    uint32_t* thash;
    SNN_TRY(ar.alloc(&tpins, L.P));
    SNN_TRY(ar.alloc(&tlen, E));
    SNN_TRY(ar.alloc(&tsd, E));
    SNN_TRY(ar.alloc(&thash, E));
    ContractJob job{L.hoff, L.hpins, L.hsd, L.hk, L.cid, tpins, tlen, tsd, thash, ns.inint};
    SNN_TRY(seg_run(job, X.seg, E, ar, s));

    // 4. duplicate hyperedges
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
    int32_t V2 = (int32_t)(h->h_scal[SC_A] & 0xffffffff);
    int32_t E2 = (int32_t)(h->h_scal[SC_B] & 0xffffffff);
    int64_t P2 = h->h_scal[SC_C];

    // 5. next level
    h->levels.emplace_back();
    h->extra.emplace_back();
    Level& N = h->levels.back();
    LevelExtra& NX = h->extra.back();
    Level& Lp = h->levels[h->levels.size() - 2];
    SNN_TRY(level_alloc(h, N, NX, V2, E2, P2));
    N.maxlen = Lp.maxlen;
    prof.reset(new ProfScope(h, PS_CONTRACT));
    if (V2 > 0) {
        SNN_CUDA(cudaMemcpyAsync(N.vsize, ns.size, (size_t)V2 * 4, cudaMemcpyDeviceToDevice, s));
        SNN_CUDA(cudaMemcpyAsync(N.vinpins, ns.inpins, (size_t)V2 * 4, cudaMemcpyDeviceToDevice, s));
        SNN_CUDA(cudaMemcpyAsync(N.vincnt, ns.incnt, (size_t)V2 * 4, cudaMemcpyDeviceToDevice, s));
        SNN_CUDA(cudaMemcpyAsync(N.vinint, ns.inint, (size_t)V2 * 4, cudaMemcpyDeviceToDevice, s));
    }
    if (E > 0) {
        SNN_L k_dedup_emit<<<grid_for((int64_t)E * 32, 256), 256, 0, s>>>(
            E, vals, rep, gid, Lp.hoff, tpins, tlen, tsd, tw, tk, newoff, N);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_L k_set_off_end<<<1, 1, 0, s>>>(N.hoff, E2, P2);
    SNN_CUDA(cudaGetLastError());
    prof.reset();
    SNN_TRY(build_incidence(h, N));
    SNN_CUDA(cudaMemsetAsync(h->d_scal + SC_W2, 0, sizeof(int64_t), s));
    SNN_TRY(seg_classify(N.hoff, E2, N.maxlen, NX.seg, ar, s, h->d_scal + SC_W2));
    h->have_matching = false;
    SNN_TRY(read_scalars(h));
    NX.pair_terms = h->h_scal[SC_W2];
    ar.reset();
    return Status{};
}

}  // namespace snn
