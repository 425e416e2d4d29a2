// Neighbour scores as a dense matrix for the coarsening levels with few
// vertices (Sec. 4.1, Coarsening; Eq. neigh_histogram).
//
// When a level has at most about sqrt(budget / 16) vertices and few of them
// against its pair count (see mat_fits), score(n, m)
// (summed omega over hyperedges holding both) and the shared inbound count
// ov(n, m) (summed k over hyperedges where both are destinations) are kept
// for every pair in V x V int32 matrices. The candidate of n is then a scan
// of row n with the validity test of the histogram path, instead of a
// histogram over n's neighbourhood.
//
// Contraction keeps the entries of two unmatched vertices exact: their
// common hyperedges map one to one onto common hyperedges of the coarse
// level with the same summed omega and k and the same destination roles (a
// hyperedge can only vanish if all its pins fall into one super-node). So
// the next level's matrix is a gather of the previous one at the
// representatives, plus fresh rows (a histogram, ScorePol) for the merged
// super-nodes, mirrored into their columns.
#include "histo.cuh"
#include "internal.cuh"

namespace snn {

template <typename S_>
struct ScorePol {
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
    const int32_t* fresh;   // rows to compute (null: every vertex)
    int32_t* Sm;
    int32_t* OVm;
    int64_t Vs;

    __device__ bool skip(int32_t n) const { return fresh && !fresh[n]; }
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
    template <class Tb>
    __device__ bool elem(int32_t n, const Seg<S>& g, int32_t off, const Tb& t, Acc&) const
    {
        int32_t m = L.hpins[g.b + off];
        if (m == n) return true;
        int md = off != 0 || g.sd;   // pin 0 is the source
        return t.add(m, g.w, (g.nd && md) ? g.k : 0u);
    }
    // every neighbour lands in the row (stores: a vertex redone by a later
    // tier overwrites its partial entries)
    __device__ void consider(int32_t n, int32_t m, int64_t s, uint32_t o, const Acc&, int64_t&,
                             int32_t&, uint32_t&) const
    {
        int64_t r = (int64_t)n * Vs + m;
        Sm[r] = (int32_t)s;
        OVm[r] = (int32_t)o;
    }
    __device__ void write(int32_t, int64_t, int32_t, uint32_t, const Acc&) const {}
};

__global__ void k_mat_min(Level L, int32_t* vmin)
{
    int32_t ms = 0x7fffffff, mi = 0x7fffffff;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < L.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        ms = min(ms, L.vsize[n]);
        mi = min(mi, L.vinpins[n]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ms = min(ms, __shfl_xor_sync(FULL, ms, o));
        mi = min(mi, __shfl_xor_sync(FULL, mi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&vmin[0], ms);
        atomicMin(&vmin[1], mi);
    }
}

// candidate of n: the valid neighbour with the largest score, ties to the
// lower id (the rules of the histogram path, including its skip of vertices
// that cannot merge even with the smallest vertex)
__global__ void __launch_bounds__(256)
    k_mat_best(Level L, const int32_t* __restrict__ vmin, const int32_t* __restrict__ Sm,
               const int32_t* __restrict__ OVm, int64_t Vs, int32_t omega, int32_t delta,
               int32_t phi, int32_t* cand, int64_t* cscore, int32_t* cov)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t n = gw; n < L.V; n += nw) {
        int64_t sz = L.vsize[n], ip = L.vinpins[n], ic = L.vincnt[n];
        int64_t r0 = n * Vs;
        int64_t bs = 0;
        int32_t bk = -1;
        if (sz + vmin[0] <= omega && ip + vmin[1] <= phi) {
            const int4* row = reinterpret_cast<const int4*>(Sm + r0);
            for (int64_t q = lane; 4 * q < L.V; q += 32) {
                int4 c4 = row[q];
                int cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    int32_t m = (int32_t)(4 * q + u);
                    int64_t sc = cv[u];
                    if (m < L.V && sc > bs && m != n && sz + L.vsize[m] <= omega &&
                        ip + L.vinpins[m] <= phi &&
                        ic + L.vincnt[m] - (int64_t)OVm[r0 + m] <= delta) {
                        bs = sc;
                        bk = m;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                int64_t s2 = __shfl_xor_sync(FULL, bs, o);
                int32_t m2 = __shfl_xor_sync(FULL, bk, o);
                if (better(s2, m2, bs, bk)) {
                    bs = s2;
                    bk = m2;
                }
            }
        }
        if (lane == 0) {
            cand[n] = bk;
            cscore[n] = bk < 0 ? 0 : bs;
            cov[n] = bk < 0 ? 0 : OVm[r0 + bk];
        }
    }
}

// coarse vertex cid(n)'s representative (its smaller member) and whether it
// merged two vertices
__global__ void k_mat_reps(int32_t V, const int32_t* __restrict__ cid,
                           const int32_t* __restrict__ match, int32_t* repof, int32_t* fresh)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = match[n];
        if (m >= 0 && m < (int32_t)n) continue;
        repof[cid[n]] = (int32_t)n;
        fresh[cid[n]] = m >= 0;
    }
}

// S2[i][j] = S[rep(i)][rep(j)] (one block per row)
__global__ void __launch_bounds__(256)
    k_mat_gather(int32_t V2, const int32_t* __restrict__ repof, const int32_t* __restrict__ Sm,
                 const int32_t* __restrict__ OVm, int64_t Vs, int32_t* S2, int32_t* OV2, int64_t Vs2)
{
    for (int64_t i = blockIdx.x; i < V2; i += gridDim.x) {
        int64_t src = (int64_t)repof[i] * Vs;
        int64_t dst = i * Vs2;
        for (int64_t j = threadIdx.x; j < V2; j += blockDim.x) {
            int64_t c = repof[j];
            S2[dst + j] = Sm[src + c];
            OV2[dst + j] = OVm[src + c];
        }
    }
}

// rows of fresh vertices cleared (one warp per vertex)
__global__ void k_mat_zero(int32_t V, const int32_t* __restrict__ fresh, int32_t* Sm, int32_t* OVm,
                           int64_t Vs)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t n = gw; n < V; n += nw) {
        if (!fresh[n]) continue;
        int4* s = reinterpret_cast<int4*>(Sm + n * Vs);
        int4* o = reinterpret_cast<int4*>(OVm + n * Vs);
        for (int64_t q = lane; q < Vs / 4; q += 32) {
            s[q] = make_int4(0, 0, 0, 0);
            o[q] = make_int4(0, 0, 0, 0);
        }
    }
}

// column u of every fresh vertex u mirrors its row (one warp per vertex)
__global__ void k_mat_mirror(int32_t V, const int32_t* __restrict__ fresh, int32_t* Sm, int32_t* OVm,
                             int64_t Vs)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = gw; u < V; u += nw) {
        if (!fresh[u]) continue;
        for (int64_t x = lane; x < V; x += 32) {
            Sm[x * Vs + u] = Sm[u * Vs + x];
            OVm[x * Vs + u] = OVm[u * Vs + x];
        }
    }
}

static Status mat_rows(snnmap_hgraph* h, const Level& L, const int32_t* fresh)
{
    ScoreMat& M = h->mat;
    ScorePol<uint32_t> pol;
    pol.L = L;
    pol.V = L.V;
    pol.keys = L.V;
    pol.fresh = fresh;
    pol.Sm = M.S;
    pol.OVm = M.OV;
    pol.Vs = M.Vs;
    int64_t* cnt;
    SNN_TRY(h->scratch.alloc(&cnt, HT_NCNT));
    return run_histogram(pol, h->scratch, h->stream, cnt, h->h_scal + 12, h->d_scal, h->tiers);
}

void mat_close(snnmap_hgraph* h)
{
    ScoreMat& M = h->mat;
    for (int32_t* p : {M.S, M.OV, M.S2, M.OV2})
        if (p) cudaFreeAsync(p, h->stream);
    M = ScoreMat{};
}

// The matrix is entered on a level when it fits the budget and pays: one
// level costs about 24 V^2 bytes of HBM traffic (gather 16, scan 8) against
// the histogram's pair_terms hash updates, which run roughly five times
// slower per item than bytes stream; so V^2 <= 5 * pair_terms. Once entered
// it stays (V shrinks while pair_terms barely does).
static bool mat_fits(const snnmap_hgraph* h, int32_t level)
{
    if (h->wide || h->wzero || h->wsum > INT32_MAX) return false;
    int64_t Vs = ((int64_t)h->levels[level].V + 3) & ~(int64_t)3;
    return 16 * Vs * Vs <= dense_row_budget(h) &&
           (double)Vs * (double)Vs <= 5.0 * (double)h->extra[level].pair_terms;
}

Status mat_affinity(snnmap_hgraph* h, int32_t level, bool* done)
{
    *done = false;
    ScoreMat& M = h->mat;
    const Level& L = h->levels[level];
    cudaStream_t s = h->stream;
    if (M.level != level) {
        mat_close(h);
        if (!mat_fits(h, level)) return Status{};
        int64_t Vs = ((int64_t)L.V + 3) & ~(int64_t)3;
        size_t bytes = (size_t)(Vs * Vs) * 4;
        cudaError_t e = dev_malloc(&M.S, bytes, s);
        if (e == cudaSuccess) e = dev_malloc(&M.OV, bytes, s);
        if (e == cudaSuccess) e = dev_malloc(&M.S2, bytes, s);
        if (e == cudaSuccess) e = dev_malloc(&M.OV2, bytes, s);
        if (e != cudaSuccess) {
            // no room: this level and the next ones use histograms
            cudaGetLastError();
            mat_close(h);
            return Status{};
        }
        M.cap = Vs * Vs;
        M.Vs = Vs;
        SNN_CUDA(cudaMemsetAsync(M.S, 0, bytes, s));
        SNN_CUDA(cudaMemsetAsync(M.OV, 0, bytes, s));
        SNN_TRY(mat_rows(h, L, nullptr));
        M.level = level;
    }
    int32_t* vmin;
    SNN_TRY(h->scratch.alloc(&vmin, 2));
    SNN_TRY(fill_i32(vmin, 0x7fffffff, 2, s));
    if (L.V > 0) {
        SNN_L k_mat_min<<<grid_for(L.V, 256), 256, 0, s>>>(L, vmin);
        SNN_L k_mat_best<<<grid_for((int64_t)L.V * 32, 256), 256, 0, s>>>(
            L, vmin, M.S, M.OV, M.Vs, h->prm.omega, h->prm.delta, h->prm.phi, h->cand, h->cscore,
            h->cov);
        SNN_CUDA(cudaGetLastError());
    }
    h->extra[level].n_block = 0;
    h->extra[level].n_global = 0;
    h->extra[level].carried = 2;
    h->extra[level].n_full = 0;
    h->extra[level].hist_work = 0;
    *done = true;
    return Status{};
}

Status mat_descend(snnmap_hgraph* h, int32_t src)
{
    ScoreMat& M = h->mat;
    if (M.level != src) return Status{};
    const Level& F = h->levels[src];
    const Level& L = h->levels[src + 1];
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    int64_t Vs2 = ((int64_t)L.V + 3) & ~(int64_t)3;
    if (Vs2 * Vs2 > M.cap) {
        mat_close(h);
        return Status{};
    }
    int32_t *repof, *fresh;
    SNN_TRY(ar.alloc(&repof, L.V));
    SNN_TRY(ar.alloc(&fresh, L.V));
    if (F.V > 0) {
        SNN_L k_mat_reps<<<grid_for(F.V, 256), 256, 0, s>>>(F.V, F.cid, h->match, repof, fresh);
        SNN_CUDA(cudaGetLastError());
    }
    if (L.V > 0) {
        SNN_L k_mat_gather<<<(int)std::min<int64_t>(L.V, 152 * 16), 256, 0, s>>>(
            L.V, repof, M.S, M.OV, M.Vs, M.S2, M.OV2, Vs2);
        SNN_CUDA(cudaGetLastError());
    }
    std::swap(M.S, M.S2);
    std::swap(M.OV, M.OV2);
    M.Vs = Vs2;
    if (L.V > 0) {
        SNN_L k_mat_zero<<<grid_for((int64_t)L.V * 32, 256), 256, 0, s>>>(L.V, fresh, M.S, M.OV, M.Vs);
        SNN_CUDA(cudaGetLastError());
        SNN_TRY(mat_rows(h, L, fresh));
        SNN_L k_mat_mirror<<<grid_for((int64_t)L.V * 32, 256), 256, 0, s>>>(L.V, fresh, M.S, M.OV, M.Vs);
        SNN_CUDA(cudaGetLastError());
    }
    M.level = src + 1;
    return Status{};
}

}  // namespace snn
