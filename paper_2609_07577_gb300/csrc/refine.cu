// Uncoarsening and refinement (Sec. 4.1).
//
// Projection: rho_l(n) = rho_{l+1}(cid(n)).
//
// One refinement round:
//  S6  pins(p, e): per hyperedge, the sorted keys rho(q)*2 + [q is a
//      destination] are run-length encoded into (p, cnt, dcnt) entries;
//      e is inbound to p iff dcnt > 0. Partition state: size, inbound pins,
//      and distinct inbound axons (internal axons + k of inbound hyperedges).
//      Conn = sum omega(e) (lambda(e) - 1) comes out of the same pass.
//  S7  per vertex: save = omega of incident hyperedges where it is its
//      partition's last pin; for every other adjacent partition p the
//      connection weight conn(p) (loss = W - conn) and the k of hyperedges
//      where it is a destination and that are already inbound to p; gain =
//      save - loss; the best feasible move (ties to the lower p) is proposed
//      if its gain is positive.
//  S8  moves sorted by decreasing gain, ties by vertex id (stable radix sort
//      of compacted proposals, which are in vertex order).
//  S9  per hyperedge, its moved pins are replayed in move order: each
//      move's gain contribution omega([cnt(from)=1] - [cnt(to)=0]) is taken
//      with every earlier move applied, and when a destination leaves the
//      last / enters the first destination slot of a partition an inbound
//      event (p, move, -/+k) is emitted. Prefix sums give each prefix's gain.
//  S10 validity: per partition, its events (size/pins of every move, inbound
//      events) sorted by move and scanned; after each move that touches the
//      partition its limits are checked and changes of "violating" are added
//      to the move's violation delta. A prefix is valid iff the prefix sum of
//      violation deltas is zero.
//  S11 the valid prefix with the largest positive gain (shortest on ties) is
//      enacted.
#include "histo.cuh"
#include "internal.cuh"

#include <algorithm>
#include <climits>
#include <memory>

namespace snn {

enum : int {
    RS_M = SC_A,       // proposals
    RS_MAXG = SC_B,    // largest proposed gain
    RS_BEST = SC_C,    // best valid prefix gain
    RS_ISTAR = SC_D,   // index of its last move
    RS_COST = SC_E,    // Conn at round start
    RS_NEV = SC_F,     // inbound events emitted
    RS_NHV = SC_G,     // hyperedges replayed by the block tier
    RS_DEG = 8,        // incidences of proposing vertices
    RS_ACT = 10,       // vertices evaluated
    RS_MING = 11,      // smallest proposed gain (<= 0)
};

constexpr int REPLAY_WARP_MAX = 32;
constexpr int PSTAR_MAX = 16;   // partitions of P* the column update takes

struct PinCounts {
    int32_t* p;
    int32_t* cnt;
    int32_t* dcnt;
    int32_t* lam;
};

struct PState {
    int64_t* size;
    int64_t* inpins;
    int64_t* pincnt;
};

// ---------------------------------------------------------------------------
// S5

__global__ void k_project(int32_t V, const int32_t* __restrict__ cid,
                          const int32_t* __restrict__ rc, int32_t* rf)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        rf[n] = rc[cid[n]];
}

Status project(snnmap_hgraph* h, int32_t level, const int32_t* rho_coarse, int32_t* rho_fine)
{
    Level& L = h->levels[level];
    if (L.V > 0) {
        SNN_L k_project<<<grid_for(L.V, 256), 256, 0, h->stream>>>(L.V, L.cid, rho_coarse, rho_fine);
        SNN_CUDA(cudaGetLastError());
    }
    return Status{};
}

// ---------------------------------------------------------------------------
// S6

// Conn is summed into COST_SLOTS partial sums (hyperedge id modulo) rather
// than one word, so the per-hyperedge atomics do not all meet on one address
constexpr int COST_SLOTS = 256;

__global__ void k_cost_slots(const int64_t* __restrict__ slots, int64_t* out)
{
    int64_t v = 0;
    for (int i = threadIdx.x; i < COST_SLOTS; i += blockDim.x) v += slots[i];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd((unsigned long long*)out, (unsigned long long)v);
}

struct PinCountJob {
    const int64_t* hoff;
    const int32_t* hpins;
    const uint8_t* hsd;
    const int32_t* hk;
    const int64_t* hw;
    const int32_t* rho;
    PinCounts pc;
    int64_t* pincnt;
    int64_t* cost;     // COST_SLOTS partial sums of Conn
    __device__ int len(int32_t a) const { return (int)(hoff[a + 1] - hoff[a]); }
    __device__ uint32_t load(int32_t a, int i) const
    {
        int64_t j = hoff[a] + i;
        uint32_t d = (i > 0 || hsd[a]) ? 1u : 0u;
        return ((uint32_t)rho[hpins[j]] << 1) | d;
    }
    __device__ void finish(int32_t a, const uint32_t* s, int n) const
    {
        int lane = threadIdx.x & 31;
        int64_t base = hoff[a];
        unsigned le = lanemask_lt() | (1u << lane);
        int R = 0;
        // pass 1: run starts (partition changes) and first destination of each run
        for (int c = 0; c < n; c += 32) {
            int i = c + lane;
            bool valid = i < n;
            uint32_t v = valid ? s[i] : KEY_PAD;
            uint32_t pv = (valid && i > 0) ? s[i - 1] : KEY_PAD;
            bool rs = valid && (i == 0 || (v >> 1) != (pv >> 1));
            bool ds = valid && (v & 1) && (i == 0 || v != pv);
            unsigned mr = __ballot_sync(FULL, rs);
            int r = R + __popc(mr & le) - 1;
            if (rs) {
                pc.p[base + r] = (int32_t)(v >> 1);
                pc.cnt[base + r] = i;
                pc.dcnt[base + r] = -1;
            }
            __syncwarp();
            if (ds) pc.dcnt[base + r] = i;
            __syncwarp();
            R += __popc(mr);
        }
        // pass 2: starts -> counts
        for (int c = 0; c < R; c += 32) {
            int r = c + lane;
            int st = 0, nx = 0, dsx = -1;
            if (r < R) {
                st = pc.cnt[base + r];
                nx = (r + 1 < R) ? pc.cnt[base + r + 1] : n;
                dsx = pc.dcnt[base + r];
            }
            __syncwarp();
            if (r < R) {
                int dc = dsx >= 0 ? nx - dsx : 0;
                pc.cnt[base + r] = nx - st;
                pc.dcnt[base + r] = dc;
                if (dc > 0) atomicAdd((unsigned long long*)&pincnt[pc.p[base + r]], (unsigned long long)hk[a]);
            }
            __syncwarp();
        }
        if (lane == 0) {
            pc.lam[a] = R;
            if (R > 1) atomicAdd((unsigned long long*)&cost[a & (COST_SLOTS - 1)], (unsigned long long)(hw[a] * (R - 1)));
        }
    }
    __device__ void finish_thread(int32_t a, const uint32_t* s, int n, int st) const
    {
        int64_t base = hoff[a];
        int R = 0, c = 0, d = 0;
        for (int i = 0; i < n; i++) {
            uint32_t p = s[(i) * st] >> 1;
            if (i > 0 && p != (s[(i - 1) * st] >> 1)) {
                pc.p[base + R] = (int32_t)(s[(i - 1) * st] >> 1);
                pc.cnt[base + R] = c;
                pc.dcnt[base + R] = d;
                if (d > 0) atomicAdd((unsigned long long*)&pincnt[s[(i - 1) * st] >> 1], (unsigned long long)hk[a]);
                R++;
                c = 0;
                d = 0;
            }
            c++;
            d += (int)(s[(i) * st] & 1);
        }
        if (n > 0) {
            pc.p[base + R] = (int32_t)(s[(n - 1) * st] >> 1);
            pc.cnt[base + R] = c;
            pc.dcnt[base + R] = d;
            if (d > 0) atomicAdd((unsigned long long*)&pincnt[s[(n - 1) * st] >> 1], (unsigned long long)hk[a]);
            R++;
        }
        pc.lam[a] = R;
        if (R > 1) atomicAdd((unsigned long long*)&cost[a & (COST_SLOTS - 1)], (unsigned long long)(hw[a] * (R - 1)));
    }
};

__global__ void k_pstate_vertices(Level L, const int32_t* __restrict__ rho, PState ps)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < L.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = rho[n];
        atomicAdd((unsigned long long*)&ps.size[p], (unsigned long long)L.vsize[n]);
        atomicAdd((unsigned long long*)&ps.inpins[p], (unsigned long long)L.vinpins[n]);
        if (L.vinint[n]) atomicAdd((unsigned long long*)&ps.pincnt[p], (unsigned long long)L.vinint[n]);
    }
}

__device__ __forceinline__ bool violates(int64_t sz, int64_t ip, int64_t pc, int32_t omega,
                                         int32_t delta, int32_t phi)
{
    return sz > omega || ip > phi || pc > delta;
}

__global__ void k_check_pstate(int32_t K, PState ps, int32_t omega, int32_t delta, int32_t phi,
                               int64_t* scal)
{
    int bad = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < K;
         p += (int64_t)gridDim.x * blockDim.x)
        if (violates(ps.size[p], ps.inpins[p], ps.pincnt[p], omega, delta, phi)) bad = 1;
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicOr((int*)&scal[SC_STATUS], ST_BADSTATE);
}

// counts of partition p in hyperedge a at round start (entries sorted by p)
__device__ __forceinline__ void lookup_count(const PinCounts& pc, int64_t b, int32_t lam, int32_t p,
                                             int32_t& cnt, int32_t& dcnt)
{
    int32_t lo = 0, hi = lam;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (pc.p[b + mid] < p) lo = mid + 1;
        else hi = mid;
    }
    if (lo < lam && pc.p[b + lo] == p) {
        cnt = pc.cnt[b + lo];
        dcnt = pc.dcnt[b + lo];
    } else {
        cnt = 0;
        dcnt = 0;
    }
}

// save(n) = omega of incident hyperedges in which n is the last pin of its
// partition, W(n) = omega of all incident hyperedges. A move of n gains
// save(n) - W(n) + conn(n, p) <= save(n), so a vertex with save(n) = 0
// never proposes. A group of G lanes per hyperedge, lanes over its pins
// (both arrays cleared before).
template <int G>
__global__ void __launch_bounds__(256)
    k_save(Level L, PinCounts pc, const int32_t* __restrict__ rho, int64_t* savev, int64_t* Wv)
{
    int lane = threadIdx.x & (G - 1);
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) / G;
    for (int64_t a = gw; a < L.E; a += nw) {
        int64_t b = L.hoff[a], e = L.hoff[a + 1];
        int32_t lam = pc.lam[a];
        unsigned long long w = (unsigned long long)L.hw[a];
        for (int64_t j = b + lane; j < e; j += G) {
            int32_t x = L.hpins[j];
            atomicAdd((unsigned long long*)&Wv[x], w);
            int32_t c, d;
            lookup_count(pc, b, lam, rho[x], c, d);
            if (c == 1) atomicAdd((unsigned long long*)&savev[x], w);
        }
    }
}

// ---------------------------------------------------------------------------
// S7: partition connection histogram per vertex

template <typename S_>
struct GainPol {
    using S = S_;
    // a vertex meets few partitions even when its bound is large
    static constexpr bool kOptimistic = true;
    struct Acc {
        int64_t W, save;   // summed omega of incident hyperedges; of those n is the last pin of
        __device__ Acc() : W(0), save(0) {}
        __device__ void add(const Acc& o)
        {
            W += o.W;
            save += o.save;
        }
        __device__ void atomic_into(Acc* g) const
        {
            if (W) atomicAdd((unsigned long long*)&g->W, (unsigned long long)W);
            if (save) atomicAdd((unsigned long long*)&g->save, (unsigned long long)save);
        }
    };
    static __device__ Acc warp_reduce(const Acc& a)
    {
        Acc r;
        r.W = warp_sum(a.W);
        r.save = warp_sum(a.save);
        return r;
    }

    Level L;
    PinCounts pc;
    PState ps;
    const int32_t* rho;
    int32_t V;
    int64_t keys;
    int32_t omega, delta, phi;
    int32_t* pto;
    int64_t* pgain;
    const int64_t* savev;
    const int32_t* dirty;   // vertices to evaluate; the others keep pto/pgain
    bool nonpos;            // propose the best feasible move whatever its gain

    __device__ bool skip(int32_t n) const { return (!nonpos && savev[n] == 0) || !dirty[n]; }
    __device__ int64_t vb(int32_t n) const { return L.voff[n]; }
    __device__ int64_t ve(int32_t n) const { return L.voff[n + 1]; }
    __device__ int64_t seg_len(int64_t i) const
    {
        return pc.lam[(int32_t)((uint32_t)L.vinc[i] & ~SRC_BIT)];
    }
    __device__ Seg<S> seg(int64_t i, Acc& acc) const
    {
        uint32_t inc = (uint32_t)L.vinc[i];
        int32_t a = (int32_t)(inc & ~SRC_BIT);
        Seg<S> g;
        g.sd = L.hsd[a];
        g.nd = !(inc & SRC_BIT) || g.sd;
        g.b = L.hoff[a];
        g.len = pc.lam[a];
        g.w = (S)L.hw[a];
        g.k = (uint32_t)L.hk[a];
        acc.W += L.hw[a];
        return g;
    }
    template <class Tb>
    __device__ bool elem(int32_t n, const Seg<S>& g, int32_t off, const Tb& t, Acc& acc) const
    {
        int64_t e = g.b + off;
        int32_t p = pc.p[e];
        if (p == rho[n]) {
            if (pc.cnt[e] == 1) acc.save += (int64_t)g.w;
            return true;
        }
        // a partition that cannot take n by size or inbound pins is never
        // the chosen move: leave it out of the table
        if (ps.size[p] + L.vsize[n] > omega || ps.inpins[p] + L.vinpins[n] > phi) return true;
        return t.add(p, g.w, (g.nd && pc.dcnt[e] > 0) ? g.k : 0u);
    }
    // gain = save - loss with loss = W - conn(p); feasible if p stays within
    // Omega, Phi, and Delta on its inbound set grown by n's axons not yet
    // inbound to p
    __device__ void consider(int32_t n, int32_t p, int64_t conn, uint32_t o, const Acc& tot,
                             int64_t& bs, int32_t& bk, uint32_t& bo) const
    {
        int64_t gain = tot.save - tot.W + conn;
        bool feas = ps.size[p] + L.vsize[n] <= omega && ps.inpins[p] + L.vinpins[n] <= phi &&
                    ps.pincnt[p] + L.vincnt[n] - (int64_t)o <= delta;
        if (feas && better(gain, p, bs, bk)) {
            bs = gain;
            bk = p;
            bo = o;
        }
    }
    __device__ void write(int32_t n, int64_t bs, int32_t bk, uint32_t, const Acc&) const
    {
        if (!dirty[n]) return;
        bool prop = bk >= 0 && (bs > 0 || nonpos);
        pto[n] = prop ? bk : -1;
        pgain[n] = prop ? bs : 0;
    }
};

struct Moves {
    int32_t* n;
    int32_t* from;
    int32_t* to;
};

// Hyperedges holding a proposed move (k_prop_hedges builds the list): a
// round's replay, row updates, re-evaluation flags and pin-count updates
// iterate it instead of every hyperedge of the level.
struct HedgeList {
    const int32_t* a;   // hyperedge ids
    const int32_t* n;   // their number (device)
};

// ---------------------------------------------------------------------------
// Connection rows (refinement levels whose rows fit the memory budget)
//
// Row r of vertex n (r = rowid[n]) holds, for every partition p,
// C[r][p] = conn(n, p) = sum of omega(e) over incident e with cnt(p, e) > 0,
// and O[r][p] = sum of k(e) over e in which n is a destination and
// dcnt(p, e) > 0. A round then needs no histogram: the best move of n is a
// scan of its row against the partition state. Rows change only when a
// partition's count in a hyperedge crosses zero, which applied moves report
// (k_dense_cross). Projection to the next finer level leaves the rows of
// unmatched vertices exact (their hyperedges map one to one onto hyperedges
// of the same omega, k, destination role and partition set); the two
// members of each contracted pair get fresh rows (RowPol).

template <typename S_>
struct RowPol {
    using S = S_;
    // a row holds every adjacent partition: warp tables would overflow
    static constexpr bool kOptimistic = false;
    struct Acc {
        __device__ Acc() {}
        __device__ void add(const Acc&) {}
        __device__ void atomic_into(Acc*) const {}
    };
    static __device__ Acc warp_reduce(const Acc& a) { return a; }

    Level L;
    PinCounts pc;
    int32_t V;
    int64_t keys;
    const int32_t* fresh;
    const int32_t* rowid;
    int32_t* C;
    int32_t* O;
    int64_t Kp;
    unsigned long long* M;
    int32_t cw;

    __device__ bool skip(int32_t n) const { return fresh[n] == 0; }
    __device__ int64_t vb(int32_t n) const { return L.voff[n]; }
    __device__ int64_t ve(int32_t n) const { return L.voff[n + 1]; }
    __device__ int64_t seg_len(int64_t i) const
    {
        return pc.lam[(int32_t)((uint32_t)L.vinc[i] & ~SRC_BIT)];
    }
    __device__ Seg<S> seg(int64_t i, Acc&) const
    {
        uint32_t inc = (uint32_t)L.vinc[i];
        int32_t a = (int32_t)(inc & ~SRC_BIT);
        Seg<S> g;
        g.sd = L.hsd[a];
        g.nd = !(inc & SRC_BIT) || g.sd;
        g.b = L.hoff[a];
        g.len = pc.lam[a];
        g.w = (S)L.hw[a];
        g.k = (uint32_t)L.hk[a];
        return g;
    }
    template <class Tb>
    __device__ bool elem(int32_t, const Seg<S>& g, int32_t off, const Tb& t, Acc&) const
    {
        int64_t e = g.b + off;
        return t.add(pc.p[e], g.w, (g.nd && pc.dcnt[e] > 0) ? g.k : 0u);
    }
    // every key of the finished histogram lands in the row (stores, so a
    // vertex redone by a later tier overwrites its partial entries)
    __device__ void consider(int32_t n, int32_t p, int64_t conn, uint32_t o, const Acc&, int64_t&,
                             int32_t&, uint32_t&) const
    {
        int32_t row = rowid[n];
        int64_t r = (int64_t)row * Kp + p;
        C[r] = (int32_t)conn;
        O[r] = (int32_t)o;
        unsigned long long bit = 1ull << (p / cw);
        if (!(M[row] & bit)) atomicOr(&M[row], bit);   // a set bit is never cleared here
    }
    __device__ void write(int32_t, int64_t, int32_t, uint32_t, const Acc&) const {}
};

// best move per vertex from its row: largest gain = C - (W - save) over
// partitions p != rho(n) that can take n, ties to the lower p; proposed if
// positive. Only the chunks of the row that the mask M marks are read (an
// entry outside them is 0, and a partition with conn 0 is never taken);
// each lane still visits its partitions in increasing order.
__global__ void __launch_bounds__(256)
    k_dense_best(Level L, const int32_t* __restrict__ rho, PState ps,
                 const int64_t* __restrict__ savev, const int64_t* __restrict__ Wv,
                 const int32_t* __restrict__ rowid, const int32_t* __restrict__ C,
                 const int32_t* __restrict__ O, const unsigned long long* __restrict__ M,
                 int32_t cw, int64_t Kp, int32_t K, int32_t omega, int32_t delta, int32_t phi,
                 int nonpos, int32_t* pto, int64_t* pgain, const int32_t* __restrict__ dirty)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t n = gw; n < L.V; n += nw) {
        if (dirty && !dirty[n]) continue;   // proposal kept from the previous round
        int64_t sv = savev[n];
        if (sv == 0 && !nonpos) {
            if (lane == 0) {
                pto[n] = -1;
                pgain[n] = 0;
            }
            continue;
        }
        int64_t T = Wv[n] - sv;
        int32_t own = rho[n];
        int64_t sz = L.vsize[n], ip = L.vinpins[n], ic = L.vincnt[n];
        int32_t rw = rowid[n];
        int64_t r0 = (int64_t)rw * Kp;
        const int4* row = reinterpret_cast<const int4*>(C + r0);
        int64_t bs = 0;
        int32_t bk = -1;
        const int64_t nq = ((int64_t)K + 3) >> 2;
        unsigned long long msk = M[rw];   // the same word in every lane
        while (msk) {
            int c = __ffsll((long long)msk) - 1;
            msk &= msk - 1;
            int64_t q0 = (int64_t)c * (cw >> 2);
            int64_t q1 = q0 + (cw >> 2) < nq ? q0 + (cw >> 2) : nq;
            for (int64_t q = q0 + lane; q < q1; q += 32) {
                int4 c4 = row[q];
                int cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    int32_t p = (int32_t)(4 * q + u);
                    int64_t g = (int64_t)cv[u] - T;
                    // default: positive gains only (bs starts at 0); variant:
                    // any adjacent partition (conn > 0), the first one found
                    // seeds bs
                    if (p < K && (g > bs || (nonpos && bk < 0 && cv[u] > 0)) && cv[u] > 0 &&
                        p != own && ps.size[p] + sz <= omega && ps.inpins[p] + ip <= phi &&
                        ps.pincnt[p] + ic - (int64_t)O[r0 + p] <= delta) {
                        bs = g;
                        bk = p;
                    }
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
        if (lane == 0) {
            pto[n] = bk;
            pgain[n] = bk >= 0 ? bs : 0;
        }
    }
}

// Row updates for the enacted prefix: per hyperedge, the moves of its pins
// with index <= i* give each touched partition's count after the prefix;
// where cnt(p, e) crosses zero every pin's C[.][p] changes by omega(e), and
// where dcnt(p, e) crosses zero every destination's O[.][p] by k(e). One
// warp per hyperedge; buf (one word per pin) collects the enacted moves.
__global__ void __launch_bounds__(256)
    k_dense_cross(Level L, PinCounts pc, const int32_t* __restrict__ moveidx, Moves mv,
                  const int64_t* __restrict__ scal, const int32_t* __restrict__ rowid, int32_t* C,
                  int32_t* O, unsigned long long* M, int32_t cw, int64_t Kp, uint32_t* buf,
                  HedgeList hl)
{
    int64_t istar = scal[RS_BEST] > 0 ? scal[RS_ISTAR] : -1;
    if (istar < 0) return;
    int lane = threadIdx.x & 31;
    unsigned lt = lanemask_lt();
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t nh = *hl.n;
    for (int64_t x = gw; x < nh; x += nw) {
        int32_t a = hl.a[x];
        int64_t b = L.hoff[a], e = L.hoff[a + 1];
        int sd = L.hsd[a];
        int m = 0;
        for (int64_t cb = b; cb < e; cb += 32) {
            int64_t j = cb + lane;
            int32_t mi = -1;
            if (j < e) mi = moveidx[L.hpins[j]];
            bool ap = mi >= 0 && mi <= istar;
            unsigned mk = __ballot_sync(FULL, ap);
            if (ap) buf[b + m + __popc(mk & lt)] = ((uint32_t)mi << 1) | ((j != b || sd) ? 1u : 0u);
            m += __popc(mk);
        }
        if (m == 0) continue;
        __syncwarp();
        int32_t lam = pc.lam[a];
        int64_t w = L.hw[a];
        int32_t k = L.hk[a];
        for (int ib = 0; ib < m; ib += 32) {
            int ii = ib + lane;
            // up to two crossing records per lane: partition, C sign, O sign
            int32_t rp[2] = {-1, -1};
            int rc[2] = {0, 0}, rd[2] = {0, 0};
            if (ii < m) {
                int32_t mi = (int32_t)(buf[b + ii] >> 1);
                int32_t cand[2] = {mv.from[mi], mv.to[mi]};
                for (int u = 0; u < 2; u++) {
                    int32_t p = cand[u];
                    bool first = true;
                    int nc = 0, nd = 0;
                    for (int jj = 0; jj < m; jj++) {
                        uint32_t rj = buf[b + jj];
                        int32_t mj = (int32_t)(rj >> 1);
                        int32_t fj = mv.from[mj], tj = mv.to[mj];
                        if (jj < ii && (fj == p || tj == p)) first = false;
                        int dlt = (tj == p) - (fj == p);
                        nc += dlt;
                        if (rj & 1) nd += dlt;
                    }
                    if (!first) continue;
                    int32_t c0, d0;
                    lookup_count(pc, b, lam, p, c0, d0);
                    int cs = ((c0 + nc) > 0) - (c0 > 0);
                    int ds = ((d0 + nd) > 0) - (d0 > 0);
                    if (cs || ds) {
                        rp[u] = p;
                        rc[u] = cs;
                        rd[u] = ds;
                    }
                }
            }
            for (int u = 0; u < 2; u++) {
                unsigned has = __ballot_sync(FULL, rp[u] >= 0);
                while (has) {
                    int src = __ffs(has) - 1;
                    has &= has - 1;
                    int32_t p = __shfl_sync(FULL, rp[u], src);
                    int cs = __shfl_sync(FULL, rc[u], src);
                    int ds = __shfl_sync(FULL, rd[u], src);
                    for (int64_t j = b + lane; j < e; j += 32) {
                        int32_t rw = rowid[L.hpins[j]];
                        int64_t r = (int64_t)rw * Kp + p;
                        if (cs) atomicAdd(&C[r], (int32_t)(cs * w));
                        unsigned long long bit = 1ull << (p / cw);
                        if (cs > 0 && !(M[rw] & bit)) atomicOr(&M[rw], bit);
                        if (ds && (j != b || sd)) atomicAdd(&O[r], ds * k);
                    }
                }
            }
        }
    }
}

// descent to the next finer level: member counts and smallest member per
// coarse vertex
__global__ void k_dense_members(int32_t V, const int32_t* __restrict__ cid, int32_t* mcount,
                                int32_t* first)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(&mcount[cid[n]], 1);
        atomicMin(&first[cid[n]], (int32_t)n);
    }
}

__global__ void k_dense_flags(int32_t V, const int32_t* __restrict__ cid,
                              const int32_t* __restrict__ mcount, const int32_t* __restrict__ first,
                              int32_t* nonrep, int32_t* fresh)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = cid[n];
        nonrep[n] = first[c] != (int32_t)n;
        fresh[n] = mcount[c] > 1;
    }
}

// the smaller member keeps its super-node's row, the other takes row
// Vc + (its rank among non-representatives)
__global__ void k_dense_rowid(int32_t V, int32_t Vc, const int32_t* __restrict__ cid,
                              const int32_t* __restrict__ nonrep, const int32_t* __restrict__ idx,
                              const int32_t* __restrict__ rowc, int32_t* rowf)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        rowf[n] = nonrep[n] ? Vc + idx[n] : rowc[cid[n]];
}

// clears the rows of vertices flagged fresh (one warp per vertex)
__global__ void k_dense_zero(int32_t V, const int32_t* __restrict__ fresh,
                             const int32_t* __restrict__ rowid, int32_t* C, int32_t* O,
                             unsigned long long* M, int64_t Kp)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t n = gw; n < V; n += nw) {
        if (!fresh[n]) continue;
        if (lane == 0) M[rowid[n]] = 0;
        int4* c = reinterpret_cast<int4*>(C + (int64_t)rowid[n] * Kp);
        int4* o = reinterpret_cast<int4*>(O + (int64_t)rowid[n] * Kp);
        for (int64_t q = lane; q < Kp / 4; q += 32) {
            c[q] = make_int4(0, 0, 0, 0);
            o[q] = make_int4(0, 0, 0, 0);
        }
    }
}

// ---------------------------------------------------------------------------
// Incremental rounds on histogram levels. After an enacted prefix, a
// vertex's best move can change only if (a) one of its hyperedges holds a
// moved pin (its conn, overlap and save change only there), (b) it is
// adjacent to a partition that lost load (a source of an enacted move) and
// was tight before -- a partition with room for the largest vertex of the
// level in all three limits was feasible for every vertex before and still
// is, and partitions that only gained load lose feasibility, which matters
// only for (c) -- or (c) its proposed target changed state. Every other
// vertex keeps its proposal, which a full evaluation would reproduce.

__global__ void k_level_max(Level L, int32_t* vmax)
{
    int32_t a = 0, b = 0, c = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < L.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        a = max(a, L.vsize[n]);
        b = max(b, L.vinpins[n]);
        c = max(c, L.vincnt[n]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = max(a, __shfl_xor_sync(FULL, a, o));
        b = max(b, __shfl_xor_sync(FULL, b, o));
        c = max(c, __shfl_xor_sync(FULL, c, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&vmax[0], a);
        atomicMax(&vmax[1], b);
        atomicMax(&vmax[2], c);
    }
}

// partitions touched by the enacted prefix (pchg) and the tight sources
// among them (prel), with the round-start state
__global__ void k_inc_parts(int32_t M, Moves mv, const int64_t* __restrict__ scal, PState ps,
                            const int32_t* __restrict__ vmax, int32_t omega, int32_t delta,
                            int32_t phi, uint8_t* pchg, uint8_t* prel,
                            const int32_t* __restrict__ pstar_n)
{
    if (*pstar_n <= PSTAR_MAX) return;   // the column update below handles this round
    int64_t istar = scal[RS_BEST] > 0 ? scal[RS_ISTAR] : -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= istar && i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t f = mv.from[i], t = mv.to[i];
        pchg[f] = 1;
        pchg[t] = 1;
        if (ps.size[f] + vmax[0] > omega || ps.inpins[f] + vmax[1] > phi ||
            ps.pincnt[f] + vmax[2] > delta)
            prel[f] = 1;
    }
}

// (a) and (b). A hyperedge holding enacted moved pins changes the other
// pins' conn, overlap or save only where a partition's count or
// destination count crosses zero or its count moves between 1 and 2; then
// all its pins are marked, otherwise only the moved pins. A hyperedge
// holding a partition of prel (round-start pin counts) marks all its pins.
// One warp per hyperedge; buf (one word per pin) collects the moves.
__global__ void __launch_bounds__(256)
    k_inc_hedges(Level L, PinCounts pc, const int32_t* __restrict__ moveidx, Moves mv,
                 const int64_t* __restrict__ scal, const uint8_t* __restrict__ prel, uint32_t* buf,
                 int32_t* dirty, const int32_t* __restrict__ pstar_n)
{
    if (*pstar_n <= PSTAR_MAX) return;
    int64_t istar = scal[RS_BEST] > 0 ? scal[RS_ISTAR] : -1;
    if (istar < 0) return;
    int lane = threadIdx.x & 31;
    unsigned lt = lanemask_lt();
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = gw; a < L.E; a += nw) {
        int64_t b = L.hoff[a], e = L.hoff[a + 1];
        int sd = L.hsd[a];
        int m = 0;
        for (int64_t cb = b; cb < e; cb += 32) {
            int64_t j = cb + lane;
            int32_t mi = -1;
            if (j < e) mi = moveidx[L.hpins[j]];
            bool ap = mi >= 0 && mi <= istar;
            unsigned mk = __ballot_sync(FULL, ap);
            if (ap) buf[b + m + __popc(mk & lt)] = ((uint32_t)mi << 1) | ((j != b || sd) ? 1u : 0u);
            m += __popc(mk);
        }
        __syncwarp();
        int32_t lam = pc.lam[a];
        bool all = false;
        for (int32_t r = lane; r < lam && !all; r += 32)
            if (prel[pc.p[b + r]]) all = true;
        all = __any_sync(FULL, all);   // uniform before the warp-wide loop below
        for (int ib = 0; ib < m && !all; ib += 32) {
            int ii = ib + lane;
            if (ii < m) {
                int32_t mi = (int32_t)(buf[b + ii] >> 1);
                int32_t cand[2] = {mv.from[mi], mv.to[mi]};
                for (int u = 0; u < 2 && !all; u++) {
                    int32_t p = cand[u];
                    int nc = 0, nd = 0;
                    for (int jj = 0; jj < m; jj++) {
                        uint32_t rj = buf[b + jj];
                        int32_t mj = (int32_t)(rj >> 1);
                        int dlt = (mv.to[mj] == p) - (mv.from[mj] == p);
                        nc += dlt;
                        if (rj & 1) nd += dlt;
                    }
                    int32_t c0, d0;
                    lookup_count(pc, b, lam, p, c0, d0);
                    int c1 = c0 + nc, d1 = d0 + nd;
                    if ((c0 > 0) != (c1 > 0) || (d0 > 0) != (d1 > 0) || (c0 == 1) != (c1 == 1))
                        all = true;
                }
            }
            all = __any_sync(FULL, all);
        }
        all = __any_sync(FULL, all);
        if (all) {
            for (int64_t j = b + lane; j < e; j += 32) dirty[L.hpins[j]] = 1;
        } else {
            for (int ii = lane; ii < m; ii += 32) dirty[mv.n[buf[b + ii] >> 1]] = 1;
        }
    }
}

// (c)
__global__ void k_inc_targets(int32_t V, const int32_t* __restrict__ pto,
                              const uint8_t* __restrict__ pchg, int32_t* dirty,
                              const int32_t* __restrict__ pstar_n)
{
    if (*pstar_n <= PSTAR_MAX) return;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        if (pto[n] >= 0 && pchg[pto[n]]) dirty[n] = 1;
}


// ---------------------------------------------------------------------------
// Proposals after a short enacted prefix (at most PSTAR_MAX partitions
// touched). Moves change the state of their source and target partitions
// only (the set P*), and in every hyperedge only the counts of those
// partitions. For a vertex n that did not move, an option q outside P*
// therefore keeps conn(n, q), ov(n, q) and its feasibility, and its gain
// shifts by the change of save(n) alone; the previous best option outside
// P* stays the best outside P*. The options inside P* are recomputed from
// their columns conn(n, p), ov(n, p), summed over the hyperedges that hold
// a pin of p (found through p's members' incidence lists). n is evaluated
// in full (flagged for the next round's histogram) only if it moved, if its
// previous proposal targeted P*, or, when only positive gains are proposed,
// if it had no proposal and its save grew (its best option outside P* is
// then unknown). The other vertices get their exact proposal here.

struct PStar {
    int32_t* pslot = nullptr;   // [K] slot of a partition of P*; -1 none
    int32_t* slots = nullptr;   // [PSTAR_MAX] partition of each slot
    int32_t* cnt = nullptr;     // [0] distinct partitions of P*, [1] marked hyperedges,
                                // [2] value cnt[0] restarts from (> PSTAR_MAX: path off)
    uint32_t* hmask = nullptr;  // [E] slots whose partition has a pin in the hyperedge
    int32_t* hl = nullptr;      // [E] hyperedges with a nonzero mask
    int64_t* colc = nullptr;    // [PSTAR_MAX * V] conn(n, slot)
    int32_t* colo = nullptr;    // [PSTAR_MAX * V] ov(n, slot)
    uint32_t* vt = nullptr;     // [V] slots adjacent to n (some incident hyperedge has a pin there)
    int64_t* save0 = nullptr;   // [V] save at round start
};

__device__ __forceinline__ bool pstar_on(const int64_t* scal, const int32_t* cnt)
{
    return scal[RS_BEST] > 0 && cnt[0] <= PSTAR_MAX;
}

// P* from the enacted moves; the moved vertices are flagged for a full
// evaluation
__global__ void k_ps_slots(int32_t M, Moves mv, const int64_t* __restrict__ scal, PStar ps,
                           int32_t* dirty)
{
    int64_t istar = scal[RS_BEST] > 0 ? scal[RS_ISTAR] : -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= istar && i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        dirty[mv.n[i]] = 1;
        int32_t pp[2] = {mv.from[i], mv.to[i]};
        for (int u = 0; u < 2; u++) {
            int32_t p = pp[u];
            if (atomicCAS(&ps.pslot[p], -1, -2) != -1) continue;
            int32_t sl = atomicAdd(&ps.cnt[0], 1);
            if (sl < PSTAR_MAX) {
                ps.slots[sl] = p;
                ps.pslot[p] = sl;
            }
        }
    }
}

// every hyperedge incident to a member of a P* partition gets that slot's
// bit (warp over 32 consecutive vertices, then over each member's
// incidences)
__global__ void __launch_bounds__(256)
    k_ps_mark(Level L, const int32_t* __restrict__ rho, const int64_t* __restrict__ scal, PStar ps)
{
    if (!pstar_on(scal, ps.cnt)) return;
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < L.V; base += nw * 32) {
        int64_t n = base + lane;
        int32_t sl = n < L.V ? ps.pslot[rho[n]] : -1;
        unsigned mem = __ballot_sync(FULL, sl >= 0);
        while (mem) {
            int src = __ffs(mem) - 1;
            mem &= mem - 1;
            int32_t m = (int32_t)__shfl_sync(FULL, (int32_t)n, src);
            uint32_t bit = 1u << __shfl_sync(FULL, sl, src);
            for (int64_t i = L.voff[m] + lane; i < L.voff[m + 1]; i += 32) {
                int32_t a = (int32_t)((uint32_t)L.vinc[i] & ~SRC_BIT);
                uint32_t old = atomicOr(&ps.hmask[a], bit);
                if (old == 0) ps.hl[atomicAdd(&ps.cnt[1], 1)] = a;
            }
        }
    }
}

// columns: for each marked hyperedge and each of its slots p, every pin n
// outside p adds omega to conn(n, p) and, as a destination of a hyperedge
// inbound to p, k to ov(n, p) (counts after the moves); masks are cleared
__global__ void __launch_bounds__(256)
    k_ps_cols(Level L, PinCounts pc, const int32_t* __restrict__ rho,
              const int64_t* __restrict__ scal, PStar ps)
{
    if (!pstar_on(scal, ps.cnt)) return;
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t nh = ps.cnt[1];
    int64_t V = L.V;
    for (int64_t idx = gw; idx < nh; idx += nw) {
        int32_t a = ps.hl[idx];
        uint32_t mask = ps.hmask[a];
        int64_t b = L.hoff[a], e = L.hoff[a + 1];
        int32_t lam = pc.lam[a];
        int64_t w = L.hw[a];
        int32_t k = L.hk[a];
        int sd = L.hsd[a];
        while (mask) {
            int sl = __ffs(mask) - 1;
            mask &= mask - 1;
            int32_t p = ps.slots[sl];
            int32_t c, d;
            lookup_count(pc, b, lam, p, c, d);
            int64_t* cc = ps.colc + (int64_t)sl * V;
            int32_t* co = ps.colo + (int64_t)sl * V;
            for (int64_t j = b + lane; j < e; j += 32) {
                int32_t n = L.hpins[j];
                if (rho[n] == p) continue;
                atomicAdd((unsigned long long*)&cc[n], (unsigned long long)w);
                if (d > 0 && (j != b || sd)) atomicAdd(&co[n], k);
                atomicOr(&ps.vt[n], 1u << sl);
            }
        }
        __syncwarp();
        if (lane == 0) ps.hmask[a] = 0;
    }
}

// each vertex's proposal for the next round (or its flag for a full
// evaluation); columns read are cleared
__global__ void k_ps_combine(Level L, const int32_t* __restrict__ rho,
                             const int64_t* __restrict__ scal, PStar ps, PState st,
                             const int64_t* __restrict__ savev, const int64_t* __restrict__ Wv,
                             int32_t omega, int32_t delta, int32_t phi, int nonpos, int32_t* pto,
                             int64_t* pgain, int32_t* dirty)
{
    if (!pstar_on(scal, ps.cnt)) return;
    int32_t ns = ps.cnt[0];
    int64_t V = L.V;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        uint32_t adj = ps.vt[n];
        if (!dirty[n]) {
            int64_t ds = savev[n] - ps.save0[n];
            int32_t q = pto[n];
            if ((q >= 0 && ps.pslot[q] >= 0) || (!nonpos && q < 0 && ds > 0)) {
                dirty[n] = 1;
            } else {
                int64_t bs = q >= 0 ? pgain[n] + ds : 0;
                int32_t bk = q;
                if (adj) {
                    int64_t sw = savev[n] - Wv[n];
                    for (int sl = 0; sl < ns; sl++) {
                        if (!((adj >> sl) & 1u)) continue;
                        int32_t p = ps.slots[sl];
                        int64_t c = ps.colc[(int64_t)sl * V + n];
                        int64_t o = ps.colo[(int64_t)sl * V + n];
                        bool feas = st.size[p] + L.vsize[n] <= omega &&
                                    st.inpins[p] + L.vinpins[n] <= phi &&
                                    st.pincnt[p] + L.vincnt[n] - o <= delta;
                        if (feas && better(sw + c, p, bs, bk)) {
                            bs = sw + c;
                            bk = p;
                        }
                    }
                }
                bool prop = bk >= 0 && (bs > 0 || nonpos);
                pto[n] = prop ? bk : -1;
                pgain[n] = prop ? bs : 0;
            }
        }
        if (adj) {
            for (int sl = 0; sl < ns; sl++) {
                if (!((adj >> sl) & 1u)) continue;
                ps.colc[(int64_t)sl * V + n] = 0;
                ps.colo[(int64_t)sl * V + n] = 0;
            }
            ps.vt[n] = 0;
        }
    }
}

// The same update on levels refined from connection rows: a vertex's
// columns of P* are entries of its row (already updated by k_dense_cross;
// adjacency is a positive entry there, rows being used only when every
// omega is positive). With more than PSTAR_MAX partitions in P*, every
// vertex is flagged for a row scan.
__global__ void k_ps_rows(Level L, const int32_t* __restrict__ rho,
                          const int64_t* __restrict__ scal, PStar ps, PState st,
                          const int64_t* __restrict__ savev, const int64_t* __restrict__ Wv,
                          const int32_t* __restrict__ rowid, const int32_t* __restrict__ C,
                          const int32_t* __restrict__ O, int64_t Kp, int32_t omega,
                          int32_t delta, int32_t phi, int nonpos, int32_t* pto, int64_t* pgain,
                          int32_t* dirty)
{
    if (scal[RS_BEST] <= 0) return;
    bool on = ps.cnt[0] <= PSTAR_MAX;
    int32_t ns = on ? ps.cnt[0] : 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < L.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        if (!on) {
            dirty[n] = 1;
            continue;
        }
        if (dirty[n]) continue;   // moved
        int64_t ds = savev[n] - ps.save0[n];
        int32_t q = pto[n];
        if ((q >= 0 && ps.pslot[q] >= 0) || (!nonpos && q < 0 && ds > 0)) {
            dirty[n] = 1;
            continue;
        }
        int64_t bs = q >= 0 ? pgain[n] + ds : 0;
        int32_t bk = q;
        int64_t r0 = (int64_t)rowid[n] * Kp;
        int64_t sw = savev[n] - Wv[n];
        int32_t own = rho[n];
        for (int sl = 0; sl < ns; sl++) {
            int32_t p = ps.slots[sl];
            int64_t c = C[r0 + p];
            if (p == own || c <= 0) continue;
            bool feas = st.size[p] + L.vsize[n] <= omega && st.inpins[p] + L.vinpins[n] <= phi &&
                        st.pincnt[p] + L.vincnt[n] - (int64_t)O[r0 + p] <= delta;
            if (feas && better(sw + c, p, bs, bk)) {
                bs = sw + c;
                bk = p;
            }
        }
        bool prop = bk >= 0 && (bs > 0 || nonpos);
        pto[n] = prop ? bk : -1;
        pgain[n] = prop ? bs : 0;
    }
}

// slot map and counters back to empty
__global__ void k_ps_reset(int32_t M, Moves mv, const int64_t* __restrict__ scal, PStar ps)
{
    int64_t istar = scal[RS_BEST] > 0 ? scal[RS_ISTAR] : -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= istar && i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        ps.pslot[mv.from[i]] = -1;
        ps.pslot[mv.to[i]] = -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ps.cnt[0] = ps.cnt[2];
        ps.cnt[1] = 0;
    }
}

// ---------------------------------------------------------------------------
// S8

__global__ void k_prop_stats(Level L, const int32_t* __restrict__ pto,
                             const int64_t* __restrict__ pgain,
                             const int64_t* __restrict__ savev,
                             const int32_t* __restrict__ dirty, int nonpos, int32_t* flag,
                             int64_t* scal)
{
    int64_t mg = 0, ng = 0, deg = 0;
    int act = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < L.V;
         n += (int64_t)gridDim.x * blockDim.x) {
        act += (nonpos || savev[n] > 0) && (!dirty || dirty[n]);
        int f = pto[n] >= 0;
        flag[n] = f;
        if (f) {
            mg = pgain[n] > mg ? pgain[n] : mg;
            ng = pgain[n] < ng ? pgain[n] : ng;
            deg += L.voff[n + 1] - L.voff[n];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int64_t m2 = __shfl_xor_sync(FULL, mg, o);
        mg = m2 > mg ? m2 : mg;
        int64_t n2 = __shfl_xor_sync(FULL, ng, o);
        ng = n2 < ng ? n2 : ng;
        deg += __shfl_xor_sync(FULL, deg, o);
    }
    act = warp_sum(act);
    if ((threadIdx.x & 31) == 0) {
        if (mg) atomicMax((unsigned long long*)&scal[RS_MAXG], (unsigned long long)mg);
        if (deg) atomicAdd((unsigned long long*)&scal[RS_DEG], (unsigned long long)deg);
        if (act) atomicAdd((unsigned long long*)&scal[RS_ACT], (unsigned long long)act);
        if (ng < 0) atomicMin((long long*)&scal[RS_MING], (long long)ng);
    }
}

__global__ void k_prop_keys(int32_t V, const int32_t* __restrict__ pto,
                            const int64_t* __restrict__ pgain, const int32_t* __restrict__ pos,
                            int64_t maxg, uint64_t* keys, uint32_t* vals)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        if (pto[n] < 0) continue;
        int32_t i = pos[n];
        keys[i] = (uint64_t)(maxg - pgain[n]);
        vals[i] = (uint32_t)n;
    }
}

__global__ void k_moves(int32_t M, const uint32_t* __restrict__ vals, const int32_t* __restrict__ rho,
                        const int32_t* __restrict__ pto, Moves mv, int32_t* moveidx)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = (int32_t)vals[i];
        mv.n[i] = n;
        mv.from[i] = rho[n];
        mv.to[i] = pto[n];
        moveidx[n] = (int32_t)i;
    }
}

// ---------------------------------------------------------------------------
// The list of hyperedges holding a proposed move, from the proposers'
// incidence lists.

__global__ void __launch_bounds__(256)
    k_prop_hedges(int32_t M, Moves mv, Level L, int32_t* hmark, int32_t* list, int32_t* n)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < M; i += nw) {
        int32_t v = mv.n[i];
        for (int64_t j = L.voff[v] + lane; j < L.voff[v + 1]; j += 32) {
            int32_t a = (int32_t)((uint32_t)L.vinc[j] & ~SRC_BIT);
            if (atomicExch(&hmark[a], 1) == 0) list[atomicAdd(n, 1)] = a;
        }
    }
}

// the marks of the listed hyperedges back to zero for the next round
__global__ void k_hedges_clear(HedgeList hl, int32_t* hmark, int32_t* hdirty)
{
    int32_t nh = *hl.n;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nh;
         x += (int64_t)gridDim.x * blockDim.x) {
        hmark[hl.a[x]] = 0;
        hdirty[hl.a[x]] = 0;
    }
}

// ---------------------------------------------------------------------------
// S9 / S10 events

struct Events {
    uint64_t* key;   // partition << ibits | move
    uint32_t* idx;   // 0..n-1 (sort values)
    int32_t* dsize;
    int32_t* dinp;
    int32_t* dpc;
    int64_t cap;
    int ibits;
};

__global__ void k_size_events(int32_t M, Moves mv, Level L, Events ev)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = mv.n[i];
        int64_t e0 = 2 * i, e1 = 2 * i + 1;
        ev.key[e0] = ((uint64_t)mv.from[i] << ev.ibits) | (uint64_t)i;
        ev.key[e1] = ((uint64_t)mv.to[i] << ev.ibits) | (uint64_t)i;
        ev.idx[e0] = (uint32_t)e0;
        ev.idx[e1] = (uint32_t)e1;
        ev.dsize[e0] = -L.vsize[n];
        ev.dsize[e1] = L.vsize[n];
        ev.dinp[e0] = -L.vinpins[n];
        ev.dinp[e1] = L.vinpins[n];
        ev.dpc[e0] = -L.vinint[n];
        ev.dpc[e1] = L.vinint[n];
    }
}

__device__ __forceinline__ void emit_inbound(const Events& ev, int64_t* scal, int64_t base,
                                             int32_t p, int32_t mi, int32_t d)
{
    int64_t pos = base + (int64_t)atomicAdd((unsigned long long*)&scal[RS_NEV], 1ull);
    if (pos >= ev.cap) {
        atomicOr((int*)&scal[SC_STATUS], ST_CAPACITY);
        return;
    }
    ev.key[pos] = ((uint64_t)p << ev.ibits) | (uint64_t)mi;
    ev.idx[pos] = (uint32_t)pos;
    ev.dsize[pos] = 0;
    ev.dinp[pos] = 0;
    ev.dpc[pos] = d;
}

// one moved pin's replay given the deltas of earlier moves of the same hyperedge
__device__ __forceinline__ void replay_one(const Level& L, const PinCounts& pc, int32_t a,
                                           int32_t mi, int32_t f, int32_t t, int d, int dcf_c,
                                           int dct_c, int dcf_d, int dct_d, int64_t* gp,
                                           const Events& ev, int64_t* scal, int64_t evbase)
{
    int64_t b = L.hoff[a];
    int32_t lam = pc.lam[a];
    int32_t c0f, d0f, c0t, d0t;
    lookup_count(pc, b, lam, f, c0f, d0f);
    lookup_count(pc, b, lam, t, c0t, d0t);
    int32_t cf = c0f + dcf_c, ct = c0t + dct_c;
    int64_t g = (int64_t)L.hw[a] * ((cf == 1 ? 1 : 0) - (ct == 0 ? 1 : 0));
    if (g) atomicAdd((unsigned long long*)&gp[mi], (unsigned long long)g);
    if (d) {
        if (d0f + dcf_d == 1) emit_inbound(ev, scal, evbase, f, mi, -L.hk[a]);
        if (d0t + dct_d == 0) emit_inbound(ev, scal, evbase, t, mi, L.hk[a]);
    }
}

__global__ void __launch_bounds__(256)
    k_replay_warp(Level L, PinCounts pc, const int32_t* __restrict__ moveidx, Moves mv,
                  uint32_t* mvbuf, int64_t* gp, Events ev, int64_t evbase, int32_t* heavy,
                  int32_t* heavycnt, int64_t* scal, HedgeList hl)
{
    int lane = threadIdx.x & 31;
    unsigned lt = lanemask_lt();
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t nh = *hl.n;
    for (int64_t x = gw; x < nh; x += nw) {
        int32_t a = hl.a[x];
        int64_t b = L.hoff[a], e = L.hoff[a + 1];
        int sd = L.hsd[a];
        int cnt = 0;
        for (int64_t cb = b; cb < e; cb += 32) {
            int64_t j = cb + lane;
            int32_t mi = -1;
            if (j < e) mi = moveidx[L.hpins[j]];
            bool moved = mi >= 0;
            unsigned mk = __ballot_sync(FULL, moved);
            if (moved) {
                uint32_t d = (j != b || sd) ? 1u : 0u;
                mvbuf[b + cnt + __popc(mk & lt)] = ((uint32_t)mi << 1) | d;
            }
            cnt += __popc(mk);
        }
        if (cnt == 0) continue;
        __syncwarp();
        if (cnt > REPLAY_WARP_MAX) {
            if (lane == 0) {
                int32_t pos = atomicAdd((int*)&scal[RS_NHV], 1);
                heavy[pos] = (int32_t)a;
                heavycnt[pos] = cnt;
            }
            continue;
        }
        uint32_t rec = lane < cnt ? mvbuf[b + lane] : 0u;
        int32_t mi = (int32_t)(rec >> 1);
        int d = rec & 1;
        int32_t f = lane < cnt ? mv.from[mi] : -1;
        int32_t t = lane < cnt ? mv.to[mi] : -1;
        int dcf_c = 0, dct_c = 0, dcf_d = 0, dct_d = 0;
        for (int jj = 0; jj < cnt; jj++) {
            int32_t mj = __shfl_sync(FULL, mi, jj);
            int32_t fj = __shfl_sync(FULL, f, jj);
            int32_t tj = __shfl_sync(FULL, t, jj);
            int dj = __shfl_sync(FULL, d, jj);
            if (mj < mi) {
                int ef = (tj == f) - (fj == f), et = (tj == t) - (fj == t);
                dcf_c += ef;
                dct_c += et;
                if (dj) {
                    dcf_d += ef;
                    dct_d += et;
                }
            }
        }
        if (lane < cnt)
            replay_one(L, pc, (int32_t)a, mi, f, t, d, dcf_c, dct_c, dcf_d, dct_d, gp, ev, scal, evbase);
    }
}

__global__ void __launch_bounds__(256)
    k_replay_block(Level L, PinCounts pc, Moves mv, const uint32_t* __restrict__ mvbuf, int64_t* gp,
                   Events ev, int64_t evbase, const int32_t* __restrict__ heavy,
                   const int32_t* __restrict__ heavycnt, int64_t* scal)
{
    int32_t nh = (int32_t)scal[RS_NHV];
    for (int32_t h = blockIdx.x; h < nh; h += gridDim.x) {
        int32_t a = heavy[h];
        int32_t cnt = heavycnt[h];
        int64_t b = L.hoff[a];
        for (int32_t x = threadIdx.x; x < cnt; x += blockDim.x) {
            uint32_t rec = mvbuf[b + x];
            int32_t mi = (int32_t)(rec >> 1);
            int d = rec & 1;
            int32_t f = mv.from[mi], t = mv.to[mi];
            int dcf_c = 0, dct_c = 0, dcf_d = 0, dct_d = 0;
            for (int32_t y = 0; y < cnt; y++) {
                uint32_t ry = mvbuf[b + y];
                int32_t mj = (int32_t)(ry >> 1);
                if (mj >= mi) continue;
                int32_t fj = mv.from[mj], tj = mv.to[mj];
                int ef = (tj == f) - (fj == f), et = (tj == t) - (fj == t);
                dcf_c += ef;
                dct_c += et;
                if (ry & 1) {
                    dcf_d += ef;
                    dct_d += et;
                }
            }
            replay_one(L, pc, a, mi, f, t, d, dcf_c, dct_c, dcf_d, dct_d, gp, ev, scal, evbase);
        }
    }
}

// ---------------------------------------------------------------------------
// S10

__global__ void k_part_bounds(int64_t T, const uint64_t* __restrict__ key, int ibits, int32_t* pbeg,
                              int32_t* pend)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < T;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t p = key[e] >> ibits;
        if (e == 0 || (key[e - 1] >> ibits) != p) pbeg[p] = (int32_t)e;
        if (e == T - 1 || (key[e + 1] >> ibits) != p) pend[p] = (int32_t)(e + 1);
    }
}

__global__ void __launch_bounds__(256)
    k_part_validity(int32_t K, const int32_t* __restrict__ pbeg, const int32_t* __restrict__ pend,
                    Events ev, PState ps, int32_t omega, int32_t delta, int32_t phi, int32_t* dv)
{
    int lane = threadIdx.x & 31;
    unsigned lt = lanemask_lt();
    uint64_t imask = (ev.ibits >= 64) ? ~0ull : ((1ull << ev.ibits) - 1);
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = gw; p < K; p += nw) {
        int32_t beg = pbeg[p], end = pend[p];
        if (beg >= end) continue;
        int64_t s0 = ps.size[p], i0 = ps.inpins[p], c0 = ps.pincnt[p];
        int64_t cs = 0, ci = 0, cc = 0;
        int prev_viol = 0;
        for (int32_t cb = beg; cb < end; cb += 32) {
            int32_t e = cb + lane;
            bool valid = e < end;
            int64_t mi = -1, ds = 0, di = 0, dc = 0;
            if (valid) {
                mi = (int64_t)(ev.key[e] & imask);
                uint32_t x = ev.idx[e];
                ds = ev.dsize[x];
                di = ev.dinp[x];
                dc = ev.dpc[x];
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int64_t a1 = __shfl_up_sync(FULL, ds, o);
                int64_t a2 = __shfl_up_sync(FULL, di, o);
                int64_t a3 = __shfl_up_sync(FULL, dc, o);
                if (lane >= o) {
                    ds += a1;
                    di += a2;
                    dc += a3;
                }
            }
            int64_t nmi = __shfl_down_sync(FULL, mi, 1);
            if (lane == 31) nmi = (e + 1 < end) ? (int64_t)(ev.key[e + 1] & imask) : -1;
            if (valid && e + 1 >= end) nmi = -1;
            bool gend = valid && nmi != mi;
            int viol = gend ? (violates(s0 + cs + ds, i0 + ci + di, c0 + cc + dc, omega, delta, phi) ? 1 : 0) : 0;
            unsigned gm = __ballot_sync(FULL, gend);
            unsigned below = gm & lt;
            int src = below ? 31 - __clz(below) : lane;
            int pv = __shfl_sync(FULL, viol, src);
            if (!below) pv = prev_viol;
            if (gend && viol != pv) atomicAdd(&dv[mi], viol - pv);
            if (gm) prev_viol = __shfl_sync(FULL, viol, 31 - __clz(gm));
            cs += __shfl_sync(FULL, ds, 31);
            ci += __shfl_sync(FULL, di, 31);
            cc += __shfl_sync(FULL, dc, 31);
        }
    }
}

// ---------------------------------------------------------------------------
// S11

__global__ void k_best1(int32_t M, const int64_t* __restrict__ G, const int32_t* __restrict__ nviol,
                        int64_t* scal)
{
    int64_t best = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x)
        if (nviol[i] == 0 && G[i] > best) best = G[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int64_t b2 = __shfl_xor_sync(FULL, best, o);
        best = b2 > best ? b2 : best;
    }
    if ((threadIdx.x & 31) == 0 && best > 0)
        atomicMax((unsigned long long*)&scal[RS_BEST], (unsigned long long)best);
}

__global__ void k_best2(int32_t M, const int64_t* __restrict__ G, const int32_t* __restrict__ nviol,
                        int64_t* scal)
{
    int64_t best = scal[RS_BEST];
    if (best <= 0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x)
        if (nviol[i] == 0 && G[i] == best) atomicMin((unsigned long long*)&scal[RS_ISTAR], (unsigned long long)i);
}

__global__ void k_apply(int32_t M, Moves mv, int32_t* rho, int32_t* moveidx, const int64_t* scal)
{
    int64_t istar = scal[RS_BEST] > 0 ? scal[RS_ISTAR] : -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i <= istar) rho[mv.n[i]] = mv.to[i];
        moveidx[mv.n[i]] = -1;
    }
}

__global__ void k_round_init(int64_t* scal) { scal[RS_ISTAR] = INT64_MAX; }

// ---------------------------------------------------------------------------

template <typename S>
static Status gains(snnmap_hgraph* h, Level& L, const PinCounts& pc, const int32_t* rho,
                    const PState& ps, int32_t K, int32_t* pto, int64_t* pgain,
                    const int64_t* savev, const int32_t* dirty)
{
    GainPol<S> pol;
    pol.savev = savev;
    pol.dirty = dirty;
    pol.nonpos = h->prm.refine_nonpositive != 0;
    pol.L = L;
    pol.pc = pc;
    pol.ps = ps;
    pol.rho = rho;
    pol.V = L.V;
    pol.keys = K;
    pol.omega = h->prm.omega;
    pol.delta = h->prm.delta;
    pol.phi = h->prm.phi;
    pol.pto = pto;
    pol.pgain = pgain;
    int64_t* cnt;
    SNN_TRY(h->scratch.alloc(&cnt, HT_NCNT));
    return run_histogram(pol, h->scratch, h->stream, cnt, h->h_scal + 12, h->d_scal, h->tiers);
}

// rows of the vertices flagged fresh, from the round's pin counts
static Status dense_fresh(snnmap_hgraph* h, Level& L, const PinCounts& pc)
{
    DenseRows& D = h->dense;
    RowPol<uint32_t> pol;
    pol.L = L;
    pol.pc = pc;
    pol.V = L.V;
    pol.keys = D.K;
    pol.fresh = D.fresh;
    pol.rowid = D.rowid;
    pol.C = D.C;
    pol.O = D.O;
    pol.Kp = D.Kp;
    pol.M = D.M;
    pol.cw = D.cw;
    int64_t* cnt;
    SNN_TRY(h->scratch.alloc(&cnt, HT_NCNT));
    return run_histogram(pol, h->scratch, h->stream, cnt, h->h_scal + 12, h->d_scal, h->tiers);
}

int64_t dense_row_budget(const snnmap_hgraph* h)
{
    if (h->row_budget >= 0) return h->row_budget;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
    return (int64_t)(tot / 4);
}

Status dense_open(snnmap_hgraph* h, int32_t K, int64_t rows)
{
    dense_close(h);
    DenseRows& D = h->dense;
    cudaStream_t s = h->stream;
    D.K = K;
    D.Kp = ((int64_t)K + 3) & ~(int64_t)3;
    D.cap = rows > 0 ? rows : 1;
    SNN_CUDA(dev_malloc(&D.C, (size_t)(D.cap * D.Kp) * 4, s));
    SNN_CUDA(dev_malloc(&D.O, (size_t)(D.cap * D.Kp) * 4, s));
    SNN_CUDA(dev_malloc(&D.rowid, (size_t)D.cap * 4, s));
    SNN_CUDA(dev_malloc(&D.rowid2, (size_t)D.cap * 4, s));
    SNN_CUDA(dev_malloc(&D.fresh, (size_t)D.cap * 4, s));
    SNN_CUDA(dev_malloc(&D.M, (size_t)D.cap * 8, s));
    D.cw = 32;
    while ((int64_t)D.cw * 64 < D.Kp) D.cw <<= 1;
    D.level = -1;
    D.pending = false;
    return Status{};
}

void dense_close(snnmap_hgraph* h)
{
    DenseRows& D = h->dense;
    for (int32_t* p : {D.C, D.O, D.rowid, D.rowid2, D.fresh})
        if (p) cudaFreeAsync(p, h->stream);
    if (D.M) cudaFreeAsync(D.M, h->stream);
    D = DenseRows{};
}

Status dense_begin(snnmap_hgraph* h, int32_t level)
{
    DenseRows& D = h->dense;
    const Level& L = h->levels[level];
    if (!D.C || L.V > D.cap) return Status{SNNMAP_ERR_STATE, "connection rows: capacity"};
    SNN_TRY(iota_i32(D.rowid, L.V, h->stream));
    SNN_TRY(fill_i32(D.fresh, 1, L.V, h->stream));
    if (L.V > 0) {
        SNN_L k_dense_zero<<<grid_for((int64_t)L.V * 32, 256), 256, 0, h->stream>>>(L.V, D.fresh, D.rowid,
                                                                            D.C, D.O, D.M, D.Kp);
        SNN_CUDA(cudaGetLastError());
    }
    D.level = level;
    D.pending = true;
    return Status{};
}

Status dense_descend(snnmap_hgraph* h, int32_t level)
{
    DenseRows& D = h->dense;
    const Level& L = h->levels[level];
    int32_t Vc = h->levels[level + 1].V;
    if (!D.C || D.level != level + 1 || L.V > D.cap)
        return Status{SNNMAP_ERR_STATE, "connection rows: descent out of order"};
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    int32_t *mcount, *first, *nonrep, *idx;
    SNN_TRY(ar.alloc(&mcount, Vc));
    SNN_TRY(ar.alloc(&first, Vc));
    SNN_TRY(ar.alloc(&nonrep, L.V));
    SNN_TRY(ar.alloc(&idx, L.V));
    SNN_CUDA(cudaMemsetAsync(mcount, 0, (size_t)(Vc > 0 ? Vc : 1) * 4, s));
    SNN_TRY(fill_i32(first, INT_MAX, Vc, s));
    if (L.V > 0) {
        int g = grid_for(L.V, 256);
        SNN_L k_dense_members<<<g, 256, 0, s>>>(L.V, L.cid, mcount, first);
        SNN_L k_dense_flags<<<g, 256, 0, s>>>(L.V, L.cid, mcount, first, nonrep, D.fresh);
        SNN_CUDA(cudaGetLastError());
        SNN_TRY(scan_exclusive_i32(nonrep, idx, L.V, nullptr, ar, s));
        SNN_L k_dense_rowid<<<g, 256, 0, s>>>(L.V, Vc, L.cid, nonrep, idx, D.rowid, D.rowid2);
        SNN_CUDA(cudaGetLastError());
        std::swap(D.rowid, D.rowid2);
        SNN_L k_dense_zero<<<grid_for((int64_t)L.V * 32, 256), 256, 0, s>>>(L.V, D.fresh, D.rowid, D.C,
                                                                     D.O, D.M, D.Kp);
        SNN_CUDA(cudaGetLastError());
    }
    D.level = level;
    D.pending = true;
    return Status{};
}

// pin counts + partition state + Conn for rho, into buffers the caller owns
// (Conn is added to *cost)
static Status pin_counts_into(snnmap_hgraph* h, Level& L, LevelExtra& X, int32_t K,
                              const int32_t* rho, PinCounts& pc, PState& ps, int64_t* cost)
{
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    SNN_CUDA(cudaMemsetAsync(ps.size, 0, (size_t)K * 8, s));
    SNN_CUDA(cudaMemsetAsync(ps.inpins, 0, (size_t)K * 8, s));
    SNN_CUDA(cudaMemsetAsync(ps.pincnt, 0, (size_t)K * 8, s));
    if (L.V > 0) {
        SNN_L k_pstate_vertices<<<grid_for(L.V, 256), 256, 0, s>>>(L, rho, ps);
        SNN_CUDA(cudaGetLastError());
    }
    int64_t* slots;
    SNN_TRY(ar.alloc(&slots, COST_SLOTS));
    SNN_CUDA(cudaMemsetAsync(slots, 0, COST_SLOTS * sizeof(int64_t), s));
    PinCountJob job{L.hoff, L.hpins, L.hsd, L.hk, L.hw, rho, pc, ps.pincnt, slots};
    SNN_TRY(seg_run(job, X.seg, L.E, ar, s));
    SNN_L k_cost_slots<<<1, 256, 0, s>>>(slots, cost);
    SNN_CUDA(cudaGetLastError());
    return Status{};
}

static Status pin_counts(snnmap_hgraph* h, Level& L, LevelExtra& X, int32_t K, const int32_t* rho,
                         PinCounts& pc, PState& ps)
{
    Arena& ar = h->scratch;
    SNN_TRY(ar.alloc(&pc.p, L.P));
    SNN_TRY(ar.alloc(&pc.cnt, L.P));
    SNN_TRY(ar.alloc(&pc.dcnt, L.P));
    SNN_TRY(ar.alloc(&pc.lam, L.E));
    SNN_TRY(ar.alloc(&ps.size, K));
    SNN_TRY(ar.alloc(&ps.inpins, K));
    SNN_TRY(ar.alloc(&ps.pincnt, K));
    return pin_counts_into(h, L, X, K, rho, pc, ps, h->d_scal + RS_COST);
}

Status level_cost(snnmap_hgraph* h, int32_t level, int32_t K, const int32_t* rho, int64_t* cost)
{
    Level& L = h->levels[level];
    LevelExtra& X = h->extra[level];
    SNN_TRY(zero_scalars(h));
    PinCounts pc;
    PState ps;
    SNN_TRY(pin_counts(h, L, X, K, rho, pc, ps));
    SNN_TRY(read_scalars(h));
    h->scratch.reset();
    *cost = h->h_scal[RS_COST];
    return Status{};
}

// ---------------------------------------------------------------------------
// Carried pin counts. Only hyperedges holding a pin of the enacted prefix
// change their counts; their old contributions (inbound k per partition,
// omega (lambda - 1) to Conn, omega to the save of a pin alone in its
// partition) are taken out before the moves, the moves' own size, inbound
// pins and internal axons move between partitions, the hyperedges are
// counted again, and their new contributions added back.

__global__ void __launch_bounds__(256)
    k_pc_mark(Level L, const int32_t* __restrict__ moveidx, const int64_t* __restrict__ scal,
              int32_t* hdirty, HedgeList hl)
{
    int64_t istar = scal[RS_BEST] > 0 ? scal[RS_ISTAR] : -1;
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t nh = *hl.n;
    for (int64_t x = gw; x < nh; x += nw) {
        int32_t a = hl.a[x];
        bool hit = false;
        if (istar >= 0)
            for (int64_t j = L.hoff[a] + lane; j < L.hoff[a + 1] && !hit; j += 32) {
                int32_t mi = moveidx[L.hpins[j]];
                if (mi >= 0 && mi <= istar) hit = true;
            }
        hit = __any_sync(FULL, hit);
        if (lane == 0) hdirty[a] = hit ? 1 : 0;
    }
}

// sign -1: remove the contributions of the marked hyperedges under the
// current counts and rho; sign +1: add them
__global__ void __launch_bounds__(256)
    k_pc_contrib(Level L, PinCounts pc, const int32_t* __restrict__ hdirty,
                 const int32_t* __restrict__ rho, PState ps, int64_t* savev, int64_t* costv,
                 int sign, HedgeList hl)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t nh = *hl.n;
    for (int64_t x = gw; x < nh; x += nw) {
        int32_t a = hl.a[x];
        if (!hdirty[a]) continue;
        int64_t b = L.hoff[a], e = L.hoff[a + 1];
        int32_t lam = pc.lam[a];
        int64_t w = L.hw[a];
        int64_t k = L.hk[a];
        if (sign < 0) {
            // the count pass adds inbound k and Conn itself for sign +1
            for (int32_t r = lane; r < lam; r += 32)
                if (pc.dcnt[b + r] > 0) atomicAdd((unsigned long long*)&ps.pincnt[pc.p[b + r]],
                                                  (unsigned long long)(-k));
            if (lane == 0 && lam > 1)
                atomicAdd((unsigned long long*)costv, (unsigned long long)(-(w * (lam - 1))));
        }
        for (int64_t j = b + lane; j < e; j += 32) {
            int32_t x = L.hpins[j];
            int32_t c, d;
            lookup_count(pc, b, lam, rho[x], c, d);
            if (c == 1) atomicAdd((unsigned long long*)&savev[x], (unsigned long long)(sign * w));
        }
    }
}

// the enacted moves' own size, inbound pins and internal axons change
// partition
__global__ void k_ps_moves(int32_t M, Moves mv, Level L, const int64_t* __restrict__ scal, PState ps)
{
    int64_t istar = scal[RS_BEST] > 0 ? scal[RS_ISTAR] : -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= istar && i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = mv.n[i], f = mv.from[i], t = mv.to[i];
        int64_t sz = L.vsize[n], ip = L.vinpins[n], ii = L.vinint[n];
        atomicAdd((unsigned long long*)&ps.size[f], (unsigned long long)(-sz));
        atomicAdd((unsigned long long*)&ps.size[t], (unsigned long long)sz);
        atomicAdd((unsigned long long*)&ps.inpins[f], (unsigned long long)(-ip));
        atomicAdd((unsigned long long*)&ps.inpins[t], (unsigned long long)ip);
        if (ii) {
            atomicAdd((unsigned long long*)&ps.pincnt[f], (unsigned long long)(-ii));
            atomicAdd((unsigned long long*)&ps.pincnt[t], (unsigned long long)ii);
        }
    }
}

// the level's size buckets restricted to marked hyperedges (each bucket keeps
// its start; counts by atomics, order irrelevant)
__global__ void k_seg_filter(const int32_t* __restrict__ list, const int32_t* __restrict__ meta,
                             int32_t E, const int32_t* __restrict__ hdirty, int32_t* out,
                             int32_t* meta2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = list[i];
        if (!hdirty[a]) continue;
        int b = 0;
        while (b + 1 < SEG_NB && i >= meta[b + 1]) b++;
        int32_t pos = atomicAdd(&meta2[SEG_NB + b], 1);
        out[meta[b] + pos] = a;
    }
}

__global__ void k_seg_meta_copy(const int32_t* __restrict__ meta, int32_t* meta2)
{
    for (int b = threadIdx.x; b < SEG_NB; b += blockDim.x) meta2[b] = meta[b];
}

__global__ void k_copy_i64(const int64_t* __restrict__ src, int64_t* dst) { *dst = *src; }

// Per-level buffers that outlive a round: proposals (kept by vertices the
// previous round did not touch), the vertices to evaluate, partition flags
// and the level's largest vertex state.
struct IncState {
    int32_t* pto = nullptr;
    int64_t* pgain = nullptr;
    int32_t* dirty = nullptr;
    uint8_t* pchg = nullptr;
    uint8_t* prel = nullptr;
    int32_t* vmax = nullptr;
    // pin counts, partition state, Conn (costv), save and W carried from
    // round to round: a round after the first starts from them, and the
    // enacted prefix updates them for the hyperedges holding a moved pin
    PinCounts pc;
    PState ps;
    int64_t* costv = nullptr;
    int64_t* savev = nullptr;
    int64_t* Wv = nullptr;
    int32_t* hdirty = nullptr;   // per hyperedge
    int32_t* hmark = nullptr;    // per hyperedge: listed this round (k_prop_hedges)
    int32_t* hlist = nullptr;    // bucket lists filtered to dirty hyperedges
    int32_t* hmeta = nullptr;    // their bucket starts and counts (2 * SEG_NB)
    bool ready = false;          // set once the first round computed them
    PStar pst;                   // column update of proposals after short prefixes
};

// One round; *applied = moves enacted, *gain = Conn removed, *cost = Conn at
// round start.
static Status refine_round(snnmap_hgraph* h, int32_t level, int32_t K, int32_t* rho,
                           int32_t* moveidx, const IncState& inc, int32_t* n_props,
                           int32_t* applied, int64_t* gain, int64_t* cost, int32_t* n_active,
                           int32_t* rows)
{
    cudaStream_t s = h->stream;
    Arena& ar = h->scratch;
    Level& L = h->levels[level];
    LevelExtra& X = h->extra[level];
    const snnmap_params& prm = h->prm;
    int32_t V = L.V;
    *n_props = 0;
    *n_active = 0;
    *rows = 0;
    *applied = 0;
    *gain = 0;
    SNN_TRY(zero_scalars(h));
    SNN_L k_round_init<<<1, 1, 0, s>>>(h->d_scal);
    SNN_CUDA(cudaGetLastError());

    PinCounts pc = inc.pc;
    PState ps = inc.ps;
    {
        ProfScope prof(h, PS_PINCOUNT);
        if (!inc.ready) {
            SNN_CUDA(cudaMemsetAsync(inc.costv, 0, sizeof(int64_t), s));
            SNN_TRY(pin_counts_into(h, L, X, K, rho, pc, ps, inc.costv));
        }
        SNN_L k_copy_i64<<<1, 1, 0, s>>>(inc.costv, h->d_scal + RS_COST);
        SNN_L k_check_pstate<<<grid_for(K, 256), 256, 0, s>>>(K, ps, prm.omega, prm.delta, prm.phi, h->d_scal);
        SNN_CUDA(cudaGetLastError());
    }
    DenseRows& D = h->dense;
    const bool dense = D.C && D.level == level;
    std::unique_ptr<ProfScope> prof;
    if (dense && D.pending) {
        prof.reset(new ProfScope(h, PS_ROWS));
        SNN_TRY(dense_fresh(h, L, pc));
        D.pending = false;
    }
    int32_t* pto = inc.pto;
    int64_t* pgain = inc.pgain;
    int32_t *flag, *pos;
    int64_t* savev = inc.savev;
    int64_t* Wv = inc.Wv;
    SNN_TRY(ar.alloc(&flag, V));
    SNN_TRY(ar.alloc(&pos, V));
    if (!inc.ready) {
        prof.reset(new ProfScope(h, PS_SAVE));
        SNN_CUDA(cudaMemsetAsync(savev, 0, (size_t)(V > 0 ? V : 1) * 8, s));
        SNN_CUDA(cudaMemsetAsync(Wv, 0, (size_t)(V > 0 ? V : 1) * 8, s));
        if (L.E > 0) {
            SNN_HEDGE_LAUNCH(hedge_lanes(L.P, L.E), k_save, L.E, s, L, pc, rho, savev, Wv);
            SNN_CUDA(cudaGetLastError());
        }
    }
    prof.reset(new ProfScope(h, PS_GAINS));
    if (dense) {
        if (V > 0) {
            SNN_L k_dense_best<<<grid_for((int64_t)V * 32, 256), 256, 0, s>>>(
                L, rho, ps, savev, Wv, D.rowid, D.C, D.O, D.M, D.cw, D.Kp, K, prm.omega, prm.delta,
                prm.phi, prm.refine_nonpositive, pto, pgain, inc.dirty);
            SNN_CUDA(cudaGetLastError());
        }
    } else if (h->wide) {
        SNN_TRY(gains<unsigned long long>(h, L, pc, rho, ps, K, pto, pgain, savev, inc.dirty));
    } else {
        SNN_TRY(gains<uint32_t>(h, L, pc, rho, ps, K, pto, pgain, savev, inc.dirty));
    }
    int gv = grid_for(V, 256);
    SNN_L k_prop_stats<<<gv, 256, 0, s>>>(L, pto, pgain, savev, dense ? nullptr : inc.dirty,
                                          prm.refine_nonpositive, flag, h->d_scal);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(scan_exclusive_i32(flag, pos, V, (int32_t*)(h->d_scal + RS_M), ar, s));
    prof.reset();
    SNN_TRY(read_scalars(h));
    *cost = h->h_scal[RS_COST];
    *n_active = (int32_t)h->h_scal[RS_ACT];
    *rows = dense ? 1 : 0;
    if (h->h_scal[SC_STATUS] & ST_BADSTATE)
        return Status{SNNMAP_ERR_INVALID, "refinement input breaks a per-core limit"};
    int32_t M = (int32_t)(h->h_scal[RS_M] & 0xffffffff);
    int64_t maxg = h->h_scal[RS_MAXG];
    int64_t ming = h->h_scal[RS_MING];   // <= 0: keys maxg - gain span maxg - ming
    int64_t deg = h->h_scal[RS_DEG];
    *n_props = M;
    if (M == 0) return Status{};

    // S8
    prof.reset(new ProfScope(h, PS_SORTMOVES));
    uint64_t *keys, *keys2;
    uint32_t *vals, *vals2;
    SNN_TRY(ar.alloc(&keys, M));
    SNN_TRY(ar.alloc(&keys2, M));
    SNN_TRY(ar.alloc(&vals, M));
    SNN_TRY(ar.alloc(&vals2, M));
    SNN_L k_prop_keys<<<gv, 256, 0, s>>>(V, pto, pgain, pos, maxg, keys, vals);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(radix_sort_pairs(keys, vals, keys2, vals2, M, bits_for((uint64_t)(maxg - ming)), ar, s));
    Moves mv;
    SNN_TRY(ar.alloc(&mv.n, M));
    SNN_TRY(ar.alloc(&mv.from, M));
    SNN_TRY(ar.alloc(&mv.to, M));
    int gm = grid_for(M, 256);
    SNN_L k_moves<<<gm, 256, 0, s>>>(M, vals, rho, pto, mv, moveidx);
    SNN_CUDA(cudaGetLastError());
    // the hyperedges holding a proposed move
    int64_t nhl = std::max<int64_t>(1, std::min<int64_t>(L.E, deg));
    int32_t *hla, *hln;
    SNN_TRY(ar.alloc(&hla, nhl));
    SNN_TRY(ar.alloc(&hln, 1));
    SNN_CUDA(cudaMemsetAsync(hln, 0, sizeof(int32_t), s));
    SNN_L k_prop_hedges<<<grid_for((int64_t)M * 32, 256), 256, 0, s>>>(M, mv, L, inc.hmark, hla, hln);
    SNN_CUDA(cudaGetLastError());
    HedgeList hl{hla, hln};
    const int ghl = grid_for(nhl * 32, 256);

    // S9
    prof.reset(new ProfScope(h, PS_REPLAY));
    int64_t *gp, *G;
    int32_t *dv, *nviol;
    SNN_TRY(ar.alloc(&gp, M));
    SNN_TRY(ar.alloc(&G, M));
    SNN_TRY(ar.alloc(&dv, M));
    SNN_TRY(ar.alloc(&nviol, M));
    SNN_CUDA(cudaMemsetAsync(gp, 0, (size_t)M * 8, s));
    SNN_CUDA(cudaMemsetAsync(dv, 0, (size_t)M * 4, s));
    Events ev;
    ev.cap = 2 * (int64_t)M + 2 * deg;
    ev.ibits = bits_for((uint64_t)M);
    SNN_TRY(ar.alloc(&ev.key, ev.cap));
    SNN_TRY(ar.alloc(&ev.idx, ev.cap));
    SNN_TRY(ar.alloc(&ev.dsize, ev.cap));
    SNN_TRY(ar.alloc(&ev.dinp, ev.cap));
    SNN_TRY(ar.alloc(&ev.dpc, ev.cap));
    SNN_L k_size_events<<<gm, 256, 0, s>>>(M, mv, L, ev);
    SNN_CUDA(cudaGetLastError());
    uint32_t* mvbuf;
    int32_t *hv, *hvc;
    SNN_TRY(ar.alloc(&mvbuf, L.P));
    SNN_TRY(ar.alloc(&hv, L.E));
    SNN_TRY(ar.alloc(&hvc, L.E));
    if (L.E > 0) {
        SNN_L k_replay_warp<<<ghl, 256, 0, s>>>(L, pc, moveidx, mv, mvbuf, gp, ev, 2 * (int64_t)M, hv,
                                                hvc, h->d_scal, hl);
        SNN_CUDA(cudaGetLastError());
        SNN_L k_replay_block<<<152 * 2, 256, 0, s>>>(L, pc, mv, mvbuf, gp, ev, 2 * (int64_t)M, hv, hvc,
                                               h->d_scal);
        SNN_CUDA(cudaGetLastError());
    }
    prof.reset();
    SNN_TRY(read_scalars(h));
    if (h->h_scal[SC_STATUS] & ST_CAPACITY) return Status{SNNMAP_ERR_CUDA, "event buffer overflow"};
    int64_t T = 2 * (int64_t)M + h->h_scal[RS_NEV];

    // S10
    prof.reset(new ProfScope(h, PS_VALIDITY));
    uint64_t* ekey2;
    uint32_t* eidx2;
    SNN_TRY(ar.alloc(&ekey2, T));
    SNN_TRY(ar.alloc(&eidx2, T));
    int kbits = bits_for((uint64_t)K);
    SNN_TRY(radix_sort_pairs(ev.key, ev.idx, ekey2, eidx2, T, ev.ibits + kbits, ar, s));
    int32_t *pbeg, *pend;
    SNN_TRY(ar.alloc(&pbeg, K));
    SNN_TRY(ar.alloc(&pend, K));
    SNN_CUDA(cudaMemsetAsync(pbeg, 0, (size_t)K * 4, s));
    SNN_CUDA(cudaMemsetAsync(pend, 0, (size_t)K * 4, s));
    SNN_L k_part_bounds<<<grid_for(T, 256), 256, 0, s>>>(T, ev.key, ev.ibits, pbeg, pend);
    SNN_CUDA(cudaGetLastError());
    SNN_L k_part_validity<<<grid_for((int64_t)K * 32, 256), 256, 0, s>>>(K, pbeg, pend, ev, ps, prm.omega,
                                                                  prm.delta, prm.phi, dv);
    SNN_CUDA(cudaGetLastError());

    // S11
    prof.reset(new ProfScope(h, PS_APPLY));
    SNN_TRY(scan_inclusive_i64(gp, G, M, ar, s));
    SNN_TRY(scan_inclusive_i32(dv, nviol, M, ar, s));
    SNN_L k_best1<<<gm, 256, 0, s>>>(M, G, nviol, h->d_scal);
    SNN_L k_best2<<<gm, 256, 0, s>>>(M, G, nviol, h->d_scal);
    if (dense && L.E > 0) {
        prof.reset(new ProfScope(h, PS_CROSS));
        SNN_L k_dense_cross<<<ghl, 256, 0, s>>>(L, pc, moveidx, mv, h->d_scal, D.rowid, D.C, D.O,
                                                D.M, D.cw, D.Kp, mvbuf, hl);
        prof.reset(new ProfScope(h, PS_APPLY));
    }
    if (dense) {
        // P* of the enacted prefix; k_ps_rows below decides the next round's
        // proposals from the rows
        SNN_CUDA(cudaMemsetAsync(inc.dirty, 0, (size_t)(V > 0 ? V : 1) * 4, s));
        SNN_L k_ps_slots<<<gm, 256, 0, s>>>(M, mv, h->d_scal, inc.pst, inc.dirty);
        SNN_CUDA(cudaGetLastError());
        if (inc.pst.save0 && V > 0)
            SNN_CUDA(cudaMemcpyAsync(inc.pst.save0, savev, (size_t)V * 8, cudaMemcpyDeviceToDevice, s));
    } else {
        // vertices the enacted prefix can affect, for the next round
        SNN_CUDA(cudaMemsetAsync(inc.dirty, 0, (size_t)(V > 0 ? V : 1) * 4, s));
        SNN_CUDA(cudaMemsetAsync(inc.pchg, 0, (size_t)(K > 0 ? K : 1), s));
        SNN_CUDA(cudaMemsetAsync(inc.prel, 0, (size_t)(K > 0 ? K : 1), s));
        // P* of the enacted prefix; when it is short the column update after
        // the pin counts below decides the next round's proposals, otherwise
        // the flags of the three rules below do
        SNN_L k_ps_slots<<<gm, 256, 0, s>>>(M, mv, h->d_scal, inc.pst, inc.dirty);
        SNN_L k_inc_parts<<<gm, 256, 0, s>>>(M, mv, h->d_scal, ps, inc.vmax, prm.omega, prm.delta,
                                             prm.phi, inc.pchg, inc.prel, inc.pst.cnt);
        if (L.E > 0)
            SNN_L k_inc_hedges<<<grid_for((int64_t)L.E * 32, 256), 256, 0, s>>>(
                L, pc, moveidx, mv, h->d_scal, inc.prel, mvbuf, inc.dirty, inc.pst.cnt);
        SNN_L k_inc_targets<<<gv, 256, 0, s>>>(V, pto, inc.pchg, inc.dirty, inc.pst.cnt);
        SNN_CUDA(cudaGetLastError());
        if (inc.pst.save0 && V > 0)
            SNN_CUDA(cudaMemcpyAsync(inc.pst.save0, savev, (size_t)V * 8, cudaMemcpyDeviceToDevice, s));
    }
    // carried pin counts: take out the hyperedges the prefix touches (old
    // counts, old rho), move, count them again, add them back
    prof.reset(new ProfScope(h, PS_PINCOUNT));
    if (L.E > 0) {
        SNN_L k_pc_mark<<<ghl, 256, 0, s>>>(L, moveidx, h->d_scal, inc.hdirty, hl);
        SNN_L k_pc_contrib<<<ghl, 256, 0, s>>>(L, pc, inc.hdirty, rho, ps, savev, inc.costv, -1, hl);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_L k_ps_moves<<<gm, 256, 0, s>>>(M, mv, L, h->d_scal, ps);
    SNN_L k_apply<<<gm, 256, 0, s>>>(M, mv, rho, moveidx, h->d_scal);
    SNN_CUDA(cudaGetLastError());
    if (L.E > 0) {
        SNN_CUDA(cudaMemsetAsync(inc.hmeta, 0, 2 * SEG_NB * sizeof(int32_t), s));
        SNN_L k_seg_meta_copy<<<1, 32, 0, s>>>(X.seg.meta, inc.hmeta);
        SNN_L k_seg_filter<<<grid_for(L.E, 256), 256, 0, s>>>(X.seg.list, X.seg.meta, L.E, inc.hdirty,
                                                             inc.hlist, inc.hmeta);
        SNN_CUDA(cudaGetLastError());
        SegBuckets db = X.seg;
        db.list = inc.hlist;
        db.meta = inc.hmeta;
        int64_t* slots;
        SNN_TRY(ar.alloc(&slots, COST_SLOTS));
        SNN_CUDA(cudaMemsetAsync(slots, 0, COST_SLOTS * sizeof(int64_t), s));
        PinCountJob job{L.hoff, L.hpins, L.hsd, L.hk, L.hw, rho, pc, ps.pincnt, slots};
        SNN_TRY(seg_run(job, db, L.E, ar, s));
        SNN_L k_cost_slots<<<1, 256, 0, s>>>(slots, inc.costv);
        SNN_L k_pc_contrib<<<ghl, 256, 0, s>>>(L, pc, inc.hdirty, rho, ps, savev, inc.costv, 1, hl);
        SNN_L k_hedges_clear<<<grid_for(nhl, 256), 256, 0, s>>>(hl, inc.hmark, inc.hdirty);
        SNN_CUDA(cudaGetLastError());
    }
    if (!dense) {
        prof.reset(new ProfScope(h, PS_GAINS));
        if (inc.pst.colc && V > 0) {
            SNN_L k_ps_mark<<<grid_for(V, 256), 256, 0, s>>>(L, rho, h->d_scal, inc.pst);
            SNN_L k_ps_cols<<<152 * 8, 256, 0, s>>>(L, pc, rho, h->d_scal, inc.pst);
            SNN_L k_ps_combine<<<gv, 256, 0, s>>>(L, rho, h->d_scal, inc.pst, ps, savev, Wv, prm.omega,
                                                  prm.delta, prm.phi, prm.refine_nonpositive, pto,
                                                  pgain, inc.dirty);
        }
        SNN_L k_ps_reset<<<gm, 256, 0, s>>>(M, mv, h->d_scal, inc.pst);
        SNN_CUDA(cudaGetLastError());
    } else {
        prof.reset(new ProfScope(h, PS_GAINS));
        if (V > 0)
            SNN_L k_ps_rows<<<gv, 256, 0, s>>>(L, rho, h->d_scal, inc.pst, ps, savev, Wv, D.rowid, D.C,
                                               D.O, D.Kp, prm.omega, prm.delta, prm.phi,
                                               prm.refine_nonpositive, pto, pgain, inc.dirty);
        SNN_L k_ps_reset<<<gm, 256, 0, s>>>(M, mv, h->d_scal, inc.pst);
        SNN_CUDA(cudaGetLastError());
    }
    prof.reset();
    SNN_TRY(read_scalars(h));
    int64_t best = h->h_scal[RS_BEST];
    int64_t istar = h->h_scal[RS_ISTAR];
    if (best > 0 && istar < M) {
        *applied = (int32_t)(istar + 1);
        *gain = best;
    }
    return Status{};
}

__global__ void k_check_rho(int32_t V, const int32_t* __restrict__ rho, int32_t K, int64_t* scal)
{
    int bad = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        if (rho[n] < 0 || rho[n] >= K) bad = 1;
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicOr((int*)&scal[SC_STATUS], ST_INVALID);
}

Status check_rho(snnmap_hgraph* h, int32_t level, int32_t K, const int32_t* rho)
{
    Level& L = h->levels[level];
    SNN_TRY(zero_scalars(h));
    if (L.V > 0) {
        SNN_L k_check_rho<<<grid_for(L.V, 256), 256, 0, h->stream>>>(L.V, rho, K, h->d_scal);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_TRY(read_scalars(h));
    if (h->h_scal[SC_STATUS] & ST_INVALID) return Status{SNNMAP_ERR_INVALID, "rho value outside [0, n_parts)"};
    return Status{};
}

// Proposals carried to the next finer level: an unmatched vertex keeps its
// super-node's proposal, gain and flag (its conn, overlap, save, W and the
// partition state are unchanged by projection); both members of a pair are
// evaluated.
__global__ void k_carry_count(int32_t V, const int32_t* __restrict__ cid, int32_t* mcount)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&mcount[cid[n]], 1);
}

__global__ void k_carry(int32_t V, const int32_t* __restrict__ cid, const int32_t* __restrict__ mcount,
                        const int32_t* __restrict__ pto_c, const int64_t* __restrict__ pgain_c,
                        const int32_t* __restrict__ dirty_c, int32_t* pto, int64_t* pgain,
                        int32_t* dirty)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = cid[n];
        pto[n] = pto_c[c];
        pgain[n] = pgain_c[c];
        dirty[n] = (mcount[c] > 1 || dirty_c[c]) ? 1 : 0;
    }
}

Status carry_open(snnmap_hgraph* h, int64_t cap)
{
    carry_close(h);
    Carry& C = h->carry;
    size_t n = (size_t)(cap > 0 ? cap : 1);
    for (int b = 0; b < 2; b++) {
        SNN_CUDA(dev_malloc(&C.pto[b], n * 4, h->stream));
        SNN_CUDA(dev_malloc(&C.pgain[b], n * 8, h->stream));
        SNN_CUDA(dev_malloc(&C.dirty[b], n * 4, h->stream));
    }
    C.cap = cap;
    C.level = -1;
    C.cur = 0;
    return Status{};
}

void carry_close(snnmap_hgraph* h)
{
    Carry& C = h->carry;
    for (int b = 0; b < 2; b++)
        for (void* p : {(void*)C.pto[b], (void*)C.pgain[b], (void*)C.dirty[b]})
            if (p) cudaFreeAsync(p, h->stream);
    C = Carry{};
}

Status refine_level(snnmap_hgraph* h, int32_t level, int32_t K, int32_t* rho, int64_t* cost,
                    int64_t* cost_start)
{
    Level& L = h->levels[level];
    cudaStream_t s = h->stream;
    size_t nv = (size_t)(L.V > 0 ? L.V : 1), nk = (size_t)(K > 0 ? K : 1);
    int32_t* moveidx;
    IncState inc;
    Carry& CA = h->carry;
    const bool dense_level = h->dense.C && h->dense.level == level;
    const bool use_carry = CA.pto[0] && L.V <= CA.cap;
    bool inherited = false;
    SNN_CUDA(dev_malloc(&moveidx, nv * sizeof(int32_t), s));
    if (use_carry) {
        int nb = 1 - CA.cur;
        inc.pto = CA.pto[nb];
        inc.pgain = CA.pgain[nb];
        inc.dirty = CA.dirty[nb];
        if (!dense_level && CA.level == level + 1 && L.V > 0) {
            const Level& Lc = h->levels[level + 1];
            int32_t* mcount;
            SNN_TRY(h->scratch.alloc(&mcount, Lc.V));
            SNN_CUDA(cudaMemsetAsync(mcount, 0, (size_t)(Lc.V > 0 ? Lc.V : 1) * 4, s));
            SNN_L k_carry_count<<<grid_for(L.V, 256), 256, 0, s>>>(L.V, L.cid, mcount);
            SNN_L k_carry<<<grid_for(L.V, 256), 256, 0, s>>>(L.V, L.cid, mcount, CA.pto[CA.cur],
                                                            CA.pgain[CA.cur], CA.dirty[CA.cur],
                                                            inc.pto, inc.pgain, inc.dirty);
            SNN_CUDA(cudaGetLastError());
            inherited = true;
        }
        CA.cur = nb;
        CA.level = -1;
    } else {
        SNN_CUDA(dev_malloc(&inc.pto, nv * 4, s));
        SNN_CUDA(dev_malloc(&inc.pgain, nv * 8, s));
        SNN_CUDA(dev_malloc(&inc.dirty, nv * 4, s));
    }
    SNN_CUDA(dev_malloc(&inc.pchg, nk, s));
    SNN_CUDA(dev_malloc(&inc.prel, nk, s));
    SNN_CUDA(dev_malloc(&inc.vmax, 3 * 4, s));
    size_t np = (size_t)(L.P > 0 ? L.P : 1), ne = (size_t)(L.E > 0 ? L.E : 1);
    SNN_CUDA(dev_malloc(&inc.pc.p, np * 4, s));
    SNN_CUDA(dev_malloc(&inc.pc.cnt, np * 4, s));
    SNN_CUDA(dev_malloc(&inc.pc.dcnt, np * 4, s));
    SNN_CUDA(dev_malloc(&inc.pc.lam, ne * 4, s));
    SNN_CUDA(dev_malloc(&inc.ps.size, nk * 8, s));
    SNN_CUDA(dev_malloc(&inc.ps.inpins, nk * 8, s));
    SNN_CUDA(dev_malloc(&inc.ps.pincnt, nk * 8, s));
    SNN_CUDA(dev_malloc(&inc.costv, 8, s));
    SNN_CUDA(dev_malloc(&inc.savev, nv * 8, s));
    SNN_CUDA(dev_malloc(&inc.Wv, nv * 8, s));
    SNN_CUDA(dev_malloc(&inc.hdirty, ne * 4, s));
    SNN_CUDA(dev_malloc(&inc.hmark, ne * 4, s));
    SNN_CUDA(cudaMemsetAsync(inc.hdirty, 0, ne * 4, s));
    SNN_CUDA(cudaMemsetAsync(inc.hmark, 0, ne * 4, s));
    SNN_CUDA(dev_malloc(&inc.hlist, ne * 4, s));
    SNN_CUDA(dev_malloc(&inc.hmeta, 2 * SEG_NB * 4, s));
    PStar& pst = inc.pst;
    SNN_CUDA(dev_malloc(&pst.pslot, nk * 4, s));
    SNN_CUDA(dev_malloc(&pst.slots, PSTAR_MAX * 4, s));
    SNN_CUDA(dev_malloc(&pst.cnt, 4 * 4, s));
    if (dense_level) {
        // rows levels need only the round-start saves besides the slot map
        if (dev_malloc(&pst.save0, nv * 8, s) != cudaSuccess) {
            cudaGetLastError();
            pst.save0 = nullptr;
        }
    } else {
        // the column buffers are optional: without them every round takes
        // the flag rules
        size_t cols = (size_t)PSTAR_MAX * nv;
        bool ok = dev_malloc(&pst.hmask, ne * 4, s) == cudaSuccess &&
                  dev_malloc(&pst.hl, ne * 4, s) == cudaSuccess &&
                  dev_malloc(&pst.colc, cols * 8, s) == cudaSuccess &&
                  dev_malloc(&pst.colo, cols * 4, s) == cudaSuccess &&
                  dev_malloc(&pst.vt, nv * 4, s) == cudaSuccess &&
                  dev_malloc(&pst.save0, nv * 8, s) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            for (void* p : {(void*)pst.hmask, (void*)pst.hl, (void*)pst.colc, (void*)pst.colo,
                            (void*)pst.vt, (void*)pst.save0})
                if (p) cudaFreeAsync(p, s);
            pst.hmask = nullptr;
            pst.hl = nullptr;
            pst.colc = nullptr;
            pst.colo = nullptr;
            pst.vt = nullptr;
            pst.save0 = nullptr;
        } else {
            SNN_CUDA(cudaMemsetAsync(pst.hmask, 0, ne * 4, s));
            SNN_CUDA(cudaMemsetAsync(pst.colc, 0, cols * 8, s));
            SNN_CUDA(cudaMemsetAsync(pst.colo, 0, cols * 4, s));
            SNN_CUDA(cudaMemsetAsync(pst.vt, 0, nv * 4, s));
        }
    }
    {
        int32_t base = (pst.colc || (dense_level && pst.save0)) ? 0 : (1 << 30);
        int32_t hc[4] = {base, 0, base, 0};
        SNN_CUDA(cudaMemcpyAsync(pst.cnt, hc, sizeof(hc), cudaMemcpyHostToDevice, s));
        SNN_TRY(fill_i32(pst.pslot, -1, nk, s));
    }
    SNN_CUDA(cudaMemsetAsync(inc.vmax, 0, 3 * 4, s));
    if (L.V > 0) SNN_L k_level_max<<<grid_for(L.V, 256), 256, 0, s>>>(L, inc.vmax);
    SNN_CUDA(cudaGetLastError());
    Status st = fill_i32(moveidx, -1, L.V, s);
    if (st.ok() && !inherited) st = fill_i32(inc.dirty, 1, L.V, s);
    int64_t c = 0;
    bool have_cost = false;
    for (int32_t r = 0; st.ok() && r < h->prm.max_refine_rounds; r++) {
        int32_t props = 0, applied = 0, act = 0, rows = 0;
        int64_t g = 0, c0 = 0;
        st = refine_round(h, level, K, rho, moveidx, inc, &props, &applied, &g, &c0, &act, &rows);
        inc.ready = true;
        h->scratch.reset();
        if (!st.ok()) break;
        h->rlog.push_back(snnmap_round_log{level, r, props, applied, act, rows, g});
        if (!have_cost && cost_start) *cost_start = c0;
        c = c0 - g;
        have_cost = true;
        if (applied == 0) break;
    }
    cudaFreeAsync(moveidx, s);
    if (!use_carry)
        for (void* p : {(void*)inc.pto, (void*)inc.pgain, (void*)inc.dirty}) cudaFreeAsync(p, s);
    else if (st.ok() && !dense_level)
        CA.level = level;   // the next finer level may inherit these proposals
    for (void* p : {(void*)inc.pchg,
                    (void*)inc.prel, (void*)inc.vmax, (void*)inc.pc.p, (void*)inc.pc.cnt,
                    (void*)inc.pc.dcnt, (void*)inc.pc.lam, (void*)inc.ps.size,
                    (void*)inc.ps.inpins, (void*)inc.ps.pincnt, (void*)inc.costv,
                    (void*)inc.savev, (void*)inc.Wv, (void*)inc.hdirty, (void*)inc.hmark,
                    (void*)inc.hlist,
                    (void*)inc.hmeta, (void*)pst.pslot, (void*)pst.slots, (void*)pst.cnt,
                    (void*)pst.hmask, (void*)pst.hl, (void*)pst.colc, (void*)pst.colo,
                    (void*)pst.vt, (void*)pst.save0})
        if (p) cudaFreeAsync(p, s);
    if (!st.ok()) return st;
    if (!have_cost) {
        SNN_TRY(level_cost(h, level, K, rho, &c));
        if (cost_start) *cost_start = c;
    }
    *cost = c;
    return Status{};
}

}  // namespace snn
