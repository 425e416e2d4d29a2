// Initial placement of the partition hypergraph G_P (Sec. 4.2, "Initial
// Placement"; snnmap_place_initial and snnmap_hilbert_order in
// include/snnmap.h), for many starts at once.
//
// The bisection tree depends only on the number of nodes, so it is built
// once (breadth-first, the host's bookkeeping of interval bounds) and
// shared by every start. Sections of one depth are disjoint, so the label
// propagation of every sibling pair of a depth, in every start, runs as one
// set of jobs; each job stops on its own. At the start of a depth:
//   k_ip_gain     one thread per position: the single-move cut drop G of
//                 the node there (counts of its hyperedges on each side)
//   k_ip_corr     one thread per L position: its row of the job's nL x nR
//                 correction matrix (the thread is the row's only writer)
// Then one round of all active jobs:
//   k_ip_best_*   one thread per (x, y) pair: the steepest swap, ties to
//                 the lowest x then y, in three passes of integer atomics
//   k_ip_update   one block per job: stop, or swap and bring G and the
//                 matrix up to date through the hyperedges of x and y only
//                 (G deltas, weight changes of pairs of non-moving pins,
//                 and the rebuilt row and column of the two moved nodes)
// Folding reads only the node sets of the sections, fixed once the label
// propagation is done: k_ip_conn sums each child's connection to its
// parent's sibling, k_ip_flip decides each orientation, and k_ip_fold gives
// every node its final position by one descent of the tree. Nodes then take
// the cores in Hilbert order (k_ip_hkeys and a radix sort).
#include "internal.cuh"
#include "initial_items.cuh"

#include <climits>
#include <new>
#include <vector>

namespace {

using namespace snn;
namespace ip = snn::initial;

constexpr int kMaxStarts = 65535;   // gridDim.y

// a pin repeated within its hyperedge; degrees of the nodes
__global__ void k_ip_distinct(int64_t P, const int64_t* __restrict__ off,
                              const int32_t* __restrict__ pins, const int32_t* __restrict__ hid,
                              int32_t* deg, int32_t* err)
{
    int bad = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t q = pins[j];
        int64_t e = off[hid[j] + 1];
        for (int64_t t = j + 1; t < e; t++)
            if (pins[t] == q) bad = 1;
        atomicAdd(&deg[q], 1);
    }
    if (bad) atomicOr(err, 2);
}

// incidence lists: vinc[voff[q] ..] the hyperedges of node q (any order)
__global__ void k_ip_fill(int64_t P, const int32_t* __restrict__ pins,
                          const int32_t* __restrict__ hid, const int64_t* __restrict__ voff,
                          int32_t* cursor, int32_t* vinc)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t q = pins[j];
        vinc[voff[q] + atomicAdd(&cursor[q], 1)] = hid[j];
    }
}

// seq and pos of every start from the initial orders; an order that is not
// a permutation of the nodes is an error (pos filled with -1 before)
__global__ void k_ip_seq(int32_t np, const int32_t* __restrict__ seq0, int32_t* seq, int32_t* pos,
                         int32_t* err)
{
    int64_t s = blockIdx.y;
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t q = seq0[s * np + i];
        seq[s * np + i] = q;
        if (q < 0 || q >= np) bad = 1;
        else if (atomicCAS(&pos[s * np + q], -1, (int32_t)i) != -1) bad = 1;
    }
    if (bad) atomicOr(err, 4);
}

// job of every position at one depth (-1: a section that does not split)
__global__ void k_ip_jobof(int32_t J, const int32_t* __restrict__ jlo, const int32_t* __restrict__ jhi,
                           int32_t* jobof)
{
    for (int32_t k = blockIdx.x; k < J; k += gridDim.x)
        for (int32_t i = jlo[k] + threadIdx.x; i < jhi[k]; i += blockDim.x) jobof[i] = k;
}

struct Jobs {
    int32_t J;
    const int32_t *lo, *mid, *hi, *cap, *jobof;
    const int64_t* pairoff;
};

__global__ void k_ip_reset(int32_t S, int32_t J, const int32_t* __restrict__ done, int64_t* bd,
                           int32_t* bx, int32_t* by)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)S * J;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (done[t]) continue;
        bd[t] = 0;
        bx[t] = INT32_MAX;
        by[t] = INT32_MAX;
    }
}

__global__ void k_ip_gain(int32_t np, Jobs jb, const int32_t* __restrict__ done,
                          const int64_t* __restrict__ voff, const int32_t* __restrict__ vinc,
                          const int64_t* __restrict__ off, const int32_t* __restrict__ pins,
                          const int64_t* __restrict__ eta, const int32_t* __restrict__ seq,
                          const int32_t* __restrict__ pos, int64_t* G)
{
    int64_t s = blockIdx.y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t k = jb.jobof[i];
        if (k < 0 || done[s * jb.J + k]) continue;
        int32_t x = seq[s * np + i];
        int sd = ip::side_of((int32_t)i, jb.lo[k], jb.mid[k], jb.hi[k]);
        G[s * np + x] = ip::single_gain(vinc, voff[x], voff[x + 1], off, pins, eta, pos + s * np, sd,
                                        jb.lo[k], jb.mid[k], jb.hi[k]);
    }
}

struct RowAdd {
    int64_t* row;
    __device__ void operator()(int32_t j, int64_t w) const { row[j] += w; }
};

__global__ void k_ip_corr(int32_t np, int64_t pairs, Jobs jb, const int32_t* __restrict__ done,
                          const int64_t* __restrict__ voff, const int32_t* __restrict__ vinc,
                          const int64_t* __restrict__ off, const int32_t* __restrict__ pins,
                          const int64_t* __restrict__ eta, const int32_t* __restrict__ seq,
                          const int32_t* __restrict__ pos, int64_t* M)
{
    int64_t s = blockIdx.y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t k = jb.jobof[i];
        if (k < 0 || done[s * jb.J + k] || i >= jb.mid[k]) continue;
        int32_t x = seq[s * np + i];
        int32_t nr = jb.hi[k] - jb.mid[k];
        RowAdd add{M + s * pairs + jb.pairoff[k] + (i - jb.lo[k]) * (int64_t)nr};
        ip::corr_row(vinc, voff[x], voff[x + 1], off, pins, eta, pos + s * np, jb.lo[k], jb.mid[k],
                     jb.hi[k], add);
    }
}

// pair p of a depth's jobs: its job (binary search in pairoff) and nodes
__device__ __forceinline__ int32_t job_of_pair(const Jobs& jb, int64_t p)
{
    int32_t a = 0, b = jb.J - 1;
    while (a < b) {
        int32_t m = (a + b + 1) >> 1;
        if (jb.pairoff[m] <= p) a = m;
        else b = m - 1;
    }
    return a;
}

template <int PASS>
__global__ void k_ip_best(int32_t np, int64_t pairs, Jobs jb, const int32_t* __restrict__ done,
                          const int32_t* __restrict__ seq, const int64_t* __restrict__ G,
                          const int64_t* __restrict__ M, int64_t* bd, int32_t* bx, int32_t* by)
{
    int64_t s = blockIdx.y;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t k = job_of_pair(jb, p);
        int64_t t = s * jb.J + k;
        if (done[t]) continue;
        int64_t q = p - jb.pairoff[k];
        int32_t nr = jb.hi[k] - jb.mid[k];
        int32_t x = seq[s * np + jb.lo[k] + (int32_t)(q / nr)];
        int32_t y = seq[s * np + jb.mid[k] + (int32_t)(q % nr)];
        int64_t d = G[s * np + x] + G[s * np + y] - M[s * pairs + p];
        if (d <= 0) continue;
        if (PASS == 0) atomicMax((long long*)&bd[t], (long long)d);
        else if (PASS == 1) {
            if (d == bd[t]) atomicMin(&bx[t], x);
        } else {
            if (d == bd[t] && x == bx[t]) atomicMin(&by[t], y);
        }
    }
}

struct GAddAtomic {
    int64_t* G;
    __device__ void operator()(int32_t v, int64_t d) const
    {
        atomicAdd((unsigned long long*)&G[v], (unsigned long long)d);
    }
};

struct MAddAtomic {
    int64_t* M;
    int32_t nr;
    __device__ void operator()(int32_t i, int32_t j, int64_t d) const
    {
        atomicAdd((unsigned long long*)&M[(int64_t)i * nr + j], (unsigned long long)d);
    }
};

struct RowAddAtomic {
    int64_t* row;
    __device__ void operator()(int32_t j, int64_t w) const
    {
        atomicAdd((unsigned long long*)&row[j], (unsigned long long)w);
    }
};

struct ColAddAtomic {
    int64_t* col;
    int32_t nr;
    __device__ void operator()(int32_t i, int64_t w) const
    {
        atomicAdd((unsigned long long*)&col[(int64_t)i * nr], (unsigned long long)w);
    }
};

// One block per (job, start): stop when no swap lowers the cut, else swap
// x and y and update G and the job's matrix incrementally.
__global__ void k_ip_update(int32_t np, int64_t pairs, Jobs jb, int32_t* done, int32_t* it,
                            const int64_t* __restrict__ bd, const int32_t* __restrict__ bx,
                            const int32_t* __restrict__ by, const int64_t* __restrict__ voff,
                            const int32_t* __restrict__ vinc, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ pins, const int64_t* __restrict__ eta,
                            int32_t* seq, int32_t* pos, int64_t* G, int64_t* M, int32_t* active)
{
    __shared__ int s_mode;   // 0 skip, 1 swap then stop, 2 swap and go on
    const int64_t s = blockIdx.y;
    const int32_t k = blockIdx.x;
    const int64_t t = s * jb.J + k;
    if (threadIdx.x == 0) {
        int mode = 0;
        if (!done[t]) {
            if (bd[t] <= 0) done[t] = 1;
            else mode = it[t] + 1 >= jb.cap[k] ? 1 : 2;
        }
        s_mode = mode;
    }
    __syncthreads();
    const int mode = s_mode;
    if (mode == 0) return;
    const int32_t lo = jb.lo[k], mid = jb.mid[k], hi = jb.hi[k], nr = hi - mid;
    const int32_t x = bx[t], y = by[t];
    int32_t* ps = pos + s * np;
    int64_t* Gs = G + s * np;
    int64_t* Mk = M + s * pairs + jb.pairoff[k];
    const int32_t px = ps[x], py = ps[y];
    if (mode == 2) {
        // hyperedges of x, then those of y not holding x, before the swap
        const int64_t nx = voff[x + 1] - voff[x], ny = voff[y + 1] - voff[y];
        GAddAtomic gadd{Gs};
        MAddAtomic madd{Mk, nr};
        for (int64_t u = threadIdx.x; u < nx + ny; u += blockDim.x) {
            bool from_y = u >= nx;
            int32_t a = from_y ? vinc[voff[y] + (u - nx)] : vinc[voff[x] + u];
            ip::swap_hedge_update(pins, off[a], off[a + 1], ps, lo, mid, hi, x, y, eta[a], from_y,
                                  gadd, madd);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t* qs = seq + s * np;
        qs[px] = y;
        qs[py] = x;
        ps[x] = py;
        ps[y] = px;
        it[t] += 1;
        if (mode == 1) done[t] = 1;
        else atomicAdd(active, 1);
    }
    if (mode == 1) return;
    __syncthreads();
    // the moved nodes' row (y now at px in L) and column (x now at py in R)
    int64_t* row = Mk + (int64_t)(px - lo) * nr;
    int64_t* col = Mk + (py - mid);
    for (int32_t j = threadIdx.x; j < nr; j += blockDim.x) row[j] = 0;
    for (int32_t i = threadIdx.x; i < mid - lo; i += blockDim.x) col[(int64_t)i * nr] = 0;
    __syncthreads();
    const int64_t nyi = voff[y + 1] - voff[y], nxi = voff[x + 1] - voff[x];
    for (int64_t u = threadIdx.x; u < nyi + nxi; u += blockDim.x) {
        if (u < nyi) {
            ip::corr_row(vinc, voff[y] + u, voff[y] + u + 1, off, pins, eta, ps, lo, mid, hi,
                         RowAddAtomic{row});
        } else {
            int64_t v = voff[x] + (u - nyi);
            ip::corr_col(vinc, v, v + 1, off, pins, eta, ps, lo, mid, hi, y, ColAddAtomic{col, nr});
        }
    }
}

struct Tree {
    const int32_t *lo, *hi, *par, *kid;
    int32_t nn;
};

// conn[c]: summed eta of hyperedges with pins in section c and in the
// sibling of c's parent, for every section c two or more levels deep
__global__ void k_ip_conn(int64_t P, int32_t np, Tree T, const int32_t* __restrict__ hid,
                          const int64_t* __restrict__ off, const int32_t* __restrict__ pins,
                          const int64_t* __restrict__ eta, const int32_t* __restrict__ pos,
                          int64_t* conn)
{
    int64_t s = blockIdx.y;
    const int32_t* ps = pos + s * np;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = hid[j];
        int32_t i = ps[pins[j]];
        int32_t cur = 0;
        while (T.kid[cur] >= 0) {
            int32_t c = ip::child_holding(T.lo, T.hi, T.kid, cur, i);
            int32_t p = T.par[cur];
            if (p >= 0) {
                int32_t sib = T.kid[p] == cur ? T.kid[p] + 1 : T.kid[p];
                bool first, meets;
                ip::fold_checks(pins, off[a], off[a + 1], ps, j, T.lo[c], T.hi[c], T.lo[sib],
                                T.hi[sib], &first, &meets);
                if (first && meets)
                    atomicAdd((unsigned long long*)&conn[s * T.nn + c], (unsigned long long)eta[a]);
            }
            cur = c;
        }
    }
}

// orientation of every section: a split section with a sibling is reversed
// when its child more connected to the sibling does not face it
__global__ void k_ip_flip(Tree T, const int64_t* __restrict__ conn, uint8_t* flip)
{
    int64_t s = blockIdx.y;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < T.nn; v += gridDim.x * blockDim.x) {
        uint8_t f = 0;
        int32_t p = T.par[v];
        if (T.kid[v] >= 0 && p >= 0) {
            int64_t ca = conn[s * T.nn + T.kid[v]], cb = conn[s * T.nn + T.kid[v] + 1];
            bool left = T.kid[p] == v;   // the sibling lies to the right
            f = left ? (ca > cb) : (cb > ca);
        }
        flip[s * T.nn + v] = f;
    }
}

__global__ void k_ip_fold(int32_t np, Tree T, const uint8_t* __restrict__ flip,
                          const int32_t* __restrict__ seq, int32_t* seq_out)
{
    int64_t s = blockIdx.y;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x)
        seq_out[s * np + ip::folded_position(T.lo, T.hi, T.kid, flip + s * T.nn, i)] =
            seq[s * np + i];
}

__global__ void k_ip_hkeys(int32_t width, int32_t nh, uint32_t n2, uint64_t* keys, uint32_t* vals)
{
    for (int32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        keys[h] = ip::hilbert_index(n2, (uint32_t)(h % width), (uint32_t)(h / width));
        vals[h] = (uint32_t)h;
    }
}

__global__ void k_ip_gamma(int32_t np, const int32_t* __restrict__ seq_out,
                           const uint32_t* __restrict__ order, int32_t* gamma)
{
    int64_t s = blockIdx.y;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x)
        gamma[s * np + seq_out[s * np + i]] = (int32_t)order[i];
}

dim3 grid2(int64_t n, int32_t S)
{
    int cap = 152 * 32 / S;
    return dim3((unsigned)grid_for(n, 256, cap > 0 ? cap : 1), (unsigned)S);
}

Status invalid(const char* msg) { return Status{SNNMAP_ERR_INVALID, msg}; }

// cores in Hilbert order into order (device uint32[nh])
Status hilbert_order(int32_t width, int32_t height, uint32_t* order, Arena& ar, cudaStream_t s)
{
    int32_t nh = width * height;
    uint32_t n2 = 1;
    while (n2 < (uint32_t)width || n2 < (uint32_t)height) n2 <<= 1;
    uint64_t *keys, *keys2;
    uint32_t* vals2;
    SNN_TRY(ar.alloc(&keys, nh));
    SNN_TRY(ar.alloc(&keys2, nh));
    SNN_TRY(ar.alloc(&vals2, nh));
    SNN_L k_ip_hkeys<<<grid_for(nh, 256), 256, 0, s>>>(width, nh, n2, keys, order);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(radix_sort_pairs(keys, order, keys2, vals2, nh, bits_for((uint64_t)n2 * n2 - 1), ar, s));
    return Status{};
}

// the bisection tree of n positions, breadth-first
struct HostTree {
    std::vector<int32_t> lo, hi, par, kid, depth;
    int32_t maxd = 0;
    explicit HostTree(int32_t n)
    {
        lo.push_back(0);
        hi.push_back(n);
        par.push_back(-1);
        kid.push_back(-1);
        depth.push_back(0);
        for (size_t v = 0; v < lo.size(); v++) {
            int32_t len = hi[v] - lo[v];
            if (len <= 1) continue;
            int32_t mid = lo[v] + (len + 1) / 2;
            kid[v] = (int32_t)lo.size();
            for (int t = 0; t < 2; t++) {
                lo.push_back(t ? mid : lo[v]);
                hi.push_back(t ? hi[v] : mid);
                par.push_back((int32_t)v);
                kid.push_back(-1);
                depth.push_back(depth[v] + 1);
                if (depth.back() > maxd) maxd = depth.back();
            }
        }
    }
};

template <typename T>
Status upload(const std::vector<T>& h, T** d, Arena& ar, cudaStream_t s)
{
    SNN_TRY(ar.alloc(d, (int64_t)h.size()));
    if (!h.empty())
        SNN_CUDA(cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
    return Status{};
}

Status initial_impl(int32_t np, int32_t ne, const int64_t* off, const int32_t* pins,
                    const int64_t* eta, int32_t width, int32_t height, int32_t S,
                    const int32_t* seq0, int32_t* seq_out_user, int32_t* gamma, cudaStream_t s)
{
    if (np < 0 || ne < 0 || width < 1 || height < 1 || S < 1 || S > kMaxStarts)
        return invalid("negative sizes, width or height < 1, or n_starts outside [1, 65535]");
    int64_t nh = (int64_t)width * height;
    if (nh >= ((int64_t)1 << 31) || (int64_t)np * S >= ((int64_t)1 << 31))
        return invalid("width * height or n_starts * n_nodes >= 2^31");
    if (np > nh) return invalid("more nodes than cores");
    if ((np > 0 && (!device_pointer(seq0) || !device_pointer(gamma))) ||
        (seq_out_user && !device_pointer(seq_out_user)))
        return invalid("buffers must be device memory");
    Arena ar;
    ar.stream = s;
    struct Guard {
        Arena& a;
        ~Guard() { a.release(); }
    } guard{ar};
    int32_t *err, *hid;
    int64_t P = 0;
    SNN_TRY(ar.alloc(&err, 1));
    SNN_TRY(gp_input(np, ne, off, pins, eta, ar, s, err, &P, &hid));
    if (np == 0) return Status{};

    int32_t *deg, *cursor, *vinc, *seq, *pos, *seq2;
    int64_t* voff;
    SNN_TRY(ar.alloc(&deg, np));
    SNN_TRY(ar.alloc(&cursor, np));
    SNN_TRY(ar.alloc(&vinc, P));
    SNN_TRY(ar.alloc(&voff, (int64_t)np + 1));
    SNN_TRY(ar.alloc(&seq, (int64_t)S * np));
    SNN_TRY(ar.alloc(&seq2, (int64_t)S * np));
    SNN_TRY(ar.alloc(&pos, (int64_t)S * np));
    SNN_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    SNN_TRY(fill_i32(pos, -1, (int64_t)S * np, s));
    SNN_L k_ip_seq<<<grid2(np, S), 256, 0, s>>>(np, seq0, seq, pos, err);
    SNN_CUDA(cudaGetLastError());
    int32_t herr = 0;
    SNN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (herr) return invalid("an initial order that is not a permutation of the nodes");
    SNN_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * np, s));
    SNN_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * np, s));
    if (P > 0) {
        SNN_L k_ip_distinct<<<grid_for(P, 256), 256, 0, s>>>(P, off, pins, hid, deg, err);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (herr) return invalid("a pin repeated within a hyperedge");
    SNN_TRY(scan_exclusive_i32_to_i64(deg, voff, np, voff + np, ar, s));
    if (P > 0) {
        SNN_L k_ip_fill<<<grid_for(P, 256), 256, 0, s>>>(P, pins, hid, voff, cursor, vinc);
        SNN_CUDA(cudaGetLastError());
    }

    // the bisection tree, shared by all starts
    HostTree ht(np);
    Tree T;
    int32_t *d_lo, *d_hi, *d_par, *d_kid;
    SNN_TRY(upload(ht.lo, &d_lo, ar, s));
    SNN_TRY(upload(ht.hi, &d_hi, ar, s));
    SNN_TRY(upload(ht.par, &d_par, ar, s));
    SNN_TRY(upload(ht.kid, &d_kid, ar, s));
    T.lo = d_lo;
    T.hi = d_hi;
    T.par = d_par;
    T.kid = d_kid;
    T.nn = (int32_t)ht.lo.size();

    // label propagation, depth by depth
    int64_t max_pairs = 0;
    int32_t max_jobs = 0;
    std::vector<std::vector<int32_t>> jobs_at(ht.maxd + 1);
    for (int32_t v = 0; v < T.nn; v++)
        if (ht.kid[v] >= 0) jobs_at[ht.depth[v]].push_back(v);
    for (auto& js : jobs_at) {
        int64_t pr = 0;
        for (int32_t v : js) {
            int32_t len = ht.hi[v] - ht.lo[v], nl = (len + 1) / 2;
            pr += (int64_t)nl * (len - nl);
        }
        if (pr > max_pairs) max_pairs = pr;
        if ((int32_t)js.size() > max_jobs) max_jobs = (int32_t)js.size();
    }
    int64_t *G, *M, *bd;
    int32_t *jobof, *done, *it, *bx, *by, *active;
    SNN_TRY(ar.alloc(&G, (int64_t)S * np));
    SNN_TRY(ar.alloc(&M, (int64_t)S * max_pairs));
    SNN_TRY(ar.alloc(&jobof, np));
    SNN_TRY(ar.alloc(&done, (int64_t)S * max_jobs));
    SNN_TRY(ar.alloc(&it, (int64_t)S * max_jobs));
    SNN_TRY(ar.alloc(&bd, (int64_t)S * max_jobs));
    SNN_TRY(ar.alloc(&bx, (int64_t)S * max_jobs));
    SNN_TRY(ar.alloc(&by, (int64_t)S * max_jobs));
    SNN_TRY(ar.alloc(&active, 1));
    const dim3 gpos = grid2(np, S);
    for (int32_t d = 0; d <= ht.maxd; d++) {
        const std::vector<int32_t>& js = jobs_at[d];
        if (js.empty()) continue;
        Arena::Mark mk = ar.mark();
        int32_t J = (int32_t)js.size();
        std::vector<int32_t> hlo(J), hmid(J), hhi(J), hcap(J);
        std::vector<int64_t> hpo(J + 1, 0);
        for (int32_t k = 0; k < J; k++) {
            int32_t v = js[k], len = ht.hi[v] - ht.lo[v], nl = (len + 1) / 2, nr = len - nl;
            hlo[k] = ht.lo[v];
            hmid[k] = ht.lo[v] + nl;
            hhi[k] = ht.hi[v];
            hcap[k] = 4 * (nl < nr ? nl : nr);
            hpo[k + 1] = hpo[k] + (int64_t)nl * nr;
        }
        const int64_t pairs = hpo[J];
        Jobs jb;
        int32_t *jlo, *jmid, *jhi, *jcap;
        int64_t* jpo;
        SNN_TRY(upload(hlo, &jlo, ar, s));
        SNN_TRY(upload(hmid, &jmid, ar, s));
        SNN_TRY(upload(hhi, &jhi, ar, s));
        SNN_TRY(upload(hcap, &jcap, ar, s));
        SNN_TRY(upload(hpo, &jpo, ar, s));
        jb.J = J;
        jb.lo = jlo;
        jb.mid = jmid;
        jb.hi = jhi;
        jb.cap = jcap;
        jb.pairoff = jpo;
        jb.jobof = jobof;
        SNN_TRY(fill_i32(jobof, -1, np, s));
        SNN_L k_ip_jobof<<<grid_for(J, 1, 152 * 8), 128, 0, s>>>(J, jlo, jhi, jobof);
        SNN_CUDA(cudaMemsetAsync(done, 0, sizeof(int32_t) * S * J, s));
        SNN_CUDA(cudaMemsetAsync(it, 0, sizeof(int32_t) * S * J, s));
        SNN_CUDA(cudaGetLastError());
        const dim3 gpair = grid2(pairs, S);
        const int gjob = grid_for((int64_t)S * J, 256);
        SNN_L k_ip_gain<<<gpos, 256, 0, s>>>(np, jb, done, voff, vinc, off, pins, eta, seq, pos, G);
        SNN_CUDA(cudaMemsetAsync(M, 0, sizeof(int64_t) * S * pairs, s));
        SNN_L k_ip_corr<<<gpos, 256, 0, s>>>(np, pairs, jb, done, voff, vinc, off, pins, eta, seq,
                                             pos, M);
        SNN_CUDA(cudaGetLastError());
        const dim3 gupd((unsigned)J, (unsigned)S);
        for (;;) {
            SNN_L k_ip_reset<<<gjob, 256, 0, s>>>(S, J, done, bd, bx, by);
            SNN_L k_ip_best<0><<<gpair, 256, 0, s>>>(np, pairs, jb, done, seq, G, M, bd, bx, by);
            SNN_L k_ip_best<1><<<gpair, 256, 0, s>>>(np, pairs, jb, done, seq, G, M, bd, bx, by);
            SNN_L k_ip_best<2><<<gpair, 256, 0, s>>>(np, pairs, jb, done, seq, G, M, bd, bx, by);
            SNN_CUDA(cudaMemsetAsync(active, 0, sizeof(int32_t), s));
            SNN_L k_ip_update<<<gupd, 128, 0, s>>>(np, pairs, jb, done, it, bd, bx, by, voff, vinc, off,
                                                   pins, eta, seq, pos, G, M, active);
            SNN_CUDA(cudaGetLastError());
            int32_t hact = 0;
            SNN_CUDA(cudaMemcpyAsync(&hact, active, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            SNN_CUDA(cudaStreamSynchronize(s));
            if (hact == 0) break;
        }
        ar.rewind(mk);
    }

    // folding, then the cores in Hilbert order
    int64_t* conn;
    uint8_t* flip;
    uint32_t* order;
    SNN_TRY(ar.alloc(&conn, (int64_t)S * T.nn));
    SNN_TRY(ar.alloc(&flip, (int64_t)S * T.nn));
    SNN_TRY(ar.alloc(&order, nh));
    SNN_CUDA(cudaMemsetAsync(conn, 0, sizeof(int64_t) * S * T.nn, s));
    if (P > 0) {
        SNN_L k_ip_conn<<<grid2(P, S), 256, 0, s>>>(P, np, T, hid, off, pins, eta, pos, conn);
    }
    SNN_L k_ip_flip<<<grid2(T.nn, S), 256, 0, s>>>(T, conn, flip);
    int32_t* seq_out = seq_out_user ? seq_out_user : seq2;
    SNN_L k_ip_fold<<<gpos, 256, 0, s>>>(np, T, flip, seq, seq_out);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(hilbert_order(width, height, order, ar, s));
    SNN_L k_ip_gamma<<<gpos, 256, 0, s>>>(np, seq_out, order, gamma);
    SNN_CUDA(cudaGetLastError());
    SNN_CUDA(cudaStreamSynchronize(s));
    return Status{};
}

int finish(const Status& st)
{
    set_last_error(st.msg);
    return st.code;
}

}  // namespace

extern "C" {

int snnmap_place_initial(int32_t n_nodes, int32_t n_hedges, const int64_t* d_offsets,
                         const int32_t* d_pins, const int64_t* d_eta, int32_t width,
                         int32_t height, int32_t n_starts, const int32_t* d_seq0,
                         int32_t* d_seq_out, int32_t* d_gamma_out, void* stream)
{
    try {
        return finish(initial_impl(n_nodes, n_hedges, d_offsets, d_pins, d_eta, width, height,
                                   n_starts, d_seq0, d_seq_out, d_gamma_out, (cudaStream_t)stream));
    } catch (const std::bad_alloc&) {
        return finish(Status{SNNMAP_ERR_OOM, "host allocation failed"});
    } catch (...) {
        return finish(Status{SNNMAP_ERR_CUDA, "internal error"});
    }
}

int snnmap_hilbert_order(int32_t width, int32_t height, int32_t* d_order_out, void* stream)
{
    try {
        if (width < 1 || height < 1 || (int64_t)width * height >= ((int64_t)1 << 31))
            return finish(invalid("width and height must be >= 1 and width * height < 2^31"));
        if (!device_pointer(d_order_out)) return finish(invalid("d_order_out must be device memory"));
        cudaStream_t s = (cudaStream_t)stream;
        Arena ar;
        ar.stream = s;
        struct Guard {
            Arena& a;
            ~Guard() { a.release(); }
        } guard{ar};
        Status st = hilbert_order(width, height, (uint32_t*)d_order_out, ar, s);
        if (st.ok()) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = Status{SNNMAP_ERR_CUDA, cudaGetErrorString(e)};
        }
        return finish(st);
    } catch (const std::bad_alloc&) {
        return finish(Status{SNNMAP_ERR_OOM, "host allocation failed"});
    } catch (...) {
        return finish(Status{SNNMAP_ERR_CUDA, "internal error"});
    }
}

}  // extern "C"
