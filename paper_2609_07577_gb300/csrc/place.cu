// Placement swap refinement and total residual distance of the partition
// hypergraph G_P on a lattice of cores (Sec. 4.2; snnmap_place_refine and
// snnmap_place_trd in include/snnmap.h).
//
// Several starts share every launch (the paper refines its Pi starts
// concurrently): start s owns cores [s*nh, (s+1)*nh) of each per-core array
// and nodes [s*np, (s+1)*np) of each per-node array, and 2-D grids carry the
// start in blockIdx.y. The starts' proposal forests never share a vertex, so
// one matching call covers all of them.
//
// One round:
//   k_pl_force    one thread per pin entry: its hyperedge's share of Eq.
//                 force of the pin's node towards the four adjacent cores,
//                 added into F with int64 atomics (exact, order-free)
//   k_pl_propose  one thread per core: Eq. tension and the core's proposal
//   match_forest  Eq. matching with tension as the score
//   k_pl_flag     one swap per matched pair, counted per start
//   k_pl_compact  the swap list (ascending core), key INT64_MAX - tension
//   radix sorts   stable by key, then stable by start: per start,
//                 decreasing tension, ties by the lower core
//   k_pl_rank     each swapping core's rank within its start, and its mate
//   k_pl_reeval   one thread per pin entry of a swapping node: its
//                 hyperedge's share of the re-evaluated tension
//   scan, k_pl_best, k_pl_first   the best positive prefix per start
//   k_pl_apply    the prefix's swaps applied to gamma and pi
#include "internal.cuh"

#include <algorithm>
#include <vector>
#include "place_items.cuh"

#include <climits>
#include <new>
#include <vector>

namespace {

// offsets non-decreasing, pins in [0, np)
__global__ void k_gp_check(int32_t ne, int64_t P, int32_t np, const int64_t* __restrict__ off,
                           const int32_t* __restrict__ pins, int32_t* err)
{
    int bad = 0;
    int64_t n = (int64_t)ne > P ? (int64_t)ne : P;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < ne && off[i] > off[i + 1]) bad = 1;
        if (i < P && (pins[i] < 0 || pins[i] >= np)) bad = 1;
    }
    if (bad) atomicOr(err, 1);
}

// hyperedge of every pin entry (offsets already checked)
__global__ void k_gp_hid(int32_t ne, const int64_t* __restrict__ off, int32_t* hid)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < ne;
         a += (int64_t)gridDim.x * blockDim.x)
        for (int64_t j = off[a]; j < off[a + 1]; j++) hid[j] = (int32_t)a;
}

}  // namespace

namespace snn {

bool device_pointer(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

Status gp_input(int32_t np, int32_t ne, const int64_t* off, const int32_t* pins,
                const int64_t* eta, Arena& ar, cudaStream_t s, int32_t* err, int64_t* P_out,
                int32_t** hid_out)
{
    if (!device_pointer(off)) return Status{SNNMAP_ERR_INVALID, "buffers must be device memory"};
    int64_t ends[2] = {0, 0};
    SNN_CUDA(cudaMemcpyAsync(&ends[0], off, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaMemcpyAsync(&ends[1], off + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (ends[0] != 0 || ends[1] < 0)
        return Status{SNNMAP_ERR_INVALID, "offsets must start at 0 and not decrease"};
    const int64_t P = ends[1];
    if (P > 0 && (!device_pointer(pins) || !device_pointer(eta)))
        return Status{SNNMAP_ERR_INVALID, "buffers must be device memory"};
    int32_t* hid;
    SNN_TRY(ar.alloc(&hid, P));
    SNN_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    if (ne > 0 || P > 0) {
        SNN_L k_gp_check<<<grid_for(ne > P ? ne : P, 256), 256, 0, s>>>(ne, P, np, off, pins, err);
        SNN_CUDA(cudaGetLastError());
    }
    int32_t herr = 0;
    SNN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (herr) return Status{SNNMAP_ERR_INVALID, "malformed offsets or a pin out of range"};
    if (ne > 0) {
        SNN_L k_gp_hid<<<grid_for(ne, 256), 256, 0, s>>>(ne, off, hid);
        SNN_CUDA(cudaGetLastError());
    }
    *P_out = P;
    *hid_out = hid;
    return Status{};
}

}  // namespace snn

namespace {

using namespace snn;
using place::NO_RANK;

// stats slots, each int64[S]
enum { PS_PROPS = 0, PS_SWAPS = 1, PS_BEST = 2, PS_FIRST = 3, PS_N = 4 };
constexpr int kMaxStarts = 65535;   // gridDim.y

// pi from gamma (pi filled with -1): a core out of range or taken twice
// within a start is an error
__global__ void k_pl_occupy(int32_t np, int32_t nh, const int32_t* __restrict__ g, int32_t* pi,
                            int32_t* err)
{
    int64_t s = blockIdx.y;
    int bad = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = g[s * np + p];
        if (c < 0 || c >= nh) bad = 1;
        else if (atomicCAS(&pi[s * nh + c], -1, (int32_t)p) != -1) bad = 1;
    }
    if (bad) atomicOr(err, 1);
}

__global__ void k_pl_init_stats(int32_t S, int64_t* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)PS_N * S;
         i += (int64_t)gridDim.x * blockDim.x)
        st[i] = i >= (int64_t)PS_FIRST * S ? INT64_MAX : 0;
}

__global__ void k_pl_force(int64_t P, int32_t np, int32_t width, int32_t height,
                           const int32_t* __restrict__ hid, const int64_t* __restrict__ off,
                           const int32_t* __restrict__ pins, const int64_t* __restrict__ eta,
                           const int32_t* __restrict__ g, const int32_t* __restrict__ act,
                           int64_t* F)
{
    int64_t s = blockIdx.y;
    if (!act[s]) return;
    const int32_t* gs = g + s * np;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = hid[j], p = pins[j];
        int32_t h = gs[p];
        int32_t nb[4];
        place::neighbours(width, height, h, nb);
        int64_t f[4] = {0, 0, 0, 0};
        place::force_terms(pins, off[a], off[a + 1], gs, p, h, nb, width, f);
        int64_t w = eta[a];
        unsigned long long* Fp = (unsigned long long*)(F + (s * np + p) * 4);
        for (int d = 0; d < 4; d++)
            if (f[d] != 0 && w != 0) atomicAdd(&Fp[d], (unsigned long long)(w * f[d]));
    }
}

__global__ void k_pl_propose(int32_t nh, int32_t np, int32_t width, int32_t height,
                             const int32_t* __restrict__ act, const int32_t* __restrict__ pi,
                             const int64_t* __restrict__ F, int32_t* cand, int64_t* cscore,
                             int64_t* st_props)
{
    int64_t s = blockIdx.y;
    bool on = act[s] != 0;
    int c = 0;
    for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < nh;
         h += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = s * nh + h;
        int64_t sc = 0;
        int32_t k = on ? place::propose(width, height, pi + s * nh, F + s * np * 4, (int32_t)h, &sc)
                       : -1;
        cand[x] = k < 0 ? -1 : (int32_t)(s * nh + k);
        cscore[x] = sc;
        c += k >= 0;
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)&st_props[s], (unsigned long long)c);
}

// one swap per matched pair, held by its lower core
__global__ void k_pl_flag(int32_t nh, const int32_t* __restrict__ match, int32_t* flag,
                          int64_t* st_swaps)
{
    int64_t s = blockIdx.y;
    int c = 0;
    for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < nh;
         h += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = s * nh + h;
        int f = match[x] > x;
        flag[x] = f;
        c += f;
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)&st_swaps[s], (unsigned long long)c);
}

__global__ void k_pl_compact(int32_t nh, int32_t np, int32_t width, int32_t height,
                             const int32_t* __restrict__ match, const int32_t* __restrict__ pi,
                             const int64_t* __restrict__ F, const int32_t* __restrict__ flag,
                             const int32_t* __restrict__ pos, uint64_t* keys, uint32_t* vals,
                             int32_t* err)
{
    int64_t s = blockIdx.y;
    int bad = 0;
    for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < nh;
         h += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = s * nh + h;
        if (!flag[x]) continue;
        int64_t k = (int64_t)match[x] - s * nh;
        int d = (k >= 0 && k < nh) ? place::direction(width, height, (int32_t)h, (int32_t)k) : -1;
        int64_t t = 0;
        if (d < 0) bad = 1;
        else t = place::tension(pi + s * nh, F + s * np * 4, (int32_t)h, (int32_t)k, d);
        if (t <= 0) bad = 1;   // a matched pair always carries a proposal's positive tension
        keys[pos[x]] = t > 0 ? (uint64_t)INT64_MAX - (uint64_t)t : (uint64_t)INT64_MAX;
        vals[pos[x]] = (uint32_t)x;
    }
    if (bad) atomicOr(err, 2);
}

__global__ void k_pl_startkey(int64_t ns, int32_t nh, const uint32_t* __restrict__ vals,
                              uint64_t* keys)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = vals[i] / (uint32_t)nh;
}

__global__ void k_pl_rank(int64_t ns, int32_t nh, const uint32_t* __restrict__ vals,
                          const int32_t* __restrict__ match, const int32_t* __restrict__ segbeg,
                          int32_t* rank, int32_t* mate)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = vals[i];
        int64_t s = x / nh;
        int64_t y = match[x];
        int32_t r = (int32_t)(i - segbeg[s]);
        rank[x] = r;
        rank[y] = r;
        mate[x] = (int32_t)(y - s * nh);
        mate[y] = (int32_t)(x - s * nh);
    }
}

__global__ void k_pl_reeval(int64_t P, int32_t np, int32_t nh, int32_t width,
                            const int32_t* __restrict__ hid, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ pins, const int64_t* __restrict__ eta,
                            const int32_t* __restrict__ g, const int32_t* __restrict__ rank,
                            const int32_t* __restrict__ mate, const int32_t* __restrict__ segbeg,
                            int64_t* Tn)
{
    int64_t s = blockIdx.y;
    const int32_t* gs = g + s * np;
    const int32_t* rs = rank + s * nh;
    const int32_t* ms = mate + s * nh;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = pins[j];
        int32_t h = gs[p];
        int32_t r = rs[h];
        if (r == NO_RANK) continue;
        int32_t a = hid[j];
        int64_t v = place::reeval_terms(pins, off[a], off[a + 1], gs, rs, ms, p, h, ms[h], r, width);
        if (v != 0 && eta[a] != 0)
            atomicAdd((unsigned long long*)&Tn[segbeg[s] + r], (unsigned long long)(eta[a] * v));
    }
}

// prefix sum of swap i within its start, from the inclusive scan C
__device__ __forceinline__ int64_t local_prefix(const int64_t* C, int64_t i, int32_t b)
{
    return C[i] - (b > 0 ? C[b - 1] : 0);
}

__global__ void k_pl_best(int64_t ns, int32_t nh, const uint32_t* __restrict__ vals,
                          const int32_t* __restrict__ segbeg, const int64_t* __restrict__ C,
                          int64_t* st_best)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = vals[i] / (uint32_t)nh;
        int64_t G = local_prefix(C, i, segbeg[s]);
        if (G > 0) atomicMax((long long*)&st_best[s], (long long)G);
    }
}

__global__ void k_pl_first(int64_t ns, int32_t nh, const uint32_t* __restrict__ vals,
                           const int32_t* __restrict__ segbeg, const int64_t* __restrict__ C,
                           const int64_t* __restrict__ st_best, int64_t* st_first)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = vals[i] / (uint32_t)nh;
        int64_t G = local_prefix(C, i, segbeg[s]);
        if (G > 0 && G == st_best[s])
            atomicMin((long long*)&st_first[s], (long long)(i - segbeg[s]));
    }
}

__global__ void k_pl_apply(int64_t ns, int32_t nh, int32_t np, const uint32_t* __restrict__ vals,
                           const int32_t* __restrict__ match, const int32_t* __restrict__ segbeg,
                           const int64_t* __restrict__ st_first, int32_t* pi, int32_t* g)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = vals[i];
        int64_t s = x / nh;
        int64_t f = st_first[s];
        if (f == INT64_MAX || i - segbeg[s] > f) continue;
        int64_t y = match[x];
        int32_t a = pi[x], b = pi[y];
        pi[x] = b;
        pi[y] = a;
        if (a >= 0) g[s * np + a] = (int32_t)(y - s * nh);
        if (b >= 0) g[s * np + b] = (int32_t)(x - s * nh);
    }
}

__global__ void k_pl_trd(int64_t P, int32_t np, int32_t width, const int32_t* __restrict__ hid,
                         const int64_t* __restrict__ off, const int32_t* __restrict__ pins,
                         const int64_t* __restrict__ eta, const int32_t* __restrict__ g,
                         int64_t* acc)
{
    int64_t s = blockIdx.y;
    const int32_t* gs = g + s * np;
    int64_t sum = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = hid[j];
        sum += eta[a] * place::trd_terms(pins, j, off[a + 1], gs, width);
    }
    sum = warp_sum(sum);
    if ((threadIdx.x & 31) == 0 && sum != 0) atomicAdd((unsigned long long*)&acc[s], (unsigned long long)sum);
}

// blocks along x for a 2-D launch over S starts of n items each
dim3 grid2(int64_t n, int32_t S)
{
    int cap = 152 * 32 / S;
    return dim3((unsigned)grid_for(n, 256, cap > 0 ? cap : 1), (unsigned)S);
}

struct Input {
    int32_t np, ne, width, height, S;
    int64_t P = 0, nh = 0;
    const int64_t* off;
    const int32_t* pins;
    const int64_t* eta;
};

Status invalid(const char* msg) { return Status{SNNMAP_ERR_INVALID, msg}; }

// Argument checks, G_P (gp_input: its pin count and the hyperedge of every
// pin entry) and the inverse placement pi of every start (from the arena).
Status prepare(Input& in, const int32_t* g, Arena& ar, cudaStream_t s, int32_t** hid_out,
               int32_t** pi_out, int32_t* err)
{
    if (in.np < 0 || in.ne < 0 || in.width < 1 || in.height < 1 || in.S < 1 || in.S > kMaxStarts)
        return invalid("negative sizes, width or height < 1, or n_starts outside [1, 65535]");
    in.nh = (int64_t)in.width * in.height;
    if (in.nh * in.S >= ((int64_t)1 << 31)) return invalid("n_starts * width * height >= 2^31");
    if (in.np > in.nh) return invalid("more nodes than cores");
    if (in.np > 0 && !device_pointer(g)) return invalid("buffers must be device memory");
    SNN_TRY(gp_input(in.np, in.ne, in.off, in.pins, in.eta, ar, s, err, &in.P, hid_out));
    int32_t* pi;
    SNN_TRY(ar.alloc(&pi, in.nh * in.S));
    SNN_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    SNN_TRY(fill_i32(pi, -1, in.nh * in.S, s));
    if (in.np > 0) {
        SNN_L k_pl_occupy<<<grid2(in.np, in.S), 256, 0, s>>>(in.np, (int32_t)in.nh, g, pi, err);
        SNN_CUDA(cudaGetLastError());
    }
    int32_t herr = 0;
    SNN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SNN_CUDA(cudaStreamSynchronize(s));
    if (herr) return invalid("a core out of range or taken twice");
    *pi_out = pi;
    return Status{};
}

Status refine_impl(Input& in, int32_t* g, int32_t max_rounds, cudaStream_t s, int32_t* rounds_out,
                   snnmap_place_log* log, int32_t log_cap)
{
    if (max_rounds < 0 || log_cap < 0) return invalid("max_rounds and log_cap must be >= 0");
    Arena ar;
    ar.stream = s;
    struct Guard {
        Arena& a;
        ~Guard() { a.release(); }
    } guard{ar};
    int32_t* err;
    SNN_TRY(ar.alloc(&err, 1));
    int32_t *hid, *pi;
    SNN_TRY(prepare(in, g, ar, s, &hid, &pi, err));
    const int32_t S = in.S, np = in.np, nh = (int32_t)in.nh;
    const int64_t V = in.nh * S;
    int64_t *F, *cscore, *st, *scal;
    int32_t *cand, *match, *flag, *pos, *rank, *mate, *act, *segbeg;
    SNN_TRY(ar.alloc(&F, (int64_t)S * np * 4));
    SNN_TRY(ar.alloc(&cscore, V));
    SNN_TRY(ar.alloc(&st, (int64_t)PS_N * S));
    SNN_TRY(ar.alloc(&scal, SC_COUNT));
    SNN_TRY(ar.alloc(&cand, V));
    SNN_TRY(ar.alloc(&match, V));
    SNN_TRY(ar.alloc(&flag, V));
    SNN_TRY(ar.alloc(&pos, V));
    SNN_TRY(ar.alloc(&rank, V));
    SNN_TRY(ar.alloc(&mate, V));
    SNN_TRY(ar.alloc(&act, S));
    SNN_TRY(ar.alloc(&segbeg, S));
    std::vector<int32_t> h_act(S, 1), h_rounds(S, 0), h_seg(S, 0);
    std::vector<int64_t> h_st((size_t)PS_N * S);
    std::vector<std::vector<snnmap_place_log>> logs(S);
    SNN_CUDA(cudaMemcpyAsync(act, h_act.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
    int32_t active = S;
    const dim3 gn = grid2(in.P, S), gc = grid2(nh, S);
    for (int32_t round = 0; round < max_rounds && active > 0; round++) {
        Arena::Mark mk = ar.mark();
        SNN_CUDA(cudaMemsetAsync(F, 0, sizeof(int64_t) * S * (int64_t)np * 4, s));
        SNN_L k_pl_init_stats<<<1, 256, 0, s>>>(S, st);
        if (in.P > 0) {
            SNN_L k_pl_force<<<gn, 256, 0, s>>>(in.P, np, in.width, in.height, hid, in.off,
                                                in.pins, in.eta, g, act, F);
        }
        SNN_L k_pl_propose<<<gc, 256, 0, s>>>(nh, np, in.width, in.height, act, pi, F, cand,
                                              cscore, st + (int64_t)PS_PROPS * S);
        SNN_CUDA(cudaGetLastError());
        int64_t pairs = 0;
        SNN_TRY(match_forest((int32_t)V, cand, cscore, match, scal, ar, s, &pairs));
        SNN_L k_pl_flag<<<gc, 256, 0, s>>>(nh, match, flag, st + (int64_t)PS_SWAPS * S);
        SNN_CUDA(cudaGetLastError());
        SNN_CUDA(cudaMemcpyAsync(h_st.data(), st, sizeof(int64_t) * PS_N * S, cudaMemcpyDeviceToHost, s));
        SNN_CUDA(cudaStreamSynchronize(s));
        int64_t ns = 0;
        for (int32_t i = 0; i < S; i++) {
            h_seg[i] = (int32_t)ns;
            ns += h_st[(size_t)PS_SWAPS * S + i];
        }
        if (ns != pairs) return Status{SNNMAP_ERR_CUDA, "placement: swap count mismatch"};
        if (ns > 0) {
            SNN_CUDA(cudaMemcpyAsync(segbeg, h_seg.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
            SNN_TRY(scan_exclusive_i32(flag, pos, V, nullptr, ar, s));
            uint64_t *keys, *keys2;
            uint32_t *vals, *vals2;
            int64_t *Tn, *C;
            SNN_TRY(ar.alloc(&keys, ns));
            SNN_TRY(ar.alloc(&keys2, ns));
            SNN_TRY(ar.alloc(&vals, ns));
            SNN_TRY(ar.alloc(&vals2, ns));
            SNN_TRY(ar.alloc(&Tn, ns));
            SNN_TRY(ar.alloc(&C, ns));
            SNN_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
            SNN_L k_pl_compact<<<gc, 256, 0, s>>>(nh, np, in.width, in.height, match, pi, F, flag,
                                                  pos, keys, vals, err);
            SNN_CUDA(cudaGetLastError());
            SNN_TRY(radix_sort_pairs(keys, vals, keys2, vals2, ns, 63, ar, s));
            if (S > 1) {
                SNN_L k_pl_startkey<<<grid_for(ns, 256), 256, 0, s>>>(ns, nh, vals, keys);
                SNN_CUDA(cudaGetLastError());
                SNN_TRY(radix_sort_pairs(keys, vals, keys2, vals2, ns, bits_for((uint64_t)(S - 1)),
                                         ar, s));
            }
            SNN_TRY(fill_i32(rank, NO_RANK, V, s));
            SNN_L k_pl_rank<<<grid_for(ns, 256), 256, 0, s>>>(ns, nh, vals, match, segbeg, rank, mate);
            SNN_CUDA(cudaMemsetAsync(Tn, 0, sizeof(int64_t) * ns, s));
            if (in.P > 0) {
                SNN_L k_pl_reeval<<<gn, 256, 0, s>>>(in.P, np, nh, in.width, hid, in.off, in.pins,
                                                     in.eta, g, rank, mate, segbeg, Tn);
            }
            SNN_CUDA(cudaGetLastError());
            SNN_TRY(scan_inclusive_i64(Tn, C, ns, ar, s));
            SNN_L k_pl_best<<<grid_for(ns, 256), 256, 0, s>>>(ns, nh, vals, segbeg, C,
                                                              st + (int64_t)PS_BEST * S);
            SNN_L k_pl_first<<<grid_for(ns, 256), 256, 0, s>>>(ns, nh, vals, segbeg, C,
                                                               st + (int64_t)PS_BEST * S,
                                                               st + (int64_t)PS_FIRST * S);
            SNN_L k_pl_apply<<<grid_for(ns, 256), 256, 0, s>>>(ns, nh, np, vals, match, segbeg,
                                                               st + (int64_t)PS_FIRST * S, pi, g);
            SNN_CUDA(cudaGetLastError());
            int32_t herr = 0;
            SNN_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            SNN_CUDA(cudaMemcpyAsync(h_st.data(), st, sizeof(int64_t) * PS_N * S, cudaMemcpyDeviceToHost, s));
            SNN_CUDA(cudaStreamSynchronize(s));
            if (herr) return Status{SNNMAP_ERR_CUDA, "placement: a matched pair without positive tension"};
        }
        bool changed = false;
        for (int32_t i = 0; i < S; i++) {
            if (!h_act[i]) continue;
            int64_t first = h_st[(size_t)PS_FIRST * S + i];
            snnmap_place_log L;
            L.props = (int32_t)h_st[(size_t)PS_PROPS * S + i];
            L.swaps = (int32_t)h_st[(size_t)PS_SWAPS * S + i];
            L.applied = first == INT64_MAX ? 0 : (int32_t)(first + 1);
            L.reserved = 0;
            L.gain = first == INT64_MAX ? 0 : h_st[(size_t)PS_BEST * S + i];
            if ((int64_t)logs[i].size() < log_cap) logs[i].push_back(L);
            h_rounds[i]++;
            if (L.applied == 0) {
                h_act[i] = 0;
                active--;
                changed = true;
            }
        }
        if (changed && active > 0)
            SNN_CUDA(cudaMemcpyAsync(act, h_act.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
        ar.rewind(mk);
    }
    SNN_CUDA(cudaStreamSynchronize(s));
    for (int32_t i = 0; i < S; i++) {
        if (rounds_out) rounds_out[i] = h_rounds[i];
        if (log)
            for (size_t r = 0; r < logs[i].size(); r++) log[(int64_t)i * log_cap + (int64_t)r] = logs[i][r];
    }
    return Status{};
}

Status trd_impl(Input& in, const int32_t* g, cudaStream_t s, int64_t* trd_out)
{
    Arena ar;
    ar.stream = s;
    struct Guard {
        Arena& a;
        ~Guard() { a.release(); }
    } guard{ar};
    int32_t* err;
    SNN_TRY(ar.alloc(&err, 1));
    int32_t *hid, *pi;
    SNN_TRY(prepare(in, g, ar, s, &hid, &pi, err));
    int64_t* acc;
    SNN_TRY(ar.alloc(&acc, in.S));
    SNN_CUDA(cudaMemsetAsync(acc, 0, sizeof(int64_t) * in.S, s));
    if (in.P > 0) {
        SNN_L k_pl_trd<<<grid2(in.P, in.S), 256, 0, s>>>(in.P, in.np, in.width, hid, in.off,
                                                         in.pins, in.eta, g, acc);
        SNN_CUDA(cudaGetLastError());
    }
    SNN_CUDA(cudaMemcpyAsync(trd_out, acc, sizeof(int64_t) * in.S, cudaMemcpyDeviceToHost, s));
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

int snnmap_place_refine(int32_t n_nodes, int32_t n_hedges, const int64_t* d_offsets,
                        const int32_t* d_pins, const int64_t* d_eta, int32_t width,
                        int32_t height, int32_t n_starts, int32_t* d_gamma, int32_t max_rounds,
                        void* stream, int32_t* h_rounds_out, snnmap_place_log* h_log,
                        int32_t log_cap)
{
    try {
        Input in{n_nodes, n_hedges, width, height, n_starts, 0, 0, d_offsets, d_pins, d_eta};
        return finish(refine_impl(in, d_gamma, max_rounds, (cudaStream_t)stream, h_rounds_out,
                                  h_log, log_cap));
    } catch (const std::bad_alloc&) {
        return finish(Status{SNNMAP_ERR_OOM, "host allocation failed"});
    } catch (...) {
        return finish(Status{SNNMAP_ERR_CUDA, "internal error"});
    }
}

int snnmap_place_trd(int32_t n_nodes, int32_t n_hedges, const int64_t* d_offsets,
                     const int32_t* d_pins, const int64_t* d_eta, int32_t width, int32_t height,
                     int32_t n_starts, const int32_t* d_gamma, void* stream, int64_t* h_trd_out)
{
    try {
        if (!h_trd_out) return finish(Status{SNNMAP_ERR_INVALID, "h_trd_out is NULL"});
        Input in{n_nodes, n_hedges, width, height, n_starts, 0, 0, d_offsets, d_pins, d_eta};
        return finish(trd_impl(in, d_gamma, (cudaStream_t)stream, h_trd_out));
    } catch (const std::bad_alloc&) {
        return finish(Status{SNNMAP_ERR_OOM, "host allocation failed"});
    } catch (...) {
        return finish(Status{SNNMAP_ERR_CUDA, "internal error"});
    }
}

int snnmap_place_best(int32_t n_nodes, int32_t n_hedges, const int64_t* d_offsets,
                      const int32_t* d_pins, const int64_t* d_eta, int32_t width, int32_t height,
                      int32_t n_starts, const int32_t* d_gamma, void* stream, int32_t* best_out,
                      int64_t* trd_out, int64_t* h_trd_out)
{
    try {
        if (!best_out) return finish(Status{SNNMAP_ERR_INVALID, "best_out is NULL"});
        Input in{n_nodes, n_hedges, width, height, n_starts, 0, 0, d_offsets, d_pins, d_eta};
        std::vector<int64_t> trd((size_t)(n_starts > 0 ? n_starts : 1));
        Status st = trd_impl(in, d_gamma, (cudaStream_t)stream, trd.data());
        if (!st.ok()) return finish(st);
        // Sec. 4.2: the start of smallest total residual distance; the
        // lowest start on ties
        int32_t best = 0;
        for (int32_t s = 1; s < n_starts; s++)
            if (trd[(size_t)s] < trd[(size_t)best]) best = s;
        *best_out = best;
        if (trd_out) *trd_out = trd[(size_t)best];
        if (h_trd_out) std::copy(trd.begin(), trd.begin() + n_starts, h_trd_out);
        return finish(Status{});
    } catch (const std::bad_alloc&) {
        return finish(Status{SNNMAP_ERR_OOM, "host allocation failed"});
    } catch (...) {
        return finish(Status{SNNMAP_ERR_CUDA, "internal error"});
    }
}

}  // extern "C"
