// Per-item steps of placement swap refinement (Sec. 4.2, "Swap Proposals"
// and "Placement Refinement") on a width x height lattice of cores, core
// h = y * width + x. The kernels of place.cu run one item per thread; the
// header uses no CUDA type, so the same steps also compile as plain host
// code and can be run one item at a time.
//
// Per start, g[p] is the core of node p and pi[h] the node on core h (-1:
// empty). Forces are kept four per node, one per direction d of the
// adjacent core: 0 up (h - width), 1 left (h - 1), 2 right (h + 1), 3 down
// (h + width), which is ascending core id order; d and 3 - d are opposite.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define PL_HD __host__ __device__ __forceinline__
#else
#define PL_HD inline
#endif

namespace snn {
namespace place {

constexpr int32_t NO_RANK = 0x7fffffff;   // rank of a core that is in no swap

// Manhattan distance between cores u and v
PL_HD int32_t dist(int32_t width, int32_t u, int32_t v)
{
    int32_t dx = u % width - v % width, dy = u / width - v / width;
    return (dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy);
}

// the cores adjacent to h (the set J(h) of Eq. force) by direction, -1 past
// the lattice's border
PL_HD void neighbours(int32_t width, int32_t height, int32_t h, int32_t nb[4])
{
    int32_t x = h % width, y = h / width;
    nb[0] = y > 0 ? h - width : -1;
    nb[1] = x > 0 ? h - 1 : -1;
    nb[2] = x + 1 < width ? h + 1 : -1;
    nb[3] = y + 1 < height ? h + width : -1;
}

// direction of core k seen from core h, -1 if k is not adjacent to h
PL_HD int direction(int32_t width, int32_t height, int32_t h, int32_t k)
{
    int32_t nb[4];
    neighbours(width, height, h, nb);
    for (int d = 0; d < 4; d++)
        if (nb[d] >= 0 && nb[d] == k) return d;
    return -1;
}

// One hyperedge's share of Eq. force, without its factor eta: for node p on
// core h and each adjacent core nb[d], s[d] += sum over the hyperedge's pins
// q != p (pins[b..e)) of dist(h, g[q]) - max(dist(nb[d], g[q]), 1). s[d] is
// left alone where nb[d] < 0.
PL_HD void force_terms(const int32_t* pins, int64_t b, int64_t e, const int32_t* g, int32_t p,
                       int32_t h, const int32_t nb[4], int32_t width, int64_t s[4])
{
    for (int64_t j = b; j < e; j++) {
        int32_t q = pins[j];
        if (q == p) continue;
        int32_t c = g[q];
        int32_t d0 = dist(width, h, c);
        for (int d = 0; d < 4; d++) {
            if (nb[d] < 0) continue;
            int32_t dk = dist(width, nb[d], c);
            s[d] += d0 - (dk > 1 ? dk : 1);
        }
    }
}

// Eq. tension between core h and its adjacent core k in direction d, from
// the forces F (four per node) of the nodes on them; an empty core adds
// nothing
PL_HD int64_t tension(const int32_t* pi, const int64_t* F, int32_t h, int32_t k, int d)
{
    int64_t t = 0;
    int32_t a = pi[h], b = pi[k];
    if (a >= 0) t += F[(int64_t)a * 4 + d];
    if (b >= 0) t += F[(int64_t)b * 4 + (3 - d)];
    return t;
}

// The swap proposed by core h: the adjacent core of largest tension, the
// lowest core id on ties, if that tension is positive; an empty core
// proposes nothing. Returns the core (or -1) and its tension in *score
// (0 without a proposal).
PL_HD int32_t propose(int32_t width, int32_t height, const int32_t* pi, const int64_t* F,
                      int32_t h, int64_t* score)
{
    *score = 0;
    if (pi[h] < 0) return -1;
    int32_t nb[4];
    neighbours(width, height, h, nb);
    int32_t best = -1;
    int64_t bt = 0;
    for (int d = 0; d < 4; d++) {
        if (nb[d] < 0) continue;
        int64_t t = tension(pi, F, h, nb[d], d);
        if (best < 0 || t > bt) {
            best = nb[d];
            bt = t;
        }
    }
    if (best < 0 || bt <= 0) return -1;
    *score = bt;
    return best;
}

// Core of the node now on core c once every swap ranked before r is
// applied: rank[c] is the rank of c's swap (NO_RANK if none) and mate[c]
// the other core of that swap.
PL_HD int32_t core_before(const int32_t* rank, const int32_t* mate, int32_t c, int32_t r)
{
    return rank[c] < r ? mate[c] : c;
}

// One hyperedge's share of Eq. force for node p moving from core h to core
// k in the swap of rank r, evaluated with every swap ranked before r
// applied (p and the node on k have not moved yet: each core is in one swap
// at most), without the factor eta.
PL_HD int64_t reeval_terms(const int32_t* pins, int64_t b, int64_t e, const int32_t* g,
                           const int32_t* rank, const int32_t* mate, int32_t p, int32_t h,
                           int32_t k, int32_t r, int32_t width)
{
    int64_t s = 0;
    for (int64_t j = b; j < e; j++) {
        int32_t q = pins[j];
        if (q == p) continue;
        int32_t c = core_before(rank, mate, g[q], r);
        int32_t dk = dist(width, k, c);
        s += dist(width, h, c) - (dk > 1 ? dk : 1);
    }
    return s;
}

// Distances from pin j of a hyperedge to the pins after it (pins[j+1..e)):
// one pin's share of the total residual distance, without eta.
PL_HD int64_t trd_terms(const int32_t* pins, int64_t j, int64_t e, const int32_t* g, int32_t width)
{
    int64_t s = 0;
    int32_t h = g[pins[j]];
    for (int64_t i = j + 1; i < e; i++) s += dist(width, h, g[pins[i]]);
    return s;
}

}  // namespace place
}  // namespace snn
