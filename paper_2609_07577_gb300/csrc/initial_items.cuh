// Per-item steps of the initial placement (Sec. 4.2, "Initial Placement")
// of G_P: the Hilbert index of a core, the sides and cut changes of the
// label propagation between two sibling sections, and the folding of the
// bisection tree. The kernels of initial.cu run one item per thread; the
// header uses no CUDA type, so the same steps also compile as plain host
// code and can be run one item at a time.
//
// Sections are intervals of a start's node sequence; pos[q] is the position
// of node q in it. For the label propagation between sibling sections
// L = [lo, mid) and R = [mid, hi), a hyperedge's pins outside both are
// ignored and a hyperedge is cut when it has pins on both sides; its pins
// must be distinct.
//
// Cut change of one swap (x of L with y of R). Moving x across alone lowers
// the cut by delta_L(a) = [cL = 1 and cR > 0] - [cL >= 2 and cR = 0] per
// hyperedge a holding x (cL, cR: its pins in L and R), and y alike. Where a
// holds both x and y the swap leaves a's counts, hence its cut, unchanged,
// while the two single moves counted [cL = 1] + [cR = 1] for it. So the
// swap lowers the cut by G(x) + G(y) - corr(x, y), with G(v) the summed
// eta-weighted single-move changes of v and corr(x, y) the sum over
// hyperedges holding both of eta(a) ([cL = 1] + [cR = 1]).
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define IP_HD __host__ __device__ __forceinline__
#else
#define IP_HD inline
#endif

namespace snn {
namespace initial {

// Index of cell (x, y) along the Hilbert curve over an n x n square (n a
// power of two), by the usual quadrant descent: at each scale s the
// quadrant gives s*s*((3*rx) ^ ry), and the cell is rotated (and mirrored
// for rx = 1) into the frame of that quadrant when ry = 0.
IP_HD uint32_t hilbert_index(uint32_t n, uint32_t x, uint32_t y)
{
    uint32_t d = 0;
    for (uint32_t s = n >> 1; s > 0; s >>= 1) {
        uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = s - 1 - x;
                y = s - 1 - y;
            }
            uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// 1: position i in L, 2: in R, 0: outside the pair
IP_HD int side_of(int32_t i, int32_t lo, int32_t mid, int32_t hi)
{
    return (i >= lo && i < mid) ? 1 : (i >= mid && i < hi) ? 2 : 0;
}

// pins of one hyperedge (pins[b..e)) in L and in R
IP_HD void side_counts(const int32_t* pins, int64_t b, int64_t e, const int32_t* pos, int32_t lo,
                       int32_t mid, int32_t hi, int32_t* cL, int32_t* cR)
{
    int32_t l = 0, r = 0;
    for (int64_t j = b; j < e; j++) {
        int sd = side_of(pos[pins[j]], lo, mid, hi);
        l += sd == 1;
        r += sd == 2;
    }
    *cL = l;
    *cR = r;
}

// cut drop of moving one node of side sd (1: L, 2: R) across alone
IP_HD int32_t move_delta(int sd, int32_t cL, int32_t cR)
{
    int32_t own = sd == 1 ? cL : cR, other = sd == 1 ? cR : cL;
    if (own == 1 && other > 0) return 1;
    if (own >= 2 && other == 0) return -1;
    return 0;
}

// G(x) of node x on side sd: incidences inc[ib..ie) (hyperedge ids)
IP_HD int64_t single_gain(const int32_t* inc, int64_t ib, int64_t ie, const int64_t* off,
                          const int32_t* pins, const int64_t* eta, const int32_t* pos, int sd,
                          int32_t lo, int32_t mid, int32_t hi)
{
    int64_t g = 0;
    for (int64_t t = ib; t < ie; t++) {
        int32_t a = inc[t], cL, cR;
        side_counts(pins, off[a], off[a + 1], pos, lo, mid, hi, &cL, &cR);
        g += eta[a] * move_delta(sd, cL, cR);
    }
    return g;
}

// corr(x, .) of node x in L over its incidences: add(j, w) receives
// corr contributions for the node at position mid + j of R. A hyperedge
// with x as its only L pin pairs x with each of its R pins (weight
// eta (1 + [cR = 1])); one with several L pins and a single R pin pairs x
// with that pin (weight eta); no other hyperedge contributes.
template <typename Add>
IP_HD void corr_row(const int32_t* inc, int64_t ib, int64_t ie, const int64_t* off,
                    const int32_t* pins, const int64_t* eta, const int32_t* pos, int32_t lo,
                    int32_t mid, int32_t hi, Add add)
{
    for (int64_t t = ib; t < ie; t++) {
        int32_t a = inc[t], cL, cR;
        side_counts(pins, off[a], off[a + 1], pos, lo, mid, hi, &cL, &cR);
        if (cR == 0 || (cL != 1 && cR != 1)) continue;
        int64_t w = cL == 1 ? eta[a] * (1 + (cR == 1)) : eta[a];
        for (int64_t j = off[a]; j < off[a + 1]; j++) {
            int32_t i = pos[pins[j]];
            if (side_of(i, lo, mid, hi) == 2) add(i - mid, w);
        }
    }
}

// corr(., x) of node x in R over its incidences, the mirror of corr_row:
// add(i, w) receives contributions for the node at position lo + i of L,
// except the node skip (whose row is rebuilt by corr_row).
template <typename Add>
IP_HD void corr_col(const int32_t* inc, int64_t ib, int64_t ie, const int64_t* off,
                    const int32_t* pins, const int64_t* eta, const int32_t* pos, int32_t lo,
                    int32_t mid, int32_t hi, int32_t skip, Add add)
{
    for (int64_t t = ib; t < ie; t++) {
        int32_t a = inc[t], cL, cR;
        side_counts(pins, off[a], off[a + 1], pos, lo, mid, hi, &cL, &cR);
        if (cL == 0 || (cL != 1 && cR != 1)) continue;
        int64_t w = cR == 1 ? eta[a] * (1 + (cL == 1)) : eta[a];
        for (int64_t j = off[a]; j < off[a + 1]; j++) {
            int32_t u = pins[j];
            int32_t i = pos[u];
            if (u != skip && side_of(i, lo, mid, hi) == 1) add(i - lo, w);
        }
    }
}

// What the swap of x (in L) with y (in R) changes through one hyperedge
// (pins[b..e), weight w_eta), with pos the positions before the swap:
// gadd(v, d) for every pin v whose single-move gain G(v) changes (the
// hyperedge's side counts change, or v is x or y and changes side), and
// madd(i, j, d) for the correction entries of pairs of non-moving pins
// (L position lo + i, R position mid + j), whose weight eta ([cL = 1] +
// [cR = 1]) changes with the counts. Such a change needs a side count to
// cross 1, which leaves at most one non-moving pin on that side, so the
// pairs are O(|a|). Pairs with x or y are left to the rebuild of their row
// and column. skip_if_x: the hyperedge came from y's incidence list and is
// handled from x's if it holds x too.
template <typename GAdd, typename MAdd>
IP_HD void swap_hedge_update(const int32_t* pins, int64_t b, int64_t e, const int32_t* pos,
                             int32_t lo, int32_t mid, int32_t hi, int32_t x, int32_t y,
                             int64_t w_eta, bool skip_if_x, GAdd gadd, MAdd madd)
{
    int32_t cL = 0, cR = 0;
    bool hx = false, hy = false;
    for (int64_t j = b; j < e; j++) {
        int32_t q = pins[j];
        int sd = side_of(pos[q], lo, mid, hi);
        cL += sd == 1;
        cR += sd == 2;
        hx = hx || q == x;
        hy = hy || q == y;
    }
    if (skip_if_x && hx) return;
    int32_t nL = cL - hx + hy, nR = cR + hx - hy;   // counts after the swap
    for (int64_t j = b; j < e; j++) {
        int32_t q = pins[j];
        int so = side_of(pos[q], lo, mid, hi);
        if (so == 0) continue;
        int sn = q == x ? 2 : q == y ? 1 : so;
        int32_t d = move_delta(sn, nL, nR) - move_delta(so, cL, cR);
        if (d != 0) gadd(q, w_eta * d);
    }
    int32_t dw = ((nL == 1) + (nR == 1)) - ((cL == 1) + (cR == 1));
    int32_t mL = cL - hx, mR = cR - hy;   // non-moving pins on each side
    if (dw == 0 || mL == 0 || mR == 0) return;
    int outer = mL <= mR ? 1 : 2;
    for (int64_t j = b; j < e; j++) {
        int32_t u = pins[j];
        int32_t iu = pos[u];
        if (u == x || u == y || side_of(iu, lo, mid, hi) != outer) continue;
        for (int64_t t = b; t < e; t++) {
            int32_t v = pins[t];
            int32_t iv = pos[v];
            if (v == x || v == y || side_of(iv, lo, mid, hi) != 3 - outer) continue;
            if (outer == 1) madd(iu - lo, iv - mid, w_eta * dw);
            else madd(iv - lo, iu - mid, w_eta * dw);
        }
    }
}

// Bisection tree of a sequence of n nodes, breadth-first: node 0 = [0, n);
// a node of more than one position splits into its first ceil(len/2)
// positions and the rest, children numbered consecutively. Descending
// from the root to position i: the child holding i.
IP_HD int32_t child_holding(const int32_t* lo, const int32_t* hi, const int32_t* kid, int32_t s,
                            int32_t i)
{
    int32_t n = hi[s] - lo[s];
    int32_t mid = lo[s] + (n + 1) / 2;
    return i < mid ? kid[s] : kid[s] + 1;
}

// whether pin entry j of hyperedge [b, e) is its lowest-position pin in
// [c0, c1), and whether the hyperedge has a pin in [s0, s1)
IP_HD void fold_checks(const int32_t* pins, int64_t b, int64_t e, const int32_t* pos, int64_t j,
                       int32_t c0, int32_t c1, int32_t s0, int32_t s1, bool* first, bool* meets)
{
    int32_t pj = pos[pins[j]];
    bool f = true, m = false;
    for (int64_t t = b; t < e; t++) {
        int32_t p = pos[pins[t]];
        if (p >= c0 && p < c1 && p < pj) f = false;
        if (p >= s0 && p < s1) m = true;
    }
    *first = f;
    *meets = m;
}

// Final position of the node at position i after folding: from the root
// down, a section whose accumulated orientation (its own flip xor its
// ancestors') is reversed puts its second child first.
IP_HD int32_t folded_position(const int32_t* lo, const int32_t* hi, const int32_t* kid,
                              const uint8_t* flip, int32_t i)
{
    int32_t s = 0, off = 0;
    int f = 0;
    while (kid[s] >= 0) {
        f ^= flip[s];
        int32_t c0 = kid[s], c1 = kid[s] + 1;
        int32_t n0 = hi[c0] - lo[c0], n1 = hi[c1] - lo[c1];
        int32_t c = child_holding(lo, hi, kid, s, i);
        if (c == c0) off += f ? n1 : 0;
        else off += f ? 0 : n0;
        s = c;
    }
    return off;
}

}  // namespace initial
}  // namespace snn
