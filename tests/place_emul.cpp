// Host run of the placement refinement kernels' steps: the per-item
// functions of csrc/place_items.cuh, called one item at a time in the phase
// order of the kernels in csrc/place.cu (forces summed per pin entry,
// proposals per core over all starts, Eq. matching in the matching kernels'
// formulation, swaps sorted by tension then by start, re-evaluation through
// ranks, per-start best prefix, apply). It checks that decomposition against
// the oracle without a GPU. Test infrastructure only; built by the tests.
#include "place_items.cuh"

#include <algorithm>
#include <climits>
#include <cstdint>
#include <vector>

using namespace snn::place;

namespace {

// Eq. matching as the matching kernels compute it: best child per vertex
// (largest score, lowest id), a link to the parent for a best child outside
// a root two-cycle, the parity of the distance to the chain's top, then the
// parent at odd distance (or the root partner), else the best child.
void match_forest(int32_t V, const std::vector<int32_t>& cand, const std::vector<int64_t>& cscore,
                  std::vector<int32_t>& match)
{
    std::vector<int64_t> bestsc(V, INT64_MIN);
    std::vector<int32_t> bc(V, INT32_MAX), link(V, -1);
    std::vector<uint8_t> par(V, 0);
    for (int32_t n = 0; n < V; n++)
        if (cand[n] >= 0) bestsc[cand[n]] = std::max(bestsc[cand[n]], cscore[n]);
    for (int32_t n = 0; n < V; n++)
        if (cand[n] >= 0 && cscore[n] == bestsc[cand[n]]) bc[cand[n]] = std::min(bc[cand[n]], n);
    auto is_root = [&](int32_t n) { return cand[n] >= 0 && cand[cand[n]] == n; };
    for (int32_t n = 0; n < V; n++) {
        int32_t c = cand[n];
        if (c >= 0 && cand[c] != n && !is_root(c) && bc[c] == n) link[n] = c;
    }
    for (int32_t n = 0; n < V; n++) {
        int d = 0;
        for (int32_t x = n; link[x] >= 0; x = link[x]) d++;
        par[n] = (uint8_t)(d & 1);
    }
    for (int32_t n = 0; n < V; n++) {
        int32_t c = cand[n];
        if (c >= 0 && (cand[c] == n || par[n] == 1)) match[n] = c;
        else match[n] = bc[n] != INT32_MAX ? bc[n] : -1;
    }
}

struct Swap {
    uint64_t key;
    uint32_t x;
};

}  // namespace

extern "C" {

// Same contract as snnmap_place_refine on host arrays; logs are per start,
// start-major with log_cap entries each. Returns 0, 1 (invalid input) or 2
// (a matched pair without positive tension).
int emul_place_refine(int32_t np, int32_t ne, const int64_t* off, const int32_t* pins,
                      const int64_t* eta, int32_t width, int32_t height, int32_t S, int32_t* g,
                      int32_t max_rounds, int32_t* rounds_out, int32_t* log_props,
                      int32_t* log_swaps, int32_t* log_applied, int64_t* log_gain, int32_t log_cap)
{
    const int32_t nh = width * height, V = nh * S;
    const int64_t P = off[ne];
    std::vector<int32_t> hid((size_t)P), pi((size_t)V, -1);
    for (int32_t a = 0; a < ne; a++)
        for (int64_t j = off[a]; j < off[a + 1]; j++) hid[j] = a;
    for (int32_t s = 0; s < S; s++)
        for (int32_t p = 0; p < np; p++) {
            int32_t c = g[(int64_t)s * np + p];
            if (c < 0 || c >= nh || pi[(size_t)s * nh + c] >= 0) return 1;
            pi[(size_t)s * nh + c] = p;
        }
    std::vector<int32_t> act(S, 1), rounds(S, 0);
    int32_t active = S;
    for (int32_t round = 0; round < max_rounds && active > 0; round++) {
        // k_pl_force
        std::vector<int64_t> F((size_t)S * np * 4, 0);
        for (int32_t s = 0; s < S; s++) {
            if (!act[s]) continue;
            const int32_t* gs = g + (int64_t)s * np;
            for (int64_t j = 0; j < P; j++) {
                int32_t a = hid[j], p = pins[j], h = gs[p];
                int32_t nb[4];
                neighbours(width, height, h, nb);
                int64_t f[4] = {0, 0, 0, 0};
                force_terms(pins, off[a], off[a + 1], gs, p, h, nb, width, f);
                for (int d = 0; d < 4; d++) F[((size_t)s * np + p) * 4 + d] += eta[a] * f[d];
            }
        }
        // k_pl_propose
        std::vector<int32_t> cand(V), match(V);
        std::vector<int64_t> cscore(V), props(S, 0), nsw(S, 0);
        for (int32_t s = 0; s < S; s++)
            for (int32_t h = 0; h < nh; h++) {
                int32_t x = s * nh + h;
                int64_t sc = 0;
                int32_t k = act[s] ? propose(width, height, &pi[(size_t)s * nh], &F[(size_t)s * np * 4],
                                             h, &sc)
                                   : -1;
                cand[x] = k < 0 ? -1 : s * nh + k;
                cscore[x] = sc;
                props[s] += k >= 0;
            }
        match_forest(V, cand, cscore, match);
        // k_pl_flag, k_pl_compact
        std::vector<Swap> sw;
        for (int32_t x = 0; x < V; x++) {
            if (match[x] <= x) continue;
            int32_t s = x / nh, h = x % nh, k = match[x] - s * nh;
            int d = direction(width, height, h, k);
            if (d < 0) return 2;
            int64_t t = tension(&pi[(size_t)s * nh], &F[(size_t)s * np * 4], h, k, d);
            if (t <= 0) return 2;
            sw.push_back({(uint64_t)INT64_MAX - (uint64_t)t, (uint32_t)x});
            nsw[s]++;
        }
        // the two stable sorts
        std::stable_sort(sw.begin(), sw.end(), [](const Swap& a, const Swap& b) { return a.key < b.key; });
        std::stable_sort(sw.begin(), sw.end(),
                         [nh](const Swap& a, const Swap& b) { return a.x / nh < b.x / nh; });
        std::vector<int32_t> segbeg(S, 0);
        for (int32_t s = 1; s < S; s++) segbeg[s] = segbeg[s - 1] + (int32_t)nsw[s - 1];
        // k_pl_rank
        std::vector<int32_t> rank(V, NO_RANK), mate(V, -1);
        for (size_t i = 0; i < sw.size(); i++) {
            int32_t x = (int32_t)sw[i].x, s = x / nh, y = match[x];
            int32_t r = (int32_t)i - segbeg[s];
            rank[x] = rank[y] = r;
            mate[x] = y - s * nh;
            mate[y] = x - s * nh;
        }
        // k_pl_reeval
        std::vector<int64_t> Tn(sw.size(), 0), C(sw.size(), 0);
        for (int32_t s = 0; s < S; s++) {
            const int32_t* gs = g + (int64_t)s * np;
            const int32_t* rs = &rank[(size_t)s * nh];
            const int32_t* ms = &mate[(size_t)s * nh];
            for (int64_t j = 0; j < P; j++) {
                int32_t p = pins[j], h = gs[p], r = rs[h];
                if (r == NO_RANK) continue;
                int32_t a = hid[j];
                Tn[segbeg[s] + r] += eta[a] * reeval_terms(pins, off[a], off[a + 1], gs, rs, ms, p, h,
                                                           ms[h], r, width);
            }
        }
        int64_t run = 0;
        for (size_t i = 0; i < sw.size(); i++) C[i] = run += Tn[i];
        // k_pl_best, k_pl_first
        std::vector<int64_t> best(S, 0), first(S, INT64_MAX);
        auto local = [&](size_t i, int32_t s) {
            return C[i] - (segbeg[s] > 0 ? C[segbeg[s] - 1] : 0);
        };
        for (size_t i = 0; i < sw.size(); i++) {
            int32_t s = (int32_t)(sw[i].x / nh);
            int64_t G = local(i, s);
            if (G > 0) best[s] = std::max(best[s], G);
        }
        for (size_t i = 0; i < sw.size(); i++) {
            int32_t s = (int32_t)(sw[i].x / nh);
            int64_t G = local(i, s);
            if (G > 0 && G == best[s]) first[s] = std::min(first[s], (int64_t)i - segbeg[s]);
        }
        // k_pl_apply
        for (size_t i = 0; i < sw.size(); i++) {
            int32_t x = (int32_t)sw[i].x, s = x / nh, y = match[x];
            if (first[s] == INT64_MAX || (int64_t)i - segbeg[s] > first[s]) continue;
            int32_t a = pi[x], b = pi[y];
            pi[x] = b;
            pi[y] = a;
            if (a >= 0) g[(int64_t)s * np + a] = y - s * nh;
            if (b >= 0) g[(int64_t)s * np + b] = x - s * nh;
        }
        for (int32_t s = 0; s < S; s++) {
            if (!act[s]) continue;
            int32_t applied = first[s] == INT64_MAX ? 0 : (int32_t)(first[s] + 1);
            int32_t r = rounds[s];
            if (r < log_cap) {
                size_t at = (size_t)s * log_cap + r;
                log_props[at] = (int32_t)props[s];
                log_swaps[at] = (int32_t)nsw[s];
                log_applied[at] = applied;
                log_gain[at] = applied ? best[s] : 0;
            }
            rounds[s]++;
            if (applied == 0) {
                act[s] = 0;
                active--;
            }
        }
    }
    for (int32_t s = 0; s < S; s++) rounds_out[s] = rounds[s];
    return 0;
}

// Same contract as snnmap_place_trd on host arrays.
void emul_place_trd(int32_t np, int32_t ne, const int64_t* off, const int32_t* pins,
                    const int64_t* eta, int32_t width, int32_t S, const int32_t* g, int64_t* out)
{
    for (int32_t s = 0; s < S; s++) {
        int64_t acc = 0;
        for (int32_t a = 0; a < ne; a++)
            for (int64_t j = off[a]; j < off[a + 1]; j++)
                acc += eta[a] * trd_terms(pins, j, off[a + 1], g + (int64_t)s * np, width);
        out[s] = acc;
    }
}

}  // extern "C"
