// Host run of the placement kernels' steps. Refinement: the per-item
// functions of csrc/place_items.cuh, called one item at a time in the phase
// order of the kernels in csrc/place.cu (forces summed per pin entry,
// proposals per core over all starts, Eq. matching in the matching kernels'
// formulation, swaps sorted by tension then by start, re-evaluation through
// ranks, per-start best prefix, apply). Initial placement: those of
// csrc/initial_items.cuh in the order of csrc/initial.cu (label propagation
// of all jobs of a depth in lockstep rounds through single-move gains and a
// correction matrix built once per depth and updated swap by swap, folding
// from the post-propagation section sets, Hilbert order). It checks those decompositions against the oracle without a GPU.
// Test infrastructure only; built by the tests.
#include "initial_items.cuh"
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


// Same contract as snnmap_place_initial on host arrays (seq_out and gamma:
// int32[S * np]). Returns 0 or 1 (invalid input).
int emul_place_initial(int32_t np, int32_t ne, const int64_t* off, const int32_t* pins,
                       const int64_t* eta, int32_t width, int32_t height, int32_t S,
                       const int32_t* seq0, int32_t* seq_out, int32_t* gamma)
{
    namespace ip = snn::initial;
    const int64_t P = off[ne];
    std::vector<int32_t> hid((size_t)P), deg(np, 0);
    for (int32_t a = 0; a < ne; a++)
        for (int64_t j = off[a]; j < off[a + 1]; j++) {
            hid[j] = a;
            for (int64_t t = j + 1; t < off[a + 1]; t++)
                if (pins[t] == pins[j]) return 1;
            deg[pins[j]]++;
        }
    std::vector<int64_t> voff(np + 1, 0);
    for (int32_t q = 0; q < np; q++) voff[q + 1] = voff[q] + deg[q];
    std::vector<int32_t> vinc((size_t)P), cur(np, 0);
    for (int64_t j = P - 1; j >= 0; j--) vinc[voff[pins[j]] + cur[pins[j]]++] = hid[j];   // any order
    std::vector<int32_t> seq((size_t)S * np), pos((size_t)S * np, -1);
    for (int64_t t = 0; t < (int64_t)S * np; t++) {
        int32_t q = seq0[t];
        int64_t s = t / np;
        if (q < 0 || q >= np || pos[s * np + q] >= 0) return 1;
        seq[t] = q;
        pos[s * np + q] = (int32_t)(t - s * np);
    }
    // the bisection tree
    std::vector<int32_t> lo{0}, hi{np}, par{-1}, kid{-1}, depth{0};
    for (size_t v = 0; v < lo.size(); v++) {
        int32_t len = hi[v] - lo[v];
        if (len <= 1) continue;
        int32_t mid = lo[v] + (len + 1) / 2;
        kid[v] = (int32_t)lo.size();
        lo.push_back(lo[v]); hi.push_back(mid); par.push_back((int32_t)v); kid.push_back(-1);
        depth.push_back(depth[v] + 1);
        lo.push_back(mid); hi.push_back(hi[v]); par.push_back((int32_t)v); kid.push_back(-1);
        depth.push_back(depth[v] + 1);
    }
    const int32_t nn = (int32_t)lo.size();
    int32_t maxd = 0;
    for (int32_t v = 0; v < nn; v++) maxd = std::max(maxd, depth[v]);
    std::vector<int64_t> G((size_t)S * np, 0);
    for (int32_t d = 0; d <= maxd; d++) {
        std::vector<int32_t> js;
        for (int32_t v = 0; v < nn; v++)
            if (depth[v] == d && kid[v] >= 0) js.push_back(v);
        const int32_t J = (int32_t)js.size();
        if (!J) continue;
        std::vector<int32_t> jlo(J), jmid(J), jhi(J), jcap(J), jobof(np, -1);
        std::vector<int64_t> po(J + 1, 0);
        for (int32_t k = 0; k < J; k++) {
            int32_t v = js[k], len = hi[v] - lo[v], nl = (len + 1) / 2, nr = len - nl;
            jlo[k] = lo[v]; jmid[k] = lo[v] + nl; jhi[k] = hi[v];
            jcap[k] = 4 * std::min(nl, nr);
            po[k + 1] = po[k] + (int64_t)nl * nr;
            for (int32_t i = lo[v]; i < hi[v]; i++) jobof[i] = k;
        }
        const int64_t pairs = po[J];
        std::vector<int32_t> done((size_t)S * J, 0), it((size_t)S * J, 0), bx((size_t)S * J),
            by((size_t)S * J);
        std::vector<int64_t> bd((size_t)S * J), M((size_t)S * pairs);
        // k_ip_gain, k_ip_corr: once per depth
        for (int32_t s = 0; s < S; s++)
            for (int32_t i = 0; i < np; i++) {
                int32_t k = jobof[i];
                if (k < 0) continue;
                int32_t x = seq[(size_t)s * np + i];
                G[(size_t)s * np + x] = ip::single_gain(
                    vinc.data(), voff[x], voff[x + 1], off, pins, eta, &pos[(size_t)s * np],
                    ip::side_of(i, jlo[k], jmid[k], jhi[k]), jlo[k], jmid[k], jhi[k]);
            }
        std::fill(M.begin(), M.end(), 0);
        for (int32_t s = 0; s < S; s++)
            for (int32_t i = 0; i < np; i++) {
                int32_t k = jobof[i];
                if (k < 0 || i >= jmid[k]) continue;
                int32_t x = seq[(size_t)s * np + i], nr = jhi[k] - jmid[k];
                int64_t* row = &M[(size_t)s * pairs + po[k] + (int64_t)(i - jlo[k]) * nr];
                ip::corr_row(vinc.data(), voff[x], voff[x + 1], off, pins, eta,
                             &pos[(size_t)s * np], jlo[k], jmid[k], jhi[k],
                             [row](int32_t j, int64_t w) { row[j] += w; });
            }
        for (;;) {
            for (size_t t = 0; t < done.size(); t++)
                if (!done[t]) { bd[t] = 0; bx[t] = INT32_MAX; by[t] = INT32_MAX; }
            // k_ip_best, three passes
            for (int pass = 0; pass < 3; pass++)
                for (int32_t s = 0; s < S; s++)
                    for (int32_t k = 0; k < J; k++) {
                        size_t t = (size_t)s * J + k;
                        if (done[t]) continue;
                        int32_t nr = jhi[k] - jmid[k];
                        for (int64_t q = 0; q < po[k + 1] - po[k]; q++) {
                            int32_t x = seq[(size_t)s * np + jlo[k] + q / nr];
                            int32_t y = seq[(size_t)s * np + jmid[k] + q % nr];
                            int64_t dd = G[(size_t)s * np + x] + G[(size_t)s * np + y] -
                                         M[(size_t)s * pairs + po[k] + q];
                            if (dd <= 0) continue;
                            if (pass == 0) bd[t] = std::max(bd[t], dd);
                            else if (pass == 1 && dd == bd[t]) bx[t] = std::min(bx[t], x);
                            else if (pass == 2 && dd == bd[t] && x == bx[t]) by[t] = std::min(by[t], y);
                        }
                    }
            // k_ip_update
            int active = 0;
            for (int32_t s = 0; s < S; s++)
                for (int32_t k = 0; k < J; k++) {
                    size_t t = (size_t)s * J + k;
                    if (done[t]) continue;
                    if (bd[t] <= 0) { done[t] = 1; continue; }
                    bool last = it[t] + 1 >= jcap[k];
                    const int32_t lo = jlo[k], mid = jmid[k], hi = jhi[k], nr = hi - mid;
                    int32_t* ps = &pos[(size_t)s * np];
                    int32_t* qs = &seq[(size_t)s * np];
                    int64_t* Gs = &G[(size_t)s * np];
                    int64_t* Mk = &M[(size_t)s * pairs + po[k]];
                    int32_t x = bx[t], y = by[t], px = ps[x], py = ps[y];
                    if (!last) {
                        auto gadd = [Gs](int32_t v, int64_t d) { Gs[v] += d; };
                        auto madd = [Mk, nr](int32_t i, int32_t j, int64_t d) {
                            Mk[(int64_t)i * nr + j] += d;
                        };
                        for (int64_t u = voff[x]; u < voff[x + 1]; u++) {
                            int32_t a = vinc[u];
                            ip::swap_hedge_update(pins, off[a], off[a + 1], ps, lo, mid, hi, x, y,
                                                  eta[a], false, gadd, madd);
                        }
                        for (int64_t u = voff[y]; u < voff[y + 1]; u++) {
                            int32_t a = vinc[u];
                            ip::swap_hedge_update(pins, off[a], off[a + 1], ps, lo, mid, hi, x, y,
                                                  eta[a], true, gadd, madd);
                        }
                    }
                    qs[px] = y; qs[py] = x; ps[x] = py; ps[y] = px;
                    it[t]++;
                    if (last) { done[t] = 1; continue; }
                    active++;
                    int64_t* row = Mk + (int64_t)(px - lo) * nr;
                    int64_t* col = Mk + (py - mid);
                    for (int32_t j = 0; j < nr; j++) row[j] = 0;
                    for (int32_t i = 0; i < mid - lo; i++) col[(int64_t)i * nr] = 0;
                    ip::corr_row(vinc.data(), voff[y], voff[y + 1], off, pins, eta, ps, lo, mid, hi,
                                 [row](int32_t j, int64_t w) { row[j] += w; });
                    ip::corr_col(vinc.data(), voff[x], voff[x + 1], off, pins, eta, ps, lo, mid, hi,
                                 y, [col, nr](int32_t i, int64_t w) { col[(int64_t)i * nr] += w; });
                }
            if (!active) break;
        }
    }
    // k_ip_conn, k_ip_flip, k_ip_fold
    std::vector<int64_t> conn((size_t)S * nn, 0);
    std::vector<uint8_t> flip((size_t)S * nn, 0);
    for (int32_t s = 0; s < S; s++) {
        const int32_t* ps = &pos[(size_t)s * np];
        for (int64_t j = 0; j < P; j++) {
            int32_t a = hid[j], i = ps[pins[j]], v = 0;
            while (kid[v] >= 0) {
                int32_t c = ip::child_holding(lo.data(), hi.data(), kid.data(), v, i);
                int32_t p = par[v];
                if (p >= 0) {
                    int32_t sib = kid[p] == v ? kid[p] + 1 : kid[p];
                    bool first, meets;
                    ip::fold_checks(pins, off[a], off[a + 1], ps, j, lo[c], hi[c], lo[sib], hi[sib],
                                    &first, &meets);
                    if (first && meets) conn[(size_t)s * nn + c] += eta[a];
                }
                v = c;
            }
        }
        for (int32_t v = 0; v < nn; v++) {
            int32_t p = par[v];
            if (kid[v] < 0 || p < 0) continue;
            int64_t ca = conn[(size_t)s * nn + kid[v]], cb = conn[(size_t)s * nn + kid[v] + 1];
            flip[(size_t)s * nn + v] = kid[p] == v ? (ca > cb) : (cb > ca);
        }
        for (int32_t i = 0; i < np; i++)
            seq_out[(size_t)s * np +
                    ip::folded_position(lo.data(), hi.data(), kid.data(), &flip[(size_t)s * nn], i)] =
                seq[(size_t)s * np + i];
    }
    // k_ip_hkeys + sort, k_ip_gamma
    uint32_t n2 = 1;
    while (n2 < (uint32_t)width || n2 < (uint32_t)height) n2 <<= 1;
    std::vector<std::pair<uint64_t, int32_t>> cells;
    for (int32_t h = 0; h < width * height; h++)
        cells.push_back({ip::hilbert_index(n2, (uint32_t)(h % width), (uint32_t)(h / width)), h});
    std::stable_sort(cells.begin(), cells.end(),
                     [](const std::pair<uint64_t, int32_t>& a, const std::pair<uint64_t, int32_t>& b) {
                         return a.first < b.first;
                     });
    for (int32_t s = 0; s < S; s++)
        for (int32_t i = 0; i < np; i++) gamma[(size_t)s * np + seq_out[(size_t)s * np + i]] = cells[i].second;
    return 0;
}

}  // extern "C"
