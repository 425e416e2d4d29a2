/*
 * CPU oracle for the multilevel hypergraph partitioning pass of Ronzani &
 * Silvano, "GPU-Accelerated Hypergraph Partitioning and Placement to Map SNNs
 * on Neuromorphic Hardware", Sec. 4.1 (Partitioning).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, single-threaded
 * statement of what the partitioning pass computes. Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it. It
 * shares no code, header, table or helper with the CUDA implementation.
 *
 * Everything is integer: weights and scores are summed in int64, so the
 * order of summation cannot change any result.
 *
 * Readings of points the paper leaves open (each one is marked where used):
 *  R1  "tie-breaking by node id" (Eq. neigh_histogram): the lower id wins.
 *  R2  Eq. matching, second case: among children of equal score, the lower id.
 *  R3  Weights are integers (omega in the paper is real-valued).
 *  R4  Delta counts distinct original axons; a coarse hyperedge carries the
 *      multiplicity k = number of original axons merged into it.
 *  R5  A coarse hyperedge keeps a flag selfdst = "some merged axon has a
 *      destination inside the source super-node"; the inbound test of the
 *      paper (pins(p,e) - [src(e) in p] > 0) becomes "some destination of e
 *      lies in p".
 *  R6  A hyperedge whose pins all fall in one super-node is dropped; its k is
 *      kept in the super-node's in_internal count.
 *  R7  Coarse vertex c is numbered by ascending minimum member id; coarse
 *      hyperedges are stored in a canonical order (source, selfdst, size,
 *      destination list), which no result depends on.
 *  R8  Coarsening stops when no vertex has a candidate, or after
 *      max_levels contractions.
 *  R9  A vertex proposes its best feasible move to an adjacent partition,
 *      only if its gain is positive; ties go to the lower partition id.
 *  R10 Moves are sorted by decreasing gain, ties by increasing vertex id.
 *  R11 The enacted prefix is the valid prefix with the largest positive
 *      cumulative gain; ties go to the shortest prefix.
 *  R12 Refinement rounds repeat until none enacts a move, at most
 *      max_refine_rounds per level.
 *  R13 Validity is evaluated after each whole move.
 *  R14 Refinement also runs on the coarsest level.
 *  R15 Partitions may end up empty; ids are those of the coarsest vertices.
 *  R19 Variant (refine_nonpositive = 1): every vertex with a feasible move
 *      to an adjacent partition proposes its best one (max gain, lower
 *      partition id) whatever the sign of its gain; a non-positive move can
 *      still belong to an enacted prefix, whose cumulative gain and
 *      validity are judged with every earlier move applied.
 *  R18 G_P (Sec. 3): the image of an axon keeps its direction: source
 *      partition rho(src), destinations the other partitions of its pins
 *      (a destination inside the source's partition is discarded). Axons
 *      with equal (source, destination set) merge and eta sums their
 *      omega; an axon left without destination is not in A and its omega
 *      counts as internal weight.
 *
 * Error codes: 0 ok, 1 invalid input, 2 infeasible (one neuron alone breaks
 * a limit), 3 out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_INFEASIBLE 2
#define ORC_ERR_OOM 3

typedef struct {
    int32_t omega;              /* max neurons per core (Omega, Sec. 2) */
    int32_t delta;              /* max distinct inbound axons per core (Delta) */
    int32_t phi;                /* max inbound synapses per core (Phi) */
    int32_t max_levels;         /* R8 */
    int32_t max_refine_rounds;  /* R12 */
    int32_t refine_nonpositive; /* R19: 1 = propose the best feasible move whatever its gain */
} orc_params;

/* One level of the hierarchy (Sec. 4.1: "each level's hgraph is
 * materialized from its predecessor while propagating each super-node's
 * constrained state"). */
typedef struct {
    int32_t V, E;
    int64_t P;
    int64_t *off;        /* E+1: pins of hyperedge a are pins[off[a]..off[a+1]) */
    int32_t *pins;       /* pins[off[a]] = source; then destinations ascending */
    int64_t *w;          /* E: summed spike frequency (omega(e)) */
    int32_t *k;          /* E: number of original axons merged (R4) */
    uint8_t *selfdst;    /* E: R5 */
    int32_t *size;       /* V: neurons in the super-node */
    int32_t *inpins;     /* V: sum over member neurons of |in(n)| (Phi weight) */
    int32_t *in_count;   /* V: |union of in(n)| over members, original axons (Delta weight) */
    int32_t *in_internal;/* V: original axons with every pin inside the super-node (R6) */
    int64_t *voff;       /* V+1: incidence lists */
    int32_t *vinc;       /* P: hyperedges incident to each vertex, ascending */
} orc_level;

typedef struct {
    int32_t level, round, n_props, istar;
    int64_t gain;
} orc_round_log;

typedef struct {
    int32_t V, E;
    int64_t P;
    int32_t n_cand, n_pairs;
} orc_level_log;

typedef struct {
    int32_t levels;          /* contractions performed */
    int32_t n_parts;         /* K = vertices of the coarsest level */
    int32_t nonempty_parts;
    int32_t rounds;          /* refinement rounds that enacted moves */
    int64_t moves;           /* moves enacted in total */
    int64_t cost_initial;    /* Conn at the coarsest level before refinement */
    int64_t cost;            /* final Conn */
} orc_stats;

/* ------------------------------------------------------------------------ */

static void level_free(orc_level *L)
{
    if (!L) return;
    free(L->off); free(L->pins); free(L->w); free(L->k); free(L->selfdst);
    free(L->size); free(L->inpins); free(L->in_count); free(L->in_internal);
    free(L->voff); free(L->vinc);
    free(L);
}

void orc_free(orc_level *L) { level_free(L); }

static orc_level *level_alloc(int32_t V, int32_t E, int64_t P)
{
    orc_level *L = (orc_level *)calloc(1, sizeof(orc_level));
    if (!L) return NULL;
    L->V = V; L->E = E; L->P = P;
    L->off = (int64_t *)calloc((size_t)E + 1, sizeof(int64_t));
    L->pins = (int32_t *)calloc((size_t)P + 1, sizeof(int32_t));
    L->w = (int64_t *)calloc((size_t)E + 1, sizeof(int64_t));
    L->k = (int32_t *)calloc((size_t)E + 1, sizeof(int32_t));
    L->selfdst = (uint8_t *)calloc((size_t)E + 1, 1);
    L->size = (int32_t *)calloc((size_t)V + 1, sizeof(int32_t));
    L->inpins = (int32_t *)calloc((size_t)V + 1, sizeof(int32_t));
    L->in_count = (int32_t *)calloc((size_t)V + 1, sizeof(int32_t));
    L->in_internal = (int32_t *)calloc((size_t)V + 1, sizeof(int32_t));
    L->voff = (int64_t *)calloc((size_t)V + 1, sizeof(int64_t));
    L->vinc = (int32_t *)calloc((size_t)P + 1, sizeof(int32_t));
    if (!L->off || !L->pins || !L->w || !L->k || !L->selfdst || !L->size || !L->inpins ||
        !L->in_count || !L->in_internal || !L->voff || !L->vinc) {
        level_free(L);
        return NULL;
    }
    return L;
}

/* n is a destination of hyperedge a (R5): a listed destination, or the
 * source itself when some merged axon ends inside it. */
static int is_dest(const orc_level *L, int32_t a, int32_t n)
{
    return n != L->pins[L->off[a]] || L->selfdst[a];
}

/* Incidence lists I(n) of Sec. 2, in ascending hyperedge order. */
static int build_incidence(orc_level *L)
{
    int32_t V = L->V;
    int64_t *fill;
    memset(L->voff, 0, ((size_t)V + 1) * sizeof(int64_t));
    for (int32_t a = 0; a < L->E; a++)
        for (int64_t j = L->off[a]; j < L->off[a + 1]; j++)
            L->voff[L->pins[j] + 1]++;
    for (int32_t n = 0; n < V; n++) L->voff[n + 1] += L->voff[n];
    fill = (int64_t *)malloc(((size_t)V + 1) * sizeof(int64_t));
    if (!fill) return ORC_ERR_OOM;
    memcpy(fill, L->voff, ((size_t)V + 1) * sizeof(int64_t));
    for (int32_t a = 0; a < L->E; a++)
        for (int64_t j = L->off[a]; j < L->off[a + 1]; j++)
            L->vinc[fill[L->pins[j]]++] = a;
    free(fill);
    return ORC_OK;
}

static int cmp_i32(const void *x, const void *y)
{
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* ------------------------------------------------------------------------ */
/* Level 0 from the SNN (Sec. 2): one vertex per neuron, one hyperedge per
 * axon with pin 0 its source and the rest its destinations. Hyperedges with
 * no destination are dropped (they can never be cut). Vertex state:
 * size 1, inpins = in_count = |in(n)|, in_internal = 0. A neuron that alone
 * exceeds Phi or Delta makes the problem infeasible. */
int orc_build(const orc_params *prm, int32_t V, int32_t E, const int64_t *off,
              const int32_t *pins, const int32_t *w, orc_level **out)
{
    int32_t Ek = 0;
    int64_t Pk = 0, maxlen = 0;
    int32_t *tmp;
    orc_level *L;
    *out = NULL;
    if (!prm || prm->omega < 1 || prm->delta < 0 || prm->phi < 0 || prm->max_levels < 0 ||
        prm->max_refine_rounds < 0 || V < 0 || E < 0)
        return ORC_ERR_INVALID;
    if (off[0] != 0) return ORC_ERR_INVALID;
    for (int32_t a = 0; a < E; a++) {
        int64_t len = off[a + 1] - off[a];
        if (len < 1) return ORC_ERR_INVALID;
        if (w[a] < 0) return ORC_ERR_INVALID;
        if (len > maxlen) maxlen = len;
    }
    tmp = (int32_t *)malloc(((size_t)maxlen + 1) * sizeof(int32_t));
    if (!tmp) return ORC_ERR_OOM;
    for (int32_t a = 0; a < E; a++) {
        int64_t len = off[a + 1] - off[a];
        int32_t s = pins[off[a]];
        for (int64_t j = 0; j < len; j++) {
            int32_t q = pins[off[a] + j];
            if (q < 0 || q >= V) { free(tmp); return ORC_ERR_INVALID; }
            tmp[j] = q;
        }
        /* destinations must be distinct and differ from the source */
        qsort(tmp + 1, (size_t)(len - 1), sizeof(int32_t), cmp_i32);
        for (int64_t j = 1; j < len; j++) {
            if (tmp[j] == s || (j > 1 && tmp[j] == tmp[j - 1])) { free(tmp); return ORC_ERR_INVALID; }
        }
        if (len > 1) { Ek++; Pk += len; }
    }
    L = level_alloc(V, Ek, Pk);
    if (!L) { free(tmp); return ORC_ERR_OOM; }
    {
        int32_t e = 0;
        int64_t pos = 0;
        for (int32_t a = 0; a < E; a++) {
            int64_t len = off[a + 1] - off[a];
            if (len < 2) continue;
            L->off[e] = pos;
            L->pins[pos] = pins[off[a]];
            memcpy(L->pins + pos + 1, pins + off[a] + 1, (size_t)(len - 1) * sizeof(int32_t));
            qsort(L->pins + pos + 1, (size_t)(len - 1), sizeof(int32_t), cmp_i32);
            L->w[e] = w[a];
            L->k[e] = 1;
            L->selfdst[e] = 0;
            pos += len;
            e++;
        }
        L->off[Ek] = pos;
    }
    free(tmp);
    for (int32_t n = 0; n < V; n++) {
        L->size[n] = 1;
        L->inpins[n] = 0;
        L->in_internal[n] = 0;
    }
    for (int32_t a = 0; a < L->E; a++)
        for (int64_t j = L->off[a] + 1; j < L->off[a + 1]; j++)
            L->inpins[L->pins[j]]++;
    for (int32_t n = 0; n < V; n++) L->in_count[n] = L->inpins[n];
    if (build_incidence(L) != ORC_OK) { level_free(L); return ORC_ERR_OOM; }
    for (int32_t n = 0; n < V; n++) {
        if ((int64_t)L->inpins[n] > prm->phi || (int64_t)L->in_count[n] > prm->delta) {
            level_free(L);
            return ORC_ERR_INFEASIBLE;
        }
    }
    *out = L;
    return ORC_OK;
}

void orc_level_dims(const orc_level *L, int32_t *V, int32_t *E, int64_t *P)
{
    *V = L->V; *E = L->E; *P = L->P;
}

void orc_level_copy(const orc_level *L, int64_t *off, int32_t *pins, int64_t *w, int32_t *k,
                    uint8_t *selfdst, int32_t *size, int32_t *inpins, int32_t *in_count,
                    int32_t *in_internal)
{
    memcpy(off, L->off, ((size_t)L->E + 1) * sizeof(int64_t));
    memcpy(pins, L->pins, (size_t)L->P * sizeof(int32_t));
    memcpy(w, L->w, (size_t)L->E * sizeof(int64_t));
    memcpy(k, L->k, (size_t)L->E * sizeof(int32_t));
    memcpy(selfdst, L->selfdst, (size_t)L->E);
    memcpy(size, L->size, (size_t)L->V * sizeof(int32_t));
    memcpy(inpins, L->inpins, (size_t)L->V * sizeof(int32_t));
    memcpy(in_count, L->in_count, (size_t)L->V * sizeof(int32_t));
    memcpy(in_internal, L->in_internal, (size_t)L->V * sizeof(int32_t));
}

/* ------------------------------------------------------------------------ */
/* Coarsening, neighbour histogram (Eq. neigh_histogram): for n, every
 * neighbour m accumulates score(n,m) = sum of omega(e) over hyperedges e
 * incident to n that contain m, and the shared inbound count
 * |in(n) & in(m)| (each coarse hyperedge in which both are destinations
 * contributes its k, R4/R5). Neighbours that break Omega, Phi, or Delta on
 * the merged inbound set are discarded; cand(n) is the valid maximum, ties
 * to the lower id (R1). No valid neighbour: cand = -1, score = ov = 0. */

typedef struct {
    int64_t *score, *ov;
    uint8_t *seen;
    int32_t *list;
} spa;

static int spa_init(spa *s, int32_t n)
{
    s->score = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    s->ov = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    s->seen = (uint8_t *)calloc((size_t)n + 1, 1);
    s->list = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!s->score || !s->ov || !s->seen || !s->list) {
        free(s->score); free(s->ov); free(s->seen); free(s->list);
        return ORC_ERR_OOM;
    }
    return ORC_OK;
}

static void spa_free(spa *s)
{
    free(s->score); free(s->ov); free(s->seen); free(s->list);
}

static int pair_valid(const orc_level *L, const orc_params *prm, int32_t n, int32_t m, int64_t ov)
{
    return (int64_t)L->size[n] + L->size[m] <= prm->omega &&
           (int64_t)L->inpins[n] + L->inpins[m] <= prm->phi &&
           (int64_t)L->in_count[n] + L->in_count[m] - ov <= prm->delta;
}

static void cand_of(const orc_level *L, const orc_params *prm, spa *s, int32_t n,
                    int32_t *cand, int64_t *cscore, int32_t *cov)
{
    int32_t cnt = 0, best = -1;
    int64_t bs = 0, bo = 0;
    for (int64_t i = L->voff[n]; i < L->voff[n + 1]; i++) {
        int32_t a = L->vinc[i];
        int nd = is_dest(L, a, n);
        for (int64_t j = L->off[a]; j < L->off[a + 1]; j++) {
            int32_t m = L->pins[j];
            if (m == n) continue;
            if (!s->seen[m]) {
                s->seen[m] = 1;
                s->score[m] = 0;
                s->ov[m] = 0;
                s->list[cnt++] = m;
            }
            s->score[m] += L->w[a];
            if (nd && is_dest(L, a, m)) s->ov[m] += L->k[a];
        }
    }
    for (int32_t i = 0; i < cnt; i++) {
        int32_t m = s->list[i];
        s->seen[m] = 0;
        if (!pair_valid(L, prm, n, m, s->ov[m])) continue;
        if (best < 0 || s->score[m] > bs || (s->score[m] == bs && m < best)) {
            best = m;
            bs = s->score[m];
            bo = s->ov[m];
        }
    }
    *cand = best;
    *cscore = best < 0 ? 0 : bs;
    *cov = best < 0 ? 0 : (int32_t)bo;
}

int orc_affinity(const orc_level *L, const orc_params *prm, int32_t *cand, int64_t *cscore,
                 int32_t *cov)
{
    spa s;
    if (spa_init(&s, L->V) != ORC_OK) return ORC_ERR_OOM;
    for (int32_t n = 0; n < L->V; n++) cand_of(L, prm, &s, n, cand + n, cscore + n, cov + n);
    spa_free(&s);
    return ORC_OK;
}

/* One vertex only, by sorting its (neighbour, weight, overlap) terms: used to
 * spot-check vertices of hypergraphs too large for a full oracle run. */
typedef struct { int32_t m; int32_t k; int64_t w; } term;

static int cmp_term(const void *x, const void *y)
{
    const term *a = (const term *)x, *b = (const term *)y;
    return (a->m > b->m) - (a->m < b->m);
}

int orc_cand_one(const orc_level *L, const orc_params *prm, int32_t n, int32_t *cand,
                 int64_t *cscore, int32_t *cov)
{
    int64_t nt = 0, t = 0;
    term *T;
    int32_t best = -1;
    int64_t bs = 0, bo = 0;
    for (int64_t i = L->voff[n]; i < L->voff[n + 1]; i++) {
        int32_t a = L->vinc[i];
        nt += L->off[a + 1] - L->off[a];
    }
    T = (term *)malloc(((size_t)nt + 1) * sizeof(term));
    if (!T) return ORC_ERR_OOM;
    for (int64_t i = L->voff[n]; i < L->voff[n + 1]; i++) {
        int32_t a = L->vinc[i];
        int nd = is_dest(L, a, n);
        for (int64_t j = L->off[a]; j < L->off[a + 1]; j++) {
            int32_t m = L->pins[j];
            if (m == n) continue;
            T[t].m = m;
            T[t].w = L->w[a];
            T[t].k = (nd && is_dest(L, a, m)) ? L->k[a] : 0;
            t++;
        }
    }
    qsort(T, (size_t)t, sizeof(term), cmp_term);
    for (int64_t i = 0; i < t;) {
        int64_t sc = 0, ov = 0, j = i;
        while (j < t && T[j].m == T[i].m) { sc += T[j].w; ov += T[j].k; j++; }
        if (pair_valid(L, prm, n, T[i].m, ov) &&
            (best < 0 || sc > bs || (sc == bs && T[i].m < best))) {
            best = T[i].m; bs = sc; bo = ov;
        }
        i = j;
    }
    free(T);
    *cand = best;
    *cscore = best < 0 ? 0 : bs;
    *cov = best < 0 ? 0 : (int32_t)bo;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Matching (Eq. matching). The candidate graph is a pseudo-forest rooted at
 * two-cycles, or at nodes without a candidate that others point to (never in
 * coarsening, where validity is symmetric; empty cores in placement). By the
 * second case of the equation such a root takes its best child. Evaluated
 * top-down in synchronous rounds by depth: the two
 * nodes of each root two-cycle match each other; then every node of depth d
 * that is still free (not taken by its parent) takes its best child, the
 * child m with cand(m) = n of highest score(n, m) = cscore(m), ties to the
 * lower id (R2). Returns the number of matched pairs, or -1 if some node with
 * a candidate is not reached from a root (no such graph should exist). */
int32_t orc_match(int32_t V, const int32_t *cand, const int64_t *cscore, int32_t *match)
{
    int64_t *coff = (int64_t *)calloc((size_t)V + 1, sizeof(int64_t));
    int32_t *child = (int32_t *)malloc(((size_t)V + 1) * sizeof(int32_t));
    int32_t *front = (int32_t *)malloc(((size_t)V + 1) * sizeof(int32_t));
    int32_t *next = (int32_t *)malloc(((size_t)V + 1) * sizeof(int32_t));
    uint8_t *reached = (uint8_t *)calloc((size_t)V + 1, 1);
    int32_t nf = 0, pairs = 0;
    if (!coff || !child || !front || !next || !reached) {
        free(coff); free(child); free(front); free(next); free(reached);
        return -2;
    }
    for (int32_t n = 0; n < V; n++) match[n] = -1;
    for (int32_t n = 0; n < V; n++)
        if (cand[n] >= 0) coff[cand[n] + 1]++;
    for (int32_t n = 0; n < V; n++) coff[n + 1] += coff[n];
    {
        int64_t *fill = (int64_t *)malloc(((size_t)V + 1) * sizeof(int64_t));
        if (!fill) { free(coff); free(child); free(front); free(next); free(reached); return -2; }
        memcpy(fill, coff, ((size_t)V + 1) * sizeof(int64_t));
        for (int32_t n = 0; n < V; n++)
            if (cand[n] >= 0) child[fill[cand[n]]++] = n;
        free(fill);
    }
    /* depth 0: the root two-cycles */
    for (int32_t n = 0; n < V; n++) {
        if (cand[n] >= 0 && cand[cand[n]] == n) {
            match[n] = cand[n];
            reached[n] = 1;
            front[nf++] = n;
            if (n < cand[n]) pairs++;
        } else if (cand[n] < 0 && coff[n + 1] > coff[n]) {
            reached[n] = 1;            /* a free root */
            front[nf++] = n;
        }
    }
    while (nf > 0) {
        int32_t nn = 0;
        for (int32_t i = 0; i < nf; i++) {
            int32_t x = front[i];
            if (match[x] < 0) {
                int32_t best = -1;
                for (int64_t j = coff[x]; j < coff[x + 1]; j++) {
                    int32_t c = child[j];
                    if (best < 0 || cscore[c] > cscore[best] || (cscore[c] == cscore[best] && c < best))
                        best = c;
                }
                if (best >= 0) {
                    match[x] = best;
                    match[best] = x;
                    pairs++;
                }
            }
        }
        for (int32_t i = 0; i < nf; i++) {
            int32_t x = front[i];
            for (int64_t j = coff[x]; j < coff[x + 1]; j++) {
                int32_t c = child[j];
                if (reached[c]) continue; /* the root partner */
                reached[c] = 1;
                next[nn++] = c;
            }
        }
        memcpy(front, next, (size_t)nn * sizeof(int32_t));
        nf = nn;
    }
    for (int32_t n = 0; n < V; n++)
        if (cand[n] >= 0 && !reached[n]) pairs = -1;
    free(coff); free(child); free(front); free(next); free(reached);
    return pairs;
}

/* ------------------------------------------------------------------------ */
/* Contraction (Sec. 4.1: "each level's hgraph is materialized from its
 * predecessor"). Super-node of a matched pair {n, m}: numbered by ascending
 * minimum member (R7); size, inpins and in_internal add up, and in_count is
 * the size of the merged inbound set, in_count(n) + in_count(m) - ov(n, m).
 * Every hyperedge is mapped through cid: source s' = cid(s); destinations
 * D' = distinct cid(d) other than s'; selfdst' = selfdst or s' in cid(D).
 * If D' is empty the hyperedge is dropped and its k added to in_internal(s')
 * (R6). Hyperedges with equal (s', selfdst', D') merge: omega and k add up. */

static const int32_t *g_pool;   /* comparator context (single-threaded) */
typedef struct { int32_t s, sd, len; int64_t start, w; int64_t k; } hrec;

static int cmp_hrec(const void *x, const void *y)
{
    const hrec *a = (const hrec *)x, *b = (const hrec *)y;
    if (a->s != b->s) return a->s < b->s ? -1 : 1;
    if (a->sd != b->sd) return a->sd < b->sd ? -1 : 1;
    if (a->len != b->len) return a->len < b->len ? -1 : 1;
    for (int32_t i = 0; i < a->len; i++) {
        int32_t u = g_pool[a->start + i], v = g_pool[b->start + i];
        if (u != v) return u < v ? -1 : 1;
    }
    return 0;
}

int orc_contract(const orc_level *L, const int32_t *match, const int32_t *cand, const int32_t *cov,
                 int32_t *cid, orc_level **out)
{
    int32_t V = L->V, V2 = 0, nrec = 0;
    int32_t *pool = NULL, *tmp = NULL;
    hrec *rec = NULL;
    int32_t *internal = NULL;
    int64_t poolpos = 0, maxlen = 0, P2 = 0;
    int32_t E2 = 0;
    orc_level *C;
    *out = NULL;
    for (int32_t n = 0; n < V; n++)
        if (match[n] < 0 || n < match[n]) cid[n] = V2++;
    for (int32_t n = 0; n < V; n++)
        if (match[n] >= 0 && n > match[n]) cid[n] = cid[match[n]];
    for (int32_t a = 0; a < L->E; a++)
        if (L->off[a + 1] - L->off[a] > maxlen) maxlen = L->off[a + 1] - L->off[a];
    pool = (int32_t *)malloc(((size_t)L->P + 1) * sizeof(int32_t));
    tmp = (int32_t *)malloc(((size_t)maxlen + 1) * sizeof(int32_t));
    rec = (hrec *)malloc(((size_t)L->E + 1) * sizeof(hrec));
    internal = (int32_t *)calloc((size_t)V2 + 1, sizeof(int32_t));
    if (!pool || !tmp || !rec || !internal) goto oom;
    for (int32_t a = 0; a < L->E; a++) {
        int32_t s2 = cid[L->pins[L->off[a]]];
        int32_t nd = 0, sd = L->selfdst[a], len = 0;
        for (int64_t j = L->off[a] + 1; j < L->off[a + 1]; j++) tmp[nd++] = cid[L->pins[j]];
        qsort(tmp, (size_t)nd, sizeof(int32_t), cmp_i32);
        for (int32_t i = 0; i < nd; i++) {
            if (i > 0 && tmp[i] == tmp[i - 1]) continue;
            if (tmp[i] == s2) { sd = 1; continue; }
            pool[poolpos + len++] = tmp[i];
        }
        if (len == 0) {
            /* every pin inside s': the axons become internal to it; they
             * always have a destination there (sd is set) */
            if (sd) internal[s2] += L->k[a];
            continue;
        }
        rec[nrec].s = s2; rec[nrec].sd = sd; rec[nrec].len = len;
        rec[nrec].start = poolpos; rec[nrec].w = L->w[a]; rec[nrec].k = L->k[a];
        nrec++;
        poolpos += len;
    }
    g_pool = pool;
    qsort(rec, (size_t)nrec, sizeof(hrec), cmp_hrec);
    /* merge equal neighbours */
    {
        int32_t i = 0;
        while (i < nrec) {
            int32_t j = i + 1;
            while (j < nrec && cmp_hrec(&rec[i], &rec[j]) == 0) {
                rec[i].w += rec[j].w;
                rec[i].k += rec[j].k;
                j++;
            }
            rec[E2] = rec[i];
            E2++;
            P2 += 1 + rec[i].len;
            i = j;
        }
    }
    C = level_alloc(V2, E2, P2);
    if (!C) goto oom;
    {
        int64_t pos = 0;
        for (int32_t e = 0; e < E2; e++) {
            C->off[e] = pos;
            C->pins[pos++] = rec[e].s;
            memcpy(C->pins + pos, pool + rec[e].start, (size_t)rec[e].len * sizeof(int32_t));
            pos += rec[e].len;
            C->w[e] = rec[e].w;
            C->k[e] = (int32_t)rec[e].k;
            C->selfdst[e] = (uint8_t)rec[e].sd;
        }
        C->off[E2] = pos;
    }
    for (int32_t n = 0; n < V; n++) {
        int32_t c = cid[n];
        C->size[c] += L->size[n];
        C->inpins[c] += L->inpins[n];
        C->in_internal[c] += L->in_internal[n];
        if (match[n] < 0) {
            C->in_count[c] = L->in_count[n];
        } else if (n < match[n]) {
            int32_t m = match[n];
            int32_t ov = cand[n] == m ? cov[n] : cov[m];
            C->in_count[c] = L->in_count[n] + L->in_count[m] - ov;
        }
    }
    for (int32_t c = 0; c < V2; c++) C->in_internal[c] += internal[c];
    if (build_incidence(C) != ORC_OK) { level_free(C); goto oom; }
    free(pool); free(tmp); free(rec); free(internal);
    *out = C;
    return ORC_OK;
oom:
    free(pool); free(tmp); free(rec); free(internal);
    return ORC_ERR_OOM;
}

/* ------------------------------------------------------------------------ */
/* Partition hypergraph G_P = (P, A, eta) of Sec. 3 ("Partitioning
 * Definition"), R18: A = { rho(e) }, eta(a) = sum of omega(e) over the axons
 * e with rho(e) = a. Output in canonical order (source, size, destination
 * list); capacities: off E+1, pins P, eta and axons E (level 0's sizes). */
int orc_gp(const orc_level *L, const int32_t *rho, int64_t *off, int32_t *pins, int64_t *eta,
           int32_t *axons, int32_t *n_hedges, int64_t *n_pins, int64_t *internal)
{
    int32_t nrec = 0, E2 = 0;
    int64_t poolpos = 0, maxlen = 0, P2 = 0, inw = 0;
    int32_t *pool, *tmp;
    hrec *rec;
    for (int32_t a = 0; a < L->E; a++)
        if (L->off[a + 1] - L->off[a] > maxlen) maxlen = L->off[a + 1] - L->off[a];
    pool = (int32_t *)malloc(((size_t)L->P + 1) * sizeof(int32_t));
    tmp = (int32_t *)malloc(((size_t)maxlen + 1) * sizeof(int32_t));
    rec = (hrec *)malloc(((size_t)L->E + 1) * sizeof(hrec));
    if (!pool || !tmp || !rec) {
        free(pool); free(tmp); free(rec);
        return ORC_ERR_OOM;
    }
    for (int32_t a = 0; a < L->E; a++) {
        int32_t s2 = rho[L->pins[L->off[a]]];
        int32_t nd = 0, len = 0;
        for (int64_t j = L->off[a] + 1; j < L->off[a + 1]; j++) tmp[nd++] = rho[L->pins[j]];
        qsort(tmp, (size_t)nd, sizeof(int32_t), cmp_i32);
        for (int32_t i = 0; i < nd; i++) {
            if (i > 0 && tmp[i] == tmp[i - 1]) continue;
            if (tmp[i] == s2) continue;            /* self-cycle broken */
            pool[poolpos + len++] = tmp[i];
        }
        if (len == 0) {
            inw += L->w[a];
            continue;
        }
        rec[nrec].s = s2; rec[nrec].sd = 0; rec[nrec].len = len;
        rec[nrec].start = poolpos; rec[nrec].w = L->w[a]; rec[nrec].k = L->k[a];
        nrec++;
        poolpos += len;
    }
    g_pool = pool;
    qsort(rec, (size_t)nrec, sizeof(hrec), cmp_hrec);
    {
        int32_t i = 0;
        while (i < nrec) {
            int32_t j = i + 1;
            int64_t w = rec[i].w, k = rec[i].k;
            while (j < nrec && cmp_hrec(&rec[i], &rec[j]) == 0) {
                w += rec[j].w;
                k += rec[j].k;
                j++;
            }
            off[E2] = P2;
            pins[P2++] = rec[i].s;
            memcpy(pins + P2, pool + rec[i].start, (size_t)rec[i].len * sizeof(int32_t));
            P2 += rec[i].len;
            eta[E2] = w;
            axons[E2] = (int32_t)k;
            E2++;
            i = j;
        }
        off[E2] = P2;
    }
    *n_hedges = E2;
    *n_pins = P2;
    *internal = inw;
    free(pool); free(tmp); free(rec);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Connectivity objective (Eq. connectivity): sum over hyperedges of
 * omega(e) * (number of distinct partitions among its pins - 1). */
int64_t orc_conn(const orc_level *L, const int32_t *rho)
{
    int64_t cost = 0, maxlen = 0;
    int32_t *tmp;
    for (int32_t a = 0; a < L->E; a++)
        if (L->off[a + 1] - L->off[a] > maxlen) maxlen = L->off[a + 1] - L->off[a];
    tmp = (int32_t *)malloc(((size_t)maxlen + 1) * sizeof(int32_t));
    if (!tmp) return -1;
    for (int32_t a = 0; a < L->E; a++) {
        int64_t len = L->off[a + 1] - L->off[a], lam = 0;
        for (int64_t j = 0; j < len; j++) tmp[j] = rho[L->pins[L->off[a] + j]];
        qsort(tmp, (size_t)len, sizeof(int32_t), cmp_i32);
        for (int64_t j = 0; j < len; j++)
            if (j == 0 || tmp[j] != tmp[j - 1]) lam++;
        cost += L->w[a] * (lam - 1);
    }
    free(tmp);
    return cost;
}

/* ------------------------------------------------------------------------ */
/* Refinement (Sec. 4.1, "Uncoarsening and Refinement"), one level.
 *
 * A round:
 *  1. pins(p, e) for every hyperedge: cnt(p,e) over all pins, dcnt(p,e)
 *     over destinations. e is inbound to p iff dcnt(p,e) > 0 (R5).
 *     Partition state: psize = sum of size, pinp = sum of inpins,
 *     pin_cnt = sum of in_internal + sum over inbound e of k(e).
 *  2. save(n) = sum of omega(e), e incident to n with cnt(rho(n), e) = 1;
 *     loss(n,p) = sum of omega(e), e incident to n with cnt(p, e) = 0;
 *     gain = save - loss. A move is feasible alone iff p stays within
 *     Omega, Phi and Delta with n added (the new inbound set adds the axons
 *     of n not already inbound to p). n proposes the feasible move of
 *     largest gain to an adjacent partition, ties to the lower p, if the
 *     gain is positive (R9).
 *  3. Proposals are sorted by decreasing gain, ties by vertex id (R10).
 *  4. Each move's gain is recomputed as if all earlier moves were applied
 *     (the Conn change of that single move), and a prefix sum gives the
 *     improvement of each prefix.
 *  5. A prefix is valid iff no partition breaks a limit after it (R13).
 *  6. The moves of the best valid improving prefix are enacted (R11).
 * Rounds repeat until none enacts a move, at most max_refine_rounds (R12).
 */

typedef struct { int32_t n, from, to; int64_t gain; } move;

static int cmp_move(const void *x, const void *y)
{
    const move *a = (const move *)x, *b = (const move *)y;
    if (a->gain != b->gain) return a->gain > b->gain ? -1 : 1;
    return (a->n > b->n) - (a->n < b->n);
}

typedef struct { int64_t size, inpins, pin_cnt; } pstate;

static int violates(const pstate *s, const orc_params *prm)
{
    return s->size > prm->omega || s->inpins > prm->phi || s->pin_cnt > prm->delta;
}

typedef struct {
    int64_t *off;
    int32_t *p, *cnt, *dcnt;
} pincounts;

/* per-hyperedge (partition, cnt, dcnt) lists, in order of first appearance;
 * stamp[p] = a + 1 marks partitions already listed for hyperedge a */
static int pin_counts(const orc_level *L, int32_t K, const int32_t *rho, pincounts *pc)
{
    int64_t pos = 0;
    int32_t *stamp = (int32_t *)calloc((size_t)K + 1, sizeof(int32_t));
    int64_t *slot = (int64_t *)malloc(((size_t)K + 1) * sizeof(int64_t));
    pc->off = (int64_t *)calloc((size_t)L->E + 1, sizeof(int64_t));
    pc->p = (int32_t *)malloc(((size_t)L->P + 1) * sizeof(int32_t));
    pc->cnt = (int32_t *)malloc(((size_t)L->P + 1) * sizeof(int32_t));
    pc->dcnt = (int32_t *)malloc(((size_t)L->P + 1) * sizeof(int32_t));
    if (!pc->off || !pc->p || !pc->cnt || !pc->dcnt || !stamp || !slot) {
        free(pc->off); free(pc->p); free(pc->cnt); free(pc->dcnt); free(stamp); free(slot);
        return ORC_ERR_OOM;
    }
    for (int32_t a = 0; a < L->E; a++) {
        pc->off[a] = pos;
        for (int64_t j = L->off[a]; j < L->off[a + 1]; j++) {
            int32_t q = L->pins[j];
            int32_t p = rho[q];
            if (stamp[p] != a + 1) {
                stamp[p] = a + 1;
                slot[p] = pos;
                pc->p[pos] = p; pc->cnt[pos] = 0; pc->dcnt[pos] = 0;
                pos++;
            }
            pc->cnt[slot[p]]++;
            if (is_dest(L, a, q)) pc->dcnt[slot[p]]++;
        }
    }
    pc->off[L->E] = pos;
    free(stamp);
    free(slot);
    return ORC_OK;
}

static void pin_counts_free(pincounts *pc)
{
    free(pc->off); free(pc->p); free(pc->cnt); free(pc->dcnt);
}

/* cnt and dcnt of partition p in hyperedge a, under the assignment rho,
 * counted from the definition pins(p, e) = |{n in e : rho(n) = p}|. */
static void count_in(const orc_level *L, const int32_t *rho, int32_t a, int32_t p,
                     int32_t *cnt, int32_t *dcnt)
{
    int32_t c = 0, d = 0;
    for (int64_t j = L->off[a]; j < L->off[a + 1]; j++) {
        int32_t q = L->pins[j];
        if (rho[q] == p) {
            c++;
            if (is_dest(L, a, q)) d++;
        }
    }
    *cnt = c;
    *dcnt = d;
}

/* One refinement round. Returns the number of moves enacted (0: none), or
 * a negative value on allocation failure; fills *props, *gain_out. */
static int64_t refine_round(const orc_level *L, int32_t K, int32_t *rho, const orc_params *prm,
                            int32_t *props_out, int64_t *gain_out, int32_t *bad_state)
{
    int32_t V = L->V;
    pincounts pc;
    pstate *ps = NULL, *ps2 = NULL;
    move *mv = NULL;
    int32_t nm = 0;
    int32_t *rho2 = NULL, *plist = NULL;
    int64_t *conn = NULL, *ovp = NULL;
    uint8_t *seen = NULL;
    int64_t result = 0;
    *props_out = 0;
    *gain_out = 0;
    if (pin_counts(L, K, rho, &pc) != ORC_OK) return -1;
    ps = (pstate *)calloc((size_t)K + 1, sizeof(pstate));
    ps2 = (pstate *)calloc((size_t)K + 1, sizeof(pstate));
    mv = (move *)malloc(((size_t)V + 1) * sizeof(move));
    rho2 = (int32_t *)malloc(((size_t)V + 1) * sizeof(int32_t));
    plist = (int32_t *)malloc(((size_t)K + 1) * sizeof(int32_t));
    conn = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
    ovp = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
    seen = (uint8_t *)calloc((size_t)K + 1, 1);
    if (!ps || !ps2 || !mv || !rho2 || !plist || !conn || !ovp || !seen) { result = -1; goto done; }

    /* 1. partition state */
    for (int32_t n = 0; n < V; n++) {
        ps[rho[n]].size += L->size[n];
        ps[rho[n]].inpins += L->inpins[n];
        ps[rho[n]].pin_cnt += L->in_internal[n];
    }
    for (int32_t a = 0; a < L->E; a++)
        for (int64_t j = pc.off[a]; j < pc.off[a + 1]; j++)
            if (pc.dcnt[j] > 0) ps[pc.p[j]].pin_cnt += L->k[a];
    for (int32_t p = 0; p < K; p++)
        if (violates(&ps[p], prm)) *bad_state = 1;

    /* 2. gains and proposals */
    for (int32_t n = 0; n < V; n++) {
        int32_t home = rho[n], np = 0, best = -1;
        int64_t W = 0, save = 0, bg = 0;
        for (int64_t i = L->voff[n]; i < L->voff[n + 1]; i++) {
            int32_t a = L->vinc[i];
            int nd = is_dest(L, a, n);
            W += L->w[a];
            for (int64_t j = pc.off[a]; j < pc.off[a + 1]; j++) {
                int32_t p = pc.p[j];
                if (p == home) {
                    if (pc.cnt[j] == 1) save += L->w[a];
                    continue;
                }
                if (!seen[p]) { seen[p] = 1; conn[p] = 0; ovp[p] = 0; plist[np++] = p; }
                conn[p] += L->w[a];
                if (nd && pc.dcnt[j] > 0) ovp[p] += L->k[a];
            }
        }
        for (int32_t i = 0; i < np; i++) {
            int32_t p = plist[i];
            int64_t loss = W - conn[p];          /* omega of e with cnt(p,e) = 0 */
            int64_t gain = save - loss;
            int feasible = ps[p].size + L->size[n] <= prm->omega &&
                           ps[p].inpins + L->inpins[n] <= prm->phi &&
                           ps[p].pin_cnt + L->in_count[n] - ovp[p] <= prm->delta;
            seen[p] = 0;
            if (!feasible) continue;
            if (best < 0 || gain > bg || (gain == bg && p < best)) { best = p; bg = gain; }
        }
        if (best >= 0 && (bg > 0 || prm->refine_nonpositive)) {     /* R9, R19 */
            mv[nm].n = n; mv[nm].from = home; mv[nm].to = best; mv[nm].gain = bg;
            nm++;
        }
    }
    *props_out = nm;

    /* 3. order */
    qsort(mv, (size_t)nm, sizeof(move), cmp_move);

    /* 4-5. replay the sequence on a copy */
    memcpy(rho2, rho, (size_t)V * sizeof(int32_t));
    memcpy(ps2, ps, (size_t)K * sizeof(pstate));
    {
        int64_t G = 0, bestG = 0;
        int32_t istar = 0, nviol = 0;
        for (int32_t i = 0; i < nm; i++) {
            int32_t n = mv[i].n, f = mv[i].from, t = mv[i].to;
            int64_t g = 0;
            int vf0 = violates(&ps2[f], prm), vt0 = violates(&ps2[t], prm);
            for (int64_t x = L->voff[n]; x < L->voff[n + 1]; x++) {
                int32_t a = L->vinc[x];
                int32_t cf, dcf, ct, dct;
                count_in(L, rho2, a, f, &cf, &dcf);
                count_in(L, rho2, a, t, &ct, &dct);
                g += L->w[a] * ((cf == 1 ? 1 : 0) - (ct == 0 ? 1 : 0));
                if (is_dest(L, a, n)) {
                    if (dcf == 1) ps2[f].pin_cnt -= L->k[a];   /* e stops being inbound to f */
                    if (dct == 0) ps2[t].pin_cnt += L->k[a];   /* e becomes inbound to t */
                }
            }
            rho2[n] = t;
            ps2[f].size -= L->size[n];   ps2[t].size += L->size[n];
            ps2[f].inpins -= L->inpins[n]; ps2[t].inpins += L->inpins[n];
            ps2[f].pin_cnt -= L->in_internal[n]; ps2[t].pin_cnt += L->in_internal[n];
            nviol += violates(&ps2[f], prm) - vf0;
            nviol += violates(&ps2[t], prm) - vt0;
            G += g;
            if (nviol == 0 && G > 0 && G > bestG) { bestG = G; istar = i + 1; }
        }
        /* 6. enact */
        for (int32_t i = 0; i < istar; i++) rho[mv[i].n] = mv[i].to;
        *gain_out = bestG;
        result = istar;
    }
done:
    pin_counts_free(&pc);
    free(ps); free(ps2); free(mv); free(rho2); free(plist); free(conn); free(ovp); free(seen);
    return result;
}

/* Refines rho (values in [0, K)) on one level. Returns the number of rounds
 * that enacted moves, -1 on allocation failure, -2 if a round started from a
 * state that breaks a limit (never expected). */
int32_t orc_refine(const orc_level *L, int32_t K, int32_t *rho, const orc_params *prm,
                   int32_t level, orc_round_log *log, int32_t log_cap, int32_t *log_len,
                   int64_t *moves)
{
    int32_t rounds = 0, bad = 0;
    for (int32_t r = 0; r < prm->max_refine_rounds; r++) {
        int32_t props = 0;
        int64_t gain = 0;
        int64_t applied = refine_round(L, K, rho, prm, &props, &gain, &bad);
        if (applied < 0) return -1;
        if (log && *log_len < log_cap) {
            log[*log_len].level = level; log[*log_len].round = r; log[*log_len].n_props = props;
            log[*log_len].istar = (int32_t)applied; log[*log_len].gain = gain;
            (*log_len)++;
        }
        if (bad) return -2;
        if (applied == 0) break;
        rounds++;
        if (moves) *moves += applied;
    }
    return rounds;
}

/* ------------------------------------------------------------------------ */
/* The whole pass (Fig. partitioning_flow): coarsen until no candidate
 * remains (R8), take one partition per coarsest vertex, then project and
 * refine level by level. */
int orc_partition(const orc_params *prm, int32_t V, int32_t E, const int64_t *off,
                  const int32_t *pins, const int32_t *w, int32_t *rho_out, int64_t *cost_out,
                  orc_stats *st, orc_level_log *llog, int32_t llog_cap, int32_t *llog_len,
                  orc_round_log *rlog, int32_t rlog_cap, int32_t *rlog_len)
{
    orc_level **lv = NULL;
    int32_t **cids = NULL;
    int32_t nl = 0, err = ORC_OK, cap;
    int32_t *cand = NULL, *cov = NULL, *match = NULL, *rho = NULL, *rho2 = NULL;
    int64_t *cscore = NULL;
    orc_level *L0;
    memset(st, 0, sizeof(*st));
    *llog_len = 0;
    *rlog_len = 0;
    err = orc_build(prm, V, E, off, pins, w, &L0);
    if (err != ORC_OK) return err;
    cap = prm->max_levels + 1;
    lv = (orc_level **)calloc((size_t)cap, sizeof(orc_level *));
    cids = (int32_t **)calloc((size_t)cap, sizeof(int32_t *));
    cand = (int32_t *)malloc(((size_t)V + 1) * sizeof(int32_t));
    cov = (int32_t *)malloc(((size_t)V + 1) * sizeof(int32_t));
    match = (int32_t *)malloc(((size_t)V + 1) * sizeof(int32_t));
    cscore = (int64_t *)malloc(((size_t)V + 1) * sizeof(int64_t));
    rho = (int32_t *)malloc(((size_t)V + 1) * sizeof(int32_t));
    rho2 = (int32_t *)malloc(((size_t)V + 1) * sizeof(int32_t));
    if (!lv || !cids || !cand || !cov || !match || !cscore || !rho || !rho2) { err = ORC_ERR_OOM; goto done; }
    lv[0] = L0;
    nl = 1;
    for (;;) {
        orc_level *L = lv[nl - 1], *C = NULL;
        int32_t ncand = 0, npairs;
        if (nl - 1 >= prm->max_levels) break;
        if (orc_affinity(L, prm, cand, cscore, cov) != ORC_OK) { err = ORC_ERR_OOM; goto done; }
        for (int32_t n = 0; n < L->V; n++) ncand += cand[n] >= 0;
        if (ncand == 0) {
            if (llog && *llog_len < llog_cap) {
                orc_level_log *g = &llog[(*llog_len)++];
                g->V = L->V; g->E = L->E; g->P = L->P; g->n_cand = 0; g->n_pairs = 0;
            }
            break;
        }
        npairs = orc_match(L->V, cand, cscore, match);
        if (npairs <= 0) { err = ORC_ERR_INVALID; goto done; }
        if (llog && *llog_len < llog_cap) {
            orc_level_log *g = &llog[(*llog_len)++];
            g->V = L->V; g->E = L->E; g->P = L->P; g->n_cand = ncand; g->n_pairs = npairs;
        }
        cids[nl - 1] = (int32_t *)malloc(((size_t)L->V + 1) * sizeof(int32_t));
        if (!cids[nl - 1]) { err = ORC_ERR_OOM; goto done; }
        if (orc_contract(L, match, cand, cov, cids[nl - 1], &C) != ORC_OK) { err = ORC_ERR_OOM; goto done; }
        lv[nl++] = C;
    }
    st->levels = nl - 1;
    {
        orc_level *Lc = lv[nl - 1];
        int32_t K = Lc->V;
        st->n_parts = K;
        for (int32_t n = 0; n < K; n++) rho[n] = n;
        st->cost_initial = orc_conn(Lc, rho);
        for (int32_t l = nl - 1; l >= 0; l--) {
            int32_t r;
            if (l < nl - 1) {
                /* projection: rho_l(n) = rho_{l+1}(cid_l(n)) */
                for (int32_t n = 0; n < lv[l]->V; n++) rho2[n] = rho[cids[l][n]];
                memcpy(rho, rho2, (size_t)lv[l]->V * sizeof(int32_t));
            }
            r = orc_refine(lv[l], K, rho, prm, l, rlog, rlog_cap, rlog_len, &st->moves);
            if (r < 0) { err = r == -1 ? ORC_ERR_OOM : ORC_ERR_INVALID; goto done; }
            st->rounds += r;
        }
        memcpy(rho_out, rho, (size_t)V * sizeof(int32_t));
        st->cost = orc_conn(lv[0], rho);
        *cost_out = st->cost;
        {
            uint8_t *used = (uint8_t *)calloc((size_t)K + 1, 1);
            if (!used) { err = ORC_ERR_OOM; goto done; }
            for (int32_t n = 0; n < V; n++) used[rho[n]] = 1;
            for (int32_t p = 0; p < K; p++) st->nonempty_parts += used[p];
            free(used);
        }
    }
done:
    if (lv) for (int32_t i = 0; i < nl; i++) level_free(lv[i]);
    if (cids) for (int32_t i = 0; i < cap; i++) free(cids[i]);
    free(lv); free(cids); free(cand); free(cov); free(match); free(cscore); free(rho); free(rho2);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Placement refinement (Sec. 4.2, "Swap Proposals" and "Placement
 * Refinement") of the partition hypergraph G_P on a width x height lattice
 * (core id = y * width + x, Manhattan distance).
 *
 *  RP1 The cores adjacent to h are its 4-neighbours on the lattice.
 *  RP2 force(p, k) = sum over hyperedges a incident to p of eta(a) times the
 *      sum over the other pins q of a of dist(h, g(q)) - max(dist(k, g(q)), 1),
 *      h = g(p) (Eq. force); tension(h, k) = force(pi(h), k) + force(pi(k), h)
 *      over occupied cores (Eq. tension).
 *  RP3 A node at h proposes the adjacent core with the largest tension, ties
 *      to the lower core id, if that tension is positive.
 *  RP4 Proposals over cores are matched by Eq. matching with tension as the
 *      score (orc_match); matched pairs are disjoint swaps.
 *  RP5 Swaps are ordered by decreasing tension, ties by the lower smaller
 *      core id; each swap's tension is evaluated again with every earlier
 *      swap of the sequence applied; the prefix with the largest positive
 *      sum (shortest on ties) is applied. Rounds repeat until none is
 *      applied, at most max_rounds.
 *  RP6 The total residual distance is the sum over hyperedges of eta(a)
 *      times the Manhattan distances of all unordered pairs of its pins; a
 *      swap's tension is exactly its decrease, so every applied prefix
 *      lowers it by its sum. */

typedef struct { int32_t h, k; int64_t t; } swp;

static int cmp_swp(const void *x, const void *y)
{
    const swp *a = (const swp *)x, *b = (const swp *)y;
    if (a->t != b->t) return a->t > b->t ? -1 : 1;
    return (a->h > b->h) - (a->h < b->h);
}

static int32_t mdist(int32_t width, int32_t u, int32_t v)
{
    int32_t dx = u % width - v % width, dy = u / width - v / width;
    return (dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy);
}

/* force of node p (at g[p]) towards core k */
static int64_t place_force(int32_t np, const int64_t *voff, const int32_t *vinc, const int64_t *off,
                           const int32_t *pins, const int64_t *eta, int32_t width,
                           const int32_t *g, int32_t p, int32_t k)
{
    int64_t f = 0;
    int32_t h = g[p];
    (void)np;
    for (int64_t i = voff[p]; i < voff[p + 1]; i++) {
        int32_t a = vinc[i];
        int64_t s = 0;
        for (int64_t j = off[a]; j < off[a + 1]; j++) {
            int32_t q = pins[j];
            if (q == p) continue;
            int32_t dk = mdist(width, k, g[q]);
            s += mdist(width, h, g[q]) - (dk > 1 ? dk : 1);
        }
        f += eta[a] * s;
    }
    return f;
}

static int64_t place_tension(int32_t np, const int64_t *voff, const int32_t *vinc,
                             const int64_t *off, const int32_t *pins, const int64_t *eta,
                             int32_t width, const int32_t *g, const int32_t *pi, int32_t h,
                             int32_t k)
{
    int64_t t = 0;
    if (pi[h] >= 0) t += place_force(np, voff, vinc, off, pins, eta, width, g, pi[h], k);
    if (pi[k] >= 0) t += place_force(np, voff, vinc, off, pins, eta, width, g, pi[k], h);
    return t;
}

int64_t orc_place_trd(int32_t np, int32_t ne, const int64_t *off, const int32_t *pins,
                      const int64_t *eta, int32_t width, const int32_t *g)
{
    int64_t d = 0;
    (void)np;
    for (int32_t a = 0; a < ne; a++)
        for (int64_t i = off[a]; i < off[a + 1]; i++)
            for (int64_t j = i + 1; j < off[a + 1]; j++)
                d += eta[a] * mdist(width, g[pins[i]], g[pins[j]]);
    return d;
}

/* Refines the placement g (int32[np], distinct cores in [0, width*height)).
 * Per round logs (capacity log_cap): proposals, swaps matched, swaps applied
 * and the residual distance removed. Returns the rounds run, or a negative
 * error code. */
int32_t orc_place_refine(int32_t np, int32_t ne, const int64_t *off, const int32_t *pins,
                         const int64_t *eta, int32_t width, int32_t height, int32_t *g,
                         int32_t max_rounds, int32_t *log_props, int32_t *log_swaps,
                         int32_t *log_applied, int64_t *log_gain, int32_t log_cap)
{
    int32_t nh = width * height, rounds = 0, err = 0;
    int64_t *voff = (int64_t *)calloc((size_t)np + 1, sizeof(int64_t));
    int64_t P = off[ne];
    int32_t *vinc = (int32_t *)malloc(((size_t)P + 1) * sizeof(int32_t));
    int32_t *fill = (int32_t *)calloc((size_t)np + 1, sizeof(int32_t));
    int32_t *pi = (int32_t *)malloc(((size_t)nh + 1) * sizeof(int32_t));
    int32_t *cand = (int32_t *)malloc(((size_t)nh + 1) * sizeof(int32_t));
    int64_t *cscore = (int64_t *)malloc(((size_t)nh + 1) * sizeof(int64_t));
    int32_t *match = (int32_t *)malloc(((size_t)nh + 1) * sizeof(int32_t));
    int32_t *g2 = (int32_t *)malloc(((size_t)np + 1) * sizeof(int32_t));
    int32_t *pi2 = (int32_t *)malloc(((size_t)nh + 1) * sizeof(int32_t));
    swp *sw = (swp *)malloc(((size_t)nh + 1) * sizeof(swp));
    if (!voff || !vinc || !fill || !pi || !cand || !cscore || !match || !g2 || !pi2 || !sw) {
        err = -ORC_ERR_OOM;
        goto done;
    }
    /* incident hyperedges of every node (each once) */
    for (int32_t a = 0; a < ne; a++)
        for (int64_t j = off[a]; j < off[a + 1]; j++) voff[pins[j] + 1]++;
    for (int32_t p = 0; p < np; p++) voff[p + 1] += voff[p];
    for (int32_t a = 0; a < ne; a++)
        for (int64_t j = off[a]; j < off[a + 1]; j++) vinc[voff[pins[j]] + fill[pins[j]]++] = a;
    for (int32_t h = 0; h < nh; h++) pi[h] = -1;
    for (int32_t p = 0; p < np; p++) {
        if (g[p] < 0 || g[p] >= nh || pi[g[p]] >= 0) { err = -ORC_ERR_INVALID; goto done; }
        pi[g[p]] = p;
    }
    while (rounds < max_rounds) {
        int32_t props = 0, ns = 0, istar = 0;
        int64_t G = 0, bestG = 0;
        /* RP3: proposals over occupied cores */
        for (int32_t h = 0; h < nh; h++) {
            cand[h] = -1;
            cscore[h] = 0;
            if (pi[h] < 0) continue;
            int32_t x = h % width, y = h / width;
            int32_t nb[4] = {y > 0 ? h - width : -1, x > 0 ? h - 1 : -1,
                             x + 1 < width ? h + 1 : -1, y + 1 < height ? h + width : -1};
            int32_t best = -1;
            int64_t bt = 0;
            for (int u = 0; u < 4; u++) {   /* ascending core ids */
                int32_t k = nb[u];
                if (k < 0) continue;
                int64_t t = place_tension(np, voff, vinc, off, pins, eta, width, g, pi, h, k);
                if (best < 0 || t > bt) { best = k; bt = t; }   /* ties: lower id */
            }
            if (best >= 0 && bt > 0) {
                cand[h] = best;
                cscore[h] = bt;
                props++;
            }
        }
        /* RP4 */
        orc_match(nh, cand, cscore, match);
        for (int32_t h = 0; h < nh; h++)
            if (match[h] > h) {
                sw[ns].h = h;
                sw[ns].k = match[h];
                sw[ns].t = place_tension(np, voff, vinc, off, pins, eta, width, g, pi, h, match[h]);
                ns++;
            }
        /* RP5 */
        qsort(sw, (size_t)ns, sizeof(swp), cmp_swp);
        memcpy(g2, g, (size_t)np * sizeof(int32_t));
        memcpy(pi2, pi, (size_t)nh * sizeof(int32_t));
        for (int32_t i = 0; i < ns; i++) {
            int32_t h = sw[i].h, k = sw[i].k;
            G += place_tension(np, voff, vinc, off, pins, eta, width, g2, pi2, h, k);
            int32_t a = pi2[h], b = pi2[k];
            pi2[h] = b;
            pi2[k] = a;
            if (a >= 0) g2[a] = k;
            if (b >= 0) g2[b] = h;
            if (G > 0 && G > bestG) { bestG = G; istar = i + 1; }
        }
        for (int32_t i = 0; i < istar; i++) {
            int32_t h = sw[i].h, k = sw[i].k;
            int32_t a = pi[h], b = pi[k];
            pi[h] = b;
            pi[k] = a;
            if (a >= 0) g[a] = k;
            if (b >= 0) g[b] = h;
        }
        if (rounds < log_cap) {
            if (log_props) log_props[rounds] = props;
            if (log_swaps) log_swaps[rounds] = ns;
            if (log_applied) log_applied[rounds] = istar;
            if (log_gain) log_gain[rounds] = bestG;
        }
        rounds++;
        if (istar == 0) break;
    }
done:
    free(voff); free(vinc); free(fill); free(pi); free(cand); free(cscore); free(match);
    free(g2); free(pi2); free(sw);
    return err ? err : rounds;
}

/* ------------------------------------------------------------------------ */
/* Initial placement (Sec. 4.2, "Initial Placement") of G_P on a width x
 * height lattice, for one start (the multi-start runs several initial
 * orders).
 *
 *  RI1 Cores are ordered by their index on the Hilbert curve of the
 *      smallest power-of-two square covering the lattice (cells outside the
 *      lattice skipped); node i of the final sequence goes to the i-th core.
 *  RI2 Section s_0 holds every node in the given initial (random) order.
 *      Each section of more than one node splits into its first ceil(n/2)
 *      and its remaining nodes; recursion stops at single nodes.
 *  RI3 Label propagation between two sibling sections L and R: the cut is
 *      the summed eta of hyperedges with pins in both L and R (pins outside
 *      L and R ignored). Swaps of one node of L with one of R are applied
 *      one at a time, each time the swap lowering the cut the most (ties:
 *      the lower node of L, then of R), while some swap lowers it, at most
 *      4 * min(|L|, |R|) swaps; swapped nodes take each other's positions.
 *  RI4 Folding, bottom-up: a section whose sibling S' exists is reversed
 *      if its child more strongly connected to S' (summed eta of hyperedges
 *      with pins in both) does not face S' -- the last child when S' lies
 *      to its right, the first when to its left; ties keep the order.
 *      Reversing a section reverses the order of its children and of the
 *      nodes inside them. */

static uint32_t hilbert_d(uint32_t n, uint32_t x, uint32_t y)
{
    uint32_t d = 0;
    for (uint32_t s = n / 2; s > 0; s /= 2) {
        uint32_t rx = (x & s) > 0, ry = (y & s) > 0;
        d += s * s * ((3 * rx) ^ ry);
        if (ry == 0) {                    /* rotate the quadrant */
            if (rx == 1) { x = s - 1 - x; y = s - 1 - y; }
            uint32_t t = x; x = y; y = t;
        }
    }
    return d;
}

typedef struct { uint32_t d; int32_t core; } hcell;

static int cmp_hcell(const void *x, const void *y)
{
    const hcell *a = (const hcell *)x, *b = (const hcell *)y;
    return (a->d > b->d) - (a->d < b->d);
}

/* cores in Hilbert order (RI1) */
int orc_hilbert_order(int32_t width, int32_t height, int32_t *order)
{
    uint32_t n = 1;
    int32_t nh = width * height;
    while (n < (uint32_t)width || n < (uint32_t)height) n <<= 1;
    hcell *c = (hcell *)malloc(((size_t)nh + 1) * sizeof(hcell));
    if (!c) return ORC_ERR_OOM;
    for (int32_t k = 0; k < nh; k++) {
        c[k].d = hilbert_d(n, (uint32_t)(k % width), (uint32_t)(k / width));
        c[k].core = k;
    }
    qsort(c, (size_t)nh, sizeof(hcell), cmp_hcell);
    for (int32_t i = 0; i < nh; i++) order[i] = c[i].core;
    free(c);
    return ORC_OK;
}

typedef struct {
    int32_t np, ne;
    const int64_t *off;
    const int32_t *pins;
    const int64_t *eta;
    int32_t *side;    /* per node: 0 outside, 1 in L (or X), 2 in R (or S') */
} ip_ctx;

/* summed eta of hyperedges with pins on both sides 1 and 2 */
static int64_t ip_cut(const ip_ctx *c)
{
    int64_t cut = 0;
    for (int32_t a = 0; a < c->ne; a++) {
        int in1 = 0, in2 = 0;
        for (int64_t j = c->off[a]; j < c->off[a + 1]; j++) {
            int32_t s = c->side[c->pins[j]];
            if (s == 1) in1 = 1;
            if (s == 2) in2 = 1;
        }
        if (in1 && in2) cut += c->eta[a];
    }
    return cut;
}

/* RI3 on seq[lo..mid) and seq[mid..hi): steepest-descent swaps */
static int ip_label_propagation(ip_ctx *c, int32_t *seq, int32_t lo, int32_t mid, int32_t hi,
                                int32_t *pos)
{
    int32_t nl = mid - lo, nr = hi - mid;
    int32_t cap = 4 * (nl < nr ? nl : nr);
    for (int32_t i = lo; i < hi; i++) {
        c->side[seq[i]] = i < mid ? 1 : 2;
        pos[seq[i]] = i;
    }
    int64_t cur = ip_cut(c);
    for (int32_t it = 0; it < cap && cur > 0; it++) {
        int32_t ba = -1, bb = -1;
        int64_t bd = 0;
        for (int32_t i = lo; i < mid; i++) {
            for (int32_t j = mid; j < hi; j++) {
                int32_t x = seq[i], y = seq[j];
                c->side[x] = 2;
                c->side[y] = 1;
                int64_t d = cur - ip_cut(c);
                c->side[x] = 1;
                c->side[y] = 2;
                if (d > bd || (d == bd && d > 0 && (x < ba || (x == ba && y < bb)))) {
                    bd = d;
                    ba = x;
                    bb = y;
                }
            }
        }
        if (bd <= 0) break;
        int32_t pa = pos[ba], pb = pos[bb];
        seq[pa] = bb; seq[pb] = ba;
        pos[ba] = pb; pos[bb] = pa;
        c->side[ba] = 2;
        c->side[bb] = 1;
        cur -= bd;
    }
    for (int32_t i = lo; i < hi; i++) c->side[seq[i]] = 0;
    return ORC_OK;
}

/* connection of seq[a0..a1) to seq[b0..b1) (RI4) */
static int64_t ip_conn(ip_ctx *c, const int32_t *seq, int32_t a0, int32_t a1, int32_t b0,
                       int32_t b1)
{
    for (int32_t i = a0; i < a1; i++) c->side[seq[i]] = 1;
    for (int32_t i = b0; i < b1; i++) c->side[seq[i]] = 2;
    int64_t x = ip_cut(c);
    for (int32_t i = a0; i < a1; i++) c->side[seq[i]] = 0;
    for (int32_t i = b0; i < b1; i++) c->side[seq[i]] = 0;
    return x;
}

static void ip_reverse(int32_t *seq, int32_t lo, int32_t hi)
{
    for (int32_t i = lo, j = hi - 1; i < j; i++, j--) {
        int32_t t = seq[i]; seq[i] = seq[j]; seq[j] = t;
    }
}

/* node sequence of one start (RI2-RI4), in place on seq (initial order in,
 * final order out) */
int orc_initial_sequence(int32_t np, int32_t ne, const int64_t *off, const int32_t *pins,
                         const int64_t *eta, int32_t *seq)
{
    int32_t *side = (int32_t *)calloc((size_t)np + 1, sizeof(int32_t));
    int32_t *pos = (int32_t *)malloc(((size_t)np + 1) * sizeof(int32_t));
    /* the bisection tree as intervals of seq, level by level */
    int32_t cap = 2 * (np > 0 ? np : 1) + 2;
    int32_t *lo = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int32_t *hi = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int32_t *par = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int32_t *depth = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int32_t *kid = (int32_t *)malloc((size_t)cap * sizeof(int32_t));   /* first child or -1 */
    int err = ORC_OK;
    ip_ctx c = {np, ne, off, pins, eta, side};
    if (!side || !pos || !lo || !hi || !par || !depth || !kid) { err = ORC_ERR_OOM; goto done; }
    if (np <= 1) goto done;
    {
        int32_t nn = 1, maxd = 0;
        lo[0] = 0; hi[0] = np; par[0] = -1; depth[0] = 0; kid[0] = -1;
        /* RI2 + RI3: split breadth-first, propagate labels between siblings */
        for (int32_t s = 0; s < nn; s++) {
            int32_t n = hi[s] - lo[s];
            if (n <= 1) continue;
            int32_t mid = lo[s] + (n + 1) / 2;
            err = ip_label_propagation(&c, seq, lo[s], mid, hi[s], pos);
            if (err) goto done;
            kid[s] = nn;
            for (int t = 0; t < 2; t++) {
                lo[nn] = t ? mid : lo[s];
                hi[nn] = t ? hi[s] : mid;
                par[nn] = s;
                depth[nn] = depth[s] + 1;
                kid[nn] = -1;
                if (depth[nn] > maxd) maxd = depth[nn];
                nn++;
            }
        }
        /* RI4: deepest sections first; a section's sibling is the other
         * child of its parent (the root has none) */
        for (int32_t d = maxd; d >= 1; d--) {
            for (int32_t s = 0; s < nn; s++) {
                if (depth[s] != d || kid[s] < 0) continue;   /* leaves need no orientation */
                int32_t p = par[s];
                int32_t sib = kid[p] == s ? kid[p] + 1 : kid[p];
                int32_t a = kid[s], b = kid[s] + 1;         /* first and last child */
                int64_t ca = ip_conn(&c, seq, lo[a], hi[a], lo[sib], hi[sib]);
                int64_t cb = ip_conn(&c, seq, lo[b], hi[b], lo[sib], hi[sib]);
                int right = lo[sib] > lo[s];              /* sibling to the right */
                int flip = right ? (ca > cb) : (cb > ca);
                if (flip) {
                    ip_reverse(seq, lo[s], hi[s]);
                    /* children swap places; their intervals follow */
                    int32_t na = hi[a] - lo[a];
                    int32_t nb2 = hi[b] - lo[b];
                    (void)na;
                    lo[b] = lo[s]; hi[b] = lo[s] + nb2;
                    lo[a] = hi[b]; hi[a] = hi[s];
                    /* deeper descendants were final already; their intervals
                     * are not read again */
                }
            }
        }
    }
done:
    free(side); free(pos); free(lo); free(hi); free(par); free(depth); free(kid);
    return err;
}
