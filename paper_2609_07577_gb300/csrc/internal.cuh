// Handle layout and the host-side entry points of each pipeline stage.
#pragma once
#include "../../include/snnmap.h"
#include "common.cuh"
#include "segsort.cuh"
#include "histo_tiers.cuh"

#include <vector>

namespace snn {

// Device scalar slots (int64) read back by the host at synchronization points.
enum Scalar : int {
    SC_STATUS = 0,   // int32 status bits live in the low word of this slot
    SC_A, SC_B, SC_C, SC_D, SC_E, SC_F, SC_G,
    SC_W2 = 9,       // pair terms of the level being classified
    SC_COUNT = 16,
};

struct LevelExtra {
    SegBuckets seg;          // hyperedge size buckets
    int64_t pair_terms = 0;  // sum of |e|(|e|-1)
    int32_t n_block = 0;     // last histogram: vertices on the block tier
    int32_t n_global = 0;    //                 and on the global-memory tier
    int32_t carried = 0;     // candidates: 0 full histogram, 1 carried, 2 score matrix
    int32_t n_full = 0;      // vertices given a full neighbour histogram
    int64_t hist_work = 0;   // elements visited by the neighbour histograms
};

// pipeline stages timed by the profiler
enum ProfStage : int {
    PS_BUILD, PS_AFFINITY, PS_MATCH, PS_CONTRACT, PS_INCIDENCE, PS_PINCOUNT, PS_GAINS,
    PS_SORTMOVES, PS_REPLAY, PS_VALIDITY, PS_APPLY, PS_SAVE, PS_ROWS, PS_CROSS, PS_N
};
extern const char* const kStageNames[PS_N];

}  // namespace snn

namespace snn {
// Connection rows of the refinement levels that fit the row budget: C and O
// hold cap rows of Kp (K rounded up to 4) int32 entries; rowid maps the
// current level's vertices to rows.
struct DenseRows {
    int32_t K = 0;
    int64_t Kp = 0;
    int64_t cap = 0;
    int32_t* C = nullptr;
    int32_t* O = nullptr;
    int32_t* rowid = nullptr;
    int32_t* rowid2 = nullptr;
    int32_t* fresh = nullptr;
    // per row: bit c set when entries [c cw, (c + 1) cw) of its C row may be
    // nonzero (set wherever an entry becomes nonzero, cleared with the row);
    // cw is the smallest power of two >= 32 giving at most 64 chunks
    unsigned long long* M = nullptr;
    int32_t cw = 32;
    int32_t level = -1;       // level the rows describe
    bool pending = false;     // fresh rows of this level not computed yet
};

// Neighbour score and shared inbound count of every vertex pair of the
// coarsest level when it is small: S and OV are V x Vs int32 (Vs = V rounded
// up to 4), S2/OV2 the buffers the next level is gathered into.
struct ScoreMat {
    int64_t cap = 0;   // entries per buffer
    int64_t Vs = 0;
    int32_t* S = nullptr;
    int32_t* OV = nullptr;
    int32_t* S2 = nullptr;
    int32_t* OV2 = nullptr;
    int32_t level = -1;   // level the matrix describes
};

// Proposals, gains and re-evaluation flags of the last histogram-refined
// level, double-buffered so the next finer level can inherit them through
// its cid map (cap vertices each).
struct Carry {
    int32_t* pto[2] = {nullptr, nullptr};
    int64_t* pgain[2] = {nullptr, nullptr};
    int32_t* dirty[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t cap = 0;
    int32_t level = -1;   // level whose final state buffers[cur] hold (-1: none)
};

// Candidates carried through a contraction (coarsen.cu, aff_carry): for each
// vertex of `level`, what its previous-level candidate says about it
// (kind), and the carried candidate, score and shared count.
struct AffCarry {
    int32_t* cand = nullptr;
    int64_t* score = nullptr;
    int32_t* ov = nullptr;
    uint8_t* kind = nullptr;
    uint8_t* full = nullptr;    // vertices needing a full histogram
    int64_t cap = 0;
    int32_t level = -1;         // level the carry describes (-1: none)
};

// The partition hypergraph G_P of the last snnmap_partition_graph call.
struct GpOut {
    int64_t* hoff = nullptr;
    int32_t* hpins = nullptr;
    int64_t* eta = nullptr;
    int32_t* axons = nullptr;
    uint8_t* hsd = nullptr;
    int32_t E = 0, K = 0;
    int64_t P = 0;
    int64_t internal = 0;
};
}  // namespace snn

struct snnmap_hgraph {
    snnmap_params prm{};
    int device = 0;
    cudaStream_t stream = 0;
    std::vector<snn::Level> levels;
    std::vector<snn::LevelExtra> extra;
    snn::Arena scratch;
    int64_t* d_scal = nullptr;   // SC_COUNT device slots
    int64_t* h_scal = nullptr;   // pinned mirror
    // pinned: the counters of a level's neighbour histograms (two sets for the
    // carried form), copied without a wait and folded into the level's extra
    // record once the stream has been synchronized (tier_fold)
    int64_t* h_tier = nullptr;
    int32_t tier_level = -1;     // level whose counters are in flight, else -1
    int32_t tier_form = 0;       // 1 full histogram, 2 carried form
    // results of the last coarsening step (for the current coarsest level)
    int32_t* cand = nullptr;
    int64_t* cscore = nullptr;
    int32_t* cov = nullptr;
    int32_t* match = nullptr;
    int32_t cap_v = 0;           // capacity of the four arrays above
    int64_t level_budget = 0;    // bytes of intermediate levels kept resident
    int32_t keep_stride = 1;     // intermediate levels kept: multiples of this
    int64_t peak_bytes = 0;      // largest held_bytes() seen at a checkpoint
    bool have_matching = false;
    int32_t last_pairs = 0;
    bool wide = false;           // some neighbour score may reach 2^32
    int64_t wsum = 0;            // sum of omega over the input hyperedges
    bool wzero = false;          // some kept hyperedge has omega 0: adjacency is not a
                                 // nonzero score, so no score matrix and no connection rows
    int64_t row_budget = -1;     // bytes for connection rows (-1: default, 0: none)
    snn::DenseRows dense;
    snn::ScoreMat mat;
    snn::GpOut gp;
    snn::Carry carry;
    snn::AffCarry icar;
    int32_t coarsen_mode = 0;    // 0 auto, 1 full histograms, 2 carried whenever possible
    snn::HtTiers tiers;          // histogram tier thresholds
    std::vector<snnmap_round_log> rlog;
    std::vector<snnmap_level_log> llog;
    // profiler
    bool prof_on = false;
    struct Pend {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Pend> prof_pend;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[snn::PS_N] = {};
    int64_t prof_calls[snn::PS_N] = {};
};

namespace snn {

// Times the enclosed launches of one stage with a pair of events.
struct ProfScope {
    snnmap_hgraph* h;
    int stage;
    cudaEvent_t a = nullptr, b = nullptr;
    uint64_t range = 0;   // NVTX range id
    ProfScope(snnmap_hgraph* h_, int stage_);
    ~ProfScope();
};
// folds finished event pairs into the counters (call after a stream sync)
void prof_collect(snnmap_hgraph* h);
void prof_release(snnmap_hgraph* h);

// text of snnmap_last_error for the calling thread (api.cu)
void set_last_error(const std::string& msg);

// folds the histogram counters in flight into their level's extra record
// (synchronizes the handle's stream first)
void tier_fold(snnmap_hgraph* h);
constexpr int TIER_SLOTS = 16;   // int64 per counter set in h_tier (two sets)

// scalars: copy the SC_COUNT slots device->host and synchronize the stream
Status read_scalars(snnmap_hgraph* h);
Status zero_scalars(snnmap_hgraph* h);

// device bytes the handle holds now (levels, cid maps, scratch, per-vertex
// arrays), and the running maximum of that figure
int64_t held_bytes(const snnmap_hgraph* h);
void note_bytes(snnmap_hgraph* h);

// level memory
Status level_alloc(snnmap_hgraph* h, Level& L, LevelExtra& X, int32_t V, int32_t E, int64_t P);
void level_free(snnmap_hgraph* h, Level& L);
// frees a level's arrays, keeping its sizes and cid map
void level_release(snnmap_hgraph* h, Level& L);

// S0: level 0 from the caller's arrays
Status build_level0(snnmap_hgraph* h, int32_t V, int32_t E, const int64_t* d_off,
                    const int32_t* d_pins, const int32_t* d_w);
// incidence lists (CSC) of a level whose hoff/hpins are final
Status build_incidence(snnmap_hgraph* h, Level& L);

// S1 + S2 on the coarsest level: fills h->cand/cscore/cov/match
Status coarsen_level(snnmap_hgraph* h, int32_t* n_cand, int32_t* n_pairs);
// Eq. matching of a candidate pseudo-forest (cand[v] = -1: none) into match
// (-1: unmatched); d_scal: device int64[SC_COUNT] scratch; *n_pairs: pairs.
Status match_forest(int32_t V, const int32_t* cand, const int64_t* cscore, int32_t* match,
                    int64_t* d_scal, Arena& ar, cudaStream_t s, int64_t* n_pairs);
// a device (or managed) pointer; host pointers would fault inside kernels
bool device_pointer(const void* p);
// Input G_P of the placement calls (place.cu): device pointers, offsets from
// 0 and non-decreasing, pins in [0, np); *P_out = offsets[ne]; *hid_out
// (arena) = the hyperedge of every pin entry. err: device int32 scratch.
Status gp_input(int32_t np, int32_t ne, const int64_t* off, const int32_t* pins,
                const int64_t* eta, Arena& ar, cudaStream_t s, int32_t* err, int64_t* P_out,
                int32_t** hid_out);
// S3: next level from h->match
Status contract_level(snnmap_hgraph* h);
// after a contraction of `src`: candidates of src carried to src + 1
Status aff_carry(snnmap_hgraph* h, int32_t src);
void aff_carry_free(snnmap_hgraph* h);
// materializes levels[dst] from resident levels[src] through map (V(src) ids);
// with the matching that produced map (match, and the candidates and their
// overlaps), in_count comes from the pairs instead of a pass over the pins
Status build_coarse(snnmap_hgraph* h, int32_t src, const int32_t* map, const int64_t* d_V2,
                    int32_t dst, const int32_t* match = nullptr, const int32_t* cand = nullptr,
                    const int32_t* cov = nullptr);
// rebuilds a released level from the nearest resident level below it
Status ensure_resident(snnmap_hgraph* h, int32_t level);
// releases intermediate levels while their memory exceeds the budget
void thin_levels(snnmap_hgraph* h);
// S5
Status project(snnmap_hgraph* h, int32_t level, const int32_t* rho_coarse, int32_t* rho_fine);
// S6-S12 on one level; rho in place
// G_P of a level-0 partition (kept in h->gp until the next call or free)
Status emit_gp(snnmap_hgraph* h, int32_t K, const int32_t* rho);
void gp_free(snnmap_hgraph* h);

// score matrix: candidates of `level` from the matrix (built on the first
// small level; *done false when the level is too large or memory short),
// carried through a contraction of `src`, released
Status mat_affinity(snnmap_hgraph* h, int32_t level, bool* done);
Status mat_descend(snnmap_hgraph* h, int32_t src);
void mat_close(snnmap_hgraph* h);

// connection rows: allocation for `rows` vertices and K partitions; rows of
// every vertex of `level` (the coarsest refined level) marked fresh; descent
// from level+1 to `level` after projection; release
Status dense_open(snnmap_hgraph* h, int32_t K, int64_t rows);
Status dense_begin(snnmap_hgraph* h, int32_t level);
Status dense_descend(snnmap_hgraph* h, int32_t level);
void dense_close(snnmap_hgraph* h);
int64_t dense_row_budget(const snnmap_hgraph* h);

// proposal carry for snnmap_partition's uncoarsening (vertices of level 0)
Status carry_open(snnmap_hgraph* h, int64_t cap);
void carry_close(snnmap_hgraph* h);

Status refine_level(snnmap_hgraph* h, int32_t level, int32_t K, int32_t* rho, int64_t* cost,
                    int64_t* cost_start);
// caller-provided rho must index existing partitions
Status check_rho(snnmap_hgraph* h, int32_t level, int32_t K, const int32_t* rho);
// S12 alone
Status level_cost(snnmap_hgraph* h, int32_t level, int32_t K, const int32_t* rho, int64_t* cost);

}  // namespace snn
