// C ABI of libsnnmap (declared in include/snnmap.h): argument checks, handle
// lifetime, and the driver loop of the whole pass (Sec. 4.1, Fig.
// partitioning_flow): coarsen/contract until no candidate remains, one
// partition per coarsest vertex, then project and refine down to level 0.
#include "internal.cuh"

#include <climits>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace {

thread_local std::string g_err;

int fail(const snn::Status& st)
{
    g_err = st.msg;
    return st.code;
}

int fail(int code, const char* msg)
{
    g_err = msg;
    return code;
}

#define API_TRY(expr)                     \
    do {                                  \
        snn::Status s_ = (expr);          \
        if (!s_.ok()) return fail(s_);    \
    } while (0)

bool params_ok(const snnmap_params* p)
{
    return p && p->omega >= 1 && p->delta >= 0 && p->phi >= 0 && p->max_levels >= 0 &&
           p->max_refine_rounds >= 0 && (p->refine_nonpositive == 0 || p->refine_nonpositive == 1);
}

// a device (or managed) pointer; host pointers would fault inside kernels
bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void bind(snnmap_hgraph* h, void* stream)
{
    h->stream = (cudaStream_t)stream;
    h->scratch.stream = h->stream;
}

// process-wide histogram tier table (snnmap_set_tier_table): rows by
// ascending level-0 pin count
struct TierRow {
    int64_t max_pins;
    snn::HtTiers t;
};
std::mutex g_tier_mu;
std::vector<TierRow> g_tier_rows;

snn::HtTiers tiers_for(int64_t pins)
{
    std::lock_guard<std::mutex> lk(g_tier_mu);
    for (const TierRow& r : g_tier_rows)
        if (pins <= r.max_pins) return r.t;
    return snn::HtTiers{};   // sizes the table does not cover keep the built-in defaults
}

void drop_levels_above(snnmap_hgraph* h, size_t keep)
{
    h->icar.level = -1;
    while (h->levels.size() > keep) {
        snn::level_free(h, h->levels.back());
        h->levels.pop_back();
        h->extra.pop_back();
    }
}

__global__ void k_mark_used(int32_t V, const int32_t* __restrict__ rho, uint8_t* used)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        used[rho[n]] = 1;
}

__global__ void k_count_used(int32_t K, const uint8_t* __restrict__ used, int64_t* out)
{
    int c = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < K;
         p += (int64_t)gridDim.x * blockDim.x)
        c += used[p];
    c = snn::warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)out, (unsigned long long)c);
}

snn::Status count_nonempty(snnmap_hgraph* h, int32_t V, int32_t K, const int32_t* rho, int32_t* out)
{
    uint8_t* used;
    SNN_TRY(h->scratch.alloc(&used, K));
    SNN_CUDA(cudaMemsetAsync(used, 0, (size_t)K, h->stream));
    SNN_TRY(snn::zero_scalars(h));
    if (V > 0) SNN_L k_mark_used<<<snn::grid_for(V, 256), 256, 0, h->stream>>>(V, rho, used);
    if (K > 0) SNN_L k_count_used<<<snn::grid_for(K, 256), 256, 0, h->stream>>>(K, used, h->d_scal + snn::SC_A);
    SNN_CUDA(cudaGetLastError());
    SNN_TRY(snn::read_scalars(h));
    *out = (int32_t)h->h_scal[snn::SC_A];
    h->scratch.reset();
    return snn::Status{};
}

}  // namespace

namespace snn {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace snn

extern "C" {

snnmap_params snnmap_default_params(int32_t omega, int32_t delta, int32_t phi)
{
    snnmap_params p;
    p.omega = omega;
    p.delta = delta;
    p.phi = phi;
    p.max_levels = 1024;
    p.max_refine_rounds = 16;
    p.refine_nonpositive = 0;
    return p;
}

const char* snnmap_last_error(void) { return g_err.c_str(); }

int64_t snnmap_launch_count(void) { return snn::launch_count(); }

void snnmap_free(snnmap_hgraph* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    snn::prof_release(h);
    snn::dense_close(h);
    snn::mat_close(h);
    snn::carry_close(h);
    snn::aff_carry_free(h);
    snn::gp_free(h);
    drop_levels_above(h, 0);
    h->scratch.release();
    if (h->cand) cudaFreeAsync(h->cand, h->stream);
    if (h->cscore) cudaFreeAsync(h->cscore, h->stream);
    if (h->cov) cudaFreeAsync(h->cov, h->stream);
    if (h->match) cudaFreeAsync(h->match, h->stream);
    if (h->d_scal) cudaFreeAsync(h->d_scal, h->stream);
    cudaStreamSynchronize(h->stream);
    if (h->h_scal) cudaFreeHost(h->h_scal);
    if (h->h_tier) cudaFreeHost(h->h_tier);
    delete h;
    snn::pool_handles(-1);
}

static int snnmap_build_hgraph_impl(const snnmap_params* params, int32_t n_vertices, int32_t n_hedges,
                        const int64_t* d_offsets, const int32_t* d_pins, const int32_t* d_w,
                        void* stream, snnmap_hgraph** out)
{
    g_err.clear();
    if (!out) return fail(SNNMAP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!params_ok(params)) return fail(SNNMAP_ERR_INVALID, "bad params");
    if (n_vertices < 0 || n_hedges < 0) return fail(SNNMAP_ERR_INVALID, "negative sizes");
    if (!is_device_ptr(d_offsets)) return fail(SNNMAP_ERR_INVALID, "d_offsets is not device memory");
    if (n_hedges > 0 && (!is_device_ptr(d_pins) || !is_device_ptr(d_w)))
        return fail(SNNMAP_ERR_INVALID, "d_pins / d_w are not device memory");
    snnmap_hgraph* h = new (std::nothrow) snnmap_hgraph;
    if (!h) return fail(SNNMAP_ERR_OOM, "host allocation failed");
    snn::pool_handles(1);
    h->prm = *params;
    bind(h, stream);
    cudaGetDevice(&h->device);
    h->levels.reserve((size_t)params->max_levels + 2);
    h->extra.reserve((size_t)params->max_levels + 2);
    int32_t cap = n_vertices > 0 ? n_vertices : 1;
    h->cap_v = cap;
    {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) h->level_budget = (int64_t)(tot * 2 / 5);
        else h->level_budget = (int64_t)1 << 34;
    }
    cudaError_t e = cudaMallocHost(&h->h_scal, snn::SC_COUNT * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_tier, 2 * snn::TIER_SLOTS * sizeof(int64_t));
    if (e == cudaSuccess) memset(h->h_tier, 0, 2 * snn::TIER_SLOTS * sizeof(int64_t));
    if (e == cudaSuccess) e = snn::dev_malloc(&h->d_scal, snn::SC_COUNT * sizeof(int64_t), h->stream);
    if (e == cudaSuccess) e = snn::dev_malloc(&h->cand, (size_t)cap * 4, h->stream);
    if (e == cudaSuccess) e = snn::dev_malloc(&h->cov, (size_t)cap * 4, h->stream);
    if (e == cudaSuccess) e = snn::dev_malloc(&h->match, (size_t)cap * 4, h->stream);
    if (e == cudaSuccess) e = snn::dev_malloc(&h->cscore, (size_t)cap * 8, h->stream);
    if (e != cudaSuccess) {
        snnmap_free(h);
        return fail(e == cudaErrorMemoryAllocation ? SNNMAP_ERR_OOM : SNNMAP_ERR_CUDA,
                    cudaGetErrorString(e));
    }
    snn::Status st = snn::build_level0(h, n_vertices, n_hedges, d_offsets, d_pins, d_w);
    if (!st.ok()) {
        snnmap_free(h);
        return fail(st);
    }
    h->tiers = tiers_for(h->levels[0].P);
    *out = h;
    return SNNMAP_OK;
}

static int snnmap_coarsen_level_impl(snnmap_hgraph* h, void* stream, int32_t* n_cand_out, int32_t* n_pairs_out)
{
    g_err.clear();
    if (!h || !n_cand_out || !n_pairs_out) return fail(SNNMAP_ERR_INVALID, "NULL argument");
    bind(h, stream);
    int32_t nc = 0, np = 0;
    snn::Status st = snn::coarsen_level(h, &nc, &np);
    h->scratch.reset();
    if (!st.ok()) return fail(st);
    snn::tier_fold(h);
    const snn::Level& L = h->levels.back();
    const snn::LevelExtra& X = h->extra.back();
    h->llog.push_back(snnmap_level_log{L.V, L.E, L.P, nc, np, X.pair_terms, X.n_block,
                                        X.n_global, X.carried, X.n_full, X.hist_work});
    *n_cand_out = nc;
    *n_pairs_out = np;
    return SNNMAP_OK;
}

static int snnmap_contract_impl(snnmap_hgraph* h, void* stream, int32_t* V_out, int32_t* E_out, int64_t* P_out)
{
    g_err.clear();
    if (!h) return fail(SNNMAP_ERR_INVALID, "NULL handle");
    bind(h, stream);
    API_TRY(snn::contract_level(h));
    snn::thin_levels(h);
    const snn::Level& N = h->levels.back();
    if (V_out) *V_out = N.V;
    if (E_out) *E_out = N.E;
    if (P_out) *P_out = N.P;
    return SNNMAP_OK;
}

int snnmap_num_levels(const snnmap_hgraph* h, int32_t* n_levels)
{
    if (!h || !n_levels) return fail(SNNMAP_ERR_INVALID, "NULL argument");
    *n_levels = (int32_t)h->levels.size();
    return SNNMAP_OK;
}

int snnmap_level_dims(const snnmap_hgraph* h, int32_t level, int32_t* V, int32_t* E, int64_t* P)
{
    if (!h || level < 0 || level >= (int32_t)h->levels.size())
        return fail(SNNMAP_ERR_INVALID, "no such level");
    const snn::Level& L = h->levels[level];
    if (V) *V = L.V;
    if (E) *E = L.E;
    if (P) *P = L.P;
    return SNNMAP_OK;
}

int snnmap_project(snnmap_hgraph* h, int32_t level, const int32_t* d_rho_coarse, int32_t* d_rho_fine,
                   void* stream)
{
    g_err.clear();
    if (!h || level < 0 || level + 1 >= (int32_t)h->levels.size())
        return fail(SNNMAP_ERR_INVALID, "level has no coarser level");
    if (!is_device_ptr(d_rho_coarse) || !is_device_ptr(d_rho_fine))
        return fail(SNNMAP_ERR_INVALID, "rho buffers must be device memory");
    bind(h, stream);
    API_TRY(snn::project(h, level, d_rho_coarse, d_rho_fine));
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(SNNMAP_ERR_CUDA, cudaGetErrorString(e));
    return SNNMAP_OK;
}

static int snnmap_refine_impl(snnmap_hgraph* h, int32_t level, int32_t n_parts, int32_t* d_rho, void* stream,
                  int64_t* cost_out)
{
    g_err.clear();
    if (!h || level < 0 || level >= (int32_t)h->levels.size())
        return fail(SNNMAP_ERR_INVALID, "no such level");
    if (n_parts < 1 || !is_device_ptr(d_rho)) return fail(SNNMAP_ERR_INVALID, "bad rho / n_parts");
    bind(h, stream);
    int64_t c = 0;
    API_TRY(snn::ensure_resident(h, level));
    API_TRY(snn::check_rho(h, level, n_parts, d_rho));
    API_TRY(snn::refine_level(h, level, n_parts, d_rho, &c, nullptr));
    if (cost_out) *cost_out = c;
    return SNNMAP_OK;
}

int snnmap_connectivity(snnmap_hgraph* h, int32_t n_parts, const int32_t* d_rho, void* stream,
                        int64_t* cost_out)
{
    g_err.clear();
    if (!h || !h->levels.size() || !cost_out) return fail(SNNMAP_ERR_INVALID, "NULL argument");
    if (n_parts < 1 || !is_device_ptr(d_rho)) return fail(SNNMAP_ERR_INVALID, "bad rho / n_parts");
    bind(h, stream);
    API_TRY(snn::check_rho(h, 0, n_parts, d_rho));
    API_TRY(snn::level_cost(h, 0, n_parts, d_rho, cost_out));
    return SNNMAP_OK;
}

static int snnmap_partition_impl(snnmap_hgraph* h, void* stream, int32_t* d_rho_out, int64_t* cost_out,
                     snnmap_stats* stats)
{
    g_err.clear();
    if (!h || !h->levels.size()) return fail(SNNMAP_ERR_INVALID, "NULL handle");
    if (!is_device_ptr(d_rho_out)) return fail(SNNMAP_ERR_INVALID, "d_rho_out must be device memory");
    bind(h, stream);
    drop_levels_above(h, 1);
    snn::mat_close(h);
    h->keep_stride = 1;
    h->rlog.clear();
    h->llog.clear();
    snnmap_stats st{};
    // coarsening
    while ((int32_t)h->levels.size() - 1 < h->prm.max_levels) {
        int32_t nc = 0, np = 0;
        snn::Status s1 = snn::coarsen_level(h, &nc, &np);
        h->scratch.reset();
        if (!s1.ok()) return fail(s1);
        snn::tier_fold(h);
        const snn::Level& L = h->levels.back();
        const snn::LevelExtra& X = h->extra.back();
        h->llog.push_back(snnmap_level_log{L.V, L.E, L.P, nc, np, X.pair_terms, X.n_block,
                                            X.n_global, X.carried, X.n_full, X.hist_work});
        if (nc == 0 || np == 0) break;
        API_TRY(snn::contract_level(h));
        snn::note_bytes(h);
        snn::thin_levels(h);
    }
    int32_t nl = (int32_t)h->levels.size();
    int32_t V0 = h->levels[0].V;
    int32_t K = h->levels.back().V;
    st.levels = nl - 1;
    st.n_parts = K;
    for (auto& L : h->levels) st.pins_total += L.P;
    // uncoarsening
    int32_t* tmp = nullptr;
    cudaError_t e = snn::dev_malloc(&tmp, (size_t)(V0 > 0 ? V0 : 1) * 4, h->stream);
    if (e != cudaSuccess) return fail(SNNMAP_ERR_OOM, cudaGetErrorString(e));
    // rho of the current level lives in `cur`; projection writes `oth`
    int32_t* cur = ((nl - 1) % 2 == 0) ? d_rho_out : tmp;
    int32_t* oth = cur == d_rho_out ? tmp : d_rho_out;
    snn::mat_close(h);
    snn::Status s2 = snn::iota_i32(cur, K, h->stream);
    // Connection rows serve the levels from the coarsest down to the finest
    // one whose rows fit the row budget (conn is stored in int32: needs the
    // summed omega below 2^31). Going down, a level keeps the rows (descent:
    // fresh rows for the pairs only) unless it re-creates more than a quarter
    // of them (2 x pairs > V / 4) while the level above needed few
    // evaluations; a histogram level hands back to rows (every row fresh)
    // once the level above needed at least four evaluations per vertex
    // (rounds times the share of vertices evaluated), as on power-law
    // graphs whose levels run many rounds with every vertex active.
    int32_t lb = nl;
    {
        int64_t rb = snn::dense_row_budget(h);
        int64_t per = ((((int64_t)K + 3) & ~(int64_t)3) * 8 + 20);
        if (rb > 0 && !h->wide && !h->wzero && h->wsum <= INT32_MAX)
            for (int32_t l = nl - 1; l >= 0 && (int64_t)h->levels[l].V * per <= rb; l--) lb = l;
        if (lb < nl && !snn::dense_open(h, K, h->levels[lb].V).ok()) {
            snn::dense_close(h);
            cudaGetLastError();
            lb = nl;
        }
    }
    if (s2.ok()) s2 = snn::carry_open(h, V0);
    int64_t cost = 0;
    double evals_above = 0;   // evaluations per vertex at the level above
    for (int32_t l = nl - 1; s2.ok() && l >= 0; l--) {
        bool rows_here = false;
        if (l < nl - 1) {
            // a level rebuilt for its refinement is released again
            if (l + 1 < nl - 1 && (l + 1) % h->keep_stride != 0)
                snn::level_release(h, h->levels[l + 1]);
            s2 = snn::ensure_resident(h, l);
            if (!s2.ok()) break;
            snn::note_bytes(h);
            s2 = snn::project(h, l, cur, oth);
            if (!s2.ok()) break;
            std::swap(cur, oth);
            if (l >= lb) {
                int64_t V = h->levels[l].V;
                int64_t fresh = 2 * (V - h->levels[l + 1].V);
                bool busy = evals_above >= 4.0;
                snn::ProfScope prof(h, snn::PS_ROWS);
                if (h->dense.level == l + 1 && (4 * fresh <= V || busy)) {
                    s2 = snn::dense_descend(h, l);
                    rows_here = true;
                } else if (h->dense.level != l + 1 && busy) {
                    s2 = snn::dense_begin(h, l);
                    rows_here = true;
                }
            } else if (h->dense.C) {
                snn::dense_close(h);
            }
            if (!s2.ok()) break;
        } else if (lb <= l) {
            s2 = snn::dense_begin(h, l);
            rows_here = true;
            if (!s2.ok()) break;
        }
        if (!rows_here && h->dense.C) h->dense.level = -1;
        int64_t c0 = 0;
        size_t r0 = h->rlog.size();
        s2 = snn::refine_level(h, l, K, cur, &cost, l == nl - 1 ? &c0 : nullptr);
        if (l == nl - 1) st.cost_initial = c0;
        snn::note_bytes(h);
        double act = 0;
        for (size_t r = r0; r < h->rlog.size(); r++) act += h->rlog[r].n_active;
        evals_above = h->levels[l].V > 0 ? act / h->levels[l].V : 0;
    }
    cudaFreeAsync(tmp, h->stream);
    snn::dense_close(h);
    snn::carry_close(h);
    if (!s2.ok()) return fail(s2);
    if (cur != d_rho_out) return fail(SNNMAP_ERR_CUDA, "internal: level parity");
    int32_t ne = 0;
    API_TRY(count_nonempty(h, V0, K, d_rho_out, &ne));
    st.nonempty_parts = ne;
    for (auto& r : h->rlog) {
        if (r.istar > 0) {
            st.rounds++;
            st.moves += r.istar;
        }
    }
    st.cost = cost;
    if (cost_out) *cost_out = cost;
    if (stats) *stats = st;
    return SNNMAP_OK;
}

static int snnmap_partition_host_impl(const snnmap_params* params, int32_t n_vertices, int32_t n_hedges,
                          const int64_t* h_offsets, const int32_t* h_pins, const int32_t* h_w,
                          int32_t* h_rho_out, int64_t* cost_out, snnmap_stats* stats, void* stream)
{
    g_err.clear();
    if (!params_ok(params) || n_vertices < 0 || n_hedges < 0 || !h_offsets || !h_rho_out ||
        (n_hedges > 0 && (!h_pins || !h_w)))
        return fail(SNNMAP_ERR_INVALID, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t P = h_offsets[n_hedges];
    if (h_offsets[0] != 0 || P < 0) return fail(SNNMAP_ERR_INVALID, "bad offsets");
    int64_t *d_off = nullptr;
    int32_t *d_pins = nullptr, *d_w = nullptr, *d_rho = nullptr;
    cudaError_t e = snn::dev_malloc(&d_off, ((size_t)n_hedges + 1) * 8, s);
    if (e == cudaSuccess) e = snn::dev_malloc(&d_pins, (size_t)(P > 0 ? P : 1) * 4, s);
    if (e == cudaSuccess) e = snn::dev_malloc(&d_w, (size_t)(n_hedges > 0 ? n_hedges : 1) * 4, s);
    if (e == cudaSuccess) e = snn::dev_malloc(&d_rho, (size_t)(n_vertices > 0 ? n_vertices : 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, h_offsets, ((size_t)n_hedges + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && P > 0) e = cudaMemcpyAsync(d_pins, h_pins, (size_t)P * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_hedges > 0) e = cudaMemcpyAsync(d_w, h_w, (size_t)n_hedges * 4, cudaMemcpyHostToDevice, s);
    int rc = SNNMAP_OK;
    if (e != cudaSuccess) rc = fail(SNNMAP_ERR_CUDA, cudaGetErrorString(e));
    snnmap_hgraph* h = nullptr;
    if (rc == SNNMAP_OK) rc = snnmap_build_hgraph(params, n_vertices, n_hedges, d_off, d_pins, d_w, stream, &h);
    if (rc == SNNMAP_OK) rc = snnmap_partition(h, stream, d_rho, cost_out, stats);
    if (rc == SNNMAP_OK && n_vertices > 0) {
        e = cudaMemcpyAsync(h_rho_out, d_rho, (size_t)n_vertices * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(SNNMAP_ERR_CUDA, cudaGetErrorString(e));
    }
    std::string keep = g_err;
    if (h) snnmap_free(h);
    cudaFreeAsync(d_off, s);
    cudaFreeAsync(d_pins, s);
    cudaFreeAsync(d_w, s);
    cudaFreeAsync(d_rho, s);
    cudaStreamSynchronize(s);
    snn::pool_handles(0);   // hands the pool back when no handle is live
    g_err = keep;
    return rc;
}

int snnmap_level_copy(const snnmap_hgraph* h, int32_t level, int64_t* d_off, int32_t* d_pins,
                      int64_t* d_w, int32_t* d_k, uint8_t* d_selfdst, int32_t* d_size,
                      int32_t* d_inpins, int32_t* d_in_count, int32_t* d_in_internal, void* stream)
{
    g_err.clear();
    if (!h || level < 0 || level >= (int32_t)h->levels.size())
        return fail(SNNMAP_ERR_INVALID, "no such level");
    snnmap_hgraph* hm = const_cast<snnmap_hgraph*>(h);
    bind(hm, stream);
    API_TRY(snn::ensure_resident(hm, level));
    const snn::Level& L = h->levels[level];
    cudaStream_t s = (cudaStream_t)stream;
    struct Item {
        void* dst;
        const void* src;
        size_t bytes;
    } items[] = {
        {d_off, L.hoff, ((size_t)L.E + 1) * 8}, {d_pins, L.hpins, (size_t)L.P * 4},
        {d_w, L.hw, (size_t)L.E * 8},           {d_k, L.hk, (size_t)L.E * 4},
        {d_selfdst, L.hsd, (size_t)L.E},        {d_size, L.vsize, (size_t)L.V * 4},
        {d_inpins, L.vinpins, (size_t)L.V * 4}, {d_in_count, L.vincnt, (size_t)L.V * 4},
        {d_in_internal, L.vinint, (size_t)L.V * 4},
    };
    for (auto& it : items) {
        if (!it.dst || it.bytes == 0) continue;
        if (!is_device_ptr(it.dst)) return fail(SNNMAP_ERR_INVALID, "outputs must be device memory");
        cudaError_t e = cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return fail(SNNMAP_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SNNMAP_ERR_CUDA, cudaGetErrorString(e));
    return SNNMAP_OK;
}

int snnmap_last_matching(const snnmap_hgraph* h, int32_t* d_cand, int64_t* d_cscore, int32_t* d_cov,
                         int32_t* d_match, void* stream)
{
    g_err.clear();
    if (!h || !h->have_matching) return fail(SNNMAP_ERR_STATE, "no matching available");
    cudaStream_t s = (cudaStream_t)stream;
    size_t V = (size_t)h->levels.back().V;
    if (V == 0) return SNNMAP_OK;
    struct Item {
        void* dst;
        const void* src;
        size_t bytes;
    } items[] = {{d_cand, h->cand, V * 4}, {d_cscore, h->cscore, V * 8}, {d_cov, h->cov, V * 4},
                 {d_match, h->match, V * 4}};
    for (auto& it : items) {
        if (!it.dst) continue;
        if (!is_device_ptr(it.dst)) return fail(SNNMAP_ERR_INVALID, "outputs must be device memory");
        cudaError_t e = cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return fail(SNNMAP_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SNNMAP_ERR_CUDA, cudaGetErrorString(e));
    return SNNMAP_OK;
}

int snnmap_level_cid(const snnmap_hgraph* h, int32_t level, int32_t* d_cid, void* stream)
{
    g_err.clear();
    if (!h || level < 0 || level + 1 >= (int32_t)h->levels.size())
        return fail(SNNMAP_ERR_INVALID, "level has no coarser level");
    if (!is_device_ptr(d_cid)) return fail(SNNMAP_ERR_INVALID, "d_cid must be device memory");
    const snn::Level& L = h->levels[level];
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d_cid, L.cid, (size_t)L.V * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SNNMAP_ERR_CUDA, cudaGetErrorString(e));
    return SNNMAP_OK;
}

int snnmap_round_logs(const snnmap_hgraph* h, snnmap_round_log* out, int32_t cap, int32_t* n)
{
    if (!h || !n) return fail(SNNMAP_ERR_INVALID, "NULL argument");
    *n = (int32_t)h->rlog.size();
    for (int32_t i = 0; out && i < cap && i < *n; i++) out[i] = h->rlog[i];
    return SNNMAP_OK;
}

int snnmap_level_logs(const snnmap_hgraph* h, snnmap_level_log* out, int32_t cap, int32_t* n)
{
    if (!h || !n) return fail(SNNMAP_ERR_INVALID, "NULL argument");
    *n = (int32_t)h->llog.size();
    for (int32_t i = 0; out && i < cap && i < *n; i++) out[i] = h->llog[i];
    return SNNMAP_OK;
}

int snnmap_profile(snnmap_hgraph* h, int32_t on)
{
    if (!h) return fail(SNNMAP_ERR_INVALID, "NULL handle");
    cudaStreamSynchronize(h->stream);
    snn::prof_collect(h);
    if (on) {
        for (int i = 0; i < snn::PS_N; i++) {
            h->prof_ms[i] = 0;
            h->prof_calls[i] = 0;
        }
    }
    h->prof_on = on != 0;
    return SNNMAP_OK;
}

int snnmap_stage_times(snnmap_hgraph* h, snnmap_stage_time* out, int32_t cap, int32_t* n)
{
    if (!h || !n) return fail(SNNMAP_ERR_INVALID, "NULL argument");
    cudaStreamSynchronize(h->stream);
    snn::prof_collect(h);
    *n = snn::PS_N;
    for (int32_t i = 0; out && i < cap && i < snn::PS_N; i++) {
        out[i].name = snn::kStageNames[i];
        out[i].calls = h->prof_calls[i];
        out[i].ms = h->prof_ms[i];
    }
    return SNNMAP_OK;
}

int snnmap_device_bytes(const snnmap_hgraph* h, int64_t* bytes)
{
    if (!h || !bytes) return fail(SNNMAP_ERR_INVALID, "NULL argument");
    *bytes = snn::held_bytes(h);
    return SNNMAP_OK;
}

int snnmap_peak_bytes(const snnmap_hgraph* h, int64_t* bytes)
{
    if (!h || !bytes) return fail(SNNMAP_ERR_INVALID, "NULL argument");
    snn::note_bytes(const_cast<snnmap_hgraph*>(h));
    *bytes = h->peak_bytes;
    return SNNMAP_OK;
}

int snnmap_partition_graph(snnmap_hgraph* h, int32_t n_parts, const int32_t* d_rho, void* stream,
                           int32_t* n_hedges_out, int64_t* n_pins_out, int64_t* internal_out)
{
    g_err.clear();
    if (!h || !h->levels.size() || n_parts < 1) return fail(SNNMAP_ERR_INVALID, "bad arguments");
    if (h->levels[0].V > 0 && !is_device_ptr(d_rho))
        return fail(SNNMAP_ERR_INVALID, "d_rho must be device memory");
    bind(h, stream);
    API_TRY(snn::check_rho(h, 0, n_parts, d_rho));
    API_TRY(snn::emit_gp(h, n_parts, d_rho));
    if (n_hedges_out) *n_hedges_out = h->gp.E;
    if (n_pins_out) *n_pins_out = h->gp.P;
    if (internal_out) *internal_out = h->gp.internal;
    return SNNMAP_OK;
}

int snnmap_partition_graph_copy(const snnmap_hgraph* h, int64_t* d_offsets, int32_t* d_pins,
                                int64_t* d_eta, int32_t* d_axons, void* stream)
{
    g_err.clear();
    if (!h || !h->gp.hoff) return fail(SNNMAP_ERR_STATE, "no partition graph computed");
    const snn::GpOut& G = h->gp;
    cudaStream_t s = (cudaStream_t)stream;
    struct Item {
        void* dst;
        const void* src;
        size_t bytes;
    } items[] = {{d_offsets, G.hoff, ((size_t)G.E + 1) * 8}, {d_pins, G.hpins, (size_t)G.P * 4},
                 {d_eta, G.eta, (size_t)G.E * 8}, {d_axons, G.axons, (size_t)G.E * 4}};
    for (auto& it : items) {
        if (!it.dst || it.bytes == 0) continue;
        if (!is_device_ptr(it.dst)) return fail(SNNMAP_ERR_INVALID, "outputs must be device memory");
        cudaError_t e = cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return fail(SNNMAP_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SNNMAP_ERR_CUDA, cudaGetErrorString(e));
    return SNNMAP_OK;
}

int snnmap_set_row_budget(snnmap_hgraph* h, int64_t bytes)
{
    if (!h || bytes < -1) return fail(SNNMAP_ERR_INVALID, "bad arguments");
    h->row_budget = bytes;
    return SNNMAP_OK;
}

int snnmap_set_coarsen_mode(snnmap_hgraph* h, int32_t mode)
{
    g_err.clear();
    if (!h) return fail(SNNMAP_ERR_INVALID, "NULL handle");
    if (mode < 0 || mode > 2) return fail(SNNMAP_ERR_INVALID, "mode must be 0, 1 or 2");
    h->coarsen_mode = mode;
    if (mode == 1) h->icar.level = -1;
    return SNNMAP_OK;
}

int snnmap_set_tier_table(int32_t n, const int64_t* max_pins, const int64_t* wwork,
                          const int64_t* bwork, const int64_t* gwork)
{
    g_err.clear();
    if (n < 0 || (n > 0 && (!max_pins || !wwork || !bwork || !gwork)))
        return fail(SNNMAP_ERR_INVALID, "n < 0 or a NULL array");
    std::vector<TierRow> rows;
    try {
        for (int32_t i = 0; i < n; i++) {
            if (wwork[i] < 0 || bwork[i] < 0 || gwork[i] < 0 || (i > 0 && max_pins[i] <= max_pins[i - 1]))
                return fail(SNNMAP_ERR_INVALID, "negative thresholds or max_pins not increasing");
            rows.push_back(TierRow{max_pins[i], snn::HtTiers{wwork[i], bwork[i], gwork[i]}});
        }
    } catch (const std::bad_alloc&) {
        return fail(SNNMAP_ERR_OOM, "host allocation failed");
    }
    std::lock_guard<std::mutex> lk(g_tier_mu);
    g_tier_rows.swap(rows);
    return SNNMAP_OK;
}

int snnmap_set_histogram_tiers(snnmap_hgraph* h, int64_t wwork, int64_t bwork, int64_t gwork)
{
    g_err.clear();
    if (!h) return fail(SNNMAP_ERR_INVALID, "NULL handle");
    if (wwork >= 0) h->tiers.wwork = wwork;
    if (bwork >= 0) h->tiers.bwork = bwork;
    if (gwork >= 0) h->tiers.gwork = gwork;
    return SNNMAP_OK;
}

int snnmap_set_level_budget(snnmap_hgraph* h, int64_t bytes)
{
    if (!h || bytes < 0) return fail(SNNMAP_ERR_INVALID, "bad arguments");
    if (bytes == 0) {
        size_t fr = 0, tot = 0;
        bytes = cudaMemGetInfo(&fr, &tot) == cudaSuccess ? (int64_t)(tot * 2 / 5) : ((int64_t)1 << 34);
    }
    h->level_budget = bytes;
    h->keep_stride = 1;
    snn::thin_levels(h);
    return SNNMAP_OK;
}

// The entry points above never let a C++ exception (a failed host
// allocation inside a standard container) cross the C ABI.
int snnmap_build_hgraph(const snnmap_params* params, int32_t n_vertices, int32_t n_hedges,
                        const int64_t* d_offsets, const int32_t* d_pins, const int32_t* d_w,
                        void* stream, snnmap_hgraph** out)
{
    try {
        return snnmap_build_hgraph_impl(params, n_vertices, n_hedges, d_offsets, d_pins, d_w, stream, out);
    } catch (const std::bad_alloc&) {
        return fail(SNNMAP_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(SNNMAP_ERR_CUDA, "internal error");
    }
}

int snnmap_coarsen_level(snnmap_hgraph* h, void* stream, int32_t* n_cand_out, int32_t* n_pairs_out)
{
    try {
        return snnmap_coarsen_level_impl(h, stream, n_cand_out, n_pairs_out);
    } catch (const std::bad_alloc&) {
        return fail(SNNMAP_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(SNNMAP_ERR_CUDA, "internal error");
    }
}

int snnmap_contract(snnmap_hgraph* h, void* stream, int32_t* V_out, int32_t* E_out, int64_t* P_out)
{
    try {
        return snnmap_contract_impl(h, stream, V_out, E_out, P_out);
    } catch (const std::bad_alloc&) {
        return fail(SNNMAP_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(SNNMAP_ERR_CUDA, "internal error");
    }
}

int snnmap_refine(snnmap_hgraph* h, int32_t level, int32_t n_parts, int32_t* d_rho, void* stream,
                  int64_t* cost_out)
{
    try {
        return snnmap_refine_impl(h, level, n_parts, d_rho, stream, cost_out);
    } catch (const std::bad_alloc&) {
        return fail(SNNMAP_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(SNNMAP_ERR_CUDA, "internal error");
    }
}

int snnmap_partition(snnmap_hgraph* h, void* stream, int32_t* d_rho_out, int64_t* cost_out,
                     snnmap_stats* stats)
{
    try {
        return snnmap_partition_impl(h, stream, d_rho_out, cost_out, stats);
    } catch (const std::bad_alloc&) {
        return fail(SNNMAP_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(SNNMAP_ERR_CUDA, "internal error");
    }
}

int snnmap_partition_host(const snnmap_params* params, int32_t n_vertices, int32_t n_hedges,
                          const int64_t* h_offsets, const int32_t* h_pins, const int32_t* h_w,
                          int32_t* h_rho_out, int64_t* cost_out, snnmap_stats* stats, void* stream)
{
    try {
        return snnmap_partition_host_impl(params, n_vertices, n_hedges, h_offsets, h_pins, h_w, h_rho_out, cost_out, stats, stream);
    } catch (const std::bad_alloc&) {
        return fail(SNNMAP_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(SNNMAP_ERR_CUDA, "internal error");
    }
}

}  // extern "C"
