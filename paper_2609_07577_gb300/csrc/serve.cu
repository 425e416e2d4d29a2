// Batched and served forms (snnmap_serve_* and snnmap_batch_partition in
// include/snnmap.h): a host scheduler that runs independent mapping jobs on
// one GPU at once.
//
// Each worker slot is one host thread with its own non-blocking CUDA stream.
// A worker takes the job at the head of the FIFO queue when the job's
// predicted footprint fits in the memory budget next to the footprints
// already reserved (or when nothing is reserved), runs the whole pass of
// snnmap_partition for it on its stream, and marks it done. The pass reads a
// few scalars back to the host per level, so one job alone leaves the GPU
// idle between its small kernels; jobs on other slots fill those gaps.
// Results are the single-job results: every job has its own handle, and
// nothing in a job's arithmetic depends on the others.
#include "internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>

namespace {

using Clock = std::chrono::steady_clock;

// Device bytes of one level as level_alloc lays it out (arrays rounded up
// to 256 bytes) plus its cid map.
int64_t level_bytes(int64_t V, int64_t E, int64_t P)
{
    auto r = [](int64_t b) { return ((b > 0 ? b : 1) + 255) / 256 * 256; };
    return r(8 * (E + 1)) + 2 * r(4 * P) + r(8 * E) + 2 * r(4 * E) + r(E) + r(8 * (V + 1)) +
           4 * r(4 * V) + r(4 * V) + 4096;
}

// Footprint model of one pass: level 0, the newest contracted level (at most
// the size of level 0), the intermediate levels kept under a budget of one
// level 0, the scratch arena (sort buffers, pin counts and the hash-table
// pools, which the histogram engine bounds by max(64 MiB, 4 bytes per pin)),
// the per-vertex matching arrays, a fixed allowance for the arena's 64 MiB
// minimum chunk and the split tier's minimum pool, and the job's budget for
// refinement connection rows and the coarsening score matrix.
constexpr int64_t kFootLevels = 3;
constexpr int64_t kFootScratch = 3;
constexpr int64_t kFootFixed = (int64_t)160 << 20;

// connection rows / score matrix memory granted to a job (part of its
// footprint)
int64_t job_row_budget(int64_t L0) { return 4 * L0 + ((int64_t)256 << 20); }

int64_t input_bytes(int64_t V, int64_t E, int64_t P)
{
    return 8 * (E + 1) + 4 * P + 4 * E + 4 * V;
}

int64_t footprint(int64_t V, int64_t E, int64_t P, bool on_host)
{
    int64_t L0 = level_bytes(V, E, P);
    // 20 B per vertex of candidate arrays, 17 B of carried candidates, and the
    // refinement's column update of short prefixes (16 slots of 12 B, 16 B of
    // flags and saves per vertex, 8 B per hyperedge)
    int64_t f = (kFootLevels + kFootScratch) * L0 + (20 + 17 + 208) * V + 8 * E + kFootFixed +
                job_row_budget(L0);
    if (on_host) f += input_bytes(V, E, P);
    return f;
}

struct Ticket {
    int64_t id = 0;
    snnmap_job* job = nullptr;
    int64_t fp = 0;
    int64_t rows = 0;              // row budget granted to the job
    int state = 0;                 // 0 queued, 1 running, 2 done
    snnmap_hgraph* h = nullptr;    // kept hierarchy
};

void set_err(snnmap_job* j, const char* msg)
{
    std::strncpy(j->error, msg ? msg : "", sizeof(j->error) - 1);
    j->error[sizeof(j->error) - 1] = 0;
}

}  // namespace

struct snnmap_server {
    int device = 0;
    int32_t slots = 8;
    int32_t dry_us = 0;
    int64_t budget = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Ticket*> queue;
    std::map<int64_t, Ticket*> tickets;
    int64_t next_id = 1;
    int64_t reserved = 0;
    int32_t running = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;

    double now_ms() const
    {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }
    bool admissible(const Ticket* t) const { return reserved == 0 || reserved + t->fp <= budget; }
    // row budget of a job: at least the footprint model's, and a quarter of
    // the memory budget shared by the slots (power-law jobs refine from
    // connection rows at most levels with it)
    int64_t row_grant(int64_t L0) const
    {
        int64_t share = budget / (4 * (int64_t)slots);
        return std::max(job_row_budget(L0), share);
    }
    void work(int slot);
    void run(Ticket* t, int slot);
};

void snnmap_server::run(Ticket* t, int slot)
{
    snnmap_job* j = t->job;
    j->slot = slot;
    if (dry_us > 0) {
        int64_t P = j->offsets && j->n_hedges >= 0 && j->on_host ? j->offsets[j->n_hedges] : 0;
        int64_t us = std::max<int64_t>(1000, (int64_t)dry_us * (P / 1000000 + 1));
        std::this_thread::sleep_for(std::chrono::microseconds(us));
        j->status = SNNMAP_OK;
        j->peak_bytes = 0;
        return;
    }
    cudaStream_t s = streams[slot];
    const int64_t* off = j->offsets;
    const int32_t *pins = j->pins, *w = j->w;
    int32_t* rho = j->rho_out;
    int64_t *d_off = nullptr;
    int32_t *d_pins = nullptr, *d_w = nullptr, *d_rho = nullptr;
    int64_t in_bytes = 0;
    int rc = SNNMAP_OK;
    std::string msg;
    if (j->on_host) {
        int64_t E = j->n_hedges, V = j->n_vertices;
        int64_t P = off[E];
        if (off[0] != 0 || P < 0) {
            rc = SNNMAP_ERR_INVALID;
            msg = "bad offsets";
        } else {
            in_bytes = input_bytes(V, E, P);
            cudaError_t e = snn::dev_malloc(&d_off, (size_t)(E + 1) * 8, s);
            if (e == cudaSuccess) e = snn::dev_malloc(&d_pins, (size_t)(P > 0 ? P : 1) * 4, s);
            if (e == cudaSuccess) e = snn::dev_malloc(&d_w, (size_t)(E > 0 ? E : 1) * 4, s);
            if (e == cudaSuccess) e = snn::dev_malloc(&d_rho, (size_t)(V > 0 ? V : 1) * 4, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off, (size_t)(E + 1) * 8, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && P > 0)
                e = cudaMemcpyAsync(d_pins, pins, (size_t)P * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && E > 0)
                e = cudaMemcpyAsync(d_w, w, (size_t)E * 4, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                rc = e == cudaErrorMemoryAllocation ? SNNMAP_ERR_OOM : SNNMAP_ERR_CUDA;
                msg = cudaGetErrorString(e);
            }
            off = d_off;
            pins = d_pins;
            w = d_w;
            rho = d_rho;
        }
    }
    snnmap_hgraph* h = nullptr;
    if (rc == SNNMAP_OK) {
        rc = snnmap_build_hgraph(&j->params, j->n_vertices, j->n_hedges, off, pins, w, s, &h);
        if (rc != SNNMAP_OK) msg = snnmap_last_error();
    }
    if (rc == SNNMAP_OK) {
        int64_t L0 = level_bytes(j->n_vertices, j->n_hedges, h->levels[0].P);
        snnmap_set_level_budget(h, L0);
        snnmap_set_row_budget(h, t->rows);
        rc = snnmap_partition(h, s, rho, &j->cost, &j->stats);
        if (rc != SNNMAP_OK) msg = snnmap_last_error();
    }
    if (rc == SNNMAP_OK && j->on_host && j->n_vertices > 0) {
        cudaError_t e = cudaMemcpyAsync(j->rho_out, d_rho, (size_t)j->n_vertices * 4,
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = SNNMAP_ERR_CUDA;
            msg = cudaGetErrorString(e);
        }
    }
    int64_t peak = 0;
    if (h) snnmap_peak_bytes(h, &peak);
    j->peak_bytes = peak + in_bytes;
    if (d_off) cudaFreeAsync(d_off, s);
    if (d_pins) cudaFreeAsync(d_pins, s);
    if (d_w) cudaFreeAsync(d_w, s);
    if (d_rho) cudaFreeAsync(d_rho, s);
    if (h && (rc != SNNMAP_OK || !j->keep_hierarchy)) {
        snnmap_free(h);
        h = nullptr;
    }
    cudaStreamSynchronize(s);
    t->h = h;
    j->status = rc;
    set_err(j, rc == SNNMAP_OK ? "" : msg.c_str());
}

void snnmap_server::work(int slot)
{
    if (dry_us == 0) cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv_work.wait(lk, [&] { return stop || (!queue.empty() && admissible(queue.front())); });
        if (stop) return;
        Ticket* t = queue.front();
        queue.pop_front();
        reserved += t->fp;
        running++;
        t->state = 1;
        t->job->t_start_ms = now_ms();
        lk.unlock();
        try {
            run(t, slot);
        } catch (...) {
            // a failed host allocation ends this job, not the process
            t->h = nullptr;
            t->job->status = SNNMAP_ERR_OOM;
            set_err(t->job, "host allocation failed");
        }
        lk.lock();
        t->job->t_end_ms = now_ms();
        t->state = 2;
        running--;
        if (!t->h) reserved -= t->fp;
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

extern "C" {

int snnmap_job_footprint(int32_t n_vertices, int32_t n_hedges, int64_t n_pins, int32_t on_host,
                         int64_t* bytes)
{
    if (n_vertices < 0 || n_hedges < 0 || n_pins < 0 || !bytes) {
        snn::set_last_error("negative sizes or NULL output");
        return SNNMAP_ERR_INVALID;
    }
    *bytes = footprint(n_vertices, n_hedges, n_pins, on_host != 0);
    return SNNMAP_OK;
}

int snnmap_serve_create(const snnmap_serve_opts* opts, snnmap_server** out)
{
    if (!out) {
        snn::set_last_error("out is NULL");
        return SNNMAP_ERR_INVALID;
    }
    *out = nullptr;
    snnmap_serve_opts o{};
    if (opts) o = *opts;
    if (o.slots < 0 || o.slots > 256 || o.dry_run_us < 0 || o.mem_budget < 0) {
        snn::set_last_error("slots must lie in [0, 256]; dry_run_us and mem_budget >= 0");
        return SNNMAP_ERR_INVALID;
    }
    snnmap_server* s = new (std::nothrow) snnmap_server;
    if (!s) {
        snn::set_last_error("host allocation failed");
        return SNNMAP_ERR_OOM;
    }
    s->slots = o.slots ? o.slots : 8;
    s->dry_us = o.dry_run_us;
    s->t0 = Clock::now();
    if (s->dry_us == 0) {
        cudaError_t e = cudaGetDevice(&s->device);
        size_t fr = 0, tot = 0;
        if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) {
            snn::set_last_error(cudaGetErrorString(e));
            delete s;
            return SNNMAP_ERR_CUDA;
        }
        s->budget = o.mem_budget ? o.mem_budget : (int64_t)(fr / 5 * 4);
        s->streams.resize(s->slots);
        for (int i = 0; i < s->slots; i++) {
            e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                for (int k = 0; k < i; k++) cudaStreamDestroy(s->streams[k]);
                snn::set_last_error(cudaGetErrorString(e));
                delete s;
                return SNNMAP_ERR_CUDA;
            }
        }
    } else {
        s->budget = o.mem_budget ? o.mem_budget : ((int64_t)1 << 36);
    }
    for (int i = 0; i < s->slots; i++) s->workers.emplace_back([s, i] { s->work(i); });
    *out = s;
    return SNNMAP_OK;
}

int snnmap_serve_submit(snnmap_server* s, snnmap_job* job, int64_t* ticket)
{
    if (!s || !job || job->n_vertices < 0 || job->n_hedges < 0 || !job->offsets || !job->rho_out ||
        (job->n_hedges > 0 && (!job->pins || !job->w))) {
        snn::set_last_error("NULL server, job or buffer, or negative sizes");
        return SNNMAP_ERR_INVALID;
    }
    int64_t P = 0;
    if (job->on_host) P = job->offsets[job->n_hedges];
    else if (s->dry_us == 0) {
        cudaError_t e = cudaMemcpy(&P, job->offsets + job->n_hedges, sizeof(int64_t),
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            snn::set_last_error(cudaGetErrorString(e));
            return SNNMAP_ERR_CUDA;
        }
    }
    Ticket* t = new (std::nothrow) Ticket;
    if (!t) {
        snn::set_last_error("host allocation failed");
        return SNNMAP_ERR_OOM;
    }
    t->job = job;
    {
        int64_t Pc = P < 0 ? 0 : P;
        int64_t L0 = level_bytes(job->n_vertices, job->n_hedges, Pc);
        t->rows = s->row_grant(L0);
        t->fp = footprint(job->n_vertices, job->n_hedges, Pc, job->on_host != 0) - job_row_budget(L0) +
                t->rows;
    }
    job->footprint = t->fp;
    job->cost = 0;
    job->stats = snnmap_stats{};
    job->peak_bytes = 0;
    job->status = -1;
    job->slot = -1;
    job->error[0] = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete t;
            snn::set_last_error("server is shutting down");
            return SNNMAP_ERR_STATE;
        }
        t->id = s->next_id++;
        job->t_submit_ms = s->now_ms();
        s->tickets[t->id] = t;
        s->queue.push_back(t);
    }
    s->cv_work.notify_all();
    if (ticket) *ticket = t->id;
    return SNNMAP_OK;
}

int snnmap_serve_wait(snnmap_server* s, int64_t ticket, double timeout_ms, int32_t* done)
{
    if (!s) {
        snn::set_last_error("NULL server");
        return SNNMAP_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        snn::set_last_error("unknown ticket");
        return SNNMAP_ERR_INVALID;
    }
    Ticket* t = it->second;
    auto pred = [&] { return t->state == 2; };
    if (timeout_ms < 0) s->cv_done.wait(lk, pred);
    else
        s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred);
    if (done) *done = t->state == 2;
    return SNNMAP_OK;
}

int snnmap_serve_hgraph(snnmap_server* s, int64_t ticket, snnmap_hgraph** out)
{
    if (!s || !out) {
        snn::set_last_error("NULL argument");
        return SNNMAP_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        snn::set_last_error("unknown ticket");
        return SNNMAP_ERR_INVALID;
    }
    if (it->second->state != 2 || !it->second->h) {
        snn::set_last_error("job not done, failed, or submitted without keep_hierarchy");
        return SNNMAP_ERR_STATE;
    }
    *out = it->second->h;
    return SNNMAP_OK;
}

int snnmap_serve_release(snnmap_server* s, int64_t ticket)
{
    if (!s) {
        snn::set_last_error("NULL server");
        return SNNMAP_ERR_INVALID;
    }
    Ticket* t = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) {
            snn::set_last_error("unknown ticket");
            return SNNMAP_ERR_INVALID;
        }
        if (it->second->state != 2) {
            snn::set_last_error("job not done");
            return SNNMAP_ERR_STATE;
        }
        t = it->second;
        s->tickets.erase(it);
        if (t->h) s->reserved -= t->fp;
    }
    if (t->h) snnmap_free(t->h);
    delete t;
    s->cv_work.notify_all();
    return SNNMAP_OK;
}

int snnmap_serve_info(snnmap_server* s, int32_t* queued, int32_t* running, int64_t* reserved)
{
    if (!s) {
        snn::set_last_error("NULL server");
        return SNNMAP_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int32_t)s->queue.size();
    if (running) *running = s->running;
    if (reserved) *reserved = s->reserved;
    return SNNMAP_OK;
}

int snnmap_serve_destroy(snnmap_server* s)
{
    if (!s) return SNNMAP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Ticket* t : s->queue) {
            t->job->status = SNNMAP_ERR_STATE;
            set_err(t->job, "server destroyed before the job started");
            t->state = 2;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    for (auto& th : s->workers) th.join();
    s->cv_done.notify_all();
    for (auto& kv : s->tickets) {
        if (kv.second->h) snnmap_free(kv.second->h);
        delete kv.second;
    }
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete s;
    snn::pool_handles(0);   // hands the pool back when no handle is live
    return SNNMAP_OK;
}

int snnmap_batch_partition(snnmap_job* jobs, int32_t n_jobs, const snnmap_serve_opts* opts)
{
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) {
        snn::set_last_error("bad job array");
        return SNNMAP_ERR_INVALID;
    }
    snnmap_server* s = nullptr;
    int rc = snnmap_serve_create(opts, &s);
    if (rc != SNNMAP_OK) return rc;
    // largest first, so the longest jobs do not start last
    std::vector<int64_t> pins(n_jobs, 0);
    for (int32_t i = 0; i < n_jobs; i++) {
        const snnmap_job& j = jobs[i];
        if (!j.offsets || j.n_hedges < 0) continue;
        if (j.on_host) pins[i] = j.offsets[j.n_hedges];
        else if (!(opts && opts->dry_run_us > 0) &&
                 cudaMemcpy(&pins[i], j.offsets + j.n_hedges, sizeof(int64_t),
                            cudaMemcpyDeviceToHost) != cudaSuccess)
            pins[i] = 0;
    }
    std::vector<int32_t> order(n_jobs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return pins[a] > pins[b]; });
    std::vector<int64_t> tk(n_jobs, 0);
    int first_bad = SNNMAP_OK;
    for (int32_t i : order) {
        jobs[i].keep_hierarchy = 0;
        int r = snnmap_serve_submit(s, &jobs[i], &tk[i]);
        if (r != SNNMAP_OK) {
            jobs[i].status = r;
            set_err(&jobs[i], snnmap_last_error());
            tk[i] = 0;
        }
    }
    for (int32_t i = 0; i < n_jobs; i++) {
        if (tk[i]) {
            snnmap_serve_wait(s, tk[i], -1.0, nullptr);
            snnmap_serve_release(s, tk[i]);
        }
        if (first_bad == SNNMAP_OK && jobs[i].status != SNNMAP_OK) first_bad = jobs[i].status;
    }
    snnmap_serve_destroy(s);
    if (first_bad != SNNMAP_OK) snn::set_last_error("a job failed; see its status and error");
    return first_bad;
}

}  // extern "C"
