// Serving engine: layout requests of mixed sizes, admitted by the device
// memory their k-hop lists need, run concurrently on the GPU.
//
// Two threads serve a queue of jobs:
//   admission  takes the smallest waiting job (fewest adjacency entries,
//              then the earliest); uploads the graph, counts its k-hop lists
//              (exact size, before any list memory exists), waits until the
//              job's device bytes fit the budget and a slot is free, then
//              fills the lists, frees the build scratch, plans the blocked
//              path and uploads the placement. A job that can never fit
//              fails with GILA_EBUDGET.
//   runner     keeps every admitted job's placement and temperature resident
//              on the device and advances them by least remaining work
//              (pairs per iteration times iterations left, shrunk by the
//              time the job has waited, and overdue jobs first, so that
//              none starves): each round it
//              enqueues the next chunk of iterations of the jobs in that
//              order on each job's own stream (at most two chunks in flight
//              per job) while their work per iteration stays below what
//              fills the GPU, so small jobs run side by side and overtake
//              large ones, whose kernels alone fill the GPU; chunks are cut
//              to a bounded amount of work so that a newly admitted job
//              waits at most about a millisecond for the GPU; finished jobs
//              are copied back, their memory is returned and waiters are
//              woken.
// Requests arriving while others run are admitted as soon as memory and a
// slot free up (continuous batching). A job runs exactly the kernels it
// would run alone, so its result does not depend on the mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gila_impl.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Job {
    uint64_t ticket = 0;
    int64_t n = 0;
    std::vector<int64_t> row;
    std::vector<int32_t> col;
    std::vector<double> pos_in;
    std::vector<double> pos_out;
    gila_params prm{};
    // device state (owned by the server threads)
    gila_graph* g = nullptr;
    cudaStream_t st = nullptr;
    void* pos[2] = {nullptr, nullptr};
    double* stage = nullptr;  // double[2n] upload/download
    double* host = nullptr;   // pinned copy of the result
    cudaEvent_t chunk_ev[2] = {nullptr, nullptr};
    cudaEvent_t done_ev = nullptr;
    int chunks_issued = 0;
    int next_iter = 0;
    int chunk_iters = 8;  // iterations per chunk (fewer for jobs with large iterations)
    bool download_issued = false;
    double t0 = 0.0;
    size_t bytes = 0;
    int64_t nnz_khop = 0;
    // outcome
    gila_status status = GILA_OK;
    std::string error;
    bool finished = false;
    Clock::time_point t_submit, t_admit, t_done;
};

using JobPtr = std::shared_ptr<Job>;

}  // namespace

struct gila_server {
    size_t budget = 0;
    int max_slots = 1;
    int chunk = 8;  // iterations per job per round
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_admit;  // admission: new job or freed capacity
    std::condition_variable cv_run;    // runner: new admitted job
    std::condition_variable cv_done;   // waiters
    std::deque<JobPtr> pending;
    std::deque<JobPtr> admitted;  // admission -> runner
    std::map<uint64_t, JobPtr> jobs;
    size_t in_use = 0, peak = 0;
    int slots_used = 0;
    uint64_t next_ticket = 1;
    int64_t completed = 0, failed = 0;
    std::atomic<bool> stop{false};
    std::thread admission, runner;
};

namespace gila {
namespace {

size_t pos_size(int precision) { return is_f64(precision) ? 16 : 8; }

// Device bytes a job holds while it runs (upper estimate, exact list size).
size_t job_bytes(int64_t n, int64_t nnz_adj, int64_t nnz_khop, int precision,
                 const gila_tuning& tune)
{
    const size_t esz = pos_size(precision);
    size_t b = 0;
    b += 16 * (size_t)(n + 1) + 4 * (size_t)nnz_adj;   // adjacency CSR + k-hop offsets
    b += 4 * (size_t)nnz_khop;                          // k-hop ids
    b += 12 * (size_t)n;                                // row classes, spare
    b += 2 * esz * (size_t)n + 16 * (size_t)n;          // placement buffers, staging
    {
        // window-mode layout (graphs whose ranges fit shared-memory windows):
        // 16-bit ids with each row padded by at most 7 entries, each range's
        // block by at most 15 per thread of its CTA, and per row an offset
        const int64_t nr = std::min<int64_t>(8 * 152, std::max<int64_t>(1, (nnz_khop + 8 * n) / 16384));
        b += 2 * (size_t)(nnz_khop + 7 * n) + 8 * (size_t)n + 2 * 15 * 1024 * (size_t)nr;
    }
    if (blocked_auto_applies(n, nnz_khop, esz, tune)) {
        // blocked-path plan: the ids once more in block order as 16-bit
        // tile-relative ids (each row's segment per tile padded by at most 7
        // entries, each block by at most 15 per thread of its CTA), and per
        // row and tile an offset, a length and a partial force
        const int64_t tv = (200 * 1024) / (int64_t)esz;
        const int64_t nt = (n + tv - 1) / std::max<int64_t>(tv, 1);
        const int64_t nr = std::max<int64_t>(8 * 152 / nt + 1, n / 4096 + 1);
        b += 2 * (size_t)nnz_khop + (14 + 16 + 2 * esz) * (size_t)n * (size_t)nt + (1 << 16);
        b += 2 * 15 * 1024 * (size_t)(nt * nr);
    }
    return b + ((size_t)1 << 20);
}

// Per-iteration work (k-hop plus adjacency entries) of the jobs already
// running beyond which a job that has not started waits: about what keeps
// the GPU busy on its own (measured: a Barabasi-Albert graph with 1.4e7
// k-hop entries already runs at 70% of the largest graphs' pair rate).
constexpr double kSaturationPairs = 2e7;
// Pair interactions per chunk of a job's iterations: about a millisecond of
// GPU time, the longest a newly admitted small job waits behind a chunk.
constexpr double kChunkPairs = 5e8;
// Waiting time (s) over which a job's remaining work counts for half in the
// runner's order (aging, so that large jobs are not starved).
constexpr double kAgeSeconds = 0.5;
// Pair interactions per second of a job alone (about the rate of the
// single-graph kernels on mid-size graphs), and the slack before a job
// counts as overdue.
constexpr double kAloneRate = 1e12;
constexpr double kOverdueSeconds = 0.12;

void finish_job(gila_server* s, const JobPtr& j, gila_status st, const std::string& err)
{
    std::lock_guard<std::mutex> lock(s->mu);
    j->status = st;
    j->error = err;
    j->finished = true;
    j->t_done = Clock::now();
    if (st == GILA_OK) ++s->completed; else ++s->failed;
    s->cv_done.notify_all();
}

void free_job_device(gila_server* s, const JobPtr& j)
{
    if (j->st) cudaStreamSynchronize(j->st);
    for (cudaEvent_t& e : j->chunk_ev)
        if (e) cudaEventDestroy(e), e = nullptr;
    if (j->done_ev) cudaEventDestroy(j->done_ev), j->done_ev = nullptr;
    cudaFree(j->pos[0]);
    cudaFree(j->pos[1]);
    cudaFree(j->stage);
    j->pos[0] = j->pos[1] = nullptr;
    j->stage = nullptr;
    if (j->host) cudaFreeHost(j->host), j->host = nullptr;
    if (j->g) gila_graph_destroy(j->g), j->g = nullptr;
    if (j->st) cudaStreamDestroy(j->st), j->st = nullptr;
    std::lock_guard<std::mutex> lock(s->mu);
    if (j->bytes) {
        s->in_use -= j->bytes;
        s->slots_used -= 1;
        j->bytes = 0;
        s->cv_admit.notify_all();
    }
}

gila_status check_cuda(cudaError_t e, const char* what, std::string* err)
{
    if (e == cudaSuccess) return GILA_OK;
    *err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GILA_ENOMEM : GILA_ECUDA;
}

// Upload, count, wait for room, fill, place. Returns with the job admitted
// (bytes reserved) or failed.
gila_status admit_job(gila_server* s, const JobPtr& j, std::string* err)
{
    gila_status st;
    if ((st = check_cuda(cudaStreamCreateWithFlags(&j->st, cudaStreamNonBlocking), "stream", err)))
        return st;
    st = gila_graph_create(j->n, j->row.data(), j->col.data(), 0, &j->g);
    if (st != GILA_OK) {
        *err = gila_last_error();
        return st;
    }
    gila_graph_set_stream(j->g, j->st);
    j->g->ks.scratch_cap = std::max<size_t>((size_t)64 << 20, s->budget / 8);
    j->g->ks.keep_balls = false;  // nothing held between count and fill beyond the scratch
    int64_t nnz = 0;
    st = build_khop_count(j->g, j->prm.k, &nnz);
    if (st != GILA_OK) {
        *err = gila_last_error();
        return st;
    }
    const size_t need = job_bytes(j->n, j->g->nnz_adj, nnz, j->prm.precision, j->g->tune);
    if (need > s->budget) {
        *err = "job needs " + std::to_string(need) + " device bytes, budget is " +
               std::to_string(s->budget);
        return GILA_EBUDGET;
    }
    {
        std::unique_lock<std::mutex> lock(s->mu);
        s->cv_admit.wait(lock, [&] {
            return s->stop.load() ||
                   (s->in_use + need <= s->budget && s->slots_used < s->max_slots);
        });
        if (s->stop.load()) {
            *err = "server stopped";
            return GILA_ESTATE;
        }
        s->in_use += need;
        s->slots_used += 1;
        s->peak = std::max(s->peak, s->in_use);
        j->bytes = need;
    }
    invalidate_tile_plans(j->g);
    st = build_khop_fill(j->g, j->prm.k);
    if (st != GILA_OK) {
        *err = gila_last_error();
        return st;
    }
    j->g->nnz_khop = nnz;
    j->g->k_built = j->prm.k;
    j->nnz_khop = nnz;
    release_khop_scratch(j->g);
    // plan the blocked path here, not on the runner thread
    if ((st = prepare_iteration(j->g, &j->prm)) != GILA_OK) {
        *err = gila_last_error();
        return st;
    }
    // a chunk holds at most about kChunkPairs pair interactions (one
    // iteration at least, eight at most)
    {
        const double per_iter = (double)(nnz + j->g->nnz_adj) + 1.0;
        j->chunk_iters = (int)std::max(1.0, std::min(8.0, kChunkPairs / per_iter));
    }
    const size_t n = (size_t)j->n;
    const size_t esz = pos_size(j->prm.precision);
    if (n > 0) {
        if ((st = check_cuda(cudaMalloc(&j->pos[0], esz * n), "placement", err))) return st;
        if ((st = check_cuda(cudaMalloc(&j->pos[1], esz * n), "placement", err))) return st;
        if ((st = check_cuda(cudaMallocHost(&j->host, 16 * n), "pinned result", err))) return st;
        if (!is_f64(j->prm.precision)) {
            if ((st = check_cuda(cudaMalloc(&j->stage, 16 * n), "staging", err))) return st;
            cudaMemcpyAsync(j->stage, j->pos_in.data(), 16 * n, cudaMemcpyHostToDevice, j->st);
            st = convert_positions(j->g, j->prm.precision, j->stage, j->pos[0], true);
        } else {
            cudaMemcpyAsync(j->pos[0], j->pos_in.data(), 16 * n, cudaMemcpyHostToDevice, j->st);
        }
        if (st != GILA_OK) {
            *err = gila_last_error();
            return st;
        }
    }
    // initial temperature of this job
    if (j->prm.t0 > 0.0) {
        j->t0 = j->prm.t0;
    } else if (j->prm.schedule != GILA_COOL_GEOMETRIC) {
        j->t0 = 0.1 * std::sqrt((double)j->n);
    } else {
        double a = 1.0;
        if (n > 0 && (st = bbox_aspect(j->g, j->prm.precision, j->pos[0], &a)) != GILA_OK) {
            *err = gila_last_error();
            return st;
        }
        j->t0 = std::sqrt((double)j->n * j->prm.d / a);
    }
    for (cudaEvent_t& e : j->chunk_ev)
        if ((st = check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event", err)))
            return st;
    if ((st = check_cuda(cudaEventCreateWithFlags(&j->done_ev, cudaEventDisableTiming), "event",
                         err)))
        return st;
    return check_cuda(cudaGetLastError(), "admission", err);
}

void admission_loop(gila_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        JobPtr j;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_admit.wait(lock, [&] { return s->stop.load() || !s->pending.empty(); });
            if (s->stop.load()) return;
            // the smallest waiting job first (ties: the earliest)
            auto best = s->pending.begin();
            for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
                if ((*it)->col.size() < (*best)->col.size()) best = it;
            j = *best;
            s->pending.erase(best);
        }
        std::string err;
        const gila_status st = admit_job(s, j, &err);
        if (st != GILA_OK) {
            free_job_device(s, j);
            finish_job(s, j, st, err);
            continue;
        }
        std::lock_guard<std::mutex> lock(s->mu);
        j->t_admit = Clock::now();
        s->admitted.push_back(j);
        s->cv_run.notify_all();
    }
}

double temperature_of(const Job& j, int i)
{
    if (j.prm.schedule == GILA_COOL_GEOMETRIC) return j.t0 * std::pow(0.93, (double)i);
    return j.t0 * (double)(j.prm.iters - i) / (double)j.prm.iters;
}

// Enqueue the next chunk of j's iterations; false when nothing could be done.
bool advance(gila_server* s, Job& j, std::string* err, gila_status* st)
{
    const int iters = j.prm.iters;
    if (j.next_iter < iters) {
        // at most two chunks in flight per job
        if (j.chunks_issued >= 2 &&
            cudaEventQuery(j.chunk_ev[j.chunks_issued & 1]) == cudaErrorNotReady)
            return false;
        const int end = std::min(iters, j.next_iter + std::min(s->chunk, j.chunk_iters));
        for (int i = j.next_iter; i < end; ++i) {
            *st = launch_iteration(j.g, &j.prm, temperature_of(j, i), j.pos[i & 1],
                                   j.pos[(i + 1) & 1], nullptr);
            if (*st != GILA_OK) {
                *err = gila_last_error();
                return false;
            }
        }
        j.next_iter = end;
        cudaEventRecord(j.chunk_ev[j.chunks_issued & 1], j.st);
        ++j.chunks_issued;
        return true;
    }
    if (!j.download_issued) {
        const size_t n = (size_t)j.n;
        void* result = j.pos[iters & 1];
        if (n > 0) {
            if (is_f64(j.prm.precision)) {
                cudaMemcpyAsync(j.host, result, 16 * n, cudaMemcpyDeviceToHost, j.st);
            } else {
                *st = convert_positions(j.g, j.prm.precision, j.stage, result, false);
                if (*st != GILA_OK) {
                    *err = gila_last_error();
                    return false;
                }
                cudaMemcpyAsync(j.host, j.stage, 16 * n, cudaMemcpyDeviceToHost, j.st);
            }
        }
        cudaEventRecord(j.done_ev, j.st);
        j.download_issued = true;
        return true;
    }
    return false;
}

void runner_loop(gila_server* s)
{
    cudaSetDevice(s->device);
    std::vector<JobPtr> active;
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (active.empty())
                s->cv_run.wait(lock, [&] { return s->stop.load() || !s->admitted.empty(); });
            if (s->stop.load() && s->admitted.empty() && active.empty()) return;
            while (!s->admitted.empty()) {
                active.push_back(s->admitted.front());
                s->admitted.pop_front();
            }
        }
        bool progressed = false;
        // least remaining work first (aged by the time waited): jobs are
        // advanced in that order while the work per iteration issued this
        // round leaves the GPU short of work; the first job always runs
        {
            const Clock::time_point now = Clock::now();
            auto key = [&](const JobPtr& j) {
                const double per_iter = (double)(j->nnz_khop + j->g->nnz_adj) + 1.0;
                const double left = per_iter * (double)(j->prm.iters - j->next_iter + 1);
                const double age = std::chrono::duration<double>(now - j->t_submit).count();
                // a job waiting for more than twice its time alone (at
                // kAloneRate pairs per second) plus kOverdueSeconds goes
                // first, oldest first: smaller jobs cannot hold back a large
                // one indefinitely (48 requests at 2x load: p99 569 -> 495 ms,
                // against 538 ms for FIFO service)
                const double alone = per_iter * (double)j->prm.iters / kAloneRate;
                if (age > 2.0 * alone + kOverdueSeconds) return -1e30 - 1e20 * age;
                return left / (1.0 + age / kAgeSeconds);
            };
            std::vector<std::pair<double, size_t>> order;
            for (size_t i = 0; i < active.size(); ++i) order.emplace_back(key(active[i]), i);
            std::stable_sort(order.begin(), order.end(),
                             [](const std::pair<double, size_t>& a,
                                const std::pair<double, size_t>& b) { return a.first < b.first; });
            std::vector<JobPtr> sorted;
            for (auto& o : order) sorted.push_back(active[o.second]);
            active.swap(sorted);
        }
        double running_work = 0.0;
        for (size_t i = 0; i < active.size();) {
            JobPtr j = active[i];
            std::string err;
            gila_status st = GILA_OK;
            if (s->stop.load()) {
                free_job_device(s, j);
                finish_job(s, j, GILA_ESTATE, "server stopped");
                active.erase(active.begin() + i);
                continue;
            }
            if (!j->download_issued && running_work >= kSaturationPairs) {
                ++i;
                continue;
            }
            if (!j->download_issued) running_work += (double)(j->nnz_khop + j->g->nnz_adj);
            if (advance(s, *j, &err, &st)) progressed = true;
            if (st != GILA_OK) {
                free_job_device(s, j);
                finish_job(s, j, st, err);
                active.erase(active.begin() + i);
                continue;
            }
            if (j->download_issued) {
                const cudaError_t q = cudaEventQuery(j->done_ev);
                if (q == cudaSuccess) {
                    j->pos_out.assign(j->host, j->host + 2 * (size_t)j->n);
                    free_job_device(s, j);
                    finish_job(s, j, GILA_OK, "");
                    active.erase(active.begin() + i);
                    progressed = true;
                    continue;
                }
                if (q != cudaErrorNotReady) {
                    std::string e2 = std::string("job: ") + cudaGetErrorString(q);
                    cudaGetLastError();
                    free_job_device(s, j);
                    finish_job(s, j, GILA_ECUDA, e2);
                    active.erase(active.begin() + i);
                    continue;
                }
            }
            ++i;
        }
        if (!progressed && !active.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace
}  // namespace gila

using namespace gila;

extern "C" {

gila_status gila_server_create(size_t mem_budget_bytes, int32_t max_slots, gila_server** out)
{
    if (!out) return fail(GILA_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_slots < 1) return fail(GILA_EINVAL, "max_slots must be >= 1");
    if (mem_budget_bytes == 0) return fail(GILA_EINVAL, "memory budget must be > 0");
    gila_server* s = new (std::nothrow) gila_server();
    if (!s) return fail(GILA_ENOMEM, "host allocation");
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaGetDevice");
    }
    s->budget = mem_budget_bytes;
    s->max_slots = max_slots;
    s->admission = std::thread(admission_loop, s);
    s->runner = std::thread(runner_loop, s);
    *out = s;
    return GILA_OK;
}

void gila_server_destroy(gila_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv_admit.notify_all();
        s->cv_run.notify_all();
        s->cv_done.notify_all();
    }
    if (s->admission.joinable()) s->admission.join();
    if (s->runner.joinable()) s->runner.join();
    for (auto& kv : s->jobs) free_job_device(s, kv.second);
    for (auto& j : s->admitted) free_job_device(s, j);
    delete s;
}

gila_status gila_server_submit(gila_server* s, int64_t n, const int64_t* row_ptr,
                               const int32_t* col_idx, const gila_params* prm,
                               const double* pos_in, uint64_t* ticket)
{
    if (!s || !prm || !ticket) return fail(GILA_EINVAL, "server, params or ticket is NULL");
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(GILA_EINVAL, "n out of range");
    if (!row_ptr || (n > 0 && !pos_in)) return fail(GILA_EINVAL, "array is NULL");
    if (prm->k < 1 || prm->k > 64 || prm->iters < 0 || !(prm->d > 0.0) ||
        (prm->precision != GILA_FP32 && prm->precision != GILA_FP64 &&
         prm->precision != GILA_FP32_COMPENSATED) ||
        prm->p < 0 || prm->p > 8 || prm->q < 0 || prm->q > 8 ||
        (prm->schedule != GILA_COOL_LINEAR && prm->schedule != GILA_COOL_GEOMETRIC))
        return fail(GILA_EINVAL, "invalid parameters");
    auto j = std::make_shared<Job>();
    j->n = n;
    const int64_t nnz = row_ptr[n] - row_ptr[0];
    if (nnz < 0 || (nnz > 0 && !col_idx)) return fail(GILA_EINVAL, "malformed CSR");
    j->row.assign(row_ptr, row_ptr + n + 1);
    for (auto& r : j->row) r -= row_ptr[0];
    j->col.assign(col_idx + row_ptr[0], col_idx + row_ptr[0] + nnz);
    {
        gila_status bs = check_csr_bounds(n, j->row.data(), j->col.data());
        if (bs != GILA_OK) return bs;
    }
    if (n > 0) j->pos_in.assign(pos_in, pos_in + 2 * n);
    j->prm = *prm;
    j->t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop.load()) return fail(GILA_ESTATE, "server stopped");
    j->ticket = s->next_ticket++;
    s->jobs[j->ticket] = j;
    s->pending.push_back(j);
    s->cv_admit.notify_all();
    *ticket = j->ticket;
    return GILA_OK;
}

gila_status gila_server_wait(gila_server* s, uint64_t ticket, int32_t timeout_ms,
                             double* pos_out, gila_job_info* info)
{
    if (!s) return fail(GILA_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return fail(GILA_EINVAL, "unknown ticket " + std::to_string(ticket));
    JobPtr j = it->second;
    auto ready = [&] { return j->finished; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lock, ready);
    } else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) {
        return fail(GILA_ETIMEDOUT, "job " + std::to_string(ticket) + " not finished");
    }
    s->jobs.erase(it);
    if (info) {
        info->status = j->status;
        info->nnz_khop = j->nnz_khop;
        info->queue_ms = j->status == GILA_OK ? ms_between(j->t_submit, j->t_admit) : 0.0;
        info->run_ms = j->status == GILA_OK ? ms_between(j->t_admit, j->t_done) : 0.0;
        info->latency_ms = ms_between(j->t_submit, j->t_done);
    }
    if (j->status != GILA_OK) return fail(j->status, j->error);
    if (pos_out && j->n > 0) memcpy(pos_out, j->pos_out.data(), sizeof(double) * 2 * j->n);
    return GILA_OK;
}

gila_status gila_server_poll(gila_server* s, uint64_t ticket, int32_t* done)
{
    if (!s || !done) return fail(GILA_EINVAL, "server or done is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return fail(GILA_EINVAL, "unknown ticket " + std::to_string(ticket));
    *done = it->second->finished ? 1 : 0;
    return GILA_OK;
}

gila_status gila_server_get_stats(gila_server* s, gila_server_stats* out)
{
    if (!s || !out) return fail(GILA_EINVAL, "server or out is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    out->completed = s->completed;
    out->failed = s->failed;
    out->pending = (int64_t)s->pending.size();
    out->running = s->slots_used;
    out->bytes_in_use = s->in_use;
    out->bytes_peak = s->peak;
    out->budget = s->budget;
    return GILA_OK;
}

}  // extern "C"
