// Continuous-batching layout server.
//
// A worker thread owns one stream and runs "ticks". Each tick it admits queued
// requests in arrival order while their working memory fits the budget (and,
// for jobs that need the whole GPU, while a slot is free), then advances every
// admitted job by one chunk of iterations:
//   - exact jobs of at most 16,384 vertices and n^2 x iterations <= 2.5e9 share
//     one persistent batched launch (one CTA per graph, 50 iterations per tick);
//   - larger exact jobs and Barnes-Hut jobs take the whole GPU for a chunk whose
//     length depends only on the job's size and mode (about 25 ms of work).
// Jobs that finish are copied to host memory and their device memory returns to
// the budget at once, so requests that arrive while others run are admitted as
// memory and slots free up. A job's chunk boundaries depend only on the job, and
// both engines give the same positions however the iterations are split, so a
// result is the same alone and in any mix.
// Each whole-GPU job has a stream of its own. A tick first queues a chunk of every
// whole-GPU job, each on its stream, then the batched launch on the worker's
// stream, and only then waits for them: the jobs' work overlaps on the device
// (Barnes-Hut iterations of mid-size graphs leave most of the GPU idle while their
// sweeps wait on dependency chains). The engines' grid-wide waits need all of a
// kernel's CTAs resident; next to other kernels some may start late, which only
// delays a wait (every wait is bounded, and the kernels sharing the GPU are
// chunks of about 25 ms that need nothing from it).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bl_internal.cuh"

namespace bl {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kSmallChunk = 50;          // iterations per tick of a batched job
constexpr int kBigSlots = 4;             // whole-GPU jobs admitted at a time (BL_SERVE_SLOTS overrides)
constexpr double kBigChunkMs = 25.0;     // target work per whole-GPU chunk
constexpr int kAutoExactBelow = 50000;   // BL_AUTO: exact below this many vertices
constexpr double kBatchedWorkMax = 2.5e9; // n^2 x iterations of a job the batched launch takes

enum class JobState { Queued, Active, Done, Failed, Canceled };

struct Job {
    uint64_t ticket = 0;
    const bl_graph* g = nullptr;
    uint64_t seed = 0;
    int iters = 0, BS = 0, chunk = 1, done = 0;
    bl_mode mode = BL_EXACT;
    float theta = 1.2f;
    bool small = false;
    size_t bytes = 0;
    bl_layout* L = nullptr;
    JobState state = JobState::Queued;
    bl_status err = BL_OK;
    std::string msg;
    Clock::time_point t_submit, t_done;
    std::vector<float> result;
    cudaStream_t st = nullptr;   // whole-GPU jobs: the job's own stream (else the worker's)
};

// Working memory a job holds on the device while admitted.
size_t job_bytes(const Job& j) {
    const size_t n = (size_t)j.g->n;
    const size_t it = (size_t)j.iters;
    // Barnes-Hut: 17 n + 1 tree-node slots of 64 B (build fields, sums, walk
    // records, level buckets) and ~110 B per vertex of sort, sweep and positions
    if (j.mode == BL_BH) return 1200 * n + 16 * it + (4u << 20);
    if (j.small) return 8 * n + 8 * it + 4096;
    return 16 * n + 8 * it + (size_t)8 * 160 * j.chunk + 65536;
}

// Iterations per chunk of a whole-GPU job, from its size and mode alone.
int big_chunk(const Job& j) {
    const double n = (double)j.g->n;
    const double ms_per_it = j.mode == BL_BH ? 7.5e-6 * n / 1.0e3 + 0.3 : n * n / 2.5e9 + 0.05;
    const int c = (int)(kBigChunkMs / ms_per_it);
    return std::max(1, std::min(c, 100));
}

}  // namespace
}  // namespace bl

using namespace bl;

struct bl_server {
    int device = 0;
    int big_slots = kBigSlots;
    cudaStream_t st = nullptr;
    size_t budget = 0, in_use = 0, peak = 0;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::thread worker;
    uint64_t next_ticket = 1;
    std::deque<Job*> queue;
    std::vector<Job*> active;
    std::unordered_map<uint64_t, Job*> jobs;
    std::vector<double> latencies;
    uint64_t completed = 0;
};

namespace {

bl_status read_status(bl_layout* L, cudaStream_t st) {
    int v = 0;
    BL_CUDA_TRY(cudaMemcpyAsync(&v, L->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BL_CUDA_TRY(cudaStreamSynchronize(st));
    if (v != 0) {
        cudaMemsetAsync(L->status.p, 0, sizeof(int), st);
        return set_error((bl_status)v, "a bounded device-side wait timed out");
    }
    return BL_OK;
}

// Ends a job (done or failed): result to host, device memory back to the budget.
void retire(bl_server* S, Job* j, bl_status err) {
    cudaStream_t st = j->st ? j->st : S->st;
    if (err == BL_OK && j->L) {
        j->result.resize(2 * (size_t)j->g->n);
        cudaError_t e = cudaMemcpyAsync(j->result.data(), j->L->pos.p, j->result.size() * sizeof(float),
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) err = cuda_error(e, "server: result copy");
    }
    if (err != BL_OK && j->msg.empty()) j->msg = bl_last_error();
    if (j->L) {
        cudaStreamSynchronize(st);   // nothing of the job may still be running
        layout_destroy(j->L);
    }
    j->L = nullptr;
    if (j->st) {
        cudaStreamDestroy(j->st);
        j->st = nullptr;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    j->t_done = Clock::now();
    S->in_use -= j->bytes;
    S->active.erase(std::remove(S->active.begin(), S->active.end(), j), S->active.end());
    if (err == BL_OK) {
        j->state = JobState::Done;
        S->latencies.push_back(std::chrono::duration<double>(j->t_done - j->t_submit).count());
        S->completed++;
    } else {
        j->state = JobState::Failed;
        j->err = err;
        j->result.clear();
    }
}

void worker_main(bl_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Job*> admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->active.empty(); });
            if (S->stop) break;
            int big_active = 0;
            for (Job* j : S->active) big_active += j->small ? 0 : 1;
            while (!S->queue.empty()) {
                Job* j = S->queue.front();
                if (S->in_use + j->bytes > S->budget) break;
                if (!j->small && big_active >= S->big_slots) break;
                S->queue.pop_front();
                S->in_use += j->bytes;
                S->peak = std::max(S->peak, S->in_use);
                j->state = JobState::Active;
                big_active += j->small ? 0 : 1;
                S->active.push_back(j);
                admitted.push_back(j);
            }
        }
        for (Job* j : admitted) {
            bl_status s = BL_OK;
            if (!j->small) {
                const cudaError_t e = cudaStreamCreateWithFlags(&j->st, cudaStreamNonBlocking);
                if (e != cudaSuccess) {
                    j->st = nullptr;
                    s = cuda_error(e, "server: job stream");
                }
            }
            if (s == BL_OK) s = layout_create(j->g, nullptr, j->seed, 0, nullptr, true, j->st ? j->st : S->st, &j->L);
            if (s != BL_OK) {
                j->msg = bl_last_error();
                retire(S, j, s);   // j may be deleted by a poll from here on
            }
        }
        // The jobs of this tick, split before anything runs: once a job is retired
        // a poll may delete it, so no job is touched after its own retire().
        std::vector<BatchJob> bj;
        std::vector<Job*> bjobs, big;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Job* j : S->active) {
                if (j->small) {
                    bj.push_back(BatchJob{j->L, std::min(kSmallChunk, j->iters - j->done), j->BS});
                    bjobs.push_back(j);
                } else {
                    big.push_back(j);
                }
            }
        }
        // one tick: a chunk of each whole-GPU job queued on its stream, then the
        // batched launch (which waits for its own stream only), then the jobs' ends
        std::vector<int> its(big.size(), 0);
        std::vector<bl_status> issued(big.size(), BL_OK);
        for (size_t q = 0; q < big.size(); q++) {
            Job* j = big[q];
            its[q] = std::min(j->chunk, j->iters - j->done);
            issued[q] = j->mode == BL_EXACT ? exact_run(j->L, its[q], j->BS, false, nullptr, j->st)
                                            : bh_run(j->L, its[q], j->BS, j->theta, j->st, false);
        }
        if (!bj.empty()) {
            const bl_status s = batch_launch(bj.data(), (int)bj.size(), 0, S->st);
            for (size_t q = 0; q < bjobs.size(); q++) {
                Job* j = bjobs[q];
                if (s != BL_OK) {
                    retire(S, j, s);
                    continue;
                }
                j->done += bj[q].iters;
                if (j->done >= j->iters) retire(S, j, BL_OK);
            }
        }
        for (size_t q = 0; q < big.size(); q++) {
            Job* j = big[q];
            const int it = its[q];
            bl_status s = issued[q];
            if (s == BL_OK) s = read_status(j->L, j->st);
            if (s != BL_OK) {
                retire(S, j, s);
                continue;
            }
            const double n = (double)j->g->n;
            j->L->t += it;
            j->L->last_iters = it;
            j->L->vupd += n * it;
            if (j->mode == BL_EXACT) j->L->pairs += n * (n - 1.0) * it;
            j->done += it;
            if (j->done >= j->iters) retire(S, j, BL_OK);
        }
    }
    // shutdown: drop what is still admitted
    std::vector<Job*> left;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        left = S->active;
    }
    cudaStreamSynchronize(S->st);
    for (Job* j : left) {
        if (j->st) cudaStreamSynchronize(j->st);
        if (j->L) layout_destroy(j->L);
        j->L = nullptr;
        if (j->st) cudaStreamDestroy(j->st);
        j->st = nullptr;
    }
}

}  // namespace

extern "C" {

bl_status bl_server_create(size_t mem_budget_bytes, bl_server** out) {
    if (!out) return set_error(BL_EINVAL, "bl_server_create: out is NULL");
    *out = nullptr;
    if (mem_budget_bytes == 0) return set_error(BL_EINVAL, "bl_server_create: budget must be positive");
    bl_server* S = new bl_server();
    S->budget = mem_budget_bytes;
    if (const char* e = std::getenv("BL_SERVE_SLOTS")) S->big_slots = std::max(1, std::min(64, std::atoi(e)));
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete S;
        return cuda_error(e, "bl_server_create");
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return BL_OK;
}

bl_status bl_serve_submit(bl_server* S, const bl_graph* g, uint64_t seed, int32_t iters, int32_t batch,
                          bl_mode mode, float theta, uint64_t* ticket) {
    if (!S || !g || !ticket) return set_error(BL_EINVAL, "bl_serve_submit: NULL argument");
    if (iters < 0) return set_error(BL_EINVAL, "bl_serve_submit: iters < 0");
    if (batch < 1 || batch > kMaxBatch) return set_error(BL_EINVAL, "bl_serve_submit: batch must be in [1, 8192]");
    if (mode != BL_EXACT && mode != BL_BH && mode != BL_AUTO)
        return set_error(BL_EINVAL, "bl_serve_submit: bad mode");
    if (mode == BL_AUTO) mode = g->n < kAutoExactBelow ? BL_EXACT : BL_BH;
    if (mode == BL_BH && !(theta >= 0.0f)) return set_error(BL_EINVAL, "bl_serve_submit: theta must be >= 0");
    if (mode == BL_BH && (int64_t)g->n > kBHMaxN)
        return set_error(BL_EINVAL, "bl_serve_submit: graph too large for Barnes-Hut mode");
    Job* j = new Job();
    j->g = g;
    j->seed = seed;
    j->iters = iters;
    j->BS = batch;
    j->mode = mode;
    j->theta = theta;
    // one CTA holds a batched job for all its iterations: above about 0.1 s of one
    // SM's work, the whole GPU finishes the job sooner
    j->small = mode == BL_EXACT && g->n <= kBatchMaxN && batch <= kBatchMaxBS &&
               (double)g->n * g->n * iters <= kBatchedWorkMax;
    j->chunk = j->small ? kSmallChunk : big_chunk(*j);
    j->bytes = job_bytes(*j);
    if (j->bytes > S->budget) {
        delete j;
        return set_error(BL_EBUDGET, "bl_serve_submit: the request needs more memory than the server's budget");
    }
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        j->ticket = S->next_ticket++;
        S->jobs[j->ticket] = j;
        if (iters == 0) {   // nothing to run: done with the seeded positions
            j->state = JobState::Done;
            j->result.resize(2 * (size_t)g->n);
            seeded_positions(g->n, seed, j->result.data());
            j->t_done = j->t_submit;
            S->latencies.push_back(0.0);
            S->completed++;
        } else {
            S->queue.push_back(j);
        }
        *ticket = j->ticket;
    }
    S->cv.notify_one();
    return BL_OK;
}

bl_status bl_serve_poll(bl_server* S, uint64_t ticket, float* xy, int64_t cap, double* latency_s) {
    if (!S) return set_error(BL_EINVAL, "bl_serve_poll: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return set_error(BL_EINVAL, "bl_serve_poll: unknown ticket");
    Job* j = it->second;
    switch (j->state) {
        case JobState::Queued:
        case JobState::Active:
            return BL_ENOTREADY;
        case JobState::Canceled:
            S->jobs.erase(it);
            delete j;
            return set_error(BL_ECANCELED, "bl_serve_poll: the request was canceled");
        case JobState::Failed: {
            const bl_status e = j->err;
            const std::string msg = j->msg;
            S->jobs.erase(it);
            delete j;
            return set_error(e, "bl_serve_poll: the request failed: " + msg);
        }
        case JobState::Done:
            break;
    }
    if (!xy || cap < (int64_t)j->result.size())
        return set_error(BL_EINVAL, "bl_serve_poll: output needs 2n floats");
    std::memcpy(xy, j->result.data(), j->result.size() * sizeof(float));
    if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
    S->jobs.erase(it);
    delete j;
    return BL_OK;
}

bl_status bl_serve_cancel(bl_server* S, uint64_t ticket) {
    if (!S) return set_error(BL_EINVAL, "bl_serve_cancel: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return set_error(BL_EINVAL, "bl_serve_cancel: unknown ticket");
    Job* j = it->second;
    if (j->state != JobState::Queued)
        return set_error(BL_EBUSY, "bl_serve_cancel: the request is already on the GPU or finished");
    S->queue.erase(std::remove(S->queue.begin(), S->queue.end(), j), S->queue.end());
    j->state = JobState::Canceled;
    return BL_OK;
}

bl_status bl_server_stats(bl_server* S, double* out, int64_t cap) {
    if (!S || !out) return set_error(BL_EINVAL, "bl_server_stats: NULL argument");
    if (cap < 6) return set_error(BL_EINVAL, "bl_server_stats: output needs 6 doubles");
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> lat = S->latencies;
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
        if (lat.empty()) return 0.0;
        const size_t k = (size_t)std::min<double>((double)lat.size() - 1, std::ceil(p * lat.size()) - 1);
        return lat[k];
    };
    out[0] = (double)S->completed;
    out[1] = (double)S->active.size();
    out[2] = (double)S->queue.size();
    out[3] = (double)S->in_use;
    out[4] = pct(0.50);
    out[5] = pct(0.99);
    if (cap >= 7) out[6] = (double)S->peak;
    return BL_OK;
}

void bl_server_free(bl_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->jobs) delete kv.second;
    if (S->st) cudaStreamDestroy(S->st);
    delete S;
}

}  // extern "C"
