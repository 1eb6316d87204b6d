// Batch / serving runner: many independent scenes advanced concurrently.
//
// A batch owns W worker threads, each with its own CUDA stream.  Admitted
// scenes (jobs) are bound to the stream of the worker with the least
// pending work; a worker advances its jobs one time step at a time in
// round-robin order, so scenes admitted while others run join at the next
// round (continuous batching) and the kernels of W scenes overlap on the
// device.  Admission is refused (BF_E_BUDGET) when the device bytes of the
// unfinished jobs plus the new scene would exceed the batch's HBM budget.
// With autotuning on (bf_batch_set_autotune), the PCG execution
// configuration is tuned once per size bucket (log2 of the matrix block
// count, which grows with the vertex count): the first scene of a bucket is
// tuned after its first step (bf_autotune_pcg, on its worker), and every
// scene of the bucket takes that configuration at its next turn.
// The runner only uses the public scene API; the time steps are the same
// calls a single scene makes (Alg. 1 per step), so a scene's result does not
// depend on what else runs beside it beyond the order of floating-point
// atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "bf.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    int64_t ticket = 0;
    bf_scene *scene = nullptr;
    int n_steps = 0, done = 0, status = BF_OK, worker = 0;
    int64_t bytes = 0, work = 0;  // device bytes; work estimate per step
    int bucket = 0, mode = -1;    // autotuning size bucket; PCG mode set by the runner (-1: default)
    double t_admit = 0.0;
    std::vector<double> t_step;  // completion time of each step (s since batch creation)
    std::vector<bf_step_stats> stats;
    bool finished = false;
};

}  // namespace

struct bf_batch {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> threads;
    std::vector<cudaStream_t> streams;
    std::vector<std::deque<Job *>> queues;  // unfinished jobs per worker
    std::vector<int64_t> pending;           // pending work per worker
    std::unordered_map<int64_t, std::unique_ptr<Job>> jobs;
    int64_t budget = 0, resident = 0, next_ticket = 1;
    int device = 0, finished = 0;
    bool stop = false;
    bool autotune = false;
    bool blocking = false;  // admitted scenes wait with blocking-sync events
    std::unordered_map<int, int> tuned;  // size bucket -> PCG mode
    std::unordered_set<int> tuning;     // buckets being tuned right now
    Clock::time_point epoch;

    double now() const { return std::chrono::duration<double>(Clock::now() - epoch).count(); }

    void work(int w)
    {
        cudaSetDevice(device);
        for (;;) {
            Job *job = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || !queues[w].empty(); });
                if (stop) return;
                job = queues[w].front();
                queues[w].pop_front();
            }
            int apply = -1;
            bool tune = false;
            if (autotune) {
                std::lock_guard<std::mutex> lk(mu);
                auto it = tuned.find(job->bucket);
                if (it != tuned.end()) {
                    if (job->mode != it->second) apply = it->second;
                } else if (job->done >= 1 && !tuning.count(job->bucket)) {
                    tuning.insert(job->bucket);  // this worker tunes the bucket
                    tune = true;
                }
            }
            if (apply >= 0 && bf_set_pcg_mode(job->scene, apply) == BF_OK) job->mode = apply;
            if (tune) {  // the scene has assembled a system in its first step
                int32_t best = -1;
                const int rc = bf_autotune_pcg(job->scene, 32, 0, nullptr, nullptr, nullptr, &best);
                std::lock_guard<std::mutex> lk(mu);
                if (rc == BF_OK && best >= 0) {
                    tuned[job->bucket] = best;
                    job->mode = best;
                }
                tuning.erase(job->bucket);
            }
            bf_step_stats st{};
            const int rc = bf_step(job->scene, 1, &st);
            const double t = now();
            std::lock_guard<std::mutex> lk(mu);
            job->t_step.push_back(t);
            job->stats.push_back(st);
            ++job->done;
            pending[w] -= job->work;
            if (rc != BF_OK || job->done >= job->n_steps) {
                job->status = rc;
                job->finished = true;
                pending[w] -= job->work * (job->n_steps - job->done);
                resident -= job->bytes;
                ++finished;
                cv_done.notify_all();
            } else {
                queues[w].push_back(job);  // round robin: one step per turn
            }
        }
    }
};

extern "C" {

int bf_batch_create(int32_t n_workers, int64_t hbm_budget_bytes, bf_batch **out)
{
    if (!out || n_workers < 1 || n_workers > 256 || hbm_budget_bytes <= 0) return BF_E_ARG;
    auto b = std::make_unique<bf_batch>();
    if (cudaGetDevice(&b->device) != cudaSuccess) return BF_E_CUDA;
    b->budget = hbm_budget_bytes;
    b->epoch = Clock::now();
    b->queues.resize(n_workers);
    b->pending.assign(n_workers, 0);
    for (int w = 0; w < n_workers; ++w) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t t : b->streams) cudaStreamDestroy(t);
            return BF_E_CUDA;
        }
        b->streams.push_back(s);
    }
    bf_batch *p = b.release();
    for (int w = 0; w < n_workers; ++w) p->threads.emplace_back([p, w] { p->work(w); });
    *out = p;
    return BF_OK;
}

int bf_batch_destroy(bf_batch *b)
{
    if (!b) return BF_E_ARG;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->stop = true;
    }
    b->cv_work.notify_all();
    for (auto &t : b->threads) t.join();
    for (auto &kv : b->jobs) bf_set_stream(kv.second->scene, nullptr);  // unreleased scenes: default stream
    for (cudaStream_t s : b->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    delete b;
    return BF_OK;
}

int bf_batch_admit(bf_batch *b, bf_scene *scene, int32_t n_steps, int64_t *ticket)
{
    if (!b || !scene || n_steps < 1 || !ticket) return BF_E_ARG;
    int64_t bytes = 0;
    int32_t info[5] = {0, 0, 0, 0, 0};
    int rc = bf_scene_bytes(scene, &bytes);
    if (!rc) rc = bf_scene_info(scene, info);
    if (rc) return rc;
    const int64_t work = (int64_t)info[3] + 1;  // matrix blocks: a proxy for the work of one step
    int bucket = 0;
    while ((int64_t)1 << (bucket + 1) <= work) ++bucket;  // floor(log2(blocks + 1))
    std::unique_lock<std::mutex> lk(b->mu);
    if (b->stop) return BF_E_ARG;
    if (b->resident + bytes > b->budget) return BF_E_BUDGET;
    const int w = (int)(std::min_element(b->pending.begin(), b->pending.end()) - b->pending.begin());
    b->resident += bytes;  // reserved before the lock is dropped
    b->pending[w] += work * n_steps;
    lk.unlock();
    rc = bf_set_stream(scene, b->streams[w]);  // the scene is not running yet
    if (!rc && b->blocking) rc = bf_set_sync_mode(scene, 1);
    lk.lock();
    if (rc) {
        b->resident -= bytes;
        b->pending[w] -= work * n_steps;
        return rc;
    }
    auto job = std::make_unique<Job>();
    job->ticket = b->next_ticket++;
    job->scene = scene;
    job->n_steps = n_steps;
    job->worker = w;
    job->bytes = bytes;
    job->work = work;
    job->bucket = bucket;
    job->t_admit = b->now();
    job->t_step.reserve(n_steps);
    job->stats.reserve(n_steps);
    b->queues[w].push_back(job.get());
    *ticket = job->ticket;
    b->jobs.emplace(job->ticket, std::move(job));
    lk.unlock();
    b->cv_work.notify_all();
    return BF_OK;
}

int bf_batch_wait(bf_batch *b, int64_t ticket, int32_t timeout_ms, int32_t *done)
{
    if (!b || !done) return BF_E_ARG;
    std::unique_lock<std::mutex> lk(b->mu);
    auto it = b->jobs.find(ticket);
    if (it == b->jobs.end()) return BF_E_NOT_FOUND;
    Job *job = it->second.get();
    auto pred = [&] { return job->finished; };
    if (timeout_ms < 0) b->cv_done.wait(lk, pred);
    else b->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
    *done = job->finished ? 1 : 0;
    return BF_OK;
}

int bf_batch_result(bf_batch *b, int64_t ticket, int32_t cap, int32_t *steps_done, int32_t *status, double *t_admit,
                    double *t_steps, bf_step_stats *stats)
{
    if (!b || cap < 0) return BF_E_ARG;
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->jobs.find(ticket);
    if (it == b->jobs.end()) return BF_E_NOT_FOUND;
    const Job *job = it->second.get();
    if (steps_done) *steps_done = job->done;
    if (status) *status = job->status;
    if (t_admit) *t_admit = job->t_admit;
    const int n = std::min<int>(cap, (int)job->t_step.size());
    for (int i = 0; i < n; ++i) {
        if (t_steps) t_steps[i] = job->t_step[i];
        if (stats) stats[i] = job->stats[i];
    }
    return BF_OK;
}

int bf_batch_release(bf_batch *b, int64_t ticket)
{
    if (!b) return BF_E_ARG;
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->jobs.find(ticket);
    if (it == b->jobs.end()) return BF_E_NOT_FOUND;
    if (!it->second->finished) return BF_E_ARG;
    bf_set_stream(it->second->scene, nullptr);  // the scene goes back to the default stream
    bf_set_sync_mode(it->second->scene, 0);
    b->jobs.erase(it);
    return BF_OK;
}

int bf_batch_info(bf_batch *b, int64_t *info)
{
    if (!b || !info) return BF_E_ARG;
    std::lock_guard<std::mutex> lk(b->mu);
    int64_t queued = 0;
    for (auto &q : b->queues) queued += (int64_t)q.size();
    info[0] = b->resident;
    info[1] = b->budget;
    info[2] = (int64_t)b->threads.size();
    info[3] = queued;
    info[4] = b->finished;
    info[5] = b->next_ticket - 1;
    return BF_OK;
}

double bf_batch_now(bf_batch *b) { return b ? b->now() : -1.0; }

int bf_batch_set_blocking_sync(bf_batch *b, int32_t on)
{
    if (!b) return BF_E_ARG;
    std::lock_guard<std::mutex> lk(b->mu);
    b->blocking = on != 0;
    return BF_OK;
}

int bf_batch_set_autotune(bf_batch *b, int32_t on)
{
    if (!b) return BF_E_ARG;
    std::lock_guard<std::mutex> lk(b->mu);
    b->autotune = on != 0;
    return BF_OK;
}

int bf_batch_tuned(bf_batch *b, int32_t cap, int32_t *buckets, int32_t *modes, int32_t *n)
{
    if (!b || cap < 0 || (cap > 0 && (!buckets || !modes))) return BF_E_ARG;
    std::lock_guard<std::mutex> lk(b->mu);
    std::vector<std::pair<int, int>> v(b->tuned.begin(), b->tuned.end());
    std::sort(v.begin(), v.end());
    for (int i = 0; i < (int)v.size() && i < cap; ++i) {
        buckets[i] = v[i].first;
        modes[i] = v[i].second;
    }
    if (n) *n = (int)v.size();
    return BF_OK;
}

}  // extern "C"
