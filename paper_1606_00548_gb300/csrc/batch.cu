// Ensemble runtime: many independent simulators (geological realisations on
// grids of different sizes) advanced together on one GPU.
//
// Each member owns a CUDA stream and replays its FGMRES restart cycles as a
// CUDA graph; a pool of persistent host worker threads drives the members'
// Newton loops, so the kernels of different members overlap on the device
// (a single member of ~10^5 cells leaves most of the 152 SMs idle between
// its latency-bound launches).  Members never exchange data.
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "sim_internal.cuh"

struct sim_batch {
    std::vector<sim_t *> members;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    // current job
    const double *dt = nullptr;
    sim_step_info *infos = nullptr;
    std::vector<sim_status> status;
    std::atomic<int> next{0};
    int active = 0;          // workers still working on the current job
    int64_t generation = 0;  // job counter
    bool quit = false;
    int nthreads = 0;
};

static void worker_main(sim_batch *b) {
    int64_t seen = 0;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(b->mu);
            b->cv_work.wait(lk, [&] { return b->quit || b->generation != seen; });
            if (b->quit) return;
            seen = b->generation;
        }
        for (;;) {
            const int k = b->next.fetch_add(1);
            if (k >= (int)b->members.size()) break;
            sim_step_info info;
            memset(&info, 0, sizeof(info));
            b->status[k] = sim_step(b->members[k], b->dt[k], &info);
            if (b->infos) b->infos[k] = info;
        }
        {
            std::lock_guard<std::mutex> lk(b->mu);
            if (--b->active == 0) b->cv_done.notify_all();
        }
    }
}

extern "C" {

sim_status sim_batch_create(int32_t n, sim_t *const *members, int32_t nthreads, sim_batch_t **out) {
    if (!out || n < 1 || !members) return sim_fail(nullptr, SIM_EINVAL, "sim_batch_create: bad arguments");
    *out = nullptr;
    for (int k = 0; k < n; k++)
        if (!members[k]) return sim_fail(nullptr, SIM_EINVAL, "sim_batch_create: NULL member");
    for (int k = 0; k < n; k++)
        for (int j = 0; j < k; j++)
            if (members[k]->stream == members[j]->stream)
                return sim_fail(nullptr, SIM_EINVAL, "sim_batch_create: members must own distinct streams");
    sim_batch *b = new sim_batch();
    b->members.assign(members, members + n);
    b->status.assign(n, SIM_OK);
    b->nthreads = nthreads > 0 ? (nthreads < n ? nthreads : n) : (n < 64 ? n : 64);
    for (int t = 0; t < b->nthreads; t++) b->workers.emplace_back(worker_main, b);
    *out = b;
    return SIM_OK;
}

void sim_batch_destroy(sim_batch_t *b) {
    if (!b) return;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->quit = true;
    }
    b->cv_work.notify_all();
    for (auto &t : b->workers) t.join();
    delete b;
}

sim_status sim_batch_step(sim_batch_t *b, const double *dt, sim_step_info *infos, sim_status *member_status) {
    if (!b || !dt) return SIM_EINVAL;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->dt = dt;
        b->infos = infos;
        b->next.store(0);
        b->active = b->nthreads;
        b->generation++;
    }
    b->cv_work.notify_all();
    {
        std::unique_lock<std::mutex> lk(b->mu);
        b->cv_done.wait(lk, [&] { return b->active == 0; });
    }
    sim_status first = SIM_OK;
    for (size_t k = 0; k < b->members.size(); k++) {
        if (member_status) member_status[k] = b->status[k];
        if (first == SIM_OK && b->status[k] != SIM_OK) first = b->status[k];
    }
    return first;
}

}  // extern "C"
