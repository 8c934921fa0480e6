// Ensemble runtime: many independent simulators (geological realisations on
// grids of different sizes) advanced together on one GPU.
//
// Lockstep (the default): the members' Newton loops advance in rounds.  In a
// round every member still in its step assembles and tests CNV (accepting
// converged substeps, halving failed ones), and those that need a Newton
// correction set up their CPR preconditioner -- these per-member phases run
// concurrently, one host worker thread and one CUDA stream per member.  Then
// ONE batched FGMRES solves all the members' systems together: each Krylov
// operation (SpMV, every CPR stage, the Gram-Schmidt passes) is one launch
// over a work list of (member, block) items, a restart cycle is one CUDA
// graph, and a member whose estimate meets its tolerance drops out of the
// remaining launches (its control word masks it).  Each member's arithmetic
// is that of its own solve, so a member computes what sim_step computes.
//
// Concurrent: each member's whole sim_step runs on its own stream from a pool
// worker (kernels of different members overlap; launches scale with members).
// Members never exchange data.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "sim_internal.cuh"

struct sim_batch {
    std::vector<sim_t *> members;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    // current job: fn(k) for k in items
    std::function<void(int)> fn;
    std::vector<int> items;
    std::atomic<int> next{0};
    int active = 0;          // workers still working on the current job
    int64_t generation = 0;  // job counter
    bool quit = false;
    int nthreads = 0;
    int mode = SIM_BATCH_LOCKSTEP;
    cudaStream_t stream = nullptr;   // the batched solve's stream
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    KrylovBatch *kb = nullptr;
    bool batchable = false;
    int64_t rounds = 0, batched_solves = 0;
    double t_newton = 0.0, t_solve = 0.0, t_update = 0.0;   // host seconds of the lockstep phases
    std::string msg;
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
            const int q = b->next.fetch_add(1);
            if (q >= (int)b->items.size()) break;
            b->fn(b->items[q]);
        }
        {
            std::lock_guard<std::mutex> lk(b->mu);
            if (--b->active == 0) b->cv_done.notify_all();
        }
    }
}

// fn(k) for every k in items, on the worker threads; returns when all are done
static void run_parallel(sim_batch *b, const std::vector<int> &items, std::function<void(int)> fn) {
    if (items.empty()) return;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->fn = std::move(fn);
        b->items = items;
        b->next.store(0);
        b->active = b->nthreads;
        b->generation++;
    }
    b->cv_work.notify_all();
    std::unique_lock<std::mutex> lk(b->mu);
    b->cv_done.wait(lk, [&] { return b->active == 0; });
}

// the Newton state of one member within a sim_batch_step call
struct MemberStep {
    double dt = 0.0, remaining = 0.0, h = 0.0;
    int l = 0;                 // Newton iterations of the current substep
    bool finished = false, solving = false;
    sim_status st = SIM_OK;
    sim_step_info si;
    sim_linear_info li;
};

// a failed Newton solve: back to the step's start, half the step
static void cut(sim_t *s, MemberStep &m) {
    if (nl_restore(s) != SIM_OK) { m.st = s->err; m.finished = true; return; }
    m.si.cuts++;
    if (m.si.cuts > s->opt.max_cuts) { m.st = SIM_ENOCONV_NEWTON; m.finished = true; return; }
    m.h *= 0.5;
    m.l = 0;
}

// assemble / test / accept / cut until the member needs a solve or its step is done
static void phase_newton(sim_t *s, MemberStep &m) {
    m.solving = false;
    while (!m.finished) {
        if (m.remaining <= 1e-12 * m.dt) { m.finished = true; break; }
        if (m.h > m.remaining) m.h = m.remaining;
        int state = 0;
        if (nl_assemble_test(s, m.h, &state, &m.si.phase) != SIM_OK) { m.st = s->err; m.finished = true; break; }
        if (state == 1) {
            if (accept_step(s, m.h) != SIM_OK) { m.st = s->err; m.finished = true; break; }
            m.remaining -= m.h;
            m.si.substeps++;
            m.si.mb_error = fmax(m.si.mb_error, s->last_mb);
            m.l = 0;
            continue;
        }
        if (state == 2 || m.l >= s->opt.newton_max) { cut(s, m); continue; }
        if (nl_prepare_solve(s, &m.si.phase) != SIM_OK) { m.st = s->err; m.finished = true; break; }
        m.solving = true;
        break;
    }
}

static void phase_update(sim_t *s, MemberStep &m, double solve_us) {
    bool fin = true;
    m.si.phase.solve_us += solve_us;
    if (nl_finish_solve(s, m.li, &fin, &m.si.phase) != SIM_OK) { m.st = s->err; m.finished = true; return; }
    m.si.newton_iterations++;
    m.si.linear_iterations += m.li.iterations;
    s->run_lin_failures += !m.li.converged;
    m.l++;
    if (!fin) cut(s, m);
}

static sim_status step_lockstep(sim_batch *b, const double *dt, sim_step_info *infos, sim_status *mst) {
    const int n = (int)b->members.size();
    std::vector<MemberStep> ms(n);
    std::vector<int> all;
    for (int k = 0; k < n; k++) {
        MemberStep &m = ms[k];
        memset(&m.si, 0, sizeof(m.si));
        m.dt = m.remaining = m.h = dt[k];
        if (!(dt[k] > 0)) { m.st = sim_fail(b->members[k], SIM_EINVAL, "dt must be positive"); m.finished = true; }
        else if (b->members[k]->err != SIM_OK) { m.st = b->members[k]->err; m.finished = true; }
        else all.push_back(k);
    }
    sim_status batch_err = SIM_OK;
    while (batch_err == SIM_OK) {
        std::vector<int> live;
        for (int k : all) if (!ms[k].finished) live.push_back(k);
        if (live.empty()) break;
        auto t0 = std::chrono::steady_clock::now();
        {
            NvtxRange range("batch_newton_phase");
            run_parallel(b, live, [&](int k) { phase_newton(b->members[k], ms[k]); });
        }
        auto t1 = std::chrono::steady_clock::now();
        b->t_newton += std::chrono::duration<double>(t1 - t0).count();
        std::vector<int> solve;
        for (int k : live) if (ms[k].solving && !ms[k].finished) solve.push_back(k);
        if (solve.empty()) continue;
        std::vector<sim_t *> sm;
        for (int k : solve) sm.push_back(b->members[k]);
        std::vector<sim_linear_info> li(solve.size());
        float ms_solve = 0.f;
        sim_status st;
        bool synced;
        {
            NvtxRange solve_range("batched_fgmres");
            cudaEventRecord(b->e0, b->stream);
            st = k_fgmres_batch(b->kb, sm.data(), (int)sm.size(), b->stream, li.data(), &b->msg);
            cudaEventRecord(b->e1, b->stream);
            synced = st == SIM_OK && cudaEventSynchronize(b->e1) == cudaSuccess;
        }
        if (st != SIM_OK || !synced) {
            batch_err = st != SIM_OK ? st : SIM_ECUDA;
            for (int k : solve) { ms[k].st = batch_err; ms[k].finished = true; }
            break;
        }
        cudaEventElapsedTime(&ms_solve, b->e0, b->e1);
        auto t2 = std::chrono::steady_clock::now();
        b->t_solve += std::chrono::duration<double>(t2 - t1).count();
        b->rounds++;
        b->batched_solves += (int64_t)solve.size();
        for (size_t q = 0; q < solve.size(); q++) ms[solve[q]].li = li[q];
        run_parallel(b, solve, [&](int k) { phase_update(b->members[k], ms[k], 1e3 * ms_solve); });
        b->t_update += std::chrono::duration<double>(std::chrono::steady_clock::now() - t2).count();
    }
    sim_status first = SIM_OK;
    for (int k = 0; k < n; k++) {
        sim_t *s = b->members[k];
        MemberStep &m = ms[k];
        if (m.st == SIM_OK && s->stream) {
            if (cudaStreamSynchronize(s->stream) != cudaSuccess) m.st = SIM_ECUDA;
        }
        m.si.ok = m.st == SIM_OK;
        run_record_step(s, m.si, m.st);
        if (infos) infos[k] = m.si;
        if (mst) mst[k] = m.st;
        if (first == SIM_OK && m.st != SIM_OK) first = m.st;
    }
    return first;
}

static sim_status step_concurrent(sim_batch *b, const double *dt, sim_step_info *infos, sim_status *mst) {
    const int n = (int)b->members.size();
    std::vector<sim_status> st(n, SIM_OK);
    std::vector<int> all(n);
    for (int k = 0; k < n; k++) all[k] = k;
    run_parallel(b, all, [&](int k) {
        sim_step_info info;
        memset(&info, 0, sizeof(info));
        st[k] = sim_step(b->members[k], dt[k], &info);
        if (infos) infos[k] = info;
    });
    sim_status first = SIM_OK;
    for (int k = 0; k < n; k++) {
        if (mst) mst[k] = st[k];
        if (first == SIM_OK && st[k] != SIM_OK) first = st[k];
    }
    return first;
}

extern "C" {

sim_status sim_batch_create(int32_t n, sim_t *const *members, int32_t nthreads, sim_batch_t **out) {
    if (!out || n < 1 || !members) return sim_fail(nullptr, SIM_EINVAL, "sim_batch_create: bad arguments");
    *out = nullptr;
    for (int k = 0; k < n; k++)
        if (!members[k]) return sim_fail(nullptr, SIM_EINVAL, "sim_batch_create: NULL member");
    for (int k = 0; k < n; k++)
        for (int j = 0; j < k; j++) {
            if (members[k] == members[j]) return sim_fail(nullptr, SIM_EINVAL, "sim_batch_create: a member appears twice");
            if (members[k]->stream == members[j]->stream)
                return sim_fail(nullptr, SIM_EINVAL, "sim_batch_create: members must own distinct streams");
        }
    sim_batch *b = new sim_batch();
    b->members.assign(members, members + n);
    b->nthreads = nthreads > 0 ? (nthreads < n ? nthreads : n) : (n < 64 ? n : 64);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess) {
        if (b->stream) cudaStreamDestroy(b->stream);
        delete b;
        return sim_fail(nullptr, SIM_ECUDA, "sim_batch_create: stream / event creation failed");
    }
    b->kb = k_batch_new();
    bool fixed = true;
    for (int k = 0; k < n; k++) fixed = fixed && members[k]->opt.forcing == SIM_FORCING_FIXED;
    b->batchable = fixed && cpr_batchable(members, n);
    b->mode = b->batchable ? SIM_BATCH_LOCKSTEP : SIM_BATCH_CONCURRENT;
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
    if (b->stream) cudaStreamSynchronize(b->stream);
    k_batch_free(b->kb);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

sim_status sim_batch_set_mode(sim_batch_t *b, int32_t mode) {
    if (!b || (mode != SIM_BATCH_LOCKSTEP && mode != SIM_BATCH_CONCURRENT)) return SIM_EINVAL;
    if (mode == SIM_BATCH_LOCKSTEP && !b->batchable) return SIM_EINVAL;
    b->mode = mode;
    return SIM_OK;
}

int32_t sim_batch_mode(sim_batch_t *b) { return b ? b->mode : -1; }

sim_status sim_batch_stats(sim_batch_t *b, int64_t *rounds, int64_t *solves, int64_t *launches) {
    if (!b) return SIM_EINVAL;
    if (rounds) *rounds = b->rounds;
    if (solves) *solves = b->batched_solves;
    if (launches) *launches = k_batch_launches(b->kb);
    return SIM_OK;
}

const char *sim_batch_last_error(sim_batch_t *b) { return b ? b->msg.c_str() : ""; }

sim_status sim_batch_phase_seconds(sim_batch_t *b, double *newton, double *solve, double *update) {
    if (!b) return SIM_EINVAL;
    if (newton) *newton = b->t_newton;
    if (solve) *solve = b->t_solve;
    if (update) *update = b->t_update;
    return SIM_OK;
}

sim_status sim_batch_step(sim_batch_t *b, const double *dt, sim_step_info *infos, sim_status *member_status) {
    if (!b || !dt) return SIM_EINVAL;
    return b->mode == SIM_BATCH_LOCKSTEP ? step_lockstep(b, dt, infos, member_status)
                                         : step_concurrent(b, dt, infos, member_status);
}

}  // extern "C"
