// server.cuh -- continuous batching of scattering runs on one GPU (serving).
//
// Included at the end of api.cu (it drives mot_run internals).  A worker thread
// owns up to max_slots active runs, each with its own context stream, problem
// (Lambda0 and history spectra resident) and run (history ring resident).
// Requests queue in arrival order and are admitted whenever a slot is free and
// their estimated device memory fits under the budget and in free memory; a
// run that arrives while others are on the GPU joins at the next worker pass.
// Each pass launches one MOT step (one CUDA graph launch after the first,
// host-driven step) for every active run whose previous step has finished, so
// the steps of different runs overlap on the device.  A finished run's last J
// is copied to the request's host buffer and its slot and memory are freed.
// Waits on the host are bounded by the caller's timeout; nothing spins on the
// GPU.

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>

struct ServeJob {
    uint64_t ticket = 0;
    // the request, copied
    int32_t n[3] = {0, 0, 0};
    double h = 0.0, alpha = 0.0;
    int32_t precision = MOT_MIXED, nrhs = 1, nsteps = 0;
    std::vector<double> eps;
    std::vector<mot_planewave> exc;
    mot_options opt;
    bool has_opt = false;
    double *J_final = nullptr;
    size_t est_bytes = 0;
    // execution
    mot_ctx *ctx = nullptr;
    mot_problem *prob = nullptr;
    mot_run *run = nullptr;
    int done_steps = 0;
    bool inflight = false;
    bool graph_started = false;
    // set-up (context, problem incl. quadrature, run) on a thread of its own, so
    // the worker keeps stepping the other runs meanwhile
    std::thread setup;
    std::atomic<int> setup_state{0};  // 0 running, 1 done, 2 failed
    mot_status setup_status = MOT_OK;
    std::string setup_error;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<float> step_ms;
    int32_t status = MOT_OK;
    std::chrono::steady_clock::time_point t_submit, t_admit, t_done;
    mot_result result;
    bool finished = false;
};

struct mot_server {
    int device = 0;
    size_t budget = 0;
    int max_slots = 1;
    size_t used = 0;
    uint64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServeJob *> pending;
    std::vector<ServeJob *> starting;  // admitted, set-up thread running
    std::vector<ServeJob *> active;
    std::map<uint64_t, ServeJob *> jobs;  // every ticket not yet collected
    bool stop = false;
    std::thread worker;
};

namespace {

constexpr size_t kServeQueueCap = 4096;

// device bytes a run of this request holds (problem + run), with headroom
size_t serve_estimate(const ServeJob &j) {
    const double rho = j.alpha / sqrt(3.0);
    const double rmax = sqrt((double)j.n[0] * j.n[0] + (double)j.n[1] * j.n[1] + (double)j.n[2] * j.n[2]);
    const long ell = (long)ceil(rmax / rho - 1e-12) + 2;
    const int r0 = lag_reach(0, rho);
    long M0[3], Mh[3];
    for (int i = 0; i < 3; ++i) {
        M0[i] = smooth235(j.n[i] + std::min(r0, j.n[i] - 1));
        Mh[i] = smooth235(std::max(1, 2 * j.n[i] - 1));
    }
    const long H0 = M0[0] / 2 + 1, Hh = Mh[0] / 2 + 1;
    const bool mixed = j.precision == MOT_MIXED;
    const size_t cs = mixed ? 8 : 16;
    const size_t nv = (size_t)j.n[0] * j.n[1] * j.n[2], n3 = 3 * nv * j.nrhs;
    size_t b = 12 * nv;                                                                   // eps_r FP64 + FP32
    b += 12 * 6 * (size_t)(M0[2] / 2 + 1) * (M0[1] / 2 + 1) * H0;                        // Lambda0 FP64 + FP32
    b += (size_t)(ell + 1) * 6 * (Mh[2] / 2 + 1) * (Mh[1] / 2 + 1) * Hh * (mixed ? 4 : 8);  // history spectra
    b += (size_t)j.nrhs * 3 * j.n[2] * (j.n[1] + M0[1]) * H0 * 16;                        // product workspace
    const bool inner32 = j.precision != MOT_FP64;  // FP32 Krylov vectors (mixed, double-float refined)
    b += 5 * n3 * 8 + 10 * n3 * (inner32 ? 4 : 8) + (inner32 ? 2 * n3 * 4 : 0);          // J, b, r, Krylov
    if (j.has_opt && j.opt.guess == 2) b += n3 * 8;                                       // J_{n-3}
    const long tb = mixed ? 8 : 4;  // time block of the history: 2 tb partial sums
    b += (size_t)(ell + 1 + 2 * tb) * j.nrhs * 3 * Mh[2] * Mh[1] * Hh * cs;  // history ring, sum, partial sums
    b += (size_t)j.nrhs * 3 * j.n[2] * (j.n[1] + Mh[1]) * Hh * cs;                       // history workspace
    return b + b / 10 + ((size_t)64 << 20);
}

void serve_finish(mot_server *s, ServeJob *j, int32_t status) {
    if (j->run) mot_run_destroy(j->run);
    if (j->prob) mot_problem_destroy(j->prob);
    if (j->ctx) mot_ctx_destroy(j->ctx);
    if (j->e0) cudaEventDestroy(j->e0);
    if (j->e1) cudaEventDestroy(j->e1);
    j->run = nullptr;
    j->prob = nullptr;
    j->ctx = nullptr;
    j->e0 = j->e1 = nullptr;
    j->t_done = std::chrono::steady_clock::now();
    mot_result &r = j->result;
    memset(&r, 0, sizeof(r));
    r.status = status == MOT_OK ? j->status : status;
    r.steps = j->done_steps;
    r.queue_ms = std::chrono::duration<double, std::milli>(j->t_admit - j->t_submit).count();
    r.run_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_admit).count();
    if (!j->step_ms.empty()) {
        std::vector<float> v = j->step_ms;
        std::sort(v.begin(), v.end());
        r.step_p50_ms = v[v.size() / 2];
        r.step_p99_ms = v[std::min(v.size() - 1, (size_t)ceil(0.99 * v.size()) - 1)];
    }
    r.device_bytes = j->est_bytes;
    std::lock_guard<std::mutex> lk(s->mu);
    s->used -= j->est_bytes;
    j->finished = true;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// create the job's context (private non-blocking stream), problem and run
mot_status serve_start(mot_server *s, ServeJob *j) {
    MOT_TRY(mot_ctx_create(s->device, nullptr, &j->ctx));
    MOT_CUDA_TRY(cudaStreamCreateWithFlags(&j->ctx->stream, cudaStreamNonBlocking));
    j->ctx->own_stream = true;
    MOT_TRY(mot_problem_create(j->ctx, j->n, j->h, j->eps.data(), j->alpha, j->has_opt ? &j->opt : nullptr,
                               &j->prob));
    MOT_TRY(mot_run_create(j->prob, j->nrhs, j->exc.data(), j->precision, &j->run));
    MOT_CUDA_TRY(cudaEventCreate(&j->e0));
    MOT_CUDA_TRY(cudaEventCreate(&j->e1));
    return MOT_OK;
}

// launch the job's next step without waiting for it (graph mode), or run it
// host-driven (the first step, and runs whose options ask for host-driven steps)
mot_status serve_launch(ServeJob *j) {
    mot_run *r = j->run;
    cudaStream_t st = r->p->ctx->stream;
    if (!r->warmed || r->p->opt.graph != 1) {
        mot_step_stats ss;
        MOT_CUDA_TRY(cudaEventRecord(j->e0, st));
        mot_status rs = mot_run_step(r, 1, nullptr, &ss);
        MOT_CUDA_TRY(cudaEventRecord(j->e1, st));
        if (rs == MOT_ENOTCONV) j->status = MOT_ENOTCONV;
        else if (rs != MOT_OK) return rs;
        j->inflight = true;
        return MOT_OK;
    }
    if (!r->step_exec) MOT_TRY(build_step_graph(r));
    if (!j->graph_started) {
        long long n0 = r->n;
        MOT_CUDA_TRY(cudaMemcpyAsync(r->sdev.p, &n0, sizeof(long long), cudaMemcpyHostToDevice, st));
        MOT_CUDA_TRY(cudaStreamSynchronize(st));
        j->graph_started = true;
    }
    MOT_CUDA_TRY(cudaMemsetAsync((char *)r->sdev.p + offsetof(StepDev, nstat), 0, sizeof(int), st));
    MOT_CUDA_TRY(cudaEventRecord(j->e0, st));
    MOT_TRY(hist_prime(r, st));
    MOT_CUDA_TRY(cudaGraphLaunch(r->step_exec, st));
    MOT_CUDA_TRY(cudaEventRecord(j->e1, st));
    r->n += 1;
    j->inflight = true;
    return MOT_OK;
}

// the job's launched step has finished: collect its statistics
mot_status serve_collect(ServeJob *j) {
    mot_run *r = j->run;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, j->e0, j->e1) == cudaSuccess) j->step_ms.push_back(ms);
    else cudaGetLastError();
    if (j->graph_started) {
        StepStatDev hs;
        MOT_CUDA_TRY(cudaMemcpyAsync(&hs, r->sstats.p, sizeof(hs), cudaMemcpyDeviceToHost, r->p->ctx->stream));
        MOT_CUDA_TRY(cudaStreamSynchronize(r->p->ctx->stream));
        g_launches.fetch_add((unsigned long long)(r->k_fixed + r->k_outer * hs.sweeps + r->k_inner * hs.loops));
        if (hs.notconv) j->status = MOT_ENOTCONV;
    }
    j->inflight = false;
    j->done_steps += 1;
    return MOT_OK;
}

void serve_worker(mot_server *s) {
    cudaSetDevice(s->device);
    size_t free_b = 0, total_b = 0;
    while (true) {
        std::vector<ServeJob *> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            if (s->active.empty() && s->pending.empty() && s->starting.empty())
                s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
            if (s->stop) break;
            // admission in arrival order; a request that does not fit waits
            // while later, smaller ones may go ahead of it
            cudaMemGetInfo(&free_b, &total_b);
            size_t head = free_b > ((size_t)256 << 20) ? free_b - ((size_t)256 << 20) : 0;
            for (auto it = s->pending.begin();
                 it != s->pending.end() &&
                 (int)s->active.size() + (int)s->starting.size() + (int)admit.size() < s->max_slots;) {
                ServeJob *j = *it;
                if (j->est_bytes > s->budget) {  // can never fit
                    j->status = MOT_ENOMEM;
                    admit.push_back(j);
                    it = s->pending.erase(it);
                    continue;
                }
                if (s->used + j->est_bytes <= s->budget && j->est_bytes <= head) {
                    s->used += j->est_bytes;
                    head -= j->est_bytes;
                    admit.push_back(j);
                    it = s->pending.erase(it);
                } else {
                    ++it;
                }
            }
            // nothing running or starting and the oldest request does not fit in free memory: it never will
            if (s->active.empty() && s->starting.empty() && admit.empty() && !s->pending.empty()) {
                ServeJob *j = s->pending.front();
                s->pending.pop_front();
                j->status = MOT_ENOMEM;
                admit.push_back(j);
            }
        }
        for (ServeJob *j : admit) {
            j->t_admit = std::chrono::steady_clock::now();
            if (j->status == MOT_ENOMEM) {
                set_error("request needs more device memory than the server's budget or the free memory");
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->used += j->est_bytes;  // serve_finish subtracts it again
                }
                serve_finish(s, j, MOT_ENOMEM);
                continue;
            }
            j->setup = std::thread([s, j] {
                cudaSetDevice(s->device);
                const mot_status st = serve_start(s, j);
                j->setup_status = st;
                if (st != MOT_OK) j->setup_error = get_error();
                j->setup_state.store(st == MOT_OK ? 1 : 2);
                std::lock_guard<std::mutex> lk(s->mu);
                s->cv_work.notify_all();
            });
            std::lock_guard<std::mutex> lk(s->mu);
            s->starting.push_back(j);
        }
        // runs whose set-up has finished join the active ones
        bool progressed = false;
        {
            std::vector<ServeJob *> ready, still;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                for (ServeJob *j : s->starting) (j->setup_state.load() ? ready : still).push_back(j);
                s->starting = still;
            }
            for (ServeJob *j : ready) {
                j->setup.join();
                progressed = true;
                if (j->setup_state.load() == 2) {
                    set_error(j->setup_error);
                    serve_finish(s, j, j->setup_status);
                    continue;
                }
                std::lock_guard<std::mutex> lk(s->mu);
                s->active.push_back(j);
            }
        }
        // one pass over the active runs: collect finished steps, launch the next ones
        std::vector<ServeJob *> keep, act;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            act = s->active;
        }
        for (ServeJob *j : act) {
            mot_status st = MOT_OK;
            if (j->inflight) {
                cudaError_t q = cudaEventQuery(j->e1);
                if (q == cudaErrorNotReady) {
                    keep.push_back(j);
                    continue;
                }
                if (q != cudaSuccess) {
                    set_error(std::string("step failed: ") + cudaGetErrorString(q));
                    st = MOT_ECUDA;
                } else {
                    st = serve_collect(j);
                }
                progressed = true;
            }
            if (st == MOT_OK && j->done_steps < j->nsteps) {
                st = serve_launch(j);
                progressed = true;
            }
            if (st != MOT_OK) {
                serve_finish(s, j, st);
                continue;
            }
            if (j->done_steps >= j->nsteps && !j->inflight) {
                if (j->J_final) {
                    const size_t bytes = sizeof(double) * 3 * (size_t)j->n[0] * j->n[1] * j->n[2] * j->nrhs;
                    cudaError_t ce = cudaMemcpy(j->J_final, j->run->J.p, bytes, cudaMemcpyDeviceToHost);
                    if (ce != cudaSuccess) {
                        set_error(std::string("result copy: ") + cudaGetErrorString(ce));
                        serve_finish(s, j, MOT_ECUDA);
                        continue;
                    }
                }
                serve_finish(s, j, MOT_OK);
                continue;
            }
            keep.push_back(j);
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->active = keep;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" {

mot_status mot_server_create(mot_ctx *ctx, size_t mem_budget, int max_slots, mot_server **out) {
    if (!ctx || !out) MOT_FAIL(MOT_EINVAL, "NULL argument");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 256) MOT_FAIL(MOT_EINVAL, "max_slots out of range [1, 256]");
    MOT_CUDA_TRY(cudaSetDevice(ctx->device));
    size_t free_b = 0, total_b = 0;
    MOT_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    mot_server *s = new mot_server();
    s->device = ctx->device;
    s->budget = mem_budget ? mem_budget : free_b / 10 * 8;  // default: 80% of the free memory now
    s->max_slots = max_slots;
    s->worker = std::thread(serve_worker, s);
    *out = s;
    return MOT_OK;
}

mot_status mot_server_submit(mot_server *s, const mot_request *q, uint64_t *ticket) {
    if (!s || !q || !ticket) MOT_FAIL(MOT_EINVAL, "NULL argument");
    if (!q->eps_r || !q->exc) MOT_FAIL(MOT_EINVAL, "request: eps_r and exc are required");
    if (q->nsteps < 0) MOT_FAIL(MOT_EINVAL, "request: nsteps < 0");
    if (q->nrhs < 1 || q->nrhs > 1024) MOT_FAIL(MOT_EINVAL, "request: nrhs out of range [1, 1024]");
    for (int i = 0; i < 3; ++i)
        if (q->n[i] < 1 || q->n[i] > 4096) MOT_FAIL(MOT_EINVAL, "request: grid size out of range [1, 4096]");
    if (!(q->alpha > 0.0) || !(q->h > 0.0)) MOT_FAIL(MOT_EINVAL, "request: alpha and h must be > 0");
    ServeJob *j = new ServeJob();
    for (int i = 0; i < 3; ++i) j->n[i] = q->n[i];
    j->h = q->h;
    j->alpha = q->alpha;
    j->precision = q->precision;
    j->nrhs = q->nrhs;
    j->nsteps = q->nsteps;
    j->eps.assign(q->eps_r, q->eps_r + (size_t)q->n[0] * q->n[1] * q->n[2]);
    j->exc.assign(q->exc, q->exc + q->nrhs);
    if (q->opt) {
        j->opt = *q->opt;
        j->has_opt = true;
    }
    j->J_final = q->J_final;
    j->est_bytes = serve_estimate(*j);
    j->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->pending.size() >= kServeQueueCap) {
        delete j;
        MOT_FAIL(MOT_EBUSY, "request queue full");
    }
    j->ticket = s->next_ticket++;
    s->jobs[j->ticket] = j;
    s->pending.push_back(j);
    *ticket = j->ticket;
    s->cv_work.notify_all();
    return MOT_OK;
}

mot_status mot_server_wait(mot_server *s, uint64_t ticket, double timeout_s, mot_result *res) {
    if (!s || !res) MOT_FAIL(MOT_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) MOT_FAIL(MOT_EINVAL, "unknown or already collected ticket");
    ServeJob *j = it->second;
    const auto limit = std::chrono::duration<double>(timeout_s < 0 ? 0.0 : timeout_s);
    if (!s->cv_done.wait_for(lk, limit, [&] { return j->finished; }))
        MOT_FAIL(MOT_ETIMEOUT, "request not finished within the timeout");
    *res = j->result;
    s->jobs.erase(it);
    delete j;
    return MOT_OK;
}

void mot_server_destroy(mot_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    // set-ups in flight finish first; their runs are then cancelled with the active ones
    for (ServeJob *j : s->starting) {
        if (j->setup.joinable()) j->setup.join();
        if (j->setup_state.load() == 1) s->active.push_back(j);
        else serve_finish(s, j, MOT_ECANCELLED);
    }
    s->starting.clear();
    // runs on the GPU finish their current step and are abandoned; waiting ones are cancelled
    for (ServeJob *j : s->active) {
        if (j->ctx) cudaStreamSynchronize(j->ctx->stream);
        serve_finish(s, j, MOT_ECANCELLED);
    }
    for (ServeJob *j : s->pending) {
        j->t_admit = j->t_submit;
        j->status = MOT_ECANCELLED;
        j->finished = true;
    }
    for (auto &kv : s->jobs) delete kv.second;
    delete s;
}

}  // extern "C"
