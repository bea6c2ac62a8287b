// Request loop over independent LLG integrations (continuous batching of runs of different grid sizes
// and materials on one GPU).  Each run is the single-mesh integration of the library (the same step
// graphs and device-side step control as nm_run_until), so a run's result does not depend on what else
// is running: runs share no device buffer, each steps on its own stream, and every reduction is
// deterministic.
//
// Threads: nm_server_submit / nm_server_poll / nm_server_stats_get take the server mutex only; all CUDA
// work, admission and mesh management happen on the worker thread.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>

#include "mesh.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

struct Key {
    int n[3];
    double dx[3];
    int prec;
    bool operator==(const Key &o) const
    {
        return n[0] == o.n[0] && n[1] == o.n[1] && n[2] == o.n[2] && dx[0] == o.dx[0] && dx[1] == o.dx[1] &&
               dx[2] == o.dx[2] && prec == o.prec;
    }
};

// a pooled mesh: idle, or owned by one running request
struct Slot {
    Key key;
    nm_mesh M = nullptr;
    long fp = 0;
    cudaEvent_t ev = nullptr;
    long last_use = 0;
    bool busy = false;
};

struct Run {
    nm_request req;
    Clock::time_point t_submit, t_admit;
    Slot *slot = nullptr;
    int phase = 0;          // 0: stepping; 1: copying m out
    bool in_flight = false; // a chunk (or the copy-out) and its control read-back are enqueued
    int n_active_at_admit = 0;
};

constexpr int kMaxChunk = 32;  // step graphs enqueued between two control read-backs

}  // namespace

struct nm_server_s {
    long budget = 0;
    int max_active = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Run *> queue;          // guarded by mu
    std::deque<nm_result> results;    // guarded by mu
    nm_server_stats st{};             // guarded by mu
    bool stop = false;                // guarded by mu
    std::vector<Run *> active;        // worker only
    std::vector<Slot *> pool;         // worker only
    long use_clock = 0;               // worker only
    Clock::time_point t0, t_tick;     // worker only (t0 read-only after create)
    std::thread worker;
};

namespace {

Key key_of(const nm_request &r)
{
    Key k;
    for (int i = 0; i < 3; ++i) {
        k.n[i] = r.n[i];
        k.dx[i] = r.dx[i];
    }
    k.prec = r.precision;
    return k;
}

void push_result(nm_server S, Run *r, int status, long n_acc, long n_rej, double t_final)
{
    const Clock::time_point now = Clock::now();
    nm_result res{};
    res.tag = r->req.tag;
    res.status = status;
    res.n_accepted = n_acc;
    res.n_rejected = n_rej;
    res.t_final = t_final;
    const bool admitted = r->slot != nullptr || r->t_admit != Clock::time_point();
    res.queue_s = admitted ? secs(r->t_submit, r->t_admit) : secs(r->t_submit, now);
    res.run_s = admitted ? secs(r->t_admit, now) : 0.0;
    res.latency_s = secs(r->t_submit, now);
    res.n_active_at_admit = r->n_active_at_admit;
    if (status != NM_OK) {
        strncpy(res.message, nm_last_error(), sizeof res.message - 1);
        res.message[sizeof res.message - 1] = 0;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->results.push_back(res);
        S->st.completed += 1;
        if (status != NM_OK) S->st.failed += 1;
    }
    S->cv_done.notify_all();
}

void destroy_slot(nm_server S, Slot *s)
{
    nm_destroy_mesh(s->M);
    if (s->ev) cudaEventDestroy(s->ev);
    S->pool.erase(std::find(S->pool.begin(), S->pool.end(), s));
    delete s;
}

long pool_bytes(nm_server S)
{
    long b = 0;
    for (Slot *s : S->pool) b += s->fp;
    return b;
}

// Configure the slot's mesh for the request and enqueue the FSAL slope; the run is then ready to step.
int start_run(nm_server S, Run *r)
{
    const nm_request &q = r->req;
    nm_mesh M = r->slot->M;
    int rc;
    const double zero[3] = {0, 0, 0};
    if ((rc = nm_set_material(M, nullptr, q.Ms, nullptr, q.A, nullptr, q.Ku, q.axis, q.alpha, q.gamma))) return rc;
    if ((rc = nm_set_field(M, NM_FIELD_HEXT_CELL, nullptr, zero, 0.0, 0.0))) return rc;
    if ((rc = nm_set_field(M, NM_FIELD_HEXT_UNIFORM, nullptr, q.h, 0.0, 0.0))) return rc;
    if ((rc = nm_set_terms(M, q.terms))) return rc;
    if ((rc = nm_set_state(M, q.m0, NM_MEM_HOST, 0.0, q.dt0))) return rc;
    StepCtl *h = M->hctl;  // nm_set_state left the stream idle and the mirror equal to the device block
    h->dt = std::min(q.dt0, q.t_end);
    h->t_end = q.t_end;
    h->rtol = q.rtol;
    h->atol = q.atol;
    h->done = 0;
    h->status = NM_OK;
    h->dt_min = M->dt_min;
    if ((rc = push_ctl(M))) return rc;
    if ((rc = ensure_k1(M, q.method))) return rc;
    (void)S;
    return NM_OK;
}

// Admit the head of the queue if a slot and memory allow.  Returns true when the queue head changed.
bool admit_one(nm_server S)
{
    Run *r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->queue.empty() || (int)S->active.size() >= S->max_active) return false;
        r = S->queue.front();
    }
    auto pop = [&]() {
        std::lock_guard<std::mutex> lk(S->mu);
        S->queue.pop_front();
    };
    const Key k = key_of(r->req);
    const long fp = mesh_footprint(k.n[0], k.n[1], k.n[2], k.prec);
    if (fp > S->budget) {
        pop();
        fail(NM_ERR_OOM, "request footprint %ld B exceeds the server budget %ld B", fp, S->budget);
        push_result(S, r, NM_ERR_OOM, 0, 0, 0.0);
        delete r;
        return true;
    }
    Slot *slot = nullptr;
    for (Slot *s : S->pool)
        if (!s->busy && s->key == k) { slot = s; break; }
    if (!slot) {
        while (pool_bytes(S) + fp > S->budget) {
            Slot *lru = nullptr;
            for (Slot *s : S->pool)
                if (!s->busy && (!lru || s->last_use < lru->last_use)) lru = s;
            if (!lru) return false;  // wait for running requests to finish
            destroy_slot(S, lru);
            std::lock_guard<std::mutex> lk(S->mu);
            S->st.meshes_evicted += 1;
        }
        nm_mesh src = nullptr;
        for (Slot *s : S->pool)
            if (s->key == k) { src = s->M; break; }
        nm_mesh M = nullptr;
        int rc = create_mesh(k.n[0], k.n[1], k.n[2], k.dx[0], k.dx[1], k.dx[2], k.prec, nullptr, src, &M);
        if (rc == NM_OK) {
            slot = new Slot();
            slot->key = k;
            slot->M = M;
            slot->fp = fp;
            if (cudaEventCreateWithFlags(&slot->ev, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                nm_destroy_mesh(M);
                delete slot;
                slot = nullptr;
                rc = fail(NM_ERR_CUDA, "cudaEventCreate failed");
            }
        }
        if (rc != NM_OK) {
            pop();
            push_result(S, r, rc, 0, 0, 0.0);
            delete r;
            return true;
        }
        S->pool.push_back(slot);
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.meshes_created += 1;
        if (src) S->st.tensor_copies += 1;
    }
    pop();
    slot->busy = true;
    slot->last_use = ++S->use_clock;
    r->slot = slot;
    r->t_admit = Clock::now();
    r->n_active_at_admit = (int)S->active.size() + 1;
    int rc = start_run(S, r);
    if (rc != NM_OK) {
        slot->busy = false;
        r->slot = nullptr;
        push_result(S, r, rc, 0, 0, 0.0);
        delete r;
        return true;
    }
    S->active.push_back(r);
    return true;
}

// Enqueue the next chunk of step graphs (or the copy-out) and the control read-back.
int enqueue_chunk(Run *r)
{
    nm_mesh M = r->slot->M;
    const StepCtl *h = M->hctl;
    long n = kMaxChunk;
    if (h->dt > 0) {
        const double left = (r->req.t_end - h->t) / h->dt;
        if (left + 1 < n) n = std::max(1L, (long)ceil(left) + 1);
    }
    int rc;
    for (long i = 0; i < n; ++i)
        if ((rc = launch_step(M, r->req.method))) return rc;
    CUDA_TRY(cudaMemcpyAsync(M->hctl, M->ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, M->st));
    CUDA_TRY(cudaEventRecord(r->slot->ev, M->st));
    r->in_flight = true;
    return NM_OK;
}

int enqueue_copy_out(Run *r)
{
    nm_mesh M = r->slot->M;
    const Geom &g = M->g;
    if (void *mapped = r->req.m_out ? mapped_host(r->req.m_out) : nullptr) {
        launch_soa_to_aos<double, double>(g, M->m, (double *)mapped, M->st);  // page-locked: written directly
        CHECK_LAUNCH();
    } else if (r->req.m_out) {
        double *tmp = nullptr;
        CUDA_TRY(cudaMallocAsync(&tmp, g.n_nodes * 3 * sizeof(double), M->st));
        launch_soa_to_aos<double, double>(g, M->m, tmp, M->st);
        CHECK_LAUNCH();
        CUDA_TRY(cudaMemcpyAsync(r->req.m_out, tmp, g.n_nodes * 3 * sizeof(double), cudaMemcpyDeviceToHost, M->st));
        CUDA_TRY(cudaFreeAsync(tmp, M->st));
    }
    CUDA_TRY(cudaEventRecord(r->slot->ev, M->st));
    r->in_flight = true;
    r->phase = 1;
    return NM_OK;
}

void finish(nm_server S, Run *r, int status)
{
    const StepCtl *h = r->slot->M->hctl;
    if (status != NM_OK) cudaStreamSynchronize(r->slot->M->st);
    r->slot->busy = false;
    r->slot->last_use = ++S->use_clock;
    push_result(S, r, status, h->n_acc, h->n_rej, h->t);
    S->active.erase(std::find(S->active.begin(), S->active.end(), r));
    delete r;
}

// Advance one run by at most one state change.  Returns true when something happened.
bool advance(nm_server S, Run *r)
{
    if (r->in_flight) {
        cudaError_t e = cudaEventQuery(r->slot->ev);
        if (e == cudaErrorNotReady) return false;
        r->in_flight = false;
        if (e != cudaSuccess) {
            fail(NM_ERR_CUDA, "run %ld: %s", r->req.tag, cudaGetErrorString(e));
            finish(S, r, NM_ERR_CUDA);
            return true;
        }
        if (r->phase == 1) {
            finish(S, r, NM_OK);
            return true;
        }
        const StepCtl *h = r->slot->M->hctl;
        if (h->status != NM_OK) {
            fail(h->status, "run %ld failed at t=%g (err %g)", r->req.tag, h->t, h->err);
            finish(S, r, h->status);
            return true;
        }
        if (h->done) {
            int rc = enqueue_copy_out(r);
            if (rc != NM_OK) finish(S, r, rc);
            return true;
        }
    }
    int rc = enqueue_chunk(r);
    if (rc != NM_OK) finish(S, r, rc);
    return true;
}

void tick(nm_server S)
{
    const Clock::time_point now = Clock::now();
    const double dt = secs(S->t_tick, now);
    S->t_tick = now;
    const int na = (int)S->active.size();
    std::lock_guard<std::mutex> lk(S->mu);
    if (na > 0) S->st.busy_s += dt;
    S->st.active_s += dt * na;
    S->st.active = na;
    S->st.peak_active = std::max(S->st.peak_active, na);
    S->st.pooled = (int)S->pool.size();
    long b = 0;
    for (Slot *s : S->pool) b += s->fp;
    S->st.bytes_in_use = b;
    S->st.peak_bytes = std::max(S->st.peak_bytes, b);
    S->st.queued = (int)S->queue.size();
}

void worker_main(nm_server S)
{
    cudaSetDevice(S->device);
    S->t_tick = Clock::now();
    while (true) {
        bool progressed = false;
        while (admit_one(S)) progressed = true;
        std::vector<Run *> snapshot = S->active;
        for (Run *r : snapshot) progressed |= advance(S, r);
        tick(S);
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->stop && S->queue.empty() && S->active.empty()) break;
        if (!progressed) {
            if (S->active.empty() && (S->queue.empty() || (int)S->active.size() >= S->max_active))
                S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            else
                S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
    while (!S->pool.empty()) destroy_slot(S, S->pool.back());
}

int check_request(const nm_request *q)
{
    if (!q) return fail(NM_ERR_ARG, "request is NULL");
    for (int i = 0; i < 3; ++i) {
        if (q->n[i] < 1) return fail(NM_ERR_ARG, "cell counts must be >= 1");
        if (!(q->dx[i] > 0) || !isfinite(q->dx[i])) return fail(NM_ERR_ARG, "cell sizes must be positive and finite");
        if (!isfinite(q->axis[i]) || !isfinite(q->h[i])) return fail(NM_ERR_ARG, "axis/h must be finite");
    }
    if (q->n[0] > 1024 || q->n[1] > 1024 || q->n[2] > 64)
        return fail(NM_ERR_ARG, "grid beyond the supported range (N1, N2 <= 1024; N3 <= 64)");
    if (q->precision != NM_F32 && q->precision != NM_F64) return fail(NM_ERR_ARG, "precision must be NM_F32 or NM_F64");
    if (!isfinite(q->Ms) || q->Ms < 0 || !isfinite(q->A) || !isfinite(q->Ku))
        return fail(NM_ERR_ARG, "material must be finite with Ms >= 0");
    if (!(q->axis[0] * q->axis[0] + q->axis[1] * q->axis[1] + q->axis[2] * q->axis[2] > 0))
        return fail(NM_ERR_ARG, "axis must be non-zero");
    if (!isfinite(q->alpha) || q->alpha < 0 || !isfinite(q->gamma)) return fail(NM_ERR_ARG, "alpha/gamma invalid");
    if (q->terms & ~NM_TERMS_MASK) return fail(NM_ERR_ARG, "unknown term bits 0x%x", q->terms);
    if (q->method != NM_RK4 && q->method != NM_DP54) return fail(NM_ERR_ARG, "unknown method %d", q->method);
    if (!(q->t_end > 0) || !isfinite(q->t_end)) return fail(NM_ERR_ARG, "t_end must be positive and finite");
    if (!(q->dt0 > 0) || !isfinite(q->dt0)) return fail(NM_ERR_ARG, "dt0 must be positive and finite");
    if (q->method == NM_DP54 && (!(q->rtol >= 0) || !(q->atol >= 0) || (q->rtol == 0 && q->atol == 0) ||
                                 !isfinite(q->rtol) || !isfinite(q->atol)))
        return fail(NM_ERR_ARG, "tolerances must be finite, >= 0 and not both 0");
    if (!q->m0) return fail(NM_ERR_ARG, "m0 is NULL");
    return NM_OK;
}

}  // namespace

extern "C" int nm_server_create(long hbm_budget_bytes, int max_active, nm_server *out)
{
    clear_error();
    if (!out) return fail(NM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes <= 0) return fail(NM_ERR_ARG, "hbm_budget_bytes must be positive");
    if (max_active < 1 || max_active > 256) return fail(NM_ERR_ARG, "max_active must be in [1, 256]");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    nm_server S = new nm_server_s();
    S->budget = hbm_budget_bytes;
    S->max_active = max_active;
    S->device = dev;
    S->t0 = Clock::now();
    S->worker = std::thread(worker_main, S);
    *out = S;
    return NM_OK;
}

extern "C" int nm_server_submit(nm_server S, const nm_request *req)
{
    clear_error();
    int rc = check_request(req);
    if (rc) return rc;
    if (!S) return fail(NM_ERR_ARG, "server is NULL");
    Run *r = new Run();
    r->req = *req;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            return fail(NM_ERR_STATE, "server is stopping");
        }
        S->queue.push_back(r);
        S->st.submitted += 1;
        S->st.queued = (int)S->queue.size();
    }
    S->cv_work.notify_one();
    return NM_OK;
}

extern "C" int nm_server_poll(nm_server S, nm_result *out, int max_results, double wait_s, int *n_out)
{
    clear_error();
    if (!S || !n_out || (max_results > 0 && !out)) return fail(NM_ERR_ARG, "bad poll arguments");
    if (!(wait_s >= 0) || !isfinite(wait_s)) return fail(NM_ERR_ARG, "wait_s must be finite and >= 0");
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->results.empty() && wait_s > 0)
        S->cv_done.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return !S->results.empty(); });
    int n = 0;
    while (n < max_results && !S->results.empty()) {
        out[n++] = S->results.front();
        S->results.pop_front();
    }
    *n_out = n;
    return NM_OK;
}

extern "C" int nm_server_stats_get(nm_server S, nm_server_stats *out)
{
    clear_error();
    if (!S || !out) return fail(NM_ERR_ARG, "bad arguments");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->wall_s = secs(S->t0, Clock::now());
    return NM_OK;
}

extern "C" int nm_server_destroy(nm_server S)
{
    clear_error();
    if (!S) return NM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    delete S;
    return NM_OK;
}
