// fr_server.cu -- backtests as requests, served with continuous batching.
//
// A server owns one env batch of `capacity` slots over one market and one
// worker thread.  The worker loops: admit queued requests into free slots
// (arrival order; the head waits until it fits), run the ensemble's rollout
// over the whole pool for `chunk_steps` steps, retire the requests whose
// windows are complete (their slots' episode metrics to the caller's host
// buffer) and park their slots.  Parked slots are done envs: the rollout
// kernels leave them frozen, so the pool runs one launch sequence whatever
// mix of requests occupies it.  Every request starts at a chunk boundary
// and all of its envs share one window, so its completion is known on the
// host from the number of chunks run.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fr_common.cuh"

namespace fr {
namespace {

// Constants of one admitted env: its window, asset count and the draw of
// its price perturbations (request seed, range, index in the request).
struct SlotCst {
    int32_t start, window, ke, range, index, pad;
    uint64_t seed;
};

// Reset admitted slots; stock slots draw their perturbations on the device
// (perturb_bps of the request's seed for assets below the market's K).
__global__ void k_slot_assign(EnvView v, const int32_t *slot, const SlotCst *cst, int n)
{
    const int i = blockIdx.x;
    if (i >= n) return;
    const int e = slot[i];
    const int lane = threadIdx.x;
    const SlotCst c = cst[i];
    if (v.task == FR_TASK_STOCK) {
        v.hold[(int64_t)e * KP + lane] = 0;
        ((int16_t *)v.bps)[(int64_t)e * KP + lane] =
            (lane < v.K && c.range > 0) ? perturb_bps(c.seed, (uint32_t)c.index, (uint32_t)lane, c.range)
                                        : (int16_t)0;
    } else if (lane == 0) {
        v.hold[e] = 0;
    }
    if (lane == 0) {
        ((int32_t *)v.start)[e] = c.start;
        ((int32_t *)v.W)[e] = c.window;
        ((int32_t *)v.Ke)[e] = c.ke;
        v.cash[e] = v.init_cash;
        v.t[e] = 0;
        v.done[e] = 0;
        v.mu[e] = 0.0;
        v.m2[e] = 0.0;
        v.mdd[e] = 0.0;
        v.peak[e] = v.init_cash;
        v.vlast[e] = v.init_cash;
        for (int j = 0; j < 4; ++j) v.latched[(int64_t)e * 4 + j] = 0.0;
    }
}

__global__ void k_slot_park(EnvView v, const int32_t *slot, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v.done[slot[i]] = 1;
}

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SrvReq {
    uint64_t ticket;
    fr_request r;
    std::vector<int32_t> slots;
    int steps_run = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = FR_OK;
    bool cancel = false;       // set by backtest_cancel while running
};

// FR_OK, or why a request must leave now: cancelled or past its deadline.
int leave_reason(const SrvReq *q, double t)
{
    if (q->cancel) return FR_ECANCELED;
    if (q->r.timeout_s > 0.0 && t - q->t_submit > q->r.timeout_s) return FR_ETIMEDOUT;
    return FR_OK;
}

}  // namespace
}  // namespace fr

using namespace fr;

struct fr_server {
    fr_ctx *ctx;
    const fr_market *mkt;
    const fr_ensemble *ens;
    fr_server_desc d;
    fr_env *env = nullptr;
    cudaStream_t stream = nullptr;
    // device / pinned staging
    int32_t *d_slot = nullptr, *h_slot = nullptr;
    SlotCst *d_cst = nullptr, *h_cst = nullptr;
    double *d_met = nullptr, *h_met = nullptr;
    std::vector<int32_t> ke_mirror;
    // scheduler state (under mu)
    std::mutex mu;
    std::condition_variable cv;
    std::deque<SrvReq *> queue;
    std::vector<SrvReq *> running;
    std::unordered_map<uint64_t, SrvReq *> live;     // queued or running
    std::unordered_map<uint64_t, SrvReq *> finished;
    std::vector<int32_t> free_slots;                 // kept sorted, popped from the front
    uint64_t next_ticket = 1;
    int sticky = FR_OK;
    bool stop = false;
    fr_server_stats st{};
    std::thread worker;
};

namespace {

void release_all(fr_server *s)
{
    for (auto &kv : s->live) delete kv.second;
    for (auto &kv : s->finished) delete kv.second;
    s->live.clear();
    s->finished.clear();
    s->queue.clear();
    s->running.clear();
}

// Upload the slot constants of newly admitted requests and reset their
// slots; returns a CUDA status.
cudaError_t assign(fr_server *s, const std::vector<SrvReq *> &adm, bool &ke_changed)
{
    const bool stock = s->env->v.task == FR_TASK_STOCK;
    int n = 0;
    for (SrvReq *q : adm) {
        const fr_request &r = q->r;
        const int ke = stock ? (r.n_assets > 0 ? r.n_assets : s->env->v.K) : 1;
        for (int i = 0; i < r.n_envs; ++i, ++n) {
            const int32_t e = q->slots[i];
            s->h_slot[n] = e;
            SlotCst &c = s->h_cst[n];
            c.start = r.start + i * r.start_stride;
            c.window = r.window;
            c.ke = ke;
            c.range = stock ? r.bps_range : 0;
            c.index = i;
            c.pad = 0;
            c.seed = r.seed;
            if (s->ke_mirror[e] != ke) ke_changed = true;
            s->ke_mirror[e] = ke;
        }
    }
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(s->d_slot, s->h_slot, 4ull * n, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_cst, s->h_cst, sizeof(SlotCst) * n, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return e;
    k_slot_assign<<<n, KP, 0, s->stream>>>(s->env->v, s->d_slot, s->d_cst, n);
    e = cudaGetLastError();
    // the staging buffers are reused by the next admission: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e;
}

void fail_all(fr_server *s, int rc)
{
    std::lock_guard<std::mutex> lk(s->mu);
    s->sticky = rc;
    const double t = now_s();
    for (SrvReq *q : s->running) {
        q->status = rc;
        q->t_done = t;
        s->live.erase(q->ticket);
        s->finished[q->ticket] = q;
        s->st.failed += 1;
    }
    for (SrvReq *q : s->queue) {
        q->status = rc;
        q->t_done = t;
        s->live.erase(q->ticket);
        s->finished[q->ticket] = q;
        s->st.failed += 1;
    }
    s->running.clear();
    s->queue.clear();
    s->st.running = 0;
    s->st.queued = 0;
}

// A chunk failed without a CUDA error (the context is still usable): the
// running requests finish with status rc, their slots are parked and freed,
// and the queued requests stay.  Returns a CUDA status (parking the slots).
cudaError_t fail_running(fr_server *s, int rc)
{
    int n = 0;
    for (SrvReq *q : s->running)
        for (int32_t e : q->slots) s->h_slot[n++] = e;
    cudaError_t ce = cudaSuccess;
    if (n > 0) {
        ce = cudaMemcpyAsync(s->d_slot, s->h_slot, 4ull * n, cudaMemcpyHostToDevice, s->stream);
        if (ce == cudaSuccess) {
            k_slot_park<<<ceil_div(n, 128), 128, 0, s->stream>>>(s->env->v, s->d_slot, n);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
    }
    if (ce != cudaSuccess) return ce;
    std::lock_guard<std::mutex> lk(s->mu);
    const double t = now_s();
    for (SrvReq *q : s->running) {
        q->status = rc;
        q->t_done = t;
        s->free_slots.insert(s->free_slots.end(), q->slots.begin(), q->slots.end());
        s->live.erase(q->ticket);
        s->finished[q->ticket] = q;
        s->st.failed += 1;
    }
    s->running.clear();
    std::sort(s->free_slots.begin(), s->free_slots.end());
    s->st.running = 0;
    return cudaSuccess;
}

// At a chunk boundary: queued requests past their deadline finish at once;
// running ones that were cancelled or are past their deadline are parked
// and their slots freed.  Returns a CUDA status (parking the slots).
cudaError_t retire_leavers(fr_server *s)
{
    std::vector<SrvReq *> gone;
    std::vector<int> why;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const double t = now_s();
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            SrvReq *q = *it;
            const int st = leave_reason(q, t);
            if (st == FR_OK) {
                ++it;
                continue;
            }
            q->status = st;
            q->t_done = t;
            s->live.erase(q->ticket);
            s->finished[q->ticket] = q;
            s->st.failed += 1;
            it = s->queue.erase(it);
        }
        s->st.queued = s->queue.size();
        for (SrvReq *q : s->running) {
            const int st = leave_reason(q, t);
            if (st != FR_OK) {
                gone.push_back(q);
                why.push_back(st);
            }
        }
    }
    if (gone.empty()) return cudaSuccess;
    int n = 0;
    for (SrvReq *q : gone)
        for (int32_t e : q->slots) s->h_slot[n++] = e;
    cudaError_t ce = cudaMemcpyAsync(s->d_slot, s->h_slot, 4ull * n, cudaMemcpyHostToDevice, s->stream);
    if (ce == cudaSuccess) {
        k_slot_park<<<ceil_div(n, 128), 128, 0, s->stream>>>(s->env->v, s->d_slot, n);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
    if (ce != cudaSuccess) return ce;
    std::lock_guard<std::mutex> lk(s->mu);
    const double t = now_s();
    for (size_t i = 0; i < gone.size(); ++i) {
        SrvReq *q = gone[i];
        q->status = why[i];
        q->t_done = t;
        s->running.erase(std::find(s->running.begin(), s->running.end(), q));
        s->free_slots.insert(s->free_slots.end(), q->slots.begin(), q->slots.end());
        s->live.erase(q->ticket);
        s->finished[q->ticket] = q;
        s->st.failed += 1;
    }
    std::sort(s->free_slots.begin(), s->free_slots.end());
    s->st.running = s->running.size();
    return cudaSuccess;
}

void worker_loop(fr_server *s)
{
    cudaSetDevice(s->ctx->device);
    const int chunk = s->d.chunk_steps;
    const int N = s->d.capacity;
    for (;;) {
        std::vector<SrvReq *> admitted;
        {
            const cudaError_t rc = retire_leavers(s);
            if (rc != cudaSuccess) {
                cuda_fail(rc, "server: retiring cancelled requests");
                fail_all(s, FR_ECUDA);
                return;
            }
        }
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::milliseconds(2),
                           [&] { return s->stop || !s->queue.empty() || !s->running.empty(); });
            if (s->stop) return;
            while (!s->queue.empty() && (int)s->free_slots.size() >= s->queue.front()->r.n_envs) {
                SrvReq *q = s->queue.front();
                s->queue.pop_front();
                q->slots.assign(s->free_slots.begin(), s->free_slots.begin() + q->r.n_envs);
                s->free_slots.erase(s->free_slots.begin(), s->free_slots.begin() + q->r.n_envs);
                q->t_admit = now_s();
                s->running.push_back(q);
                admitted.push_back(q);
            }
            s->st.queued = s->queue.size();
            s->st.running = s->running.size();
            if (s->running.empty()) continue;
        }
        const double t0 = now_s();
        bool ke_changed = false;
        cudaError_t ce = assign(s, admitted, ke_changed);
        if (ce != cudaSuccess) {
            cuda_fail(ce, "server: slot assignment");
            fail_all(s, FR_ECUDA);
            return;
        }
        if (!admitted.empty()) s->env->pack_state = 0;       // windows changed: re-pack the tiles
        if (ke_changed && s->env->slot_of_env) {
            // the fused stock kernel rebuilds its asset-count slots
            dev_free(s->ctx, s->env->slot_of_env, 4ull * N + 4ull * 32);
            s->env->slot_of_env = nullptr;
            s->env->slot_ke = nullptr;
        }
        int rc = rollout(s->env, s->ens, chunk, nullptr, nullptr, s->stream);
        if (rc == FR_ECUDA) {
            fail_all(s, rc);
            return;
        }
        if (rc) {
            ce = fail_running(s, rc);
            if (ce != cudaSuccess) {
                cuda_fail(ce, "server: parking failed requests");
                fail_all(s, FR_ECUDA);
                return;
            }
            continue;
        }
        // the worker alone touches running requests' progress
        std::vector<SrvReq *> done;
        for (SrvReq *q : s->running) {
            q->steps_run += chunk;
            if (q->steps_run >= q->r.window - 1) done.push_back(q);
        }
        if (!done.empty()) {
            ce = launch_env_metrics(s->env->v, s->d_met, s->stream);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(s->h_met, s->d_met, 24ull * N, cudaMemcpyDeviceToHost, s->stream);
            int n = 0;
            for (SrvReq *q : done)
                for (int32_t e : q->slots) s->h_slot[n++] = e;
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_slot, s->h_slot, 4ull * n, cudaMemcpyHostToDevice, s->stream);
            if (ce == cudaSuccess) {
                k_slot_park<<<ceil_div(n, 128), 128, 0, s->stream>>>(s->env->v, s->d_slot, n);
                ce = cudaGetLastError();
            }
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
            if (ce != cudaSuccess) {
                cuda_fail(ce, "server: retiring requests");
                fail_all(s, FR_ECUDA);
                return;
            }
            const double t = now_s();
            for (SrvReq *q : done) {
                for (int i = 0; i < q->r.n_envs; ++i)
                    for (int j = 0; j < 3; ++j) q->r.metrics[3 * i + j] = s->h_met[3 * (size_t)q->slots[i] + j];
                q->t_done = t;
            }
        } else {
            ce = cudaStreamSynchronize(s->stream);
            if (ce != cudaSuccess) {
                cuda_fail(ce, "server: rollout chunk");
                fail_all(s, FR_ECUDA);
                return;
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (SrvReq *q : done) {
                s->running.erase(std::find(s->running.begin(), s->running.end(), q));
                s->free_slots.insert(s->free_slots.end(), q->slots.begin(), q->slots.end());
                s->live.erase(q->ticket);
                s->finished[q->ticket] = q;
                s->st.completed += 1;
                s->st.env_steps += (double)q->r.n_envs * (q->r.window - 1);
            }
            if (!done.empty()) std::sort(s->free_slots.begin(), s->free_slots.end());
            s->st.pool_steps += (double)N * chunk;
            s->st.busy_s += now_s() - t0;
            s->st.running = s->running.size();
        }
    }
}

void server_free(fr_server *s)
{
    if (s->env) env_destroy(s->env);
    if (s->d_slot) cudaFree(s->d_slot);
    if (s->d_cst) cudaFree(s->d_cst);
    if (s->d_met) cudaFree(s->d_met);
    if (s->h_slot) cudaFreeHost(s->h_slot);
    if (s->h_cst) cudaFreeHost(s->h_cst);
    if (s->h_met) cudaFreeHost(s->h_met);
    if (s->stream) cudaStreamDestroy(s->stream);
    release_all(s);
    delete s;
}

}  // namespace

extern "C" {

int fr_server_create(fr_ctx *ctx, const fr_server_desc *d, fr_server **out)
{
    FR_NVTX("fr_server_create");
    FR_CHECK(ctx && d && out && d->market && d->ens, FR_EINVAL, "fr_server_create: NULL argument");
    *out = nullptr;
    FR_CHECK(d->capacity >= 1 && d->chunk_steps >= 1, FR_EINVAL,
             "fr_server_create: capacity %d and chunk_steps %d must be >= 1", d->capacity, d->chunk_steps);
    const fr_market *m = d->market;
    const fr_ensemble *e = d->ens;
    const bool stock = m->task == FR_TASK_STOCK;
    FR_CHECK(e->dims[0] == (stock ? 1 + 2 * m->K + m->I * m->K : FR_CRYPTO_OBS_DIM), FR_EINVAL,
             "fr_server_create: ensemble input %d does not match the market's observation", e->dims[0]);
    FR_CHECK(stock ? (e->combine == FR_COMBINE_MEAN && e->dims[e->L] == m->K)
                   : (e->combine == FR_COMBINE_VOTE && e->n_act == 3),
             FR_EINVAL, "fr_server_create: ensemble combine/output does not match the task");
    FR_CUDA(cudaSetDevice(ctx->device));
    int rc = FR_OK;
    fr_server *s = new (std::nothrow) fr_server();
    FR_CHECK(s, FR_ENOMEM, "fr_server_create: out of host memory");
    s->ctx = ctx;
    s->mkt = m;
    s->ens = e;
    s->d = *d;
    const int N = d->capacity;
    std::vector<int32_t> win(N, 2), start(N, 0);
    fr_env_desc ed{};
    ed.task = m->task;
    ed.n_envs = N;
    ed.window = win.data();
    ed.start = start.data();
    ed.init_cash = d->init_cash;
    ed.hmax = d->hmax;
    ed.fee_bps = d->fee_bps;
    ed.pmax = d->pmax;
    rc = env_create(ctx, &ed, m, &s->env);
    if (rc) {
        server_free(s);
        return rc;
    }
    s->ke_mirror.assign(N, stock ? m->K : 1);
    cudaError_t ce = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_slot, 4ull * N);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_cst, sizeof(SlotCst) * N);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->d_met, 24ull * N);
    if (ce == cudaSuccess) ce = cudaMallocHost(&s->h_slot, 4ull * N);
    if (ce == cudaSuccess) ce = cudaMallocHost(&s->h_cst, sizeof(SlotCst) * N);
    if (ce == cudaSuccess) ce = cudaMallocHost(&s->h_met, 24ull * N);
    if (ce != cudaSuccess) {
        server_free(s);
        return cuda_fail(ce, "fr_server_create");
    }
    // every slot starts parked
    for (int i = 0; i < N; ++i) s->h_slot[i] = i;
    ce = cudaMemcpy(s->d_slot, s->h_slot, 4ull * N, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
        k_slot_park<<<ceil_div(N, 128), 128, 0, s->stream>>>(s->env->v, s->d_slot, N);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
    if (ce != cudaSuccess) {
        server_free(s);
        return cuda_fail(ce, "fr_server_create: parking slots");
    }
    s->free_slots.resize(N);
    for (int i = 0; i < N; ++i) s->free_slots[i] = i;
    try {
        s->worker = std::thread(worker_loop, s);
    } catch (...) {
        server_free(s);
        set_error("fr_server_create: cannot start the worker thread");
        return FR_ENOMEM;
    }
    *out = s;
    return FR_OK;
}

void fr_server_destroy(fr_server *s)
{
    FR_NVTX("fr_server_destroy");
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->ctx->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    server_free(s);
}

int backtest_submit(fr_server *s, const fr_request *r, uint64_t *ticket)
{
    FR_NVTX("backtest_submit");
    FR_CHECK(s && r && ticket, FR_EINVAL, "backtest_submit: NULL argument");
    FR_CHECK(r->n_envs >= 1 && r->window >= 2 && r->start >= 0 && r->start_stride >= 0 && r->metrics, FR_EINVAL,
             "backtest_submit: need n_envs >= 1, window >= 2, start >= 0, start_stride >= 0, metrics");
    FR_CHECK(!r->want_traj, FR_EINVAL, "backtest_submit: the server returns metrics only (want_traj must be 0)");
    FR_CHECK(r->timeout_s >= 0.0 && r->timeout_s < 1e12, FR_EINVAL, "backtest_submit: timeout_s %g not in [0, 1e12)",
             r->timeout_s);
    const fr_market *m = s->mkt;
    const bool stock = m->task == FR_TASK_STOCK;
    const int64_t horizon = stock ? m->n_days : m->S;
    const int64_t last = (int64_t)r->start + (int64_t)(r->n_envs - 1) * r->start_stride + r->window;
    FR_CHECK(last <= horizon, FR_EINVAL, "backtest_submit: the last env's window ends at %lld, past the market end %lld",
             (long long)last - 1, (long long)horizon);
    if (stock) {
        FR_CHECK(r->n_assets >= 0 && r->n_assets <= m->K, FR_EINVAL, "backtest_submit: n_assets %d not in 0..%d",
                 r->n_assets, m->K);
        FR_CHECK(r->bps_range >= 0 && r->bps_range <= 100, FR_EINVAL, "backtest_submit: bps_range %d not in 0..100",
                 r->bps_range);
    }
    FR_CHECK(r->n_envs <= s->d.capacity, FR_ENOMEM,
             "backtest_submit: %d envs can never fit the server's %d slots", r->n_envs, s->d.capacity);
    FR_CHECK(!fault_hit(FR_FAULT_SUBMIT), FR_EBUSY, "backtest_submit: request rejected (injected fault)");
    SrvReq *q = new (std::nothrow) SrvReq();
    FR_CHECK(q, FR_ENOMEM, "backtest_submit: out of host memory");
    q->r = *r;
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->sticky != FR_OK) {
            delete q;
            set_error("backtest_submit: the server's worker failed earlier");
            return s->sticky;
        }
        q->ticket = s->next_ticket++;
        s->queue.push_back(q);
        s->live[q->ticket] = q;
        s->st.submitted += 1;
        s->st.queued = s->queue.size();
        *ticket = q->ticket;
    }
    s->cv.notify_all();
    return FR_OK;
}

int backtest_poll(fr_server *s, uint64_t ticket, fr_result *out, int32_t *done)
{
    FR_NVTX("backtest_poll");
    FR_CHECK(s && out && done, FR_EINVAL, "backtest_poll: NULL argument");
    *done = 0;
    if (fault_hit(FR_FAULT_POLL)) {
        set_error("backtest_poll: answer dropped (injected fault)");
        return FR_ENOTREADY;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->finished.find(ticket);
    if (it != s->finished.end()) {
        SrvReq *q = it->second;
        out->status = q->status;
        out->n_envs = q->r.n_envs;
        out->queue_s = (q->t_admit > 0 ? q->t_admit : q->t_done) - q->t_submit;
        out->latency_s = q->t_done - q->t_submit;
        *done = 1;
        s->finished.erase(it);
        delete q;
        return FR_OK;
    }
    if (s->live.count(ticket)) return FR_ENOTREADY;
    set_error("backtest_poll: unknown ticket %llu", (unsigned long long)ticket);
    return FR_ENOTFOUND;
}

int backtest_cancel(fr_server *s, uint64_t ticket)
{
    FR_NVTX("backtest_cancel");
    FR_CHECK(s, FR_EINVAL, "backtest_cancel: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->finished.count(ticket)) return FR_OK;                  // complete: no effect
    auto it = s->live.find(ticket);
    if (it == s->live.end()) {
        set_error("backtest_cancel: unknown ticket %llu", (unsigned long long)ticket);
        return FR_ENOTFOUND;
    }
    SrvReq *q = it->second;
    auto qi = std::find(s->queue.begin(), s->queue.end(), q);
    if (qi != s->queue.end()) {                                   // queued: finish now
        s->queue.erase(qi);
        q->status = FR_ECANCELED;
        q->t_done = now_s();
        s->live.erase(it);
        s->finished[ticket] = q;
        s->st.failed += 1;
        s->st.queued = s->queue.size();
    } else {
        q->cancel = true;                                         // running: next chunk boundary
    }
    s->cv.notify_all();
    return FR_OK;
}

int fr_server_stats_get(fr_server *s, fr_server_stats *out)
{
    FR_NVTX("fr_server_stats_get");
    FR_CHECK(s && out, FR_EINVAL, "fr_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    return FR_OK;
}

}  // extern "C"
