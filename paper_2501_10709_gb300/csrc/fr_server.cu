// fr_server.cu -- backtests as requests, served with continuous batching.
//
// A server owns one or more pools.  A pool is one env batch of `capacity`
// slots over one market, run with one ensemble, with its own stream and
// worker thread; requests name their pool by task and ensemble.  Each
// worker loops: retire the requests that leave (cancelled, past their
// deadline), admit its queued requests into free slots in arrival order
// while the server's HBM budget covers them (the head waits until it
// fits), run the ensemble's rollout over the whole pool for `chunk_steps`
// steps, copy the steps of trajectory-recording requests out of the chunk,
// and retire the requests whose windows are complete (their slots' episode
// metrics to the caller's host buffer; their trajectory stays on the device
// until fetched).  Parked slots are done envs: the rollout kernels leave
// them frozen, so a pool runs one launch sequence whatever mix of requests
// occupies it, and the pools' chunks overlap on the device.  Every request
// starts at a chunk boundary and all of its envs share one window, so its
// completion is known on the host from the number of chunks run.
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

// Copy `steps` rows of a chunk's trajectory (pool layout [chunk][cap][.])
// for the request's envs slot[0..n) into the request's trajectory (layout
// [W - 1][n][.]) starting at its row t0.  One warp per (row, env): the
// observation row by lanes, then the action, reward and done flag.
__global__ void k_traj_gather(fr_traj src, int cap, int D, int K, int stock, const int32_t *slot, int n,
                              int steps, fr_traj dst, int t0)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)steps * n) return;
    const int t = (int)(w / n), i = (int)(w % n);
    const int64_t s = (int64_t)t * cap + slot[i];
    const int64_t d = ((int64_t)(t0 + t)) * n + i;
    for (int k = lane; k < D; k += 32) dst.obs[d * D + k] = src.obs[s * src.obs_ld + k];
    if (stock) {
        for (int k = lane; k < K; k += 32) ((float *)dst.act)[d * K + k] = ((const float *)src.act)[s * K + k];
    } else if (lane == 0) {
        ((uint8_t *)dst.act)[d] = ((const uint8_t *)src.act)[s];
    }
    if (lane == 0) {
        dst.rew[d] = src.rew[s];
        dst.done[d] = src.done[s];
    }
}

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Pool;

struct SrvReq {
    uint64_t ticket;
    fr_request r;
    Pool *pool = nullptr;
    std::vector<int32_t> slots;
    int steps_run = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = FR_OK;
    bool cancel = false;       // set by backtest_cancel while running
    uint64_t slot_bytes = 0;   // budget charge of the slots while running
    uint64_t traj_bytes = 0;   // budget charge of the trajectory until fetched or released
    fr_traj traj{};            // device, [W - 1][n][.], when want_traj
    void *traj_block = nullptr;
};

// FR_OK, or why a request must leave now: cancelled or past its deadline.
int leave_reason(const SrvReq *q, double t)
{
    if (q->cancel) return FR_ECANCELED;
    if (q->r.timeout_s > 0.0 && t - q->t_submit > q->r.timeout_s) return FR_ETIMEDOUT;
    return FR_OK;
}

// Trajectory bytes of one env-step: observation, action, reward, done.
uint64_t traj_row_bytes(int task, int D, int K)
{
    return 4ull * D + (task == FR_TASK_STOCK ? 4ull * K : 1ull) + 8ull + 1ull;
}

}  // namespace
}  // namespace fr

using namespace fr;

namespace fr {
namespace {

struct Pool {
    fr_server *srv = nullptr;
    const fr_market *mkt = nullptr;
    const fr_ensemble *ens = nullptr;
    int task = 0, capacity = 0, chunk = 0;
    fr_env *env = nullptr;
    cudaStream_t stream = nullptr;
    uint64_t slot_bytes = 0;                         // budget charge per admitted env
    uint64_t row_bytes = 0;                          // trajectory bytes per env-step
    // device / pinned staging
    int32_t *d_slot = nullptr, *h_slot = nullptr;
    int32_t *d_gslot = nullptr, *h_gslot = nullptr;  // slots of the trajectory gathers
    SlotCst *d_cst = nullptr, *h_cst = nullptr;
    double *d_met = nullptr, *h_met = nullptr;
    std::vector<int32_t> ke_mirror;
    // the chunk's trajectory for the whole pool, while a request records one
    fr_traj ctraj{};
    void *ctraj_block = nullptr;
    uint64_t ctraj_bytes = 0;
    // scheduler state (under the server's mutex)
    std::deque<SrvReq *> queue;
    std::vector<SrvReq *> running;
    std::vector<int32_t> free_slots;                 // kept sorted, popped from the front
    std::thread worker;
};

}  // namespace
}  // namespace fr

struct fr_server {
    fr_ctx *ctx;
    fr_server_desc d;
    std::vector<Pool *> pools;
    std::mutex mu;
    std::condition_variable cv;
    std::unordered_map<uint64_t, SrvReq *> live;     // queued or running
    std::unordered_map<uint64_t, SrvReq *> finished; // complete, not yet polled / fetched
    uint64_t next_ticket = 1;
    uint64_t budget = 0;                             // 0: no limit beyond the context's
    uint64_t reserved = 0;                           // budget bytes charged to requests
    int sticky = FR_OK;
    bool stop = false;
    fr_server_stats st{};
};

namespace {

// Budget charge of a request, the trajectory included.
uint64_t request_bytes(const Pool *p, const fr_request &r)
{
    uint64_t b = (uint64_t)r.n_envs * p->slot_bytes;
    if (r.want_traj) b += (uint64_t)(r.window - 1) * r.n_envs * p->row_bytes;
    return b;
}

void free_traj(fr_server *s, SrvReq *q)
{
    if (q->traj_block) dev_free(s->ctx, q->traj_block, q->traj_bytes);
    q->traj_block = nullptr;
}

// Under s->mu: a request leaves the scheduler with `status`.  Its slot
// charge is returned now; a trajectory charge stays until the trajectory is
// fetched or released (a failed request's trajectory is released here).
void finish_locked(fr_server *s, SrvReq *q, int status, double t)
{
    q->status = status;
    q->t_done = t;
    s->reserved -= q->slot_bytes;
    q->slot_bytes = 0;
    if (status != FR_OK && q->traj_bytes) {
        free_traj(s, q);
        s->reserved -= q->traj_bytes;
        q->traj_bytes = 0;
    }
    s->live.erase(q->ticket);
    s->finished[q->ticket] = q;
    if (status == FR_OK)
        s->st.completed += 1;
    else if (status == FR_ECANCELED)
        s->st.canceled += 1;
    else if (status == FR_ETIMEDOUT)
        s->st.timed_out += 1;
    else
        s->st.failed += 1;
    s->st.bytes_reserved = s->reserved;
}

void release_all(fr_server *s)
{
    for (auto &kv : s->live) {
        free_traj(s, kv.second);
        delete kv.second;
    }
    for (auto &kv : s->finished) {
        free_traj(s, kv.second);
        delete kv.second;
    }
    s->live.clear();
    s->finished.clear();
    for (Pool *p : s->pools) {
        p->queue.clear();
        p->running.clear();
    }
}

void recount_locked(fr_server *s)
{
    uint64_t q = 0, r = 0;
    for (Pool *p : s->pools) {
        q += p->queue.size();
        r += p->running.size();
    }
    s->st.queued = q;
    s->st.running = r;
}

// Park slots on the pool's stream (they become done envs) and wait.
cudaError_t park(Pool *p, const std::vector<SrvReq *> &reqs)
{
    int n = 0;
    for (SrvReq *q : reqs)
        for (int32_t e : q->slots) p->h_slot[n++] = e;
    if (n == 0) return cudaSuccess;
    cudaError_t ce = cudaMemcpyAsync(p->d_slot, p->h_slot, 4ull * n, cudaMemcpyHostToDevice, p->stream);
    if (ce == cudaSuccess) {
        k_slot_park<<<ceil_div(n, 128), 128, 0, p->stream>>>(p->env->v, p->d_slot, n);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(p->stream);
    return ce;
}

// Upload the slot constants of newly admitted requests and reset their
// slots; returns a CUDA status.
cudaError_t assign(Pool *p, const std::vector<SrvReq *> &adm, bool &ke_changed)
{
    const bool stock = p->task == FR_TASK_STOCK;
    int n = 0;
    for (SrvReq *q : adm) {
        const fr_request &r = q->r;
        const int ke = stock ? (r.n_assets > 0 ? r.n_assets : p->env->v.K) : 1;
        for (int i = 0; i < r.n_envs; ++i, ++n) {
            const int32_t e = q->slots[i];
            p->h_slot[n] = e;
            SlotCst &c = p->h_cst[n];
            c.start = r.start + i * r.start_stride;
            c.window = r.window;
            c.ke = ke;
            c.range = stock ? r.bps_range : 0;
            c.index = i;
            c.pad = 0;
            c.seed = r.seed;
            if (p->ke_mirror[e] != ke) ke_changed = true;
            p->ke_mirror[e] = ke;
        }
    }
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(p->d_slot, p->h_slot, 4ull * n, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_cst, p->h_cst, sizeof(SlotCst) * n, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return e;
    k_slot_assign<<<n, KP, 0, p->stream>>>(p->env->v, p->d_slot, p->d_cst, n);
    e = cudaGetLastError();
    // the staging buffers are reused by the next admission: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    return e;
}

void fail_all(fr_server *s, int rc)
{
    std::lock_guard<std::mutex> lk(s->mu);
    s->sticky = rc;
    const double t = now_s();
    for (Pool *p : s->pools) {
        for (SrvReq *q : p->running) finish_locked(s, q, rc, t);
        for (SrvReq *q : p->queue) finish_locked(s, q, rc, t);
        p->running.clear();
        p->queue.clear();
        p->free_slots.resize(p->capacity);
        for (int i = 0; i < p->capacity; ++i) p->free_slots[i] = i;
    }
    recount_locked(s);
    s->cv.notify_all();
}

// A chunk failed without a CUDA error (the context is still usable): the
// pool's running requests finish with status rc, their slots are parked
// and freed, and the queued requests stay.  Returns a CUDA status.
cudaError_t fail_running(Pool *p, int rc)
{
    fr_server *s = p->srv;
    const cudaError_t ce = park(p, p->running);
    if (ce != cudaSuccess) return ce;
    std::lock_guard<std::mutex> lk(s->mu);
    const double t = now_s();
    for (SrvReq *q : p->running) {
        p->free_slots.insert(p->free_slots.end(), q->slots.begin(), q->slots.end());
        finish_locked(s, q, rc, t);
    }
    p->running.clear();
    std::sort(p->free_slots.begin(), p->free_slots.end());
    recount_locked(s);
    s->cv.notify_all();
    return cudaSuccess;
}

// At a chunk boundary: queued requests past their deadline finish at once;
// running ones that were cancelled or are past their deadline are parked
// and their slots freed.  Returns a CUDA status (parking the slots).
cudaError_t retire_leavers(Pool *p)
{
    fr_server *s = p->srv;
    std::vector<SrvReq *> gone;
    std::vector<int> why;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const double t = now_s();
        for (auto it = p->queue.begin(); it != p->queue.end();) {
            SrvReq *q = *it;
            const int st = leave_reason(q, t);
            if (st == FR_OK) {
                ++it;
                continue;
            }
            finish_locked(s, q, st, t);
            it = p->queue.erase(it);
        }
        for (SrvReq *q : p->running) {
            const int st = leave_reason(q, t);
            if (st != FR_OK) {
                gone.push_back(q);
                why.push_back(st);
            }
        }
        recount_locked(s);
    }
    if (gone.empty()) return cudaSuccess;
    const cudaError_t ce = park(p, gone);
    if (ce != cudaSuccess) return ce;
    std::lock_guard<std::mutex> lk(s->mu);
    const double t = now_s();
    for (size_t i = 0; i < gone.size(); ++i) {
        SrvReq *q = gone[i];
        p->running.erase(std::find(p->running.begin(), p->running.end(), q));
        p->free_slots.insert(p->free_slots.end(), q->slots.begin(), q->slots.end());
        finish_locked(s, q, why[i], t);
    }
    std::sort(p->free_slots.begin(), p->free_slots.end());
    recount_locked(s);
    s->cv.notify_all();
    return cudaSuccess;
}

// The chunk's trajectory buffer for the whole pool (device, charged to the
// context), made when a running request first records one.
int ensure_chunk_traj(Pool *p)
{
    if (p->ctraj_block) return FR_OK;
    const EnvView &v = p->env->v;
    const uint64_t rows = (uint64_t)p->chunk * p->capacity;
    const uint64_t ob = (4ull * v.D * rows + 255) & ~255ull;
    const uint64_t ab = ((p->task == FR_TASK_STOCK ? 4ull * v.K : 1ull) * rows + 255) & ~255ull;
    const uint64_t rb = (8ull * rows + 255) & ~255ull;
    const uint64_t db = (rows + 255) & ~255ull;
    int rc = dev_alloc(p->env->ctx, &p->ctraj_block, ob + ab + rb + db);
    if (rc) return rc;
    p->ctraj_bytes = ob + ab + rb + db;
    char *b = (char *)p->ctraj_block;
    p->ctraj.obs = (float *)b;
    p->ctraj.obs_ld = v.D;
    p->ctraj.act = b + ob;
    p->ctraj.rew = (int64_t *)(b + ob + ab);
    p->ctraj.rew_f32 = nullptr;
    p->ctraj.done = (uint8_t *)(b + ob + ab + rb);
    return FR_OK;
}

// The request's own trajectory buffer (device, [W - 1][n][.]).
int alloc_request_traj(Pool *p, SrvReq *q)
{
    const EnvView &v = p->env->v;
    const uint64_t rows = (uint64_t)(q->r.window - 1) * q->r.n_envs;
    const uint64_t ob = (4ull * v.D * rows + 255) & ~255ull;
    const uint64_t ab = ((p->task == FR_TASK_STOCK ? 4ull * v.K : 1ull) * rows + 255) & ~255ull;
    const uint64_t rb = (8ull * rows + 255) & ~255ull;
    const uint64_t db = (rows + 255) & ~255ull;
    int rc = dev_alloc(p->env->ctx, &q->traj_block, ob + ab + rb + db);
    if (rc) return rc;
    char *b = (char *)q->traj_block;
    q->traj.obs = (float *)b;
    q->traj.obs_ld = v.D;
    q->traj.act = b + ob;
    q->traj.rew = (int64_t *)(b + ob + ab);
    q->traj.rew_f32 = nullptr;
    q->traj.done = (uint8_t *)(b + ob + ab + rb);
    // the budget charge stays the request's planned bytes; the block is
    // released with dev_free of its own size
    q->traj_bytes = ob + ab + rb + db;
    return FR_OK;
}

void worker_loop(Pool *p)
{
    fr_server *s = p->srv;
    cudaSetDevice(s->ctx->device);
    const int chunk = p->chunk;
    const int N = p->capacity;
    const EnvView &v = p->env->v;
    for (;;) {
        {
            const cudaError_t rc = retire_leavers(p);
            if (rc != cudaSuccess) {
                cuda_fail(rc, "server: retiring cancelled requests");
                fail_all(s, FR_ECUDA);
                return;
            }
        }
        std::vector<SrvReq *> admitted, no_memory;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::milliseconds(2),
                           [&] { return s->stop || !p->queue.empty() || !p->running.empty(); });
            if (s->stop) return;
            // the head of the queue waits until its slots and bytes fit
            while (!p->queue.empty()) {
                SrvReq *q = p->queue.front();
                const uint64_t need = request_bytes(p, q->r);
                if ((int)p->free_slots.size() < q->r.n_envs || (s->budget && s->reserved + need > s->budget)) break;
                p->queue.pop_front();
                q->slots.assign(p->free_slots.begin(), p->free_slots.begin() + q->r.n_envs);
                p->free_slots.erase(p->free_slots.begin(), p->free_slots.begin() + q->r.n_envs);
                q->t_admit = now_s();
                q->slot_bytes = (uint64_t)q->r.n_envs * p->slot_bytes;
                q->traj_bytes = need - q->slot_bytes;
                s->reserved += need;
                s->st.bytes_peak = std::max(s->st.bytes_peak, s->reserved);
                s->st.bytes_reserved = s->reserved;
                admitted.push_back(q);
            }
            recount_locked(s);
        }
        // trajectory buffers of the admitted recording requests (outside the
        // lock: device allocations); one the context cannot hold fails
        for (SrvReq *q : admitted) {
            if (!q->r.want_traj) continue;
            const uint64_t charge = q->traj_bytes;
            int rc = alloc_request_traj(p, q);
            if (rc == FR_OK) rc = ensure_chunk_traj(p);
            if (rc) {
                std::lock_guard<std::mutex> lk(s->mu);
                free_traj(s, q);
                q->traj_bytes = charge;
                p->free_slots.insert(p->free_slots.end(), q->slots.begin(), q->slots.end());
                std::sort(p->free_slots.begin(), p->free_slots.end());
                q->slots.clear();
                finish_locked(s, q, rc, now_s());
                no_memory.push_back(q);
                continue;
            }
            // keep the planned charge (rounding of the block is the context's)
            std::lock_guard<std::mutex> lk(s->mu);
            const uint64_t got = q->traj_bytes;
            s->reserved = s->reserved - charge + got;
            s->st.bytes_peak = std::max(s->st.bytes_peak, s->reserved);
            s->st.bytes_reserved = s->reserved;
        }
        if (!no_memory.empty()) {
            std::vector<SrvReq *> keep;
            for (SrvReq *q : admitted)
                if (std::find(no_memory.begin(), no_memory.end(), q) == no_memory.end()) keep.push_back(q);
            admitted.swap(keep);
            std::lock_guard<std::mutex> lk(s->mu);
            s->cv.notify_all();
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            p->running.insert(p->running.end(), admitted.begin(), admitted.end());
            recount_locked(s);
            if (p->running.empty()) continue;
        }
        const double t0 = now_s();
        bool ke_changed = false;
        cudaError_t ce = assign(p, admitted, ke_changed);
        if (ce != cudaSuccess) {
            cuda_fail(ce, "server: slot assignment");
            fail_all(s, FR_ECUDA);
            return;
        }
        if (!admitted.empty()) p->env->pack_state = 0;       // windows changed: re-pack the tiles
        if (ke_changed && p->env->slot_of_env) {
            // the fused stock kernel rebuilds its asset-count slots
            dev_free(s->ctx, p->env->slot_of_env, 4ull * N + 4ull * 32);
            p->env->slot_of_env = nullptr;
            p->env->slot_ke = nullptr;
        }
        bool recording = false;
        for (SrvReq *q : p->running) recording = recording || q->r.want_traj;
        int rc = rollout(p->env, p->ens, chunk, recording ? &p->ctraj : nullptr, nullptr, p->stream);
        if (rc == FR_ECUDA) {
            fail_all(s, rc);
            return;
        }
        if (rc) {
            ce = fail_running(p, rc);
            if (ce != cudaSuccess) {
                cuda_fail(ce, "server: parking failed requests");
                fail_all(s, FR_ECUDA);
                return;
            }
            continue;
        }
        // the recording requests' steps of this chunk into their own buffers
        if (recording) {
            int off = 0;
            for (SrvReq *q : p->running) {
                if (!q->r.want_traj) continue;
                const int steps = std::min(chunk, q->r.window - 1 - q->steps_run);
                if (steps <= 0) continue;
                std::copy(q->slots.begin(), q->slots.end(), p->h_gslot + off);
                ce = cudaMemcpyAsync(p->d_gslot + off, p->h_gslot + off, 4ull * q->slots.size(), cudaMemcpyHostToDevice,
                                     p->stream);
                if (ce != cudaSuccess) break;
                const int64_t warps = (int64_t)steps * q->r.n_envs;
                k_traj_gather<<<(unsigned)ceil_div(warps * 32, 256), 256, 0, p->stream>>>(
                    p->ctraj, N, v.D, v.K, p->task == FR_TASK_STOCK, p->d_gslot + off, q->r.n_envs, steps, q->traj,
                    q->steps_run);
                ce = cudaGetLastError();
                if (ce != cudaSuccess) break;
                off += (int)q->slots.size();
            }
            if (ce != cudaSuccess) {
                cuda_fail(ce, "server: trajectory copy");
                fail_all(s, FR_ECUDA);
                return;
            }
        }
        // the worker alone touches running requests' progress
        std::vector<SrvReq *> done;
        for (SrvReq *q : p->running) {
            q->steps_run += chunk;
            if (q->steps_run >= q->r.window - 1) done.push_back(q);
        }
        if (!done.empty()) {
            ce = launch_env_metrics(v, p->d_met, p->stream);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(p->h_met, p->d_met, 24ull * N, cudaMemcpyDeviceToHost, p->stream);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(p->stream);
            if (ce == cudaSuccess) ce = park(p, done);
            if (ce != cudaSuccess) {
                cuda_fail(ce, "server: retiring requests");
                fail_all(s, FR_ECUDA);
                return;
            }
            for (SrvReq *q : done)
                for (int i = 0; i < q->r.n_envs; ++i)
                    for (int j = 0; j < 3; ++j) q->r.metrics[3 * i + j] = p->h_met[3 * (size_t)q->slots[i] + j];
        } else {
            ce = cudaStreamSynchronize(p->stream);
            if (ce != cudaSuccess) {
                cuda_fail(ce, "server: rollout chunk");
                fail_all(s, FR_ECUDA);
                return;
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            const double t = now_s();
            for (SrvReq *q : done) {
                p->running.erase(std::find(p->running.begin(), p->running.end(), q));
                p->free_slots.insert(p->free_slots.end(), q->slots.begin(), q->slots.end());
                s->st.env_steps += (double)q->r.n_envs * (q->r.window - 1);
                finish_locked(s, q, FR_OK, t);
            }
            if (!done.empty()) std::sort(p->free_slots.begin(), p->free_slots.end());
            s->st.pool_steps += (double)N * chunk;
            s->st.busy_s += now_s() - t0;
            recount_locked(s);
            if (!done.empty()) s->cv.notify_all();
        }
    }
}

void pool_free(fr_server *s, Pool *p)
{
    if (p->env) env_destroy(p->env);
    if (p->ctraj_block) dev_free(s->ctx, p->ctraj_block, p->ctraj_bytes);
    if (p->d_slot) cudaFree(p->d_slot);
    if (p->d_gslot) cudaFree(p->d_gslot);
    if (p->d_cst) cudaFree(p->d_cst);
    if (p->d_met) cudaFree(p->d_met);
    if (p->h_slot) cudaFreeHost(p->h_slot);
    if (p->h_gslot) cudaFreeHost(p->h_gslot);
    if (p->h_cst) cudaFreeHost(p->h_cst);
    if (p->h_met) cudaFreeHost(p->h_met);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

void server_free(fr_server *s)
{
    release_all(s);
    for (Pool *p : s->pools) pool_free(s, p);
    s->pools.clear();
    delete s;
}

// A pool for (market, ensemble): its env batch, stream and staging; every
// slot starts parked.  The worker is started by the caller.
int pool_create(fr_server *s, const fr_market *m, const fr_ensemble *e, int capacity, int chunk_steps, Pool **out)
{
    *out = nullptr;
    FR_CHECK(m && e, FR_EINVAL, "server pool: NULL market or ensemble");
    FR_CHECK(capacity >= 1 && chunk_steps >= 1, FR_EINVAL, "server pool: capacity %d and chunk_steps %d must be >= 1",
             capacity, chunk_steps);
    FR_CHECK(m->ctx == s->ctx && e->ctx == s->ctx, FR_EINVAL, "server pool: market and ensemble of another context");
    const bool stock = m->task == FR_TASK_STOCK;
    FR_CHECK(e->dims[0] == (stock ? 1 + 2 * m->K + m->I * m->K : FR_CRYPTO_OBS_DIM), FR_EINVAL,
             "server pool: ensemble input %d does not match the market's observation", e->dims[0]);
    FR_CHECK(stock ? (e->combine == FR_COMBINE_MEAN && e->dims[e->L] == m->K)
                   : (e->combine == FR_COMBINE_VOTE && e->n_act == 3),
             FR_EINVAL, "server pool: ensemble combine/output does not match the task");
    for (Pool *q : s->pools)
        FR_CHECK(q->ens != e, FR_EINVAL, "server pool: the ensemble already has a pool in this server");
    Pool *p = new (std::nothrow) Pool();
    FR_CHECK(p, FR_ENOMEM, "server pool: out of host memory");
    p->srv = s;
    p->mkt = m;
    p->ens = e;
    p->task = m->task;
    p->capacity = capacity;
    p->chunk = chunk_steps;
    const int N = capacity;
    std::vector<int32_t> win(N, 2), start(N, 0);
    fr_env_desc ed{};
    ed.task = m->task;
    ed.n_envs = N;
    ed.window = win.data();
    ed.start = start.data();
    ed.init_cash = s->d.init_cash;
    ed.hmax = s->d.hmax;
    ed.fee_bps = s->d.fee_bps;
    ed.pmax = s->d.pmax;
    int rc = env_create(s->ctx, &ed, m, &p->env);
    if (rc) {
        pool_free(s, p);
        return rc;
    }
    p->slot_bytes = (p->env->bytes + (uint64_t)N - 1) / (uint64_t)N;
    p->row_bytes = traj_row_bytes(p->task, p->env->v.D, p->env->v.K);
    p->ke_mirror.assign(N, stock ? m->K : 1);
    cudaError_t ce = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->d_slot, 4ull * N);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->d_gslot, 4ull * N);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->d_cst, sizeof(SlotCst) * N);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->d_met, 24ull * N);
    if (ce == cudaSuccess) ce = cudaMallocHost(&p->h_slot, 4ull * N);
    if (ce == cudaSuccess) ce = cudaMallocHost(&p->h_gslot, 4ull * N);
    if (ce == cudaSuccess) ce = cudaMallocHost(&p->h_cst, sizeof(SlotCst) * N);
    if (ce == cudaSuccess) ce = cudaMallocHost(&p->h_met, 24ull * N);
    if (ce != cudaSuccess) {
        pool_free(s, p);
        return cuda_fail(ce, "server pool");
    }
    for (int i = 0; i < N; ++i) p->h_slot[i] = i;
    ce = cudaMemcpy(p->d_slot, p->h_slot, 4ull * N, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
        k_slot_park<<<ceil_div(N, 128), 128, 0, p->stream>>>(p->env->v, p->d_slot, N);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(p->stream);
    if (ce != cudaSuccess) {
        pool_free(s, p);
        return cuda_fail(ce, "server pool: parking slots");
    }
    p->free_slots.resize(N);
    for (int i = 0; i < N; ++i) p->free_slots[i] = i;
    *out = p;
    return FR_OK;
}

int start_worker(Pool *p)
{
    try {
        p->worker = std::thread(worker_loop, p);
    } catch (...) {
        set_error("server pool: cannot start the worker thread");
        return FR_ENOMEM;
    }
    return FR_OK;
}

void stop_workers(fr_server *s)
{
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (Pool *p : s->pools)
        if (p->worker.joinable()) p->worker.join();
}

// The pool that serves a request: its ensemble's, else the first of its task.
Pool *route(fr_server *s, const fr_request *r)
{
    for (Pool *p : s->pools)
        if (r->ens ? p->ens == r->ens : p->task == r->task) return p;
    return nullptr;
}

}  // namespace

extern "C" {

int fr_server_create(fr_ctx *ctx, const fr_server_desc *d, fr_server **out)
{
    FR_NVTX("fr_server_create");
    FR_CHECK(ctx && d && out && d->market && d->ens, FR_EINVAL, "fr_server_create: NULL argument");
    *out = nullptr;
    FR_CUDA(cudaSetDevice(ctx->device));
    fr_server *s = new (std::nothrow) fr_server();
    FR_CHECK(s, FR_ENOMEM, "fr_server_create: out of host memory");
    s->ctx = ctx;
    s->d = *d;
    s->budget = d->hbm_budget;
    s->st.budget = s->budget;
    Pool *p = nullptr;
    int rc = pool_create(s, d->market, d->ens, d->capacity, d->chunk_steps, &p);
    if (rc) {
        server_free(s);
        return rc;
    }
    s->pools.push_back(p);
    s->st.pools = 1;
    if ((rc = start_worker(p))) {
        server_free(s);
        return rc;
    }
    *out = s;
    return FR_OK;
}

int fr_server_add_pool(fr_server *s, const fr_market *market, const fr_ensemble *ens, int32_t capacity,
                       int32_t chunk_steps)
{
    FR_NVTX("fr_server_add_pool");
    FR_CHECK(s, FR_EINVAL, "fr_server_add_pool: NULL server");
    FR_CUDA(cudaSetDevice(s->ctx->device));
    Pool *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        FR_CHECK(s->sticky == FR_OK, s->sticky, "fr_server_add_pool: the server's worker failed earlier");
    }
    int rc = pool_create(s, market, ens, capacity, chunk_steps, &p);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->pools.push_back(p);
        s->st.pools = s->pools.size();
    }
    return start_worker(p);
}

void fr_server_destroy(fr_server *s)
{
    FR_NVTX("fr_server_destroy");
    if (!s) return;
    stop_workers(s);
    cudaSetDevice(s->ctx->device);
    for (Pool *p : s->pools)
        if (p->stream) cudaStreamSynchronize(p->stream);
    server_free(s);
}

int backtest_submit(fr_server *s, const fr_request *r, uint64_t *ticket)
{
    FR_NVTX("backtest_submit");
    FR_CHECK(s && r && ticket, FR_EINVAL, "backtest_submit: NULL argument");
    FR_CHECK(r->n_envs >= 1 && r->window >= 2 && r->start >= 0 && r->start_stride >= 0 && r->metrics, FR_EINVAL,
             "backtest_submit: need n_envs >= 1, window >= 2, start >= 0, start_stride >= 0, metrics");
    FR_CHECK(r->want_traj == 0 || r->want_traj == 1, FR_EINVAL, "backtest_submit: want_traj %d not 0 or 1",
             r->want_traj);
    FR_CHECK(r->task == FR_TASK_STOCK || r->task == FR_TASK_CRYPTO, FR_EINVAL, "backtest_submit: task %d", r->task);
    FR_CHECK(r->timeout_s >= 0.0 && r->timeout_s < 1e12, FR_EINVAL, "backtest_submit: timeout_s %g not in [0, 1e12)",
             r->timeout_s);
    Pool *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        p = route(s, r);
    }
    FR_CHECK(p, FR_EINVAL, "backtest_submit: no pool of this server serves the request's %s",
             r->ens ? "ensemble" : "task");
    FR_CHECK(p->task == r->task, FR_EINVAL, "backtest_submit: the ensemble's pool runs task %d, the request is task %d",
             p->task, r->task);
    const fr_market *m = p->mkt;
    const bool stock = p->task == FR_TASK_STOCK;
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
    FR_CHECK(r->n_envs <= p->capacity, FR_ENOMEM, "backtest_submit: %d envs can never fit the pool's %d slots",
             r->n_envs, p->capacity);
    const uint64_t need = request_bytes(p, *r);
    FR_CHECK(!s->budget || need <= s->budget, FR_ENOMEM,
             "backtest_submit: the request needs %llu bytes on the device, more than the server's budget %llu",
             (unsigned long long)need, (unsigned long long)s->budget);
    FR_CHECK(!fault_hit(FR_FAULT_SUBMIT), FR_EBUSY, "backtest_submit: request rejected (injected fault)");
    SrvReq *q = new (std::nothrow) SrvReq();
    FR_CHECK(q, FR_ENOMEM, "backtest_submit: out of host memory");
    q->r = *r;
    q->pool = p;
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->sticky != FR_OK) {
            delete q;
            set_error("backtest_submit: the server's worker failed earlier");
            return s->sticky;
        }
        q->ticket = s->next_ticket++;
        p->queue.push_back(q);
        s->live[q->ticket] = q;
        s->st.submitted += 1;
        recount_locked(s);
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
        out->task = q->pool ? q->pool->task : q->r.task;
        out->traj_steps = q->traj_block ? q->r.window - 1 : 0;
        out->traj_bytes = q->traj_block ? q->traj_bytes : 0;
        *done = 1;
        if (!q->traj_block) {                          // nothing left on the device: the ticket ends
            s->finished.erase(it);
            delete q;
        }
        return FR_OK;
    }
    if (s->live.count(ticket)) return FR_ENOTREADY;
    set_error("backtest_poll: unknown ticket %llu", (unsigned long long)ticket);
    return FR_ENOTFOUND;
}

int backtest_fetch_traj(fr_server *s, uint64_t ticket, const fr_traj *dst, void *stream)
{
    FR_NVTX("backtest_fetch_traj");
    FR_CHECK(s && dst, FR_EINVAL, "backtest_fetch_traj: NULL argument");
    SrvReq *q = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->finished.find(ticket);
        if (it == s->finished.end() || !it->second->traj_block) {
            set_error("backtest_fetch_traj: ticket %llu has no trajectory to fetch", (unsigned long long)ticket);
            return s->live.count(ticket) ? FR_ENOTREADY : FR_ENOTFOUND;
        }
        q = it->second;
        s->finished.erase(it);                         // the caller now owns the fetch
    }
    FR_CUDA(cudaSetDevice(s->ctx->device));
    const Pool *p = q->pool;
    const uint64_t rows = (uint64_t)(q->r.window - 1) * q->r.n_envs;
    const int D = p->env->v.D;
    const int ld = dst->obs_ld ? dst->obs_ld : D;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t ce = cudaSuccess;
    if (dst->obs && ld < D) ce = cudaErrorInvalidValue;
    if (ce == cudaSuccess && dst->obs)
        ce = cudaMemcpy2DAsync(dst->obs, 4ull * ld, q->traj.obs, 4ull * D, 4ull * D, rows, cudaMemcpyDefault, st);
    if (ce == cudaSuccess && dst->act)
        ce = cudaMemcpyAsync(dst->act, q->traj.act, (p->task == FR_TASK_STOCK ? 4ull * p->env->v.K : 1ull) * rows,
                             cudaMemcpyDefault, st);
    if (ce == cudaSuccess && dst->rew) ce = cudaMemcpyAsync(dst->rew, q->traj.rew, 8ull * rows, cudaMemcpyDefault, st);
    if (ce == cudaSuccess && dst->done) ce = cudaMemcpyAsync(dst->done, q->traj.done, rows, cudaMemcpyDefault, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    std::lock_guard<std::mutex> lk(s->mu);
    free_traj(s, q);
    s->reserved -= q->traj_bytes;
    s->st.bytes_reserved = s->reserved;
    delete q;
    s->cv.notify_all();
    if (ce != cudaSuccess) return cuda_fail(ce, "backtest_fetch_traj");
    return FR_OK;
}

int backtest_release(fr_server *s, uint64_t ticket)
{
    FR_NVTX("backtest_release");
    FR_CHECK(s, FR_EINVAL, "backtest_release: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->finished.find(ticket);
    if (it == s->finished.end()) {
        set_error("backtest_release: ticket %llu is not complete", (unsigned long long)ticket);
        return s->live.count(ticket) ? FR_ENOTREADY : FR_ENOTFOUND;
    }
    SrvReq *q = it->second;
    s->finished.erase(it);
    free_traj(s, q);
    s->reserved -= q->traj_bytes;
    s->st.bytes_reserved = s->reserved;
    delete q;
    s->cv.notify_all();
    return FR_OK;
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
    auto qi = std::find(q->pool->queue.begin(), q->pool->queue.end(), q);
    if (qi != q->pool->queue.end()) {                             // queued: finish now
        q->pool->queue.erase(qi);
        finish_locked(s, q, FR_ECANCELED, now_s());
        recount_locked(s);
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
