// Serving of single-particle adsorption requests (the experiment of §4 of
// Günther et al., arXiv:1109.3277: one ellipsoid released near a flat
// interface, run until its tilt settles) by continuous batching.
//
// One worker thread owns the GPU work.  Its loop:
//   1. admit queued requests in arrival order while a slot is free and the
//      HBM budget holds their footprint (lbe_footprint), creating their
//      lattices; creation overlaps the chunk running on the GPU;
//   2. when the set of running boxes changed, rebuild the batch (one
//      persistent fused kernel and batched particle kernels over all boxes,
//      replayed as a CUDA graph);
//   3. advance every running box by one chunk of CHUNK steps;
//   4. read every box's particle orientation in one gather and retire the
//      boxes whose tilt changed by less than the request's tolerance over
//      the chunk, or that reached their step limit.
// A box's result does not depend on what else runs beside it: batched
// stepping is bit-identical to stepping alone, and each box is checked on
// its own 100-step schedule counted from its admission.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lbe.h"

namespace {

constexpr int CHUNK = 100;  // steps between convergence checks
using Clock = std::chrono::steady_clock;

enum { QUEUED = 0, RUNNING = 1, DONE = 2, FAILED = 3 };

struct Request {
    uint64_t id = 0;
    lbe_lattice_desc d{};
    std::vector<double> rho0;
    int np = 0;
    std::vector<double> blob;  // np x LBE_PARTICLE_IN
    int max_steps = 0;
    double tol = 0.0;
    size_t bytes = 0;
    int state = QUEUED;
    lbe_status err = LBE_OK;
    lbe_ctx *ctx = nullptr;
    int steps = 0;
    double tilt = 0.0;             // at the last check
    std::vector<double> out;       // np x LBE_PARTICLE_OUT
    Clock::time_point t_submit, t_admit, t_done;
};

// Tilt of the body x axis against the z normal, in [0, π/2].
double tilt_of(const double *q)
{
    const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(n > 0)) return 0.0;
    const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    const double az = 2.0 * (x * z - w * y);
    return std::acos(std::min(1.0, std::fabs(az)));
}

}  // namespace

struct lbe_server {
    size_t budget = 0, used = 0;
    int max_slots = 1, storage = 0, device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    // worker-only state
    std::vector<Request *> running;   // in the batch, in batch member order
    std::vector<Request *> joining;   // admitted, not yet in the batch
    lbe_batch *batch = nullptr;
    std::vector<double> quat;
    // statistics
    int64_t completed = 0, node_steps = 0, max_running = 0, chunks = 0;
};

namespace {

void finish(lbe_server *s, Request *r, lbe_status err)
{
    if (r->ctx) {
        if (err == LBE_OK) {
            r->out.assign((size_t)r->np * LBE_PARTICLE_OUT, 0.0);
            std::vector<double> pos(3 * r->np), q(4 * r->np), v(3 * r->np), w(3 * r->np), F(3 * r->np),
                T(3 * r->np);
            err = lbe_read_particles(r->ctx, pos.data(), q.data(), v.data(), w.data(), F.data(), T.data());
            for (int p = 0; p < r->np && err == LBE_OK; p++) {
                double *o = r->out.data() + (size_t)p * LBE_PARTICLE_OUT;
                for (int k = 0; k < 3; k++) {
                    o[k] = pos[3 * p + k];
                    o[7 + k] = v[3 * p + k];
                    o[10 + k] = w[3 * p + k];
                    o[13 + k] = F[3 * p + k];
                    o[16 + k] = T[3 * p + k];
                }
                for (int k = 0; k < 4; k++) o[3 + k] = q[4 * p + k];
                // a run that diverged is a failure, whatever stopped it
                for (int k = 0; k < LBE_PARTICLE_OUT; k++)
                    if (!std::isfinite(o[k])) err = LBE_ENUMERIC;
            }
        }
        lbe_destroy(r->ctx);
        r->ctx = nullptr;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    s->used -= r->bytes;
    r->err = err;
    r->state = err == LBE_OK ? DONE : FAILED;
    r->t_done = Clock::now();
    s->completed++;
    s->cv.notify_all();
}

// Create the lattice of one admitted request (worker thread).
void start(lbe_server *s, Request *r)
{
    lbe_lattice_desc d = r->d;
    d.storage = s->storage;
    d.device = s->device;
    d.cuda_stream = nullptr;
    d.flags = 0;
    lbe_status st = lbe_init_lattice(&d, r->rho0.data(), &r->ctx);
    if (st == LBE_OK && r->np > 0) {
        const int n = r->np;
        std::vector<double> pos(3 * n), q(4 * n), v(3 * n), w(3 * n), rp(n), ro(n), dr(n);
        for (int p = 0; p < n; p++) {
            const double *b = r->blob.data() + (size_t)p * LBE_PARTICLE_IN;
            for (int k = 0; k < 3; k++) {
                pos[3 * p + k] = b[k];
                v[3 * p + k] = b[7 + k];
                w[3 * p + k] = b[10 + k];
            }
            for (int k = 0; k < 4; k++) q[4 * p + k] = b[3 + k];
            rp[p] = b[13];
            ro[p] = b[14];
            dr[p] = b[15];
        }
        st = lbe_add_particles(r->ctx, n, pos.data(), q.data(), v.data(), w.data(), rp.data(), ro.data(),
                               dr.data());
        r->tilt = tilt_of(q.data());
    }
    std::vector<double>().swap(r->rho0);
    if (st != LBE_OK) {
        finish(s, r, st);
        return;
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        r->t_admit = Clock::now();
        r->state = RUNNING;
    }
    s->joining.push_back(r);
}

// Admit queued requests while slots and memory allow (arrival order: a
// request that does not fit blocks the ones behind it, so none starves).
void admit(lbe_server *s)
{
    for (;;) {
        Request *r = nullptr;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->queue.empty()) return;
            const int active = (int)(s->running.size() + s->joining.size());
            Request *h = s->queue.front();
            if (active >= s->max_slots || s->used + h->bytes > s->budget) return;
            s->queue.pop_front();
            s->used += h->bytes;
            r = h;
        }
        start(s, r);
    }
}

void rebuild(lbe_server *s)
{
    if (s->batch) {
        lbe_batch_destroy(s->batch);
        s->batch = nullptr;
    }
    for (Request *r : s->joining) s->running.push_back(r);
    s->joining.clear();
    if (s->running.empty()) return;
    std::vector<lbe_ctx *> m;
    for (Request *r : s->running) m.push_back(r->ctx);
    lbe_status st = lbe_batch_create(m.data(), (int32_t)m.size(), &s->batch);
    if (st != LBE_OK) {
        for (Request *r : s->running) finish(s, r, st);
        s->running.clear();
        s->batch = nullptr;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    s->max_running = std::max<int64_t>(s->max_running, (int64_t)s->running.size());
}

void work(lbe_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        admit(s);
        if (!s->joining.empty()) rebuild(s);
        if (s->running.empty()) {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->stop) break;
            s->cv.wait_for(lock, std::chrono::milliseconds(20));
            continue;
        }
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->stop) break;
        }
        lbe_status st = lbe_batch_step(s->batch, CHUNK);
        // lattices of newly admitted requests are set up while the chunk runs
        admit(s);
        s->quat.assign(4 * s->running.size(), 0.0);
        if (st == LBE_OK) st = lbe_batch_first_quat(s->batch, s->quat.data());
        bool changed = !s->joining.empty();
        std::vector<Request *> keep, done;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->chunks++;
            for (size_t k = 0; k < s->running.size(); k++) {
                Request *r = s->running[k];
                if (st != LBE_OK) {
                    done.push_back(r);
                    continue;
                }
                r->steps += CHUNK;
                s->node_steps += (int64_t)CHUNK * r->d.nx * r->d.ny * r->d.nz;
                const double t = r->np > 0 ? tilt_of(&s->quat[4 * k]) : 0.0;
                const bool settled = r->np > 0 && std::fabs(t - r->tilt) < r->tol;
                r->tilt = t;
                if (settled || r->steps >= r->max_steps || !std::isfinite(t))
                    done.push_back(r);
                else
                    keep.push_back(r);
            }
        }
        if (!done.empty()) {
            changed = true;
            lbe_batch_destroy(s->batch);
            s->batch = nullptr;
            for (Request *r : done) finish(s, r, st != LBE_OK ? st : (std::isfinite(r->tilt) ? LBE_OK : LBE_ENUMERIC));
            s->running = keep;
        }
        if (changed) rebuild(s);
    }
    // shutting down: drop what is left
    if (s->batch) lbe_batch_destroy(s->batch);
    s->batch = nullptr;
    for (Request *r : s->running) finish(s, r, LBE_EBUSY);
    for (Request *r : s->joining) finish(s, r, LBE_EBUSY);
    s->running.clear();
    s->joining.clear();
}

}  // namespace

extern "C" {

lbe_status lbe_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t storage, lbe_server **out)
{
    if (!out || max_slots < 1 || hbm_budget_bytes == 0) return LBE_EINVAL;
    if (storage < LBE_STORE_F32 || storage > LBE_STORE_F16_OFS) return LBE_EINVAL;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBE_ECUDA;
    lbe_server *s = new (std::nothrow) lbe_server();
    if (!s) return LBE_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->storage = storage;
    s->device = dev;
    try {
        s->worker = std::thread(work, s);
    } catch (...) {
        delete s;
        return LBE_ENOMEM;
    }
    *out = s;
    return LBE_OK;
}

lbe_status lbe_server_submit(lbe_server *s, const lbe_lattice_desc *d, const double *rho0, int32_t nparticles,
                             const double *particle_blob, int32_t max_steps, double tilt_tol, uint64_t *req_id)
{
    if (!s || !d || !rho0 || !req_id || nparticles < 0 || (nparticles > 0 && !particle_blob) || max_steps < 1 ||
        !(tilt_tol >= 0))
        return LBE_EINVAL;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || (long long)d->nx * d->ny * d->nz > 0x7fffffffLL) return LBE_EINVAL;
    lbe_lattice_desc dd = *d;
    dd.storage = s->storage;
    const size_t bytes = lbe_footprint(&dd, nparticles);
    if (bytes == 0) return LBE_EINVAL;
    if (bytes > s->budget) return LBE_ENOMEM;
    Request *r = new (std::nothrow) Request();
    if (!r) return LBE_ENOMEM;
    const size_t N = (size_t)d->nx * d->ny * d->nz;
    try {
        r->rho0.assign(rho0, rho0 + 2 * N);
        if (nparticles > 0) r->blob.assign(particle_blob, particle_blob + (size_t)nparticles * LBE_PARTICLE_IN);
    } catch (...) {
        delete r;
        return LBE_ENOMEM;
    }
    r->d = dd;
    r->np = nparticles;
    r->max_steps = ((max_steps + CHUNK - 1) / CHUNK) * CHUNK;
    r->tol = tilt_tol;
    r->bytes = bytes;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) {
            delete r;
            return LBE_EBUSY;
        }
        r->id = s->next_id++;
        s->all[r->id] = r;
        s->queue.push_back(r);
    }
    s->cv.notify_all();
    *req_id = r->id;
    return LBE_OK;
}

lbe_status lbe_server_poll(lbe_server *s, uint64_t req_id, int32_t *done, int32_t *steps_run, double *particle_out)
{
    if (!s) return LBE_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(req_id);
    if (it == s->all.end()) return LBE_EINVAL;
    Request *r = it->second;
    const bool fin = r->state == DONE || r->state == FAILED;
    if (done) *done = fin ? 1 : 0;
    if (steps_run) *steps_run = r->steps;
    if (!fin) return LBE_OK;
    if (r->state == FAILED) return r->err;
    if (particle_out && !r->out.empty()) std::memcpy(particle_out, r->out.data(), r->out.size() * sizeof(double));
    return LBE_OK;
}

lbe_status lbe_server_wait(lbe_server *s, uint64_t req_id, int32_t timeout_ms)
{
    if (!s) return LBE_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->all.find(req_id);
    if (it == s->all.end()) return LBE_EINVAL;
    Request *r = it->second;
    const bool ok = s->cv.wait_for(lock, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                   [&] { return r->state == DONE || r->state == FAILED; });
    return ok ? LBE_OK : LBE_ETIMEOUT;
}

lbe_status lbe_server_timing(lbe_server *s, uint64_t req_id, double *queued_s, double *latency_s)
{
    if (!s) return LBE_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(req_id);
    if (it == s->all.end()) return LBE_EINVAL;
    Request *r = it->second;
    if (r->state != DONE && r->state != FAILED) return LBE_EBUSY;
    using sec = std::chrono::duration<double>;
    if (queued_s) *queued_s = r->state == DONE ? sec(r->t_admit - r->t_submit).count() : 0.0;
    if (latency_s) *latency_s = sec(r->t_done - r->t_submit).count();
    return LBE_OK;
}

lbe_status lbe_server_stats(lbe_server *s, int64_t out[4])
{
    if (!s || !out) return LBE_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    out[0] = s->completed;
    out[1] = s->node_steps;
    out[2] = s->max_running;
    out[3] = s->chunks;
    return LBE_OK;
}

void lbe_server_destroy(lbe_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->all) delete kv.second;
    delete s;
}

}  // extern "C"
