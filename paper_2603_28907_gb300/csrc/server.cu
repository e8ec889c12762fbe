// server.cu -- continuous-batching inversion server on one GPU.
//
// Requests (a problem, its data, its chains and a step budget) arrive at any
// time.  A scheduler thread admits them in arrival order while the device
// memory they would hold fits the budget and a slot is free, builds each one
// its own context on the slot's CUDA stream (chain state stays resident; its
// device memory comes from the server's stream-ordered pool, filled at
// creation, so admission and completion neither allocate from the driver nor
// synchronise the device), and keeps
// every admitted request busy: whenever a request's previous super-step has
// finished on the GPU it launches the next one (one CUDA-graph replay of
// n_within Metropolis steps), so super-steps of different requests overlap on
// the device.  Finished requests read back their chains, free their memory
// and slot, and the next queued requests are admitted.  Latency of every
// super-step (CUDA events on the request's stream) and time from submission
// to posterior (host clock) are recorded.  Each request's result depends
// only on its own inputs and seeds, so it is the same alone and in a mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using clock_t_ = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    mt_request spec{};
    // owned copies of the inputs
    std::vector<double> box, rho, mu, sensors, dirs, h_true;
    std::vector<int32_t> counts;
    std::vector<unsigned char> heights0;
    size_t footprint = 0;
    double t_submit = 0, t_admit = -1, t_done = -1;
    // run state
    mt_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    int slot = -1;
    bool inflight = false;
    double gpu_start = NAN, gpu_end = NAN, gpu_busy = 0.0;  // device clock, ms
    std::atomic<bool> cancel{false};
    int supers_done = 0;
    std::vector<float> superstep_ms;
    // results
    int status = MT_OK;
    std::string error;
    std::vector<unsigned char> heights;
    std::vector<double> ll, lp;
    std::vector<int64_t> accepts;
    bool done = false;
};

size_t elem_size(int precision) { return precision == MT_PREC_F64 ? 8 : 4; }

// Device memory a request holds while admitted (a conservative estimate of
// what its context allocates).
size_t footprint_of(const mt_request &r)
{
    const size_t L = r.n_layers, N = (size_t)r.n_rows * r.n_cols, C = r.n_chains;
    const size_t rays = (size_t)r.n_sensors * r.n_pixels, es = elem_size(r.cfg.precision);
    size_t b = 2 * C * L * N * es;                 // double-buffered heights
    b += C * 64;                                    // per-chain scalars
    b += rays * (16 + 16 + 8 * L + 8 * L + 8 + 24 + 24 + 8 + 8 + 8 + 8 + 4 + 8);  // ray table, counts
    b += C * ((rays + 4095) / 4096) * 8;            // partial sums
    b += L * N * 8 * 2;                             // prior mean, staging
    const size_t rpb = std::min<size_t>(MT_RAYS_PER_CTA, (rays + 255) / 256 * 256);
    if (N * L * 8 + MT_SMEM_STATIC > MT_MAX_SMEM && N * 8 + rpb * 8 + MT_SMEM_STATIC > MT_MAX_SMEM)
        b += C * N * L * 8;                         // HBM (h, dx) planes (not even one plane fits)
    if (r.kernel == MT_KERNEL_MALA)                 // gradients: two slots, accumulator,
        b += 4 * C * L * N * 8 + C * 8 + C * rays * 4;  // staging; Hastings terms; dll/dO
    b += rays * 16 + C * L * N * es;                // output staging
    return b + (8u << 20);                          // allocator slack
}

double now_s(clock_t_::time_point t0)
{
    return std::chrono::duration<double>(clock_t_::now() - t0).count();
}

double pct(std::vector<double> v, double p)
{
    if (v.empty()) return NAN;
    std::sort(v.begin(), v.end());
    const double pos = p * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

struct mt_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_active = 0;
    cudaMemPool_t pool = nullptr;     // device memory of the requests' contexts
    size_t pool_start = 0;            // bytes the pool held once filled
    struct Slot {
        cudaStream_t stream = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
        bool used = false;
    };
    std::vector<Slot> slots;          // max_active streams and events, reused
    cudaEvent_t ev_ref = nullptr;     // device-clock origin
    clock_t_::time_point t0;
    std::mutex mu;
    std::condition_variable cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::vector<std::shared_ptr<Request>> active;
    std::map<int64_t, std::shared_ptr<Request>> all;
    int64_t next_id = 1;
    std::atomic<bool> stop{false};
    std::atomic<int64_t> n_active{0};  // active.size(), which only the scheduler touches
    std::thread worker;
    std::string err;
    // aggregate statistics
    std::vector<double> superstep_ms, ttp_s;
    double chain_ray_evals = 0, first_admit = -1, last_done = -1;
    int64_t n_done = 0;
};

static thread_local std::string g_srv_err;

static mt_status srv_fail(mt_server *s, mt_status st, const std::string &m)
{
    if (s) s->err = m;
    else g_srv_err = m;
    return st;
}

// Set a request up on the device; false (with r->error) on failure.
static bool setup_request(mt_server *s, Request *r)
{
    const mt_request &q = r->spec;
    mt_status st;
    for (size_t i = 0; i < s->slots.size(); ++i)  // a free slot exists: active < max_active
        if (!s->slots[i].used) {
            s->slots[i].used = true;
            r->slot = (int)i;
            r->stream = s->slots[i].stream;
            r->ev_a = s->slots[i].a;
            r->ev_b = s->slots[i].b;
            break;
        }
    if (r->slot < 0) {
        r->error = "no free stream slot";
        r->status = MT_ESTATE;
        return false;
    }
    st = mt::ctx_create_pooled(&r->ctx, s->device, &q.cfg, r->stream, s->pool);
    if (st != MT_OK) {
        r->error = mt_last_error(nullptr);
        r->status = st;
        return false;
    }
    auto chk = [&](mt_status x) {
        if (x != MT_OK && r->status == MT_OK) {
            r->status = x;
            r->error = mt_last_error(r->ctx);
        }
        return x == MT_OK;
    };
    if (!chk(mt_set_grid(r->ctx, q.n_layers, q.n_rows, q.n_cols, r->box.data(), r->rho.data(),
                         r->mu.empty() ? nullptr : r->mu.data())))
        return false;
    if (!chk(mt_set_sensors(r->ctx, q.n_sensors, r->sensors.data()))) return false;
    if (!chk(mt_set_pixels(r->ctx, q.n_pixels, r->dirs.data()))) return false;
    if (!r->counts.empty()) {
        if (!chk(mt_set_counts(r->ctx, r->counts.data()))) return false;
    } else {
        if (!chk(mt_generate_data(r->ctx, r->h_true.data(), q.data_seed, MT_COUNTS_POISSON, nullptr,
                                  nullptr)))
            return false;
    }
    if (!chk(mt_init_chains(r->ctx, q.n_chains, r->heights0.data(), q.seed))) return false;
    return true;
}

static void finish_request(mt_server *s, Request *r)
{
    const mt_request &q = r->spec;
    if (r->status == MT_OK && r->ctx) {
        const size_t n = (size_t)q.n_chains * q.n_layers * q.n_rows * q.n_cols;
        r->heights.resize(n * elem_size(q.cfg.precision));
        r->ll.resize(q.n_chains);
        r->lp.resize(q.n_chains);
        r->accepts.resize(q.n_chains);
        int64_t stp = 0;
        mt_status st = mt_get_state(r->ctx, r->heights.data(), r->ll.data(), r->lp.data(),
                                    r->accepts.data(), &stp);
        if (st != MT_OK) {
            r->status = st;
            r->error = mt_last_error(r->ctx);
        }
    }
    if (r->ctx) mt_destroy(r->ctx);  // its memory goes back to the pool on its stream
    r->ctx = nullptr;
    if (r->slot >= 0) s->slots[r->slot].used = false;  // stream and events are reused
    r->slot = -1;
    r->ev_a = r->ev_b = nullptr;
    r->stream = nullptr;
    std::lock_guard<std::mutex> g(s->mu);
    r->t_done = now_s(s->t0);
    s->used -= r->footprint;
    if (r->status == MT_OK) {
        for (float m : r->superstep_ms) s->superstep_ms.push_back(m);
        s->ttp_s.push_back(r->t_done - r->t_submit);
        s->chain_ray_evals += (double)q.n_chains * q.n_sensors * q.n_pixels * (double)q.n_super *
                              (double)q.n_within;
        s->last_done = r->t_done;
    }
    s->n_done += 1;
    r->done = true;
    s->cv_done.notify_all();
}

// The device memory, streams and events of a server, made once at creation:
// a stream-ordered pool that keeps up to the budget (release threshold) and is
// filled with min(budget, 32 GiB) in 2 GiB blocks, max_active stream slots,
// and the device-clock origin event.  False (with s->err) on failure.
static bool server_reserve(mt_server *s)
{
    auto bad = [&](cudaError_t e, const char *what) {
        cudaGetLastError();
        s->err = std::string("mt_server_create: ") + what + ": " + cudaGetErrorString(e);
        return false;
    };
    cudaError_t e = cudaSetDevice(s->device);
    if (e != cudaSuccess) return bad(e, "cudaSetDevice");
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if ((e = cudaMemPoolCreate(&s->pool, &props)) != cudaSuccess) return bad(e, "cudaMemPoolCreate");
    uint64_t thr = s->budget;
    if ((e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr)) != cudaSuccess)
        return bad(e, "pool release threshold");
    s->slots.resize(s->max_active);
    for (auto &sl : s->slots) {
        if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreate(&sl.a)) != cudaSuccess || (e = cudaEventCreate(&sl.b)) != cudaSuccess)
            return bad(e, "stream / event");
    }
    cudaStream_t st = s->slots[0].stream;
    const size_t block = (size_t)2 << 30, fill = std::min(s->budget, (size_t)32 << 30);
    std::vector<void *> blocks;
    for (size_t got = 0; got < fill;) {
        const size_t want = std::min(block, fill - got);
        void *p = nullptr;
        if (cudaMallocFromPoolAsync(&p, want, s->pool, st) != cudaSuccess) {
            cudaGetLastError();  // the device is fuller than the budget: keep what was reserved
            break;
        }
        blocks.push_back(p);
        got += want;
    }
    for (void *p : blocks) cudaFreeAsync(p, st);
    if ((e = cudaEventCreate(&s->ev_ref)) != cudaSuccess) return bad(e, "cudaEventCreate");
    if ((e = cudaEventRecord(s->ev_ref, st)) != cudaSuccess) return bad(e, "cudaEventRecord");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bad(e, "pool fill");
    uint64_t held = 0;
    cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrReservedMemCurrent, &held);
    s->pool_start = (size_t)held;
    return true;
}

static void server_release(mt_server *s)
{
    cudaSetDevice(s->device);
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.a) cudaEventDestroy(sl.a);
        if (sl.b) cudaEventDestroy(sl.b);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    s->slots.clear();
    if (s->ev_ref) cudaEventDestroy(s->ev_ref);
    s->ev_ref = nullptr;
    if (s->pool) cudaMemPoolDestroy(s->pool);
    s->pool = nullptr;
}

static void worker_loop(mt_server *s)
{
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        bool progress = false;
        // admission: arrival order, memory budget, free slot
        std::vector<std::shared_ptr<Request>> admit;
        {
            std::lock_guard<std::mutex> g(s->mu);
            while (!s->pending.empty() && (int)(s->active.size() + admit.size()) < s->max_active &&
                   s->used + s->pending.front()->footprint <= s->budget) {
                auto r = s->pending.front();
                s->pending.pop_front();
                s->used += r->footprint;
                r->t_admit = now_s(s->t0);
                if (s->first_admit < 0) s->first_admit = r->t_admit;
                admit.push_back(r);
            }
        }
        for (auto &r : admit) {
            progress = true;
            if (setup_request(s, r.get())) {
                s->active.push_back(r);
                s->n_active.store((int64_t)s->active.size());
            } else {
                finish_request(s, r.get());
            }
        }
        // keep every admitted request's stream busy with its next super-step
        for (size_t i = 0; i < s->active.size();) {
            Request *r = s->active[i].get();
            if (r->inflight) {
                cudaError_t e = cudaEventQuery(r->ev_b);
                if (e == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                r->inflight = false;
                progress = true;
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    r->status = MT_ECUDA;
                    r->error = cudaGetErrorString(e);
                } else {
                    float ms = 0.f, ta = 0.f, tb = 0.f;
                    cudaEventElapsedTime(&ms, r->ev_a, r->ev_b);
                    cudaEventElapsedTime(&ta, s->ev_ref, r->ev_a);
                    cudaEventElapsedTime(&tb, s->ev_ref, r->ev_b);
                    if (!(r->gpu_start <= ta)) r->gpu_start = ta;
                    r->gpu_end = tb;
                    r->gpu_busy += ms;
                    r->superstep_ms.push_back(ms);
                    r->supers_done += 1;
                }
            }
            if (r->status == MT_OK && r->cancel.load()) {
                r->status = MT_ECANCELED;
                r->error = "request cancelled";
            }
            if (r->status != MT_OK || r->supers_done >= r->spec.n_super) {
                finish_request(s, r);
                s->active.erase(s->active.begin() + (long)i);
                s->n_active.store((int64_t)s->active.size());
                continue;
            }
            cudaEventRecord(r->ev_a, r->stream);
            mt_status st = mt_run(r->ctx, r->spec.kernel, r->spec.step, 1, r->spec.n_within);
            cudaEventRecord(r->ev_b, r->stream);
            if (st != MT_OK) {
                r->status = st;
                r->error = mt_last_error(r->ctx);
            } else {
                r->inflight = true;
            }
            progress = true;
            ++i;
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    // drain on shutdown
    for (auto &r : s->active) {
        if (r->stream) cudaStreamSynchronize(r->stream);
        r->status = r->status == MT_OK ? MT_ESTATE : r->status;
        r->error = "server shut down before the request finished";
        finish_request(s, r.get());
    }
    s->active.clear();
    s->n_active.store(0);
    // requests never admitted end the same way
    std::lock_guard<std::mutex> g(s->mu);
    for (auto &r : s->pending) {
        r->status = MT_ESTATE;
        r->error = "server shut down before the request was admitted";
        r->t_done = now_s(s->t0);
        s->n_done += 1;
        r->done = true;
    }
    s->pending.clear();
    s->cv_done.notify_all();
}

extern "C" {

MT_API mt_status mt_server_create(mt_server **out, int device, size_t hbm_budget_bytes,
                                  int max_active)
{
    if (!out || hbm_budget_bytes == 0 || max_active < 1)
        return srv_fail(nullptr, MT_EINVAL, "mt_server_create: need out, a budget and max_active >= 1");
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return srv_fail(nullptr, MT_ECUDA, "mt_server_create: no such CUDA device");
    }
    mt_server *s = new (std::nothrow) mt_server();
    if (!s) return srv_fail(nullptr, MT_ENOMEM, "out of host memory");
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->max_active = max_active;
    s->t0 = clock_t_::now();
    if (!server_reserve(s)) {
        std::string m = s->err;
        server_release(s);
        delete s;
        return srv_fail(nullptr, MT_ECUDA, m);
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return MT_OK;
}

MT_API mt_status mt_server_submit(mt_server *s, const mt_request *q, int64_t *id_out)
{
    if (!s || !q) return srv_fail(s, MT_EINVAL, "null argument");
    if (q->n_layers < 1 || q->n_layers > MT_MAX_L || q->n_rows < 2 || q->n_cols < 2 ||
        q->n_sensors < 1 || q->n_pixels < 1 || q->n_chains < 1 || q->n_super < 0 ||
        (q->kernel != MT_KERNEL_RW && q->kernel != MT_KERNEL_MALA) ||
        q->n_within < 1 || !q->box || !q->unit_density || !q->sensors || !q->dirs ||
        !q->heights0 || (!q->counts && !q->h_true))
        return srv_fail(s, MT_EINVAL, "mt_server_submit: incomplete or out-of-range request");
    auto r = std::make_shared<Request>();
    r->spec = *q;
    const size_t L = q->n_layers, N = (size_t)q->n_rows * q->n_cols;
    r->box.assign(q->box, q->box + 3);
    r->rho.assign(q->unit_density, q->unit_density + L + 1);
    if (q->prior_mean) r->mu.assign(q->prior_mean, q->prior_mean + L * N);
    r->sensors.assign(q->sensors, q->sensors + 3 * (size_t)q->n_sensors);
    r->dirs.assign(q->dirs, q->dirs + 3 * (size_t)q->n_pixels);
    if (q->counts) r->counts.assign(q->counts, q->counts + (size_t)q->n_sensors * q->n_pixels);
    else r->h_true.assign(q->h_true, q->h_true + L * N);
    const unsigned char *h0 = (const unsigned char *)q->heights0;
    r->heights0.assign(h0, h0 + (size_t)q->n_chains * L * N * elem_size(q->cfg.precision));
    r->footprint = footprint_of(*q);
    std::lock_guard<std::mutex> g(s->mu);
    if (r->footprint > s->budget)
        return srv_fail(s, MT_ENOMEM, "request needs more device memory than the server's budget");
    r->id = s->next_id++;
    r->t_submit = now_s(s->t0);
    s->pending.push_back(r);
    s->all[r->id] = r;
    if (id_out) *id_out = r->id;
    return MT_OK;
}

MT_API mt_status mt_server_wait(mt_server *s, int64_t id, double timeout_s, void *heights_out,
                                double *loglik_out, double *logprior_out, int64_t *accepts_out,
                                mt_request_info *info)
{
    if (!s) return srv_fail(nullptr, MT_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return srv_fail(s, MT_EINVAL, "unknown request id");
    auto r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
            return srv_fail(s, MT_ETIMEDOUT, "request still running");
    } else {
        s->cv_done.wait(lk, pred);
    }
    if (info) {
        info->status = r->status;
        info->submit_s = r->t_submit;
        info->admit_s = r->t_admit;
        info->done_s = r->t_done;
        std::vector<double> v(r->superstep_ms.begin(), r->superstep_ms.end());
        info->superstep_ms_p50 = pct(v, 0.5);
        info->superstep_ms_p99 = pct(v, 0.99);
        info->n_supersteps = (int)v.size();
        info->gpu_start_ms = r->gpu_start;
        info->gpu_end_ms = r->gpu_end;
        info->gpu_busy_ms = r->gpu_busy;
    }
    if (r->status != MT_OK) return srv_fail(s, (mt_status)r->status, r->error);
    if (heights_out) memcpy(heights_out, r->heights.data(), r->heights.size());
    if (loglik_out) memcpy(loglik_out, r->ll.data(), r->ll.size() * 8);
    if (logprior_out) memcpy(logprior_out, r->lp.data(), r->lp.size() * 8);
    if (accepts_out) memcpy(accepts_out, r->accepts.data(), r->accepts.size() * 8);
    return MT_OK;
}

MT_API mt_status mt_server_cancel(mt_server *s, int64_t id)
{
    if (!s) return srv_fail(nullptr, MT_EINVAL, "null server");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return srv_fail(s, MT_EINVAL, "unknown request id");
    auto r = it->second;
    if (r->done) return srv_fail(s, MT_ESTATE, "request already finished");
    for (auto p = s->pending.begin(); p != s->pending.end(); ++p) {
        if (p->get() != r.get()) continue;
        // never admitted: nothing on the device to release
        s->pending.erase(p);
        r->status = MT_ECANCELED;
        r->error = "request cancelled";
        r->t_done = now_s(s->t0);
        s->n_done += 1;
        r->done = true;
        s->cv_done.notify_all();
        return MT_OK;
    }
    r->cancel.store(true);  // admitted: the scheduler stops it at a super-step boundary
    return MT_OK;
}

MT_API mt_status mt_server_stats(mt_server *s, mt_server_stats_t *out)
{
    if (!s || !out) return srv_fail(s, MT_EINVAL, "null argument");
    std::lock_guard<std::mutex> g(s->mu);
    out->n_done = s->n_done;
    out->n_pending = (int64_t)s->pending.size();
    out->n_active = s->n_active.load();
    out->superstep_ms_p50 = pct(s->superstep_ms, 0.5);
    out->superstep_ms_p99 = pct(s->superstep_ms, 0.99);
    out->ttp_s_p50 = pct(s->ttp_s, 0.5);
    out->ttp_s_p99 = pct(s->ttp_s, 0.99);
    const double span = s->last_done - s->first_admit;
    out->chain_ray_evals_per_s = span > 0 ? s->chain_ray_evals / span : NAN;
    out->bytes_in_use = s->used;
    uint64_t held = 0;
    cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrReservedMemCurrent, &held);
    out->pool_bytes_at_start = s->pool_start;
    out->pool_bytes_now = (size_t)held;
    return MT_OK;
}

MT_API mt_status mt_server_destroy(mt_server *s)
{
    if (!s) return MT_OK;
    s->stop.store(true);
    if (s->worker.joinable()) s->worker.join();
    server_release(s);
    delete s;
    return MT_OK;
}

MT_API const char *mt_server_last_error(const mt_server *s)
{
    return s ? s->err.c_str() : g_srv_err.c_str();
}

}  // extern "C"
