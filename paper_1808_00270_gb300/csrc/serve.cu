// serve.cu -- the serving loop of include/gld.h (gld_server_*): requests for
// GLD simulations of different sizes, densities and memory lengths are
// admitted by the device bytes their systems need, keep all state on the
// device, and are stepped together as one batch (continuous batching: the
// composition may change at every 64-step block boundary, while the next
// block is already queued on the device).
//
// Streams: every batched block, tail step and result read-back runs on the
// server's stream S; contexts are created (and freed) on a private admission
// stream A, so that admitting a request never waits for the blocks in flight.
// Member memory comes from a private stream-ordered pool (no device-wide
// synchronisation on allocation or release).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include "ctx.h"

namespace {

enum ReqState { kQueued = 0, kActive = 1, kRetiring = 2, kDone = 3, kFailed = 4, kCancelling = 5 };

struct Slab {  // pinned host memory for a result in flight
    char* p = nullptr;
    size_t cap = 0;
};

struct Req {
    int64_t id = 0;
    gld_params prm{};
    std::vector<double> pos, vel, Ks, g, f, gs, fs;
    int32_t Q = 0, Qs = 0, nr = 2, conv = GLD_KCONT, keep_state = 0, pn_deg = 0;
    double dr = 1.0;
    int64_t steps = 0, left = 0;
    double arrival = 0, admitted = -1, done = -1;
    size_t bytes = 0;
    int state = kQueued;
    gld_status status = GLD_OK;
    std::string msg;
    gld_ctx* ctx = nullptr;
    cudaEvent_t ev = nullptr;
    Slab slab;
    std::vector<double> vacf, out_pos, out_vel;
    int64_t n_origins = 0;
};

}  // namespace

struct gld_server {
    gld_server_params sp{};
    cudaStream_t S = nullptr, A = nullptr;
    bool own_S = false;
    cudaMemPool_t pool = nullptr;
    gld_batch* batch = nullptr;
    std::vector<Req*> reqs;     // by id
    std::deque<Req*> queue;     // arrival order
    std::vector<Req*> active;   // members of the batch
    std::vector<Req*> retiring; // results in flight
    std::vector<Req*> cancelling; // cancelled members waiting for their queued blocks
    std::deque<cudaEvent_t> inflight;
    std::vector<cudaEvent_t> spare_ev;
    std::vector<Slab> spare_slab;
    size_t used = 0, budget = 0, peak = 0;
    int64_t blocks = 0, psteps = 0, n_done = 0, n_failed = 0, peak_members = 0;
    std::chrono::steady_clock::time_point t0;
    std::string msg;
};

namespace {

double now_s(const gld_server* s)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

void* pool_alloc(size_t bytes, void*, void* user)
{
    gld_server* s = (gld_server*)user;
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, s->pool, s->A) != cudaSuccess) return nullptr;
    return p;
}

void pool_free(void* p, void*, void* user)
{
    gld_server* s = (gld_server*)user;
    cudaFreeAsync(p, s->A);
}

cudaEvent_t take_event(gld_server* s)
{
    if (!s->spare_ev.empty()) {
        cudaEvent_t e = s->spare_ev.back();
        s->spare_ev.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

bool take_slab(gld_server* s, size_t need, Slab& out)
{
    for (size_t k = 0; k < s->spare_slab.size(); ++k)
        if (s->spare_slab[k].cap >= need) {
            out = s->spare_slab[k];
            s->spare_slab.erase(s->spare_slab.begin() + (long)k);
            return true;
        }
    out.cap = std::max(need, (size_t)1 << 16);
    if (cudaHostAlloc((void**)&out.p, out.cap, cudaHostAllocDefault) != cudaSuccess) {
        out = Slab{};
        return false;
    }
    return true;
}

void fail_req(gld_server* s, Req* r, gld_status st, const std::string& m)
{
    r->status = st;
    r->msg = m;
    r->state = kFailed;
    r->done = now_s(s);
    ++s->n_failed;
}

void release_ctx(gld_server* s, Req* r)
{
    if (!r->ctx) return;
    r->ctx->st = s->A;  // its last work on S has finished; destroy waits on A only
    gld_destroy(r->ctx);
    r->ctx = nullptr;
    s->used -= r->bytes;
}

// Creates the context of a request on the admission stream.
gld_status admit(gld_server* s, Req* r)
{
    gld_params p = r->prm;
    p.stream = s->A;
    p.alloc = pool_alloc;
    p.free = pool_free;
    p.alloc_user = s;
    p.order = nullptr;
    p.use_graphs = 0;
    gld_ctx* c = nullptr;
    gld_status st = gld_create(&p, r->pos.data(), r->vel.data(), &c);
    if (st != GLD_OK) return st;
    st = gld_set_kernels(c, r->Ks.data(), r->Q, r->Q ? r->g.data() : nullptr, r->Q ? r->f.data() : nullptr, r->nr,
                         r->dr, r->Qs ? r->gs.data() : nullptr, r->Qs ? r->fs.data() : nullptr, r->Qs, r->conv);
    if (st == GLD_OK && r->pn_deg > 0) st = gld_set_pair_noise(c, r->pn_deg, nullptr, nullptr);
    if (st != GLD_OK) {
        r->msg = gld_last_error(c);
        gld_destroy(c);
        return st;
    }
    c->st = s->S;  // creation finished on A (the calls above synchronised it)
    r->ctx = c;
    r->bytes = c->bytes;
    s->used += r->bytes;
    s->peak = std::max(s->peak, s->used);
    std::vector<double>().swap(r->pos);  // inputs are on the device now
    std::vector<double>().swap(r->vel);
    return GLD_OK;
}

// Runs the tail steps (fewer than one block) alone, then queues the read-back
// of the results behind them on S.
gld_status retire(gld_server* s, Req* r)
{
    gld_ctx* c = r->ctx;
    if (r->left > 0) {
        const gld_status st = gld_step(c, r->left);
        if (st != GLD_OK) return st;
        s->psteps += r->left * (int64_t)c->P.n;
        r->left = 0;
    }
    const int L = c->P.vacf_len;
    const size_t n = (size_t)c->P.n;
    const size_t need = 64 + 16 * (size_t)std::max(L, 1) + (r->keep_state ? 32 * n : 0);
    if (!take_slab(s, need, r->slab)) return GLD_E_NOMEM;
    char* h = r->slab.p;
    cudaError_t e = launch_vacf_flush(c->P, c->B, s->S);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, &c->B.ctrl->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s->S);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + 8, c->B.norig, 8, cudaMemcpyDeviceToHost, s->S);
    if (e == cudaSuccess && L > 0) e = cudaMemcpyAsync(h + 64, c->B.csum, 8 * (size_t)L, cudaMemcpyDeviceToHost, s->S);
    if (e == cudaSuccess && L > 0)
        e = cudaMemcpyAsync(h + 64 + 8 * (size_t)L, c->B.ccnt, 8 * (size_t)L, cudaMemcpyDeviceToHost, s->S);
    const size_t off = 64 + 16 * (size_t)std::max(L, 1);
    if (e == cudaSuccess && r->keep_state) {
        e = cudaMemcpyAsync(h + off, c->B.pos, 16 * n, cudaMemcpyDeviceToHost, s->S);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h + off + 16 * n, c->B.vel, 16 * n, cudaMemcpyDeviceToHost, s->S);
    }
    if (e == cudaSuccess) {
        r->ev = take_event(s);
        e = r->ev ? cudaEventRecord(r->ev, s->S) : cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        r->msg = cudaGetErrorString(e);
        return GLD_E_CUDA;
    }
    r->state = kRetiring;
    return GLD_OK;
}

void finalize(gld_server* s, Req* r)
{
    gld_ctx* c = r->ctx;
    const char* h = r->slab.p;
    unsigned err = 0;
    std::memcpy(&err, h, sizeof(unsigned));
    const gld_status st = ctx_check_err(c, err);
    const int L = c->P.vacf_len;
    std::memcpy(&r->n_origins, h + 8, 8);
    r->vacf.assign((size_t)L, 0.0);
    for (int l = 0; l < L; ++l) {
        double sum;
        long long cnt;
        std::memcpy(&sum, h + 64 + 8 * (size_t)l, 8);
        std::memcpy(&cnt, h + 64 + 8 * (size_t)L + 8 * (size_t)l, 8);
        r->vacf[(size_t)l] = cnt > 0 ? sum / (3.0 * c->P.n * (double)cnt) : 0.0;
    }
    if (r->keep_state) {
        const size_t n = (size_t)c->P.n, off = 64 + 16 * (size_t)std::max(L, 1);
        r->out_pos.resize(3 * n);
        r->out_vel.resize(3 * n);
        ctx_to_caller(c, (const float4*)(h + off), r->out_pos.data());
        ctx_to_caller(c, (const float4*)(h + off + 16 * n), r->out_vel.data());
    }
    s->spare_slab.push_back(r->slab);
    r->slab = Slab{};
    s->spare_ev.push_back(r->ev);
    r->ev = nullptr;
    r->done = now_s(s);
    if (st != GLD_OK) {
        r->msg = c->msg;
        r->status = st;
        r->state = kFailed;
        ++s->n_failed;
    } else {
        r->state = kDone;
        ++s->n_done;
    }
    release_ctx(s, r);
}

void reap(gld_server* s)
{
    size_t keep = 0;
    for (Req* r : s->retiring) {
        if (cudaEventQuery(r->ev) == cudaSuccess) finalize(s, r);
        else s->retiring[keep++] = r;
    }
    s->retiring.resize(keep);
    keep = 0;
    for (Req* r : s->cancelling) {
        if (cudaEventQuery(r->ev) == cudaSuccess) {
            s->spare_ev.push_back(r->ev);
            r->ev = nullptr;
            release_ctx(s, r);
            fail_req(s, r, GLD_E_CANCELLED, "cancelled");
        } else {
            s->cancelling[keep++] = r;
        }
    }
    s->cancelling.resize(keep);
}

void drop_active(gld_server* s, Req* r, gld_status st, const std::string& m)
{
    if (r->ctx) {
        gld_batch_remove(s->batch, r->ctx);
        cudaStreamSynchronize(s->S);
        release_ctx(s, r);
    }
    fail_req(s, r, st, m);
}

}  // namespace

extern "C" {

void gld_server_params_default(gld_server_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->in_flight = 2;
    p->tuning = 1;
}

gld_status gld_server_create(const gld_server_params* sp, gld_server** out)
{
    if (!out) return GLD_E_INVAL;
    *out = nullptr;
    gld_server_params d;
    gld_server_params_default(&d);
    if (!sp) sp = &d;
    if (sp->hbm_budget < 0 || sp->max_members < 0 || sp->in_flight < 0 || sp->tuning < 0 || sp->tuning > 1)
        return GLD_E_INVAL;
    gld_server* s = new gld_server();
    s->sp = *sp;
    if (s->sp.in_flight == 0) s->sp.in_flight = 2;
    s->t0 = std::chrono::steady_clock::now();
    int dev = 0;
    bool ok = cudaGetDevice(&dev) == cudaSuccess;
    if (ok && sp->stream) {
        s->S = (cudaStream_t)sp->stream;
    } else if (ok) {
        ok = cudaStreamCreateWithFlags(&s->S, cudaStreamNonBlocking) == cudaSuccess;
        s->own_S = ok;
    }
    ok = ok && cudaStreamCreateWithFlags(&s->A, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        ok = cudaMemPoolCreate(&s->pool, &props) == cudaSuccess;
        if (ok) {
            uint64_t keep = ~0ull;  // freed memory stays in the pool
            cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    size_t free_b = 0, total_b = 0;
    ok = ok && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess;
    ok = ok && gld_batch_create(s->S, &s->batch) == GLD_OK;
    if (!ok) {
        gld_server_destroy(s);
        return GLD_E_CUDA;
    }
    gld_batch_set_tuning(s->batch, s->sp.tuning);
    s->budget = sp->hbm_budget > 0 ? (size_t)sp->hbm_budget : (size_t)(0.85 * (double)free_b);
    *out = s;
    return GLD_OK;
}

gld_status gld_server_submit(gld_server* s, const gld_request* q, int64_t* id)
{
    if (!s || !q) return GLD_E_INVAL;
    const gld_params& p = q->params;
    const int M = p.m_max;
    if (!q->pos || !q->vel || !q->Ks || q->steps < 0 || p.n < 1 || M < 2 || q->Q < 0 || q->Qs < 0 ||
        (q->Q > 0 && (!q->g || !q->f)) || (q->Qs > 0 && (!q->dKs_g || !q->dKs_f)) ||
        (q->Q + q->Qs > 0 && q->nr < 2) || q->pair_noise < 0 || q->pair_noise > kMaxPnDegree) {
        s->msg = "gld_server_submit: invalid request";
        return GLD_E_INVAL;
    }
    if (!s->queue.empty() && q->arrival < s->queue.back()->arrival) {
        s->msg = "gld_server_submit: arrivals must not decrease";
        return GLD_E_INVAL;
    }
    Req* r = new Req();
    r->id = (int64_t)s->reqs.size();
    r->prm = p;
    const size_t n3 = 3 * (size_t)p.n;
    r->pos.assign(q->pos, q->pos + n3);
    r->vel.assign(q->vel, q->vel + n3);
    r->Ks.assign(q->Ks, q->Ks + M);
    if (q->Q) {
        r->g.assign(q->g, q->g + (size_t)q->Q * M);
        r->f.assign(q->f, q->f + (size_t)q->Q * q->nr);
    }
    if (q->Qs) {
        r->gs.assign(q->dKs_g, q->dKs_g + (size_t)q->Qs * M);
        r->fs.assign(q->dKs_f, q->dKs_f + (size_t)q->Qs * q->nr);
    }
    r->Q = q->Q;
    r->Qs = q->Qs;
    r->nr = q->nr;
    r->dr = q->dr;
    r->conv = q->kernel_convention;
    r->keep_state = q->keep_state;
    r->pn_deg = q->pair_noise;
    r->steps = r->left = q->steps;
    r->arrival = q->arrival;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    r->bytes = ctx_bytes_needed(&p, q->Q, q->Qs, q->nr, sms) + pn_bytes_needed(&p, r->pn_deg);
    s->reqs.push_back(r);
    s->queue.push_back(r);
    if (id) *id = r->id;
    return GLD_OK;
}

gld_status gld_server_pump(gld_server* s, int32_t* active)
{
    if (!s) return GLD_E_INVAL;
    reap(s);
    const double now = now_s(s);
    // admission: arrived requests in order, while memory and slots allow
    while (!s->queue.empty() && s->queue.front()->arrival <= now) {
        Req* r = s->queue.front();
        if (r->bytes > s->budget) {
            s->queue.pop_front();
            fail_req(s, r, GLD_E_NOMEM, "request needs more device memory than the server's budget");
            continue;
        }
        if (s->sp.max_members > 0 && (int)s->active.size() >= s->sp.max_members) break;
        if (s->used + r->bytes > s->budget) break;
        s->queue.pop_front();
        gld_status st = admit(s, r);
        if (st != GLD_OK) {
            fail_req(s, r, st, r->msg.empty() ? "admission failed" : r->msg);
            continue;
        }
        r->admitted = now_s(s);
        r->state = kActive;
        if (r->left < kMaxNoiseBlock) {
            st = retire(s, r);
            if (st != GLD_OK) drop_active(s, r, st, "retire failed");
            else s->retiring.push_back(r);
            continue;
        }
        st = gld_batch_add(s->batch, r->ctx);
        if (st != GLD_OK) {
            drop_active(s, r, st, gld_batch_last_error(s->batch));
            continue;
        }
        s->active.push_back(r);
    }
    s->peak_members = std::max<int64_t>(s->peak_members, (int64_t)s->active.size());
    if (!s->active.empty()) {
        while ((int)s->inflight.size() >= s->sp.in_flight) {  // bounded run-ahead
            cudaEventSynchronize(s->inflight.front());
            s->spare_ev.push_back(s->inflight.front());
            s->inflight.pop_front();
        }
        gld_status st = gld_batch_step(s->batch, kMaxNoiseBlock);
        if (st != GLD_OK) {
            s->msg = gld_batch_last_error(s->batch);
            return st;
        }
        cudaEvent_t e = take_event(s);
        if (e && cudaEventRecord(e, s->S) == cudaSuccess) s->inflight.push_back(e);
        else if (e) s->spare_ev.push_back(e);
        ++s->blocks;
        size_t keep = 0;
        for (Req* r : s->active) {
            r->left -= kMaxNoiseBlock;
            s->psteps += (int64_t)kMaxNoiseBlock * r->prm.n;
            if (r->left >= kMaxNoiseBlock) {
                s->active[keep++] = r;
                continue;
            }
            gld_batch_remove(s->batch, r->ctx);
            st = retire(s, r);
            if (st != GLD_OK) drop_active(s, r, st, "retire failed");
            else s->retiring.push_back(r);
        }
        s->active.resize(keep);
    }
    if (active) *active = (int32_t)s->active.size();
    return GLD_OK;
}

gld_status gld_server_drain(gld_server* s, double timeout_s)
{
    if (!s) return GLD_E_INVAL;
    const double t_end = now_s(s) + (timeout_s > 0 ? timeout_s : 1e30);
    for (;;) {
        const gld_status st = gld_server_pump(s, nullptr);
        if (st != GLD_OK) return st;
        if (s->queue.empty() && s->active.empty() && s->retiring.empty() && s->cancelling.empty()) break;
        const double now = now_s(s);
        if (now > t_end) {
            s->msg = "gld_server_drain: timeout";
            return GLD_E_TIMEOUT;
        }
        if (s->active.empty()) {  // idle until the next arrival or result
            double wait = 5e-5;
            if (s->retiring.empty() && s->cancelling.empty() && !s->queue.empty())
                wait = std::min(1e-3, std::max(0.0, s->queue.front()->arrival - now));
            std::this_thread::sleep_for(std::chrono::duration<double>(wait));
        }
    }
    return GLD_OK;
}

gld_status gld_server_clock(const gld_server* s, double* t)
{
    if (!s || !t) return GLD_E_INVAL;
    *t = now_s(s);
    return GLD_OK;
}

gld_status gld_server_result(gld_server* s, int64_t id, double* vacf, int64_t* n_origins, double* pos, double* vel,
                             double* times)
{
    if (!s || id < 0 || id >= (int64_t)s->reqs.size()) return GLD_E_INVAL;
    const Req* r = s->reqs[(size_t)id];
    if (times) {
        times[0] = r->arrival;
        times[1] = r->admitted;
        times[2] = r->done;
    }
    if (r->state == kFailed) {
        s->msg = r->msg;
        return r->status;
    }
    if (r->state != kDone) return GLD_E_STATE;
    if (vacf) std::copy(r->vacf.begin(), r->vacf.end(), vacf);
    if (n_origins) *n_origins = r->n_origins;
    if (r->keep_state) {
        if (pos) std::copy(r->out_pos.begin(), r->out_pos.end(), pos);
        if (vel) std::copy(r->out_vel.begin(), r->out_vel.end(), vel);
    } else if (pos || vel) {
        s->msg = "gld_server_result: the request did not keep its state";
        return GLD_E_STATE;
    }
    return GLD_OK;
}

gld_status gld_server_cancel(gld_server* s, int64_t id)
{
    if (!s || id < 0 || id >= (int64_t)s->reqs.size()) return GLD_E_INVAL;
    Req* r = s->reqs[(size_t)id];
    if (r->state == kQueued) {
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
        fail_req(s, r, GLD_E_CANCELLED, "cancelled");
        return GLD_OK;
    }
    if (r->state != kActive) {
        s->msg = "gld_server_cancel: the request has finished or is being read back";
        return GLD_E_STATE;
    }
    s->active.erase(std::find(s->active.begin(), s->active.end(), r));
    gld_batch_remove(s->batch, r->ctx);
    r->ev = take_event(s);
    if (!r->ev || cudaEventRecord(r->ev, s->S) != cudaSuccess) {  // cannot track it: wait
        cudaStreamSynchronize(s->S);
        if (r->ev) s->spare_ev.push_back(r->ev);
        r->ev = nullptr;
        release_ctx(s, r);
        fail_req(s, r, GLD_E_CANCELLED, "cancelled");
        return GLD_OK;
    }
    r->state = kCancelling;
    s->cancelling.push_back(r);
    return GLD_OK;
}

gld_status gld_server_stats(gld_server* s, int64_t* out, int32_t count)
{
    if (!s || !out || count < 0) return GLD_E_INVAL;
    const int64_t v[GLD_SRV_N] = {(int64_t)s->queue.size(), (int64_t)s->active.size(), (int64_t)s->retiring.size(),
                                  s->n_done, s->n_failed, s->blocks, s->psteps, (int64_t)s->used,
                                  (int64_t)s->peak, s->peak_members, (int64_t)s->budget};
    for (int k = 0; k < count && k < GLD_SRV_N; ++k) out[k] = v[k];
    return GLD_OK;
}

const char* gld_server_last_error(const gld_server* s) { return s ? s->msg.c_str() : "null server"; }

gld_status gld_server_destroy(gld_server* s)
{
    if (!s) return GLD_E_INVAL;
    if (s->S) cudaStreamSynchronize(s->S);
    for (Req* r : s->reqs) {
        if (r->ctx) {
            if (s->batch) gld_batch_remove(s->batch, r->ctx);
            release_ctx(s, r);
        }
        if (r->slab.p) cudaFreeHost(r->slab.p);
        if (r->ev) cudaEventDestroy(r->ev);
        delete r;
    }
    if (s->batch) gld_batch_destroy(s->batch);
    for (cudaEvent_t e : s->inflight) cudaEventDestroy(e);
    for (cudaEvent_t e : s->spare_ev) cudaEventDestroy(e);
    for (Slab& b : s->spare_slab) cudaFreeHost(b.p);
    if (s->A) {
        cudaStreamSynchronize(s->A);
        cudaStreamDestroy(s->A);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (s->own_S && s->S) cudaStreamDestroy(s->S);
    delete s;
    return GLD_OK;
}

}  // extern "C"
