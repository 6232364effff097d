// Serving engine behind lbm_server_* (include/lbm.h): melting runs arrive as
// requests, are admitted while slots and the HBM budget allow, advance
// together through one lbm_batch, and leave with their FP64
// diagnostics as soon as their step count is reached -- continuous batching:
// a request that arrives while others run joins them at the next tick.
// With batched = 0 the engine serves one request at a time in arrival order
// (the plain form, for comparison).  Host-only code on the public C ABI.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "lbm.h"

namespace {

using Clock = std::chrono::steady_clock;

// NVTX range for the lifetime of a scope (a no-op unless a profiler that
// records NVTX ranges is attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

struct Request {
    int64_t id = 0;
    lbm_params p{};
    int64_t steps = 0, remaining = 0, bytes = 0, nodes = 0;
    int64_t history_bytes = 0;   // the second exchange history of batch map 5
    double submit_s = 0.0, admit_s = 0.0;
    lbm_handle* h = nullptr;
};

}  // namespace

struct lbm_server {
    int64_t budget = 0, used = 0, peak_used = 0;
    int max_active = 1, batched = 1, quantum = 256, width_cap = 128, mapping = 4;
    int precision = LBM_F32, thermal_q = 5, flow = 1;
    cudaStream_t stream = nullptr;
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn release = nullptr;
    void* ctx = nullptr;
    std::deque<Request> queue;
    std::vector<Request> active;
    std::vector<lbm_request_result> done;
    lbm_batch* batch = nullptr;
    bool changed = true;
    int64_t next_id = 1;
    int64_t node_steps = 0;
    Clock::time_point t0;
    double busy_s = 0.0;
};

namespace {

double since(const lbm_server* s) {
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

void drop_batch(lbm_server* s) {
    if (s->batch) lbm_batch_destroy(s->batch);
    s->batch = nullptr;
    s->changed = true;
}

void finish(lbm_server* s, Request& r, int status) {
    lbm_request_result out;
    std::memset(&out, 0, sizeof out);
    out.id = r.id;
    out.steps = r.steps - r.remaining;
    out.nodes = r.nodes;
    out.submit_s = r.submit_s;
    out.admit_s = r.admit_s;
    double m = NAN, nu = NAN, e = NAN, ms = NAN;
    int rc = status;
    if (r.h) {
        const int d = lbm_diag(r.h, &m, &nu, &e, &ms);
        if (rc == LBM_OK) rc = d;
    }
    out.status = rc;
    out.melt_frac = m;
    out.nu_hot = nu;
    out.enthalpy = e;
    out.mass = ms;
    out.finish_s = since(s);
    if (r.h) lbm_destroy(r.h);
    r.h = nullptr;
    s->used -= r.bytes;
    s->done.push_back(out);
}

// Device bytes an active request holds: its state, and under batch map 5 the
// second exchange history that the two-step launches use.
int64_t charge(const lbm_server* s, const Request& r) {
    return r.bytes + (s->batched && s->mapping == 5 ? r.history_bytes : 0);
}

// Admission in arrival order, while a slot and the budget allow.  A request
// that the budget can never hold under the map in force (its second history
// counts only under map 5) is refused here.
void admit(lbm_server* s) {
    const Range range("admit");
    while (!s->queue.empty() && charge(s, s->queue.front()) > s->budget) {
        Request r = s->queue.front();
        s->queue.pop_front();
        r.admit_s = since(s);
        r.bytes = 0;
        finish(s, r, LBM_ERR_ARG);
    }
    while (!s->queue.empty() && (int)s->active.size() < s->max_active &&
           s->used + charge(s, s->queue.front()) <= s->budget) {
        Request r = s->queue.front();
        const int rc = lbm_create_ex(&r.p, s->stream, s->alloc, s->release, s->ctx, &r.h);
        if (rc == LBM_ERR_OOM && !s->active.empty()) break;   // wait for memory to come back
        s->queue.pop_front();
        r.bytes = charge(s, r);   // what this run holds while active
        r.admit_s = since(s);
        s->used += r.bytes;
        s->peak_used = std::max(s->peak_used, s->used);
        if (rc != LBM_OK) {
            r.h = nullptr;
            finish(s, r, rc);
            continue;
        }
        s->active.push_back(r);
        s->changed = true;
    }
}

}  // namespace

extern "C" {

int lbm_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t batched, int32_t quantum,
                      int32_t precision, int32_t thermal_q, int32_t flow, void* cuda_stream, lbm_alloc_fn alloc,
                      lbm_free_fn release, void* ctx, lbm_server** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || max_active < 1 || quantum < 1 || (batched != 0 && batched != 1) ||
        precision < LBM_F64 || precision > LBM_BF16 || (thermal_q != 5 && thermal_q != 9) ||
        (flow != 0 && flow != 1) || ((alloc == nullptr) != (release == nullptr)))
        return LBM_ERR_ARG;
    lbm_server* s = new (std::nothrow) lbm_server();
    if (!s) return LBM_ERR_OOM;
    s->budget = hbm_budget_bytes;
    s->batched = batched;
    s->max_active = batched ? max_active : 1;
    s->quantum = quantum;
    s->precision = precision;
    s->thermal_q = thermal_q;
    s->flow = flow;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->alloc = alloc;
    s->release = release;
    s->ctx = ctx;
    s->t0 = Clock::now();
    *out = s;
    return LBM_OK;
}

int lbm_server_configure(lbm_server* s, int32_t width_cap, int32_t mapping) {
    if (!s || (width_cap != 32 && width_cap != 64 && width_cap != 128 && width_cap != 256) || mapping < 0 ||
        mapping > 5 || (mapping == 5 && (s->precision == LBM_F64 || !s->flow)))
        return LBM_ERR_ARG;
    s->width_cap = width_cap;
    s->mapping = mapping;
    drop_batch(s);
    return LBM_OK;
}

int lbm_server_submit(lbm_server* s, const lbm_params* p, int64_t nsteps, int64_t* id) {
    if (!s || !p || nsteps < 1) return LBM_ERR_ARG;
    if (p->precision != s->precision || p->thermal_q != s->thermal_q || p->flow != s->flow) return LBM_ERR_ARG;
    const int64_t bytes = lbm_state_bytes(p);
    if (bytes < 0) {
        lbm_derived d;
        return lbm_derive(p, &d);   // the reason: malformed or unstable parameters
    }
    const int64_t history = lbm_history_bytes(p);
    Request r;
    r.id = s->next_id++;
    r.p = *p;
    r.steps = r.remaining = nsteps;
    r.bytes = bytes;
    r.history_bytes = history;
    if (charge(s, r) > s->budget) return LBM_ERR_ARG;   // could never be admitted
    r.nodes = (int64_t)p->nx * p->ny;
    r.submit_s = since(s);
    s->queue.push_back(r);
    if (id) *id = r.id;
    return LBM_OK;
}

int lbm_server_tick(lbm_server* s, int32_t* n_active, int32_t* n_queued, int32_t* n_done) {
    if (!s) return LBM_ERR_ARG;
    const Range tick_range("lbm_server_tick");
    admit(s);
    int rc = LBM_OK;
    if (!s->active.empty()) {
        const Range advance_range("advance");
        int64_t q = s->quantum;
        for (const Request& r : s->active) q = std::min(q, r.remaining);
        const auto t = Clock::now();
        if (s->batched) {
            if (s->changed || !s->batch) {
                drop_batch(s);
                std::vector<lbm_handle*> hs;
                for (const Request& r : s->active) hs.push_back(r.h);
                rc = lbm_batch_create(hs.data(), (int32_t)hs.size(), 0, s->stream, &s->batch);
                if (rc == LBM_OK) rc = lbm_batch_configure(s->batch, s->width_cap, s->mapping);
                s->changed = false;
            }
            if (rc == LBM_OK) rc = lbm_batch_step(s->batch, q);
        } else {
            rc = lbm_step(s->active.front().h, q);
        }
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
            cudaGetLastError();
            rc = LBM_ERR_CUDA;
        }
        s->busy_s += std::chrono::duration<double>(Clock::now() - t).count();
        for (Request& r : s->active) {
            r.remaining -= q;
            s->node_steps += q * r.nodes;
        }
        // retire finished runs (and every run if the step failed)
        bool any = false;
        for (const Request& r : s->active) any = any || r.remaining == 0 || rc != LBM_OK;
        if (any) {
            const Range retire_range("retire");
            drop_batch(s);
            std::vector<Request> keep;
            for (Request& r : s->active) {
                if (r.remaining == 0 || rc != LBM_OK) finish(s, r, rc);
                else keep.push_back(r);
            }
            s->active.swap(keep);
        }
    }
    if (n_active) *n_active = (int32_t)s->active.size();
    if (n_queued) *n_queued = (int32_t)s->queue.size();
    if (n_done) *n_done = (int32_t)s->done.size();
    return rc;
}

int lbm_server_results(lbm_server* s, lbm_request_result* out, int32_t max_results, int32_t* n) {
    if (!s || !n || (max_results > 0 && !out)) return LBM_ERR_ARG;
    const int k = std::min<int>(max_results, (int)s->done.size());
    for (int i = 0; i < k; ++i) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + k);
    *n = k;
    return LBM_OK;
}

int lbm_server_stats(const lbm_server* s, int64_t* node_steps, double* busy_s, double* elapsed_s, int64_t* used_bytes,
                     int64_t* peak_used_bytes) {
    if (!s) return LBM_ERR_ARG;
    if (node_steps) *node_steps = s->node_steps;
    if (busy_s) *busy_s = s->busy_s;
    if (elapsed_s) *elapsed_s = since(s);
    if (used_bytes) *used_bytes = s->used;
    if (peak_used_bytes) *peak_used_bytes = s->peak_used;
    return LBM_OK;
}

int lbm_server_destroy(lbm_server* s) {
    if (!s) return LBM_OK;
    drop_batch(s);
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (Request& r : s->active)
        if (r.h) lbm_destroy(r.h);
    cudaGetLastError();
    delete s;
    return LBM_OK;
}

}  // extern "C"
