// Serving loop: parareal solves of different sizes, flows and eps that arrive over time
// share one GPU (continuous batching).  Host code on top of the public C ABI.
//
// A request waits in a FIFO until its context's workspace fits the memory budget and the
// cap on resident requests; it is then admitted (workspace allocated, initial state
// copied, iteration 0 issued on its own stream) and stays resident until it finishes.
// Requests advance on their own iteration clocks, not in lock-step: each resident request
// has at most one iteration in flight on its stream, followed by an event.  A
// pr_server_step
//   1. admits waiting requests while memory and the resident cap allow;
//   2. finds the requests whose in-flight work has completed (event queries; if none has,
//      it polls for up to about a millisecond), runs their convergence checks, retires the
//      finished ones: U^k_N is copied to host memory and the workspace released, so the
//      next waiting requests are admitted in the same step;
//   3. issues the next iteration of every ready request: fine sweeps of ready requests
//      with the same n, box and precision share one persistent launch
//      (pr_fine_sweep_batch, up to FINE_MAX_JOBS requests per launch), then each request's
//      POD update and coarse sweep on its own stream, then its event.
// A small request therefore finishes while a large one is mid-solve, and its iterations
// never wait for another request's.  The CTA-group size of the fine launch is tuned once
// per (n, precision) by pr_tune_fine on the first request admitted with group_ctas = 0,
// and reused for every later request of that shape, so that batched and single launches
// tile a subinterval the same way (results are then identical alone and in the mix).
#include "../../include/parareal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

namespace {

constexpr int kMaxJobsPerLaunch = 16;   // FINE_MAX_JOBS of the fine kernel

struct Req {
    int id = 0;
    int state = PR_REQ_PENDING;
    pr_request r{};
    std::vector<double> u0, f, pert;   // host copies; r.flow.pert points into pert
    pr_ctx* ctx = nullptr;
    void* ws = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;      // recorded after the work in flight
    bool in_flight = false;        // iteration k + 1 (or iteration 0) issued, not checked
    int k = 0;
    int issued_k = 0;              // iteration in flight (k + 1) or last issued
    int k_max = 0;
    double inc = INFINITY;
    std::vector<double> result;
    std::string err;
};

// n, box length, precision, fine integrator, stored perturbation (one launch runs one
// stencil kind)
using ShapeKey = std::tuple<int, double, int, int, int>;

ShapeKey shape_of(const pr_request& r) {
    return ShapeKey(r.grid.n, r.grid.L, r.opts.precision, r.opts.fine, r.flow.pert ? 1 : 0);
}

}  // namespace

struct pr_server {
    pr_server_opts o{};
    size_t budget = 0;
    size_t used = 0;
    std::vector<std::unique_ptr<Req>> reqs;
    std::deque<int> pending;
    std::vector<int> active;
    std::map<ShapeKey, int> tuned;
    std::string err;
};

namespace {

pr_status server_fail(pr_server* s, pr_status st, const std::string& msg) {
    s->err = msg;
    return st;
}

// Release the request's device resources; keep its result and error text.
void release(pr_server* s, Req& q) {
    if (q.ctx) {
        pr_destroy(q.ctx);
        q.ctx = nullptr;
    }
    if (q.st) {
        cudaStreamSynchronize(q.st);
        cudaStreamDestroy(q.st);
        q.st = nullptr;
    }
    if (q.ev) {
        cudaEventDestroy(q.ev);
        q.ev = nullptr;
    }
    q.in_flight = false;
    if (q.ws) {
        cudaFree(q.ws);
        q.ws = nullptr;
        s->used -= q.bytes;
    }
    q.u0.clear();
    q.u0.shrink_to_fit();
    q.f.clear();
    q.f.shrink_to_fit();
}

void mark_failed(pr_server* s, Req& q, pr_status st, const char* where) {
    std::string m = where;
    if (q.ctx) {
        m += ": ";
        m += pr_last_error(q.ctx);
    }
    m += " (";
    m += pr_status_string(st);
    m += ")";
    q.err = m;
    q.state = PR_REQ_FAILED;
    release(s, q);
}

// Admit waiting requests in arrival order while memory and the resident cap allow.
void admit(pr_server* s) {
    while (!s->pending.empty()) {
        Req& q = *s->reqs[s->pending.front()];
        if (s->o.max_active > 0 && (int)s->active.size() >= s->o.max_active) return;
        if (!q.ctx) {
            pr_opts op = q.r.opts;
            auto it = s->tuned.find(shape_of(q.r));
            if (op.group_ctas <= 0 && it != s->tuned.end()) op.group_ctas = it->second;
            pr_status st = pr_create(&q.r.grid, &q.r.flow, q.r.eps, q.r.T, q.r.n_sub, q.r.dt_fine,
                                     q.r.pod_tol, &op, &q.ctx);
            if (st != PR_OK) {
                s->pending.pop_front();
                mark_failed(s, q, st, "pr_create");
                continue;
            }
            q.bytes = pr_workspace_bytes(q.ctx);
        }
        if (q.bytes > s->budget) {
            s->pending.pop_front();
            q.err = "workspace larger than the whole memory budget";
            q.state = PR_REQ_FAILED;
            release(s, q);
            continue;
        }
        if (s->used + q.bytes > s->budget) return;   // wait until others finish
        if (cudaMalloc(&q.ws, q.bytes) != cudaSuccess) {
            cudaGetLastError();
            q.ws = nullptr;
            return;                                  // memory held elsewhere: retry later
        }
        s->used += q.bytes;
        s->pending.pop_front();
        pr_status st = pr_bind_workspace(q.ctx, q.ws, q.bytes);
        if (st == PR_OK && cudaStreamCreateWithFlags(&q.st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            q.st = nullptr;
            st = PR_ERR_CUDA;
        }
        if (st == PR_OK && cudaEventCreateWithFlags(&q.ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            q.ev = nullptr;
            st = PR_ERR_CUDA;
        }
        if (st == PR_OK) st = pr_set_stream(q.ctx, q.st);
        if (st == PR_OK) st = pr_set_initial(q.ctx, q.u0.data(), q.f.empty() ? nullptr : q.f.data());
        if (st == PR_OK) st = pr_iteration0(q.ctx);
        if (st == PR_OK && q.r.opts.group_ctas <= 0 && !s->tuned.count(shape_of(q.r))) {
            int G = 0;
            st = pr_tune_fine(q.ctx, 8, &G, nullptr);
            if (st == PR_OK) s->tuned[shape_of(q.r)] = G;
        }
        if (st != PR_OK) {
            mark_failed(s, q, st, "admission");
            continue;
        }
        q.u0.clear();
        q.u0.shrink_to_fit();
        q.f.clear();
        q.f.shrink_to_fit();
        if (cudaEventRecord(q.ev, q.st) != cudaSuccess) {
            cudaGetLastError();
            mark_failed(s, q, PR_ERR_CUDA, "admission");
            continue;
        }
        q.state = PR_REQ_ACTIVE;
        q.k = 0;
        q.in_flight = true;   // iteration 0
        s->active.push_back(q.id);
    }
}

// Has the request's in-flight work completed?  (An event error fails the request.)
bool work_done(pr_server* s, Req& q) {
    const cudaError_t e = cudaEventQuery(q.ev);
    if (e == cudaErrorNotReady) return false;
    if (e != cudaSuccess) {
        cudaGetLastError();
        mark_failed(s, q, PR_ERR_CUDA, "event query");
    }
    return true;
}

// A request whose in-flight work completed: check the iteration it ran (none after
// iteration 0) and retire it if it is finished.  Returns true if it stays active.
bool settle(pr_server* s, Req& q) {
    q.in_flight = false;
    if (q.state != PR_REQ_ACTIVE) return false;
    if (q.issued_k > q.k) {
        double inc = 0.0, e = 0.0;
        pr_status st = pr_check(q.ctx, q.issued_k, &inc, &e);
        if (st != PR_OK) {
            mark_failed(s, q, st, "convergence check");
            return false;
        }
        q.k = q.issued_k;
        q.inc = inc;
        if (inc <= q.r.tol || q.k >= q.k_max) {
            const long long Ng = (long long)q.r.grid.n * q.r.grid.n * q.r.grid.n;
            q.result.resize((size_t)Ng);
            st = pr_get_interface(q.ctx, q.r.n_sub, q.result.data());
            if (st != PR_OK) {
                mark_failed(s, q, st, "result read-back");
                return false;
            }
            q.state = PR_REQ_DONE;
            release(s, q);
            return false;
        }
    }
    return true;
}

}  // namespace

extern "C" {

void pr_server_opts_init(pr_server_opts* o) {
    if (!o) return;
    o->hbm_budget = 0;
    o->max_active = 0;
    o->batch_fine = 1;
}

pr_status pr_server_create(const pr_server_opts* opts, pr_server** out) {
    if (!out) return PR_ERR_INVALID_ARG;
    *out = nullptr;
    auto s = std::make_unique<pr_server>();
    pr_server_opts_init(&s->o);
    if (opts) s->o = *opts;
    if (s->o.max_active < 0) return PR_ERR_INVALID_ARG;
    s->budget = s->o.hbm_budget;
    if (s->budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return PR_ERR_CUDA;
        }
        s->budget = fr / 10 * 9;
    }
    *out = s.release();
    return PR_OK;
}

void pr_server_destroy(pr_server* s) {
    if (!s) return;
    for (auto& q : s->reqs) release(s, *q);
    delete s;
}

pr_status pr_server_submit(pr_server* s, const pr_request* r, int* id) {
    if (!s || !r || !id || !r->u0) return PR_ERR_INVALID_ARG;
    if (r->grid.n < 4 || !(r->tol > 0)) return server_fail(s, PR_ERR_INVALID_ARG, "grid n >= 4 and tol > 0 needed");
    const long long Ng = (long long)r->grid.n * r->grid.n * r->grid.n;
    auto q = std::make_unique<Req>();
    q->id = (int)s->reqs.size();
    q->r = *r;
    q->u0.assign(r->u0, r->u0 + Ng);
    if (r->f) q->f.assign(r->f, r->f + Ng);
    if (r->flow.pert) {
        q->pert.assign(r->flow.pert, r->flow.pert + 3 * Ng);
        q->r.flow.pert = q->pert.data();
    }
    q->r.u0 = nullptr;
    q->r.f = nullptr;
    q->k_max = (r->k_max <= 0 || r->k_max > r->n_sub) ? r->n_sub : r->k_max;
    *id = q->id;
    s->pending.push_back(q->id);
    s->reqs.push_back(std::move(q));
    return PR_OK;
}

pr_status pr_server_step(pr_server* s, int* n_active, int* n_pending) {
    if (!s) return PR_ERR_INVALID_ARG;
    admit(s);
    // 1. requests whose in-flight work completed; wait (polling) until at least one has,
    //    for at most about a millisecond, so that the caller can submit new arrivals
    std::vector<Req*> ready;
    const auto t_start = std::chrono::steady_clock::now();
    for (int pass = 0;; ++pass) {
        bool any_active = false;
        for (int id : s->active) {
            Req* q = s->reqs[id].get();
            if (q->state != PR_REQ_ACTIVE) continue;
            any_active = true;
            if (q->in_flight && work_done(s, *q) && settle(s, *q)) ready.push_back(q);
            else if (!q->in_flight && q->state == PR_REQ_ACTIVE) ready.push_back(q);
        }
        if (!ready.empty() || !any_active) break;
        bool left = false;
        for (int id : s->active) left = left || s->reqs[id]->state == PR_REQ_ACTIVE;
        if (!left) break;   // every resident request finished in this pass
        if (std::chrono::steady_clock::now() - t_start > std::chrono::microseconds(1000)) break;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    // finished requests left: their memory lets waiting requests in now
    {
        std::vector<int> still;
        for (int id : s->active)
            if (s->reqs[id]->state == PR_REQ_ACTIVE) still.push_back(id);
        s->active.swap(still);
    }
    admit(s);
    // 2. the next iteration of every ready request: fine sweeps batched by shape
    std::map<ShapeKey, std::vector<Req*>> by_shape;
    for (Req* q : ready)
        if (q->state == PR_REQ_ACTIVE) by_shape[shape_of(q->r)].push_back(q);
    for (auto& kv : by_shape) {
        auto& v = kv.second;
        const size_t per = s->o.batch_fine ? kMaxJobsPerLaunch : 1;
        for (size_t i0 = 0; i0 < v.size(); i0 += per) {
            const size_t i1 = std::min(v.size(), i0 + per);
            std::vector<pr_ctx*> cs;
            std::vector<int> ks;
            for (size_t i = i0; i < i1; ++i) {
                cs.push_back(v[i]->ctx);
                ks.push_back(v[i]->k + 1);
            }
            pr_status st = pr_fine_sweep_batch(cs.data(), ks.data(), (int)cs.size());
            if (st != PR_OK)
                for (size_t i = i0; i < i1; ++i) mark_failed(s, *v[i], st, "fine sweep");
        }
    }
    // 3. POD update, coarse sweep and the completion event on each request's stream
    for (Req* q : ready) {
        if (q->state != PR_REQ_ACTIVE) continue;
        pr_status st = pr_pod_update(q->ctx, q->k + 1);
        if (st == PR_OK) st = pr_coarse_sweep(q->ctx, q->k + 1);
        if (st == PR_OK && cudaEventRecord(q->ev, q->st) != cudaSuccess) {
            cudaGetLastError();
            st = PR_ERR_CUDA;
        }
        if (st != PR_OK) {
            mark_failed(s, *q, st, "POD update / coarse sweep");
            continue;
        }
        q->issued_k = q->k + 1;
        q->in_flight = true;
    }
    {
        std::vector<int> still;
        for (int id : s->active)
            if (s->reqs[id]->state == PR_REQ_ACTIVE) still.push_back(id);
        s->active.swap(still);
    }
    if (n_active) *n_active = (int)s->active.size();
    if (n_pending) *n_pending = (int)s->pending.size();
    return PR_OK;
}

pr_status pr_server_query(pr_server* s, int id, int* state, int* k, double* max_inc) {
    if (!s || id < 0 || id >= (int)s->reqs.size()) return PR_ERR_INVALID_ARG;
    const Req& q = *s->reqs[id];
    if (state) *state = q.state;
    if (k) *k = q.k;
    if (max_inc) *max_inc = q.inc;
    return PR_OK;
}

pr_status pr_server_result(pr_server* s, int id, double* host_out) {
    if (!s || !host_out || id < 0 || id >= (int)s->reqs.size()) return PR_ERR_INVALID_ARG;
    const Req& q = *s->reqs[id];
    if (q.state == PR_REQ_FAILED) return server_fail(s, PR_ERR_STATE, "request failed: " + q.err);
    if (q.state != PR_REQ_DONE) return server_fail(s, PR_ERR_STATE, "request not finished");
    std::copy(q.result.begin(), q.result.end(), host_out);
    return PR_OK;
}

const char* pr_server_request_error(const pr_server* s, int id) {
    if (!s || id < 0 || id >= (int)s->reqs.size()) return "";
    return s->reqs[id]->err.c_str();
}

const char* pr_server_last_error(const pr_server* s) { return s ? s->err.c_str() : ""; }

}  // extern "C"
