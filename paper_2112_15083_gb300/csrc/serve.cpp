// Continuous-batching sampling server on top of the C-ABI (tn_server_*).
//
// Requests (circuit, open qubits, precision, target fidelity f, N, seed) are planned on
// planner threads (tn_plan + tn_select + tn_plan_estimate, each request on its own CUDA
// stream), admitted by a scheduler thread (shortest estimated job first, aged by waiting
// time) while the sum of admitted device-memory estimates stays within the HBM budget,
// and then advanced one batch group at a time:
// every active request always has one group in flight on its own stream, so the groups
// of different requests overlap on the device and a request that arrives while others
// run is admitted as soon as a slot and memory are free.  A request's samples depend only
// on its own inputs (deterministic plan, counter-based draws, fixed-order sums), so they
// are the same alone and in any mix.  Requests whose estimated GPU time exceeds the
// configured limit are rejected instead of blocking the queue.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "tn.h"
#include "serve_policy.h"

namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Req {
    int64_t id = 0;
    std::vector<unsigned char> circuit;
    std::vector<int32_t> open;
    int32_t precision = TN_PREC_C64, n_sliced = 0;
    double est_s = 0;  // estimated GPU seconds (admission order)
    double f = 1.0, alpha = 2.0;
    int64_t N = 0;
    uint64_t seed = 0;
    int32_t status = TN_REQ_QUEUED;
    int32_t error = TN_OK;
    std::string message;
    tn_circuit_h circ = nullptr;
    tn_plan_h plan = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<uint64_t> slices;
    double F = 0, flops_first = 0, flops_next = 0, flops_done = 0;
    int64_t est_bytes = 0;
    int64_t T = 0, t_next = 0, steps = 0, accepted = 0, max_steps = 0;
    int group = 0;
    bool inflight = false;
    uint8_t *d_acc = nullptr, *h_acc = nullptr;
    uint64_t *d_bits = nullptr, *h_bits = nullptr;
    std::vector<uint64_t> result;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct tn_server_s {
    tn_server_opts o{};
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_plan, cv_sched, cv_done;
    std::map<int64_t, std::shared_ptr<Req>> reqs;
    std::deque<std::shared_ptr<Req>> to_plan, planned;
    std::vector<std::shared_ptr<Req>> active;
    double bytes_in_use = 0;
    int64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> planners;
    std::thread sched;
};

namespace {

void release(Req &r) {
    if (r.stream) cudaStreamSynchronize(r.stream);
    if (r.d_acc) cudaFree(r.d_acc);
    if (r.d_bits) cudaFree(r.d_bits);
    if (r.h_acc) cudaFreeHost(r.h_acc);
    if (r.h_bits) cudaFreeHost(r.h_bits);
    r.d_acc = r.h_acc = nullptr;
    r.d_bits = r.h_bits = nullptr;
    if (r.plan) tn_plan_destroy(r.plan);
    if (r.circ) tn_circuit_destroy(r.circ);
    r.plan = nullptr;
    r.circ = nullptr;
    if (r.ev) cudaEventDestroy(r.ev);
    if (r.stream) cudaStreamDestroy(r.stream);
    r.ev = nullptr;
    r.stream = nullptr;
}

void fail(tn_server_s *s, Req &r, int code, int32_t status) {
    r.message = tn_last_error();
    release(r);
    std::lock_guard<std::mutex> lk(s->mu);
    r.error = code;
    r.status = status;
    r.t_done = now_s(s->t0);
    s->cv_done.notify_all();
}

// Assumed device rate of a request's precision (for the time estimates).
double rate_of(const tn_server_s *s, int32_t precision) {
    return precision == TN_PREC_C64 ? s->o.assumed_flops_c64 : s->o.assumed_flops;
}

void planner_loop(tn_server_s *s) {
    cudaSetDevice(s->o.device);
    for (;;) {
        std::shared_ptr<Req> r;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_plan.wait(lk, [&] { return s->stop || !s->to_plan.empty(); });
            if (s->stop) return;
            r = s->to_plan.front();
            s->to_plan.pop_front();
            r->status = TN_REQ_PLANNING;
        }
        int rc = TN_OK;
        if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess)
            rc = TN_EDEVICE;
        if (!rc) rc = tn_circuit_load(r->circuit.data(), r->circuit.size(), &r->circ);
        if (!rc) {
            tn_plan_opts po;
            tn_plan_opts_default(&po);
            po.precision = r->precision;
            // the smallest group holding the request's expected batches, within the bounds
            int lb = std::max(0, s->o.log2_batches);
            const double want = 1.1 * r->alpha * (double)r->N;
            while (lb < s->o.max_log2_batches && std::ldexp(1.0, lb) < want) lb++;
            po.log2_batches = lb;
            // the order search minimises the request's whole job: its expected groups
            po.job_groups = (int32_t)std::max(1.0, std::ceil(want / std::ldexp(1.0, lb)));
            po.autotune = 0;
            po.order_trials = s->o.order_trials;
            po.n_auto_sliced = r->n_sliced;
            po.hbm_budget_bytes = s->o.hbm_budget_bytes;
            po.stream = r->stream;
            po.max_norm_flops = s->o.max_request_seconds * rate_of(s, r->precision);
            rc = tn_plan(r->circ, nullptr, 0, nullptr, 0, r->open.data(), (int32_t)r->open.size(), &po, &r->plan);
        }
        int64_t n = 0;
        if (!rc) rc = tn_select(r->plan, r->f, nullptr, 0, &n, &r->F);
        if (!rc) {
            r->slices.resize((size_t)n);
            rc = tn_select(r->plan, r->f, r->slices.data(), n, &n, &r->F);
        }
        if (!rc) rc = tn_plan_estimate(r->plan, r->slices.data(), n, &r->est_bytes, &r->flops_first, &r->flops_next);
        if (rc == TN_EUNSUPPORTED) {  // e.g. a norm network over the time limit: a rejection
            fail(s, *r, rc, TN_REQ_REJECTED);
            continue;
        }
        if (rc) {
            fail(s, *r, rc, TN_REQ_FAILED);
            continue;
        }
        tn_plan_info info;
        tn_plan_get_info(r->plan, &info);
        r->T = 1LL << info.log2_batches;
        r->max_steps = (int64_t)std::ceil(8.0 * r->alpha * (double)r->N) + 4096;
        const double groups = std::ceil(1.1 * r->alpha * (double)r->N / (double)r->T);
        const double est_s =
            (r->flops_first + std::max(0.0, groups - 1) * r->flops_next) / rate_of(s, r->precision);
        r->est_s = est_s;
        if (est_s > s->o.max_request_seconds || (double)r->est_bytes > s->o.hbm_budget_bytes) {
            r->message = "rejected: estimated " + std::to_string(est_s) + " s / " + std::to_string(r->est_bytes) +
                         " bytes exceed the server limits";
            release(*r);
            std::lock_guard<std::mutex> lk(s->mu);
            r->error = TN_ENOMEM;
            r->status = TN_REQ_REJECTED;
            r->t_done = now_s(s->t0);
            s->cv_done.notify_all();
            continue;
        }
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {  // the server is shutting down: nobody will run it
            release(*r);
            r->status = TN_REQ_FAILED;
            s->cv_done.notify_all();
            continue;
        }
        r->status = TN_REQ_PLANNED;
        s->planned.push_back(r);
        s->cv_sched.notify_all();
    }
}

// Launch the next batch group of an active request on its stream.
int launch_group(Req &r) {
    int rc = tn_sample_step(r.plan, r.slices.data(), (int64_t)r.slices.size(), r.F, r.seed, (uint64_t)r.t_next,
                            r.alpha, r.group > 0, r.d_acc, r.d_bits, TN_DEVICE_BUFFERS);
    if (rc) return rc;
    if (cudaMemcpyAsync(r.h_acc, r.d_acc, r.T, cudaMemcpyDeviceToHost, r.stream) != cudaSuccess ||
        cudaMemcpyAsync(r.h_bits, r.d_bits, r.T * sizeof(uint64_t), cudaMemcpyDeviceToHost, r.stream) != cudaSuccess ||
        cudaEventRecord(r.ev, r.stream) != cudaSuccess)
        return TN_EDEVICE;
    r.inflight = true;
    r.group++;
    return TN_OK;
}

void sched_loop(tn_server_s *s) {
    cudaSetDevice(s->o.device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->active.empty())
                s->cv_sched.wait(lk, [&] { return s->stop || !s->planned.empty(); });
            if (s->stop && s->active.empty()) return;
            // admission (serve_policy.h): shortest estimated job first, aged by waiting
            // time, first fit within the budget and the slot count
            if (!s->planned.empty()) {
                const int n = (int)s->planned.size();
                std::vector<double> est(n), sub(n), bytes(n);
                for (int i = 0; i < n; i++) {
                    est[i] = s->planned[i]->est_s;
                    sub[i] = s->planned[i]->t_submit;
                    bytes[i] = (double)s->planned[i]->est_bytes;
                }
                std::vector<int> order(n), admit(n);
                tn_admission(n, est.data(), sub.data(), bytes.data(), now_s(s->t0), s->o.hbm_budget_bytes,
                             s->bytes_in_use, (int)s->active.size(), s->o.max_active, order.data(), admit.data());
                std::deque<std::shared_ptr<Req>> rest;
                for (int k = 0; k < n; k++) {
                    const int i = order[k];
                    auto &rp = s->planned[i];
                    if (admit[i]) {
                        s->bytes_in_use += (double)rp->est_bytes;
                        rp->status = TN_REQ_ACTIVE;
                        rp->t_admit = now_s(s->t0);
                        s->active.push_back(rp);
                    } else {
                        rest.push_back(rp);
                    }
                }
                s->planned.assign(rest.begin(), rest.end());
            }
        }
        bool idle = true;
        std::vector<std::shared_ptr<Req>> finished;
        for (auto &rp : s->active) {
            Req &r = *rp;
            if (!r.d_acc) {  // first time: buffers
                if (cudaMalloc(&r.d_acc, r.T) != cudaSuccess || cudaMalloc(&r.d_bits, r.T * sizeof(uint64_t)) != cudaSuccess ||
                    cudaMallocHost(&r.h_acc, r.T) != cudaSuccess ||
                    cudaMallocHost(&r.h_bits, r.T * sizeof(uint64_t)) != cudaSuccess) {
                    r.error = TN_ENOMEM;
                    finished.push_back(rp);
                    continue;
                }
            }
            if (r.inflight) {
                cudaError_t q = cudaEventQuery(r.ev);
                if (q == cudaErrorNotReady) continue;
                idle = false;
                r.inflight = false;
                if (q != cudaSuccess) {
                    r.error = TN_EDEVICE;
                    finished.push_back(rp);
                    continue;
                }
                const int64_t take = std::min<int64_t>(r.T, r.max_steps - r.steps);
                int64_t acc = 0;
                for (int64_t i = 0; i < take; i++)
                    if (r.h_acc[i]) {
                        acc++;
                        if ((int64_t)r.result.size() < r.N) r.result.push_back(r.h_bits[i]);
                    }
                {  // progress counters are read by tn_server_query under the lock
                    std::lock_guard<std::mutex> lk(s->mu);
                    r.accepted += acc;
                    r.steps += take;
                }
                r.t_next += r.T;
                if ((int64_t)r.result.size() >= r.N || r.steps >= r.max_steps) {
                    finished.push_back(rp);
                    continue;
                }
            }
            idle = false;
            const double fl = r.group == 0 ? r.flops_first : r.flops_next;
            int rc = launch_group(r);
            if (rc) {
                r.error = rc;
                finished.push_back(rp);
            } else {
                std::lock_guard<std::mutex> lk(s->mu);
                r.flops_done += fl;
            }
        }
        for (auto &rp : finished) {
            Req &r = *rp;
            int rc = r.error ? r.error : (r.plan ? tn_plan_sync(r.plan) : TN_OK);
            if (!rc && (int64_t)r.result.size() < r.N) rc = TN_EINVAL;  // step limit reached
            if (rc) r.message = tn_last_error();
            release(r);
            std::lock_guard<std::mutex> lk(s->mu);
            s->bytes_in_use -= (double)r.est_bytes;
            r.error = rc;
            r.status = rc ? TN_REQ_FAILED : TN_REQ_DONE;
            r.t_done = now_s(s->t0);
            s->active.erase(std::find(s->active.begin(), s->active.end(), rp));
            s->cv_done.notify_all();
        }
        if (idle && finished.empty()) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Called with the server's lock held.  The planner thread writes a request's plan fields
// without the lock and publishes them with its status change, so they are read only past
// planning; the scheduler updates the progress counters under the lock.
void fill_info(const Req &r, tn_request_info *info) {
    std::memset(info, 0, sizeof(*info));
    info->status = r.status;
    info->error = r.error;
    const bool planned = r.status != TN_REQ_QUEUED && r.status != TN_REQ_PLANNING;
    info->F = planned ? r.F : 0.0;
    info->steps = r.steps;
    info->accepted = r.accepted;
    info->n_slices = planned ? (int64_t)r.slices.size() : 0;
    info->est_bytes = planned ? r.est_bytes : 0;
    info->flops = r.flops_done;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
}

}  // namespace

extern "C" {

void tn_server_opts_default(tn_server_opts *o) {
    std::memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = 150e9;
    o->max_active = 8;
    o->planner_threads = 2;
    o->log2_batches = 8;
    o->max_log2_batches = 14;
    o->order_trials = 64;
    o->max_request_seconds = 600;
    o->assumed_flops = 3e14;
    o->assumed_flops_c64 = 3e13;
    o->device = 0;
}

int tn_server_create(const tn_server_opts *opts, tn_server_h *out) {
    if (!out) return TN_EINVAL;
    auto *s = new (std::nothrow) tn_server_s;
    if (!s) return TN_ENOMEM;
    if (opts) s->o = *opts;
    else tn_server_opts_default(&s->o);
    if (s->o.max_active < 1) s->o.max_active = 1;
    if (s->o.planner_threads < 1) s->o.planner_threads = 1;
    if (!(s->o.assumed_flops > 0)) s->o.assumed_flops = 3e14;
    if (!(s->o.assumed_flops_c64 > 0)) s->o.assumed_flops_c64 = 3e13;
    s->t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < s->o.planner_threads; i++) s->planners.emplace_back(planner_loop, s);
    s->sched = std::thread(sched_loop, s);
    *out = s;
    return TN_OK;
}

int tn_server_submit(tn_server_h s, const void *circuit, size_t len, const int32_t *open, int32_t n_open,
                     int32_t precision, int32_t n_sliced, double f, int64_t N, uint64_t seed, double alpha,
                     int64_t *id) {
    if (!s || !circuit || !len || !open || n_open <= 0 || N <= 0 || !(f > 0) || !(alpha > 1) || !id)
        return TN_EINVAL;
    auto r = std::make_shared<Req>();
    r->circuit.assign(static_cast<const unsigned char *>(circuit), static_cast<const unsigned char *>(circuit) + len);
    r->open.assign(open, open + n_open);
    r->precision = precision;
    r->n_sliced = n_sliced;
    r->f = f;
    r->N = N;
    r->seed = seed;
    r->alpha = alpha;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return TN_EINVAL;
    r->id = s->next_id++;
    r->t_submit = now_s(s->t0);
    s->reqs[r->id] = r;
    s->to_plan.push_back(r);
    s->cv_plan.notify_one();
    *id = r->id;
    return TN_OK;
}

int tn_server_query(tn_server_h s, int64_t id, tn_request_info *info) {
    if (!s || !info) return TN_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return TN_EINVAL;
    fill_info(*it->second, info);
    return TN_OK;
}

int tn_server_wait(tn_server_h s, int64_t id, double timeout_s, uint64_t *bitstrings, int64_t cap,
                   tn_request_info *info) {
    if (!s) return TN_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return TN_EINVAL;
    std::shared_ptr<Req> r = it->second;
    auto done = [&] { return r->status == TN_REQ_DONE || r->status == TN_REQ_FAILED || r->status == TN_REQ_REJECTED; };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) return TN_ETIMEOUT;
    } else {
        s->cv_done.wait(lk, done);
    }
    if (info) fill_info(*r, info);
    if (bitstrings && r->status == TN_REQ_DONE)
        std::copy(r->result.begin(), r->result.begin() + std::min<int64_t>(cap, (int64_t)r->result.size()), bitstrings);
    return r->status == TN_REQ_DONE ? TN_OK : (r->error ? r->error : TN_EINVAL);
}

int tn_server_get_stats(tn_server_h s, tn_server_stats *st) {
    if (!s || !st) return TN_EINVAL;
    std::memset(st, 0, sizeof(*st));
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &kv : s->reqs) {
        st->submitted++;
        switch (kv.second->status) {
            case TN_REQ_QUEUED: st->queued++; break;
            case TN_REQ_PLANNING: st->planning++; break;
            case TN_REQ_PLANNED: st->planned++; break;
            case TN_REQ_ACTIVE: st->active++; break;
            case TN_REQ_DONE: st->done++; break;
            case TN_REQ_FAILED: st->failed++; break;
            case TN_REQ_REJECTED: st->rejected++; break;
        }
    }
    st->bytes_in_use = s->bytes_in_use;
    st->time_s = now_s(s->t0);
    return TN_OK;
}

void tn_server_destroy(tn_server_h s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto &r : s->to_plan) r->status = TN_REQ_FAILED;
        for (auto &r : s->planned) {
            r->status = TN_REQ_FAILED;
            release(*r);
        }
        s->to_plan.clear();
        s->planned.clear();
        s->cv_plan.notify_all();
        s->cv_sched.notify_all();
        s->cv_done.notify_all();
    }
    for (auto &t : s->planners) t.join();
    s->sched.join();  // finishes the active requests
    delete s;
}

}  // extern "C"
