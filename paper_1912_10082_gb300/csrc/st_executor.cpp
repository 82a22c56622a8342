// Executor for many independent space-time solves on one GPU: the batched and
// served workloads of the library (no counterpart in the paper, which solves
// one problem at a time; each solve here is the paper's Section 4 method).
//
// Design.  `slots` worker threads each own a CUDA stream.  Problem handles
// live in a pool shared by the slots and keyed by geometry, so operators and
// fast-diagonalisation tables stay on the device between requests; a request
// takes an idle handle of its geometry (rebound to the slot's stream) and a
// new diffusion coefficient only re-runs the assembly kernel.  Handle memory
// comes from the stream-ordered pool, so no slot's allocation stalls another.  Requests wait in one queue and are
// admitted in arrival order (or, under the HRRN policy, highest response ratio
// first), skipping requests whose estimated device footprint does not fit the
// free part of the HBM budget (a request larger than the whole budget runs
// when nothing else does).  A slot takes
// the next admissible request as soon as its previous one finishes, so work
// of requests that arrived at different times overlaps on the device
// (continuous batching).  Each solve touches only its own handle, so a
// result does not depend on what else is running.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "st_common.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kExecutorUSlot = 31;   // workspace slot of a dense U staged for a request (ids below are the solver's)

struct Job {
    st_request req;
    int retries = 0;      // re-queued after running out of device memory next to other requests
    double t_submit = 0.0;
    double est = 0.0;     // admission estimate of device bytes
    double units = 0.0;   // n_h * n_t: the work measure of the service estimate
    int cls = 0;          // (operator, method, dimension) class of the learned rate
};

constexpr double kServiceOverhead = 2e-3;   // seconds of a request beyond its n_h * n_t work

int class_of(const st_request& r) { return (r.desc.op == ST_CONVDIFF ? 8 : 0) + (r.method == ST_METHOD_CN ? 4 : 0) + r.desc.dim; }

double prior_rate(int cls) {
    if (cls & 4) return 1e-9;
    return (cls & 8) ? 2e-8 : 3e-9;
}

struct GeomKey {
    int dim, n0, n1, n2, n_t, precision, maxit, max_basis;
    double l0, l1, l2, T, tol;
    bool operator==(const GeomKey& o) const { return std::memcmp(this, &o, sizeof(GeomKey)) == 0; }
};

GeomKey key_of(const st_desc& d) {
    GeomKey k;
    std::memset(&k, 0, sizeof(k));
    k.dim = d.dim;
    k.n0 = d.n[0];
    k.n1 = d.dim > 1 ? d.n[1] : 1;
    k.n2 = d.dim > 2 ? d.n[2] : 1;
    k.n_t = d.n_t;
    k.precision = d.precision;
    k.maxit = d.maxit;
    k.max_basis = d.max_basis;
    k.l0 = d.length[0];
    k.l1 = d.dim > 1 ? d.length[1] : 0.0;
    k.l2 = d.dim > 2 ? d.length[2] : 0.0;
    k.T = d.T;
    k.tol = d.tol;
    return k;
}

}  // namespace

struct PoolEntry {
    GeomKey key;
    st_problem* h = nullptr;
    bool busy = false;
    unsigned long long last_use = 0;
};

struct st_executor {
    int device = 0;
    std::vector<PoolEntry> pool;      // problem handles shared by all slots, keyed by geometry
    unsigned long long use_clock = 0;
    int nslots = 0;
    double budget = 0.0, used = 0.0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job> queue;
    std::deque<st_result> done;
    std::vector<std::thread> threads;
    bool stop = false;
    int running = 0;
    int policy = ST_SCHED_FIFO;
    double rate[16] = {};   // learned seconds per n_h * n_t unit, per class (0: not yet seen)
    Clock::time_point t0;
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

// Estimated device bytes of one solve: operators, fast-diagonalisation tables,
// a basis V and M V of k_est columns, the N_h-sized work blocks and Y.
extern "C" double st_request_bytes(const st_desc* d, int p) {
    if (!d || d->dim < 1 || d->dim > 3 || p < 1) return 0.0;
    double nh = 1.0, nnz = 1.0, tab = 0.0;
    for (int i = 0; i < d->dim; ++i) {
        nh *= d->n[i];
        nnz *= 3.0 * d->n[i] - 2.0;
        tab += 12.0 * d->n[i] * d->n[i] + 16.0 * d->n[i];
    }
    int maxit = d->maxit > 0 ? d->maxit : 400;
    int maxb = d->max_basis > 0 ? d->max_basis : 2048;
    // convection-diffusion needs more iterations (up to about 200 at eps = 0.01)
    const int it_est = d->op == ST_CONVDIFF ? 200 : 80;
    double k_est = std::min<double>(maxb + 16, (double)p * (std::min(maxit, it_est) + 1));
    double csr = nnz * (4.0 + 4 * 8.0 + 4 * 4.0) + 4.0 * (nh + 1);
    // V and M V (and the double-float V in mixed precision)
    double blocks = 8.0 * nh * ((d->precision == ST_MIXED ? 3.0 : 2.0) * k_est + 12.0 * p);
    double y = 8.0 * k_est * d->n_t;
    if (d->op == ST_CONVDIFF) {
        // flexible GMRES: 40-step Krylov and preconditioned blocks for up to 16 columns, within 4 GB
        double per_col = 8.0 * nh * 84.0;
        double mg = std::max(1.0, std::min({(double)p, 16.0, std::floor(4e9 / per_col)}));
        blocks += per_col * mg;
    }
    return csr + tab + blocks + y;
}

namespace {

double service_estimate(const st_executor* ex, const Job& j) {
    double r = ex->rate[j.cls] > 0 ? ex->rate[j.cls] : prior_rate(j.cls);
    return kServiceOverhead + r * j.units;
}

// The request to admit next (caller holds ex->mu).  FIFO: the first that fits
// the free budget.  HRRN: the request of highest (wait + service) / service;
// if it does not fit, nothing is admitted until memory frees up, so a large
// request is not starved by small ones that keep fitting.  With nothing
// running, the head (FIFO) or the top request (HRRN) runs whatever its size,
// so the queue cannot stall.
bool pick(st_executor* ex, size_t* idx) {
    if (ex->queue.empty()) return false;
    if (ex->policy != ST_SCHED_HRRN) {
        for (size_t i = 0; i < ex->queue.size(); ++i)
            if (ex->used + ex->queue[i].est <= ex->budget) {
                *idx = i;
                return true;
            }
        *idx = 0;
        return ex->running == 0;
    }
    const double now = ex->now();
    double best = -1.0;
    for (size_t i = 0; i < ex->queue.size(); ++i) {
        const Job& j = ex->queue[i];
        const double sv = service_estimate(ex, j);
        const double ratio = (now - j.t_submit + sv) / sv;
        if (ratio > best) {
            best = ratio;
            *idx = i;
        }
    }
    return ex->running == 0 || ex->used + ex->queue[*idx].est <= ex->budget;
}

// Take an idle pooled handle of this geometry (rebound to the slot's stream;
// the slot that used it last synchronised its stream when it finished), or
// build a new one.
st_problem* checkout(st_executor* ex, const GeomKey& key, const st_desc& d, cudaStream_t s, int* status) {
    *status = ST_OK;
    {
        std::lock_guard<std::mutex> lk(ex->mu);
        for (auto& e : ex->pool)
            if (!e.busy && e.key == key) {
                e.busy = true;
                e.h->stream = s;
                e.h->d.stream = s;
                return e.h;
            }
    }
    st_problem* h = nullptr;
    *status = st_setup(&d, &h);
    return *status == ST_OK ? h : nullptr;
}

// Return a handle to the pool.  Handles whose operators exceed 512 MB are not
// kept; beyond 4 handles per slot the least recently used idle one goes.
void checkin(st_executor* ex, const GeomKey& key, st_problem* h) {
    st_problem* drop = nullptr;
    {
        std::lock_guard<std::mutex> lk(ex->mu);
        bool found = false;
        for (auto& e : ex->pool)
            if (e.h == h) {
                e.busy = false;
                e.last_use = ++ex->use_clock;
                found = true;
            }
        if (!found) {
            if ((double)h->nnz * 52.0 > 512.0 * 1024 * 1024) {
                drop = h;
            } else {
                ex->pool.push_back(PoolEntry{key, h, false, ++ex->use_clock});
            }
        }
        if (!drop && ex->pool.size() > (size_t)4 * ex->nslots) {
            size_t victim = ex->pool.size();
            for (size_t i = 0; i < ex->pool.size(); ++i)
                if (!ex->pool[i].busy && (victim == ex->pool.size() || ex->pool[i].last_use < ex->pool[victim].last_use))
                    victim = i;
            if (victim < ex->pool.size()) {
                drop = ex->pool[victim].h;
                ex->pool.erase(ex->pool.begin() + (long)victim);
            }
        }
    }
    if (drop) st_destroy(drop);
}

int run_one(st_executor* ex, cudaStream_t s, const Job& job, st_result& res) {
    st_desc d = job.req.desc;
    d.stream = s;
    GeomKey key = key_of(d);
    int st0 = ST_OK;
    st_problem* h = checkout(ex, key, d, s, &st0);
    if (!h) return st0;
    struct Release {
        st_executor* ex;
        const GeomKey& key;
        st_problem* h;
        ~Release() {
            cudaStreamSynchronize(h->stream);   // nothing of this request in flight when another slot takes it
            checkin(ex, key, h);
        }
    } release{ex, key, h};
    ST_TRY(st_set_coefficients(h, d.op, d.kappa, d.eps, d.beta));
    st_solution sol{};
    double* Ud = nullptr;
    bool host_out = false;
    const bool cn = job.req.method == ST_METHOD_CN;
    if (!job.req.U_out && cn) {
        int st = st_slot(h, kExecutorUSlot, sizeof(double) * (size_t)h->n_h * h->n_t, (void**)&Ud);
        if (st != ST_OK) return st;
        sol.ldu = h->n_h;
    } else if (job.req.U_out) {
        if (st_is_device_ptr(job.req.U_out)) {
            Ud = job.req.U_out;
            sol.ldu = job.req.ldu;
        } else {
            host_out = true;
            int st = st_slot(h, kExecutorUSlot, sizeof(double) * (size_t)h->n_h * h->n_t, (void**)&Ud);
            if (st != ST_OK) return st;
            sol.ldu = h->n_h;
        }
        sol.U_dense = Ud;
    }
    int st;
    if (cn) {
        st = st_timestep_cn(h, job.req.F1, job.req.ldf1, job.req.F2, job.req.ldf2, job.req.p, Ud, sol.ldu);
        cudaError_t e = cudaStreamSynchronize(s);
        if (st == ST_OK && e != cudaSuccess) {
            st_note_cuda(e, "executor CN", __FILE__, __LINE__);
            st = ST_ECUDA;
        }
        res.k = 0;
    } else {
        st = st_solve(h, job.req.F1, job.req.ldf1, job.req.F2, job.req.ldf2, job.req.p, &sol, &res.stats);
        res.k = sol.k;
    }
    if (host_out && (st == ST_OK || st == ST_ENOTCONV)) {
        cudaError_t e = cudaMemcpy2DAsync(job.req.U_out, sizeof(double) * job.req.ldu, Ud, sizeof(double) * h->n_h,
                                          sizeof(double) * h->n_h, h->n_t, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st_note_cuda(e, "executor result copy", __FILE__, __LINE__);
            st = ST_ECUDA;
        }
    }
    return st;
}

void worker(st_executor* ex, int slot) {
    cudaSetDevice(ex->device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    while (true) {
        Job job;
        {
            std::unique_lock<std::mutex> lk(ex->mu);
            size_t idx = 0;
            ex->cv_work.wait(lk, [&] { return ex->stop || pick(ex, &idx); });
            if (ex->stop) break;
            job = ex->queue[idx];
            ex->queue.erase(ex->queue.begin() + (long)idx);
            ex->used += job.est;
            ex->running++;
        }
        st_result res{};
        res.tag = job.req.tag;
        res.slot = slot;
        res.bytes_reserved = job.est;
        res.t_submit = job.t_submit;
        res.t_start = ex->now();
        st_note_msg("");
        res.status = run_one(ex, s, job, res);
        res.t_end = ex->now();
        if (res.status != ST_OK) std::snprintf(res.message, sizeof(res.message), "%s", st_last_error());
        {
            std::lock_guard<std::mutex> lk(ex->mu);
            ex->used -= job.est;
            ex->running--;
            if (res.status == ST_ENOMEM && ex->running > 0 && job.retries < 2) {
                // the estimate fell short while others held memory: run it again, alone
                job.retries++;
                job.est = std::max(job.est, ex->budget);
                ex->queue.push_front(job);
                ex->cv_work.notify_all();
                continue;
            }
            if (res.status == ST_OK && job.units > 0) {
                // exponential average of the observed rate of this class
                double obs = std::max(0.0, res.t_end - res.t_start - kServiceOverhead) / job.units;
                double& r = ex->rate[job.cls];
                r = r > 0 ? 0.7 * r + 0.3 * obs : obs;
            }
            ex->done.push_back(res);
        }
        ex->cv_done.notify_all();
        ex->cv_work.notify_all();
    }
    if (s) cudaStreamDestroy(s);
}

}  // namespace

extern "C" int st_executor_create(int slots, double hbm_budget_bytes, st_executor** out) {
    if (!out) return ST_EINVAL;
    *out = nullptr;
    if (slots < 1 || slots > 256) return ST_EINVAL;
    st_executor* ex = new st_executor();
    if (cudaGetDevice(&ex->device) != cudaSuccess) {
        cudaGetLastError();
        delete ex;
        return ST_ECUDA;
    }
    if (hbm_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete ex;
            return ST_ECUDA;
        }
        hbm_budget_bytes = 0.8 * (double)fr;
    }
    ex->budget = hbm_budget_bytes;
    ex->nslots = slots;
    ex->t0 = Clock::now();
    for (int i = 0; i < slots; ++i) ex->threads.emplace_back(worker, ex, i);
    *out = ex;
    return ST_OK;
}

extern "C" double st_executor_now(st_executor* ex) { return ex ? ex->now() : 0.0; }

extern "C" int st_executor_submit(st_executor* ex, const st_request* req) {
    if (!ex || !req || !req->F1 || !req->F2 || req->p < 1 || req->p > 16) return ST_EINVAL;
    if (req->method != ST_METHOD_RKSM && req->method != ST_METHOD_CN) return ST_EINVAL;
    const st_desc& d = req->desc;
    if (d.dim < 1 || d.dim > 3 || d.n_t < 1 || !(d.T > 0)) return ST_EINVAL;
    Job job;
    job.req = *req;
    job.t_submit = ex->now();
    job.est = st_request_bytes(&d, req->p);
    // a dense U staged on the device: CN's output, or U = V Y bound for host memory
    double nh = 1.0;
    for (int i = 0; i < d.dim; ++i) nh *= d.n[i];
    job.units = nh * d.n_t;
    job.cls = class_of(*req);
    if (req->method == ST_METHOD_CN || (req->U_out && !st_is_device_ptr(req->U_out))) job.est += 8.0 * nh * d.n_t;
    {
        std::lock_guard<std::mutex> lk(ex->mu);
        if (ex->stop) return ST_EINVAL;
        ex->queue.push_back(job);
    }
    ex->cv_work.notify_one();
    return ST_OK;
}

extern "C" int st_executor_wait(st_executor* ex, st_result* out, int max, int* count, double timeout_s) {
    if (!ex || !count || max < 0) return ST_EINVAL;
    *count = 0;
    std::unique_lock<std::mutex> lk(ex->mu);
    auto ready = [&] { return !ex->done.empty(); };
    if (timeout_s > 0)
        ex->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
    int n = 0;
    while (n < max && !ex->done.empty()) {
        if (out) out[n] = ex->done.front();
        ex->done.pop_front();
        ++n;
    }
    *count = n;
    return ST_OK;
}

extern "C" int st_executor_set_policy(st_executor* ex, int policy) {
    if (!ex || (policy != ST_SCHED_FIFO && policy != ST_SCHED_HRRN)) return ST_EINVAL;
    {
        std::lock_guard<std::mutex> lk(ex->mu);
        ex->policy = policy;
    }
    ex->cv_work.notify_all();
    return ST_OK;
}

extern "C" int st_executor_pending(st_executor* ex, int* queued, int* running) {
    if (!ex) return ST_EINVAL;
    std::lock_guard<std::mutex> lk(ex->mu);
    if (queued) *queued = (int)ex->queue.size();
    if (running) *running = ex->running;
    return ST_OK;
}

extern "C" int st_executor_destroy(st_executor* ex) {
    if (!ex) return ST_OK;
    {
        std::lock_guard<std::mutex> lk(ex->mu);
        ex->stop = true;
        ex->queue.clear();
    }
    ex->cv_work.notify_all();
    for (auto& t : ex->threads) t.join();
    // the slots' streams are gone with their workers: release the pooled
    // handles on the default stream
    for (auto& e : ex->pool) {
        e.h->stream = nullptr;
        e.h->d.stream = nullptr;
        st_destroy(e.h);
    }
    delete ex;
    return ST_OK;
}
