// Serving loop: continuous admission of LBP inference requests.
//
// Requests (a factor-graph description, log-potentials, evidence, T, damping,
// iterations) are queued in arrival order. A fixed number of in-flight slots, each a
// worker thread with its own CUDA stream, take requests from the head of the queue as
// soon as a slot is free and the request's device memory fits the budget: the worker
// compiles the graph, allocates and uploads everything stream-ordered (no device-wide
// synchronisation), runs the iterations, reads the normalised log-beliefs and the MAP
// decode back to host memory and frees its memory. Requests that arrive while others are
// on the GPU are therefore admitted as slots and memory free up, and the kernels of all
// in-flight requests overlap on the device; with one slot the loop is a plain FIFO that
// runs one request at a time. Each request's messages stay resident on the device for
// its lifetime. Latency = submission to results in host memory.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pgm.h"
#include "pgm_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// Deep copy of a pgm_graph_desc (the caller's arrays may be freed after submission).
struct DescCopy {
    std::vector<int32_t> num_states;
    std::vector<std::vector<int32_t>> e_cfg, e_vars, l_paroff, l_parents, l_child;
    std::vector<pgm_enum_group> eg;
    std::vector<pgm_logic_group> lg;
    pgm_graph_desc desc{};
    int64_t n_potentials = 0, n_var_states = 0;

    // Returns "" on success.
    std::string copy_from(const pgm_graph_desc *d) {
        if (!d || d->n_vars < 1 || !d->num_states) return "invalid description";
        if (d->n_enum_groups < 0 || d->n_logic_groups < 0) return "negative group count";
        if ((d->n_enum_groups > 0 && !d->enum_groups) || (d->n_logic_groups > 0 && !d->logic_groups))
            return "NULL group array";
        num_states.assign(d->num_states, d->num_states + d->n_vars);
        n_var_states = 0;
        for (int32_t k : num_states) n_var_states += k;
        for (int i = 0; i < d->n_enum_groups; ++i) {
            pgm_enum_group g = d->enum_groups[i];
            if (g.arity < 1 || g.n_cfg < 1 || g.n_fac < 0 || !g.cfg || (g.n_fac > 0 && !g.vars))
                return "invalid enumeration group";
            e_cfg.emplace_back(g.cfg, g.cfg + (int64_t)g.n_cfg * g.arity);
            e_vars.emplace_back(g.vars ? g.vars : g.cfg, g.vars ? g.vars + (int64_t)g.n_fac * g.arity : g.cfg);
            n_potentials += g.shared_potentials ? g.n_cfg : (int64_t)g.n_cfg * g.n_fac;
            eg.push_back(g);
        }
        for (int i = 0; i < d->n_logic_groups; ++i) {
            pgm_logic_group g = d->logic_groups[i];
            if (g.n_fac < 0 || !g.par_off || (g.n_fac > 0 && !g.child)) return "invalid logical group";
            l_paroff.emplace_back(g.par_off, g.par_off + g.n_fac + 1);
            const int64_t np = g.par_off[g.n_fac];
            if (np < 0 || (np > 0 && !g.parents)) return "invalid logical group";
            l_parents.emplace_back(g.parents ? g.parents : g.par_off, g.parents ? g.parents + np : g.par_off);
            l_child.emplace_back(g.child ? g.child : g.par_off, g.child ? g.child + g.n_fac : g.par_off);
            lg.push_back(g);
        }
        for (size_t i = 0; i < eg.size(); ++i) {
            eg[i].cfg = e_cfg[i].data();
            eg[i].vars = e_vars[i].data();
        }
        for (size_t i = 0; i < lg.size(); ++i) {
            lg[i].par_off = l_paroff[i].data();
            lg[i].parents = l_parents[i].data();
            lg[i].child = l_child[i].data();
        }
        desc.n_vars = d->n_vars;
        desc.num_states = num_states.data();
        desc.n_enum_groups = (int32_t)eg.size();
        desc.enum_groups = eg.data();
        desc.n_logic_groups = (int32_t)lg.size();
        desc.logic_groups = lg.data();
        return "";
    }
};

enum ReqState : int32_t { kPending = 1, kRunning = 2, kDone = 0 };

struct Request {
    int64_t id = 0;
    DescCopy d;
    std::vector<float> log_pot, evidence;
    float T = 1.f, damping = 0.f;
    int32_t n_iters = 0;        // iterations (the limit when check_every > 0)
    float tol = 0.f;            // early exit: residual tolerance
    // borrowed requests (pgm_serve_submit_borrowed): the caller's description and arrays
    const pgm_graph_desc *b_desc = nullptr;
    const float *b_lp = nullptr, *b_ev = nullptr;
    const pgm_graph_desc *desc() const { return b_desc ? b_desc : &d.desc; }
    const float *lp() const { return b_desc ? b_lp : log_pot.data(); }
    const float *ev() const { return b_desc ? b_ev : evidence.data(); }
    int32_t check_every = 0;    // early exit: residual checked every check_every iterations; 0 = off
    Clock::time_point t_submit, t_pop, t_compiled, t_admitted, t_done;
    int32_t state = kPending;
    pgm_status status = PGM_OK;
    std::string error;
    std::vector<float> beliefs;
    std::vector<int32_t> decode;
    int64_t updates = 0;
};

}  // namespace

struct pgm_server {
    pgm_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_mem;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<int64_t, std::shared_ptr<Request>> all;
    int64_t next_id = 1, bytes_in_use = 0, peak_bytes = 0;
    int64_t submitted = 0, completed = 0, failed = 0, updates_done = 0;
    int32_t in_flight = 0;
    // admission in arrival order: a worker takes the queue's head with a ticket, compiles
    // it (in parallel with the other workers), then waits until its ticket is the next to
    // be admitted and its memory fits
    int64_t next_ticket = 0, next_admit = 0;
    // seconds summed over completed requests: queue (submission to a worker), host
    // compile, admission wait, device work (build, upload, run, read-back)
    double sum_queue_s = 0.0, sum_compile_s = 0.0, sum_admit_s = 0.0, sum_run_s = 0.0;
    bool stop = false;
    Clock::time_point t_first_submit, t_last_done;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
};

namespace {

void finish(pgm_server *s, const std::shared_ptr<Request> &r, pgm_status st, const std::string &err, int64_t bytes) {
    std::lock_guard<std::mutex> lk(s->mu);
    r->t_done = Clock::now();
    r->status = st;
    r->error = err;
    r->state = kDone;
    if (bytes > 0) {
        s->bytes_in_use -= bytes;
        s->in_flight -= 1;
    }
    if (st == PGM_OK) {
        s->completed += 1;
        s->updates_done += r->updates;
        s->t_last_done = r->t_done;
        auto sec = [](Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); };
        s->sum_queue_s += sec(r->t_submit, r->t_pop);
        s->sum_compile_s += sec(r->t_pop, r->t_compiled);
        s->sum_admit_s += sec(r->t_compiled, r->t_admitted);
        s->sum_run_s += sec(r->t_admitted, r->t_done);
    } else {
        s->failed += 1;
    }
    s->cv_done.notify_all();
    s->cv_mem.notify_all();
    s->cv_work.notify_all();
}

// One request on one slot's stream, from its compiled layout. Returns the status; `err`
// gets the message.
pgm_status run_request(Request &r, const pgm::HostLayout &H, cudaStream_t st, std::string &err) {
    pgm_graph *g = nullptr;
    pgm_status rc = pgm::build_layout_on_stream(H, st, &g);
    if (rc != PGM_OK) {
        err = pgm_last_error();
        return rc;
    }
    pgm_info I{};
    pgm_graph_info(g, &I);
    r.updates = I.n_edge_states * (int64_t)r.n_iters;  // (early exit: iterations run)
    char *mem = nullptr;
    auto up = [](int64_t n) { return (size_t)((std::max<int64_t>(n, 1) * 4 + 255) / 256 * 256); };
    const size_t b_lp = up(I.n_potentials), b_vs = up(I.n_var_states), b_es = up(I.n_edge_states), b_v = up(I.n_vars);
    cudaError_t e = cudaMallocAsync(&mem, b_lp + 2 * b_vs + b_es + b_v, st);
    if (e != cudaSuccess) {
        pgm_free(g);
        err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
        return PGM_ENOMEM;
    }
    float *lp = reinterpret_cast<float *>(mem), *ev = reinterpret_cast<float *>(mem + b_lp);
    float *bel = reinterpret_cast<float *>(mem + b_lp + b_vs), *msgs = reinterpret_cast<float *>(mem + b_lp + 2 * b_vs);
    int32_t *dec = reinterpret_cast<int32_t *>(mem + b_lp + 2 * b_vs + b_es);
    if (I.n_potentials > 0)
        e = cudaMemcpyAsync(lp, r.lp(), I.n_potentials * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ev, r.ev(), I.n_var_states * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && I.n_edge_states > 0) e = cudaMemsetAsync(msgs, 0, I.n_edge_states * sizeof(float), st);
    rc = (e == cudaSuccess) ? PGM_OK : PGM_ECUDA;
    if (rc == PGM_OK && r.check_every > 0) {
        int32_t done = 0;
        float res = 0.f;
        rc = pgm_run_bp_until(g, lp, ev, r.T, r.damping, r.n_iters, r.tol, r.check_every, msgs, &done, &res, st);
        r.updates = I.n_edge_states * (int64_t)done;
    } else if (rc == PGM_OK) {
        rc = pgm_run_bp(g, lp, ev, r.T, r.damping, r.n_iters, msgs, st);
    }
    if (rc == PGM_OK) rc = pgm_beliefs(g, ev, msgs, bel, 1, st);
    if (rc == PGM_OK) rc = pgm_decode(g, ev, msgs, dec, st);
    if (rc == PGM_OK) {
        r.beliefs.resize(I.n_var_states);
        r.decode.resize(I.n_vars);
        e = cudaMemcpyAsync(r.beliefs.data(), bel, I.n_var_states * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r.decode.data(), dec, I.n_vars * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = PGM_ECUDA;
    }
    if (rc != PGM_OK && err.empty()) err = (e != cudaSuccess) ? cudaGetErrorString(e) : pgm_last_error();
    cudaFreeAsync(mem, st);
    pgm_free(g);  // stream-ordered
    return rc;
}

// Device bytes a request holds while in flight (graph + its input/output buffers, and
// with an early exit the residual buffers of pgm_run_bp_until).
int64_t request_bytes(const pgm::HostLayout &H, bool until) {
    return pgm::layout_device_bytes(H) + 4 * (H.P + 2 * H.VS + H.ES + H.V) + 2048 + (until ? 4 * H.ES + 512 : 0);
}

void worker_loop(pgm_server *s, int w) {
    cudaSetDevice(s->device);
    cudaStream_t st = s->streams[w];
    for (;;) {
        std::shared_ptr<Request> r;
        int64_t ticket = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
            if (s->pending.empty()) {
                if (s->stop) return;
                continue;
            }
            r = s->pending.front();
            s->pending.pop_front();
            ticket = s->next_ticket++;
        }
        r->t_pop = Clock::now();
        // compile once (the layout sizes the request and is built on the device below)
        pgm::HostLayout H;
        const void *one = r->desc();
        std::string err = pgm::compile_graph(&one, 1, &H);
        pgm_status rc = err.empty() ? PGM_OK : PGM_EINVAL;
        if (rc == PGM_OK && H.P > 0 && !r->lp()) {
            rc = PGM_EINVAL;
            err = "log_pot is NULL";
        }
        int64_t need = 0;
        if (rc == PGM_OK) {
            need = request_bytes(H, r->check_every > 0);
            if (need > s->cfg.memory_budget_bytes) {
                rc = PGM_ENOMEM;
                err = "request exceeds the server's memory budget";
            }
        }
        r->t_compiled = Clock::now();
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_mem.wait(lk, [&] {
                return s->stop ||
                       (ticket == s->next_admit && (rc != PGM_OK || s->bytes_in_use + need <= s->cfg.memory_budget_bytes));
            });
            if (ticket == s->next_admit) s->next_admit += 1;
            if (rc == PGM_OK) {
                s->bytes_in_use += need;
                s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_use);
                s->in_flight += 1;
                r->state = kRunning;
            }
            s->cv_mem.notify_all();  // the next ticket
        }
        r->t_admitted = Clock::now();
        if (rc != PGM_OK) {
            finish(s, r, rc, err, 0);
            continue;
        }
        rc = run_request(*r, H, st, err);
        finish(s, r, rc, err, need);
    }
}

}  // namespace

extern "C" {

pgm_status pgm_serve_create(const pgm_server_config *cfg, pgm_server **out) {
    if (!cfg || !out) return pgm::set_last_error(PGM_EINVAL, "NULL argument");
    if (cfg->max_in_flight < 1 || cfg->max_in_flight > 64)
        return pgm::set_last_error(PGM_EINVAL, "max_in_flight must be in 1..64");
    if (cfg->memory_budget_bytes <= 0) return pgm::set_last_error(PGM_EINVAL, "memory_budget_bytes must be > 0");
    if (cfg->max_pending < 1) return pgm::set_last_error(PGM_EINVAL, "max_pending must be >= 1");
    *out = nullptr;
    pgm_server *s = new (std::nothrow) pgm_server();
    if (!s) return pgm::set_last_error(PGM_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&s->device);
    for (int i = 0; i < cfg->max_in_flight && e == cudaSuccess; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->streams.push_back(st);
    }
    if (e != cudaSuccess) {
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        delete s;
        return pgm::set_last_error(PGM_ECUDA, std::string("pgm_serve_create: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < cfg->max_in_flight; ++i) s->workers.emplace_back(worker_loop, s, i);
    *out = s;
    return PGM_OK;
}

static pgm_status submit(pgm_server *s, const pgm_graph_desc *desc, const float *log_pot, const float *evidence,
                         float T, float damping, int32_t n_iters, float tol, int32_t check_every, bool borrowed,
                         int64_t *id) {
    if (!s || !id) return pgm::set_last_error(PGM_EINVAL, "NULL argument");
    if (!(T >= 0.f) || !std::isfinite(T)) return pgm::set_last_error(PGM_EINVAL, "T must be finite and >= 0");
    if (!(damping >= 0.f && damping < 1.f)) return pgm::set_last_error(PGM_EINVAL, "damping must be in [0, 1)");
    if (n_iters < 0 || !evidence) return pgm::set_last_error(PGM_EINVAL, "invalid n_iters or NULL evidence");
    auto r = std::make_shared<Request>();
    if (borrowed) {  // checked by the worker that admits it
        if (!desc) return pgm::set_last_error(PGM_EINVAL, "invalid description");
        r->b_desc = desc;
        r->b_lp = log_pot;
        r->b_ev = evidence;
    } else {
        std::string err = r->d.copy_from(desc);
        if (!err.empty()) return pgm::set_last_error(PGM_EINVAL, err);
        if (r->d.n_potentials > 0 && !log_pot) return pgm::set_last_error(PGM_EINVAL, "log_pot is NULL");
        r->log_pot.assign(log_pot ? log_pot : evidence, log_pot ? log_pot + r->d.n_potentials : evidence);
        r->evidence.assign(evidence, evidence + r->d.n_var_states);
    }
    r->T = T;
    r->damping = damping;
    r->n_iters = n_iters;
    r->tol = tol;
    r->check_every = check_every;
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int64_t)s->pending.size() >= s->cfg.max_pending)
        return pgm::set_last_error(PGM_EBUSY, "the pending queue is full");
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    if (s->submitted == 0) s->t_first_submit = r->t_submit;
    s->submitted += 1;
    s->pending.push_back(r);
    s->all[r->id] = r;
    *id = r->id;
    s->cv_work.notify_one();
    return PGM_OK;
}

pgm_status pgm_serve_submit(pgm_server *s, const pgm_graph_desc *desc, const float *log_pot,
                            const float *evidence, float T, float damping, int32_t n_iters, int64_t *id) {
    return submit(s, desc, log_pot, evidence, T, damping, n_iters, 0.f, 0, false, id);
}

pgm_status pgm_serve_submit_borrowed(pgm_server *s, const pgm_graph_desc *desc, const float *log_pot,
                                     const float *evidence, float T, float damping, int32_t max_iters, float tol,
                                     int32_t check_every, int64_t *id) {
    if (check_every < 0) return pgm::set_last_error(PGM_EINVAL, "check_every must be >= 0");
    if (check_every > 0 && !(tol >= 0.f)) return pgm::set_last_error(PGM_EINVAL, "tol must be >= 0");
    return submit(s, desc, log_pot, evidence, T, damping, max_iters, tol, check_every, true, id);
}

pgm_status pgm_serve_submit_until(pgm_server *s, const pgm_graph_desc *desc, const float *log_pot,
                                  const float *evidence, float T, float damping, int32_t max_iters, float tol,
                                  int32_t check_every, int64_t *id) {
    if (check_every < 1) return pgm::set_last_error(PGM_EINVAL, "check_every must be >= 1");
    if (!(tol >= 0.f)) return pgm::set_last_error(PGM_EINVAL, "tol must be >= 0");
    return submit(s, desc, log_pot, evidence, T, damping, max_iters, tol, check_every, false, id);
}

static pgm_status take_result(pgm_server *s, std::unordered_map<int64_t, std::shared_ptr<Request>>::iterator it,
                              float *beliefs, int32_t *decode, double *latency_s) {
    std::shared_ptr<Request> r = it->second;
    s->all.erase(it);
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    if (r->status != PGM_OK) return pgm::set_last_error(r->status, r->error);
    if (beliefs) std::memcpy(beliefs, r->beliefs.data(), r->beliefs.size() * sizeof(float));
    if (decode) std::memcpy(decode, r->decode.data(), r->decode.size() * sizeof(int32_t));
    return PGM_OK;
}

pgm_status pgm_serve_poll(pgm_server *s, int64_t id, float *beliefs, int32_t *decode, double *latency_s) {
    if (!s) return pgm::set_last_error(PGM_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return pgm::set_last_error(PGM_EINVAL, "unknown request id");
    if (it->second->state != kDone) return PGM_EBUSY;
    return take_result(s, it, beliefs, decode, latency_s);
}

pgm_status pgm_serve_wait(pgm_server *s, int64_t id, int64_t timeout_us, float *beliefs, int32_t *decode,
                          double *latency_s) {
    if (!s) return pgm::set_last_error(PGM_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return pgm::set_last_error(PGM_EINVAL, "unknown request id");
    std::shared_ptr<Request> r = it->second;
    if (!s->cv_done.wait_for(lk, std::chrono::microseconds(std::max<int64_t>(timeout_us, 0)),
                             [&] { return r->state == kDone; }))
        return pgm::set_last_error(PGM_ETIMEDOUT, "request not finished within the timeout");
    return take_result(s, s->all.find(id), beliefs, decode, latency_s);
}

pgm_status pgm_serve_stats(pgm_server *s, pgm_server_stats *out) {
    if (!s || !out) return pgm::set_last_error(PGM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->pending = (int64_t)s->pending.size();
    out->in_flight = s->in_flight;
    out->bytes_in_use = s->bytes_in_use;
    out->peak_bytes = s->peak_bytes;
    out->updates_done = s->updates_done;
    out->span_s = (s->completed > 0) ? std::chrono::duration<double>(s->t_last_done - s->t_first_submit).count() : 0.0;
    out->queue_s = s->sum_queue_s;
    out->compile_s = s->sum_compile_s;
    out->admit_s = s->sum_admit_s;
    out->run_s = s->sum_run_s;
    return PGM_OK;
}

void pgm_serve_destroy(pgm_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->pending.clear();
    }
    s->cv_work.notify_all();
    s->cv_mem.notify_all();
    for (std::thread &t : s->workers) t.join();
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
