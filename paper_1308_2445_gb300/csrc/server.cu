// Request loop of the served form: solves of different problems, sizes and nev arrive over
// time (SCF steps and k-points of several runs); each is admitted when a slot and its device-
// memory estimate fit, runs on its own stream next to the others (their kernels overlap on the
// GPU), and its result is collected by ticket.  Sessions (matrix, factor and last block) stay
// resident, so a follow-up request -- new H values on the same pattern, warm-started from the
// previous block, Sec. 3 -- reuses the factorisation of its session's first H (reading R2).
//
// Host code only: worker threads, a queue scanned in arrival order (a request that cannot run
// yet -- session busy, or memory -- does not hold back later ones), least-recently-used
// eviction of idle sessions when memory is short.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.h"

namespace hbsd {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    bool is_new = false;
    // new problem (copied at submission)
    int64_t n = 0, nnz = 0;
    int is_complex = 0;              // values are (re, im) pairs; the session solves the 2n real pencil
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col_idx, dof_node, dof_cluster;
    std::vector<double> hval, sval;
    int32_t grid[3] = {0, 0, 0};
    hbsd_options opt{};
    int nl_k = 0;                    // nonlocal term F (n x nl_k, row-major) and G
    std::vector<double> nl_F, nl_G;
    // follow-up
    int64_t session_id = -1;
    std::vector<double> hval_new;
    int warm = 0;
    // solve
    int nev = 0;
    double tol = 0.0;
    std::vector<double> X0;
    double* lam_out = nullptr;
    double* X_out = nullptr;
    size_t est_raw = 0;      // footprint estimate from n, nnz, nev (new problem)
    size_t est_bytes = 0;    // what admission reserved: est_raw times the server's calibration
    Clock::time_point t_submit;
};

struct ResultRec {
    bool done = false;
    hbsd_result r{};
};

struct SessionRec {
    hbsd_handle* h = nullptr;
    cudaStream_t stream = nullptr;
    bool busy = false;
    size_t bytes = 0;
    Clock::time_point last_use;
};

size_t estimate_bytes(int64_t n, int64_t nnz, int nev, int nl_k) {
    // matrix: ~1.2 nnz stored SELL entries x (index, FP64 pair, FP32 pair, double-float pair);
    // factor: 24 bytes per entry (FP64 panels and their explicit inverses, two FP32 copies), its
    // fill nnz(L)/nnz measured at 16.5 on the 32^3 workload (n = 47,620) and growing as n^0.35
    // (39 at 64^3), plus a quarter for the factorisation's fronts; ~20 blocks of n x (nev + m0)
    // doubles (the solve's blocks, MINRES vectors, FP32 and double-float copies, start block and
    // warm-start copy); with a nonlocal term the dense Fhat (FP64 + FP32) and its setup block.
    // The server scales this by the largest measured footprint / estimate seen so far.
    const int64_t w = nev + std::max(3, (nev + 9) / 10);
    const double fill = 16.5 * std::pow((double)std::max<int64_t>(n, 1000) / 47620.0, 0.35);
    return (size_t)(56.0 * (double)nnz + 30.0 * fill * (double)nnz + 160.0 * (double)n * (double)w +
                    20.0 * (double)n * (double)nl_k + (double)(64 << 20));
}

}  // namespace
}  // namespace hbsd

struct hbsd_server {
    hbsd_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::unique_ptr<hbsd::Request>> queue;
    std::unordered_map<uint64_t, hbsd::ResultRec> results;
    std::unordered_map<int64_t, hbsd::SessionRec> sessions;
    std::vector<std::thread> workers;
    size_t used = 0;   // device bytes of resident sessions (measured) and running requests (reserved)
    double est_scale = 1.25;  // largest measured peak footprint / estimate so far (only grows)
    uint64_t next_ticket = 1;
    int64_t next_session = 0;
    int running = 0;
    bool stop = false;
    std::vector<hbsd::SessionRec> graveyard;   // evicted sessions, destroyed outside the lock
};

namespace hbsd {
namespace {

// Evict idle sessions, least recently used first, until `need` more bytes fit.  mu held.
void evict_for(hbsd_server* sv, size_t need) {
    while (sv->used + need > sv->opts.hbm_budget_bytes) {
        int64_t victim = -1;
        Clock::time_point oldest = Clock::time_point::max();
        for (auto& kv : sv->sessions)
            if (!kv.second.busy && kv.second.last_use < oldest) {
                oldest = kv.second.last_use;
                victim = kv.first;
            }
        if (victim < 0) return;
        SessionRec rec = sv->sessions[victim];
        sv->sessions.erase(victim);
        sv->used -= std::min(sv->used, rec.bytes);
        sv->graveyard.push_back(rec);
    }
}

// Destroys the evicted sessions (device frees synchronise the device: never under mu).
void bury(hbsd_server* sv) {
    std::vector<SessionRec> dead;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        dead.swap(sv->graveyard);
    }
    for (auto& rec : dead) {
        hbsd_destroy(rec.h);
        if (rec.stream) cudaStreamDestroy(rec.stream);
    }
}

// Evicts every idle session and destroys the evicted ones now (a request that met a device
// out-of-memory error retries after this).  mu not held.
void free_idle(hbsd_server* sv) {
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        evict_for(sv, sv->opts.hbm_budget_bytes + 1);   // as much as possible: every idle session
    }
    bury(sv);
}

// Next runnable request in arrival order, or null.  mu held.
std::unique_ptr<Request> take_runnable(hbsd_server* sv) {
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
        Request& r = **it;
        if (!r.is_new) {
            auto s = sv->sessions.find(r.session_id);
            if (s == sv->sessions.end()) {   // unknown or evicted session: fail the request
                std::unique_ptr<Request> out = std::move(*it);
                sv->queue.erase(it);
                return out;
            }
            if (s->second.busy) continue;
        }
        const size_t need = r.is_new ? (size_t)((double)r.est_raw * sv->est_scale) : 0;
        if (sv->used + need > sv->opts.hbm_budget_bytes) {
            evict_for(sv, need);
            if (sv->used + need > sv->opts.hbm_budget_bytes && sv->running > 0) continue;   // wait for memory
        }
        std::unique_ptr<Request> out = std::move(*it);
        sv->queue.erase(it);
        return out;
    }
    return nullptr;
}

void run_request(hbsd_server* sv, Request& rq) {
    const Clock::time_point t_start = Clock::now();
    const int64_t dev0 = tl_dev_bytes();   // this thread's device bytes before the request
    tl_dev_peak() = dev0;
    hbsd_result res{};
    res.ticket = rq.ticket;
    int64_t sid = rq.session_id;
    hbsd_handle* h = nullptr;
    int rc = HBSD_OK;
    if (rq.is_new) {
        cudaStream_t stream = nullptr;
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
            rc = fail(HBSD_ERR_CUDA, "server: cudaStreamCreateWithFlags failed");
        } else {
            hbsd_csr H{rq.n, rq.nnz, rq.row_ptr.data(), rq.col_idx.data(), rq.hval.data(), rq.is_complex};
            hbsd_csr S{rq.n, rq.nnz, rq.row_ptr.data(), rq.col_idx.data(), rq.sval.data(), rq.is_complex};
            hbsd_local_blocks lb{};
            lb.dof_node = rq.dof_node.data();
            lb.dof_cluster = rq.dof_cluster.empty() ? nullptr : rq.dof_cluster.data();
            std::memcpy(lb.grid, rq.grid, sizeof(lb.grid));
            rc = hbsd_create(&H, &S, &lb, &rq.opt, stream, &h);
            if (rc == HBSD_ERR_OOM) {   // the device ran short despite admission: free every idle session, retry once
                free_idle(sv);
                rc = hbsd_create(&H, &S, &lb, &rq.opt, stream, &h);
            }
            if (rc >= 0 && rq.nl_k > 0) {
                rc = hbsd_set_nonlocal(h, rq.nl_k, rq.nl_F.data(), rq.nl_k, rq.nl_G.data());
                if (rc < 0) {
                    hbsd_destroy(h);
                    h = nullptr;
                }
            }
            std::lock_guard<std::mutex> lk(sv->mu);
            if (rc < 0) {
                cudaStreamDestroy(stream);
                sv->used -= std::min(sv->used, rq.est_bytes);
                rq.est_bytes = 0;
            } else {
                sid = sv->next_session++;
                SessionRec rec;
                rec.h = h;
                rec.stream = stream;
                rec.busy = true;
                rec.bytes = 0;   // set from the measured footprint when the request ends
                rec.last_use = Clock::now();
                sv->sessions[sid] = rec;
            }
        }
    } else {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto s = sv->sessions.find(sid);
        if (s == sv->sessions.end()) rc = fail(HBSD_ERR_ARG, "server: unknown or evicted session");
        else h = s->second.h;
    }
    if (rc >= 0 && !rq.hval_new.empty()) rc = hbsd_update_H(h, rq.hval_new.data());
    if (rc >= 0) {
        int iters = 0;
        hbsd_stats st{};
        rc = hbsd_solve(h, rq.nev, rq.tol, rq.X0.empty() ? nullptr : rq.X0.data(), rq.warm, rq.lam_out, rq.X_out,
                        &iters, &st);
        if (rc == HBSD_ERR_OOM) {
            free_idle(sv);
            rc = hbsd_solve(h, rq.nev, rq.tol, rq.X0.empty() ? nullptr : rq.X0.data(), rq.warm, rq.lam_out, rq.X_out,
                            &iters, &st);
        }
        res.iters = iters;
        res.res_max = st.res_max;
    }
    const Clock::time_point t_end = Clock::now();
    // the session's footprint: what this request left allocated (all of a new session: its
    // matrix, factor and solve buffers; a follow-up's growth), replacing the reservation
    const int64_t grown = std::max<int64_t>(0, tl_dev_bytes() - dev0);
    const int64_t peak = std::max<int64_t>(grown, tl_dev_peak() - dev0);   // with the factorisation's fronts
    res.status = rc;
    res.session_id = rc >= 0 || !rq.is_new ? sid : -1;
    res.queue_ms = std::chrono::duration<double, std::milli>(t_start - rq.t_submit).count();
    res.run_ms = std::chrono::duration<double, std::milli>(t_end - t_start).count();
    res.latency_ms = std::chrono::duration<double, std::milli>(t_end - rq.t_submit).count();
    std::lock_guard<std::mutex> lk(sv->mu);
    auto s = sv->sessions.find(sid);
    if (s != sv->sessions.end()) {
        s->second.busy = false;
        s->second.last_use = Clock::now();
        if (rq.is_new) {
            sv->used -= std::min(sv->used, rq.est_bytes);
            s->second.bytes = (size_t)grown;
            if (rq.est_raw > 0) sv->est_scale = std::max(sv->est_scale, (double)peak / (double)rq.est_raw);
        } else {
            s->second.bytes += (size_t)grown;
        }
        sv->used += (size_t)grown;
    }
    ResultRec& rr = sv->results[rq.ticket];
    rr.r = res;
    rr.done = true;
}

void worker(hbsd_server* sv) {
    for (;;) {
        std::unique_ptr<Request> rq;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stop) return;
                rq = take_runnable(sv);
                if (rq) break;
                sv->cv.wait(lk);
            }
            if (!rq->is_new) {
                auto s = sv->sessions.find(rq->session_id);
                if (s != sv->sessions.end()) s->second.busy = true;
            } else {
                rq->est_bytes = (size_t)((double)rq->est_raw * sv->est_scale);
                sv->used += rq->est_bytes;
            }
            ++sv->running;
        }
        bury(sv);
        const int rc = guarded([&]() -> int {
            run_request(sv, *rq);
            return HBSD_OK;
        });
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            --sv->running;
            if (rc < 0) {   // a host exception before the result was recorded: record the failure
                auto s = sv->sessions.find(rq->session_id);
                if (s != sv->sessions.end()) s->second.busy = false;
                auto it = sv->results.find(rq->ticket);
                if (it != sv->results.end() && !it->second.done) {
                    it->second.r = hbsd_result{};
                    it->second.r.ticket = rq->ticket;
                    it->second.r.status = rc;
                    it->second.r.session_id = -1;
                    it->second.done = true;
                }
            }
        }
        sv->cv.notify_all();
    }
}

}  // namespace
}  // namespace hbsd

using namespace hbsd;

extern "C" {

void hbsd_server_opts_default(hbsd_server_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = 0;
    o->max_slots = 4;
}

int hbsd_server_create(const hbsd_server_opts* opts, hbsd_server** out) {
    return guarded([&]() -> int {
        if (!out) return fail(HBSD_ERR_ARG, "out is NULL");
        *out = nullptr;
        hbsd_server_opts o;
        hbsd_server_opts_default(&o);
        if (opts) o = *opts;
        if (o.max_slots < 1 || o.max_slots > 64) return fail(HBSD_ERR_ARG, "max_slots must lie in [1, 64]");
        if (o.hbm_budget_bytes == 0) {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(HBSD_ERR_CUDA, "cudaMemGetInfo failed");
            o.hbm_budget_bytes = fr / 10 * 8;
        }
        hbsd_server* sv = new hbsd_server();
        sv->opts = o;
        try {
            for (int i = 0; i < o.max_slots; ++i) sv->workers.emplace_back(worker, sv);
        } catch (...) {   // a thread could not start: stop and join the ones that did
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->stop = true;
            }
            sv->cv.notify_all();
            for (auto& t : sv->workers) t.join();
            delete sv;
            throw;
        }
        *out = sv;
        return HBSD_OK;
    });
}

int hbsd_submit(hbsd_server* sv, const hbsd_request* rq, double* lambda_out, double* X_out, uint64_t* ticket) {
    return guarded([&]() -> int {
        if (!sv || !rq || !lambda_out || !ticket) return fail(HBSD_ERR_ARG, "NULL argument");
        if (rq->nev < 1 || !(rq->tol > 0)) return fail(HBSD_ERR_ARG, "nev >= 1 and tol > 0 required");
        auto r = std::make_unique<Request>();
        r->nev = rq->nev;
        r->tol = rq->tol;
        r->lam_out = lambda_out;
        r->X_out = X_out;
        r->warm = rq->warm;
        int64_t n = 0;
        if (rq->session_id < 0) {   // new problem: H, S, local blocks and options copied here
            if (!rq->H || !rq->S || !rq->lb || !rq->opt) return fail(HBSD_ERR_ARG, "a new problem needs H, S, lb, opt");
            if (rq->H->n <= 0 || rq->H->n != rq->S->n || rq->H->nnz != rq->S->nnz || rq->H->is_complex != rq->S->is_complex)
                return fail(HBSD_ERR_ARG, "H and S must have the same n, nnz and value type");
            if (rq->H->is_complex && rq->nl_k > 0) return fail(HBSD_ERR_UNSUPPORTED, "nonlocal term on complex input");
            if (!rq->lb->dof_node || !rq->H->row_ptr || !rq->H->col_idx || !rq->H->val || !rq->S->val)
                return fail(HBSD_ERR_ARG, "NULL array in the problem");
            if (rq->warm) return fail(HBSD_ERR_ARG, "a new problem cannot warm-start");
            n = rq->H->n;
            r->is_new = true;
            r->n = n;
            r->nnz = rq->H->nnz;
            r->row_ptr.assign(rq->H->row_ptr, rq->H->row_ptr + n + 1);
            r->col_idx.assign(rq->H->col_idx, rq->H->col_idx + r->nnz);
            r->is_complex = rq->H->is_complex ? 1 : 0;
            const int64_t vals = r->nnz * (r->is_complex ? 2 : 1);
            r->hval.assign(rq->H->val, rq->H->val + vals);
            r->sval.assign(rq->S->val, rq->S->val + vals);
            r->dof_node.assign(rq->lb->dof_node, rq->lb->dof_node + n);
            if (rq->lb->dof_cluster) r->dof_cluster.assign(rq->lb->dof_cluster, rq->lb->dof_cluster + n);
            std::memcpy(r->grid, rq->lb->grid, sizeof(r->grid));
            r->opt = *rq->opt;
            if (rq->nl_k < 0 || (rq->nl_k > 0 && (!rq->nl_F || !rq->nl_G || rq->nl_ldf < rq->nl_k)))
                return fail(HBSD_ERR_ARG, "nonlocal term: nl_F, nl_G required and nl_ldf >= nl_k");
            if (rq->nl_k > 0) {
                r->nl_k = rq->nl_k;
                r->nl_F.resize((size_t)n * rq->nl_k);
                for (int64_t i = 0; i < n; ++i)
                    std::memcpy(r->nl_F.data() + i * rq->nl_k, rq->nl_F + i * rq->nl_ldf, rq->nl_k * sizeof(double));
                r->nl_G.assign(rq->nl_G, rq->nl_G + (size_t)rq->nl_k * rq->nl_k);
            }
            // a complex problem runs as the real pencil of size 2n (4 nnz entries, 2 nev columns)
            r->est_raw = r->is_complex ? estimate_bytes(2 * n, 4 * r->nnz, 2 * rq->nev, 0)
                                       : estimate_bytes(n, r->nnz, rq->nev, r->nl_k);
            if (r->est_raw > sv->opts.hbm_budget_bytes) return fail(HBSD_ERR_OOM, "request exceeds the server's memory budget");
        } else {   // follow-up of a resident session: new H values (optional), warm start or X0
            std::lock_guard<std::mutex> lk(sv->mu);
            auto s = sv->sessions.find(rq->session_id);
            if (s == sv->sessions.end()) return fail(HBSD_ERR_ARG, "unknown or evicted session");
            const Session& ses = s->second.h->s;
            const int cw = ses.cplx ? 2 : 1;                    // doubles per value
            n = ses.cplx ? ses.n_c : ses.n;
            r->is_complex = ses.cplx ? 1 : 0;
            r->session_id = rq->session_id;
            if (rq->H_val) r->hval_new.assign(rq->H_val, rq->H_val + (ses.cplx ? 2 * (int64_t)ses.c_row_ptr.back() : ses.nnz));
            if (rq->X0) {
                const int64_t w = rq->nev + (ses.opt.m0 >= 0 ? ses.opt.m0 : std::max(3, (rq->nev + 9) / 10));
                r->X0.assign(rq->X0, rq->X0 + (size_t)n * w * cw);
            }
        }
        if (rq->X0 && r->is_new) {
            const int64_t w = rq->nev + (rq->opt->m0 >= 0 ? rq->opt->m0 : std::max(3, (rq->nev + 9) / 10));
            r->X0.assign(rq->X0, rq->X0 + (size_t)n * w * (r->is_complex ? 2 : 1));
        }
        r->t_submit = Clock::now();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r->ticket = sv->next_ticket++;
            *ticket = r->ticket;
            sv->results[r->ticket] = ResultRec{};
            sv->queue.push_back(std::move(r));
        }
        sv->cv.notify_all();
        return HBSD_OK;
    });
}

int hbsd_poll(hbsd_server* sv, uint64_t ticket, hbsd_result* out) {
    return guarded([&]() -> int {
        if (!sv || !out) return fail(HBSD_ERR_ARG, "NULL argument");
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->results.find(ticket);
        if (it == sv->results.end()) return fail(HBSD_ERR_ARG, "unknown ticket");
        if (!it->second.done) return HBSD_BUSY;
        *out = it->second.r;
        sv->results.erase(it);
        return HBSD_OK;
    });
}

int hbsd_session_release(hbsd_server* sv, int64_t session_id) {
    return guarded([&]() -> int {
        if (!sv) return fail(HBSD_ERR_ARG, "NULL server");
        std::unique_lock<std::mutex> lk(sv->mu);
        auto s = sv->sessions.find(session_id);
        if (s == sv->sessions.end()) return fail(HBSD_ERR_ARG, "unknown session");
        if (s->second.busy) return HBSD_BUSY;
        SessionRec rec = s->second;
        sv->sessions.erase(s);
        sv->used -= std::min(sv->used, rec.bytes);
        sv->graveyard.push_back(rec);
        lk.unlock();
        bury(sv);
        sv->cv.notify_all();
        return HBSD_OK;
    });
}

void hbsd_server_destroy(hbsd_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    for (auto& t : sv->workers) t.join();
    bury(sv);
    for (auto& kv : sv->sessions) {
        hbsd_destroy(kv.second.h);
        if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
    }
    delete sv;
}

}  // extern "C"
