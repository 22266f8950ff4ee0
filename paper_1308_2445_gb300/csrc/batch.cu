// Batched form: many resident sessions solved in one call, and the autotuner that picks the launch
// shapes of the fused SpMM (steps 3/7) and the cooperative MINRES (step 6(b)) for each session.
//
// The sessions are independent eigenproblems (k-points, SCF runs, configurations; Sec. 5 solves
// each separately with the same method).  Worker threads take them longest-first and run each
// solve on the session's own stream, so kernels of different sessions share the GPU: the small
// problems' launches, which fill only a few SMs each, overlap with each other and with the large
// problems' work.  The MINRES launch is cooperative and by default occupies every SM; the tuner
// gives small problems a smaller grid, which both shortens their grid barriers and lets the other
// sessions run beside them.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <thread>
#include <vector>

#include "common.h"

namespace hbsd {
namespace {

// deterministic fill in [-1, 1) (a 64-bit mix of the index; timing data only)
__global__ void k_tune_fill(double* x, int64_t count, uint64_t salt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + salt;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
}

struct TuneKey {
    int precision, width, cplx;
    int64_t n, nnz;
};

struct TuneEntry {
    TuneKey key;
    hbsd_tune t;
};

std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune_table;

bool same_class(const TuneKey& a, const TuneKey& b) {
    auto close = [](int64_t x, int64_t y) { return std::fabs((double)x - (double)y) <= 0.2 * (double)std::max(x, y); };
    return a.precision == b.precision && a.width == b.width && a.cplx == b.cplx && close(a.n, b.n) && close(a.nnz, b.nnz);
}

// CUDA-event time of fn() on stream st: one untimed run, then the best of `reps`
template <class Fn>
int time_best(cudaStream_t st, int reps, double* ms, Fn&& fn) {
    cudaEvent_t e0, e1;
    HBSD_CUDA(cudaEventCreate(&e0));
    HBSD_CUDA(cudaEventCreate(&e1));
    int rc = fn();
    double best = 1e300;
    for (int r = 0; r < reps && rc == 0; ++r) {
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = fail(HBSD_ERR_CUDA, "event record"); break; }
        rc = fn();
        if (rc) break;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = fail(HBSD_ERR_CUDA, "event wait");
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        best = std::min(best, (double)t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return rc;
}

}  // namespace

int autotune(Session* s, int width, hbsd_tune* out) {
    if (width < 1) return fail(HBSD_ERR_ARG, "autotune: width >= 1 required");
    const TuneKey key{s->opt.precision, width, s->cplx ? 1 : 0, s->n, s->nnz};
    hbsd_tune t{};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const TuneEntry& e : g_tune_table)
            if (same_class(e.key, key)) {
                t = e.t;
                t.from_table = 1;
                break;
            }
    }
    if (!t.from_table) {
        const cudaStream_t st = s->stream;
        const int64_t n = s->n;
        const int w = std::min<int64_t>(width, n);
        const int64_t ld = round_up(w, 4);
        DBuf<double> X, Y0, Y1, e;
        HBSD_TRY(X.alloc((size_t)n * ld));
        HBSD_TRY(Y0.alloc((size_t)n * ld));
        HBSD_TRY(Y1.alloc((size_t)n * ld));
        HBSD_TRY(e.alloc(64));
        k_tune_fill<<<1024, 256, 0, st>>>(X.p, n * ld, 0x5EEDull);
        HBSD_CUDA(cudaGetLastError());
        HBSD_CUDA(cudaMemsetAsync(e.p, 0, 64 * sizeof(double), st));
        const bool df = s->opt.precision == HBSD_PRECISION_MIXED && s->opt_df64 && s->opt.spmm_df64 && s->A.hsdf.p;
        const int saved_lpr = s->tune_spmm_lpr, saved_grid = s->tune_mr_grid;
        // 1. fused SpMM: most lanes per row
        static const int lanes[4] = {4, 8, 16, 32};
        double best = 1e300;
        int best_l = 32;
        for (int c = 0; c < 4; ++c) {
            s->tune_spmm_lpr = lanes[c];
            double ms = 0.0;
            int rc = time_best(st, 3, &ms, [&]() -> int {
                return df ? spmm_pair_df64(s, s->A, X.p, ld, w, Y0.p, ld, Y1.p, ld, st)
                          : spmm_pair<double>(s, s->A, X.p, ld, w, Y0.p, ld, Y1.p, ld, st);
            });
            if (rc) {
                s->tune_spmm_lpr = saved_lpr;
                return rc;
            }
            t.spmm_ms[c] = ms;
            if (ms < best * 0.98) { best = ms; best_l = lanes[c]; }   // ties go to the wider rows
        }
        // 2. cooperative MINRES: CTA count (10 steps; eta = 0 runs every step)
        s->tune_spmm_lpr = best_l;
        s->tune_mr_grid = 0;
        const int km = std::min(w, 32);
        HBSD_TRY(s->ws.alloc((size_t)304 * 2 * std::max(km, 1) + 64));
        int full = 0;
        double mr_best = 1e300;
        double mr_ms[6] = {0, 0, 0, 0, 0, 0};
        for (int c = 0; c < 6; ++c) {
            if (c > 0) {
                const int g = full >> c;
                if (g < 2) break;
                s->tune_mr_grid = g;
            }
            double ms = 0.0;
            int rc = time_best(st, 2, &ms, [&]() -> int {
                return minres_batch<double>(s, X.p, ld, e.p, km, 0.0, 10, Y0.p, ld, nullptr, nullptr, st,
                                            HBSD_LOCAL_MINRES);
            });
            if (rc) {
                s->tune_spmm_lpr = saved_lpr;
                s->tune_mr_grid = saved_grid;
                return rc;
            }
            if (c == 0) full = s->mr_blk_grid;
            mr_ms[c] = ms;
            mr_best = std::min(mr_best, ms);
        }
        int grid = full;
        for (int c = 0; c < 6; ++c)
            if (mr_ms[c] > 0.0 && mr_ms[c] <= 1.10 * mr_best) grid = c == 0 ? full : (full >> c);
        t.width = width;
        t.spmm_lanes = best_l;
        t.minres_ctas = grid;
        t.minres_ctas_full = full;
        for (int c = 0; c < 6; ++c) t.minres_ms[c] = mr_ms[c];
        HBSD_CUDA(cudaStreamSynchronize(st));
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_table.push_back(TuneEntry{key, t});
    }
    s->tune_spmm_lpr = t.spmm_lanes;
    s->tune_mr_grid = t.minres_ctas == t.minres_ctas_full ? 0 : t.minres_ctas;
    s->tuned_width = width;
    if (out) *out = t;
    return 0;
}

}  // namespace hbsd

using namespace hbsd;

void hbsd_batch_opts_default(hbsd_batch_opts* o) {
    if (!o) return;
    o->max_concurrent = 8;
    o->autotune = 1;
    o->longest_first = 1;
}

int hbsd_autotune(hbsd_handle* h, int width, hbsd_tune* out) {
    return guarded([&]() -> int {
        if (!h) return fail(HBSD_ERR_ARG, "NULL handle");
        return autotune(&h->s, width, out);
    });
}

int hbsd_solve_batch(hbsd_batch_item* items, int count, const hbsd_batch_opts* opts) {
    return guarded([&]() -> int {
        hbsd_batch_opts o;
        hbsd_batch_opts_default(&o);
        if (opts) o = *opts;
        if (count < 0 || (count > 0 && !items)) return fail(HBSD_ERR_ARG, "bad item list");
        if (o.max_concurrent < 1 || o.max_concurrent > 64) return fail(HBSD_ERR_ARG, "max_concurrent outside [1, 64]");
        std::vector<const hbsd_handle*> seen;
        for (int i = 0; i < count; ++i) {
            if (!items[i].h) return fail(HBSD_ERR_ARG, "NULL handle in the batch");
            if (items[i].nev < 1) return fail(HBSD_ERR_ARG, "nev >= 1 required");
            seen.push_back(items[i].h);
        }
        std::sort(seen.begin(), seen.end());
        if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
            return fail(HBSD_ERR_ARG, "a session appears twice in the batch");
        if (count == 0) return HBSD_OK;
        // tuning runs before the concurrent phase, one session at a time, so its timings see an idle GPU
        if (o.autotune) {
            for (int i = 0; i < count; ++i) {
                Session* S = &items[i].h->s;
                const int w = block_width(*S, items[i].nev);
                if (S->tuned_width != w) {
                    const int rc = autotune(S, w, nullptr);
                    if (rc) return rc;
                }
            }
        }
        std::vector<int> order(count);
        for (int i = 0; i < count; ++i) order[i] = i;
        if (o.longest_first) {
            std::vector<double> cost(count);
            for (int i = 0; i < count; ++i) {
                const Session& S = items[i].h->s;
                const double w = block_width(S, items[i].nev);
                cost[i] = w * ((double)S.nnz + (double)S.n * w);
            }
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        }
        std::atomic<int> next{0};
        const auto t0 = std::chrono::steady_clock::now();
        auto work = [&]() {
            for (;;) {
                const int j = next.fetch_add(1);
                if (j >= count) return;
                hbsd_batch_item& it = items[order[j]];
                const auto ts = std::chrono::steady_clock::now();
                hbsd_stats st{};
                int iters = 0;
                it.status = hbsd_solve_device(it.h, it.nev, it.tol, it.X0_dev, it.ldx0, it.lambda_dev, it.X_dev,
                                              it.ldx, &iters, &st);
                const auto te = std::chrono::steady_clock::now();
                it.iters = iters;
                it.res_max = st.res_max;
                it.start_ms = std::chrono::duration<double, std::milli>(ts - t0).count();
                it.run_ms = std::chrono::duration<double, std::milli>(te - ts).count();
            }
        };
        const int nt = std::min(o.max_concurrent, count);
        std::vector<std::thread> pool;
        int started = 0;
        try {
            for (; started < nt - 1; ++started) pool.emplace_back(work);
        } catch (...) {   // fewer threads than asked: the ones that started and this one finish the batch
        }
        work();
        for (std::thread& th : pool) th.join();
        for (int i = 0; i < count; ++i)
            if (items[i].status != HBSD_OK) return items[i].status;
        return HBSD_OK;
    });
}
