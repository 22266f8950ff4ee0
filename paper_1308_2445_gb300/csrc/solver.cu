// LABPSD driver (Sec. 3 outline, steps 1-12, with remarks 1-6) on the GB300 kernels, and the
// C ABI of include/hbsd.h.  The host runs the outer loop and decides, from the per-column
// relative residuals read back each iteration, which columns are preconditioned (remark 3)
// and which are refined locally (remark 4); every block operation runs in the kernels of
// sell.cu, dense.cu, chol.cu and minres.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <type_traits>

#include "common.h"

namespace hbsd {

static thread_local std::string g_last_error;

int64_t& tl_dev_bytes() {
    static thread_local int64_t bytes = 0;
    return bytes;
}

int64_t& tl_dev_peak() {
    static thread_local int64_t peak = 0;
    return peak;
}

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
void count_launch(Session* s) {
    if (s) s->launches++;
}

// ---- small kernels of the outer loop -----------------------------------------------------
namespace {

inline int grid_for(int64_t work) {
    return (int)std::min<int64_t>(std::max<int64_t>(1, (work + 255) / 256), 8192);
}

// R_U(:, j) = PsiH(:, U_j) - PsiS(:, U_j) E_{U_j}  (step 4 restricted to the unconverged columns)
template <class T>
__global__ void k_gather_residual(const T* __restrict__ PH, int64_t ldh, const T* __restrict__ PS, int64_t lds,
                                  const double* __restrict__ E, const int* __restrict__ U, int p, int64_t n,
                                  T* __restrict__ R, int64_t ldr) {
    const int64_t total = n * p;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / p;
        const int j = (int)(idx % p);
        const int c = U[j];
        R[i * ldr + j] = PH[i * ldh + c] - PS[i * lds + c] * (T)E[c];
    }
}

template <class T>
__global__ void k_gather_cols(const T* __restrict__ src, int64_t lds, const int* __restrict__ idx, int k, int64_t n,
                              T* __restrict__ dst, int64_t ldd) {
    const int64_t total = n * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int j = (int)(t % k);
        dst[i * ldd + j] = src[i * lds + idx[j]];
    }
}

template <class T>
__global__ void k_scatter_cols(const T* __restrict__ src, int64_t lds, const int* __restrict__ idx, int k, int64_t n,
                               T* __restrict__ dst, int64_t ldd) {
    const int64_t total = n * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int j = (int)(t % k);
        dst[i * ldd + idx[j]] = src[i * lds + j];
    }
}

template <class T>
__global__ void k_copy_block(const T* __restrict__ src, int64_t lds, int k, int64_t n, T* __restrict__ dst, int64_t ldd) {
    const int64_t total = n * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int j = (int)(t % k);
        dst[i * ldd + j] = src[i * lds + j];
    }
}

__global__ void k_shift_add(const double* __restrict__ E, int k, double sigma0, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) out[j] = E[j] + sigma0;
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator + Box-Muller
constexpr uint64_t GOLDEN = 0x9E3779B97F4A7C15ull;
inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
void seed_normals(uint64_t seed, uint64_t stream, int64_t count, double* out) {
    const uint64_t key = mix64((seed ^ (stream * GOLDEN)) + GOLDEN);
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t t = 0; t < count; t += 2) {
        const uint64_t z1 = mix64(key + (uint64_t)(t + 1) * GOLDEN);
        const uint64_t z2 = mix64(key + (uint64_t)(t + 2) * GOLDEN);
        const double u1 = (double)(z1 >> 11) * (1.0 / 9007199254740992.0);
        const double u2 = (double)(z2 >> 11) * (1.0 / 9007199254740992.0);
        const double rad = std::sqrt(-2.0 * std::log1p(-u1));
        out[t] = rad * std::cos(two_pi * u2);
        if (t + 1 < count) out[t + 1] = rad * std::sin(two_pi * u2);
    }
}

}  // namespace

// ---- trace (HBSD_TRACE=1): one stderr line per outer iteration ----------------------------------
static bool trace_on() {
    static int on = -1;
    if (on < 0) {
        const char* e = std::getenv("HBSD_TRACE");
        on = (e && e[0] && e[0] != '0') ? 1 : 0;
    }
    return on == 1;
}

// number of non-finite entries of a device array (trace only)
static int count_nonfinite(const double* p, int64_t n, cudaStream_t st) {
    std::vector<double> h(n);
    if (cudaMemcpyAsync(h.data(), p, n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    int c = 0;
    for (double v : h) c += !std::isfinite(v);
    return c;
}

// ---- step timers: CUDA events on the session stream, read back after host syncs ------------------
struct StepTimer {
    enum { MATVEC, RESID, PRECOND, LOCAL, GRAM, RR, UPDATE, NCLS };
    static constexpr int NEV = 32;
    cudaEvent_t ev[NEV][2];
    int cls[NEV];
    int used = 0;
    double acc[NCLS] = {};
    bool ok = false;
    StepTimer() {
        ok = true;
        for (int i = 0; i < NEV && ok; ++i)
            ok = cudaEventCreate(&ev[i][0]) == cudaSuccess && cudaEventCreate(&ev[i][1]) == cudaSuccess;
    }
    ~StepTimer() {
        for (int i = 0; i < NEV; ++i) { cudaEventDestroy(ev[i][0]); cudaEventDestroy(ev[i][1]); }
    }
    int begin(int c, cudaStream_t st) {
        if (!ok) return -1;
        if (used == NEV) flush();
        const int i = used++;
        cls[i] = c;
        cudaEventRecord(ev[i][0], st);
        return i;
    }
    void end(int i, cudaStream_t st) {
        if (i >= 0) cudaEventRecord(ev[i][1], st);
    }
    void flush() {  // waits for the recorded pairs
        for (int i = 0; i < used; ++i) {
            float ms = 0.f;
            if (cudaEventSynchronize(ev[i][1]) == cudaSuccess && cudaEventElapsedTime(&ms, ev[i][0], ev[i][1]) == cudaSuccess)
                acc[cls[i]] += ms;
        }
        used = 0;
    }
};

// Gram and update of the loop: the mixed form computes them in double-float arithmetic on the
// FP32 pipes (FP64 accumulation across 128-row tiles for the Gram sums), the FP64 form in FP64.
template <class T>
static int gram_step(Session* S, bool df, const T* Z0, int64_t ld0, int q0, const T* Z1, int64_t ld1, int q1,
                     const T* H0, int64_t ldh0, const T* H1, int64_t ldh1, const T* S0, int64_t lds0, const T* S1,
                     int64_t lds1, int64_t n, double* HR, double* SR, cudaStream_t st) {
    if constexpr (std::is_same<T, double>::value) {
        if (df) return gram2_df64(S, Z0, ld0, q0, Z1, ld1, q1, H0, ldh0, H1, ldh1, S0, lds0, S1, lds1, n, HR, SR, st);
    }
    return gram2<T>(S, Z0, ld0, q0, Z1, ld1, q1, H0, ldh0, H1, ldh1, S0, lds0, S1, lds1, n, HR, SR, st);
}
// Steps 10-11 for one block: Zb(:, 0:k) := [Zb Z1] W.  With tc, on the tensor cores from exact bf16
// slices into the spare block, which then takes Zb's place (k = q0: every column is replaced).
template <class T>
static int update_block(Session* S, bool df, bool tc, SolveBufs<T>& B, DBuf<T>& Zb, int64_t ld0, int q0,
                        const T* Z1, int64_t ld1, int q1, int64_t n, const double* W, int k, cudaStream_t st,
                        bool first);
template <class T>
static int update_step(Session* S, bool df, T* Z0, int64_t ld0, int q0, const T* Z1, int64_t ld1, int q1, int64_t n,
                       const double* W, int k, cudaStream_t st, bool first) {
    if constexpr (std::is_same<T, double>::value) {
        if (df) return update2_df64(S, Z0, ld0, q0, Z1, ld1, q1, n, W, k, st, first);
    }
    (void)first;
    return update2<T>(S, Z0, ld0, q0, Z1, ld1, q1, n, W, k, st);
}

template <class T>
static int update_block(Session* S, bool df, bool tc, SolveBufs<T>& B, DBuf<T>& Zb, int64_t ld0, int q0,
                        const T* Z1, int64_t ld1, int q1, int64_t n, const double* W, int k, cudaStream_t st,
                        bool first) {
    if constexpr (std::is_same<T, double>::value) {
        if (tc && k == q0 && q0 <= OZ_MAX_Q_SEG && q1 <= OZ_MAX_Q_SEG) {
            HBSD_TRY(B.upd.alloc((size_t)n * ld0));
            HBSD_TRY(update_oz(S, Zb.p, ld0, q0, Z1, ld1, q1, n, W, k, B.upd.p, ld0, st, S->oz_status.p));
            std::swap(Zb.p, B.upd.p);
            std::swap(Zb.n, B.upd.n);
            return 0;
        }
    }
    return update_step<T>(S, df, Zb.p, ld0, q0, Z1, ld1, q1, n, W, k, st, first);
}

// ---- per-solve buffers -----------------------------------------------------------------------

template <class S_, class D_>
__global__ void k_convert_block(const S_* __restrict__ src, int64_t lds, int k, int64_t n, D_* __restrict__ dst,
                                int64_t ldd, const double* __restrict__ d, int pw);
template <class T>
__global__ void k_neg_block(const T* __restrict__ src, int64_t lds, int k, int64_t n, T* __restrict__ dst,
                            int64_t ldd);

// Stopping rule of one precision phase.
struct PhaseRule {
    double tol;          // Res_max target (remark 2)
    int max_iters;       // outer iterations allowed in this phase
    bool stagnation;     // stop when Res_max has not halved over `window` iterations (FP32 floor)
    int window;
};

// True when Res_max has stalled: more than `win` entries since `mark`, the best of the entries
// before the last `win` is below `below`, and the best of the last `win` is above half of it.
static bool res_stalled(const double* hist, size_t len, size_t mark, int win, double below) {
    if (win < 1 || len < mark || (int64_t)(len - mark) <= win) return false;
    double best_before = hist[0];
    for (size_t i = 0; i + win < len; ++i) best_before = std::min(best_before, hist[i]);
    double best_recent = hist[len - win];
    for (size_t i = len - win; i < len; ++i) best_recent = std::min(best_recent, hist[i]);
    return best_before < below && best_recent > 0.5 * best_before;
}

// LABPSD outline (Sec. 3) in precision T on the blocks of B, starting from Psi (n x w, ld ldw):
// steps 1-3 (Rayleigh-Ritz on span(Psi)) then steps 4-11 until the rule stops it.  E_host and
// Eprev carry the Ritz values across phases (remark 4 needs the previous ones).
template <class T>
static int labpsd_phase(Session* S, SolveBufs<T>& B, SolveCommon& C, int m, int w, int64_t ldw, int64_t ldp,
                        const PhaseRule& rule, std::vector<double>& E, std::vector<double>& Eprev, int* iters_done,
                        bool* converged, StepTimer& tm) {
    cudaStream_t st = S->stream;
    const hbsd_options& o = S->opt;
    const int64_t n = S->n;
    hbsd_stats& stt = S->stats;
    int ti;
    int info[2];
    *converged = false;
    // FP64 keeps the reading of the paper (R13).  An FP32 instantiation (which no solve form
    // runs) would treat scaled-S_R pivots below 1e-6 as dependent directions: its Gram entries
    // carry ~1e-7 relative noise.
    const double drop_tol = sizeof(T) == 4 ? 1e-6 : 0.0;
    bool dfp = o.precision == HBSD_PRECISION_MIXED && S->opt_df64;   // double-float Gram / update
    const bool tcu = o.precision == HBSD_PRECISION_MIXED && o.tc_update != 0;   // tensor-core update
    // products of steps 3/7 and the Psi_H, Psi_S recomputation: double-float on the scaled pencil
    // in the mixed form (spmm_df64), FP64 otherwise
    bool dfs = std::is_same<T, double>::value && o.precision == HBSD_PRECISION_MIXED && o.spmm_df64 != 0;
    stt.fp64_from_iter = stt.fp64_gram_from_iter = -1;
    size_t esc_mark = 0;   // history length at the last precision switch
    auto products = [&](const T* Xp, int64_t ldx, int k, T* HXp, int64_t ldh, T* SXp, int64_t lds) -> int {
        if constexpr (std::is_same<T, double>::value) {
            if (dfs) return spmm_pair_df64(S, S->A, Xp, ldx, k, HXp, ldh, SXp, lds, st);
        }
        return spmm_pair<T>(S, S->A, Xp, ldx, k, HXp, ldh, SXp, lds, st);
    };
    // Psi_H, Psi_S updated with W (steps 10-11 as printed) or recomputed from the new Psi by the
    // fused SpMM: the same blocks up to rounding, the SpMM costing less than two block updates here
    // per update of width q: update_hs = 1 updates, 0 recomputes; -1 (auto) updates in the FP64
    // form and, in the mixed form, recomputes when the SpMM's FP64 work (2 nnz per column) is below
    // that of two double-float block updates (2 n q per column at ~3.5x the FP64 rate)
    auto upd_hs_for = [&](int qq) -> bool {
        if (o.update_hs >= 0) return o.update_hs > 0;
        if (o.precision == HBSD_PRECISION_FP64) return true;
        return !((double)qq * (double)n > (dfs ? 1.5 : 3.5) * (double)S->nnz);
    };
    bool hs_fresh = false;   // Psi_H, Psi_S recomputed in FP64 by the last update step
    bool certified = false;   // Psi_H, Psi_S freshly recomputed in FP64 (mixed form)
    // steps 1-3: Psi_H, Psi_S, Rayleigh-Ritz on span(Psi)
    ti = tm.begin(StepTimer::MATVEC, st);
    HBSD_TRY(products(B.Psi.p, ldw, w, B.PsiH.p, ldw, B.PsiS.p, ldw));
    tm.end(ti, st);
    stt.matvec_cols += w;
    ti = tm.begin(StepTimer::GRAM, st);
    HBSD_TRY(gram_step<T>(S, dfp, B.Psi.p, ldw, w, (const T*)nullptr, 0, 0, B.PsiH.p, ldw, (const T*)nullptr, 0, B.PsiS.p,
                      ldw, (const T*)nullptr, 0, n, C.HR.p, C.SR.p, st));
    tm.end(ti, st);
    stt.gram_fma += (double)n * w * (w + 1);
    if (trace_on())
        std::fprintf(stderr, "[hbsd] %s start: Rayleigh-Ritz on the start block, nonfinite HR %d SR %d\n",
                     sizeof(T) == 4 ? "fp32" : "fp64", count_nonfinite(C.HR.p, (int64_t)w * w, st),
                     count_nonfinite(C.SR.p, (int64_t)w * w, st));
    ti = tm.begin(StepTimer::RR, st);
    HBSD_TRY(rayleigh_ritz_cluster(S, C.HR.p, C.SR.p, w, w, C.theta.p, C.W.p, info, st, drop_tol));
    tm.end(ti, st);
    stt.rr_fallbacks += info[0];
    bool upd_hs = upd_hs_for(w);
    hs_fresh = !upd_hs && !dfs;
    ti = tm.begin(StepTimer::UPDATE, st);
    HBSD_TRY(update_block<T>(S, dfp, tcu, B, B.Psi, ldw, w, (const T*)nullptr, 0, 0, n, C.W.p, w, st, true));
    if (upd_hs) {
        HBSD_TRY(update_block<T>(S, dfp, tcu, B, B.PsiH, ldw, w, (const T*)nullptr, 0, 0, n, C.W.p, w, st, false));
        HBSD_TRY(update_block<T>(S, dfp, tcu, B, B.PsiS, ldw, w, (const T*)nullptr, 0, 0, n, C.W.p, w, st, false));
    }
    tm.end(ti, st);
    stt.update_fma += (upd_hs ? 3.0 : 1.0) * n * w * w;
    if (!upd_hs) {   // Psi_H = Hs Psi, Psi_S = S Psi by the fused SpMM of steps 3/7
        ti = tm.begin(StepTimer::MATVEC, st);
        HBSD_TRY(products(B.Psi.p, ldw, w, B.PsiH.p, ldw, B.PsiS.p, ldw));
        tm.end(ti, st);
        stt.matvec_cols += w;
    }
    HBSD_CUDA(cudaMemcpyAsync(C.E.p, C.theta.p, w * 8, cudaMemcpyDeviceToDevice, st));
    HBSD_CUDA(cudaMemcpyAsync(E.data(), C.theta.p, w * 8, cudaMemcpyDeviceToHost, st));
    std::vector<double> res(m);
    std::vector<int> U, Lpos;
    std::vector<T> shifts;
    std::vector<double> hist;
    const bool hybrid = o.precond == HBSD_PRECOND_HYBRID || o.precond == HBSD_PRECOND_LOCAL;   // localization on
    const bool local_only = o.precond == HBSD_PRECOND_LOCAL;   // no step 6(a) (reading R16)
    int iters = 0;
    for (;;) {
        // steps 4-5
        ti = tm.begin(StepTimer::RESID, st);
        HBSD_TRY(residual<T>(S, B.PsiH.p, ldw, B.PsiS.p, ldw, C.E.p, m, (T*)nullptr, 0, n, C.res.p, nullptr, st));
        tm.end(ti, st);
        HBSD_CUDA(cudaMemcpyAsync(res.data(), C.res.p, m * 8, cudaMemcpyDeviceToHost, st));
        HBSD_CUDA(cudaStreamSynchronize(st));
        double rmax = 0.0;
        for (double r : res) {
            if (!std::isfinite(r)) return fail(HBSD_ERR_RR_RANK, "non-finite residual norm");
            rmax = std::max(rmax, r);
        }
        stt.res_max = rmax;
        hist.push_back(rmax);
        if (rmax <= rule.tol) {
            // the mixed form carries Psi_H, Psi_S through double-float updates: before accepting,
            // recompute them from Psi in FP64 and test the residual again (a failing test just
            // continues the iteration from the recomputed blocks)
            if ((dfp || dfs) && !hs_fresh && !certified) {
                certified = true;
                hs_fresh = true;
                ti = tm.begin(StepTimer::MATVEC, st);
                HBSD_TRY(spmm_pair<T>(S, S->A, B.Psi.p, ldw, w, B.PsiH.p, ldw, B.PsiS.p, ldw, st));
                tm.end(ti, st);
                stt.matvec_cols += w;
                hist.pop_back();
                continue;
            }
            *converged = true;
            break;
        }
        certified = false;
        if (iters >= rule.max_iters) break;
        // precision escalation: double-float sums carry ~48 bits, and where the terms of H x, or of
        // the Gram and update sums, cancel strongly the residuals stall above tol (measured: near
        // 1e-6 on enriched 16^3-40^3 problems whose FP64 solves converge in 23-160 iterations; on
        // some FP64 products restore convergence, on others only FP64 products with an FP64 Gram
        // and update).  A stall -- no halving of the best Res_max over the last 10 iterations once
        // it has been below 1e4 tol, or over the last 30 at any level -- first moves the products
        // of steps 3/7 to FP64 (Psi_H and Psi_S recomputed from Psi in FP64, the residual test
        // repeated); a further stall, counted from that switch, moves the Gram and the update to
        // FP64 too.  The first stage is cheap, so a false alarm on a slow but healthy trajectory
        // (a plateau of a cluster cut by the block edge) costs little.
        auto stalled = [&](int win, double below) -> bool {
            return res_stalled(hist.data(), hist.size(), esc_mark, win, below);
        };
        if ((dfs || dfp) && (stalled(10, 1e4 * rule.tol) || stalled(30, 1e300))) {
            if (dfs) {
                dfs = false;
                stt.fp64_from_iter = iters;
            } else {
                dfp = false;
                stt.fp64_gram_from_iter = iters;
            }
            esc_mark = hist.size() - 1;
            hs_fresh = true;
            ti = tm.begin(StepTimer::MATVEC, st);
            HBSD_TRY(spmm_pair<T>(S, S->A, B.Psi.p, ldw, w, B.PsiH.p, ldw, B.PsiS.p, ldw, st));
            tm.end(ti, st);
            stt.matvec_cols += w;
            hist.pop_back();
            continue;
        }
        if (rule.stagnation && (int)hist.size() > rule.window) {
            double best_before = hist[0];
            for (size_t i = 0; i + rule.window < hist.size(); ++i) best_before = std::min(best_before, hist[i]);
            double best_recent = hist[hist.size() - rule.window];
            for (size_t i = hist.size() - rule.window; i < hist.size(); ++i) best_recent = std::min(best_recent, hist[i]);
            if (best_recent > 0.5 * best_before) break;
        }
        // step 6: unconverged columns (remark 3), localized among them (remark 4)
        U.clear(); Lpos.clear(); shifts.clear();
        for (int i = 0; i < m; ++i)
            if (res[i] > rule.tol) U.push_back(i);
        const int p = (int)U.size();
        if (hybrid && !Eprev.empty()) {
            for (int j = 0; j < p; ++j) {
                const int i = U[j];
                if (res[i] <= o.tau1 && std::fabs(E[i] - Eprev[i]) <= o.tau2 * std::fabs(Eprev[i])) {
                    Lpos.push_back(j);
                    shifts.push_back((T)E[i]);
                }
            }
        }
        const int a = (int)Lpos.size();
        HBSD_CUDA(cudaMemcpyAsync(C.Ulist.p, U.data(), p * sizeof(int), cudaMemcpyHostToDevice, st));
        ti = tm.begin(StepTimer::RESID, st);
        k_gather_residual<T><<<grid_for(n * p), 256, 0, st>>>(B.PsiH.p, ldw, B.PsiS.p, ldw, C.E.p, C.Ulist.p, p, n,
                                                             B.RU.p, ldp);
        HBSD_LAUNCHED(S);
        tm.end(ti, st);
        const bool fp32_dirs = sizeof(T) == 8 && o.precision == HBSD_PRECISION_MIXED && !local_only;
        ti = tm.begin(StepTimer::PRECOND, st);
        if (local_only) {   // P = -R on the unconverged columns
            k_neg_block<T><<<grid_for(n * p), 256, 0, st>>>(B.RU.p, ldp, p, n, B.P.p, ldp);
            HBSD_LAUNCHED(S);
        } else if (fp32_dirs) {
            // 6(a) in FP32 on the scaled pencil: P^ = -(D A D)^{-1} (D R); P^ stays scaled for 6(b)
            k_convert_block<T, float><<<grid_for(n * p), 256, 0, st>>>(B.RU.p, ldp, p, n, S->r32.p, ldp,
                                                                      S->A.dscale.p, +1);
            HBSD_LAUNCHED(S);
            HBSD_TRY(factor_solve<float>(S, S->F, S->r32.p, ldp, p, S->p32.p, ldp, st));
            HBSD_TRY(nl_smw_correct<float>(S, S->p32.p, ldp, p, st));            // SMW step 6 (scaled)
        } else {
            HBSD_TRY(factor_solve<T>(S, S->F, B.RU.p, ldp, p, B.P.p, ldp, st));   // 6(a)
            HBSD_TRY(nl_smw_correct<T>(S, B.P.p, ldp, p, st));                    // SMW step 6
        }
        tm.end(ti, st);
        stt.precond_cols += p;
        stt.precond_calls += 1;
        if (a > 0) {                                                          // 6(b)
            ti = tm.begin(StepTimer::LOCAL, st);
            HBSD_CUDA(cudaMemcpyAsync(C.Llist.p, Lpos.data(), a * sizeof(int), cudaMemcpyHostToDevice, st));
            int64_t msteps = 0;
            if (fp32_dirs) {   // P = D P^ (6(a) in FP32), the refinement in FP64
                k_convert_block<float, T><<<grid_for(n * p), 256, 0, st>>>(S->p32.p, ldp, p, n, B.P.p, ldp,
                                                                          S->A.dscale.p, +1);
                HBSD_LAUNCHED(S);
            }
            HBSD_CUDA(cudaMemcpyAsync(B.shifts.p, shifts.data(), a * sizeof(T), cudaMemcpyHostToDevice, st));
            if (local_only) {   // MINRES from zero
                HBSD_CUDA(cudaMemsetAsync(B.Xa.p, 0, (size_t)n * ldp * sizeof(T), st));
            } else {
                k_gather_cols<T><<<grid_for(n * a), 256, 0, st>>>(B.P.p, ldp, C.Llist.p, a, n, B.Xa.p, ldp);
                HBSD_LAUNCHED(S);
            }
            k_gather_cols<T><<<grid_for(n * a), 256, 0, st>>>(B.RU.p, ldp, C.Llist.p, a, n, B.Ra.p, ldp);
            HBSD_LAUNCHED(S);
            HBSD_TRY(minres_batch<T>(S, B.Ra.p, ldp, B.shifts.p, a, o.eta, o.max_minres, B.Xa.p, ldp, C.steps.p,
                                     &msteps, st, o.local_solver));
            k_scatter_cols<T><<<grid_for(n * a), 256, 0, st>>>(B.Xa.p, ldp, C.Llist.p, a, n, B.P.p, ldp);
            HBSD_LAUNCHED(S);
            tm.end(ti, st);
            stt.minres_steps += msteps;
            stt.local_cols += a;
            stt.local_calls += 1;
        }
        if (fp32_dirs && a == 0) {   // P = D P^ (no refinement this iteration)
            k_convert_block<float, T><<<grid_for(n * p), 256, 0, st>>>(S->p32.p, ldp, p, n, B.P.p, ldp,
                                                                      S->A.dscale.p, +1);
            HBSD_LAUNCHED(S);
        }
        // step 7
        ti = tm.begin(StepTimer::MATVEC, st);
        HBSD_TRY(products(B.P.p, ldp, p, B.PH.p, ldp, B.PS.p, ldp));
        tm.end(ti, st);
        stt.matvec_cols += p;
        // step 8
        const int q = w + p;
        ti = tm.begin(StepTimer::GRAM, st);
        HBSD_TRY(gram_step<T>(S, dfp, B.Psi.p, ldw, w, B.P.p, ldp, p, B.PsiH.p, ldw, B.PH.p, ldp, B.PsiS.p, ldw, B.PS.p, ldp,
                          n, C.HR.p, C.SR.p, st));
        tm.end(ti, st);
        stt.gram_fma += (double)n * q * (q + 1);
        // step 9
        if (trace_on())
            std::fprintf(stderr, "[hbsd] %s it %d res_max %.3e p %d a %d nonfinite HR %d SR %d\n",
                         sizeof(T) == 4 ? "fp32" : "fp64", iters + 1, hist.back(), p, a,
                         count_nonfinite(C.HR.p, (int64_t)q * q, st), count_nonfinite(C.SR.p, (int64_t)q * q, st));
        ti = tm.begin(StepTimer::RR, st);
        const auto h0 = std::chrono::steady_clock::now();
        HBSD_TRY(rayleigh_ritz_cluster(S, C.HR.p, C.SR.p, q, w, C.theta.p, C.W.p, info, st, drop_tol));
        S->dbg_rr_host_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h0).count();
        tm.end(ti, st);
        stt.rr_fallbacks += info[0];
        if (trace_on())
            std::fprintf(stderr, "[hbsd]   RR q %d rank %d branch %d nonfinite theta %d W %d\n", q, info[1], info[0],
                         count_nonfinite(C.theta.p, w, st), count_nonfinite(C.W.p, (int64_t)q * w, st));
        // steps 10-11
        upd_hs = upd_hs_for(q);
        hs_fresh = !upd_hs && !dfs;
        ti = tm.begin(StepTimer::UPDATE, st);
        HBSD_TRY(update_block<T>(S, dfp, tcu, B, B.Psi, ldw, w, B.P.p, ldp, p, n, C.W.p, w, st, true));
        if (upd_hs) {
            HBSD_TRY(update_block<T>(S, dfp, tcu, B, B.PsiH, ldw, w, B.PH.p, ldp, p, n, C.W.p, w, st, false));
            HBSD_TRY(update_block<T>(S, dfp, tcu, B, B.PsiS, ldw, w, B.PS.p, ldp, p, n, C.W.p, w, st, false));
        }
        tm.end(ti, st);
        stt.update_fma += (upd_hs ? 3.0 : 1.0) * n * q * w;
        if (!upd_hs) {   // Psi_H = Hs Psi, Psi_S = S Psi by the fused SpMM of steps 3/7
            ti = tm.begin(StepTimer::MATVEC, st);
            HBSD_TRY(products(B.Psi.p, ldw, w, B.PsiH.p, ldw, B.PsiS.p, ldw));
            tm.end(ti, st);
            stt.matvec_cols += w;
        }
        Eprev = E;
        HBSD_CUDA(cudaMemcpyAsync(C.E.p, C.theta.p, w * 8, cudaMemcpyDeviceToDevice, st));
        HBSD_CUDA(cudaMemcpyAsync(E.data(), C.theta.p, w * 8, cudaMemcpyDeviceToHost, st));
        ++iters;
    }
    *iters_done = iters;
    S->res_hist = hist;
    return 0;
}

template <class T>
static int alloc_blocks(SolveBufs<T>& B, int64_t n, int64_t ldw, int64_t ldp, int m) {
    HBSD_TRY(B.Psi.alloc(n * ldw)); HBSD_TRY(B.PsiH.alloc(n * ldw)); HBSD_TRY(B.PsiS.alloc(n * ldw));
    HBSD_TRY(B.P.alloc(n * ldp)); HBSD_TRY(B.PH.alloc(n * ldp)); HBSD_TRY(B.PS.alloc(n * ldp));
    HBSD_TRY(B.RU.alloc(n * ldp)); HBSD_TRY(B.Xa.alloc(n * ldp)); HBSD_TRY(B.Ra.alloc(n * ldp));
    HBSD_TRY(B.shifts.alloc(m));
    return 0;
}

// dst(i, j) = -src(i, j)
template <class T>
__global__ void k_neg_block(const T* __restrict__ src, int64_t lds, int k, int64_t n, T* __restrict__ dst,
                            int64_t ldd) {
    const int64_t total = n * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int j = (int)(t % k);
        dst[i * ldd + j] = -src[i * lds + j];
    }
}

// dst(i, j) = src(i, j) * d_i^pow  (pow = -1: into scaled coordinates y = D^{-1} x; +1: back)
template <class S_, class D_>
__global__ void k_convert_block(const S_* __restrict__ src, int64_t lds, int k, int64_t n, D_* __restrict__ dst,
                                int64_t ldd, const double* __restrict__ d, int pw) {
    const int64_t total = n * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int j = (int)(t % k);
        const double f = pw > 0 ? d[i] : 1.0 / d[i];
        dst[i * ldd + j] = (D_)((double)src[i * lds + j] * f);
    }
}

// Whole solve.  FP64: every step in FP64.  Mixed: the same iteration with step 6(a) -- the global
// preconditioner, which only shapes the search directions -- in FP32 on the diagonally scaled
// pencil (D A D, D = diag(S)^{-1/2}, which keeps the numbers inside the FP32 range); the operator
// products inside MINRES in FP32 on that pencil (vectors and recurrences FP64); the block
// products of steps 3/7, the Gram and the update in double-float (~48 bits) on the FP32 pipes,
// with the products escalated to FP64 when the residual stalls; residual norms, Rayleigh-Ritz and
// the final convergence test in FP64.  The directions K r carry components along the shared
// near-null space of H and S amplified ~1e11: extracting the subspace from them in plain FP32
// diverges (measured on the 32^3 workload), hence the double-float Gram and update.
static int labpsd_solve(Session* S, int m, double tol, const double* X0, int64_t ldx0, double* lam_dev,
                        double* X_dev, int64_t ldx, int* iters_out, int m0_force = -1) {
    cudaStream_t st = S->stream;
    const hbsd_options& o = S->opt;
    const int64_t n = S->n;
    const int m0 = m0_force >= 0 ? m0_force : o.m0 >= 0 ? o.m0 : std::max(3, (m + 9) / 10);
    const int w = m + m0;
    if (m < 1 || w > n) return fail(HBSD_ERR_ARG, "nev + m0 must lie in [1, n]");
    const bool mixed = o.precision == HBSD_PRECISION_MIXED;
    const int64_t ldw = round_up(w, 4), ldp = round_up(std::max(m, 1), 4);
    const int qmax = w + m;
    SolveCommon& C = S->sc;   // session-resident: the DBufs only grow, so repeated solves do not allocate
    HBSD_TRY(C.E.alloc(w)); HBSD_TRY(C.res.alloc(m)); HBSD_TRY(C.theta.alloc(w));
    HBSD_TRY(C.HR.alloc((size_t)qmax * qmax)); HBSD_TRY(C.SR.alloc((size_t)qmax * qmax));
    HBSD_TRY(C.W.alloc((size_t)qmax * w));
    HBSD_TRY(C.Ulist.alloc(m)); HBSD_TRY(C.Llist.alloc(m)); HBSD_TRY(C.steps.alloc(m));
    {   // scratch of the reductions and the Gram partials, sized once (no reallocation mid-solve)
        const int tiles = ceil_div(qmax, 32);
        HBSD_TRY(S->ws.alloc((size_t)2 * 1024 * (1216 + tiles * tiles) + (size_t)304 * 2 * qmax + 1024));
        HBSD_TRY(S->rr_info.alloc(4));
    }
    HBSD_TRY(S->oz_status.alloc(1));
    HBSD_CUDA(cudaMemsetAsync(S->oz_status.p, 0, sizeof(int), st));
    hbsd_stats& stt = S->stats;
    stt.iters = stt.iters_fp64 = 0;
    stt.minres_steps = stt.precond_cols = stt.local_cols = 0;
    stt.rr_fallbacks = 0;
    stt.matvec_cols = stt.minres_spmm_cols = 0;
    stt.local_calls = 0;
    stt.precond_calls = 0;
    stt.gram_fma = stt.update_fma = 0.0;
    StepTimer tm;
    std::vector<double> E(w), Eprev;
    SolveBufs<double>& B64 = S->sb;
    HBSD_TRY(alloc_blocks(B64, n, ldw, ldp, m));
    int it64 = 0;
    bool conv = false;
    if (mixed && S->has_factor) {
        HBSD_TRY(factor_make_fp32(S->F, S->A.dscale.p, st));
        HBSD_TRY(S->r32.alloc((size_t)n * ldp));
        HBSD_TRY(S->p32.alloc((size_t)n * ldp));
        HBSD_TRY(S->xa32.alloc((size_t)n * ldp));
        HBSD_TRY(S->ra32.alloc((size_t)n * ldp));
        HBSD_TRY(S->sh32.alloc(m));
    }
    k_copy_block<double><<<grid_for(n * w), 256, 0, st>>>(X0, ldx0, w, n, B64.Psi.p, ldw);
    HBSD_LAUNCHED(S);
    // one FP64 outer loop in both forms; the mixed form differs inside it (FP32 directions of
    // step 6(a), double-float Gram and update)
    PhaseRule r64{tol, std::max(0, o.max_outer), false, 0};
    HBSD_TRY(labpsd_phase<double>(S, B64, C, m, w, ldw, ldp, r64, E, Eprev, &it64, &conv, tm));
    const int iters = it64;
    stt.iters = iters;
    stt.iters_fp64 = it64;
    tm.flush();
    stt.t_matvec_ms = tm.acc[StepTimer::MATVEC];
    stt.t_resid_ms = tm.acc[StepTimer::RESID];
    stt.t_precond_ms = tm.acc[StepTimer::PRECOND];
    stt.t_local_ms = tm.acc[StepTimer::LOCAL];
    stt.t_gram_ms = tm.acc[StepTimer::GRAM];
    stt.t_rr_ms = tm.acc[StepTimer::RR];
    if (std::getenv("HBSD_RRDBG"))
        std::fprintf(stderr, "[hbsd] RR step timer %.1f ms, kernel events %.1f ms, host call %.1f ms, sync-to-next-event %.1f ms\n",
                     tm.acc[StepTimer::RR], S->dbg_rr_kernel_ms, S->dbg_rr_host_ms, S->dbg_rr_wake_ms);
    stt.t_update_ms = tm.acc[StepTimer::UPDATE];
    if (lam_dev) {
        k_shift_add<<<ceil_div(m, 128), 128, 0, st>>>(C.E.p, m, S->sigma0, lam_dev);
        HBSD_LAUNCHED(S);
    }
    if (X_dev) {
        k_copy_block<double><<<grid_for(n * m), 256, 0, st>>>(B64.Psi.p, ldw, m, n, X_dev, ldx);
        HBSD_LAUNCHED(S);
    }
    // keep the block for a warm start
    HBSD_TRY(S->psi_keep.alloc(n * ldw));
    HBSD_CUDA(cudaMemcpyAsync(S->psi_keep.p, B64.Psi.p, n * ldw * 8, cudaMemcpyDeviceToDevice, st));
    S->keep_w = w;
    S->keep_ld = ldw;
    int oz_fail = 0;
    HBSD_CUDA(cudaMemcpyAsync(&oz_fail, S->oz_status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (oz_fail) return fail(HBSD_ERR_TIMEOUT, "tensor-core update: an MMA completion wait gave up");
    if (iters_out) *iters_out = iters;
    return conv ? HBSD_OK : HBSD_NOT_CONVERGED;
}

}  // namespace hbsd

using namespace hbsd;

// ---- C ABI ------------------------------------------------------------------------------
extern "C" {

void hbsd_options_default(hbsd_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->sigma_bar = std::numeric_limits<double>::quiet_NaN();
    opt->sigma0 = std::numeric_limits<double>::quiet_NaN();
    opt->m0 = -1;
    opt->tau1 = 0.1;
    opt->tau2 = 0.1;
    opt->eta = 0.25;
    opt->max_minres = 20;
    opt->max_outer = 1000;
    opt->precision = HBSD_PRECISION_FP64;
    opt->precond = HBSD_PRECOND_HYBRID;
    opt->seed = 1;
    opt->local_solver = HBSD_LOCAL_MINRES;
    opt->tc_update = 0;
    opt->update_hs = -1;
    opt->minres_f32 = 1;
    opt->spmm_df64 = 1;
}

const char* hbsd_status_string(int status) {
    switch (status) {
        case HBSD_OK: return "ok";
        case HBSD_NOT_CONVERGED: return "not converged";
        case HBSD_BUSY: return "busy";
        case HBSD_ERR_ARG: return "invalid argument";
        case HBSD_ERR_OOM: return "out of device memory";
        case HBSD_ERR_NOT_SPD: return "H - sigma_bar S is not positive definite";
        case HBSD_ERR_RR_RANK: return "search space rank too small";
        case HBSD_ERR_TIMEOUT: return "device wait timed out";
        case HBSD_ERR_CUDA: return "CUDA error";
        case HBSD_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

const char* hbsd_last_error(void) { return g_last_error.c_str(); }

int hbsd_create(const hbsd_csr* H, const hbsd_csr* Sm, const hbsd_local_blocks* lb, const hbsd_options* opt,
                void* stream, hbsd_handle** out) {
    return guarded([&]() -> int {
        if (!out) return fail(HBSD_ERR_ARG, "out is NULL");
        *out = nullptr;
        if (!H || !Sm || !lb || !opt) return fail(HBSD_ERR_ARG, "H, S, local blocks and options are required");
        if (H->is_complex != Sm->is_complex) return fail(HBSD_ERR_ARG, "H and S must both be real or both complex");
        if (!H->row_ptr || !H->col_idx || !H->val || !Sm->val || !Sm->row_ptr || !Sm->col_idx)
            return fail(HBSD_ERR_ARG, "NULL CSR array");
        if (H->n <= 0 || H->n != Sm->n || H->nnz != Sm->nnz || H->nnz != H->row_ptr[H->n])
            return fail(HBSD_ERR_ARG, "H and S must have the same n and nnz");
        if (std::memcmp(H->row_ptr, Sm->row_ptr, (H->n + 1) * 8) != 0 ||
            std::memcmp(H->col_idx, Sm->col_idx, H->nnz * 4) != 0)
            return fail(HBSD_ERR_ARG, "H and S must share one sparsity pattern");
        for (int64_t e = 0; e < H->nnz; ++e)
            if (H->col_idx[e] < 0 || H->col_idx[e] >= H->n) return fail(HBSD_ERR_ARG, "column index out of range");
        if (!std::isfinite(opt->sigma_bar)) return fail(HBSD_ERR_ARG, "sigma_bar must be set");
        if (opt->precond < HBSD_PRECOND_HYBRID || opt->precond > HBSD_PRECOND_LOCAL)
            return fail(HBSD_ERR_ARG, "unknown preconditioner mode");
        if (opt->local_solver != HBSD_LOCAL_MINRES && opt->local_solver != HBSD_LOCAL_ONESTEP)
            return fail(HBSD_ERR_ARG, "hbsd_create: local_solver must be HBSD_LOCAL_MINRES or HBSD_LOCAL_ONESTEP");
        if (!lb->dof_node || lb->grid[0] <= 0 || lb->grid[1] <= 0 || lb->grid[2] <= 0)
            return fail(HBSD_ERR_ARG, "local blocks need dof_node and a positive grid");
        // complex Hermitian input: the real-equivalent pencil of size 2n (complex.cu)
        std::vector<int64_t> rp2;
        std::vector<int32_t> ci2, node2;
        std::vector<double> hv2, sv2;
        const int64_t* row_ptr = H->row_ptr;
        const int32_t* col_idx = H->col_idx;
        const double* hval = H->val;
        const double* sval = Sm->val;
        const int32_t* dof_node = lb->dof_node;
        int64_t n_dofs = H->n, nnz = H->nnz;
        if (H->is_complex) {
            for (int64_t e = 0; e < 2 * H->nnz; ++e)
                if (!std::isfinite(H->val[e]) || !std::isfinite(Sm->val[e])) return fail(HBSD_ERR_ARG, "non-finite value");
            complex_realify_csr(H->n, H->row_ptr, H->col_idx, H->val, Sm->val, lb->dof_node, rp2, ci2, hv2, sv2, node2);
            row_ptr = rp2.data();
            col_idx = ci2.data();
            hval = hv2.data();
            sval = sv2.data();
            dof_node = node2.data();
            n_dofs = 2 * H->n;
            nnz = 4 * H->nnz;
        }
        hbsd_handle* h = new hbsd_handle();
        Session* S = &h->s;
        S->n = n_dofs;
        S->nnz = nnz;
        S->opt = *opt;
        if (H->is_complex) {
            S->cplx = true;
            S->n_c = H->n;
            S->c_row_ptr.assign(H->row_ptr, H->row_ptr + H->n + 1);
        }
        {
            const char* e = std::getenv("HBSD_NO_DF64");
            S->opt_df64 = !(e && e[0] && e[0] != '0');
        }
        S->sigma0 = std::isnan(opt->sigma0) ? opt->sigma_bar : opt->sigma0;
        if (stream) {
            S->stream = (cudaStream_t)stream;
        } else {
            if (cudaStreamCreate(&S->stream) != cudaSuccess) {  // blocking: ordered with the legacy default stream
                delete h;
                return fail(HBSD_ERR_CUDA, "cudaStreamCreate failed");
            }
            S->own_stream = true;
        }
        int rc = sell_build(S->A, S->n, row_ptr, col_idx, hval, sval, S->sigma0);
        if (rc < 0) { hbsd_destroy(h); return rc; }
        S->h_sval.assign(sval, sval + S->nnz);
        std::vector<double> aval(S->nnz);
        for (int64_t e = 0; e < S->nnz; ++e) aval[e] = hval[e] - opt->sigma_bar * sval[e];
        if (opt->precond != HBSD_PRECOND_LOCAL) {   // the local-only mode has no global step
            rc = factor_build(S, S->F, S->n, row_ptr, col_idx, aval.data(), dof_node, lb->grid, S->stream);
            if (rc < 0) { std::string keep = g_last_error; hbsd_destroy(h); g_last_error = keep; return rc; }
            S->has_factor = true;
        }
        *out = h;
        return HBSD_OK;
    });
}

int hbsd_update_H(hbsd_handle* h, const double* H_val) {
    return guarded([&]() -> int {
        if (!h || !H_val) return fail(HBSD_ERR_ARG, "NULL argument");
        if (h->s.cplx) {   // 2 nnz interleaved (re, im) values of the complex pattern
            std::vector<double> v2;
            complex_realify_values(h->s.n_c, h->s.c_row_ptr.data(), H_val, v2);
            return sell_update_h(h->s.A, v2.data(), h->s.h_sval.data(), h->s.sigma0);
        }
        return sell_update_h(h->s.A, H_val, h->s.h_sval.data(), h->s.sigma0);
    });
}

void hbsd_destroy(hbsd_handle* h) {
    if (!h) return;
    if (h->s.stream) cudaStreamSynchronize(h->s.stream);
    if (h->s.own_stream && h->s.stream) cudaStreamDestroy(h->s.stream);
    delete h;
}

int64_t hbsd_n(const hbsd_handle* h) { return h ? (h->s.cplx ? h->s.n_c : h->s.n) : -1; }
int hbsd_is_complex(const hbsd_handle* h) { return h && h->s.cplx ? 1 : 0; }
double hbsd_sigma0(const hbsd_handle* h) { return h ? h->s.sigma0 : 0.0; }
void hbsd_get_stats(const hbsd_handle* h, hbsd_stats* st) {
    if (h && st) *st = h->s.stats;
}

static int m0_of(const Session& S, int nev) { return S.opt.m0 >= 0 ? S.opt.m0 : std::max(3, (nev + 9) / 10); }

extern "C++" {
int hbsd::block_width(const Session& s, int nev) { return (nev + m0_of(s, nev)) * (s.cplx ? 2 : 1); }
}

// Complex session: LABPSD on the real-equivalent pencil for 2 nev pairs from the realified start
// block Yb (2 n_c x 2 (nev + m0), ld ldy; columns J-paired), then the complex recovery.
static int complex_solve_block(Session* S, int nev, double tol, const double* Yb, int64_t ldy, double* lambda_dev,
                               double* X_dev, int64_t ldx, int* iters) {
    const int m0c = m0_of(*S, nev);
    S->launches = 0;
    auto t0 = std::chrono::steady_clock::now();
    int rc = labpsd_solve(S, 2 * nev, tol, Yb, ldy, nullptr, nullptr, 0, iters, 2 * m0c);
    if (rc >= 0) {
        const int rr = complex_recover(S, nev, lambda_dev, X_dev, ldx);
        if (rr < 0) rc = rr;
        else if (cudaStreamSynchronize(S->stream) != cudaSuccess) rc = fail(HBSD_ERR_CUDA, "complex recovery");
    }
    auto t1 = std::chrono::steady_clock::now();
    S->stats.t_solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    S->stats.gpu_launches = S->launches;
    return rc;
}

static int complex_solve_device(Session* S, int nev, double tol, const double* X0_dev, int64_t ldx0,
                                double* lambda_dev, double* X_dev, int64_t ldx, int* iters) {
    const int wc = nev + m0_of(*S, nev);
    if (wc > S->n_c) return fail(HBSD_ERR_ARG, "nev + m0 exceeds n");
    if (X_dev && ldx < nev) return fail(HBSD_ERR_ARG, "ldx < nev");
    if (2 * nev > 1024) return fail(HBSD_ERR_ARG, "complex input: nev <= 512");
    if (!X0_dev) {   // seed-normal complex block: real part from stream 2, imaginary part from stream 6
        const int64_t cnt = S->n_c * wc;
        std::vector<double> re(cnt), im(cnt), hx(2 * cnt);
        seed_normals(S->opt.seed, 2, cnt, re.data());
        seed_normals(S->opt.seed, 6, cnt, im.data());
        for (int64_t t = 0; t < cnt; ++t) { hx[2 * t] = re[t]; hx[2 * t + 1] = im[t]; }
        HBSD_TRY(S->cx_x0.alloc(hx.size()));
        HBSD_CUDA(cudaMemcpyAsync(S->cx_x0.p, hx.data(), hx.size() * 8, cudaMemcpyHostToDevice, S->stream));
        HBSD_CUDA(cudaStreamSynchronize(S->stream));
        X0_dev = S->cx_x0.p;
        ldx0 = wc;
    } else if (ldx0 < wc) {
        return fail(HBSD_ERR_ARG, "ldx0 < nev + m0");
    }
    const int64_t w = 2 * (int64_t)wc;
    HBSD_TRY(S->cx_y0.alloc((size_t)S->n * w));
    HBSD_TRY(complex_start_block(S, X0_dev, ldx0, wc, S->cx_y0.p, w));
    return complex_solve_block(S, nev, tol, S->cx_y0.p, w, lambda_dev, X_dev, ldx, iters);
}

int hbsd_solve_device(hbsd_handle* h, int nev, double tol, const double* X0_dev, int64_t ldx0, double* lambda_dev,
                      double* X_dev, int64_t ldx, int* iters, hbsd_stats* st) {
    return guarded([&]() -> int {
        if (!h || !lambda_dev) return fail(HBSD_ERR_ARG, "NULL handle or lambda");
        Session* S = &h->s;
        if (nev < 1 || !(tol > 0)) return fail(HBSD_ERR_ARG, "nev >= 1 and tol > 0 required");
        if (S->opt.precision != HBSD_PRECISION_FP64 && S->opt.precision != HBSD_PRECISION_MIXED)
            return fail(HBSD_ERR_ARG, "unknown precision mode");
        if (S->cplx) {
            const int rc = complex_solve_device(S, nev, tol, X0_dev, ldx0, lambda_dev, X_dev, ldx, iters);
            if (st) *st = S->stats;
            return rc;
        }
        if (X_dev && ldx < nev) return fail(HBSD_ERR_ARG, "ldx < nev");
        const int w = nev + m0_of(*S, nev);
        if (w > S->n) return fail(HBSD_ERR_ARG, "nev + m0 exceeds n");
        if (S->opt.precision != HBSD_PRECISION_FP64 && S->opt.precision != HBSD_PRECISION_MIXED)
            return fail(HBSD_ERR_ARG, "unknown precision mode");
        if (!X0_dev) {
            std::vector<double> hx((size_t)S->n * w);
            seed_normals(S->opt.seed, 2, (int64_t)hx.size(), hx.data());
            HBSD_TRY(S->io_x0.alloc(hx.size()));
            HBSD_CUDA(cudaMemcpyAsync(S->io_x0.p, hx.data(), hx.size() * 8, cudaMemcpyHostToDevice, S->stream));
            HBSD_CUDA(cudaStreamSynchronize(S->stream));   // hx is released at the end of this block
            X0_dev = S->io_x0.p;
            ldx0 = w;
        } else if (ldx0 < w) {
            return fail(HBSD_ERR_ARG, "ldx0 < nev + m0");
        }
        S->launches = 0;
        auto t0 = std::chrono::steady_clock::now();
        int rc = labpsd_solve(S, nev, tol, X0_dev, ldx0, lambda_dev, X_dev, ldx, iters);
        auto t1 = std::chrono::steady_clock::now();
        S->stats.t_solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        S->stats.gpu_launches = S->launches;
        if (st) *st = S->stats;
        return rc;
    });
}

// hbsd_solve on a complex session: X0 host n_c x (nev + m0) complex (interleaved re, im), X host
// n_c x nev complex; warm: the session's last real-equivalent block.
static int complex_solve_host(Session* S, int nev, double tol, const double* X0, int warm, double* lambda, double* X,
                              int* iters, hbsd_stats* st) {
    if (!(tol > 0)) return fail(HBSD_ERR_ARG, "tol > 0 required");
    if (S->opt.precision != HBSD_PRECISION_FP64 && S->opt.precision != HBSD_PRECISION_MIXED)
        return fail(HBSD_ERR_ARG, "unknown precision mode");
    const int wc = nev + m0_of(*S, nev);
    if (wc > S->n_c) return fail(HBSD_ERR_ARG, "nev + m0 exceeds n");
    if (2 * nev > 1024) return fail(HBSD_ERR_ARG, "complex input: nev <= 512");
    HBSD_TRY(S->io_lam.alloc(nev));
    if (X) HBSD_TRY(S->io_x.alloc((size_t)S->n_c * nev * 2));
    int rc;
    if (warm) {
        if (X0) return fail(HBSD_ERR_ARG, "warm start takes X0 = NULL");
        if (!S->psi_keep.p || S->keep_w != 2 * wc)
            return fail(HBSD_ERR_ARG, "no previous block of this width to warm-start from");
        HBSD_TRY(S->cx_y0.alloc(S->psi_keep.n));
        HBSD_CUDA(cudaMemcpyAsync(S->cx_y0.p, S->psi_keep.p, S->psi_keep.n * 8, cudaMemcpyDeviceToDevice, S->stream));
        rc = complex_solve_block(S, nev, tol, S->cx_y0.p, S->keep_ld, S->io_lam.p, X ? S->io_x.p : nullptr, nev, iters);
    } else {
        const double* x0p = nullptr;
        if (X0) {
            HBSD_TRY(S->io_x0.alloc((size_t)S->n_c * wc * 2));
            HBSD_CUDA(cudaMemcpyAsync(S->io_x0.p, X0, (size_t)S->n_c * wc * 16, cudaMemcpyHostToDevice, S->stream));
            x0p = S->io_x0.p;
        }
        rc = complex_solve_device(S, nev, tol, x0p, wc, S->io_lam.p, X ? S->io_x.p : nullptr, nev, iters);
    }
    if (st) *st = S->stats;
    if (rc < 0) return rc;
    HBSD_CUDA(cudaMemcpyAsync(lambda, S->io_lam.p, nev * 8, cudaMemcpyDeviceToHost, S->stream));
    if (X) HBSD_CUDA(cudaMemcpyAsync(X, S->io_x.p, (size_t)S->n_c * nev * 16, cudaMemcpyDeviceToHost, S->stream));
    HBSD_CUDA(cudaStreamSynchronize(S->stream));
    return rc;
}

int hbsd_solve(hbsd_handle* h, int nev, double tol, const double* X0, int warm, double* lambda, double* X, int* iters,
               hbsd_stats* st) {
    return guarded([&]() -> int {
        if (!h || !lambda) return fail(HBSD_ERR_ARG, "NULL handle or lambda");
        Session* S = &h->s;
        if (nev < 1) return fail(HBSD_ERR_ARG, "nev >= 1 required");
        if (S->cplx) return complex_solve_host(S, nev, tol, X0, warm, lambda, X, iters, st);
        const int w = nev + m0_of(*S, nev);
        if (w > S->n) return fail(HBSD_ERR_ARG, "nev + m0 exceeds n");
        // host <-> device traffic goes through session-resident buffers on the session's stream
        // (no allocation after the first solve of a size, no legacy-stream synchronisation)
        const double* x0p = nullptr;
        int64_t ld0 = w;
        if (warm) {
            if (X0) return fail(HBSD_ERR_ARG, "warm start takes X0 = NULL");
            if (!S->psi_keep.p || S->keep_w != w) return fail(HBSD_ERR_ARG, "no previous block of this width to warm-start from");
            // the solve overwrites psi_keep; start from a copy
            HBSD_TRY(S->io_x0.alloc(S->psi_keep.n));
            HBSD_CUDA(cudaMemcpyAsync(S->io_x0.p, S->psi_keep.p, S->psi_keep.n * 8, cudaMemcpyDeviceToDevice, S->stream));
            x0p = S->io_x0.p;
            ld0 = S->keep_ld;
        } else if (X0) {
            HBSD_TRY(S->io_x0.alloc((size_t)S->n * w));
            HBSD_CUDA(cudaMemcpyAsync(S->io_x0.p, X0, (size_t)S->n * w * 8, cudaMemcpyHostToDevice, S->stream));
            x0p = S->io_x0.p;
        }
        HBSD_TRY(S->io_lam.alloc(nev));
        if (X) HBSD_TRY(S->io_x.alloc((size_t)S->n * nev));
        int rc = hbsd_solve_device(h, nev, tol, x0p, ld0, S->io_lam.p, X ? S->io_x.p : nullptr, nev, iters, st);
        if (rc < 0) return rc;
        HBSD_CUDA(cudaMemcpyAsync(lambda, S->io_lam.p, nev * 8, cudaMemcpyDeviceToHost, S->stream));
        if (X) HBSD_CUDA(cudaMemcpyAsync(X, S->io_x.p, (size_t)S->n * nev * 8, cudaMemcpyDeviceToHost, S->stream));
        HBSD_CUDA(cudaStreamSynchronize(S->stream));
        return rc;
    });
}

int hbsd_probe_barrier_timeout(double limit_s, void* stream) {
    return guarded([&]() -> int {
        return barrier_timeout_probe(limit_s, (cudaStream_t)stream);
    });
}

int hbsd_seed_normals(uint64_t seed, uint64_t stream, int64_t count, double* out) {
    return guarded([&]() -> int {
        if (!out || count < 0) return fail(HBSD_ERR_ARG, "bad arguments");
        seed_normals(seed, stream, count, out);
        return HBSD_OK;
    });
}

// ---- step-level entry points ---------------------------------------------------------------
// A row-major block of `width` columns needs ld >= width (kernels would read past a row).
static bool ld_ok(int64_t ld, int64_t width) { return width <= 0 || ld >= width; }

int hbsd_res_stalled(const double* hist, int len, int mark, int win, double below) {
    return guarded([&]() -> int {
        if (len < 0 || mark < 0 || mark > len || win < 1 || (len > 0 && !hist)) return fail(HBSD_ERR_ARG, "bad arguments");
        return res_stalled(hist, (size_t)len, (size_t)mark, win, below) ? 1 : 0;
    });
}

int hbsd_res_history(const hbsd_handle* h, double* out, int cap) {
    return guarded([&]() -> int {
        if (!h || cap < 0 || (cap > 0 && !out)) return fail(HBSD_ERR_ARG, "bad arguments");
        const std::vector<double>& v = h->s.res_hist;
        for (int i = 0; i < cap && i < (int)v.size(); ++i) out[i] = v[i];
        return (int)v.size();
    });
}

int hbsd_set_nonlocal(hbsd_handle* h, int k, const double* F, int64_t ldf, const double* G) {
    return guarded([&]() -> int {
        if (!h) return fail(HBSD_ERR_ARG, "bad arguments");
        if (h->s.cplx && k > 0) return fail(HBSD_ERR_UNSUPPORTED, "nonlocal term on a complex session");
        HBSD_CUDA(cudaStreamSynchronize(h->s.stream));   // no work of this session reads the old term any more
        return nl_set(&h->s, k, F, ldf, G);
    });
}

int hbsd_spmm_pair(hbsd_handle* h, const double* X, int64_t ldx, int k, double* HX, int64_t ldhx, double* SX,
                   int64_t ldsx) {
    return guarded([&]() -> int {
        if (!h || !X || !HX || !SX || k < 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldx, k) || !ld_ok(ldhx, k) || !ld_ok(ldsx, k)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        return spmm_pair<double>(&h->s, h->s.A, X, ldx, k, HX, ldhx, SX, ldsx, h->s.stream);
    });
}

int hbsd_spmm_pair_df64(hbsd_handle* h, const double* X, int64_t ldx, int k, double* HX, int64_t ldhx, double* SX,
                        int64_t ldsx) {
    return guarded([&]() -> int {
        if (!h || !X || !HX || !SX || k < 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldx, k) || !ld_ok(ldhx, k) || !ld_ok(ldsx, k)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        return spmm_pair_df64(&h->s, h->s.A, X, ldx, k, HX, ldhx, SX, ldsx, h->s.stream);
    });
}

int hbsd_spmm_pair_f32(hbsd_handle* h, const float* X, int64_t ldx, int k, float* HX, int64_t ldhx, float* SX,
                       int64_t ldsx) {
    return guarded([&]() -> int {
        if (!h || !X || !HX || !SX || k < 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldx, k) || !ld_ok(ldhx, k) || !ld_ok(ldsx, k)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        return spmm_pair<float>(&h->s, h->s.A, X, ldx, k, HX, ldhx, SX, ldsx, h->s.stream);
    });
}

int hbsd_precond_apply_f32(hbsd_handle* h, const float* R, int64_t ldr, int k, float* P, int64_t ldp) {
    return guarded([&]() -> int {
        if (!h || !R || !P || k < 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldr, k) || !ld_ok(ldp, k)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        HBSD_TRY(factor_make_fp32(h->s.F, h->s.A.dscale.p, h->s.stream));
        HBSD_TRY(factor_solve<float>(&h->s, h->s.F, R, ldr, k, P, ldp, h->s.stream));
        return nl_smw_correct<float>(&h->s, P, ldp, k, h->s.stream);
    });
}

int hbsd_dscale(const hbsd_handle* h, double* d_host) {
    return guarded([&]() -> int {
        if (!h || !d_host) return fail(HBSD_ERR_ARG, "bad arguments");
        std::memcpy(d_host, h->s.A.h_dscale.data(), h->s.n * sizeof(double));
        return HBSD_OK;
    });
}

int hbsd_spmm_shifted(hbsd_handle* h, const double* X, int64_t ldx, int k, const double* e, double* Y, int64_t ldy) {
    return guarded([&]() -> int {
        if (!h || !X || !e || !Y || k < 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldx, k) || !ld_ok(ldy, k)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        return spmm_shifted<double>(&h->s, h->s.A, X, ldx, k, e, Y, ldy, h->s.stream);
    });
}

int hbsd_residual(hbsd_handle* h, const double* PsiH, int64_t ldh, const double* PsiS, int64_t lds, const double* E,
                  int m, double* R, int64_t ldr, double* res) {
    return guarded([&]() -> int {
        if (!h || !PsiH || !PsiS || !E || !res || m <= 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldh, m) || !ld_ok(lds, m) || (R && !ld_ok(ldr, m))) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        Session* S = &h->s;
        HBSD_TRY(S->ws.alloc((size_t)304 * 2 * m + 64));
        return residual<double>(S, PsiH, ldh, PsiS, lds, E, m, R, ldr, S->n, res, nullptr, S->stream);
    });
}

int hbsd_precond_apply(hbsd_handle* h, const double* R, int64_t ldr, int k, double* P, int64_t ldp) {
    return guarded([&]() -> int {
        if (!h || !R || !P || k < 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldr, k) || !ld_ok(ldp, k)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        HBSD_TRY(factor_solve<double>(&h->s, h->s.F, R, ldr, k, P, ldp, h->s.stream));
        return nl_smw_correct<double>(&h->s, P, ldp, k, h->s.stream);
    });
}

int hbsd_minres(hbsd_handle* h, const double* R, int64_t ldr, const double* e, int k, double eta, int max_minres,
                double* P, int64_t ldp, int* steps) {
    return guarded([&]() -> int {
        if (!h || !R || !e || !P || k < 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldr, k) || !ld_ok(ldp, k)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        Session* S = &h->s;
        HBSD_TRY(S->ws.alloc((size_t)304 * 2 * std::max(k, 1) + 64));
        return minres_batch<double>(S, R, ldr, e, k, eta, max_minres, P, ldp, steps, nullptr, S->stream);
    });
}

int hbsd_onestep(hbsd_handle* h, const double* R, int64_t ldr, const double* e, int k, double eta, int max_steps,
                 double* P, int64_t ldp, int* steps) {
    return guarded([&]() -> int {
        if (!h || !R || !e || !P || k < 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldr, k) || !ld_ok(ldp, k)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        Session* S = &h->s;
        return minres_batch<double>(S, R, ldr, e, k, eta, max_steps, P, ldp, steps, nullptr, S->stream,
                                    HBSD_LOCAL_ONESTEP);
    });
}

// Step-level calls without a session run on a temporary one that only carries scratch.
static Session* scratch_session() {
    static thread_local Session* s = nullptr;
    if (!s) s = new Session();
    return s;
}

int hbsd_gram(const double* Z, int64_t ldz, const double* ZH, int64_t ldzh, const double* ZS, int64_t ldzs, int64_t n,
              int q, double* HR, double* SR, void* stream) {
    return guarded([&]() -> int {
        if (!Z || !ZH || !ZS || !HR || !SR || n <= 0 || q <= 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldz, q) || !ld_ok(ldzh, q) || !ld_ok(ldzs, q)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        Session* S = scratch_session();
        const int tiles = ceil_div(q, 32);
        HBSD_TRY(S->ws.alloc((size_t)2 * 1024 * (1216 + tiles * tiles) + 1024));
        return gram2<double>(S, Z, ldz, q, nullptr, 0, 0, ZH, ldzh, nullptr, 0, ZS, ldzs, nullptr, 0, n, HR, SR,
                             (cudaStream_t)stream);
    });
}

int hbsd_gram_noalloc(const double* Z, int64_t ldz, const double* ZH, int64_t ldzh, const double* ZS,
                      int64_t ldzs, int64_t n, int q, double* HR, double* SR, void* stream) {
    return guarded([&]() -> int {
        if (!Z || !ZH || !ZS || !HR || !SR) return fail(HBSD_ERR_ARG, "bad arguments");
        // the scratch limit is reported before any other size check, whatever the ld
        if (q > GRAM_NOALLOC_MAX_Q)
            return fail(HBSD_ERR_ARG, "gram_noalloc: q = " + std::to_string(q) +
                                          " exceeds the static scratch (2 q^2 <= 2^21 doubles, q <= 1024)");
        if (!ld_ok(ldz, q) || !ld_ok(ldzh, q) || !ld_ok(ldzs, q)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        return gram_noalloc(Z, ldz, ZH, ldzh, ZS, ldzs, n, q, HR, SR, (cudaStream_t)stream);
    });
}

int hbsd_update_oz(const double* Z0, int64_t ld0, int q0, const double* Z1, int64_t ld1, int q1, int64_t n,
                   const double* W, int k, double* Y, int64_t ldy, void* stream) {
    return guarded([&]() -> int {
        if (!Z0 || !W || !Y || (q1 > 0 && !Z1)) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ld0, q0) || (q1 > 0 && !ld_ok(ld1, q1)) || !ld_ok(ldy, k))
            return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        return update_oz(scratch_session(), Z0, ld0, q0, Z1, ld1, q1, n, W, k, Y, ldy, (cudaStream_t)stream);
    });
}

int hbsd_rayleigh_ritz(const double* HR, const double* SR, int q, int k, double* theta, double* W, int* info,
                       void* stream) {
    return guarded([&]() -> int {
        if (!HR || !SR || !theta || !W) return fail(HBSD_ERR_ARG, "bad arguments");
        Session* S = scratch_session();
        int hinfo[2] = {0, 0};
        int rc = rayleigh_ritz_cluster(S, HR, SR, q, k, theta, W, hinfo, (cudaStream_t)stream);
        if (info) {
            int tmp[2] = {hinfo[0], hinfo[1]};
            cudaError_t e = cudaMemcpy(info, tmp, sizeof(tmp), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail(HBSD_ERR_CUDA, cudaGetErrorString(e));
        }
        return rc;
    });
}

int hbsd_update(double* Z, int64_t ldz, int64_t n, int q, const double* W, int k, void* stream) {
    return guarded([&]() -> int {
        if (!Z || !W || n <= 0 || q <= 0 || k <= 0 || k > q) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldz, q)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        return update2<double>(scratch_session(), Z, ldz, q, nullptr, 0, 0, n, W, k, (cudaStream_t)stream);
    });
}

int hbsd_gram_df64(const double* Z, int64_t ldz, const double* ZH, int64_t ldzh, const double* ZS, int64_t ldzs,
                   int64_t n, int q, double* HR, double* SR, void* stream) {
    return guarded([&]() -> int {
        if (!Z || !ZH || !ZS || !HR || !SR || n <= 0 || q <= 0) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldz, q) || !ld_ok(ldzh, q) || !ld_ok(ldzs, q)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        return gram2_df64(scratch_session(), Z, ldz, q, nullptr, 0, 0, ZH, ldzh, nullptr, 0, ZS, ldzs, nullptr, 0, n, HR,
                          SR, (cudaStream_t)stream);
    });
}

int hbsd_update_df64(double* Z, int64_t ldz, int64_t n, int q, const double* W, int k, void* stream) {
    return guarded([&]() -> int {
        if (!Z || !W || n <= 0 || q <= 0 || k <= 0 || k > q) return fail(HBSD_ERR_ARG, "bad arguments");
        if (!ld_ok(ldz, q)) return fail(HBSD_ERR_ARG, "leading dimension below the block width");
        return update2_df64(scratch_session(), Z, ldz, q, nullptr, 0, 0, n, W, k, (cudaStream_t)stream, true);
    });
}

}  // extern "C"
