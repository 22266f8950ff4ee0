// Step 6(b) of LABPSD: locally accelerated refinement (Sec. 3 hybrid scheme, Sec. 4, Eq. indls).
// For each refined column j, MINRES (Paige & Saunders 1975) on the Hermitian indefinite system
// (H - eps_j S) p = -r_j started from the globally preconditioned p_j, stopped when the
// recurrence residual estimate drops to eta ||r_j|| (Eq. approxp) or after max_minres steps.
//
// All refined columns advance in lockstep: one shifted SpMM per step serves every column still
// iterating (gathered into a compact block once some have stopped), the Lanczos inner products
// are deterministic two-pass column reductions, and the Givens / QR recurrences are per-column
// scalars updated by one thread per column.  A column that has met its tolerance keeps its
// iterate and stops updating.
#include <cmath>

#include "common.h"

namespace hbsd {

struct MrCol {
    double beta_old, c_prev, s_prev, c_pp, s_pp, phibar, tol;
    double alpha, beta_next, phi, gamma, delta, eps;
    int active;     // still iterating
    int upd;        // this step updates the iterate
    int cont;       // a next Lanczos vector is needed
    int steps;
};

template <class T>
int col_dots(Session* s, const T* A, int64_t lda, const T* B, int64_t ldb, int64_t n, int k, double* out,
             cudaStream_t st);

namespace {

// V = -R - U  (r0 = b - A x0 with b = -r_j)
template <class T>
__global__ void k_mr_r0(const T* __restrict__ R, int64_t ldr, const T* __restrict__ U, int64_t ldu,
                        T* __restrict__ V, int64_t ldv, int64_t n, int k) {
    const int64_t total = n * k;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / k;
        const int j = (int)(idx % k);
        V[i * ldv + j] = -R[i * ldr + j] - U[i * ldu + j];
    }
}

__global__ void k_mr_init(MrCol* __restrict__ col, const double* __restrict__ rr, const double* __restrict__ bb,
                          int k, double eta, int maxit, int* __restrict__ any) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    MrCol c{};
    const double beta = sqrt(rr[j]);
    c.tol = eta * sqrt(bb[j]);
    c.beta_old = 0.0;
    c.c_prev = 1.0; c.s_prev = 0.0; c.c_pp = 1.0; c.s_pp = 0.0;
    c.phibar = beta;
    c.beta_next = beta;         // used to normalise v_1
    c.steps = 0;
    c.active = (beta > c.tol && maxit > 0) ? 1 : 0;
    c.upd = 0;
    c.cont = c.active;
    col[j] = c;
    if (c.active) atomicOr(any, 1);
}

// v_1 = r0 / beta_1; v_0 = w_0 = w_{-1} = 0
template <class T>
__global__ void k_mr_start(const MrCol* __restrict__ col, T* __restrict__ V, T* __restrict__ Vp, T* __restrict__ Wp,
                           T* __restrict__ Wpp, int64_t ld, int64_t n, int k) {
    const int64_t total = n * k;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / k;
        const int j = (int)(idx % k);
        const int64_t o = i * ld + j;
        if (col[j].active) V[o] = (T)((double)V[o] / col[j].beta_next);
        Vp[o] = T(0); Wp[o] = T(0); Wpp[o] = T(0);
    }
}

__global__ void k_mr_set_alpha(MrCol* __restrict__ col, const double* __restrict__ a, int k) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) col[j].alpha = a[j];
}

// U = U - alpha V - beta_old Vp
template <class T>
__global__ void k_mr_lanczos(const MrCol* __restrict__ col, T* __restrict__ U, const T* __restrict__ V,
                             const T* __restrict__ Vp, int64_t ld, int64_t n, int k) {
    const int64_t total = n * k;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / k;
        const int j = (int)(idx % k);
        if (!col[j].active) continue;
        const int64_t o = i * ld + j;
        U[o] = U[o] - (T)col[j].alpha * V[o] - (T)col[j].beta_old * Vp[o];
    }
}

// Givens update of the QR factorisation of the Lanczos tridiagonal, one thread per column.
__global__ void k_mr_scalars(MrCol* __restrict__ col, const double* __restrict__ uu, int k, int step,
                             int* __restrict__ any) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    MrCol c = col[j];
    c.upd = 0;
    c.cont = 0;
    if (c.active) {
        const double beta_next = sqrt(uu[j]);
        const double eps = c.s_pp * c.beta_old;
        const double dbar = c.c_pp * c.beta_old;
        const double delta = c.c_prev * dbar + c.s_prev * c.alpha;
        const double gbar = -c.s_prev * dbar + c.c_prev * c.alpha;
        const double gamma = hypot(gbar, beta_next);
        if (gamma == 0.0) {
            c.active = 0;
        } else {
            const double ck = gbar / gamma, sk = beta_next / gamma;
            c.phi = ck * c.phibar;
            c.phibar = -sk * c.phibar;
            c.gamma = gamma;
            c.delta = delta;
            c.eps = eps;
            c.steps = step;
            c.upd = 1;
            const bool done = fabs(c.phibar) <= c.tol || beta_next == 0.0;
            c.cont = done ? 0 : 1;
            c.beta_next = beta_next;
            c.beta_old = beta_next;
            c.c_pp = c.c_prev; c.s_pp = c.s_prev;
            c.c_prev = ck; c.s_prev = sk;
            if (done) c.active = 0;
        }
    }
    col[j] = c;
    if (c.active) atomicOr(any, 1);
}

// w = (v - delta w_prev - eps w_pp) / gamma;  x += phi w;  shift w;  v_prev = v; v = u / beta
template <class T>
__global__ void k_mr_vectors(const MrCol* __restrict__ col, T* __restrict__ X, int64_t ldx, T* __restrict__ V,
                             T* __restrict__ Vp, const T* __restrict__ U, T* __restrict__ Wp, T* __restrict__ Wpp,
                             int64_t ld, int64_t n, int k) {
    const int64_t total = n * k;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / k;
        const int j = (int)(idx % k);
        const MrCol& c = col[j];
        if (!c.upd) continue;
        const int64_t o = i * ld + j;
        const double v = (double)V[o];
        const double w = (v - c.delta * (double)Wp[o] - c.eps * (double)Wpp[o]) / c.gamma;
        X[i * ldx + j] = (T)((double)X[i * ldx + j] + c.phi * w);
        Wpp[o] = Wp[o];
        Wp[o] = (T)w;
        if (c.cont) {
            Vp[o] = V[o];
            V[o] = (T)((double)U[o] / c.beta_next);
        }
    }
}

__global__ void k_mr_steps(const MrCol* __restrict__ col, int k, int* __restrict__ steps) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) steps[j] = col[j].steps;
}

inline int grid_for(int64_t work) {
    return (int)std::min<int64_t>(std::max<int64_t>(1, (work + 255) / 256), 4096);
}

__global__ void k_mr_active(const MrCol* __restrict__ col, int k, int* __restrict__ flags) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) flags[j] = col[j].active;
}

template <class T>
__global__ void k_mr_gather(const T* __restrict__ V, int64_t ld, const T* __restrict__ e, const int* __restrict__ idx,
                            int na, int64_t n, T* __restrict__ Vc, int64_t ldc, T* __restrict__ ec) {
    const int64_t total = n * na;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / na;
        const int j = (int)(t % na);
        Vc[i * ldc + j] = V[i * ld + idx[j]];
        if (i == 0) ec[j] = e[idx[j]];
    }
}

template <class T>
__global__ void k_mr_scatter(const T* __restrict__ Uc, int64_t ldc, const int* __restrict__ idx, int na, int64_t n,
                             T* __restrict__ U, int64_t ld) {
    const int64_t total = n * na;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / na;
        const int j = (int)(t % na);
        U[i * ld + idx[j]] = Uc[i * ldc + j];
    }
}

}  // namespace

static int k_active_flags(Session* s, const MrCol* col, int k, int* flags, cudaStream_t st) {
    k_mr_active<<<ceil_div(k, 128), 128, 0, st>>>(col, k, flags);
    HBSD_LAUNCHED(s);
    return 0;
}

template <class T> static DBuf<T>& mr_vecs(Session* s);
template <> DBuf<double>& mr_vecs<double>(Session* s) { return s->mr_d; }
template <> DBuf<float>& mr_vecs<float>(Session* s) { return s->mr_f; }
// compact block of the active columns (V, U and the shifts), after the 5 state blocks
template <class T>
static T* mr_compact(Session* s) { return mr_vecs<T>(s).p + 5 * s->n * s->mr_ld; }

// X (n x k, ldx): start vectors on entry, refined vectors on exit.  R: residual columns.
// e: shifts eps_j relative to sigma0 (device, k entries of T).  steps: device ints (nullable).
template <class T>
int minres_batch(Session* s, const T* R, int64_t ldr, const T* e, int k, double eta, int maxit, T* X,
                 int64_t ldx, int* steps, int64_t* total_steps, cudaStream_t st) {
    if (k <= 0) return 0;
    const int64_t n = s->n;
    const int64_t ld = round_up(k, 4);
    HBSD_TRY(mr_vecs<T>(s).alloc((size_t)7 * n * ld + ld));
    HBSD_TRY(s->mr_idx.alloc(k));
    s->mr_ld = ld;
    HBSD_TRY(s->mr_col.alloc((size_t)k * sizeof(MrCol) / sizeof(double) + 1));
    HBSD_TRY(s->mr_red.alloc((size_t)3 * k));
    HBSD_TRY(s->mr_any.alloc(1));
    HBSD_TRY(s->mr_steps.alloc(k));
    MrCol* colp = reinterpret_cast<MrCol*>(s->mr_col.p);
    int* anyp = s->mr_any.p;
    T* V = mr_vecs<T>(s).p;
    T* Vp = V + n * ld;
    T* U = Vp + n * ld;
    T* Wp = U + n * ld;
    T* Wpp = Wp + n * ld;
    double* rr = s->mr_red.p;
    double* bb = rr + k;
    double* al = bb + k;
    const int g = grid_for(n * k);
    // r0 = -R - A X
    HBSD_TRY(spmm_shifted<T>(s, s->A, X, ldx, k, e, U, ld, st));
    k_mr_r0<T><<<g, 256, 0, st>>>(R, ldr, U, ld, V, ld, n, k);
    HBSD_LAUNCHED(s);
    HBSD_TRY(col_dots<T>(s, V, ld, V, ld, n, k, rr, st));
    HBSD_TRY(col_dots<T>(s, R, ldr, R, ldr, n, k, bb, st));
    HBSD_CUDA(cudaMemsetAsync(anyp, 0, sizeof(int), st));
    k_mr_init<<<ceil_div(k, 128), 128, 0, st>>>(colp, rr, bb, k, eta, maxit, anyp);
    HBSD_LAUNCHED(s);
    k_mr_start<T><<<g, 256, 0, st>>>(colp, V, Vp, Wp, Wpp, ld, n, k);
    HBSD_LAUNCHED(s);
    s->stats.minres_spmm_cols += k;
    // columns still iterating; the shifted SpMM of a step runs on those only (gathered into a
    // compact block), the cheap memory-bound kernels run on all columns with masks
    std::vector<int> act(k), flags(k);
    for (int j = 0; j < k; ++j) act[j] = j;
    HBSD_TRY(k_active_flags(s, colp, k, s->mr_steps.p, st));
    HBSD_CUDA(cudaMemcpyAsync(flags.data(), s->mr_steps.p, k * sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    act.clear();
    for (int j = 0; j < k; ++j)
        if (flags[j]) act.push_back(j);
    for (int step = 1; step <= maxit && !act.empty(); ++step) {
        const int na = (int)act.size();
        if (na == k) {
            HBSD_TRY(spmm_shifted<T>(s, s->A, V, ld, k, e, U, ld, st));
        } else {
            const int64_t ldc = round_up(na, 4);
            HBSD_CUDA(cudaMemcpyAsync(s->mr_idx.p, act.data(), na * sizeof(int), cudaMemcpyHostToDevice, st));
            T* Vc = mr_compact<T>(s);
            T* Uc = Vc + n * ldc;
            T* ec = Uc + n * ldc;
            k_mr_gather<T><<<grid_for(n * na), 256, 0, st>>>(V, ld, e, s->mr_idx.p, na, n, Vc, ldc, ec);
            HBSD_LAUNCHED(s);
            HBSD_TRY(spmm_shifted<T>(s, s->A, Vc, ldc, na, ec, Uc, ldc, st));
            k_mr_scatter<T><<<grid_for(n * na), 256, 0, st>>>(Uc, ldc, s->mr_idx.p, na, n, U, ld);
            HBSD_LAUNCHED(s);
        }
        s->stats.minres_spmm_cols += na;
        HBSD_TRY(col_dots<T>(s, V, ld, U, ld, n, k, al, st));
        k_mr_set_alpha<<<ceil_div(k, 128), 128, 0, st>>>(colp, al, k);
        HBSD_LAUNCHED(s);
        k_mr_lanczos<T><<<g, 256, 0, st>>>(colp, U, V, Vp, ld, n, k);
        HBSD_LAUNCHED(s);
        HBSD_TRY(col_dots<T>(s, U, ld, U, ld, n, k, rr, st));
        HBSD_CUDA(cudaMemsetAsync(anyp, 0, sizeof(int), st));
        k_mr_scalars<<<ceil_div(k, 128), 128, 0, st>>>(colp, rr, k, step, anyp);
        HBSD_LAUNCHED(s);
        k_mr_vectors<T><<<g, 256, 0, st>>>(colp, X, ldx, V, Vp, U, Wp, Wpp, ld, n, k);
        HBSD_LAUNCHED(s);
        HBSD_TRY(k_active_flags(s, colp, k, s->mr_steps.p, st));
        HBSD_CUDA(cudaMemcpyAsync(flags.data(), s->mr_steps.p, k * sizeof(int), cudaMemcpyDeviceToHost, st));
        HBSD_CUDA(cudaStreamSynchronize(st));
        act.clear();
        for (int j = 0; j < k; ++j)
            if (flags[j]) act.push_back(j);
    }
    if (steps || total_steps) {
        int* sp = steps ? steps : s->mr_steps.p;
        k_mr_steps<<<ceil_div(k, 128), 128, 0, st>>>(colp, k, sp);
        HBSD_LAUNCHED(s);
        if (total_steps) {
            std::vector<int> h(k);
            HBSD_CUDA(cudaMemcpyAsync(h.data(), sp, k * sizeof(int), cudaMemcpyDeviceToHost, st));
            HBSD_CUDA(cudaStreamSynchronize(st));
            int64_t tot = 0;
            for (int v : h) tot += v;
            *total_steps = tot;
        }
    }
    return 0;
}

template int minres_batch<double>(Session*, const double*, int64_t, const double*, int, double, int, double*,
                                  int64_t, int*, int64_t*, cudaStream_t);
template int minres_batch<float>(Session*, const float*, int64_t, const float*, int, double, int, float*,
                                 int64_t, int*, int64_t*, cudaStream_t);

}  // namespace hbsd
