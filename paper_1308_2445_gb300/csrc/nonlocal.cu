// Nonlocal low-rank term of the Hamiltonian, H = H_loc + F G F^T (Sec. 4, Eq. fgf), and the
// Sherman-Morrison-Woodbury form of the global preconditioner (Sec. 4, steps 1-6):
//   setup, once per factor and precision:  Fh = -(H_loc - eps_bar S)^{-1} F = -Fhat     (step 1)
//                                          T  = I + G F^T Fhat                          (steps 2-3)
//                                          M  = T^{-1} G                                (step 4)
//   every application:                     P  = -(H_loc - eps_bar S)^{-1} R             (step 5)
//                                          P -= Fhat (M (F^T P))                        (step 6)
// Step 4 stores F := F G T^{-H}; step 6 then needs (F G T^{-H})^T P = T^{-1} G F^T P = M F^T P,
// so holding M instead keeps F sparse (G symmetric).
// Every product with H adds F (G (F^T X)): F^T X as partial sums over work items (at most
// NL_ITEM entries of one projector each) reduced in a fixed order, then G, then F by rows.
// Everything is deterministic: fixed summation orders, no atomics.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"

namespace hbsd {

namespace {

constexpr int NL_ITEM = 128;     // F entries per F^T X work item
constexpr int NL_KMAX = 4096;    // projectors (the reduction keeps one column of F^T X in shared memory)

inline int grid_for(int64_t work, int threads = 256) {
    const int64_t g = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

// part[it * ldp + j] = sum over the entries e of item it of val[e] * X[row[e], j]
template <class T>
__global__ void k_nl_ft_partial(const int64_t* __restrict__ item_e, const int32_t* __restrict__ row,
                                const T* __restrict__ val, const T* __restrict__ X, int64_t ldx, int w,
                                T* __restrict__ part, int64_t ldp) {
    const int it = blockIdx.x;
    const int64_t e0 = item_e[2 * it], e1 = item_e[2 * it + 1];
    for (int j = threadIdx.x; j < w; j += blockDim.x) {
        T a0 = T(0), a1 = T(0);
        int64_t e = e0;
        for (; e + 1 < e1; e += 2) {
            a0 = fma(val[e], X[(int64_t)row[e] * ldx + j], a0);
            a1 = fma(val[e + 1], X[(int64_t)row[e + 1] * ldx + j], a1);
        }
        if (e < e1) a0 = fma(val[e], X[(int64_t)row[e] * ldx + j], a0);
        part[(int64_t)it * ldp + j] = a0 + a1;
    }
}

// Z[l, j] = sum_e mval[e] * z[mcol[e]] over row l of M, z = F^T X(:, j) summed from the items in
// order; one block per column j.
template <class T, class TO>
__global__ void k_nl_reduce(const int32_t* __restrict__ item_ptr, const T* __restrict__ part, int64_t ldp, int k,
                            const int32_t* __restrict__ mptr, const int32_t* __restrict__ mcol,
                            const double* __restrict__ mval, TO* __restrict__ Z, int64_t ldz) {
    extern __shared__ double zs[];
    const int j = blockIdx.x;
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
        double s = 0.0;
        for (int it = item_ptr[l]; it < item_ptr[l + 1]; ++it) s += (double)part[(int64_t)it * ldp + j];
        zs[l] = s;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
        double s = 0.0;
        for (int e = mptr[l]; e < mptr[l + 1]; ++e) s = fma(mval[e], zs[mcol[e]], s);
        Z[(int64_t)l * ldz + j] = (TO)s;
    }
}

// Y[i, j] += sum_e val[e] * Z[col[e], j] over row i of F, for the rows with entries
template <class T>
__global__ void k_nl_apply(const int32_t* __restrict__ frows, int64_t nfr, const int64_t* __restrict__ rptr,
                           const int32_t* __restrict__ col, const T* __restrict__ val, const T* __restrict__ Z,
                           int64_t ldz, int w, T* __restrict__ Y, int64_t ldy) {
    const int64_t total = nfr * w;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / w;
        const int j = (int)(t - r * w);
        const int64_t i = frows[r];
        T s = T(0);
        for (int64_t e = rptr[i]; e < rptr[i + 1]; ++e) s = fma(val[e], Z[(int64_t)col[e] * ldz + j], s);
        Y[i * ldy + j] += s;
    }
}

// P[i, j] += sum_l Fh[i, l] * Z[l, j]   (step 6 with Fh = -Fhat)
template <class T>
__global__ void k_nl_lowrank_add(const T* __restrict__ Fh, int64_t ldf, int k, const T* __restrict__ Z, int64_t ldz,
                                 int64_t n, int p, T* __restrict__ P, int64_t ldp) {
    const int64_t total = n * p;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / p;
        const int j = (int)(t - i * p);
        const T* f = Fh + i * ldf;
        T s = T(0);
        for (int l = 0; l < k; ++l) s = fma(f[l], Z[(int64_t)l * ldz + j], s);
        P[i * ldp + j] += s;
    }
}

// D[i, col[e]] = val[e] (D zeroed before)
template <class T>
__global__ void k_nl_densify(const int32_t* __restrict__ frows, int64_t nfr, const int64_t* __restrict__ rptr,
                             const int32_t* __restrict__ col, const T* __restrict__ val, T* __restrict__ D,
                             int64_t ldd) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nfr; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = frows[r];
        for (int64_t e = rptr[i]; e < rptr[i + 1]; ++e) D[i * ldd + col[e]] = val[e];
    }
}

// FP32 copies of D F in both orders (D = diag(S)^{-1/2}, the scaling of the FP32 pencil)
__global__ void k_nl_scale_cols(const int32_t* __restrict__ crow, const double* __restrict__ cval, int64_t nnz,
                                const double* __restrict__ d, float* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (float)(cval[e] * d[crow[e]]);
}
__global__ void k_nl_scale_rows(const int32_t* __restrict__ frows, int64_t nfr, const int64_t* __restrict__ rptr,
                                const double* __restrict__ rval, const double* __restrict__ d, float* __restrict__ out) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nfr; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = frows[r];
        for (int64_t e = rptr[i]; e < rptr[i + 1]; ++e) out[e] = (float)(rval[e] * d[i]);
    }
}

// A = I - Z (Z = G F^T Fh, k x k, ld ldz) and B = G dense; one block
__global__ void k_nl_make_t(const double* __restrict__ Z, int64_t ldz, int k, const int32_t* __restrict__ gptr,
                            const int32_t* __restrict__ gcol, const double* __restrict__ gval, double* __restrict__ A,
                            double* __restrict__ B) {
    const int64_t kk = (int64_t)k * k;
    for (int64_t t = threadIdx.x; t < kk; t += blockDim.x) {
        const int64_t l = t / k, m = t - l * k;
        A[t] = (l == m ? 1.0 : 0.0) - Z[l * ldz + m];
        B[t] = 0.0;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < k; l += blockDim.x)
        for (int e = gptr[l]; e < gptr[l + 1]; ++e) B[(int64_t)l * k + gcol[e]] = gval[e];
}

// B := A^{-1} B (k x k, row-major; A destroyed) by Gauss-Jordan elimination with partial
// pivoting, one block.  info[0] = 1 when a pivot is zero or not finite (B is then undefined).
__global__ void k_nl_gauss_jordan(double* __restrict__ A, double* __restrict__ B, int k, int* __restrict__ info) {
    extern __shared__ double fs[];   // k column factors
    __shared__ int piv;
    __shared__ double pmax;
    const int lane = threadIdx.x & 31;
    const int64_t kk = (int64_t)k * k;
    for (int c = 0; c < k; ++c) {
        if (threadIdx.x < 32) {
            double best = -1.0;
            int bi = c;
            for (int r = c + lane; r < k; r += 32) {
                const double v = fabs(A[(int64_t)r * k + c]);
                if (v > best) { best = v; bi = r; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) { piv = bi; pmax = best; }
        }
        __syncthreads();
        if (!(pmax > 0.0) || !isfinite(pmax)) {
            if (threadIdx.x == 0) info[0] = 1;
            return;
        }
        const int p = piv;
        if (p != c)
            for (int m = threadIdx.x; m < k; m += blockDim.x) {
                const double a = A[(int64_t)p * k + m], b = B[(int64_t)p * k + m];
                A[(int64_t)p * k + m] = A[(int64_t)c * k + m];
                B[(int64_t)p * k + m] = B[(int64_t)c * k + m];
                A[(int64_t)c * k + m] = a;
                B[(int64_t)c * k + m] = b;
            }
        __syncthreads();
        const double inv = 1.0 / A[(int64_t)c * k + c];
        __syncthreads();
        for (int m = threadIdx.x; m < k; m += blockDim.x) {
            A[(int64_t)c * k + m] *= inv;
            B[(int64_t)c * k + m] *= inv;
        }
        __syncthreads();
        for (int r = threadIdx.x; r < k; r += blockDim.x) fs[r] = r == c ? 0.0 : A[(int64_t)r * k + c];
        __syncthreads();
        for (int64_t t = threadIdx.x; t < kk; t += blockDim.x) {
            const int64_t r = t / k, m = t - r * k;
            if (r == c) continue;
            A[t] -= fs[r] * A[(int64_t)c * k + m];
            B[t] -= fs[r] * B[(int64_t)c * k + m];
        }
        __syncthreads();
    }
}

template <class T> struct NlData;
template <> struct NlData<double> {
    static const double* cval(Nonlocal& nl) { return nl.cval.p; }
    static const double* rval(Nonlocal& nl) { return nl.rval.p; }
    static DBuf<double>& part(Nonlocal& nl) { return nl.part; }
    static DBuf<double>& z(Nonlocal& nl) { return nl.z; }
    static DBuf<double>& Fh(Nonlocal& nl) { return nl.Fh; }
    static DBuf<double>& M(Nonlocal& nl) { return nl.M64; }
    static bool& ready(Nonlocal& nl) { return nl.smw64; }
};
template <> struct NlData<float> {
    static const float* cval(Nonlocal& nl) { return nl.cval32.p; }
    static const float* rval(Nonlocal& nl) { return nl.rval32.p; }
    static DBuf<float>& part(Nonlocal& nl) { return nl.part32; }
    static DBuf<float>& z(Nonlocal& nl) { return nl.z32; }
    static DBuf<float>& Fh(Nonlocal& nl) { return nl.Fh32; }
    static DBuf<double>& M(Nonlocal& nl) { return nl.M32; }
    static bool& ready(Nonlocal& nl) { return nl.smw32; }
};

// FP32 paths work on the scaled pencil: build D F once
template <class T>
int nl_prepare(Session* s, cudaStream_t st) {
    Nonlocal& nl = s->nl;
    if constexpr (sizeof(T) == 8) return 0;
    if (nl.scaled32) return 0;
    HBSD_TRY(nl.cval32.alloc(nl.nnz));
    HBSD_TRY(nl.rval32.alloc(nl.nnz));
    k_nl_scale_cols<<<grid_for(nl.nnz), 256, 0, st>>>(nl.crow.p, nl.cval.p, nl.nnz, s->A.dscale.p, nl.cval32.p);
    HBSD_LAUNCHED(s);
    k_nl_scale_rows<<<grid_for(nl.nfr), 256, 0, st>>>(nl.frows.p, nl.nfr, nl.rptr.p, nl.rval.p, s->A.dscale.p,
                                                      nl.rval32.p);
    HBSD_LAUNCHED(s);
    nl.scaled32 = true;
    return 0;
}

// z[l, j] = (M F^T X)[l, j] for w columns of X; M given by rows (mptr, mcol, mval)
template <class T, class TO>
int nl_ft(Session* s, const T* X, int64_t ldx, int w, const int32_t* mptr, const int32_t* mcol, const double* mval,
          TO* Z, int64_t ldz, cudaStream_t st) {
    Nonlocal& nl = s->nl;
    const int64_t ldp = round_up(w, 4);
    DBuf<T>& part = NlData<T>::part(nl);
    HBSD_TRY(part.alloc((size_t)nl.n_items * ldp));
    const int tb = w >= 128 ? 128 : (w > 32 ? 64 : 32);
    k_nl_ft_partial<T><<<nl.n_items, tb, 0, st>>>(nl.item_e.p, nl.crow.p, NlData<T>::cval(nl), X, ldx, w, part.p, ldp);
    HBSD_LAUNCHED(s);
    k_nl_reduce<T, TO><<<w, 128, (size_t)nl.k * sizeof(double), st>>>(nl.item_ptr.p, part.p, ldp, nl.k, mptr, mcol,
                                                                      mval, Z, ldz);
    HBSD_LAUNCHED(s);
    return 0;
}

// SMW steps 1-4 for precision T (T = float: on the scaled pencil with the FP32 factor)
template <class T>
int nl_smw_prepare(Session* s, cudaStream_t st) {
    Nonlocal& nl = s->nl;
    if (NlData<T>::ready(nl)) return 0;
    if (!s->has_factor) return fail(HBSD_ERR_ARG, "SMW: no global factor in this session");
    if (sizeof(T) == 4) HBSD_TRY(factor_make_fp32(s->F, s->A.dscale.p, st));
    HBSD_TRY(nl_prepare<T>(s, st));
    const int64_t n = s->n;
    const int k = nl.k;
    nl.ldf = round_up(k, 4);
    const int64_t ldf = nl.ldf;
    DBuf<T>& Fh = NlData<T>::Fh(nl);
    HBSD_TRY(Fh.alloc((size_t)n * ldf));
    {   // step 1: Fh = -(H_loc - eps_bar S)^{-1} F  (factor_solve returns -K R)
        DBuf<T> dense;
        HBSD_TRY(dense.alloc((size_t)n * ldf));
        HBSD_CUDA(cudaMemsetAsync(dense.p, 0, (size_t)n * ldf * sizeof(T), st));
        k_nl_densify<T><<<grid_for(nl.nfr), 256, 0, st>>>(nl.frows.p, nl.nfr, nl.rptr.p, nl.rcol.p,
                                                          NlData<T>::rval(nl), dense.p, ldf);
        HBSD_LAUNCHED(s);
        HBSD_TRY(factor_solve<T>(s, s->F, dense.p, ldf, k, Fh.p, ldf, st));
        HBSD_CUDA(cudaStreamSynchronize(st));   // `dense` is freed on return
    }
    // steps 2-3: T = I + G F^T Fhat = I - G F^T Fh;  step 4: M = T^{-1} G
    const int64_t kk = (int64_t)k * k;
    HBSD_TRY(nl.tmat.alloc((size_t)k * ldf + 2 * kk));
    double* Zd = nl.tmat.p;
    double* A = Zd + (int64_t)k * ldf;
    double* B = A + kk;
    HBSD_TRY((nl_ft<T, double>(s, Fh.p, ldf, k, nl.gptr.p, nl.gcol.p, nl.gval.p, Zd, ldf, st)));
    k_nl_make_t<<<1, 256, 0, st>>>(Zd, ldf, k, nl.gptr.p, nl.gcol.p, nl.gval.p, A, B);
    HBSD_LAUNCHED(s);
    HBSD_TRY(nl.info.alloc(1));
    HBSD_CUDA(cudaMemsetAsync(nl.info.p, 0, sizeof(int), st));
    k_nl_gauss_jordan<<<1, 256, (size_t)k * sizeof(double), st>>>(A, B, k, nl.info.p);
    HBSD_LAUNCHED(s);
    int info = 0;
    HBSD_CUDA(cudaMemcpyAsync(&info, nl.info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (info) return fail(HBSD_ERR_ARG, "SMW: I + G F^T Fhat is singular");
    DBuf<double>& M = NlData<T>::M(nl);
    HBSD_TRY(M.alloc(kk));
    HBSD_CUDA(cudaMemcpyAsync(M.p, B, kk * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (!nl.mptr.p) {   // dense pattern of M in CSR form
        std::vector<int32_t> mp(k + 1), mc(kk);
        for (int l = 0; l <= k; ++l) mp[l] = l * k;
        for (int64_t t = 0; t < kk; ++t) mc[t] = (int32_t)(t % k);
        HBSD_TRY(nl.mptr.alloc(k + 1));
        HBSD_TRY(nl.mcol.alloc(kk));
        HBSD_CUDA(cudaMemcpy(nl.mptr.p, mp.data(), (k + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
        HBSD_CUDA(cudaMemcpy(nl.mcol.p, mc.data(), kk * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    NlData<T>::ready(nl) = true;
    return 0;
}

template <class T>
int upload(DBuf<T>& d, const std::vector<T>& h) {
    HBSD_TRY(d.alloc(std::max<size_t>(h.size(), 1)));
    if (!h.empty()) HBSD_CUDA(cudaMemcpy(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return 0;
}

}  // namespace

int nl_set(Session* s, int k, const double* F, int64_t ldf, const double* G) {
    Nonlocal& nl = s->nl;
    if (k < 0 || k > NL_KMAX) return fail(HBSD_ERR_ARG, "nonlocal: k must lie in [0, 4096]");
    if (k > 0 && (!F || !G || ldf < k)) return fail(HBSD_ERR_ARG, "nonlocal: F, G required and ldf >= k");
    if (k > 0) {   // G must be symmetric (Eq. fgf: Hermitian)
        double gmax = 0.0;
        for (int64_t t = 0; t < (int64_t)k * k; ++t) {
            if (!std::isfinite(G[t])) return fail(HBSD_ERR_ARG, "nonlocal: G has a non-finite entry");
            gmax = std::max(gmax, std::fabs(G[t]));
        }
        for (int l = 0; l < k; ++l)
            for (int m = 0; m < l; ++m)
                if (std::fabs(G[(int64_t)l * k + m] - G[(int64_t)m * k + l]) > 1e-14 * gmax)
                    return fail(HBSD_ERR_ARG, "nonlocal: G is not symmetric");
    }
    const int64_t n = s->n;
    // by rows
    std::vector<int64_t> rptr(n + 1, 0);
    std::vector<int32_t> rcol, frows;
    std::vector<double> rval;
    if (k > 0)
        for (int64_t i = 0; i < n; ++i) {
            for (int l = 0; l < k; ++l) {
                const double v = F[i * ldf + l];
                if (!std::isfinite(v)) return fail(HBSD_ERR_ARG, "nonlocal: F has a non-finite entry");
                if (v != 0.0) {
                    rcol.push_back(l);
                    rval.push_back(v);
                }
            }
            rptr[i + 1] = (int64_t)rcol.size();
            if (rptr[i + 1] > rptr[i]) frows.push_back((int32_t)i);
        }
    const int64_t nnz = (int64_t)rcol.size();
    nl.version++;
    nl.smw64 = nl.smw32 = nl.scaled32 = false;
    nl.mr_grid = -1;
    nl.mptr.release();
    nl.mcol.release();
    nl.k = k;
    nl.nnz = nnz;
    nl.nfr = (int64_t)frows.size();
    if (k == 0) {
        nl.n_items = 0;
        return 0;
    }
    // by projector (counting sort of the row entries), and the work items
    std::vector<int64_t> cptr(k + 1, 0);
    for (int32_t l : rcol) cptr[l + 1]++;
    for (int l = 0; l < k; ++l) cptr[l + 1] += cptr[l];
    std::vector<int32_t> crow(nnz);
    std::vector<double> cval(nnz);
    {
        std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = rptr[i]; e < rptr[i + 1]; ++e) {
                const int64_t d = fill[rcol[e]]++;
                crow[d] = (int32_t)i;
                cval[d] = rval[e];
            }
    }
    std::vector<int64_t> item_e;
    std::vector<int32_t> item_ptr(k + 1, 0);
    for (int l = 0; l < k; ++l) {
        for (int64_t e = cptr[l]; e < cptr[l + 1]; e += NL_ITEM) {
            item_e.push_back(e);
            item_e.push_back(std::min<int64_t>(e + NL_ITEM, cptr[l + 1]));
        }
        item_ptr[l + 1] = (int32_t)(item_e.size() / 2);
    }
    nl.n_items = (int)(item_e.size() / 2);
    // G by rows (its nonzero entries)
    std::vector<int32_t> gptr(k + 1, 0), gcol;
    std::vector<double> gval;
    for (int l = 0; l < k; ++l) {
        for (int m = 0; m < k; ++m)
            if (G[(int64_t)l * k + m] != 0.0) {
                gcol.push_back(m);
                gval.push_back(G[(int64_t)l * k + m]);
            }
        gptr[l + 1] = (int32_t)gcol.size();
    }
    HBSD_TRY(upload(nl.cptr, cptr)); HBSD_TRY(upload(nl.crow, crow)); HBSD_TRY(upload(nl.cval, cval));
    HBSD_TRY(upload(nl.item_e, item_e)); HBSD_TRY(upload(nl.item_ptr, item_ptr));
    HBSD_TRY(upload(nl.rptr, rptr)); HBSD_TRY(upload(nl.rcol, rcol)); HBSD_TRY(upload(nl.rval, rval));
    HBSD_TRY(upload(nl.frows, frows));
    HBSD_TRY(upload(nl.gptr, gptr)); HBSD_TRY(upload(nl.gcol, gcol)); HBSD_TRY(upload(nl.gval, gval));
    nl.h_rptr = std::move(rptr);
    nl.h_rcol = std::move(rcol);
    nl.h_rval = std::move(rval);
    nl.h_frows = std::move(frows);
    nl.h_gptr = std::move(gptr);
    nl.h_gcol = std::move(gcol);
    nl.h_gval = std::move(gval);
    return 0;
}

template <class T>
int nl_apply_add(Session* s, const T* X, int64_t ldx, int w, T* Y, int64_t ldy, cudaStream_t st) {
    Nonlocal& nl = s->nl;
    if (nl.k == 0 || nl.nnz == 0 || w <= 0) return 0;
    HBSD_TRY(nl_prepare<T>(s, st));
    const int64_t ldz = round_up(w, 4);
    DBuf<T>& z = NlData<T>::z(nl);
    HBSD_TRY(z.alloc((size_t)nl.k * ldz));
    HBSD_TRY((nl_ft<T, T>(s, X, ldx, w, nl.gptr.p, nl.gcol.p, nl.gval.p, z.p, ldz, st)));
    k_nl_apply<T><<<grid_for(nl.nfr * w), 256, 0, st>>>(nl.frows.p, nl.nfr, nl.rptr.p, nl.rcol.p, NlData<T>::rval(nl),
                                                        z.p, ldz, w, Y, ldy);
    HBSD_LAUNCHED(s);
    return 0;
}

template <class T>
int nl_smw_correct(Session* s, T* P, int64_t ldp, int p, cudaStream_t st) {
    Nonlocal& nl = s->nl;
    if (nl.k == 0 || nl.nnz == 0 || p <= 0) return 0;
    HBSD_TRY(nl_smw_prepare<T>(s, st));
    const int64_t ldz = round_up(p, 4);
    DBuf<T>& z = NlData<T>::z(nl);
    HBSD_TRY(z.alloc((size_t)nl.k * ldz));
    HBSD_TRY((nl_ft<T, T>(s, P, ldp, p, nl.mptr.p, nl.mcol.p, NlData<T>::M(nl).p, z.p, ldz, st)));
    k_nl_lowrank_add<T><<<grid_for(s->n * p), 256, 0, st>>>(NlData<T>::Fh(nl).p, nl.ldf, nl.k, z.p, ldz, s->n, p, P,
                                                            ldp);
    HBSD_LAUNCHED(s);
    return 0;
}

template int nl_apply_add<double>(Session*, const double*, int64_t, int, double*, int64_t, cudaStream_t);
template int nl_apply_add<float>(Session*, const float*, int64_t, int, float*, int64_t, cudaStream_t);
template int nl_smw_correct<double>(Session*, double*, int64_t, int, cudaStream_t);
template int nl_smw_correct<float>(Session*, float*, int64_t, int, cudaStream_t);

// Index of the fused MINRES kernel for `grid` blocks with SELL slot ranges blk (minres.cu):
//  * chunk c (worked by block c): a contiguous range of the rows with F entries, about equal in
//    entries; its projectors (slots ch_lptr[c] .. ch_lptr[c+1]) and a dense panel rows x slots;
//  * per projector l: the chunk slots holding a partial of row l of F^T U, in chunk order;
//  * per block b: the projectors met by the F entries of its SpMM rows (N_b, applied) followed
//    by those only coupled to them through G, with lmap[b * k + l] = local index or -1.
int nl_minres_index(Session* s, int grid, const std::vector<int64_t>& blk, int64_t kp) {
    Nonlocal& nl = s->nl;
    const int k = nl.k;
    if (nl.mr_grid != grid || nl.mr_version != nl.version) {
        const std::vector<int64_t>& rptr = nl.h_rptr;
        const std::vector<int32_t>& rcol = nl.h_rcol;
        // rows with F entries ordered by their first projector (then row): a chunk then covers
        // the rows of one atom's projectors, so it meets few projectors and each projector's
        // partials sit in few chunks
        std::vector<int32_t> frows = nl.h_frows;
        std::stable_sort(frows.begin(), frows.end(), [&](int32_t x, int32_t y) {
            return rcol[rptr[x]] < rcol[rptr[y]];
        });
        const int64_t nfr = (int64_t)frows.size();
        // chunks
        std::vector<int64_t> row_off(grid + 1, nfr);
        row_off[0] = 0;
        {
            int64_t r = 0, acc = 0;
            for (int c = 1; c < grid; ++c) {
                const double target = (double)nl.nnz * c / grid;
                while (r < nfr && (double)acc < target) {
                    acc += rptr[frows[r] + 1] - rptr[frows[r]];
                    ++r;
                }
                row_off[c] = r;
            }
        }
        std::vector<int32_t> lptr(grid + 1, 0), lids;
        std::vector<int64_t> pan_off(grid + 1, 0);
        std::vector<double> pan;
        std::vector<int32_t> loc(k, -1);
        for (int c = 0; c < grid; ++c) {
            std::vector<int32_t> ls;
            for (int64_t r = row_off[c]; r < row_off[c + 1]; ++r)
                for (int64_t e = rptr[frows[r]]; e < rptr[frows[r] + 1]; ++e) ls.push_back(rcol[e]);
            std::sort(ls.begin(), ls.end());
            ls.erase(std::unique(ls.begin(), ls.end()), ls.end());
            for (size_t t = 0; t < ls.size(); ++t) loc[ls[t]] = (int32_t)t;
            const int64_t nr = row_off[c + 1] - row_off[c], nlc = (int64_t)ls.size();
            const int64_t base = (int64_t)pan.size();
            pan.resize(base + nr * nlc, 0.0);
            for (int64_t r = 0; r < nr; ++r) {
                const int64_t i = frows[row_off[c] + r];
                for (int64_t e = rptr[i]; e < rptr[i + 1]; ++e) pan[base + r * nlc + loc[rcol[e]]] = nl.h_rval[e];
            }
            lids.insert(lids.end(), ls.begin(), ls.end());
            lptr[c + 1] = (int32_t)lids.size();
            pan_off[c + 1] = (int64_t)pan.size();
        }
        // contributors of each projector
        std::vector<int32_t> cl_ptr(k + 1, 0), cl_slot(lids.size());
        for (int32_t l : lids) cl_ptr[l + 1]++;
        for (int l = 0; l < k; ++l) cl_ptr[l + 1] += cl_ptr[l];
        {
            std::vector<int32_t> fill(cl_ptr.begin(), cl_ptr.end() - 1);
            for (size_t sl = 0; sl < lids.size(); ++sl) cl_slot[fill[lids[sl]]++] = (int32_t)sl;
        }
        // needed projectors of each block
        const Sell& A = s->A;
        std::vector<int32_t> nb_ptr(grid + 1, 0), nb_napply(grid, 0), nb_l;
        std::vector<int32_t> lmap((size_t)grid * k, -1);
        std::vector<char> mark(k, 0);
        for (int b = 0; b < grid; ++b) {
            std::vector<int32_t> ap;
            for (int64_t slot = blk[b]; slot < blk[b + 1]; ++slot) {
                const int row = A.h_slot_row[slot];
                if (row < 0) continue;
                for (int64_t e = rptr[row]; e < rptr[row + 1]; ++e)
                    if (!mark[rcol[e]]) { mark[rcol[e]] = 1; ap.push_back(rcol[e]); }
            }
            std::sort(ap.begin(), ap.end());
            std::vector<int32_t> extra;
            for (int32_t l : ap)
                for (int e = nl.h_gptr[l]; e < nl.h_gptr[l + 1]; ++e) {
                    const int32_t m = nl.h_gcol[e];
                    if (!mark[m]) { mark[m] = 1; extra.push_back(m); }
                }
            std::sort(extra.begin(), extra.end());
            for (int32_t l : ap) mark[l] = 0;
            for (int32_t l : extra) mark[l] = 0;
            nb_napply[b] = (int32_t)ap.size();
            for (size_t t = 0; t < ap.size(); ++t) lmap[(size_t)b * k + ap[t]] = (int32_t)t;
            for (size_t t = 0; t < extra.size(); ++t) lmap[(size_t)b * k + extra[t]] = (int32_t)(ap.size() + t);
            nb_l.insert(nb_l.end(), ap.begin(), ap.end());
            nb_l.insert(nb_l.end(), extra.begin(), extra.end());
            nb_ptr[b + 1] = (int32_t)nb_l.size();
        }
        // F entries of every SELL slot with the zg row of its block they read
        std::vector<int32_t> sf_ptr(A.n_slots + 1, 0), sf_off;
        std::vector<double> sf_val;
        for (int b = 0; b < grid; ++b)
            for (int64_t slot = blk[b]; slot < blk[b + 1]; ++slot) {
                const int row = A.h_slot_row[slot];
                if (row >= 0)
                    for (int64_t e = rptr[row]; e < rptr[row + 1]; ++e) {
                        sf_off.push_back(nb_ptr[b] + lmap[(size_t)b * k + rcol[e]]);
                        sf_val.push_back(nl.h_rval[e]);
                    }
                sf_ptr[slot + 1] = (int32_t)sf_off.size();
            }
        HBSD_TRY(upload(nl.sf_ptr, sf_ptr)); HBSD_TRY(upload(nl.sf_off, sf_off)); HBSD_TRY(upload(nl.sf_val, sf_val));
        HBSD_TRY(upload(nl.ch_rows, frows));
        HBSD_TRY(upload(nl.ch_row_off, row_off)); HBSD_TRY(upload(nl.ch_lptr, lptr));
        HBSD_TRY(upload(nl.pan_off, pan_off)); HBSD_TRY(upload(nl.pan, pan));
        HBSD_TRY(upload(nl.cl_ptr, cl_ptr)); HBSD_TRY(upload(nl.cl_slot, cl_slot));
        HBSD_TRY(upload(nl.nb_ptr, nb_ptr)); HBSD_TRY(upload(nl.nb_napply, nb_napply));
        HBSD_TRY(upload(nl.nb_l, nb_l)); HBSD_TRY(upload(nl.lmap, lmap));
        nl.mr_grid = grid;
        nl.mr_version = nl.version;
        nl.mr_nslots = lptr[grid];
        nl.mr_nneed = nb_ptr[grid];
    }
    // partial sums (one row of kp per chunk slot) and the per-block reduced values
    HBSD_TRY(nl.mr_part.alloc((size_t)std::max(nl.mr_nslots, 1) * kp));
    HBSD_TRY(nl.zv.alloc((size_t)std::max(nl.mr_nneed, 1) * kp));
    HBSD_TRY(nl.zg.alloc((size_t)std::max(nl.mr_nneed, 1) * kp));
    return 0;
}

}  // namespace hbsd
