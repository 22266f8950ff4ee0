// Complex Hermitian input (Sec. 2: at a Bloch vector k != 0 the pencil H x = lambda S x has H
// Hermitian and S Hermitian positive definite) on the real kernels of the library.
//
// H = Hr + i Hi with Hr symmetric and Hi antisymmetric acts on x = a + i b like the real
// symmetric matrix [[Hr, -Hi], [Hi, Hr]] on (a, b); likewise S.  That real pencil of size 2n has
// every eigenvalue of the complex one twice, with eigenvectors (a, b) and J (a, b) = (-b, a), the
// realifications of x and i x, and H - eps_bar S positive definite stays positive definite.  The
// session stores it with the two real dofs of a complex dof next to each other (row 2i: real
// part, row 2i+1: imaginary part), so a complex entry becomes a 2 x 2 block [[a, -b], [b, a]] and
// nested dissection keeps both halves of a dof in one supernode (they share a mesh node).
//
// The solve runs LABPSD (Sec. 3) on the real pencil from the start block [x~_c, J x~_c]: its span
// is invariant under J, and every step keeps it so (K, the MINRES operator and the Rayleigh-Ritz
// of the real pencil commute with J; MINRES on a Hermitian operator has real Lanczos
// coefficients), so the iteration is the complex LABPSD of the same start block, written in real
// arithmetic, with 2 nev real columns for nev complex ones.
//
// Recovery: the 2 nev real eigenvectors y_k give complex vectors z_k (rows 2i + i * rows 2i+1)
// whose complex span has dimension nev.  Their complex S-Gram is G = Y^T S~ Y - i Y^T J S~ Y.
// A Cholesky elimination of G that takes the columns in ascending eigenvalue order and keeps a
// column when its remaining diagonal exceeds 1/2 (G is twice a projector: remaining diagonals are
// near 0 for a column already in the span and at least 2/3 for some column of every cluster not
// yet covered) selects nev of them; X = Z_P L_P^{-H} is the S-orthonormal complex basis, and the
// eigenvalue of column a is the Ritz value of its selected y.
#include <cmath>

#include "common.h"

namespace hbsd {

int complex_realify_csr(int64_t n, const int64_t* rp, const int32_t* ci, const double* hv, const double* sv,
                        const int32_t* dof_node, std::vector<int64_t>& rp2, std::vector<int32_t>& ci2,
                        std::vector<double>& hv2, std::vector<double>& sv2, std::vector<int32_t>& node2) {
    const int64_t nnz = rp[n];
    rp2.assign(2 * n + 1, 0);
    ci2.resize(4 * nnz);
    hv2.resize(4 * nnz);
    sv2.resize(4 * nnz);
    node2.resize(2 * n);
    int64_t pos = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int t = 0; t < 2; ++t) {           // t = 0: row of the real part, 1: imaginary part
            rp2[2 * i + t] = pos;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                const int32_t j = ci[e];
                const double ha = hv[2 * e], hb = hv[2 * e + 1], sa = sv[2 * e], sb = sv[2 * e + 1];
                // [[a, -b], [b, a]] at rows (2i, 2i+1), columns (2j, 2j+1)
                ci2[pos] = 2 * j;
                hv2[pos] = t == 0 ? ha : hb;
                sv2[pos] = t == 0 ? sa : sb;
                ++pos;
                ci2[pos] = 2 * j + 1;
                hv2[pos] = t == 0 ? -hb : ha;
                sv2[pos] = t == 0 ? -sb : sa;
                ++pos;
            }
        }
        node2[2 * i] = node2[2 * i + 1] = dof_node[i];
    }
    rp2[2 * n] = pos;
    return 0;
}

void complex_realify_values(int64_t n, const int64_t* rp, const double* v, std::vector<double>& out) {
    out.resize(4 * rp[n]);
    int64_t pos = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int t = 0; t < 2; ++t)
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                const double a = v[2 * e], b = v[2 * e + 1];
                out[pos++] = t == 0 ? a : b;
                out[pos++] = t == 0 ? -b : a;
            }
}

namespace {

// Y(:, 2c) = x~_c (realified column c of the complex block), Y(:, 2c+1) = J x~_c
__global__ void k_realify_start(const double* __restrict__ X0c, int64_t ldc, int wc, int64_t nc,
                                double* __restrict__ Y, int64_t ldy) {
    const int64_t total = nc * wc;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / wc;
        const int c = (int)(t % wc);
        const double re = X0c[2 * (i * ldc + c)], im = X0c[2 * (i * ldc + c) + 1];
        Y[(2 * i) * ldy + 2 * c] = re;
        Y[(2 * i + 1) * ldy + 2 * c] = im;
        Y[(2 * i) * ldy + 2 * c + 1] = -im;
        Y[(2 * i + 1) * ldy + 2 * c + 1] = re;
    }
}

// B = J A for a realified block of nc complex rows: (J y)_{2i} = -y_{2i+1}, (J y)_{2i+1} = y_{2i}
__global__ void k_apply_J(const double* __restrict__ A, int64_t lda, int k, int64_t nc, double* __restrict__ B,
                          int64_t ldb) {
    const int64_t total = nc * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int j = (int)(t % k);
        const double re = A[(2 * i) * lda + j], im = A[(2 * i + 1) * lda + j];
        B[(2 * i) * ldb + j] = -im;
        B[(2 * i + 1) * ldb + j] = re;
    }
}

// complex output: Xc(i, j) = (Xr(2i, j), Xr(2i+1, j)), ld in complex elements
__global__ void k_interleave_out(const double* __restrict__ Xr, int64_t ldr, int k, int64_t nc,
                                 double* __restrict__ Xc, int64_t ldc) {
    const int64_t total = nc * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int j = (int)(t % k);
        Xc[2 * (i * ldc + j)] = Xr[(2 * i) * ldr + j];
        Xc[2 * (i * ldc + j) + 1] = Xr[(2 * i + 1) * ldr + j];
    }
}

__global__ void k_copy_cols(const double* __restrict__ A, int64_t lda, int k, int64_t n, double* __restrict__ B,
                            int64_t ldb) {
    const int64_t total = n * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int j = (int)(t % k);
        B[i * ldb + j] = A[i * lda + j];
    }
}

__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline double2 cmul_conj(double2 a, double2 b) {   // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

constexpr int SEL_THREADS = 1024;
constexpr int SEL_MAX_Q = 1024;

// One CTA.  G = Gr - i Gc (q x q Hermitian, q = 2 nev), eliminated in place in A; selected columns
// piv[0..nev); Wt ((2q) x nev row-major): rows 0..q-1 the real and rows q..2q-1 the imaginary part
// of the coefficients W (X = Z W, W = E_P L_P^{-H}); lam[a] = E[piv[a]] + sigma0.  info[0] = number
// of columns selected.
__global__ void __launch_bounds__(SEL_THREADS) k_complex_select(const double* __restrict__ Gr,
                                                                const double* __restrict__ Gc, int q, int nev,
                                                                double thresh, double2* __restrict__ A,
                                                                double2* __restrict__ Lc, double2* __restrict__ M,
                                                                int* __restrict__ piv, double* __restrict__ Wt,
                                                                const double* __restrict__ E, double sigma0,
                                                                double* __restrict__ lam, int* __restrict__ info) {
    __shared__ double2 lcol[SEL_MAX_Q];
    __shared__ int s_acc;
    const int tid = threadIdx.x;
    const int64_t qq = (int64_t)q * q;
    for (int64_t t = tid; t < qq; t += blockDim.x) A[t] = make_double2(Gr[t], -Gc[t]);
    __syncthreads();
    int cnt = 0;   // uniform across the block
    for (int k = 0; k < q && cnt < nev; ++k) {
        if (tid == 0) s_acc = A[(int64_t)k * q + k].x > thresh ? 1 : 0;
        __syncthreads();
        const int acc = s_acc;
        __syncthreads();
        if (!acc) continue;
        const double r = sqrt(A[(int64_t)k * q + k].x);
        const double rinv = 1.0 / r;
        for (int i = k + 1 + tid; i < q; i += blockDim.x) {
            const double2 a = A[(int64_t)i * q + k];
            const double2 l = make_double2(a.x * rinv, a.y * rinv);
            lcol[i] = l;
            Lc[(int64_t)i * nev + cnt] = l;
        }
        if (tid == 0) {
            Lc[(int64_t)k * nev + cnt] = make_double2(r, 0.0);
            piv[cnt] = k;
        }
        __syncthreads();
        const int m = q - k - 1;
        const int64_t mm = (int64_t)m * m;
        for (int64_t t = tid; t < mm; t += blockDim.x) {
            const int i = k + 1 + (int)(t / m), j = k + 1 + (int)(t % m);
            const double2 u = cmul_conj(lcol[i], lcol[j]);
            double2& a = A[(int64_t)i * q + j];
            a.x -= u.x;
            a.y -= u.y;
        }
        __syncthreads();
        ++cnt;
    }
    if (tid == 0) info[0] = cnt;
    if (cnt < nev) return;
    // L_P (nev x nev, lower): rows piv[a] of the stored Cholesky columns, kept in A
    for (int64_t t = tid; t < (int64_t)nev * nev; t += blockDim.x) {
        const int a = (int)(t / nev), b = (int)(t % nev);
        A[t] = b <= a ? Lc[(int64_t)piv[a] * nev + b] : make_double2(0.0, 0.0);
    }
    for (int64_t t = tid; t < 2 * (int64_t)q * nev; t += blockDim.x) Wt[t] = 0.0;
    __syncthreads();
    // M = L_P^{-1} by forward substitution, one column per thread (the diagonal of L_P is real)
    for (int c = tid; c < nev; c += blockDim.x) {
        M[(int64_t)c * nev + c] = make_double2(1.0 / A[(int64_t)c * nev + c].x, 0.0);
        for (int r2 = c + 1; r2 < nev; ++r2) {
            double2 s = make_double2(0.0, 0.0);
            for (int t = c; t < r2; ++t) {
                const double2 p = cmul(A[(int64_t)r2 * nev + t], M[(int64_t)t * nev + c]);
                s.x += p.x;
                s.y += p.y;
            }
            const double dinv = 1.0 / A[(int64_t)r2 * nev + r2].x;
            M[(int64_t)r2 * nev + c] = make_double2(-s.x * dinv, -s.y * dinv);
        }
    }
    __syncthreads();
    // W = M^H (upper): W(a, b) = conj(M(b, a)), b >= a, placed on row piv[a] of the coefficients
    for (int64_t t = tid; t < (int64_t)nev * nev; t += blockDim.x) {
        const int a = (int)(t / nev), b = (int)(t % nev);
        if (b < a) continue;
        const double2 mba = M[(int64_t)b * nev + a];
        Wt[(int64_t)piv[a] * nev + b] = mba.x;
        Wt[((int64_t)q + piv[a]) * nev + b] = -mba.y;
    }
    for (int a = tid; a < nev; a += blockDim.x) lam[a] = E[piv[a]] + sigma0;
}

inline int grid_for(int64_t work) {
    return (int)std::min<int64_t>(std::max<int64_t>(1, (work + 255) / 256), 8192);
}

}  // namespace

int complex_start_block(Session* s, const double* X0c, int64_t ldc, int wc, double* Y, int64_t ldy) {
    k_realify_start<<<grid_for(s->n_c * wc), 256, 0, s->stream>>>(X0c, ldc, wc, s->n_c, Y, ldy);
    HBSD_LAUNCHED(s);
    return 0;
}

// After a solve of the real pencil for 2 nev pairs (the block in s->sb.Psi, ld s->keep_ld; the
// shifted Ritz values in s->sc.E): nev complex eigenvalues (lam_dev, unshifted, ascending) and the
// S-orthonormal complex eigenvectors (Xc_dev, row-major n_c x nev complex with ld ldxc, or NULL).
int complex_recover(Session* s, int nev, double* lam_dev, double* Xc_dev, int64_t ldxc) {
    cudaStream_t st = s->stream;
    const int q = 2 * nev;
    if (q > SEL_MAX_Q) return fail(HBSD_ERR_ARG, "complex input: nev <= 512");
    const int64_t n = s->n, nc = s->n_c;
    SolveBufs<double>& B = s->sb;
    const double* Y = B.Psi.p;
    const int64_t ldw = s->keep_ld;
    const int64_t ldp = round_up(q, 4);   // the solve's P-block width for m = 2 nev
    if (B.P.n < (size_t)(n * ldp)) return fail(HBSD_ERR_ARG, "complex recovery: solve blocks too small");
    // S~ Y, J S~ Y
    HBSD_TRY(spmm_pair<double>(s, s->A, Y, ldw, q, B.PH.p, ldp, B.PS.p, ldp, st));
    k_apply_J<<<grid_for(nc * q), 256, 0, st>>>(B.PS.p, ldp, q, nc, B.RU.p, ldp);
    HBSD_LAUNCHED(s);
    HBSD_TRY(s->cx_gr.alloc((size_t)q * q));
    HBSD_TRY(s->cx_gc.alloc((size_t)q * q));
    // Gc = skew(Y^T J S~ Y), Gr = sym(Y^T S~ Y)
    HBSD_TRY(gram_skew(s, Y, ldw, B.RU.p, ldp, B.PS.p, ldp, n, q, s->cx_gc.p, s->cx_gr.p, st));
    HBSD_TRY(s->cx_a.alloc((size_t)q * q));
    HBSD_TRY(s->cx_l.alloc((size_t)q * nev));
    HBSD_TRY(s->cx_m.alloc((size_t)nev * nev));
    HBSD_TRY(s->cx_piv.alloc(nev + 1));
    HBSD_TRY(s->cx_w.alloc((size_t)2 * q * nev));
    HBSD_TRY(s->io_lam.alloc(nev));
    double* lam = lam_dev ? lam_dev : s->io_lam.p;
    int* info = s->cx_piv.p + nev;
    k_complex_select<<<1, SEL_THREADS, 0, st>>>(s->cx_gr.p, s->cx_gc.p, q, nev, 0.5, s->cx_a.p, s->cx_l.p, s->cx_m.p,
                                                s->cx_piv.p, s->cx_w.p, s->sc.E.p, s->sigma0, lam, info);
    HBSD_LAUNCHED(s);
    int cnt = 0;
    HBSD_CUDA(cudaMemcpyAsync(&cnt, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (cnt < nev)
        return fail(HBSD_ERR_RR_RANK, "complex recovery: the computed block spans " + std::to_string(cnt) +
                                          " < nev complex directions");
    if (!Xc_dev) return 0;
    // X~ = Y W_r + (J Y) W_i, formed in place in a copy of Y
    k_copy_cols<<<grid_for(n * q), 256, 0, st>>>(Y, ldw, q, n, B.P.p, ldp);
    HBSD_LAUNCHED(s);
    k_apply_J<<<grid_for(nc * q), 256, 0, st>>>(Y, ldw, q, nc, B.Xa.p, ldp);
    HBSD_LAUNCHED(s);
    HBSD_TRY(update2<double>(s, B.P.p, ldp, q, B.Xa.p, ldp, q, n, s->cx_w.p, nev, st));
    k_interleave_out<<<grid_for(nc * nev), 256, 0, st>>>(B.P.p, ldp, nev, nc, Xc_dev, ldxc);
    HBSD_LAUNCHED(s);
    return 0;
}

}  // namespace hbsd
