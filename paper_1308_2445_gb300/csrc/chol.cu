// Global preconditioner of LABPSD step 6(a): K = (H - eps_bar S)^{-1} (Eq. globalprecond,
// Eq. k1p), applied through a sparse factorisation computed once per session (Sec. 4,
// Eq. ldl: "computed just once and used throughout").  eps_bar lies below the spectrum, so
// H - eps_bar S is positive definite and the factorisation is a Cholesky L L^T.
//
//  * ordering (host): geometric nested dissection of the periodic node grid; the dofs of a
//    node stay together.  A periodic direction is cut by two planes, an open one by one.
//    Each dissection-tree node (separator or leaf box) is one supernode.
//  * symbolic (host): below-diagonal row structure of every supernode, child->parent
//    extend-add maps, storage offsets.
//  * numeric (GPU): multifrontal, one tree level at a time; a front is assembled from the
//    matrix entries and the children's update matrices, then partially factorised by a
//    blocked right-looking Cholesky (NB x NB diagonal blocks in shared memory, their
//    inverses kept for the solves).  Only the lower triangle of a front is referenced.
//  * solve (GPU): forward multifrontal sweep with front vectors (levels bottom-up), backward
//    sweep gathering the ancestors' solution (levels top-down); within a supernode both are
//    blocked by NB with the inverted diagonal blocks.
#include <algorithm>
#include <array>
#include <chrono>
#include <mutex>
#include <numeric>
#include <type_traits>

#include "common.h"

namespace hbsd {

namespace {

constexpr int NB = Factor::NB;
constexpr int LEAF_NODES = 64;

struct SnDev {
    int64_t first, L_off, Dinv_off, fv_off, struct_off, ea_off, front_off;
    int ns, nu, child0, child1;
};

struct NDTree {
    int g[3];
    std::vector<std::vector<int32_t>> nodes;   // mesh nodes of each tree node
    std::vector<std::array<int, 2>> kids;
    std::vector<int> parent;

    int add(std::vector<int32_t>&& v) {
        nodes.push_back(std::move(v));
        kids.push_back({-1, -1});
        parent.push_back(-1);
        return (int)nodes.size() - 1;
    }
    void box_nodes(const int lo[3], const int hi[3], std::vector<int32_t>& out) const {
        for (int z = lo[2]; z < hi[2]; ++z)
            for (int y = lo[1]; y < hi[1]; ++y)
                for (int x = lo[0]; x < hi[0]; ++x) {
                    const int xx = ((x % g[0]) + g[0]) % g[0];
                    const int yy = ((y % g[1]) + g[1]) % g[1];
                    const int zz = ((z % g[2]) + g[2]) % g[2];
                    out.push_back(xx + g[0] * (yy + g[1] * zz));
                }
    }
    int build(const int lo[3], const int hi[3], const bool per[3]) {
        int size[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
        if (size[0] <= 0 || size[1] <= 0 || size[2] <= 0) return -1;
        const int64_t vol = (int64_t)size[0] * size[1] * size[2];
        if (vol <= LEAF_NODES) {
            std::vector<int32_t> v;
            box_nodes(lo, hi, v);
            return add(std::move(v));
        }
        int d = 0;
        for (int e = 1; e < 3; ++e)
            if (size[e] > size[d]) d = e;
        const int mid = lo[d] + size[d] / 2;
        std::vector<int> planes;
        int alo[3], ahi[3], blo[3], bhi[3];
        bool per2[3] = {per[0], per[1], per[2]};
        for (int e = 0; e < 3; ++e) { alo[e] = blo[e] = lo[e]; ahi[e] = bhi[e] = hi[e]; }
        if (per[d]) {
            planes.push_back(lo[d]);
            if (mid != lo[d]) planes.push_back(mid);
            alo[d] = lo[d] + 1; ahi[d] = mid;
            blo[d] = mid + 1; bhi[d] = hi[d];
            per2[d] = false;
        } else {
            planes.push_back(mid);
            ahi[d] = mid;
            blo[d] = mid + 1;
        }
        const int ca = build(alo, ahi, per2);
        const int cb = build(blo, bhi, per2);
        std::vector<int32_t> sep;
        for (int pl : planes) {
            int slo[3] = {lo[0], lo[1], lo[2]}, shi[3] = {hi[0], hi[1], hi[2]};
            slo[d] = pl; shi[d] = pl + 1;
            box_nodes(slo, shi, sep);
        }
        const int id = add(std::move(sep));
        kids[id] = {ca, cb};
        if (ca >= 0) parent[ca] = id;
        if (cb >= 0) parent[cb] = id;
        return id;
    }
};

// ---- numeric factorisation kernels ---------------------------------------------------------
__global__ void k_zero(double* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0.0;
}

__global__ void k_scatter_entries(const int64_t* __restrict__ pos, const int64_t* __restrict__ src,
                                  int64_t count, const double* __restrict__ aval, double* __restrict__ F) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        F[pos[i]] = aval[src[i]];
}

// parent front += child update matrix (lower triangle), jobs = (parent, child) pairs
__global__ void k_extend_add_matrix(const SnDev* __restrict__ sn, const int* __restrict__ jobs, int njobs,
                                    const int32_t* __restrict__ ea, double* __restrict__ F) {
    const int job = blockIdx.y;
    if (job >= njobs) return;
    const SnDev p = sn[jobs[2 * job]];
    const SnDev c = sn[jobs[2 * job + 1]];
    const int nu = c.nu;
    const int nfc = c.ns + c.nu, nfp = p.ns + p.nu;
    const int64_t total = (int64_t)nu * nu;
    const int32_t* map = ea + c.ea_off;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % nu), j = (int)(idx / nu);
        if (i < j) continue;
        const double u = F[c.front_off + (int64_t)(c.ns + j) * nfc + c.ns + i];
        F[p.front_off + (int64_t)map[j] * nfp + map[i]] += u;
    }
}

// Cholesky of the diagonal block [k0, k0+kb) of each front in shared memory, plus its inverse.
// SIGNED: the LDL^T form with 1 x 1 pivots, held as A = Lt Sg Lt^T with Sg = diag(+-1) and
// Lt = L |D|^{1/2}: a pivot d gives Lt_cc = sqrt|d|, sign(d) goes to sgn[] (permuted order) and
// the column below is divided by Lt_cc sign(d); negative pivots are counted in err[1].  Only a
// zero or non-finite pivot fails (err[0]).  Without SIGNED a non-positive pivot fails.
template <bool SIGNED>
__global__ void __launch_bounds__(256) k_potrf_block(const SnDev* __restrict__ sn, const int* __restrict__ ids,
                                                     int nids, int k0, double* __restrict__ F,
                                                     double* __restrict__ Dinv, int* __restrict__ err,
                                                     double* __restrict__ sgn) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto A = reinterpret_cast<double(*)[NB + 1]>(smem_raw);
    auto X = reinterpret_cast<double(*)[NB + 1]>(smem_raw + sizeof(double) * NB * (NB + 1));
    __shared__ int bad, nneg;
    __shared__ double sg[NB];
    const SnDev s = sn[ids[blockIdx.x]];
    if (k0 >= s.ns) return;
    const int kb = min(NB, s.ns - k0);
    const int nf = s.ns + s.nu;
    double* Fb = F + s.front_off + (int64_t)k0 * nf + k0;
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        const int i = t % NB, j = t / NB;
        A[i][j] = (i < kb && j < kb && i >= j) ? Fb[(int64_t)j * nf + i] : 0.0;
        X[i][j] = 0.0;
    }
    if (threadIdx.x == 0) bad = nneg = 0;
    __syncthreads();
    for (int c = 0; c < kb; ++c) {
        if (threadIdx.x == 0) {
            const double piv = A[c][c];
            if constexpr (SIGNED) {
                if (!(fabs(piv) > 0.0) || !isfinite(piv)) { bad = 1; A[c][c] = 1.0; sg[c] = 1.0; }
                else {
                    A[c][c] = sqrt(fabs(piv));
                    sg[c] = piv < 0.0 ? -1.0 : 1.0;
                    if (piv < 0.0) ++nneg;
                }
            } else {
                if (!(piv > 0.0)) { bad = 1; A[c][c] = 1.0; }
                else A[c][c] = sqrt(piv);
            }
        }
        __syncthreads();
        const double l = A[c][c];
        if constexpr (SIGNED) {
            const double sc = sg[c];
            for (int i = c + 1 + threadIdx.x; i < kb; i += blockDim.x) A[i][c] = A[i][c] / l * sc;
            __syncthreads();
            const int m = kb - c - 1;
            for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
                const int i = c + 1 + t % m, j = c + 1 + t / m;
                if (i >= j) A[i][j] -= (A[i][c] * sc) * A[j][c];
            }
        } else {
            for (int i = c + 1 + threadIdx.x; i < kb; i += blockDim.x) A[i][c] /= l;
            __syncthreads();
            const int m = kb - c - 1;
            for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
                const int i = c + 1 + t % m, j = c + 1 + t / m;
                if (i >= j) A[i][j] -= A[i][c] * A[j][c];
            }
        }
        __syncthreads();
    }
    if (bad && threadIdx.x == 0) atomicExch(err, 1);
    if constexpr (SIGNED) {
        if (threadIdx.x == 0 && nneg) atomicAdd(err + 1, nneg);
        for (int c = threadIdx.x; c < kb; c += blockDim.x) sgn[s.first + k0 + c] = sg[c];
    }
    // inverse of the lower-triangular block, one column per thread
    for (int c = threadIdx.x; c < kb; c += blockDim.x) {
        X[c][c] = 1.0 / A[c][c];
        for (int i = c + 1; i < kb; ++i) {
            double acc = 0.0;
            for (int t = c; t < i; ++t) acc += A[i][t] * X[t][c];
            X[i][c] = -acc / A[i][i];
        }
    }
    __syncthreads();
    double* Db = Dinv + s.Dinv_off + (int64_t)(k0 / NB) * NB * NB;
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        const int i = t % NB, j = t / NB;
        if (i < kb && j < kb && i >= j) Fb[(int64_t)j * nf + i] = A[i][j];
        Db[t] = (i < kb && j < kb) ? X[i][j] : 0.0;  // column-major NB x NB
    }
}

// Panel: F[k0+kb : nf, k0 : k0+kb] := F[...] * L_kk^{-T}  (row tiles of 64); SIGNED: then column
// c times its pivot sign
template <bool SIGNED>
__global__ void __launch_bounds__(256) k_trsm_panel(const SnDev* __restrict__ sn, const int* __restrict__ ids,
                                                    int k0, double* __restrict__ F, const double* __restrict__ Dinv,
                                                    const double* __restrict__ sgn) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto Ar = reinterpret_cast<double(*)[NB + 1]>(smem_raw);
    auto Di = reinterpret_cast<double(*)[NB + 1]>(smem_raw + sizeof(double) * 64 * (NB + 1));
    const SnDev s = sn[ids[blockIdx.y]];
    if (k0 >= s.ns) return;
    const int kb = min(NB, s.ns - k0);
    const int nf = s.ns + s.nu;
    const int r0 = k0 + kb + blockIdx.x * 64;
    if (r0 >= nf) return;
    const int rows = min(64, nf - r0);
    double* Fc = F + s.front_off + (int64_t)k0 * nf;
    const double* Db = Dinv + s.Dinv_off + (int64_t)(k0 / NB) * NB * NB;
    for (int t = threadIdx.x; t < 64 * NB; t += blockDim.x) {
        const int i = t % 64, j = t / 64;
        Ar[i][j] = (i < rows && j < kb) ? Fc[(int64_t)j * nf + r0 + i] : 0.0;
    }
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) Di[t % NB][t / NB] = Db[t];
    __syncthreads();
    // out[i][c] = sum_{t <= c} A[i][t] * Dinv[c][t]
    for (int t = threadIdx.x; t < 64 * NB; t += blockDim.x) {
        const int i = t % 64, c = t / 64;
        if (i >= rows || c >= kb) continue;
        double acc = 0.0;
        for (int u = 0; u <= c; ++u) acc += Ar[i][u] * Di[c][u];
        if constexpr (SIGNED) acc *= sgn[s.first + k0 + c];
        Fc[(int64_t)c * nf + r0 + i] = acc;
    }
}

// Trailing update F22 -= L21 L21^T over 64 x 64 tiles of the lower triangle (SIGNED:
// F22 -= L21 Sg L21^T).
template <bool SIGNED>
__global__ void __launch_bounds__(256) k_syrk_update(const SnDev* __restrict__ sn, const int* __restrict__ ids,
                                                     int k0, double* __restrict__ F, const double* __restrict__ sgn) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto Li = reinterpret_cast<double(*)[NB + 1]>(smem_raw);
    auto Lj = reinterpret_cast<double(*)[NB + 1]>(smem_raw + sizeof(double) * 64 * (NB + 1));
    const SnDev s = sn[ids[blockIdx.y]];
    if (k0 >= s.ns) return;
    const int kb = min(NB, s.ns - k0);
    const int nf = s.ns + s.nu;
    const int base = k0 + kb;
    const int m = nf - base;
    if (m <= 0) return;
    const int T = (m + 63) / 64;
    const int x = blockIdx.x;
    if (x >= T * (T + 1) / 2) return;
    int ti = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= x) ++ti;
    while (ti * (ti + 1) / 2 > x) --ti;
    const int tj = x - ti * (ti + 1) / 2;
    const int i0 = base + ti * 64, j0 = base + tj * 64;
    const double* Fc = F + s.front_off + (int64_t)k0 * nf;
    for (int t = threadIdx.x; t < 64 * NB; t += blockDim.x) {
        const int r = t % 64, c = t / 64;
        Li[r][c] = (i0 + r < nf && c < kb) ? Fc[(int64_t)c * nf + i0 + r] : 0.0;
        Lj[r][c] = (j0 + r < nf && c < kb) ? Fc[(int64_t)c * nf + j0 + r] : 0.0;
    }
    __syncthreads();
    const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;  // 4 x 4 outputs each
    double acc[4][4] = {};
    for (int c = 0; c < kb; ++c) {
        double a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { a[u] = Li[tr + 16 * u][c]; b[u] = Lj[tc + 16 * u][c]; }
        if constexpr (SIGNED) {
            const double sc = sgn[s.first + k0 + c];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] *= sc;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    double* Fo = F + s.front_off;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + tr + 16 * u, j = j0 + tc + 16 * v;
            if (i < nf && j < nf && i >= j) Fo[(int64_t)j * nf + i] -= acc[u][v];
        }
}

__global__ void k_copy_panels(const SnDev* __restrict__ sn, int nsn, const double* __restrict__ F,
                              double* __restrict__ L) {
    const SnDev s = sn[blockIdx.y];
    const int64_t count = (int64_t)(s.ns + s.nu) * s.ns;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        L[s.L_off + i] = F[s.front_off + i];
}


// ---- explicit panels G = [L11^{-1}; -L21 L11^{-1}] (factor time) ----------------------------------
// Running the blocked forward substitution of a supernode on the right-hand side [I; 0] yields
// L11^{-1} in the first ns rows and -L21 L11^{-1} below, so that the per-iteration solves become
// products with G only:  forward  [y; u] = G f_top + [0; f_bot],   backward  x = G^T [y; x_struct].
// G has the shape and column-major layout of the L panel (nf x ns, ld nf).

__global__ void k_g_init(const SnDev* __restrict__ sn, const int* __restrict__ ids, double* __restrict__ G) {
    const SnDev s = sn[ids[blockIdx.y]];
    const int nf = s.ns + s.nu;
    const int64_t total = (int64_t)nf * s.ns;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx % nf), c = (int)(idx / nf);
        G[s.L_off + idx] = (r == c) ? 1.0 : 0.0;
    }
}

// block row [k0, k0+kb) of G, columns [0, k0+kb):  G_blk := Dinv_blk G_blk   (column chunks of 64)
__global__ void __launch_bounds__(256) k_g_diag(const SnDev* __restrict__ sn, const int* __restrict__ ids, int k0,
                                                const double* __restrict__ Dinv, double* __restrict__ G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto Y = reinterpret_cast<double(*)[65]>(smem_raw);
    auto D = reinterpret_cast<double(*)[NB + 1]>(smem_raw + sizeof(double) * NB * 65);
    const SnDev s = sn[ids[blockIdx.y]];
    if (k0 >= s.ns) return;
    const int kb = min(NB, s.ns - k0);
    const int ncols = k0 + kb;
    const int c0 = blockIdx.x * 64;
    if (c0 >= ncols) return;
    const int cc = min(64, ncols - c0);
    const int nf = s.ns + s.nu;
    double* Gc = G + s.L_off;
    const double* Db = Dinv + s.Dinv_off + (int64_t)(k0 / NB) * NB * NB;
    for (int t = threadIdx.x; t < NB * 64; t += blockDim.x) {
        const int r = t % NB, j = t / NB;
        Y[r][j] = (r < kb && j < cc) ? Gc[(int64_t)(c0 + j) * nf + k0 + r] : 0.0;
    }
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) D[t % NB][t / NB] = Db[t];
    __syncthreads();
    for (int t = threadIdx.x; t < NB * 64; t += blockDim.x) {
        const int r = t % NB, j = t / NB;
        if (r >= kb || j >= cc) continue;
        double acc = 0.0;
        for (int u = 0; u <= r; ++u) acc = fma(D[r][u], Y[u][j], acc);
        Gc[(int64_t)(c0 + j) * nf + k0 + r] = acc;
    }
}

// rows >= k0+kb, columns [0, k0+kb):  G -= L[:, k0:k0+kb] G_blk   (64 x 64 tiles)
__global__ void __launch_bounds__(256) k_g_update(const SnDev* __restrict__ sn, const int* __restrict__ ids, int k0,
                                                  const double* __restrict__ L, double* __restrict__ G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto Lt = reinterpret_cast<double(*)[NB + 1]>(smem_raw);
    auto Yt = reinterpret_cast<double(*)[65]>(smem_raw + sizeof(double) * 64 * (NB + 1));
    const SnDev s = sn[ids[blockIdx.z]];
    if (k0 >= s.ns) return;
    const int kb = min(NB, s.ns - k0);
    const int nf = s.ns + s.nu;
    const int r0 = k0 + kb + blockIdx.x * 64;
    const int c0 = blockIdx.y * 64;
    if (r0 >= nf || c0 >= k0 + kb) return;
    const int rows = min(64, nf - r0), cols = min(64, k0 + kb - c0);
    const double* Lc = L + s.L_off;
    double* Gc = G + s.L_off;
    for (int t = threadIdx.x; t < 64 * NB; t += blockDim.x) {
        const int i = t % 64, c = t / 64;
        Lt[i][c] = (i < rows && c < kb) ? Lc[(int64_t)(k0 + c) * nf + r0 + i] : 0.0;
    }
    for (int t = threadIdx.x; t < NB * 64; t += blockDim.x) {
        const int r = t % NB, j = t / NB;
        Yt[r][j] = (r < kb && j < cols) ? Gc[(int64_t)(c0 + j) * nf + k0 + r] : 0.0;
    }
    __syncthreads();
    const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int c = 0; c < kb; ++c) {
        double a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { a[u] = Lt[tr + 16 * u][c]; b[u] = Yt[c][tc + 16 * u]; }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = tr + 16 * u, j = tc + 16 * v;
            if (i < rows && j < cols) Gc[(int64_t)(c0 + j) * nf + r0 + i] -= acc[u][v];
        }
}

// ---- per-iteration solve kernels (T = double or float) ---------------------------------------
// Forward: front vector f (nf rows) <- [R(perm) rows of the supernode; 0] + the children's
// bottom parts (each front row has at most one source row per child; src = -1 for none).
template <class T>
__global__ void k_fwd_assemble(const SnDev* __restrict__ sn, const int* __restrict__ ids,
                               const int32_t* __restrict__ perm, const int2* __restrict__ src,
                               const T* __restrict__ R, int64_t ldr, int p, T* __restrict__ fv, int64_t ldf) {
    const SnDev s = sn[ids[blockIdx.y]];
    const int nf = s.ns + s.nu;
    const int64_t total = (int64_t)nf * p;
    const SnDev* c0 = s.child0 >= 0 ? sn + s.child0 : nullptr;
    const SnDev* c1 = s.child1 >= 0 ? sn + s.child1 : nullptr;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / p), j = (int)(idx % p);
        T v = (r < s.ns) ? R[(int64_t)perm[s.first + r] * ldr + j] : T(0);
        const int2 sr = src[s.fv_off + r];
        if (sr.x >= 0) v += fv[(c0->fv_off + c0->ns + sr.x) * ldf + j];
        if (sr.y >= 0) v += fv[(c1->fv_off + c1->ns + sr.y) * ldf + j];
        fv[(s.fv_off + r) * ldf + j] = v;
    }
}

// One tile of a split-K product with G.  FWD: out rows [t0, t0+64) of nf, reduction over G
// columns [k0, k1) against f_top.  BWD: out columns [t0, t0+64) of ns, reduction over G rows
// [k0, k1) against z = [y; x(struct)].  Unsplit items write the result; split items write a
// partial that k_*_reduce sums in split order (deterministic).
struct SolveItem {
    int sn, t0, k0, k1, split, nsplit;
    int64_t part_row;   // first partial row of this supernode's split block (level-relative)
};

template <class T, int RC, bool BWD>
__global__ void __launch_bounds__(256) k_solve_gemm(const SnDev* __restrict__ sn, const SolveItem* __restrict__ items,
                                                    const T* __restrict__ G, const int64_t* __restrict__ srows,
                                                    int p, T* __restrict__ fv, int64_t ldf,
                                                    T* __restrict__ Y, T* __restrict__ X, int64_t ldx,
                                                    T* __restrict__ part) {
    __shared__ T Gt[32][65];
    __shared__ T Zt[32][RC + 1];
    const SolveItem it = items[blockIdx.x];
    const SnDev s = sn[it.sn];
    const int nf = s.ns + s.nu;
    const int j0 = blockIdx.y * RC;
    const int kc = min(RC, p - j0);
    const int nout = BWD ? s.ns : nf;
    constexpr int CPT = RC / 16;         // columns per thread
    const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;
    T acc[4][CPT];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < CPT; ++v) acc[u][v] = T(0);
    const T* Gs = G + s.L_off;
    for (int kk = it.k0; kk < it.k1; kk += 32) {
        if (!BWD) {
            for (int t = threadIdx.x; t < 32 * 64; t += blockDim.x) {
                const int i = t % 64, q = t / 64;   // coalesced over output rows
                const int row = it.t0 + i, k = kk + q;
                Gt[q][i] = (row < nf && k < it.k1) ? Gs[(int64_t)k * nf + row] : T(0);
            }
            for (int t = threadIdx.x; t < 32 * RC; t += blockDim.x) {
                const int q = t / RC, j = t % RC;
                const int k = kk + q;
                Zt[q][j] = (k < it.k1 && j < kc) ? fv[(s.fv_off + k) * ldf + j0 + j] : T(0);
            }
        } else {
            for (int t = threadIdx.x; t < 32 * 64; t += blockDim.x) {
                const int q = t % 32, i = t / 32;   // coalesced over G rows
                const int col = it.t0 + i, r = kk + q;
                Gt[q][i] = (col < s.ns && r < it.k1) ? Gs[(int64_t)col * nf + r] : T(0);
            }
            for (int t = threadIdx.x; t < 32 * RC; t += blockDim.x) {
                const int q = t / RC, j = t % RC;
                const int r = kk + q;
                T z = T(0);
                if (r < it.k1 && j < kc)
                    z = (r < s.ns) ? Y[(s.first + r) * ldx + j0 + j] : X[srows[s.struct_off + r - s.ns] * ldx + j0 + j];
                Zt[q][j] = z;
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < 32; ++q) {
            T a[4], b[CPT];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = Gt[q][tr + 16 * u];
#pragma unroll
            for (int v = 0; v < CPT; ++v) b[v] = Zt[q][tc + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < CPT; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int o = it.t0 + tr + 16 * u;
        if (o >= nout) continue;
#pragma unroll
        for (int v = 0; v < CPT; ++v) {
            const int j = tc + 16 * v;
            if (j >= kc) continue;
            if (it.nsplit > 1) {
                part[(it.part_row + (int64_t)it.split * nout + o) * ldf + j0 + j] = acc[u][v];
            } else if (BWD) {
                X[(s.first + o) * ldx + j0 + j] = acc[u][v];
            } else if (o < s.ns) {
                Y[(s.first + o) * ldx + j0 + j] = acc[u][v];
            } else {
                fv[(s.fv_off + o) * ldf + j0 + j] += acc[u][v];
            }
        }
    }
}

// ---- FP32 sweep products (the mixed form's step 6(a)) --------------------------------------------
// The same work items as k_solve_gemm, for T = float, shaped for the FP32 pipes and for HBM:
//  - a CTA computes a 64-row output tile for up to 32 TN columns of the right-hand sides, so for
//    k <= 256 columns every panel entry is read from HBM once per sweep;
//  - each thread holds an 8 x TN register tile (8 TN FMAs per 2 + TN/4 shared-memory vector loads);
//  - panel and right-hand-side tiles are staged by cp.async, two stages in flight;
//  - the forward sweep reads the column-major panels, the backward sweep a row-major copy, so both
//    stream contiguous rows of the panel for consecutive output indices.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(pred ? 4 : 0));
}
__device__ __forceinline__ void cp_async16(float* smem, const float* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

constexpr int SW_KT = 32;   // reduction rows per stage

template <int TN>
constexpr size_t sweep32_smem() { return (size_t)2 * SW_KT * (64 + 32 * TN) * sizeof(float); }

// column of the thread's v-th accumulator: for TN = 4 and 8 groups of 4 interleaved across the warp
// (each 16-byte shared load of a warp then covers 512 contiguous bytes), contiguous otherwise
template <int TN>
__device__ __forceinline__ int sweep_col(int cg, int v) {
    return (TN % 4 == 0) ? (v >> 2) * 128 + cg * 4 + (v & 3) : cg * TN + v;
}

template <int TN, bool BWD>
__global__ void __launch_bounds__(256) k_sweep32(const SnDev* __restrict__ sn, const SolveItem* __restrict__ items,
                                                 const float* __restrict__ Gc, const float* __restrict__ Gr,
                                                 const int64_t* __restrict__ srows, int p, float* __restrict__ fv,
                                                 int64_t ldf, float* __restrict__ Y, float* __restrict__ X,
                                                 int64_t ldx, float* __restrict__ part) {
    constexpr int COLS = 32 * TN;
    extern __shared__ __align__(16) float sw_smem[];
    float* Gt = sw_smem;                      // [2][SW_KT][64]
    float* Zt = sw_smem + 2 * SW_KT * 64;     // [2][SW_KT][COLS]
    const SolveItem it = items[blockIdx.x];
    const SnDev s = sn[it.sn];
    const int nf = s.ns + s.nu;
    const int j0 = blockIdx.y * COLS;
    const int kc = min(COLS, p - j0);
    const int nout = BWD ? s.ns : nf;
    const int r8 = threadIdx.x >> 5;          // output rows r8*8 .. r8*8+7 of the tile
    const int cg = threadIdx.x & 31;
    // panel entry (reduction index k, output index o): forward G(o, k) column-major, backward
    // G(k, o) from the row-major copy
    const float* Gb = (BWD ? Gr : Gc) + s.L_off;
    const int64_t gld = BWD ? s.ns : nf;

    auto load_stage = [&](int buf, int kk) {
        float* gt = Gt + buf * SW_KT * 64;
        float* zt = Zt + buf * SW_KT * COLS;
        for (int e = threadIdx.x; e < SW_KT * 64; e += 256) {
            const int q = e >> 6, i = e & 63;
            const int k = kk + q, o = it.t0 + i;
            const bool ok = k < it.k1 && o < nout;
            cp_async4(gt + e, ok ? Gb + (int64_t)k * gld + o : Gb, ok);
        }
        constexpr int V = COLS / 4;
        for (int e = threadIdx.x; e < SW_KT * V; e += 256) {
            const int q = e / V, j = (e % V) * 4;
            const int k = kk + q;
            int nb = 0;
            const float* src = fv;   // 16-byte aligned; nothing is read when nb = 0
            if (k < it.k1 && j < kc) {
                nb = 4 * min(4, kc - j);
                if (!BWD) src = fv + (s.fv_off + k) * ldf + j0 + j;
                else src = (k < s.ns) ? Y + (s.first + k) * ldx + j0 + j
                                      : X + srows[s.struct_off + k - s.ns] * ldx + j0 + j;
            }
            cp_async16(zt + q * COLS + j, src, nb);
        }
        cp_async_commit();
    };

    float acc[8][TN];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < TN; ++v) acc[u][v] = 0.f;
    const int nk = (it.k1 - it.k0 + SW_KT - 1) / SW_KT;
    load_stage(0, it.k0);
    for (int t = 0; t < nk; ++t) {
        if (t + 1 < nk) {
            load_stage((t + 1) & 1, it.k0 + (t + 1) * SW_KT);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float* gt = Gt + (t & 1) * SW_KT * 64 + r8 * 8;
        const float* zt = Zt + (t & 1) * SW_KT * COLS;
#pragma unroll 4
        for (int q = 0; q < SW_KT; ++q) {
            const float4 a0 = *reinterpret_cast<const float4*>(gt + q * 64);
            const float4 a1 = *reinterpret_cast<const float4*>(gt + q * 64 + 4);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float b[TN];
            if constexpr (TN % 4 == 0) {
#pragma unroll
                for (int g = 0; g < TN / 4; ++g) {
                    const float4 bv = *reinterpret_cast<const float4*>(zt + q * COLS + g * 128 + cg * 4);
                    b[4 * g] = bv.x; b[4 * g + 1] = bv.y; b[4 * g + 2] = bv.z; b[4 * g + 3] = bv.w;
                }
            } else if constexpr (TN % 2 == 0) {
#pragma unroll
                for (int g = 0; g < TN / 2; ++g) {
                    const float2 bv = *reinterpret_cast<const float2*>(zt + q * COLS + cg * TN + 2 * g);
                    b[2 * g] = bv.x; b[2 * g + 1] = bv.y;
                }
            } else {   // odd TN: scalar loads at an odd word stride, conflict-free
#pragma unroll
                for (int v = 0; v < TN; ++v) b[v] = zt[q * COLS + cg * TN + v];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < TN; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int o = it.t0 + r8 * 8 + u;
        if (o >= nout) continue;
#pragma unroll
        for (int v = 0; v < TN; ++v) {
            const int j = sweep_col<TN>(cg, v);
            if (j >= kc) continue;
            if (it.nsplit > 1) {
                part[(it.part_row + (int64_t)it.split * nout + o) * ldf + j0 + j] = acc[u][v];
            } else if (BWD) {
                X[(s.first + o) * ldx + j0 + j] = acc[u][v];
            } else if (o < s.ns) {
                Y[(s.first + o) * ldx + j0 + j] = acc[u][v];
            } else {
                fv[(s.fv_off + o) * ldf + j0 + j] += acc[u][v];
            }
        }
    }
}

// Sum the split partials of the supernodes listed in items (one item per (supernode, tile)),
// in split order, skipping the splits whose tiles were empty (see solve_items()).
template <class T, bool BWD>
__global__ void k_solve_reduce(const SnDev* __restrict__ sn, const SolveItem* __restrict__ items, int p,
                               const T* __restrict__ part, int64_t ldf, T* __restrict__ fv, T* __restrict__ Y,
                               T* __restrict__ X, int64_t ldx, int KS) {
    const SolveItem it = items[blockIdx.y];
    const SnDev s = sn[it.sn];
    const int nf = s.ns + s.nu;
    const int nout = BWD ? s.ns : nf;
    const int64_t total = (int64_t)64 * p;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int o = it.t0 + (int)(idx / p), j = (int)(idx % p);
        if (o >= nout) continue;
        T acc = T(0);
        for (int sp = 0; sp < it.nsplit; ++sp) {
            const int k0 = sp * KS;
            bool empty;
            if (BWD) empty = (k0 + KS <= it.t0);                               // rows all above the tile
            else empty = (it.t0 + 64 <= s.ns) && (k0 > it.t0 + 63);            // columns all right of the tile
            if (empty) continue;
            acc += part[(it.part_row + (int64_t)sp * nout + o) * ldf + j];
        }
        if (BWD) X[(s.first + o) * ldx + j] = acc;
        else if (o < s.ns) Y[(s.first + o) * ldx + j] = acc;
        else fv[(s.fv_off + o) * ldf + j] += acc;
    }
}

// P[perm[i]] = -x[i]
// Y[i, j] *= sgn[i]
template <class T>
__global__ void k_scale_rows(const double* __restrict__ sgn, T* __restrict__ Y, int64_t ld, int64_t n, int k) {
    const int64_t total = n * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int j = (int)(t - i * k);
        Y[i * ld + j] *= (T)sgn[i];
    }
}

template <class T>
__global__ void k_unpermute_neg(const int32_t* __restrict__ perm, const T* __restrict__ xp, int64_t ldx,
                                int64_t n, int k, T* __restrict__ P, int64_t ldp) {
    const int64_t total = n * k;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / k;
        const int j = (int)(idx % k);
        P[(int64_t)perm[i] * ldp + j] = -xp[i * ldx + j];
    }
}

inline int grid_for(int64_t work, int threads = 256) {
    return (int)std::min<int64_t>(std::max<int64_t>(1, (work + threads - 1) / threads), 1 << 16);
}

// two 64 x 65 tiles of T
template <class T>
constexpr size_t tile2_bytes() { return 2 * sizeof(T) * 64 * 65; }

template <class K>
int allow_smem(K kernel, size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return fail(HBSD_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    return 0;
}

// Split-K chunk of the solve products (columns of G forward, rows of G backward)
constexpr int SOLVE_KS = 128;

// Work items of one sweep of one level (see k_solve_gemm); partial rows are level-relative.
void solve_items(const Factor& f, int h, bool bwd, std::vector<SolveItem>& items, std::vector<SolveItem>& red,
                 int64_t* part_rows) {
    int64_t pr = 0;
    for (int q : f.levels[h]) {
        const Supernode& sn = f.sn[q];
        const int nf = sn.ns + sn.nu;
        const int nout = bwd ? sn.ns : nf;
        const int klen = bwd ? nf : sn.ns;
        const int nsplit = std::max(1, ceil_div(klen, SOLVE_KS));
        const int64_t base = pr;
        if (nsplit > 1) pr += (int64_t)nsplit * nout;
        for (int t0 = 0; t0 < nout; t0 += 64) {
            for (int sp = 0; sp < nsplit; ++sp) {
                const int k0 = sp * SOLVE_KS, k1 = std::min(klen, k0 + SOLVE_KS);
                const bool empty = bwd ? (k1 <= t0) : (t0 + 64 <= sn.ns && k0 > t0 + 63);
                if (empty) continue;
                items.push_back(SolveItem{q, t0, k0, k1, sp, nsplit, base});
            }
            if (nsplit > 1) red.push_back(SolveItem{q, t0, 0, klen, 0, nsplit, base});
        }
    }
    *part_rows = pr;
}

// Largest row count below the diagonal block [k0, k0+kb) over the fronts of a level, and the
// largest number of 64 x 64 lower-triangle tiles of the trailing matrix (grids must cover every
// front of the level, whose ns and nf differ).
void level_extent(const Factor& f, int h, int k0, int* max_rows, int* max_pairs) {
    int mr = 0, mp = 0;
    for (int q : f.levels[h]) {
        const Supernode& sn = f.sn[q];
        if (k0 >= sn.ns) continue;
        const int kb = std::min(NB, sn.ns - k0);
        const int rem = sn.ns + sn.nu - k0 - kb;
        mr = std::max(mr, rem);
        const int T = (rem + 63) / 64;
        mp = std::max(mp, T * (T + 1) / 2);
    }
    *max_rows = mr;
    *max_pairs = mp;
}

}  // namespace

int factor_build(Session* s, Factor& f, int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* aval, const int32_t* dof_node, const int32_t* grid, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    f.n = n;
    NDTree T;
    for (int e = 0; e < 3; ++e) T.g[e] = grid[e];
    const int64_t nnodes = (int64_t)grid[0] * grid[1] * grid[2];
    for (int64_t i = 0; i < n; ++i)
        if (dof_node[i] < 0 || dof_node[i] >= nnodes) return fail(HBSD_ERR_ARG, "dof_node out of range");
    const int lo[3] = {0, 0, 0}, hi[3] = {grid[0], grid[1], grid[2]};
    const bool per[3] = {true, true, true};
    const int root = T.build(lo, hi, per);
    if (root < 0) return fail(HBSD_ERR_ARG, "empty grid");
    // dofs of every mesh node
    std::vector<int64_t> nd_ptr(nnodes + 1, 0);
    for (int64_t i = 0; i < n; ++i) nd_ptr[dof_node[i] + 1]++;
    for (int64_t v = 0; v < nnodes; ++v) nd_ptr[v + 1] += nd_ptr[v];
    std::vector<int32_t> nd_dofs(n);
    {
        std::vector<int64_t> fill(nd_ptr.begin(), nd_ptr.end() - 1);
        for (int64_t i = 0; i < n; ++i) nd_dofs[fill[dof_node[i]]++] = (int32_t)i;
    }
    // postorder of the dissection tree -> supernodes (tree nodes without dofs are skipped)
    std::vector<int> post;
    {
        std::vector<std::pair<int, int>> stack{{root, 0}};
        while (!stack.empty()) {
            auto& top = stack.back();
            if (top.second < 2) {
                int c = T.kids[top.first][top.second++];
                if (c >= 0) stack.push_back({c, 0});
            } else {
                post.push_back(top.first);
                stack.pop_back();
            }
        }
    }
    std::vector<int> sn_of_tree(T.nodes.size(), -1);
    f.h_perm.clear();
    f.h_perm.reserve(n);
    f.sn.clear();
    for (int t : post) {
        std::vector<int32_t> mesh = T.nodes[t];
        std::sort(mesh.begin(), mesh.end());
        Supernode sn{};
        sn.first = (int64_t)f.h_perm.size();
        for (int32_t v : mesh)
            for (int64_t q = nd_ptr[v]; q < nd_ptr[v + 1]; ++q) f.h_perm.push_back(nd_dofs[q]);
        sn.ns = (int)((int64_t)f.h_perm.size() - sn.first);
        sn.parent = -1;
        sn.child[0] = sn.child[1] = -1;
        if (sn.ns == 0) continue;
        sn_of_tree[t] = (int)f.sn.size();
        f.sn.push_back(sn);
    }
    if ((int64_t)f.h_perm.size() != n) return fail(HBSD_ERR_ARG, "ordering does not cover every dof");
    // parent links: nearest ancestor that owns dofs
    for (int t : post) {
        const int me = sn_of_tree[t];
        if (me < 0) continue;
        int a = T.parent[t];
        while (a >= 0 && sn_of_tree[a] < 0) a = T.parent[a];
        if (a >= 0) {
            const int p = sn_of_tree[a];
            f.sn[me].parent = p;
            if (f.sn[p].child[0] < 0) f.sn[p].child[0] = me;
            else if (f.sn[p].child[1] < 0) f.sn[p].child[1] = me;
            else return fail(HBSD_ERR_ARG, "dissection tree node with more than two children");
        }
    }
    std::vector<int32_t> iperm(n);
    for (int64_t i = 0; i < n; ++i) iperm[f.h_perm[i]] = (int32_t)i;
    // symbolic: below-diagonal structure of each supernode (postorder = index order)
    const int nsn = (int)f.sn.size();
    std::vector<std::vector<int64_t>> st_rows(nsn);
    for (int q = 0; q < nsn; ++q) {
        Supernode& sn = f.sn[q];
        const int64_t last = sn.first + sn.ns;
        std::vector<int64_t> rows;
        for (int64_t c = sn.first; c < last; ++c) {
            const int32_t old = f.h_perm[c];
            for (int64_t e = row_ptr[old]; e < row_ptr[old + 1]; ++e) {
                const int64_t r = iperm[col_idx[e]];
                if (r >= last) rows.push_back(r);
            }
        }
        for (int ci = 0; ci < 2; ++ci) {
            const int c = sn.child[ci];
            if (c < 0) continue;
            for (int64_t r : st_rows[c])
                if (r >= last) rows.push_back(r);
        }
        std::sort(rows.begin(), rows.end());
        rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
        sn.nu = (int)rows.size();
        st_rows[q] = std::move(rows);
    }
    // heights
    int H = 0;
    for (int q = 0; q < nsn; ++q) {
        int h = 0;
        for (int ci = 0; ci < 2; ++ci)
            if (f.sn[q].child[ci] >= 0) h = std::max(h, f.sn[f.sn[q].child[ci]].level + 1);
        f.sn[q].level = h;
        H = std::max(H, h);
    }
    f.levels.assign(H + 1, {});
    for (int q = 0; q < nsn; ++q) f.levels[f.sn[q].level].push_back(q);
    // offsets (front storage ordered by level so a level is one contiguous range)
    std::vector<int64_t> front_off(nsn), level_front_begin(H + 2, 0);
    int64_t fo = 0;
    f.nnz_L = 0; f.fv_total = 0; f.dinv_total = 0; f.ea_total = 0;
    f.h_struct.clear();
    f.max_front = 0; f.max_ns = 0;
    int64_t L_tot = 0;
    for (int h = 0; h <= H; ++h) {
        level_front_begin[h] = fo;
        for (int q : f.levels[h]) {
            const int64_t nf = (int64_t)f.sn[q].ns + f.sn[q].nu;
            front_off[q] = fo;
            fo += nf * nf;
        }
    }
    level_front_begin[H + 1] = fo;
    for (int q = 0; q < nsn; ++q) {
        Supernode& sn = f.sn[q];
        const int64_t nf = (int64_t)sn.ns + sn.nu;
        sn.L_off = L_tot;
        L_tot += nf * sn.ns;
        f.nnz_L += nf * sn.ns - (int64_t)sn.ns * (sn.ns - 1) / 2;
        sn.Dinv_off = f.dinv_total;
        f.dinv_total += (int64_t)ceil_div(sn.ns, NB) * NB * NB;
        sn.fv_off = f.fv_total;
        f.fv_total += nf;
        sn.struct_off = (int64_t)f.h_struct.size();
        f.h_struct.insert(f.h_struct.end(), st_rows[q].begin(), st_rows[q].end());
        sn.ea_off = f.ea_total;
        f.ea_total += sn.nu;
        f.max_front = std::max<int>(f.max_front, (int)nf);
        f.max_ns = std::max(f.max_ns, sn.ns);
    }
    // extend-add maps: child struct row -> parent front row
    std::vector<int32_t> ea(std::max<int64_t>(1, f.ea_total));
    for (int q = 0; q < nsn; ++q) {
        const Supernode& c = f.sn[q];
        if (c.parent < 0) continue;
        const Supernode& p = f.sn[c.parent];
        const std::vector<int64_t>& prow = st_rows[c.parent];
        for (int r = 0; r < c.nu; ++r) {
            const int64_t g = st_rows[q][r];
            int32_t pos;
            if (g < p.first + p.ns) {
                if (g < p.first) return fail(HBSD_ERR_ARG, "symbolic: child row before parent columns");
                pos = (int32_t)(g - p.first);
            } else {
                auto it = std::lower_bound(prow.begin(), prow.end(), g);
                if (it == prow.end() || *it != g) return fail(HBSD_ERR_ARG, "symbolic: child row missing in parent");
                pos = (int32_t)(p.ns + (it - prow.begin()));
            }
            ea[c.ea_off + r] = pos;
        }
    }
    // matrix entries of each supernode's columns (lower triangle, permuted) -> front positions
    LevelLists& LL = f.LL;
    LL.offs.assign(H + 1, 0); LL.counts.assign(H + 1, 0);
    LL.max_ns.assign(H + 1, 0); LL.max_nf.assign(H + 1, 0); LL.max_nu.assign(H + 1, 0);
    for (int c = 0; c < 2; ++c) { LL.job_offs[c].assign(H + 1, 0); LL.job_counts[c].assign(H + 1, 0); }
    LL.entry_offs.assign(H + 2, 0);
    std::vector<int> ids, jobs;
    std::vector<int64_t> epos, esrc;
    for (int h = 0; h <= H; ++h) {
        LL.offs[h] = (int)ids.size();
        LL.counts[h] = (int)f.levels[h].size();
        for (int q : f.levels[h]) {
            ids.push_back(q);
            LL.max_ns[h] = std::max(LL.max_ns[h], f.sn[q].ns);
            LL.max_nu[h] = std::max(LL.max_nu[h], f.sn[q].nu);
            LL.max_nf[h] = std::max(LL.max_nf[h], f.sn[q].ns + f.sn[q].nu);
        }
    }
    for (int slot = 0; slot < 2; ++slot)
        for (int h = 0; h <= H; ++h) {
            LL.job_offs[slot][h] = (int)jobs.size() / 2;
            for (int q : f.levels[h])
                if (f.sn[q].child[slot] >= 0) { jobs.push_back(q); jobs.push_back(f.sn[q].child[slot]); }
            LL.job_counts[slot][h] = (int)jobs.size() / 2 - LL.job_offs[slot][h];
        }
    for (int h = 0; h <= H; ++h) {
        LL.entry_offs[h] = (int64_t)epos.size();
        for (int q : f.levels[h]) {
            const Supernode& sn = f.sn[q];
            const int64_t nf = (int64_t)sn.ns + sn.nu;
            const int64_t last = sn.first + sn.ns;
            const std::vector<int64_t>& rows = st_rows[q];
            for (int64_t c = sn.first; c < last; ++c) {
                const int32_t old = f.h_perm[c];
                for (int64_t e = row_ptr[old]; e < row_ptr[old + 1]; ++e) {
                    const int64_t r = iperm[col_idx[e]];
                    if (r < c) continue;
                    int64_t pr;
                    if (r < last) pr = r - sn.first;
                    else pr = sn.ns + (std::lower_bound(rows.begin(), rows.end(), r) - rows.begin());
                    epos.push_back(front_off[q] + (c - sn.first) * nf + pr);
                    esrc.push_back(e);
                }
            }
        }
    }
    LL.entry_offs[H + 1] = (int64_t)epos.size();
    // ---- device copies ----
    std::vector<SnDev> sd(nsn);
    for (int q = 0; q < nsn; ++q) {
        const Supernode& sn = f.sn[q];
        sd[q] = SnDev{sn.first, sn.L_off, sn.Dinv_off, sn.fv_off, sn.struct_off, sn.ea_off, front_off[q],
                      sn.ns, sn.nu, sn.child[0], sn.child[1]};
    }
    HBSD_TRY(f.d_sn.alloc(nsn * sizeof(SnDev) / sizeof(int) + 1));
    HBSD_CUDA(cudaMemcpy(f.d_sn.p, sd.data(), nsn * sizeof(SnDev), cudaMemcpyHostToDevice));
    HBSD_TRY(f.perm.alloc(n));
    HBSD_CUDA(cudaMemcpy(f.perm.p, f.h_perm.data(), n * 4, cudaMemcpyHostToDevice));
    HBSD_TRY(f.d_struct.alloc(std::max<size_t>(1, f.h_struct.size())));
    if (!f.h_struct.empty())
        HBSD_CUDA(cudaMemcpy(f.d_struct.p, f.h_struct.data(), f.h_struct.size() * 8, cudaMemcpyHostToDevice));
    HBSD_TRY(f.ea.alloc(ea.size()));
    HBSD_CUDA(cudaMemcpy(f.ea.p, ea.data(), ea.size() * 4, cudaMemcpyHostToDevice));
    HBSD_TRY(LL.ids.alloc(std::max<size_t>(1, ids.size())));
    HBSD_CUDA(cudaMemcpy(LL.ids.p, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice));
    HBSD_TRY(LL.jobs.alloc(std::max<size_t>(2, jobs.size())));
    if (!jobs.empty()) HBSD_CUDA(cudaMemcpy(LL.jobs.p, jobs.data(), jobs.size() * 4, cudaMemcpyHostToDevice));
    HBSD_TRY(LL.entry_pos.alloc(std::max<size_t>(1, epos.size())));
    HBSD_TRY(LL.entry_src.alloc(std::max<size_t>(1, esrc.size())));
    HBSD_CUDA(cudaMemcpy(LL.entry_pos.p, epos.data(), epos.size() * 8, cudaMemcpyHostToDevice));
    HBSD_CUDA(cudaMemcpy(LL.entry_src.p, esrc.data(), esrc.size() * 8, cudaMemcpyHostToDevice));
    DBuf<double> d_aval;
    HBSD_TRY(d_aval.alloc(row_ptr[n]));
    HBSD_CUDA(cudaMemcpy(d_aval.p, aval, row_ptr[n] * 8, cudaMemcpyHostToDevice));
    DBuf<double> fronts;
    HBSD_TRY(fronts.alloc(std::max<int64_t>(1, fo)));
    HBSD_TRY(f.Dinv.alloc(std::max<int64_t>(1, f.dinv_total)));
    DBuf<int> err;
    HBSD_TRY(err.alloc(2));
    const SnDev* dsn = reinterpret_cast<const SnDev*>(f.d_sn.p);
    HBSD_TRY(allow_smem(k_potrf_block<false>, tile2_bytes<double>()));
    HBSD_TRY(allow_smem(k_trsm_panel<false>, tile2_bytes<double>()));
    HBSD_TRY(allow_smem(k_syrk_update<false>, tile2_bytes<double>()));
    HBSD_TRY(allow_smem(k_potrf_block<true>, tile2_bytes<double>()));
    HBSD_TRY(allow_smem(k_trsm_panel<true>, tile2_bytes<double>()));
    HBSD_TRY(allow_smem(k_syrk_update<true>, tile2_bytes<double>()));
    // ---- numeric factorisation, level by level: Cholesky; on a non-positive pivot (eps_bar
    // inside the spectrum) once more in the signed LDL^T form ----
    f.signed_form = false;
    f.neg_pivots = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
    const bool sgnd = attempt == 1;
    if (sgnd) {
        HBSD_TRY(f.sgn.alloc(std::max<int64_t>(1, n)));
        f.signed_form = true;
    }
    HBSD_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(int), st));
    for (int h = 0; h <= H; ++h) {
        const int64_t fb = level_front_begin[h], fe = level_front_begin[h + 1];
        k_zero<<<grid_for(fe - fb), 256, 0, st>>>(fronts.p + fb, fe - fb);
        HBSD_LAUNCHED(s);
        const int64_t e0 = LL.entry_offs[h], e1 = LL.entry_offs[h + 1];
        if (e1 > e0) {
            k_scatter_entries<<<grid_for(e1 - e0), 256, 0, st>>>(LL.entry_pos.p + e0, LL.entry_src.p + e0, e1 - e0,
                                                                 d_aval.p, fronts.p);
            HBSD_LAUNCHED(s);
        }
        for (int slot = 0; slot < 2; ++slot) {
            const int nj = LL.job_counts[slot][h];
            if (nj == 0) continue;
            int64_t maxw = 0;
            for (int q : f.levels[h])
                if (f.sn[q].child[slot] >= 0) maxw = std::max<int64_t>(maxw, (int64_t)f.sn[f.sn[q].child[slot]].nu * f.sn[f.sn[q].child[slot]].nu);
            dim3 g(std::min(grid_for(maxw), 2048), nj);
            k_extend_add_matrix<<<g, 256, 0, st>>>(dsn, LL.jobs.p + 2 * LL.job_offs[slot][h], nj, f.ea.p, fronts.p);
            HBSD_LAUNCHED(s);
        }
        const int* lid = LL.ids.p + LL.offs[h];
        const int cnt = LL.counts[h];
        for (int k0 = 0; k0 < LL.max_ns[h]; k0 += NB) {
            if (sgnd) k_potrf_block<true><<<cnt, 256, tile2_bytes<double>(), st>>>(dsn, lid, cnt, k0, fronts.p, f.Dinv.p, err.p, f.sgn.p);
            else k_potrf_block<false><<<cnt, 256, tile2_bytes<double>(), st>>>(dsn, lid, cnt, k0, fronts.p, f.Dinv.p, err.p, nullptr);
            HBSD_LAUNCHED(s);
            int rem = 0, pairs = 0;
            level_extent(f, h, k0, &rem, &pairs);
            if (rem <= 0) continue;
            dim3 gt(ceil_div(rem, 64), cnt);
            if (sgnd) k_trsm_panel<true><<<gt, 256, tile2_bytes<double>(), st>>>(dsn, lid, k0, fronts.p, f.Dinv.p, f.sgn.p);
            else k_trsm_panel<false><<<gt, 256, tile2_bytes<double>(), st>>>(dsn, lid, k0, fronts.p, f.Dinv.p, nullptr);
            HBSD_LAUNCHED(s);
            dim3 gs(pairs, cnt);
            if (sgnd) k_syrk_update<true><<<gs, 256, tile2_bytes<double>(), st>>>(dsn, lid, k0, fronts.p, f.sgn.p);
            else k_syrk_update<false><<<gs, 256, tile2_bytes<double>(), st>>>(dsn, lid, k0, fronts.p, nullptr);
            HBSD_LAUNCHED(s);
        }
    }
    int herr[2] = {0, 0};
    HBSD_CUDA(cudaMemcpyAsync(herr, err.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (!herr[0]) {
        f.neg_pivots = herr[1];
        break;
    }
    if (sgnd) return fail(HBSD_ERR_NOT_SPD, "factorisation of H - sigma_bar S met a zero or non-finite pivot");
    }
    HBSD_TRY(f.L.alloc(std::max<int64_t>(1, L_tot)));
    {
        int64_t maxp = 1;
        for (int q = 0; q < nsn; ++q) maxp = std::max<int64_t>(maxp, ((int64_t)f.sn[q].ns + f.sn[q].nu) * f.sn[q].ns);
        dim3 g(std::min(grid_for(maxp), 1024), nsn);
        k_copy_panels<<<g, 256, 0, st>>>(dsn, nsn, fronts.p, f.L.p);
        HBSD_LAUNCHED(s);
    }
    HBSD_CUDA(cudaStreamSynchronize(st));
    fronts.release();
    // explicit panels G = [L11^{-1}; -L21 L11^{-1}]: forward substitution on [I; 0], level-batched
    HBSD_TRY(f.G.alloc(std::max<int64_t>(1, L_tot)));
    HBSD_TRY(allow_smem(k_g_diag, tile2_bytes<double>()));
    HBSD_TRY(allow_smem(k_g_update, tile2_bytes<double>()));
    for (int h = 0; h <= H; ++h) {
        const int* lid = LL.ids.p + LL.offs[h];
        const int cnt = LL.counts[h];
        int64_t maxp = 1;
        for (int q : f.levels[h]) maxp = std::max<int64_t>(maxp, ((int64_t)f.sn[q].ns + f.sn[q].nu) * f.sn[q].ns);
        dim3 gi(std::min(grid_for(maxp), 1024), cnt);
        k_g_init<<<gi, 256, 0, st>>>(dsn, lid, f.G.p);
        HBSD_LAUNCHED(s);
        for (int k0 = 0; k0 < LL.max_ns[h]; k0 += NB) {
            const int ncols = k0 + std::min(NB, LL.max_ns[h] - k0);
            dim3 gd(ceil_div(ncols, 64), cnt);
            k_g_diag<<<gd, 256, tile2_bytes<double>(), st>>>(dsn, lid, k0, f.Dinv.p, f.G.p);
            HBSD_LAUNCHED(s);
            int rem = 0, pairs = 0;
            level_extent(f, h, k0, &rem, &pairs);
            if (rem <= 0) continue;
            dim3 gu(ceil_div(rem, 64), ceil_div(ncols, 64), cnt);
            k_g_update<<<gu, 256, tile2_bytes<double>(), st>>>(dsn, lid, k0, f.L.p, f.G.p);
            HBSD_LAUNCHED(s);
        }
    }
    // extend-add sources of every front row (pull form of the solve's extend-add)
    {
        std::vector<int2> src(std::max<int64_t>(1, f.fv_total), make_int2(-1, -1));
        for (int q = 0; q < nsn; ++q) {
            const Supernode& c = f.sn[q];
            if (c.parent < 0) continue;
            const Supernode& pa = f.sn[c.parent];
            const int slot = (pa.child[0] == q) ? 0 : 1;
            for (int r = 0; r < c.nu; ++r) {
                int2& e = src[pa.fv_off + ea[c.ea_off + r]];
                if (slot == 0) e.x = r; else e.y = r;
            }
        }
        HBSD_TRY(f.src.alloc(src.size()));
        HBSD_CUDA(cudaMemcpy(f.src.p, src.data(), src.size() * sizeof(int2), cudaMemcpyHostToDevice));
    }
    // solve work lists
    {
        f.sweep.assign(2 * (H + 1), {});
        std::vector<SolveItem> all_items, all_red;
        f.part_rows = 0;
        for (int h = 0; h <= H; ++h)
            for (int b = 0; b < 2; ++b) {
                std::vector<SolveItem> items, red;
                int64_t pr = 0;
                solve_items(f, h, b == 1, items, red, &pr);
                Factor::Sweep& sw = f.sweep[2 * h + b];
                sw.item_off = (int)all_items.size();
                sw.n_items = (int)items.size();
                sw.red_off = (int)all_red.size();
                sw.n_red = (int)red.size();
                all_items.insert(all_items.end(), items.begin(), items.end());
                all_red.insert(all_red.end(), red.begin(), red.end());
                f.part_rows = std::max(f.part_rows, pr);
            }
        const size_t isz = sizeof(SolveItem);
        HBSD_TRY(f.items.alloc((std::max<size_t>(1, all_items.size()) * isz + 7) / 8));
        HBSD_TRY(f.red_items.alloc((std::max<size_t>(1, all_red.size()) * isz + 7) / 8));
        if (!all_items.empty())
            HBSD_CUDA(cudaMemcpy(f.items.p, all_items.data(), all_items.size() * isz, cudaMemcpyHostToDevice));
        if (!all_red.empty())
            HBSD_CUDA(cudaMemcpy(f.red_items.p, all_red.data(), all_red.size() * isz, cudaMemcpyHostToDevice));
    }
    HBSD_CUDA(cudaStreamSynchronize(st));
    auto t1 = std::chrono::steady_clock::now();
    s->stats.t_factor_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    s->stats.nnz_L = f.nnz_L;
    s->stats.neg_pivots = f.neg_pivots;
    s->stats.n_supernodes = nsn;
    return 0;
}

// FP32 panels of the diagonally scaled matrix D A D (D in the permuted order): with
// L^ = D L, the panel G^ = [L11^{-1} D_s^{-1}; D_u M21 D_s^{-1}], i.e. column c divided by the
// scale of the supernode's c-th dof and rows below the diagonal block multiplied by theirs.
__global__ void k_g_to_float_scaled(const SnDev* __restrict__ sn, const double* __restrict__ G,
                                    const int32_t* __restrict__ perm, const int64_t* __restrict__ srows,
                                    const double* __restrict__ d, float* __restrict__ G32) {
    const SnDev s = sn[blockIdx.y];
    const int nf = s.ns + s.nu;
    const int64_t total = (int64_t)nf * s.ns;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx % nf), c = (int)(idx / nf);
        const double rho = (r < s.ns) ? 1.0 : d[perm[srows[s.struct_off + r - s.ns]]];
        G32[s.L_off + idx] = (float)(rho * G[s.L_off + idx] / d[perm[s.first + c]]);
    }
}

// The same FP32 panel values row-major: entry (r, c) of a supernode's panel at L_off + r ns + c.
__global__ void k_panel_transpose32(const SnDev* __restrict__ sn, const float* __restrict__ Gc,
                                    float* __restrict__ Gr) {
    const SnDev s = sn[blockIdx.y];
    const int nf = s.ns + s.nu;
    const int64_t total = (int64_t)nf * s.ns;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / s.ns), c = (int)(idx % s.ns);
        Gr[s.L_off + idx] = Gc[s.L_off + (int64_t)c * nf + r];
    }
}

int factor_make_fp32(Factor& f, const double* dscale, cudaStream_t st) {
    if (f.G32.p) return 0;
    HBSD_TRY(f.G32.alloc(f.G.n));
    HBSD_TRY(f.G32T.alloc(f.G.n));
    const int nsn = (int)f.sn.size();
    int64_t maxp = 1;
    for (int q = 0; q < nsn; ++q) maxp = std::max<int64_t>(maxp, ((int64_t)f.sn[q].ns + f.sn[q].nu) * f.sn[q].ns);
    dim3 g(std::min(grid_for(maxp), 1024), nsn);
    k_g_to_float_scaled<<<g, 256, 0, st>>>(reinterpret_cast<const SnDev*>(f.d_sn.p), f.G.p, f.perm.p, f.d_struct.p,
                                           dscale, f.G32.p);
    HBSD_CUDA(cudaPeekAtLastError());
    k_panel_transpose32<<<g, 256, 0, st>>>(reinterpret_cast<const SnDev*>(f.d_sn.p), f.G32.p, f.G32T.p);
    HBSD_CUDA(cudaPeekAtLastError());
    return 0;
}

template <int TN, bool BWD>
static int launch_sweep32(Session* s, Factor& f, dim3 g, const SolveItem* it, int k, float* fv, int64_t ld, float* Y,
                          float* X, float* part, cudaStream_t st) {
    constexpr size_t smem = sweep32_smem<TN>();
    if (smem > 48 * 1024) {   // the cap, once: concurrent sessions never lower it under each other
        static std::once_flag once;
        static cudaError_t e = cudaSuccess;
        std::call_once(once, [] {
            e = cudaFuncSetAttribute(k_sweep32<TN, BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        });
        HBSD_CUDA(e);
    }
    k_sweep32<TN, BWD><<<g, 256, smem, st>>>(reinterpret_cast<const SnDev*>(f.d_sn.p), it, f.G32.p, f.G32T.p,
                                             f.d_struct.p, k, fv, ld, Y, X, ld, part);
    HBSD_LAUNCHED(s);
    return 0;
}

template <class T> struct FactorData;
template <> struct FactorData<double> {
    static const double* G(Factor& f) { return f.G.p; }
    static DBuf<double>& ws(Factor& f) { return f.sws; }
};
template <> struct FactorData<float> {
    static const float* G(Factor& f) { return f.G32.p; }
    static DBuf<float>& ws(Factor& f) { return f.sws32; }
};

// P = -(L L^T)^{-1} R for a k-column block: forward sweep (levels bottom-up), backward sweep
// (levels top-down), each level one split-K product with G plus, for split supernodes, one
// deterministic reduction.
template <class T>
int factor_solve(Session* s, Factor& f, const T* R, int64_t ldr, int k, T* P, int64_t ldp, cudaStream_t st) {
    if (k <= 0) return 0;
    const T* G = FactorData<T>::G(f);
    if (!G) return fail(HBSD_ERR_ARG, "factor_solve: factor not available in this precision");
    const int64_t ld = round_up(k, 4);
    // workspace: front vectors | y | x | split partials
    const int64_t rows = f.fv_total + 2 * f.n + f.part_rows;
    HBSD_TRY(FactorData<T>::ws(f).alloc((size_t)rows * ld));
    T* fv = FactorData<T>::ws(f).p;
    T* Y = fv + f.fv_total * ld;
    T* X = Y + f.n * ld;
    T* part = X + f.n * ld;
    LevelLists& LL = f.LL;
    const SnDev* dsn = reinterpret_cast<const SnDev*>(f.d_sn.p);
    const SolveItem* items = reinterpret_cast<const SolveItem*>(f.items.p);
    const SolveItem* red = reinterpret_cast<const SolveItem*>(f.red_items.p);
    const int H = (int)f.levels.size() - 1;
    const bool narrow = k <= 16;
    const int rc = narrow ? 16 : 64;
    const int rchunks = ceil_div(k, rc);
    // FP32: TN columns per thread, 32 TN per CTA, the smallest TN whose tile holds all k columns
    const int tn = std::min(8, ceil_div(k, 32));
    auto gemm = [&](int h, bool bwd) -> int {
        const Factor::Sweep& sw = f.sweep[2 * h + (bwd ? 1 : 0)];
        if (sw.n_items > 0 && std::is_same<T, float>::value && f.G32T.p) {
            float* fv32 = reinterpret_cast<float*>(fv);
            float* Y32 = reinterpret_cast<float*>(Y);
            float* X32 = reinterpret_cast<float*>(X);
            float* part32 = reinterpret_cast<float*>(part);
            dim3 g(sw.n_items, ceil_div(k, 32 * tn));
            const SolveItem* it = items + sw.item_off;
            int rc = 0;
            auto go = [&](auto tn_c, auto bwd_c) {
                return launch_sweep32<decltype(tn_c)::value, decltype(bwd_c)::value>(s, f, g, it, k, fv32, ld, Y32,
                                                                                      X32, part32, st);
            };
            auto pick = [&](auto bwd_c) {
                switch (tn) {
                    case 1: return go(std::integral_constant<int, 1>{}, bwd_c);
                    case 2: return go(std::integral_constant<int, 2>{}, bwd_c);
                    case 3: return go(std::integral_constant<int, 3>{}, bwd_c);
                    case 4: return go(std::integral_constant<int, 4>{}, bwd_c);
                    case 5: return go(std::integral_constant<int, 5>{}, bwd_c);
                    case 6: return go(std::integral_constant<int, 6>{}, bwd_c);
                    case 7: return go(std::integral_constant<int, 7>{}, bwd_c);
                    default: return go(std::integral_constant<int, 8>{}, bwd_c);
                }
            };
            rc = bwd ? pick(std::true_type{}) : pick(std::false_type{});
            HBSD_TRY(rc);
        } else if (sw.n_items > 0) {
            dim3 g(sw.n_items, rchunks);
            const SolveItem* it = items + sw.item_off;
            if (bwd) {
                if (narrow) k_solve_gemm<T, 16, true><<<g, 256, 0, st>>>(dsn, it, G, f.d_struct.p, k, fv, ld, Y, X, ld, part);
                else k_solve_gemm<T, 64, true><<<g, 256, 0, st>>>(dsn, it, G, f.d_struct.p, k, fv, ld, Y, X, ld, part);
            } else {
                if (narrow) k_solve_gemm<T, 16, false><<<g, 256, 0, st>>>(dsn, it, G, f.d_struct.p, k, fv, ld, Y, X, ld, part);
                else k_solve_gemm<T, 64, false><<<g, 256, 0, st>>>(dsn, it, G, f.d_struct.p, k, fv, ld, Y, X, ld, part);
            }
            HBSD_LAUNCHED(s);
        }
        if (sw.n_red > 0) {
            dim3 g(ceil_div((int64_t)64 * k, 256), sw.n_red);
            if (bwd) k_solve_reduce<T, true><<<g, 256, 0, st>>>(dsn, red + sw.red_off, k, part, ld, fv, Y, X, ld, SOLVE_KS);
            else k_solve_reduce<T, false><<<g, 256, 0, st>>>(dsn, red + sw.red_off, k, part, ld, fv, Y, X, ld, SOLVE_KS);
            HBSD_LAUNCHED(s);
        }
        return 0;
    };
    for (int h = 0; h <= H; ++h) {
        dim3 gi(std::min(grid_for((int64_t)LL.max_nf[h] * k), 1024), LL.counts[h]);
        k_fwd_assemble<T><<<gi, 256, 0, st>>>(dsn, LL.ids.p + LL.offs[h], f.perm.p, f.src.p, R, ldr, k, fv, ld);
        HBSD_LAUNCHED(s);
        HBSD_TRY(gemm(h, false));
    }
    if (f.signed_form) {   // x = Lt^{-T} Sg Lt^{-1} r: the pivot signs between the sweeps
        k_scale_rows<T><<<grid_for(f.n * k), 256, 0, st>>>(f.sgn.p, Y, ld, f.n, k);
        HBSD_LAUNCHED(s);
    }
    for (int h = H; h >= 0; --h) HBSD_TRY(gemm(h, true));
    k_unpermute_neg<T><<<grid_for(f.n * k), 256, 0, st>>>(f.perm.p, X, ld, f.n, k, P, ldp);
    HBSD_LAUNCHED(s);
    return 0;
}

template int factor_solve<double>(Session*, Factor&, const double*, int64_t, int, double*, int64_t, cudaStream_t);
template int factor_solve<float>(Session*, Factor&, const float*, int64_t, int, float*, int64_t, cudaStream_t);

}  // namespace hbsd
