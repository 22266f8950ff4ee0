// Step 6(b) of LABPSD: locally accelerated refinement (Sec. 3 hybrid scheme, Sec. 4, Eq. indls).
// For each refined column j, MINRES (Paige & Saunders 1975) on the Hermitian indefinite system
// (H - eps_j S) p = -r_j started from the globally preconditioned p_j, stopped when the
// recurrence residual estimate drops to eta ||r_j|| (Eq. approxp) or after max_minres steps.
//
// One cooperative (co-resident) launch runs every step of every column.  The refined columns
// advance in lockstep; each step is three phases separated by grid barriers:
//   A. U = (H - e_j S) V for the columns still iterating (SELL-C-sigma rows, lanes over the
//      columns), with per-block partial sums of alpha_j = v_j . u_j;
//   B. u_j -= alpha_j v_j + beta_j v_{j-1}, with per-block partials of ||u_j||^2;
//   C. the Givens update of the QR factorisation of the Lanczos tridiagonal, then the
//      direction, iterate and Lanczos-vector updates.
// The per-column scalar recurrences are replicated in every block's shared memory: every block
// reduces the per-block partials in the same fixed order, so all copies agree bit for bit and
// nothing has to be broadcast.  A column that has met its tolerance keeps its iterate, stops
// updating and leaves the SpMM.  The grid barrier is an arrival counter whose wait is bounded
// by %globaltimer: a block that waits past the limit raises the error flag and every block
// returns; the host reports HBSD_ERR_TIMEOUT.
// With a nonlocal term H_nl = F G F^T (Eq. fgf) phase A adds F (G (F^T v_j)) to each row.
// F^T v_{j+1} = F^T u_j / beta_{j+1} is gathered in phase C, when every u_j is final: block c
// sums the rows of its chunk of F against U into per-chunk partials; after the barrier each
// block reduces, in a fixed order, only the projectors its own rows meet (and those coupled to
// them through G), so the step keeps its three barriers.  The start takes one more.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "common.h"

namespace hbsd {

namespace {

constexpr int MR_THREADS = 512;
constexpr int MR_PASS = 128;                      // columns per pass (>= 4 rows per block step)
constexpr uint64_t MR_WAIT_NS = 2000000000ull;   // grid-barrier wait limit (2 s)
constexpr size_t MR_SMEM_MAX = 64 * 1024;

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// bar[0]: arrivals, bar[1]: generation.  Returns false (for the whole block) when the wait
// timed out here or another block has raised the error flag.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned& gen, int* err, int* ok_sm,
                             uint64_t wait_ns = MR_WAIT_NS) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned old = atomicAdd(&bar[0], 1u);
        if (old == nblocks - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            const uint64_t t0 = gtimer();
            while (ld_acquire(&bar[1]) == gen) {
                if (ld_relaxed(err)) { ok = 0; break; }
                if (gtimer() - t0 > wait_ns) { atomicExch(err, 1); ok = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        gen += 1;
        *ok_sm = ok;
    }
    __syncthreads();
    return *ok_sm != 0;
}

// Failure path of the grid barrier: the blocks of this launch wait for one more arrival than
// there are blocks, so the wait can only end by its time limit; each block then raises the error
// flag and returns (err[1] counts the blocks that returned).
__global__ void k_barrier_probe(unsigned* bar, int* err, uint64_t wait_ns) {
    __shared__ int ok_sm;
    unsigned gen = 0;
    const bool ok = grid_barrier(bar, gridDim.x + 1, gen, err, &ok_sm, wait_ns);
    if (!ok && threadIdx.x == 0) atomicAdd(err + 1, 1);
}

struct MrArgs {
    // SELL-C-sigma pattern with interleaved (h - sigma0 s, s)
    const int64_t* slice_ptr;
    const int32_t* slice_len;
    const int32_t* cols;
    const void* hs;
    const int32_t* slot_row;
    int64_t n_slots;
    const int64_t* blk;   // gridDim + 1 slot boundaries, balanced by stored entries
    int C;
    int64_t n;
    int k;
    const void* R;
    int64_t ldr;
    const void* e;
    void* X;
    int64_t ldx;
    void *V, *Vp, *U, *Wp, *Wpp;
    int64_t ld;
    double* part;   // [2][gridDim][kp] per-block partial sums
    int64_t kp;
    double eta;
    int maxit;
    int* steps_out;   // k ints (block 0 writes)
    unsigned* bar;
    int* err;
    unsigned long long* stamps;   // nullable: phase times (ns) seen by block 0, for tracing
    // nonlocal term (nl_k = 0: none); index built by nl_minres_index for this grid
    int nl_k;
    const int64_t* nl_rptr;       // F by row (all n rows)
    const int32_t* nl_rcol;
    const double* nl_rval;
    const int32_t* nl_frows;      // rows with F entries, in chunk order
    const int64_t* nl_ch_row_off; // chunk c: frows[ch_row_off[c] .. ch_row_off[c+1])
    const int32_t* nl_ch_lptr;    // chunk c: projector slots [ch_lptr[c], ch_lptr[c+1])
    const double* nl_pan;         // chunk c: rows x slots panel at pan_off[c]
    const int64_t* nl_pan_off;
    const int32_t* nl_cl_ptr;     // projector l: chunk slots cl_slot[cl_ptr[l] .. cl_ptr[l+1])
    const int32_t* nl_cl_slot;
    const int32_t* nl_nb_ptr;     // block b: projectors nb_l[nb_ptr[b] ..], the first napply[b] applied
    const int32_t* nl_nb_napply;
    const int32_t* nl_nb_l;
    const int32_t* nl_lmap;       // [b * nl_k + l]: local index of projector l in block b, or -1
    const int32_t* nl_sf_ptr;     // per SELL slot: F entries sf_ptr[slot] .. sf_ptr[slot+1] with
    const int32_t* nl_sf_off;     //   the zg row they read (nb_ptr[b] + local index)
    const double* nl_sf_val;      //   and the value F(row, l)
    const int32_t* nl_gptr;       // G by rows
    const int32_t* nl_gcol;
    const double* nl_gval;
    double* nl_part;              // [chunk slot][kp] partials of F^T U
    double* nl_zv;                // [block slot][kp] F^T v
    double* nl_zg;                // [block slot][kp] G F^T v
    // operator products of the Lanczos steps from the FP32 scaled pencil (f32 = 1):
    // (Hs - e S) v = D^-1 [(D Hs D) - e (D S D)] (D^-1 v), v^ = D^-1 v kept in FP32 beside V
    int f32;
    const float2* hs32;           // (D Hs D, D S D) per stored entry
    const double* dinv;           // D^-1 (n)
    float* V32;                   // v^ = D^-1 v, layout of V
};

template <class T> struct Pair;
template <> struct Pair<double> { using P = double2; };
template <> struct Pair<float> { using P = float2; };

// One pass over nc (<= MR_PASS) columns: the block's threads are flattened over (row, column)
// pairs, thread t -> row r = t / nc of the current group of rb = blockDim / nc rows, column
// c = t % nc, so that almost every lane does useful work for any column count.
struct Pass {
    int c0, nc, rb, r, c;
};
__device__ __forceinline__ Pass make_pass(int c0, int na) {
    Pass p;
    p.c0 = c0;
    p.nc = min(MR_PASS, na - c0);
    p.rb = (int)blockDim.x / p.nc;
    p.r = (int)threadIdx.x / p.nc;
    p.c = (int)threadIdx.x - p.r * p.nc;
    return p;
}

// Block reduction of the per-thread partials (one column per thread) into part_row[c0 + c]:
// a pairwise tree over the rb row slots, the same order in every block and every run.
__device__ void block_partials(double acc, const Pass& p, double* red, double* part_row) {
    const bool on = p.r < p.rb;
    if (on) red[threadIdx.x] = acc;
    __syncthreads();
    int top = 1;
    while (top < p.rb) top <<= 1;
    for (int sdist = top >> 1; sdist >= 1; sdist >>= 1) {
        if (on && p.r < sdist && p.r + sdist < p.rb) red[threadIdx.x] += red[threadIdx.x + sdist * p.nc];
        __syncthreads();
    }
    if (on && p.r == 0) part_row[p.c0 + p.c] = red[p.c];
    __syncthreads();
}

// out[pos] = sum over blocks of part[b * kp + pos] in a fixed order (one warp per position,
// lanes stride over the blocks, then a shuffle tree); every block computes identical values.
__device__ void grid_sum(const double* part, int64_t kp, int na, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int pos = warp; pos < na; pos += nw) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += part[(int64_t)b * kp + pos];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[pos] = s;
    }
    __syncthreads();
}

// Shared-memory column state (k entries per field), replicated in every block: one base
// pointer and k, fields at fixed multiples of k (keeps the state out of registers).
enum DField { F_BETA_OLD, F_C_PREV, F_S_PREV, F_C_PP, F_S_PP, F_PHIBAR, F_TOL, F_ALPHA, F_BETA_NEXT, F_PHI, F_GINV,
              F_BINV, F_DELTA, F_EPS, F_RED1, F_RED2, MR_DFIELDS };
enum IField { I_ACTIVE, I_UPD, I_CONT, I_STEPS, I_ACT, MR_IFIELDS };
struct ColState {
    double* d;   // MR_DFIELDS x k
    int* i;      // MR_IFIELDS x k, then nact
    int k;
    double* red; // blockDim doubles for block_partials
    __device__ __forceinline__ double* f(DField x) const { return d + (int64_t)x * k; }
    __device__ __forceinline__ int* g(IField x) const { return i + (int64_t)x * k; }
    __device__ __forceinline__ int* nact() const { return i + (int64_t)MR_IFIELDS * k; }
};

__device__ __forceinline__ ColState col_state(double* smem, int k) {
    ColState s;
    s.red = smem;
    s.d = smem + MR_THREADS;
    s.i = reinterpret_cast<int*>(s.d + (int64_t)MR_DFIELDS * k);
    s.k = k;
    return s;
}

size_t mr_smem_bytes(int k) {
    return ((size_t)MR_THREADS + (size_t)MR_DFIELDS * k) * sizeof(double) +
           (size_t)(MR_IFIELDS * k + 2) * sizeof(int);
}

// Nonlocal row term sum_e F(row, l_e) (G F^T v)(l_e, j) of one SELL slot, from this block's
// reduced values: the slot's entries carry the row of zg they read.
__device__ __forceinline__ double nl_slot(const MrArgs& a, int64_t slot, int j) {
    double s = 0.0;
    const int e1 = a.nl_sf_ptr[slot + 1];
    for (int e = a.nl_sf_ptr[slot]; e < e1; ++e) s = fma(a.nl_sf_val[e], a.nl_zg[(int64_t)a.nl_sf_off[e] * a.kp + j], s);
    return s;
}

// Chunk partials of F^T Src for the columns jcol(0 .. cnt-1) with keep(j): block c writes
// nl_part[(ch_lptr[c] + t) * kp + j] = scale(j) * sum_r panel(r, t) Src(frows[r], j).
// Threads form groups of rs lanes (a power of two); a group takes one column and its lanes
// interleave over the chunk's rows, four projectors at a time, then a shuffle tree sums the
// group (fixed order).  One load of Src per (row, column) and group of four projectors.
template <class J, class K, class Sc>
__device__ void nl_chunk_partial(const MrArgs& a, const double* Src, int64_t lds, int cnt, J&& jcol, K&& keep,
                                 Sc&& scale) {
    const int c = blockIdx.x;
    const int l0 = a.nl_ch_lptr[c], nlc = a.nl_ch_lptr[c + 1] - l0;
    const int64_t r0 = a.nl_ch_row_off[c];
    const int nr = (int)(a.nl_ch_row_off[c + 1] - r0);
    if (nlc == 0 || cnt == 0) return;
    const double* pan = a.nl_pan + a.nl_pan_off[c];
    int rs = 32;
    while (rs > 1 && rs * cnt > (int)blockDim.x) rs >>= 1;
    const int sub = threadIdx.x & (rs - 1);
    const int ngrp = (int)blockDim.x / rs;
    for (int q = threadIdx.x / rs; q - (int)threadIdx.x / rs < cnt; q += ngrp) {
        // every lane of a warp runs the same trip count (its groups share the loop bounds), so
        // the shuffles below see full warps; idle groups carry zeros
        const bool on = q < cnt;
        const int j = on ? jcol(q) : 0;
        const bool use = on && keep(j);
        for (int t0 = 0; t0 < nlc; t0 += 4) {
            double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
            if (use) {
                // four rows per trip: their index and value loads are issued together
                for (int rb = sub; rb < nr; rb += 4 * rs) {
                    int ri[4];
                    double x[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int r = rb + u * rs;
                        ri[u] = r < nr ? a.nl_frows[r0 + r] : -1;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) x[u] = ri[u] >= 0 ? Src[(int64_t)ri[u] * lds + j] : 0.0;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int r = rb + u * rs;
                        if (r >= nr) break;
                        const double* pr = pan + (int64_t)r * nlc + t0;
                        acc0 = fma(pr[0], x[u], acc0);
                        if (t0 + 1 < nlc) acc1 = fma(pr[1], x[u], acc1);
                        if (t0 + 2 < nlc) acc2 = fma(pr[2], x[u], acc2);
                        if (t0 + 3 < nlc) acc3 = fma(pr[3], x[u], acc3);
                    }
                }
            }
            for (int o = rs >> 1; o > 0; o >>= 1) {
                acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
                acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
                acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
                acc3 += __shfl_xor_sync(0xffffffffu, acc3, o);
            }
            if (use && sub == 0) {
                const double sc = scale(j);
                double* out = a.nl_part + (int64_t)(l0 + t0) * a.kp + j;
                out[0] = acc0 * sc;
                if (t0 + 1 < nlc) out[a.kp] = acc1 * sc;
                if (t0 + 2 < nlc) out[2 * a.kp] = acc2 * sc;
                if (t0 + 3 < nlc) out[3 * a.kp] = acc3 * sc;
            }
        }
    }
}

// This block's F^T v (projectors it needs) from the chunk partials in chunk order, then
// G F^T v for the projectors its rows apply.  Block-uniform control flow.
template <class J>
__device__ void nl_reduce(const MrArgs& a, int cnt, J&& jcol) {
    const int b = blockIdx.x;
    const int n0 = a.nl_nb_ptr[b], nn = a.nl_nb_ptr[b + 1] - n0, napp = a.nl_nb_napply[b];
    if (nn == 0) return;
    // a group of g lanes (a power of two) per (projector, column): its lanes stride over the
    // contributing chunks, then a shuffle tree; every warp runs the same trip count
    const int pairs = nn * cnt;
    int g = 32;
    while (g > 1 && g * pairs > (int)blockDim.x) g >>= 1;
    const int sub = threadIdx.x & (g - 1), g0 = threadIdx.x / g, ng = (int)blockDim.x / g;
    for (int pidx = g0; pidx - g0 < pairs; pidx += ng) {
        const bool on = pidx < pairs;
        double s0 = 0.0, s1 = 0.0;
        int t = 0, j = 0;
        if (on) {
            t = pidx / cnt;
            j = jcol(pidx - t * cnt);
            const int l = a.nl_nb_l[n0 + t];
            const int u1 = a.nl_cl_ptr[l + 1];
            int u = a.nl_cl_ptr[l] + sub;
            for (; u + g < u1; u += 2 * g) {
                s0 += a.nl_part[(int64_t)a.nl_cl_slot[u] * a.kp + j];
                s1 += a.nl_part[(int64_t)a.nl_cl_slot[u + g] * a.kp + j];
            }
            if (u < u1) s0 += a.nl_part[(int64_t)a.nl_cl_slot[u] * a.kp + j];
        }
        s0 += s1;
        for (int o = g >> 1; o > 0; o >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        if (on && sub == 0) a.nl_zv[(int64_t)(n0 + t) * a.kp + j] = s0;
    }
    __syncthreads();
    const int32_t* lm = a.nl_lmap + (int64_t)b * a.nl_k;
    for (int pidx = threadIdx.x; pidx < napp * cnt; pidx += blockDim.x) {
        const int t = pidx / cnt, q = pidx - t * cnt;
        const int j = jcol(q);
        const int l = a.nl_nb_l[n0 + t];
        double s = 0.0;
        for (int e = a.nl_gptr[l]; e < a.nl_gptr[l + 1]; ++e)
            s = fma(a.nl_gval[e], a.nl_zv[(int64_t)(n0 + lm[a.nl_gcol[e]]) * a.kp + j], s);
        a.nl_zg[(int64_t)(n0 + t) * a.kp + j] = s;
    }
    __syncthreads();
}

// Shifted SpMM of one pass over this block's slot range: thread (r, c) takes the slots
// b0 + r, b0 + r + rb, ... and column j = jcol(c0 + c); f(row, j, y) receives
// y = ((Hs - e_j S) Xin)(row, j).
template <class T, class P, class J, class F>
__device__ __forceinline__ void spmm_pass(const MrArgs& a, const P* hs, const T* E, const T* Xin, int64_t ldxin,
                                          const Pass& p, J&& jcol, F&& f) {
    if (p.r >= p.rb) return;
    const int j = jcol(p.c0 + p.c);
    const T ej = E[j];
    const int64_t s1 = a.blk[blockIdx.x + 1];
    for (int64_t slot = a.blk[blockIdx.x] + p.r; slot < s1; slot += p.rb) {
        const int64_t sl = slot / a.C;
        const int t = (int)(slot - sl * a.C);
        const int64_t base = a.slice_ptr[sl] + t;
        const int len = a.slice_len[sl];
        T ah = T(0), as = T(0);
#pragma unroll 4
        for (int jj = 0; jj < len; ++jj) {
            const int64_t ee = base + (int64_t)jj * a.C;
            const int cj = __ldg(a.cols + ee);
            const P hv = __ldg(hs + ee);
            const T x = Xin[(int64_t)cj * ldxin + j];
            ah = fma(hv.x, x, ah);
            as = fma(hv.y, x, as);
        }
        const int row = a.slot_row[slot];
        if (row >= 0) {
            T y = ah - ej * as;
            if (a.nl_k) y += (T)nl_slot(a, slot, j);
            f((int64_t)row, j, y);
        }
    }
}

// The same product from the FP32 scaled pencil on v^ = D^-1 v (FP32 multiply-adds), scaled back by
// D^-1 per row in FP64: f(row, j, y) receives ((Hs - e_j S) v)(row, j) to FP32 accuracy.
template <class J, class F>
__device__ __forceinline__ void spmm_pass_f32(const MrArgs& a, const double* E, int64_t ld, const Pass& p, J&& jcol,
                                              F&& f) {
    if (p.r >= p.rb) return;
    const int j = jcol(p.c0 + p.c);
    const float ej = (float)E[j];
    const int64_t s1 = a.blk[blockIdx.x + 1];
    for (int64_t slot = a.blk[blockIdx.x] + p.r; slot < s1; slot += p.rb) {
        const int64_t sl = slot / a.C;
        const int t = (int)(slot - sl * a.C);
        const int64_t base = a.slice_ptr[sl] + t;
        const int len = a.slice_len[sl];
        float ah = 0.f, as = 0.f;
#pragma unroll 4
        for (int jj = 0; jj < len; ++jj) {
            const int64_t ee = base + (int64_t)jj * a.C;
            const int cj = __ldg(a.cols + ee);
            const float2 hv = __ldg(a.hs32 + ee);
            const float x = a.V32[(int64_t)cj * ld + j];
            ah = fmaf(hv.x, x, ah);
            as = fmaf(hv.y, x, as);
        }
        const int row = a.slot_row[slot];
        if (row >= 0) {
            double y = (double)fmaf(-ej, as, ah) * a.dinv[row];
            if (a.nl_k) y += nl_slot(a, slot, j);
            f((int64_t)row, j, y);
        }
    }
}

// Row-wise visit of one pass over this block's slot range: f(row, j).
template <class J, class F>
__device__ __forceinline__ void rows_pass(const MrArgs& a, const Pass& p, J&& jcol, F&& f) {
    if (p.r >= p.rb) return;
    const int j = jcol(p.c0 + p.c);
    const int64_t s1 = a.blk[blockIdx.x + 1];
    for (int64_t slot = a.blk[blockIdx.x] + p.r; slot < s1; slot += p.rb) {
        const int row = a.slot_row[slot];
        if (row >= 0) f((int64_t)row, j);
    }
}

template <class T>
__global__ void __launch_bounds__(MR_THREADS, 2) k_minres(MrArgs a) {
    using P = typename Pair<T>::P;
    extern __shared__ __align__(16) double smem[];
    __shared__ int ok_sm;
    const int k = a.k;
    ColState S = col_state(smem, k);
    const T* R = static_cast<const T*>(a.R);
    const T* E = static_cast<const T*>(a.e);
    T* X = static_cast<T*>(a.X);
    T* V = static_cast<T*>(a.V);
    T* Vp = static_cast<T*>(a.Vp);
    T* U = static_cast<T*>(a.U);
    T* Wp = static_cast<T*>(a.Wp);
    T* Wpp = static_cast<T*>(a.Wpp);
    const P* hs = static_cast<const P*>(a.hs);
    const int64_t ld = a.ld;
    double* partA = a.part;
    double* partB = a.part + (int64_t)gridDim.x * a.kp;
    double* rowA = partA + (int64_t)blockIdx.x * a.kp;
    double* rowB = partB + (int64_t)blockIdx.x * a.kp;
    unsigned gen = 0;
    // tracing: block 0 adds the time since its previous mark to stamps[slot]
    unsigned long long tmark = 0;
    const bool tr = a.stamps != nullptr && blockIdx.x == 0 && threadIdx.x == 0;
    if (tr) tmark = gtimer();
    auto mark = [&](int slot) {
        if (tr) {
            const unsigned long long t = gtimer();
            a.stamps[slot] += t - tmark;
            tmark = t;
        }
    };
    auto identity = [](int pos) { return pos; };
    auto active_col = [&](int pos) { return S.g(I_ACT)[pos]; };

    // ---- nonlocal: F^T X for the start product ----
    if (a.nl_k) {
        nl_chunk_partial(a, reinterpret_cast<const double*>(X), a.ldx, k, identity, [](int) { return true; },
                         [](int) { return 1.0; });
        if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
        nl_reduce(a, k, identity);
    }
    // ---- start: U = A_e X, V = r0 = -R - U, ||r0||^2 and ||R||^2 per column ----
    for (int c0 = 0; c0 < k; c0 += MR_PASS) {
        const Pass p = make_pass(c0, k);
        double acc1 = 0.0, acc2 = 0.0;
        spmm_pass<T>(a, hs, E, X, a.ldx, p, identity, [&](int64_t row, int j, T u) {
            const T r = R[row * a.ldr + j];
            const T v = -r - u;
            V[row * ld + j] = v;
            acc1 += (double)v * (double)v;
            acc2 += (double)r * (double)r;
        });
        block_partials(acc1, p, S.red, rowA);
        block_partials(acc2, p, S.red, rowB);
    }
    mark(0);
    if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
    mark(4);
    grid_sum(partA, a.kp, k, S.f(F_RED1));
    grid_sum(partB, a.kp, k, S.f(F_RED2));
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double beta = sqrt(S.f(F_RED1)[j]);
        S.f(F_TOL)[j] = a.eta * sqrt(S.f(F_RED2)[j]);
        S.f(F_BETA_OLD)[j] = 0.0;
        S.f(F_C_PREV)[j] = 1.0; S.f(F_S_PREV)[j] = 0.0; S.f(F_C_PP)[j] = 1.0; S.f(F_S_PP)[j] = 0.0;
        S.f(F_PHIBAR)[j] = beta;
        S.f(F_BETA_NEXT)[j] = beta;
        S.f(F_BINV)[j] = beta > 0.0 ? 1.0 / beta : 0.0;
        S.g(I_STEPS)[j] = 0;
        S.g(I_ACTIVE)[j] = (beta > S.f(F_TOL)[j] && a.maxit > 0) ? 1 : 0;
        S.g(I_UPD)[j] = 0;
        S.g(I_CONT)[j] = S.g(I_ACTIVE)[j];
    }
    __syncthreads();
    // v_1 = r0 / beta_1 for the active columns, written to U (V keeps r0, which the nonlocal
    // partials read from every block); v_0 = w_0 = w_{-1} = 0.  V and U swap roles below.
    for (int c0 = 0; c0 < k; c0 += MR_PASS) {
        const Pass p = make_pass(c0, k);
        rows_pass(a, p, identity, [&](int64_t i, int j) {
            const int64_t o = i * ld + j;
            U[o] = S.g(I_ACTIVE)[j] ? (T)((double)V[o] * S.f(F_BINV)[j]) : V[o];
            if (a.f32) a.V32[o] = (float)((double)U[o] * a.dinv[i]);
            Vp[o] = T(0);
            Wp[o] = T(0);
            Wpp[o] = T(0);
        });
    }
    if (a.nl_k)
        nl_chunk_partial(a, reinterpret_cast<const double*>(V), ld, k, identity,
                         [&](int j) { return S.g(I_ACTIVE)[j] != 0; }, [&](int j) { return S.f(F_BINV)[j]; });
    if (threadIdx.x == 0) {
        int na = 0;
        for (int j = 0; j < k; ++j)
            if (S.g(I_ACTIVE)[j]) S.g(I_ACT)[na++] = j;
        S.nact()[0] = na;
    }
    mark(0);
    if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
    mark(4);
    {
        T* t = V;
        V = U;
        U = t;
    }

    for (int step = 1; step <= a.maxit && S.nact()[0] > 0; ++step) {
        const int na = S.nact()[0];
        // ---- A: U = A_e V on the active columns, partial alpha ----
        if (a.nl_k) {
            nl_reduce(a, na, active_col);
            mark(6);
        }
        const unsigned long long ta = (a.stamps && threadIdx.x == 0) ? gtimer() : 0ull;
        for (int c0 = 0; c0 < na; c0 += MR_PASS) {
            const Pass p = make_pass(c0, na);
            double acc = 0.0;
            auto take = [&](int64_t row, int j, T u) {
                U[row * ld + j] = u;
                acc += (double)V[row * ld + j] * (double)u;
            };
            if (a.f32) spmm_pass_f32(a, reinterpret_cast<const double*>(E), ld, p, active_col, take);
            else spmm_pass<T>(a, hs, E, V, ld, p, active_col, take);
            block_partials(acc, p, S.red, rowA);
        }
        if (a.stamps && threadIdx.x == 0) a.stamps[8 + blockIdx.x] += gtimer() - ta;   // per-block phase A (tracing)
        mark(1);
        if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
        mark(4);
        grid_sum(partA, a.kp, na, S.f(F_RED1));
        for (int q = threadIdx.x; q < na; q += blockDim.x) S.f(F_ALPHA)[S.g(I_ACT)[q]] = S.f(F_RED1)[q];
        __syncthreads();
        // ---- B: Lanczos three-term update, partial ||u||^2 ----
        for (int c0 = 0; c0 < na; c0 += MR_PASS) {
            const Pass p = make_pass(c0, na);
            double acc = 0.0;
            rows_pass(a, p, active_col, [&](int64_t i, int j) {
                const int64_t o = i * ld + j;
                const T u = U[o] - (T)S.f(F_ALPHA)[j] * V[o] - (T)S.f(F_BETA_OLD)[j] * Vp[o];
                U[o] = u;
                acc += (double)u * (double)u;
            });
            block_partials(acc, p, S.red, rowB);
        }
        mark(2);
        if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
        mark(4);
        grid_sum(partB, a.kp, na, S.f(F_RED2));
        // ---- C: Givens update (replicated per block), then the vector updates ----
        for (int q = threadIdx.x; q < na; q += blockDim.x) {
            const int j = S.g(I_ACT)[q];
            S.g(I_UPD)[j] = 0;
            S.g(I_CONT)[j] = 0;
            const double beta_next = sqrt(S.f(F_RED2)[q]);
            const double eps = S.f(F_S_PP)[j] * S.f(F_BETA_OLD)[j];
            const double dbar = S.f(F_C_PP)[j] * S.f(F_BETA_OLD)[j];
            const double delta = S.f(F_C_PREV)[j] * dbar + S.f(F_S_PREV)[j] * S.f(F_ALPHA)[j];
            const double gbar = -S.f(F_S_PREV)[j] * dbar + S.f(F_C_PREV)[j] * S.f(F_ALPHA)[j];
            const double gamma = hypot(gbar, beta_next);
            if (gamma == 0.0) {
                S.g(I_ACTIVE)[j] = 0;
            } else {
                const double ck = gbar / gamma, sk = beta_next / gamma;
                S.f(F_PHI)[j] = ck * S.f(F_PHIBAR)[j];
                S.f(F_PHIBAR)[j] = -sk * S.f(F_PHIBAR)[j];
                S.f(F_GINV)[j] = 1.0 / gamma;
                S.f(F_DELTA)[j] = delta;
                S.f(F_EPS)[j] = eps;
                S.g(I_STEPS)[j] = step;
                S.g(I_UPD)[j] = 1;
                const bool done = fabs(S.f(F_PHIBAR)[j]) <= S.f(F_TOL)[j] || beta_next == 0.0;
                S.g(I_CONT)[j] = done ? 0 : 1;
                S.f(F_BETA_NEXT)[j] = beta_next;
                S.f(F_BINV)[j] = beta_next > 0.0 ? 1.0 / beta_next : 0.0;
                S.f(F_BETA_OLD)[j] = beta_next;
                S.f(F_C_PP)[j] = S.f(F_C_PREV)[j]; S.f(F_S_PP)[j] = S.f(F_S_PREV)[j];
                S.f(F_C_PREV)[j] = ck; S.f(F_S_PREV)[j] = sk;
                if (done) S.g(I_ACTIVE)[j] = 0;
            }
        }
        __syncthreads();
        // F^T v_{j+1} = F^T u_j / beta_{j+1} for the columns that go on (U is final here)
        if (a.nl_k && step < a.maxit) {
            mark(3);
            nl_chunk_partial(a, reinterpret_cast<const double*>(U), ld, na, active_col,
                             [&](int j) { return S.g(I_CONT)[j] != 0; }, [&](int j) { return S.f(F_BINV)[j]; });
            mark(5);
        }
        for (int c0 = 0; c0 < na; c0 += MR_PASS) {
            const Pass p = make_pass(c0, na);
            rows_pass(a, p, active_col, [&](int64_t i, int j) {
                if (!S.g(I_UPD)[j]) return;
                const int64_t o = i * ld + j;
                const double v = (double)V[o];
                const double w = (v - S.f(F_DELTA)[j] * (double)Wp[o] - S.f(F_EPS)[j] * (double)Wpp[o]) * S.f(F_GINV)[j];
                T* xp = X + i * a.ldx + j;
                *xp = (T)((double)*xp + S.f(F_PHI)[j] * w);
                Wpp[o] = Wp[o];
                Wp[o] = (T)w;
                if (S.g(I_CONT)[j]) {
                    Vp[o] = V[o];
                    V[o] = (T)((double)U[o] * S.f(F_BINV)[j]);
                    if (a.f32) a.V32[o] = (float)((double)V[o] * a.dinv[i]);
                }
            });
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int nn = 0;
            for (int q = 0; q < na; ++q)
                if (S.g(I_ACTIVE)[S.g(I_ACT)[q]]) S.g(I_ACT)[nn++] = S.g(I_ACT)[q];
            S.nact()[0] = nn;
        }
        __syncthreads();
        mark(3);
        if (S.nact()[0] > 0 && step < a.maxit) {
            if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
            mark(4);
        }
    }
    if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < k; j += blockDim.x) a.steps_out[j] = S.g(I_STEPS)[j];
}

// First-order one-step refinement (Sec. 6, future work; reading R18): for each column j,
// d = (H - e_j S) p + r_j, p <- p - alpha d with alpha = (A d . d) / (A d . A d), the step that
// minimises ||d - alpha A d||; ||d|| is recomputed after each step and the column stops when it
// is <= eta ||r_j|| (Eq. approxp) or after maxit steps.  Same launch, layout and barrier as
// k_minres; each step is three phases:
//   A. U = A d on the active columns, partials of A d . d and A d . A d;
//   B. alpha, p -= alpha d, d -= alpha U, partials of ||d||^2;
//   C. the stopping test, the nonlocal partials of F^T d for the next step, compaction.
template <class T>
__global__ void __launch_bounds__(MR_THREADS, 2) k_onestep(MrArgs a) {
    using P = typename Pair<T>::P;
    extern __shared__ __align__(16) double smem[];
    __shared__ int ok_sm;
    const int k = a.k;
    ColState S = col_state(smem, k);
    const T* R = static_cast<const T*>(a.R);
    const T* E = static_cast<const T*>(a.e);
    T* X = static_cast<T*>(a.X);
    T* V = static_cast<T*>(a.V);   // d
    T* U = static_cast<T*>(a.U);   // A d
    const P* hs = static_cast<const P*>(a.hs);
    const int64_t ld = a.ld;
    double* partA = a.part;
    double* partB = a.part + (int64_t)gridDim.x * a.kp;
    double* rowA = partA + (int64_t)blockIdx.x * a.kp;
    double* rowB = partB + (int64_t)blockIdx.x * a.kp;
    unsigned gen = 0;
    unsigned long long tmark = 0;
    const bool tr = a.stamps != nullptr && blockIdx.x == 0 && threadIdx.x == 0;
    if (tr) tmark = gtimer();
    auto mark = [&](int slot) {
        if (tr) {
            const unsigned long long t = gtimer();
            a.stamps[slot] += t - tmark;
            tmark = t;
        }
    };
    auto identity = [](int pos) { return pos; };
    auto active_col = [&](int pos) { return S.g(I_ACT)[pos]; };

    if (a.nl_k) {
        nl_chunk_partial(a, reinterpret_cast<const double*>(X), a.ldx, k, identity, [](int) { return true; },
                         [](int) { return 1.0; });
        if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
        nl_reduce(a, k, identity);
    }
    // ---- start: d = A_e p + r into V, ||d||^2 and ||r||^2 per column ----
    for (int c0 = 0; c0 < k; c0 += MR_PASS) {
        const Pass p = make_pass(c0, k);
        double acc1 = 0.0, acc2 = 0.0;
        spmm_pass<T>(a, hs, E, X, a.ldx, p, identity, [&](int64_t row, int j, T u) {
            const T r = R[row * a.ldr + j];
            const T d = u + r;
            V[row * ld + j] = d;
            acc1 += (double)d * (double)d;
            acc2 += (double)r * (double)r;
        });
        block_partials(acc1, p, S.red, rowA);
        block_partials(acc2, p, S.red, rowB);
    }
    mark(0);
    if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
    mark(4);
    grid_sum(partA, a.kp, k, S.f(F_RED1));
    grid_sum(partB, a.kp, k, S.f(F_RED2));
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double dn = sqrt(S.f(F_RED1)[j]);
        S.f(F_TOL)[j] = a.eta * sqrt(S.f(F_RED2)[j]);
        S.f(F_PHIBAR)[j] = dn;
        S.g(I_STEPS)[j] = 0;
        S.g(I_ACTIVE)[j] = (dn > S.f(F_TOL)[j] && a.maxit > 0) ? 1 : 0;
    }
    __syncthreads();
    if (a.nl_k)
        nl_chunk_partial(a, reinterpret_cast<const double*>(V), ld, k, identity,
                         [&](int j) { return S.g(I_ACTIVE)[j] != 0; }, [](int) { return 1.0; });
    if (threadIdx.x == 0) {
        int na = 0;
        for (int j = 0; j < k; ++j)
            if (S.g(I_ACTIVE)[j]) S.g(I_ACT)[na++] = j;
        S.nact()[0] = na;
    }
    mark(0);
    if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
    mark(4);

    for (int step = 1; step <= a.maxit && S.nact()[0] > 0; ++step) {
        const int na = S.nact()[0];
        // ---- A: U = A d, partials of A d . d and A d . A d ----
        if (a.nl_k) {
            nl_reduce(a, na, active_col);
            mark(6);
        }
        for (int c0 = 0; c0 < na; c0 += MR_PASS) {
            const Pass p = make_pass(c0, na);
            double acc1 = 0.0, acc2 = 0.0;
            spmm_pass<T>(a, hs, E, V, ld, p, active_col, [&](int64_t row, int j, T u) {
                U[row * ld + j] = u;
                acc1 += (double)u * (double)V[row * ld + j];
                acc2 += (double)u * (double)u;
            });
            block_partials(acc1, p, S.red, rowA);
            block_partials(acc2, p, S.red, rowB);
        }
        mark(1);
        if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
        mark(4);
        // ---- B: alpha, p -= alpha d, d -= alpha A d, partial ||d||^2 ----
        grid_sum(partA, a.kp, na, S.f(F_RED1));
        grid_sum(partB, a.kp, na, S.f(F_RED2));
        for (int q = threadIdx.x; q < na; q += blockDim.x) {
            const int j = S.g(I_ACT)[q];
            const double uu = S.f(F_RED2)[q];
            S.g(I_UPD)[j] = uu > 0.0 ? 1 : 0;
            S.f(F_ALPHA)[j] = uu > 0.0 ? S.f(F_RED1)[q] / uu : 0.0;
        }
        __syncthreads();
        for (int c0 = 0; c0 < na; c0 += MR_PASS) {
            const Pass p = make_pass(c0, na);
            double acc = 0.0;
            rows_pass(a, p, active_col, [&](int64_t i, int j) {
                if (!S.g(I_UPD)[j]) return;
                const int64_t o = i * ld + j;
                const double al = S.f(F_ALPHA)[j];
                const double d = (double)V[o];
                T* xp = X + i * a.ldx + j;
                *xp = (T)((double)*xp - al * d);
                const double dn = d - al * (double)U[o];
                V[o] = (T)dn;
                acc += dn * dn;
            });
            block_partials(acc, p, S.red, rowA);
        }
        mark(2);
        if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
        mark(4);
        // ---- C: stopping test, F^T d for the next step, compaction ----
        grid_sum(partA, a.kp, na, S.f(F_RED1));
        for (int q = threadIdx.x; q < na; q += blockDim.x) {
            const int j = S.g(I_ACT)[q];
            int cont = 0;
            if (S.g(I_UPD)[j]) {
                const double dn = sqrt(S.f(F_RED1)[q]);
                S.f(F_PHIBAR)[j] = dn;
                S.g(I_STEPS)[j] = step;
                cont = dn > S.f(F_TOL)[j] && step < a.maxit;
            }
            S.g(I_CONT)[j] = cont;
            if (!cont) S.g(I_ACTIVE)[j] = 0;
        }
        __syncthreads();
        if (a.nl_k && step < a.maxit) {
            mark(3);
            nl_chunk_partial(a, reinterpret_cast<const double*>(V), ld, na, active_col,
                             [&](int j) { return S.g(I_CONT)[j] != 0; }, [](int) { return 1.0; });
            mark(5);
        }
        if (threadIdx.x == 0) {
            int nn = 0;
            for (int q = 0; q < na; ++q)
                if (S.g(I_ACTIVE)[S.g(I_ACT)[q]]) S.g(I_ACT)[nn++] = S.g(I_ACT)[q];
            S.nact()[0] = nn;
        }
        __syncthreads();
        mark(3);
        if (S.nact()[0] > 0 && step < a.maxit) {
            if (!grid_barrier(a.bar, gridDim.x, gen, a.err, &ok_sm)) return;
            mark(4);
        }
    }
    if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < k; j += blockDim.x) a.steps_out[j] = S.g(I_STEPS)[j];
}

}  // namespace

// Runs k_barrier_probe on two blocks with a wait limit of limit_s seconds: HBSD_ERR_TIMEOUT when
// both blocks gave up and returned (the expected outcome), HBSD_ERR_CUDA otherwise.
int barrier_timeout_probe(double limit_s, cudaStream_t st) {
    DBuf<int> w;
    HBSD_TRY(w.alloc(4));
    HBSD_CUDA(cudaMemsetAsync(w.p, 0, 4 * sizeof(int), st));
    const uint64_t ns = (uint64_t)(std::max(0.001, std::min(limit_s, 5.0)) * 1e9);
    k_barrier_probe<<<2, 64, 0, st>>>(reinterpret_cast<unsigned*>(w.p), w.p + 2, ns);
    HBSD_CUDA(cudaPeekAtLastError());
    int h[4] = {0, 0, 0, 0};
    HBSD_CUDA(cudaMemcpyAsync(h, w.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (h[2] == 1 && h[3] == 2) return fail(HBSD_ERR_TIMEOUT, "barrier probe: the wait ran out as expected");
    return fail(HBSD_ERR_CUDA, "barrier probe: unexpected outcome");
}

template <class T> static DBuf<T>& mr_vecs(Session* s);
template <> DBuf<double>& mr_vecs<double>(Session* s) { return s->mr_d; }

// X (n x k, ldx): start vectors on entry, refined vectors on exit.  R: residual columns.
// e: shifts eps_j relative to sigma0 (device, k entries of T).  steps: device ints (nullable).
template <class T>
int minres_batch(Session* s, const T* R, int64_t ldr, const T* e, int k, double eta, int maxit, T* X,
                 int64_t ldx, int* steps, int64_t* total_steps, cudaStream_t st, int solver) {
    if (solver != HBSD_LOCAL_MINRES && solver != HBSD_LOCAL_ONESTEP) return fail(HBSD_ERR_ARG, "unknown local solver");
    const void* kern = solver == HBSD_LOCAL_ONESTEP ? (const void*)k_onestep<T> : (const void*)k_minres<T>;
    if (k <= 0) return 0;
    const size_t smem = mr_smem_bytes(k);
    if (smem > MR_SMEM_MAX) return fail(HBSD_ERR_ARG, "minres: too many columns for one launch");
    const int64_t n = s->n;
    const int64_t ld = round_up(k, 4);
    HBSD_TRY(mr_vecs<T>(s).alloc((size_t)5 * n * ld));
    HBSD_TRY(s->mr_steps.alloc(k));
    HBSD_TRY(s->mr_any.alloc(4));   // [0..1] grid barrier, [2] error flag
    static int blocks_per_sm[2] = {-1, -1};
    static int num_sms = 0;
    static std::mutex init_mu;
    const int ti = sizeof(T) == 8 ? 0 : 1;
    std::unique_lock<std::mutex> init_lk(init_mu);
    if (blocks_per_sm[ti] < 0) {
        int dev = 0;
        HBSD_CUDA(cudaGetDevice(&dev));
        HBSD_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
        // one grid size for both kernels (the slot partition and the nonlocal index follow it)
        HBSD_CUDA(cudaFuncSetAttribute(k_minres<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MR_SMEM_MAX));
        HBSD_CUDA(cudaFuncSetAttribute(k_onestep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MR_SMEM_MAX));
        int nb = 0, nb2 = 0;
        HBSD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_minres<T>, MR_THREADS, MR_SMEM_MAX));
        HBSD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, k_onestep<T>, MR_THREADS, MR_SMEM_MAX));
        blocks_per_sm[ti] = std::min(nb, nb2);
    }
    if (blocks_per_sm[ti] < 1) return fail(HBSD_ERR_UNSUPPORTED, "minres: kernel cannot be resident");
    // the whole GPU, or fewer CTAs where the autotuner found them as fast (small problems: cheaper
    // grid barriers, and SMs left to the other sessions of a batch)
    const int full = blocks_per_sm[ti] * num_sms;
    const int grid = s->tune_mr_grid > 0 ? std::min(s->tune_mr_grid, full) : full;
    init_lk.unlock();
    const int64_t kp = round_up(k, 4);
    HBSD_TRY(s->mr_red.alloc((size_t)2 * grid * kp));
    const bool nl = s->nl.k > 0 && s->nl.nnz > 0;
    const int nl_ver = nl ? s->nl.version : -1;
    if (s->mr_blk_grid != grid || s->mr_blk_nl != nl_ver) {
        // contiguous slot ranges per block with about equal work: stored entries, +2 per row for
        // the per-row work outside the nonzero loop, +2 per entry of F in the row (nonlocal term)
        const Sell& A = s->A;
        std::vector<int64_t> wcum(A.n_slots + 1, 0);
        for (int64_t sl = 0; sl < A.n_slices; ++sl) {
            const int64_t len = (A.h_slice_ptr[sl + 1] - A.h_slice_ptr[sl]) / A.C;
            for (int t = 0; t < A.C; ++t) {
                const int64_t slot = sl * A.C + t;
                if (slot >= A.n_slots) continue;
                wcum[slot + 1] = len + 2;
                const int row = A.h_slot_row[slot];
                if (nl && row >= 0) wcum[slot + 1] += 2 * (s->nl.h_rptr[row + 1] - s->nl.h_rptr[row]);
            }
        }
        for (int64_t i = 0; i < A.n_slots; ++i) wcum[i + 1] += wcum[i];
        std::vector<int64_t> blk(grid + 1, A.n_slots);
        blk[0] = 0;
        int64_t slot = 0;
        for (int b = 1; b < grid; ++b) {
            const double target = (double)wcum[A.n_slots] * b / grid;
            while (slot < A.n_slots && (double)wcum[slot] < target) ++slot;
            blk[b] = slot;
        }
        HBSD_TRY(s->mr_blk.alloc(grid + 1));
        HBSD_CUDA(cudaMemcpy(s->mr_blk.p, blk.data(), (grid + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
        s->h_mr_blk = std::move(blk);
        s->mr_blk_grid = grid;
        s->mr_blk_nl = nl_ver;
        s->nl.mr_grid = -1;   // the nonlocal index follows the partition
    }
    if (nl) HBSD_TRY(nl_minres_index(s, grid, s->h_mr_blk, kp));
    HBSD_CUDA(cudaMemsetAsync(s->mr_any.p, 0, 4 * sizeof(int), st));
    T* V = mr_vecs<T>(s).p;
    MrArgs a;
    a.slice_ptr = s->A.slice_ptr.p;
    a.slice_len = s->A.slice_len.p;
    a.cols = s->A.cols.p;
    a.hs = sizeof(T) == 8 ? static_cast<const void*>(s->A.hs.p) : static_cast<const void*>(s->A.hs32.p);
    a.slot_row = s->A.slot_row.p;
    a.n_slots = s->A.n_slots;
    a.blk = s->mr_blk.p;
    a.C = s->A.C;
    a.n = n;
    a.k = k;
    a.R = R;
    a.ldr = ldr;
    a.e = e;
    a.X = X;
    a.ldx = ldx;
    a.V = V;
    a.Vp = V + n * ld;
    a.U = V + 2 * n * ld;
    a.Wp = V + 3 * n * ld;
    a.Wpp = V + 4 * n * ld;
    a.ld = ld;
    a.part = s->mr_red.p;
    a.kp = kp;
    a.eta = eta;
    a.maxit = maxit;
    int* sp = steps ? steps : s->mr_steps.p;
    a.steps_out = sp;
    a.bar = reinterpret_cast<unsigned*>(s->mr_any.p);
    a.err = s->mr_any.p + 2;
    static const bool trace = std::getenv("HBSD_TRACE") != nullptr;
    a.stamps = nullptr;
    if (trace) {
        HBSD_TRY(s->mr_stamps.alloc(8 + grid));
        HBSD_CUDA(cudaMemsetAsync(s->mr_stamps.p, 0, (8 + grid) * sizeof(unsigned long long), st));
        a.stamps = s->mr_stamps.p;
    }
    a.nl_k = nl ? s->nl.k : 0;
    a.f32 = 0;
    a.hs32 = nullptr;
    a.dinv = nullptr;
    a.V32 = nullptr;
    if (sizeof(T) == 8 && solver == HBSD_LOCAL_MINRES && s->opt.precision == HBSD_PRECISION_MIXED &&
        s->opt.minres_f32 && s->A.dinv.p) {
        HBSD_TRY(s->mr_v32.alloc((size_t)n * ld));
        a.f32 = 1;
        a.hs32 = s->A.hs32.p;
        a.dinv = s->A.dinv.p;
        a.V32 = s->mr_v32.p;
    }
    {
        Nonlocal& q = s->nl;
        a.nl_rptr = q.rptr.p; a.nl_rcol = q.rcol.p; a.nl_rval = q.rval.p; a.nl_frows = q.ch_rows.p;
        a.nl_ch_row_off = q.ch_row_off.p; a.nl_ch_lptr = q.ch_lptr.p; a.nl_pan = q.pan.p; a.nl_pan_off = q.pan_off.p;
        a.nl_cl_ptr = q.cl_ptr.p; a.nl_cl_slot = q.cl_slot.p;
        a.nl_nb_ptr = q.nb_ptr.p; a.nl_nb_napply = q.nb_napply.p; a.nl_nb_l = q.nb_l.p; a.nl_lmap = q.lmap.p;
        a.nl_gptr = q.gptr.p; a.nl_gcol = q.gcol.p; a.nl_gval = q.gval.p;
        a.nl_sf_ptr = q.sf_ptr.p; a.nl_sf_off = q.sf_off.p; a.nl_sf_val = q.sf_val.p;
        a.nl_part = q.mr_part.p; a.nl_zv = q.zv.p; a.nl_zg = q.zg.p;
    }
    void* args[] = {&a};
    HBSD_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(MR_THREADS), args, smem, st));
    HBSD_LAUNCHED(s);
    std::vector<int> h(k);
    int flags[4] = {0, 0, 0, 0};
    HBSD_CUDA(cudaMemcpyAsync(flags, s->mr_any.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaMemcpyAsync(h.data(), sp, k * sizeof(int), cudaMemcpyDeviceToHost, st));
    HBSD_CUDA(cudaStreamSynchronize(st));
    if (flags[2]) return fail(HBSD_ERR_TIMEOUT, "minres: a grid barrier wait timed out");
    int64_t tot = 0;
    int mx = 0;
    for (int v : h) { tot += v; mx = std::max(mx, v); }
    if (trace) {
        unsigned long long t[8];
        HBSD_CUDA(cudaMemcpy(t, s->mr_stamps.p, sizeof(t), cudaMemcpyDeviceToHost));
        std::fprintf(stderr, "[hbsd]   %s k %d grid %d steps max %d sum %lld | us: start %.0f A %.0f B %.0f C %.0f barriers %.0f nl-partial %.0f nl-reduce %.0f\n",
                     solver == HBSD_LOCAL_ONESTEP ? "ONESTEP" : "MINRES", k, grid, mx, (long long)tot, t[0] * 1e-3, t[1] * 1e-3, t[2] * 1e-3, t[3] * 1e-3, t[4] * 1e-3,
                     t[5] * 1e-3, t[6] * 1e-3);
        std::vector<unsigned long long> pb(grid);
        HBSD_CUDA(cudaMemcpy(pb.data(), s->mr_stamps.p + 8, grid * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        std::vector<unsigned long long> srt(pb);
        std::sort(srt.begin(), srt.end());
        double mean = 0.0;
        for (auto v : pb) mean += (double)v;
        mean /= grid;
        int imax = (int)(std::max_element(pb.begin(), pb.end()) - pb.begin());
        std::fprintf(stderr, "[hbsd]     phase A per block us: min %.0f p10 %.0f median %.0f p90 %.0f max %.0f (block %d) mean %.0f\n",
                     srt[0] * 1e-3, srt[grid / 10] * 1e-3, srt[grid / 2] * 1e-3, srt[grid * 9 / 10] * 1e-3, srt[grid - 1] * 1e-3,
                     imax, mean * 1e-3);
        if (std::getenv("HBSD_TRACE_BLOCKS")) {
            std::fprintf(stderr, "[hbsd]     phase A blocks:");
            for (int b = 0; b < grid; ++b) std::fprintf(stderr, " %.0f", pb[b] * 1e-3);
            std::fprintf(stderr, "\n");
        }
    }
    s->stats.minres_spmm_cols += tot + k;   // the start SpMM plus one column per step
    if (total_steps) *total_steps = tot;
    return 0;
}

template int minres_batch<double>(Session*, const double*, int64_t, const double*, int, double, int, double*,
                                  int64_t, int*, int64_t*, cudaStream_t, int);

}  // namespace hbsd
