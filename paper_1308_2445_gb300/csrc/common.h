// Internal declarations shared by the translation units of libhbsd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <new>
#include <string>
#include <vector>

#include "hbsd.h"

namespace hbsd {

// ---- errors -------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

// Runs the body of a C entry point so that no exception crosses the ABI: std::bad_alloc becomes
// HBSD_ERR_OOM (with a message short enough to need no allocation), any other exception
// HBSD_ERR_ARG.
template <class F>
int guarded(F&& body) noexcept {
    try {
        return body();
    } catch (const std::bad_alloc&) {
        return fail(HBSD_ERR_OOM, "no host memory");
    } catch (const std::exception& e) {
        try {
            return fail(HBSD_ERR_ARG, std::string("host exception: ") + e.what());
        } catch (...) {
            return HBSD_ERR_ARG;
        }
    } catch (...) {
        return fail(HBSD_ERR_ARG, "host exception");
    }
}

#define HBSD_CUDA(call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return ::hbsd::fail(HBSD_ERR_CUDA, std::string(#call) + ": " +               \
                                                   cudaGetErrorString(e_));              \
    } while (0)

#define HBSD_TRY(call)                                                                   \
    do {                                                                                 \
        int s_ = (call);                                                                 \
        if (s_ < 0) return s_;                                                           \
    } while (0)

#define HBSD_LAUNCHED(h)                                                                 \
    do {                                                                                 \
        cudaError_t e_ = cudaPeekAtLastError();                                          \
        if (e_ != cudaSuccess)                                                           \
            return ::hbsd::fail(HBSD_ERR_CUDA, std::string("launch: ") +                 \
                                                   cudaGetErrorString(e_));              \
        ::hbsd::count_launch(h);                                                         \
    } while (0)

struct Session;
void count_launch(Session* s);
// device bytes held by the DBufs this thread allocated minus those it released (a thread's
// difference across a call is what the call left allocated; the served form's footprints)
int64_t& tl_dev_bytes();
int64_t& tl_dev_peak();   // the largest value tl_dev_bytes() has reached on this thread

// ---- device memory owned by a session ---------------------------------------------------
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    int alloc(size_t count);
    void release();
    ~DBuf() { release(); }
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
};

template <class T>
int DBuf<T>::alloc(size_t count) {
    if (count <= n && p) return 0;
    release();
    if (count == 0) return 0;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
        p = nullptr;
        (void)cudaGetLastError();
        return fail(HBSD_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    n = count;
    tl_dev_bytes() += (int64_t)(count * sizeof(T));
    if (tl_dev_bytes() > tl_dev_peak()) tl_dev_peak() = tl_dev_bytes();
    return 0;
}

template <class T>
void DBuf<T>::release() {
    if (p) {
        cudaFree(p);
        tl_dev_bytes() -= (int64_t)(n * sizeof(T));
    }
    p = nullptr;
    n = 0;
}

// ---- SELL-C-sigma matrix with interleaved (h, s) values -----------------------------------
struct Sell {
    int C = 8;                  // slice height
    int sigma = 256;            // sorting window
    int64_t n = 0, nnz = 0;
    int64_t n_slices = 0, n_slots = 0, stored = 0;
    DBuf<int64_t> slice_ptr;    // first entry of each slice
    DBuf<int32_t> slice_len;    // padded row length of each slice
    DBuf<int32_t> cols;         // stored column indices, slice-major, then entry-major, then row
    DBuf<double2> hs;           // (h - sigma0 s, s) per stored entry
    DBuf<float2> hs32;          // FP32 values of the scaled pencil (D Hs D, D S D) for the mixed path
    DBuf<float4> hsdf;          // the scaled pencil in double-float: (hi, lo) of D Hs D, then of D S D
    DBuf<double> dscale;        // D = diag(S)^{-1/2}
    DBuf<double> dinv;          // D^-1
    std::vector<double> h_dscale;
    std::vector<int64_t> h_slice_ptr;
    std::vector<int32_t> h_slot_row, h_cols;
    DBuf<int32_t> slot_row;     // original row of each slot (-1 for padding slots)
    std::vector<int64_t> h_entry_of_csr;  // stored position of each CSR entry (host, for updates)
};

int sell_build(Sell& m, int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
               const double* hval, const double* sval, double sigma0);
int sell_update_h(Sell& m, const double* hval, const double* sval, double sigma0);
int sell_fill_fp32(Sell& m, const double2* hs, const int32_t* cols, const int32_t* slot_row);

// Y_h = Hs X, Y_s = S X for k columns; X, Y row-major.
template <class T>
int spmm_pair(Session* s, const Sell& m, const T* X, int64_t ldx, int k, T* HX, int64_t ldhx,
              T* SX, int64_t ldsx, cudaStream_t st);
// Y_h = Hs X, Y_s = S X in double-float arithmetic on the scaled pencil (mixed form): about 48 bits
// per product, the FP64 inputs and outputs scaled by D^-1 on the way in and out
int spmm_pair_df64(Session* s, const Sell& m, const double* X, int64_t ldx, int k, double* HX, int64_t ldhx,
                   double* SX, int64_t ldsx, cudaStream_t st);
// Y(:, j) = (Hs - e_j S) X(:, j)
template <class T>
int spmm_shifted(Session* s, const Sell& m, const T* X, int64_t ldx, int k, const T* e, T* Y,
                 int64_t ldy, cudaStream_t st);

// ---- supernodal Cholesky of H - sigma_bar S ----------------------------------------------
struct Supernode {
    int64_t first;       // first column (permuted order)
    int ns;              // columns
    int nu;              // rows below the diagonal block
    int parent;          // -1 for a root
    int level;           // height: leaves 0
    int child[2];        // up to two children (-1 none)
    int64_t struct_off;  // offset of the below-diagonal row list in Factor::h_struct
    int64_t L_off;       // offset of the (ns+nu) x ns column-major panel in Factor::L
    int64_t Dinv_off;    // offset of the inverted NB x NB diagonal blocks
    int64_t ea_off;      // offset of this node's child->parent map (nu entries) in Factor::ea
    int64_t fv_off;      // offset of this node's front vector (ns+nu rows) in the solve workspace
};

// per-level work lists of the factor (device copies used by the batched kernels)
struct LevelLists {
    std::vector<int> offs;                        // offset of each level's id list in ids
    std::vector<int> counts;
    std::vector<int> max_ns, max_nf, max_nu;
    std::vector<int> job_offs[2], job_counts[2];  // (parent, child) pairs per level per child slot
    std::vector<int64_t> entry_offs;              // matrix-entry scatter list per level
    DBuf<int> ids;
    DBuf<int> jobs;
    DBuf<int64_t> entry_pos, entry_src;
};

struct Factor {
    static constexpr int NB = 64;
    LevelLists LL;
    int64_t n = 0;
    std::vector<Supernode> sn;
    std::vector<int64_t> h_struct;               // below-diagonal rows of every supernode
    std::vector<std::vector<int>> levels;        // supernodes by height
    std::vector<int32_t> h_perm;                 // new -> old
    int64_t nnz_L = 0, fv_total = 0, dinv_total = 0, ea_total = 0;
    DBuf<int32_t> perm;                          // new -> old
    DBuf<int64_t> d_struct;
    DBuf<int32_t> ea;                            // child row -> parent front row
    DBuf<double> L;                              // panels
    DBuf<double> Dinv;                           // inverted diagonal blocks
    DBuf<int> d_sn;                              // packed per-supernode descriptors (see chol.cu)
    int max_front = 0;
    int max_ns = 0;
    // explicit panels G = [L11^{-1}; -L21 L11^{-1}] used by the solves (layout of L)
    DBuf<double> G;
    DBuf<float> G32;
    DBuf<float> G32T;                            // the FP32 panels row-major (backward sweep)
    DBuf<int2> src;                              // extend-add sources of each front row (child 0, child 1)
    struct Sweep { int item_off, n_items, red_off, n_red; };
    std::vector<Sweep> sweep;                    // [2*level + (0 forward, 1 backward)]
    DBuf<int64_t> items, red_items;              // packed work items (see chol.cu)
    int64_t part_rows = 0;                       // split partial rows needed by the largest level
    // solve workspace: front vectors | y | x | partials
    DBuf<double> sws;
    DBuf<float> sws32;
    // signed LDL^T form (eps_bar inside the spectrum): pivot signs in permuted order
    bool signed_form = false;
    int64_t neg_pivots = 0;
    DBuf<double> sgn;
};

int factor_build(Session* s, Factor& f, int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* aval, const int32_t* dof_node, const int32_t* grid, cudaStream_t st);
template <class T>
int factor_solve(Session* s, Factor& f, const T* R, int64_t ldr, int k, T* P, int64_t ldp,
                 cudaStream_t st);
int factor_make_fp32(Factor& f, const double* dscale, cudaStream_t st);

// ---- dense helpers -------------------------------------------------------------------
// column sums over rows of a row-major block: out[j] = sum_i A(i, j) * B(i, j)  (B may be A)
template <class T>
int col_dots(Session* s, const T* A, int64_t lda, const T* B, int64_t ldb, int64_t n, int k,
             double* out, cudaStream_t st);
template <class T>
int gram2(Session* s, const T* Z0, int64_t ld0, int q0, const T* Z1, int64_t ld1, int q1, const T* H0,
          int64_t ldh0, const T* H1, int64_t ldh1, const T* S0, int64_t lds0, const T* S1, int64_t lds1,
          int64_t n, double* HR, double* SR, cudaStream_t st);
// A1 = antisymmetric part of Z^T V1, A2 = symmetric part of Z^T V2 (q x q, row-major)
int gram_skew(Session* s, const double* Z, int64_t ldz, const double* V1, int64_t ldv1, const double* V2,
              int64_t ldv2, int64_t n, int q, double* A1, double* A2, cudaStream_t st);
// largest q the allocation-free Gram's static scratch holds (2 q^2 doubles per row chunk, 2^21 in all)
constexpr int GRAM_NOALLOC_MAX_Q = 1024;
int gram_noalloc(const double* Z, int64_t ldz, const double* ZH, int64_t ldzh, const double* ZS, int64_t ldzs,
                 int64_t n, int q, double* HR, double* SR, cudaStream_t st);
template <class T>
int update2(Session* s, T* Z0, int64_t ld0, int q0, const T* Z1, int64_t ld1, int q1, int64_t n,
            const double* W, int k, cudaStream_t st);
int rayleigh_ritz(Session* s, const double* HR, const double* SR, int q, int k, double* theta,
                  double* W, int* info_host, cudaStream_t st);
// double-float (hi + lo float pairs) forms of the Gram and update products, for the mixed form
int gram2_df64(Session* s, const double* Z0, int64_t ld0, int q0, const double* Z1, int64_t ld1, int q1,
               const double* H0, int64_t ldh0, const double* H1, int64_t ldh1, const double* S0, int64_t lds0,
               const double* S1, int64_t lds1, int64_t n, double* HR, double* SR, cudaStream_t st);
int update2_df64(Session* s, double* Z0, int64_t ld0, int q0, const double* Z1, int64_t ld1, int q1, int64_t n,
                 const double* W, int k, cudaStream_t st, bool split_w);
// Y = [Z0 Z1] W on the tensor cores by exact bf16 slices (oz.cu); Y must not alias Z0 or Z1
// status: device int that a timed-out MMA wait sets to 1 (the call is then asynchronous), or NULL
// (the call checks its own flag and synchronises)
int update_oz(Session* s, const double* Z0, int64_t ld0, int q0, const double* Z1, int64_t ld1, int q1, int64_t n,
              const double* W, int k, double* Y, int64_t ldy, cudaStream_t st, int* status = nullptr);
constexpr int OZ_MAX_Q_SEG = 640;   // largest block width update_oz takes
int rayleigh_ritz_cluster(Session* s, const double* HR, const double* SR, int q, int k, double* theta,
                          double* W, int* info_host, cudaStream_t st, double drop_tol = 0.0);
template <class T>
int residual(Session* s, const T* PH, int64_t ldh, const T* PS, int64_t lds, const double* E, int m,
             T* R, int64_t ldr, int64_t n, double* res, double* rnorm, cudaStream_t st);
// step 6(b) for k columns: MINRES (solver = HBSD_LOCAL_MINRES) or the first-order one-step
// refinement (HBSD_LOCAL_ONESTEP)
template <class T>
int minres_batch(Session* s, const T* R, int64_t ldr, const T* e, int k, double eta, int maxit, T* X,
                 int64_t ldx, int* steps, int64_t* total_steps, cudaStream_t st, int solver = HBSD_LOCAL_MINRES);

// ---- nonlocal low-rank term H_nl = F G F^T (Eq. fgf) and its SMW data (Sec. 4) -----------
// F is kept by its nonzero entries (projectors of compact support make it sparse) in two
// orders: by projector (F^T X products) and by row (F Z products).  SMW steps 1-4 are held as
// Fh = -(H_loc - eps_bar S)^{-1} F (dense) and M = T^{-1} G, so that step 6 reads
// P -= Fhat (M (F^T P)); this equals the stored F := F G T^{-H} of step 4 and keeps F sparse.
struct Nonlocal {
    int k = 0;                      // projectors (0: no nonlocal term)
    int version = 0;                // bumped by every nl_set (invalidates derived data)
    int64_t nnz = 0, nfr = 0;       // stored entries of F; rows with entries
    int n_items = 0;                // F^T X work items
    std::vector<int64_t> h_rptr;    // host copies used to build the fused-MINRES index
    std::vector<int32_t> h_rcol, h_frows, h_gptr, h_gcol;
    std::vector<double> h_rval, h_gval;
    DBuf<int64_t> cptr, item_e;     // F by projector; entry range of each work item
    DBuf<int32_t> crow, item_ptr;   // row of each entry; first work item of each projector
    DBuf<double> cval;
    DBuf<float> cval32;             // D F (scaled pencil of the FP32 paths)
    DBuf<int64_t> rptr;             // F by row, over all n rows
    DBuf<int32_t> rcol, frows;      // projector of each entry; rows with entries
    DBuf<double> rval;
    DBuf<float> rval32;
    bool scaled32 = false;
    DBuf<int32_t> gptr, gcol;       // G by rows
    DBuf<double> gval;
    int64_t ldf = 0;                // SMW: Fh (n x k, ld ldf); M = T^{-1} G dense (CSR form)
    bool smw64 = false, smw32 = false;
    DBuf<double> Fh, M64, M32;
    DBuf<float> Fh32;
    DBuf<int32_t> mptr, mcol;
    DBuf<double> part, z, tmat;     // work
    DBuf<float> part32, z32;
    DBuf<int> info;
    // fused-MINRES index for one grid size (see minres.cu)
    int mr_grid = -1, mr_version = -1, mr_nslots = 0, mr_nneed = 0;
    DBuf<int64_t> ch_row_off, pan_off;
    DBuf<int32_t> ch_rows, ch_lptr, cl_ptr, cl_slot, nb_ptr, nb_napply, nb_l, lmap, sf_ptr, sf_off;
    DBuf<double> pan, mr_part, zv, zg, sf_val;
};

// ---- session -----------------------------------------------------------------------
// Block buffers of one solve (steps 1-11), kept in the session between solves.
template <class T>
struct SolveBufs {
    DBuf<T> Psi, PsiH, PsiS, P, PH, PS, RU, Xa, Ra, shifts;
    DBuf<T> upd;                // out-of-place target of the tensor-core update, swapped in
};

struct SolveCommon {
    DBuf<double> E, res, HR, SR, W, theta;
    DBuf<int> Ulist, Llist, steps;
};

struct Session {
    int64_t n = 0, nnz = 0;
    hbsd_options opt{};
    double sigma0 = 0.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Sell A;                     // (Hs, S) pattern
    Factor F;
    bool has_factor = false;
    hbsd_stats stats{};
    int launches = 0;
    // CSR kept on host for hbsd_update_H
    std::vector<double> h_sval;
    // workspaces (FP64 driver)
    DBuf<double> ws;            // generic scratch for reductions
    DBuf<double> rr_ws;         // Rayleigh-Ritz workspace
    DBuf<int> rr_info;
    // MINRES workspace (minres.cu)
    DBuf<double> mr_d;
    DBuf<double> mr_red;        // per-block partial sums of the fused MINRES kernel
    DBuf<float> mr_v32;         // D^-1 v in FP32 for the FP32 operator products of MINRES
    DBuf<float2> x2;            // D^-1 X in double-float for spmm_pair_df64
    DBuf<int> mr_any, mr_steps; // grid barrier + error flag; per-column step counts
    DBuf<unsigned long long> mr_stamps;   // MINRES phase times when tracing
    DBuf<int64_t> mr_blk;       // per-block SELL slot ranges of the fused MINRES kernel
    DBuf<float2> df_w;          // double-float copy of the Rayleigh-Ritz coefficients W
    DBuf<double> oz_ws;         // split-slice update: exponents and bf16 slices of W (oz.cu)
    DBuf<int> oz_status;        // set by a timed-out MMA wait of the solve's tensor-core updates
    SolveBufs<double> sb;       // per-solve blocks, resident (grow only)
    SolveCommon sc;
    DBuf<double> io_x0, io_lam, io_x;   // host API staging of X0, lambda, X
    bool opt_df64 = true;       // mixed form: Gram and update in double-float (HBSD_NO_DF64=1 turns off)
    double dbg_rr_kernel_ms = 0.0, dbg_rr_host_ms = 0.0, dbg_rr_wake_ms = 0.0;   // Rayleigh-Ritz timing accounting (HBSD_RRDBG)
    int mr_blk_grid = 0;
    int mr_blk_nl = -1;              // nonlocal version the partition was weighted for (-1: none)
    std::vector<int64_t> h_mr_blk;   // host copy of mr_blk
    // mixed-precision preconditioner buffers (FP32 scaled R and P)
    DBuf<float> r32, p32, xa32, ra32, sh32;
    // warm-start state
    DBuf<double> psi_keep;
    int keep_w = 0;
    int64_t keep_ld = 0;
    Nonlocal nl;                // H_nl = F G F^T (k = 0: none)
    // complex Hermitian input: the session holds the real-equivalent pencil of size n = 2 n_c
    // with the dofs interleaved (row 2i: real part of complex dof i, row 2i+1: imaginary part)
    bool cplx = false;
    int64_t n_c = 0;
    std::vector<int64_t> c_row_ptr;  // complex pattern, kept to realify new H values
    std::vector<int32_t> c_col_idx;
    DBuf<double> cx_gr, cx_gc, cx_w, cx_x0, cx_y0;   // recovery: Gram parts, coefficients; start blocks
    DBuf<double2> cx_a, cx_l, cx_m;  // recovery: Gram (eliminated in place), Cholesky columns, inverse
    DBuf<int> cx_piv;
    std::vector<double> res_hist;   // Res_max at each convergence test of the last solve
    // launch shapes picked by the autotuner (batch.cu); 0 = the built-in choice
    int tune_spmm_lpr = 0;          // most lanes per row of the fused SpMM (4, 8, 16 or 32)
    int tune_mr_grid = 0;           // CTAs of the cooperative MINRES launch
    int tuned_width = 0;            // block width the session was tuned for (0: not tuned)
};

// nev + m0 real columns of the block a solve of nev pairs runs on (twice that on a complex session)
int block_width(const Session& s, int nev);
// time the candidate launch shapes on this session and keep the fastest (batch.cu)
int autotune(Session* s, int width, hbsd_tune* out);

// nonlocal term (nonlocal.cu)
int nl_set(Session* s, int k, const double* F, int64_t ldf, const double* G);
template <class T>   // Y += F G F^T X (T = float: the scaled pencil, D F G F^T D)
int nl_apply_add(Session* s, const T* X, int64_t ldx, int w, T* Y, int64_t ldy, cudaStream_t st);
template <class T>   // SMW step 6 on P = -K R (T = float: scaled P^ of the mixed form)
int nl_smw_correct(Session* s, T* P, int64_t ldp, int p, cudaStream_t st);
int nl_minres_index(Session* s, int grid, const std::vector<int64_t>& blk, int64_t kp);
int barrier_timeout_probe(double limit_s, cudaStream_t st);

// complex Hermitian input through the real-equivalent pencil (complex.cu)
int complex_realify_csr(int64_t n, const int64_t* rp, const int32_t* ci, const double* hv, const double* sv,
                        const int32_t* dof_node, std::vector<int64_t>& rp2, std::vector<int32_t>& ci2,
                        std::vector<double>& hv2, std::vector<double>& sv2, std::vector<int32_t>& node2);
void complex_realify_values(int64_t n, const int64_t* rp, const double* v, std::vector<double>& out);
int complex_start_block(Session* s, const double* X0c, int64_t ldc, int wc, double* Y, int64_t ldy);
int complex_recover(Session* s, int nev, double* lam_dev, double* Xc_dev, int64_t ldxc);

// ---- small utilities -----------------------------------------------------------------
inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace hbsd

struct hbsd_handle {
    hbsd::Session s;
};
