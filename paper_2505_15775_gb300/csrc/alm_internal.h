// Internal declarations shared by the translation units of the ALM-BM library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "alm.h"

namespace alm {

constexpr int kMaxLR = 4;        // low-rank terms of C
constexpr int kMaxRank = 32;     // rank cap (r_max)
constexpr int kLzMax = 64;       // Lanczos basis length per cycle
constexpr int kBlock = 256;      // threads per block of the row kernels
constexpr int kNumSMs = 152;     // GB300
constexpr int kPartStride = 160; // doubles of partial sums per block (>= kLzMax + 4, >= 1 + kMaxLR*kMaxRank)

// ------------------------------------------------------------------------------------
// host-built pattern (pattern.cpp)
// ------------------------------------------------------------------------------------
struct HostPattern {
    int64_t n = 0, m = 0;
    std::vector<int32_t> up_ptr, up_col;     // strict upper CSR
    std::vector<int32_t> up_row;             // row of each upper entry (COO)
    int ell_kf = 0, ell_ku = 0;              // ELL widths (0: no ELL layout)
    std::vector<int32_t> f_ell_col, u_ell_col;  // n x ell_kf / n x ell_ku, padded with the row itself
    std::vector<double> f_ell_val, u_ell_val;   // C_ij on them, 0 in the padding
    int ell_kn = 0;                          // narrow upper ELL width (<= ell_ku): most rows fit,
    std::vector<int32_t> un_col, ov_i, ov_j; // the rest of a longer row goes to an overflow list
    std::vector<double> un_val, ov_v;
    std::vector<double> up_c;                // C_ij on it (0 where only constraints)
    std::vector<int32_t> up_sel_k;           // selector constraint per upper entry (-1), if any
    std::vector<double> up_sel_a;
    std::vector<double> d_c;                 // C_ii
    std::vector<int32_t> d_sel_k;            // selector constraint of the diagonal entry (-1)
    std::vector<double> d_sel_a;
    std::vector<int32_t> f_ptr, f_col;       // full off-diagonal CSR
    std::vector<double> f_c;
    std::vector<int32_t> up_slot;            // 2 per upper entry: its (i,j) and (j,i) full slots
                                             // (when off_dynamic)
    std::vector<int32_t> g_con, g_ptr, g_i, g_j;  // general constraints, constraint-major
    std::vector<double> g_a;
    std::vector<int32_t> gd_ptr, gd_k;       // general constraints on diagonal entries, per row
    std::vector<double> gd_a;
    std::vector<int32_t> gu_ptr, gu_k;       // general constraints on upper entries, per entry
    std::vector<double> gu_a;
    bool has_off_sel = false, has_gen_diag = false, has_gen_off = false, off_dynamic = false;
    int64_t n_sel = 0, m_gen = 0;
    int lr_k = 0;
    std::vector<double> lr_u, lr_s;
    std::vector<double> b;
    double norm_b = 0.0, norm_C = 0.0;
};

std::string build_pattern(const alm_problem *p, HostPattern *hp);

// message returned by alm_last_error(NULL) (errors of calls without a handle)
void set_global_error(const std::string &msg);

// ------------------------------------------------------------------------------------
// device-side scalar state (one per handle, in device memory)
// ------------------------------------------------------------------------------------
struct DevState {
    // control of the inner loop
    int done;          // 0 run; 1 stop now; 2 stop after this step's update
    int iters;         // inner steps taken
    int status;        // alm_status raised on the device
    int max_inner;
    int restart;       // next CG direction is -G
    int method;        // ALM_INNER_CG / ALM_INNER_GD
    int lz_stop;       // Lanczos breakdown: skip the remaining steps of the cycle
    int lz_m;          // Lanczos steps done in this cycle
    int precond;       // 1: row-block Jacobi preconditioned CG directions
    int k1count;       // fused step+SpMM launches that ran in this inner solve (R ping-pong parity)
    float xcap2;       // staged FP32 step kernel: bound on |r_i|^2 for its next launch (0: none yet)
    unsigned int rmax2_bits;  // its running maximum of |r_i'|^2 (float bits) within one launch
    double pc_floor;   // lower bound of the diagonal 2 S_ii used by the preconditioner
    double zg, zg_prev;  // <Z, G> of the current / previous preconditioned gradient
    // scalars of the current iterate
    double sigma, tau_abs;
    double c0, yres, res2, bw, L;
    double gg, gg_prev, g_gprev, g_dprev, beta;
    double c1, c2, wa1, wa2, a11, a12, a22;
    double q[5];
    double alpha;
    double z[kMaxLR][kMaxRank];     // R^T u_l
    double zd[kMaxLR][kMaxRank];    // D^T u_l
    // Lanczos
    double lz_alpha[kLzMax], lz_beta[kLzMax];
    double h1[kLzMax + 1], h2[kLzMax + 1];
    double nrm2, anorm, theta, resid_est;
    double lz_s[kLzMax];
    double qu[kMaxLR];              // u_l^T q (current Lanczos vector)
    double red[8];                  // scratch results of small reductions
    unsigned int counter[16];       // last-block counters
};

enum Counter { CNT_EVAL = 0, CNT_DUAL, CNT_SPMM, CNT_LS, CNT_LZ, CNT_RED, CNT_GEN, CNT_AXPY };

// Per-row records read by the staged (cp.async) inner-step kernels, one 16-byte aligned
// record per row so that a row's scalars arrive with one or two 16-byte copies.
struct StepRec {      // fused step + SpMM, FP32 form (32 bytes)
    float base_hi, base_lo;  // C_ii - a_i y_k(i) as a float pair (rewritten per outer iteration)
    float b_hi, b_lo;        // b_k(i) of the row's diagonal selector as a float pair
    float af;                // a_i as float
    int k;                   // the row's diagonal selector constraint (-1: none)
    float rabs;              // sum of |C_ij| over the row's ELL entries
    float pad;
};
template <typename T>
struct LsRec;          // direction + line search: the row's selector and S_ii
template <>
struct alignas(16) LsRec<float> {   // 16 bytes
    float a;   // a_i of the row's diagonal selector (0 without one)
    int k;     // its constraint (-1: none)
    float ds;  // S_ii (leading float of the pair), rewritten by every slack-diagonal update
    int pad;
};
template <>
struct alignas(16) LsRec<double> {  // 32 bytes
    double a;
    double ds;
    int k;
    int pad[3];
};
static_assert(sizeof(StepRec) == 32 && sizeof(LsRec<float>) == 16 && sizeof(LsRec<double>) == 32, "record layout");

// ------------------------------------------------------------------------------------
// kernel-side views of the pattern
// ------------------------------------------------------------------------------------
template <typename T>
struct SparseView {
    int n, m;
    int64_t nnz_u;
    const int *up_row, *up_col;     // strict upper pattern in COO, sorted by row
    const int *up_ptr;              // ... and its row pointers (CSR)
    const T *up_c;                  // C_ij on it
    T *up_s;                        // S_ij on it (aliases up_c while S_off = C_off is static)
    const int *up_sel_k;            // may be null
    const double *up_sel_a;
    const T *d_c;
    const int *d_sel_k;
    const double *d_sel_a;
    const int *f_ptr, *f_col;
    T *f_val;                        // S_ij on the full pattern
    T *d_s;                          // S_ii (FP32 form: the leading float of a float pair)
    T *d_s_lo;                       // FP32 form: S_ii - d_s as a float (null in the FP64 form)
    const T *base_hi, *base_lo;      // C_ii - a_i y_k(i) for diagonal selectors, per outer iteration
    const T *b_hi, *b_lo;            // b_k(i) of the diagonal selector of row i, as a float pair
    const float *d_sel_af;           // a_i as float (diagonal selectors)
    const int *gd_ptr, *gd_k;        // may be null
    const double *gd_a;
    const int *gu_ptr, *gu_k;        // may be null
    const double *gu_a;
    int m_gen;
    const int *g_con, *g_ptr, *g_i, *g_j;
    const double *g_a;
    double *g_a1, *g_a2;             // per general constraint: A1, A2 of the line search
    int lr_k;
    const double *lr_u, *lr_s;
    const double *b;
    int off_dynamic, has_off_sel;
    int fused_dual;                  // every constraint is a diagonal selector: the dual update
                                     // and slack diagonal are computed inside k_eval
    int ell_kf, ell_ku;              // ELL widths of the full / strict upper pattern (0: none)
    const int *f_ell_col, *u_ell_col;
    const T *f_ell_val, *u_ell_val;  // S_ij = C_ij (ELL is built only when S_off is static)
    int ell_kn;                      // narrow strict-upper ELL (width ell_kn) plus overflow entries
    const int *un_col;
    const T *un_val;
    int64_t n_ov;
    const int *ov_i, *ov_j;
    const T *ov_v;
    StepRec *step_rec;               // per-row records of the staged step kernel (FP32, may be null)
    LsRec<T> *ls_rec;                // per-row records of the staged line-search kernel (may be null)
};

// Launch shape of the two kernels of an inner CG step (the fused step + SpMM and the fused
// direction + line search of the ELL form); chosen per handle by alm_autotune.
struct InnerCfg {
    int variant = 1;   // 0: rows loaded into registers; 1: rows staged by cp.async pipelines
    int stages = 2;    // variant 1: ring buffers per row group, rows in flight + 1 (2..4)
    int threads = 128; // variant 1: threads per CTA (128 or 256)
};

struct LaunchCtx {
    cudaStream_t stream;
    int sms;                  // multiprocessors of the device
    int grid;                 // upper bound on blocks (partials hold grid * kPartStride)
    double *partials;         // grid * kPartStride doubles
    DevState *st;
    int64_t *launches;        // host counter of kernel launches
    InnerCfg icfg;            // launch shape of the inner-step kernels
};

// kernels_sparse.cu
template <typename T>
void launch_eval(const LaunchCtx &c, const SparseView<T> &v, const T *R, int r, int ldr, double *AX,
                 const int *done, const double *y = nullptr, double *w = nullptr);
template <typename T>
void launch_dual_slack(const LaunchCtx &c, const SparseView<T> &v, const double *y, const double *AX,
                       double *w, const int *done, const int2 *up_slot);
template <typename T>
void launch_inner_slack(const LaunchCtx &c, const SparseView<T> &v, T *R, const T *D, int r, int ldr,
                        const int *done);
template <typename T>
void launch_prep_base(const LaunchCtx &c, const SparseView<T> &v, const double *y, T *base_hi, T *base_lo);
template <typename T>
void launch_spmm(const LaunchCtx &c, const SparseView<T> &v, const T *R, int r, int ldr, T *G,
                 const T *D, int mode, const int *done);
template <typename T>
void launch_dir(const LaunchCtx &c, const T *G, T *D, int64_t count, const int *done);
template <typename T>
void launch_ls(const LaunchCtx &c, const SparseView<T> &v, const T *R, const T *D, int r, int ldr,
               const double *w, int mode, const int *done);
template <typename T>
void launch_axpy(const LaunchCtx &c, T *R, const T *D, int64_t count, const int *done, int final_only = 0);
// inner-loop line search with the CG direction fused in (ELL form): D_new = -Z + beta D_old
template <typename T>
void launch_ls_dir(const LaunchCtx &c, const SparseView<T> &v, const T *R, const T *Z, const T *Dold, T *Dnew, int r,
                   int ldr, const int *done);
template <typename T>
bool ls_dir_fusable(const SparseView<T> &v);
// inner-loop SpMM with the pending step R_out = R_in + alpha D and the slack diagonal fused in
// (ELL, diagonal selectors; R_in and R_out different buffers)
template <typename T>
void launch_spmm_step(const LaunchCtx &c, const SparseView<T> &v, const T *Rin, T *Rout, int r, int ldr, T *G,
                      const T *D, const int *done);
template <typename T>
bool spmm_step_fusable(const SparseView<T> &v);
template <typename T>
void launch_relayout(const LaunchCtx &c, const T *src, int ld_src, T *dst, int ld_dst, int r, int64_t n,
                     const T *col, double scale);
template <typename T>
void launch_sumsq(const LaunchCtx &c, const double *x, int64_t m);

// kernels_growth.cu: rank growth along several eigenvectors (diagonal-selector problems)
template <typename T>
void launch_grow_moments(const LaunchCtx &c, const SparseView<T> &v, const T *V, int k, double *mom);
void launch_grow_sdp(const LaunchCtx &c, const double *mom, const double *lam, int k, double sigma, double *sqrtS,
                     int *info, double *dec);
template <typename T>
void launch_grow_append(const LaunchCtx &c, const T *V, int64_t n, int k, const double *sqrtS, T *dst, int ld,
                        int col0);
template <typename T>
void launch_to_double(const LaunchCtx &c, const T *src, int64_t n, double *dst);

// kernels_lanczos.cu
template <typename T>
void launch_lz_start(const LaunchCtx &c, T *q, int64_t n, uint64_t seed);
// q += (0.05 / sqrt(st->nrm2)) u, then st->nrm2 = |q|^2 (u from launch_lz_start)
template <typename T>
void launch_lz_mix(const LaunchCtx &c, T *q, const T *u, int64_t n);
template <typename T>
void launch_lz_spmv(const LaunchCtx &c, const SparseView<T> &v, const T *q, T *w);
template <typename T>
void launch_lz_reorth(const LaunchCtx &c, const T *Q, int64_t ldq, int nvec, T *w, int64_t n,
                      const double *h_in, double *h_out, int j, int stage);
template <typename T>
void launch_lz_spmv_reorth(const LaunchCtx &c, const SparseView<T> &v, const T *q, const T *Q, int64_t ldq, int nvec,
                           T *w, double *h_out, int j);
template <typename T>
void launch_lz_normalize(const LaunchCtx &c, const SparseView<T> &v, const T *src, T *dst, int64_t n,
                         int mode, int j);
void launch_lz_tridiag(const LaunchCtx &c, int m);
void launch_lz_reset(const LaunchCtx &c);
template <typename T>
void launch_lz_ritz(const LaunchCtx &c, const T *Q, int64_t ldq, int m, T *dst, int64_t n);
template <typename T>
void launch_lz_resid(const LaunchCtx &c, const T *w, const T *v, int64_t n);
void launch_set_state(const LaunchCtx &c, double sigma, double tau_abs, int max_inner, int method, int precond,
                      double pc_floor);

}  // namespace alm
