// C ABI of the ALM-BM library (include/alm.h) and the ALORA driver (arXiv
// 2505.15775, Alg. 1).  Host code here only orchestrates: every step of the path
// runs in the kernels of kernels_sparse.cu and kernels_lanczos.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "alm_internal.h"
#include "dev_util.cuh"

// A named NVTX range (solve, outer iteration, inner solve, eigensolve) for timeline
// profilers; NVTX does nothing unless a tool is attached.
struct NvtxRange {
    bool open = true;
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    void end() {
        if (open) {
            nvtxRangePop();
            open = false;
        }
    }
    ~NvtxRange() { end(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

using namespace alm;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct alm_handle {
    std::string err;
    std::string log_path;     // per-outer-iteration JSON lines (alm_set_log); empty: off
    bool inject_oom = false;  // ALM_FAULT_INJECT=oom: the next device allocation fails
    cudaStream_t stream = nullptr;
    alm_options opt{};
    int prec = ALM_FP64;
    size_t esz = 8;  // bytes of one element of R
    int64_t n = 0, m = 0, nnz_u = 0, nnz_f = 0, n_sel = 0, m_gen = 0;
    int lr_k = 0;
    bool off_sel = false, off_dynamic = false;
    double norm_b = 0.0, norm_C = 0.0;
    uint64_t problem_hash = 0;  // FNV-1a of the problem arrays (a checkpoint names its problem)
    InnerCfg icfg;              // launch shape of the inner-step kernels (alm_autotune)
    double pc_floor = 0.0;  // floor of S_ii in the CG preconditioner: 1e-2 (1 + mean |C_ii|)
    int grid = 0;
    int64_t launches = 0;
    std::vector<DevBuf> bufs;
    // pattern
    int *up_row = nullptr, *up_col = nullptr, *up_sel_k = nullptr, *d_sel_k = nullptr;
    int *f_ptr = nullptr, *f_col = nullptr;
    int2 *up_slot = nullptr;
    int *gd_ptr = nullptr, *gd_k = nullptr, *gu_ptr = nullptr, *gu_k = nullptr;
    int *g_con = nullptr, *g_ptr = nullptr, *g_i = nullptr, *g_j = nullptr;
    void *up_c = nullptr, *up_s = nullptr, *d_c = nullptr, *f_val = nullptr, *d_s = nullptr;
    void *d_s_lo = nullptr, *base_hi = nullptr, *base_lo = nullptr, *b_hi = nullptr, *b_lo = nullptr;
    int *up_ptr = nullptr;
    float *d_sel_af = nullptr;
    int ell_kf = 0, ell_ku = 0;
    int *f_ell_col = nullptr, *u_ell_col = nullptr;
    void *f_ell_val = nullptr, *u_ell_val = nullptr;
    int ell_kn = 0;
    int64_t n_ov = 0;
    int *un_col = nullptr, *ov_i = nullptr, *ov_j = nullptr;
    void *un_val = nullptr, *ov_v = nullptr;
    StepRec *step_rec = nullptr;
    void *ls_rec = nullptr;  // LsRec<float> or LsRec<double> per row
    bool fused_dual = false;
    int sms = 0;
    double *up_sel_a = nullptr, *d_sel_a = nullptr, *gd_a = nullptr, *gu_a = nullptr, *g_a = nullptr;
    double *g_a1 = nullptr, *g_a2 = nullptr, *lr_u = nullptr, *lr_s = nullptr, *b = nullptr;
    // state and work
    DevState *st = nullptr;
    double *partials = nullptr;
    int *zero_flag = nullptr;
    double *AX = nullptr, *AXtmp = nullptr, *w = nullptr, *y = nullptr, *zeros_m = nullptr;
    // solver / Lanczos buffers (allocated on first use)
    void *Rb[2] = {nullptr, nullptr};
    void *G = nullptr, *D = nullptr, *D2 = nullptr, *Q = nullptr, *lzw = nullptr;  // D2: ping-pong partner of D
    int Q_cols = 0;
    int work_rmax = 0;
    // host mirrors
    DevState *h_st = nullptr;  // pinned
    cudaEvent_t prof_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t graph = nullptr;
    int graph_r = -1, graph_ldr = -1, graph_cur = -1;
    int64_t graph_launches = 0;
    cudaGraphExec_t lz_graph = nullptr;  // one Lanczos restart cycle (kk steps), captured
    int lz_graph_k = -1, lz_graph_lr = -1;
    // rank growth along several eigenvectors: the found eigenvectors deflated as low-rank
    // terms of S (after C's own), the directions V (n x 4), and the small SDP's data
    double *defl_u = nullptr, *defl_s = nullptr;
    void *grow_V = nullptr;
    double *grow_mom = nullptr, *grow_lam = nullptr, *grow_sqrt = nullptr, *grow_dec = nullptr;
    int *grow_info = nullptr;
    const void *lz_graph_Q = nullptr;
    int64_t lz_graph_launches = 0;
    bool fused_step = false;  // the last enqueued inner chunk used the fused step+SpMM kernel
    // state of the last solve at its end (what alm_checkpoint saves and alm_resume restores):
    // the factor is in Rb[ss_cur] (row stride ss_ldr), y in y, the last Ritz vector in Q[:, 0]
    struct SolveState {
        int32_t valid = 0, r = 0, ldr = 0, cur = 0, outer_done = 0, lz_before = 0, growth_steps = 0, pad = 0;
        double sigma = 0.0, tau_in = 0.0, kkt_prev = -1.0, p_prev = 0.0, lam = 0.0;
        int64_t inner_total = 0, lanczos_matvecs = 0;
    } ss;
};

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return e_ == cudaErrorMemoryAllocation ? ALM_ERR_OOM : ALM_ERR_CUDA;          \
        }                                                                                 \
    } while (0)

#define FAIL(code, msg)      \
    do {                     \
        h->err = (msg);      \
        return (code);       \
    } while (0)

#define TRY(expr)                              \
    do {                                       \
        alm_status s_ = (expr);                \
        if (s_ != ALM_OK) return s_;           \
    } while (0)

namespace alm {

void set_global_error(const std::string &msg) { g_create_error = msg; }

__global__ void k_set_state(DevState *st, double sigma, double tau_abs, int max_inner, int method, int precond,
                            double pc_floor) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->precond = precond;
        st->pc_floor = pc_floor;
        st->zg_prev = 0.0;
        st->sigma = sigma;
        st->tau_abs = tau_abs;
        st->max_inner = max_inner;
        st->method = method;
        st->done = 0;
        st->iters = 0;
        st->status = 0;
        st->restart = 1;
        st->gg_prev = 0.0;
        st->beta = 0.0;
        st->alpha = 0.0;  // no pending step at the start of an inner solve
        st->k1count = 0;
        st->xcap2 = 0.f;
        st->rmax2_bits = 0u;
    }
}

void launch_set_state(const LaunchCtx &c, double sigma, double tau_abs, int max_inner, int method, int precond,
                      double pc_floor) {
    k_set_state<<<1, 32, 0, c.stream>>>(c.st, sigma, tau_abs, max_inner, method, precond, pc_floor);
    ++*c.launches;
}

}  // namespace alm

static alm_status dalloc(alm_handle *h, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return ALM_OK;
    if (h->inject_oom) {
        h->inject_oom = false;
        FAIL(ALM_ERR_OOM, "cudaMalloc: out of memory (injected by ALM_FAULT_INJECT=oom)");
    }
    CK(cudaMalloc(p, bytes));
    h->bufs.push_back({*p, bytes});
    return ALM_OK;
}

template <typename V>
static alm_status upload(alm_handle *h, V **dst, const std::vector<V> &src) {
    *dst = nullptr;
    if (src.empty()) return ALM_OK;
    void *p = nullptr;
    TRY(dalloc(h, &p, sizeof(V) * src.size()));
    CK(cudaMemcpyAsync(p, src.data(), sizeof(V) * src.size(), cudaMemcpyHostToDevice, h->stream));
    *dst = static_cast<V *>(p);
    return ALM_OK;
}

// upload doubles converted to the working precision (scaled)
static alm_status upload_T(alm_handle *h, void **dst, const std::vector<double> &src, double scale) {
    *dst = nullptr;
    if (src.empty()) return ALM_OK;
    if (h->prec == ALM_FP64) {
        std::vector<double> t(src.size());
        for (size_t k = 0; k < src.size(); ++k) t[k] = scale * src[k];
        double *p = nullptr;
        TRY(upload(h, &p, t));
        CK(cudaStreamSynchronize(h->stream));
        *dst = p;
    } else {
        std::vector<float> t(src.size());
        for (size_t k = 0; k < src.size(); ++k) t[k] = float(scale * src[k]);
        float *p = nullptr;
        TRY(upload(h, &p, t));
        CK(cudaStreamSynchronize(h->stream));
        *dst = p;
    }
    return ALM_OK;
}

template <typename T>
static SparseView<T> view(const alm_handle *h) {
    SparseView<T> v{};
    v.n = int(h->n);
    v.m = int(h->m);
    v.nnz_u = h->nnz_u;
    v.up_row = h->up_row;
    v.up_col = h->up_col;
    v.up_ptr = h->up_ptr;
    v.d_s_lo = static_cast<T *>(h->d_s_lo);
    v.base_hi = static_cast<const T *>(h->base_hi);
    v.base_lo = static_cast<const T *>(h->base_lo);
    v.b_hi = static_cast<const T *>(h->b_hi);
    v.b_lo = static_cast<const T *>(h->b_lo);
    v.d_sel_af = h->d_sel_af;
    v.ell_kf = h->ell_kf;
    v.ell_ku = h->ell_ku;
    v.f_ell_col = h->f_ell_col;
    v.u_ell_col = h->u_ell_col;
    v.f_ell_val = static_cast<const T *>(h->f_ell_val);
    v.u_ell_val = static_cast<const T *>(h->u_ell_val);
    v.ell_kn = h->ell_kn;
    v.un_col = h->un_col;
    v.un_val = static_cast<const T *>(h->un_val);
    v.n_ov = h->n_ov;
    v.ov_i = h->ov_i;
    v.ov_j = h->ov_j;
    v.ov_v = static_cast<const T *>(h->ov_v);
    v.step_rec = h->step_rec;
    v.ls_rec = static_cast<LsRec<T> *>(h->ls_rec);
    v.up_c = static_cast<const T *>(h->up_c);
    v.up_s = static_cast<T *>(h->up_s);
    v.up_sel_k = h->up_sel_k;
    v.up_sel_a = h->up_sel_a;
    v.d_c = static_cast<const T *>(h->d_c);
    v.d_sel_k = h->d_sel_k;
    v.d_sel_a = h->d_sel_a;
    v.f_ptr = h->f_ptr;
    v.f_col = h->f_col;
    v.f_val = static_cast<T *>(h->f_val);
    v.d_s = static_cast<T *>(h->d_s);
    v.gd_ptr = h->gd_ptr;
    v.gd_k = h->gd_k;
    v.gd_a = h->gd_a;
    v.gu_ptr = h->gu_ptr;
    v.gu_k = h->gu_k;
    v.gu_a = h->gu_a;
    v.m_gen = int(h->m_gen);
    v.g_con = h->g_con;
    v.g_ptr = h->g_ptr;
    v.g_i = h->g_i;
    v.g_j = h->g_j;
    v.g_a = h->g_a;
    v.g_a1 = h->g_a1;
    v.g_a2 = h->g_a2;
    v.lr_k = h->lr_k;
    v.lr_u = h->lr_u;
    v.lr_s = h->lr_s;
    v.b = h->b;
    v.off_dynamic = h->off_dynamic ? 1 : 0;
    v.has_off_sel = h->off_sel ? 1 : 0;
    v.fused_dual = h->fused_dual ? 1 : 0;
    return v;
}

static LaunchCtx ctx(alm_handle *h) {
    LaunchCtx c;
    c.stream = h->stream;
    c.sms = h->sms;
    c.grid = h->grid;
    c.partials = h->partials;
    c.st = h->st;
    c.launches = &h->launches;
    c.icfg = h->icfg;
    return c;
}

static int vec_width(const alm_handle *h) { return h->prec == ALM_FP64 ? 2 : 4; }
static int pad_rank(const alm_handle *h, int r) {
    const int W = vec_width(h);
    return (r + W - 1) / W * W;
}

static alm_status check_factor(alm_handle *h, const void *R, int r, int ldr, bool allow_null = false) {
    if (!R) {
        if (allow_null && r == 0) return ALM_OK;
        FAIL(ALM_ERR_INVALID_ARG, "factor pointer is NULL");
    }
    if (r < 1 || r > kMaxRank) FAIL(ALM_ERR_INVALID_ARG, "rank r must be in 1..32");
    if (ldr < r) FAIL(ALM_ERR_INVALID_ARG, "ldr must be >= r");
    if ((size_t(ldr) * h->esz) % 16 != 0) FAIL(ALM_ERR_INVALID_ARG, "ldr * element size must be a multiple of 16 bytes");
    if (reinterpret_cast<uintptr_t>(R) % 16 != 0) FAIL(ALM_ERR_INVALID_ARG, "factor pointer must be 16-byte aligned");
    return ALM_OK;
}

static alm_status sync_state(alm_handle *h) {
    CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ALM_OK;
}

// ------------------------------------------------------------------------------------
// create / destroy
// ------------------------------------------------------------------------------------
extern "C" void alm_default_options(alm_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = ALM_FP64;
    o->r_max = 32;
    o->sigma0 = 1.0;
    o->sigma_rule = ALM_SIGMA_FIXED;
    o->sigma_max = 1e6;
    o->eps = 1e-6;
    o->max_outer = 200;
    o->max_inner = 5000;
    o->inner_method = ALM_INNER_CG;
    o->inner_rel = 0.1;
    o->inner_floor = 0.1;
    o->inner_start = 0.1;
    o->inner_decay = 0.7;
    o->lanczos_k = 32;
    o->lanczos_max_restarts = 400;
    o->lanczos_tol = 1e-10;
    o->seed = 0x5eed;
    o->chunk = 16;
    o->use_graph = 1;
    o->profile = 0;
    o->verbose = 0;
    o->inner_precond = 1;
    o->lanczos_warm = 0;
    o->growth_k = 1;
}

// 64-bit FNV-1a over the bytes of the problem's arrays, in a fixed order
static uint64_t problem_fingerprint(const alm_problem *p) {
    uint64_t x = 0xcbf29ce484222325ULL;
    auto mix = [&x](const void *data, size_t bytes) {
        const unsigned char *c = static_cast<const unsigned char *>(data);
        for (size_t k = 0; k < bytes; ++k) x = (x ^ c[k]) * 0x100000001b3ULL;
    };
    mix(&p->n, sizeof(p->n));
    mix(&p->m, sizeof(p->m));
    mix(&p->c_nnz, sizeof(p->c_nnz));
    mix(&p->a_nnz, sizeof(p->a_nnz));
    mix(&p->c_lr_k, sizeof(p->c_lr_k));
    const size_t cn = size_t(p->c_nnz), an = size_t(p->a_nnz), lk = size_t(p->c_lr_k);
    if (cn) {
        mix(p->c_i, cn * sizeof(int32_t));
        mix(p->c_j, cn * sizeof(int32_t));
        mix(p->c_v, cn * sizeof(double));
    }
    if (an) {
        mix(p->a_k, an * sizeof(int32_t));
        mix(p->a_i, an * sizeof(int32_t));
        mix(p->a_j, an * sizeof(int32_t));
        mix(p->a_v, an * sizeof(double));
    }
    if (lk) {
        mix(p->c_lr_u, lk * size_t(p->n) * sizeof(double));
        mix(p->c_lr_s, lk * sizeof(double));
    }
    if (p->m > 0) mix(p->b, size_t(p->m) * sizeof(double));
    return x;
}

static alm_status create_impl(alm_handle *h, const alm_problem *p, const alm_options *o) {
    HostPattern hp;
    std::string e = build_pattern(p, &hp);
    if (!e.empty()) FAIL(ALM_ERR_INVALID_ARG, e);
    h->problem_hash = problem_fingerprint(p);
    h->n = hp.n;
    h->m = hp.m;
    h->nnz_u = int64_t(hp.up_col.size());
    h->nnz_f = int64_t(hp.f_col.size());
    h->n_sel = hp.n_sel;
    h->m_gen = hp.m_gen;
    h->lr_k = hp.lr_k;
    h->off_sel = hp.has_off_sel;
    h->off_dynamic = hp.off_dynamic;
    h->norm_b = hp.norm_b;
    h->norm_C = hp.norm_C;
    {
        double acd = 0.0;
        for (double v : hp.d_c) acd += std::fabs(v);
        h->pc_floor = 1e-2 * (1.0 + acd / double(hp.n));
    }
    int dev = 0, sms = kNumSMs;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    h->sms = sms;
    h->grid = sms * (2048 / kBlock);
    // all constraints are diagonal selectors (MaxCut-like): the dual update is fused into k_eval
    h->fused_dual = hp.m_gen == 0 && !hp.has_off_sel && hp.n_sel == hp.m;

    TRY(upload(h, &h->up_row, hp.up_row));
    h->ell_kf = hp.ell_kf;
    h->ell_ku = hp.ell_ku;
    if (hp.ell_kf > 0) {
        TRY(upload(h, &h->f_ell_col, hp.f_ell_col));
        TRY(upload(h, &h->u_ell_col, hp.u_ell_col));
        TRY(upload_T(h, &h->f_ell_val, hp.f_ell_val, 1.0));
        TRY(upload_T(h, &h->u_ell_val, hp.u_ell_val, 1.0));
        h->ell_kn = hp.ell_kn;
        h->n_ov = int64_t(hp.ov_i.size());
        TRY(upload(h, &h->un_col, hp.un_col));
        TRY(upload_T(h, &h->un_val, hp.un_val, 1.0));
        TRY(upload(h, &h->ov_i, hp.ov_i));
        TRY(upload(h, &h->ov_j, hp.ov_j));
        TRY(upload_T(h, &h->ov_v, hp.ov_v, 1.0));
    }
    TRY(upload(h, &h->up_ptr, hp.up_ptr));
    TRY(upload(h, &h->up_col, hp.up_col));
    {
        std::vector<float> af(hp.d_sel_a.begin(), hp.d_sel_a.end());
        TRY(upload(h, &h->d_sel_af, af));
    }
    if (h->prec == ALM_FP32) TRY(dalloc(h, &h->d_s_lo, sizeof(float) * size_t(h->n)));
    if (h->fused_dual) {
        // b of the diagonal selector of each row, as a float pair (FP32 form) or a double
        std::vector<double> bh(size_t(h->n), 0.0), bl(size_t(h->n), 0.0);
        for (int64_t i = 0; i < h->n; ++i) {
            const int32_t k = hp.d_sel_k[size_t(i)];
            if (k < 0) continue;
            const double bk = hp.b[size_t(k)];
            if (h->prec == ALM_FP32) {
                bh[size_t(i)] = double(float(bk));
                bl[size_t(i)] = bk - bh[size_t(i)];
            } else {
                bh[size_t(i)] = bk;
            }
        }
        TRY(upload_T(h, &h->b_hi, bh, 1.0));
        TRY(dalloc(h, &h->base_hi, h->esz * size_t(h->n)));
        if (h->prec == ALM_FP32) {
            TRY(upload_T(h, &h->b_lo, bl, 1.0));
            TRY(dalloc(h, &h->base_lo, sizeof(float) * size_t(h->n)));
        }
        if (hp.ell_kf > 0) {
            // per-row records of the staged inner-step kernels (the step kernel's: FP32 form;
            // its base fields are written per outer iteration by launch_prep_base)
            auto ls_records = [&](auto tag) -> alm_status {
                using Rec = LsRec<decltype(tag)>;
                std::vector<Rec> lr(size_t(h->n));
                for (int64_t i = 0; i < h->n; ++i) {
                    lr[size_t(i)] = Rec{};
                    lr[size_t(i)].a = decltype(lr[size_t(i)].a)(hp.d_sel_a[size_t(i)]);
                    lr[size_t(i)].k = hp.d_sel_k[size_t(i)];
                }
                Rec *d = nullptr;
                TRY(upload(h, &d, lr));
                h->ls_rec = d;
                return ALM_OK;
            };
            if (h->prec == ALM_FP32) TRY(ls_records(float{}));
            else TRY(ls_records(double{}));
            if (h->prec == ALM_FP32) {
                std::vector<StepRec> sr(size_t(h->n));
                for (int64_t i = 0; i < h->n; ++i) {
                    StepRec &q = sr[size_t(i)];
                    q.base_hi = q.base_lo = 0.f;
                    q.b_hi = float(bh[size_t(i)]);
                    q.b_lo = float(bl[size_t(i)]);
                    q.af = float(hp.d_sel_a[size_t(i)]);
                    q.k = hp.d_sel_k[size_t(i)];
                    double ra = 0.0;
                    for (int t = 0; t < hp.ell_kf; ++t) ra += std::fabs(hp.f_ell_val[size_t(i) * hp.ell_kf + t]);
                    q.rabs = float(ra * (1.0 + 1e-6));  // rounded up
                    q.pad = 0.f;
                }
                TRY(upload(h, &h->step_rec, sr));
            }
        }
    }
    TRY(upload_T(h, &h->up_c, hp.up_c, 1.0));
    if (hp.off_dynamic) TRY(upload_T(h, &h->up_s, hp.up_c, 1.0));  // S_ij, rewritten by every slack update
    else h->up_s = h->up_c;                                         // S_ij = C_ij for good
    TRY(upload(h, &h->up_sel_k, hp.up_sel_k));
    TRY(upload(h, &h->up_sel_a, hp.up_sel_a));
    TRY(upload_T(h, &h->d_c, hp.d_c, 1.0));
    TRY(upload(h, &h->d_sel_k, hp.d_sel_k));
    TRY(upload(h, &h->d_sel_a, hp.d_sel_a));
    TRY(upload(h, &h->f_ptr, hp.f_ptr));
    TRY(upload(h, &h->f_col, hp.f_col));
    TRY(upload_T(h, &h->f_val, hp.f_c, 1.0));  // S_off = C_off until a slack update
    if (hp.off_dynamic) {
        int32_t *slot = nullptr;
        TRY(upload(h, &slot, hp.up_slot));
        h->up_slot = reinterpret_cast<int2 *>(slot);
    }
    TRY(dalloc(h, &h->d_s, h->esz * size_t(h->n)));
    TRY(upload(h, &h->gd_ptr, hp.gd_ptr));
    TRY(upload(h, &h->gd_k, hp.gd_k));
    TRY(upload(h, &h->gd_a, hp.gd_a));
    TRY(upload(h, &h->gu_ptr, hp.gu_ptr));
    TRY(upload(h, &h->gu_k, hp.gu_k));
    TRY(upload(h, &h->gu_a, hp.gu_a));
    TRY(upload(h, &h->g_con, hp.g_con));
    TRY(upload(h, &h->g_ptr, hp.g_ptr));
    TRY(upload(h, &h->g_i, hp.g_i));
    TRY(upload(h, &h->g_j, hp.g_j));
    TRY(upload(h, &h->g_a, hp.g_a));
    if (hp.m_gen > 0) {
        TRY(dalloc(h, reinterpret_cast<void **>(&h->g_a1), sizeof(double) * size_t(hp.m_gen)));
        TRY(dalloc(h, reinterpret_cast<void **>(&h->g_a2), sizeof(double) * size_t(hp.m_gen)));
    }
    TRY(upload(h, &h->lr_u, hp.lr_u));
    TRY(upload(h, &h->lr_s, hp.lr_s));
    TRY(upload(h, &h->b, hp.b));
    TRY(dalloc(h, reinterpret_cast<void **>(&h->st), sizeof(DevState)));
    CK(cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream));
    TRY(dalloc(h, reinterpret_cast<void **>(&h->partials), sizeof(double) * size_t(h->grid) * kPartStride));
    TRY(dalloc(h, reinterpret_cast<void **>(&h->zero_flag), sizeof(int) * 4));
    CK(cudaMemsetAsync(h->zero_flag, 0, sizeof(int) * 4, h->stream));
    TRY(dalloc(h, reinterpret_cast<void **>(&h->AX), sizeof(double) * size_t(h->m)));
    TRY(dalloc(h, reinterpret_cast<void **>(&h->AXtmp), sizeof(double) * size_t(h->m)));
    TRY(dalloc(h, reinterpret_cast<void **>(&h->w), sizeof(double) * size_t(h->m)));
    TRY(dalloc(h, reinterpret_cast<void **>(&h->y), sizeof(double) * size_t(h->m)));
    TRY(dalloc(h, reinterpret_cast<void **>(&h->zeros_m), sizeof(double) * size_t(h->m)));
    CK(cudaMemsetAsync(h->zeros_m, 0, sizeof(double) * size_t(h->m), h->stream));
    CK(cudaMallocHost(reinterpret_cast<void **>(&h->h_st), sizeof(DevState)));
    for (auto &e : h->prof_ev) CK(cudaEventCreate(&e));
    CK(cudaStreamSynchronize(h->stream));
    (void)o;
    return ALM_OK;
}

extern "C" alm_status alm_create(alm_handle **out, const alm_problem *p, const alm_options *o, alm_stream_t s) {
    if (!out) {
        g_create_error = "output handle pointer is NULL";
        return ALM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    alm_handle *h = new (std::nothrow) alm_handle();
    if (!h) {
        g_create_error = "host allocation failed";
        return ALM_ERR_OOM;
    }
    if (o) h->opt = *o;
    else alm_default_options(&h->opt);
    const alm_options &op = h->opt;
    alm_status st = ALM_OK;
    if (op.precision != ALM_FP64 && op.precision != ALM_FP32) st = ALM_ERR_INVALID_ARG, h->err = "precision must be ALM_FP64 or ALM_FP32";
    else if (op.r_max < 1 || op.r_max > kMaxRank) st = ALM_ERR_INVALID_ARG, h->err = "r_max must be in 1..32";
    else if (op.lanczos_k < 2 || op.lanczos_k > kLzMax) st = ALM_ERR_INVALID_ARG, h->err = "lanczos_k must be in 2..64";
    else if (!(op.sigma0 > 0.0) || !(op.eps > 0.0)) st = ALM_ERR_INVALID_ARG, h->err = "sigma0 and eps must be > 0";
    else if (op.chunk < 1 || op.chunk > 256) st = ALM_ERR_INVALID_ARG, h->err = "chunk must be in 1..256";
    else if (op.growth_k < 1 || op.growth_k > 4) st = ALM_ERR_INVALID_ARG, h->err = "growth_k must be in 1..4";
    // host-side fault injection: corrupt a private copy of the problem, or fail an allocation
    alm_problem pf{};
    std::vector<double> b_bad;
    std::vector<int32_t> ai_bad;
    if (st == ALM_OK && p) {
        if (const char *fi = std::getenv("ALM_FAULT_INJECT")) {
            const std::string mode(fi);
            pf = *p;
            if (mode == "nan_b" && p->m > 0 && p->b) {
                b_bad.assign(p->b, p->b + p->m);
                b_bad[0] = std::nan("");
                pf.b = b_bad.data();
                p = &pf;
            } else if (mode == "csr" && p->a_nnz > 0 && p->a_i) {
                ai_bad.assign(p->a_i, p->a_i + p->a_nnz);
                ai_bad[0] = int32_t(p->n);
                pf.a_i = ai_bad.data();
                p = &pf;
            } else if (mode == "oom") {
                h->inject_oom = true;
            } else if (!mode.empty() && mode != "nan_b" && mode != "csr") {
                st = ALM_ERR_INVALID_ARG, h->err = "unknown ALM_FAULT_INJECT value (nan_b, csr or oom)";
            }
        }
    }
    if (st == ALM_OK) {
        h->prec = op.precision;
        h->esz = op.precision == ALM_FP64 ? 8 : 4;
        h->stream = static_cast<cudaStream_t>(s);
        st = create_impl(h, p, o);
    }
    if (st != ALM_OK) {
        g_create_error = h->err;
        alm_destroy(h);
        return st;
    }
    *out = h;
    return ALM_OK;
}

extern "C" void alm_destroy(alm_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->lz_graph) cudaGraphExecDestroy(h->lz_graph);
    for (void *p : {static_cast<void *>(h->defl_u), static_cast<void *>(h->defl_s), h->grow_V,
                    static_cast<void *>(h->grow_mom), static_cast<void *>(h->grow_lam),
                    static_cast<void *>(h->grow_sqrt), static_cast<void *>(h->grow_dec),
                    static_cast<void *>(h->grow_info)})
        if (p) cudaFree(p);
    for (auto &b : h->bufs) cudaFree(b.p);
    for (void *p : {h->Rb[0], h->Rb[1], h->G, h->D, h->D2, h->Q, h->lzw})
        if (p) cudaFree(p);
    for (auto e : h->prof_ev)
        if (e) cudaEventDestroy(e);
    if (h->h_st) cudaFreeHost(h->h_st);
    delete h;
}

extern "C" const char *alm_last_error(const alm_handle *h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

extern "C" const char *alm_version(void) { return "alm-bm sm_103a (fp64 + fp32 kernels)"; }

extern "C" alm_status alm_pattern_info(const alm_handle *h, int64_t *out) {
    if (!h || !out) return ALM_ERR_INVALID_ARG;
    out[0] = h->n;
    out[1] = h->m;
    out[2] = h->nnz_u;
    out[3] = h->nnz_f;
    out[4] = h->n_sel;
    out[5] = h->m_gen;
    out[6] = h->off_dynamic ? 1 : 0;
    return ALM_OK;
}

// A(RR^T), <C, RR^T>, w = y - sigma(A(RR^T) - b), S = C - A^*(w) and L at the factor R:
// one fused kernel for diagonal-selector problems, eval + dual/slack update otherwise.
template <typename T>
static void eval_dual(alm_handle *h, const LaunchCtx &c, const SparseView<T> &v, const T *R, int r, int ldr,
                      const double *y, double *AX, const int *done) {
    if (h->fused_dual) {
        launch_eval<T>(c, v, R, r, ldr, AX, done, y, h->w);
    } else {
        launch_eval<T>(c, v, R, r, ldr, AX, done);
        launch_dual_slack<T>(c, v, y, AX, h->w, done, h->up_slot);
    }
}

// ------------------------------------------------------------------------------------
// primitives
// ------------------------------------------------------------------------------------
template <typename T>
static alm_status eval_and_dual(alm_handle *h, const void *R, int r, int ldr, const double *y, double sigma,
                                double *AXbuf) {
    LaunchCtx c = ctx(h);
    const SparseView<T> v = view<T>(h);
    launch_set_state(c, sigma, 0.0, 0, ALM_INNER_GD, 0, 0.0);
    if (R) {
        eval_dual<T>(h, c, v, static_cast<const T *>(R), r, ldr, y ? y : h->zeros_m, AXbuf, h->zero_flag);
    } else {
        CK(cudaMemsetAsync(AXbuf, 0, sizeof(double) * size_t(h->m), h->stream));
        CK(cudaMemsetAsync(&h->st->c0, 0, sizeof(double), h->stream));
        launch_dual_slack<T>(c, v, y ? y : h->zeros_m, AXbuf, h->w, h->zero_flag, h->up_slot);
    }
    CK(cudaGetLastError());
    return ALM_OK;
}

template <typename T>
static alm_status eval_prim(alm_handle *h, const void *R, int r, int ldr, const double *y, double sigma, double *L_out,
                            double *AX_out, double *CX_out) {
    TRY(eval_and_dual<T>(h, R, r, ldr, y, sigma, AX_out ? AX_out : h->AX));
    if (L_out || CX_out) {
        TRY(sync_state(h));
        if (L_out) *L_out = h->h_st->L;
        if (CX_out) *CX_out = h->h_st->c0;
        if (h->h_st->status) FAIL(alm_status(h->h_st->status), "non-finite value in the augmented Lagrangian");
    }
    return ALM_OK;
}

extern "C" alm_status alm_eval(alm_handle *h, const void *R, int32_t r, int32_t ldr, const double *y, double sigma,
                               double *L_out, double *AX_out, double *CX_out) {
    if (!h) return ALM_ERR_INVALID_ARG;
    TRY(check_factor(h, R, r, ldr));
    if (!std::isfinite(sigma) || sigma < 0) FAIL(ALM_ERR_INVALID_ARG, "sigma must be finite and >= 0");
    if (h->prec == ALM_FP64) return eval_prim<double>(h, R, r, ldr, y, sigma, L_out, AX_out, CX_out);
    return eval_prim<float>(h, R, r, ldr, y, sigma, L_out, AX_out, CX_out);
}

template <typename T>
static alm_status grad_prim(alm_handle *h, const void *R, int r, int ldr, const double *y, double sigma, void *G,
                            double *gnorm2_out) {
    TRY(eval_and_dual<T>(h, R, r, ldr, y, sigma, h->AX));
    const int W = vec_width(h);
    int L = 1;
    while (L * W < r) L <<= 1;
    if (ldr > L * W) CK(cudaMemsetAsync(G, 0, h->esz * size_t(h->n) * size_t(ldr), h->stream));
    launch_spmm<T>(ctx(h), view<T>(h), static_cast<const T *>(R), r, ldr, static_cast<T *>(G), nullptr, 0,
                   h->zero_flag);
    CK(cudaGetLastError());
    if (gnorm2_out) {
        TRY(sync_state(h));
        *gnorm2_out = h->h_st->gg;
    }
    return ALM_OK;
}

extern "C" alm_status alm_grad(alm_handle *h, const void *R, int32_t r, int32_t ldr, const double *y, double sigma,
                               void *G, double *gnorm2_out) {
    if (!h) return ALM_ERR_INVALID_ARG;
    TRY(check_factor(h, R, r, ldr));
    TRY(check_factor(h, G, r, ldr));
    if (G == R) FAIL(ALM_ERR_INVALID_ARG, "G may not alias R");
    if (!std::isfinite(sigma) || sigma < 0) FAIL(ALM_ERR_INVALID_ARG, "sigma must be finite and >= 0");
    if (h->prec == ALM_FP64) return grad_prim<double>(h, R, r, ldr, y, sigma, G, gnorm2_out);
    return grad_prim<float>(h, R, r, ldr, y, sigma, G, gnorm2_out);
}

template <typename T>
static alm_status ls_prim(alm_handle *h, const void *R, const void *D, int r, int ldr, const double *y, double sigma,
                          double *coeffs_out, double *alpha_out) {
    TRY(eval_and_dual<T>(h, R, r, ldr, y, sigma, h->AX));
    launch_ls<T>(ctx(h), view<T>(h), static_cast<const T *>(R), static_cast<const T *>(D), r, ldr, h->w, 0,
                 h->zero_flag);
    CK(cudaGetLastError());
    TRY(sync_state(h));
    if (coeffs_out)
        for (int k = 0; k < 5; ++k) coeffs_out[k] = h->h_st->q[k];
    if (alpha_out) *alpha_out = h->h_st->alpha;
    if (h->h_st->status == ALM_ERR_UNBOUNDED) FAIL(ALM_ERR_UNBOUNDED, "phi(alpha) is unbounded below on alpha >= 0");
    if (h->h_st->status) FAIL(alm_status(h->h_st->status), "non-finite value in the line search");
    return ALM_OK;
}

extern "C" alm_status alm_linesearch(alm_handle *h, const void *R, const void *D, int32_t r, int32_t ldr,
                                     const double *y, double sigma, double *coeffs_out, double *alpha_out) {
    if (!h) return ALM_ERR_INVALID_ARG;
    TRY(check_factor(h, R, r, ldr));
    TRY(check_factor(h, D, r, ldr));
    if (!std::isfinite(sigma) || sigma < 0) FAIL(ALM_ERR_INVALID_ARG, "sigma must be finite and >= 0");
    if (h->prec == ALM_FP64) return ls_prim<double>(h, R, D, r, ldr, y, sigma, coeffs_out, alpha_out);
    return ls_prim<float>(h, R, D, r, ldr, y, sigma, coeffs_out, alpha_out);
}

// ------------------------------------------------------------------------------------
// Lanczos driver
// ------------------------------------------------------------------------------------
static alm_status ensure_lanczos(alm_handle *h, int k) {
    if (h->Q && h->Q_cols >= k + 1) return ALM_OK;
    if (h->lz_graph) {  // it holds the old basis pointers
        cudaStreamSynchronize(h->stream);
        cudaGraphExecDestroy(h->lz_graph);
        h->lz_graph = nullptr;
    }
    if (h->Q) cudaFree(h->Q);
    if (h->lzw) cudaFree(h->lzw);
    h->Q = h->lzw = nullptr;
    CK(cudaMalloc(&h->Q, h->esz * size_t(h->n) * size_t(k + 1)));
    CK(cudaMalloc(&h->lzw, h->esz * size_t(h->n)));
    h->Q_cols = k + 1;
    return ALM_OK;
}

// smallest eigenpair of the S currently held by the handle (d_s, f_val and the
// low-rank part).  On return the unit Ritz vector is Q[:, 0].
template <typename T>
static alm_status lanczos(alm_handle *h, int k, int max_restarts, double tol_rel, double tol_abs, uint64_t seed,
                          double *theta_out, double *resid_out, int64_t *matvecs, bool warm = false, int nlock = 0) {
    TRY(ensure_lanczos(h, k));
    // FP32 vectors keep orthogonality to about 1e-7: a residual below ~1e-5 ||S|| is not reachable
    if (h->prec == ALM_FP32) tol_rel = std::max(tol_rel, 1e-5);
    const LaunchCtx c = ctx(h);
    SparseView<T> v = view<T>(h);
    if (nlock > 0) {  // S + mu sum_l v_l v_l^T: the eigenpairs already found are moved out of the way
        v.lr_k = h->lr_k + nlock;
        v.lr_u = h->defl_u;
        v.lr_s = h->defl_s;
    }
    const int64_t n = h->n;
    T *Q = static_cast<T *>(h->Q);
    T *w = static_cast<T *>(h->lzw);
    double *h1 = &h->st->h1[0];
    double *h2 = &h->st->h2[0];
    const int kk = int(std::min<int64_t>(k, n));
    if (warm) {  // Q[:, 0] holds the previous Ritz vector: perturb it by a seeded vector of norm 0.05
        launch_lz_start<T>(c, w, n, seed);
        launch_lz_mix<T>(c, Q, w, n);
    } else {
        launch_lz_start<T>(c, Q, n, seed);
    }
    launch_lz_normalize<T>(c, v, Q, Q, n, 0, 0);
    // one restart cycle: kk steps (SpMV, CGS2 in three passes, normalisation), the tridiagonal
    // eigensolve and the Ritz vector; captured once as a CUDA graph (its launches are many
    // and, at small n, short)
    auto cycle_launches = [&]() {
        launch_lz_reset(c);
        for (int j = 0; j < kk; ++j) {
            launch_lz_spmv_reorth<T>(c, v, Q + int64_t(j) * n, Q, n, j + 1, w, h1, j);
            launch_lz_reorth<T>(c, Q, n, j + 1, w, n, h1, h2, j, 1);
            launch_lz_reorth<T>(c, Q, n, j + 1, w, n, h2, nullptr, j, 2);
            launch_lz_normalize<T>(c, v, w, Q + int64_t(j + 1) * n, n, 1, j);
        }
        launch_lz_tridiag(c, kk);
        launch_lz_ritz<T>(c, Q, n, kk, w, n);
        launch_lz_normalize<T>(c, v, w, Q, n, 0, 0);
    };
    const bool graphs = h->opt.use_graph && h->stream != nullptr;
    if (graphs && (!h->lz_graph || h->lz_graph_k != kk || h->lz_graph_Q != h->Q || h->lz_graph_lr != nlock)) {
        if (h->lz_graph) {
            cudaGraphExecDestroy(h->lz_graph);
            h->lz_graph = nullptr;
        }
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = h->launches;
        cycle_launches();
        h->lz_graph_launches = h->launches - l0;
        h->launches = l0;
        CK(cudaStreamEndCapture(h->stream, &g));
        CK(cudaGraphInstantiate(&h->lz_graph, g, 0));
        cudaGraphDestroy(g);
        h->lz_graph_k = kk;
        h->lz_graph_Q = h->Q;
        h->lz_graph_lr = nlock;
    }
    double theta = 0.0, resid = INFINITY;
    for (int cycle = 0; cycle < max_restarts; ++cycle) {
        if (graphs) {
            CK(cudaGraphLaunch(h->lz_graph, h->stream));
            h->launches += h->lz_graph_launches;
        } else {
            cycle_launches();
        }
        CK(cudaGetLastError());
        TRY(sync_state(h));
        const DevState &s = *h->h_st;
        *matvecs += s.lz_m;
        theta = s.theta;
        resid = s.resid_est;
        if (!std::isfinite(theta)) FAIL(ALM_ERR_NUMERIC, "non-finite Ritz value in Lanczos");
        if (resid <= std::max(tol_rel * s.anorm, tol_abs) || s.lz_stop) break;
    }
    // true residual of the final pair
    launch_lz_reset(c);
    launch_lz_spmv<T>(c, v, Q, w);
    launch_lz_resid<T>(c, w, Q, n);
    CK(cudaGetLastError());
    TRY(sync_state(h));
    *matvecs += 1;
    *theta_out = theta;
    *resid_out = std::sqrt(std::max(h->h_st->red[1], 0.0));
    return ALM_OK;
}

// buffers of the rank growth along several eigenvectors (allocated on first use)
static alm_status ensure_growth(alm_handle *h) {
    if (h->grow_V) return ALM_OK;
    const size_t n = size_t(h->n);
    CK(cudaMalloc(&h->defl_u, sizeof(double) * n * kMaxLR));
    CK(cudaMalloc(&h->defl_s, sizeof(double) * kMaxLR));
    if (h->lr_k > 0) {  // C's own low-rank terms come first
        CK(cudaMemcpyAsync(h->defl_u, h->lr_u, sizeof(double) * n * size_t(h->lr_k), cudaMemcpyDeviceToDevice,
                           h->stream));
        CK(cudaMemcpyAsync(h->defl_s, h->lr_s, sizeof(double) * size_t(h->lr_k), cudaMemcpyDeviceToDevice,
                           h->stream));
    }
    CK(cudaMalloc(&h->grow_V, h->esz * n * 4));
    CK(cudaMalloc(&h->grow_mom, sizeof(double) * 35));
    CK(cudaMalloc(&h->grow_lam, sizeof(double) * 4));
    CK(cudaMalloc(&h->grow_sqrt, sizeof(double) * 16));
    CK(cudaMalloc(&h->grow_dec, sizeof(double)));
    CK(cudaMalloc(&h->grow_info, sizeof(int) * 2));
    return ALM_OK;
}

// Alg. 1's growth along several eigenvectors of Z(w) = grad_X L (diagonal-selector
// problems): the eigenpair in Q[:, 0] (eigenvalue lam1) and up to kmax - 1 more found by
// Lanczos on S + mu sum_l v_l v_l^T (the found ones deflated), those below -tau_lam kept;
// then the k x k SDP for S on the device and R <- [R, V S^{1/2}].  *added = the number of
// columns appended (0: fewer than two directions qualified; Q[:, 0] then holds v_1 again
// and the caller takes the one-direction step).
template <typename T>
static alm_status grow_block(alm_handle *h, double lam1, double sigma, double tau_lam, double tol_abs, int kmax,
                             uint64_t seed, T **Rp, int *r, int *ldr, int *cur, alm_stats *S, int *added) {
    *added = 0;
    kmax = std::min(kmax, std::min(4, kMaxLR - h->lr_k + 1));
    if (kmax < 2 || !h->fused_dual) return ALM_OK;
    TRY(ensure_growth(h));
    const alm_options &o = h->opt;
    const LaunchCtx c = ctx(h);
    const SparseView<T> v = view<T>(h);
    const int64_t n = h->n;
    const size_t col = h->esz * size_t(n);
    T *V = static_cast<T *>(h->grow_V);
    CK(cudaMemcpyAsync(V, h->Q, col, cudaMemcpyDeviceToDevice, h->stream));
    std::vector<double> lams{lam1};
    const double mu = 2.0 * (std::fabs(h->h_st->anorm) + std::fabs(lam1));
    for (int j = 1; j < kmax; ++j) {
        launch_to_double<T>(c, V + int64_t(j - 1) * n, n, h->defl_u + size_t(h->lr_k + j - 1) * size_t(n));
        CK(cudaMemcpyAsync(h->defl_s + h->lr_k + j - 1, &mu, sizeof(double), cudaMemcpyHostToDevice, h->stream));
        double th = 0.0, res = 0.0;
        int64_t mv = 0;
        TRY(lanczos<T>(h, o.lanczos_k, o.lanczos_max_restarts, o.lanczos_tol, tol_abs, seed + uint64_t(j), &th, &res,
                       &mv, false, j));
        S->lanczos_matvecs += mv;
        if (!(th < -tau_lam)) break;
        CK(cudaMemcpyAsync(V + int64_t(j) * n, h->Q, col, cudaMemcpyDeviceToDevice, h->stream));
        lams.push_back(th);
    }
    CK(cudaMemcpyAsync(h->Q, V, col, cudaMemcpyDeviceToDevice, h->stream));  // v_1 back in Q[:, 0]
    const int k = int(lams.size());
    if (k < 2) {
        CK(cudaStreamSynchronize(h->stream));
        return ALM_OK;
    }
    CK(cudaMemcpyAsync(h->grow_lam, lams.data(), sizeof(double) * size_t(k), cudaMemcpyHostToDevice, h->stream));
    launch_grow_moments<T>(c, v, V, k, h->grow_mom);
    launch_grow_sdp(c, h->grow_mom, h->grow_lam, k, sigma, h->grow_sqrt, h->grow_info, h->grow_dec);
    int info[2] = {0, 0};
    CK(cudaMemcpyAsync(info, h->grow_info, sizeof(info), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (info[0] == 1) FAIL(ALM_ERR_UNBOUNDED, "L_sigma unbounded below along the eigenvectors (A(V S V^T) can vanish)");
    const int ldr2 = pad_rank(h, *r + k);
    T *dst = static_cast<T *>(h->Rb[1 - *cur]);
    launch_relayout<T>(c, *Rp, *ldr, dst, ldr2, *r, n, nullptr, 0.0);
    launch_grow_append<T>(c, V, n, k, h->grow_sqrt, dst, ldr2, *r);
    *cur = 1 - *cur;
    *r += k;
    *ldr = ldr2;
    *Rp = dst;
    *added = k;
    return ALM_OK;
}

template <typename T>
static alm_status lambda_prim(alm_handle *h, const void *R, int r, int ldr, const double *y, double sigma,
                              double *lambda_out, void *v_out, double *resid_out) {
    TRY(eval_and_dual<T>(h, R, r, ldr, y, sigma, h->AX));
    double theta = 0.0, resid = 0.0;
    int64_t mv = 0;
    TRY(lanczos<T>(h, h->opt.lanczos_k, h->opt.lanczos_max_restarts, h->opt.lanczos_tol, 0.0, h->opt.seed, &theta,
                   &resid, &mv));
    if (v_out) CK(cudaMemcpyAsync(v_out, h->Q, h->esz * size_t(h->n), cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *lambda_out = theta;
    if (resid_out) *resid_out = resid;
    return ALM_OK;
}

extern "C" alm_status alm_lambda_min(alm_handle *h, const void *R, int32_t r, int32_t ldr, const double *y,
                                     double sigma, double *lambda_out, void *v_out, double *resid_out) {
    if (!h || !lambda_out) return ALM_ERR_INVALID_ARG;
    if (R) TRY(check_factor(h, R, r, ldr));
    else if (r != 0) FAIL(ALM_ERR_INVALID_ARG, "r must be 0 when R is NULL");
    if (!std::isfinite(sigma) || sigma < 0) FAIL(ALM_ERR_INVALID_ARG, "sigma must be finite and >= 0");
    if (h->prec == ALM_FP64) return lambda_prim<double>(h, R, r, ldr, y, sigma, lambda_out, v_out, resid_out);
    return lambda_prim<float>(h, R, r, ldr, y, sigma, lambda_out, v_out, resid_out);
}

// ------------------------------------------------------------------------------------
// ALORA
// ------------------------------------------------------------------------------------
static alm_status ensure_solver(alm_handle *h) {
    const int rp = pad_rank(h, h->opt.r_max + 1 > kMaxRank ? kMaxRank : h->opt.r_max);
    if (h->Rb[0] && h->work_rmax >= rp) return ALM_OK;
    for (void **p : {&h->Rb[0], &h->Rb[1], &h->G, &h->D, &h->D2})
        if (*p) { cudaFree(*p); *p = nullptr; }
    const size_t bytes = h->esz * size_t(h->n) * size_t(rp);
    for (void **p : {&h->Rb[0], &h->Rb[1], &h->G, &h->D, &h->D2}) {
        CK(cudaMalloc(p, bytes));
        CK(cudaMemsetAsync(*p, 0, bytes, h->stream));
    }
    h->work_rmax = rp;
    return ALM_OK;
}

// ev: optional 6 timing events around the kernel classes of the chunk's first step
// (slack, SpMM, direction, line search, update); recorded as external event nodes when
// the chunk is being captured into a graph.
template <typename T>
static void enqueue_inner_chunk(alm_handle *h, T *R, T *Rpart, int r, int ldr, int chunk, cudaEvent_t *ev,
                                bool capturing) {
    const LaunchCtx c = ctx(h);
    const SparseView<T> v = view<T>(h);
    T *G = static_cast<T *>(h->G);
    T *D = static_cast<T *>(h->D);
    T *D2 = static_cast<T *>(h->D2);
    const int64_t cnt = h->n * int64_t(ldr);
    int *done = &h->st->done;
    auto mark = [&](int it, int k) {
        if (ev && it == 0) cudaEventRecordWithFlags(ev[k], h->stream, capturing ? cudaEventRecordExternal : 0);
    };
    // Direction fused into the line search: the new direction goes to the other buffer of
    // the pair (D, D2), so that neighbours' old directions stay readable.  Step it reads the
    // current direction from buffer it % 2 and writes the next one to (it + 1) % 2; a chunk
    // has an even number of steps, so every chunk starts with the direction in D.  (At the
    // start of an inner solve alpha = beta = 0, so the buffers' contents are not read.)
    const bool fuse_dir = h->fused_dual && ls_dir_fusable<T>(v) && chunk % 2 == 0 && D2 != nullptr;
    // The pending step and the slack diagonal fused into the SpMM as well: the factor then
    // alternates between R and Rpart like the direction (step it reads R from buffer it % 2
    // and writes the stepped factor to the other); the host counts the fused launches
    // (DevState::k1count) and moves the factor back to R at the end of the inner solve.
    const bool fuse_step = fuse_dir && Rpart != nullptr && spmm_step_fusable<T>(v);
    h->fused_step = fuse_step;
    for (int it = 0; it < chunk; ++it) {
        T *Dc = fuse_dir && (it % 2) ? D2 : D;
        T *Dn = fuse_dir ? ((it % 2) ? D : D2) : D;
        if (fuse_step) {
            T *Rin = (it % 2) ? Rpart : R;
            T *Rout = (it % 2) ? R : Rpart;
            mark(it, 0);
            mark(it, 1);
            launch_spmm_step<T>(c, v, Rin, Rout, r, ldr, G, Dc, done);
            mark(it, 2);
            mark(it, 3);
            launch_ls_dir<T>(c, v, Rout, G, Dc, Dn, r, ldr, done);
            mark(it, 4);
            mark(it, 5);  // the step that reaches the iteration cap is applied by the host (solve_impl)
            continue;
        }
        mark(it, 0);
        // slack diagonal only (y is fixed during the inner solve), after applying the step of
        // the previous line search
        if (h->fused_dual) launch_inner_slack<T>(c, v, R, Dc, r, ldr, done);
        else eval_dual<T>(h, c, v, R, r, ldr, h->y, h->AX, done);
        mark(it, 1);
        launch_spmm<T>(c, v, R, r, ldr, G, Dc, 1, done);
        mark(it, 2);
        if (fuse_dir) {
            mark(it, 3);
            launch_ls_dir<T>(c, v, R, G, Dc, Dn, r, ldr, done);
        } else {
            launch_dir<T>(c, G, D, cnt, done);
            mark(it, 3);
            launch_ls<T>(c, v, R, D, r, ldr, h->w, 1, done);
        }
        mark(it, 4);
        launch_axpy<T>(c, R, Dn, cnt, done, h->fused_dual ? 1 : 0);  // fused form: only the last step
        mark(it, 5);
    }
}

// the solve's per-outer-iteration log (alm_set_log): open for appending while a solve runs
struct SolveLog {
    FILE *f = nullptr;
    ~SolveLog() {
        if (f) std::fclose(f);
    }
};
static std::string jnum(double x) {
    if (!std::isfinite(x)) return "null";
    char b[40];
    std::snprintf(b, sizeof b, "%.17g", x);
    return b;
}

template <typename T>
static alm_status solve_impl(alm_handle *h, void *R_user, int ldr_user, int *r_inout, double *y_user, alm_stats *stats,
                             bool resume = false) {
    const auto t0 = std::chrono::steady_clock::now();
    const alm_options &o = h->opt;
    if (!y_user) FAIL(ALM_ERR_INVALID_ARG, "y is NULL");
    if (ldr_user < o.r_max) FAIL(ALM_ERR_INVALID_ARG, "ldr must be >= r_max");
    int r = resume ? h->ss.r : *r_inout;
    if (r < 1 || r > o.r_max) FAIL(ALM_ERR_INVALID_ARG, "initial rank must be in 1..r_max");
    TRY(check_factor(h, R_user, r, ldr_user));
    TRY(ensure_solver(h));
    TRY(ensure_lanczos(h, o.lanczos_k));
    const int64_t launches0 = h->launches;
    alm_stats S{};
    const LaunchCtx c = ctx(h);
    const SparseView<T> v = view<T>(h);
    int cur = 0;
    int ldr = pad_rank(h, r);
    double sigma = o.sigma0, tau_in = o.inner_start, kkt_prev = -1.0, p_prev = INFINITY;
    double lam = 0.0;
    bool lz_before = false;  // a Lanczos ran earlier in this solve (its Ritz vector is in Q[:, 0])
    int outer_first = 1;
    if (resume) {  // continue the saved trajectory: factor, y and Ritz vector are in the handle
        const auto &q = h->ss;
        cur = q.cur;
        ldr = q.ldr;
        sigma = q.sigma;
        tau_in = q.tau_in;
        kkt_prev = q.kkt_prev;
        p_prev = q.p_prev;
        lam = q.lam;
        lz_before = q.lz_before != 0;
        outer_first = q.outer_done + 1;
        S.inner_total = int32_t(q.inner_total);
        S.lanczos_matvecs = q.lanczos_matvecs;
        S.growth_steps = q.growth_steps;
    } else {
        launch_relayout<T>(c, static_cast<const T *>(R_user), ldr_user, static_cast<T *>(h->Rb[cur]), ldr, r, h->n,
                           nullptr, 0.0);
        CK(cudaMemcpyAsync(h->y, y_user, sizeof(double) * size_t(h->m), cudaMemcpyDeviceToDevice, h->stream));
    }
    const double tau_lam = o.eps * (1.0 + h->norm_C);
    alm_status result = ALM_ERR_NOT_CONVERGED;
    SolveLog log;
    if (!h->log_path.empty()) {
        log.f = std::fopen(h->log_path.c_str(), "a");
        if (!log.f) FAIL(ALM_ERR_INVALID_ARG, "cannot open the log file for appending: " + h->log_path);
    }
    NvtxRange solve_range("alm_solve");
    int outer = 0;
    for (outer = outer_first; outer <= o.max_outer; ++outer) {
        NvtxRange outer_range("alm_outer");
        const auto to0 = std::chrono::steady_clock::now();
        double lz_ms = 0.0;
        const double sigma_used = sigma;
        if (outer > 1) {
            double cap = o.inner_decay * tau_in;
            if (kkt_prev >= 0.0) cap = std::min(cap, o.inner_rel * kkt_prev);
            tau_in = std::max(o.inner_floor * o.eps, cap);
        }
        T *R = static_cast<T *>(h->Rb[cur]);
        T *Rpart = static_cast<T *>(h->Rb[1 - cur]);  // ping-pong partner of the fused inner step
        launch_set_state(c, sigma, tau_in * (1.0 + h->norm_C), o.max_inner, o.inner_method, o.inner_precond,
                         h->pc_floor);
        if (h->fused_dual)
            launch_prep_base<T>(c, v, h->y, static_cast<T *>(h->base_hi), static_cast<T *>(h->base_lo));
        // ---- inner solve: chunks of `chunk` steps, each step a fixed kernel sequence that
        //      turns into no-ops once the device sets `done` --------------------------------
        int iters = 0;
        cudaEvent_t *ev = o.profile ? h->prof_ev : nullptr;
        NvtxRange inner_range("alm_inner_solve");
        for (;;) {
            if (o.use_graph && h->stream != nullptr) {  // no capture on the legacy default stream
                if (!h->graph || h->graph_r != r || h->graph_ldr != ldr || h->graph_cur != cur) {
                    if (h->graph) {
                        cudaGraphExecDestroy(h->graph);
                        h->graph = nullptr;
                    }
                    cudaGraph_t g;
                    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
                    const int64_t l0 = h->launches;
                    enqueue_inner_chunk<T>(h, R, Rpart, r, ldr, o.chunk, ev, true);
                    h->graph_launches = h->launches - l0;
                    h->launches = l0;
                    CK(cudaStreamEndCapture(h->stream, &g));
                    CK(cudaGraphInstantiate(&h->graph, g, 0));
                    cudaGraphDestroy(g);
                    h->graph_r = r;
                    h->graph_ldr = ldr;
                    h->graph_cur = cur;
                }
                CK(cudaGraphLaunch(h->graph, h->stream));
                h->launches += h->graph_launches;
            } else {
                enqueue_inner_chunk<T>(h, R, Rpart, r, ldr, o.chunk, ev, false);
            }
            CK(cudaGetLastError());
            TRY(sync_state(h));
            if (ev) {
                float ms = 0.f, cls[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                bool ok = true;
                for (int k = 0; k < 5 && ok; ++k) ok = cudaEventElapsedTime(&cls[k], ev[k], ev[k + 1]) == cudaSuccess;
                ms = cls[1];
                if (!ok) {
                    (void)cudaGetLastError();  // clear it: a missing sample is not a failure
                } else {
                    for (int k = 0; k < 5; ++k) S.step_ms[k] += cls[k];
                    S.spmm_ms += ms;
                    S.spmm_launches += 1;
                    // pattern, diag(S), and the n x ldr blocks the kernel streams: R, Z_old, D_old
                    // read and Z written; the fused step kernel also writes the stepped R and reads
                    // the slack's per-row data (base and b pairs, selector) instead of diag(S)
                    const double blk = h->fused_step ? 5.0 : 4.0;
                    const double rowb = h->fused_step ? double(6 * h->esz + 8) : double(h->esz);
                    S.spmm_bytes += double(4 * (h->n + 1)) + double(h->nnz_f) * double(4 + h->esz) +
                                    double(h->n) * rowb + blk * double(h->n) * double(ldr) * double(h->esz);
                    S.spmm_rank_pad = ldr;
                    // line search (fused direction form): R, Z, D_old read, D_new written; the
                    // strict upper pattern (narrow ELL and its overflow list when present)
                    // and the per-row record
                    const double upat = h->ell_kn > 0
                                            ? double(h->n) * h->ell_kn * double(4 + h->esz) +
                                                  double(h->n_ov) * double(8 + h->esz)
                                            : double(4 * (h->n + 1)) + double(h->nnz_u) * double(4 + h->esz);
                    const double rec = h->esz == 4 ? 16.0 : 32.0;
                    S.ls_bytes += upat + double(h->n) * rec + 4.0 * double(h->n) * double(ldr) * double(h->esz);
                }
            }
            iters = h->h_st->iters;
            if (h->h_st->done) break;
        }
        inner_range.end();
        const double inner_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - to0).count();
        S.inner_total += iters;
        if (h->fused_step && h->h_st->done == 2) {
            // the inner solve stopped at the iteration cap: the fused loop leaves the last step
            // R_out += alpha D_new to the next step kernel, which did not run, so apply it here.
            // Step k of the solve wrote R_out = (k odd ? R : Rpart), D_new = (k odd ? D : D2)
            // (chunks have an even number of steps); the last one is k = k1count - 1.
            const int last = h->h_st->k1count - 1;
            T *Dn = static_cast<T *>((last % 2) ? h->D : h->D2);
            launch_axpy<T>(c, (last % 2) ? R : Rpart, Dn, h->n * int64_t(ldr), &h->st->done, 1);
        }
        if (h->h_st->k1count % 2 == 1)  // the factor ended in the partner buffer: move it back
            CK(cudaMemcpyAsync(R, Rpart, h->esz * size_t(h->n) * size_t(ldr), cudaMemcpyDeviceToDevice, h->stream));
        if (h->h_st->status == ALM_ERR_NUMERIC) FAIL(ALM_ERR_NUMERIC, "non-finite value in the inner solve");
        if (h->h_st->status == ALM_ERR_UNBOUNDED) FAIL(ALM_ERR_UNBOUNDED, "L_sigma unbounded below along a CG direction");
        // ---- spectral information of grad_X L at X = RR^T ------------------------------
        eval_dual<T>(h, c, v, R, r, ldr, h->y, h->AX, h->zero_flag);
        // lambda_min serves the rank growth (only while r < r_max) and the dual KKT term
        // (which decides only once the primal and gap terms are <= eps): skip it otherwise
        TRY(sync_state(h));
        bool have_lam = r < o.r_max;
        if (!have_lam) {
            const DevState &s0 = *h->h_st;
            const double p0 = std::sqrt(std::max(s0.res2, 0.0)) / (1.0 + h->norm_b);
            const double g0 = std::fabs(s0.c0 - s0.bw) / (1.0 + std::fabs(s0.c0) + std::fabs(s0.bw));
            have_lam = p0 <= o.eps && g0 <= o.eps;
        }
        if (have_lam) {
            double resid = 0.0;
            int64_t mv = 0;
            const double tol_abs = 0.1 * o.eps * (1.0 + h->norm_C);
            const auto tl0 = std::chrono::steady_clock::now();
            NvtxRange lz_range("alm_lanczos");
            TRY(lanczos<T>(h, o.lanczos_k, o.lanczos_max_restarts, o.lanczos_tol, tol_abs,
                           o.seed + uint64_t(outer) * 0x100000001ULL, &lam, &resid, &mv, o.lanczos_warm && lz_before));
            lz_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tl0).count();
            S.lanczos_ms += lz_ms;
            S.lanczos_matvecs += mv;
            lz_before = true;
        }
        bool grew = false;
        int added = 0;
        if (have_lam && lam < -tau_lam && r < o.r_max && o.growth_k > 1) {
            TRY(grow_block<T>(h, lam, sigma, tau_lam, 0.1 * o.eps * (1.0 + h->norm_C),
                              std::min(o.growth_k, o.r_max - r), o.seed + uint64_t(outer) * 0x100000001ULL + 7,
                              &R, &r, &ldr, &cur, &S, &added));
            if (added > 0) {
                CK(cudaMemsetAsync(h->G, 0, h->esz * size_t(h->n) * size_t(h->work_rmax), h->stream));
                CK(cudaMemsetAsync(h->D, 0, h->esz * size_t(h->n) * size_t(h->work_rmax), h->stream));
                CK(cudaMemsetAsync(h->D2, 0, h->esz * size_t(h->n) * size_t(h->work_rmax), h->stream));
                eval_dual<T>(h, c, v, R, r, ldr, h->y, h->AX, h->zero_flag);
                grew = true;
                S.growth_steps += 1;
            }
        }
        if (!grew && have_lam && lam < -tau_lam && r < o.r_max) {
            // ||A(v v^T)||^2 with v = Q[:, 0]: evaluate the constraint map on the n x W factor [v 0]
            const int W = vec_width(h);
            T *tmp = static_cast<T *>(h->D);
            launch_relayout<T>(c, static_cast<const T *>(h->Q), 1, tmp, W, 1, h->n, nullptr, 0.0);
            launch_eval<T>(c, v, tmp, 1, W, h->AXtmp, h->zero_flag);
            launch_sumsq<T>(c, h->AXtmp, h->m);
            CK(cudaGetLastError());
            TRY(sync_state(h));
            const double av2 = h->h_st->red[0];
            if (!(av2 > 0.0)) FAIL(ALM_ERR_UNBOUNDED, "L_sigma unbounded below along the eigenvector (A(vv^T) = 0)");
            const double s = -lam / (sigma * av2);
            const int ldr2 = pad_rank(h, r + 1);
            launch_relayout<T>(c, R, ldr, static_cast<T *>(h->Rb[1 - cur]), ldr2, r, h->n,
                               static_cast<const T *>(h->Q), std::sqrt(s));
            cur = 1 - cur;
            r += 1;
            ldr = ldr2;
            R = static_cast<T *>(h->Rb[cur]);
            // the CG buffers change layout with the rank: clear them
            CK(cudaMemsetAsync(h->G, 0, h->esz * size_t(h->n) * size_t(h->work_rmax), h->stream));
            CK(cudaMemsetAsync(h->D, 0, h->esz * size_t(h->n) * size_t(h->work_rmax), h->stream));
            CK(cudaMemsetAsync(h->D2, 0, h->esz * size_t(h->n) * size_t(h->work_rmax), h->stream));
            eval_dual<T>(h, c, v, R, r, ldr, h->y, h->AX, h->zero_flag);
            grew = true;
            S.growth_steps += 1;
        }
        // ---- dual update (Eq. ALM): y <- w ----------------------------------------------
        CK(cudaMemcpyAsync(h->y, h->w, sizeof(double) * size_t(h->m), cudaMemcpyDeviceToDevice, h->stream));
        TRY(sync_state(h));
        if (o.verbose)
            std::fprintf(stderr, "[alm] outer %4d inner %6d (total %8d) r %2d sigma %.3g lambda %+.4e%s t %.1f ms\n",
                         outer, iters, S.inner_total, r, sigma, lam, grew ? " grew" : "",
                         std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
        const DevState &s = *h->h_st;
        const double p = std::sqrt(std::max(s.res2, 0.0)) / (1.0 + h->norm_b);
        const double d = have_lam ? std::fabs(std::min(0.0, lam)) / (1.0 + h->norm_C) : 0.0;
        const double g = std::fabs(s.c0 - s.bw) / (1.0 + std::fabs(s.c0) + std::fabs(s.bw));
        if (log.f) {
            const double now_ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            std::fprintf(log.f,
                         "{\"outer\": %d, \"inner\": %d, \"inner_total\": %d, \"rank\": %d, \"sigma\": %s, "
                         "\"lambda_min\": %s, \"grew\": %s, \"kkt\": [%s, %s, %s], \"objective\": %s, "
                         "\"alpha_last\": %s, \"time_ms\": {\"inner\": %s, \"lanczos\": %s, \"total\": %s}}\n",
                         outer, iters, S.inner_total, r, jnum(sigma_used).c_str(),
                         have_lam ? jnum(lam).c_str() : "null", grew ? "true" : "false", jnum(p).c_str(),
                         jnum(d).c_str(), jnum(g).c_str(), jnum(s.c0).c_str(), jnum(s.alpha).c_str(),
                         jnum(inner_ms).c_str(), jnum(lz_ms).c_str(), jnum(now_ms).c_str());
            std::fflush(log.f);
        }
        if (grew) continue;
        S.kkt[0] = p;
        S.kkt[1] = d;
        S.kkt[2] = g;
        S.objective = s.c0;
        if (o.sigma_rule == ALM_SIGMA_ADAPTIVE && kkt_prev >= 0.0 && p > 0.25 * p_prev)
            sigma = std::min(2.0 * sigma, o.sigma_max);
        p_prev = p;
        kkt_prev = std::max(p, std::max(d, g));
        if (o.verbose) std::fprintf(stderr, "[alm]   kkt p %.3e d %.3e g %.3e\n", p, d, g);
        if (have_lam && kkt_prev <= o.eps) {
            result = ALM_OK;
            break;
        }
    }
    // ---- the state a checkpoint saves ------------------------------------------------------
    {
        auto &q = h->ss;
        q.valid = 1;
        q.r = r;
        q.ldr = ldr;
        q.cur = cur;
        q.outer_done = std::min(outer, o.max_outer);
        q.lz_before = lz_before ? 1 : 0;
        q.growth_steps = S.growth_steps;
        q.sigma = sigma;
        q.tau_in = tau_in;
        q.kkt_prev = kkt_prev;
        q.p_prev = p_prev;
        q.lam = lam;
        q.inner_total = S.inner_total;
        q.lanczos_matvecs = S.lanczos_matvecs;
    }
    // ---- outputs ------------------------------------------------------------------------
    launch_eval<T>(c, v, static_cast<T *>(h->Rb[cur]), r, ldr, h->AX, h->zero_flag);
    launch_relayout<T>(c, static_cast<const T *>(h->Rb[cur]), ldr, static_cast<T *>(R_user), ldr_user, r, h->n,
                       nullptr, 0.0);
    CK(cudaMemcpyAsync(y_user, h->y, sizeof(double) * size_t(h->m), cudaMemcpyDeviceToDevice, h->stream));
    TRY(sync_state(h));
    S.objective = h->h_st->c0;
    S.status = result;
    S.outer = std::min(outer, o.max_outer);
    S.rank = r;
    S.sigma = sigma;
    S.lambda_min = lam;
    S.kernel_launches = h->launches - launches0;
    S.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *r_inout = r;
    if (stats) *stats = S;
    if (result != ALM_OK) h->err = "outer iteration cap reached before KKT <= eps";
    return result;
}

extern "C" alm_status alm_solve(alm_handle *h, void *R, int32_t ldr, int32_t *r_inout, double *y, alm_stats *stats) {
    if (!h || !r_inout) return ALM_ERR_INVALID_ARG;
    h->ss.valid = 0;
    if (h->prec == ALM_FP64) return solve_impl<double>(h, R, ldr, r_inout, y, stats);
    return solve_impl<float>(h, R, ldr, r_inout, y, stats);
}

// ------------------------------------------------------------------------------------
// one inner CG step of the fused loop from a caller-given state
// ------------------------------------------------------------------------------------
namespace alm {
__global__ void k_cg_state(DevState *st, double alpha, double zg_prev) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->alpha = alpha;
        st->zg_prev = zg_prev;
        st->restart = zg_prev > 0.0 ? 0 : 1;
    }
}
template <typename T>
__global__ void k_diag_out(const T *__restrict__ hi, const T *__restrict__ lo, int64_t n, double *__restrict__ out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = double(hi[i]) + (lo ? double(lo[i]) : 0.0);
}
}  // namespace alm

template <typename T>
static alm_status cg_step_impl(alm_handle *h, const void *R, const void *D, int r, int ldr, const double *y,
                               double sigma, double alpha, double zg_prev, void *R_out, void *Z, void *D_new,
                               double *diag_out, double *out) {
    const void *bufs[5] = {R, D, R_out, Z, D_new};
    for (const void *p : bufs) TRY(check_factor(h, p, r, ldr));
    if (!y) FAIL(ALM_ERR_INVALID_ARG, "y is NULL");
    if (R_out == R || D_new == D || Z == R || Z == D || R_out == Z || D_new == Z)
        FAIL(ALM_ERR_INVALID_ARG, "R_out, Z and D_new must be buffers of their own");
    if (!std::isfinite(sigma) || sigma < 0 || !std::isfinite(alpha) || !std::isfinite(zg_prev))
        FAIL(ALM_ERR_INVALID_ARG, "sigma, alpha and zg_prev must be finite (sigma >= 0)");
    TRY(ensure_solver(h));
    const LaunchCtx c = ctx(h);
    const SparseView<T> v = view<T>(h);
    if (!(h->fused_dual && ls_dir_fusable<T>(v)))
        FAIL(ALM_ERR_INVALID_ARG, "the fused inner step needs constraints X_ii = b_i and rows of at most 16 entries");
    h->ss.valid = 0;
    const alm_options &o = h->opt;
    int *done = &h->st->done;
    CK(cudaMemcpyAsync(h->y, y, sizeof(double) * size_t(h->m), cudaMemcpyDeviceToDevice, h->stream));
    launch_set_state(c, sigma, 0.0, 1 << 30, o.inner_method, o.inner_precond, h->pc_floor);
    k_cg_state<<<1, 32, 0, h->stream>>>(h->st, alpha, zg_prev);
    launch_prep_base<T>(c, v, h->y, static_cast<T *>(h->base_hi), static_cast<T *>(h->base_lo));
    T *Ro = static_cast<T *>(R_out);
    T *Zb = static_cast<T *>(Z);
    if (spmm_step_fusable<T>(v)) {
        launch_spmm_step<T>(c, v, static_cast<const T *>(R), Ro, r, ldr, Zb, static_cast<const T *>(D), done);
    } else {
        CK(cudaMemcpyAsync(Ro, R, h->esz * size_t(h->n) * size_t(ldr), cudaMemcpyDeviceToDevice, h->stream));
        launch_inner_slack<T>(c, v, Ro, static_cast<const T *>(D), r, ldr, done);
        launch_spmm<T>(c, v, Ro, r, ldr, Zb, static_cast<const T *>(D), 1, done);
    }
    launch_ls_dir<T>(c, v, Ro, Zb, static_cast<const T *>(D), static_cast<T *>(D_new), r, ldr, done);
    if (diag_out)
        k_diag_out<T><<<std::max<int64_t>(1, std::min<int64_t>(h->grid, (h->n + 255) / 256)), 256, 0, h->stream>>>(
            static_cast<const T *>(h->d_s), static_cast<const T *>(h->d_s_lo), h->n, diag_out);
    CK(cudaGetLastError());
    TRY(sync_state(h));
    const DevState &s = *h->h_st;
    if (s.status == ALM_ERR_NUMERIC) FAIL(ALM_ERR_NUMERIC, "non-finite value in the inner step");
    const double vals[11] = {s.gg, s.g_gprev, s.g_dprev, s.zg, s.beta, s.q[0], s.q[1], s.q[2], s.q[3], s.q[4], s.alpha};
    for (int k = 0; k < 11; ++k) out[k] = vals[k];
    return ALM_OK;
}

extern "C" alm_status alm_cg_step(alm_handle *h, const void *R, const void *D, int32_t r, int32_t ldr,
                                  const double *y, double sigma, double alpha, double zg_prev, void *R_out, void *Z,
                                  void *D_new, double *diag_out, double *out) {
    if (!h || !out) return ALM_ERR_INVALID_ARG;
    if (h->prec == ALM_FP64)
        return cg_step_impl<double>(h, R, D, r, ldr, y, sigma, alpha, zg_prev, R_out, Z, D_new, diag_out, out);
    return cg_step_impl<float>(h, R, D, r, ldr, y, sigma, alpha, zg_prev, R_out, Z, D_new, diag_out, out);
}

// ------------------------------------------------------------------------------------
// launch shape of the inner-step kernels, and its autotuner
// ------------------------------------------------------------------------------------
static bool shape_valid(const alm_inner_shape &s) {
    if (s.variant == 0) return true;
    return s.variant == 1 && s.stages >= 2 && s.stages <= 4 && (s.threads == 128 || s.threads == 256);
}

static void drop_graph(alm_handle *h) {
    if (h->graph) {
        cudaStreamSynchronize(h->stream);
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
}

static void set_shape(alm_handle *h, const alm_inner_shape &s) {
    h->icfg.variant = s.variant;
    if (s.variant == 1) {
        h->icfg.stages = s.stages;
        h->icfg.threads = s.threads;
    }
    drop_graph(h);  // the captured chunk holds the previous shape's kernels
}

extern "C" alm_status alm_set_inner_shape(alm_handle *h, const alm_inner_shape *shape) {
    if (!h || !shape) return ALM_ERR_INVALID_ARG;
    if (!shape_valid(*shape)) FAIL(ALM_ERR_INVALID_ARG, "inner shape: variant 0, or variant 1 with stages 2..4 and 128 or 256 threads");
    set_shape(h, *shape);
    return ALM_OK;
}

extern "C" alm_status alm_get_inner_shape(const alm_handle *h, alm_inner_shape *shape) {
    if (!h || !shape) return ALM_ERR_INVALID_ARG;
    shape->variant = h->icfg.variant;
    shape->stages = h->icfg.stages;
    shape->threads = h->icfg.threads;
    return ALM_OK;
}

// the candidates the autotuner times, in this order
static const alm_inner_shape kShapes[] = {{0, 0, 0},   {1, 2, 128}, {1, 2, 256}, {1, 3, 128},
                                          {1, 3, 256}, {1, 4, 128}};
constexpr int kNumShapes = int(sizeof(kShapes) / sizeof(kShapes[0]));

// Time `steps` inner CG steps of the fused ELL loop (from R, y at sigma0) in each shape.
template <typename T>
static alm_status autotune_impl(alm_handle *h, const void *R_user, int r, int ldr_user, const double *y_user,
                                int steps, double *times_ms, int32_t *count) {
    TRY(check_factor(h, R_user, r, ldr_user));
    if (!y_user) FAIL(ALM_ERR_INVALID_ARG, "y is NULL");
    TRY(ensure_solver(h));
    const alm_options &o = h->opt;
    const SparseView<T> v = view<T>(h);
    *count = 0;
    if (!(h->fused_dual && ls_dir_fusable<T>(v) && spmm_step_fusable<T>(v) && h->D2)) return ALM_OK;  // nothing to tune
    h->ss.valid = 0;  // the solver buffers are overwritten: no solve state to checkpoint any more
    const int ldr = pad_rank(h, r);
    const size_t bytes = h->esz * size_t(h->n) * size_t(ldr);
    const alm_inner_shape keep{h->icfg.variant, h->icfg.stages, h->icfg.threads};
    double best = INFINITY;
    alm_inner_shape best_s = keep;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    alm_status result = ALM_OK;
    for (int k = 0; k < kNumShapes && result == ALM_OK; ++k) {
        set_shape(h, kShapes[k]);
        const LaunchCtx c = ctx(h);
        float msb = INFINITY;
        for (int rep = 0; rep < 2; ++rep) {  // the first run also loads the kernels
            launch_relayout<T>(c, static_cast<const T *>(R_user), ldr_user, static_cast<T *>(h->Rb[0]), ldr, r, h->n,
                               nullptr, 0.0);
            cudaError_t e = cudaMemcpyAsync(h->y, y_user, sizeof(double) * size_t(h->m), cudaMemcpyDeviceToDevice,
                                            h->stream);
            for (void *b : {h->G, h->D, h->D2})
                if (e == cudaSuccess) e = cudaMemsetAsync(b, 0, bytes, h->stream);
            if (e != cudaSuccess) {
                h->err = std::string("autotune: ") + cudaGetErrorString(e);
                result = ALM_ERR_CUDA;
                break;
            }
            launch_set_state(c, o.sigma0, 0.0, steps + 1, o.inner_method, o.inner_precond, h->pc_floor);
            launch_prep_base<T>(c, v, h->y, static_cast<T *>(h->base_hi), static_cast<T *>(h->base_lo));
            cudaEventRecord(e0, h->stream);
            enqueue_inner_chunk<T>(h, static_cast<T *>(h->Rb[0]), static_cast<T *>(h->Rb[1]), r, ldr, steps, nullptr,
                                   false);
            cudaEventRecord(e1, h->stream);
            e = cudaStreamSynchronize(h->stream);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                h->err = std::string("autotune: ") + cudaGetErrorString(e);
                result = ALM_ERR_CUDA;
                break;
            }
            msb = std::min(msb, ms);
        }
        if (result != ALM_OK) break;
        if (times_ms) times_ms[k] = msb;
        if (msb < best) {
            best = msb;
            best_s = kShapes[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_shape(h, result == ALM_OK ? best_s : keep);
    if (result == ALM_OK) *count = kNumShapes;
    return result;
}

// The cache key of a tuned shape: the sizes that decide which kernels run and how long.
static std::string tune_key(const alm_handle *h, int r) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "n=%lld nnz=%lld r=%d prec=%d kf=%d kn=%d", static_cast<long long>(h->n),
                  static_cast<long long>(h->nnz_f), r, h->prec, h->ell_kf, h->ell_kn);
    return buf;
}

// Look `key` up in a JSON-lines cache file (one object per line, written by cache_store).
static bool cache_lookup(const char *path, const std::string &key, alm_inner_shape *s) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    const std::string want = "\"key\": \"" + key + "\"";
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        if (!std::strstr(line, want.c_str())) continue;
        const char *pv = std::strstr(line, "\"variant\": ");
        const char *ps = std::strstr(line, "\"stages\": ");
        const char *pt = std::strstr(line, "\"threads\": ");
        alm_inner_shape q{};
        if (pv && ps && pt && std::sscanf(pv + 11, "%d", &q.variant) == 1 && std::sscanf(ps + 10, "%d", &q.stages) == 1 &&
            std::sscanf(pt + 11, "%d", &q.threads) == 1 && shape_valid(q)) {
            *s = q;  // the last matching line wins
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

static void cache_store(const char *path, const std::string &key, const alm_inner_shape &s, double ms) {
    FILE *f = std::fopen(path, "a");
    if (!f) return;  // an unwritable cache only costs the next call a retune
    std::fprintf(f, "{\"key\": \"%s\", \"variant\": %d, \"stages\": %d, \"threads\": %d, \"ms\": %.4f}\n",
                 key.c_str(), s.variant, s.stages, s.threads, ms);
    std::fclose(f);
}

extern "C" alm_status alm_autotune(alm_handle *h, const void *R, int32_t r, int32_t ldr, const double *y,
                                   int32_t steps, const char *cache_path, alm_inner_shape *best, double *times_ms,
                                   int32_t *count, int32_t *from_cache) {
    if (!h || !count) return ALM_ERR_INVALID_ARG;
    if (steps < 2 || steps > 256 || steps % 2) FAIL(ALM_ERR_INVALID_ARG, "steps must be even and in 2..256");
    if (from_cache) *from_cache = 0;
    *count = 0;
    const std::string key = tune_key(h, r);
    alm_inner_shape cached{};
    if (cache_path && cache_lookup(cache_path, key, &cached)) {
        set_shape(h, cached);
        if (best) *best = cached;
        if (from_cache) *from_cache = 1;
        return ALM_OK;
    }
    const alm_status st = h->prec == ALM_FP64 ? autotune_impl<double>(h, R, r, ldr, y, steps, times_ms, count)
                                              : autotune_impl<float>(h, R, r, ldr, y, steps, times_ms, count);
    if (st != ALM_OK) return st;
    alm_inner_shape b{};
    alm_get_inner_shape(h, &b);
    if (best) *best = b;
    if (cache_path && *count > 0 && times_ms) {
        double ms = INFINITY;
        for (int k = 0; k < *count; ++k) ms = std::min(ms, times_ms[k]);
        cache_store(cache_path, key, b, ms);
    } else if (cache_path && *count > 0) {
        cache_store(cache_path, key, b, 0.0);
    }
    return ALM_OK;
}

extern "C" int32_t alm_inner_shapes(alm_inner_shape *out) {
    if (out)
        for (int k = 0; k < kNumShapes; ++k) out[k] = kShapes[k];
    return kNumShapes;
}

// ------------------------------------------------------------------------------------
// checkpoint / resume of the ALORA state at the end of a solve
// ------------------------------------------------------------------------------------
namespace {
constexpr char kCkptMagic[8] = {'A', 'L', 'M', 'C', 'K', 'P', 'T', '2'};
struct CkptHeader {
    char magic[8];
    int64_t n, m;
    int32_t precision, esz;
    uint64_t problem_hash;  // fingerprint of C, the A_k and b: resume only on the same problem
};
}  // namespace

extern "C" alm_status alm_set_log(alm_handle *h, const char *path) {
    if (!h) return ALM_ERR_INVALID_ARG;
    if (!path || !*path) {
        h->log_path.clear();
        return ALM_OK;
    }
    FILE *f = std::fopen(path, "a");
    if (!f) FAIL(ALM_ERR_INVALID_ARG, std::string("cannot open the log file for appending: ") + path);
    std::fclose(f);
    h->log_path = path;
    return ALM_OK;
}

extern "C" alm_status alm_checkpoint(alm_handle *h, const char *path) {
    if (!h || !path) return ALM_ERR_INVALID_ARG;
    if (!h->ss.valid) FAIL(ALM_ERR_INVALID_ARG, "no solve state to save: run alm_solve or alm_resume first");
    const auto &q = h->ss;
    const size_t nr = size_t(h->n) * size_t(q.ldr);
    std::vector<char> R(h->esz * nr), Q(h->esz * size_t(h->n));
    std::vector<double> y(size_t(h->m));
    CK(cudaMemcpyAsync(R.data(), h->Rb[q.cur], R.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(y.data(), h->y, sizeof(double) * y.size(), cudaMemcpyDeviceToHost, h->stream));
    if (q.lz_before) CK(cudaMemcpyAsync(Q.data(), h->Q, Q.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    FILE *f = std::fopen(path, "wb");
    if (!f) FAIL(ALM_ERR_INVALID_ARG, std::string("cannot open ") + path + " for writing");
    CkptHeader hd{};
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.n = h->n;
    hd.m = h->m;
    hd.precision = h->prec;
    hd.esz = int32_t(h->esz);
    hd.problem_hash = h->problem_hash;
    bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 && std::fwrite(&q, sizeof(q), 1, f) == 1 &&
              std::fwrite(R.data(), 1, R.size(), f) == R.size() &&
              std::fwrite(y.data(), sizeof(double), y.size(), f) == y.size() &&
              (!q.lz_before || std::fwrite(Q.data(), 1, Q.size(), f) == Q.size());
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) FAIL(ALM_ERR_INVALID_ARG, std::string("write to ") + path + " failed");
    return ALM_OK;
}

template <typename T>
static alm_status resume_impl(alm_handle *h, const char *path, void *R_user, int32_t ldr_user, int32_t *r_inout,
                              double *y_user, alm_stats *stats) {
    FILE *f = std::fopen(path, "rb");
    if (!f) FAIL(ALM_ERR_INVALID_ARG, std::string("cannot open ") + path);
    CkptHeader hd{};
    alm_handle::SolveState q;
    bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, kCkptMagic, 8) == 0 &&
              std::fread(&q, sizeof(q), 1, f) == 1;
    if (ok && (hd.n != h->n || hd.m != h->m || hd.precision != h->prec || hd.esz != int32_t(h->esz))) {
        std::fclose(f);
        FAIL(ALM_ERR_INVALID_ARG, "checkpoint is for another problem size or precision");
    }
    if (ok && hd.problem_hash != h->problem_hash) {
        std::fclose(f);
        FAIL(ALM_ERR_INVALID_ARG, "checkpoint was saved for another problem (C, A or b differ)");
    }
    ok = ok && q.valid && q.r >= 1 && q.r <= h->opt.r_max && q.ldr >= q.r && (q.cur == 0 || q.cur == 1);
    if (!ok) {
        std::fclose(f);
        FAIL(ALM_ERR_INVALID_ARG, std::string("malformed checkpoint ") + path);
    }
    const alm_status es = ensure_solver(h);
    const alm_status el = es == ALM_OK ? ensure_lanczos(h, h->opt.lanczos_k) : es;
    if (el != ALM_OK || q.ldr > h->work_rmax) {
        std::fclose(f);
        if (el != ALM_OK) return el;
        FAIL(ALM_ERR_INVALID_ARG, "checkpoint row stride exceeds this handle's r_max");
    }
    const size_t nr = size_t(h->n) * size_t(q.ldr);
    std::vector<char> R(h->esz * nr), Q(h->esz * size_t(h->n));
    std::vector<double> y(size_t(h->m));
    ok = std::fread(R.data(), 1, R.size(), f) == R.size() && std::fread(y.data(), sizeof(double), y.size(), f) == y.size() &&
         (!q.lz_before || std::fread(Q.data(), 1, Q.size(), f) == Q.size());
    std::fclose(f);
    if (!ok) FAIL(ALM_ERR_INVALID_ARG, std::string("truncated checkpoint ") + path);
    CK(cudaMemcpyAsync(h->Rb[q.cur], R.data(), R.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->y, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, h->stream));
    if (q.lz_before) CK(cudaMemcpyAsync(h->Q, Q.data(), Q.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->ss = q;
    return solve_impl<T>(h, R_user, ldr_user, r_inout, y_user, stats, true);
}

extern "C" alm_status alm_resume(alm_handle *h, const char *path, void *R, int32_t ldr, int32_t *r_out, double *y,
                                 alm_stats *stats) {
    if (!h || !path || !r_out) return ALM_ERR_INVALID_ARG;
    if (h->prec == ALM_FP64) return resume_impl<double>(h, path, R, ldr, r_out, y, stats);
    return resume_impl<float>(h, path, R, ldr, r_out, y, stats);
}
