// C ABI of the warm-start network (include/alm.h, alm_gnn_*): parameter storage, the
// activation buffers sized for a batch, and the forward / loss-gradient / Adam sequences.
// Every arithmetic step runs in kernels_gnn.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "batch_internal.h"
#include "gnn_internal.h"

using namespace alm;

namespace {
thread_local std::string g_gnn_error;
}

struct alm_gnn {
    std::string err;
    cudaStream_t stream = nullptr;
    int storage = ALM_GNN_BF16;
    uint64_t feat_seed = 0;
    int sms = 0;
    int np = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    int step = 0;
    // buffers for the rows of the last batch seen
    int64_t cap_rows = 0;
    bool trainbufs = false;         // fbuf also holds the training buffers
    void *act = nullptr;            // H and AGG (storage type)
    float *fbuf = nullptr;          // rhat, yhat and the training buffers
    GnnActs<float> a32;
    GnnActs<__nv_bfloat16> a16;
    float *rhat = nullptr, *yhat = nullptr;
    double *loss = nullptr;
    double *lpart = nullptr;        // loss partials, one per CTA of the loss kernel (<= 8 per SM)
    int64_t launches = 0;
};

#define GCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            g->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return e_ == cudaErrorMemoryAllocation ? ALM_ERR_OOM : ALM_ERR_CUDA;          \
        }                                                                                 \
    } while (0)
#define GFAIL(code, msg)     \
    do {                     \
        g->err = (msg);      \
        return (code);       \
    } while (0)
#define GTRY(expr)                   \
    do {                             \
        alm_status s_ = (expr);      \
        if (s_ != ALM_OK) return s_; \
    } while (0)

namespace {

GnnGraph graph_of(const alm_batch *hb) {
    GnnGraph gr{};
    gr.rows = hb->rows;
    gr.row_inst = hb->row_inst;
    gr.row_off = hb->row_off;
    gr.rowptr = hb->rowptr;
    gr.col = hb->col;
    gr.val = hb->val;
    gr.scal = hb->gnn_scal;
    return gr;
}

template <typename T>
void carve(alm_gnn *g, GnnActs<T> &a, int64_t rows, bool training) {
    T *p = static_cast<T *>(g->act);
    a.H[0] = p;
    p += rows * kGnnFeat;
    for (int l = 1; l <= kGnnLayers; ++l) {
        a.H[l] = p;
        p += rows * kGnnHid;
    }
    a.AGG[0] = p;
    p += rows * kGnnFeat;
    for (int l = 1; l < kGnnLayers; ++l) {
        a.AGG[l] = p;
        p += rows * kGnnHid;
    }
    float *f = g->fbuf;
    g->rhat = f;
    f += rows * kGnnRank;
    g->yhat = f;
    f += rows;
    if (training) {
        a.dR = f;
        f += rows * kGnnRank;
        a.dY = f;
        f += rows;
        a.dH = f;
        f += rows * kGnnHid;
        a.dZ = f;
        f += rows * kGnnHid;
        a.dHp = f;
        f += rows * kGnnHid;
        a.U = f;
        f += rows * kGnnHid;
        a.part = f;
        a.lpart = g->lpart;
    }
    a.nblk = std::max(1, std::min(2 * g->sms, int((rows + 31) / 32)));
    a.ldp = kGnnLdp;
}

alm_status ensure_buffers(alm_gnn *g, int64_t rows, bool training) {
    if (!(g->act && g->cap_rows >= rows && (!training || g->trainbufs))) {
        const bool tr = training || g->trainbufs;
        const int64_t cap = std::max(rows, g->cap_rows);
        if (g->act) cudaFree(g->act);
        if (g->fbuf) cudaFree(g->fbuf);
        g->act = nullptr;
        g->fbuf = nullptr;
        g->cap_rows = 0;
        g->trainbufs = false;
        const size_t esz = g->storage == ALM_GNN_BF16 ? 2 : 4;
        const size_t acts = size_t(cap) * (2 * kGnnFeat + (2 * kGnnLayers - 1) * kGnnHid);
        size_t fl = size_t(cap) * (kGnnRank + 1);
        if (tr) {
            const int nblk = std::max(1, std::min(2 * g->sms, int((cap + 31) / 32)));
            fl += size_t(cap) * (kGnnRank + 1 + 4 * kGnnHid) + size_t(nblk) * size_t(kGnnLdp);
        }
        GCK(cudaMalloc(&g->act, esz * acts));
        GCK(cudaMalloc(&g->fbuf, sizeof(float) * fl));
        g->cap_rows = cap;
        g->trainbufs = tr;
    }
    g->a32 = GnnActs<float>();
    g->a16 = GnnActs<__nv_bfloat16>();
    if (g->storage == ALM_GNN_BF16) carve(g, g->a16, rows, g->trainbufs);
    else carve(g, g->a32, rows, g->trainbufs);
    if (!g->loss) GCK(cudaMalloc(&g->loss, sizeof(double)));
    return ALM_OK;
}

alm_status forward(alm_gnn *g, const alm_batch *hb) {
    const GnnGraph gr = graph_of(hb);
    const GnnParams p = gnn_views(g->theta);
    cudaError_t e;
    if (g->storage == ALM_GNN_BF16) e = gnn_forward(gr, p, g->feat_seed, g->a16, g->rhat, g->yhat, g->sms, g->stream);
    else e = gnn_forward(gr, p, g->feat_seed, g->a32, g->rhat, g->yhat, g->sms, g->stream);
    g->launches += 2 + kGnnLayers;
    GCK(e);
    return ALM_OK;
}

// loss and gradient into g->grad (device); the loss in g->loss (device)
alm_status loss_grad(alm_gnn *g, const alm_batch *hb, const float *Rs, const double *ys, double lam) {
    GTRY(forward(g, hb));
    const GnnGraph gr = graph_of(hb);
    const GnnParams p = gnn_views(g->theta);
    const GnnParams gp = gnn_views(g->grad);
    const double npat = double(hb->rows) + 0.5 * double(hb->nnz);  // diagonal + strict upper entries
    cudaError_t e;
    if (g->storage == ALM_GNN_BF16)
        e = gnn_loss_grad(gr, p, gp, g->a16, g->rhat, g->yhat, Rs, ys, hb->cbar, lam, npat, double(hb->rows), g->loss,
                          g->sms, g->stream);
    else
        e = gnn_loss_grad(gr, p, gp, g->a32, g->rhat, g->yhat, Rs, ys, hb->cbar, lam, npat, double(hb->rows), g->loss,
                          g->sms, g->stream);
    g->launches += 30;
    GCK(e);
    return ALM_OK;
}

// SplitMix64-based uniform initialisation: U(-1, 1) sqrt(3 / fan_in) weights, zero biases
void init_host(std::vector<float> &th, uint64_t seed) {
    auto smx = [](uint64_t s, uint64_t i) {
        uint64_t z = s + (i + 1) * 0x9e3779b97f4a7c15ULL;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        return 2.0 * (double(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    };
    th.assign(size_t(gnn_num_params()), 0.f);
    size_t o = 0;
    uint64_t k = 0;
    auto mat = [&](int rows, int cols) {
        const double sc = std::sqrt(3.0 / double(cols));
        for (int t = 0; t < rows * cols; ++t) th[o++] = float(smx(seed, k++) * sc);
    };
    int din = kGnnFeat;
    for (int l = 0; l < kGnnLayers; ++l) {
        mat(kGnnHid, din);
        mat(kGnnHid, din);
        o += kGnnHid;
        din = kGnnHid;
    }
    mat(kGnnRank, kGnnHid);
    mat(1, kGnnHid);
}

// the batch's pattern is static after alm_batch_create (uploaded and synchronised), so the
// network may read it from its own stream
alm_status check_batch_arrays(alm_gnn *g, const alm_batch *hb) {
    if (!hb) GFAIL(ALM_ERR_INVALID_ARG, "batch handle is NULL");
    return ALM_OK;
}

}  // namespace

extern "C" int32_t alm_gnn_num_params(void) { return gnn_num_params(); }

extern "C" alm_status alm_gnn_create(alm_gnn **out, int32_t storage, uint64_t feat_seed, uint64_t init_seed,
                                     alm_stream_t s) {
    if (!out) {
        g_gnn_error = "g is NULL";
        return ALM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (storage != ALM_GNN_FP32 && storage != ALM_GNN_BF16) {
        g_gnn_error = "storage must be ALM_GNN_FP32 or ALM_GNN_BF16";
        return ALM_ERR_INVALID_ARG;
    }
    alm_gnn *g = new (std::nothrow) alm_gnn();
    if (!g) {
        g_gnn_error = "host allocation failed";
        return ALM_ERR_OOM;
    }
    g->stream = static_cast<cudaStream_t>(s);
    g->storage = storage;
    g->feat_seed = feat_seed;
    g->np = gnn_num_params();
    auto fail = [&](alm_status st) {
        g_gnn_error = g->err;
        alm_gnn_destroy(g);
        return st;
    };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
    for (float **p : {&g->theta, &g->grad, &g->m, &g->v})
        if (e == cudaSuccess) e = cudaMalloc(p, sizeof(float) * size_t(g->np));
    if (e == cudaSuccess) e = cudaMalloc(&g->lpart, sizeof(double) * size_t(8 * std::max(g->sms, 1)));
    if (e == cudaSuccess) e = cudaMemsetAsync(g->m, 0, sizeof(float) * size_t(g->np), g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->v, 0, sizeof(float) * size_t(g->np), g->stream);
    std::vector<float> th;
    init_host(th, init_seed);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->theta, th.data(), sizeof(float) * th.size(), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        g->err = std::string("alm_gnn_create: ") + cudaGetErrorString(e);
        return fail(e == cudaErrorMemoryAllocation ? ALM_ERR_OOM : ALM_ERR_CUDA);
    }
    *out = g;
    return ALM_OK;
}

extern "C" void alm_gnn_destroy(alm_gnn *g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (void *p : {(void *)g->theta, (void *)g->grad, (void *)g->m, (void *)g->v, g->act, (void *)g->fbuf,
                    (void *)g->loss, (void *)g->lpart})
        if (p) cudaFree(p);
    delete g;
}

extern "C" const char *alm_gnn_last_error(const alm_gnn *g) { return g ? g->err.c_str() : g_gnn_error.c_str(); }

extern "C" alm_status alm_gnn_set_params(alm_gnn *g, const float *theta) {
    if (!g || !theta) return ALM_ERR_INVALID_ARG;
    GCK(cudaMemcpyAsync(g->theta, theta, sizeof(float) * size_t(g->np), cudaMemcpyHostToDevice, g->stream));
    GCK(cudaMemsetAsync(g->m, 0, sizeof(float) * size_t(g->np), g->stream));
    GCK(cudaMemsetAsync(g->v, 0, sizeof(float) * size_t(g->np), g->stream));
    GCK(cudaStreamSynchronize(g->stream));
    g->step = 0;
    return ALM_OK;
}

extern "C" alm_status alm_gnn_get_params(alm_gnn *g, float *theta) {
    if (!g || !theta) return ALM_ERR_INVALID_ARG;
    GCK(cudaMemcpyAsync(theta, g->theta, sizeof(float) * size_t(g->np), cudaMemcpyDeviceToHost, g->stream));
    GCK(cudaStreamSynchronize(g->stream));
    return ALM_OK;
}

extern "C" alm_status alm_gnn_forward(alm_gnn *g, const alm_batch *hb, float *rhat, float *yhat) {
    if (!g) return ALM_ERR_INVALID_ARG;
    GTRY(check_batch_arrays(g, hb));
    GTRY(ensure_buffers(g, hb->rows, false));
    GTRY(forward(g, hb));
    if (rhat)
        GCK(cudaMemcpyAsync(rhat, g->rhat, sizeof(float) * size_t(hb->rows) * kGnnRank, cudaMemcpyDeviceToDevice,
                            g->stream));
    if (yhat)
        GCK(cudaMemcpyAsync(yhat, g->yhat, sizeof(float) * size_t(hb->rows), cudaMemcpyDeviceToDevice, g->stream));
    GCK(cudaStreamSynchronize(g->stream));
    return ALM_OK;
}

extern "C" alm_status alm_gnn_warm_start(alm_gnn *g, const alm_batch *hb, double mix, float *R0, int32_t *rank,
                                         double *y0) {
    if (!g || !R0 || !rank || !y0) return ALM_ERR_INVALID_ARG;
    GTRY(check_batch_arrays(g, hb));
    if (reinterpret_cast<uintptr_t>(R0) % 16 != 0) GFAIL(ALM_ERR_INVALID_ARG, "R0 must be 16-byte aligned");
    GTRY(ensure_buffers(g, hb->rows, false));
    GTRY(forward(g, hb));
    if (!(mix >= 0.0) || !std::isfinite(mix)) GFAIL(ALM_ERR_INVALID_ARG, "mix must be finite and >= 0");
    GCK(gnn_warm(graph_of(hb), g->rhat, g->yhat, hb->cbar, float(mix), g->feat_seed ^ 0x3a1dULL, R0, y0, g->sms,
                 g->stream));
    std::vector<int32_t> r(size_t(hb->count), int32_t(std::min(kGnnRank, hb->opt.r_max)));
    GCK(cudaMemcpyAsync(rank, r.data(), sizeof(int32_t) * r.size(), cudaMemcpyHostToDevice, g->stream));
    GCK(cudaStreamSynchronize(g->stream));
    g->launches += 1;
    return ALM_OK;
}

extern "C" alm_status alm_gnn_loss_grad(alm_gnn *g, const alm_batch *hb, const float *Rstar, const double *ystar,
                                        double lam, double *loss_out, float *grad_out) {
    if (!g || !Rstar || !ystar) return ALM_ERR_INVALID_ARG;
    GTRY(check_batch_arrays(g, hb));
    GTRY(ensure_buffers(g, hb->rows, true));
    GTRY(loss_grad(g, hb, Rstar, ystar, lam));
    if (loss_out) GCK(cudaMemcpyAsync(loss_out, g->loss, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    if (grad_out)
        GCK(cudaMemcpyAsync(grad_out, g->grad, sizeof(float) * size_t(g->np), cudaMemcpyDeviceToHost, g->stream));
    GCK(cudaStreamSynchronize(g->stream));
    return ALM_OK;
}

extern "C" alm_status alm_gnn_train(alm_gnn *g, const alm_batch *hb, const float *Rstar, const double *ystar,
                                    double lam, int32_t steps, double lr, double *loss_out) {
    if (!g || !Rstar || !ystar || steps < 0 || !(lr > 0.0)) return ALM_ERR_INVALID_ARG;
    GTRY(check_batch_arrays(g, hb));
    GTRY(ensure_buffers(g, hb->rows, true));
    std::vector<double> losses(size_t(std::max(steps, 0)));
    for (int k = 0; k < steps; ++k) {
        GTRY(loss_grad(g, hb, Rstar, ystar, lam));
        if (loss_out) GCK(cudaMemcpyAsync(&losses[size_t(k)], g->loss, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
        g->step += 1;
        GCK(gnn_adam(g->theta, g->grad, g->m, g->v, g->np, lr, g->step, g->stream));
        g->launches += 1;
    }
    GCK(cudaStreamSynchronize(g->stream));
    if (loss_out)
        for (int k = 0; k < steps; ++k) loss_out[k] = losses[size_t(k)];
    return ALM_OK;
}
