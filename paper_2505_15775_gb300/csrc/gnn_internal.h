// Internal interface of the warm-start network (kernels_gnn.cu, gnn_api.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

namespace alm {

constexpr int kGnnFeat = 8;     // input features per row
constexpr int kGnnHid = 64;     // hidden width
constexpr int kGnnLayers = 3;   // message-passing layers
constexpr int kGnnRank = 32;    // columns of the factor head (the batch's row stride)

// Parameter vector layout (floats): per layer Ws (64 x din), Wn (64 x din), b (64); then
// W_R (32 x 64), w_y (64), b_y (1).  din = 8 for the first layer, 64 after.
inline int gnn_num_params() {
    int n = 0, din = kGnnFeat;
    for (int l = 0; l < kGnnLayers; ++l) {
        n += 2 * kGnnHid * din + kGnnHid;
        din = kGnnHid;
    }
    return n + kGnnRank * kGnnHid + kGnnHid + 1;
}

struct GnnParams {
    float *Ws[kGnnLayers], *Wn[kGnnLayers], *b[kGnnLayers], *WR, *wy, *by;
};
inline GnnParams gnn_views(float *base) {
    GnnParams p{};
    int o = 0, din = kGnnFeat;
    for (int l = 0; l < kGnnLayers; ++l) {
        p.Ws[l] = base + o;
        o += kGnnHid * din;
        p.Wn[l] = base + o;
        o += kGnnHid * din;
        p.b[l] = base + o;
        o += kGnnHid;
        din = kGnnHid;
    }
    p.WR = base + o;
    o += kGnnRank * kGnnHid;
    p.wy = base + o;
    o += kGnnHid;
    p.by = base + o;
    return p;
}

// The pattern the network runs on (device pointers of a batch handle).
struct GnnGraph {
    int64_t rows;
    const int32_t *row_inst;  // instance of each row
    const int64_t *row_off;   // first row of each instance
    const int32_t *rowptr;    // full symmetric off-diagonal CSR over global rows
    const int32_t *col;       // local column index
    const float *val;         // C_ij
    const float4 *scal;       // per instance: 1/dbar, 1/cbar, 1/sbar, log(n)/8
};

// Activations (T = float or __nv_bfloat16) and FP32 training buffers.
template <typename T>
struct GnnActs {
    T *H[kGnnLayers + 1] = {nullptr, nullptr, nullptr, nullptr};  // H[0]: rows x 8, H[1..3]: rows x 64
    T *AGG[kGnnLayers] = {nullptr, nullptr, nullptr};               // rows x din of each layer
    float *dR = nullptr, *dY = nullptr, *dH = nullptr, *dZ = nullptr, *dHp = nullptr, *U = nullptr;
    float *part = nullptr;   // nblk x ldp weight-gradient partials
    double *lpart = nullptr; // loss partials (one per CTA of the loss kernel)
    int nblk = 0;
    int64_t ldp = 0;
};
constexpr int64_t kGnnLdp = int64_t(kGnnHid) * kGnnHid + kGnnHid;  // widest partial: 64 x 64 + 64

template <typename T>
cudaError_t gnn_forward(const GnnGraph &g, const GnnParams &p, uint64_t feat_seed, GnnActs<T> &a, float *rhat,
                        float *yhat, int sms, cudaStream_t s);
cudaError_t gnn_warm(const GnnGraph &g, const float *rhat, const float *yhat, const double *cbar, float mix,
                     uint64_t mix_seed, float *R0, double *y0, int sms, cudaStream_t s);
template <typename T>
cudaError_t gnn_loss_grad(const GnnGraph &g, const GnnParams &p, const GnnParams &grad, GnnActs<T> &a,
                          const float *rhat, const float *yhat, const float *Rs, const double *ys, const double *cbar,
                          double lam, double n_pattern, double n_rows, double *loss_dev, int sms, cudaStream_t s);
cudaError_t gnn_adam(float *theta, const float *grad, float *m, float *v, int cnt, double lr, int step,
                     cudaStream_t s);

}  // namespace alm
