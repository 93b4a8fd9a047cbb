// Internal interface of the batched persistent solver: the device view of a batch of
// unit-diagonal SDPs (min <C_b, X_b> s.t. diag(X_b) = 1, X_b >= 0; the MaxCut SDP form of
// Sec. 6.1) and the launcher of the persistent kernel.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "alm.h"
#include "alm_internal.h"

namespace alm {

constexpr int kBatchLanes = 8;  // lanes per row group: 8 x float4 = the 32 columns of a row
constexpr int64_t kBatchMaxRows = 16384;  // rows of one instance (the per-CTA scratch grows with it)

// Every pointer is device memory.  Row i of instance b is global row row_off[b] + i; the
// off-diagonal pattern of C_b is full symmetric CSR over global rows with LOCAL column
// indices.  R is row-major with a fixed stride of kMaxRank floats.
struct BatchArgs {
    int32_t count;             // entries of `order` to process (the queue length)
    const int64_t *row_off;    // instances + 1
    const int32_t *rowptr;     // total rows + 1 (global offsets into col/val)
    const int32_t *col;        // local column index
    const float *val;          // C_ij
    const double *cdiag;       // C_ii, per global row
    const double *norm_c;      // ||C_b||_F
    const double *pc_floor;    // preconditioner floor of S_ii, per instance
    const int32_t *order;      // queue position -> instance
    float *R;                  // total rows x kMaxRank
    int32_t *rank;             // per instance, in/out
    double *y;                 // per global row, in/out
    alm_instance_stats *out;   // per instance
    int32_t *queue;            // work counter, 0 before the launch
    // per-CTA scratch: CTA k uses scr_f + k * scr_f_stride and scr_d + k * scr_d_stride
    float *scr_f;
    double *scr_d;
    int64_t nmax;              // rows of the largest instance
    int64_t scr_f_stride, scr_d_stride;
    // options (alm_options)
    double sigma0, sigma_max, eps, inner_rel, inner_floor, inner_start, inner_decay, lanczos_tol;
    int32_t sigma_rule, max_outer, max_inner, inner_method, precond, lanczos_k, lanczos_max_restarts, r_max;
    int32_t lanczos_warm, fallback_inner;
    uint64_t seed;
};

// float scratch of one CTA: Z and D (nmax x 32 each), the Lanczos basis (lanczos_k + 1
// columns of nmax), the Lanczos work vector, diag(S) and the base C_ii - y_i as float pairs
inline int64_t batch_scr_f_floats(int64_t nmax, int lanczos_k) {
    return nmax * (2 * kMaxRank) + int64_t(lanczos_k + 1) * nmax + 5 * nmax;
}
inline int64_t batch_scr_d_doubles(int64_t nmax) { return nmax; }  // the dual candidate w

// Threads per CTA the kernel is compiled for.
constexpr int kBatchThreads[3] = {256, 512, 1024};

// Launch the persistent kernel with `threads` per CTA on `grid` CTAs.
cudaError_t launch_batch_solve(const BatchArgs &a, int threads, int grid, cudaStream_t s);
// Resident CTAs per SM of the kernel compiled for `threads` (cudaOccupancy...).
int batch_ctas_per_sm(int threads);

}  // namespace alm

// The batch handle (opaque in the C ABI); shared with the warm-start network, which runs
// on a batch's pattern.
struct alm_batch {
    std::string err;
    cudaStream_t stream = nullptr;
    alm_options opt{};
    int32_t count = 0;
    int64_t rows = 0, nmax = 0, nnz = 0;
    int sms = 0;
    int threads = 512;
    std::vector<int64_t> h_row_off;
    std::vector<int32_t> h_order;
    // device
    int64_t *row_off = nullptr;
    int32_t *rowptr = nullptr, *col = nullptr, *order = nullptr, *sample = nullptr, *queue = nullptr;
    int32_t *row_inst = nullptr;  // instance of each global row
    float4 *gnn_scal = nullptr;   // per instance: 1/dbar, 1/cbar, 1/sbar, log(n)/8 (warm-start network)
    double *cbar = nullptr;       // per instance: mean |C_ij| over the off-diagonal entries
    float *val = nullptr;
    double *cdiag = nullptr, *norm_c = nullptr, *pc_floor = nullptr;
    alm_instance_stats *out = nullptr;
    float *scr_f = nullptr;
    double *scr_d = nullptr;
    int scr_ctas = 0;
    int64_t scr_f_stride = 0, scr_d_stride = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_threads = 0;
    const void *graph_R = nullptr, *graph_rank = nullptr, *graph_y = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};
