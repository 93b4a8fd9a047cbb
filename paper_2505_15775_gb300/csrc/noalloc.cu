// alm_grad_unitdiag_noalloc: the gradient G = 2 S R of the augmented Lagrangian for
// problems whose constraints are X_ii = b_i, one per row (the MaxCut SDP form), computed
// from device arrays the caller owns, without allocating any device memory.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not wanted -- inside
// a region with a fixed, pre-reserved memory budget, a caller whose allocator must not be
// re-entered, or a deployment that forbids allocation after start-up.  Such callers cannot
// use alm_create (it allocates the pattern copies and work buffers), but can hand over the
// problem in CSR form themselves.
//
// The only working memory is diag(S) = C_ii - w_i, w_i = y_i - sigma (X_ii - b_i), kept in a
// file-scope device array of kNoAllocMaxRows doubles (8 MiB).  Every GPU that loads the
// library holds that array until the process exits.  Each call writes every entry it later
// reads, so nothing has to start at zero; calls that overlap on the GPU (two streams, or
// two host threads) share the array and race.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "alm_internal.h"
#include "dev_util.cuh"

namespace alm {

constexpr int64_t kNoAllocMaxRows = int64_t(1) << 20;  // rows the scratch array holds

// the scratch array (file scope, one per device that loads the library)
static __device__ __align__(256) double g_slack_diag_scratch[kNoAllocMaxRows];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_addr_mu;
double *g_addr[kMaxDevices] = {};  // device address of the array, per device

// S_ii = C_ii - (y_i - sigma (|r_i|^2 - b_i)) for every row (compensated |r_i|^2 in FP32)
template <typename T, int LANES>
__global__ void __launch_bounds__(kBlock) k_na_slack(int64_t n, const T *__restrict__ cdiag,
                                                     const double *__restrict__ b, const double *__restrict__ y,
                                                     double sigma, const T *__restrict__ R, int r, int ldr,
                                                     double *__restrict__ sdiag) {
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LANES - 1);
    const unsigned gmask = group_mask<LANES>(lane);
    const int gpb = kBlock / LANES;
    const int64_t ng = int64_t(gridDim.x) * gpb;
    const bool active = gl * W < r;
    for (int64_t i = int64_t(blockIdx.x) * gpb + threadIdx.x / LANES; i < n; i += ng) {
        const V ri = mask_tail(active ? ldro(R + i * ldr + gl * W) : vzero(T()), gl * W, r);
        const double xii = ff_norm2<LANES>(ri, gmask);
        if (gl == 0) sdiag[i] = double(cdiag[i]) - (y[i] - sigma * (xii - b[i]));
    }
}

// G = 2 (S_off R + diag(S) R), one row per group; columns r..ldr-1 of G are zeroed
template <typename T, int LANES>
__global__ void __launch_bounds__(kBlock) k_na_spmm(int64_t n, const int *__restrict__ rowptr,
                                                    const int *__restrict__ col, const T *__restrict__ val,
                                                    const double *__restrict__ sdiag, const T *__restrict__ R, int r,
                                                    int ldr, T *__restrict__ G) {
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LANES - 1);
    const int gpb = kBlock / LANES;
    const int64_t ng = int64_t(gridDim.x) * gpb;
    const bool active = gl * W < r;
    const int nv = ldr / W;
    for (int64_t i = int64_t(blockIdx.x) * gpb + threadIdx.x / LANES; i < n; i += ng) {
        const V ri = mask_tail(active ? ldro(R + i * ldr + gl * W) : vzero(T()), gl * W, r);
        const double d = sdiag[i];
        const T dh = T(d);
        const T dl = T(d - double(dh));
        V acc = fma4(dl, ri, scale4(dh, ri));
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
            acc = fma4(val[e], active ? ldro(R + int64_t(col[e]) * ldr + gl * W) : vzero(T()), acc);
        const V g = mask_tail(scale4(T(2), acc), gl * W, r);
        if (gl < nv) stv(G + i * ldr + gl * W, g);
        for (int q = LANES + gl; q < nv; q += LANES) stv(G + i * ldr + q * W, vzero(T()));
    }
}

template <typename T>
void na_launch(int64_t n, const int *rowptr, const int *col, const T *val, const T *cdiag, const double *b,
               const double *y, double sigma, const T *R, int r, int ldr, T *G, double *scratch, int grid,
               cudaStream_t s) {
    constexpr int W = VecT<T>::W;
    const int nvec = (r + W - 1) / W;
    int L = 1;
    while (L < nvec) L <<= 1;
    switch (L) {
#define ALM_NA_CASE(LN)                                                                                   \
    case LN:                                                                                              \
        k_na_slack<T, LN><<<grid, kBlock, 0, s>>>(n, cdiag, b, y, sigma, R, r, ldr, scratch);             \
        k_na_spmm<T, LN><<<grid, kBlock, 0, s>>>(n, rowptr, col, val, scratch, R, r, ldr, G);             \
        break;
        ALM_NA_CASE(1)
        ALM_NA_CASE(2)
        ALM_NA_CASE(4)
        ALM_NA_CASE(8)
        default:
            ALM_NA_CASE(16)
#undef ALM_NA_CASE
    }
}

}  // namespace

}  // namespace alm

using namespace alm;

extern "C" alm_status alm_grad_unitdiag_noalloc(int32_t precision, int64_t n, const int32_t *rowptr,
                                                const int32_t *col, const void *val, const void *cdiag,
                                                const double *b, const double *y, double sigma, const void *R,
                                                int32_t r, int32_t ldr, void *G, alm_stream_t s) {
    auto fail = [](alm_status st, const char *msg) {
        set_global_error(msg);
        return st;
    };
    if (precision != ALM_FP64 && precision != ALM_FP32) return fail(ALM_ERR_INVALID_ARG, "precision must be ALM_FP64 or ALM_FP32");
    if (n < 1) return fail(ALM_ERR_INVALID_ARG, "n must be >= 1");
    if (n > kNoAllocMaxRows)
        return fail(ALM_ERR_INVALID_ARG, "n exceeds the 1048576 rows the no-allocation scratch array holds");
    if (!rowptr || !col || !val || !cdiag || !b || !y || !R || !G) return fail(ALM_ERR_INVALID_ARG, "a pointer argument is NULL");
    if (r < 1 || r > kMaxRank) return fail(ALM_ERR_INVALID_ARG, "rank r must be in 1..32");
    const size_t esz = precision == ALM_FP64 ? 8 : 4;
    if (ldr < r || (size_t(ldr) * esz) % 16 != 0) return fail(ALM_ERR_INVALID_ARG, "ldr must be >= r and ldr * element size a multiple of 16 bytes");
    if (reinterpret_cast<uintptr_t>(R) % 16 || reinterpret_cast<uintptr_t>(G) % 16)
        return fail(ALM_ERR_INVALID_ARG, "R and G must be 16-byte aligned");
    if (G == R) return fail(ALM_ERR_INVALID_ARG, "G may not alias R");
    if (!std::isfinite(sigma) || sigma < 0) return fail(ALM_ERR_INVALID_ARG, "sigma must be finite and >= 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ALM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(ALM_ERR_INVALID_ARG, "device index beyond 63");
    double *scratch = nullptr;
    {
        // one-time set-up per device (with that device current): the device address of the
        // scratch array; host code may not use the array's name as an address
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_slack_diag_scratch);
            if (e != cudaSuccess) return fail(ALM_ERR_CUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
            g_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_addr[dev];
    }
    int sms = kNumSMs;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        sms = kNumSMs;
    }
    const int grid = sms * 4;
    cudaStream_t st = static_cast<cudaStream_t>(s);
    if (precision == ALM_FP64)
        na_launch<double>(n, rowptr, col, static_cast<const double *>(val), static_cast<const double *>(cdiag), b, y,
                          sigma, static_cast<const double *>(R), r, ldr, static_cast<double *>(G), scratch, grid, st);
    else
        na_launch<float>(n, rowptr, col, static_cast<const float *>(val), static_cast<const float *>(cdiag), b, y,
                         sigma, static_cast<const float *>(R), r, ldr, static_cast<float *>(G), scratch, grid, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ALM_ERR_CUDA, cudaGetErrorString(e));
    return ALM_OK;
}
