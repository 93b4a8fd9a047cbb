// C ABI of the batched persistent solver (include/alm.h, alm_batch_*): host-side
// validation and pattern build of many small unit-diagonal SDPs, the queue order, the
// per-CTA scratch, the CUDA graph around the one persistent launch, and the autotuner of
// its CTA size.  Every step of every solve runs in kernels_batch.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "batch_internal.h"

using namespace alm;

namespace {
thread_local std::string g_batch_error;
}


#define BCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            hb->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return e_ == cudaErrorMemoryAllocation ? ALM_ERR_OOM : ALM_ERR_CUDA;          \
        }                                                                                 \
    } while (0)
#define BFAIL(code, msg)     \
    do {                     \
        hb->err = (msg);     \
        return (code);       \
    } while (0)
#define BTRY(expr)                   \
    do {                             \
        alm_status s_ = (expr);      \
        if (s_ != ALM_OK) return s_; \
    } while (0)

namespace {

template <typename T>
alm_status upload(alm_batch *hb, T **dst, const std::vector<T> &src) {
    BCK(cudaMalloc(reinterpret_cast<void **>(dst), sizeof(T) * std::max<size_t>(src.size(), 1)));
    if (!src.empty())
        BCK(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, hb->stream));
    return ALM_OK;
}

// Pattern of one instance: C_ii into cdiag, the off-diagonal entries in full symmetric
// CSR (rows sorted by column, repeated entries merged) appended to col/val, row pointers
// relative to the instance's first entry.
struct InstPattern {
    std::vector<int32_t> ptr, col;
    std::vector<float> val;
    std::vector<double> diag;
    double norm_c = 0.0, pc_floor = 0.0;
    double dbar = 1.0, cbar = 1.0, sbar = 1.0;  // scales of the warm-start network's inputs
    std::string err;
};

void build_instance(const alm_batch_problem *p, int b, InstPattern *out) {
    const int64_t n = p->row_off[b + 1] - p->row_off[b];
    const int64_t e0 = p->nnz_off[b], e1 = p->nnz_off[b + 1];
    out->diag.assign(static_cast<size_t>(n), 0.0);
    std::vector<int64_t> cnt(static_cast<size_t>(n) + 1, 0);
    for (int64_t e = e0; e < e1; ++e) {
        const int64_t i = p->c_i[e], j = p->c_j[e];
        const double v = p->c_v[e];
        if (i < 0 || j < 0 || i >= n || j >= n || i > j) {
            out->err = "instance " + std::to_string(b) + ": entry " + std::to_string(e - e0) +
                       " is not an upper-triangle index pair of an n_b x n_b matrix";
            return;
        }
        if (!std::isfinite(v)) {
            out->err = "instance " + std::to_string(b) + ": non-finite value of C";
            return;
        }
        if (i == j) out->diag[size_t(i)] += v;
        else {
            cnt[size_t(i) + 1] += 1;
            cnt[size_t(j) + 1] += 1;
        }
    }
    for (int64_t i = 0; i < n; ++i) cnt[size_t(i) + 1] += cnt[size_t(i)];
    std::vector<std::pair<int32_t, double>> ent(static_cast<size_t>(cnt[size_t(n)]));
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (int64_t e = e0; e < e1; ++e) {
        const int32_t i = p->c_i[e], j = p->c_j[e];
        if (i == j) continue;
        ent[size_t(pos[size_t(i)]++)] = {j, p->c_v[e]};
        ent[size_t(pos[size_t(j)]++)] = {i, p->c_v[e]};
    }
    out->ptr.assign(size_t(n) + 1, 0);
    double nc = 0.0, acd = 0.0, asum = 0.0, arow = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double srow = 0.0;
        auto first = ent.begin() + cnt[size_t(i)], last = ent.begin() + cnt[size_t(i) + 1];
        std::sort(first, last, [](const auto &x, const auto &y) { return x.first < y.first; });
        for (auto it = first; it != last;) {
            int32_t c = it->first;
            double v = 0.0;
            for (; it != last && it->first == c; ++it) v += it->second;
            out->col.push_back(c);
            out->val.push_back(float(v));
            nc += v * v;  // each off-diagonal pair appears twice: 2 C_ij^2 in total
            asum += std::fabs(v);
            srow += v;
        }
        arow += std::fabs(srow);
        out->ptr[size_t(i) + 1] = int32_t(out->col.size());
        nc += out->diag[size_t(i)] * out->diag[size_t(i)];
        acd += std::fabs(out->diag[size_t(i)]);
    }
    out->norm_c = std::sqrt(nc);
    out->pc_floor = 1e-2 * (1.0 + acd / double(n));
    const double ne = double(out->col.size());
    out->dbar = std::max(ne / double(n), 1.0);
    out->cbar = ne > 0 ? asum / ne : 1.0;
    out->sbar = arow > 0 ? arow / double(n) : 1.0;
}

alm_status create_impl(alm_batch *hb, const alm_batch_problem *p) {
    const alm_options &o = hb->opt;
    if (o.precision != ALM_FP32) BFAIL(ALM_ERR_INVALID_ARG, "the batched solver computes in the ALM_FP32 form only");
    if (o.r_max < 1 || o.r_max > kMaxRank) BFAIL(ALM_ERR_INVALID_ARG, "r_max must be in 1..32");
    if (o.lanczos_k < 2 || o.lanczos_k > kLzMax) BFAIL(ALM_ERR_INVALID_ARG, "lanczos_k must be in 2..64");
    if (!(o.sigma0 > 0.0) || !(o.eps > 0.0)) BFAIL(ALM_ERR_INVALID_ARG, "sigma0 and eps must be > 0");
    if (o.max_outer < 1 || o.max_inner < 1 || o.lanczos_max_restarts < 1)
        BFAIL(ALM_ERR_INVALID_ARG, "max_outer, max_inner and lanczos_max_restarts must be >= 1");
    if (!p || p->count < 1 || !p->row_off || !p->nnz_off) BFAIL(ALM_ERR_INVALID_ARG, "empty batch or NULL offsets");
    const int count = p->count;
    if (p->row_off[0] != 0 || p->nnz_off[0] != 0) BFAIL(ALM_ERR_INVALID_ARG, "row_off[0] and nnz_off[0] must be 0");
    for (int b = 0; b < count; ++b) {
        const int64_t n = p->row_off[b + 1] - p->row_off[b];
        if (n < 1 || n >= (int64_t(1) << 31)) BFAIL(ALM_ERR_INVALID_ARG, "every instance needs 1 <= n_b < 2^31 rows");
        if (p->nnz_off[b + 1] < p->nnz_off[b]) BFAIL(ALM_ERR_INVALID_ARG, "nnz_off must be non-decreasing");
    }
    if (p->nnz_off[count] > 0 && (!p->c_i || !p->c_j || !p->c_v)) BFAIL(ALM_ERR_INVALID_ARG, "NULL entry arrays");
    hb->count = count;
    hb->rows = p->row_off[count];
    hb->h_row_off.assign(p->row_off, p->row_off + count + 1);
    std::vector<InstPattern> ip(static_cast<size_t>(count));
    {
        const int nt = std::max(1, std::min<int>(int(std::thread::hardware_concurrency()), 32));
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t)
            pool.emplace_back([&, t] {
                for (int b = t; b < count; b += nt) build_instance(p, b, &ip[size_t(b)]);
            });
        for (auto &th : pool) th.join();
    }
    int64_t nnz = 0;
    for (int b = 0; b < count; ++b) {
        if (!ip[size_t(b)].err.empty()) BFAIL(ALM_ERR_INVALID_ARG, ip[size_t(b)].err);
        nnz += int64_t(ip[size_t(b)].col.size());
        hb->nmax = std::max<int64_t>(hb->nmax, hb->h_row_off[size_t(b) + 1] - hb->h_row_off[size_t(b)]);
    }
    if (nnz >= (int64_t(1) << 31)) BFAIL(ALM_ERR_INVALID_ARG, "the batch has more than 2^31 - 1 off-diagonal entries");
    hb->nnz = nnz;
    std::vector<int32_t> rowptr(static_cast<size_t>(hb->rows) + 1), col(static_cast<size_t>(nnz));
    std::vector<float> val(static_cast<size_t>(nnz));
    std::vector<double> cdiag(static_cast<size_t>(hb->rows)), norm_c(static_cast<size_t>(count)),
        pcf(static_cast<size_t>(count)), work(static_cast<size_t>(count)), cbar(static_cast<size_t>(count));
    std::vector<int32_t> row_inst(static_cast<size_t>(hb->rows));
    std::vector<float4> scal(static_cast<size_t>(count));
    int64_t base = 0;
    for (int b = 0; b < count; ++b) {
        const InstPattern &q = ip[size_t(b)];
        const int64_t r0 = hb->h_row_off[size_t(b)];
        const int64_t n = hb->h_row_off[size_t(b) + 1] - r0;
        for (int64_t i = 0; i <= n; ++i) rowptr[size_t(r0 + i)] = int32_t(base + q.ptr[size_t(i)]);
        std::copy(q.col.begin(), q.col.end(), col.begin() + base);
        std::copy(q.val.begin(), q.val.end(), val.begin() + base);
        std::copy(q.diag.begin(), q.diag.end(), cdiag.begin() + r0);
        norm_c[size_t(b)] = q.norm_c;
        pcf[size_t(b)] = q.pc_floor;
        work[size_t(b)] = double(q.col.size()) + 8.0 * double(n);  // row passes touch n x 32 floats
        cbar[size_t(b)] = q.cbar;
        scal[size_t(b)] = make_float4(float(1.0 / q.dbar), float(1.0 / q.cbar), float(1.0 / q.sbar),
                                      float(std::log(double(n)) / 8.0));
        std::fill(row_inst.begin() + r0, row_inst.begin() + r0 + n, int32_t(b));
        base += int64_t(q.col.size());
    }
    // largest work first (longest-processing-time order), ties by index
    hb->h_order.resize(size_t(count));
    for (int b = 0; b < count; ++b) hb->h_order[size_t(b)] = b;
    std::stable_sort(hb->h_order.begin(), hb->h_order.end(),
                     [&](int32_t x, int32_t y) { return work[size_t(x)] > work[size_t(y)]; });
    BTRY(upload(hb, &hb->row_off, hb->h_row_off));
    BTRY(upload(hb, &hb->rowptr, rowptr));
    BTRY(upload(hb, &hb->col, col));
    BTRY(upload(hb, &hb->val, val));
    BTRY(upload(hb, &hb->cdiag, cdiag));
    BTRY(upload(hb, &hb->norm_c, norm_c));
    BTRY(upload(hb, &hb->pc_floor, pcf));
    BTRY(upload(hb, &hb->order, hb->h_order));
    BTRY(upload(hb, &hb->row_inst, row_inst));
    BTRY(upload(hb, &hb->gnn_scal, scal));
    BTRY(upload(hb, &hb->cbar, cbar));
    BCK(cudaMalloc(&hb->sample, sizeof(int32_t) * size_t(count)));
    BCK(cudaMalloc(&hb->queue, sizeof(int32_t)));
    BCK(cudaMalloc(&hb->out, sizeof(alm_instance_stats) * size_t(count)));
    int dev = 0;
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&hb->sms, cudaDevAttrMultiProcessorCount, dev));
    BCK(cudaEventCreate(&hb->ev[0]));
    BCK(cudaEventCreate(&hb->ev[1]));
    BCK(cudaStreamSynchronize(hb->stream));
    return ALM_OK;
}

int grid_for(alm_batch *hb, int threads) {
    const int per = batch_ctas_per_sm(threads);
    return std::max(1, per) * hb->sms;
}

alm_status ensure_scratch(alm_batch *hb, int ctas) {
    if (hb->scr_f && hb->scr_ctas >= ctas) return ALM_OK;
    // the cached graph's kernel arguments hold the old scratch pointers: drop it (the stream
    // is idle here, every caller synchronises before it returns)
    if (hb->graph) {
        cudaGraphExecDestroy(hb->graph);
        hb->graph = nullptr;
    }
    if (hb->scr_f) cudaFree(hb->scr_f);
    if (hb->scr_d) cudaFree(hb->scr_d);
    hb->scr_f = nullptr;
    hb->scr_d = nullptr;
    hb->scr_ctas = 0;
    auto round64 = [](int64_t x) { return (x + 63) / 64 * 64; };  // 256-byte aligned CTA slices
    hb->scr_f_stride = round64(batch_scr_f_floats(hb->nmax, hb->opt.lanczos_k));
    hb->scr_d_stride = round64(batch_scr_d_doubles(hb->nmax));
    BCK(cudaMalloc(&hb->scr_f, sizeof(float) * size_t(hb->scr_f_stride) * size_t(ctas)));
    BCK(cudaMalloc(&hb->scr_d, sizeof(double) * size_t(hb->scr_d_stride) * size_t(ctas)));
    hb->scr_ctas = ctas;
    return ALM_OK;
}

BatchArgs args_for(alm_batch *hb, float *R, int32_t *rank, double *y, const int32_t *order, int count) {
    const alm_options &o = hb->opt;
    BatchArgs a{};
    a.count = count;
    a.row_off = hb->row_off;
    a.rowptr = hb->rowptr;
    a.col = hb->col;
    a.val = hb->val;
    a.cdiag = hb->cdiag;
    a.norm_c = hb->norm_c;
    a.pc_floor = hb->pc_floor;
    a.order = order;
    a.R = R;
    a.rank = rank;
    a.y = y;
    a.out = hb->out;
    a.queue = hb->queue;
    a.scr_f = hb->scr_f;
    a.scr_d = hb->scr_d;
    a.nmax = hb->nmax;
    a.scr_f_stride = hb->scr_f_stride;
    a.scr_d_stride = hb->scr_d_stride;
    a.sigma0 = o.sigma0;
    a.sigma_max = o.sigma_max;
    a.eps = o.eps;
    a.inner_rel = o.inner_rel;
    a.inner_floor = o.inner_floor;
    a.inner_start = o.inner_start;
    a.inner_decay = o.inner_decay;
    a.lanczos_tol = o.lanczos_tol;
    a.sigma_rule = o.sigma_rule;
    a.max_outer = o.max_outer;
    a.max_inner = o.max_inner;
    a.inner_method = o.inner_method;
    a.precond = o.inner_precond;
    a.lanczos_k = o.lanczos_k;
    a.lanczos_max_restarts = o.lanczos_max_restarts;
    a.r_max = o.r_max;
    a.lanczos_warm = o.lanczos_warm;
    a.fallback_inner = o.fallback_inner;
    a.seed = o.seed;
    return a;
}

// the counter reset and the persistent launch, on hb->stream
alm_status enqueue(alm_batch *hb, const BatchArgs &a, int threads, int grid) {
    BCK(cudaMemsetAsync(hb->queue, 0, sizeof(int32_t), hb->stream));
    BCK(launch_batch_solve(a, threads, grid, hb->stream));
    return ALM_OK;
}

alm_status check_arrays(alm_batch *hb, const void *R, const void *rank, const void *y) {
    if (hb->nmax > kBatchMaxRows)
        BFAIL(ALM_ERR_INVALID_ARG, "the batched solver takes instances of at most 16384 rows (alm_solve takes larger ones)");
    if (!R || !rank || !y) BFAIL(ALM_ERR_INVALID_ARG, "R, rank and y must be device pointers");
    if (reinterpret_cast<uintptr_t>(R) % 16 != 0) BFAIL(ALM_ERR_INVALID_ARG, "R must be 16-byte aligned");
    for (const void *ptr : {R, rank, y}) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            (void)cudaGetLastError();
            BFAIL(ALM_ERR_INVALID_ARG, "R, rank and y must be device memory");
        }
    }
    return ALM_OK;
}

}  // namespace

extern "C" alm_status alm_batch_create(alm_batch **out, const alm_batch_problem *p, const alm_options *o,
                                       alm_stream_t s) {
    if (!out) {
        g_batch_error = "hb is NULL";
        return ALM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    alm_batch *hb = new (std::nothrow) alm_batch();
    if (!hb) {
        g_batch_error = "host allocation failed";
        return ALM_ERR_OOM;
    }
    hb->stream = static_cast<cudaStream_t>(s);
    if (o) hb->opt = *o;
    else {
        alm_default_options(&hb->opt);
        hb->opt.precision = ALM_FP32;
        hb->opt.lanczos_warm = 1;
    }
    const alm_status st = create_impl(hb, p);
    if (st != ALM_OK) {
        g_batch_error = hb->err;
        alm_batch_destroy(hb);
        return st;
    }
    *out = hb;
    return ALM_OK;
}

extern "C" void alm_batch_destroy(alm_batch *hb) {
    if (!hb) return;
    if (hb->stream) cudaStreamSynchronize(hb->stream);
    if (hb->graph) cudaGraphExecDestroy(hb->graph);
    for (cudaEvent_t e : hb->ev)
        if (e) cudaEventDestroy(e);
    void *ptrs[] = {hb->row_off, hb->rowptr, hb->col, hb->order, hb->sample, hb->queue, hb->val, hb->cdiag,
                    hb->norm_c, hb->pc_floor, hb->out, hb->scr_f, hb->scr_d, hb->row_inst, hb->gnn_scal,
                    hb->cbar};
    for (void *ptr : ptrs)
        if (ptr) cudaFree(ptr);
    delete hb;
}

extern "C" const char *alm_batch_last_error(const alm_batch *hb) {
    return hb ? hb->err.c_str() : g_batch_error.c_str();
}

extern "C" alm_status alm_batch_solve(alm_batch *hb, float *R, int32_t *rank, double *y, alm_batch_stats *stats,
                                      alm_instance_stats *per_instance) {
    if (!hb) return ALM_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    BTRY(check_arrays(hb, R, rank, y));
    const int threads = hb->threads;
    const int grid = std::min<int>(grid_for(hb, threads), hb->count);
    BTRY(ensure_scratch(hb, grid));
    const BatchArgs a = args_for(hb, R, rank, y, hb->order, hb->count);
    int64_t launches = 0;
    if (hb->stream != nullptr) {  // no capture on the legacy default stream
        if (!hb->graph || hb->graph_threads != threads || hb->graph_R != R || hb->graph_rank != rank ||
            hb->graph_y != y) {
            if (hb->graph) {
                cudaGraphExecDestroy(hb->graph);
                hb->graph = nullptr;
            }
            cudaGraph_t g;
            BCK(cudaStreamBeginCapture(hb->stream, cudaStreamCaptureModeThreadLocal));
            const alm_status st = enqueue(hb, a, threads, grid);
            const cudaError_t ee = cudaStreamEndCapture(hb->stream, &g);
            BTRY(st);
            BCK(ee);
            BCK(cudaGraphInstantiate(&hb->graph, g, 0));
            cudaGraphDestroy(g);
            hb->graph_threads = threads;
            hb->graph_R = R;
            hb->graph_rank = rank;
            hb->graph_y = y;
        }
        BCK(cudaEventRecord(hb->ev[0], hb->stream));
        BCK(cudaGraphLaunch(hb->graph, hb->stream));
        BCK(cudaEventRecord(hb->ev[1], hb->stream));
    } else {
        BCK(cudaEventRecord(hb->ev[0], hb->stream));
        BTRY(enqueue(hb, a, threads, grid));
        BCK(cudaEventRecord(hb->ev[1], hb->stream));
    }
    launches = 1;
    std::vector<alm_instance_stats> h(static_cast<size_t>(hb->count));
    BCK(cudaMemcpyAsync(h.data(), hb->out, sizeof(alm_instance_stats) * h.size(), cudaMemcpyDeviceToHost,
                        hb->stream));
    BCK(cudaStreamSynchronize(hb->stream));
    float ms = 0.f;
    BCK(cudaEventElapsedTime(&ms, hb->ev[0], hb->ev[1]));
    alm_batch_stats S{};
    S.status = ALM_OK;
    for (const auto &x : h) {
        if (x.status == ALM_OK) S.converged += 1;
        else if (S.status == ALM_OK) S.status = x.status;
        S.inner_total += x.inner_total;
        S.lanczos_matvecs += x.lanczos_matvecs;
    }
    S.threads = threads;
    S.ctas_per_sm = batch_ctas_per_sm(threads);
    S.grid = grid;
    S.kernel_launches = launches;
    S.device_ms = ms;
    S.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S;
    if (per_instance) std::memcpy(per_instance, h.data(), sizeof(alm_instance_stats) * h.size());
    if (S.status != ALM_OK) hb->err = "some instances did not converge (see the per-instance statuses)";
    return alm_status(S.status);
}

extern "C" alm_status alm_batch_autotune(alm_batch *hb, const float *R, const int32_t *rank, const double *y,
                                         int32_t *threads_out, double *times_ms) {
    if (!hb) return ALM_ERR_INVALID_ARG;
    BTRY(check_arrays(hb, R, rank, y));
    // sample: about two instances per resident CTA of the largest grid, spread evenly over
    // the queue order (so over the size range), kept in that order
    int gmax = 0;
    for (int t : kBatchThreads) gmax = std::max(gmax, grid_for(hb, t));
    const int ns = std::min<int>(hb->count, 2 * gmax);
    std::vector<int32_t> smp(static_cast<size_t>(ns));
    for (int k = 0; k < ns; ++k) smp[size_t(k)] = hb->h_order[size_t((int64_t(k) * hb->count) / ns)];
    BCK(cudaMemcpyAsync(hb->sample, smp.data(), sizeof(int32_t) * size_t(ns), cudaMemcpyHostToDevice, hb->stream));
    BTRY(ensure_scratch(hb, std::min(gmax, ns)));
    float *Rt = nullptr;
    int32_t *rt = nullptr;
    double *yt = nullptr;
    const size_t rbytes = sizeof(float) * size_t(hb->rows) * kMaxRank;
    BCK(cudaMalloc(&Rt, rbytes));
    BCK(cudaMalloc(&rt, sizeof(int32_t) * size_t(hb->count)));
    BCK(cudaMalloc(&yt, sizeof(double) * size_t(hb->rows)));
    alm_status result = ALM_OK;
    double best = INFINITY;
    int best_t = hb->threads;
    for (int ci = 0; ci < 3 && result == ALM_OK; ++ci) {
        const int t = kBatchThreads[ci];
        const int grid = std::min(grid_for(hb, t), ns);
        BatchArgs a = args_for(hb, Rt, rt, yt, hb->sample, ns);
        a.max_outer = 1;
        float msb = INFINITY;
        for (int rep = 0; rep < 2; ++rep) {  // the first run also loads the kernel
            cudaError_t e = cudaMemcpyAsync(Rt, R, rbytes, cudaMemcpyDeviceToDevice, hb->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(rt, rank, sizeof(int32_t) * size_t(hb->count), cudaMemcpyDeviceToDevice,
                                    hb->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(yt, y, sizeof(double) * size_t(hb->rows), cudaMemcpyDeviceToDevice, hb->stream);
            if (e == cudaSuccess) e = cudaEventRecord(hb->ev[0], hb->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(hb->queue, 0, sizeof(int32_t), hb->stream);
            if (e == cudaSuccess) e = launch_batch_solve(a, t, grid, hb->stream);
            if (e == cudaSuccess) e = cudaEventRecord(hb->ev[1], hb->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(hb->stream);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, hb->ev[0], hb->ev[1]);
            if (e != cudaSuccess) {
                hb->err = std::string("autotune launch: ") + cudaGetErrorString(e);
                result = ALM_ERR_CUDA;
                break;
            }
            msb = std::min(msb, ms);
        }
        if (times_ms) times_ms[ci] = msb;
        if (msb < best) {
            best = msb;
            best_t = t;
        }
    }
    cudaFree(Rt);
    cudaFree(rt);
    cudaFree(yt);
    BTRY(result);
    hb->threads = best_t;
    if (threads_out) *threads_out = best_t;
    return ALM_OK;
}

extern "C" alm_status alm_batch_set_threads(alm_batch *hb, int32_t threads) {
    if (!hb) return ALM_ERR_INVALID_ARG;
    if (threads != 256 && threads != 512 && threads != 1024)
        BFAIL(ALM_ERR_INVALID_ARG, "threads per CTA must be 256, 512 or 1024");
    hb->threads = threads;
    return ALM_OK;
}
