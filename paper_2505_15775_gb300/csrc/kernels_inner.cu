// The two kernels of one inner CG step of the ELL form (diagonal-selector problems such as
// the MaxCut SDP; Sec. 6.1), each in two launch shapes:
//
//   step + SpMM   R' = R + alpha D (the pending step of the previous line search), the slack
//                 diagonal S_ii from |r_i'|^2 in float pairs, G = 2 S R', the row-block
//                 preconditioner Z = P^{-1} G and the CG inner products (Sec. 4.2: the BM
//                 gradient 2 grad f(RR^T) R)
//   dir + LS      D_new = -Z + beta D_old and the quartic coefficients of the exact step
//                 along D_new (Eq. AL expanded in alpha), with the FP64 cubic solve in the
//                 last block
//
// Shape 0 loads a row group's own rows and the gathered neighbour rows into registers.
// Shape 1 stages them in shared memory with cp.async (16-byte asynchronous global->shared
// copies, one per lane and row vector, plus the row's ELL values and per-row scalars), in a
// ring of `stages` buffers per row group: while a group computes row t, the copies of rows
// t+1 .. t+stages-1 are in flight, so a warp never waits for a load it issued in the same
// iteration.  Every lane consumes only the vectors it copied itself (its 16-byte column
// slice of each row); the ELL values and scalars of a row are copied by a few lanes of the
// group and read by all of them after cp.async.wait_group and __syncwarp.  The waits are
// hardware waits on the thread's own copies (no spinning on memory).
#include <type_traits>

#include "sparse_common.cuh"

namespace alm {

// ---------------------------------------------------------------------------------------
// shape 0: rows in registers
// ---------------------------------------------------------------------------------------
// Inner-loop SpMM with the pending step and the slack update fused in (ELL form, diagonal-
// selector problems).  R_in is the factor before the step and stays unmodified: the group's
// own row becomes r_i' = r_i + alpha d_i (written to R_out, a different buffer), S_ii is
// formed from |r_i'|^2 in float-pair arithmetic as in k_inner_slack (and stored for the
// line search), the neighbours' rows are formed on the fly as r_j + alpha d_j from R_in and
// D.  Then G = 2 S R', Z = P^{-1} G and the CG inner products, as in k_spmm_ell (MODE 1).
template <typename T, int LANES, int KF>
__global__ void __launch_bounds__(kBlock, 3) k_spmm_ell_step(SparseView<T> v, const T *__restrict__ Rin,
                                                          T *__restrict__ Rout, int r, int ldr, T *G, const T *D,
                                                          DevState *st, double *partials, const int *done) {
    if (*done) return;
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    __shared__ double shm[32];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LANES - 1);
    const unsigned gmask = group_mask<LANES>(lane);
    const int gpb = kBlock / LANES;
    const int64_t ng = int64_t(gridDim.x) * gpb;
    const bool active = gl * W < r;
    const bool writer = gl * W < ldr;
    const bool pc = st->precond;
    const T sig = T(st->sigma);
    const T pc_floor = T(st->pc_floor);
    const T alpha = T(st->alpha);
    const bool step = alpha != T(0);
    T pgg = T(0), pgo = T(0), pgd = T(0), pzg = T(0);
    int jc[KF];
    T sc[KF];
    int64_t i = int64_t(blockIdx.x) * gpb + threadIdx.x / LANES;
    if (i < v.n) ell_fetch<T, KF>(v.f_ell_col, v.f_ell_val, i, jc, sc);
    for (; i < v.n; i += ng) {
        const int64_t inext = i + ng;
        int jn[KF];
        T sn[KF];
        if (inext < v.n) ell_fetch<T, KF>(v.f_ell_col, v.f_ell_val, inext, jn, sn);
        V ri = load_row(Rin, i, ldr, gl, active);
        const V dold = active ? ld(D + i * ldr + gl * W) : vzero(T());
        const V gold = active ? ld(G + i * ldr + gl * W) : vzero(T());
        V gth[KF];
#pragma unroll
        for (int k = 0; k < KF; ++k) gth[k] = load_row(Rin, jc[k], ldr, gl, active);
        if (step) {
#pragma unroll
            for (int k = 0; k < KF; ++k) gth[k] = fma4(alpha, load_row(D, jc[k], ldr, gl, active), gth[k]);
            ri = fma4(alpha, dold, ri);
        }
        ri = mask_tail(ri, gl * W, r);
        if (writer) stv(Rout + i * ldr + gl * W, ri);
        T xh, xl;
        norm2_pair(ri, gmask, LANES, xh, xl);
        T dsi, dlo;
        slack_pair<T>(v, i, xh, xl, sig, dsi, dlo);
        if (gl == 0) {
            v.d_s[i] = dsi;
            if (v.d_s_lo) v.d_s_lo[i] = dlo;
            if (v.ls_rec) v.ls_rec[i].ds = dsi;
        }
        using Acc = typename AccOf<T>::type;
        Acc acc;
        acc.init();
        acc.add(dsi, ri);
        acc.add_lo(dlo, ri);
#pragma unroll
        for (int k = 0; k < KF; ++k) acc.add(sc[k], gth[k]);
        const V g = mask_tail(scale4(T(2), acc.value()), gl * W, r);
        pgg += dot(g, g);
        V z = g;
        if (pc) {
            const T rg = group_sum<LANES>(dot(ri, g), gmask);
            const T rr = xh + xl;
            T sdi = dsi + dlo;
            sdi = sdi > pc_floor ? sdi : pc_floor;
            const int k = v.d_sel_k[i];
            const T a = k >= 0 ? T(v.d_sel_a[i]) : T(0);
            const T ka = T(4) * sig * a * a;
            const T coef = ka * rg / (T(2) * sdi + ka * rr);
            z = scale4(T(1) / (T(2) * sdi), fma4(-coef, ri, g));
        }
        pzg += dot(z, g);
        pgo += dot(g, gold);
        pgd += dot(g, dold);
        if (writer) stv(G + i * ldr + gl * W, z);
#pragma unroll
        for (int k = 0; k < KF; ++k) {
            jc[k] = jn[k];
            sc[k] = sn[k];
        }
    }
    double *part = partials + size_t(blockIdx.x) * kPartStride;
    const double vals[4] = {double(pgg), double(pgo), double(pgd), double(pzg)};
    block_partials<4>(vals, part, shm);
    if (!last_block(&st->counter[CNT_SPMM])) return;
    double tot[4];
    sum_partials_n<4>(partials, tot, shm);
    if (threadIdx.x == 0) {
        spmm_finish(st, tot[0], tot[1], tot[2], tot[3]);
        st->k1count += 1;
    }
}

// Inner-loop (MODE 1) line search with the CG direction fused in, for the ELL form:
//   D_new = -Z + beta D_old   (written for the group's own row; the upper neighbours'
//                              directions are formed on the fly from Z and D_old)
// then the quartic of the exact step along D_new.  In the inner loop q1 comes from the
// SpMM's inner products, so only <S, D D^T> and the diagonal selector terms a1 = 2 r_i.d_i,
// a2 = |d_i|^2 are needed: no R row is gathered.  D_old and D_new are different buffers.
template <typename T, int LANES, int KU>
__global__ void __launch_bounds__(kBlock, 4) k_ls_ell_dir(SparseView<T> v, const T *__restrict__ R,
                                                       const T *__restrict__ Z, const T *__restrict__ Dold,
                                                       T *__restrict__ Dnew, int r, int ldr, DevState *st,
                                                       double *partials, const int *done) {
    if (*done) return;
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    __shared__ double shm[32];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LANES - 1);
    const unsigned gmask = group_mask<LANES>(lane);
    const int gpb = kBlock / LANES;
    const int64_t ng = int64_t(gridDim.x) * gpb;
    const bool active = gl * W < r;
    const bool writer = gl * W < ldr;
    const T beta = T(st->beta);
    const bool use_old = beta != T(0);  // D_old may hold stale values when beta = 0
    T p2 = T(0), p11 = T(0), p12 = T(0), p22 = T(0);
    int jc[KU];
    T sc[KU];
    auto fetch = [&](int64_t row, int (&jj)[KU], T (&ss)[KU]) {
        if constexpr (KU == 2) ell_fetch2<T, KU>(v.u_ell_col, v.u_ell_val, row, jj, ss);
        else ell_fetch<T, KU>(v.u_ell_col, v.u_ell_val, row, jj, ss);
    };
    auto dir_of = [&](V z, V d) { return fma4(beta, use_old ? d : vzero(T()), scale4(T(-1), z)); };
    int64_t i = int64_t(blockIdx.x) * gpb + threadIdx.x / LANES;
    if (i < v.n) fetch(i, jc, sc);
    for (; i < v.n; i += ng) {
        const V ri = mask_tail(load_row(R, i, ldr, gl, active), gl * W, r);
        const V zi = load_row(Z, i, ldr, gl, active);
        const V doi = use_old ? load_row(Dold, i, ldr, gl, active) : vzero(T());
        V zj[KU], dj[KU];
#pragma unroll
        for (int k = 0; k < KU; ++k) {
            zj[k] = load_row(Z, jc[k], ldr, gl, active);
            dj[k] = use_old ? load_row(Dold, jc[k], ldr, gl, active) : vzero(T());
        }
        T sq[KU];
#pragma unroll
        for (int k = 0; k < KU; ++k) sq[k] = T(2) * sc[k];
        if (i + ng < v.n) fetch(i + ng, jc, sc);
        const V di = mask_tail(dir_of(zi, doi), gl * W, r);
        if (writer) stv(Dnew + i * ldr + gl * W, di);
        const T rdi = dot(ri, di), ddi = dot(di, di);
        T l2 = v.d_s[i] * ddi;
#pragma unroll
        for (int k = 0; k < KU; ++k) l2 += sq[k] * dot(di, dir_of(zj[k], dj[k]));
        p2 += l2;
        const int ksel = v.d_sel_k[i];
        if (ksel >= 0) {  // group-uniform
            const T a1 = T(2) * group_sum<LANES>(rdi, gmask);
            const T a2 = group_sum<LANES>(ddi, gmask);
            if (gl == 0) {
                const T a = T(v.d_sel_a[i]);
                const T A1 = a * a1, A2 = a * a2;
                p11 += A1 * A1;
                p12 += A1 * A2;
                p22 += A2 * A2;
            }
        }
    }
    const double vals[5] = {0.0, double(p2), double(p11), double(p12), double(p22)};
    block_partials<5>(vals, partials + size_t(blockIdx.x) * kPartStride, shm);
    if (!last_block(&st->counter[CNT_LS])) return;
    double tot[5];
    sum_partials_n<5>(partials, tot, shm);
    if (threadIdx.x == 0) ls_finish<T, 1, false>(v, st, r, tot);
}


// ---------------------------------------------------------------------------------------
// shape 1: rows staged by cp.async
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// 16-byte copy that bypasses L1 (streams read once)
__device__ __forceinline__ void cpa16_cg(void *s, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
// 16-byte copy cached in L1 (gathered rows: neighbours of nearby rows hit L1)
__device__ __forceinline__ void cpa16_ca(void *s, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cpa8(void *s, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cpa4(void *s, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
// the K column indices of an ELL row into registers (K = 2: one 8-byte load; K >= 4: 16-byte loads)
template <int K>
__device__ __forceinline__ void ell_cols(const int *__restrict__ cols, int64_t row, int (&jj)[K]) {
    if constexpr (K == 2) {
        const int2 c = __ldg(reinterpret_cast<const int2 *>(cols + row * K));
        jj[0] = c.x;
        jj[1] = c.y;
    } else {
        const int4 *cp = reinterpret_cast<const int4 *>(cols + row * K);
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const int4 c = __ldg(cp + q);
            jj[4 * q] = c.x;
            jj[4 * q + 1] = c.y;
            jj[4 * q + 2] = c.z;
            jj[4 * q + 3] = c.w;
        }
    }
}
template <int BYTES>
__device__ __forceinline__ void cpa_scalar(void *s, const void *g) {
    if constexpr (BYTES == 8) cpa8(s, g);
    else cpa4(s, g);
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most `pending` of this thread's committed groups are still in flight
__device__ __forceinline__ void cpa_wait(int pending) {
    if (pending <= 0) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    else if (pending == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else if (pending == 2) asm volatile("cp.async.wait_group 2;\n" ::: "memory");
    else asm volatile("cp.async.wait_group 3;\n" ::: "memory");
}

// Shape-1 work decomposition: a group of LANES lanes owns a row (lane gl holds the 16-byte
// vector of columns [gl W, gl W + W)), NT threads per CTA, the row groups of the grid walk
// the rows with stride (grid x NT / LANES).  Shared memory per stage: SLOTS row vectors per
// thread ([stage][slot][thread], consecutive threads on consecutive 16-byte words), then
// one block of per-row data (ELL values and the row's record) per row group.

// Error-free accumulation against a power-of-two bias (the extraction step of Rump, Ogita and
// Oishi, "Accurate floating-point summation", SIAM J. Sci. Comput. 31, 2008).  `sg` starts at
// bias = 1.5 * 2^e with 2^e above twice every partial sum, so sg stays in (2^e, 2^(e+1)).  One
// FMA rounds the exact sum sg + c x; q = s - sg is then exact (Sterbenz: s and sg lie within a
// factor of two) and c x - q, the part of c x that the rounding dropped, is exact when c x is
// a float (c a power of two) and otherwise off by 2^-24 of a unit in the last place of sg:
// it goes to `lo`.  Four operations per term, the product included, against eight to ten for a
// product error plus a two-sum.  If a bound is exceeded the sum loses only the exactness of
// that step (plain FP32 rounding).
__device__ __forceinline__ void ext_fma(float &sg, float &lo, float c, float x) {
    const float s = fmaf(c, x, sg);
    const float q = s - sg;
    lo += fmaf(c, x, -q);
    sg = s;
}
// 1.5 * 2^e with 2^e the power of two just above 2 b (b >= 0), capped below the overflow range
__device__ __forceinline__ float ext_bias(float b) {
    unsigned u = __float_as_uint(2.f * b) & 0x7f800000u;
    u = u < 0x7e000000u ? u : 0x7e000000u;
    return __uint_as_float(u + 0x00c00000u);
}
// c x accumulated into (sg, lo) per component
__device__ __forceinline__ void ext_term(float (&sg)[4], float (&lo)[4], float c, float4 x) {
    ext_fma(sg[0], lo[0], c, x.x);
    ext_fma(sg[1], lo[1], c, x.y);
    ext_fma(sg[2], lo[2], c, x.z);
    ext_fma(sg[3], lo[3], c, x.w);
}

template <int KF>
constexpr int step_aux_bytes() { return KF * 4 + int(sizeof(StepRec)); }  // ELL values, record
template <int KF>
constexpr int step_slots() { return 3 + 2 * KF; }  // own R, D, Z_old; gathered R_j, D_j

// Fused step + SpMM (FP32 form; see the file comment), shape 1.  FULL: every lane of a row
// group holds live columns (r = LANES W = ldr) and every element offset fits in 32 bits, so
// the lane predicates, the tail masks and the 64-bit offsets drop out.
template <int LANES, int KF, int NT, bool FULL>
__global__ void __launch_bounds__(NT, 512 / NT) k_spmm_step_pipe(SparseView<float> v, const float *__restrict__ Rin,
                                                                float *__restrict__ Rout, int r, int ldr, float *G,
                                                                const float *D, int stages, DevState *st,
                                                                double *partials, const int *done) {
    if (*done) return;
    constexpr int W = 4;
    constexpr int SLOTS = step_slots<KF>();
    constexpr int AUXB = step_aux_bytes<KF>();
    constexpr int NAUX = AUXB / 16;  // 16-byte copies of a row's per-row data
    constexpr int GPB = NT / LANES;
    static_assert(NAUX <= LANES, "a row's per-row data is copied by one lane per 16 bytes");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double shm[32];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int gl = lane & (LANES - 1);
    const unsigned gmask = group_mask<LANES>(lane);
    const int grp = tid / LANES;
    const int64_t ng = int64_t(gridDim.x) * GPB;
    const int col = gl * W;
    const bool active = FULL || col < r;
    const bool writer = FULL || col < ldr;
    const bool pc = st->precond;
    const float sig = float(st->sigma);
    const float pc_floor = float(st->pc_floor);
    const float alpha = float(st->alpha);
    const bool step = alpha != 0.f;
    // bound xc on the entries of the rows for the extraction bias of G: twice the largest row
    // norm of the previous step within an inner solve, 8 at its first step (so that the sums
    // depend on the iterate alone)
    const float xc = sqrtf(st->xcap2 > 0.f ? st->xcap2 : 64.f);
    float rmax2 = 0.f;
    float4 *vec = reinterpret_cast<float4 *>(smem) + tid;
    unsigned char *auxg = smem + size_t(stages) * SLOTS * NT * 16 + size_t(grp) * AUXB;
    const size_t aux_stage = size_t(GPB) * AUXB;
    // row index arithmetic in 32 bits when every element offset fits
    const bool idx32 = FULL || int64_t(v.n) * ldr < (int64_t(1) << 31);
    auto off = [&](int64_t row) -> int64_t {
        return idx32 ? int64_t(unsigned(row) * unsigned(ldr) + unsigned(col)) : row * ldr + col;
    };
    const int64_t row0 = int64_t(blockIdx.x) * GPB + grp;
    const int64_t wrow0 = int64_t(blockIdx.x) * GPB + (tid >> 5) * (32 / LANES);
    int jn[KF];  // column indices of the next row to issue, loaded one iteration ahead
    auto fetch_cols = [&](int64_t row) {
        if (row < v.n) ell_cols<KF>(v.f_ell_col, row, jn);
    };
    auto issue = [&](int64_t row, int s) {
        if (row >= v.n) return;
        float4 *sl = vec + size_t(s) * SLOTS * NT;
        if (active) {
            const int64_t o = off(row);
            cpa16_cg(sl, Rin + o);
            cpa16_cg(sl + NT, D + o);
            cpa16_cg(sl + 2 * NT, G + o);
#pragma unroll
            for (int k = 0; k < KF; ++k) {
                const int64_t oj = off(jn[k]);
                cpa16_ca(sl + (3 + k) * NT, Rin + oj);
                if (step) cpa16_ca(sl + (3 + KF + k) * NT, D + oj);
            }
        }
        if (gl < NAUX) {
            unsigned char *a = auxg + size_t(s) * aux_stage + 16 * gl;
            const unsigned char *src =
                gl < KF / 4 ? reinterpret_cast<const unsigned char *>(v.f_ell_val + row * KF) + 16 * gl
                            : reinterpret_cast<const unsigned char *>(v.step_rec + row) + 16 * (gl - KF / 4);
            cpa16_ca(a, src);
        }
    };
    float pgg = 0.f, pgo = 0.f, pgd = 0.f, pzg = 0.f;
    for (int s = 0; s < stages - 1; ++s) {
        fetch_cols(row0 + s * ng);
        issue(row0 + s * ng, s);
        cpa_commit();
    }
    fetch_cols(row0 + int64_t(stages - 1) * ng);
    int s_cur = 0;
    for (int64_t t = 0; wrow0 + t * ng < v.n; ++t) {
        const int64_t i = row0 + t * ng;
        // refill the buffer of the row computed in the previous iteration
        __syncwarp();
        int s_new = s_cur + stages - 1;
        if (s_new >= stages) s_new -= stages;
        issue(i + int64_t(stages - 1) * ng, s_new);
        cpa_commit();
        fetch_cols(i + int64_t(stages) * ng);
        cpa_wait(stages - 1);
        __syncwarp();
        if (i < v.n) {
            const float4 *sl = vec + size_t(s_cur) * SLOTS * NT;
            const unsigned char *a = auxg + size_t(s_cur) * aux_stage;
            const float *sv = reinterpret_cast<const float *>(a);
            const StepRec sa = *reinterpret_cast<const StepRec *>(a + KF * 4);
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            const int64_t oi = off(i);
            float4 ri = active ? sl[0] : zero;
            const float4 dold = active ? sl[NT] : zero;
            const float4 gold = active ? sl[2 * NT] : zero;
            if (step) ri = fma4(alpha, dold, ri);
            if (!FULL) ri = mask_tail(ri, col, r);
            if (writer) stv(Rout + oi, ri);
            float xh, xl;
            norm2_pair(ri, gmask, LANES, xh, xl);
            rmax2 = fmaxf(rmax2, xh + xl);
            // S_ii = base_i + sigma a_i (a_i |r_i'|^2 - b_k) in float pairs (as slack_pair)
            float dsi = sa.base_hi, dlo = sa.base_lo;
            if (sa.k >= 0) {
                const float aa = sa.af;
                const float ph = aa * xh;
                const float pe = fmaf(aa, xh, -ph) + aa * xl;
                const float s0 = ph - sa.b_hi;
                const float bb = s0 - ph;
                const float e0 = (ph - (s0 - bb)) + (-sa.b_hi - bb);
                const float res = s0 + (e0 + pe - sa.b_lo);
                const float corr = sig * aa * res;
                const float s1 = dsi + corr;
                const float b1 = s1 - dsi;
                dlo += (dsi - (s1 - b1)) + (corr - b1);
                dsi = s1;
            }
            if (gl == 0) {
                v.d_s[i] = dsi;
                v.d_s_lo[i] = dlo;
                if (v.ls_rec) v.ls_rec[i].ds = dsi;
            }
            // G = 2 (S_ii r_i' + sum_j C_ij r_j'): every partial sum is below (|S_ii| + rabs_i) xc
            const float gb = ext_bias((fabsf(dsi) + sa.rabs) * xc);
            float sg[4] = {gb, gb, gb, gb}, lo[4] = {0.f, 0.f, 0.f, 0.f};
            ext_term(sg, lo, dsi, ri);
            lo[0] = fmaf(dlo, ri.x, lo[0]);
            lo[1] = fmaf(dlo, ri.y, lo[1]);
            lo[2] = fmaf(dlo, ri.z, lo[2]);
            lo[3] = fmaf(dlo, ri.w, lo[3]);
#pragma unroll
            for (int k = 0; k < KF; ++k) {
                float4 x = active ? sl[(3 + k) * NT] : zero;
                if (step && active) x = fma4(alpha, sl[(3 + KF + k) * NT], x);
                ext_term(sg, lo, sv[k], x);
            }
            float4 g = make_float4(2.f * ((sg[0] - gb) + lo[0]), 2.f * ((sg[1] - gb) + lo[1]),
                                   2.f * ((sg[2] - gb) + lo[2]), 2.f * ((sg[3] - gb) + lo[3]));
            if (!FULL) g = mask_tail(g, col, r);
            pgg += dot(g, g);
            float4 z = g;
            if (pc) {
                const float rg = group_sum<LANES>(dot(ri, g), gmask);
                const float rr = xh + xl;
                float sdi = dsi + dlo;
                sdi = sdi > pc_floor ? sdi : pc_floor;
                const float aa = sa.k >= 0 ? sa.af : 0.f;
                const float ka = 4.f * sig * aa * aa;
                // the preconditioner needs no correctly rounded division
                const float coef = __fdividef(ka * rg, 2.f * sdi + ka * rr);
                z = scale4(__fdividef(1.f, 2.f * sdi), fma4(-coef, ri, g));
            }
            pzg += dot(z, g);
            pgo += dot(g, gold);
            pgd += dot(g, dold);
            if (writer) stv(G + oi, z);
        }
        s_cur = s_cur + 1 == stages ? 0 : s_cur + 1;
    }
    cpa_wait(0);
    // the launch's maximum of |r_i'|^2 (non-negative floats order as their bits)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax2 = fmaxf(rmax2, __shfl_xor_sync(0xffffffffu, rmax2, o));
    if (lane == 0) atomicMax(&st->rmax2_bits, __float_as_uint(rmax2));
    double *part = partials + size_t(blockIdx.x) * kPartStride;
    const double vals[4] = {double(pgg), double(pgo), double(pgd), double(pzg)};
    block_partials<4>(vals, part, shm);
    if (!last_block(&st->counter[CNT_SPMM])) return;
    double tot[4];
    sum_partials_n<4>(partials, tot, shm);
    if (threadIdx.x == 0) {
        spmm_finish(st, tot[0], tot[1], tot[2], tot[3]);
        st->k1count += 1;
        const float m = __uint_as_float(atomicExch(&st->rmax2_bits, 0u));
        st->xcap2 = (m == m && m < 1e30f) ? fmaxf(4.f * m, 1e-30f) : 0.f;
    }
}

// per-row data block of the line-search kernel: the upper ELL values (padded to 16 bytes),
// then the row's record (selector and S_ii)
template <typename T, int KU>
constexpr int ls_val_bytes() { return (KU * int(sizeof(T)) + 15) / 16 * 16; }
template <typename T, int KU>
constexpr int ls_aux_bytes() { return ls_val_bytes<T, KU>() + int(sizeof(LsRec<T>)); }
template <int KU>
constexpr int ls_slots() { return 3 + 2 * KU; }  // own R', Z, D_old; gathered Z_j, D_old_j

// Fused direction + line search (see the file comment), shape 1.  FULL as for the step kernel.
template <typename T, int LANES, int KU, int NT, bool FULL>
__global__ void __launch_bounds__(NT, 512 / NT) k_ls_dir_pipe(SparseView<T> v, const T *__restrict__ R,
                                                             const T *__restrict__ Z, const T *__restrict__ Dold,
                                                             T *__restrict__ Dnew, int r, int ldr, int stages,
                                                             DevState *st, double *partials, const int *done) {
    if (*done) return;
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    constexpr int SLOTS = ls_slots<KU>();
    constexpr int VB = KU * int(sizeof(T));  // bytes of a row's upper ELL values
    constexpr int VBP = ls_val_bytes<T, KU>();
    constexpr int AUXB = ls_aux_bytes<T, KU>();
    constexpr int NVAL = VBP / 16;
    constexpr int NITEM = NVAL + int(sizeof(LsRec<T>)) / 16;  // 16-byte copies (one 8-byte when VB = 8)
    constexpr int GPB = NT / LANES;
    static_assert(NITEM <= LANES, "a row's per-row data is copied by one lane per 16 bytes");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double shm[32];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int gl = lane & (LANES - 1);
    const unsigned gmask = group_mask<LANES>(lane);
    const int grp = tid / LANES;
    const int64_t ng = int64_t(gridDim.x) * GPB;
    const int col = gl * W;
    const bool active = FULL || col < r;
    const bool writer = FULL || col < ldr;
    const T beta = T(st->beta);
    const bool use_old = beta != T(0);  // D_old may hold stale values when beta = 0
    V *vec = reinterpret_cast<V *>(smem) + tid;
    unsigned char *auxg = smem + size_t(stages) * SLOTS * NT * 16 + size_t(grp) * AUXB;
    const size_t aux_stage = size_t(GPB) * AUXB;
    const bool idx32 = FULL || int64_t(v.n) * ldr < (int64_t(1) << 31);
    auto off = [&](int64_t row) -> int64_t {
        return idx32 ? int64_t(unsigned(row) * unsigned(ldr) + unsigned(col)) : row * ldr + col;
    };
    const int64_t row0 = int64_t(blockIdx.x) * GPB + grp;
    const int64_t wrow0 = int64_t(blockIdx.x) * GPB + (tid >> 5) * (32 / LANES);
    int jn[KU];
    auto fetch_cols = [&](int64_t row) {
        if (row < v.n) ell_cols<KU>(v.un_col, row, jn);
    };
    // per-row data: lanes 0..NVAL-1 the ELL values (one 8-byte copy when VB = 8), the next
    // lanes the record
    auto issue = [&](int64_t row, int s) {
        if (row >= v.n) return;
        V *sl = vec + size_t(s) * SLOTS * NT;
        if (active) {
            const int64_t o = off(row);
            cpa16_cg(sl, R + o);
            cpa16_cg(sl + NT, Z + o);
            if (use_old) cpa16_cg(sl + 2 * NT, Dold + o);
#pragma unroll
            for (int k = 0; k < KU; ++k) {
                const int64_t oj = off(jn[k]);
                cpa16_ca(sl + (3 + k) * NT, Z + oj);
                if (use_old) cpa16_ca(sl + (3 + KU + k) * NT, Dold + oj);
            }
        }
        unsigned char *a = auxg + size_t(s) * aux_stage;
        if (gl < NITEM) {
            if (VB >= 16 || gl >= NVAL) {
                const unsigned char *src =
                    gl < NVAL ? reinterpret_cast<const unsigned char *>(v.un_val + row * KU) + 16 * gl
                              : reinterpret_cast<const unsigned char *>(v.ls_rec + row) + 16 * (gl - NVAL);
                cpa16_ca(a + 16 * gl, src);
            } else {
                cpa8(a, v.un_val + row * KU);
            }
        }
    };
    auto dir_of = [&](V z, V d) { return fma4(beta, use_old ? d : vzero(T()), scale4(T(-1), z)); };
    T p2 = T(0), p11 = T(0), p12 = T(0), p22 = T(0);
    for (int s = 0; s < stages - 1; ++s) {
        fetch_cols(row0 + s * ng);
        issue(row0 + s * ng, s);
        cpa_commit();
    }
    fetch_cols(row0 + int64_t(stages - 1) * ng);
    int s_cur = 0;
    for (int64_t t = 0; wrow0 + t * ng < v.n; ++t) {
        const int64_t i = row0 + t * ng;
        __syncwarp();
        int s_new = s_cur + stages - 1;
        if (s_new >= stages) s_new -= stages;
        issue(i + int64_t(stages - 1) * ng, s_new);
        cpa_commit();
        fetch_cols(i + int64_t(stages) * ng);
        cpa_wait(stages - 1);
        __syncwarp();
        if (i < v.n) {
            const V *sl = vec + size_t(s_cur) * SLOTS * NT;
            const unsigned char *a = auxg + size_t(s_cur) * aux_stage;
            const T *sv = reinterpret_cast<const T *>(a);
            const LsRec<T> rec = *reinterpret_cast<const LsRec<T> *>(a + VBP);
            const T ds = rec.ds;
            V ri = active ? sl[0] : vzero(T());
            if (!FULL) ri = mask_tail(ri, col, r);
            const V zi = active ? sl[NT] : vzero(T());
            const V doi = (active && use_old) ? sl[2 * NT] : vzero(T());
            V di = dir_of(zi, doi);
            if (!FULL) di = mask_tail(di, col, r);
            if (writer) stv(Dnew + off(i), di);
            const T rdi = dot(ri, di), ddi = dot(di, di);
            T l2 = ds * ddi;
#pragma unroll
            for (int k = 0; k < KU; ++k) {
                const V zj = active ? sl[(3 + k) * NT] : vzero(T());
                const V dj = (active && use_old) ? sl[(3 + KU + k) * NT] : vzero(T());
                l2 += T(2) * sv[k] * dot(di, dir_of(zj, dj));
            }
            p2 += l2;
            if (rec.k >= 0) {  // group-uniform
                const T a1 = T(2) * group_sum<LANES>(rdi, gmask);
                const T a2 = group_sum<LANES>(ddi, gmask);
                if (gl == 0) {
                    const T aa = rec.a;
                    const T A1 = aa * a1, A2 = aa * a2;
                    p11 += A1 * A1;
                    p12 += A1 * A2;
                    p22 += A2 * A2;
                }
            }
        }
        s_cur = s_cur + 1 == stages ? 0 : s_cur + 1;
    }
    cpa_wait(0);
    // entries of rows longer than the narrow ELL: 2 s_ij d_i . d_j, one entry per row group
    for (int64_t e = int64_t(blockIdx.x) * GPB + grp; e < v.n_ov; e += ng) {
        if (!active) continue;
        const int64_t oi = off(v.ov_i[e]), oj = off(v.ov_j[e]);
        V di = dir_of(ldro(Z + oi), use_old ? ldro(Dold + oi) : vzero(T()));
        if (!FULL) di = mask_tail(di, col, r);
        const V dj = dir_of(ldro(Z + oj), use_old ? ldro(Dold + oj) : vzero(T()));
        p2 += T(2) * v.ov_v[e] * dot(di, dj);
    }
    const double vals[5] = {0.0, double(p2), double(p11), double(p12), double(p22)};
    block_partials<5>(vals, partials + size_t(blockIdx.x) * kPartStride, shm);
    if (!last_block(&st->counter[CNT_LS])) return;
    double tot[5];
    sum_partials_n<5>(partials, tot, shm);
    if (threadIdx.x == 0) ls_finish<T, 1, false>(v, st, r, tot);
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------
// resident CTAs per SM of a shape-1 kernel at a launch shape (cached).  The kernel's dynamic
// shared memory limit is raised once to the device maximum, so that every shape (and every
// graph captured with one) stays launchable.
template <typename K>
static int pipe_resident(K *fn, int threads, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<const void *, std::unordered_map<size_t, int>> cache;
    std::lock_guard<std::mutex> lk(mu);
    const void *key = reinterpret_cast<const void *>(fn);
    auto &per = cache[key];
    if (per.empty()) {
        int dev = 0, maxsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm - 1024) != cudaSuccess)
            (void)cudaGetLastError();
        per[0] = maxsm - 1024;  // the dynamic limit that was set
    }
    const size_t tag = (smem << 12) | size_t(threads);
    auto it = per.find(tag);
    if (it != per.end()) return it->second;
    int b = 0;
    if (smem > size_t(per[0]) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem) != cudaSuccess || b < 1) {
        (void)cudaGetLastError();
        b = 0;
    }
    per[tag] = b;
    return b;
}

static size_t step_pipe_smem(int kf, int stages, int threads, int lanes) {
    const int aux = kf == 4 ? step_aux_bytes<4>() : step_aux_bytes<8>();
    return size_t(stages) * (size_t(3 + 2 * kf) * threads * 16 + size_t(threads / lanes) * aux);
}
template <typename T>
static size_t ls_pipe_smem(int ku, int stages, int threads, int lanes) {
    const int aux = ku == 2 ? ls_aux_bytes<T, 2>() : ku == 4 ? ls_aux_bytes<T, 4>() : ls_aux_bytes<T, 8>();
    return size_t(stages) * (size_t(3 + 2 * ku) * threads * 16 + size_t(threads / lanes) * aux);
}

// Shape 1 covers ELL widths up to 8 and ranks of at least 16 columns' worth of 16-byte
// vectors per row group (4 lanes in FP32, 8 in FP64); other cases use shape 0.
static bool pipe_ok(const LaunchCtx &c, int width, int lanes, int min_lanes) {
    return c.icfg.variant == 1 && width <= 8 && c.icfg.stages >= 2 && c.icfg.stages <= 4 &&
           (c.icfg.threads == 128 || c.icfg.threads == 256) && lanes >= min_lanes;
}

template <typename K>
static bool pipe_launch_grid(const LaunchCtx &c, K *fn, int th, size_t smem, int64_t n, int lanes, int &grid) {
    const int b = pipe_resident(fn, th, smem);
    if (b < 1) return false;
    const int64_t need = (n + th / lanes - 1) / (th / lanes);
    const int64_t g = std::min<int64_t>(need, int64_t(c.sms) * b);
    grid = int(std::max<int64_t>(1, std::min<int64_t>(g, c.grid)));
    return true;
}

// FULL launches: r fills the row groups (r = LANES W = ldr) and n ldr < 2^31
static bool full_shape(int64_t n, int r, int ldr, int lanes, int W) {
    return r == lanes * W && ldr == r && n * ldr < (int64_t(1) << 31);
}

template <int LN, int KF, int NT, bool FULL>
static bool spmm_step_pipe_one(const LaunchCtx &c, const SparseView<float> &v, const float *Rin, float *Rout, int r,
                               int ldr, float *G, const float *D, const int *done) {
    auto *fn = k_spmm_step_pipe<LN, KF, NT, FULL>;
    const size_t smem = step_pipe_smem(KF, c.icfg.stages, NT, LN);
    int grid = 0;
    if (!pipe_launch_grid(c, fn, NT, smem, v.n, LN, grid)) return false;
    fn<<<grid, NT, smem, c.stream>>>(v, Rin, Rout, r, ldr, G, D, c.icfg.stages, c.st, c.partials, done);
    return true;
}

template <int LN, int KF>
static bool spmm_step_pipe_nt(const LaunchCtx &c, const SparseView<float> &v, const float *Rin, float *Rout, int r,
                              int ldr, float *G, const float *D, const int *done) {
    if constexpr (LN == 8) {
        if (full_shape(v.n, r, ldr, LN, 4)) {
            if (c.icfg.threads == 128) return spmm_step_pipe_one<LN, KF, 128, true>(c, v, Rin, Rout, r, ldr, G, D, done);
            return spmm_step_pipe_one<LN, KF, 256, true>(c, v, Rin, Rout, r, ldr, G, D, done);
        }
    }
    if (c.icfg.threads == 128) return spmm_step_pipe_one<LN, KF, 128, false>(c, v, Rin, Rout, r, ldr, G, D, done);
    return spmm_step_pipe_one<LN, KF, 256, false>(c, v, Rin, Rout, r, ldr, G, D, done);
}

template <typename T, int LN, int KU, int NT, bool FULL>
static bool ls_dir_pipe_one(const LaunchCtx &c, const SparseView<T> &v, const T *R, const T *Z, const T *Dold,
                            T *Dnew, int r, int ldr, const int *done) {
    auto *fn = k_ls_dir_pipe<T, LN, KU, NT, FULL>;
    const size_t smem = ls_pipe_smem<T>(KU, c.icfg.stages, NT, LN);
    int grid = 0;
    if (!pipe_launch_grid(c, fn, NT, smem, v.n, LN, grid)) return false;
    fn<<<grid, NT, smem, c.stream>>>(v, R, Z, Dold, Dnew, r, ldr, c.icfg.stages, c.st, c.partials, done);
    return true;
}

template <typename T, int LN, int KU>
static bool ls_dir_pipe_nt(const LaunchCtx &c, const SparseView<T> &v, const T *R, const T *Z, const T *Dold, T *Dnew,
                           int r, int ldr, const int *done) {
    constexpr int W = VecT<T>::W;
    if constexpr (LN * W == 32) {
        if (full_shape(v.n, r, ldr, LN, W)) {
            if (c.icfg.threads == 128)
                return ls_dir_pipe_one<T, LN, KU, 128, true>(c, v, R, Z, Dold, Dnew, r, ldr, done);
            return ls_dir_pipe_one<T, LN, KU, 256, true>(c, v, R, Z, Dold, Dnew, r, ldr, done);
        }
    }
    if (c.icfg.threads == 128) return ls_dir_pipe_one<T, LN, KU, 128, false>(c, v, R, Z, Dold, Dnew, r, ldr, done);
    return ls_dir_pipe_one<T, LN, KU, 256, false>(c, v, R, Z, Dold, Dnew, r, ldr, done);
}

template <typename T, int LN, int KF>
static void spmm_step_one(const LaunchCtx &c, const SparseView<T> &v, const T *Rin, T *Rout, int r, int ldr, T *G,
                          const T *D, const int *done) {
    auto *fn = k_spmm_ell_step<T, LN, KF>;
    fn<<<grid_for(c, fn, v.n, kBlock / LN), kBlock, 0, c.stream>>>(v, Rin, Rout, r, ldr, G, D, c.st, c.partials, done);
}

template <typename T, int LN, int KU>
static void ls_ell_dir_one(const LaunchCtx &c, const SparseView<T> &v, const T *R, const T *Z, const T *Dold, T *Dnew,
                           int r, int ldr, const int *done) {
    auto *fn = k_ls_ell_dir<T, LN, KU>;
    fn<<<grid_for(c, fn, v.n, kBlock / LN), kBlock, 0, c.stream>>>(v, R, Z, Dold, Dnew, r, ldr, c.st, c.partials,
                                                                      done);
}

template <typename T>
bool spmm_step_fusable(const SparseView<T> &v) {
    return v.ell_kf > 0 && v.lr_k == 0 && v.fused_dual && v.d_s_lo != nullptr;
}

template <typename T>
void launch_spmm_step(const LaunchCtx &c, const SparseView<T> &v, const T *Rin, T *Rout, int r, int ldr, T *G,
                      const T *D, const int *done) {
    constexpr int W = VecT<T>::W;
    if constexpr (sizeof(T) == 4) {
        const int L = lanes_for(r, W);
        if (pipe_ok(c, v.ell_kf, L, 4) && v.step_rec) {
            const bool ok = L == 4 ? (v.ell_kf == 4 ? spmm_step_pipe_nt<4, 4>(c, v, Rin, Rout, r, ldr, G, D, done)
                                                    : spmm_step_pipe_nt<4, 8>(c, v, Rin, Rout, r, ldr, G, D, done))
                                   : (v.ell_kf == 4 ? spmm_step_pipe_nt<8, 4>(c, v, Rin, Rout, r, ldr, G, D, done)
                                                    : spmm_step_pipe_nt<8, 8>(c, v, Rin, Rout, r, ldr, G, D, done));
            if (ok) {
                ++*c.launches;
                return;
            }
        }
    }
    const int L = lanes_for(r, W);
    ALM_DISPATCH_LANES(L, {
        if (v.ell_kf == 4) spmm_step_one<T, LN, 4>(c, v, Rin, Rout, r, ldr, G, D, done);
        else if (v.ell_kf == 8) spmm_step_one<T, LN, 8>(c, v, Rin, Rout, r, ldr, G, D, done);
        else spmm_step_one<T, LN, 16>(c, v, Rin, Rout, r, ldr, G, D, done);
    });
    ++*c.launches;
}

template <typename T>
bool ls_dir_fusable(const SparseView<T> &v) {
    return v.ell_ku > 0 && v.lr_k == 0 && !v.has_off_sel && v.m_gen == 0;
}

template <typename T>
void launch_ls_dir(const LaunchCtx &c, const SparseView<T> &v, const T *R, const T *Z, const T *Dold, T *Dnew, int r,
                   int ldr, const int *done) {
    constexpr int W = VecT<T>::W;
    {
        constexpr int MINL = sizeof(T) == 4 ? 4 : 8;  // 16 columns or more
        const int L = lanes_for(r, W);
        if (pipe_ok(c, v.ell_kn, L, MINL) && v.ls_rec && v.un_col) {
            auto go = [&](auto lanes_tag) -> bool {
                constexpr int LN = decltype(lanes_tag)::value;
                if (v.ell_kn == 2) return ls_dir_pipe_nt<T, LN, 2>(c, v, R, Z, Dold, Dnew, r, ldr, done);
                if (v.ell_kn == 4) return ls_dir_pipe_nt<T, LN, 4>(c, v, R, Z, Dold, Dnew, r, ldr, done);
                return ls_dir_pipe_nt<T, LN, 8>(c, v, R, Z, Dold, Dnew, r, ldr, done);
            };
            const bool ok = L == MINL ? go(std::integral_constant<int, MINL>{})
                                      : go(std::integral_constant<int, 2 * MINL>{});
            if (ok) {
                ++*c.launches;
                return;
            }
        }
    }
    const int L = lanes_for(r, W);
    ALM_DISPATCH_LANES(L, {
        if (v.ell_ku == 2) ls_ell_dir_one<T, LN, 2>(c, v, R, Z, Dold, Dnew, r, ldr, done);
        else if (v.ell_ku == 4) ls_ell_dir_one<T, LN, 4>(c, v, R, Z, Dold, Dnew, r, ldr, done);
        else if (v.ell_ku == 8) ls_ell_dir_one<T, LN, 8>(c, v, R, Z, Dold, Dnew, r, ldr, done);
        else ls_ell_dir_one<T, LN, 16>(c, v, R, Z, Dold, Dnew, r, ldr, done);
    });
    ++*c.launches;
}

#define ALM_INNER_INST(T)                                                                                       \
    template void launch_ls_dir<T>(const LaunchCtx &, const SparseView<T> &, const T *, const T *, const T *, T *, \
                                   int, int, const int *);                                                      \
    template bool ls_dir_fusable<T>(const SparseView<T> &);                                                      \
    template bool spmm_step_fusable<T>(const SparseView<T> &);                                                   \
    template void launch_spmm_step<T>(const LaunchCtx &, const SparseView<T> &, const T *, T *, int, int, T *,    \
                                      const T *, const int *);

// ALM_INST_ONLY (1: float, 2: double): see kernels_sparse.cu
#if !defined(ALM_INST_ONLY) || ALM_INST_ONLY == 1
ALM_INNER_INST(float)
#endif
#if !defined(ALM_INST_ONLY) || ALM_INST_ONLY == 2
ALM_INNER_INST(double)
#endif

}  // namespace alm
