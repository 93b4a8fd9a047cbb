// Host-side builder of the aggregated sparsity pattern of (P) (arXiv 2505.15775,
// Sec. 1.2: C, the A_k and b).  It validates the coordinate input of alm_create
// and lays the data out the way the kernels read it:
//
//  * the strict upper triangle of P = nnz(C) u nnz(A_0) u ... (CSR, for the SDDMMs:
//    every off-diagonal pair once, since X_ij = X_ji);
//  * the diagonal (C_ii and, per row, the selector constraint e_i e_i^T if any);
//  * the full off-diagonal pattern (CSR with both (i,j) and (j,i), for the SpMM
//    and the Lanczos SpMV) and, when S's off-diagonal values depend on y, the map
//    from each full slot back to its upper entry;
//  * the constraints split into "selectors" (one entry, and no other selector on
//    that entry: A(X)_k = kappa a X_ij is written directly by the SDDMM) and
//    "general" constraints (constraint-major lists), plus entry-major lists of the
//    general constraints for the slack update S = C - A^*(w).
#include "alm_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <sstream>

namespace alm {

namespace {

struct Entry {            // one upper-triangle coordinate of some input matrix
    int32_t i, j;
    int32_t k;            // -1: C, else constraint index
    double v;
};

}  // namespace

std::string build_pattern(const alm_problem *p, HostPattern *hp) {
    std::ostringstream err;
    if (!p) return "problem is NULL";
    if (p->n < 1 || p->m < 1) return "n and m must be >= 1";
    if (p->n >= (int64_t(1) << 31) - 1 || p->m >= (int64_t(1) << 31) - 1) return "n and m must be < 2^31 - 1";
    if (p->c_nnz < 0 || p->a_nnz < 1) return "c_nnz must be >= 0 and a_nnz >= 1";
    if (p->c_nnz > 0 && (!p->c_i || !p->c_j || !p->c_v)) return "C arrays are NULL";
    if (!p->a_k || !p->a_i || !p->a_j || !p->a_v || !p->b) return "constraint arrays are NULL";
    if (p->c_lr_k < 0 || p->c_lr_k > kMaxLR) return "c_lr_k must be in 0..4";
    if (p->c_lr_k > 0 && (!p->c_lr_u || !p->c_lr_s)) return "low-rank arrays are NULL";
    const int64_t n = p->n, m = p->m;
    hp->n = n;
    hp->m = m;

    // ---- validate and gather entries -------------------------------------------
    std::vector<Entry> ent;
    ent.reserve(size_t(p->c_nnz + p->a_nnz));
    for (int64_t e = 0; e < p->c_nnz; ++e) {
        int32_t i = p->c_i[e], j = p->c_j[e];
        double v = p->c_v[e];
        if (i < 0 || j < 0 || i >= n || j >= n || i > j) {
            err << "C entry " << e << " = (" << i << "," << j << ") is out of range or not upper-triangular";
            return err.str();
        }
        if (!std::isfinite(v)) { err << "C entry " << e << " is not finite"; return err.str(); }
        ent.push_back({i, j, -1, v});
    }
    std::vector<int64_t> con_count(size_t(m), 0);
    for (int64_t e = 0; e < p->a_nnz; ++e) {
        int32_t k = p->a_k[e], i = p->a_i[e], j = p->a_j[e];
        double v = p->a_v[e];
        if (k < 0 || k >= m) { err << "constraint entry " << e << " has index " << k << " outside 0..m-1"; return err.str(); }
        if (i < 0 || j < 0 || i >= n || j >= n || i > j) {
            err << "constraint entry " << e << " = (" << i << "," << j << ") is out of range or not upper-triangular";
            return err.str();
        }
        if (!std::isfinite(v)) { err << "constraint entry " << e << " is not finite"; return err.str(); }
        ent.push_back({i, j, k, v});
    }
    for (int64_t k = 0; k < m; ++k)
        if (!std::isfinite(p->b[k])) { err << "b[" << k << "] is not finite"; return err.str(); }
    for (int l = 0; l < p->c_lr_k; ++l) {
        if (!std::isfinite(p->c_lr_s[l])) return "c_lr_s is not finite";
        for (int64_t i = 0; i < n; ++i)
            if (!std::isfinite(p->c_lr_u[l * n + i])) return "c_lr_u is not finite";
    }

    // ---- sort entries by (i, j, k): counting sort on i, then per-row sort --------
    std::vector<int64_t> rcount(size_t(n) + 1, 0);
    for (const Entry &x : ent) rcount[size_t(x.i) + 1]++;
    for (int64_t i = 0; i < n; ++i) rcount[size_t(i) + 1] += rcount[size_t(i)];
    std::vector<Entry> sorted(ent.size());
    {
        std::vector<int64_t> pos(rcount.begin(), rcount.end() - 1);
        for (const Entry &x : ent) sorted[size_t(pos[size_t(x.i)]++)] = x;
    }
    ent.clear();
    ent.shrink_to_fit();
    for (int64_t i = 0; i < n; ++i) {
        auto b = sorted.begin() + rcount[size_t(i)], e = sorted.begin() + rcount[size_t(i) + 1];
        std::sort(b, e, [](const Entry &a, const Entry &c) {
            if (a.j != c.j) return a.j < c.j;
            return a.k < c.k;
        });
    }

    // ---- merge into unique (i, j) pattern entries ----------------------------------
    // per unique off-diagonal entry: C value and its list of (k, a) (duplicates per k summed)
    hp->d_c.assign(size_t(n), 0.0);
    hp->up_ptr.assign(size_t(n) + 1, 0);
    hp->up_col.clear();
    hp->up_c.clear();
    std::vector<int64_t> up_con_ptr(1, 0);            // CSR over upper entries -> (k, a)
    std::vector<int32_t> up_con_k;
    std::vector<double> up_con_a;
    std::vector<int64_t> dg_con_ptr(size_t(n) + 1, 0);  // per row diagonal -> (k, a)
    std::vector<int32_t> dg_con_k;
    std::vector<double> dg_con_a;
    int64_t s = 0;
    const int64_t total = int64_t(sorted.size());
    for (int64_t i = 0; i < n; ++i) {
        int64_t e = rcount[size_t(i)], end = rcount[size_t(i) + 1];
        while (e < end) {
            const int32_t j = sorted[size_t(e)].j;
            double cval = 0.0;
            int64_t f = e;
            // entries of this (i, j), ordered by k (C first, k = -1)
            std::vector<std::pair<int32_t, double>> cons;
            while (f < end && sorted[size_t(f)].j == j) {
                const Entry &x = sorted[size_t(f)];
                if (x.k < 0) cval += x.v;
                else if (!cons.empty() && cons.back().first == x.k) cons.back().second += x.v;
                else cons.push_back({x.k, x.v});
                ++f;
            }
            if (j == i) {
                hp->d_c[size_t(i)] = cval;
                for (auto &c : cons) { dg_con_k.push_back(c.first); dg_con_a.push_back(c.second); }
            } else {
                hp->up_col.push_back(j);
                hp->up_c.push_back(cval);
                for (auto &c : cons) { up_con_k.push_back(c.first); up_con_a.push_back(c.second); }
                up_con_ptr.push_back(int64_t(up_con_k.size()));
            }
            e = f;
        }
        hp->up_ptr[size_t(i) + 1] = int32_t(hp->up_col.size());
        dg_con_ptr[size_t(i) + 1] = int64_t(dg_con_k.size());
        if (hp->up_col.size() >= size_t(INT32_MAX) / 2) return "pattern too large (>= 2^30 upper entries)";
    }
    (void)s;
    (void)total;
    sorted.clear();
    sorted.shrink_to_fit();
    const int64_t nnz_u = int64_t(hp->up_col.size());

    // ---- classify constraints ------------------------------------------------------
    // entries per constraint after merging
    std::fill(con_count.begin(), con_count.end(), 0);
    for (int32_t k : up_con_k) con_count[size_t(k)]++;
    for (int32_t k : dg_con_k) con_count[size_t(k)]++;
    for (int64_t k = 0; k < m; ++k)
        if (con_count[size_t(k)] == 0) {
            err << "constraint " << k << " has no entries (A_k = 0)";
            return err.str();
        }
    // a selector: exactly one entry, and the first selector on its pattern entry
    std::vector<char> is_sel(size_t(m), 0);
    hp->d_sel_k.assign(size_t(n), -1);
    hp->d_sel_a.assign(size_t(n), 0.0);
    std::vector<int32_t> up_sel_k(size_t(nnz_u), -1);
    std::vector<double> up_sel_a(size_t(nnz_u), 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t t = dg_con_ptr[size_t(i)]; t < dg_con_ptr[size_t(i) + 1]; ++t) {
            int32_t k = dg_con_k[size_t(t)];
            if (con_count[size_t(k)] == 1 && hp->d_sel_k[size_t(i)] < 0) {
                hp->d_sel_k[size_t(i)] = k;
                hp->d_sel_a[size_t(i)] = dg_con_a[size_t(t)];
                is_sel[size_t(k)] = 1;
            }
        }
    bool has_off_sel = false;
    for (int64_t e = 0; e < nnz_u; ++e)
        for (int64_t t = up_con_ptr[size_t(e)]; t < up_con_ptr[size_t(e) + 1]; ++t) {
            int32_t k = up_con_k[size_t(t)];
            if (con_count[size_t(k)] == 1 && up_sel_k[size_t(e)] < 0) {
                up_sel_k[size_t(e)] = k;
                up_sel_a[size_t(e)] = up_con_a[size_t(t)];
                is_sel[size_t(k)] = 1;
                has_off_sel = true;
            }
        }
    hp->has_off_sel = has_off_sel;
    if (has_off_sel) {
        hp->up_sel_k.swap(up_sel_k);
        hp->up_sel_a.swap(up_sel_a);
    } else {
        hp->up_sel_k.clear();
        hp->up_sel_a.clear();
    }
    hp->n_sel = 0;
    for (int64_t k = 0; k < m; ++k) hp->n_sel += is_sel[size_t(k)];

    // general constraints: constraint-major lists of (i, j, a), and entry-major lists
    std::vector<int32_t> gidx(size_t(m), -1);
    hp->g_con.clear();
    for (int64_t k = 0; k < m; ++k)
        if (!is_sel[size_t(k)]) { gidx[size_t(k)] = int32_t(hp->g_con.size()); hp->g_con.push_back(int32_t(k)); }
    hp->m_gen = int64_t(hp->g_con.size());
    hp->g_ptr.assign(size_t(hp->m_gen) + 1, 0);
    hp->gd_ptr.assign(size_t(n) + 1, 0);
    hp->gd_k.clear();
    hp->gd_a.clear();
    hp->gu_ptr.clear();
    hp->gu_k.clear();
    hp->gu_a.clear();
    hp->has_gen_diag = false;
    hp->has_gen_off = false;
    if (hp->m_gen > 0) {
        std::vector<int64_t> gcount(size_t(hp->m_gen) + 1, 0);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t t = dg_con_ptr[size_t(i)]; t < dg_con_ptr[size_t(i) + 1]; ++t) {
                int32_t k = dg_con_k[size_t(t)];
                bool sel_here = hp->d_sel_k[size_t(i)] == k;
                if (!sel_here) gcount[size_t(gidx[size_t(k)]) + 1]++;
            }
        for (int64_t e = 0; e < nnz_u; ++e)
            for (int64_t t = up_con_ptr[size_t(e)]; t < up_con_ptr[size_t(e) + 1]; ++t) {
                int32_t k = up_con_k[size_t(t)];
                bool sel_here = has_off_sel && hp->up_sel_k[size_t(e)] == k;
                if (!sel_here) gcount[size_t(gidx[size_t(k)]) + 1]++;
            }
        for (int64_t g = 0; g < hp->m_gen; ++g) gcount[size_t(g) + 1] += gcount[size_t(g)];
        if (gcount[size_t(hp->m_gen)] >= INT32_MAX) return "too many general constraint entries";
        for (int64_t g = 0; g <= hp->m_gen; ++g) hp->g_ptr[size_t(g)] = int32_t(gcount[size_t(g)]);
        const size_t gtot = size_t(gcount[size_t(hp->m_gen)]);
        hp->g_i.assign(gtot, 0);
        hp->g_j.assign(gtot, 0);
        hp->g_a.assign(gtot, 0.0);
        std::vector<int64_t> gpos(gcount.begin(), gcount.end() - 1);
        // diagonal general entries (also entry-major per row)
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t t = dg_con_ptr[size_t(i)]; t < dg_con_ptr[size_t(i) + 1]; ++t) {
                int32_t k = dg_con_k[size_t(t)];
                if (hp->d_sel_k[size_t(i)] == k) continue;
                size_t q = size_t(gpos[size_t(gidx[size_t(k)])]++);
                hp->g_i[q] = int32_t(i);
                hp->g_j[q] = int32_t(i);
                hp->g_a[q] = dg_con_a[size_t(t)];
                hp->gd_k.push_back(k);
                hp->gd_a.push_back(dg_con_a[size_t(t)]);
                hp->has_gen_diag = true;
            }
            hp->gd_ptr[size_t(i) + 1] = int32_t(hp->gd_k.size());
        }
        // off-diagonal general entries (entry-major per upper entry)
        std::vector<int32_t> gu_ptr(size_t(nnz_u) + 1, 0);
        std::vector<int32_t> gu_k;
        std::vector<double> gu_a;
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = hp->up_ptr[size_t(i)]; e < hp->up_ptr[size_t(i) + 1]; ++e) {
                for (int64_t t = up_con_ptr[size_t(e)]; t < up_con_ptr[size_t(e) + 1]; ++t) {
                    int32_t k = up_con_k[size_t(t)];
                    if (has_off_sel && hp->up_sel_k[size_t(e)] == k) continue;
                    size_t q = size_t(gpos[size_t(gidx[size_t(k)])]++);
                    hp->g_i[q] = int32_t(i);
                    hp->g_j[q] = hp->up_col[size_t(e)];
                    hp->g_a[q] = up_con_a[size_t(t)];
                    gu_k.push_back(k);
                    gu_a.push_back(up_con_a[size_t(t)]);
                    hp->has_gen_off = true;
                }
                gu_ptr[size_t(e) + 1] = int32_t(gu_k.size());
            }
        if (hp->has_gen_off) {
            hp->gu_ptr.swap(gu_ptr);
            hp->gu_k.swap(gu_k);
            hp->gu_a.swap(gu_a);
        }
        if (!hp->has_gen_diag) { hp->gd_ptr.clear(); }
    } else {
        hp->gd_ptr.clear();
    }
    hp->off_dynamic = has_off_sel || hp->has_gen_off;

    // ---- full off-diagonal CSR (both triangles) ---------------------------------------
    hp->f_ptr.assign(size_t(n) + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        int32_t deg_up = hp->up_ptr[size_t(i) + 1] - hp->up_ptr[size_t(i)];
        hp->f_ptr[size_t(i) + 1] += deg_up;
        for (int64_t e = hp->up_ptr[size_t(i)]; e < hp->up_ptr[size_t(i) + 1]; ++e)
            hp->f_ptr[size_t(hp->up_col[size_t(e)]) + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) hp->f_ptr[size_t(i) + 1] += hp->f_ptr[size_t(i)];
    const size_t nnz_f = size_t(hp->f_ptr[size_t(n)]);
    hp->f_col.assign(nnz_f, 0);
    hp->f_c.assign(nnz_f, 0.0);
    hp->up_slot.assign(hp->off_dynamic ? 2 * size_t(nnz_u) : 0, 0);
    {
        // lower part first (column index < i, ascending since rows are visited in order),
        // then the upper part (j > i, ascending): each row ends up sorted.
        std::vector<int32_t> pos(hp->f_ptr.begin(), hp->f_ptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = hp->up_ptr[size_t(i)]; e < hp->up_ptr[size_t(i) + 1]; ++e) {
                int32_t j = hp->up_col[size_t(e)];
                size_t q = size_t(pos[size_t(j)]++);
                hp->f_col[q] = int32_t(i);
                hp->f_c[q] = hp->up_c[size_t(e)];
                if (hp->off_dynamic) hp->up_slot[2 * size_t(e) + 1] = int32_t(q);
            }
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = hp->up_ptr[size_t(i)]; e < hp->up_ptr[size_t(i) + 1]; ++e) {
                size_t q = size_t(pos[size_t(i)]++);
                hp->f_col[q] = hp->up_col[size_t(e)];
                hp->f_c[q] = hp->up_c[size_t(e)];
                if (hp->off_dynamic) hp->up_slot[2 * size_t(e)] = int32_t(q);
            }
    }
    hp->up_row.assign(size_t(nnz_u), 0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = hp->up_ptr[size_t(i)]; e < hp->up_ptr[size_t(i) + 1]; ++e) hp->up_row[size_t(e)] = int32_t(i);

    // ELL copies (fixed row width, padded with the row itself and value 0) when S's
    // off-diagonal values never change and every row is short: column indices then sit at
    // computable addresses, so the kernels can fetch them ahead of the row gathers
    int32_t maxf = 0, maxu = 0;
    for (int64_t i = 0; i < n; ++i) {
        maxf = std::max(maxf, hp->f_ptr[size_t(i) + 1] - hp->f_ptr[size_t(i)]);
        maxu = std::max(maxu, hp->up_ptr[size_t(i) + 1] - hp->up_ptr[size_t(i)]);
    }
    hp->ell_kf = hp->ell_ku = 0;
    hp->f_ell_col.clear();
    hp->f_ell_val.clear();
    hp->u_ell_col.clear();
    hp->u_ell_val.clear();
    if (!hp->off_dynamic && maxf <= 16 && p->c_lr_k == 0) {
        const int kf = maxf <= 4 ? 4 : maxf <= 8 ? 8 : 16;
        const int ku = maxu <= 2 ? 2 : maxu <= 4 ? 4 : maxu <= 8 ? 8 : 16;
        hp->ell_kf = kf;
        hp->ell_ku = ku;
        hp->f_ell_col.assign(size_t(n) * kf, 0);
        hp->f_ell_val.assign(size_t(n) * kf, 0.0);
        hp->u_ell_col.assign(size_t(n) * ku, 0);
        hp->u_ell_val.assign(size_t(n) * ku, 0.0);
        for (int64_t i = 0; i < n; ++i) {
            int t = 0;
            for (int64_t e = hp->f_ptr[size_t(i)]; e < hp->f_ptr[size_t(i) + 1]; ++e, ++t) {
                hp->f_ell_col[size_t(i) * kf + t] = hp->f_col[size_t(e)];
                hp->f_ell_val[size_t(i) * kf + t] = hp->f_c[size_t(e)];
            }
            for (; t < kf; ++t) hp->f_ell_col[size_t(i) * kf + t] = int32_t(i);
            t = 0;
            for (int64_t e = hp->up_ptr[size_t(i)]; e < hp->up_ptr[size_t(i) + 1]; ++e, ++t) {
                hp->u_ell_col[size_t(i) * ku + t] = hp->up_col[size_t(e)];
                hp->u_ell_val[size_t(i) * ku + t] = hp->up_c[size_t(e)];
            }
            for (; t < ku; ++t) hp->u_ell_col[size_t(i) * ku + t] = int32_t(i);
        }
        // narrow upper ELL: the width of {2, 4, 8} (at most ku) that minimises the padded
        // entries plus twice the overflow entries (an overflow entry costs about two)
        int best = ku;
        int64_t best_cost = int64_t(ku) * n;
        for (int w : {2, 4, 8}) {
            if (w >= ku) break;
            int64_t ov = 0;
            for (int64_t i = 0; i < n; ++i)
                ov += std::max<int64_t>(0, int64_t(hp->up_ptr[size_t(i) + 1] - hp->up_ptr[size_t(i)]) - w);
            const int64_t cost = int64_t(w) * n + 2 * ov;
            if (cost < best_cost) {
                best_cost = cost;
                best = w;
            }
        }
        hp->ell_kn = best;
        hp->un_col.assign(size_t(n) * best, 0);
        hp->un_val.assign(size_t(n) * best, 0.0);
        hp->ov_i.clear();
        hp->ov_j.clear();
        hp->ov_v.clear();
        for (int64_t i = 0; i < n; ++i) {
            int t = 0;
            for (int64_t e = hp->up_ptr[size_t(i)]; e < hp->up_ptr[size_t(i) + 1]; ++e, ++t) {
                if (t < best) {
                    hp->un_col[size_t(i) * best + t] = hp->up_col[size_t(e)];
                    hp->un_val[size_t(i) * best + t] = hp->up_c[size_t(e)];
                } else {
                    hp->ov_i.push_back(int32_t(i));
                    hp->ov_j.push_back(hp->up_col[size_t(e)]);
                    hp->ov_v.push_back(hp->up_c[size_t(e)]);
                }
            }
            for (; t < best; ++t) hp->un_col[size_t(i) * best + t] = int32_t(i);
        }
    }

    // ---- b, low-rank part, norms -------------------------------------------------------
    hp->b.assign(p->b, p->b + m);
    hp->lr_k = p->c_lr_k;
    hp->lr_u.assign(size_t(p->c_lr_k) * size_t(n), 0.0);
    hp->lr_s.assign(size_t(p->c_lr_k), 0.0);
    for (int l = 0; l < p->c_lr_k; ++l) {
        hp->lr_s[size_t(l)] = p->c_lr_s[l];
        std::memcpy(&hp->lr_u[size_t(l) * size_t(n)], p->c_lr_u + size_t(l) * size_t(n), sizeof(double) * size_t(n));
    }
    double nb = 0.0;
    for (double v : hp->b) nb += v * v;
    hp->norm_b = std::sqrt(nb);
    // ||C||_F^2 = ||C_s||_F^2 + 2 sum_l s_l u_l^T C_s u_l + sum_{l,q} s_l s_q (u_l . u_q)^2
    double nc = 0.0;
    for (int64_t i = 0; i < n; ++i) nc += hp->d_c[size_t(i)] * hp->d_c[size_t(i)];
    for (double v : hp->up_c) nc += 2.0 * v * v;
    for (int l = 0; l < hp->lr_k; ++l) {
        const double *u = &hp->lr_u[size_t(l) * size_t(n)];
        double quad = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            quad += hp->d_c[size_t(i)] * u[i] * u[i];
            for (int64_t e = hp->up_ptr[size_t(i)]; e < hp->up_ptr[size_t(i) + 1]; ++e)
                quad += 2.0 * hp->up_c[size_t(e)] * u[i] * u[hp->up_col[size_t(e)]];
        }
        nc += 2.0 * hp->lr_s[size_t(l)] * quad;
        for (int q = 0; q < hp->lr_k; ++q) {
            const double *uq = &hp->lr_u[size_t(q) * size_t(n)];
            double d = 0.0;
            for (int64_t i = 0; i < n; ++i) d += u[i] * uq[i];
            nc += hp->lr_s[size_t(l)] * hp->lr_s[size_t(q)] * d * d;
        }
    }
    hp->norm_C = std::sqrt(std::max(nc, 0.0));
    return "";
}

}  // namespace alm
