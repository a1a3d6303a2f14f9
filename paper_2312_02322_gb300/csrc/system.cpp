// mqct_create_system: validation, internal state order, spline tables and coupling
// layouts (host), then upload to device memory.
//
// Spline (Sec. III): clamped cubic on the uniform grid, solved here in the slope form
//   d_{i-1} + 4 d_i + d_{i+1} = 3 (y_{i+1} - y_{i-1}) / h,  d_0, d_{n-1} given,
// whose piecewise cubics are the same clamped spline as any other construction.
// Because the spline is linear in the data, the table of M_nm(R) = sum_l G^l_nm v_l(R)
// is sum_l G^l_nm (coefficients of v_l): the PLAIN and FACTORISED paths evaluate the same
// function (Eq. 12).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace mqct {

namespace {
thread_local std::string g_err;
thread_local long long g_launches = 0;
}

void reset_launches() { g_launches = 0; }
void count_launches(long long n) { g_launches += n; }

void set_error(const std::string &msg) { g_err = msg; }
const char *last_error_cstr() { return g_err.c_str(); }
mqct_status fail(mqct_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}
mqct_status cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MQCT_ERR_OOM : MQCT_ERR_CUDA;
}

namespace {

// clamped cubic spline in slope form; coef[i] = (c0, c1, c2, c3) on [R_i, R_i+1]
void clamped_spline(int n, double h, const double *y, double d0, double dn, std::vector<dbl4> &coef)
{
    std::vector<double> d(n), cp(n), rp(n);
    d[0] = d0;
    d[n - 1] = dn;
    int m = n - 2;  // interior unknowns d_1..d_{n-2}
    if (m > 0) {
        // forward sweep: rows i = 1..n-2, diag 4, off-diagonals 1
        for (int i = 1; i <= m; ++i) {
            double rhs = 3.0 * (y[i + 1] - y[i - 1]) / h;
            if (i == 1) rhs -= d0;
            if (i == m) rhs -= dn;
            double diag = 4.0;
            if (i > 1) {
                diag -= cp[i - 1];
                rhs -= rp[i - 1];
            }
            cp[i] = 1.0 / diag;
            rp[i] = rhs / diag;
        }
        d[m] = rp[m];
        for (int i = m - 1; i >= 1; --i) d[i] = rp[i] - cp[i] * d[i + 1];
    }
    coef.resize(n - 1);
    for (int i = 0; i < n - 1; ++i) {
        double del = (y[i + 1] - y[i]) / h;
        coef[i] = make_dbl4(y[i], d[i], (3.0 * del - 2.0 * d[i] - d[i + 1]) / h, (d[i] + d[i + 1] - 2.0 * del) / (h * h));
    }
}

struct Entry {
    int r, c;
    double v;
};

template <class T>
mqct_status upload(System &S, const std::vector<T> &v, const T **dst)
{
    *dst = nullptr;
    if (v.empty()) return MQCT_OK;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * v.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    S.allocs.push_back(p);
    e = cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    *dst = static_cast<const T *>(p);
    S.info.device_bytes += (int64_t)(sizeof(T) * v.size());
    return MQCT_OK;
}

void release(System &S)
{
    for (void *p : S.allocs) cudaFree(p);
    S.allocs.clear();
    if (S.d) cudaFree(S.d);
    S.d = nullptr;
}

// sliced-ELL layout of per-row entry lists: slices of kSlice consecutive rows, width = max
// row length in the slice, entry (slice, k, lane) at off[slice] + k * kSlice + lane.
struct Sell {
    std::vector<int> off;   // [n_slices + 1]
    std::vector<int> cols;  // [nnz_pad]
    std::vector<int> src;   // [nnz_pad] index into the row's entry list, -1 for padding
    std::vector<int> row_of;
};

Sell make_sell(int n, const std::vector<std::vector<Entry>> &rows)
{
    Sell S;
    int ns = (n + kSlice - 1) / kSlice;
    S.off.assign(ns + 1, 0);
    for (int s = 0; s < ns; ++s) {
        int w = 0;
        for (int l = 0; l < kSlice; ++l) {
            int r = s * kSlice + l;
            if (r < n) w = std::max<int>(w, (int)rows[r].size());
        }
        S.off[s + 1] = S.off[s] + w * kSlice;
    }
    S.cols.assign(S.off[ns], 0);
    S.src.assign(S.off[ns], -1);
    S.row_of.assign(S.off[ns], 0);
    for (int s = 0; s < ns; ++s) {
        int w = (S.off[s + 1] - S.off[s]) / kSlice;
        for (int l = 0; l < kSlice; ++l) {
            int r = s * kSlice + l;
            for (int k = 0; k < w; ++k) {
                int e = S.off[s] + k * kSlice + l;
                S.row_of[e] = r;
                if (r < n && k < (int)rows[r].size()) {
                    S.cols[e] = rows[r][k].c;
                    S.src[e] = k;
                } else {
                    S.cols[e] = r < n ? r : 0;  // in-bounds dummy column, zero coefficient
                }
            }
        }
    }
    return S;
}

}  // namespace
}  // namespace mqct

using namespace mqct;

extern "C" mqct_status mqct_create_system(const mqct_system_desc *d, mqct_system *out)
{
    if (!d || !out) return fail(MQCT_ERR_INVALID_ARG, "mqct_create_system: NULL argument");
    *out = nullptr;
    const int n = d->n_states, L = d->n_terms, ng = d->n_grid, P = d->n_params;
    if (n < 1) return fail(MQCT_ERR_INVALID_ARG, "n_states < 1");
    if (L < 1 || L > kMaxTerms) return fail(MQCT_ERR_INVALID_ARG, "n_terms outside [1, 64]");
    if (ng < 4) return fail(MQCT_ERR_INVALID_ARG, "n_grid < 4");
    if (!(d->r_max > d->r_min) || !std::isfinite(d->r_min) || !std::isfinite(d->r_max))
        return fail(MQCT_ERR_INVALID_ARG, "r_max must exceed r_min (finite)");
    if (!(d->mu > 0) || !std::isfinite(d->mu)) return fail(MQCT_ERR_INVALID_ARG, "mu must be finite and > 0");
    if (!d->energy || !d->level || !d->j || !d->m || !d->v || !d->dv_ends)
        return fail(MQCT_ERR_INVALID_ARG, "NULL array in system description");
    if (d->path != MQCT_PATH_PLAIN && d->path != MQCT_PATH_FACTORISED) return fail(MQCT_ERR_INVALID_ARG, "unknown path");
    if (d->precision != MQCT_FP64 && d->precision != MQCT_FP32 && d->precision != MQCT_BF16X3)
        return fail(MQCT_ERR_INVALID_ARG, "unknown precision");
    if (d->precision == MQCT_BF16X3 && d->path != MQCT_PATH_FACTORISED)
        return fail(MQCT_ERR_UNSUPPORTED, "MQCT_BF16X3 runs on the factorised path only");
    if (d->grid_kind != MQCT_GRID_UNIFORM && d->grid_kind != MQCT_GRID_LOG)
        return fail(MQCT_ERR_INVALID_ARG, "unknown grid_kind");
    if (d->grid_kind == MQCT_GRID_LOG && !(d->r_min > 0))
        return fail(MQCT_ERR_INVALID_ARG, "MQCT_GRID_LOG needs r_min > 0");
    if (d->grid_kind == MQCT_GRID_LOG && d->precision != MQCT_FP64 && d->path == MQCT_PATH_FACTORISED)
        return fail(MQCT_ERR_UNSUPPORTED, "MQCT_GRID_LOG runs on FP64 systems and on the PLAIN path");
    if (!std::isfinite(d->trunc_threshold)) return fail(MQCT_ERR_INVALID_ARG, "non-finite trunc_threshold");
    if (!std::isfinite(d->adapt_tol) || d->adapt_tol < 0.0) return fail(MQCT_ERR_INVALID_ARG, "adapt_tol must be finite and >= 0");
    if (d->adapt_tol > 0.0) {
        const int hm = d->adapt_hmax;
        if (hm < 0 || hm > 1024 || (hm & (hm - 1)) != 0)
            return fail(MQCT_ERR_INVALID_ARG, "adapt_hmax must be 0 or a power of 2 up to 1024");
        if (d->precision != MQCT_FP64) return fail(MQCT_ERR_UNSUPPORTED, "adaptive steps need precision MQCT_FP64");
        if (d->flags & MQCT_PRESCRIBED_TRAJ)
            return fail(MQCT_ERR_UNSUPPORTED, "adaptive steps do not run with MQCT_PRESCRIBED_TRAJ");
    }
    if (d->trunc_threshold > 0.0) {
        if (d->path != MQCT_PATH_PLAIN) return fail(MQCT_ERR_UNSUPPORTED, "truncation needs the PLAIN path");
        if (!(d->trunc_r[0] > 0) || !(d->trunc_r[1] > 0) || !std::isfinite(d->trunc_r[0]) || !std::isfinite(d->trunc_r[1]))
            return fail(MQCT_ERR_INVALID_ARG, "trunc_r must be finite and > 0");
    }
    if (d->flags & ~(MQCT_PRESCRIBED_TRAJ | MQCT_DECOUPLED_TRAJ)) return fail(MQCT_ERR_INVALID_ARG, "unknown flags");
    if ((d->flags & MQCT_PRESCRIBED_TRAJ) && (d->flags & MQCT_DECOUPLED_TRAJ))
        return fail(MQCT_ERR_INVALID_ARG, "MQCT_PRESCRIBED_TRAJ and MQCT_DECOUPLED_TRAJ exclude each other");
    if ((d->flags & MQCT_PRESCRIBED_TRAJ) && d->precision != MQCT_FP64)
        return fail(MQCT_ERR_UNSUPPORTED, "MQCT_PRESCRIBED_TRAJ needs precision MQCT_FP64");
    if ((d->flags & MQCT_DECOUPLED_TRAJ) && d->precision != MQCT_FP64)
        return fail(MQCT_ERR_UNSUPPORTED, "MQCT_DECOUPLED_TRAJ needs precision MQCT_FP64");
    if (P < 0 || (P > 0 && (!d->dv_dparam || !d->ddv_ends))) return fail(MQCT_ERR_INVALID_ARG, "bad parameter tables");
    if (!d->G && d->g_nnz > 0 && (!d->g_term || !d->g_row || !d->g_col || !d->g_val))
        return fail(MQCT_ERR_INVALID_ARG, "NULL triplet array");
    if (!d->G && d->g_nnz < 0) return fail(MQCT_ERR_INVALID_ARG, "g_nnz < 0");

    // ---- labels and levels
    int n_levels = 0;
    for (int s = 0; s < n; ++s) {
        if (!std::isfinite(d->energy[s])) return fail(MQCT_ERR_INVALID_ARG, "non-finite energy");
        if (d->level[s] < 0 || d->level[s] >= n) return fail(MQCT_ERR_INVALID_ARG, "level id outside [0, N)");
        if (d->j[s] >= 0 && std::abs(d->m[s]) > d->j[s]) return fail(MQCT_ERR_INVALID_ARG, "|m| > j");
        n_levels = std::max(n_levels, d->level[s] + 1);
    }
    std::vector<double> lev_e(n_levels, NAN);
    for (int s = 0; s < n; ++s) {
        double &e = lev_e[d->level[s]];
        if (std::isnan(e)) e = d->energy[s];
        else if (e != d->energy[s]) return fail(MQCT_ERR_INVALID_ARG, "states of one level have different energies");
    }
    for (auto &e : lev_e)
        if (std::isnan(e)) e = 0.0;  // unused level id

    // ---- coupling entries per term (caller indices): sorted by (row, column), duplicates summed
    // in the order given
    struct Trip {
        int r, c;
        double v;
    };
    std::vector<std::vector<Trip>> G(L);
    double gmax = 0.0;
    if (d->G) {
        for (int l = 0; l < L; ++l)
            for (int r = 0; r < n; ++r)
                for (int c = 0; c < n; ++c) {
                    double v = d->G[((size_t)l * n + r) * n + c];
                    if (!std::isfinite(v)) return fail(MQCT_ERR_INVALID_ARG, "non-finite G");
                    if (v != 0.0) G[l].push_back({r, c, v});
                }
    } else {
        for (int64_t i = 0; i < d->g_nnz; ++i) {
            int l = d->g_term[i], r = d->g_row[i], c = d->g_col[i];
            double v = d->g_val[i];
            if (l < 0 || l >= L || r < 0 || r >= n || c < 0 || c >= n) return fail(MQCT_ERR_INVALID_ARG, "G triplet out of range");
            if (!std::isfinite(v)) return fail(MQCT_ERR_INVALID_ARG, "non-finite G");
            G[l].push_back({r, c, v});
        }
    }
    auto trip_less = [](const Trip &a, const Trip &b) { return a.r != b.r ? a.r < b.r : a.c < b.c; };
    for (auto &t : G) {
        std::stable_sort(t.begin(), t.end(), trip_less);
        size_t k = 0;
        for (size_t i = 0; i < t.size(); ++i) {
            if (k > 0 && t[k - 1].r == t[i].r && t[k - 1].c == t[i].c) t[k - 1].v += t[i].v;
            else t[k++] = t[i];
        }
        t.resize(k);
    }
    for (int l = 0; l < L; ++l)
        for (const Trip &e : G[l]) gmax = std::max(gmax, std::fabs(e.v));
    for (int l = 0; l < L; ++l)
        for (const Trip &e : G[l]) {
            if (d->m[e.r] != d->m[e.c]) return fail(MQCT_ERR_INVALID_ARG, "G couples states of different m (Eq. 6)");
            const Trip key{e.c, e.r, 0.0};
            auto it = std::lower_bound(G[l].begin(), G[l].end(), key, trip_less);
            double vt = (it != G[l].end() && it->r == e.c && it->c == e.r) ? it->v : 0.0;
            if (std::fabs(vt - e.v) > 1e-12 * gmax) return fail(MQCT_ERR_INVALID_ARG, "G is not symmetric");
        }

    // ---- grid data
    for (size_t i = 0; i < (size_t)L * ng; ++i)
        if (!std::isfinite(d->v[i])) return fail(MQCT_ERR_INVALID_ARG, "non-finite v");
    for (int i = 0; i < 2 * L; ++i)
        if (!std::isfinite(d->dv_ends[i])) return fail(MQCT_ERR_INVALID_ARG, "non-finite dv_ends");

    mqct_system_s *hs = new (std::nothrow) mqct_system_s();
    if (!hs) return fail(MQCT_ERR_OOM, "host allocation failed");
    System &S = hs->s;

    // ---- internal order: blocks of equal m, largest block first, caller order inside
    std::map<int, std::vector<int>> blocks;
    for (int s = 0; s < n; ++s) blocks[d->m[s]].push_back(s);
    std::vector<std::vector<int>> bl;
    for (auto &kv : blocks) bl.push_back(kv.second);
    std::stable_sort(bl.begin(), bl.end(), [](const std::vector<int> &a, const std::vector<int> &b) { return a.size() > b.size(); });
    S.perm.clear();
    for (auto &b : bl) {
        S.max_block = std::max<int>(S.max_block, (int)b.size());
        for (int s : b) S.perm.push_back(s);
    }
    S.inv.assign(n, 0);
    for (int i = 0; i < n; ++i) S.inv[S.perm[i]] = i;
    S.lev.resize(n);
    for (int i = 0; i < n; ++i) S.lev[i] = d->level[S.perm[i]];

    // ---- Coriolis partners (same level and j, m +- 1), internal indices
    std::map<std::tuple<int, int, int>, int> where;
    for (int i = 0; i < n; ++i) where[{d->level[S.perm[i]], d->j[S.perm[i]], d->m[S.perm[i]]}] = i;
    std::vector<int> up(n), dn(n);
    std::vector<double> aup(n, 0.0), adn(n, 0.0);
    for (int i = 0; i < n; ++i) {
        int s = S.perm[i], j = d->j[s], m = d->m[s], lv = d->level[s];
        up[i] = dn[i] = i;
        if (j < 0) continue;
        auto iu = where.find({lv, j, m + 1}), id = where.find({lv, j, m - 1});
        double jj = (double)j * (j + 1);
        if (iu != where.end()) { up[i] = iu->second; aup[i] = std::sqrt(jj - (double)m * (m + 1)); }
        if (id != where.end()) { dn[i] = id->second; adn[i] = std::sqrt(jj - (double)m * (m - 1)); }
    }

    // ---- splines of v_lambda and of the parameter derivatives
    // on the logarithmic grid the spline variable is x = ln R (uniform knots), end slopes R dv/dR
    const int n_int = ng - 1;
    const bool glog = d->grid_kind == MQCT_GRID_LOG;
    const double x0 = glog ? std::log(d->r_min) : d->r_min;
    const double h = glog ? (std::log(d->r_max) - std::log(d->r_min)) / (ng - 1) : (d->r_max - d->r_min) / (ng - 1);
    const double e0 = glog ? d->r_min : 1.0, e1 = glog ? d->r_max : 1.0;
    std::vector<std::vector<dbl4>> vc(L);
    std::vector<dbl4> vcoef((size_t)L * n_int);
    for (int l = 0; l < L; ++l) {
        clamped_spline(ng, h, d->v + (size_t)l * ng, e0 * d->dv_ends[2 * l], e1 * d->dv_ends[2 * l + 1], vc[l]);
        std::copy(vc[l].begin(), vc[l].end(), vcoef.begin() + (size_t)l * n_int);
    }
    std::vector<dbl4> dvcoef;
    if (P > 0) {
        dvcoef.resize((size_t)P * L * n_int);
        std::vector<dbl4> tmp;
        for (int p = 0; p < P; ++p)
            for (int l = 0; l < L; ++l) {
                size_t o = (size_t)p * L + l;
                for (int k = 0; k < ng; ++k)
                    if (!std::isfinite(d->dv_dparam[o * ng + k])) { delete hs; return fail(MQCT_ERR_INVALID_ARG, "non-finite dv_dparam"); }
                clamped_spline(ng, h, d->dv_dparam + o * ng, e0 * d->ddv_ends[2 * o], e1 * d->ddv_ends[2 * o + 1], tmp);
                std::copy(tmp.begin(), tmp.end(), dvcoef.begin() + o * n_int);
            }
    }

    // ---- G in internal indices, per term row lists; diagonal
    std::vector<double> diag_g((size_t)L * n, 0.0);
    std::vector<std::vector<std::vector<Entry>>> grows(L, std::vector<std::vector<Entry>>(n));
    for (int l = 0; l < L; ++l)
        for (const Trip &e : G[l]) {
            int r = S.inv[e.r], c = S.inv[e.c];
            if (e.v == 0.0) continue;
            grows[l][r].push_back({r, c, e.v});
            if (r == c) diag_g[(size_t)l * n + r] = e.v;
        }
    for (int l = 0; l < L; ++l)
        for (auto &row : grows[l]) std::sort(row.begin(), row.end(), [](const Entry &a, const Entry &b) { return a.c < b.c; });

    // ---- terms whose G is the identity (the isotropic part of the potential, e.g. lambda = 0 of a
    // Legendre expansion), up to the rounding of their construction
    unsigned long long iso_mask = 0;
    for (int l = 0; l < L; ++l) {
        bool ident = true;
        for (int r = 0; r < n && ident; ++r)
            if (grows[l][r].size() != 1 || grows[l][r][0].c != r || std::fabs(grows[l][r][0].v - 1.0) > 1e-13) ident = false;
        if (ident) iso_mask |= 1ull << l;
    }
    if ((d->flags & MQCT_DECOUPLED_TRAJ) && !iso_mask) {
        delete hs;
        return fail(MQCT_ERR_INVALID_ARG, "MQCT_DECOUPLED_TRAJ needs an expansion term whose G is the identity");
    }

    // ---- truncation (Sec. III): M_rc = sum_l G^l_rc v_l(R) from the splines at the two
    // reference distances; an element at or below the threshold at both is dropped from every term
    int64_t n_dropped = 0;
    if (d->trunc_threshold > 0.0) {
        double va[2][kMaxTerms];
        for (int q = 0; q < 2; ++q) {
            const double R = d->trunc_r[q], X = glog ? std::log(R) : R;
            int k = (int)std::floor((X - x0) / h);
            k = std::max(0, std::min(n_int - 1, k));
            const double x = X - (x0 + k * h);
            for (int l = 0; l < L; ++l) {
                const dbl4 &c = vc[l][k];
                va[q][l] = c.x + x * (c.y + x * (c.z + x * c.w));
            }
        }
        const double thr = d->trunc_threshold;
        for (int r = 0; r < n; ++r) {
            std::map<int, std::pair<double, double>> mrow;  // column -> (M(R_a), M(R_b)), terms in order
            for (int l = 0; l < L; ++l)
                for (auto &e : grows[l][r]) {
                    auto &m = mrow[e.c];
                    m.first += va[0][l] * e.v;
                    m.second += va[1][l] * e.v;
                }
            for (auto &kv : mrow) {
                if (std::fabs(kv.second.first) > thr || std::fabs(kv.second.second) > thr) continue;
                ++n_dropped;
                const int c = kv.first;
                for (int l = 0; l < L; ++l) {
                    auto &row = grows[l][r];
                    row.erase(std::remove_if(row.begin(), row.end(), [c](const Entry &e) { return e.c == c; }), row.end());
                }
                if (c == r)
                    for (int l = 0; l < L; ++l) diag_g[(size_t)l * n + r] = 0.0;
            }
        }
    }

    const int n_slices = (n + kSlice - 1) / kSlice;
    DevSys &D = S.h;
    std::memset(&D, 0, sizeof(D));
    D.n = n; D.n_levels = n_levels; D.L = L; D.n_int = n_int; D.n_slices = n_slices; D.P = P;
    D.path = d->path; D.precision = d->precision; D.flags = d->flags;
    D.mu = d->mu; D.r_min = d->r_min; D.h = h; D.inv_h = 1.0 / h;
    D.grid_log = glog ? 1 : 0; D.x0 = x0;
    D.id_mask = iso_mask;
    D.adapt_tol = d->adapt_tol;
    D.adapt_hmax = d->adapt_tol > 0.0 ? (d->adapt_hmax > 0 ? (double)d->adapt_hmax : 16.0) : 1.0;

    mqct_status st = MQCT_OK;
    auto up_ = [&](auto &v, auto **dst) { if (st == MQCT_OK) st = upload(S, v, dst); };
    up_(lev_e, &D.lev_energy);
    if (d->precision != MQCT_FP64) {
        std::vector<float> lev_ef(lev_e.begin(), lev_e.end());
        up_(lev_ef, &D.lev_energy_f);
    }
    up_(S.lev, &D.lev);
    up_(S.perm, &D.perm);
    up_(S.inv, &D.inv);
    up_(up, &D.up);
    up_(dn, &D.dn);
    up_(aup, &D.aup);
    up_(adn, &D.adn);
    up_(diag_g, &D.diag_g);
    up_(vcoef, &D.vcoef);
    if (P > 0) up_(dvcoef, &D.dvcoef);
    if (P > 0 && d->precision != MQCT_FP64) {
        // FP32 copy for the mixed-precision adjoint
        std::vector<float4> dvf(dvcoef.size());
        for (size_t i = 0; i < dvcoef.size(); ++i)
            dvf[i] = make_float4((float)dvcoef[i].x, (float)dvcoef[i].y, (float)dvcoef[i].z, (float)dvcoef[i].w);
        up_(dvf, &D.dvcoef_f);
    }

    S.info.n_states = n;
    S.info.n_levels = n_levels;
    S.info.n_terms = L;
    S.info.n_grid = ng;
    S.info.n_blocks = (int)bl.size();
    S.info.max_block = S.max_block;
    S.info.path = d->path;
    S.info.trunc_dropped = n_dropped;
    S.info.grid_kind = d->grid_kind;
    S.info.precision = d->precision;

    if (d->path == MQCT_PATH_PLAIN) {
        // union pattern of all terms, coefficients sum_l G^l_rc coef_l[k]
        std::vector<std::vector<Entry>> rows(n);
        for (int r = 0; r < n; ++r) {
            std::map<int, int> cs;
            for (int l = 0; l < L; ++l)
                for (auto &e : grows[l][r]) cs[e.c] = 0;
            for (auto &kv : cs) rows[r].push_back({r, kv.first, 0.0});
        }
        Sell sl = make_sell(n, rows);
        const size_t nnz_pad = sl.cols.size();
        // per row: map column -> position, and per term the G values in that order
        std::vector<std::vector<std::vector<double>>> gv(n);
        for (int r = 0; r < n; ++r) {
            gv[r].assign(rows[r].size(), std::vector<double>(L, 0.0));
            for (int l = 0; l < L; ++l)
                for (auto &e : grows[l][r]) {
                    auto it = std::lower_bound(rows[r].begin(), rows[r].end(), e.c, [](const Entry &a, int c) { return a.c < c; });
                    gv[r][it - rows[r].begin()][l] = e.v;
                }
        }
        // FP64 systems: (c0, c1) and (c2, c3) planes; FP32 systems (stage-synchronous sparse path):
        // one float4 per element and interval
        const bool f32 = d->precision == MQCT_FP32;
        std::vector<double2> T01(f32 ? 0 : nnz_pad * n_int), T23(f32 ? 0 : nnz_pad * n_int);
        std::vector<float4> T4(f32 ? nnz_pad * n_int : 0);
        for (size_t e = 0; e < nnz_pad; ++e) {
            int r = sl.row_of[e], k0 = sl.src[e];
            for (int k = 0; k < n_int; ++k) {
                double c[4] = {0, 0, 0, 0};
                if (k0 >= 0)
                    for (int l = 0; l < L; ++l) {
                        double g = gv[r][k0][l];
                        if (g == 0.0) continue;
                        const dbl4 &q = vc[l][k];
                        c[0] += g * q.x; c[1] += g * q.y; c[2] += g * q.z; c[3] += g * q.w;
                    }
                if (f32) {
                    T4[(size_t)k * nnz_pad + e] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)c[3]);
                } else {
                    T01[(size_t)k * nnz_pad + e] = make_double2(c[0], c[1]);
                    T23[(size_t)k * nnz_pad + e] = make_double2(c[2], c[3]);
                }
            }
        }
        int64_t nnz = 0;
        for (auto &r : rows) nnz += (int64_t)r.size();
        D.nnz_pad = (long long)nnz_pad;
        up_(sl.off, &D.sl_off);
        up_(sl.cols, &D.cols);
        if (f32) {
            up_(T4, &D.T4f);
            std::vector<float> aupf(aup.begin(), aup.end()), adnf(adn.begin(), adn.end());
            up_(aupf, &D.aupf);
            up_(adnf, &D.adnf);
        } else {
            up_(T01, &D.T01);
            up_(T23, &D.T23);
        }
        S.info.table_nnz = nnz;
        S.info.table_bytes = (int64_t)nnz_pad * n_int * (f32 ? 16 : 32);
    }
    if (d->path == MQCT_PATH_FACTORISED || P > 0) {
        // identity terms are applied directly; others get one sliced-ELL matrix each (the
        // adjoint always works on the per-term form, so it is built whenever P > 0)
        std::vector<int> fterm, foff, fcols;
        std::vector<double> fval;
        unsigned long long idm = 0;
        int64_t gnnz = 0;
        for (int l = 0; l < L; ++l) {
            // the identity (e.g. G^0 of a Legendre expansion) up to rounding of its construction
            bool ident = true;
            for (int r = 0; r < n && ident; ++r) {
                if (grows[l][r].size() != 1 || grows[l][r][0].c != r || std::fabs(grows[l][r][0].v - 1.0) > 1e-13)
                    ident = false;
            }
            bool empty = true;
            for (int r = 0; r < n; ++r) if (!grows[l][r].empty()) empty = false;
            if (ident) { idm |= 1ull << l; continue; }
            if (empty) continue;
            Sell sl = make_sell(n, grows[l]);
            fterm.push_back(l);
            int base = (int)fcols.size();
            for (int s2 = 0; s2 <= n_slices; ++s2) foff.push_back(base + sl.off[s2]);
            for (size_t e = 0; e < sl.cols.size(); ++e) {
                fcols.push_back(sl.cols[e]);
                int r = sl.row_of[e], k0 = sl.src[e];
                fval.push_back(k0 >= 0 ? grows[l][r][k0].v : 0.0);
            }
            for (int r = 0; r < n; ++r) gnnz += (int64_t)grows[l][r].size();
        }
        D.n_f = (int)fterm.size();
        D.id_mask = idm;
        up_(fterm, &D.f_term);
        up_(foff, &D.f_sl_off);
        up_(fcols, &D.f_cols);
        up_(fval, &D.f_val);
        if (d->precision != MQCT_FP64) {
            // FP32 copies for the mixed-precision kernels: the sliced-ELL values, the spline
            // coefficients of v_lambda and the Coriolis ladder factors
            std::vector<float> fvalf(fval.begin(), fval.end());
            std::vector<float4> vf(vcoef.size());
            for (size_t i = 0; i < vcoef.size(); ++i)
                vf[i] = make_float4((float)vcoef[i].x, (float)vcoef[i].y, (float)vcoef[i].z, (float)vcoef[i].w);
            std::vector<float> aupf(aup.begin(), aup.end()), adnf(adn.begin(), adn.end());
            up_(fvalf, &D.f_valf);
            std::vector<int2> fcv(fcols.size());
            for (size_t i = 0; i < fcols.size(); ++i) {
                int bits;
                std::memcpy(&bits, &fvalf[i], sizeof bits);
                fcv[i] = make_int2(fcols[i], bits);
            }
            up_(fcv, &D.f_cvf);
            up_(aupf, &D.aupf);
            up_(adnf, &D.adnf);
            up_(vf, &D.vcoef_f);
        }
        if (d->precision == MQCT_BF16X3) {
            // pack whole m-blocks (contiguous in the internal order) into row tiles of <= 128 rows
            std::vector<int> t0{0};
            int rows = 0;
            for (auto &b : bl) {
                const int sz = (int)b.size();
                if (sz > 128) {
                    release(S);
                    delete hs;
                    return fail(MQCT_ERR_UNSUPPORTED, "BF16X3: an m-block has more than 128 states");
                }
                if (rows + sz > 128) { t0.push_back(t0.back() + rows); rows = 0; }
                rows += sz;
            }
            t0.push_back(t0.back() + rows);
            const int nt = (int)t0.size() - 1;
            // block-diagonal 128 x 128 tiles, BF16 hi/lo split, canonical K-major MMA layout:
            // element (r, k) at byte (r/8)*2048 + (k/8)*128 + (r%8)*16 + (k%8)*2; per tile the
            // mask of its 16-column K chunks that hold a non-zero (the others are skipped)
            auto bf16_bits = [](float x) -> uint16_t {
                uint32_t u;
                std::memcpy(&u, &x, 4);
                u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
                return (uint16_t)(u >> 16);
            };
            auto bf16_val = [](uint16_t h) -> float {
                uint32_t u = (uint32_t)h << 16;
                float x;
                std::memcpy(&x, &u, 4);
                return x;
            };
            std::vector<uint16_t> tiles((size_t)fterm.size() * nt * 2 * 16384, 0);
            std::vector<uint8_t> kmask((size_t)fterm.size() * nt, 0);
            for (size_t f = 0; f < fterm.size(); ++f) {
                const int l = fterm[f];
                for (int t = 0; t < nt; ++t) {
                    uint16_t *hi = tiles.data() + (((size_t)f * nt + t) * 2) * 16384, *lo = hi + 16384;
                    uint8_t &km = kmask[(size_t)f * nt + t];
                    for (int r = t0[t]; r < t0[t + 1]; ++r)
                        for (auto &e : grows[l][r]) {
                            const int rr = r - t0[t], kk = e.c - t0[t];
                            km |= (uint8_t)(1u << (kk >> 4));
                            const float v = (float)e.v;
                            const uint16_t h = bf16_bits(v);
                            const size_t off = ((size_t)(rr >> 3) * 2048 + (size_t)(kk >> 3) * 128 + (rr & 7) * 16 + (kk & 7) * 2) / 2;
                            hi[off] = h;
                            lo[off] = bf16_bits(v - bf16_val(h));
                        }
                    if (!km) km = 1;  // an all-zero tile still writes its (zero) product
                    S.info.tc_kchunks += __builtin_popcount(km);
                }
            }
            D.n_tiles = nt;
            up_(t0, &D.tile_r0);
            up_(tiles, &D.g_tiles);
            up_(kmask, &D.g_kmask);
        }
        S.info.glambda_nnz = gnnz;
        S.info.n_coupling_terms = D.n_f;
        S.info.n_row_tiles = D.n_tiles;
    }
    if (st == MQCT_OK) {
        cudaError_t e = cudaMalloc(&S.d, sizeof(DevSys));
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc");
        else {
            S.info.device_bytes += sizeof(DevSys);
            e = cudaMemcpy(S.d, &D, sizeof(DevSys), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpy");
        }
    }
    if (st != MQCT_OK) {
        release(S);
        delete hs;
        return st;
    }
    *out = hs;
    return MQCT_OK;
}

extern "C" mqct_status mqct_destroy_system(mqct_system sys)
{
    if (!sys) return MQCT_OK;
    release(sys->s);
    delete sys;
    return MQCT_OK;
}

extern "C" mqct_status mqct_system_info(mqct_system sys, mqct_system_info_t *out)
{
    if (!sys || !out) return fail(MQCT_ERR_INVALID_ARG, "mqct_system_info: NULL argument");
    *out = sys->s.info;
    return MQCT_OK;
}

extern "C" const char *mqct_last_error(void) { return last_error_cstr(); }

extern "C" int64_t mqct_last_launch_count(void) { return g_launches; }

extern "C" const char *mqct_version(void) { return "mqct-gb300 0.1 (sm_103a)"; }
