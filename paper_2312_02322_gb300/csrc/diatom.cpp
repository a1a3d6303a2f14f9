// Built-in atom + linear rotor system (host only).
//
// Basis (Eq. 2): Y_jm, j <= jmax, all m, j-major order s = j^2 + j + m, E_j = B j(j+1).
// Coupling (Eq. 6 with the Legendre expansion of Eq. 12): G^lambda_{(j''m),(j'm)} =
// <j'' m | P_lambda(cos theta) | j' m>, the Gaunt integral of Eq. 15.  Here it is
// evaluated as the exact Gauss-Legendre quadrature of the normalised associated
// Legendre functions (the integrand is a polynomial of degree j'' + j' + lambda in
// cos theta), with the selection rules of Eq. 15 (m'' = m', triangle rule,
// j' + j'' + lambda even) applied to the structural zeros.
// PES: V(R, theta) = sum_l A_l exp(-beta_l R) P_l(cos theta) - C6 R^-6 (1 - exp(-(R/Rd)^6)).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace mqct {

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace mqct

namespace {

// theta[j] = normalised associated Legendre function of order m (int_{-1}^{1} theta^2 dx = 1)
// at x for j = m..jmax (entries j < m are left at zero).
void norm_assoc_legendre(int jmax, int m, double x, std::vector<double> &th)
{
    th.assign(jmax + 1, 0.0);
    if (m > jmax) return;
    double s = std::sqrt(std::fmax(0.0, 1.0 - x * x));
    double t = 1.0 / std::sqrt(2.0);
    for (int k = 1; k <= m; ++k) t *= std::sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
    th[m] = t;
    if (m + 1 <= jmax) th[m + 1] = std::sqrt(2.0 * m + 3.0) * x * t;
    for (int j = m + 2; j <= jmax; ++j) {
        double a = std::sqrt((4.0 * j * j - 1.0) / ((double)j * j - (double)m * m));
        double b = std::sqrt((((double)(j - 1) * (j - 1)) - (double)m * m) / (4.0 * (j - 1) * (j - 1) - 1.0));
        th[j] = a * (x * th[j - 1] - b * th[j - 2]);
    }
}

double legendre(int l, double x)
{
    double p0 = 1.0, p1 = x;
    if (l == 0) return 1.0;
    for (int k = 2; k <= l; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

template <class T>
T *alloc_copy(const std::vector<T> &v)
{
    T *p = static_cast<T *>(std::malloc(sizeof(T) * (v.empty() ? 1 : v.size())));
    if (p && !v.empty()) std::memcpy(p, v.data(), sizeof(T) * v.size());
    return p;
}

}  // namespace

namespace mqct {

// Grid tables of the expansion coefficients v_l(R) = A_l exp(-beta_l R) (+ the damped -C6 R^-6
// dispersion on term 0), their analytic end slopes for the clamped spline and, with
// with_params, the derivative tables for theta = (A_0..A_{L-1}, beta_0..beta_{L-1}); then the
// host arrays of *out (freed by mqct_free_desc).
mqct_status finish_desc(mqct_system_desc *out, const char *who, const std::vector<double> &energy,
                        const std::vector<int32_t> &level, const std::vector<int32_t> &jq,
                        const std::vector<int32_t> &mq, double mu, int L, const std::vector<int32_t> &gt,
                        const std::vector<int32_t> &gr, const std::vector<int32_t> &gc, const std::vector<double> &gv,
                        const double *A, const double *beta, double c6, double rd, int ng, double r_min, double r_max,
                        bool with_params, int path, int precision, int grid_kind)
{
    const int n = (int)energy.size();
    // grid point k: uniform in R, or in ln R (MQCT_GRID_LOG)
    const double h = (r_max - r_min) / (ng - 1);
    const double hl = grid_kind == MQCT_GRID_LOG ? (std::log(r_max) - std::log(r_min)) / (ng - 1) : 0.0;
    auto grid_r = [&](int k) { return grid_kind == MQCT_GRID_LOG ? r_min * std::exp(k * hl) : r_min + k * h; };
    std::vector<double> v((size_t)L * ng), ends((size_t)L * 2);
    auto c6term = [&](double R) { return -c6 * std::pow(R, -6.0) * (1.0 - std::exp(-std::pow(R / rd, 6.0))); };
    auto c6slope = [&](double R) {
        double u = std::pow(R / rd, 6.0);
        return 6.0 * c6 * std::pow(R, -7.0) * (1.0 - std::exp(-u)) - 6.0 * c6 * u * std::exp(-u) * std::pow(R, -7.0);
    };
    for (int l = 0; l < L; ++l) {
        for (int k = 0; k < ng; ++k) {
            double R = grid_r(k);
            v[(size_t)l * ng + k] = A[l] * std::exp(-beta[l] * R) + (l == 0 ? c6term(R) : 0.0);
        }
        for (int e = 0; e < 2; ++e) {
            double R = e ? r_max : r_min;
            ends[2 * l + e] = -beta[l] * A[l] * std::exp(-beta[l] * R) + (l == 0 ? c6slope(R) : 0.0);
        }
    }
    std::vector<double> dvp, dvpe;
    int P = 0;
    if (with_params) {
        P = 2 * L;
        dvp.assign((size_t)P * L * ng, 0.0);
        dvpe.assign((size_t)P * L * 2, 0.0);
        for (int l = 0; l < L; ++l) {
            for (int k = 0; k < ng; ++k) {
                double R = grid_r(k), ex = std::exp(-beta[l] * R);
                dvp[((size_t)l * L + l) * ng + k] = ex;                      // d/dA_l
                dvp[((size_t)(L + l) * L + l) * ng + k] = -R * A[l] * ex;    // d/dbeta_l
            }
            for (int e = 0; e < 2; ++e) {
                double R = e ? r_max : r_min, ex = std::exp(-beta[l] * R);
                dvpe[((size_t)l * L + l) * 2 + e] = -beta[l] * ex;
                dvpe[((size_t)(L + l) * L + l) * 2 + e] = A[l] * ex * (beta[l] * R - 1.0);
            }
        }
    }

    out->n_states = n;
    out->energy = alloc_copy(energy);
    out->level = alloc_copy(level);
    out->j = alloc_copy(jq);
    out->m = alloc_copy(mq);
    out->mu = mu;
    out->n_terms = L;
    out->G = nullptr;
    out->g_nnz = (int64_t)gv.size();
    out->g_term = alloc_copy(gt);
    out->g_row = alloc_copy(gr);
    out->g_col = alloc_copy(gc);
    out->g_val = alloc_copy(gv);
    out->n_grid = ng;
    out->r_min = r_min;
    out->r_max = r_max;
    out->v = alloc_copy(v);
    out->dv_ends = alloc_copy(ends);
    out->n_params = P;
    out->dv_dparam = P ? alloc_copy(dvp) : nullptr;
    out->ddv_ends = P ? alloc_copy(dvpe) : nullptr;
    out->path = path;
    out->precision = precision;
    out->flags = 0;
    out->grid_kind = grid_kind;
    if (!out->energy || !out->level || !out->j || !out->m || !out->g_term || !out->g_row || !out->g_col ||
        !out->g_val || !out->v || !out->dv_ends || (P && (!out->dv_dparam || !out->ddv_ends))) {
        mqct_free_desc(out);
        return fail(MQCT_ERR_OOM, std::string(who) + ": host allocation failed");
    }
    return MQCT_OK;
}

}  // namespace mqct

extern "C" mqct_status mqct_build_diatom(const mqct_diatom_params *p, mqct_system_desc *out)
{
    using namespace mqct;
    if (!p || !out) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_diatom: NULL argument");
    std::memset(out, 0, sizeof(*out));
    const int jmax = p->jmax, L = p->n_terms, ng = p->n_grid;
    if (jmax < 0 || jmax > 500) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_diatom: jmax outside [0, 500]");
    if (L < 1 || L > 16) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_diatom: n_terms outside [1, 16]");
    if (ng < 4) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_diatom: n_grid < 4");
    if (!(p->r_max > p->r_min) || !(p->r_min > 0)) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_diatom: bad grid range");
    if (!(p->mu > 0)) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_diatom: mu <= 0");
    if (!(p->rd > 0)) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_diatom: rd <= 0");
    if (p->grid_kind != MQCT_GRID_UNIFORM && p->grid_kind != MQCT_GRID_LOG)
        return fail(MQCT_ERR_INVALID_ARG, "mqct_build_diatom: unknown grid_kind");
    const int n = (jmax + 1) * (jmax + 1);

    std::vector<double> energy(n);
    std::vector<int32_t> level(n), jq(n), mq(n);
    for (int j = 0; j <= jmax; ++j)
        for (int m = -j; m <= j; ++m) {
            int s = j * j + j + m;
            energy[s] = p->bconst * j * (j + 1);
            level[s] = j;
            jq[s] = j;
            mq[s] = m;
        }

    // G^lambda by exact Gauss-Legendre quadrature, m-block by m-block
    const int nq = jmax + L + 4;
    std::vector<double> xq, wq;
    gauss_legendre(nq, xq, wq);
    std::vector<std::vector<double>> th(nq);
    std::vector<double> pl((size_t)L * nq);
    for (int l = 0; l < L; ++l)
        for (int q = 0; q < nq; ++q) pl[(size_t)l * nq + q] = legendre(l, xq[q]);
    std::vector<int32_t> gt, gr, gc;
    std::vector<double> gv;
    for (int m = 0; m <= jmax; ++m) {
        // the normalised associated Legendre functions of order m at the nodes, once per m
        for (int q = 0; q < nq; ++q) norm_assoc_legendre(jmax, m, xq[q], th[q]);
        for (int l = 0; l < L; ++l) {
            const double *plq = pl.data() + (size_t)l * nq;
            for (int j2 = m; j2 <= jmax; ++j2)
                for (int j1 = std::max(m, j2 - l); j1 <= std::min(jmax, j2 + l); ++j1) {
                    if (l > j1 + j2 || ((j1 + j2 + l) & 1)) continue;
                    double acc = 0.0;
                    for (int q = 0; q < nq; ++q) acc += wq[q] * th[q][j2] * plq[q] * th[q][j1];
                    for (int sm = (m == 0 ? 1 : -1); sm <= 1; sm += 2) {
                        int mm = sm * m;
                        gt.push_back(l);
                        gr.push_back(j2 * j2 + j2 + mm);
                        gc.push_back(j1 * j1 + j1 + mm);
                        gv.push_back(acc);
                    }
                }
        }
    }

    const mqct_status st = mqct::finish_desc(out, "mqct_build_diatom", energy, level, jq, mq, p->mu, L, gt, gr, gc, gv,
                                             p->A, p->beta, p->c6, p->rd, ng, p->r_min, p->r_max, p->with_params != 0,
                                             p->path, p->precision, p->grid_kind);
    if (st == MQCT_OK) {
        out->trunc_threshold = p->trunc_threshold;
        out->trunc_r[0] = p->trunc_r[0];
        out->trunc_r[1] = p->trunc_r[1];
    }
    return st;
}

extern "C" void mqct_free_desc(mqct_system_desc *d)
{
    if (!d) return;
    std::free((void *)d->energy);
    std::free((void *)d->level);
    std::free((void *)d->j);
    std::free((void *)d->m);
    std::free((void *)d->G);
    std::free((void *)d->g_term);
    std::free((void *)d->g_row);
    std::free((void *)d->g_col);
    std::free((void *)d->g_val);
    std::free((void *)d->v);
    std::free((void *)d->dv_ends);
    std::free((void *)d->dv_dparam);
    std::free((void *)d->ddv_ends);
    std::memset(d, 0, sizeof(*d));
}
