// Built-in atom + rigid asymmetric-top system (host only).
//
// Rotor states (Eq. 1): psi_{J tau M} = sum_K b_K sqrt((2J+1)/(8 pi^2)) D^{J*}_{MK}, with the b_K
// from diagonalising A Ja^2 + B Jb^2 + C Jc^2 in the symmetric-top functions (K along a).
// Here the rotor matrix is first brought to Wang's symmetrised functions, where it splits into
// four tridiagonal classes (K even / odd, (|K> +- |-K>)/sqrt2); each class is diagonalised by
// Sturm-sequence bisection followed by inverse iteration.  Eigenvectors never mix classes, so
// near-degenerate pairs of different symmetry (the K-doublets of high K_a) stay well defined.
//
// Coupling: G^{lam mu}_{s'' s'} = <J'' tau'' M | f_{lam mu} | J' tau' M> with the real angular
// function f_{lam mu} = (D^{lam*}_{0 mu} + (-1)^mu D^{lam*}_{0,-mu}) / (1 + delta_{mu 0}) -- the
// +-mu combination of Eq. 14 for an atom partner.  The alpha and gamma integrals are done in
// closed form (they select K'' = K' +- mu); the beta integral of three Wigner d-functions is an
// exact Gauss-Legendre quadrature in cos(beta) (the integrand is a polynomial of degree
// J'' + J' + lam).  This is the quadrature counterpart of the Eq. 16 closed form.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

struct Level {
    double E;
    int J, tau;
    std::vector<double> b;  // b[K + J]
};

// number of eigenvalues of the symmetric tridiagonal (d, e) below x
int sturm_count(const std::vector<double> &d, const std::vector<double> &e, double x)
{
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < d.size(); ++i) {
        double off = i ? e[i - 1] * e[i - 1] : 0.0;
        q = d[i] - x - (i ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// eigenpairs of a symmetric tridiagonal matrix: eigenvalues by bisection on the Sturm count,
// eigenvectors by two steps of inverse iteration (dense elimination with partial pivoting;
// the classes are at most jmax/2 + 1 long)
void tridiag_eigen(const std::vector<double> &d, const std::vector<double> &e, std::vector<double> &w,
                   std::vector<std::vector<double>> &vec)
{
    const int n = (int)d.size();
    double lo = d[0], hi = d[0], scale = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = (i ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    scale = std::max(std::fabs(lo), std::fabs(hi));
    if (!(scale > 0.0)) scale = 1.0;
    w.assign(n, 0.0);
    vec.assign(n, std::vector<double>(n, 0.0));
    if (n == 1) {
        w[0] = d[0];
        vec[0][0] = 1.0;
        return;
    }
    for (int k = 0; k < n; ++k) {
        double a = lo - 1e-12 * scale, b = hi + 1e-12 * scale;
        for (int it = 0; it < 200 && b - a > 2e-16 * scale; ++it) {
            double c = 0.5 * (a + b);
            if (sturm_count(d, e, c) > k) b = c; else a = c;
        }
        w[k] = 0.5 * (a + b);
        std::vector<double> x(n, 1.0);
        for (int it = 0; it < 3; ++it) {
            // solve (T - (w + delta) I) y = x
            const double shift = w[k] + 1e-14 * scale;
            std::vector<double> M((size_t)n * n, 0.0), y = x;
            for (int i = 0; i < n; ++i) {
                M[(size_t)i * n + i] = d[i] - shift;
                if (i + 1 < n) M[(size_t)i * n + i + 1] = M[(size_t)(i + 1) * n + i] = e[i];
            }
            for (int c = 0; c < n; ++c) {
                int p = c;
                for (int r = c + 1; r < n; ++r)
                    if (std::fabs(M[(size_t)r * n + c]) > std::fabs(M[(size_t)p * n + c])) p = r;
                if (p != c) {
                    for (int j = 0; j < n; ++j) std::swap(M[(size_t)p * n + j], M[(size_t)c * n + j]);
                    std::swap(y[p], y[c]);
                }
                double piv = M[(size_t)c * n + c];
                if (piv == 0.0) piv = M[(size_t)c * n + c] = 1e-300;
                for (int r = c + 1; r < n; ++r) {
                    double f = M[(size_t)r * n + c] / piv;
                    if (f == 0.0) continue;
                    for (int j = c; j < n; ++j) M[(size_t)r * n + j] -= f * M[(size_t)c * n + j];
                    y[r] -= f * y[c];
                }
            }
            for (int r = n - 1; r >= 0; --r) {
                double s = y[r];
                for (int j = r + 1; j < n; ++j) s -= M[(size_t)r * n + j] * y[j];
                y[r] = s / M[(size_t)r * n + r];
            }
            double nrm = 0.0;
            for (double t : y) nrm += t * t;
            nrm = std::sqrt(nrm);
            for (int i = 0; i < n; ++i) x[i] = y[i] / nrm;
        }
        vec[k] = x;
    }
}

// all 2J+1 eigenstates of one J, ascending energy; b in the |J K> functions
void rotor_levels(int J, double A, double B, double C, std::vector<Level> &out)
{
    const double jj = (double)J * (J + 1);
    auto h = [&](int K) { return 0.5 * (B + C) * (jj - (double)K * K) + A * (double)K * K; };
    auto o = [&](int K) {  // <K+2|H|K>
        return 0.25 * (B - C) * std::sqrt((double)(J - K) * (J - K - 1) * (J + K + 1) * (J + K + 2));
    };
    std::vector<Level> lv;
    for (int cls = 0; cls < 4; ++cls) {
        const int par = cls >> 1;               // K parity
        const int minus = cls & 1;              // (|K> - |-K>) combination
        const int k0 = par ? 1 : (minus ? 2 : 0);
        std::vector<int> Ks;
        for (int K = k0; K <= J; K += 2) Ks.push_back(K);
        if (Ks.empty()) continue;
        const int n = (int)Ks.size();
        std::vector<double> d(n), e(n > 1 ? n - 1 : 0);
        for (int i = 0; i < n; ++i) {
            d[i] = h(Ks[i]);
            if (Ks[i] == 1) d[i] += (minus ? -1.0 : 1.0) * 0.25 * (B - C) * jj;
            if (i + 1 < n) e[i] = o(Ks[i]) * (Ks[i] == 0 ? std::sqrt(2.0) : 1.0);
        }
        std::vector<double> w;
        std::vector<std::vector<double>> v;
        tridiag_eigen(d, e, w, v);
        for (int k = 0; k < n; ++k) {
            int big = 0;
            for (int i = 1; i < n; ++i)
                if (std::fabs(v[k][i]) > std::fabs(v[k][big])) big = i;
            const double sg = v[k][big] < 0 ? -1.0 : 1.0;
            Level L;
            L.E = w[k];
            L.J = J;
            L.tau = 0;
            L.b.assign(2 * J + 1, 0.0);
            for (int i = 0; i < n; ++i) {
                const int K = Ks[i];
                const double c = sg * v[k][i];
                if (K == 0) { L.b[J] = c; continue; }
                L.b[K + J] = c * std::sqrt(0.5);
                L.b[-K + J] = (minus ? -c : c) * std::sqrt(0.5);
            }
            lv.push_back(std::move(L));
        }
    }
    std::sort(lv.begin(), lv.end(), [](const Level &a, const Level &b) { return a.E < b.E; });
    for (size_t i = 0; i < lv.size(); ++i) lv[i].tau = (int)i - J;
    for (auto &L : lv) out.push_back(std::move(L));
}

// Wigner d^j_{m' m}(beta) at x = cos(beta), Wigner's explicit sum (long double)
double wigner_d(int j, int mp, int m, double x)
{
    const long double c = std::sqrt((long double)(1.0 + x) / 2.0L), s = std::sqrt((long double)(1.0 - x) / 2.0L);
    auto lf = [](int k) { return std::lgamma((long double)k + 1.0L); };
    const long double pre = 0.5L * (lf(j + mp) + lf(j - mp) + lf(j + m) + lf(j - m));
    long double acc = 0.0L;
    const int smin = std::max(0, m - mp), smax = std::min(j + m, j - mp);
    for (int k = smin; k <= smax; ++k) {
        const int pc = 2 * j + m - mp - 2 * k, ps = mp - m + 2 * k;
        long double t = std::exp(pre - lf(j + m - k) - lf(k) - lf(mp - m + k) - lf(j - mp - k));
        t *= (pc ? std::pow(c, (long double)pc) : 1.0L) * (ps ? std::pow(s, (long double)ps) : 1.0L);
        acc += ((mp - m + k) & 1) ? -t : t;
    }
    return (double)acc;
}

}  // namespace

extern "C" mqct_status mqct_build_asym_top(const mqct_asym_params *p, mqct_system_desc *out)
{
    using namespace mqct;
    if (!p || !out) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: NULL argument");
    std::memset(out, 0, sizeof(*out));
    const int jmax = p->jmax, L = p->n_terms, ng = p->n_grid;
    if (jmax < 0 || jmax > 20) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: jmax outside [0, 20]");
    if (!(p->A >= p->B && p->B >= p->C && p->C > 0 && p->A > p->C))
        return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: need A >= B >= C > 0 and A > C");
    if (p->max_states < 1) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: max_states < 1");
    if (L < 1 || L > 64) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: n_terms outside [1, 64]");
    int lam_max = 0;
    for (int t = 0; t < L; ++t) {
        if (p->lam[t] < 0 || p->lam[t] > 8 || p->mproj[t] < 0 || p->mproj[t] > p->lam[t])
            return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: term needs 0 <= mu <= lambda <= 8");
        lam_max = std::max(lam_max, p->lam[t]);
    }
    if (ng < 4) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: n_grid < 4");
    if (!(p->r_max > p->r_min) || !(p->r_min > 0)) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: bad grid range");
    if (!(p->mu > 0)) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: mu <= 0");
    if (!(p->rd > 0)) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: rd <= 0");

    // ---- levels: all J <= jmax, ascending energy (ties: smaller J), whole multiplets
    std::vector<Level> all;
    for (int J = 0; J <= jmax; ++J) rotor_levels(J, p->A, p->B, p->C, all);
    std::stable_sort(all.begin(), all.end(), [](const Level &a, const Level &b) {
        return a.E < b.E || (a.E == b.E && a.J < b.J);
    });
    std::vector<Level> lv;
    int n = 0;
    for (auto &l : all) {
        if (n + 2 * l.J + 1 > p->max_states) break;
        n += 2 * l.J + 1;
        lv.push_back(l);
    }
    if (lv.empty()) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_asym_top: max_states below the first level");
    const int nl = (int)lv.size();
    std::vector<int> first(nl + 1, 0);
    for (int l = 0; l < nl; ++l) first[l + 1] = first[l] + 2 * lv[l].J + 1;
    std::vector<double> energy(n);
    std::vector<int32_t> level(n), jq(n), mq(n);
    for (int l = 0; l < nl; ++l)
        for (int M = -lv[l].J; M <= lv[l].J; ++M) {
            const int s = first[l] + M + lv[l].J;
            energy[s] = lv[l].E;
            level[s] = l;
            jq[s] = lv[l].J;
            mq[s] = M;
        }
    if (p->tau_out)
        for (int l = 0; l < nl; ++l) p->tau_out[l] = lv[l].tau;

    // ---- G by quadrature over cos(beta)
    int jtop = 0;
    for (auto &l : lv) jtop = std::max(jtop, l.J);
    const int nq = jtop + (lam_max + 1) / 2 + 2;  // 2 nq - 1 >= 2 jtop + lam_max
    std::vector<double> xq, wq;
    gauss_legendre(nq, xq, wq);
    // dJ[J][(M+J)(2J+1) + K+J][q]
    std::vector<std::vector<double>> dJ(jtop + 1);
    for (int J = 0; J <= jtop; ++J) {
        const int w = 2 * J + 1;
        dJ[J].assign((size_t)w * w * nq, 0.0);
        for (int M = -J; M <= J; ++M)
            for (int K = -J; K <= J; ++K)
                for (int q = 0; q < nq; ++q) dJ[J][(((size_t)(M + J) * w) + K + J) * nq + q] = wigner_d(J, M, K, xq[q]);
    }
    // dl[t][0/1][q] = d^lam_{0, +mu}, d^lam_{0, -mu}
    std::vector<double> dl((size_t)L * 2 * nq);
    for (int t = 0; t < L; ++t)
        for (int q = 0; q < nq; ++q) {
            dl[((size_t)t * 2 + 0) * nq + q] = wigner_d(p->lam[t], 0, p->mproj[t], xq[q]);
            dl[((size_t)t * 2 + 1) * nq + q] = wigner_d(p->lam[t], 0, -p->mproj[t], xq[q]);
        }
    std::vector<std::vector<int>> terms_of_mu(lam_max + 1);
    for (int t = 0; t < L; ++t) terms_of_mu[p->mproj[t]].push_back(t);
    std::vector<int32_t> gt, gr, gc;
    std::vector<double> gv;
    std::vector<double> Pp(nq), Pm(nq);
    for (int l2 = 0; l2 < nl; ++l2)
        for (int l1 = 0; l1 <= l2; ++l1) {
            const int J2 = lv[l2].J, J1 = lv[l1].J, w2 = 2 * J2 + 1, w1 = 2 * J1 + 1;
            if (std::abs(J2 - J1) > lam_max) continue;
            const double pref = 0.5 * std::sqrt((double)w2 * w1);
            const int Mmax = std::min(J1, J2);
            for (int M = -Mmax; M <= Mmax; ++M) {
                const double *d2 = dJ[J2].data() + (size_t)(M + J2) * w2 * nq;
                const double *d1 = dJ[J1].data() + (size_t)(M + J1) * w1 * nq;
                for (int mu = 0; mu <= lam_max; ++mu) {
                    if (terms_of_mu[mu].empty()) continue;
                    // K sums for K'' = K' + mu and K'' = K' - mu (independent of lambda)
                    std::fill(Pp.begin(), Pp.end(), 0.0);
                    std::fill(Pm.begin(), Pm.end(), 0.0);
                    for (int K1 = -J1; K1 <= J1; ++K1) {
                        const double b1 = lv[l1].b[K1 + J1];
                        if (b1 == 0.0) continue;
                        for (int sgn = 0; sgn < (mu ? 2 : 1); ++sgn) {
                            const int K2 = sgn ? K1 - mu : K1 + mu;
                            if (K2 < -J2 || K2 > J2) continue;
                            const double bb = lv[l2].b[K2 + J2] * b1;
                            if (bb == 0.0) continue;
                            double *P = sgn ? Pm.data() : Pp.data();
                            const double *x2 = d2 + (size_t)(K2 + J2) * nq, *x1 = d1 + (size_t)(K1 + J1) * nq;
                            for (int q = 0; q < nq; ++q) P[q] += bb * x2[q] * x1[q];
                        }
                    }
                    const double sg = (mu & 1) ? -1.0 : 1.0;
                    for (int t : terms_of_mu[mu]) {
                        const int lam = p->lam[t];
                        if (std::abs(J2 - J1) > lam || J2 + J1 < lam) continue;
                        const double *dp = dl.data() + (size_t)t * 2 * nq, *dm = dp + nq;
                        double acc = 0.0;
                        for (int q = 0; q < nq; ++q) acc += wq[q] * (Pp[q] * dp[q] + (mu ? sg * Pm[q] * dm[q] : 0.0));
                        const double g = pref * acc;
                        if (std::fabs(g) < 1e-14) continue;  // class selection rules: zero up to rounding
                        const int r = first[l2] + M + J2, c = first[l1] + M + J1;
                        gt.push_back(t); gr.push_back(r); gc.push_back(c); gv.push_back(g);
                        if (r != c) { gt.push_back(t); gr.push_back(c); gc.push_back(r); gv.push_back(g); }
                    }
                }
            }
        }
    std::vector<double> A(L), beta(L);
    for (int t = 0; t < L; ++t) { A[t] = p->coef[t]; beta[t] = p->beta[t]; }
    return finish_desc(out, "mqct_build_asym_top", energy, level, jq, mq, p->mu, L, gt, gr, gc, gv, A.data(),
                       beta.data(), p->c6, p->rd, ng, p->r_min, p->r_max, p->with_params != 0, p->path, p->precision, MQCT_GRID_UNIFORM);
}

namespace {

// Clebsch-Gordan coefficients <j1 m1 j2 m2 | J M> for all J, M, m1 of one (j1, j2), built from the
// angular-momentum algebra itself: the top state |J J> is the vector of the M = J subspace orthogonal
// to every |J' J>, J' > J (Gram-Schmidt), signed so that <j1 j1, j2 J-j1 | J J> > 0 (Condon-Shortley),
// and the others follow by the lowering operator J- = J1- + J2-.
struct CgTable {
    int j1 = 0, j2 = 0;
    std::vector<double> c;  // [(J - |j1-j2|)][M + J][m1 + j1]
    double get(int m1, int m2, int J, int M) const
    {
        if (m1 + m2 != M || std::abs(m1) > j1 || std::abs(m2) > j2 || J < std::abs(j1 - j2) || J > j1 + j2 ||
            std::abs(M) > J)
            return 0.0;
        const int w1 = 2 * j1 + 1, wJ = 2 * (j1 + j2) + 1;
        return c[((size_t)(J - std::abs(j1 - j2)) * wJ + (M + J)) * w1 + (m1 + j1)];
    }
};

CgTable cg_build(int j1, int j2)
{
    CgTable T;
    T.j1 = j1;
    T.j2 = j2;
    const int Jmin = std::abs(j1 - j2), Jmax = j1 + j2, w1 = 2 * j1 + 1, wJ = 2 * Jmax + 1;
    T.c.assign((size_t)(Jmax - Jmin + 1) * wJ * w1, 0.0);
    auto at = [&](int J, int M, int m1) -> double & {
        return T.c[((size_t)(J - Jmin) * wJ + (M + J)) * w1 + (m1 + j1)];
    };
    auto ok = [&](int m1, int M) { return std::abs(m1) <= j1 && std::abs(M - m1) <= j2; };
    for (int J = Jmax; J >= Jmin; --J) {
        // the M = J subspace: vectors over m1; residuals of the unit vectors after removing |J' J>
        std::vector<double> best;
        double bn = -1.0;
        for (int u = -j1; u <= j1; ++u) {
            if (!ok(u, J)) continue;
            std::vector<double> v(w1, 0.0);
            v[u + j1] = 1.0;
            for (int Jp = Jmax; Jp > J; --Jp) {
                double dot = 0.0;
                for (int m1 = -j1; m1 <= j1; ++m1) dot += at(Jp, J, m1) * v[m1 + j1];
                for (int m1 = -j1; m1 <= j1; ++m1) v[m1 + j1] -= dot * at(Jp, J, m1);
            }
            double nn = 0.0;
            for (double x : v) nn += x * x;
            if (nn > bn) { bn = nn; best = v; }
        }
        const double nrm = std::sqrt(bn);
        // Condon-Shortley: the component with m1 = j1 positive
        const double sg = best[2 * j1] < 0 ? -1.0 : 1.0;
        for (int m1 = -j1; m1 <= j1; ++m1) at(J, J, m1) = ok(m1, J) ? sg * best[m1 + j1] / nrm : 0.0;
        for (int M = J; M > -J; --M) {
            // J- |J M> = sqrt(J(J+1) - M(M-1)) |J M-1>
            const double f = std::sqrt((double)J * (J + 1) - (double)M * (M - 1));
            for (int m1 = -j1; m1 <= j1; ++m1) {
                if (!ok(m1, M - 1)) continue;
                const int m2 = M - 1 - m1;
                double v = 0.0;
                // from |m1 + 1, m2> by J1- and from |m1, m2 + 1> by J2-
                if (ok(m1 + 1, M)) v += std::sqrt((double)j1 * (j1 + 1) - (double)(m1 + 1) * m1) * at(J, M, m1 + 1);
                if (ok(m1, M)) v += std::sqrt((double)j2 * (j2 + 1) - (double)(m2 + 1) * m2) * at(J, M, m1);
                at(J, M - 1, m1) = v / f;
            }
        }
    }
    return T;
}

}  // namespace

extern "C" mqct_status mqct_build_molmol(const mqct_molmol_params *p, mqct_system_desc *out)
{
    using namespace mqct;
    if (!p || !out) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_molmol: NULL argument");
    std::memset(out, 0, sizeof(*out));
    const int L = p->n_terms, ng = p->n_grid;
    if (p->j1max < 0 || p->j1max > 8) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_molmol: j1max outside [0, 8]");
    if (!(p->A >= p->B && p->B >= p->C && p->C > 0 && p->A > p->C))
        return fail(MQCT_ERR_INVALID_ARG, "mqct_build_molmol: need A >= B >= C > 0 and A > C");
    if (p->n_j2 < 1 || p->n_j2 > 8) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_molmol: n_j2 outside [1, 8]");
    for (int i = 0; i < p->n_j2; ++i)
        if (p->j2[i] < 0 || p->j2[i] > 8) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_molmol: j2 outside [0, 8]");
    if (L < 1 || L > 64) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_molmol: n_terms outside [1, 64]");
    int lmax = 0;
    for (int t = 0; t < L; ++t) {
        const int a = p->lam1[t], m = p->mu1[t], b = p->lam2[t], c = p->lam[t];
        if (a < 0 || a > 8 || m < 0 || m > a || b < 0 || b > 8 || c < std::abs(a - b) || c > a + b)
            return fail(MQCT_ERR_INVALID_ARG, "mqct_build_molmol: term outside 0 <= mu1 <= lam1 <= 8, lam2 <= 8, triangle");
        lmax = std::max(lmax, std::max(a, b));
    }
    if (ng < 4) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_molmol: n_grid < 4");
    if (!(p->r_max > p->r_min) || !(p->r_min > 0)) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_molmol: bad grid range");
    if (!(p->mu > 0) || !(p->rd > 0)) return fail(MQCT_ERR_INVALID_ARG, "mqct_build_molmol: mu and rd must be > 0");

    // ---- molecule 1 levels (ascending j1, then energy) and the composite states of Eq. 3
    std::vector<Level> lv;
    for (int J = 0; J <= p->j1max; ++J) rotor_levels(J, p->A, p->B, p->C, lv);
    const int nl = (int)lv.size(), nj2 = p->n_j2;
    struct St { int l1, a, j, m; };
    std::vector<St> st;
    std::vector<double> energy;
    std::vector<int32_t> level, jq, mq;
    int j2max = 0;
    for (int i = 0; i < nj2; ++i) j2max = std::max(j2max, p->j2[i]);
    for (int l = 0; l < nl; ++l)
        for (int i = 0; i < nj2; ++i) {
            const int J1 = lv[l].J, a = p->j2[i];
            for (int j = std::abs(J1 - a); j <= J1 + a; ++j)
                for (int m = -j; m <= j; ++m) {
                    st.push_back({l, a, j, m});
                    energy.push_back(lv[l].E + p->bconst2 * a * (a + 1));
                    level.push_back(l * nj2 + i);
                    jq.push_back(j);
                    mq.push_back(m);
                }
        }
    const int n = (int)st.size();
    // ---- Clebsch-Gordan tables of the couplings j1 x j2 -> j and lam1 x lam2 -> lam
    const int jtop = std::max(p->j1max, j2max);
    std::vector<CgTable> cgt((size_t)(jtop + 1) * (jtop + 1));
    for (int a = 0; a <= jtop; ++a)
        for (int b = 0; b <= jtop; ++b) cgt[(size_t)a * (jtop + 1) + b] = cg_build(a, b);
    auto CG = [&](int a, int ma, int b, int mb, int J, int M) {
        return cgt[(size_t)a * (jtop + 1) + b].get(ma, mb, J, M);
    };
    std::vector<CgTable> cgl((size_t)(lmax + 1) * (lmax + 1));
    for (int a = 0; a <= lmax; ++a)
        for (int b = 0; b <= lmax; ++b) cgl[(size_t)a * (lmax + 1) + b] = cg_build(a, b);
    // ---- one-molecule integrals over x = cos(beta) (Gauss-Legendre, exact for these polynomials)
    const int nq = jtop + lmax / 2 + 3;
    std::vector<double> xq, wq;
    gauss_legendre(nq, xq, wq);
    const double pi = 3.14159265358979323846;
    // d^j_{m k}(beta) at the nodes, j <= dmax
    const int dmax = std::max(jtop, lmax), wd = 2 * dmax + 1;
    std::vector<double> dtab((size_t)(dmax + 1) * wd * wd * nq, 0.0);
    auto dref = [&](int j, int mm, int k) -> double * {
        return dtab.data() + ((((size_t)j * wd + (mm + dmax)) * wd) + (k + dmax)) * nq;
    };
    for (int j = 0; j <= dmax; ++j)
        for (int mm = -j; mm <= j; ++mm)
            for (int k = -j; k <= j; ++k)
                for (int q = 0; q < nq; ++q) dref(j, mm, k)[q] = wigner_d(j, mm, k, xq[q]);
    // molecule 1: I1 = <J'' tau'' m1+eta| D^{lam1*}_{eta nu} |J' tau' m1> (Eq. 16's integral: 4 pi^2 from
    // alpha and gamma, the product of three d-functions over beta, the b_K of Eq. 1); memoised
    std::unordered_map<long long, double> memo1, memo2;
    auto I1 = [&](int l2, int l1, int m1, int eta, int lam1, int nu) {
        const int J2 = lv[l2].J, J1 = lv[l1].J, n1 = m1 + eta;
        if (std::abs(n1) > J2 || std::abs(m1) > J1 || std::abs(eta) > lam1 || std::abs(nu) > lam1) return 0.0;
        const long long key = ((((((long long)l2 * 256 + l1) * 32 + (m1 + 16)) * 32 + (eta + 16)) * 16 + lam1) * 32) + (nu + 16);
        auto it = memo1.find(key);
        if (it != memo1.end()) return it->second;
        double acc = 0.0;
        for (int K1 = -J1; K1 <= J1; ++K1) {
            const int K2 = K1 + nu;
            if (K2 < -J2 || K2 > J2) continue;
            const double bb = lv[l2].b[K2 + J2] * lv[l1].b[K1 + J1];
            if (bb == 0.0) continue;
            const double *x2 = dref(J2, n1, K2), *xl = dref(lam1, eta, nu), *x1 = dref(J1, m1, K1);
            double sum = 0.0;
            for (int q = 0; q < nq; ++q) sum += wq[q] * x2[q] * xl[q] * x1[q];
            acc += bb * sum;
        }
        const double v = std::sqrt((2.0 * J2 + 1.0) * (2.0 * J1 + 1.0)) / (8.0 * pi * pi) * 4.0 * pi * pi * acc;
        memo1.emplace(key, v);
        return v;
    };
    // molecule 2: I2 = <Y^{a2}_{m2-eta} | Y^{lam2}_{-eta} | Y^{a1}_{m2}>
    auto I2 = [&](int a2, int a1, int m2, int eta, int lam2) {
        const int n2 = m2 - eta;
        if (std::abs(n2) > a2 || std::abs(m2) > a1 || std::abs(eta) > lam2) return 0.0;
        const long long key = ((((long long)a2 * 16 + a1) * 32 + (m2 + 16)) * 32 + (eta + 16)) * 16 + lam2;
        auto it = memo2.find(key);
        if (it != memo2.end()) return it->second;
        const double *x2 = dref(a2, n2, 0), *xl = dref(lam2, -eta, 0), *x1 = dref(a1, m2, 0);
        double sum = 0.0;
        for (int q = 0; q < nq; ++q) sum += wq[q] * x2[q] * xl[q] * x1[q];
        const double v = std::sqrt((2.0 * a2 + 1.0) * (2.0 * lam2 + 1.0) * (2.0 * a1 + 1.0)) / std::pow(4.0 * pi, 1.5) *
                         2.0 * pi * sum;
        memo2.emplace(key, v);
        return v;
    };
    std::vector<int32_t> gt, gr, gc;
    std::vector<double> gv;
    for (int t = 0; t < L; ++t) {
        const int lam1 = p->lam1[t], mu1 = p->mu1[t], lam2 = p->lam2[t], lam = p->lam[t];
        const double sg = ((lam1 + mu1 + lam2 + lam) & 1) ? -1.0 : 1.0;
        const double pre = std::sqrt((2.0 * lam1 + 1.0) / (4.0 * pi));
        const int emax = std::min(lam1, lam2);
        for (int r = 0; r < n; ++r)
            for (int c = 0; c <= r; ++c) {
                if (st[r].m != st[c].m) continue;
                const int m = st[r].m, J2 = lv[st[r].l1].J, J1 = lv[st[c].l1].J;
                double acc = 0.0;
                for (int eta = -emax; eta <= emax; ++eta) {
                    const double ce = cgl[(size_t)lam1 * (lmax + 1) + lam2].get(eta, -eta, lam, 0);
                    if (ce == 0.0) continue;
                    for (int m1 = -J1; m1 <= J1; ++m1) {
                        const int m2 = m - m1;
                        const double cin = CG(J1, m1, st[c].a, m2, st[c].j, m);
                        const double cout = CG(J2, m1 + eta, st[r].a, m2 - eta, st[r].j, m);
                        if (cin == 0.0 || cout == 0.0) continue;
                        const double i1 = I1(st[r].l1, st[c].l1, m1, eta, lam1, mu1) +
                                          (mu1 > 0 ? sg * I1(st[r].l1, st[c].l1, m1, eta, lam1, -mu1)
                                                   : sg * I1(st[r].l1, st[c].l1, m1, eta, lam1, 0));
                        if (i1 == 0.0) continue;
                        acc += ce * cin * cout * i1 * I2(st[r].a, st[c].a, m2, eta, lam2);
                    }
                }
                const double g = pre * acc;
                if (std::fabs(g) < 1e-14) continue;  // selection rules: zero up to rounding
                gt.push_back(t); gr.push_back(r); gc.push_back(c); gv.push_back(g);
                if (r != c) { gt.push_back(t); gr.push_back(c); gc.push_back(r); gv.push_back(g); }
            }
    }
    std::vector<double> A(L), beta(L);
    for (int t = 0; t < L; ++t) { A[t] = p->coef[t]; beta[t] = p->beta[t]; }
    return finish_desc(out, "mqct_build_molmol", energy, level, jq, mq, p->mu, L, gt, gr, gc, gv, A.data(), beta.data(),
                       p->c6, p->rd, ng, p->r_min, p->r_max, false, p->path, p->precision, MQCT_GRID_UNIFORM);
}
