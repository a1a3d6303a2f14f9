/*
 * MQCT oracle -- a plain, slow, FP64 CPU implementation of the mixed
 * quantum/classical (Ehrenfest mean-field) trajectory method of
 * Joy, Mandal, Bostan, Dubernet & Babikov (arXiv 2312.02322).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this file.  It shares no code, header,
 * table or helper with the CUDA library; the two are compared on the same
 * seeded inputs.
 *
 * What it follows (paper sections / equations):
 *   Eq. 4       amplitudes a_n in the interaction picture; c_n = exp(-i E_n t) a_n
 *   Eq. 5       quantum equations of motion: potential coupling summed over the
 *               states of the same m, plus the Coriolis m +- 1 term driven by dPhi/dt
 *   Eq. 6       M(R) = <Psi_n'' m | V | Psi_n' m>: real, symmetric, diagonal in m
 *   Eqs. 7-10   classical R, Phi, P_R, P_Phi in the collision plane (Theta = pi/2)
 *   Eq. 12      V = sum_lambda v_lambda(R) tau_lambda, hence M(R) = sum_lambda v_lambda(R) G^lambda
 *   Eq. 15      integral of three spherical harmonics (G^lambda of a linear rotor)
 *   Eq. 1       asymmetric-top eigenstates as sums of symmetric-top functions (Wang's
 *               symmetrised functions, Jacobi rotations)
 *   Eq. 16      integral of three Wigner D-functions (G^{lambda mu} of an asymmetric top)
 *   Sec. III    cubic-spline interpolation of the coupling along R
 *   Sec. II     final |a|^2 summed over final and averaged over initial degenerate states
 *
 * Readings where the printed text is garbled or silent:
 *   - Eq. 5 Coriolis term: written as the anti-Hermitian generator
 *       (K a)_{j m} = (dPhi/dt / 2) [ A-_{jm} a_{j,m-1} - A+_{jm} a_{j,m+1} ],
 *     A+-_{jm} = sqrt(j(j+1) - m(m+-1)), i.e. H_q = H_rot + V - dPhi/dt J_y.
 *   - Eq. 10 torque: dP_Phi/dt = i <[J_y, V]> = Re( c^dag D M c ),  D = J+ - J-,
 *     the unique form that conserves E_tot and P_Phi + <J_y> with the above.
 *   - Initial conditions: a = e_s0, R = R0, Phi = 0, P_Phi = b sqrt(2 mu E),
 *     P_R = -sqrt(2 mu (E - M_s0s0(R0)) - P_Phi^2 / R0^2).
 *   - Spline: clamped cubic on a uniform grid with given end slopes; outside the
 *     grid the first / last cubic is extrapolated.  Interval k = floor((R-r_min)/h)
 *     clamped to [0, n_grid-2], x = R - (r_min + k h).  On the logarithmic grid of
 *     Sec. III the spline is the clamped cubic in ln R on its uniform grid (end slopes
 *     R dv/dR), R-derivatives by the chain rule.
 *   - Truncation (Sec. III): an element M_rc is dropped for the whole propagation when
 *     |M_rc(R)| <= threshold at both reference distances, M from the splines.
 *   - Time stepping: classical 4-stage RK4 with fixed dt, stage times
 *     n dt, n dt + dt/2, n dt + dt/2, (n+1) dt.  A trajectory stops after the
 *     first step that ends with R >= r_end and P_R > 0, or after max_steps.
 *
 * Everything is FP64, written for clarity: per-state complex exponentials,
 * per-element M_rc = sum_lambda v_lambda G^lambda_rc, sums in state order.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_OK 0
#define ORA_EINVAL 1
#define ORA_ENOMEM 2

/* trajectory status bits */
#define ORA_ST_MAX_STEPS 1
#define ORA_ST_TABLE_RANGE 2
#define ORA_ST_NONFINITE 4

/* propagation flags */
#define ORA_F_NO_STOP 1     /* only max_steps ends a trajectory                   */
#define ORA_F_PRESCRIBED 2  /* classical motion fixed to a straight line (test)   */
#define ORA_F_FLIP_JY 4     /* J_y -> -J_y in the Coriolis term and in the torque */
/* planted mistakes, used only by the tests that show the conservation pins catch them */
#define ORA_F_PLANT_TORQUE 8     /* reverse the sign of the torque alone          */
#define ORA_F_PLANT_CORIOLIS 16  /* drop the factor 1/2 of the Coriolis term      */
/* decoupled classical motion (the AT-MQCT decoupling of Sec. III, read as): R, Phi move in the
 * isotropic potential v_0(R) alone (term 0, whose G must be the identity) with no torque; the
 * amplitudes follow Eq. 5 along that trajectory */
#define ORA_F_DECOUPLED 32

/* ------------------------------------------------------------------ */
/* Clebsch-Gordan coefficients: Racah's closed formula, long double.  */
/* ------------------------------------------------------------------ */
/* ln n! = lgammal(n + 1); the values for n < ORA_LFAC_N are computed once (the same calls, so
   the same numbers) because every coefficient of a large basis needs dozens of them */
#define ORA_LFAC_N 4096
static long double lfac_tab[ORA_LFAC_N];
static pthread_once_t lfac_once = PTHREAD_ONCE_INIT;
static void lfac_fill(void)
{
    for (int n = 0; n < ORA_LFAC_N; ++n) lfac_tab[n] = lgammal((long double)n + 1.0L);
}
static long double lfac(int n)
{
    if (n >= 0 && n < ORA_LFAC_N) {
        pthread_once(&lfac_once, lfac_fill);
        return lfac_tab[n];
    }
    return lgammal((long double)n + 1.0L);
}

double ora_cg(int j1, int m1, int j2, int m2, int J, int M)
{
    if (m1 + m2 != M) return 0.0;
    if (j1 < 0 || j2 < 0 || J < 0) return 0.0;
    if (abs(m1) > j1 || abs(m2) > j2 || abs(M) > J) return 0.0;
    if (J < abs(j1 - j2) || J > j1 + j2) return 0.0;
    if (m1 == 0 && m2 == 0 && ((j1 + j2 + J) & 1)) return 0.0; /* parity: vanishes exactly */
    long double pre = 0.5L * (logl(2.0L * J + 1.0L) + lfac(J + j1 - j2) + lfac(J - j1 + j2) +
                              lfac(j1 + j2 - J) - lfac(j1 + j2 + J + 1) + lfac(J + M) + lfac(J - M) +
                              lfac(j1 - m1) + lfac(j1 + m1) + lfac(j2 - m2) + lfac(j2 + m2));
    int kmin = 0;
    if (j2 - J - m1 > kmin) kmin = j2 - J - m1;
    if (j1 + m2 - J > kmin) kmin = j1 + m2 - J;
    int kmax = j1 + j2 - J;
    if (j1 - m1 < kmax) kmax = j1 - m1;
    if (j2 + m2 < kmax) kmax = j2 + m2;
    long double s = 0.0L;
    for (int k = kmin; k <= kmax; ++k) {
        long double den = lfac(k) + lfac(j1 + j2 - J - k) + lfac(j1 - m1 - k) + lfac(j2 + m2 - k) +
                          lfac(J - j2 + m1 + k) + lfac(J - j1 - m2 + k);
        long double t = expl(pre - den);
        s += (k & 1) ? -t : t;
    }
    return (double)s;
}

/* ------------------------------------------------------------------ */
/* Linear rotor basis and G^lambda (Eq. 2, Eq. 15)                     */
/* ------------------------------------------------------------------ */
/* States in j-major order: s = j*j + (m + j), j = 0..jmax, m = -j..j.  */
int ora_diatom_n(int jmax) { return (jmax + 1) * (jmax + 1); }

void ora_diatom_basis(int jmax, double bconst, double *energy, int *level, int *jq, int *mq)
{
    for (int j = 0; j <= jmax; ++j)
        for (int m = -j; m <= j; ++m) {
            int s = j * j + (m + j);
            energy[s] = bconst * j * (j + 1);
            level[s] = j;
            jq[s] = j;
            mq[s] = m;
        }
}

/* <j'' m | P_lambda(cos theta) | j' m>: Eq. 15 with P_lambda = sqrt(4 pi/(2 lambda+1)) Y_lambda0:
 *   sqrt((2j'+1)/(2j''+1)) C^{j'' 0}_{j' 0 lambda 0} C^{j'' m}_{j' m lambda 0};  zero unless m'' = m'. */
void ora_diatom_G(int jmax, int lam, double *G)
{
    int n = ora_diatom_n(jmax);
    memset(G, 0, sizeof(double) * (size_t)n * n);
    for (int j2 = 0; j2 <= jmax; ++j2)        /* j''  (row)    */
        for (int j1 = 0; j1 <= jmax; ++j1) {  /* j'   (column) */
            double c0 = ora_cg(j1, 0, lam, 0, j2, 0);
            if (c0 == 0.0) continue;
            double f = sqrt((2.0 * j1 + 1.0) / (2.0 * j2 + 1.0)) * c0;
            int mm = j1 < j2 ? j1 : j2;
            for (int m = -mm; m <= mm; ++m) {
                int r = j2 * j2 + (m + j2), c = j1 * j1 + (m + j1);
                G[(size_t)r * n + c] = f * ora_cg(j1, m, lam, 0, j2, m);
            }
        }
}

/* Synthetic atom + diatom PES of the form
 *   V(R, theta) = sum_{lambda=0}^{4} A_l exp(-beta_l R) P_l(cos theta)
 *                 - C6 R^-6 (1 - exp(-(R/Rd)^6))          (isotropic, lambda = 0)
 * evaluated on a uniform grid; all quantities in atomic units.
 * Outputs v[L][n_grid], dv_ends[L][2] (analytic dv/dR at both ends) and, if
 * dvp != NULL, the derivatives with respect to theta = (A_0..A_{L-1}, beta_0..beta_{L-1}):
 * dvp[2L][L][n_grid], dvp_ends[2L][L][2]. */
/* grid point k: uniform in R, or (grid_log) uniform in ln R (Sec. III: logarithmic spacing) */
static double grid_r(int grid_log, int n_grid, double r_min, double r_max, int k)
{
    if (grid_log) {
        double hl = (log(r_max) - log(r_min)) / (n_grid - 1);
        return r_min * exp(k * hl);
    }
    double h = (r_max - r_min) / (n_grid - 1);
    return r_min + k * h;
}

void ora_diatom_pes_grid(int L, const double *A, const double *beta, double c6, double rd, int n_grid,
                         double r_min, double r_max, int grid_log, double *v, double *dv_ends, double *dvp,
                         double *dvp_ends)
{
    for (int l = 0; l < L; ++l) {
        for (int k = 0; k < n_grid; ++k) {
            double R = grid_r(grid_log, n_grid, r_min, r_max, k);
            double val = A[l] * exp(-beta[l] * R);
            if (l == 0) val -= c6 * pow(R, -6.0) * (1.0 - exp(-pow(R / rd, 6.0)));
            v[l * n_grid + k] = val;
        }
        for (int e = 0; e < 2; ++e) {
            double R = e ? r_max : r_min;
            double d = -beta[l] * A[l] * exp(-beta[l] * R);
            if (l == 0) {
                double u = pow(R / rd, 6.0);
                d += 6.0 * c6 * pow(R, -7.0) * (1.0 - exp(-u)) - c6 * pow(R, -6.0) * exp(-u) * 6.0 * u / R;
            }
            dv_ends[l * 2 + e] = d;
        }
    }
    if (!dvp) return;
    memset(dvp, 0, sizeof(double) * (size_t)2 * L * L * n_grid);
    memset(dvp_ends, 0, sizeof(double) * (size_t)2 * L * L * 2);
    for (int l = 0; l < L; ++l) {
        double *pa = dvp + ((size_t)l * L + l) * n_grid;        /* d v_l / d A_l    */
        double *pb = dvp + ((size_t)(L + l) * L + l) * n_grid;  /* d v_l / d beta_l */
        for (int k = 0; k < n_grid; ++k) {
            double R = grid_r(grid_log, n_grid, r_min, r_max, k);
            pa[k] = exp(-beta[l] * R);
            pb[k] = -R * A[l] * exp(-beta[l] * R);
        }
        for (int e = 0; e < 2; ++e) {
            double R = e ? r_max : r_min;
            double ex = exp(-beta[l] * R);
            dvp_ends[((size_t)l * L + l) * 2 + e] = -beta[l] * ex;
            dvp_ends[((size_t)(L + l) * L + l) * 2 + e] = -A[l] * ex + beta[l] * R * A[l] * ex;
        }
    }
}

void ora_diatom_pes(int L, const double *A, const double *beta, double c6, double rd, int n_grid,
                    double r_min, double r_max, double *v, double *dv_ends, double *dvp, double *dvp_ends)
{
    ora_diatom_pes_grid(L, A, beta, c6, rd, n_grid, r_min, r_max, 0, v, dv_ends, dvp, dvp_ends);
}

/* G^lambda of the linear rotor (Eq. 15) as triplets (row, col, value) of the non-zero
 * entries, for bases too large for a dense N x N array; returns the count written (at most
 * cap) or -1 if cap is too small. */
long long ora_diatom_G_triplets(int jmax, int lam, long long cap, int *row, int *col, double *val)
{
    long long k = 0;
    for (int j2 = 0; j2 <= jmax; ++j2)
        for (int j1 = 0; j1 <= jmax; ++j1) {
            double c0 = ora_cg(j1, 0, lam, 0, j2, 0);
            if (c0 == 0.0) continue;
            double f = sqrt((2.0 * j1 + 1.0) / (2.0 * j2 + 1.0)) * c0;
            int mm = j1 < j2 ? j1 : j2;
            for (int m = -mm; m <= mm; ++m) {
                double g = f * ora_cg(j1, m, lam, 0, j2, m);
                if (g == 0.0) continue;
                if (k >= cap) return -1;
                row[k] = j2 * j2 + (m + j2);
                col[k] = j1 * j1 + (m + j1);
                val[k] = g;
                ++k;
            }
        }
    return k;
}

/* ------------------------------------------------------------------ */
/* Clamped cubic spline on a uniform grid (second-derivative form).   */
/* ------------------------------------------------------------------ */
/* coef[i][0..3]: y(R) = c0 + c1 x + c2 x^2 + c3 x^3 on [R_i, R_{i+1}], x = R - R_i. */
int ora_spline(int n, double h, const double *y, double d0, double dn, double *coef)
{
    if (n < 2 || !(h > 0)) return ORA_EINVAL;
    double *a = malloc(sizeof(double) * n), *b = malloc(sizeof(double) * n), *c = malloc(sizeof(double) * n),
           *r = malloc(sizeof(double) * n), *s = malloc(sizeof(double) * n);
    if (!a || !b || !c || !r || !s) {
        free(a); free(b); free(c); free(r); free(s);
        return ORA_ENOMEM;
    }
    /* tridiagonal system for the second derivatives s_i */
    a[0] = 0.0; b[0] = 2.0; c[0] = 1.0;
    r[0] = 6.0 / h * ((y[1] - y[0]) / h - d0);
    for (int i = 1; i < n - 1; ++i) {
        a[i] = 1.0; b[i] = 4.0; c[i] = 1.0;
        r[i] = 6.0 / (h * h) * (y[i + 1] - 2.0 * y[i] + y[i - 1]);
    }
    a[n - 1] = 1.0; b[n - 1] = 2.0; c[n - 1] = 0.0;
    r[n - 1] = 6.0 / h * (dn - (y[n - 1] - y[n - 2]) / h);
    /* Thomas algorithm */
    for (int i = 1; i < n; ++i) {
        double w = a[i] / b[i - 1];
        b[i] -= w * c[i - 1];
        r[i] -= w * r[i - 1];
    }
    s[n - 1] = r[n - 1] / b[n - 1];
    for (int i = n - 2; i >= 0; --i) s[i] = (r[i] - c[i] * s[i + 1]) / b[i];
    for (int i = 0; i < n - 1; ++i) {
        double *q = coef + 4 * (size_t)i;
        q[0] = y[i];
        q[1] = (y[i + 1] - y[i]) / h - h * (2.0 * s[i] + s[i + 1]) / 6.0;
        q[2] = 0.5 * s[i];
        q[3] = (s[i + 1] - s[i]) / (6.0 * h);
    }
    free(a); free(b); free(c); free(r); free(s);
    return ORA_OK;
}

/* value, first and second derivative of a spline built by ora_spline */
static void spline_at(const double *coef, int n_int, double r_min, double h, double R, double *f, double *df,
                      double *d2f)
{
    int k = (int)floor((R - r_min) / h);
    if (k < 0) k = 0;
    if (k > n_int - 1) k = n_int - 1;
    double x = R - (r_min + k * h);
    const double *q = coef + 4 * (size_t)k;
    *f = q[0] + x * (q[1] + x * (q[2] + x * q[3]));
    *df = q[1] + x * (2.0 * q[2] + 3.0 * x * q[3]);
    *d2f = 2.0 * q[2] + 6.0 * x * q[3];
}

void ora_spline_eval(const double *coef, int n_grid, double r_min, double r_max, int npts, const double *R,
                     double *f, double *df, double *d2f)
{
    double h = (r_max - r_min) / (n_grid - 1);
    for (int i = 0; i < npts; ++i) spline_at(coef, n_grid - 1, r_min, h, R[i], f + i, df + i, d2f + i);
}

/* ------------------------------------------------------------------ */
/* System: states, coupling terms, spline of v_lambda.                */
/* ------------------------------------------------------------------ */
typedef struct {
    int n, n_terms, n_grid;
    double mu, r_min, r_max;
    const double *energy;  /* [n]            */
    const int *level;      /* [n]            */
    const int *jq, *mq;    /* [n]; jq < 0 switches the Coriolis term off for the state */
    const double *G;       /* [L][n][n]      */
    const double *v;       /* [L][n_grid]    */
    const double *dv_ends; /* [L][2]         */
    int n_params;          /* derivative tables for ora_tangent (0 if unused) */
    const double *dvp;     /* [P][L][n_grid] */
    const double *dvp_ends;/* [P][L][2]      */
    /* grid_log: grid uniform in ln R (R_k = r_min (r_max/r_min)^(k/(n_grid-1))), spline in ln R */
    int grid_log;
    /* truncation (Sec. III): M_rc is dropped when |M_rc(R)| <= trunc_thr at both trunc_r;
       trunc_thr <= 0 keeps every element */
    double trunc_thr;
    double trunc_r[2];
    /* G in triplet form when G == NULL: g_nnz entries (term, row, col, value), summed */
    long long g_nnz;
    const int *g_term, *g_row, *g_col;
    const double *g_val;
    /* adaptive step control: adapt_tol > 0 switches it on; the largest step is adapt_hmax_factor x
       the trajectory's dt (16 when 0) and the smallest is dt */
    double adapt_tol;
    int adapt_hmax_factor;
} ora_system_desc;

typedef struct {
    double e_coll, b, r0, r_end, dt;
    int init_state, max_steps;
} ora_traj;

typedef struct {
    int steps, status;
    double norm_dev, energy_dev, angmom_dev, t_final;
    double R, PR, Phi, PPhi;
} ora_result;

typedef struct {
    int n, L, n_int, P;
    double mu, r_min, h;
    int grid_log;      /* spline variable x = ln R instead of R          */
    double x0;         /* first knot in the spline variable             */
    const double *E;
    int n_blk;
    int *blk_start, *blk_size, *members; /* members grouped by block (same m) */
    double *Gb;                          /* per block: [L][nb][nb]            */
    size_t *blk_goff;
    int *up, *dn;                        /* Coriolis partners (-1: none)      */
    double *aup, *adn;                   /* A+ and A- ladder factors          */
    unsigned char *keep;                 /* per block: [nb][nb] truncation mask (NULL: keep all) */
    double *coef;                        /* [L][n_int][4]                     */
    double *dcoef;                       /* [P][L][n_int][4]                  */
} ora_sys;

static void sys_free(ora_sys *S)
{
    free(S->blk_start); free(S->blk_size); free(S->members); free(S->Gb); free(S->blk_goff);
    free(S->up); free(S->dn); free(S->aup); free(S->adn); free(S->coef); free(S->dcoef); free(S->keep);
    memset(S, 0, sizeof(*S));
}

/* sort key of the Coriolis partner search: states of one level and one j, ordered by m */
typedef struct { int level, j, m, s; } ora_key;

static int key_cmp(const void *pa, const void *pb)
{
    const ora_key *a = pa, *b = pb;
    if (a->level != b->level) return a->level < b->level ? -1 : 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    if (a->m != b->m) return a->m < b->m ? -1 : 1;
    return 0;
}

static void eval_terms(const ora_sys *S, const double *coef, double R, double *v, double *dv, double *d2v);

static int sys_build(const ora_system_desc *d, ora_sys *S)
{
    memset(S, 0, sizeof(*S));
    int n = d->n, L = d->n_terms;
    if (n < 1 || L < 1 || d->n_grid < 2 || !(d->mu > 0) || !(d->r_max > d->r_min)) return ORA_EINVAL;
    if (d->grid_log && !(d->r_min > 0)) return ORA_EINVAL;
    if (!d->G && d->g_nnz > 0 && (!d->g_term || !d->g_row || !d->g_col || !d->g_val)) return ORA_EINVAL;
    S->n = n; S->L = L; S->n_int = d->n_grid - 1; S->P = d->n_params;
    S->mu = d->mu; S->r_min = d->r_min;
    S->grid_log = d->grid_log != 0;
    S->x0 = S->grid_log ? log(d->r_min) : d->r_min;
    S->h = ((S->grid_log ? log(d->r_max) : d->r_max) - S->x0) / (d->n_grid - 1);
    S->E = d->energy;
    /* blocks of equal m (Eq. 5 couples states only within each m) */
    int *blk_of = malloc(sizeof(int) * n), *pos_of = malloc(sizeof(int) * n);
    S->blk_start = malloc(sizeof(int) * (n + 1));
    S->blk_size = malloc(sizeof(int) * n);
    S->members = malloc(sizeof(int) * n);
    S->up = malloc(sizeof(int) * n); S->dn = malloc(sizeof(int) * n);
    S->aup = malloc(sizeof(double) * n); S->adn = malloc(sizeof(double) * n);
    int *mvals = malloc(sizeof(int) * n);
    ora_key *keys = malloc(sizeof(ora_key) * n);
    if (!blk_of || !pos_of || !S->blk_start || !S->blk_size || !S->members || !S->up || !S->dn || !S->aup ||
        !S->adn || !mvals || !keys) {
        free(blk_of); free(pos_of); free(mvals); free(keys); sys_free(S);
        return ORA_ENOMEM;
    }
    int nb = 0;
    for (int s = 0; s < n; ++s) {
        int b = -1;
        for (int q = 0; q < nb; ++q)
            if (mvals[q] == d->mq[s]) b = q;
        if (b < 0) { b = nb; mvals[nb++] = d->mq[s]; }
        blk_of[s] = b;
    }
    S->n_blk = nb;
    for (int b = 0; b < nb; ++b) S->blk_size[b] = 0;
    for (int s = 0; s < n; ++s) S->blk_size[blk_of[s]]++;
    int pos = 0;
    for (int b = 0; b < nb; ++b) { S->blk_start[b] = pos; pos += S->blk_size[b]; S->blk_size[b] = 0; }
    S->blk_start[nb] = pos;
    for (int s = 0; s < n; ++s) {   /* members in state order within each block */
        int b = blk_of[s];
        pos_of[s] = S->blk_size[b]++;
        S->members[S->blk_start[b] + pos_of[s]] = s;
    }
    /* coupling must vanish between different m (Eq. 6) */
    int bad = 0;
    if (d->G) {
        for (int l = 0; l < L && !bad; ++l)
            for (int r = 0; r < n && !bad; ++r)
                for (int c = 0; c < n; ++c)
                    if (blk_of[r] != blk_of[c] && d->G[((size_t)l * n + r) * n + c] != 0.0) { bad = 1; break; }
    } else {
        for (long long e = 0; e < d->g_nnz && !bad; ++e) {
            int l = d->g_term[e], r = d->g_row[e], c = d->g_col[e];
            if (l < 0 || l >= L || r < 0 || r >= n || c < 0 || c >= n) bad = 1;
            else if (blk_of[r] != blk_of[c] && d->g_val[e] != 0.0) bad = 1;
        }
    }
    if (bad) { free(blk_of); free(pos_of); free(mvals); free(keys); sys_free(S); return ORA_EINVAL; }
    S->blk_goff = malloc(sizeof(size_t) * (nb + 1));
    size_t tot = 0;
    for (int b = 0; b < nb; ++b) { S->blk_goff[b] = tot; tot += (size_t)L * S->blk_size[b] * S->blk_size[b]; }
    S->blk_goff[nb] = tot;
    S->Gb = calloc(tot ? tot : 1, sizeof(double));
    if (!S->Gb) { free(blk_of); free(pos_of); free(mvals); free(keys); sys_free(S); return ORA_ENOMEM; }
    if (d->G) {
        for (int b = 0; b < nb; ++b) {
            int sz = S->blk_size[b];
            const int *mem = S->members + S->blk_start[b];
            for (int l = 0; l < L; ++l)
                for (int r = 0; r < sz; ++r)
                    for (int c = 0; c < sz; ++c)
                        S->Gb[S->blk_goff[b] + ((size_t)l * sz + r) * sz + c] = d->G[((size_t)l * n + mem[r]) * n + mem[c]];
        }
    } else {
        for (long long e = 0; e < d->g_nnz; ++e) {
            int l = d->g_term[e], r = d->g_row[e], c = d->g_col[e], b = blk_of[r], sz = S->blk_size[b];
            S->Gb[S->blk_goff[b] + ((size_t)l * sz + pos_of[r]) * sz + pos_of[c]] += d->g_val[e];
        }
    }
    /* Coriolis partners: same level and j, m +- 1 (neighbours after sorting by level, j, m) */
    for (int s = 0; s < n; ++s) {
        S->up[s] = S->dn[s] = -1;
        S->aup[s] = S->adn[s] = 0.0;
        keys[s].level = d->level[s]; keys[s].j = d->jq[s]; keys[s].m = d->mq[s]; keys[s].s = s;
    }
    qsort(keys, n, sizeof(ora_key), key_cmp);
    for (int i = 0; i + 1 < n; ++i) {
        const ora_key *a = keys + i, *b = keys + i + 1;
        if (a->j < 0 || a->level != b->level || a->j != b->j || b->m != a->m + 1) continue;
        S->up[a->s] = b->s;
        S->dn[b->s] = a->s;
    }
    for (int s = 0; s < n; ++s) {
        int j = d->jq[s], m = d->mq[s];
        if (j < 0) { S->up[s] = S->dn[s] = -1; continue; }
        double jj = (double)j * (j + 1);
        if (S->up[s] >= 0) S->aup[s] = sqrt(jj - (double)m * (m + 1));
        if (S->dn[s] >= 0) S->adn[s] = sqrt(jj - (double)m * (m - 1));
    }
    free(blk_of); free(pos_of); free(mvals); free(keys);
    /* splines of the expansion coefficients (and of their parameter derivatives); on the log
       grid the spline variable is x = ln R and the end slopes are dv/dx = R dv/dR */
    double e0 = S->grid_log ? d->r_min : 1.0, e1 = S->grid_log ? d->r_max : 1.0;
    S->coef = malloc(sizeof(double) * (size_t)L * S->n_int * 4);
    for (int l = 0; l < L; ++l) {
        int e = ora_spline(d->n_grid, S->h, d->v + (size_t)l * d->n_grid, e0 * d->dv_ends[2 * l],
                           e1 * d->dv_ends[2 * l + 1], S->coef + (size_t)l * S->n_int * 4);
        if (e) { sys_free(S); return e; }
    }
    if (S->P > 0) {
        S->dcoef = malloc(sizeof(double) * (size_t)S->P * L * S->n_int * 4);
        for (int p = 0; p < S->P; ++p)
            for (int l = 0; l < L; ++l) {
                size_t o = (size_t)p * L + l;
                int e = ora_spline(d->n_grid, S->h, d->dvp + o * d->n_grid, e0 * d->dvp_ends[2 * o],
                                   e1 * d->dvp_ends[2 * o + 1], S->dcoef + o * S->n_int * 4);
                if (e) { sys_free(S); return e; }
            }
    }
    /* truncation (Sec. III): keep M_rc where |M_rc| exceeds the threshold at either reference
       distance, M evaluated from the splines above */
    if (d->trunc_thr > 0.0) {
        size_t ktot = tot / (size_t)L;
        S->keep = malloc(ktot ? ktot : 1);
        double *va = malloc(sizeof(double) * 6 * L);
        if (!S->keep || !va) { free(va); sys_free(S); return ORA_ENOMEM; }
        eval_terms(S, S->coef, d->trunc_r[0], va, va + L, va + 2 * L);
        eval_terms(S, S->coef, d->trunc_r[1], va + 3 * L, va + 4 * L, va + 5 * L);
        for (int b = 0; b < nb; ++b) {
            int sz = S->blk_size[b];
            const double *Gb = S->Gb + S->blk_goff[b];
            unsigned char *kp = S->keep + S->blk_goff[b] / L;
            for (int r = 0; r < sz; ++r)
                for (int c = 0; c < sz; ++c) {
                    double ma = 0.0, mb = 0.0;
                    for (int l = 0; l < L; ++l) {
                        double g = Gb[((size_t)l * sz + r) * sz + c];
                        ma += va[l] * g;
                        mb += va[3 * L + l] * g;
                    }
                    kp[(size_t)r * sz + c] = (fabs(ma) > d->trunc_thr || fabs(mb) > d->trunc_thr) ? 1 : 0;
                }
        }
        free(va);
    }
    return ORA_OK;
}

/* whether M_rc of block b is kept by the truncation */
static int kept(const ora_sys *S, int b, int r, int c)
{
    if (!S->keep) return 1;
    int sz = S->blk_size[b];
    return S->keep[S->blk_goff[b] / S->L + (size_t)r * sz + c];
}

/* v_lambda and its first two R-derivatives; table_range set if R < r_min */
static void eval_terms(const ora_sys *S, const double *coef, double R, double *v, double *dv, double *d2v)
{
    double x = S->grid_log ? log(R) : R;
    for (int l = 0; l < S->L; ++l)
        spline_at(coef + (size_t)l * S->n_int * 4, S->n_int, S->x0, S->h, x, v + l, dv + l, d2v + l);
    if (S->grid_log)  /* chain rule from x = ln R: f' = f_x / R, f'' = (f_xx - f_x) / R^2 */
        for (int l = 0; l < S->L; ++l) {
            double d1 = dv[l] / R;
            d2v[l] = (d2v[l] - dv[l]) / (R * R);
            dv[l] = d1;
        }
}

/* y = sum over the m-blocks of (sum_lambda f_lambda G^lambda) x   (Eq. 5 / Eq. 12) */
static void couple(const ora_sys *S, const double *f, const double complex *x, double complex *y)
{
    for (int b = 0; b < S->n_blk; ++b) {
        int sz = S->blk_size[b];
        const int *mem = S->members + S->blk_start[b];
        const double *Gb = S->Gb + S->blk_goff[b];
        for (int r = 0; r < sz; ++r) {
            double complex acc = 0.0;
            for (int c = 0; c < sz; ++c) {
                if (!kept(S, b, r, c)) continue;
                double mrc = 0.0;
                for (int l = 0; l < S->L; ++l) mrc += f[l] * Gb[((size_t)l * sz + r) * sz + c];
                acc += mrc * x[mem[c]];
            }
            y[mem[r]] = acc;
        }
    }
}

/* (D x)_s = A-_s x_{m-1} - A+_s x_{m+1},  D = J+ - J- */
static double complex ladder(const ora_sys *S, const double complex *x, int s)
{
    double complex r = 0.0;
    if (S->dn[s] >= 0) r += S->adn[s] * x[S->dn[s]];
    if (S->up[s] >= 0) r -= S->aup[s] * x[S->up[s]];
    return r;
}

typedef struct {
    double complex *c, *w, *u, *u2, *tmp, *tmp2;
    double *v, *dv, *d2v, *pv, *pdv, *pd2v;
} ora_work;

static int work_alloc(ora_work *W, int n, int L)
{
    W->c = malloc(sizeof(double complex) * n);
    W->w = malloc(sizeof(double complex) * n);
    W->u = malloc(sizeof(double complex) * n);
    W->u2 = malloc(sizeof(double complex) * n);
    W->tmp = malloc(sizeof(double complex) * n);
    W->tmp2 = malloc(sizeof(double complex) * n);
    W->v = malloc(sizeof(double) * L * 6);
    if (!W->c || !W->w || !W->u || !W->u2 || !W->tmp || !W->tmp2 || !W->v) return ORA_ENOMEM;
    W->dv = W->v + L; W->d2v = W->v + 2 * L; W->pv = W->v + 3 * L; W->pdv = W->v + 4 * L; W->pd2v = W->v + 5 * L;
    return ORA_OK;
}

static void work_free(ora_work *W)
{
    free(W->c); free(W->w); free(W->u); free(W->u2); free(W->tmp); free(W->tmp2); free(W->v);
}

/* classical state q = (R, P_R, Phi, P_Phi) */
typedef struct {
    int flags;
    double jy_sign; /* +1, or -1 with ORA_F_FLIP_JY */
    double line_b, line_v, line_t0; /* prescribed straight line (ORA_F_PRESCRIBED) */
    double tol;                     /* > 0: adaptive step control (step doubling), else fixed dt */
    double hmax_factor;             /* largest adaptive step / dt                                */
} ora_opts;

/* quantities of a right-hand-side evaluation, for the diagnostics */
typedef struct {
    double vc;   /* Re(c^dag M c) */
    double jy;   /* <J_y> = Im(a^dag D a)/2 */
    double norm; /* sum |a|^2 */
    double erot; /* sum E |a|^2 */
    double viso; /* v_0(R) (decoupled mode) */
    int below;   /* R < r_min */
} ora_eval;

/* f(t, y): Eqs. 5 and 7-10 in the reading stated in the header */
static void rhs(const ora_sys *S, const ora_opts *o, double t, const double complex *a, const double *q,
                double complex *da, double *dq, ora_work *W, ora_eval *ev)
{
    int n = S->n;
    double R = q[0], PR = q[1], PPhi = q[3], phidot;
    if (o->flags & ORA_F_PRESCRIBED) {
        double s = o->line_v * (t - o->line_t0);
        R = sqrt(o->line_b * o->line_b + s * s);
        phidot = o->line_b * o->line_v / (R * R);
    } else {
        phidot = PPhi / (S->mu * R * R);
    }
    eval_terms(S, S->coef, R, W->v, W->dv, W->d2v);
    for (int s = 0; s < n; ++s) W->c[s] = cexp(-I * S->E[s] * t) * a[s];
    couple(S, W->v, W->c, W->w);  /* w = M c   */
    couple(S, W->dv, W->c, W->u); /* u = M' c  */
    double force = 0.0, torque = 0.0;
    for (int s = 0; s < n; ++s) {
        force -= creal(conj(W->c[s]) * W->u[s]);
        torque += creal(conj(W->c[s]) * ladder(S, W->w, s));
    }
    if (o->flags & ORA_F_DECOUPLED) {
        /* no back-reaction of the amplitudes: the isotropic potential alone, no torque */
        force = -W->dv[0];
        torque = 0.0;
    }
    force += PPhi * PPhi / (S->mu * R * R * R);
    torque *= o->jy_sign;
    if (o->flags & ORA_F_PLANT_TORQUE) torque = -torque;
    double kc = (o->flags & ORA_F_PLANT_CORIOLIS) ? 1.0 : 0.5;
    for (int s = 0; s < n; ++s)
        da[s] = -I * cexp(I * S->E[s] * t) * W->w[s] + o->jy_sign * kc * phidot * ladder(S, a, s);
    if (o->flags & ORA_F_PRESCRIBED) {
        dq[0] = dq[1] = dq[2] = dq[3] = 0.0;
    } else {
        dq[0] = PR / S->mu;
        dq[1] = force;
        dq[2] = phidot;
        dq[3] = torque;
    }
    if (ev) {
        double vc = 0.0, jy = 0.0, nrm = 0.0, er = 0.0;
        for (int s = 0; s < n; ++s) {
            vc += creal(conj(W->c[s]) * W->w[s]);
            jy += cimag(conj(a[s]) * ladder(S, a, s));
            double p = creal(a[s]) * creal(a[s]) + cimag(a[s]) * cimag(a[s]);
            nrm += p;
            er += S->E[s] * p;
        }
        ev->vc = vc;
        ev->jy = 0.5 * o->jy_sign * jy;
        ev->norm = nrm;
        ev->erot = er;
        ev->viso = W->v[0];
        ev->below = R < S->r_min;
    }
}

static double total_energy(const ora_sys *S, const ora_opts *o, const double *q, const ora_eval *ev)
{
    double R = q[0];
    if (o->flags & ORA_F_DECOUPLED)  /* the classical energy, conserved on its own */
        return q[1] * q[1] / (2.0 * S->mu) + q[3] * q[3] / (2.0 * S->mu * R * R) + ev->viso;
    return q[1] * q[1] / (2.0 * S->mu) + q[3] * q[3] / (2.0 * S->mu * R * R) + ev->erot + ev->vc;
}

/* the conserved angular momentum: P_Phi + <J_y>, or P_Phi alone with decoupled motion */
static double total_angmom(const ora_opts *o, const double *q, const ora_eval *ev)
{
    return (o->flags & ORA_F_DECOUPLED) ? q[3] : q[3] + ev->jy;
}

static int finite_state(int n, const double complex *a, const double *q)
{
    for (int i = 0; i < 4; ++i)
        if (!isfinite(q[i])) return 0;
    for (int s = 0; s < n; ++s)
        if (!isfinite(creal(a[s])) || !isfinite(cimag(a[s]))) return 0;
    return 1;
}

static void initial_state(const ora_sys *S, const ora_traj *tr, int decoupled, double complex *a, double *q,
                          double *m00_out)
{
    for (int s = 0; s < S->n; ++s) a[s] = 0.0;
    a[tr->init_state] = 1.0;
    /* diagonal coupling of the initial state at R0 */
    double *pv = malloc(sizeof(double) * 3 * S->L);
    eval_terms(S, S->coef, tr->r0, pv, pv + S->L, pv + 2 * S->L);
    int s0 = tr->init_state, b = -1, r = -1;
    for (int q2 = 0; q2 < S->n_blk && b < 0; ++q2)
        for (int i = 0; i < S->blk_size[q2]; ++i)
            if (S->members[S->blk_start[q2] + i] == s0) { b = q2; r = i; }
    int sz = S->blk_size[b];
    double m00 = 0.0;
    if (decoupled)
        m00 = pv[0];  /* the isotropic potential: the classical motion does not see the state */
    else if (kept(S, b, r, r))
        for (int l = 0; l < S->L; ++l) m00 += pv[l] * S->Gb[S->blk_goff[b] + ((size_t)l * sz + r) * sz + r];
    free(pv);
    double lz = tr->b * sqrt(2.0 * S->mu * tr->e_coll);
    q[0] = tr->r0;
    q[2] = 0.0;
    q[3] = lz;
    q[1] = -sqrt(2.0 * S->mu * (tr->e_coll - m00) - lz * lz / (tr->r0 * tr->r0));
    if (m00_out) *m00_out = m00;
}

/* one RK4 step of length h from (t, a, q); ev receives the evaluation at the start of the step;
 * returns the TABLE_RANGE bit of its four evaluations */
static int rk4_step(const ora_sys *S, const ora_opts *o, double t, double h, double complex *a, double *q,
                    ora_work *W, double complex *k1, double complex *k2, double complex *k3, double complex *k4,
                    double complex *ys, ora_eval *ev)
{
    int n = S->n, status = 0;
    double qs[4], l1[4], l2[4], l3[4], l4[4];
    ora_eval e2;
    rhs(S, o, t, a, q, k1, l1, W, ev);
    if (ev->below) status |= ORA_ST_TABLE_RANGE;
    for (int s = 0; s < n; ++s) ys[s] = a[s] + 0.5 * h * k1[s];
    for (int i = 0; i < 4; ++i) qs[i] = q[i] + 0.5 * h * l1[i];
    rhs(S, o, t + 0.5 * h, ys, qs, k2, l2, W, &e2);
    if (e2.below) status |= ORA_ST_TABLE_RANGE;
    for (int s = 0; s < n; ++s) ys[s] = a[s] + 0.5 * h * k2[s];
    for (int i = 0; i < 4; ++i) qs[i] = q[i] + 0.5 * h * l2[i];
    rhs(S, o, t + 0.5 * h, ys, qs, k3, l3, W, &e2);
    if (e2.below) status |= ORA_ST_TABLE_RANGE;
    for (int s = 0; s < n; ++s) ys[s] = a[s] + h * k3[s];
    for (int i = 0; i < 4; ++i) qs[i] = q[i] + h * l3[i];
    rhs(S, o, t + h, ys, qs, k4, l4, W, &e2);
    if (e2.below) status |= ORA_ST_TABLE_RANGE;
    for (int s = 0; s < n; ++s) a[s] += h / 6.0 * (k1[s] + 2.0 * k2[s] + 2.0 * k3[s] + k4[s]);
    for (int i = 0; i < 4; ++i) q[i] += h / 6.0 * (l1[i] + 2.0 * l2[i] + 2.0 * l3[i] + l4[i]);
    return status;
}

static int propagate_one(const ora_sys *S, const ora_traj *tr, const ora_opts *o, double complex *a_out, ora_result *res)
{
    int n = S->n, status = 0;
    ora_work W;
    double complex *a = malloc(sizeof(double complex) * n * 8);
    if (!a || work_alloc(&W, n, S->L)) { free(a); work_free(&W); return ORA_ENOMEM; }
    double complex *k1 = a + n, *k2 = a + 2 * n, *k3 = a + 3 * n, *k4 = a + 4 * n, *ys = a + 5 * n;
    double complex *a0 = a + 6 * n, *a1 = a + 7 * n;
    double q[4];
    initial_state(S, tr, (o->flags & ORA_F_DECOUPLED) != 0, a, q, NULL);
    if (o->flags & ORA_F_PRESCRIBED) {
        double s = o->line_v * (0.0 - o->line_t0);
        q[0] = sqrt(o->line_b * o->line_b + s * s);
        q[1] = q[2] = q[3] = 0.0;
    }
    double dt = tr->dt, t = 0.0, e0 = 0.0, j0 = 0.0, ndev = 0.0, edev = 0.0, jdev = 0.0;
    ora_eval ev;
    int steps = 0, stopped = 0;
    /* Step control.  Fixed: every step dt.  Adaptive (o->tol > 0; the algorithm of ADAPTOL in
       Sec. III is not given, so this is a reading of it): step doubling -- one RK4 step of h against two of
       h/2 from the same state, error = max_n |a_n(two halves) - a_n(one step)|.  The two-half result
       is kept when the error is at most tol or h is already dt (the smallest step); otherwise h is
       halved and the step retried from the same state.  After an accepted step h doubles, up to
       hmax_factor dt, when the error was at most tol / 64.  h starts at hmax_factor dt. */
    const int adaptive = o->tol > 0.0;
    const double hmax = dt * o->hmax_factor;
    double h = adaptive ? hmax : dt;
    while (steps < tr->max_steps) {
        double qstart[4], q1[4], err = 0.0, tn;
        for (int i = 0; i < 4; ++i) qstart[i] = q[i];
        if (!adaptive) {
            status |= rk4_step(S, o, steps * dt, dt, a, q, &W, k1, k2, k3, k4, ys, &ev);
            tn = (steps + 1) * dt;
        } else {
            ora_eval eh;
            for (int s = 0; s < n; ++s) { a0[s] = a[s]; a1[s] = a[s]; }
            for (int i = 0; i < 4; ++i) q1[i] = q[i];
            status |= rk4_step(S, o, t, h, a1, q1, &W, k1, k2, k3, k4, ys, &ev);
            status |= rk4_step(S, o, t, 0.5 * h, a, q, &W, k1, k2, k3, k4, ys, &eh);
            status |= rk4_step(S, o, t + 0.5 * h, 0.5 * h, a, q, &W, k1, k2, k3, k4, ys, &eh);
            for (int s = 0; s < n; ++s) err = fmax(err, cabs(a[s] - a1[s]));
            if (!(err <= o->tol) && h > dt) {
                for (int s = 0; s < n; ++s) a[s] = a0[s];
                for (int i = 0; i < 4; ++i) q[i] = qstart[i];
                h *= 0.5;
                continue;
            }
            tn = t + h;
        }
        /* diagnostics of the state the step started from */
        {
            double et = total_energy(S, o, qstart, &ev), jt = total_angmom(o, qstart, &ev);
            if (steps == 0) { e0 = et; j0 = jt; }
            if (fabs(ev.norm - 1.0) > ndev) ndev = fabs(ev.norm - 1.0);
            if (fabs(et - e0) > edev) edev = fabs(et - e0);
            if (fabs(jt - j0) > jdev) jdev = fabs(jt - j0);
        }
        if (o->flags & ORA_F_PRESCRIBED) {
            double s = o->line_v * (tn - o->line_t0);
            q[0] = sqrt(o->line_b * o->line_b + s * s);
        }
        steps += 1;
        t = tn;
        if (adaptive && 64.0 * err <= o->tol && h < hmax) h *= 2.0;
        if (!finite_state(n, a, q)) { status |= ORA_ST_NONFINITE; stopped = 1; break; }
        if (!(o->flags & (ORA_F_NO_STOP | ORA_F_PRESCRIBED)) && q[0] >= tr->r_end && q[1] > 0.0) { stopped = 1; break; }
    }
    if (!stopped) status |= ORA_ST_MAX_STEPS;
    if (!(status & ORA_ST_NONFINITE)) {
        /* diagnostics of the final state */
        double lf[4];
        rhs(S, o, t, a, q, k1, lf, &W, &ev);
        double et = total_energy(S, o, q, &ev), jt = total_angmom(o, q, &ev);
        if (steps == 0) { e0 = et; j0 = jt; }
        if (fabs(ev.norm - 1.0) > ndev) ndev = fabs(ev.norm - 1.0);
        if (fabs(et - e0) > edev) edev = fabs(et - e0);
        if (fabs(jt - j0) > jdev) jdev = fabs(jt - j0);
    }
    for (int s = 0; s < n; ++s) a_out[s] = a[s];
    res->steps = steps;
    res->status = status;
    res->norm_dev = ndev;
    res->energy_dev = edev;
    res->angmom_dev = jdev;
    res->t_final = t;
    res->R = q[0]; res->PR = q[1]; res->Phi = q[2]; res->PPhi = q[3];
    free(a);
    work_free(&W);
    return ORA_OK;
}

/* Propagate n_traj trajectories (Sec. II / III).  final_amp: [n_traj][n] complex (interleaved re, im).
 * line_speed: prescribed-line speed per trajectory (only with ORA_F_PRESCRIBED; the line is
 * time-symmetric about max_steps*dt/2 with impact parameter b). */
/* v_lambda(R) and its first two R-derivatives from the system's splines at npts distances
 * (out: [npts][L] each) */
int ora_sys_terms(const ora_system_desc *d, int npts, const double *R, double *v, double *dv, double *d2v)
{
    ora_sys S;
    int e = sys_build(d, &S);
    if (e) return e;
    for (int i = 0; i < npts; ++i)
        eval_terms(&S, S.coef, R[i], v + (size_t)i * S.L, dv + (size_t)i * S.L, d2v + (size_t)i * S.L);
    sys_free(&S);
    return ORA_OK;
}

/* the truncation's decision per element: keep[r * n + c] = 1 for a retained M_rc (0 for a
 * dropped one and for every pair of different m); dense n x n output, small systems only */
int ora_sys_kept(const ora_system_desc *d, unsigned char *keep)
{
    ora_sys S;
    int e = sys_build(d, &S);
    if (e) return e;
    int n = S.n;
    memset(keep, 0, (size_t)n * n);
    for (int b = 0; b < S.n_blk; ++b) {
        int sz = S.blk_size[b];
        const int *mem = S.members + S.blk_start[b];
        for (int r = 0; r < sz; ++r)
            for (int c = 0; c < sz; ++c) keep[(size_t)mem[r] * n + mem[c]] = (unsigned char)kept(&S, b, r, c);
    }
    sys_free(&S);
    return ORA_OK;
}

int ora_propagate(const ora_system_desc *d, const ora_traj *tr, int n_traj, int flags, const double *line_speed,
                  int n_threads, double *final_amp, ora_result *res)
{
    ora_sys S;
    int e = sys_build(d, &S);
    if (e) return e;
    for (int i = 0; i < n_traj; ++i)
        if (tr[i].init_state < 0 || tr[i].init_state >= d->n || !(tr[i].dt > 0) || tr[i].max_steps < 0) {
            sys_free(&S);
            return ORA_EINVAL;
        }
    if ((flags & ORA_F_DECOUPLED) && (flags & ORA_F_PRESCRIBED)) { sys_free(&S); return ORA_EINVAL; }
    if (flags & ORA_F_DECOUPLED) {
        /* term 0 must be the isotropic term: G^0 = identity (to the rounding of its construction) */
        for (int b = 0; b < S.n_blk; ++b) {
            int sz = S.blk_size[b];
            for (int r = 0; r < sz; ++r)
                for (int c = 0; c < sz; ++c) {
                    double g = S.Gb[S.blk_goff[b] + (size_t)r * sz + c];
                    if (fabs(g - (r == c ? 1.0 : 0.0)) > 1e-13) { sys_free(&S); return ORA_EINVAL; }
                }
        }
    }
    int err = 0;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int i = 0; i < n_traj; ++i) {
        ora_opts o;
        o.flags = flags;
        o.jy_sign = (flags & ORA_F_FLIP_JY) ? -1.0 : 1.0;
        o.line_b = tr[i].b;
        o.line_v = line_speed ? line_speed[i] : 0.0;
        o.line_t0 = 0.5 * tr[i].max_steps * tr[i].dt;
        o.tol = d->adapt_tol;
        o.hmax_factor = d->adapt_hmax_factor > 0 ? (double)d->adapt_hmax_factor : 16.0;
        if (propagate_one(&S, tr + i, &o, (double complex *)(final_amp + 2 * (size_t)i * d->n), res + i))
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = ORA_ENOMEM;
    }
    sys_free(&S);
    return err;
}

/* ------------------------------------------------------------------ */
/* Forward tangent: exact derivative of the same discrete RK4 map with */
/* respect to the parameters whose dv_lambda/dtheta tables are given.  */
/* ------------------------------------------------------------------ */
typedef struct {
    double complex *da;
    double dq[4];
} tan_state;

/* tangent right-hand side for parameter p: given (a, q), the tangents (ta, tq) and the forward
 * quantities already in W (c, w = M c, u = M' c) */
static void rhs_tangent(const ora_sys *S, const ora_opts *o, double t, int p, const double complex *a, const double *q,
                        const double complex *ta, const double *tq, double complex *dta, double *dtq, ora_work *W,
                        double complex *tc, double complex *tw, double complex *tu, double complex *scr)
{
    int n = S->n, L = S->L;
    double R = q[0], PPhi = q[3], mu = S->mu;
    double phidot = PPhi / (mu * R * R);
    double tphidot = tq[3] / (mu * R * R) - 2.0 * PPhi * tq[0] / (mu * R * R * R);
    eval_terms(S, S->dcoef + (size_t)p * L * S->n_int * 4, R, W->pv, W->pdv, W->pd2v);
    for (int s = 0; s < n; ++s) tc[s] = cexp(-I * S->E[s] * t) * ta[s];
    /* tw = M tc + tR M' c + M_theta c */
    couple(S, W->v, tc, tw);
    couple(S, W->pv, W->c, scr);
    for (int s = 0; s < n; ++s) tw[s] += tq[0] * W->u[s] + scr[s];
    /* tu = M' tc + tR M'' c + M'_theta c */
    couple(S, W->dv, tc, tu);
    couple(S, W->pdv, W->c, scr);
    for (int s = 0; s < n; ++s) tu[s] += tq[0] * W->u2[s] + scr[s];
    double tforce = 0.0, ttorque = 0.0;
    for (int s = 0; s < n; ++s) {
        tforce -= creal(conj(tc[s]) * W->u[s] + conj(W->c[s]) * tu[s]);
        ttorque += creal(conj(tc[s]) * ladder(S, W->w, s) + conj(W->c[s]) * ladder(S, tw, s));
    }
    tforce += 2.0 * PPhi * tq[3] / (mu * R * R * R) - 3.0 * PPhi * PPhi * tq[0] / (mu * R * R * R * R);
    ttorque *= o->jy_sign;
    for (int s = 0; s < n; ++s)
        dta[s] = -I * cexp(I * S->E[s] * t) * tw[s] +
                 o->jy_sign * 0.5 * (tphidot * ladder(S, a, s) + phidot * ladder(S, ta, s));
    dtq[0] = tq[1] / mu;
    dtq[1] = tforce;
    dtq[2] = tphidot;
    dtq[3] = ttorque;
}

static int tangent_one(const ora_sys *S, const ora_traj *tr, double complex *a_out, double *dpop, ora_result *res)
{
    int n = S->n, P = S->P;
    ora_opts o;
    memset(&o, 0, sizeof(o));
    o.jy_sign = 1.0;
    ora_work W;
    if (work_alloc(&W, n, S->L)) { work_free(&W); return ORA_ENOMEM; }
    size_t na = (size_t)n;
    /* forward: a, k1..k4, ys; tangents: ta[P], tk[4][P], tys; scratch */
    double complex *buf = malloc(sizeof(double complex) * na * (6 + 6 * (size_t)P + 4));
    double *tqbuf = malloc(sizeof(double) * 4 * 6 * (size_t)(P > 0 ? P : 1));
    if (!buf || !tqbuf) { free(buf); free(tqbuf); work_free(&W); return ORA_ENOMEM; }
    double complex *a = buf, *k[4] = {buf + na, buf + 2 * na, buf + 3 * na, buf + 4 * na}, *ys = buf + 5 * na;
    double complex *ta = buf + 6 * na;                          /* [P][n]    */
    double complex *tk = ta + (size_t)P * na;                   /* [4][P][n] */
    double complex *tys = tk + 4 * (size_t)P * na;              /* [P][n]    */
    double complex *tc = tys + (size_t)P * na, *tw = tc + na, *tu = tw + na, *scr = tu + na;
    double *tq = tqbuf, *tl = tqbuf + 4 * P, *tqs = tqbuf + 20 * P; /* tq[P][4], tl[4][P][4], tqs[P][4] */
    double q[4], qs[4], l[4][4];
    double m00;
    initial_state(S, tr, 0, a, q, &m00);
    /* tangent of the initial state: only P_R depends on theta through M_s0s0(R0) */
    memset(ta, 0, sizeof(double complex) * (size_t)P * na);
    memset(tq, 0, sizeof(double) * 4 * P);
    {
        int s0 = tr->init_state, b = -1, r = -1;
        for (int q2 = 0; q2 < S->n_blk && b < 0; ++q2)
            for (int i = 0; i < S->blk_size[q2]; ++i)
                if (S->members[S->blk_start[q2] + i] == s0) { b = q2; r = i; }
        int sz = S->blk_size[b];
        for (int p = 0; p < P; ++p) {
            eval_terms(S, S->dcoef + (size_t)p * S->L * S->n_int * 4, tr->r0, W.pv, W.pdv, W.pd2v);
            double dm00 = 0.0;
            if (kept(S, b, r, r))
                for (int l2 = 0; l2 < S->L; ++l2) dm00 += W.pv[l2] * S->Gb[S->blk_goff[b] + ((size_t)l2 * sz + r) * sz + r];
            tq[4 * p + 1] = -S->mu * dm00 / q[1];
        }
    }
    double dt = tr->dt;
    int steps = 0, stopped = 0, status = 0;
    static const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    for (int step = 0; step < tr->max_steps; ++step) {
        double t = step * dt;
        for (int st = 0; st < 4; ++st) {
            double ts = t + cst[st] * dt;
            const double complex *ya = a;
            const double *yq = q;
            if (st > 0) {
                double f = cst[st] * dt;
                for (int s = 0; s < n; ++s) ys[s] = a[s] + f * k[st - 1][s];
                for (int i = 0; i < 4; ++i) qs[i] = q[i] + f * l[st - 1][i];
                for (int p = 0; p < P; ++p) {
                    for (int s = 0; s < n; ++s)
                        tys[(size_t)p * na + s] = ta[(size_t)p * na + s] + f * tk[((size_t)(st - 1) * P + p) * na + s];
                    for (int i = 0; i < 4; ++i) tqs[4 * p + i] = tq[4 * p + i] + f * tl[((st - 1) * P + p) * 4 + i];
                }
                ya = ys;
                yq = qs;
            } else {
                memcpy(tys, ta, sizeof(double complex) * (size_t)P * na);
                memcpy(tqs, tq, sizeof(double) * 4 * P);
            }
            ora_eval ev;
            rhs(S, &o, ts, ya, yq, k[st], l[st], &W, &ev);
            if (ev.below) status |= ORA_ST_TABLE_RANGE;
            couple(S, W.d2v, W.c, W.u2); /* M'' c for the tangents */
            for (int p = 0; p < P; ++p)
                rhs_tangent(S, &o, ts, p, ya, yq, tys + (size_t)p * na, tqs + 4 * p,
                            tk + ((size_t)st * P + p) * na, tl + (st * P + p) * 4, &W, tc, tw, tu, scr);
        }
        for (int s = 0; s < n; ++s) a[s] += dt / 6.0 * (k[0][s] + 2.0 * k[1][s] + 2.0 * k[2][s] + k[3][s]);
        for (int i = 0; i < 4; ++i) q[i] += dt / 6.0 * (l[0][i] + 2.0 * l[1][i] + 2.0 * l[2][i] + l[3][i]);
        for (int p = 0; p < P; ++p) {
            for (int s = 0; s < n; ++s) {
                size_t o2 = (size_t)p * na + s;
                ta[o2] += dt / 6.0 * (tk[o2] + 2.0 * tk[(size_t)P * na + o2] + 2.0 * tk[2 * (size_t)P * na + o2] +
                                      tk[3 * (size_t)P * na + o2]);
            }
            for (int i = 0; i < 4; ++i)
                tq[4 * p + i] += dt / 6.0 * (tl[(0 * P + p) * 4 + i] + 2.0 * tl[(1 * P + p) * 4 + i] +
                                             2.0 * tl[(2 * P + p) * 4 + i] + tl[(3 * P + p) * 4 + i]);
        }
        steps = step + 1;
        if (!finite_state(n, a, q)) { status |= ORA_ST_NONFINITE; stopped = 1; break; }
        if (q[0] >= tr->r_end && q[1] > 0.0) { stopped = 1; break; }
    }
    if (!stopped) status |= ORA_ST_MAX_STEPS;
    for (int s = 0; s < n; ++s) a_out[s] = a[s];
    /* d|a_s|^2 / d theta_p = 2 Re(conj(a_s) ta_s) */
    for (int p = 0; p < P; ++p)
        for (int s = 0; s < n; ++s) dpop[(size_t)p * n + s] = 2.0 * creal(conj(a[s]) * ta[(size_t)p * na + s]);
    memset(res, 0, sizeof(*res));
    res->steps = steps;
    res->status = status;
    res->t_final = steps * dt;
    res->R = q[0]; res->PR = q[1]; res->Phi = q[2]; res->PPhi = q[3];
    free(buf);
    free(tqbuf);
    work_free(&W);
    return ORA_OK;
}

/* final amplitudes and d|a|^2/dtheta: dpop[n_traj][P][n] */
int ora_tangent(const ora_system_desc *d, const ora_traj *tr, int n_traj, int n_threads, double *final_amp,
                double *dpop, ora_result *res)
{
    if (d->n_params < 1 || !d->dvp || !d->dvp_ends) return ORA_EINVAL;
    ora_sys S;
    int e = sys_build(d, &S);
    if (e) return e;
    for (int i = 0; i < n_traj; ++i)
        if (tr[i].init_state < 0 || tr[i].init_state >= d->n || !(tr[i].dt > 0) || tr[i].max_steps < 0) {
            sys_free(&S);
            return ORA_EINVAL;
        }
    int err = 0;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int i = 0; i < n_traj; ++i)
        if (tangent_one(&S, tr + i, (double complex *)(final_amp + 2 * (size_t)i * d->n),
                        dpop + (size_t)i * d->n_params * d->n, res + i))
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = ORA_ENOMEM;
    sys_free(&S);
    return err;
}

/* ------------------------------------------------------------------ */
/* Cross sections (Sec. II): populations summed over the final level,  */
/* weighted (impact-parameter quadrature and initial-m average) and    */
/* summed over the trajectories of each group.                         */
/* ------------------------------------------------------------------ */
void ora_cross_sections(int n, const int *level, int n_levels, int n_traj, const double *pop, const double *weight,
                        const int *group, int n_groups, double *sigma)
{
    memset(sigma, 0, sizeof(double) * (size_t)n_groups * n_levels);
    for (int t = 0; t < n_traj; ++t) {
        if (group[t] < 0 || group[t] >= n_groups) continue;
        for (int s = 0; s < n; ++s)
            sigma[(size_t)group[t] * n_levels + level[s]] += weight[t] * pop[(size_t)t * n + s];
    }
}

int ora_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Rigid asymmetric top (Eq. 1 basis) and its coupling to an atom      */
/* (Eq. 16 integrals of three Wigner D-functions)                      */
/* ------------------------------------------------------------------ */
/* Rotor Hamiltonian A Ja^2 + B Jb^2 + C Jc^2 for one J in the symmetric-top functions
 * |J K> (K = projection on the a axis, index K + J), with Jb, Jc taken as Jx, Jy:
 *   <K|H|K>   = (B+C)/2 (J(J+1) - K^2) + A K^2
 *   <K+2|H|K> = (B-C)/4 sqrt((J-K)(J-K-1)(J+K+1)(J+K+2)). */
static void asym_h(int J, double A, double B, double C, double *H)
{
    int n = 2 * J + 1;
    memset(H, 0, sizeof(double) * n * n);
    for (int K = -J; K <= J; ++K) {
        H[(K + J) * n + (K + J)] = 0.5 * (B + C) * ((double)J * (J + 1) - (double)K * K) + A * (double)K * K;
        if (K + 2 <= J) {
            double x = 0.25 * (B - C) * sqrt((double)(J - K) * (J - K - 1) * (J + K + 1) * (J + K + 2));
            H[(K + 2 + J) * n + (K + J)] = x;
            H[(K + J) * n + (K + 2 + J)] = x;
        }
    }
}

/* Wang's symmetrised functions, column w of U (|K> rows): w = 0 is |0>, then for
 * K = 1..J the pair (|K> + |-K>)/sqrt2, (|K> - |-K>)/sqrt2.  H is invariant under K -> -K,
 * so U^T H U has no element between the + and - combinations (nor between even and odd K):
 * every eigenvector stays inside one symmetry class, also for near-degenerate pairs. */
static void wang_basis(int J, double *U)
{
    int n = 2 * J + 1;
    double r = sqrt(0.5);
    memset(U, 0, sizeof(double) * n * n);
    U[J * n + 0] = 1.0;
    for (int K = 1; K <= J; ++K) {
        int wp = 2 * K - 1, wm = 2 * K;
        U[(K + J) * n + wp] = r;  U[(-K + J) * n + wp] = r;
        U[(K + J) * n + wm] = r;  U[(-K + J) * n + wm] = -r;
    }
}

/* cyclic Jacobi rotations on the symmetric matrix a (destroyed); v = eigenvectors (columns), w = eigenvalues */
static void jacobi_eigen(int n, double *a, double *v, double *w)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) v[i * n + j] = (i == j);
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p) {
            diag += a[p * n + p] * a[p * n + p];
            for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
        }
        if (off <= 1e-34 * diag || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = a[p * n + q];
                if (apq == 0.0) continue;
                double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = v[k * n + p], vkq = v[k * n + q];
                    v[k * n + p] = c * vkp - s * vkq;
                    v[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = a[i * n + i];
}

/* Eigenstates of one J (Eq. 1): E[e] ascending (e = 0..2J, tau = e - J), b[e][K + J] the expansion
 * coefficients b_K.  Sign: the largest-magnitude Wang component of each eigenvector is positive
 * (first such component on a tie). */
int ora_asym_levels(int J, double A, double B, double C, double *E, double *b)
{
    int n = 2 * J + 1;
    double *H = malloc(sizeof(double) * n * n), *U = malloc(sizeof(double) * n * n);
    double *Hw = malloc(sizeof(double) * n * n), *V = malloc(sizeof(double) * n * n);
    double *w = malloc(sizeof(double) * n);
    int *idx = malloc(sizeof(int) * n);
    if (!H || !U || !Hw || !V || !w || !idx) {
        free(H); free(U); free(Hw); free(V); free(w); free(idx);
        return ORA_ENOMEM;
    }
    asym_h(J, A, B, C, H);
    wang_basis(J, U);
    for (int p = 0; p < n; ++p)          /* Hw = U^T H U, zero between classes (exactly, not to rounding) */
        for (int q = 0; q < n; ++q) {
            int Kp = (p + 1) / 2, Kq = (q + 1) / 2;
            int sp = p > 0 && p % 2 == 0, sq = q > 0 && q % 2 == 0;  /* 1 for the (|K> - |-K>) combination */
            double s = 0.0;
            if ((Kp - Kq) % 2 == 0 && sp == sq)
                for (int k = 0; k < n; ++k)
                    for (int l = 0; l < n; ++l) s += U[k * n + p] * H[k * n + l] * U[l * n + q];
            Hw[p * n + q] = s;
        }
    jacobi_eigen(n, Hw, V, w);
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int i = 0; i < n; ++i)          /* ascending energy */
        for (int j = i + 1; j < n; ++j)
            if (w[idx[j]] < w[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int e = 0; e < n; ++e) {
        int src = idx[e], big = 0;
        for (int k = 1; k < n; ++k)
            if (fabs(V[k * n + src]) > fabs(V[big * n + src])) big = k;
        double sg = V[big * n + src] < 0 ? -1.0 : 1.0;
        E[e] = w[src];
        for (int K = 0; K < n; ++K) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += U[K * n + k] * V[k * n + src];
            b[e * n + K] = sg * s;
        }
    }
    free(H); free(U); free(Hw); free(V); free(w); free(idx);
    return ORA_OK;
}

/* Levels (J, tau) for J <= jmax in ascending energy (ties: smaller J first), keeping whole
 * multiplets (all 2J+1 values of M) while the total number of states stays <= max_states.
 * Output arrays hold (jmax+1)^2 levels; lev_b[l][K + jmax] (row length 2 jmax + 1).
 * Returns the number of levels kept, or -1 on allocation failure. */
int ora_asym_basis(int jmax, double A, double B, double C, int max_states, int *lev_J, int *lev_tau,
                   double *lev_E, double *lev_b)
{
    int nall = (jmax + 1) * (jmax + 1), w = 2 * jmax + 1;
    int *aJ = malloc(sizeof(int) * nall), *at = malloc(sizeof(int) * nall), *ord = malloc(sizeof(int) * nall);
    double *aE = malloc(sizeof(double) * nall), *ab = calloc((size_t)nall * w, sizeof(double));
    double *E = malloc(sizeof(double) * w), *b = malloc(sizeof(double) * w * w);
    if (!aJ || !at || !ord || !aE || !ab || !E || !b) {
        free(aJ); free(at); free(ord); free(aE); free(ab); free(E); free(b);
        return -1;
    }
    int k = 0;
    for (int J = 0; J <= jmax; ++J) {
        int n = 2 * J + 1;
        ora_asym_levels(J, A, B, C, E, b);
        for (int e = 0; e < n; ++e, ++k) {
            aJ[k] = J; at[k] = e - J; aE[k] = E[e];
            for (int K = -J; K <= J; ++K) ab[(size_t)k * w + K + jmax] = b[e * n + K + J];
        }
    }
    for (int i = 0; i < nall; ++i) ord[i] = i;
    for (int i = 0; i < nall; ++i)       /* stable selection by (E, J) */
        for (int j = i + 1; j < nall; ++j) {
            int a = ord[i], c = ord[j];
            if (aE[c] < aE[a] || (aE[c] == aE[a] && aJ[c] < aJ[a])) { ord[i] = c; ord[j] = a; }
        }
    int nl = 0, ns = 0;
    for (int i = 0; i < nall; ++i) {
        int s = ord[i];
        if (ns + 2 * aJ[s] + 1 > max_states) break;
        ns += 2 * aJ[s] + 1;
        lev_J[nl] = aJ[s]; lev_tau[nl] = at[s]; lev_E[nl] = aE[s];
        memcpy(lev_b + (size_t)nl * w, ab + (size_t)s * w, sizeof(double) * w);
        ++nl;
    }
    free(aJ); free(at); free(ord); free(aE); free(ab); free(E); free(b);
    return nl;
}

/* Coupling matrix of one expansion term (Eq. 12) between the states (level, M), levels in the given
 * order and M = -J..J inside each level.  The angular function is
 *   f_{lam mu} = (D^{lam*}_{0 mu} + (-1)^mu D^{lam*}_{0,-mu}) / (1 + delta_{mu 0}),  0 <= mu <= lam,
 * real (2 d^lam_{0 mu}(beta) cos(mu gamma), or P_lam(cos beta) for mu = 0).  With Eq. 16 and the
 * normalisation sqrt((2J+1)/(8 pi^2)) of Eq. 1,
 *   <J'' K'' M | D^{lam*}_{0 nu} | J' K' M> = sqrt((2J'+1)/(2J''+1)) C^{J''M}_{J'M lam 0} C^{J''K''}_{J'K' lam nu},
 * and the eigenstates add these with weights b''_{K''} b'_{K'}.  G[n][n], row = final state. */
void ora_asym_G(int n_lev, const int *lev_J, const double *lev_b, int jmax, int lam, int mu, int n, double *G)
{
    int w = 2 * jmax + 1;
    int *first = malloc(sizeof(int) * (n_lev + 1));
    first[0] = 0;
    for (int l = 0; l < n_lev; ++l) first[l + 1] = first[l] + 2 * lev_J[l] + 1;
    memset(G, 0, sizeof(double) * (size_t)n * n);
    double sgn = (mu & 1) ? -1.0 : 1.0;
#pragma omp parallel for schedule(dynamic)
    for (int l2 = 0; l2 < n_lev; ++l2)
        for (int l1 = 0; l1 < n_lev; ++l1) {
            int J2 = lev_J[l2], J1 = lev_J[l1];
            if (abs(J2 - J1) > lam || J2 + J1 < lam) continue;
            const double *b2 = lev_b + (size_t)l2 * w + jmax, *b1 = lev_b + (size_t)l1 * w + jmax;
            double S = 0.0;  /* the K sum: independent of M */
            for (int K1 = -J1; K1 <= J1; ++K1) {
                int Kp = K1 + mu, Km = K1 - mu;
                if (Kp >= -J2 && Kp <= J2) S += b2[Kp] * b1[K1] * ora_cg(J1, K1, lam, mu, J2, Kp);
                if (mu > 0 && Km >= -J2 && Km <= J2) S += sgn * b2[Km] * b1[K1] * ora_cg(J1, K1, lam, -mu, J2, Km);
            }
            if (S == 0.0) continue;
            double pre = sqrt((2.0 * J1 + 1.0) / (2.0 * J2 + 1.0)) * S;
            int Mmax = J1 < J2 ? J1 : J2;
            for (int M = -Mmax; M <= Mmax; ++M) {
                int r = first[l2] + M + J2, c = first[l1] + M + J1;
                if (r < n && c < n) G[(size_t)r * n + c] = pre * ora_cg(J1, M, lam, 0, J2, M);
            }
        }
    free(first);
}

/* ------------------------------------------------------------------ */
/* Asymmetric top + linear rotor (Eqs. 3, 13-17)                      */
/* ------------------------------------------------------------------ */
/* Coupling matrix of one expansion term tau_{lam1 mu1 lam2 lam} (Eq. 13) between the composite states
 * |n m> of Eq. 3.  State s is given by its molecule-1 level l1[s] (J = lev_J[l1], eigenvector
 * lev_b[l1][K + jmax1] of Eq. 1), the rotor's j2[s], the total j[s] and the projection m[s].  With
 * Eq. 16 for molecule 1 (normalisation sqrt((2j1+1)/(8 pi^2)) of Eq. 3):
 *   <j1'' m1'' K''| D^{lam1*}_{eta nu} |j1' m1' K'> = sqrt((2j1'+1)/(2j1''+1)) C^{j1'' m1''}_{j1' m1' lam1 eta}
 *                                                   C^{j1'' K''}_{j1' K' lam1 nu},
 * Eq. 15 for molecule 2, and the couplings of Eq. 3 for both states (Eq. 17 before the CG
 * selection rules are used).  G[n][n], row = final state, zero between different m. */
void ora_molmol_G(int n, const int *l1, const int *j2, const int *jt, const int *mt, const int *lev_J,
                  const double *lev_b, int jmax1, int lam1, int mu1, int lam2, int lam, double *G)
{
    const double pi = 3.14159265358979323846;
    const int w = 2 * jmax1 + 1;
    const double sgn = ((lam1 + mu1 + lam2 + lam) & 1) ? -1.0 : 1.0;
    memset(G, 0, sizeof(double) * (size_t)n * n);
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            if (mt[r] != mt[c]) continue;
            const int m = mt[r];
            const int J2 = lev_J[l1[r]], J1 = lev_J[l1[c]], a2 = j2[r], a1 = j2[c];
            const double *b2 = lev_b + (size_t)l1[r] * w + jmax1, *b1 = lev_b + (size_t)l1[c] * w + jmax1;
            /* molecule 1: the K sums of the two D functions of Eq. 13 (independent of m1) */
            double Kp = 0.0, Km = 0.0;
            for (int K1 = -J1; K1 <= J1; ++K1) {
                if (K1 + mu1 >= -J2 && K1 + mu1 <= J2) Kp += b2[K1 + mu1] * b1[K1] * ora_cg(J1, K1, lam1, mu1, J2, K1 + mu1);
                if (K1 - mu1 >= -J2 && K1 - mu1 <= J2) Km += b2[K1 - mu1] * b1[K1] * ora_cg(J1, K1, lam1, -mu1, J2, K1 - mu1);
            }
            const double Ksum = Kp + sgn * Km;
            if (Ksum == 0.0) continue;
            const double c2 = ora_cg(a1, 0, lam2, 0, a2, 0);
            if (c2 == 0.0) continue;
            const double pre1 = sqrt((2.0 * J1 + 1.0) / (2.0 * J2 + 1.0));
            const double pre2 = sqrt((2.0 * a1 + 1.0) * (2.0 * lam2 + 1.0) / (4.0 * pi * (2.0 * a2 + 1.0))) * c2;
            double acc = 0.0;
            const int emax = lam1 < lam2 ? lam1 : lam2;
            for (int eta = -emax; eta <= emax; ++eta) {
                const double ce = ora_cg(lam1, eta, lam2, -eta, lam, 0);
                if (ce == 0.0) continue;
                for (int m1 = -J1; m1 <= J1; ++m1) {
                    const int m2 = m - m1, n1 = m1 + eta, n2 = m2 - eta;   /* m1'' = m1' + eta, m2'' = m2' - eta */
                    if (abs(m2) > a1 || abs(n1) > J2 || abs(n2) > a2) continue;
                    const double cin = ora_cg(J1, m1, a1, m2, jt[c], m);
                    const double cout = ora_cg(J2, n1, a2, n2, jt[r], m);
                    if (cin == 0.0 || cout == 0.0) continue;
                    acc += ce * cin * cout * pre1 * ora_cg(J1, m1, lam1, eta, J2, n1) * Ksum * pre2 *
                           ora_cg(a1, m2, lam2, -eta, a2, n2);
                }
            }
            G[(size_t)r * n + c] = sqrt((2.0 * lam1 + 1.0) / (4.0 * pi)) * acc;
        }
}
