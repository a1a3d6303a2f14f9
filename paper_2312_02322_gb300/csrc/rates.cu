// Post-processing of cross sections (Sec. III): the symmetrised cross sections of Eq. 20 and
// the Maxwell-Boltzmann rate coefficients of both directions of every transition.
//
// Readings (the paper defers the integration to its ref. [44]):
//   R1  U, the energy at which Eq. 19 compares both directions, is the mean of the incoming and
//       outgoing translational energies;
//   R2  k_{a->b}(T) = (8/(pi mu))^(1/2) (kT)^(-3/2) exp(-(E_b - E_a)/(2kT)) / g_a
//                      * int_{u0}^inf sigma~_ab(U) U exp(-U/kT) dU,
//       so that g_a k_{a->b} = g_b k_{b->a} exp(-(E_b - E_a)/kT) holds exactly;
//   R3  natural cubic spline of sigma~ in U through the computed energies, negative values
//       taken as zero;
//   R4  u0 = |E_b - E_a| / 2; below U_1 a linear ramp from zero at u0, or the spline cut at u0
//       when u0 >= U_1;
//   R5  above U_K the power law sigma~_K (U/U_K)^p, p the log-log slope of the last two points
//       clipped to [-1, 0], integrated in closed form with the upper incomplete gamma function.
//
// One thread per (unordered pair of levels, temperature).  The spline's second derivatives are
// a fixed linear map of the knot values (set up on the host from the energy grid), the finite
// pieces are integrated by 16-point Gauss-Legendre panels no wider than 4 kT (the exponential at the
// nodes as a panel factor times node factors shared by the panels of a piece), and the integrand
// carries exp(-(U - u0)/kT) so that neither exponential factor of R2 overflows.  The walk stops at
// the first panel whose remainder bound (4 max|y| kT (U + kT) exp(-(U - u0)/kT) at its lower edge U)
// is below 1e-17 of the integral so far; the tail is then dropped too.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace mqct {

namespace {

constexpr int kRateMaxK = MQCT_RATE_MAX_ENERGIES;
constexpr int kRateMaxT = MQCT_RATE_MAX_TEMPS;
constexpr int kGl = 16;

struct RateArgs {
    double u[kRateMaxK];
    double Q[kRateMaxK][kRateMaxK];  // second derivatives of the natural spline: M = Q y
    double gx[kGl], gw[kGl];         // Gauss-Legendre nodes and weights on [-1, 1]
    double kT[kRateMaxT];
    double pref;                     // (8 / (pi mu))^(1/2)
    int K, L, n_T;
    long long n_pairs;
};

// Gamma(s, x) e^x for 1 <= s <= 2, x > 0.  Below x = s + 1 the power series of the lower
// function gamma(s, x) = x^s e^-x sum_n x^n / (s (s+1) ... (s+n)) (Abramowitz & Stegun 6.5.29)
// is subtracted from Gamma(s); above, Legendre's continued fraction (A&S 6.5.31) is evaluated
// by the modified Lentz algorithm.
__device__ double upper_gamma_scaled(double s, double x)
{
    if (s == 1.0) return 1.0;
    if (s == 2.0) return 1.0 + x;
    if (x < s + 1.0) {
        double term = 1.0 / s, sum = term;
        for (int n = 1; n < 200; ++n) {
            term *= x / (s + n);
            sum += term;
            if (fabs(term) < 1e-17 * sum) break;
        }
        return tgamma(s) * exp(x) - pow(x, s) * sum;
    }
    const double tiny = 1e-300;
    double b = x + 1.0 - s, c = 1.0 / tiny, d = 1.0 / b, f = d;
    for (int i = 1; i < 300; ++i) {
        const double an = -i * (i - s);
        b += 2.0;
        d = an * d + b;
        if (fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        const double del = d * c;
        f *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    return pow(x, s) * f;
}

__global__ void k_rate_sym(const double *sigma, const double *g, int K, int L, double *out)
{
    const long long n = (long long)K * L * L;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i % L), a = (int)((i / L) % L);
        const long long k = i / ((long long)L * L);
        out[i] = 0.5 * (g[a] * sigma[i] + g[b] * sigma[(k * L + b) * L + a]);
    }
}

__global__ void __launch_bounds__(128) k_rates(const __grid_constant__ RateArgs A, const double *sigma,
                                                const double *g, const double *E, double *rate)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= A.n_pairs * A.n_T) return;
    // temperature is the slow index: the lanes of a warp share kT and so take similar panel counts
    const int t = (int)(i / A.n_pairs);
    const long long q = i % A.n_pairs;
    // q = b (b + 1) / 2 + a with a <= b
    long long b = (long long)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
    while (b * (b + 1) / 2 > q) --b;
    while ((b + 1) * (b + 2) / 2 <= q) ++b;
    const int ib = (int)b, ia = (int)(q - b * (b + 1) / 2);
    const int K = A.K, L = A.L;
    const double ga = g[ia], gb = g[ib];
    double y[kRateMaxK], M[kRateMaxK];
    double ymax = 0.0;
    for (int k = 0; k < K; ++k) {
        const size_t base = (size_t)k * L * L;
        y[k] = 0.5 * (ga * sigma[base + (size_t)ia * L + ib] + gb * sigma[base + (size_t)ib * L + ia]);
        ymax = fmax(ymax, fabs(y[k]));
    }
    for (int k = 0; k < K; ++k) {
        double m = 0.0;
        for (int j = 0; j < K; ++j) m = fma(A.Q[k][j], y[j], m);
        M[k] = m;
    }
    const double th = A.kT[t], ith = 1.0 / th;
    const double dE = E[ib] - E[ia], u0 = 0.5 * fabs(dE);
    // acc = int sigma~ U exp(-(U - u0)/kT) dU, piece by piece in increasing U
    double acc = 0.0;
    bool done = false;
    auto piece = [&](double lo, double hi, int kind, int k) {
        // remainder above lo bounded by 4 max|y| kT (lo + kT) exp(-(lo - u0)/kT)
        if (done || hi <= lo) return;
        if (4.0 * ymax * th * (lo + th) * exp(-(lo - u0) * ith) <= 1e-17 * acc) { done = true; return; }
        const int np = (int)fmin(256.0, fmax(1.0, ceil((hi - lo) * 0.25 * ith)));
        const double hp = (hi - lo) / np;
        const double h = kind ? A.u[k + 1] - A.u[k] : 0.0;
        // reciprocals once per piece (an FP64 division costs ~10 FMA slots on this GPU's FP64 pipe)
        const double ih = kind ? 1.0 / h : 0.0, iramp = kind ? 0.0 : y[0] / (A.u[0] - u0);
        const double h26 = h * h * (1.0 / 6.0);
        // exp(-(U - u0)/kT) = exp(-(c - u0)/kT) exp(-(hp/2) x_j / kT): the node factors are the same
        // for every panel of the piece
        double ef[kGl];
#pragma unroll
        for (int j = 0; j < kGl; ++j) ef[j] = exp(-0.5 * hp * A.gx[j] * ith);
        // the same remainder bound at each panel's lower edge c - hp/2, from the panel factor:
        // exp(-(c - hp/2 - u0)/kT) = exp(-(c - u0)/kT) exp(hp/(2kT))
        const double bnd = 4.0 * ymax * th * exp(0.5 * hp * ith);
        for (int p = 0; p < np; ++p) {
            const double c = lo + hp * (p + 0.5);
            const double ec = exp(-(c - u0) * ith);
            if (p > 0 && bnd * (c - 0.5 * hp + th) * ec <= 1e-17 * acc) { done = true; return; }
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < kGl; ++j) {
                const double U = fma(0.5 * hp, A.gx[j], c);
                double v;
                if (kind == 0) {
                    v = (U - u0) * iramp;
                } else {
                    const double tt = (U - A.u[k]) * ih, st = 1.0 - tt;
                    v = st * y[k] + tt * y[k + 1] + h26 * ((st * st * st - st) * M[k] + (tt * tt * tt - tt) * M[k + 1]);
                    v = fmax(v, 0.0);
                }
                s = fma(A.gw[j], v * U * (ec * ef[j]), s);
            }
            acc = fma(0.5 * hp, s, acc);
        }
    };
    if (u0 < A.u[0]) piece(u0, A.u[0], 0, 0);
    for (int k = 0; k + 1 < K; ++k) piece(fmax(A.u[k], u0), A.u[k + 1], 1, k);
    {
        // tail: y_K U_K^-p int_a^inf U^(1+p) exp(-(U - u0)/kT) dU
        //     = y_K U_K^-p kT^s [Gamma(s, a/kT) e^(a/kT)] exp(-(a - u0)/kT),  s = 2 + p
        const double a = fmax(A.u[K - 1], u0), yK = y[K - 1], yJ = y[K - 2];
        double p = 0.0;
        if (yK > 0.0 && yJ > 0.0) p = fmin(0.0, fmax(-1.0, log(yK / yJ) / log(A.u[K - 1] / A.u[K - 2])));
        if (yK != 0.0 && !done) {
            const double s = 2.0 + p, x = a * ith;
            acc += yK * pow(A.u[K - 1], -p) * pow(th, s) * upper_gamma_scaled(s, x) * exp(-(a - u0) * ith);
        }
    }
    const double c = A.pref * pow(th, -1.5) * acc;
    // exp(-dE/(2kT)) exp(-u0/kT): exp(-dE/kT) for an excitation, 1 for a quenching
    const double ab = c * exp(-(0.5 * dE + u0) * ith) / ga;
    const double ba = c * exp((0.5 * dE - u0) * ith) / gb;
    const size_t plane = (size_t)t * L * L;
    rate[plane + (size_t)ia * L + ib] = ab;
    rate[plane + (size_t)ib * L + ia] = ba;
}

// Gauss-Legendre nodes and weights by Newton's iteration on P_n (three-term recurrence)
void gauss_legendre(int n, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Q[k][j] = d M_k / d y_j for the natural spline on the knots u (M_0 = M_{K-1} = 0)
void natural_spline_map(const double *u, int K, double Q[kRateMaxK][kRateMaxK])
{
    for (int k = 0; k < kRateMaxK; ++k)
        for (int j = 0; j < kRateMaxK; ++j) Q[k][j] = 0.0;
    const int n = K - 2;
    if (n <= 0) return;
    std::vector<double> lo(n), di(n), up(n), cp(n), r(n);
    for (int i = 0; i < n; ++i) {
        const double h0 = u[i + 1] - u[i], h1 = u[i + 2] - u[i + 1];
        lo[i] = h0;
        di[i] = 2.0 * (h0 + h1);
        up[i] = h1;
    }
    for (int j = 0; j < K; ++j) {
        // right-hand side 6 [(y_{i+2} - y_{i+1}) / h1 - (y_{i+1} - y_i) / h0] for y = e_j
        for (int i = 0; i < n; ++i) {
            const double h0 = u[i + 1] - u[i], h1 = u[i + 2] - u[i + 1];
            const double yi = (j == i), yi1 = (j == i + 1), yi2 = (j == i + 2);
            r[i] = 6.0 * ((yi2 - yi1) / h1 - (yi1 - yi) / h0);
        }
        // Thomas
        cp[0] = up[0] / di[0];
        r[0] /= di[0];
        for (int i = 1; i < n; ++i) {
            const double m = di[i] - lo[i] * cp[i - 1];
            cp[i] = up[i] / m;
            r[i] = (r[i] - lo[i] * r[i - 1]) / m;
        }
        for (int i = n - 2; i >= 0; --i) r[i] -= cp[i] * r[i + 1];
        for (int i = 0; i < n; ++i) Q[i + 1][j] = r[i];
    }
}

bool rate_is_dev(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace mqct

using namespace mqct;

extern "C" mqct_status mqct_rate_coefficients(const mqct_rate_desc *d, const double *sigma, double *sigma_sym,
                                              double *rate, void *cuda_stream)
{
    reset_launches();
    if (!d || !sigma || !rate) return fail(MQCT_ERR_INVALID_ARG, "mqct_rate_coefficients: NULL argument");
    const int K = d->n_energies, L = d->n_levels, nT = d->n_temps;
    if (d->reserved != 0) return fail(MQCT_ERR_INVALID_ARG, "mqct_rate_coefficients: reserved must be 0");
    if (L < 1 || K < 2 || K > kRateMaxK || nT < 1 || nT > kRateMaxT)
        return fail(MQCT_ERR_INVALID_ARG, "mqct_rate_coefficients: sizes out of range");
    if (!d->u || !d->kT || !d->level_energy || !d->degeneracy)
        return fail(MQCT_ERR_INVALID_ARG, "mqct_rate_coefficients: NULL array in the descriptor");
    if (!(d->mu > 0.0) || !std::isfinite(d->mu)) return fail(MQCT_ERR_INVALID_ARG, "mqct_rate_coefficients: mu must be > 0");
    if (rate_is_dev(d->u) || rate_is_dev(d->kT) || rate_is_dev(d->level_energy) || rate_is_dev(d->degeneracy))
        return fail(MQCT_ERR_INVALID_ARG, "mqct_rate_coefficients: descriptor arrays must be host memory");
    RateArgs A;
    std::memset(&A, 0, sizeof(A));
    for (int k = 0; k < K; ++k) {
        A.u[k] = d->u[k];
        if (!(A.u[k] > 0.0) || !std::isfinite(A.u[k]) || (k > 0 && !(A.u[k] > A.u[k - 1])))
            return fail(MQCT_ERR_INVALID_ARG, "mqct_rate_coefficients: energies must be finite, > 0 and increasing");
    }
    for (int t = 0; t < nT; ++t) {
        A.kT[t] = d->kT[t];
        if (!(A.kT[t] > 0.0) || !std::isfinite(A.kT[t])) return fail(MQCT_ERR_INVALID_ARG, "mqct_rate_coefficients: kT must be > 0");
    }
    for (int l = 0; l < L; ++l) {
        if (!(d->degeneracy[l] > 0.0) || !std::isfinite(d->degeneracy[l]) || !std::isfinite(d->level_energy[l]))
            return fail(MQCT_ERR_INVALID_ARG, "mqct_rate_coefficients: degeneracies must be > 0, energies finite");
    }
    natural_spline_map(A.u, K, A.Q);
    gauss_legendre(kGl, A.gx, A.gw);
    A.pref = std::sqrt(8.0 / (3.14159265358979323846 * d->mu));
    A.K = K;
    A.L = L;
    A.n_T = nT;
    A.n_pairs = (long long)L * (L + 1) / 2;

    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e;
    std::vector<void *> tmp;
    auto get = [&](void **p, size_t b) {
        cudaError_t r = cudaMallocAsync(p, b ? b : 16, st);
        if (r == cudaSuccess) tmp.push_back(*p);
        return r;
    };
    auto cleanup = [&]() { for (void *p : tmp) cudaFreeAsync(p, st); };
    const size_t sig_bytes = sizeof(double) * (size_t)K * L * L, rate_bytes = sizeof(double) * (size_t)nT * L * L;
    const double *dsig = sigma;
    double *dsym = sigma_sym, *drate = rate, *dgE = nullptr;
    const bool host_rate = !rate_is_dev(rate), host_sym = sigma_sym && !rate_is_dev(sigma_sym);
    if (!rate_is_dev(sigma)) {
        double *p;
        if ((e = get((void **)&p, sig_bytes)) != cudaSuccess ||
            (e = cudaMemcpyAsync(p, sigma, sig_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "staging sigma");
        }
        dsig = p;
    }
    // degeneracies and level energies, one device buffer [g | E]; pageable copies are staged
    // by the runtime before cudaMemcpyAsync returns
    if ((e = get((void **)&dgE, sizeof(double) * 2 * (size_t)L)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dgE, d->degeneracy, sizeof(double) * L, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dgE + L, d->level_energy, sizeof(double) * L, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "staging levels");
    }
    if (host_rate && (e = get((void **)&drate, rate_bytes)) != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaMallocAsync"); }
    if (host_sym && (e = get((void **)&dsym, sig_bytes)) != cudaSuccess) { cleanup(); return cuda_fail(e, "cudaMallocAsync"); }
    if (dsym) {
        const long long n = (long long)K * L * L;
        const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 16);
        k_rate_sym<<<blocks, 256, 0, st>>>(dsig, dgE, K, L, dsym);
    }
    const long long work = A.n_pairs * nT;
    k_rates<<<(unsigned)((work + 127) / 128), 128, 0, st>>>(A, dsig, dgE, dgE + L, drate);
    count_launches(dsym ? 2 : 1);
    if ((e = cudaGetLastError()) != cudaSuccess) { cleanup(); return cuda_fail(e, "rate kernels"); }
    if (host_rate && (e = cudaMemcpyAsync(rate, drate, rate_bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMemcpyAsync");
    }
    if (host_sym && (e = cudaMemcpyAsync(sigma_sym, dsym, sig_bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaMemcpyAsync");
    }
    cleanup();
    if (host_rate || host_sym) {
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return MQCT_OK;
}
