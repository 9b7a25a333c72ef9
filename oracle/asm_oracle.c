/*
 * asm_oracle.c -- plain FP64 CPU oracle of the average spectrum method with
 * blocked modes sampling (Ghanem & Koch, arXiv:1912.01379).
 *
 * TEST INFRASTRUCTURE ONLY (see asm_oracle.h).  Slow on purpose: every block
 * visit recomputes the data seen by the block from scratch and every move
 * recomputes the mode coordinate by a dot product, exactly as Sec. IV.D counts
 * the work.  No blocking, fusion or incremental bookkeeping.
 *
 * Readings of the paper that this file fixes:
 *  R1 moves draw delta = e' - e from the 1-D conditional with ONE uniform u
 *     through the inverse CDF of the truncated normal (Sec. IV.A cites a
 *     rejection sampler; an inverse CDF samples the same distribution).  The
 *     inverse CDF is evaluated in the form that keeps delta - lo accurate
 *     relative to hi - lo: Gauss-Legendre + Newton on intervals narrower than
 *     the Gaussian's curvature, Phi^{-1} in the centre, log Q in the tails.
 *  R2 zero modes (d = 0, Sec. IV.B) are flat on their interval; singular
 *     values d <= d_1 max(M, n) 2^-52 count as zero, and so do those up to
 *     d_1 max(M, n) 2^-40 whose vector changes sign (R2).
 *  R3 the bounds of Eq. modeLimits are used as delta in [max_{V>0} -f/V,
 *     min_{V<0} -f/V]; entries |V| < 2^-40 max|V| are left out of the bounds;
 *     after the move f is clamped at 0 so A >= 0 holds exactly.
 *  R17 gamma prior prod f_n^(a_n - 1) (Eq. compat, a_n >= 1): each move's
 *     draw from the 1-D conditional of the fit is a proposal, accepted with
 *     probability min(1, prior ratio) by a second uniform (word t mod 4 of
 *     ctr {t/4, s, q, problem xor 2^63}).
 *  R4 sweep order: modes in index order (largest d first) within a block,
 *     blocks left to right; one level per sweep drawn uniformly (Sec. IV.C).
 *  R5 random numbers: Philox4x64-10, key {seed, 0}; move t of sweep s of chain
 *     q of problem p uses word t mod 4 of ctr {t div 4, s, q, p}; the level of
 *     sweep s uses word 0 of ctr {2^64-1, s, 0, p}; u = (w>>12 + 1/2) 2^-52.
 *  R6 sign convention: the largest |component| of every V_j is positive
 *     (lowest index on ties).
 */
#include "asm_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_SQRT2 1.41421356237309504880
#define ORA_SQRT_2_OVER_PI 0.79788456080286535588
#define ORA_INV_SQRT_PI 0.56418958354775628695

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 from its published definition (Salmon et al., SC'11,       */
/* Sec. 4.3): 10 rounds of two 64x64->128 multiplies; the key is bumped by   */
/* the Weyl constants before every round after the first.                   */
/* ------------------------------------------------------------------------ */
void ora_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static double ora_u01(uint64_t w) { return ((double)(w >> 12) + 0.5) * 0x1p-52; }

/* ------------------------------------------------------------------------ */
/* Normal distribution.  erfc comes from the C library; erfcx for x >= 2   */
/* from its continued fraction (Abramowitz & Stegun 7.1.14).               */
/* ------------------------------------------------------------------------ */
double ora_norm_cdf(double z) { return 0.5 * erfc(-z / ORA_SQRT2); }
static double ora_q(double z) { return 0.5 * erfc(z / ORA_SQRT2); }

double ora_erfcx(double x)
{
    if (x < 0.0) return 2.0 * exp(x * x) - ora_erfcx(-x);
    if (x < 2.0) return exp(x * x) * erfc(x);
    /* Laplace continued fraction (Abramowitz & Stegun 7.1.14), evaluated
     * backwards from a fixed depth: 1/(sqrt(pi) (x + (1/2)/(x + 1/(x + ...)))) */
    double t = x;
    for (int k = 120; k >= 1; --k) t = x + 0.5 * k / t;
    return ORA_INV_SQRT_PI / t;
}

double ora_log_q(double x)
{
    /* Q(x) = exp(-x^2/2) erfcx(x/sqrt2) / 2 */
    return log(0.5 * ora_erfcx(x / ORA_SQRT2)) - 0.5 * x * x;
}

/* log Phi(x) and phi(x)/Phi(x) without underflow. */
static double ora_log_phi_cdf(double x)
{
    if (x < 0.0) return log(0.5 * ora_erfcx(-x / ORA_SQRT2)) - 0.5 * x * x;
    return log1p(-ora_q(x));
}
static double ora_mills_inv(double x)
{
    if (x < 0.0) return ORA_SQRT_2_OVER_PI / ora_erfcx(-x / ORA_SQRT2);
    return exp(-0.5 * x * x) / (sqrt(2.0 * M_PI) * ora_norm_cdf(x));
}

/* Phi^{-1}(p): rational start (Abramowitz & Stegun 26.2.23) refined by
 * Newton's method on log Phi(x) = log p, which converges monotonically
 * because log Phi is concave. */
double ora_norm_quantile(double p)
{
    if (!(p > 0.0)) return -INFINITY;
    if (!(p < 1.0)) return INFINITY;
    if (p > 0.5) return -ora_norm_quantile(1.0 - p);
    double t = sqrt(-2.0 * log(p));
    double x = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                     (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
    double lp = log(p);
    for (int it = 0; it < 100; ++it) {
        double g = ora_log_phi_cdf(x) - lp;
        double dx = -g / ora_mills_inv(x);
        x += dx;
        if (fabs(dx) <= 1e-16 * fmax(1.0, fabs(x))) break;
    }
    return x;
}

/* ------------------------------------------------------------------------ */
/* Truncated normal by the inverse CDF (R1): the draw is the root x of       */
/* P(a <= X <= x) = u P(a <= X <= b), X ~ N(0,1), found by a bracketing root */
/* finder on a mass function that keeps its relative accuracy.              */
/* ------------------------------------------------------------------------ */

/* Mass of N(0,1) on [c, c + y] relative to its density at c, for c >= 0 and
 * y >= 0 (y = inf allowed):  E(c, y) = int_0^y exp(-c s - s^2/2) ds.
 * For y (c + y) <= 1: the Taylor series of the Gaussian about c, whose k-th
 * derivative is (-1)^k He_k(c) phi(c) (probabilists' Hermite polynomials,
 * He_0 = 1, He_1 = x, He_{k+1} = x He_k - k He_{k-1}), integrated term by
 * term: E = sum_k (-1)^k He_k(c) y^(k+1) / (k+1)!.
 * Otherwise the difference of two upper tails, Q(c) - Q(c + y), written with
 * Q(x) = phi(x) sqrt(pi/2) erfcx(x/sqrt2): the subtracted term is at most
 * exp(-1/2) of the first one here, so the difference loses no accuracy. */
static double ora_tail_mass(double c, double y)
{
    if (!(y > 0.0)) return 0.0;
    if (isfinite(y) && y * (c + y) <= 1.0) {
        double hm1 = 0.0, h = 1.0;     /* He_{k-1}(c), He_k(c) */
        double pw = y;                 /* y^(k+1) / (k+1)! */
        double sum = 0.0;
        int small = 0;
        for (int k = 0; k < 200; ++k) {
            const double term = ((k & 1) ? -h : h) * pw;
            sum += term;
            if (fabs(term) <= 1e-18 * fabs(sum)) {
                if (++small == 2) break;
            } else {
                small = 0;
            }
            const double hp1 = c * h - k * hm1;
            hm1 = h;
            h = hp1;
            pw *= y / (k + 2);
        }
        return sum;
    }
    const double first = ora_erfcx(c / ORA_SQRT2);
    const double second = isinf(y) ? 0.0 : ora_erfcx((c + y) / ORA_SQRT2) * exp(-y * (c + 0.5 * y));
    return 1.25331413731550025121 * (first - second);   /* sqrt(pi/2) */
}

/* P(z <= X <= c) / phi(0) for 0 <= z <= c (c = inf allowed): decreasing in z. */
static double ora_upper_mass(double z, double c)
{
    return exp(-0.5 * z * z) * ora_tail_mass(z, c - z);
}

/* The doubles in [lo, hi] (0 <= lo < hi) ordered by their bit patterns: the
 * pattern halfway between those of lo and hi.  Halving the pattern interval
 * halves a range of exponents when lo and hi are far apart and the range of
 * values when they are close, so at most 64 such steps separate any two
 * non-negative doubles. */
static double ora_bits_mid(double lo, double hi)
{
    uint64_t a, b;
    memcpy(&a, &lo, 8);
    memcpy(&b, &hi, 8);
    uint64_t m = a + (b - a) / 2;
    double r;
    memcpy(&r, &m, 8);
    return r;
}

/* Root of g(y) = F(y) - target on [lo, hi], 0 <= lo < hi finite, for F
 * monotone with g(lo) and g(hi) of opposite signs (or zero): regula falsi
 * with the Illinois modification (Dowell and Jarratt, BIT 11 (1971) 168),
 * which keeps the root bracketed, and a step of ora_bits_mid whenever a false-
 * position step leaves more than half of the bracket.  Stops when the bracket
 * holds no double between its ends; returns the end where g has the sign of
 * g(hi).  *capped counts solves that hit the iteration cap. */
typedef double (*ora_mass_fn)(double y, const double *par);

static double ora_bracket_root(ora_mass_fn F, const double *par, double target, double lo, double hi,
                               int *capped)
{
    double glo = F(lo, par) - target, ghi = F(hi, par) - target;
    if (glo == 0.0) return lo;
    if (ghi == 0.0 || (glo > 0.0) == (ghi > 0.0)) return hi;
    const int hi_positive = ghi > 0.0;
    int side = 0, it;
    for (it = 0; it < 400; ++it) {
        if (ora_bits_mid(lo, hi) == lo) break;   /* adjacent doubles */
        double y = hi - ghi * (hi - lo) / (ghi - glo);
        if (!(y > lo && y < hi)) y = ora_bits_mid(lo, hi);
        const double width = hi - lo;
        const double gy = F(y, par) - target;
        if (gy == 0.0) return y;
        if ((gy > 0.0) == hi_positive) {
            hi = y; ghi = gy;
            if (side == -1) glo *= 0.5;   /* Illinois: the end kept twice has its value halved */
            side = -1;
        } else {
            lo = y; glo = gy;
            if (side == 1) ghi *= 0.5;
            side = 1;
        }
        if (hi - lo > 0.5 * width) {      /* slow progress: a bisection step of the bit patterns */
            const double m = ora_bits_mid(lo, hi);
            if (m == lo) break;
            const double gm = F(m, par) - target;
            if (gm == 0.0) return m;
            if ((gm > 0.0) == hi_positive) { hi = m; ghi = gm; }
            else { lo = m; glo = gm; }
            side = 0;
        }
    }
    if (it == 400 && capped) ++*capped;
    return hi;
}

static double ora_tail_mass_fn(double y, const double *par) { return ora_tail_mass(par[0], y); }
static double ora_upper_mass_fn(double z, const double *par) { return ora_upper_mass(z, par[0]); }
/* P(c + y <= X <= c + w) / phi(c): the mass above the offset y, decreasing in y */
static double ora_rest_mass_fn(double y, const double *par)
{
    const double c = par[0], w = par[1];
    return exp(-y * (c + 0.5 * y)) * ora_tail_mass(c + y, w - y);
}

/* Upper end of a bracket [0, y] for an offset on [c, inf): doubling from the
 * scale of the density's decay until F passes the target (F increasing) or
 * drops below it (F decreasing). */
static double ora_tail_bracket(ora_mass_fn F, const double *par, double target, int increasing)
{
    double y = 1.0 / (par[0] + 1.0);
    for (int k = 0; k < 2100; ++k, y *= 2.0) {
        const double v = F(y, par);
        if (increasing ? v >= target : v <= target) break;
    }
    return y;
}

/* delta ~ N(mu, sigma^2) restricted to [lo, hi] (lo < hi) by the inverse CDF
 * at u.  In standard units the interval is [a, b] = [(lo-mu)/sigma,
 * (hi-mu)/sigma].  The root is always sought from the side whose share of the
 * mass is the smaller one (u or 1 - u), so that the function solved is steep
 * where the root lies:
 *  - a >= 0: the offset y = x - a from the lower end solves E(a, y) = u Z
 *    (u <= 1/2) or P(a + y <= X <= b) / phi(a) = (1 - u) Z (u > 1/2), with
 *    Z = E(a, b - a); delta = lo + sigma y.
 *  - b <= 0: the mirror image, measured down from hi with 1 - u (exact: u lies
 *    on the 2^-52 grid).
 *  - a < 0 < b: the mass left of 0 is sqrt(pi/2) erf(|a|/sqrt2).  A root left
 *    of 0 is x = -z with P(z <= -X <= |a|) = u P(a <= X <= b); a root right of
 *    0 is x = z with P(z <= X <= b) = (1 - u) P(a <= X <= b).  Both keep z
 *    accurate near 0 and near the end it is measured from.
 * Any root of the straddling case lies within 40 of 0 (the targets are at
 * least 2^-53 of a mass of order one there), which bounds the brackets. */
static double ora_truncnorm_impl(double mu, double sigma, double lo, double hi, double u,
                                 int *capped)
{
    if (!(hi > lo)) return lo;
    const double a = (lo - mu) / sigma, b = (hi - mu) / sigma;
    double d;
    if (a >= 0.0 || b <= 0.0) {
        const int mirror = a < 0.0;
        const double c = mirror ? -b : a;
        const double w = (hi - lo) / sigma;
        const double uu = mirror ? 1.0 - u : u;
        const double par[2] = {c, w};
        const double Z = ora_tail_mass(c, w);
        double y;
        if (uu <= 0.5) {
            const double top = isfinite(w) ? w : ora_tail_bracket(ora_tail_mass_fn, par, uu * Z, 1);
            y = ora_bracket_root(ora_tail_mass_fn, par, uu * Z, 0.0, top, capped);
        } else {
            const double top = isfinite(w) ? w : ora_tail_bracket(ora_rest_mass_fn, par, (1.0 - uu) * Z, 0);
            y = ora_bracket_root(ora_rest_mass_fn, par, (1.0 - uu) * Z, 0.0, top, capped);
        }
        d = mirror ? hi - sigma * y : lo + sigma * y;
    } else {
        const double mass_left = 1.25331413731550025121 * erf(-a / ORA_SQRT2);
        const double mass_right = 1.25331413731550025121 * erf(b / ORA_SQRT2);
        const double total = mass_left + mass_right;
        double x;
        if (u * total <= mass_left) {
            const double par[1] = {-a};
            x = -ora_bracket_root(ora_upper_mass_fn, par, u * total, 0.0, fmin(-a, 40.0), capped);
        } else {
            const double par[1] = {b};
            x = ora_bracket_root(ora_upper_mass_fn, par, (1.0 - u) * total, 0.0, fmin(b, 40.0), capped);
        }
        d = mu + sigma * x;
    }
    if (d < lo) d = lo;
    if (d > hi) d = hi;
    return d;
}

double ora_truncnorm(double mu, double sigma, double lo, double hi, double u)
{
    return ora_truncnorm_impl(mu, sigma, lo, hi, u, &(int){0});
}

/* ------------------------------------------------------------------------ */
/* Robert's rejection sampler (C. P. Robert, "Simulation of truncated normal */
/* variables", Statistics and Computing 5 (1995) 121-125): an independent   */
/* route to the same distribution, used only to cross-check the inverse CDF */
/* above in distribution.  Uniforms come from Philox4x64-10 with key        */
/* {seed, 0x526f62657274} and counter {k/4, stream, 0, 0}.                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t key[2], stream, k, w[4];
} ora_ustream;

static double ora_next_u(ora_ustream *s)
{
    if ((s->k & 3) == 0) {
        const uint64_t ctr[4] = {s->k >> 2, s->stream, 0, 0};
        ora_philox4x64_10(ctr, s->key, s->w);
    }
    return ora_u01(s->w[s->k++ & 3]);
}

/* One draw of X ~ N(0,1) restricted to [a, b] (a < b, either may be infinite).
 * Proposals (Robert 1995, Sec. 2): for a >= 0, the exponential translated to a
 * with the optimal rate l = (a + sqrt(a^2 + 4))/2, accepted with probability
 * exp(-(z - l)^2/2) and rejected beyond b, unless the interval is short
 * enough that the uniform proposal on [a, b] (accepted with probability
 * exp((a^2 - z^2)/2)) is the better one; for a < 0 < b, the uniform proposal
 * (accepted with exp(-z^2/2)) on intervals shorter than sqrt(2 pi), else
 * N(0,1) itself by Box-Muller, rejected outside [a, b]; b <= 0 by symmetry. */
static double ora_robert_draw(double a, double b, ora_ustream *s, long *tries)
{
    if (b <= 0.0) return -ora_robert_draw(-b, -a, s, tries);
    for (;;) {
        ++*tries;
        if (a >= 0.0) {
            const double r = sqrt(a * a + 4.0);
            const double l = 0.5 * (a + r);
            const double b_switch = a + 2.0 / (a + r) * exp(0.25 * (a * a - a * r) + 0.5);
            if (b <= b_switch) {
                const double z = a + (b - a) * ora_next_u(s);
                if (ora_next_u(s) <= exp(0.5 * (a - z) * (a + z))) return z;
            } else {
                const double z = a - log(ora_next_u(s)) / l;
                const double acc = exp(-0.5 * (z - l) * (z - l));
                if (ora_next_u(s) <= acc && z <= b) return z;
            }
        } else if (b - a < 2.50662827463100050242) {   /* sqrt(2 pi) */
            const double z = a + (b - a) * ora_next_u(s);
            if (ora_next_u(s) <= exp(-0.5 * z * z)) return z;
        } else {
            const double u1 = ora_next_u(s), u2 = ora_next_u(s);
            const double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
            if (z >= a && z <= b) return z;
        }
    }
}

long ora_truncnorm_robert(double a, double b, uint64_t seed, uint64_t stream, int n, double *out)
{
    ora_ustream s = {{seed, 0x526f62657274ULL}, stream, 0, {0, 0, 0, 0}};
    long tries = 0;
    for (int i = 0; i < n; ++i) out[i] = ora_robert_draw(a, b, &s, &tries);
    return tries;
}

/* ------------------------------------------------------------------------ */
/* Linear algebra                                                           */
/* ------------------------------------------------------------------------ */
int ora_cholesky(int n, const double *C, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j) {
        double s = C[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return -2;
        double ljj = sqrt(s);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = C[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / ljj;
        }
    }
    return 0;
}

/* One-sided (Hestenes) Jacobi: rotate column pairs of W = A until all pairs
 * are orthogonal; then s_j = |W_j|, U_j = W_j / s_j and V collects the
 * rotations.  For n > m the n - m surplus columns converge to zero and V
 * still is a full orthogonal basis, which gives the zero modes of Sec. IV.B. */
int ora_jacobi_svd(int m, int n, const double *A, double *s, double *U, double *V)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)m * n);  /* column-major */
    double *Z = (double *)malloc(sizeof(double) * (size_t)n * n);  /* column-major */
    if (!W || !Z) { free(W); free(Z); return -1; }
    double norm2 = 0.0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            W[(size_t)j * m + i] = A[(size_t)i * n + j];
            norm2 += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Z[(size_t)j * n + i] = (i == j) ? 1.0 : 0.0;
    int sweep, converged = 0;
    for (sweep = 1; sweep <= 80 && !converged; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double *wp = W + (size_t)p * m, *wq = W + (size_t)q * m;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < m; ++i) {
                    al += wp[i] * wp[i];
                    be += wq[i] * wq[i];
                    ga += wp[i] * wq[i];
                }
                if (fabs(ga) <= 1e-15 * sqrt(al * be) || fabs(ga) <= 1e-30 * norm2) continue;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                for (int i = 0; i < m; ++i) {
                    double a = wp[i], b = wq[i];
                    wp[i] = c * a - sn * b;
                    wq[i] = sn * a + c * b;
                }
                double *zp = Z + (size_t)p * n, *zq = Z + (size_t)q * n;
                for (int i = 0; i < n; ++i) {
                    double a = zp[i], b = zq[i];
                    zp[i] = c * a - sn * b;
                    zq[i] = sn * a + c * b;
                }
                rotated = 1;
            }
        if (!rotated) converged = 1;
    }
    /* column norms, then sort descending (selection sort: n is small) */
    int *ord = (int *)malloc(sizeof(int) * n);
    double *sv = (double *)malloc(sizeof(double) * n);
    for (int j = 0; j < n; ++j) {
        double t = 0.0;
        for (int i = 0; i < m; ++i) t += W[(size_t)j * m + i] * W[(size_t)j * m + i];
        sv[j] = sqrt(t);
        ord[j] = j;
    }
    for (int a = 0; a < n; ++a) {
        int best = a;
        for (int b = a + 1; b < n; ++b)
            if (sv[ord[b]] > sv[ord[best]]) best = b;
        int tmp = ord[a]; ord[a] = ord[best]; ord[best] = tmp;
    }
    for (int a = 0; a < n; ++a) {
        int j = ord[a];
        double *z = Z + (size_t)j * n, *w = W + (size_t)j * m;
        /* sign convention R6 */
        int imax = 0;
        for (int i = 1; i < n; ++i)
            if (fabs(z[i]) > fabs(z[imax])) imax = i;
        double sg = z[imax] < 0.0 ? -1.0 : 1.0;
        s[a] = sv[j];
        for (int i = 0; i < n; ++i) V[(size_t)i * n + a] = sg * z[i];
        for (int i = 0; i < m; ++i) U[(size_t)i * n + a] = sv[j] > 0.0 ? sg * w[i] / sv[j] : 0.0;
    }
    free(ord); free(sv); free(W); free(Z);
    return converged ? sweep - 1 : -2;
}

/* ------------------------------------------------------------------------ */
/* Problem set-up: whitening (Sec. IV, C^{-1} = T^T T with T = L^{-1}) and   */
/* the SVD of every block of every level (Sec. IV.B-C).                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int start, n, np;    /* first column, width, number of U columns min(M, n) */
    double *d;           /* n singular values, 0 for zero modes (R2) */
    double *V;           /* n x n mode-major */
    double *U;           /* np x M mode-major */
} ora_block;

struct ora_problem {
    int M, N, n_levels;
    int *level_nblocks, *level_first;
    int n_blocks;
    ora_block *blk;
    double *Kt, *gt;     /* whitened kernel (M x N row-major) and data */
    double *prior_am1;   /* a_n - 1 of the gamma prior prod f_n^(a_n - 1) (Eq. compat), NULL: flat */
    int flat_exp;        /* R2: sign-changing modes with d <= d_1 max(M,n) 2^-flat_exp are flat */
    int jitter;          /* test of rounding sensitivity: 0 off, else every conditional mean and
                          * interval end moved by one rounding at unit roundoff 2^-jitter */
    int jitter_shift;    /* the directions come from bits jitter_shift + 1..3 of the move's word */
};

void ora_free(ora_problem *p)
{
    if (!p) return;
    for (int b = 0; b < p->n_blocks; ++b) {
        free(p->blk[b].d); free(p->blk[b].V); free(p->blk[b].U);
    }
    free(p->blk); free(p->level_nblocks); free(p->level_first);
    free(p->Kt); free(p->gt); free(p->prior_am1);
    free(p);
}

static int ora_block_svd(const ora_problem *p, ora_block *b)
{
    int M = p->M, n = b->n;
    double *A = (double *)malloc(sizeof(double) * (size_t)M * n);
    double *s = (double *)malloc(sizeof(double) * n);
    double *U = (double *)malloc(sizeof(double) * (size_t)M * n);
    double *V = (double *)malloc(sizeof(double) * (size_t)n * n);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = p->Kt[(size_t)i * p->N + b->start + j];
    int rc = ora_jacobi_svd(M, n, A, s, U, V);
    if (rc < 0) { free(A); free(s); free(U); free(V); return -1; }
    b->np = M < n ? M : n;
    b->d = (double *)calloc(n, sizeof(double));
    b->V = (double *)malloc(sizeof(double) * (size_t)n * n);
    b->U = (double *)calloc((size_t)b->np * M, sizeof(double));
    /* R2 zero modes.  d <= d_1 max(M,n) 2^-52 is numerically zero.  Up to
     * d_1 max(M,n) 2^-40 the left vector U_j = K~ V_j / d_j cannot be formed
     * in FP64 to better than about 2^-52 d_1 / d_j, which moves the
     * conditional mean by a visible fraction of its width, while the
     * likelihood varies by only exp(-(d Delta)^2/2) ~ 1 over the positivity
     * interval Delta: such a mode is sampled flat when its vector changes sign
     * (so that the interval is finite) and keeps its Gaussian otherwise. */
    const double dmax = (double)(M > n ? M : n);
    const double thr0 = s[0] * dmax * 0x1p-52, thr = s[0] * dmax * ldexp(1.0, -p->flat_exp);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) b->V[(size_t)j * n + i] = V[(size_t)i * n + j];
    for (int j = 0; j < n; ++j) {
        const double *v = b->V + (size_t)j * n;
        double vmax = 0.0;
        for (int i = 0; i < n; ++i) vmax = fmax(vmax, fabs(v[i]));
        int pos = 0, neg = 0;
        for (int i = 0; i < n; ++i) {
            if (fabs(v[i]) < 0x1p-40 * vmax) continue;
            if (v[i] > 0.0) pos = 1;
            if (v[i] < 0.0) neg = 1;
        }
        const double sj = j < b->np ? s[j] : 0.0;
        const int zero = sj <= thr0 || (sj <= thr && pos && neg);
        if (zero && !(pos && neg)) { free(A); free(s); free(U); free(V); return -4; }   /* improper */
        b->d[j] = zero ? 0.0 : sj;
        if (!zero)
            for (int m = 0; m < M; ++m) b->U[(size_t)j * M + m] = U[(size_t)m * n + j];
    }
    free(A); free(s); free(U); free(V);
    return 0;
}

ora_problem *ora_setup_ex(int M, int N, const double *K, const double *G, const double *C,
                          int n_levels, const int *level_nblocks, const int *block_start, int flat_exp,
                          int *err)
{
    *err = 0;
    if (M < 1 || N < 1 || n_levels < 1 || flat_exp < 1 || flat_exp > 52) { *err = -1; return NULL; }
    for (long i = 0; i < (long)M * N; ++i) if (!isfinite(K[i])) { *err = -3; return NULL; }
    for (int i = 0; i < M; ++i) if (!isfinite(G[i])) { *err = -3; return NULL; }
    for (long i = 0; i < (long)M * M; ++i) if (!isfinite(C[i])) { *err = -3; return NULL; }
    ora_problem *p = (ora_problem *)calloc(1, sizeof(ora_problem));
    p->M = M; p->N = N; p->n_levels = n_levels;
    p->flat_exp = flat_exp;
    p->level_nblocks = (int *)malloc(sizeof(int) * n_levels);
    p->level_first = (int *)malloc(sizeof(int) * n_levels);
    int nb = 0;
    for (int l = 0; l < n_levels; ++l) {
        if (level_nblocks[l] < 1) { *err = -1; ora_free(p); return NULL; }
        p->level_nblocks[l] = level_nblocks[l];
        p->level_first[l] = nb;
        nb += level_nblocks[l];
    }
    p->n_blocks = nb;
    p->blk = (ora_block *)calloc(nb, sizeof(ora_block));
    for (int l = 0; l < n_levels; ++l) {
        const int *st = block_start + p->level_first[l];
        for (int b = 0; b < level_nblocks[l]; ++b) {
            int s0 = st[b], s1 = (b + 1 < level_nblocks[l]) ? st[b + 1] : N;
            if ((b == 0 && s0 != 0) || s1 <= s0 || s1 > N) { *err = -1; ora_free(p); return NULL; }
            p->blk[p->level_first[l] + b].start = s0;
            p->blk[p->level_first[l] + b].n = s1 - s0;
        }
    }
    /* whitening: C = L L^T, T = L^{-1}, K~ = T K, g~ = T G (forward substitution) */
    double *L = (double *)malloc(sizeof(double) * (size_t)M * M);
    if (ora_cholesky(M, C, L) != 0) { free(L); *err = -2; ora_free(p); return NULL; }
    p->Kt = (double *)malloc(sizeof(double) * (size_t)M * N);
    p->gt = (double *)malloc(sizeof(double) * M);
    for (int i = 0; i < M; ++i) {
        for (int j = 0; j < N; ++j) {
            double t = K[(size_t)i * N + j];
            for (int k = 0; k < i; ++k) t -= L[(size_t)i * M + k] * p->Kt[(size_t)k * N + j];
            p->Kt[(size_t)i * N + j] = t / L[(size_t)i * M + i];
        }
        double t = G[i];
        for (int k = 0; k < i; ++k) t -= L[(size_t)i * M + k] * p->gt[k];
        p->gt[i] = t / L[(size_t)i * M + i];
    }
    free(L);
    for (int b = 0; b < nb; ++b) {
        int rc = ora_block_svd(p, &p->blk[b]);
        if (rc != 0) { *err = rc == -4 ? -4 : -1; ora_free(p); return NULL; }
    }
    return p;
}

ora_problem *ora_setup(int M, int N, const double *K, const double *G, const double *C,
                       int n_levels, const int *level_nblocks, const int *block_start, int *err)
{
    return ora_setup_ex(M, N, K, G, C, n_levels, level_nblocks, block_start, 40, err);
}

void ora_set_jitter(ora_problem *p, int unit_exp, int pattern)
{
    p->jitter = (unit_exp >= 1 && unit_exp <= 60) ? unit_exp : 0;
    p->jitter_shift = (pattern >= 0 && pattern < 16) ? 3 * pattern : 0;
}

void ora_sizes(const ora_problem *p, long *n_d, long *n_V, long *n_U)
{
    long a = 0, b = 0, c = 0;
    for (int k = 0; k < p->n_blocks; ++k) {
        a += p->blk[k].n;
        b += (long)p->blk[k].n * p->blk[k].n;
        c += (long)p->blk[k].np * p->M;
    }
    *n_d = a; *n_V = b; *n_U = c;
}

void ora_export(const ora_problem *p, double *Kt, double *gt, double *d, double *V, double *U)
{
    memcpy(Kt, p->Kt, sizeof(double) * (size_t)p->M * p->N);
    memcpy(gt, p->gt, sizeof(double) * p->M);
    for (int k = 0; k < p->n_blocks; ++k) {
        const ora_block *b = &p->blk[k];
        memcpy(d, b->d, sizeof(double) * b->n); d += b->n;
        memcpy(V, b->V, sizeof(double) * (size_t)b->n * b->n); V += (size_t)b->n * b->n;
        memcpy(U, b->U, sizeof(double) * (size_t)b->np * p->M); U += (size_t)b->np * p->M;
    }
}

void ora_initial_f(const ora_problem *p, double *f0)
{
    /* s* = argmin_{s >= 0} | g~ - s K~ 1 |^2 */
    double num = 0.0, den = 0.0;
    for (int i = 0; i < p->M; ++i) {
        double k = 0.0;
        for (int j = 0; j < p->N; ++j) k += p->Kt[(size_t)i * p->N + j];
        num += k * p->gt[i];
        den += k * k;
    }
    double s = den > 0.0 ? num / den : 0.0;
    if (!(s > 0.0) || !isfinite(s)) s = 1.0 / p->N;
    for (int j = 0; j < p->N; ++j) f0[j] = s;
}

double ora_chi2(const ora_problem *p, const double *f)
{
    double c = 0.0;
    for (int i = 0; i < p->M; ++i) {
        double r = p->gt[i];
        for (int j = 0; j < p->N; ++j) r -= p->Kt[(size_t)i * p->N + j] * f[j];
        c += r * r;
    }
    return c;
}

/* Data seen by block b: h_b = U_b^T (g~ - sum_{blocks b' != b} K~_{b'} f_{b'})
 * (Sec. IV.D: the contribution of the other blocks).  habs (may be NULL)
 * receives sum_m |U_jm| (|g~_m| + sum_{n not in b} |K~_mn f_n|), the size of
 * the terms whose roundings h_j carries. */
static void ora_block_h(const ora_problem *p, const ora_block *b, const double *f, double *gp,
                        double *h, double *habs)
{
    double *gabs = habs ? (double *)malloc(sizeof(double) * p->M) : NULL;
    for (int i = 0; i < p->M; ++i) {
        double t = p->gt[i], ta = fabs(p->gt[i]);
        for (int j = 0; j < p->N; ++j) {
            if (j >= b->start && j < b->start + b->n) continue;
            t -= p->Kt[(size_t)i * p->N + j] * f[j];
            ta += fabs(p->Kt[(size_t)i * p->N + j] * f[j]);
        }
        gp[i] = t;
        if (gabs) gabs[i] = ta;
    }
    for (int j = 0; j < b->np; ++j) {
        double t = 0.0, ta = 0.0;
        for (int i = 0; i < p->M; ++i) {
            t += b->U[(size_t)j * p->M + i] * gp[i];
            if (gabs) ta += fabs(b->U[(size_t)j * p->M + i]) * gabs[i];
        }
        h[j] = t;
        if (habs) habs[j] = ta;
    }
    free(gabs);
}

/* Interval of delta = e_j' - e_j that keeps f + delta V_j >= 0 (Eq. modeLimits, R3). */
static void ora_bounds(const ora_block *b, int j, const double *f, double *lo, double *hi)
{
    const double *v = b->V + (size_t)j * b->n;
    const double *fb = f + b->start;
    double vmax = 0.0;
    for (int i = 0; i < b->n; ++i) vmax = fmax(vmax, fabs(v[i]));
    double l = -INFINITY, h = INFINITY;
    for (int i = 0; i < b->n; ++i) {
        if (fabs(v[i]) < 0x1p-40 * vmax) continue;
        double fi = fb[i] > 0.0 ? fb[i] : 0.0;
        double t = -fi / v[i];
        if (v[i] > 0.0) { if (t > l) l = t; }
        else { if (t < h) h = t; }
    }
    *lo = l; *hi = h;
}

/* Conditional of mode j of block b given the rest (Sec. IV.B-C):
 * e_j' ~ N(h_j/d_j, 1/d_j^2), so delta ~ N(h_j/d_j - e_j, 1/d_j^2). */
static void ora_mode_conditional(const ora_block *b, int j, const double *f, const double *h,
                                 const double *habs, double *mu, double *sigma, double *mu_scale)
{
    const double *v = b->V + (size_t)j * b->n;
    double e = 0.0, ea = 0.0;
    for (int i = 0; i < b->n; ++i) {
        e += v[i] * f[b->start + i];
        ea += fabs(v[i] * f[b->start + i]);
    }
    if (b->d[j] > 0.0) {
        *mu = h[j] / b->d[j] - e;
        *sigma = 1.0 / b->d[j];
        /* the size of every term rounded on the way to mu */
        if (mu_scale) *mu_scale = (habs ? habs[j] : fabs(h[j])) / b->d[j] + ea;
    } else {
        *mu = 0.0;
        *sigma = 0.0;
        if (mu_scale) *mu_scale = 0.0;
    }
}

int ora_conditional(const ora_problem *p, int level, int block, int j, const double *f,
                    double *mu, double *sigma, double *lo, double *hi)
{
    if (level < 0 || level >= p->n_levels || block < 0 || block >= p->level_nblocks[level]) return -1;
    const ora_block *b = &p->blk[p->level_first[level] + block];
    if (j < 0 || j >= b->n) return -1;
    double *gp = (double *)malloc(sizeof(double) * p->M);
    double *h = (double *)malloc(sizeof(double) * (b->np > 0 ? b->np : 1));
    ora_block_h(p, b, f, gp, h, NULL);
    ora_mode_conditional(b, j, f, h, NULL, mu, sigma, NULL);
    ora_bounds(b, j, f, lo, hi);
    free(gp); free(h);
    return 0;
}

/* Prior prod_n f_n^(a_n - 1) of Eq. compat (Sec. V.C, simulating one grid on
 * another); a_n >= 1 (shape NULL or all 1: flat).  Returns -1 for a shape below 1
 * or not finite. */
int ora_set_prior(ora_problem *p, const double *shape)
{
    free(p->prior_am1);
    p->prior_am1 = NULL;
    if (!shape) return 0;
    int any = 0;
    for (int n = 0; n < p->N; ++n) {
        if (!(shape[n] >= 1.0) || !isfinite(shape[n])) return -1;
        if (shape[n] != 1.0) any = 1;
    }
    if (!any) return 0;
    p->prior_am1 = (double *)malloc(sizeof(double) * p->N);
    for (int n = 0; n < p->N; ++n) p->prior_am1[n] = shape[n] - 1.0;
    return 0;
}

/* Log of the prior ratio prod ((f + delta v)_+ / f)^(a - 1) over a block
 * (R17): -inf if a proposed value is exactly 0 where a > 1 (density 0), +inf if
 * a current value is exactly 0 there (and no proposed one is), else the sum. */
static double ora_prior_logratio(const ora_problem *p, const ora_block *b, const double *v, const double *f,
                                 double delta)
{
    int zero_new = 0, zero_old = 0;
    double sum = 0.0;
    for (int i = 0; i < b->n; ++i) {
        const double am1 = p->prior_am1[b->start + i];
        if (am1 == 0.0) continue;
        const double x0 = f[b->start + i];
        double x1 = x0 + delta * v[i];
        if (!(x1 > 0.0)) x1 = 0.0;
        if (x1 == 0.0) zero_new = 1;
        else if (x0 == 0.0) zero_old = 1;
        else sum += am1 * (log(x1) - log(x0));
    }
    if (zero_new) return -INFINITY;
    if (zero_old) return INFINITY;
    return sum;
}

static void ora_chain(const ora_problem *p, uint64_t q, double *f, long sweep0, long burn_in,
                      long sweeps, uint64_t seed, uint64_t problem_id, double *S1, double *S2,
                      double *trace, long *stats)
{
    int M = p->M, N = p->N;
    double *gp = (double *)malloc(sizeof(double) * M);
    double *h = (double *)malloc(sizeof(double) * (M > 0 ? M : 1));
    double *habs = p->jitter ? (double *)malloc(sizeof(double) * (M > 0 ? M : 1)) : NULL;
    const uint64_t key[2] = {seed, 0};
    long viol = 0, degen = 0, flat = 0;
    int capped = 0;
    for (long s = sweep0; s < sweep0 + burn_in + sweeps; ++s) {
        uint64_t w[4];
        uint64_t lc[4] = {~(uint64_t)0, (uint64_t)s, 0, problem_id};
        ora_philox4x64_10(lc, key, w);
        int level = (int)(ora_u01(w[0]) * p->n_levels);
        if (level >= p->n_levels) level = p->n_levels - 1;
        for (int bi = 0; bi < p->level_nblocks[level]; ++bi) {
            const ora_block *b = &p->blk[p->level_first[level] + bi];
            ora_block_h(p, b, f, gp, h, habs);
            for (int j = 0; j < b->n; ++j) {
                long t = b->start + j;
                uint64_t ctr[4] = {(uint64_t)t >> 2, (uint64_t)s, (uint64_t)q, problem_id};
                ora_philox4x64_10(ctr, key, w);
                double u = ora_u01(w[t & 3]);
                double mu, sigma, lo, hi, delta, mu_scale;
                ora_mode_conditional(b, j, f, h, habs, &mu, &sigma, &mu_scale);
                ora_bounds(b, j, f, &lo, &hi);
                if (p->jitter) {   /* one rounding each, up or down by three bits of the move's word */
                    const double ulp = ldexp(1.0, -p->jitter);
                    const uint64_t bits = w[t & 3] >> p->jitter_shift;
                    if (sigma > 0.0) mu += ((bits & 2) ? 1.0 : -1.0) * ulp * mu_scale;
                    if (isfinite(lo)) lo += ((bits & 4) ? 1.0 : -1.0) * ulp * fabs(lo);
                    if (isfinite(hi)) hi += ((bits & 8) ? 1.0 : -1.0) * ulp * fabs(hi);
                }
                if (!(hi > lo)) {
                    delta = 0.0;
                    ++degen;
                } else if (sigma == 0.0) {
                    delta = lo + u * (hi - lo);
                    ++flat;
                } else {
                    delta = ora_truncnorm_impl(mu, sigma, lo, hi, u, &capped);
                }
                const double *v = b->V + (size_t)j * b->n;
                if (p->prior_am1 && delta != 0.0) {
                    /* Metropolis-Hastings on the gamma prior (R17): the 1-D conditional of
                     * the fit is the proposal; accept with prob. min(1, prior ratio),
                     * uniform: word t mod 4 of ctr {t/4, s, q, problem xor 2^63} */
                    const double lr = ora_prior_logratio(p, b, v, f, delta);
                    uint64_t wa[4];
                    uint64_t ca[4] = {(uint64_t)t >> 2, (uint64_t)s, (uint64_t)q, problem_id ^ ((uint64_t)1 << 63)};
                    ora_philox4x64_10(ca, key, wa);
                    const double ua = ora_u01(wa[t & 3]);
                    if (!(log(ua) < lr)) delta = 0.0;
                }
                for (int i = 0; i < b->n; ++i) {
                    double x = f[b->start + i] + delta * v[i];
                    if (x < -1e-12 * (fabs(f[b->start + i]) + 1e-300)) ++viol;
                    f[b->start + i] = x > 0.0 ? x : 0.0;
                }
            }
        }
        long k = s - sweep0;
        if (k >= burn_in && S1) {
            for (int j = 0; j < N; ++j) {
                S1[j] += f[j];
                S2[j] += f[j] * f[j];
            }
        }
        if (trace) memcpy(trace + (size_t)k * N, f, sizeof(double) * N);
    }
    if (stats) {
        stats[0] = viol; stats[1] = degen; stats[2] = flat; stats[3] = capped;
    }
    free(gp); free(h); free(habs);
}

int ora_run_ids(const ora_problem *p, int chains, const double *f_start, long sweep0,
                long burn_in, long sweeps, uint64_t seed, uint64_t problem_id, uint64_t chain0,
                int n_threads, double *f_final, double *S1, double *S2, double *chi2_final,
                double *trace, int n_traced, long *stats)
{
    int N = p->N;
    long tot[4] = {0, 0, 0, 0};
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        long loc[4] = {0, 0, 0, 0};
        double *f = (double *)malloc(sizeof(double) * N);
        double *s1 = (double *)malloc(sizeof(double) * N);
        double *s2 = (double *)malloc(sizeof(double) * N);
#pragma omp for schedule(dynamic, 1)
        for (int q = 0; q < chains; ++q) {
            long st[4] = {0, 0, 0, 0};
            memcpy(f, f_start + (size_t)q * N, sizeof(double) * N);
            memset(s1, 0, sizeof(double) * N);
            memset(s2, 0, sizeof(double) * N);
            double *tr = (trace && q < n_traced) ? trace + (size_t)q * (burn_in + sweeps) * N : NULL;
            ora_chain(p, chain0 + (uint64_t)q, f, sweep0, burn_in, sweeps, seed, problem_id, s1, s2, tr, st);
            if (f_final) memcpy(f_final + (size_t)q * N, f, sizeof(double) * N);
            if (S1) memcpy(S1 + (size_t)q * N, s1, sizeof(double) * N);
            if (S2) memcpy(S2 + (size_t)q * N, s2, sizeof(double) * N);
            if (chi2_final) chi2_final[q] = ora_chi2(p, f);
            for (int k = 0; k < 4; ++k) loc[k] += st[k];
        }
#pragma omp critical
        for (int k = 0; k < 4; ++k) tot[k] += loc[k];
        free(f); free(s1); free(s2);
    }
    if (stats) for (int k = 0; k < 4; ++k) stats[k] = tot[k];
    return 0;
}

int ora_run_from(const ora_problem *p, int chains, const double *f_start, long sweep0,
                 long burn_in, long sweeps, uint64_t seed, uint64_t problem_id, int n_threads,
                 double *f_final, double *S1, double *S2, double *chi2_final,
                 double *trace, int n_traced, long *stats)
{
    return ora_run_ids(p, chains, f_start, sweep0, burn_in, sweeps, seed, problem_id, 0, n_threads,
                       f_final, S1, S2, chi2_final, trace, n_traced, stats);
}

int ora_run(const ora_problem *p, int chains, long burn_in, long sweeps, uint64_t seed,
            uint64_t problem_id, int n_threads, double *f_final, double *S1, double *S2,
            double *chi2_final, double *trace, int n_traced, long *stats)
{
    double *f0 = (double *)malloc(sizeof(double) * (size_t)chains * p->N);
    ora_initial_f(p, f0);
    for (int q = 1; q < chains; ++q) memcpy(f0 + (size_t)q * p->N, f0, sizeof(double) * p->N);
    int rc = ora_run_from(p, chains, f0, 0, burn_in, sweeps, seed, problem_id, n_threads,
                          f_final, S1, S2, chi2_final, trace, n_traced, stats);
    free(f0);
    return rc;
}
