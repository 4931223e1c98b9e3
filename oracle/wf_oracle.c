/*
 * Oracle for the messenger-field Wiener filter: CPU, FP64, deliberately plain.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA library.
 *
 * What it computes (Elsner & Wandelt 2013, "Efficient Wiener filtering
 * without preconditioning"):
 *   - the HEALPix RING pixelisation on which the paper's CMB maps live
 *     (Sect. 3; geometry from Gorski et al. 2005, which the paper cites);
 *   - the normalised associated Legendre functions lambda_lm(cos theta),
 *     from the textbook three-term recurrence, FP64, with an explicit binary
 *     exponent carried for the sin^m(theta) seed so nothing underflows;
 *   - spherical-harmonic synthesis (the basis change of Sect. 2.1) and its
 *     adjoint, by a direct Legendre sum per ring followed by a direct
 *     (naive) Fourier sum over the pixels of the ring.  No FFT, no folding,
 *     no ring-pair symmetry, no cut-offs: every term of the definition is
 *     evaluated.
 *
 * Conventions (the same ones the library documents):
 *   Y_lm(theta, phi) = lambda_lm(cos theta) e^{i m phi}, Condon-Shortley
 *   phase included, orthonormal on the sphere.  a_lm is stored for m >= 0
 *   only, m-major: index(l, m) = m(2 lmax + 3 - m)/2 + (l - m), complex
 *   interleaved (re, im).  A real map is f = sum_l [a_l0 Y_l0 + 2 Re sum_{m>0}
 *   a_lm Y_lm].  The adjoint of that synthesis is
 *   (Y^T f)_lm = sum_p f_p lambda_lm(theta_p) e^{-i m phi_p}.
 *
 * Parallelism: OpenMP over rings (synthesis) and over m (adjoint); each
 * output element is written by exactly one thread, so results do not depend
 * on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* HEALPix RING geometry (Gorski et al. 2005).                                */
/* Rings i = 1 .. 4 nside - 1 from north to south.  In the polar caps         */
/* (i < nside, or 4nside - i < nside) a ring has 4k pixels, k the ring's      */
/* distance from its pole, at z = +-(1 - k^2 / (3 nside^2)) and              */
/* phi_j = (j + 1/2) pi / (2k).  In the equatorial belt a ring has 4 nside    */
/* pixels at z = 4/3 - 2 i / (3 nside), phi_j = (j + 1 - f) pi / (2 nside)    */
/* with f = 1 when i + nside is odd and f = 1/2 otherwise (j = 0-based).      */
/* ------------------------------------------------------------------------- */
int or_nrings(int nside) { return 4 * nside - 1; }

int64_t or_npix(int nside) { return 12LL * nside * nside; }

void or_healpix_rings(int nside, double *z, double *sintheta, double *phi0,
                      int64_t *nr, int64_t *offset)
{
    const int R = 4 * nside - 1;
    int64_t off = 0;
    for (int i = 1; i <= R; ++i) {
        const int k = (i <= 2 * nside) ? i : 4 * nside - i;
        double zz, st, p0;
        int64_t n;
        if (k < nside) {
            const double omz = (double)k * k / (3.0 * nside * nside); /* 1 - |z| */
            zz = 1.0 - omz;
            st = sqrt(omz * (2.0 - omz));
            n = 4LL * k;
            p0 = M_PI / (4.0 * k);
            if (i > 2 * nside) zz = -zz;
        } else {
            zz = 4.0 / 3.0 - 2.0 * i / (3.0 * nside);
            st = sqrt((1.0 - zz) * (1.0 + zz));
            n = 4LL * nside;
            p0 = ((i + nside) & 1) ? 0.0 : M_PI / (4.0 * nside);
        }
        z[i - 1] = zz;
        sintheta[i - 1] = st;
        phi0[i - 1] = p0;
        nr[i - 1] = n;
        offset[i - 1] = off;
        off += n;
    }
}

/* ------------------------------------------------------------------------- */
/* Normalised associated Legendre functions.                                  */
/*   lambda_lm(x) = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_lm(x),               */
/*   P_lm with the Condon-Shortley phase (-1)^m.                              */
/* Seed: lambda_mm = (-1)^m sqrt((2m+1)/(4 pi) prod_{k=1..m} (2k-1)/(2k))     */
/*                   sin^m(theta).                                            */
/* Step: lambda_{m+1,m} = sqrt(2m+3) x lambda_mm,                             */
/*       lambda_lm = a_lm (x lambda_{l-1,m} - lambda_{l-2,m} / a_{l-1,m}),    */
/*       a_lm = sqrt((4 l^2 - 1) / (l^2 - m^2)).                              */
/* The running values are kept as v * 2^E with |v| moderate; out[] receives   */
/* the plain double v * 2^E (which is 0 when it is below the double range).   */
/* ------------------------------------------------------------------------- */
static double log_seed_coef(int m)
{
    /* log of sqrt((2m+1)/(4 pi) prod_{k=1..m} (2k-1)/(2k)) */
    double s = log((2.0 * m + 1.0) / (4.0 * M_PI));
    for (int k = 1; k <= m; ++k) s += log((2.0 * k - 1.0) / (2.0 * k));
    return 0.5 * s;
}

static double coef_a(int l, int m)
{
    return sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
}

static void legendre_column(int lmax, int m, double x, double st, double logc,
                            double *out /* lmax - m + 1 values */)
{
    const int n = lmax - m + 1;
    if (n <= 0) return;
    if (m > 0 && st == 0.0) {
        for (int i = 0; i < n; ++i) out[i] = 0.0;
        return;
    }
    const double lg = logc + (m > 0 ? m * log(st) : 0.0); /* natural log of |lambda_mm| */
    const double ln2 = log(2.0);
    int E = (int)floor(lg / ln2);
    double v0 = exp(lg - E * ln2);
    if (m & 1) v0 = -v0;
    out[0] = ldexp(v0, E);
    if (n == 1) return;
    double v1 = sqrt(2.0 * m + 3.0) * x * v0;
    out[1] = ldexp(v1, E);
    for (int l = m + 2; l <= lmax; ++l) {
        const double v2 = coef_a(l, m) * (x * v1 - v0 / coef_a(l - 1, m));
        v0 = v1;
        v1 = v2;
        if (fabs(v1) > 0x1p+300) {
            v0 = ldexp(v0, -300);
            v1 = ldexp(v1, -300);
            E += 300;
        }
        out[l - m] = ldexp(v1, E);
    }
}

/* lambda_lm(x) for l = m..lmax; sintheta must equal sqrt(1 - x^2). */
void or_legendre(int lmax, int m, double x, double sintheta, double *out)
{
    legendre_column(lmax, m, x, sintheta, log_seed_coef(m), out);
}

static inline int64_t alm_index(int lmax, int l, int m)
{
    return (int64_t)m * (2 * lmax + 3 - m) / 2 + (l - m);
}

int64_t or_nalm(int lmax) { return (int64_t)(lmax + 1) * (lmax + 2) / 2; }

/* ------------------------------------------------------------------------- */
/* Synthesis f = Y a restricted to l <= L (a stored up to lmax).              */
/* Rings [ring_lo, ring_hi) (0-based) are computed; map holds the full        */
/* pixel vector (only those rings' pixels are written).                       */
/*   G_m(theta_r) = sum_{l=m..L} a_lm lambda_lm(cos theta_r)                  */
/*   f_j = Re G_0 + 2 sum_{m=1..L} Re(G_m e^{i m phi_j}),                     */
/*   phi_j = phi0_r + 2 pi j / n_r, evaluated term by term.  Every HEALPix    */
/*   longitude is (2j + q) pi / n_r with q = 0 or 1, so m phi_j is reduced    */
/*   modulo 2 pi exactly in integers before cos/sin.                          */
/* ------------------------------------------------------------------------- */
void or_synthesis(int nside, int lmax, int L, const double *alm, double *map,
                  int ring_lo, int ring_hi)
{
    const int R = 4 * nside - 1;
    double *z = malloc(sizeof(double) * R), *st = malloc(sizeof(double) * R);
    double *p0 = malloc(sizeof(double) * R);
    int64_t *nr = malloc(sizeof(int64_t) * R), *off = malloc(sizeof(int64_t) * R);
    or_healpix_rings(nside, z, st, p0, nr, off);
    double *logc = malloc(sizeof(double) * (L + 1));
    for (int m = 0; m <= L; ++m) logc[m] = log_seed_coef(m);
    if (ring_lo < 0) ring_lo = 0;
    if (ring_hi > R) ring_hi = R;

#pragma omp parallel
    {
        double *lam = malloc(sizeof(double) * (L + 1));
        double *Gr = malloc(sizeof(double) * (L + 1));
        double *Gi = malloc(sizeof(double) * (L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int r = ring_lo; r < ring_hi; ++r) {
            for (int m = 0; m <= L; ++m) {
                legendre_column(L, m, z[r], st[r], logc[m], lam);
                double sr = 0.0, si = 0.0;
                for (int l = m; l <= L; ++l) {
                    const int64_t k = alm_index(lmax, l, m);
                    sr += alm[2 * k] * lam[l - m];
                    si += alm[2 * k + 1] * lam[l - m];
                }
                Gr[m] = sr;
                Gi[m] = si;
            }
            const int64_t n = nr[r];
            const int64_t q = p0[r] != 0.0; /* phi0 = q pi / n */
            for (int64_t j = 0; j < n; ++j) {
                double f = Gr[0];
                for (int m = 1; m <= L; ++m) {
                    /* m phi_j = 2 pi (m (2j + q) mod 2n) / (2n), reduced exactly */
                    const int64_t p = ((int64_t)m * (2 * j + q)) % (2 * n);
                    const double ang = M_PI * (double)p / (double)n;
                    f += 2.0 * (Gr[m] * cos(ang) - Gi[m] * sin(ang));
                }
                map[off[r] + j] = f;
            }
        }
        free(lam);
        free(Gr);
        free(Gi);
    }
    free(z); free(st); free(p0); free(nr); free(off); free(logc);
}

/* ------------------------------------------------------------------------- */
/* Adjoint synthesis b = Y^T f restricted to l <= L, for m in [m_lo, m_hi).   */
/*   F_m(theta_r) = sum_j f_j e^{-i m phi_j}                                  */
/*   b_lm = sum_r lambda_lm(cos theta_r) F_m(theta_r)                         */
/* Entries of alm outside the computed (l, m) range are left untouched.       */
/* ------------------------------------------------------------------------- */
void or_adjoint_synthesis(int nside, int lmax, int L, const double *map,
                          double *alm, int m_lo, int m_hi)
{
    const int R = 4 * nside - 1;
    double *z = malloc(sizeof(double) * R), *st = malloc(sizeof(double) * R);
    double *p0 = malloc(sizeof(double) * R);
    int64_t *nr = malloc(sizeof(int64_t) * R), *off = malloc(sizeof(int64_t) * R);
    or_healpix_rings(nside, z, st, p0, nr, off);
    if (m_lo < 0) m_lo = 0;
    if (m_hi > L + 1) m_hi = L + 1;

#pragma omp parallel
    {
        double *lam = malloc(sizeof(double) * (L + 1));
        double *Fr = malloc(sizeof(double) * R);
        double *Fi = malloc(sizeof(double) * R);
        double *br = malloc(sizeof(double) * (L + 1));
        double *bi = malloc(sizeof(double) * (L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int m = m_lo; m < m_hi; ++m) {
            const double logc = log_seed_coef(m);
            for (int r = 0; r < R; ++r) {
                const int64_t n = nr[r];
                const int64_t q = p0[r] != 0.0;
                double sr = 0.0, si = 0.0;
                for (int64_t j = 0; j < n; ++j) {
                    const int64_t p = ((int64_t)m * (2 * j + q)) % (2 * n);
                    const double ang = M_PI * (double)p / (double)n;
                    const double f = map[off[r] + j];
                    sr += f * cos(ang);
                    si -= f * sin(ang);
                }
                Fr[r] = sr;
                Fi[r] = si;
            }
            for (int l = m; l <= L; ++l) br[l] = bi[l] = 0.0;
            for (int r = 0; r < R; ++r) {
                legendre_column(L, m, z[r], st[r], logc, lam);
                for (int l = m; l <= L; ++l) {
                    br[l] += lam[l - m] * Fr[r];
                    bi[l] += lam[l - m] * Fi[r];
                }
            }
            for (int l = m; l <= L; ++l) {
                const int64_t k = alm_index(lmax, l, m);
                alm[2 * k] = br[l];
                alm[2 * k + 1] = bi[l];
            }
        }
        free(lam); free(Fr); free(Fi); free(br); free(bi);
    }
    free(z); free(st); free(p0); free(nr); free(off);
}

/* ------------------------------------------------------------------------- */
/* Spin-weighted harmonics (polarisation, Eqs. 10-11 of the paper work on     */
/* I, Q, U maps).  Convention:                                                */
/*   sY_lm(theta, phi) = slambda_lm(theta) e^{i m phi},                       */
/*   slambda_lm(theta) = sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta),               */
/* with Wigner's small d (explicit sum below); for s = 0 this is the          */
/* Condon-Shortley Y_lm above.  Polarisation:                                 */
/*   (Q + iU)(n) = sum_{l >= 2} sum_{m=-l..l} 2a_lm 2Y_lm(n),                 */
/*   2a_lm = -(E_lm + i B_lm), E_{l,-m} = (-1)^m conj(E_lm) (B alike),        */
/* E, B stored like a_lm (m >= 0).                                            */
/* d^j_{ab}(beta) = sum_k (-1)^(a-b+k) sqrt((j+a)!(j-a)!(j+b)!(j-b)!)         */
/*                  c^(2j+b-a-2k) s^(a-b+2k) / ((j+b-k)! k! (a-b+k)! (j-a-k)!)*/
/* with c = cos(beta/2), s = sin(beta/2); at j = max(|a|, |b|) exactly one k  */
/* is allowed, which gives the seed.  Upward in l (a, b fixed):               */
/*   d^l = l(2l-1)/sqrt((l^2-a^2)(l^2-b^2)) (x - ab/(l(l-1))) d^{l-1}         */
/*       - l sqrt(((l-1)^2-a^2)((l-1)^2-b^2)) / ((l-1) sqrt((l^2-a^2)(l^2-b^2))) d^{l-2}. */
/* ------------------------------------------------------------------------- */
static double lfact(int n) { return lgamma((double)n + 1.0); }

/* slambda_lm(theta) for l = l0 .. lmax, l0 = max(|m|, |s|); out[l - l0].      */
/* ch = cos(theta/2), sh = sin(theta/2), x = cos(theta).  Returns l0.          */
static int spin_column(int lmax, int m, int s, double x, double ch, double sh, double *out)
{
    const int a = m, b = -s;
    const int l0 = abs(a) > abs(b) ? abs(a) : abs(b);
    if (l0 > lmax) return l0;
    /* seed: the single k of the explicit sum at j = l0 */
    const int j = l0;
    int kk = 0;
    if (a == j) kk = 0;
    else if (a == -j) kk = j + b;
    else if (b == j) kk = j - a;
    else kk = 0; /* b == -j */
    const int ec = 2 * j + b - a - 2 * kk, es = a - b + 2 * kk;
    double lg = 0.5 * (lfact(j + a) + lfact(j - a) + lfact(j + b) + lfact(j - b)) -
                (lfact(j + b - kk) + lfact(kk) + lfact(a - b + kk) + lfact(j - a - kk));
    const int sign = ((a - b + kk) & 1) ? -1 : 1;
    if ((ec > 0 && ch == 0.0) || (es > 0 && sh == 0.0)) {
        for (int l = l0; l <= lmax; ++l) out[l - l0] = 0.0;
        return l0;
    }
    if (ec > 0) lg += ec * log(ch);
    if (es > 0) lg += es * log(sh);
    const double ln2 = log(2.0);
    int E = (int)floor(lg / ln2);
    double v1 = sign * exp(lg - E * ln2), v0 = 0.0; /* d^{l0} and d^{l0-1} = 0, as v * 2^E */
    out[0] = ldexp(v1, E) * sqrt((2.0 * l0 + 1.0) / (4.0 * M_PI));
    for (int l = l0 + 1; l <= lmax; ++l) {
        const double ll = l, d1 = sqrt((ll * ll - (double)a * a) * (ll * ll - (double)b * b));
        double v2;
        if (l == 1) {
            v2 = x * v1; /* a = b = 0: d^1_00 = cos(theta) */
        } else {
            const double c1 = ll * (2.0 * ll - 1.0) / d1 * (x - (double)a * b / (ll * (ll - 1.0)));
            const double lm1 = ll - 1.0;
            const double c2 = ll * sqrt((lm1 * lm1 - (double)a * a) * (lm1 * lm1 - (double)b * b)) / (lm1 * d1);
            v2 = c1 * v1 - c2 * v0;
        }
        v0 = v1;
        v1 = v2;
        if (fabs(v1) > 0x1p+300) {
            v0 = ldexp(v0, -300);
            v1 = ldexp(v1, -300);
            E += 300;
        }
        out[l - l0] = ldexp(v1, E) * sqrt((2.0 * ll + 1.0) / (4.0 * M_PI));
    }
    return l0;
}

static void half_angles(double x, double st, double *ch, double *sh)
{
    if (x >= 0.0) {
        *ch = sqrt(0.5 * (1.0 + x));
        *sh = st / (2.0 * *ch);
    } else {
        *sh = sqrt(0.5 * (1.0 - x));
        *ch = st / (2.0 * *sh);
    }
}

/* slambda_lm(theta) for l = 0 .. lmax (zero below max(|m|, |s|)). */
void or_spin_legendre(int lmax, int m, int s, double x, double sintheta, double *out)
{
    double ch, sh;
    half_angles(x, sintheta, &ch, &sh);
    double *col = malloc(sizeof(double) * (lmax + 1));
    for (int l = 0; l <= lmax; ++l) out[l] = 0.0;
    const int l0 = spin_column(lmax, m, s, x, ch, sh, col);
    for (int l = l0; l <= lmax; ++l) out[l] = col[l - l0];
    free(col);
}

/* 2a_lm for any m from E, B stored for m >= 0 (re, im interleaved). */
static inline void two_a(int lmax, const double *E, const double *B, int l, int m, double *re, double *im)
{
    const int am = abs(m);
    const int64_t k = alm_index(lmax, l, am);
    double er = E[2 * k], ei = E[2 * k + 1], br = B[2 * k], bi = B[2 * k + 1];
    if (m < 0) { /* E_{l,-m} = (-1)^m conj(E_lm), B alike */
        const double sg = (am & 1) ? -1.0 : 1.0;
        er *= sg; ei *= -sg; br *= sg; bi *= -sg;
    }
    /* -(E + i B) */
    *re = -(er - bi);
    *im = -(ei + br);
}

/* Polarisation synthesis (Q, U) from (E, B), l <= L, rings [ring_lo, ring_hi):
 *   P_m(theta_r) = sum_l 2a_lm 2lambda_lm(theta_r),  m = -L..L,
 *   (Q + iU)_j = sum_m P_m e^{i m phi_j},  evaluated term by term. */
void or_synthesis_pol(int nside, int lmax, int L, const double *E, const double *B, double *Q, double *U,
                      int ring_lo, int ring_hi)
{
    const int R = 4 * nside - 1;
    double *z = malloc(sizeof(double) * R), *st = malloc(sizeof(double) * R);
    double *p0 = malloc(sizeof(double) * R);
    int64_t *nr = malloc(sizeof(int64_t) * R), *off = malloc(sizeof(int64_t) * R);
    or_healpix_rings(nside, z, st, p0, nr, off);
    if (ring_lo < 0) ring_lo = 0;
    if (ring_hi > R) ring_hi = R;
#pragma omp parallel
    {
        double *col = malloc(sizeof(double) * (L + 1));
        double *Pr = malloc(sizeof(double) * (2 * L + 1)), *Pi = malloc(sizeof(double) * (2 * L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int r = ring_lo; r < ring_hi; ++r) {
            double ch, sh;
            half_angles(z[r], st[r], &ch, &sh);
            for (int m = -L; m <= L; ++m) {
                double sr = 0.0, si = 0.0;
                const int l0 = spin_column(L, m, 2, z[r], ch, sh, col);
                for (int l = l0; l <= L; ++l) {
                    double ar, ai;
                    two_a(lmax, E, B, l, m, &ar, &ai);
                    sr += ar * col[l - l0];
                    si += ai * col[l - l0];
                }
                Pr[m + L] = sr;
                Pi[m + L] = si;
            }
            const int64_t n = nr[r];
            const int64_t q = p0[r] != 0.0;
            for (int64_t j = 0; j < n; ++j) {
                double fr = 0.0, fi = 0.0;
                for (int m = -L; m <= L; ++m) {
                    const int64_t pp = ((((int64_t)m * (2 * j + q)) % (2 * n)) + 2 * n) % (2 * n);
                    const double ang = M_PI * (double)pp / (double)n, c = cos(ang), s = sin(ang);
                    fr += Pr[m + L] * c - Pi[m + L] * s;
                    fi += Pr[m + L] * s + Pi[m + L] * c;
                }
                Q[off[r] + j] = fr;
                U[off[r] + j] = fi;
            }
        }
        free(col);
        free(Pr);
        free(Pi);
    }
    free(z); free(st); free(p0); free(nr); free(off);
}

/* Adjoint of or_synthesis_pol under sum_p (Q Q' + U U') and
 * Re sum_{l, all m} (conj(E) E' + conj(B) B'):
 *   2t_lm = sum_p (Q + iU)_p conj(2Y_lm(p))                 (m = -L..L)
 *   E_lm = -(2t_lm + (-1)^m conj(2t_{l,-m})) / 2
 *   B_lm = (i/2) (2t_lm - (-1)^m conj(2t_{l,-m}))            (m >= 0, 2 <= l <= L)
 * E, B: all entries written (zero outside 2 <= l <= L). */
void or_adjoint_pol(int nside, int lmax, int L, const double *Q, const double *U, double *E, double *B)
{
    const int R = 4 * nside - 1;
    double *z = malloc(sizeof(double) * R), *st = malloc(sizeof(double) * R);
    double *p0 = malloc(sizeof(double) * R);
    int64_t *nr = malloc(sizeof(int64_t) * R), *off = malloc(sizeof(int64_t) * R);
    or_healpix_rings(nside, z, st, p0, nr, off);
    const int64_t na = or_nalm(lmax);
    for (int64_t i = 0; i < 2 * na; ++i) E[i] = B[i] = 0.0;
    /* t[m + L][l] for m = -L..L, l = 0..L (complex) */
    double *tr = calloc((size_t)(2 * L + 1) * (L + 1), sizeof(double));
    double *ti = calloc((size_t)(2 * L + 1) * (L + 1), sizeof(double));
#pragma omp parallel
    {
        double *col = malloc(sizeof(double) * (L + 1));
        double *Fr = malloc(sizeof(double) * R), *Fi = malloc(sizeof(double) * R);
        double *chs = malloc(sizeof(double) * R), *shs = malloc(sizeof(double) * R);
        for (int r = 0; r < R; ++r) half_angles(z[r], st[r], &chs[r], &shs[r]);
#pragma omp for schedule(dynamic, 1)
        for (int m = -L; m <= L; ++m) {
            for (int r = 0; r < R; ++r) {
                const int64_t n = nr[r];
                const int64_t q = p0[r] != 0.0;
                double sr = 0.0, si = 0.0;
                for (int64_t j = 0; j < n; ++j) {
                    const int64_t pp = ((((int64_t)m * (2 * j + q)) % (2 * n)) + 2 * n) % (2 * n);
                    const double ang = M_PI * (double)pp / (double)n, c = cos(ang), s = sin(ang);
                    const double qr = Q[off[r] + j], ui = U[off[r] + j];
                    /* (Q + iU) e^{-i ang} */
                    sr += qr * c + ui * s;
                    si += ui * c - qr * s;
                }
                Fr[r] = sr;
                Fi[r] = si;
            }
            double *rowr = tr + (size_t)(m + L) * (L + 1), *rowi = ti + (size_t)(m + L) * (L + 1);
            for (int r = 0; r < R; ++r) {
                const int l0 = spin_column(L, m, 2, z[r], chs[r], shs[r], col);
                for (int l = l0; l <= L; ++l) {
                    rowr[l] += col[l - l0] * Fr[r];
                    rowi[l] += col[l - l0] * Fi[r];
                }
            }
        }
        free(col); free(Fr); free(Fi); free(chs); free(shs);
    }
    for (int m = 0; m <= L; ++m) {
        const double sg = (m & 1) ? -1.0 : 1.0;
        for (int l = (m > 2 ? m : 2); l <= L; ++l) {
            const double ar = tr[(size_t)(m + L) * (L + 1) + l], ai = ti[(size_t)(m + L) * (L + 1) + l];
            const double cr = sg * tr[(size_t)(-m + L) * (L + 1) + l], ci = -sg * ti[(size_t)(-m + L) * (L + 1) + l];
            const int64_t k = alm_index(lmax, l, m);
            E[2 * k] = -0.5 * (ar + cr);
            E[2 * k + 1] = -0.5 * (ai + ci);
            /* (i/2)(t - c) */
            B[2 * k] = -0.5 * (ai - ci);
            B[2 * k + 1] = 0.5 * (ar - cr);
        }
    }
    free(tr); free(ti);
    free(z); free(st); free(p0); free(nr); free(off);
}

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
