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
