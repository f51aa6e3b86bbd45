/*
 * sht_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU reference for scalar spherical
 * harmonic synthesis on iso-latitude ring grids (HEALPix in particular) and
 * for its real-inner-product adjoint.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load this library; the product path
 * never does.  It shares no code with the CUDA path.
 *
 * What it computes (Seljebotn, "Wavemoth", arXiv 1110.4874):
 *   - the synthesis sum, Eq. (shdef), evaluated at the pixels (Sec. 2.2);
 *   - via the separation of sums, Eq. (sh-baseline):
 *       q_m(z_k) = sum_{l=m}^{L} a_lm Ptilde_l^m(z_k)       (Eq. legendre-transform)
 *       f(theta_k, phi_kj) = sum_{m=-L}^{L} q_m(z_k) e^{i m phi_kj}
 *     with q_{-m} = conj(q_m) for a real field (Sec. 2.1, a_{l,-m} = (-1)^m a*_lm)
 *     and phi_kj = phi_k0 + 2 pi j / J_k (Eq. phi);
 *   - Ptilde_l^m is the normalised associated Legendre function of Eq. (Y-def),
 *     with the Condon-Shortley phase (-1)^m.
 *
 * Deliberate choices that keep it independent of the fast method:
 *   - its own ONE-step recurrence in l (the textbook one), not the paper's
 *     jump-two relation of Eq. (three-term);
 *   - the recurrence and every sum are carried in double-double (unevaluated
 *     pairs of FP64 numbers built from error-free transformations: TwoSum,
 *     and TwoProd by fma), so the oracle's own rounding error stays near
 *     1e-30 relative instead of growing with l as a plain FP64 recurrence
 *     does (about 1e-13 at l = 4096 away from the poles, worse near them);
 *   - recurrence values carry a separate power-of-two exponent, so nothing
 *     underflows near the poles (sin^m theta reaches 1e-13900 at m = 4096);
 *   - no even/odd split: every ring is evaluated directly;
 *   - a direct O(L J) DFT per ring (no FFT), with the angle m*phi reduced
 *     exactly in integers: phi_kj = pi (2j + s_k) / J_k, so m*phi_kj is
 *     2 pi n / (2 J_k) with n = m (2j + s_k) mod 2 J_k.
 *
 * Ring grid description shared by every routine: nrings rings, ring k has
 * z = cos(theta_k) and sin(theta_k), each as a double-double pair
 * (z[k] + zlo[k], sinth[k] + sinlo[k]) so that the ring position is known to
 * far better than a double, J[k] pixels and a half-pixel shift flag
 * s[k] in {0,1}: phi_kj = pi (2 j + s_k) / J_k, j = 0..J_k-1.  Pixel values
 * of ring k are stored contiguously, rings in the given order.
 *
 * a_lm layout: complex128 interleaved (re, im), index m(2L+1-m)/2 + l,
 * i.e. m-major with l = m..L contiguous; Im a_l0 is ignored.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------- double-double */
typedef struct { double hi, lo; } dd;

static inline dd two_sum(double a, double b)
{
    double s = a + b, bb = s - a;
    dd r = {s, (a - (s - bb)) + (b - bb)};
    return r;
}

static inline dd quick_two_sum(double a, double b)
{
    double s = a + b;
    dd r = {s, b - (s - a)};
    return r;
}

static inline dd dd_from(double a) { dd r = {a, 0.0}; return r; }

static inline dd dd_add(dd x, dd y)
{
    dd s = two_sum(x.hi, y.hi), t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

static inline dd dd_neg(dd x) { dd r = {-x.hi, -x.lo}; return r; }
static inline dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

static inline dd dd_mul(dd x, dd y)
{
    double p = x.hi * y.hi;
    double e = fma(x.hi, y.hi, -p);
    e += x.hi * y.lo + x.lo * y.hi;
    return quick_two_sum(p, e);
}

static inline dd dd_mul_d(dd x, double d)
{
    double p = x.hi * d;
    double e = fma(x.hi, d, -p);
    e += x.lo * d;
    return quick_two_sum(p, e);
}

static inline dd dd_div(dd x, dd y)
{
    double q1 = x.hi / y.hi;
    dd r = dd_sub(x, dd_mul_d(y, q1));
    double q2 = r.hi / y.hi;
    r = dd_sub(r, dd_mul_d(y, q2));
    double q3 = r.hi / y.hi;
    dd q = quick_two_sum(q1, q2);
    return dd_add(q, dd_from(q3));
}

static inline dd dd_sqrt(dd x)
{
    if (x.hi <= 0.0) return dd_from(0.0);
    double s = sqrt(x.hi);
    double p = s * s;
    double e = fma(s, s, -p);
    double r = ((x.hi - p) - e + x.lo) / (2.0 * s);
    return quick_two_sum(s, r);
}

static inline dd dd_ldexp(dd x, int e) { dd r = {ldexp(x.hi, e), ldexp(x.lo, e)}; return r; }

/* pi as a double-double */
static const dd DD_PI = {3.141592653589793116e+00, 1.224646799147353207e-16};

long long orc_nalm(int lmax) { return (long long)(lmax + 1) * (lmax + 2) / 2; }

static long long alm_index(int lmax, int l, int m)
{
    return (long long)m * (2 * lmax + 1 - m) / 2 + l;
}

/* ------------------------------------------------------- HEALPix geometry */
/*
 * HEALPix RING scheme (Gorski et al. 2005, the grid the paper targets):
 *   north polar ring i = 1..N-1 : z = 1 - i^2/(3N^2), J = 4i, phi = pi(2j+1)/(4i)
 *   belt ring i = N..2N          : z = (4N - 2i)/(3N), J = 4N,
 *                                  phi = pi(2j+s)/(4N), s = 1 iff (i+N) even
 *   south ring 4N-i              : mirror of ring i (z -> -z, same J and phi)
 * Pixels are numbered ring by ring from the north pole.
 * z and sin(theta) are returned as double-double pairs (hi, lo), formed
 * from exact integer ratios:
 *   polar: z = (3N^2 - i^2)/(3N^2),  sin^2 = i^2 (6N^2 - i^2) / (9N^4)
 *   belt : z = (4N - 2i)/(3N),       sin^2 = (2i - N)(7N - 2i) / (9N^2)
 * (a rounded double z alone moves theta by ~1e-10 relative on the first
 * ring at Nside = 2048, where 1 - z ~ 8e-8).
 */
int orc_healpix_nrings(int nside) { return 4 * nside - 1; }

int orc_healpix_rings(int nside, double *z, double *zlo, double *sinth,
                      double *sinlo, int *J, int *s, long long *start)
{
    if (nside < 1) return -1;
    const long long N = nside;
    const int nr = 4 * nside - 1;
    long long pix = 0;
    for (int r = 1; r <= nr; ++r) {
        const long long i = r <= 2 * nside ? r : 4 * nside - r;
        long long zn, zd, sn, sd;     /* z = zn/zd, sin^2 = sn/sd, exact integers */
        int Ji, si;
        if (i < N) {
            zn = 3 * N * N - i * i;  zd = 3 * N * N;
            sn = i * i * (6 * N * N - i * i);  sd = 9 * N * N * N * N;
            Ji = (int)(4 * i);
            si = 1;
        } else {
            zn = 4 * N - 2 * i;  zd = 3 * N;
            sn = (2 * i - N) * (7 * N - 2 * i);  sd = 9 * N * N;
            Ji = (int)(4 * N);
            si = ((i + N) % 2 == 0) ? 1 : 0;
        }
        dd zz = dd_div(dd_from((double)zn), dd_from((double)zd));
        dd ss = dd_sqrt(dd_div(dd_from((double)sn), dd_from((double)sd)));
        const int k = r - 1;
        if (r > 2 * nside) zz = dd_neg(zz);
        z[k] = zz.hi;
        zlo[k] = zz.lo;
        sinth[k] = ss.hi;
        sinlo[k] = ss.lo;
        J[k] = Ji;
        s[k] = si;
        if (start) start[k] = pix;
        pix += Ji;
    }
    return 0;
}

/* sin(theta) = sqrt((1-z)(1+z)) in double-double for rings given by a double z */
void orc_sin_from_cos(int n, const double *z, double *sinth, double *sinlo)
{
    for (int k = 0; k < n; ++k) {
        dd a = two_sum(1.0, -z[k]), b = two_sum(1.0, z[k]);
        dd ss = dd_sqrt(dd_mul(a, b));
        sinth[k] = ss.hi;
        sinlo[k] = ss.lo;
    }
}

/* --------------------------------------------------- Legendre functions */
/*
 * Ptilde_l^m(z), l = m..lmax (Eq. Y-def normalisation, Condon-Shortley
 * phase), by the one-step recurrence
 *   Ptilde_m^m     = (-1)^m c_m sin^m(theta),
 *                    c_m^2 = (1/(4 pi)) prod_{i=1}^{m} (2i+1)/(2i)
 *   Ptilde_{m+1}^m = sqrt(2m+3) z Ptilde_m^m
 *   Ptilde_l^m     = (z Ptilde_{l-1}^m - b_{l-1} Ptilde_{l-2}^m) / b_l,
 *   b_l = sqrt((l^2 - m^2)/(4 l^2 - 1)),
 * all in double-double.  The per-m coefficients are tabulated once in a
 * plm_table and reused for every ring.
 */
typedef struct {
    int m, lmax;
    dd cm;            /* c_m                     */
    dd sq;            /* sqrt(2m+3)              */
    dd *b;            /* b_l,   l = m+1..lmax    (index l-m) */
    dd *ib;           /* 1/b_l, l = m+1..lmax    (index l-m) */
} plm_table;

static void plm_table_init(plm_table *t, int m, int lmax)
{
    t->m = m;
    t->lmax = lmax;
    dd c2 = dd_div(dd_from(1.0), dd_mul_d(DD_PI, 4.0));
    for (int i = 1; i <= m; ++i)
        c2 = dd_mul(c2, dd_div(dd_from(2.0 * i + 1.0), dd_from(2.0 * i)));
    t->cm = dd_sqrt(c2);
    t->sq = dd_sqrt(dd_from(2.0 * m + 3.0));
    int n = lmax - m + 1;
    t->b = (dd *)malloc(sizeof(dd) * (size_t)(n > 0 ? n : 1));
    t->ib = (dd *)malloc(sizeof(dd) * (size_t)(n > 0 ? n : 1));
    for (int l = m + 1; l <= lmax; ++l) {
        /* (l-m)(l+m) and (2l-1)(2l+1) are exact integers in doubles */
        dd num = dd_from((double)(l - m) * (double)(l + m));
        dd den = dd_from((double)(2 * l - 1) * (double)(2 * l + 1));
        dd b = dd_sqrt(dd_div(num, den));
        t->b[l - m] = b;
        t->ib[l - m] = dd_div(dd_from(1.0), b);
    }
}

static void plm_table_free(plm_table *t)
{
    free(t->b);
    free(t->ib);
}

/* mantissa * 2^E with the mantissa's leading double in [0.5, 1) */
static dd dd_normalise(dd x, int *E)
{
    if (x.hi == 0.0) return x;
    int e;
    frexp(x.hi, &e);
    *E += e;
    return dd_ldexp(x, -e);
}

/* s^m as (mantissa, exponent) by binary powering */
static dd dd_pow_scaled(dd s, int m, int *E)
{
    dd r = dd_from(1.0);
    int Er = 0, Eb = 0;
    dd b = dd_normalise(s, &Eb);
    while (m > 0) {
        if (m & 1) {
            r = dd_mul(r, b);
            Er += Eb;
            r = dd_normalise(r, &Er);
        }
        m >>= 1;
        if (m) {
            b = dd_mul(b, b);
            Eb *= 2;
            b = dd_normalise(b, &Eb);
        }
    }
    *E = Er;
    return r;
}

/* Values at one point for l = m..lmax, as double-double (hi, lo arrays). */
static void plm_eval(const plm_table *t, dd z, dd sinth, double *ohi, double *olo)
{
    const int m = t->m, lmax = t->lmax;
    int E;
    dd p0 = dd_pow_scaled(sinth, m, &E);
    p0 = dd_mul(p0, t->cm);
    if (m & 1) p0 = dd_neg(p0);
#define EMIT(idx, v)                                                        \
    do {                                                                    \
        if (E == 0) { ohi[idx] = (v).hi; olo[idx] = (v).lo; }               \
        else { ohi[idx] = ldexp((v).hi, E); olo[idx] = ldexp((v).lo, E); }  \
    } while (0)
    EMIT(0, p0);
    if (m == lmax) return;
    dd p1 = dd_mul(dd_mul(t->sq, p0), z);
    EMIT(1, p1);
    for (int l = m + 2; l <= lmax; ++l) {
        dd a = dd_mul(p1, z);
        dd c = dd_mul(t->b[l - 1 - m], p0);
        dd p2 = dd_mul(dd_sub(a, c), t->ib[l - m]);
        p0 = p1;
        p1 = p2;
        if (E != 0 && p1.hi != 0.0) {
            /* bring the pair back to a zero exponent once it is representable */
            int e;
            frexp(p1.hi, &e);
            if (e + E > -900) {
                p0 = dd_ldexp(p0, E);
                p1 = dd_ldexp(p1, E);
                E = 0;
            } else if (e > 512) {
                p0 = dd_ldexp(p0, -256);
                p1 = dd_ldexp(p1, -256);
                E += 256;
            }
        }
        EMIT(l - m, p1);
    }
#undef EMIT
}

void orc_legendre(int m, int lmax, double z, double zlo, double sinth,
                  double sinlo, double *out)
{
    if (m < 0 || m > lmax) return;
    plm_table t;
    plm_table_init(&t, m, lmax);
    double *lo = (double *)malloc(sizeof(double) * (size_t)(lmax - m + 1));
    const dd zz = {z, zlo}, ss = {sinth, sinlo};
    plm_eval(&t, zz, ss, out, lo);
    for (int i = 0; i <= lmax - m; ++i) out[i] += lo[i];
    free(lo);
    plm_table_free(&t);
}

/* ------------------------------------------------------------ synthesis */
/*
 * Legendre stage: q[map][k][m] (complex, interleaved) = sum_l a_lm Ptilde_l^m(z_k)
 * for m = 0..lmax at each of the given rings (Eq. legendre-transform).
 * Parallel over m; the sum over l is accumulated in double-double.
 */
int orc_legendre_q(int nrings, const double *z, const double *zlo,
                   const double *sinth, const double *sinlo, int lmax,
                   int nmaps, const double *alm, double *q, int nthreads)
{
    if (nrings < 0 || lmax < 0 || nmaps < 1) return -1;
    const long long nalm = orc_nalm(lmax);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *ph = (double *)malloc(sizeof(double) * (size_t)(lmax + 1));
        double *pl = (double *)malloc(sizeof(double) * (size_t)(lmax + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int m = 0; m <= lmax; ++m) {
            plm_table t;
            plm_table_init(&t, m, lmax);
            for (int k = 0; k < nrings; ++k) {
                const dd zk = {z[k], zlo[k]}, sk = {sinth[k], sinlo[k]};
                plm_eval(&t, zk, sk, ph, pl);
                for (int b = 0; b < nmaps; ++b) {
                    const double *a = alm + 2 * (size_t)nalm * b;
                    dd re = dd_from(0.0), im = dd_from(0.0);
                    for (int l = m; l <= lmax; ++l) {
                        const long long idx = alm_index(lmax, l, m);
                        const dd P = {ph[l - m], pl[l - m]};
                        re = dd_add(re, dd_mul_d(P, a[2 * idx]));
                        if (m > 0) im = dd_add(im, dd_mul_d(P, a[2 * idx + 1]));
                    }
                    double *qo = q + 2 * (((size_t)b * nrings + k) * (lmax + 1) + m);
                    qo[0] = re.hi + re.lo;
                    qo[1] = im.hi + im.lo;
                }
            }
            plm_table_free(&t);
        }
        free(ph);
        free(pl);
    }
    return 0;
}

/*
 * cos and sin of 2 pi n / D for n = 0..D-1 (the exact angles of one ring),
 * from libm with the integer n folded so that the angle lies in [-pi, pi].
 */
static void ring_phase_table(int D, double *c, double *s)
{
    for (int n = 0; n < D; ++n) {
        int k = n;
        if (2 * k > D) k -= D;
        double ang = 2.0 * DD_PI.hi * ((double)k / (double)D);
        c[n] = cos(ang);
        s[n] = sin(ang);
    }
}

/*
 * Fourier stage: map values from q (Eq. sh-baseline / Eq. phi), as a direct
 * sum over m for every pixel, accumulated in double-double:
 *   f_kj = Re q_0 + 2 sum_{m=1}^{L} (Re q_m cos(m phi_kj) - Im q_m sin(m phi_kj)).
 */
int orc_phi_synth(int nrings, const int *J, const int *s, int lmax, int nmaps,
                  const double *q, double *map, int nthreads)
{
    if (nrings < 0 || lmax < 0 || nmaps < 1) return -1;
    long long *start = (long long *)malloc(sizeof(long long) * (size_t)(nrings + 1));
    start[0] = 0;
    for (int k = 0; k < nrings; ++k) start[k + 1] = start[k] + J[k];
    const long long npix = start[nrings];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int k = 0; k < nrings; ++k) {
            const int Jk = J[k], D = 2 * J[k];
            double *ct = (double *)malloc(sizeof(double) * (size_t)D);
            double *st = (double *)malloc(sizeof(double) * (size_t)D);
            ring_phase_table(D, ct, st);
            for (int b = 0; b < nmaps; ++b) {
                const double *qk = q + 2 * (((size_t)b * nrings + k) * (lmax + 1));
                double *out = map + (size_t)b * npix + start[k];
                for (int j = 0; j < Jk; ++j) {
                    const long long step = 2LL * j + s[k];   /* m*phi = 2 pi m step / D */
                    dd acc = dd_from(qk[0]);
                    long long n = 0;
                    for (int m = 1; m <= lmax; ++m) {
                        n = (n + step) % D;
                        acc = dd_add(acc, dd_mul_d(dd_from(2.0 * qk[2 * m]), ct[n]));
                        acc = dd_add(acc, dd_mul_d(dd_from(-2.0 * qk[2 * m + 1]), st[n]));
                    }
                    out[j] = acc.hi + acc.lo;
                }
            }
            free(ct);
            free(st);
        }
    }
    free(start);
    return 0;
}

/* Full synthesis: Legendre stage then Fourier stage. */
int orc_synth(int nrings, const double *z, const double *zlo, const double *sinth,
              const double *sinlo, const int *J, const int *s, int lmax, int nmaps,
              const double *alm, double *map, int nthreads)
{
    size_t nq = 2 * (size_t)nmaps * nrings * (lmax + 1);
    double *q = (double *)malloc(sizeof(double) * (nq ? nq : 1));
    if (!q) return -2;
    int rc = orc_legendre_q(nrings, z, zlo, sinth, sinlo, lmax, nmaps, alm, q, nthreads);
    if (rc == 0) rc = orc_phi_synth(nrings, J, s, lmax, nmaps, q, map, nthreads);
    free(q);
    return rc;
}

/* -------------------------------------------------------------- adjoint */
/*
 * Fourier-stage adjoint: F[map][k][m] = sum_j f_kj e^{-i m phi_kj}, m = 0..L.
 */
int orc_phi_adjoint(int nrings, const int *J, const int *s, int lmax, int nmaps,
                    const double *map, double *F, int nthreads)
{
    if (nrings < 0 || lmax < 0 || nmaps < 1) return -1;
    long long *start = (long long *)malloc(sizeof(long long) * (size_t)(nrings + 1));
    start[0] = 0;
    for (int k = 0; k < nrings; ++k) start[k + 1] = start[k] + J[k];
    const long long npix = start[nrings];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int k = 0; k < nrings; ++k) {
            const int Jk = J[k], D = 2 * J[k];
            double *ct = (double *)malloc(sizeof(double) * (size_t)D);
            double *st = (double *)malloc(sizeof(double) * (size_t)D);
            ring_phase_table(D, ct, st);
            for (int b = 0; b < nmaps; ++b) {
                const double *f = map + (size_t)b * npix + start[k];
                double *Fk = F + 2 * (((size_t)b * nrings + k) * (lmax + 1));
                for (int m = 0; m <= lmax; ++m) {
                    dd re = dd_from(0.0), im = dd_from(0.0);
                    for (int j = 0; j < Jk; ++j) {
                        long long n = ((long long)m * (2LL * j + s[k])) % D;
                        re = dd_add(re, dd_mul_d(dd_from(f[j]), ct[n]));
                        im = dd_add(im, dd_mul_d(dd_from(-f[j]), st[n]));
                    }
                    Fk[2 * m] = re.hi + re.lo;
                    Fk[2 * m + 1] = im.hi + im.lo;
                }
            }
            free(ct);
            free(st);
        }
    }
    free(start);
    return 0;
}

/*
 * Legendre-stage adjoint: alm[l,m] = c_m sum_k Ptilde_l^m(z_k) F_m(k), with
 * c_0 = 1 (and Im a_l0 = 0) and c_m = 2 for m >= 1.  Together with the
 * Fourier-stage adjoint this is the transpose of the real-linear synthesis
 * map (Re a_lm, Im a_lm) -> f under the plain real inner products, i.e.
 *   (Y^T f)_l0 = sum_p f_p Ptilde_l^0(z_p),
 *   (Y^T f)_lm = 2 sum_p f_p Ptilde_l^m(z_p) e^{-i m phi_p}   (m >= 1);
 * it is the Y^dagger of Eq. (wiener) up to the factor 2 for m >= 1.
 */
int orc_legendre_adjoint(int nrings, const double *z, const double *zlo,
                         const double *sinth, const double *sinlo,
                         int lmax, int nmaps, const double *F, double *alm,
                         int nthreads)
{
    if (nrings < 0 || lmax < 0 || nmaps < 1) return -1;
    const long long nalm = orc_nalm(lmax);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *ph = (double *)malloc(sizeof(double) * (size_t)(lmax + 1));
        double *pl = (double *)malloc(sizeof(double) * (size_t)(lmax + 1));
        dd *acc = (dd *)malloc(sizeof(dd) * 2 * (size_t)(lmax + 1) * nmaps);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int m = 0; m <= lmax; ++m) {
            const int n = lmax - m + 1;
            for (size_t i = 0; i < 2 * (size_t)n * nmaps; ++i) acc[i] = dd_from(0.0);
            plm_table t;
            plm_table_init(&t, m, lmax);
            for (int k = 0; k < nrings; ++k) {
                const dd zk = {z[k], zlo[k]}, sk = {sinth[k], sinlo[k]};
                plm_eval(&t, zk, sk, ph, pl);
                for (int b = 0; b < nmaps; ++b) {
                    const double *Fk = F + 2 * (((size_t)b * nrings + k) * (lmax + 1) + m);
                    dd *ab = acc + 2 * (size_t)n * b;
                    for (int i = 0; i < n; ++i) {
                        const dd P = {ph[i], pl[i]};
                        ab[2 * i] = dd_add(ab[2 * i], dd_mul_d(P, Fk[0]));
                        ab[2 * i + 1] = dd_add(ab[2 * i + 1], dd_mul_d(P, Fk[1]));
                    }
                }
            }
            plm_table_free(&t);
            const double cm = m == 0 ? 1.0 : 2.0;
            for (int b = 0; b < nmaps; ++b) {
                dd *ab = acc + 2 * (size_t)n * b;
                for (int i = 0; i < n; ++i) {
                    const long long idx = alm_index(lmax, m + i, m);
                    double *o = alm + 2 * ((size_t)nalm * b + idx);
                    o[0] = cm * (ab[2 * i].hi + ab[2 * i].lo);
                    o[1] = m == 0 ? 0.0 : cm * (ab[2 * i + 1].hi + ab[2 * i + 1].lo);
                }
            }
        }
        free(ph);
        free(pl);
        free(acc);
    }
    return 0;
}

/* Full adjoint: Fourier-stage adjoint then Legendre-stage adjoint. */
int orc_adjoint(int nrings, const double *z, const double *zlo, const double *sinth,
                const double *sinlo, const int *J, const int *s, int lmax, int nmaps,
                const double *map, double *alm, int nthreads)
{
    size_t nF = 2 * (size_t)nmaps * nrings * (lmax + 1);
    double *F = (double *)malloc(sizeof(double) * (nF ? nF : 1));
    if (!F) return -2;
    int rc = orc_phi_adjoint(nrings, J, s, lmax, nmaps, map, F, nthreads);
    if (rc == 0)
        rc = orc_legendre_adjoint(nrings, z, zlo, sinth, sinlo, lmax, nmaps, F, alm, nthreads);
    free(F);
    return rc;
}

/* ------------------------------------------------ spin-weighted functions */
/*
 * Spin-weighted harmonics, for the polarised transform the paper points to
 * (Sec. 5, "spin-weighted spherical harmonic transforms"):
 *   sY_lm(theta, phi) = s_lambda_lm(theta) e^{i m phi},
 *   s_lambda_lm(theta) = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta),
 * with d^l_{m1 m2}(theta) = <l m1| exp(-i theta J_y) |l m2> the Wigner
 * small-d function.  This is the Newman-Penrose convention, in which the
 * spin-raising operator takes s_Y to (s+1)_Y; at s = 0 it is Eq. (Y-def)
 * with the Condon-Shortley phase.  d is evaluated from its closed form in
 * Jacobi polynomials (DLMF 18.5, Varshalovich et al. Sec. 4.3.4): with
 * k = min(l+m2, l-m2, l+m1, l-m1) and, by which of the four attains k,
 *   a = |m1 - m2|, b = 2l - 2k - a, sign (-1)^(m1-m2) when k = l+m2 or
 *   l-m1 (else +1),
 *   d = sign sqrt(C(2l-k, k+a) / C(k+b, b)) sin(theta/2)^a cos(theta/2)^b
 *       P_k^(a,b)(cos theta),
 * P_k^(a,b) by its three-term recurrence in the degree (DLMF 18.9.1), all in
 * long double.  This is a different route from the product path's plan
 * builder, which runs the Wigner recurrence in l.
 */
/* P_k^(a,b)(x) for k = 0..n into p[0..n] */
static void jacobi_all(int n, long double a, long double b, long double x, long double *p)
{
    p[0] = 1.0L;
    if (n == 0) return;
    p[1] = (a + 1.0L) + 0.5L * (a + b + 2.0L) * (x - 1.0L);
    for (int k = 2; k <= n; ++k) {
        const long double c = 2.0L * k + a + b;
        p[k] = ((c - 1.0L) * (c * (c - 2.0L) * x + a * a - b * b) * p[k - 1] -
                2.0L * (k + a - 1.0L) * (k + b - 1.0L) * c * p[k - 2]) /
               (2.0L * k * (k + a + b) * (c - 2.0L));
    }
}

static long double log_binom(int n, int r)
{
    return lgammal(n + 1.0L) - lgammal(r + 1.0L) - lgammal(n - r + 1.0L);
}

/* half-angle sine and cosine from cos(theta), sin(theta) (double-double
   inputs), without cancellation on either hemisphere */
static void half_angles(dd z, dd st, long double *sh, long double *ch)
{
    const long double zz = (long double)z.hi + z.lo, ss = (long double)st.hi + st.lo;
    if (zz >= 0) {
        *ch = sqrtl(0.5L * (1.0L + zz));
        *sh = ss / (2.0L * *ch);
    } else {
        *sh = sqrtl(0.5L * (1.0L - zz));
        *ch = ss / (2.0L * *sh);
    }
}

/* s_lambda_lm at one point for l = 0..lmax (0 where l < max(|m|, |s|)).
   For fixed (m1, m2) = (m, -s) the case of the closed form, hence (a, b)
   and the sign, is the same for every l >= l0 = max(|m1|, |m2|), and
   k = l - l0, so one pass of the degree recurrence serves all l. */
static void spin_lambda_eval(int s, int m, int lmax, dd z, dd st, long double *out)
{
    for (int l = 0; l <= lmax; ++l) out[l] = 0.0L;
    const int m1 = m, m2 = -s;
    const int l0 = abs(m1) > abs(m2) ? abs(m1) : abs(m2);
    if (l0 > lmax) return;
    long double sh, ch;
    half_angles(z, st, &sh, &ch);
    const long double x = (long double)z.hi + z.lo;
    /* which of l+m2, l-m2, l+m1, l-m1 is smallest (they differ by l-free amounts) */
    const int k1 = m2, k2 = -m2, k3 = m1, k4 = -m1;
    int kk = k1, a, sgn;
    if (k2 < kk) kk = k2;
    if (k3 < kk) kk = k3;
    if (k4 < kk) kk = k4;
    if (kk == k1) { a = m1 - m2; sgn = (a & 1) ? -1 : 1; }
    else if (kk == k2) { a = m2 - m1; sgn = 1; }
    else if (kk == k3) { a = m2 - m1; sgn = 1; }
    else { a = m1 - m2; sgn = (a & 1) ? -1 : 1; }
    const int n = lmax - l0;
    long double *p = (long double *)malloc(sizeof(long double) * (size_t)(n + 1));
    const long double lsh = logl(sh), lch = logl(ch);
    const long double sign_s = (s & 1) ? -1.0L : 1.0L;
    const long double four_pi = 4.0L * 3.14159265358979323846264338327950288L;
    int b0 = -1;
    for (int l = l0; l <= lmax; ++l) {
        const int k = l - l0, b = 2 * l - 2 * k - a;
        if (b0 < 0) {                   /* b = 2 l0 - a is the same for every l */
            b0 = b;
            jacobi_all(n, a, b, x, p);
        }
        const long double lp = 0.5L * (log_binom(2 * l - k, k + a) - log_binom(k + b, b)) +
                               (a ? a * lsh : 0.0L) + (b ? b * lch : 0.0L);
        const long double d = lp < -11000.0L ? 0.0L : sgn * expl(lp) * p[k];
        out[l] = sign_s * sqrtl((2.0L * l + 1.0L) / four_pi) * d;
    }
    free(p);
}

void orc_spin_lambda(int s, int m, int lmax, double z, double zlo, double sinth, double sinlo,
                     double *out)
{
    long double *v = (long double *)malloc(sizeof(long double) * (size_t)(lmax + 1));
    const dd zz = {z, zlo}, ss = {sinth, sinlo};
    spin_lambda_eval(s, m, lmax, zz, ss, v);
    for (int l = 0; l <= lmax; ++l) out[l] = (double)v[l];
    free(v);
}

/*
 * Polarised (spin-2) Legendre stage at the given rings, HEALPix convention
 * (Q + iU) = -sum (aE + i aB) 2Y, (Q - iU) = -sum (aE - i aB) (-2)Y:
 * with F+- = (2_lambda +- (-2)_lambda)/2,
 *   Q_m(z) = -sum_l [aE F+ + i aB F-],   U_m(z) = -sum_l [aB F+ - i aE F-],
 * so that Q = Re Q_0 + 2 sum_{m>=1} Re(Q_m e^{i m phi}) and the same for U
 * (both maps real).  qQ, qU: [nmaps][nrings][lmax+1] complex.
 */
int orc_spin_q(int nrings, const double *z, const double *zlo, const double *sinth,
               const double *sinlo, int lmax, int nmaps, const double *aE, const double *aB,
               double *qQ, double *qU, int nthreads)
{
    if (nrings < 0 || lmax < 0 || nmaps < 1) return -1;
    const long long nalm = orc_nalm(lmax);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        long double *lp = (long double *)malloc(sizeof(long double) * (size_t)(lmax + 1));
        long double *lm = (long double *)malloc(sizeof(long double) * (size_t)(lmax + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int k = 0; k < nrings; ++k) {
            const dd zk = {z[k], zlo[k]}, sk = {sinth[k], sinlo[k]};
            for (int m = 0; m <= lmax; ++m) {
                spin_lambda_eval(2, m, lmax, zk, sk, lp);
                spin_lambda_eval(-2, m, lmax, zk, sk, lm);
                for (int b = 0; b < nmaps; ++b) {
                    const double *e = aE + 2 * (size_t)nalm * b, *bb = aB + 2 * (size_t)nalm * b;
                    long double qr = 0, qi = 0, ur = 0, ui = 0;
                    for (int l = m; l <= lmax; ++l) {
                        const long long idx = alm_index(lmax, l, m);
                        const long double Fp = 0.5L * (lp[l] + lm[l]), Fm = 0.5L * (lp[l] - lm[l]);
                        const long double er = e[2 * idx], ei = m ? e[2 * idx + 1] : 0.0;
                        const long double br = bb[2 * idx], bi = m ? bb[2 * idx + 1] : 0.0;
                        /* Q_m -= aE F+ + i aB F-;  U_m -= aB F+ - i aE F- */
                        qr -= er * Fp - bi * Fm;
                        qi -= ei * Fp + br * Fm;
                        ur -= br * Fp + ei * Fm;
                        ui -= bi * Fp - er * Fm;
                    }
                    double *qo = qQ + 2 * (((size_t)b * nrings + k) * (lmax + 1) + m);
                    double *uo = qU + 2 * (((size_t)b * nrings + k) * (lmax + 1) + m);
                    qo[0] = (double)qr;
                    qo[1] = (double)qi;
                    uo[0] = (double)ur;
                    uo[1] = (double)ui;
                }
            }
        }
        free(lp);
        free(lm);
    }
    return 0;
}

/*
 * Transpose of the polarised Legendre stage under real inner products over
 * (Re, Im) pairs: given GQ_m(k), GU_m(k) = sum_j f_kj e^{-i m phi_kj} of the
 * Q and U maps (orc_phi_adjoint), and c_0 = 1, c_m = 2 (the -m terms),
 *   gE_lm = c_m sum_k [-F+ GQ - i F- GU],   gB_lm = c_m sum_k [i F- GQ - F+ GU],
 * the derivatives of sum_p (Q'_p Q_p + U'_p U_p) with respect to Re and Im
 * of aE_lm and aB_lm (written as Re + i Im).  Im of the m = 0 entries is 0.
 */
int orc_spin_legendre_adjoint(int nrings, const double *z, const double *zlo, const double *sinth,
                              const double *sinlo, int lmax, int nmaps, const double *GQ,
                              const double *GU, double *gE, double *gB, int nthreads)
{
    if (nrings < 0 || lmax < 0 || nmaps < 1) return -1;
    const long long nalm = orc_nalm(lmax);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        long double *lp = (long double *)malloc(sizeof(long double) * (size_t)(lmax + 1));
        long double *lm = (long double *)malloc(sizeof(long double) * (size_t)(lmax + 1));
        long double *acc = (long double *)malloc(sizeof(long double) * 4 * (size_t)(lmax + 1) * nmaps);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int m = 0; m <= lmax; ++m) {
            memset(acc, 0, sizeof(long double) * 4 * (size_t)(lmax + 1) * nmaps);
            for (int k = 0; k < nrings; ++k) {
                const dd zk = {z[k], zlo[k]}, sk = {sinth[k], sinlo[k]};
                spin_lambda_eval(2, m, lmax, zk, sk, lp);
                spin_lambda_eval(-2, m, lmax, zk, sk, lm);
                for (int b = 0; b < nmaps; ++b) {
                    const double *q = GQ + 2 * (((size_t)b * nrings + k) * (lmax + 1) + m);
                    const double *u = GU + 2 * (((size_t)b * nrings + k) * (lmax + 1) + m);
                    long double *ab = acc + 4 * (size_t)b * (lmax + 1);
                    for (int l = m; l <= lmax; ++l) {
                        const long double Fp = 0.5L * (lp[l] + lm[l]), Fm = 0.5L * (lp[l] - lm[l]);
                        /* -F+ GQ - i F- GU  and  i F- GQ - F+ GU */
                        ab[4 * l + 0] += -Fp * q[0] + Fm * u[1];
                        ab[4 * l + 1] += -Fp * q[1] - Fm * u[0];
                        ab[4 * l + 2] += -Fm * q[1] - Fp * u[0];
                        ab[4 * l + 3] += Fm * q[0] - Fp * u[1];
                    }
                }
            }
            const long double c = m == 0 ? 1.0L : 2.0L;
            for (int b = 0; b < nmaps; ++b) {
                const long double *ab = acc + 4 * (size_t)b * (lmax + 1);
                for (int l = m; l <= lmax; ++l) {
                    const long long idx = alm_index(lmax, l, m);
                    double *e = gE + 2 * ((size_t)nalm * b + idx), *bb = gB + 2 * ((size_t)nalm * b + idx);
                    e[0] = (double)(c * ab[4 * l + 0]);
                    e[1] = m ? (double)(c * ab[4 * l + 1]) : 0.0;
                    bb[0] = (double)(c * ab[4 * l + 2]);
                    bb[1] = m ? (double)(c * ab[4 * l + 3]) : 0.0;
                }
            }
        }
        free(lp);
        free(lm);
        free(acc);
    }
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
