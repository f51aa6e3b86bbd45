// Host-side plan builder: HEALPix ring geometry, the per-(l, m) constants of
// the rescaled jump-two Legendre recurrence, the recurrence start values past
// the 1e-30 crop, and the ring-FFT tables.  Everything is computed once per
// (nside, L) in double-double where rounding matters and uploaded to the
// device (Sec. 4.2: "the precomputation ... once"; Appendix, "Efficient code
// for Legendre transforms").
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <tuple>
#include <thread>
#include <vector>

#include "shtb_butterfly.h"
#include "shtb_dd.h"
#include "shtb_internal.h"
#include "shtb_plan_detail.h"

using shtb::DD;
using shtb::dd;
using shtb::HalfRing;
using shtb::kCrop;
using shtb::parallel_for;


// ------------------------------------------------------------ shared helpers
namespace shtb {

HalfRing half_ring(long long N, long long i)
{
    long long zn, zd, sn, sd, en;
    if (i < N) {
        zn = 3 * N * N - i * i;
        zd = 3 * N * N;
        sn = i * i * (6 * N * N - i * i);
        sd = 9 * N * N * N * N;
        en = i * i;                 // 1 - z = i^2 / (3N^2)
    } else {
        zn = 4 * N - 2 * i;
        zd = 3 * N;
        sn = (2 * i - N) * (7 * N - 2 * i);
        sd = 9 * N * N;
        en = 2 * i - N;             // 1 - z = (2i - N) / (3N)
    }
    HalfRing h;
    DD zq = dd((double)zn) / dd((double)zd);
    h.z = to_double(zq);
    h.z2 = to_double(ddmul((double)zn, (double)zn) / ddmul((double)zd, (double)zd));
    DD s2 = dd((double)sn) / dd((double)sd);
    h.s2 = to_double(s2);
    h.eps1 = to_double(dd((double)en) / dd((double)zd));
    h.sdd = sqrt(s2);
    return h;
}

// c_m = sqrt(1/(4 pi) prod_{i=1}^m (2i+1)/(2i)) as dd, m = 0..L
std::vector<DD> diag_norms(int L)
{
    std::vector<DD> out(L + 1);
    DD c2 = dd(1.0) / (DD{shtb::kPiHi, shtb::kPiLo} * 4.0);
    out[0] = shtb::sqrt(c2);
    for (int i = 1; i <= L; ++i) {
        c2 = c2 * (dd(2.0 * i + 1.0) / dd(2.0 * i));
        out[i] = shtb::sqrt(c2);
    }
    return out;
}

// x^m as (mantissa dd in [0.5,1), exponent) by binary powering
DD dd_pow(DD x, int m, int *E)
{
    auto norm = [](DD v, int *e) {
        int k;
        std::frexp(v.hi, &k);
        *e += k;
        return DD{std::ldexp(v.hi, -k), std::ldexp(v.lo, -k)};
    };
    DD r = dd(1.0), b = x;
    int er = 0, eb = 0;
    b = norm(b, &eb);
    while (m > 0) {
        if (m & 1) { r = r * b; er += eb; r = norm(r, &er); }
        m >>= 1;
        if (m) { b = b * b; eb *= 2; b = norm(b, &eb); }
    }
    *E = er;
    return r;
}

// b_l = sqrt((l^2 - m^2)/(4 l^2 - 1)) for l = m+1..L (index l - m) of the
// textbook one-step recurrence Ptilde_l = (z Ptilde_{l-1} - b_{l-1} Ptilde_{l-2}) / b_l
std::vector<double> one_step_coefs(int L, int m)
{
    std::vector<double> b(L - m + 2, 0.0);
    for (int l = m + 1; l <= L; ++l)
        b[l - m] = std::sqrt(((double)(l - m) * (double)(l + m)) /
                             ((double)(2 * l - 1) * (double)(2 * l + 1)));
    return b;
}


void legendre_column(int L, int m, const HalfRing &h, DD cm, const std::vector<double> &b,
                     double *out)
{
    const double sq = std::sqrt(2.0 * m + 3.0);
    const bool near_pole = h.z > 0.5;
    auto zmul = [&](double v) { return near_pole ? v - h.eps1 * v : h.z * v; };
    int E = 0;
    DD pm = dd_pow(h.sdd, m, &E) * cm;
    double P0 = to_double(pm);
    if (m & 1) P0 = -P0;
    auto emit = [&](int l, double Pm) {
        const double v = E == 0 ? Pm : std::ldexp(Pm, E);
        out[l - m] = std::fabs(v) >= kCrop ? v : 0.0;
    };
    emit(m, P0);
    if (m == L) return;
    double P1 = sq * zmul(P0);
    emit(m + 1, P1);
    for (int l = m + 2; l <= L; ++l) {
        double P2 = (zmul(P1) - b[l - 1 - m] * P0) / b[l - m];
        P0 = P1;
        P1 = P2;
        if (E != 0 && P1 != 0.0) {
            int k;
            std::frexp(P1, &k);
            if (k + E > -900) {
                P0 = std::ldexp(P0, E);
                P1 = std::ldexp(P1, E);
                E = 0;
            } else if (k > 600) {
                P0 = std::ldexp(P0, -512);
                P1 = std::ldexp(P1, -512);
                E += 512;
            }
        }
        emit(l, P1);
    }
}

// Spin-weighted s_lambda_lm (s = +-2) at one half-ring for l = m..L: the
// Wigner three-term recurrence in l for d^l_{m,-s} on the normalised
// functions s_lambda = (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s}:
//   l sqrt(((l+1)^2-m^2)((l+1)^2-s^2)) d^{l+1}
//     = (2l+1)(l(l+1) z + m s) d^l - (l+1) sqrt((l^2-m^2)(l^2-s^2)) d^{l-1},
// from l0 = max(m, 2).  Start values: for m >= 2, s_lambda_mm =
// Ptilde_m^m sqrt(m(m-1)/((m+1)(m+2))) tan(theta/2)^s (the closed form
// of d^m_{m,-s}, since sin^m = 2^m sin^m(theta/2) cos^m(theta/2)); for
// m = 0, 1 the l = 2 closed forms.  The same power-of-two exponent
// bookkeeping and 1e-30 crop as the scalar column.
void spin_column(int L, int m, int s, const HalfRing &h, DD cm, double *out)
{
    for (int l = m; l <= L; ++l) out[l - m] = 0.0;
    const int l0 = std::max(m, 2);
    if (l0 > L) return;
    const double z = h.z, st = to_double(h.sdd);
    const bool near_pole = h.z > 0.5;
    auto zmul = [&](double v) { return near_pole ? v - h.eps1 * v : z * v; };
    const double tan_half = st / (1.0 + z);            // tan(theta/2), z >= 0
    int E = 0;
    double V0;
    if (m >= 2) {
        DD pm = dd_pow(h.sdd, m, &E) * cm;             // |Ptilde_m^m| = c_m sin^m
        double v = to_double(pm) * std::sqrt((double)m * (m - 1) / ((double)(m + 1) * (m + 2)));
        v *= s > 0 ? tan_half * tan_half : 1.0 / (tan_half * tan_half);
        V0 = (m & 1) ? -v : v;                         // Condon-Shortley phase of Ptilde_m^m
    } else {
        const double c5 = std::sqrt(5.0 / (4.0 * shtb::kPiHi));
        const double sh = std::sqrt(0.5 * h.eps1), ch = std::sqrt(0.5 * (1.0 + z));   // half angles
        if (m == 0) V0 = c5 * std::sqrt(6.0) * sh * sh * ch * ch;
        else if (s > 0) V0 = -c5 * 2.0 * sh * sh * sh * ch;
        else V0 = c5 * 2.0 * sh * ch * ch * ch;
    }
    auto emit = [&](int l, double v) {
        const double x = E == 0 ? v : std::ldexp(v, E);
        out[l - m] = std::fabs(x) >= kCrop ? x : 0.0;
    };
    emit(l0, V0);
    double Vp = 0.0, V = V0;
    const double mm = (double)m * m, ss = (double)s * s;
    for (int l = l0; l < L; ++l) {
        const double dl = l;
        const double den = dl * std::sqrt(((dl + 1) * (dl + 1) - mm) * ((dl + 1) * (dl + 1) - ss));
        const double nrm = std::sqrt((2 * dl + 3) / (2 * dl + 1));
        const double a = nrm * (2 * dl + 1) / den;
        const double bcoef = l == l0 ? 0.0
                                     : nrm * (dl + 1) * std::sqrt((dl * dl - mm) * (dl * dl - ss)) *
                                           std::sqrt((2 * dl + 1) / (2 * dl - 1)) / den;
        const double Vn = a * (dl * (dl + 1) * zmul(V) + (double)m * s * V) - bcoef * Vp;
        Vp = V;
        V = Vn;
        if (E != 0 && V != 0.0) {
            int k;
            std::frexp(V, &k);
            if (k + E > -900) {
                Vp = std::ldexp(Vp, E);
                V = std::ldexp(V, E);
                E = 0;
            } else if (k > 600) {
                Vp = std::ldexp(Vp, -512);
                V = std::ldexp(V, -512);
                E += 512;
            }
        }
        emit(l + 1, V);
    }
}

}  // namespace shtb

using shtb::diag_norms;
using shtb::dd_pow;
using shtb::half_ring;
using shtb::one_step_coefs;

namespace {

// -------------------------------------------- cos/sin of rational angles
// (cos, sin)(pi * num / den) with the angle folded by integer symmetries
// into [0, pi/4] and evaluated from a double-double argument.
void sincospi_frac(long long num, long long den, double *c, double *s)
{
    long long twoden = 2 * den;
    long long q = ((num % twoden) + twoden) % twoden;   // angle pi q/den in [0, 2pi)
    double sc = 1.0, ss = 1.0;                          // signs for cos, sin
    if (q >= den) { q -= den; sc = -sc; ss = -ss; }     // theta - pi
    if (2 * q > den) { q = den - q; sc = -sc; }         // pi - theta
    // now angle = pi q / den in [0, pi/2]; swap to the complement above pi/4
    bool swap = 4 * q > den;
    long long n = swap ? den - 2 * q : q;               // angle' = pi n / d
    long long d = swap ? 2 * den : den;
    DD a = DD{shtb::kPiHi, shtb::kPiLo} * (double)n / dd((double)d);
    double ch = std::cos(a.hi), sh = std::sin(a.hi);
    double cv = ch - sh * a.lo, sv = sh + ch * a.lo;
    if (swap) std::swap(cv, sv);
    *c = sc * cv;
    *s = ss * sv;
}

// Radices of a mixed-radix transform of length n over 4, 2, 3, 5, 7, 11, 13
// (4s first, at most one 2); false if n has another prime factor.
bool radix_list(long long n, std::vector<int> &rl)
{
    rl.clear();
    if (n < 1) return false;
    int twos = 0;
    while (n % 2 == 0) { n /= 2; ++twos; }
    for (; twos >= 2; twos -= 2) rl.push_back(4);
    if (twos) rl.push_back(2);
    for (int pr : {3, 5, 7, 11, 13})
        while (n % pr == 0) { n /= pr; rl.push_back(pr); }
    return n == 1;
}

bool is_prime(long long n)
{
    if (n < 2) return false;
    for (long long d = 2; d * d <= n; ++d)
        if (n % d == 0) return false;
    return true;
}

// The prime p of Rader's algorithm for a transform of length K, or 0: K is
// p times a product of 2, 3, 5, 7, 11, 13 with p > 13 prime (once), and
// p - 1 factors over 2, 3, 5, 7, 11, 13, so that the cyclic convolution of
// length p - 1 is itself a mixed-radix transform.
long long rader_prime(long long K)
{
    long long n = K;
    for (int pr : {2, 3, 5, 7, 11, 13})
        while (n % pr == 0) n /= pr;
    std::vector<int> rl;
    if (n <= 13 || !is_prime(n) || !radix_list(n - 1, rl)) return 0;
    return n;
}

// smallest primitive root modulo the prime p
long long primitive_root(long long p)
{
    std::vector<long long> f;
    long long n = p - 1;
    for (long long d = 2; d * d <= n; ++d)
        if (n % d == 0) {
            f.push_back(d);
            while (n % d == 0) n /= d;
        }
    if (n > 1) f.push_back(n);
    auto powmod = [p](long long b, long long e) {
        long long r = 1;
        b %= p;
        for (; e; e >>= 1, b = b * b % p)
            if (e & 1) r = r * b % p;
        return r;
    };
    for (long long g = 2;; ++g) {
        bool ok = true;
        for (long long q : f)
            if (powmod(g, (p - 1) / q) == 1) { ok = false; break; }
        if (ok) return g;
    }
}

// smallest 7-smooth integer >= n
long long smooth_at_least(long long n)
{
    for (long long m = std::max(1LL, n);; ++m) {
        long long x = m;
        for (int pr : {2, 3, 5, 7})
            while (x % pr == 0) x /= pr;
        if (x == 1) return m;
    }
}

// In-place mixed-radix decimation in frequency with exponent -1 (the device
// kernels' pass structure): natural-order input, position-order output.
void mixed_dif_forward(std::vector<std::complex<double>> &x, const std::vector<int> &rl)
{
    const long long N = (long long)x.size();
    std::vector<std::complex<double>> w(N);          // e^{-2 pi i t / N}
    for (long long t = 0; t < N; ++t) {
        double c, sn;
        sincospi_frac(2 * t, N, &c, &sn);
        w[t] = {c, -sn};
    }
    long long B = N;
    std::vector<std::complex<double>> a, y;
    for (int r : rl) {
        const long long Ns = B / r, step = N / B, rs = N / r;
        a.resize(r);
        y.resize(r);
        for (long long b = 0; b < N; b += B) {
            for (long long j = 0; j < Ns; ++j) {
                for (int q = 0; q < r; ++q) a[q] = x[b + j + q * Ns];
                for (int p = 0; p < r; ++p) {
                    std::complex<double> acc = 0.0;
                    for (int q = 0; q < r; ++q) acc += a[q] * w[((p * q) % r) * rs];
                    y[p] = acc * w[p * j * step];
                }
                for (int p = 0; p < r; ++p) x[b + j + p * Ns] = y[p];
            }
        }
        B = Ns;
    }
}

// ------------------------------------------------ recurrence constants
// Jump-two recurrence of Eq. (three-term):
//   P_{l+2} = ((z^2 - d_l)/c_l) P_l - (c_{l-2}/c_l) P_{l-2}
//   c_l^m = sqrt((l-m+1)(l-m+2)(l+m+1)(l+m+2) / ((2l+1)(2l+3)^2(2l+5)))
//   d_l^m = (2l(l+1) - 2m^2 - 1) / ((2l-1)(2l+3))
// Rescaled by P_l = sigma_l V_l with sigma_{m+t} = sigma_{m+t+2} = 1 and
// sigma_{l+2} = sigma_{l-2} c_{l-2} / c_l, it becomes
//   V_{l+2} = mu_l (z^2 - d_l) V_l - V_{l-2},   mu_l = sigma_l / (c_{l-2} sigma_{l-2}),
// two FMAs per step: w = mu_l x + C, V_{l+2} = w V_l - V_{l-2} with
// (x, C) = (z^2, -mu_l d_l) or (-sin^2, mu_l (1 - d_l)).  The sin^2 form keeps
// the argument exact near the poles, where z^2 rounded to a double would
// move theta by up to 1e-10 relative at Nside = 2048.
DD c_coef(long long l, long long m)
{
    DD num = shtb::ddmul((double)((l - m + 1) * (l - m + 2)), (double)((l + m + 1) * (l + m + 2)));
    DD den = shtb::ddmul((double)((2 * l + 1) * (2 * l + 5)), (double)((2 * l + 3) * (2 * l + 3)));
    return shtb::sqrt(num / den);
}

DD d_coef(long long l, long long m)
{
    return dd((double)(2 * l * (l + 1) - 2 * m * m - 1)) / dd((double)((2 * l - 1) * (2 * l + 3)));
}

DD one_minus_d(long long l, long long m)
{
    return dd((double)(2 * (l * l + l - 1 + m * m))) / dd((double)((2 * l - 1) * (2 * l + 3)));
}

void build_coefficients(int L, int m, RecCoef *out /* indexed by l - m */)
{
    for (int t = 0; t < 2; ++t) {
        const int n = chain_len(L, m, t);
        if (n == 0) continue;
        // chain j: l_j = m + t + 2j
        std::vector<DD> c(n), sig(n);
        for (int j = 0; j < n; ++j) c[j] = c_coef(m + t + 2 * j, m);
        sig[0] = dd(1.0);
        if (n > 1) sig[1] = dd(1.0);
        for (int j = 1; j + 1 < n; ++j) sig[j + 1] = sig[j - 1] * c[j - 1] / c[j];
        for (int j = 0; j < n; ++j) {
            const int l = m + t + 2 * j;
            RecCoef e;
            e.sig = shtb::to_double(sig[j]);
            if (j >= 1) {
                DD mu = sig[j] / (c[j - 1] * sig[j - 1]);
                e.mu = shtb::to_double(mu);
                e.cz = shtb::to_double(-(mu * d_coef(l, m)));
                e.cs = shtb::to_double(mu * one_minus_d(l, m));
            } else {
                e.mu = e.cz = e.cs = 0.0;   // first element of a chain: no step starts there
            }
            out[l - m] = e;
        }
    }
}


// For order m at one half-ring: per parity t the first chain index js[t]
// with |Ptilde_{m+t+2j}^m| >= 1e-30 and the rescaled values V = Ptilde/sigma
// there and one chain step later (js[t] = chain length if none).  Found by
// the one-step recurrence in l from Ptilde_m^m = (-1)^m c_m sin^m(theta),
// with a separate power-of-two exponent so that nothing underflows; near the
// poles z*P is formed as P - (1-z) P so that 1 - z enters exactly.
void chain_starts(int L, int m, const HalfRing &h, DD cm, const std::vector<double> &b,
                  const RecCoef *cf, int js[2], double2 vs[2])
{
    const int n0 = chain_len(L, m, 0), n1 = chain_len(L, m, 1);
    const double sq = std::sqrt(2.0 * m + 3.0);
    const bool near_pole = h.z > 0.5;
    auto zmul = [&](double v) { return near_pole ? v - h.eps1 * v : h.z * v; };
    js[0] = js[1] = -1;
    double v0[2] = {0, 0}, v1[2] = {0, 0};
    bool res[2] = {n0 == 0, n1 == 0};   // chain resolved
    int E = 0;
    DD pm = dd_pow(h.sdd, m, &E) * cm;
    double P0 = shtb::to_double(pm);
    if (m & 1) P0 = -P0;
    double P1 = 0.0;
    auto visit = [&](int l, double Pm) {   // Pm: mantissa at exponent E
        const int t = (l - m) & 1;
        if (res[t]) return;
        const int j = (l - m - t) / 2;
        const double v = E == 0 ? Pm : std::ldexp(Pm, E);
        if (js[t] < 0) {
            if (std::fabs(v) >= kCrop) {
                js[t] = j;
                v0[t] = v;
                if (l + 2 > L) res[t] = true;
            }
        } else {                            // the chain's next element
            v1[t] = v;
            res[t] = true;
        }
    };
    visit(m, P0);
    if (m < L) {
        P1 = sq * zmul(P0);
        visit(m + 1, P1);
    }
    for (int l = m + 2; l <= L && !(res[0] && res[1]); ++l) {
        double P2 = (zmul(P1) - b[l - 1 - m] * P0) / b[l - m];
        P0 = P1;
        P1 = P2;
        if (E != 0 && P1 != 0.0) {
            int k;
            std::frexp(P1, &k);
            if (k + E > -900) {
                P0 = std::ldexp(P0, E);
                P1 = std::ldexp(P1, E);
                E = 0;
            } else if (k > 600) {
                P0 = std::ldexp(P0, -512);
                P1 = std::ldexp(P1, -512);
                E += 512;
            }
        }
        visit(l, P1);
    }
    for (int t = 0; t < 2; ++t) {
        const int nt = t == 0 ? n0 : n1;
        if (js[t] < 0 || nt == 0) {
            js[t] = nt;                          // nothing above the crop
            vs[t] = make_double2(0.0, 0.0);
        } else {
            const int l0 = m + t + 2 * js[t];
            const double s0 = cf[l0 - m].sig;
            const double s1 = l0 + 2 <= L ? cf[l0 + 2 - m].sig : 1.0;
            vs[t] = make_double2(v0[t] / s0, l0 + 2 <= L ? v1[t] / s1 : 0.0);
        }
    }
}

}  // namespace

// ------------------------------------------------------------------------
int plan_alloc_upload(shtb_plan_s *p, void **dst, const void *src, size_t bytes)
{
    void *d = nullptr;
    size_t nb = bytes ? bytes : 16;
    cudaError_t e = cudaMalloc(&d, nb);
    if (e != cudaSuccess)
        return shtb_fail(SHTB_ENOMEM, std::string("cudaMalloc plan table: ") + cudaGetErrorString(e));
    p->allocations.push_back(d);
    p->alloc_bytes.push_back(nb);
    if (src && bytes) {
        e = cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return shtb_fail(SHTB_ECUDA, std::string("cudaMemcpy plan table: ") + cudaGetErrorString(e));
    }
    p->stats.plan_device_bytes += (long long)nb;
    *dst = d;
    return SHTB_OK;
}

int shtb_build_dense_plan(shtb_plan_s *p)
{
    const int N = p->nside, L = p->lmax;
    const int nthreads = p->opts.nthreads;
    const int Z = 2 * N;   // rings with z >= 0, equator last
    p->nhalf = Z;
    p->nrings = 4 * N - 1;
    p->npix = 12LL * N * N;
    p->nalm = (long long)(L + 1) * (L + 2) / 2;

    // ---------------------------------------------------------- geometry
    std::vector<HalfRing> hr(Z);
    std::vector<double> xarg(Z);
    std::vector<int> xform(Z);
    for (int r = 0; r < Z; ++r) {
        hr[r] = half_ring(N, r + 1);
        if (hr[r].s2 < 0.5) { xarg[r] = -hr[r].s2; xform[r] = 1; }
        else { xarg[r] = hr[r].z2; xform[r] = 0; }
    }
    p->ring_J.resize(p->nrings);
    p->ring_s.resize(p->nrings);
    p->ring_start.resize(p->nrings);
    long long pix = 0;
    for (int r = 0; r < p->nrings; ++r) {
        long long i = r < Z ? r + 1 : 4LL * N - (r + 1);
        p->ring_J[r] = (int)(i < N ? 4 * i : 4LL * N);
        p->ring_s[r] = i < N ? 1 : (((i + N) % 2 == 0) ? 1 : 0);
        p->ring_start[r] = pix;
        pix += p->ring_J[r];
    }

    // --------------------------------------- recurrence constants (Eq. three-term)
    std::vector<RecCoef> coef((size_t)p->nalm);
    parallel_for(L + 1, nthreads, [&](int m) {
        build_coefficients(L, m, coef.data() + alm_index(L, m, m));
    });

    // --------------------------------------------- start values past the crop
    // For each (m, parity t, half-ring r): first chain index j with
    // |Ptilde_{m+t+2j}^m(z_r)| >= 1e-30 and the rescaled values V there and
    // one chain step later.  Found by the one-step recurrence in l from
    // Ptilde_m^m = (-1)^m c_m sin^m(theta), carried with a separate
    // power-of-two exponent so that nothing underflows.
    const std::vector<DD> cm = diag_norms(L);
    std::vector<int> jstart((size_t)(L + 1) * 2 * Z);
    std::vector<double2> vstart((size_t)(L + 1) * 2 * Z);
    parallel_for(L + 1, nthreads, [&](int m) {
        const std::vector<double> b = one_step_coefs(L, m);
        const RecCoef *cf = coef.data() + alm_index(L, m, m);
        for (int r = 0; r < Z; ++r) {
            int js[2];
            double2 vs[2];
            chain_starts(L, m, hr[r], cm[m], b, cf, js, vs);
            for (int t = 0; t < 2; ++t) {
                const size_t idx = ((size_t)m * 2 + t) * Z + r;
                jstart[idx] = js[t];
                vstart[idx] = vs[t];
            }
        }
    });

    // statistics of the recurrence work
    long long n_rec = 0, n_exec = 0;
    const int nchunk = (Z + 31) / 32;
    for (int m = 0; m <= L; ++m) {
        const int n0 = chain_len(L, m, 0), n1 = chain_len(L, m, 1);
        for (int c = 0; c < nchunk; ++c) {
            int jlo = n0;
            for (int r = c * 32; r < std::min(Z, c * 32 + 32); ++r) {
                for (int t = 0; t < 2; ++t) {
                    const int nt = t == 0 ? n0 : n1;
                    int j = jstart[((size_t)m * 2 + t) * Z + r];
                    n_rec += nt - j;
                    if (j < nt) jlo = std::min(jlo, j);
                }
            }
            if (jlo < n0) n_exec += 32LL * ((n0 - jlo) + std::max(0, n1 - jlo));
        }
    }
    p->stats.n_recurrence = n_rec;
    p->stats.n_recurrence_exec = n_exec;
    p->stats.recurrence_flops = 4.0 * (double)n_rec;
    p->stats.legendre_flops_per_map = 4.0 * (double)n_rec;

    // ------------------------------------------------------- ring FFT tables
    std::vector<long long> ring_tw(p->nrings);

    // e^{i pi n / J} tables, one per distinct J (north and south rings share)
    std::vector<double2> tw;
    std::vector<long long> tw_of_J(4 * N + 1, -1);
    for (int r = 0; r < p->nrings; ++r) {
        int J = p->ring_J[r];
        if (tw_of_J[J] < 0) {
            tw_of_J[J] = (long long)tw.size();
            for (int n = 0; n < J; ++n) {
                double c, s;
                sincospi_frac(n, J, &c, &s);
                tw.push_back(make_double2(c, s));
            }
        }
        ring_tw[r] = tw_of_J[J];
    }
    // Mixed-radix tables of the stand-alone ring kernels: K factoring over
    // 2, 3, 5, 7, 11, 13 -> direct transform of length K; otherwise Bluestein
    // through the smallest 7-smooth length M >= 2K - 1.
    std::vector<int> rad, ring_rad(p->nrings), ring_mx(p->nrings, 0), chunk_list;
    std::vector<long long> ring_mfb(p->nrings, 0), ring_mtw(p->nrings, 0);
    std::vector<double2> mfb, mtw;
    std::vector<int> ring_rdr(p->nrings, -1), ring_smem(p->nrings, 0), rdr_int;
    std::vector<RaderInfo> rdr;
    std::vector<double2> rdr_dbl;
    std::vector<long long> ring_ab(p->nrings, 0);
    std::vector<double2> ab;
    {
        std::map<long long, int> rad_of_len;
        std::map<long long, long long> mtw_of_len;
        std::vector<long long> mfb_of_J(4 * N + 1, -1);
        auto radix_off = [&](long long n) {
            auto it = rad_of_len.find(n);
            if (it != rad_of_len.end()) return it->second;
            std::vector<int> rl;
            radix_list(n, rl);
            const int off = (int)rad.size();
            rad.push_back((int)rl.size());
            rad.insert(rad.end(), rl.begin(), rl.end());
            rad_of_len[n] = off;
            return off;
        };
        std::vector<int> blue_J;
        p->direct_rings.clear();
        p->blue_rings.clear();
        p->big_rings.clear();
        p->max_K_direct = 0;
        p->max_M_mx = 0;
        p->max_K_big = 0;
        // Rader primes: per prime p its tables (generator powers, the
        // transformed convolution kernel, the length-(p-1) roots)
        std::map<long long, int> rdr_of_p;
        auto rader_off = [&](long long pr) {
            auto it = rdr_of_p.find(pr);
            if (it != rdr_of_p.end()) return it->second;
            RaderInfo ri{};
            ri.p = (int)pr;
            ri.n = (int)(pr - 1);
            ri.rl = radix_off(pr - 1);
            const long long g = primitive_root(pr);
            ri.ga = (int)rdr_int.size();
            std::vector<long long> gp(pr - 1);
            long long x = 1;
            for (long long v = 0; v < pr - 1; ++v, x = x * g % pr) gp[v] = x;
            for (long long v = 0; v < pr - 1; ++v) rdr_int.push_back((int)gp[v]);
            ri.gi = (int)rdr_int.size();
            for (long long v = 0; v < pr - 1; ++v) rdr_int.push_back((int)gp[(pr - 1 - v) % (pr - 1)]);
            // beta_t = e^{2 pi i g^t / p}, DIF-transformed (exponent -1,
            // position order) and scaled by 1/(p-1)
            std::vector<std::complex<double>> beta(pr - 1);
            for (long long t = 0; t < pr - 1; ++t) {
                double c, sn;
                sincospi_frac(2 * gp[t], pr, &c, &sn);
                beta[t] = {c, sn};
            }
            std::vector<int> rl;
            radix_list(pr - 1, rl);
            mixed_dif_forward(beta, rl);
            ri.G = (long long)rdr_dbl.size();
            for (long long t = 0; t < pr - 1; ++t)
                rdr_dbl.push_back(make_double2(beta[t].real() / (double)(pr - 1), beta[t].imag() / (double)(pr - 1)));
            ri.tw = (long long)rdr_dbl.size();
            for (long long t = 0; t < pr - 1; ++t) {
                double c, sn;
                sincospi_frac(2 * t, pr - 1, &c, &sn);
                rdr_dbl.push_back(make_double2(c, sn));
            }
            rdr.push_back(ri);
            return rdr_of_p[pr] = (int)rdr.size() - 1;
        };
        for (int r = 0; r < p->nrings; ++r) {
            const long long K = p->ring_J[r] / 2;
            std::vector<int> rl;
            const long long pr = radix_list(K, rl) ? 0 : rader_prime(K);
            if (pr) {
                // mixed radix over the smooth part, the Rader pass last in the
                // list (so first, untwiddled, in the synthesis transform)
                auto it = rad_of_len.find(K);
                if (it == rad_of_len.end()) {
                    radix_list(K / pr, rl);
                    rl.push_back((int)pr);
                    const int off = (int)rad.size();
                    rad.push_back((int)rl.size());
                    rad.insert(rad.end(), rl.begin(), rl.end());
                    it = rad_of_len.emplace(K, off).first;
                }
                ring_rad[r] = it->second;
                ring_rdr[r] = rader_off(pr);
                p->big_rings.push_back(r);
                const long long entries = K + (K / pr) * (pr - 1);
                ring_smem[r] = (int)entries;
                p->max_K_big = std::max<int>(p->max_K_big, (int)entries);
            } else if (radix_list(K, rl)) {
                ring_rad[r] = radix_off(K);
                const bool big = std::any_of(rl.begin(), rl.end(), [](int x) { return x > 7; });
                (big ? p->big_rings : p->direct_rings).push_back(r);
                int &mx = big ? p->max_K_big : p->max_K_direct;
                mx = std::max<int>(mx, (int)K);
                ring_smem[r] = (int)K;
            } else {
                const long long M = smooth_at_least(2 * K - 1);
                ring_mx[r] = (int)M;
                ring_smem[r] = (int)M;
                ring_rad[r] = radix_off(M);
                p->blue_rings.push_back(r);
                p->max_M_mx = std::max<long long>(p->max_M_mx, M);
                if (!mtw_of_len.count(M)) {
                    mtw_of_len[M] = (long long)mtw.size();
                    for (long long t = 0; t < M; ++t) {
                        double c, sn;
                        sincospi_frac(2 * t, M, &c, &sn);
                        mtw.push_back(make_double2(c, sn));
                    }
                }
                ring_mtw[r] = mtw_of_len[M];
                if (mfb_of_J[p->ring_J[r]] < 0) {
                    mfb_of_J[p->ring_J[r]] = 0;
                    blue_J.push_back(p->ring_J[r]);
                }
            }
        }
        if ((long long)std::max({p->max_K_direct, p->max_M_mx, p->max_K_big}) * 16 > 200 * 1024)
            return shtb_fail(SHTB_ENOTSUP, "ring FFT does not fit in shared memory (nside too large)");
        // Bluestein filters, one per distinct J: the DIF transform of
        // b_j = conj(c_j) (|j| < K, cyclic in M) in position order, / M
        std::vector<long long> off(blue_J.size());
        long long total = 0;
        for (size_t d = 0; d < blue_J.size(); ++d) {
            off[d] = total;
            mfb_of_J[blue_J[d]] = total;
            total += smooth_at_least(2 * (blue_J[d] / 2) - 1);
        }
        mfb.resize((size_t)total);
        parallel_for((int)blue_J.size(), nthreads, [&](int d) {
            const long long K = blue_J[d] / 2, M = smooth_at_least(2 * K - 1);
            std::vector<std::complex<double>> bv(M, 0.0);
            for (long long j = 0; j < K; ++j) {
                double c, sn;
                sincospi_frac((j * j) % (2 * K), K, &c, &sn);
                std::complex<double> b(c, -sn);
                bv[j] = b;
                if (j > 0) bv[M - j] = b;
            }
            std::vector<int> rl;
            radix_list(M, rl);
            mixed_dif_forward(bv, rl);
            for (long long k = 0; k < M; ++k)
                mfb[off[d] + k] = make_double2(bv[k].real() / M, bv[k].imag() / M);
        });
        for (int r : p->blue_rings) ring_mfb[r] = mfb_of_J[p->ring_J[r]];
        // Fold weights per distinct (J, s, Bluestein or not): with
        // G_r = sum_{m = r mod J, |m| <= L} (-1)^{s t} q_m (m = r + tJ),
        // g_r = e^{i pi r s / J} G_r, and Z_k = E_k + i e^{2 pi i k/J} O_k,
        // E, O = g_k +- g_{k+K}, one finds Z_k = G_k A_k + G_{k+K} B_k with
        //   A_k = e^{i pi a/J} + i e^{i pi b/J},  B_k = i^s (e^{i pi a/J} - i e^{i pi b/J}),
        //   a = k s, b = k (s + 2), both + 2 k^2 on Bluestein rings (the
        // chirp e^{i pi k^2 / K} of the convolution's input).  Each
        // exponential comes from an exact integer argument, so A and B are
        // within one rounding of exact.
        {
            std::map<std::tuple<int, int, int>, long long> ab_of;
            for (int r = 0; r < p->nrings; ++r) {
                const int J = p->ring_J[r], sr = p->ring_s[r], blue = ring_mx[r] ? 1 : 0;
                const auto key = std::make_tuple(J, sr, blue);
                auto it = ab_of.find(key);
                if (it == ab_of.end()) {
                    const long long off = (long long)ab.size();
                    const long long K = J / 2;
                    ab.resize(ab.size() + 2 * K);
                    for (long long k = 0; k < K; ++k) {
                        const long long ch = blue ? (2 * k * k) % (2LL * J) : 0;
                        double c1, s1, c2, s2;
                        sincospi_frac(k * sr + ch, J, &c1, &s1);
                        sincospi_frac(k * (sr + 2) + ch, J, &c2, &s2);
                        ab[off + 2 * k] = make_double2(c1 - s2, s1 + c2);
                        ab[off + 2 * k + 1] = sr ? make_double2(c2 - s1, c1 + s2) : make_double2(c1 + s2, s1 - c2);
                    }
                    it = ab_of.emplace(key, off).first;
                }
                ring_ab[r] = it->second;
            }
        }
        // heaviest rings first
        std::stable_sort(p->direct_rings.begin(), p->direct_rings.end(),
                         [&](int a, int b) { return p->ring_J[a] > p->ring_J[b]; });
        std::stable_sort(p->big_rings.begin(), p->big_rings.end(),
                         [&](int a, int b) { return ring_smem[a] > ring_smem[b]; });
        std::stable_sort(p->blue_rings.begin(), p->blue_rings.end(),
                         [&](int a, int b) { return ring_mx[a] > ring_mx[b]; });
        constexpr int kSmallM = shtb_plan_s::kBlueSmallM;
        p->blue_split = 0;
        while (p->blue_split < (int)p->blue_rings.size() && ring_mx[p->blue_rings[p->blue_split]] > kSmallM)
            ++p->blue_split;
        p->max_M_small = p->blue_split < (int)p->blue_rings.size() ? ring_mx[p->blue_rings[p->blue_split]] : 0;
        // chunks of consecutive rings with about equal pixel counts
        constexpr int NCH = shtb_plan_s::kPhiChunks;
        std::vector<int> chunk_of(p->nrings);
        {
            int c = 0;
            for (int r = 0; r < p->nrings; ++r) {
                while (c < NCH - 1 && p->ring_start[r] >= (c + 1) * p->npix / NCH) ++c;
                chunk_of[r] = c;
            }
            for (int cc = 0; cc <= NCH; ++cc) p->chunk_pix[cc] = cc == NCH ? p->npix : -1;
            for (int r = p->nrings - 1; r >= 0; --r) p->chunk_pix[chunk_of[r]] = p->ring_start[r];
            for (int cc = NCH - 1; cc >= 0; --cc)       // an empty chunk starts where the next one does
                if (p->chunk_pix[cc] < 0) p->chunk_pix[cc] = p->chunk_pix[cc + 1];
        }
        const std::vector<int> *lists[3] = {&p->direct_rings, &p->blue_rings, &p->big_rings};
        for (int cc = 0; cc < NCH; ++cc)
            for (int k = 0; k < 3; ++k) {
                auto &ck = p->chunk_kind[cc][k];
                ck.off = (int)chunk_list.size();
                ck.len = 0;
                ck.split = 0;
                ck.len_small = 0;
                for (int r : *lists[k])
                    if (chunk_of[r] == cc) {
                        chunk_list.push_back(r);
                        const int len = ring_smem[r];
                        ck.len = std::max(ck.len, len);
                        if (k == 1 && len <= kSmallM) ck.len_small = std::max(ck.len_small, len);
                        else ++ck.split;              // lists are sorted longest first
                    }
                ck.n = (int)chunk_list.size() - ck.off;
            }
    }

    // algorithmic FFT flops: 2.5 J log2 J per real ring transform of length J
    double phi_flops = 0.0;
    for (int r = 0; r < p->nrings; ++r)
        phi_flops += 2.5 * p->ring_J[r] * std::log2((double)p->ring_J[r]);
    p->stats.phi_flops_per_map = phi_flops;

    // --------------------------------------------------------------- upload
    PlanView &v = p->view;
    v.nside = N;
    v.lmax = L;
    v.nrings = p->nrings;
    v.nhalf = Z;
    v.npix = p->npix;
    v.nalm = p->nalm;
    int rc;
#define UP(field, vec)                                                                  \
    do {                                                                                \
        void *d_;                                                                       \
        rc = plan_alloc_upload(p, &d_, (vec).data(), sizeof((vec)[0]) * (vec).size());  \
        if (rc) return rc;                                                              \
        v.field = (decltype(v.field))d_;                                                \
    } while (0)
    UP(coef, coef);
    UP(xarg, xarg);
    UP(xform, xform);
    UP(jstart, jstart);
    UP(vstart, vstart);
    UP(ring_J, p->ring_J);
    UP(ring_s, p->ring_s);
    UP(ring_start, p->ring_start);
    UP(ring_tw, ring_tw);
    UP(tw, tw);
    UP(ring_rad, ring_rad);
    UP(rad, rad);
    UP(ring_mx, ring_mx);
    UP(ring_mfb, ring_mfb);
    UP(mfb, mfb);
    UP(ring_mtw, ring_mtw);
    UP(mtw, mtw);
    UP(ring_ab, ring_ab);
    UP(ab, ab);
    UP(ring_rdr, ring_rdr);
    if (rdr.empty()) rdr.push_back(RaderInfo{});          // non-empty uploads
    if (rdr_int.empty()) rdr_int.push_back(0);
    if (rdr_dbl.empty()) rdr_dbl.push_back(make_double2(0.0, 0.0));
    UP(rdr, rdr);
    UP(rdr_int, rdr_int);
    UP(rdr_dbl, rdr_dbl);
#undef UP
    void *d;
    rc = plan_alloc_upload(p, &d, p->direct_rings.data(), sizeof(int) * p->direct_rings.size());
    if (rc) return rc;
    p->d_direct_rings = (int *)d;
    rc = plan_alloc_upload(p, &d, p->blue_rings.data(), sizeof(int) * p->blue_rings.size());
    if (rc) return rc;
    p->d_blue_rings = (int *)d;
    rc = plan_alloc_upload(p, &d, p->big_rings.data(), sizeof(int) * p->big_rings.size());
    if (rc) return rc;
    p->d_big_rings = (int *)d;
    rc = plan_alloc_upload(p, &d, chunk_list.data(), sizeof(int) * chunk_list.size());
    if (rc) return rc;
    p->d_chunk_list = (int *)d;

    // bytes one call reads from the plan (Legendre tables + start values)
    p->stats.plan_read_bytes = (long long)(sizeof(RecCoef) * coef.size() + sizeof(int) * jstart.size() +
                                           sizeof(double2) * vstart.size());
    return SHTB_OK;
}

// ------------------------------------------------------------------------
// Private host-only check of the plan tables (no GPU): Ptilde_l^m at HEALPix
// half-ring r (0-based from the north pole) for l = m..lmax, evaluated with
// exactly the tables and the two-FMA step the kernels use.
extern "C" int shtb_test_host_recurrence(int nside, int lmax, int m, int r, double *out)
{
    if (nside < 1 || lmax < 0 || m < 0 || m > lmax || r < 0 || r >= 2 * nside || !out)
        return shtb_fail(SHTB_EINVAL, "bad arguments");
    const HalfRing h = half_ring(nside, r + 1);
    std::vector<RecCoef> cf(lmax - m + 1);
    build_coefficients(lmax, m, cf.data());
    const std::vector<DD> cm = diag_norms(lmax);
    const std::vector<double> b = one_step_coefs(lmax, m);
    int js[2];
    double2 vs[2];
    chain_starts(lmax, m, h, cm[m], b, cf.data(), js, vs);
    const bool sform = h.s2 < 0.5;
    const double x = sform ? -h.s2 : h.z2;
    for (int l = m; l <= lmax; ++l) out[l - m] = 0.0;
    for (int t = 0; t < 2; ++t) {
        const int n = chain_len(lmax, m, t);
        double cur = 0.0, prev = 0.0;
        for (int j = js[t]; j < n; ++j) {
            const int l = m + t + 2 * j;
            double nxt;
            if (j == js[t]) { cur = vs[t].x; nxt = vs[t].y; }
            else {
                const RecCoef &c = cf[l - m];
                const double w = std::fma(c.mu, x, sform ? c.cs : c.cz);
                nxt = std::fma(w, cur, -prev);
            }
            out[l - m] = cf[l - m].sig * cur;
            prev = cur;
            cur = nxt;
        }
    }
    return SHTB_OK;
}

// Private host-only check of regenerated residual blocks (no GPU): builds
// chain (m, t) of a compressed plan, then every residual block's R again from
// its per-column recurrence starts (the start records a residual_recurrence
// plan keeps, stepped as the kernel steps them, times sigma) and compares
// them with the stored blocks.  info[0..3] = {blocks, regenerated elements,
// elements that differ in the crop (one side zero), depth}; *max_rel = the
// largest |R_regen - R_stored| over the largest |R| of the block's column.
extern "C" int shtb_test_host_rec_blocks(int nside, int lmax, double eps, int m, int t, int leaf_cols,
                                         double *max_rel, long long *info)
{
    if (nside < 1 || lmax < 0 || m < 0 || m > lmax || t < 0 || t > 1 || !(eps > 0) || leaf_cols < 1 ||
        leaf_cols > shtb::kMaxCand || !max_rel || !info)
        return shtb_fail(SHTB_EINVAL, "bad arguments");
    const int Z = 2 * nside, n = chain_len(lmax, m, t);
    if (n < 1) return shtb_fail(SHTB_EINVAL, "empty chain");
    std::vector<HalfRing> hr(Z);
    for (int r = 0; r < Z; ++r) hr[r] = half_ring(nside, r + 1);
    const std::vector<DD> cm = diag_norms(lmax);
    std::vector<double> lam0, lam1;
    shtb::build_lambda(lmax, m, Z, hr, cm[m], lam0, lam1);
    shtb::BfParams prm;
    prm.eps = eps;
    prm.leaf_cols = leaf_cols;
    shtb::BfChain ch;
    int rc = shtb::compress_chain(t ? lam1.data() : lam0.data(), n, Z, prm, &ch);
    if (rc) return rc;
    std::vector<RecCoef> cf(lmax - m + 1);
    build_coefficients(lmax, m, cf.data());
    const std::vector<double> b = one_step_coefs(lmax, m);
    *max_rel = 0.0;
    long long nb = 0, ne = 0, ncrop = 0;
    for (const auto &rb : ch.rblocks) {
        ++nb;
        for (int s = 0; s < rb.k; ++s) {
            const int r = rb.cols[s];
            const HalfRing &h = hr[r];
            const bool sform = h.s2 < 0.5;
            const double x = sform ? -h.s2 : h.z2;
            int js[2];
            double2 vs[2];
            chain_starts(lmax, m, h, cm[m], b, cf.data(), js, vs);
            const RecStart st = shtb::block_column_start(n, t, rb.j0, rb.nrows, r, x, sform, cf.data(), js[t], vs[t]);
            double cmax = 0.0;
            for (int j = 0; j < rb.nrows; ++j) cmax = std::max(cmax, std::fabs(rb.data[(size_t)j * rb.k + s]));
            double cur = st.start == 0 ? st.v0 : 0.0, prev = 0.0;
            for (int j = 0; j < rb.nrows; ++j) {
                const int dl = t + 2 * (rb.j0 + j);
                const double regen = cf[dl].sig * cur, stored = rb.data[(size_t)j * rb.k + s];
                if ((regen == 0.0) != (stored == 0.0)) ++ncrop;
                if (cmax > 0) *max_rel = std::max(*max_rel, std::fabs(regen - stored) / cmax);
                ++ne;
                const RecCoef &c = cf[dl];
                const double w = std::fma(c.mu, x, sform ? c.cs : c.cz);
                double nxt = std::fma(w, cur, -prev);
                if (j == st.start) nxt = st.v1;
                if (j + 1 == st.start) nxt = st.v0;
                prev = cur;
                cur = nxt;
            }
        }
    }
    info[0] = nb;
    info[1] = ne;
    info[2] = ncrop;
    info[3] = ch.depth;
    return SHTB_OK;
}

// s_lambda_lm (s = +-2) at half-ring r (0-based from the north pole) for
// l = m..lmax, as the plan builder of spin plans computes it.
extern "C" int shtb_test_host_spin_column(int nside, int lmax, int m, int s, int r, double *out)
{
    if (nside < 1 || lmax < 0 || m < 0 || m > lmax || (s != 2 && s != -2) || r < 0 || r >= 2 * nside || !out)
        return shtb_fail(SHTB_EINVAL, "bad arguments");
    const HalfRing h = half_ring(nside, r + 1);
    const std::vector<DD> cm = diag_norms(lmax);
    shtb::spin_column(lmax, m, s, h, cm[m], out);
    return SHTB_OK;
}
