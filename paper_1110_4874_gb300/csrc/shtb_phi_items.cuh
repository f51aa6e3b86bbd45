// Device bodies of the ring stage (Eq. sh-baseline, Eq. tau): complex
// helpers, the mixed-radix and Bluestein FFTs in shared memory and the
// per-ring synthesis used by the ring kernels of shtb_phi.cu and by the
// persistent batch kernel of shtb_batch.cu.
#pragma once

#include <cuda_runtime.h>

#include "shtb_internal.h"

namespace shtb_dev {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul_conj(double2 a, double2 b)   // a * conj(b)
{
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ double2 times_i(double2 a) { return make_double2(-a.y, a.x); }

// sign flips as integer operations on the sign bit (no FP64 instruction)
__device__ __forceinline__ double dneg_if(double x, int neg)
{
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)(neg & 1) << 63));
}
__device__ __forceinline__ double2 cneg_if(double2 a, int neg)
{
    return make_double2(dneg_if(a.x, neg), dneg_if(a.y, neg));
}
__device__ __forceinline__ double2 cconj_i(double2 a) { return make_double2(a.x, dneg_if(a.y, 1)); }

// e^{i pi n / J} for any integer n >= 0 from the half-circle table T (n < J)
__device__ __forceinline__ double2 ring_root(const double2 *__restrict__ T, int J, long long n)
{
    long long k = n % (2LL * J);
    if (k < J) return __ldg(T + k);
    double2 t = __ldg(T + (k - J));
    return make_double2(-t.x, -t.y);
}

// ... for 0 <= n < 2^31, in 32-bit integer arithmetic
__device__ __forceinline__ double2 ring_root32(const double2 *__restrict__ T, int J, int n)
{
    const int k = n % (2 * J);
    if (k < J) return __ldg(T + k);
    return cneg_if(__ldg(T + (k - J)), 1);
}

template <bool CG>
__device__ __forceinline__ double2 ldq(const double2 *p)
{
    return CG ? __ldcg(p) : __ldg(p);
}

// G_r = sum over m = r (mod J), |m| <= L, of (-1)^{s t} q_m (m = r + tJ),
// with q_m = conj(q_{-m}) for m < 0.  The first term starts the sum (no add
// to zero) and the signs are flipped bitwise, so every FP64 instruction here
// is one of the sum's additions.
template <class QAt>
__device__ __forceinline__ double2 fold_G(QAt qat, int L, int J, int s, int r)
{
    double2 acc;
    int mp, tt;                         // negative terms m = -mp, mp = tt J - r
    if (r <= L) {
        acc = qat(r);
        int t = 1;
        for (int m = r + J; m <= L; m += J, ++t) acc = cadd(acc, cneg_if(qat(m), s & t));
        mp = J - r;
        tt = 1;
    } else {
        mp = J - r;                     // r in (L, J): only negative terms
        if (mp > L) return make_double2(0.0, 0.0);
        acc = cneg_if(cconj_i(qat(mp)), s);
        mp += J;
        tt = 2;
    }
    for (; mp <= L; mp += J, ++tt) acc = cadd(acc, cneg_if(cconj_i(qat(mp)), s & tt));
    return acc;
}

// ------------------------------------------------ mixed-radix ring FFTs
// A transform of length N = r_0 r_1 ... r_{n-1} (radices 2, 3, 4, 5, 7, 11,
// 13; list rl = {n, r_0, .., r_{n-1}}) runs in place in shared memory in n
// passes.  Pass i works on blocks of B_i = N / (r_0 .. r_{i-1}) points and
// combines the r_i points base + q N_i (N_i = B_i / r_i, q < r_i) of each of
// its B_i / r_i butterflies.  Decimation in frequency (exponent -1, passes
// 0..n-1: radix-r DFT, then the twiddles w_{B_i}^{-p j}) takes natural order
// to "position" order, in which X_k, k = p_0 + r_0 (p_1 + r_1 (p_2 + ..)),
// sits at pos(k) = sum_i p_i N_i.  Decimation in time (exponent +1, passes
// n-1..0, twiddles first) is its conjugate transpose: position order in,
// natural order out, unnormalised.  So no permutation pass is ever needed:
// the fold writes straight to pos(k), and a Bluestein filter is stored in
// position order.

// e^{2 pi i k / R} for the odd radices, k < R: R = 3, 5, 7, 11, 13 at offsets
// 0, 3, 8, 15, 26
static __constant__ double kRootCos[39] = {
    1.00000000000000000e+00, -5.00000000000000000e-01, -5.00000000000000000e-01,
    1.00000000000000000e+00, 3.09016994374947451e-01, -8.09016994374947451e-01, -8.09016994374947451e-01,
    3.09016994374947451e-01,
    1.00000000000000000e+00, 6.23489801858733483e-01, -2.22520933956314393e-01, -9.00968867902419146e-01,
    -9.00968867902419146e-01, -2.22520933956314393e-01, 6.23489801858733483e-01,
    1.00000000000000000e+00, 8.41253532831181206e-01, 4.15415013001886435e-01, -1.42314838273285144e-01,
    -6.54860733945285101e-01, -9.59492973614497369e-01, -9.59492973614497369e-01, -6.54860733945285101e-01,
    -1.42314838273285144e-01, 4.15415013001886435e-01, 8.41253532831181206e-01,
    1.00000000000000000e+00, 8.85456025653209911e-01, 5.68064746731155812e-01, 1.20536680255323048e-01,
    -3.54604887042535621e-01, -7.48510748171101081e-01, -9.70941817426052012e-01, -9.70941817426052012e-01,
    -7.48510748171101081e-01, -3.54604887042535621e-01, 1.20536680255323048e-01, 5.68064746731155812e-01,
    8.85456025653209911e-01};
static __constant__ double kRootSin[39] = {
    0.00000000000000000e+00, 8.66025403784438597e-01, -8.66025403784438597e-01,
    0.00000000000000000e+00, 9.51056516295153531e-01, 5.87785252292473137e-01, -5.87785252292473137e-01,
    -9.51056516295153531e-01,
    0.00000000000000000e+00, 7.81831482468029804e-01, 9.74927912181823619e-01, 4.33883739117558120e-01,
    -4.33883739117558120e-01, -9.74927912181823619e-01, -7.81831482468029804e-01,
    0.00000000000000000e+00, 5.40640817455597555e-01, 9.09631995354518330e-01, 9.89821441880932684e-01,
    7.55749574354258269e-01, 2.81732556841429671e-01, -2.81732556841429671e-01, -7.55749574354258269e-01,
    -9.89821441880932684e-01, -9.09631995354518330e-01, -5.40640817455597555e-01,
    0.00000000000000000e+00, 4.64723172043768562e-01, 8.22983865893656352e-01, 9.92708874098053973e-01,
    9.35016242685414833e-01, 6.63122658240795193e-01, 2.39315664287557767e-01, -2.39315664287557767e-01,
    -6.63122658240795193e-01, -9.35016242685414833e-01, -9.92708874098053973e-01, -8.22983865893656352e-01,
    -4.64723172043768562e-01};

template <int R>
__device__ __forceinline__ constexpr int root_off()
{
    return R == 3 ? 0 : R == 5 ? 3 : R == 7 ? 8 : R == 11 ? 15 : 26;
}

// y_q = sum_p a_p e^{S 2 pi i p q / R}, in place (S = +1 or -1)
template <int R, int S>
__device__ __forceinline__ void dft_small(double2 (&a)[R])
{
    if constexpr (R == 2) {
        const double2 u = a[0];
        a[0] = cadd(u, a[1]);
        a[1] = csub(u, a[1]);
    } else if constexpr (R == 4) {
        const double2 s0 = cadd(a[0], a[2]), s1 = csub(a[0], a[2]);
        const double2 s2 = cadd(a[1], a[3]), d = csub(a[1], a[3]);
        const double2 s3 = S > 0 ? times_i(d) : make_double2(d.y, -d.x);   // S i (a1 - a3)
        a[0] = cadd(s0, s2);
        a[1] = cadd(s1, s3);
        a[2] = csub(s0, s2);
        a[3] = csub(s1, s3);
    } else {
        // odd R: pair p with R - p, y_q = A_q + S i B_q, y_{R-q} = A_q - S i B_q
        constexpr int H = (R - 1) / 2, O = root_off<R>();
        double2 sp[H], dp[H];
#pragma unroll
        for (int p = 1; p <= H; ++p) {
            sp[p - 1] = cadd(a[p], a[R - p]);
            dp[p - 1] = csub(a[p], a[R - p]);
        }
        const double2 a0 = a[0];
        double2 y0 = a0;
#pragma unroll
        for (int p = 0; p < H; ++p) y0 = cadd(y0, sp[p]);
#pragma unroll
        for (int q = 1; q <= H; ++q) {
            double2 A = a0, B = make_double2(0.0, 0.0);
#pragma unroll
            for (int p = 1; p <= H; ++p) {
                const double c = kRootCos[O + (p * q) % R], sn = kRootSin[O + (p * q) % R];
                A.x = fma(sp[p - 1].x, c, A.x);
                A.y = fma(sp[p - 1].y, c, A.y);
                B.x = fma(dp[p - 1].x, sn, B.x);
                B.y = fma(dp[p - 1].y, sn, B.y);
            }
            const double2 iB = S > 0 ? make_double2(-B.y, B.x) : make_double2(B.y, -B.x);
            a[q] = cadd(A, iB);
            a[R - q] = csub(A, iB);
        }
        a[0] = y0;
    }
}

// s = a + w b, d = a - w b as s and 2a - s: six FP64 instructions (four
// fused multiply-adds, two for d) instead of a complex product and two sums
__device__ __forceinline__ void bfly_fma(double2 a, double2 b, double2 w, double2 &s, double2 &d)
{
    s.x = fma(w.x, b.x, fma(-w.y, b.y, a.x));
    s.y = fma(w.x, b.y, fma(w.y, b.x, a.y));
    d.x = fma(2.0, a.x, -s.x);
    d.y = fma(2.0, a.y, -s.y);
}

// one pass of radix R over Ntot points: back-to-back sequences of Nseq
// points (Nseq a multiple of B), in blocks of B; tw(t) = e^{2 pi i t / Nseq}
template <int R, bool INV, class TW>
__device__ __forceinline__ void mx_pass(double2 *x, int Ntot, int Nseq, int B, const TW &tw)
{
    const int Ns = B / R, step = Nseq / B;
    if constexpr (INV) {
        if (Ns == 1) {
            // the first pass of decimation in time: every twiddle is 1, so
            // only the R-point DFT remains (16 adds for radix 4, not 24 FMAs)
            for (int t = threadIdx.x; t < Ntot / R; t += blockDim.x) {
                double2 a[R];
#pragma unroll
                for (int q = 0; q < R; ++q) a[q] = x[t * R + q];
                dft_small<R, 1>(a);
#pragma unroll
                for (int q = 0; q < R; ++q) x[t * R + q] = a[q];
            }
            return;
        }
    }
    for (int t = threadIdx.x; t < Ntot / R; t += blockDim.x) {
        const int j = t % Ns, base = (t - j) * R + j;
        double2 a[R];
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = x[base + q * Ns];
        if constexpr (INV && R == 2) {
            // y_0,1 = a_0 +- w a_1, w = w_B^j
            double2 y0, y1;
            bfly_fma(a[0], a[1], tw(j * step), y0, y1);
            a[0] = y0;
            a[1] = y1;
        } else if constexpr (INV && R == 4) {
            // twiddles w_B^{pj} then the 4-point DFT (exponent +1), as two
            // layers of fused radix-2 butterflies: u0 = a0 +- w2 a2,
            // u1 = a1 +- w2 a3 (w2 = w_B^{2j}), then y_0,2 = u0+ +- w1 u1+,
            // y_1,3 = u0- +- i w1 u1- (w1 = w_B^j)
            const double2 w1 = tw(j * step), w2 = tw(2 * j * step);
            double2 u0p, u0m, u1p, u1m;
            bfly_fma(a[0], a[2], w2, u0p, u0m);
            bfly_fma(a[1], a[3], w2, u1p, u1m);
            bfly_fma(u0p, u1p, w1, a[0], a[2]);
            bfly_fma(u0m, u1m, make_double2(-w1.y, w1.x), a[1], a[3]);
        } else if (INV) {
            if (j) {
#pragma unroll
                for (int p = 1; p < R; ++p) a[p] = cmul(a[p], tw(p * j * step));
            }
            dft_small<R, 1>(a);
        } else {
            dft_small<R, -1>(a);
            if (j) {
#pragma unroll
                for (int p = 1; p < R; ++p) a[p] = cmul_conj(a[p], tw(p * j * step));
            }
        }
#pragma unroll
        for (int q = 0; q < R; ++q) x[base + q * Ns] = a[q];
    }
}

// Rader pass context: the ring's prime tables, and shared-memory scratch
// for its convolutions ((N / p) (p - 1) points after the N of the ring)
struct RaderCtx {
    const RaderInfo *ri;
    const int *rad;
    const int *ints;
    const double2 *dbl;
    double2 *scratch;
};

template <bool CONJ>
__device__ void rader_pass(double2 *x, int N, const RaderCtx &c);

// BIG: the radix-11 and radix-13 butterflies are compiled in (they need many
// more registers; only lengths with those factors are run with BIG); RADER:
// a radix above 13 is a prime done by Rader's algorithm (BIG kernels only)
template <bool INV, bool BIG, bool RADER, class TW>
__device__ __forceinline__ void mx_pass_any(int r, double2 *x, int Ntot, int Nseq, int B, const TW &tw,
                                            const RaderCtx *rc)
{
    switch (r) {
    case 4: mx_pass<4, INV>(x, Ntot, Nseq, B, tw); break;
    case 2: mx_pass<2, INV>(x, Ntot, Nseq, B, tw); break;
    case 3: mx_pass<3, INV>(x, Ntot, Nseq, B, tw); break;
    case 5: mx_pass<5, INV>(x, Ntot, Nseq, B, tw); break;
    case 7: mx_pass<7, INV>(x, Ntot, Nseq, B, tw); break;
    default:
        if constexpr (BIG) {
            if (r == 11) mx_pass<11, INV>(x, Ntot, Nseq, B, tw);
            else if (r == 13) mx_pass<13, INV>(x, Ntot, Nseq, B, tw);
            else if constexpr (RADER) rader_pass<!INV>(x, Ntot, *rc);
        }
        break;
    }
}

// natural order in, position order out, exponent -1; Ntot / Nseq
// sequences of Nseq points transformed side by side
template <bool BIG, bool RADER, class TW>
__device__ void fft_mx_dif(double2 *x, int Ntot, int Nseq, const int *__restrict__ rl, const TW &tw,
                           const RaderCtx *rc = nullptr)
{
    const int n = rl[0];
    int B = Nseq;
    for (int i = 0; i < n; ++i) {
        const int r = rl[1 + i];
        __syncthreads();
        mx_pass_any<false, BIG, RADER>(r, x, Ntot, Nseq, B, tw, rc);
        B /= r;
    }
    __syncthreads();
}

// position order in, natural order out, exponent +1 (unnormalised)
template <bool BIG, bool RADER, class TW>
__device__ void fft_mx_dit(double2 *x, int Ntot, int Nseq, const int *__restrict__ rl, const TW &tw,
                           const RaderCtx *rc = nullptr)
{
    const int n = rl[0];
    int B = 1;
    for (int i = n - 1; i >= 0; --i) {
        const int r = rl[1 + i];
        B *= r;
        __syncthreads();
        mx_pass_any<true, BIG, RADER>(r, x, Ntot, Nseq, B, tw, rc);
    }
    __syncthreads();
}

// ring transform kinds: direct mixed radix over 2, 3, 4, 5, 7; Bluestein
// (7-smooth convolution length); direct with radix 11 or 13 among the
// radices, or with one prime above 13 done by Rader's algorithm
enum RingFft { kDirect = 0, kBluestein = 1, kDirectBig = 2 };

// position of X_k in position order
__device__ __forceinline__ int fft_pos(int k, int N, const int *__restrict__ rl)
{
    const int n = rl[0];
    int pos = 0, Nc = N;
    for (int i = 0; i < n; ++i) {
        const int r = rl[1 + i];
        Nc /= r;
        pos += (k % r) * Nc;
        k /= r;
    }
    return pos;
}

// e^{2 pi i t / K} (t < K) from the ring's half-circle table of J = 2K roots
struct TwRing {
    const double2 *T;
    int J;
    __device__ __forceinline__ double2 operator()(int t) const
    {
        const int n = 4 * t;             // e^{2 pi i t / K} = e^{i pi 4t / J}, 4t < 2J
        if (n < J) return __ldg(T + n);
        const double2 u = __ldg(T + (n - J));
        return make_double2(-u.x, -u.y);
    }
};

// e^{2 pi i t / M} (t < M) from a table of M roots
struct TwTable {
    const double2 *R;
    __device__ __forceinline__ double2 operator()(int t) const { return __ldg(R + t); }
};

// x[0..K) holds the input; computes x[n] = sum_k x_k e^{2 pi i k n / K} in
// place for n < K through Bluestein's chirp transform: a cyclic convolution
// of length M (smooth, >= 2K - 1) with the chirp filter, stored transformed
// in position order and scaled by 1/M.  x must hold M entries.  T is the
// ring's e^{i pi n/J} table (J = 2K): the chirp c_j = e^{i pi j^2 / K} is
// the root of index 2 j^2 mod 2J.  PRECHIRP = false: the input already
// carries its chirp c_k (the synthesis fold weights include it).
template <bool PRECHIRP>
__device__ void bluestein_mx(double2 *x, int K, int M, const double2 *__restrict__ T,
                             const double2 *__restrict__ fb, const int *__restrict__ rl, const TwTable &tw)
{
    const int J = 2 * K;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        if (k >= K) x[k] = make_double2(0.0, 0.0);
        else if (PRECHIRP) x[k] = cmul(x[k], ring_root32(T, J, 2 * k * k));
    }
    fft_mx_dif<false, false>(x, M, M, rl, tw);
    for (int k = threadIdx.x; k < M; k += blockDim.x) x[k] = cmul(x[k], __ldg(fb + k));
    fft_mx_dit<false, false>(x, M, M, rl, tw);
    for (int n = threadIdx.x; n < K; n += blockDim.x) x[n] = cmul(x[n], ring_root32(T, J, 2 * n * n));
    __syncthreads();
}

// Rader's algorithm for the p-point DFTs of one pass over N points (blocks
// of p contiguous points, no twiddles: the pass is the first of decimation
// in time, or the last of decimation in frequency).  With g a primitive
// root mod p, y_{g^w} = a_0 + sum_v a_{g^{-v}} e^{2 pi i g^{w-v} / p}: a
// cyclic convolution of alpha_v = a_{g^{-v}} with beta_t = e^{2 pi i g^t / p},
// done as forward transform, product with the stored transform of beta
// (scaled by 1/(p-1)), inverse transform, all of length p - 1 and side by
// side for the N / p blocks in the scratch.  a_0 joins every output through
// the product's zero frequency, and y_0 = a_0 + (sum of alpha) is that
// frequency before the product.  Exponent +1; CONJ = true gives exponent -1
// as conj(DFT(conj a)).  Barriers: the transform's passes sync before they
// start and after they end; the caller syncs before the next pass.
template <bool CONJ>
__device__ void rader_pass(double2 *x, int N, const RaderCtx &c)
{
    const RaderInfo ri = *c.ri;
    const int p = ri.p, n = ri.n, tot = (N / p) * n;
    const int *__restrict__ ga = c.ints + ri.ga;
    const int *__restrict__ gi = c.ints + ri.gi;
    const double2 *__restrict__ G = c.dbl + ri.G;
    const int *__restrict__ rl = c.rad + ri.rl;
    const TwTable tw{c.dbl + ri.tw};
    double2 *S = c.scratch;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int b = e / n, v = e - b * n;
        const double2 a = x[b * p + __ldg(gi + v)];
        S[e] = CONJ ? cconj_i(a) : a;
    }
    fft_mx_dif<true, false>(S, tot, n, rl, tw);
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int b = e / n, v = e - b * n;
        const double2 A = S[e];
        double2 C = cmul(A, __ldg(G + v));
        if (v == 0) {
            const double2 a0 = CONJ ? cconj_i(x[b * p]) : x[b * p];
            const double2 y0 = cadd(a0, A);
            x[b * p] = CONJ ? cconj_i(y0) : y0;
            C = cadd(C, a0);
        }
        S[e] = C;
    }
    fft_mx_dit<true, false>(S, tot, n, rl, tw);
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int b = e / n, w = e - b * n;
        const double2 y = S[e];
        x[b * p + __ldg(ga + w)] = CONJ ? cconj_i(y) : y;
    }
}

// The Rader context of a ring of a BIG kernel (nullptr for other rings):
// its scratch follows the ring's K points in shared memory.
__device__ __forceinline__ const RaderCtx *rader_ctx(const PlanView &v, int ring, int K, double2 *sm, RaderCtx &rc)
{
    const int ri = v.ring_rdr[ring];
    if (ri < 0) return nullptr;
    rc = RaderCtx{v.rdr + ri, v.rad, v.rdr_int, v.rdr_dbl, sm + K};
    return &rc;
}

// Pixels of one ring from its q_m (m = 0..L): fold (Eq. tau) and pack the
// Hermitian spectrum into a half-length complex FFT in one step,
// Z_k = G_k A_k + G_{k+K} B_k (8 FP64 instructions per k; the plan's fold
// weights A, B hold the phi_0 phase, the packing twiddle and, on Bluestein
// rings, the chirp), transform, and write f_{2n}, f_{2n+1} as the real and
// imaginary parts of z_n.  All threads of the block take part; sm holds K
// (direct), K plus the Rader scratch, or M (Bluestein) entries.
template <int KIND, class QAt>
__device__ void phi_synth_ring_at(const PlanView &v, int ring, QAt qat, double *out_ring, double2 *sm)
{
    constexpr bool BLUE = KIND == kBluestein, BIG = KIND == kDirectBig;
    const int L = v.lmax;
    const int J = v.ring_J[ring], K = J / 2, s = v.ring_s[ring];
    const double2 *__restrict__ T = v.tw + v.ring_tw[ring];
    const double2 *__restrict__ AB = v.ab + v.ring_ab[ring];
    const int *__restrict__ rl = v.rad + v.ring_rad[ring];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double2 G0 = fold_G(qat, L, J, s, k);
        const double2 G1 = fold_G(qat, L, J, s, k + K);
        const double2 A = __ldg(AB + 2 * k), B = __ldg(AB + 2 * k + 1);
        double2 Z;
        Z.x = fma(G0.x, A.x, fma(-G0.y, A.y, fma(G1.x, B.x, -(G1.y * B.y))));
        Z.y = fma(G0.x, A.y, fma(G0.y, A.x, fma(G1.x, B.y, G1.y * B.x)));
        if (BLUE) sm[k] = Z;
        else sm[fft_pos(k, K, rl)] = Z;
    }
    if constexpr (BLUE) {
        __syncthreads();
        bluestein_mx<false>(sm, K, v.ring_mx[ring], T, v.mfb + v.ring_mfb[ring], rl,
                            TwTable{v.mtw + v.ring_mtw[ring]});
    } else {
        RaderCtx rc;
        const RaderCtx *rcp = BIG ? rader_ctx(v, ring, K, sm, rc) : nullptr;
        fft_mx_dit<BIG, BIG>(sm, K, K, rl, TwRing{T, J}, rcp);
    }
    double2 *out = reinterpret_cast<double2 *>(out_ring);
    for (int n = threadIdx.x; n < K; n += blockDim.x) out[n] = sm[n];
    __syncthreads();
}

// ... with q_m read from a ring-major array qr[m]
template <int KIND, bool CG>
__device__ void phi_synth_ring(const PlanView &v, int ring, const double2 *qr, double *out_ring,
                               double2 *sm)
{
    phi_synth_ring_at<KIND>(v, ring, [qr](int m) { return ldq<CG>(qr + m); }, out_ring, sm);
}

// ... with q_m formed from the two parity halves of the butterfly output,
// stored map-major: qt[((b * 2 + t) * nhalf + r) * (L + 1) + m] (complex);
// north rings (ring < nhalf) take q^0 + q^1, their mirrors q^0 - q^1.
template <int KIND, bool CG>
__device__ void phi_synth_ring_qt(const PlanView &v, int ring, const double2 *qt, int b,
                                  double *out_ring, double2 *sm)
{
    const int Z = v.nhalf, L = v.lmax;
    const bool north = ring < Z;
    const int r = north ? ring : v.nrings - 1 - ring;
    const double2 *q0 = qt + ((size_t)(b * 2) * Z + r) * (L + 1);
    const double2 *q1 = q0 + (size_t)Z * (L + 1);
    auto qat = [=](int m) {
        const double2 x0 = ldq<CG>(q0 + m);
        if (m + 1 > L) return x0;
        return cadd(x0, cneg_if(ldq<CG>(q1 + m), !north));
    };
    phi_synth_ring_at<KIND>(v, ring, qat, out_ring, sm);
}

}  // namespace shtb_dev
