// Device bodies of the ring stage (Eq. sh-baseline, Eq. tau): complex
// helpers, the radix-4 and Bluestein FFTs in shared memory and the per-ring
// synthesis used by the ring kernels of shtb_phi.cu (the persistent batch
// kernel keeps its own copies, shtb_batch_items.cuh).
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

// e^{i pi n / J} for any integer n >= 0 from the half-circle table T (n < J)
__device__ __forceinline__ double2 ring_root(const double2 *__restrict__ T, int J, long long n)
{
    long long k = n % (2LL * J);
    if (k < J) return __ldg(T + k);
    double2 t = __ldg(T + (k - J));
    return make_double2(-t.x, -t.y);
}

// G_r = sum over m = r (mod J), |m| <= L, of (-1)^{s t} q_m  (m = r + tJ)
template <bool CG>
__device__ __forceinline__ double2 ldq(const double2 *p)
{
    return CG ? __ldcg(p) : __ldg(p);
}

template <class QAt>
__device__ double2 fold_G(QAt qat, int L, int J, int s, int r)
{
    double2 acc = make_double2(0.0, 0.0);
    int t = 0;
    for (int m = r; m <= L; m += J, ++t) {
        double2 v = qat(m);
        if (s & t & 1) { v.x = -v.x; v.y = -v.y; }
        acc = cadd(acc, v);
    }
    for (int tt = 1;; ++tt) {           // m = r - tt J < 0: q_m = conj(q_{-m})
        const int mp = tt * J - r;
        if (mp > L) break;
        double2 v = cconj(qat(mp));
        if (s & tt & 1) { v.x = -v.x; v.y = -v.y; }
        acc = cadd(acc, v);
    }
    return acc;
}

__device__ __forceinline__ double2 times_mi(double2 a) { return make_double2(a.y, -a.x); }

__device__ __forceinline__ int ilog2(int m)
{
    return 31 - __clz(m);
}

// Decimation in time, positive exponent: bit-reversed in, natural out.
// Radix-4 passes, each fusing the radix-2 stages of half-size h and 2h: with
// t1 = W^{2j} b, t2 = W^{j} c, t3 = W^{3j} d (W the 4h-th root),
//   a' = (a+t1) + (t2+t3),  b' = (a-t1) + i (t2-t3),
//   c' = (a+t1) - (t2+t3),  d' = (a-t1) - i (t2-t3);
// an odd number of stages starts with one twiddle-free radix-2 pass.
static __device__ void fft_dit_inverse(double2 *x, int M, const double2 *__restrict__ W, int Wlen)
{
    int h = 1;
    if (ilog2(M) & 1) {
        __syncthreads();
        for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
            const double2 u = x[2 * b], v = x[2 * b + 1];
            x[2 * b] = cadd(u, v);
            x[2 * b + 1] = csub(u, v);
        }
        h = 2;
    }
    for (; h < M; h *= 4) {
        __syncthreads();
        const int S = Wlen / (4 * h);
        for (int b = threadIdx.x; b < M / 4; b += blockDim.x) {
            const int j = b % h;
            const int base = (b - j) * 4 + j;
            const double2 a = x[base];
            const double2 t1 = cmul(__ldg(W + (size_t)2 * j * S), x[base + h]);
            const double2 t2 = cmul(__ldg(W + (size_t)j * S), x[base + 2 * h]);
            const double2 t3 = cmul(__ldg(W + (size_t)3 * j * S), x[base + 3 * h]);
            const double2 p = cadd(a, t1), m = csub(a, t1);
            const double2 sp = cadd(t2, t3), sm = times_i(csub(t2, t3));
            x[base] = cadd(p, sp);
            x[base + h] = cadd(m, sm);
            x[base + 2 * h] = csub(p, sp);
            x[base + 3 * h] = csub(m, sm);
        }
    }
    __syncthreads();
}

// Decimation in frequency, negative exponent: natural in, bit-reversed out.
// Radix-4 passes fusing the stages of half-size H and H/2 (w = conj of the
// 2H-th root): with s0 = a+c, s1 = a-c, s2 = b+d, s3 = b-d,
//   a' = s0+s2,  b' = (s0-s2) w^{2j},  c' = (s1 - i s3) w^{j},  d' = (s1 + i s3) w^{3j};
// an odd number of stages ends with one twiddle-free radix-2 pass.
static __device__ void fft_dif_forward(double2 *x, int M, const double2 *__restrict__ W, int Wlen)
{
    int H = M / 2;
    for (; H >= 2; H /= 4) {
        __syncthreads();
        const int S = Wlen / (2 * H), Q = H / 2;
        for (int b = threadIdx.x; b < M / 4; b += blockDim.x) {
            const int j = b % Q;
            const int base = (b - j) * 4 + j;
            const double2 a = x[base], bb = x[base + Q], c = x[base + H], d = x[base + H + Q];
            const double2 s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(bb, d), s3 = csub(bb, d);
            x[base] = cadd(s0, s2);
            x[base + Q] = cmul_conj(csub(s0, s2), __ldg(W + (size_t)2 * j * S));
            x[base + H] = cmul_conj(cadd(s1, times_mi(s3)), __ldg(W + (size_t)j * S));
            x[base + H + Q] = cmul_conj(cadd(s1, times_i(s3)), __ldg(W + (size_t)3 * j * S));
        }
    }
    if (H == 1) {
        __syncthreads();
        for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
            const double2 u = x[2 * b], v = x[2 * b + 1];
            x[2 * b] = cadd(u, v);
            x[2 * b + 1] = csub(u, v);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int bitrev(int k, int logn)
{
    return logn == 0 ? 0 : (int)(__brev((unsigned)k) >> (32 - logn));
}

// x[0..K) holds the input; computes x[n] = sum_k x_k e^{2 pi i k n / K} in
// place for n < K (x must hold M entries).  T is the ring's e^{i pi n/J}
// table with J = 2K, so the chirp c_j = e^{i pi j^2 / K} = T-root(2 j^2).
static __device__ void bluestein_inverse(double2 *x, int K, int M, const double2 *__restrict__ T,
                                  const double2 *__restrict__ fb, const double2 *__restrict__ W,
                                  int Wlen)
{
    const int J = 2 * K;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        if (k < K) x[k] = cmul(x[k], ring_root(T, J, 2LL * k * k));
        else x[k] = make_double2(0.0, 0.0);
    }
    fft_dif_forward(x, M, W, Wlen);
    for (int k = threadIdx.x; k < M; k += blockDim.x) x[k] = cmul(x[k], __ldg(fb + k));
    fft_dit_inverse(x, M, W, Wlen);
    for (int n = threadIdx.x; n < K; n += blockDim.x) x[n] = cmul(x[n], ring_root(T, J, 2LL * n * n));
    __syncthreads();
}

// Pixels of one ring from its q_m (m = 0..L): fold (Eq. tau), pack the
// Hermitian spectrum into a half-length complex FFT, transform, and write
// f_{2n}, f_{2n+1} as the real and imaginary parts of z_n.  All threads of
// the block take part; sm holds K (power of two) or M (Bluestein) entries.
template <bool BLUE, class QAt>
__device__ void phi_synth_ring_at(const PlanView &v, int ring, QAt qat, double *out_ring, double2 *sm)
{
    const int L = v.lmax;
    const int J = v.ring_J[ring], K = J / 2, s = v.ring_s[ring];
    const double2 *__restrict__ T = v.tw + v.ring_tw[ring];
    int logK = 0;
    while ((1 << logK) < K) ++logK;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double2 g0 = fold_G(qat, L, J, s, k);
        double2 g1 = fold_G(qat, L, J, s, k + K);
        if (s) g1 = times_i(g1);                           // e^{i pi K s / J} = i^s
        const double2 E = cadd(g0, g1), O = csub(g0, g1);
        double2 Zk = cadd(E, times_i(cmul(ring_root(T, J, 2LL * k), O)));
        if (s) Zk = cmul(Zk, ring_root(T, J, k));          // common factor e^{i pi k s / J}
        if (BLUE) sm[k] = Zk;
        else sm[bitrev(k, logK)] = Zk;
    }
    if (BLUE) {
        __syncthreads();
        bluestein_inverse(sm, K, v.ring_M[ring], T, v.fb + v.ring_fb[ring], v.W, v.Wlen);
    } else {
        fft_dit_inverse(sm, K, v.W, v.Wlen);
    }
    double2 *out = reinterpret_cast<double2 *>(out_ring);
    for (int n = threadIdx.x; n < K; n += blockDim.x) out[n] = sm[n];
    __syncthreads();
}

// ... with q_m read from a ring-major array qr[m]
template <bool BLUE, bool CG>
__device__ void phi_synth_ring(const PlanView &v, int ring, const double2 *qr, double *out_ring,
                               double2 *sm)
{
    phi_synth_ring_at<BLUE>(v, ring, [qr](int m) { return ldq<CG>(qr + m); }, out_ring, sm);
}

// ... with q_m formed from the two parity halves of the butterfly output,
// stored map-major: qt[((b * 2 + t) * nhalf + r) * (L + 1) + m] (complex);
// north rings (ring < nhalf) take q^0 + q^1, their mirrors q^0 - q^1.
template <bool BLUE, bool CG>
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
        const double2 x1 = ldq<CG>(q1 + m);
        return north ? make_double2(x0.x + x1.x, x0.y + x1.y) : make_double2(x0.x - x1.x, x0.y - x1.y);
    };
    phi_synth_ring_at<BLUE>(v, ring, qat, out_ring, sm);
}

}  // namespace shtb_dev
