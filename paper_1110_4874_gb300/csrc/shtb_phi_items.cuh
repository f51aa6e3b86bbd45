// Device bodies of the ring stage (Eq. sh-baseline, Eq. tau): complex
// helpers, the radix-2 and Bluestein FFTs in shared memory and the per-ring
// synthesis, shared by the stand-alone ring kernels (shtb_phi.cu) and the
// persistent batch kernel (shtb_batch.cu).
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
    return CG ? __ldcg(p) : *p;
}

template <bool CG>
__device__ double2 fold_G(const double2 *__restrict__ qr, int L, int J, int s, int r)
{
    double2 acc = make_double2(0.0, 0.0);
    int t = 0;
    for (int m = r; m <= L; m += J, ++t) {
        double2 v = ldq<CG>(qr + m);
        if (s & t & 1) { v.x = -v.x; v.y = -v.y; }
        acc = cadd(acc, v);
    }
    for (int tt = 1;; ++tt) {           // m = r - tt J < 0: q_m = conj(q_{-m})
        const int mp = tt * J - r;
        if (mp > L) break;
        double2 v = cconj(ldq<CG>(qr + mp));
        if (s & tt & 1) { v.x = -v.x; v.y = -v.y; }
        acc = cadd(acc, v);
    }
    return acc;
}

// radix-2 decimation in time, positive exponent: bit-reversed in, natural out
static __device__ void fft_dit_inverse(double2 *x, int M, const double2 *__restrict__ W, int Wlen)
{
    for (int half = 1; half < M; half <<= 1) {
        __syncthreads();
        const int stride = Wlen / (2 * half);
        for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
            const int j = b & (half - 1);
            const int i0 = ((b - j) << 1) + j, i1 = i0 + half;
            const double2 t = cmul(__ldg(W + (size_t)j * stride), x[i1]);
            const double2 u = x[i0];
            x[i0] = cadd(u, t);
            x[i1] = csub(u, t);
        }
    }
    __syncthreads();
}

// radix-2 decimation in frequency, negative exponent: natural in, bit-reversed out
static __device__ void fft_dif_forward(double2 *x, int M, const double2 *__restrict__ W, int Wlen)
{
    for (int half = M / 2; half >= 1; half >>= 1) {
        __syncthreads();
        const int stride = Wlen / (2 * half);
        for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
            const int j = b & (half - 1);
            const int i0 = ((b - j) << 1) + j, i1 = i0 + half;
            const double2 u = x[i0], w = x[i1];
            x[i0] = cadd(u, w);
            x[i1] = cmul_conj(csub(u, w), __ldg(W + (size_t)j * stride));
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
template <bool BLUE, bool CG>
__device__ void phi_synth_ring(const PlanView &v, int ring, const double2 *qr, double *out_ring,
                               double2 *sm)
{
    const int L = v.lmax;
    const int J = v.ring_J[ring], K = J / 2, s = v.ring_s[ring];
    const double2 *__restrict__ T = v.tw + v.ring_tw[ring];
    int logK = 0;
    while ((1 << logK) < K) ++logK;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double2 g0 = fold_G<CG>(qr, L, J, s, k);
        double2 g1 = fold_G<CG>(qr, L, J, s, k + K);
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

}  // namespace shtb_dev
