// Kernel (c): the ring stage of Eq. (sh-baseline) -- per iso-latitude ring,
// the phase shift and wrap of Eq. (tau) followed by a backward real FFT of
// the ring's length J (Eq. pad-and-wrap), and its exact adjoint.
//
// With phi_kj = pi (2j + s)/J (s = 0 or 1) and q_{-m} = conj(q_m),
//   f_j = sum_{r=0}^{J-1} g_r e^{2 pi i r j / J},
//   g_r = sum_{m = r mod J, |m| <= L} q_m e^{i pi m s / J}
//       = e^{i pi r s / J} sum_t (-1)^{s t} q_{r + tJ}.
// g is Hermitian, so the real FFT of length J = 2K is done as one complex FFT
// of length K: Z_k = E_k + i e^{2 pi i k/J} O_k with E_k = g_k + g_{k+K},
// O_k = g_k - g_{k+K}; then z_n = sum_k Z_k e^{2 pi i k n / K} holds the
// pixels as f_{2n} + i f_{2n+1}.
// One CTA per (ring, map); the ring's data live in shared memory.  K a power
// of two: in-place radix-2 FFT from bit-reversed input.  Otherwise Bluestein's
// chirp transform through a power-of-two convolution of length M >= 2K-1
// (decimation in frequency, pointwise product with a precomputed filter in
// bit-reversed order, decimation in time), so no permutation pass is needed.
#include <cuda_runtime.h>

#include "shtb_internal.h"

namespace {

constexpr int kPhiThreads = 256;

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
__device__ double2 fold_G(const double2 *__restrict__ qr, int L, int J, int s, int r)
{
    double2 acc = make_double2(0.0, 0.0);
    int t = 0;
    for (int m = r; m <= L; m += J, ++t) {
        double2 v = qr[m];
        if (s & t & 1) { v.x = -v.x; v.y = -v.y; }
        acc = cadd(acc, v);
    }
    for (int tt = 1;; ++tt) {           // m = r - tt J < 0: q_m = conj(q_{-m})
        const int mp = tt * J - r;
        if (mp > L) break;
        double2 v = cconj(qr[mp]);
        if (s & tt & 1) { v.x = -v.x; v.y = -v.y; }
        acc = cadd(acc, v);
    }
    return acc;
}

// radix-2 decimation in time, positive exponent: bit-reversed in, natural out
__device__ void fft_dit_inverse(double2 *x, int M, const double2 *__restrict__ W, int Wlen)
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
__device__ void fft_dif_forward(double2 *x, int M, const double2 *__restrict__ W, int Wlen)
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
__device__ void bluestein_inverse(double2 *x, int K, int M, const double2 *__restrict__ T,
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

template <bool BLUE>
__global__ void __launch_bounds__(kPhiThreads)
phi_synth_kernel(PlanView v, const int *__restrict__ rings, const double2 *__restrict__ q,
                 double *__restrict__ map)
{
    extern __shared__ double2 sm[];
    const int ring = rings[blockIdx.x];
    const int b = blockIdx.y;
    const int L = v.lmax;
    const int J = v.ring_J[ring], K = J / 2, s = v.ring_s[ring];
    const double2 *__restrict__ T = v.tw + v.ring_tw[ring];
    const double2 *__restrict__ qr = q + ((size_t)b * v.nrings + ring) * (L + 1);
    int logK = 0;
    while ((1 << logK) < K) ++logK;

    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double2 g0 = fold_G(qr, L, J, s, k);
        double2 g1 = fold_G(qr, L, J, s, k + K);
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
    double2 *out = reinterpret_cast<double2 *>(map + (size_t)b * v.npix + v.ring_start[ring]);
    for (int n = threadIdx.x; n < K; n += blockDim.x) out[n] = sm[n];
}

template <bool BLUE>
__global__ void __launch_bounds__(kPhiThreads)
phi_adjoint_kernel(PlanView v, const int *__restrict__ rings, const double *__restrict__ map,
                   double2 *__restrict__ qa)
{
    extern __shared__ double2 sm[];
    const int ring = rings[blockIdx.x];
    const int b = blockIdx.y;
    const int L = v.lmax;
    const int J = v.ring_J[ring], K = J / 2, s = v.ring_s[ring];
    const double2 *__restrict__ T = v.tw + v.ring_tw[ring];
    int logK = 0;
    while ((1 << logK) < K) ++logK;

    // z_n = f_{2n} + i f_{2n+1}; forward DFT Zf_k = sum_n z_n e^{-2 pi i k n/K}
    const double2 *in = reinterpret_cast<const double2 *>(map + (size_t)b * v.npix + v.ring_start[ring]);
    for (int n = threadIdx.x; n < K; n += blockDim.x) {
        const double2 z = in[n];
        sm[n] = BLUE ? cconj(z) : z;     // Bluestein: forward = conj(inverse(conj))
    }
    if (BLUE) {
        __syncthreads();
        bluestein_inverse(sm, K, v.ring_M[ring], T, v.fb + v.ring_fb[ring], v.W, v.Wlen);
        for (int n = threadIdx.x; n < K; n += blockDim.x) sm[n] = cconj(sm[n]);
        __syncthreads();
    } else {
        fft_dif_forward(sm, K, v.W, v.Wlen);   // bit-reversed order
    }

    // F_r = E'_r + e^{-2 pi i r/J} O'_r with E' = (Zf_r + conj Zf_{K-r})/2,
    // O' = (Zf_r - conj Zf_{K-r})/(2i), K-periodic; then
    // q_adj[m] = e^{-i pi m s / J} F_{m mod J}.
    double2 *outq = qa + ((size_t)b * v.nrings + ring) * (L + 1);
    for (int m = threadIdx.x; m <= L; m += blockDim.x) {
        const int r = m % J;
        const int rho = r < K ? r : r - K;
        const int rho2 = rho == 0 ? 0 : K - rho;
        const double2 A = BLUE ? sm[rho] : sm[bitrev(rho, logK)];
        const double2 B = cconj(BLUE ? sm[rho2] : sm[bitrev(rho2, logK)]);
        const double2 Ep = make_double2(0.5 * (A.x + B.x), 0.5 * (A.y + B.y));
        const double2 D = make_double2(0.5 * (A.x - B.x), 0.5 * (A.y - B.y));   // (A - B)/2
        const double2 Op = make_double2(D.y, -D.x);                             // D / i
        const double2 F = cadd(Ep, cmul_conj(Op, ring_root(T, J, 2LL * r)));
        outq[m] = s ? cmul_conj(F, ring_root(T, J, (long long)m)) : F;
    }
}

int launch_set(const shtb_plan_s *p, bool synth, const void *in, void *out, int nmaps,
               cudaStream_t st)
{
    if (!p->pow2_rings.empty()) {
        const size_t smem = sizeof(double2) * (size_t)p->max_K_pow2;
        const dim3 grid((unsigned)p->pow2_rings.size(), (unsigned)nmaps);
        if (synth) {
            SHTB_CUDA_TRY(cudaFuncSetAttribute(phi_synth_kernel<false>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            phi_synth_kernel<false><<<grid, kPhiThreads, smem, st>>>(
                p->view, p->d_pow2_rings, (const double2 *)in, (double *)out);
        } else {
            SHTB_CUDA_TRY(cudaFuncSetAttribute(phi_adjoint_kernel<false>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            phi_adjoint_kernel<false><<<grid, kPhiThreads, smem, st>>>(
                p->view, p->d_pow2_rings, (const double *)in, (double2 *)out);
        }
        SHTB_CUDA_TRY(cudaGetLastError());
        ++p->launches;
    }
    if (!p->blue_rings.empty()) {
        const size_t smem = sizeof(double2) * (size_t)p->max_M_blue;
        const dim3 grid((unsigned)p->blue_rings.size(), (unsigned)nmaps);
        if (synth) {
            SHTB_CUDA_TRY(cudaFuncSetAttribute(phi_synth_kernel<true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            phi_synth_kernel<true><<<grid, kPhiThreads, smem, st>>>(
                p->view, p->d_blue_rings, (const double2 *)in, (double *)out);
        } else {
            SHTB_CUDA_TRY(cudaFuncSetAttribute(phi_adjoint_kernel<true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            phi_adjoint_kernel<true><<<grid, kPhiThreads, smem, st>>>(
                p->view, p->d_blue_rings, (const double *)in, (double2 *)out);
        }
        SHTB_CUDA_TRY(cudaGetLastError());
        ++p->launches;
    }
    return SHTB_OK;
}

}  // namespace

int launch_phi_synth(const shtb_plan_s *p, const double2 *q, double *map, int nmaps, cudaStream_t st)
{
    return launch_set(p, true, q, map, nmaps, st);
}

int launch_phi_adjoint(const shtb_plan_s *p, const double *map, double2 *q, int nmaps,
                       cudaStream_t st)
{
    return launch_set(p, false, map, q, nmaps, st);
}
