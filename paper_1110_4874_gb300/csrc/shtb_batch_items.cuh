// Item bodies of the persistent batch kernel (shtb_batch.cu).  The batch
// keeps its own copies of the butterfly and ring-stage bodies in the layout it
// was validated with on the GPU: q^t entry-major ([entry][2 x maps]), a parity
// combine pass into ring-major q (Eq. q-even-odd2), radix-2 FFTs and the
// pointer form of the Eq. tau fold.  The stand-alone stage kernels use the
// map-major q^t bodies of shtb_bf_items.cuh / shtb_phi_items.cuh.  All data
// produced earlier in the same launch is read through L2 only (CG = true,
// ld.global.cg): L1 is not coherent between SMs within one launch.
#pragma once

#include <cuda_runtime.h>

#include "shtb_butterfly.h"
#include "shtb_internal.h"

namespace shtb_bdev {

// Warp tiling of a (rows x C) output with C = 2 x maps real components: the
// components are cut into groups of CPL, each group taken by LD lanes, and
// each lane owns RPL rows, so all 32 lanes are busy for any row count >= LD
// and a lane carries only RPL x CPL accumulators.
template <int C>
struct Tile {
    static constexpr int CPL = C >= 4 ? 4 : C;   // components per lane
    static constexpr int NG = C / CPL;           // component groups
    static constexpr int LD = 32 / NG;           // lanes per group
    static constexpr int RPL = 2;                // rows per lane
    static constexpr int CH = LD * RPL;          // rows per pass
};

template <bool CG>
__device__ __forceinline__ double ldp(const double *p)
{
    return CG ? __ldcg(p) : __ldg(p);
}

__device__ __forceinline__ long long alm_off(int L, int m)
{
    return (long long)m * (2 * L + 1 - m) / 2 + m;
}

// u = R^T a over one residual block (lane tile over the block's k columns).
// ai: [idx][nmaps] complex, the group's maps at b0 .. b0+NB-1.
template <int NB, bool CG>
__device__ __forceinline__ void bf_r_item(const BfRItem &it, int L, const int *__restrict__ ints,
                                          const double *__restrict__ dbl, const double2 *ai, int nmaps,
                                          int b0, double *ubuf, double *qt, int lane)
{
    constexpr int C = 2 * NB;
    using Tl = Tile<C>;
    const double *__restrict__ R = dbl + it.data_off;
    const long long aoff = alm_off(L, it.m) + it.t;   // chain row j at aoff + 2j
    const int sl = lane % Tl::LD, cg = lane / Tl::LD;
    for (int s0 = 0; s0 < it.k; s0 += Tl::CH) {
        double acc[Tl::RPL][Tl::CPL];
#pragma unroll
        for (int r = 0; r < Tl::RPL; ++r)
#pragma unroll
            for (int c = 0; c < Tl::CPL; ++c) acc[r][c] = 0.0;
        for (int j = 0; j < it.nrows; ++j) {
            const double *aj = reinterpret_cast<const double *>(
                ai + (size_t)(aoff + 2 * (it.j0 + j)) * nmaps + b0) + cg * Tl::CPL;
            double av[Tl::CPL];
#pragma unroll
            for (int c = 0; c < Tl::CPL; ++c) av[c] = ldp<CG>(aj + c);
#pragma unroll
            for (int r = 0; r < Tl::RPL; ++r) {
                const int sidx = s0 + sl + r * Tl::LD;
                const double t = sidx < it.k ? R[(size_t)j * it.k + sidx] : 0.0;
#pragma unroll
                for (int c = 0; c < Tl::CPL; ++c) acc[r][c] = fma(t, av[c], acc[r][c]);
            }
        }
#pragma unroll
        for (int r = 0; r < Tl::RPL; ++r) {
            const int sidx = s0 + sl + r * Tl::LD;
            if (sidx >= it.k) continue;
            double *dst = it.to_rings ? qt + (size_t)ints[it.out_off + sidx] * C
                                      : ubuf + (size_t)(it.out_off + sidx) * C;
#pragma unroll
            for (int c = 0; c < Tl::CPL; ++c) dst[cg * Tl::CPL + c] = acc[r][c];
        }
    }
}

// One level item: v = T_top^T u_top + T_bot^T u_bot over the shared
// candidate list, written to the parent level's u (or to q^t at level 1).
// out: this warp's shared-memory scratch of kMaxCand x C doubles.
template <int NB, bool CG>
__device__ __forceinline__ void bf_level_item(const BfItem &it, const int *__restrict__ ints,
                                              const double *__restrict__ dbl, const double *uin,
                                              double *uout, double *qt, double *out, int lane)
{
    constexpr int C = 2 * NB;
    using Tl = Tile<C>;
    for (int i = lane; i < it.nc * C; i += 32) out[i] = 0.0;
    __syncwarp();
    // dense parts of both children as one list of nd0 + nd1 rows (LD rows per
    // pass), each row a k-long dot product with its child's u; the top child's
    // rows are added before the bottom child's, so two rows that hit the same
    // candidate never update it at the same time
    const int dl = lane % Tl::LD, cg = lane / Tl::LD;
    const int nd0 = it.nd[0], ndt = it.nd[0] + it.nd[1];
    const int kmax = max(it.k[0], it.k[1]);
    for (int q0 = 0; q0 < ndt; q0 += Tl::LD) {
        const int q = q0 + dl;
        const bool valid = q < ndt;
        const int s = (valid && q >= nd0) ? 1 : 0;
        const int d = s ? q - nd0 : (valid ? q : 0);
        const int k = s ? it.k[1] : it.k[0], nd = s ? it.nd[1] : it.nd[0];
        const double *u = uin + (size_t)(s ? it.u_off[1] : it.u_off[0]) * C + cg * Tl::CPL;
        const double *__restrict__ T = dbl + (s ? it.T_off[1] : it.T_off[0]) + d;
        double acc[Tl::CPL];
#pragma unroll
        for (int c = 0; c < Tl::CPL; ++c) acc[c] = 0.0;
        for (int i = 0; i < kmax; ++i) {
            const bool live = valid && i < k;
            const double t = live ? T[(size_t)i * nd] : 0.0;
            const double *ui = u + (size_t)(live ? i : 0) * C;
#pragma unroll
            for (int c = 0; c < Tl::CPL; ++c) acc[c] = fma(t, ldp<CG>(ui + c), acc[c]);
        }
        double *o = out + (valid ? ints[(s ? it.dpos_off[1] : it.dpos_off[0]) + d] : 0) * C + cg * Tl::CPL;
        if (valid && s == 0) {
#pragma unroll
            for (int c = 0; c < Tl::CPL; ++c) o[c] += acc[c];
        }
        __syncwarp();
        if (valid && s == 1) {
#pragma unroll
            for (int c = 0; c < Tl::CPL; ++c) o[c] += acc[c];
        }
        __syncwarp();
    }
    // identity parts: out[skeleton position] += u (top child, then bottom)
    for (int s = 0; s < 2; ++s) {
        const int k = s ? it.k[1] : it.k[0];
        const double *u = uin + (size_t)(s ? it.u_off[1] : it.u_off[0]) * C;
        const int *__restrict__ ipos = ints + (s ? it.ipos_off[1] : it.ipos_off[0]);
        for (int i = lane; i < k; i += 32) {
            double *o = out + ipos[i] * C;
            const double *ui = u + (size_t)i * C;
#pragma unroll
            for (int c = 0; c < C; ++c) o[c] += ldp<CG>(ui + c);
        }
        __syncwarp();
    }
    if (it.to_rings) {
        const int *__restrict__ ent = ints + it.out_off;
        for (int i = lane; i < it.nc * C; i += 32) {
            const int cpos = i / C, c = i - cpos * C;
            qt[(size_t)ent[cpos] * C + c] = out[i];
        }
    } else {
        double *dst = uout + (size_t)it.out_off * C;
        for (int i = lane; i < it.nc * C; i += 32) dst[i] = out[i];
    }
    __syncwarp();
}

// q[b][ring][m] of order m for half-rings r = r0, r0 + rs, ...: north ring r
// gets q^0 + q^1, its mirror q^0 - q^1 (Eq. q-even-odd2); q_of(b) gives map
// b's q base ([nrings][L+1] complex).
template <int NB, bool CG, class QOf>
__device__ __forceinline__ void bf_combine_m(int m, int L, int Z, int nrings, const double *qt,
                                             QOf q_of, int r0, int rs)
{
    constexpr int C = 2 * NB;
    const bool odd = m + 1 <= L;    // chain t = 1 exists
    for (int r = r0; r < Z; r += rs) {
        const double *e0 = qt + ((size_t)(m * 2 + 0) * Z + r) * C;
        const double *e1 = qt + ((size_t)(m * 2 + 1) * Z + r) * C;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const double x0 = ldp<CG>(e0 + 2 * b), y0 = ldp<CG>(e0 + 2 * b + 1);
            const double x1 = odd ? ldp<CG>(e1 + 2 * b) : 0.0, y1 = odd ? ldp<CG>(e1 + 2 * b + 1) : 0.0;
            double2 *qb = q_of(b);
            qb[(size_t)r * (L + 1) + m] = make_double2(x0 + x1, y0 + y1);
            if (r < Z - 1) qb[(size_t)(nrings - 1 - r) * (L + 1) + m] = make_double2(x0 - x1, y0 - y1);
        }
    }
}

// ---------------------------------------------------------------- ring stage

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

}  // namespace shtb_bdev
