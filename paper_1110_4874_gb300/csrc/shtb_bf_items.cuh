// Per-work-item device bodies of the butterfly synthesis (Sec. 3.2), shared
// by the stand-alone stage kernels (shtb_butterfly.cu) and the persistent
// batch kernel (shtb_batch.cu).  CG = true reads data produced earlier in the
// same launch through L2 only (ld.global.cg), as the persistent kernel must:
// L1 is not coherent between SMs within one launch.
#pragma once

#include <cuda_runtime.h>

#include "shtb_butterfly.h"

namespace shtb_dev {

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

}  // namespace shtb_dev
