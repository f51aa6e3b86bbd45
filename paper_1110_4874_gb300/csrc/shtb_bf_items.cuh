// Per-work-item device bodies of the butterfly synthesis (Sec. 3.2) used by
// the stage kernels of shtb_butterfly.cu (the persistent batch kernel keeps
// its own copies, shtb_batch_items.cuh).  CG = true reads data through L2
// only (ld.global.cg), for data produced earlier in the same launch: L1 is
// not coherent between SMs within one launch.
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

// q^t of a map group is stored map-major as complex values:
// qt[((b * 2 + t) * nhalf + r) * (L + 1) + m], so the ring stage reads each
// map's q_m of one ring contiguously in m.  Leaf outputs are addressed by the
// entry e = (m * 2 + t) * nhalf + r; this writes the C = 2 NB components of e.
__device__ __forceinline__ void qt_store(double *qt, long long e, int nhalf, int L, int c, double v)
{
    const long long mt = e / nhalf, r = e - mt * nhalf;
    const long long m = mt >> 1, t = mt & 1;
    const int b = c >> 1;
    qt[((((long long)b * 2 + t) * nhalf + r) * (L + 1) + m) * 2 + (c & 1)] = v;
}

// u = R^T a over one residual block (lane tile over the block's k columns).
// ai: [idx][nmaps] complex, the group's maps at b0 .. b0+NB-1.
template <int NB, bool CG>
__device__ __forceinline__ void bf_r_item(const BfRItem &it, int L, int nhalf, const int *__restrict__ ints,
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
#pragma unroll 2
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
            if (it.to_rings) {
                const long long e = ints[it.out_off + sidx];
#pragma unroll
                for (int c = 0; c < Tl::CPL; ++c) qt_store(qt, e, nhalf, L, cg * Tl::CPL + c, acc[r][c]);
            } else {
                double *dst = ubuf + (size_t)(it.out_off + sidx) * C;
#pragma unroll
                for (int c = 0; c < Tl::CPL; ++c) dst[cg * Tl::CPL + c] = acc[r][c];
            }
        }
    }
}

// One level item: v = T_top^T u_top + T_bot^T u_bot over the shared
// candidate list, written to the parent level's u (or to q^t at level 1).
// out: this warp's shared-memory scratch of nc x (C + 1) doubles (the odd row
// stride spreads the lanes' rows over the banks).
template <int C>
__host__ __device__ constexpr int out_stride()
{
    return C + 1;
}

template <int NB, bool CG>
__device__ __forceinline__ void bf_level_item(const BfItem &it, int L, int nhalf, const int *__restrict__ ints,
                                              const double *__restrict__ dbl, const double *uin,
                                              double *uout, double *qt, double *out, int lane)
{
    constexpr int C = 2 * NB;
    constexpr int OS = out_stride<C>();
    using Tl = Tile<C>;
    for (int i = lane; i < it.nc * OS; i += 32) out[i] = 0.0;
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
#pragma unroll 4
        for (int i = 0; i < kmax; ++i) {
            const bool live = valid && i < k;
            const double t = live ? T[(size_t)i * nd] : 0.0;
            const double *ui = u + (size_t)(live ? i : 0) * C;
#pragma unroll
            for (int c = 0; c < Tl::CPL; ++c) acc[c] = fma(t, ldp<CG>(ui + c), acc[c]);
        }
        double *o = out + (valid ? ints[(s ? it.dpos_off[1] : it.dpos_off[0]) + d] : 0) * OS + cg * Tl::CPL;
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
            double *o = out + ipos[i] * OS;
            const double *ui = u + (size_t)i * C;
#pragma unroll
            for (int c = 0; c < C; ++c) o[c] += ldp<CG>(ui + c);
        }
        __syncwarp();
    }
    if (it.to_rings) {
        const int *__restrict__ ent = ints + it.out_off;
        for (int i = lane; i < it.nc * C; i += 32) {
            const int c = i / it.nc, cpos = i - c * it.nc;
            qt_store(qt, ent[cpos], nhalf, L, c, out[cpos * OS + c]);
        }
    } else {
        double *dst = uout + (size_t)it.out_off * C;
        for (int i = lane; i < it.nc * C; i += 32) {
            const int cpos = i / C, c = i - cpos * C;
            dst[i] = out[cpos * OS + c];
        }
    }
    __syncwarp();
}

}  // namespace shtb_dev
