// Per-work-item device bodies of the butterfly synthesis (Sec. 3.2) used by
// the stage kernels of shtb_butterfly.cu and by the persistent batch kernel
// of shtb_batch.cu.  CG = true reads data through L2
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

// Warp layout of the synthesis items: each lane owns ONE real component c of
// the C = 2 x maps carried per entry, and the LD = 32 / C lanes that share a
// component split the rows (level items) or columns (residual blocks) of the
// item, so a pass wastes at most LD - 1 rows or columns (1 at 8 maps).
template <int C>
struct Lanes {
    static_assert(C >= 2 && C <= 16 && 32 % C == 0, "2..16 real components per entry");
    static constexpr int LD = 32 / C;    // lanes per component
    static constexpr int NRMAX = C < 8 ? C : 8;   // residual columns per lane and pass
};

// NR columns per lane of one residual block, columns s0 + sl + r LD (r < NR):
// u_s = sum_j R[j][s] a_j for component c, then stored to u (or q^t).
template <int NB, int NR, bool CG>
__device__ __forceinline__ void bf_r_pass(const BfRItem &it, int L, int nhalf, const int *__restrict__ ints,
                                          const double *__restrict__ R, const double *a0, int astride,
                                          int s0, int sl, int c, double *ubuf, double *qt)
{
    constexpr int C = 2 * NB, LD = Lanes<C>::LD;
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0;
    const int k = it.k;
#pragma unroll 2
    for (int j = 0; j < it.nrows; ++j) {
        const double a = ldp<CG>(a0 + (size_t)j * astride);
        const double *__restrict__ Rj = R + (size_t)j * k + s0 + sl;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const double t = s0 + sl + r * LD < k ? Rj[r * LD] : 0.0;
            acc[r] = fma(t, a, acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int sidx = s0 + sl + r * LD;
        if (sidx >= k) continue;
        if (it.to_rings) qt_store(qt, ints[it.out_off + sidx], nhalf, L, c, acc[r]);
        else ubuf[(size_t)(it.out_off + sidx) * C + c] = acc[r];
    }
}

template <int NB, int NR, bool CG>
__device__ __forceinline__ void bf_r_dispatch(int nr, const BfRItem &it, int L, int nhalf, const int *ints,
                                              const double *R, const double *a0, int astride, int s0, int sl,
                                              int c, double *ubuf, double *qt)
{
    if constexpr (NR > 1) {
        if (nr < NR) {
            bf_r_dispatch<NB, NR - 1, CG>(nr, it, L, nhalf, ints, R, a0, astride, s0, sl, c, ubuf, qt);
            return;
        }
    }
    bf_r_pass<NB, NR, CG>(it, L, nhalf, ints, R, a0, astride, s0, sl, c, ubuf, qt);
}

// Few maps (C = 2 NB <= 4): a lane owns every component of its columns, so
// one load of R[j][s] feeds C FMAs; the 32 lanes split the columns and each
// column's sum runs over the rows in order, as with more maps (results do not
// depend on how maps are grouped).  The row's C values of a are NB double2
// loads shared by the warp.
template <int NB, int NR, bool CG>
__device__ __forceinline__ void bf_r_pass_cl(const BfRItem &it, int L, int nhalf, const int *__restrict__ ints,
                                             const double *__restrict__ R, const double2 *a0, int astride,
                                             int s0, int lane, double *ubuf, double *qt)
{
    constexpr int C = 2 * NB;
    double acc[NR][C];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] = 0.0;
    const int k = it.k;
#pragma unroll 4
    for (int j = 0; j < it.nrows; ++j) {
        double2 a[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) a[b] = CG ? __ldcg(a0 + (size_t)j * astride + b) : __ldg(a0 + (size_t)j * astride + b);
        const double *__restrict__ Rj = R + (size_t)j * k + s0 + lane;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const double t = s0 + lane + 32 * r < k ? Rj[32 * r] : 0.0;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                acc[r][2 * b] = fma(t, a[b].x, acc[r][2 * b]);
                acc[r][2 * b + 1] = fma(t, a[b].y, acc[r][2 * b + 1]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int sidx = s0 + lane + 32 * r;
        if (sidx >= k) continue;
        if (it.to_rings) {
            const long long e = ints[it.out_off + sidx];
#pragma unroll
            for (int c = 0; c < C; ++c) qt_store(qt, e, nhalf, L, c, acc[r][c]);
        } else {
            double *dst = ubuf + (size_t)(it.out_off + sidx) * C;
#pragma unroll
            for (int c = 0; c < C; ++c) dst[c] = acc[r][c];
        }
    }
}

template <int NB, int NR, bool CG>
__device__ __forceinline__ void bf_r_dispatch_cl(int nr, const BfRItem &it, int L, int nhalf, const int *ints,
                                                 const double *R, const double2 *a0, int astride, int s0,
                                                 int lane, double *ubuf, double *qt)
{
    if constexpr (NR > 1) {
        if (nr < NR) {
            bf_r_dispatch_cl<NB, NR - 1, CG>(nr, it, L, nhalf, ints, R, a0, astride, s0, lane, ubuf, qt);
            return;
        }
    }
    bf_r_pass_cl<NB, NR, CG>(it, L, nhalf, ints, R, a0, astride, s0, lane, ubuf, qt);
}

// u = R^T a over one residual block.  ai: [idx][nmaps] complex, the group's
// maps at b0 .. b0+NB-1; chain row j of (m, t) is a_{m+t+2j}.  A pass covers
// up to LD x NRMAX columns; its per-lane column count is exact (the block's
// columns rounded up to LD).
template <int NB, bool CG>
__device__ __forceinline__ void bf_r_item(const BfRItem &it, int L, int nhalf, const int *__restrict__ ints,
                                          const double *__restrict__ dbl, const double2 *ai, int nmaps,
                                          int b0, double *ubuf, double *qt, int lane)
{
    constexpr int C = 2 * NB, LD = Lanes<C>::LD;
    const double *__restrict__ R = dbl + it.data_off;
    const long long aoff = alm_off(L, it.m) + it.t;   // chain row j at aoff + 2j
    if constexpr (NB <= 2) {
        constexpr int NRMAX = 4;
        const double2 *a0 = ai + (size_t)(aoff + 2 * it.j0) * nmaps + b0;
        for (int s0 = 0; s0 < it.k; s0 += 32 * NRMAX) {
            const int nr = min(NRMAX, (it.k - s0 + 31) / 32);
            bf_r_dispatch_cl<NB, NRMAX, CG>(nr, it, L, nhalf, ints, R, a0, 2 * nmaps, s0, lane, ubuf, qt);
        }
        return;
    }
    const int sl = lane % LD, c = lane / LD;
    const double *a0 = reinterpret_cast<const double *>(ai + (size_t)(aoff + 2 * it.j0) * nmaps + b0) + c;
    const int astride = 4 * nmaps;                    // doubles between chain rows j and j + 1
    for (int s0 = 0; s0 < it.k; s0 += LD * Lanes<C>::NRMAX) {
        const int nr = min(Lanes<C>::NRMAX, (it.k - s0 + LD - 1) / LD);
        bf_r_dispatch<NB, Lanes<C>::NRMAX, CG>(nr, it, L, nhalf, ints, R, a0, astride, s0, sl, c, ubuf, qt);
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

// NR dense rows per lane of one child, rows q0 + dl + r LD (r < NR): each a
// k-long dot product of the child's T column with its u (component c); every
// u value loaded serves the lane's NR rows.
template <int NB, int NR, bool CG>
__device__ __forceinline__ void bf_dense_pass(int k, int nd, const double *__restrict__ T,
                                              const int *__restrict__ dpos, const double *uc, int q0, int dl,
                                              int c, double *out, bool second)
{
    constexpr int C = 2 * NB, LD = Lanes<C>::LD, OS = out_stride<C>();
    // every dot product starts from zero; the first child's rows are then
    // stored, the second child's added to what the first child left (one
    // order for every map-group width, see bf_level_item_pair)
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0;
    const double *__restrict__ Tq = T + q0 + dl;
#pragma unroll 2
    for (int i = 0; i < k; ++i) {
        const double uv = ldp<CG>(uc + (size_t)i * C);
        const double *__restrict__ Ti = Tq + (size_t)i * nd;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const double t = q0 + dl + r * LD < nd ? Ti[r * LD] : 0.0;
            acc[r] = fma(t, uv, acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int d = q0 + dl + r * LD;
        if (d < nd) {
            double *o = out + dpos[d] * OS + c;
            *o = second ? *o + acc[r] : acc[r];
        }
    }
}

template <int NB, int NR, bool CG>
__device__ __forceinline__ void bf_dense_dispatch(int nr, int k, int nd, const double *T, const int *dpos,
                                                  const double *uc, int q0, int dl, int c, double *out,
                                                  bool second)
{
    if constexpr (NR > 1) {
        if (nr < NR) {
            bf_dense_dispatch<NB, NR - 1, CG>(nr, k, nd, T, dpos, uc, q0, dl, c, out, second);
            return;
        }
    }
    bf_dense_pass<NB, NR, CG>(k, nd, T, dpos, uc, q0, dl, c, out, second);
}

// Few maps (C = 2 NB <= 4): the two children run side by side, lanes 16 h
// to 16 h + 15 on child h, each lane owning every component of its dense
// rows d = dl + 16 r (r < NR; nd < 128 = 16 x 8, so one pass), so one load
// of T[i][d] feeds C FMAs.  Each row's dot product runs over i in order from
// zero, as in bf_dense_pass; the first child's rows and identity entries are
// stored, then the second child's are added: the same arithmetic as with
// more maps, bit for bit.
template <int NB, int NR, bool CG>
__device__ __forceinline__ void bf_pair_rows(const BfItem &it, const int *__restrict__ ints,
                                             const double *__restrict__ dbl, const double *uin, double *out,
                                             int lane)
{
    constexpr int C = 2 * NB, OS = out_stride<C>();
    const int h = lane >> 4, dl = lane & 15;
    const int k = it.k[h], nd = it.nd[h];
    const int kmax = max(it.nd[0], it.nd[1]) ? max(it.k[0], it.k[1]) : 0;
    const double2 *u2 = reinterpret_cast<const double2 *>(uin + (size_t)it.u_off[h] * C);
    const double *__restrict__ Tq = dbl + it.T_off[h] + dl;
    const int *__restrict__ dpos = ints + it.dpos_off[h];
    double acc[NR][C];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] = 0.0;
#pragma unroll 2
    for (int i = 0; i < kmax; ++i) {
        if (i < k) {
            double2 uv[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) uv[b] = CG ? __ldcg(u2 + (size_t)i * NB + b) : __ldg(u2 + (size_t)i * NB + b);
            const double *__restrict__ Ti = Tq + (size_t)i * nd;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const double t = dl + 16 * r < nd ? Ti[16 * r] : 0.0;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    acc[r][2 * b] = fma(t, uv[b].x, acc[r][2 * b]);
                    acc[r][2 * b + 1] = fma(t, uv[b].y, acc[r][2 * b + 1]);
                }
            }
        }
    }
    for (int s = 0; s < 2; ++s) {
        if (h == s) {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int d = dl + 16 * r;
                if (d < nd) {
                    double *o = out + dpos[d] * OS;
#pragma unroll
                    for (int c = 0; c < C; ++c) o[c] = s ? o[c] + acc[r][c] : acc[r][c];
                }
            }
        }
        // identity entries of child s: a store for the first child, an add
        // for the second
        const double *us = uin + (size_t)it.u_off[s] * C;
        const int *__restrict__ ipos = ints + it.ipos_off[s];
        for (int x = lane; x < it.k[s] * C; x += 32) {
            const int i = x / C, cc = x - i * C;
            double *o = out + ipos[i] * OS + cc;
            *o = s ? *o + ldp<CG>(us + x) : ldp<CG>(us + x);
        }
        __syncwarp();
    }
}

template <int NB, int NR, bool CG>
__device__ __forceinline__ void bf_pair_dispatch(int nr, const BfItem &it, const int *ints, const double *dbl,
                                                 const double *uin, double *out, int lane)
{
    if constexpr (NR > 1) {
        if (nr < NR) {
            bf_pair_dispatch<NB, NR - 1, CG>(nr, it, ints, dbl, uin, out, lane);
            return;
        }
    }
    bf_pair_rows<NB, NR, CG>(it, ints, dbl, uin, out, lane);
}

// Each child in turn: its dense rows (passes of up to LD x NRMAX rows, the
// per-lane row count exact), then its identity entries.  A child's dense and
// identity positions are distinct, so lanes never update the same scratch
// entry within a child; the warp syncs between the children, whose positions
// may coincide.
template <int NB, bool CG>
__device__ __forceinline__ void bf_level_item(const BfItem &it, int L, int nhalf, const int *__restrict__ ints,
                                              const double *__restrict__ dbl, const double *uin,
                                              double *uout, double *qt, double *out, int lane)
{
    constexpr int C = 2 * NB, LD = Lanes<C>::LD, NRMAX = Lanes<C>::NRMAX;
    constexpr int OS = out_stride<C>();
    for (int i = lane; i < it.nc * OS; i += 32) out[i] = 0.0;
    __syncwarp();
    const int dl = lane % LD, c = lane / LD;
    if constexpr (NB <= 2) {
        const int nr = (max(it.nd[0], it.nd[1]) + 15) / 16;      // <= 8: nd < kMaxCand
        bf_pair_dispatch<NB, 8, CG>(max(nr, 1), it, ints, dbl, uin, out, lane);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if constexpr (NB <= 2) break;
        const int k = it.k[s], nd = it.nd[s];
        const double *u = uin + (size_t)it.u_off[s] * C;
        const double *__restrict__ T = dbl + it.T_off[s];
        const int *__restrict__ dpos = ints + it.dpos_off[s];
        for (int q0 = 0; q0 < nd; q0 += LD * NRMAX) {
            const int nr = min(NRMAX, (nd - q0 + LD - 1) / LD);
            bf_dense_dispatch<NB, NRMAX, CG>(nr, k, nd, T, dpos, u + c, q0, dl, c, out, s == 1);
        }
        // identity entries: the first child's land on zeroed scratch (a store),
        // the second child's on whatever the first child left there
        const int *__restrict__ ipos = ints + it.ipos_off[s];
        for (int x = lane; x < k * C; x += 32) {
            const int i = x / C, cc = x - i * C;
            double *o = out + ipos[i] * OS + cc;
            *o = s ? *o + ldp<CG>(u + x) : ldp<CG>(u + x);
        }
        __syncwarp();
    }
    if (it.to_rings) {
        const int *__restrict__ ent = ints + it.out_off;
        for (int i = lane; i < it.nc * C; i += 32) {
            const int cc = i / it.nc, cpos = i - cc * it.nc;
            qt_store(qt, ent[cpos], nhalf, L, cc, out[cpos * OS + cc]);
        }
    } else {
        double *dst = uout + (size_t)it.out_off * C;
        for (int i = lane; i < it.nc * C; i += 32) {
            const int cpos = i / C, cc = i - cpos * C;
            dst[i] = out[cpos * OS + cc];
        }
    }
    __syncwarp();
}

}  // namespace shtb_dev
