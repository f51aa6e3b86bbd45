// Device body of regenerated residual blocks (plans built with
// residual_recurrence), used by bf_r_rec_kernel in shtb_butterfly.cu.
#pragma once

#include <cuda_runtime.h>

#include "shtb_bf_items.cuh"

namespace shtb_dev {

// ---- regenerated residual blocks (plans with residual_recurrence): each
// column's R values come from the jump-two recurrence of Eq. (three-term),
// V_{j+1} = (mu_j x + C_j) V_j - V_{j-1}, started from the column's RecStart;
// the a_lm rows are pre-scaled by sigma (Ptilde = sigma V), so
// u_s = sum_j V_j(x_s) (sigma a)_j, a dot product from zero over the rows in
// order for every component, at any map count.  A lane owns CPL components
// of one column and runs the column's recurrence itself (the S lanes of a
// column repeat it); the coefficients of a row are one broadcast load.
template <int NB, bool CG>
__device__ __forceinline__ void bf_r_rec_item(const BfRItem &it, const PlanView &v,
                                              const RecStart *__restrict__ rs, const int *__restrict__ ints,
                                              const double2 *ai, int nmaps, int b0, double *ubuf, double *qt,
                                              int lane)
{
    constexpr int C = 2 * NB, CPL = C < 8 ? C : 8, S = C / CPL, CPP = 32 / S;
    const int L = v.lmax, nhalf = v.nhalf;
    const int c0 = (lane % S) * CPL;
    const long long arow = alm_off(L, it.m) + it.t + 2 * it.j0;       // chain row j0
    const double *a0 = reinterpret_cast<const double *>(ai + (size_t)arow * nmaps + b0) + c0;
    const size_t astride = (size_t)4 * nmaps;                         // doubles per chain row
    const RecCoef *__restrict__ cf = v.coef + arow;                   // block row j at cf[2 j]
    for (int s0 = 0; s0 < it.k; s0 += CPP) {
        const int s = s0 + lane / S;
        const bool ok = s < it.k;
        const RecStart st = ok ? rs[it.rs_off + s] : RecStart{0, it.nrows, 0.0, 0.0};
        const double x = v.xarg[st.ring];
        const bool sform = v.xform[st.ring] != 0;
        double acc[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[c] = 0.0;
        double cur = st.start == 0 ? st.v0 : 0.0, prev = 0.0;
#pragma unroll 2
        for (int j = 0; j < it.nrows; ++j) {
            const double *aj = a0 + (size_t)j * astride;
#pragma unroll
            for (int c = 0; c < CPL; c += 2) {
                const double2 a = CG ? __ldcg(reinterpret_cast<const double2 *>(aj + c))
                                     : __ldg(reinterpret_cast<const double2 *>(aj + c));
                acc[c] = fma(cur, a.x, acc[c]);
                acc[c + 1] = fma(cur, a.y, acc[c + 1]);
            }
            const RecCoef k = cf[2 * j];
            const double w = fma(k.mu, x, sform ? k.cs : k.cz);
            double nxt = fma(w, cur, -prev);
            if (j == st.start) nxt = st.v1;
            if (j + 1 == st.start) nxt = st.v0;
            prev = cur;
            cur = nxt;
        }
        if (!ok) continue;
        if (it.to_rings) {
            const int e = ints[it.out_off + s];
#pragma unroll
            for (int c = 0; c < CPL; ++c) qt_store(qt, e, nhalf, L, c0 + c, acc[c]);
        } else {
            double *dst = ubuf + (size_t)(it.out_off + s) * C + c0;
#pragma unroll
            for (int c = 0; c < CPL; ++c) dst[c] = acc[c];
        }
    }
}

// Adjoint of the regenerated residual blocks of one (chain, row interval)
// group: a_j = sigma_j sum over the group's blocks and their columns s of
// V_j(x_s) x_s, x the block's u (or g at depth 0); sigma is applied by the
// final staging.  Each block is taken 32 columns and 32 rows at a time: the
// column lanes continue their recurrences over the chunk's rows into a
// shared tile Vt, then the row lanes add the chunk to their rows of ad
// (zeroed first), running over blocks and columns in order like the stored
// blocks' adjoint.  smem: this warp's 32 x 33 + 32 x C doubles.
template <int NB>
__device__ __forceinline__ void bf_adj_r_rec_group(const BfRGroup &gr, const PlanView &v,
                                                   const BfRItem *__restrict__ ritems,
                                                   const RecStart *__restrict__ rs, const int *__restrict__ ints,
                                                   const double *ubuf, const double *gd, int nmaps, int b0,
                                                   double *ad, double *smem, int lane)
{
    constexpr int C = 2 * NB, TS = 33;
    double *Vt = smem, *X = smem + 32 * TS;
    const int L = v.lmax;
    const long long aoff = alm_off(L, gr.m) + gr.t;
    for (int j = gr.r0 + lane; j < gr.r1; j += 32)
#pragma unroll
        for (int c = 0; c < C; ++c) ad[((size_t)(aoff + 2 * j) * nmaps + b0) * 2 + c] = 0.0;
    __syncwarp();
    for (int q = 0; q < gr.nblk; ++q) {
        const BfRItem it = ritems[ints[gr.blk_off + q]];
        if (it.nrows == 0) continue;
        const RecCoef *__restrict__ cf = v.coef + aoff + 2 * it.j0;   // block row j at cf[2 j]
        for (int s0 = 0; s0 < it.k; s0 += 32) {
            const int s = s0 + lane, ncol = min(32, it.k - s0);
            const bool ok = s < it.k;
            const RecStart st = ok ? rs[it.rs_off + s] : RecStart{0, it.nrows, 0.0, 0.0};
            const double x = v.xarg[st.ring];
            const bool sform = v.xform[st.ring] != 0;
            if (ok)
#pragma unroll
                for (int c = 0; c < C; ++c)
                    X[lane * C + c] = it.to_rings ? __ldg(gd + ((size_t)ints[it.out_off + s] * nmaps + b0) * 2 + c)
                                                  : ubuf[(size_t)(it.out_off + s) * C + c];
            double cur = st.start == 0 ? st.v0 : 0.0, prev = 0.0;
            for (int r0 = 0; r0 < it.nrows; r0 += 32) {
                const int nr = min(32, it.nrows - r0);
                for (int r = 0; r < nr; ++r) {
                    const int j = r0 + r;
                    Vt[r * TS + lane] = cur;
                    const RecCoef k = cf[2 * j];
                    const double w = fma(k.mu, x, sform ? k.cs : k.cz);
                    double nxt = fma(w, cur, -prev);
                    if (j == st.start) nxt = st.v1;
                    if (j + 1 == st.start) nxt = st.v0;
                    prev = cur;
                    cur = nxt;
                }
                __syncwarp();
                if (lane < nr) {
                    const int j = it.j0 + r0 + lane;
                    double *a = ad + ((size_t)(aoff + 2 * j) * nmaps + b0) * 2;
                    double acc[C];
#pragma unroll
                    for (int c = 0; c < C; ++c) acc[c] = a[c];
                    for (int sc = 0; sc < ncol; ++sc) {
                        const double vv = Vt[lane * TS + sc];
#pragma unroll
                        for (int c = 0; c < C; ++c) acc[c] = fma(vv, X[sc * C + c], acc[c]);
                    }
#pragma unroll
                    for (int c = 0; c < C; ++c) a[c] = acc[c];
                }
                __syncwarp();
            }
        }
    }
}

}  // namespace shtb_dev
