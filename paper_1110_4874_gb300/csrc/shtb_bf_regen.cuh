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

}  // namespace shtb_dev
