// Kernel (a): application of the butterfly-compressed Legendre operator
// (Sec. 3.2, Eq. factor-into-block-diagonal) for synthesis, q^t = Lambda^T a,
// level by level over all (m, parity) chains at once.
//
//   bf_r_kernel      u = R^T a_I for every residual block (top level of each
//                    chain; depth-0 chains write q^t directly);
//   bf_level_kernel  one item = two sibling nodes sharing a candidate list:
//                    v = T_top^T u_top + T_bot^T u_bot, split into the parent
//                    level's two u vectors (or q^t on a leaf block at level 1);
//                    identity part = adds, dense part = k x nd dot products
//                    (Appendix: the identity-embedded interpolation matrices);
// and the ring stage of each map group then reads q_m(+z) = q^0 + q^1 and
// q_m(-z) = q^0 - q^1 (Eq. q-even-odd2) straight from the two parity halves.
// One warp per work item; all maps of a group (up to 8, 2 real components
// each) are carried per entry so every stored matrix element is read once
// per group and used for 2 x maps FMAs.  All stages are FP64-bound on GB300.
#include <cuda_runtime.h>

#include <algorithm>

#include "shtb_bf_items.cuh"
#include "shtb_bf_regen.cuh"
#include "shtb_butterfly.h"

namespace {

using shtb_dev::Tile;

constexpr int kBfWarps = 4;
// with one or two maps, a warp takes this many consecutive level items or
// residual blocks (their dot products packed on its lanes)
constexpr int kBfLevelPack = 2;
constexpr int kBfResidualPack = 8;

template <int NB>
__host__ __device__ constexpr int items_per_warp_level()
{
    return NB <= 2 ? kBfLevelPack : 1;
}

template <int NB>
__host__ __device__ constexpr int items_per_warp_residual()
{
    return NB <= 2 ? kBfResidualPack : 1;
}

// level-item scratch of one warp (doubles)
template <int NB>
__host__ __device__ constexpr size_t level_scratch_doubles(int maxnc)
{
    return (size_t)items_per_warp_level<NB>() * maxnc * shtb_dev::level_scratch_per_cand(2 * NB);
}


// Staging between the caller's stacked a_lm [map][idx] and the butterfly's
// interleaved ai [idx][map]: tiles of T coefficients x MB maps pass through
// shared memory, so that both the map-major side and the interleaved side are
// read or written along consecutive addresses (one map is a plain copy).  The
// tile row is padded by one entry so the column walk spreads over the banks.
constexpr int kStageTile = 256;

struct StageTile {
    int T, MB;
    __device__ __forceinline__ explicit StageTile(int nmaps)
        : T(nmaps >= kStageTile ? 1 : kStageTile / nmaps), MB(nmaps < kStageTile ? nmaps : kStageTile) {}
};

// ai[idx][b] = a_lm[b][idx] (Im a_l0 = 0, Sec. 2.1: idx <= L is m = 0), times
// sigma_lm when sig is non-null (plans that regenerate R by the rescaled
// recurrence, Ptilde = sigma V)
__device__ __forceinline__ double2 staged(double2 a, long long i, long long L, const RecCoef *sig)
{
    const double s = sig ? sig[i].sig : 1.0;
    return sig ? make_double2(a.x * s, i <= L ? 0.0 : a.y * s) : make_double2(a.x, i <= L ? 0.0 : a.y);
}

__global__ void __launch_bounds__(256) bf_interleave_kernel(PlanView v, const double2 *__restrict__ alm,
                                                            double2 *__restrict__ ai, int nmaps,
                                                            const RecCoef *__restrict__ sig)
{
    __shared__ double2 tile[2 * kStageTile];
    const long long nalm = v.nalm, L = v.lmax;
    if (nmaps == 1) {
        for (long long i = blockIdx.x * 256LL + threadIdx.x; i < nalm; i += 256LL * gridDim.x)
            ai[i] = staged(alm[i], i, L, sig);
        return;
    }
    const StageTile st(nmaps);
    for (long long i0 = (long long)blockIdx.x * st.T; i0 < nalm; i0 += (long long)st.T * gridDim.x) {
        const int nt = (int)min((long long)st.T, nalm - i0);
        for (int b0 = 0; b0 < nmaps; b0 += st.MB) {
            const int mb = min(st.MB, nmaps - b0);
            for (int e = threadIdx.x; e < nt * mb; e += blockDim.x) {
                const int b = e / nt, t = e - b * nt;
                tile[b * (st.T + 1) + t] = alm[(size_t)(b0 + b) * nalm + i0 + t];
            }
            __syncthreads();
            for (int e = threadIdx.x; e < nt * mb; e += blockDim.x) {
                const int t = e / mb, b = e - t * mb;
                ai[(size_t)(i0 + t) * nmaps + b0 + b] = staged(tile[b * (st.T + 1) + t], i0 + t, L, sig);
            }
            __syncthreads();
        }
    }
}

// grid of the staging kernels: every tile once, at most 16 blocks per SM
unsigned stage_grid(const shtb_plan_s *p, int nmaps)
{
    const long long T = nmaps >= kStageTile ? 1 : kStageTile / nmaps;
    const long long tiles = nmaps == 1 ? (p->nalm + 255) / 256 : (p->nalm + T - 1) / T;
    return (unsigned)std::max(1LL, std::min(tiles, 152LL * 16));
}

template <int NB>
__global__ void __launch_bounds__(32 * kBfWarps)
bf_r_kernel(PlanView v, const BfRItem *__restrict__ items, int nitems, const int *__restrict__ ints,
            const double *__restrict__ dbl, const double2 *__restrict__ ai, int nmaps, int b0,
            double *__restrict__ ubuf0, double *__restrict__ ubuf1, const int *__restrict__ depth_par,
            double *__restrict__ qt)
{
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * kBfWarps + (threadIdx.x >> 5);
    if constexpr (NB <= 2) {
        constexpr int G = kBfResidualPack;
        const int i0 = w * G;
        if (i0 >= nitems) return;
        shtb_dev::bf_r_items_few<NB, G, false>(items + i0, min(G, nitems - i0), v.lmax, v.nhalf, ints, dbl, ai,
                                               nmaps, b0, ubuf0, ubuf1, depth_par, qt, lane);
        return;
    }
    if (w >= nitems) return;
    const BfRItem it = items[w];
    double *ubuf = depth_par[it.m * 2 + it.t] ? ubuf1 : ubuf0;
    shtb_dev::bf_r_item<NB, false>(it, v.lmax, v.nhalf, ints, dbl, ai, nmaps, b0, ubuf, qt, lane);
}

// RING: the launch is the plan's level 1, whose items all write q^t (no
// other level's do), so each instantiation holds one output path.
template <int NB, bool RING>
__global__ void __launch_bounds__(32 * kBfWarps, NB <= 2 ? 6 : 8)
bf_level_kernel(const BfItem *__restrict__ items, int nitems, int L, int nhalf, int maxnc,
                const int *__restrict__ ints, const double *__restrict__ dbl,
                const double *__restrict__ uin, double *__restrict__ uout, double *__restrict__ qt)
{
    extern __shared__ double sout[];     // [kBfWarps][level_scratch_doubles<NB>(maxnc)]
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int w = blockIdx.x * kBfWarps + wib;
    double *scr = sout + (size_t)wib * level_scratch_doubles<NB>(maxnc);
    if constexpr (NB <= 2) {
        constexpr int G = kBfLevelPack;
        const int i0 = w * G;
        if (i0 >= nitems) return;
        const int n = min(G, nitems - i0);
        BfItem it[G];
#pragma unroll
        for (int q = 0; q < G; ++q) it[q] = items[i0 + min(q, n - 1)];
        shtb_dev::bf_level_items_few<NB, G, false>(it, n, L, nhalf, ints, dbl, uin, uout, qt, scr, maxnc, lane);
        return;
    }
    if (w >= nitems) return;
    shtb_dev::bf_level_item<NB, false, RING ? 1 : 0>(items[w], L, nhalf, ints, dbl, uin, uout, qt, scr, lane);
}

// regenerated residual blocks (residual_recurrence plans), one per warp
template <int NB>
__global__ void __launch_bounds__(32 * kBfWarps)
bf_r_rec_kernel(PlanView v, const BfRItem *__restrict__ items, int nitems, const RecStart *__restrict__ rs,
                const int *__restrict__ ints, const double2 *__restrict__ ai, int nmaps, int b0,
                double *__restrict__ ubuf0, double *__restrict__ ubuf1, const int *__restrict__ depth_par,
                double *__restrict__ qt)
{
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * kBfWarps + (threadIdx.x >> 5);
    if (w >= nitems) return;
    const BfRItem it = items[w];
    double *ubuf = depth_par[it.m * 2 + it.t] ? ubuf1 : ubuf0;
    shtb_dev::bf_r_rec_item<NB, false>(it, v, rs, ints, ai, nmaps, b0, ubuf, qt, lane);
}

// residual blocks of one map group (maps b0 .. b0+NB-1 of ai)
template <int NB>
int launch_r(const shtb_plan_s *p, const double2 *ai, int nmaps, int b0, double *u0, double *u1,
             double *qt, cudaStream_t st)
{
    const BfPlanDev &bf = *p->bf;
    if (bf.n_ritems == 0) return SHTB_OK;
    if (bf.rec) {
        const unsigned grid = (unsigned)((bf.n_ritems + kBfWarps - 1) / kBfWarps);
        bf_r_rec_kernel<NB><<<grid, 32 * kBfWarps, 0, st>>>(p->view, bf.ritems, bf.n_ritems, bf.rstart, bf.ints,
                                                            ai, nmaps, b0, u0, u1, bf.depth_parity, qt);
        SHTB_CUDA_TRY(cudaGetLastError());
        ++p->launches;
        return SHTB_OK;
    }
    const long long warps = (bf.n_ritems + items_per_warp_residual<NB>() - 1) / items_per_warp_residual<NB>();
    const unsigned grid = (unsigned)((warps + kBfWarps - 1) / kBfWarps);
    bf_r_kernel<NB><<<grid, 32 * kBfWarps, 0, st>>>(p->view, bf.ritems, bf.n_ritems, bf.ints, bf.dbl, ai,
                                                    nmaps, b0, u0, u1, bf.depth_parity, qt);
    SHTB_CUDA_TRY(cudaGetLastError());
    ++p->launches;
    return SHTB_OK;
}

// butterfly levels of one map group, top down; level 1 writes q^t
template <int NB>
int launch_levels(const shtb_plan_s *p, double *u0, double *u1, double *qt, cudaStream_t st)
{
    const BfPlanDev &bf = *p->bf;
    for (int lev = bf.depth_max; lev >= 1; --lev) {
        const int n = bf.level_counts[lev - 1];
        if (n == 0) continue;
        double *uin = (lev % 2) ? u1 : u0;
        double *uout = ((lev - 1) % 2) ? u1 : u0;
        const int warps = (n + items_per_warp_level<NB>() - 1) / items_per_warp_level<NB>();
        const unsigned grid = (unsigned)((warps + kBfWarps - 1) / kBfWarps);
        const int maxnc = bf.level_maxnc[lev - 1];
        const size_t smem = sizeof(double) * kBfWarps * level_scratch_doubles<NB>(maxnc);
        auto *kern = lev == 1 ? bf_level_kernel<NB, true> : bf_level_kernel<NB, false>;
        SHTB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, 32 * kBfWarps, smem, st>>>(bf.level_items[lev - 1], n, p->lmax, p->nhalf, maxnc, bf.ints,
                                                bf.dbl, uin, uout, qt);
        SHTB_CUDA_TRY(cudaGetLastError());
        ++p->launches;
    }
    return SHTB_OK;
}

// One map group: residual blocks, butterfly levels, then (map != nullptr)
// the ring stage.  With map == nullptr the group's q^t is the caller's
// array (the Legendre stage alone).
template <int NB>
int run_group(const shtb_plan_s *p, const double2 *ai, int nmaps, int b0, double *u0, double *u1,
              double *qt, double *map, cudaStream_t st)
{
    shtb_plan_s *pp = const_cast<shtb_plan_s *>(p);
    const int ev_leg = profile_begin(pp, st);
    int ev = profile_begin(pp, st);
    int rc = launch_r<NB>(p, ai, nmaps, b0, u0, u1, qt, st);
    if (rc) return rc;
    profile_end(pp, st, 5, ev);
    ev = profile_begin(pp, st);
    if ((rc = launch_levels<NB>(p, u0, u1, qt, st))) return rc;
    profile_end(pp, st, 6, ev);
    profile_end(pp, st, 0, ev_leg);
    if (!map) return SHTB_OK;
    // ring stage of this group straight from q^0, q^1 (parity combine fused)
    ev = profile_begin(pp, st);
    rc = launch_phi_synth_qt(p, qt, NB, map, b0, st);
    profile_end(pp, st, 1, ev);
    return rc;
}

// a_lm of merged maps (one device pointer per map) into ai[idx][map]
__global__ void bf_gather_kernel(PlanView v, const double2 *const *__restrict__ alm_of_map,
                                 double2 *__restrict__ ai, int nmaps)
{
    const int m = blockIdx.x;
    const int L = v.lmax;
    const long long off = shtb_dev::alm_off(L, m);
    const int n = L - m + 1;
    for (int i = threadIdx.x; i < n * nmaps; i += blockDim.x) {
        const int b = i / n, dl = i - b * n;
        const long long idx = off + dl;
        const double2 a = alm_of_map[b][idx];
        ai[(size_t)idx * nmaps + b] = make_double2(a.x, m == 0 ? 0.0 : a.y);
    }
}

// ------------------------------------------------------------------ adjoint
// a^t = Lambda g^t: the transposed butterfly.  Level items run bottom-up:
// item (parent P, group G) gathers its candidate vector (g on a leaf block at
// level 1, else the u of level l-1) and applies both children's T:
// u_s = [I | T_s] v  (identity entries copy, dense rows are k x nd dots).

// NR rows of child s per lane, rows q0 + dl + r LD (r < NR), component c
template <int NB, int NR>
__device__ __forceinline__ void adj_rows(const BfItem &it, int s, const int *__restrict__ ints,
                                         const double *__restrict__ dbl, const double *in, int q0, int dl,
                                         int c, double *__restrict__ uout)
{
    constexpr int C = 2 * NB, LD = shtb_dev::Lanes<C>::LD;
    const int k = it.k[s], nd = it.nd[s];
    const double *__restrict__ T = dbl + it.T_off[s];        // k x nd, row-major
    const int *__restrict__ dpos = ints + it.dpos_off[s];
    const int *__restrict__ ipos = ints + it.ipos_off[s];
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int i = q0 + dl + r * LD;
        acc[r] = i < k ? in[ipos[i] * C + c] : 0.0;
    }
#pragma unroll 2
    for (int d = 0; d < nd; ++d) {
        const double x = in[dpos[d] * C + c];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int i = q0 + dl + r * LD;
            const double t = i < k ? T[(size_t)i * nd + d] : 0.0;
            acc[r] = fma(t, x, acc[r]);
        }
    }
    double *dst = uout + (size_t)it.u_off[s] * C + c;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int i = q0 + dl + r * LD;
        if (i < k) dst[(size_t)i * C] = acc[r];
    }
}

template <int NB, int NR>
__device__ __forceinline__ void adj_rows_dispatch(int nr, const BfItem &it, int s, const int *ints,
                                                  const double *dbl, const double *in, int q0, int dl, int c,
                                                  double *uout)
{
    if constexpr (NR > 1) {
        if (nr < NR) {
            adj_rows_dispatch<NB, NR - 1>(nr, it, s, ints, dbl, in, q0, dl, c, uout);
            return;
        }
    }
    adj_rows<NB, NR>(it, s, ints, dbl, in, q0, dl, c, uout);
}
template <int NB>
__global__ void __launch_bounds__(32 * kBfWarps)
bf_adj_level_kernel(const BfItem *__restrict__ items, int nitems, const int *__restrict__ ints,
                    const double *__restrict__ dbl, const double *__restrict__ uin,
                    const double2 *__restrict__ g, int nmaps, int b0, double *__restrict__ uout)
{
    constexpr int C = 2 * NB;
    extern __shared__ double sin_[];     // [kBfWarps][kMaxCand * C]
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int w = blockIdx.x * kBfWarps + wib;
    if (w >= nitems) return;
    const BfItem it = items[w];
    double *in = sin_ + (size_t)wib * shtb::kMaxCand * C;
    if (it.to_rings) {
        const int *__restrict__ ent = ints + it.out_off;
        for (int i = lane; i < it.nc * NB; i += 32) {
            const int cpos = i / NB, b = i - cpos * NB;
            const double2 x = g[(size_t)ent[cpos] * nmaps + b0 + b];
            in[cpos * C + 2 * b] = x.x;
            in[cpos * C + 2 * b + 1] = x.y;
        }
    } else {
        const double *src = uin + (size_t)it.out_off * C;
        for (int i = lane; i < it.nc * C; i += 32) in[i] = src[i];
    }
    __syncwarp();
    // each child in turn, its k rows over the lanes (one component per lane,
    // an exact per-lane row count): identity entry plus a dot product of the
    // row of T with the candidates' dense part
    using shtb_dev::Lanes;
    constexpr int LD = Lanes<C>::LD, NRMAX = Lanes<C>::NRMAX;
    const int dl = lane % LD, c = lane / LD;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int k = it.k[s];
        for (int q0 = 0; q0 < k; q0 += LD * NRMAX) {
            const int nr = min(NRMAX, (k - q0 + LD - 1) / LD);
            adj_rows_dispatch<NB, NRMAX>(nr, it, s, ints, dbl, in, q0, dl, c, uout);
        }
    }
}

// NR rows per lane of one (chain, row interval) group, rows j0 + dl + r LD
// (r < NR), component c: a_j = sum over the group's residual blocks of
// R[j, :] x, x the block's u (or g at depth 0)
template <int NB, int NR>
__device__ __forceinline__ void adj_r_rows(const BfRGroup &gr, const BfRItem *__restrict__ ritems,
                                           const int *__restrict__ ints, const double *__restrict__ dbl,
                                           const double *ubuf, const double *gd, int nmaps, int b0, int j0,
                                           int dl, int c, double *ad, long long aoff)
{
    constexpr int C = 2 * NB, LD = shtb_dev::Lanes<C>::LD;
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0;
    const int jend = min(gr.r1, j0 + NR * LD);
    for (int q = 0; q < gr.nblk; ++q) {
        const BfRItem it = ritems[ints[gr.blk_off + q]];
        if (it.j0 >= jend || it.j0 + it.nrows <= j0) continue;       // no row of this pass
        const double *__restrict__ R = dbl + it.data_off;
        for (int s = 0; s < it.k; ++s) {
            const double x = it.to_rings ? __ldg(gd + ((size_t)ints[it.out_off + s] * nmaps + b0) * 2 + c)
                                         : __ldg(ubuf + (size_t)(it.out_off + s) * C + c);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int j = j0 + dl + r * LD;
                const bool in_blk = j >= it.j0 && j < it.j0 + it.nrows;
                const double t = in_blk ? R[(size_t)(j - it.j0) * it.k + s] : 0.0;
                acc[r] = fma(t, x, acc[r]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int j = j0 + dl + r * LD;
        if (j < gr.r1) ad[((size_t)(aoff + 2 * j) * nmaps + b0) * 2 + c] = acc[r];
    }
}

template <int NB, int NR>
__device__ __forceinline__ void adj_r_dispatch(int nr, const BfRGroup &gr, const BfRItem *ritems,
                                               const int *ints, const double *dbl, const double *ubuf,
                                               const double *gd, int nmaps, int b0, int j0, int dl, int c,
                                               double *ad, long long aoff)
{
    if constexpr (NR > 1) {
        if (nr < NR) {
            adj_r_dispatch<NB, NR - 1>(nr, gr, ritems, ints, dbl, ubuf, gd, nmaps, b0, j0, dl, c, ad, aoff);
            return;
        }
    }
    adj_r_rows<NB, NR>(gr, ritems, ints, dbl, ubuf, gd, nmaps, b0, j0, dl, c, ad, aoff);
}

// a rows of one (chain, row interval): every row of the interval is written
// (zero when no block reaches it), so each chain row has exactly one writer
template <int NB>
__global__ void __launch_bounds__(32 * kBfWarps)
bf_adj_r_kernel(PlanView v, const BfRGroup *__restrict__ groups, int ngroups,
                const BfRItem *__restrict__ ritems, const int *__restrict__ ints,
                const double *__restrict__ dbl, const double *__restrict__ u0,
                const double *__restrict__ u1, const int *__restrict__ depth_par,
                const double2 *__restrict__ g, int nmaps, int b0, double2 *__restrict__ aacc)
{
    constexpr int C = 2 * NB, LD = shtb_dev::Lanes<C>::LD, NRMAX = shtb_dev::Lanes<C>::NRMAX;
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * kBfWarps + (threadIdx.x >> 5);
    if (w >= ngroups) return;
    const BfRGroup gr = groups[w];
    const double *ubuf = depth_par[gr.m * 2 + gr.t] ? u1 : u0;
    const long long aoff = shtb_dev::alm_off(v.lmax, gr.m) + gr.t;
    const int dl = lane % LD, c = lane / LD;
    for (int j0 = gr.r0; j0 < gr.r1; j0 += LD * NRMAX) {
        const int nr = min(NRMAX, (gr.r1 - j0 + LD - 1) / LD);
        adj_r_dispatch<NB, NRMAX>(nr, gr, ritems, ints, dbl, ubuf, reinterpret_cast<const double *>(g), nmaps,
                                  b0, j0, dl, c, reinterpret_cast<double *>(aacc), aoff);
    }
}

// adjoint of regenerated residual blocks, one (chain, row interval) per warp
template <int NB>
__global__ void __launch_bounds__(32 * kBfWarps)
bf_adj_r_rec_kernel(PlanView v, const BfRGroup *__restrict__ groups, int ngroups,
                    const BfRItem *__restrict__ ritems, const RecStart *__restrict__ rs,
                    const int *__restrict__ ints, const double *__restrict__ u0, const double *__restrict__ u1,
                    const int *__restrict__ depth_par, const double2 *__restrict__ g, int nmaps, int b0,
                    double2 *__restrict__ aacc)
{
    extern __shared__ double smem_rec[];     // [kBfWarps][32 x 33 + 32 x C]
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int w = blockIdx.x * kBfWarps + wib;
    if (w >= ngroups) return;
    const BfRGroup gr = groups[w];
    const double *ubuf = depth_par[gr.m * 2 + gr.t] ? u1 : u0;
    shtb_dev::bf_adj_r_rec_group<NB>(gr, v, ritems, rs, ints, ubuf, reinterpret_cast<const double *>(g), nmaps, b0,
                                     reinterpret_cast<double *>(aacc),
                                     smem_rec + (size_t)wib * (32 * 33 + 32 * 2 * NB), lane);
}

// alm[b][idx] = c_m aacc[idx][b] (c_0 = 1 with Im a_l0 = 0, c_m = 2), the
// transposed staging of bf_interleave_kernel; times sigma_lm when sig is
// non-null (plans that regenerate R: the residual adjoint sums V, not
// Ptilde = sigma V)
__global__ void __launch_bounds__(256) bf_finish_kernel(PlanView v, const double2 *__restrict__ aacc,
                                                        double2 *__restrict__ alm, int nmaps,
                                                        const RecCoef *__restrict__ sig)
{
    __shared__ double2 tile[2 * kStageTile];
    const long long nalm = v.nalm, L = v.lmax;
    auto scaled = [L, sig](double2 a, long long idx) {
        const double cs = (idx <= L ? 1.0 : 2.0) * (sig ? sig[idx].sig : 1.0);
        return idx <= L ? make_double2(sig ? a.x * cs : a.x, 0.0)
                        : make_double2(sig ? cs * a.x : 2.0 * a.x, sig ? cs * a.y : 2.0 * a.y);
    };
    if (nmaps == 1) {
        for (long long i = blockIdx.x * 256LL + threadIdx.x; i < nalm; i += 256LL * gridDim.x)
            alm[i] = scaled(aacc[i], i);
        return;
    }
    const StageTile st(nmaps);
    for (long long i0 = (long long)blockIdx.x * st.T; i0 < nalm; i0 += (long long)st.T * gridDim.x) {
        const int nt = (int)min((long long)st.T, nalm - i0);
        for (int b0 = 0; b0 < nmaps; b0 += st.MB) {
            const int mb = min(st.MB, nmaps - b0);
            for (int e = threadIdx.x; e < nt * mb; e += blockDim.x) {
                const int t = e / mb, b = e - t * mb;
                tile[b * (st.T + 1) + t] = aacc[(size_t)(i0 + t) * nmaps + b0 + b];
            }
            __syncthreads();
            for (int e = threadIdx.x; e < nt * mb; e += blockDim.x) {
                const int b = e / nt, t = e - b * nt;
                alm[(size_t)(b0 + b) * nalm + i0 + t] = scaled(tile[b * (st.T + 1) + t], i0 + t);
            }
            __syncthreads();
        }
    }
}

template <int NB>
int run_adj_group(const shtb_plan_s *p, const double2 *g, int nmaps, int b0, double *u0, double *u1,
                  double2 *aacc, cudaStream_t st)
{
    const BfPlanDev &bf = *p->bf;
    for (int lev = 1; lev <= bf.depth_max; ++lev) {
        const int n = bf.level_counts[lev - 1];
        if (n == 0) continue;
        const double *uin = ((lev - 1) % 2) ? u1 : u0;
        double *uout = (lev % 2) ? u1 : u0;
        const unsigned grid = (unsigned)((n + kBfWarps - 1) / kBfWarps);
        const size_t smem = sizeof(double) * kBfWarps * shtb::kMaxCand * 2 * NB;
        SHTB_CUDA_TRY(cudaFuncSetAttribute(bf_adj_level_kernel<NB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        bf_adj_level_kernel<NB><<<grid, 32 * kBfWarps, smem, st>>>(bf.level_items[lev - 1], n, bf.ints,
                                                                   bf.dbl, uin, g, nmaps, b0, uout);
        SHTB_CUDA_TRY(cudaGetLastError());
        ++p->launches;
    }
    if (bf.n_rgroups > 0 && bf.rec) {
        const unsigned grid = (unsigned)((bf.n_rgroups + kBfWarps - 1) / kBfWarps);
        const size_t smem = sizeof(double) * kBfWarps * (32 * 33 + 32 * 2 * NB);
        SHTB_CUDA_TRY(cudaFuncSetAttribute(bf_adj_r_rec_kernel<NB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        bf_adj_r_rec_kernel<NB><<<grid, 32 * kBfWarps, smem, st>>>(p->view, bf.rgroups, bf.n_rgroups, bf.ritems,
                                                                   bf.rstart, bf.ints, u0, u1, bf.depth_parity,
                                                                   g, nmaps, b0, aacc);
        SHTB_CUDA_TRY(cudaGetLastError());
        ++p->launches;
    } else if (bf.n_rgroups > 0) {
        const unsigned grid = (unsigned)((bf.n_rgroups + kBfWarps - 1) / kBfWarps);
        bf_adj_r_kernel<NB><<<grid, 32 * kBfWarps, 0, st>>>(p->view, bf.rgroups, bf.n_rgroups, bf.ritems,
                                                            bf.ints, bf.dbl, u0, u1, bf.depth_parity, g,
                                                            nmaps, b0, aacc);
        SHTB_CUDA_TRY(cudaGetLastError());
        ++p->launches;
    }
    return SHTB_OK;
}

}  // namespace

size_t bf_workspace_bytes(const shtb_plan_s *p)
{
    if (!p->bf) return 0;
    const size_t entry = sizeof(double) * 16;   // up to 8 maps x (re, im) per group
    return (2 * (size_t)p->bf->u_entries + (size_t)p->bf->qt_entries) * entry + 512;
}

int launch_bf_synth(const shtb_plan_s *p, const double2 *alm, double2 *ai, void *ws, double *map,
                    int nmaps, cudaStream_t st, double *qt_out)
{
    const BfPlanDev &bf = *p->bf;
    const size_t entry = 16;
    double *u0 = (double *)ws;
    double *u1 = u0 + (size_t)bf.u_entries * entry;
    double *qt_ws = u1 + (size_t)bf.u_entries * entry;
    // q^t of map b in the caller's [nmaps][2][nhalf][L+1] array (Legendre stage alone)
    const size_t qt_map = (size_t)4 * p->nhalf * (p->lmax + 1);
    auto qt_of = [&](int b0) { return qt_out ? qt_out + (size_t)b0 * qt_map : qt_ws; };
    const int ev = profile_begin(const_cast<shtb_plan_s *>(p), st);
    bf_interleave_kernel<<<stage_grid(p, nmaps), 256, 0, st>>>(p->view, alm, ai, nmaps,
                                                               p->bf->rec ? p->view.coef : nullptr);
    SHTB_CUDA_TRY(cudaGetLastError());
    ++p->launches;
    profile_end(const_cast<shtb_plan_s *>(p), st, 4, ev);
    for (int b0 = 0; b0 < nmaps;) {
        const int left = nmaps - b0;
        int rc;
        double *qt = qt_of(b0);
        if (left >= 8) { rc = run_group<8>(p, ai, nmaps, b0, u0, u1, qt, map, st); b0 += 8; }
        else if (left >= 4) { rc = run_group<4>(p, ai, nmaps, b0, u0, u1, qt, map, st); b0 += 4; }
        else if (left >= 2) { rc = run_group<2>(p, ai, nmaps, b0, u0, u1, qt, map, st); b0 += 2; }
        else { rc = run_group<1>(p, ai, nmaps, b0, u0, u1, qt, map, st); b0 += 1; }
        if (rc) return rc;
    }
    return SHTB_OK;
}

int launch_bf_synth_to_host(shtb_plan_s *p, const double2 *alm, double2 *ai, void *ws, double *map,
                            double *map_host, int nmaps, cudaStream_t st)
{
    constexpr int NCH = shtb_plan_s::kPhiChunks;
    if (!p->copy_stream) {
        SHTB_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
        for (auto &e : p->chunk_ev) SHTB_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const BfPlanDev &bf = *p->bf;
    const size_t entry = 16;
    double *u0 = (double *)ws;
    double *u1 = u0 + (size_t)bf.u_entries * entry;
    double *qt = u1 + (size_t)bf.u_entries * entry;
    bf_interleave_kernel<<<stage_grid(p, nmaps), 256, 0, st>>>(p->view, alm, ai, nmaps,
                                                               p->bf->rec ? p->view.coef : nullptr);
    SHTB_CUDA_TRY(cudaGetLastError());
    ++p->launches;
    for (int b0 = 0; b0 < nmaps;) {
        const int left = nmaps - b0;
        const int nb = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        int rc = launch_bf_legendre_group(p, ai, nmaps, b0, nb, u0, u1, qt, st);
        if (rc) return rc;
        // ring stage chunk by chunk; each chunk's pixels go back while the
        // next chunk (or the next map group) computes
        for (int c = 0; c < NCH; ++c) {
            if ((rc = launch_phi_synth_qt_chunk(p, qt, nb, map, b0, c, st))) return rc;
            const long long p0 = p->chunk_pix[c], p1 = p->chunk_pix[c + 1];
            if (p1 == p0) continue;
            SHTB_CUDA_TRY(cudaEventRecord(p->chunk_ev[c], st));
            SHTB_CUDA_TRY(cudaStreamWaitEvent(p->copy_stream, p->chunk_ev[c], 0));
            for (int b = b0; b < b0 + nb; ++b)
                SHTB_CUDA_TRY(cudaMemcpyAsync(map_host + (size_t)b * p->npix + p0, map + (size_t)b * p->npix + p0,
                                              sizeof(double) * (size_t)(p1 - p0), cudaMemcpyDeviceToHost,
                                              p->copy_stream));
        }
        b0 += nb;
    }
    // the caller's stream completes after the last copy
    SHTB_CUDA_TRY(cudaEventRecord(p->chunk_ev[0], p->copy_stream));
    SHTB_CUDA_TRY(cudaStreamWaitEvent(st, p->chunk_ev[0], 0));
    return SHTB_OK;
}

int launch_bf_adjoint(const shtb_plan_s *p, const double2 *g, double2 *aacc, void *ws, double2 *alm,
                      int nmaps, cudaStream_t st)
{
    const BfPlanDev &bf = *p->bf;
    const size_t entry = 16;
    double *u0 = (double *)ws;
    double *u1 = u0 + (size_t)bf.u_entries * entry;
    for (int b0 = 0; b0 < nmaps;) {
        const int left = nmaps - b0;
        int rc;
        if (left >= 8) { rc = run_adj_group<8>(p, g, nmaps, b0, u0, u1, aacc, st); b0 += 8; }
        else if (left >= 4) { rc = run_adj_group<4>(p, g, nmaps, b0, u0, u1, aacc, st); b0 += 4; }
        else if (left >= 2) { rc = run_adj_group<2>(p, g, nmaps, b0, u0, u1, aacc, st); b0 += 2; }
        else { rc = run_adj_group<1>(p, g, nmaps, b0, u0, u1, aacc, st); b0 += 1; }
        if (rc) return rc;
    }
    bf_finish_kernel<<<stage_grid(p, nmaps), 256, 0, st>>>(p->view, aacc, alm, nmaps,
                                                           p->bf->rec ? p->view.coef : nullptr);
    SHTB_CUDA_TRY(cudaGetLastError());
    ++p->launches;
    return SHTB_OK;
}

int launch_bf_gather(const shtb_plan_s *p, const double2 *const *alm_of_map, double2 *ai, int nmaps,
                     cudaStream_t st)
{
    bf_gather_kernel<<<p->lmax + 1, 256, 0, st>>>(p->view, alm_of_map, ai, nmaps);
    SHTB_CUDA_TRY(cudaGetLastError());
    ++p->launches;
    return SHTB_OK;
}

int launch_bf_legendre_group(const shtb_plan_s *p, const double2 *ai, int nmaps, int b0, int nb, double *u0,
                             double *u1, double *qt, cudaStream_t st)
{
    int rc;
    switch (nb) {
    case 8: if ((rc = launch_r<8>(p, ai, nmaps, b0, u0, u1, qt, st))) return rc;
            return launch_levels<8>(p, u0, u1, qt, st);
    case 4: if ((rc = launch_r<4>(p, ai, nmaps, b0, u0, u1, qt, st))) return rc;
            return launch_levels<4>(p, u0, u1, qt, st);
    case 2: if ((rc = launch_r<2>(p, ai, nmaps, b0, u0, u1, qt, st))) return rc;
            return launch_levels<2>(p, u0, u1, qt, st);
    case 1: if ((rc = launch_r<1>(p, ai, nmaps, b0, u0, u1, qt, st))) return rc;
            return launch_levels<1>(p, u0, u1, qt, st);
    default: return shtb_fail(SHTB_EINVAL, "map group width must be 1, 2, 4 or 8");
    }
}
