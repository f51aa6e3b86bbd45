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
// Entries fit 32 bits (e < 2 (L + 1) nhalf), so the split of e runs as a
// 32-bit division.
__device__ __forceinline__ size_t qt_index(int e, int nhalf, int L, int c)
{
    const unsigned mt = (unsigned)e / (unsigned)nhalf, r = (unsigned)e - mt * (unsigned)nhalf;
    const unsigned m = mt >> 1, t = mt & 1;
    const unsigned b = (unsigned)c >> 1;
    return ((((size_t)b * 2 + t) * nhalf + r) * (L + 1) + m) * 2 + (c & 1);
}

__device__ __forceinline__ void qt_store(double *qt, int e, int nhalf, int L, int c, double v)
{
    qt[qt_index(e, nhalf, L, c)] = v;
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

// ---- level items with few maps (C = 2 NB <= 4): packed dot products.
// Every output of a residual block (one column) and of a level child (one
// dense row) is a dot product from zero over its inputs in order, whatever
// the map count, so the results do not depend on how maps are grouped.  With
// C <= 4 components a lane owns all components of its dot products (one load
// of the operator feeds C FMAs), and the products of several children share
// the warp: group g gets ceil(njobs_g / R) contiguous lanes, R the fewest
// rounds that fit all groups on 32 lanes, and each lane runs its R products
// side by side over the warp's longest input length (shorter groups idle
// there).  Up to 4 (8) products per lane share each input load.

// njobs dot products of length len: product x reads element i at
// T[i * ld + x] and the NB complex inputs of entry i at v + i * vstep.
struct DotGroup {
    const double *T;
    const double2 *v;
    int len, njobs, ld, vstep;
};

// Sink: select(q) binds the lane's group (q a compile-time index after
// unrolling), key(x) fetches what put needs to place product x, put(key, x,
// acc) stores its C sums.
template <int NB, int NR, bool CG, class Sink>
__device__ __forceinline__ void packed_pass(const double *__restrict__ T, const double2 *v, int len, int ld,
                                            int vstep, int kmax, int x0, int nl, int njobs, Sink &sink)
{
    constexpr int C = 2 * NB;
    double acc[NR][C];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] = 0.0;
    bool ok[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) ok[r] = x0 + r * nl < njobs;
    const double *__restrict__ Ti = T + x0;
    const double2 *vi = v;
#pragma unroll 2
    for (int i = 0; i < kmax; ++i) {
        const bool on = i < len;
        double2 u[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            u[b] = make_double2(0.0, 0.0);
            if (on) u[b] = CG ? __ldcg(vi + b) : __ldg(vi + b);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            double t = 0.0;
            if (on && ok[r]) t = __ldg(Ti + r * nl);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                acc[r][2 * b] = fma(t, u[b].x, acc[r][2 * b]);
                acc[r][2 * b + 1] = fma(t, u[b].y, acc[r][2 * b + 1]);
            }
        }
        Ti += ld;
        vi += vstep;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r)
        if (ok[r]) {
            const int x = x0 + r * nl;
            sink.put(sink.key(x), x, acc[r]);
        }
}

template <int NB, int NR, bool CG, class Sink>
__device__ __forceinline__ void packed_pass_dispatch(int nr, const double *T, const double2 *v, int len, int ld,
                                                     int vstep, int kmax, int x0, int nl, int njobs, Sink &sink)
{
    if constexpr (NR > 1) {
        if (nr < NR) {
            packed_pass_dispatch<NB, NR - 1, CG>(nr, T, v, len, ld, vstep, kmax, x0, nl, njobs, sink);
            return;
        }
    }
    packed_pass<NB, NR, CG>(T, v, len, ld, vstep, kmax, x0, nl, njobs, sink);
}

template <int NB, int NG, bool CG, class Sink>
__device__ __forceinline__ void packed_dots(const DotGroup (&g)[NG], int lane, Sink &sink)
{
    static_assert(NG <= 32, "one lane per group at least");
    constexpr int NRMAX = NB == 1 ? 4 : 2;       // rounds per pass
    int kmax = 0, jobs = 0;
#pragma unroll
    for (int q = 0; q < NG; ++q)
        if (g[q].len > 0 && g[q].njobs > 0) {
            kmax = max(kmax, g[q].len);
            jobs += g[q].njobs;
        }
    if (kmax == 0) return;
    int R = max(1, (jobs + 31) / 32);
    for (;; ++R) {
        int need = 0;
#pragma unroll
        for (int q = 0; q < NG; ++q)
            if (g[q].len > 0 && g[q].njobs > 0) need += (g[q].njobs + R - 1) / R;
        if (need <= 32) break;
    }
    int x0 = 0, nl = 1, njobs = 0, len = 0, ld = 0, vstep = 0;
    const double *T = nullptr;
    const double2 *v = nullptr;
    int l0 = 0;
#pragma unroll
    for (int q = 0; q < NG; ++q) {
        const int n = g[q].len > 0 && g[q].njobs > 0 ? (g[q].njobs + R - 1) / R : 0;
        if (lane >= l0 && lane < l0 + n) {
            sink.select(q);
            x0 = lane - l0;
            nl = n;
            njobs = g[q].njobs;
            len = g[q].len;
            ld = g[q].ld;
            vstep = g[q].vstep;
            T = g[q].T;
            v = g[q].v;
        }
        l0 += n;
    }
    for (int r0 = 0; r0 < R; r0 += NRMAX)
        packed_pass_dispatch<NB, NRMAX, CG>(min(NRMAX, R - r0), T, v, len, ld, vstep, kmax, x0 + r0 * nl, nl,
                                            njobs, sink);
}

// ---- residual blocks with few maps: dot products packed in rounds.  One
// warp takes the columns of several blocks (each column, per real component,
// a dot product from zero over the block's rows in order, as above): a lane
// owns CPL components of one column (S = C / CPL lanes per column), the
// warp's columns are ordered by length, longest first, and cut into rounds of
// 32 lanes; a round runs over its longest column, so columns of similar
// length share a round and few FMA slots idle.  (Tried on the level items
// too, where every lane loading its own input for one product measured
// slower than the packing above.)

// Group descriptor, held by lane q for group q: rows dot products of length
// len, row x reading element i at T[i * ld + x] and the components of input
// entry i at v + i * vstep (doubles); row x lands on output slot pos[x] (x
// when pos is null), slot s at base[s * C + c], or at q^t entry ent[s] when
// base is null.
struct RoundGroup {
    const double *T;
    const double *v;
    const int *pos;
    double *base;
    const int *ent;
    int len, rows, ld, vstep;
};

template <class P>
__device__ __forceinline__ P shfl_ptr(P p, int src)
{
    return (P)__shfl_sync(0xffffffffu, (unsigned long long)p, src);
}

// address of component c of q^t entry e (see qt_store)
__device__ __forceinline__ double *qt_ptr(double *qt, int e, int nhalf, int L, int c)
{
    return qt + qt_index(e, nhalf, L, c);
}

template <int C>
__device__ __forceinline__ double *slot_ptr(double *base, const int *ent, int slot, int c, double *qt, int nhalf,
                                            int L)
{
    return base ? base + (size_t)slot * C + c : qt_ptr(qt, __ldg(ent + slot), nhalf, L, c);
}

// The rows of the NG groups (lane q < NG holds group q in g) on one warp;
// ADD: outputs are added to what is there, else stored.
template <int NB, int CPL, int NG, bool CG, bool ADD>
__device__ __forceinline__ void round_dots(const RoundGroup &g, int L, int nhalf, double *qt,
                                           const double *safe, int lane)
{
    constexpr int C = 2 * NB, S = C / CPL;
    static_assert(NG <= 32 && S * CPL == C, "lane layout");
    // every lane: each group's length and lane count, then the groups ordered
    // by length (longest first, ties by index) and their first lanes
    int len[NG], jobs[NG];
#pragma unroll
    for (int q = 0; q < NG; ++q) {
        len[q] = __shfl_sync(0xffffffffu, lane < NG ? g.len : 0, q);
        const int rows = __shfl_sync(0xffffffffu, lane < NG ? g.rows : 0, q);
        jobs[q] = len[q] > 0 ? S * rows : 0;
        if (jobs[q] == 0) len[q] = 0;
    }
    int start[NG], total = 0;
#pragma unroll
    for (int q = 0; q < NG; ++q) {
        int st = 0;
#pragma unroll
        for (int p = 0; p < NG; ++p)
            if (len[p] > len[q] || (len[p] == len[q] && p < q)) st += jobs[p];
        start[q] = st;
        total += jobs[q];
    }
    for (int r0 = 0; r0 < total; r0 += 32) {
        const int rho = r0 + lane;
        int q = -1;
#pragma unroll
        for (int p = 0; p < NG; ++p)
            if (rho >= start[p] && rho < start[p] + jobs[p]) q = p;
        const int src = q < 0 ? 0 : q;
        const double *__restrict__ T = shfl_ptr(g.T, src);
        const double *v = shfl_ptr(g.v, src);
        const int ld = __shfl_sync(0xffffffffu, g.ld, src);
        const int vstep = __shfl_sync(0xffffffffu, g.vstep, src);
        const int *pos = shfl_ptr(g.pos, src);
        double *base = shfl_ptr(g.base, src);
        const int *ent = shfl_ptr(g.ent, src);
        int mylen = 0, x = 0, c0 = 0;
#pragma unroll
        for (int p = 0; p < NG; ++p)
            if (p == q) {
                mylen = len[p];
                x = (rho - start[p]) / S;
                c0 = (rho - start[p] - x * S) * CPL;
            }
        const int kmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)mylen);
        const int slot = q >= 0 && pos ? __ldg(pos + x) : x;      // issued before the sums
        double acc[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[c] = 0.0;
        const double *__restrict__ Ti = T + x;
        const double *vi = v + c0;
        // blocks of U inputs: all U loads issued before their FMAs (past its
        // own length a lane reads a fixed valid, 16-byte aligned address and
        // adds zero products); FMAs past the round's longest input are skipped
        constexpr int U = 8;
        for (int i0 = 0; i0 < kmax; i0 += U) {
            double t[U], u[U][CPL];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const bool on = i0 + j < mylen;
                const double tl = __ldg(on ? Ti : safe);
                if constexpr (CPL == 1) {
                    const double w = CG ? __ldcg(on ? vi : safe) : __ldg(on ? vi : safe);
                    u[j][0] = on ? w : 0.0;
                } else {
                    const double2 *w2 = reinterpret_cast<const double2 *>(on ? vi : safe);
                    const double2 w = CG ? __ldcg(w2) : __ldg(w2);
                    u[j][0] = on ? w.x : 0.0;
                    u[j][1] = on ? w.y : 0.0;
                }
                t[j] = on ? tl : 0.0;
                Ti += ld;
                vi += vstep;
            }
#pragma unroll
            for (int j = 0; j < U; ++j) {
                if (i0 + j >= kmax) break;
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[c] = fma(t[j], u[j][c], acc[c]);
            }
        }
        if (q >= 0) {
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                double *o = slot_ptr<C>(base, ent, slot, c0 + c, qt, nhalf, L);
                *o = ADD ? *o + acc[c] : acc[c];
            }
        }
    }
}

// Up to G residual blocks on one warp at C = 2 NB <= 4 (items[q] for
// q < n): u_s = sum_j R[j][s] a_j, column s of each block one dot product.
// Block q writes u1 if depth_par (non-null) marks its chain's depth odd,
// else u0.
template <int NB, int G, bool CG>
__device__ __forceinline__ void bf_r_items_few(const BfRItem *__restrict__ items, int n, int L, int nhalf,
                                               const int *__restrict__ ints, const double *__restrict__ dbl,
                                               const double2 *ai, int nmaps, int b0, double *u0, double *u1,
                                               const int *__restrict__ depth_par, double *qt, int lane)
{
    constexpr int C = 2 * NB;
    // one component per lane at one map, one map's pair at two
    constexpr int CPL = NB == 1 ? 1 : 2;
    RoundGroup g{};
    if (lane < n) {
        const BfRItem it = items[lane];
        const long long aoff = alm_off(L, it.m) + it.t + 2 * it.j0;
        double *ubuf = depth_par && depth_par[it.m * 2 + it.t] ? u1 : u0;
        g.T = dbl + it.data_off;
        g.v = reinterpret_cast<const double *>(ai + (size_t)aoff * nmaps + b0);
        g.pos = nullptr;
        g.base = it.to_rings ? nullptr : ubuf + (size_t)it.out_off * C;
        g.ent = it.to_rings ? ints + it.out_off : nullptr;
        g.len = it.nrows;
        g.rows = it.k;
        g.ld = it.k;
        g.vstep = 4 * nmaps;
    }
    // a block without rows (a cropped chain range) still writes its columns:
    // zero sums
#pragma unroll
    for (int q = 0; q < G; ++q) {
        const int len = __shfl_sync(0xffffffffu, g.len, q), rows = __shfl_sync(0xffffffffu, g.rows, q);
        double *base = shfl_ptr(g.base, q);
        const int *ent = shfl_ptr(g.ent, q);
        if (q >= n || len > 0) continue;
        for (int x = lane; x < rows * C; x += 32)
            *slot_ptr<C>(base, ent, x / C, x % C, qt, nhalf, L) = 0.0;
    }
    round_dots<NB, CPL, G, CG, false>(g, L, nhalf, qt, dbl, lane);
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
        bf_r_items_few<NB, 1, CG>(&it, 1, L, nhalf, ints, dbl, ai, nmaps, b0, ubuf, ubuf, nullptr, qt, lane);
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
// out: this warp's shared-memory scratch of nc x level_scratch_per_cand(C)
// doubles (from 4 maps up, rows of C + 1: the odd stride spreads the lanes'
// rows over the banks).
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

// Level-item scratch per candidate (doubles) and map group: C + 1 (one
// padded row per candidate) from 4 maps up; with fewer maps each child sums
// into its own zeroed nc x C half, so 2 C.
__host__ __device__ constexpr int level_scratch_per_cand(int C)
{
    return C <= 4 ? 2 * C : C + 1;
}

// level children: dense row x of child h lands on its candidate position in
// that child's half of the item's scratch
template <int NB, int NG>
struct LSink {
    static constexpr int C = 2 * NB;
    double *S[NG];
    const int *pos[NG];
    double *my_S;
    const int *my_pos;
    __device__ __forceinline__ void select(int q)
    {
        my_S = S[q];
        my_pos = pos[q];
    }
    __device__ __forceinline__ int key(int x) const { return __ldg(my_pos + x); }
    __device__ __forceinline__ void put(int key, int, const double (&acc)[C]) const
    {
#pragma unroll
        for (int c = 0; c < C; ++c) my_S[key * C + c] = acc[c];
    }
};

// Up to G level items (it[q] for q < n) on one warp at C = 2 NB <= 4.  Each
// child h sums into its own zeroed half S_h (identity entries copied, dense
// rows as packed dot products); the output is S_0 + S_1, which is what the
// wider groups' store-then-add order gives, bit for bit: 0 + v = v, and a
// position with both children is c_0 + c_1 in both.  scr: G x 2 x maxnc x C
// doubles of this warp's shared memory.
template <int NB, int G, bool CG>
__device__ __forceinline__ void bf_level_items_few(const BfItem (&it)[G], int n, int L, int nhalf,
                                                   const int *__restrict__ ints, const double *__restrict__ dbl,
                                                   const double *uin, double *uout, double *qt, double *scr,
                                                   int maxnc, int lane)
{
    constexpr int C = 2 * NB;
    DotGroup g[2 * G];
    LSink<NB, 2 * G> sink;
#pragma unroll
    for (int q = 0; q < G; ++q) {
        const int nc = q < n ? it[q].nc : 0;
        double *S0 = scr + (size_t)q * 2 * maxnc * C;
        for (int i = lane; i < 2 * nc * C; i += 32) S0[i] = 0.0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const bool on = q < n;
            const double *u = uin + (on ? (size_t)it[q].u_off[h] * C : 0);
            DotGroup &d = g[2 * q + h];
            d.T = dbl + (on ? it[q].T_off[h] : 0);
            d.v = reinterpret_cast<const double2 *>(u);
            d.len = on ? it[q].k[h] : 0;
            d.njobs = on ? it[q].nd[h] : 0;
            d.ld = d.njobs;
            d.vstep = NB;
            sink.S[2 * q + h] = S0 + (size_t)h * nc * C;
            sink.pos[2 * q + h] = ints + (on ? it[q].dpos_off[h] : 0);
        }
    }
    __syncwarp();
    // identity entries (positions distinct from the same child's dense rows)
#pragma unroll
    for (int q = 0; q < G; ++q) {
        if (q >= n) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double *u = uin + (size_t)it[q].u_off[h] * C;
            const int *__restrict__ ipos = ints + it[q].ipos_off[h];
            double *S = sink.S[2 * q + h];
            for (int x = lane; x < it[q].k[h] * C; x += 32) {
                const int i = x / C, cc = x - i * C;
                S[ipos[i] * C + cc] = ldp<CG>(u + x);
            }
        }
    }
    packed_dots<NB, 2 * G, CG>(g, lane, sink);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < G; ++q) {
        if (q >= n) break;
        const int nc = it[q].nc;
        const double *S0 = sink.S[2 * q], *S1 = S0 + (size_t)nc * C;
        if (it[q].to_rings) {
            const int *__restrict__ ent = ints + it[q].out_off;
            for (int i = lane; i < nc * C; i += 32) {
                const int cpos = i / C, cc = i - cpos * C;
                qt_store(qt, ent[cpos], nhalf, L, cc, S0[i] + S1[i]);
            }
        } else {
            double *dst = uout + (size_t)it[q].out_off * C;
            for (int i = lane; i < nc * C; i += 32) dst[i] = S0[i] + S1[i];
        }
    }
    __syncwarp();
}

// Each child in turn: its dense rows (passes of up to LD x NRMAX rows, the
// per-lane row count exact), then its identity entries.  A child's dense and
// identity positions are distinct, so lanes never update the same scratch
// entry within a child; the warp syncs between the children, whose positions
// may coincide.
// RING: 1 when every item of the launch writes q^t (the plan's level 1), 0
// when none does, -1 to follow each item's to_rings flag.
template <int NB, bool CG, int RING = -1>
__device__ __forceinline__ void bf_level_item_wide(const BfItem &it, int L, int nhalf, const int *__restrict__ ints,
                                                   const double *__restrict__ dbl, const double *uin,
                                                   double *uout, double *qt, double *out, int lane)
{
    constexpr int C = 2 * NB, LD = Lanes<C>::LD, NRMAX = Lanes<C>::NRMAX;
    constexpr int OS = out_stride<C>();
    for (int i = lane; i < it.nc * OS; i += 32) out[i] = 0.0;
    __syncwarp();
    const int dl = lane % LD, c = lane / LD;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
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
    if (RING == 1 || (RING < 0 && it.to_rings)) {
        const int *__restrict__ ent = ints + it.out_off;
        for (int i = lane; i < it.nc * C; i += 32) {
            const int cpos = i / C, cc = i - cpos * C;
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

template <int NB, bool CG, int RING = -1>
__device__ __forceinline__ void bf_level_item(const BfItem &it, int L, int nhalf, const int *__restrict__ ints,
                                              const double *__restrict__ dbl, const double *uin,
                                              double *uout, double *qt, double *out, int lane)
{
    if constexpr (NB <= 2) {
        const BfItem one[1] = {it};
        bf_level_items_few<NB, 1, CG>(one, 1, L, nhalf, ints, dbl, uin, uout, qt, out, it.nc, lane);
    } else {
        bf_level_item_wide<NB, CG, RING>(it, L, nhalf, ints, dbl, uin, uout, qt, out, lane);
    }
}

}  // namespace shtb_dev
