// Kernel (b): the Legendre stage by the jump-two recurrence of Eq. (three-term),
// uncompressed ("zero levels of compression", Sec. 3.3) and split by l - m
// parity over rings mirrored about the equator (Eq. q-even-odd, q-even-odd2).
//
// Synthesis: for every order m and half-ring r (z_r >= 0)
//   q^t_m(z_r) = sum_j a_{m+t+2j, m} Ptilde_{m+t+2j}^m(z_r),  t = 0 (even), 1 (odd),
// then q_m(+z_r) = q^0 + q^1 and q_m(-z_r) = q^0 - q^1 (the mirror ring).
// A warp owns 32 consecutive half-rings of one m, each lane runs both parity
// chains of its ring in registers and accumulates all maps of the batch, so
// the per-l constants and a_lm are warp-uniform (broadcast) loads.  Each
// chain starts at its own crop point (first |Ptilde| >= 1e-30, Appendix) with
// two precomputed values and advances by two FMAs per step:
//   w_j = mu_j x_r + C_j,   V_{j+1} = w_j V_j - V_{j-1},   Ptilde = sigma V,
// the scale sigma being folded into a_lm by the prescale kernel.
//
// Adjoint: a^t_{m+t+2j} = sum_r V_j(r) g^t_r with g^0 = F(+z) + F(-z) and
// g^1 = F(+z) - F(-z).  The sum runs across the rings, i.e. across lanes, so
// each warp writes a 32 (j) x 32 (ring) tile of V to shared memory and then
// lets lane = j accumulate over the tile's rings with FMAs; the partial sums
// of a block's warps are added in shared memory and written once.
#include <cuda_runtime.h>

#include "shtb_internal.h"

namespace {

constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ int warp_min(int v)
{
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ int dchain_len(int L, int m, int t)
{
    return m + t > L ? 0 : (L - m - t) / 2 + 1;
}

__device__ __forceinline__ long long dalm_index(int L, int l, int m)
{
    return (long long)m * (2 * L + 1 - m) / 2 + l;
}

// a'[idx][b] = a_lm[b][idx] * sigma_lm   (Im a_l0 dropped: real-field input, Sec. 2.1)
__global__ void alm_prescale_kernel(PlanView v, const double2 *__restrict__ alm,
                                    double2 *__restrict__ ap, int nmaps)
{
    const int m = blockIdx.x;
    const int L = v.lmax;
    const long long off = dalm_index(L, m, m);
    const int n = L - m + 1;
    for (int i = threadIdx.x; i < n * nmaps; i += blockDim.x) {
        const int b = i / n, dl = i - b * n;
        const long long idx = off + dl;
        double2 a = alm[(size_t)b * v.nalm + idx];
        const double s = v.coef[idx].sig;
        ap[(size_t)idx * nmaps + b] = make_double2(a.x * s, m == 0 ? 0.0 : a.y * s);
    }
}

template <int NB>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
legendre_synth_kernel(PlanView v, const double2 *__restrict__ ap, double2 *__restrict__ q,
                      int nmaps, int b0)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int Z = v.nhalf, L = v.lmax;
    const int nchunk = (Z + 31) >> 5;
    const long long item = (long long)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= (long long)(L + 1) * nchunk) return;
    const int m = (int)(item / nchunk);
    const int chunk = (int)(item - (long long)m * nchunk);
    const int r = chunk * 32 + lane;
    const bool valid = r < Z;
    const int rr = valid ? r : Z - 1;
    const int n0 = dchain_len(L, m, 0), n1 = dchain_len(L, m, 1);

    const double x = v.xarg[rr];
    const bool sform = v.xform[rr] != 0;
    const size_t base0 = ((size_t)m * 2) * Z + rr, base1 = base0 + Z;
    const int js0 = valid ? v.jstart[base0] : n0;
    const int js1 = valid ? v.jstart[base1] : n1;
    const double2 s0 = v.vstart[base0], s1 = v.vstart[base1];

    int lo = n0;
    if (js0 < n0) lo = js0;
    if (js1 < n1) lo = min(lo, js1);
    const int jlo = warp_min(lo);
    if (jlo >= n0) {
        // nothing above the crop for any lane: q is zero for these rings
        if (valid) {
            for (int b = 0; b < NB; ++b) {
                double2 *qb = q + (size_t)(b0 + b) * v.nrings * (L + 1);
                qb[(size_t)r * (L + 1) + m] = make_double2(0.0, 0.0);
                if (r < Z - 1) qb[(size_t)(v.nrings - 1 - r) * (L + 1) + m] = make_double2(0.0, 0.0);
            }
        }
        return;
    }

    double2 acc0[NB], acc1[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        acc0[b] = make_double2(0.0, 0.0);
        acc1[b] = make_double2(0.0, 0.0);
    }
    double cur0 = (js0 == jlo) ? s0.x : 0.0, prev0 = 0.0;
    double cur1 = (js1 == jlo) ? s1.x : 0.0, prev1 = 0.0;

    const long long off = dalm_index(L, m, m);
    const RecCoef *__restrict__ cf = v.coef + off;
    const double2 *__restrict__ a = ap + (size_t)off * nmaps + b0;

    for (int j = jlo; j < n0; ++j) {
        // ---- even chain, l = m + 2j
        {
            const int dl = 2 * j;
            const double2 *aj = a + (size_t)dl * nmaps;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const double2 av = __ldg(aj + b);
                acc0[b].x = fma(av.x, cur0, acc0[b].x);
                acc0[b].y = fma(av.y, cur0, acc0[b].y);
            }
            const RecCoef c = cf[dl];
            const double w = fma(c.mu, x, sform ? c.cs : c.cz);
            double nxt = fma(w, cur0, -prev0);
            if (j == js0) nxt = s0.y;
            if (j + 1 == js0) nxt = s0.x;
            prev0 = cur0;
            cur0 = nxt;
        }
        // ---- odd chain, l = m + 1 + 2j
        if (j < n1) {
            const int dl = 2 * j + 1;
            const double2 *aj = a + (size_t)dl * nmaps;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const double2 av = __ldg(aj + b);
                acc1[b].x = fma(av.x, cur1, acc1[b].x);
                acc1[b].y = fma(av.y, cur1, acc1[b].y);
            }
            const RecCoef c = cf[dl];
            const double w = fma(c.mu, x, sform ? c.cs : c.cz);
            double nxt = fma(w, cur1, -prev1);
            if (j == js1) nxt = s1.y;
            if (j + 1 == js1) nxt = s1.x;
            prev1 = cur1;
            cur1 = nxt;
        }
    }

    if (!valid) return;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        double2 *qb = q + (size_t)(b0 + b) * v.nrings * (L + 1);
        qb[(size_t)r * (L + 1) + m] = make_double2(acc0[b].x + acc1[b].x, acc0[b].y + acc1[b].y);
        if (r < Z - 1)   // the equator ring (r = Z-1) has no mirror
            qb[(size_t)(v.nrings - 1 - r) * (L + 1) + m] =
                make_double2(acc0[b].x - acc1[b].x, acc0[b].y - acc1[b].y);
    }
}


// ------------------------------------------------------------------ adjoint
// g[((m*2 + t)*Z + r)*nmaps + b]: parity combination of the ring-stage
// adjoint output, g^0 = F(+z_r) + F(-z_r), g^1 = F(+z_r) - F(-z_r); the
// equator ring (r = Z-1) has no mirror and contributes once.
// One CTA per (half-ring r, run of 64 orders m): reads each map's run of q_adj
// on ring r and its mirror, and writes the maps of one (m, t, r) entry of g
// next to each other, up to 16 maps at a time.  Shared memory turns the
// map-major reads into the entry-major writes, so both are coalesced.
constexpr int kParityM = 64, kParityMaps = 16;

__global__ void __launch_bounds__(256) adjoint_parity_kernel(PlanView v, const double2 *__restrict__ qa,
                                                             double2 *__restrict__ g, int nmaps)
{
    __shared__ double2 tile[2][kParityMaps][kParityM];     // north, south
    const int r = blockIdx.x, m0 = blockIdx.y * kParityM;
    const int Z = v.nhalf, L = v.lmax;
    const int nm = min(kParityM, L + 1 - m0);
    const bool equator = r == Z - 1;
    for (int b0 = 0; b0 < nmaps; b0 += kParityMaps) {
        const int nb = min(kParityMaps, nmaps - b0);
        for (int i = threadIdx.x; i < nb * nm; i += blockDim.x) {
            const int b = i / nm, ml = i - b * nm;
            const size_t row = (size_t)(b0 + b) * v.nrings;
            tile[0][b][ml] = qa[(row + r) * (L + 1) + m0 + ml];
            tile[1][b][ml] = equator ? make_double2(0.0, 0.0) : qa[(row + (v.nrings - 1 - r)) * (L + 1) + m0 + ml];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb * nm; i += blockDim.x) {
            const int ml = i / nb, b = i - ml * nb;
            const double2 a = tile[0][b][ml], c = tile[1][b][ml];
            const size_t m = (size_t)(m0 + ml);
            g[((m * 2 + 0) * Z + r) * nmaps + b0 + b] = make_double2(a.x + c.x, a.y + c.y);
            g[((m * 2 + 1) * Z + r) * nmaps + b0 + b] = make_double2(a.x - c.x, a.y - c.y);
        }
        __syncthreads();
    }
}

constexpr int kAdjWarps = 4;
constexpr int kTilePad = 33;   // row stride (doubles) of the 32x32 tile: no bank conflicts

template <int NB>
__host__ __device__ constexpr size_t adjoint_warp_smem_doubles()
{
    return 2 * 32 * kTilePad + 2 * 32 * NB * 2;
}

template <int NB>
__global__ void __launch_bounds__(32 * kAdjWarps)
legendre_adjoint_kernel(PlanView v, const double2 *__restrict__ g, double2 *__restrict__ aacc,
                        RecState *__restrict__ state, int nmaps, int b0)
{
    extern __shared__ double smd[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int Z = v.nhalf, L = v.lmax;
    const int m = blockIdx.x;
    const int n0 = dchain_len(L, m, 0), n1 = dchain_len(L, m, 1);
    const int nchunk = (Z + 31) >> 5;
    const long long off = dalm_index(L, m, m);
    const RecCoef *__restrict__ cf = v.coef + off;
    double *tile = smd + (size_t)warp * adjoint_warp_smem_doubles<NB>();   // [2][32][kTilePad]
    double2 *gs = reinterpret_cast<double2 *>(tile + 2 * 32 * kTilePad);    // [2][32][NB]
    RecState *st = state + (size_t)blockIdx.x * Z;
    const int ntiles = (n0 + 31) >> 5;

    for (int ti = 0; ti < ntiles; ++ti) {
        const int jt = ti * 32;
        double2 acc0[NB], acc1[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            acc0[b] = make_double2(0.0, 0.0);
            acc1[b] = make_double2(0.0, 0.0);
        }
        for (int c = warp; c < nchunk; c += kAdjWarps) {
            const int r = c * 32 + lane;
            const bool valid = r < Z;
            const int rr = valid ? r : Z - 1;
            const size_t base0 = ((size_t)m * 2) * Z + rr, base1 = base0 + Z;
            const int js0 = valid ? v.jstart[base0] : n0;
            const int js1 = valid ? v.jstart[base1] : n1;
            int lo = n0;
            if (js0 < n0) lo = js0;
            if (js1 < n1) lo = min(lo, js1);
            const int clo = warp_min(lo);
            if (clo >= n0 || jt + 32 <= clo) continue;   // chunk is zero in this tile
            const double2 s0 = v.vstart[base0], s1 = v.vstart[base1];
            const double x = v.xarg[rr];
            const bool sform = v.xform[rr] != 0;
            double cur0, prev0, cur1, prev1;
            if (ti == (clo >> 5)) {
                cur0 = (js0 == jt) ? s0.x : 0.0;
                cur1 = (js1 == jt) ? s1.x : 0.0;
                prev0 = prev1 = 0.0;
            } else {
                const RecState sv = st[rr];
                cur0 = sv.cur0; prev0 = sv.prev0; cur1 = sv.cur1; prev1 = sv.prev1;
            }
            // phase 1: lane = ring; V_j for the tile's 32 chain steps
            for (int jj = 0; jj < 32; ++jj) {
                const int j = jt + jj;
                double e0 = 0.0, e1 = 0.0;
                if (j < n0) {
                    e0 = cur0;
                    const RecCoef cc = cf[2 * j];
                    const double w = fma(cc.mu, x, sform ? cc.cs : cc.cz);
                    double nxt = fma(w, cur0, -prev0);
                    if (j == js0) nxt = s0.y;
                    if (j + 1 == js0) nxt = s0.x;
                    prev0 = cur0;
                    cur0 = nxt;
                }
                if (j < n1) {
                    e1 = cur1;
                    const RecCoef cc = cf[2 * j + 1];
                    const double w = fma(cc.mu, x, sform ? cc.cs : cc.cz);
                    double nxt = fma(w, cur1, -prev1);
                    if (j == js1) nxt = s1.y;
                    if (j + 1 == js1) nxt = s1.x;
                    prev1 = cur1;
                    cur1 = nxt;
                }
                tile[jj * kTilePad + lane] = e0;
                tile[(32 + jj) * kTilePad + lane] = e1;
            }
            if (valid) {
                RecState sv;
                sv.cur0 = cur0; sv.prev0 = prev0; sv.cur1 = cur1; sv.prev1 = prev1;
                st[r] = sv;
            }
            for (int i = lane; i < 2 * 32 * NB; i += 32) {
                const int t = i / (32 * NB), rem = i - t * 32 * NB;
                const int r2 = rem / NB, b = rem - r2 * NB;
                const int ring = c * 32 + r2;
                gs[i] = ring < Z ? g[(((size_t)m * 2 + t) * Z + ring) * nmaps + b0 + b]
                                 : make_double2(0.0, 0.0);
            }
            __syncwarp();
            // phase 2: lane = chain step jj, sum over the tile's 32 rings
            const double *row0 = tile + lane * kTilePad;
            const double *row1 = tile + (32 + lane) * kTilePad;
            for (int r2 = 0; r2 < 32; ++r2) {
                const double V0 = row0[r2], V1 = row1[r2];
                const double2 *g0 = gs + r2 * NB, *g1 = gs + (32 + r2) * NB;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const double2 ga = g0[b], gb = g1[b];
                    acc0[b].x = fma(V0, ga.x, acc0[b].x);
                    acc0[b].y = fma(V0, ga.y, acc0[b].y);
                    acc1[b].x = fma(V1, gb.x, acc1[b].x);
                    acc1[b].y = fma(V1, gb.y, acc1[b].y);
                }
            }
            __syncwarp();
        }
        // add the warps' partial sums for this tile and store them
        __syncthreads();
        double2 *red = reinterpret_cast<double2 *>(smd);   // [warp][t][jj][b]
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            red[((warp * 2 + 0) * 32 + lane) * NB + b] = acc0[b];
            red[((warp * 2 + 1) * 32 + lane) * NB + b] = acc1[b];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 2 * 32 * NB; i += blockDim.x) {
            const int t = i / (32 * NB), rem = i - t * 32 * NB;
            const int jj = rem / NB, b = rem - jj * NB;
            const int j = jt + jj;
            if (j >= (t == 0 ? n0 : n1)) continue;
            double2 sum = make_double2(0.0, 0.0);
            for (int w = 0; w < kAdjWarps; ++w) {
                const double2 pv = red[((w * 2 + t) * 32 + jj) * NB + b];
                sum.x += pv.x;
                sum.y += pv.y;
            }
            aacc[(size_t)(off + t + 2 * j) * nmaps + b0 + b] = sum;
        }
        __syncthreads();
    }
}

// alm[b][idx] = c_m sigma_idx aacc[idx][b], c_0 = 1 (Im a_l0 = 0), c_m = 2
__global__ void alm_finish_kernel(PlanView v, const double2 *__restrict__ aacc,
                                  double2 *__restrict__ alm, int nmaps)
{
    const int m = blockIdx.x;
    const int L = v.lmax;
    const long long off = dalm_index(L, m, m);
    const int n = L - m + 1;
    const double cm = m == 0 ? 1.0 : 2.0;
    for (int i = threadIdx.x; i < n * nmaps; i += blockDim.x) {
        const int b = i / n, dl = i - b * n;
        const long long idx = off + dl;
        const double s = cm * v.coef[idx].sig;
        const double2 a = aacc[(size_t)idx * nmaps + b];
        alm[(size_t)b * v.nalm + idx] = make_double2(a.x * s, m == 0 ? 0.0 : a.y * s);
    }
}

template <int NB>
int launch_adjoint_nb(const shtb_plan_s *p, const double2 *g, double2 *aacc, RecState *state,
                      int nmaps, int b0, cudaStream_t st)
{
    const size_t smem = sizeof(double) * adjoint_warp_smem_doubles<NB>() * kAdjWarps;
    SHTB_CUDA_TRY(cudaFuncSetAttribute(legendre_adjoint_kernel<NB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    legendre_adjoint_kernel<NB><<<p->lmax + 1, 32 * kAdjWarps, smem, st>>>(p->view, g, aacc, state,
                                                                           nmaps, b0);
    ++p->launches;
    SHTB_CUDA_TRY(cudaGetLastError());
    return SHTB_OK;
}

}  // namespace

int launch_alm_prescale(const shtb_plan_s *p, const double2 *alm, double2 *ap, int nmaps,
                        cudaStream_t st)
{
    alm_prescale_kernel<<<p->lmax + 1, 256, 0, st>>>(p->view, alm, ap, nmaps);
    ++p->launches;
    SHTB_CUDA_TRY(cudaGetLastError());
    return SHTB_OK;
}

int launch_legendre_synth(const shtb_plan_s *p, const double2 *ap, double2 *q, int nmaps,
                          cudaStream_t st)
{
    const int nchunk = (p->nhalf + 31) / 32;
    const long long items = (long long)(p->lmax + 1) * nchunk;
    const unsigned grid = (unsigned)((items + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const dim3 block(32 * kWarpsPerBlock);
    for (int b0 = 0; b0 < nmaps;) {
        const int left = nmaps - b0;
        if (left >= 8) {
            legendre_synth_kernel<8><<<grid, block, 0, st>>>(p->view, ap, q, nmaps, b0);
            b0 += 8;
        } else if (left >= 4) {
            legendre_synth_kernel<4><<<grid, block, 0, st>>>(p->view, ap, q, nmaps, b0);
            b0 += 4;
        } else if (left >= 2) {
            legendre_synth_kernel<2><<<grid, block, 0, st>>>(p->view, ap, q, nmaps, b0);
            b0 += 2;
        } else {
            legendre_synth_kernel<1><<<grid, block, 0, st>>>(p->view, ap, q, nmaps, b0);
            b0 += 1;
        }
        SHTB_CUDA_TRY(cudaGetLastError());
        ++p->launches;
    }
    return SHTB_OK;
}

size_t legendre_adjoint_state_bytes(const shtb_plan_s *p)
{
    return sizeof(RecState) * (size_t)(p->lmax + 1) * p->nhalf;
}

int launch_adjoint_parity(const shtb_plan_s *p, const double2 *qadj, double2 *g, int nmaps,
                          cudaStream_t st)
{
    adjoint_parity_kernel<<<dim3(p->nhalf, (p->lmax + kParityM) / kParityM), 256, 0, st>>>(p->view, qadj, g,
                                                                                           nmaps);
    ++p->launches;
    SHTB_CUDA_TRY(cudaGetLastError());
    return SHTB_OK;
}

int launch_legendre_adjoint(const shtb_plan_s *p, const double2 *qadj, double2 *aacc, int nmaps,
                            void *ws, cudaStream_t st)
{
    // ws: [g: (L+1)*2*Z*nmaps double2][state: (L+1)*Z RecState]
    double2 *g = (double2 *)ws;
    RecState *state = (RecState *)(g + (size_t)(p->lmax + 1) * 2 * p->nhalf * nmaps);
    int rc0 = launch_adjoint_parity(p, qadj, g, nmaps, st);
    if (rc0) return rc0;
    for (int b0 = 0; b0 < nmaps;) {
        const int left = nmaps - b0;
        int rc;
        if (left >= 8) { rc = launch_adjoint_nb<8>(p, g, aacc, state, nmaps, b0, st); b0 += 8; }
        else if (left >= 4) { rc = launch_adjoint_nb<4>(p, g, aacc, state, nmaps, b0, st); b0 += 4; }
        else if (left >= 2) { rc = launch_adjoint_nb<2>(p, g, aacc, state, nmaps, b0, st); b0 += 2; }
        else { rc = launch_adjoint_nb<1>(p, g, aacc, state, nmaps, b0, st); b0 += 1; }
        if (rc) return rc;
    }
    return SHTB_OK;
}

int launch_alm_finish(const shtb_plan_s *p, const double2 *aacc, double2 *alm, int nmaps,
                      cudaStream_t st)
{
    alm_finish_kernel<<<p->lmax + 1, 256, 0, st>>>(p->view, aacc, alm, nmaps);
    ++p->launches;
    SHTB_CUDA_TRY(cudaGetLastError());
    return SHTB_OK;
}
