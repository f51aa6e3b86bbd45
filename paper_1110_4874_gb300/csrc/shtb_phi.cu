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
// One CTA per (ring, map); the ring's data live in shared memory.  K factoring
// over 2, 3, 5, 7, 11, 13: in-place mixed-radix FFT (radices 4, 2, 3, 5, 7,
// 11, 13) from position-order input.  Otherwise Bluestein's chirp transform
// through a convolution of 7-smooth length M >= 2K-1 (decimation in
// frequency, pointwise product with a precomputed filter in position order,
// decimation in time), so no permutation pass is needed.
#include <cuda_runtime.h>

#include "shtb_internal.h"
#include "shtb_phi_items.cuh"

namespace {

using namespace shtb_dev;

// threads per ring CTA: the Bluestein variant holds up to ~8.4k complex
// values of shared memory per CTA (one CTA per SM at the longest rings), so
// it runs twice the threads to keep the FP64 pipe fed
template <int KIND>
constexpr int phi_threads()
{
    return KIND == kBluestein ? 512 : 256;
}

// CTAs per SM the synthesis kernels are compiled for: the common mixed-radix
// kind fits in 64 registers without spilling, so four share an SM wherever
// their shared memory allows it (transforms of up to 3.5k points); the
// radix-11/13 kind keeps two per SM (128 registers) and Bluestein one (512
// threads).  The adjoint kernels need more registers and keep the default.
template <int KIND>
constexpr int phi_synth_min_blocks()
{
    return KIND == kDirect ? 4 : KIND == kDirectBig ? 2 : 1;
}

template <int KIND>
__global__ void __launch_bounds__(phi_threads<KIND>(), phi_synth_min_blocks<KIND>())
phi_synth_kernel(PlanView v, const int *__restrict__ rings, const double2 *__restrict__ q,
                 double *__restrict__ map)
{
    extern __shared__ double2 sm[];
    const int ring = rings[blockIdx.x];
    const int b = blockIdx.y;
    shtb_dev::phi_synth_ring<KIND, false>(v, ring, q + ((size_t)b * v.nrings + ring) * (v.lmax + 1),
                                          map + (size_t)b * v.npix + v.ring_start[ring], sm);
}

// ring stage of a compressed plan's map group, straight from the parity
// halves q^0, q^1 of the butterfly output (no separate combine pass)
// maps: either stacked at map + (b0 + b) npix, or one pointer per map
struct MapOut {
    double *map;
    double *const *table;
};

template <int KIND>
__global__ void __launch_bounds__(phi_threads<KIND>(), phi_synth_min_blocks<KIND>())
phi_synth_qt_kernel(PlanView v, const int *__restrict__ rings, const double2 *__restrict__ qt,
                    MapOut mo, int b0)
{
    extern __shared__ double2 sm[];
    const int ring = rings[blockIdx.x];
    const int b = blockIdx.y;
    double *base = mo.table ? mo.table[b0 + b] : mo.map + (size_t)(b0 + b) * v.npix;
    shtb_dev::phi_synth_ring_qt<KIND, false>(v, ring, qt, b, base + v.ring_start[ring], sm);
}

template <int KIND>
__global__ void __launch_bounds__(phi_threads<KIND>())
phi_adjoint_kernel(PlanView v, const int *__restrict__ rings, const double *__restrict__ map,
                   double2 *__restrict__ qa)
{
    constexpr bool BLUE = KIND == kBluestein;
    extern __shared__ double2 sm[];
    const int ring = rings[blockIdx.x];
    const int b = blockIdx.y;
    const int L = v.lmax;
    const int J = v.ring_J[ring], K = J / 2, s = v.ring_s[ring];
    const double2 *__restrict__ T = v.tw + v.ring_tw[ring];
    const int *__restrict__ rl = v.rad + v.ring_rad[ring];

    // z_n = f_{2n} + i f_{2n+1}; forward DFT Zf_k = sum_n z_n e^{-2 pi i k n/K}
    const double2 *in = reinterpret_cast<const double2 *>(map + (size_t)b * v.npix + v.ring_start[ring]);
    for (int n = threadIdx.x; n < K; n += blockDim.x) {
        const double2 z = in[n];
        sm[n] = BLUE ? cconj(z) : z;     // Bluestein: forward = conj(inverse(conj))
    }
    if (BLUE) {
        __syncthreads();
        bluestein_mx<true>(sm, K, v.ring_mx[ring], T, v.mfb + v.ring_mfb[ring], rl,
                           TwTable{v.mtw + v.ring_mtw[ring]});
        for (int n = threadIdx.x; n < K; n += blockDim.x) sm[n] = cconj(sm[n]);
        __syncthreads();
    } else {
        constexpr bool BIG = KIND == kDirectBig;
        RaderCtx rc;
        const RaderCtx *rcp = BIG ? rader_ctx(v, ring, K, sm, rc) : nullptr;
        fft_mx_dif<BIG, BIG>(sm, K, K, rl, TwRing{T, J}, rcp);   // position order
    }

    // F_r = E'_r + e^{-2 pi i r/J} O'_r with E' = (Zf_r + conj Zf_{K-r})/2,
    // O' = (Zf_r - conj Zf_{K-r})/(2i), K-periodic; then
    // q_adj[m] = e^{-i pi m s / J} F_{m mod J}.
    double2 *outq = qa + ((size_t)b * v.nrings + ring) * (L + 1);
    for (int m = threadIdx.x; m <= L; m += blockDim.x) {
        const int r = m % J;
        const int rho = r < K ? r : r - K;
        const int rho2 = rho == 0 ? 0 : K - rho;
        const double2 A = BLUE ? sm[rho] : sm[fft_pos(rho, K, rl)];
        const double2 B = cconj(BLUE ? sm[rho2] : sm[fft_pos(rho2, K, rl)]);
        const double2 Ep = make_double2(0.5 * (A.x + B.x), 0.5 * (A.y + B.y));
        const double2 D = make_double2(0.5 * (A.x - B.x), 0.5 * (A.y - B.y));   // (A - B)/2
        const double2 Op = make_double2(D.y, -D.x);                             // D / i
        const double2 F = cadd(Ep, cmul_conj(Op, ring_root(T, J, 2LL * r)));
        outq[m] = s ? cmul_conj(F, ring_root(T, J, (long long)m)) : F;
    }
}

// one launch per ring kind: grid (rings of that kind) x maps, shared memory
// for the kind's longest transform.  The Bluestein list is cut in two:
// rings [0, split) at phi_threads (one CTA per SM at the longest lengths),
// rings [split, n) -- transforms of at most kBlueSmallM points -- at half the
// threads with shared memory for their own longest transform, so that two
// CTAs share an SM and one's barriers between FFT passes are covered by the
// other's work.  Every body loops over blockDim.x.
struct RingSet {
    const int *rings;
    int n, len;
    int split, len_small;
};

RingSet ring_set(const shtb_plan_s *p, int kind)
{
    if (kind == kDirect)
        return {p->d_direct_rings, (int)p->direct_rings.size(), p->max_K_direct, (int)p->direct_rings.size(), 0};
    if (kind == kBluestein)
        return {p->d_blue_rings, (int)p->blue_rings.size(), p->max_M_mx, p->blue_split, p->max_M_small};
    return {p->d_big_rings, (int)p->big_rings.size(), p->max_K_big, (int)p->big_rings.size(), 0};
}

// launch(rings, n, threads, smem bytes) for each non-empty part of rs
template <int KIND, class Launch>
int launch_parts(const shtb_plan_s *p, const RingSet &rs, const void *kernel, Launch launch)
{
    if (rs.n == 0) return SHTB_OK;
    SHTB_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double2) * (size_t)rs.len)));
    if (rs.split > 0) {
        launch(rs.rings, rs.split, phi_threads<KIND>(), sizeof(double2) * (size_t)rs.len);
        SHTB_CUDA_TRY(cudaGetLastError());
        ++p->launches;
    }
    if (rs.split < rs.n) {
        launch(rs.rings + rs.split, rs.n - rs.split, phi_threads<KIND>() / 2,
               sizeof(double2) * (size_t)rs.len_small);
        SHTB_CUDA_TRY(cudaGetLastError());
        ++p->launches;
    }
    return SHTB_OK;
}

template <int KIND>
int launch_kind(const shtb_plan_s *p, bool synth, const void *in, void *out, int nmaps, cudaStream_t st)
{
    const RingSet rs = ring_set(p, KIND);
    const PlanView v = p->view;
    if (synth)
        return launch_parts<KIND>(p, rs, (const void *)phi_synth_kernel<KIND>,
                                  [&](const int *rings, int n, int threads, size_t smem) {
                                      phi_synth_kernel<KIND><<<dim3((unsigned)n, (unsigned)nmaps), threads, smem,
                                                               st>>>(v, rings, (const double2 *)in, (double *)out);
                                  });
    return launch_parts<KIND>(p, rs, (const void *)phi_adjoint_kernel<KIND>,
                              [&](const int *rings, int n, int threads, size_t smem) {
                                  phi_adjoint_kernel<KIND><<<dim3((unsigned)n, (unsigned)nmaps), threads, smem,
                                                             st>>>(v, rings, (const double *)in, (double2 *)out);
                              });
}

int launch_set(const shtb_plan_s *p, bool synth, const void *in, void *out, int nmaps,
               cudaStream_t st)
{
    int rc;
    if ((rc = launch_kind<kBluestein>(p, synth, in, out, nmaps, st))) return rc;
    if ((rc = launch_kind<kDirect>(p, synth, in, out, nmaps, st))) return rc;
    return launch_kind<kDirectBig>(p, synth, in, out, nmaps, st);
}

template <int KIND>
int launch_qt_set(const shtb_plan_s *p, const double2 *qt, int nb, MapOut map, int b0, const RingSet &rs,
                  cudaStream_t st)
{
    const PlanView v = p->view;
    return launch_parts<KIND>(p, rs, (const void *)phi_synth_qt_kernel<KIND>,
                              [&](const int *rings, int n, int threads, size_t smem) {
                                  phi_synth_qt_kernel<KIND><<<dim3((unsigned)n, (unsigned)nb), threads, smem, st>>>(
                                      v, rings, qt, map, b0);
                              });
}

template <int KIND>
int launch_qt_kind(const shtb_plan_s *p, const double2 *qt, int nb, MapOut map, int b0, cudaStream_t st)
{
    return launch_qt_set<KIND>(p, qt, nb, map, b0, ring_set(p, KIND), st);
}

template <int KIND>
int launch_qt_list(const shtb_plan_s *p, const double2 *qt, int nb, MapOut map, int b0,
                   const shtb_plan_s::ChunkKind &ck, cudaStream_t st)
{
    return launch_qt_set<KIND>(p, qt, nb, map, b0, RingSet{p->d_chunk_list + ck.off, ck.n, ck.len,
                                                           KIND == kBluestein ? ck.split : ck.n, ck.len_small}, st);
}

int launch_qt_all(const shtb_plan_s *p, const double *qt, int nb, MapOut mo, int b0, cudaStream_t st)
{
    const double2 *q2 = (const double2 *)qt;
    int rc;
    if ((rc = launch_qt_kind<kBluestein>(p, q2, nb, mo, b0, st))) return rc;
    if ((rc = launch_qt_kind<kDirect>(p, q2, nb, mo, b0, st))) return rc;
    return launch_qt_kind<kDirectBig>(p, q2, nb, mo, b0, st);
}

}  // namespace

// The three ring kinds write disjoint rings, so they run side by side: the
// Bluestein rings on the caller's stream, the direct and the radix-11/13 or
// Rader rings on two plan-owned streams forked from it and joined back, and
// each launch's last wave overlaps the others' work.
int launch_phi_synth_qt(const shtb_plan_s *p, const double *qt, int nb, double *map, int b0,
                        cudaStream_t st)
{
    shtb_plan_s *pp = const_cast<shtb_plan_s *>(p);
    if (!pp->ring_stream[0]) {
        for (auto &s2 : pp->ring_stream) SHTB_CUDA_TRY(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
        for (auto &e : pp->ring_ev) SHTB_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const double2 *q2 = (const double2 *)qt;
    const MapOut mo{map, nullptr};
    SHTB_CUDA_TRY(cudaEventRecord(pp->ring_ev[0], st));
    for (cudaStream_t s2 : pp->ring_stream) SHTB_CUDA_TRY(cudaStreamWaitEvent(s2, pp->ring_ev[0], 0));
    int rc;
    if ((rc = launch_qt_kind<kBluestein>(p, q2, nb, mo, b0, st))) return rc;
    if ((rc = launch_qt_kind<kDirect>(p, q2, nb, mo, b0, pp->ring_stream[0]))) return rc;
    if ((rc = launch_qt_kind<kDirectBig>(p, q2, nb, mo, b0, pp->ring_stream[1]))) return rc;
    for (int i = 0; i < 2; ++i) {
        SHTB_CUDA_TRY(cudaEventRecord(pp->ring_ev[1 + i], pp->ring_stream[i]));
        SHTB_CUDA_TRY(cudaStreamWaitEvent(st, pp->ring_ev[1 + i], 0));
    }
    return SHTB_OK;
}

int launch_phi_synth_qt_chunk(const shtb_plan_s *p, const double *qt, int nb, double *map, int b0, int chunk,
                              cudaStream_t st)
{
    const double2 *q2 = (const double2 *)qt;
    const MapOut mo{map, nullptr};
    const auto *ck = p->chunk_kind[chunk];
    int rc;
    if ((rc = launch_qt_list<kBluestein>(p, q2, nb, mo, b0, ck[1], st))) return rc;
    if ((rc = launch_qt_list<kDirect>(p, q2, nb, mo, b0, ck[0], st))) return rc;
    return launch_qt_list<kDirectBig>(p, q2, nb, mo, b0, ck[2], st);
}

int launch_phi_synth_qt_ptr(const shtb_plan_s *p, const double *qt, int nb, double *const *map_of_map,
                            int b0, cudaStream_t st)
{
    return launch_qt_all(p, qt, nb, MapOut{nullptr, map_of_map}, b0, st);
}

int launch_phi_synth(const shtb_plan_s *p, const double2 *q, double *map, int nmaps, cudaStream_t st)
{
    return launch_set(p, true, q, map, nmaps, st);
}

int launch_phi_adjoint(const shtb_plan_s *p, const double *map, double2 *q, int nmaps,
                       cudaStream_t st)
{
    return launch_set(p, false, map, q, nmaps, st);
}
