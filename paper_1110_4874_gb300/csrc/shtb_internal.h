// Internal declarations shared by the host plan builder, the kernels and the
// C-ABI layer.  Nothing here is part of the public interface (include/shtb.h).
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "shtb.h"

// ---------------------------------------------------------------- errors
// Record a detailed message for shtb_last_error_message() and return code.
int shtb_fail(int code, const std::string &msg);

// NVTX range over one library call (header-only NVTX 3: free unless a
// profiler is attached), so that timelines show the calls by name
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

#define SHTB_CUDA_TRY(expr)                                                            \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return shtb_fail(e_ == cudaErrorMemoryAllocation ? SHTB_ENOMEM : SHTB_ECUDA, \
                             std::string(#expr) + ": " + cudaGetErrorString(e_));      \
    } while (0)

// ------------------------------------------------------------ plan layout
// Index of coefficient (l, m) in the m-major a_lm layout.
inline long long alm_index(int lmax, int l, int m)
{
    return (long long)m * (2 * lmax + 1 - m) / 2 + l;
}

// Number of l values of parity t (l - m = t mod 2) for order m: l = m+t, m+t+2, ... <= L.
inline int chain_len(int lmax, int m, int t)
{
    return m + t > lmax ? 0 : (lmax - m - t) / 2 + 1;
}

// Constants of one step of the rescaled jump-two recurrence at (l, m):
// w = mu * x + (cz or cs), V_{l+2} = w V_l - V_{l-2}; sig = sigma_l.
struct alignas(32) RecCoef {
    double mu, cz, cs, sig;
};

// Running state of the two parity chains of one ring (adjoint kernel).
struct alignas(32) RecState {
    double cur0, prev0, cur1, prev1;
};

// Rader's algorithm for a ring transform with one prime factor p > 13
// (its own exponent 1) whose p - 1 factors over 2, 3, 5, 7, 11, 13: the
// p-point DFTs become cyclic convolutions of length n = p - 1.  Offsets are
// into the plan's rad (radix list of n), rdr_int (g^v and g^{-v} mod p,
// v < n, g a primitive root) and rdr_dbl (the position-order DFT of
// beta_t = e^{2 pi i g^t / p} scaled by 1/n, and e^{2 pi i t / n}).
struct RaderInfo {
    int p, n, rl, ga, gi, pad;
    long long G, tw;
};

// Everything a kernel needs to know about a plan, by value.
struct PlanView {
    int nside, lmax, nrings, nhalf;   // nhalf = 2 nside rings with z >= 0 (incl. equator)
    long long npix, nalm;

    // Legendre stage (Eq. three-term in the rescaled two-FMA form, see the
    // plan builder): per (l, m) at alm_index(l, m): {mu, Cz, Cs, sigma}.
    const RecCoef *coef;
    // per half-ring r in [0, nhalf): signed recurrence argument and which
    // constant (Cz or Cs) goes with it
    const double *xarg;
    const int *xform;
    // start of each (m, parity, half-ring) chain after the 1e-30 crop:
    // index ((m * 2) + t) * nhalf + r
    const int *jstart;
    const double2 *vstart;

    // ring stage
    const int *ring_J;               // pixels per ring
    const int *ring_s;               // half-pixel shift flag (phi_0 = pi s / J)
    const long long *ring_start;     // first pixel of each ring
    const long long *ring_tw;        // offset of the ring's e^{i pi n / J} table in tw
    const double2 *tw;
    // mixed-radix transforms (the stand-alone ring kernels): per ring the
    // radix list {n, r_0 .. r_{n-1}} (rad + ring_rad[ring]) of its transform
    // length -- K = J/2 when K factors over 2, 3, 5, 7, 11, 13 (ring_mx = 0),
    // else the Bluestein length ring_mx (smooth, >= 2K - 1) with the filter
    // at mfb + ring_mfb (position order, scaled by 1/ring_mx) and the
    // e^{2 pi i t / ring_mx} table at mtw + ring_mtw
    const int *ring_rad;
    const int *rad;
    const int *ring_mx;
    const long long *ring_mfb;
    const double2 *mfb;
    const long long *ring_mtw;
    const double2 *mtw;
    // fold weights of the synthesis ring kernels: ab + ring_ab[ring] holds,
    // for k < K = J/2, {A_k, B_k} with Z_k = G_k A_k + G_{k+K} B_k (G the
    // ring's folded spectrum without its phi_0 phase); the half-pixel phase,
    // the half-length packing and, on Bluestein rings, the chirp are in them
    const long long *ring_ab;
    const double2 *ab;
    // Rader rings: ring_rdr[ring] indexes rdr (-1 for other rings)
    const int *ring_rdr;
    const RaderInfo *rdr;
    const int *rdr_int;
    const double2 *rdr_dbl;
};

struct BfPlanDev;

struct shtb_plan_s {
    int nside = 0, lmax = 0;
    double eps = 0;
    // operator: 0 the scalar Legendre functions; 1 and 2 the spin-2
    // F+ and F- of a polarised plan (1 is the plan the caller holds, and it
    // owns the F- plan as its partner)
    int kind = 0;
    shtb_plan_s *partner = nullptr;
    int device = 0;
    int nrings = 0, nhalf = 0;
    long long npix = 0, nalm = 0;
    shtb_plan_opts opts{};

    // host copies of the ring description
    std::vector<int> ring_J, ring_s;
    std::vector<long long> ring_start;

    // ring lists of the three ring-kernel variants (mixed radix: direct
    // transform of length K over radices 2..7, Bluestein, direct with a
    // radix 11 or 13 or a Rader pass), heaviest rings first; the max_ values
    // are the shared-memory entries (complex) of the longest ring of each
    // (a Rader ring also holds its convolution scratch)
    std::vector<int> direct_rings, blue_rings, big_rings;
    int max_K_direct = 0, max_M_mx = 0, max_K_big = 0;
    // Bluestein rings blue_rings[blue_split..] have transforms of at most
    // kBlueSmallM points (the longest max_M_small): they run at half the
    // threads per CTA, two CTAs per SM
    static constexpr int kBlueSmallM = 7168;
    int blue_split = 0, max_M_small = 0;
    int *d_direct_rings = nullptr, *d_blue_rings = nullptr, *d_big_rings = nullptr;
    // the rings cut into kPhiChunks runs of consecutive rings with about equal
    // pixel counts, per run and ring variant a device list (chunk_list + off)
    // and its longest transform; pixels [chunk_pix[c], chunk_pix[c+1]) of a
    // map are written by run c (host-buffer synthesis overlaps their copy
    // back with the next run)
    static constexpr int kPhiChunks = 4;
    struct ChunkKind {
        int off, n, len;
        int split, len_small;   // as blue_split / max_M_small, within this list
    };
    ChunkKind chunk_kind[kPhiChunks][3] = {};
    long long chunk_pix[kPhiChunks + 1] = {};
    int *d_chunk_list = nullptr;
    cudaStream_t copy_stream = nullptr;            // created on first use, owned
    cudaEvent_t chunk_ev[kPhiChunks] = {};
    // the ring stage's three transform kinds run side by side on the
    // caller's stream and two plan-owned streams (created on first use)
    cudaStream_t ring_stream[2] = {};
    cudaEvent_t ring_ev[3] = {};

    // device allocations owned by the plan (freed in destroy), with their sizes
    std::vector<void *> allocations;
    std::vector<size_t> alloc_bytes;
    PlanView view{};

    // butterfly-compressed operator (eps > 0), owned
    BfPlanDev *bf = nullptr;

    // workspace (grown on demand)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int ws_nmaps = 0;

    // statistics
    shtb_plan_stats_t stats{};
    mutable long long launches = 0;   // kernels launched on behalf of this plan

    // stage profiling
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { int stage; int ev0, ev1; };
    std::vector<Rec> recs;
    int ev_next = 0;
    int prof_calls = 0;      // transforms run since the last profile read
};

// Stage timing (shtb_profile_enable): event pair around a stage on stream st;
// profile_begin returns -1 when profiling is off or the event pool is full.
int profile_begin(shtb_plan_s *p, cudaStream_t st);
void profile_end(shtb_plan_s *p, cudaStream_t st, int stage, int ev);

// ------------------------------------------------------- host plan build
// Fills every host-side table and uploads it; defined in shtb_plan_host.cpp.
int shtb_build_dense_plan(shtb_plan_s *p);

// Device allocation helper that registers the pointer with the plan.
int plan_alloc_upload(shtb_plan_s *p, void **dst, const void *src, size_t bytes);

// Plan cache files (shtb_plan_cache.cpp): write a built plan; fill a fresh
// plan whose key (nside, lmax, eps, opts) and device are set; the file name
// of a plan in a cache directory.
int plan_save(shtb_plan_s *p, const char *path);
int plan_load(shtb_plan_s *p, const char *path);
std::string plan_cache_path(const shtb_plan_s *p, const char *dir);
int plan_read_key(const char *path, int *nside, int *lmax, double *eps, shtb_plan_opts *opts);

// ---------------------------------------------------------- kernel launches
// shtb_legendre.cu
int launch_alm_prescale(const shtb_plan_s *p, const double2 *alm, double2 *aprime, int nmaps,
                        cudaStream_t st);
int launch_legendre_synth(const shtb_plan_s *p, const double2 *aprime, double2 *q, int nmaps,
                          cudaStream_t st);
int launch_legendre_adjoint(const shtb_plan_s *p, const double2 *qadj, double2 *aacc,
                            int nmaps, void *state_ws, cudaStream_t st);
int launch_alm_finish(const shtb_plan_s *p, const double2 *aacc, double2 *alm, int nmaps,
                      cudaStream_t st);
int launch_adjoint_parity(const shtb_plan_s *p, const double2 *qadj, double2 *g, int nmaps,
                          cudaStream_t st);
size_t legendre_adjoint_state_bytes(const shtb_plan_s *p);

// shtb_phi.cu
int launch_phi_synth(const shtb_plan_s *p, const double2 *q, double *map, int nmaps,
                     cudaStream_t st);
int launch_phi_adjoint(const shtb_plan_s *p, const double *map, double2 *q, int nmaps,
                       cudaStream_t st);
int launch_phi_synth_qt(const shtb_plan_s *p, const double *qt, int nb, double *map, int b0,
                        cudaStream_t st);
// ... for the rings of chunk `chunk` only (shtb_plan_s::kPhiChunks runs)
int launch_phi_synth_qt_chunk(const shtb_plan_s *p, const double *qt, int nb, double *map, int b0, int chunk,
                              cudaStream_t st);
// ... writing map b0 + b to map_of_map[b0 + b] (device array of map pointers)
int launch_phi_synth_qt_ptr(const shtb_plan_s *p, const double *qt, int nb, double *const *map_of_map,
                            int b0, cudaStream_t st);

// shtb_butterfly.cu
// polarised synthesis (shtb_spin.cu): parity halves of F+ and F- (map-major,
// inputs E, B per pair) -> ring-major Q_m, U_m spectra
int launch_spin_combine(const shtb_plan_s *p, const double *qt_plus, const double *qt_minus, double2 *qring,
                        int npairs, cudaStream_t st);
// ... and its transpose: ring sums of Q, U -> entry-major parity gradients of
// the F+ and F- butterflies; alm += add over n complex entries
int launch_spin_uncombine(const shtb_plan_s *p, const double2 *G, double2 *g_plus, double2 *g_minus, int npairs,
                          cudaStream_t st);
int launch_alm_add(const shtb_plan_s *p, double2 *alm, const double2 *add, size_t n, cudaStream_t st);

// analysis (shtb_analysis.cu): quadrature weighting of a map or a residual,
// and alm += h_m g with h_0 = 1, h_m = 1/2
int launch_ring_weight(const shtb_plan_s *p, const double *f, const double *y, const double *ring_w,
                       double w0, double *r, int nmaps, cudaStream_t st);
int launch_alm_quadrature_add(const shtb_plan_s *p, const double2 *g, double2 *alm, int nmaps,
                              bool first, cudaStream_t st);

size_t bf_workspace_bytes(const shtb_plan_s *p);
// map != nullptr: the whole synthesis; map == nullptr: the Legendre stage
// alone, q^t of map b written to qt_out + b [2][nhalf][L+1] complex
int launch_bf_synth(const shtb_plan_s *p, const double2 *alm, double2 *ai, void *ws, double *map,
                    int nmaps, cudaStream_t st, double *qt_out = nullptr);
// whole synthesis with the maps copied back to host memory as the ring
// stage finishes each chunk of rings (the copies overlap the rest)
int launch_bf_synth_to_host(shtb_plan_s *p, const double2 *alm, double2 *ai, void *ws, double *map,
                            double *map_host, int nmaps, cudaStream_t st);
void bf_release(shtb_plan_s *p);
// batched serving (stage-kernel schedule): a_lm of merged maps, given one
// device pointer per map, into ai[idx][map]; residual blocks + butterfly
// levels of maps b0 .. b0+nb-1 of ai (nb = 1, 2, 4, 8) into that group's q^t
int launch_bf_gather(const shtb_plan_s *p, const double2 *const *alm_of_map, double2 *ai, int nmaps,
                     cudaStream_t st);
int launch_bf_legendre_group(const shtb_plan_s *p, const double2 *ai, int nmaps, int b0, int nb, double *u0,
                             double *u1, double *qt, cudaStream_t st);
int launch_bf_adjoint(const shtb_plan_s *p, const double2 *g, double2 *aacc, void *ws, double2 *alm,
                      int nmaps, cudaStream_t st);

// shtb_util.cu
int measure_fp64_peak(int device, double *dfma, double *dmma);
