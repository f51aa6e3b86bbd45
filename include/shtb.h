/*
 * shtb.h -- C ABI of a GB300 (sm_103a) implementation of scalar spherical
 * harmonic synthesis on the HEALPix grid by butterfly-compressed Legendre
 * transforms, after D. S. Seljebotn, "Wavemoth -- Fast spherical harmonic
 * transforms by butterfly matrix compression" (arXiv 1110.4874).
 *
 * Conventions shared by every call
 * ---------------------------------
 * Transform (Sec. 2.1-2.2, Eq. shdef, Eq. sh-baseline):
 *     f(theta_k, phi_kj) = sum_{l=0}^{L} sum_{m=-l}^{l} a_lm Y_lm(theta_k, phi_kj)
 *   for a real field, a_{l,-m} = (-1)^m conj(a_lm), with Y_lm =
 *   Ptilde_l^m(cos theta) e^{i m phi} and Ptilde the normalised associated
 *   Legendre function of Eq. (Y-def), Condon-Shortley phase included.
 * a_lm buffers: complex128 as interleaved doubles (re, im), only m >= 0,
 *   m-major: coefficient (l, m) of map b sits at complex index
 *   b * nalm + m*(2L+1-m)/2 + l, nalm = (L+1)(L+2)/2.  Im a_l0 is ignored on
 *   input and written as 0 on output.
 * Maps: float64, [nmaps][12 nside^2], HEALPix RING order (rings north to
 *   south, pixels in increasing phi), maps stacked (not interleaved).
 * Adjoint: the transpose of the real-linear synthesis map under the plain
 *   real inner products over (Re a_lm, Im a_lm) and pixels:
 *     (Y^T f)_l0 = sum_p f_p Ptilde_l^0(z_p)
 *     (Y^T f)_lm = 2 sum_p f_p Ptilde_l^m(z_p) e^{-i m phi_p}   (m >= 1),
 *   i.e. the Y^dagger of Eq. (wiener) with a factor 2 for m >= 1, which is
 *   the gradient convention of torch for complex parameters.
 * Device pointers: every pointer named *_dev lives in the memory of the plan's
 *   CUDA device and must be 8-byte aligned (16-byte for complex arrays); the
 *   caller owns it.  Host pointers (*_host) should be pinned for overlap.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *   default stream).  Calls enqueue work and return without synchronising,
 *   except the *_host variants, which return once the result is on the host.
 * Errors: every int-returning call returns SHTB_OK (0) or a negative SHTB_E*
 *   code; nothing aborts.  shtb_strerror() names a code and
 *   shtb_last_error_message() gives the calling thread's last detailed
 *   message.
 * Threads: one plan may be used from one host thread at a time.
 */
#ifndef SHTB_H
#define SHTB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SHTB_ABI_VERSION 1

enum {
    SHTB_OK = 0,
    SHTB_EINVAL = -1,     /* invalid argument (sizes, null pointers, nside, lmax, eps) */
    SHTB_ENOMEM = -2,     /* host or device allocation failed                        */
    SHTB_ECUDA = -3,      /* a CUDA runtime call failed                               */
    SHTB_EMISMATCH = -4,  /* plan used on another device than it was built for       */
    SHTB_ETIMEOUT = -5,   /* a bounded device wait gave up                             */
    SHTB_ENOTSUP = -6,    /* size or option outside what the library supports         */
    SHTB_EIO = -7,        /* plan cache file could not be read or written              */
    SHTB_ECORRUPT = -8    /* plan cache file failed its checks                         */
};

typedef struct shtb_plan_s *shtb_plan;

/* Plan options (all fields have defaults set by shtb_plan_opts_init). */
typedef struct {
    int leaf_cols;     /* columns (rings) per butterfly leaf block, Sec. 3.2 ("64 columns"
                          in the text, 32 in Fig. compression-efficiency); default 32  */
    int max_depth;     /* cap on butterfly levels per (m, parity); -1 = no cap        */
    double rho;        /* cost of one stored-matrix element relative to one recurrence
                          step, the rho of Sec. 4.2 used to choose where to stop
                          compressing; <= 0 = library default                         */
    int nthreads;      /* host threads used while building the plan; 0 = all cores   */
    int device;        /* CUDA device ordinal; -1 = the calling thread's current one  */
    const char *cache_dir; /* NULL, or a directory of plan files: shtb_plan_create loads
                          the plan of this (nside, lmax, eps, options) from it if a
                          valid file is there, else builds the plan and writes the
                          file (a missing, unreadable or corrupt file is rebuilt)   */
    int gpu_build;     /* 1: the plan builder runs the interpolative decompositions of
                          each butterfly level as one batch on the plan's GPU (same
                          algorithm and truncation rule as the host); 0: on the host */
    int spin;          /* 0: scalar plan; 2: polarised (spin-2) plan, whose transforms
                          are shtb_synthesize_spin (the spin-weighted transforms of
                          Sec. 5, by compressing the spin-weighted operators)      */
    int residual_recurrence; /* compressed scalar plans: 0 (default) stores each
                          residual block R = Lambda[I, skeleton] (Sec. 3.2); 1 keeps
                          two start values per (block, column) instead and
                          regenerates R during synthesis by the jump-two recurrence
                          of Eq. (three-term), as Sec. 3.3 does to save memory (and
                          its transpose in the adjoint).  Batches (shtb_batch_create)
                          return SHTB_ENOTSUP on such plans.  Needs eps > 0 and
                          spin = 0, else SHTB_ENOTSUP.                            */
} shtb_plan_opts;

/* Plan statistics (algorithmic counts; used for roofline accounting). */
typedef struct {
    int nside, lmax;
    double eps;
    int nrings;                 /* 4 nside - 1                                        */
    long long npix;             /* 12 nside^2                                         */
    long long nalm;             /* (L+1)(L+2)/2                                       */
    int compressed;             /* 0: eps <= 0, uncompressed (zero levels, Sec. 3.3)  */
    long long n_recurrence;     /* (l, ring) pairs evaluated by the Legendre recurrence
                                   after the 1e-30 crop, summed over m and parity    */
    long long n_recurrence_exec;/* lane-steps the kernel issues for them (incl. idle
                                   lanes of a warp)                                   */
    long long n_dense;          /* stored dense interpolation-matrix elements (S)     */
    long long n_rstored;        /* stored residual-block elements (R)                 */
    long long plan_device_bytes;/* HBM held by the plan (excluding workspace)         */
    long long plan_read_bytes;  /* plan bytes one transform of a map batch reads      */
    double legendre_flops_per_map;  /* FP64 flops of the Legendre stage per map
                                       (recurrence flops amortised at 1 map)          */
    double recurrence_flops;        /* FP64 flops of the recurrence per call           */
    double phi_flops_per_map;       /* FP64 flops of the ring FFT stage per map       */
    double build_seconds;           /* host + device time of shtb_plan_create         */
    long long kernel_launches;      /* CUDA kernels this plan has launched so far     */
    long long n_ident;              /* identity entries of the interpolation matrices  */
    int depth_hist[16];             /* (m, parity) count per butterfly depth          */
    int from_cache;                 /* 1: the plan was read from a plan file          */
    int spin;                       /* 0 scalar, 2 polarised; for a polarised plan the
                                       element and byte counts cover both operators  */
    long long n_rgen;               /* residual-block elements regenerated by the
                                       recurrence per synthesis (residual_recurrence
                                       plans; n_rstored is then 0)                    */
} shtb_plan_stats_t;

/*
 * sizeof of the public structs as this library was compiled, so that a
 * binding can check its own layouts: opts = shtb_plan_opts, stats =
 * shtb_plan_stats_t, request = shtb_request, batch_opts = shtb_batch_opts.
 * Any pointer may be NULL.  Needs no GPU.  Returns SHTB_OK.
 */
int shtb_struct_sizes(int *opts, int *stats, int *request, int *batch_opts);

/* Fill *opts with defaults.  Returns SHTB_EINVAL on NULL. */
int shtb_plan_opts_init(shtb_plan_opts *opts);

/*
 * Build a synthesis plan for HEALPix resolution nside and band limit lmax
 * (Sec. 2.2) on a CUDA device: ring geometry, the per-(l, m) coefficients of
 * the jump-two Legendre recurrence (Eq. three-term), the recurrence start
 * values past the 1e-30 crop (Appendix, "Efficient code for Legendre
 * transforms"), the ring phase/FFT tables of Eq. (tau), and, when eps > 0,
 * the butterfly-compressed operator of Sec. 3.2 at ID tolerance eps
 * (Eq. ID-approximation), with eps the relative tolerance of every ID (each
 * block's truncated pivoted QR stops once the largest remaining column norm
 * is at most eps times the block's first pivot).  eps <= 0 gives the
 * uncompressed transform (the "zero levels of compression" limit of
 * Sec. 3.3); the adjoint of a compressed plan applies the transposed
 * compressed operator, so it is the exact transpose of that plan's synthesis.
 * nside >= 1, 0 <= lmax <= 8192; opts may be NULL.  On success *out holds a
 * plan that owns all its device memory; release it with shtb_plan_destroy.
 * Errors: SHTB_EINVAL, SHTB_ENOTSUP, SHTB_ENOMEM, SHTB_ECUDA.
 */
int shtb_plan_create(int nside, int lmax, double eps, const shtb_plan_opts *opts,
                     shtb_plan *out);

/*
 * Polarised plans (opts->spin = 2).  The spin-2 transform needs two real
 * operators per m, F+ and F- = (2_lambda +- (-2)_lambda)/2, where
 * sY_lm = s_lambda_lm(theta) e^{i m phi} (Newman-Penrose convention).  F+
 * has the mirror parity (-1)^(l+m) of the scalar functions and F- the
 * opposite one.  A polarised plan holds both, each compressed by the
 * butterfly of Sec. 3.2 at tolerance eps.  With eps <= 0 both are stored
 * uncompressed, as residual blocks at depth 0, which suits small sizes only.
 * The paper's Sec. 5 offers two routes: a reduction to three scalar
 * transforms, or compressing the spin-weighted operators.  This plan takes
 * the second.  Polarised plans serve shtb_synthesize_spin,
 * shtb_adjoint_spin and shtb_analyze_spin; the scalar calls and batches
 * return SHTB_ENOTSUP on them.  Plan files and cache_dir hold both
 * operators.
 */

/* Release a plan and all device memory it owns (NULL is accepted). */
int shtb_plan_destroy(shtb_plan plan);

/*
 * Plan files (the paper's precomputed-data files).  shtb_plan_save writes
 * the plan -- host tables and every device array, with a format version, the
 * plan's key (nside, lmax, eps, leaf_cols, max_depth, rho, spin) and a
 * checksum; a polarised plan's file holds both of its operators --
 * to `path` (written to path.tmp, then renamed).  shtb_plan_load builds a
 * plan on opts->device (or the current device; other opts fields are taken
 * from the file) from such a file.  Errors: SHTB_EIO (cannot open, read or
 * write), SHTB_ECORRUPT (wrong magic, version or key, truncated, checksum
 * mismatch), SHTB_EINVAL, SHTB_ENOMEM, SHTB_ECUDA.
 */
int shtb_plan_save(shtb_plan plan, const char *path);
int shtb_plan_load(const char *path, const shtb_plan_opts *opts, shtb_plan *out);

/* Copy the plan's statistics into *out. */
int shtb_plan_stats(shtb_plan plan, shtb_plan_stats_t *out);

/*
 * Make sure the plan's internal workspace can serve transforms of up to
 * nmaps maps, allocating now (so later calls allocate nothing and may be
 * captured into a CUDA graph).  Errors: SHTB_EINVAL, SHTB_ENOMEM.
 */
int shtb_plan_reserve(shtb_plan plan, int nmaps);

/*
 * Synthesis f = Y a for nmaps maps (Eq. shdef via Eq. sh-baseline):
 * Legendre stage q_m(z_k) = sum_l a_lm Ptilde_l^m(z_k) split by l-m parity
 * over mirrored rings (Eq. q-even-odd, q-even-odd2), then per ring the phase
 * shift and wrap of Eq. (tau) and a backward real FFT.
 * alm_dev: [nmaps][nalm] complex128; map_dev: [nmaps][12 nside^2] float64.
 * Errors: SHTB_EINVAL (NULL, nmaps < 1, misaligned), SHTB_EMISMATCH,
 * SHTB_ENOMEM (workspace growth), SHTB_ECUDA.
 */
int shtb_synthesize(shtb_plan plan, const double *alm_dev, double *map_dev, int nmaps,
                    void *stream);

/*
 * Adjoint synthesis a = Y^T f for nmaps maps (the Y^dagger of Eq. wiener
 * under the real inner product, see the header comment): per ring a forward
 * real FFT and the unwrap of Eq. (tau), then the transposed Legendre stage
 * (Eq. legendre-transform-linalg-backwards without quadrature weights).
 * map_dev: [nmaps][12 nside^2]; alm_dev: [nmaps][nalm] complex128 (written).
 * Errors as shtb_synthesize.
 */
int shtb_adjoint(shtb_plan plan, const double *map_dev, double *alm_dev, int nmaps,
                 void *stream);

/*
 * Polarised synthesis, HEALPix convention: (Q + iU) = -sum (aE + i aB) 2Y and
 * (Q - iU) = -sum (aE - i aB) (-2)Y.  Per m and ring this is
 * Q_m = -sum_l [aE F+ + i aB F-] and U_m = -sum_l [aB F+ - i aE F-], with
 * Q = Re Q_0 + 2 sum_{m>=1} Re(Q_m e^{i m phi}), and the same for U.  Each
 * operator is applied to the E and B coefficients of all pairs together
 * (one read of its plan data per 8 inputs), then a combine pass and the
 * ring stage of shtb_synthesize run.
 * alm_dev: [npairs][2][nalm] complex128, E then B per pair; l < 2 terms
 * contribute nothing, and Im a_l0 is ignored.
 * map_dev: [npairs][2][12 nside^2] float64, Q then U.
 * Errors: as shtb_synthesize; SHTB_ENOTSUP if the plan is not polarised.
 */
int shtb_synthesize_spin(shtb_plan plan, const double *alm_dev, double *map_dev, int npairs,
                         void *stream);

/*
 * Transpose of shtb_synthesize_spin under real inner products over the
 * (Re, Im) pairs of aE and aB (the convention of shtb_adjoint):
 * <synthesize_spin(a), f> = <a, adjoint_spin(f)>.  The steps are the ring
 * sums of the Q and U maps (forward FFT and unwrap, as in shtb_adjoint), the
 * transposed combine (E: -G_Q for F+ and -i G_U for F-; B: -G_U for F+ and
 * i G_Q for F-, folded by each operator's mirror parity), and the
 * transposed butterflies of F+ and F-, whose outputs are summed, x2 for
 * m >= 1.  The compressed plan's adjoint is the exact transpose of its
 * synthesis.
 * map_dev: [npairs][2][12 nside^2] (Q, U); alm_dev: [npairs][2][nalm]
 * complex128 (E, B; written, Im a_l0 = 0).  Errors as shtb_synthesize_spin.
 */
int shtb_adjoint_spin(shtb_plan plan, const double *map_dev, double *alm_dev, int npairs,
                      void *stream);

/*
 * Polarised analysis by the same ring quadrature as shtb_analyze (Eq.
 * sh-forward-quadrature for the spin-2 harmonics, which are orthonormal
 * like the scalar ones): (aE, aB) = h_m shtb_adjoint_spin(w Q, w U) with
 * h_0 = 1 and h_m = 1/2, then niter Jacobi steps a += A (f - Y a).  Layouts
 * are those of shtb_adjoint_spin; ring_weight_dev and niter are as for
 * shtb_analyze.  Errors as shtb_synthesize_spin, plus SHTB_EINVAL for niter
 * or aliasing as in shtb_analyze.
 */
int shtb_analyze_spin(shtb_plan plan, const double *map_dev, double *alm_dev, int npairs,
                      const double *ring_weight_dev, int niter, void *stream);

/*
 * Spherical-harmonic analysis by ring quadrature (Eq. sh-forward-quadrature):
 * a_lm = sum_p w_p f_p conj(Y_lm(p)), w_p = ring_weight_dev[ring of p], then
 * niter Jacobi refinement steps a <- a + A (f - Y a), A the quadrature rule
 * (the HEALPix quadrature is not exact, Sec. 2.3; each step costs one
 * synthesis and one adjoint and shrinks the error of a band-limited map by
 * a roughly constant factor for lmax <= 2 nside).
 * map_dev: [nmaps][12 nside^2] float64 (read only); alm_dev: [nmaps][nalm]
 * complex128 (written; Im a_l0 = 0).  ring_weight_dev: device, one double
 * per ring (4 nside - 1), the weight of every pixel of that ring; NULL means
 * the equal-area HEALPix weight 4 pi / (12 nside^2).  The plan's workspace
 * holds the residual map, so calls on one plan are stream-ordered.
 * Errors as shtb_synthesize; SHTB_EINVAL also for niter outside
 * 0..SHTB_MAX_ANALYSIS_ITER or map_dev == alm_dev.
 */
#define SHTB_MAX_ANALYSIS_ITER 64
int shtb_analyze(shtb_plan plan, const double *map_dev, double *alm_dev, int nmaps,
                 const double *ring_weight_dev, int niter, void *stream);

/*
 * The same two transforms between HOST buffers: the call copies the inputs
 * to the device on `stream`, transforms, copies the result back and waits
 * for it.  Buffers should be pinned (cudaHostAlloc) for full copy speed.
 */
int shtb_synthesize_host(shtb_plan plan, const double *alm_host, double *map_host,
                         int nmaps, void *stream);
int shtb_adjoint_host(shtb_plan plan, const double *map_host, double *alm_host,
                      int nmaps, void *stream);

/* ------------------------------------------------------------------------
 * Batched serving.  A batch holds synthesis requests for any number of
 * compressed plans (any mix of nside / lmax / eps); requests sharing a plan
 * are merged along the map axis so that the plan's compressed operator is
 * read once per group of up to 8 maps (Sec. 3.3: many simultaneous
 * transforms amortise the precomputed data).  shtb_batch_run executes the
 * whole batch -- a_lm gather, residual blocks, every butterfly level, parity
 * combine, ring FFTs -- as ONE persistent kernel launch whose blocks pull
 * work packs in dependency order from a queue; the launch is captured into a
 * CUDA graph on the first run and replayed afterwards.
 * ------------------------------------------------------------------------ */
typedef struct {
    shtb_plan plan;          /* a compressed plan (eps > 0) on the current device   */
    const double *alm_dev;   /* [nmaps][nalm] complex128, as shtb_synthesize         */
    double *map_dev;         /* [nmaps][12 nside^2] float64 (written)                 */
    int nmaps;
    int dir;                 /* 0 = synthesis (the only direction served)            */
} shtb_request;

typedef struct shtb_batch_s *shtb_batch;

typedef struct {
    int autotune;            /* 1: time the candidate schedules on this batch at
                                creation (runs it several times) and keep the fastest */
    int warps_per_block;     /* 4 or 8 (0 = default 4; overridden by autotune)         */
    int group_width;         /* maps per operator read, 1..8 (default 8)               */
    int lpt;                 /* 1: largest items first inside each stage               */
    long long spin_limit;    /* polls before a stage wait gives up (0 = 2e7)           */
    int schedule;            /* without autotune: 0 = one persistent kernel launch,
                                1 = graph of the stage kernels over merged map groups  */
    int streams;             /* streams of schedule 1 (0 = 4)                           */
} shtb_batch_opts;

int shtb_batch_opts_init(shtb_batch_opts *opts);

/*
 * Build a batch over nreq requests (buffers must stay valid while the batch
 * is used; they are read and written at creation when autotune is on).  The
 * batch owns its workspace and schedule; creation allocates, runs allocate
 * nothing.  Errors: SHTB_EINVAL, SHTB_ENOTSUP (uncompressed plan, dir != 0),
 * SHTB_EMISMATCH, SHTB_ENOMEM, SHTB_ECUDA.
 */
int shtb_batch_create(const shtb_request *reqs, int nreq, const shtb_batch_opts *opts,
                      shtb_batch *out);

/*
 * Run the batch on `stream` (NULL: the batch's own stream, and wait for it).
 * The first call captures the launch into a CUDA graph.  Check the outcome
 * with shtb_batch_status.  Errors: SHTB_EINVAL, SHTB_EMISMATCH, SHTB_ECUDA.
 */
int shtb_batch_run(shtb_batch batch, void *stream);

/* Wait for the batch's work on `stream` and report SHTB_ETIMEOUT if a stage
   wait of the persistent kernel gave up (its bounded spin ran out). */
int shtb_batch_status(shtb_batch batch, void *stream);

/* Schedule chosen for the batch: warps per block, persistent grid size,
   number of work packs (all 0 for the stage-kernel schedule) and the
   autotuner's best time (ms, 0 if not tuned). */
int shtb_batch_info(shtb_batch batch, int *warps_per_block, int *grid, int *npacks,
                    double *tuned_ms);

int shtb_batch_destroy(shtb_batch batch);
/* The schedule in use: 0 = persistent kernel, 1 = stage-kernel graph, and
   the stream count of schedule 1 (0 for schedule 0). */
int shtb_batch_schedule(shtb_batch batch, int *schedule, int *streams);

/* Private test hook: with on = 1 the batch's first stage claims one item more
   than it has, so every later stage's bounded wait runs out and the next run
   ends with SHTB_ETIMEOUT; on = 0 restores it. */
int shtb_test_batch_stall(shtb_batch batch, int on);

/* Name of an error code (static string). */
const char *shtb_strerror(int code);

/* Detailed message of the calling thread's last failing call ("" if none). */
const char *shtb_last_error_message(void);

/*
 * Per-stage device timing.  While enabled, each transform records CUDA
 * events around its stages on the stream it runs on; shtb_profile_read
 * waits for them and returns the summed milliseconds per stage:
 *   ms[0] Legendre stage (synthesis), ms[1] ring FFT stage (synthesis),
 *   ms[2] ring FFT stage (adjoint),   ms[3] Legendre stage (adjoint),
 *   ms[4] a_lm staging kernels (scaling / interleave / scatter),
 *   and, inside ms[0] for compressed plans: ms[5] residual blocks,
 *   ms[6] butterfly levels (ms[7] is unused);
 * and the number of profiled transforms.  Reading resets the sums.  Up to 4096
 * calls are kept between reads.
 */
int shtb_profile_enable(shtb_plan plan, int on);
int shtb_profile_read(shtb_plan plan, double *ms, int nstages, int *ncalls);

/*
 * Measure this device's FP64 throughput with two microkernels (a chain of
 * independent DFMA per thread, and warp-level DMMA m8n8k4 f64 tensor-core
 * MMA), each timed with CUDA events after a warm-up.  Results in GFLOP/s
 * (2 flops per FMA).  Used only to state roofline denominators.
 */
int shtb_measure_fp64_peak(int device, double *dfma_gflops, double *dmma_gflops);

/* ------------------------------------------------------------------------
 * Private entry points for testing single stages in isolation (the paper's
 * "private API ... used from Python to test individual C routines",
 * Sec. 4.1).  Buffers are device pointers.
 *   q layout: complex128 [nmaps][4 nside - 1][lmax + 1], q[b][ring][m].
 * ------------------------------------------------------------------------ */

/* Legendre stage only: q_m(z_k) for every ring (Eq. legendre-transform). */
int shtb_test_legendre(shtb_plan plan, const double *alm_dev, double *q_dev, int nmaps,
                       void *stream);
/* Compressed Legendre stage only (Sec. 3.2, Eq. factor-into-block-diagonal):
   residual blocks and butterfly levels of a compressed plan (eps > 0), giving
   the two parity halves q^t_m(z_r) = sum_j a_{m+t+2j,m} Ptilde_{m+t+2j}^m(z_r)
   (t = 0, 1) at the 2 nside half-rings r with z_r >= 0, north to the equator.
   qt_dev: device, [nmaps][2][2 nside][lmax+1] complex128 (written; the empty
   chain t = 1, m = lmax is 0).  The maps are q^0 + q^1 on ring r and
   q^0 - q^1 on its mirror (Eq. q-even-odd2).  Errors: SHTB_ENOTSUP for an
   uncompressed plan, as shtb_synthesize otherwise. */
int shtb_test_butterfly(shtb_plan plan, const double *alm_dev, double *qt_dev, int nmaps,
                        void *stream);
/* Ring stage only: pixels from q (Eq. sh-baseline, Eq. phi, Eq. tau). */
int shtb_test_phi(shtb_plan plan, const double *q_dev, double *map_dev, int nmaps,
                  void *stream);
/* Ring stage adjoint: q_adj[b][ring][m] = sum_j f_kj e^{-i m phi_kj}. */
int shtb_test_phi_adjoint(shtb_plan plan, const double *map_dev, double *q_dev,
                          int nmaps, void *stream);
/* Legendre stage adjoint: a_lm = c_m sum_k Ptilde_l^m(z_k) q_adj[k][m],
   c_0 = 1, c_m = 2 (m >= 1). */
int shtb_test_legendre_adjoint(shtb_plan plan, const double *q_dev, double *alm_dev,
                               int nmaps, void *stream);

/*
 * Synthesis without any device allocation.  Same arguments as
 * shtb_synthesize and, for uncompressed plans (eps <= 0), the same maps bit
 * for bit; for compressed plans it evaluates the uncompressed operator,
 * which agrees with shtb_synthesize to within the plan's tolerance.  Its scratch (the scaled a_lm and the q_m(z_k) work
 * array) lives in one static device array of SHTB_NOALLOC_SCRATCH_BYTES
 * instead of the plan's workspace.  This has no counterpart in the paper; it
 * serves callers that cannot allocate device memory when they transform:
 * processes whose device memory is already held by another allocator (a
 * framework's caching pool or a preallocating runtime), and loops that must
 * not pay for the implicit device synchronisation of cudaMalloc.  The plan
 * itself is still created, and allocated, beforehand.
 *  - Limit: 16 nmaps (L+1)(L+2)/2 bytes (rounded up to 256) plus
 *    16 nmaps (4 nside - 1)(L+1) bytes must fit in SHTB_NOALLOC_SCRATCH_BYTES
 *    (64 MiB), e.g. one map at nside = 512, L = 1024; larger requests return
 *    SHTB_ENOTSUP and leave the output untouched.
 *  - The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress (that device current) and caches it; make that
 *    first call before any stream capture.  Every GPU that loads the library
 *    holds the array until the process exits.  The cached address belongs
 *    to the device's primary context: after cudaDeviceReset (or anything
 *    else that destroys and recreates that context) this call is not
 *    supported in the same process.
 *  - All calls share the one array, which keeps the last call's contents:
 *    calls whose work overlaps on the GPU (other streams, other threads)
 *    race on it and must be ordered by the caller.  No state is carried from
 *    call to call: every scratch entry is written before it is read.
 * Errors: SHTB_EINVAL, SHTB_EMISMATCH, SHTB_ENOTSUP, SHTB_ECUDA.
 */
#define SHTB_NOALLOC_SCRATCH_BYTES (64u << 20)
int shtb_synthesize_noalloc(shtb_plan plan, const double *alm_dev, double *map_dev, int nmaps,
                            void *stream);

/*
 * Host-only check of the plan tables (needs no GPU): Ptilde_l^m(z_r) for
 * l = m..lmax at HEALPix half-ring r (0-based from the north pole, r < 2 nside),
 * evaluated on the CPU with the same per-(l, m) constants, start values and
 * two-FMA recurrence step as the Legendre kernels (Eq. three-term, rescaled).
 * out: lmax - m + 1 doubles (host).  Errors: SHTB_EINVAL.
 */
int shtb_test_host_recurrence(int nside, int lmax, int m, int r, double *out);

/*
 * Host-only check of the interpolative decomposition (Sec. 3.1, Eq. ID) used
 * by the butterfly compression: for the rows x n column-major block A and
 * relative tolerance eps, writes the rank k, the k skeleton column indices
 * (skel_out, n slots) and the full k x n interpolation matrix (T_out, n*n
 * slots, row-major; identity on the skeleton, 0 on all-zero columns) such
 * that A ~= A[:, skel] * T.  Errors: SHTB_EINVAL.
 */
int shtb_test_host_id(int rows, int n, const double *A, double eps, int *k_out, int *skel_out,
                      double *T_out);

/*
 * The same decomposition through the GPU plan builder's batched kernel, on
 * the current device (A on the host; n <= 128).  Outputs as
 * shtb_test_host_id.  Errors: SHTB_EINVAL, SHTB_ENOMEM, SHTB_ECUDA.
 */
int shtb_test_gpu_id(int rows, int n, const double *A, double eps, int *k_out, int *skel_out,
                     double *T_out);

/*
 * Host-only check of the butterfly compression (Sec. 3.2) of one Legendre
 * matrix Lambda^{m,t} (rows l = m+t+2j, columns the HEALPix rings with
 * z >= 0): builds the compressed operator exactly as shtb_plan_create does
 * and applies it on the CPU, the way the device kernels do, to the real
 * vector a (chain_len = floor((lmax-m-t)/2)+1 entries).  q_out (2 nside
 * doubles) receives the compressed Lambda^T a, q_exact the dense product;
 * info[0..3] = {depth, dense interpolation elements, stored residual
 * elements, identity entries}.  Errors: SHTB_EINVAL.
 */
int shtb_test_host_butterfly(int nside, int lmax, double eps, int m, int t, int leaf_cols,
                             const double *a, double *q_out, double *q_exact, long long *info);

/*
 * Host-only measurement of the interpolation variant of the Legendre stage
 * (Sec. 3.4 "Notes on interpolation", Eq. interpolation) for one chain
 * (order m, parity t; rows l = m+t+2j, j < n): q is evaluated at the n
 * positive roots z_i of P_{m+t+2n}^m and interpolated to the 2 nside
 * half-rings by W(y, z_i) = P_{l*}(y) 2 z_i / (P'_{l*}(z_i) (y^2 - z_i^2)),
 * l* = m+t+2n.  a: the chain's n coefficients (host); q_interp (2 nside
 * doubles) receives the two-step result, q_exact the direct product
 * Lambda^T a at the half-rings.  info[0..7] = {n, stored elements of Lambda
 * at the roots compressed by the plan's butterfly builder, of W compressed
 * by the same builder, of W compressed hierarchically (off-diagonal blocks
 * by interpolative decomposition, the algebraic form of the FMM), of Lambda
 * at the half-rings compressed by the butterfly builder, n * 2 nside,
 * n^2 + n * 2 nside, depth of the half-rings' butterfly}.
 * Errors: SHTB_EINVAL.
 */
int shtb_test_host_interp(int nside, int lmax, double eps, int m, int t, int leaf_cols, const double *a,
                          double *q_interp, double *q_exact, long long *info);

/*
 * Private host-only check (no GPU) of residual_recurrence plans: compresses
 * chain (m, t) as a plan of tolerance eps does, then regenerates every
 * residual block R = Lambda[I, skeleton] from the per-column recurrence
 * starts such a plan keeps (the jump-two recurrence of Eq. three-term,
 * stepped as the kernel steps it, times sigma) and compares it with the
 * stored block.  *max_rel: largest |R_regen - R_stored| relative to the
 * largest |R| of the same column.  info[0..3] = {blocks, elements, elements
 * zero on one side only (the 1e-30 crop), chain depth}.
 * Errors: SHTB_EINVAL, SHTB_ENOTSUP.
 */
int shtb_test_host_rec_blocks(int nside, int lmax, double eps, int m, int t, int leaf_cols, double *max_rel,
                              long long *info);

/*
 * Host-only check of the spin-weighted functions of spin plans (the
 * polarised transform, Sec. 5): s_lambda_lm(z_r) for s = +2 or -2 and
 * l = m..lmax at HEALPix half-ring r (0-based from the north pole), as the
 * plan builder computes them (Wigner recurrence in l, Newman-Penrose
 * convention: sY_lm = s_lambda_lm e^{i m phi}).  out: lmax - m + 1 doubles
 * (host; 0 for l < 2).  Errors: SHTB_EINVAL.
 */
int shtb_test_host_spin_column(int nside, int lmax, int m, int s, int r, double *out);

#ifdef __cplusplus
}
#endif

#endif /* SHTB_H */
