// C-ABI entry points (include/shtb.h): plan lifetime, workspace, the
// synthesis / adjoint pipelines, host-buffer variants, stage profiling and
// the private single-stage test entry points.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>

#include "shtb_butterfly.h"
#include "shtb_internal.h"

namespace {

thread_local std::string g_last_error;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Workspace {
    // synthesis
    double2 *ap = nullptr;      // [nalm][nmaps]
    double2 *q = nullptr;       // [nmaps][nrings][L+1]  (also the adjoint's q_adj)
    // adjoint
    void *adj = nullptr;        // g + recurrence state
    double2 *aacc = nullptr;    // [nalm][nmaps]
    // host-buffer variants
    double2 *alm = nullptr;     // [nmaps][nalm]
    double *map = nullptr;      // [nmaps][npix]
    // butterfly apply (compressed plans): two u buffers and q^t
    void *bf = nullptr;
};

size_t q_bytes(const shtb_plan_s *p, int nmaps)
{
    return sizeof(double2) * (size_t)nmaps * p->nrings * (p->lmax + 1);
}

size_t alm_bytes(const shtb_plan_s *p, int nmaps) { return sizeof(double2) * (size_t)nmaps * p->nalm; }

size_t adj_bytes(const shtb_plan_s *p, int nmaps)
{
    return sizeof(double2) * (size_t)(p->lmax + 1) * 2 * p->nhalf * nmaps +
           legendre_adjoint_state_bytes(p);
}

size_t ws_total(const shtb_plan_s *p, int nmaps)
{
    return align256(alm_bytes(p, nmaps)) * 2 + align256(q_bytes(p, nmaps)) +
           align256(adj_bytes(p, nmaps)) + align256(alm_bytes(p, nmaps)) +
           align256(sizeof(double) * (size_t)nmaps * p->npix) + align256(bf_workspace_bytes(p));
}

Workspace carve(shtb_plan_s *p, int nmaps)
{
    Workspace w;
    char *c = (char *)p->ws;
    w.ap = (double2 *)c;    c += align256(alm_bytes(p, nmaps));
    w.q = (double2 *)c;     c += align256(q_bytes(p, nmaps));
    w.adj = c;              c += align256(adj_bytes(p, nmaps));
    w.aacc = (double2 *)c;  c += align256(alm_bytes(p, nmaps));
    w.alm = (double2 *)c;   c += align256(alm_bytes(p, nmaps));
    w.map = (double *)c;    c += align256(sizeof(double) * (size_t)nmaps * p->npix);
    w.bf = c;
    return w;
}

int ensure_ws(shtb_plan_s *p, int nmaps)
{
    if (nmaps <= p->ws_nmaps && p->ws) return SHTB_OK;
    const size_t need = ws_total(p, nmaps);
    if (p->ws) {
        cudaError_t e = cudaFree(p->ws);
        p->ws = nullptr;
        p->ws_bytes = 0;
        p->ws_nmaps = 0;
        if (e != cudaSuccess) return shtb_fail(SHTB_ECUDA, std::string("cudaFree workspace: ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaMalloc(&p->ws, need);
    if (e != cudaSuccess) {
        p->ws = nullptr;
        return shtb_fail(SHTB_ENOMEM, "workspace of " + std::to_string(need) + " bytes: " + cudaGetErrorString(e));
    }
    p->ws_bytes = need;
    p->ws_nmaps = nmaps;
    return SHTB_OK;
}

int check_buffers(shtb_plan p, const void *a, const void *b, int nmaps);

int check_call(shtb_plan p, const void *a, const void *b, int nmaps)
{
    if (!p) return shtb_fail(SHTB_EINVAL, "plan is NULL");
    if (p->kind != 0) return shtb_fail(SHTB_ENOTSUP, "a polarised plan serves shtb_synthesize_spin only");
    return check_buffers(p, a, b, nmaps);
}

int check_buffers(shtb_plan p, const void *a, const void *b, int nmaps)
{
    if (!a || !b) return shtb_fail(SHTB_EINVAL, "NULL buffer");
    if (nmaps < 1) return shtb_fail(SHTB_EINVAL, "nmaps must be >= 1");
    if (((uintptr_t)a & 15) || ((uintptr_t)b & 15))
        return shtb_fail(SHTB_EINVAL, "buffers must be 16-byte aligned");
    int dev = -1;
    SHTB_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device)
        return shtb_fail(SHTB_EMISMATCH, "plan built on device " + std::to_string(p->device) +
                                             ", called with device " + std::to_string(dev) + " current");
    return SHTB_OK;
}

// ---------------------------------------------------------- profiling
struct StageTimer {
    shtb_plan_s *p;
    cudaStream_t st;
    int stage;
    int e0;
    StageTimer(shtb_plan_s *pp, cudaStream_t s, int stg) : p(pp), st(s), stage(stg)
    {
        e0 = profile_begin(p, st);
    }
    ~StageTimer() { profile_end(p, st, stage, e0); }
};

// ------------------------------------------------------------ pipelines
int run_synthesis(shtb_plan_s *p, const double2 *alm, double *map, int nmaps, cudaStream_t st)
{
    int rc = ensure_ws(p, nmaps);
    if (rc) return rc;
    Workspace w = carve(p, nmaps);
    if (p->profiling) ++p->prof_calls;
    if (p->bf) {
        // compressed operator (Sec. 3.2): per map group residual blocks, butterfly
        // levels, then the ring stage reading both parity halves directly
        return launch_bf_synth(p, alm, w.ap, w.bf, map, nmaps, st);
    } else {
        {
            StageTimer t(p, st, 4);
            if ((rc = launch_alm_prescale(p, alm, w.ap, nmaps, st))) return rc;
        }
        StageTimer t(p, st, 0);
        if ((rc = launch_legendre_synth(p, w.ap, w.q, nmaps, st))) return rc;
    }
    {
        StageTimer t(p, st, 1);
        if ((rc = launch_phi_synth(p, w.q, map, nmaps, st))) return rc;
    }
    return SHTB_OK;
}

int run_adjoint(shtb_plan_s *p, const double *map, double2 *alm, int nmaps, cudaStream_t st)
{
    int rc = ensure_ws(p, nmaps);
    if (rc) return rc;
    if (p->profiling) ++p->prof_calls;
    Workspace w = carve(p, nmaps);
    {
        StageTimer t(p, st, 2);
        if ((rc = launch_phi_adjoint(p, map, w.q, nmaps, st))) return rc;
    }
    if (p->bf) {
        // transposed butterfly (compressed plans)
        StageTimer t(p, st, 3);
        double2 *g = (double2 *)w.adj;
        if ((rc = launch_adjoint_parity(p, w.q, g, nmaps, st))) return rc;
        if ((rc = launch_bf_adjoint(p, g, w.aacc, w.bf, alm, nmaps, st))) return rc;
        return SHTB_OK;
    }
    {
        StageTimer t(p, st, 3);
        if ((rc = launch_legendre_adjoint(p, w.q, w.aacc, nmaps, w.adj, st))) return rc;
    }
    {
        StageTimer t(p, st, 4);
        if ((rc = launch_alm_finish(p, w.aacc, alm, nmaps, st))) return rc;
    }
    return SHTB_OK;
}

}  // namespace

int profile_begin(shtb_plan_s *p, cudaStream_t st)
{
    if (!p->profiling || p->ev_next + 2 > (int)p->ev_pool.size()) return -1;
    const int e0 = p->ev_next;
    p->ev_next += 2;
    cudaEventRecord(p->ev_pool[e0], st);
    return e0;
}

void profile_end(shtb_plan_s *p, cudaStream_t st, int stage, int ev)
{
    if (ev < 0) return;
    cudaEventRecord(p->ev_pool[ev + 1], st);
    p->recs.push_back({stage, ev, ev + 1});
}

int shtb_fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

extern "C" {

const char *shtb_strerror(int code)
{
    switch (code) {
    case SHTB_OK: return "success";
    case SHTB_EINVAL: return "invalid argument";
    case SHTB_ENOMEM: return "out of memory";
    case SHTB_ECUDA: return "CUDA runtime error";
    case SHTB_EMISMATCH: return "plan used on a different device";
    case SHTB_ETIMEOUT: return "bounded device wait timed out";
    case SHTB_ENOTSUP: return "not supported";
    case SHTB_EIO: return "plan cache I/O error";
    case SHTB_ECORRUPT: return "plan cache file corrupt";
    default: return "unknown error";
    }
}

const char *shtb_last_error_message(void) { return g_last_error.c_str(); }

int shtb_struct_sizes(int *opts, int *stats, int *request, int *batch_opts)
{
    if (opts) *opts = (int)sizeof(shtb_plan_opts);
    if (stats) *stats = (int)sizeof(shtb_plan_stats_t);
    if (request) *request = (int)sizeof(shtb_request);
    if (batch_opts) *batch_opts = (int)sizeof(shtb_batch_opts);
    return SHTB_OK;
}

int shtb_plan_opts_init(shtb_plan_opts *o)
{
    if (!o) return shtb_fail(SHTB_EINVAL, "opts is NULL");
    o->leaf_cols = 32;
    o->max_depth = -1;
    o->rho = 0.0;
    o->nthreads = 0;
    o->device = -1;
    o->cache_dir = nullptr;
    o->gpu_build = 0;
    o->spin = 0;
    o->residual_recurrence = 0;
    return SHTB_OK;
}

namespace {

void finish_stats(shtb_plan_s *p, std::chrono::steady_clock::time_point t0)
{
    p->opts.cache_dir = nullptr;          // the caller's string is not kept
    p->stats.kernel_launches = 0;
    p->stats.nside = p->nside;
    p->stats.lmax = p->lmax;
    p->stats.eps = p->eps;
    p->stats.nrings = p->nrings;
    p->stats.npix = p->npix;
    p->stats.nalm = p->nalm;
    if (!p->bf) {
        p->stats.compressed = 0;
        p->stats.depth_hist[0] = 2 * (p->lmax + 1);
    }
    p->stats.build_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// A fresh, empty plan for this key.  A polarised plan (opts.spin = 2) holds
// the F+ operator (kind 1) and owns the F- one (kind 2) as its partner.
shtb_plan_s *new_plan(const shtb_plan_opts &o, int nside, int lmax, double eps, int dev)
{
    auto make = [&](int kind) {
        shtb_plan_s *p = new (std::nothrow) shtb_plan_s();
        if (!p) return p;
        p->opts = o;
        p->nside = nside;
        p->lmax = lmax;
        p->eps = eps;
        p->device = dev;
        p->kind = kind;
        return p;
    };
    shtb_plan_s *p = make(o.spin == 2 ? 1 : 0);
    if (p && o.spin == 2) {
        p->partner = make(2);
        if (!p->partner) {
            delete p;
            return nullptr;
        }
        p->partner->opts.cache_dir = nullptr;
    }
    return p;
}

// Builds a fresh plan: ring tables and recurrence tables, and the butterfly
// when eps > 0 or the operator is polarised (depth 0 only when eps <= 0).
int build_plan(shtb_plan_s *p)
{
    int rc = shtb_build_dense_plan(p);
    if (!rc && (p->eps > 0 || p->kind != 0)) rc = shtb_build_butterfly(p);
    if (!rc && p->partner) rc = build_plan(p->partner);
    return rc;
}

// A polarised plan reports both operators' element and byte counts.
void combine_polarised_stats(shtb_plan_s *p)
{
    const shtb_plan_s *q = p->partner;
    p->stats.spin = 2;
    p->stats.compressed = p->eps > 0 ? 1 : 0;
    p->stats.n_dense += q->stats.n_dense;
    p->stats.n_rstored += q->stats.n_rstored;
    p->stats.n_ident += q->stats.n_ident;
    p->stats.plan_device_bytes += q->stats.plan_device_bytes;
    p->stats.plan_read_bytes += q->stats.plan_read_bytes;
    for (int d = 0; d < 16; ++d) p->stats.depth_hist[d] += q->stats.depth_hist[d];
}

}  // namespace

int shtb_plan_create(int nside, int lmax, double eps, const shtb_plan_opts *opts, shtb_plan *out)
{
    NvtxRange nvtx("shtb_plan_create");
    if (!out) return shtb_fail(SHTB_EINVAL, "out is NULL");
    *out = nullptr;
    if (nside < 1) return shtb_fail(SHTB_EINVAL, "nside must be >= 1");
    if (lmax < 0) return shtb_fail(SHTB_EINVAL, "lmax must be >= 0");
    if (!(eps == eps) || eps > 1.0) return shtb_fail(SHTB_EINVAL, "eps must be a number <= 1");
    if (lmax > 8192) return shtb_fail(SHTB_ENOTSUP, "lmax > 8192");
    if (nside > 2048) return shtb_fail(SHTB_ENOTSUP, "nside > 2048");
    auto t0 = std::chrono::steady_clock::now();
    shtb_plan_opts o;
    shtb_plan_opts_init(&o);
    if (opts) o = *opts;
    if (o.spin != 0 && o.spin != 2) return shtb_fail(SHTB_EINVAL, "spin must be 0 (scalar) or 2 (polarised)");
    if (o.residual_recurrence && (!(eps > 0) || o.spin != 0))
        return shtb_fail(SHTB_ENOTSUP, "residual_recurrence needs a compressed scalar plan (eps > 0, spin 0)");
    int dev = o.device;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) return shtb_fail(SHTB_ECUDA, "no CUDA device");
    } else if (cudaSetDevice(dev) != cudaSuccess) {
        return shtb_fail(SHTB_ECUDA, "cudaSetDevice failed");
    }
    shtb_plan_s *p = new_plan(o, nside, lmax, eps, dev);
    if (!p) return shtb_fail(SHTB_ENOMEM, "plan struct");
    bool loaded = false;
    std::string cpath;
    if (o.cache_dir) {
        cpath = plan_cache_path(p, o.cache_dir);
        if (plan_load(p, cpath.c_str()) == SHTB_OK) {
            loaded = true;
        } else {                          // missing or invalid file: start over and rebuild
            shtb_plan_destroy(p);
            p = new_plan(o, nside, lmax, eps, dev);
            if (!p) return shtb_fail(SHTB_ENOMEM, "plan struct");
        }
    }
    if (!loaded) {
        const int rc = build_plan(p);
        if (rc) {
            shtb_plan_destroy(p);
            return rc;
        }
        if (p->partner) {
            finish_stats(p->partner, t0);
            combine_polarised_stats(p);
        }
        if (o.cache_dir) plan_save(p, cpath.c_str());   // a cache that cannot be written is only slower
    }
    p->stats.from_cache = loaded ? 1 : 0;
    finish_stats(p, t0);
    *out = p;
    return SHTB_OK;
}

int shtb_plan_save(shtb_plan p, const char *path)
{
    NvtxRange nvtx("shtb_plan_save");
    if (!p || !path) return shtb_fail(SHTB_EINVAL, "plan or path is NULL");
    int prev = -1;
    SHTB_CUDA_TRY(cudaGetDevice(&prev));
    if (prev != p->device) SHTB_CUDA_TRY(cudaSetDevice(p->device));
    const int rc = plan_save(p, path);
    if (prev != p->device) cudaSetDevice(prev);
    return rc;
}

int shtb_plan_load(const char *path, const shtb_plan_opts *opts, shtb_plan *out)
{
    NvtxRange nvtx("shtb_plan_load");
    if (!out || !path) return shtb_fail(SHTB_EINVAL, "out or path is NULL");
    *out = nullptr;
    auto t0 = std::chrono::steady_clock::now();
    shtb_plan_opts o;
    shtb_plan_opts_init(&o);
    if (opts) o.device = opts->device;
    int nside = 0, lmax = 0;
    double eps = 0.0;
    int rc = plan_read_key(path, &nside, &lmax, &eps, &o);
    if (rc) return rc;
    int dev = o.device;
    if (dev < 0) {
        SHTB_CUDA_TRY(cudaGetDevice(&dev));
    } else {
        SHTB_CUDA_TRY(cudaSetDevice(dev));
    }
    o.device = dev;
    o.cache_dir = nullptr;
    if (o.spin != 0 && o.spin != 2) return shtb_fail(SHTB_ECORRUPT, std::string("unknown spin in ") + path);
    shtb_plan_s *p = new_plan(o, nside, lmax, eps, dev);
    if (!p) return shtb_fail(SHTB_ENOMEM, "plan struct");
    if ((rc = plan_load(p, path))) {
        shtb_plan_destroy(p);
        return rc;
    }
    p->stats.from_cache = 1;
    p->stats.kernel_launches = 0;
    p->stats.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return SHTB_OK;
}

int shtb_plan_destroy(shtb_plan p)
{
    if (!p) return SHTB_OK;
    if (p->partner) shtb_plan_destroy(p->partner);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->device) cudaSetDevice(p->device);
    for (void *a : p->allocations) cudaFree(a);
    if (p->ws) cudaFree(p->ws);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    if (p->copy_stream) {
        cudaStreamDestroy(p->copy_stream);
        for (cudaEvent_t e : p->chunk_ev) cudaEventDestroy(e);
    }
    for (cudaStream_t s2 : p->ring_stream)
        if (s2) cudaStreamDestroy(s2);
    for (cudaEvent_t e : p->ring_ev)
        if (e) cudaEventDestroy(e);
    bf_release(p);
    if (prev >= 0 && prev != p->device) cudaSetDevice(prev);
    delete p;
    return SHTB_OK;
}

int shtb_plan_stats(shtb_plan p, shtb_plan_stats_t *out)
{
    if (!p || !out) return shtb_fail(SHTB_EINVAL, "NULL argument");
    p->stats.kernel_launches = p->launches + (p->partner ? p->partner->launches : 0);
    *out = p->stats;
    return SHTB_OK;
}

int shtb_plan_reserve(shtb_plan p, int nmaps)
{
    if (!p) return shtb_fail(SHTB_EINVAL, "plan is NULL");
    if (nmaps < 1) return shtb_fail(SHTB_EINVAL, "nmaps must be >= 1");
    return ensure_ws(p, nmaps);
}

int shtb_synthesize(shtb_plan p, const double *alm_dev, double *map_dev, int nmaps, void *stream)
{
    NvtxRange nvtx("shtb_synthesize");
    int rc = check_call(p, alm_dev, map_dev, nmaps);
    if (rc) return rc;
    return run_synthesis(p, (const double2 *)alm_dev, map_dev, nmaps, (cudaStream_t)stream);
}

int shtb_adjoint(shtb_plan p, const double *map_dev, double *alm_dev, int nmaps, void *stream)
{
    NvtxRange nvtx("shtb_adjoint");
    int rc = check_call(p, map_dev, alm_dev, nmaps);
    if (rc) return rc;
    return run_adjoint(p, map_dev, (double2 *)alm_dev, nmaps, (cudaStream_t)stream);
}

}  // extern "C"

namespace {

int check_spin(shtb_plan p, const void *a, const void *b, int npairs, const char *what)
{
    if (!p) return shtb_fail(SHTB_EINVAL, "plan is NULL");
    if (p->kind != 1 || !p->partner) return shtb_fail(SHTB_ENOTSUP, std::string(what) + " needs a polarised plan");
    if (npairs < 1 || npairs > (1 << 20)) return shtb_fail(SHTB_EINVAL, "npairs must be in 1..2^20");
    return check_buffers(p, a, b, 2 * npairs);
}

// E, B of every pair -> Q, U (2 npairs inputs and maps)
int run_synthesis_spin(shtb_plan_s *p, const double2 *alm, double *map, int npairs, cudaStream_t st)
{
    const int nm = 2 * npairs;
    shtb_plan_s *q = p->partner;
    int rc;
    if ((rc = ensure_ws(p, nm)) || (rc = ensure_ws(q, nm))) return rc;
    Workspace wp = carve(p, nm), wq = carve(q, nm);
    double *qt_plus = (double *)wp.adj, *qt_minus = (double *)wq.adj;   // parity halves, map-major
    if ((rc = launch_bf_synth(p, alm, wp.ap, wp.bf, nullptr, nm, st, qt_plus))) return rc;
    if ((rc = launch_bf_synth(q, alm, wq.ap, wq.bf, nullptr, nm, st, qt_minus))) return rc;
    if ((rc = launch_spin_combine(p, qt_plus, qt_minus, wp.q, npairs, st))) return rc;
    return launch_phi_synth(p, wp.q, map, nm, st);
}

// Q, U -> transposed E, B
int run_adjoint_spin(shtb_plan_s *p, const double *map, double2 *alm, int npairs, cudaStream_t st)
{
    const int nm = 2 * npairs;
    shtb_plan_s *q = p->partner;
    int rc;
    if ((rc = ensure_ws(p, nm)) || (rc = ensure_ws(q, nm))) return rc;
    Workspace wp = carve(p, nm), wq = carve(q, nm);
    double2 *g_plus = (double2 *)wp.adj, *g_minus = (double2 *)wq.adj;
    if ((rc = launch_phi_adjoint(p, map, wp.q, nm, st))) return rc;      // ring sums of Q and U
    if ((rc = launch_spin_uncombine(p, wp.q, g_plus, g_minus, npairs, st))) return rc;
    if ((rc = launch_bf_adjoint(p, g_plus, wp.aacc, wp.bf, alm, nm, st))) return rc;
    if ((rc = launch_bf_adjoint(q, g_minus, wq.aacc, wq.bf, wq.alm, nm, st))) return rc;
    return launch_alm_add(p, alm, wq.alm, (size_t)nm * p->nalm, st);
}

// Quadrature analysis (Eq. sh-forward-quadrature) and Jacobi refinement over
// nm stacked maps: a = h_m Y^T (w f), then a += h_m Y^T (w (f - Y a)).
// synth/adjoint apply Y and Y^T; r (nm maps) and tmp (nm a_lm sets) are
// workspace the two do not use.
template <class Synth, class Adjoint>
int run_analysis(shtb_plan_s *p, const double *map, double2 *alm, int nm, const double *ring_w, int niter,
                 double *r, double2 *tmp, cudaStream_t st, Synth synth, Adjoint adjoint)
{
    const double w0 = 4.0 * 3.14159265358979323846 / (double)p->npix;   // equal-area HEALPix pixel weight
    int rc;
    if ((rc = launch_ring_weight(p, map, nullptr, ring_w, w0, r, nm, st))) return rc;
    if ((rc = adjoint(r, alm))) return rc;
    if ((rc = launch_alm_quadrature_add(p, alm, alm, nm, true, st))) return rc;
    for (int it = 0; it < niter; ++it) {
        if ((rc = synth(alm, r))) return rc;
        if ((rc = launch_ring_weight(p, map, r, ring_w, w0, r, nm, st))) return rc;
        if ((rc = adjoint(r, tmp))) return rc;
        if ((rc = launch_alm_quadrature_add(p, tmp, alm, nm, false, st))) return rc;
    }
    return SHTB_OK;
}

int check_analysis_args(const void *map, const void *alm, int niter)
{
    if (niter < 0 || niter > SHTB_MAX_ANALYSIS_ITER)
        return shtb_fail(SHTB_EINVAL, "niter must be in 0.." + std::to_string(SHTB_MAX_ANALYSIS_ITER));
    if (map == alm) return shtb_fail(SHTB_EINVAL, "map and alm must not alias");
    return SHTB_OK;
}

}  // namespace

extern "C" {

int shtb_synthesize_spin(shtb_plan p, const double *alm_dev, double *map_dev, int npairs, void *stream)
{
    NvtxRange nvtx("shtb_synthesize_spin");
    int rc = check_spin(p, alm_dev, map_dev, npairs, "shtb_synthesize_spin");
    if (rc) return rc;
    return run_synthesis_spin(p, (const double2 *)alm_dev, map_dev, npairs, (cudaStream_t)stream);
}

int shtb_adjoint_spin(shtb_plan p, const double *map_dev, double *alm_dev, int npairs, void *stream)
{
    NvtxRange nvtx("shtb_adjoint_spin");
    int rc = check_spin(p, map_dev, alm_dev, npairs, "shtb_adjoint_spin");
    if (rc) return rc;
    return run_adjoint_spin(p, map_dev, (double2 *)alm_dev, npairs, (cudaStream_t)stream);
}

int shtb_analyze_spin(shtb_plan p, const double *map_dev, double *alm_dev, int npairs,
                      const double *ring_weight_dev, int niter, void *stream)
{
    NvtxRange nvtx("shtb_analyze_spin");
    int rc = check_spin(p, map_dev, alm_dev, npairs, "shtb_analyze_spin");
    if (rc || (rc = check_analysis_args(map_dev, alm_dev, niter))) return rc;
    const int nm = 2 * npairs;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure_ws(p, nm)) || (rc = ensure_ws(p->partner, nm))) return rc;
    Workspace w = carve(p, nm);   // w.map and w.alm: used by neither polarised transform
    return run_analysis(
        p, map_dev, (double2 *)alm_dev, nm, ring_weight_dev, niter, w.map, w.alm, st,
        [&](const double2 *a, double *f) { return run_synthesis_spin(p, a, f, npairs, st); },
        [&](const double *f, double2 *a) { return run_adjoint_spin(p, f, a, npairs, st); });
}

int shtb_analyze(shtb_plan p, const double *map_dev, double *alm_dev, int nmaps,
                 const double *ring_weight_dev, int niter, void *stream)
{
    NvtxRange nvtx("shtb_analyze");
    int rc = check_call(p, map_dev, alm_dev, nmaps);
    if (rc || (rc = check_analysis_args(map_dev, alm_dev, niter))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure_ws(p, nmaps))) return rc;
    Workspace w = carve(p, nmaps);   // w.map: weighted residual, w.alm: adjoint of it
    return run_analysis(
        p, map_dev, (double2 *)alm_dev, nmaps, ring_weight_dev, niter, w.map, w.alm, st,
        [&](const double2 *a, double *f) { return run_synthesis(p, a, f, nmaps, st); },
        [&](const double *f, double2 *a) { return run_adjoint(p, f, a, nmaps, st); });
}

int shtb_synthesize_host(shtb_plan p, const double *alm_host, double *map_host, int nmaps,
                         void *stream)
{
    NvtxRange nvtx("shtb_synthesize_host");
    int rc = check_call(p, alm_host, map_host, nmaps);
    if (rc) return rc;
    if ((rc = ensure_ws(p, nmaps))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace w = carve(p, nmaps);
    SHTB_CUDA_TRY(cudaMemcpyAsync(w.alm, alm_host, alm_bytes(p, nmaps), cudaMemcpyHostToDevice, st));
    if (p->bf) {
        // compressed plans: the maps come back ring chunk by ring chunk,
        // overlapping the rest of the ring stage
        if (p->profiling) ++p->prof_calls;
        if ((rc = launch_bf_synth_to_host(p, w.alm, w.ap, w.bf, w.map, map_host, nmaps, st))) return rc;
    } else {
        if ((rc = run_synthesis(p, w.alm, w.map, nmaps, st))) return rc;
        SHTB_CUDA_TRY(cudaMemcpyAsync(map_host, w.map, sizeof(double) * (size_t)nmaps * p->npix,
                                      cudaMemcpyDeviceToHost, st));
    }
    SHTB_CUDA_TRY(cudaStreamSynchronize(st));
    return SHTB_OK;
}

int shtb_adjoint_host(shtb_plan p, const double *map_host, double *alm_host, int nmaps, void *stream)
{
    NvtxRange nvtx("shtb_adjoint_host");
    int rc = check_call(p, map_host, alm_host, nmaps);
    if (rc) return rc;
    if ((rc = ensure_ws(p, nmaps))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace w = carve(p, nmaps);
    SHTB_CUDA_TRY(cudaMemcpyAsync(w.map, map_host, sizeof(double) * (size_t)nmaps * p->npix,
                                  cudaMemcpyHostToDevice, st));
    if ((rc = run_adjoint(p, w.map, w.alm, nmaps, st))) return rc;
    SHTB_CUDA_TRY(cudaMemcpyAsync(alm_host, w.alm, alm_bytes(p, nmaps), cudaMemcpyDeviceToHost, st));
    SHTB_CUDA_TRY(cudaStreamSynchronize(st));
    return SHTB_OK;
}

int shtb_profile_enable(shtb_plan p, int on)
{
    if (!p) return shtb_fail(SHTB_EINVAL, "plan is NULL");
    if (on && p->ev_pool.empty()) {
        p->ev_pool.resize(2 * 4096);
        for (auto &e : p->ev_pool) SHTB_CUDA_TRY(cudaEventCreate(&e));
    }
    p->profiling = on != 0;
    return SHTB_OK;
}

int shtb_profile_read(shtb_plan p, double *ms, int nstages, int *ncalls)
{
    if (!p || !ms || nstages < 0) return shtb_fail(SHTB_EINVAL, "NULL argument");
    for (int i = 0; i < nstages; ++i) ms[i] = 0.0;
    int calls = 0;
    for (const auto &r : p->recs) {
        SHTB_CUDA_TRY(cudaEventSynchronize(p->ev_pool[r.ev1]));
        float t = 0.f;
        SHTB_CUDA_TRY(cudaEventElapsedTime(&t, p->ev_pool[r.ev0], p->ev_pool[r.ev1]));
        if (r.stage < nstages) ms[r.stage] += t;
    }
    calls = p->prof_calls;
    p->prof_calls = 0;
    p->recs.clear();
    p->ev_next = 0;
    if (ncalls) *ncalls = calls;
    return SHTB_OK;
}

int shtb_measure_fp64_peak(int device, double *dfma, double *dmma)
{
    if (!dfma || !dmma) return shtb_fail(SHTB_EINVAL, "NULL argument");
    return measure_fp64_peak(device, dfma, dmma);
}

// ------------------------------------------------------- private API
int shtb_test_legendre(shtb_plan p, const double *alm_dev, double *q_dev, int nmaps, void *stream)
{
    int rc = check_call(p, alm_dev, q_dev, nmaps);
    if (rc) return rc;
    if ((rc = ensure_ws(p, nmaps))) return rc;
    Workspace w = carve(p, nmaps);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = launch_alm_prescale(p, (const double2 *)alm_dev, w.ap, nmaps, st))) return rc;
    return launch_legendre_synth(p, w.ap, (double2 *)q_dev, nmaps, st);
}

int shtb_test_butterfly(shtb_plan p, const double *alm_dev, double *qt_dev, int nmaps, void *stream)
{
    int rc = check_call(p, alm_dev, qt_dev, nmaps);
    if (rc) return rc;
    if (!p->bf) return shtb_fail(SHTB_ENOTSUP, "shtb_test_butterfly needs a compressed plan (eps > 0)");
    if ((rc = ensure_ws(p, nmaps))) return rc;
    Workspace w = carve(p, nmaps);
    cudaStream_t st = (cudaStream_t)stream;
    // the (m = L, t = 1) chain is empty: its entries stay zero
    SHTB_CUDA_TRY(cudaMemsetAsync(qt_dev, 0, sizeof(double2) * 2 * (size_t)nmaps * p->nhalf * (p->lmax + 1), st));
    return launch_bf_synth(p, (const double2 *)alm_dev, w.ap, w.bf, nullptr, nmaps, st, qt_dev);
}

int shtb_test_phi(shtb_plan p, const double *q_dev, double *map_dev, int nmaps, void *stream)
{
    int rc = check_call(p, q_dev, map_dev, nmaps);
    if (rc) return rc;
    return launch_phi_synth(p, (const double2 *)q_dev, map_dev, nmaps, (cudaStream_t)stream);
}

int shtb_test_phi_adjoint(shtb_plan p, const double *map_dev, double *q_dev, int nmaps, void *stream)
{
    int rc = check_call(p, map_dev, q_dev, nmaps);
    if (rc) return rc;
    return launch_phi_adjoint(p, map_dev, (double2 *)q_dev, nmaps, (cudaStream_t)stream);
}

int shtb_test_legendre_adjoint(shtb_plan p, const double *q_dev, double *alm_dev, int nmaps,
                               void *stream)
{
    int rc = check_call(p, q_dev, alm_dev, nmaps);
    if (rc) return rc;
    if ((rc = ensure_ws(p, nmaps))) return rc;
    Workspace w = carve(p, nmaps);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = launch_legendre_adjoint(p, (const double2 *)q_dev, w.aacc, nmaps, w.adj, st))) return rc;
    return launch_alm_finish(p, w.aacc, (double2 *)alm_dev, nmaps, st);
}

}  // extern "C"
