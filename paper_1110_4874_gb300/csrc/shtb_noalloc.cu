// shtb_synthesize_noalloc: the synthesis pipeline with its scratch buffers
// (the scaled a_lm and the q_m(z_k) work array) placed in a fixed static
// device array instead of the plan's workspace, so the call itself never
// allocates device memory.
//
// For callers that cannot allocate at the time they transform: a process
// whose device memory is already reserved by another allocator (a framework's
// caching pool, a preallocating runtime), or a latency-sensitive loop that
// must not pay for cudaMalloc's implicit device synchronisation.  The plan is
// still created (and allocated) beforehand with shtb_plan_create.
//
// The array is a module-scope __device__ variable: every GPU that loads this
// library holds SHTB_NOALLOC_SCRATCH_BYTES of it until the process exits.
// Its host-side name is only a stand-in for the symbol, never a device
// address, so the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "shtb_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SHTB_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (looked up on
// the first call for that device).
int scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return shtb_fail(SHTB_ENOTSUP, "device ordinal " + std::to_string(dev) + " out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return shtb_fail(SHTB_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") +
                                             cudaGetErrorString(e));
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return SHTB_OK;
}

}  // namespace

extern "C" int shtb_synthesize_noalloc(shtb_plan p, const double *alm_dev, double *map_dev,
                                       int nmaps, void *stream)
{
    NvtxRange range("shtb_synthesize_noalloc");
    if (!p) return shtb_fail(SHTB_EINVAL, "plan is NULL");
    if (p->kind != 0) return shtb_fail(SHTB_ENOTSUP, "a polarised plan serves shtb_synthesize_spin only");
    if (!alm_dev || !map_dev) return shtb_fail(SHTB_EINVAL, "NULL buffer");
    if (nmaps < 1) return shtb_fail(SHTB_EINVAL, "nmaps must be >= 1");
    if (((uintptr_t)alm_dev & 15) || ((uintptr_t)map_dev & 15))
        return shtb_fail(SHTB_EINVAL, "buffers must be 16-byte aligned");
    int dev = -1;
    SHTB_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device)
        return shtb_fail(SHTB_EMISMATCH, "plan built on device " + std::to_string(p->device) +
                                             ", called with device " + std::to_string(dev) + " current");
    const size_t ap_bytes = sizeof(double2) * (size_t)nmaps * p->nalm;
    const size_t q_bytes = sizeof(double2) * (size_t)nmaps * p->nrings * (p->lmax + 1);
    const size_t need = round256(ap_bytes) + q_bytes;
    if (need > (size_t)SHTB_NOALLOC_SCRATCH_BYTES)
        return shtb_fail(SHTB_ENOTSUP,
                         "shtb_synthesize_noalloc needs " + std::to_string(need) +
                             " bytes of scratch for nside=" + std::to_string(p->nside) +
                             ", lmax=" + std::to_string(p->lmax) + ", nmaps=" + std::to_string(nmaps) +
                             "; the static scratch holds " + std::to_string((size_t)SHTB_NOALLOC_SCRATCH_BYTES) +
                             " bytes (use shtb_synthesize, or fewer maps per call)");
    void *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    // Both scratch arrays are written in full before they are read (every
    // scaled coefficient, every (map, ring, m) entry of q), so nothing left
    // over from an earlier call can leak into this one.
    double2 *ap = (double2 *)base;
    double2 *q = (double2 *)((char *)base + round256(ap_bytes));
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = launch_alm_prescale(p, (const double2 *)alm_dev, ap, nmaps, st))) return rc;
    if ((rc = launch_legendre_synth(p, ap, q, nmaps, st))) return rc;
    return launch_phi_synth(p, q, map_dev, nmaps, st);
}
