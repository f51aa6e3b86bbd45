// Batched interpolative decompositions on the GPU for the plan builder
// (Sec. 3.1, Eq. ID): the same column-pivoted Householder QR, truncation rule
// and interpolation matrix as the host routine interp_decomp, one CTA per
// block.  Internal; not part of the C ABI.
#pragma once

#include <vector>

#include "shtb_butterfly.h"

namespace shtb {

// One block: rows x nc, column-major with leading dimension rows, at
// element offset `off` of the batch's data array.
struct IdBlock {
    long long off;
    int rows, nc;
};

class GpuIdPool;   // per-thread device buffers and streams

// A pool for up to nthreads concurrent callers on `device`; nullptr on failure.
GpuIdPool *gpu_id_pool_create(int device, int nthreads);
void gpu_id_pool_destroy(GpuIdPool *pool);

// A pinned host buffer of at least nelem doubles owned by the caller's slot,
// for gathering the blocks straight into (gpu_id_run then copies nothing on
// the host); nullptr on allocation failure.  Valid until the slot's next call.
double *gpu_id_staging(GpuIdPool *pool, int slot, long long nelem);

// IDs of every block of `data` (host memory, the blocks' elements), into
// out[i] exactly as interp_decomp(data + blocks[i].off, rows, nc, rows, eps,
// abs_floor) defines them (up to the order of floating-point sums).
// slot: the caller's thread index (< nthreads).  Returns SHTB_OK or an error.
int gpu_id_run(GpuIdPool *pool, int slot, const double *data, long long nelem,
               const std::vector<IdBlock> &blocks, double eps, double abs_floor,
               std::vector<IdResult> &out);

}  // namespace shtb
