// Butterfly-compressed Legendre operator: host-side build structures and the
// flat device work-item format consumed by the apply kernels.  Internal.
#pragma once

#include <climits>
#include <vector>

#include "shtb_internal.h"

namespace shtb {

constexpr int kMaxCand = 128;        // candidate columns per node (shared-memory bound)
constexpr int kZeroCol = INT_MIN;    // column in the crop: contributes nothing

// One interpolative decomposition A[:, C] ~= A[:, skel] [I | T].
struct IdResult {
    int k = 0;                       // rank
    std::vector<int> skel;           // positions in C of the skeleton, in u order
    std::vector<int> kind;           // per position: >= 0 identity index, -1-d dense column d, kZeroCol
    std::vector<int> dense_pos;      // dense column d -> position in C (ascending)
    std::vector<double> T;           // k x nd, row-major
};

IdResult interp_decomp(const double *A, int rows, int n, int lda, double eps, double abs_floor);

class GpuIdPool;

struct BfParams {
    double eps = 1e-10;
    double abs_floor = 1e-30;        // the Appendix's negligible magnitude
    int leaf_cols = 32;
    int max_depth = -1;
    GpuIdPool *gpu = nullptr;        // non-null: the IDs of each level run batched on the GPU
    int slot = 0;                    // the calling thread's slot in that pool
};

// Residual block of one chain (local offsets).
struct BfRLocal {
    int j0 = 0, nrows = 0, k = 0;
    int interval = 0;                // index of its row interval at the chain's depth
    bool to_rings = false;           // depth 0: outputs go straight to q^t rings
    long long out_off = 0;           // u entry offset (within the chain's region)
    std::vector<int> rings;
    std::vector<int> cols;           // the half-ring of each column
    std::vector<double> data;        // nrows x k, row-major
};

// One level item: two sibling nodes that share a candidate list.
struct BfItemLocal {
    int level = 0, nc = 0;
    int k[2] = {0, 0};
    long long u_off[2] = {0, 0};
    std::vector<int> dense_pos[2];
    std::vector<int> ident_pos[2];
    std::vector<double> T[2];
    bool to_rings = false;
    long long out_off = 0;
    std::vector<int> rings;
};

struct BfChain {
    int n = 0, depth = 0;
    long long cost = 0;
    long long region = 0;            // u entries per buffer
    std::vector<BfRLocal> rblocks;
    std::vector<BfItemLocal> items;  // ordered from the top level down
    std::vector<std::pair<int, int>> top_rows;   // row intervals at the chosen depth
};

int compress_chain(const double *Lam, int n, int Z, const BfParams &prm, BfChain *out);
void apply_chain_host(const BfChain &ch, int Z, const double *a, double *q);

}  // namespace shtb

// ------------------------------------------------------------ device format
// All offsets are absolute within the plan-wide arrays.  A u "entry" holds
// one value per real component of the map group (2 x maps doubles).
struct BfRItem {
    int m, t;
    int j0, nrows, k;
    int to_rings;                    // 1: write q^t entries listed at idx_off
    long long data_off;              // doubles: nrows x k row-major (stored R)
    long long out_off;               // u entry offset (to_rings = 0) or int offset of entry list
    long long rs_off;                // first of the block's k RecStart (regenerated R)
};

// Start of the jump-two recurrence for one column of a residual block, in
// plans that regenerate R (Eq. three-term; Ptilde = sigma V): the column's
// half-ring, the first block row at or past the 1e-30 crop (nrows: the
// column is zero in this block), and V at that row and the next.
struct RecStart {
    int ring, start;
    double v0, v1;
};

struct BfItem {
    int nc;
    int k[2], nd[2];
    int to_rings;                    // 1: outputs to q^t entries listed at out_off (ints)
    long long u_off[2];              // u entry offsets of the two children
    long long dpos_off[2];           // int offsets: dense column -> candidate position
    long long ipos_off[2];           // int offsets: identity index -> candidate position
    long long T_off[2];              // double offsets: k x nd row-major
    long long out_off;               // u entry offset of the output, or int offset of q^t entries
};

// Adjoint: all residual blocks of one (chain, row interval), so that each
// chain row of a_lm is written by exactly one warp.
struct BfRGroup {
    int m, t, r0, r1, nblk;
    long long blk_off;               // int offset: indices into the residual item list
};

// Per-plan device data of the compressed operator.
struct BfPlanDev {
    int depth_max = 0;
    const BfRItem *ritems = nullptr;
    int n_ritems = 0;
    const BfRGroup *rgroups = nullptr;
    int n_rgroups = 0;
    std::vector<const BfItem *> level_items;    // level l at [l-1]
    std::vector<int> level_counts;
    std::vector<int> level_maxnc;               // largest candidate list per level
    const int *ints = nullptr;
    const double *dbl = nullptr;
    const int *depth_parity = nullptr;   // per chain (m*2 + t): depth % 2 (u buffer of its R output)
    const RecStart *rstart = nullptr;    // regenerated R: one per (block, column)
    bool rec = false;                    // R regenerated by the recurrence, not stored
    long long n_rgen = 0;
    long long u_entries = 0;         // entries per u buffer
    long long qt_entries = 0;        // (L+1) * 2 * nhalf
    long long n_dense = 0, n_r = 0, n_ident = 0;
};

namespace shtb {
RecStart block_column_start(int n, int t, int j0, int nrows, int ring, double x, bool sform, const RecCoef *cf,
                            int js, double2 vs);
}

// Builds the compressed operator of a plan (eps > 0) and uploads it.
int shtb_build_butterfly(shtb_plan_s *p);
