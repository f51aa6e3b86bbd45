// Batched serving: many synthesis requests of different (Nside, L, eps) in
// ONE persistent kernel launch, captured in a CUDA graph on the first run --
// or, where the autotuner finds it faster, a CUDA graph of the stand-alone
// stage kernels over the merged map groups on several streams.
//
// Requests that share a plan are merged along the map axis, so every stored
// element of that plan's compressed operator is read once per group of up to
// 8 maps (the paper's remark that many simultaneous transforms amortise the
// precomputed data, Sec. 3.3).  The persistent kernel runs the same item
// bodies as the stand-alone stage kernels (shtb_bf_items.cuh,
// shtb_phi_items.cuh), reading everything produced earlier in the launch
// through L2 only, so every map it writes equals the single-request result
// bit for bit.  The work of the whole batch is one list of items -- a_lm
// gather (a warp per order m), residual blocks and butterfly levels (a warp
// per item), ring transforms (a block per ring and map) -- cut into packs of
// one map group's stage.  A pack first waits for the last non-empty earlier
// stage of its own map group (the gather of its plan for the residual
// blocks), so a small plan's rings can run while a large plan's levels are
// still going.  Resident blocks claim packs from a global counter in phase
// order (every dependency lies in an earlier phase), so a claimed pack only
// ever waits on packs claimed before it and every wait ends; it is still
// bounded (spin_limit polls), after which the kernel sets an error flag and
// returns, and the host reports SHTB_ETIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "shtb_bf_items.cuh"
#include "shtb_butterfly.h"
#include "shtb_internal.h"
#include "shtb_phi_items.cuh"

namespace {

enum WorkType { W_GATHER = 0, W_RES = 1, W_LEVEL = 2, W_PHI = 3 };

struct BatchWork {
    int type;
    int g;        // plan group
    int mg;       // map group (index into the flat map-group table)
    int idx;      // m (gather), residual item, level item or ring
    int aux;      // level (W_LEVEL); map within the group (W_PHI)
    int kind;     // ring transform kind (W_PHI)
};

struct BatchPack {
    int first, count, block;          // block = 1: one ring item for the whole block
    int dep, need;                    // wait until counter dep reaches need (dep < 0: no wait)
    int cnt;                          // counter the pack adds its item count to
};

struct BatchMG {                      // one map group of one plan group
    double *u0, *u1, *qt;
    int b0, nb;
};

struct BatchGroupDev {
    PlanView v;
    const BfRItem *ritems;
    const BfItem *litems[16];
    const int *ints;
    const double *dbl;
    const int *depth_parity;
    double2 *ai;                      // [nalm][nmaps]
    int nmaps;
    const double2 *const *alm_of_map; // request a_lm of each merged map
    double *const *map_of_map;        // request output map of each merged map
};

struct BatchDev {
    const BatchWork *work;
    const BatchPack *packs;
    int npacks;
    const BatchGroupDev *groups;
    const BatchMG *mgs;
    int *counters;                    // zeroed before every run
    int *next;                        // pack claims
    int *err;
    int scratch;                      // doubles of level-item scratch per warp
    long long spin_limit;
};

template <int NB>
__device__ void warp_item(const BatchDev &bd, const BatchWork &w, double *wsm, int lane)
{
    const BatchGroupDev &G = bd.groups[w.g];
    const BatchMG &M = bd.mgs[w.mg];
    if (w.type == W_RES) {
        const BfRItem it = G.ritems[w.idx];
        double *ubuf = G.depth_parity[it.m * 2 + it.t] ? M.u1 : M.u0;
        shtb_dev::bf_r_item<NB, true>(it, G.v.lmax, G.v.nhalf, G.ints, G.dbl, G.ai, G.nmaps, M.b0, ubuf, M.qt,
                                      lane);
    } else {
        const double *uin = (w.aux % 2) ? M.u1 : M.u0;
        double *uout = ((w.aux - 1) % 2) ? M.u1 : M.u0;
        shtb_dev::bf_level_item<NB, true>(G.litems[w.aux - 1][w.idx], G.v.lmax, G.v.nhalf, G.ints, G.dbl, uin,
                                          uout, M.qt, wsm, lane);
    }
}

// a_lm of the merged maps into ai[idx][map] (Im a_l0 = 0), one order m
__device__ void gather_item(const BatchDev &bd, const BatchWork &w, int lane)
{
    const BatchGroupDev &G = bd.groups[w.g];
    const int m = w.idx, L = G.v.lmax;
    const long long off = shtb_dev::alm_off(L, m);
    const int n = L - m + 1;
    for (int i = lane; i < n * G.nmaps; i += 32) {
        const int b = i / n, dl = i - b * n;
        const long long idx = off + dl;
        const double2 a = G.alm_of_map[b][idx];
        G.ai[(size_t)idx * G.nmaps + b] = make_double2(a.x, m == 0 ? 0.0 : a.y);
    }
}

// one ring of one map of a map group, by the whole block, from the group's
// parity halves (fused combine, as in phi_synth_qt_kernel)
__device__ void ring_item(const BatchDev &bd, const BatchWork &w, double2 *sm)
{
    const BatchGroupDev &G = bd.groups[w.g];
    const BatchMG &M = bd.mgs[w.mg];
    const double2 *qt = reinterpret_cast<const double2 *>(M.qt);
    double *out = G.map_of_map[M.b0 + w.aux] + G.v.ring_start[w.idx];
    switch (w.kind) {
    case shtb_dev::kBluestein:
        shtb_dev::phi_synth_ring_qt<shtb_dev::kBluestein, true>(G.v, w.idx, qt, w.aux, out, sm);
        break;
    case shtb_dev::kDirectBig:
        shtb_dev::phi_synth_ring_qt<shtb_dev::kDirectBig, true>(G.v, w.idx, qt, w.aux, out, sm);
        break;
    default:
        shtb_dev::phi_synth_ring_qt<shtb_dev::kDirect, true>(G.v, w.idx, qt, w.aux, out, sm);
        break;
    }
}

// at most 8 warps per block, two blocks per SM (128 registers a thread:
// the radix-11/13 and Rader ring bodies need about that many)
__global__ void __launch_bounds__(256, 2) batch_kernel(BatchDev bd)
{
    extern __shared__ double bsm[];
    __shared__ int s_pack, s_abort;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            s_pack = atomicAdd(bd.next, 1);
            s_abort = 0;
        }
        __syncthreads();
        const int pk = s_pack;
        if (pk >= bd.npacks) return;
        const BatchPack P = bd.packs[pk];
        if (P.dep >= 0 && threadIdx.x == 0) {
            long long polls = 0;
            while (atomicAdd(&bd.counters[P.dep], 0) < P.need) {
                if (atomicAdd(bd.err, 0) != 0 || ++polls > bd.spin_limit) {
                    atomicExch(bd.err, 1);
                    s_abort = 1;
                    break;
                }
                __nanosleep(200);
            }
            __threadfence();
        }
        __syncthreads();
        if (s_abort) return;
        if (P.block) {
            ring_item(bd, bd.work[P.first], reinterpret_cast<double2 *>(bsm));
        } else if (wib < P.count) {
            const BatchWork w = bd.work[P.first + wib];
            if (w.type == W_GATHER) {
                gather_item(bd, w, lane);
            } else {
                double *wsm = bsm + (size_t)wib * bd.scratch;
                switch (bd.mgs[w.mg].nb) {
                case 8: warp_item<8>(bd, w, wsm, lane); break;
                case 4: warp_item<4>(bd, w, wsm, lane); break;
                case 2: warp_item<2>(bd, w, wsm, lane); break;
                default: warp_item<1>(bd, w, wsm, lane); break;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&bd.counters[P.cnt], P.count);
        }
    }
}


}  // namespace

struct shtb_batch_s {
    int device = 0;
    shtb_batch_opts opts{};
    std::vector<shtb_request> reqs;
    struct Group {
        shtb_plan_s *plan;
        int nmaps = 0;
        std::vector<const double2 *> alm_of_map;
        std::vector<double *> map_of_map;
    };
    std::vector<Group> groups;
    std::vector<void *> allocs;
    // device tables of the current schedule
    BatchDev dev{};
    int ncounters = 0, warps = 4, grid = 0;
    int stall_counter = -1;           // the gather counter shtb_test_batch_stall holds back
    std::vector<char> host_packs;     // the uploaded pack table (BatchPack records)
    size_t smem = 0;
    std::vector<void *> sched_allocs;
    // stage-kernel schedule: per plan group the merged a_lm and pointer
    // tables, per map group its u buffers and q^t, and the stream it runs on
    int mode = 0;                     // 0 persistent kernel, 1 stage-kernel graph
    int nstreams = 1;
    struct GMapGroup {
        int b0, nb, stream;
        double *u0, *u1, *qt;
        double cost;
    };
    struct GPlanGroup {
        shtb_plan_s *plan;
        int nmaps;
        double2 *ai;
        const double2 *const *alm_tab;
        double *const *map_tab;
        std::vector<GMapGroup> mgs;
    };
    std::vector<GPlanGroup> gg;
    std::vector<cudaStream_t> side;   // streams 1 .. nstreams-1 (stream 0 is the caller's)
    std::vector<cudaEvent_t> fork_join;
    // graph
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    cudaStream_t own_stream = nullptr;
    double tuned_ms = 0.0;
};

namespace {

int balloc(std::vector<void *> &list, void **p, size_t bytes, const void *src = nullptr)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess)
        return shtb_fail(SHTB_ENOMEM, std::string("batch allocation: ") + cudaGetErrorString(e));
    list.push_back(*p);
    if (src && bytes) {
        e = cudaMemcpy(*p, src, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return shtb_fail(SHTB_ECUDA, std::string("batch upload: ") + cudaGetErrorString(e));
    }
    return SHTB_OK;
}

void free_schedule(shtb_batch_s *b)
{
    for (void *p : b->sched_allocs) cudaFree(p);
    b->sched_allocs.clear();
    b->gg.clear();
    b->dev = BatchDev{};
    b->ncounters = 0;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
}

// relative work of one ring transform (for the largest-first order)
long long ring_cost(const shtb_plan_s *p, int kind, int r)
{
    const long long K = p->ring_J[r] / 2;
    long long lg = 1;
    while ((1LL << lg) < K) ++lg;
    return kind == shtb_dev::kBluestein ? 8 * K * (lg + 1) : K * lg;
}

// Builds the work list, packs and device tables for `warps` warps per block
// and map groups of at most `width` maps; work inside a phase in decreasing
// size (lpt = 1) or in plan order (lpt = 0).
int build_schedule(shtb_batch_s *b, int warps, int width, int lpt)
{
    free_schedule(b);
    b->mode = 0;
    std::vector<BatchGroupDev> gdev(b->groups.size());
    std::vector<BatchMG> mgs;
    int dmax = 0, cmax = 2, maxnc = 1;
    for (auto &G : b->groups) {
        const BfPlanDev &bf = *G.plan->bf;
        dmax = std::max(dmax, bf.depth_max);
        for (int nc : bf.level_maxnc) maxnc = std::max(maxnc, nc);
    }
    // phases: gather 0, residual blocks 1, level l at 2 + (dmax - l), rings 2 + dmax
    const int nphase = 3 + dmax;
    struct Unit {                     // the items of one stage of one map group (or one plan's gather)
        int phase, dep, need, cnt, block;
        std::vector<BatchWork> items;
        std::vector<long long> cost;
    };
    std::vector<Unit> units;
    int ncounters = 0;
    size_t ring_entries = 1;
    int rc;
    for (size_t g = 0; g < b->groups.size(); ++g) {
        auto &G = b->groups[g];
        shtb_plan_s *p = G.plan;
        const BfPlanDev &bf = *p->bf;
        if (bf.depth_max > 16) return shtb_fail(SHTB_ENOTSUP, "butterfly deeper than the batch tables");
        BatchGroupDev &D = gdev[g];
        D.v = p->view;
        D.ritems = bf.ritems;
        for (int l = 0; l < 16; ++l) D.litems[l] = l < bf.depth_max ? bf.level_items[l] : nullptr;
        D.ints = bf.ints;
        D.dbl = bf.dbl;
        D.depth_parity = bf.depth_parity;
        D.nmaps = G.nmaps;
        void *d;
        if ((rc = balloc(b->sched_allocs, &d, sizeof(double2) * (size_t)p->nalm * G.nmaps))) return rc;
        D.ai = (double2 *)d;
        if ((rc = balloc(b->sched_allocs, &d, sizeof(void *) * G.nmaps, G.alm_of_map.data()))) return rc;
        D.alm_of_map = (const double2 *const *)d;
        if ((rc = balloc(b->sched_allocs, &d, sizeof(void *) * G.nmaps, G.map_of_map.data()))) return rc;
        D.map_of_map = (double *const *)d;
        ring_entries = std::max<size_t>(ring_entries, (size_t)std::max({p->max_K_direct, p->max_M_mx, p->max_K_big}));
        // ring transform kind of every ring, from the plan's ring lists
        std::vector<int> kind(p->nrings, shtb_dev::kDirect);
        for (int r : p->blue_rings) kind[r] = shtb_dev::kBluestein;
        for (int r : p->big_rings) kind[r] = shtb_dev::kDirectBig;
        // ---- gather of this plan group
        Unit ug{0, -1, 0, ncounters++, 0, {}, {}};
        const int gather_cnt = ug.cnt;
        for (int m = 0; m <= p->lmax; ++m) {
            ug.items.push_back({W_GATHER, (int)g, 0, m, 0, 0});
            ug.cost.push_back((long long)(p->lmax - m + 1) * G.nmaps);
        }
        const int gather_total = (int)ug.items.size();
        units.push_back(std::move(ug));
        // host copies of the item lists, for the costs
        std::vector<BfRItem> rh(bf.n_ritems);
        if (bf.n_ritems)
            SHTB_CUDA_TRY(cudaMemcpy(rh.data(), bf.ritems, sizeof(BfRItem) * bf.n_ritems, cudaMemcpyDeviceToHost));
        std::vector<std::vector<BfItem>> lh(bf.depth_max);
        for (int l = 1; l <= bf.depth_max; ++l) {
            lh[l - 1].resize(bf.level_counts[l - 1]);
            if (!lh[l - 1].empty())
                SHTB_CUDA_TRY(cudaMemcpy(lh[l - 1].data(), bf.level_items[l - 1], sizeof(BfItem) * lh[l - 1].size(),
                                         cudaMemcpyDeviceToHost));
        }
        // ---- map groups of power-of-two widths up to `width`
        for (int b0 = 0; b0 < G.nmaps;) {
            const int left = G.nmaps - b0;
            int nb = 1;
            while (nb * 2 <= std::min(left, width)) nb *= 2;
            cmax = std::max(cmax, 2 * nb);
            BatchMG M{};
            M.b0 = b0;
            M.nb = nb;
            const size_t entry = sizeof(double) * 2 * nb;
            if ((rc = balloc(b->sched_allocs, &d, entry * (size_t)bf.u_entries))) return rc;
            M.u0 = (double *)d;
            if ((rc = balloc(b->sched_allocs, &d, entry * (size_t)bf.u_entries))) return rc;
            M.u1 = (double *)d;
            if ((rc = balloc(b->sched_allocs, &d, entry * (size_t)bf.qt_entries))) return rc;
            M.qt = (double *)d;
            const int mg = (int)mgs.size();
            mgs.push_back(M);
            // each stage waits for the last non-empty stage before it
            int dep = gather_cnt, need = gather_total;
            if (bf.n_ritems > 0) {
                Unit u{1, dep, need, ncounters++, 0, {}, {}};
                for (int i = 0; i < bf.n_ritems; ++i) {
                    u.items.push_back({W_RES, (int)g, mg, i, 0, 0});
                    u.cost.push_back((long long)rh[i].nrows * rh[i].k * nb);
                }
                dep = u.cnt;
                need = (int)u.items.size();
                units.push_back(std::move(u));
            }
            for (int l = bf.depth_max; l >= 1; --l) {
                if (lh[l - 1].empty()) continue;
                Unit u{2 + (dmax - l), dep, need, ncounters++, 0, {}, {}};
                for (size_t i = 0; i < lh[l - 1].size(); ++i) {
                    const BfItem &it = lh[l - 1][i];
                    u.items.push_back({W_LEVEL, (int)g, mg, (int)i, l, 0});
                    u.cost.push_back(((long long)it.k[0] * it.nd[0] + (long long)it.k[1] * it.nd[1] + it.nc) * nb);
                }
                dep = u.cnt;
                need = (int)u.items.size();
                units.push_back(std::move(u));
            }
            Unit ur{2 + dmax, dep, need, ncounters++, 1, {}, {}};
            for (int bl = 0; bl < nb; ++bl)
                for (int r = 0; r < p->nrings; ++r) {
                    ur.items.push_back({W_PHI, (int)g, mg, r, bl, kind[r]});
                    ur.cost.push_back(ring_cost(p, kind[r], r));
                }
            units.push_back(std::move(ur));
            b0 += nb;
        }
    }
    // ---- packs in phase order; within a phase the heaviest work first
    std::vector<BatchWork> work;
    std::vector<BatchPack> packs;
    std::vector<std::pair<long long, std::pair<int, int>>> order;   // (cost, (unit, first item))
    for (int ph = 0; ph < nphase; ++ph) {
        order.clear();
        for (size_t u = 0; u < units.size(); ++u) {
            Unit &U = units[u];
            if (U.phase != ph) continue;
            std::vector<int> ord(U.items.size());
            for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
            if (lpt) std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return U.cost[a] > U.cost[c]; });
            std::vector<BatchWork> it2;
            std::vector<long long> c2;
            for (int i : ord) {
                it2.push_back(U.items[i]);
                c2.push_back(U.cost[i]);
            }
            U.items.swap(it2);
            U.cost.swap(c2);
            const int per = U.block ? 1 : warps;
            for (int i = 0; i < (int)U.items.size(); i += per) {
                long long c = 0;
                for (int k = i; k < std::min<int>(i + per, (int)U.items.size()); ++k) c += U.cost[k];
                order.push_back({c, {(int)u, i}});
            }
        }
        if (lpt) std::stable_sort(order.begin(), order.end(), [](const auto &a, const auto &c) { return a.first > c.first; });
        for (auto &o : order) {
            Unit &U = units[o.second.first];
            const int i = o.second.second, per = U.block ? 1 : warps;
            const int n = std::min(per, (int)U.items.size() - i);
            packs.push_back({(int)work.size(), n, U.block, U.dep, U.need, U.cnt});
            for (int k = i; k < i + n; ++k) work.push_back(U.items[k]);
        }
    }
    void *d;
    if ((rc = balloc(b->sched_allocs, &d, sizeof(BatchWork) * work.size(), work.data()))) return rc;
    b->dev.work = (const BatchWork *)d;
    if ((rc = balloc(b->sched_allocs, &d, sizeof(BatchPack) * packs.size(), packs.data()))) return rc;
    b->dev.packs = (const BatchPack *)d;
    b->host_packs.assign((const char *)packs.data(), (const char *)(packs.data() + packs.size()));
    b->dev.npacks = (int)packs.size();
    if ((rc = balloc(b->sched_allocs, &d, sizeof(BatchGroupDev) * gdev.size(), gdev.data()))) return rc;
    b->dev.groups = (const BatchGroupDev *)d;
    if ((rc = balloc(b->sched_allocs, &d, sizeof(BatchMG) * mgs.size(), mgs.data()))) return rc;
    b->dev.mgs = (const BatchMG *)d;
    if ((rc = balloc(b->sched_allocs, &d, sizeof(int) * (size_t)(ncounters + 2)))) return rc;
    b->dev.counters = (int *)d;
    b->dev.next = b->dev.counters + ncounters;
    b->dev.err = b->dev.counters + ncounters + 1;
    b->dev.spin_limit = b->opts.spin_limit > 0 ? b->opts.spin_limit : 20000000LL;
    // level-item scratch per warp: the batch's longest candidate list x the
    // most doubles per candidate any of its map groups needs (C + 1 from 4
    // maps up, 2 C below; C = 2 x maps)
    if (cmax > 16 || maxnc > shtb::kMaxCand) return shtb_fail(SHTB_EINVAL, "map group or candidate list too large");
    b->dev.scratch = maxnc * std::max(shtb_dev::level_scratch_per_cand(cmax),
                                      shtb_dev::level_scratch_per_cand(std::min(cmax, 4)));
    b->ncounters = ncounters;
    b->stall_counter = 0;             // the first plan group's gather
    b->warps = warps;
    b->smem = std::max(sizeof(double2) * ring_entries, sizeof(double) * (size_t)warps * b->dev.scratch);
    if (b->smem > 227 * 1024) return shtb_fail(SHTB_ENOTSUP, "batch kernel shared memory above 227 KB");
    SHTB_CUDA_TRY(cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    int per_sm = 0, nsm = 0;
    SHTB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, 32 * warps, b->smem));
    SHTB_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
    if (per_sm < 1) return shtb_fail(SHTB_ENOTSUP, "batch kernel does not fit on an SM");
    b->grid = std::min(b->dev.npacks, nsm * per_sm);
    return SHTB_OK;
}

// Stage-kernel schedule: the stand-alone stage kernels over merged map
// groups of up to `width` maps (residual blocks, butterfly levels, ring
// FFTs writing each map through its pointer), the map groups spread over
// `nstreams` streams by decreasing work so that small plans overlap big ones.
int build_graph_schedule(shtb_batch_s *b, int width, int nstreams)
{
    free_schedule(b);
    b->mode = 1;
    b->nstreams = nstreams;
    int rc;
    void *d;
    std::vector<std::pair<double, std::pair<int, int>>> order;   // (cost, (group, map group))
    for (size_t g = 0; g < b->groups.size(); ++g) {
        auto &G = b->groups[g];
        shtb_plan_s *p = G.plan;
        const BfPlanDev &bf = *p->bf;
        shtb_batch_s::GPlanGroup P{};
        P.plan = p;
        P.nmaps = G.nmaps;
        if ((rc = balloc(b->sched_allocs, &d, sizeof(double2) * (size_t)p->nalm * G.nmaps))) return rc;
        P.ai = (double2 *)d;
        if ((rc = balloc(b->sched_allocs, &d, sizeof(void *) * G.nmaps, G.alm_of_map.data()))) return rc;
        P.alm_tab = (const double2 *const *)d;
        if ((rc = balloc(b->sched_allocs, &d, sizeof(void *) * G.nmaps, G.map_of_map.data()))) return rc;
        P.map_tab = (double *const *)d;
        const double per_map = 4.0 * (double)(bf.n_dense + bf.n_r) + 2.0 * (double)bf.n_ident +
                               p->stats.phi_flops_per_map;
        for (int b0 = 0; b0 < G.nmaps;) {
            const int left = G.nmaps - b0;
            int nb = 1;
            while (nb * 2 <= std::min(left, width)) nb *= 2;
            shtb_batch_s::GMapGroup M{};
            M.b0 = b0;
            M.nb = nb;
            M.cost = per_map * nb;
            const size_t entry = sizeof(double) * 2 * nb;
            if ((rc = balloc(b->sched_allocs, &d, entry * (size_t)bf.u_entries))) return rc;
            M.u0 = (double *)d;
            if ((rc = balloc(b->sched_allocs, &d, entry * (size_t)bf.u_entries))) return rc;
            M.u1 = (double *)d;
            if ((rc = balloc(b->sched_allocs, &d, entry * (size_t)bf.qt_entries))) return rc;
            M.qt = (double *)d;
            order.push_back({M.cost, {(int)g, (int)P.mgs.size()}});
            P.mgs.push_back(M);
            b0 += nb;
        }
        b->gg.push_back(std::move(P));
    }
    // longest processing time first onto the least loaded stream
    std::sort(order.begin(), order.end(), [](const auto &a, const auto &c) { return a.first > c.first; });
    std::vector<double> load(nstreams, 0.0);
    for (auto &o : order) {
        const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[s] += o.first;
        b->gg[o.second.first].mgs[o.second.second].stream = s;
    }
    while ((int)b->side.size() < nstreams - 1) {
        cudaStream_t s2;
        SHTB_CUDA_TRY(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
        b->side.push_back(s2);
    }
    while ((int)b->fork_join.size() < nstreams) {
        cudaEvent_t e;
        SHTB_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->fork_join.push_back(e);
    }
    b->warps = 0;
    b->grid = 0;
    return SHTB_OK;
}

int enqueue_graph(shtb_batch_s *b, cudaStream_t st)
{
    int rc;
    for (auto &P : b->gg)
        if ((rc = launch_bf_gather(P.plan, P.alm_tab, P.ai, P.nmaps, st))) return rc;
    // fork: every side stream starts after the gathers
    SHTB_CUDA_TRY(cudaEventRecord(b->fork_join[0], st));
    for (int s = 1; s < b->nstreams; ++s) SHTB_CUDA_TRY(cudaStreamWaitEvent(b->side[s - 1], b->fork_join[0], 0));
    for (auto &P : b->gg) {
        for (auto &M : P.mgs) {
            cudaStream_t ss = M.stream == 0 ? st : b->side[M.stream - 1];
            if ((rc = launch_bf_legendre_group(P.plan, P.ai, P.nmaps, M.b0, M.nb, M.u0, M.u1, M.qt, ss)))
                return rc;
            if ((rc = launch_phi_synth_qt_ptr(P.plan, M.qt, M.nb, P.map_tab, M.b0, ss))) return rc;
        }
    }
    // join
    for (int s = 1; s < b->nstreams; ++s) {
        SHTB_CUDA_TRY(cudaEventRecord(b->fork_join[s], b->side[s - 1]));
        SHTB_CUDA_TRY(cudaStreamWaitEvent(st, b->fork_join[s], 0));
    }
    return SHTB_OK;
}

int enqueue(shtb_batch_s *b, cudaStream_t st)
{
    if (b->mode == 1) return enqueue_graph(b, st);
    SHTB_CUDA_TRY(cudaMemsetAsync(b->dev.counters, 0, sizeof(int) * (b->ncounters + 2), st));
    batch_kernel<<<b->grid, 32 * b->warps, b->smem, st>>>(b->dev);
    SHTB_CUDA_TRY(cudaGetLastError());
    return SHTB_OK;
}

int read_status(shtb_batch_s *b, cudaStream_t st)
{
    int err = 0;
    if (b->mode == 0)
        SHTB_CUDA_TRY(cudaMemcpyAsync(&err, b->dev.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SHTB_CUDA_TRY(cudaStreamSynchronize(st));
    SHTB_CUDA_TRY(cudaGetLastError());
    if (err) return shtb_fail(SHTB_ETIMEOUT, "batch kernel: a stage wait gave up (error flag set)");
    return SHTB_OK;
}

double time_schedule(shtb_batch_s *b, cudaStream_t st, int reps)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    enqueue(b, st);                      // warm-up
    cudaEventRecord(e0, st);
    for (int i = 0; i < reps; ++i) enqueue(b, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (read_status(b, st) != SHTB_OK) return 1e30;
    return ms / reps;
}

}  // namespace

extern "C" {

int shtb_batch_opts_init(shtb_batch_opts *o)
{
    if (!o) return shtb_fail(SHTB_EINVAL, "opts is NULL");
    o->autotune = 1;
    o->warps_per_block = 0;
    o->group_width = 8;
    o->lpt = 1;
    o->spin_limit = 0;
    o->schedule = 0;
    o->streams = 0;
    return SHTB_OK;
}

int shtb_batch_create(const shtb_request *reqs, int nreq, const shtb_batch_opts *opts, shtb_batch *out)
{
    if (!out) return shtb_fail(SHTB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!reqs || nreq < 1) return shtb_fail(SHTB_EINVAL, "no requests");
    int dev = -1;
    SHTB_CUDA_TRY(cudaGetDevice(&dev));
    std::map<shtb_plan_s *, int> gid;
    auto *b = new shtb_batch_s();
    b->device = dev;
    shtb_batch_opts_init(&b->opts);
    if (opts) b->opts = *opts;
    for (int i = 0; i < nreq; ++i) {
        const shtb_request &r = reqs[i];
        if (!r.plan || !r.alm_dev || !r.map_dev || r.nmaps < 1 || ((uintptr_t)r.alm_dev & 15) ||
            ((uintptr_t)r.map_dev & 15)) {
            delete b;
            return shtb_fail(SHTB_EINVAL, "request " + std::to_string(i) + " is invalid");
        }
        if (r.dir != 0) {
            delete b;
            return shtb_fail(SHTB_ENOTSUP, "batches serve synthesis requests (dir = 0) only");
        }
        if (!r.plan->bf || r.plan->kind != 0) {
            delete b;
            return shtb_fail(SHTB_ENOTSUP, "batches need compressed scalar plans (eps > 0)");
        }
        if (r.plan->bf->rec) {
            delete b;
            return shtb_fail(SHTB_ENOTSUP, "batches need plans that store their residual blocks");
        }
        if (r.plan->device != dev) {
            delete b;
            return shtb_fail(SHTB_EMISMATCH, "request " + std::to_string(i) + " uses a plan of another device");
        }
        b->reqs.push_back(r);
        auto it = gid.find(r.plan);
        if (it == gid.end()) {
            gid[r.plan] = (int)b->groups.size();
            b->groups.push_back({});
            b->groups.back().plan = r.plan;
            it = gid.find(r.plan);
        }
        auto &G = b->groups[it->second];
        for (int k = 0; k < r.nmaps; ++k) {
            G.alm_of_map.push_back((const double2 *)r.alm_dev + (size_t)k * r.plan->nalm);
            G.map_of_map.push_back(r.map_dev + (size_t)k * r.plan->npix);
        }
        G.nmaps += r.nmaps;
    }
    int rc;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return shtb_fail(SHTB_ECUDA, "stream creation failed");
    }
    b->own_stream = st;
    const int w0 = b->opts.warps_per_block > 0 ? b->opts.warps_per_block : 4;
    const int gw = b->opts.group_width > 0 ? b->opts.group_width : 8;
    if (b->opts.autotune) {
        // autotuner, timed on this batch: the persistent kernel (warps per
        // block x work order) and the stage-kernel graph (streams)
        double best = 1e30;
        int bw = w0, bl = b->opts.lpt, bs = 0, bn = 1;
        for (int warps : {4, 8}) {
            for (int lpt : {1, 0}) {
                if ((rc = build_schedule(b, warps, gw, lpt))) { shtb_batch_destroy(b); return rc; }
                const double ms = time_schedule(b, st, 2);
                if (ms < best) { best = ms; bw = warps; bl = lpt; bs = 0; }
            }
        }
        for (int ns : {1, 2, 4, 8}) {
            if ((rc = build_graph_schedule(b, gw, ns))) { shtb_batch_destroy(b); return rc; }
            const double ms = time_schedule(b, st, 2);
            if (ms < best) { best = ms; bs = 1; bn = ns; }
        }
        b->opts.warps_per_block = bw;
        b->opts.lpt = bl;
        b->opts.schedule = bs;
        b->opts.streams = bn;
        b->tuned_ms = best;
    }
    if (b->opts.schedule == 1)
        rc = build_graph_schedule(b, gw, b->opts.streams > 0 ? b->opts.streams : 4);
    else
        rc = build_schedule(b, b->opts.warps_per_block > 0 ? b->opts.warps_per_block : w0, gw, b->opts.lpt);
    if (rc) {
        shtb_batch_destroy(b);
        return rc;
    }
    *out = b;
    return SHTB_OK;
}

int shtb_batch_run(shtb_batch b, void *stream)
{
    NvtxRange nvtx("shtb_batch_run");
    if (!b) return shtb_fail(SHTB_EINVAL, "batch is NULL");
    int dev = -1;
    SHTB_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != b->device) return shtb_fail(SHTB_EMISMATCH, "batch used on another device");
    cudaStream_t st = stream ? (cudaStream_t)stream : b->own_stream;
    if (!b->exec) {
        cudaGraph_t graph;
        SHTB_CUDA_TRY(cudaStreamBeginCapture(b->own_stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue(b, b->own_stream);
        cudaError_t e = cudaStreamEndCapture(b->own_stream, &graph);
        if (rc) return rc;
        if (e != cudaSuccess) return shtb_fail(SHTB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return shtb_fail(SHTB_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    SHTB_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    if (!stream) SHTB_CUDA_TRY(cudaStreamSynchronize(st));
    return SHTB_OK;
}

int shtb_batch_status(shtb_batch b, void *stream)
{
    if (!b) return shtb_fail(SHTB_EINVAL, "batch is NULL");
    return read_status(b, stream ? (cudaStream_t)stream : b->own_stream);
}

int shtb_batch_info(shtb_batch b, int *warps_per_block, int *grid, int *npacks, double *tuned_ms)
{
    if (!b) return shtb_fail(SHTB_EINVAL, "batch is NULL");
    if (warps_per_block) *warps_per_block = b->warps;
    if (grid) *grid = b->grid;
    if (npacks) *npacks = b->dev.npacks;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    return SHTB_OK;
}

int shtb_batch_schedule(shtb_batch b, int *schedule, int *streams)
{
    if (!b) return shtb_fail(SHTB_EINVAL, "batch is NULL");
    if (schedule) *schedule = b->mode;
    if (streams) *streams = b->mode == 1 ? b->nstreams : 0;
    return SHTB_OK;
}

int shtb_test_batch_stall(shtb_batch b, int on)
{
    if (b && b->mode != 0) return shtb_fail(SHTB_ENOTSUP, "stage waits exist in the persistent schedule only");
    if (!b || b->ncounters < 2 || b->stall_counter < 0) return shtb_fail(SHTB_EINVAL, "batch is NULL or empty");
    // every pack waiting on the first plan group's gather waits for one item
    // more than that gather has, so its wait runs out (on) or not (off)
    std::vector<BatchPack> packs(b->host_packs.size() / sizeof(BatchPack));
    memcpy(packs.data(), b->host_packs.data(), b->host_packs.size());
    for (auto &P : packs)
        if (P.dep == b->stall_counter) P.need += on ? 1 : 0;
    SHTB_CUDA_TRY(cudaMemcpy((void *)b->dev.packs, packs.data(), sizeof(BatchPack) * packs.size(),
                             cudaMemcpyHostToDevice));
    return SHTB_OK;
}

int shtb_batch_destroy(shtb_batch b)
{
    if (!b) return SHTB_OK;
    free_schedule(b);
    for (void *p : b->allocs) cudaFree(p);
    for (cudaStream_t s2 : b->side) cudaStreamDestroy(s2);
    for (cudaEvent_t e : b->fork_join) cudaEventDestroy(e);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
    return SHTB_OK;
}

}  // extern "C"
