// Batched serving: many synthesis requests of different (Nside, L, eps) in
// ONE persistent kernel launch, captured in a CUDA graph on the first run --
// or, where the autotuner finds it faster, a CUDA graph of the stand-alone
// stage kernels over the merged map groups on several streams.
//
// Requests that share a plan are merged along the map axis, so every stored
// element of that plan's compressed operator is read once per group of up to
// 8 maps (the paper's remark that many simultaneous transforms amortise the
// precomputed data, Sec. 3.3).  The work of the whole batch is one list of
// items in dependency order -- a_lm gather, residual blocks, each butterfly
// level from the top down, parity combine, per-ring FFT -- grouped into packs
// (a warp per item for the butterfly stages, a block per ring for the FFT).
// Resident blocks claim packs in list order from a global counter; a pack of
// stage s first waits until every item of stage s-1 is done.  Packs are
// claimed in order and a claimed pack never waits on a later stage, so the
// wait always ends; it is still bounded (spin_limit polls), after which the
// kernel sets an error flag and returns, and the host reports SHTB_ETIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "shtb_batch_items.cuh"
#include "shtb_butterfly.h"
#include "shtb_internal.h"

namespace {

enum WorkType { W_GATHER = 0, W_RES = 1, W_LEVEL = 2, W_COMBINE = 3, W_PHI = 4 };

struct BatchWork {
    int type;
    int g;        // plan group
    int mg;       // map group (butterfly stages) or map (ring stage)
    int idx;      // m, residual item, level item or ring
    int level;
};

struct BatchPack {
    int stage, first, count, block;   // block = 1: one item for the whole block
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
    double2 *q;                       // [nmaps][nrings][L+1]
    int nmaps;
    const double2 *const *alm_of_map; // request a_lm of each merged map
    double *const *map_of_map;        // request output map of each merged map
};

struct BatchDev {
    const BatchWork *work;
    const BatchPack *packs;
    int npacks;
    const BatchGroupDev *groups;
    const BatchMG *mgs;               // flat, mg index = group's mg_base + local
    const int *mg_base;
    const int *stage_total;
    int *done;
    int *next;
    int *err;
    long long spin_limit;
};

template <int NB>
__device__ void warp_item(const BatchDev &bd, const BatchWork &w, double *wsm, int lane)
{
    const BatchGroupDev &G = bd.groups[w.g];
    const BatchMG &M = bd.mgs[bd.mg_base[w.g] + w.mg];
    switch (w.type) {
    case W_RES: {
        const BfRItem it = G.ritems[w.idx];
        double *ubuf = G.depth_parity[it.m * 2 + it.t] ? M.u1 : M.u0;
        shtb_bdev::bf_r_item<NB, true>(it, G.v.lmax, G.ints, G.dbl, G.ai, G.nmaps, M.b0, ubuf, M.qt, lane);
        break;
    }
    case W_LEVEL: {
        const double *uin = (w.level % 2) ? M.u1 : M.u0;
        double *uout = ((w.level - 1) % 2) ? M.u1 : M.u0;
        shtb_bdev::bf_level_item<NB, true>(G.litems[w.level - 1][w.idx], G.ints, G.dbl, uin, uout, M.qt,
                                          wsm, lane);
        break;
    }
    case W_COMBINE: {
        const size_t per_map = (size_t)G.v.nrings * (G.v.lmax + 1);
        shtb_bdev::bf_combine_m<NB, true>(w.idx, G.v.lmax, G.v.nhalf, G.v.nrings, M.qt,
                                         [&](int b) { return G.q + (size_t)(M.b0 + b) * per_map; }, lane,
                                         32);
        break;
    }
    default:
        break;
    }
}

// a_lm of the merged maps into ai[idx][map] (Im a_l0 = 0), one order m
__device__ void gather_item(const BatchDev &bd, const BatchWork &w, int lane)
{
    const BatchGroupDev &G = bd.groups[w.g];
    const int m = w.idx, L = G.v.lmax;
    const long long off = shtb_bdev::alm_off(L, m);
    const int n = L - m + 1;
    for (int i = lane; i < n * G.nmaps; i += 32) {
        const int b = i / n, dl = i - b * n;
        const long long idx = off + dl;
        const double2 a = G.alm_of_map[b][idx];
        G.ai[(size_t)idx * G.nmaps + b] = make_double2(a.x, m == 0 ? 0.0 : a.y);
    }
}

__global__ void __launch_bounds__(256) batch_kernel(BatchDev bd)
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
        if (P.stage > 0 && threadIdx.x == 0) {
            long long polls = 0;
            while (atomicAdd(&bd.done[P.stage - 1], 0) < bd.stage_total[P.stage - 1]) {
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
            const BatchWork w = bd.work[P.first];
            const BatchGroupDev &G = bd.groups[w.g];
            const int ring = w.idx, b = w.mg;
            const double2 *qr = G.q + ((size_t)b * G.v.nrings + ring) * (G.v.lmax + 1);
            double *out = G.map_of_map[b] + G.v.ring_start[ring];
            if (G.v.ring_M[ring] > 0)
                shtb_bdev::phi_synth_ring<true, true>(G.v, ring, qr, out, reinterpret_cast<double2 *>(bsm));
            else
                shtb_bdev::phi_synth_ring<false, true>(G.v, ring, qr, out, reinterpret_cast<double2 *>(bsm));
        } else if (wib < P.count) {
            const BatchWork w = bd.work[P.first + wib];
            if (w.type == W_GATHER) {
                gather_item(bd, w, lane);
            } else {
                const BatchMG &M = bd.mgs[bd.mg_base[w.g] + w.mg];
                double *wsm = bsm + (size_t)wib * shtb::kMaxCand * 16;
                switch (M.nb) {
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
            atomicAdd(&bd.done[P.stage], P.count);
        }
    }
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

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
    int nstages = 0, warps = 4, grid = 0;
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
    b->nstages = 0;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
}

// Builds the work list, packs and device tables for `warps` warps per block
// and map groups of at most `width` maps; work inside a stage in decreasing
// size (lpt = 1) or in plan order (lpt = 0).
int build_schedule(shtb_batch_s *b, int warps, int width, int lpt)
{
    free_schedule(b);
    b->mode = 0;
    std::vector<BatchGroupDev> gdev(b->groups.size());
    std::vector<BatchMG> mgs;
    std::vector<int> mg_base(b->groups.size());
    std::vector<std::vector<BatchWork>> stages;
    int dmax = 0;
    for (auto &G : b->groups) dmax = std::max(dmax, G.plan->bf->depth_max);
    const int S_GATHER = 0, S_RES = 1, S_COMB = 2 + dmax, S_PHI = 3 + dmax;
    stages.resize(S_PHI + 1);
    std::vector<std::vector<long long>> cost(stages.size());
    size_t smem_fft = 0;
    int rc;
    for (size_t g = 0; g < b->groups.size(); ++g) {
        auto &G = b->groups[g];
        shtb_plan_s *p = G.plan;
        const BfPlanDev &bf = *p->bf;
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
        if ((rc = balloc(b->sched_allocs, &d, sizeof(double2) * (size_t)G.nmaps * p->nrings * (p->lmax + 1))))
            return rc;
        D.q = (double2 *)d;
        if ((rc = balloc(b->sched_allocs, &d, sizeof(void *) * G.nmaps, G.alm_of_map.data()))) return rc;
        D.alm_of_map = (const double2 *const *)d;
        if ((rc = balloc(b->sched_allocs, &d, sizeof(void *) * G.nmaps, G.map_of_map.data()))) return rc;
        D.map_of_map = (double *const *)d;
        // map groups of power-of-two widths up to `width`
        mg_base[g] = (int)mgs.size();
        for (int b0 = 0; b0 < G.nmaps;) {
            const int left = G.nmaps - b0;
            int nb = 1;
            while (nb * 2 <= std::min(left, width)) nb *= 2;
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
            mgs.push_back(M);
            b0 += nb;
        }
        const int nmg2 = (int)mgs.size() - mg_base[g];
        // ---- work
        for (int m = 0; m <= p->lmax; ++m) {
            stages[S_GATHER].push_back({W_GATHER, (int)g, 0, m, 0});
            cost[S_GATHER].push_back((long long)(p->lmax - m + 1) * G.nmaps);
        }
        std::vector<BfRItem> rh(bf.n_ritems);
        cudaMemcpy(rh.data(), bf.ritems, sizeof(BfRItem) * bf.n_ritems, cudaMemcpyDeviceToHost);
        for (int mg = 0; mg < nmg2; ++mg) {
            const int nb = mgs[mg_base[g] + mg].nb;
            for (int i = 0; i < bf.n_ritems; ++i) {
                stages[S_RES].push_back({W_RES, (int)g, mg, i, 0});
                cost[S_RES].push_back((long long)rh[i].nrows * rh[i].k * nb);
            }
            for (int l = bf.depth_max; l >= 1; --l) {
                const int st = 2 + (dmax - l);
                std::vector<BfItem> lh(bf.level_counts[l - 1]);
                cudaMemcpy(lh.data(), bf.level_items[l - 1], sizeof(BfItem) * lh.size(), cudaMemcpyDeviceToHost);
                for (size_t i = 0; i < lh.size(); ++i) {
                    stages[st].push_back({W_LEVEL, (int)g, mg, (int)i, l});
                    cost[st].push_back(((long long)lh[i].k[0] * lh[i].nd[0] + (long long)lh[i].k[1] * lh[i].nd[1] +
                                        lh[i].nc) * nb);
                }
            }
            for (int m = 0; m <= p->lmax; ++m) {
                stages[S_COMB].push_back({W_COMBINE, (int)g, mg, m, 0});
                cost[S_COMB].push_back((long long)p->nhalf * nb);
            }
        }
        for (int mp = 0; mp < G.nmaps; ++mp)
            for (int r = 0; r < p->nrings; ++r) {
                stages[S_PHI].push_back({W_PHI, (int)g, mp, r, 0});
                const long long K = p->ring_J[r] / 2, M = p->ring_M[r];
                cost[S_PHI].push_back(M > 0 ? 3 * M : K);
            }
        smem_fft = std::max(smem_fft, sizeof(double2) * (size_t)std::max(p->max_K_pow2, p->max_M_blue));
    }
    // ---- order, packs
    std::vector<BatchWork> work;
    std::vector<BatchPack> packs;
    std::vector<int> totals(stages.size(), 0);
    for (size_t s = 0; s < stages.size(); ++s) {
        std::vector<int> ord(stages[s].size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
        if (lpt) std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return cost[s][a] > cost[s][c]; });
        const int first = (int)work.size();
        for (int i : ord) work.push_back(stages[s][i]);
        totals[s] = (int)ord.size();
        const bool block = (int)s == S_PHI;
        const int per = block ? 1 : warps;
        for (int i = 0; i < (int)ord.size(); i += per)
            packs.push_back({(int)s, first + i, std::min(per, (int)ord.size() - i), block ? 1 : 0});
    }
    void *d;
    if ((rc = balloc(b->sched_allocs, &d, sizeof(BatchWork) * work.size(), work.data()))) return rc;
    b->dev.work = (const BatchWork *)d;
    if ((rc = balloc(b->sched_allocs, &d, sizeof(BatchPack) * packs.size(), packs.data()))) return rc;
    b->dev.packs = (const BatchPack *)d;
    b->dev.npacks = (int)packs.size();
    if ((rc = balloc(b->sched_allocs, &d, sizeof(BatchGroupDev) * gdev.size(), gdev.data()))) return rc;
    b->dev.groups = (const BatchGroupDev *)d;
    if ((rc = balloc(b->sched_allocs, &d, sizeof(BatchMG) * mgs.size(), mgs.data()))) return rc;
    b->dev.mgs = (const BatchMG *)d;
    if ((rc = balloc(b->sched_allocs, &d, sizeof(int) * mg_base.size(), mg_base.data()))) return rc;
    b->dev.mg_base = (const int *)d;
    if ((rc = balloc(b->sched_allocs, &d, sizeof(int) * totals.size(), totals.data()))) return rc;
    b->dev.stage_total = (const int *)d;
    if ((rc = balloc(b->sched_allocs, &d, sizeof(int) * (totals.size() + 2)))) return rc;
    b->dev.done = (int *)d;
    b->dev.next = b->dev.done + totals.size();
    b->dev.err = b->dev.done + totals.size() + 1;
    b->dev.spin_limit = b->opts.spin_limit > 0 ? b->opts.spin_limit : 20000000LL;
    b->nstages = (int)totals.size();
    b->warps = warps;
    b->smem = std::max(smem_fft, sizeof(double) * (size_t)warps * shtb::kMaxCand * 16);
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
    SHTB_CUDA_TRY(cudaMemsetAsync(b->dev.done, 0, sizeof(int) * (b->nstages + 2), st));
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
    if (!b || b->nstages < 2) return shtb_fail(SHTB_EINVAL, "batch is NULL or empty");
    int t0 = 0;
    SHTB_CUDA_TRY(cudaMemcpy(&t0, b->dev.stage_total, sizeof(int), cudaMemcpyDeviceToHost));
    // one more item than stage 0 has: every later stage waits until its bound runs out
    const int want = on ? t0 + 1 : t0 - 1;
    if ((on && t0 < 0) || (!on && t0 < 1)) return shtb_fail(SHTB_EINVAL, "stall state");
    SHTB_CUDA_TRY(cudaMemcpy((void *)b->dev.stage_total, &want, sizeof(int), cudaMemcpyHostToDevice));
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
