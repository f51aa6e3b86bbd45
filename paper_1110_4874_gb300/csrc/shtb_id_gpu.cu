// Batched interpolative decompositions for the plan builder on the GPU
// (Sec. 3.1, Eq. ID; the ID of Cheng, Gimbutas, Martinsson & Rokhlin 2005).
// Each CTA takes one block A (rows x nc, column-major) and runs the same
// algorithm as the host routine interp_decomp:
//   columns with norm <= abs_floor are zero columns and take no part;
//   column-pivoted Householder QR over the others, stopping once the largest
//   remaining column norm is <= max(eps |R_00|, abs_floor); norms are
//   downdated and recomputed exactly when they lose 8 digits;
//   X = R_11^{-1} R_12 by back substitution, one dense column per warp.
// Pivoting swaps column indices, not data.  The block is transformed in
// place in global memory (it stays in L2 while its CTA works on it); the
// Householder vector lives in shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "shtb_id_gpu.h"
#include "shtb_internal.h"

namespace {

constexpr int kIdThreads = 256;
constexpr int kIdWarps = kIdThreads / 32;

struct IdDesc {
    long long off;      // block data (element offset)
    long long x_off;    // output X (element offset), room for kMaxCand^2 / 4 + kMaxCand
    int rows, nc;
    int col_off;        // output column order (int offset), nc slots
    int pad;
};

__device__ __forceinline__ double warp_sum(double s)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// sum over threads of the block (every thread gets the result)
__device__ double block_sum(double s, double *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    s = warp_sum(s);
    __syncthreads();
    if (lane == 0) red[w] = s;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < kIdWarps; ++i) t += red[i];
    return t;
}

__global__ void __launch_bounds__(kIdThreads)
id_kernel(double *__restrict__ data, const IdDesc *__restrict__ descs, double eps, double abs_floor,
          int *__restrict__ out_k, int *__restrict__ out_nzc, int *__restrict__ out_col, double *__restrict__ out_x)
{
    extern __shared__ double v[];                       // Householder vector, rows entries
    __shared__ double norms[shtb::kMaxCand], ref[shtb::kMaxCand], red[kIdWarps];
    __shared__ int col[shtb::kMaxCand];
    __shared__ int s_nzc, s_p, s_stop;
    __shared__ double s_r00, s_alpha, s_beta;
    const IdDesc d = descs[blockIdx.x];
    double *A = data + d.off;
    const int rows = d.rows, nc = d.nc;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;

    // column norms; nonzero columns in their original order
    for (int c = w; c < nc; c += kIdWarps) {
        double s = 0.0;
        for (int r = lane; r < rows; r += 32) s += A[(size_t)c * rows + r] * A[(size_t)c * rows + r];
        s = warp_sum(s);
        if (lane == 0) norms[c] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int n = 0;
        for (int c = 0; c < nc; ++c)
            if (sqrt(norms[c]) > abs_floor) {
                ref[n] = norms[c];
                col[n++] = c;
            }
        for (int j = 0; j < n; ++j) norms[j] = ref[j];
        s_nzc = n;
    }
    __syncthreads();
    const int nzc = s_nzc;
    const int kmax = rows == 0 ? 0 : min(rows, nzc);
    int k = 0;
    for (int i = 0; i < kmax; ++i) {
        if (threadIdx.x == 0) {
            int p = i;
            for (int j = i + 1; j < nzc; ++j)
                if (norms[j] > norms[p]) p = j;
            s_p = p;
        }
        __syncthreads();
        const int p = s_p;
        const double *cp = A + (size_t)col[p] * rows;
        double s = 0.0;
        for (int r = i + threadIdx.x; r < rows; r += kIdThreads) s += cp[r] * cp[r];
        const double n2 = block_sum(s, red);
        if (threadIdx.x == 0) {
            norms[p] = n2;
            const double nrm = sqrt(n2);
            if (i == 0) s_r00 = nrm;
            s_stop = nrm <= fmax(eps * s_r00, abs_floor);
            if (!s_stop) {
                if (p != i) {
                    const double tn = norms[p]; norms[p] = norms[i]; norms[i] = tn;
                    const double tr = ref[p]; ref[p] = ref[i]; ref[i] = tr;
                    const int tc = col[p]; col[p] = col[i]; col[i] = tc;
                }
                const double x0 = A[(size_t)col[i] * rows + i];
                s_alpha = x0 >= 0 ? -nrm : nrm;
                const double vn2 = 2.0 * nrm * (nrm + fabs(x0));
                s_beta = vn2 > 0 ? 2.0 / vn2 : 0.0;
            }
        }
        __syncthreads();
        if (s_stop) break;
        double *ci = A + (size_t)col[i] * rows;
        for (int r = i + threadIdx.x; r < rows; r += kIdThreads) v[r] = ci[r] - (r == i ? s_alpha : 0.0);
        __syncthreads();
        const double beta = s_beta;
        for (int j = i + 1 + w; j < nzc; j += kIdWarps) {
            double *cj = A + (size_t)col[j] * rows;
            double t = 0.0;
            for (int r = i + lane; r < rows; r += 32) t += v[r] * cj[r];
            t = warp_sum(t) * beta;
            for (int r = i + lane; r < rows; r += 32) cj[r] -= t * v[r];
            __syncwarp();
            double nj = 0.0;
            int redo = 0;
            if (lane == 0) {
                nj = norms[j] - cj[i] * cj[i];
                redo = nj <= 1e-8 * ref[j];
            }
            redo = __shfl_sync(0xffffffffu, redo, 0);
            if (redo) {
                double e = 0.0;
                for (int r = i + 1 + lane; r < rows; r += 32) e += cj[r] * cj[r];
                e = warp_sum(e);
                if (lane == 0) ref[j] = norms[j] = e;
            } else if (lane == 0) {
                norms[j] = nj;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) ci[i] = s_alpha;
        k = i + 1;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out_k[blockIdx.x] = k;
        out_nzc[blockIdx.x] = nzc;
    }
    for (int j = threadIdx.x; j < nzc; j += kIdThreads) out_col[d.col_off + j] = col[j];
    // X = R_11^{-1} R_12: dense column c = k + q, rows 0..k-1 of the transformed block
    double *X = out_x + d.x_off;
    for (int q = w; q < nzc - k; q += kIdWarps) {
        const double *cc = A + (size_t)col[k + q] * rows;
        double *x = X + (size_t)q * k;
        for (int i = k - 1; i >= 0; --i) {
            double t = 0.0;
            for (int qq = i + 1 + lane; qq < k; qq += 32) t += A[(size_t)col[qq] * rows + i] * x[qq];
            t = warp_sum(t);
            if (lane == 0) x[i] = (cc[i] - t) / A[(size_t)col[i] * rows + i];
            __syncwarp();
        }
    }
}

}  // namespace

namespace shtb {

struct GpuIdSlot {
    cudaStream_t st = nullptr;
    double *h_data = nullptr, *d_data = nullptr, *h_x = nullptr, *d_x = nullptr;
    IdDesc *h_desc = nullptr, *d_desc = nullptr;
    int *h_int = nullptr, *d_int = nullptr;
    long long cap_data = 0, cap_x = 0;
    int cap_blocks = 0, cap_int = 0;
};

class GpuIdPool {
public:
    int device = 0;
    std::vector<GpuIdSlot> slots;
};

namespace {

void release(GpuIdSlot &s)
{
    if (s.st) cudaStreamSynchronize(s.st);
    cudaFreeHost(s.h_data);
    cudaFree(s.d_data);
    cudaFreeHost(s.h_x);
    cudaFree(s.d_x);
    cudaFreeHost(s.h_desc);
    cudaFree(s.d_desc);
    cudaFreeHost(s.h_int);
    cudaFree(s.d_int);
    if (s.st) cudaStreamDestroy(s.st);
    s = GpuIdSlot{};
}

template <class T>
bool grow(T *&h, T *&d, long long &cap, long long need)
{
    if (need <= cap) return true;
    cudaFreeHost(h);
    cudaFree(d);
    h = nullptr;
    d = nullptr;
    cap = 0;
    const long long n = std::max(need, 2 * cap + 1024);
    if (cudaMallocHost((void **)&h, sizeof(T) * n) != cudaSuccess) return false;
    if (cudaMalloc((void **)&d, sizeof(T) * n) != cudaSuccess) return false;
    cap = n;
    return true;
}

}  // namespace

GpuIdPool *gpu_id_pool_create(int device, int nthreads)
{
    auto *pool = new (std::nothrow) GpuIdPool();
    if (!pool) return nullptr;
    pool->device = device;
    pool->slots.resize(std::max(1, nthreads));
    return pool;
}

void gpu_id_pool_destroy(GpuIdPool *pool)
{
    if (!pool) return;
    cudaSetDevice(pool->device);
    for (auto &s : pool->slots) release(s);
    delete pool;
}

double *gpu_id_staging(GpuIdPool *pool, int slot, long long nelem)
{
    if (cudaSetDevice(pool->device) != cudaSuccess) return nullptr;
    GpuIdSlot &s = pool->slots[slot];
    if (!grow(s.h_data, s.d_data, s.cap_data, std::max(1LL, nelem))) return nullptr;
    return s.h_data;
}

int gpu_id_run(GpuIdPool *pool, int slot, const double *data, long long nelem, const std::vector<IdBlock> &blocks,
               double eps, double abs_floor, std::vector<IdResult> &out)
{
    const int nb = (int)blocks.size();
    out.assign(nb, IdResult{});
    if (nb == 0) return SHTB_OK;
    if (cudaSetDevice(pool->device) != cudaSuccess) return shtb_fail(SHTB_ECUDA, "plan build: cudaSetDevice");
    GpuIdSlot &s = pool->slots[slot];
    if (!s.st && cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess)
        return shtb_fail(SHTB_ECUDA, "plan build: stream");
    // descriptors and output layout
    constexpr int kXPer = kMaxCand * kMaxCand / 4 + kMaxCand;   // k (nzc - k) <= nzc^2 / 4
    long long cap_b = s.cap_blocks, cap_i = s.cap_int;
    if (!grow(s.h_desc, s.d_desc, cap_b, nb)) return shtb_fail(SHTB_ENOMEM, "plan build: id descriptors");
    s.cap_blocks = (int)cap_b;
    long long nint = 2LL * nb;
    for (const auto &b : blocks) nint += b.nc;
    if (!grow(s.h_int, s.d_int, cap_i, nint)) return shtb_fail(SHTB_ENOMEM, "plan build: id outputs");
    s.cap_int = (int)cap_i;
    if (data != s.h_data && !grow(s.h_data, s.d_data, s.cap_data, std::max(1LL, nelem)))
        return shtb_fail(SHTB_ENOMEM, "plan build: id data");
    if (!grow(s.h_x, s.d_x, s.cap_x, (long long)nb * kXPer)) return shtb_fail(SHTB_ENOMEM, "plan build: id X");
    int col_off = 2 * nb, max_rows = 1;
    for (int i = 0; i < nb; ++i) {
        const IdBlock &b = blocks[i];
        if (b.nc > kMaxCand || b.nc < 0 || b.rows < 0 || b.off < 0 || b.off + (long long)b.rows * b.nc > nelem)
            return shtb_fail(SHTB_EINVAL, "plan build: bad id block");
        s.h_desc[i] = IdDesc{b.off, (long long)i * kXPer, b.rows, b.nc, col_off, 0};
        col_off += b.nc;
        max_rows = std::max(max_rows, b.rows);
    }
    const size_t smem = sizeof(double) * (size_t)max_rows;
    if (smem > 160 * 1024) return shtb_fail(SHTB_ENOTSUP, "plan build: id block too tall for the GPU builder");
    if (data != s.h_data) std::copy(data, data + nelem, s.h_data);
    SHTB_CUDA_TRY(cudaMemcpyAsync(s.d_data, s.h_data, sizeof(double) * nelem, cudaMemcpyHostToDevice, s.st));
    SHTB_CUDA_TRY(cudaMemcpyAsync(s.d_desc, s.h_desc, sizeof(IdDesc) * nb, cudaMemcpyHostToDevice, s.st));
    if (smem > 48 * 1024)
        SHTB_CUDA_TRY(cudaFuncSetAttribute(id_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    id_kernel<<<nb, kIdThreads, smem, s.st>>>(s.d_data, s.d_desc, eps, abs_floor, s.d_int, s.d_int + nb,
                                              s.d_int, s.d_x);
    SHTB_CUDA_TRY(cudaGetLastError());
    SHTB_CUDA_TRY(cudaMemcpyAsync(s.h_int, s.d_int, sizeof(int) * nint, cudaMemcpyDeviceToHost, s.st));
    SHTB_CUDA_TRY(cudaMemcpyAsync(s.h_x, s.d_x, sizeof(double) * (size_t)nb * kXPer, cudaMemcpyDeviceToHost, s.st));
    SHTB_CUDA_TRY(cudaStreamSynchronize(s.st));
    // results in the host routine's form
    for (int i = 0; i < nb; ++i) {
        const IdBlock &b = blocks[i];
        IdResult &res = out[i];
        const int k = s.h_int[i], nzc = s.h_int[nb + i];
        const int *cols = s.h_int + s.h_desc[i].col_off;
        const double *X = s.h_x + s.h_desc[i].x_off;
        res.k = k;
        res.kind.assign(b.nc, kZeroCol);
        res.skel.assign(cols, cols + k);
        for (int q = 0; q < k; ++q) res.kind[cols[q]] = q;
        const int nd = nzc - k;
        std::vector<std::pair<int, int>> dense;      // (block column, X column)
        for (int q = 0; q < nd; ++q) dense.push_back({cols[k + q], q});
        std::sort(dense.begin(), dense.end());
        res.dense_pos.resize(nd);
        res.T.assign((size_t)k * nd, 0.0);
        for (int dd = 0; dd < nd; ++dd) {
            res.dense_pos[dd] = dense[dd].first;
            res.kind[dense[dd].first] = -1 - dd;
            const double *x = X + (size_t)dense[dd].second * k;
            for (int q = 0; q < k; ++q) res.T[(size_t)q * nd + dd] = x[q];
        }
    }
    return SHTB_OK;
}

}  // namespace shtb
