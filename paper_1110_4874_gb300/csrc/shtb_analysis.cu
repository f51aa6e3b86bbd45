// Spherical-harmonic analysis by ring quadrature (Eq. sh-forward-quadrature):
// a_lm = sum_p w_p f_p conj(Y_lm(p)).  conj(Y_lm) = Ptilde_l^m e^{-i m phi},
// so the sum is the adjoint synthesis of the weighted map (the adjoint
// kernels) halved for m >= 1, where the real-inner-product adjoint carries
// the factor 2 of the -m terms.  The two kernels here are the parts the
// adjoint does not already do: weighting the map (optionally the residual
// f - Y a of a Jacobi refinement step) and folding the adjoint's output into
// the estimate.  Both are HBM streams, one pass each.
#include "shtb_internal.h"

namespace {

// r[b][p] = w_ring(p) (f[b][p] - y[b][p]) (y == nullptr: w f).  One CTA per
// (ring, map); y may alias r.
__global__ void ring_weight_kernel(PlanView v, const double *__restrict__ f, const double *y,
                                   const double *__restrict__ ring_w, double w0, double *r)
{
    const int ring = blockIdx.x;
    const size_t base = (size_t)blockIdx.y * v.npix + v.ring_start[ring];
    const int J = v.ring_J[ring];
    const double w = ring_w ? ring_w[ring] : w0;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        double x = f[base + j];
        if (y) x -= y[base + j];
        r[base + j] = w * x;
    }
}

// alm[b] = (first ? 0 : alm[b]) + h_m g[b], h_0 = 1, h_m = 1/2 (m >= 1).
// One CTA per m; g may alias alm when first.
__global__ void alm_quadrature_add_kernel(PlanView v, const double2 *g, double2 *alm, int nmaps,
                                          int first)
{
    const int m = blockIdx.x;
    const int L = v.lmax;
    const long long off = (long long)m * (2 * L + 1 - m) / 2 + m;
    const int n = L - m + 1;
    const double h = m == 0 ? 1.0 : 0.5;
    for (int i = threadIdx.x; i < n * nmaps; i += blockDim.x) {
        const int b = i / n, dl = i - b * n;
        const size_t idx = (size_t)b * v.nalm + off + dl;
        double2 x = g[idx];
        x.x *= h;
        x.y *= h;
        if (!first) {
            const double2 a = alm[idx];
            x.x += a.x;
            x.y += a.y;
        }
        alm[idx] = x;
    }
}

}  // namespace

int launch_ring_weight(const shtb_plan_s *p, const double *f, const double *y, const double *ring_w,
                       double w0, double *r, int nmaps, cudaStream_t st)
{
    if (p->nrings < 1) return SHTB_OK;
    ring_weight_kernel<<<dim3(p->nrings, nmaps), 256, 0, st>>>(p->view, f, y, ring_w, w0, r);
    ++p->launches;
    SHTB_CUDA_TRY(cudaGetLastError());
    return SHTB_OK;
}

int launch_alm_quadrature_add(const shtb_plan_s *p, const double2 *g, double2 *alm, int nmaps,
                              bool first, cudaStream_t st)
{
    alm_quadrature_add_kernel<<<p->lmax + 1, 256, 0, st>>>(p->view, g, alm, nmaps, first ? 1 : 0);
    ++p->launches;
    SHTB_CUDA_TRY(cudaGetLastError());
    return SHTB_OK;
}
