// Polarised (spin-2) synthesis: the combine of the two operators' outputs
// into the Q and U spectra of every ring.  The operators F+ and F- =
// (2_lambda +- (-2)_lambda)/2 are applied by the butterfly kernels of the
// scalar path (a polarised plan is two compressed plans).  For each map they
// leave the parity halves q^0, q^1 on the half-rings.  This kernel mirrors
// them onto all rings and forms Q_m and U_m (HEALPix convention, Sec. 5's
// spin-weighted transforms); the scalar ring stage then makes the maps.
//   F+ mirrors like the scalar functions: q(-z) = q^0 - q^1.
//   F- has the opposite parity:          q(-z) = -(q^0 - q^1).
//   Q_m = -(E+ + i B-),  U_m = -(B+ - i E-),
// where X+- is F+- applied to input X (E or B) of the pair.
#include "shtb_internal.h"

namespace {

// qp, qm: map-major parity halves, q[((b * 2 + t) * nhalf + r) * (L + 1) + m],
// inputs b = 2 pair (E) and 2 pair + 1 (B).  qring: ring-major
// [2 npairs][nrings][L + 1], Q then U per pair.  One CTA per (ring, pair).
__global__ void spin_combine_kernel(int L, int nhalf, int nrings, const double2 *__restrict__ qp,
                                    const double2 *__restrict__ qm, double2 *__restrict__ qring)
{
    const int ring = blockIdx.x, pair = blockIdx.y;
    const bool north = ring < nhalf;
    const int r = north ? ring : nrings - 1 - ring;
    const size_t half = (size_t)nhalf * (L + 1);
    auto at = [&](const double2 *q, int b, int m, bool odd_mirror) {
        const double2 *q0 = q + ((size_t)(b * 2) * nhalf + r) * (L + 1);
        const double2 x0 = q0[m];
        const double2 x1 = m + 1 <= L ? q0[half + m] : make_double2(0.0, 0.0);   // chain t = 1 exists
        if (north) return make_double2(x0.x + x1.x, x0.y + x1.y);
        return odd_mirror ? make_double2(x1.x - x0.x, x1.y - x0.y) : make_double2(x0.x - x1.x, x0.y - x1.y);
    };
    double2 *Q = qring + ((size_t)(2 * pair) * nrings + ring) * (L + 1);
    double2 *U = Q + (size_t)nrings * (L + 1);
    for (int m = threadIdx.x; m <= L; m += blockDim.x) {
        const double2 Ep = at(qp, 2 * pair, m, false), Bp = at(qp, 2 * pair + 1, m, false);
        const double2 Em = at(qm, 2 * pair, m, true), Bm = at(qm, 2 * pair + 1, m, true);
        Q[m] = make_double2(-(Ep.x - Bm.y), -(Ep.y + Bm.x));
        U[m] = make_double2(-(Bp.x + Em.y), -(Bp.y - Em.x));
    }
}

// Transpose of the combine, feeding the transposed butterflies: from the
// ring sums G_m(ring) = sum_j f_j e^{-i m phi_j} of the Q and U maps
// (ring-major [2 npairs][nrings][L + 1], Q then U), the gradients of the
// four operator outputs,
//   g(E+) = -G_Q,  g(B+) = -G_U,  g(E-) = -i G_U,  g(B-) = i G_Q,
// folded onto the half-rings by the transposed mirror (F+: g^0 = g_N + g_S,
// g^1 = g_N - g_S; F-: g^0 = g_N - g_S, g^1 = g_N + g_S; the equator has no
// mirror), in the entry-major layout of the adjoint butterflies,
// g[((m * 2 + t) * nhalf + r) * nmaps + b] with b = 2 pair (E), 2 pair + 1 (B).
// One CTA per (half-ring, block of kSpinM orders); threads run over
// (order, input) with the input fastest, so the stores are contiguous.
constexpr int kSpinM = 32;

__global__ void spin_uncombine_kernel(int L, int nhalf, int nrings, int npairs, const double2 *__restrict__ G,
                                      double2 *__restrict__ gp, double2 *__restrict__ gm)
{
    const int r = blockIdx.x, m0 = blockIdx.y * kSpinM;
    const int nm = min(kSpinM, L + 1 - m0), nb = 2 * npairs;
    const bool equator = r == nhalf - 1;
    const int south = nrings - 1 - r;
    for (int i = threadIdx.x; i < nm * nb; i += blockDim.x) {
        const int ml = i / nb, b = i - ml * nb, pair = b >> 1;
        const size_t m = (size_t)(m0 + ml);
        const double2 *gq = G + (size_t)(2 * pair) * nrings * (L + 1) + m;
        const double2 *gu = gq + (size_t)nrings * (L + 1);
        const double2 zero = make_double2(0.0, 0.0);
        const double2 qn = gq[(size_t)r * (L + 1)], qs = equator ? zero : gq[(size_t)south * (L + 1)];
        const double2 un = gu[(size_t)r * (L + 1)], us = equator ? zero : gu[(size_t)south * (L + 1)];
        double2 p0, p1, n0, n1;
        if ((b & 1) == 0) {   // E: g(E+) = -G_Q, g(E-) = -i G_U
            p0 = make_double2(-(qn.x + qs.x), -(qn.y + qs.y));
            p1 = make_double2(-(qn.x - qs.x), -(qn.y - qs.y));
            const double2 d = make_double2(un.x - us.x, un.y - us.y), a = make_double2(un.x + us.x, un.y + us.y);
            n0 = make_double2(d.y, -d.x);                                 // -i d
            n1 = make_double2(a.y, -a.x);                                 // -i a
        } else {              // B: g(B+) = -G_U, g(B-) = i G_Q
            p0 = make_double2(-(un.x + us.x), -(un.y + us.y));
            p1 = make_double2(-(un.x - us.x), -(un.y - us.y));
            const double2 d = make_double2(qn.x - qs.x, qn.y - qs.y), a = make_double2(qn.x + qs.x, qn.y + qs.y);
            n0 = make_double2(-d.y, d.x);                                 // i d
            n1 = make_double2(-a.y, a.x);                                 // i a
        }
        const size_t e0 = ((m * 2 + 0) * nhalf + r) * nb + b, e1 = ((m * 2 + 1) * nhalf + r) * nb + b;
        gp[e0] = p0;
        gp[e1] = p1;
        gm[e0] = n0;
        gm[e1] = n1;
    }
}

// alm += add (both [n] complex)
__global__ void alm_add_kernel(double2 *__restrict__ alm, const double2 *__restrict__ add, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = alm[i], b = add[i];
        alm[i] = make_double2(a.x + b.x, a.y + b.y);
    }
}

}  // namespace

int launch_spin_uncombine(const shtb_plan_s *p, const double2 *G, double2 *g_plus, double2 *g_minus, int npairs,
                          cudaStream_t st)
{
    spin_uncombine_kernel<<<dim3((unsigned)p->nhalf, (unsigned)((p->lmax + kSpinM) / kSpinM)), 256, 0, st>>>(
        p->lmax, p->nhalf, p->nrings, npairs, G, g_plus, g_minus);
    ++p->launches;
    SHTB_CUDA_TRY(cudaGetLastError());
    return SHTB_OK;
}

int launch_alm_add(const shtb_plan_s *p, double2 *alm, const double2 *add, size_t n, cudaStream_t st)
{
    alm_add_kernel<<<4 * 152, 256, 0, st>>>(alm, add, n);
    ++p->launches;
    SHTB_CUDA_TRY(cudaGetLastError());
    return SHTB_OK;
}

int launch_spin_combine(const shtb_plan_s *p, const double *qt_plus, const double *qt_minus, double2 *qring,
                        int npairs, cudaStream_t st)
{
    spin_combine_kernel<<<dim3((unsigned)p->nrings, (unsigned)npairs), 256, 0, st>>>(
        p->lmax, p->nhalf, p->nrings, (const double2 *)qt_plus, (const double2 *)qt_minus, qring);
    ++p->launches;
    SHTB_CUDA_TRY(cudaGetLastError());
    return SHTB_OK;
}
