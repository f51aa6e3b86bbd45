// Host-side helpers shared by the plan builders (dense tables and butterfly
// compression).  Internal; not part of the C ABI.
#pragma once

#include <vector>

#include "shtb_dd.h"
#include "shtb_internal.h"

namespace shtb {

// One ring with z >= 0 of the HEALPix RING grid (i = ring number from the
// north pole), with every quantity formed from exact integer ratios:
//   polar i < N : z = 1 - i^2/(3N^2), sin^2 = i^2 (6N^2 - i^2)/(9N^4)
//   belt        : z = (4N - 2i)/(3N),  sin^2 = (2i - N)(7N - 2i)/(9N^2)
struct HalfRing {
    double z;        // cos(theta), correctly rounded
    double z2;       // z^2, correctly rounded from the exact ratio
    double s2;       // sin^2(theta), correctly rounded from the exact ratio
    double eps1;     // 1 - z, correctly rounded from the exact ratio
    DD sdd;          // sin(theta) as dd
};

HalfRing half_ring(long long N, long long i);

// c_m = sqrt(1/(4 pi) prod_{i=1}^m (2i+1)/(2i)) as dd, m = 0..L
std::vector<DD> diag_norms(int L);

// b_l = sqrt((l^2 - m^2)/(4 l^2 - 1)) for l = m+1..L (index l - m)
std::vector<double> one_step_coefs(int L, int m);

// x^m as (mantissa in [0.5,1), power-of-two exponent)
DD dd_pow(DD x, int m, int *E);

// Ptilde_l^m at one half-ring for l = m..L by the one-step recurrence from
// Ptilde_m^m, with a power-of-two exponent while values are below the double
// range; entries below the 1e-30 crop are set to 0.  out has L - m + 1 slots.
void legendre_column(int L, int m, const HalfRing &h, DD cm, const std::vector<double> &b,
                     double *out);

// Spin-weighted s_lambda_lm (s = +-2) at one half-ring for l = m..L (zero
// below l = 2), by the Wigner recurrence in l; out has L - m + 1 slots.
void spin_column(int L, int m, int s, const HalfRing &h, DD cm, double *out);
// Lambda^{m,t} of both parities of one m (column-major, n_t rows x Z columns)
void build_lambda(int L, int m, int Z, const std::vector<HalfRing> &hr, DD cm, std::vector<double> &lam0,
                  std::vector<double> &lam1);

constexpr double kCrop = 1e-30;   // Appendix: values below 1e-30 are neglected

template <class F>
void parallel_for(int n, int nthreads, F &&fn);

}  // namespace shtb

#include <atomic>
#include <thread>

template <class F>
void shtb::parallel_for(int n, int nthreads, F &&fn)
{
    if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
    nthreads = std::min(nthreads, std::max(n, 1));
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (;;) {
            int i = next.fetch_add(1);
            if (i >= n) break;
            fn(i);
        }
    };
    if (nthreads == 1) {
        worker();
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; ++t) th.emplace_back(worker);
    for (auto &t : th) t.join();
}
