// Extreme eigenvalues of a symmetric tridiagonal matrix, for the condition
// number estimates drawn from CG's coefficients (the Lanczos connection:
// the step lengths alpha_j and direction coefficients beta_j of preconditioned
// CG define the tridiagonal matrix of the Lanczos process on B L, whose
// eigenvalues approximate those of B L from inside its spectrum).
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "lap_internal.h"

namespace lap {
namespace {

// Number of eigenvalues below x of the tridiagonal (a, b): the negative
// pivots of the LDL^T factorisation of T - x I (Sturm sequence count).
int count_below(const std::vector<double> &a, const std::vector<double> &b, double x, double tiny)
{
    int neg = 0;
    double d = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        d = (a[i] - x) - (i ? b[i - 1] * b[i - 1] / d : 0.0);
        if (d == 0.0) d = -tiny;                 // step past an exact zero pivot
        if (d < 0.0) ++neg;
    }
    return neg;
}

// The j-th smallest eigenvalue (1-based) by bisection inside [lo, hi].
double kth_eigenvalue(const std::vector<double> &a, const std::vector<double> &b, int j, double lo,
                      double hi, double tiny)
{
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;      // interval at machine resolution
        if (count_below(a, b, mid, tiny) >= j) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

bool tridiag_extremes(const std::vector<double> &a, const std::vector<double> &b, double *lo, double *hi)
{
    const size_t k = a.size();
    if (k == 0 || b.size() + 1 < k) return false;
    // Gershgorin interval
    double glo = std::numeric_limits<double>::infinity(), ghi = -glo, scale = 0.0;
    for (size_t i = 0; i < k; ++i) {
        const double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
        glo = std::min(glo, a[i] - r);
        ghi = std::max(ghi, a[i] + r);
        scale = std::max(scale, std::fabs(a[i]) + r);
        if (!std::isfinite(a[i]) || !std::isfinite(r)) return false;
    }
    const double tiny = std::numeric_limits<double>::min() + scale * 1e-300;
    *lo = kth_eigenvalue(a, b, 1, glo, ghi, tiny);
    *hi = kth_eigenvalue(a, b, static_cast<int>(k), glo, ghi, tiny);
    return true;
}

bool lanczos_tridiagonal(const double *alpha, const double *beta, int k, std::vector<double> &a,
                         std::vector<double> &b)
{
    a.assign(static_cast<size_t>(std::max(k, 0)), 0.0);
    b.assign(static_cast<size_t>(std::max(k - 1, 0)), 0.0);
    for (int j = 0; j < k; ++j) {
        if (!(alpha[j] > 0.0) || !std::isfinite(alpha[j])) return false;
        a[j] = 1.0 / alpha[j] + (j ? beta[j - 1] / alpha[j - 1] : 0.0);
        if (j + 1 < k) {
            if (!(beta[j] >= 0.0)) return false;
            b[j] = std::sqrt(beta[j]) / alpha[j];
        }
    }
    return true;
}

}  // namespace lap
