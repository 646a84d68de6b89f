// poisson.cuh -- log-space Poisson weights F_{d,i} = lambda^i e^{-lambda} / i!
// (Eq. Fmatrix) in double, by the saddle-point form of C. Loader, "Fast and
// accurate computation of binomial probabilities" (2000):
//     ln p(i; lambda) = -1/2 ln(2 pi i) - stirlerr(i) - bd0(i, lambda),   i >= 1,
// with stirlerr(n) = ln n! - (n + 1/2) ln n + n - 1/2 ln(2 pi) (the error of
// Stirling's formula) and bd0(x, m) = x ln(x/m) + m - x, both evaluated
// without the cancellation of the naive i ln(lambda) - lambda - ln i!, whose
// terms reach 1e7 at i ~ 1e6.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace tomo {

// stirlerr(n) for integer n >= 1.  n <= 15: from ln n! of the exactly
// representable integer n!; n > 15: the asymptotic series of ln Gamma with
// the Bernoulli coefficients B_2k / (2k (2k-1)) = 1/12, -1/360, 1/1260,
// -1/1680, 1/1188 (next term < 2e-16 relative at n = 16).
__device__ __forceinline__ double stirlerr(double n)
{
    const double half_ln_2pi = 0.91893853320467274178;  // ln(2 pi) / 2
    if (n <= 15.0) {
        double fact = 1.0;
        for (int k = 2; k <= int(n); ++k) fact *= double(k);
        return log(fact) - (n + 0.5) * log(n) + n - half_ln_2pi;
    }
    const double nn = n * n;
    const double S0 = 1.0 / 12.0, S1 = 1.0 / 360.0, S2 = 1.0 / 1260.0,
                 S3 = 1.0 / 1680.0, S4 = 1.0 / 1188.0;
    return (S0 - (S1 - (S2 - (S3 - S4 / nn) / nn) / nn) / nn) / n;
}

// bd0(x, m) = x ln(x/m) + m - x.  Near x = m it is summed from
// v = (x-m)/(x+m):  ln(x/m) = 2 atanh(v), hence
//     bd0 = v (x - m) + 2 x sum_{j>=1} v^(2j+1) / (2j+1).
__device__ __forceinline__ double bd0(double x, double m)
{
    if (fabs(x - m) < 0.1 * (x + m)) {
        const double v = (x - m) / (x + m);
        const double v2 = v * v;
        double s = (x - m) * v;
        double ej = 2.0 * x * v;
        for (int j = 1; j < 200; ++j) {
            ej *= v2;
            const double s1 = s + ej / double(2 * j + 1);
            if (s1 == s) return s1;
            s = s1;
        }
        return s;
    }
    return x * log(x / m) + m - x;
}

// ln F_{d,i} for lambda > 0 (Eq. Fmatrix in log space).
__device__ __forceinline__ double log_poisson(double i, double lam)
{
    if (i == 0.0) return -lam;
    const double ln_2pi = 1.83787706640934548356;
    return -0.5 * (ln_2pi + log(i)) - stirlerr(i) - bd0(i, lam);
}

__device__ __forceinline__ double poisson_weight(int64_t i, double lam)
{
    if (lam == 0.0) return i == 0 ? 1.0 : 0.0;
    return exp(log_poisson(double(i), lam));
}

}  // namespace tomo
