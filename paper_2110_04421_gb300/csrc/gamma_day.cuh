// gamma_day.cuh -- the integral of Eq. 1 (Sec. 3 "Infection Transmission"): the
// gamma(shape, scale) density integrated over one day [t-1, t], in FP64.
//
// Regularized incomplete gamma functions: P(s,x) by its power series (for
// x < s+1) and Q(s,x) = 1 - P(s,x) by Legendre's continued fraction evaluated
// with the modified Lentz method (Lentz 1976; Thompson and Barnett 1986), for
// x >= s+1.  Both table builders of the library (a context's set-up and the
// no-allocation entry point) include this one definition, so their tables are
// the same bit for bit.
#pragma once
#include <cstdint>

namespace deabm {

__device__ __forceinline__ double gamma_p_series(double s, double x)
{
    if (x <= 0.0) return 0.0;
    double ap = s, del = 1.0 / s, sum = del;
    for (int n = 0; n < 2000; ++n) {
        ap += 1.0;
        del *= x / ap;
        sum += del;
        if (fabs(del) < fabs(sum) * 1e-17) break;
    }
    return sum * exp(-x + s * log(x) - lgamma(s));
}

__device__ __forceinline__ double gamma_q_contfrac(double s, double x)
{
    const double tiny = 1e-300;
    double b = x + 1.0 - s, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 2000; ++i) {
        const double an = -(double)i * ((double)i - s);
        b += 2.0;
        d = an * d + b;
        if (fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        const double del = d * c;
        h *= del;
        if (fabs(del - 1.0) < 1e-17) break;
    }
    return exp(-x + s * log(x) - lgamma(s)) * h;
}

// integral of the gamma(shape, scale) density over day [t-1, t], t >= 1, taking
// each difference where it does not cancel
__device__ __forceinline__ double gamma_day(double shape, double scale, uint32_t t)
{
    const double a = ((double)t - 1.0) / scale, b = (double)t / scale, edge = shape + 1.0;
    if (b <= edge) return gamma_p_series(shape, b) - gamma_p_series(shape, a);
    if (a >= edge) return gamma_q_contfrac(shape, a) - gamma_q_contfrac(shape, b);
    return (1.0 - gamma_q_contfrac(shape, b)) - gamma_p_series(shape, a);
}

}  // namespace deabm
