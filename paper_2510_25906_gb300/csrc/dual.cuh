// dual.cuh -- forward-mode dual numbers (value + K tangents) in FP64.
//
// The adjoint differentiates the Riemann solvers and the nonlinear
// reconstructions by evaluating the very same templated code on Dual<K>:
// every operation carries K directional derivatives, and every comparison
// acts on the value, so a branch (HLLC wave pattern, limiter bound, |x|) is
// taken as in the plain evaluation and differentiated as taken.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define DHD __host__ __device__ __forceinline__
#else
#define DHD inline
#endif

namespace hfv {

template <int K>
struct Dual {
    double v;
    double d[K];
    DHD Dual() : v(0.0)
    {
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] = 0.0;
    }
    DHD Dual(double x) : v(x)
    {
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] = 0.0;
    }
    DHD Dual& operator+=(const Dual& b)
    {
        v += b.v;
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] += b.d[k];
        return *this;
    }
    DHD Dual& operator-=(const Dual& b)
    {
        v -= b.v;
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] -= b.d[k];
        return *this;
    }
    DHD Dual& operator*=(const Dual& b)
    {
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] = d[k] * b.v + v * b.d[k];
        v *= b.v;
        return *this;
    }
};

template <int K>
DHD Dual<K> operator-(const Dual<K>& a)
{
    Dual<K> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
    return r;
}
template <int K>
DHD Dual<K> operator+(Dual<K> a, const Dual<K>& b) { return a += b; }
template <int K>
DHD Dual<K> operator-(Dual<K> a, const Dual<K>& b) { return a -= b; }
template <int K>
DHD Dual<K> operator*(Dual<K> a, const Dual<K>& b) { return a *= b; }
template <int K>
DHD Dual<K> operator/(const Dual<K>& a, const Dual<K>& b)
{
    Dual<K> r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
template <int K>
DHD Dual<K> operator+(Dual<K> a, double b) { a.v += b; return a; }
template <int K>
DHD Dual<K> operator+(double b, Dual<K> a) { a.v += b; return a; }
template <int K>
DHD Dual<K> operator-(Dual<K> a, double b) { a.v -= b; return a; }
template <int K>
DHD Dual<K> operator-(double b, const Dual<K>& a) { return Dual<K>(b) - a; }
template <int K>
DHD Dual<K> operator*(Dual<K> a, double b)
{
    a.v *= b;
#pragma unroll
    for (int k = 0; k < K; ++k) a.d[k] *= b;
    return a;
}
template <int K>
DHD Dual<K> operator*(double b, Dual<K> a) { return a * b; }
template <int K>
DHD Dual<K> operator/(const Dual<K>& a, double b) { return a * (1.0 / b); }
template <int K>
DHD Dual<K> operator/(double a, const Dual<K>& b) { return Dual<K>(a) / b; }

#define HFV_DUAL_CMP(op)                                                                  \
    template <int K>                                                                      \
    DHD bool operator op(const Dual<K>& a, const Dual<K>& b) { return a.v op b.v; }        \
    template <int K>                                                                      \
    DHD bool operator op(const Dual<K>& a, double b) { return a.v op b; }                  \
    template <int K>                                                                      \
    DHD bool operator op(double a, const Dual<K>& b) { return a op b.v; }
HFV_DUAL_CMP(<)
HFV_DUAL_CMP(>)
HFV_DUAL_CMP(<=)
HFV_DUAL_CMP(>=)
#undef HFV_DUAL_CMP

template <int K>
DHD Dual<K> sqrt(const Dual<K>& a)
{
    Dual<K> r;
    r.v = ::sqrt(a.v);
    const double h = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * h;
    return r;
}

// x^e for a constant exponent
template <int K>
DHD Dual<K> tpow(const Dual<K>& a, double e)
{
    Dual<K> r;
    r.v = ::pow(a.v, e);
    const double g = a.v != 0.0 ? e * ::pow(a.v, e - 1.0) : (e == 1.0 ? 1.0 : 0.0);
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * g;
    return r;
}

}  // namespace hfv
