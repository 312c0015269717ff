// physics.cuh -- perfect-gas Euler physics at a face point (Sec. 2):
// pressure, normal physical flux, and the Rusanov / HLL / HLLC Riemann
// solvers (Sec. 2.4 names HLLC and HLL; Rusanov is the local Lax-Friedrichs
// flux).  Davis wave-speed estimates; HLLC star states after Toro.
#pragma once

#ifdef __CUDACC__
#define HD __host__ __device__
#define HDI __host__ __device__ __forceinline__
#else
#define HD
#define HDI inline
#endif

namespace hfv {

enum { kRusanov = 0, kHLLC = 1, kHLL = 2 };

template <class T, int D>
HDI T pressure(const T* U, T g)
{
    T m2 = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) m2 += U[1 + k] * U[1 + k];
    return (g - T(1)) * (U[D + 1] - T(0.5) * m2 / U[0]);
}

// normal flux F(U).n and the normal velocity / pressure it used
template <class T, int D>
HDI void normal_flux(const T* U, const T* n, T g, T* F, T& un, T& p)
{
    T inv = T(1) / U[0];
    un = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) un += U[1 + k] * n[k];
    un *= inv;
    p = pressure<T, D>(U, g);
    F[0] = U[0] * un;
#pragma unroll
    for (int k = 0; k < D; ++k) F[1 + k] = U[1 + k] * un + p * n[k];
    F[D + 1] = (U[D + 1] + p) * un;
}

template <class T>
HDI T tsqrt(T x);
template <>
HDI float tsqrt<float>(float x) { return sqrtf(x); }
template <>
HDI double tsqrt<double>(double x) { return sqrt(x); }

template <class T, int D, int KIND>
HDI void riemann(const T* UL, const T* UR, const T* n, T g, T* F)
{
    constexpr int NV = D + 2;
    T FL[NV], FR[NV], unl, unr, pl, pr;
    normal_flux<T, D>(UL, n, g, FL, unl, pl);
    normal_flux<T, D>(UR, n, g, FR, unr, pr);
    T cl = tsqrt<T>(g * pl / UL[0]), cr = tsqrt<T>(g * pr / UR[0]);
    if (KIND == kRusanov) {
        T al = (unl < T(0) ? -unl : unl) + cl, ar = (unr < T(0) ? -unr : unr) + cr;
        T s = al > ar ? al : ar;
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = T(0.5) * (FL[v] + FR[v]) - T(0.5) * s * (UR[v] - UL[v]);
        return;
    }
    T a = unl - cl, b = unr - cr, SL = a < b ? a : b;
    a = unl + cl;
    b = unr + cr;
    T SR = a > b ? a : b;
    if (SL >= T(0)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = FL[v];
        return;
    }
    if (SR <= T(0)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = FR[v];
        return;
    }
    if (KIND == kHLL) {
        T inv = T(1) / (SR - SL);
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) * inv;
        return;
    }
    // contact wave speed
    T ml = UL[0] * (SL - unl), mr = UR[0] * (SR - unr);
    T Ss = (pr - pl + ml * unl - mr * unr) / (ml - mr);
    const bool left = Ss >= T(0);
    const T* UK = left ? UL : UR;
    const T* FK = left ? FL : FR;
    T SK = left ? SL : SR, unk = left ? unl : unr, pk = left ? pl : pr, mk = left ? ml : mr;
    T rk = UK[0];
    T fac = mk / (SK - Ss);   // rho*
    T dS = Ss - unk;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        T us = fac * (UK[1 + k] / rk + dS * n[k]);
        F[1 + k] = FK[1 + k] + SK * (us - UK[1 + k]);
    }
    F[0] = FK[0] + SK * (fac - UK[0]);
    T Es = fac * (UK[D + 1] / rk + dS * (Ss + pk / mk));
    F[D + 1] = FK[D + 1] + SK * (Es - UK[D + 1]);
}

}  // namespace hfv
