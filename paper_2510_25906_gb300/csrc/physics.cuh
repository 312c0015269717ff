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

// generic forms; FP32 and FP64 below
template <class T>
HDI T tsqrt(T x) { return sqrt(x); }
template <>
HDI float tsqrt<float>(float x) { return ::sqrtf(x); }
template <>
HDI double tsqrt<double>(double x) { return ::sqrt(x); }

// reciprocal and square root.  FP32: the hardware approximations (about
// 2 ulp), far inside the FP32 path's 1e-5 bar.  FP64 square root: IEEE.
// FP64 reciprocal on the device: the hardware's approximate reciprocal as
// the seed y0, then two Newton-Raphson steps for f(y) = 1/y - x,
//   e = 1 - x y,  y <- y + y e  (each step squares the relative error),
// with fused multiply-adds: within about an ulp of 1/x for x and 1/x
// normal, one seed and four FMAs where the correctly rounded division
// takes several more FP64 instructions (this GPU's FP64 pipe executes two
// lanes per clock per SM, and the FP64 flux kernels keep it ~88 % busy).
template <class T>
HDI T trcp(T x) { return T(1) / x; }
template <>
HDI double trcp<double>(double x)
{
#ifdef __CUDA_ARCH__
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
#else
    return 1.0 / x;
#endif
}
template <>
HDI float trcp<float>(float x)
{
#ifdef __CUDA_ARCH__
    return __fdividef(1.0f, x);
#else
    return 1.0f / x;
#endif
}
template <class T>
HDI T fsqrt(T x) { return x > T(0) ? sqrt(x) : T(0); }
template <>
HDI double fsqrt<double>(double x) { return ::sqrt(x); }
template <>
HDI float fsqrt<float>(float x)
{
#ifdef __CUDA_ARCH__
    return x > 0.0f ? x * rsqrtf(x) : 0.0f;
#else
    return sqrtf(x);
#endif
}

template <class T, int D>
HDI T pressure(const T* U, T g)
{
    T m2 = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) m2 += U[1 + k] * U[1 + k];
    return (g - T(1)) * (U[D + 1] - T(0.5) * m2 * trcp<T>(U[0]));
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

template <class T, int D, int KIND>
HDI void riemann(const T* UL, const T* UR, const T* n, T g, T* F)
{
    constexpr int NV = D + 2;
    const T il = trcp<T>(UL[0]), ir = trcp<T>(UR[0]);
    T ml2 = T(0), mr2 = T(0), mnl = T(0), mnr = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        ml2 += UL[1 + k] * UL[1 + k];
        mr2 += UR[1 + k] * UR[1 + k];
        mnl += UL[1 + k] * n[k];
        mnr += UR[1 + k] * n[k];
    }
    const T unl = mnl * il, unr = mnr * ir;
    const T pl = (g - T(1)) * (UL[D + 1] - T(0.5) * ml2 * il);
    const T pr = (g - T(1)) * (UR[D + 1] - T(0.5) * mr2 * ir);
    T FL[NV], FR[NV];
    FL[0] = mnl;
    FR[0] = mnr;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        FL[1 + k] = UL[1 + k] * unl + pl * n[k];
        FR[1 + k] = UR[1 + k] * unr + pr * n[k];
    }
    FL[D + 1] = (UL[D + 1] + pl) * unl;
    FR[D + 1] = (UR[D + 1] + pr) * unr;
    const T cl = fsqrt<T>(g * pl * il), cr = fsqrt<T>(g * pr * ir);
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
        const T inv = trcp<T>(SR - SL);
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) * inv;
        return;
    }
    // contact wave speed and the star state on its upwind side
    const T ml = UL[0] * (SL - unl), mr = UR[0] * (SR - unr);
    const T Ss = (pr - pl + ml * unl - mr * unr) * trcp<T>(ml - mr);
    const bool left = Ss >= T(0);
    const T* UK = left ? UL : UR;
    const T* FK = left ? FL : FR;
    const T SK = left ? SL : SR, unk = left ? unl : unr, pk = left ? pl : pr, mk = left ? ml : mr, ik = left ? il : ir;
    const T fac = mk * trcp<T>(SK - Ss);   // rho*
    const T dS = Ss - unk;
#pragma unroll
    for (int k = 0; k < D; ++k) F[1 + k] = FK[1 + k] + SK * (fac * (UK[1 + k] * ik + dS * n[k]) - UK[1 + k]);
    F[0] = FK[0] + SK * (fac - UK[0]);
    const T Es = fac * (UK[D + 1] * ik + dS * (Ss + pk * trcp<T>(mk)));
    F[D + 1] = FK[D + 1] + SK * (Es - UK[D + 1]);
}

// Viscous flux F_v . n at one face point (Sec. 2: eqs. Terms1, Stresses,
// HeatConduct, sutherlandlaw, viscous_jump).  wl, wr: the two sides'
// conserved states; gl, gr: their gradients [D + 1][D] of the velocity
// components and of T = p / rho; inv_lint = 1 / (distance between the cells'
// centres), 0 on an open boundary.  Face state: the mean of the two sides'
// velocity and temperature; face gradient: the mean of the two sides'
// gradients plus (alpha / L_int)(W_R - W_L) n;
//   tau_ij = mu (d_j u_i + d_i u_j - 2/3 div u delta_ij),
//   Theta_j = sum_i u_i tau_ij + mu / Pr gamma / (gamma - 1) dT/dx_j,
//   mu = mu0 (T / T0)^(3/2) (T0 + S) / (T + S).
// (in the residual's precision: FP32 kernels convert no FP64 operand)
template <class T>
struct ViscParams {
    T mu0, t0, suth, inv_pr, alpha;
};

template <class T, int D>
HDI void viscous_flux(const T* wl, const T* wr, const T* gl, const T* gr, const T* n, T inv_lint, T g,
                      const ViscParams<T>& vp, T* F)
{
    T ql[D + 1], qr[D + 1];
    {
        const T il = T(1) / wl[0], ir = T(1) / wr[0];
        T ul2 = T(0), ur2 = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            ql[k] = wl[1 + k] * il;
            qr[k] = wr[1 + k] * ir;
            ul2 += ql[k] * ql[k];
            ur2 += qr[k] * qr[k];
        }
        ql[D] = (g - T(1)) * (wl[D + 1] - T(0.5) * wl[0] * ul2) * il;
        qr[D] = (g - T(1)) * (wr[D + 1] - T(0.5) * wr[0] * ur2) * ir;
    }
    T Gm[D + 1][D];
#pragma unroll
    for (int k = 0; k <= D; ++k) {
        const T pen = vp.alpha * inv_lint * (qr[k] - ql[k]);
#pragma unroll
        for (int j = 0; j < D; ++j) Gm[k][j] = T(0.5) * (gl[k * D + j] + gr[k * D + j]) + pen * n[j];
    }
    const T Tm = T(0.5) * (ql[D] + qr[D]), t0 = vp.t0, S = vp.suth;
    const T tr = Tm / t0;
    const T mu = vp.mu0 * tr * tsqrt<T>(tr) * (t0 + S) / (Tm + S);
    T div = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) div += Gm[k][k];
    const T kap = mu * vp.inv_pr * g / (g - T(1));
    F[0] = T(0);
    T fe = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T fi = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const T tij = mu * (Gm[i][j] + Gm[j][i] - (i == j ? T(2) / T(3) * div : T(0)));
            fi += tij * n[j];
        }
        F[1 + i] = fi;
        // sum_j (sum_i u_i tau_ij) n_j = sum_i u_i (tau . n)_i (tau symmetric)
        fe += T(0.5) * (ql[i] + qr[i]) * fi;
    }
#pragma unroll
    for (int j = 0; j < D; ++j) fe += kap * Gm[D][j] * n[j];
    F[D + 1] = fe;
}

}  // namespace hfv
