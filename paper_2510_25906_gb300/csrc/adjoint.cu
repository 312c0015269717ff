// adjoint.cu -- vector-Jacobian product of the residual, g = lam^T dR/dU,
// with the cell classes frozen (FP64).
//
// R_c = -(1/|V_c|) sum_q w_q F(W_cq, W_nq, n_q)  (eq. EulerEquationsDetails):
// the residual depends on U only through the face-point states W, so the
// product is taken in two steps.
//   1. k_flux_vjp: mu_cq = dR/dW_cq^T lam, one group per cell, lane per
//      face point.  W_cq enters the cell's own flux evaluation as the left
//      state and the neighbour's evaluation of the same face as the right
//      state (each face is evaluated by both cells), so
//        mu_cq = -w_q J_L(W_cq, W_nq, n)^T lam_c / |V_c|
//                - w'_q J_R(W_nq, W_cq, -n)^T lam_n / |V_n|,
//      with J_L + J_R at an open boundary (outside state = inside state).
//      The Rusanov, HLL and HLLC fluxes are conservative under the exchange
//      of the sides, F(b, a, -n) = -F(a, b, n) (the wave speeds map to
//      minus each other), so J_R(W_nq, W_cq, -n) = -J_L(W_cq, W_nq, n) and
//        mu_cq = J_L(W_cq, W_nq, n)^T (w'_q lam_n / |V_n| - w_q lam_c / |V_c|):
//      one vector-Jacobian product per face point, by the reverse mode of
//      the solver (riemann_vjp; the wave pattern taken as in the plain
//      evaluation).
//   2. The face states per class (the detector, tagging and Harten decisions
//      frozen):
//        LINEAR (Sec. 2.1)  W_q = U_0 + sum_m L_qm (U_m - U_0):
//          a_cm = sum_q L_qm mu_cq,  a_c0 = sum_q mu_cq - sum_m a_cm
//        FIRST              W_q = U_0:  a_c0 = sum_q mu_cq
//        CWENOZ (Sec. 2.3), MUSCL + Barth-Jespersen or Venkatakrishnan
//          (Sec. 2.2): the reverse mode of the per-variable reconstruction,
//          one thread per (cell, variable), limiter bounds and minima taken
//          as in the plain evaluation.
//      a_cm is the contribution to the m-th stencil cell of c.
//   3. k_gather_vjp: g_j = a_j0 + sum over the (c, m) with sten[c][m] = j of
//      a_cm, in ascending (c, m): deterministic, no atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "hfv_internal.h"
#include "kernels.cuh"
#include "launch.cuh"

namespace hfv {
namespace {

struct AdjParams {
    int64_t nc;
    const int32_t* sten;
    const int32_t* nbr;
    const int8_t* nbrf;
    const int32_t* nfs;
    const uint8_t* nfc;
    const int64_t* loff;
    const uint8_t* dir;
    const double* L;
    const double* P;
    const double* Phil;
    const double* OI;
    const double* Dd;
    const double* G;
    const double* W;
    const double* nrm;
    const double* ivol;
    const double* UA;    // cell-major state of the forward evaluation, [nc][P]
    const double* FS;    // face-point states of the forward evaluation
    const uint8_t* cls;  // classes after the forward evaluation (Harten fallbacks included)
    const int32_t* queue;
    const int32_t* counts;
    const double* lam;   // [nv][nc]
    double* MU;          // [qtot][nv] adjoint of the face-point states
    double* A;           // [nc][M][nv] contributions to the stencil cells
    double* S0;          // [nc][nv] contributions to the cell itself
    const int64_t* inv_ptr;
    const int32_t* inv_idx;
    double* g;           // [nv][nc]
    double gamma, lam1, eps_cw, b_cw;
    int limiter;
    double venk_k;
};

template <int NV>
struct AoS {
    static constexpr int P = NV == 4 ? 4 : 8;
};

// ---------------------------------------------------------------------------
// 1. Riemann flux
// ---------------------------------------------------------------------------
// Reverse mode of riemann<double, D, KIND> (physics.cuh): gL += (dF/dUL)^T y
// and gR += (dF/dUR)^T y at (UL, UR, n), every branch taken as in the plain
// evaluation.  The plain statements are recomputed first; then each one's
// adjoint, last to first (x_b denotes dJ/dx for J = y . F).
template <int D, int KIND>
__device__ __forceinline__ void riemann_vjp(const double* UL, const double* UR, const double* n, double g,
                                            const double* y, double* gL, double* gR)
{
    constexpr int NV = D + 2;
    // ---- plain evaluation ----
    const double il = 1.0 / UL[0], ir = 1.0 / UR[0];
    double ml2 = 0.0, mr2 = 0.0, mnl = 0.0, mnr = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        ml2 += UL[1 + k] * UL[1 + k];
        mr2 += UR[1 + k] * UR[1 + k];
        mnl += UL[1 + k] * n[k];
        mnr += UR[1 + k] * n[k];
    }
    const double unl = mnl * il, unr = mnr * ir;
    const double pl = (g - 1.0) * (UL[D + 1] - 0.5 * ml2 * il);
    const double pr = (g - 1.0) * (UR[D + 1] - 0.5 * mr2 * ir);
    double FL[NV], FR[NV];
    FL[0] = mnl;
    FR[0] = mnr;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        FL[1 + k] = UL[1 + k] * unl + pl * n[k];
        FR[1 + k] = UR[1 + k] * unr + pr * n[k];
    }
    FL[D + 1] = (UL[D + 1] + pl) * unl;
    FR[D + 1] = (UR[D + 1] + pr) * unr;
    const double cl = ::sqrt(g * pl * il), cr = ::sqrt(g * pr * ir);
    // ---- adjoints ----
    double FL_b[NV], FR_b[NV], UL_b[NV], UR_b[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { FL_b[v] = 0.0; FR_b[v] = 0.0; UL_b[v] = 0.0; UR_b[v] = 0.0; }
    double unl_b = 0.0, unr_b = 0.0, pl_b = 0.0, pr_b = 0.0, cl_b = 0.0, cr_b = 0.0, il_b = 0.0, ir_b = 0.0;
    if (KIND == kRusanov) {
        // F = (FL + FR) / 2 - s (UR - UL) / 2,  s = max(|unl| + cl, |unr| + cr)
        const double al = (unl < 0.0 ? -unl : unl) + cl, ar = (unr < 0.0 ? -unr : unr) + cr;
        const double sp = al > ar ? al : ar;
        double s_b = 0.0;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            FL_b[v] += 0.5 * y[v];
            FR_b[v] += 0.5 * y[v];
            UR_b[v] -= 0.5 * sp * y[v];
            UL_b[v] += 0.5 * sp * y[v];
            s_b -= 0.5 * y[v] * (UR[v] - UL[v]);
        }
        if (al > ar) {
            unl_b += unl < 0.0 ? -s_b : s_b;
            cl_b += s_b;
        } else {
            unr_b += unr < 0.0 ? -s_b : s_b;
            cr_b += s_b;
        }
    } else {
        const bool lmin = unl - cl < unr - cr, rmax = unl + cl > unr + cr;
        const double SL = lmin ? unl - cl : unr - cr, SR = rmax ? unl + cl : unr + cr;
        double SL_b = 0.0, SR_b = 0.0;
        if (SL >= 0.0) {
#pragma unroll
            for (int v = 0; v < NV; ++v) FL_b[v] += y[v];
        } else if (SR <= 0.0) {
#pragma unroll
            for (int v = 0; v < NV; ++v) FR_b[v] += y[v];
        } else if (KIND == kHLL) {
            // F = N inv,  N = SR FL - SL FR + SL SR (UR - UL),  inv = 1 / (SR - SL)
            const double inv = 1.0 / (SR - SL);
            double inv_b = 0.0;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const double dU = UR[v] - UL[v];
                const double N = SR * FL[v] - SL * FR[v] + SL * SR * dU;
                const double N_b = y[v] * inv;
                inv_b += y[v] * N;
                FL_b[v] += SR * N_b;
                FR_b[v] -= SL * N_b;
                UR_b[v] += SL * SR * N_b;
                UL_b[v] -= SL * SR * N_b;
                SR_b += N_b * (FL[v] + SL * dU);
                SL_b += N_b * (SR * dU - FR[v]);
            }
            SR_b -= inv * inv * inv_b;
            SL_b += inv * inv * inv_b;
        } else {
            // HLLC: the contact speed and the star state on its upwind side K
            const double ml = UL[0] * (SL - unl), mr = UR[0] * (SR - unr);
            const double num = pr - pl + ml * unl - mr * unr, rden = 1.0 / (ml - mr);
            const double Ss = num * rden;
            const bool left = Ss >= 0.0;
            const double* UK = left ? UL : UR;
            const double* FK = left ? FL : FR;
            const double SK = left ? SL : SR, unk = left ? unl : unr, pk = left ? pl : pr, mk = left ? ml : mr;
            const double ik = left ? il : ir;
            const double rS = 1.0 / (SK - Ss), fac = mk * rS, dS = Ss - unk, rm = 1.0 / mk;
            const double E1 = UK[D + 1] * ik + dS * (Ss + pk * rm), Es = fac * E1;
            double FK_b[NV], UK_b[NV];
            double SK_b = 0.0, fac_b = 0.0, ik_b = 0.0, dS_b = 0.0;
#pragma unroll
            for (int v = 0; v < NV; ++v) { FK_b[v] = y[v]; UK_b[v] = 0.0; }
            // F[1+k] = FK[1+k] + SK (fac (UK[1+k] ik + dS n_k) - UK[1+k])
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double yk = y[1 + k], inner = UK[1 + k] * ik + dS * n[k];
                SK_b += yk * (fac * inner - UK[1 + k]);
                fac_b += yk * SK * inner;
                UK_b[1 + k] += yk * SK * (fac * ik - 1.0);
                ik_b += yk * SK * fac * UK[1 + k];
                dS_b += yk * SK * fac * n[k];
            }
            // F[0] = FK[0] + SK (fac - UK[0])
            SK_b += y[0] * (fac - UK[0]);
            fac_b += y[0] * SK;
            UK_b[0] -= y[0] * SK;
            // F[D+1] = FK[D+1] + SK (Es - UK[D+1]),  Es = fac E1
            SK_b += y[D + 1] * (Es - UK[D + 1]);
            UK_b[D + 1] -= y[D + 1] * SK;
            const double Es_b = y[D + 1] * SK;
            fac_b += Es_b * E1;
            const double E1_b = Es_b * fac;
            // E1 = UK[D+1] ik + dS (Ss + pk rm)
            UK_b[D + 1] += E1_b * ik;
            ik_b += E1_b * UK[D + 1];
            dS_b += E1_b * (Ss + pk * rm);
            double Ss_b = E1_b * dS;
            const double pk_b = E1_b * dS * rm;
            double mk_b = -rm * rm * (E1_b * dS * pk);
            // dS = Ss - unk;  fac = mk rS;  rS = 1 / (SK - Ss)
            Ss_b += dS_b;
            const double unk_b = -dS_b;
            mk_b += fac_b * rS;
            const double rS_b = fac_b * mk;
            SK_b -= rS * rS * rS_b;
            Ss_b += rS * rS * rS_b;
            // Ss = num rden;  rden = 1 / (ml - mr);  num = pr - pl + ml unl - mr unr
            const double num_b = Ss_b * rden, den_b = -rden * rden * (Ss_b * num);
            double ml_b = den_b + num_b * unl, mr_b = -den_b - num_b * unr;
            pr_b += num_b;
            pl_b -= num_b;
            unl_b += num_b * ml;
            unr_b -= num_b * mr;
            // the upwind side's quantities back to their own side
            if (left) {
#pragma unroll
                for (int v = 0; v < NV; ++v) { FL_b[v] += FK_b[v]; UL_b[v] += UK_b[v]; }
                SL_b += SK_b; unl_b += unk_b; pl_b += pk_b; ml_b += mk_b; il_b += ik_b;
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) { FR_b[v] += FK_b[v]; UR_b[v] += UK_b[v]; }
                SR_b += SK_b; unr_b += unk_b; pr_b += pk_b; mr_b += mk_b; ir_b += ik_b;
            }
            // ml = UL0 (SL - unl),  mr = UR0 (SR - unr)
            UL_b[0] += ml_b * (SL - unl);
            SL_b += ml_b * UL[0];
            unl_b -= ml_b * UL[0];
            UR_b[0] += mr_b * (SR - unr);
            SR_b += mr_b * UR[0];
            unr_b -= mr_b * UR[0];
        }
        // SL = min(unl - cl, unr - cr),  SR = max(unl + cl, unr + cr)
        if (lmin) { unl_b += SL_b; cl_b -= SL_b; } else { unr_b += SL_b; cr_b -= SL_b; }
        if (rmax) { unl_b += SR_b; cl_b += SR_b; } else { unr_b += SR_b; cr_b += SR_b; }
    }
    // the sides' fluxes, sound speeds, pressures and normal velocities
    auto side = [&](const double* U, double i, double un, double p, double c, double m2, double mn, const double* F_b,
                    double un_b, double p_b, double c_b, double i_b, double* U_b) {
        // F[0] = mn;  F[1+k] = U[1+k] un + p n_k;  F[D+1] = (U[D+1] + p) un
        double mn_b = F_b[0];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            U_b[1 + k] += F_b[1 + k] * un;
            un_b += F_b[1 + k] * U[1 + k];
            p_b += F_b[1 + k] * n[k];
        }
        U_b[D + 1] += F_b[D + 1] * un;
        p_b += F_b[D + 1] * un;
        un_b += F_b[D + 1] * (U[D + 1] + p);
        // c = sqrt(g p i)
        const double z_b = c_b * 0.5 / c;
        p_b += z_b * g * i;
        i_b += z_b * g * p;
        // p = (g - 1) (U[D+1] - m2 i / 2)
        U_b[D + 1] += (g - 1.0) * p_b;
        const double m2_b = -0.5 * (g - 1.0) * i * p_b;
        i_b -= 0.5 * (g - 1.0) * m2 * p_b;
        // un = mn i
        mn_b += un_b * i;
        i_b += un_b * mn;
        // mn = sum_k U[1+k] n_k;  m2 = sum_k U[1+k]^2;  i = 1 / U[0]
#pragma unroll
        for (int k = 0; k < D; ++k) U_b[1 + k] += mn_b * n[k] + 2.0 * U[1 + k] * m2_b;
        U_b[0] -= i * i * i_b;
    };
    side(UL, il, unl, pl, cl, ml2, mnl, FL_b, unl_b, pl_b, cl_b, il_b, UL_b);
    side(UR, ir, unr, pr, cr, mr2, mnr, FR_b, unr_b, pr_b, cr_b, ir_b, UR_b);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        gL[v] += UL_b[v];
        gR[v] += UR_b[v];
    }
}

template <class C, int KIND>
__global__ void __launch_bounds__(128) k_flux_vjp(AdjParams p)
{
    constexpr int NV = C::NV, D = C::D, NFP = C::NFP, G = GroupSize<C::QMAX>::value, CPB = 128 / G;
    const int lane = threadIdx.x % G;
    const int64_t c = (int64_t)blockIdx.x * CPB + threadIdx.x / G;
    if (c >= p.nc || lane >= C::QMAX) return;
    const int f = lane / NFP, a = lane - f * NFP;
    const int32_t nb = p.nfs[c * 6 + f];
    const int64_t q = c * C::QMAX + lane;
    double mu[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) mu[v] = 0.0;
    if (nb == -2) return;   // no such face
    double wl[NV], wr[NV], lc[NV], n[3];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        wl[v] = p.FS[q * NV + v];
        lc[v] = p.lam[(int64_t)v * p.nc + c];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] = p.nrm[(c * 6 + f) * 3 + k];
    const double wq = p.W[q];
    if (nb < 0) {
        // open boundary: the outside state is the inside one, J_L + J_R
        double gr[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) gr[v] = 0.0;
        riemann_vjp<D, KIND>(wl, wl, n, p.gamma, lc, mu, gr);
#pragma unroll
        for (int v = 0; v < NV; ++v) mu[v] = (mu[v] + gr[v]) * (-wq * p.ivol[c]);
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) wr[v] = p.FS[((int64_t)nb + a) * NV + v];
        // the cell's and the neighbour's weights of this face point, through
        // the one Jacobian of the cell's own evaluation
        const int64_t j = p.nbr[c * 6 + f];
        const double sc = -wq * p.ivol[c], sj = p.W[(int64_t)nb + a] * p.ivol[j];
        double y[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) y[v] = sc * lc[v] + sj * p.lam[(int64_t)v * p.nc + j];
        double gr[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) gr[v] = 0.0;
        riemann_vjp<D, KIND>(wl, wr, n, p.gamma, y, mu, gr);   // gr unused: dropped by the compiler
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) p.MU[q * NV + v] = mu[v];
}

// ---------------------------------------------------------------------------
// 2. face states: linear and first-order cells
// ---------------------------------------------------------------------------
// L_qm in a cell's block (FP64: column chunks of two, [M/2][Q][2])
__device__ __forceinline__ double l_at(const double* Lc, int q, int m, int Q) { return Lc[(m >> 1) * Q * 2 + q * 2 + (m & 1)]; }

// one thread per (cell, variable): a_cm = sum_q L_qm mu_cq for every m, and
// a_c0 = sum_q mu_cq - sum_m a_cm (FP64 instructions are this GPU's scarce
// resource: no lane idles on a short stencil and no sum goes through shuffles)
template <class C>
__global__ void __launch_bounds__(128) k_recon_lin_vjp(AdjParams p)
{
    constexpr int NV = C::NV, M = C::M, NFP = C::NFP;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.nc * NV) return;
    const int64_t c = t / NV;
    const int v = (int)(t - c * NV);
    const int cl = p.cls[c];
    const int Q = (p.nfc[c] & 15) * NFP;
    const double* mu = p.MU + c * C::QMAX * NV + v;
    double* A = p.A + c * M * NV + v;
    double sq = 0.0;
    for (int q = 0; q < Q; ++q) sq += mu[q * NV];
    double sa = 0.0;
    if (cl == CLS_LIN) {
        const double* Lc = p.L + p.loff[c];
        for (int m = 0; m < M; ++m) {
            double am = 0.0;
            for (int q = 0; q < Q; ++q) am += l_at(Lc, q, m, Q) * mu[q * NV];
            A[m * NV] = am;
            sa += am;
        }
    } else {
        for (int m = 0; m < M; ++m) A[m * NV] = 0.0;
    }
    p.S0[c * NV + v] = (cl == CLS_LIN || cl == CLS_FIRST) ? sq - sa : 0.0;
}

// ---------------------------------------------------------------------------
// 2. face states: CWENOZ and MUSCL cells, reverse mode
// ---------------------------------------------------------------------------
// Reverse mode of the CWENOZ face values of one variable (Sec. 2.3), formed
// as the forward kernel forms them: p_opt from P, the directional degree-1
// polynomials from D, p_1, the indicators through OI, tau and the weights,
// and
//   W_q = U_0 + (omega_1 / lambda_1) lin_q + sum_k Phi_qk g_k,
//   lin_q = sum_m L_qm (U_m - U_0),  g_k = sum_s coef_s sd_sk.
// Given wb[q] = dJ/dW_q, returns dJ/dU_0 and dJ/dU_m.  The plain values are
// evaluated first, then the adjoints last to first (x_b = dJ/dx); |x| takes
// slope +1 at 0 and tau = x^b slope b x^(b-1) (1 at x = 0 for b = 1).
template <class C>
__device__ void cweno_var_vjp(const AdjParams& p, int64_t c, int nf, double u0, const double* um, const double* wb,
                              double& u0_b, double* um_b)
{
    constexpr int M = C::M, N = C::N, D = C::D, MD = C::MD, NFP = C::NFP;
    // ---- plain values ----
    double du[M];
    for (int m = 0; m < M; ++m) du[m] = um[m] - u0;
    const double* P = p.P + c * (int64_t)N * M;
    double a[N];
    for (int k = 0; k < N; ++k) {
        double acc = 0.0;
        for (int m = 0; m < M; ++m) acc += P[k * M + m] * du[m];
        a[k] = acc;
    }
    double sd[6][D];
    for (int f = 0; f < nf; ++f)
        for (int k = 0; k < D; ++k) {
            const uint8_t* idx = p.dir + (c * 6 + f) * MD;
            const double* Dm = p.Dd + ((c * 6 + f) * D + k) * (int64_t)MD;
            double acc = 0.0;
            for (int b = 0; b < MD; ++b) acc += Dm[b] * du[idx[b]];
            sd[f][k] = acc;
        }
    const double lam1 = p.lam1, lams = (1.0 - lam1) / nf, eps = p.eps_cw;
    const double* OI = p.OI + c * (int64_t)C::NOI;
    // OI packed by rows of its upper triangle: entry (k, l >= k) at k N - k (k - 1) / 2 + l - k
    auto oi = [&](int k, int l) { return k <= l ? OI[k * N - k * (k - 1) / 2 + (l - k)] : OI[l * N - l * (l - 1) / 2 + (k - l)]; };
    double a1[N];
    for (int k = 0; k < N; ++k) {
        double sl = 0.0;
        if (k < D)
            for (int f = 0; f < nf; ++f) sl += sd[f][k];
        a1[k] = (a[k] - lams * sl) / lam1;
    }
    double OIa1[N], si1 = 0.0;
    for (int k = 0; k < N; ++k) {
        double t = 0.0;
        for (int l = 0; l < N; ++l) t += oi(k, l) * a1[l];
        OIa1[k] = t;
        si1 += a1[k] * t;
    }
    double sis[6], e[6], OIsd[6][D], tsum = 0.0;
    for (int f = 0; f < nf; ++f) {
        double s0 = 0.0;
        for (int k = 0; k < D; ++k) {
            double t = 0.0;
            for (int l = 0; l < D; ++l) t += oi(k, l) * sd[f][l];
            OIsd[f][k] = t;
            s0 += sd[f][k] * t;
        }
        sis[f] = s0;
        e[f] = s0 - si1;
        tsum += e[f] < 0.0 ? -e[f] : e[f];
    }
    const double x = tsum / (double)nf, tau = ::pow(x, p.b_cw);
    const double w1 = lam1 * (1.0 + tau / (eps + si1));
    double ws[6], wsum = w1;
    for (int f = 0; f < nf; ++f) {
        ws[f] = lams * (1.0 + tau / (eps + sis[f]));
        wsum += ws[f];
    }
    const double om1 = w1 / wsum, c0 = om1 / lam1;
    // ---- adjoints ----
    // W_q = U_0 + c0 lin_q + sum_k Phi_qk g_k
    const int Q = nf * NFP;
    const double* Lc = p.L + p.loff[c];
    double du_b[M], gk_b[D], c0_b = 0.0;
    for (int m = 0; m < M; ++m) du_b[m] = 0.0;
    for (int k = 0; k < D; ++k) gk_b[k] = 0.0;
    u0_b = 0.0;
    for (int q = 0; q < Q; ++q) {
        const double wq = wb[q], cw = c0 * wq;
        u0_b += wq;
        double lin = 0.0;
        for (int m = 0; m < M; ++m) {
            const double l = l_at(Lc, q, m, Q);
            lin += l * du[m];
            du_b[m] += cw * l;
        }
        c0_b += wq * lin;
        for (int k = 0; k < D; ++k) gk_b[k] += wq * p.Phil[(c * C::QMAX + q) * D + k];
    }
    // g_k = sum_s coef_s sd_sk,  coef_s = ws_s / wsum - om1 lams / lam1
    double sd_b[6][D], ws_b[6], wsum_b = 0.0, om1_b = 0.0;
    for (int f = 0; f < nf; ++f) {
        const double coef = ws[f] / wsum - om1 * lams / lam1;
        double coef_b = 0.0;
        for (int k = 0; k < D; ++k) {
            sd_b[f][k] = coef * gk_b[k];
            coef_b += gk_b[k] * sd[f][k];
        }
        ws_b[f] = coef_b / wsum;
        wsum_b -= coef_b * ws[f] / (wsum * wsum);
        om1_b -= coef_b * lams / lam1;
    }
    // c0 = om1 / lam1;  om1 = w1 / wsum;  wsum = w1 + sum_s ws_s
    om1_b += c0_b / lam1;
    double w1_b = om1_b / wsum;
    wsum_b -= om1_b * w1 / (wsum * wsum);
    w1_b += wsum_b;
    // ws_s = lams (1 + tau / (eps + SI_s)),  w1 = lam1 (1 + tau / (eps + SI_1))
    double tau_b = w1_b * lam1 / (eps + si1), si1_b = -w1_b * lam1 * tau / ((eps + si1) * (eps + si1)), sis_b[6];
    for (int f = 0; f < nf; ++f) {
        ws_b[f] += wsum_b;
        tau_b += ws_b[f] * lams / (eps + sis[f]);
        sis_b[f] = -ws_b[f] * lams * tau / ((eps + sis[f]) * (eps + sis[f]));
    }
    // tau = x^b, x = tsum / nf;  tsum = sum_s |SI_s - SI_1|
    const double slope = x != 0.0 ? p.b_cw * ::pow(x, p.b_cw - 1.0) : (p.b_cw == 1.0 ? 1.0 : 0.0);
    const double tsum_b = tau_b * slope / (double)nf;
    for (int f = 0; f < nf; ++f) {
        const double sg = e[f] < 0.0 ? -tsum_b : tsum_b;
        sis_b[f] += sg;
        si1_b -= sg;
    }
    // SI_s = sd_s^T OI sd_s (its D x D block);  SI_1 = a1^T OI a1
    for (int f = 0; f < nf; ++f)
        for (int k = 0; k < D; ++k) sd_b[f][k] += 2.0 * sis_b[f] * OIsd[f][k];
    // a1_k = (a_k - lams sum_s sd_sk [k < D]) / lam1
    double a_b[N];
    for (int k = 0; k < N; ++k) {
        const double a1_b = 2.0 * si1_b * OIa1[k];
        a_b[k] = a1_b / lam1;
        if (k < D)
            for (int f = 0; f < nf; ++f) sd_b[f][k] -= lams * a1_b / lam1;
    }
    // sd_sk = sum_b Dm_skb du[idx_s[b]];  a_k = sum_m P_km du_m
    for (int f = 0; f < nf; ++f)
        for (int k = 0; k < D; ++k) {
            const uint8_t* idx = p.dir + (c * 6 + f) * MD;
            const double* Dm = p.Dd + ((c * 6 + f) * D + k) * (int64_t)MD;
            for (int b = 0; b < MD; ++b) du_b[idx[b]] += Dm[b] * sd_b[f][k];
        }
    for (int m = 0; m < M; ++m) {
        double acc = du_b[m];
        for (int k = 0; k < N; ++k) acc += P[k * M + m] * a_b[k];
        um_b[m] = acc;            // du_m = U_m - U_0
        u0_b -= acc;
    }
}

// Reverse mode of the MUSCL face values of one variable (Sec. 2.2): the
// degree-1 gradient from the first Md stencil cells, Barth-Jespersen or
// Venkatakrishnan limiter with bounds over the cell and its face neighbours,
// one limiter value for all points, W_q = U_0 + theta dl_q.  The minima and
// maxima take the later operand on ties, as the forward kernel does; the
// adjoint follows the operand that was taken.
template <class C>
__device__ void muscl_var_vjp(const AdjParams& p, int64_t c, int nf, int n1, double u0, const double* um,
                              const double* wb, double& u0_b, double* um_b)
{
    constexpr int M = C::M, D = C::D, MD = C::MD, NFP = C::NFP;
    const double* Gm = p.G + c * (int64_t)D * MD;
    double gr[D];
    for (int k = 0; k < D; ++k) {
        double acc = 0.0;
        for (int b = 0; b < MD; ++b) acc += Gm[k * MD + b] * (um[b] - u0);
        gr[k] = acc;
    }
    double lo = u0, hi = u0;
    int lo_i = -1, hi_i = -1;   // -1: the cell itself
    for (int m = 0; m < n1; ++m) {
        if (!(lo < um[m])) { lo = um[m]; lo_i = m; }
        if (!(hi > um[m])) { hi = um[m]; hi_i = m; }
    }
    double eps2 = 0.0;
    if (p.limiter == 1) {
        const double vol = 1.0 / p.ivol[c];
        const double kd = p.venk_k * (D == 2 ? ::sqrt(vol) : ::cbrt(vol));
        eps2 = kd * kd * kd;
    }
    const int Q = nf * NFP;
    double dl[C::QMAX];
    double th = 1.0;
    int th_q = -1;   // the point whose limiter ratio theta is; -1: theta is the constant 1
    for (int q = 0; q < Q; ++q) {
        double d0 = 0.0;
        for (int k = 0; k < D; ++k) d0 += p.Phil[(c * C::QMAX + q) * D + k] * gr[k];
        dl[q] = d0;
        double t = 1.0;
        bool ratio = false;
        if (p.limiter == 1) {
            if (d0 > 0.0 || d0 < 0.0) {
                const double d1 = (d0 > 0.0 ? hi : lo) - u0;
                const double r = ((d1 * d1 + eps2) * d0 + 2.0 * d0 * d0 * d1) / (d0 * (d1 * d1 + 2.0 * d0 * d0 + d1 * d0 + eps2));
                ratio = !(1.0 < r);
                t = ratio ? r : 1.0;
            }
        } else if (d0 > 0.0 || d0 < 0.0) {
            const double r = ((d0 > 0.0 ? hi : lo) - u0) / d0;
            ratio = !(1.0 < r);
            t = ratio ? r : 1.0;
        }
        if (!(th < t)) { th = t; th_q = ratio ? q : -1; }
    }
    // ---- adjoints ----
    double dl_b[C::QMAX], th_b = 0.0;
    u0_b = 0.0;
    for (int m = 0; m < M; ++m) um_b[m] = 0.0;
    for (int q = 0; q < Q; ++q) {
        u0_b += wb[q];
        th_b += wb[q] * dl[q];
        dl_b[q] = th * wb[q];
    }
    if (th_q >= 0) {
        const double d0 = dl[th_q];
        const bool up = d0 > 0.0;
        double ext_b, d0_b;
        if (p.limiter == 1) {
            const double d1 = (up ? hi : lo) - u0;
            const double num = (d1 * d1 + eps2) * d0 + 2.0 * d0 * d0 * d1;
            const double den = d0 * (d1 * d1 + 2.0 * d0 * d0 + d1 * d0 + eps2);
            const double num_b = th_b / den, den_b = -th_b * num / (den * den);
            d0_b = num_b * (d1 * d1 + eps2 + 4.0 * d0 * d1) + den_b * (d1 * d1 + 6.0 * d0 * d0 + 2.0 * d1 * d0 + eps2);
            ext_b = num_b * (2.0 * d1 * d0 + 2.0 * d0 * d0) + den_b * (2.0 * d0 * d1 + d0 * d0);
        } else {
            const double r = ((up ? hi : lo) - u0) / d0;
            ext_b = th_b / d0;
            d0_b = -th_b * r / d0;
        }
        u0_b -= ext_b;   // d1 (or the bound's gap) = bound - U_0
        const int ei = up ? hi_i : lo_i;
        if (ei < 0) u0_b += ext_b;
        else um_b[ei] += ext_b;
        dl_b[th_q] += d0_b;
    }
    // dl_q = sum_k Phi_qk gr_k;  gr_k = sum_b G_kb (U_b - U_0)
    double gr_b[D];
    for (int k = 0; k < D; ++k) {
        double acc = 0.0;
        for (int q = 0; q < Q; ++q) acc += p.Phil[(c * C::QMAX + q) * D + k] * dl_b[q];
        gr_b[k] = acc;
    }
    for (int b = 0; b < MD; ++b) {
        double acc = 0.0;
        for (int k = 0; k < D; ++k) acc += Gm[k * MD + b] * gr_b[k];
        um_b[b] += acc;
        u0_b -= acc;
    }
}

// one item per (queued cell, variable): the face values' adjoints of that
// variable back to U_0 (S0) and to the stencil values (A)
template <class C>
__device__ void nl_vjp_item(const AdjParams& p, int which, int64_t t)
{
    constexpr int NV = C::NV, M = C::M, NFP = C::NFP, P4 = AoS<NV>::P;
    const int v = (int)(t % NV);
    const int64_t c = p.queue[which * p.nc + t / NV];
    const int cl = p.cls[c];
    if (cl != (which == 0 ? CLS_CW : CLS_MU)) return;   // fell back to first order: handled as such
    const int nfv = p.nfc[c], nf = nfv & 15, n1 = nfv >> 4, Q = nf * NFP;
    const double u0 = p.UA[c * P4 + v];
    double um[M], wb[C::QMAX], um_b[M], u0_b;
    const int32_t* st = p.sten + c * M;
    for (int m = 0; m < M; ++m) um[m] = p.UA[(int64_t)st[m] * P4 + v];
    const double* mu = p.MU + c * C::QMAX * NV;
    for (int q = 0; q < Q; ++q) wb[q] = mu[q * NV + v];
    if (which == 0) cweno_var_vjp<C>(p, c, nf, u0, um, wb, u0_b, um_b);
    else muscl_var_vjp<C>(p, c, nf, n1, u0, um, wb, u0_b, um_b);
    p.S0[c * NV + v] = u0_b;
    for (int m = 0; m < M; ++m) p.A[(c * M + m) * NV + v] = um_b[m];
}

// the items of one queue, the grid striding over them (the queue length is
// on the device: a grid sized for the worst case would be mostly empty)
template <class C>
__global__ void __launch_bounds__(64) k_recon_nl_vjp(AdjParams p, int which)
{
    const int64_t n = (int64_t)p.counts[which] * C::NV;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        nl_vjp_item<C>(p, which, t);
}

// ---------------------------------------------------------------------------
// 3. gather
// ---------------------------------------------------------------------------
template <int NV, int M>
__global__ void __launch_bounds__(256) k_gather_vjp(AdjParams p)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.nc) return;
    double s[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = p.S0[j * NV + v];
    for (int64_t e = p.inv_ptr[j]; e < p.inv_ptr[j + 1]; ++e) {
        const int64_t x = p.inv_idx[e];
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] += p.A[x * NV + v];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) p.g[(int64_t)v * p.nc + j] = s[v];
}

template <class C>
int run_vjp(hfv_scheme* s, const double* lam, double* g, cudaStream_t st)
{
    const hfv_dev_arrays& a = s->a;
    AdjParams p;
    p.nc = s->mesh->nc;
    p.sten = a.sten; p.nbr = a.nbr; p.nbrf = a.nbrf; p.nfs = a.nfs; p.nfc = a.nfc; p.loff = a.loff; p.dir = a.dir;
    p.L = (const double*)a.L; p.P = (const double*)a.P; p.Phil = (const double*)a.Phil; p.OI = (const double*)a.OI;
    p.Dd = (const double*)a.D; p.G = (const double*)a.G; p.W = (const double*)a.W; p.nrm = (const double*)a.nrm;
    p.ivol = (const double*)a.ivol; p.UA = (const double*)a.UA; p.FS = (const double*)a.FS; p.cls = a.cls;
    p.queue = a.queue; p.counts = a.counts; p.lam = lam;
    p.MU = s->adj.MU; p.A = s->adj.A; p.S0 = s->adj.S0; p.inv_ptr = s->adj.inv_ptr; p.inv_idx = s->adj.inv_idx; p.g = g;
    p.gamma = s->p.gamma; p.lam1 = 1.0 - 1.0 / s->p.lambda1_prime; p.eps_cw = s->p.cweno_eps; p.b_cw = s->p.cweno_b;
    p.limiter = s->p.limiter; p.venk_k = s->p.venkat_k;
    const int64_t nc = p.nc;
    constexpr int CPB = 128 / GroupSize<C::QMAX>::value;
    const unsigned gf = (unsigned)((nc + CPB - 1) / CPB);
    {
        Launch l(s, KID_VJP_FLUX, st);
        switch (s->p.flux) {
        case HFV_RUSANOV: k_flux_vjp<C, kRusanov><<<gf, 128, 0, st>>>(p); break;
        case HFV_HLL: k_flux_vjp<C, kHLL><<<gf, 128, 0, st>>>(p); break;
        default: k_flux_vjp<C, kHLLC><<<gf, 128, 0, st>>>(p); break;
        }
    }
    {
        Launch l(s, KID_VJP_RECON, st);
        k_recon_lin_vjp<C><<<(unsigned)((nc * C::NV + 127) / 128), 128, 0, st>>>(p);
    }
    // queued cells: at most nc per queue (the count itself lives on the
    // device); at most 64 blocks of 64 threads per SM, striding
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 1;
    }
    const unsigned gn = (unsigned)std::min<int64_t>((nc * C::NV + 63) / 64, (int64_t)sms * 32);
    for (int which = 0; which < 2; ++which) {
        Launch l(s, KID_VJP_RECON, st);
        k_recon_nl_vjp<C><<<gn, 64, 0, st>>>(p, which);
    }
    {
        Launch l(s, KID_VJP_GATHER, st);
        k_gather_vjp<C::NV, C::M><<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(p);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("hfv_residual_vjp: ") + cudaGetErrorString(e));
        return HFV_ERR_CUDA;
    }
    return HFV_OK;
}

// scratch of the adjoint and the inverse stencil map, made on first use
int adjoint_prepare(hfv_scheme* s, cudaStream_t st)
{
    if (s->adj.base) return HFV_OK;
    const int64_t nc = s->mesh->nc, M = s->M, nv = s->nv;
    const int64_t qtot = nc * s->nfmax * s->nfp;
    std::vector<int64_t> ptr(nc + 1, 0);
    std::vector<int32_t> idx(nc * M);
    for (int64_t e = 0; e < nc * M; ++e) ++ptr[s->sten[e] + 1];
    for (int64_t j = 0; j < nc; ++j) ptr[j + 1] += ptr[j];
    {
        std::vector<int64_t> pos(ptr.begin(), ptr.end() - 1);
        for (int64_t e = 0; e < nc * M; ++e) idx[pos[s->sten[e]]++] = (int32_t)e;   // ascending (c, m)
    }
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_mu = al(qtot * nv * 8), b_a = al(nc * M * nv * 8), b_s0 = al(nc * nv * 8), b_ptr = al((nc + 1) * 8),
                 b_idx = al(nc * M * 4), b_x = al(nc * nv * 8);
    void* base = nullptr;
    if (cudaMalloc(&base, b_mu + b_a + b_s0 + b_ptr + b_idx + 5 * b_x) != cudaSuccess) {
        set_error("hfv_residual_vjp: out of device memory for the adjoint scratch");
        return HFV_ERR_OOM;
    }
    char* b = (char*)base;
    s->adj.base = base;
    s->adj.MU = (double*)b;
    s->adj.A = (double*)(b + b_mu);
    s->adj.S0 = (double*)(b + b_mu + b_a);
    s->adj.inv_ptr = (int64_t*)(b + b_mu + b_a + b_s0);
    s->adj.inv_idx = (int32_t*)(b + b_mu + b_a + b_s0 + b_ptr);
    char* x = b + b_mu + b_a + b_s0 + b_ptr + b_idx;
    s->adj.X1 = (double*)x;
    s->adj.X2 = (double*)(x + b_x);
    s->adj.T = (double*)(x + 2 * b_x);
    s->adj.G = (double*)(x + 3 * b_x);
    s->adj.L2 = (double*)(x + 4 * b_x);
    if (cudaMemsetAsync(base, 0, b_mu + b_a + b_s0, st) != cudaSuccess ||
        cudaMemcpyAsync(s->adj.inv_ptr, ptr.data(), (nc + 1) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->adj.inv_idx, idx.data(), nc * M * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("hfv_residual_vjp: upload of the inverse stencil map failed");
        return HFV_ERR_CUDA;
    }
    return HFV_OK;
}

}  // namespace

int launch_vjp(hfv_scheme* s, const double* U, const uint8_t* cls, const double* lam, double* g, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = adjoint_prepare(s, st);
    if (rc != HFV_OK) return rc;
    // forward evaluation at U with the classes given: face states, final
    // classes (Harten fallbacks) and the CWENOZ / MUSCL queues
    rc = launch_residual(s, U, s->a.Rs, cls, nullptr, stream);
    if (rc != HFV_OK) return rc;
    if (s->d == 2) {
        switch (s->r) {
        case 1: return run_vjp<Cfg<2, 1>>(s, lam, g, st);
        case 2: return run_vjp<Cfg<2, 2>>(s, lam, g, st);
        case 3: return run_vjp<Cfg<2, 3>>(s, lam, g, st);
        case 4: return run_vjp<Cfg<2, 4>>(s, lam, g, st);
        }
    } else if (s->fam == 1) {
        switch (s->r) {
        case 1: return run_vjp<Cfg<3, 1, 1>>(s, lam, g, st);
        case 2: return run_vjp<Cfg<3, 2, 1>>(s, lam, g, st);
        }
    } else if (s->fam == 2) {
        switch (s->r) {
        case 1: return run_vjp<Cfg<3, 1, 2>>(s, lam, g, st);
        case 2: return run_vjp<Cfg<3, 2, 2>>(s, lam, g, st);
        }
    } else {
        switch (s->r) {
        case 1: return run_vjp<Cfg<3, 1>>(s, lam, g, st);
        case 2: return run_vjp<Cfg<3, 2>>(s, lam, g, st);
        case 3: return run_vjp<Cfg<3, 3>>(s, lam, g, st);
        }
    }
    set_error("hfv_residual_vjp: order not built");
    return HFV_ERR_ARG;
}

// out = a U0 + b (Us + dt R)  (a = 0: U0 unread)
__global__ void __launch_bounds__(256) k_stage_combine(int64_t n, const double* __restrict__ U0,
                                                      const double* __restrict__ Us, const double* __restrict__ R,
                                                      double a, double b, double dt, double* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = b * (Us[i] + dt * R[i]);
    if (a != 0.0) x += a * U0[i];
    out[i] = x;
}

// out = cx x + cy y + cz z + cg g  (null terms skipped)
__global__ void __launch_bounds__(256) k_lincomb(int64_t n, double* __restrict__ out, double cx,
                                                const double* __restrict__ x, double cy, const double* __restrict__ y,
                                                double cz, const double* __restrict__ z, double cg,
                                                const double* __restrict__ g)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = cx * x[i];
    if (y) v += cy * y[i];
    if (z) v += cz * z[i];
    if (g) v += cg * g[i];
    out[i] = v;
}

// One SSP-RK3 step, Shu-Osher form, from the residual with its classes
// output (forced = 0) or given (forced != 0): cls [3][nc], one per stage.
int launch_step_classes(hfv_scheme* s, const double* U, double dt, uint8_t* cls, int forced, double* out, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = adjoint_prepare(s, st);
    if (rc != HFV_OK) return rc;
    const int64_t nc = s->mesh->nc, n = (int64_t)s->nv * nc;
    const unsigned g = (unsigned)((n + 255) / 256);
    double* R = (double*)s->a.Rs;
    const double A[3] = {0.0, 0.75, 1.0 / 3.0}, B[3] = {1.0, 0.25, 2.0 / 3.0};
    const double* Us = U;
    double* outs[3] = {s->adj.X1, s->adj.X2, out};
    for (int k = 0; k < 3; ++k) {
        uint8_t* c = cls + k * nc;
        rc = forced ? launch_residual(s, Us, R, c, nullptr, stream) : launch_residual(s, Us, R, nullptr, c, stream);
        if (rc != HFV_OK) return rc;
        note_launch();
        k_stage_combine<<<g, 256, 0, st>>>(n, U, Us, R, A[k], B[k], dt, outs[k]);
        Us = outs[k];
    }
    return cudaGetLastError() == cudaSuccess ? HFV_OK : HFV_ERR_CUDA;
}

// The adjoint of one SSP-RK3 step with the stages' classes frozen: lam holds
// dJ/dU_{n+1} on entry and dJ/dU_n on return.  With U1 = U + h R(U),
// U2 = 3/4 U + 1/4 (U1 + h R(U1)), U3 = 1/3 U + 2/3 (U2 + h R(U2)):
//   l2 = 2/3 lam + h J2^T (2/3 lam)
//   l1 = 1/4 l2 + h J1^T (1/4 l2)
//   lam <- 1/3 lam + 3/4 l2 + l1 + h J0^T l1
// (J_k = dR/dU at stage k with its classes).
int launch_step_vjp(hfv_scheme* s, const double* U, const uint8_t* cls, double dt, double* lam, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nc = s->mesh->nc, n = (int64_t)s->nv * nc;
    int rc = launch_step_classes(s, U, dt, const_cast<uint8_t*>(cls), 1, s->adj.L2, stream);   // U1, U2 (U3 unused)
    if (rc != HFV_OK) return rc;
    const unsigned g = (unsigned)((n + 255) / 256);
    hfv_adjoint_arrays& a = s->adj;
    // stage 3
    note_launch();
    k_lincomb<<<g, 256, 0, st>>>(n, a.T, 2.0 / 3.0, lam, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr);
    if ((rc = launch_vjp(s, a.X2, cls + 2 * nc, a.T, a.G, stream)) != HFV_OK) return rc;
    note_launch();
    k_lincomb<<<g, 256, 0, st>>>(n, a.L2, 1.0, a.T, dt, a.G, 0.0, nullptr, 0.0, nullptr);
    // stage 2
    note_launch();
    k_lincomb<<<g, 256, 0, st>>>(n, a.T, 0.25, a.L2, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr);
    if ((rc = launch_vjp(s, a.X1, cls + nc, a.T, a.G, stream)) != HFV_OK) return rc;
    note_launch();
    k_lincomb<<<g, 256, 0, st>>>(n, a.T, 1.0, a.T, dt, a.G, 0.0, nullptr, 0.0, nullptr);   // T = l1
    // stage 1
    if ((rc = launch_vjp(s, U, cls, a.T, a.G, stream)) != HFV_OK) return rc;
    note_launch();
    k_lincomb<<<g, 256, 0, st>>>(n, lam, 1.0 / 3.0, lam, 0.75, a.L2, 1.0, a.T, dt, a.G);
    return cudaGetLastError() == cudaSuccess ? HFV_OK : HFV_ERR_CUDA;
}

void adjoint_free(hfv_scheme* s)
{
    if (s->adj.base) cudaFree(s->adj.base);
    s->adj = hfv_adjoint_arrays{};
}

}  // namespace hfv
