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
//      one Jacobian per face point.  It comes from the solver itself
//      evaluated on dual numbers (the wave pattern taken as in the plain
//      evaluation).
//   2. The face states per class (the detector, tagging and Harten decisions
//      frozen):
//        LINEAR (Sec. 2.1)  W_q = U_0 + sum_m L_qm (U_m - U_0):
//          a_cm = sum_q L_qm mu_cq,  a_c0 = sum_q mu_cq - sum_m a_cm
//        FIRST              W_q = U_0:  a_c0 = sum_q mu_cq
//        CWENOZ (Sec. 2.3), MUSCL + Barth-Jespersen (Sec. 2.2): the
//          per-variable reconstruction re-evaluated on dual numbers seeded
//          on U_0 and the stencil values, limiter bounds and minima taken as
//          in the plain evaluation.
//      a_cm is the contribution to the m-th stencil cell of c.
//   3. k_gather_vjp: g_j = a_j0 + sum over the (c, m) with sten[c][m] = j of
//      a_cm, in ascending (c, m): deterministic, no atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "dual.cuh"
#include "hfv_internal.h"
#include "kernels.cuh"

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
template <int D, int KIND>
__device__ void flux_jt(const double* WL, const double* WR, const double* n, double g, const double* lam, int which,
                        double* out)
{
    // out += J^T lam, J = dF/dW_L (which = 0), dF/dW_R (1), or both (2)
    constexpr int NV = D + 2;
    using DT = Dual<NV>;
    DT L[NV], R[NV], nn[3], F[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        L[v] = DT(WL[v]);
        R[v] = DT(WR[v]);
        if (which == 0 || which == 2) L[v].d[v] = 1.0;
        if (which == 1 || which == 2) R[v].d[v] = 1.0;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) nn[k] = DT(n[k]);
    riemann<DT, D, KIND>(L, R, nn, DT(g), F);
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        double s = 0.0;
#pragma unroll
        for (int v = 0; v < NV; ++v) s += lam[v] * F[v].d[j];
        out[j] += s;
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
        flux_jt<D, KIND>(wl, wl, n, p.gamma, lc, 2, mu);
#pragma unroll
        for (int v = 0; v < NV; ++v) mu[v] *= -wq * p.ivol[c];
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
        flux_jt<D, KIND>(wl, wr, n, p.gamma, y, 0, mu);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) p.MU[q * NV + v] = mu[v];
}

// ---------------------------------------------------------------------------
// 2. face states: linear and first-order cells, one warp per cell
// ---------------------------------------------------------------------------
// L_qm in a cell's block (FP64: column chunks of two, [M/2][Q][2])
__device__ __forceinline__ double l_at(const double* Lc, int q, int m, int Q) { return Lc[(m >> 1) * Q * 2 + q * 2 + (m & 1)]; }

template <class C>
__global__ void __launch_bounds__(128) k_recon_lin_vjp(AdjParams p)
{
    constexpr int NV = C::NV, M = C::M, NFP = C::NFP;
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (c >= p.nc) return;
    const int cl = p.cls[c];
    const int Q = (p.nfc[c] & 15) * NFP;
    const double* mu = p.MU + c * C::QMAX * NV;
    double* A = p.A + c * M * NV;
    double sq[NV], sa[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { sq[v] = 0.0; sa[v] = 0.0; }
    for (int q = lane; q < Q; q += 32)
#pragma unroll
        for (int v = 0; v < NV; ++v) sq[v] += mu[q * NV + v];
    const double* Lc = p.L + p.loff[c];
    for (int m = lane; m < M; m += 32) {
        double am[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) am[v] = 0.0;
        if (cl == CLS_LIN) {
            for (int q = 0; q < Q; ++q) {
                const double l = l_at(Lc, q, m, Q);
#pragma unroll
                for (int v = 0; v < NV; ++v) am[v] += l * mu[q * NV + v];
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            A[m * NV + v] = am[v];
            sa[v] += am[v];
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sq[v] += __shfl_xor_sync(0xffffffffu, sq[v], o);
            sa[v] += __shfl_xor_sync(0xffffffffu, sa[v], o);
        }
    if (lane < NV) {
        double x = 0.0;
#pragma unroll
        for (int v = 0; v < NV; ++v)
            if (v == lane) x = (cl == CLS_LIN || cl == CLS_FIRST) ? sq[v] - sa[v] : 0.0;
        p.S0[c * NV + lane] = x;
    }
}

// ---------------------------------------------------------------------------
// 2. face states: CWENOZ and MUSCL cells, dual numbers
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T dabs(const T& x) { return x < 0.0 ? -x : x; }
template <class T>
__device__ __forceinline__ T dmin(const T& a, const T& b) { return a < b ? a : b; }
template <class T>
__device__ __forceinline__ T dmax(const T& a, const T& b) { return a > b ? a : b; }
__device__ __forceinline__ double tpow(double x, double e) { return pow(x, e); }

// CWENOZ face values of one variable (Sec. 2.3), as the forward kernel forms
// them: p_opt from P, the directional degree-1 polynomials from D, p_1,
// the indicators through OI, tau and the weights, and
// W_q = U_0 + (omega_1 / lambda_1) (p_opt(x_q) - U_0) + sum_k Phi_qk G_k
template <class C, class S>
__device__ void cweno_var(const AdjParams& p, int64_t c, int nf, const S& u0, const S* um, S* w)
{
    constexpr int M = C::M, N = C::N, D = C::D, MD = C::MD, NFP = C::NFP;
    S du[M];
    for (int m = 0; m < M; ++m) du[m] = um[m] - u0;
    S a[N];
    const double* P = p.P + c * (int64_t)N * M;
    for (int k = 0; k < N; ++k) {
        S acc(0.0);
        for (int m = 0; m < M; ++m) acc += P[k * M + m] * du[m];
        a[k] = acc;
    }
    S sd[6][D];
    for (int f = 0; f < nf; ++f)
        for (int k = 0; k < D; ++k) {
            const uint8_t* idx = p.dir + (c * 6 + f) * MD;
            const double* Dm = p.Dd + ((c * 6 + f) * D + k) * (int64_t)MD;
            S acc(0.0);
            for (int b = 0; b < MD; ++b) acc += Dm[b] * du[idx[b]];
            sd[f][k] = acc;
        }
    const double lam1 = p.lam1, lams = (1.0 - lam1) / nf;
    const double* OI = p.OI + c * (int64_t)C::NOI;
    S a1[N];
    for (int k = 0; k < N; ++k) {
        S sl(0.0);
        if (k < D)
            for (int f = 0; f < nf; ++f) sl += sd[f][k];
        a1[k] = (a[k] - lams * sl) / lam1;
    }
    S si1(0.0);
    {
        int o = 0;
        for (int k = 0; k < N; ++k) {
            S t = OI[o++] * a1[k];
            for (int l = k + 1; l < N; ++l) t += 2.0 * OI[o++] * a1[l];
            si1 += a1[k] * t;
        }
    }
    S sis[6], tsum(0.0);
    for (int f = 0; f < nf; ++f) {
        S s0(0.0);
        for (int k = 0; k < D; ++k) {
            const int o = k * N - k * (k - 1) / 2;
            S t = OI[o] * sd[f][k];
            for (int l = k + 1; l < D; ++l) t += 2.0 * OI[o + (l - k)] * sd[f][l];
            s0 += sd[f][k] * t;
        }
        sis[f] = s0;
        tsum += dabs(s0 - si1);
    }
    const S tau = tpow(tsum / (double)nf, p.b_cw);
    const S w1 = lam1 * (1.0 + tau / (p.eps_cw + si1));
    S wsum = w1, ws[6];
    for (int f = 0; f < nf; ++f) {
        ws[f] = lams * (1.0 + tau / (p.eps_cw + sis[f]));
        wsum += ws[f];
    }
    const S om1 = w1 / wsum;
    const S c0 = om1 / lam1;
    S gk[D];
    for (int k = 0; k < D; ++k) {
        S acc(0.0);
        for (int f = 0; f < nf; ++f) acc += (ws[f] / wsum - om1 * lams / lam1) * sd[f][k];
        gk[k] = acc;
    }
    const int Q = nf * NFP;
    const double* Lc = p.L + p.loff[c];
    for (int q = 0; q < Q; ++q) {
        S lin(0.0);
        for (int m = 0; m < M; ++m) lin += l_at(Lc, q, m, Q) * du[m];
        S s0 = u0 + c0 * lin;
        for (int k = 0; k < D; ++k) s0 += p.Phil[(c * C::QMAX + q) * D + k] * gk[k];
        w[q] = s0;
    }
}

// MUSCL face values of one variable (Sec. 2.2): degree-1 gradient from the
// first Md stencil cells, Barth-Jespersen limiter with bounds over the cell
// and its face neighbours, one limiter value for all points
template <class C, class S>
__device__ void muscl_var(const AdjParams& p, int64_t c, int nf, int n1, const S& u0, const S* um, S* w)
{
    constexpr int D = C::D, MD = C::MD, NFP = C::NFP;
    S gr[D];
    const double* Gm = p.G + c * (int64_t)D * MD;
    for (int k = 0; k < D; ++k) {
        S acc(0.0);
        for (int b = 0; b < MD; ++b) acc += Gm[k * MD + b] * (um[b] - u0);
        gr[k] = acc;
    }
    S lo = u0, hi = u0;
    for (int m = 0; m < n1; ++m) {
        lo = dmin(lo, um[m]);
        hi = dmax(hi, um[m]);
    }
    double eps2 = 0.0;
    if (p.limiter == 1) {
        const double vol = 1.0 / p.ivol[c];
        const double kd = p.venk_k * (D == 2 ? ::sqrt(vol) : ::cbrt(vol));
        eps2 = kd * kd * kd;
    }
    const int Q = nf * NFP;
    S th(1.0);
    S dl[C::QMAX];
    for (int q = 0; q < Q; ++q) {
        S d0(0.0);
        for (int k = 0; k < D; ++k) d0 += p.Phil[(c * C::QMAX + q) * D + k] * gr[k];
        dl[q] = d0;
        S t(1.0);
        if (p.limiter == 1) {
            if (d0 > 0.0 || d0 < 0.0) {
                const S d1 = (d0 > 0.0 ? hi : lo) - u0;
                const S num = (d1 * d1 + eps2) * d0 + 2.0 * d0 * d0 * d1;
                const S den = d0 * (d1 * d1 + 2.0 * d0 * d0 + d1 * d0 + eps2);
                t = dmin(S(1.0), num / den);
            }
        } else {
            if (d0 > 0.0) t = dmin(S(1.0), (hi - u0) / d0);
            else if (d0 < 0.0) t = dmin(S(1.0), (lo - u0) / d0);
        }
        th = dmin(th, t);
    }
    for (int q = 0; q < Q; ++q) w[q] = u0 + th * dl[q];
}

constexpr int kTan = 8;   // tangents per dual evaluation

// one item per (queued cell, variable, chunk of kTan inputs): inputs are
// U_0 (index 0) and the stencil values U_m (index m + 1)
template <class C>
__device__ void nl_vjp_item(const AdjParams& p, int which, int64_t t)
{
    constexpr int NV = C::NV, M = C::M, NFP = C::NFP, P4 = AoS<NV>::P;
    constexpr int NCH = (M + 1 + kTan - 1) / kTan;
    using S = Dual<kTan>;
    const int ch = (int)(t % NCH);
    const int v = (int)((t / NCH) % NV);
    const int64_t c = p.queue[which * p.nc + t / (NCH * NV)];
    const int cl = p.cls[c];
    if (cl != (which == 0 ? CLS_CW : CLS_MU)) return;   // fell back to first order: handled as such
    const int nfv = p.nfc[c], nf = nfv & 15, n1 = nfv >> 4, Q = nf * NFP;
    S u0(p.UA[c * P4 + v]);
    S um[M];
    const int32_t* st = p.sten + c * M;
    for (int m = 0; m < M; ++m) um[m] = S(p.UA[(int64_t)st[m] * P4 + v]);
    const int e0 = ch * kTan;
    for (int k = 0; k < kTan; ++k) {
        const int e = e0 + k;
        if (e == 0) u0.d[k] = 1.0;
        else if (e <= M) um[e - 1].d[k] = 1.0;
    }
    S w[C::QMAX];
    if (which == 0) cweno_var<C, S>(p, c, nf, u0, um, w);
    else muscl_var<C, S>(p, c, nf, n1, u0, um, w);
    const double* mu = p.MU + c * C::QMAX * NV;
    for (int k = 0; k < kTan; ++k) {
        const int e = e0 + k;
        if (e > M) break;
        double s = 0.0;
        for (int q = 0; q < Q; ++q) s += mu[q * NV + v] * w[q].d[k];
        if (e == 0) p.S0[c * NV + v] = s;
        else p.A[(c * M + (e - 1)) * NV + v] = s;
    }
}

// the items of one queue, the grid striding over them (the queue length is
// on the device: a grid sized for the worst case would be mostly empty)
template <class C>
__global__ void __launch_bounds__(64) k_recon_nl_vjp(AdjParams p, int which)
{
    constexpr int NCH = (C::M + 1 + kTan - 1) / kTan;
    const int64_t n = (int64_t)p.counts[which] * C::NV * NCH;
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
    note_launch();
    switch (s->p.flux) {
    case HFV_RUSANOV: k_flux_vjp<C, kRusanov><<<gf, 128, 0, st>>>(p); break;
    case HFV_HLL: k_flux_vjp<C, kHLL><<<gf, 128, 0, st>>>(p); break;
    default: k_flux_vjp<C, kHLLC><<<gf, 128, 0, st>>>(p); break;
    }
    note_launch();
    k_recon_lin_vjp<C><<<(unsigned)((nc + 3) / 4), 128, 0, st>>>(p);
    // queued cells: at most nc per queue (the count itself lives on the
    // device); at most 64 blocks of 64 threads per SM, striding
    constexpr int NCH = (C::M + 1 + kTan - 1) / kTan;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 1;
    }
    const unsigned gn = (unsigned)std::min<int64_t>((nc * C::NV * NCH + 63) / 64, (int64_t)sms * 32);
    for (int which = 0; which < 2; ++which) {
        note_launch();
        k_recon_nl_vjp<C><<<gn, 64, 0, st>>>(p, which);
    }
    note_launch();
    k_gather_vjp<C::NV, C::M><<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(p);
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
