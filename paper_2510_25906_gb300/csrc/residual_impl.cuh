// residual_impl.cuh -- the kernels of one residual evaluation R(U) of the
// hybrid scheme (Sec. 2.5) and their launch sequence (run_residual), shared by
// the translation units that instantiate them per mesh family and order
// (residual_2d.cu, residual_2d_high.cu, residual_3d.cu, residual_hex.cu, residual_hex5.cu,
// residual_hex6.cu);
// residual.cu holds the dispatch and the Runge-Kutta steps.
//
//   K1 k_linear   all cells: stencil gather, linear candidate at the face
//                 points (U_0 + L (U_m - U_0), Sec. 2.1), detector raw class
//                 (eqs. DMP, NADMUSCL, NADCWENOZ, marginm, marginw,
//                 NADDeactivatedCriteria), Harten test of the candidate
//   K2 k_tag      class of a cell = max over itself and its face neighbours
//                 (tagging of the flagged cells' neighbourhood); linear cells
//                 that fail the Harten bound become first-order; the CWENOZ
//                 and MUSCL cells go into two queues (warp ballots, one
//                 atomic range reservation per block and queue)
//   K3 k_cweno    CWENOZ on the CWENOZ queue (Sec. 2.3)
//   K4 k_muscl    MUSCL + Barth-Jespersen on the MUSCL queue (Sec. 2.2)
//      (both apply the Harten bound, eq. harten_jump_fix)
//   K6 k_flux     Riemann fluxes at every face point, summed per cell
//                 (eq. EulerEquationsDetails); cell-centred, atomic-free
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <utility>

#include "device_common.cuh"
#include "hfv_internal.h"
#include "launch.cuh"
#include "k_linear.cuh"
#include "kernels.cuh"
#include "tma.cuh"

namespace hfv {

// The stable time step of one cell from its state u (the precision of the
// residual; FP64 for FP64 schemes):
//   dt = cfl |V| / (sum_f (|u . n_f| + a) |S_f| [+ 4 nu sum_f |S_f|^2 / |V|])
// with the diffusion limit when mu0 > 0 (nu = max(4/3, gamma / Pr) mu / rho);
// 0 for a non-physical state (it stops the step).  One function for the
// stage-in kernel and the chained flux epilogue, so that both give the same bits.
// in three parts, so that the flux kernel can spread the face terms over
// its face lanes and still sum them in the same order with the same FMAs
template <class T, int NV, int P>
__device__ __forceinline__ void cell_dt_state(const T (&u)[P], T g, T (&vel)[3], T& a, T& pr)
{
    constexpr int D = NV - 2;
    const T rho = u[0];
    T m2 = T(0);
    vel[0] = vel[1] = vel[2] = T(0);
    if constexpr (sizeof(T) == 4) {
        // FP32: a stability estimate; one fast reciprocal (as the Riemann solver)
        const T ir = trcp<T>(rho);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            vel[k] = u[1 + k] * ir;
            m2 += u[1 + k] * u[1 + k];
        }
        pr = (g - T(1)) * (u[D + 1] - T(0.5) * m2 * ir);
        a = fsqrt<T>(g * pr * ir);
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            vel[k] = u[1 + k] / rho;
            m2 += u[1 + k] * u[1 + k];
        }
        pr = (g - T(1)) * (u[D + 1] - T(0.5) * m2 / rho);
        a = tsqrt<T>(g * pr / rho);
    }
}
template <class T>
__device__ __forceinline__ T cell_dt_face(const T (&vel)[3], T a, const T* n)
{
    const T un = vel[0] * n[0] + vel[1] * n[1] + vel[2] * n[2];
    return tabs(un) + a;
}
// lam = sum_f face_f area_f (accumulated by the caller in face order), s2 =
// sum_f area_f^2; the step in the residual's precision (kept there for the
// minimum: FP64 instructions are scarce on this GPU, and the minimum of FP32
// values converted to FP64 is the conversion of their minimum)
template <class T, bool VISC>
__device__ __forceinline__ T cell_dt_finish(T lam, T s2, T rho, T pr, T ivol, T g, T cfl, const ViscParams<T>& vp)
{
    if constexpr (VISC) {
        const T tt = pr / rho, t0 = vp.t0, S = vp.suth, tr = tt / t0;
        const T mu = vp.mu0 * tr * tsqrt<T>(tr) * (t0 + S) / (tt + S);
        const T nu = tmax(T(4) / T(3), g * vp.inv_pr) * mu / rho;
        lam += T(4) * nu * s2 * ivol;
    }
    T dtc = cfl * (T(1) / ivol) / lam;
    if (sizeof(T) == 8) dtc = cfl / (ivol * lam);
    return dtc > T(0) ? dtc : T(0);   // a non-physical state stops the step at dt = 0
}
// a time step as the bits of the FP64 value, for the atomic minimum over cells
template <class T>
__device__ __forceinline__ unsigned long long dt_bits(T dtc)
{
    if constexpr (sizeof(T) == 4) return (unsigned long long)__double_as_longlong(f32_to_f64(dtc));
    else return (unsigned long long)__double_as_longlong(dtc);
}
template <class T, int NV, int P>
__device__ __forceinline__ T cell_dt(const T (&u)[P], int64_t c, const T* __restrict__ ivol,
                                          const T* __restrict__ area, const T* __restrict__ nrm, int nf, T g,
                                          T cfl, const ViscParams<T>& vp)
{
    T vel[3], a, pr;
    cell_dt_state<T, NV>(u, g, vel, a, pr);
    T lam = T(0), s2 = T(0);
    for (int f = 0; f < nf; ++f) {
        const T ar = area[c * 6 + f];
        const T t = cell_dt_face<T>(vel, a, nrm + (c * 6 + f) * 3);
        lam += t * ar;
        s2 += ar * ar;
    }
    return vp.mu0 > T(0) ? cell_dt_finish<T, true>(lam, s2, u[0], pr, ivol[c], g, cfl, vp)
                        : cell_dt_finish<T, false>(lam, s2, u[0], pr, ivol[c], g, cfl, vp);
}

// a first-order cell's face points all carry its cell mean
template <class T>
__device__ __forceinline__ void write_mean(const KParams<T>& p, int64_t c)
{
    const int nv = p.nv, P = nv == 4 ? 4 : 8, nfp = p.nfp;
    const int Q = (p.nfc[c] & 15) * nfp;
    const T* u = p.UA + c * P;
    T* fs = p.FS + c * (int64_t)p.qmax * nv;
    for (int q = 0; q < Q; ++q)
        for (int v = 0; v < nv; ++v) fs[q * nv + v] = u[v];
}

// K2: tagging of the flagged cells' face neighbourhood (class = max over the
// cell and its face neighbours), first-order for linear cells that broke the
// Harten bound, and the CWENOZ / MUSCL queues.  A block of 256 cells counts
// its queued cells with warp ballots, reserves its ranges of the two queues
// with one atomic add each on counts[0..1] (zeroed by the candidate kernel
// of the same residual) and writes its cells there in ascending order.  The
// blocks' ranges follow the order of their atomics, so the queues hold each
// class's cells in a run-dependent block order; a queued cell's
// reconstruction depends only on the cell, so the residual does not.
template <class T>
__global__ void __launch_bounds__(256) k_tag(KParams<T> p)
{
    pdl_wait();
    __shared__ int sc[2][8];
    __shared__ int base[2];
    if (p.dt_pending && blockIdx.x == 0) {
        // one warp per problem folds its slots (two per lane, loaded together)
        // and resets them; the minimum of the bits does not depend on the order
        static_assert(kDtSlots == 64, "two slots per lane");
        const int wq = threadIdx.x >> 5, lq = threadIdx.x & 31;
        for (int k = wq; k < p.nseg; k += 8) {
            const int64_t e0 = ((int64_t)k * kDtSlots + lq) * kDtStride, e1 = e0 + 32 * kDtStride;
            const unsigned long long x0 = p.dt_pending[e0], x1 = p.dt_pending[e1];
            unsigned long long m = x0 < x1 ? x0 : x1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
                m = y < m ? y : m;
            }
            p.dt_pending[e0] = 0x7ff0000000000000ull;
            p.dt_pending[e1] = 0x7ff0000000000000ull;
            if (lq == 0) p.dt_cur[k] = __longlong_as_double((long long)m);
        }
    }
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    int t = 255;
    if (c < p.nc) {
        const uint8_t r = p.raw[c];
        t = r & 3;
        if (!p.forced && p.scheme == HFV_HYBRID) {
            // the six neighbour slots in three 8-byte loads (slots past the
            // cell's faces hold -1), then the neighbours' classes together
            const int2* nb2 = reinterpret_cast<const int2*>(p.nbr + c * 6);
            const int2 a = nb2[0], b = nb2[1], d = nb2[2];
            const int32_t nbj[6] = {a.x, a.y, b.x, b.y, d.x, d.y};
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (nbj[f] >= 0) {
                    const int tj = p.raw[nbj[f]] & 3;
                    t = tj > t ? tj : t;
                }
            }
        }
        if (t == CLS_LIN && (r & HARTEN_FAIL)) t = CLS_FIRST;
        p.cls[c] = (uint8_t)t;
        if (t == CLS_FIRST) write_mean<T>(p, c);
    }
    const unsigned b1 = __ballot_sync(0xffffffffu, t == CLS_CW);
    const unsigned b2 = __ballot_sync(0xffffffffu, t == CLS_MU);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sc[0][w] = __popc(b1); sc[1][w] = __popc(b2); }
    __syncthreads();
    if (threadIdx.x < 2) {
        int sum = 0;
        for (int k = 0; k < 8; ++k) sum += sc[threadIdx.x][k];
        base[threadIdx.x] = sum ? atomicAdd(p.counts + threadIdx.x, sum) : 0;
    }
    __syncthreads();
    if (t == CLS_CW || t == CLS_MU) {
        const int q = t == CLS_CW ? 0 : 1;
        int off = base[q] + __popc((q == 0 ? b1 : b2) & ((1u << lane) - 1u));
        for (int k = 0; k < w; ++k) off += sc[q][k];
        p.queue[q * p.nc + off] = (int32_t)c;
    }
}

// K3: CWENOZ on the CWENOZ queue, one group per queued cell (Sec. 2.3).
// Lanes share the stencil gather; lane k forms coefficient k of p_opt;
// lane (f, k) forms the directional degree-1 coefficients; lane v forms the
// indicators and weights of variable v; lane q writes face point q.  With
// CHAR the variables are characteristic per face: lane f forms the face's
// eigenvectors, lane (f, w) the weights of characteristic variable w there.
template <class C, class T, bool CHAR>
__device__ __forceinline__ void cweno_part(const KParams<T>& p, unsigned bid, unsigned nbl);
template <class C, class T>
__device__ __forceinline__ void muscl_part(const KParams<T>& p, unsigned bid, unsigned nbl);

// block shape of the CWENOZ / MUSCL kernel: groups of G lanes, one cell each;
// 128 threads, or 64 / 32 where the per-cell shared arrays of the high
// orders (stencil rows, p_opt coefficients, OI, directional operators) would
// pass 46 KB of static shared memory
template <class C, class T>
struct NLShape {
    static constexpr int G = GroupSize<C::QMAX>::value;
    static constexpr int bytes(int threads)
    {
        const int cpb = threads / G, NV = C::NV, D = C::D, N = C::N, M = C::M, NF = C::NFMAX;
        const bool stage_p = (size_t)cpb * N * M * sizeof(T) <= 16384;
        const int per = M * NV + N * NV + 6 * D * NV + NF * NV * (D + 1) + 2 * NF * NV * NV + (stage_p ? N * M : 0) +
                        C::NOI + NF * D * C::MD + C::MD * NV + NV * D + D * C::MD;
        return cpb * (per * (int)sizeof(T) + 4 * ((NF * C::MD + 3) / 4));
    }
    static constexpr int THREADS = bytes(128) <= 46 * 1024 ? 128 : bytes(64) <= 46 * 1024 ? 64 : 32;
    static constexpr int CPB = THREADS / G;
    static constexpr int PPL = (C::QMAX + G - 1) / G;   // face points per lane (two on hexahedra at orders 5-6)
};

// K3 + K4 in one launch: the first `split` blocks work through the CWENOZ
// queue, the others through the MUSCL queue (no divergence between them)
template <class C, class T, bool CHAR>
__global__ void __launch_bounds__(128) k_nonlinear(KParams<T> p, unsigned split)
{
    pdl_wait();
    if (blockIdx.x < split) cweno_part<C, T, CHAR>(p, blockIdx.x, split);
    else muscl_part<C, T>(p, blockIdx.x - split, gridDim.x - split);
}

// the CWENOZ combination of one variable from its p_opt coefficients a[N]
// and directional coefficients s[nf][D]: omega_1 / lambda_1 in c0 and the
// degree-1 part sum_s (omega_s - omega_1 lambda_s / lambda_1) p_s in g[D]
//   p_1 = (p_opt - sum_s lambda_s p_s) / lambda_1, SI = a^T OI a,
//   tau = (sum_s |SI_s - SI_1| / nf)^b, w_s = lambda_s (1 + tau / (eps + SI_s))
template <class C, class T>
__device__ __forceinline__ void cweno_weights(const KParams<T>& p, const T* OI, int nf, const T (&a)[C::N],
                                              const T (&s)[6][C::D], T& c0, T (&g)[C::D])
{
    constexpr int N = C::N, D = C::D;
    const T lam1 = p.lam1, lams = (T(1) - lam1) / T(nf);
    T sumlin[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        T s0 = T(0);
#pragma unroll
        for (int f = 0; f < C::NFMAX; ++f)
            if (f < nf) s0 += s[f][k];
        sumlin[k] = s0;
    }
    T a1[N];
#pragma unroll
    for (int k = 0; k < N; ++k) a1[k] = (a[k] - (k < D ? lams * sumlin[k < D ? k : 0] : T(0))) / lam1;
    T si1 = T(0);
    {
        int o = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            T t = OI[o++] * a1[k];
#pragma unroll
            for (int l = k + 1; l < N; ++l) t += T(2) * OI[o++] * a1[l];
            si1 += a1[k] * t;
        }
    }
    T sis[C::NFMAX], tsum = T(0);
#pragma unroll
    for (int f = 0; f < C::NFMAX; ++f) {
        if (f >= nf) break;
        T s0 = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int o = k * N - k * (k - 1) / 2;
            T t = OI[o] * s[f][k];
#pragma unroll
            for (int l = k + 1; l < D; ++l) t += T(2) * OI[o + (l - k)] * s[f][l];
            s0 += s[f][k] * t;
        }
        sis[f] = s0;
        tsum += tabs(s0 - si1);
    }
    const T tau = tpow(tsum / T(nf), p.b_cw);
    const T w1 = lam1 * (T(1) + tau / (p.eps_cw + si1));
    T wsum = w1, ws[C::NFMAX];
#pragma unroll
    for (int f = 0; f < C::NFMAX; ++f) {
        if (f >= nf) break;
        ws[f] = lams * (T(1) + tau / (p.eps_cw + sis[f]));
        wsum += ws[f];
    }
    const T om1 = w1 / wsum;
    // p_cweno = (omega_1/lambda_1) p_opt + sum_s (omega_s - omega_1 lambda_s / lambda_1) p_s
    c0 = om1 / lam1;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        T gk = T(0);
#pragma unroll
        for (int f = 0; f < C::NFMAX; ++f)
            if (f < nf) gk += (ws[f] / wsum - om1 * lams / lam1) * s[f][k];
        g[k] = gk;
    }
}

// eigenvectors of the Euler flux Jacobian dF.n/dU at the conserved state u
// along the unit normal n: R columns, L = R^-1 rows, ordered u.n - c,
// entropy, shear (t; in 3D t1, t2), u.n + c.  2D t = (-n_y, n_x); 3D t1 =
// n x e_a / |n x e_a| for the axis a of the smallest |n_a|, t2 = n x t1.
template <class T, int D>
__device__ __forceinline__ void euler_eigenvectors(const T* u, const T* n, T g, T (*L)[D + 2], T (*R)[D + 2])
{
    constexpr int NV = D + 2;
    T vel[3] = {T(0), T(0), T(0)}, q2 = T(0), qn = T(0);
    const T ir = T(1) / u[0];
#pragma unroll
    for (int k = 0; k < D; ++k) { vel[k] = u[1 + k] * ir; q2 += vel[k] * vel[k]; qn += vel[k] * n[k]; }
    const T pr = (g - T(1)) * (u[D + 1] - T(0.5) * u[0] * q2);
    const T c = tsqrt<T>(g * pr * ir), H = (u[D + 1] + pr) * ir;
    T t[2][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
    if (D == 2) {
        t[0][0] = -n[1];
        t[0][1] = n[0];
    } else {
        int ax = 0;
        for (int k = 1; k < 3; ++k)
            if (tabs(n[k]) < tabs(n[ax])) ax = k;
        T e[3] = {T(0), T(0), T(0)};
        e[ax] = T(1);
        T a[3] = {n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]};
        const T an = tsqrt<T>(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int k = 0; k < 3; ++k) t[0][k] = a[k] / an;
        t[1][0] = n[1] * t[0][2] - n[2] * t[0][1];
        t[1][1] = n[2] * t[0][0] - n[0] * t[0][2];
        t[1][2] = n[0] * t[0][1] - n[1] * t[0][0];
    }
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int j = 0; j < NV; ++j) { L[i][j] = T(0); R[i][j] = T(0); }
    R[0][0] = T(1); R[0][1] = T(1); R[0][NV - 1] = T(1);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        R[1 + k][0] = vel[k] - c * n[k];
        R[1 + k][1] = vel[k];
        R[1 + k][NV - 1] = vel[k] + c * n[k];
    }
    R[D + 1][0] = H - c * qn;
    R[D + 1][1] = T(0.5) * q2;
    R[D + 1][NV - 1] = H + c * qn;
    const T b1 = (g - T(1)) / (c * c), b2 = T(0.5) * b1 * q2;
    L[0][0] = T(0.5) * (b2 + qn / c);
    L[NV - 1][0] = T(0.5) * (b2 - qn / c);
    L[1][0] = T(1) - b2;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        L[0][1 + k] = T(0.5) * (-b1 * vel[k] - n[k] / c);
        L[NV - 1][1 + k] = T(0.5) * (-b1 * vel[k] + n[k] / c);
        L[1][1 + k] = b1 * vel[k];
    }
    L[0][D + 1] = T(0.5) * b1;
    L[NV - 1][D + 1] = T(0.5) * b1;
    L[1][D + 1] = -b1;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) {
        T ut = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            R[1 + k][2 + j] = t[j][k];
            L[2 + j][1 + k] = t[j][k];
            ut += vel[k] * t[j][k];
        }
        R[D + 1][2 + j] = ut;
        L[2 + j][0] = -ut;
    }
}

template <class C, class T, bool CHAR>
__device__ __forceinline__ void cweno_part(const KParams<T>& p, unsigned bid, unsigned nbl)
{
    constexpr int M = C::M, NV = C::NV, D = C::D, NFP = C::NFP, N = C::N, MD = C::MD;
    constexpr int G = NLShape<C, T>::G, CPB = NLShape<C, T>::CPB;
    constexpr int NFC = CHAR ? C::NFMAX : 1;   // faces with their own weights
    constexpr int NVC = CHAR ? NV : 1;
    __shared__ T sU[CPB][M][NV];
    __shared__ T sA[CPB][N][NV];          // p_opt coefficients
    __shared__ T sS[CPB][6][D][NV];       // directional coefficients
    __shared__ T sC[CPB][NFC][NV][D + 1]; // per (face,) variable: omega_1 / lambda_1 and the degree-1 part
    __shared__ T sL[CPB][NFC][NVC][NV];   // characteristic projection of each face (CHAR)
    __shared__ T sR[CPB][NFC][NV][NVC];
    // the cell's operators, copied asynchronously while the stencil states
    // are gathered (P only where CPB copies of it fit in 16 KB)
    constexpr int NOI = C::NOI, NDD = C::NFMAX * D * MD, NDIR = (C::NFMAX * MD + 3) / 4;
    constexpr bool STAGE_P = (size_t)CPB * N * M * sizeof(T) <= 16384;
    __shared__ __align__(16) T sP[STAGE_P ? CPB : 1][STAGE_P ? N * M : 1];
    __shared__ T sOI[CPB][NOI];
    __shared__ T sDd[CPB][NDD];
    __shared__ uint32_t sDir[CPB][NDIR];  // directional stencil indices, four per word
    const Grp<G> grp;
    const int gi = threadIdx.x / G, lane = grp.lane;
    const int cnt = p.counts[0];
    for (int64_t i = (int64_t)bid * CPB + gi; i < cnt; i += (int64_t)nbl * CPB) {
        const int64_t c = p.queue[i];
        const int nf = p.nfc[c] & 15;
        if constexpr (STAGE_P) {
            const T* P = p.P + c * (int64_t)N * M;
            for (int e = lane; e < N * M; e += G) cp_async(&sP[gi][e], P + e);
        }
        {
            const T* O = p.OI + c * (int64_t)NOI;
            for (int e = lane; e < NOI; e += G) cp_async(&sOI[gi][e], O + e);
            const T* Dm = p.Dd + c * (int64_t)(6 * D * MD);
            for (int e = lane; e < nf * D * MD; e += G) cp_async(&sDd[gi][e], Dm + e);
            // 6 MD bytes per cell, a multiple of four
            const uint32_t* di = reinterpret_cast<const uint32_t*>(p.dir + c * 6 * MD);
            for (int e = lane; e < (nf * MD + 3) / 4; e += G) cp_async(&sDir[gi][e], di + e);
        }
        // the face points' own inputs: quadrature map and linear candidate
        constexpr int PPL = NLShape<C, T>::PPL;
        const int Q = nf * NFP;
        const int64_t q0 = c * C::QMAX;
        T ph[PPL][D], wc[PPL][NV];
#pragma unroll
        for (int j = 0; j < PPL; ++j) {
            const int q = lane + j * G;
            if (q < Q) {
#pragma unroll
                for (int k = 0; k < D; ++k) ph[j][k] = p.Phil[(q0 + q) * D + k];
                load_state<T, NV>(p.FS + (q0 + q) * NV, wc[j]);
            }
        }
        T uc[NV];
        load_cell<T, NV>(p.UA, c, uc);
        const int32_t* st = p.sten + c * M;
        for (int m = lane; m < M; m += G) {
            T uj[NV];
            load_cell<T, NV>(p.UA, st[m], uj);
#pragma unroll
            for (int v = 0; v < NV; ++v) sU[gi][m][v] = uj[v] - uc[v];
        }
        if constexpr (CHAR) {
            if (lane < nf) {
                const T* n = p.nrm + (c * 6 + lane) * 3;
                const T nn[3] = {n[0], n[1], n[2]};
                euler_eigenvectors<T, D>(uc, nn, p.gamma, sL[gi][lane], sR[gi][lane]);
            }
        }
        cp_async_wait_all();
        grp.sync();
        // p_opt: a_k = sum_m P_km (U_m - U_0)
        const T* P = p.P + c * (int64_t)N * M;
        for (int k = lane; k < N; k += G) {
            T acc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] = T(0);
            if constexpr (M <= 40) {
                T row[M];
                if constexpr (STAGE_P) load_row_smem<T, M>(&sP[gi][k * M], row);
                else load_row<T, M>(P + k * M, row);
#pragma unroll
                for (int m = 0; m < M; ++m)
#pragma unroll
                    for (int v = 0; v < NV; ++v) acc[v] += row[m] * sU[gi][m][v];
            } else {
                // long rows (orders 6-7): streamed, a row would not fit in registers
                for (int m = 0; m < M; ++m) {
                    const T pk = STAGE_P ? sP[gi][STAGE_P ? k * M + m : 0] : __ldg(P + k * M + m);
#pragma unroll
                    for (int v = 0; v < NV; ++v) acc[v] += pk * sU[gi][m][v];
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) sA[gi][k][v] = acc[v];
        }
        // directional degree-1 polynomials
        for (int t = lane; t < nf * D; t += G) {
            const int f = t / D, k = t % D;
            const uint8_t* idx = reinterpret_cast<const uint8_t*>(sDir[gi]) + f * MD;
            const T* Dm = &sDd[gi][(f * D + k) * MD];
            T acc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] = T(0);
#pragma unroll
            for (int b = 0; b < MD; ++b) {
                const T dk = Dm[b];
                const int m = idx[b];
#pragma unroll
                for (int v = 0; v < NV; ++v) acc[v] += dk * sU[gi][m][v];
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) sS[gi][f][k][v] = acc[v];
        }
        grp.sync();
        // indicators and weights: one lane per variable, or per (face,
        // characteristic variable)
        const T* OI = sOI[gi];
        for (int t = lane; t < (CHAR ? nf * NV : NV); t += G) {
            const int f = CHAR ? t / NV : 0, w = CHAR ? t % NV : t;
            T a[N], sd[6][D], c0, g[D];
#pragma unroll
            for (int k = 0; k < N; ++k) {
                if constexpr (CHAR) {
                    T x = T(0);
#pragma unroll
                    for (int u = 0; u < NV; ++u) x += sL[gi][f][w][u] * sA[gi][k][u];
                    a[k] = x;
                } else {
                    a[k] = sA[gi][k][w];
                }
            }
#pragma unroll
            for (int h = 0; h < C::NFMAX; ++h)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    sd[h][k] = T(0);
                    if (h >= nf) continue;
                    if constexpr (CHAR) {
                        T x = T(0);
#pragma unroll
                        for (int u = 0; u < NV; ++u) x += sL[gi][f][w][u] * sS[gi][h][k][u];
                        sd[h][k] = x;
                    } else {
                        sd[h][k] = sS[gi][h][k][w];
                    }
                }
            cweno_weights<C, T>(p, OI, nf, a, sd, c0, g);
            sC[gi][f][w][0] = c0;
#pragma unroll
            for (int k = 0; k < D; ++k) sC[gi][f][w][1 + k] = g[k];
        }
        grp.sync();
        bool fail = false;
        T w[PPL][NV];
        const T rb = uc[0], pb = pressure<T, D>(uc, p.gamma);
        const T rlim = p.h_theta * tmax(tabs(rb), p.h_eps), plim = p.h_theta * tmax(tabs(pb), p.h_eps);
#pragma unroll
        for (int j = 0; j < PPL; ++j) {
            const int q = lane + j * G;
            if (q >= Q) continue;
#pragma unroll
            for (int v = 0; v < NV; ++v) w[j][v] = wc[j][v];
            if constexpr (CHAR) {
                // the linear candidate's increment in the face's
                // characteristic variables, combined there, projected back
                const int f = q / NFP;
                T dl[NV], cw[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) dl[v] = w[j][v] - uc[v];
#pragma unroll
                for (int x = 0; x < NV; ++x) {
                    T d0 = T(0);
#pragma unroll
                    for (int u = 0; u < NV; ++u) d0 += sL[gi][f][x][u] * dl[u];
                    T s0 = sC[gi][f][x][0] * d0;
#pragma unroll
                    for (int k = 0; k < D; ++k) s0 += ph[j][k] * sC[gi][f][x][1 + k];
                    cw[x] = s0;
                }
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    T s0 = uc[v];
#pragma unroll
                    for (int x = 0; x < NV; ++x) s0 += sR[gi][f][v][x] * cw[x];
                    w[j][v] = s0;
                }
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    T s0 = uc[v] + sC[gi][0][v][0] * (w[j][v] - uc[v]);
#pragma unroll
                    for (int k = 0; k < D; ++k) s0 += ph[j][k] * sC[gi][0][v][1 + k];
                    w[j][v] = s0;
                }
            }
            fail = fail || !(tabs(w[j][0] - rb) <= rlim) || !(tabs(pressure<T, D>(w[j], p.gamma) - pb) <= plim);
        }
        // a cell failing the Harten bound falls back to its mean at every point
        const bool anyf = grp.any(fail);
#pragma unroll
        for (int j = 0; j < PPL; ++j) {
            const int q = lane + j * G;
            if (q >= Q) continue;
            T o[NV];   // chosen element by element: the arrays stay in registers
#pragma unroll
            for (int v = 0; v < NV; ++v) o[v] = anyf ? uc[v] : w[j][v];
            store_state<T, NV>(p.FS + (q0 + q) * NV, o);
        }
        if (anyf && lane == 0) p.cls[c] = CLS_FIRST;
        grp.sync();
    }
}

// Venkatakrishnan's smooth limiter value at one face point (d2 != 0 the
// unlimited increment, d1 the distance to the bound on its side,
// eps2 = (K dx)^3), capped at 1
template <class T>
__device__ __forceinline__ T venk_phi(T d1, T d2, T eps2)
{
    const T num = (d1 * d1 + eps2) * d2 + T(2) * d2 * d2 * d1;
    const T den = d2 * (d1 * d1 + T(2) * d2 * d2 + d1 * d2 + eps2);
    return tmin(T(1), num / den);
}
__device__ __forceinline__ float tcbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double tcbrt(double x) { return cbrt(x); }

// K4: MUSCL on the MUSCL queue (Sec. 2.2), one group per queued cell:
// degree-1 gradient from the first Md stencil cells, limiter bounds from the
// cell and its face neighbours (the first stencil layer); Barth-Jespersen, or
// Venkatakrishnan's limiter with its threshold (K dx)^3.
template <class C, class T>
__device__ __forceinline__ void muscl_part(const KParams<T>& p, unsigned bid, unsigned nbl)
{
    constexpr int M = C::M, NV = C::NV, D = C::D, NFP = C::NFP, MD = C::MD;
    constexpr int G = NLShape<C, T>::G, CPB = NLShape<C, T>::CPB;
    __shared__ T sU[CPB][MD][NV];
    __shared__ T sG[CPB][NV][D];
    __shared__ T sGm[CPB][D * MD];        // the gradient operator, copied during the gather
    const Grp<G> grp;
    const int gi = threadIdx.x / G, lane = grp.lane;
    const int64_t nc = p.nc;
    const int cnt = p.counts[1];
    for (int64_t i = (int64_t)bid * CPB + gi; i < cnt; i += (int64_t)nbl * CPB) {
        const int64_t c = p.queue[nc + i];
        const int nfv = p.nfc[c];
        const int nf = nfv & 15, n1 = nfv >> 4, Q = nf * NFP;
        {
            const T* Gsrc = p.G + c * (int64_t)D * MD;
            for (int e = lane; e < D * MD; e += G) cp_async(&sGm[gi][e], Gsrc + e);
        }
        constexpr int PPL = NLShape<C, T>::PPL;
        const int64_t q0 = c * C::QMAX;
        T ph[PPL][D];
#pragma unroll
        for (int j = 0; j < PPL; ++j)
            if (lane + j * G < Q)
#pragma unroll
                for (int k = 0; k < D; ++k) ph[j][k] = p.Phil[(q0 + lane + j * G) * D + k];
        const T ivc = p.ivol[c];
        T uc[NV];
        load_cell<T, NV>(p.UA, c, uc);
        const int32_t* st = p.sten + c * M;
        for (int m = lane; m < MD; m += G) {
            T uj[NV];
            load_cell<T, NV>(p.UA, st[m], uj);
#pragma unroll
            for (int v = 0; v < NV; ++v) sU[gi][m][v] = uj[v];
        }
        cp_async_wait_all();
        grp.sync();
        const T* Gm = sGm[gi];
        for (int t = lane; t < NV * D; t += G) {
            const int v = t / D, k = t % D;
            T acc = T(0);
#pragma unroll
            for (int b = 0; b < MD; ++b) acc += Gm[k * MD + b] * (sU[gi][b][v] - uc[v]);
            sG[gi][v][k] = acc;
        }
        grp.sync();
        T w[PPL][NV];
        T eps2 = T(0);
        if (p.limiter == 1) {
            const T vol = T(1) / ivc;
            const T dx = D == 2 ? tsqrt<T>(vol) : tcbrt(vol);
            const T kd = p.venk_k * dx;
            eps2 = kd * kd * kd;
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            T lo = uc[v], hi = uc[v];
            for (int m = 0; m < n1; ++m) {
                lo = tmin(lo, sU[gi][m][v]);
                hi = tmax(hi, sU[gi][m][v]);
            }
            T dl[PPL], t = T(1);
#pragma unroll
            for (int j = 0; j < PPL; ++j) {
                dl[j] = T(0);
                if (lane + j * G >= Q) continue;
#pragma unroll
                for (int k = 0; k < D; ++k) dl[j] += ph[j][k] * sG[gi][v][k];
                T tj = T(1);
                if (p.limiter == 1) {
                    if (dl[j] > T(0)) tj = venk_phi(hi - uc[v], dl[j], eps2);
                    else if (dl[j] < T(0)) tj = venk_phi(lo - uc[v], dl[j], eps2);
                } else {
                    if (dl[j] > T(0)) tj = tmin(T(1), (hi - uc[v]) / dl[j]);
                    else if (dl[j] < T(0)) tj = tmin(T(1), (lo - uc[v]) / dl[j]);
                }
                t = tmin(t, tj);
            }
            const T th = grp.min(t);
#pragma unroll
            for (int j = 0; j < PPL; ++j) w[j][v] = uc[v] + th * dl[j];
        }
        bool fail = false;
        const T rb = uc[0], pb = pressure<T, D>(uc, p.gamma);
        const T rlim = p.h_theta * tmax(tabs(rb), p.h_eps), plim = p.h_theta * tmax(tabs(pb), p.h_eps);
#pragma unroll
        for (int j = 0; j < PPL; ++j)
            if (lane + j * G < Q)
                fail = fail || !(tabs(w[j][0] - rb) <= rlim) || !(tabs(pressure<T, D>(w[j], p.gamma) - pb) <= plim);
        // a cell failing the Harten bound falls back to its mean at every point
        const bool anyf = grp.any(fail);
#pragma unroll
        for (int j = 0; j < PPL; ++j) {
            const int q = lane + j * G;
            if (q >= Q) continue;
            T o[NV];   // chosen element by element: the arrays stay in registers
#pragma unroll
            for (int v = 0; v < NV; ++v) o[v] = anyf ? uc[v] : w[j][v];
            store_state<T, NV>(p.FS + (q0 + q) * NV, o);
        }
        if (anyf && lane == 0) p.cls[c] = CLS_FIRST;
        grp.sync();
    }
}

// exponents of the monomial basis psi_k = xi^a eta^b zeta^c, 1 <= a+b+c <= R,
// in the order of the operator setup (total degree, then a, then b, falling)
template <int D, int R>
struct MonoExp {
    int e[cK(R, D) - 1][3];
    constexpr MonoExp() : e{}
    {
        int k = 0;
        for (int deg = 1; deg <= R; ++deg)
            for (int ea = deg; ea >= 0; --ea) {
                if (D == 2) {
                    e[k][0] = ea; e[k][1] = deg - ea; e[k][2] = 0; ++k;
                } else {
                    for (int eb = deg - ea; eb >= 0; --eb) { e[k][0] = ea; e[k][1] = eb; e[k][2] = deg - ea - eb; ++k; }
                }
            }
    }
};

// Viscous gradients (Sec. 2: the gradients of the viscous flux come from the
// constrained least-squares reconstruction), one group per cell, every cell:
// a = P (U_m - U_0) as for p_opt, then at each face point the gradient in
// physical coordinates of the unlimited polynomial, sum_k a_k J^-T
// grad_xi psi_k(xi_q) (xi_q = Phi_lin + mean(xi); the subtracted means do not
// change a gradient), and the chain rule to the velocity and temperature
// gradients at the cell's final face-point state U_L (in FS: this kernel runs
// after the CWENOZ / MUSCL kernel and the Harten bound, just before the
// fluxes), the state that also enters the convective flux.
template <class C, class T>
__global__ void __launch_bounds__(128) k_grad(KParams<T> p)
{
    constexpr int M = C::M, NV = C::NV, D = C::D, N = C::N, NFP = C::NFP, R = C::R;
    constexpr int G = GroupSize<C::QMAX>::value, CPB = 128 / G, NGR = (D + 1) * D, NVX = D + D * D;
    constexpr MonoExp<D, R> EX{};
    __shared__ T sU[CPB][M][NV];
    __shared__ T sA[CPB][N][NV];
    const Grp<G> grp;
    const int gi = threadIdx.x / G, lane = grp.lane;
    const int64_t c = (int64_t)blockIdx.x * CPB + gi;
    pdl_wait();
    if (c >= p.nc) return;   // a whole group leaves; only group-masked collectives follow
    T uc[NV];
    load_cell<T, NV>(p.UA, c, uc);
    const int32_t* st = p.sten + c * M;
    for (int m = lane; m < M; m += G) {
        T uj[NV];
        load_cell<T, NV>(p.UA, st[m], uj);
#pragma unroll
        for (int v = 0; v < NV; ++v) sU[gi][m][v] = uj[v] - uc[v];
    }
    grp.sync();
    const T* P = p.P + c * (int64_t)N * M;
    for (int k = lane; k < N; k += G) {
        T acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = T(0);
        for (int m = 0; m < M; ++m) {
            const T pk = __ldg(P + k * M + m);
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += pk * sU[gi][m][v];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) sA[gi][k][v] = acc[v];
    }
    grp.sync();
    const int Q = (p.nfc[c] & 15) * NFP;
    const T* vx = p.VX + c * NVX;
    T Ji[D][D];
#pragma unroll
    for (int b = 0; b < D; ++b)
#pragma unroll
        for (int j = 0; j < D; ++j) Ji[b][j] = vx[D + b * D + j];
    const T g = p.gamma;
    for (int q = lane; q < Q; q += G) {
        const int64_t qi = c * C::QMAX + q;
        T pw[D][R + 1];
#pragma unroll
        for (int b = 0; b < D; ++b) {
            const T x = p.Phil[qi * D + b] + vx[b];
            pw[b][0] = T(1);
#pragma unroll
            for (int e = 1; e <= R; ++e) pw[b][e] = pw[b][e - 1] * x;
        }
        T gc[NV][D];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int j = 0; j < D; ++j) gc[v][j] = T(0);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            T dx[D];
#pragma unroll
            for (int j = 0; j < D; ++j) dx[j] = T(0);
#pragma unroll
            for (int b = 0; b < D; ++b) {
                const int eb = EX.e[k][b];
                if (eb == 0) continue;
                T dpsi = T(eb) * pw[b][eb - 1];
#pragma unroll
                for (int a = 0; a < D; ++a)
                    if (a != b) dpsi *= pw[a][EX.e[k][a]];
#pragma unroll
                for (int j = 0; j < D; ++j) dx[j] += Ji[b][j] * dpsi;
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const T ak = sA[gi][k][v];
#pragma unroll
                for (int j = 0; j < D; ++j) gc[v][j] += ak * dx[j];
            }
        }
        T w[NV];
        load_state<T, NV>(p.FS + qi * NV, w);
        const T ir = T(1) / w[0];
        T u[D], u2 = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) { u[k] = w[1 + k] * ir; u2 += u[k] * u[k]; }
        const T tt = (g - T(1)) * (w[D + 1] - T(0.5) * w[0] * u2) * ir;
        T* out = p.GS + qi * NGR;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            // grad u_k = (grad m_k - u_k grad rho) / rho
#pragma unroll
            for (int k = 0; k < D; ++k) out[k * D + j] = (gc[1 + k][j] - u[k] * gc[0][j]) * ir;
            // grad p = (g - 1)(grad E - sum_k u_k grad m_k + |u|^2 / 2 grad rho),
            // grad T = (grad p - T grad rho) / rho
            T gp = gc[D + 1][j] + T(0.5) * u2 * gc[0][j];
#pragma unroll
            for (int k = 0; k < D; ++k) gp -= u[k] * gc[1 + k][j];
            out[D * D + j] = ((g - T(1)) * gp - tt * gc[0][j]) * ir;
        }
    }
}

// K6: Riemann fluxes at the face points and the residual, a group of FG
// lanes per cell, lane f taking the NFP points of face f (they share the
// face's normal and neighbour offset and lie next to each other in FS, on
// both sides of the face).  Both sides' states come from FS (a first-order
// cell carries its mean there).  The lanes' point sums are added in a fixed
// butterfly; lanes v, v + FG, ... < nv finish variable v, with the
// Runge-Kutta stage fused when one is given.  Every lane of the warp reaches
// the shuffles (cells past the end carry no faces), so they take the full
// mask.
// resident blocks per SM aimed for: 2D FP32 ten (48 registers, measured
// 5 % faster than 54), 3D FP32 nine (56), FP64 four (128)
template <class C, class T>
struct FluxShape {
    static constexpr int FG = C::NFMAX <= 4 ? 4 : 8;
    static constexpr int CPB = 128 / FG;
    // 2D FP32 with at most two points per face: every face point's states
    // are loaded before the first Riemann solve (PRE), at eight blocks per
    // SM (64 registers); 5 % faster per step on the quadrant than ten
    // blocks with point-by-point loads
    static constexpr bool PRE = sizeof(T) == 4 && C::D == 2 && C::NFP <= 2;
    static constexpr int MINB = sizeof(T) == 8 ? 4 : C::D == 2 ? (PRE ? 8 : 10) : 9;
};

template <class C, class T, int KIND, bool VISC = false, bool CHAIN = false>
__global__ void __launch_bounds__(128, FluxShape<C, T>::MINB) k_flux(KParams<T> p, T* __restrict__ R)
{
    constexpr int NV = C::NV, D = C::D, NFP = C::NFP, G = FluxShape<C, T>::FG, CPB = FluxShape<C, T>::CPB;
    const int lane = threadIdx.x & (G - 1);
    const int64_t nc = p.nc;
    const int64_t c = (int64_t)blockIdx.x * CPB + threadIdx.x / G;
    const bool valid = c < nc;
    const int64_t cs = valid ? c : nc - 1;
    const int f = lane;
    int32_t nb = -2;
    T nn[3] = {T(0), T(0), T(0)};
    if (valid && f < C::NFMAX) {
        nb = p.nfs[cs * 6 + f];
        const T* n = p.nrm + (cs * 6 + f) * 3;
        nn[0] = n[0]; nn[1] = n[1]; nn[2] = n[2];
    }
    // the Runge-Kutta operands (independent of the fluxes)
    constexpr int NVL = (NV + G - 1) / G;   // variables finished per lane
    constexpr bool F32 = sizeof(T) == 4;
    const bool rk = p.rk_mode & 1, rk_a = p.rk_mode & 2;
    double u0[NVL], us[NVL], cdt = 0.0;
    float cdtf = 0.0f;
#pragma unroll
    for (int k = 0; k < NVL; ++k) {
        u0[k] = 0.0; us[k] = 0.0;
        const int v = lane + k * G;
        if (valid && rk && v < NV) {
            us[k] = p.Us[(int64_t)v * nc + c];
            if (rk_a) u0[k] = p.U0[(int64_t)v * nc + c];
        }
    }
    if (valid && rk) {
        const double dtk = p.dt[p.seg ? p.seg[c] : 0];
        if constexpr (F32) cdtf = p.rk_bw * f64_to_f32(dtk);
        else cdt = p.rk_w * dtk;
    }
    const T ivol = valid ? p.ivol[cs] : T(0);
    T linv = T(0);
    if (VISC && valid && f < C::NFMAX) linv = p.LINV[cs * 6 + f];
    // quadrature weights x face area (constant): ahead of the wait where
    // every face point is preloaded
    constexpr bool PRE = FluxShape<C, T>::PRE && !VISC;
    T wqa[PRE ? NFP : 1];
    if constexpr (PRE) {
#pragma unroll
        for (int a = 0; a < NFP; ++a) wqa[a] = nb != -2 ? p.W[cs * C::QMAX + f * NFP + a] : T(0);
    }
    // the chained time step's geometry, loaded here: after the state stores
    // below the compiler could not move these loads ahead of them, and each
    // block would wait on two more memory round trips at its end
    T af = T(0);
    int dseg = 0;   // the problem the atomic goes to, or -1 - the cell's problem when the warp spans two
    if constexpr (CHAIN) {
        if (nb != -2) af = p.areaT[cs * 6 + f];
        if (p.seg) {
            constexpr int CPW = 32 / G;
            const int64_t w0 = min((int64_t)blockIdx.x * CPB + (threadIdx.x >> 5) * CPW, nc - 1);
            const int64_t w1 = min(w0 + (int64_t)CPW, nc) - 1;
            dseg = p.seg[w0];
            if (p.seg[w1] != dseg) dseg = -1 - p.seg[cs];
        }
    }
    // geometry and the stage operands above are constant or written two or
    // more kernels back; the face states are the predecessor's output
    pdl_wait();
    T acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = T(0);
    if (nb != -2) {
        const int64_t q = cs * C::QMAX + f * NFP;
        constexpr int NP = PRE ? NFP : 1;
        T WL[NP][NV], WR[NP][NV];
        if constexpr (PRE) {
#pragma unroll
            for (int a = 0; a < NFP; ++a) {
                // an open boundary's outside state is the inside one: the
                // same load again (branch-free)
                load_state<T, NV>(p.FS + (q + a) * NV, WL[a]);
                load_state<T, NV>(p.FS + (nb < 0 ? q + a : (int64_t)nb + a) * NV, WR[a]);
            }
        }
#pragma unroll
        for (int a = 0; a < NFP; ++a) {
            T wl[NV], wr[NV], F[NV];
            if constexpr (PRE) {
#pragma unroll
                for (int v = 0; v < NV; ++v) { wl[v] = WL[a][v]; wr[v] = WR[a][v]; }
            } else {
                load_state<T, NV>(p.FS + (q + a) * NV, wl);
                if (nb < 0) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) wr[v] = wl[v];
                } else {
                    load_state<T, NV>(p.FS + ((int64_t)nb + a) * NV, wr);
                }
            }
            T wq;
            if constexpr (PRE) wq = wqa[a];
            else wq = p.W[q + a];
            riemann<T, D, KIND>(wl, wr, nn, p.gamma, F);
            if constexpr (VISC) {
                // minus the viscous flux (eq. EulerEquationsDetails); an open
                // boundary's outside copies the inside gradient
                constexpr int NGR = (D + 1) * D;
                T gl[NGR], gr[NGR], Fv[NV];
                const T* pl = p.GS + (q + a) * NGR;
                const T* pr = nb < 0 ? pl : p.GS + ((int64_t)nb + a) * NGR;
#pragma unroll
                for (int e = 0; e < NGR; ++e) { gl[e] = pl[e]; gr[e] = pr[e]; }
                viscous_flux<T, D>(wl, wr, gl, gr, nn, linv, p.gamma, p.vp, Fv);
#pragma unroll
                for (int v = 0; v < NV; ++v) F[v] -= Fv[v];
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += F[v] * wq;
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
    T xs[NVL];   // the new state in the residual's precision (the next stage's copy)
#pragma unroll
    for (int k = 0; k < NVL; ++k) {
        xs[k] = T(0);
        const int v = lane + k * G;
        if (!valid || v >= NV) continue;
        T val = acc[0];
#pragma unroll
        for (int x = 1; x < NV; ++x) val = v == x ? acc[x] : val;
        const T r = -val * ivol;
        const int64_t e = (int64_t)v * nc + c;
        if (!rk) {
            R[e] = r;
        } else {
            // Runge-Kutta stage update of variable v of cell c into the FP64 state
            double x;
            if constexpr (F32) {
                x = fma(p.rk_b, us[k], f32_to_f64(cdtf * r));
                if (rk_a) x = fma(p.rk_a, u0[k], x);
                xs[k] = f64_to_f32(x);
            } else {
                x = p.rk_b * (us[k] + cdt * (double)r);
                if (rk_a) x += p.rk_a * u0[k];
                xs[k] = x;
            }
            if (p.Rcopy) p.Rcopy[e] = r;
            p.out[e] = x;
            if (p.ua_next) p.ua_next[c * AoSP<NV>::P + v] = xs[k];
        }
    }
    if constexpr (CHAIN) {
        // chained steps (the last stage's launch): the next step's time step
        // from the new state; a warp inside one problem reduces first, a warp
        // across a boundary takes one atomic per cell
        constexpr int P = AoSP<NV>::P;
        const int base = (threadIdx.x & 31) & ~(G - 1);
        T u[P];
#pragma unroll
        for (int v = 0; v < P; ++v) u[v] = T(0);
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = __shfl_sync(0xffffffffu, xs[v / G], base + v % G);
        // every lane holds the new state; lane f takes face f's term with the
        // normal it already has, the first lane sums them in face order
        T vel[3], a, pr;
        cell_dt_state<T, NV>(u, p.gamma, vel, a, pr);
        T tf = T(0);
        if (nb != -2) tf = cell_dt_face<T>(vel, a, nn);
        // a lane past the cell's faces holds tf = af = 0: its term adds an
        // exact zero, so the sums equal those over the cell's own faces
        T lam = T(0), s2 = T(0);
#pragma unroll
        for (int h = 0; h < C::NFMAX; ++h) {
            const T th = __shfl_sync(0xffffffffu, tf, base + h), ah = __shfl_sync(0xffffffffu, af, base + h);
            lam += th * ah;
            s2 += ah * ah;
        }
        T dtc = T(INFINITY);
        if (valid && lane == 0) dtc = cell_dt_finish<T, false>(lam, s2, u[0], pr, ivol, p.gamma, p.cfl, p.vp);
        constexpr int CPW = 32 / G;   // cells per warp
        const int64_t w0 = (int64_t)blockIdx.x * CPB + (threadIdx.x >> 5) * CPW;
        const int slot = (blockIdx.x * 4 + (threadIdx.x >> 5)) & (kDtSlots - 1);
        if (w0 < nc) {
            if (dseg < 0) {
                if (valid && lane == 0)
                    atomicMin(p.dt_next + ((int64_t)(-1 - dseg) * kDtSlots + slot) * kDtStride, dt_bits(dtc));
            } else {
#pragma unroll
                for (int o = 16; o >= G; o >>= 1) dtc = tmin(dtc, __shfl_xor_sync(0xffffffffu, dtc, o));
                if ((threadIdx.x & 31) == 0)
                    atomicMin(p.dt_next + ((int64_t)dseg * kDtSlots + slot) * kDtStride, dt_bits(dtc));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host launch
// ---------------------------------------------------------------------------

#define HFV_CUDA_CHECK(x)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (x);                                                                  \
        if (e_ != cudaSuccess) {                                                               \
            set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x);             \
            return HFV_ERR_CUDA;                                                               \
        }                                                                                      \
    } while (0)

// Launch with programmatic stream serialization: the kernel may be scheduled
// while its predecessor drains and waits for it in pdl_wait() (every kernel
// launched this way calls it before touching the predecessor's output).
constexpr int kPdl = 1;
template <class... KA, class... A>
static void pdl(void (*k)(KA...), unsigned grid, unsigned block, size_t smem, cudaStream_t st, A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = kPdl;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// the viscous constants in the residual's precision
template <class T>
ViscParams<T> visc_params(const hfv_scheme* s)
{
    ViscParams<T> vp;
    vp.mu0 = (T)s->p.mu0;
    vp.t0 = (T)s->p.t0;
    vp.suth = (T)s->p.sutherland_s;
    vp.inv_pr = (T)(1.0 / s->p.prandtl);
    vp.alpha = (T)s->p.visc_alpha;
    return vp;
}

template <class T>
KParams<T> make_params(hfv_scheme* s, const uint8_t* forced)
{
    const hfv_dev_arrays& a = s->a;
    KParams<T> p;
    p.nc = s->mesh->nc;
    p.scheme = s->p.scheme;
    p.nad_vars = s->p.nad_vars;
    p.forced = forced != nullptr;
    p.forced_cls = forced;
    p.sten = a.sten; p.nbr = a.nbr; p.nbrf = a.nbrf; p.nfc = a.nfc; p.qoff = a.qoff; p.loff = a.loff; p.dir = a.dir;
    p.L = (const T*)a.L; p.P = (const T*)a.P; p.Phil = (const T*)a.Phil; p.OI = (const T*)a.OI;
    p.Dd = (const T*)a.D; p.G = (const T*)a.G; p.W = (const T*)a.W; p.nrm = (const T*)a.nrm;
    p.ivol = (const T*)a.ivol; p.dxthr = (const T*)a.dxthr;
    p.UA = (const T*)a.UA;
    p.nfs = a.nfs;
    p.nv = s->nv;
    p.nfp = s->nfp;
    p.qmax = s->nfmax * s->nfp;
    p.FS = (T*)a.FS; p.raw = a.raw; p.cls = a.cls; p.queue = a.queue; p.counts = a.counts;
    p.status = a.status;
    p.gamma = (T)s->p.gamma; p.alpha_m = (T)s->p.alpha_m; p.beta_m = (T)s->p.beta_m;
    p.alpha_w = (T)s->p.alpha_w; p.beta_w = (T)s->p.beta_w;
    p.lam1 = (T)(1.0 - 1.0 / s->p.lambda1_prime);
    p.eps_cw = (T)s->p.cweno_eps; p.b_cw = (T)s->p.cweno_b;
    p.h_theta = (T)s->p.harten_theta; p.h_eps = (T)s->p.harten_eps;
    p.limiter = s->p.limiter;
    p.venk_k = (T)s->p.venkat_k;
    p.VX = (const T*)a.VX;
    p.LINV = (const T*)a.LINV;
    p.GS = (T*)a.GS;
    p.vp = visc_params<T>(s);
    p.wait_ns = s->wait_ns;
    p.withhold_copies = s->withhold_copies;
    p.dt_next = nullptr;
    p.dt_pending = nullptr;
    p.dt_cur = a.dt;
    p.areaT = (const T*)a.areaT;
    p.cfl = T(0);
    p.rk_mode = 0;
    p.rk_bw = 0.0f;
    p.nseg = s->nseg;
    return p;
}

// structure-of-arrays state -> cell-major rows of the stage state
template <class Tin, class T, int NV>
__global__ void k_to_aos(int64_t nc, const Tin* __restrict__ U, T* __restrict__ UA)
{
    pdl_wait();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    constexpr int P = AoSP<NV>::P;
    T u[P];
#pragma unroll
    for (int v = 0; v < P; ++v) u[v] = v < NV ? (T)U[v * nc + c] : T(0);
    T* q = UA + c * P;
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int v = 0; v < P; v += 4) *reinterpret_cast<float4*>(q + v) = make_float4(u[v], u[v + 1], u[v + 2], u[v + 3]);
    } else {
#pragma unroll
        for (int v = 0; v < P; v += 2) *reinterpret_cast<double2*>(q + v) = make_double2(u[v], u[v + 1]);
    }
}

// fused Runge-Kutta stage applied in the flux kernel's epilogue (see KParams)
struct StageRK {
    double a = 0.0, b = 0.0;
    double w = 1.0;           // the stage's step c = w dt
    const double* U0 = nullptr;
    const double* Us = nullptr;
    double* out = nullptr;
    void* ua_next = nullptr;
    bool keep_R = false;      // also store R (into Rs)
    // chained steps: reduce the next step's time step into dt_next (last stage,
    // with cfl), or move dt_pending into the current step's (first stage)
    unsigned long long* dt_next = nullptr;
    unsigned long long* dt_pending = nullptr;
    double cfl = 0.0;
};

// the persistent candidate kernel in tile shape WIDE: one CTA per (SM x
// resident CTAs), fewer if the tuned count says so
template <class C, class T, bool WIDE>
static int launch_linear(hfv_scheme* s, const KParams<T>& p, cudaStream_t st)
{
    using S1 = K1Shape<C, T, WIDE>;
    static int sms = 0, per_max = 0;   // per instantiation: SMs and resident CTAs per SM
    if (!sms) {
        HFV_CUDA_CHECK(cudaFuncSetAttribute(k_linear<C, T, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, S1::SMEM));
        int dev = 0, n = 0, per = 0;
        HFV_CUDA_CHECK(cudaGetDevice(&dev));
        HFV_CUDA_CHECK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        HFV_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_linear<C, T, WIDE>, S1::THREADS, S1::SMEM));
        per_max = per > 0 ? per : 1;
        sms = n;
    }
    s->sms = sms;
    s->linear_per_sm_max = per_max;
    const int per = s->tune_linear_per_sm > 0 ? std::min(s->tune_linear_per_sm, per_max) : per_max;
    const int64_t ntiles = (p.nc + S1::NG - 1) / S1::NG;
    const unsigned g1 = (unsigned)std::min<int64_t>(ntiles, (int64_t)sms * per);
    Launch l(s, KID_LINEAR, st);
    pdl(k_linear<C, T, WIDE>, g1, S1::THREADS, S1::SMEM, st, p);
    return HFV_OK;
}

template <class C, class T>
int run_residual(hfv_scheme* s, const T* U, T* R, const uint8_t* forced, uint8_t* cls_out, cudaStream_t st,
                 const T* ua, const StageRK* rk)
{
    KParams<T> p = make_params<T>(s, forced);
    const int64_t nc = p.nc;
    constexpr int CPB = 128 / GroupSize<C::QMAX>::value;
    const unsigned g256 = (unsigned)((nc + 255) / 256);
    if (!ua) {
        Launch l(s, KID_CVT, st);
        pdl(k_to_aos<T, T, C::NV>, g256, 256, 0, st, nc, U, (T*)s->a.UA);
        ua = (const T*)s->a.UA;
    }
    p.UA = ua;
    if (rk) {
        p.rk_a = rk->a; p.rk_b = rk->b; p.U0 = rk->U0; p.Us = rk->Us; p.seg = s->a.seg;
        p.dt = s->a.dt;
        p.rk_w = rk->w;
        p.rk_bw = (float)(rk->b * rk->w);
        p.rk_mode = (rk->b != 0.0 ? 1 : 0) | (rk->a != 0.0 ? 2 : 0);
        p.out = rk->out; p.ua_next = (T*)rk->ua_next;
        p.Rcopy = rk->keep_R ? (T*)s->a.Rs : nullptr;
        p.dt_next = rk->dt_next;
        p.dt_pending = rk->dt_pending;
        p.cfl = (T)rk->cfl;
    } else {
        p.rk_a = 0.0; p.rk_b = 0.0; p.rk_w = 0.0; p.rk_bw = 0.0f; p.rk_mode = 0;
        p.U0 = nullptr; p.Us = nullptr; p.dt = nullptr;
        p.seg = nullptr; p.out = nullptr; p.ua_next = nullptr; p.Rcopy = nullptr;
    }
    {
        // the candidate kernel in the scheme's tile shape (2D FP32 orders 2-3
        // have two, hfv_autotune picks one)
        constexpr bool ALT = K1Shape<C, T>::HAS_WIDE;
        s->linear_tiles = ALT ? 2 : 1;
        int rc1;
        if (ALT && s->tune_linear_tile == 1) rc1 = launch_linear<C, T, ALT>(s, p, st);
        else rc1 = launch_linear<C, T, false>(s, p, st);
        if (rc1 != HFV_OK) return rc1;
    }
    const bool visc = s->p.mu0 > 0.0;
    { Launch l(s, KID_TAG, st); pdl(k_tag<T>, s->nblocks, 256, 0, st, p); }
    {
        // CWENOZ cells cost several times a MUSCL cell: by default 3/4 of the
        // blocks take the CWENOZ queue
        using NL = NLShape<C, T>;
        const unsigned gq = (unsigned)std::max<int64_t>(
            2, std::min<int64_t>((nc + NL::CPB - 1) / NL::CPB, (int64_t)s->sms * s->tune_nl_per_sm * (128 / NL::THREADS)));
        const unsigned split = std::min<unsigned>(gq - 1, std::max<unsigned>(1, gq * s->tune_nl_cweno_pct / 100));
        Launch l(s, KID_CWENO, st);
        if (s->p.cweno_vars == HFV_CHARACTERISTIC) pdl(k_nonlinear<C, T, true>, gq, NL::THREADS, 0, st, p, split);
        else pdl(k_nonlinear<C, T, false>, gq, NL::THREADS, 0, st, p, split);
    }
    if (visc) {
        Launch l(s, KID_GRAD, st);
        pdl(k_grad<C, T>, (unsigned)((nc + CPB - 1) / CPB), 128, 0, st, p);
    }
    {
        Launch l(s, KID_FLUX, st);
        const unsigned gf = (unsigned)((nc + FluxShape<C, T>::CPB - 1) / FluxShape<C, T>::CPB);
        switch (s->p.flux + (visc ? 3 : p.dt_next ? 6 : 0)) {
        case HFV_RUSANOV: pdl(k_flux<C, T, kRusanov>, gf, 128, 0, st, p, R); break;
        case HFV_HLL: pdl(k_flux<C, T, kHLL>, gf, 128, 0, st, p, R); break;
        case HFV_HLLC: pdl(k_flux<C, T, kHLLC>, gf, 128, 0, st, p, R); break;
        case 3 + HFV_RUSANOV: pdl(k_flux<C, T, kRusanov, true>, gf, 128, 0, st, p, R); break;
        case 3 + HFV_HLL: pdl(k_flux<C, T, kHLL, true>, gf, 128, 0, st, p, R); break;
        case 3 + HFV_HLLC: pdl(k_flux<C, T, kHLLC, true>, gf, 128, 0, st, p, R); break;
        case 6 + HFV_RUSANOV: pdl(k_flux<C, T, kRusanov, false, true>, gf, 128, 0, st, p, R); break;
        case 6 + HFV_HLL: pdl(k_flux<C, T, kHLL, false, true>, gf, 128, 0, st, p, R); break;
        default: pdl(k_flux<C, T, kHLLC, false, true>, gf, 128, 0, st, p, R); break;
        }
    }
    if (cls_out) HFV_CUDA_CHECK(cudaMemcpyAsync(cls_out, s->a.cls, nc, cudaMemcpyDeviceToDevice, st));
    HFV_CUDA_CHECK(cudaGetLastError());
    return HFV_OK;
}

}  // namespace hfv
