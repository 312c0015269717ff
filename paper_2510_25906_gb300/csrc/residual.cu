// residual.cu -- the hot path: one residual evaluation R(U) of the hybrid
// scheme (Sec. 2.5) and the SSP-RK3 stage updates.
//
//   K1 k_linear   all cells: stencil gather, linear candidate at the face
//                 points (U_0 + L (U_m - U_0), Sec. 2.1), detector raw class
//                 (eqs. DMP, NADMUSCL, NADCWENOZ, marginm, marginw,
//                 NADDeactivatedCriteria), Harten test of the candidate
//   K2 k_tag      class of a cell = max over itself and its face neighbours
//                 (tagging of the flagged cells' neighbourhood); linear cells
//                 that fail the Harten bound become first-order
//      k_count / k_scan / k_scatter: warp-ballot compaction of the CWENOZ and
//                 MUSCL cells into two queues in ascending cell order
//   K3 k_cweno    CWENOZ on the CWENOZ queue (Sec. 2.3)
//   K4 k_muscl    MUSCL + Barth-Jespersen on the MUSCL queue (Sec. 2.2)
//      (both apply the Harten bound, eq. harten_jump_fix)
//   K6 k_flux     Riemann fluxes at every face point, summed per cell
//                 (eq. EulerEquationsDetails); cell-centred, atomic-free
#include <cuda_runtime.h>

#include <cstdio>

#include "hfv_internal.h"
#include "kernels.cuh"

namespace hfv {

template <class T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }
template <class T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <class T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

__device__ __forceinline__ float tpow(float x, float e) { return powf(x, e); }
__device__ __forceinline__ double tpow(double x, double e) { return pow(x, e); }

// detector quantity of kind k: 0 density, 1 pressure, 2.. conserved variable k-1
template <class T, int D>
__device__ __forceinline__ T nad_value(const T* u, int k, T g)
{
    if (k == 0) return u[0];
    if (k == 1) return pressure<T, D>(u, g);
    return u[k - 1];
}

template <class C, class T>
__global__ void __launch_bounds__(128) k_linear(KParams<T> p, const T* __restrict__ U)
{
    constexpr int M = C::M, NV = C::NV, D = C::D, NFP = C::NFP;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.nc) return;
    const int64_t nc = p.nc;
    T uc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) uc[v] = U[v * nc + c];
    {
        T pc = pressure<T, D>(uc, p.gamma);
        bool bad = !(uc[0] > T(0)) || !(pc > T(0));
#pragma unroll
        for (int v = 0; v < NV; ++v) bad |= !isfinite(uc[v]);
        if (bad) atomicOr(p.status, 1);
    }
    T du[M][NV];
    const int32_t* st = p.sten + c * M;
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        int64_t j = st[m];
#pragma unroll
        for (int v = 0; v < NV; ++v) du[m][v] = U[v * nc + j] - uc[v];
    }
    const int nf = p.nfc[c];
    const int Q = nf * NFP;
    const int64_t q0 = p.qoff[c];
    const T* L = p.L + q0 * M;

    // detector bounds over the cell and its face neighbours
    const bool detect = !p.forced && p.scheme == HFV_HYBRID;
    constexpr int KMAX = NV + 1;
    T mn[KMAX], mx[KMAX], dm[KMAX], dw[KMAX];
    bool on[KMAX];
    int nk = 0;
    int kinds[KMAX];
    if (detect) {
        if (p.nad_vars & 1) kinds[nk++] = 0;
        if (p.nad_vars & 2) kinds[nk++] = 1;
        if (p.nad_vars & 4)
            for (int v = 1; v < NV; ++v) kinds[nk++] = v + 1;
        const T thr = p.dxthr[c];
        for (int a = 0; a < nk; ++a) {
            T qi = nad_value<T, D>(uc, kinds[a], p.gamma);
            T lo = qi, hi = qi, dlo = T(0), dhi = T(0);
            int nn = 0;
            for (int f = 0; f < nf; ++f) {
                int64_t j = p.nbr[c * 6 + f];
                if (j < 0) continue;
                T uj[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) uj[v] = U[v * nc + j];
                T qj = nad_value<T, D>(uj, kinds[a], p.gamma);
                lo = tmin(lo, qj);
                hi = tmax(hi, qj);
                T dd = tabs(qj - qi);
                if (nn == 0) { dlo = dd; dhi = dd; }
                else { dlo = tmin(dlo, dd); dhi = tmax(dhi, dd); }
                ++nn;
            }
            on[a] = nn > 0 && !(dhi - dlo < thr);
            T range = hi - lo;
            mn[a] = lo;
            mx[a] = hi;
            dm[a] = tmax(p.alpha_m, p.beta_m * range);
            T sg = p.beta_w > T(0) ? T(1) : (p.beta_w < T(0) ? T(-1) : T(0));
            dw[a] = sg * tmax(p.alpha_w, tabs(p.beta_w * range));
        }
    }
    const T rb = uc[0], pb = pressure<T, D>(uc, p.gamma);
    const T rlim = p.h_theta * tmax(tabs(rb), p.h_eps), plim = p.h_theta * tmax(tabs(pb), p.h_eps);
    int cl = CLS_LIN;
    bool hfail = false;
    T* FS = p.FS + q0 * NV;
    for (int q = 0; q < Q; ++q) {
        T w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = uc[v];
#pragma unroll 4
        for (int m = 0; m < M; ++m) {
            T l = L[(int64_t)m * Q + q];
#pragma unroll
            for (int v = 0; v < NV; ++v) w[v] += l * du[m][v];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) FS[q * NV + v] = w[v];
        for (int a = 0; a < nk; ++a) {
            if (!on[a]) continue;
            T x = nad_value<T, D>(w, kinds[a], p.gamma);
            int k;
            if (x <= mn[a] - dm[a] || x >= mx[a] + dm[a]) k = CLS_MU;
            else if (mn[a] - dw[a] < x && x < mx[a] + dw[a]) k = CLS_LIN;
            else k = CLS_CW;
            cl = k > cl ? k : cl;
        }
        T pw = pressure<T, D>(w, p.gamma);
        if (!(tabs(w[0] - rb) <= rlim) || !(tabs(pw - pb) <= plim)) hfail = true;
    }
    uint8_t out;
    if (p.forced) out = p.forced_cls[c];
    else if (p.scheme == HFV_HYBRID) out = (uint8_t)cl;
    else out = p.scheme == HFV_PURE_LINEAR ? CLS_LIN : p.scheme == HFV_PURE_CWENOZ ? CLS_CW : CLS_MU;
    p.raw[c] = out | (hfail ? HARTEN_FAIL : 0);
}

template <class T>
__global__ void k_tag(KParams<T> p)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.nc) return;
    uint8_t r = p.raw[c];
    int t = r & 3;
    if (!p.forced && p.scheme == HFV_HYBRID) {
        int nf = p.nfc[c];
        for (int f = 0; f < nf; ++f) {
            int64_t j = p.nbr[c * 6 + f];
            if (j >= 0) {
                int tj = p.raw[j] & 3;
                t = tj > t ? tj : t;
            }
        }
    }
    if (t == CLS_LIN && (r & HARTEN_FAIL)) t = CLS_FIRST;
    p.cls[c] = (uint8_t)t;
}

// per-block counts of CWENOZ / MUSCL cells (blocks of 256 cells)
__global__ void __launch_bounds__(256) k_count(const uint8_t* __restrict__ cls, int64_t nc, int32_t* bcount, int nblocks)
{
    __shared__ int s[2][8];
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    int t = c < nc ? cls[c] : 255;
    unsigned b1 = __ballot_sync(0xffffffffu, t == CLS_CW);
    unsigned b2 = __ballot_sync(0xffffffffu, t == CLS_MU);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s[0][w] = __popc(b1); s[1][w] = __popc(b2); }
    __syncthreads();
    if (threadIdx.x < 2) {
        int sum = 0;
        for (int k = 0; k < 8; ++k) sum += s[threadIdx.x][k];
        bcount[threadIdx.x * nblocks + blockIdx.x] = sum;
    }
}

// exclusive scan of the block counts (one block of 1024 threads); totals to counts[0..1]
__global__ void __launch_bounds__(1024) k_scan(int32_t* bcount, int nblocks, int32_t* counts)
{
    __shared__ int part[1024];
    for (int q = 0; q < 2; ++q) {
        int32_t* b = bcount + q * nblocks;
        int per = (nblocks + 1023) / 1024;
        int lo = threadIdx.x * per, hi = min(lo + per, nblocks);
        int sum = 0;
        for (int i = lo; i < hi; ++i) sum += b[i];
        part[threadIdx.x] = sum;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {    // Hillis-Steele inclusive scan
            int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        int run = part[threadIdx.x] - sum;              // exclusive prefix of this thread's chunk
        for (int i = lo; i < hi; ++i) {
            int v = b[i];
            b[i] = run;
            run += v;
        }
        if (threadIdx.x == 1023) counts[q] = part[1023];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_scatter(const uint8_t* __restrict__ cls, int64_t nc, const int32_t* bcount,
                                                 int nblocks, int32_t* queue)
{
    __shared__ int s[2][8];
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    int t = c < nc ? cls[c] : 255;
    unsigned b1 = __ballot_sync(0xffffffffu, t == CLS_CW);
    unsigned b2 = __ballot_sync(0xffffffffu, t == CLS_MU);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s[0][w] = __popc(b1); s[1][w] = __popc(b2); }
    __syncthreads();
    unsigned lt = (1u << lane) - 1u;
    if (t == CLS_CW || t == CLS_MU) {
        int q = t == CLS_CW ? 0 : 1;
        unsigned b = q == 0 ? b1 : b2;
        int off = bcount[q * nblocks + blockIdx.x];
        for (int k = 0; k < w; ++k) off += s[q][k];
        off += __popc(b & lt);
        queue[q * nc + off] = (int32_t)c;
    }
}

template <class C, class T>
__global__ void __launch_bounds__(128) k_cweno(KParams<T> p, const T* __restrict__ U)
{
    constexpr int M = C::M, NV = C::NV, D = C::D, NFP = C::NFP, N = C::N, MD = C::MD;
    const int64_t nc = p.nc;
    const int cnt = p.counts[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int64_t c = p.queue[i];
        T uc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) uc[v] = U[v * nc + c];
        T du[M][NV];
        const int32_t* st = p.sten + c * M;
        for (int m = 0; m < M; ++m) {
            int64_t j = st[m];
#pragma unroll
            for (int v = 0; v < NV; ++v) du[m][v] = U[v * nc + j] - uc[v];
        }
        const int nf = p.nfc[c];
        const T lam1 = p.lam1, lams = (T(1) - lam1) / T(nf);
        const T* P = p.P + c * (int64_t)N * M;
        const T* OI = p.OI + c * (int64_t)C::NOI;
        T c1[NV], g[NV][D];
        for (int v = 0; v < NV; ++v) {
            T aopt[N];
            for (int k = 0; k < N; ++k) {
                T s = T(0);
                for (int m = 0; m < M; ++m) s += P[k * M + m] * du[m][v];
                aopt[k] = s;
            }
            T as[6][D];
            T sumlin[D];
#pragma unroll
            for (int k = 0; k < D; ++k) sumlin[k] = T(0);
            for (int f = 0; f < nf; ++f) {
                const uint8_t* idx = p.dir + (c * 6 + f) * MD;
                const T* Dm = p.Dd + (c * 6 + f) * (int64_t)D * MD;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    T s = T(0);
                    for (int b = 0; b < MD; ++b) s += Dm[k * MD + b] * du[idx[b]][v];
                    as[f][k] = s;
                    sumlin[k] += s;
                }
            }
            // p_1 = (p_opt - sum_s lambda_s p_s) / lambda_1
            T a1[N];
            for (int k = 0; k < N; ++k) a1[k] = (aopt[k] - (k < D ? lams * sumlin[k] : T(0))) / lam1;
            // smoothness indicators SI = a^T OI a (packed upper triangle)
            T si1 = T(0);
            for (int k = 0, o = 0; k < N; ++k) {
                T s = OI[o++] * a1[k];
                for (int l = k + 1; l < N; ++l) s += T(2) * OI[o++] * a1[l];
                si1 += a1[k] * s;
            }
            T sis[6];
            T tsum = T(0);
            for (int f = 0; f < nf; ++f) {
                T s = T(0);
                for (int k = 0; k < D; ++k) {
                    int o = k * N - k * (k - 1) / 2;
                    T t = OI[o] * as[f][k];
                    for (int l = k + 1; l < D; ++l) t += T(2) * OI[o + (l - k)] * as[f][l];
                    s += as[f][k] * t;
                }
                sis[f] = s;
                tsum += tabs(s - si1);
            }
            const T tau = tpow(tsum / T(nf), p.b_cw);
            T w1 = lam1 * (T(1) + tau / (p.eps_cw + si1));
            T wsum = w1;
            T ws[6];
            for (int f = 0; f < nf; ++f) {
                ws[f] = lams * (T(1) + tau / (p.eps_cw + sis[f]));
                wsum += ws[f];
            }
            const T om1 = w1 / wsum;
            c1[v] = om1 / lam1;
#pragma unroll
            for (int k = 0; k < D; ++k) g[v][k] = T(0);
            for (int f = 0; f < nf; ++f) {
                T cf = ws[f] / wsum - om1 * lams / lam1;
#pragma unroll
                for (int k = 0; k < D; ++k) g[v][k] += cf * as[f][k];
            }
        }
        // p_cweno = (omega_1/lambda_1) p_opt + sum_s (omega_s - omega_1 lambda_s / lambda_1) p_s
        const int Q = nf * NFP;
        const int64_t q0 = p.qoff[c];
        T* FS = p.FS + q0 * NV;
        const T* Phil = p.Phil + q0 * D;
        const T rb = uc[0], pb = pressure<T, D>(uc, p.gamma);
        const T rlim = p.h_theta * tmax(tabs(rb), p.h_eps), plim = p.h_theta * tmax(tabs(pb), p.h_eps);
        bool fail = false;
        for (int q = 0; q < Q; ++q) {
            T w[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                T s = uc[v] + c1[v] * (FS[q * NV + v] - uc[v]);
#pragma unroll
                for (int k = 0; k < D; ++k) s += Phil[q * D + k] * g[v][k];
                w[v] = s;
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) FS[q * NV + v] = w[v];
            T pw = pressure<T, D>(w, p.gamma);
            if (!(tabs(w[0] - rb) <= rlim) || !(tabs(pw - pb) <= plim)) fail = true;
        }
        if (fail) p.cls[c] = CLS_FIRST;
    }
}

template <class C, class T>
__global__ void __launch_bounds__(128) k_muscl(KParams<T> p, const T* __restrict__ U)
{
    constexpr int M = C::M, NV = C::NV, D = C::D, NFP = C::NFP, MD = C::MD;
    const int64_t nc = p.nc;
    const int cnt = p.counts[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int64_t c = p.queue[nc + i];
        T uc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) uc[v] = U[v * nc + c];
        const int nf = p.nfc[c];
        const int Q = nf * NFP;
        const int64_t q0 = p.qoff[c];
        const T* Phil = p.Phil + q0 * D;
        const T* G = p.G + c * (int64_t)D * MD;
        const int32_t* st = p.sten + c * M;
        T grad[NV][D], theta[NV];
        for (int v = 0; v < NV; ++v) {
#pragma unroll
            for (int k = 0; k < D; ++k) grad[v][k] = T(0);
            for (int b = 0; b < MD; ++b) {
                T dv = U[v * nc + st[b]] - uc[v];
#pragma unroll
                for (int k = 0; k < D; ++k) grad[v][k] += G[k * MD + b] * dv;
            }
            T lo = uc[v], hi = uc[v];
            for (int f = 0; f < nf; ++f) {
                int64_t j = p.nbr[c * 6 + f];
                if (j < 0) continue;
                T uj = U[v * nc + j];
                lo = tmin(lo, uj);
                hi = tmax(hi, uj);
            }
            T th = T(1);
            for (int q = 0; q < Q; ++q) {
                T dl = T(0);
#pragma unroll
                for (int k = 0; k < D; ++k) dl += Phil[q * D + k] * grad[v][k];
                T t = T(1);
                if (dl > T(0)) t = tmin(T(1), (hi - uc[v]) / dl);
                else if (dl < T(0)) t = tmin(T(1), (lo - uc[v]) / dl);
                th = tmin(th, t);
            }
            theta[v] = th;
        }
        T* FS = p.FS + q0 * NV;
        const T rb = uc[0], pb = pressure<T, D>(uc, p.gamma);
        const T rlim = p.h_theta * tmax(tabs(rb), p.h_eps), plim = p.h_theta * tmax(tabs(pb), p.h_eps);
        bool fail = false;
        for (int q = 0; q < Q; ++q) {
            T w[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                T dl = T(0);
#pragma unroll
                for (int k = 0; k < D; ++k) dl += Phil[q * D + k] * grad[v][k];
                w[v] = uc[v] + theta[v] * dl;
                FS[q * NV + v] = w[v];
            }
            T pw = pressure<T, D>(w, p.gamma);
            if (!(tabs(w[0] - rb) <= rlim) || !(tabs(pw - pb) <= plim)) fail = true;
        }
        if (fail) p.cls[c] = CLS_FIRST;
    }
}

template <class C, class T, int KIND>
__global__ void __launch_bounds__(128) k_flux(KParams<T> p, const T* __restrict__ U, T* __restrict__ R)
{
    constexpr int NV = C::NV, D = C::D, NFP = C::NFP;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.nc) return;
    const int64_t nc = p.nc;
    T uc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) uc[v] = U[v * nc + c];
    const int cc = p.cls[c];
    const int nf = p.nfc[c];
    const int64_t q0 = p.qoff[c];
    T acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = T(0);
    for (int f = 0; f < nf; ++f) {
        const int64_t j = p.nbr[c * 6 + f];
        const int fj = p.nbrf[c * 6 + f];
        const T* n = p.nrm + (c * 6 + f) * 3;
        T nn[3] = {n[0], n[1], n[2]};
        T uj[NV];
        int cj = CLS_LIN;
        if (j >= 0) {
            cj = p.cls[j];
            if (cj == CLS_FIRST)
#pragma unroll
                for (int v = 0; v < NV; ++v) uj[v] = U[v * nc + j];
        }
        for (int a = 0; a < NFP; ++a) {
            const int q = f * NFP + a;
            T wl[NV], wr[NV], F[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) wl[v] = cc == CLS_FIRST ? uc[v] : p.FS[(q0 + q) * NV + v];
            if (j < 0) {
#pragma unroll
                for (int v = 0; v < NV; ++v) wr[v] = wl[v];
            } else if (cj == CLS_FIRST) {
#pragma unroll
                for (int v = 0; v < NV; ++v) wr[v] = uj[v];
            } else {
                const int64_t qj = p.qoff[j] + fj * NFP + a;
#pragma unroll
                for (int v = 0; v < NV; ++v) wr[v] = p.FS[qj * NV + v];
            }
            riemann<T, D, KIND>(wl, wr, nn, p.gamma, F);
            const T w = p.W[q0 + q];
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += F[v] * w;
        }
    }
    const T iv = p.ivol[c];
#pragma unroll
    for (int v = 0; v < NV; ++v) R[v * nc + c] = -acc[v] * iv;
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

// scope guard: counts the launch and, when the scheme's timer is on, brackets
// it with a pair of events on the launch stream
struct Launch {
    KernelTimer* t;
    cudaStream_t st;
    int pair = -1;
    Launch(hfv_scheme* s, int kid, cudaStream_t stream) : t(&s->timer), st(stream)
    {
        note_launch();
        if (t->on && 2 * (t->used + 1) <= (int)t->ev.size()) {
            pair = t->used++;
            t->kid[pair] = kid;
            cudaEventRecord((cudaEvent_t)t->ev[2 * pair], st);
        }
    }
    ~Launch()
    {
        if (pair >= 0) cudaEventRecord((cudaEvent_t)t->ev[2 * pair + 1], st);
    }
};

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
    p.sten = a.sten; p.nbr = a.nbr; p.nbrf = a.nbrf; p.nfc = a.nfc; p.qoff = a.qoff; p.dir = a.dir;
    p.L = (const T*)a.L; p.P = (const T*)a.P; p.Phil = (const T*)a.Phil; p.OI = (const T*)a.OI;
    p.Dd = (const T*)a.D; p.G = (const T*)a.G; p.W = (const T*)a.W; p.nrm = (const T*)a.nrm;
    p.ivol = (const T*)a.ivol; p.dxthr = (const T*)a.dxthr;
    p.FS = (T*)a.FS; p.raw = a.raw; p.cls = a.cls; p.queue = a.queue; p.counts = a.counts;
    p.bcount = a.bcount; p.nblocks = s->nblocks; p.status = a.status;
    p.gamma = (T)s->p.gamma; p.alpha_m = (T)s->p.alpha_m; p.beta_m = (T)s->p.beta_m;
    p.alpha_w = (T)s->p.alpha_w; p.beta_w = (T)s->p.beta_w;
    p.lam1 = (T)(1.0 - 1.0 / s->p.lambda1_prime);
    p.eps_cw = (T)s->p.cweno_eps; p.b_cw = (T)s->p.cweno_b;
    p.h_theta = (T)s->p.harten_theta; p.h_eps = (T)s->p.harten_eps;
    return p;
}

template <class C, class T>
int run_residual(hfv_scheme* s, const T* U, T* R, const uint8_t* forced, uint8_t* cls_out, cudaStream_t st)
{
    KParams<T> p = make_params<T>(s, forced);
    const int64_t nc = p.nc;
    const unsigned g128 = (unsigned)((nc + 127) / 128), g256 = (unsigned)((nc + 255) / 256);
    { Launch l(s, KID_LINEAR, st); k_linear<C, T><<<g128, 128, 0, st>>>(p, U); }
    { Launch l(s, KID_TAG, st); k_tag<T><<<g256, 256, 0, st>>>(p); }
    { Launch l(s, KID_COUNT, st); k_count<<<s->nblocks, 256, 0, st>>>(s->a.cls, nc, s->a.bcount, s->nblocks); }
    { Launch l(s, KID_SCAN, st); k_scan<<<1, 1024, 0, st>>>(s->a.bcount, s->nblocks, s->a.counts); }
    { Launch l(s, KID_SCATTER, st); k_scatter<<<s->nblocks, 256, 0, st>>>(s->a.cls, nc, s->a.bcount, s->nblocks, s->a.queue); }
    const unsigned gq = (unsigned)std::min<int64_t>((nc + 127) / 128, 152 * 8);
    { Launch l(s, KID_CWENO, st); k_cweno<C, T><<<gq, 128, 0, st>>>(p, U); }
    { Launch l(s, KID_MUSCL, st); k_muscl<C, T><<<gq, 128, 0, st>>>(p, U); }
    {
        Launch l(s, KID_FLUX, st);
        switch (s->p.flux) {
        case HFV_RUSANOV: k_flux<C, T, kRusanov><<<g128, 128, 0, st>>>(p, U, R); break;
        case HFV_HLL: k_flux<C, T, kHLL><<<g128, 128, 0, st>>>(p, U, R); break;
        default: k_flux<C, T, kHLLC><<<g128, 128, 0, st>>>(p, U, R); break;
        }
    }
    if (cls_out) HFV_CUDA_CHECK(cudaMemcpyAsync(cls_out, s->a.cls, nc, cudaMemcpyDeviceToDevice, st));
    HFV_CUDA_CHECK(cudaGetLastError());
    return HFV_OK;
}


// ---------------------------------------------------------------------------
// time stepping (three-stage SSP Runge-Kutta, FP64 accumulation)
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_rk(int64_t n, double a, double b, const double* __restrict__ U0, const double* __restrict__ Us,
                     const T* __restrict__ R, const double* __restrict__ dt, double* out, float* outf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = b * (Us[i] + dt[0] * (double)R[i]);
    if (a != 0.0) v += a * U0[i];
    out[i] = v;
    if (outf) outf[i] = (float)v;
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ in, float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

__global__ void k_set(double* x, double v) { *x = v; }

__global__ void k_dt_init(unsigned long long* x) { *x = 0x7ff0000000000000ull; }

// dt_c = cfl |V_c| / sum_f (|u_c . n_f| + a_c) |S_f|; min over cells (order-free, exact)
__global__ void __launch_bounds__(256) k_dt(int64_t nc, int d, const double* __restrict__ U, const double* __restrict__ vol,
                                            const double* __restrict__ area, const double* __restrict__ nrm,
                                            const uint8_t* __restrict__ nfc, double gamma, double cfl,
                                            unsigned long long* out)
{
    __shared__ double red[8];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dtc = INFINITY;
    if (c < nc) {
        double rho = U[c], m2 = 0.0, u[3] = {0, 0, 0};
        for (int k = 0; k < d; ++k) {
            u[k] = U[(1 + k) * nc + c] / rho;
            m2 += U[(1 + k) * nc + c] * U[(1 + k) * nc + c];
        }
        double p = (gamma - 1.0) * (U[(d + 1) * nc + c] - 0.5 * m2 / rho);
        double a = sqrt(gamma * p / rho);
        double lam = 0.0;
        for (int f = 0; f < nfc[c]; ++f) {
            const double* n = nrm + (c * 6 + f) * 3;
            double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
            lam += (fabs(un) + a) * area[c * 6 + f];
        }
        dtc = cfl * vol[c] / lam;
        if (!(dtc > 0.0)) dtc = 0.0;  // a non-physical state stops the step at dt = 0
    }
    for (int o = 16; o > 0; o >>= 1) dtc = fmin(dtc, __shfl_xor_sync(0xffffffffu, dtc, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dtc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = red[0];
        for (int k = 1; k < 8; ++k) m = fmin(m, red[k]);
        atomicMin(out, (unsigned long long)__double_as_longlong(m));
    }
}

using Res64 = int (*)(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t);
using Res32 = int (*)(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t);

template <class T>
static auto pick(int d, int r) -> int (*)(hfv_scheme*, const T*, T*, const uint8_t*, uint8_t*, cudaStream_t)
{
    if (d == 2) {
        switch (r) {
        case 1: return run_residual<Cfg<2, 1>, T>;
        case 2: return run_residual<Cfg<2, 2>, T>;
        case 3: return run_residual<Cfg<2, 3>, T>;
        case 4: return run_residual<Cfg<2, 4>, T>;
        }
    } else {
        switch (r) {
        case 1: return run_residual<Cfg<3, 1>, T>;
        case 2: return run_residual<Cfg<3, 2>, T>;
        case 3: return run_residual<Cfg<3, 3>, T>;
        }
    }
    return nullptr;
}

bool residual_supported(int d, int r) { return pick<double>(d, r) != nullptr; }

int launch_residual(hfv_scheme* s, const void* U, void* R, const uint8_t* forced, uint8_t* cls_out, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (s->p.precision == HFV_FP32)
        return pick<float>(s->d, s->r)(s, (const float*)U, (float*)R, forced, cls_out, st);
    return pick<double>(s->d, s->r)(s, (const double*)U, (double*)R, forced, cls_out, st);
}

int launch_dt(hfv_scheme* s, const double* U, double cfl, double* dt_dev, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nc = s->mesh->nc;
    { Launch l(s, KID_DT, st); k_dt_init<<<1, 1, 0, st>>>((unsigned long long*)dt_dev); }
    {
        Launch l(s, KID_DT, st);
        k_dt<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(nc, s->d, U, s->a.vol, s->a.area, s->a.nrm64, s->a.nfc,
                                                             s->p.gamma, cfl, (unsigned long long*)dt_dev);
    }
    HFV_CUDA_CHECK(cudaGetLastError());
    return HFV_OK;
}

int launch_step(hfv_scheme* s, double* U, double cfl, double dt, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)s->nv * s->mesh->nc;
    const unsigned g = (unsigned)((n + 255) / 256);
    int rc;
    if (dt > 0.0) { Launch l(s, KID_DT, st); k_set<<<1, 1, 0, st>>>(s->a.dt, dt); }
    else if ((rc = launch_dt(s, U, cfl, s->a.dt, stream)) != HFV_OK) return rc;
    const double A[3] = {0.0, 0.75, 1.0 / 3.0}, B[3] = {1.0, 0.25, 2.0 / 3.0};
    double* outs[3] = {s->a.U1, s->a.U2, U};
    const double* ins[3] = {U, s->a.U1, s->a.U2};
    if (s->p.precision == HFV_FP32) {
        { Launch l(s, KID_CVT, st); k_to_f32<<<g, 256, 0, st>>>(n, U, s->a.Uf); }
        for (int k = 0; k < 3; ++k) {
            if ((rc = launch_residual(s, s->a.Uf, s->a.Rs, nullptr, nullptr, stream)) != HFV_OK) return rc;
            Launch l(s, KID_RK, st);
            k_rk<float><<<g, 256, 0, st>>>(n, A[k], B[k], U, ins[k], (const float*)s->a.Rs, s->a.dt, outs[k],
                                           k < 2 ? s->a.Uf : nullptr);
        }
    } else {
        for (int k = 0; k < 3; ++k) {
            if ((rc = launch_residual(s, ins[k], s->a.Rs, nullptr, nullptr, stream)) != HFV_OK) return rc;
            Launch l(s, KID_RK, st);
            k_rk<double><<<g, 256, 0, st>>>(n, A[k], B[k], U, ins[k], (const double*)s->a.Rs, s->a.dt, outs[k], nullptr);
        }
    }
    HFV_CUDA_CHECK(cudaGetLastError());
    return HFV_OK;
}

}  // namespace hfv
