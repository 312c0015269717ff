// residual.cu -- the hot path's entry points: residual dispatch by mesh
// family and order, the SSP Runge-Kutta steps (Sec. 2.4) and the time step.
// The residual kernels themselves are in residual_impl.cuh, instantiated in
// residual_2d.cu, residual_2d_high.cu, residual_3d.cu, residual_hex.cu,
// residual_hex5.cu and residual_hex6.cu.
#include "residual_impl.cuh"

namespace hfv {

// instantiated in the per-family translation units
extern template int run_residual<Cfg<2, 1, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<2, 1, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<2, 2, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<2, 2, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<2, 3, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<2, 3, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<2, 4, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<2, 4, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<2, 5, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<2, 5, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<2, 6, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<2, 6, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<3, 1, 1>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<3, 1, 1>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<3, 2, 1>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<3, 2, 1>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<3, 1, 2>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<3, 1, 2>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<3, 2, 2>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<3, 2, 2>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<3, 1, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<3, 1, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<3, 2, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<3, 2, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<3, 3, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<3, 3, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<3, 4, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<3, 4, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
extern template int run_residual<Cfg<3, 5, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
extern template int run_residual<Cfg<3, 5, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);

// ---------------------------------------------------------------------------
// time stepping (three-stage SSP Runge-Kutta, FP64 accumulation)
// ---------------------------------------------------------------------------
__global__ void k_set(double* x, double v, int n)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__global__ void k_dt_init(unsigned long long* x, int n)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = 0x7ff0000000000000ull;
}

// SSP-RK(5,4): the part of the last stage known after stage 4,
//   P = a52 u2 + a53 (u3 + c R(u3)),  c = w5 dt,  w5 = beta_53 / alpha_53
template <class T>
__global__ void __launch_bounds__(256) k_rk_partial(int64_t n, int64_t nc, const double* __restrict__ u2,
                                                   const double* __restrict__ u3, const T* __restrict__ R3,
                                                   const double* __restrict__ dt, double w5,
                                                   const int32_t* __restrict__ seg, double a52, double a53,
                                                   double* __restrict__ P)
{
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t cell = i % nc;
    P[i] = a52 * u2[i] + a53 * (u3[i] + w5 * dt[seg ? seg[cell] : 0] * (double)R3[i]);
}

// FP64 state (structure of arrays) -> the first stage's cell-major copy, and,
// when dt_out is given, the stable step
//   dt = cfl min_c |V_c| / sum_f (|u_c . n_f| + a_c) |S_f|
// from the copy (FP64 with FP64 geometry, or FP32 with FP32 geometry: then a
// stability estimate, not part of the conserved update), one minimum per
// problem (seg: the problem of each cell, null for one problem).  The min is
// order-free and exact.
template <class T, int NV>
__global__ void __launch_bounds__(256) k_stage_in(int64_t nc, const double* __restrict__ U, T* __restrict__ UA,
                                                  const T* __restrict__ ivol, const T* __restrict__ area,
                                                  const T* __restrict__ nrm, const uint8_t* __restrict__ nfc,
                                                  const int32_t* __restrict__ seg, double gamma, double cfl,
                                                  unsigned long long* dt_out, ViscParams<T> vp)
{
    pdl_wait();
    constexpr int P = AoSP<NV>::P;
    __shared__ T red[8];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T dtc = T(INFINITY);
    if (c < nc) {
        T u[P];
#pragma unroll
        for (int v = 0; v < P; ++v) u[v] = v < NV ? to_t<T>(U[v * nc + c]) : T(0);
        T* q = UA + c * P;
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int v = 0; v < P; v += 4) *reinterpret_cast<float4*>(q + v) = make_float4(u[v], u[v + 1], u[v + 2], u[v + 3]);
        } else {
#pragma unroll
            for (int v = 0; v < P; v += 2) *reinterpret_cast<double2*>(q + v) = make_double2(u[v], u[v + 1]);
        }
        if (dt_out) dtc = cell_dt<T, NV>(u, c, ivol, area, nrm, nfc[c] & 15, (T)gamma, (T)cfl, vp);
    }
    if (!dt_out) return;
    // problems are runs of consecutive cells: a block inside one problem
    // reduces first, a block across a boundary takes one atomic per cell
    int k0 = 0;
    if (seg) {
        const int64_t c0 = (int64_t)blockIdx.x * blockDim.x;
        const int64_t c1 = min(c0 + (int64_t)blockDim.x, nc) - 1;
        k0 = seg[c0];
        if (seg[c1] != k0) {
            if (c < nc) atomicMin(dt_out + seg[c], (unsigned long long)__double_as_longlong((double)dtc));
            return;
        }
    }
    // the minimum in the residual's precision (see cell_dt_finish), one
    // conversion to FP64 for the atomic
    for (int o = 16; o > 0; o >>= 1) dtc = tmin(dtc, __shfl_xor_sync(0xffffffffu, dtc, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dtc;
    __syncthreads();
    if (threadIdx.x == 0) {
        T m = red[0];
        for (int k = 1; k < 8; ++k) m = tmin(m, red[k]);
        atomicMin(dt_out + k0, (unsigned long long)__double_as_longlong((double)m));
    }
}

template <class T>
static auto pick(int d, int r, int fam)
    -> int (*)(hfv_scheme*, const T*, T*, const uint8_t*, uint8_t*, cudaStream_t, const T*, const StageRK*)
{
    if (d == 2) {
        switch (r) {
        case 1: return run_residual<Cfg<2, 1>, T>;
        case 2: return run_residual<Cfg<2, 2>, T>;
        case 3: return run_residual<Cfg<2, 3>, T>;
        case 4: return run_residual<Cfg<2, 4>, T>;
        case 5: return run_residual<Cfg<2, 5>, T>;
        case 6: return run_residual<Cfg<2, 6>, T>;
        }
    } else if (fam == 1) {
        switch (r) {
        case 1: return run_residual<Cfg<3, 1, 1>, T>;
        case 2: return run_residual<Cfg<3, 2, 1>, T>;
        }
    } else if (fam == 2) {
        switch (r) {
        case 1: return run_residual<Cfg<3, 1, 2>, T>;
        case 2: return run_residual<Cfg<3, 2, 2>, T>;
        }
    } else {
        switch (r) {
        case 1: return run_residual<Cfg<3, 1>, T>;
        case 2: return run_residual<Cfg<3, 2>, T>;
        case 3: return run_residual<Cfg<3, 3>, T>;
        case 4: return run_residual<Cfg<3, 4>, T>;
        case 5: return run_residual<Cfg<3, 5>, T>;
        }
    }
    return nullptr;
}

bool residual_supported(int d, int r, int fam) { return pick<double>(d, r, fam) != nullptr; }

static int residual_any(hfv_scheme* s, const void* U, void* R, const uint8_t* forced, uint8_t* cls_out,
                        cudaStream_t st, const void* ua, const StageRK* rk)
{
    if (s->p.precision == HFV_FP32)
        return pick<float>(s->d, s->r, s->fam)(s, (const float*)U, (float*)R, forced, cls_out, st, (const float*)ua, rk);
    return pick<double>(s->d, s->r, s->fam)(s, (const double*)U, (double*)R, forced, cls_out, st, (const double*)ua, rk);
}

int launch_residual(hfv_scheme* s, const void* U, void* R, const uint8_t* forced, uint8_t* cls_out, void* stream)
{
    s->chain_ok = false;   // the stage copy is overwritten
    return residual_any(s, U, R, forced, cls_out, (cudaStream_t)stream, nullptr, nullptr);
}

// FP64 state -> cell-major copy in UA (and the step into dt_dev when given)
static int stage_in(hfv_scheme* s, const double* U, double cfl, double* dt_dev, cudaStream_t st)
{
    const int64_t nc = s->mesh->nc;
    const unsigned g = (unsigned)((nc + 255) / 256);
    const hfv_dev_arrays& a = s->a;
    auto* out = (unsigned long long*)dt_dev;
    const ViscParams<float> vpf = visc_params<float>(s);
    const ViscParams<double> vpd = visc_params<double>(s);
    if (dt_dev) { Launch l(s, KID_DT, st); pdl(k_dt_init, (s->nseg + 255) / 256, 256, 0, st, out, s->nseg); }
    Launch l(s, KID_CVT, st);
    const bool f32 = s->p.precision == HFV_FP32;
    if (s->nv == 4) {
        if (f32) pdl(k_stage_in<float, 4>, g, 256, 0, st, nc, U, (float*)a.UA, (const float*)a.ivol, (const float*)a.areaT, (const float*)a.nrm, a.nfc, a.seg, s->p.gamma, cfl, out, vpf);
        else pdl(k_stage_in<double, 4>, g, 256, 0, st, nc, U, (double*)a.UA, (const double*)a.ivol, (const double*)a.areaT, (const double*)a.nrm, a.nfc, a.seg, s->p.gamma, cfl, out, vpd);
    } else {
        if (f32) pdl(k_stage_in<float, 5>, g, 256, 0, st, nc, U, (float*)a.UA, (const float*)a.ivol, (const float*)a.areaT, (const float*)a.nrm, a.nfc, a.seg, s->p.gamma, cfl, out, vpf);
        else pdl(k_stage_in<double, 5>, g, 256, 0, st, nc, U, (double*)a.UA, (const double*)a.ivol, (const double*)a.areaT, (const double*)a.nrm, a.nfc, a.seg, s->p.gamma, cfl, out, vpd);
    }
    HFV_CUDA_CHECK(cudaGetLastError());
    return HFV_OK;
}

int launch_dt(hfv_scheme* s, const double* U, double cfl, double* dt_dev, void* stream)
{
    s->chain_ok = false;
    return stage_in(s, U, cfl, dt_dev, (cudaStream_t)stream);
}

int launch_step(hfv_scheme* s, double* U, double cfl, double dt, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    // chained steps (step_chain): the previous call's last stage already wrote
    // this step's stage copy (and, in CFL mode, its time step into dt_next)
    // when this call repeats its state, mode and CFL number
    // (the viscous residual takes the stage-in pass: its flux kernel carries no chained epilogue)
    const bool chain = s->p.step_chain && s->p.time_scheme == HFV_SSPRK3 && !(s->p.mu0 > 0.0);
    const bool fixed = dt > 0.0;
    const bool warm = chain && s->chain_ok && s->chain_U == U && s->chain_fixed == fixed && (fixed || s->chain_cfl == cfl);
    s->chain_ok = false;
    if (fixed) {
        { Launch l(s, KID_DT, st); pdl(k_set, (s->nseg + 255) / 256, 256, 0, st, s->a.dt, dt, s->nseg); }
        if (!warm && (rc = stage_in(s, U, cfl, nullptr, st)) != HFV_OK) return rc;
    } else if (!warm && (rc = stage_in(s, U, cfl, s->a.dt, st)) != HFV_OK) {
        return rc;
    }
    if (chain && !fixed && !warm) {
        // the first step of a chain: dt_next starts at +inf for the last stage's minimum
        Launch l(s, KID_DT, st);
        pdl(k_dt_init, (s->nseg * kDtSlots * kDtStride + 255) / 256, 256, 0, st, (unsigned long long*)s->a.dt_next,
            s->nseg * kDtSlots * kDtStride);
    }
    // stages alternate the cell-major copies UA, UB, UA, ...; each stage's
    // flux kernel writes the next one
    void* uab[2] = {s->a.UA, s->a.UB};
    if (s->p.time_scheme == HFV_SSPRK54) {
        // u_i = sum_j alpha_ij u_j + beta_ij dt L(u_j) (Spiteri and Ruuth's
        // SSP-RK(5,4), Shu-Osher form): stage i reads u_{i-1} and writes
        //   u_i = alpha_i0 u_0 + alpha_i,i-1 (u_{i-1} + (beta_i,i-1 / alpha_i,i-1) dt L(u_{i-1}));
        // after stage 4, P = alpha_52 u_2 + alpha_53 (u_3 + (beta_53 / alpha_53) dt L(u_3))
        // from the kept L(u_3), and stage 5 writes
        //   u_5 = P + alpha_54 (u_4 + (beta_54 / alpha_54) dt L(u_4))
        static const double a10 = 1.0, b10 = 0.391752226571890;
        static const double a20 = 0.444370493651235, a21 = 0.555629506348765, b21 = 0.368410593050371;
        static const double a30 = 0.620101851488403, a32 = 0.379898148511597, b32 = 0.251891774271694;
        static const double a40 = 0.178079954393132, a43 = 0.821920045606868, b43 = 0.544974750228521;
        static const double a52 = 0.517231671970585, a53 = 0.096059710526147, b53 = 0.063692468666290;
        static const double a54 = 0.386708617503269, b54 = 0.226007483236906;
        double* u[5] = {U, s->a.U1, s->a.U2, s->a.U3, s->a.U4};
        const double A0[5] = {0.0, a20, a30, a40, 1.0};
        const double Bk[5] = {a10, a21, a32, a43, a54};
        // c_k = (beta_k,k-1 / alpha_k,k-1) dt; (beta_53 / alpha_53) dt for P
        const double W[6] = {b10 / a10, b21 / a21, b32 / a32, b43 / a43, b54 / a54, b53 / a53};
        const int64_t nvc = (int64_t)s->nv * s->mesh->nc;
        for (int k = 0; k < 5; ++k) {
            StageRK rk;
            rk.a = A0[k];
            rk.b = Bk[k];
            rk.w = W[k];
            rk.U0 = k == 4 ? s->a.U5 : U;
            rk.Us = u[k];
            rk.out = k == 4 ? U : u[k + 1];
            rk.ua_next = k < 4 ? uab[(k + 1) & 1] : nullptr;
            rk.keep_R = k == 3;
            if ((rc = residual_any(s, nullptr, s->a.Rs, nullptr, nullptr, st, uab[k & 1], &rk)) != HFV_OK) return rc;
            if (k == 3) {
                Launch l(s, KID_RK, st);
                const unsigned g = (unsigned)((nvc + 255) / 256);
                if (s->p.precision == HFV_FP32)
                    pdl(k_rk_partial<float>, g, 256, 0, st, nvc, s->mesh->nc, s->a.U2, s->a.U3, (const float*)s->a.Rs,
                        (const double*)s->a.dt, W[5], s->a.seg, a52, a53, s->a.U5);
                else
                    pdl(k_rk_partial<double>, g, 256, 0, st, nvc, s->mesh->nc, s->a.U2, s->a.U3, (const double*)s->a.Rs,
                        (const double*)s->a.dt, W[5], s->a.seg, a52, a53, s->a.U5);
            }
        }
        HFV_CUDA_CHECK(cudaGetLastError());
        return HFV_OK;
    }
    double* outs[3] = {s->a.U1, s->a.U2, U};
    const double* ins[3] = {U, s->a.U1, s->a.U2};
    const double A[3] = {0.0, 0.75, 1.0 / 3.0}, B[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int k = 0; k < 3; ++k) {
        StageRK rk;
        rk.a = A[k];
        rk.b = B[k];
        rk.w = 1.0;
        rk.U0 = U;
        rk.Us = ins[k];
        rk.out = outs[k];
        rk.ua_next = k < 2 ? uab[(k + 1) & 1] : chain ? uab[0] : nullptr;
        if (chain && !fixed) {
            if (k == 0 && warm) rk.dt_pending = (unsigned long long*)s->a.dt_next;
            if (k == 2) { rk.dt_next = (unsigned long long*)s->a.dt_next; rk.cfl = cfl; }
        }
        if ((rc = residual_any(s, nullptr, s->a.Rs, nullptr, nullptr, st, uab[k & 1], &rk)) != HFV_OK) return rc;
    }
    HFV_CUDA_CHECK(cudaGetLastError());
    if (chain) {
        s->chain_ok = true;
        s->chain_U = U;
        s->chain_fixed = fixed;
        s->chain_cfl = cfl;
    }
    return HFV_OK;
}

}  // namespace hfv
