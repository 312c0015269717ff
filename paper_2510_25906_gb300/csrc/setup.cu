// setup.cu -- device memory of a scheme and the FP64 operator build on the
// GPU (one thread per cell, chunked), see setup_math.cuh for the steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hfv_internal.h"
#include "kernels.cuh"
#include "setup_math.cuh"

namespace hfv {

#define SETUP_CHECK(x)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (x);                                                                 \
        if (e_ != cudaSuccess) {                                                              \
            set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x);            \
            return e_ == cudaErrorMemoryAllocation ? HFV_ERR_OOM : HFV_ERR_CUDA;               \
        }                                                                                     \
    } while (0)

namespace {

// Gauss-Legendre rule on [0, 1]: roots of P_n by Newton's method from the
// Chebyshev-like initial guesses, weights 1 / ((1 - z^2) P_n'(z)^2).
void gauss01(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        double d = 1.0;
        for (int it = 0; it < 60; ++it) {
            double pm = 1.0, pc = z;
            for (int k = 1; k < n; ++k) {
                double pn = ((2 * k + 1) * z * pc - k * pm) / (k + 1);
                pm = pc;
                pc = pn;
            }
            if (n == 0) pc = 1.0;
            d = n * (pm - z * pc) / (1.0 - z * z);
            double step = pc / d;
            z -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        double pm = 1.0, pc = z;
        for (int k = 1; k < n; ++k) {
            double pn = ((2 * k + 1) * z * pc - k * pm) / (k + 1);
            pm = pc;
            pc = pn;
        }
        d = n * (pm - z * pc) / (1.0 - z * z);
        x[n - 1 - i] = 0.5 * (1.0 + z);
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * d * d);
    }
}

__global__ void k_setup(SetupParams S, SetupOut O, double* ws, int64_t stride, int64_t c0, int64_t cn)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cn) return;
    const int64_t c = c0 + t;
    SetupWork W{ws + t, stride};
    if (!setup_cell(S, O, W, c)) atomicMin(O.err, (int)c);
}

template <class T>
__global__ void k_cvt(int64_t n, const double* __restrict__ in, T* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

template <class T>
void convert(const double* in, void* out, int64_t n, cudaStream_t st)
{
    if (n <= 0) return;
    unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32);
    k_cvt<T><<<g, 256, 0, st>>>(n, in, (T*)out);
}

}  // namespace

// Allocate the scheme's device memory (one arena) and build every operator.
int build_operators(hfv_scheme* s, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const hfv_mesh* m = s->mesh;
    const int64_t nc = m->nc, qt = s->qtot;
    const int d = s->d, M = s->M, N = s->N, Md = s->Md, nv = s->nv;
    const int NOI = N * (N + 1) / 2;
    const bool f32 = s->p.precision == HFV_FP32;
    const size_t b = f32 ? 4 : 8;
    s->nblocks = (int)((nc + 255) / 256);
    s->nseg = (int)m->seg_off.size() - 1;

    // ---- arena layout ----
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += al(bytes); return o; };
    const int64_t ncp = s->nc_pad, lt = s->ltot;
    size_t o_nfs = take(nc * 6 * 4);
    size_t o_sten = take(ncp * M * 4), o_nbr = take(nc * 6 * 4), o_nbrf = take(nc * 6), o_nfc = take(nc),
           o_qoff = take((nc + 1) * 8), o_loff = take((ncp + 1) * 8), o_dir = take(nc * 6 * Md);
    size_t o_L = take(lt * b), o_P = take(nc * N * M * b), o_Phil = take(qt * d * b), o_OI = take(nc * NOI * b),
           o_D = take(nc * 6 * d * Md * b), o_G = take(nc * d * Md * b), o_W = take(qt * b), o_nrm = take(nc * 18 * b),
           o_ivol = take(nc * b), o_thr = take(nc * b);
    size_t o_vol = take(nc * 8), o_area = take(nc * 6 * 8), o_nrm64 = take(nc * 18 * 8);
    size_t o_FS = take(qt * nv * b), o_raw = take(nc), o_cls = take(nc), o_queue = take(2 * nc * 4), o_counts = take(64),
           o_status = take(64);
    size_t o_U1 = take(nv * nc * 8), o_U2 = take(nv * nc * 8), o_Rs = take(nv * nc * b), o_UA = take(nc * (nv == 4 ? 4 : 8) * b), o_UB = take(nc * (nv == 4 ? 4 : 8) * b),
           o_areaT = take(nc * 6 * b),
           o_dt = take(std::max<int64_t>(64, 8 * (int64_t)s->nseg)), o_dtn = take(8 * kDtSlots * kDtStride * (int64_t)s->nseg),
           o_Uio = take(nv * nc * 8),
           o_seg = take(s->nseg > 1 ? nc * 4 : 0);
    const bool rk54 = s->p.time_scheme == HFV_SSPRK54;
    size_t o_U3 = take(rk54 ? nv * nc * 8 : 0), o_U4 = take(rk54 ? nv * nc * 8 : 0), o_U5 = take(rk54 ? nv * nc * 8 : 0);
    const bool visc = s->p.mu0 > 0.0;
    const int nvx = d + d * d;
    size_t o_VX = take(visc ? nc * nvx * b : 0), o_LINV = take(visc ? nc * 6 * b : 0),
           o_GS = take(visc ? qt * (d + 1) * d * b : 0);
    s->arena_bytes = off;
    SETUP_CHECK(cudaMalloc(&s->arena, off));
    char* A = (char*)s->arena;
    hfv_dev_arrays& a = s->a;
    a.sten = (int32_t*)(A + o_sten); a.nbr = (int32_t*)(A + o_nbr); a.nbrf = (int8_t*)(A + o_nbrf);
    a.nfc = (uint8_t*)(A + o_nfc); a.qoff = (int64_t*)(A + o_qoff); a.dir = (uint8_t*)(A + o_dir);
    a.loff = (int64_t*)(A + o_loff);
    a.nfs = (int32_t*)(A + o_nfs);
    a.L = A + o_L; a.P = A + o_P; a.Phil = A + o_Phil; a.OI = A + o_OI; a.D = A + o_D; a.G = A + o_G; a.W = A + o_W;
    a.nrm = A + o_nrm; a.ivol = A + o_ivol; a.dxthr = A + o_thr;
    a.vol = (double*)(A + o_vol); a.area = (double*)(A + o_area); a.nrm64 = (double*)(A + o_nrm64);
    a.FS = A + o_FS; a.raw = (uint8_t*)(A + o_raw); a.cls = (uint8_t*)(A + o_cls); a.queue = (int32_t*)(A + o_queue);
    a.counts = (int32_t*)(A + o_counts); a.status = (int*)(A + o_status);
    a.U1 = (double*)(A + o_U1); a.U2 = (double*)(A + o_U2); a.Rs = A + o_Rs; a.UA = A + o_UA; a.UB = A + o_UB; a.areaT = A + o_areaT;
    a.dt = (double*)(A + o_dt);
    a.dt_next = (double*)(A + o_dtn);
    a.seg = s->nseg > 1 ? (int32_t*)(A + o_seg) : nullptr;
    a.U3 = rk54 ? (double*)(A + o_U3) : nullptr;
    a.U4 = rk54 ? (double*)(A + o_U4) : nullptr;
    a.U5 = rk54 ? (double*)(A + o_U5) : nullptr;
    a.Uio = (double*)(A + o_Uio);
    a.VX = visc ? A + o_VX : nullptr;
    a.LINV = visc ? A + o_LINV : nullptr;
    a.GS = visc ? A + o_GS : nullptr;
    SETUP_CHECK(cudaMemsetAsync(s->arena, 0, off, st));

    // ---- host-side per-cell data ----
    std::vector<int32_t> nbr(m->nbr.begin(), m->nbr.end());
    std::vector<int32_t> nfs(nc * 6, -1);
    {
        const int64_t qs = (int64_t)s->nfmax * s->nfp;
        if (nc * qs >= (int64_t(1) << 31)) {
            set_error("hfv_scheme_create: mesh too large for 32-bit face-point offsets");
            return HFV_ERR_ARG;
        }
        for (int64_t c = 0; c < nc; ++c)
            for (int f = 0; f < 6; ++f) {
                const int32_t j = m->nbr[c * kMaxFaces + f];
                if (f >= type_nfaces(m->type[c])) nfs[c * 6 + f] = -2;
                else if (j >= 0) nfs[c * 6 + f] = (int32_t)(j * qs + m->nbrf[c * kMaxFaces + f] * s->nfp);
            }
    }
    std::vector<uint8_t> nfc(nc);
    std::vector<int32_t> fvtx(nc * 24, 0);
    std::vector<int8_t> fk(nc * 18, 0);
    std::vector<double> ivol(nc), thr(nc);
    for (int64_t c = 0; c < nc; ++c) {
        int t = m->type[c];
        nfc[c] = (uint8_t)(type_nfaces(t) | (s->n1[c] << 4));
        for (int f = 0; f < type_nfaces(t); ++f) {
            int64_t cf = c * kMaxFaces + f;
            int64_t oc = c;
            int of = f;
            if (!m->own[cf]) {
                oc = m->nbr[cf];
                of = m->nbrf[cf];
                for (int k = 0; k < 3; ++k) fk[cf * 3 + k] = m->nshift[cf * 3 + k];
            }
            int ot = m->type[oc];
            for (int q = 0; q < face_nverts(ot, of); ++q) fvtx[cf * 4 + q] = m->cidx[m->cptr[oc] + type_face_vertex(ot, of, q)];
        }
        ivol[c] = 1.0 / m->vol[c];
        double dx = d == 2 ? std::sqrt(m->vol[c]) : std::cbrt(m->vol[c]);
        thr[c] = std::pow(s->p.kappa * dx, s->p.n_exp);
    }
    SETUP_CHECK(cudaMemcpyAsync(a.sten, s->sten.data(), nc * M * 4, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(a.nbr, nbr.data(), nc * 6 * 4, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(a.nfs, nfs.data(), nc * 6 * 4, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(a.nbrf, m->nbrf.data(), nc * 6, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(a.nfc, nfc.data(), nc, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(a.qoff, s->qoff.data(), (nc + 1) * 8, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(a.loff, s->loff.data(), (ncp + 1) * 8, cudaMemcpyHostToDevice, st));
    std::vector<int32_t> seg;
    if (a.seg) {
        seg.resize(nc);
        for (int k = 0; k < s->nseg; ++k)
            for (int64_t c = m->seg_off[k]; c < m->seg_off[k + 1]; ++c) seg[c] = k;
        SETUP_CHECK(cudaMemcpyAsync(a.seg, seg.data(), nc * 4, cudaMemcpyHostToDevice, st));
    }
    SETUP_CHECK(cudaMemcpyAsync(a.dir, s->dir.data(), nc * 6 * Md, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(a.vol, m->vol.data(), nc * 8, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(a.area, m->farea.data(), nc * 6 * 8, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(a.nrm64, m->fnorm.data(), nc * 18 * 8, cudaMemcpyHostToDevice, st));

    // ---- temporaries of the FP64 build ----
    const int64_t chunk = std::min<int64_t>(nc, 131072);
    size_t t_off = 0;
    auto ttake = [&](size_t bytes) { size_t o = t_off; t_off += al(bytes); return o; };
    size_t t_xyz = ttake(m->nn * 3 * 8), t_cptr = ttake((nc + 1) * 8), t_cidx = ttake(m->cidx.size() * 4),
           t_type = ttake(nc), t_sshift = ttake(nc * M * 3), t_nd = ttake(nc * 6), t_fvtx = ttake(nc * 24 * 4),
           t_fk = ttake(nc * 18), t_ws = ttake((size_t)chunk * M * N * 8), t_err = ttake(64);
    // FP32 schemes build their operators in FP64 one chunk of cells at a time
    // and convert each chunk into the arena, so the FP64 copies never exceed
    // one chunk (hexahedra at order 6 carry 24 KB of L per cell in FP32)
    const int64_t qs = (int64_t)s->nfmax * s->nfp;
    int64_t lchunk = 0;
    for (int64_t c0 = 0; c0 < nc; c0 += chunk)
        lchunk = std::max<int64_t>(lchunk, s->loff[std::min(c0 + chunk, nc)] - s->loff[c0]);
    size_t t_L = 0, t_P = 0, t_Phil = 0, t_OI = 0, t_D = 0, t_G = 0, t_W = 0, t_VX = 0;
    if (f32) {
        t_L = ttake(lchunk * 8); t_P = ttake(chunk * N * M * 8); t_Phil = ttake(chunk * qs * d * 8);
        t_OI = ttake(chunk * NOI * 8); t_D = ttake(chunk * 6 * d * Md * 8); t_G = ttake(chunk * d * Md * 8);
        t_W = ttake(chunk * qs * 8);
        if (visc) t_VX = ttake(chunk * nvx * 8);
    }
    char* T = nullptr;
    SETUP_CHECK(cudaMalloc(&T, t_off));
    SETUP_CHECK(cudaMemcpyAsync(T + t_xyz, m->xyz.data(), m->nn * 3 * 8, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(T + t_cptr, m->cptr.data(), (nc + 1) * 8, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(T + t_cidx, m->cidx.data(), m->cidx.size() * 4, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(T + t_type, m->type.data(), nc, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(T + t_sshift, s->sshift.data(), nc * M * 3, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(T + t_nd, s->nd.data(), nc * 6, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(T + t_fvtx, fvtx.data(), nc * 24 * 4, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(T + t_fk, fk.data(), nc * 18, cudaMemcpyHostToDevice, st));
    const int big = 0x7fffffff;
    SETUP_CHECK(cudaMemcpyAsync(T + t_err, &big, 4, cudaMemcpyHostToDevice, st));

    SetupParams S;
    std::memset(&S, 0, sizeof S);
    S.xyz = (const double*)(T + t_xyz); S.cptr = (const int64_t*)(T + t_cptr); S.cidx = (const int32_t*)(T + t_cidx);
    S.type = (const uint8_t*)(T + t_type); S.sten = a.sten; S.sshift = (const int8_t*)(T + t_sshift); S.dir = a.dir;
    S.nd = (const uint8_t*)(T + t_nd); S.fvtx = (const int32_t*)(T + t_fvtx); S.fk = (const int8_t*)(T + t_fk);
    S.farea = a.area; S.qoff = a.qoff; S.loff = a.loff;
    for (int k = 0; k < 3; ++k) S.period[k] = m->period[k];
    S.d = d; S.r = s->r; S.N = N; S.M = M; S.Md = Md; S.nq = s->nq; S.nfp = s->nfp;
    S.nvq = d == 2 ? s->r + 1 : s->r + 2;
    S.lcw = f32 ? 4 : 2;
    gauss01(s->nq, S.gfx, S.gfw);
    gauss01(S.nvq, S.gvx, S.gvw);
    {
        int k = 0;
        for (int deg = 1; deg <= s->r; ++deg)
            for (int ea = deg; ea >= 0; --ea) {
                if (d == 2) { S.ex[k][0] = (int8_t)ea; S.ex[k][1] = (int8_t)(deg - ea); S.ex[k][2] = 0; ++k; }
                else
                    for (int eb = deg - ea; eb >= 0; --eb) {
                        S.ex[k][0] = (int8_t)ea; S.ex[k][1] = (int8_t)eb; S.ex[k][2] = (int8_t)(deg - ea - eb); ++k;
                    }
            }
    }
    SetupOut O;
    O.L = (double*)(f32 ? T + t_L : (char*)a.L);
    O.P = (double*)(f32 ? T + t_P : (char*)a.P);
    O.Phil = (double*)(f32 ? T + t_Phil : (char*)a.Phil);
    O.OI = (double*)(f32 ? T + t_OI : (char*)a.OI);
    O.D = (double*)(f32 ? T + t_D : (char*)a.D);
    O.G = (double*)(f32 ? T + t_G : (char*)a.G);
    O.W = (double*)(f32 ? T + t_W : (char*)a.W);
    O.VX = visc ? (double*)(f32 ? T + t_VX : (char*)a.VX) : nullptr;
    O.err = (int*)(T + t_err);
    double* ws = (double*)(T + t_ws);
    // the per-cell build keeps its small matrices in local memory (~12 KB
    // of stack per thread): raise this context's stack limit for the build
    constexpr size_t kStack = 16384;
    size_t old_stack = 0;
    SETUP_CHECK(cudaDeviceGetLimit(&old_stack, cudaLimitStackSize));
    if (old_stack < kStack) SETUP_CHECK(cudaDeviceSetLimit(cudaLimitStackSize, kStack));
    for (int64_t c0 = 0; c0 < nc; c0 += chunk) {
        int64_t cn = std::min(chunk, nc - c0);
        if (f32) { O.cbase = c0; O.qbase = s->qoff[c0]; O.lbase = s->loff[c0]; }
        k_setup<<<(unsigned)((cn + 63) / 64), 64, 0, st>>>(S, O, ws, chunk, c0, cn);
        SETUP_CHECK(cudaGetLastError());
        if (f32) {
            const int64_t l0 = s->loff[c0], q0 = s->qoff[c0];
            convert<float>(O.L, (float*)a.L + l0, s->loff[c0 + cn] - l0, st);
            convert<float>(O.P, (float*)a.P + c0 * N * M, cn * N * M, st);
            convert<float>(O.Phil, (float*)a.Phil + q0 * d, (s->qoff[c0 + cn] - q0) * d, st);
            convert<float>(O.OI, (float*)a.OI + c0 * NOI, cn * NOI, st);
            convert<float>(O.D, (float*)a.D + c0 * 6 * d * Md, cn * 6 * d * Md, st);
            convert<float>(O.G, (float*)a.G + c0 * d * Md, cn * d * Md, st);
            convert<float>(O.W, (float*)a.W + q0, s->qoff[c0 + cn] - q0, st);
            if (visc) convert<float>(O.VX, (float*)a.VX + c0 * nvx, cn * nvx, st);
        }
    }
    int err_cell = big;
    SETUP_CHECK(cudaMemcpyAsync(&err_cell, O.err, 4, cudaMemcpyDeviceToHost, st));
    SETUP_CHECK(cudaStreamSynchronize(st));
    if (old_stack < kStack) SETUP_CHECK(cudaDeviceSetLimit(cudaLimitStackSize, old_stack));
    if (err_cell != big) {
        cudaFree(T);
        set_error("hfv_scheme_create: rank-deficient least-squares system at cell " + std::to_string(err_cell));
        return HFV_ERR_STENCIL;
    }
    // per-precision copies of the small geometric arrays
    std::vector<double> nrm(m->fnorm.begin(), m->fnorm.end());
    // viscous penalty (eq. viscous_jump): 1 / distance between the cell's and
    // each face neighbour's centre (vertex means; the neighbour moved by its
    // periodic shift), 0 on open boundaries
    std::vector<double> linv(visc ? nc * 6 : 0, 0.0);
    for (int64_t c = 0; visc && c < nc; ++c)
        for (int f = 0; f < type_nfaces(m->type[c]); ++f) {
            const int32_t j = m->nbr[c * kMaxFaces + f];
            if (j < 0) continue;
            double l2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double dx = m->vmean[3 * j + k] + m->nshift[(c * kMaxFaces + f) * 3 + k] * m->period[k] -
                                  m->vmean[3 * c + k];
                l2 += dx * dx;
            }
            linv[c * 6 + f] = 1.0 / std::sqrt(l2);
        }
    double* h64 = nullptr;
    SETUP_CHECK(cudaMalloc(&h64, al(nc * 8) * 2 + al(nc * 18 * 8) + al(linv.size() * 8)));
    double* d_ivol = h64;
    double* d_thr = (double*)((char*)h64 + al(nc * 8));
    double* d_nrm = (double*)((char*)h64 + 2 * al(nc * 8));
    double* d_linv = (double*)((char*)h64 + 2 * al(nc * 8) + al(nc * 18 * 8));
    if (visc) SETUP_CHECK(cudaMemcpyAsync(d_linv, linv.data(), nc * 6 * 8, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(d_ivol, ivol.data(), nc * 8, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(d_thr, thr.data(), nc * 8, cudaMemcpyHostToDevice, st));
    SETUP_CHECK(cudaMemcpyAsync(d_nrm, nrm.data(), nc * 18 * 8, cudaMemcpyHostToDevice, st));
    if (f32) {
        convert<float>(d_ivol, a.ivol, nc, st); convert<float>(d_thr, a.dxthr, nc, st); convert<float>(d_nrm, a.nrm, nc * 18, st);
        convert<float>(a.area, a.areaT, nc * 6, st);
        if (visc) convert<float>(d_linv, a.LINV, nc * 6, st);
    } else {
        SETUP_CHECK(cudaMemcpyAsync(a.ivol, d_ivol, nc * 8, cudaMemcpyDeviceToDevice, st));
        SETUP_CHECK(cudaMemcpyAsync(a.dxthr, d_thr, nc * 8, cudaMemcpyDeviceToDevice, st));
        SETUP_CHECK(cudaMemcpyAsync(a.nrm, d_nrm, nc * 18 * 8, cudaMemcpyDeviceToDevice, st));
        SETUP_CHECK(cudaMemcpyAsync(a.areaT, a.area, nc * 6 * 8, cudaMemcpyDeviceToDevice, st));
        if (visc) SETUP_CHECK(cudaMemcpyAsync(a.LINV, d_linv, nc * 6 * 8, cudaMemcpyDeviceToDevice, st));
    }
    SETUP_CHECK(cudaGetLastError());
    SETUP_CHECK(cudaStreamSynchronize(st));
    cudaFree(h64);
    cudaFree(T);
    return HFV_OK;
}

}  // namespace hfv
