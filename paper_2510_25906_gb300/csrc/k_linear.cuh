// k_linear.cuh -- K1, the candidate kernel of the residual: stencil gather,
// the linear candidate at the face points (Sec. 2.1), the detector (Sec. 2.5)
// and the Harten test, fed by bulk copies into a shared-memory ring.
#pragma once

#include "../../include/hfv.h"
#include "device_common.cuh"
#include "tma.cuh"

namespace hfv {

// K1: persistent, warp-specialised.  Tiles of NG consecutive cells: a
// producer warp streams each tile's contiguous L blocks and stencil ids into a
// ring of shared-memory stages with bulk copies (TMA engine, mbarrier
// completion); eight consumer warps hold NG groups of G lanes, one group per
// cell.  A group gathers the M stencil states into rows of U_m - U_0, lane l
// forms the candidate at face points l, l + G, ... (PPL of them) from their
// rows of L, and the group runs the detector (bounds from the first stencil
// layer = the face neighbours) and the Harten test.
//
// L block of a cell with Q face points: columns in chunks of W = 16 bytes /
// sizeof(T); chunk j holds [Q][W] (the W values of every row for columns
// jW .. jW+W-1), a last partial chunk of width M mod W holds [Q][M mod W].
// One 16-byte load gives a lane W columns of its row, and the eight lanes of
// a group read 128 contiguous bytes.
template <class C, class T, bool WIDE = false>
struct K1Shape {
    // 2D orders 2-4: four lanes per cell (one per face neighbour) with up to
    // two face points each, so that the per-cell work of the detector and of
    // the Harten test is shared by eight cells per warp instruction; one
    // face point per lane elsewhere (more points per lane in 3D would need
    // more cells per tile than a ring of stages of L holds: 3.8 KB of L per
    // hexahedron at order 4)
    static constexpr bool SMALL = C::D == 2 && C::QMAX <= 8;
    // 3D with up to 32 face points and M <= 20 (order 3; hexahedra, prisms,
    // pyramids): sixteen lanes per cell, two points each
    static constexpr bool SMALL3 = C::D == 3 && C::QMAX > 16 && C::QMAX <= 32 && C::M <= 20;
    static constexpr int G = SMALL ? 4 : SMALL3 ? 16 : GroupSize<C::QMAX>::value;   // lanes per cell
    // face points per lane: two in the layouts above, and two where a
    // hexahedron has more points than a warp has lanes (orders 5-6, 54 points)
    static constexpr int PPL = SMALL ? C::QMAX / 4 : SMALL3 ? 2 : (C::QMAX + G - 1) / G;
    static constexpr int SLOT = C::NFMAX <= 4 ? 4 : 8;       // lanes of one face-neighbour reduction
    // lanes past the first SLOT take the bounds from the group's first lane
    static constexpr bool NB_BCAST = G > SLOT;
    static constexpr int PER16 = 16 / (int)sizeof(T);
    static constexpr int LMAX = (C::QMAX * C::M + PER16 - 1) / PER16 * PER16;  // elements per cell block
    // rows of U_m - U_0 per cell: [M][4] and, with five variables, [M] of the
    // fifth; cells 16 bytes apart modulo 128 so that the four cells of a warp
    // read different banks
    static constexpr int DU4 = C::M * 4 * (int)sizeof(T);
    static constexpr int DU5 = C::NV == 5 ? (C::M * (int)sizeof(T) + 15) / 16 * 16 : 0;
    static constexpr int CSTRIDE = (DU4 + DU5 + 127) / 128 * 128 + 16;
    // shared memory of two ring stages and the U_m - U_0 rows for a tile of
    // `consumers` / G cells
    static constexpr int two_stages(int consumers)
    {
        const int ng = consumers / G;
        const int stage = (ng * LMAX * (int)sizeof(T) + ng * C::M * 4 + 127) / 128 * 128;
        return 2 * stage + (ng * CSTRIDE + 127) / 128 * 128 + 4 * 8 + 1024;
    }
    // eight consumer warps, or four or two where a tile of the large blocks
    // of L (orders 6-7 in 2D, FP64) would not leave room for two ring stages.
    // 2D orders 2-3 in FP32: six consumer warps (48-cell tiles) and three
    // CTAs per SM, each with a three-stage ring: 3 % faster per quadrant step
    // than two CTAs of eight warps (29.1 against 31.0 us per launch), where
    // two CTAs of six warps with four stages measured 4 % slower and three
    // CTAs of eight warps with two stages 13 % slower
    // (WIDE: the two-CTA shape, the autotuner's alternative for these)
    static constexpr bool TRIPLE = !WIDE && SMALL && C::M <= 12 && sizeof(T) == 4;
    static constexpr bool HAS_WIDE = WIDE || TRIPLE;
    static constexpr int CONSUMERS = TRIPLE ? 192
                                     : two_stages(256) <= 227 * 1024 ? 256
                                     : two_stages(128) <= 227 * 1024 ? 128 : 64;
    static constexpr int NG = CONSUMERS / G;                 // cells per tile
    // the per-cell arrays are padded to a multiple of 192 cells (nc_pad): the
    // last tile's bulk copies stay inside them
    static_assert(192 % NG == 0, "tile size must divide the cell padding");
    static constexpr int LBYTES = NG * LMAX * (int)sizeof(T);
    static constexpr int SBYTES = NG * C::M * 4;
    static constexpr int STAGE = (LBYTES + SBYTES + 127) / 128 * 128;
    static constexpr int SU = NG * CSTRIDE;
    // resident CTAs per SM aimed for (register and shared-memory budget)
    static constexpr int MINB = sizeof(T) == 8 ? 1 : TRIPLE ? 3 : 2;
    static constexpr int BUDGET = 227 * 1024 / MINB - (SU + 127) / 128 * 128 - 1024;
    static constexpr int FIT = BUDGET / STAGE;
    static constexpr int STAGES = FIT >= 4 ? 4 : FIT >= 3 ? 3 : 2;
    static constexpr int SMEM = STAGES * STAGE + (SU + 127) / 128 * 128 + 2 * STAGES * 8;
    static constexpr int THREADS = CONSUMERS + 32;
    static_assert(SMEM <= 227 * 1024, "staging ring exceeds shared memory");
};

// min / max over the SLOT aligned lanes of a segment (xor offsets below SLOT
// stay inside it).  The whole warp takes part (full mask): callers keep the
// control flow warp-uniform.  Operands are finite or +-inf.
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }

// FP64 decisions in integer instructions.  An FP64 compare, minimum or
// maximum occupies this GPU's FP64 pipe (two lanes per clock per SM) as long
// as an FMA does; on the key below, a signed 64-bit integer that orders as
// the double does (the sign-magnitude bits with the magnitude bits of a
// negative number flipped; -0 taken as +0), they take a few integer
// instructions and give the same decisions for every non-NaN operand.  The
// key maps back to the value (a zero comes back as +0, which changes no sum
// or product the detector forms from it).  FP32 keeps the plain operations.
__device__ __forceinline__ long long okey(double x)
{
    long long b = __double_as_longlong(x);
    b = (b << 1) == 0 ? 0 : b;
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double okey_inv(long long k) { return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL)); }
__device__ __forceinline__ bool dle(float a, float b) { return a <= b; }
__device__ __forceinline__ bool dle(double a, double b) { return okey(a) <= okey(b); }
__device__ __forceinline__ bool dlt(float a, float b) { return a < b; }
__device__ __forceinline__ bool dlt(double a, double b) { return okey(a) < okey(b); }
__device__ __forceinline__ float dmaxv(float a, float b) { return a > b ? a : b; }
__device__ __forceinline__ double dmaxv(double a, double b) { return okey(a) > okey(b) ? a : b; }
__device__ __forceinline__ float dabsv(float x) { return x < 0.0f ? -x : x; }
__device__ __forceinline__ double dabsv(double x) { return fabs(x); }   // a sign-bit operation

template <int SLOT, class T>
__device__ __forceinline__ T seg_min(T v)
{
    if constexpr (sizeof(T) == 8) {
        long long k = okey(v);
#pragma unroll
        for (int o = SLOT / 2; o > 0; o >>= 1) {
            const long long y = __shfl_xor_sync(0xffffffffu, k, o);
            k = y < k ? y : k;
        }
        return okey_inv(k);
    } else {
#pragma unroll
        for (int o = SLOT / 2; o > 0; o >>= 1) v = vmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
}
template <int SLOT, class T>
__device__ __forceinline__ T seg_max(T v)
{
    if constexpr (sizeof(T) == 8) {
        long long k = okey(v);
#pragma unroll
        for (int o = SLOT / 2; o > 0; o >>= 1) {
            const long long y = __shfl_xor_sync(0xffffffffu, k, o);
            k = y > k ? y : k;
        }
        return okey_inv(k);
    } else {
#pragma unroll
        for (int o = SLOT / 2; o > 0; o >>= 1) v = vmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
}

template <class C, class T, bool WIDE = false>
__global__ void __launch_bounds__(K1Shape<C, T, WIDE>::THREADS, K1Shape<C, T, WIDE>::MINB) k_linear(KParams<T> p)
{
    using S = K1Shape<C, T, WIDE>;
    constexpr int M = C::M, NV = C::NV, D = C::D, G = S::G, NG = S::NG, ST = S::STAGES, PPL = S::PPL;
    constexpr int SLOT = S::SLOT, W = S::PER16, M4 = M / W * W, TW = M - M4;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* sU = smem + ST * S::STAGE;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + ST * S::STAGE + (S::SU + 127) / 128 * 128);
    uint64_t* empty = full + ST;
    const int64_t nc = p.nc;
    const int64_t ntiles = (nc + NG - 1) / NG;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], S::CONSUMERS / 32);
        }
        mbar_init_fence();
    }
    __syncthreads();

    if (threadIdx.x >= S::CONSUMERS) {
        // ---------------- producer warp ----------------
        // (with withhold_copies nothing is issued: the consumers' first wait
        // runs out and the launch reports the timeout; no copy is in flight)
        if (threadIdx.x == S::CONSUMERS && !p.withhold_copies) {
            int k = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
                const int s = k % ST;
                if (k >= ST && !(ok = mbar_wait(&empty[s], ((k / ST) - 1) & 1))) break;
                const int64_t c0 = tile * NG;
                const int64_t lb = p.loff[c0], le = p.loff[c0 + NG];
                const uint32_t lbytes = (uint32_t)((le - lb) * (int64_t)sizeof(T));
                unsigned char* stage = smem + s * S::STAGE;
                mbar_arrive_expect_tx(&full[s], lbytes + S::SBYTES);
                if (lbytes) bulk_g2s(stage, p.L + lb, lbytes, &full[s]);
                bulk_g2s(stage + S::LBYTES, p.sten + c0 * M, S::SBYTES, &full[s]);
            }
            if (!ok) atomicOr(p.status, 4);
            // every issued copy has landed before the CTA may exit
            const int issued = k;
            for (int j = issued - ST > 0 ? issued - ST : 0; j < issued; ++j)
                if (!mbar_wait(&full[j % ST], (j / ST) & 1)) { atomicOr(p.status, 4); break; }
        }
        return;
    }

    // ---------------- consumer warps ----------------
    // Software pipeline: while tile k is computed from shared memory, the
    // stencil states of tile k+1 are already in flight into registers.
    constexpr int MI = (M + G - 1) / G;    // stencil cells per lane
    const Grp<G> grp;
    const int gi = threadIdx.x / G, lane = grp.lane;
    T* dU4 = reinterpret_cast<T*>(sU + gi * S::CSTRIDE);          // [M][4]
    T* dU5 = reinterpret_cast<T*>(sU + gi * S::CSTRIDE + S::DU4); // [M] (five variables)
    T nu[MI][NV];                          // in-flight stencil states of the next tile
    T nuc[NV];                             // the cell
    int nnfv = 0;
    int64_t nlrel = 0;
    T nthr = T(0);
    auto fetch = [&](int64_t tile_f, int stage_f) {
        const int64_t cf = tile_f * NG + gi;
        if (cf >= nc) {
            // with several cells per warp, a group past the last cell runs on
            // a quiet dummy cell with no faces (Q = n1 = 0) and stores
            // nothing: the warp stays converged (a whole warp past the last
            // cell skips the tile)
            if constexpr (G < 32) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    nuc[v] = v == 0 ? T(1) : v == NV - 1 ? T(2.5) : T(0);
#pragma unroll
                    for (int i = 0; i < MI; ++i) nu[i][v] = nuc[v];
                }
                nnfv = 0;
                nthr = T(0);
                nlrel = 0;
            }
            return;
        }
        const int32_t* st = reinterpret_cast<const int32_t*>(smem + stage_f * S::STAGE + S::LBYTES) + gi * M;
#pragma unroll
        for (int i = 0; i < MI; ++i) {
            const int m = lane + i * G;
            if (m < M) load_cell<T, NV>(p.UA, st[m], nu[i]);
        }
        load_cell<T, NV>(p.UA, cf, nuc);
        nnfv = p.nfc[cf];
        nthr = p.dxthr[cf];
        nlrel = p.loff[cf] - p.loff[tile_f * NG];
    };
    // the producer streams constant data only; the states are the
    // predecessor's output
    pdl_wait();
    // the queue counts of this residual start at zero for the tagging
    // kernel's range reservations (their readers of the previous residual
    // have completed: they ran before the predecessor)
    if (blockIdx.x == 0 && threadIdx.x == 0) { p.counts[0] = 0; p.counts[1] = 0; }
    int k = 0;
    int64_t tile = blockIdx.x;
    bool alive = true;
    if (tile < ntiles) {
        if (!__all_sync(0xffffffffu, mbar_wait(&full[0], 0, p.wait_ns))) {
            if ((threadIdx.x & 31) == 0) atomicOr(p.status, 4);
            alive = false;
        } else {
            fetch(tile, 0);
        }
    }
    while (alive && tile < ntiles) {
        const int s = k % ST;
        const int64_t c = tile * NG + gi;
        T uc[NV], nb[NV];                  // the cell's state; face neighbour `lane` (lane < SLOT)
        const int nfv = nnfv;
        const int64_t lrel = nlrel;
        const T thr = nthr;
        const bool valid = c < nc;
        const bool run = G < 32 || valid;   // warp-uniform
        if (run) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                uc[v] = nuc[v];
                nb[v] = lane < M ? nu[0][v] : uc[v];
            }
#pragma unroll
            for (int i = 0; i < MI; ++i) {
                const int m = lane + i * G;
                if (m < M) {
                    T row[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) row[v] = nu[i][v] - uc[v];
                    if constexpr (sizeof(T) == 4) {
                        *reinterpret_cast<float4*>(dU4 + m * 4) = make_float4(row[0], row[1], row[2], row[3]);
                    } else {
                        *reinterpret_cast<double2*>(dU4 + m * 4) = make_double2(row[0], row[1]);
                        *reinterpret_cast<double2*>(dU4 + m * 4 + 2) = make_double2(row[2], row[3]);
                    }
                    if constexpr (NV == 5) dU5[m] = row[4];
                }
            }
        }
        const int64_t next = tile + gridDim.x;
        if (next < ntiles) {
            const int s1 = (k + 1) % ST;
            if (!__all_sync(0xffffffffu, mbar_wait(&full[s1], ((k + 1) / ST) & 1, p.wait_ns))) {
                if ((threadIdx.x & 31) == 0) atomicOr(p.status, 4);
                alive = false;
            } else {
                fetch(next, s1);
            }
        }
        const unsigned char* stage = smem + s * S::STAGE;
        if (run) {
            const int nf = nfv & 15, n1 = nfv >> 4, Q = nf * C::NFP;
            T w[PPL][NV];
#pragma unroll
            for (int j = 0; j < PPL; ++j)
#pragma unroll
                for (int v = 0; v < NV; ++v) w[j][v] = uc[v];
            __syncwarp();
            const T* lb = reinterpret_cast<const T*>(stage) + lrel;
            // candidate: w = U_0 + sum_m L_qm (U_m - U_0), one chunk of W
            // columns of L per 16-byte load
            if constexpr (sizeof(T) == 4) {
                float2 w01[PPL], w23[PPL];
#pragma unroll
                for (int j = 0; j < PPL; ++j) { w01[j] = make_float2(w[j][0], w[j][1]); w23[j] = make_float2(w[j][2], w[j][3]); }
#pragma unroll
                for (int m0 = 0; m0 < M4; m0 += 4) {
                    float lv[PPL][4];
#pragma unroll
                    for (int j = 0; j < PPL; ++j) {
                        const int q = lane + j * G;
                        if (q < Q) {
                            const float4 t = *reinterpret_cast<const float4*>(lb + m0 * Q + q * 4);
                            lv[j][0] = t.x; lv[j][1] = t.y; lv[j][2] = t.z; lv[j][3] = t.w;
                        } else {
                            lv[j][0] = lv[j][1] = lv[j][2] = lv[j][3] = 0.0f;
                        }
                    }
                    float4 e5 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if constexpr (NV == 5) e5 = *reinterpret_cast<const float4*>(dU5 + m0);
                    const float e5a[4] = {e5.x, e5.y, e5.z, e5.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 d = *reinterpret_cast<const float4*>(dU4 + (m0 + i) * 4);
                        const float2 d01 = make_float2(d.x, d.y), d23 = make_float2(d.z, d.w);
#pragma unroll
                        for (int j = 0; j < PPL; ++j) {
                            const float2 l2 = make_float2(lv[j][i], lv[j][i]);
                            w01[j] = __ffma2_rn(l2, d01, w01[j]);
                            w23[j] = __ffma2_rn(l2, d23, w23[j]);
                            if constexpr (NV == 5) w[j][4] = fmaf(lv[j][i], e5a[i], w[j][4]);
                        }
                    }
                }
                if constexpr (TW == 2) {
                    float lt[PPL][2];
#pragma unroll
                    for (int j = 0; j < PPL; ++j) {
                        const int q = lane + j * G;
                        if (q < Q) {
                            const float2 t = *reinterpret_cast<const float2*>(lb + M4 * Q + q * 2);
                            lt[j][0] = t.x; lt[j][1] = t.y;
                        } else {
                            lt[j][0] = lt[j][1] = 0.0f;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const float4 d = *reinterpret_cast<const float4*>(dU4 + (M4 + i) * 4);
                        const float2 d01 = make_float2(d.x, d.y), d23 = make_float2(d.z, d.w);
#pragma unroll
                        for (int j = 0; j < PPL; ++j) {
                            const float2 l2 = make_float2(lt[j][i], lt[j][i]);
                            w01[j] = __ffma2_rn(l2, d01, w01[j]);
                            w23[j] = __ffma2_rn(l2, d23, w23[j]);
                            if constexpr (NV == 5) w[j][4] = fmaf(lt[j][i], dU5[M4 + i], w[j][4]);
                        }
                    }
                }
                static_assert(TW == 0 || TW == 2, "FP32 stencil sizes are even");
#pragma unroll
                for (int j = 0; j < PPL; ++j) { w[j][0] = w01[j].x; w[j][1] = w01[j].y; w[j][2] = w23[j].x; w[j][3] = w23[j].y; }
            } else {
                static_assert(sizeof(T) == 4 || TW == 0, "FP64 stencil sizes are even");
#pragma unroll 2
                for (int m0 = 0; m0 < M; m0 += 2) {
                    double lv[PPL][2];
#pragma unroll
                    for (int j = 0; j < PPL; ++j) {
                        const int q = lane + j * G;
                        if (q < Q) {
                            const double2 t = *reinterpret_cast<const double2*>(lb + m0 * Q + q * 2);
                            lv[j][0] = t.x; lv[j][1] = t.y;
                        } else {
                            lv[j][0] = lv[j][1] = 0.0;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const double2 a = *reinterpret_cast<const double2*>(dU4 + (m0 + i) * 4);
                        const double2 b = *reinterpret_cast<const double2*>(dU4 + (m0 + i) * 4 + 2);
                        const double d[4] = {a.x, a.y, b.x, b.y};
#pragma unroll
                        for (int j = 0; j < PPL; ++j) {
#pragma unroll
                            for (int v = 0; v < 4; ++v) w[j][v] = fma(lv[j][i], d[v], w[j][v]);
                            if constexpr (NV == 5) w[j][4] = fma(lv[j][i], dU5[m0 + i], w[j][4]);
                        }
                    }
                }
            }
            const int64_t q0 = c * C::QMAX;
            const T rb = uc[0], pb = pressure<T, D>(uc, p.gamma);
            if (valid && lane == 0 && !(rb > T(0) && pb > T(0))) atomicOr(p.status, 1);
            // Harten test of the candidate at the lane's points
            const T rlim = p.h_theta * tmax(tabs(rb), p.h_eps), plim = p.h_theta * tmax(tabs(pb), p.h_eps);
            T pw[PPL];
            bool fail = false;
#pragma unroll
            for (int j = 0; j < PPL; ++j) {
                const int q = lane + j * G;
                pw[j] = pressure<T, D>(w[j], p.gamma);
                if (q < Q) {
                    store_state<T, NV>(p.FS + (q0 + q) * NV, w[j]);
                    fail = fail || !dle(dabsv(w[j][0] - rb), rlim) || !dle(dabsv(pw[j] - pb), plim);
                }
            }
            int cl = CLS_LIN;
            if (!p.forced && p.scheme == HFV_HYBRID) {
                // detector: lane l < SLOT takes face neighbour l for the
                // bounds, every lane its own face points for the classification
                const bool has = lane < n1;
                const int src = (threadIdx.x & 31) & ~(G - 1);   // the group's first lane
                const bool det = n1 > 0;
                const T pn = pressure<T, D>(nb, p.gamma);
                const T sg = p.beta_w > T(0) ? T(1) : (p.beta_w < T(0) ? T(-1) : T(0));
#pragma unroll
                for (int kind = 0; kind < NV + 1; ++kind) {
                    const bool use = kind == 0 ? (p.nad_vars & 1) : kind == 1 ? (p.nad_vars & 2) : (p.nad_vars & 4);
                    if (!use) continue;
                    const T qi = kind == 0 ? rb : kind == 1 ? pb : uc[kind - 1];
                    const T qn = kind == 0 ? nb[0] : kind == 1 ? pn : nb[kind - 1];
                    const T qj = has ? qn : qi;
                    const T dd = dabsv(qj - qi);
                    T lo = seg_min<SLOT>(qj), hi = seg_max<SLOT>(qj);
                    T dlo = seg_min<SLOT>(has ? dd : T(INFINITY));
                    T dhi = seg_max<SLOT>(has ? dd : T(-INFINITY));
                    if constexpr (S::NB_BCAST) {
                        lo = __shfl_sync(0xffffffffu, lo, src);
                        hi = __shfl_sync(0xffffffffu, hi, src);
                        dlo = __shfl_sync(0xffffffffu, dlo, src);
                        dhi = __shfl_sync(0xffffffffu, dhi, src);
                    }
                    // deactivated (smooth) unless the neighbour differences spread by thr
                    if (det && !dlt(dhi - dlo, thr)) {
                        const T range = hi - lo;
                        const T dm = dmaxv(p.alpha_m, p.beta_m * range);
                        const T dw = sg * dmaxv(p.alpha_w, dabsv(p.beta_w * range));
#pragma unroll
                        for (int j = 0; j < PPL; ++j) {
                            const int q = lane + j * G;
                            if (q < Q) {
                                const T x = kind == 0 ? w[j][0] : kind == 1 ? pw[j] : w[j][kind - 1];
                                int kc;
                                if (dle(x, lo - dm) || dle(hi + dm, x)) kc = CLS_MU;
                                else if (dlt(lo - dw, x) && dlt(x, hi + dw)) kc = CLS_LIN;
                                else kc = CLS_CW;
                                cl = kc > cl ? kc : cl;
                            }
                        }
                    }
                }
            }
            const unsigned gbits = grp.mask;
            const bool hfail = (__ballot_sync(0xffffffffu, fail) & gbits) != 0u;
            const bool any_mu = (__ballot_sync(0xffffffffu, cl == CLS_MU) & gbits) != 0u;
            const bool any_cw = (__ballot_sync(0xffffffffu, cl == CLS_CW) & gbits) != 0u;
            if (valid && lane == 0) {
                uint8_t out;
                if (p.forced) out = p.forced_cls[c];
                else if (p.scheme == HFV_HYBRID) out = any_mu ? CLS_MU : any_cw ? CLS_CW : CLS_LIN;
                else out = p.scheme == HFV_PURE_LINEAR ? CLS_LIN : p.scheme == HFV_PURE_CWENOZ ? CLS_CW : CLS_MU;
                p.raw[c] = out | (hfail ? HARTEN_FAIL : 0);
            }
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[s]);
        ++k;
        tile = next;
    }
}

}  // namespace hfv
