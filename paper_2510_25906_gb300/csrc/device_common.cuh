// device_common.cuh -- device helpers shared by the residual kernels: small
// math, cell groups of lanes, vector loads and stores of state rows.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace hfv {

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization is scheduled as its predecessor's CTAs exit, ahead of the
// predecessor's completion and memory flush; pdl_wait() returns once the
// predecessor has completed and its writes are visible (at once for a kernel
// launched without the attribute).  No kernel here triggers its dependents
// early: CTAs of a wide dependent grid waiting beside the running kernel
// slowed the quadrant step by 17 %.  So when a kernel starts, the kernel two
// places back in the stream has completed: the code ahead of a kernel's wait
// reads only constant data or data written two or more kernels back, and
// writes nothing.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// asynchronous copy of one 4- or 8-byte element from global to shared
// memory (completed by cp_async_wait_all in the issuing thread; other lanes
// read it after a barrier)
template <class T>
__device__ __forceinline__ void cp_async(T* dst, const T* src)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element copies only");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"((int)sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }
template <class T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <class T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

// FP32 <-> FP64 conversions in integer arithmetic on the IEEE 754 binary32 /
// binary64 bit layouts, for the FP32 kernels: the conversion instructions
// issue to the FP64 pipe, which on this GPU executes two lanes per clock per
// SM (a warp's conversion holds it for 16 cycles), while these take a few
// integer instructions.  Normal numbers and zeros take the integer path and
// give exactly the conversion instruction's result (FP32 -> FP64 is exact;
// FP64 -> FP32 rounds to nearest, ties to even); subnormal, out-of-range,
// infinite and NaN operands fall back to the instruction.
__device__ __forceinline__ double f32_to_f64(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e - 1u < 254u) {
        // sign | exponent rebiased 127 -> 1023 | the 23 fraction bits, the
        // top 20 in the high word and the last 3 at the top of the low word
        const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
        return __hiloint2double((int)hi, (int)(b << 29));
    }
    if ((b << 1) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    return (double)f;
}
__device__ __forceinline__ float f64_to_f32(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t e = (hi >> 20) & 0x7ffu;
    if (e - 897u < 254u) {
        // a normal FP32 exponent (1..254 after rebiasing): keep 23 of the 52
        // fraction bits and round on the 29 dropped ones; a carry out of
        // the fraction steps the exponent (to infinity past the largest float)
        uint32_t r = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
        const uint32_t rest = lo & 0x1fffffffu;
        r += (uint32_t)(rest > 0x10000000u) | ((uint32_t)(rest == 0x10000000u) & (r & 1u));
        return __uint_as_float(r);
    }
    if (((hi << 1) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    return (float)x;
}

// an FP64 state value in the residual's precision T
template <class T>
__device__ __forceinline__ T to_t(double x)
{
    if constexpr (sizeof(T) == 4) return f64_to_f32(x);
    else return x;
}

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

// ---------------------------------------------------------------------------
// cell groups: G lanes (a power of two <= 32, inside one warp) own one cell;
// lane q handles face point q.  Reductions stay inside the group.
// ---------------------------------------------------------------------------
template <int G>
struct Grp {
    unsigned mask;
    int lane;
    __device__ __forceinline__ Grp()
    {
        lane = threadIdx.x & (G - 1);
        const int base = (threadIdx.x & 31) & ~(G - 1);
        mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << base);
    }
    template <class T>
    __device__ __forceinline__ T max(T v) const
    {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) { T w = __shfl_xor_sync(mask, v, o); v = w > v ? w : v; }
        return v;
    }
    template <class T>
    __device__ __forceinline__ T min(T v) const
    {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) { T w = __shfl_xor_sync(mask, v, o); v = w < v ? w : v; }
        return v;
    }

    template <class T>
    __device__ __forceinline__ T sum(T v) const
    {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
        return v;
    }
    __device__ __forceinline__ bool any(bool b) const { return (__ballot_sync(mask, b) & mask) != 0u; }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
};

// contiguous row of M values with the widest aligned vector loads (rows start
// at (c * QMAX + q) * M elements: 16-byte aligned when M * sizeof(T) % 16 == 0)
template <class T, int M>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T (&r)[M])
{
    if constexpr (sizeof(T) == 4 && M % 4 == 0) {
#pragma unroll
        for (int m = 0; m < M; m += 4) {
            float4 v = __ldg(reinterpret_cast<const float4*>(p + m));
            r[m] = v.x; r[m + 1] = v.y; r[m + 2] = v.z; r[m + 3] = v.w;
        }
    } else if constexpr (sizeof(T) == 4 && M % 2 == 0) {
#pragma unroll
        for (int m = 0; m < M; m += 2) {
            float2 v = __ldg(reinterpret_cast<const float2*>(p + m));
            r[m] = v.x; r[m + 1] = v.y;
        }
    } else if constexpr (sizeof(T) == 8 && M % 2 == 0) {
#pragma unroll
        for (int m = 0; m < M; m += 2) {
            double2 v = __ldg(reinterpret_cast<const double2*>(p + m));
            r[m] = v.x; r[m + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int m = 0; m < M; ++m) r[m] = __ldg(p + m);
    }
}

template <class T, int M>
__device__ __forceinline__ void load_row_smem(const T* p, T (&r)[M])
{
    if constexpr (sizeof(T) == 4 && M % 4 == 0) {
#pragma unroll
        for (int m = 0; m < M; m += 4) {
            float4 v = *reinterpret_cast<const float4*>(p + m);
            r[m] = v.x; r[m + 1] = v.y; r[m + 2] = v.z; r[m + 3] = v.w;
        }
    } else if constexpr (sizeof(T) == 4 && M % 2 == 0) {
#pragma unroll
        for (int m = 0; m < M; m += 2) {
            float2 v = *reinterpret_cast<const float2*>(p + m);
            r[m] = v.x; r[m + 1] = v.y;
        }
    } else if constexpr (sizeof(T) == 8 && M % 2 == 0) {
#pragma unroll
        for (int m = 0; m < M; m += 2) {
            double2 v = *reinterpret_cast<const double2*>(p + m);
            r[m] = v.x; r[m + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int m = 0; m < M; ++m) r[m] = p[m];
    }
}

template <class T, int NV>
__device__ __forceinline__ void store_state(T* __restrict__ p, const T (&w)[NV])
{
    if constexpr (sizeof(T) == 4 && NV == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(w[0], w[1], w[2], w[3]);
    } else if constexpr (sizeof(T) == 8 && NV == 4) {
        reinterpret_cast<double2*>(p)[0] = make_double2(w[0], w[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(w[2], w[3]);
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) p[v] = w[v];
    }
}

template <class T, int NV>
__device__ __forceinline__ void load_state(const T* __restrict__ p, T (&w)[NV])
{
    if constexpr (sizeof(T) == 4 && NV == 4) {
        float4 v = *reinterpret_cast<const float4*>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if constexpr (sizeof(T) == 8 && NV == 4) {
        double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = p[v];
    }
}

// cell-major state rows: P = 4 values (2D) or 8 (3D, 5 used), 16-byte aligned
template <int NV>
struct AoSP {
    static constexpr int P = NV == 4 ? 4 : 8;
};

template <class T, int NV>
__device__ __forceinline__ void load_cell(const T* __restrict__ UA, int64_t c, T (&u)[NV])
{
    const T* q = UA + c * AoSP<NV>::P;
    if constexpr (sizeof(T) == 4) {
        float4 a = __ldg(reinterpret_cast<const float4*>(q));
        u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
    } else {
        double2 a = __ldg(reinterpret_cast<const double2*>(q)), b = __ldg(reinterpret_cast<const double2*>(q) + 1);
        u[0] = a.x; u[1] = a.y; u[2] = b.x; u[3] = b.y;
    }
    if constexpr (NV == 5) u[4] = __ldg(q + 4);
}

}  // namespace hfv
