// peak.cu -- CUDA-core fused multiply-add throughput of the current device:
// the ALU ceiling against which the FP64 (and FP32) residual paths are
// reported next to the HBM ceiling.  Instrumentation; the paper has no
// counterpart.  Also the FP32 kernels' integer FP32 <-> FP64 conversions and
// the FP64 kernels' reciprocal applied to an array, so that they can be
// checked against the hardware's conversions and against 1/x.
//
// Each thread runs eight independent chains of dependent FMAs (x <- a x + b
// with |a| < 1, so the values stay normal and bounded), enough independent
// work per warp to keep the FMA pipe issuing every cycle; the grid fills
// every SM with 2,048 resident threads.  The chains' sum is compared with a
// value it never takes, so the compiler keeps every FMA.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "device_common.cuh"
#include "physics.cuh"
#include "hfv_internal.h"

namespace hfv {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

static __device__ double g_fma_sink;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kUnroll; ++j)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == T(-1)) g_fma_sink = (double)s;
}

// packed FP32: two FMAs per instruction (FFMA2)
__global__ void __launch_bounds__(kThreads) k_ffma2_peak(int iters, float a, float b)
{
    float2 x[kChains / 2];
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) x[k] = make_float2((threadIdx.x + 2 * k) * 1e-3f, (threadIdx.x + 2 * k + 1) * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kUnroll; ++j)
#pragma unroll
            for (int k = 0; k < kChains / 2; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) s += x[k].x + x[k].y;
    if (s == -1.0f) g_fma_sink = (double)s;
}

int launch_peak(int kind, int iters, unsigned grid, cudaStream_t st)
{
    note_launch();
    if (kind == 0) k_fma_peak<double><<<grid, kThreads, 0, st>>>(iters, 0.999, 1e-3);
    else if (kind == 1) k_fma_peak<float><<<grid, kThreads, 0, st>>>(iters, 0.999f, 1e-3f);
    else k_ffma2_peak<<<grid, kThreads, 0, st>>>(iters, 0.999f, 1e-3f);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("hfv_fma_rate: ") + cudaGetErrorString(e));
        return HFV_ERR_CUDA;
    }
    return HFV_OK;
}

__global__ void k_rcp64(int64_t n, const double* __restrict__ in, double* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = trcp<double>(in[i]);
}

__global__ void k_convert(int to_f32, int64_t n, const void* __restrict__ in, void* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (to_f32) static_cast<float*>(out)[i] = f64_to_f32(static_cast<const double*>(in)[i]);
    else static_cast<double*>(out)[i] = f32_to_f64(static_cast<const float*>(in)[i]);
}

}  // namespace
}  // namespace hfv

using namespace hfv;

// one thread per element in blocks of 256: the grid stays below 2^31 blocks
static constexpr int64_t kMaxElems = ((int64_t(1) << 31) - 1) * 255;

extern "C" int hfv_rcp64(int64_t n, const double* in, double* out, void* stream)
{
    if (n < 0 || n > kMaxElems || (n > 0 && (!in || !out))) {
        set_error("hfv_rcp64: 0 <= n <= (2^31 - 1) * 255 and non-null buffers");
        return HFV_ERR_ARG;
    }
    if (n == 0) return HFV_OK;
    note_launch();
    k_rcp64<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, in, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("hfv_rcp64: ") + cudaGetErrorString(e));
        return HFV_ERR_CUDA;
    }
    return HFV_OK;
}

extern "C" int hfv_convert(int to_f32, int64_t n, const void* in, void* out, void* stream)
{
    if (n < 0 || n > kMaxElems || (n > 0 && (!in || !out)) || (to_f32 != 0 && to_f32 != 1)) {
        set_error("hfv_convert: to_f32 must be 0 or 1, 0 <= n <= (2^31 - 1) * 255, buffers non-null");
        return HFV_ERR_ARG;
    }
    if (n == 0) return HFV_OK;
    note_launch();
    k_convert<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(to_f32, n, in, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("hfv_convert: ") + cudaGetErrorString(e));
        return HFV_ERR_CUDA;
    }
    return HFV_OK;
}

extern "C" int hfv_fma_rate(int kind, double target_ms, double* flops_per_s, void* stream)
{
    if (!flops_per_s || kind < 0 || kind > 2 || !(target_ms > 0.0) || target_ms > 2000.0) {
        set_error("hfv_fma_rate: kind must be 0 (FP64), 1 (FP32) or 2 (packed FP32), target 0 < ms <= 2000");
        return HFV_ERR_ARG;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_error("hfv_fma_rate: no device");
        return HFV_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned grid = (unsigned)sms * (2048 / kThreads);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        set_error("hfv_fma_rate: cudaEventCreate failed");
        return HFV_ERR_CUDA;
    }
    auto timed = [&](int iters, float* ms) -> int {
        cudaEventRecord(e0, st);
        int rc = launch_peak(kind, iters, grid, st);
        cudaEventRecord(e1, st);
        if (rc != HFV_OK) return rc;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) {
            set_error("hfv_fma_rate: event timing failed");
            return HFV_ERR_CUDA;
        }
        return HFV_OK;
    };
    // calibrate the loop count to the target duration, then keep the best of three
    int iters = 64, rc;
    float ms = 0.0f;
    if ((rc = timed(iters, &ms)) == HFV_OK) {
        const double scale = target_ms / std::max(ms, 1e-3f);
        iters = (int)std::min(1e8, std::max(64.0, iters * scale));
        double best = 0.0;
        for (int rep = 0; rep < 3 && rc == HFV_OK; ++rep) {
            if ((rc = timed(iters, &ms)) != HFV_OK) break;
            const double fmas = (double)grid * kThreads * kChains * kUnroll * (double)iters;
            best = std::max(best, 2.0 * fmas / (ms * 1e-3));
        }
        *flops_per_s = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
