// noalloc.cu -- class-queue compaction that allocates nothing.
//
// Some callers cannot call cudaMalloc when they need the queues: code that
// runs inside a CUDA stream capture (an allocation there breaks the capture),
// solvers hosted by a framework whose pool allocator owns all device memory,
// or real-time host code that may not allocate after start-up.  This entry
// point gives them the same compaction as the residual pipeline (stable, in
// ascending cell order) with its block-count scratch in a file-scope device
// array instead of any allocation.  The caller still passes the class array
// and the output buffers.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hfv_internal.h"

namespace hfv {
namespace {

constexpr int kBlock = 256;                        // cells per block
constexpr int kMaxBlocks = 1 << 16;                // scratch rows: up to 16,777,216 cells
constexpr int64_t kMaxCells = (int64_t)kMaxBlocks * kBlock;

// per-block counts of the two queues; every call overwrites the entries it
// uses before reading them, so nothing needs clearing between calls
static __device__ __align__(256) int32_t g_queue_scratch[2 * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
int32_t* g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array for the current device (host code
// only knows a stand-in for it); looked up once per device
int scratch_for_current_device(int32_t** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("hfv_class_queues_static: cudaGetDevice: ") + cudaGetErrorString(e));
        return HFV_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("hfv_class_queues_static: device index " + std::to_string(dev) + " is beyond the " +
                  std::to_string(kMaxDevices) + " devices whose scratch address this library keeps");
        return HFV_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_queue_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("hfv_class_queues_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return HFV_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<int32_t*>(p);
    }
    *out = g_scratch_ptr[dev];
    return HFV_OK;
}

__device__ __forceinline__ void block_ballots(int t, int& c1, int& c2, unsigned& b1, unsigned& b2, int* s)
{
    b1 = __ballot_sync(0xffffffffu, t == 1);
    b2 = __ballot_sync(0xffffffffu, t == 2);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s[w] = __popc(b1); s[8 + w] = __popc(b2); }
    __syncthreads();
    c1 = 0;
    c2 = 0;
    for (int k = 0; k < w; ++k) { c1 += s[k]; c2 += s[8 + k]; }
}

__global__ void __launch_bounds__(kBlock) k_sq_count(const uint8_t* __restrict__ cls, int64_t n, int32_t* scratch, int nb)
{
    __shared__ int s[16];
    const int64_t c = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    const int t = c < n ? cls[c] : 255;
    int c1, c2;
    unsigned b1, b2;
    block_ballots(t, c1, c2, b1, b2, s);
    if (threadIdx.x == kBlock - 1) {
        scratch[blockIdx.x] = c1 + __popc(b1);
        scratch[nb + blockIdx.x] = c2 + __popc(b2);
    }
}

// exclusive scan of the block counts in one block; totals to counts[0..1]
__global__ void __launch_bounds__(1024) k_sq_scan(int32_t* scratch, int nb, int32_t* counts)
{
    __shared__ int part[1024];
    for (int q = 0; q < 2; ++q) {
        int32_t* b = scratch + q * nb;
        const int per = (nb + 1023) / 1024;
        const int lo = threadIdx.x * per, hi = min(lo + per, nb);
        int sum = 0;
        for (int i = lo; i < hi; ++i) sum += b[i];
        part[threadIdx.x] = sum;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        int run = part[threadIdx.x] - sum;
        for (int i = lo; i < hi; ++i) {
            const int v = b[i];
            b[i] = run;
            run += v;
        }
        if (threadIdx.x == 1023) counts[q] = part[1023];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) k_sq_scatter(const uint8_t* __restrict__ cls, int64_t n,
                                                      const int32_t* scratch, int nb, int32_t* queues)
{
    __shared__ int s[16];
    const int64_t c = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    const int t = c < n ? cls[c] : 255;
    int c1, c2;
    unsigned b1, b2;
    block_ballots(t, c1, c2, b1, b2, s);
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    if (t == 1) queues[scratch[blockIdx.x] + c1 + __popc(b1 & lt)] = (int32_t)c;
    if (t == 2) queues[n + scratch[nb + blockIdx.x] + c2 + __popc(b2 & lt)] = (int32_t)c;
}

}  // namespace
}  // namespace hfv

using namespace hfv;

extern "C" int hfv_class_queues_static(const uint8_t* cls, int64_t n_cells, int32_t* counts, int32_t* queues, void* stream)
{
    if (!cls || !counts || !queues || n_cells <= 0) {
        set_error("hfv_class_queues_static: NULL pointer or non-positive size");
        return HFV_ERR_ARG;
    }
    if (n_cells > kMaxCells) {
        set_error("hfv_class_queues_static: " + std::to_string(n_cells) + " cells exceed the static scratch limit of " +
                  std::to_string(kMaxCells));
        return HFV_ERR_ARG;
    }
    int32_t* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != HFV_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)((n_cells + kBlock - 1) / kBlock);
    note_launch();
    k_sq_count<<<nb, kBlock, 0, st>>>(cls, n_cells, scratch, nb);
    note_launch();
    k_sq_scan<<<1, 1024, 0, st>>>(scratch, nb, counts);
    note_launch();
    k_sq_scatter<<<nb, kBlock, 0, st>>>(cls, n_cells, scratch, nb, queues);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("hfv_class_queues_static: ") + cudaGetErrorString(e));
        return HFV_ERR_CUDA;
    }
    return HFV_OK;
}
