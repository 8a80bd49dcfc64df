// Tissue sum of one field without any device allocation.
//
// Some callers cannot allocate device memory: code that runs inside a
// framework which owns every allocation through its own pool, a real-time
// loop that must never call cudaMalloc (it may synchronise the device and
// has unbounded latency), or a context with a fixed memory budget that was
// reserved up front.  bbx_total_noalloc serves them: the caller passes the
// field, the mask and the output; the per-block partial sums and the
// completion ticket live in a fixed, file-scope device array that the
// library image holds for the lifetime of the process on every GPU that
// loads it.
#include <cuda_runtime.h>

#include <mutex>

#include "bbx_device.cuh"

namespace {

// Scratch shared by every call: one double per block plus the ticket.
constexpr int kNoallocMaxBlocks = 4096;
constexpr long long kNoallocNodesPerBlock = 65536;  // nodes summed by one block
constexpr long long kNoallocMaxNodes = kNoallocMaxBlocks * kNoallocNodesPerBlock;  // 2^28

struct NoallocScratch {
    double partials[kNoallocMaxBlocks];
    unsigned int ticket;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
NoallocScratch* g_scratch_ptr[kMaxDevices] = {};
std::once_flag g_scratch_once[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices] = {};

// Each block sums its own range of kNoallocNodesPerBlock nodes (compensated
// float pairs per thread, doubles across warps); the last block to finish
// adds the per-block partials in a fixed order.
__global__ void k_total_noalloc(const float* __restrict__ u, const uint8_t* __restrict__ mask, int nx, int ny,
                                int nz, int px, NoallocScratch* scr, double* out) {
    __shared__ double scratch[32];
    const long long n = (long long)nx * ny * nz;
    const long long b0 = (long long)blockIdx.x * kNoallocNodesPerBlock;
    const long long b1 = b0 + kNoallocNodesPerBlock < n ? b0 + kNoallocNodesPerBlock : n;
    const long long plane = (long long)px * ny;
    bbx::F2 acc = {0.0f, 0.0f};
    for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const int x = int(i % nx);
        const long long r = i / nx;
        const int y = int(r % ny);
        const int z = int(r / ny);
        const long long gi = z * plane + (long long)y * px + x;
        if (!mask || mask[gi]) bbx::two_sum_add(acc, u[gi]);
    }
    const double bs = bbx::block_sum_double((double)acc.hi + (double)acc.lo, scratch);
    bbx::grid_total_finalize(bs, scr->partials, &scr->ticket, out, nullptr, false, scratch);
}

}  // namespace

extern "C" int bbx_total_noalloc(const float* field_dev, const uint8_t* mask_dev, int nx, int ny, int nz,
                                 int pitch, double* out_dev, void* cuda_stream) {
    if (!field_dev || !out_dev || nx <= 0 || ny <= 0 || nz <= 0 || pitch < nx) return BBX_ERR_ARG;
    const long long n = (long long)nx * ny * nz;
    if (n > kNoallocMaxNodes) return BBX_ERR_ARG;  // beyond the fixed scratch: at most 2^28 nodes
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    // Set-up, once per device, with that device current: the device address
    // of the scratch array (its host-side name is only a stand-in).
    std::call_once(g_scratch_once[dev], [dev] {
        void* p = nullptr;
        g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (g_scratch_err[dev] == cudaSuccess) g_scratch_ptr[dev] = static_cast<NoallocScratch*>(p);
        else cudaGetLastError();
    });
    if (g_scratch_err[dev] != cudaSuccess || !g_scratch_ptr[dev]) return BBX_ERR_CUDA;
    NoallocScratch* scr = g_scratch_ptr[dev];
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the ticket must start at zero (a call cut short could have left it set)
    if (cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    const int blocks = (int)((n + kNoallocNodesPerBlock - 1) / kNoallocNodesPerBlock);
    k_total_noalloc<<<blocks, 256, 0, s>>>(field_dev, mask_dev, nx, ny, nz, pitch, scr, out_dev);
    if (cudaGetLastError() != cudaSuccess) return BBX_ERR_CUDA;
    return BBX_OK;
}
