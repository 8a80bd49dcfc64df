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
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "bbx_device.cuh"

namespace {

// Scratch shared by every call: one double per block plus the ticket.
constexpr int kNoallocMaxBlocks = 4096;
constexpr long long kNoallocNodesPerBlock = 65536;  // nodes summed by one block (at most)
constexpr long long kNoallocMaxNodes = kNoallocMaxBlocks * kNoallocNodesPerBlock;  // 2^28
constexpr int kNoallocThreads = 256;

struct NoallocScratch {
    double partials[kNoallocMaxBlocks];
    unsigned int ticket;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// The scratch array's device address, looked up once per CUDA context: a
// device reset (or the release and re-creation of the primary context)
// reloads the module, so the address is looked up again when the current
// context's id differs from the one it was found in.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    unsigned long long ctx_id;  // 0: not looked up yet
    NoallocScratch* ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mu;

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;
std::once_flag g_ctx_fn_once;

// Id of the calling thread's current context (0 if it cannot be read).
unsigned long long current_context_id() {
    std::call_once(g_ctx_fn_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(fn);
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(fn);
    });
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Block b sums the rows [b R / B, (b+1) R / B) of the R = ny nz rows of the
// field (B blocks): each warp takes every (blockDim/32)-th of them, its lanes
// walking x with coalesced loads (compensated float pairs per thread, doubles
// across warps).  The last block to finish adds the per-block partials in a
// fixed order.  A row holds at most 2^28 nodes, so x and the in-row offsets
// stay 32-bit; the row's base offset is 64-bit and computed once per row.
__global__ void k_total_noalloc(const float* __restrict__ u, const uint8_t* __restrict__ mask, int nx, int ny,
                                int nz, int px, NoallocScratch* scr, double* out) {
    __shared__ double scratch[32];
    const long long rows = (long long)ny * nz;
    const long long r0 = (long long)blockIdx.x * rows / gridDim.x;
    const long long r1 = ((long long)blockIdx.x + 1) * rows / gridDim.x;
    const long long plane = (long long)px * ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    bbx::F2 acc = {0.0f, 0.0f};
    for (long long r = r0 + warp; r < r1; r += nwarps) {
        const int z = (int)(r / ny), y = (int)(r - (long long)z * ny);
        const long long base = (long long)z * plane + (long long)y * px;
        const float* ur = u + base;
        if (mask) {
            const uint8_t* mr = mask + base;
            for (unsigned x = lane; x < (unsigned)nx; x += 32)
                if (mr[x]) bbx::two_sum_add(acc, ur[x]);
        } else {
            for (unsigned x = lane; x < (unsigned)nx; x += 32) bbx::two_sum_add(acc, ur[x]);
        }
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
    // An error left by the caller's earlier work is not ours to clear or to
    // report as this call's: refuse to start, and leave it in place.
    if (cudaPeekAtLastError() != cudaSuccess) return BBX_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();  // our own failure (none was pending)
        return BBX_ERR_CUDA;
    }
    // Set-up, once per device and context, with that device current: the
    // device address of the scratch array (its host-side name is only a
    // stand-in).
    NoallocScratch* scr = nullptr;
    {
        const unsigned long long ctx = current_context_id();
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        ScratchAddr& a = g_scratch[dev];
        if (!a.ptr || ctx == 0 || a.ctx_id != ctx) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                a.ptr = nullptr;
                a.ctx_id = 0;
                return BBX_ERR_CUDA;
            }
            a.ptr = static_cast<NoallocScratch*>(p);
            a.ctx_id = ctx;
        }
        scr = a.ptr;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the ticket must start at zero (a call cut short could have left it set)
    if (cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    const long long rows = (long long)ny * nz;
    long long blocks = (n + kNoallocNodesPerBlock - 1) / kNoallocNodesPerBlock;
    if (blocks < 152) blocks = 152 < rows ? 152 : rows;  // every SM, as far as there are rows
    if (blocks > rows) blocks = rows;
    if (blocks > kNoallocMaxBlocks) blocks = kNoallocMaxBlocks;
    k_total_noalloc<<<(int)blocks, kNoallocThreads, 0, s>>>(field_dev, mask_dev, nx, ny, nz, pitch, scr, out_dev);
    if (cudaGetLastError() != cudaSuccess) return BBX_ERR_CUDA;
    return BBX_OK;
}
