// Host runtime of the C ABI in include/bbx.h, plus the set-up kernels
// (fibre normalisation, tissue bricks, rest state) and the standalone
// double-precision tissue reduction.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "bbx_device.cuh"

namespace bbx {
StepKernel step_kernel_fhn(bool masked, bool aniso, int ty);
StepKernel step_kernel_barkley(bool masked, bool aniso, int ty);
StepKernel step_kernel_br(bool masked, bool aniso, int ty);
StepKernel step_kernel_zfk(bool masked, bool aniso, int ty);
StepKernel step_kernel_diffusion(bool masked, bool aniso, int ty);
}  // namespace bbx

using namespace bbx;

namespace {

constexpr long long kWaitLimitCycles = 4000000000LL;  // about 2 s of SM clock
constexpr long long kPoisonWaitLimit = 2000000LL;     // about 1 ms
constexpr int kMaxPartials = 152 * 32;
constexpr int kErrFibre = 4;

int model_nvars(int model) {
    switch (model) {
        case BBX_FHN: return 2;
        case BBX_BARKLEY: return 2;
        case BBX_BR: return 8;
        case BBX_ZFK: return 1;
        case BBX_DIFFUSION: return 1;
    }
    return 0;
}

double model_threshold(int model) {
    switch (model) {
        case BBX_FHN: return 0.0;
        case BBX_BR: return -40.0;
        default: return 0.5;
    }
}

// defaults of each model's parameter list (bbx.h)
int model_defaults(int model, double* p) {
    switch (model) {
        case BBX_FHN: p[0] = 0.3; p[1] = 0.71; p[2] = 0.5; return 3;
        case BBX_BARKLEY: p[0] = 0.75; p[1] = 0.02; p[2] = 0.02; return 3;
        case BBX_BR: p[0] = 4.0; p[1] = 0.003; p[2] = 50.0; p[3] = 0.09; return 4;
        case BBX_ZFK: p[0] = 0.13; return 1;
        case BBX_DIFFUSION: return 0;
    }
    return -1;
}

// parameters in the form the kernels use (see Model<> in bbx_device.cuh)
void model_kernel_params(int model, const double* p, float* mp) {
    for (int i = 0; i < 8; ++i) mp[i] = 0.0f;
    switch (model) {
        case BBX_FHN: mp[0] = float(1.0 / p[0]); mp[1] = float(p[0]); mp[2] = float(p[1]); mp[3] = float(p[2]); break;
        case BBX_BARKLEY: mp[0] = float(1.0 / p[0]); mp[1] = float(p[1]); mp[2] = float(1.0 / p[2]); break;
        case BBX_BR: for (int i = 0; i < 4; ++i) mp[i] = float(p[i]); break;
        case BBX_ZFK: mp[0] = float(p[0]); break;
        default: break;
    }
}

StepKernel lookup_kernel(int model, bool masked, bool aniso, int ty) {
    switch (model) {
        case BBX_FHN: return step_kernel_fhn(masked, aniso, ty);
        case BBX_BARKLEY: return step_kernel_barkley(masked, aniso, ty);
        case BBX_BR: return step_kernel_br(masked, aniso, ty);
        case BBX_ZFK: return step_kernel_zfk(masked, aniso, ty);
        case BBX_DIFFUSION: return step_kernel_diffusion(masked, aniso, ty);
    }
    return StepKernel{nullptr, 0, 0, 0};
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool get_encoder() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode != nullptr;
}

bool encode(CUtensorMap* m, CUtensorMapDataType dt, int rank, void* base, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box) {
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = g_encode(m, dt, rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------------------
// set-up kernels
// ------------------------------------------------------------------------

// Normalise interleaved fibres into the SoA field [3][nz][ny][pxf] whose rows
// are stored from x = -4 (storage column x + 4) with the x-padding filled by
// the nearest in-array fibre (clamped); a zero vector at a tissue node sets
// the error bit.  Void nodes get 0.
__global__ void k_fibres(const float* __restrict__ in, int nx, int ny, int nz, int pxf, long long fplane,
                         long long fvol, const uint8_t* __restrict__ mask, int px, long long plane,
                         float* __restrict__ out, int* err) {
    const long long n = (long long)pxf * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int xs = int(i % pxf);
        const long long r = i / pxf;
        const int y = int(r % ny);
        const int z = int(r / ny);
        const int x = min(max(xs - 4, 0), nx - 1);
        const bool real = (xs - 4) == x;
        const long long src = (long long)x + (long long)nx * (y + (long long)ny * z);
        const bool tissue = mask ? mask[z * plane + (long long)y * px + x] != 0 : true;
        const float fx = in[3 * src], fy = in[3 * src + 1], fz = in[3 * src + 2];
        const float n2 = fx * fx + fy * fy + fz * fz;
        float ox = 0.f, oy = 0.f, oz = 0.f;
        if (tissue) {
            if (!(n2 > 0.0f) || !isfinite(n2)) {
                if (real) atomicOr(err, kErrFibre);
            } else {
                const float nr = __fsqrt_rn(n2);
                ox = __fdiv_rn(fx, nr);
                oy = __fdiv_rn(fy, nr);
                oz = __fdiv_rn(fz, nr);
            }
        }
        const long long o = z * fplane + (long long)y * pxf + xs;
        out[o] = ox;
        out[fvol + o] = oy;
        out[2 * fvol + o] = oz;
    }
}

// Device mask byte: bit 0 tissue, bit 1 set when all 18 neighbours of the
// 19-point stencil (faces and edges) are tissue nodes inside the array.
__global__ void k_mask_interior(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int nx, int ny, int nz,
                                int px, long long plane) {
    const long long n = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = int(i % nx);
        const long long r = i / nx;
        const int y = int(r % ny);
        const int z = int(r / ny);
        const long long gi = z * plane + (long long)y * px + x;
        uint8_t m = in[gi] ? MASK_TISSUE : 0;
        if (m) {
            bool all = true;
            for (int dz = -1; dz <= 1 && all; ++dz)
                for (int dy = -1; dy <= 1 && all; ++dy)
                    for (int dx = -1; dx <= 1 && all; ++dx) {
                        const int nnz = (dx != 0) + (dy != 0) + (dz != 0);
                        if (nnz == 0 || nnz == 3) continue;
                        const int X = x + dx, Y = y + dy, Z = z + dz;
                        if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) all = false;
                        else if (!in[Z * plane + (long long)Y * px + X]) all = false;
                    }
            if (all) m |= MASK_INTERIOR;
        }
        out[gi] = m;
    }
}

// One block per brick: does the brick hold any tissue node?
__global__ void k_brick_flags(const uint8_t* __restrict__ mask, int nx, int ny, int nz, int px, long long plane,
                              int ty, int zb, int nbx, int nby, uint8_t* flags) {
    const int id = blockIdx.x;
    const int bx = id % nbx, by = (id / nbx) % nby, bz = id / (nbx * nby);
    const int x0 = bx * kTileX, y0 = by * ty, z0 = bz * zb;
    const int cells = kTileX * ty * zb;
    int any = 0;
    for (int c = threadIdx.x; c < cells && !any; c += blockDim.x) {
        const int x = x0 + c % kTileX;
        const int y = y0 + (c / kTileX) % ty;
        const int z = z0 + c / (kTileX * ty);
        if (x < nx && y < ny && z < nz) any = mask[z * plane + (long long)y * px + x] != 0;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) flags[id] = any ? 1 : 0;
}

// Ordered stream compaction of the flags by one block (1024 threads).
__global__ void k_compact(const uint8_t* __restrict__ flags, long long n, int* __restrict__ out,
                          long long* count) {
    __shared__ int warp_sums[32];
    __shared__ long long base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long c0 = 0; c0 < n; c0 += blockDim.x) {
        const long long i = c0 + threadIdx.x;
        const int f = (i < n) ? flags[i] : 0;
        int incl = f;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int ws = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += v;
            }
            warp_sums[lane] = ws;  // inclusive over warps
        }
        __syncthreads();
        const int before = (warp > 0 ? warp_sums[warp - 1] : 0) + incl - f;
        if (f) out[base + before] = (int)i;
        __syncthreads();
        if (threadIdx.x == 0) base += warp_sums[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

// Rest state of a model, one thread.  FHN: Newton on the cubic (double);
// BR: the space-clamped cell integrated for 10 s (dt = 0.05 ms) by the
// kernel's own update; Barkley, ZFK, diffusion: 0.
__global__ void k_rest(int model, const float* mp, double beta_d, double gamma_d, float* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < 8; ++i) out[i] = 0.0f;
    if (model == BBX_FHN) {
        double u = -1.0;
        for (int it = 0; it < 100; ++it) {
            const double F = u - u * u * u / 3.0 - (u + beta_d) / gamma_d;
            const double dF = 1.0 - u * u - 1.0 / gamma_d;
            u -= F / dF;
        }
        out[0] = float(u);
        out[1] = float((u + beta_d) / gamma_d);
    } else if (model == BBX_BR) {
        float y[8] = {-84.0f, 1e-7f, 0.0f, 0.0f, 1.0f, 1.0f, 0.0f, 1.0f};
        float p[8];
        for (int i = 0; i < 8; ++i) p[i] = mp[i];
        for (int n = 0; n < 200000; ++n) Model<BBX_BR>::update(p, y, 0.0f, 0.0f, 0.05f);
        for (int i = 0; i < 8; ++i) out[i] = y[i];
    }
}

__global__ void k_fill_state(float* __restrict__ st, int S, long long vol, const float* __restrict__ rest) {
    const long long n = (long long)S * vol;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        st[i] = rest[i / vol];
}

__global__ void k_fill_int(int32_t* __restrict__ p, long long n, int32_t v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// Tissue sum of one pitched field: compensated float pairs per thread,
// doubles across warps and blocks, deterministic last-block finalisation.
// Uses a scratch array of one double per block and a ticket counter.
__global__ void k_total(const float* __restrict__ u, const uint8_t* __restrict__ mask, int nx, int ny, int nz,
                        int px, long long plane, double* partials, unsigned int* ticket, double* out, int* err) {
    __shared__ double scratch[32];
    const long long n = (long long)nx * ny * nz;
    F2 acc = {0.0f, 0.0f};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = int(i % nx);
        const long long r = i / nx;
        const int y = int(r % ny);
        const int z = int(r / ny);
        const long long gi = z * plane + (long long)y * px + x;
        if (!mask || mask[gi]) two_sum_add(acc, u[gi]);
    }
    const double bs = block_sum_double((double)acc.hi + (double)acc.lo, scratch);
    grid_total_finalize(bs, partials, ticket, out, err, false, scratch);
}

template <typename T>
cudaError_t dmalloc(T** p, size_t bytes) {
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

}  // namespace

// ---------------------------------------------------------------------------
// the grid object
// ---------------------------------------------------------------------------

struct bbx_grid {
    int nx = 0, ny = 0, nz = 0, px = 0;
    double h = 1.0;
    long long plane = 0, vol = 0, ncell = 0;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;

    uint8_t* d_mask = nullptr;
    long long n_tissue = 0;
    float* d_fib = nullptr;  // [3][nz][ny][pxf], x stored from -4 (clamped padding)
    int pxf = 0;
    long long fplane = 0, fvol = 0;
    bool aniso = false;
    double Dpar = 1.0, Dperp = 1.0;

    int model = 0, S = 0;
    double par[8] = {0};
    double theta = 0.0;
    float* d_state[2] = {nullptr, nullptr};
    bool bound = false;
    int cur = 0;
    int32_t* d_act = nullptr;
    float* d_rest = nullptr;  // 8 floats
    float* d_mp = nullptr;    // 8 floats

    uint8_t* d_stim = nullptr;
    double stim_amp = 0, t_on = 0, t_off = 0;

    double t = 0.0;
    long long n = 0;
    bool stepped = false;

    int ty = 8, zb = 16;
    int nbx = 0, nby = 0, nbz = 0;
    int* d_bricks = nullptr;
    long long n_bricks = 0;
    std::vector<int> h_bricks;      // host copy of the active brick ids (masked grids)
    int4* d_pieces = nullptr;       // balanced per-CTA work schedule
    int* d_cta_off = nullptr;
    size_t pieces_cap = 0, off_cap = 0;
    long long n_planes = 0;         // column-planes in the schedule

    double* d_partials = nullptr;
    unsigned int* d_ticket = nullptr;
    double* d_total = nullptr;   // written by each step
    double* d_total2 = nullptr;  // written by bbx_total
    int* d_err = nullptr;

    CUtensorMap tm_u[2], tm_s[2], tm_f, tm_m;
    bool maps_ok = false;
    StepKernel kern = {nullptr, 0, 0, 0};
    int grid_ctas = 0;
    int poison = 0;
};

namespace {

int fail_cuda(cudaError_t e) {
    (void)e;
    cudaGetLastError();  // do not let a failed call's error surface in a later launch check
    return BBX_ERR_CUDA;
}

#define BBX_CUDA(call)                                       \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return fail_cuda(e_);         \
    } while (0)

int n_blocks_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return (int)b;
}

// (Re)build the brick list for the current tile shape.
int build_bricks(bbx_grid* g) {
    g->nbx = (g->nx + kTileX - 1) / kTileX;
    g->nby = (g->ny + g->ty - 1) / g->ty;
    g->nbz = (g->nz + g->zb - 1) / g->zb;
    const long long nb = (long long)g->nbx * g->nby * g->nbz;
    if (nb > 0x7fffffffLL) return BBX_ERR_ARG;
    if (g->d_bricks) {
        cudaFree(g->d_bricks);
        g->d_bricks = nullptr;
    }
    if (!g->d_mask) {
        g->n_bricks = nb;
        return BBX_OK;
    }
    uint8_t* flags = nullptr;
    long long* d_count = nullptr;
    if (dmalloc(&flags, nb) != cudaSuccess) return BBX_ERR_NOMEM;
    if (dmalloc(&g->d_bricks, sizeof(int) * nb) != cudaSuccess || dmalloc(&d_count, sizeof(long long)) != cudaSuccess) {
        cudaFree(flags);
        return BBX_ERR_NOMEM;
    }
    k_brick_flags<<<(unsigned)nb, 256, 0, g->stream>>>(g->d_mask, g->nx, g->ny, g->nz, g->px, g->plane, g->ty,
                                                        g->zb, g->nbx, g->nby, flags);
    k_compact<<<1, 1024, 0, g->stream>>>(flags, nb, g->d_bricks, d_count);
    long long cnt = 0;
    cudaError_t e = cudaMemcpyAsync(&cnt, d_count, sizeof(long long), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    cudaFree(flags);
    cudaFree(d_count);
    if (e != cudaSuccess) return BBX_ERR_CUDA;
    g->n_bricks = cnt;
    g->h_bricks.resize((size_t)cnt);
    if (cnt > 0) {
        if (cudaMemcpy(g->h_bricks.data(), g->d_bricks, sizeof(int) * cnt, cudaMemcpyDeviceToHost) != cudaSuccess)
            return BBX_ERR_CUDA;
    }
    return BBX_OK;
}

// Balanced work schedule for `ctas` CTAs: the active columns (64 x TY nodes
// in x, y) with their active z-runs are concatenated column by column, and
// each CTA receives an equal share of the column-planes as contiguous pieces,
// so no CTA idles while others finish a last brick.
int build_schedule(bbx_grid* g, int ctas) {
    struct Seg {
        int x0, y0, z0, z1;
    };
    std::vector<Seg> segs;
    if (!g->d_mask) {
        for (int by = 0; by < g->nby; ++by)
            for (int bx = 0; bx < g->nbx; ++bx) segs.push_back({bx * kTileX, by * g->ty, 0, g->nz});
    } else {
        // brick ids are bx + nbx*(by + nby*bz); regroup by column, z ascending
        const long long ncol = (long long)g->nbx * g->nby;
        std::vector<std::vector<int>> col((size_t)ncol);
        for (int id : g->h_bricks) col[(size_t)(id % ncol)].push_back((int)(id / ncol));
        for (long long cidx = 0; cidx < ncol; ++cidx) {
            const std::vector<int>& zs = col[(size_t)cidx];
            const int bx = (int)(cidx % g->nbx), by = (int)(cidx / g->nbx);
            size_t i = 0;
            while (i < zs.size()) {
                size_t j = i;
                while (j + 1 < zs.size() && zs[j + 1] == zs[j] + 1) ++j;
                segs.push_back({bx * kTileX, by * g->ty, zs[i] * g->zb, std::min((zs[j] + 1) * g->zb, g->nz)});
                i = j + 1;
            }
        }
    }
    long long T = 0;
    for (const Seg& sg : segs) T += sg.z1 - sg.z0;
    g->n_planes = T;
    if (T == 0) return BBX_OK;
    if (ctas > T) ctas = (int)T;
    std::vector<int4> pieces;
    std::vector<int> off((size_t)ctas + 1, 0);
    size_t si = 0;
    long long consumed = 0;  // planes of segs[si] already handed out
    for (int c = 0; c < ctas; ++c) {
        off[c] = (int)pieces.size();
        long long need = (long long)(c + 1) * T / ctas - (long long)c * T / ctas;
        while (need > 0 && si < segs.size()) {
            const Seg& sg = segs[si];
            const long long avail = (sg.z1 - sg.z0) - consumed;
            const long long take = std::min(avail, need);
            const int z0 = sg.z0 + (int)consumed;
            pieces.push_back(make_int4(sg.x0, sg.y0, z0, z0 + (int)take));
            need -= take;
            consumed += take;
            if (consumed == sg.z1 - sg.z0) {
                ++si;
                consumed = 0;
            }
        }
    }
    off[ctas] = (int)pieces.size();
    if (pieces.size() > g->pieces_cap) {
        cudaFree(g->d_pieces);
        g->d_pieces = nullptr;
        if (dmalloc(&g->d_pieces, sizeof(int4) * pieces.size()) != cudaSuccess) return BBX_ERR_NOMEM;
        g->pieces_cap = pieces.size();
    }
    if (off.size() > g->off_cap) {
        cudaFree(g->d_cta_off);
        g->d_cta_off = nullptr;
        if (dmalloc(&g->d_cta_off, sizeof(int) * off.size()) != cudaSuccess) return BBX_ERR_NOMEM;
        g->off_cap = off.size();
    }
    if (cudaMemcpy(g->d_pieces, pieces.data(), sizeof(int4) * pieces.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->d_cta_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return BBX_ERR_CUDA;
    g->grid_ctas = ctas;
    return BBX_OK;
}

// Tensor maps and kernel choice for the current model / tiling / buffers.
int prepare(bbx_grid* g) {
    g->maps_ok = false;
    if (!g->model || !g->d_state[0]) return BBX_ERR_STATE;
    if (!get_encoder()) return BBX_ERR_CUDA;
    StepKernel k = lookup_kernel(g->model, g->d_mask != nullptr, g->aniso, g->ty);
    if (!k.fn) return BBX_ERR_UNSUPPORTED;
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    if (k.smem + 2048 > smem_optin) return BBX_ERR_UNSUPPORTED;  // this tile shape does not fit this model
    if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, k.threads, k.smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return BBX_ERR_UNSUPPORTED;
    }
    long long ctas = (long long)per_sm * g->num_sms;
    if (ctas > kMaxPartials) ctas = kMaxPartials;
    g->grid_ctas = 1;
    g->kern = k;
    {
        int rc = build_schedule(g, (int)ctas);
        if (rc) return rc;
    }

    const int ty = g->ty;
    const cuuint64_t fdims3[3] = {(cuuint64_t)g->nx, (cuuint64_t)g->ny, (cuuint64_t)g->nz};
    const cuuint64_t fstr3[2] = {(cuuint64_t)g->px * 4, (cuuint64_t)g->plane * 4};
    const cuuint32_t ubox[3] = {(cuuint32_t)(kTileX + 8), (cuuint32_t)(ty + 2), 1};
    const cuuint64_t sdims4[4] = {(cuuint64_t)g->nx, (cuuint64_t)g->ny, (cuuint64_t)g->nz, (cuuint64_t)g->S};
    const cuuint64_t str4[3] = {(cuuint64_t)g->px * 4, (cuuint64_t)g->plane * 4, (cuuint64_t)g->vol * 4};
    const cuuint32_t sbox[4] = {(cuuint32_t)kTileX, (cuuint32_t)ty, 1, (cuuint32_t)(g->S > 1 ? g->S - 1 : 1)};
    for (int b = 0; b < 2; ++b) {
        if (!encode(&g->tm_u[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, g->d_state[b], fdims3, fstr3, ubox))
            return BBX_ERR_CUDA;
        if (g->S > 1) {
            if (!encode(&g->tm_s[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->d_state[b], sdims4, str4, sbox))
                return BBX_ERR_CUDA;
        } else {
            g->tm_s[b] = g->tm_u[b];
        }
    }
    if (g->aniso) {
        const cuuint64_t fd4[4] = {(cuuint64_t)g->pxf, (cuuint64_t)g->ny, (cuuint64_t)g->nz, 3};
        const cuuint64_t fstr4[3] = {(cuuint64_t)g->pxf * 4, (cuuint64_t)g->fplane * 4, (cuuint64_t)g->fvol * 4};
        const cuuint32_t fbox[4] = {(cuuint32_t)(kTileX + 8), (cuuint32_t)(ty + 2), 1, 3};
        if (!encode(&g->tm_f, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->d_fib, fd4, fstr4, fbox)) return BBX_ERR_CUDA;
    } else {
        g->tm_f = g->tm_u[0];
    }
    if (g->d_mask) {
        const cuuint64_t mstr[2] = {(cuuint64_t)g->px, (cuuint64_t)g->plane};
        const cuuint32_t mbox[3] = {(cuuint32_t)(kTileX + 32), (cuuint32_t)(ty + 2), 1};
        if (!encode(&g->tm_m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, g->d_mask, fdims3, mstr, mbox)) return BBX_ERR_CUDA;
    } else {
        g->tm_m = g->tm_u[0];
    }
    g->maps_ok = true;
    return BBX_OK;
}

int check_sticky(bbx_grid* g) {
    int err = 0;
    BBX_CUDA(cudaMemcpyAsync(&err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    if (err & ERRBIT_TIMEOUT) return BBX_ERR_TIMEOUT;
    if (err & ERRBIT_NAN) return BBX_ERR_NAN;
    return BBX_OK;
}

int copy_in(bbx_grid* g, void* dst, const void* src, size_t elem) {
    BBX_CUDA(cudaMemcpy2DAsync(dst, (size_t)g->px * elem, src, (size_t)g->nx * elem, (size_t)g->nx * elem,
                               (size_t)g->ny * g->nz, cudaMemcpyHostToDevice, g->stream));
    return BBX_OK;
}

int copy_out(bbx_grid* g, void* dst, const void* src, size_t elem) {
    BBX_CUDA(cudaMemcpy2DAsync(dst, (size_t)g->nx * elem, src, (size_t)g->px * elem, (size_t)g->nx * elem,
                               (size_t)g->ny * g->nz, cudaMemcpyDeviceToHost, g->stream));
    return BBX_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char* bbx_status_string(int s) {
    switch (s) {
        case BBX_OK: return "ok";
        case BBX_ERR_ARG: return "invalid argument";
        case BBX_ERR_CUDA: return "CUDA call failed";
        case BBX_ERR_FIBRE: return "zero fibre vector at a tissue node";
        case BBX_ERR_UNSTABLE: return "time step above the explicit diffusion stability bound";
        case BBX_ERR_NAN: return "non-finite V produced by a step";
        case BBX_ERR_TIMEOUT: return "bounded in-kernel wait timed out";
        case BBX_ERR_STATE: return "call out of order";
        case BBX_ERR_NOMEM: return "device allocation failed";
        case BBX_ERR_UNSUPPORTED: return "no compiled kernel for this configuration";
    }
    return "unknown status";
}

void bbx_destroy_grid(bbx_grid* g) {
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    cudaFree(g->d_mask);
    cudaFree(g->d_fib);
    if (!g->bound) {
        cudaFree(g->d_state[0]);
        cudaFree(g->d_state[1]);
    }
    cudaFree(g->d_act);
    cudaFree(g->d_rest);
    cudaFree(g->d_mp);
    cudaFree(g->d_stim);
    cudaFree(g->d_bricks);
    cudaFree(g->d_pieces);
    cudaFree(g->d_cta_off);
    cudaFree(g->d_partials);
    cudaFree(g->d_ticket);
    cudaFree(g->d_total);
    cudaFree(g->d_total2);
    cudaFree(g->d_err);
    delete g;
}

int bbx_create_grid(bbx_grid** out, int nx, int ny, int nz, double h, const uint8_t* mask_host,
                    void* cuda_stream) {
    if (!out) return BBX_ERR_ARG;
    *out = nullptr;
    if (nx <= 0 || ny <= 0 || nz <= 0 || !(h > 0.0) || !std::isfinite(h)) return BBX_ERR_ARG;
    const long long ncell = (long long)nx * ny * nz;
    if (ncell >= 0x7fffffffLL) return BBX_ERR_ARG;
    bbx_grid* g = new (std::nothrow) bbx_grid();
    if (!g) return BBX_ERR_NOMEM;
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->h = h;
    g->px = (nx + 31) / 32 * 32;
    g->plane = (long long)g->px * ny;
    g->vol = g->plane * nz;
    g->ncell = ncell;
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    g->zb = (nz == 1) ? 1 : 16;
    g->ty = 16;
    int rc = BBX_OK;
    do {
        if (cudaGetDevice(&g->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
            rc = BBX_ERR_CUDA;
            break;
        }
        if (dmalloc(&g->d_partials, sizeof(double) * kMaxPartials) != cudaSuccess ||
            dmalloc(&g->d_ticket, sizeof(unsigned int)) != cudaSuccess ||
            dmalloc(&g->d_total, sizeof(double)) != cudaSuccess ||
            dmalloc(&g->d_total2, sizeof(double)) != cudaSuccess || dmalloc(&g->d_err, sizeof(int)) != cudaSuccess ||
            dmalloc(&g->d_rest, sizeof(float) * 8) != cudaSuccess ||
            dmalloc(&g->d_mp, sizeof(float) * 8) != cudaSuccess) {
            rc = BBX_ERR_NOMEM;
            break;
        }
        if (cudaMemsetAsync(g->d_ticket, 0, sizeof(unsigned int), g->stream) != cudaSuccess ||
            cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream) != cudaSuccess) {
            rc = BBX_ERR_CUDA;
            break;
        }
        if (mask_host) {
            long long nt = 0;
            for (long long i = 0; i < ncell; ++i) nt += mask_host[i] != 0;
            g->n_tissue = nt;
            if (dmalloc(&g->d_mask, (size_t)g->vol) != cudaSuccess) {
                rc = BBX_ERR_NOMEM;
                break;
            }
            if (cudaMemsetAsync(g->d_mask, 0, (size_t)g->vol, g->stream) != cudaSuccess) {
                rc = BBX_ERR_CUDA;
                break;
            }
            // store 0/1 exactly
            std::vector<uint8_t> m01(ncell);
            for (long long i = 0; i < ncell; ++i) m01[i] = mask_host[i] ? 1 : 0;
            uint8_t* tmp = nullptr;
            if (dmalloc(&tmp, (size_t)g->vol) != cudaSuccess) {
                rc = BBX_ERR_NOMEM;
                break;
            }
            if (cudaMemsetAsync(tmp, 0, (size_t)g->vol, g->stream) != cudaSuccess ||
                (rc = copy_in(g, tmp, m01.data(), 1)) != BBX_OK) {
                cudaFree(tmp);
                if (rc == BBX_OK) rc = BBX_ERR_CUDA;
                break;
            }
            k_mask_interior<<<n_blocks_for(ncell, 256), 256, 0, g->stream>>>(tmp, g->d_mask, nx, ny, nz, g->px,
                                                                             g->plane);
            const cudaError_t e1 = cudaGetLastError();
            const cudaError_t e2 = cudaStreamSynchronize(g->stream);
            cudaFree(tmp);
            if (e1 != cudaSuccess || e2 != cudaSuccess) {
                rc = BBX_ERR_CUDA;
                break;
            }
        } else {
            g->n_tissue = ncell;
        }
        rc = build_bricks(g);
    } while (0);
    if (rc != BBX_OK) {
        bbx_destroy_grid(g);
        return rc;
    }
    *out = g;
    return BBX_OK;
}

int bbx_set_fibres(bbx_grid* g, const float* f, double D_par, double D_perp) {
    if (!g || !(D_par >= 0.0) || !(D_perp >= 0.0) || !std::isfinite(D_par) || !std::isfinite(D_perp))
        return BBX_ERR_ARG;
    if (!f) {
        cudaFree(g->d_fib);
        g->d_fib = nullptr;
        g->aniso = false;
        g->Dpar = g->Dperp = D_par;
    } else {
        float* tmp = nullptr;
        float* fib = nullptr;
        const int pxf = (g->nx + 8 + 31) / 32 * 32;
        const long long fplane = (long long)pxf * g->ny, fvol = fplane * g->nz;
        if (dmalloc(&tmp, sizeof(float) * 3 * g->ncell) != cudaSuccess) return BBX_ERR_NOMEM;
        if (dmalloc(&fib, sizeof(float) * 3 * fvol) != cudaSuccess) {
            cudaFree(tmp);
            return BBX_ERR_NOMEM;
        }
        int rc = BBX_OK, err = 0;
        cudaError_t e = cudaMemcpyAsync(tmp, f, sizeof(float) * 3 * g->ncell, cudaMemcpyHostToDevice, g->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream);
        if (e == cudaSuccess) {
            k_fibres<<<n_blocks_for(fvol, 256), 256, 0, g->stream>>>(tmp, g->nx, g->ny, g->nz, pxf, fplane, fvol,
                                                                      g->d_mask, g->px, g->plane, fib, g->d_err);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream);
        cudaFree(tmp);
        if (e != cudaSuccess) rc = BBX_ERR_CUDA;
        else if (err & kErrFibre) rc = BBX_ERR_FIBRE;
        if (rc != BBX_OK) {
            cudaFree(fib);
            return rc;
        }
        cudaFree(g->d_fib);
        g->d_fib = fib;
        g->pxf = pxf;
        g->fplane = fplane;
        g->fvol = fvol;
        g->aniso = true;
        g->Dpar = D_par;
        g->Dperp = D_perp;
    }
    if (g->model) return prepare(g);
    return BBX_OK;
}

int bbx_set_ionic_model(bbx_grid* g, int model, const double* params, int n_params) {
    if (!g) return BBX_ERR_ARG;
    const int S = model_nvars(model);
    if (S == 0 || n_params < 0 || (n_params > 0 && !params)) return BBX_ERR_ARG;
    double p[8] = {0};
    const int nd = model_defaults(model, p);
    for (int i = 0; i < n_params && i < nd; ++i) p[i] = params[i];
    for (int i = 0; i < nd; ++i)
        if (!std::isfinite(p[i])) return BBX_ERR_ARG;
    if (g->bound && S != g->S) {
        g->bound = false;  // the caller's buffers no longer fit: back to library buffers
        g->d_state[0] = g->d_state[1] = nullptr;
    }
    if (!g->bound && (S != g->S || !g->d_state[0])) {
        cudaFree(g->d_state[0]);
        cudaFree(g->d_state[1]);
        g->d_state[0] = g->d_state[1] = nullptr;
        if (dmalloc(&g->d_state[0], sizeof(float) * S * g->vol) != cudaSuccess ||
            dmalloc(&g->d_state[1], sizeof(float) * S * g->vol) != cudaSuccess)
            return BBX_ERR_NOMEM;
    }
    if (!g->d_act && dmalloc(&g->d_act, sizeof(int32_t) * g->vol) != cudaSuccess) return BBX_ERR_NOMEM;
    g->model = model;
    g->S = S;
    for (int i = 0; i < 8; ++i) g->par[i] = p[i];
    g->theta = model_threshold(model);
    float mp[8];
    model_kernel_params(model, p, mp);
    BBX_CUDA(cudaMemcpyAsync(g->d_mp, mp, sizeof(mp), cudaMemcpyHostToDevice, g->stream));
    k_rest<<<1, 1, 0, g->stream>>>(model, g->d_mp, p[1], p[2], g->d_rest);
    for (int b = 0; b < 2; ++b)
        k_fill_state<<<n_blocks_for((long long)S * g->vol, 256), 256, 0, g->stream>>>(g->d_state[b], S, g->vol,
                                                                                         g->d_rest);
    k_fill_int<<<n_blocks_for(g->vol, 256), 256, 0, g->stream>>>(g->d_act, g->vol, BBX_ACT_NONE);
    BBX_CUDA(cudaGetLastError());
    BBX_CUDA(cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    g->cur = 0;
    g->t = 0.0;
    g->n = 0;
    g->stepped = false;
    return prepare(g);
}

int bbx_bind_state(bbx_grid* g, void* a, void* b, size_t bytes) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (!a || !b || a == b || (reinterpret_cast<uintptr_t>(a) & 15) || (reinterpret_cast<uintptr_t>(b) & 15) ||
        bytes < sizeof(float) * g->S * (size_t)g->vol)
        return BBX_ERR_ARG;
    if (!g->bound) {
        cudaStreamSynchronize(g->stream);
        cudaFree(g->d_state[0]);
        cudaFree(g->d_state[1]);
    }
    g->d_state[0] = static_cast<float*>(a);
    g->d_state[1] = static_cast<float*>(b);
    g->bound = true;
    for (int k = 0; k < 2; ++k)
        k_fill_state<<<n_blocks_for((long long)g->S * g->vol, 256), 256, 0, g->stream>>>(g->d_state[k], g->S,
                                                                                            g->vol, g->d_rest);
    BBX_CUDA(cudaGetLastError());
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    g->cur = 0;
    return prepare(g);
}

int bbx_write_state(bbx_grid* g, int var, const float* host, size_t n) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (var < 0 || var >= g->S || !host || n != (size_t)g->ncell) return BBX_ERR_ARG;
    float* cur = g->d_state[g->cur] + (size_t)var * g->vol;
    float* oth = g->d_state[1 - g->cur] + (size_t)var * g->vol;
    int rc = copy_in(g, cur, host, sizeof(float));
    if (rc) return rc;
    // the other ping-pong buffer gets the same values (void nodes are never
    // rewritten by a step, so both buffers must agree there)
    BBX_CUDA(cudaMemcpyAsync(oth, cur, sizeof(float) * (size_t)g->vol, cudaMemcpyDeviceToDevice, g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    return BBX_OK;
}

int bbx_set_stimulus(bbx_grid* g, const uint8_t* region, double amp, double t_on, double t_off) {
    if (!g || !std::isfinite(amp) || std::isnan(t_on) || std::isnan(t_off)) return BBX_ERR_ARG;
    if (!region) {
        cudaFree(g->d_stim);
        g->d_stim = nullptr;
        g->stim_amp = 0.0;
        return BBX_OK;
    }
    if (!g->d_stim) {
        if (dmalloc(&g->d_stim, (size_t)g->vol) != cudaSuccess) return BBX_ERR_NOMEM;
        BBX_CUDA(cudaMemsetAsync(g->d_stim, 0, (size_t)g->vol, g->stream));
    }
    std::vector<uint8_t> r01(g->ncell);
    for (long long i = 0; i < g->ncell; ++i) r01[i] = region[i] ? 1 : 0;
    int rc = copy_in(g, g->d_stim, r01.data(), 1);
    if (rc) return rc;
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    g->stim_amp = amp;
    g->t_on = t_on;
    g->t_off = t_off;
    return BBX_OK;
}

int bbx_set_threshold(bbx_grid* g, double theta) {
    if (!g || !std::isfinite(theta)) return BBX_ERR_ARG;
    g->theta = theta;
    return BBX_OK;
}

int bbx_debug_poison_first_load(bbx_grid* g, int on) {
    if (!g) return BBX_ERR_ARG;
    g->poison = on ? 1 : 0;
    return BBX_OK;
}

int bbx_clear_device_error(bbx_grid* g) {
    if (!g) return BBX_ERR_ARG;
    BBX_CUDA(cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    return BBX_OK;
}

int bbx_step(bbx_grid* g, double dt, int n_steps) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (!(dt > 0.0) || !std::isfinite(dt) || n_steps < 0) return BBX_ERR_ARG;
    const double Dmax = g->aniso ? std::max(g->Dpar, g->Dperp) : g->Dpar;
    const double trD = g->aniso ? (g->Dpar + 2.0 * g->Dperp) : 3.0 * g->Dpar;
    const double dD = g->aniso ? std::fabs(g->Dpar - g->Dperp) : 0.0;
    (void)Dmax;
    // Gershgorin bound on the spectrum of the discrete operator:
    // |lambda| <= (4 tr D + 2 |Dpar - Dperp|) / h^2; forward Euler needs dt |lambda| <= 2.
    if (dt * (4.0 * trD + 2.0 * dD) > 2.0 * g->h * g->h) return BBX_ERR_UNSTABLE;
    if (n_steps == 0) return BBX_OK;
    if (!g->maps_ok) {
        int rc = prepare(g);
        if (rc) return rc;
    }
    if (g->n_bricks == 0 || g->n_planes == 0) {
        // no tissue: nothing moves, only time advances
        g->t += dt * n_steps;
        g->n += n_steps;
        double zero = 0.0;
        BBX_CUDA(cudaMemcpyAsync(g->d_total, &zero, sizeof(double), cudaMemcpyHostToDevice, g->stream));
        BBX_CUDA(cudaStreamSynchronize(g->stream));
        g->stepped = true;
        return BBX_OK;
    }
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = g->nx;
    a.ny = g->ny;
    a.nz = g->nz;
    a.px = g->px;
    a.plane = g->plane;
    a.vol = g->vol;
    a.pieces = g->d_pieces;
    a.cta_off = g->d_cta_off;
    a.act = g->d_act;
    a.theta = (float)g->theta;
    a.stim = g->d_stim;
    a.dt = (float)dt;
    {
        const double ih2 = 1.0 / (g->h * g->h);
        const double cd = (g->Dpar - g->Dperp) * ih2;
        a.c_perp = (float)(g->Dperp * ih2);
        a.c_d = (float)cd;
        a.c_dh = (float)(0.5 * cd);
        a.c_s = (float)(0.25 * cd);
        a.c_iso = (float)(g->Dpar * ih2);
    }
    model_kernel_params(g->model, g->par, a.mp);
    a.partials = g->d_partials;
    a.ticket = g->d_ticket;
    a.total_out = g->d_total;
    a.err = g->d_err;
    a.poison_first_load = g->poison;
    a.wait_limit = g->poison ? kPoisonWaitLimit : kWaitLimitCycles;
    for (int s = 0; s < n_steps; ++s) {
        const int src = g->cur, dst = 1 - g->cur;
        a.dst = g->d_state[dst];
        a.step_next = (int)(g->n + 1);
        const bool on = g->d_stim && g->stim_amp != 0.0 && g->t >= g->t_on && g->t < g->t_off;
        a.stim_amp = on ? (float)g->stim_amp : 0.0f;
        void* args[] = {(void*)&g->tm_u[src], (void*)&g->tm_s[src], (void*)&g->tm_f, (void*)&g->tm_m, (void*)&a};
        cudaError_t e = cudaLaunchKernel(g->kern.fn, dim3(g->grid_ctas), dim3(g->kern.threads), args,
                                         (size_t)g->kern.smem, g->stream);
        if (e != cudaSuccess) return BBX_ERR_CUDA;
        g->cur = dst;
        g->t += dt;
        g->n += 1;
        g->stepped = true;
    }
    return BBX_OK;
}

int bbx_read_state(bbx_grid* g, int var, float* host, size_t n) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (var < 0 || var >= g->S || !host || n != (size_t)g->ncell) return BBX_ERR_ARG;
    int rc = copy_out(g, host, g->d_state[g->cur] + (size_t)var * g->vol, sizeof(float));
    if (rc) return rc;
    return check_sticky(g);
}

int bbx_read_activation(bbx_grid* g, int32_t* host, size_t n) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (!host || n != (size_t)g->ncell) return BBX_ERR_ARG;
    int rc = copy_out(g, host, g->d_act, sizeof(int32_t));
    if (rc) return rc;
    return check_sticky(g);
}

int bbx_write_activation(bbx_grid* g, const int32_t* host, size_t n) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (!host || n != (size_t)g->ncell) return BBX_ERR_ARG;
    int rc = copy_in(g, g->d_act, host, sizeof(int32_t));
    if (rc) return rc;
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    return BBX_OK;
}

int bbx_total(bbx_grid* g, int var, double* out) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (var < 0 || var >= g->S || !out) return BBX_ERR_ARG;
    int blocks = g->num_sms * 4;
    if (blocks > kMaxPartials) blocks = kMaxPartials;
    k_total<<<blocks, 256, 0, g->stream>>>(g->d_state[g->cur] + (size_t)var * g->vol, g->d_mask, g->nx, g->ny,
                                           g->nz, g->px, g->plane, g->d_partials, g->d_ticket, g->d_total2, g->d_err);
    BBX_CUDA(cudaGetLastError());
    BBX_CUDA(cudaMemcpyAsync(out, g->d_total2, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    return check_sticky(g);
}

int bbx_step_total(bbx_grid* g, double* out) {
    if (!g || !out) return BBX_ERR_ARG;
    if (!g->stepped) return BBX_ERR_STATE;
    BBX_CUDA(cudaMemcpyAsync(out, g->d_total, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    return check_sticky(g);
}

int bbx_get_time(bbx_grid* g, double* t, long long* step) {
    if (!g) return BBX_ERR_ARG;
    if (t) *t = g->t;
    if (step) *step = g->n;
    return BBX_OK;
}

int bbx_set_time(bbx_grid* g, double t, long long step) {
    if (!g || !std::isfinite(t) || step < 0 || step >= 0x7fffffffLL) return BBX_ERR_ARG;
    g->t = t;
    g->n = step;
    return BBX_OK;
}

int bbx_get_info(bbx_grid* g, bbx_info* o) {
    if (!g || !o) return BBX_ERR_ARG;
    o->nx = g->nx;
    o->ny = g->ny;
    o->nz = g->nz;
    o->px = g->px;
    o->nvars = g->S;
    o->model = g->model;
    o->masked = g->d_mask != nullptr;
    o->anisotropic = g->aniso;
    o->tile_x = kTileX;
    o->tile_y = g->ty;
    o->tile_z = g->zb;
    o->n_bricks = g->n_bricks;
    o->n_tissue = g->n_tissue;
    o->step = g->n;
    o->t = g->t;
    return BBX_OK;
}

int bbx_read_active_bricks(bbx_grid* g, int32_t* out, size_t cap, long long* count) {
    if (!g || !count) return BBX_ERR_ARG;
    *count = g->n_bricks;
    if ((size_t)g->n_bricks > cap || (!out && g->n_bricks > 0)) return BBX_ERR_ARG;
    if (g->d_bricks) {
        BBX_CUDA(cudaMemcpyAsync(out, g->d_bricks, sizeof(int32_t) * g->n_bricks, cudaMemcpyDeviceToHost, g->stream));
        BBX_CUDA(cudaStreamSynchronize(g->stream));
    } else {
        for (long long i = 0; i < g->n_bricks; ++i) out[i] = (int32_t)i;
    }
    return BBX_OK;
}

int bbx_set_tiling(bbx_grid* g, int tile_y, int tile_z) {
    if (!g || (tile_y != 8 && tile_y != 16 && tile_y != 32) || tile_z < 1) return BBX_ERR_ARG;
    const int old_ty = g->ty, old_zb = g->zb;
    g->ty = tile_y;
    g->zb = tile_z > g->nz ? g->nz : tile_z;
    int rc = build_bricks(g);
    if (rc == BBX_OK && g->model) rc = prepare(g);
    if (rc == BBX_ERR_UNSUPPORTED) {
        // keep the previous, working tile shape
        g->ty = old_ty;
        g->zb = old_zb;
        if (build_bricks(g) == BBX_OK && g->model) prepare(g);
    }
    return rc;
}

int bbx_state_device_ptr(bbx_grid* g, int var, void** p) {
    if (!g || !p) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (var < 0 || var >= g->S) return BBX_ERR_ARG;
    *p = g->d_state[g->cur] + (size_t)var * g->vol;
    return BBX_OK;
}

int bbx_autotune(bbx_grid* g, double dt, double* best_ms) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    // save the state so the trial steps leave no trace
    const size_t sbytes = sizeof(float) * g->S * (size_t)g->vol;
    float* save = nullptr;
    int32_t* save_act = nullptr;
    if (dmalloc(&save, sbytes) != cudaSuccess) return BBX_ERR_NOMEM;
    if (dmalloc(&save_act, sizeof(int32_t) * g->vol) != cudaSuccess) {
        cudaFree(save);
        return BBX_ERR_NOMEM;
    }
    BBX_CUDA(cudaMemcpyAsync(save, g->d_state[g->cur], sbytes, cudaMemcpyDeviceToDevice, g->stream));
    BBX_CUDA(cudaMemcpyAsync(save_act, g->d_act, sizeof(int32_t) * g->vol, cudaMemcpyDeviceToDevice, g->stream));
    const int cur0 = g->cur;
    const double t0 = g->t;
    const long long n0 = g->n;
    const bool stepped0 = g->stepped;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int tys[3] = {8, 16, 32};
    std::vector<int> zbs;
    if (g->nz == 1 || !g->d_mask) {
        zbs.push_back(g->zb);  // unmasked columns are marched whole; only the tile rows matter
    } else {
        for (int z : {4, 8, 16, 32, 64})
            if (z <= g->nz) zbs.push_back(z);
        if (g->nz > 64) zbs.push_back(g->nz);
    }
    double best = 1e30;
    int bty = g->ty, bzb = g->zb;
    int rc = BBX_OK;
    for (int ty : tys) {
        for (int zb : zbs) {
            if ((rc = bbx_set_tiling(g, ty, zb)) != BBX_OK) {
                if (rc == BBX_ERR_UNSUPPORTED) { rc = BBX_OK; continue; }
                break;
            }
            if ((rc = bbx_step(g, dt, 2)) != BBX_OK) break;
            cudaEventRecord(e0, g->stream);
            if ((rc = bbx_step(g, dt, 6)) != BBX_OK) break;
            cudaEventRecord(e1, g->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / 6.0 < best) {
                best = ms / 6.0;
                bty = ty;
                bzb = zb;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc2 = bbx_set_tiling(g, bty, bzb);
    g->cur = cur0;
    cudaMemcpyAsync(g->d_state[g->cur], save, sbytes, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(g->d_state[1 - g->cur], save, sbytes, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(g->d_act, save_act, sizeof(int32_t) * g->vol, cudaMemcpyDeviceToDevice, g->stream);
    cudaStreamSynchronize(g->stream);
    cudaFree(save);
    cudaFree(save_act);
    g->t = t0;
    g->n = n0;
    g->stepped = stepped0;
    if (best_ms) *best_ms = best;
    if (rc) return rc;
    if (rc2) return rc2;
    return check_sticky(g);
}

}  // extern "C"
