// Host runtime of the C ABI in include/bbx.h, plus the set-up kernels
// (fibre normalisation, tissue bricks, rest state) and the standalone
// double-precision tissue reduction.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <map>
#include <vector>

#include "bbx_device.cuh"
#include "bbx_mlp.cuh"

namespace bbx {
StepKernel step_kernel_fhn(bool masked, int aniso, int ty, bool planar, bool general);
StepKernel step_kernel_barkley(bool masked, int aniso, int ty, bool planar, bool general);
StepKernel step_kernel_br(bool masked, int aniso, int ty, bool planar, bool general);
StepKernel step_kernel_zfk(bool masked, int aniso, int ty, bool planar, bool general);
StepKernel step_kernel_diffusion(bool masked, int aniso, int ty, bool planar, bool general);
StepKernel step_kernel_br_mrl(bool masked, int aniso, int ty, bool planar, bool general);
StepKernel step_kernel_br_fca(bool masked, int aniso, int ty, bool planar, bool general);
cudaError_t mrl_build_table(float4* tab, double dt, cudaStream_t s);
cudaError_t br_build_rl_table(float4* tab, double dt, double tau_c, cudaStream_t s);
StepKernel step_kernel_br_surrogate(bool masked, bool aniso, int ty);
StepKernel step_kernel_br16(bool masked, bool aniso, int ty, bool planar, bool general, int gates);
cudaError_t launch_ppm(const float* s0, const float* s1, const int* cur, const uint8_t* mask, long long vol, int nx,
                       int ny, int nz, int px, long long plane, const int layer[3], const float lo[3],
                       const float hi[3], uint8_t* out, int num_sms, cudaStream_t s);
cudaError_t resident_sheet_steps(int model, const TissueArgs* d_t, int nx, int ny, int n_steps, int* d_err,
                                 cudaStream_t s, bool check_only, bool* ok);
cudaError_t launch_singz(const float* s0, const float* s1, const int* cur, long long off_a, long long off_b,
                         float iso_a, float iso_b, const uint8_t* mask, int nx, int ny, int nz, int px,
                         long long plane, float* xyz, int max_points, int* d_count, int num_sms, cudaStream_t s);
}  // namespace bbx

using namespace bbx;

namespace {

constexpr long long kWaitLimitCycles = 4000000000LL;  // about 2 s of SM clock
constexpr long long kPoisonWaitLimit = 2000000LL;     // about 1 ms
constexpr int kMaxPartials = 152 * 32;
constexpr int kErrFibre = 4;
constexpr int kChunkX = 16;  // x granularity of a masked grid's piece origins (the mask copy's 16-byte rule)

int model_nvars(int model) {
    switch (model) {
        case BBX_FHN: return 2;
        case BBX_BARKLEY: return 2;
        case BBX_BR: return 8;
        case BBX_ZFK: return 1;
        case BBX_DIFFUSION: return 1;
        case BBX_BR_MRL: return 11;
        case BBX_BR_FCA: return 11;
    }
    return 0;
}

double model_threshold(int model) {
    switch (model) {
        case BBX_FHN: return 0.0;
        case BBX_BR:
        case BBX_BR_MRL:
        case BBX_BR_FCA: return -40.0;
        default: return 0.5;
    }
}

// defaults of each model's parameter list (bbx.h)
int model_defaults(int model, double* p) {
    switch (model) {
        case BBX_FHN: p[0] = 0.3; p[1] = 0.71; p[2] = 0.5; return 3;
        case BBX_BARKLEY: p[0] = 0.75; p[1] = 0.02; p[2] = 0.02; return 3;
        case BBX_BR:
        case BBX_BR_MRL: p[0] = 4.0; p[1] = 0.003; p[2] = 50.0; p[3] = 0.09; return 4;
        case BBX_BR_FCA:
            p[0] = 4.0; p[1] = 0.003; p[2] = 50.0; p[3] = 0.09; p[4] = 5e-6; p[5] = 2.0; p[6] = 0.05; p[7] = 0.0;
            return 8;  // ..., Kc (mol/L), tau_c (ms), eps, onfly
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
        case BBX_BR:
        case BBX_BR_MRL: for (int i = 0; i < 4; ++i) mp[i] = float(p[i]); break;
        case BBX_BR_FCA:
            for (int i = 0; i < 5; ++i) mp[i] = float(p[i]);
            mp[5] = float(p[6]);
            mp[6] = float(1.0 / p[5]);
            mp[7] = p[7] != 0.0 ? 1.0f : 0.0f;
            break;
        case BBX_ZFK: mp[0] = float(p[0]); break;
        default: break;
    }
}

// planar: a grid with nz = 1 (sheet kernels, tiles marched along y).  The
// surrogate kernels exist for 3D grids only.  general: the grid uses the Lie
// scheme or the RK4 solver (kernels for 7- and 14-row tiles).
// aniso: AN_ISO, AN_SUMS or AN_NO_SUMS (the last only for the plain kernels of
// unmasked grids; the 16-bit-gate and surrogate variants read the sums)
StepKernel lookup_kernel(int model, bool masked, int aniso, int ty, bool surrogate, bool planar, bool general,
                         int gates = GATES_F32) {
    if (gates != GATES_F32)  // 16-bit gates: Beeler-Reuter without surrogate
        return model == BBX_BR && !surrogate && aniso != AN_NO_SUMS
                   ? step_kernel_br16(masked, aniso != AN_ISO, ty, planar, general, gates)
                   : StepKernel{nullptr, 0, 0, 0};
    if (surrogate)
        return model == BBX_BR && !planar && aniso != AN_NO_SUMS
                   ? step_kernel_br_surrogate(masked, aniso != AN_ISO, ty)
                   : StepKernel{nullptr, 0, 0, 0};
    switch (model) {
        case BBX_FHN: return step_kernel_fhn(masked, aniso, ty, planar, general);
        case BBX_BARKLEY: return step_kernel_barkley(masked, aniso, ty, planar, general);
        case BBX_BR: return step_kernel_br(masked, aniso, ty, planar, general);
        case BBX_ZFK: return step_kernel_zfk(masked, aniso, ty, planar, general);
        case BBX_DIFFUSION: return step_kernel_diffusion(masked, aniso, ty, planar, general);
        case BBX_BR_MRL: return step_kernel_br_mrl(masked, aniso, ty, planar, general);
        case BBX_BR_FCA: return step_kernel_br_fca(masked, aniso, ty, planar, general);
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

// The W-tilde ingredient of the weights (section "Monodomain diffusion and
// boundary conditions"): per tissue node p, S_k = sum_j (f_j f_k at p + q_j
// minus at p - q_j), f the unit fibre, with a void or out-of-array neighbour's
// fibre replaced by f at p (D^p in place of its tensor; the D_perp parts of
// D cancel in the difference).  The fibre field is fixed, so the three sums
// are computed once, in double precision, and read by every step.  Layout
// [3][nz][ny][px]; 0 at void nodes.  *nonzero is set to 1 if any stored sum
// differs from 0 (the step kernel skips loading sums that all vanish).
__global__ void k_divergence(const float* __restrict__ fib, int nx, int ny, int nz, int pxf, long long fplane,
                             long long fvol, const uint8_t* __restrict__ mask, int px, long long plane,
                             long long vol, float* __restrict__ div, int* __restrict__ nonzero) {
    const long long n = (long long)nx * ny * nz;
    bool any = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = int(i % nx);
        const long long r = i / nx;
        const int y = int(r % ny);
        const int z = int(r / ny);
        const long long o = z * plane + (long long)y * px + x;
        auto tissue = [&](int xx, int yy, int zz) {
            if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) return false;
            return mask ? (mask[zz * plane + (long long)yy * px + xx] & 1) != 0 : true;
        };
        auto fibre = [&](int xx, int yy, int zz, double* f) {
            const long long q = zz * fplane + (long long)yy * pxf + (xx + 4);
            f[0] = fib[q];
            f[1] = fib[fvol + q];
            f[2] = fib[2 * fvol + q];
        };
        double acc[3] = {0.0, 0.0, 0.0};
        if (tissue(x, y, z)) {
            double fp[3];
            fibre(x, y, z, fp);
            for (int j = 0; j < 3; ++j) {
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    int c[3] = {x, y, z};
                    c[j] += sgn;
                    double fn[3] = {fp[0], fp[1], fp[2]};
                    if (tissue(c[0], c[1], c[2])) fibre(c[0], c[1], c[2], fn);
                    for (int k = 0; k < 3; ++k) acc[k] += sgn * fn[j] * fn[k];
                }
            }
        }
        const float s0 = (float)acc[0], s1 = (float)acc[1], s2 = (float)acc[2];
        div[o] = s0;
        div[vol + o] = s1;
        div[2 * vol + o] = s2;
        any = any || s0 != 0.0f || s1 != 0.0f || s2 != 0.0f;
    }
    if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(nonzero, 1);
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
                        if (nz == 1 && dz != 0) continue;  // a sheet has no z neighbours
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

// One block per 16-node-wide chunk of a brick row band: does the chunk
// (16 x ty x zb nodes) hold any tissue node?  Block id = cx + ncx (by + nby bz).
__global__ void k_chunk_flags(const uint8_t* __restrict__ mask, int nx, int ny, int nz, int px, long long plane,
                              int ty, int zb, int ncx, int nby, uint8_t* flags) {
    const long long id = blockIdx.x;
    const int cx = (int)(id % ncx), by = (int)((id / ncx) % nby), bz = (int)(id / ((long long)ncx * nby));
    const int x0 = cx * kChunkX, y0 = by * ty, z0 = bz * zb;
    const int cells = kChunkX * ty * zb;
    int any = 0;
    for (int c = threadIdx.x; c < cells && !any; c += blockDim.x) {
        const int x = x0 + c % kChunkX;
        const int y = y0 + (c / kChunkX) % ty;
        const int z = z0 + c / (kChunkX * ty);
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
    for (int i = 0; i < 16; ++i) out[i] = 0.0f;
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
    } else if (model == BBX_BR_MRL) {
        // the Beeler-Reuter rest state, with the chain at the binomial
        // distribution of the rest value of m (independent subunits)
        float y[8] = {-84.0f, 1e-7f, 0.0f, 0.0f, 1.0f, 1.0f, 0.0f, 1.0f};
        float p[8];
        for (int i = 0; i < 8; ++i) p[i] = mp[i];
        for (int n = 0; n < 200000; ++n) Model<BBX_BR>::update(p, y, 0.0f, 0.0f, 0.05f);
        const double m = y[3];
        out[0] = y[0]; out[1] = y[1]; out[2] = y[2];
        out[3] = y[4]; out[4] = y[5]; out[5] = y[6]; out[6] = y[7];
        out[7] = float((1 - m) * (1 - m) * (1 - m));
        out[8] = float(3 * m * (1 - m) * (1 - m));
        out[9] = float(3 * m * m * (1 - m));
        out[10] = float(m * m * m);
    } else if (model == BBX_BR_FCA) {
        // from the Beeler-Reuter rest state with the channel at the product
        // of the gates' steady states, the cell integrated for another 10 s
        // (the calcium gate moves the rest state)
        float y[11] = {-84.0f, 1e-7f, 0.0f, 0.0f, 1.0f, 1.0f, 0.0f, 1.0f, 0.0f, 0.0f, 0.0f};
        float p[8];
        for (int i = 0; i < 8; ++i) p[i] = mp[i];
        for (int n = 0; n < 200000; ++n) Model<BBX_BR>::update(p, y, 0.0f, 0.0f, 0.05f);
        const float f = y[7], c = p[4] / (p[4] + y[1]);
        y[7] = (1.0f - f) * (1.0f - c);
        y[8] = f * (1.0f - c);
        y[9] = (1.0f - f) * c;
        y[10] = f * c;
        for (int n = 0; n < 200000; ++n) Model<BBX_BR_FCA>::update(p, y, 0.0f, 0.0f, 0.05f);
        for (int i = 0; i < 11; ++i) out[i] = y[i];
    }
}

// Device-to-device copy of n4 float4 by the SMs (the asynchronous exchange's
// stage copies, which would otherwise take a copy engine from the host copies
// they are meant to overlap); up to two destinations.
__global__ void k_copy4(float4* __restrict__ d0, float4* __restrict__ d1, const float4* __restrict__ src,
                        long long n4) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 v = __ldcs(src + i);
        d0[i] = v;
        if (d1) d1[i] = v;
    }
}

__global__ void k_fill_state(float* __restrict__ st, int S, long long vol, const float* __restrict__ rest) {
    const long long n = (long long)S * vol;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        st[i] = rest[i / vol];
}

// 16-bit gate storage (Beeler-Reuter): V and Ca as float planes, then the
// six gates as uint16 planes (binary16 or fixed point u / 65535).
__device__ __forceinline__ uint16_t enc16(float y, int mode) {
    if (mode == GATES_F16) return __half_as_ushort(__float2half_rn(y));
    return (uint16_t)__float2uint_rn(__saturatef(y) * 65535.0f);
}
__device__ __forceinline__ float dec16(uint16_t u, int mode) {
    if (mode == GATES_F16) return __half2float(__ushort_as_half(u));
    return (float)u * (1.0f / 65535.0f);
}

// Every node of a buffer to the rest state (in the buffer's layout).
__global__ void k_fill_state16(float* __restrict__ st, long long vol, const float* __restrict__ rest, int mode) {
    uint16_t* g16 = reinterpret_cast<uint16_t*>(st + 2 * vol);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < vol;
         i += (long long)gridDim.x * blockDim.x) {
        st[i] = rest[0];
        st[vol + i] = rest[1];
        for (int g = 0; g < 6; ++g) g16[g * vol + i] = enc16(rest[2 + g], mode);
    }
}

// One 16-bit plane of variable-sized data to and from floats.
__global__ void k_pack16(const float* __restrict__ src, uint16_t* __restrict__ dst, long long n, int mode) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = enc16(src[i], mode);
}
__global__ void k_unpack16(const uint16_t* __restrict__ src, float* __restrict__ dst, long long n, int mode) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = dec16(src[i], mode);
}

__global__ void k_set_parity(TissueDyn* dyn, int cur) {
    if (threadIdx.x == 0 && blockIdx.x == 0) dyn->cur = cur;
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

// The total of a grid's last single-grid step, summed from the step's
// per-piece partials in slot order (unused slots hold 0) when it is asked
// for; nothing happens if no total is pending.  One CTA.
__global__ void k_finish_total(const double* __restrict__ partials, int n_slots, TissueDyn* dyn, int* err) {
    __shared__ double scratch[32];
    if (!dyn->total_pending) return;  // uniform: every thread reads the same flag
    double s = 0.0;
    for (int k = threadIdx.x; k < n_slots; k += blockDim.x) s += partials[k];
    const double total = block_sum_double(s, scratch);
    if (threadIdx.x == 0) {
        if (!isfinite(total)) atomicOr(err, ERRBIT_NAN);
        dyn->total = total;
        dyn->total_pending = 0;
    }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Training pairs for the reaction surrogate: n tissue nodes drawn by a
// counter-based hash, their current Beeler-Reuter state s and the exact
// reaction increment of one step (no diffusion, no stimulus) s' - s.
__global__ void k_sample_pairs_br(const TissueArgs* __restrict__ T, const uint8_t* __restrict__ mask, long long n,
                                  unsigned long long seed, float* __restrict__ X, float* __restrict__ Y) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long cells = (long long)T->nx * T->ny * T->nz;
    long long node = 0, gi = 0;
    for (int attempt = 0; attempt < 256; ++attempt) {
        node = (long long)(mix64(seed ^ mix64((unsigned long long)i * 256ull + attempt)) % (unsigned long long)cells);
        const int x = int(node % T->nx);
        const long long r = node / T->nx;
        const int y = int(r % T->ny);
        const int z = int(r / T->ny);
        gi = z * T->plane + (long long)y * T->px + x;
        if (!mask || mask[gi]) break;
    }
    const float* st = T->state[T->dyn->cur];
    float s[8], d[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) s[v] = st[(long long)v * T->vol + gi];
    float mp[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) mp[k] = T->mp[k];
    Model<BBX_BR>::increment(mp, s, 0.0f, 0.0f, T->dt, d);
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        X[i * 8 + v] = s[v];
        Y[i * 8 + v] = d[v];
    }
}

// The step kernel's copy of a trained network: BF16 weights in row-major
// 32-bit pairs (W1 padded from 8 to 16 inputs), FP32 biases, normalisation.
__global__ void k_build_surrogate(const float* __restrict__ P, const float* __restrict__ norm, float v_up,
                                  SurrogateData* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    auto pair = [](float lo, float hi) {
        __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&v);
    };
    // MMA-fragment order (see SurrogateData): word (lane t, k-step kk, half h)
    // of a row holds input columns 16 kk + 2 t + 8 h and the next one
    if (i < 64 * 8) {  // W1 [64][16], inputs 8..15 are zero padding
        const int n = i / 8, t = (i % 8) / 2, h = i % 2, c = 2 * t + 8 * h;
        out->W1[i] = pair(c < 8 ? P[kOffW1 + n * 8 + c] : 0.0f, c + 1 < 8 ? P[kOffW1 + n * 8 + c + 1] : 0.0f);
    }
    if (i < 64 * 32) {
        const int n = i / 32, t = (i % 32) / 8, kk = (i % 8) / 2, h = i % 2, c = 16 * kk + 2 * t + 8 * h;
        out->W2[i] = pair(P[kOffW2 + n * 64 + c], P[kOffW2 + n * 64 + c + 1]);
    }
    if (i < 8 * 32) {
        const int n = i / 32, t = (i % 32) / 8, kk = (i % 8) / 2, h = i % 2, c = 16 * kk + 2 * t + 8 * h;
        out->W3[i] = pair(P[kOffW3 + n * 64 + c], P[kOffW3 + n * 64 + c + 1]);
    }
    if (i < 64) {
        out->b1[i] = P[kOffB1 + i];
        out->b2[i] = P[kOffB2 + i];
    }
    if (i < 8) out->b3[i] = P[kOffB3 + i];
    if (i < kNormSize) out->norm[i] = norm[i];
    if (i < 8) out->inv_sd_in[i] = 1.0f / norm[8 + i];
    if (i == 0) out->v_up = v_up;
}

template <typename T>
cudaError_t dmalloc(T** p, size_t bytes) {
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

}  // namespace

// ---------------------------------------------------------------------------
// launch plans: a balanced schedule of pieces over a list of grids
// ---------------------------------------------------------------------------

namespace {

struct Seg {
    int tissue, x0, y0, z0, z1;
};

struct LaunchPlan {
    StepKernel k = {nullptr, 0, 0, 0};
    int ctas = 0;
    int n_tissues = 0;
    long long n_planes = 0;
    int4* d_pieces = nullptr;
    int* d_piece_tissue = nullptr;
    int* d_cta_count = nullptr;
    int* d_tissue_off = nullptr;
    int* d_tissue_pieces = nullptr;
    double* d_partials = nullptr;
    unsigned int* d_ticket = nullptr;
    unsigned int* d_tissue_done = nullptr;  // per grid, zero between launches
    int* d_empty = nullptr;                 // grids without pieces
    int n_empty = 0;
    size_t cap_pieces = 0, cap_cta = 0, cap_tis = 0, cap_tlist = 0, cap_done = 0, cap_empty = 0;
    int cta_stride = 1, n_slots = 0;

    void release() {
        cudaFree(d_pieces);
        cudaFree(d_piece_tissue);
        cudaFree(d_cta_count);
        cudaFree(d_tissue_off);
        cudaFree(d_tissue_pieces);
        cudaFree(d_partials);
        cudaFree(d_ticket);
        cudaFree(d_tissue_done);
        cudaFree(d_empty);
        *this = LaunchPlan();
    }
};

template <typename T>
int upload(T** d, size_t* cap, const std::vector<T>& h) {
    const size_t n = h.size() ? h.size() : 1;
    if (n > *cap) {
        cudaFree(*d);
        *d = nullptr;
        if (dmalloc(d, sizeof(T) * n) != cudaSuccess) {
            cudaGetLastError();
            *cap = 0;
            return BBX_ERR_NOMEM;
        }
        *cap = n;
    }
    if (!h.empty() && cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    return BBX_OK;
}

// Each CTA receives an equal share of the column-planes of all segments (in
// segment order) as contiguous pieces, so that no CTA idles while others
// finish: CTA c takes column-planes [c T / ctas, (c+1) T / ctas) of the T in
// all segments.  Returns the CTA count used (at most T); per[c] and per_t[c]
// get CTA c's pieces and their grids.  Host-only.
int plan_shares(const std::vector<Seg>& segs, int ctas, std::vector<std::vector<int4>>* per_out,
                std::vector<std::vector<int>>* per_t_out, int* stride_out) {
    long long T = 0;
    for (const Seg& sg : segs) T += sg.z1 - sg.z0;
    if (ctas > T) ctas = (int)std::max<long long>(T, 1);
    std::vector<std::vector<int4>>& per = *per_out;
    std::vector<std::vector<int>>& per_t = *per_t_out;
    per.assign((size_t)ctas, {});
    per_t.assign((size_t)ctas, {});
    size_t si = 0;
    long long consumed = 0;
    int stride = 1;
    for (int c = 0; c < ctas; ++c) {
        long long need = (long long)(c + 1) * T / ctas - (long long)c * T / ctas;
        while (need > 0 && si < segs.size()) {
            const Seg& sg = segs[si];
            const long long avail = (sg.z1 - sg.z0) - consumed;
            const long long take = std::min(avail, need);
            const int z0 = sg.z0 + (int)consumed;
            per[(size_t)c].push_back(make_int4(sg.x0, sg.y0, z0, z0 + (int)take));
            per_t[(size_t)c].push_back(sg.tissue);
            need -= take;
            consumed += take;
            if (consumed == sg.z1 - sg.z0) {
                ++si;
                consumed = 0;
            }
        }
        stride = std::max(stride, (int)per[(size_t)c].size());
    }
    *stride_out = stride;
    return ctas;
}

// The launch plan of a list of segments (plan_shares), uploaded; per grid,
// the pieces are listed for the fixed-order totals.
int build_plan(LaunchPlan* lp, const std::vector<Seg>& segs, int n_tissues, int ctas) {
    long long T = 0;
    for (const Seg& sg : segs) T += sg.z1 - sg.z0;
    lp->n_planes = T;
    lp->n_tissues = n_tissues;
    std::vector<std::vector<int4>> per;
    std::vector<std::vector<int>> per_t;
    int stride = 1;
    ctas = plan_shares(segs, ctas, &per, &per_t, &stride);
    // slot c*stride + i holds piece i of CTA c; unused slots stay zero
    const size_t nslot = (size_t)ctas * (size_t)stride;
    std::vector<int4> pieces(nslot, make_int4(0, 0, 0, 0));
    std::vector<int> ptis(nslot, 0), cnt((size_t)ctas, 0);
    std::vector<int> toff((size_t)n_tissues + 1, 0);
    for (int c = 0; c < ctas; ++c) {
        cnt[(size_t)c] = (int)per[(size_t)c].size();
        for (size_t i = 0; i < per[(size_t)c].size(); ++i) {
            pieces[(size_t)c * stride + i] = per[(size_t)c][i];
            ptis[(size_t)c * stride + i] = per_t[(size_t)c][i];
            toff[(size_t)per_t[(size_t)c][i] + 1]++;
        }
    }
    for (int t = 0; t < n_tissues; ++t) toff[(size_t)t + 1] += toff[t];
    std::vector<int> tlist((size_t)toff[(size_t)n_tissues]);
    {
        std::vector<int> fill(toff.begin(), toff.end() - 1);
        for (int c = 0; c < ctas; ++c)
            for (int i = 0; i < cnt[(size_t)c]; ++i) {
                const size_t k = (size_t)c * stride + i;
                tlist[(size_t)fill[(size_t)ptis[k]]++] = (int)k;
            }
    }
    int rc;
    size_t cap_pt = lp->cap_pieces, cap_part = lp->cap_pieces;
    if ((rc = upload(&lp->d_pieces, &lp->cap_pieces, pieces))) return rc;
    if ((rc = upload(&lp->d_piece_tissue, &cap_pt, ptis))) return rc;
    if ((rc = upload(&lp->d_tissue_pieces, &lp->cap_tlist, tlist))) return rc;
    if ((rc = upload(&lp->d_cta_count, &lp->cap_cta, cnt))) return rc;
    if ((rc = upload(&lp->d_tissue_off, &lp->cap_tis, toff))) return rc;
    std::vector<double> zeros(nslot, 0.0);
    if ((rc = upload(&lp->d_partials, &cap_part, zeros))) return rc;
    std::vector<unsigned int> done((size_t)n_tissues, 0u);
    if ((rc = upload(&lp->d_tissue_done, &lp->cap_done, done))) return rc;
    std::vector<int> empty;
    for (int t = 0; t < n_tissues; ++t)
        if (toff[(size_t)t + 1] == toff[(size_t)t]) empty.push_back(t);
    if ((rc = upload(&lp->d_empty, &lp->cap_empty, empty))) return rc;
    lp->n_empty = (int)empty.size();
    lp->cta_stride = stride;
    lp->n_slots = (int)nslot;
    if (!lp->d_ticket) {
        if (dmalloc(&lp->d_ticket, sizeof(unsigned int)) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_NOMEM;
        }
        if (cudaMemset(lp->d_ticket, 0, sizeof(unsigned int)) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_CUDA;
        }
    }
    lp->ctas = ctas;
    return BBX_OK;
}

// h_single: the host copy of the TissueArgs of a single-grid launch (carried in
// the kernel parameters), or nullptr.
LaunchArgs launch_args(const LaunchPlan& lp, const TissueArgs* d_tissues, int* d_err, int poison,
                       const TissueArgs* h_single = nullptr) {
    LaunchArgs L;
    memset((void*)&L, 0, sizeof(L));
    if (h_single && lp.n_tissues == 1) {
        L.t0 = *h_single;
        L.single = 1;
    }
    L.tissues = d_tissues;
    L.pieces = lp.d_pieces;
    L.piece_tissue = lp.d_piece_tissue;
    L.cta_count = lp.d_cta_count;
    L.cta_stride = lp.cta_stride;
    L.n_slots = lp.n_slots;
    L.tissue_off = lp.d_tissue_off;
    L.tissue_pieces = lp.d_tissue_pieces;
    L.n_tissues = lp.n_tissues;
    L.partials = lp.d_partials;
    L.ticket = lp.d_ticket;
    L.tissue_done = lp.d_tissue_done;
    L.empty_tissues = lp.d_empty;
    L.n_empty = lp.n_empty;
    L.err = d_err;
    L.poison_first_load = poison;
    L.cur_hint = -1;
    L.wait_limit = poison ? kPoisonWaitLimit : kWaitLimitCycles;
    return L;
}

// A step launch, allowed to start while the previous kernel on the stream
// finishes (programmatic stream serialization: the step kernel waits for it
// with griddepcontrol.wait before it reads or writes anything that kernel may
// touch; each grid is at most one wave of resident CTAs, so the early CTAs
// never hold back the previous grid's).
cudaError_t launch(const LaunchPlan& lp, const LaunchArgs& L, cudaStream_t s) {
    if (lp.n_planes == 0) return cudaSuccess;
    void* args[] = {(void*)&L};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(lp.ctas);
    cfg.blockDim = dim3(lp.k.threads);
    cfg.dynamicSmemBytes = (size_t)lp.k.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, lp.k.fn, args);
}

// Select the kernel for a configuration, check it fits, and return the CTA
// budget (resident CTAs on the whole GPU).
int select_kernel(int model, bool masked, int aniso, int ty, int device, int num_sms, StepKernel* out,
                  int* ctas, bool surrogate, bool planar, bool general, int gates = GATES_F32) {
    StepKernel k = lookup_kernel(model, masked, aniso, ty, surrogate, planar, general, gates);
    if (!k.fn) return BBX_ERR_UNSUPPORTED;
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
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
    *out = k;
    *ctas = per_sm * num_sms;
    return BBX_OK;
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
    float* d_div = nullptr;  // [3][nz][ny][px]: the fixed W-tilde sums of every node (k_divergence)
    bool wsum_zero = false;  // every W-tilde sum is exactly 0 (the step need not load them)
    bool wsum_elide = true;  // skip loading vanishing sums (bbx_set_wsum_elision)
    int pxf = 0;
    long long fplane = 0, fvol = 0;
    bool aniso = false;
    double Dpar = 1.0, Dperp = 1.0;

    int model = 0, S = 0;
    double par[8] = {0};
    double theta = 0.0;
    double dt = 0.0;
    float* d_state[2] = {nullptr, nullptr};
    bool bound = false;
    size_t bound_bytes = 0;
    int32_t* d_act = nullptr;
    float* d_rest = nullptr;  // 16 floats
    float4* d_tab = nullptr;  // V-table: chain matrices (BBX_BR_MRL) or Rush-Larsen coefficients (BBX_BR)
    double tab_dt = 0.0;      // the time step d_tab was built for
    int h_cur = 0;            // buffer parity as the enqueued work leaves it (mirror of d_dyn->cur)
    cudaStream_t copy_stream = nullptr;          // bbx_exchange_state: device-to-host copies
    cudaEvent_t ev_enter = nullptr, ev_out = nullptr;
    // bbx_exchange_state_async: two input and two output stages on the device,
    // a host-to-device and a device-to-host stream, and per stage the events
    // that order them against the grid's stream
    float* d_xin[2] = {nullptr, nullptr};
    float* d_xout[2] = {nullptr, nullptr};
    size_t x_bytes = 0;
    cudaStream_t xs_in = nullptr, xs_out = nullptr;
    cudaEvent_t xev_in_ready[2] = {}, xev_in_used[2] = {}, xev_out_ready[2] = {}, xev_out_done[2] = {};
    long long x_issued = 0;  // asynchronous exchanges issued since the stages were allocated
    int tab_model = 0;        // the model d_tab was built for
    double tab_tau_c = 0.0;   // and its tau_c (BBX_BR_FCA; 0 otherwise)
    bool tab_on = false;      // Beeler-Reuter with tabulated Rush-Larsen coefficients (bbx_set_tabulation)
    float* d_mp = nullptr;    // 8 floats

    uint8_t* d_stim = nullptr;
    double stim_amp = 0, t_on = 0, t_off = 0;
    bool stepped = false;

    int ty = 16, zb = 16;
    int nbx = 0, nby = 0, nbz = 0;
    int* d_bricks = nullptr;
    long long n_bricks = 0;
    std::vector<int> h_bricks;  // host copy of the active brick ids (masked grids)
    std::vector<uint8_t> h_chunks;  // masked 3D grids: tissue flag of each 16-wide chunk of each brick band

    TissueArgs h_t;                // host copy of the kernel's view of this grid
    TissueArgs* d_t = nullptr;     // device copy
    TissueDyn* d_dyn = nullptr;    // device-updated time, step, parity, total
    LaunchPlan lp;                 // single-grid launch
    bool ready = false;            // h_t, d_t and lp match the current settings
    unsigned long long version = 1;  // bumped whenever the kernel's view changes

    SurrogateData* d_surr = nullptr;  // reaction surrogate (Beeler-Reuter), owned
    bool surr_on = false;
    int split = 0;  // time-stepping scheme (bbx_set_scheme)
    int rk4 = 0;    // kinetics solver (bbx_set_solver)
    int resident = 0;  // multi-step resident kernel requested (bbx_set_resident)

    // z-slab of a decomposed grid: the first halo_lo and last halo_hi planes
    // are halo planes (a neighbour slab's boundary V, read by the stencil,
    // never computed); plane_tissue: tissue nodes per plane
    int halo_lo = 0, halo_hi = 0;
    // storage of the Beeler-Reuter gates (GATES_F32, GATES_F16, GATES_U16);
    // with 16 bits the buffers hold V and Ca as float planes, then the six
    // gates as uint16 planes.  d_stage: float staging plane for host copies.
    int gates = GATES_F32;
    float* d_stage = nullptr;
    std::vector<long long> plane_tissue;
    cudaEvent_t ev_halo = nullptr;

    double* d_partials = nullptr;  // bbx_total scratch
    unsigned int* d_ticket = nullptr;
    double* d_total2 = nullptr;
    int* d_err = nullptr;
    int* d_count = nullptr;  // phase-singularity counter (allocated on first use)
    int* h_small = nullptr;  // pinned host words: a small result and the error bits, read in one wait
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

// Float-sized words of one state buffer: S planes, or with 16-bit gates two
// float planes and six half-size planes.
size_t state_words(const bbx_grid* g) {
    return (size_t)(g->gates != GATES_F32 ? 5 : g->S) * (size_t)g->vol;
}
bool var_is16(const bbx_grid* g, int var) { return g->gates != GATES_F32 && var >= 2; }
int ensure_stage(bbx_grid* g) {  // the float staging plane of 16-bit host copies
    if (g->d_stage) return BBX_OK;
    if (dmalloc(&g->d_stage, sizeof(float) * (size_t)g->vol) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_NOMEM;
    }
    return BBX_OK;
}
uint16_t* gate_plane(const bbx_grid* g, int b, int var) {
    return reinterpret_cast<uint16_t*>(g->d_state[b] + 2 * (size_t)g->vol) + (size_t)(var - 2) * g->vol;
}

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
    g->h_bricks.clear();
    if (!g->d_mask) {
        g->n_bricks = nb;
        return BBX_OK;
    }
    uint8_t* flags = nullptr;
    long long* d_count = nullptr;
    if (dmalloc(&flags, nb) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_NOMEM;
        }
    if (dmalloc(&g->d_bricks, sizeof(int) * nb) != cudaSuccess || dmalloc(&d_count, sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
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
    if (e != cudaSuccess) return fail_cuda(e);
    g->n_bricks = cnt;
    g->h_bricks.resize((size_t)cnt);
    if (cnt > 0) BBX_CUDA(cudaMemcpy(g->h_bricks.data(), g->d_bricks, sizeof(int) * cnt, cudaMemcpyDeviceToHost));
    g->h_chunks.clear();
    if (g->nz > 1) {
        // 16-wide chunk flags, from which the pieces of a masked 3D grid are cut
        const int ncx = (g->nx + kChunkX - 1) / kChunkX;
        const long long nc = (long long)ncx * g->nby * g->nbz;
        uint8_t* cflags = nullptr;
        if (nc > 0x7fffffffLL || dmalloc(&cflags, nc) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_NOMEM;
        }
        k_chunk_flags<<<(unsigned)nc, 256, 0, g->stream>>>(g->d_mask, g->nx, g->ny, g->nz, g->px, g->plane, g->ty,
                                                            g->zb, ncx, g->nby, cflags);
        g->h_chunks.resize((size_t)nc);
        cudaError_t e2 = cudaGetLastError();
        if (e2 == cudaSuccess)
            e2 = cudaMemcpyAsync(g->h_chunks.data(), cflags, nc, cudaMemcpyDeviceToHost, g->stream);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(g->stream);
        cudaFree(cflags);
        if (e2 != cudaSuccess) return fail_cuda(e2);
    }
    return BBX_OK;
}

// Masked 3D grid: in each band of ty rows by zb planes, the 16-wide chunks
// that hold tissue (flags [bz][by][cx]) are covered from the left by 64-wide
// pieces starting at a chunk (so a wall that crosses a 64-column boundary
// costs one piece, not two); pieces with the same origin in consecutive bands
// of a row band merge into one z-run.  Every tissue node lies in exactly one
// piece.  Host-only.
void cover_chunks(const uint8_t* flags, int ncx, int nby, int nbz, int ty, int zb, int nz, int tissue,
                  std::vector<Seg>* segs) {
    const int per = kTileX / kChunkX;
    for (int by = 0; by < nby; ++by) {
        std::map<int, std::vector<int>> runs;  // piece origin x0 -> bands bz holding a piece there
        for (int bz = 0; bz < nbz; ++bz) {
            const uint8_t* f = flags + ((size_t)bz * nby + by) * ncx;
            for (int c = 0; c < ncx;) {
                if (!f[c]) {
                    ++c;
                    continue;
                }
                runs[c * kChunkX].push_back(bz);
                c += per;
            }
        }
        for (const auto& kv : runs) {
            const std::vector<int>& zs = kv.second;
            size_t i = 0;
            while (i < zs.size()) {
                size_t j = i;
                while (j + 1 < zs.size() && zs[j + 1] == zs[j] + 1) ++j;
                segs->push_back({tissue, kv.first, by * ty, zs[i] * zb, std::min((zs[j] + 1) * zb, nz)});
                i = j + 1;
            }
        }
    }
}

// Active columns (64 x ty nodes) of a grid with their active z-runs, for the
// given tile rows (the brick list must have been built for g->ty).
void grid_segments(const bbx_grid* g, int tissue, std::vector<Seg>* segs) {
    if (g->nz == 1) {
        // a sheet: runs of tiles down each column, (z0, z1) = tile range
        if (!g->d_mask) {
            for (int bx = 0; bx < g->nbx; ++bx) segs->push_back({tissue, bx * kTileX, 0, 0, g->nby});
            return;
        }
        std::vector<std::vector<int>> col((size_t)g->nbx);
        for (int id : g->h_bricks) col[(size_t)(id % g->nbx)].push_back(id / g->nbx);  // (nz = 1: by = id / nbx)
        for (int bx = 0; bx < g->nbx; ++bx) {
            const std::vector<int>& ys = col[(size_t)bx];
            size_t i = 0;
            while (i < ys.size()) {
                size_t j = i;
                while (j + 1 < ys.size() && ys[j + 1] == ys[j] + 1) ++j;
                segs->push_back({tissue, bx * kTileX, 0, ys[i], ys[j] + 1});
                i = j + 1;
            }
        }
        return;
    }
    // a z-slab computes only the planes between its halo planes
    const int zlo = g->halo_lo, zhi = g->nz - g->halo_hi;
    if (!g->d_mask) {
        for (int by = 0; by < g->nby; ++by)
            for (int bx = 0; bx < g->nbx; ++bx) segs->push_back({tissue, bx * kTileX, by * g->ty, zlo, zhi});
        return;
    }
    std::vector<Seg> all;
    cover_chunks(g->h_chunks.data(), (g->nx + kChunkX - 1) / kChunkX, g->nby, g->nbz, g->ty, g->zb, g->nz, tissue,
                 &all);
    for (Seg sg : all) {
        sg.z0 = std::max(sg.z0, zlo);
        sg.z1 = std::min(sg.z1, zhi);
        if (sg.z1 > sg.z0) segs->push_back(sg);
    }
}

// The kernel's view of a grid for tile rows `ty` (tensor maps depend on it).
int encode_targs(const bbx_grid* g, int ty, TissueArgs* t) {
    if (!get_encoder()) return BBX_ERR_CUDA;
    memset((void*)t, 0, sizeof(TissueArgs));
    const cuuint64_t dims3[3] = {(cuuint64_t)g->nx, (cuuint64_t)g->ny, (cuuint64_t)g->nz};
    const cuuint64_t str3[2] = {(cuuint64_t)g->px * 4, (cuuint64_t)g->plane * 4};
    const cuuint32_t ubox[3] = {(cuuint32_t)(kTileX + 8), (cuuint32_t)(ty + 2), 1};
    const bool g16 = g->gates != GATES_F32;
    const int s32 = g16 ? 2 : g->S;  // 32-bit variables (V first)
    const cuuint64_t sdims4[4] = {(cuuint64_t)g->nx, (cuuint64_t)g->ny, (cuuint64_t)g->nz, (cuuint64_t)s32};
    const cuuint64_t str4[3] = {(cuuint64_t)g->px * 4, (cuuint64_t)g->plane * 4, (cuuint64_t)g->vol * 4};
    const cuuint32_t sbox[4] = {(cuuint32_t)kTileX, (cuuint32_t)ty, 1, (cuuint32_t)(s32 > 1 ? s32 - 1 : 1)};
    const cuuint64_t gdims4[4] = {(cuuint64_t)g->nx, (cuuint64_t)g->ny, (cuuint64_t)g->nz, 6};
    const cuuint64_t gstr4[3] = {(cuuint64_t)g->px * 2, (cuuint64_t)g->plane * 2, (cuuint64_t)g->vol * 2};
    const cuuint32_t gbox[4] = {(cuuint32_t)kTileX, (cuuint32_t)ty, 1, 6};
    for (int b = 0; b < 2; ++b) {
        if (!encode(&t->tm_u[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, g->d_state[b], dims3, str3, ubox))
            return BBX_ERR_CUDA;
        if (g->S > 1) {
            if (!encode(&t->tm_s[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->d_state[b], sdims4, str4, sbox))
                return BBX_ERR_CUDA;
        } else {
            t->tm_s[b] = t->tm_u[b];
        }
        if (g16) {
            if (!encode(&t->tm_g[b], CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, gate_plane(g, b, 2), gdims4, gstr4, gbox))
                return BBX_ERR_CUDA;
            t->gate16[b] = gate_plane(g, b, 2);
        } else {
            t->tm_g[b] = t->tm_u[b];
            t->gate16[b] = nullptr;
        }
    }
    if (g->aniso) {
        const cuuint64_t fd4[4] = {(cuuint64_t)g->pxf, (cuuint64_t)g->ny, (cuuint64_t)g->nz, 3};
        const cuuint64_t fstr4[3] = {(cuuint64_t)g->pxf * 4, (cuuint64_t)g->fplane * 4, (cuuint64_t)g->fvol * 4};
        const cuuint32_t fbox[4] = {(cuuint32_t)kTileX, (cuuint32_t)ty, 1, 3};  // a tile's own fibres
        if (!encode(&t->tm_f, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->d_fib, fd4, fstr4, fbox)) return BBX_ERR_CUDA;
        const cuuint64_t dd4[4] = {(cuuint64_t)g->nx, (cuuint64_t)g->ny, (cuuint64_t)g->nz, 3};
        if (!encode(&t->tm_d, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->d_div, dd4, str4, fbox)) return BBX_ERR_CUDA;
    } else {
        t->tm_f = t->tm_u[0];
        t->tm_d = t->tm_u[0];
    }
    if (g->d_mask) {
        const cuuint64_t mstr[2] = {(cuuint64_t)g->px, (cuuint64_t)g->plane};
        const cuuint32_t mbox[3] = {(cuuint32_t)(kTileX + 32), (cuuint32_t)(ty + 2), 1};
        if (!encode(&t->tm_m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, g->d_mask, dims3, mstr, mbox)) return BBX_ERR_CUDA;
    } else {
        t->tm_m = t->tm_u[0];
    }
    t->state[0] = g->d_state[0];
    t->state[1] = g->d_state[1];
    t->act = g->d_act;
    t->stim = g->d_stim;
    t->dyn = g->d_dyn;
    t->plane = g->plane;
    t->vol = g->vol;
    t->t_on = g->t_on;
    t->t_off = g->t_off;
    t->dt_d = g->dt;
    t->nx = g->nx;
    t->ny = g->ny;
    t->nz = g->nz;
    t->px = g->px;
    t->dt = (float)g->dt;
    t->theta = (float)g->theta;
    t->split = g->split;
    t->rk4 = g->rk4;
    t->wsum_zero = (g->aniso && g->wsum_zero && g->wsum_elide) ? 1 : 0;
    t->stim_amp = g->d_stim ? (float)g->stim_amp : 0.0f;
    const double ih2 = 1.0 / (g->h * g->h);
    const double cd = (g->Dpar - g->Dperp) * ih2;
    t->c_perp = (float)(g->Dperp * ih2);
    t->c_d = (float)cd;
    t->c_dh = (float)(0.5 * cd);
    t->c_s = (float)(0.25 * cd);
    t->c_iso = (float)(g->Dpar * ih2);
    model_kernel_params(g->model, g->par, t->mp);
    t->surr = (g->surr_on && g->model == BBX_BR) ? g->d_surr : nullptr;
    t->tab = (g->model == BBX_BR_MRL || g->model == BBX_BR_FCA || (g->model == BBX_BR && g->tab_on)) ? g->d_tab
                                                                                                    : nullptr;
    return BBX_OK;
}

int finish_total(bbx_grid* g);

// A grid that needs the general kernel variants (7- and 14-row tiles): the
// Lie scheme, the RK4 solver, or Beeler-Reuter with tabulated coefficients.
bool wants_general(const bbx_grid* g) { return g->split || g->rk4 || (g->tab_on && g->model == BBX_BR); }

// The V-table of a grid that uses one (the Rush-Larsen coefficients of BBX_BR
// with tabulation on and of BBX_BR_FCA; those and the chain matrices of
// BBX_BR_MRL), allocated on first use and rebuilt on the grid's stream
// whenever the model, the time step or tau_c differs from the ones it was
// built for.
// The asynchronous exchange's stages, streams and events, after its copies end.
void exchange_release(bbx_grid* g) {
    if (g->xs_out) cudaStreamSynchronize(g->xs_out);
    if (g->xs_in) cudaStreamSynchronize(g->xs_in);
    for (int j = 0; j < 2; ++j) {
        cudaFree(g->d_xin[j]);
        cudaFree(g->d_xout[j]);
        g->d_xin[j] = g->d_xout[j] = nullptr;
        for (cudaEvent_t* e : {&g->xev_in_ready[j], &g->xev_in_used[j], &g->xev_out_ready[j], &g->xev_out_done[j]}) {
            if (*e) cudaEventDestroy(*e);
            *e = nullptr;
        }
    }
    if (g->xs_in) cudaStreamDestroy(g->xs_in);
    if (g->xs_out) cudaStreamDestroy(g->xs_out);
    g->xs_in = g->xs_out = nullptr;
    g->x_bytes = 0;
    g->x_issued = 0;
}

int tab_refresh(bbx_grid* g) {
    const bool want = g->model == BBX_BR_MRL || g->model == BBX_BR_FCA || (g->model == BBX_BR && g->tab_on);
    if (!want) return BBX_OK;
    if (!g->d_tab) {  // room for both tables of BBX_BR_MRL
        if (dmalloc(&g->d_tab, sizeof(float4) * 8 * (size_t)kTabN) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_NOMEM;
        }
        g->tab_model = 0;
    }
    const double tau_c = g->model == BBX_BR_FCA ? g->par[5] : 0.0;
    if (!(g->dt > 0.0) || (g->tab_dt == g->dt && g->tab_model == g->model && g->tab_tau_c == tau_c)) return BBX_OK;
    BBX_CUDA(br_build_rl_table(g->d_tab, g->dt, tau_c, g->stream));
    if (g->model == BBX_BR_MRL) BBX_CUDA(mrl_build_table(g->d_tab + 4 * (size_t)kTabN, g->dt, g->stream));
    g->tab_dt = g->dt;
    g->tab_model = g->model;
    g->tab_tau_c = tau_c;
    return BBX_OK;
}

// Bring h_t, d_t and the single-grid launch plan in line with the settings.
int prepare(bbx_grid* g) {
    g->ready = false;
    ++g->version;
    if (!g->model || !g->d_state[0]) return BBX_ERR_STATE;
    int rc0 = finish_total(g);  // the plan's partials are about to be replaced
    if (rc0 || (rc0 = tab_refresh(g))) return rc0;
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    StepKernel k;
    int ctas = 0;
    const bool surr = g->surr_on && g->model == BBX_BR;
    int rc = BBX_ERR_UNSUPPORTED;
    if (g->aniso && g->wsum_zero && g->wsum_elide && !g->d_mask)  // the variant without W-tilde sums, if built
        rc = select_kernel(g->model, false, AN_NO_SUMS, g->ty, g->device, g->num_sms, &k, &ctas, surr, g->nz == 1,
                           wants_general(g), g->gates);
    if (rc == BBX_ERR_UNSUPPORTED)
        rc = select_kernel(g->model, g->d_mask != nullptr, g->aniso ? AN_SUMS : AN_ISO, g->ty, g->device,
                           g->num_sms, &k, &ctas, surr, g->nz == 1, wants_general(g), g->gates);
    if (rc) return rc;
    if ((rc = encode_targs(g, g->ty, &g->h_t))) return rc;
    BBX_CUDA(cudaMemcpyAsync(g->d_t, &g->h_t, sizeof(TissueArgs), cudaMemcpyHostToDevice, g->stream));
    std::vector<Seg> segs;
    grid_segments(g, 0, &segs);
    g->lp.k = k;
    if ((rc = build_plan(&g->lp, segs, 1, ctas))) return rc;
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    g->ready = true;
    return BBX_OK;
}

// Refresh only the scalar fields of the kernel's view (threshold, stimulus,
// time step) without rebuilding the plan.
int refresh_targs(bbx_grid* g) {
    if (!g->ready) return prepare(g);
    int rc = tab_refresh(g);
    if (rc) return rc;
    ++g->version;
    g->h_t.t_on = g->t_on;
    g->h_t.t_off = g->t_off;
    g->h_t.dt_d = g->dt;
    g->h_t.dt = (float)g->dt;
    g->h_t.theta = (float)g->theta;
    g->h_t.split = g->split;
    g->h_t.rk4 = g->rk4;
    g->h_t.stim = g->d_stim;
    g->h_t.stim_amp = g->d_stim ? (float)g->stim_amp : 0.0f;
    BBX_CUDA(cudaMemcpyAsync(g->d_t, &g->h_t, sizeof(TissueArgs), cudaMemcpyHostToDevice, g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    return BBX_OK;
}

int read_dyn(bbx_grid* g, TissueDyn* d) {
    BBX_CUDA(cudaMemcpyAsync(d, g->d_dyn, sizeof(TissueDyn), cudaMemcpyDeviceToHost, g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    g->h_cur = d->cur;  // nothing is in flight: the device value is the parity
    return BBX_OK;
}

int write_dyn(bbx_grid* g, const TissueDyn& d) {
    BBX_CUDA(cudaMemcpyAsync(g->d_dyn, &d, sizeof(TissueDyn), cudaMemcpyHostToDevice, g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    g->h_cur = d.cur;
    return BBX_OK;
}

// Enqueue the sum of a pending single-grid total from the plan's partials
// (nothing happens on the device when none is pending).  Called before
// anything that reads the total or overwrites the partials.
int finish_total(bbx_grid* g) {
    if (!g->lp.d_partials || g->lp.n_slots <= 0 || !g->d_dyn) return BBX_OK;
    k_finish_total<<<1, 256, 0, g->stream>>>(g->lp.d_partials, g->lp.n_slots, g->d_dyn, g->d_err);
    BBX_CUDA(cudaGetLastError());
    return BBX_OK;
}

int check_sticky_ptr(cudaStream_t s, int* d_err) {
    int err = 0;
    BBX_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BBX_CUDA(cudaStreamSynchronize(s));
    if (err & ERRBIT_TIMEOUT) return BBX_ERR_TIMEOUT;
    if (err & ERRBIT_NAN) return BBX_ERR_NAN;
    if (err & ERRBIT_HINT) return BBX_ERR_STATE;  // host and device disagreed on the schedule or parity
    return BBX_OK;
}

int check_sticky(bbx_grid* g) { return check_sticky_ptr(g->stream, g->d_err); }

// A 4-byte device result and the grid's error bits copied to pinned host
// memory together, with one wait for the stream (one round trip instead of
// two); then the sticky-error check as check_sticky.
int read_word_and_sticky(bbx_grid* g, const int* d_word, int* out) {
    if (!g->h_small && cudaMallocHost(&g->h_small, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        g->h_small = nullptr;
        BBX_CUDA(cudaMemcpyAsync(out, d_word, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
        return check_sticky(g);
    }
    BBX_CUDA(cudaMemcpyAsync(g->h_small, d_word, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    BBX_CUDA(cudaMemcpyAsync(g->h_small + 1, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    *out = g->h_small[0];
    const int err = g->h_small[1];
    if (err & ERRBIT_TIMEOUT) return BBX_ERR_TIMEOUT;
    if (err & ERRBIT_NAN) return BBX_ERR_NAN;
    if (err & ERRBIT_HINT) return BBX_ERR_STATE;
    return BBX_OK;
}

// Dense host field <-> pitched device field; one linear copy when the rows
// are not padded (nx a multiple of 32).
int copy_in(bbx_grid* g, void* dst, const void* src, size_t elem) {
    if (g->px == g->nx) {
        BBX_CUDA(cudaMemcpyAsync(dst, src, (size_t)g->ncell * elem, cudaMemcpyHostToDevice, g->stream));
        return BBX_OK;
    }
    BBX_CUDA(cudaMemcpy2DAsync(dst, (size_t)g->px * elem, src, (size_t)g->nx * elem, (size_t)g->nx * elem,
                               (size_t)g->ny * g->nz, cudaMemcpyHostToDevice, g->stream));
    return BBX_OK;
}

int copy_out(bbx_grid* g, void* dst, const void* src, size_t elem) {
    if (g->px == g->nx) {
        BBX_CUDA(cudaMemcpyAsync(dst, src, (size_t)g->ncell * elem, cudaMemcpyDeviceToHost, g->stream));
        return BBX_OK;
    }
    BBX_CUDA(cudaMemcpy2DAsync(dst, (size_t)g->nx * elem, src, (size_t)g->px * elem, (size_t)g->nx * elem,
                               (size_t)g->ny * g->nz, cudaMemcpyDeviceToHost, g->stream));
    return BBX_OK;
}

// Forward Euler stability of the diffusion part: Gershgorin bound on the
// spectrum of the discrete operator, |lambda| <= (4 tr D + 2 |Dpar - Dperp|)/h^2.
bool stable(const bbx_grid* g, double dt) {
    const double trD = g->aniso ? (g->Dpar + 2.0 * g->Dperp) : 3.0 * g->Dpar;
    const double dD = g->aniso ? std::fabs(g->Dpar - g->Dperp) : 0.0;
    return dt * (4.0 * trD + 2.0 * dD) <= 2.0 * g->h * g->h;
}

int set_dt(bbx_grid* g, double dt) {
    if (!(dt > 0.0) || !std::isfinite(dt)) return BBX_ERR_ARG;
    if (!stable(g, dt)) return BBX_ERR_UNSTABLE;
    if (dt != g->dt || !g->ready) {
        g->dt = dt;
        return refresh_targs(g);
    }
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
    exchange_release(g);
    if (g->copy_stream) {
        cudaStreamSynchronize(g->copy_stream);
        cudaStreamDestroy(g->copy_stream);
    }
    if (g->ev_enter) cudaEventDestroy(g->ev_enter);
    if (g->ev_out) cudaEventDestroy(g->ev_out);
    if (g->ev_halo) cudaEventDestroy(g->ev_halo);
    cudaFree(g->d_stage);
    cudaFree(g->d_mask);
    cudaFree(g->d_fib);
    cudaFree(g->d_div);
    if (!g->bound) {
        cudaFree(g->d_state[0]);
        cudaFree(g->d_state[1]);
    }
    cudaFree(g->d_act);
    cudaFree(g->d_rest);
    cudaFree(g->d_tab);
    cudaFree(g->d_mp);
    cudaFree(g->d_stim);
    cudaFree(g->d_bricks);
    cudaFree(g->d_t);
    cudaFree(g->d_dyn);
    cudaFree(g->d_surr);
    g->lp.release();
    cudaFree(g->d_partials);
    cudaFree(g->d_ticket);
    cudaFree(g->d_total2);
    cudaFree(g->d_err);
    cudaFree(g->d_count);
    if (g->h_small) cudaFreeHost(g->h_small);
    cudaGetLastError();
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
    g->ty = 14;
    int rc = BBX_OK;
    do {
        if (cudaGetDevice(&g->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
            cudaGetLastError();
            rc = BBX_ERR_CUDA;
            break;
        }
        if (dmalloc(&g->d_partials, sizeof(double) * kMaxPartials) != cudaSuccess ||
            dmalloc(&g->d_ticket, sizeof(unsigned int)) != cudaSuccess ||
            dmalloc(&g->d_total2, sizeof(double)) != cudaSuccess || dmalloc(&g->d_err, sizeof(int)) != cudaSuccess ||
            dmalloc(&g->d_rest, sizeof(float) * 16) != cudaSuccess ||
            dmalloc(&g->d_mp, sizeof(float) * 8) != cudaSuccess ||
            dmalloc(&g->d_t, sizeof(TissueArgs)) != cudaSuccess ||
            dmalloc(&g->d_dyn, sizeof(TissueDyn)) != cudaSuccess) {
            cudaGetLastError();
            rc = BBX_ERR_NOMEM;
            break;
        }
        if (cudaMemsetAsync(g->d_ticket, 0, sizeof(unsigned int), g->stream) != cudaSuccess ||
            cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream) != cudaSuccess ||
            cudaMemsetAsync(g->d_dyn, 0, sizeof(TissueDyn), g->stream) != cudaSuccess) {
            cudaGetLastError();
            rc = BBX_ERR_CUDA;
            break;
        }
        g->plane_tissue.assign((size_t)nz, (long long)nx * ny);
        if (mask_host) {
            long long nt = 0;
            for (int z = 0; z < nz; ++z) {
                long long c = 0;
                const uint8_t* m = mask_host + (size_t)z * nx * ny;
                for (long long i = 0; i < (long long)nx * ny; ++i) c += m[i] != 0;
                g->plane_tissue[(size_t)z] = c;
                nt += c;
            }
            g->n_tissue = nt;
            if (dmalloc(&g->d_mask, (size_t)g->vol) != cudaSuccess) {
                cudaGetLastError();
                rc = BBX_ERR_NOMEM;
                break;
            }
            if (cudaMemsetAsync(g->d_mask, 0, (size_t)g->vol, g->stream) != cudaSuccess) {
                cudaGetLastError();
                rc = BBX_ERR_CUDA;
                break;
            }
            std::vector<uint8_t> m01(ncell);
            for (long long i = 0; i < ncell; ++i) m01[i] = mask_host[i] ? 1 : 0;
            uint8_t* tmp = nullptr;
            if (dmalloc(&tmp, (size_t)g->vol) != cudaSuccess) {
                cudaGetLastError();
                rc = BBX_ERR_NOMEM;
                break;
            }
            if (cudaMemsetAsync(tmp, 0, (size_t)g->vol, g->stream) != cudaSuccess ||
                (rc = copy_in(g, tmp, m01.data(), 1)) != BBX_OK) {
                cudaGetLastError();
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
                cudaGetLastError();
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
        cudaStreamSynchronize(g->stream);
        cudaFree(g->d_fib);
        cudaFree(g->d_div);
        g->d_fib = nullptr;
        g->d_div = nullptr;
        g->aniso = false;
        g->Dpar = g->Dperp = D_par;
    } else {
        float* tmp = nullptr;
        float* fib = nullptr;
        const int pxf = (g->nx + 8 + 31) / 32 * 32;
        const long long fplane = (long long)pxf * g->ny, fvol = fplane * g->nz;
        if (dmalloc(&tmp, sizeof(float) * 3 * g->ncell) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_NOMEM;
        }
        if (dmalloc(&fib, sizeof(float) * 3 * fvol) != cudaSuccess) {
            cudaGetLastError();
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
        if (e != cudaSuccess) rc = fail_cuda(e);
        else if (err & kErrFibre) rc = BBX_ERR_FIBRE;
        float* div = nullptr;
        if (rc == BBX_OK) {
            if (dmalloc(&div, sizeof(float) * 3 * (size_t)g->vol) != cudaSuccess) {
                cudaGetLastError();
                rc = BBX_ERR_NOMEM;
            } else {
                e = cudaMemsetAsync(div, 0, sizeof(float) * 3 * (size_t)g->vol, g->stream);
                if (e == cudaSuccess) {
                    // g->d_err is clear here (reset after the fibre check); it
                    // carries the "some sum is nonzero" word for this one call
                    k_divergence<<<n_blocks_for(g->ncell, 256), 256, 0, g->stream>>>(
                        fib, g->nx, g->ny, g->nz, pxf, fplane, fvol, g->d_mask, g->px, g->plane, g->vol, div,
                        g->d_err);
                    e = cudaGetLastError();
                }
                int nonzero = 1;
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(&nonzero, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream);
                if (e == cudaSuccess) e = cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
                if (e != cudaSuccess) rc = fail_cuda(e);
                else g->wsum_zero = (nonzero == 0);
            }
        }
        if (rc != BBX_OK) {
            cudaFree(fib);
            cudaFree(div);
            return rc;
        }
        cudaStreamSynchronize(g->stream);
        cudaFree(g->d_fib);
        cudaFree(g->d_div);
        g->d_fib = fib;
        g->d_div = div;
        g->pxf = pxf;
        g->fplane = fplane;
        g->fvol = fvol;
        g->aniso = true;
        g->Dpar = D_par;
        g->Dperp = D_perp;
    }
    if (g->dt > 0.0 && !stable(g, g->dt)) g->dt = 0.0;  // the next step must choose a stable dt
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
    // parameters the kernels divide by, and the calcium gate's constants
    if ((model == BBX_FHN && p[0] == 0.0) || (model == BBX_BARKLEY && (p[0] == 0.0 || p[2] == 0.0)) ||
        (model == BBX_BR_FCA && (!(p[4] > 0.0) || !(p[5] > 0.0) || p[6] < 0.0)))
        return BBX_ERR_ARG;
    cudaStreamSynchronize(g->stream);
    const size_t old_words = g->d_state[0] ? state_words(g) : 0;
    g->gates = GATES_F32;  // a new model starts with 32-bit storage
    if (g->bound && S != g->S) {
        g->bound = false;  // the caller's buffers no longer fit: back to library buffers
        g->d_state[0] = g->d_state[1] = nullptr;
    }
    if (!g->bound && ((size_t)S * g->vol != old_words || !g->d_state[0])) {
        cudaFree(g->d_state[0]);
        cudaFree(g->d_state[1]);
        g->d_state[0] = g->d_state[1] = nullptr;
        if (dmalloc(&g->d_state[0], sizeof(float) * S * g->vol) != cudaSuccess ||
            dmalloc(&g->d_state[1], sizeof(float) * S * g->vol) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_NOMEM;
        }
    }
    if (!g->d_act && dmalloc(&g->d_act, sizeof(int32_t) * g->vol) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_NOMEM;
    }
    if (model != BBX_BR) g->surr_on = false;
    if (model == BBX_BR || model == BBX_BR_MRL || model == BBX_BR_FCA) g->rk4 = 0;  // Euler / Rush-Larsen
    if (model == BBX_BR_MRL || model == BBX_BR_FCA) g->split = 0;  // unsplit only (no Lie-scheme kernels)
    if (model != BBX_BR) g->tab_on = false;
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
    BBX_CUDA(cudaMemsetAsync(g->d_dyn, 0, sizeof(TissueDyn), g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    g->h_cur = 0;
    g->stepped = false;
    return prepare(g);
}

int bbx_bind_state(bbx_grid* g, void* a, void* b, size_t bytes) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (!a || !b || a == b || (reinterpret_cast<uintptr_t>(a) & 15) || (reinterpret_cast<uintptr_t>(b) & 15) ||
        bytes < sizeof(float) * state_words(g))
        return BBX_ERR_ARG;
    cudaStreamSynchronize(g->stream);
    if (!g->bound) {
        cudaFree(g->d_state[0]);
        cudaFree(g->d_state[1]);
    }
    g->d_state[0] = static_cast<float*>(a);
    g->d_state[1] = static_cast<float*>(b);
    g->bound = true;
    g->bound_bytes = bytes;
    for (int k = 0; k < 2; ++k) {
        if (g->gates != GATES_F32)
            k_fill_state16<<<n_blocks_for(g->vol, 256), 256, 0, g->stream>>>(g->d_state[k], g->vol, g->d_rest,
                                                                              g->gates);
        else
            k_fill_state<<<n_blocks_for((long long)g->S * g->vol, 256), 256, 0, g->stream>>>(g->d_state[k], g->S,
                                                                                                g->vol, g->d_rest);
    }
    BBX_CUDA(cudaGetLastError());
    TissueDyn d;
    int rc = read_dyn(g, &d);
    if (rc) return rc;
    d.cur = 0;
    if ((rc = write_dyn(g, d))) return rc;
    return prepare(g);
}

int bbx_write_state(bbx_grid* g, int var, const float* host, size_t n) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (var < 0 || var >= g->S || !host || n != (size_t)g->ncell) return BBX_ERR_ARG;
    // both ping-pong buffers get the values (void nodes are never rewritten
    // by a step, so the buffers must agree there): one copy from the host,
    // one on the device
    if (var_is16(g, var)) {
        int rc = ensure_stage(g);
        if (rc || (rc = copy_in(g, g->d_stage, host, sizeof(float)))) return rc;
        k_pack16<<<n_blocks_for(g->vol, 256), 256, 0, g->stream>>>(g->d_stage, gate_plane(g, 0, var), g->vol,
                                                                     g->gates);
        BBX_CUDA(cudaGetLastError());
        BBX_CUDA(cudaMemcpyAsync(gate_plane(g, 1, var), gate_plane(g, 0, var), sizeof(uint16_t) * (size_t)g->vol,
                                 cudaMemcpyDeviceToDevice, g->stream));
        BBX_CUDA(cudaStreamSynchronize(g->stream));
        return BBX_OK;
    }
    float* b0 = g->d_state[0] + (size_t)var * g->vol;
    float* b1 = g->d_state[1] + (size_t)var * g->vol;
    int rc = copy_in(g, b0, host, sizeof(float));
    if (rc) return rc;
    BBX_CUDA(cudaMemcpyAsync(b1, b0, sizeof(float) * (size_t)g->vol, cudaMemcpyDeviceToDevice, g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    return BBX_OK;
}

int bbx_write_all(bbx_grid* g, const float* host, size_t n) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (!host || n != (size_t)g->S * (size_t)g->ncell) return BBX_ERR_ARG;
    if (g->gates != GATES_F32) {  // 16-bit gates: variable by variable, through the float staging plane
        for (int v = 0; v < g->S; ++v) {
            int rc = bbx_write_state(g, v, host + (size_t)v * g->ncell, (size_t)g->ncell);
            if (rc) return rc;
        }
        return BBX_OK;
    }
    // every variable into buffer 0, then buffer 0 into buffer 1 in one
    // device copy (both hold the state, as bbx_write_state leaves them); one
    // synchronisation at the end
    if (g->px == g->nx) {
        BBX_CUDA(cudaMemcpyAsync(g->d_state[0], host, sizeof(float) * n, cudaMemcpyHostToDevice, g->stream));
    } else {
        for (int v = 0; v < g->S; ++v) {
            int rc = copy_in(g, g->d_state[0] + (size_t)v * g->vol, host + (size_t)v * g->ncell, sizeof(float));
            if (rc) return rc;
        }
    }
    BBX_CUDA(cudaMemcpyAsync(g->d_state[1], g->d_state[0], sizeof(float) * (size_t)g->S * g->vol,
                             cudaMemcpyDeviceToDevice, g->stream));
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    return BBX_OK;
}

int bbx_set_stimulus(bbx_grid* g, const uint8_t* region, double amp, double t_on, double t_off) {
    if (!g || !std::isfinite(amp) || std::isnan(t_on) || std::isnan(t_off)) return BBX_ERR_ARG;
    if (!region) {
        cudaStreamSynchronize(g->stream);
        cudaFree(g->d_stim);
        g->d_stim = nullptr;
        g->stim_amp = 0.0;
        return g->model ? refresh_targs(g) : BBX_OK;
    }
    if (!g->d_stim) {
        if (dmalloc(&g->d_stim, (size_t)g->vol) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_NOMEM;
        }
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
    return g->model ? refresh_targs(g) : BBX_OK;
}

int bbx_set_threshold(bbx_grid* g, double theta) {
    if (!g || !std::isfinite(theta)) return BBX_ERR_ARG;
    g->theta = theta;
    return g->model ? refresh_targs(g) : BBX_OK;
}

// The resident multi-step kernel serves small unmasked isotropic sheets of the
// models given by a right-hand side, with the default scheme and solver.
static bool resident_eligible(const bbx_grid* g) {
    return g->nz == 1 && !g->d_mask && !g->aniso && !g->split && !g->rk4 && !g->surr_on && !g->poison &&
           (g->model == BBX_FHN || g->model == BBX_BARKLEY || g->model == BBX_ZFK || g->model == BBX_DIFFUSION);
}

static int apply_kinetics_setting(bbx_grid* g);

int bbx_set_tabulation(bbx_grid* g, int on) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (g->model != BBX_BR) return BBX_ERR_UNSUPPORTED;
    g->tab_on = on != 0;
    return apply_kinetics_setting(g);
}

int bbx_set_wsum_elision(bbx_grid* g, int on) {
    if (!g) return BBX_ERR_ARG;
    g->wsum_elide = on != 0;
    return g->model ? prepare(g) : BBX_OK;
}

int bbx_set_resident(bbx_grid* g, int on) {
    if (!g) return BBX_ERR_ARG;
    if (!on) {
        g->resident = 0;
        return BBX_OK;
    }
    if (!g->model) return BBX_ERR_STATE;
    if (!resident_eligible(g)) return BBX_ERR_UNSUPPORTED;
    bool ok = false;
    if (resident_sheet_steps(g->model, nullptr, g->nx, g->ny, 0, nullptr, g->stream, true, &ok) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_CUDA;
    }
    if (!ok) return BBX_ERR_UNSUPPORTED;
    g->resident = 1;
    return BBX_OK;
}

// The scheme and solver select the kernel variant (the general one has no
// 28-row tiles: such a grid moves to 14 rows).
static int apply_kinetics_setting(bbx_grid* g) {
    if (!g->model) return BBX_OK;
    if (wants_general(g) && g->ty == 28) return bbx_set_tiling(g, 14, g->zb);
    return prepare(g);
}

int bbx_set_scheme(bbx_grid* g, int scheme) {
    if (!g || (scheme != BBX_SCHEME_UNSPLIT && scheme != BBX_SCHEME_LIE)) return BBX_ERR_ARG;
    if (scheme == BBX_SCHEME_LIE && (g->model == BBX_BR_MRL || g->model == BBX_BR_FCA)) return BBX_ERR_UNSUPPORTED;
    g->split = scheme == BBX_SCHEME_LIE ? 1 : 0;
    return apply_kinetics_setting(g);
}

int bbx_set_solver(bbx_grid* g, int solver) {
    if (!g || (solver != BBX_SOLVER_EULER && solver != BBX_SOLVER_RK4)) return BBX_ERR_ARG;
    if (solver == BBX_SOLVER_RK4 && (g->model == BBX_BR || g->model == BBX_BR_MRL || g->model == BBX_BR_FCA))
        return BBX_ERR_UNSUPPORTED;
    g->rk4 = solver == BBX_SOLVER_RK4 ? 1 : 0;
    return apply_kinetics_setting(g);
}

int bbx_set_timestep(bbx_grid* g, double dt) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    return set_dt(g, dt);
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
    int rc = set_dt(g, dt);
    if (rc) return rc;
    if (n_steps == 0) return BBX_OK;
    if (!g->ready && (rc = prepare(g))) return rc;
    if (g->lp.n_planes == 0) {
        // no tissue: nothing moves, only time advances
        TissueDyn d;
        if ((rc = read_dyn(g, &d))) return rc;
        for (int s = 0; s < n_steps; ++s) {
            d.t += dt;
            d.n += 1;
        }
        d.total = 0.0;
        d.total_pending = 0;
        if ((rc = write_dyn(g, d))) return rc;
        g->stepped = true;
        return BBX_OK;
    }
    if (g->resident && n_steps >= 2 && resident_eligible(g)) {
        int done = 0;
        while (done < n_steps) {
            const int chunk = std::min(n_steps - done, 1 << 16);
            bool ok = false;
            const cudaError_t e = resident_sheet_steps(g->model, g->d_t, g->nx, g->ny, chunk, g->d_err, g->stream,
                                                       false, &ok);
            if (e != cudaSuccess) return fail_cuda(e);
            if (!ok) break;  // not launchable after all: the tiled kernel takes the rest
            done += chunk;
            g->h_cur ^= chunk & 1;
        }
        if (done > 0) g->stepped = true;
        n_steps -= done;
        if (n_steps == 0) return BBX_OK;
    }
    LaunchArgs L = launch_args(g->lp, g->d_t, g->d_err, g->poison, &g->h_t);
    if (!g->d_mask) {
        // unmasked grid: whole columns in order (nz planes, or a sheet's nby
        // tile rows), equal shares (build_plan)
        L.reg_len = g->nz > 1 ? g->nz - g->halo_lo - g->halo_hi : g->nby;
        L.reg_z0 = g->nz > 1 ? g->halo_lo : 0;
        L.reg_nbx = g->nbx;
        L.reg_ty = g->ty;
        L.reg_ctas = g->lp.ctas;
        L.reg_planes = g->lp.n_planes;
    }
    for (int s = 0; s < n_steps; ++s) {
        L.cur_hint = g->h_cur;
        const cudaError_t e = launch(g->lp, L, g->stream);
        if (e != cudaSuccess) return fail_cuda(e);
        g->h_cur ^= 1;
    }
    g->stepped = true;
    return BBX_OK;
}

int bbx_read_state(bbx_grid* g, int var, float* host, size_t n) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (var < 0 || var >= g->S || !host || n != (size_t)g->ncell) return BBX_ERR_ARG;
    TissueDyn d;
    int rc = read_dyn(g, &d);
    if (rc) return rc;
    if (var_is16(g, var)) {
        if ((rc = ensure_stage(g))) return rc;
        k_unpack16<<<n_blocks_for(g->vol, 256), 256, 0, g->stream>>>(gate_plane(g, d.cur, var), g->d_stage, g->vol,
                                                                       g->gates);
        BBX_CUDA(cudaGetLastError());
        rc = copy_out(g, host, g->d_stage, sizeof(float));
    } else {
        rc = copy_out(g, host, g->d_state[d.cur] + (size_t)var * g->vol, sizeof(float));
    }
    if (rc) return rc;
    return check_sticky(g);
}

int bbx_read_all(bbx_grid* g, float* host, size_t n) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (!host || n != (size_t)g->S * (size_t)g->ncell) return BBX_ERR_ARG;
    if (g->gates != GATES_F32) {
        for (int v = 0; v < g->S; ++v) {
            int rc = bbx_read_state(g, v, host + (size_t)v * g->ncell, (size_t)g->ncell);
            if (rc) return rc;
        }
        return BBX_OK;
    }
    TissueDyn d;
    int rc = read_dyn(g, &d);
    if (rc) return rc;
    const float* src = g->d_state[d.cur];
    if (g->px == g->nx) {
        BBX_CUDA(cudaMemcpyAsync(host, src, sizeof(float) * n, cudaMemcpyDeviceToHost, g->stream));
    } else {
        for (int v = 0; v < g->S; ++v)
            if ((rc = copy_out(g, host + (size_t)v * g->ncell, src + (size_t)v * g->vol, sizeof(float)))) return rc;
    }
    return check_sticky(g);
}

int bbx_exchange_state(bbx_grid* g, const float* host_in, float* host_out, size_t n) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (g->x_issued) {  // asynchronous exchanges still writing the caller's buffers
        const int rc = bbx_exchange_wait(g);
        if (rc) return rc;
    }
    if (!host_in || !host_out || n != (size_t)g->S * (size_t)g->ncell) return BBX_ERR_ARG;
    if (g->px != g->nx || g->gates != GATES_F32) {  // padded rows or 16-bit gates: one direction after the other
        int rc = bbx_read_all(g, host_out, n);
        return rc ? rc : bbx_write_all(g, host_in, n);
    }
    if (!g->copy_stream) {
        if (cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g->ev_enter, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_CUDA;
        }
    }
    const int cur = g->h_cur, oth = cur ^ 1;
    const size_t bytes = sizeof(float) * n;
    // the current state out on the copy stream, after everything enqueued so far ...
    BBX_CUDA(cudaEventRecord(g->ev_enter, g->stream));
    BBX_CUDA(cudaStreamWaitEvent(g->copy_stream, g->ev_enter, 0));
    BBX_CUDA(cudaMemcpyAsync(host_out, g->d_state[cur], bytes, cudaMemcpyDeviceToHost, g->copy_stream));
    // ... while the new one comes into the other buffer on the grid's stream
    BBX_CUDA(cudaMemcpyAsync(g->d_state[oth], host_in, bytes, cudaMemcpyHostToDevice, g->stream));
    BBX_CUDA(cudaEventRecord(g->ev_out, g->copy_stream));
    BBX_CUDA(cudaStreamWaitEvent(g->stream, g->ev_out, 0));  // nothing overwrites the old buffer before it is out
    if (g->d_mask)  // void nodes hold the same values in both buffers
        BBX_CUDA(cudaMemcpyAsync(g->d_state[cur], g->d_state[oth], bytes, cudaMemcpyDeviceToDevice, g->stream));
    k_set_parity<<<1, 1, 0, g->stream>>>(g->d_dyn, oth);
    BBX_CUDA(cudaGetLastError());
    g->h_cur = oth;
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    return check_sticky(g);
}

int bbx_exchange_state_async(bbx_grid* g, const float* host_in, float* host_out, size_t n) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (!host_in || !host_out || n != (size_t)g->S * (size_t)g->ncell) return BBX_ERR_ARG;
    if (g->px != g->nx || g->gates != GATES_F32) return BBX_ERR_UNSUPPORTED;
    const size_t bytes = sizeof(float) * n;
    if (g->x_bytes != bytes) {  // first use, or a model with another number of variables
        exchange_release(g);
        bool ok = cudaStreamCreateWithFlags(&g->xs_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&g->xs_out, cudaStreamNonBlocking) == cudaSuccess;
        for (int j = 0; j < 2 && ok; ++j)
            ok = cudaEventCreateWithFlags(&g->xev_in_ready[j], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&g->xev_in_used[j], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&g->xev_out_ready[j], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&g->xev_out_done[j], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            exchange_release(g);
            return BBX_ERR_CUDA;
        }
        for (int j = 0; j < 2 && ok; ++j)
            ok = dmalloc(&g->d_xin[j], bytes) == cudaSuccess && dmalloc(&g->d_xout[j], bytes) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            exchange_release(g);
            return BBX_ERR_NOMEM;
        }
        g->x_bytes = bytes;
        g->x_issued = 0;
    }
    const int j = (int)(g->x_issued & 1);
    const bool reuse = g->x_issued >= 2;  // stage j was used two exchanges ago
    const int cur = g->h_cur;
    // the current state into output stage j (once that stage's previous copy to
    // the host is done), then to the host on the output stream
    const long long n4 = (long long)(bytes / 16);  // vol is a multiple of 32 floats (rows padded to 32)
    const int cb = g->num_sms * 4;
    if (reuse) BBX_CUDA(cudaStreamWaitEvent(g->stream, g->xev_out_done[j], 0));
    k_copy4<<<cb, 256, 0, g->stream>>>(reinterpret_cast<float4*>(g->d_xout[j]), nullptr,
                                       reinterpret_cast<const float4*>(g->d_state[cur]), n4);
    BBX_CUDA(cudaGetLastError());
    BBX_CUDA(cudaEventRecord(g->xev_out_ready[j], g->stream));
    BBX_CUDA(cudaStreamWaitEvent(g->xs_out, g->xev_out_ready[j], 0));
    BBX_CUDA(cudaMemcpyAsync(host_out, g->d_xout[j], bytes, cudaMemcpyDeviceToHost, g->xs_out));
    BBX_CUDA(cudaEventRecord(g->xev_out_done[j], g->xs_out));
    // the new state into input stage j on the input stream (once the grid's
    // stream has taken what the stage held before), then into the state
    if (reuse) BBX_CUDA(cudaStreamWaitEvent(g->xs_in, g->xev_in_used[j], 0));
    BBX_CUDA(cudaMemcpyAsync(g->d_xin[j], host_in, bytes, cudaMemcpyHostToDevice, g->xs_in));
    BBX_CUDA(cudaEventRecord(g->xev_in_ready[j], g->xs_in));
    BBX_CUDA(cudaStreamWaitEvent(g->stream, g->xev_in_ready[j], 0));
    // (void nodes hold the same values in both buffers of a masked grid)
    k_copy4<<<cb, 256, 0, g->stream>>>(reinterpret_cast<float4*>(g->d_state[cur]),
                                       g->d_mask ? reinterpret_cast<float4*>(g->d_state[cur ^ 1]) : nullptr,
                                       reinterpret_cast<const float4*>(g->d_xin[j]), n4);
    BBX_CUDA(cudaGetLastError());
    BBX_CUDA(cudaEventRecord(g->xev_in_used[j], g->stream));
    ++g->x_issued;
    return BBX_OK;
}

int bbx_exchange_wait(bbx_grid* g) {
    if (!g) return BBX_ERR_ARG;
    if (!g->xs_in) return BBX_OK;
    const cudaError_t a = cudaStreamSynchronize(g->xs_out);
    const cudaError_t b = cudaStreamSynchronize(g->xs_in);
    if (a != cudaSuccess) return fail_cuda(a);
    if (b != cudaSuccess) return fail_cuda(b);
    return BBX_OK;
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
    if (var_is16(g, var)) return BBX_ERR_UNSUPPORTED;
    TissueDyn d;
    int rc = read_dyn(g, &d);
    if (rc) return rc;
    int blocks = g->num_sms * 4;
    if (blocks > kMaxPartials) blocks = kMaxPartials;
    const long long z0 = g->halo_lo;  // a z-slab sums its own planes, not its halo planes
    k_total<<<blocks, 256, 0, g->stream>>>(g->d_state[d.cur] + (size_t)var * g->vol + z0 * g->plane,
                                           g->d_mask ? g->d_mask + z0 * g->plane : nullptr, g->nx, g->ny,
                                           g->nz - g->halo_lo - g->halo_hi, g->px, g->plane, g->d_partials,
                                           g->d_ticket, g->d_total2, g->d_err);
    BBX_CUDA(cudaGetLastError());
    BBX_CUDA(cudaMemcpyAsync(out, g->d_total2, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    return check_sticky(g);
}

int bbx_ppm_frame(bbx_grid* g, const int* layers, const double* lo, const double* hi, uint8_t* out_dev) {
    if (!g || !layers || !lo || !hi || !out_dev) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    int ly[3];
    float l[3], h[3];
    for (int c = 0; c < 3; ++c) {
        ly[c] = layers[c];
        l[c] = (float)lo[c];
        h[c] = (float)hi[c];
        if (ly[c] < -1 || ly[c] >= g->S) return BBX_ERR_ARG;
        if (ly[c] >= 0 && !(std::isfinite(l[c]) && std::isfinite(h[c]) && h[c] != l[c])) return BBX_ERR_ARG;
        if (ly[c] >= 0 && var_is16(g, ly[c])) return BBX_ERR_UNSUPPORTED;  // 16-bit gate layers
    }
    BBX_CUDA(launch_ppm(g->d_state[0], g->d_state[1], &g->d_dyn->cur, g->d_mask, g->vol, g->nx, g->ny, g->nz, g->px,
                        g->plane, ly, l, h, out_dev, g->num_sms, g->stream));
    return BBX_OK;
}

int bbx_phase_singularities(bbx_grid* g, int var_a, double iso_a, int var_b, double iso_b, float* xyz_dev,
                            int max_points, int* n_found) {
    if (!g || !n_found || max_points < 0 || (max_points > 0 && !xyz_dev)) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (var_a < 0 || var_a >= g->S || var_b < 0 || var_b >= g->S || !std::isfinite(iso_a) || !std::isfinite(iso_b))
        return BBX_ERR_ARG;
    if (var_is16(g, var_a) || var_is16(g, var_b)) return BBX_ERR_UNSUPPORTED;
    if (!g->d_count && dmalloc(&g->d_count, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_NOMEM;
    }
    BBX_CUDA(launch_singz(g->d_state[0], g->d_state[1], &g->d_dyn->cur, (long long)var_a * g->vol,
                          (long long)var_b * g->vol, (float)iso_a, (float)iso_b, g->d_mask, g->nx, g->ny, g->nz, g->px,
                          g->plane, xyz_dev, max_points, g->d_count, g->num_sms, g->stream));
    return read_word_and_sticky(g, g->d_count, n_found);
}

int bbx_step_total(bbx_grid* g, double* out) {
    if (!g || !out) return BBX_ERR_ARG;
    if (!g->stepped) return BBX_ERR_STATE;
    int rc = finish_total(g);
    if (rc) return rc;
    TissueDyn d;
    if ((rc = read_dyn(g, &d))) return rc;
    *out = d.total;
    return check_sticky(g);
}

int bbx_get_time(bbx_grid* g, double* t, long long* step) {
    if (!g) return BBX_ERR_ARG;
    TissueDyn d;
    int rc = read_dyn(g, &d);
    if (rc) return rc;
    if (t) *t = d.t;
    if (step) *step = d.n;
    return BBX_OK;
}

int bbx_set_time(bbx_grid* g, double t, long long step) {
    if (!g || !std::isfinite(t) || step < 0 || step >= 0x7fffffffLL) return BBX_ERR_ARG;
    TissueDyn d;
    int rc = read_dyn(g, &d);
    if (rc) return rc;
    d.t = t;
    d.n = step;
    return write_dyn(g, d);
}

int bbx_get_info(bbx_grid* g, bbx_info* o) {
    if (!g || !o) return BBX_ERR_ARG;
    TissueDyn d;
    memset(&d, 0, sizeof(d));
    int rc = read_dyn(g, &d);
    if (rc) return rc;
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
    long long owned = 0;  // tissue nodes the step computes (a z-slab's halo planes excluded)
    for (int z = g->halo_lo; z < g->nz - g->halo_hi; ++z) owned += g->plane_tissue[(size_t)z];
    o->n_tissue = owned;
    o->step = d.n;
    o->t = d.t;
    o->wsum_skipped = (g->aniso && g->wsum_zero && g->wsum_elide) ? 1 : 0;
    return BBX_OK;
}

int bbx_read_active_bricks(bbx_grid* g, int32_t* out, size_t cap, long long* count) {
    if (!g || !count) return BBX_ERR_ARG;
    *count = g->n_bricks;
    if ((size_t)g->n_bricks > cap || (!out && g->n_bricks > 0)) return BBX_ERR_ARG;
    if (g->d_mask) {
        for (long long i = 0; i < g->n_bricks; ++i) out[i] = g->h_bricks[(size_t)i];
    } else {
        for (long long i = 0; i < g->n_bricks; ++i) out[i] = (int32_t)i;
    }
    return BBX_OK;
}

int bbx_set_tiling(bbx_grid* g, int tile_y, int tile_z) {
    if (!g || (tile_y != 7 && tile_y != 14 && tile_y != 28) || tile_z < 1) return BBX_ERR_ARG;
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
    TissueDyn d;
    int rc = read_dyn(g, &d);
    if (rc) return rc;
    *p = var_is16(g, var) ? (void*)gate_plane(g, d.cur, var) : (void*)(g->d_state[d.cur] + (size_t)var * g->vol);
    return BBX_OK;
}

int bbx_set_gate_storage(bbx_grid* g, int mode) {
    if (!g || (mode != BBX_GATES_FP32 && mode != BBX_GATES_FP16 && mode != BBX_GATES_UNORM16)) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (mode == g->gates) return BBX_OK;
    if (g->model != BBX_BR || (mode != BBX_GATES_FP32 && g->surr_on)) return BBX_ERR_UNSUPPORTED;
    if (mode != BBX_GATES_FP32 && g->ty == 28) {  // 16-bit kernels have 7- and 14-row tiles
        g->ty = 14;
        int rc0 = build_bricks(g);
        if (rc0) return rc0;
    }
    // the current state through the host, in the new layout
    std::vector<float> host((size_t)g->S * g->ncell);
    int rc = bbx_read_all(g, host.data(), host.size());
    if (rc) return rc;
    const int old = g->gates;
    const size_t need = (size_t)(mode != BBX_GATES_FP32 ? 5 : g->S) * g->vol;
    if (g->bound && sizeof(float) * need > g->bound_bytes) return BBX_ERR_STATE;  // the caller's buffers are too small
    if (!g->bound) {
        float* nb[2] = {nullptr, nullptr};
        if (dmalloc(&nb[0], sizeof(float) * need) != cudaSuccess ||
            dmalloc(&nb[1], sizeof(float) * need) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(nb[0]);
            return BBX_ERR_NOMEM;
        }
        cudaStreamSynchronize(g->stream);
        cudaFree(g->d_state[0]);
        cudaFree(g->d_state[1]);
        g->d_state[0] = nb[0];
        g->d_state[1] = nb[1];
    }
    g->gates = mode;
    // every node (void ones included) to rest in the new layout, then the state
    for (int k = 0; k < 2; ++k) {
        if (mode != BBX_GATES_FP32)
            k_fill_state16<<<n_blocks_for(g->vol, 256), 256, 0, g->stream>>>(g->d_state[k], g->vol, g->d_rest, mode);
        else
            k_fill_state<<<n_blocks_for((long long)g->S * g->vol, 256), 256, 0, g->stream>>>(g->d_state[k], g->S,
                                                                                                g->vol, g->d_rest);
    }
    BBX_CUDA(cudaGetLastError());
    TissueDyn d;
    if ((rc = read_dyn(g, &d))) return rc;
    d.cur = 0;
    if ((rc = write_dyn(g, d))) return rc;
    g->ready = false;
    if ((rc = prepare(g))) {
        (void)old;
        return rc;
    }
    return bbx_write_all(g, host.data(), host.size());
}

int bbx_set_halo_planes(bbx_grid* g, int lo, int hi) {
    if (!g || lo < 0 || lo > 1 || hi < 0 || hi > 1) return BBX_ERR_ARG;
    if ((lo || hi) && (g->nz < 2 || g->nz <= lo + hi)) return BBX_ERR_ARG;
    if (lo == g->halo_lo && hi == g->halo_hi) return BBX_OK;
    if (g->model) {
        int rc = finish_total(g);  // the plan's partials are about to be replaced
        if (rc) return rc;
    }
    g->halo_lo = lo;
    g->halo_hi = hi;
    g->ready = false;
    return g->model ? prepare(g) : BBX_OK;
}

int bbx_halo_plane(bbx_grid* g, int side, int halo, void** dev_ptr, size_t* bytes) {
    if (!g || !dev_ptr || (side != 0 && side != 1) || (halo != 0 && halo != 1)) return BBX_ERR_ARG;
    if (!g->model || !g->d_state[0]) return BBX_ERR_STATE;
    const int has = side == 0 ? g->halo_lo : g->halo_hi;
    if (!has) return BBX_ERR_STATE;  // no halo plane on that side
    int z;
    if (side == 0) z = halo ? 0 : 1;
    else z = halo ? g->nz - 1 : g->nz - 2;
    *dev_ptr = g->d_state[g->h_cur] + (size_t)z * g->plane;  // V of the buffer the next step reads
    if (bytes) *bytes = (size_t)g->plane * sizeof(float);
    return BBX_OK;
}

int bbx_halo_exchange(bbx_grid* lower, bbx_grid* upper) {
    if (!lower || !upper || lower == upper) return BBX_ERR_ARG;
    if (!lower->model || !upper->model) return BBX_ERR_STATE;
    if (!lower->halo_hi || !upper->halo_lo) return BBX_ERR_STATE;
    if (lower->nx != upper->nx || lower->ny != upper->ny || lower->device != upper->device) return BBX_ERR_ARG;
    const size_t bytes = (size_t)lower->plane * sizeof(float);
    float* lo_send = lower->d_state[lower->h_cur] + (size_t)(lower->nz - 2) * lower->plane;
    float* lo_recv = lower->d_state[lower->h_cur] + (size_t)(lower->nz - 1) * lower->plane;
    float* up_send = upper->d_state[upper->h_cur] + (size_t)1 * upper->plane;
    float* up_recv = upper->d_state[upper->h_cur];
    const bool two = lower->stream != upper->stream;
    if (two) {
        // the copies run on the lower grid's stream after the upper grid's
        // enqueued work, and the upper grid's later work waits for them
        if (!upper->ev_halo) BBX_CUDA(cudaEventCreateWithFlags(&upper->ev_halo, cudaEventDisableTiming));
        if (!lower->ev_halo) BBX_CUDA(cudaEventCreateWithFlags(&lower->ev_halo, cudaEventDisableTiming));
        BBX_CUDA(cudaEventRecord(upper->ev_halo, upper->stream));
        BBX_CUDA(cudaStreamWaitEvent(lower->stream, upper->ev_halo, 0));
    }
    BBX_CUDA(cudaMemcpyAsync(up_recv, lo_send, bytes, cudaMemcpyDeviceToDevice, lower->stream));
    BBX_CUDA(cudaMemcpyAsync(lo_recv, up_send, bytes, cudaMemcpyDeviceToDevice, lower->stream));
    if (two) {
        BBX_CUDA(cudaEventRecord(lower->ev_halo, lower->stream));
        BBX_CUDA(cudaStreamWaitEvent(upper->stream, lower->ev_halo, 0));
    }
    return BBX_OK;
}

int bbx_autotune(bbx_grid* g, double dt, double* best_ms) {
    if (!g) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    int rc = set_dt(g, dt);
    if (rc) return rc;
    // save the state so the trial steps leave no trace
    const size_t sbytes = sizeof(float) * state_words(g);
    float* save = nullptr;
    int32_t* save_act = nullptr;
    if (dmalloc(&save, sbytes) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_NOMEM;
        }
    if (dmalloc(&save_act, sizeof(int32_t) * g->vol) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(save);
        return BBX_ERR_NOMEM;
    }
    TissueDyn d0;
    if ((rc = finish_total(g)) || (rc = read_dyn(g, &d0))) {
        cudaFree(save);
        cudaFree(save_act);
        return rc;
    }
    BBX_CUDA(cudaMemcpyAsync(save, g->d_state[d0.cur], sbytes, cudaMemcpyDeviceToDevice, g->stream));
    BBX_CUDA(cudaMemcpyAsync(save_act, g->d_act, sizeof(int32_t) * g->vol, cudaMemcpyDeviceToDevice, g->stream));
    const bool stepped0 = g->stepped;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int tys[3] = {7, 14, 28};
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
    rc = BBX_OK;
    for (int ty : tys) {
        for (int zb : zbs) {
            if ((rc = bbx_set_tiling(g, ty, zb)) != BBX_OK) {
                if (rc == BBX_ERR_UNSUPPORTED) {
                    rc = BBX_OK;
                    continue;
                }
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
    cudaMemcpyAsync(g->d_state[0], save, sbytes, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(g->d_state[1], save, sbytes, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(g->d_act, save_act, sizeof(int32_t) * g->vol, cudaMemcpyDeviceToDevice, g->stream);
    cudaStreamSynchronize(g->stream);
    cudaFree(save);
    cudaFree(save_act);
    d0.cur = 0;
    int rc3 = write_dyn(g, d0);
    g->stepped = stepped0;
    if (best_ms) *best_ms = best;
    if (rc) return rc;
    if (rc2) return rc2;
    if (rc3) return rc3;
    return check_sticky(g);
}

}  // extern "C"

extern "C" int bbx_set_surrogate(bbx_grid* g, const bbx_mlp* m, double v_upstroke) {
    if (!g || !std::isfinite(v_upstroke)) return BBX_ERR_ARG;
    if (!m) {
        g->surr_on = false;
        return g->model ? prepare(g) : BBX_OK;
    }
    if (!g->model) return BBX_ERR_STATE;
    if (g->model != BBX_BR || g->gates != GATES_F32) return BBX_ERR_UNSUPPORTED;
    if (!g->d_surr && dmalloc(&g->d_surr, sizeof(SurrogateData)) != cudaSuccess) {
        cudaGetLastError();
        return BBX_ERR_NOMEM;
    }
    k_build_surrogate<<<(64 * 32 + 255) / 256, 256, 0, g->stream>>>(bbx_mlp_device_params(m), bbx_mlp_device_norm(m),
                                                                    (float)v_upstroke, g->d_surr);
    BBX_CUDA(cudaGetLastError());
    BBX_CUDA(cudaStreamSynchronize(g->stream));
    const bool was = g->surr_on;
    g->surr_on = true;
    int rc = prepare(g);
    if (rc) {
        g->surr_on = was;
        prepare(g);
    }
    return rc;
}

extern "C" int bbx_sample_reaction_pairs(bbx_grid* g, long long n, unsigned long long seed, float* x_dev,
                                         float* t_dev) {
    if (!g || n <= 0 || !x_dev || !t_dev) return BBX_ERR_ARG;
    if (!g->model) return BBX_ERR_STATE;
    if (g->model != BBX_BR || g->gates != GATES_F32) return BBX_ERR_UNSUPPORTED;
    if (!(g->dt > 0.0)) return BBX_ERR_STATE;
    if (g->n_tissue == 0) return BBX_ERR_ARG;
    if (!g->ready) {
        int rc = prepare(g);
        if (rc) return rc;
    }
    k_sample_pairs_br<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(g->d_t, g->d_mask, n, seed, x_dev, t_dev);
    BBX_CUDA(cudaGetLastError());
    return BBX_OK;
}

// ---------------------------------------------------------------------------
// batches of independent grids
// ---------------------------------------------------------------------------

struct bbx_batch {
    struct Group {
        int model = 0;
        bool masked = false, aniso = false, surr = false, planar = false, general = false;
        int ty = 14;
        std::vector<int> members;  // indices into grids
        TissueArgs* d_t = nullptr;  // one TissueArgs per member (tensor maps for this group's ty)
        LaunchPlan lp;
        cudaStream_t s = nullptr;
        cudaEvent_t done = nullptr;
        long long work = 0;
    };
    std::vector<bbx_grid*> grids;
    std::vector<unsigned long long> versions;
    cudaStream_t stream = nullptr;  // the members' stream (may be the legacy default stream)
    cudaStream_t ps = nullptr;      // the batch's own stream: graph capture and launches
    cudaEvent_t enter = nullptr, leave = nullptr;
    int device = 0, num_sms = 0;
    std::vector<Group> groups;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_steps = 0;
    int* d_err = nullptr;
    bool built = false;
};

namespace {

void batch_release_groups(bbx_batch* b) {
    for (auto& gr : b->groups) {
        cudaFree(gr.d_t);
        gr.lp.release();
        if (gr.s) cudaStreamDestroy(gr.s);
        if (gr.done) cudaEventDestroy(gr.done);
    }
    b->groups.clear();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->graph_steps = 0;
    b->built = false;
}

// Group the grids by kernel type; give each group a share of the GPU's
// resident CTAs proportional to its column-planes, so that all groups of a
// step run side by side and finish together.
int batch_build(bbx_batch* b, const std::vector<int>* tys) {
    cudaStreamSynchronize(b->stream);
    if (b->ps) cudaStreamSynchronize(b->ps);
    std::vector<int> keep_ty;
    for (auto& gr : b->groups) keep_ty.push_back(gr.ty);
    batch_release_groups(b);
    for (size_t i = 0; i < b->grids.size(); ++i) {
        bbx_grid* g = b->grids[i];
        size_t gi = 0;
        for (; gi < b->groups.size(); ++gi) {
            auto& gr = b->groups[gi];
            if (gr.model == g->model && gr.masked == (g->d_mask != nullptr) && gr.aniso == g->aniso &&
                gr.surr == (g->surr_on && g->model == BBX_BR) && gr.planar == (g->nz == 1) &&
                gr.general == wants_general(g))
                break;
        }
        if (gi == b->groups.size()) {
            bbx_batch::Group gr;
            gr.model = g->model;
            gr.masked = g->d_mask != nullptr;
            gr.aniso = g->aniso;
            gr.surr = g->surr_on && g->model == BBX_BR;
            gr.planar = g->nz == 1;
            gr.general = wants_general(g);
            b->groups.push_back(gr);
        }
        b->groups[gi].members.push_back((int)i);
    }
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        auto& gr = b->groups[gi];
        if (tys && gi < tys->size()) gr.ty = (*tys)[gi];
        else if (gi < keep_ty.size()) gr.ty = keep_ty[gi];
    }
    long long total_work = 0;
    std::vector<std::vector<Seg>> segs(b->groups.size());
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        auto& gr = b->groups[gi];
        std::vector<TissueArgs> ta(gr.members.size());
        for (size_t m = 0; m < gr.members.size(); ++m) {
            bbx_grid* g = b->grids[(size_t)gr.members[m]];
            // columns for this group's tile rows
            const int ty0 = g->ty;
            if (g->ty != gr.ty) {
                g->ty = gr.ty;
                int rc = build_bricks(g);
                if (rc) { g->ty = ty0; build_bricks(g); return rc; }
            }
            grid_segments(g, (int)m, &segs[gi]);
            int rc = encode_targs(g, gr.ty, &ta[m]);
            if (g->ty != ty0) {
                g->ty = ty0;
                build_bricks(g);
            }
            if (rc) return rc;
        }
        for (const Seg& sg : segs[gi]) gr.work += (long long)(sg.z1 - sg.z0);
        total_work += gr.work;
        if (dmalloc(&gr.d_t, sizeof(TissueArgs) * ta.size()) != cudaSuccess) {
            cudaGetLastError();
            return BBX_ERR_NOMEM;
        }
        BBX_CUDA(cudaMemcpy(gr.d_t, ta.data(), sizeof(TissueArgs) * ta.size(), cudaMemcpyHostToDevice));
        BBX_CUDA(cudaStreamCreateWithFlags(&gr.s, cudaStreamNonBlocking));
        BBX_CUDA(cudaEventCreateWithFlags(&gr.done, cudaEventDisableTiming));
    }
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        auto& gr = b->groups[gi];
        int ctas = 0;
        int rc = select_kernel(gr.model, gr.masked, gr.aniso ? AN_SUMS : AN_ISO, gr.ty, b->device, b->num_sms, &gr.lp.k, &ctas, gr.surr,
                               gr.planar, gr.general);
        if (rc) return rc;
        long long share = total_work > 0 ? (long long)((double)ctas * gr.work / total_work + 0.5) : 1;
        if (share < 1) share = 1;
        if ((rc = build_plan(&gr.lp, segs[gi], (int)gr.members.size(), (int)share))) return rc;
    }
    b->versions.clear();
    for (bbx_grid* g : b->grids) b->versions.push_back(g->version);
    b->built = true;
    return BBX_OK;
}

// One batch step of grids that hold no tissue (a group without pieces):
// nothing moves, time, step count and parity advance as for the others.
__global__ void k_advance_empty(const TissueArgs* __restrict__ T, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        TissueDyn* d = T[i].dyn;
        d->total = 0.0;
        d->t = d->t + T[i].dt_d;
        d->n = d->n + 1;
        d->cur = d->cur ^ 1;
        d->total_pending = 0;
    }
}

int batch_launch_step(bbx_batch* b) {
    BBX_CUDA(cudaEventRecord(b->fork, b->ps));
    for (auto& gr : b->groups) {
        if (gr.lp.n_planes == 0) {
            if (gr.members.empty()) continue;
            BBX_CUDA(cudaStreamWaitEvent(gr.s, b->fork, 0));
            k_advance_empty<<<1, 32, 0, gr.s>>>(gr.d_t, (int)gr.members.size());
            BBX_CUDA(cudaGetLastError());
            BBX_CUDA(cudaEventRecord(gr.done, gr.s));
            BBX_CUDA(cudaStreamWaitEvent(b->ps, gr.done, 0));
            continue;
        }
        BBX_CUDA(cudaStreamWaitEvent(gr.s, b->fork, 0));
        const LaunchArgs L = launch_args(gr.lp, gr.d_t, b->d_err, 0);
        BBX_CUDA(launch(gr.lp, L, gr.s));
        BBX_CUDA(cudaEventRecord(gr.done, gr.s));
        BBX_CUDA(cudaStreamWaitEvent(b->ps, gr.done, 0));
    }
    return BBX_OK;
}

int batch_capture(bbx_batch* b, int steps) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->graph_steps = 0;
    BBX_CUDA(cudaStreamBeginCapture(b->ps, cudaStreamCaptureModeThreadLocal));
    int rc = BBX_OK;
    for (int s = 0; s < steps && rc == BBX_OK; ++s) rc = batch_launch_step(b);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->ps, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail_cuda(e);
    b->graph = graph;
    BBX_CUDA(cudaGraphInstantiate(&b->gexec, graph, 0));
    b->graph_steps = steps;
    return BBX_OK;
}

}  // namespace

extern "C" {

int bbx_batch_create(bbx_batch** out, bbx_grid* const* grids, int n) {
    if (!out || !grids || n <= 0) return BBX_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!grids[i]) return BBX_ERR_ARG;
        if (!grids[i]->model || !(grids[i]->dt > 0.0)) return BBX_ERR_STATE;
        if (grids[i]->gates != GATES_F32) return BBX_ERR_UNSUPPORTED;  // 16-bit gates: stepped alone
        if (grids[i]->stream != grids[0]->stream || grids[i]->device != grids[0]->device) return BBX_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (grids[j] == grids[i]) return BBX_ERR_ARG;
    }
    bbx_batch* b = new (std::nothrow) bbx_batch();
    if (!b) return BBX_ERR_NOMEM;
    b->grids.assign(grids, grids + n);
    b->stream = grids[0]->stream;
    b->device = grids[0]->device;
    b->num_sms = grids[0]->num_sms;
    int rc = BBX_OK;
    if (cudaStreamCreateWithFlags(&b->ps, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->enter, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->leave, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        dmalloc(&b->d_err, sizeof(int)) != cudaSuccess || cudaMemset(b->d_err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        rc = BBX_ERR_CUDA;
    }
    if (rc == BBX_OK) rc = batch_build(b, nullptr);
    if (rc) {
        bbx_batch_destroy(b);
        return rc;
    }
    *out = b;
    return BBX_OK;
}

void bbx_batch_destroy(bbx_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->ps) cudaStreamSynchronize(b->ps);
    batch_release_groups(b);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->enter) cudaEventDestroy(b->enter);
    if (b->leave) cudaEventDestroy(b->leave);
    if (b->ps) cudaStreamDestroy(b->ps);
    cudaFree(b->d_err);
    cudaGetLastError();
    delete b;
}

int bbx_batch_step(bbx_batch* b, int n_steps) {
    if (!b || n_steps < 0) return BBX_ERR_ARG;
    if (n_steps == 0) return BBX_OK;
    for (size_t i = 0; i < b->grids.size(); ++i) {
        bbx_grid* g = b->grids[i];
        if (!g->model || !(g->dt > 0.0)) return BBX_ERR_STATE;
        if (g->version != b->versions[i]) b->built = false;  // a member changed since the batch was built
    }
    int rc;
    if (!b->built && (rc = batch_build(b, nullptr))) return rc;
    const int chunk = n_steps < 16 ? n_steps : 16;
    if (n_steps >= 2 && b->graph_steps != chunk && (rc = batch_capture(b, chunk))) return rc;
    // order the batch's stream after the members' stream, and back
    BBX_CUDA(cudaEventRecord(b->enter, b->stream));
    BBX_CUDA(cudaStreamWaitEvent(b->ps, b->enter, 0));
    int done = 0;
    if (n_steps >= 2) {
        for (; done + chunk <= n_steps; done += chunk) BBX_CUDA(cudaGraphLaunch(b->gexec, b->ps));
    }
    for (; done < n_steps; ++done)
        if ((rc = batch_launch_step(b))) return rc;
    BBX_CUDA(cudaEventRecord(b->leave, b->ps));
    BBX_CUDA(cudaStreamWaitEvent(b->stream, b->leave, 0));
    for (bbx_grid* g : b->grids) {
        g->stepped = true;
        g->h_cur ^= n_steps & 1;  // every batch step flips every member's parity
    }
    return BBX_OK;
}

int bbx_batch_sync(bbx_batch* b) {
    if (!b) return BBX_ERR_ARG;
    BBX_CUDA(cudaStreamSynchronize(b->ps));
    const int rc = check_sticky_ptr(b->stream, b->d_err);
    if (rc)  // a launch cut short (a timeout) may have left per-grid piece counts behind
        for (auto& gr : b->groups)
            if (gr.lp.d_tissue_done) cudaMemset(gr.lp.d_tissue_done, 0, sizeof(unsigned int) * gr.lp.n_tissues);
    return rc;
}

int bbx_batch_autotune(bbx_batch* b, double* best_ms) {
    if (!b) return BBX_ERR_ARG;
    int rc;
    if (!b->built && (rc = batch_build(b, nullptr))) return rc;
    // save every member so the trial steps leave no trace
    struct Saved {
        float* st;
        int32_t* act;
        TissueDyn dyn;
    };
    std::vector<Saved> saved;
    for (bbx_grid* g : b->grids) {
        Saved sv{nullptr, nullptr, {}};
        const size_t sbytes = sizeof(float) * g->S * (size_t)g->vol;
        if (read_dyn(g, &sv.dyn) || dmalloc(&sv.st, sbytes) != cudaSuccess ||
            dmalloc(&sv.act, sizeof(int32_t) * g->vol) != cudaSuccess) {
            cudaGetLastError();
            for (auto& s2 : saved) { cudaFree(s2.st); cudaFree(s2.act); }
            cudaFree(sv.st);
            return BBX_ERR_NOMEM;
        }
        cudaMemcpyAsync(sv.st, g->d_state[sv.dyn.cur], sbytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(sv.act, g->d_act, sizeof(int32_t) * g->vol, cudaMemcpyDeviceToDevice, b->stream);
        saved.push_back(sv);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<int> tys;
    for (auto& gr : b->groups) tys.push_back(gr.ty);
    double best_total = 0;
    rc = BBX_OK;
    // one group at a time, the others at their current shape
    for (size_t gi = 0; gi < tys.size() && rc == BBX_OK; ++gi) {
        double best = 1e30;
        int bty = tys[gi];
        for (int ty : {7, 14, 28}) {
            std::vector<int> trial = tys;
            trial[gi] = ty;
            int r = batch_build(b, &trial);
            if (r == BBX_ERR_UNSUPPORTED) continue;
            if (r) { rc = r; break; }
            cudaStreamSynchronize(b->stream);
            for (int s = 0; s < 2 && rc == BBX_OK; ++s) rc = batch_launch_step(b);
            cudaEventRecord(e0, b->ps);
            for (int s = 0; s < 4 && rc == BBX_OK; ++s) rc = batch_launch_step(b);
            cudaEventRecord(e1, b->ps);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / 4.0 < best) {
                best = ms / 4.0;
                bty = ty;
            }
        }
        tys[gi] = bty;
        best_total = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(b->ps);
    int rc2 = batch_build(b, &tys);
    for (size_t i = 0; i < b->grids.size(); ++i) {
        bbx_grid* g = b->grids[i];
        const size_t sbytes = sizeof(float) * g->S * (size_t)g->vol;
        cudaMemcpyAsync(g->d_state[0], saved[i].st, sbytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(g->d_state[1], saved[i].st, sbytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(g->d_act, saved[i].act, sizeof(int32_t) * g->vol, cudaMemcpyDeviceToDevice, b->stream);
        TissueDyn d = saved[i].dyn;
        d.cur = 0;
        cudaMemcpyAsync(g->d_dyn, &d, sizeof(TissueDyn), cudaMemcpyHostToDevice, b->stream);
        g->h_cur = 0;
        cudaStreamSynchronize(b->stream);
        cudaFree(saved[i].st);
        cudaFree(saved[i].act);
    }
    if (best_ms) *best_ms = best_total;
    if (rc) return rc;
    if (rc2) return rc2;
    return check_sticky_ptr(b->stream, b->d_err);
}

int bbx_batch_info(bbx_batch* b, int* n_groups, int* tile_y, int cap) {
    if (!b || !n_groups) return BBX_ERR_ARG;
    *n_groups = (int)b->groups.size();
    for (int i = 0; i < *n_groups && tile_y && i < cap; ++i) tile_y[i] = b->groups[(size_t)i].ty;
    return BBX_OK;
}

}  // extern "C"

// Host-only test hooks (no device work): the piece covering of a masked 3D
// grid and the CTA shares of a launch plan, as the library computes them.
extern "C" int bbx_debug_cover_chunks(const uint8_t* flags, int ncx, int nby, int nbz, int ty, int zb, int nz,
                                      int* out, int cap, int* count) {
    if (!flags || !count || ncx <= 0 || nby <= 0 || nbz <= 0 || ty <= 0 || zb <= 0 || nz <= 0 || cap < 0 ||
        (cap > 0 && !out))
        return BBX_ERR_ARG;
    std::vector<Seg> segs;
    cover_chunks(flags, ncx, nby, nbz, ty, zb, nz, 0, &segs);
    *count = (int)segs.size();
    if ((int)segs.size() > cap) return BBX_ERR_ARG;
    for (size_t i = 0; i < segs.size(); ++i) {
        out[4 * i] = segs[i].x0;
        out[4 * i + 1] = segs[i].y0;
        out[4 * i + 2] = segs[i].z0;
        out[4 * i + 3] = segs[i].z1;
    }
    return BBX_OK;
}

namespace {
// The step kernels' e^x - 1 next to CUDA's expm1f, for the accuracy test.
__global__ void k_debug_expm1(const float* __restrict__ x, float* __restrict__ y, float* __restrict__ ref, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        y[i] = expm1_br(x[i]);
        ref[i] = expm1f(x[i]);
    }
}
}  // namespace

extern "C" int bbx_debug_expm1(const float* x_dev, float* out_dev, float* ref_dev, int n, void* cuda_stream) {
    if (!x_dev || !out_dev || !ref_dev || n <= 0) return BBX_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_debug_expm1<<<n_blocks_for(n, 256), 256, 0, s>>>(x_dev, out_dev, ref_dev, n);
    BBX_CUDA(cudaGetLastError());
    BBX_CUDA(cudaStreamSynchronize(s));
    return BBX_OK;
}

extern "C" int bbx_debug_plan_first_pieces(const int* segs4, int nsegs, int ctas, int* out, int cap, int* used) {
    if (!segs4 || nsegs <= 0 || ctas <= 0 || !out || !used) return BBX_ERR_ARG;
    std::vector<Seg> segs((size_t)nsegs);
    for (int i = 0; i < nsegs; ++i)
        segs[(size_t)i] = {0, segs4[4 * i], segs4[4 * i + 1], segs4[4 * i + 2], segs4[4 * i + 3]};
    std::vector<std::vector<int4>> per;
    std::vector<std::vector<int>> per_t;
    int stride = 1;
    const int n = plan_shares(segs, ctas, &per, &per_t, &stride);
    *used = n;
    if (n > cap) return BBX_ERR_ARG;
    for (int c = 0; c < n; ++c) {
        const int4 p = per[(size_t)c].empty() ? make_int4(0, 0, 0, 0) : per[(size_t)c][0];
        out[4 * c] = p.x;
        out[4 * c + 1] = p.y;
        out[4 * c + 2] = p.z;
        out[4 * c + 3] = p.w;
    }
    return BBX_OK;
}
