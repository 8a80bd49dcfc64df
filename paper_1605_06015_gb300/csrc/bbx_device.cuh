// Device-side building blocks of the sm_103a monodomain step: TMA/mbarrier
// wrappers (inline PTX), the cell models, and the fused step kernel template.
//
// The step kernel is one pass of the paper's unsplit scheme (section
// "Computation of intermediate expressions": diff followed by euler /
// rushlarsen) for every tissue node of a brick list:
//   - 2.5D z-marching over bricks of 64 x TY x ZB nodes; each z-plane of V
//     (with a one-node halo, widened in x to the 16-byte TMA rule), of the
//     fibres (with halo), of the tissue mask (with halo) and of the
//     non-diffusing variables is staged into shared memory by
//     cp.async.bulk.tensor on an mbarrier ring of NS planes, loads running up
//     to NS-3 planes ahead of the plane being computed;
//   - the weights W = Wbar + Wtilde of Eq. (Lu) are rebuilt per node from the
//     unit fibre vectors of the node and of its six face neighbours, Eq.
//     (sigma); nothing per-weight is stored in HBM;
//   - the reaction update (Eq. (Euler) for V and non-gates, Eq. (RL) for
//     gates) is fused, the new state is stored straight from registers;
//   - the activation map is written on the first upward crossing only;
//   - the sum of the new V over tissue nodes is reduced in the same pass
//     (compensated float pairs per thread and warp, double across warps and
//     CTAs, deterministic last-CTA finalisation).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bbx.h"

namespace bbx {

// ---------------------------------------------------------------------------
// launch arguments
// ---------------------------------------------------------------------------

enum : int { ERRBIT_TIMEOUT = 1, ERRBIT_NAN = 2 };

struct StepArgs {
    int nx, ny, nz, px;
    long long plane;  // px * ny
    long long vol;    // px * ny * nz
    int nbx, nby, zb;
    const int* bricks;  // active brick ids, or nullptr = all bricks in order
    int n_bricks;
    float* dst;  // destination state buffer (var v at dst + v*vol)
    int32_t* act;
    float theta;
    int step_next;  // n+1 for this step
    const uint8_t* stim;
    float stim_amp;  // 0: stimulus off for this step
    float dt, inv_h2;
    float Dperp, dD, Diso;  // anisotropic: D = Dperp I + dD f f^T; isotropic: Diso I
    float mp[8];            // model parameters (already in kernel form)
    double* partials;       // >= gridDim.x doubles
    unsigned int* ticket;   // zero between launches
    double* total_out;      // tissue sum of the new V
    int* err;               // sticky error bits
    long long wait_limit;   // clock64 cycles a wait may spin before giving up
    int poison_first_load;  // fault injection: CTA 0's first plane never completes
};

// ---------------------------------------------------------------------------
// PTX wrappers: shared-memory barriers and tensor-map bulk copies
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the barrier phase with the given parity; gives up (returns false)
// after `limit` SM clock cycles instead of spinning forever.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------------------
// compensated float accumulation (Knuth's TwoSum) for the V reduction
// ---------------------------------------------------------------------------

struct F2 {
    float hi, lo;
};

__device__ __forceinline__ void two_sum_add(F2& a, float b) {
    float s = a.hi + b;
    float bb = s - a.hi;
    float err = (a.hi - (s - bb)) + (b - bb);
    a.hi = s;
    a.lo += err;
}

// Sum a per-thread double over the block (any blockDim that is a multiple of
// 32, at most 1024); result valid in thread 0.
__device__ __forceinline__ double block_sum_double(double v, double* scratch32) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) scratch32[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) s += scratch32[w];
    }
    return s;
}

// Per-CTA partial -> deterministic grid total by the last CTA to finish.
__device__ __forceinline__ void grid_total_finalize(double block_partial, double* partials,
                                                    unsigned int* ticket, double* out, int* err,
                                                    bool flag_nonfinite) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = block_partial;
        if (flag_nonfinite && !isfinite(block_partial)) atomicOr(err, ERRBIT_NAN);
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned int b = 0; b < gridDim.x; ++b) s += ((volatile double*)partials)[b];
        *out = s;
        *ticket = 0u;
    }
}

// ---------------------------------------------------------------------------
// cell models (kernel form of the parameters is prepared on the host)
// ---------------------------------------------------------------------------

template <int MODEL>
struct Model;

// FitzHugh-Nagumo, Eq. (FHN) with the cubic: mp = {1/eps, eps, beta, gamma}.
template <>
struct Model<BBX_FHN> {
    static constexpr int S = 2;
    __device__ static __forceinline__ void update(const float* mp, float* y, float L, float Is, float dt) {
        const float u = y[0], v = y[1];
        const float du = (u - u * u * u * (1.0f / 3.0f) - v) * mp[0] + L + Is;
        const float dv = mp[1] * (u + mp[2] - mp[3] * v);
        y[0] = u + dt * du;
        y[1] = v + dt * dv;
    }
};

// Barkley (1991): mp = {1/a, b, 1/eps}.
template <>
struct Model<BBX_BARKLEY> {
    static constexpr int S = 2;
    __device__ static __forceinline__ void update(const float* mp, float* y, float L, float Is, float dt) {
        const float u = y[0], v = y[1];
        const float du = u * (1.0f - u) * (u - (v + mp[1]) * mp[0]) * mp[2] + L + Is;
        y[0] = u + dt * du;
        y[1] = v + dt * (u - v);
    }
};

// ZFK / Nagumo reaction of Eq. (ZFKbidomV): mp = {alpha}.
template <>
struct Model<BBX_ZFK> {
    static constexpr int S = 1;
    __device__ static __forceinline__ void update(const float* mp, float* y, float L, float Is, float dt) {
        const float u = y[0];
        y[0] = u + dt * (u * (u - mp[0]) * (1.0f - u) + L + Is);
    }
};

// Diffusion equation alone.
template <>
struct Model<BBX_DIFFUSION> {
    static constexpr int S = 1;
    __device__ static __forceinline__ void update(const float*, float* y, float L, float Is, float dt) {
        y[0] = y[0] + dt * (L + Is);
    }
};

// Beeler-Reuter (1977).  State (V, Ca, x1, m, h, j, d, f); mp = {gNa, gNaC,
// ENa, gs}.  V in mV, t in ms, Ca in mol/L, currents in uA/cm^2, Cm = 1.
// Rate constants of the 1977 publication, written out per gate.
__device__ __forceinline__ float br_ratio(float num, float den) { return __fdividef(num, den); }

template <>
struct Model<BBX_BR> {
    static constexpr int S = 8;

    // One Rush-Larsen gate step, Eq. (RL) read as y' = A y + B, in the
    // algebraically equal form y' = y + (1 - A)(y_inf - y), with 1 - A taken
    // by expm1f (no cancellation when (alpha+beta) dt is small).
    __device__ static __forceinline__ float rl(float y, float al, float be, float dt) {
        const float s = al + be;
        const float one_minus_A = -expm1f(-s * dt);
        return y + one_minus_A * (__fdividef(al, s) - y);
    }

    __device__ static __forceinline__ void update(const float* mp, float* y, float L, float Is, float dt) {
        const float V = y[0], Ca = y[1];
        const float x1 = y[2], m = y[3], h = y[4], j = y[5], d = y[6], f = y[7];

        // membrane currents
        const float INa = (mp[0] * m * m * m * h * j + mp[1]) * (V - mp[2]);
        const float Es = -82.3f - 13.0287f * __logf(Ca);
        const float Is_ = mp[3] * d * f * (V - Es);
        const float Ix1 = x1 * 0.8f * (__expf(0.04f * (V + 77.0f)) - 1.0f) * __expf(-0.04f * (V + 35.0f));
        const float w = V + 23.0f;
        const float lin = (w == 0.0f) ? 5.0f : br_ratio(0.2f * w, -expm1f(-0.04f * w));
        const float IK1 = 0.35f * (br_ratio(4.0f * (__expf(0.04f * (V + 85.0f)) - 1.0f),
                                            __expf(0.08f * (V + 53.0f)) + __expf(0.04f * (V + 53.0f))) +
                                   lin);
        const float Iion = INa + Is_ + Ix1 + IK1;
        const float dCa = -1e-7f * Is_ + 0.07f * (1e-7f - Ca);

        // gate rates, 1/ms
        const float a_x1 = br_ratio(0.0005f * __expf(0.083f * (V + 50.0f)), __expf(0.057f * (V + 50.0f)) + 1.0f);
        const float b_x1 = br_ratio(0.0013f * __expf(-0.06f * (V + 20.0f)), __expf(-0.04f * (V + 20.0f)) + 1.0f);
        const float xm = V + 47.0f;
        const float a_m = (xm == 0.0f) ? 10.0f : br_ratio(-xm, expm1f(-0.1f * xm));
        const float b_m = 40.0f * __expf(-0.056f * (V + 72.0f));
        const float a_h = 0.126f * __expf(-0.25f * (V + 77.0f));
        const float b_h = br_ratio(1.7f, __expf(-0.082f * (V + 22.5f)) + 1.0f);
        const float a_j = br_ratio(0.055f * __expf(-0.25f * (V + 78.0f)), __expf(-0.2f * (V + 78.0f)) + 1.0f);
        const float b_j = br_ratio(0.3f, __expf(-0.1f * (V + 32.0f)) + 1.0f);
        const float a_d = br_ratio(0.095f * __expf(-0.01f * (V - 5.0f)), __expf(-0.072f * (V - 5.0f)) + 1.0f);
        const float b_d = br_ratio(0.07f * __expf(-0.017f * (V + 44.0f)), __expf(0.05f * (V + 44.0f)) + 1.0f);
        const float a_f = br_ratio(0.012f * __expf(-0.008f * (V + 28.0f)), __expf(0.15f * (V + 28.0f)) + 1.0f);
        const float b_f = br_ratio(0.0065f * __expf(-0.02f * (V + 30.0f)), __expf(-0.2f * (V + 30.0f)) + 1.0f);

        y[0] = V + dt * (-(Iion - Is) + L);  // Cm = 1
        y[1] = Ca + dt * dCa;
        y[2] = rl(x1, a_x1, b_x1, dt);
        y[3] = rl(m, a_m, b_m, dt);
        y[4] = rl(h, a_h, b_h, dt);
        y[5] = rl(j, a_j, b_j, dt);
        y[6] = rl(d, a_d, b_d, dt);
        y[7] = rl(f, a_f, b_f, dt);
    }
};

// ---------------------------------------------------------------------------
// shared-memory plan of the step kernel
// ---------------------------------------------------------------------------

constexpr int kTileX = 64;
constexpr int align128(int b) { return (b + 127) & ~127; }

template <int MODEL, bool MASKED, bool ANISO, int TY>
struct Plan {
    static constexpr int S = Model<MODEL>::S;
    static constexpr int TX = kTileX;
    static constexpr int UW = TX + 8;   // x from x0-4 to x0+TX+3 (16-byte aligned start)
    static constexpr int UH = TY + 2;   // y from y0-1 to y0+TY
    static constexpr int MW = TX + 32;  // mask bytes: x from x0-16 (16-byte aligned start)
    static constexpr int U_RAW = UW * UH * 4;
    static constexpr int F_RAW = ANISO ? 3 * UW * UH * 4 : 0;
    static constexpr int M_RAW = MASKED ? MW * UH : 0;
    static constexpr int S_RAW = (S > 1) ? (S - 1) * TX * TY * 4 : 0;
    static constexpr int U_OFF = 0;
    static constexpr int F_OFF = U_OFF + align128(U_RAW);
    static constexpr int M_OFF = F_OFF + align128(F_RAW);
    static constexpr int S_OFF = M_OFF + align128(M_RAW);
    static constexpr int STAGE = S_OFF + align128(S_RAW);
    static constexpr uint32_t TX_BYTES = U_RAW + F_RAW + M_RAW + S_RAW;
    static constexpr int NS_FIT = (200 * 1024) / STAGE;
    static constexpr int NS = NS_FIT > 6 ? 6 : (NS_FIT < 4 ? 4 : NS_FIT);
    static constexpr int SMEM = 128 + NS * STAGE + NS * 8;
    static constexpr int THREADS = TX * TY;
};

struct Brick {
    int x0, y0, z0, z1;
};

__device__ __forceinline__ Brick decode_brick(const StepArgs& a, int i) {
    const int id = a.bricks ? a.bricks[i] : i;
    const int bx = id % a.nbx;
    const int r = id / a.nbx;
    const int by = r % a.nby;
    const int bz = r / a.nby;
    Brick b;
    b.x0 = bx * kTileX;
    b.y0 = by;  // scaled by TY in the kernel
    b.z0 = bz * a.zb;
    b.z1 = min(b.z0 + a.zb, a.nz);
    return b;
}

// ---------------------------------------------------------------------------
// the fused step kernel
// ---------------------------------------------------------------------------

template <int MODEL, bool MASKED, bool ANISO, int TY>
__global__ void __launch_bounds__(kTileX * TY)
step_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_s,
            const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_m,
            const StepArgs a) {
    using P = Plan<MODEL, MASKED, ANISO, TY>;
    constexpr int S = P::S, TX = P::TX, UW = P::UW, MW = P::MW, NS = P::NS;

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NS * P::STAGE);
    __shared__ double red_scratch[32];

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
        prefetch_map(&tm_u);
        if (S > 1) prefetch_map(&tm_s);
        if (ANISO) prefetch_map(&tm_f);
        if (MASKED) prefetch_map(&tm_m);
    }
    __syncthreads();

    // ---- producer state (thread 0 only) ----
    int p_iter = 0, p_off = 0, issued = 0;
    auto issue_next = [&]() -> bool {
        const int bi = blockIdx.x + p_iter * gridDim.x;
        if (bi >= a.n_bricks) return false;
        Brick b = decode_brick(a, bi);
        const int y0 = b.y0 * TY;
        const int nload = b.z1 - b.z0 + 2;
        const int z = b.z0 - 1 + p_off;
        const int slot = issued % NS;
        uint64_t* bar = &bars[slot];
        unsigned char* st = smem + slot * P::STAGE;
        if (a.poison_first_load && blockIdx.x == 0 && issued == 0) {
            // fault injection: expect bytes that no copy will deliver
            mbar_arrive_expect_tx(bar, 16);
        } else if (z < 0 || z >= a.nz) {
            mbar_arrive(bar);  // plane outside the array: nothing to load
        } else {
            mbar_arrive_expect_tx(bar, P::TX_BYTES);
            tma_load_3d(st + P::U_OFF, &tm_u, b.x0 - 4, y0 - 1, z, bar);
            if (ANISO) tma_load_4d(st + P::F_OFF, &tm_f, b.x0 - 4, y0 - 1, z, 0, bar);
            if (MASKED) tma_load_3d(st + P::M_OFF, &tm_m, b.x0 - 16, y0 - 1, z, bar);
            if (S > 1) tma_load_4d(st + P::S_OFF, &tm_s, b.x0, y0, z, 1, bar);
        }
        ++issued;
        if (++p_off == nload) {
            p_off = 0;
            ++p_iter;
        }
        return true;
    };
    if (tid == 0) {
        while (issued < NS && issue_next()) {
        }
    }

    // ---- consumer ----
    F2 vsum = {0.0f, 0.0f};
    bool timed_out = false, abort = false;
    int jb = 0;  // load index of the first plane of the current brick
    const float theta = a.theta;

    for (int it = 0;; ++it) {
        const int bi = blockIdx.x + it * gridDim.x;
        if (bi >= a.n_bricks) break;
        const Brick b = decode_brick(a, bi);
        const int y0 = b.y0 * TY;
        const int x = b.x0 + tx, y = y0 + ty;
        const bool in_xy = (x < a.nx) && (y < a.ny);
        const int ncomp = b.z1 - b.z0;

        for (int w = 0; w < 2; ++w) {
            const int j = jb + w;
            if (!mbar_wait_bounded(&bars[j % NS], (j / NS) & 1, a.wait_limit)) timed_out = true;
        }
        for (int t = 0; t < ncomp; ++t) {
            {
                const int j = jb + t + 2;
                if (!mbar_wait_bounded(&bars[j % NS], (j / NS) & 1, a.wait_limit)) timed_out = true;
            }
            const int k = b.z0 + t;
            const unsigned char* stp = smem + ((jb + t) % NS) * P::STAGE;
            const unsigned char* stc = smem + ((jb + t + 1) % NS) * P::STAGE;
            const unsigned char* stn = smem + ((jb + t + 2) % NS) * P::STAGE;
            const float* Up = reinterpret_cast<const float*>(stp + P::U_OFF);
            const float* Uc = reinterpret_cast<const float*>(stc + P::U_OFF);
            const float* Un = reinterpret_cast<const float*>(stn + P::U_OFF);
            const int c = (ty + 1) * UW + (tx + 4);
            const bool zp_ok = k > 0, zn_ok = k + 1 < a.nz;

            // psi of the 18 neighbours
            bool ps_c, ps_xp, ps_xm, ps_yp, ps_ym, ps_zp, ps_zm;
            bool ps_pp, ps_mm, ps_pm, ps_mp;        // (x,y) edges in plane k
            bool ps_xpzp, ps_xmzm, ps_xpzm, ps_xmzp;  // (x,z) edges
            bool ps_ypzp, ps_ymzm, ps_ypzm, ps_ymzp;  // (y,z) edges
            if (MASKED) {
                const unsigned char* Mp = stp + P::M_OFF;
                const unsigned char* Mc = stc + P::M_OFF;
                const unsigned char* Mn = stn + P::M_OFF;
                const int m = (ty + 1) * MW + (tx + 16);
                ps_c = Mc[m] != 0;
                ps_xp = Mc[m + 1] != 0;
                ps_xm = Mc[m - 1] != 0;
                ps_yp = Mc[m + MW] != 0;
                ps_ym = Mc[m - MW] != 0;
                ps_zp = zn_ok && Mn[m] != 0;
                ps_zm = zp_ok && Mp[m] != 0;
                ps_pp = Mc[m + MW + 1] != 0;
                ps_mm = Mc[m - MW - 1] != 0;
                ps_pm = Mc[m - MW + 1] != 0;
                ps_mp = Mc[m + MW - 1] != 0;
                ps_xpzp = zn_ok && Mn[m + 1] != 0;
                ps_xmzm = zp_ok && Mp[m - 1] != 0;
                ps_xpzm = zp_ok && Mp[m + 1] != 0;
                ps_xmzp = zn_ok && Mn[m - 1] != 0;
                ps_ypzp = zn_ok && Mn[m + MW] != 0;
                ps_ymzm = zp_ok && Mp[m - MW] != 0;
                ps_ypzm = zp_ok && Mp[m + MW] != 0;
                ps_ymzp = zn_ok && Mn[m - MW] != 0;
            } else {
                const bool xp = x + 1 < a.nx, xm = x > 0, yp = y + 1 < a.ny, ym = y > 0;
                ps_c = true;
                ps_xp = xp; ps_xm = xm; ps_yp = yp; ps_ym = ym;
                ps_zp = zn_ok; ps_zm = zp_ok;
                ps_pp = xp && yp; ps_mm = xm && ym; ps_pm = xp && ym; ps_mp = xm && yp;
                ps_xpzp = xp && zn_ok; ps_xmzm = xm && zp_ok; ps_xpzm = xp && zp_ok; ps_xmzp = xm && zn_ok;
                ps_ypzp = yp && zn_ok; ps_ymzm = ym && zp_ok; ps_ypzm = yp && zp_ok; ps_ymzp = ym && zn_ok;
            }

            if (in_xy && ps_c) {
                const float up = Uc[c];
                auto dlt = [&](bool ps, float uq) { return ps ? (uq - up) : 0.0f; };
                const float e_xp = dlt(ps_xp, Uc[c + 1]), e_xm = dlt(ps_xm, Uc[c - 1]);
                const float e_yp = dlt(ps_yp, Uc[c + UW]), e_ym = dlt(ps_ym, Uc[c - UW]);
                const float e_zp = dlt(ps_zp, Un[c]), e_zm = dlt(ps_zm, Up[c]);
                float L;
                if (ANISO) {
                    const float* Fp = reinterpret_cast<const float*>(stp + P::F_OFF);
                    const float* Fc = reinterpret_cast<const float*>(stc + P::F_OFF);
                    const float* Fn = reinterpret_cast<const float*>(stn + P::F_OFF);
                    constexpr int FC = UW * P::UH;  // component stride
                    const float fx = Fc[c], fy = Fc[c + FC], fz = Fc[c + 2 * FC];
                    const float dD = a.dD, Dperp = a.Dperp;
                    const float Dxx = Dperp + dD * fx * fx, Dyy = Dperp + dD * fy * fy, Dzz = Dperp + dD * fz * fz;
                    const float Dxy = dD * fx * fy, Dxz = dD * fx * fz, Dyz = dD * fy * fz;
                    // S_k = sum_j (D^{p+q_j}_jk - D^{p-q_j}_jk); a void neighbour
                    // takes D^p.  The Dperp delta_jk parts cancel.
                    float Sx = 0.f, Sy = 0.f, Sz = 0.f;
                    auto acc_nb = [&](bool ps, const float* F, int off, int jdir, float sgn) {
                        float gx = fx, gy = fy, gz = fz;
                        if (ps) {
                            gx = F[off];
                            gy = F[off + FC];
                            gz = F[off + 2 * FC];
                        }
                        const float gj = (jdir == 0) ? gx : ((jdir == 1) ? gy : gz);
                        const float s = sgn * gj;
                        Sx += s * gx;
                        Sy += s * gy;
                        Sz += s * gz;
                    };
                    acc_nb(ps_xp, Fc, c + 1, 0, 1.f);
                    acc_nb(ps_xm, Fc, c - 1, 0, -1.f);
                    acc_nb(ps_yp, Fc, c + UW, 1, 1.f);
                    acc_nb(ps_ym, Fc, c - UW, 1, -1.f);
                    acc_nb(ps_zp, Fn, c, 2, 1.f);
                    acc_nb(ps_zm, Fp, c, 2, -1.f);
                    Sx *= dD; Sy *= dD; Sz *= dD;
                    const float faces = Dxx * (e_xp + e_xm) + Dyy * (e_yp + e_ym) + Dzz * (e_zp + e_zm);
                    const float divt = 0.25f * ((ps_xp && ps_xm ? Sx * (Uc[c + 1] - Uc[c - 1]) : 0.f) +
                                                (ps_yp && ps_ym ? Sy * (Uc[c + UW] - Uc[c - UW]) : 0.f) +
                                                (ps_zp && ps_zm ? Sz * (Un[c] - Up[c]) : 0.f));
                    const float exy = dlt(ps_pp, Uc[c + UW + 1]) + dlt(ps_mm, Uc[c - UW - 1]) -
                                      dlt(ps_pm, Uc[c - UW + 1]) - dlt(ps_mp, Uc[c + UW - 1]);
                    const float exz = dlt(ps_xpzp, Un[c + 1]) + dlt(ps_xmzm, Up[c - 1]) -
                                      dlt(ps_xpzm, Up[c + 1]) - dlt(ps_xmzp, Un[c - 1]);
                    const float eyz = dlt(ps_ypzp, Un[c + UW]) + dlt(ps_ymzm, Up[c - UW]) -
                                      dlt(ps_ypzm, Up[c + UW]) - dlt(ps_ymzp, Un[c - UW]);
                    const float edges = 0.5f * (Dxy * exy + Dxz * exz + Dyz * eyz);
                    L = a.inv_h2 * (faces + divt + edges);
                } else {
                    L = a.Diso * a.inv_h2 * ((e_xp + e_xm) + (e_yp + e_ym) + (e_zp + e_zm));
                }

                float yv[S];
                yv[0] = up;
                if (S > 1) {
                    const float* Sv = reinterpret_cast<const float*>(stc + P::S_OFF);
#pragma unroll
                    for (int v = 1; v < S; ++v) yv[v] = Sv[(v - 1) * TX * TY + ty * TX + tx];
                }
                const long long gi = (long long)k * a.plane + (long long)y * a.px + x;
                float Is = 0.0f;
                if (a.stim_amp != 0.0f && a.stim[gi]) Is = a.stim_amp;
                Model<MODEL>::update(a.mp, yv, L, Is, a.dt);
#pragma unroll
                for (int v = 0; v < S; ++v) a.dst[(long long)v * a.vol + gi] = yv[v];
                if (up < theta && theta <= yv[0]) {
                    if (a.act[gi] == BBX_ACT_NONE) a.act[gi] = a.step_next;
                }
                two_sum_add(vsum, yv[0]);
            }

            abort = __syncthreads_or(timed_out);
            if (abort) break;
            if (tid == 0) {
                const int freed = (t < ncomp - 1) ? (jb + t + 1) : (jb + ncomp + 2);
                while (issued < freed + NS && issue_next()) {
                }
            }
        }
        if (abort) break;
        jb += ncomp + 2;
    }

    if (abort && tid == 0) {
        // Give loads still in flight a bounded chance to land before exit.
        atomicOr(a.err, ERRBIT_TIMEOUT);
        for (int j = jb; j < issued; ++j) {
            if (a.poison_first_load && blockIdx.x == 0 && j == 0) continue;
            (void)mbar_wait_bounded(&bars[j % NS], (j / NS) & 1, a.wait_limit);
        }
    }

    const double mine = (double)vsum.hi + (double)vsum.lo;
    const double bs = block_sum_double(mine, red_scratch);
    grid_total_finalize(bs, a.partials, a.ticket, a.total_out, a.err, true);
}

// host-visible description of one compiled step kernel
typedef void (*StepFn)(CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, StepArgs);
struct StepKernel {
    const void* fn;
    int smem;
    int threads;
    int ty;
};

}  // namespace bbx
