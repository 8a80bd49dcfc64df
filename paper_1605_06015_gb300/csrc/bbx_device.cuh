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
//     (compensated float pairs per thread and warp, one double per piece;
//     the fixed-order sum of the pieces when the total is read, or at the
//     end of a batch launch).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/bbx.h"

namespace bbx {

// ---------------------------------------------------------------------------
// launch arguments
// ---------------------------------------------------------------------------

enum : int { ERRBIT_TIMEOUT = 1, ERRBIT_NAN = 2, ERRBIT_HINT = 4 };

// Device-updated state of one grid: written once per step, by the CTA that
// takes the last start ticket (single-grid launch) or by the last CTA to
// finish (batch launch), and by the on-demand sum of a pending total.
struct TissueDyn {
    double t;       // model time t_n
    double total;   // tissue sum of V after the most recent step
    long long n;    // steps taken
    int cur;        // buffer holding the current state (0 or 1)
    int total_pending;  // 1: total is still to be summed from the per-piece
                        // partials of the grid's last single-grid launch
};

// Host-written description of one grid for the step kernel (in device memory,
// so that one launch, or one graph node, can serve any number of grids).
struct TissueArgs {  // (CUtensorMap members impose its alignment)
    CUtensorMap tm_u[2];  // V of buffer b with halo (box TX+8 x TY+2)
    CUtensorMap tm_s[2];  // non-diffusing variables of buffer b (box TX x TY x S-1; with 16-bit gates: Ca only)
    CUtensorMap tm_g[2];  // 16-bit gates of buffer b (box TX x TY x 6 uint16), when stored so
    CUtensorMap tm_f;     // unit fibres, x stored from -4 with clamped padding (box TX x TY x 3, no halo)
    CUtensorMap tm_d;     // the W-tilde sums of every node (box TX x TY x 3)
    CUtensorMap tm_m;     // tissue mask bytes
    float* state[2];      // the ping-pong buffers, var v at state[b] + v*vol (32-bit variables)
    uint16_t* gate16[2];  // 16-bit gates: gate g (variable 2 + g) at gate16[b] + g*vol, or nullptr
    int32_t* act;         // activation steps
    const uint8_t* stim;  // stimulus region (nullptr: none)
    TissueDyn* dyn;
    long long plane, vol;  // px*ny, px*ny*nz
    double t_on, t_off;    // stimulus window, compared with t_n
    double dt_d;           // time step, for t_{n+1} = t_n + dt
    int nx, ny, nz, px;
    float dt, theta, stim_amp;
    int split;  // 1: Lie operator splitting (diffusion substep, then kinetics); 0: unsplit
    int rk4;    // kinetics solver: 1 classical RK4 (right-hand-side models), 0 forward Euler / Rush-Larsen
    int wsum_zero;  // 1: every W-tilde sum of the grid is exactly 0 (a single-grid launch then skips their copies)
    // diffusion constants over h^2: anisotropic D = Dperp I + (Dpar-Dperp) f f^T
    // gives c_perp = Dperp/h^2, c_d = (Dpar-Dperp)/h^2, c_dh = c_d/2 (edge
    // weights), c_s = c_d/4 (Wtilde); isotropic D gives c_iso = D/h^2.
    float c_perp, c_d, c_dh, c_s, c_iso;
    float mp[8];  // model parameters in kernel form
    const struct SurrogateData* surr;  // reaction surrogate (Beeler-Reuter), or nullptr
    const float4* tab;                 // V-table of the model (kTabN x 4 float4), or nullptr
};

// One launch: a balanced schedule of pieces over the grids of one kernel type.
// CTA c marches through the slots c*cta_stride .. c*cta_stride + cta_count[c]
// of pieces[]; a piece (x0, y0, z0, z1) is one 64 x TY column of grid
// piece_tissue[i] over the z-range [z0, z1).  A fixed stride lets a CTA find
// its first piece with one load.
//
// A launch over one grid (`single`) carries that grid's TissueArgs in the
// kernel parameters (t0): its tensor maps, constants and the pointer to its
// TissueDyn are then read from parameter space instead of through a chain of
// dependent global loads at the start of every CTA.
struct LaunchArgs {
    TissueArgs t0;             // the grid of a single-grid launch
    const TissueArgs* tissues;
    const int4* pieces;        // ctas x cta_stride slots
    const int* piece_tissue;   // per slot
    const int* cta_count;      // pieces of each CTA
    const int* tissue_off;     // grid t owns slots tissue_pieces[tissue_off[t] .. tissue_off[t+1])
    const int* tissue_pieces;  // (for the per-grid sums, in a fixed order)
    int n_tissues;
    int single;                // one grid: t0 is valid and slots are summed in index order
    int cta_stride;
    int n_slots;               // ctas x cta_stride; unused slots keep a zero partial
    double* partials;          // one per slot
    unsigned int* ticket;      // zero between launches
    unsigned int* tissue_done; // per grid: pieces finished in this launch (zero between launches)
    const int* empty_tissues;  // the grids with no piece (their time still advances)
    int n_empty;
    int* err;                  // sticky error bits
    long long wait_limit;      // clock64 cycles a wait may spin before giving up
    int poison_first_load;     // fault injection: CTA 0's first plane never completes
    // Single-grid launch: the buffer parity the host expects (-1: read it),
    // and for an unmasked 3D grid the schedule's shape, from which a CTA finds
    // its first piece without a memory read (reg_len = 0: read the list).  A
    // CTA then issues its first plane copies before any global load returns;
    // both are checked against device memory (ERRBIT_HINT on a mismatch).
    int cur_hint;
    int reg_len, reg_nbx, reg_ty, reg_ctas;  // column length (nz), columns in x, tile rows, CTAs
    long long reg_planes;                    // column-planes of the schedule
    int reg_z0;                              // first computed plane of every column (0; 1 below a halo plane)
};

struct Coef {
    float c_perp, c_d, c_dh, c_s, c_iso;
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

// Expect bytes on the barrier without arriving (the arrival comes later).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
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

// Stores of the new state: st.global states the address space, so the
// compiler need not assume they overwrite the shared-memory piece context
// (which it would otherwise reload after every store).
__device__ __forceinline__ void st_global(float* p, float2 v) {
    asm volatile("st.global.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ void st_global(float* p, float v) { asm volatile("st.global.f32 [%0], %1;" ::"l"(p), "f"(v)); }

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

// Per-CTA partial -> deterministic grid total by the last CTA to finish.  The
// last CTA sums the partials with all its threads (fixed strided order, then
// a fixed tree), so the result does not depend on which CTA finished last.
__device__ __forceinline__ void grid_total_finalize(double block_partial, double* partials,
                                                    unsigned int* ticket, double* out, int* err,
                                                    bool flag_nonfinite, double* scratch32) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = block_partial;
        if (flag_nonfinite && !isfinite(block_partial)) atomicOr(err, ERRBIT_NAN);
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += __ldcg(&partials[b]);
    __syncthreads();  // scratch32 may still be read by the caller's block sum
    const double total = block_sum_double(s, scratch32);
    if (threadIdx.x == 0) {
        *out = total;
        *ticket = 0u;
    }
}

// Single-grid launch, producer lane of every CTA, once its t, n and parity
// are read: the CTA that arrives last (all others have read them too)
// advances them, marks the total as pending and resets the ticket.
__device__ __forceinline__ void start_ticket(const LaunchArgs& L, const TissueDyn& d0) {
    __threadfence();
    const unsigned int t = atomicAdd(L.ticket, 1u);
    if (t == gridDim.x - 1) {
        TissueDyn* d = L.t0.dyn;
        d->t = d0.t + L.t0.dt_d;
        d->n = d0.n + 1;
        d->cur = d0.cur ^ 1;
        d->total_pending = 1;
        *L.ticket = 0u;
    }
}

// The fixed-order sum of a grid's per-piece partials tissue_pieces[k0 .. k1):
// each of `stride` threads takes every stride-th piece from `first`, four
// loads at a time so their L2 latencies overlap; then a shuffle tree over
// the warp (the caller adds the warps' results in order).
__device__ __forceinline__ double grid_partials_sum(const LaunchArgs& L, int k0, int k1, int first, int stride) {
    double s = 0.0;
    for (int k = k0 + first; k < k1; k += 4 * stride) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int kk = k + u * stride;
            v[u] = kk < k1 ? __ldcg(&L.partials[__ldcg(&L.tissue_pieces[kk])]) : 0.0;
        }
        s += (v[0] + v[1]) + (v[2] + v[3]);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// The end of a grid's step in a launch over several grids: its total, then
// t += dt, n += 1 and the buffer parity flip.
__device__ __forceinline__ void finish_grid(const LaunchArgs& L, int ti, double s) {
    const TissueArgs* T = L.tissues + ti;
    TissueDyn* d = T->dyn;
    if (!isfinite(s)) atomicOr(L.err, ERRBIT_NAN);
    d->total = s;
    d->t = d->t + T->dt_d;
    d->n = d->n + 1;
    d->cur = d->cur ^ 1;
    d->total_pending = 0;
}

// Launch over several grids, one warp of the CTA that has just written the
// partial of piece pi (lane 0 wrote it): the piece counts towards its grid,
// and the CTA that completes a grid finishes it at once (per-grid sums spread
// over the CTAs while the others still compute, instead of one CTA summing
// every grid at the end).  A grid's pieces all precede its finish, so no
// producer reads the grid's parity after it flips.
__device__ __forceinline__ void grid_piece_done(const LaunchArgs& L, int pi, int lane) {
    int fin = -1;
    if (lane == 0) {
        __threadfence();  // the piece's partial before its count
        const int ti = L.piece_tissue[pi];
        const unsigned int npc = (unsigned int)(L.tissue_off[ti + 1] - L.tissue_off[ti]);
        if (atomicAdd(&L.tissue_done[ti], 1u) == npc - 1u) fin = ti;
    }
    fin = __shfl_sync(0xffffffffu, fin, 0);
    if (fin < 0) return;
    __threadfence();
    const double s = grid_partials_sum(L, __ldcg(&L.tissue_off[fin]), __ldcg(&L.tissue_off[fin + 1]), lane, 32);
    if (lane == 0) {
        finish_grid(L, fin, s);
        L.tissue_done[fin] = 0u;
    }
}

// End of a launch over several grids: the grids without pieces (no tissue)
// advance t, n and the parity in the last CTA to finish; the others were
// finished by grid_piece_done.  A single-grid launch has no end step: its
// producers advance t, n and the parity as soon as every CTA has read them
// (start_ticket), and the grid's total is summed from the partials when it
// is asked for.
__device__ __forceinline__ void step_finalize(const LaunchArgs& L, double* scratch32) {
    __shared__ bool last;
    (void)scratch32;
    if (L.single || L.n_empty == 0) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(L.ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    for (int e = threadIdx.x; e < L.n_empty; e += blockDim.x) finish_grid(L, __ldcg(&L.empty_tissues[e]), 0.0);
    __syncthreads();
    if (threadIdx.x == 0) *L.ticket = 0u;
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
    // right-hand side with the source I (diffusion term + stimulus) on u
    __device__ static __forceinline__ void rhs(const float* mp, const float* y, float I, float* dy) {
        const float u = y[0], v = y[1];
        dy[0] = (u - u * u * u * (1.0f / 3.0f) - v) * mp[0] + I;
        dy[1] = mp[1] * (u + mp[2] - mp[3] * v);
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
    __device__ static __forceinline__ void rhs(const float* mp, const float* y, float I, float* dy) {
        const float u = y[0], v = y[1];
        dy[0] = u * (1.0f - u) * (u - (v + mp[1]) * mp[0]) * mp[2] + I;
        dy[1] = u - v;
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
    __device__ static __forceinline__ void rhs(const float* mp, const float* y, float I, float* dy) {
        const float u = y[0];
        dy[0] = u * (u - mp[0]) * (1.0f - u) + I;
    }
};

// Diffusion equation alone.
template <>
struct Model<BBX_DIFFUSION> {
    static constexpr int S = 1;
    __device__ static __forceinline__ void update(const float*, float* y, float L, float Is, float dt) {
        y[0] = y[0] + dt * (L + Is);
    }
    __device__ static __forceinline__ void rhs(const float*, const float*, float I, float* dy) { dy[0] = I; }
};

// One classical fourth-order Runge-Kutta step (the rk4 kinetics solver of
// section "Explicit solvers") of a model given by its right-hand side, with
// the diffusion term and stimulus held fixed over the step as a source on the
// first variable: stages at t, t + dt/2, t + dt/2, t + dt; weights 1, 2, 2, 1
// over 6.
template <int MODEL>
__device__ __forceinline__ void rk4_update(const float* mp, float* y, float L, float Is, float dt) {
    constexpr int S = Model<MODEL>::S;
    const float I = L + Is, h2 = 0.5f * dt;
    float k1[S], k2[S], k3[S], k4[S], t[S];
    Model<MODEL>::rhs(mp, y, I, k1);
#pragma unroll
    for (int v = 0; v < S; ++v) t[v] = y[v] + h2 * k1[v];
    Model<MODEL>::rhs(mp, t, I, k2);
#pragma unroll
    for (int v = 0; v < S; ++v) t[v] = y[v] + h2 * k2[v];
    Model<MODEL>::rhs(mp, t, I, k3);
#pragma unroll
    for (int v = 0; v < S; ++v) t[v] = y[v] + dt * k3[v];
    Model<MODEL>::rhs(mp, t, I, k4);
#pragma unroll
    for (int v = 0; v < S; ++v) y[v] += (dt * (1.0f / 6.0f)) * ((k1[v] + k4[v]) + 2.0f * (k2[v] + k3[v]));
}

// Beeler-Reuter (1977).  State (V, Ca, x1, m, h, j, d, f); mp = {gNa, gNaC,
// ENa, gs}.  V in mV, t in ms, Ca in mol/L, currents in uA/cm^2, Cm = 1.
// Rate constants of the 1977 publication, written out per gate.
__device__ __forceinline__ float br_ratio(float num, float den) { return __fdividef(num, den); }

// e^x - 1 in FP32: near 0 the Taylor series of e^x - 1 about 0 up to x^7/5040
// (|x| < 0.25: the first omitted term is below 2e-9 of the value), elsewhere
// the difference e^x - 1, whose cancellation is bounded there (e^x - 1 >= 0.22
// for x >= 0.25, <= -0.22 for x <= -0.25).
__device__ __forceinline__ float expm1_br(float x) {
    if (fabsf(x) < 0.25f) {
        float p = fmaf(x, 1.0f / 5040.0f, 1.0f / 720.0f);
        p = fmaf(x, p, 1.0f / 120.0f);
        p = fmaf(x, p, 1.0f / 24.0f);
        p = fmaf(x, p, 1.0f / 6.0f);
        p = fmaf(x, p, 0.5f);
        p = fmaf(x, p, 1.0f);
        return x * p;
    }
    return __expf(x) - 1.0f;
}

// Voltage tables of the Beeler-Reuter models: kTabN entries kTabDv mV apart
// from kTabVmin (-120 to +80 mV), 16 floats (4 float4) each; V outside the
// range takes the end entry.  Entry index and interpolation weight of V.
constexpr float kTabVmin = -120.0f, kTabDv = 0.025f, kTabInvDv = 40.0f;
constexpr int kTabN = 8001;
__device__ __forceinline__ int tab_index(float V, float* w) {
    float xi = (V - kTabVmin) * kTabInvDv;
    xi = fminf(fmaxf(xi, 0.0f), (float)(kTabN - 1));
    int i = (int)xi;
    if (i > kTabN - 2) i = kTabN - 2;
    *w = xi - (float)i;
    return i;
}

template <>
struct Model<BBX_BR> {
    static constexpr int S = 8;


    // The change of every variable over one step (the update is y + d): the
    // Euler increments of V and Ca, and the Rush-Larsen increments of the
    // gates, Eq. (RL) read as y' = A y + B, i.e. d = (1 - A)(y_inf - y) with
    // 1 - A by expm1_br (no cancellation when (alpha+beta) dt is small).
    __device__ static __forceinline__ void increment(const float* mp, const float* y, float L, float Is, float dt,
                                                     float* d) {
        increment_m3(mp, y, y[3] * y[3] * y[3], L, Is, dt, d);
    }

    // The same with the open probability m3 of the sodium activation given
    // (y[3] only feeds the m-gate increment d[3]).
    __device__ static __forceinline__ void increment_m3(const float* mp, const float* y, float m3, float L,
                                                        float Is, float dt, float* d) {
        const float V = y[0], Ca = y[1];
        const float x1 = y[2], m = y[3], h = y[4], j = y[5], dd = y[6], f = y[7];

        // membrane currents
        const float INa = (mp[0] * m3 * h * j + mp[1]) * (V - mp[2]);
        const float Es = -82.3f - 13.0287f * __logf(Ca);
        const float Is_ = mp[3] * dd * f * (V - Es);
        const float Ix1 = x1 * 0.8f * (__expf(0.04f * (V + 77.0f)) - 1.0f) * __expf(-0.04f * (V + 35.0f));
        const float w = V + 23.0f;
        const float lin = (w == 0.0f) ? 5.0f : br_ratio(0.2f * w, -expm1_br(-0.04f * w));
        const float IK1 = 0.35f * (br_ratio(4.0f * (__expf(0.04f * (V + 85.0f)) - 1.0f),
                                            __expf(0.08f * (V + 53.0f)) + __expf(0.04f * (V + 53.0f))) +
                                   lin);
        const float Iion = INa + Is_ + Ix1 + IK1;
        const float dCa = -1e-7f * Is_ + 0.07f * (1e-7f - Ca);

        // gate rates, 1/ms
        const float a_x1 = br_ratio(0.0005f * __expf(0.083f * (V + 50.0f)), __expf(0.057f * (V + 50.0f)) + 1.0f);
        const float b_x1 = br_ratio(0.0013f * __expf(-0.06f * (V + 20.0f)), __expf(-0.04f * (V + 20.0f)) + 1.0f);
        const float xm = V + 47.0f;
        const float a_m = (xm == 0.0f) ? 10.0f : br_ratio(-xm, expm1_br(-0.1f * xm));
        const float b_m = 40.0f * __expf(-0.056f * (V + 72.0f));
        const float a_h = 0.126f * __expf(-0.25f * (V + 77.0f));
        const float b_h = br_ratio(1.7f, __expf(-0.082f * (V + 22.5f)) + 1.0f);
        const float a_j = br_ratio(0.055f * __expf(-0.25f * (V + 78.0f)), __expf(-0.2f * (V + 78.0f)) + 1.0f);
        const float b_j = br_ratio(0.3f, __expf(-0.1f * (V + 32.0f)) + 1.0f);
        const float a_d = br_ratio(0.095f * __expf(-0.01f * (V - 5.0f)), __expf(-0.072f * (V - 5.0f)) + 1.0f);
        const float b_d = br_ratio(0.07f * __expf(-0.017f * (V + 44.0f)), __expf(0.05f * (V + 44.0f)) + 1.0f);
        float a_f, b_f;
        f_rates(V, &a_f, &b_f);

        d[0] = dt * (-(Iion - Is) + L);  // Cm = 1
        d[1] = dt * dCa;
        d[2] = rl_inc(x1, a_x1, b_x1, dt);
        d[3] = rl_inc(m, a_m, b_m, dt);
        d[4] = rl_inc(h, a_h, b_h, dt);
        d[5] = rl_inc(j, a_j, b_j, dt);
        d[6] = rl_inc(dd, a_d, b_d, dt);
        d[7] = rl_inc(f, a_f, b_f, dt);
    }

    // alpha_f and beta_f, the rates of the slow inward current's inactivation
    __device__ static __forceinline__ void f_rates(float V, float* a_f, float* b_f) {
        *a_f = br_ratio(0.012f * __expf(-0.008f * (V + 28.0f)), __expf(0.15f * (V + 28.0f)) + 1.0f);
        *b_f = br_ratio(0.0065f * __expf(-0.02f * (V + 30.0f)), __expf(-0.2f * (V + 30.0f)) + 1.0f);
    }

    __device__ static __forceinline__ float rl_inc(float y, float al, float be, float dt) {
        const float s = al + be;
        const float one_minus_A = -expm1_br(-s * dt);
        return one_minus_A * (__fdividef(al, s) - y);
    }

    __device__ static __forceinline__ void update(const float* mp, float* y, float L, float Is, float dt) {
        float d[8];
        increment(mp, y, L, Is, dt, d);
#pragma unroll
        for (int v = 0; v < 8; ++v) y[v] = y[v] + d[v];
    }

    // The same step with the Rush-Larsen coefficients tabulated in V (the
    // rushlarsen device's tabulation, section "Exponential solvers"): per
    // entry A and B of Eq. (RL) for x1, m, h, j, d, f, then the V factors of
    // I_x1 (I_x1 = x1 K(V)) and I_K1, interpolated linearly; gates by
    // y' = A y + B.  The table is built for the grid's dt.
    __device__ static __forceinline__ void update_tab(const float* mp, const float4* __restrict__ tab, float* y,
                                                      float L, float Is, float dt) {
        const float V = y[0], Ca = y[1];
        float w;
        const int i = tab_index(V, &w);
        float c[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 a = __ldg(tab + 4 * i + q), b = __ldg(tab + 4 * i + 4 + q);
            c[4 * q + 0] = fmaf(w, b.x - a.x, a.x);
            c[4 * q + 1] = fmaf(w, b.y - a.y, a.y);
            c[4 * q + 2] = fmaf(w, b.z - a.z, a.z);
            c[4 * q + 3] = fmaf(w, b.w - a.w, a.w);
        }
        const float m = y[3];
        const float INa = (mp[0] * m * m * m * y[4] * y[5] + mp[1]) * (V - mp[2]);
        const float Es = -82.3f - 13.0287f * __logf(Ca);
        const float Is_ = mp[3] * y[6] * y[7] * (V - Es);
        const float Iion = INa + Is_ + y[2] * c[12] + c[13];
        const float dCa = -1e-7f * Is_ + 0.07f * (1e-7f - Ca);
        y[0] = V + dt * (-(Iion - Is) + L);  // Cm = 1
        y[1] = Ca + dt * dCa;
#pragma unroll
        for (int g = 0; g < 6; ++g) y[2 + g] = fmaf(c[2 * g], y[2 + g], c[2 * g + 1]);
    }
};

// Beeler-Reuter with the sodium activation m^3 in its Markov form: the
// probabilities P0..P3 that k = 0..3 of the three activation subunits are
// open (P3 in place of m^3), du/dt = A(V) u with k -> k+1 at (3-k) alpha_m
// and k -> k-1 at k beta_m, advanced by the matrix Rush-Larsen scheme
// u_{n+1} = T(V_n) u_n, T = exp(dt A) (section "Exponential solvers").  T is
// tabulated in V (kTabN entries kTabDv mV apart from kTabVmin, 16 floats
// each, row-major; built on the device for the grid's dt) and interpolated
// linearly; V outside the table takes the end entry.  x1, h, j, d, f by
// Eq. (RL) with tabulated coefficients (as Model<BBX_BR>::update_tab), V and
// Ca by Eq. (Euler).
// State: V, Ca, x1, h, j, d, f, P0, P1, P2, P3.

template <>
struct Model<BBX_BR_MRL> {
    static constexpr int S = 11;

    // tab: the Rush-Larsen table of Model<BBX_BR>::update_tab (kTabN x 4
    // float4), followed by the chain's transition matrices (kTabN x 4 float4).
    __device__ static __forceinline__ void update_tab(const float* mp, const float4* __restrict__ tab, float* y,
                                                      float L, float Is, float dt) {
        const float V = y[0], Ca = y[1];
        float w;
        const int i = tab_index(V, &w);
        float c[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 a = __ldg(tab + 4 * i + q), b = __ldg(tab + 4 * i + 4 + q);
            c[4 * q + 0] = fmaf(w, b.x - a.x, a.x);
            c[4 * q + 1] = fmaf(w, b.y - a.y, a.y);
            c[4 * q + 2] = fmaf(w, b.z - a.z, a.z);
            c[4 * q + 3] = fmaf(w, b.w - a.w, a.w);
        }
        // the chain, from V at the start of the step
        const float4* t0 = tab + 4 * kTabN + 4 * i;
        float pn[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float4 a = __ldg(t0 + r), b = __ldg(t0 + 4 + r);
            const float qa = fmaf(a.x, y[7], fmaf(a.y, y[8], fmaf(a.z, y[9], a.w * y[10])));
            const float qb = fmaf(b.x, y[7], fmaf(b.y, y[8], fmaf(b.z, y[9], b.w * y[10])));
            pn[r] = fmaf(w, qb - qa, qa);
        }
        // currents with P3 in place of m^3; x1, h, j, d, f by y' = A y + B
        const float INa = (mp[0] * y[10] * y[3] * y[4] + mp[1]) * (V - mp[2]);
        const float Es = -82.3f - 13.0287f * __logf(Ca);
        const float Is_ = mp[3] * y[5] * y[6] * (V - Es);
        const float Iion = INa + Is_ + y[2] * c[12] + c[13];
        const float dCa = -1e-7f * Is_ + 0.07f * (1e-7f - Ca);
        y[0] = V + dt * (-(Iion - Is) + L);  // Cm = 1
        y[1] = Ca + dt * dCa;
        y[2] = fmaf(c[0], y[2], c[1]);  // x1
#pragma unroll
        for (int g = 0; g < 4; ++g) y[3 + g] = fmaf(c[4 + 2 * g], y[3 + g], c[5 + 2 * g]);  // h, j, d, f
#pragma unroll
        for (int r = 0; r < 4; ++r) y[7 + r] = pn[r];
    }
};

// Beeler-Reuter with the slow inward current's inactivation as a two-gate
// channel: the voltage gate f (alpha_f, beta_f of the 1977 model) and a
// calcium gate c (closed -> open at c_inf / tau_c, open -> closed at
// (1 - c_inf) / tau_c, c_inf = Kc / (Kc + Ca)), the four states q = f + 2 c
// with probabilities Q0..Q3, and a small direct transition (f open, c
// closed) -> (f closed, c open) at eps alpha_f (1 - c_inf).  The generator
// A(V, Ca) of Eq. (markov-generic) is the sum of a V-univariate matrix (the
// f gate), a Ca-univariate matrix (the c gate) and that multivariate
// remainder; section "Exponential solvers" advances such a chain by Lie
// splitting: each univariate part by its exact step from the values of V
// and Ca at the start of the step, the remainder by forward Euler.  The f
// gate's step comes from the Rush-Larsen V-table; the c gate's rates sum to
// 1/tau_c at every Ca, so its step has the closed form open' = open +
// (1 - e^{-dt/tau_c}) (c_inf total - open) with one constant.  Both gate steps
// move probability within pairs of states (total of the pair kept exactly).
// With the parameter onfly set, the channel takes the step the same section
// gives for a generator with no such decomposition instead: the exponential
// of the whole A(V, Ca) applied at run time, with no table and no splitting.
// I_s = g_s d Q3 (V - E_s); x1, m, h, j, d by Rush-Larsen; V, Ca by Euler.
// State: V, Ca, x1, m, h, j, d, Q0, Q1, Q2, Q3.
// Kernel parameters mp: gNa, gNaC, ENa, gs, Kc, eps, 1/tau_c, onfly (0 or 1).

template <>
struct Model<BBX_BR_FCA> {
    static constexpr int S = 11;

    // the channel step (u = Q0..Q3): f gate by open' = A_f open + B_f total,
    // c gate as above with omc = 1 - e^{-dt/tau_c}, then the remainder
    __device__ static __forceinline__ void channel(const float* mp, float A_f, float B_f, float a_f, float omc,
                                                   float Ca, float dt, float* u) {
        const float pc0 = u[0] + u[1], pc1 = u[2] + u[3];  // c closed, c open
        const float fo0 = fmaf(A_f, u[1], B_f * pc0), fo1 = fmaf(A_f, u[3], B_f * pc1);
        u[0] = pc0 - fo0;
        u[1] = fo0;
        u[2] = pc1 - fo1;
        u[3] = fo1;
        const float inv = __fdividef(1.0f, mp[4] + Ca);
        const float ci = mp[4] * inv, one_minus_ci = Ca * inv;
        const float pf0 = u[0] + u[2], pf1 = u[1] + u[3];  // f closed, f open
        const float co0 = fmaf(omc, fmaf(ci, pf0, -u[2]), u[2]), co1 = fmaf(omc, fmaf(ci, pf1, -u[3]), u[3]);
        u[0] = pf0 - co0;
        u[2] = co0;
        u[1] = pf1 - co1;
        u[3] = co1;
        const float flow = dt * mp[5] * a_f * one_minus_ci * u[1];
        u[1] -= flow;
        u[2] += flow;
    }

    // u <- exp(dt A(V, Ca)) u with every rate evaluated at the node: the
    // Taylor series of the exponential's action on u to nine terms, on 2^s
    // substeps, s the smallest (at most 6) that brings dt / 2^s times the
    // largest absolute column sum of A (twice the largest outflow) to 1/2.
    __device__ static __forceinline__ void channel_onfly(const float* mp, float V, float Ca, float dt, float* u) {
        float a_f, b_f;
        Model<BBX_BR>::f_rates(V, &a_f, &b_f);
        const float inv = __fdividef(1.0f, mp[4] + Ca);
        const float a_c = mp[4] * inv * mp[6], b_c = Ca * inv * mp[6];
        const float r = mp[5] * a_f * (Ca * inv);
        // outflow of each state q = f + 2 c
        const float o0 = a_f + a_c, o1 = b_f + a_c + r, o2 = a_f + b_c, o3 = b_f + b_c;
        float nrm = 2.0f * dt * fmaxf(fmaxf(o0, o1), fmaxf(o2, o3)), h = dt;
        int s = 0;
        while (nrm > 0.5f && s < 6) {
            nrm *= 0.5f;
            h *= 0.5f;
            ++s;
        }
        for (int k = 0; k < (1 << s); ++k) {
            float t0 = u[0], t1 = u[1], t2 = u[2], t3 = u[3];
            float s0 = t0, s1 = t1, s2 = t2, s3 = t3;
#pragma unroll
            for (int n = 1; n <= 9; ++n) {
                const float c = h * (1.0f / (float)n);
                const float n0 = fmaf(-o0, t0, fmaf(b_f, t1, b_c * t2));
                const float n1 = fmaf(a_f, t0, fmaf(-o1, t1, b_c * t3));
                const float n2 = fmaf(a_c, t0, fmaf(r, t1, fmaf(-o2, t2, b_f * t3)));
                const float n3 = fmaf(a_c, t1, fmaf(a_f, t2, -o3 * t3));
                t0 = c * n0;
                t1 = c * n1;
                t2 = c * n2;
                t3 = c * n3;
                s0 += t0;
                s1 += t1;
                s2 += t2;
                s3 += t3;
            }
            u[0] = s0;
            u[1] = s1;
            u[2] = s2;
            u[3] = s3;
        }
    }

    // tab: the Rush-Larsen table of Model<BBX_BR>::update_tab (kTabN x 4
    // float4) with entry 14 = alpha_f(V) and entry 15 = 1 - e^{-dt/tau_c}.
    __device__ static __forceinline__ void update_tab(const float* mp, const float4* __restrict__ tab, float* y,
                                                      float L, float Is, float dt) {
        const float V = y[0], Ca = y[1];
        float w;
        const int i = tab_index(V, &w);
        float c[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 a = __ldg(tab + 4 * i + q), b = __ldg(tab + 4 * i + 4 + q);
            c[4 * q + 0] = fmaf(w, b.x - a.x, a.x);
            c[4 * q + 1] = fmaf(w, b.y - a.y, a.y);
            c[4 * q + 2] = fmaf(w, b.z - a.z, a.z);
            c[4 * q + 3] = fmaf(w, b.w - a.w, a.w);
        }
        const float m = y[3];
        const float INa = (mp[0] * m * m * m * y[4] * y[5] + mp[1]) * (V - mp[2]);
        const float Es = -82.3f - 13.0287f * __logf(Ca);
        const float Is_ = mp[3] * y[6] * y[10] * (V - Es);
        const float Iion = INa + Is_ + y[2] * c[12] + c[13];
        const float dCa = -1e-7f * Is_ + 0.07f * (1e-7f - Ca);
        y[0] = V + dt * (-(Iion - Is) + L);  // Cm = 1
        y[1] = Ca + dt * dCa;
#pragma unroll
        for (int g = 0; g < 5; ++g) y[2 + g] = fmaf(c[2 * g], y[2 + g], c[2 * g + 1]);  // x1, m, h, j, d
        if (mp[7] != 0.0f)
            channel_onfly(mp, V, Ca, dt, y + 7);
        else
            channel(mp, c[10], c[11], c[14], c[15], Ca, dt, y + 7);
    }

    // The same step with every rate evaluated at V (no table): the rest-state
    // integration uses it.
    __device__ static __forceinline__ void update(const float* mp, float* y, float L, float Is, float dt) {
        const float V = y[0], Ca = y[1];
        float y8[8] = {y[0], y[1], y[2], y[3], y[4], y[5], y[6], y[10]};  // Q3 in the place of f
        float d[8];
        Model<BBX_BR>::increment_m3(mp, y8, y[3] * y[3] * y[3], L, Is, dt, d);
        float a_f, b_f;
        Model<BBX_BR>::f_rates(V, &a_f, &b_f);
        const float omA = -expm1_br(-(a_f + b_f) * dt);
        const float omc = -expm1_br(-dt * mp[6]);
#pragma unroll
        for (int v = 0; v < 7; ++v) y[v] += d[v];
        if (mp[7] != 0.0f)
            channel_onfly(mp, V, Ca, dt, y + 7);
        else
            channel(mp, 1.0f - omA, __fdividef(a_f, a_f + b_f) * omA, a_f, omc, Ca, dt, y + 7);
    }
};

// ---------------------------------------------------------------------------
// shared-memory plan of the step kernel
// ---------------------------------------------------------------------------

constexpr int kTileX = 64;  // nodes per brick along x: 32 threads x 2 nodes
// Consumer warps per CTA (plus one producer warp) for a tile of TY rows: 7
// warps of 1 or 2 rows each for TY = 7, 14 (two CTAs per SM), 14 warps of 2
// rows for TY = 28 (one CTA of 480 threads per SM, whose warps share one
// ring of planes and so finish together).
__host__ __device__ constexpr int rows_of_threads(int ty) { return ty == 28 ? 14 : 7; }

// Anisotropy of a step kernel variant: isotropic (c_iso only), anisotropic
// with the W-tilde sums read from memory, or anisotropic for grids whose
// W-tilde sums all vanish (no sums in the stage ring, no W-tilde arithmetic).
enum : int { AN_ISO = 0, AN_SUMS = 1, AN_NO_SUMS = 2 };

// Resident CTAs per SM a kernel variant is built for (the register budget:
// two CTAs of 256 threads allow 128 registers a thread; the masked
// anisotropic stencil with 2 rows a thread and the surrogate need more; the
// unmasked isotropic variants fit in 64, so four CTAs hide more latency).
__host__ __device__ constexpr int ctas_per_sm(bool masked, bool aniso, int ty, bool surr) {
    return (masked && aniso && ty != 7) || ty == 28 || (surr && ty != 7) ? 1 : (!masked && !aniso && !surr ? 4 : 2);
}
constexpr int align128(int b) { return (b + 127) & ~127; }

// Tissue-mask byte on the device: bit 0 = tissue, bit 1 = tissue node whose
// 18 stencil neighbours are all tissue inside the array ("interior").
enum : uint8_t { MASK_TISSUE = 1, MASK_INTERIOR = 2 };

// Storage of the Beeler-Reuter gates (variables 2..7) between steps: FP32
// (default), IEEE binary16, or 16-bit unsigned fixed point y = u / 65535
// (uniform steps of 1.5e-5 over [0, 1]); arithmetic is FP32 in every case,
// the new values rounded to nearest when stored.
enum : int { GATES_F32 = 0, GATES_F16 = 1, GATES_U16 = 2 };

template <int GATES>
__device__ __forceinline__ float2 gate_decode2(uint32_t w) {
    if (GATES == GATES_F16) {
        __half2 h = *reinterpret_cast<__half2*>(&w);
        return __half22float2(h);
    }
    constexpr float k = 1.0f / 65535.0f;
    return make_float2((float)(w & 0xffffu) * k, (float)(w >> 16) * k);
}

template <int GATES>
__device__ __forceinline__ uint16_t gate_encode(float y) {
    if (GATES == GATES_F16) return __half_as_ushort(__float2half_rn(y));
    return (uint16_t)__float2uint_rn(__saturatef(y) * 65535.0f);
}

template <int GATES>
__device__ __forceinline__ uint32_t gate_encode2(float lo, float hi) {
    return (uint32_t)gate_encode<GATES>(lo) | ((uint32_t)gate_encode<GATES>(hi) << 16);
}

__device__ __forceinline__ void st_global_u32(uint16_t* p, uint32_t v) {
    asm volatile("st.global.u32 [%0], %1;" ::"l"(p), "r"(v));
}
__device__ __forceinline__ void st_global_u16(uint16_t* p, uint16_t v) {
    asm volatile("st.global.u16 [%0], %1;" ::"l"(p), "h"(v));
}

template <int MODEL, bool MASKED, int ANISO, int TY, bool SURR = false, int GATES = GATES_F32>
struct Plan {
    static constexpr int S = Model<MODEL>::S;
    static constexpr int NG = GATES ? 6 : 0;  // variables stored in 16 bits (the gates, last in the state)
    static constexpr int TX = kTileX;
    static constexpr int RY = rows_of_threads(TY);
    static constexpr int CTAS = ctas_per_sm(MASKED, ANISO != AN_ISO, TY, SURR);
    static constexpr int CY = TY / RY;  // nodes per thread along y (each a pair in x)
    static constexpr int THREADS = 32 * RY + 32;  // consumer warps + producer warp
    static constexpr int UW = TX + 8;   // x from x0-4 to x0+TX+3 (16-byte aligned start)
    static constexpr int UH = TY + 2;   // y from y0-1 to y0+TY
    static constexpr int MW = TX + 32;  // mask bytes: x from x0-16 (16-byte aligned start)
    // ring A, one stage per loaded plane (the computed planes and the z-halo
    // planes): V with its one-node halo, the mask with its halo
    static constexpr int U_RAW = UW * UH * 4;
    static constexpr int M_RAW = MASKED ? MW * UH : 0;
    static constexpr int U_OFF = 0;
    static constexpr int M_OFF = U_OFF + align128(U_RAW);
    static constexpr int A_STAGE = M_OFF + align128(M_RAW);
    static constexpr uint32_t A_BYTES = U_RAW + M_RAW;
    // ring B, one stage per computed plane: the node's own unit fibre and
    // W-tilde sums (3 x TX x TY floats each), the other variables
    static constexpr int F_RAW = ANISO ? 3 * TX * TY * 4 : 0;
    static constexpr int D_RAW = ANISO == AN_SUMS ? 3 * TX * TY * 4 : 0;
    static constexpr int S32_RAW = (S > 1) ? (S - 1 - NG) * TX * TY * 4 : 0;  // 32-bit non-diffusing variables
    static constexpr int G_RAW = NG * TX * TY * 2;                              // 16-bit gates
    static constexpr int S_RAW = S32_RAW + G_RAW;
    static constexpr int F_OFF = 0;
    static constexpr int D_OFF = F_OFF + F_RAW;    // (each part a multiple of 128 bytes)
    static constexpr int S_OFF = D_OFF + D_RAW;
    static constexpr int G_OFF = S_OFF + S32_RAW;
    static constexpr int B_STAGE = align128(F_RAW + D_RAW + S_RAW);
    static constexpr uint32_t B_BYTES = F_RAW + D_RAW + S_RAW;
    static constexpr bool HAS_B = B_BYTES > 0;
    static constexpr int BUDGET = (CTAS == 1 ? 200 : 112) * 1024;  // dynamic shared memory per CTA
    static constexpr int NB = !HAS_B ? 0 : (3 * B_STAGE + 5 * A_STAGE <= BUDGET ? 3 : 2);
    static constexpr int NA_FIT = (BUDGET - NB * B_STAGE) / A_STAGE;
    static constexpr int NA = NA_FIT > 8 ? 8 : (NA_FIT < 4 ? 4 : NA_FIT);
    static constexpr int WBUF = SURR ? RY * 2048 : 0;  // per consumer warp: 64 rows of 32 bytes
    static constexpr int BAR_OFF = NA * A_STAGE + NB * B_STAGE + WBUF;
    // stages, warp buffers, full/empty barriers of both rings, piece contexts
    static constexpr int SMEM = 128 + BAR_OFF + 2 * (NA + NB) * 8 + NA * 176;
    static_assert(TY % RY == 0 && CY >= 1, "tile rows must be a multiple of the thread rows");
    static_assert(U_RAW % 16 == 0 && F_RAW % 128 == 0 && D_RAW % 128 == 0 && S32_RAW % 128 == 0, "stage layout");
};

struct F3 {
    float x, y, z;
};

// Neighbour values of one node: faces, then the 12 edges of the 19-point
// stencil ("pm" = x+1,y-1 etc.).
struct Nb {
    float u0, xp, xm, yp, ym, zp, zm;
    float pp, mm, pm, mp;          // (x,y) edges
    float xpzp, xmzm, xpzm, xmzp;  // (x,z) edges
    float ypzp, ymzm, ypzm, ymzp;  // (y,z) edges
};

// The precomputed ingredients of Eq. (Lu) at a node: the unit fibre f (D =
// Dperp I + (Dpar - Dperp) f f^T, Eq. (sigma)) and the W-tilde sums sd_k =
// sum_j (f_j f_k at p + q_j minus at p - q_j), with a void neighbour's fibre
// replaced by f at p (computed once per grid, k_divergence).

// (L u)_p for a node whose 18 neighbours are all tissue: the weights of
// Eq. (Lu) with psi = 1 everywhere, in difference form.  c_perp = Dperp/h^2,
// c_d = (Dpar-Dperp)/h^2, c_dh = c_d/2, c_s = c_d/4.
template <int ANISO>
__device__ __forceinline__ float lap_interior(const Coef& a, const Nb& n, F3 f, F3 sd) {
    if (!ANISO) {
        return a.c_iso * (((n.xp + n.xm) + (n.yp + n.ym)) + (n.zp + n.zm) - 6.0f * n.u0);
    }
    const float Dxx = fmaf(a.c_d, f.x * f.x, a.c_perp);
    const float Dyy = fmaf(a.c_d, f.y * f.y, a.c_perp);
    const float Dzz = fmaf(a.c_d, f.z * f.z, a.c_perp);
    const float hx = a.c_dh * f.x;
    const float Dxy = hx * f.y, Dxz = hx * f.z, Dyz = a.c_dh * f.y * f.z;
    const float two_u = 2.0f * n.u0;
    float L = Dxx * ((n.xp + n.xm) - two_u);
    L = fmaf(Dyy, (n.yp + n.ym) - two_u, L);
    L = fmaf(Dzz, (n.zp + n.zm) - two_u, L);
    if (ANISO == AN_SUMS) {
        float dv = sd.x * (n.xp - n.xm);
        dv = fmaf(sd.y, n.yp - n.ym, dv);
        dv = fmaf(sd.z, n.zp - n.zm, dv);
        L = fmaf(a.c_s, dv, L);
    }
    L = fmaf(Dxy, (n.pp + n.mm) - (n.pm + n.mp), L);
    L = fmaf(Dxz, (n.xpzp + n.xmzm) - (n.xpzm + n.xmzp), L);
    L = fmaf(Dyz, (n.ypzp + n.ymzm) - (n.ypzm + n.ymzp), L);
    return L;
}

// (L u)_p for a node of an unmasked grid whose y and z neighbours are inside
// the array; px, mx in {0, 1} are psi of the x+1 and x-1 neighbours (0 only
// at the array's x faces).
template <int ANISO>
__device__ __forceinline__ float lap_xbound(const Coef& a, const Nb& n, float px, float mx, F3 f, F3 sd) {
    const float ex = px * (n.xp - n.u0) + mx * (n.xm - n.u0);
    if (!ANISO) {
        return a.c_iso * ((ex + (n.yp + n.ym)) + (n.zp + n.zm) - 4.0f * n.u0);
    }
    const float Dxx = fmaf(a.c_d, f.x * f.x, a.c_perp);
    const float Dyy = fmaf(a.c_d, f.y * f.y, a.c_perp);
    const float Dzz = fmaf(a.c_d, f.z * f.z, a.c_perp);
    const float hx = a.c_dh * f.x;
    const float Dxy = hx * f.y, Dxz = hx * f.z, Dyz = a.c_dh * f.y * f.z;
    const float two_u = 2.0f * n.u0;
    float L = Dxx * ex;
    L = fmaf(Dyy, (n.yp + n.ym) - two_u, L);
    L = fmaf(Dzz, (n.zp + n.zm) - two_u, L);
    if (ANISO == AN_SUMS) {
        float dv = (px * mx) * sd.x * (n.xp - n.xm);
        dv = fmaf(sd.y, n.yp - n.ym, dv);
        dv = fmaf(sd.z, n.zp - n.zm, dv);
        L = fmaf(a.c_s, dv, L);
    }
    L = fmaf(Dxy, px * (n.pp - n.pm) + mx * (n.mm - n.mp), L);
    L = fmaf(Dxz, px * (n.xpzp - n.xpzm) + mx * (n.xmzm - n.xmzp), L);
    L = fmaf(Dyz, (n.ypzp + n.ymzm) - (n.ypzm + n.ymzp), L);
    return L;
}

// Grid indicator psi of the 18 neighbours (bit order: xp xm yp ym zp zm, then
// pp mm pm mp, xpzp xmzm xpzm xmzp, ypzp ymzm ypzm ymzp).
struct Psi {
    bool xp, xm, yp, ym, zp, zm;
    bool pp, mm, pm, mp;
    bool xpzp, xmzm, xpzm, xmzp;
    bool ypzp, ymzm, ypzm, ymzp;
};

// (L u)_p for any tissue node: every weight carries its psi (a void or
// out-of-array neighbour contributes nothing); the W-tilde sums already hold
// a void neighbour's tensor replaced by D^p.
template <int ANISO>
__device__ __forceinline__ float lap_general(const Coef& a, const Nb& n, const Psi& q, F3 f, F3 sd) {
    auto d = [&](bool ps, float uq) { return ps ? (uq - n.u0) : 0.0f; };
    const float exp_ = d(q.xp, n.xp), exm = d(q.xm, n.xm), eyp = d(q.yp, n.yp), eym = d(q.ym, n.ym);
    const float ezp = d(q.zp, n.zp), ezm = d(q.zm, n.zm);
    if (!ANISO) {
        return a.c_iso * (((exp_ + exm) + (eyp + eym)) + (ezp + ezm));
    }
    const float Dxx = fmaf(a.c_d, f.x * f.x, a.c_perp);
    const float Dyy = fmaf(a.c_d, f.y * f.y, a.c_perp);
    const float Dzz = fmaf(a.c_d, f.z * f.z, a.c_perp);
    const float hx = a.c_dh * f.x;
    const float Dxy = hx * f.y, Dxz = hx * f.z, Dyz = a.c_dh * f.y * f.z;
    float L = Dxx * (exp_ + exm);
    L = fmaf(Dyy, eyp + eym, L);
    L = fmaf(Dzz, ezp + ezm, L);
    if (ANISO == AN_SUMS) {
        float dv = (q.xp && q.xm) ? sd.x * (n.xp - n.xm) : 0.0f;
        if (q.yp && q.ym) dv = fmaf(sd.y, n.yp - n.ym, dv);
        if (q.zp && q.zm) dv = fmaf(sd.z, n.zp - n.zm, dv);
        L = fmaf(a.c_s, dv, L);
    }
    L = fmaf(Dxy, (d(q.pp, n.pp) + d(q.mm, n.mm)) - (d(q.pm, n.pm) + d(q.mp, n.mp)), L);
    L = fmaf(Dxz, (d(q.xpzp, n.xpzp) + d(q.xmzm, n.xmzm)) - (d(q.xpzm, n.xpzm) + d(q.xmzp, n.xmzp)), L);
    L = fmaf(Dyz, (d(q.ypzp, n.ypzp) + d(q.ymzm, n.ymzm)) - (d(q.ypzm, n.ypzm) + d(q.ymzp, n.ymzp)), L);
    return L;
}


// ---------------------------------------------------------------------------
// the fused step kernel
// ---------------------------------------------------------------------------

// The reaction surrogate as the step kernel uses it (built on the device from
// a trained network, bbx_set_surrogate): BF16 weights laid out row-major
// [out][in] as 32-bit pairs (W1 padded to 16 inputs), FP32 biases, the
// normalisation and envelope, and the upstroke threshold.
struct SurrogateData {
    // BF16 pairs in MMA-fragment order: for output row n and lane t (of
    // the 4 lanes sharing a row group), the words holding input columns
    // (2t, 2t+1) and (2t+8, 2t+9) of each 16-wide k-step are adjacent.
    uint32_t W1[64 * 8];   // [64 rows][4 lanes][b0, b1]      (inputs padded to 16)
    uint32_t W2[64 * 32];  // [64 rows][4 lanes][4 k-steps][b0, b1]
    uint32_t W3[8 * 32];   // [8 rows][4 lanes][4 k-steps][b0, b1]
    float b1[64], b2[64], b3[8];
    float norm[48];        // mu_in, sd_in, mu_out, sd_out, lo, hi (8 each)
    float inv_sd_in[8];    // 1 / sd_in
    float v_up;            // the exact model runs where V >= v_up
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ReLU and BF16 packing of two FP32 values in one instruction (lo in the low
// half, as the MMA fragments expect).
__device__ __forceinline__ uint32_t relu_pack_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// The network on the 64 nodes of one warp row (2 per lane) with tensor-core
// MMAs (m16n8k16, BF16 inputs, FP32 accumulation), four m-tiles of 16 nodes.
// Hidden activations stay in registers: the accumulators of two adjacent
// 8-column tiles are the A fragment of the next layer's 16-wide k-tile.  The
// accumulators start from the bias, ReLU and BF16 packing are one instruction
// per pair, and each lane's B fragments are stored contiguously
// (k_build_surrogate), one 64- or 128-bit load per MMA or pair of MMAs.
// wbuf: this warp's 2 KB of shared memory (64 rows of 32 bytes), first the
// BF16 inputs of a row, then, row by row, its 8 FP32 outputs.  All 32 lanes
// must call it.  s: the two nodes' raw states; d: their raw increments.
__device__ __forceinline__ void surrogate_warp64(const SurrogateData* __restrict__ W, unsigned char* wbuf,
                                                 const float (*s)[8], float (*d)[8]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float* nrm = W->norm;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        uint32_t* row = reinterpret_cast<uint32_t*>(wbuf + (lane * 2 + e) * 32);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            row[k] = pack_bf16((s[e][2 * k] - nrm[2 * k]) * W->inv_sd_in[2 * k],
                               (s[e][2 * k + 1] - nrm[2 * k + 1]) * W->inv_sd_in[2 * k + 1]);
#pragma unroll
        for (int k = 4; k < 8; ++k) row[k] = 0u;
    }
    __syncwarp();
    const uint2* W1 = reinterpret_cast<const uint2*>(W->W1);  // [row][lane t]: (b0, b1)
    const uint4* W2 = reinterpret_cast<const uint4*>(W->W2);  // [row][lane t][kk pair]: (b0, b1, b0', b1')
    const uint4* W3 = reinterpret_cast<const uint4*>(W->W3);
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        uint32_t* X = reinterpret_cast<uint32_t*>(wbuf + q * 16 * 32);
        uint32_t a[4] = {X[g * 8 + t], X[(g + 8) * 8 + t], X[g * 8 + t + 4], X[(g + 8) * 8 + t + 4]};
        __syncwarp();  // every lane holds its fragment before the rows are overwritten
        uint32_t h[4][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 bias = *reinterpret_cast<const float2*>(W->b1 + 8 * j + 2 * t);
            float c[4] = {bias.x, bias.y, bias.x, bias.y};
            const uint2 b = W1[(8 * j + g) * 4 + t];
            mma_bf16(c, a, b.x, b.y);
            const uint32_t lo = relu_pack_bf16(c[0], c[1]), hi = relu_pack_bf16(c[2], c[3]);
            if (j & 1) { h[j >> 1][2] = lo; h[j >> 1][3] = hi; }
            else { h[j >> 1][0] = lo; h[j >> 1][1] = hi; }
        }
        uint32_t h2[4][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 bias = *reinterpret_cast<const float2*>(W->b2 + 8 * j + 2 * t);
            float c[4] = {bias.x, bias.y, bias.x, bias.y};
            const uint4 b01 = W2[((8 * j + g) * 4 + t) * 2], b23 = W2[((8 * j + g) * 4 + t) * 2 + 1];
            mma_bf16(c, h[0], b01.x, b01.y);
            mma_bf16(c, h[1], b01.z, b01.w);
            mma_bf16(c, h[2], b23.x, b23.y);
            mma_bf16(c, h[3], b23.z, b23.w);
            const uint32_t lo = relu_pack_bf16(c[0], c[1]), hi = relu_pack_bf16(c[2], c[3]);
            if (j & 1) { h2[j >> 1][2] = lo; h2[j >> 1][3] = hi; }
            else { h2[j >> 1][0] = lo; h2[j >> 1][1] = hi; }
        }
        const float2 b3 = *reinterpret_cast<const float2*>(W->b3 + 2 * t);
        float c[4] = {b3.x, b3.y, b3.x, b3.y};
        const uint4 b01 = W3[(g * 4 + t) * 2], b23 = W3[(g * 4 + t) * 2 + 1];
        mma_bf16(c, h2[0], b01.x, b01.y);
        mma_bf16(c, h2[1], b01.z, b01.w);
        mma_bf16(c, h2[2], b23.x, b23.y);
        mma_bf16(c, h2[3], b23.z, b23.w);
        float* Y = reinterpret_cast<float*>(X);
        *reinterpret_cast<float2*>(Y + g * 8 + 2 * t) = make_float2(c[0], c[1]);
        *reinterpret_cast<float2*>(Y + (g + 8) * 8 + 2 * t) = make_float2(c[2], c[3]);
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float4* y = reinterpret_cast<const float4*>(wbuf + (lane * 2 + e) * 32);
        const float4 y0 = y[0], y1 = y[1];
        const float yy[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) d[e][k] = fmaf(yy[k], nrm[24 + k], nrm[16 + k]);
    }
    __syncwarp();  // the buffer is reused by the next row
}

// Per-piece context, written into a shared ring by the producer warp when it
// issues the piece's first plane load, and read by the consumer warps once
// that load has landed (the mbarrier orders the two).
struct PieceSlot : Coef {
    int x0, y0, z0, z1;
    int nx, ny, nz, px;
    long long plane, vol;
    float* dst;
    uint16_t* dst16;  // the 16-bit gates of the buffer written (nullptr: all variables 32-bit)
    int32_t* act;
    const uint8_t* stim;
    float stim_amp, dt, theta;
    int step_next;
    int split, rk4;
    const SurrogateData* surr;  // nullptr: exact reaction everywhere
    const float4* tab;          // V-table of the model, or nullptr
    float mp[8];
};
static_assert(sizeof(PieceSlot) <= 176, "piece ring slot size");


// Barrier over the consumer warps only (named barrier 1), returning the OR of
// a per-thread predicate.
__device__ __forceinline__ bool consumers_sync_or(bool p, int nthreads) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, 1, %2, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void consumers_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// First row of the tile of load off of a piece: a 3D piece keeps its tile
// (pc.y); a sheet's piece is a run of tile rows pc.z .. pc.w of a column.
template <bool PLANAR, int TY>
__device__ __forceinline__ int tile_row_of(int4 pc, int off) {
    return PLANAR ? (pc.z + off) * TY : pc.y;
}

// Warp-specialised step kernel: warps 0..RY-1 compute (2 x CY nodes per
// thread), warp RY is the producer.
//
// GEN: the variant that honours the per-grid scheme and solver settings (Lie
// splitting, RK4 kinetics); the default variant (unsplit, Euler/Rush-Larsen)
// carries no code for them.
//
// PLANAR (grids with nz = 1): a piece is a run of tiles down one column of
// the sheet, pieces[i] = (x0, -, first tile, end tile); each stage holds one
// tile with its one-row halo and the consumers march along y.  The z
// neighbours of a plane are the plane itself (the previous and next stage
// pointers alias the current one): every z term of the stencil is then zero
// (faces and edges exactly, the W-tilde divergence up to rounding), which is
// the 5-point (isotropic) or 9-point (anisotropic) sheet operator.  Stage slots cycle through two mbarrier
// rings: full[s] completes when the plane's bulk copies have landed, empty[s]
// when all RY consumer warps are done with the plane.  No CTA-wide barrier is
// taken per plane.
template <int MODEL, bool MASKED, int ANISO, int TY, bool SURR = false, bool PLANAR = false, bool GEN = false,
          int GATES = GATES_F32>
__global__ void __launch_bounds__(32 * rows_of_threads(TY) + 32, ctas_per_sm(MASKED, ANISO != AN_ISO, TY, SURR))
step_kernel(const __grid_constant__ LaunchArgs L) {
    using P = Plan<MODEL, MASKED, ANISO, TY, SURR, GATES>;
    static_assert(GATES == GATES_F32 || (MODEL == BBX_BR && !SURR), "16-bit gates: Beeler-Reuter without surrogate");
    constexpr int NG = P::NG, S32 = P::S - NG;  // 16-bit variables last
    constexpr int S = P::S, TX = P::TX, UW = P::UW, MW = P::MW, CY = P::CY;
    constexpr int NS = P::NA;            // ring A: loaded planes
    constexpr int NB = P::NB;            // ring B: computed planes (0: nothing beyond V and the mask)
    constexpr bool HB = P::HAS_B;
    constexpr int NCW = P::RY;  // consumer warps
    constexpr int NCT = 32 * NCW;        // consumer threads
    static_assert(TX == 64, "pair mapping assumes 64-node rows");
    constexpr int CB = TX * TY;  // component stride in a ring-B stage

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    unsigned char* bstages = smem + NS * P::A_STAGE;    // ring B
    unsigned char* wbufs = bstages + NB * P::B_STAGE;   // surrogate buffers (SURR only)
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + P::BAR_OFF);
    uint64_t* empty = full + NS;
    uint64_t* fullb = empty + NS;
    uint64_t* emptyb = fullb + NB;
    PieceSlot* ring = reinterpret_cast<PieceSlot*>(emptyb + NB);
    __shared__ double red_scratch[32];
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid / 32, lane = tid % 32;

    // W-tilde sums that vanish at every node of the grid (a fibre field whose
    // tensor does not change along the directions the sums difference, e.g.
    // fibres in the x-y plane turning with z only, or uniform fibres), in a
    // variant that keeps them (masked grids, the general, surrogate and
    // 16-bit-gate kernels; unmasked plain kernels run AN_NO_SUMS instead): a
    // single-grid launch does not copy them, and their part of every ring-B
    // stage holds zeros for the whole launch, so the arithmetic is unchanged
    // and the result is bitwise the one with the sums loaded.  (Batch launches
    // share stages between grids and always copy them.)
    const bool skip_d = ANISO == AN_SUMS && L.single && L.t0.wsum_zero;
    if (skip_d) {
        for (int s = 0; s < NB; ++s) {
            float4* zd = reinterpret_cast<float4*>(bstages + s * P::B_STAGE + P::D_OFF);
            for (int i = tid; i < P::D_RAW / 16; i += P::THREADS) zd[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    const uint32_t b_bytes = skip_d ? P::B_BYTES - P::D_RAW : P::B_BYTES;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        for (int s = 0; s < NB; ++s) {
            mbar_init(&fullb[s], 1);
            mbar_init(&emptyb[s], NCW);
        }
        abort_flag = 0;
        mbar_init_fence();
    }
    __syncthreads();
    // Programmatic dependent launch: the next step's grid may be scheduled from
    // here on (its CTAs take the SMs this grid's CTAs leave), and every thread
    // waits until the previous grid on the stream has completed and its writes
    // are visible before it touches memory that grid wrote (state, t, n,
    // parity, activation map); with no such grid the wait returns at once.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    const int piece_begin = blockIdx.x * L.cta_stride, piece_end = piece_begin + L.cta_count[blockIdx.x];
    int issued = 0;   // producer lane 0: plane loads issued (ring A)
    int issuedb = 0;  // producer lane 0: computed planes issued (ring B)

    if (warp == NCW) {
        // ---------------- producer warp ----------------
        if (lane == 0) {
            bool stop = false;
            int lp = 0;
            // the loads the first plane waits for, issued together: the first
            // piece (its slot always exists) and, for one grid, its t, n, parity
            int4 pc_next = L.pieces[piece_begin];
            TissueDyn d0 = {};
            bool ticketed = !L.single;  // a single-grid launch takes one start ticket per CTA
            if (L.single) {
                const TissueDyn* D = L.t0.dyn;
                d0.t = D->t;
                d0.n = D->n;
                d0.cur = D->cur;
            }
            // Single-grid launch of an unmasked grid with a known parity: the
            // first piece from the schedule's shape and its first plane copies
            // (three planes; two tile rows of a sheet) issued now, expected on
            // their barriers but not yet arrived on (the arrival follows the
            // piece context, below).
            // ring B copies of the computed plane z (tile rows from y0) of grid T
            auto load_b = [&](const TissueArgs* T, int src, int x0, int y0, int z, int bslot, uint64_t* bar) {
                unsigned char* sb = bstages + bslot * P::B_STAGE;
                if (ANISO) {
                    tma_load_4d(sb + P::F_OFF, &T->tm_f, x0 + 4, y0, z, 0, bar);  // fibres stored from x = -4
                    if (ANISO == AN_SUMS && !skip_d) tma_load_4d(sb + P::D_OFF, &T->tm_d, x0, y0, z, 0, bar);
                }
                if (S > 1 && S32 > 1) tma_load_4d(sb + P::S_OFF, &T->tm_s[src], x0, y0, z, 1, bar);
                if (NG) tma_load_4d(sb + P::G_OFF, &T->tm_g[src], x0, y0, z, 0, bar);
            };
            bool early = false;
            int n_early = 0;
            int4 pc_early = make_int4(0, 0, 0, 0);
            if (L.single && L.cur_hint >= 0 && L.reg_len > 0 && !L.poison_first_load) {
                const long long p0 = (long long)blockIdx.x * L.reg_planes / L.reg_ctas;
                const long long p1 = ((long long)blockIdx.x + 1) * L.reg_planes / L.reg_ctas;
                if (p1 > p0) {
                    const int col = (int)(p0 / L.reg_len), z0 = L.reg_z0 + (int)(p0 % L.reg_len);
                    const int z1 = (int)min((long long)(L.reg_z0 + L.reg_len), z0 + (p1 - p0));
                    pc_early = make_int4((col % L.reg_nbx) * TX, (col / L.reg_nbx) * L.reg_ty, z0, z1);
                    early = true;
                    const TissueArgs* T = &L.t0;
                    const int src = L.cur_hint;
                    const int nl = PLANAR ? z1 - z0 : z1 - z0 + 2;
                    n_early = PLANAR ? min(nl, 2) : 3;  // (3D: at most 2 computed planes; NB >= 2)
                    if (HB && PLANAR && n_early > NB) n_early = NB;
#pragma unroll 1
                    for (int off = 0; off < n_early; ++off) {
                        const int z = PLANAR ? 0 : z0 - 1 + off;
                        if (z < 0 || z >= T->nz) continue;
                        const int y0 = tile_row_of<PLANAR, TY>(pc_early, off);
                        uint64_t* bar = &full[off];
                        unsigned char* st = smem + off * P::A_STAGE;
                        const bool halo = !PLANAR && ((off == 0) || (off == nl - 1));
                        mbar_expect_tx(bar, P::A_BYTES);
                        tma_load_3d(st + P::U_OFF, &T->tm_u[src], pc_early.x - 4, y0 - 1, z, bar);
                        if (MASKED) tma_load_3d(st + P::M_OFF, &T->tm_m, pc_early.x - 16, y0 - 1, z, bar);
                        if (HB && !halo) {  // computed plane b = off - 1 (3D) or off (sheet): slot b
                            const int b = PLANAR ? off : off - 1;
                            mbar_expect_tx(&fullb[b], b_bytes);
                            load_b(T, src, pc_early.x, y0, z, b, &fullb[b]);
                        }
                    }
                }
            }
            if (L.single && L.cur_hint >= 0 &&
                (d0.cur != L.cur_hint ||
                 (early && (pc_early.x != pc_next.x || pc_early.y != pc_next.y || pc_early.z != pc_next.z ||
                            pc_early.w != pc_next.w))))
                atomicOr(L.err, ERRBIT_HINT);
            for (int pi = piece_begin; pi < piece_end && !stop; ++pi, ++lp) {
                const int4 pc = pc_next;
                if (pi + 1 < piece_end) pc_next = L.pieces[pi + 1];
                const TissueArgs* T = L.single ? &L.t0 : L.tissues + L.piece_tissue[pi];
                const TissueDyn* D = T->dyn;
                const int src = L.single ? (L.cur_hint >= 0 ? L.cur_hint : d0.cur) : D->cur;
                const int nz = T->nz;
                const int nload = PLANAR ? pc.w - pc.z : pc.w - pc.z + 2;
                for (int off = 0; off < nload; ++off) {
                    const int slot = issued % NS;
                    const bool comp = PLANAR || (off >= 1 && off <= pc.w - pc.z);  // a computed plane: ring B too
                    const int bslot = NB ? issuedb % NB : 0;
                    if (!ticketed && issued == NS) {
                        // the ring is full: the ticket's round trip overlaps the copies
                        start_ticket(L, d0);
                        ticketed = true;
                    }
                    if (L.poison_first_load && blockIdx.x == 0 && issued == 0) {
                        // fault injection: wait for an empty-slot phase that no
                        // consumer completes; the bounded wait runs out
                        (void)mbar_wait_bounded(&empty[slot], 0, L.wait_limit);
                        stop = true;
                    } else if (issued >= NS &&
                               !mbar_wait_bounded(&empty[slot], ((issued / NS) - 1) & 1, L.wait_limit)) {
                        stop = true;
                    } else if (HB && comp && issuedb >= NB &&
                               !mbar_wait_bounded(&emptyb[bslot], ((issuedb / NB) - 1) & 1, L.wait_limit)) {
                        stop = true;
                    }
                    if (stop || abort_flag) {
                        stop = true;
                        break;
                    }
                    if (off == 0) {
                        PieceSlot& r = ring[lp % NS];
                        const double tn = L.single ? d0.t : D->t;
                        r.x0 = pc.x; r.y0 = pc.y; r.z0 = pc.z; r.z1 = pc.w;
                        r.nx = T->nx; r.ny = T->ny; r.nz = nz; r.px = T->px;
                        r.plane = T->plane; r.vol = T->vol;
                        r.dst = T->state[src ^ 1];
                        r.dst16 = T->gate16[src ^ 1];
                        r.act = T->act;
                        r.stim = T->stim;
                        r.stim_amp = (T->stim && T->stim_amp != 0.0f && tn >= T->t_on && tn < T->t_off) ? T->stim_amp
                                                                                                       : 0.0f;
                        r.dt = T->dt;
                        r.theta = T->theta;
                        r.step_next = (int)((L.single ? d0.n : D->n) + 1);
                        r.split = T->split;
                        r.rk4 = T->rk4;
                        r.c_perp = T->c_perp; r.c_d = T->c_d; r.c_dh = T->c_dh; r.c_s = T->c_s; r.c_iso = T->c_iso;
                        r.surr = T->surr;
                        r.tab = T->tab;
#pragma unroll
                        for (int i = 0; i < 8; ++i) r.mp[i] = T->mp[i];
                    }
                    const int z = PLANAR ? 0 : pc.z - 1 + off;
                    const int y0 = tile_row_of<PLANAR, TY>(pc, off);  // first row of the tile
                    uint64_t* bar = &full[slot];
                    unsigned char* st = smem + slot * P::A_STAGE;
                    if (early && lp == 0 && off < n_early) {
                        mbar_arrive(bar);  // its copies were issued at the start
                        if (HB && comp) mbar_arrive(&fullb[bslot]);
                    } else if (z < 0 || z >= nz) {
                        mbar_arrive(bar);  // plane outside the array: nothing to load (never a computed one)
                    } else {
                        mbar_arrive_expect_tx(bar, P::A_BYTES);
                        tma_load_3d(st + P::U_OFF, &T->tm_u[src], pc.x - 4, y0 - 1, z, bar);
                        if (MASKED) tma_load_3d(st + P::M_OFF, &T->tm_m, pc.x - 16, y0 - 1, z, bar);
                        if (HB && comp) {
                            mbar_arrive_expect_tx(&fullb[bslot], b_bytes);
                            load_b(T, src, pc.x, y0, z, bslot, &fullb[bslot]);
                        }
                    }
                    ++issued;
                    if (HB && comp) ++issuedb;
                }
            }
            if (!ticketed) start_ticket(L, d0);  // every CTA takes it, also on a short or aborted run
            if (stop) abort_flag = 1;
        }
        __syncwarp();
    } else {
        // ---------------- consumer warps ----------------
        const int tx = tid % 32, row0 = (tid / 32) * CY;  // node pair (x, x+1) = x0 + 2 tx
        F2 vsum = {0.0f, 0.0f};
        bool timed_out = false;
        int jb = 0, lp = 0;  // load index of the first plane of the piece, local piece index
        int sb = 0, pb = 0;  // ring B: slot and phase parity of the next computed plane
        auto wait_bar = [&](uint64_t* bar, int parity) {
            if (timed_out || abort_flag) {
                timed_out = true;
                return;
            }
            if (!mbar_wait_bounded(bar, parity, L.wait_limit)) {
                timed_out = true;
                abort_flag = 1;
            }
        };
        auto wait_slot = [&](int slot, int parity) { wait_bar(&full[slot], parity); };
        auto wait_full = [&](int j) { wait_slot(j % NS, (j / NS) & 1); };
        for (int pi = piece_begin; pi < piece_end; ++pi, ++lp) {
            wait_full(jb);  // the piece's first load carries its context
            const PieceSlot& a = ring[lp % NS];  // read from shared memory where used
            const float* mp = a.mp;
            const float theta = a.theta;
            int4 pc = make_int4(a.x0, a.y0, a.z0, a.z1);
            if (timed_out) pc.w = pc.z = 0;  // context unreliable: compute nothing
            const int x = pc.x + 2 * tx;  // first node of this thread's pair
            const bool x_in = x < a.nx && !timed_out;  // (folded into the per-node flags)
            const int ncomp = pc.w - pc.z;
            if (!PLANAR) wait_full(jb + 1);
            // stage slots of loads jb + t (sp), jb + t + 1 (sc), jb + t + 2 (sn)
            // and the slot and phase parity of the next load to wait for,
            // advanced per plane without divisions
            int sp = jb % NS;
            int sc = sp + 1 == NS ? 0 : sp + 1;
            int sn = sc + 1 == NS ? 0 : sc + 1;
            const int jw = jb + (PLANAR ? 1 : 2);
            int sw = jw % NS, pw = (jw / NS) & 1;
            for (int t = 0; t < ncomp; ++t) {
                if (!PLANAR || t > 0) {
                    wait_slot(sw, pw);
                    if (++sw == NS) {
                        sw = 0;
                        pw ^= 1;
                    }
                }
                if (HB) wait_bar(&fullb[sb], pb);  // the plane's own fibres, W-tilde sums, other variables
                const int k = PLANAR ? 0 : pc.z + t;
                const int yb = (PLANAR ? (pc.z + t) * TY : pc.y) + row0;  // y of this thread's first row
                const unsigned char* stc = smem + (PLANAR ? sp : sc) * P::A_STAGE;
                const unsigned char* stp = PLANAR ? stc : smem + sp * P::A_STAGE;
                const unsigned char* stn = PLANAR ? stc : smem + sn * P::A_STAGE;
                const unsigned char* stb = bstages + sb * P::B_STAGE;
                const float* Up = reinterpret_cast<const float*>(stp + P::U_OFF);
                const float* Uc = reinterpret_cast<const float*>(stc + P::U_OFF);
                const float* Un = reinterpret_cast<const float*>(stn + P::U_OFF);
                const float* Fb = reinterpret_cast<const float*>(stb + P::F_OFF);  // [3][TY][TX]
                const float* Db = reinterpret_cast<const float*>(stb + P::D_OFF);  // [3][TY][TX]
                const unsigned char* Mp = stp + P::M_OFF;
                const unsigned char* Mc = stc + P::M_OFF;
                const unsigned char* Mn = stn + P::M_OFF;
                const float* Sv = reinterpret_cast<const float*>(stb + P::S_OFF);
                const bool zn_ok = k + 1 < a.nz, zp_ok = k > 0;
                const int c0 = (row0 + 1) * UW + (2 * tx + 4);   // stage index of node (x, yb), even
                const int m0 = (row0 + 1) * MW + (2 * tx + 16);  // mask index of node (x, yb)
    
                {
                    auto ld2 = [&](const float* U, int o) { return *reinterpret_cast<const float2*>(U + o); };
                    const bool x1_in = x + 1 < a.nx;
                    // psi of the x neighbours of the two nodes (unmasked grids)
                    const float px0 = x1_in ? 1.0f : 0.0f, mx0 = (x > 0) ? 1.0f : 0.0f;
                    const float px1 = (x + 2 < a.nx) ? 1.0f : 0.0f, mx1 = 1.0f;
    
                    // phase 1: the stencil for the 2 x CY nodes of this thread.
                    // Sliding window down the rows: plane k at x-2..x+3 (three
                    // float2), own pair of planes k+-1, own pair of fibres.
                    float Lr[CY][2], u0r[CY][2];
                    bool live[CY][2];
                    float2 wA[3], wB[3], wC[3], wN[3], wP[3];
    #pragma unroll
                    for (int w = 0; w < 2; ++w) {
                        const int o = c0 + (w - 1) * UW;
                        wA[w] = ld2(Uc, o - 2); wB[w] = ld2(Uc, o); wC[w] = ld2(Uc, o + 2);
                        wN[w] = ld2(Un, o); wP[w] = ld2(Up, o);
                    }
    #pragma unroll
                    for (int r = 0; r < CY; ++r) {
                        const int y = yb + r;
                        const int c = c0 + r * UW;
                        const int m = m0 + r * MW;
                        {
                            const int o = c + UW;  // row r+1
                            wA[2] = ld2(Uc, o - 2); wB[2] = ld2(Uc, o); wC[2] = ld2(Uc, o + 2);
                            wN[2] = ld2(Un, o); wP[2] = ld2(Up, o);
                        }
                        bool tis[2] = {x_in && y < a.ny, x_in && y < a.ny && x1_in}, intr[2];
                        if (MASKED) {
                            const unsigned char mc0 = Mc[m], mc1 = Mc[m + 1];
                            tis[0] = tis[0] && (mc0 & MASK_TISSUE);
                            tis[1] = tis[1] && (mc1 & MASK_TISSUE);
                            intr[0] = (mc0 & MASK_INTERIOR) != 0;
                            intr[1] = (mc1 & MASK_INTERIOR) != 0;
                        } else {
                            intr[0] = intr[1] = (y > 0) && (y + 1 < a.ny) && (PLANAR || (zp_ok && zn_ok));  // warp-uniform
                        }
                        Nb n[2];
                        F3 f[2], sd[2];
                        n[0].u0 = wB[1].x; n[0].xp = wB[1].y; n[0].xm = wA[1].y;
                        n[0].yp = wB[2].x; n[0].ym = wB[0].x; n[0].zp = wN[1].x; n[0].zm = wP[1].x;
                        n[1].u0 = wB[1].y; n[1].xp = wC[1].x; n[1].xm = wB[1].x;
                        n[1].yp = wB[2].y; n[1].ym = wB[0].y; n[1].zp = wN[1].y; n[1].zm = wP[1].y;
                        if (ANISO) {
                            const float2 nA = ld2(Un, c - 2), nC = ld2(Un, c + 2);
                            const float2 pA = ld2(Up, c - 2), pC = ld2(Up, c + 2);
                            n[0].pp = wB[2].y; n[0].mm = wA[0].y; n[0].pm = wB[0].y; n[0].mp = wA[2].y;
                            n[0].xpzp = wN[1].y; n[0].xmzm = pA.y; n[0].xpzm = wP[1].y; n[0].xmzp = nA.y;
                            n[0].ypzp = wN[2].x; n[0].ymzm = wP[0].x; n[0].ypzm = wP[2].x; n[0].ymzp = wN[0].x;
                            n[1].pp = wC[2].x; n[1].mm = wB[0].x; n[1].pm = wC[0].x; n[1].mp = wB[2].x;
                            n[1].xpzp = nC.x; n[1].xmzm = wP[1].x; n[1].xpzm = pC.x; n[1].xmzp = wN[1].x;
                            n[1].ypzp = wN[2].y; n[1].ymzm = wP[0].y; n[1].ypzm = wP[2].y; n[1].ymzp = wN[0].y;
                            // the pair's own fibres and W-tilde sums ([comp][row][x] in ring B)
                            const int bo = (row0 + r) * TX + 2 * tx;
                            const float2 fx = ld2(Fb, bo), fy = ld2(Fb + CB, bo), fz = ld2(Fb + 2 * CB, bo);
                            f[0] = F3{fx.x, fy.x, fz.x};
                            f[1] = F3{fx.y, fy.y, fz.y};
                            if (ANISO == AN_SUMS) {
                                const float2 dx = ld2(Db, bo), dy = ld2(Db + CB, bo), dz = ld2(Db + 2 * CB, bo);
                                sd[0] = F3{dx.x, dy.x, dz.x};
                                sd[1] = F3{dx.y, dy.y, dz.y};
                            } else {
                                sd[0] = sd[1] = F3{0.f, 0.f, 0.f};
                            }
                        } else {
    #pragma unroll
                            for (int e = 0; e < 2; ++e) f[e] = sd[e] = F3{0.f, 0.f, 0.f};
                        }
    #pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            live[r][e] = tis[e];
                            u0r[r][e] = n[e].u0;
                            // fast formula for every node (values of void or
                            // out-of-array nodes are finite and never stored) ...
                            if (MASKED)
                                Lr[r][e] = lap_interior<ANISO>(a, n[e], f[e], sd[e]);
                            else
                                Lr[r][e] = lap_xbound<ANISO>(a, n[e], e ? px1 : px0, e ? mx1 : mx0, f[e], sd[e]);
                        }
                        // ... and the general one where a y/z neighbour (or, in a
                        // masked grid, any neighbour) may be void: rare, and
                        // warp-uniform on unmasked grids
                        if (!((intr[0] || !tis[0]) && (intr[1] || !tis[1]))) {
    #pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                if (!tis[e] || intr[e]) continue;
                                const int xe = x + e, me = m + e;
                                Psi q;
                                if (MASKED) {
                                    q.xp = Mc[me + 1] != 0; q.xm = Mc[me - 1] != 0;
                                    q.yp = Mc[me + MW] != 0; q.ym = Mc[me - MW] != 0;
                                    q.zp = zn_ok && Mn[me] != 0; q.zm = zp_ok && Mp[me] != 0;
                                    q.pp = Mc[me + MW + 1] != 0; q.mm = Mc[me - MW - 1] != 0;
                                    q.pm = Mc[me - MW + 1] != 0; q.mp = Mc[me + MW - 1] != 0;
                                    q.xpzp = zn_ok && Mn[me + 1] != 0; q.xmzm = zp_ok && Mp[me - 1] != 0;
                                    q.xpzm = zp_ok && Mp[me + 1] != 0; q.xmzp = zn_ok && Mn[me - 1] != 0;
                                    q.ypzp = zn_ok && Mn[me + MW] != 0; q.ymzm = zp_ok && Mp[me - MW] != 0;
                                    q.ypzm = zp_ok && Mp[me + MW] != 0; q.ymzp = zn_ok && Mn[me - MW] != 0;
                                } else {
                                    const bool xp = xe + 1 < a.nx, xm = xe > 0, yp = y + 1 < a.ny, ym = y > 0;
                                    q.xp = xp; q.xm = xm; q.yp = yp; q.ym = ym; q.zp = zn_ok; q.zm = zp_ok;
                                    q.pp = xp && yp; q.mm = xm && ym; q.pm = xp && ym; q.mp = xm && yp;
                                    q.xpzp = xp && zn_ok; q.xmzm = xm && zp_ok; q.xpzm = xp && zp_ok; q.xmzp = xm && zn_ok;
                                    q.ypzp = yp && zn_ok; q.ymzm = ym && zp_ok; q.ypzm = yp && zp_ok; q.ymzp = ym && zn_ok;
                                }
                                Lr[r][e] = lap_general<ANISO>(a, n[e], q, f[e], sd[e]);
                            }
                        }
                        // slide the window down one row
                        wA[0] = wA[1]; wA[1] = wA[2]; wB[0] = wB[1]; wB[1] = wB[2]; wC[0] = wC[1]; wC[1] = wC[2];
                        wN[0] = wN[1]; wN[1] = wN[2]; wP[0] = wP[1]; wP[1] = wP[2];
                    }
    
                    // phase 2: reaction, stores, activation, tissue sum (predicated)
                    const bool stim_on = a.stim_amp != 0.0f;
    #pragma unroll
                    for (int r = 0; r < CY; ++r) {
                        const int y = yb + r;
                        const long long gi = (long long)k * a.plane + (long long)y * a.px + x;  // even
                        float yv[2][S];
    #pragma unroll
                        for (int e = 0; e < 2; ++e) yv[e][0] = u0r[r][e];
    #pragma unroll
                        for (int v = 1; v < S32; ++v) {
                            const float2 sv = *reinterpret_cast<const float2*>(Sv + (v - 1) * TX * TY + (row0 + r) * TX + 2 * tx);
                            yv[0][v] = sv.x;
                            yv[1][v] = sv.y;
                        }
    #pragma unroll
                        for (int v = S32; v < S; ++v) {  // 16-bit gates, decoded to FP32
                            const uint32_t w = *reinterpret_cast<const uint32_t*>(
                                stb + P::G_OFF + 2 * ((v - S32) * TX * TY + (row0 + r) * TX + 2 * tx));
                            const float2 gv = gate_decode2<GATES>(w);
                            yv[0][v] = gv.x;
                            yv[1][v] = gv.y;
                        }
                            float Isr[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            Isr[e] = 0.0f;
                            if (stim_on && live[r][e] && a.stim[gi + e]) Isr[e] = a.stim_amp;
                        }
                        if (GEN && a.split) {
                            // Lie splitting: the diffusion substep on its own, then
                            // the kinetics step from the half-step voltage
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                yv[e][0] += a.dt * Lr[r][e];
                                Lr[r][e] = 0.0f;
                            }
                        }
                        if constexpr (SURR && MODEL == BBX_BR) {
                            // the surrogate where the state is inside the training
                            // envelope and V below the upstroke threshold; the
                            // exact model elsewhere
                            const SurrogateData* W = a.surr;
                            bool want[2] = {false, false};
                            if (W) {
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    bool in = live[r][e] && yv[e][0] < W->v_up;
#pragma unroll
                                    for (int v = 0; v < S; ++v)
                                        in = in && yv[e][v] >= W->norm[32 + v] && yv[e][v] <= W->norm[40 + v];
                                    want[e] = in;
                                }
                            }
                            if (__any_sync(0xffffffffu, want[0] || want[1])) {
                                float dsur[2][8];
                                surrogate_warp64(W, wbufs + (tid >> 5) * 2048, yv, dsur);
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    if (want[e]) {
#pragma unroll
                                        for (int v = 0; v < S; ++v) yv[e][v] += dsur[e][v];
                                        yv[e][0] += a.dt * (Lr[r][e] + Isr[e]);
                                    } else {
                                        Model<MODEL>::update(mp, yv[e], Lr[r][e], Isr[e], a.dt);
                                    }
                                }
                            } else {
#pragma unroll
                                for (int e = 0; e < 2; ++e) Model<MODEL>::update(mp, yv[e], Lr[r][e], Isr[e], a.dt);
                            }
                        } else if constexpr (MODEL != BBX_BR && GEN) {
                            if (a.rk4) {
#pragma unroll
                                for (int e = 0; e < 2; ++e) rk4_update<MODEL>(mp, yv[e], Lr[r][e], Isr[e], a.dt);
                            } else {
#pragma unroll
                                for (int e = 0; e < 2; ++e) Model<MODEL>::update(mp, yv[e], Lr[r][e], Isr[e], a.dt);
                            }
                        } else if constexpr (MODEL == BBX_BR_MRL || MODEL == BBX_BR_FCA) {
#pragma unroll
                            for (int e = 0; e < 2; ++e)
                                Model<MODEL>::update_tab(mp, a.tab, yv[e], Lr[r][e], Isr[e], a.dt);
                        } else if constexpr (MODEL == BBX_BR && GEN) {
                            // tabulated Rush-Larsen coefficients (the general
                            // variants only, so the default kernel is unchanged)
                            if (a.tab) {
#pragma unroll
                                for (int e = 0; e < 2; ++e)
                                    Model<MODEL>::update_tab(mp, a.tab, yv[e], Lr[r][e], Isr[e], a.dt);
                            } else {
#pragma unroll
                                for (int e = 0; e < 2; ++e) Model<MODEL>::update(mp, yv[e], Lr[r][e], Isr[e], a.dt);
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 2; ++e) Model<MODEL>::update(mp, yv[e], Lr[r][e], Isr[e], a.dt);
                        }
                        if (live[r][0] && live[r][1]) {
    #pragma unroll
                            for (int v = 0; v < S32; ++v)
                                st_global(a.dst + (long long)v * a.vol + gi, make_float2(yv[0][v], yv[1][v]));
    #pragma unroll
                            for (int v = S32; v < S; ++v)
                                st_global_u32(a.dst16 + (long long)(v - S32) * a.vol + gi,
                                              gate_encode2<GATES>(yv[0][v], yv[1][v]));
                        } else if (live[r][0] || live[r][1]) {
    #pragma unroll
                            for (int e = 0; e < 2; ++e)
                                if (live[r][e]) {
    #pragma unroll
                                    for (int v = 0; v < S32; ++v) st_global(a.dst + (long long)v * a.vol + gi + e, yv[e][v]);
    #pragma unroll
                                    for (int v = S32; v < S; ++v)
                                        st_global_u16(a.dst16 + (long long)(v - S32) * a.vol + gi + e,
                                                      gate_encode<GATES>(yv[e][v]));
                                }
                        }
    #pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            if (live[r][e] && u0r[r][e] < theta && theta <= yv[e][0]) {
                                if (a.act[gi + e] == BBX_ACT_NONE) a.act[gi + e] = a.step_next;
                            }
                            two_sum_add(vsum, live[r][e] ? yv[e][0] : 0.0f);
                        }
                    }
                }
    
                    __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&empty[sp]);
                    if (HB) mbar_arrive(&emptyb[sb]);
                }
                if (HB && ++sb == NB) {
                    sb = 0;
                    pb ^= 1;
                }
                sp = sc;
                sc = sn;
                sn = sn + 1 == NS ? 0 : sn + 1;
            }
            __syncwarp();
            if (!PLANAR && lane == 0) {
                // release the piece's last two planes (or all of a piece cut short)
                for (int j = jb + (ncomp > 0 ? ncomp : 0); j < jb + (ncomp > 0 ? ncomp + 2 : 2); ++j)
                    mbar_arrive(&empty[j % NS]);
            }
            jb += (ncomp > 0 ? ncomp : 0) + (PLANAR ? 0 : 2);
            // per-piece partial of the tissue sum, and a vote on timeouts
            double v = (double)vsum.hi + (double)vsum.lo;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red_scratch[warp] = v;
            const bool any_to = consumers_sync_or(timed_out, NCT);
            if (tid == 0) {
                double s = 0.0;
                for (int w = 0; w < NCW; ++w) s += red_scratch[w];
                L.partials[pi] = s;
                if (!isfinite(s)) atomicOr(L.err, ERRBIT_NAN);
            }
            consumers_sync(NCT);
            if (!L.single && warp == 0 && !any_to) grid_piece_done(L, pi, lane);
            vsum.hi = vsum.lo = 0.0f;
            if (any_to) break;
        }
        if (timed_out) abort_flag = 1;
    }
    __syncthreads();

    if (abort_flag && warp == NCW && lane == 0) {
        // Give the loads that may still be in flight a bounded chance to land.
        atomicOr(L.err, ERRBIT_TIMEOUT);
        for (int j = issued > NS ? issued - NS : 0; j < issued; ++j)
            (void)mbar_wait_bounded(&full[j % NS], (j / NS) & 1, L.wait_limit);
        for (int j = issuedb > NB ? issuedb - NB : 0; j < issuedb; ++j)
            (void)mbar_wait_bounded(&fullb[j % NB], (j / NB) & 1, L.wait_limit);
    }
    step_finalize(L, red_scratch);
}

// host-visible description of one compiled step kernel
struct StepKernel {
    const void* fn;
    int smem;
    int threads;
    int ty;
};

}  // namespace bbx
