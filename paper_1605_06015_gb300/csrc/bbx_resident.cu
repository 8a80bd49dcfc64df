// Resident multi-step kernel for small sheets: a cluster of CTAs holds the
// whole sheet in distributed shared memory and advances many time steps in
// one launch.  Each CTA owns a band of rows; the stencil reads the rows next
// to its band from the neighbouring CTAs' shared memory, and one cluster
// barrier per step separates a step's writes from the next step's reads.
// Nothing goes through global memory between steps except activation events,
// so a step costs neither a launch nor a DRAM round trip: the unsplit step of
// section "Computation of intermediate expressions" with the 5-point
// operator of an isotropic sheet (faces only; no-flux edges: a missing
// neighbour contributes nothing).
#include <cooperative_groups.h>

#include "bbx_device.cuh"

namespace cg = cooperative_groups;

namespace bbx {

namespace {

// CTAs in the cluster: 16 (a non-portable cluster size the launch asks for),
// else the portable 8
constexpr int kResCtasLarge = 16, kResCtasPortable = 8;
constexpr int kResThreads = 1024;
constexpr int kResMaxSmem = 200 * 1024;

__device__ __forceinline__ void res_two_sum(double& hi, double& lo, double b) {
    const double s = hi + b, bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}

// Launched with NC CTAs forming one cluster.  Shared memory per CTA:
// two buffers of the band's V (maxr rows of nx) and S-1 buffers of the other
// variables, updated in place (only V is read by neighbours).
template <int MODEL, int NC>
__global__ void __cluster_dims__(NC, 1, 1) __launch_bounds__(kResThreads, 1)
    k_resident_sheet(const TissueArgs* __restrict__ T, int n_steps, int* __restrict__ err) {
    constexpr int S = Model<MODEL>::S;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    extern __shared__ float sm[];
    __shared__ double red_hi[kResThreads / 32], red_lo[kResThreads / 32];
    __shared__ double cl_part[NC];

    const int nx = T->nx, ny = T->ny, px = T->px;
    const long long vol = T->vol;
    const int maxr = (ny + NC - 1) / NC;
    const int rb0 = (int)((long long)ny * rank / NC), rb1 = (int)((long long)ny * (rank + 1) / NC);
    const int nr = rb1 - rb0;
    const int nb = nr * nx;
    float* V[2] = {sm, sm + maxr * nx};
    float* Wv = sm + 2 * maxr * nx;  // the other variables, (S-1) x maxr x nx
    // the neighbouring bands' V buffers (rows rb0-1 and rb1 live there)
    const int up = rank > 0 ? rank - 1 : rank, dn = rank + 1 < NC ? rank + 1 : rank;
    const int nr_up = rb0 - (int)((long long)ny * up / NC);
    float* Vu[2] = {cl.map_shared_rank(V[0], up), cl.map_shared_rank(V[1], up)};
    float* Vd[2] = {cl.map_shared_rank(V[0], dn), cl.map_shared_rank(V[1], dn)};

    TissueDyn* D = T->dyn;
    const int cur0 = D->cur;
    double t = D->t;
    long long n = D->n;
    const float* src = T->state[cur0];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const int r = i / nx, x = i - r * nx;
        const long long gi = (long long)(rb0 + r) * px + x;
        V[0][i] = src[gi];
#pragma unroll
        for (int v = 1; v < S; ++v) Wv[(v - 1) * maxr * nx + i] = src[v * vol + gi];
    }
    cl.sync();

    const float c = T->c_iso, dt = T->dt, theta = T->theta;
    float mp[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) mp[k] = T->mp[k];
    const int dr = (int)blockDim.x / nx, dx = (int)blockDim.x - dr * nx;
    int p = 0;
    for (int s = 0; s < n_steps; ++s) {
        const bool stim_on = T->stim && T->stim_amp != 0.0f && t >= T->t_on && t < T->t_off;
        const float* Vo = V[p];
        float* Vn = V[p ^ 1];
        const float* Vup = Vu[p];
        const float* Vdn = Vd[p];
        // node i = r nx + x of the band, advanced by blockDim without divisions
        int r = (int)threadIdx.x / nx, x = (int)threadIdx.x - r * nx;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const int y = rb0 + r;
            const float u0 = Vo[i];
            const float xp = x + 1 < nx ? Vo[i + 1] : u0;
            const float xm = x > 0 ? Vo[i - 1] : u0;
            const float ym = r > 0 ? Vo[i - nx] : (y > 0 ? Vup[(nr_up - 1) * nx + x] : u0);
            const float yp = r + 1 < nr ? Vo[i + nx] : (y + 1 < ny ? Vdn[x] : u0);
            const float L = c * (((xp - u0) + (xm - u0)) + ((yp - u0) + (ym - u0)));
            float yv[S];
            yv[0] = u0;
#pragma unroll
            for (int v = 1; v < S; ++v) yv[v] = Wv[(v - 1) * maxr * nx + i];
            const long long gi = (long long)y * px + x;
            const float Is = (stim_on && T->stim[gi]) ? T->stim_amp : 0.0f;
            Model<MODEL>::update(mp, yv, L, Is, dt);
            Vn[i] = yv[0];
#pragma unroll
            for (int v = 1; v < S; ++v) Wv[(v - 1) * maxr * nx + i] = yv[v];
            if (u0 < theta && theta <= yv[0] && T->act[gi] == BBX_ACT_NONE) T->act[gi] = (int32_t)(n + 1);
            x += dx;
            r += dr;
            if (x >= nx) {
                x -= nx;
                ++r;
            }
        }
        cl.sync();  // every band's new V is written before any band reads it
        p ^= 1;
        t = t + T->dt_d;
        n += 1;
    }

    // the new state into the buffer that becomes current, and the FP64 total of V
    const int cur1 = cur0 ^ (n_steps & 1);
    float* dst = T->state[cur1];
    double hi = 0.0, lo = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const int r = i / nx, x = i - r * nx;
        const long long gi = (long long)(rb0 + r) * px + x;
        const float u = V[p][i];
        dst[gi] = u;
#pragma unroll
        for (int v = 1; v < S; ++v) dst[v * vol + gi] = Wv[(v - 1) * maxr * nx + i];
        res_two_sum(hi, lo, (double)u);
    }
    double part = hi + lo;
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red_hi[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kResThreads / 32; ++w) b += red_hi[w];
        double* root = cl.map_shared_rank(cl_part, 0);
        root[rank] = b;
    }
    (void)red_lo;
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < NC; ++k) tot += cl_part[k];
        if (!isfinite(tot)) atomicOr(err, ERRBIT_NAN);
        D->total = tot;
        D->total_pending = 0;
        D->t = t;
        D->n = n;
        D->cur = cur1;
    }
    cl.sync();  // no CTA leaves while its shared memory may still be read
}

template <int MODEL, int NC>
int resident_smem(int nx, int ny) {
    const int maxr = (ny + NC - 1) / NC;
    return (int)(sizeof(float) * (size_t)(Model<MODEL>::S + 1) * maxr * nx);
}

// One cluster of NC CTAs, if the grid fits and the GPU can hold such a
// cluster (*ok); returns launch errors.
template <int MODEL, int NC>
cudaError_t resident_try(const TissueArgs* d_t, int nx, int ny, int n_steps, int* d_err, cudaStream_t s,
                         bool check_only, bool* ok) {
    const int smem = resident_smem<MODEL, NC>(nx, ny);
    *ok = false;
    if (smem > kResMaxSmem || ny < NC) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_resident_sheet<MODEL, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (NC > kResCtasPortable &&
        cudaFuncSetAttribute(k_resident_sheet<MODEL, NC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
        cudaGetLastError();  // not offered here: the caller tries the portable size
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(NC);
    cfg.blockDim = dim3(kResThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_resident_sheet<MODEL, NC>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;
    }
    if (clusters < 1) return cudaSuccess;
    *ok = true;
    if (check_only) return cudaSuccess;
    k_resident_sheet<MODEL, NC><<<NC, kResThreads, smem, s>>>(d_t, n_steps, d_err);
    return cudaGetLastError();
}

template <int MODEL>
cudaError_t resident_launch(const TissueArgs* d_t, int nx, int ny, int n_steps, int* d_err, cudaStream_t s,
                            bool check_only, bool* ok) {
    cudaError_t e = resident_try<MODEL, kResCtasLarge>(d_t, nx, ny, n_steps, d_err, s, check_only, ok);
    if (e != cudaSuccess || *ok) return e;
    return resident_try<MODEL, kResCtasPortable>(d_t, nx, ny, n_steps, d_err, s, check_only, ok);
}

}  // namespace

// Run n_steps on a small isotropic, unmasked sheet with the resident kernel.
// check_only: only report (in *ok) whether this grid shape can run resident.
cudaError_t resident_sheet_steps(int model, const TissueArgs* d_t, int nx, int ny, int n_steps, int* d_err,
                                 cudaStream_t s, bool check_only, bool* ok) {
    switch (model) {
        case BBX_FHN: return resident_launch<BBX_FHN>(d_t, nx, ny, n_steps, d_err, s, check_only, ok);
        case BBX_BARKLEY: return resident_launch<BBX_BARKLEY>(d_t, nx, ny, n_steps, d_err, s, check_only, ok);
        case BBX_ZFK: return resident_launch<BBX_ZFK>(d_t, nx, ny, n_steps, d_err, s, check_only, ok);
        case BBX_DIFFUSION: return resident_launch<BBX_DIFFUSION>(d_t, nx, ny, n_steps, d_err, s, check_only, ok);
    }
    *ok = false;
    return cudaSuccess;
}

}  // namespace bbx
