// Headless output kernels: the 1-byte quantisation of three layers of the
// grid (the ppmout device of section "Input and output"), and phase
// singularities in z cross-sections as intersections of the isolines of two
// fields inside a grid cell (the singz device of the same section).  Both
// read the current state in its padded device layout; neither allocates.
#include <cstdint>

#include <cuda_runtime.h>

namespace bbx {

namespace {

constexpr uint8_t kTissue = 1;  // mask bit 0: the node is tissue

// t = (v - lo) / (hi - lo) clamped to [0, 1]; code = floor(255 t + 0.5), each
// operation rounded once (no contraction), so the host can reproduce it.
// The quotient is first formed as (v - lo) times the rounded reciprocal of the
// span: it differs from the rounded quotient by at most about 3 units in its
// last place, i.e. 255 t + 0.5 by less than 1e-4, so the floor is the same
// unless 255 t + 0.5 lies within 1e-4 of an integer; there the exact division
// decides.  (The division's own slow path, which denormal inputs such as a
// decaying resting variable take, is then rarely reached.)
__device__ __forceinline__ uint8_t quantise(float v, float lo, float span, float rspan) {
    const float d = __fsub_rn(v, lo);
    float t = fminf(fmaxf(__fmul_rn(d, rspan), 0.0f), 1.0f);
    float q = __fadd_rn(__fmul_rn(t, 255.0f), 0.5f);
    const float fr = q - floorf(q);
    if (fr < 1e-4f || fr > 1.0f - 1e-4f) {
        t = fminf(fmaxf(__fdiv_rn(d, span), 0.0f), 1.0f);
        q = __fadd_rn(__fmul_rn(t, 255.0f), 0.5f);
    }
    return (uint8_t)floorf(q);
}

// Each warp takes whole rows (y, z): its lanes walk the row in groups of 4
// consecutive nodes, float4 loads from the padded rows (px is a multiple of
// 32) and three 32-bit stores of the 12 bytes of a group, except in a row's
// last partial group or where the output row is not 4-byte aligned.  Rows are
// spread over the warps of the grid, so the only divisions are one per row.
// The current buffer is picked on the device from the grid's parity, so the
// call does not synchronise.
__global__ void k_ppm(const float* __restrict__ s0, const float* __restrict__ s1, const int* __restrict__ cur,
                      const uint8_t* __restrict__ mask, long long vol, int nx, int ny, int nz, int px,
                      long long plane, int3 layer, float3 lo, float3 span, uint8_t* __restrict__ out) {
    const float* state = *cur ? s1 : s0;
    const int gx = (nx + 3) / 4;
    const long long rows = (long long)ny * nz;
    const int ly[3] = {layer.x, layer.y, layer.z};
    const float l[3] = {lo.x, lo.y, lo.z}, sp[3] = {span.x, span.y, span.z};
    const float rs[3] = {__frcp_rn(span.x), __frcp_rn(span.y), __frcp_rn(span.z)};
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        const int z = (int)(r / ny), y = (int)(r - (long long)z * ny);
        const float* row = state + z * plane + (long long)y * px;
        const uint8_t* mrow = mask ? mask + z * plane + (long long)y * px : nullptr;
        uint8_t* orow = out + 3 * (((long long)z * ny + y) * nx);
        const bool aligned = ((((long long)z * ny + y) * nx) & 3) == 0;
        for (int g = lane; g < gx; g += 32) {
            const int x = 4 * g;
            uint8_t c[4][3] = {};
            bool tis[4] = {true, true, true, true};
            if (mrow) {
                const uchar4 m = *reinterpret_cast<const uchar4*>(mrow + x);
                tis[0] = m.x & kTissue; tis[1] = m.y & kTissue; tis[2] = m.z & kTissue; tis[3] = m.w & kTissue;
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                if (ly[ch] < 0) continue;
                const float4 v = *reinterpret_cast<const float4*>(row + ly[ch] * vol + x);
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) c[k][ch] = tis[k] ? quantise(vv[k], l[ch], sp[ch], rs[ch]) : 0;
            }
            if (x + 4 <= nx && aligned) {
                uint32_t w[3];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    w[b] = 0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int byte = 4 * b + k;  // byte of the 12-byte group
                        w[b] |= (uint32_t)c[byte / 3][byte % 3] << (8 * k);
                    }
                }
                uint32_t* o = reinterpret_cast<uint32_t*>(orow + 3 * x);
                o[0] = w[0];
                o[1] = w[1];
                o[2] = w[2];
            } else {
                for (int k = 0; k < 4 && x + k < nx; ++k)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) orow[3 * (x + k) + ch] = c[k][ch];
            }
        }
    }
}

// Crossings of the isoline f = 0 (g = f - f*) with the four edges of a cell
// (corners (0,0), (1,0), (1,1), (0,1)); an edge is crossed where g > 0 at one
// end only.  Returns the number of crossings; the first two are in p.
__device__ __forceinline__ int cell_crossings(const float g[4], float2 p[2]) {
    const float cx[4] = {0.0f, 1.0f, 1.0f, 0.0f}, cy[4] = {0.0f, 0.0f, 1.0f, 1.0f};
    int n = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int j = (i + 1) & 3;
        if ((g[i] > 0.0f) != (g[j] > 0.0f)) {
            const float s = __fdividef(g[i], __fsub_rn(g[i], g[j]));  // |g[i] - g[j]| > 0, far below 2^126
            if (n < 2) p[n] = make_float2(cx[i] + s * (cx[j] - cx[i]), cy[i] + s * (cy[j] - cy[i]));
            ++n;
        }
    }
    return n;
}

// Number of the four cell edges whose ends lie on different sides of the
// isoline (g > 0 at one end only): the same test cell_crossings applies.
__device__ __forceinline__ int edge_changes(const float g[4]) {
    const unsigned s = (g[0] > 0.0f ? 1u : 0u) | (g[1] > 0.0f ? 2u : 0u) | (g[2] > 0.0f ? 4u : 0u) |
                       (g[3] > 0.0f ? 8u : 0u);
    return __popc(s ^ (((s >> 1) | (s << 3)) & 15u));
}

// Each warp takes whole rows of cells (y, z); each lane four consecutive
// cells x .. x+3, from float4 loads of rows y and y+1 of both fields (px is a
// multiple of 32, so x + 3 stays inside the padded row) and the corner column
// x + 4 from the next lane, or loaded where no next lane holds it.  A cell is
// examined further only where both isolines change sides exactly twice
// around it; that examination is cell_crossings and the intersection below.
__global__ void k_singz(const float* __restrict__ s0, const float* __restrict__ s1, const int* __restrict__ cur,
                        long long off_a, long long off_b, float iso_a, float iso_b, const uint8_t* __restrict__ mask,
                        int nx, int ny, int nz, int px, long long plane, float* __restrict__ xyz, int max_points,
                        int* __restrict__ count) {
    const float* st = *cur ? s1 : s0;  // the current buffer, from the grid's parity
    const float* fa = st + off_a;
    const float* fb = st + off_b;
    const int cx = nx - 1, cy = ny - 1;
    const int gx = (cx + 3) / 4;  // groups of four cells in a row
    const long long rows = (long long)cy * nz;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long rr = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); rr < rows; rr += warps) {
        const int z = (int)(rr / cy), y = (int)(rr - (long long)z * cy);
        const long long r0 = z * plane + (long long)y * px, r1 = r0 + px;
        for (int gb = 0; gb < gx; gb += 32) {
            const int g = gb + lane;
            const bool act = g < gx;
            const int x = 4 * g;
            float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
            uint32_t m0 = 0xffffffffu, m1 = 0xffffffffu;  // four mask bytes of each row (all tissue without a mask)
            if (act) {
                a0 = *reinterpret_cast<const float4*>(fa + r0 + x);
                a1 = *reinterpret_cast<const float4*>(fa + r1 + x);
                b0 = *reinterpret_cast<const float4*>(fb + r0 + x);
                b1 = *reinterpret_cast<const float4*>(fb + r1 + x);
                if (mask) {
                    m0 = *reinterpret_cast<const uint32_t*>(mask + r0 + x);
                    m1 = *reinterpret_cast<const uint32_t*>(mask + r1 + x);
                }
            }
            float a0e = __shfl_down_sync(0xffffffffu, a0.x, 1), a1e = __shfl_down_sync(0xffffffffu, a1.x, 1);
            float b0e = __shfl_down_sync(0xffffffffu, b0.x, 1), b1e = __shfl_down_sync(0xffffffffu, b1.x, 1);
            uint32_t m0e = __shfl_down_sync(0xffffffffu, m0, 1), m1e = __shfl_down_sync(0xffffffffu, m1, 1);
            if (!act) continue;
            if ((lane == 31 || g + 1 >= gx) && x + 4 < nx) {  // column x + 4 of the last cell
                a0e = fa[r0 + x + 4];
                a1e = fa[r1 + x + 4];
                b0e = fb[r0 + x + 4];
                b1e = fb[r1 + x + 4];
                if (mask) {
                    m0e = mask[r0 + x + 4];
                    m1e = mask[r1 + x + 4];
                }
            }
            const float A0[5] = {a0.x, a0.y, a0.z, a0.w, a0e}, A1[5] = {a1.x, a1.y, a1.z, a1.w, a1e};
            const float B0[5] = {b0.x, b0.y, b0.z, b0.w, b0e}, B1[5] = {b1.x, b1.y, b1.z, b1.w, b1e};
            const uint32_t t0 = (m0 & 0x01010101u) | ((m0e & 1u) << 31);  // tissue bits, column k at bit 8k
            const uint32_t t1 = (m1 & 0x01010101u) | ((m1e & 1u) << 31);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (x + k >= cx) break;
                if (mask) {
                    const uint32_t n0 = k < 3 ? (t0 >> (8 * (k + 1))) & 1u : t0 >> 31;
                    const uint32_t n1 = k < 3 ? (t1 >> (8 * (k + 1))) & 1u : t1 >> 31;
                    if (!(((t0 >> (8 * k)) & 1u) && n0 && n1 && ((t1 >> (8 * k)) & 1u))) continue;
                }
                // corners in cell order: (x, y), (x+1, y), (x+1, y+1), (x, y+1)
                const float ga[4] = {__fsub_rn(A0[k], iso_a), __fsub_rn(A0[k + 1], iso_a), __fsub_rn(A1[k + 1], iso_a),
                                     __fsub_rn(A1[k], iso_a)};
                const float gbv[4] = {__fsub_rn(B0[k], iso_b), __fsub_rn(B0[k + 1], iso_b),
                                      __fsub_rn(B1[k + 1], iso_b), __fsub_rn(B1[k], iso_b)};
                if (edge_changes(ga) != 2 || edge_changes(gbv) != 2) continue;
                float2 pa[2], pb[2];
                if (cell_crossings(ga, pa) != 2 || cell_crossings(gbv, pb) != 2) continue;
                // pa0 + al (pa1 - pa0) = pb0 + be (pb1 - pb0)
                const float d1x = pa[1].x - pa[0].x, d1y = pa[1].y - pa[0].y;
                const float d2x = pb[1].x - pb[0].x, d2y = pb[1].y - pb[0].y;
                const float det = d1y * d2x - d1x * d2y;
                if (det == 0.0f) continue;
                const float rx = pb[0].x - pa[0].x, ry = pb[0].y - pa[0].y;
                const float rdet = __frcp_rn(det);
                const float al = (ry * d2x - rx * d2y) * rdet;
                const float be = (d1x * ry - d1y * rx) * rdet;
                if (!(al >= 0.0f && al <= 1.0f && be >= 0.0f && be <= 1.0f)) continue;
                const int slot = atomicAdd(count, 1);
                if (slot < max_points) {
                    xyz[3 * slot] = (float)(x + k) + pa[0].x + al * d1x;
                    xyz[3 * slot + 1] = (float)y + pa[0].y + al * d1y;
                    xyz[3 * slot + 2] = (float)z;
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_ppm(const float* s0, const float* s1, const int* cur, const uint8_t* mask, long long vol, int nx,
                       int ny, int nz, int px, long long plane, const int layer[3], const float lo[3],
                       const float hi[3], uint8_t* out, int num_sms, cudaStream_t s) {
    const long long rows = (long long)ny * nz;  // one warp per row, 8 rows per block
    long long nb = (rows + 7) / 8;
    if (nb > (long long)num_sms * 16) nb = (long long)num_sms * 16;
    k_ppm<<<(int)(nb < 1 ? 1 : nb), 256, 0, s>>>(s0, s1, cur, mask, vol, nx, ny, nz, px, plane,
                                                 make_int3(layer[0], layer[1], layer[2]),
                                                 make_float3(lo[0], lo[1], lo[2]),
                                                 make_float3(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]), out);
    return cudaGetLastError();
}

cudaError_t launch_singz(const float* s0, const float* s1, const int* cur, long long off_a, long long off_b,
                         float iso_a, float iso_b, const uint8_t* mask, int nx, int ny, int nz, int px,
                         long long plane, float* xyz, int max_points, int* d_count, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const long long n = (long long)(nx - 1) * (ny - 1) * nz;
    if (n <= 0) return cudaSuccess;
    long long nb = ((long long)(ny - 1) * nz + 7) / 8;  // one warp per row of cells, 8 rows per block
    if (nb > (long long)num_sms * 16) nb = (long long)num_sms * 16;
    k_singz<<<(int)(nb < 1 ? 1 : nb), 256, 0, s>>>(s0, s1, cur, off_a, off_b, iso_a, iso_b, mask, nx, ny, nz, px,
                                                   plane, xyz, max_points, d_count);
    return cudaGetLastError();
}

}  // namespace bbx
