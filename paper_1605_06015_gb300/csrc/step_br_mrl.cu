// Explicit instantiations of the fused step kernel for Beeler-Reuter with the
// Markov-form sodium activation (matrix Rush-Larsen), and the kernel that
// tabulates the chain's one-step transition matrix T(V) = exp(dt A(V)).
#include "bbx_device.cuh"

namespace bbx {

template <bool MA, int AN, int TY, bool PL = false>
static StepKernel make_br_mrl() {
    using P = Plan<BBX_BR_MRL, MA, AN, TY, false>;
    return StepKernel{reinterpret_cast<const void*>(&step_kernel<BBX_BR_MRL, MA, AN, TY, false, PL, false>),
                      P::SMEM, P::THREADS, TY};
}

// Tile rows 7 and 14 (the eleven variables make a 28-row stage too large for
// shared memory); unsplit Euler / Rush-Larsen only.
StepKernel step_kernel_br_mrl(bool masked, int aniso, int ty, bool planar, bool general) {
    if (general) return StepKernel{nullptr, 0, 0, 0};
    // unmasked grids whose W-tilde sums all vanish: no sums in the stage ring
    if (!masked && aniso == AN_NO_SUMS && (ty == 7 || ty == 14))
        return ty == 7 ? (planar ? make_br_mrl<false, AN_NO_SUMS, 7, true>() : make_br_mrl<false, AN_NO_SUMS, 7>())
                       : (planar ? make_br_mrl<false, AN_NO_SUMS, 14, true>() : make_br_mrl<false, AN_NO_SUMS, 14>());
#define BBX_CASE(MA, AN, T) \
    if (masked == MA && aniso == AN && ty == T) \
        return planar ? make_br_mrl<MA, AN, T, true>() : make_br_mrl<MA, AN, T>();
    BBX_CASE(false, false, 7) BBX_CASE(false, false, 14)
    BBX_CASE(false, true, 7) BBX_CASE(false, true, 14)
    BBX_CASE(true, false, 7) BBX_CASE(true, false, 14)
    BBX_CASE(true, true, 7) BBX_CASE(true, true, 14)
#undef BBX_CASE
    return StepKernel{nullptr, 0, 0, 0};
}

namespace {

// alpha_m and beta_m of Beeler & Reuter (1977) in double precision, 1/ms.
__device__ double mrl_alpha_m(double V) {
    const double x = V + 47.0;
    return x == 0.0 ? 10.0 : -x / expm1(-0.1 * x);
}
__device__ double mrl_beta_m(double V) { return 40.0 * exp(-0.056 * (V + 72.0)); }

__device__ void mrl_mul4(const double* X, const double* Y, double* Z) {
    double t[16];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) s = fma(X[i * 4 + k], Y[k * 4 + j], s);
            t[i * 4 + j] = s;
        }
#pragma unroll
    for (int i = 0; i < 16; ++i) Z[i] = t[i];
}

// One entry per thread: the generator A(V) of the chain (column j = from
// state j), M = dt A / 2^s with s the smallest power that brings the largest
// absolute column sum of dt A to 1/4 or below, exp(M) by its Taylor series to
// degree 18 (Horner form), then s squarings.  FP64 throughout; stored as
// float, row-major.
__global__ void k_mrl_table(float4* __restrict__ tab, int n, double vmin, double dv, double dt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double V = vmin + dv * e;
    const double a = mrl_alpha_m(V), b = mrl_beta_m(V);
    double M[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) M[i] = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double out = 0.0;
        if (k < 3) {
            M[(k + 1) * 4 + k] = (3 - k) * a;
            out += (3 - k) * a;
        }
        if (k > 0) {
            M[(k - 1) * 4 + k] = k * b;
            out += k * b;
        }
        M[k * 4 + k] = -out;
    }
    // column sums of |dt A| are 2 x the outflow rate
    double nrm = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) nrm = fmax(nrm, -2.0 * M[k * 4 + k] * dt);
    int s = 0;
    while (nrm > 0.25 && s < 60) {
        nrm *= 0.5;
        ++s;
    }
    const double scale = ldexp(dt, -s);
#pragma unroll
    for (int i = 0; i < 16; ++i) M[i] *= scale;
    // Horner: E = I + M (I + M/2 (I + M/3 (... (I + M/18))))
    double E[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) E[i] = (i % 5 == 0) ? 1.0 : 0.0;
    for (int k = 18; k >= 1; --k) {
        double P[16];
        mrl_mul4(M, E, P);
#pragma unroll
        for (int i = 0; i < 16; ++i) E[i] = ((i % 5 == 0) ? 1.0 : 0.0) + P[i] / k;
    }
    for (int q = 0; q < s; ++q) mrl_mul4(E, E, E);
#pragma unroll
    for (int r = 0; r < 4; ++r)
        tab[e * 4 + r] = make_float4((float)E[r * 4 + 0], (float)E[r * 4 + 1], (float)E[r * 4 + 2], (float)E[r * 4 + 3]);
}

}  // namespace

// Tabulate T(V) for the time step dt into tab (kTabN x 4 float4).
cudaError_t mrl_build_table(float4* tab, double dt, cudaStream_t s) {
    k_mrl_table<<<(kTabN + 127) / 128, 128, 0, s>>>(tab, kTabN, (double)kTabVmin, (double)kTabDv, dt);
    return cudaGetLastError();
}

}  // namespace bbx
