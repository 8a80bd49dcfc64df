// Explicit instantiations of the fused step kernel for the br model.
#include "bbx_device.cuh"

namespace bbx {

template <bool MA, int AN, int TY, bool SU = false, bool PL = false, bool GE = false>
static StepKernel make_br() {
    using P = Plan<BBX_BR, MA, AN, TY, SU>;
    return StepKernel{reinterpret_cast<const void*>(&step_kernel<BBX_BR, MA, AN, TY, SU, PL, GE>), P::SMEM,
                      P::THREADS, TY};
}

// planar: grids with nz = 1 (tiles marched along y); general: the variant
// for the Lie scheme (7- and 14-row tiles)
StepKernel step_kernel_br(bool masked, int aniso, int ty, bool planar, bool general) {
    // unmasked grids whose W-tilde sums all vanish: no sums in the stage ring
    // (plain variants; the general ones read the sums, or skip their copies)
#define BBX_CASE_NS(T) \
    if (!masked && aniso == AN_NO_SUMS && ty == T) \
        return general ? StepKernel{nullptr, 0, 0, 0} \
                       : (planar ? make_br<false, AN_NO_SUMS, T, false, true>() : make_br<false, AN_NO_SUMS, T>());
    BBX_CASE_NS(7) BBX_CASE_NS(14) BBX_CASE_NS(28)
#undef BBX_CASE_NS
#define BBX_CASE(MA, AN, T) \
    if (masked == MA && aniso == AN && ty == T) { \
        if (general && T == 28) return StepKernel{nullptr, 0, 0, 0}; \
        if (general) \
            return planar ? make_br<MA, AN, T, false, true, T != 28>() : make_br<MA, AN, T, false, false, T != 28>(); \
        return planar ? make_br<MA, AN, T, false, true>() : make_br<MA, AN, T>(); \
    }
    BBX_CASE(false, false, 7) BBX_CASE(false, false, 14) BBX_CASE(false, false, 28)
    BBX_CASE(false, true, 7) BBX_CASE(false, true, 14) BBX_CASE(false, true, 28)
    BBX_CASE(true, false, 7) BBX_CASE(true, false, 14) BBX_CASE(true, false, 28)
    BBX_CASE(true, true, 7) BBX_CASE(true, true, 14) BBX_CASE(true, true, 28)
#undef BBX_CASE
    return StepKernel{nullptr, 0, 0, 0};
}

// With the reaction surrogate (tensor-core MLP with exact fallback); these
// variants also honour the scheme setting.
StepKernel step_kernel_br_surrogate(bool masked, bool aniso, int ty) {
#define BBX_CASE(MA, AN, T) \
    if (masked == MA && aniso == AN && ty == T) return make_br<MA, AN, T, true, false, true>();
    BBX_CASE(false, false, 7) BBX_CASE(false, false, 14)
    BBX_CASE(false, true, 7) BBX_CASE(false, true, 14)
    BBX_CASE(true, false, 7) BBX_CASE(true, false, 14)
    BBX_CASE(true, true, 7) BBX_CASE(true, true, 14)
#undef BBX_CASE
    return StepKernel{nullptr, 0, 0, 0};
}

namespace {

// Beeler & Reuter (1977) rates in double precision, 1/ms: alpha and beta of
// x1, m, h, j, d, f (the expressions of Model<BBX_BR>).
__device__ void br_rates_d(double V, double* al, double* be) {
    const double xm = V + 47.0;
    al[0] = 0.0005 * exp(0.083 * (V + 50.0)) / (exp(0.057 * (V + 50.0)) + 1.0);
    be[0] = 0.0013 * exp(-0.06 * (V + 20.0)) / (exp(-0.04 * (V + 20.0)) + 1.0);
    al[1] = xm == 0.0 ? 10.0 : -xm / expm1(-0.1 * xm);
    be[1] = 40.0 * exp(-0.056 * (V + 72.0));
    al[2] = 0.126 * exp(-0.25 * (V + 77.0));
    be[2] = 1.7 / (exp(-0.082 * (V + 22.5)) + 1.0);
    al[3] = 0.055 * exp(-0.25 * (V + 78.0)) / (exp(-0.2 * (V + 78.0)) + 1.0);
    be[3] = 0.3 / (exp(-0.1 * (V + 32.0)) + 1.0);
    al[4] = 0.095 * exp(-0.01 * (V - 5.0)) / (exp(-0.072 * (V - 5.0)) + 1.0);
    be[4] = 0.07 * exp(-0.017 * (V + 44.0)) / (exp(0.05 * (V + 44.0)) + 1.0);
    al[5] = 0.012 * exp(-0.008 * (V + 28.0)) / (exp(0.15 * (V + 28.0)) + 1.0);
    be[5] = 0.0065 * exp(-0.02 * (V + 30.0)) / (exp(-0.2 * (V + 30.0)) + 1.0);
}

// One entry per thread: A = exp(-(alpha+beta) dt) and B = alpha/(alpha+beta)
// (1 - A) of Eq. (RLcoeff) for the six gates, then K(V) with I_x1 = x1 K(V),
// I_K1(V), alpha_f(V) and 1 - exp(-dt/tau_c) (the calcium gate of BBX_BR_FCA;
// 0 when tau_c = 0); FP64, stored as float.
__global__ void k_rl_table(float4* __restrict__ tab, int n, double vmin, double dv, double dt, double tau_c) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double V = vmin + dv * e;
    double al[6], be[6], c[16];
    br_rates_d(V, al, be);
    for (int g = 0; g < 6; ++g) {
        const double A = exp(-(al[g] + be[g]) * dt);
        c[2 * g] = A;
        c[2 * g + 1] = al[g] / (al[g] + be[g]) * (1.0 - A);
    }
    c[12] = 0.8 * (exp(0.04 * (V + 77.0)) - 1.0) * exp(-0.04 * (V + 35.0));
    const double w = V + 23.0;
    const double lin = w == 0.0 ? 5.0 : 0.2 * w / (-expm1(-0.04 * w));
    c[13] = 0.35 * (4.0 * (exp(0.04 * (V + 85.0)) - 1.0) / (exp(0.08 * (V + 53.0)) + exp(0.04 * (V + 53.0))) + lin);
    c[14] = al[5];
    c[15] = tau_c > 0.0 ? -expm1(-dt / tau_c) : 0.0;
    for (int q = 0; q < 4; ++q)
        tab[e * 4 + q] = make_float4((float)c[4 * q], (float)c[4 * q + 1], (float)c[4 * q + 2], (float)c[4 * q + 3]);
}

}  // namespace

// Tabulate the Rush-Larsen coefficients of Beeler-Reuter for the time step
// dt into tab (kTabN x 4 float4); tau_c > 0 adds the calcium gate's constant.
cudaError_t br_build_rl_table(float4* tab, double dt, double tau_c, cudaStream_t s) {
    k_rl_table<<<(kTabN + 127) / 128, 128, 0, s>>>(tab, kTabN, (double)kTabVmin, (double)kTabDv, dt, tau_c);
    return cudaGetLastError();
}

}  // namespace bbx
