// Explicit instantiations of the fused step kernel for the br model.
#include "bbx_device.cuh"

namespace bbx {

template <bool MA, bool AN, int TY, bool SU = false, bool PL = false>
static StepKernel make_br() {
    using P = Plan<BBX_BR, MA, AN, TY, SU>;
    return StepKernel{reinterpret_cast<const void*>(&step_kernel<BBX_BR, MA, AN, TY, SU, PL>), P::SMEM, P::THREADS,
                      TY};
}

// planar: grids with nz = 1 (tiles marched along y)
StepKernel step_kernel_br(bool masked, bool aniso, int ty, bool planar) {
#define BBX_CASE(MA, AN, T) \
    if (masked == MA && aniso == AN && ty == T) \
        return planar ? make_br<MA, AN, T, false, true>() : make_br<MA, AN, T>();
    BBX_CASE(false, false, 7) BBX_CASE(false, false, 14) BBX_CASE(false, false, 28)
    BBX_CASE(false, true, 7) BBX_CASE(false, true, 14) BBX_CASE(false, true, 28)
    BBX_CASE(true, false, 7) BBX_CASE(true, false, 14) BBX_CASE(true, false, 28)
    BBX_CASE(true, true, 7) BBX_CASE(true, true, 14) BBX_CASE(true, true, 28)
#undef BBX_CASE
    return StepKernel{nullptr, 0, 0, 0};
}

// With the reaction surrogate (tensor-core MLP with exact fallback).
StepKernel step_kernel_br_surrogate(bool masked, bool aniso, int ty) {
#define BBX_CASE(MA, AN, T) \
    if (masked == MA && aniso == AN && ty == T) return make_br<MA, AN, T, true>();
    BBX_CASE(false, false, 7) BBX_CASE(false, false, 14)
    BBX_CASE(false, true, 7) BBX_CASE(false, true, 14)
    BBX_CASE(true, false, 7) BBX_CASE(true, false, 14)
    BBX_CASE(true, true, 7) BBX_CASE(true, true, 14)
#undef BBX_CASE
    return StepKernel{nullptr, 0, 0, 0};
}

}  // namespace bbx
