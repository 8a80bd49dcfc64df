// Explicit instantiations of the fused step kernel for the br model.
#include "bbx_device.cuh"

namespace bbx {

template <bool MA, bool AN, int TY, bool SU = false, bool PL = false, bool GE = false>
static StepKernel make_br() {
    using P = Plan<BBX_BR, MA, AN, TY, SU>;
    return StepKernel{reinterpret_cast<const void*>(&step_kernel<BBX_BR, MA, AN, TY, SU, PL, GE>), P::SMEM,
                      P::THREADS, TY};
}

// planar: grids with nz = 1 (tiles marched along y); general: the variant
// for the Lie scheme (7- and 14-row tiles)
StepKernel step_kernel_br(bool masked, bool aniso, int ty, bool planar, bool general) {
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

}  // namespace bbx
