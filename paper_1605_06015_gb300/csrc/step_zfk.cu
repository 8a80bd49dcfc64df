// Explicit instantiations of the fused step kernel for the zfk model.
#include "bbx_device.cuh"

namespace bbx {

template <bool MA, int AN, int TY, bool PL, bool GE>
static StepKernel make_zfk() {
    using P = Plan<BBX_ZFK, MA, AN, TY>;
    return StepKernel{reinterpret_cast<const void*>(&step_kernel<BBX_ZFK, MA, AN, TY, false, PL, GE>), P::SMEM,
                      P::THREADS, TY};
}

// planar: grids with nz = 1 (tiles marched along y); general: the variant
// for the Lie scheme or the RK4 solver (7- and 14-row tiles)
StepKernel step_kernel_zfk(bool masked, int aniso, int ty, bool planar, bool general) {
    // unmasked grids whose W-tilde sums all vanish: no sums in the stage ring
    // (plain variants; the general ones read the sums, or skip their copies)
#define BBX_CASE_NS(T) \
    if (!masked && aniso == AN_NO_SUMS && ty == T) \
        return general ? StepKernel{nullptr, 0, 0, 0} \
                       : (planar ? make_zfk<false, AN_NO_SUMS, T, true, false>() : make_zfk<false, AN_NO_SUMS, T, false, false>());
    BBX_CASE_NS(7) BBX_CASE_NS(14) BBX_CASE_NS(28)
#undef BBX_CASE_NS
#define BBX_CASE(MA, AN, T) \
    if (masked == MA && aniso == AN && ty == T) { \
        if (general && T == 28) return StepKernel{nullptr, 0, 0, 0}; \
        if (general) return planar ? make_zfk<MA, AN, T, true, T != 28>() : make_zfk<MA, AN, T, false, T != 28>(); \
        return planar ? make_zfk<MA, AN, T, true, false>() : make_zfk<MA, AN, T, false, false>(); \
    }
    BBX_CASE(false, false, 7) BBX_CASE(false, false, 14) BBX_CASE(false, false, 28)
    BBX_CASE(false, true, 7) BBX_CASE(false, true, 14) BBX_CASE(false, true, 28)
    BBX_CASE(true, false, 7) BBX_CASE(true, false, 14) BBX_CASE(true, false, 28)
    BBX_CASE(true, true, 7) BBX_CASE(true, true, 14) BBX_CASE(true, true, 28)
#undef BBX_CASE
    return StepKernel{nullptr, 0, 0, 0};
}

}  // namespace bbx
