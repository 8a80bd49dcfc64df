// Explicit instantiations of the fused step kernel for Beeler-Reuter with the
// six gates stored in 16 bits (binary16 or unsigned fixed point), tile rows 7
// and 14; general: the variants that honour the Lie scheme and the tabulated
// Rush-Larsen coefficients.
#include "bbx_device.cuh"

namespace bbx {

template <bool MA, int AN, int TY, bool PL, bool GE, int GA>
static StepKernel make_br16() {
    using P = Plan<BBX_BR, MA, AN, TY, false, GA>;
    return StepKernel{reinterpret_cast<const void*>(&step_kernel<BBX_BR, MA, AN, TY, false, PL, GE, GA>), P::SMEM,
                      P::THREADS, TY};
}

template <bool MA, int AN, int TY, int GA>
static StepKernel pick_br16(bool planar, bool general) {
    if (general) return planar ? make_br16<MA, AN, TY, true, true, GA>() : make_br16<MA, AN, TY, false, true, GA>();
    return planar ? make_br16<MA, AN, TY, true, false, GA>() : make_br16<MA, AN, TY, false, false, GA>();
}

StepKernel step_kernel_br16(bool masked, bool aniso, int ty, bool planar, bool general, int gates) {
#define BBX_CASE(MA, AN, T)                                                                 \
    if (masked == MA && aniso == AN && ty == T) {                                           \
        if (gates == GATES_F16) return pick_br16<MA, AN, T, GATES_F16>(planar, general);    \
        if (gates == GATES_U16) return pick_br16<MA, AN, T, GATES_U16>(planar, general);    \
    }
    BBX_CASE(false, false, 7) BBX_CASE(false, false, 14)
    BBX_CASE(false, true, 7) BBX_CASE(false, true, 14)
    BBX_CASE(true, false, 7) BBX_CASE(true, false, 14)
    BBX_CASE(true, true, 7) BBX_CASE(true, true, 14)
#undef BBX_CASE
    return StepKernel{nullptr, 0, 0, 0};
}

}  // namespace bbx
