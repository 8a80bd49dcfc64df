// Explicit instantiations of the fused step kernel for Beeler-Reuter with the
// calcium-gated slow inward channel (Model<BBX_BR_FCA>: the multivariate
// chain split into its univariate gates and a small remainder).
#include "bbx_device.cuh"

namespace bbx {

template <bool MA, int AN, int TY, bool PL = false>
static StepKernel make_br_fca() {
    using P = Plan<BBX_BR_FCA, MA, AN, TY, false>;
    return StepKernel{reinterpret_cast<const void*>(&step_kernel<BBX_BR_FCA, MA, AN, TY, false, PL, false>),
                      P::SMEM, P::THREADS, TY};
}

// Tile rows 7 and 14 (eleven variables, as the Markov sodium form); unsplit
// Euler / Rush-Larsen only.
StepKernel step_kernel_br_fca(bool masked, int aniso, int ty, bool planar, bool general) {
    if (general) return StepKernel{nullptr, 0, 0, 0};
    // unmasked grids whose W-tilde sums all vanish: no sums in the stage ring
    if (!masked && aniso == AN_NO_SUMS && (ty == 7 || ty == 14))
        return ty == 7 ? (planar ? make_br_fca<false, AN_NO_SUMS, 7, true>() : make_br_fca<false, AN_NO_SUMS, 7>())
                       : (planar ? make_br_fca<false, AN_NO_SUMS, 14, true>() : make_br_fca<false, AN_NO_SUMS, 14>());
#define BBX_CASE(MA, AN, T) \
    if (masked == MA && aniso == AN && ty == T) \
        return planar ? make_br_fca<MA, AN, T, true>() : make_br_fca<MA, AN, T>();
    BBX_CASE(false, false, 7) BBX_CASE(false, false, 14)
    BBX_CASE(false, true, 7) BBX_CASE(false, true, 14)
    BBX_CASE(true, false, 7) BBX_CASE(true, false, 14)
    BBX_CASE(true, true, 7) BBX_CASE(true, true, 14)
#undef BBX_CASE
    return StepKernel{nullptr, 0, 0, 0};
}

}  // namespace bbx
