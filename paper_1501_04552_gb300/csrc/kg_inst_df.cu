// kg_inst_df.cu -- pass launchers for the PrecDF precision.
#include "kg_launch_impl.cuh"

namespace kg {
template struct Launchers<PrecDF>;
const PassLaunch kLaunchDF = {
    &Launchers<PrecDF>::pass_x, &Launchers<PrecDF>::col, &Launchers<PrecDF>::col_from_f64, &Launchers<PrecDF>::update, &Launchers<PrecDF>::update_parts, &Launchers<PrecDF>::ens_step, &Launchers<PrecDF>::ens_blocks_per_sm, &Launchers<PrecDF>::x_parts, sizeof(PrecDF::S),
    &Launchers<PrecDF>::passc_x, &Launchers<PrecDF>::xc_parts, &Launchers<PrecDF>::colc, &Launchers<PrecDF>::colc_from_f64, &Launchers<PrecDF>::updatec, &Launchers<PrecDF>::updatec_parts,
    &Launchers<PrecDF>::zstep, &Launchers<PrecDF>::zstep_parts,
    &Launchers<PrecDF>::x_setup, &Launchers<PrecDF>::x_readout, &Launchers<PrecDF>::col_to_f64,
    &Launchers<PrecDF>::xc_setup, &Launchers<PrecDF>::xc_readout, &Launchers<PrecDF>::colc_to_f64};
}  // namespace kg
