// kg_inst_f32.cu -- pass launchers for the PrecF32 precision.
#include "kg_launch_impl.cuh"

namespace kg {
template struct Launchers<PrecF32>;
const PassLaunch kLaunchF32 = {
    &Launchers<PrecF32>::pass_x, &Launchers<PrecF32>::col, &Launchers<PrecF32>::col_from_f64, &Launchers<PrecF32>::update, &Launchers<PrecF32>::update_parts, &Launchers<PrecF32>::ens_step, &Launchers<PrecF32>::ens_blocks_per_sm, &Launchers<PrecF32>::x_parts, sizeof(PrecF32::S),
    &Launchers<PrecF32>::passc_x, &Launchers<PrecF32>::xc_parts, &Launchers<PrecF32>::colc, &Launchers<PrecF32>::colc_from_f64, &Launchers<PrecF32>::updatec, &Launchers<PrecF32>::updatec_parts,
    &Launchers<PrecF32>::zstep, &Launchers<PrecF32>::zstep_parts,
    nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};   // set-up and read-out stay FP64
}  // namespace kg
