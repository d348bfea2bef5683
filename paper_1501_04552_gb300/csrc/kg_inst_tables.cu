// kg_inst_tables.cu -- the pass-launcher tables of the three FFT precisions, built from
// the per-share functions of kg_inst.cu.
#include "kg_inst.h"
#include "../../include/kg.h"

namespace kg {

#define KG_TABLE_COMMON(ns, S)                                                                                 \
    &ns::pass_x, &ns::col, &ns::col_from_f64, &ns::update, &ns::update_parts, &ns::ens_step,                 \
        &ns::ens_blocks_per_sm, &ns::x_parts, S, &ns::passc_x, &ns::xc_parts, &ns::colc, &ns::colc_from_f64, \
        &ns::updatec, &ns::updatec_parts

const PassLaunch kLaunchF64 = {
    KG_TABLE_COMMON(inst_f64, 16),
    nullptr, nullptr,   // no fused z pass: the three-kernel form is faster for FP64
    nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,    // set-up and read-out: the FP64 kernels
    nullptr, nullptr};                                       // no fused xy pass
const PassLaunch kLaunchDF = {
    KG_TABLE_COMMON(inst_df, 16),
    &inst_df::zstep, &inst_df::zstep_parts,
    &inst_df::x_setup, &inst_df::x_readout, &inst_df::col_to_f64,
    &inst_df::xc_setup, &inst_df::xc_readout, &inst_df::colc_to_f64,
    nullptr, nullptr};   // no fused xy pass: the double-float passes are bound by the FMA pipes, not HBM
const PassLaunch kLaunchF32 = {
    KG_TABLE_COMMON(inst_f32, 8),
    &inst_f32::zstep, &inst_f32::zstep_parts,
    nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,    // set-up and read-out stay FP64
    &inst_f32::xy_fused, &inst_f32::xy_parts};

}  // namespace kg
