// kg_inst.h -- the pass launchers of one precision as plain functions.
//
// Launchers<P> (kg_launch_impl.cuh) instantiates every kernel template of a precision;
// compiled as one unit per precision the double-float share alone took minutes.  So
// kg_inst.cu is compiled once per (precision, share) with KG_PREC_ID and KG_PART set,
// each compile defining the functions of one share in namespace kg::inst_f64,
// kg::inst_df or kg::inst_f32, and kg_inst_tables.cu builds the three PassLaunch
// tables from the declarations below.
#pragma once
#include <type_traits>

#include "kg_launch.h"

#define KG_INST_FN(m) std::remove_pointer_t<decltype(::kg::PassLaunch::m)>

#define KG_INST_DECLARE(ns)                                                            \
    namespace ns {                                                                     \
    KG_INST_FN(pass_x) pass_x;                /* share 0: x pass, x set-up/read-out */ \
    KG_INST_FN(x_parts) x_parts;                                                       \
    KG_INST_FN(x_setup) x_setup;                                                       \
    KG_INST_FN(x_readout) x_readout;                                                   \
    KG_INST_FN(xy_fused) xy_fused;                                                     \
    KG_INST_FN(xy_parts) xy_parts;                                                     \
    KG_INST_FN(col) col;                      /* share 1: column passes */             \
    KG_INST_FN(col_from_f64) col_from_f64;                                             \
    KG_INST_FN(col_to_f64) col_to_f64;                                                 \
    KG_INST_FN(zstep) zstep;                  /* share 2: z pass and update */         \
    KG_INST_FN(zstep_parts) zstep_parts;                                               \
    KG_INST_FN(update) update;                                                         \
    KG_INST_FN(update_parts) update_parts;                                             \
    KG_INST_FN(passc_x) passc_x;              /* share 3: complex field */             \
    KG_INST_FN(xc_parts) xc_parts;                                                     \
    KG_INST_FN(colc) colc;                                                             \
    KG_INST_FN(colc_from_f64) colc_from_f64;                                           \
    KG_INST_FN(updatec) updatec;                                                       \
    KG_INST_FN(updatec_parts) updatec_parts;                                           \
    KG_INST_FN(xc_setup) xc_setup;                                                     \
    KG_INST_FN(xc_readout) xc_readout;                                                 \
    KG_INST_FN(colc_to_f64) colc_to_f64;                                               \
    KG_INST_FN(ens_step) ens_step;            /* share 4: ensemble step */             \
    KG_INST_FN(ens_blocks_per_sm) ens_blocks_per_sm;                                   \
    }

namespace kg {
KG_INST_DECLARE(inst_f64)
KG_INST_DECLARE(inst_df)
KG_INST_DECLARE(inst_f32)
}  // namespace kg
