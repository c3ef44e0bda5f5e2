// FP32 temporally-blocked sweeps with two rows per thread (512-thread CTAs),
// compiled at the depths where they run faster than one row per thread: depth 2
// (60 registers, two CTAs per SM) and depth 3 (registers capped for two CTAs per
// SM, a few spilled).
#include "tb_inst.cuh"

namespace jac {

static const TBEntry kTB[] = {
    JAC_TBR(F32, 2, 16, 2, 2, MODE_PLAIN, 6),
    JAC_TBM(F32, 2, 16, 2, 3, MODE_PLAIN, 6, 2),
    JAC_TBM(F32, 2, 16, 2, 3, MODE_ADJ, 6, 2),
};
JAC_TABLE(tb_entries_f32_rows, kTB)

}  // namespace jac
