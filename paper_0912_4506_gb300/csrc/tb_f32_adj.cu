// FP32 adjoint (transpose) sweeps with boundary-gradient accumulation.
#include "tb_inst.cuh"

namespace jac {

static const TBEntry kTB[] = {
    JAC_TB(F32, 2, 32, 1, MODE_ADJ, 6), JAC_TB(F32, 2, 32, 2, MODE_ADJ, 6),
    JAC_TB(F32, 2, 32, 3, MODE_ADJ, 6), JAC_TB(F32, 2, 32, 4, MODE_ADJ, 6),
    JAC_TB(F32, 2, 32, 5, MODE_ADJ, 6), JAC_TB(F32, 2, 32, 6, MODE_ADJ, 6),
    JAC_TB(F32, 2, 32, 7, MODE_ADJ, 6), JAC_TB(F32, 2, 32, 8, MODE_ADJ, 6),
};
JAC_TABLE(tb_entries_f32_adj, kTB)

}  // namespace jac
