// FP32 adjoint (transpose) sweeps with boundary-gradient accumulation.
#include "tb_inst.cuh"

namespace jac {

// depths 1..4: deeper passes need more registers than 1024-thread CTAs have
// (they spill) and run slower than depth 4
static const TBEntry kTB[] = {
    JAC_TB(F32, 2, 32, 1, MODE_ADJ, 6),
    JAC_TB(F32, 2, 32, 2, MODE_ADJ, 6),
    JAC_TB(F32, 2, 32, 3, MODE_ADJ, 6),
    JAC_TB(F32, 2, 32, 4, MODE_ADJ, 6),
};
JAC_TABLE(tb_entries_f32_adj, kTB)

}  // namespace jac
