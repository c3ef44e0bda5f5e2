// FP64 adjoint (transpose) sweeps with boundary-gradient accumulation.
#include "tb_inst.cuh"

namespace jac {

static const TBEntry kTB[] = {
    JAC_TB(F64, 2, 16, 1, MODE_ADJ, 6), JAC_TB(F64, 2, 16, 2, MODE_ADJ, 6),
    JAC_TB(F64, 2, 16, 3, MODE_ADJ, 6), JAC_TB(F64, 2, 16, 4, MODE_ADJ, 6),
};
JAC_TABLE(tb_entries_f64_adj, kTB)

}  // namespace jac
