// FP32 correction sweeps of the iterative refinement (temporally blocked).
#include "tb_inst.cuh"

namespace jac {

// depths 1..4: deeper passes need more registers than 1024-thread CTAs have
// (they spill) and run slower than depth 4
static const TBEntry kTB[] = {
    JAC_TB(F32, 2, 32, 1, MODE_RHS, 6),
    JAC_TB(F32, 2, 32, 2, MODE_RHS, 6),
    JAC_TB(F32, 2, 32, 3, MODE_RHS, 6),
    JAC_TB(F32, 2, 32, 4, MODE_RHS, 6),
};
JAC_TABLE(tb_entries_f32_rhs, kTB)

}  // namespace jac
