// bf16-storage correction sweeps of the iterative refinement.
#include "tb_inst.cuh"

namespace jac {

// depths 1..4: deeper passes need more registers than 1024-thread CTAs have
// (they spill) and run slower than depth 4
static const TBEntry kTB[] = {
    JAC_TB(BF16, 2, 32, 1, MODE_RHS, 6),
    JAC_TB(BF16, 2, 32, 2, MODE_RHS, 6),
    JAC_TB(BF16, 2, 32, 3, MODE_RHS, 6),
    JAC_TB(BF16, 2, 32, 4, MODE_RHS, 6),
};
JAC_TABLE(tb_entries_bf16_rhs, kTB)

}  // namespace jac
