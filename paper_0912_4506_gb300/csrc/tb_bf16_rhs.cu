// bf16-storage correction sweeps of the iterative refinement.
#include "tb_inst.cuh"

namespace jac {

// the right-hand side is staged in shared memory by TMA (NS + T slots), which
// bounds the depth at 6 (227 KB of shared memory per CTA for FP32) and the tiles
// at 128 x 20 for depths 3-4; shapes per depth measured at 512^3 on GB300
static const TBEntry kTB[] = {
    JAC_TB(BF16, 2, 32, 1, MODE_RHS, 6), JAC_TB(BF16, 4, 16, 2, MODE_RHS, 6),
    JAC_TB(BF16, 4, 20, 3, MODE_RHS, 6), JAC_TB(BF16, 4, 20, 4, MODE_RHS, 6),
    JAC_TB(BF16, 2, 32, 5, MODE_RHS, 6), JAC_TB(BF16, 2, 32, 6, MODE_RHS, 6),
};
JAC_TABLE(tb_entries_bf16_rhs, kTB)

}  // namespace jac
