// FP32 adjoint (transpose) sweeps with boundary-gradient accumulation.
#include "tb_inst.cuh"

namespace jac {

// The adjoint k-march is the plain sweep on a zero boundary; the face values
// leave through shared memory after each step, and the registers they need on
// top of a 128-wide march cost a CTA per SM (or spill) at depths 2-4, where 64 x 32
// tiles measured faster (256^3, 50 sweeps: 460 / 500 / 420 GLUP/s at depths 2 / 3
// / 4 against 359 / 403 / 345 for 128-wide tiles); depth 1 takes 128 x 12.
static const TBEntry kTB[] = {
    JAC_TB(F32, 4, 12, 1, MODE_ADJ, 6),
    JAC_TB(F32, 2, 32, 2, MODE_ADJ, 6),
    JAC_TB(F32, 2, 32, 3, MODE_ADJ, 6),
    JAC_TB(F32, 2, 32, 4, MODE_ADJ, 6),
};
JAC_TABLE(tb_entries_f32_adj, kTB)

}  // namespace jac
