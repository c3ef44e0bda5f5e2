// bf16 temporally-blocked sweeps with two rows per thread (512-thread CTAs),
// compiled at the depths where they run faster than one row per thread.
#include "tb_inst.cuh"

namespace jac {

static const TBEntry kTB[] = {
    JAC_TBR(BF16, 2, 16, 2, 2, MODE_PLAIN, 6),
    JAC_TBM(BF16, 2, 16, 2, 3, MODE_PLAIN, 6, 2),
};
JAC_TABLE(tb_entries_bf16_rows, kTB)

}  // namespace jac
