// bf16-storage kernels (FP32 arithmetic): plain streaming sweep and
// temporally-blocked sweep (tile shapes per depth as for FP32).
#include "tb_inst.cuh"

namespace jac {

static const TBEntry kTB[] = {
    JAC_TB(BF16, 4, 12, 1, MODE_PLAIN, 6), JAC_TB(BF16, 4, 16, 2, MODE_PLAIN, 6),
    JAC_TB(BF16, 4, 32, 3, MODE_PLAIN, 6), JAC_TB(BF16, 4, 24, 4, MODE_PLAIN, 6),
    JAC_TB(BF16, 2, 32, 5, MODE_PLAIN, 6), JAC_TB(BF16, 2, 32, 6, MODE_PLAIN, 6),
    JAC_TB(BF16, 2, 32, 7, MODE_PLAIN, 6), JAC_TB(BF16, 2, 32, 8, MODE_PLAIN, 6),
};
JAC_TABLE(tb_entries_bf16, kTB)

static const PlainEntry kPlain = JAC_PLAIN(BF16, 4, 8, 0);
const PlainEntry* plain_entry_bf16() { return &kPlain; }

}  // namespace jac
