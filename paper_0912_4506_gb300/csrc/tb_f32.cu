// FP32 kernels: plain streaming sweep and temporally-blocked sweep.
#include "tb_inst.cuh"

namespace jac {

static const TBEntry kTB[] = {
    JAC_TB(F32, 2, 32, 1, MODE_PLAIN, 6), JAC_TB(F32, 2, 32, 2, MODE_PLAIN, 6),
    JAC_TB(F32, 2, 32, 3, MODE_PLAIN, 6), JAC_TB(F32, 2, 32, 4, MODE_PLAIN, 6),
    JAC_TB(F32, 2, 32, 5, MODE_PLAIN, 6), JAC_TB(F32, 2, 32, 6, MODE_PLAIN, 6),
    JAC_TB(F32, 2, 32, 7, MODE_PLAIN, 6), JAC_TB(F32, 2, 32, 8, MODE_PLAIN, 6),
};
JAC_TABLE(tb_entries_f32, kTB)

static const PlainEntry kPlain = JAC_PLAIN(F32, 4, 8, 0);
const PlainEntry* plain_entry_f32() { return &kPlain; }

}  // namespace jac
