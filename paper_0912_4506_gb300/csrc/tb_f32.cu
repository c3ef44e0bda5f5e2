// FP32 kernels: plain streaming sweep and temporally-blocked sweep (depth 1 on
// 128 x 12 extended tiles, the fastest one-sweep-per-pass shape at 512^3; deeper
// passes on 64 x 32 tiles).
#include "tb_inst.cuh"

namespace jac {

static const TBEntry kTB[] = {
    JAC_TB(F32, 4, 12, 1, MODE_PLAIN, 6), JAC_TB(F32, 2, 32, 2, MODE_PLAIN, 6),
    JAC_TB(F32, 2, 32, 3, MODE_PLAIN, 6), JAC_TB(F32, 2, 32, 4, MODE_PLAIN, 6),
    JAC_TB(F32, 2, 32, 5, MODE_PLAIN, 6), JAC_TB(F32, 2, 32, 6, MODE_PLAIN, 6),
    JAC_TB(F32, 2, 32, 7, MODE_PLAIN, 6), JAC_TB(F32, 2, 32, 8, MODE_PLAIN, 6),
};
JAC_TABLE(tb_entries_f32, kTB)

static const PlainEntry kPlain = JAC_PLAIN(F32, 4, 8, 0);
const PlainEntry* plain_entry_f32() { return &kPlain; }

}  // namespace jac
