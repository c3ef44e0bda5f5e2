// FP64 kernels: plain streaming sweep, temporally-blocked sweep, adjoint sweep.
#include "tb_inst.cuh"

namespace jac {

static const TBEntry kTB[] = {
    JAC_TB(F64, 2, 16, 1, MODE_PLAIN, 6), JAC_TB(F64, 2, 16, 2, MODE_PLAIN, 6),
    JAC_TB(F64, 2, 16, 3, MODE_PLAIN, 6), JAC_TB(F64, 2, 16, 4, MODE_PLAIN, 6),
    JAC_TB(F64, 2, 16, 1, MODE_ADJ, 6),   JAC_TB(F64, 2, 16, 2, MODE_ADJ, 6),
    JAC_TB(F64, 2, 16, 3, MODE_ADJ, 6),   JAC_TB(F64, 2, 16, 4, MODE_ADJ, 6),
};
JAC_TABLE(tb_entries_f64, kTB)

static const PlainEntry kPlain = JAC_PLAIN(F64, 1, 8);
const PlainEntry* plain_entry_f64() { return &kPlain; }

}  // namespace jac
