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

// plain sweeps with 0..4 of the additions on the integer pipes, in half
// additions per plane (see plain_march); entry 0 is the all-FP64-unit kernel
static const PlainEntry kPlain[] = {JAC_PLAIN(F64, 2, 8, 0), JAC_PLAIN(F64, 2, 8, 2),
                                    JAC_PLAIN(F64, 2, 8, 4), JAC_PLAIN(F64, 2, 8, 5),
                                    JAC_PLAIN(F64, 2, 8, 6), JAC_PLAIN(F64, 2, 8, 7),
                                    JAC_PLAIN(F64, 2, 8, 8)};
const PlainEntry* plain_entries_f64(int* n) {
    *n = (int)(sizeof(kPlain) / sizeof(kPlain[0]));
    return kPlain;
}
const PlainEntry* plain_entry_f64() { return &kPlain[0]; }

}  // namespace jac
