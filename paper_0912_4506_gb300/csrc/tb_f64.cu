// FP64 kernels: plain streaming sweep and temporally-blocked sweep.  The blocked
// sweep carries the integer-pipe additions (3 of the 5 additions of an update,
// valid when the call's range check passes), like the plain sweep.
#include "tb_inst.cuh"

namespace jac {

// Extended tiles 64 x 32 (depths 1-2) and 64 x 24 (depths 3-4): the tallest
// whose registers fit without spills; depths 5-8 are in tb_f64_deep.cu.
static const TBEntry kTB[] = {
    JAC_TBE(F64, 2, 32, 1, MODE_PLAIN, 6, 3), JAC_TBE(F64, 2, 32, 2, MODE_PLAIN, 6, 3),
    JAC_TBE(F64, 2, 24, 3, MODE_PLAIN, 6, 3), JAC_TBE(F64, 2, 24, 4, MODE_PLAIN, 6, 3),
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
