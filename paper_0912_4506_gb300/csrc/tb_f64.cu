// FP64 kernels: plain streaming sweep and temporally-blocked sweep.  The blocked
// sweep carries the integer-pipe additions (3 of the 5 additions of an update,
// valid when the call's range check passes), like the plain sweep.
#include "tb_inst.cuh"

namespace jac {

// Extended tiles 64 x 32 (depths 1-2) and 64 x 24 (depths 3-4): the tallest
// whose registers fit without spills; depths 5-8 are in tb_f64_deep.cu.
static const TBEntry kTB[] = {
    JAC_TBE(F64, 2, 32, 1, MODE_PLAIN, 6, 20), JAC_TBE(F64, 2, 32, 2, MODE_PLAIN, 6, 20),
    JAC_TBE(F64, 2, 24, 3, MODE_PLAIN, 6, 20), JAC_TBE(F64, 2, 24, 4, MODE_PLAIN, 6, 20),
};
JAC_TABLE(tb_entries_f64, kTB)

// plain sweeps: entry 0 keeps every addition on the FP64 unit; 6 does 3 of the
// 5 additions one at a time on the integer pipes (emu.cuh); 16 + K + 8F sends the
// first K additions through the unpacked accumulator (emusum.cuh) in word form F,
// and + 32 compiles it for 5 resident CTAs per SM (at most 51 registers).  76
// (K = 4, F = 3, capped) measured fastest at 512^3 on GB300: 202 GLUP/s, against
// 200 for F = 2 capped, 195 for F = 1 capped, 194 for F = 0 capped, 197 for F = 0,
// 167 / 156 with K = 3 / 5, 166 for entry 6 and 85 for entry 0.
static const PlainEntry kPlain[] = {JAC_PLAIN(F64, 2, 8, 0),  JAC_PLAIN(F64, 2, 8, 6),
                                    JAC_PLAIN(F64, 2, 8, 19), JAC_PLAIN(F64, 2, 8, 20),
                                    JAC_PLAIN(F64, 2, 8, 21), JAC_PLAIN(F64, 2, 8, 44),
                                    JAC_PLAIN(F64, 2, 8, 52), JAC_PLAIN(F64, 2, 8, 76)};
const PlainEntry* plain_entries_f64(int* n) {
    *n = (int)(sizeof(kPlain) / sizeof(kPlain[0]));
    return kPlain;
}
const PlainEntry* plain_entry_f64() { return &kPlain[0]; }

}  // namespace jac
