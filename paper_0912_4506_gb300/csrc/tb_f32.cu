// FP32 kernels: plain streaming sweep and temporally-blocked sweep.  Extended tile
// per depth (32*V x NW), the fastest measured at 512^3 on GB300 in sweeps of V in
// {2, 4, 8} and NW in 6..32: 128 x 12, 128 x 16, 128 x 32, 128 x 24, then 64 x 32.
// Wider tiles cut the x halo (OX/EX = 124/128 against 60/64); NW is set by the
// registers of the depth (one or two CTAs per SM).
#include "tb_inst.cuh"

namespace jac {

static const TBEntry kTB[] = {
    JAC_TB(F32, 4, 12, 1, MODE_PLAIN, 6), JAC_TB(F32, 4, 16, 2, MODE_PLAIN, 6),
    JAC_TB(F32, 4, 32, 3, MODE_PLAIN, 6), JAC_TB(F32, 4, 24, 4, MODE_PLAIN, 6),
    JAC_TB(F32, 2, 32, 5, MODE_PLAIN, 6), JAC_TB(F32, 2, 32, 6, MODE_PLAIN, 6),
    JAC_TB(F32, 2, 32, 7, MODE_PLAIN, 6), JAC_TB(F32, 2, 32, 8, MODE_PLAIN, 6),
};
JAC_TABLE(tb_entries_f32, kTB)

static const PlainEntry kPlain = JAC_PLAIN(F32, 4, 8, 0);
const PlainEntry* plain_entry_f32() { return &kPlain; }

}  // namespace jac
