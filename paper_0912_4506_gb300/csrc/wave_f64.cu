// FP64 pipelined (wavefront) kernels: 64 x 8 tiles (V = 2, the streaming sweep's
// shape), four of the five additions of every update on the integer pipes
// (accumulator word form 3) when the range check allows it.  The first entry is
// the default (four CTAs per SM: 144 GLUP/s at 512^3, t = 1, against 133 with
// three); the others are alternates for measurement runs.
#include "wave_inst.cuh"

namespace jac {

static const WaveEntry kWave[] = {
    JAC_WAVE(F64, 2, 8, kAccBaseWave + 4 + 8 * 3, 4, 0),
    JAC_WAVE(F64, 2, 8, kAccBaseWave + 4 + 8 * 3, 3, 0),
};
const WaveEntry* wave_entries_f64(int* n) {
    *n = (int)(sizeof(kWave) / sizeof(kWave[0]));
    return kWave;
}

}  // namespace jac
