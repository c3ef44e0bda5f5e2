// FP64 pipelined (wavefront) kernel: 64 x 8 tiles (V = 2, the streaming sweep's
// shape), four of the five additions of every update on the integer pipes
// (accumulator word form 3) when the range check allows it.
#include "wave_inst.cuh"

namespace jac {

static const WaveEntry kWave = JAC_WAVE(F64, 2, 8, kAccBaseWave + 4 + 8 * 3, 3);
const WaveEntry* wave_entry_f64() { return &kWave; }

}  // namespace jac
