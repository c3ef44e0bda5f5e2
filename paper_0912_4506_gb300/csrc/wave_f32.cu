// FP32 and bf16 pipelined (wavefront) kernels: 128 x 8 tiles (16-byte vectors of
// four FP32 cells, 8-byte vectors of four bf16 cells), as the streaming sweep.
#include "wave_inst.cuh"

namespace jac {

static const WaveEntry kWaveF32 = JAC_WAVE(F32, 4, 8, 0, 3);
static const WaveEntry kWaveBF16 = JAC_WAVE(BF16, 4, 8, 0, 3);
const WaveEntry* wave_entry_f32() { return &kWaveF32; }
const WaveEntry* wave_entry_bf16() { return &kWaveBF16; }

}  // namespace jac
