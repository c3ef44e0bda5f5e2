// FP32 and bf16 pipelined (wavefront) kernels: 128 x 8 tiles (16-byte vectors of
// four FP32 cells, 8-byte vectors of four bf16 cells), as the streaming sweep.
// The first entry of a table is the default, the fastest measured at 512^3
// (FP32: three CTAs per SM, 424 GLUP/s at t = 1 against 396 with four; bf16: four,
// 419 against 382); the others are alternates for measurement runs.
#include "wave_inst.cuh"

namespace jac {

static const WaveEntry kWaveF32[] = {
    JAC_WAVE(F32, 4, 8, 0, 3),
    JAC_WAVE(F32, 4, 8, 0, 4),
};
static const WaveEntry kWaveBF16[] = {
    JAC_WAVE(BF16, 4, 8, 0, 4),
    JAC_WAVE(BF16, 4, 8, 0, 3),
};
const WaveEntry* wave_entries_f32(int* n) {
    *n = (int)(sizeof(kWaveF32) / sizeof(kWaveF32[0]));
    return kWaveF32;
}
const WaveEntry* wave_entries_bf16(int* n) {
    *n = (int)(sizeof(kWaveBF16) / sizeof(kWaveBF16[0]));
    return kWaveBF16;
}

}  // namespace jac
