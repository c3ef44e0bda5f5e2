// FP32 and bf16 pipelined (wavefront) kernels: 128 x 8 tiles (16-byte vectors of
// four FP32 cells, 8-byte vectors of four bf16 cells), as the streaming sweep.
// The first entry of a table is the default, the fastest measured at 512^3: the
// TMA-staged march at four CTAs per SM (FP32 605 GLUP/s at t = 1 and 484 at t = 4,
// against 540 / 425 at five CTAs per SM and 424 / 416 for the register march; bf16
// 516 / 410 against 419 / 388).  The others are alternates for measurement runs.
#include "wave_inst.cuh"

namespace jac {

static const WaveEntry kWaveF32[] = {
    JAC_WAVE(F32, 4, 8, 0, 4, 1),
    JAC_WAVE(F32, 4, 8, 0, 5, 1),
    JAC_WAVE(F32, 4, 8, 0, 3, 0),
};
static const WaveEntry kWaveBF16[] = {
    JAC_WAVE(BF16, 4, 8, 0, 4, 1),
    JAC_WAVE(BF16, 4, 8, 0, 5, 1),
    JAC_WAVE(BF16, 4, 8, 0, 4, 0),
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
