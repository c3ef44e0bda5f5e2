// FP64 temporally-blocked sweeps of depth 5-8.  Three register planes per level
// and cell limit these depths to one cell per lane (extended tiles 32 x 32 and
// 32 x 24), so most of each pass is halo recompute: they exist for completeness
// of the depth range, and the planner's default for FP64 stays the plain sweep.
#include "tb_inst.cuh"

namespace jac {

static const TBEntry kTB[] = {
    JAC_TBE(F64, 1, 32, 5, MODE_PLAIN, 6, 20), JAC_TBE(F64, 1, 32, 6, MODE_PLAIN, 6, 20),
    JAC_TBE(F64, 1, 24, 7, MODE_PLAIN, 6, 20), JAC_TBE(F64, 1, 24, 8, MODE_PLAIN, 6, 20),
};
JAC_TABLE(tb_entries_f64_deep, kTB)

}  // namespace jac
