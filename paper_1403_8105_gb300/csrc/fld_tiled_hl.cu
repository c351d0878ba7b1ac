// fld_tiled_hl.cu -- the hi/lo-family instances of the temporally blocked
// sweeps (fld_tiled.cu), compiled as a translation unit of their own so the
// two halves of the kernel instances build in parallel.
#define FLD_TILED_HL_ONLY 1
#include "fld_tiled.cu"
