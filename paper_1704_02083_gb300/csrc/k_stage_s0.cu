// k_stage_s0.cu — the stage kernel for 32 x 16-block evaluation tiles; the sweep schedule's
// CTA walk.
#define RAPID_TILE_W 32
#define RAPID_TILE_H 16
#define RAPID_SWEEP_CTA 1
#define RAPID_SHAPE_NS s0
#include "stage_impl.cuh"
