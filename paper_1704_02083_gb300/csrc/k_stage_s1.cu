// k_stage_s1.cu — the stage kernel for 32 x 8-block evaluation tiles; the sweep schedule's
// warp walk.
#define RAPID_TILE_W 32
#define RAPID_TILE_H 8
#define RAPID_SWEEP_CTA 0
#define RAPID_SHAPE_NS s1
#include "stage_impl.cuh"
