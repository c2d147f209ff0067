// k_stage_s4.cu — the stage kernel for 32 x 8-block evaluation tiles, 512 threads per CTA
// (twice the registers per thread of the 1024-thread build: no spills, half the warps);
// the sweep schedule's warp walk.
#define RAPID_TILE_W 32
#define RAPID_TILE_H 8
#define RAPID_THREADS 512
#define RAPID_SWEEP_CTA 0
#define RAPID_SHAPE_NS s4
#include "stage_impl.cuh"
