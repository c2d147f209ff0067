// k_stage_s3.cu — the stage kernel for 32 x 16-block evaluation tiles, 512 threads per CTA
// (twice the registers per thread of the 1024-thread build: no spills, half the warps);
// the sweep schedule's CTA walk.
#define RAPID_TILE_W 32
#define RAPID_TILE_H 16
#define RAPID_THREADS 512
#define RAPID_SWEEP_CTA 1
#define RAPID_SHAPE_NS s3
#include "stage_impl.cuh"
