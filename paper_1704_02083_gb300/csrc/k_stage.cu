// k_stage.cu — dispatch of the stage kernel over its evaluation-tile shapes (kShapes in
// rapid_dev.cuh; one translation unit per shape).
#include "rapid_dev.cuh"

namespace rapid {
#define RAPID_SHAPE_DECL(NS)                                  \
  const void *stage_kernel_ptr_##NS(bool batch, bool frontier); \
  cudaError_t launch_stage_##NS(const StageArgs &a, int grid, int block, cudaStream_t s);
RAPID_SHAPE_DECL(s0)
RAPID_SHAPE_DECL(s1)
RAPID_SHAPE_DECL(s2)
RAPID_SHAPE_DECL(s3)
RAPID_SHAPE_DECL(s4)
RAPID_SHAPE_DECL(s5)
static_assert(kNumShapes == 6, "one entry per compiled shape");

int stage_block_threads(int shape) { return kShapes[(shape >= 0 && shape < kNumShapes) ? shape : 0].threads; }

const void *stage_kernel_ptr(bool batch, bool frontier, int shape) {
  switch (shape) {
    case 1: return stage_kernel_ptr_s1(batch, frontier);
    case 2: return stage_kernel_ptr_s2(batch, frontier);
    case 3: return stage_kernel_ptr_s3(batch, frontier);
    case 4: return stage_kernel_ptr_s4(batch, frontier);
    case 5: return stage_kernel_ptr_s5(batch, frontier);
    default: return stage_kernel_ptr_s0(batch, frontier);
  }
}

cudaError_t launch_stage(const StageArgs &a, int grid, int block, cudaStream_t s, int shape) {
  switch (shape) {
    case 1: return launch_stage_s1(a, grid, block, s);
    case 2: return launch_stage_s2(a, grid, block, s);
    case 3: return launch_stage_s3(a, grid, block, s);
    case 4: return launch_stage_s4(a, grid, block, s);
    case 5: return launch_stage_s5(a, grid, block, s);
    default: return launch_stage_s0(a, grid, block, s);
  }
}

}  // namespace rapid
