// k_stage.cu — dispatch of the stage kernel over its evaluation-tile shapes (kShapes in
// rapid_dev.cuh; one translation unit per shape).
#include "rapid_dev.cuh"

namespace rapid {
const void *stage_kernel_ptr_s0(bool batch);
const void *stage_kernel_ptr_s1(bool batch);
const void *stage_kernel_ptr_s2(bool batch);
cudaError_t launch_stage_s0(const StageArgs &a, int grid, int block, cudaStream_t s);
cudaError_t launch_stage_s1(const StageArgs &a, int grid, int block, cudaStream_t s);
cudaError_t launch_stage_s2(const StageArgs &a, int grid, int block, cudaStream_t s);
static_assert(kNumShapes == 3, "one entry per compiled shape");

int stage_block_threads() { return 1024; }

const void *stage_kernel_ptr(bool batch, int shape) {
  switch (shape) {
    case 1: return stage_kernel_ptr_s1(batch);
    case 2: return stage_kernel_ptr_s2(batch);
    default: return stage_kernel_ptr_s0(batch);
  }
}

cudaError_t launch_stage(const StageArgs &a, int grid, int block, cudaStream_t s, int shape) {
  switch (shape) {
    case 1: return launch_stage_s1(a, grid, block, s);
    case 2: return launch_stage_s2(a, grid, block, s);
    default: return launch_stage_s0(a, grid, block, s);
  }
}

}  // namespace rapid
