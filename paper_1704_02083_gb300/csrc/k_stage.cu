// k_stage.cu — dispatch of the stage kernel over its evaluation-tile shapes (kShapes in
// rapid_dev.cuh; one translation unit per shape).
#include "../../include/rapid.h"
#include "rapid_dev.cuh"

#include <mutex>
#include <vector>

namespace rapid {
#define RAPID_SHAPE_DECL(NS)                                  \
  const void *stage_kernel_ptr_##NS(bool batch, bool frontier, bool cluster); \
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
    case 1: return stage_kernel_ptr_s1(batch, frontier, false);
    case 2: return stage_kernel_ptr_s2(batch, frontier, false);
    case 3: return stage_kernel_ptr_s3(batch, frontier, false);
    case 4: return stage_kernel_ptr_s4(batch, frontier, false);
    case 5: return stage_kernel_ptr_s5(batch, frontier, false);
    default: return stage_kernel_ptr_s0(batch, frontier, false);
  }
}

// Cluster support per (kernel, device): the largest cluster size found to fit (16, 8 or 0).
namespace {
struct ClusterFit {
  const void *fn;
  int device, block, max_size;
};
std::mutex g_cluster_mu;
std::vector<ClusterFit> g_cluster_fit;

int cluster_fit(const void *fn, int block) {
  for (int size : {kMaxCluster, 8}) {
    if (size > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(size);
    cfg.blockDim = dim3(block);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (n >= 1) return size;
  }
  return 0;
}
}  // namespace

bool cluster_launch_ok(const void *fn, int grid, int block, cudaStream_t s) {
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lock(g_cluster_mu);
  for (const ClusterFit &c : g_cluster_fit)
    if (c.fn == fn && c.device == device && c.block == block) return grid <= c.max_size;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return false;
  }
  g_cluster_fit.push_back({fn, device, block, cluster_fit(fn, block)});
  return grid <= g_cluster_fit.back().max_size;
}

const void *stage_cluster_kernel_ptr(bool frontier, int shape) {
  switch (shape) {
    case 1: return stage_kernel_ptr_s1(false, frontier, true);
    case 2: return stage_kernel_ptr_s2(false, frontier, true);
    case 3: return stage_kernel_ptr_s3(false, frontier, true);
    case 4: return stage_kernel_ptr_s4(false, frontier, true);
    case 5: return stage_kernel_ptr_s5(false, frontier, true);
    default: return stage_kernel_ptr_s0(false, frontier, true);
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

// Three scripted write sequences through the race check on a 6 x 6 block grid, one phase
// each (g = 1, 2, 3): class-0 blocks 3 apart (no violation); a class-0 block, then a block 2
// to its right (wrong class, and within distance 2 of the first: two); the same block twice
// (one).
__global__ void race_selftest_kernel(int *wstamp, unsigned long long *out) {
  for (int i = 0; i < 36; i++) wstamp[i] = 0;
  const int A[4][2] = {{0, 0}, {3, 0}, {0, 3}, {3, 3}}, B[2][2] = {{0, 0}, {2, 0}}, Cw[2][2] = {{3, 3}, {3, 3}};
  for (int i = 0; i < 4; i++) race_check(out + 0, wstamp, 0, 6, 6, A[i][0], A[i][1], 1, 0);
  for (int i = 0; i < 2; i++) race_check(out + 1, wstamp, 0, 6, 6, B[i][0], B[i][1], 2, 0);
  for (int i = 0; i < 2; i++) race_check(out + 2, wstamp, 0, 6, 6, Cw[i][0], Cw[i][1], 3, 0);
}

}  // namespace rapid

extern "C" rapid_status rapid_race_selftest(int64_t *violations3) {
  if (!violations3) return RAPID_EINVAL;
  int *w = nullptr;
  unsigned long long *v = nullptr;
  rapid_status rs = RAPID_OK;
  if (cudaMalloc(&w, 36 * sizeof(int)) != cudaSuccess || cudaMalloc(&v, 3 * sizeof(unsigned long long)) != cudaSuccess)
    rs = RAPID_ENOMEM;
  unsigned long long h[3] = {0, 0, 0};
  if (rs == RAPID_OK && (cudaMemset(v, 0, sizeof h) != cudaSuccess ||
                         (rapid::race_selftest_kernel<<<1, 1>>>(w, v), cudaGetLastError()) != cudaSuccess ||
                         cudaMemcpy(h, v, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess))
    rs = RAPID_ECUDA;
  cudaFree(w);
  cudaFree(v);
  for (int i = 0; i < 3; i++) violations3[i] = (int64_t)h[i];
  return rs;
}
