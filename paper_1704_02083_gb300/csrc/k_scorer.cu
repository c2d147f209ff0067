// k_scorer.cu — the learned block scorer: a 3-layer 3x3 convolutional net over per-block
// features that predicts which boundary blocks will move in a stage, used only to prune
// which blocks the exact topology and energy tests evaluate (never to decide a move).
// Inference, training-data logging and training are all kernels of this file.
//
// Features of block p (label a, block mean colour c_p, snapshot means c_k of S):
//   f0..f3  for the N, W, E, S neighbour k (when it exists and k != a):
//           (|c_p - c_a| - |c_p - c_k|) / 64, the colour gain of moving to k; else 0
//   f4      boundary count: neighbours with another label / 4
//   f5      level / L
//   f6      coarse importance of a (1 before prediction)
//   f7      log2(block side) / 8
//   f8      |c_p - c_a| / 64, the block's misfit to its own superpixel
// Net: conv3x3(9 -> 16) ReLU, conv3x3(16 -> 16) ReLU, conv3x3(16 -> 1), sigmoid; every layer
// pads with zeros outside the image.  Weights and activations are rounded to bf16, sums are
// fp32.  Parameters (canonical float order): W1[16][9][3][3], b1[16], W2[16][16][3][3],
// b2[16], W3[16][3][3], b3.
#include <cuda_bf16.h>

#include <climits>
#include <cstring>

#include "../../include/rapid.h"
#include "rapid_dev.cuh"

namespace rapid {

static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int kFeat = 9, kHid = 16, kCh = 16;  // kCh: padded input channels of layer 1
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kFeat * 9, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid * 9, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * 9,
              kNParams = kOffB3 + 1;
static_assert(kNParams == RAPID_SCORER_PARAMS, "parameter count");

// Device form of the weights (ScorerDev): bf16 [tap][co][ci] for the two tensor-core
// layers (ci padded to 16), bf16-rounded fp32 [tap][ci] for the last layer, fp32 biases.
constexpr size_t kScorerDevBytes = 2 * 9 * 16 * 16 * sizeof(__nv_bfloat16) + (9 * 16 + 32) * sizeof(float);

// ---------------------------------------------------------------- features
__device__ __forceinline__ float dist3(float x0, float x1, float x2, float y0, float y1, float y2) {
  const float d0 = x0 - y0, d1 = x1 - y1, d2 = x2 - y2;
  return sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
}

__device__ __forceinline__ void label_mean(const DevStats &s, int k, float &r, float &g, float &b) {
  const float n = (float)s.N[k];
  r = n > 0.f ? (float)s.R[k] / n : 0.f;
  g = n > 0.f ? (float)s.G[k] / n : 0.f;
  b = n > 0.f ? (float)s.B[k] / n : 0.f;
}

// The 9 features of block (bx, by) of image im at the stage of a (zeros outside the image).
__device__ void block_features(const StageArgs &a, const ImageDesc &im, int L, int bx, int by, float f[kFeat]) {
  for (int i = 0; i < kFeat; i++) f[i] = 0.f;
  if (bx < 0 || by < 0 || bx >= im.nbx || by >= im.nby) return;
  const int *lab = im.lab;
  const long long i0 = (long long)by * im.nbx + bx;
  const int la = lab[i0];
  const int nb[4] = {by > 0 ? lab[i0 - im.nbx] : -1, bx > 0 ? lab[i0 - 1] : -1, bx + 1 < im.nbx ? lab[i0 + 1] : -1,
                     by + 1 < im.nby ? lab[i0 + im.nbx] : -1};
  const BlockSums bs = block_sums(a, im, bx, by);
  const float w = (float)bs.w;
  const float pr = (float)bs.r / w, pg = (float)bs.g / w, pb = (float)bs.b / w;
  float ar, ag, ab;
  label_mean(a.st, la, ar, ag, ab);
  const float da = dist3(pr, pg, pb, ar, ag, ab);
  int nbound = 0;
  for (int j = 0; j < 4; j++) {
    const int k = nb[j];
    if (k < 0 || k == la) continue;
    nbound++;
    float kr, kg, kb;
    label_mean(a.st, k, kr, kg, kb);
    f[j] = (da - dist3(pr, pg, pb, kr, kg, kb)) * (1.f / 64.f);
  }
  f[4] = 0.25f * (float)nbound;
  f[5] = (float)a.level / (float)L;
  f[6] = a.imp_on ? (float)a.st.imp[la] : 1.f;
  f[7] = log2f((float)a.side) * 0.125f;
  f[8] = da * (1.f / 64.f);
}

__global__ void features_kernel(StageArgs a, ImageDesc im, int L, float *out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)im.nbx * im.nby) return;
  float f[kFeat];
  block_features(a, im, L, (int)(i % im.nbx), (int)(i / im.nbx), f);
  for (int c = 0; c < kFeat; c++) out[i * kFeat + c] = f[c];
}

// ---------------------------------------------------------------- inference
// D += A (16 x 16 bf16, row-major) * B (16 x 8 bf16, column-major), fp32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

constexpr int kOut = 16;             // output tile side (blocks)
constexpr int kG0 = kOut + 6;        // feature grid side (halo 3)
constexpr int kG1 = kOut + 4;        // layer-1 output side
constexpr int kG2 = kOut + 2;        // layer-2 output side
constexpr int kScoreThreads = 256;

// One 3x3 convolution layer on the tensor cores: in = gin x gin positions x 16 bf16
// channels (shared), out = gout x gout x 16 (gout = gin - 2), ReLU, positions outside the
// image (origin oy0, ox0 in block coordinates) set to zero.  Warps take 16-position rows
// of the implicit GEMM [positions x (9 taps x 16 ch)] x [(9 x 16) x 16].
__device__ __forceinline__ void conv_layer_tc(const __nv_bfloat16 *in, int gin, __nv_bfloat16 *out, int gout,
                                              const __nv_bfloat16 *w, const float *bias, int oy0, int ox0,
                                              int nbx, int nby) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int npos = gout * gout, ntile = (npos + 15) / 16;
  const unsigned *in32 = reinterpret_cast<const unsigned *>(in);
  const unsigned *w32 = reinterpret_cast<const unsigned *>(w);
  for (int mt = warp; mt < ntile; mt += nw) {
    const int m0 = min(mt * 16 + g, npos - 1), m1 = min(mt * 16 + g + 8, npos - 1);
    const int y0 = m0 / gout, x0 = m0 % gout, y1 = m1 / gout, x1 = m1 % gout;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int tap = 0; tap < 9; tap++) {
      const int dy = tap / 3, dx = tap % 3;
      const int p0 = ((y0 + dy) * gin + (x0 + dx)) * 8, p1 = ((y1 + dy) * gin + (x1 + dx)) * 8;  // 32-bit units
      const unsigned a0 = in32[p0 + t], a1 = in32[p1 + t], a2 = in32[p0 + 4 + t], a3 = in32[p1 + 4 + t];
#pragma unroll
      for (int nb = 0; nb < 2; nb++) {
        const int wo = (tap * 16 + nb * 8 + g) * 8;  // [tap][co][ci] in 32-bit units
        mma_bf16(acc[nb], a0, a1, a2, a3, w32[wo + t], w32[wo + 4 + t]);
      }
    }
    // bias, ReLU, zero outside the image, round to bf16
#pragma unroll
    for (int half = 0; half < 2; half++) {
      const int m = mt * 16 + g + 8 * half;
      if (m >= npos) continue;
      const int yy = m / gout, xx = m % gout;
      const int by = oy0 + yy, bx = ox0 + xx;
      const bool inside = by >= 0 && bx >= 0 && by < nby && bx < nbx;
#pragma unroll
      for (int nb = 0; nb < 2; nb++) {
        const int co = nb * 8 + 2 * t;
        const float v0 = inside ? fmaxf(acc[nb][2 * half] + bias[co], 0.f) : 0.f;
        const float v1 = inside ? fmaxf(acc[nb][2 * half + 1] + bias[co + 1], 0.f) : 0.f;
        out[m * 16 + co] = __float2bfloat16_rn(v0);
        out[m * 16 + co + 1] = __float2bfloat16_rn(v1);
      }
    }
  }
}

// Scores of one kOut x kOut tile of image im's blocks: features (with a 3-block halo) in
// shared memory, two tensor-core layers, the last layer per thread.  Writes the sigmoid
// score (if score != null) and the pruning mask (score >= threshold).
__global__ void __launch_bounds__(kScoreThreads, 4) score_kernel(StageArgs a, ImageDesc im, int L, ScorerDev W,
                                                              float threshold, float *score, unsigned char *mask) {
  __shared__ __align__(16) __nv_bfloat16 s_f[kG0 * kG0 * kCh];
  __shared__ __align__(16) __nv_bfloat16 s_h1[kG1 * kG1 * kHid];
  __shared__ __align__(16) __nv_bfloat16 s_h2[kG2 * kG2 * kHid];
  const int tx = blockIdx.x, ty = blockIdx.y;
  const int bx0 = tx * kOut, by0 = ty * kOut;
  for (int p = threadIdx.x; p < kG0 * kG0; p += blockDim.x) {
    float f[kFeat];
    block_features(a, im, L, bx0 - 3 + p % kG0, by0 - 3 + p / kG0, f);
    for (int c = 0; c < kCh; c++) s_f[p * kCh + c] = __float2bfloat16_rn(c < kFeat ? f[c] : 0.f);
  }
  __syncthreads();
  conv_layer_tc(s_f, kG0, s_h1, kG1, (const __nv_bfloat16 *)W.w1, W.b1, by0 - 2, bx0 - 2, im.nbx, im.nby);
  __syncthreads();
  conv_layer_tc(s_h1, kG1, s_h2, kG2, (const __nv_bfloat16 *)W.w2, W.b2, by0 - 1, bx0 - 1, im.nbx, im.nby);
  __syncthreads();
  const int oy = threadIdx.x / kOut, ox = threadIdx.x % kOut;
  const int by = by0 + oy, bx = bx0 + ox;
  if (by >= im.nby || bx >= im.nbx) return;
  float z = W.b3;
  for (int tap = 0; tap < 9; tap++) {
    const __nv_bfloat16 *h = s_h2 + ((oy + tap / 3) * kG2 + (ox + tap % 3)) * kHid;
    for (int ci = 0; ci < kHid; ci++) z += __bfloat162float(h[ci]) * W.w3[tap * kHid + ci];
  }
  const float sc = 1.f / (1.f + expf(-z));
  const long long i = (long long)by * im.nbx + bx;
  if (score) score[i] = sc;
  if (mask) mask[i] = sc >= threshold ? 1 : 0;
}

static_assert(kOut * kOut == kScoreThreads, "one thread per output block");

// ---------------------------------------------------------------- training data
// Per logged stage: the block labels at the stage start are kept; afterwards every block
// that was a boundary block at the start (feature f4 > 0) becomes a sample, labelled 1
// when its label changed during the stage.  Negatives are kept with probability neg_rate
// (a hash of image, stage and block decides, so the selection is reproducible).  A sample
// is its 7 x 7 x 9 feature patch (the net's receptive field) and a 7 x 7 in-image mask.
constexpr int kPatch = 7, kPatchFeat = kPatch * kPatch * kFeat;

static_assert(kScorerPatchFloats == kPatchFeat, "patch size");

__device__ __forceinline__ unsigned hash3(unsigned a, unsigned b, unsigned c) {
  unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u ^ (c + 0x165667B1u) * 0xC2B2AE3Du;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return h;
}

// Whether block i becomes a sample, and its label y.
__device__ __forceinline__ bool is_sample(const float *feat, const int *before, const int *after, long long i,
                                          int img, int stage, unsigned neg_threshold, float *y) {
  if (feat[i * kFeat + 4] <= 0.f) return false;  // not a boundary block at the stage start
  *y = before[i] != after[i] ? 1.f : 0.f;
  return *y != 0.f || hash3((unsigned)img, (unsigned)stage, (unsigned)i) <= neg_threshold;
}

// The samples of one logged stage take consecutive slots in block order, whatever the
// thread timing: a count per CTA of kCollectThreads blocks, an exclusive scan over those
// counts (one CTA), then each CTA writes its samples at its base plus their rank in it.
constexpr int kCollectThreads = 256, kScanThreads = 1024;

__global__ void __launch_bounds__(kCollectThreads) collect_count_kernel(const float *feat, const int *before,
                                                                         const int *after, long long nb, int img,
                                                                         int stage, unsigned neg_threshold,
                                                                         int *cta_count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float y;
  const bool take = i < nb && is_sample(feat, before, after, i, img, stage, neg_threshold, &y);
  const int c = __syncthreads_count(take);
  if (threadIdx.x == 0) cta_count[blockIdx.x] = c;
}

// cta_base[j] = *ts.count + sum of cta_count[0 .. j); then *ts.count grows by the total.
__global__ void __launch_bounds__(kScanThreads) collect_scan_kernel(const int *cta_count, int nctas, int *cta_base,
                                                                    TrainSet ts) {
  __shared__ long long s_part[kScanThreads];
  const int per = (nctas + kScanThreads - 1) / kScanThreads;
  const int b0 = threadIdx.x * per, b1 = min(nctas, b0 + per);
  long long sum = 0;
  for (int j = b0; j < b1; j++) sum += cta_count[j];
  s_part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive prefix over the threads' chunks, in order
    long long run = *ts.count;
    for (int t = 0; t < kScanThreads; t++) {
      const long long v = s_part[t];
      s_part[t] = run;
      run += v;
    }
    *ts.count = (int)min(run, (long long)INT_MAX);
  }
  __syncthreads();
  long long run = s_part[threadIdx.x];
  for (int j = b0; j < b1; j++) {
    cta_base[j] = (int)min(run, (long long)INT_MAX);
    run += cta_count[j];
  }
}

__global__ void __launch_bounds__(kCollectThreads) collect_write_kernel(const float *feat, const int *before,
                                                                         const int *after, int nbx, int nby, int img,
                                                                         int stage, unsigned neg_threshold,
                                                                         const int *cta_base, TrainSet ts) {
  __shared__ int s_warp[kCollectThreads / 32];
  const long long nb = (long long)nbx * nby;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float y = 0.f;
  const bool take = i < nb && is_sample(feat, before, after, i, img, stage, neg_threshold, &y);
  const unsigned ball = __ballot_sync(0xffffffffu, take);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_warp[warp] = __popc(ball);
  __syncthreads();
  int rank = __popc(ball & ((1u << lane) - 1u));
  for (int w = 0; w < warp; w++) rank += s_warp[w];
  if (!take) return;
  const long long slot = (long long)cta_base[blockIdx.x] + rank;
  if (slot >= ts.cap) return;  // the store is full: the extra samples are dropped
  const int bx = (int)(i % nbx), by = (int)(i / nbx);
  float *x = ts.x + slot * kPatchFeat;
  unsigned long long inb = 0;
  for (int p = 0; p < kPatch * kPatch; p++) {
    const int qx = bx - 3 + p % kPatch, qy = by - 3 + p / kPatch;
    const bool in = qx >= 0 && qy >= 0 && qx < nbx && qy < nby;
    if (in) inb |= 1ull << p;
    for (int c = 0; c < kFeat; c++) x[p * kFeat + c] = in ? feat[((long long)qy * nbx + qx) * kFeat + c] : 0.f;
  }
  ts.inb[slot] = inb;
  ts.y[slot] = y;
}

// ---------------------------------------------------------------- training
// Forward and backward of the net on one sample's patch, one warp per sample, fp32 with
// bf16-rounded weights, inputs and activations and fp32 biases (the inference precision),
// and fp32 master weights updated by Adam.  The bf16 roundings pass gradients through
// unchanged.  Loss: pos_weight * y * -log p + (1 - y) * -log(1 - p).
constexpr int kTrainWarps = 8, kTrainMaxCtas = 1024;

struct WarpScratch {
  float z1[25 * kHid], h1[25 * kHid];  // layer 1 on the 5 x 5 positions around the sample
  float z2[9 * kHid], h2[9 * kHid];    // layer 2 on the 3 x 3 positions
  float d2[9 * kHid], d1[25 * kHid];   // gradients of the pre-activations
  float x[kPatchFeat];
  float z3;
};

__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Gradients are summed in a fixed order, so that a training run is reproducible: each warp
// adds its samples' gradients, one after another, into a buffer of its own (every
// parameter of a sample is written by one lane), the CTA then adds its warps' buffers in
// warp order into its row of `part`, and train_reduce_kernel adds the rows in CTA order.
struct TrainSmem {
  float w[kNParams];
  float g[kTrainWarps][kNParams];
  float loss[kTrainWarps];
  WarpScratch ws[kTrainWarps];
};
constexpr size_t kTrainSmem = sizeof(TrainSmem);
static_assert(kTrainSmem <= 227 * 1024, "the training kernel's shared memory");

__global__ void __launch_bounds__(kTrainWarps * 32) train_grad_kernel(TrainSet ts, int n, const float *wmaster,
                                                                      const int *order, int off, int batch,
                                                                      float pos_weight, float *part,
                                                                      float *part_loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem &T = *reinterpret_cast<TrainSmem *>(smem_raw);
  float *s_w = T.w;
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) {  // bf16 weights, fp32 biases: the inference precision
    const bool bias = (i >= kOffB1 && i < kOffW2) || (i >= kOffB2 && i < kOffW3) || i == kOffB3;
    s_w[i] = bias ? wmaster[i] : bf(wmaster[i]);
  }
  for (int i = threadIdx.x; i < kTrainWarps * kNParams; i += blockDim.x) (&T.g[0][0])[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpScratch &S = T.ws[warp];
  float *s_g = T.g[warp];
  float lsum = 0.f;
  for (int b = blockIdx.x * kTrainWarps + warp; b < batch; b += gridDim.x * kTrainWarps) {
    const int sidx = order[(off + b) % n];
    const float *xg = ts.x + (long long)sidx * kPatchFeat;
    for (int i = lane; i < kPatchFeat; i += 32) S.x[i] = bf(xg[i]);
    const unsigned long long inb = ts.inb[sidx];
    const float y = ts.y[sidx];
    __syncwarp();
    // layer 1: 5 x 5 positions (patch offset 1) x 16 channels
    for (int j = lane; j < 25 * kHid; j += 32) {
      const int p = j / kHid, co = j % kHid, py = p / 5 + 1, px = p % 5 + 1;
      float z = s_w[kOffB1 + co];
      for (int tap = 0; tap < 9; tap++) {
        const int q = (py - 1 + tap / 3) * kPatch + (px - 1 + tap % 3);
        for (int ci = 0; ci < kFeat; ci++) z += S.x[q * kFeat + ci] * s_w[kOffW1 + (co * kFeat + ci) * 9 + tap];
      }
      const bool in = (inb >> (py * kPatch + px)) & 1ull;
      S.z1[j] = z;
      S.h1[j] = in ? bf(fmaxf(z, 0.f)) : 0.f;
    }
    __syncwarp();
    // layer 2: 3 x 3 positions (patch offset 2)
    for (int j = lane; j < 9 * kHid; j += 32) {
      const int p = j / kHid, co = j % kHid, py = p / 3, px = p % 3;  // in layer-1 coordinates (+1)
      float z = s_w[kOffB2 + co];
      for (int tap = 0; tap < 9; tap++) {
        const int q = (py + tap / 3) * 5 + (px + tap % 3);
        for (int ci = 0; ci < kHid; ci++) z += S.h1[q * kHid + ci] * s_w[kOffW2 + (co * kHid + ci) * 9 + tap];
      }
      const bool in = (inb >> ((py + 2) * kPatch + (px + 2))) & 1ull;
      S.z2[j] = z;
      S.h2[j] = in ? bf(fmaxf(z, 0.f)) : 0.f;
    }
    __syncwarp();
    // layer 3 and the loss
    float part = 0.f;
    for (int j = lane; j < 9 * kHid; j += 32) part += S.h2[j] * s_w[kOffW3 + (j % kHid) * 9 + j / kHid];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const float z3 = part + s_w[kOffB3];
    const float p = 1.f / (1.f + expf(-z3));
    const float dz3 = y > 0.5f ? pos_weight * (p - 1.f) : p;
    if (lane == 0) {
      lsum += y > 0.5f ? -pos_weight * logf(fmaxf(p, 1e-12f)) : -logf(fmaxf(1.f - p, 1e-12f));
      s_g[kOffB3] += dz3;
    }
    // layer 3 gradients; layer 2 pre-activation gradients
    for (int j = lane; j < 9 * kHid; j += 32) {
      const int p2 = j / kHid, ci = j % kHid;
      s_g[kOffW3 + ci * 9 + p2] += dz3 * S.h2[j];
      const bool in = (inb >> ((p2 / 3 + 2) * kPatch + (p2 % 3 + 2))) & 1ull;
      S.d2[j] = (in && S.z2[j] > 0.f) ? dz3 * s_w[kOffW3 + ci * 9 + p2] : 0.f;
    }
    __syncwarp();
    // layer 2 weight and bias gradients
    for (int j = lane; j < kHid * kHid * 9 + kHid; j += 32) {
      if (j < kHid * kHid * 9) {
        const int co = j / (kHid * 9), ci = (j / 9) % kHid, tap = j % 9;
        float gsum = 0.f;
        for (int p2 = 0; p2 < 9; p2++) {
          const int q = (p2 / 3 + tap / 3) * 5 + (p2 % 3 + tap % 3);
          gsum += S.d2[p2 * kHid + co] * S.h1[q * kHid + ci];
        }
        s_g[kOffW2 + j] += gsum;
      } else {
        const int co = j - kHid * kHid * 9;
        float gsum = 0.f;
        for (int p2 = 0; p2 < 9; p2++) gsum += S.d2[p2 * kHid + co];
        s_g[kOffB2 + co] += gsum;
      }
    }
    // layer 1 pre-activation gradients
    for (int j = lane; j < 25 * kHid; j += 32) {
      const int p1 = j / kHid, ci = j % kHid, py = p1 / 5, px = p1 % 5;
      float gsum = 0.f;
      for (int tap = 0; tap < 9; tap++) {
        const int qy = py - tap / 3, qx = px - tap % 3;  // layer-2 position using p1 at this tap
        if (qy < 0 || qx < 0 || qy > 2 || qx > 2) continue;
        for (int co = 0; co < kHid; co++) gsum += S.d2[(qy * 3 + qx) * kHid + co] * s_w[kOffW2 + (co * kHid + ci) * 9 + tap];
      }
      const bool in = (inb >> ((py + 1) * kPatch + (px + 1))) & 1ull;
      S.d1[j] = (in && S.z1[j] > 0.f) ? gsum : 0.f;
    }
    __syncwarp();
    // layer 1 weight and bias gradients
    for (int j = lane; j < kHid * kFeat * 9 + kHid; j += 32) {
      if (j < kHid * kFeat * 9) {
        const int co = j / (kFeat * 9), ci = (j / 9) % kFeat, tap = j % 9;
        float gsum = 0.f;
        for (int p1 = 0; p1 < 25; p1++) {
          const int q = (p1 / 5 + tap / 3) * kPatch + (p1 % 5 + tap % 3);
          gsum += S.d1[p1 * kHid + co] * S.x[q * kFeat + ci];
        }
        s_g[kOffW1 + j] += gsum;
      } else {
        const int co = j - kHid * kFeat * 9;
        float gsum = 0.f;
        for (int p1 = 0; p1 < 25; p1++) gsum += S.d1[p1 * kHid + co];
        s_g[kOffB1 + co] += gsum;
      }
    }
    __syncwarp();
  }
  if (lane == 0) T.loss[warp] = lsum;
  __syncthreads();
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) {
    float g = 0.f;
    for (int w = 0; w < kTrainWarps; w++) g += T.g[w][i];
    part[(long long)blockIdx.x * kNParams + i] = g;
  }
  if (threadIdx.x == 0) {
    float l = 0.f;
    for (int w = 0; w < kTrainWarps; w++) l += T.loss[w];
    part_loss[blockIdx.x] = l;
  }
}

// grad[i] = sum over the CTAs' rows in CTA order; *loss += their losses in the same order.
__global__ void train_reduce_kernel(const float *part, const float *part_loss, int ctas, float *grad, float *loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kNParams) {
    float g = 0.f;
    for (int c = 0; c < ctas; c++) g += part[(long long)c * kNParams + i];
    grad[i] = g;
  }
  if (i == 0) {
    float l = 0.f;
    for (int c = 0; c < ctas; c++) l += part_loss[c];
    *loss += l;
  }
}

// Adam on the fp32 master weights (gradient averaged over the batch).
__global__ void adam_kernel(float *w, float *m, float *v, float *grad, int n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2, float inv_batch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = grad[i] * inv_batch;
  m[i] = b1 * m[i] + (1.f - b1) * gi;
  v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
  w[i] -= lr * (m[i] / bc1) / (sqrtf(v[i] / bc2) + eps);
}

// ---------------------------------------------------------------- host helpers
static unsigned short f2bf_bits(float f) {  // round to nearest even (finite inputs)
  unsigned u;
  std::memcpy(&u, &f, 4);
  const unsigned r = u + 0x7FFFu + ((u >> 16) & 1u);
  return (unsigned short)(r >> 16);
}
static float bf_round(float f) {
  const unsigned u = (unsigned)f2bf_bits(f) << 16;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// Device form of canonical weights into buf (kScorerDevBytes, device memory).
cudaError_t scorer_upload(const float *wc, void *buf, ScorerDev *out, cudaStream_t s) {
  unsigned char host[kScorerDevBytes];
  std::memset(host, 0, sizeof host);
  unsigned short *w1 = (unsigned short *)host, *w2 = w1 + 9 * 16 * 16;
  float *w3 = (float *)(w2 + 9 * 16 * 16), *b1 = w3 + 9 * 16, *b2 = b1 + 16;
  for (int tap = 0; tap < 9; tap++)
    for (int co = 0; co < 16; co++)
      for (int ci = 0; ci < 16; ci++) {
        w1[(tap * 16 + co) * 16 + ci] = ci < kFeat ? f2bf_bits(wc[kOffW1 + (co * kFeat + ci) * 9 + tap]) : 0;
        w2[(tap * 16 + co) * 16 + ci] = f2bf_bits(wc[kOffW2 + (co * kHid + ci) * 9 + tap]);
      }
  for (int tap = 0; tap < 9; tap++)
    for (int ci = 0; ci < 16; ci++) w3[tap * 16 + ci] = bf_round(wc[kOffW3 + ci * 9 + tap]);
  for (int c = 0; c < 16; c++) {
    b1[c] = wc[kOffB1 + c];
    b2[c] = wc[kOffB2 + c];
  }
  // the copy must finish before `host` goes out of scope
  cudaError_t e = cudaMemcpyAsync(buf, host, kScorerDevBytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const __nv_bfloat16 *d = (const __nv_bfloat16 *)buf;
  out->w1 = d;
  out->w2 = d + 9 * 16 * 16;
  out->w3 = (const float *)(d + 2 * 9 * 16 * 16);
  out->b1 = out->w3 + 9 * 16;
  out->b2 = out->b1 + 16;
  out->b3 = wc[kOffB3];
  return e;
}

size_t scorer_dev_bytes() { return kScorerDevBytes; }

cudaError_t launch_features(const StageArgs &a, const ImageDesc &im, int L, float *out, cudaStream_t s) {
  features_kernel<<<blocks_for((long long)im.nbx * im.nby, 256), 256, 0, s>>>(a, im, L, out);
  return cudaGetLastError();
}

cudaError_t launch_score(const StageArgs &a, const ImageDesc &im, int L, const ScorerDev &W, float threshold,
                         float *score, unsigned char *mask, cudaStream_t s) {
  const dim3 grid((im.nbx + kOut - 1) / kOut, (im.nby + kOut - 1) / kOut);
  score_kernel<<<grid, kScoreThreads, 0, s>>>(a, im, L, W, threshold, score, mask);
  return cudaGetLastError();
}

size_t collect_scratch_ints(long long blocks) { return 2 * (size_t)blocks_for(blocks, kCollectThreads) + 2; }

cudaError_t launch_collect(const float *feat, const int *before, const int *after, int nbx, int nby, int img,
                           int stage, float neg_rate, const TrainSet &ts, int *scratch, cudaStream_t s) {
  const double q = neg_rate <= 0.f ? 0.0 : neg_rate >= 1.f ? 4294967295.0 : (double)neg_rate * 4294967296.0;
  const long long nb = (long long)nbx * nby;
  const unsigned nctas = blocks_for(nb, kCollectThreads);
  int *cnt = scratch, *base = scratch + nctas;
  collect_count_kernel<<<nctas, kCollectThreads, 0, s>>>(feat, before, after, nb, img, stage, (unsigned)q, cnt);
  collect_scan_kernel<<<1, kScanThreads, 0, s>>>(cnt, (int)nctas, base, ts);
  collect_write_kernel<<<nctas, kCollectThreads, 0, s>>>(feat, before, after, nbx, nby, img, stage, (unsigned)q,
                                                         base, ts);
  return cudaGetLastError();
}

int train_max_ctas() { return kTrainMaxCtas; }

cudaError_t launch_train_step(const TrainSet &ts, int n, const float *w, const int *order, int off, int batch,
                              float pos_weight, float *part, float *part_loss, float *grad, float *loss,
                              cudaStream_t s) {
  const cudaError_t e =
      cudaFuncSetAttribute(train_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
  if (e != cudaSuccess) return e;
  const int want = (batch + kTrainWarps - 1) / kTrainWarps;
  const int ctas = want < kTrainMaxCtas ? want : kTrainMaxCtas;
  train_grad_kernel<<<ctas, kTrainWarps * 32, kTrainSmem, s>>>(ts, n, w, order, off, batch, pos_weight, part,
                                                                part_loss);
  train_reduce_kernel<<<blocks_for(kNParams, 256), 256, 0, s>>>(part, part_loss, ctas, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float *w, float *m, float *v, float *grad, float lr, float bc1, float bc2, float inv_batch,
                        cudaStream_t s) {
  adam_kernel<<<blocks_for(kNParams, 256), 256, 0, s>>>(w, m, v, grad, kNParams, lr, 0.9f, 0.999f, 1e-8f, bc1, bc2,
                                                       inv_batch);
  return cudaGetLastError();
}

}  // namespace rapid
