// rapid_api.cu — the C ABI (include/rapid.h): context, device buffers, stage schedule and
// launch orchestration for a batch of images (a single image is a batch of one).  Host
// code only; every step of the method runs in the kernels of k_prep.cu, k_stage_s*.cu
// (through the dispatcher k_stage.cu) and, for the learned scorer, k_scorer.cu.
#include <algorithm>
#include <climits>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/rapid.h"
#include "rapid_dev.cuh"

namespace rapid {
cudaError_t launch_pyramid(const unsigned char *img, long long pitch, int H, int W, int f, int Wl, int Hl,
                           int4 *out, cudaStream_t s);
cudaError_t launch_pyramid_merge(const int4 *fine, int Wf, int Hf, int m, int Wl, int Hl, int4 *out, cudaStream_t s);
cudaError_t launch_seed(const StageArgs &a, const ImageDesc *ims, const int *gx, const int *gy, int n,
                        cudaStream_t s, int *launches);
cudaError_t launch_recompute(const StageArgs &a, const ImageDesc *ims, int n, cudaStream_t s, int *launches);
cudaError_t launch_split(const int *src, int snbx, int *dst, int dnbx, int dnby, cudaStream_t s);
cudaError_t launch_predict(const ImageDesc *ims, int n, const DevStats &st, long long hT, cudaStream_t s,
                           int *launches);
cudaError_t launch_predict_linear(const StageArgs &a, const ImageDesc *ims, int n, const double *theta,
                                  cudaStream_t s, int *launches);
cudaError_t launch_upsample(const int *lab, int nbx, int side, int H, int W, int label0, int *dst,
                            long long pitch_elems, cudaStream_t s);
cudaError_t launch_pack_stats(const DevStats &st, int label0, int M, rapid_sp_stats *out, cudaStream_t s);
cudaError_t launch_simple_table(unsigned char *out, cudaStream_t s);
cudaError_t launch_init_counters(long long *cnt, const Schedule &sch, int n, cudaStream_t s);
}  // namespace rapid

using namespace rapid;

static_assert(RAPID_MAX_STAGES == 32, "the device counter layout holds 32 stages per image");
static_assert(RAPID_MAX_BATCH == kMaxBatch, "header and device batch limits differ");

static const int kMaxLevels = 8;

// One image of the context's batch.
struct ImgHost {
  int H, W, K;
  long long pitch;                // row pitch of the device copy
  size_t img_off;                 // byte offset of the copy in d_img
  size_t pyr_off[kMaxSumLevels];  // int4 offset of its cells in each sum level
  size_t lab_off;                 // int offset of its label maps in d_lab[0] and d_lab[1]
  int gx, gy, M, label0;          // seed grid, labels label0 .. label0 + M - 1
  double lam_pos;
};

struct rapid_ctx {
  rapid_params p;
  cudaStream_t stream;
  int device, nsm, coop_grid;
  rapid_status sticky;
  // images and levels
  int nimg;
  ImgHost im[kMaxBatch];
  unsigned char *d_img;
  size_t img_cap;
  int L;
  int f[kMaxLevels + 1];
  int nsf;  // box-sum levels for block sums (factors sf[i] > 1, ascending)
  int sf[kMaxSumLevels];
  int4 *d_pyr[kMaxSumLevels];
  size_t pyr_cap[kMaxSumLevels];
  // schedule
  int nstages;
  int st_level[RAPID_MAX_STAGES], st_side[RAPID_MAX_STAGES];
  int cur, cur_buf;
  bool image_set;
  int *d_lab[2];
  size_t lab_cap[2];
  int *d_full;  // full-res staging for host reads
  size_t full_cap;
  unsigned *d_qbits;  // frontier queue (schedule 1): per (tile, class), sized for the finest stage
  size_t qbits_cap;
  int *d_wl;          // frontier worklists (9 * wl_cap) and their 9 counts
  size_t wl_bytes_cap;
  int wl_cap;
  unsigned *d_cbits, *d_rbits;  // sweep schedule: per-class block bitmaps, sized for the largest stage
  int *d_wstamp;  // race check: per block, the phase that last wrote it (rapid_set_race_check)
  size_t wstamp_cap;
  unsigned long long *d_race;  // race check: violations
  int race_on;
  size_t cbits_cap, rbits_cap;
  int cwb[RAPID_MAX_STAGES][10];  // per stage: first word of each class's bitmaps (all images)
  // per (stage, image) descriptors
  ImageDesc *h_desc;  // [nstages * nimg]
  ImageDesc *d_desc;
  size_t desc_cap;
  int ntiles[RAPID_MAX_STAGES];
  int stage_grid[RAPID_MAX_STAGES];   // CTAs of each stage's launch (0 = the full co-resident grid)
  int stage_shape[RAPID_MAX_STAGES];  // evaluation-tile shape of each stage (index into kShapes)
  // labels
  int M_total, M_cap;
  void *d_label_block;
  DevStats st;
  DevMerge mg;
  rapid_sp_stats *d_pack;
  size_t pack_cap;
  // control
  void *d_ctl_block;
  CtlLayout cl;
  DevCtl ctl;
  long long *prof;  // [RAPID_MAX_STAGES][PROF_N] section times (ns)
  double lam_b2;
  int imp_on;
  long long launches;
  int profiling;
  cudaEvent_t ev[RAPID_MAX_STAGES][2];
  int ev_ok[RAPID_MAX_STAGES];
  // CUDA graph of rapid_run
  int graph_on, graph_ok, capturing;
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  long long graph_launches;
  // learned scorer: pruning weights, per-image masks (at the label maps' offsets)
  size_t lab_total;  // ints of one label-map buffer (all images)
  int scorer_on;
  int theta_on;       // Eq. predict with the linear classifier over the features
  double theta[5];
  float scorer_thr;
  int scorer_off[RAPID_MAX_STAGES];  // 1: the scorer leaves this stage unpruned (rapid_set_scorer_stages)
  void *d_scorer, *d_scorer_tmp;
  ScorerDev sdev;
  unsigned char *d_mask;
  size_t mask_cap;
  // caller-given keep masks (rapid_set_keep_mask): per (stage, image) at keep_off, 1 = kept
  unsigned char *d_keep;
  size_t keep_cap;
  size_t keep_off[RAPID_MAX_STAGES][kMaxBatch];
  int keep_stage[RAPID_MAX_STAGES];  // 1: the stage sweeps pruned with its masks
  int keep_on;
  // training-data logging
  rapid_trainer *logger;
  float *d_feat;
  size_t feat_cap;
  int *d_before;
  size_t before_cap;
  int *d_collect;  // scratch of the sample collection (per-CTA counts and bases)
  size_t collect_cap;
};

struct rapid_trainer {
  TrainSet ts;
  float neg_rate;
  int runs;  // logged runs (seedings), part of the sampling hash
  float *buf_x;
  unsigned long long *buf_inb;
  float *buf_y;
  int *buf_count;
};

// Every device allocation of the library goes through dev_malloc, so that a test can make
// the n-th one fail (rapid_debug_fail_alloc) and check that each call reports RAPID_ENOMEM
// and leaves the context destroyable.  The countdown is process-wide; 0 = off.
static std::atomic<long long> g_fail_alloc_after{0};

static cudaError_t dev_malloc(void **p, size_t bytes) {
  long long n = g_fail_alloc_after.load();
  while (n > 0) {
    if (g_fail_alloc_after.compare_exchange_weak(n, n - 1)) {
      if (n == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

extern "C" void rapid_debug_fail_alloc(int64_t n) { g_fail_alloc_after.store(n > 0 ? n : 0); }

static rapid_status cuda_fail(rapid_ctx *c) {
  if (c) c->sticky = RAPID_ECUDA;
  return RAPID_ECUDA;
}

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(ctx); \
  } while (0)

static bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
static constexpr size_t kScorerFeatures() { return RAPID_SCORER_FEATURES; }
static int ceil_div(int a, int b) { return (a + b - 1) / b; }
static size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

extern "C" void rapid_default_params(rapid_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->num_levels = 1;
  p->ratio_C = 4;
  p->init_block = 16;
  p->final_grain = 1;
  p->K = 200;
  p->size_mode = 2;
  p->lambda_pos0 = 400.0;
  p->lambda_b = 50.0;
  p->lo_num = 1;
  p->lo_den = 4;
  p->hi_num = 3;
  p->hi_den = 2;
  p->predict = 0;
  p->reuse = 1;
  p->importance_rule = 0;
  p->max_sweeps = 64;
  p->h_T = 150;
  p->spin_limit_ns = 2000000000ll;
  p->use_filter = 1;
  p->skip_tiles = 1;
  p->verify_filter = 0;
  p->schedule = 0;
}

static bool params_ok(const rapid_params *p) {
  if (!p) return false;
  if (p->num_levels < 1 || p->num_levels > kMaxLevels) return false;
  if (p->num_levels > 1 && (!is_pow2(p->ratio_C) || p->ratio_C < 2)) return false;
  if (!is_pow2(p->init_block) || !is_pow2(p->final_grain) || p->init_block > (1 << 20)) return false;
  if (p->K < 1 || p->size_mode < 0 || p->size_mode > 2 || p->max_sweeps < 1) return false;
  if (p->lo_den <= 0 || p->hi_den <= 0 || p->lo_num < 0 || p->hi_num < 0) return false;
  if (!std::isfinite(p->lambda_pos0) || !std::isfinite(p->lambda_b)) return false;
  if ((p->predict | p->reuse | p->importance_rule | p->use_filter | p->skip_tiles | p->verify_filter |
       p->schedule) & ~1)
    return false;
  if (p->spin_limit_ns < 0 || p->h_T < 0 || p->h_T > (1ll << 40)) return false;
  long long f1 = 1;
  for (int i = 1; i < p->num_levels; i++) {
    f1 *= p->ratio_C;
    if (f1 > (1 << 20)) return false;
  }
  return true;
}

extern "C" rapid_status rapid_create(const rapid_params *p, void *cuda_stream, rapid_ctx **out) {
  if (!out) return RAPID_EINVAL;
  *out = nullptr;
  if (!params_ok(p)) return RAPID_EINVAL;
  rapid_ctx *ctx = new (std::nothrow) rapid_ctx;
  if (!ctx) return RAPID_ENOMEM;
  std::memset(ctx, 0, sizeof *ctx);
  ctx->p = *p;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->cur = -1;
  ctx->sticky = RAPID_OK;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  int coop = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
  // one grid size that every compiled stage kernel can keep co-resident
  int per_sm = INT_MAX;
  for (int sh = 0; sh < kNumShapes && e == cudaSuccess; sh++)
    for (int b = 0; b < 4 && e == cudaSuccess; b++) {
      int k = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, stage_kernel_ptr(b & 1, b >> 1, sh), stage_block_threads(sh),
                                                        0);
      per_sm = std::min(per_sm, k);
    }
  if (e != cudaSuccess || !coop || per_sm < 1) {
    delete ctx;
    return RAPID_ECUDA;
  }
  ctx->coop_grid = ctx->nsm * per_sm;
  // which stage kernels can run as one thread-block cluster (decided now, outside any graph
  // capture, and remembered)
  for (int sh = 0; sh < kNumShapes; sh++)
    for (int fr = 0; fr < 2; fr++)
      cluster_launch_ok(stage_cluster_kernel_ptr(fr != 0, sh), 2, stage_block_threads(sh), ctx->stream);
  ctx->cl = ctl_layout(kMaxBatch);
  if (dev_malloc((void **)&ctx->d_ctl_block, ctx->cl.total) != cudaSuccess) {
    delete ctx;
    return RAPID_ENOMEM;
  }
  char *b = (char *)ctx->d_ctl_block;
  ctx->ctl.bar = (unsigned *)(b + ctx->cl.bar);
  ctx->ctl.err = (int *)(b + 8);
  ctx->mg.req_count = (int *)(b + 16);    // [2], by phase parity
  ctx->mg.found_count = (int *)(b + 24);  // [2], by phase parity
  ctx->mg.acc_count = (int *)(b + 32);
  ctx->ctl.last_merge = (int *)(b + ctx->cl.last_merge);
  ctx->ctl.changes = (unsigned long long *)(b + ctx->cl.changes);
  ctx->ctl.cnt = (long long *)(b + ctx->cl.cnt);
  ctx->prof = (long long *)(b + ctx->cl.prof);
  ctx->ctl.spin_ns = p->spin_limit_ns;
  if (cudaMemsetAsync(ctx->d_ctl_block, 0, ctx->cl.total, ctx->stream) != cudaSuccess) {
    cudaFree(ctx->d_ctl_block);
    delete ctx;
    return RAPID_ECUDA;
  }
  *out = ctx;
  return RAPID_OK;
}

static void drop_graph(rapid_ctx *ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->gexec = nullptr;
  ctx->graph = nullptr;
  ctx->graph_ok = 0;
}

static void free_image_buffers(rapid_ctx *ctx) {
  cudaFree(ctx->d_img);
  ctx->d_img = nullptr;
  ctx->img_cap = 0;
  for (int l = 0; l < kMaxSumLevels; l++) {
    cudaFree(ctx->d_pyr[l]);
    ctx->d_pyr[l] = nullptr;
    ctx->pyr_cap[l] = 0;
  }
  for (int b = 0; b < 2; b++) {
    cudaFree(ctx->d_lab[b]);
    ctx->d_lab[b] = nullptr;
    ctx->lab_cap[b] = 0;
  }
  cudaFree(ctx->d_full);
  ctx->d_full = nullptr;
  ctx->full_cap = 0;
  cudaFree(ctx->d_qbits);
  ctx->d_qbits = nullptr;
  ctx->qbits_cap = 0;
  cudaFree(ctx->d_wl);
  ctx->d_wl = nullptr;
  ctx->wl_bytes_cap = 0;
  cudaFree(ctx->d_wstamp);
  ctx->d_wstamp = nullptr;
  ctx->wstamp_cap = 0;
  cudaFree(ctx->d_cbits);
  ctx->d_cbits = nullptr;
  ctx->cbits_cap = 0;
  cudaFree(ctx->d_rbits);
  ctx->d_rbits = nullptr;
  ctx->rbits_cap = 0;
  cudaFree(ctx->d_desc);
  ctx->d_desc = nullptr;
  ctx->desc_cap = 0;
  std::free(ctx->h_desc);
  ctx->h_desc = nullptr;
  cudaFree(ctx->d_keep);
  ctx->d_keep = nullptr;
  ctx->keep_cap = 0;
  ctx->keep_on = 0;
  std::memset(ctx->keep_stage, 0, sizeof ctx->keep_stage);
  cudaFree(ctx->d_mask);
  ctx->d_mask = nullptr;
  ctx->mask_cap = 0;
  cudaFree(ctx->d_feat);
  ctx->d_feat = nullptr;
  ctx->feat_cap = 0;
  cudaFree(ctx->d_before);
  ctx->d_before = nullptr;
  ctx->before_cap = 0;
  cudaFree(ctx->d_collect);
  ctx->d_collect = nullptr;
  ctx->collect_cap = 0;
}

extern "C" void rapid_destroy(rapid_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  drop_graph(ctx);
  free_image_buffers(ctx);
  cudaFree(ctx->d_label_block);
  cudaFree(ctx->d_pack);
  cudaFree(ctx->d_ctl_block);
  cudaFree(ctx->d_scorer);
  cudaFree(ctx->d_scorer_tmp);
  cudaFree(ctx->d_race);
  for (int i = 0; i < RAPID_MAX_STAGES; i++)
    if (ctx->ev_ok[i]) {
      cudaEventDestroy(ctx->ev[i][0]);
      cudaEventDestroy(ctx->ev[i][1]);
    }
  delete ctx;
}

// Levels f_l = C^(L-l) and the stage schedule: the block side halves from the initial
// block (at least f_1) to the final grain; each side belongs to the coarsest level whose
// factor does not exceed it.  Depends on the parameters only.
static rapid_status make_schedule(rapid_ctx *ctx) {
  const rapid_params &p = ctx->p;
  ctx->L = p.num_levels;
  for (int l = 1; l <= ctx->L; l++) {
    int f = 1;
    for (int i = 0; i < ctx->L - l; i++) f *= p.ratio_C;
    ctx->f[l] = f;
  }
  int s = p.init_block < ctx->f[1] ? ctx->f[1] : p.init_block;
  ctx->nstages = 0;
  while (s >= 1 && s >= p.final_grain) {
    int lev = 0;
    for (int l = 1; l <= ctx->L; l++)
      if (ctx->f[l] <= s) {
        lev = l;
        break;
      }
    if (lev == 0) break;
    if (ctx->nstages >= RAPID_MAX_STAGES) return RAPID_ERANGE;
    ctx->st_level[ctx->nstages] = lev;
    ctx->st_side[ctx->nstages] = s;
    ctx->nstages++;
    s /= 2;
  }
  if (ctx->nstages == 0) {
    ctx->st_level[0] = 1;
    ctx->st_side[0] = p.init_block < ctx->f[1] ? ctx->f[1] : p.init_block;
    ctx->nstages = 1;
  }
  ctx->nsf = sum_factors(ctx->f, ctx->L, ctx->st_side[0], ctx->sf);
  return RAPID_OK;
}

// Make *pp a device buffer of at least `need` bytes (contents not kept).
template <class T>
static bool grow(T **pp, size_t *cap, size_t need) {
  if (need <= *cap && *pp) return true;
  cudaFree(*pp);
  *pp = nullptr;
  *cap = 0;
  if (dev_malloc((void **)pp, need ? need : 1) != cudaSuccess) return false;
  *cap = need;
  return true;
}

static rapid_status ensure_label_arrays(rapid_ctx *ctx, int M) {
  if (M <= ctx->M_cap) {
    carve_label_arrays(ctx->d_label_block, label_arrays_bytes(ctx->M_cap), M, &ctx->st, &ctx->mg);
    return RAPID_OK;
  }
  cudaFree(ctx->d_label_block);
  ctx->d_label_block = nullptr;
  ctx->M_cap = 0;
  const size_t bytes = label_arrays_bytes(M);
  if (dev_malloc((void **)&ctx->d_label_block, bytes) != cudaSuccess) return RAPID_ENOMEM;
  carve_label_arrays(ctx->d_label_block, bytes, M, &ctx->st, &ctx->mg);
  ctx->M_cap = M;
  return RAPID_OK;
}

// Factor of the sum level a stage reads: the coarsest box-sum level whose cells fit in a
// block (1 = the image itself).
static int stage_sum_factor(const rapid_ctx *ctx, int side) {
  int f = 1;
  for (int l = 0; l < ctx->nsf; l++)
    if (ctx->sf[l] <= side) f = ctx->sf[l];
  return f;
}

// Descriptors of every (stage, image), on the host and uploaded once.
static rapid_status build_descriptors(rapid_ctx *ctx) {
  const size_t n = (size_t)ctx->nstages * ctx->nimg;
  std::free(ctx->h_desc);
  ctx->h_desc = (ImageDesc *)std::calloc(n, sizeof(ImageDesc));
  if (!ctx->h_desc) return RAPID_ENOMEM;
  if (!grow(&ctx->d_desc, &ctx->desc_cap, n * sizeof(ImageDesc))) return RAPID_ENOMEM;
  long long words_max = 0;
  for (int s = 0; s < ctx->nstages; s++) {
    const int side = ctx->st_side[s];
    const int f = stage_sum_factor(ctx, side);
    int li = -1;
    for (int l = 0; l < ctx->nsf; l++)
      if (ctx->sf[l] == f) li = l;
    long long tile0 = 0, blk0 = 0;
    for (int i = 0; i < ctx->nimg; i++) {
      const ImgHost &h = ctx->im[i];
      ImageDesc &d = ctx->h_desc[(size_t)s * ctx->nimg + i];
      d.H = h.H;
      d.W = h.W;
      d.nbx = ceil_div(h.W, side);
      d.nby = ceil_div(h.H, side);
      const TileShape ts = kShapes[ctx->stage_shape[s]];
      d.ntx = (d.nbx + ts.w - 1) / ts.w;
      d.nty = (d.nby + ts.h - 1) / ts.h;
      d.Wl = ceil_div(h.W, f);
      d.Hl = ceil_div(h.H, f);
      d.tile0 = (int)tile0;
      d.label0 = h.label0;
      d.M = h.M;
      d.blk0 = (int)blk0;
      // single-precision decisions need blocks under 2^24 pixels and exact float block centres
      d.use_filter = ctx->p.use_filter && side <= 4096 && h.W < (1 << 22) && h.H < (1 << 22);
      d.img = ctx->d_img + h.img_off;
      d.img_pitch = h.pitch;
      d.pyr = li >= 0 ? ctx->d_pyr[li] + h.pyr_off[li] : nullptr;
      d.lab = ctx->d_lab[s & 1] + h.lab_off;
      d.mask = ctx->d_mask ? ctx->d_mask + h.lab_off : nullptr;
      d.lam_pos = h.lam_pos;
      d.lam_pos_f = (float)h.lam_pos;
      tile0 += (long long)d.ntx * d.nty;
      blk0 += (long long)d.nbx * d.nby;
    }
    if (tile0 >= INT_MAX / 9 || blk0 >= INT_MAX) return RAPID_ERANGE;
    ctx->ntiles[s] = (int)tile0;
    // sweep-schedule bitmaps: class-major, images in order within a class
    long long w = 0;
    for (int c = 0; c < 9; c++) {
      ctx->cwb[s][c] = (int)w;
      for (int i = 0; i < ctx->nimg; i++) {
        ImageDesc &d = ctx->h_desc[(size_t)s * ctx->nimg + i];
        d.cw0[c] = (int)w;
        w += class_words(d.nbx, d.nby, c);
        if (w >= INT_MAX) return RAPID_ERANGE;
      }
    }
    ctx->cwb[s][9] = (int)w;
    words_max = std::max(words_max, w);
  }
  if (!grow(&ctx->d_cbits, &ctx->cbits_cap, (size_t)words_max * sizeof(unsigned)) ||
      !grow(&ctx->d_rbits, &ctx->rbits_cap, (size_t)words_max * sizeof(unsigned)))
    return RAPID_ENOMEM;
  if (cudaMemcpy(ctx->d_desc, ctx->h_desc, n * sizeof(ImageDesc), cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_fail(ctx);
  return RAPID_OK;
}

extern "C" rapid_status rapid_set_images(rapid_ctx *ctx, int32_t n, const uint8_t *const *rgb, const int32_t *H,
                                         const int32_t *W, const int64_t *row_pitch_bytes, const int32_t *K,
                                         int32_t rgb_is_device) {
  if (!ctx || !rgb || !H || !W || !row_pitch_bytes) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (n < 1) return RAPID_EINVAL;
  if (n > kMaxBatch) return RAPID_ERANGE;
  for (int i = 0; i < n; i++) {
    if (!rgb[i] || H[i] < 1 || W[i] < 1 || row_pitch_bytes[i] < 3ll * W[i]) return RAPID_EINVAL;
    if (K && K[i] < 1) return RAPID_EINVAL;
    const long long npx = (long long)H[i] * W[i];
    if (npx >= (1ll << 31)) return RAPID_EINVAL;
    // position sums reach about H*W*max(H,W)/2; keep them exact in binary64
    if ((double)npx * (double)(H[i] > W[i] ? H[i] : W[i]) >= 9007199254740992.0) return RAPID_EINVAL;
  }
  drop_graph(ctx);
  ctx->image_set = false;
  ctx->keep_on = 0;  // keep masks belong to the previous images' block grids
  std::memset(ctx->keep_stage, 0, sizeof ctx->keep_stage);
  ctx->cur = -1;
  rapid_status rs = make_schedule(ctx);
  if (rs != RAPID_OK) return rs;
  // a sum level keeps int32 channel sums: one cell (at most f x f pixels of 255) must fit
  for (int i = 0; i < n; i++)
    for (int l = 0; l < ctx->nsf; l++)
      if ((long long)std::min(ctx->sf[l], W[i]) * std::min(ctx->sf[l], H[i]) * 255 > INT_MAX) return RAPID_ERANGE;
  // per-image layout (image copy, sum levels, label maps), seed grid and label range
  const int s0 = ctx->st_side[0], sl = ctx->st_side[ctx->nstages - 1];
  size_t img_bytes = 0, pyr_n[kMaxSumLevels] = {0}, lab_n = 0;
  long long tiles_last = 0, M_total = 0, max_M = 0, npx_max = 0, class_blocks = 0;
  for (int i = 0; i < n; i++) {
    ImgHost &h = ctx->im[i];
    h.H = H[i];
    h.W = W[i];
    h.K = K ? K[i] : ctx->p.K;
    h.pitch = (long long)round_up(3ull * h.W, 16);
    h.img_off = img_bytes;
    img_bytes = round_up(img_bytes + (size_t)h.pitch * h.H, 256);
    for (int l = 0; l < ctx->nsf; l++) {
      h.pyr_off[l] = pyr_n[l];
      pyr_n[l] = round_up(pyr_n[l] + (size_t)ceil_div(h.W, ctx->sf[l]) * ceil_div(h.H, ctx->sf[l]), 16);
    }
    const int lnbx = ceil_div(h.W, sl), lnby = ceil_div(h.H, sl);
    h.lab_off = lab_n;
    lab_n = round_up(lab_n + (size_t)lnbx * lnby, 64);
    long long most = 0;  // queue words: the shape with the most tiles at the finest stage
    for (int sh = 0; sh < kNumShapes; sh++)
      most = std::max<long long>(most, (long long)((lnbx + kShapes[sh].w - 1) / kShapes[sh].w) *
                                           ((lnby + kShapes[sh].h - 1) / kShapes[sh].h));
    tiles_last += most;
    class_blocks += (long long)((lnbx + 2) / 3) * ((lnby + 2) / 3);  // blocks of one phase class, at most
    // seed grid gx x gy (same rounding as the stated formula) on the first stage's blocks
    const int nbx0 = ceil_div(h.W, s0), nby0 = ceil_div(h.H, s0);
    int gx = (int)std::floor(std::sqrt((double)h.K * (double)h.W / (double)h.H) + 0.5);
    if (gx < 1) gx = 1;
    int gy = (int)std::floor((double)h.K / (double)gx + 0.5);
    if (gy < 1) gy = 1;
    if (gx > nbx0) gx = nbx0;
    if (gy > nby0) gy = nby0;
    h.gx = gx;
    h.gy = gy;
    h.M = gx * gy;
    h.label0 = (int)M_total;
    M_total += h.M;
    max_M = std::max<long long>(max_M, h.M);
    npx_max = std::max<long long>(npx_max, (long long)h.H * h.W);
    h.lam_pos = ctx->p.lambda_pos0 * ((double)h.M / ((double)h.H * (double)h.W));
  }
  if (M_total >= INT_MAX || lab_n >= (size_t)INT_MAX) return RAPID_ERANGE;
  ctx->nimg = n;
  ctx->lab_total = lab_n;
  ctx->M_total = (int)M_total;
  ctx->lam_b2 = 2.0 * ctx->p.lambda_b;
  if (!grow(&ctx->d_img, &ctx->img_cap, img_bytes)) return RAPID_ENOMEM;
  for (int l = 0; l < ctx->nsf; l++)
    if (!grow(&ctx->d_pyr[l], &ctx->pyr_cap[l], pyr_n[l] * sizeof(int4))) return RAPID_ENOMEM;
  for (int b = 0; b < 2; b++)
    if (!grow(&ctx->d_lab[b], &ctx->lab_cap[b], lab_n * sizeof(int))) return RAPID_ENOMEM;
  if (ctx->p.schedule == 1) {
    if (!grow(&ctx->d_qbits, &ctx->qbits_cap, (size_t)tiles_last * 9 * kQueueWords * sizeof(unsigned)))
      return RAPID_ENOMEM;
    if (!grow(&ctx->d_wl, &ctx->wl_bytes_cap, ((size_t)class_blocks * 9 + 16) * sizeof(int))) return RAPID_ENOMEM;
    ctx->wl_cap = (int)class_blocks;
  }
  if (!grow(&ctx->d_full, &ctx->full_cap, (size_t)npx_max * sizeof(int))) return RAPID_ENOMEM;
  if (!grow(&ctx->d_pack, &ctx->pack_cap, (size_t)max_M * sizeof(rapid_sp_stats))) return RAPID_ENOMEM;
  rs = ensure_label_arrays(ctx, ctx->M_total);
  if (rs != RAPID_OK) return rs;
  if (ctx->scorer_on && !grow(&ctx->d_mask, &ctx->mask_cap, lab_n)) return RAPID_ENOMEM;
  if (ctx->race_on && !grow(&ctx->d_wstamp, &ctx->wstamp_cap, lab_n * sizeof(int))) return RAPID_ENOMEM;
  if (ctx->logger) {
    if (!grow(&ctx->d_feat, &ctx->feat_cap, lab_n * kScorerFeatures() * sizeof(float))) return RAPID_ENOMEM;
    if (!grow(&ctx->d_before, &ctx->before_cap, lab_n * sizeof(int))) return RAPID_ENOMEM;
    if (!grow(&ctx->d_collect, &ctx->collect_cap, collect_scratch_ints((long long)lab_n) * sizeof(int)))
      return RAPID_ENOMEM;
  }
  rs = build_descriptors(ctx);
  if (rs != RAPID_OK) return rs;
  for (int i = 0; i < n; i++) {
    const ImgHost &h = ctx->im[i];
    CK(cudaMemcpy2DAsync(ctx->d_img + h.img_off, h.pitch, rgb[i], row_pitch_bytes[i], 3ull * h.W, h.H,
                         rgb_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  }
  if (!rgb_is_device) CK(cudaStreamSynchronize(ctx->stream));  // the host buffers may be reused at return
  ctx->image_set = true;
  return RAPID_OK;
}

extern "C" rapid_status rapid_set_image(rapid_ctx *ctx, const uint8_t *rgb, int32_t H, int32_t W,
                                        int64_t row_pitch_bytes, int32_t rgb_is_device) {
  if (!ctx) return RAPID_EINVAL;
  const uint8_t *imgs[1] = {rgb};
  const int64_t pitch[1] = {row_pitch_bytes};
  return rapid_set_images(ctx, 1, imgs, &H, &W, pitch, nullptr, rgb_is_device);
}

// Launch arguments of stage s (all images).
static StageArgs stage_args(rapid_ctx *ctx, int s) {
  StageArgs a;
  std::memset(&a, 0, sizeof a);
  a.side = ctx->st_side[s];
  a.level = ctx->st_level[s];
  a.f = stage_sum_factor(ctx, a.side);
  a.k = a.side / a.f;
  a.imgs = ctx->d_desc + (size_t)s * ctx->nimg;
  a.img0 = ctx->h_desc[(size_t)s * ctx->nimg];
  a.nimg = ctx->nimg;
  a.ntiles = ctx->ntiles[s];
  a.st = ctx->st;
  a.st.M = ctx->M_total;
  a.mg = ctx->mg;
  a.ctl = ctx->ctl;
  a.ctl.cnt = ctx->ctl.cnt + (long long)CNT_N * s;
  a.ctl.prof = ctx->profiling ? ctx->prof + (long long)PROF_N * s : nullptr;
  a.imp_on = ctx->imp_on;
  a.imp_rule = ctx->p.importance_rule;
  a.lam_b2 = ctx->lam_b2;
  a.lam_b2_f = (float)ctx->lam_b2;
  a.size_mode = ctx->p.size_mode;
  a.lo_num = ctx->p.lo_num;
  a.lo_den = ctx->p.lo_den;
  a.hi_num = ctx->p.hi_num;
  a.hi_den = ctx->p.hi_den;
  a.max_sweeps = ctx->p.max_sweeps;
  a.verify_filter = ctx->p.verify_filter;
  a.skip_tiles = ctx->p.skip_tiles;
  a.prune = (ctx->scorer_on && !ctx->scorer_off[s]) || (ctx->keep_on && ctx->keep_stage[s]);
  a.frontier = ctx->p.schedule == 1;
  a.qbits = ctx->d_qbits;
  a.wl = ctx->d_wl;
  a.wl_count = ctx->d_wl ? ctx->d_wl + (size_t)ctx->wl_cap * 9 : nullptr;
  a.wl_cap = ctx->wl_cap;
  a.cbits = ctx->d_cbits;
  a.rbits = ctx->d_rbits;
  a.wstamp = ctx->race_on ? ctx->d_wstamp : nullptr;
  a.race = ctx->d_race;
  for (int c = 0; c < 10; c++) a.cwb[c] = ctx->cwb[s][c];
  return a;
}

static const ImageDesc *host_desc(const rapid_ctx *ctx, int s) { return ctx->h_desc + (size_t)s * ctx->nimg; }

extern "C" rapid_status rapid_seed_grid(rapid_ctx *ctx, int32_t *M_out) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (!ctx->image_set) return RAPID_ESTATE;
  // level images (exact box sums, Sec. 2.2) and the extra box-sum levels for block sums
  for (int i = 0; i < ctx->nimg; i++) {
    const ImgHost &h = ctx->im[i];
    for (int l = 0; l < ctx->nsf; l++) {  // the finest level from the image, each coarser one from the last
      const int sf = ctx->sf[l];
      if (l == 0)
        CK(launch_pyramid(ctx->d_img + h.img_off, h.pitch, h.H, h.W, sf, ceil_div(h.W, sf), ceil_div(h.H, sf),
                          ctx->d_pyr[l] + h.pyr_off[l], ctx->stream));
      else
        CK(launch_pyramid_merge(ctx->d_pyr[l - 1] + h.pyr_off[l - 1], ceil_div(h.W, ctx->sf[l - 1]),
                                ceil_div(h.H, ctx->sf[l - 1]), sf / ctx->sf[l - 1], ceil_div(h.W, sf),
                                ceil_div(h.H, sf), ctx->d_pyr[l] + h.pyr_off[l], ctx->stream));
      ctx->launches++;
    }
  }
  ctx->cur = 0;
  ctx->cur_buf = 0;
  ctx->imp_on = 0;
  // counters: level and side of every stage, the rest zero; no device error pending
  Schedule sch;
  std::memset(&sch, 0, sizeof sch);
  sch.n = ctx->nstages;
  for (int i = 0; i < ctx->nstages; i++) {
    sch.level[i] = ctx->st_level[i];
    sch.side[i] = ctx->st_side[i];
  }
  CK(launch_init_counters(ctx->ctl.cnt, sch, ctx->nimg, ctx->stream));
  CK(cudaMemsetAsync(ctx->prof, 0, sizeof(long long) * PROF_N * RAPID_MAX_STAGES, ctx->stream));
  CK(cudaMemsetAsync(ctx->mg.req_count, 0, 4 * sizeof(int), ctx->stream));
  ctx->launches++;
  int gx[kMaxBatch], gy[kMaxBatch];
  for (int i = 0; i < ctx->nimg; i++) {
    gx[i] = ctx->im[i].gx;
    gy[i] = ctx->im[i].gy;
  }
  int nl = 0;
  StageArgs a = stage_args(ctx, 0);
  CK(launch_seed(a, host_desc(ctx, 0), gx, gy, ctx->nimg, ctx->stream, &nl));
  if (ctx->logger) ctx->logger->runs++;
  ctx->launches += nl;
  if (M_out) *M_out = ctx->im[0].M;
  return RAPID_OK;
}

static rapid_status read_device_error(rapid_ctx *ctx) {
  int err = 0;
  CK(cudaMemcpy(&err, ctx->ctl.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err != 0) {
    ctx->sticky = RAPID_ETIMEOUT;
    return RAPID_ETIMEOUT;
  }
  return RAPID_OK;
}

extern "C" rapid_status rapid_sync(rapid_ctx *ctx) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  CK(cudaStreamSynchronize(ctx->stream));
  return read_device_error(ctx);
}

extern "C" rapid_status rapid_refine_stage(rapid_ctx *ctx, int32_t *sweeps_out, int64_t *moves_out,
                                           int64_t *merges_out) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (ctx->cur < 0) return RAPID_ESTATE;
  const int i = ctx->cur;
  // fresh barrier counter, merge stamps, request / found counts and sweep-change slots
  CK(cudaMemsetAsync((char *)ctx->d_ctl_block + 16, 0, ctx->cl.reset_end - 16, ctx->stream));
  StageArgs a = stage_args(ctx, i);
  // events around the launch (inside a captured graph as event-record nodes)
  const unsigned evflags = ctx->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (ctx->profiling) {
    if (!ctx->ev_ok[i]) {
      CK(cudaEventCreate(&ctx->ev[i][0]));
      CK(cudaEventCreate(&ctx->ev[i][1]));
      ctx->ev_ok[i] = 1;
    }
    CK(cudaEventRecordWithFlags(ctx->ev[i][0], ctx->stream, evflags));
  }
  const ImageDesc *ds = host_desc(ctx, i);
  if (ctx->scorer_on && a.prune)  // the learned scorer's masks for this stage (pruned sweeps)
    for (int m = 0; m < ctx->nimg; m++) {
      CK(launch_score(a, ds[m], ctx->L, ctx->sdev, ctx->scorer_thr, nullptr, ctx->d_mask + ctx->im[m].lab_off,
                      ctx->stream));
      ctx->launches++;
    }
  else if (a.prune)  // the caller's keep masks for this stage
    for (int m = 0; m < ctx->nimg; m++)
      CK(cudaMemcpyAsync(ctx->d_mask + ctx->im[m].lab_off, ctx->d_keep + ctx->keep_off[i][m],
                         (size_t)ds[m].nbx * ds[m].nby, cudaMemcpyDeviceToDevice, ctx->stream));
  if (ctx->logger)  // training data: features and labels at the stage start
    for (int m = 0; m < ctx->nimg; m++) {
      const size_t off = ctx->im[m].lab_off;
      CK(launch_features(a, ds[m], ctx->L, ctx->d_feat + off * kScorerFeatures(), ctx->stream));
      CK(cudaMemcpyAsync(ctx->d_before + off, ds[m].lab, (size_t)ds[m].nbx * ds[m].nby * sizeof(int),
                         cudaMemcpyDeviceToDevice, ctx->stream));
      ctx->launches++;
    }
  const int grid = ctx->stage_grid[i] > 0 ? std::min(ctx->stage_grid[i], ctx->coop_grid) : ctx->coop_grid;
  CK(launch_stage(a, grid, stage_block_threads(ctx->stage_shape[i]), ctx->stream, ctx->stage_shape[i]));
  ctx->launches++;
  if (ctx->profiling) CK(cudaEventRecordWithFlags(ctx->ev[i][1], ctx->stream, evflags));
  if (ctx->logger)  // samples: boundary blocks at the start, moved or not by the end
    for (int m = 0; m < ctx->nimg; m++) {
      const size_t off = ctx->im[m].lab_off;
      CK(launch_collect(ctx->d_feat + off * kScorerFeatures(), ctx->d_before + off, ds[m].lab, ds[m].nbx,
                        ds[m].nby, ctx->logger->runs * kMaxBatch + m, i, ctx->logger->neg_rate, ctx->logger->ts,
                        ctx->d_collect, ctx->stream));
      ctx->launches++;
    }
  if (sweeps_out || moves_out || merges_out) {
    CK(cudaStreamSynchronize(ctx->stream));
    rapid_status rs = read_device_error(ctx);
    if (rs != RAPID_OK) return rs;
    long long c[CNT_N];
    CK(cudaMemcpy(c, ctx->ctl.cnt + (long long)CNT_N * i, sizeof c, cudaMemcpyDeviceToHost));
    if (sweeps_out) *sweeps_out = (int32_t)c[CNT_SWEEPS];
    if (moves_out) *moves_out = c[CNT_MOVES];
    if (merges_out) *merges_out = c[CNT_MERGES];
  }
  return RAPID_OK;
}

extern "C" rapid_status rapid_split(rapid_ctx *ctx) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (ctx->cur < 0 || ctx->cur + 1 >= ctx->nstages) return RAPID_ESTATE;
  const int prev_level = ctx->st_level[ctx->cur];
  const int nxt = ctx->cur + 1;
  int nl = 0;
  if (ctx->p.predict && ctx->st_level[nxt] >= 2 && prev_level < 2) {
    StageArgs a = stage_args(ctx, ctx->cur);
    if (ctx->theta_on)
      CK(launch_predict_linear(a, host_desc(ctx, ctx->cur), ctx->nimg, ctx->theta, ctx->stream, &nl));
    else
      CK(launch_predict(host_desc(ctx, ctx->cur), ctx->nimg, a.st, ctx->p.h_T, ctx->stream, &nl));
    ctx->imp_on = 1;
  }
  const ImageDesc *src = host_desc(ctx, ctx->cur), *dst = host_desc(ctx, nxt);
  for (int i = 0; i < ctx->nimg; i++) {
    CK(launch_split(src[i].lab, src[i].nbx, dst[i].lab, dst[i].nbx, dst[i].nby, ctx->stream));
    nl++;
  }
  ctx->cur_buf ^= 1;
  ctx->cur = nxt;
  if (!ctx->p.reuse && ctx->st_level[nxt] != prev_level) {
    StageArgs a = stage_args(ctx, nxt);
    CK(launch_recompute(a, dst, ctx->nimg, ctx->stream, &nl));
  }
  ctx->launches += nl;
  return RAPID_OK;
}

static rapid_status run_sequence(rapid_ctx *ctx) {
  rapid_status rs = rapid_seed_grid(ctx, nullptr);
  if (rs != RAPID_OK) return rs;
  rs = rapid_refine_stage(ctx, nullptr, nullptr, nullptr);
  if (rs != RAPID_OK) return rs;
  while (ctx->cur + 1 < ctx->nstages) {
    rs = rapid_split(ctx);
    if (rs != RAPID_OK) return rs;
    rs = rapid_refine_stage(ctx, nullptr, nullptr, nullptr);
    if (rs != RAPID_OK) return rs;
  }
  return RAPID_OK;
}

// Capture the whole schedule once into a CUDA graph (stream capture of the launches
// rapid_run makes) and instantiate it.
static rapid_status capture_run(rapid_ctx *ctx) {
  const long long l0 = ctx->launches;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  ctx->capturing = 1;
  rapid_status rs = run_sequence(ctx);
  ctx->capturing = 0;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  if (rs != RAPID_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rs != RAPID_OK ? rs : cuda_fail(ctx);
  }
  ctx->graph = g;
  CK(cudaGraphInstantiate(&ctx->gexec, g, 0));
  ctx->graph_launches = ctx->launches - l0;
  ctx->launches = l0;
  ctx->graph_ok = 1;
  return RAPID_OK;
}

extern "C" rapid_status rapid_run(rapid_ctx *ctx) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (!ctx->graph_on) return run_sequence(ctx);
  if (!ctx->image_set) return RAPID_ESTATE;
  if (!ctx->graph_ok) {
    rapid_status rs = capture_run(ctx);
    if (rs != RAPID_OK) return rs;
  }
  CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
  ctx->launches += ctx->graph_launches;
  // the host-side position after a whole run
  ctx->cur = ctx->nstages - 1;
  ctx->cur_buf = (ctx->nstages - 1) & 1;
  ctx->imp_on = 0;
  for (int s = 1; s < ctx->nstages; s++)
    if (ctx->p.predict && ctx->st_level[s] >= 2 && ctx->st_level[s - 1] < 2) ctx->imp_on = 1;
  return RAPID_OK;
}

extern "C" rapid_status rapid_set_graph(rapid_ctx *ctx, int32_t on) {
  if (!ctx) return RAPID_EINVAL;
  if (on && ctx->stream == 0) return RAPID_EINVAL;  // the legacy stream cannot be captured
  if (!on) drop_graph(ctx);
  ctx->graph_on = on ? 1 : 0;
  return RAPID_OK;
}

extern "C" rapid_status rapid_set_stage_shapes(rapid_ctx *ctx, const int32_t *shapes, int32_t n) {
  if (!ctx || n < 0 || n > RAPID_MAX_STAGES || (n > 0 && !shapes)) return RAPID_EINVAL;
  for (int i = 0; i < n; i++)
    if (shapes[i] < 0 || shapes[i] >= kNumShapes) return RAPID_EINVAL;
  for (int i = 0; i < RAPID_MAX_STAGES; i++) ctx->stage_shape[i] = i < n ? shapes[i] : 0;
  drop_graph(ctx);
  return ctx->image_set ? build_descriptors(ctx) : RAPID_OK;
}

extern "C" rapid_status rapid_set_stage_grids(rapid_ctx *ctx, const int32_t *grids, int32_t n) {
  if (!ctx || n < 0 || n > RAPID_MAX_STAGES || (n > 0 && !grids)) return RAPID_EINVAL;
  for (int i = 0; i < n; i++)
    if (grids[i] < 0) return RAPID_EINVAL;
  for (int i = 0; i < RAPID_MAX_STAGES; i++) ctx->stage_grid[i] = i < n ? grids[i] : 0;
  drop_graph(ctx);
  return RAPID_OK;
}

// Launch-geometry tuner.  A stage's result does not depend on its evaluation-tile shape or
// on how many CTAs share its work (the decisions of a phase are independent, merges are
// ordered by block index), only its time does: coarse stages with few tiles lose more to
// the grid barrier than they gain from more SMs, and the best tile shape depends on the
// stage.  First the whole schedule runs once per tile shape on the full grid, then once per
// grid size (the full co-resident grid, its halvings down to one CTA, and 16 and 8 CTAs,
// which run as one thread-block cluster) with the chosen shapes; every stage is timed with
// events and keeps its fastest setting (ties to the earlier candidate).  Each candidate runs
// twice, the first run warming up.
static rapid_status time_stages(rapid_ctx *ctx, float *ms) {
  for (int rep = 0; rep < 2; rep++) {
    rapid_status rs = run_sequence(ctx);
    if (rs == RAPID_OK) rs = rapid_sync(ctx);
    if (rs != RAPID_OK) return rs;
  }
  for (int s = 0; s < ctx->nstages; s++)
    if (cudaEventElapsedTime(&ms[s], ctx->ev[s][0], ctx->ev[s][1]) != cudaSuccess) return cuda_fail(ctx);
  return RAPID_OK;
}

extern "C" rapid_status rapid_autotune(rapid_ctx *ctx, int32_t *grids_out, int32_t *shapes_out) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (!ctx->image_set) return RAPID_ESTATE;
  const int saved_prof = ctx->profiling, saved_graph = ctx->graph_on;
  ctx->profiling = 1;
  ctx->graph_on = 0;
  drop_graph(ctx);
  float best[RAPID_MAX_STAGES], ms[RAPID_MAX_STAGES];
  int best_shape[RAPID_MAX_STAGES], best_grid[RAPID_MAX_STAGES];
  for (int s = 0; s < RAPID_MAX_STAGES; s++) {
    best[s] = 3.4e38f;
    best_shape[s] = 0;
    best_grid[s] = ctx->coop_grid;
    ctx->stage_grid[s] = 0;
  }
  rapid_status rs = RAPID_OK;
  for (int sh = 0; sh < kNumShapes && rs == RAPID_OK; sh++) {
    for (int s = 0; s < RAPID_MAX_STAGES; s++) ctx->stage_shape[s] = sh;
    rs = build_descriptors(ctx);
    if (rs == RAPID_OK) rs = time_stages(ctx, ms);
    for (int s = 0; s < ctx->nstages && rs == RAPID_OK; s++)
      if (ms[s] < best[s]) {
        best[s] = ms[s];
        best_shape[s] = sh;
      }
  }
  for (int s = 0; s < RAPID_MAX_STAGES; s++) ctx->stage_shape[s] = best_shape[s];
  if (rs == RAPID_OK) rs = build_descriptors(ctx);
  // grid candidates: the halvings of the full grid, and the cluster sizes 16 and 8 (a grid of
  // at most kMaxCluster CTAs runs as one thread-block cluster where the device allows it)
  int cand[40], nc = 0;
  for (int g = ctx->coop_grid / 2; g >= 1; g /= 2) cand[nc++] = g;
  for (int g : {kMaxCluster, 8})
    if (g < ctx->coop_grid && std::find(cand, cand + nc, g) == cand + nc) cand[nc++] = g;
  for (int ci = 0; ci < nc && rs == RAPID_OK; ci++) {
    const int g = cand[ci];
    for (int s = 0; s < RAPID_MAX_STAGES; s++) ctx->stage_grid[s] = g;
    rs = time_stages(ctx, ms);
    for (int s = 0; s < ctx->nstages && rs == RAPID_OK; s++)
      if (ms[s] < best[s]) {
        best[s] = ms[s];
        best_grid[s] = g;
      }
  }
  for (int s = 0; s < RAPID_MAX_STAGES; s++) ctx->stage_grid[s] = s < ctx->nstages ? best_grid[s] : 0;
  for (int s = 0; s < ctx->nstages; s++) {
    if (grids_out) grids_out[s] = best_grid[s];
    if (shapes_out) shapes_out[s] = best_shape[s];
  }
  ctx->profiling = saved_prof;
  ctx->graph_on = saved_graph;
  return rs;
}

// ---------------------------------------------------------------- linear classifier
extern "C" rapid_status rapid_set_classifier(rapid_ctx *ctx, const double *theta5) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (theta5)
    for (int i = 0; i < 5; i++)
      if (!std::isfinite(theta5[i])) return RAPID_EINVAL;
  drop_graph(ctx);
  ctx->theta_on = theta5 != nullptr;
  for (int i = 0; i < 5; i++) ctx->theta[i] = theta5 ? theta5[i] : 0.0;
  return RAPID_OK;
}

extern "C" rapid_status rapid_read_features(rapid_ctx *ctx, int32_t i, double *dst_host) {
  if (!ctx || !dst_host) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (!ctx->theta_on || !ctx->image_set) return RAPID_ESTATE;
  if (i < 0 || i >= ctx->nimg) return RAPID_EINVAL;
  const ImgHost &h = ctx->im[i];
  CK(cudaMemcpyAsync(dst_host, ctx->st.feat + 4ll * h.label0, sizeof(double) * 4 * (size_t)h.M,
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return RAPID_OK;
}

// ---------------------------------------------------------------- learned scorer
extern "C" rapid_status rapid_set_scorer(rapid_ctx *ctx, const float *weights, float threshold) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  drop_graph(ctx);
  if (!weights) {
    ctx->scorer_on = 0;
    return RAPID_OK;
  }
  if (!(threshold >= 0.f && threshold <= 1.f)) return RAPID_EINVAL;
  if (ctx->p.schedule != 0) return RAPID_EINVAL;  // pruned sweeps are defined for schedule 0 only
  if (ctx->keep_on) return RAPID_EINVAL;          // one source of masks at a time
  for (int i = 0; i < RAPID_SCORER_PARAMS; i++)
    if (!std::isfinite(weights[i])) return RAPID_EINVAL;
  if (!ctx->d_scorer && dev_malloc((void **)&ctx->d_scorer, scorer_dev_bytes()) != cudaSuccess) return RAPID_ENOMEM;
  CK(scorer_upload(weights, ctx->d_scorer, &ctx->sdev, ctx->stream));
  ctx->scorer_thr = threshold;
  ctx->scorer_on = 1;
  if (ctx->image_set) {
    if (!grow(&ctx->d_mask, &ctx->mask_cap, ctx->lab_total)) return RAPID_ENOMEM;
    return build_descriptors(ctx);
  }
  return RAPID_OK;
}

extern "C" rapid_status rapid_set_race_check(rapid_ctx *ctx, int32_t on) {
  if (!ctx || (on & ~1)) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  drop_graph(ctx);
  if (!on) {
    ctx->race_on = 0;
    return RAPID_OK;
  }
  if (!ctx->d_race) {
    if (dev_malloc((void **)&ctx->d_race, sizeof(unsigned long long)) != cudaSuccess) return RAPID_ENOMEM;
    CK(cudaMemsetAsync(ctx->d_race, 0, sizeof(unsigned long long), ctx->stream));
  }
  if (ctx->image_set && !grow(&ctx->d_wstamp, &ctx->wstamp_cap, ctx->lab_total * sizeof(int))) return RAPID_ENOMEM;
  ctx->race_on = 1;
  return RAPID_OK;
}

extern "C" rapid_status rapid_read_race_violations(rapid_ctx *ctx, int64_t *out) {
  if (!ctx || !out) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  unsigned long long v = 0;
  if (ctx->d_race) {
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(&v, ctx->d_race, sizeof v, cudaMemcpyDeviceToHost));
  }
  *out = (int64_t)v;
  return RAPID_OK;
}

extern "C" rapid_status rapid_set_scorer_stages(rapid_ctx *ctx, const int32_t *on, int32_t n) {
  if (!ctx || n < 0 || n > RAPID_MAX_STAGES || (n > 0 && !on)) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  for (int i = 0; i < n; i++)
    if (on[i] & ~1) return RAPID_EINVAL;
  drop_graph(ctx);
  for (int i = 0; i < RAPID_MAX_STAGES; i++) ctx->scorer_off[i] = i < n ? !on[i] : 0;
  return RAPID_OK;
}

extern "C" rapid_status rapid_set_keep_mask(rapid_ctx *ctx, int32_t i, int32_t s, const uint8_t *mask, int64_t n,
                                            int32_t mask_is_device) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (!mask) {  // clear every mask
    if (i != -1 || s != -1) return RAPID_EINVAL;
    if (ctx->keep_on) drop_graph(ctx);
    ctx->keep_on = 0;
    std::memset(ctx->keep_stage, 0, sizeof ctx->keep_stage);
    return RAPID_OK;
  }
  if (!ctx->image_set) return RAPID_ESTATE;
  if (i < 0 || i >= ctx->nimg || s < 0 || s >= ctx->nstages || (mask_is_device & ~1)) return RAPID_EINVAL;
  if (ctx->p.schedule != 0 || ctx->scorer_on) return RAPID_EINVAL;
  const ImageDesc &d = ctx->h_desc[(size_t)s * ctx->nimg + i];
  if (n != (int64_t)d.nbx * d.nby) return RAPID_EINVAL;
  drop_graph(ctx);
  if (!ctx->keep_on) {  // every (stage, image) mask starts as "keep every block"
    size_t off = 0;
    for (int st = 0; st < ctx->nstages; st++)
      for (int m = 0; m < ctx->nimg; m++) {
        const ImageDesc &e = ctx->h_desc[(size_t)st * ctx->nimg + m];
        ctx->keep_off[st][m] = off;
        off = round_up(off + (size_t)e.nbx * e.nby, 256);
      }
    if (!grow(&ctx->d_keep, &ctx->keep_cap, off)) return RAPID_ENOMEM;
    if (!grow(&ctx->d_mask, &ctx->mask_cap, ctx->lab_total)) return RAPID_ENOMEM;
    CK(cudaMemsetAsync(ctx->d_keep, 1, off, ctx->stream));
    ctx->keep_on = 1;
    std::memset(ctx->keep_stage, 0, sizeof ctx->keep_stage);
    rapid_status rs = build_descriptors(ctx);  // the descriptors now point at the mask buffer
    if (rs != RAPID_OK) return rs;
  }
  CK(cudaMemcpyAsync(ctx->d_keep + ctx->keep_off[s][i], mask, (size_t)n,
                     mask_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->keep_stage[s] = 1;
  return RAPID_OK;
}

extern "C" rapid_status rapid_scorer_features(rapid_ctx *ctx, int32_t i, float *dst_dev) {
  if (!ctx || !dst_dev) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (ctx->cur < 0) return RAPID_ESTATE;
  if (i < 0 || i >= ctx->nimg) return RAPID_EINVAL;
  StageArgs a = stage_args(ctx, ctx->cur);
  CK(launch_features(a, host_desc(ctx, ctx->cur)[i], ctx->L, dst_dev, ctx->stream));
  ctx->launches++;
  return RAPID_OK;
}

extern "C" rapid_status rapid_scorer_scores(rapid_ctx *ctx, int32_t i, const float *weights, float *dst_dev) {
  if (!ctx || !weights || !dst_dev) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (ctx->cur < 0) return RAPID_ESTATE;
  if (i < 0 || i >= ctx->nimg) return RAPID_EINVAL;
  if (!ctx->d_scorer_tmp && dev_malloc((void **)&ctx->d_scorer_tmp, scorer_dev_bytes()) != cudaSuccess) return RAPID_ENOMEM;
  ScorerDev w;
  CK(scorer_upload(weights, ctx->d_scorer_tmp, &w, ctx->stream));
  StageArgs a = stage_args(ctx, ctx->cur);
  CK(launch_score(a, host_desc(ctx, ctx->cur)[i], ctx->L, w, 0.f, dst_dev, nullptr, ctx->stream));
  ctx->launches++;
  return RAPID_OK;
}

extern "C" rapid_status rapid_trainer_create(int64_t capacity, float neg_rate, rapid_trainer **out) {
  if (!out) return RAPID_EINVAL;
  *out = nullptr;
  if (capacity < 1 || capacity > (1ll << 30) || !(neg_rate >= 0.f && neg_rate <= 1.f)) return RAPID_EINVAL;
  rapid_trainer *t = new (std::nothrow) rapid_trainer;
  if (!t) return RAPID_ENOMEM;
  std::memset(t, 0, sizeof *t);
  t->neg_rate = neg_rate;
  bool ok = dev_malloc((void **)&t->buf_x, (size_t)capacity * kScorerPatchFloats * sizeof(float)) == cudaSuccess &&
            dev_malloc((void **)&t->buf_inb, (size_t)capacity * sizeof(unsigned long long)) == cudaSuccess &&
            dev_malloc((void **)&t->buf_y, (size_t)capacity * sizeof(float)) == cudaSuccess &&
            dev_malloc((void **)&t->buf_count, sizeof(int)) == cudaSuccess &&
            cudaMemset(t->buf_count, 0, sizeof(int)) == cudaSuccess;
  if (!ok) {
    rapid_trainer_destroy(t);
    return RAPID_ENOMEM;
  }
  t->ts.x = t->buf_x;
  t->ts.inb = t->buf_inb;
  t->ts.y = t->buf_y;
  t->ts.count = t->buf_count;
  t->ts.cap = capacity;
  *out = t;
  return RAPID_OK;
}

extern "C" void rapid_trainer_destroy(rapid_trainer *t) {
  if (!t) return;
  cudaDeviceSynchronize();
  cudaFree(t->buf_x);
  cudaFree(t->buf_inb);
  cudaFree(t->buf_y);
  cudaFree(t->buf_count);
  delete t;
}

extern "C" rapid_status rapid_set_logging(rapid_ctx *ctx, rapid_trainer *t) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  drop_graph(ctx);
  ctx->logger = t;
  if (t && ctx->image_set) {
    if (!grow(&ctx->d_feat, &ctx->feat_cap, ctx->lab_total * kScorerFeatures() * sizeof(float))) return RAPID_ENOMEM;
    if (!grow(&ctx->d_before, &ctx->before_cap, ctx->lab_total * sizeof(int))) return RAPID_ENOMEM;
    if (!grow(&ctx->d_collect, &ctx->collect_cap, collect_scratch_ints((long long)ctx->lab_total) * sizeof(int)))
      return RAPID_ENOMEM;
  }
  return RAPID_OK;
}

static long long trainer_samples(rapid_trainer *t) {
  int c = 0;
  if (cudaMemcpy(&c, t->buf_count, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return std::min<long long>(c, t->ts.cap);
}

extern "C" rapid_status rapid_trainer_count(rapid_trainer *t, int64_t *samples, int64_t *positives) {
  if (!t) return RAPID_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return RAPID_ECUDA;
  const long long n = trainer_samples(t);
  if (n < 0) return RAPID_ECUDA;
  if (samples) *samples = n;
  if (positives) {
    float *y = (float *)std::malloc((size_t)std::max<long long>(n, 1) * sizeof(float));
    if (!y) return RAPID_ENOMEM;
    if (n > 0 && cudaMemcpy(y, t->buf_y, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
      std::free(y);
      return RAPID_ECUDA;
    }
    long long p = 0;
    for (long long i = 0; i < n; i++) p += y[i] > 0.5f;
    std::free(y);
    *positives = p;
  }
  return RAPID_OK;
}

// xorshift64* generator for the shuffles and the initial weights
static unsigned long long next_u64(unsigned long long &s) {
  s ^= s >> 12;
  s ^= s << 25;
  s ^= s >> 27;
  return s * 2685821657736338717ull;
}

extern "C" rapid_status rapid_trainer_fit(rapid_trainer *t, int32_t epochs, int32_t batch, float lr, float pos_weight,
                                          uint64_t seed, const float *init, float *weights_out, float *epoch_loss) {
  if (!t || !weights_out || epochs < 1 || batch < 1 || !(lr > 0.f) || !(pos_weight > 0.f)) return RAPID_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return RAPID_ECUDA;
  const long long n = trainer_samples(t);
  if (n < 1) return RAPID_ESTATE;
  const int nP = RAPID_SCORER_PARAMS;
  float w0[RAPID_SCORER_PARAMS];
  unsigned long long rng = seed * 0x9E3779B97F4A7C15ull + 1;
  if (init) {
    std::memcpy(w0, init, sizeof w0);
  } else {  // uniform Glorot start for the weights, zero biases
    auto fill = [&](int off, int count, int fan_in, int fan_out) {
      const float b = std::sqrt(6.f / (float)(fan_in + fan_out));
      for (int i = 0; i < count; i++)
        w0[off + i] = b * (2.f * (float)((next_u64(rng) >> 40) / 16777216.0) - 1.f);
    };
    std::memset(w0, 0, sizeof w0);
    fill(0, 16 * 9 * 9, 9 * 9, 16 * 9);
    fill(16 * 9 * 9 + 16, 16 * 16 * 9, 16 * 9, 16 * 9);
    fill(16 * 9 * 9 + 16 + 16 * 16 * 9 + 16, 16 * 9, 16 * 9, 9);
  }
  float *d = nullptr;  // w, m, v, grad, loss
  float *part = nullptr;  // per-CTA gradient rows and losses of a minibatch
  int *order = nullptr;
  int *horder = (int *)std::malloc((size_t)n * sizeof(int));
  rapid_status rs = RAPID_OK;
  const size_t nparts = (size_t)train_max_ctas();
  if (!horder || dev_malloc((void **)&d, (4 * (size_t)nP + 1) * sizeof(float)) != cudaSuccess ||
      dev_malloc((void **)&part, nparts * (nP + 1) * sizeof(float)) != cudaSuccess ||
      dev_malloc((void **)&order, (size_t)n * sizeof(int)) != cudaSuccess)
    rs = RAPID_ENOMEM;
  float *w = d, *m = d + nP, *v = d + 2 * nP, *grad = d + 3 * nP, *loss = d + 4 * nP;
  float *part_loss = part + nparts * nP;
  if (rs == RAPID_OK && (cudaMemcpy(w, w0, nP * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemset(m, 0, (3 * (size_t)nP + 1) * sizeof(float)) != cudaSuccess))
    rs = RAPID_ECUDA;
  for (long long i = 0; i < n && horder; i++) horder[i] = (int)i;
  long long step = 0;
  for (int e = 0; e < epochs && rs == RAPID_OK; e++) {
    for (long long i = n - 1; i > 0; i--) {  // Fisher-Yates shuffle
      const long long j = (long long)(next_u64(rng) % (unsigned long long)(i + 1));
      std::swap(horder[i], horder[j]);
    }
    if (cudaMemcpy(order, horder, (size_t)n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(loss, 0, sizeof(float)) != cudaSuccess) {
      rs = RAPID_ECUDA;
      break;
    }
    for (long long off = 0; off < n; off += batch) {
      const int bs = (int)std::min<long long>(batch, n - off);
      step++;
      const float bc1 = 1.f - std::pow(0.9f, (float)step), bc2 = 1.f - std::pow(0.999f, (float)step);
      if (launch_train_step(t->ts, (int)n, w, order, (int)off, bs, pos_weight, part, part_loss, grad, loss, 0) !=
              cudaSuccess ||
          launch_adam(w, m, v, grad, lr, bc1, bc2, 1.f / (float)bs, 0) != cudaSuccess) {
        rs = RAPID_ECUDA;
        break;
      }
    }
    float l = 0.f;
    if (rs == RAPID_OK && cudaMemcpy(&l, loss, sizeof l, cudaMemcpyDeviceToHost) != cudaSuccess) rs = RAPID_ECUDA;
    if (epoch_loss) epoch_loss[e] = l / (float)n;
  }
  if (rs == RAPID_OK && cudaMemcpy(weights_out, w, nP * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    rs = RAPID_ECUDA;
  cudaFree(d);
  cudaFree(part);
  cudaFree(order);
  std::free(horder);
  return rs;
}

extern "C" rapid_status rapid_trainer_samples(rapid_trainer *t, int64_t first, int32_t count, float *x_out,
                                              uint64_t *inb_out, float *y_out) {
  if (!t || first < 0 || count < 1) return RAPID_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return RAPID_ECUDA;
  const long long n = trainer_samples(t);
  if (n < 0) return RAPID_ECUDA;
  if (first + count > n) return RAPID_ERANGE;
  if (x_out && cudaMemcpy(x_out, t->buf_x + first * kScorerPatchFloats, (size_t)count * kScorerPatchFloats * 4,
                          cudaMemcpyDeviceToHost) != cudaSuccess)
    return RAPID_ECUDA;
  if (inb_out && cudaMemcpy(inb_out, t->buf_inb + first, (size_t)count * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return RAPID_ECUDA;
  if (y_out && cudaMemcpy(y_out, t->buf_y + first, (size_t)count * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return RAPID_ECUDA;
  return RAPID_OK;
}

extern "C" rapid_status rapid_trainer_gradient(rapid_trainer *t, const float *weights, int64_t first, int32_t count,
                                               float pos_weight, float *grad_out, float *loss_out) {
  if (!t || !weights || !grad_out || first < 0 || count < 1 || !(pos_weight > 0.f)) return RAPID_EINVAL;
  for (int i = 0; i < RAPID_SCORER_PARAMS; i++)
    if (!std::isfinite(weights[i])) return RAPID_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return RAPID_ECUDA;
  const long long n = trainer_samples(t);
  if (n < 0) return RAPID_ECUDA;
  if (first + count > n) return RAPID_ERANGE;
  const int nP = RAPID_SCORER_PARAMS;
  const size_t nparts = (size_t)train_max_ctas();
  float *d = nullptr, *part = nullptr;
  int *order = nullptr;
  int *horder = (int *)std::malloc((size_t)count * sizeof(int));
  rapid_status rs = RAPID_OK;
  if (!horder || dev_malloc((void **)&d, (2 * (size_t)nP + 1) * sizeof(float)) != cudaSuccess ||
      dev_malloc((void **)&part, nparts * (nP + 1) * sizeof(float)) != cudaSuccess ||
      dev_malloc((void **)&order, (size_t)count * sizeof(int)) != cudaSuccess)
    rs = RAPID_ENOMEM;
  for (int i = 0; i < count && horder; i++) horder[i] = (int)(first + i);
  float *w = d, *grad = d + nP, *loss = d + 2 * nP;
  if (rs == RAPID_OK &&
      (cudaMemcpy(w, weights, nP * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(order, horder, (size_t)count * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemset(loss, 0, sizeof(float)) != cudaSuccess ||
       launch_train_step(t->ts, count, w, order, 0, count, pos_weight, part, part + nparts * nP, grad, loss, 0) !=
           cudaSuccess ||
       cudaMemcpy(grad_out, grad, nP * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
       (loss_out && cudaMemcpy(loss_out, loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)))
    rs = RAPID_ECUDA;
  cudaFree(d);
  cudaFree(part);
  cudaFree(order);
  std::free(horder);
  return rs;
}

// ---------------------------------------------------------------- whole slides
static constexpr long long kSlideBatchPixels = 1ll << 30;

extern "C" rapid_status rapid_refine_slide(rapid_ctx *ctx, const uint8_t *rgb_dev, int64_t H, int64_t W,
                                           int64_t rgb_pitch_bytes, int32_t max_tile, int32_t px_per_superpixel,
                                           int32_t autotune, int32_t *labels_dev, int64_t labels_pitch_bytes,
                                           rapid_sp_stats *stats_dev, int64_t stats_capacity, int64_t *M_out,
                                           int32_t *tiles_out) {
  if (!ctx || !rgb_dev || !labels_dev) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (H < 1 || W < 1 || rgb_pitch_bytes < 3 * W || labels_pitch_bytes < 4 * W || labels_pitch_bytes % 4) return RAPID_EINVAL;
  if (max_tile < 16 || max_tile > 46340 || px_per_superpixel < 1 || (stats_dev && stats_capacity < 0)) return RAPID_EINVAL;
  // even row and column bands (Eq. parallel_spit) no longer than max_tile
  const long long nr = (H + max_tile - 1) / max_tile, nc = (W + max_tile - 1) / max_tile;
  if (nr * nc > (1ll << 24)) return RAPID_ERANGE;
  rapid_status rs = RAPID_OK;
  const uint8_t *ptrs[kMaxBatch];
  int32_t hs[kMaxBatch], ws[kMaxBatch], ks[kMaxBatch];
  int64_t pitches[kMaxBatch];
  long long r0s[kMaxBatch], c0s[kMaxBatch];
  long long id_base = 0, t = 0;
  bool tuned = false;
  while (rs == RAPID_OK && t < nr * nc) {
    // a batch: up to kMaxBatch tiles and at most kSlideBatchPixels pixels (its block and label
    // indices are 32-bit), at least one tile
    int n = 0;
    long long batch_px = 0;
    for (; n < kMaxBatch && t < nr * nc; n++, t++) {
      const long long i = t / nc, j = t % nc;
      const long long r0 = H * i / nr, r1 = H * (i + 1) / nr, c0 = W * j / nc, c1 = W * (j + 1) / nc;
      if (n > 0 && batch_px + (r1 - r0) * (c1 - c0) > kSlideBatchPixels) break;
      batch_px += (r1 - r0) * (c1 - c0);
      ptrs[n] = rgb_dev + r0 * rgb_pitch_bytes + 3 * c0;
      hs[n] = (int32_t)(r1 - r0);
      ws[n] = (int32_t)(c1 - c0);
      ks[n] = (int32_t)std::max<long long>(1, (r1 - r0) * (c1 - c0) / px_per_superpixel);
      pitches[n] = rgb_pitch_bytes;
      r0s[n] = r0;
      c0s[n] = c0;
    }
    rs = rapid_set_images(ctx, n, ptrs, hs, ws, pitches, ks, 1);
    if (rs == RAPID_OK && autotune && !tuned) {  // the first batch's geometry serves them all
      // (a context keeps the geometry it was given or tuned before: pass autotune = 0 then)
      rs = rapid_autotune(ctx, nullptr, nullptr);
      tuned = true;
    }
    if (rs == RAPID_OK) rs = rapid_run(ctx);
    if (rs != RAPID_OK) break;
    if (id_base + ctx->M_total >= INT_MAX) {
      rs = RAPID_ERANGE;
      break;
    }
    // each tile's labels go into the slide's map as slide-wide ids (id_base + its ids)
    const int side = ctx->st_side[ctx->cur];
    for (int k = 0; k < n && rs == RAPID_OK; k++) {
      const ImgHost &h = ctx->im[k];
      const ImageDesc &d = host_desc(ctx, ctx->cur)[k];
      int32_t *dst = (int32_t *)((char *)labels_dev + r0s[k] * labels_pitch_bytes) + c0s[k];
      // the context's ids are already numbered across the batch: subtract -id_base
      if (launch_upsample(d.lab, d.nbx, side, h.H, h.W, -(int)id_base, dst, labels_pitch_bytes / 4, ctx->stream) !=
          cudaSuccess)
        rs = cuda_fail(ctx);
      if (rs == RAPID_OK && stats_dev && id_base + h.label0 + h.M <= stats_capacity &&
          launch_pack_stats(ctx->st, h.label0, h.M, stats_dev + id_base + h.label0, ctx->stream) != cudaSuccess)
        rs = cuda_fail(ctx);
    }
    id_base += ctx->M_total;
    if (rs == RAPID_OK) rs = rapid_sync(ctx);  // the next batch reuses the context's buffers
  }
  if (rs == RAPID_OK && stats_dev && id_base > stats_capacity) rs = RAPID_EINVAL;
  if (M_out) *M_out = id_base;
  if (tiles_out) *tiles_out = (int32_t)(nr * nc);
  return rs;
}

extern "C" rapid_status rapid_get_state(rapid_ctx *ctx, int32_t *stage, int32_t *level, int32_t *block,
                                        int32_t *M) {
  if (!ctx) return RAPID_EINVAL;
  if (stage) *stage = ctx->cur;
  if (level) *level = ctx->cur >= 0 ? ctx->st_level[ctx->cur] : 0;
  if (block) *block = ctx->cur >= 0 ? ctx->st_side[ctx->cur] : 0;
  if (M) *M = ctx->cur >= 0 ? ctx->im[0].M : 0;
  return RAPID_OK;
}

extern "C" rapid_status rapid_get_image_info(rapid_ctx *ctx, int32_t i, int32_t *H, int32_t *W, int32_t *M) {
  if (!ctx || !ctx->image_set || i < 0 || i >= ctx->nimg) return RAPID_EINVAL;
  if (H) *H = ctx->im[i].H;
  if (W) *W = ctx->im[i].W;
  if (M) *M = ctx->im[i].M;
  return RAPID_OK;
}

extern "C" rapid_status rapid_read_image_labels(rapid_ctx *ctx, int32_t i, int32_t *dst, int64_t row_pitch_bytes,
                                                int32_t dst_is_device) {
  if (!ctx || !dst) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (ctx->cur < 0) return RAPID_ESTATE;
  if (i < 0 || i >= ctx->nimg) return RAPID_EINVAL;
  const ImgHost &h = ctx->im[i];
  const ImageDesc &d = host_desc(ctx, ctx->cur)[i];
  if (row_pitch_bytes < 4ll * h.W || (row_pitch_bytes % 4) != 0) return RAPID_EINVAL;
  const int side = ctx->st_side[ctx->cur];
  if (side == 1 && h.label0 == 0) {
    CK(cudaMemcpy2DAsync(dst, row_pitch_bytes, d.lab, 4ull * h.W, 4ull * h.W, h.H,
                         dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  } else if (dst_is_device) {
    CK(launch_upsample(d.lab, d.nbx, side, h.H, h.W, h.label0, dst, row_pitch_bytes / 4, ctx->stream));
    ctx->launches++;
  } else {
    CK(launch_upsample(d.lab, d.nbx, side, h.H, h.W, h.label0, ctx->d_full, h.W, ctx->stream));
    ctx->launches++;
    CK(cudaMemcpy2DAsync(dst, row_pitch_bytes, ctx->d_full, 4ull * h.W, 4ull * h.W, h.H, cudaMemcpyDeviceToHost,
                         ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return read_device_error(ctx);
}

extern "C" rapid_status rapid_read_labels(rapid_ctx *ctx, int32_t *dst, int64_t row_pitch_bytes,
                                          int32_t dst_is_device) {
  return rapid_read_image_labels(ctx, 0, dst, row_pitch_bytes, dst_is_device);
}

extern "C" rapid_status rapid_read_block_labels(rapid_ctx *ctx, int32_t *dst, int64_t capacity, int32_t *nbx_out,
                                                int32_t *nby_out) {
  if (!ctx || !dst) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (ctx->cur < 0) return RAPID_ESTATE;
  const ImageDesc &d = host_desc(ctx, ctx->cur)[0];  // image 0: its global ids are its own ids
  const long long n = (long long)d.nbx * d.nby;
  if (capacity < n) return RAPID_EINVAL;
  CK(cudaMemcpyAsync(dst, d.lab, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (nbx_out) *nbx_out = d.nbx;
  if (nby_out) *nby_out = d.nby;
  return read_device_error(ctx);
}

extern "C" rapid_status rapid_read_image_stats(rapid_ctx *ctx, int32_t i, rapid_sp_stats *dst, int64_t capacity,
                                               int64_t *M_out) {
  if (!ctx || !dst) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (ctx->cur < 0) return RAPID_ESTATE;
  if (i < 0 || i >= ctx->nimg) return RAPID_EINVAL;
  const ImgHost &h = ctx->im[i];
  if (capacity < h.M) return RAPID_EINVAL;
  CK(launch_pack_stats(ctx->st, h.label0, h.M, ctx->d_pack, ctx->stream));
  ctx->launches++;
  CK(cudaMemcpyAsync(dst, ctx->d_pack, (size_t)h.M * sizeof(rapid_sp_stats), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (M_out) *M_out = h.M;
  return read_device_error(ctx);
}

extern "C" rapid_status rapid_read_stats(rapid_ctx *ctx, rapid_sp_stats *dst, int64_t capacity, int64_t *M_out) {
  return rapid_read_image_stats(ctx, 0, dst, capacity, M_out);
}

extern "C" rapid_status rapid_read_image_counters(rapid_ctx *ctx, int32_t i, rapid_counters *dst) {
  if (!ctx || !dst) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (i < 0 || i >= (ctx->image_set ? ctx->nimg : 1)) return RAPID_EINVAL;
  std::memset(dst, 0, sizeof *dst);
  CK(cudaStreamSynchronize(ctx->stream));
  rapid_status rs = read_device_error(ctx);
  if (rs != RAPID_OK) return rs;
  long long c[CNT_N * RAPID_MAX_STAGES];
  CK(cudaMemcpy(c, ctx->ctl.cnt + (long long)i * kCntStride, sizeof c, cudaMemcpyDeviceToHost));
  long long pr[PROF_N * RAPID_MAX_STAGES];
  CK(cudaMemcpy(pr, ctx->prof, sizeof pr, cudaMemcpyDeviceToHost));
  dst->num_stages = ctx->cur >= 0 ? ctx->nstages : 0;
  dst->M = ctx->cur >= 0 ? ctx->im[i].M : 0;
  dst->launches = ctx->launches;
  for (int s = 0; s < dst->num_stages; s++) {
    rapid_stage_counters &o = dst->stage[s];
    const long long *ci = c + (long long)CNT_N * s;
    o.level = (int32_t)ci[CNT_LEVEL];
    o.block = (int32_t)ci[CNT_SIDE];
    o.sweeps = (int32_t)ci[CNT_SWEEPS];
    o.eligible = ci[CNT_ELIG];
    o.evaluated = ci[CNT_EVAL];
    o.moves = ci[CNT_MOVES];
    o.merge_requests = ci[CNT_REQ];
    o.merges = ci[CNT_MERGES];
    o.fp64_fallbacks = ci[CNT_FALLBACK];
    o.filter_mismatches = ci[CNT_MISMATCH];
    o.tiles_scanned = ci[CNT_SCANNED];
    o.tiles_skipped = ci[CNT_SKIPPED];
    o.merge_searches = ci[CNT_SEARCHES];
    o.merge_cache_hits = ci[CNT_CACHE_HITS];
    o.kernel_ms = -1.0f;
    for (int j = 0; j < PROF_N; j++) o.section_ms[j] = ctx->profiling ? (float)(pr[s * PROF_N + j] * 1e-6) : 0.0f;
    if (ctx->profiling && ctx->ev_ok[s] && s <= ctx->cur) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ctx->ev[s][0], ctx->ev[s][1]) == cudaSuccess) o.kernel_ms = ms;
    }
  }
  return RAPID_OK;
}

extern "C" rapid_status rapid_read_counters(rapid_ctx *ctx, rapid_counters *dst) {
  return rapid_read_image_counters(ctx, 0, dst);
}

extern "C" rapid_status rapid_set_profiling(rapid_ctx *ctx, int32_t on) {
  if (!ctx) return RAPID_EINVAL;
  ctx->profiling = on ? 1 : 0;
  return RAPID_OK;
}

extern "C" rapid_status rapid_simple_table(uint8_t *out256) {
  if (!out256) return RAPID_EINVAL;
  unsigned char *d = nullptr;
  if (dev_malloc((void **)&d, 256) != cudaSuccess) return RAPID_ENOMEM;
  cudaError_t e = launch_simple_table(d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out256, d, 256, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? RAPID_OK : RAPID_ECUDA;
}

extern "C" const char *rapid_status_string(rapid_status s) {
  switch (s) {
    case RAPID_OK: return "RAPID_OK";
    case RAPID_EINVAL: return "RAPID_EINVAL: invalid argument";
    case RAPID_ENOMEM: return "RAPID_ENOMEM: allocation failed";
    case RAPID_ECUDA: return "RAPID_ECUDA: CUDA error";
    case RAPID_ESTATE: return "RAPID_ESTATE: call out of order";
    case RAPID_ETIMEOUT: return "RAPID_ETIMEOUT: device wait gave up";
    case RAPID_ERANGE: return "RAPID_ERANGE: exactness or size limit exceeded";
  }
  return "RAPID_?: unknown status";
}
