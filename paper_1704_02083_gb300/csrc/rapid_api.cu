// rapid_api.cu — the C ABI (include/rapid.h): context, device buffers, stage schedule and
// launch orchestration.  Host code only; every step of the method runs in the kernels of
// k_prep.cu and k_stage.cu.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/rapid.h"
#include "rapid_dev.cuh"

namespace rapid {
cudaError_t launch_pyramid(const unsigned char *img, long long pitch, int H, int W, int f, int Wl, int Hl,
                           int4 *out, cudaStream_t s);
cudaError_t launch_seed(const StageArgs &a, int gx, int gy, cudaStream_t s, int *launches);
cudaError_t launch_recompute(const StageArgs &a, cudaStream_t s, int *launches);
cudaError_t launch_split(const int *src, int snbx, int *dst, int dnbx, int dnby, cudaStream_t s);
cudaError_t launch_predict(const int *lab, int nbx, int nby, const DevStats &st, long long hT, cudaStream_t s,
                           int *launches);
cudaError_t launch_upsample(const int *lab, int nbx, int side, int H, int W, int *dst, long long pitch_elems,
                            cudaStream_t s);
cudaError_t launch_pack_stats(const DevStats &st, rapid_sp_stats *out, cudaStream_t s);
cudaError_t launch_simple_table(unsigned char *out, cudaStream_t s);
cudaError_t launch_init_counters(long long *cnt, const Schedule &sch, cudaStream_t s);
}  // namespace rapid

using namespace rapid;

static const int kMaxLevels = 8;

struct rapid_ctx {
  rapid_params p;
  cudaStream_t stream;
  int device, nsm, coop_grid, coop_block;
  rapid_status sticky;
  // image and levels
  int H, W;
  long long pitch;
  unsigned char *d_img;
  size_t img_cap;
  int L;
  int f[kMaxLevels + 1], Wl[kMaxLevels + 1], Hl[kMaxLevels + 1];
  // box-sum levels for block sums (factors sf[i] > 1, ascending)
  int nsf;
  int sf[kMaxSumLevels], sfW[kMaxSumLevels], sfH[kMaxSumLevels];
  int4 *d_pyr[kMaxSumLevels];
  size_t pyr_cap[kMaxSumLevels];
  // schedule
  int nstages;
  int st_level[RAPID_MAX_STAGES], st_side[RAPID_MAX_STAGES];
  int cur, nbx, nby, cur_buf;
  bool image_set;
  int *d_lab[2];
  long long lab_cap;
  int *d_full;  // full-res staging for host reads at side > 1
  int *d_trec;  // tile scan records, sized for the finest stage
  long long trec_cap;
  long long full_cap;
  // labels
  int M, M_cap;
  void *d_label_block;
  DevStats st;
  DevMerge mg;
  rapid_sp_stats *d_pack;
  // control
  void *d_ctl_block;
  DevCtl ctl;
  double lam_pos, lam_b2;
  int imp_on;
  long long launches;
  int profiling;
  long long *prof;  // [RAPID_MAX_STAGES][PROF_N] section times (ns)
  cudaEvent_t ev[RAPID_MAX_STAGES][2];
  int ev_ok[RAPID_MAX_STAGES];
};

static rapid_status cuda_fail(rapid_ctx *c) {
  if (c) c->sticky = RAPID_ECUDA;
  return RAPID_ECUDA;
}

#define CK(call)                             \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx); \
  } while (0)

static bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
static int ceil_div(int a, int b) { return (a + b - 1) / b; }

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
}

static bool params_ok(const rapid_params *p) {
  if (!p) return false;
  if (p->num_levels < 1 || p->num_levels > kMaxLevels) return false;
  if (p->num_levels > 1 && (!is_pow2(p->ratio_C) || p->ratio_C < 2)) return false;
  if (!is_pow2(p->init_block) || !is_pow2(p->final_grain) || p->init_block > (1 << 20)) return false;
  if (p->K < 1 || p->size_mode < 0 || p->size_mode > 2 || p->max_sweeps < 1) return false;
  if (p->lo_den <= 0 || p->hi_den <= 0 || p->lo_num < 0 || p->hi_num < 0) return false;
  if (!std::isfinite(p->lambda_pos0) || !std::isfinite(p->lambda_b)) return false;
  if ((p->predict | p->reuse | p->importance_rule | p->use_filter | p->skip_tiles | p->verify_filter) & ~1)
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
  ctx->coop_block = stage_block_threads();
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_kernel_ptr(), ctx->coop_block, 0);
  if (e != cudaSuccess || !coop || per_sm < 1) {
    delete ctx;
    return RAPID_ECUDA;
  }
  ctx->coop_grid = ctx->nsm * per_sm;
  // control block: barrier (2 u32), error (i32), request/accept counts, sweep changes
  // (3 u64), counters.
  size_t ctl_bytes = 128 + sizeof(long long) * (CNT_N + PROF_N) * RAPID_MAX_STAGES;
  if (cudaMalloc(&ctx->d_ctl_block, ctl_bytes) != cudaSuccess) {
    delete ctx;
    return RAPID_ENOMEM;
  }
  char *b = (char *)ctx->d_ctl_block;
  ctx->ctl.bar = (unsigned *)(b + 0);
  ctx->ctl.err = (int *)(b + 8);
  ctx->ctl.last_merge = (int *)(b + 12);
  ctx->mg.req_count = (int *)(b + 16);    // [2], by phase parity
  ctx->mg.found_count = (int *)(b + 24);  // [2], by phase parity
  ctx->mg.acc_count = (int *)(b + 32);
  ctx->ctl.changes = (unsigned long long *)(b + 40);
  ctx->ctl.cnt = (long long *)(b + 128);
  ctx->prof = (long long *)(b + 128 + sizeof(long long) * CNT_N * RAPID_MAX_STAGES);
  ctx->ctl.spin_ns = p->spin_limit_ns;
  if (cudaMemsetAsync(ctx->d_ctl_block, 0, ctl_bytes, ctx->stream) != cudaSuccess) {
    cudaFree(ctx->d_ctl_block);
    delete ctx;
    return RAPID_ECUDA;
  }
  for (int i = 0; i < RAPID_MAX_STAGES; i++) ctx->ev_ok[i] = 0;
  *out = ctx;
  return RAPID_OK;
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
  cudaFree(ctx->d_lab[0]);
  cudaFree(ctx->d_lab[1]);
  ctx->d_lab[0] = ctx->d_lab[1] = nullptr;
  ctx->lab_cap = 0;
  cudaFree(ctx->d_full);
  ctx->d_full = nullptr;
  ctx->full_cap = 0;
  cudaFree(ctx->d_trec);
  ctx->d_trec = nullptr;
  ctx->trec_cap = 0;
}

extern "C" void rapid_destroy(rapid_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_image_buffers(ctx);
  cudaFree(ctx->d_label_block);
  cudaFree(ctx->d_pack);
  cudaFree(ctx->d_ctl_block);
  for (int i = 0; i < RAPID_MAX_STAGES; i++)
    if (ctx->ev_ok[i]) {
      cudaEventDestroy(ctx->ev[i][0]);
      cudaEventDestroy(ctx->ev[i][1]);
    }
  delete ctx;
}

// Levels f_l = C^(L-l) and the stage schedule: the block side halves from the initial
// block (at least f_1) to the final grain; each side belongs to the coarsest level whose
// factor does not exceed it.
static rapid_status make_schedule(rapid_ctx *ctx) {
  const rapid_params &p = ctx->p;
  ctx->L = p.num_levels;
  for (int l = 1; l <= ctx->L; l++) {
    int f = 1;
    for (int i = 0; i < ctx->L - l; i++) f *= p.ratio_C;
    ctx->f[l] = f;
    ctx->Wl[l] = ceil_div(ctx->W, f);
    ctx->Hl[l] = ceil_div(ctx->H, f);
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
  return RAPID_OK;
}

extern "C" rapid_status rapid_set_image(rapid_ctx *ctx, const uint8_t *rgb, int32_t H, int32_t W,
                                        int64_t row_pitch_bytes, int32_t rgb_is_device) {
  if (!ctx || !rgb) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (H < 1 || W < 1 || row_pitch_bytes < 3ll * W) return RAPID_EINVAL;
  const long long npx = (long long)H * W;
  if (npx >= (1ll << 31)) return RAPID_EINVAL;
  // position sums reach about H*W*max(H,W)/2; keep them exact in binary64
  if ((double)npx * (double)(H > W ? H : W) >= 9007199254740992.0) return RAPID_EINVAL;
  ctx->H = H;
  ctx->W = W;
  ctx->image_set = false;
  ctx->cur = -1;
  rapid_status rs = make_schedule(ctx);
  if (rs != RAPID_OK) return rs;
  ctx->pitch = ((3ll * W + 15) / 16) * 16;
  size_t need = (size_t)ctx->pitch * H;
  if (need > ctx->img_cap) {
    cudaFree(ctx->d_img);
    ctx->d_img = nullptr;
    ctx->img_cap = 0;
    if (cudaMalloc(&ctx->d_img, need) != cudaSuccess) return RAPID_ENOMEM;
    ctx->img_cap = need;
  }
  ctx->nsf = sum_factors(ctx->f, ctx->L, ctx->st_side[0], ctx->sf);
  // a sum level keeps int32 channel sums: one cell (at most f x f pixels of 255) must fit
  for (int l = 0; l < ctx->nsf; l++)
    if ((long long)std::min(ctx->sf[l], W) * std::min(ctx->sf[l], H) * 255 > INT_MAX) return RAPID_ERANGE;
  for (int l = 0; l < ctx->nsf; l++) {
    ctx->sfW[l] = ceil_div(W, ctx->sf[l]);
    ctx->sfH[l] = ceil_div(H, ctx->sf[l]);
    size_t pn = (size_t)ctx->sfW[l] * ctx->sfH[l] * sizeof(int4);
    if (pn > ctx->pyr_cap[l]) {
      cudaFree(ctx->d_pyr[l]);
      ctx->d_pyr[l] = nullptr;
      ctx->pyr_cap[l] = 0;
      if (cudaMalloc(&ctx->d_pyr[l], pn) != cudaSuccess) return RAPID_ENOMEM;
      ctx->pyr_cap[l] = pn;
    }
  }
  const int sl = ctx->st_side[ctx->nstages - 1];
  long long cap = (long long)ceil_div(W, sl) * ceil_div(H, sl);
  if (cap > ctx->lab_cap) {
    cudaFree(ctx->d_lab[0]);
    cudaFree(ctx->d_lab[1]);
    ctx->d_lab[0] = ctx->d_lab[1] = nullptr;
    ctx->lab_cap = 0;
    if (cudaMalloc(&ctx->d_lab[0], cap * sizeof(int)) != cudaSuccess) return RAPID_ENOMEM;
    if (cudaMalloc(&ctx->d_lab[1], cap * sizeof(int)) != cudaSuccess) return RAPID_ENOMEM;
    ctx->lab_cap = cap;
  }
  {
    // tile records: the finest stage has the most tiles
    const long long nbx = ceil_div(W, sl), nby = ceil_div(H, sl);
    const long long nrec = ((nbx + kTileW - 1) / kTileW) * ((nby + kTileH - 1) / kTileH) * 9 * kRecInts;
    if (nrec > ctx->trec_cap) {
      cudaFree(ctx->d_trec);
      ctx->d_trec = nullptr;
      ctx->trec_cap = 0;
      if (cudaMalloc(&ctx->d_trec, nrec * sizeof(int)) != cudaSuccess) return RAPID_ENOMEM;
      ctx->trec_cap = nrec;
    }
  }
  CK(cudaMemcpy2DAsync(ctx->d_img, ctx->pitch, rgb, row_pitch_bytes, 3ull * W, H,
                       rgb_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  if (!rgb_is_device) CK(cudaStreamSynchronize(ctx->stream));
  ctx->image_set = true;
  return RAPID_OK;
}

static StageArgs stage_args(rapid_ctx *ctx) {
  StageArgs a;
  std::memset(&a, 0, sizeof a);
  a.H = ctx->H;
  a.W = ctx->W;
  a.side = ctx->st_side[ctx->cur];
  a.nbx = ctx->nbx;
  a.nby = ctx->nby;
  a.level = ctx->st_level[ctx->cur];
  // colour sums from the coarsest box-sum level whose cells fit in a block
  a.f = 1;
  a.pyr = nullptr;
  for (int l = 0; l < ctx->nsf; l++)
    if (ctx->sf[l] <= a.side) {
      a.f = ctx->sf[l];
      a.pyr = ctx->d_pyr[l];
    }
  a.k = a.side / a.f;
  a.Wl = ceil_div(ctx->W, a.f);
  a.Hl = ceil_div(ctx->H, a.f);
  a.img = ctx->d_img;
  a.img_pitch = ctx->pitch;

  a.lab = ctx->d_lab[ctx->cur_buf];
  a.st = ctx->st;
  a.mg = ctx->mg;
  a.ctl = ctx->ctl;
  a.ctl.cnt = ctx->ctl.cnt + (long long)CNT_N * ctx->cur;
  a.ctl.prof = ctx->profiling ? ctx->prof + (long long)PROF_N * ctx->cur : nullptr;
  a.imp_on = ctx->imp_on;
  a.imp_rule = ctx->p.importance_rule;
  a.lam_pos = ctx->lam_pos;
  a.lam_b2 = ctx->lam_b2;
  a.size_mode = ctx->p.size_mode;
  a.lo_num = ctx->p.lo_num;
  a.lo_den = ctx->p.lo_den;
  a.hi_num = ctx->p.hi_num;
  a.hi_den = ctx->p.hi_den;
  a.max_sweeps = ctx->p.max_sweeps;
  a.trec = ctx->d_trec;
  a.ntx = (a.nbx + kTileW - 1) / kTileW;
  a.nty = (a.nby + kTileH - 1) / kTileH;
  a.lam_pos_f = (float)ctx->lam_pos;
  a.lam_b2_f = (float)ctx->lam_b2;
  // single-precision decisions need blocks under 2^24 pixels and exact float block centres
  a.use_filter = ctx->p.use_filter && a.side <= 4096 && ctx->W < (1 << 22) && ctx->H < (1 << 22);
  a.verify_filter = ctx->p.verify_filter;
  a.skip_tiles = ctx->p.skip_tiles;
  return a;
}

static rapid_status ensure_label_arrays(rapid_ctx *ctx, int M) {
  if (M <= ctx->M_cap) {
    carve_label_arrays(ctx->d_label_block, label_arrays_bytes(ctx->M_cap), M, &ctx->st, &ctx->mg);
    return RAPID_OK;
  }
  cudaFree(ctx->d_label_block);
  cudaFree(ctx->d_pack);
  ctx->d_label_block = nullptr;
  ctx->d_pack = nullptr;
  ctx->M_cap = 0;
  const size_t bytes = label_arrays_bytes(M);
  if (cudaMalloc(&ctx->d_label_block, bytes) != cudaSuccess) return RAPID_ENOMEM;
  if (cudaMalloc(&ctx->d_pack, (size_t)M * sizeof(rapid_sp_stats)) != cudaSuccess) return RAPID_ENOMEM;
  carve_label_arrays(ctx->d_label_block, bytes, M, &ctx->st, &ctx->mg);
  ctx->M_cap = M;
  return RAPID_OK;
}

extern "C" rapid_status rapid_seed_grid(rapid_ctx *ctx, int32_t *M_out) {
  if (!ctx) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (!ctx->image_set) return RAPID_ESTATE;
  // level images (exact box sums, Sec. 2.2) and the extra box-sum levels for block sums
  for (int l = 0; l < ctx->nsf; l++) {
    CK(launch_pyramid(ctx->d_img, ctx->pitch, ctx->H, ctx->W, ctx->sf[l], ctx->sfW[l], ctx->sfH[l], ctx->d_pyr[l],
                      ctx->stream));
    ctx->launches++;
  }

  ctx->cur = 0;
  ctx->cur_buf = 0;
  const int s0 = ctx->st_side[0];
  ctx->nbx = ceil_div(ctx->W, s0);
  ctx->nby = ceil_div(ctx->H, s0);
  // seed grid gx x gy (same rounding as the stated formula)
  double gxd = std::sqrt((double)ctx->p.K * (double)ctx->W / (double)ctx->H);
  int gx = (int)std::floor(gxd + 0.5);
  if (gx < 1) gx = 1;
  int gy = (int)std::floor((double)ctx->p.K / (double)gx + 0.5);
  if (gy < 1) gy = 1;
  if (gx > ctx->nbx) gx = ctx->nbx;
  if (gy > ctx->nby) gy = ctx->nby;
  const int M = gx * gy;
  rapid_status rs = ensure_label_arrays(ctx, M);
  if (rs != RAPID_OK) return rs;
  ctx->M = M;
  ctx->st.M = M;
  ctx->imp_on = 0;
  ctx->lam_pos = ctx->p.lambda_pos0 * ((double)M / ((double)ctx->H * (double)ctx->W));
  ctx->lam_b2 = 2.0 * ctx->p.lambda_b;
  // counters: level and side of every stage, the rest zero; no device error pending
  Schedule sch;
  std::memset(&sch, 0, sizeof sch);
  sch.n = ctx->nstages;
  for (int i = 0; i < ctx->nstages; i++) {
    sch.level[i] = ctx->st_level[i];
    sch.side[i] = ctx->st_side[i];
  }
  CK(launch_init_counters(ctx->ctl.cnt, sch, ctx->stream));
  CK(cudaMemsetAsync(ctx->prof, 0, sizeof(long long) * PROF_N * RAPID_MAX_STAGES, ctx->stream));
  CK(cudaMemsetAsync(ctx->mg.req_count, 0, 4 * sizeof(int), ctx->stream));
  int nl = 1;
  StageArgs a = stage_args(ctx);
  CK(launch_seed(a, gx, gy, ctx->stream, &nl));
  ctx->launches += nl;
  if (M_out) *M_out = M;
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
  // fresh barrier words and sweep-change slots for the launch
  CK(cudaMemsetAsync(ctx->ctl.bar, 0, 8, ctx->stream));
  // last merge, request / found counts, sweep changes, tile counters
  CK(cudaMemsetAsync((char *)ctx->d_ctl_block + 12, 0, 116, ctx->stream));

  StageArgs a = stage_args(ctx);
  if (ctx->profiling) {
    if (!ctx->ev_ok[i]) {
      CK(cudaEventCreate(&ctx->ev[i][0]));
      CK(cudaEventCreate(&ctx->ev[i][1]));
      ctx->ev_ok[i] = 1;
    }
    CK(cudaEventRecord(ctx->ev[i][0], ctx->stream));
  }
  CK(launch_stage(a, ctx->coop_grid, ctx->coop_block, ctx->stream));
  ctx->launches++;
  if (ctx->profiling) CK(cudaEventRecord(ctx->ev[i][1], ctx->stream));
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
    CK(launch_predict(ctx->d_lab[ctx->cur_buf], ctx->nbx, ctx->nby, ctx->st, ctx->p.h_T, ctx->stream, &nl));
    ctx->imp_on = 1;
  }
  const int s = ctx->st_side[nxt];
  const int dnbx = ceil_div(ctx->W, s), dnby = ceil_div(ctx->H, s);
  CK(launch_split(ctx->d_lab[ctx->cur_buf], ctx->nbx, ctx->d_lab[ctx->cur_buf ^ 1], dnbx, dnby, ctx->stream));
  nl++;
  ctx->cur_buf ^= 1;
  ctx->cur = nxt;
  ctx->nbx = dnbx;
  ctx->nby = dnby;
  if (!ctx->p.reuse && ctx->st_level[nxt] != prev_level) {
    StageArgs a = stage_args(ctx);
    CK(launch_recompute(a, ctx->stream, &nl));
  }
  ctx->launches += nl;
  return RAPID_OK;
}

extern "C" rapid_status rapid_run(rapid_ctx *ctx) {
  if (!ctx) return RAPID_EINVAL;
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

extern "C" rapid_status rapid_get_state(rapid_ctx *ctx, int32_t *stage, int32_t *level, int32_t *block,
                                        int32_t *M) {
  if (!ctx) return RAPID_EINVAL;
  if (stage) *stage = ctx->cur;
  if (level) *level = ctx->cur >= 0 ? ctx->st_level[ctx->cur] : 0;
  if (block) *block = ctx->cur >= 0 ? ctx->st_side[ctx->cur] : 0;
  if (M) *M = ctx->cur >= 0 ? ctx->M : 0;
  return RAPID_OK;
}

extern "C" rapid_status rapid_read_labels(rapid_ctx *ctx, int32_t *dst, int64_t row_pitch_bytes,
                                          int32_t dst_is_device) {
  if (!ctx || !dst) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (ctx->cur < 0) return RAPID_ESTATE;
  if (row_pitch_bytes < 4ll * ctx->W || (row_pitch_bytes % 4) != 0) return RAPID_EINVAL;
  const int side = ctx->st_side[ctx->cur];
  const int *lab = ctx->d_lab[ctx->cur_buf];
  if (side == 1) {
    CK(cudaMemcpy2DAsync(dst, row_pitch_bytes, lab, 4ull * ctx->W, 4ull * ctx->W, ctx->H,
                         dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  } else if (dst_is_device) {
    CK(launch_upsample(lab, ctx->nbx, side, ctx->H, ctx->W, dst, row_pitch_bytes / 4, ctx->stream));
    ctx->launches++;
  } else {
    const long long n = (long long)ctx->H * ctx->W;
    if (n > ctx->full_cap) {
      cudaFree(ctx->d_full);
      ctx->d_full = nullptr;
      ctx->full_cap = 0;
      if (cudaMalloc(&ctx->d_full, n * sizeof(int)) != cudaSuccess) return RAPID_ENOMEM;
      ctx->full_cap = n;
    }
    CK(launch_upsample(lab, ctx->nbx, side, ctx->H, ctx->W, ctx->d_full, ctx->W, ctx->stream));
    ctx->launches++;
    CK(cudaMemcpy2DAsync(dst, row_pitch_bytes, ctx->d_full, 4ull * ctx->W, 4ull * ctx->W, ctx->H,
                         cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return read_device_error(ctx);
}

extern "C" rapid_status rapid_read_block_labels(rapid_ctx *ctx, int32_t *dst, int64_t capacity, int32_t *nbx_out,
                                                int32_t *nby_out) {
  if (!ctx || !dst) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (ctx->cur < 0) return RAPID_ESTATE;
  const long long n = (long long)ctx->nbx * ctx->nby;
  if (capacity < n) return RAPID_EINVAL;
  CK(cudaMemcpyAsync(dst, ctx->d_lab[ctx->cur_buf], n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (nbx_out) *nbx_out = ctx->nbx;
  if (nby_out) *nby_out = ctx->nby;
  return read_device_error(ctx);
}

extern "C" rapid_status rapid_read_stats(rapid_ctx *ctx, rapid_sp_stats *dst, int64_t capacity, int64_t *M_out) {
  if (!ctx || !dst) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  if (ctx->cur < 0) return RAPID_ESTATE;
  if (capacity < ctx->M) return RAPID_EINVAL;
  CK(launch_pack_stats(ctx->st, ctx->d_pack, ctx->stream));
  ctx->launches++;
  CK(cudaMemcpyAsync(dst, ctx->d_pack, (size_t)ctx->M * sizeof(rapid_sp_stats), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (M_out) *M_out = ctx->M;
  return read_device_error(ctx);
}

extern "C" rapid_status rapid_read_counters(rapid_ctx *ctx, rapid_counters *dst) {
  if (!ctx || !dst) return RAPID_EINVAL;
  if (ctx->sticky != RAPID_OK) return ctx->sticky;
  std::memset(dst, 0, sizeof *dst);
  CK(cudaStreamSynchronize(ctx->stream));
  rapid_status rs = read_device_error(ctx);
  if (rs != RAPID_OK) return rs;
  long long c[CNT_N * RAPID_MAX_STAGES];
  CK(cudaMemcpy(c, ctx->ctl.cnt, sizeof c, cudaMemcpyDeviceToHost));
  long long pr[PROF_N * RAPID_MAX_STAGES];
  CK(cudaMemcpy(pr, ctx->prof, sizeof pr, cudaMemcpyDeviceToHost));
  dst->num_stages = ctx->cur >= 0 ? ctx->nstages : 0;
  dst->M = ctx->cur >= 0 ? ctx->M : 0;
  dst->launches = ctx->launches;
  for (int i = 0; i < dst->num_stages; i++) {
    rapid_stage_counters &o = dst->stage[i];
    const long long *ci = c + (long long)CNT_N * i;
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
    for (int j = 0; j < PROF_N; j++) o.section_ms[j] = ctx->profiling ? (float)(pr[i * PROF_N + j] * 1e-6) : 0.0f;
    if (ctx->profiling && ctx->ev_ok[i] && i <= ctx->cur) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ctx->ev[i][0], ctx->ev[i][1]) == cudaSuccess) o.kernel_ms = ms;
    }
  }
  return RAPID_OK;
}

extern "C" rapid_status rapid_set_profiling(rapid_ctx *ctx, int32_t on) {
  if (!ctx) return RAPID_EINVAL;
  ctx->profiling = on ? 1 : 0;
  return RAPID_OK;
}

extern "C" rapid_status rapid_simple_table(uint8_t *out256) {
  if (!out256) return RAPID_EINVAL;
  unsigned char *d = nullptr;
  if (cudaMalloc(&d, 256) != cudaSuccess) return RAPID_ENOMEM;
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
