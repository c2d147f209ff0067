// rapid_static.cu — rapid_run_static: the whole refinement of one small image with every
// byte of working memory taken from one fixed device array, for callers that must not
// allocate GPU memory.
//
// Who needs it: services whose device memory is fully reserved up front by another
// allocator (a framework memory pool, a multi-tenant inference server), so a library
// cudaMalloc would fail or steal from their budget; and latency-critical pipelines that
// forbid cudaMalloc / cudaFree because those calls can synchronise the device.  Such
// callers pass their input image and output buffers (device memory they already own);
// this entry point never calls cudaMalloc, cudaFree or any allocating library routine.
//
// The working memory is g_scratch below: a file-scope __device__ array of
// kStaticScratchBytes (16 MiB).  Every GPU that loads this library holds that array until
// the process exits.  All calls on one device share it, and it keeps the last call's
// contents, so each call re-initialises everything that must start at zero; two calls
// whose GPU work overlaps in time (different streams or host threads) race on it and
// must be serialised by the caller.
#include <cmath>
#include <cstring>
#include <mutex>

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
cudaError_t launch_upsample(const int *lab, int nbx, int side, int H, int W, int label0, int *dst,
                            long long pitch_elems, cudaStream_t s);
cudaError_t launch_pack_stats(const DevStats &st, int label0, int M, rapid_sp_stats *out, cudaStream_t s);
cudaError_t launch_init_counters(long long *cnt, const Schedule &sch, int n, cudaStream_t s);
}  // namespace rapid

using namespace rapid;

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;
constexpr int kMaxLevelsStatic = 8;

__device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices];    // device address of g_scratch per device
unsigned long long g_scratch_ctx[kMaxDevices];  // id of the context it was looked up in

// Unique id of the calling thread's current context (ids are never reused in a process),
// through the driver entry points the runtime hands out; 0 when unavailable.
unsigned long long current_context_id() {
  typedef int (*GetCurrent)(void **);
  typedef int (*GetId)(void *, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = (GetCurrent)f1;
      get_id = (GetId)f2;
    }
    looked_up = true;
  }
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of g_scratch on the current device, looked up at the first call on each
// device (with that device current) and again whenever the device's context is a new one
// (after cudaDeviceReset the module is loaded again and the array moves).  In host code the
// name g_scratch is only a host-side stand-in, never a device address.
rapid_status scratch_on_current_device(unsigned char **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RAPID_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  const unsigned long long id = current_context_id();  // 0 before the runtime made a context current
  if (!g_scratch_addr[dev] || id == 0 || id != g_scratch_ctx[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) return RAPID_ECUDA;
    g_scratch_addr[dev] = (unsigned char *)p;
    g_scratch_ctx[dev] = current_context_id();
  }
  *out = g_scratch_addr[dev];
  return RAPID_OK;
}

// Bump allocator over the fixed array (256-byte aligned pieces).
struct Carve {
  unsigned char *base;
  size_t used, cap;
  void *take(size_t n) {
    n = (n + 255) / 256 * 256;
    if (n > cap - used) return nullptr;
    void *r = base + used;
    used += n;
    return r;
  }
};

bool pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
int cdiv(int a, int b) { return (a + b - 1) / b; }

}  // namespace

extern "C" rapid_status rapid_run_static(const rapid_params *p, const uint8_t *rgb_dev, int32_t H, int32_t W,
                                         int64_t rgb_pitch_bytes, int32_t *labels_dev, int64_t labels_pitch_bytes,
                                         rapid_sp_stats *stats_dev, int64_t stats_capacity, int32_t *M_out,
                                         void *cuda_stream) {
  if (!p || !rgb_dev || !labels_dev || !stats_dev) return RAPID_EINVAL;
  if (H < 1 || W < 1 || rgb_pitch_bytes < 3ll * W || labels_pitch_bytes < 4ll * W || labels_pitch_bytes % 4)
    return RAPID_EINVAL;
  if (p->num_levels < 1 || p->num_levels > kMaxLevelsStatic) return RAPID_EINVAL;
  if (p->num_levels > 1 && (!pow2(p->ratio_C) || p->ratio_C < 2)) return RAPID_EINVAL;
  if (!pow2(p->init_block) || !pow2(p->final_grain) || p->init_block > (1 << 20)) return RAPID_EINVAL;
  if (p->K < 1 || p->size_mode < 0 || p->size_mode > 2 || p->max_sweeps < 1) return RAPID_EINVAL;
  if (p->lo_den <= 0 || p->hi_den <= 0 || p->lo_num < 0 || p->hi_num < 0) return RAPID_EINVAL;
  if (!std::isfinite(p->lambda_pos0) || !std::isfinite(p->lambda_b)) return RAPID_EINVAL;
  if ((p->predict | p->reuse | p->importance_rule | p->schedule | p->use_filter | p->skip_tiles | p->verify_filter) &
      ~1)
    return RAPID_EINVAL;
  if (p->spin_limit_ns < 0 || p->h_T < 0 || p->h_T > (1ll << 40)) return RAPID_EINVAL;
  if ((long long)H * W > RAPID_STATIC_MAX_PIXELS) return RAPID_ERANGE;
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  // Levels and stages (same schedule as rapid_run).
  const int L = p->num_levels;
  int f[kMaxLevelsStatic + 1];
  for (int l = 1; l <= L; l++) {
    long long ff = 1;
    for (int i = 0; i < L - l; i++) ff *= p->ratio_C;
    if (ff > (1 << 20)) return RAPID_EINVAL;
    f[l] = (int)ff;
  }
  int nst = 0, lev[RAPID_MAX_STAGES], side[RAPID_MAX_STAGES];
  int s = p->init_block < f[1] ? f[1] : p->init_block;
  while (s >= 1 && s >= p->final_grain) {
    int lv = 0;
    for (int l = 1; l <= L; l++)
      if (f[l] <= s) {
        lv = l;
        break;
      }
    if (lv == 0) break;
    if (nst >= RAPID_MAX_STAGES) return RAPID_ERANGE;
    lev[nst] = lv;
    side[nst] = s;
    nst++;
    s /= 2;
  }
  if (nst == 0) {
    lev[0] = 1;
    side[0] = p->init_block < f[1] ? f[1] : p->init_block;
    nst = 1;
  }
  const int nbx0 = cdiv(W, side[0]), nby0 = cdiv(H, side[0]);
  int gx = (int)std::floor(std::sqrt((double)p->K * (double)W / (double)H) + 0.5);
  if (gx < 1) gx = 1;
  int gy = (int)std::floor((double)p->K / (double)gx + 0.5);
  if (gy < 1) gy = 1;
  if (gx > nbx0) gx = nbx0;
  if (gy > nby0) gy = nby0;
  const int M = gx * gy;
  if (M > RAPID_STATIC_MAX_LABELS) return RAPID_ERANGE;
  if (stats_capacity < M) return RAPID_EINVAL;

  // Carve the fixed array.
  unsigned char *base = nullptr;
  rapid_status rs = scratch_on_current_device(&base);
  if (rs != RAPID_OK) return rs;
  Carve cv{base, 0, kStaticScratchBytes};
  const CtlLayout cl = ctl_layout(1);
  unsigned char *ctl = (unsigned char *)cv.take(cl.total);
  int sf[kMaxSumLevels];
  const int nsf = sum_factors(f, L, side[0], sf);
  int4 *pyr[kMaxSumLevels] = {nullptr};
  for (int l = 0; l < nsf; l++) pyr[l] = (int4 *)cv.take((size_t)cdiv(W, sf[l]) * cdiv(H, sf[l]) * sizeof(int4));
  const long long cap = (long long)cdiv(W, side[nst - 1]) * cdiv(H, side[nst - 1]);
  int *lab[2] = {(int *)cv.take(cap * sizeof(int)), (int *)cv.take(cap * sizeof(int))};
  const TileShape ts = kShapes[0];  // one tile shape for every stage here
  const int ntx_max = (cdiv(W, side[nst - 1]) + ts.w - 1) / ts.w;
  const int nty_max = (cdiv(H, side[nst - 1]) + ts.h - 1) / ts.h;
  unsigned *qbits = p->schedule == 1
                        ? (unsigned *)cv.take((size_t)ntx_max * nty_max * 9 * kQueueWords * sizeof(unsigned))
                        : nullptr;
  const int wl_cap = ((cdiv(W, side[nst - 1]) + 2) / 3) * ((cdiv(H, side[nst - 1]) + 2) / 3);
  int *wl = p->schedule == 1 ? (int *)cv.take(((size_t)wl_cap * 9 + 16) * sizeof(int)) : nullptr;
  // sweep-schedule bitmaps, sized for the largest stage
  long long words_max = 0;
  for (int i = 0; i < nst; i++) {
    long long w = 0;
    for (int c = 0; c < 9; c++) w += class_words(cdiv(W, side[i]), cdiv(H, side[i]), c);
    if (w > words_max) words_max = w;
  }
  unsigned *cbits = (unsigned *)cv.take((size_t)words_max * sizeof(unsigned));
  unsigned *rbits = (unsigned *)cv.take((size_t)words_max * sizeof(unsigned));
  ImageDesc *d_desc = (ImageDesc *)cv.take((size_t)nst * sizeof(ImageDesc));
  DevStats st;
  DevMerge mg;
  std::memset(&st, 0, sizeof st);
  std::memset(&mg, 0, sizeof mg);
  const size_t lbytes = label_arrays_bytes(M);
  void *lblock = cv.take(lbytes);
  bool ok = ctl && lab[0] && lab[1] && cbits && rbits && d_desc && lblock && ((qbits && wl) || p->schedule != 1);
  for (int l = 0; l < nsf; l++) ok = ok && pyr[l];
  if (!ok) return RAPID_ERANGE;  // this image and parameter set need more than the fixed array
  carve_label_arrays(lblock, lbytes, M, &st, &mg);
  DevCtl c;
  c.bar = (unsigned *)(ctl + cl.bar);
  c.err = (int *)(ctl + 8);
  mg.req_count = (int *)(ctl + 16);
  mg.found_count = (int *)(ctl + 24);
  mg.acc_count = (int *)(ctl + 32);
  c.last_merge = (int *)(ctl + cl.last_merge);
  c.changes = (unsigned long long *)(ctl + cl.changes);
  c.cnt = (long long *)(ctl + cl.cnt);
  c.prof = nullptr;
  c.spin_ns = p->spin_limit_ns;

  // One image descriptor per stage (the stage kernel handles batches; this is a batch of one).
  const double lam_pos = p->lambda_pos0 * ((double)M / ((double)H * (double)W));
  ImageDesc desc[RAPID_MAX_STAGES];
  std::memset(desc, 0, sizeof desc);
  int stage_f[RAPID_MAX_STAGES];
  for (int i = 0; i < nst; i++) {
    ImageDesc &d = desc[i];
    int fi = 1, li = -1;
    for (int l = 0; l < nsf; l++)
      if (sf[l] <= side[i]) {
        fi = sf[l];
        li = l;
      }
    stage_f[i] = fi;
    d.H = H;
    d.W = W;
    d.nbx = cdiv(W, side[i]);
    d.nby = cdiv(H, side[i]);
    d.ntx = (d.nbx + ts.w - 1) / ts.w;
    d.nty = (d.nby + ts.h - 1) / ts.h;
    d.Wl = cdiv(W, fi);
    d.Hl = cdiv(H, fi);
    d.M = M;
    d.use_filter = p->use_filter && side[i] <= 4096 && W < (1 << 22) && H < (1 << 22);
    d.img = rgb_dev;
    d.img_pitch = rgb_pitch_bytes;
    d.pyr = li >= 0 ? pyr[li] : nullptr;
    d.lab = lab[i & 1];
    d.lam_pos = lam_pos;
    d.lam_pos_f = (float)lam_pos;
    int w = 0;
    for (int c = 0; c < 9; c++) {
      d.cw0[c] = w;
      w += (int)class_words(d.nbx, d.nby, c);
    }
  }

  // Cooperative grid size for the stage kernel (no allocation involved).
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_kernel_ptr(false, p->schedule == 1, 0), stage_block_threads(0), 0) !=
          cudaSuccess ||
      per_sm < 1)
    return RAPID_ECUDA;

#define CKS(call)                                   \
  do {                                              \
    if ((call) != cudaSuccess) return RAPID_ECUDA; \
  } while (0)

  // Start from a clean control block: barrier, error word, request counts, counters.
  CKS(cudaMemsetAsync(ctl, 0, cl.total, stream));
  CKS(cudaMemcpyAsync(d_desc, desc, (size_t)nst * sizeof(ImageDesc), cudaMemcpyHostToDevice, stream));
  for (int l = 0; l < nsf; l++)  // the finest level from the image, each coarser one from the last
    if (l == 0)
      CKS(launch_pyramid(rgb_dev, rgb_pitch_bytes, H, W, sf[l], cdiv(W, sf[l]), cdiv(H, sf[l]), pyr[l], stream));
    else
      CKS(launch_pyramid_merge(pyr[l - 1], cdiv(W, sf[l - 1]), cdiv(H, sf[l - 1]), sf[l] / sf[l - 1], cdiv(W, sf[l]),
                               cdiv(H, sf[l]), pyr[l], stream));
  Schedule sch;
  std::memset(&sch, 0, sizeof sch);
  sch.n = nst;
  for (int i = 0; i < nst; i++) {
    sch.level[i] = lev[i];
    sch.side[i] = side[i];
  }
  CKS(launch_init_counters(c.cnt, sch, 1, stream));

  StageArgs a;
  std::memset(&a, 0, sizeof a);
  a.nimg = 1;
  a.st = st;
  a.mg = mg;
  a.lam_b2 = 2.0 * p->lambda_b;
  a.lam_b2_f = (float)a.lam_b2;
  a.imp_rule = p->importance_rule;
  a.size_mode = p->size_mode;
  a.lo_num = p->lo_num;
  a.lo_den = p->lo_den;
  a.hi_num = p->hi_num;
  a.hi_den = p->hi_den;
  a.max_sweeps = p->max_sweeps;
  a.frontier = p->schedule == 1;
  a.qbits = qbits;
  a.wl = wl;
  a.wl_count = wl ? wl + (size_t)wl_cap * 9 : nullptr;
  a.wl_cap = wl_cap;
  a.verify_filter = p->verify_filter;
  a.skip_tiles = p->skip_tiles;
  a.cbits = cbits;
  a.rbits = rbits;
  int launches = 0;
  auto set_stage = [&](int i) {
    a.side = side[i];
    a.level = lev[i];
    a.f = stage_f[i];
    a.k = a.side / a.f;
    a.imgs = d_desc + i;
    a.img0 = desc[i];
    a.ntiles = desc[i].ntx * desc[i].nty;
    a.ctl = c;
    a.ctl.cnt = c.cnt + (long long)CNT_N * i;
    for (int cl9 = 0; cl9 < 9; cl9++) a.cwb[cl9] = desc[i].cw0[cl9];
    a.cwb[9] = desc[i].cw0[8] + (int)class_words(desc[i].nbx, desc[i].nby, 8);
  };
  set_stage(0);
  const int gxa[1] = {gx}, gya[1] = {gy};
  CKS(launch_seed(a, &desc[0], gxa, gya, 1, stream, &launches));
  for (int i = 0; i < nst; i++) {
    if (i > 0) {
      if (p->predict && lev[i] >= 2 && lev[i - 1] < 2) {
        CKS(launch_predict(&desc[i - 1], 1, st, p->h_T, stream, &launches));
        a.imp_on = 1;
      }
      CKS(launch_split(desc[i - 1].lab, desc[i - 1].nbx, desc[i].lab, desc[i].nbx, desc[i].nby, stream));
      set_stage(i);
      if (!p->reuse && lev[i] != lev[i - 1]) CKS(launch_recompute(a, &desc[i], 1, stream, &launches));
    }
    CKS(cudaMemsetAsync(ctl + 16, 0, cl.reset_end - 16, stream));  // barrier, merge stamps, counts, changes
    CKS(launch_stage(a, nsm * per_sm, stage_block_threads(0), stream, 0));
  }
  // Outputs into the caller's buffers.
  const ImageDesc &dl = desc[nst - 1];
  if (side[nst - 1] == 1)
    CKS(cudaMemcpy2DAsync(labels_dev, labels_pitch_bytes, dl.lab, 4ull * W, 4ull * W, H, cudaMemcpyDeviceToDevice,
                          stream));
  else
    CKS(launch_upsample(dl.lab, dl.nbx, side[nst - 1], H, W, 0, labels_dev, labels_pitch_bytes / 4, stream));
  CKS(launch_pack_stats(st, 0, M, stats_dev, stream));
  int err = 0;
  CKS(cudaMemcpyAsync(&err, c.err, sizeof err, cudaMemcpyDeviceToHost, stream));
  CKS(cudaStreamSynchronize(stream));
#undef CKS
  if (M_out) *M_out = M;
  return err ? RAPID_ETIMEOUT : RAPID_OK;
}
