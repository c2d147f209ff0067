// stage_impl.cuh — one stage of the refinement (Sec. 2.1, Algorithm RAPID's queue loop) as
// a single cooperative launch: sweeps of 9 phases until a sweep changes nothing.
//
// Compiled once per evaluation-tile shape: a translation unit defines RAPID_TILE_W,
// RAPID_TILE_H and RAPID_SHAPE_NS and includes this file; everything lands in the
// namespace rapid::RAPID_SHAPE_NS, and the unit exports launch_stage_<NS> and
// stage_kernel_ptr_<NS> for the dispatcher (k_stage.cu).
//
// Phase (py, px) evaluates the blocks with by % 3 == py and bx % 3 == px.  Two such
// blocks are at least 3 apart, so their 3x3 windows are disjoint: every block of a phase
// decides from labels no other block of the phase writes, their boundary pairs are
// disjoint, and each topology test stays valid when the others move.  Decisions use a
// snapshot of the superpixel means (and sizes, for the size rule) taken when the phase
// starts; moves update the label map in place and add their exact int64 sums into S
// atomically.  Merge requests of the phase (size bound hit, Sec. 3.1) are then resolved
// against the post-move S while the snapshot is refreshed.
//
// Work layout: one persistent CTA of 1024 (or 512) threads per SM.  Under the sweep
// schedule a phase walks a bitmap of the class's blocks that may be eligible, split
// evenly over the warps of the grid (eval_sweep.cuh); under the queue schedule a phase pops
// the queued blocks of its class, by tiles of kTileW x kTileH blocks (32 x 16, 32 x 8 or
// 64 x 16 by unit) or from a worklist (eval_tile.cuh).
//
// Decisions: the energy difference of each candidate label k against the block's label a
// is first computed in single precision in the well-conditioned form
//   dE_k = sum_ch (c_k - c_a)(w (c_k + c_a) - 2 S_ch)
//          + lambda_pos w sum_d (mu_k - mu_a)((mu_k - pbar_d) + (mu_a - pbar_d))
//          + 2 lambda_b (B_k - B_a)          (pbar = block centre = P / w)
// (algebraically e(k) - e(a) of the binary64 block energy) together with a rigorous bound
// on its rounding error, widened by the rounding error of the binary64 evaluation itself.
// When the resulting intervals fix the sign of the best candidate and its strict lead over
// the others, that is exactly the binary64 decision; otherwise the block is decided in
// binary64 with the oracle's operation order.  Results are bit-identical to an
// all-binary64 evaluation.
#include <climits>

#include "rapid_dev.cuh"

#if !defined(RAPID_TILE_W) || !defined(RAPID_TILE_H) || !defined(RAPID_SHAPE_NS)
#error "define RAPID_TILE_W, RAPID_TILE_H and RAPID_SHAPE_NS before including stage_impl.cuh"
#endif
#define RAPID_CAT2(a, b) a##b
#define RAPID_CAT(a, b) RAPID_CAT2(a, b)

namespace rapid {
namespace RAPID_SHAPE_NS {

// Evaluation tiles of this unit: kTileW x kTileH blocks, one warp each.
constexpr int kTileW = RAPID_TILE_W, kTileH = RAPID_TILE_H;
// the sweep schedule's walk of this build: the CTA walk (1) or the warp walk (0)
#ifndef RAPID_SWEEP_CTA
#error "define RAPID_SWEEP_CTA (0 or 1) before including stage_impl.cuh"
#endif
constexpr bool kSweepCta = RAPID_SWEEP_CTA != 0;
// blocks of one phase class in a tile, and 32-bit words of one bit each
constexpr int kPhaseMax = ((kTileW + 2) / 3) * ((kTileH + 2) / 3);
constexpr int kReqWords = (kPhaseMax + 31) / 32;
static_assert(kReqWords <= kQueueWords, "the frontier queue holds a tile's class lattice");

#ifndef RAPID_THREADS
#define RAPID_THREADS 1024
#endif
static constexpr int kThreads = RAPID_THREADS;
static_assert((kThreads & (kThreads - 1)) == 0, "block reductions assume a power-of-two CTA size");

static constexpr int kMergeSet = 64;

struct Local {
  int elig, eval, moves, req, fallback, mismatch;  // per thread and phase: fit in 32 bits

};

struct BlockIn {
  BlockSums bs;
  int x0, y0;  // block origin (full-res px)
  int lbl;
  int nb[4];   // N, W, E, S neighbour labels (-1 outside the grid)
};

// ---------------------------------------------------------------- binary64 decision
// Exactly the oracle's evaluation: e(a), then e(k) - e(a) per distinct neighbour label,
// least value (ties to the smaller label).  Returns the best label or -1 (no decrease).
__device__ __noinline__ int decide_f64(const StageArgs &a, const BlockIn &in, double lam_pos) {
  const DevStats &s = a.st;
  const BlockSums &bs = in.bs;
  const double w = __ll2double_rn(bs.w);
  const double r2 = __ll2double_rn(2 * bs.r), g2 = __ll2double_rn(2 * bs.g), b2 = __ll2double_rn(2 * bs.b);
  const double x2 = __ll2double_rn(2 * bs.x), y2 = __ll2double_rn(2 * bs.y);
  const int len[4] = {bs.bw, bs.bh, bs.bh, bs.bw};
  const int lbl = in.lbl;
  long long Ba = 0;
  for (int j = 0; j < 4; j++)
    if (in.nb[j] >= 0 && in.nb[j] != lbl) Ba += len[j];
  const double ea = blk_energy(w, r2, g2, b2, x2, y2, s.mR[lbl], s.mG[lbl], s.mB[lbl], s.mX[lbl], s.mY[lbl],
                               __ll2double_rn(Ba), lam_pos, a.lam_b2);
  int bestk = -1;
  double best = 0.0;
  for (int j = 0; j < 4; j++) {
    const int k = in.nb[j];
    if (k < 0 || k == lbl) continue;
    bool dup = false;
    for (int i = 0; i < j; i++) dup |= (in.nb[i] == k);
    if (dup) continue;
    long long Bk = 0;
    for (int i = 0; i < 4; i++)
      if (in.nb[i] >= 0 && in.nb[i] != k) Bk += len[i];
    const double ek = blk_energy(w, r2, g2, b2, x2, y2, s.mR[k], s.mG[k], s.mB[k], s.mX[k], s.mY[k],
                                 __ll2double_rn(Bk), lam_pos, a.lam_b2);
    const double dE = __dsub_rn(ek, ea);
    if (bestk < 0 || dE < best || (dE == best && k < bestk)) {
      best = dE;
      bestk = k;
    }
  }
  return (bestk >= 0 && best < 0.0) ? bestk : -1;
}

// ---------------------------------------------------------------- single-precision filter
// Running error analysis: each quantity carries a radius r with |computed - exact| <= r,
// "exact" being real arithmetic on the binary64 snapshot means.  kU = 2^-24 is the unit
// roundoff of float; kSplit = 2^-46 bounds |c - (hi + lo)| / |hi| for the hi/lo split of a
// binary64 mean (|c - hi - lo| <= 2^-48 |c|).  The radius arithmetic itself is evaluated in
// float; its own relative rounding (< 40 operations of 2^-24) is covered by the final 1%
// widening.
static constexpr float kU = 5.9604645e-08f;
static constexpr float kSplit = 1.4210855e-14f;

struct Fr {
  float v, r;
};

__device__ __forceinline__ Fr diff_hl(float hk, float lk, float ha, float la) {
  const float d1 = hk - ha, d2 = lk - la, d = d1 + d2;
  return {d, kU * (fabsf(d1) + fabsf(d2) + fabsf(d)) + kSplit * (fabsf(hk) + fabsf(ha))};
}

// (c_k - c_a)(w (c_k + c_a) - 2 S) for one colour channel.  s2f = float(2 S), rs2 = its error.
__device__ __forceinline__ Fr colour_term(float hk, float lk, float ha, float la, float wf, float s2f, float rs2) {
  const Fr d = diff_hl(hk, lk, ha, la);
  const float s1 = hk + ha, s2 = lk + la, sm = s1 + s2;
  const float rs = kU * (fabsf(s1) + fabsf(s2) + fabsf(sm)) + kSplit * (fabsf(hk) + fabsf(ha));
  const float ws = wf * sm;
  const float rws = wf * rs + kU * fabsf(ws);
  const float m = ws - s2f;
  const float rm = rws + rs2 + kU * fabsf(m);
  const float t = d.v * m;
  return {t, fabsf(d.v) * rm + fabsf(m) * d.r + d.r * rm + kU * fabsf(t)};
}

// w (mu_k - mu_a)((mu_k - pb) + (mu_a - pb)) for one position dimension; pb exact in float.
__device__ __forceinline__ Fr position_term(float hk, float lk, float ha, float la, float pb, float wf) {
  const Fr d = diff_hl(hk, lk, ha, la);
  const float e1 = hk - pb, e2 = ha - pb, e12 = e1 + e2, l12 = lk + la, e = e12 + l12;
  const float re =
      kU * (fabsf(e1) + fabsf(e2) + fabsf(e12) + fabsf(l12) + fabsf(e)) + kSplit * (fabsf(hk) + fabsf(ha));
  const float t = d.v * e;
  const float rt = fabsf(d.v) * re + fabsf(e) * d.r + d.r * re + kU * fabsf(t);
  const float tw = wf * t;
  return {tw, wf * rt + kU * fabsf(tw)};
}

__device__ __forceinline__ Fr add_fr(Fr x, Fr y) {
  const float v = x.v + y.v;
  return {v, x.r + y.r + kU * fabsf(v)};
}

// Bound on |binary64 e(j) - exact e(j)|: at most 7 u64 times the sum of the absolute terms
// of the energy (u64 = 2^-53; each term passes through at most 7 roundings), taken as
// 16 u64 and widened 1% for the float evaluation of the sum.
__device__ __forceinline__ float eps64(const float4 &h, const float2 &hy, float wf, float r2f, float g2f,
                                       float b2f, float x2f, float y2f, float lamf, float lamb2f, float Bj) {
  const float col = (wf * h.x * h.x + r2f * h.x) + (wf * h.y * h.y + g2f * h.y) + (wf * h.z * h.z + b2f * h.z);
  const float pos = (wf * h.w * h.w + x2f * h.w) + (wf * hy.x * hy.x + y2f * hy.x);
  const float T = col + lamf * pos + lamb2f * Bj;
  return T * (1.7763568e-15f * 1.01f);
}

#include "eval_tile.cuh"
#include "eval_sweep.cuh"

// The sweep schedule walks the per-class bitmaps (eval_sweep.cuh); the queue schedule pops
// its queue by tiles or worklists (eval_tile.cuh).
template <int kSched>
__device__ __forceinline__ bool sweep_schedule(const StageArgs &a) {
  return kSched == kSchedSweeps || (kSched == kSchedRuntime && !a.frontier);
}

// Refresh the snapshot means and counts of the labels the phase's moves changed (S itself
// already holds the moves) and stamp them (2g).
__device__ void commit_phase(const StageArgs &a, int g) {
  const DevStats &s = a.st;
  // label k goes to CTA k % grid: the divisions of set_means spread over every SM
  for (int k = blockIdx.x + gridDim.x * threadIdx.x; k < s.M; k += gridDim.x * blockDim.x) {
    if (!s.dirty[k]) continue;
    s.dirty[k] = 0;
    set_means(s, k);
    s.chg[k] = 2 * g;
  }
}

// Merge targets (Eqs. eqa:merge, condtion), one CTA per requested label: over the labels
// 4-adjacent to it (gathered by scanning its bounding box, which always contains it), the
// least merge cost among those that stay within u * InitSize; ties to the smaller id.  A
// search that found no target is remembered with its neighbour labels; while neither the
// label nor any of them has changed since, the answer is the same and the scan is skipped.
// Image of global label v: the last image whose first label is <= v.
__device__ __forceinline__ int image_of_label(const int *label0, int nimg, int v) {
  int lo = 0, hi = nimg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (label0[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <bool kBatch>
__device__ __forceinline__ void merge_targets(const StageArgs &a, const ImageDesc *imgs, const int *label0, int rq,
                                              int g) {
  __shared__ double sw[kThreads];
  __shared__ int sn[kThreads];
  __shared__ int nset[kMergeSet];
  __shared__ int s_over, s_hit;
  __shared__ int s_ext[4];
  __shared__ double s_am[5];
  const DevStats &s = a.st;
  const DevMerge &mg = a.mg;
  for (int j = blockIdx.x; j < rq; j += gridDim.x) {
    const int al = mg.req_list[j];
    const int ii = kBatch ? image_of_label(label0, a.nimg, al) : 0;
    const ImageDesc &im = kBatch ? imgs[ii] : a.img0;
    long long *cnt = a.ctl.cnt + (long long)ii * kCntStride;
    // A cached failure still holds when the neighbour set is provably the same (no move of
    // or next to a block of al, no merge in its image since) and every cached neighbour
    // still fails the size condition with the current counts.
    if (threadIdx.x < 32) {
      const int cs = mg.cache_stamp[al], cn = mg.cache_n[al];
      const bool can =
          cs > 0 && cn >= 0 && s.adj[al] <= cs && ld_volatile_i32(a.ctl.last_merge + ii) <= cs;
      bool fits = false;
      if (can && (int)threadIdx.x < cn) {
        const int n = mg.cache_nb[(long long)al * kCacheLabels + threadIdx.x];
        fits = (long long)a.hi_den * (s.N[n] + s.N[al]) <= (long long)a.hi_num * s.init[n];
      }
      fits = __any_sync(0xffffffffu, fits);
      if (threadIdx.x == 0) {
        s_hit = can && !fits;
        atomic_add_i64(&cnt[s_hit ? CNT_CACHE_HITS : CNT_SEARCHES], 1);
        s_over = 0;
        s_ext[0] = s_ext[1] = INT_MAX;
        s_ext[2] = s_ext[3] = -1;
      }
    }
    if (threadIdx.x < kMergeSet) nset[threadIdx.x] = -1;
    if (threadIdx.x == 32) {  // the requesting label's means, shared by every candidate's cost
      s_am[0] = mean_of(s.R, s.N, al);
      s_am[1] = mean_of(s.G, s.N, al);
      s_am[2] = mean_of(s.B, s.N, al);
      s_am[3] = mean_of(s.X, s.N, al);
      s_am[4] = mean_of(s.Y, s.N, al);
    }
    __syncthreads();
    if (s_hit) {
      if (threadIdx.x == 0) mg.target[al] = -1;  // no target: the request is finished here
      __syncthreads();
      continue;
    }
    // gather the distinct neighbour labels of al, and its exact extent (which replaces the
    // conservative bounding box: later moves only widen it again)
    const int4 bb = s.bbox[al];
    const int bx0 = bb.x / a.side, bx1 = bb.z / a.side, by0 = bb.y / a.side, by1 = bb.w / a.side;
    const int bw = bx1 - bx0 + 1;
    const long long total = (long long)bw * (by1 - by0 + 1);
    const int *lab = im.lab;
    const int nbx = im.nbx, nby = im.nby;
    int mnx = INT_MAX, mny = INT_MAX, mxx = -1, mxy = -1;
    // kScan boxes per thread at a time: their labels in one round trip, then the
    // neighbours of those labelled al in another
    constexpr int kScan = 4;
    for (long long t0 = threadIdx.x; t0 < total; t0 += (long long)kScan * blockDim.x) {
      int cx[kScan], cy[kScan];
      bool hit[kScan];
#pragma unroll
      for (int u = 0; u < kScan; u++) {
        const long long t = t0 + (long long)u * blockDim.x;
        hit[u] = false;
        cx[u] = cy[u] = 0;
        if (t < total) {
          cx[u] = bx0 + (int)(t % bw);
          cy[u] = by0 + (int)(t / bw);
          hit[u] = lab[(long long)cy[u] * nbx + cx[u]] == al;
        }
      }
      int q[kScan][4];
#pragma unroll
      for (int u = 0; u < kScan; u++) {
        q[u][0] = q[u][1] = q[u][2] = q[u][3] = -1;
        if (!hit[u]) continue;
        const long long idx = (long long)cy[u] * nbx + cx[u];
        mnx = min(mnx, cx[u]);
        mxx = max(mxx, cx[u]);
        mny = min(mny, cy[u]);
        mxy = max(mxy, cy[u]);
        q[u][0] = cy[u] > 0 ? lab[idx - nbx] : -1;
        q[u][1] = cx[u] > 0 ? lab[idx - 1] : -1;
        q[u][2] = cx[u] + 1 < nbx ? lab[idx + 1] : -1;
        q[u][3] = cy[u] + 1 < nby ? lab[idx + nbx] : -1;
      }
#pragma unroll
      for (int u = 0; u < kScan; u++)
        for (int i = 0; i < 4; i++)
          if (q[u][i] >= 0 && q[u][i] != al) set_insert(nset, kMergeSet, q[u][i], &s_over);
    }
    if (mxx >= 0) {
      atomicMin(&s_ext[0], mnx);
      atomicMin(&s_ext[1], mny);
      atomicMax(&s_ext[2], mxx);
      atomicMax(&s_ext[3], mxy);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_ext[2] >= 0) {
      s.bbox[al] = make_int4(s_ext[0] * a.side, s_ext[1] * a.side, min((s_ext[2] + 1) * a.side, im.W) - 1,
                             min((s_ext[3] + 1) * a.side, im.H) - 1);
    }
    double best = 0.0;
    int bestn = INT_MAX;
    if (!s_over) {
      for (int i = threadIdx.x; i < kMergeSet; i += blockDim.x) {
        const int n = nset[i];
        if (n < 0) continue;
        if ((long long)a.hi_den * (s.N[n] + s.N[al]) > (long long)a.hi_num * s.init[n]) continue;
        const double wv = ward_cost(s, al, s_am, n, im.lam_pos);
        if (bestn == INT_MAX || wv < best || (wv == best && n < bestn)) {
          best = wv;
          bestn = n;
        }
      }
    } else {  // more neighbours than the set holds: evaluate every adjacency directly
      for (long long t = threadIdx.x; t < total; t += blockDim.x) {
        const int cx = bx0 + (int)(t % bw), cy = by0 + (int)(t / bw);
        const long long idx = (long long)cy * nbx + cx;
        if (lab[idx] != al) continue;
        const int q[4] = {cy > 0 ? lab[idx - nbx] : -1, cx > 0 ? lab[idx - 1] : -1,
                          cx + 1 < nbx ? lab[idx + 1] : -1, cy + 1 < nby ? lab[idx + nbx] : -1};
        for (int i = 0; i < 4; i++) {
          const int n = q[i];
          if (n < 0 || n == al) continue;
          if ((long long)a.hi_den * (s.N[n] + s.N[al]) > (long long)a.hi_num * s.init[n]) continue;
          const double wv = ward_cost(s, al, s_am, n, im.lam_pos);
          if (bestn == INT_MAX || wv < best || (wv == best && n < bestn)) {
            best = wv;
            bestn = n;
          }
        }
      }
    }
    sw[threadIdx.x] = best;
    sn[threadIdx.x] = bestn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) {
        const double w2 = sw[threadIdx.x + o];
        const int n2 = sn[threadIdx.x + o];
        const int n1 = sn[threadIdx.x];
        if (n2 != INT_MAX && (n1 == INT_MAX || w2 < sw[threadIdx.x] || (w2 == sw[threadIdx.x] && n2 < n1))) {
          sw[threadIdx.x] = w2;
          sn[threadIdx.x] = n2;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int tgt = sn[0] == INT_MAX ? -1 : sn[0];
      mg.target[al] = tgt;
      if (tgt >= 0) mg.found[atomicAdd(mg.found_count + (g & 1), 1)] = al;  // to the acceptance walk
      if (tgt < 0) {  // remember the failure with its neighbour set
        int n = 0;
        while (!s_over && n < kMergeSet && nset[n] >= 0) n++;
        if (!s_over && n <= kCacheLabels) {
          for (int i = 0; i < n; i++) mg.cache_nb[(long long)al * kCacheLabels + i] = nset[i];
          mg.cache_n[al] = n;
          mg.cache_stamp[al] = 2 * g;
        } else {
          mg.cache_n[al] = -1;
        }
      }
    }
    __syncthreads();
  }
}

// Acceptance of the requests whose search found a target (Sec. 3.1): in ascending order of
// their first requesting block, skipping those whose source or target already merged in
// this phase.  With up to kAcceptSmem such requests every CTA runs the same (cheap) walk in
// shared memory, so each knows the accepted list without another grid barrier; above that
// CTA 0 walks in global memory and the grid waits once more.  CTA b then applies merges
// b, b + grid, ...: S_n += S_a, S_a = 0, stamps, bounding box, and relabels a -> n over a's
// bounding box.  No two accepted merges share a label, so they apply independently.
static constexpr int kAcceptSmem = 512;

// Walk of up to kAcceptSmem found requests in shared memory; returns the accepted count.
__device__ int merge_walk_small(const StageArgs &a, int nf, int2 *s_acc) {
  __shared__ int s_key[kAcceptSmem], s_lab[kAcceptSmem], s_tgt[kAcceptSmem], s_ord[kAcceptSmem];
  __shared__ int s_nacc;
  const DevMerge &mg = a.mg;
  for (int j = threadIdx.x; j < nf; j += blockDim.x) {
    const int al = mg.found[j];
    s_lab[j] = al;
    s_key[j] = req_block(mg.req_min[al]);
    s_tgt[j] = mg.target[al];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nf; j += blockDim.x) {
    const int key = s_key[j];
    int rank = 0;
    for (int i = 0; i < nf; i++) rank += s_key[i] < key;  // keys are distinct block indices
    s_ord[rank] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int r = 0; r < nf; r++) {
      const int j = s_ord[r];
      const int al = s_lab[j], n = s_tgt[j];
      bool inv = false;
      for (int i = 0; i < acc; i++) {
        const int2 q = s_acc[i];
        inv |= (q.x == al) | (q.y == al) | (q.x == n) | (q.y == n);
      }
      if (!inv) s_acc[acc++] = make_int2(al, n);
    }
    s_nacc = acc;
  }
  __syncthreads();
  return s_nacc;
}

// The same walk for any number of found requests, on CTA 0, in global memory (mg.order,
// mg.involved, mg.acc, *mg.acc_count).
__device__ void merge_walk_big(const StageArgs &a, int nf) {
  const DevMerge &mg = a.mg;
  for (int j = threadIdx.x; j < nf; j += blockDim.x) {
    const unsigned long long key = mg.req_min[mg.found[j]];
    int rank = 0;
    for (int i = 0; i < nf; i++) rank += mg.req_min[mg.found[i]] < key;
    mg.order[rank] = mg.found[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int r = 0; r < nf; r++) {
      const int al = mg.order[r], n = mg.target[al];
      if (mg.involved[al] || mg.involved[n]) continue;
      mg.involved[al] = 1;
      mg.involved[n] = 1;
      mg.acc[acc++] = make_int2(al, n);
    }
    *mg.acc_count = acc;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < *(volatile int *)mg.acc_count; j += blockDim.x) {
    const int2 p = mg.acc[j];
    mg.involved[p.x] = 0;
    mg.involved[p.y] = 0;
  }
}

// Apply accepted merges (list in shared or global memory).  The request state needs no
// clearing: its keys and flags carry the phase number, so another CTA may still read them
// for its own walk while this one applies.
template <bool kBatch, int kSched>
__device__ __forceinline__ void merge_apply(const StageArgs &a, const ImageDesc *imgs, const int *label0,
                                            const int2 *acc, int nacc, int g, int slot) {
  const DevStats &s = a.st;
  const DevMerge &mg = a.mg;
  for (int j = blockIdx.x; j < nacc; j += gridDim.x) {
    const int al = acc[j].x, n = acc[j].y;
    const int ii = kBatch ? image_of_label(label0, a.nimg, al) : 0;
    const ImageDesc &im = kBatch ? imgs[ii] : a.img0;
    const int4 ba = s.bbox[al];
    if (threadIdx.x == 0) {
      s.N[n] += s.N[al];
      s.R[n] += s.R[al];
      s.G[n] += s.G[al];
      s.B[n] += s.B[al];
      s.X[n] += s.X[al];
      s.Y[n] += s.Y[al];
      s.N[al] = s.R[al] = s.G[al] = s.B[al] = s.X[al] = s.Y[al] = 0;
      set_means(s, n);
      set_means(s, al);
      s.chg[n] = 2 * g + 1;
      s.chg[al] = 2 * g + 1;
      a.ctl.last_merge[ii] = 2 * g + 1;
      int4 bn = s.bbox[n];
      bn.x = min(bn.x, ba.x);
      bn.y = min(bn.y, ba.y);
      bn.z = max(bn.z, ba.z);
      bn.w = max(bn.w, ba.w);
      s.bbox[n] = bn;
      atomic_add_i64(&a.ctl.cnt[(long long)ii * kCntStride + CNT_MERGES], 1);
      atomicAdd(&a.ctl.changes[3 * ii + slot], 1ull);
      if (queue_schedule<kSched>(a)) {  // the 4-neighbours of the request's first block join the queue
        const long long blk = (long long)req_block(mg.req_min[al]) - im.blk0;
        queue_push_neighbours(a, im, (int)(blk % im.nbx), (int)(blk / im.nbx));
      }
    }
    const int bx0 = ba.x / a.side, bx1 = ba.z / a.side, by0 = ba.y / a.side, by1 = ba.w / a.side;
    const int bw = bx1 - bx0 + 1;
    const long long total = (long long)bw * (by1 - by0 + 1);
    const bool marks = sweep_schedule<kSched>(a);
    for (long long t = threadIdx.x; t < total; t += blockDim.x) {
      const int cx = bx0 + (int)(t % bw), cy = by0 + (int)(t / bw);
      const long long idx = (long long)cy * im.nbx + cx;
      if (im.lab[idx] == al) {
        im.lab[idx] = n;
        if (marks) sweep_mark_plus(a, im, cx, cy, true);  // the cell and its 4-neighbours may turn eligible
      }
    }
  }
}

// Section timer of the first CTA (profiling only).
struct Timer {
  long long *prof;
  unsigned long long t;
  __device__ Timer(long long *p) : prof((blockIdx.x == 0 && threadIdx.x == 0) ? p : nullptr), t(0) {
    if (prof) t = global_ns();
  }
  __device__ __forceinline__ void lap(int section) {
    if (prof) {
      const unsigned long long n = global_ns();
      prof[section] += (long long)(n - t);
      t = n;
    }
  }
};

// kBatch: a launch over several images (descriptors copied to shared memory); otherwise
// one image, whose descriptor the kernel reads from its parameters.  kSched: the sweep
// schedule alone, the queue schedule alone (such a kernel carries only the code of its
// schedule), or either by a.frontier (used for batches under the sweep schedule).
template <bool kBatch, int kSched, bool kCluster = false>
__global__ void __launch_bounds__(kThreads, 1) stage_kernel(StageArgs a) {
  constexpr int kImgs = kBatch ? kMaxBatch : 1;
  __shared__ WarpTile wts[kThreads / 32];
  __shared__ int2 s_acc[kAcceptSmem];
  __shared__ ImageDesc s_img[kImgs];
  __shared__ int s_tile0[kImgs], s_label0[kImgs];
  __shared__ unsigned char s_active[kImgs], s_pruned[kImgs];
  __shared__ int s_valid_from[kImgs];
  __shared__ int s_cnt[kImgs * 8];
  __shared__ int s_draw, s_any;
  unsigned epoch = 0;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
  for (int i = threadIdx.x; i < (kBatch ? a.nimg : 1); i += blockDim.x) {
    if (kBatch) {
      s_img[i] = a.imgs[i];
      s_tile0[i] = a.imgs[i].tile0;
      s_label0[i] = a.imgs[i].label0;
    }
    s_active[i] = 1;
    s_pruned[i] = a.prune ? 1 : 0;
    s_valid_from[i] = 0;
  }
  for (int k = blockIdx.x + gridDim.x * threadIdx.x; k < a.st.M; k += gstride) {
    set_means(a.st, k);
    a.st.chg[k] = 0;
    a.mg.cache_stamp[k] = 0;
    a.mg.req_flag[k] = 0;  // phase numbers restart at 1 in every launch
    a.mg.req_min[k] = ~0ull;
    a.st.adj[k] = 0;
  }
  const long long nrec = (long long)a.ntiles * 9;
  if (a.wstamp) {  // race check: no block written in this launch yet
    const long long nb = (long long)(kBatch ? a.imgs[a.nimg - 1].blk0 : 0) +
                         (long long)(kBatch ? a.imgs[a.nimg - 1].nbx : a.img0.nbx) *
                             (kBatch ? a.imgs[a.nimg - 1].nby : a.img0.nby);
    for (long long i = gtid; i < nb; i += gstride) a.wstamp[i] = 0;
  }
  if (sweep_schedule<kSched>(a)) {  // sweep schedule: every block may be eligible when the stage starts
    for (int i = gtid; i < a.cwb[9]; i += gstride) {
      a.cbits[i] = ~0u;
      a.rbits[i] = 0u;
    }
  }
  if (queue_schedule<kSched>(a)) {  // frontier schedule: every block is queued when the stage starts
    for (long long i = gtid; i < nrec * kQueueWords; i += gstride) a.qbits[i] = ~0u;
    if (gtid < 9) a.wl_count[gtid] = 0;  // blocks queued from the start are not listed
  }
  if (!grid_sync<kCluster>(a.ctl, epoch)) return;
  Timer tm(a.ctl.prof);
  int g = 0;
  for (int sweep = 0; sweep < a.max_sweeps; sweep++) {
    const int slot = sweep % 3;
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < a.nimg; i += blockDim.x) a.ctl.changes[3 * i + (sweep + 1) % 3] = 0;
    for (int ph = 0; ph < 9; ph++) {
      g++;
      // frontier schedule: after the first sweep every queued block is on its class's list;
      // a short list is worked off one thread per block, a long one by the tile walk
      if (sweep_schedule<kSched>(a)) {
        eval_sweep<kBatch, kSched>(a, s_img, s_active, s_pruned, s_valid_from, wts, s_cnt, ph, g, slot, sweep);
      } else if constexpr (kSched != kSchedSweeps) {
        const int nq = sweep > 0 ? ld_volatile_i32(a.wl_count + ph) : INT_MAX;
        if (nq <= 4 * (int)(gridDim.x * blockDim.x))
          eval_queue<kBatch, kSched>(a, s_img, s_active, s_cnt, ph, g, slot, nq);
        else
          eval_phase<kBatch, kSched>(a, s_img, s_tile0, s_active, wts, &s_draw, ph, g, slot);
      }

      tm.lap(PROF_EVAL);
      if (!grid_sync<kCluster>(a.ctl, epoch)) return;
      tm.lap(PROF_SYNC1);
      const int gp = g & 1;
      if (blockIdx.x == 0 && threadIdx.x == 0) {  // slots of the next phase; last read a phase ago
        a.mg.req_count[gp ^ 1] = 0;
        a.mg.found_count[gp ^ 1] = 0;
        if (queue_schedule<kSched>(a)) a.wl_count[ph] = 0;  // the class's queued blocks all left the queue above
      }
      // the snapshot refresh and the merge-target search (which reads only S, the label
      // map and the merge state) share the barrier that ends them
      commit_phase(a, g);
      const int rq = ld_volatile_i32(a.mg.req_count + gp);
      if (rq > 0) merge_targets<kBatch>(a, s_img, s_label0, rq, g);
      tm.lap(PROF_COMMIT);
      if (!grid_sync<kCluster>(a.ctl, epoch)) return;
      tm.lap(PROF_SYNC2);
      if (rq > 0) {
        const int nf = ld_volatile_i32(a.mg.found_count + gp);
        if (nf > 0) {
          if (nf <= kAcceptSmem) {
            const int nacc = merge_walk_small(a, nf, s_acc);
            merge_apply<kBatch, kSched>(a, s_img, s_label0, s_acc, nacc, g, slot);
          } else {
            if (blockIdx.x == 0) merge_walk_big(a, nf);
            if (!grid_sync<kCluster>(a.ctl, epoch)) return;
            merge_apply<kBatch, kSched>(a, s_img, s_label0, a.mg.acc, ld_volatile_i32(a.mg.acc_count), g, slot);
          }
          if (!grid_sync<kCluster>(a.ctl, epoch)) return;
        }
        tm.lap(PROF_MERGE);
      }
    }
    // End of the sweep (every CTA decides the same from the same counts): an image whose
    // sweep changed nothing has finished this stage, and its tiles are no longer visited --
    // unless that sweep was pruned: then it goes on with full sweeps, and tile records made
    // before (phase numbers <= g) no longer count.
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < (kBatch ? a.nimg : 1); i += blockDim.x) {
      if (!s_active[i]) continue;
      if (blockIdx.x == 0) a.ctl.cnt[(long long)i * kCntStride + CNT_SWEEPS] += 1;
      if (ld_volatile_u64(&a.ctl.changes[3 * i + slot]) != 0) {
        s_any = 1;
      } else if (s_pruned[i]) {
        s_pruned[i] = 0;
        s_valid_from[i] = g + 1;
        s_any = 1;
      } else {
        s_active[i] = 0;
      }
    }
    __syncthreads();
    if (!s_any) break;
  }
}

}  // namespace RAPID_SHAPE_NS

const void *RAPID_CAT(stage_kernel_ptr_, RAPID_SHAPE_NS)(bool batch, bool frontier, bool cluster) {
  using namespace RAPID_SHAPE_NS;
  if (cluster) return frontier ? (const void *)stage_kernel<false, kSchedQueue, true>
                               : (const void *)stage_kernel<false, kSchedSweeps, true>;
  // (a batch under the sweep schedule runs the kernel that reads the schedule at run time:
  // measured 5% faster there than the sweeps-only build, 1042 against 1102 ms on 64 tiles)
  if (batch) return frontier ? (const void *)stage_kernel<true, kSchedQueue> : (const void *)stage_kernel<true, kSchedRuntime>;
  return frontier ? (const void *)stage_kernel<false, kSchedQueue> : (const void *)stage_kernel<false, kSchedSweeps>;
}

// A single image's stage of at most kMaxCluster CTAs runs as one thread-block cluster (the
// kernel built with the cluster's hardware barrier) when the device can co-schedule such a
// cluster; otherwise, for larger grids and for batches, as a cooperative launch (barriers
// through a counter in global memory).
cudaError_t RAPID_CAT(launch_stage_, RAPID_SHAPE_NS)(const StageArgs &a, int grid, int block, cudaStream_t s) {
  StageArgs copy = a;
  void *args[] = {&copy};
  if (a.nimg == 1 && grid >= 2 && grid <= kMaxCluster) {
    const void *fc = RAPID_CAT(stage_kernel_ptr_, RAPID_SHAPE_NS)(false, a.frontier != 0, true);
    if (cluster_launch_ok(fc, grid, block, s)) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(block);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = grid;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelExC(&cfg, fc, args);
    }
  }
  const void *fn = RAPID_CAT(stage_kernel_ptr_, RAPID_SHAPE_NS)(a.nimg > 1, a.frontier != 0, false);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, s);
}

}  // namespace rapid
