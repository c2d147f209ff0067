// eval_tile.cuh — the block tests and decisions shared by both schedules, and the queue
// schedule's phases (included by stage_impl.cuh, once per evaluation-tile shape).
//
// Dense queue phases: a warp takes a kTileW x kTileH-block tile, pops the tile's queued
// blocks of the phase class, stages the tile's labels with a 1-block halo in its own shared
// window ((kTileW + 2) x (kTileH + 2) int32) and gives each lane the popped blocks.  Warps
// never wait for each other inside a phase, so the SM hides the global-memory latency of
// one warp's tile behind the work of the others.  Sparse queue phases take their blocks
// from the class's worklist instead, one thread per block (eval_queue).
#pragma once

// (included inside namespace rapid)
static constexpr int kWinW = kTileW + 2, kWinH = kTileH + 2;

struct WarpTile {
  int win[kWinW * kWinH];
  int items[kPhaseMax];         // phase-class blocks (index j) that need a decision
  unsigned queue[kReqWords];    // the blocks popped from the queue now
};

// Decide a block: the target label, or -1 for no decrease (Eq. operation; ties to the
// smaller label, a move only on a strict decrease).  The candidates are visited once,
// keeping the best one's interval, the smallest lower bound among the others and the
// largest magnitude seen.
__device__ __forceinline__ int decide(const StageArgs &a, const ImageDesc &im, const BlockIn &in, Local &lc) {
  if (!im.use_filter) return decide_f64(a, in, im.lam_pos);
  const DevStats &s = a.st;
  const BlockSums &bs = in.bs;
  const int lbl = in.lbl;
  const float wf = (float)bs.w;  // exact: blocks have < 2^24 pixels when the filter is on
  const float r2f = (float)(2 * bs.r), g2f = (float)(2 * bs.g), b2f = (float)(2 * bs.b);
  const float x2f = (float)(2 * bs.x), y2f = (float)(2 * bs.y);
  const float pbx = (float)in.x0 + 0.5f * (float)(bs.bw - 1);  // P_x / w, exact
  const float pby = (float)in.y0 + 0.5f * (float)(bs.bh - 1);
  const float lamf = im.lam_pos_f, lamb2f = a.lam_b2_f;
  const float rlam = 1.0001f * kU * lamf, rlamb = 1.0001f * kU * lamb2f;  // |float - binary64| weights
  const float4 ha = s.fhi[lbl];
  const float2 ya = s.fy[lbl];
  int Ba = 0;
  if (in.nb[0] >= 0 && in.nb[0] != lbl) Ba += bs.bw;
  if (in.nb[1] >= 0 && in.nb[1] != lbl) Ba += bs.bh;
  if (in.nb[2] >= 0 && in.nb[2] != lbl) Ba += bs.bh;
  if (in.nb[3] >= 0 && in.nb[3] != lbl) Ba += bs.bw;
  const float4 la = s.flo[lbl];
  const float eps_a = eps64(ha, ya, wf, r2f, g2f, b2f, x2f, y2f, lamf, lamb2f, (float)Ba);

  int bk = -1;
  float bD = 0.f, bLo = 0.f, bHi = 0.f;
  float minLoOther = INFINITY, minLoAll = INFINITY, maxAbs = 0.f;
#pragma unroll 1
  for (int j = 0; j < 4; j++) {
    const int k = in.nb[j];
    if (k < 0 || k == lbl) continue;
    bool dup = false;
    for (int i = 0; i < j; i++) dup |= (in.nb[i] == k);
    if (dup) continue;
    int Bk = 0;
    if (in.nb[0] >= 0 && in.nb[0] != k) Bk += bs.bw;
    if (in.nb[1] >= 0 && in.nb[1] != k) Bk += bs.bh;
    if (in.nb[2] >= 0 && in.nb[2] != k) Bk += bs.bh;
    if (in.nb[3] >= 0 && in.nb[3] != k) Bk += bs.bw;
    const float4 hk = s.fhi[k], lk = s.flo[k];
    const float2 yk = s.fy[k];
    const Fr col = add_fr(add_fr(colour_term(hk.x, lk.x, ha.x, la.x, wf, r2f, kU * r2f),
                                 colour_term(hk.y, lk.y, ha.y, la.y, wf, g2f, kU * g2f)),
                          colour_term(hk.z, lk.z, ha.z, la.z, wf, b2f, kU * b2f));
    const Fr pos =
        add_fr(position_term(hk.w, lk.w, ha.w, la.w, pbx, wf), position_term(yk.x, yk.y, ya.x, ya.y, pby, wf));
    const float lp = lamf * pos.v;
    const Fr lpos = {lp, lamf * pos.r + fabsf(pos.v) * rlam + rlam * pos.r + kU * fabsf(lp)};
    const float dB = (float)(Bk - Ba);  // exact small integer
    const float bb = lamb2f * dB;
    const Fr bnd = {bb, fabsf(dB) * rlamb + kU * fabsf(bb)};
    const Fr d = add_fr(add_fr(col, lpos), bnd);
    const float eps_k = eps64(hk, yk, wf, r2f, g2f, b2f, x2f, y2f, lamf, lamb2f, (float)Bk);
    const float R = __fmul_ru(__fadd_ru(__fadd_ru(d.r, eps_k), eps_a), 1.01f);
    const float lo = __fsub_rd(d.v, R), hi = __fadd_ru(d.v, R);
    minLoAll = fminf(minLoAll, lo);
    maxAbs = fmaxf(maxAbs, fmaxf(fabsf(lo), fabsf(hi)));
    if (bk < 0 || d.v < bD || (d.v == bD && k < bk)) {
      if (bk >= 0) minLoOther = fminf(minLoOther, bLo);
      bk = k;
      bD = d.v;
      bLo = lo;
      bHi = hi;
    } else {
      minLoOther = fminf(minLoOther, lo);
    }
  }
  if (bk < 0) return -1;
  int result = -2;  // undecided
  if (minLoAll >= 0.f) {
    result = -1;  // every binary64 difference is >= 0: no move
  } else if (bHi < 0.f) {
    // strict lead of the best candidate that survives the final binary64 rounding of the
    // differences (margin 2^-50 of four times the largest magnitude)
    const float thr = __fmul_ru(maxAbs, 3.5527137e-15f);
    if (minLoOther == INFINITY || __fsub_rd(minLoOther, bHi) > thr) result = bk;
  }
  if (result == -2) {
    lc.fallback++;
    return decide_f64(a, in, im.lam_pos);
  }
  if (a.verify_filter) {
    const int ref = decide_f64(a, in, im.lam_pos);
    if (ref != result) {
      lc.mismatch++;
      return ref;
    }
  }
  return result;
}

// ---------------------------------------------------------------- one block, two passes
// Pass 1 (every phase-class block of the tile, one lane each): the cheap tests from the
// shared window -- boundary (Eq. bound), boundary superpixel (Eq. new_bound), topology
// (E_topo) -- and the counters.  Returns true when the block needs an energy decision: it
// passed the tests and, when block_skip holds (the tile was scanned before in this phase
// class and its label set is complete), its label or a neighbour label changed since, or
// it requested a merge then.  Otherwise it decides as at the previous scan: no move.
// The tests of one block from its label, its 4-neighbours (N, W, E, S) and its diagonal
// neighbours (NW, NE, SE, SW); -1 outside the grid.  Counts eligible and evaluated blocks.
__device__ __forceinline__ bool block_tests(const StageArgs &a, int lbl, int nN, int nW, int nE, int nS, int nNW,
                                            int nNE, int nSE, int nSW, const unsigned char *mask, long long blk,
                                            Local &lc) {
  const bool boundary = (nN >= 0 && nN != lbl) || (nW >= 0 && nW != lbl) || (nE >= 0 && nE != lbl) ||
                        (nS >= 0 && nS != lbl);
  if (!boundary) return false;
  const DevStats &s = a.st;
  if (a.imp_on) {
    if (a.imp_rule == 0) {
      if (!s.imp[lbl]) return false;
    } else {
      const signed char ya = s.y[lbl];
      const bool any = (nN >= 0 && nN != lbl && s.y[nN] != ya) || (nW >= 0 && nW != lbl && s.y[nW] != ya) ||
                       (nE >= 0 && nE != lbl && s.y[nE] != ya) || (nS >= 0 && nS != lbl && s.y[nS] != ya);
      if (!any) return false;
    }
  }
  lc.elig++;
  // pruned sweeps: the learned scorer decides which eligible blocks get the exact tests
  if (mask && !mask[blk]) return false;
  const unsigned m = (unsigned)(nNW == lbl) | ((unsigned)(nN == lbl) << 1) | ((unsigned)(nNE == lbl) << 2) |
                     ((unsigned)(nE == lbl) << 3) | ((unsigned)(nSE == lbl) << 4) | ((unsigned)(nS == lbl) << 5) |
                     ((unsigned)(nSW == lbl) << 6) | ((unsigned)(nW == lbl) << 7);
  if (!simple_mask(m)) return false;
  lc.eval++;
  return true;
}

// Frontier schedule: queue block (gx, gy) of image im (no-op outside the block grid).  Its
// tile, phase class and index j in the class lattice of the tile are those eval_phase
// enumerates: the class lattice of a tile starts at (lx % 3, ly % 3).
// The queue word of block (gx, gy) (inside the grid) and its bit.
__device__ __forceinline__ unsigned *queue_word(const StageArgs &a, const ImageDesc &im, int gx, int gy,
                                                unsigned *bit) {
  const int tx = gx / kTileW, ty = gy / kTileH;
  const int lx = gx - tx * kTileW, ly = gy - ty * kTileH;
  const int tw = min(kTileW, im.nbx - tx * kTileW);
  const int nx = (tw - lx % 3 + 2) / 3;
  const int j = (ly / 3) * nx + lx / 3;
  const long long t = (long long)im.tile0 + (long long)ty * im.ntx + tx;
  *bit = 1u << (j & 31);
  return a.qbits + (t * 9 + (gy % 3) * 3 + gx % 3) * kQueueWords + (j >> 5);
}

// The 4-neighbours of block (bx, by) go on the queue; those that were not queued also go on
// their class's worklist (global block index), from which sparse phases take their blocks,
// so each queued block is listed at most once.  The four flag updates are issued together,
// then the list slots together.
__device__ __forceinline__ void queue_push_neighbours(const StageArgs &a, const ImageDesc &im, int bx, int by) {
  const int nx[4] = {bx, bx - 1, bx + 1, bx}, ny[4] = {by - 1, by, by, by + 1};
  unsigned old[4], bit[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    old[q] = bit[q] = 0u;
    if (nx[q] < 0 || ny[q] < 0 || nx[q] >= im.nbx || ny[q] >= im.nby) continue;
    unsigned *w = queue_word(a, im, nx[q], ny[q], &bit[q]);
    old[q] = atomicOr(w, bit[q]);
  }
  int slot[4];
#pragma unroll
  for (int q = 0; q < 4; q++)
    slot[q] = (bit[q] && !(old[q] & bit[q])) ? atomicAdd(a.wl_count + (ny[q] % 3) * 3 + nx[q] % 3, 1) : -1;
#pragma unroll
  for (int q = 0; q < 4; q++)
    if (slot[q] >= 0)
      a.wl[(long long)((ny[q] % 3) * 3 + nx[q] % 3) * a.wl_cap + slot[q]] = im.blk0 + ny[q] * im.nbx + nx[q];
}

// Pass 2 (one compacted block per lane): block sums, the decision (Eq. operation), the size
// term (Sec. 3.1) and the move.
// Returns true when the block raised a merge request instead of moving.  Under the queue
// schedule a move queues its 4-neighbours.
template <int kSched>
__device__ __forceinline__ bool decide_block_at(const StageArgs &a, const ImageDesc &im, int lbl0, int nN, int nW,
                                                int nE, int nS, int bx, int by, int g, Local &lc) {
  const DevStats &s = a.st;
  BlockIn in;
  in.lbl = lbl0;
  in.nb[0] = nN;
  in.nb[1] = nW;
  in.nb[2] = nE;
  in.nb[3] = nS;
  in.bs = block_sums(a, im, bx, by);
  in.x0 = bx * a.side;
  in.y0 = by * a.side;
  const int lbl = in.lbl;
  const int k = decide(a, im, in, lc);
  if (k < 0) return false;
  const long long idx = (long long)by * im.nbx + bx;
  if (a.size_mode != 0 && (long long)a.lo_den * (s.mN[lbl] - in.bs.w) < (long long)a.lo_num * s.init[lbl]) {
    if (a.size_mode != 2) return false;
    lc.req++;
    atomicMin(&a.mg.req_min[lbl], req_key(g, im.blk0 + idx));  // global block order
    if (atomicExch(&a.mg.req_flag[lbl], g) != g) {
      const int slot = atomicAdd(a.mg.req_count + (g & 1), 1);
      a.mg.req_list[slot] = lbl;
    }
    return true;
  }
  // Move: relabel in place, add the exact sums to S (decisions of this phase read only the
  // snapshot means and counts, never S).
  const BlockSums &bs = in.bs;
  im.lab[idx] = k;
  if (a.wstamp) race_check(a.race, a.wstamp, im.blk0, im.nbx, im.nby, bx, by, g, (g - 1) % 9);
  atomic_add_i64(&s.N[lbl], -bs.w);
  atomic_add_i64(&s.R[lbl], -bs.r);
  atomic_add_i64(&s.G[lbl], -bs.g);
  atomic_add_i64(&s.B[lbl], -bs.b);
  atomic_add_i64(&s.X[lbl], -bs.x);
  atomic_add_i64(&s.Y[lbl], -bs.y);
  atomic_add_i64(&s.N[k], bs.w);
  atomic_add_i64(&s.R[k], bs.r);
  atomic_add_i64(&s.G[k], bs.g);
  atomic_add_i64(&s.B[k], bs.b);
  atomic_add_i64(&s.X[k], bs.x);
  atomic_add_i64(&s.Y[k], bs.y);
  s.dirty[lbl] = 1;
  s.dirty[k] = 1;
  // the adjacency of the block's old and new labels and of its 4-neighbours' labels may
  // have changed (every writer of this phase stores the same stamp)
  s.adj[lbl] = 2 * g;
  s.adj[k] = 2 * g;
  for (int q = 0; q < 4; q++)
    if (in.nb[q] >= 0) s.adj[in.nb[q]] = 2 * g;
  atomicMin(&s.bbox[k].x, in.x0);
  atomicMin(&s.bbox[k].y, in.y0);
  atomicMax(&s.bbox[k].z, in.x0 + bs.bw - 1);
  atomicMax(&s.bbox[k].w, in.y0 + bs.bh - 1);
  if (queue_schedule<kSched>(a)) queue_push_neighbours(a, im, bx, by);  // (other phase classes only)
  lc.moves++;
  return false;
}

__device__ inline int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Insert v into a shared append-only set of `cap` slots initialised to -1; sets *over when
// the set is full.
__device__ __forceinline__ void set_insert(int *set, int cap, int v, int *over) {
  for (int j = 0; j < cap; j++) {
    int cur = ((volatile int *)set)[j];
    if (cur == v) return;
    if (cur == -1) {
      cur = atomicCAS(&set[j], -1, v);
      if (cur == -1 || cur == v) return;
    }
  }
  *over = 1;
}

// ---------------------------------------------------------------- one phase
// Counters of one warp's run of tiles of one image, added to the image's counters at once.
__device__ __forceinline__ void flush_counts(const StageArgs &a, int ii, int slot, Local &lc, int &scanned,
                                             int &skipped) {
  const int lane = threadIdx.x & 31;
  const int e = warp_sum(lc.elig), v = warp_sum(lc.eval), m = warp_sum(lc.moves), r = warp_sum(lc.req);
  const int fb = warp_sum(lc.fallback), mm = warp_sum(lc.mismatch);
  const int sc = warp_sum(scanned), sk = warp_sum(skipped);
  if (lane == 0 && ii >= 0) {
    long long *cnt = a.ctl.cnt + (long long)ii * kCntStride;
    if (e) atomic_add_i64(&cnt[CNT_ELIG], e);
    if (v) atomic_add_i64(&cnt[CNT_EVAL], v);
    if (m) {
      atomic_add_i64(&cnt[CNT_MOVES], m);
      atomicAdd(&a.ctl.changes[3 * ii + slot], (unsigned long long)m);
    }
    if (r) atomic_add_i64(&cnt[CNT_REQ], r);
    if (fb) atomic_add_i64(&cnt[CNT_FALLBACK], fb);
    if (mm) atomic_add_i64(&cnt[CNT_MISMATCH], mm);
    if (sc) atomic_add_i64(&cnt[CNT_SCANNED], sc);
    if (sk) atomic_add_i64(&cnt[CNT_SKIPPED], sk);
  }
  lc = Local{0, 0, 0, 0, 0, 0};
  scanned = skipped = 0;
}

// Frontier schedule, a phase whose class has many queued blocks (and the first sweep of a
// stage, when every block is queued): one warp per tile of kTileW x kTileH blocks pops the
// tile's queued blocks of the class (skipping the tile when none is queued), stages the
// tile's labels with a 1-block halo in shared memory and decides the popped blocks.
// g: 1-based phase number within the launch; slot: the sweep's change-count slot; imgs,
// tile0 and active are the CTA's shared copies of the images, their first tiles and
// whether each still refines in this stage.
template <bool kBatch, int kSched>
__device__ __forceinline__ void eval_phase(const StageArgs &a, const ImageDesc *imgs, const int *tile0,
                                           const unsigned char *active, WarpTile *wts, int *s_draw, int phase, int g,
                                           int slot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpTile &W = wts[warp];
  const int py = phase / 3, px = phase % 3;
  if (threadIdx.x == 0) *s_draw = 0;
  __syncthreads();
  int draw = 0;
  if (lane == 0) draw = atomicAdd(s_draw, 1);
  draw = __shfl_sync(0xffffffffu, draw, 0);
  Local lc = {0, 0, 0, 0, 0, 0};
  int scanned = 0, skipped = 0, cur = -1;
  for (;;) {
    const long long tt = (long long)blockIdx.x + (long long)draw * gridDim.x;
    if (tt >= a.ntiles) break;
    const int t = (int)tt;
    int nxt = 0;
    if (lane == 0) nxt = atomicAdd(s_draw, 1);
    draw = __shfl_sync(0xffffffffu, nxt, 0);  // used by the next iteration
    // the tile's image: the last one whose first tile is <= t (a warp's tiles only go up)
    int lo = cur < 0 ? 0 : cur, hi = kBatch ? a.nimg - 1 : 0;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile0[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    if (lo != cur) {
      flush_counts(a, cur, slot, lc, scanned, skipped);
      cur = lo;
    }
    if (!active[cur]) continue;  // the image finished this stage
    const ImageDesc &im = kBatch ? imgs[cur] : a.img0;
    const int lt = t - im.tile0;
    const int tx = lt % im.ntx, ty = lt / im.ntx;
    const int bx0 = tx * kTileW, by0 = ty * kTileH;
    // pop the tile's queued blocks of this class (if any)
    unsigned *qw = a.qbits + ((long long)t * 9 + phase) * kQueueWords;
    const unsigned qv = lane < kReqWords ? qw[lane] : 0u;
    if (!__any_sync(0xffffffffu, qv != 0u)) {
      if (lane == 0) skipped++;
      continue;
    }
    if (lane < kReqWords) qw[lane] = 0u;
    if (lane == 0) scanned++;
    if (lane < kReqWords) W.queue[lane] = qv;
    // window: lane = column (lanes 0 and 1 also take columns 32 and 33)
    for (int col = lane; col < kWinW; col += 32) {
      const int gx = bx0 - 1 + col;
      const bool inx = gx >= 0 && gx < im.nbx;
#pragma unroll
      for (int wy = 0; wy < kWinH; wy++) {
        const int gy = by0 - 1 + wy;
        W.win[wy * kWinW + col] = (inx && gy >= 0 && gy < im.nby) ? im.lab[(long long)gy * im.nbx + gx] : -1;
      }
    }
    // the tile's blocks of this phase class
    const int lx0 = ((px - bx0) % 3 + 3) % 3, ly0 = ((py - by0) % 3 + 3) % 3;
    const int tw = min(kTileW, im.nbx - bx0), th = min(kTileH, im.nby - by0);
    const int nx = tw > lx0 ? (tw - lx0 + 2) / 3 : 0, ny = th > ly0 ? (th - ly0 + 2) / 3 : 0;
    __syncwarp();
    // pass 1: the tests of the popped blocks; those that need a decision are compacted
    int nitems = 0;
    for (int j0 = 0; j0 < nx * ny; j0 += 32) {
      const int j = j0 + lane;
      bool need = false;
      if (j < nx * ny && ((W.queue[j >> 5] >> (j & 31)) & 1u)) {
        const int lx = lx0 + 3 * (j % nx), ly = ly0 + 3 * (j / nx);
        const int c = (ly + 1) * kWinW + (lx + 1);
        const int *win = W.win;
        need = block_tests(a, win[c], win[c - kWinW], win[c - 1], win[c + 1], win[c + kWinW], win[c - kWinW - 1],
                           win[c - kWinW + 1], win[c + kWinW + 1], win[c + kWinW - 1], nullptr, 0, lc);
      }
      const unsigned ball = __ballot_sync(0xffffffffu, need);
      if (need) W.items[nitems + __popc(ball & ((1u << lane) - 1u))] = j;
      nitems += __popc(ball);
    }
    __syncwarp();
    // pass 2: decisions, one compacted block per lane
    for (int it = lane; it < nitems; it += 32) {
      const int j = W.items[it];
      const int lx = lx0 + 3 * (j % nx), ly = ly0 + 3 * (j / nx);
      const int c = (ly + 1) * kWinW + (lx + 1);
      const int *win = W.win;
      decide_block_at<kSched>(a, im, win[c], win[c - kWinW], win[c - 1], win[c + 1], win[c + kWinW], bx0 + lx,
                              by0 + ly, g, lc);
    }
    __syncwarp();
  }
  flush_counts(a, cur, slot, lc, scanned, skipped);
}

// ---------------------------------------------------------------- sparse frontier phase
// Frontier schedule, phase class `phase` with nq listed blocks: one thread per listed block
// (32 consecutive entries per warp, warps spread over the CTAs first), no tile walk.  The
// listed blocks are exactly the queued blocks of the class; each leaves the queue here.
// Counts go through the CTA's per-image shared counters s_cnt[image * 8 + ...].
template <bool kBatch, int kSched>
__device__ __forceinline__ void eval_queue(const StageArgs &a, const ImageDesc *imgs, const unsigned char *active,
                                           int *s_cnt, int phase, int g, int slot, int nq) {
  const int nimg = kBatch ? a.nimg : 1;
  for (int i = threadIdx.x; i < nimg * 8; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int *list = a.wl + (long long)phase * a.wl_cap;
  for (long long base = (long long)(warp * gridDim.x + blockIdx.x) * 32; base < nq; base += (long long)nwarps * 32) {
    const long long e = base + lane;
    if (e >= nq) continue;
    const int gb = list[e];
    int ii = 0;
    if (kBatch) {
      int lo = 0, hi = nimg - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].blk0 <= gb) lo = mid;
        else hi = mid - 1;
      }
      ii = lo;
    }
    if (!active[ii]) continue;
    const ImageDesc &im = kBatch ? imgs[ii] : a.img0;
    const int idx = gb - im.blk0;
    const int bx = idx % im.nbx, by = idx / im.nbx;
    const int *lab = im.lab;
    const int W = im.nbx, H = im.nby;
    const bool n_ok = by > 0, s_ok = by + 1 < H, w_ok = bx > 0, e_ok = bx + 1 < W;
    const int lbl = lab[idx];
    const int nN = n_ok ? lab[idx - W] : -1, nS = s_ok ? lab[idx + W] : -1;
    const int nW = w_ok ? lab[idx - 1] : -1, nE = e_ok ? lab[idx + 1] : -1;
    const int nNW = (n_ok && w_ok) ? lab[idx - W - 1] : -1, nNE = (n_ok && e_ok) ? lab[idx - W + 1] : -1;
    const int nSW = (s_ok && w_ok) ? lab[idx + W - 1] : -1, nSE = (s_ok && e_ok) ? lab[idx + W + 1] : -1;
    // what the tests and the decision read next, fetched into L1 at once instead of one
    // round trip after another
    prefetch_l1(a.st.imp + lbl);
    prefetch_l1(a.st.mN + lbl);
    prefetch_l1(a.st.init + lbl);
    prefetch_l1(a.st.fhi + lbl);
    prefetch_l1(a.st.flo + lbl);
    prefetch_l1(a.st.fy + lbl);
    const int nb4[4] = {nN, nW, nE, nS};
#pragma unroll
    for (int q = 0; q < 4; q++)
      if (nb4[q] >= 0 && nb4[q] != lbl) {
        prefetch_l1(a.st.fhi + nb4[q]);
        prefetch_l1(a.st.flo + nb4[q]);
        prefetch_l1(a.st.fy + nb4[q]);
      }
    if (a.f == 1) prefetch_l1(im.img + (long long)by * a.side * im.img_pitch + 3ll * bx * a.side);
    unsigned bit;
    unsigned *w = queue_word(a, im, bx, by, &bit);
    atomicAnd(w, ~bit);  // off the queue
    Local lc = {0, 0, 0, 0, 0, 0};
    if (block_tests(a, lbl, nN, nW, nE, nS, nNW, nNE, nSE, nSW, nullptr, 0, lc))
      decide_block_at<kSched>(a, im, lbl, nN, nW, nE, nS, bx, by, g, lc);
    int *c = s_cnt + ii * 8;
    if (lc.elig) atomicAdd(c + 0, lc.elig);
    if (lc.eval) atomicAdd(c + 1, lc.eval);
    if (lc.moves) atomicAdd(c + 2, lc.moves);
    if (lc.req) atomicAdd(c + 3, lc.req);
    if (lc.fallback) atomicAdd(c + 4, lc.fallback);
    if (lc.mismatch) atomicAdd(c + 5, lc.mismatch);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nimg; i += blockDim.x) {
    const int *c = s_cnt + i * 8;
    long long *cnt = a.ctl.cnt + (long long)i * kCntStride;
    if (c[0]) atomic_add_i64(&cnt[CNT_ELIG], c[0]);
    if (c[1]) atomic_add_i64(&cnt[CNT_EVAL], c[1]);
    if (c[2]) {
      atomic_add_i64(&cnt[CNT_MOVES], c[2]);
      atomicAdd(&a.ctl.changes[3 * i + slot], (unsigned long long)c[2]);
    }
    if (c[3]) atomic_add_i64(&cnt[CNT_REQ], c[3]);
    if (c[4]) atomic_add_i64(&cnt[CNT_FALLBACK], c[4]);
    if (c[5]) atomic_add_i64(&cnt[CNT_MISMATCH], c[5]);
  }
}
