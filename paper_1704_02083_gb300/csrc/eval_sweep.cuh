// eval_sweep.cuh — block decisions of one phase of the sweep schedule, from a bitmap of the
// blocks of the phase class that may be eligible (included by stage_impl.cuh, inside the
// shape's namespace).
//
// A sweep examines every block of every class (Sec. 2.1: relabel the boundary blocks; the
// 9-phase reading R10).  Only eligible blocks -- boundary blocks (Eq. bound) of important
// labels at the finer levels (Eq. new_bound) -- can move, and they are a small share of
// the grid, so a phase walks a per-class bitmap `cbits` that holds a superset of the
// class's eligible blocks, kept so by three rules:
//   * when the stage starts every bit is set;
//   * a block that is visited and found not eligible has its bit cleared;
//   * a block whose label changes (a move, or the relabelling of an accepted merge) sets
//     the bits of its 4-neighbours (its own stays set).
// Eligibility depends only on the block's label, its 4-neighbours' labels and per-label
// flags that are fixed during a stage (importance, class y), so a block can become
// eligible only when a label of its 4-neighbourhood changes, which sets its bit.  Every
// eligible block is therefore visited in every sweep, and the eligible and evaluated
// counts equal those of a walk over the whole class.
//
// A visited block that passes the tests skips the decision when neither its label nor a
// 4-neighbour label has changed S since its class's previous phase (g - 9) and it did not
// request a merge then (`rbits`): a label change in its 3x3 window changes the S of the
// old and the new label, one of which is then the block's own label or a 4-neighbour
// label whenever the change reaches the boundary test, the topology mask or the energy.
// Its window, candidates and snapshot means are then those of the previous phase, whose
// decision was no move (a move would have changed its own label).
#pragma once

// Blocks a lane tests at once: their loads are issued together.
constexpr int kPer = kThreads >= 1024 ? 2 : 4;

// N bitmap words as a walk holds them in shared memory.
template <int N>
struct SweepWords {
  unsigned bits[N];              // the words, as loaded
  int pre[N];                    // inclusive prefix sums of their set-bit counts
  unsigned clr[N];               // bits to clear: blocks found not eligible, bits past the row
  unsigned req[N];               // request-memo words as this phase leaves them
  int img[N], row[N], col0[N];   // image, lattice row and first lattice column of each word
};

// Per-warp scratch of the warp walk (overlays the warp's WarpTile).
struct WarpSweep {
  SweepWords<32> w;
  int dec[32 * kPer];            // blocks that need a decision: word << 5 | bit
};
static_assert(sizeof(WarpSweep) <= sizeof(WarpTile), "the warp walk's scratch overlays the warp's tile");

// CTA scratch of the CTA walk (overlays the CTA's warp tiles).
struct CtaSweep {
  SweepWords<kThreads> w;
  int dec[kThreads * kPer];      // blocks that need a decision: word << 5 | bit
  int wsum[32];                  // per-warp set-bit counts, then their exclusive prefix sums
  int total;                     // set bits of the CTA's words this round
  int ndec[2];                   // entries in dec (alternating between batches of tests)
};
static_assert(sizeof(CtaSweep) <= sizeof(WarpTile) * (kThreads / 32),
              "the CTA walk's scratch overlays the CTA's warp tiles");

// The word that holds set bit number e of the words: the first whose prefix sum exceeds e.
template <int N>
__device__ __forceinline__ int word_of_entry(const SweepWords<N> &W, int e) {
  int lo = 0, hi = N - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (W.pre[mid] > e) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Labels of block (x, y) and its 8 neighbours: own, N, W, E, S, NW, NE, SE, SW (-1 outside
// the grid).
__device__ __forceinline__ void load_window(const ImageDesc &im, int x, int y, int *l) {
  const int *lab = im.lab;
  const int nbx = im.nbx;
  const long long idx = (long long)y * nbx + x;
  const bool n_ok = y > 0, s_ok = y + 1 < im.nby, w_ok = x > 0, e_ok = x + 1 < nbx;
  l[0] = lab[idx];
  l[1] = n_ok ? lab[idx - nbx] : -1;
  l[2] = w_ok ? lab[idx - 1] : -1;
  l[3] = e_ok ? lab[idx + 1] : -1;
  l[4] = s_ok ? lab[idx + nbx] : -1;
  l[5] = (n_ok && w_ok) ? lab[idx - nbx - 1] : -1;
  l[6] = (n_ok && e_ok) ? lab[idx - nbx + 1] : -1;
  l[7] = (s_ok && e_ok) ? lab[idx + nbx + 1] : -1;
  l[8] = (s_ok && w_ok) ? lab[idx + nbx - 1] : -1;
}

// Block (x, y) of image im may be eligible (no-op outside the block grid).
__device__ __forceinline__ void sweep_mark(const StageArgs &a, const ImageDesc &im, int x, int y) {
  if (x < 0 || y < 0 || x >= im.nbx || y >= im.nby) return;
  const int px = x % 3, i = x / 3;
  const long long w = (long long)im.cw0[(y % 3) * 3 + px] + (long long)(y / 3) * class_wpr(im.nbx, px) + (i >> 5);
  atomicOr(a.cbits + w, 1u << (i & 31));
}

// The 4-neighbours of block (x, y), and the block itself when `self`.
__device__ __forceinline__ void sweep_mark_plus(const StageArgs &a, const ImageDesc &im, int x, int y, bool self) {
  if (self) sweep_mark(a, im, x, y);
  sweep_mark(a, im, x, y - 1);
  sweep_mark(a, im, x - 1, y);
  sweep_mark(a, im, x + 1, y);
  sweep_mark(a, im, x, y + 1);
}

// Adds a lane's counts to the CTA's per-image shared counters (8 per image: eligible,
// evaluated, moves, requests, fallbacks, filter mismatches, visited blocks, skipped
// decisions) and clears them.
__device__ __forceinline__ void flush_sweep_counts(int *s_cnt, int ii, Local &lc, int &visited, int &skipped) {
  int *c = s_cnt + ii * 8;
  if (lc.elig) atomicAdd(c + 0, lc.elig);
  if (lc.eval) atomicAdd(c + 1, lc.eval);
  if (lc.moves) atomicAdd(c + 2, lc.moves);
  if (lc.req) atomicAdd(c + 3, lc.req);
  if (lc.fallback) atomicAdd(c + 4, lc.fallback);
  if (lc.mismatch) atomicAdd(c + 5, lc.mismatch);
  if (visited) atomicAdd(c + 6, visited);
  if (skipped) atomicAdd(c + 7, skipped);
  lc = Local{0, 0, 0, 0, 0, 0};
  visited = skipped = 0;
}

// The CTA's per-image shared counters into the image counters (after a CTA barrier).
__device__ __forceinline__ void store_sweep_counts(const StageArgs &a, const int *s_cnt, int nimg, int slot) {
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
    if (c[6]) atomic_add_i64(&cnt[CNT_SCANNED], c[6]);
    if (c[7]) atomic_add_i64(&cnt[CNT_SKIPPED], c[7]);
  }
}

// Word w of the class (phase) into slot i of W: its image, row and first column, and its
// bitmap and request-memo words (zero for a word past the class or of a retired image).
template <bool kBatch, int N>
__device__ __forceinline__ unsigned sweep_load_word(const StageArgs &a, const ImageDesc *imgs,
                                                    const unsigned char *active, int nimg, int phase, int px,
                                                    int w, int w_end, SweepWords<N> &W, int i, unsigned &rw) {
  unsigned word = 0u;
  int ii = 0, row = 0, col0 = 0;
  rw = 0u;
  if (w < w_end) {
    if (kBatch) {  // the image: the last one whose class words start at or before w
      int lo = 0, hi = nimg - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].cw0[phase] <= w) lo = mid;
        else hi = mid - 1;
      }
      ii = lo;
    }
    if (active[ii]) {  // (an image that finished the stage is not visited again)
      const ImageDesc &im = kBatch ? imgs[ii] : a.img0;
      word = a.cbits[w];
      rw = a.rbits[w];
      const int wpr = class_wpr(im.nbx, px);
      const int local = w - im.cw0[phase];
      row = local / wpr;
      col0 = (local - row * wpr) * 32;
    }
  }
  W.bits[i] = word;
  W.clr[i] = 0u;
  W.req[i] = rw;
  W.img[i] = ii;
  W.row[i] = row;
  W.col0[i] = col0;
  return word;
}

// Tests of up to kPer set bits of W (entries e0 + u * stride, u < kPer, below total): their
// window loads, then their flag loads, are issued together.  dec[u]: the block needs a
// decision (its word << 5 | bit in code[u]).
template <bool kBatch, int N>
__device__ __forceinline__ void sweep_tests(const StageArgs &a, const ImageDesc *imgs, const unsigned char *pruned,
                                            const int *valid_from, SweepWords<N> &W, int e0, int stride, int total,
                                            int px, int py, int g, int sweep, bool dec[kPer], int code[kPer],
                                            Local &lc, int *s_cnt, int &cur, int &visited, int &skipped) {
  const DevStats &s = a.st;
  const int prev2 = 2 * (g - 9);  // stamps >= this changed since the class's previous phase
  int qv[kPer], bv[kPer], xv[kPer], yv[kPer];
  int L[kPer][9];  // label, N, W, E, S, NW, NE, SE, SW (-1 outside the grid)
  bool okv[kPer];
#pragma unroll
  for (int u = 0; u < kPer; u++) {
    const int e = e0 + u * stride;
    okv[u] = false;
    dec[u] = false;
    qv[u] = bv[u] = xv[u] = yv[u] = 0;
    if (e < total) {
      const int q = word_of_entry(W, e);
      const unsigned wq = W.bits[q];
      const int b = select_bit(wq, e - (W.pre[q] - __popc(wq)));
      const ImageDesc &im = kBatch ? imgs[W.img[q]] : a.img0;
      qv[u] = q;
      bv[u] = b;
      xv[u] = px + 3 * (W.col0[q] + b);
      yv[u] = py + 3 * W.row[q];
      if (xv[u] >= im.nbx) atomicOr(&W.clr[q], 1u << b);  // a bit past the row's last column: no block
      else okv[u] = true;
    }
  }
#pragma unroll
  for (int u = 0; u < kPer; u++) {
    if (!okv[u]) continue;
    const ImageDesc &im = kBatch ? imgs[W.img[qv[u]]] : a.img0;
    load_window(im, xv[u], yv[u], L[u]);
  }
#pragma unroll
  for (int u = 0; u < kPer; u++) {  // what the tests and the skip check read next
    if (!okv[u]) continue;
    if (a.imp_on) prefetch_l1(s.imp + L[u][0]);
#pragma unroll
    for (int t = 0; t < 5; t++)
      if (L[u][t] >= 0) prefetch_l1(s.chg + L[u][t]);
  }
#pragma unroll
  for (int u = 0; u < kPer; u++) {
    code[u] = (qv[u] << 5) | bv[u];
    if (!okv[u]) continue;
    const int q = qv[u], qi = W.img[q];
    const unsigned bit = 1u << bv[u];
    const ImageDesc &im = kBatch ? imgs[qi] : a.img0;
    if (kBatch && qi != cur) {
      flush_sweep_counts(s_cnt, cur, lc, visited, skipped);
      cur = qi;
    }
    visited++;
    const int *l = L[u];
    const int el0 = lc.elig;
    const unsigned char *mask = pruned[qi] ? im.mask : nullptr;
    const long long idx = (long long)yv[u] * im.nbx + xv[u];
    const bool need = block_tests(a, l[0], l[1], l[2], l[3], l[4], l[5], l[6], l[7], l[8], mask, idx, lc);
    if (lc.elig == el0) atomicOr(&W.clr[q], bit);  // not eligible: off the bitmap
    const bool memo = (W.req[q] & bit) != 0;
    if (memo) atomicAnd(&W.req[q], ~bit);  // set again if it requests again
    if (need) {
      bool same = a.skip_tiles && sweep > 0 && g - 9 >= valid_from[qi] && !memo;
      if (same) {
#pragma unroll
        for (int t = 0; t < 5; t++)
          if (l[t] >= 0) same &= s.chg[l[t]] < prev2;
      }
      if (same) skipped++;
      else dec[u] = true;
    }
  }
}

// The decision of the block listed as `code` (word << 5 | bit of W).
template <bool kBatch, int kSched, int N>
__device__ __forceinline__ void sweep_decide(const StageArgs &a, const ImageDesc *imgs, SweepWords<N> &W, int code,
                                             int px, int py, int g, Local &lc, int *s_cnt, int &cur, int &visited,
                                             int &skipped) {
  const DevStats &s = a.st;
  const int q = code >> 5, b = code & 31, qi = W.img[q];
  const ImageDesc &im = kBatch ? imgs[qi] : a.img0;
  if (kBatch && qi != cur) {
    flush_sweep_counts(s_cnt, cur, lc, visited, skipped);
    cur = qi;
  }
  const int bx = px + 3 * (W.col0[q] + b), by = py + 3 * W.row[q];
  const long long idx = (long long)by * im.nbx + bx;
  const int *lab = im.lab;
  const int lbl = lab[idx];
  const int nN = by > 0 ? lab[idx - im.nbx] : -1, nS = by + 1 < im.nby ? lab[idx + im.nbx] : -1;
  const int nW = bx > 0 ? lab[idx - 1] : -1, nE = bx + 1 < im.nbx ? lab[idx + 1] : -1;
  // the decision's reads (snapshot means, counts, the block's pixels), fetched together
  const int nb5[5] = {lbl, nN, nW, nE, nS};
#pragma unroll
  for (int t = 0; t < 5; t++)
    if (nb5[t] >= 0 && (t == 0 || nb5[t] != lbl)) {
      prefetch_l1(s.fhi + nb5[t]);
      prefetch_l1(s.flo + nb5[t]);
      prefetch_l1(s.fy + nb5[t]);
    }
  prefetch_l1(s.mN + lbl);
  prefetch_l1(s.init + lbl);
  if (a.f == 1) prefetch_l1(im.img + (long long)by * a.side * im.img_pitch + 3ll * bx * a.side);
  const int m0 = lc.moves;
  if (decide_block_at<kSched>(a, im, lbl, nN, nW, nE, nS, bx, by, g, lc)) atomicOr(&W.req[q], 1u << b);
  if (lc.moves != m0) sweep_mark_plus(a, im, bx, by, false);
}

// Warp walk (the better one for sparse classes): the class's words are split
// into equal contiguous ranges, one per warp of the grid.  A warp loads up to 32 words at a
// time (a lane each), spreads their set bits over its lanes and gives each lane kPer blocks
// at a time: tests, then the decisions, shared out again one per lane.  Warps never wait on
// one another.
template <bool kBatch, int kSched>
__device__ __forceinline__ void eval_sweep_warp(const StageArgs &a, const ImageDesc *imgs, const unsigned char *active,
                                                const unsigned char *pruned, const int *valid_from, WarpTile *wts,
                                                int *s_cnt, int phase, int g, int sweep, Local &lc, int &cur,
                                                int &visited, int &skipped) {
  const int nimg = kBatch ? a.nimg : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpSweep &X = *reinterpret_cast<WarpSweep *>(&wts[warp]);
  const int py = phase / 3, px = phase % 3;
  const int w_first = a.cwb[phase];
  const long long nw = (long long)a.cwb[phase + 1] - w_first;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  const int wb = w_first + (int)(nw * gw / nwarps), we = w_first + (int)(nw * (gw + 1) / nwarps);
  for (int base = wb; base < we; base += 32) {
    const int w = base + lane;
    unsigned rw;
    const unsigned word = sweep_load_word<kBatch>(a, imgs, active, nimg, phase, px, w, we, X.w, lane, rw);
    int pre = __popc(word);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += v;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    if (total == 0) continue;  // (warp-uniform)
    X.w.pre[lane] = pre;
    __syncwarp();
    for (int c0 = 0; c0 < total; c0 += 32 * kPer) {
      bool dec[kPer];
      int code[kPer];
      sweep_tests<kBatch>(a, imgs, pruned, valid_from, X.w, c0 + lane, 32, total, px, py, g, sweep, dec, code, lc,
                          s_cnt, cur, visited, skipped);
      int nd = 0;
#pragma unroll
      for (int u = 0; u < kPer; u++) {
        const unsigned bal = __ballot_sync(0xffffffffu, dec[u]);
        if (dec[u]) X.dec[nd + __popc(bal & ((1u << lane) - 1u))] = code[u];
        nd += __popc(bal);
      }
      __syncwarp();
      for (int d = lane; d < nd; d += 32)
        sweep_decide<kBatch, kSched>(a, imgs, X.w, X.dec[d], px, py, g, lc, s_cnt, cur, visited, skipped);
      __syncwarp();
    }
    if (w < we && word) {
      const unsigned c = X.w.clr[lane];
      if (c) atomicAnd(a.cbits + w, ~c);
      if (X.w.req[lane] != rw) a.rbits[w] = X.w.req[lane];
    }
    __syncwarp();
  }
}

// CTA walk (the better one for dense classes): the class's words
// are cut into chunks of 32, dealt to the CTAs in turn (chunk c to CTA c mod grid, so
// every CTA samples the whole image and the CTAs' shares of set bits even out).  A CTA
// takes one chunk per warp at a time (a word per lane), spreads the set bits of all its
// words evenly over its threads (CTA-wide prefix sums) for the tests, and then spreads the
// blocks that need a decision evenly over its threads again, so no warp waits long on a
// busier warp's chain.  Costs a few CTA barriers per round, which a sparse class does not
// repay.
template <bool kBatch, int kSched>
__device__ __forceinline__ void eval_sweep_cta(const StageArgs &a, const ImageDesc *imgs, const unsigned char *active,
                                               const unsigned char *pruned, const int *valid_from, WarpTile *wts,
                                               int *s_cnt, int phase, int g, int sweep, Local &lc, int &cur,
                                               int &visited, int &skipped) {
  const int nimg = kBatch ? a.nimg : 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kThreads / 32;
  CtaSweep &X = *reinterpret_cast<CtaSweep *>(wts);
  const int py = phase / 3, px = phase % 3;
  const int w_first = a.cwb[phase], w_end = a.cwb[phase + 1];
  const int nchunks = (w_end - w_first + 31) >> 5;
  const int grid = gridDim.x;
  __syncthreads();  // (the scratch overlays the warp tiles)
  for (int r = 0; (long long)r * kWarps * grid + blockIdx.x < nchunks; r++) {
    // this warp's chunk in round r: the CTA's (r * kWarps + warp)-th
    const long long chunk = ((long long)r * kWarps + warp) * grid + blockIdx.x;
    const int w = chunk < nchunks ? w_first + (int)chunk * 32 + lane : w_end;
    unsigned rw;
    const unsigned word = sweep_load_word<kBatch>(a, imgs, active, nimg, phase, px, w, w_end, X.w, tid, rw);
    int pre = __popc(word);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += v;
    }
    if (lane == 31) X.wsum[warp] = pre;
    __syncthreads();
    if (warp == 0) {  // exclusive prefix sums of the warps' counts
      const int v = lane < kWarps ? X.wsum[lane] : 0;
      int inc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
      }
      if (lane < kWarps) X.wsum[lane] = inc - v;
      if (lane == 31) {
        X.total = inc;
        X.ndec[0] = 0;
      }
    }
    __syncthreads();
    X.w.pre[tid] = pre + X.wsum[warp];
    const int total = X.total;
    __syncthreads();
    if (total == 0) continue;  // (CTA-uniform)
    for (int c0 = 0, it = 0; c0 < total; c0 += kThreads * kPer, it ^= 1) {
      bool dec[kPer];
      int code[kPer];
      sweep_tests<kBatch>(a, imgs, pruned, valid_from, X.w, c0 + tid, kThreads, total, px, py, g, sweep, dec, code,
                          lc, s_cnt, cur, visited, skipped);
#pragma unroll
      for (int u = 0; u < kPer; u++) {  // list the blocks that need a decision (one reservation per warp)
        const unsigned bal = __ballot_sync(0xffffffffu, dec[u]);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&X.ndec[it], __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (dec[u]) X.dec[base + __popc(bal & ((1u << lane) - 1u))] = code[u];
      }
      __syncthreads();
      const int nd = X.ndec[it];
      if (tid == 0) X.ndec[it ^ 1] = 0;  // the next batch's list (no thread reads it before the barrier below)
      for (int d = tid; d < nd; d += kThreads)
        sweep_decide<kBatch, kSched>(a, imgs, X.w, X.dec[d], px, py, g, lc, s_cnt, cur, visited, skipped);
      __syncthreads();
    }
    if (w < w_end && word) {  // this thread's word, as the round leaves it
      const unsigned c = X.w.clr[tid];
      if (c) atomicAnd(a.cbits + w, ~c);
      if (X.w.req[tid] != rw) a.rbits[w] = X.w.req[tid];
    }
  }
}

// Phase `phase` (class py = phase / 3, px = phase % 3) of sweep `sweep`; g is the phase
// number in the launch.  A build carries one of the two walks (kSweepCta, chosen per
// translation unit), so the launch-geometry tuner picks the walk per stage along with the
// build; either gives the same results.
template <bool kBatch, int kSched>
__device__ __forceinline__ void eval_sweep(const StageArgs &a, const ImageDesc *imgs, const unsigned char *active,
                                           const unsigned char *pruned, const int *valid_from, WarpTile *wts,
                                           int *s_cnt, int phase, int g, int slot, int sweep) {
  const int nimg = kBatch ? a.nimg : 1;
  for (int i = threadIdx.x; i < nimg * 8; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  Local lc = {0, 0, 0, 0, 0, 0};
  int cur = 0, visited = 0, skipped = 0;
  if constexpr (kSweepCta)
    eval_sweep_cta<kBatch, kSched>(a, imgs, active, pruned, valid_from, wts, s_cnt, phase, g, sweep, lc, cur,
                                   visited, skipped);
  else
    eval_sweep_warp<kBatch, kSched>(a, imgs, active, pruned, valid_from, wts, s_cnt, phase, g, sweep, lc, cur,
                                    visited, skipped);
  flush_sweep_counts(s_cnt, cur, lc, visited, skipped);
  __syncthreads();
  store_sweep_counts(a, s_cnt, nimg, slot);
}
