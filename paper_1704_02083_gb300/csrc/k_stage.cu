// k_stage.cu — one stage of the refinement (Sec. 2.1, Algorithm RAPID's queue loop) as a
// single cooperative launch: sweeps of 9 phases until a sweep changes nothing.
//
// Phase (py, px) evaluates the blocks with by % 3 == py and bx % 3 == px.  Two such
// blocks are at least 3 apart, so their 3x3 windows are disjoint: every block of a phase
// decides from labels no other block of the phase writes, their boundary pairs are
// disjoint, and each topology test stays valid when the others move.  Decisions use a
// snapshot of the statistics S taken when the phase starts; moves update the label map
// in place and accumulate exact int64 deltas that are folded into S after the phase.
// Merge requests of the phase (size bound hit, Sec. 3.1) are then resolved against the
// post-move state.
#include <climits>

#include "rapid_dev.cuh"

namespace rapid {

static constexpr int kThreads = 256;

struct Local {
  long long elig, eval, moves, req;
};

// Decide one block (Eq. bound, E_topo, Eq. operation, size term) and apply its move.
__device__ __forceinline__ void eval_block(const StageArgs &a, int bx, int by, Local &lc,
                                           unsigned long long *changes) {
  const int nbx = a.nbx, nby = a.nby;
  const int *L = a.lab;
  const long long idx = (long long)by * nbx + bx;
  const int lbl = L[idx];
  const bool hasN = by > 0, hasS = by + 1 < nby, hasW = bx > 0, hasE = bx + 1 < nbx;
  const int nN = hasN ? L[idx - nbx] : -1;
  const int nW = hasW ? L[idx - 1] : -1;
  const int nE = hasE ? L[idx + 1] : -1;
  const int nS = hasS ? L[idx + nbx] : -1;
  const bool boundary = (nN >= 0 && nN != lbl) || (nW >= 0 && nW != lbl) || (nE >= 0 && nE != lbl) ||
                        (nS >= 0 && nS != lbl);
  if (!boundary) return;
  if (a.imp_on) {
    if (a.imp_rule == 0) {
      if (!a.st.imp[lbl]) return;
    } else {
      const signed char ya = a.st.y[lbl];
      bool any = (nN >= 0 && nN != lbl && a.st.y[nN] != ya) || (nW >= 0 && nW != lbl && a.st.y[nW] != ya) ||
                 (nE >= 0 && nE != lbl && a.st.y[nE] != ya) || (nS >= 0 && nS != lbl && a.st.y[nS] != ya);
      if (!any) return;
    }
  }
  lc.elig++;
  const int nNW = (hasN && hasW) ? L[idx - nbx - 1] : -1;
  const int nNE = (hasN && hasE) ? L[idx - nbx + 1] : -1;
  const int nSE = (hasS && hasE) ? L[idx + nbx + 1] : -1;
  const int nSW = (hasS && hasW) ? L[idx + nbx - 1] : -1;
  unsigned m = (unsigned)(nNW == lbl) | ((unsigned)(nN == lbl) << 1) | ((unsigned)(nNE == lbl) << 2) |
               ((unsigned)(nE == lbl) << 3) | ((unsigned)(nSE == lbl) << 4) | ((unsigned)(nS == lbl) << 5) |
               ((unsigned)(nSW == lbl) << 6) | ((unsigned)(nW == lbl) << 7);
  if (!simple_mask(m)) return;
  lc.eval++;

  const BlockSums bs = block_sums(a, bx, by);
  const double w = __ll2double_rn(bs.w);
  const double r2 = __ll2double_rn(2 * bs.r), g2 = __ll2double_rn(2 * bs.g), b2 = __ll2double_rn(2 * bs.b);
  const double x2 = __ll2double_rn(2 * bs.x), y2 = __ll2double_rn(2 * bs.y);
  const int nb[4] = {nN, nW, nE, nS};
  const int len[4] = {bs.bw, bs.bh, bs.bh, bs.bw};
  const DevStats &s = a.st;

  long long Ba = 0;
#pragma unroll
  for (int j = 0; j < 4; j++)
    if (nb[j] >= 0 && nb[j] != lbl) Ba += len[j];
  const double ea = blk_energy(w, r2, g2, b2, x2, y2, s.mR[lbl], s.mG[lbl], s.mB[lbl], s.mX[lbl], s.mY[lbl],
                               __ll2double_rn(Ba), a.lam_pos, a.lam_b2);
  int bestk = -1;
  double best = 0.0;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const int k = nb[j];
    if (k < 0 || k == lbl) continue;
    bool dup = false;
#pragma unroll
    for (int i = 0; i < j; i++) dup |= (nb[i] == k);
    if (dup) continue;
    long long Bk = 0;
#pragma unroll
    for (int i = 0; i < 4; i++)
      if (nb[i] >= 0 && nb[i] != k) Bk += len[i];
    const double ek = blk_energy(w, r2, g2, b2, x2, y2, s.mR[k], s.mG[k], s.mB[k], s.mX[k], s.mY[k],
                                 __ll2double_rn(Bk), a.lam_pos, a.lam_b2);
    const double dE = __dsub_rn(ek, ea);
    if (bestk < 0 || dE < best || (dE == best && k < bestk)) {
      best = dE;
      bestk = k;
    }
  }
  if (bestk < 0 || !(best < 0.0)) return;
  if (a.size_mode != 0 && (long long)a.lo_den * (s.N[lbl] - bs.w) < (long long)a.lo_num * s.init[lbl]) {
    if (a.size_mode == 2) {
      lc.req++;
      atomicMin(&a.mg.req_min[lbl], (int)idx);
      if (atomicExch(&a.mg.req_flag[lbl], 1) == 0) {
        const int slot = atomicAdd(a.mg.req_count, 1);
        a.mg.req_list[slot] = lbl;
      }
    }
    return;
  }
  // Move: relabel in place, accumulate the exact deltas of both labels.
  a.lab[idx] = bestk;
  atomic_add_i64(&s.dN[lbl], -bs.w);
  atomic_add_i64(&s.dR[lbl], -bs.r);
  atomic_add_i64(&s.dG[lbl], -bs.g);
  atomic_add_i64(&s.dB[lbl], -bs.b);
  atomic_add_i64(&s.dX[lbl], -bs.x);
  atomic_add_i64(&s.dY[lbl], -bs.y);
  atomic_add_i64(&s.dN[bestk], bs.w);
  atomic_add_i64(&s.dR[bestk], bs.r);
  atomic_add_i64(&s.dG[bestk], bs.g);
  atomic_add_i64(&s.dB[bestk], bs.b);
  atomic_add_i64(&s.dX[bestk], bs.x);
  atomic_add_i64(&s.dY[bestk], bs.y);
  s.dirty[lbl] = 1;
  s.dirty[bestk] = 1;
  const int x0 = bx * a.side, y0 = by * a.side;
  atomicMin(&s.bbox[bestk].x, x0);
  atomicMin(&s.bbox[bestk].y, y0);
  atomicMax(&s.bbox[bestk].z, x0 + bs.bw - 1);
  atomicMax(&s.bbox[bestk].w, y0 + bs.bh - 1);
  lc.moves++;
  (void)changes;
}

__device__ inline long long warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ void eval_phase(const StageArgs &a, int phase, unsigned long long *changes) {
  const int py = phase / 3, px = phase % 3;
  Local lc = {0, 0, 0, 0};
  if (a.nbx > px && a.nby > py) {
    const long long nphx = (a.nbx - px + 2) / 3, nphy = (a.nby - py + 2) / 3;
    const long long total = nphx * nphy;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
      const int bx = px + 3 * (int)(i % nphx);
      const int by = py + 3 * (int)(i / nphx);
      eval_block(a, bx, by, lc, changes);
    }
  }
  const long long e = warp_sum(lc.elig), v = warp_sum(lc.eval), m = warp_sum(lc.moves), r = warp_sum(lc.req);
  if ((threadIdx.x & 31) == 0) {
    if (e) atomic_add_i64(&a.ctl.cnt[CNT_ELIG], e);
    if (v) atomic_add_i64(&a.ctl.cnt[CNT_EVAL], v);
    if (m) {
      atomic_add_i64(&a.ctl.cnt[CNT_MOVES], m);
      atomicAdd(changes, (unsigned long long)m);
    }
    if (r) atomic_add_i64(&a.ctl.cnt[CNT_REQ], r);
  }
}

// Fold the phase's deltas into S and refresh the snapshot means of changed labels.
__device__ void commit_phase(const StageArgs &a) {
  const DevStats &s = a.st;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < s.M; k += gridDim.x * blockDim.x) {
    if (!s.dirty[k]) continue;
    s.dirty[k] = 0;
    s.N[k] += s.dN[k];
    s.R[k] += s.dR[k];
    s.G[k] += s.dG[k];
    s.B[k] += s.dB[k];
    s.X[k] += s.dX[k];
    s.Y[k] += s.dY[k];
    s.dN[k] = s.dR[k] = s.dG[k] = s.dB[k] = s.dX[k] = s.dY[k] = 0;
    set_means(s, k);
  }
}

// Merge targets (Eqs. eqa:merge, condtion), one CTA per requested label: over the labels
// 4-adjacent to it (found by scanning its bounding box, which always contains it), the
// least merge cost among those that stay within u * InitSize; ties to the smaller id.
__device__ void merge_targets(const StageArgs &a, int rq) {
  __shared__ double sw[kThreads];
  __shared__ int sn[kThreads];
  const DevStats &s = a.st;
  for (int j = blockIdx.x; j < rq; j += gridDim.x) {
    const int al = a.mg.req_list[j];
    const int4 bb = s.bbox[al];
    const int bx0 = bb.x / a.side, bx1 = bb.z / a.side, by0 = bb.y / a.side, by1 = bb.w / a.side;
    const int bw = bx1 - bx0 + 1;
    const long long total = (long long)bw * (by1 - by0 + 1);
    double best = 0.0;
    int bestn = INT_MAX;
    for (long long t = threadIdx.x; t < total; t += blockDim.x) {
      const int cx = bx0 + (int)(t % bw), cy = by0 + (int)(t / bw);
      const long long idx = (long long)cy * a.nbx + cx;
      if (a.lab[idx] != al) continue;
      int nbv[4];
      nbv[0] = cy > 0 ? a.lab[idx - a.nbx] : -1;
      nbv[1] = cx > 0 ? a.lab[idx - 1] : -1;
      nbv[2] = cx + 1 < a.nbx ? a.lab[idx + 1] : -1;
      nbv[3] = cy + 1 < a.nby ? a.lab[idx + a.nbx] : -1;
      for (int q = 0; q < 4; q++) {
        const int n = nbv[q];
        if (n < 0 || n == al) continue;
        if ((long long)a.hi_den * (s.N[n] + s.N[al]) > (long long)a.hi_num * s.init[n]) continue;
        const double wv = ward_cost(s, al, n, a.lam_pos);
        if (bestn == INT_MAX || wv < best || (wv == best && n < bestn)) {
          best = wv;
          bestn = n;
        }
      }
    }
    sw[threadIdx.x] = best;
    sn[threadIdx.x] = bestn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
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
    if (threadIdx.x == 0) a.mg.target[al] = sn[0] == INT_MAX ? -1 : sn[0];
    __syncthreads();
  }
}

// Accept requests in ascending order of their first requesting block; skip those whose
// source or target already merged in this phase; fold S.  Runs on CTA 0 only.
__device__ void merge_accept(const StageArgs &a, int rq, unsigned long long *changes) {
  const DevStats &s = a.st;
  const DevMerge &g = a.mg;
  for (int j = threadIdx.x; j < rq; j += blockDim.x) {
    const int key = g.req_min[g.req_list[j]];
    int rank = 0;
    for (int i = 0; i < rq; i++) rank += g.req_min[g.req_list[i]] < key;
    g.order[rank] = g.req_list[j];
  }
  __syncthreads();
  __threadfence_block();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int r = 0; r < rq; r++) {
      const int al = g.order[r];
      const int n = g.target[al];
      if (n < 0 || g.involved[al] || g.involved[n]) continue;
      g.involved[al] = 1;
      g.involved[n] = 1;
      g.acc[acc++] = make_int2(al, n);
      s.N[n] += s.N[al];
      s.R[n] += s.R[al];
      s.G[n] += s.G[al];
      s.B[n] += s.B[al];
      s.X[n] += s.X[al];
      s.Y[n] += s.Y[al];
      s.N[al] = s.R[al] = s.G[al] = s.B[al] = s.X[al] = s.Y[al] = 0;
      set_means(s, n);
      set_means(s, al);
      int4 bn = s.bbox[n];
      const int4 ba = s.bbox[al];
      bn.x = min(bn.x, ba.x);
      bn.y = min(bn.y, ba.y);
      bn.z = max(bn.z, ba.z);
      bn.w = max(bn.w, ba.w);
      s.bbox[n] = bn;
    }
    *g.acc_count = acc;
    *g.req_count = 0;
    if (acc) {
      a.ctl.cnt[CNT_MERGES] += acc;
      *changes += (unsigned long long)acc;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < rq; j += blockDim.x) {
    const int al = g.req_list[j];
    g.req_flag[al] = 0;
    g.req_min[al] = INT_MAX;
    g.target[al] = -1;
  }
  const int nacc = *(volatile int *)g.acc_count;
  for (int j = threadIdx.x; j < nacc; j += blockDim.x) {
    const int2 p = g.acc[j];
    g.involved[p.x] = 0;
    g.involved[p.y] = 0;
  }
}

// Relabel accepted merges a -> n over a's bounding box, one CTA per merge.
__device__ void merge_relabel(const StageArgs &a, int nacc) {
  for (int j = blockIdx.x; j < nacc; j += gridDim.x) {
    const int2 p = a.mg.acc[j];
    const int4 bb = a.st.bbox[p.x];
    const int bx0 = bb.x / a.side, bx1 = bb.z / a.side, by0 = bb.y / a.side, by1 = bb.w / a.side;
    const int bw = bx1 - bx0 + 1;
    const long long total = (long long)bw * (by1 - by0 + 1);
    for (long long t = threadIdx.x; t < total; t += blockDim.x) {
      const long long idx = (long long)(by0 + (int)(t / bw)) * a.nbx + bx0 + (int)(t % bw);
      if (a.lab[idx] == p.x) a.lab[idx] = p.y;
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

__global__ void __launch_bounds__(kThreads) stage_kernel(StageArgs a) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.st.M; k += gridDim.x * blockDim.x) set_means(a.st, k);
  if (!grid_sync(a.ctl)) return;
  Timer tm(a.ctl.prof);
  for (int sweep = 0; sweep < a.max_sweeps; sweep++) {
    unsigned long long *changes = &a.ctl.changes[sweep % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl.changes[(sweep + 1) % 3] = 0;
    for (int ph = 0; ph < 9; ph++) {
      eval_phase(a, ph, changes);
      tm.lap(PROF_EVAL);
      if (!grid_sync(a.ctl)) return;
      tm.lap(PROF_SYNC1);
      const int rq = ld_volatile_i32(a.mg.req_count);
      commit_phase(a);
      tm.lap(PROF_COMMIT);
      if (!grid_sync(a.ctl)) return;
      tm.lap(PROF_SYNC2);
      if (rq > 0) {
        merge_targets(a, rq);
        if (!grid_sync(a.ctl)) return;
        if (blockIdx.x == 0) merge_accept(a, rq, changes);
        if (!grid_sync(a.ctl)) return;
        merge_relabel(a, ld_volatile_i32(a.mg.acc_count));
        if (!grid_sync(a.ctl)) return;
        tm.lap(PROF_MERGE);
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl.cnt[CNT_SWEEPS] += 1;
    if (ld_volatile_u64(changes) == 0) break;
  }
}

int stage_block_threads() { return kThreads; }
const void *stage_kernel_ptr() { return (const void *)stage_kernel; }

cudaError_t launch_stage(const StageArgs &a, int grid, int block, cudaStream_t s) {
  StageArgs copy = a;
  void *args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void *)stage_kernel, dim3(grid), dim3(block), args, 0, s);
}

}  // namespace rapid
