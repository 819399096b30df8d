// air_refine.cu -- the adaptive image (Parkin 2010, Section 2 steps iii-vi):
// truncation-error scan (Section 3, Eq. 2), 2:1 level balance between adjacent
// pixels, quadtree refinement with a warp-ballot prefix sum that compacts the
// new rays, and the leaf output with the band flux.
//
// The image quadtree is a node list: the base image row-major (node j*n0 + i),
// then four consecutive children per refined node, in the order of the
// parents. Each node stores its level, (i, j) at that level and the index of
// its first child (-1 for a leaf). The pixel at level L holding (i, j) is
// found by descending from the base node through the child links; this gives
// the deepest existing node at a level <= L, which is the value a missing
// neighbour takes in the stencil.
#include <atomic>
#include <cfloat>

#include "air_tree.cuh"

namespace air {

// Step iii: flag every leaf below max_level whose xi >= xi_crit.
// ---- warp-ballot prefix sums ------------------------------------------------
// A block covers kScanItems = kScanRounds * kScanBlock consecutive items;
// round r holds items [r * kScanBlock, (r + 1) * kScanBlock) of the block, one
// per thread, so every load is coalesced and the block-local order is the
// global order.

struct PredFlag {
  const uint32_t *flag;
  __device__ bool operator()(int64_t k) const { return flag[k] != 0; }
};
struct PredLeaf {
  const int32_t *child;
  int all;
  __device__ bool operator()(int64_t k) const { return all || child[k] < 0; }
};

template <class Pred>
__global__ void __launch_bounds__(kScanBlock) k_count(Pred pred, int64_t n, int32_t *bcount) {
  __shared__ int32_t wsum[kScanBlock / 32];
  const int64_t start = (int64_t)blockIdx.x * kScanItems;
  int32_t cnt = 0;
  for (int rr = 0; rr < kScanRounds; ++rr) {
    const int64_t k = start + (int64_t)rr * kScanBlock + threadIdx.x;
    const bool p = k < n && pred(k);
    cnt += __popc(__ballot_sync(0xffffffffu, p));
  }
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t s = 0;
    for (int w = 0; w < kScanBlock / 32; ++w) s += wsum[w];
    bcount[blockIdx.x] = s;
  }
}

// Exclusive scan of the per-block counts in one block; total -> *total.
__global__ void __launch_bounds__(1024) k_scan_blocks(const int32_t *bcount, int64_t nb,
                                                      int64_t *boff, int64_t *total) {
  __shared__ int64_t part[1024];
  const int64_t per = (nb + 1023) / 1024;
  const int64_t a = threadIdx.x * per, b = min(nb, a + per);
  int64_t s = 0;
  for (int64_t x = a; x < b; ++x) s += bcount[x];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int64_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - s;
  for (int64_t x = a; x < b; ++x) {
    boff[x] = run;
    run += bcount[x];
  }
  if (threadIdx.x == 1023) *total = part[1023];
}

// ---- open-leaf list -----------------------------------------------------------
// The leaves below the top level, in ascending node order: the only nodes a
// sweep can flag. Steps iii and iv run over this list instead of every node;
// children are still emitted in parent (node) order, so the quadtree is the
// same. Flags of nodes outside the list are kept at zero (a refined node's
// flag is cleared when its children are emitted, children start at zero).

// Level-map entries of the four children (first index c0, level l) of the
// level-(l - 1) pixel (i, j); only levels l < Lm have maps.
__device__ __forceinline__ void set_level_map(int32_t *lmap, int n0, int l, int i, int j,
                                              int64_t c0) {
  const int64_t nl = (int64_t)n0 << l;
  int32_t *row = lmap + level_map_offset(n0, l) + (int64_t)(2 * j) * nl + 2 * i;
  row[0] = (int32_t)c0;
  row[1] = (int32_t)(c0 + 1);
  row[nl] = (int32_t)(c0 + 2);
  row[nl + 1] = (int32_t)(c0 + 3);
}

__global__ void k_iota(int32_t *list, int64_t m) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) list[i] = (int32_t)i;
}

__global__ void k_xi_scan_list(TreeView t, const int32_t *__restrict__ open, int64_t m,
                               double xi_crit, int xi_norm, int refine_on,
                               uint32_t *__restrict__ flag, const int32_t *lmap) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t k = open[i];
  flag[k] = xi_flag(t, NodeLookup{0, lmap}, k, xi_crit, xi_norm, refine_on);
}

__global__ void k_balance_list(TreeView t, const int32_t *__restrict__ open, int64_t m,
                               uint32_t *__restrict__ flag, uint32_t *__restrict__ err,
                               const int32_t *lmap) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const int k = open[i];
    if (flag[k] != 0) balance_from(t, NodeLookup{0, lmap}, k, flag, err);
  }
}

// Three selections over the list, per entry k = open[i]: flagged (refined
// this sweep), kept (not flagged: stays an open leaf), and flagged with
// children below the top level (its four children join the list).
struct ListSel {
  bool f, keep, co;
};
__device__ __forceinline__ ListSel list_sel(const TreeView &t, const int32_t *open, int64_t m,
                                            const uint32_t *flag, int Lm, int64_t i, int &k) {
  ListSel q{false, false, false};
  k = 0;
  if (i < m) {
    k = open[i];
    q.f = flag[k] != 0;
    q.keep = !q.f;
    q.co = q.f && t.lvl[k] + 1 < Lm;
  }
  return q;
}

__global__ void __launch_bounds__(kScanBlock) k_count3(TreeView t, const int32_t *open, int64_t m,
                                                       const uint32_t *flag, int Lm,
                                                       int32_t *bcount, int64_t nb) {
  __shared__ int32_t wsum[3][kScanBlock / 32];
  const int64_t start = (int64_t)blockIdx.x * kScanItems;
  int32_t c0 = 0, c1 = 0, c2 = 0;
  for (int rr = 0; rr < kScanRounds; ++rr) {
    int k;
    const ListSel q = list_sel(t, open, m, flag, Lm, start + (int64_t)rr * kScanBlock + threadIdx.x, k);
    c0 += __popc(__ballot_sync(0xffffffffu, q.f));
    c1 += __popc(__ballot_sync(0xffffffffu, q.keep));
    c2 += __popc(__ballot_sync(0xffffffffu, q.co));
  }
  if ((threadIdx.x & 31) == 0) {
    wsum[0][threadIdx.x >> 5] = c0;
    wsum[1][threadIdx.x >> 5] = c1;
    wsum[2][threadIdx.x >> 5] = c2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    int32_t s = 0;
    for (int w = 0; w < kScanBlock / 32; ++w) s += wsum[threadIdx.x][w];
    bcount[threadIdx.x * nb + blockIdx.x] = s;
  }
}

// Block b of the launch scans selection b's per-block counts.
__global__ void __launch_bounds__(1024) k_scan_blocks3(const int32_t *bcount, int64_t nb,
                                                       int64_t *boff, int64_t *total) {
  __shared__ int64_t part[1024];
  const int32_t *bc = bcount + blockIdx.x * nb;
  int64_t *bo = boff + blockIdx.x * nb;
  const int64_t per = (nb + 1023) / 1024;
  const int64_t a = threadIdx.x * per, b = min(nb, a + per);
  int64_t s = 0;
  for (int64_t x = a; x < b; ++x) s += bc[x];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int64_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - s;
  for (int64_t x = a; x < b; ++x) {
    bo[x] = run;
    run += bc[x];
  }
  if (threadIdx.x == 1023) total[blockIdx.x] = part[1023];
}

// Step iv over the list, and the next list: kept entries first (in order),
// then the children below the top level (in order).
__global__ void __launch_bounds__(kScanBlock) k_emit3(TreeView t, const int32_t *open, int64_t m,
                                                      uint32_t *flag, int Lm, const int64_t *boff,
                                                      const int64_t *total, int64_t nb,
                                                      int64_t n_old, int32_t *next, int32_t *lmap) {
  __shared__ int32_t wsum[3][kScanBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t start = (int64_t)blockIdx.x * kScanItems;
  int64_t run0 = boff[blockIdx.x], run1 = boff[nb + blockIdx.x], run2 = boff[2 * nb + blockIdx.x];
  const int64_t keep_total = total[1];
  const uint32_t below = (1u << lane) - 1u;
  for (int rr = 0; rr < kScanRounds; ++rr) {
    int k;
    const ListSel q = list_sel(t, open, m, flag, Lm, start + (int64_t)rr * kScanBlock + threadIdx.x, k);
    const uint32_t b0 = __ballot_sync(0xffffffffu, q.f);
    const uint32_t b1 = __ballot_sync(0xffffffffu, q.keep);
    const uint32_t b2 = __ballot_sync(0xffffffffu, q.co);
    if (lane == 0) {
      wsum[0][warp] = __popc(b0);
      wsum[1][warp] = __popc(b1);
      wsum[2][warp] = __popc(b2);
    }
    __syncthreads();
    int32_t p0 = 0, p1 = 0, p2 = 0, t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
    for (int w = 0; w < kScanBlock / 32; ++w) {
      const int32_t v0 = wsum[0][w], v1 = wsum[1][w], v2 = wsum[2][w];
      p0 += w < warp ? v0 : 0;
      p1 += w < warp ? v1 : 0;
      p2 += w < warp ? v2 : 0;
      t0 += v0;
      t1 += v1;
      t2 += v2;
    }
    if (q.f) {
      const int64_t c0 = n_old + 4 * (run0 + p0 + __popc(b0 & below));
      const int L = t.lvl[k] + 1, i = t.pi[k], j = t.pj[k];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        t.lvl[c0 + c] = (int8_t)L;
        t.pi[c0 + c] = 2 * i + (c & 1);
        t.pj[c0 + c] = 2 * j + (c >> 1);
        t.child[c0 + c] = -1;
        flag[c0 + c] = 0u;
      }
      t.child[k] = (int32_t)c0;
      flag[k] = 0u;
      if (q.co) {
        const int64_t r2 = keep_total + 4 * (run2 + p2 + __popc(b2 & below));
#pragma unroll
        for (int c = 0; c < 4; ++c) next[r2 + c] = (int32_t)(c0 + c);
        if (lmap) set_level_map(lmap, t.n0, L, i, j, c0);
      }
    } else if (q.keep) {
      next[run1 + p1 + __popc(b1 & below)] = k;
    }
    run0 += t0;
    run1 += t1;
    run2 += t2;
    __syncthreads();
  }
}

// ---- the sweep with counts on the device ----------------------------------
// The same steps as above over open[S->cur] with m = S->m items; grids are a
// few blocks per SM and loop over the items (k_count3d and k_emit3d over scan
// chunks of kScanItems, chunk c's counts at bcount[sel * nb_cap + c]).

__global__ void k_xi_scan_dev(TreeView t, const int32_t *__restrict__ open0,
                              const int32_t *__restrict__ open1, const SweepState *__restrict__ S,
                              double xi_crit, int xi_norm, int refine_on,
                              uint32_t *__restrict__ flag, const int32_t *lmap) {
  wait_prior_grid();
  if (S->done) return;
  const int64_t m = S->m;
  const int32_t *open = S->cur ? open1 : open0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const int64_t k = open[i];
    flag[k] = xi_flag(t, NodeLookup{0, lmap}, k, xi_crit, xi_norm, refine_on);
  }
}

// Scan and balance in one pass (counts on the device). Flags of the open
// list are all zero when a sweep starts (a refined node's flag is cleared
// with its children's, new children start at zero), so a thread only ever
// sets flags: a leaf whose xi reaches xi_crit is flagged, and the thread that
// moves a flag from 0 to 1 -- the scan's or a balance expansion's -- expands
// it. Every flag is expanded once, and the flags reach the same closure as a
// scan of every leaf followed by the balance.
__global__ void k_scan_balance_dev(TreeView t, const int32_t *__restrict__ open0,
                                   const int32_t *__restrict__ open1,
                                   const SweepState *__restrict__ S, double xi_crit, int xi_norm,
                                   int refine_on, uint32_t *__restrict__ flag,
                                   uint32_t *__restrict__ err, const int32_t *lmap) {
  wait_prior_grid();
  if (S->done) return;
  const int64_t m = S->m;
  const int32_t *open = S->cur ? open1 : open0;
  const NodeLookup look{0, lmap};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const int k = open[i];
    if (xi_flag(t, look, k, xi_crit, xi_norm, refine_on) && atomicExch(flag + k, 1u) == 0u)
      balance_from(t, look, k, flag, err);
  }
}

__global__ void k_balance_dev(TreeView t, const int32_t *__restrict__ open0,
                              const int32_t *__restrict__ open1, const SweepState *__restrict__ S,
                              uint32_t *__restrict__ flag, uint32_t *__restrict__ err,
                              const int32_t *lmap) {
  wait_prior_grid();
  if (S->done) return;
  const int64_t m = S->m;
  const int32_t *open = S->cur ? open1 : open0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const int k = open[i];
    if (flag[k] != 0) balance_from(t, NodeLookup{0, lmap}, k, flag, err);
  }
}

__global__ void __launch_bounds__(kScanBlock) k_count3d(TreeView t, const int32_t *open0,
                                                        const int32_t *open1,
                                                        const SweepState *__restrict__ S,
                                                        const uint32_t *flag, int32_t *bcount,
                                                        int64_t nb_cap) {
  wait_prior_grid();
  if (S->done) return;
  __shared__ int32_t wsum[3][kScanBlock / 32];
  const int64_t m = S->m;
  const int32_t *open = S->cur ? open1 : open0;
  const int64_t nb = scan_chunks(m);
  for (int64_t c = blockIdx.x; c < nb; c += gridDim.x) {
    const int64_t start = c * kScanItems;
    int32_t c0 = 0, c1 = 0, c2 = 0;
    for (int rr = 0; rr < kScanRounds; ++rr) {
      int k;
      const ListSel q = list_sel(t, open, m, flag, t.Lm, start + (int64_t)rr * kScanBlock + threadIdx.x, k);
      c0 += __popc(__ballot_sync(0xffffffffu, q.f));
      c1 += __popc(__ballot_sync(0xffffffffu, q.keep));
      c2 += __popc(__ballot_sync(0xffffffffu, q.co));
    }
    if ((threadIdx.x & 31) == 0) {
      wsum[0][threadIdx.x >> 5] = c0;
      wsum[1][threadIdx.x >> 5] = c1;
      wsum[2][threadIdx.x >> 5] = c2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      int32_t sum = 0;
      for (int w = 0; w < kScanBlock / 32; ++w) sum += wsum[threadIdx.x][w];
      bcount[threadIdx.x * nb_cap + c] = sum;
    }
    __syncthreads();
  }
}

// Block b scans selection b's chunk counts; totals to S->tot, and block 0
// sets S->done when nothing was flagged (blocks 1 and 2 may then see it and
// return early: their totals are not needed once the loop has ended).
__global__ void __launch_bounds__(1024) k_scan_blocks3d(const int32_t *bcount, int64_t nb_cap,
                                                        int64_t *boff, SweepState *S) {
  wait_prior_grid();
  if (S->done) return;
  __shared__ int64_t part[1024];
  const int64_t nb = scan_chunks(S->m);
  const int32_t *bc = bcount + blockIdx.x * nb_cap;
  int64_t *bo = boff + blockIdx.x * nb_cap;
  const int64_t per = (nb + 1023) / 1024;
  const int64_t a = threadIdx.x * per, b = min(nb, a + per);
  int64_t s = 0;
  for (int64_t x = a; x < b; ++x) s += bc[x];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int64_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - s;
  for (int64_t x = a; x < b; ++x) {
    bo[x] = run;
    run += bc[x];
  }
  if (threadIdx.x == 1023) {
    S->tot[blockIdx.x] = part[1023];
    if (blockIdx.x == 0 && part[1023] == 0) S->done = 1;  // nothing flagged: the loop ends
  }
}

__global__ void __launch_bounds__(kScanBlock) k_emit3d(TreeView t, int32_t *open0,
                                                       int32_t *open1, const SweepState *__restrict__ S,
                                                       uint32_t *flag, const int64_t *boff,
                                                       int64_t nb_cap, int32_t *lmap) {
  wait_prior_grid();
  if (S->done) return;
  __shared__ int32_t wsum[3][kScanBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t m = S->m, n_old = S->n, keep_total = S->tot[1];
  const int32_t *open = S->cur ? open1 : open0;
  int32_t *next = S->cur ? open0 : open1;
  const int64_t nb = scan_chunks(m);
  const uint32_t below = (1u << lane) - 1u;
  for (int64_t c = blockIdx.x; c < nb; c += gridDim.x) {
    const int64_t start = c * kScanItems;
    int64_t run0 = boff[c], run1 = boff[nb_cap + c], run2 = boff[2 * nb_cap + c];
    for (int rr = 0; rr < kScanRounds; ++rr) {
      int k;
      const ListSel q = list_sel(t, open, m, flag, t.Lm, start + (int64_t)rr * kScanBlock + threadIdx.x, k);
      // a flagged node's fields, loaded before the ranks are formed
      int Lc = 0, pi = 0, pj = 0;
      if (q.f) {
        Lc = t.lvl[k] + 1;
        pi = t.pi[k];
        pj = t.pj[k];
      }
      const uint32_t b0 = __ballot_sync(0xffffffffu, q.f);
      const uint32_t b1 = __ballot_sync(0xffffffffu, q.keep);
      const uint32_t b2 = __ballot_sync(0xffffffffu, q.co);
      if (lane == 0) {
        wsum[0][warp] = __popc(b0);
        wsum[1][warp] = __popc(b1);
        wsum[2][warp] = __popc(b2);
      }
      __syncthreads();
      int32_t p0 = 0, p1 = 0, p2 = 0, t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
      for (int w = 0; w < kScanBlock / 32; ++w) {
        const int32_t v0 = wsum[0][w], v1 = wsum[1][w], v2 = wsum[2][w];
        p0 += w < warp ? v0 : 0;
        p1 += w < warp ? v1 : 0;
        p2 += w < warp ? v2 : 0;
        t0 += v0;
        t1 += v1;
        t2 += v2;
      }
      if (q.f) {
        const int64_t c0 = n_old + 4 * (run0 + p0 + __popc(b0 & below));
        const int L = Lc, i = pi, j = pj;
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
          t.lvl[c0 + ch] = (int8_t)L;
          t.pi[c0 + ch] = 2 * i + (ch & 1);
          t.pj[c0 + ch] = 2 * j + (ch >> 1);
          t.child[c0 + ch] = -1;
          flag[c0 + ch] = 0u;
        }
        t.child[k] = (int32_t)c0;
        flag[k] = 0u;
        if (q.co) {
          const int64_t r2 = keep_total + 4 * (run2 + p2 + __popc(b2 & below));
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) next[r2 + ch] = (int32_t)(c0 + ch);
          if (lmap) set_level_map(lmap, t.n0, L, i, j, c0);
        }
      } else if (q.keep) {
        next[run1 + p1 + __popc(b1 & below)] = k;
      }
      run0 += t0;
      run1 += t1;
      run2 += t2;
      __syncthreads();
    }
  }
}

// Step vi: copy the selected nodes (leaves, or all) to the output arrays.

// The fields of every round's node are loaded before the ranks are formed,
// so their latency overlaps the block's ballots and barriers.
__global__ void __launch_bounds__(kScanBlock) k_emit_out(TreeView t, OutView o, int all, int64_t n,
                                                         const int64_t *boff) {
  __shared__ int32_t wsum[kScanBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t start = (int64_t)blockIdx.x * kScanItems;
  bool sel[kScanRounds];
  int lv[kScanRounds], pi[kScanRounds], pj[kScanRounds], cl[kScanRounds];
  float N[kScanRounds], P[kScanRounds], I0[kScanRounds];
#pragma unroll
  for (int rr = 0; rr < kScanRounds; ++rr) {
    const int64_t k = start + (int64_t)rr * kScanBlock + threadIdx.x;
    sel[rr] = false;
    if (k < n) {
      cl[rr] = t.child[k];
      sel[rr] = all || cl[rr] < 0;
      lv[rr] = t.lvl[k];
      pi[rr] = t.pi[k];
      pj[rr] = t.pj[k];
      N[rr] = t.N[k];
      P[rr] = t.p[k];
      I0[rr] = o.I ? t.I[k] : 0.f;  // no tree intensities are read without o.I
    }
  }
  int64_t run = boff[blockIdx.x];
#pragma unroll
  for (int rr = 0; rr < kScanRounds; ++rr) {
    const int64_t k = start + (int64_t)rr * kScanBlock + threadIdx.x;
    const uint32_t bal = __ballot_sync(0xffffffffu, sel[rr]);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int32_t before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kScanBlock / 32; ++w) {
      const int32_t v = wsum[w];
      before += w < warp ? v : 0;
      tot += v;
    }
    if (sel[rr]) {
      const int64_t r = run + before + __popc(bal & ((1u << lane) - 1u));
      if (o.level) o.level[r] = lv[rr];
      if (o.i) o.i[r] = pi[rr];
      if (o.j) o.j[r] = pj[rr];
      if (o.is_leaf) o.is_leaf[r] = cl[rr] < 0;
      if (o.N) o.N[r] = N[rr];
      if (o.p) o.p[r] = P[rr];
      if (o.I) {
        o.I[r] = I0[rr];
        for (int b = 1; b < o.n_bands; ++b) o.I[(int64_t)b * o.stride + r] = t.I[(int64_t)b * t.cap + k];
      }
    }
    run += tot;
    __syncthreads();
  }
}

// Base image, row-major: node j*n0 + i.
__global__ void k_init_base(TreeView t) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)t.n0 * t.n0;
  if (k >= n) return;
  t.lvl[k] = 0;
  t.pi[k] = (int32_t)(k % t.n0);
  t.pj[k] = (int32_t)(k / t.n0);
  t.child[k] = -1;
}

// ---- band flux and step count --------------------------------------------
// Per block: sum over selected pixels of I_b x area(level) in FP64 and of the
// step counts (integers); a second kernel adds the block partials of each
// band in a fixed order (strided per thread, then a tree), so the result does
// not depend on scheduling. area(level) = area0 4^-L is an exact power-of-two
// scaling, applied as a product.
__device__ __forceinline__ double pow4_neg(int L) {
  return __longlong_as_double((long long)(1023 - 2 * L) << 52);
}

__global__ void __launch_bounds__(256) k_flux_partial(FluxArgs a) {
  __shared__ double sh[256];
  __shared__ unsigned long long shs[256];
  __shared__ double area[kMaxLevels];
  if (threadIdx.x < kMaxLevels) area[threadIdx.x] = a.area0 * pow4_neg(threadIdx.x);
  const int64_t start = (int64_t)blockIdx.x * a.per_block;
  const int64_t end = min(a.n, start + a.per_block);
  double *outp = a.partial + (int64_t)blockIdx.x * (a.n_bands + 1);
  unsigned long long st = 0;
  for (int64_t k = start + threadIdx.x; k < end; k += blockDim.x) st += a.steps[k];
  shs[threadIdx.x] = st;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) shs[threadIdx.x] += shs[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) outp[0] = (double)shs[0];
  for (int b = 0; b < a.n_bands; ++b) {
    // a thread's leaves summed as an unevaluated pair of FP32 numbers
    // (Knuth's two-sum: hi + lo carries the sum to ~2^-44 relative) of
    // I 4^-L, an exact scaling while the product stays a normal number; the
    // rare smaller terms go to an FP64 sum. FP64 work per thread, not per
    // leaf (FP64 issues at 1/64 of the FP32 rate here).
    float hi = 0.f, lo = 0.f;
    double tiny = 0.0;
    for (int64_t k = start + threadIdx.x; k < end; k += blockDim.x) {
      const bool leaf = a.child ? a.child[k] < 0 : true;
      if (!leaf) continue;
      const int L = a.lvl ? a.lvl[k] : 0;
      const float I = a.I[(int64_t)b * a.stride + k];
      const float x = __fmul_rn(I, __int_as_float((127 - 2 * L) << 23));
      if (fabsf(x) >= 0x1p-126f || x == 0.f) {
        const float t = __fadd_rn(hi, x);
        const float bv = __fsub_rn(t, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(x, bv)));
        hi = t;
      } else {
        tiny = fma((double)I, area[L], tiny);
      }
    }
    double s = fma(((double)hi + (double)lo), a.area0, tiny);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
      if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) outp[b + 1] = sh[0];
    __syncthreads();
  }
}

// One block per output: block 0 the step count, block b + 1 band b.
__global__ void __launch_bounds__(256) k_flux_final(const double *partial, int64_t nblocks,
                                                    int n_bands, double *flux, double *steps) {
  __shared__ double sh[256];
  const int b = (int)blockIdx.x - 1;
  double s = 0.0;
  for (int64_t x = threadIdx.x; x < nblocks; x += blockDim.x) s += partial[x * (n_bands + 1) + b + 1];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (b < 0) *steps = sh[0];
    else flux[b] = sh[0];
  }
}

// ---- host launchers ----------------------------------------------------------

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_init_base(const TreeView &t, cudaStream_t st) {
  const int64_t n = (int64_t)t.n0 * t.n0;
  k_init_base<<<nblk(n, 256), 256, 0, st>>>(t);
  return cudaGetLastError();
}

int sm_count() {
  static std::atomic<int> sms{0};
  int n = sms.load(std::memory_order_relaxed);
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 1;
    }
    sms.store(n, std::memory_order_relaxed);
  }
  return n;
}

// Blocks for a grid-stride launch: enough for `per_sm` blocks on every SM.
static unsigned stride_blocks(int64_t n, int block, int per_sm) {
  const int64_t cap = (int64_t)sm_count() * per_sm;
  const int64_t need = (n + block - 1) / block;
  return (unsigned)(need < cap ? need : cap);
}

int64_t scan_blocks(int64_t n) { return scan_chunks(n); }

cudaError_t launch_list_init(int32_t *list, int64_t m, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  k_iota<<<nblk(m, 256), 256, 0, st>>>(list, m);
  return cudaGetLastError();
}

cudaError_t launch_list_scan(const TreeView &t, const int32_t *open, int64_t m, double xi_crit,
                             int xi_norm, int refine_on, uint32_t *flag, cudaStream_t st,
                             const int32_t *lmap) {
  if (m <= 0) return cudaSuccess;
  k_xi_scan_list<<<nblk(m, 256), 256, 0, st>>>(t, open, m, xi_crit, xi_norm, refine_on, flag, lmap);
  return cudaGetLastError();
}

cudaError_t launch_list_balance(const TreeView &t, const int32_t *open, int64_t m, uint32_t *flag,
                                uint32_t *err, cudaStream_t st, const int32_t *lmap) {
  if (m <= 0) return cudaSuccess;
  k_balance_list<<<stride_blocks(m, 128, 16), 128, 0, st>>>(t, open, m, flag, err, lmap);
  return cudaGetLastError();
}

cudaError_t launch_list_count(const TreeView &t, const int32_t *open, int64_t m,
                              const uint32_t *flag, int32_t *bcount, int64_t *boff,
                              int64_t *totals, cudaStream_t st) {
  const int64_t nb = scan_blocks(m);
  if (nb == 0) return cudaMemsetAsync(totals, 0, 3 * sizeof(int64_t), st);
  k_count3<<<(unsigned)nb, kScanBlock, 0, st>>>(t, open, m, flag, t.Lm, bcount, nb);
  k_scan_blocks3<<<3, 1024, 0, st>>>(bcount, nb, boff, totals);
  return cudaGetLastError();
}

cudaError_t launch_list_emit(const TreeView &t, const int32_t *open, int64_t m, uint32_t *flag,
                             const int64_t *boff, const int64_t *totals, int64_t n_old,
                             int32_t *next, cudaStream_t st, int32_t *lmap) {
  const int64_t nb = scan_blocks(m);
  if (nb == 0) return cudaSuccess;
  k_emit3<<<(unsigned)nb, kScanBlock, 0, st>>>(t, open, m, flag, t.Lm, boff, totals, nb, n_old, next, lmap);
  return cudaGetLastError();
}

cudaError_t launch_count_flags(const uint32_t *flag, int64_t n, int32_t *bcount, int64_t *boff,
                               int64_t *total, cudaStream_t st) {
  const int64_t nb = scan_blocks(n);
  if (nb == 0) return cudaMemsetAsync(total, 0, sizeof(int64_t), st);
  k_count<<<(unsigned)nb, kScanBlock, 0, st>>>(PredFlag{flag}, n, bcount);
  k_scan_blocks<<<1, 1024, 0, st>>>(bcount, nb, boff, total);
  return cudaGetLastError();
}

cudaError_t launch_scan_offsets(const int32_t *bcount, int64_t nb, int64_t *boff, int64_t *total,
                                cudaStream_t st) {
  if (nb == 0) return cudaMemsetAsync(total, 0, sizeof(int64_t), st);
  k_scan_blocks<<<1, 1024, 0, st>>>(bcount, nb, boff, total);
  return cudaGetLastError();
}


cudaError_t launch_count_leaves(const TreeView &t, int all, int64_t n, int32_t *bcount,
                                int64_t *boff, int64_t *total, cudaStream_t st) {
  const int64_t nb = scan_blocks(n);
  if (nb == 0) return cudaMemsetAsync(total, 0, sizeof(int64_t), st);
  k_count<<<(unsigned)nb, kScanBlock, 0, st>>>(PredLeaf{t.child, all}, n, bcount);
  k_scan_blocks<<<1, 1024, 0, st>>>(bcount, nb, boff, total);
  return cudaGetLastError();
}

cudaError_t launch_emit_out(const TreeView &t, const OutView &o, int all, int64_t n,
                            const int64_t *boff, cudaStream_t st) {
  const int64_t nb = scan_blocks(n);
  if (nb == 0) return cudaSuccess;
  k_emit_out<<<(unsigned)nb, kScanBlock, 0, st>>>(t, o, all, n, boff);
  return cudaGetLastError();
}

// Blocks of the device-count sweep kernels: a few per SM, looping over items.
static unsigned sweep_blocks(int per_sm) { return (unsigned)(sm_count() * per_sm); }

cudaError_t launch_sweep_scan(const TreeView &t, int32_t *const open[2], const SweepState *S,
                              double xi_crit, int xi_norm, int refine_on, uint32_t *flag,
                              cudaStream_t st, const int32_t *lmap) {
  return launch_pdl(k_xi_scan_dev, dim3(sweep_blocks(8)), dim3(256), 0, st, t,
                    (const int32_t *)open[0], (const int32_t *)open[1], S, xi_crit, xi_norm,
                    refine_on, flag, lmap);
}

cudaError_t launch_sweep_scan_balance(const TreeView &t, int32_t *const open[2],
                                      const SweepState *S, double xi_crit, int xi_norm,
                                      int refine_on, uint32_t *flag, uint32_t *err,
                                      cudaStream_t st, const int32_t *lmap) {
  return launch_pdl(k_scan_balance_dev, dim3(sweep_blocks(8)), dim3(256), 0, st, t,
                    (const int32_t *)open[0], (const int32_t *)open[1], S, xi_crit, xi_norm,
                    refine_on, flag, err, lmap);
}

cudaError_t launch_sweep_balance(const TreeView &t, int32_t *const open[2], const SweepState *S,
                                 uint32_t *flag, uint32_t *err, cudaStream_t st,
                                 const int32_t *lmap) {
  return launch_pdl(k_balance_dev, dim3(sweep_blocks(16)), dim3(128), 0, st, t,
                    (const int32_t *)open[0], (const int32_t *)open[1], S, flag, err, lmap);
}

cudaError_t launch_sweep_count(const TreeView &t, int32_t *const open[2], SweepState *S,
                               const uint32_t *flag, int32_t *bcount, int64_t *boff,
                               int64_t nb_cap, cudaStream_t st) {
  cudaError_t e = launch_pdl(k_count3d, dim3(sweep_blocks(8)), dim3(kScanBlock), 0, st, t,
                             (const int32_t *)open[0], (const int32_t *)open[1],
                             (const SweepState *)S, flag, bcount, nb_cap);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_scan_blocks3d, dim3(3), dim3(1024), 0, st, (const int32_t *)bcount, nb_cap,
                    boff, S);
}

cudaError_t launch_sweep_emit(const TreeView &t, int32_t *const open[2], const SweepState *S,
                              uint32_t *flag, const int64_t *boff, int64_t nb_cap,
                              cudaStream_t st, int32_t *lmap) {
  return launch_pdl(k_emit3d, dim3(sweep_blocks(8)), dim3(kScanBlock), 0, st, t, open[0], open[1],
                    S, flag, boff, nb_cap, lmap);
}


int64_t flux_blocks(int64_t n) {
  const int64_t per = 8192;
  return n <= 0 ? 0 : (n + per - 1) / per;
}

cudaError_t launch_flux(FluxArgs a, double *flux, double *steps, cudaStream_t st) {
  a.per_block = 8192;
  const int64_t nb = flux_blocks(a.n);
  if (nb == 0) {
    cudaError_t e = cudaMemsetAsync(flux, 0, sizeof(double) * a.n_bands, st);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(steps, 0, sizeof(double), st);
  }
  k_flux_partial<<<(unsigned)nb, 256, 0, st>>>(a);
  k_flux_final<<<(unsigned)(a.n_bands + 1), 256, 0, st>>>(a.partial, nb, a.n_bands, flux, steps);
  return cudaGetLastError();
}

}  // namespace air
