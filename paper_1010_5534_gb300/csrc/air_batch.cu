// air_batch.cu -- batched adaptive images: many views of one grid (each view
// with all its energy bands) rendered by ONE cooperative persistent kernel.
// Parkin (2010), Section 2 steps i-vi, applied to every view at once.
//
// Inside the kernel, per sweep:
//   march   : a work queue of (ray, band chunk) items over the rays added in
//             the previous sweep, all views mixed; warps fetch 32 items at a
//             time with one atomic, so rays of uneven length, level, view and
//             band balance across the whole GPU;
//   band sum: p = sum_b I_b when the bands were split over several threads;
//   scan    : Eq. 2 on every leaf below max_level (all views);
//   balance : 2:1 closure within each view's tree;
//   refine  : per-view prefix sum of the flags (static ranges of nodes per
//             block, per-view counts, per-view offsets), four children per
//             flagged leaf, emitted view by view so every view's nodes keep
//             the order of a single-view render.
// Phases are separated by a grid barrier of the library's own (an arrival
// counter and a generation word); every wait has a time limit after which the
// kernel records AIR_ERR_TIMEOUT and returns. The launch is cooperative, so
// all blocks are resident, and the host captures it in a CUDA graph.
#include <cstring>
#include <vector>

#include "air_handle.cuh"
#include "air_march.cuh"
#include "air_tree.cuh"

namespace air {

constexpr int kBatchBlock = 128;
constexpr int kBatchMaxViews = 256;
constexpr uint32_t kErrBalance = 1u, kErrTimeout = 2u, kErrCapacity = 4u;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier with a time limit. `expected` arrivals release it.
__device__ bool grid_sync(BatchCtl *ctl, unsigned expected, long long timeout_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned *genp = &ctl->bar_gen;
    const unsigned gen = *genp;
    __threadfence();
    const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
    if (arrived == expected) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*genp == gen) {
        if ((long long)(global_ns() - t0) > timeout_ns) {
          atomicOr(&ctl->err, kErrTimeout);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Items [s0, s1) of one block, in rounds of blockDim. For every selected item
// k of view v: emit(k, v, run[v] + rank), rank = selected items of view v
// before k in the block's range. run[] (shared, V entries) advances per round.
template <class Pred, class Emit>
__device__ void block_emit_by_view(const Pred &pred, const int16_t *__restrict__ view, Emit &emit,
                                   int64_t s0, int64_t s1, int V, int64_t *run, int32_t *wcnt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t r0 = s0; r0 < s1; r0 += blockDim.x) {
    for (int x = threadIdx.x; x < nw * V; x += blockDim.x) wcnt[x] = 0;
    __syncthreads();
    const int64_t k = r0 + threadIdx.x;
    const bool sel = k < s1 && pred(k);
    const int v = sel ? (int)view[k] : -1;
    const unsigned m = __match_any_sync(0xffffffffu, v);
    const int rank_w = __popc(m & ((1u << lane) - 1u));
    if (sel && rank_w == 0) wcnt[warp * V + v] = __popc(m);
    __syncthreads();
    if (sel) {
      int64_t before = 0;
      for (int w = 0; w < warp; ++w) before += wcnt[w * V + v];
      emit(k, v, run[v] + before + rank_w);
    }
    __syncthreads();
    for (int vv = threadIdx.x; vv < V; vv += blockDim.x) {
      int64_t s = 0;
      for (int w = 0; w < nw; ++w) s += wcnt[w * V + vv];
      run[vv] += s;
    }
    __syncthreads();
  }
}

struct FlagPred {
  const uint32_t *flag;
  __device__ bool operator()(int64_t k) const { return flag[k] != 0; }
};

struct EmitChildrenV {
  TreeView t;
  int16_t *view;
  const int64_t *vbase;  // shared: first child slot of each view this sweep
  __device__ void operator()(int64_t k, int v, int64_t rank) {
    const int64_t c0 = vbase[v] + 4 * rank;
    const int L = t.lvl[k] + 1, i = t.pi[k], j = t.pj[k];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      t.lvl[c0 + c] = (int8_t)L;
      t.pi[c0 + c] = 2 * i + (c & 1);
      t.pj[c0 + c] = 2 * j + (c >> 1);
      t.child[c0 + c] = -1;
      view[c0 + c] = (int16_t)v;
    }
    t.child[k] = (int32_t)c0;
  }
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

static size_t batch_smem(const GridView &g, int V) {
  const size_t tab = align16(sizeof(float) * (size_t)g.n_bands * (g.n_tbins + 1));
  return tab + 3 * sizeof(int64_t) * V + sizeof(int32_t) * V + sizeof(int32_t) * (kBatchBlock / 32) * V;
}

// No minimum-blocks bound: with one, the compiler takes more registers (198
// instead of 152 at 8 bands per thread) and the batch runs slower; bounds of 4
// and more blocks per SM spill in the refinement phases and run 2.5x slower.
template <int NBT, bool AMR, int FMT>
__global__ void __launch_bounds__(kBatchBlock) k_air_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GridView &g = a.g;
  const int V = a.V, nb = g.n_bands, tstride = g.n_tbins + 1;
  float *tab = (float *)smem_raw;
  int64_t *run = (int64_t *)(smem_raw + align16(sizeof(float) * (size_t)nb * tstride));
  int64_t *tot = run + V;
  int64_t *vbase = tot + V;
  int32_t *cnt = (int32_t *)(vbase + V);
  int32_t *wcnt = cnt + V;
  __shared__ int64_t s_total;
  if (FMT == kCellXq)
    for (int x = threadIdx.x; x < nb * tstride; x += blockDim.x) tab[x] = g.table[x];
  __syncthreads();

  const TreeView t = a.t;
  const int n0 = t.n0;
  const int64_t nn0 = (int64_t)n0 * n0;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const unsigned nblk = gridDim.x;
  const int lane = threadIdx.x & 31;

  // step i: the base image of every view, view-major, row-major within a view
  // (mode 2 continues from the base images a mode-1 launch traced)
  const int64_t nbase = (int64_t)V * nn0;
  if (a.mode != 2) {
    for (int64_t k = gtid; k < nbase; k += gstride) {
      const int v = (int)(k / nn0);
      const int64_t r = k - (int64_t)v * nn0;
      t.lvl[k] = 0;
      t.pi[k] = (int32_t)(r % n0);
      t.pj[k] = (int32_t)(r / n0);
      t.child[k] = -1;
      a.view[k] = (int16_t)v;
    }
    if (!grid_sync(a.ctl, nblk + (a.stall ? 1u : 0u), a.timeout_ns)) return;
  }

  int64_t first = a.mode == 2 ? nbase : 0, n = nbase;
  if (a.mode == 2 && a.P > 0) {
    // the proposal wave of every view: (ray, band chunk) items from the queue
    const unsigned long long items = (unsigned long long)a.P * (unsigned long long)a.chunks;
    for (;;) {
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(&a.ctl->q_head, 32ull);
      b = __shfl_sync(0xffffffffu, b, 0);
      if (b >= items) break;
      const unsigned long long it = b + lane;
      if (it < items) {
        const int chunk = (int)(it / (unsigned long long)a.P);
        const int64_t q = (int64_t)(it - (unsigned long long)chunk * a.P);
        const int b0 = chunk * NBT;
        BandCtx bc;
        bc.tab = tab + b0 * tstride;
        bc.tstride = tstride;
        bc.nbh = min(NBT, nb - b0);
        BandRegs<NBT> br;
        band_regs<NBT>(br, g.kappa, g.invkappa, b0, bc.nbh);
        const RayGeom rg = a.geoms[a.pview[q]];
        RTState<NBT> st;
        trace_ray<NBT, AMR, FMT>(st, g, rg, a.plvl[q], a.ppi[q], a.ppj[q], a.fp64_level, bc, br);
        if (chunk == 0) {
          a.pN[q] = st.N;
          a.psteps[q] = st.steps;
        }
#pragma unroll
        for (int c = 0; c < NBT; ++c)
          if (c < bc.nbh) a.pI[(int64_t)(b0 + c) * a.P + q] = st.I[c];
        if (a.chunks == 1) {
          float p = 0.f;
#pragma unroll
          for (int c = 0; c < NBT; ++c)
            if (c < bc.nbh) p += st.I[c];
          a.pp[q] = p;
        }
      }
    }
    if (!grid_sync(a.ctl, nblk, a.timeout_ns)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->q_head = 0ull;
  }
  int sweep = 0;
  for (;; ++sweep) {
    // step ii: trace the rays added last sweep, all views and band chunks
    const int64_t cnt_r = n - first;
    const unsigned long long items = (unsigned long long)cnt_r * (unsigned long long)a.chunks;
    for (;;) {
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(&a.ctl->q_head, 32ull);
      b = __shfl_sync(0xffffffffu, b, 0);
      if (b >= items) break;
      const unsigned long long it = b + lane;
      bool todo = it < items;
      int chunk = 0, v = 0, b0 = 0;
      int64_t k = 0;
      if (todo) {
        chunk = (int)(it / (unsigned long long)cnt_r);
        k = first + (int64_t)(it - (unsigned long long)chunk * cnt_r);
        v = a.view[k];
        b0 = chunk * NBT;
      }
      if (todo && a.mode == 2) {
        // the pixel's values from its view's proposal wave when the wave
        // traced it (the same trace, so the same bits); else trace it
        const int L = t.lvl[k], i = t.pi[k], j = t.pj[k];
        const int64_t pb = (int64_t)v * nn0 + (int64_t)(j >> L) * n0 + (i >> L);
        const int64_t q = prop_index(a.pdepth + 4 * pb, a.poff[pb], L, i, j);
        if (q >= 0) {
          if (chunk == 0) {
            t.N[k] = a.pN[q];
            t.steps[k] = a.psteps[q];
          }
          const int nbh = min(NBT, nb - b0);
          for (int c = 0; c < nbh; ++c) t.I[(int64_t)(b0 + c) * t.cap + k] = a.pI[(int64_t)(b0 + c) * a.P + q];
          if (a.chunks == 1) t.p[k] = a.pp[q];
          todo = false;
        } else if (chunk == 0) {
          atomicAdd(&a.ctl->fb_rays, 1ull);
        }
      }
      if (todo) {
        BandCtx bc;
        bc.tab = tab + b0 * tstride;
        bc.tstride = tstride;
        bc.nbh = min(NBT, nb - b0);
        BandRegs<NBT> br;
        band_regs<NBT>(br, g.kappa, g.invkappa, b0, bc.nbh);
        const RayGeom rg = a.geoms[v];
        RTState<NBT> st;
        trace_ray<NBT, AMR, FMT>(st, g, rg, t.lvl[k], t.pi[k], t.pj[k], a.fp64_level, bc, br);
        if (chunk == 0) {
          t.N[k] = st.N;
          t.steps[k] = st.steps;
          if (a.mode == 1) a.maxlev[k] = (uint8_t)st.maxlev;
        }
#pragma unroll
        for (int q = 0; q < NBT; ++q)
          if (q < bc.nbh) t.I[(int64_t)(b0 + q) * t.cap + k] = st.I[q];
        if (a.chunks == 1) {
          float p = 0.f;
#pragma unroll
          for (int q = 0; q < NBT; ++q)
            if (q < bc.nbh) p += st.I[q];
          t.p[k] = p;
        }
      }
    }
    if (!grid_sync(a.ctl, nblk, a.timeout_ns)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->q_head = 0ull;  // next sweep's queue
    if (a.chunks > 1) {
      for (int64_t k = first + gtid; k < n; k += gstride) {
        float s = 0.f;
        for (int q = 0; q < nb; ++q) s += t.I[(int64_t)q * t.cap + k];
        t.p[k] = s;
      }
      if (!grid_sync(a.ctl, nblk, a.timeout_ns)) return;
    }
    if (a.mode == 1) {
      // the base images are traced (and their band sums): the host computes
      // the features and the proposal, then launches mode 2
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->n_nodes = n;
        a.ctl->sweeps = 0;
      }
      return;
    }
    // step iii: scan, then balance
    for (int64_t k = gtid; k < n; k += gstride)
      a.flag[k] = xi_flag(t, NodeLookup{(int)(a.view[k] * nn0), nullptr}, k, a.xi_crit, a.xi_norm, a.refine_on);
    if (!grid_sync(a.ctl, nblk, a.timeout_ns)) return;
    for (int64_t k = gtid; k < n; k += gstride)
      if (a.flag[k]) balance_from(t, NodeLookup{(int)(a.view[k] * nn0), nullptr}, (int)k, a.flag, &a.ctl->err);
    if (!grid_sync(a.ctl, nblk, a.timeout_ns)) return;
    // step iv: per-view prefix sum over static node ranges
    const int64_t per = (n + nblk - 1) / nblk;
    const int64_t s0 = min(n, (int64_t)blockIdx.x * per), s1 = min(n, s0 + per);
    for (int v = threadIdx.x; v < V; v += blockDim.x) cnt[v] = 0;
    __syncthreads();
    for (int64_t k = s0 + threadIdx.x; k < s1; k += blockDim.x)
      if (a.flag[k]) atomicAdd(&cnt[a.view[k]], 1);
    __syncthreads();
    for (int v = threadIdx.x; v < V; v += blockDim.x) a.bcnt[(int64_t)blockIdx.x * V + v] = cnt[v];
    if (!grid_sync(a.ctl, nblk, a.timeout_ns)) return;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
      int64_t off = 0, all = 0;
      for (unsigned b2 = 0; b2 < nblk; ++b2) {
        const int64_t c = a.bcnt[(int64_t)b2 * V + v];
        if (b2 < blockIdx.x) off += c;
        all += c;
      }
      run[v] = off;
      tot[v] = all;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t acc = 0;
      for (int v = 0; v < V; ++v) {
        vbase[v] = n + 4 * acc;
        acc += tot[v];
      }
      s_total = acc;
    }
    __syncthreads();
    const int64_t total = s_total;
    if (total == 0) break;
    if (n + 4 * total > t.cap) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->need = n + 4 * total;
        atomicOr(&a.ctl->err, kErrCapacity);
      }
      break;
    }
    EmitChildrenV em{t, a.view, vbase};
    block_emit_by_view(FlagPred{a.flag}, a.view, em, s0, s1, V, run, wcnt);
    if (blockIdx.x == 0)
      for (int v = threadIdx.x; v < V; v += blockDim.x)
        if (tot[v] > 0) {
          a.refined[v] += tot[v];
          a.vsweeps[v] += 1;
        }
    if (!grid_sync(a.ctl, nblk, a.timeout_ns)) return;
    first = n;
    n += 4 * total;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl->n_nodes = n;
    a.ctl->sweeps = sweep;
  }
}

// ---- output: per-view leaf compaction, band flux, step counts ---------------

struct LeafPred {
  const int32_t *child;
  int all;
  __device__ bool operator()(int64_t k) const { return all || child[k] < 0; }
};

// Per block of kScanItems nodes: selected nodes per view; ray-cell steps per view.
__global__ void __launch_bounds__(256) k_vcount(TreeView t, const int16_t *view, int all, int64_t n,
                                                int V, int32_t *bcnt,
                                                unsigned long long *vsteps) {
  extern __shared__ int32_t sm_cnt[];
  unsigned long long *sm_steps = (unsigned long long *)(sm_cnt + ((V + 1) & ~1));
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    sm_cnt[v] = 0;
    sm_steps[v] = 0ull;
  }
  __syncthreads();
  const int64_t s0 = (int64_t)blockIdx.x * kScanItems, s1 = min(n, s0 + kScanItems);
  for (int64_t k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
    const int v = view[k];
    if (all || t.child[k] < 0) atomicAdd(&sm_cnt[v], 1);
    atomicAdd(&sm_steps[v], (unsigned long long)t.steps[k]);
  }
  __syncthreads();
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    bcnt[(int64_t)blockIdx.x * V + v] = sm_cnt[v];
    if (sm_steps[v]) atomicAdd(&vsteps[v], sm_steps[v]);
  }
}

// One block per view: exclusive scan of that view's per-block counts.
__global__ void __launch_bounds__(256) k_vscan(const int32_t *bcnt, int64_t nblocks, int V,
                                               int64_t *boff) {
  __shared__ int64_t part[256];
  const int v = blockIdx.x;
  const int64_t per = (nblocks + 255) / 256;
  const int64_t a = threadIdx.x * per, b = min(nblocks, a + per);
  int64_t s = 0;
  for (int64_t x = a; x < b; ++x) s += bcnt[x * V + v];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const int64_t u = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += u;
    __syncthreads();
  }
  int64_t run = part[threadIdx.x] - s;
  for (int64_t x = a; x < b; ++x) {
    boff[x * V + v] = run;
    run += bcnt[x * V + v];
  }
}

struct EmitOutV {
  TreeView t;
  const OutView *outs;    // [V] (global)
  double *sm_flux;        // shared [V][n_bands]
  const RayGeom *geoms;   // [V]: level-0 pixel size of each view
  __device__ void operator()(int64_t k, int v, int64_t r) {
    const OutView &o = outs[v];
    const bool leaf = t.child[k] < 0;
    if (o.level) o.level[r] = t.lvl[k];
    if (o.i) o.i[r] = t.pi[k];
    if (o.j) o.j[r] = t.pj[k];
    if (o.is_leaf) o.is_leaf[r] = leaf;
    if (o.N) o.N[r] = t.N[k];
    if (o.p) o.p[r] = t.p[k];
    const double pix = geoms[v].pix0;
    const double area = pix * pix * __longlong_as_double((long long)(1023 - 2 * t.lvl[k]) << 52);
    for (int b = 0; b < o.n_bands; ++b) {
      const float I = t.I[(int64_t)b * t.cap + k];
      if (o.I) o.I[(int64_t)b * o.stride + r] = I;
      if (leaf) atomicAdd(&sm_flux[v * o.n_bands + b], (double)I * area);
    }
  }
};

__global__ void __launch_bounds__(256) k_vemit(TreeView t, const int16_t *view, int all, int64_t n,
                                               int V, int n_bands, const int64_t *boff,
                                               const OutView *outs, const RayGeom *geoms,
                                               double *vflux) {
  extern __shared__ __align__(16) unsigned char sm[];
  int64_t *run = (int64_t *)sm;
  double *flux = (double *)(run + V);
  int32_t *wcnt = (int32_t *)(flux + (size_t)V * n_bands);
  for (int v = threadIdx.x; v < V; v += blockDim.x) run[v] = boff[(int64_t)blockIdx.x * V + v];
  for (int x = threadIdx.x; x < V * n_bands; x += blockDim.x) flux[x] = 0.0;
  __syncthreads();
  const int64_t s0 = (int64_t)blockIdx.x * kScanItems, s1 = min(n, s0 + kScanItems);
  EmitOutV e{t, outs, flux, geoms};
  block_emit_by_view(LeafPred{t.child, all}, view, e, s0, s1, V, run, wcnt);
  __syncthreads();
  for (int x = threadIdx.x; x < V * n_bands; x += blockDim.x)
    if (flux[x] != 0.0) atomicAdd(&vflux[x], flux[x]);
}

// ---- host ---------------------------------------------------------------------

#define CU_TRY(x)                                    \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

template <int NBT, bool AMR, int FMT>
static cudaError_t batch_occupancy(int *blocks_per_sm, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_air_batch<NBT, AMR, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_air_batch<NBT, AMR, FMT>, kBatchBlock, smem);
}

template <int NBT, bool AMR, int FMT>
static cudaError_t batch_launch(const BatchArgs &a, int grid, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBatchBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_air_batch<NBT, AMR, FMT>, a);
}

typedef cudaError_t (*BatchOccFn)(int *, size_t);
typedef cudaError_t (*BatchLaunchFn)(const BatchArgs &, int, size_t, cudaStream_t);

static bool batch_fns(int nbt, bool amr, int fmt, BatchOccFn *occ, BatchLaunchFn *launch) {
  if (fmt == kCellLam) {
    // per-cell Lambda exists for one-band grids only
    if (nbt != 1) return false;
    *occ = amr ? batch_occupancy<1, true, kCellLam> : batch_occupancy<1, false, kCellLam>;
    *launch = amr ? batch_launch<1, true, kCellLam> : batch_launch<1, false, kCellLam>;
    return true;
  }
#define AIR_BATCH_CASE(N)                                                                     \
  if (nbt == N) {                                                                             \
    if (fmt == kCellXq) {                                                                     \
      *occ = amr ? batch_occupancy<N, true, kCellXq> : batch_occupancy<N, false, kCellXq>;    \
      *launch = amr ? batch_launch<N, true, kCellXq> : batch_launch<N, false, kCellXq>;       \
    } else {                                                                                  \
      *occ = amr ? batch_occupancy<N, true, kCellRho> : batch_occupancy<N, false, kCellRho>;  \
      *launch = amr ? batch_launch<N, true, kCellRho> : batch_launch<N, false, kCellRho>;     \
    }                                                                                         \
    return true;                                                                              \
  }
  AIR_BATCH_CASE(1)
  AIR_BATCH_CASE(2)
  AIR_BATCH_CASE(4)
  AIR_BATCH_CASE(8)
  AIR_BATCH_CASE(16)
#undef AIR_BATCH_CASE
  return false;
}

// Bands per thread of batched renders when the tuning leaves it open: the
// template width that holds every band, up to 8.
static int default_batch_bands_per_thread(int nb) {
  if (nb <= 1) return 1;
  if (nb <= 2) return 2;
  if (nb <= 4) return 4;
  return 8;
}

// Node count for the next attempt of a batch that outgrew its arrays at
// `need` nodes (more sweeps may follow): twice that, as far as half of the
// free device memory allows, and at least a sixteenth above it.
static int64_t batch_regrow(air_grid *g, int64_t need, int64_t bound) {
  const double per_node = 31.0 + 4.0 * g->gv.n_bands;
  size_t fr = 0, tot = 0;
  int64_t roomy = 2 * need;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
    const int64_t held = g->ws.cap;  // freed when the arrays are replaced
    const int64_t fit = (int64_t)(0.5 * (double)fr / per_node) + held;
    roomy = std::min<int64_t>(roomy, fit);
  } else {
    cudaGetLastError();
  }
  return std::min<int64_t>(bound, std::max<int64_t>(need + need / 16, roomy));
}

air_status render_batch(air_grid *g, const air_view *views, int32_t V, const air_params *pr,
                        const air_batch_opts *opts, air_image *outs, air_mlp *mlp,
                        const air_learned_opts *lopts, air_learned_stats *stats) {
  g->raster.ok = false;  // the workspace tree is about to change
  if (!views || !outs || !pr) return set_error(AIR_ERR_ARG, "views, params and outs must not be NULL");
  if (V < 1 || V > kBatchMaxViews) return set_error(AIR_ERR_ARG, "n_views must be in [1, %d]", kBatchMaxViews);
  const int n0 = pr->base_res, Lm = pr->max_level;
  if (n0 < 1 || Lm < 0 || Lm >= kMaxLevels || ((int64_t)n0 << Lm) > (1 << 20))
    return set_error(AIR_ERR_ARG, "need base_res >= 1, 0 <= max_level < %d, base_res << max_level <= 2^20", kMaxLevels);
  if (!(pr->xi_crit >= 0.0) || pr->xi_crit > 1e300) return set_error(AIR_ERR_ARG, "xi_crit must be finite and >= 0");
  if (pr->xi_norm != 0 && pr->xi_norm != 1) return set_error(AIR_ERR_ARG, "xi_norm must be 0 or 1");
  if (pr->refine_on < 0 || pr->refine_on > 2) return set_error(AIR_ERR_ARG, "refine_on must be 0, 1 or 2");
  if (pr->include_interior != 0 && pr->include_interior != 1) return set_error(AIR_ERR_ARG, "include_interior must be 0 or 1");
  air_batch_opts op{};
  op.bands_per_thread = 0;
  op.use_graph = 1;
  op.wait_timeout_ms = 2000.0;
  op.test_stall_barrier = 0;
  if (opts) op = *opts;
  if (!(op.wait_timeout_ms > 0.0)) op.wait_timeout_ms = 2000.0;
  const int nb = g->gv.n_bands;
  int nbt = op.bands_per_thread > 0 ? op.bands_per_thread
            : (g->tune.batch_bands_per_thread > 0 ? g->tune.batch_bands_per_thread : default_batch_bands_per_thread(nb));
  if (g->gv.cell_fmt == kCellLam && nbt > 0) nbt = 1;  // one band
  BatchOccFn occ;
  BatchLaunchFn launch;
  if (!batch_fns(nbt, g->gv.kind == AIR_GRID_AMR, g->gv.cell_fmt, &occ, &launch))
    return set_error(AIR_ERR_ARG, "bands_per_thread must be 1, 2, 4, 8 or 16");
  for (int v = 0; v < V; ++v) {
    air_status s = check_image(&outs[v]);
    if (s) return s;
  }
  std::vector<RayGeom> geoms(V);
  for (int v = 0; v < V; ++v) {
    Camera cam;
    air_status s = make_camera(&views[v], cam);
    if (s) return s;
    geoms[v] = make_geom(g->gv, cam, n0);
  }
  g->last.valid = false;  // the batch reuses the single-view workspace
  air_status s = init_scalars(g->ws);
  if (s) return s;
  Workspace &w = g->ws;
  BatchWork &bw = g->batch;
  cudaStream_t st = g->stream;
  const int64_t nbase = (int64_t)V * n0 * n0;
  int64_t bound = 0;
  for (int l = 0; l <= Lm; ++l) bound += ((int64_t)n0 << l) * ((int64_t)n0 << l);
  bound *= V;
  if (bound > INT32_MAX) bound = INT32_MAX;
  const size_t smem = batch_smem(g->gv, V);
  int per_sm = 0;
  int dev = 0, sms = 0;
  CU_TRY(cudaGetDevice(&dev));
  CU_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CU_TRY(occ(&per_sm, smem));
  if (per_sm < 1) return set_error(AIR_ERR_CUDA, "batched kernel cannot be resident (smem %zu B)", smem);
  if (g->tune.batch_blocks_per_sm > 0 && g->tune.batch_blocks_per_sm < per_sm) per_sm = g->tune.batch_blocks_per_sm;
  const int grid = per_sm * sms;
  // device-side state
  CU_TRY(ensure((void **)&bw.geoms, &bw.geoms_b, sizeof(RayGeom) * V));
  CU_TRY(ensure((void **)&bw.ctl, &bw.ctl_b, sizeof(BatchCtl)));
  CU_TRY(ensure((void **)&bw.bcnt, &bw.bcnt_b, sizeof(int32_t) * (size_t)std::max<int64_t>(grid, scan_blocks(bound)) * V));
  CU_TRY(ensure((void **)&bw.refined, &bw.refined_b, sizeof(int64_t) * V));
  CU_TRY(ensure((void **)&bw.vsweeps, &bw.vsweeps_b, sizeof(int32_t) * V));
  CU_TRY(ensure((void **)&bw.vsteps, &bw.vsteps_b, sizeof(unsigned long long) * V));
  CU_TRY(ensure((void **)&bw.vflux, &bw.vflux_b, sizeof(double) * V * nb));
  CU_TRY(ensure((void **)&bw.outs, &bw.outs_b, sizeof(OutView) * V));
  if (!bw.h_ctl) CU_TRY(cudaMallocHost((void **)&bw.h_ctl, sizeof(BatchCtl)));
  if (bw.h_geoms_b < sizeof(RayGeom) * V) {
    if (bw.h_geoms) cudaFreeHost(bw.h_geoms);
    bw.h_geoms = nullptr;
    bw.h_geoms_b = 0;
    CU_TRY(cudaMallocHost(&bw.h_geoms, sizeof(RayGeom) * kBatchMaxViews));
    bw.h_geoms_b = sizeof(RayGeom) * kBatchMaxViews;
  }
  std::memcpy(bw.h_geoms, geoms.data(), sizeof(RayGeom) * V);
  int64_t want = std::max<int64_t>(std::min<int64_t>(bound, 4 * nbase), w.cap);
  bool done = false;
  for (int attempt = 0; attempt < 8 && !done; ++attempt) {
    // a batch that outgrew the node arrays is rendered again with arrays of
    // the size it needed (and a sixteenth more), not the usual doubling
    if ((s = ensure_nodes(g, want, 0, bound, true, attempt > 0))) return s;
    TreeView t = w.tree(n0, Lm);
    BatchArgs a{};
    a.g = g->gv;
    a.geoms = bw.geoms;
    a.V = V;
    a.chunks = (nb + nbt - 1) / nbt;
    a.fp64_level = pr->fp64_level < 0 ? 3 : pr->fp64_level;
    a.xi_norm = pr->xi_norm;
    a.refine_on = pr->refine_on;
    a.stall = op.test_stall_barrier ? 1 : 0;
    a.xi_crit = pr->xi_crit;
    a.t = t;
    a.view = w.view;
    a.flag = w.flag;
    a.ctl = bw.ctl;
    a.bcnt = bw.bcnt;
    a.refined = bw.refined;
    a.vsweeps = bw.vsweeps;
    a.timeout_ns = (long long)(op.wait_timeout_ms * 1e6);
    CU_TRY(cudaMemcpyAsync(bw.geoms, bw.h_geoms, sizeof(RayGeom) * V, cudaMemcpyHostToDevice, st));
    g->prof.used = 0;
    if (mlp) {
      // learned proposal: the base images (mode 1), the network's proposal
      // for every view, then every proposal wave and the sweeps (mode 2)
      LearnWork &lw = g->learn;
      const double q = (lopts && lopts->quantile > 0.0 && lopts->quantile <= 1.0) ? lopts->quantile : 0.8;
      CU_TRY(ensure((void **)&lw.maxlev, &lw.maxlev_b, (size_t)nbase));
      a.mode = 1;
      a.maxlev = lw.maxlev;
      for (int phase = 1; phase <= 2; ++phase) {
        if (phase == 2) {
          int64_t P = 0;
          if ((s = batch_proposal(g, V, pr, mlp, q, lw.maxlev, &P))) return s;
          a.mode = 2;
          a.maxlev = nullptr;
          a.pdepth = lw.depth;
          a.poff = lw.off;
          a.plvl = lw.plvl;
          a.ppi = lw.ppi;
          a.ppj = lw.ppj;
          a.pview = lw.pview;
          a.P = P;
          a.pN = lw.pN;
          a.pI = lw.pI;
          a.pp = lw.pp;
          a.psteps = lw.psteps;
          if (stats) {
            std::memset(stats, 0, sizeof(*stats));
            stats->proposed_rays = P;
          }
        }
        CU_TRY(prof_open(g, AIR_PHASE_BATCH, 1));
        CU_TRY(cudaMemsetAsync(bw.ctl, 0, sizeof(BatchCtl), st));
        if (phase == 1) {
          CU_TRY(cudaMemsetAsync(bw.refined, 0, sizeof(int64_t) * V, st));
          CU_TRY(cudaMemsetAsync(bw.vsweeps, 0, sizeof(int32_t) * V, st));
        }
        CU_TRY(launch(a, grid, smem, st));
        CU_TRY(prof_close(g));
        CU_TRY(cudaMemcpyAsync(bw.h_ctl, bw.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st));
        CU_TRY(cudaStreamSynchronize(st));
        if (bw.h_ctl->err & kErrTimeout)
          return set_error(AIR_ERR_TIMEOUT, "batched kernel: a grid barrier wait exceeded %.0f ms", op.wait_timeout_ms);
        if (bw.h_ctl->err & kErrBalance) return set_error(AIR_ERR_NUMERIC, "balance closure overflowed its stack");
        if (bw.h_ctl->err & kErrCapacity) break;
      }
      const BatchCtl c = *bw.h_ctl;
      if (c.err & kErrCapacity) {
        if (c.need > bound) return set_error(AIR_ERR_NUMERIC, "quadtree exceeds its bound");
        want = batch_regrow(g, c.need, bound);
        continue;
      }
      if (stats) stats->fallback_rays = (int64_t)c.fb_rays;
      done = true;
      continue;
    }
    // the graph holds: reset of the control words, the cooperative launch
    const bool same = bw.exec && !std::memcmp(&bw.key, &a, sizeof(BatchArgs)) && bw.key_grid == grid &&
                      bw.key_smem == smem && bw.key_nbt == nbt;
    CU_TRY(prof_open(g, AIR_PHASE_BATCH, 1));
    if (op.use_graph) {
      if (!same) {
        if (bw.exec) {
          cudaGraphExecDestroy(bw.exec);
          bw.exec = nullptr;
        }
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph then runs on the caller's
        if (!bw.cap_stream) CU_TRY(cudaStreamCreateWithFlags(&bw.cap_stream, cudaStreamNonBlocking));
        cudaStream_t cs = bw.cap_stream;
        cudaGraph_t graph;
        CU_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = cudaMemsetAsync(bw.ctl, 0, sizeof(BatchCtl), cs);
        cudaError_t e2 = cudaMemsetAsync(bw.refined, 0, sizeof(int64_t) * V, cs);
        cudaError_t e3 = cudaMemsetAsync(bw.vsweeps, 0, sizeof(int32_t) * V, cs);
        cudaError_t e4 = launch(a, grid, smem, cs);
        cudaError_t e5 = cudaStreamEndCapture(cs, &graph);
        if (e1 || e2 || e3 || e4 || e5) {
          cudaGetLastError();
          return set_error(AIR_ERR_CUDA, "graph capture of the batched launch failed: %s",
                           cudaGetErrorString(e4 ? e4 : (e5 ? e5 : (e1 ? e1 : (e2 ? e2 : e3)))));
        }
        cudaError_t e6 = cudaGraphInstantiate(&bw.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e6 != cudaSuccess) return cuda_fail(e6, "cudaGraphInstantiate");
        bw.key = a;
        bw.key_grid = grid;
        bw.key_smem = smem;
        bw.key_nbt = nbt;
      }
      CU_TRY(cudaGraphLaunch(bw.exec, st));
    } else {
      CU_TRY(cudaMemsetAsync(bw.ctl, 0, sizeof(BatchCtl), st));
      CU_TRY(cudaMemsetAsync(bw.refined, 0, sizeof(int64_t) * V, st));
      CU_TRY(cudaMemsetAsync(bw.vsweeps, 0, sizeof(int32_t) * V, st));
      CU_TRY(launch(a, grid, smem, st));
    }
    CU_TRY(prof_close(g));
    CU_TRY(cudaMemcpyAsync(bw.h_ctl, bw.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st));
    CU_TRY(cudaStreamSynchronize(st));
    const BatchCtl c = *bw.h_ctl;
    if (c.err & kErrTimeout) return set_error(AIR_ERR_TIMEOUT, "batched kernel: a grid barrier wait exceeded %.0f ms", op.wait_timeout_ms);
    if (c.err & kErrBalance) return set_error(AIR_ERR_NUMERIC, "balance closure overflowed its stack");
    if (c.err & kErrCapacity) {
      if (c.need > bound) return set_error(AIR_ERR_NUMERIC, "quadtree exceeds its bound");
      want = batch_regrow(g, c.need, bound);
      continue;
    }
    done = true;
  }
  if (!done) return set_error(AIR_ERR_CAPACITY, "batched quadtree did not fit after regrowing");
  const int64_t n = bw.h_ctl->n_nodes;
  std::vector<int64_t> refined(V);
  std::vector<int32_t> vsw(V);
  CU_TRY(cudaMemcpy(refined.data(), bw.refined, sizeof(int64_t) * V, cudaMemcpyDeviceToHost));
  CU_TRY(cudaMemcpy(vsw.data(), bw.vsweeps, sizeof(int32_t) * V, cudaMemcpyDeviceToHost));
  if (mlp && stats) {
    int64_t traced = 0;  // nodes beyond the base images: from the wave or traced after it
    for (int v = 0; v < V; ++v) traced += 4 * refined[v];
    stats->used_rays = traced - stats->fallback_rays;
    stats->wasted_rays = stats->proposed_rays - stats->used_rays;
    int32_t mx = 0;
    for (int v = 0; v < V; ++v) mx = std::max(mx, vsw[v]);
    stats->sweeps = mx;
    stats->waves = 2;  // the base images, then the proposal waves and sweeps in one launch
  }
  const int all = pr->include_interior;
  // sizes and capacities
  std::vector<int64_t> n_out(V);
  bool short_cap = false;
  for (int v = 0; v < V; ++v) {
    const int64_t leaves = (int64_t)n0 * n0 + 3 * refined[v];
    const int64_t rays = (int64_t)n0 * n0 + 4 * refined[v];
    n_out[v] = all ? rays : leaves;
    outs[v].n_out = n_out[v];
    outs[v].n_leaves = leaves;
    outs[v].n_rays = rays;
    outs[v].n_sweeps = vsw[v];
    outs[v].n_steps = 0;
    if (outs[v].capacity < n_out[v]) short_cap = true;
  }
  if (short_cap) return set_error(AIR_ERR_CAPACITY, "an output image's capacity is smaller than its pixel count (n_out set per view)");
  // output views: caller device arrays, or staging slices for host memory
  std::vector<OutView> ov(V);
  int64_t stage = 0;
  for (int v = 0; v < V; ++v)
    if (outs[v].mem == AIR_HOST) stage += std::max<int64_t>(n_out[v], 1);
  if (stage > 0) {
    CU_TRY(ensure((void **)&w.o_level, &w.o_level_b, 4 * stage));
    CU_TRY(ensure((void **)&w.o_i, &w.o_i_b, 4 * stage));
    CU_TRY(ensure((void **)&w.o_j, &w.o_j_b, 4 * stage));
    CU_TRY(ensure((void **)&w.o_leaf, &w.o_leaf_b, stage));
    CU_TRY(ensure((void **)&w.o_N, &w.o_N_b, 4 * stage));
    CU_TRY(ensure((void **)&w.o_p, &w.o_p_b, 4 * stage));
    CU_TRY(ensure((void **)&w.o_I, &w.o_I_b, 4 * stage * nb));
  }
  int64_t so = 0;
  for (int v = 0; v < V; ++v) {
    const air_image &im = outs[v];
    OutView &o = ov[v];
    o.n_bands = nb;
    if (im.mem == AIR_DEVICE) {
      o.level = im.level; o.i = im.i; o.j = im.j; o.is_leaf = im.is_leaf;
      o.N = im.coldens; o.p = im.p; o.I = im.intensity;
      o.stride = im.capacity;
    } else {
      const int64_t m = std::max<int64_t>(n_out[v], 1);
      o.level = im.level ? w.o_level + so : nullptr;
      o.i = im.i ? w.o_i + so : nullptr;
      o.j = im.j ? w.o_j + so : nullptr;
      o.is_leaf = im.is_leaf ? w.o_leaf + so : nullptr;
      o.N = im.coldens ? w.o_N + so : nullptr;
      o.p = im.p ? w.o_p + so : nullptr;
      o.I = im.intensity ? w.o_I + so * nb : nullptr;
      o.stride = m;
      so += m;
    }
  }
  CU_TRY(cudaMemcpyAsync(bw.outs, ov.data(), sizeof(OutView) * V, cudaMemcpyHostToDevice, st));
  CU_TRY(cudaMemsetAsync(bw.vsteps, 0, sizeof(unsigned long long) * V, st));
  CU_TRY(cudaMemsetAsync(bw.vflux, 0, sizeof(double) * V * nb, st));
  TreeView t = w.tree(n0, Lm);
  const int64_t nblocks = scan_blocks(n);
  CU_TRY(prof_open(g, AIR_PHASE_OUTPUT, 3));
  if (nblocks > 0) {
    const size_t sm1 = sizeof(int32_t) * ((V + 1) & ~1) + sizeof(unsigned long long) * V;
    k_vcount<<<(unsigned)nblocks, 256, sm1, st>>>(t, w.view, all, n, V, bw.bcnt, bw.vsteps);
    CU_TRY(cudaGetLastError());
    CU_TRY(ensure((void **)&bw.boff, &bw.boff_b, sizeof(int64_t) * nblocks * V));
    k_vscan<<<V, 256, 0, st>>>(bw.bcnt, nblocks, V, bw.boff);
    CU_TRY(cudaGetLastError());
    const size_t sm3 = sizeof(int64_t) * V + sizeof(double) * V * nb + sizeof(int32_t) * 8 * V;
    CU_TRY(cudaFuncSetAttribute(k_vemit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
    k_vemit<<<(unsigned)nblocks, 256, sm3, st>>>(t, w.view, all, n, V, nb, bw.boff, bw.outs, bw.geoms, bw.vflux);
    CU_TRY(cudaGetLastError());
  }
  CU_TRY(prof_close(g));
  // copies out
  std::vector<double> vflux((size_t)V * nb);
  std::vector<unsigned long long> vsteps(V);
  for (int v = 0; v < V; ++v) {
    const air_image &im = outs[v];
    const OutView &o = ov[v];
    const int64_t m = n_out[v];
    if (im.mem == AIR_HOST && m > 0) {
      if (im.level) CU_TRY(cudaMemcpyAsync(im.level, o.level, 4 * m, cudaMemcpyDeviceToHost, st));
      if (im.i) CU_TRY(cudaMemcpyAsync(im.i, o.i, 4 * m, cudaMemcpyDeviceToHost, st));
      if (im.j) CU_TRY(cudaMemcpyAsync(im.j, o.j, 4 * m, cudaMemcpyDeviceToHost, st));
      if (im.is_leaf) CU_TRY(cudaMemcpyAsync(im.is_leaf, o.is_leaf, m, cudaMemcpyDeviceToHost, st));
      if (im.coldens) CU_TRY(cudaMemcpyAsync(im.coldens, o.N, 4 * m, cudaMemcpyDeviceToHost, st));
      if (im.p) CU_TRY(cudaMemcpyAsync(im.p, o.p, 4 * m, cudaMemcpyDeviceToHost, st));
      if (im.intensity)
        for (int b = 0; b < nb; ++b)
          CU_TRY(cudaMemcpyAsync(im.intensity + (size_t)b * im.capacity, o.I + (size_t)b * o.stride, 4 * m,
                                 cudaMemcpyDeviceToHost, st));
    }
    if (im.band_flux && im.mem == AIR_DEVICE)
      CU_TRY(cudaMemcpyAsync(im.band_flux, bw.vflux + (size_t)v * nb, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st));
  }
  CU_TRY(cudaMemcpyAsync(vflux.data(), bw.vflux, sizeof(double) * V * nb, cudaMemcpyDeviceToHost, st));
  CU_TRY(cudaMemcpyAsync(vsteps.data(), bw.vsteps, sizeof(unsigned long long) * V, cudaMemcpyDeviceToHost, st));
  CU_TRY(cudaStreamSynchronize(st));
  for (int v = 0; v < V; ++v) {
    if (outs[v].band_flux && outs[v].mem == AIR_HOST)
      std::memcpy(outs[v].band_flux, vflux.data() + (size_t)v * nb, sizeof(double) * nb);
    outs[v].n_steps = (int64_t)vsteps[v];
  }
  CU_TRY(prof_resolve(g));
  g->last.valid = false;
  return AIR_OK;
}

void free_batch(air_grid *g) {
  BatchWork &bw = g->batch;
  if (bw.exec) cudaGraphExecDestroy(bw.exec);
  bw.exec = nullptr;
  if (bw.cap_stream) cudaStreamDestroy(bw.cap_stream);
  void *ps[] = {bw.geoms, bw.ctl, bw.bcnt, bw.refined, bw.vsweeps, bw.vsteps, bw.vflux, bw.outs, bw.boff};
  for (void *p : ps)
    if (p) cudaFree(p);
  if (bw.h_ctl) cudaFreeHost(bw.h_ctl);
  if (bw.h_geoms) cudaFreeHost(bw.h_geoms);
  bw = BatchWork{};
}

}  // namespace air

extern "C" air_status air_render_batch(air_grid *g, const air_view *views, int32_t n_views,
                                       const air_params *params, const air_batch_opts *opts,
                                       air_image *outs) {
  air::set_error(AIR_OK, "");
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  return air::render_batch(g, views, n_views, params, opts, outs);
}

extern "C" air_status air_render_batch_learned(air_grid *g, const air_view *views, int32_t n_views,
                                               const air_params *params, const air_batch_opts *opts,
                                               air_mlp *mlp, const air_learned_opts *lopts,
                                               air_image *outs, air_learned_stats *stats) {
  air::set_error(AIR_OK, "");
  if (!g) return air::set_error(AIR_ERR_ARG, "grid is NULL");
  if (!mlp) return air::set_error(AIR_ERR_ARG, "mlp is NULL");
  if (opts && opts->test_stall_barrier) return air::set_error(AIR_ERR_ARG, "test_stall_barrier is for air_render_batch");
  return air::render_batch(g, views, n_views, params, opts, outs, mlp, lopts, stats);
}
