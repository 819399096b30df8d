// air_refine.cuh -- image quadtree layout and the refinement launchers.
#pragma once
#include "air_internal.cuh"

namespace air {

constexpr int kScanBlock = 256;
constexpr int kScanRounds = 2;
constexpr int kScanItems = kScanBlock * kScanRounds;
constexpr int kBalanceStack = 8 * kMaxLevels;

// Offset of level l's map in the level maps of a single-view tree (levels
// 1 .. Lm - 1, each a dense (n0 2^l)^2 array of node indices); the maps of
// levels below Lm take level_map_offset(n0, Lm) entries.
__host__ __device__ inline int64_t level_map_offset(int n0, int l) {
  // sum over 1 <= l' < l of (n0 2^l')^2 = n0^2 (4^l - 4) / 3
  return l <= 1 ? 0 : (int64_t)n0 * n0 * ((((int64_t)1 << (2 * l)) - 4) / 3);
}

// Scan chunks (of kScanItems) covering n items.
__host__ __device__ inline int64_t scan_chunks(int64_t n) { return (n + kScanItems - 1) / kScanItems; }

// Node arrays of the image quadtree (capacity `cap`).
struct TreeView {
  int n0, Lm;
  int64_t cap;
  int8_t *lvl;
  int32_t *pi, *pj;
  int32_t *child;   // first child index, -1 for a leaf
  float *N;         // column density
  float *I;         // [n_bands][cap]
  float *p;         // band-summed intensity
  uint32_t *steps;
};

// Output arrays (device memory), entry r of `stride`.
struct OutView {
  int32_t *level, *i, *j;
  uint8_t *is_leaf;
  float *N, *p, *I;
  int64_t stride;
  int n_bands;
};

struct FluxArgs {
  int64_t n;             // nodes or pixels
  const int32_t *child;  // NULL: every entry is a leaf
  const int8_t *lvl;     // NULL: level 0
  const float *I;        // [n_bands][stride]
  int64_t stride;
  const uint32_t *steps;
  int n_bands;
  double area0;          // pixel area at level 0
  double *partial;       // [blocks][n_bands + 1]
  int64_t per_block;
};

// Device-resident bookkeeping of the sweep loop when the counts stay on the
// device (render_adaptive without a read-back per sweep). Every kernel of a
// sweep reads its item count here; once `done` is set, every later kernel
// returns at once, so sweeps queued past the end do nothing.
struct SweepState {
  long long n;          // traced nodes so far
  long long m;          // length of the current open-leaf list
  long long n_refined;  // refined nodes so far
  long long tot[3];     // this sweep: flagged, kept, flagged with children below the top level
  int cur;              // which open-leaf list is current (0 or 1)
  int sweeps;           // sweeps that refined something
  int done;             // the last scan flagged nothing (or nothing is left to scan)
  unsigned blocks_done; // blocks of the sweep's last kernel that have finished
  unsigned long long ray_ctr[kMaxBands];  // march work counters, one per band chunk
  // with a learned proposal: pixels it missed, traced this sweep / in all
  // sweeps, and the sweeps that traced any
  unsigned long long fb_sweep, fb_total;
  int fb_waves;
};

// After the new pixels are traced: n, m, cur, sweeps and n_refined move on to
// the next sweep, and the work counters are reset. Run by one thread once no
// other thread of the sweep reads the state any more.
__device__ __forceinline__ void sweep_advance(SweepState *S) {
  const long long nflag = S->tot[0];
  S->n += 4 * nflag;
  S->n_refined += nflag;
  S->m = S->tot[1] + 4 * S->tot[2];
  S->cur ^= 1;
  S->sweeps += 1;
  if (S->m == 0) S->done = 1;  // no leaf below the top level is left
  for (int b = 0; b < kMaxBands; ++b) S->ray_ctr[b] = 0ull;
  S->blocks_done = 0u;
  if (S->fb_sweep) {
    S->fb_total += S->fb_sweep;
    S->fb_waves += 1;
    S->fb_sweep = 0ull;
  }
}

// Called by thread 0 of every block of the sweep's last kernel as the block
// finishes (after a __syncthreads): the last block to finish advances.
__device__ __forceinline__ void sweep_block_finished(SweepState *S, unsigned nblocks) {
  __threadfence();
  if (atomicAdd(&S->blocks_done, 1u) == nblocks - 1u) sweep_advance(S);
}

// Programmatic dependent launch: a kernel of the sweep chain waits here for
// the kernel before it (launched with cudaLaunchAttributeProgrammaticStream-
// Serialization, the wait returns once that kernel has completed and its
// memory is visible; launched without it, the wait returns at once).
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with programmatic stream serialization: the kernel may be scheduled
// while the one before it in the stream is finishing, and waits for it in
// wait_prior_grid(), so the launch latency between the short kernels of a
// sweep overlaps the previous kernel's tail.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_init_base(const TreeView &t, cudaStream_t st);
int64_t scan_blocks(int64_t n);
cudaError_t launch_count_flags(const uint32_t *flag, int64_t n, int32_t *bcount, int64_t *boff,
                               int64_t *total, cudaStream_t st);
cudaError_t launch_count_leaves(const TreeView &t, int all, int64_t n, int32_t *bcount,
                                int64_t *boff, int64_t *total, cudaStream_t st);
cudaError_t launch_emit_out(const TreeView &t, const OutView &o, int all, int64_t n,
                            const int64_t *boff, cudaStream_t st);
// Exclusive scan of nb per-block counts (one block) -> boff, total.
cudaError_t launch_scan_offsets(const int32_t *bcount, int64_t nb, int64_t *boff, int64_t *total,
                                cudaStream_t st);
// Open-leaf list (leaves below the top level, ascending): steps iii-iv over it.
cudaError_t launch_list_init(int32_t *list, int64_t m, cudaStream_t st);
// lmap: level maps of a single-view tree (see air_tree.cuh), or NULL to find
// stencil neighbours by descent through the child links.
cudaError_t launch_list_scan(const TreeView &t, const int32_t *open, int64_t m, double xi_crit,
                             int xi_norm, int refine_on, uint32_t *flag, cudaStream_t st,
                             const int32_t *lmap = nullptr);
cudaError_t launch_list_balance(const TreeView &t, const int32_t *open, int64_t m, uint32_t *flag,
                                uint32_t *err, cudaStream_t st, const int32_t *lmap = nullptr);
// totals[0] flagged, [1] kept, [2] flagged with children below the top level;
// bcount / boff hold 3 x scan_blocks(m) entries.
cudaError_t launch_list_count(const TreeView &t, const int32_t *open, int64_t m,
                              const uint32_t *flag, int32_t *bcount, int64_t *boff,
                              int64_t *totals, cudaStream_t st);
// Children of the flagged entries at n_old + 4 * rank; the next list into `next`.
cudaError_t launch_list_emit(const TreeView &t, const int32_t *open, int64_t m, uint32_t *flag,
                             const int64_t *boff, const int64_t *totals, int64_t n_old,
                             int32_t *next, cudaStream_t st, int32_t *lmap = nullptr);
// The same steps with every count read from the device (SweepState S; the
// current list is open[S->cur], the next one open[S->cur ^ 1]). Grids are
// sized for the GPU, not for the count, and loop over the items. nb_cap:
// scan blocks the count arrays hold per selection (scan_blocks of the
// largest list).
cudaError_t launch_sweep_scan(const TreeView &t, int32_t *const open[2], const SweepState *S,
                              double xi_crit, int xi_norm, int refine_on, uint32_t *flag,
                              cudaStream_t st, const int32_t *lmap);
// Scan and balance fused (the open list's flags must be zero on entry).
cudaError_t launch_sweep_scan_balance(const TreeView &t, int32_t *const open[2],
                                      const SweepState *S, double xi_crit, int xi_norm,
                                      int refine_on, uint32_t *flag, uint32_t *err,
                                      cudaStream_t st, const int32_t *lmap);
cudaError_t launch_sweep_balance(const TreeView &t, int32_t *const open[2], const SweepState *S,
                                 uint32_t *flag, uint32_t *err, cudaStream_t st,
                                 const int32_t *lmap);
// Count the three selections and scan them; S->tot and S->done are set.
cudaError_t launch_sweep_count(const TreeView &t, int32_t *const open[2], SweepState *S,
                               const uint32_t *flag, int32_t *bcount, int64_t *boff,
                               int64_t nb_cap, cudaStream_t st);
cudaError_t launch_sweep_emit(const TreeView &t, int32_t *const open[2], const SweepState *S,
                              uint32_t *flag, const int64_t *boff, int64_t nb_cap,
                              cudaStream_t st, int32_t *lmap);
int64_t flux_blocks(int64_t n);
cudaError_t launch_flux(FluxArgs a, double *flux, double *steps, cudaStream_t st);

}  // namespace air
