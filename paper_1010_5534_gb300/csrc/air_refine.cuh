// air_refine.cuh -- image quadtree layout and the refinement launchers.
#pragma once
#include "air_internal.cuh"

namespace air {

constexpr int kScanBlock = 256;
constexpr int kScanRounds = 2;
constexpr int kScanItems = kScanBlock * kScanRounds;
constexpr int kBalanceStack = 8 * kMaxLevels;

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
cudaError_t launch_list_scan(const TreeView &t, const int32_t *open, int64_t m, double xi_crit,
                             int xi_norm, int refine_on, uint32_t *flag, cudaStream_t st);
cudaError_t launch_list_balance(const TreeView &t, const int32_t *open, int64_t m, uint32_t *flag,
                                uint32_t *err, cudaStream_t st);
// totals[0] flagged, [1] kept, [2] flagged with children below the top level;
// bcount / boff hold 3 x scan_blocks(m) entries.
cudaError_t launch_list_count(const TreeView &t, const int32_t *open, int64_t m,
                              const uint32_t *flag, int32_t *bcount, int64_t *boff,
                              int64_t *totals, cudaStream_t st);
// Children of the flagged entries at n_old + 4 * rank; the next list into `next`.
cudaError_t launch_list_emit(const TreeView &t, const int32_t *open, int64_t m, uint32_t *flag,
                             const int64_t *boff, const int64_t *totals, int64_t n_old,
                             int32_t *next, cudaStream_t st);
int64_t flux_blocks(int64_t n);
cudaError_t launch_flux(FluxArgs a, double *flux, double *steps, cudaStream_t st);

}  // namespace air
