// air_internal.cuh -- device-side data layout and helpers shared by the
// library's translation units (grid upload, march, refinement, API).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/air.h"

namespace air {

constexpr int kMaxBands = 64;
constexpr int kMaxLevels = 16;
constexpr int kXqFracBits = 24;  // table coordinate fixed point: 8 integer, 24 fraction bits
constexpr int kMapLevelShift = 27;  // brick map entry: id | level << 27
constexpr int32_t kMapIdMask = (1 << kMapLevelShift) - 1;
enum { kCellRho = 0, kCellLam = 1, kCellXq = 2 };

// Grid as the kernels see it. Positions are in units of the finest cell
// (uniform: the cell), F = (x - lo) / h per axis.
struct GridView {
  int kind;             // AIR_GRID_UNIFORM / AIR_GRID_AMR
  int nf[3];            // finest cells per axis
  double lo[3], h[3];   // world origin and finest cell size
  // cell fields, one record per cell (cell_fmt):
  //   kCellRho  : float rho                                 (emission j = rho^2)
  //   kCellLam  : float2 {rho, rho Lambda(T)}               (one band, Lambda
  //               interpolated and multiplied by rho once per cell at upload,
  //               in FP64)
  //   kCellXq   : uint2 {rho bits, xq}, xq = round(x 2^24) the fixed-point
  //               table coordinate of T, x = (log10 T - logT_lo) / dlogT in bins
  const void *cells;
  int cell_fmt;
  // block AMR
  int B, log2B, Lm;     // brick edge (cells), log2 of it, finest level
  int nb0[3];           // level-0 bricks per axis
  const int32_t *base;  // [nb0z][nb0y][nb0x]: >= 0 leaf brick id, < 0 -(group + 1)
  const int32_t *oct;   // [groups][8] children codes (octant = bx | by<<1 | bz<<2)
  const int32_t *bmap;  // dense map at level mapL: id | level << 27, or -(group + 1)
  int mapL, nm[3];      // map level and map positions per axis
  // emission
  int emis_mode, n_bands, n_tbins;
  const float *table;   // [n_bands][n_tbins + 1] (last entry repeated)
  const float *kappa;   // [n_bands]
  const float *invkappa;// [n_bands] (0 where kappa == 0)
};

// Orthographic camera resolved on the host in FP64.
struct Camera {
  double c[3], u[3], v[3], d[3];
  double H;
};

struct SweepState;

// A learned depth proposal traced in one wave (air_learned.cu). Each base
// pixel b of an n0 x n0 image has four quadrants, its level-1 pixels
// (2 bi + (q & 1), 2 bj + (q >> 1)), q = 0..3, and quadrant q was proposed to
// depth depth[4 b + q] (an image level, 0..max_level). The rays traced for b,
// from ray off[b] on: its four level-1 pixels when any quadrant's depth is at
// least 1, then for q = 0..3 the full subtree of depth depth[4 b + q] - 1
// below level-1 pixel q (image levels 2 .. depth[4 b + q]), level by level and
// row-major within a level. Values of proposal ray r: N[r], I[c * stride + r]
// (band c), p[r], steps[r].
struct Proposal {
  const int8_t *depth;
  const int64_t *off;
  const float *N, *I, *p;
  const uint32_t *steps;
  int64_t stride;
};

// Rays in the full subtree of depth d below one pixel: 4 + 16 + ... + 4^d.
__host__ __device__ __forceinline__ int64_t prop_subtree(int d) {
  return ((int64_t)1 << (2 * d + 2)) / 3 - 1;
}
// Offset of level L (1..d) inside such a subtree.
__host__ __device__ __forceinline__ int64_t prop_level_offset(int L) {
  return L <= 1 ? 0 : prop_subtree(L - 1);
}
__host__ __device__ __forceinline__ int prop_max_depth(const int8_t *d4) {
  int m = d4[0];
  for (int q = 1; q < 4; ++q) m = d4[q] > m ? d4[q] : m;
  return m;
}
// Rays of one base pixel's proposal, from its quadrant depths d4[0..3].
__host__ __device__ __forceinline__ int64_t prop_rays(const int8_t *d4) {
  if (prop_max_depth(d4) < 1) return 0;
  int64_t s = 4;
  for (int q = 0; q < 4; ++q) s += d4[q] > 1 ? prop_subtree(d4[q] - 1) : 0;
  return s;
}
// Pixel (L, i, j) of ray r (0 <= r < prop_rays(d4)) of base pixel (bi, bj)'s
// proposal: the four level-1 pixels first, then each quadrant's subtree level
// by level, row-major within a level. prop_index inverts it.
__host__ __device__ __forceinline__ void prop_ray(const int8_t *d4, int64_t r, int bi, int bj,
                                                  int &L, int &i, int &j) {
  if (r < 4) {
    L = 1;
    i = 2 * bi + (int)(r & 1);
    j = 2 * bj + (int)(r >> 1);
    return;
  }
  int64_t rr = r - 4;
  int q = 0;
  while (q < 3) {
    const int64_t sz = d4[q] > 1 ? prop_subtree(d4[q] - 1) : 0;
    if (rr < sz) break;
    rr -= sz;
    ++q;
  }
  const int e = d4[q] - 1;  // the quadrant's subtree depth (>= 1 here)
  int Lr = 1;
  while (Lr < e && rr >= prop_level_offset(Lr + 1)) ++Lr;
  const int64_t loc = rr - prop_level_offset(Lr);
  const int w = 1 << Lr;
  L = Lr + 1;
  i = ((2 * bi + (q & 1)) << Lr) + (int)(loc % w);
  j = ((2 * bj + (q >> 1)) << Lr) + (int)(loc / w);
}

// Ray of pixel (L, i, j), L >= 1, in the proposal of the base pixel that
// holds it (quadrant depths d4, first ray off), or -1 if it was not traced.
__host__ __device__ __forceinline__ int64_t prop_index(const int8_t *d4, int64_t off, int L, int i,
                                                       int j) {
  if (L < 1) return -1;
  const int i1 = i >> (L - 1), j1 = j >> (L - 1);
  const int q = (i1 & 1) + 2 * (j1 & 1);
  if (L == 1) return prop_max_depth(d4) >= 1 ? off + q : -1;
  if (L > d4[q]) return -1;
  int64_t o = off + 4;
  for (int r = 0; r < q; ++r) o += d4[r] > 1 ? prop_subtree(d4[r] - 1) : 0;
  const int Lr = L - 1;  // level below the quadrant's level-1 pixel
  return o + prop_level_offset(Lr) + (int64_t)(j - (j1 << Lr)) * (1 << Lr) + (i - (i1 << Lr));
}

// Ray list: explicit nodes (level, i, j) of an n0 base image, the implicit
// pixels of a res x res fixed image, or the new nodes of a sweep whose count
// stays on the device.
struct RaySource {
  int mode;             // 0 nodes, 1 fixed grid, 2 nodes counted on the device
  int n0;               // base resolution (nodes) or res (grid)
  const int8_t *lvl;
  const int32_t *pi, *pj;
  int64_t first, count; // rays [first, first + count) of the list / image (modes 0, 1)
  int tile_w;           // grid mode: a warp covers tile_w x (32 / tile_w) pixels
  const int32_t *list;  // nodes mode: if set, ray r is node list[r] (first ignored)
  SweepState *sweep;    // mode 2: rays [S->n, S->n + 4 S->tot[0]), none once S->done;
                        // blocks take 128-ray chunks from S->ray_ctr[band chunk]
  int advance;          // mode 2: the launch's last block moves S on to the next sweep
  int use_prop;         // mode 2: copy a new pixel's values from `prop` when the
  Proposal prop;        // proposal traced it; trace only the pixels it missed
  // column table of an axis view (RayGeom::tab, levels of the n0 image), or NULL
  const int32_t *axtab;
  int64_t axtab_slot;
  int axtab_byj;
};

struct RayOut {
  float *N;             // [stride] column density
  float *I;             // [n_bands][stride]
  int64_t stride;
  uint32_t *steps;      // [stride]
  float *p;             // [stride] band-summed intensity (NULL: written elsewhere)
  float *tau0;          // [stride] optical depth of band 0 through the grid (optional)
  uint8_t *maxlev;      // [stride] deepest brick level the ray crossed (optional)
  int64_t ioff;         // node k's intensities sit at I[b * stride + k - ioff] (a
                        // staging buffer for the nodes from ioff on; 0 otherwise)
};

struct MarchTune {
  int block;            // threads per block
  int fp64_level;       // bricks at this level or deeper use FP64 entry/exit
  int nbt;              // bands one thread carries (1, 2, 4, 8, 16; 0 = all up to 8, else 8)
};

// Kahan-compensated sum: s += x with running compensation c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  float y = x - c;
  float t = s + y;
  c = (t - s) - y;
  s = t;
}

// (1 - e^-x) / x for 0 <= x < 0.25 from its Taylor series
// sum_{n>=0} (-x)^n / (n+1)!, truncated after x^6 (remainder < x^7/8! < 1.6e-9).
__device__ __forceinline__ float one_minus_exp_over_x(float x) {
  float g = 1.0f / 5040.0f;
  g = fmaf(g, -x, 1.0f / 720.0f);
  g = fmaf(g, -x, 1.0f / 120.0f);
  g = fmaf(g, -x, 1.0f / 24.0f);
  g = fmaf(g, -x, 1.0f / 6.0f);
  g = fmaf(g, -x, 0.5f);
  g = fmaf(g, -x, 1.0f);
  return g;
}

}  // namespace air

// ---- host-side internal API between translation units ----------------------
namespace air {

struct DeviceGrid;  // owned by the handle (defined in air_grid.cu)

// Streaming multiprocessors of the current device (read once; 1 if the query fails).
int sm_count();

// Entries per fixed axis of a column table for levels 0 .. lmax of an n0 image.
inline int64_t axis_table_slot(int n0, int lmax) {
  return (int64_t)n0 * ((((int64_t)1) << (lmax + 1)) - 1);
}
// Column table of an axis view (RayGeom::tab) for levels 0 .. lmax of an n0
// image into tab (2 * axis_table_slot(n0, lmax) entries); *ok = false (and
// nothing launched) when the view does not qualify.
cudaError_t launch_axis_table(const GridView &g, const Camera &cam, int n0, int lmax,
                              int32_t *tab, int *byj, int64_t *slot, bool *ok, cudaStream_t st);
cudaError_t launch_march(const GridView &g, const Camera &cam, const RaySource &src,
                         const RayOut &out, const MarchTune &tune, cudaStream_t st);
// Bands one thread carries when the tuning leaves it open (launch_march).
inline int default_bands_per_thread(int n_bands) { return n_bands <= 8 ? n_bands : 8; }
cudaError_t launch_band_sum(const float *I, int n_bands, int64_t stride, int64_t first,
                            int64_t count, float *p, cudaStream_t st, int64_t ioff = 0);

}  // namespace air
