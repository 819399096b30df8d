// air_march.cu -- launches of the per-ray march (device code in air_march.cuh).
#include "air_march.cuh"
#include "air_refine.cuh"

namespace air {

// Resident blocks per SM of the one-band kernels of rays parallel to an axis
// (DIR = 1 + A). Measured on the cone-shock bench image, one process, each
// variant twice (AIR / fixed 4096^2 image, ms): 12 blocks with 8-cell groups
// 5.39 / 4.89, 10 blocks 5.22 / 4.82, 8 blocks 5.02 / 4.30, 8 blocks with
// 16-cell groups 4.92 / 4.37 (the form kept). A separate form for launches
// of at most one wave (more registers, deeper load groups) is then the same
// kernel, so there is one.
constexpr int kAxisBlocks = 8;

template <int NBT, int DIR>
struct MinBlocks {
  static constexpr int value = DIR >= 1 ? kAxisBlocks
                               : (NBT <= 1 ? 6 : (NBT <= 2 ? 5 : (NBT <= 4 ? 4 : (NBT <= 8 ? 3 : 2))));
};

constexpr int kMarchBlock = 128;

// Node k's ray: trace it and store its column density, step count and band
// intensities (and their sum when one chunk holds every band).
template <int NBT, bool AMR, int FMT, int DIR>
__device__ __forceinline__ void march_one(const GridView &g, const RayGeom &rg, const RaySource &src,
                                          const RayOut &out, int fp64_level, const BandCtx &bc,
                                          const BandRegs<NBT> &br, int chunk, int b0, int nbh,
                                          int64_t k) {
  if (src.use_prop) {
    // the pixel's values from the proposal wave when it traced the pixel
    // (the same trace, so the same bits); else trace it here
    const Proposal &pr = src.prop;
    const int L = src.lvl[k], i = src.pi[k], j = src.pj[k];
    const int64_t b = (int64_t)(j >> L) * src.n0 + (i >> L);
    const int64_t q = prop_index(pr.depth + 4 * b, pr.off[b], L, i, j);
    if (q >= 0) {
      if (chunk == 0) {
        out.N[k] = pr.N[q];
        out.steps[k] = pr.steps[q];
      }
      for (int c = 0; c < nbh; ++c)
        out.I[(int64_t)(b0 + c) * out.stride + k] = pr.I[(int64_t)(b0 + c) * pr.stride + q];
      if (out.p && gridDim.y == 1) out.p[k] = pr.p[q];
      return;
    }
    if (chunk == 0) atomicAdd(&src.sweep->fb_sweep, 1ull);
  }
  RTState<NBT> st;
  trace_ray<NBT, AMR, FMT, DIR>(st, g, rg, src.lvl[k], src.pi[k], src.pj[k], fp64_level, bc, br);
  if (chunk == 0) {
    out.N[k] = st.N;
    out.steps[k] = st.steps;
    if (out.tau0) out.tau0[k] = br.kap[0] * st.N;
    if (out.maxlev) out.maxlev[k] = (uint8_t)st.maxlev;
  }
#pragma unroll
  for (int b = 0; b < NBT; ++b)
    if (b < nbh) out.I[(int64_t)(b0 + b) * out.stride + (k - out.ioff)] = st.I[b];
  if (out.p && gridDim.y == 1) {
    float p = 0.f;
#pragma unroll
    for (int b = 0; b < NBT; ++b)
      if (b < nbh) p += st.I[b];
    out.p[k] = p;
  }
}

template <int NBT, bool AMR, int FMT, int DIR>
__global__ void __launch_bounds__(kMarchBlock, MinBlocks<NBT, DIR>::value)
    k_march(GridView g, RayGeom rg, RaySource src, RayOut out, int fp64_level) {
  extern __shared__ float smem[];
  wait_prior_grid();
  const int chunk = blockIdx.y;
  const int b0 = chunk * NBT;
  const int nbh = min(NBT, g.n_bands - b0);
  const int tstride = g.n_tbins + 1;
  BandCtx bc;
  bc.tab = smem;
  bc.tstride = tstride;
  bc.nbh = nbh;
  if (FMT == kCellXq)
    for (int x = threadIdx.x; x < nbh * tstride; x += blockDim.x) smem[x] = g.table[b0 * tstride + x];
  BandRegs<NBT> br;
  band_regs<NBT>(br, g.kappa, g.invkappa, b0, nbh);
  __syncthreads();

  if (src.mode == 2) {
    // new nodes of a sweep counted on the device: blocks take chunks of
    // blockDim.x rays from a work counter until the rays run out
    // (with src.advance, the last block to finish moves the state on to the
    // next sweep)
    SweepState *S = src.sweep;
    if (S->done) return;
    const int64_t count = 4 * S->tot[0], first = S->n;
    __shared__ long long s_chunk;
    for (;;) {
      if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(S->ray_ctr + chunk, 1ull);
      __syncthreads();
      const int64_t r0 = (int64_t)s_chunk * blockDim.x;
      __syncthreads();
      if (r0 >= count) break;
      const int64_t r = r0 + threadIdx.x;
      if (r < count) march_one<NBT, AMR, FMT, DIR>(g, rg, src, out, fp64_level, bc, br, chunk, b0,
                                                   nbh, first + r);
    }
    if (src.advance && threadIdx.x == 0) sweep_block_finished(S, gridDim.x * gridDim.y);
    return;
  }
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int L, i, j;
  int64_t k;
  if (src.mode == 0) {
    if (r >= src.count) return;
    k = src.list ? (int64_t)src.list[r] : src.first + r;
    L = src.lvl[k];
    i = src.pi[k];
    j = src.pj[k];
  } else {
    const int res = src.n0;
    const int tw = src.tile_w, th = 32 / tw;
    const int tiles_x = (res + tw - 1) / tw;
    const int64_t warp = r >> 5;
    const int lane = (int)(r & 31);
    const int64_t ty = warp / tiles_x;
    const int tx = (int)(warp - ty * tiles_x);
    i = tx * tw + lane % tw;
    j = (int)ty * th + lane / tw;
    if (i >= res || j >= res) return;
    k = (int64_t)j * res + i;
    L = 0;
  }
  RTState<NBT> st;
  trace_ray<NBT, AMR, FMT, DIR>(st, g, rg, L, i, j, fp64_level, bc, br);
  if (chunk == 0) {
    out.N[k] = st.N;
    out.steps[k] = st.steps;
    if (out.tau0) out.tau0[k] = br.kap[0] * st.N;
    if (out.maxlev) out.maxlev[k] = (uint8_t)st.maxlev;
  }
#pragma unroll
  for (int b = 0; b < NBT; ++b)
    if (b < nbh) out.I[(int64_t)(b0 + b) * out.stride + (k - out.ioff)] = st.I[b];
  if (out.p && gridDim.y == 1) {
    float p = 0.f;
#pragma unroll
    for (int b = 0; b < NBT; ++b)
      if (b < nbh) p += st.I[b];
    out.p[k] = p;
  }
}

__global__ void k_band_sum(const float *__restrict__ I, int n_bands, int64_t stride, int64_t first,
                           int64_t count, const int32_t *__restrict__ list, float *__restrict__ p,
                           int64_t ioff) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= count) return;
  const int64_t k = list ? (int64_t)list[r] : first + r;
  float s = 0.f;
  for (int b = 0; b < n_bands; ++b) s += I[(int64_t)b * stride + (k - ioff)];
  p[k] = s;
}

// Band sums of a sweep counted on the device (rays [S->n, S->n + 4 S->tot[0])).
// The last block to finish moves the state on to the next sweep.
__global__ void k_band_sum_dev(const float *__restrict__ I, int n_bands, int64_t stride,
                               SweepState *__restrict__ S, float *__restrict__ p) {
  wait_prior_grid();
  if (S->done) return;
  const int64_t first = S->n, count = 4 * S->tot[0];
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  if (p)
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += step) {
      const int64_t k = first + r;
      float s = 0.f;
      for (int b = 0; b < n_bands; ++b) s += I[(int64_t)b * stride + k];
      p[k] = s;
    }
  __syncthreads();
  if (threadIdx.x == 0) sweep_block_finished(S, gridDim.x);
}

template <int NBT>
static cudaError_t launch_t(const GridView &g, const Camera &cam, const RaySource &src,
                            const RayOut &out, const MarchTune &tune, cudaStream_t st) {
  const int chunks = (g.n_bands + NBT - 1) / NBT;
  const bool dev = src.mode == 2;
  int64_t threads;
  if (src.mode == 0) {
    threads = src.count;
  } else if (src.mode == 1) {
    const int tw = src.tile_w, th = 32 / tw;
    const int64_t tiles = (int64_t)((src.n0 + tw - 1) / tw) * ((src.n0 + th - 1) / th);
    threads = tiles * 32;
  } else {
    threads = 1;  // the count is on the device; the grid is sized per form below
  }
  if (threads <= 0) return cudaSuccess;
  const int block = kMarchBlock;
  const int64_t blocks = (threads + block - 1) / block;
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  const size_t smem = g.cell_fmt == kCellXq ? sizeof(float) * (size_t)(NBT * (g.n_tbins + 1)) : 0;
  RayGeom rg = make_geom(g, cam, src.n0);
  rg.tab = src.axtab;
  rg.tab_slot = src.axtab_slot;
  rg.tab_byj = src.axtab_byj;
  const bool amr = g.kind == AIR_GRID_AMR;
  const int moving = (rg.Dhi[0] != 0.f) + (rg.Dhi[1] != 0.f) + (rg.Dhi[2] != 0.f);
  const int fp = tune.fp64_level;
  const int sms = sm_count();
  dim3 grid((unsigned)blocks, chunks);
  // device counts: a grid of one wave of the form's resident blocks, taking
  // work from the counter
#define AIR_GRID(D) \
  if (dev) grid = dim3((unsigned)(sms * MinBlocks<NBT, D>::value), chunks);
  // with the count on the device the march ends the sweep: the last block
  // advances the state, or the band sum after it does when bands are split
  RaySource s2 = src;
  s2.advance = dev && chunks == 1;
  cudaError_t le = cudaSuccess;
#define AIR_MARCH(N, A, F, D) \
  le = launch_pdl(k_march<N, A, F, D>, grid, dim3(block), smem, st, g, rg, s2, out, fp)
  if (NBT == 1 && moving == 1) {
    // every ray parallel to grid axis A: the compiled one-axis form DIR = 1 + A
    const int A = rg.Dhi[0] != 0.f ? 0 : (rg.Dhi[1] != 0.f ? 1 : 2);
#define AIR_AXIS(D)                                                                              \
  { AIR_GRID(D)                                                                                  \
  if (g.cell_fmt == kCellRho) { if (amr) AIR_MARCH(1, true, kCellRho, D); else AIR_MARCH(1, false, kCellRho, D); } \
  else if (g.cell_fmt == kCellXq) { if (amr) AIR_MARCH(1, true, kCellXq, D); else AIR_MARCH(1, false, kCellXq, D); } \
  else { if (amr) AIR_MARCH(1, true, kCellLam, D); else AIR_MARCH(1, false, kCellLam, D); } }
    if (A == 0) AIR_AXIS(1)
    else if (A == 1) AIR_AXIS(2)
    else AIR_AXIS(3)
#undef AIR_AXIS
  } else {
    AIR_GRID(0)
    if (g.cell_fmt == kCellRho) {
      if (amr) AIR_MARCH(NBT, true, kCellRho, 0); else AIR_MARCH(NBT, false, kCellRho, 0);
    } else if (g.cell_fmt == kCellXq) {
      if (amr) AIR_MARCH(NBT, true, kCellXq, 0); else AIR_MARCH(NBT, false, kCellXq, 0);
    } else {
      // per-cell Lambda exists for one-band grids only
      if (NBT != 1) return cudaErrorInvalidValue;
      if (amr) AIR_MARCH(1, true, kCellLam, 0); else AIR_MARCH(1, false, kCellLam, 0);
    }
  }
#undef AIR_MARCH
#undef AIR_GRID
  if (le != cudaSuccess) return le;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (dev && chunks > 1)  // band sums (if wanted), and the state moves on
    return launch_pdl(k_band_sum_dev, dim3((unsigned)(sms * 8)), dim3(256), 0, st,
                      (const float *)out.I, g.n_bands, out.stride, src.sweep, out.p);
  if (chunks > 1 && out.p) {
    if (dev) {
      return launch_pdl(k_band_sum_dev, dim3((unsigned)(sms * 8)), dim3(256), 0, st,
                        (const float *)out.I, g.n_bands, out.stride, src.sweep, out.p);
    }
    const int64_t first = src.mode == 0 ? src.first : 0;
    const int64_t count = src.mode == 0 ? src.count : (int64_t)src.n0 * src.n0;
    if (src.list) {
      k_band_sum<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(out.I, g.n_bands, out.stride, 0,
                                                                  count, src.list, out.p, out.ioff);
      return cudaGetLastError();
    }
    return launch_band_sum(out.I, g.n_bands, out.stride, first, count, out.p, st, out.ioff);
  }
  return cudaSuccess;
}

cudaError_t launch_march(const GridView &g, const Camera &cam, const RaySource &src,
                         const RayOut &out, const MarchTune &tune, cudaStream_t st) {
  // default: every band in one thread up to 8 bands, chunks of 8 above
  // (32-band adaptive / fixed images of the large grid, one view: 4 bands
  // 1315 / 1365 ms, 8 bands 1251 / 1328 ms, 16 bands 1512 / 1653 ms)
  int nbt = tune.nbt;
  if (nbt <= 0) nbt = default_bands_per_thread(g.n_bands);
  if (g.cell_fmt == kCellLam) nbt = 1;  // one band
  if (nbt <= 1) return launch_t<1>(g, cam, src, out, tune, st);
  if (nbt <= 2) return launch_t<2>(g, cam, src, out, tune, st);
  if (nbt <= 4) return launch_t<4>(g, cam, src, out, tune, st);
  if (nbt <= 8) return launch_t<8>(g, cam, src, out, tune, st);
  return launch_t<16>(g, cam, src, out, tune, st);
}

// Column-table entries (axis_table_entry), one per thread.
__global__ void k_axis_table(GridView g, RayGeom rg, int A, int byj, int n0, int64_t slot,
                             int32_t *tab) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= 2 * slot) return;
  const int s = x >= slot ? 1 : 0;
  const int64_t e = x - s * slot;
  int L = 0;
  while ((int64_t)n0 * ((((int64_t)1) << (L + 1)) - 1) <= e) ++L;
  const int p = (int)(e - (int64_t)n0 * ((((int64_t)1) << L) - 1));
  tab[x] = axis_table_entry(g, rg, (A + 1 + s) % 3, L, p, (byj >> s) & 1);
}

cudaError_t launch_axis_table(const GridView &g, const Camera &cam, int n0, int lmax,
                              int32_t *tab, int *byj, int64_t *slot, bool *ok, cudaStream_t st) {
  const RayGeom rg = make_geom(g, cam, n0);
  int A = 0;
  *ok = axis_table_view(rg, &A, byj);
  *slot = axis_table_slot(n0, lmax);
  if (!*ok) return cudaSuccess;
  const int64_t n = 2 * *slot;
  k_axis_table<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, rg, A, *byj, n0, *slot, tab);
  return cudaGetLastError();
}

cudaError_t launch_band_sum(const float *I, int n_bands, int64_t stride, int64_t first,
                            int64_t count, float *p, cudaStream_t st, int64_t ioff) {
  if (count <= 0) return cudaSuccess;
  const int block = 256;
  k_band_sum<<<(unsigned)((count + block - 1) / block), block, 0, st>>>(I, n_bands, stride, first,
                                                                       count, nullptr, p, ioff);
  return cudaGetLastError();
}

}  // namespace air
