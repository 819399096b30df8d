// air_grid.cu -- Section 2 step i: read the simulation grid, lay it out on the
// device and build the brick lookup.
//
// Device layout (resident for the handle's lifetime):
//   rho : float per cell. Uniform grid [nz][ny][nx]; AMR brick-major
//         [brick][z][y][x], so a warp of neighbouring rays reads neighbouring
//         words of one brick.
//   xq  : uint32 per cell (emis_mode 1 only): the emission-table coordinate of
//         T, x = (log10 T - logT_lo) / (logT_hi - logT_lo) * (n_tbins - 1),
//         clamped to [0, n_tbins - 1], in fixed point with 24 fraction bits.
//         The bin index and weight then come out exactly in FP32.
//   base: level-0 brick grid; entries >= 0 are leaf bricks, < 0 point to a
//         group of 8 child slots in `oct` (octant = bx | by << 1 | bz << 2).
//   bmap: dense brick map at level mapL (the finest level whose brick grid has
//         at most 2^24 positions): per brick position, the leaf brick covering
//         it as id | level << 27, or -(group + 1) where the octree continues
//         below mapL. The march finds most bricks with this one load.
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "air_handle.cuh"

namespace air {

// Raw fields -> cell records (see GridView::cell_fmt). The table coordinate
// of T is x = (log10 T - logT_lo) / dlogT * (n_tbins - 1), clamped; for one
// band the record holds rho Lambda with Lambda = (1 - w) tab[k] + w tab[k + 1],
// k = floor(x) (at most n_tbins - 2) and w = x - k, formed in FP64 from the
// stored FP32 rho and rounded once to FP32 (every transfer form uses Lambda
// only in the product rho Lambda).
template <typename T>
__global__ void k_convert_fields(const T *__restrict__ rho_in, const T *__restrict__ t_in,
                                 int64_t n, int fmt, void *__restrict__ out, double logT_lo,
                                 double dlogT, int n_tbins, const float *__restrict__ tab0,
                                 unsigned long long *__restrict__ bad) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double r = (double)rho_in[k];
  bool ok = isfinite(r) && r >= 0.0;
  const float rf = ok ? (float)r : 0.f;
  if (fmt == kCellRho) {
    ((float *)out)[k] = rf;
  } else {
    const double Tv = (double)t_in[k];
    const bool tok = isfinite(Tv) && Tv > 0.0;
    ok = ok && tok;
    double x = tok ? (log10(Tv) - logT_lo) / dlogT * (double)(n_tbins - 1) : 0.0;
    if (!(x > 0.0)) x = 0.0;
    if (x > (double)(n_tbins - 1)) x = (double)(n_tbins - 1);
    uint32_t aux;
    if (fmt == kCellLam) {
      int kk = (int)floor(x);
      if (kk > n_tbins - 2) kk = n_tbins - 2;
      const double w = x - (double)kk;
      const double lam = (1.0 - w) * (double)tab0[kk] + w * (double)tab0[kk + 1];
      aux = __float_as_uint((float)((double)rf * lam));
    } else {
      aux = (uint32_t)rint(x * (double)(1u << kXqFracBits));
    }
    ((uint2 *)out)[k] = make_uint2(__float_as_uint(rf), aux);
  }
  if (!ok) atomicAdd(bad, 1ull);
}

namespace {

constexpr int32_t kUnset = INT32_MIN;

struct OctBuild {
  std::vector<int32_t> base, oct;
  std::string err;
};

inline int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return (1 << l) == v ? l : -1;
}

// Brick octree from the leaf list; every slot must end up filled exactly once.
bool build_octree(const air_grid_desc *d, OctBuild &ob) {
  const int B = d->brick, Lm = d->max_level, lb = ilog2(B);
  int nb0[3];
  for (int a = 0; a < 3; ++a) nb0[a] = d->n[a] / B;
  ob.base.assign((size_t)nb0[0] * nb0[1] * nb0[2], kUnset);
  ob.oct.clear();
  for (int b = 0; b < d->n_bricks; ++b) {
    const int l = d->brick_level[b];
    if (l < 0 || l > Lm) { ob.err = "brick level out of range"; return false; }
    const int64_t S = (int64_t)B << (Lm - l);
    int64_t o[3];
    for (int a = 0; a < 3; ++a) {
      o[a] = d->brick_origin[3 * (int64_t)b + a];
      const int64_t nf = (int64_t)d->n[a] << Lm;
      if (o[a] < 0 || o[a] % S || o[a] + S > nf) { ob.err = "brick origin not aligned to its level or outside the grid"; return false; }
    }
    const int s0 = lb + Lm;
    const size_t bidx = ((size_t)(o[2] >> s0) * nb0[1] + (o[1] >> s0)) * nb0[0] + (o[0] >> s0);
    if (l == 0) {
      if (ob.base[bidx] != kUnset) { ob.err = "bricks overlap"; return false; }
      ob.base[bidx] = b;
      continue;
    }
    // walk (and create) the groups from level 0 down to the brick's parent
    int32_t code = ob.base[bidx];
    if (code >= 0) { ob.err = "bricks overlap"; return false; }
    int32_t grp;
    if (code == kUnset) {
      grp = (int32_t)(ob.oct.size() / 8);
      ob.oct.insert(ob.oct.end(), 8, kUnset);
      ob.base[bidx] = -(grp + 1);
    } else {
      grp = -code - 1;
    }
    for (int lev = 1; lev <= l; ++lev) {
      const int sh = s0 - lev;
      const int oc = (int)(((o[0] >> sh) & 1) | (((o[1] >> sh) & 1) << 1) | (((o[2] >> sh) & 1) << 2));
      const size_t si = (size_t)grp * 8 + oc;
      if (lev == l) {
        if (ob.oct[si] != kUnset) { ob.err = "bricks overlap"; return false; }
        ob.oct[si] = b;
      } else {
        code = ob.oct[si];
        if (code >= 0) { ob.err = "bricks overlap"; return false; }
        if (code == kUnset) {
          const int32_t g2 = (int32_t)(ob.oct.size() / 8);
          ob.oct.insert(ob.oct.end(), 8, kUnset);
          ob.oct[si] = -(g2 + 1);
          grp = g2;
        } else {
          grp = -code - 1;
        }
      }
    }
  }
  for (int32_t v : ob.base)
    if (v == kUnset) { ob.err = "leaf bricks do not cover the grid"; return false; }
  for (int32_t v : ob.oct)
    if (v == kUnset) { ob.err = "leaf bricks do not cover the grid"; return false; }
  return true;
}

// Dense map of the octree at level mapL (positions in level-mapL brick units).
void fill_map(const OctBuild &ob, int32_t code, int lev, int64_t px, int64_t py, int64_t pz,
              int mapL, const int64_t nm[3], std::vector<int32_t> &map) {
  if (code >= 0) {
    const int s = mapL - lev;
    const int32_t e = code | (lev << kMapLevelShift);
    for (int64_t z = pz << s; z < (pz + 1) << s; ++z)
      for (int64_t y = py << s; y < (py + 1) << s; ++y)
        for (int64_t x = px << s; x < (px + 1) << s; ++x) map[(size_t)((z * nm[1] + y) * nm[0] + x)] = e;
    return;
  }
  if (lev == mapL) {
    map[(size_t)((pz * nm[1] + py) * nm[0] + px)] = code;
    return;
  }
  const int64_t grp = -(int64_t)code - 1;
  for (int oc = 0; oc < 8; ++oc)
    fill_map(ob, ob.oct[(size_t)grp * 8 + oc], lev + 1, 2 * px + (oc & 1), 2 * py + ((oc >> 1) & 1),
             2 * pz + ((oc >> 2) & 1), mapL, nm, map);
}

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

}  // namespace

void free_grid_impl(air_grid *g) {
  dfree(g->d_cells); dfree(g->d_base); dfree(g->d_oct); dfree(g->d_bmap);
  dfree(g->d_table); dfree(g->d_kappa); dfree(g->d_invkappa);
  dfree(g->raster.scratch);
  g->raster.ok = false;
  {
    SpectraWork &sp = g->spectra;
    if (sp.copy) cudaStreamSynchronize(sp.copy);
    for (int k = 0; k < 2; ++k) {
      dfree(sp.stage[k]);
      sp.stage_b[k] = 0;
      if (sp.marched[k]) cudaEventDestroy(sp.marched[k]);
      if (sp.copied[k]) cudaEventDestroy(sp.copied[k]);
      sp.marched[k] = sp.copied[k] = nullptr;
    }
    if (sp.copy) cudaStreamDestroy(sp.copy);
    sp.copy = nullptr;
  }
  free_batch(g);
  free_learn(g);
  Workspace &w = g->ws;
  dfree(w.view);
  dfree(w.lvl); dfree(w.pi); dfree(w.pj); dfree(w.child); dfree(w.N); dfree(w.I); dfree(w.p);
  dfree(w.steps); dfree(w.flag); dfree(w.bcount); dfree(w.boff); dfree(w.d_total); dfree(w.d_err);
  dfree(w.open[0]); dfree(w.open[1]); dfree(w.lmap); dfree(w.axtab);
  w.lmap_b = 0;
  dfree(w.partial); dfree(w.d_flux); dfree(w.fN); dfree(w.fI); dfree(w.fp); dfree(w.fsteps);
  dfree(w.o_level); dfree(w.o_i); dfree(w.o_j); dfree(w.o_leaf); dfree(w.o_N); dfree(w.o_p);
  dfree(w.o_I);
  dfree(w.d_sweep);
  if (w.h_sweep) cudaFreeHost(w.h_sweep);
  w.h_sweep = nullptr;
  for (int k = 0; k < 2; ++k) {
    if (w.ev_sweep[k]) cudaEventDestroy(w.ev_sweep[k]);
    w.ev_sweep[k] = nullptr;
  }
  if (w.h_total) cudaFreeHost(w.h_total);
  if (w.h_err) cudaFreeHost(w.h_err);
  if (w.h_flux) cudaFreeHost(w.h_flux);
  w.h_total = nullptr; w.h_err = nullptr; w.h_flux = nullptr;
  for (cudaEvent_t e : g->prof.ev) cudaEventDestroy(e);
  g->prof.ev.clear();
}

#define CU_TRY(x)                                          \
  do {                                                     \
    cudaError_t e_ = (x);                                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x);       \
  } while (0)

air_status load_grid_impl(const air_grid_desc *d, air_grid *g) {
  // ---- validate the description
  if (d->kind != AIR_GRID_UNIFORM && d->kind != AIR_GRID_AMR) return set_error(AIR_ERR_ARG, "unknown grid kind %d", d->kind);
  if (!d->rho) return set_error(AIR_ERR_ARG, "rho is NULL");
  if (d->field_dtype != AIR_F32 && d->field_dtype != AIR_F64) return set_error(AIR_ERR_ARG, "field_dtype must be AIR_F32 or AIR_F64");
  if (d->n_bands < 1 || d->n_bands > kMaxBands) return set_error(AIR_ERR_ARG, "n_bands must be in [1, %d]", kMaxBands);
  if (!d->kappa) return set_error(AIR_ERR_ARG, "kappa is NULL");
  for (int b = 0; b < d->n_bands; ++b)
    if (!std::isfinite(d->kappa[b]) || d->kappa[b] < 0.0) return set_error(AIR_ERR_ARG, "kappa[%d] must be finite and >= 0", b);
  if (d->emis_mode != 0 && d->emis_mode != 1) return set_error(AIR_ERR_ARG, "emis_mode must be 0 or 1");
  if (d->emis_mode == 1) {
    if (!d->temp || !d->lambda_table) return set_error(AIR_ERR_ARG, "emis_mode 1 needs temp and lambda_table");
    if (d->n_tbins < 2 || d->n_tbins > 255) return set_error(AIR_ERR_ARG, "n_tbins must be in [2, 255]");
    if (!(d->logT_hi > d->logT_lo) || !std::isfinite(d->logT_lo) || !std::isfinite(d->logT_hi)) return set_error(AIR_ERR_ARG, "need logT_lo < logT_hi");
    for (int64_t x = 0; x < (int64_t)d->n_bands * d->n_tbins; ++x)
      if (!std::isfinite(d->lambda_table[x]) || d->lambda_table[x] < 0.f) return set_error(AIR_ERR_ARG, "lambda_table must be finite and >= 0");
  }
  for (int a = 0; a < 3; ++a) {
    if (d->n[a] < 1) return set_error(AIR_ERR_ARG, "n[%d] must be >= 1", a);
    if (!(d->hi[a] > d->lo[a]) || !std::isfinite(d->lo[a]) || !std::isfinite(d->hi[a])) return set_error(AIR_ERR_ARG, "need lo < hi on axis %d", a);
  }
  int64_t n_cells = 0;
  GridView &v = g->gv;
  v = GridView{};
  v.kind = d->kind;
  OctBuild ob;
  if (d->kind == AIR_GRID_UNIFORM) {
    n_cells = (int64_t)d->n[0] * d->n[1] * d->n[2];
    if ((int64_t)d->n[0] * d->n[1] > INT32_MAX || n_cells > ((int64_t)1 << 40)) return set_error(AIR_ERR_ARG, "grid too large");
    for (int a = 0; a < 3; ++a) v.nf[a] = d->n[a];
  } else {
    const int lb = ilog2(d->brick);
    if (d->brick < 1 || lb < 0 || d->brick > 64) return set_error(AIR_ERR_ARG, "brick must be a power of two in [1, 64]");
    if (d->max_level < 0 || d->max_level >= kMaxLevels) return set_error(AIR_ERR_ARG, "max_level must be in [0, %d]", kMaxLevels - 1);
    if (d->n_bricks < 1 || !d->brick_level || !d->brick_origin) return set_error(AIR_ERR_ARG, "AMR grid needs n_bricks >= 1, brick_level and brick_origin");
    for (int a = 0; a < 3; ++a) {
      if (d->n[a] % d->brick) return set_error(AIR_ERR_ARG, "n[%d] is not a multiple of brick", a);
      if (((int64_t)d->n[a] << d->max_level) > (1 << 30)) return set_error(AIR_ERR_ARG, "finest grid too large");
      v.nf[a] = d->n[a] << d->max_level;
      v.nb0[a] = d->n[a] / d->brick;
    }
    if (d->n_bricks >= (1 << kMapLevelShift)) return set_error(AIR_ERR_ARG, "at most 2^27 - 1 bricks");
    if (!build_octree(d, ob)) return set_error(AIR_ERR_ARG, "%s", ob.err.c_str());
    n_cells = (int64_t)d->n_bricks * d->brick * d->brick * d->brick;
    v.B = d->brick;
    v.log2B = lb;
    v.Lm = d->max_level;
  }
  for (int a = 0; a < 3; ++a) {
    v.lo[a] = d->lo[a];
    v.h[a] = (d->hi[a] - d->lo[a]) / (double)v.nf[a];
  }
  v.emis_mode = d->emis_mode;
  v.n_bands = d->n_bands;
  v.n_tbins = d->emis_mode == 1 ? d->n_tbins : 1;
  g->n_cells = n_cells;

  // ---- device copies: emission table first (the upload of one-band grids uses it)
  {
    const int ts = v.n_tbins + 1;
    std::vector<float> tab((size_t)d->n_bands * ts, 0.f), kap(d->n_bands), ik(d->n_bands);
    if (d->emis_mode == 1)
      for (int b = 0; b < d->n_bands; ++b) {
        for (int x = 0; x < d->n_tbins; ++x) tab[(size_t)b * ts + x] = d->lambda_table[(size_t)b * d->n_tbins + x];
        tab[(size_t)b * ts + d->n_tbins] = d->lambda_table[(size_t)b * d->n_tbins + d->n_tbins - 1];
      }
    for (int b = 0; b < d->n_bands; ++b) {
      kap[b] = (float)d->kappa[b];
      ik[b] = d->kappa[b] > 0.0 ? (float)(1.0 / d->kappa[b]) : 0.f;
    }
    CU_TRY(cudaMalloc((void **)&g->d_table, sizeof(float) * tab.size()));
    CU_TRY(cudaMemcpy(g->d_table, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice));
    CU_TRY(cudaMalloc((void **)&g->d_kappa, sizeof(float) * kap.size()));
    CU_TRY(cudaMemcpy(g->d_kappa, kap.data(), sizeof(float) * kap.size(), cudaMemcpyHostToDevice));
    CU_TRY(cudaMalloc((void **)&g->d_invkappa, sizeof(float) * ik.size()));
    CU_TRY(cudaMemcpy(g->d_invkappa, ik.data(), sizeof(float) * ik.size(), cudaMemcpyHostToDevice));
    v.table = g->d_table;
    v.kappa = g->d_kappa;
    v.invkappa = g->d_invkappa;
  }
  cudaStream_t st = g->stream;
  v.cell_fmt = d->emis_mode == 0 ? kCellRho : (d->n_bands == 1 ? kCellLam : kCellXq);
  CU_TRY(cudaMalloc(&g->d_cells, (v.cell_fmt == kCellRho ? sizeof(float) : sizeof(uint2)) * n_cells));
  {
    const size_t es = d->field_dtype == AIR_F64 ? 8 : 4;
    void *raw_r = nullptr, *raw_t = nullptr;
    unsigned long long *d_bad = nullptr, h_bad = 0;
    // convert in slices so the staging buffer stays bounded
    const int64_t slice = (int64_t)1 << 26;
    const int64_t sl = std::min<int64_t>(slice, n_cells);
    cudaError_t e = cudaMalloc(&raw_r, es * sl);
    if (e == cudaSuccess && d->emis_mode == 1) e = cudaMalloc(&raw_t, es * sl);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_bad, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), st);
    for (int64_t off = 0; e == cudaSuccess && off < n_cells; off += sl) {
      const int64_t m = std::min<int64_t>(sl, n_cells - off);
      e = cudaMemcpyAsync(raw_r, (const char *)d->rho + es * off, es * m, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess && raw_t)
        e = cudaMemcpyAsync(raw_t, (const char *)d->temp + es * off, es * m, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) break;
      const unsigned blocks = (unsigned)((m + 255) / 256);
      const double dlogT = d->logT_hi - d->logT_lo;
      void *dst = v.cell_fmt == kCellRho ? (void *)((float *)g->d_cells + off)
                                         : (void *)((uint2 *)g->d_cells + off);
      if (d->field_dtype == AIR_F64)
        k_convert_fields<double><<<blocks, 256, 0, st>>>((const double *)raw_r, (const double *)raw_t, m,
                                                         v.cell_fmt, dst, d->logT_lo, dlogT, d->n_tbins,
                                                         g->d_table, d_bad);
      else
        k_convert_fields<float><<<blocks, 256, 0, st>>>((const float *)raw_r, (const float *)raw_t, m,
                                                        v.cell_fmt, dst, d->logT_lo, dlogT, d->n_tbins,
                                                        g->d_table, d_bad);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, d_bad, sizeof(h_bad), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(raw_r);
    if (raw_t) cudaFree(raw_t);
    if (d_bad) cudaFree(d_bad);
    if (e != cudaSuccess) return cuda_fail(e, "field upload");
    if (h_bad) return set_error(AIR_ERR_ARG, "%llu cells have rho < 0, T <= 0 or a non-finite value", h_bad);
  }
  v.cells = g->d_cells;
  if (d->kind == AIR_GRID_AMR) {
    CU_TRY(cudaMalloc((void **)&g->d_base, sizeof(int32_t) * ob.base.size()));
    CU_TRY(cudaMemcpy(g->d_base, ob.base.data(), sizeof(int32_t) * ob.base.size(), cudaMemcpyHostToDevice));
    if (!ob.oct.empty()) {
      CU_TRY(cudaMalloc((void **)&g->d_oct, sizeof(int32_t) * ob.oct.size()));
      CU_TRY(cudaMemcpy(g->d_oct, ob.oct.data(), sizeof(int32_t) * ob.oct.size(), cudaMemcpyHostToDevice));
    }
    const int64_t nb = (int64_t)v.nb0[0] * v.nb0[1] * v.nb0[2];
    int mapL = 0;
    while (mapL < v.Lm && (nb << (3 * (mapL + 1))) <= ((int64_t)1 << 24)) ++mapL;
    int64_t nm[3];
    for (int a = 0; a < 3; ++a) {
      nm[a] = (int64_t)v.nb0[a] << mapL;
      v.nm[a] = (int)nm[a];
    }
    std::vector<int32_t> map((size_t)(nm[0] * nm[1] * nm[2]));
    for (int64_t z = 0; z < v.nb0[2]; ++z)
      for (int64_t y = 0; y < v.nb0[1]; ++y)
        for (int64_t x = 0; x < v.nb0[0]; ++x)
          fill_map(ob, ob.base[(size_t)((z * v.nb0[1] + y) * v.nb0[0] + x)], 0, x, y, z, mapL, nm, map);
    CU_TRY(cudaMalloc((void **)&g->d_bmap, sizeof(int32_t) * map.size()));
    CU_TRY(cudaMemcpy(g->d_bmap, map.data(), sizeof(int32_t) * map.size(), cudaMemcpyHostToDevice));
    v.base = g->d_base;
    v.oct = g->d_oct;
    v.bmap = g->d_bmap;
    v.mapL = mapL;
  }
  return AIR_OK;
}

}  // namespace air
