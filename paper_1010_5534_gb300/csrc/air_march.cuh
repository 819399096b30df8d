// air_march.cuh -- per-ray march (Parkin 2010, Section 1 and Section 2 step ii):
// follow one ray per pixel through the grid and sum, per crossed cell, the
// column density N = sum rho ds and the emergent intensity of the absorbed
// emission, front to back, I_b = sum_k (j_k/alpha_k)(1 - e^-dtau_k) e^-tau_<k.
//
// One thread marches one ray (x a chunk of bands). Warps hold 32 neighbouring
// pixels, so their cell fetches fall in the same or adjacent cells.
//
// Traversal: the ray's position is kept as an integer finest-level cell
// coordinate plus a ray parameter t (world length). Inside a block of cells
// (the whole uniform grid, or one AMR brick) an Amanatides-Woo DDA in FP32
// local coordinates yields the exact chord of each cell. AMR bricks are found
// through a dense map over the finest cells (at the finest brick level that
// fits 2^24 entries, with an octree descent below it); a brick is left
// through the face with the smallest exit parameter and the next brick is the
// one holding the finest cell across that face, so no cell is skipped or
// visited twice. A ray along one grid axis crosses every brick whole, and its
// walk (march_amr_axis) carries no ray parameter. Bricks at level >= fp64_level compute their entry point and
// exit parameter in FP64. Coarser bricks compute the entry point in
// double-float (pairs of FP32 with error-free sums and products), since FP64
// issues at a small fraction of the FP32 rate on this GPU. Either way the
// entry point is expressed relative to the entry cell, so FP32 rounding inside
// a brick scales with the distance marched in it.
//
// Accumulation in FP32: N and I_b are Kahan-compensated sums. The absorption
// coefficient is alpha_b = kappa_b rho with kappa_b fixed per band, so the
// optical depth is tau_b = kappa_b N exactly, taken from the compensated N;
// T_b = e^-tau_b = 2^(-kappa_b log2(e) N) is recomputed at every cell with the
// hardware base-2 exponential (ex2.approx: relative error about 2^-22, plus
// the rounding of its argument, |tau| 2^-24 relative), so no error is carried
// from one cell to the next. The cell term is j ds T (1 - e^-dtau)/dtau from
// a Taylor polynomial for dtau < 1/4, and (j/alpha)(T_prev - T_next) above.
#pragma once
#include <cfloat>

#include "air_internal.cuh"

namespace air {

template <int NBT>
struct RTState {
  float N, cN;
  float T[NBT], I[NBT], cI[NBT];
  uint32_t steps;
  int maxlev;  // deepest brick level crossed
};

struct BandCtx {
  const float *tab;  // shared: [NBT][tstride] (kCellXq)
  int tstride, nbh;
};

// Per-band constants held in registers for the whole ray.
template <int NBT>
struct BandRegs {
  float kap[NBT];  // kappa_b
  float ik[NBT];   // 1 / kappa_b (0 where kappa_b = 0)
  float nk[NBT];   // -kappa_b log2(e): T_b = 2^(nk_b N)
  float kmax;      // largest kappa_b of the chunk
};

// Per-band registers of bands [b0, b0 + nbh) (zero beyond).
template <int NBT>
__device__ __forceinline__ void band_regs(BandRegs<NBT> &br, const float *kappa,
                                          const float *invkappa, int b0, int nbh) {
#pragma unroll
  for (int b = 0; b < NBT; ++b) {
    br.kap[b] = b < nbh ? __ldg(kappa + b0 + b) : 0.f;
    br.ik[b] = b < nbh ? __ldg(invkappa + b0 + b) : 0.f;
    br.nk[b] = (float)(-(double)br.kap[b] * 1.4426950408889634);
  }
  br.kmax = 0.f;
#pragma unroll
  for (int b = 0; b < NBT; ++b) br.kmax = fmaxf(br.kmax, br.kap[b]);
}

// 2^x by the hardware approximation (PTX ex2.approx.ftz.f32).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int NBT>
__device__ __forceinline__ void rt_init(RTState<NBT> &r) {
  r.N = 0.f;
  r.cN = 0.f;
  r.steps = 0;
  r.maxlev = 0;
#pragma unroll
  for (int b = 0; b < NBT; ++b) {
    r.T[b] = 1.f;
    r.I[b] = 0.f;
    r.cI[b] = 0.f;
  }
}

// Transfer step of one cell chord of length ds: density rho, and aux =
// rho Lambda (kCellLam, as float bits) or the table coordinate of T (kCellXq).
// With dtau = 0 (kappa_b = 0 or rho = 0) the series form gives the optically
// thin term j ds T exactly, so no separate case is needed.
// Both forms of the cell term are evaluated and the one for the cell's dtau
// is selected, which keeps the loop free of divergent branches.
//
// The products that feed the compensated sums (rho ds, and each form's final
// product) are rounded explicitly (__fmul_rn), so the compiler cannot fuse
// them into the sums' subtractions: every instantiation (band chunking, form)
// rounds alike and gives the same bits.
template <int NBT, int FMT>
__device__ __forceinline__ void rt_term(RTState<NBT> &r, float rho, uint32_t aux, float ds,
                                        const BandCtx &bc, const BandRegs<NBT> &br) {
  const float rds = __fmul_rn(rho, ds);
  kahan_add(r.N, r.cN, rds);
  int k = 0;
  float w = 0.f, lam1 = 1.f;
  if (FMT == kCellXq) {
    k = (int)(aux >> kXqFracBits);
    w = (float)(aux & ((1u << kXqFracBits) - 1u)) * (1.0f / (float)(1u << kXqFracBits));
  } else if (FMT == kCellLam) {
    lam1 = __uint_as_float(aux);
  }
#pragma unroll
  for (int b = 0; b < NBT; ++b) {
    if (NBT == 1 || b < bc.nbh) {
      float lam = lam1;
      if (FMT == kCellXq) {
        const float *t = bc.tab + b * bc.tstride + k;
        lam = fmaf(w, t[1] - t[0], t[0]);
      }
      const float dtau = br.kap[b] * rds;
      const float Tn = ex2_approx(br.nk[b] * r.N);
      const float rl = FMT == kCellLam ? lam1 : rho * lam;  // rho Lambda_b
      const float t_small = __fmul_rn(rl * rds, r.T[b] * one_minus_exp_over_x(dtau));
      const float t_large = __fmul_rn(rl * br.ik[b], r.T[b] - Tn);
      const float term = dtau < 0.25f ? t_small : t_large;
      r.T[b] = Tn;
      kahan_add(r.I[b], r.cI[b], term);
    }
  }
}

// One cell chord of length ds >= 0 on the DDA path. A zero-length chord (a
// ray grazing an edge or corner) adds nothing and is not counted as a step.
// Both transfer forms are evaluated and one selected per band: a per-cell
// branch to the series form alone (same bits when kmax (rho ds) < 1/4) was
// timed and made the batched 16-band renders 15% slower.
template <int NBT, int FMT>
__device__ __forceinline__ void rt_cell(RTState<NBT> &r, float rho, uint32_t aux, float ds,
                                        const BandCtx &bc, const BandRegs<NBT> &br) {
  r.steps += ds > 0.f ? 1u : 0u;
  rt_term<NBT, FMT>(r, rho, aux, ds, bc, br);
}

// Cells of a block requested ahead of the march along its dominant axis.
constexpr int kPrefetchAhead = 3;

// Fields of cell idx: rho and the auxiliary word of the format.
template <int FMT, typename Idx>
__device__ __forceinline__ void load_cell(const void *__restrict__ cells, Idx idx, float &rho,
                                          uint32_t &aux) {
  if (FMT == kCellRho) {
    rho = __ldg((const float *)cells + idx);
    aux = 0u;
  } else {
    const uint2 c = __ldg((const uint2 *)cells + idx);
    rho = __uint_as_float(c.x);
    aux = c.y;
  }
}

// Ask L1 for the record of cell idx (a hint: nothing is loaded into registers).
template <int FMT, typename Idx>
__device__ __forceinline__ void prefetch_cell(const void *__restrict__ cells, Idx idx) {
  const void *p = FMT == kCellRho ? (const void *)((const float *)cells + idx)
                                  : (const void *)((const uint2 *)cells + idx);
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// (1 - e^-x) / x for 0 <= x < 1/64 from its Taylor series truncated after
// x^3 (remainder < x^4 / 5! < 5e-10).
__device__ __forceinline__ float one_minus_exp_over_x_short(float x) {
  float g = -1.0f / 24.0f;
  g = fmaf(g, x, 1.0f / 6.0f);
  g = fmaf(g, x, -0.5f);
  g = fmaf(g, x, 1.0f);
  return g;
}

// The transfer steps of a group of U column cells, all with chord ds. Inside
// the group the column density and the band intensities are summed in plain
// FP32 (partial sums from zero, the cell terms added with one fused
// multiply-add each), and the group's partial sums are added to the running
// sums with Kahan compensation; the error of a plain sum of U = 16 positive
// terms is at most 15 u of the group's sum (u = 2^-24), so the column's sums
// stay within about 16 u of exact. T_b at each cell is 2^(nk_b N_k) with N_k
// the running column density plus the group's partial sum, its exponent
// formed as fma(nk_b, partial, nk_b N_start).
// FORM 3: every dtau of the group below 2^-12: (1 - e^-x) / x taken to first
// order, 1 - x / 2 (remainder < x^2 / 6 < 1e-8), as T + (-kappa_b / 2 T)(rho
// ds); used for one-band grids with per-cell Lambda, the format whose
// instantiations are few enough to afford another form;
// FORM 2: below 1/64 (the short series); FORM 1: below 1/4 (the full series);
// FORM 0: the form is selected per cell and band.
template <int NBT, int FMT, int FORM, int U>
__device__ __forceinline__ void column_group(RTState<NBT> &r, const float (&rh)[U],
                                             const uint32_t (&xv)[U], float ds, const BandCtx &bc,
                                             const BandRegs<NBT> &br) {
  float pN = 0.f, pI[NBT], nN0[NBT], hk[NBT];
  const float N0 = r.N;
#pragma unroll
  for (int b = 0; b < NBT; ++b) {
    pI[b] = 0.f;
    nN0[b] = __fmul_rn(br.nk[b], N0);  // log2 T_b at the group's start
    hk[b] = -0.5f * br.kap[b];         // exact: a power-of-two scaling
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const float rho = rh[u];
    const float rds = __fmul_rn(rho, ds);
    pN = __fadd_rn(pN, rds);
    int k = 0;
    float w = 0.f, lam1 = 1.f;
    if (FMT == kCellXq) {
      k = (int)(xv[u] >> kXqFracBits);
      w = (float)(xv[u] & ((1u << kXqFracBits) - 1u)) * (1.0f / (float)(1u << kXqFracBits));
    } else if (FMT == kCellLam) {
      lam1 = __uint_as_float(xv[u]);
    }
#pragma unroll
    for (int b = 0; b < NBT; ++b) {
      if (NBT == 1 || b < bc.nbh) {
        float lam = lam1;
        if (FMT == kCellXq) {
          const float *t = bc.tab + b * bc.tstride + k;
          lam = fmaf(w, t[1] - t[0], t[0]);
        }
        const float Tn = ex2_approx(fmaf(br.nk[b], pN, nN0[b]));
        const float rl = FMT == kCellLam ? lam1 : __fmul_rn(rho, lam);  // rho Lambda_b
        float P, Q;
        if (FORM == 3) {
          // T (1 - dtau / 2) with dtau = kappa_b (rho ds)
          P = __fmul_rn(rl, rds);
          Q = fmaf(__fmul_rn(hk[b], r.T[b]), rds, r.T[b]);
        } else if (FORM == 2) {
          const float dtau = __fmul_rn(br.kap[b], rds);
          P = __fmul_rn(rl, rds);
          Q = __fmul_rn(r.T[b], one_minus_exp_over_x_short(dtau));
        } else {
          const float dtau = __fmul_rn(br.kap[b], rds);
          const float Ps = __fmul_rn(rl, rds);
          const float Qs = __fmul_rn(r.T[b], one_minus_exp_over_x(dtau));
          if (FORM == 1) {
            P = Ps;
            Q = Qs;
          } else {
            const bool small = dtau < 0.25f;
            P = small ? Ps : __fmul_rn(rl, br.ik[b]);
            Q = small ? Qs : __fsub_rn(r.T[b], Tn);
          }
        }
        pI[b] = fmaf(P, Q, pI[b]);
        r.T[b] = Tn;
      }
    }
  }
  kahan_add(r.N, r.cN, pN);
#pragma unroll
  for (int b = 0; b < NBT; ++b)
    if (NBT == 1 || b < bc.nbh) kahan_add(r.I[b], r.cI[b], pI[b]);
}

// n cells of one column (cell idx, idx + d, ...), every one crossed whole
// with the same chord ds: the path of a ray parallel to a grid axis, which
// enters each block of cells through a face and leaves through the opposite
// one. No DDA is needed. Cells are fetched U at a time (U loads in flight per
// thread) and summed as a group (column_group); the transfer form is chosen
// per group from kmax (rho_max ds) for the group's largest rho, which bounds
// every cell's dtau = kappa_b (rho ds) (FP32 rounding is monotonic).
template <int NBT, int FMT, int U, typename Idx>
__device__ __forceinline__ void march_column(RTState<NBT> &r, const void *__restrict__ cells, Idx idx,
                                             Idx d, int n, float ds, const BandCtx &bc,
                                             const BandRegs<NBT> &br) {
  r.steps += (uint32_t)n;
  int k = 0;
  for (; k + U <= n; k += U) {
    float rh[U];
    uint32_t xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) load_cell<FMT>(cells, idx + (Idx)u * d, rh[u], xv[u]);
    idx += (Idx)U * d;
    float m = rh[0];
#pragma unroll
    for (int u = 1; u < U; ++u) m = fmaxf(m, rh[u]);
    const float dmax = br.kmax * __fmul_rn(m, ds);
    if (FMT == kCellLam && dmax < 0x1p-12f) column_group<NBT, FMT, 3, U>(r, rh, xv, ds, bc, br);
    else if (dmax < 0.015625f) column_group<NBT, FMT, 2, U>(r, rh, xv, ds, bc, br);
    else if (dmax < 0.25f) column_group<NBT, FMT, 1, U>(r, rh, xv, ds, bc, br);
    else column_group<NBT, FMT, 0, U>(r, rh, xv, ds, bc, br);
  }
  for (; k < n; ++k) {
    float rh;
    uint32_t xv;
    load_cell<FMT>(cells, idx, rh, xv);
    idx += d;
    rt_term<NBT, FMT>(r, rh, xv, ds, bc, br);
  }
}

// Cells fetched per group in the column march: 16 in the compiled one-axis
// form (8 blocks per SM), 8 where the column march runs inside a general
// kernel (oblique-capable single-view and batched kernels, more registers
// taken by the 3-axis DDA).
template <int DIR>
struct ColumnUnroll {
  static constexpr int value = 16;
};

// DDA through a block of nx x ny x nz cells, entered in cell (lx, ly, lz),
// for a ray that moves along two or three grid axes (a ray along one axis
// takes march_column). Q: entry point relative to the low corner of the
// entry cell (in cells), Dl: direction (cells per unit t), inv = 1 / Dl (0
// where Dl = 0), tend: block exit relative to the entry. cells points at the
// block's cell (0, 0, 0); cell (x, y, z) is record z*sz + y*sy + x.
//
// After k steps along axis a the next face of that axis is crossed at
// t = (k + [Dl > 0] - Q) / Dl = k |inv| + q, evaluated as one fused
// multiply-add from the exact float count k, so the rounding of a boundary
// parameter does not grow with the number of cells marched. Parameters are
// measured from the entry cell, so their FP32 rounding scales with the
// distance marched inside the block, not with the ray's distance from the
// origin. The fields of the next cell are fetched before the current cell's
// transfer step, so the load latency overlaps that arithmetic, and the cell
// kPrefetchAhead steps further along the axis the ray crosses fastest is
// requested from L1 at every step (clamped into the block), so most loads
// find their line already on the way. The loop body is straight-line code
// (the axis to step, the next index and the transfer form are selected, not
// branched on); its one branch is the exit from the block.
template <int NBT, int FMT, typename Idx>
__device__ __forceinline__ void march_block(RTState<NBT> &r, const float Q[3], const float Dl[3],
                                            const float inv[3], float tend, int lx, int ly, int lz,
                                            int nx, int ny, int nz, Idx sy, Idx sz,
                                            const void *__restrict__ cells, const BandCtx &bc,
                                            const BandRegs<NBT> &br) {
  {
  const float INF = FLT_MAX;
  const bool p0 = Dl[0] > 0.f, p1 = Dl[1] > 0.f, p2 = Dl[2] > 0.f;
  const float a0 = fabsf(inv[0]), a1 = fabsf(inv[1]), a2 = fabsf(inv[2]);
  const float q0 = Dl[0] != 0.f ? ((p0 ? 1.f : 0.f) - Q[0]) * inv[0] : INF;
  const float q1 = Dl[1] != 0.f ? ((p1 ? 1.f : 0.f) - Q[1]) * inv[1] : INF;
  const float q2 = Dl[2] != 0.f ? ((p2 ? 1.f : 0.f) - Q[2]) * inv[2] : INF;
  // last step count that stays inside the block, per axis
  const float km0 = (float)(p0 ? nx - 1 - lx : lx);
  const float km1 = (float)(p1 ? ny - 1 - ly : ly);
  const float km2 = (float)(p2 ? nz - 1 - lz : lz);
  const Idx d0 = p0 ? (Idx)1 : (Idx)-1, d1 = p1 ? sy : -sy, d2 = p2 ? sz : -sz;
  float k0 = 0.f, k1 = 0.f, k2 = 0.f;
  float tm0 = q0, tm1 = q1, tm2 = q2;
  Idx idx = (Idx)lz * sz + (Idx)ly * sy + (Idx)lx;
  const float e0 = fabsf(Dl[0]), e1 = fabsf(Dl[1]), e2 = fabsf(Dl[2]);
  const Idx pstep = (e0 >= e1 && e0 >= e2) ? d0 : (e1 >= e2 ? d1 : d2);
  const Idx plast = (Idx)nz * sz - 1;
  float rh;
  uint32_t xv;
  load_cell<FMT>(cells, idx, rh, xv);
#pragma unroll
  for (int n = 2; n <= kPrefetchAhead; ++n) {
    const Idx pi = idx + (Idx)n * pstep;
    prefetch_cell<FMT>(cells, pi < 0 ? (Idx)0 : (pi > plast ? plast : pi));
  }
  float tl = 0.f;
  for (;;) {
    const float tn = fminf(fminf(tm0, tm1), fminf(tm2, tend));
    const float ds = fmaxf(tn - tl, 0.f);
    tl = tn;
    // step the axis whose face comes first (selects, no branches); an axis
    // that is not stepped keeps its count and so its boundary parameter
    const bool x0 = tm0 <= tm1 && tm0 <= tm2;
    const bool x1 = !x0 && tm1 <= tm2;
    const bool x2 = !x0 && !x1;
    k0 += x0 ? 1.f : 0.f;
    k1 += x1 ? 1.f : 0.f;
    k2 += x2 ? 1.f : 0.f;
    tm0 = fmaf(k0, a0, q0);
    tm1 = fmaf(k1, a1, q1);
    tm2 = fmaf(k2, a2, q2);
    const bool more = tn < tend && k0 <= km0 && k1 <= km1 && k2 <= km2;
    const Idx nidx = idx + (x0 ? d0 : (x1 ? d1 : d2));
    idx = more ? nidx : idx;  // past the block: reload the current cell (no use)
    float rh_n;
    uint32_t xv_n;
    load_cell<FMT>(cells, idx, rh_n, xv_n);
    if (kPrefetchAhead > 1) {
      const Idx pi = idx + (Idx)kPrefetchAhead * pstep;
      prefetch_cell<FMT>(cells, pi < 0 ? (Idx)0 : (pi > plast ? plast : pi));
    }
    rt_cell<NBT, FMT>(r, rh, xv, ds, bc, br);
    if (!more) break;  // left the block (through its far face, or by rounding)
    rh = rh_n;
    xv = xv_n;
  }
  }
}

// Per-launch ray geometry, resolved on the host in FP64: the pixel centre
// (uc, vc) is the world point C + uc u + vc v (C = image centre - grid origin),
// its grid coordinate (finest-cell units) that point divided by the cell size
// h; rays travel along D = d / h (cells per unit t).
struct RayGeom {
  double C[3], U[3], V[3], h[3], invh[3], D[3], invD[3];
  double H, pix0;  // image half-extent, pixel size at level 0
  float Dhi[3], Dlo[3];  // D as a double-float pair
  float invDhi[3];       // 1 / Dhi, correctly rounded (0 where D = 0); for a
                         // brick at 2^s finest cells per cell, 1 / (Dhi 2^-s)
                         // is exactly invDhi 2^s
  // Axis views whose u and v are grid axes too: the cell of every pixel
  // column on each fixed axis, from axis_table_entry (exactly the set-up's
  // FP64 operations, once per column instead of once per ray), or NULL.
  // Fixed axis s = (A + 1 + s) % 3 (A the ray's axis): entries
  // tab[s * tab_slot + tab_n0 (2^L - 1) + p] for levels L = 0, 1, ..., with
  // p the pixel's j when bit s of tab_byj is set, else its i; -1 where the
  // column misses the grid.
  const int32_t *tab;
  int64_t tab_slot;
  int tab_n0, tab_byj;
};

// 2^-L exactly (0 <= L < 1023).
__device__ __forceinline__ double exp2_neg(int L) {
  return __longlong_as_double((long long)(1023 - L) << 52);
}

// Pixel centre -> ray in finest-cell units, clipped to the box: F(t) = O + t D,
// t >= t0. The pixel size at level L is pix0 2^-L (exact scaling), so a pixel
// of an adaptive image and the same pixel of a fixed image get the same ray.
// The grid coordinate x / h is the correctly rounded quotient (a product with
// 1/h and one residual correction), so a pixel centre that lies exactly on a
// cell face maps exactly onto it, and the half-open rule picks the higher cell.
__device__ __forceinline__ bool ray_setup(const GridView &g, const RayGeom &rg, int L, int i,
                                          int j, double O[3], double &t0, int &eax) {
  const double pix = rg.pix0 * exp2_neg(L);
  const double uc = fma((double)i + 0.5, pix, -rg.H);
  const double vc = fma((double)j + 0.5, pix, -rg.H);
  t0 = -DBL_MAX;
  eax = -1;
  double t1 = DBL_MAX;
  bool hit = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double x = fma(vc, rg.V[a], fma(uc, rg.U[a], rg.C[a]));
    const double q = x * rg.invh[a];
    O[a] = fma(fma(-q, rg.h[a], x), rg.invh[a], q);
    if (rg.D[a] == 0.0) {
      if (!(O[a] >= 0.0 && O[a] < (double)g.nf[a])) hit = false;
    } else {
      double ta = -O[a] * rg.invD[a], tb = ((double)g.nf[a] - O[a]) * rg.invD[a];
      if (ta > tb) {
        const double y = ta;
        ta = tb;
        tb = y;
      }
      if (ta > t0) {
        t0 = ta;
        eax = a;  // the box face the ray enters through
      }
      t1 = fmin(t1, tb);
    }
  }
  return hit && t0 < t1;
}

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

// ray_setup for a ray along grid axis A: only the two fixed coordinates are
// needed (the ray enters at the grid face and crosses every cell of its
// column), computed exactly as ray_setup computes them, so the cells are the
// same; c[A] is left for the caller. Half of ray_setup's FP64 work, which
// matters on a GPU whose FP64 rate is a small fraction of FP32's.
//
// With a column table (RayGeom::tab) the two cells are read from it: where u
// and v are grid axes, x_a depends on one pixel index only (the other term is
// an exact zero), and the table holds this function's result for every
// column (axis_table_entry), so the cells are the same bits.
template <int A>
__device__ __noinline__ unsigned long long axis_cells_fp64(const GridView &g, const RayGeom &rg,
                                                           int L, int i, int j);

template <int A>
__device__ __forceinline__ bool axis_ray_setup(const GridView &g, const RayGeom &rg, int L, int i,
                                               int j, int c[3]) {
  if (rg.tab) {
    const int o = rg.tab_n0 * ((1 << L) - 1);
    const int c1 = __ldg(rg.tab + o + ((rg.tab_byj & 1) ? j : i));
    const int c2 = __ldg(rg.tab + rg.tab_slot + o + ((rg.tab_byj & 2) ? j : i));
    c[(A + 1) % 3] = c1;
    c[(A + 2) % 3] = c2;
    return c1 >= 0 && c2 >= 0;
  }
  // a separate function, so that none of its FP64 work is executed ahead of
  // the branch on views that have a table
  const unsigned long long cc = axis_cells_fp64<A>(g, rg, L, i, j);
  const int c1 = (int)(uint32_t)cc, c2 = (int)(uint32_t)(cc >> 32);
  c[(A + 1) % 3] = c1;
  c[(A + 2) % 3] = c2;
  return c1 >= 0 && c2 >= 0;
}

// The two fixed cells of pixel (L, i, j)'s ray along axis A in FP64: cell on
// axis (A + 1) % 3 in the low word, on (A + 2) % 3 in the high word, -1 where
// the ray misses the grid on that axis.
template <int A>
__device__ __noinline__ unsigned long long axis_cells_fp64(const GridView &g, const RayGeom &rg,
                                                           int L, int i, int j) {
  const double pix = rg.pix0 * exp2_neg(L);
  const double uc = fma((double)i + 0.5, pix, -rg.H);
  const double vc = fma((double)j + 0.5, pix, -rg.H);
  int c[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int a = (A + 1 + s) % 3;
    const double x = fma(vc, rg.V[a], fma(uc, rg.U[a], rg.C[a]));
    const double q = __dmul_rn(x, rg.invh[a]);
    const double o = fma(fma(-q, rg.h[a], x), rg.invh[a], q);
    c[s] = (o >= 0.0 && o < (double)g.nf[a]) ? (int)o : -1;  // o >= 0: truncation is floor
  }
  return (unsigned long long)(uint32_t)c[0] | ((unsigned long long)(uint32_t)c[1] << 32);
}

// One column-table entry: the cell on grid axis a of level-L pixel column p
// (its i when by_j is false, else its j; the other index is 0, whose term is
// an exact zero), computed with axis_ray_setup's operations; -1 where the
// column misses the grid.
__device__ __forceinline__ int axis_table_entry(const GridView &g, const RayGeom &rg, int a, int L,
                                                int p, bool by_j) {
  const double pix = rg.pix0 * exp2_neg(L);
  const double uc = fma((double)(by_j ? 0 : p) + 0.5, pix, -rg.H);
  const double vc = fma((double)(by_j ? p : 0) + 0.5, pix, -rg.H);
  const double x = fma(vc, rg.V[a], fma(uc, rg.U[a], rg.C[a]));
  const double q = __dmul_rn(x, rg.invh[a]);
  const double o = fma(fma(-q, rg.h[a], x), rg.invh[a], q);
  return (o >= 0.0 && o < (double)g.nf[a]) ? (int)o : -1;
}

template <int NBT, int FMT>
__device__ void march_uniform(RTState<NBT> &r, const GridView &g, const double O[3],
                              const RayGeom &rg, double t0, const BandCtx &bc,
                              const BandRegs<NBT> &br) {
  float Q[3], Dl[3], inv[3];
  int lc[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double F = O[a] + t0 * rg.D[a];
    lc[a] = clampi((int)floor(F), 0, g.nf[a] - 1);
    Q[a] = (float)(F - (double)lc[a]);
    Dl[a] = rg.Dhi[a];
    inv[a] = rg.invDhi[a];
  }
  // the ray leaves through a face of the grid: no end parameter needed
  march_block<NBT, FMT, int64_t>(r, Q, Dl, inv, FLT_MAX, lc[0], lc[1], lc[2], g.nf[0], g.nf[1],
                                 g.nf[2], (int64_t)g.nf[0], (int64_t)g.nf[0] * g.nf[1], g.cells,
                                 bc, br);
}

// Double-float helpers (error-free transformations: Knuth's TwoSum and the
// fused-multiply-add form of Dekker's TwoProduct).
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 f2_from(double x) {
  F2 r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ F2 f2_add_f(F2 a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e += a.lo;
  F2 r;
  r.hi = s + e;
  r.lo = e - (r.hi - s);
  return r;
}
// (O + t D - anchor) in finest cells, accurate to FP32 rounding of the result:
// the products and sums that cancel are carried in double-float.
__device__ __forceinline__ float f2_offset(F2 O, F2 t, F2 D, float anchor) {
  const float p = t.hi * D.hi;
  float pe = fmaf(t.hi, D.hi, -p);            // exact error of t.hi * D.hi
  pe = fmaf(t.hi, D.lo, fmaf(t.lo, D.hi, pe));
  float s, se;
  two_sum(O.hi, p, s, se);
  const float a = s - anchor;                  // exact: s lies within a cell of anchor
  return a + ((se + O.lo) + pe);
}

// Dense brick-map entry of finest cell c (see GridView::bmap).
__device__ __forceinline__ int map_entry(const GridView &g, int c0, int c1, int c2) {
  const int sm = g.log2B + g.Lm - g.mapL;
  return __ldg(g.bmap + ((int64_t)(c2 >> sm) * g.nm[1] + (c1 >> sm)) * g.nm[0] + (c0 >> sm));
}

// Leaf brick holding finest cell c from its map entry: id, and its level in
// `lev`. Below the map level the brick octree is descended.
__device__ __forceinline__ int brick_of(const GridView &g, int e, const int c[3], int &lev) {
  if (e >= 0) {
    lev = e >> kMapLevelShift;
    return e & kMapIdMask;
  }
  const int s0 = g.log2B + g.Lm;
  lev = g.mapL;
  while (e < 0) {
    ++lev;
    const int sh = s0 - lev;
    const int oc = ((c[0] >> sh) & 1) | (((c[1] >> sh) & 1) << 1) | (((c[2] >> sh) & 1) << 2);
    e = __ldg(g.oct + (int64_t)(-e - 1) * 8 + oc);
  }
  return e;
}

// Brick by brick: find the leaf brick holding finest cell c, compute the
// entry point in it and the exit face (FP64 at levels >= fp64_level, else
// double-float), march its cells, step to the finest cell across the exit
// face. The map entry of the next brick is fetched before the current brick
// is marched, so its latency overlaps the march. Per-launch constants
// (direction, its inverse and its double-float split) are read from the
// kernel-parameter bank, not held per thread.
template <int NBT, int FMT>
__device__ void march_amr(RTState<NBT> &r, const GridView &g, const double O[3],
                          const RayGeom &rg, double t0, int eax, int fp64_level,
                          const BandCtx &bc, const BandRegs<NBT> &br) {
  const int B = g.B, lb = g.log2B, Lm = g.Lm;
  const double *D = rg.D, *invD = rg.invD;
  F2 Of[3];
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Of[a] = f2_from(O[a]);
    c[a] = clampi((int)floor(O[a] + t0 * D[a]), 0, g.nf[a] - 1);
  }
  F2 t = f2_from(t0);
  const int max_iter = 4 * (g.nf[0] + g.nf[1] + g.nf[2]);
  int e = map_entry(g, c[0], c[1], c[2]);
  for (int it = 0; it < max_iter; ++it) {
    int lev;
    const int code = brick_of(g, e, c, lev);
    r.maxlev = max(r.maxlev, lev);
    const int shift = Lm - lev;
    const int sb = lb + shift;
    const int S = B << shift;
    const float scale = __int_as_float((127 - shift) << 23);  // 2^-shift
    const float up = __int_as_float((127 + shift) << 23);     // 2^shift
    int lc[3], anchor[3], bo[3];
    float Q[3], Dl[3], inv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      bo[a] = (c[a] >> sb) << sb;
      lc[a] = (c[a] - bo[a]) >> shift;
      anchor[a] = bo[a] + (lc[a] << shift);
      Dl[a] = rg.Dhi[a] * scale;
      inv[a] = rg.invDhi[a] * up;
    }
    const bool deep = lev >= fp64_level;
    // entry point relative to the entry cell, and the exit face: smallest
    // parameter over the axes, measured from the entry
    float tend = FLT_MAX;
    int ax = -1;
    double te = 0.0;
    // On the axis the brick is entered through, the entry point is the face
    // itself, an integer finest coordinate: its offset is exact. On an axis
    // the ray does not move along, the offset O - anchor is constant and exact
    // in double-float. Only the other axes need the FP64 (or double-float)
    // position of the entry point.
    if (deep) {
      const double td = (double)t.hi + (double)t.lo;
      double tmin = DBL_MAX;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a == eax)
          Q[a] = (float)((Dl[a] > 0.f ? c[a] : c[a] + 1) - anchor[a]) * scale;
        else if (Dl[a] == 0.f)
          Q[a] = ((Of[a].hi - (float)anchor[a]) + Of[a].lo) * scale;
        else
          Q[a] = (float)fma(td, D[a], O[a] - (double)anchor[a]) * scale;
        if (Dl[a] != 0.f) {
          const double face = (double)(Dl[a] > 0.f ? bo[a] + S : bo[a]);
          const double ta = (face - O[a]) * invD[a];
          if (ta < tmin) {
            tmin = ta;
            ax = a;
          }
        }
      }
      te = tmin < td ? td : tmin;
      tend = (float)(te - td);
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        F2 Dv;
        Dv.hi = rg.Dhi[a];
        Dv.lo = rg.Dlo[a];
        if (a == eax)
          Q[a] = (float)((Dl[a] > 0.f ? c[a] : c[a] + 1) - anchor[a]) * scale;
        else if (Dl[a] == 0.f)
          Q[a] = ((Of[a].hi - (float)anchor[a]) + Of[a].lo) * scale;
        else
          Q[a] = f2_offset(Of[a], t, Dv, (float)anchor[a]) * scale;
        if (Dl[a] != 0.f) {
          const float face = Dl[a] > 0.f ? (float)(B - lc[a]) : (float)(-lc[a]);
          const float ta = (face - Q[a]) * inv[a];
          if (ta < tend) {
            tend = ta;
            ax = a;
          }
        }
      }
      if (tend < 0.f) tend = 0.f;
    }
    // finest cell just across the exit face; the other coordinates, from the
    // exit point in this brick's frame, stay in this brick's range
    bool out = ax < 0;
    int cn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == ax) {
        cn[a] = Dl[a] > 0.f ? bo[a] + S : bo[a] - 1;
        out = out || cn[a] < 0 || cn[a] >= g.nf[a];
      } else {
        const float x = fmaf(tend, Dl[a], Q[a]);  // local cells from the entry cell
        const int f = anchor[a] + (int)floorf(x * up);
        cn[a] = clampi(f, bo[a], bo[a] + S - 1);
      }
    }
    const int en = out ? 0 : map_entry(g, cn[0], cn[1], cn[2]);
    const int64_t boff = (int64_t)code << (3 * lb);
    const void *cb = FMT == kCellRho ? (const void *)((const float *)g.cells + boff)
                                     : (const void *)((const uint2 *)g.cells + boff);
    march_block<NBT, FMT, int>(r, Q, Dl, inv, tend, lc[0], lc[1], lc[2], B, B, B, B, B * B, cb,
                               bc, br);
    if (out) break;
    // advance to the exit point
    if (deep) t = f2_from(te);
    else t = f2_add_f(t, tend);
    c[0] = cn[0];
    c[1] = cn[1];
    c[2] = cn[2];
    e = en;
    eax = ax;
  }
}

// A ray parallel to grid axis A (every face-on view: the bench's +z view, the
// paper's ring view). Such a ray enters the grid, and every brick after,
// through an A face and crosses each brick whole, through a column of B cells
// of the brick's level, each with the same chord: the cell width over the
// direction, |1 / D_A| 2^(Lm - level) (an exact power-of-two scaling of the
// per-launch FP32 reciprocal). The other two finest coordinates never change
// and the next brick is the one holding the finest cell just past the far
// face, so the walk is integer-exact: no entry or exit parameter is computed,
// in FP32 or FP64, and no cell can be skipped or counted twice. Every kernel
// form (and the batched kernel) sends such a ray here, so all give the same
// bits for it. The map entry of the next brick is fetched before the current
// brick's column is marched, so its latency overlaps the march.
template <int NBT, int FMT, int A, int U>
__device__ __forceinline__ void march_amr_axis(RTState<NBT> &r, const GridView &g, int c[3], const RayGeom &rg,
                               const BandCtx &bc, const BandRegs<NBT> &br) {
  constexpr int A1 = (A + 1) % 3, A2 = (A + 2) % 3;
  const int B = g.B, lb = g.log2B, Lm = g.Lm;
  const bool pos = rg.Dhi[A] > 0.f;
  const float a1 = fabsf(rg.invDhi[A]);
  // cell strides inside a brick, x fastest
  const int sA = A == 0 ? 1 : (A == 1 ? B : B * B);
  const int sA1 = A1 == 0 ? 1 : (A1 == 1 ? B : B * B);
  const int sA2 = A2 == 0 ? 1 : (A2 == 1 ? B : B * B);
  const int d = pos ? sA : -sA;
  c[A] = pos ? 0 : g.nf[A] - 1;  // the ray enters through the grid face
  const int max_iter = 4 * g.nf[A];
  int e = map_entry(g, c[0], c[1], c[2]);
  for (int it = 0; it < max_iter; ++it) {
    int lev;
    const int code = brick_of(g, e, c, lev);
    r.maxlev = max(r.maxlev, lev);
    const int shift = Lm - lev;
    const int S = B << shift;
    const int cn = pos ? c[A] + S : c[A] - S;
    const bool out = cn < 0 || cn >= g.nf[A];
    int nc[3];
    nc[A] = cn;
    nc[A1] = c[A1];
    nc[A2] = c[A2];
    const int en = out ? 0 : map_entry(g, nc[0], nc[1], nc[2]);
    const int idx = (pos ? 0 : (B - 1) * sA) + ((c[A1] >> shift) & (B - 1)) * sA1 +
                    ((c[A2] >> shift) & (B - 1)) * sA2;
    const float ds = a1 * __int_as_float((127 + shift) << 23);  // a1 2^shift
    const int64_t boff = (int64_t)code << (3 * lb);
    const void *cb = FMT == kCellRho ? (const void *)((const float *)g.cells + boff)
                                     : (const void *)((const uint2 *)g.cells + boff);
    march_column<NBT, FMT, U, int>(r, cb, idx, d, B, ds, bc, br);
    if (out) break;
    c[A] = cn;
    e = en;
  }
}

// The uniform grid's version: the whole column of nf[A] cells.
template <int NBT, int FMT, int A, int U>
__device__ __forceinline__ void march_uniform_axis(RTState<NBT> &r, const GridView &g, const int c[3],
                                   const RayGeom &rg, const BandCtx &bc, const BandRegs<NBT> &br) {
  constexpr int A1 = (A + 1) % 3, A2 = (A + 2) % 3;
  const bool pos = rg.Dhi[A] > 0.f;
  const int64_t st[3] = {1, (int64_t)g.nf[0], (int64_t)g.nf[0] * g.nf[1]};
  const int64_t idx = (pos ? 0 : (int64_t)(g.nf[A] - 1) * st[A]) + (int64_t)c[A1] * st[A1] +
                      (int64_t)c[A2] * st[A2];
  march_column<NBT, FMT, U, int64_t>(r, g.cells, idx, pos ? st[A] : -st[A], g.nf[A],
                                     fabsf(rg.invDhi[A]), bc, br);
}

// Pixel (L, i, j)'s ray along grid axis A through either kind of grid.
template <int NBT, bool AMR, int FMT, int A, int U>
__device__ __forceinline__ void march_axis(RTState<NBT> &st, const GridView &g, const RayGeom &rg,
                                           int L, int i, int j, const BandCtx &bc,
                                           const BandRegs<NBT> &br) {
  int c[3];
  if (!axis_ray_setup<A>(g, rg, L, i, j, c)) return;
  if (AMR) march_amr_axis<NBT, FMT, A, U>(st, g, c, rg, bc, br);
  else march_uniform_axis<NBT, FMT, A, U>(st, g, c, rg, bc, br);
}

// One ray (pixel (L, i, j)) through the grid, bands [b0, b0 + NBT) of bc/br.
// DIR = 1 + A: every ray of the launch is parallel to grid axis A.
template <int NBT, bool AMR, int FMT, int DIR = 0>
__device__ __forceinline__ void trace_ray(RTState<NBT> &st, const GridView &g, const RayGeom &rg,
                                          int L, int i, int j, int fp64_level, const BandCtx &bc,
                                          const BandRegs<NBT> &br) {
  rt_init<NBT>(st);
  constexpr int U = ColumnUnroll<DIR>::value;
  if constexpr (DIR >= 1) {
    march_axis<NBT, AMR, FMT, (DIR - 1) % 3, U>(st, g, rg, L, i, j, bc, br);
  } else {
    const bool m0 = rg.Dhi[0] != 0.f, m1 = rg.Dhi[1] != 0.f, m2 = rg.Dhi[2] != 0.f;
    if (m0 + m1 + m2 == 1) {
      if (m0) march_axis<NBT, AMR, FMT, 0, U>(st, g, rg, L, i, j, bc, br);
      else if (m1) march_axis<NBT, AMR, FMT, 1, U>(st, g, rg, L, i, j, bc, br);
      else march_axis<NBT, AMR, FMT, 2, U>(st, g, rg, L, i, j, bc, br);
      return;
    }
    double O[3], t0;
    int eax;
    if (!ray_setup(g, rg, L, i, j, O, t0, eax)) return;
    if (AMR) march_amr<NBT, FMT>(st, g, O, rg, t0, eax, fp64_level, bc, br);
    else march_uniform<NBT, FMT>(st, g, O, rg, t0, bc, br);
  }
}

// World camera -> per-launch ray geometry (FP64, host).
static inline RayGeom make_geom(const GridView &g, const Camera &cam, int n0) {
  RayGeom rg;
  for (int a = 0; a < 3; ++a) {
    rg.C[a] = cam.c[a] - g.lo[a];
    rg.U[a] = cam.u[a];
    rg.V[a] = cam.v[a];
    rg.h[a] = g.h[a];
    rg.invh[a] = 1.0 / g.h[a];
    rg.D[a] = cam.d[a] / g.h[a];
    rg.invD[a] = cam.d[a] != 0.0 ? 1.0 / rg.D[a] : 0.0;
    rg.Dhi[a] = (float)rg.D[a];
    // a direction component too small for FP32 (the ray moves less than
    // 1e-30 cells per unit length along that axis) is taken as zero
    if (!(fabsf(rg.Dhi[a]) >= 1e-30f)) {
      rg.D[a] = 0.0;
      rg.invD[a] = 0.0;
      rg.Dhi[a] = 0.f;
    }
    rg.Dlo[a] = (float)(rg.D[a] - (double)rg.Dhi[a]);
    rg.invDhi[a] = rg.Dhi[a] != 0.f ? 1.0f / rg.Dhi[a] : 0.f;
  }
  rg.H = cam.H;
  rg.pix0 = (2.0 * cam.H) / (double)n0;
  rg.tab = nullptr;
  rg.tab_slot = 0;
  rg.tab_n0 = n0;
  rg.tab_byj = 0;
  return rg;
}

// Whether the view's rays run along one grid axis A with u and v along the
// other two (each with one nonzero component); then *byj gets bit s set when
// fixed axis (A + 1 + s) % 3 follows v (the pixel's j).
static inline bool axis_table_view(const RayGeom &rg, int *A, int *byj) {
  const int moving = (rg.Dhi[0] != 0.f) + (rg.Dhi[1] != 0.f) + (rg.Dhi[2] != 0.f);
  if (moving != 1) return false;
  *A = rg.Dhi[0] != 0.f ? 0 : (rg.Dhi[1] != 0.f ? 1 : 2);
  *byj = 0;
  for (int s = 0; s < 2; ++s) {
    const int a = (*A + 1 + s) % 3;
    const bool u = rg.U[a] != 0.0, v = rg.V[a] != 0.0;
    if (u == v) return false;
    if (v) *byj |= 1 << s;
  }
  return true;
}


}  // namespace air
