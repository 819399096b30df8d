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
// by descending the brick octree from the level-0 brick; a brick is left
// through the face with the smallest exit parameter and the next brick is the
// one holding the finest cell across that face, so no cell is skipped or
// visited twice. Bricks at level >= fp64_level compute their entry point and
// exit parameter in FP64. Coarser bricks compute the entry point in
// double-float (pairs of FP32 with error-free sums and products), since FP64
// issues at a small fraction of the FP32 rate on this GPU. Either way the
// entry point is expressed relative to the entry cell, so FP32 rounding inside
// a brick scales with the distance marched in it.
//
// Accumulation in FP32: N, tau_b and I_b are Kahan-compensated sums;
// T = exp(-tau) is recomputed from the compensated tau at every cell (CUDA's
// __expf intrinsic: at most 2 + floor(1.17 |tau|) ulp, and no error carried
// from one cell to the next); the cell
// term is j ds T (1 - e^-dtau)/dtau from a Taylor polynomial for dtau < 1/4,
// and (j/alpha)(T_prev - T_next) above.
#pragma once
#include <cfloat>

#include "air_internal.cuh"

namespace air {

template <int NBT>
struct RTState {
  float N, cN;
  float tau[NBT], ctau[NBT], T[NBT], I[NBT], cI[NBT];
  uint32_t steps;
  int maxlev;  // deepest brick level crossed
};

struct BandCtx {
  const float *tab;  // shared: [NBT][tstride]
  int tstride, nbh;
  int fmt;           // cell format (kCellRho / kCellLam / kCellXq)
};

// Per-band constants held in registers for the whole ray.
template <int NBT>
struct BandRegs {
  float kap[NBT];  // kappa_b
  float ik[NBT];   // 1 / kappa_b (0 where kappa_b = 0)
};

template <int NBT>
__device__ __forceinline__ void rt_init(RTState<NBT> &r) {
  r.N = 0.f;
  r.cN = 0.f;
  r.steps = 0;
  r.maxlev = 0;
#pragma unroll
  for (int b = 0; b < NBT; ++b) {
    r.tau[b] = 0.f;
    r.ctau[b] = 0.f;
    r.T[b] = 1.f;
    r.I[b] = 0.f;
    r.cI[b] = 0.f;
  }
}

// One cell chord of length ds: density rho, and aux = Lambda (kCellLam, as
// float bits) or the table coordinate of T (kCellXq).
template <int NBT>
__device__ __forceinline__ void rt_cell(RTState<NBT> &r, float rho, uint32_t aux, float ds,
                                        const BandCtx &bc, const BandRegs<NBT> &br) {
  kahan_add(r.N, r.cN, rho * ds);
  r.steps += 1;
  int k = 0;
  float w = 0.f, lam1 = 1.f;
  if (bc.fmt == kCellXq) {
    k = (int)(aux >> kXqFracBits);
    w = (float)(aux & ((1u << kXqFracBits) - 1u)) * (1.0f / (float)(1u << kXqFracBits));
  } else if (bc.fmt == kCellLam) {
    lam1 = __uint_as_float(aux);
  }
  const float rho2ds = rho * rho * ds;
#pragma unroll
  for (int b = 0; b < NBT; ++b) {
    if (b < bc.nbh) {
      float lam = lam1;
      if (bc.fmt == kCellXq) {
        const float *t = bc.tab + b * bc.tstride + k;
        lam = fmaf(w, t[1] - t[0], t[0]);
      }
      const float alpha = br.kap[b] * rho;
      const float dtau = alpha * ds;
      float term;
      if (dtau > 0.f) {
        kahan_add(r.tau[b], r.ctau[b], dtau);
        const float Tn = __expf(-r.tau[b]);
        if (dtau < 0.25f)
          term = rho2ds * lam * r.T[b] * one_minus_exp_over_x(dtau);
        else
          term = rho * lam * br.ik[b] * (r.T[b] - Tn);
        r.T[b] = Tn;
      } else {
        term = rho2ds * lam * r.T[b];
      }
      kahan_add(r.I[b], r.cI[b], term);
    }
  }
}

// Fields of cell idx: rho and the auxiliary word of the format.
template <typename Idx>
__device__ __forceinline__ void load_cell(const void *__restrict__ cells, int fmt, Idx idx,
                                          float &rho, uint32_t &aux) {
  if (fmt == kCellRho) {
    rho = __ldg((const float *)cells + idx);
    aux = 0u;
  } else {
    const uint2 c = __ldg((const uint2 *)cells + idx);
    rho = __uint_as_float(c.x);
    aux = c.y;
  }
}

// DDA through a block of nx x ny x nz cells, entered in cell (lx, ly, lz).
// Q: entry point relative to the low corner of the entry cell (in cells),
// Dl: direction (cells per unit t), tend: block exit relative to the entry.
// cells points at the block's cell (0, 0, 0); cell (x, y, z) is record
// z*sz + y*sy + x. Boundary parameters are measured from the entry cell, so
// their FP32 rounding grows with the distance marched inside the block, not
// with the ray's distance from the origin. The fields of the next cell are
// fetched before the current cell's transfer step, so the load latency
// overlaps that arithmetic. Per-axis state is kept in scalars (registers).
template <int NBT, typename Idx>
__device__ __forceinline__ void march_block(RTState<NBT> &r, const float Q[3], const float Dl[3],
                                            float tend, int lx, int ly, int lz, int nx, int ny,
                                            int nz, Idx sy, Idx sz, const void *__restrict__ cells,
                                            const BandCtx &bc, const BandRegs<NBT> &br) {
  const float INF = FLT_MAX;
  const int s0 = Dl[0] > 0.f ? 1 : -1, s1 = Dl[1] > 0.f ? 1 : -1, s2 = Dl[2] > 0.f ? 1 : -1;
  const int p0 = Dl[0] > 0.f, p1 = Dl[1] > 0.f, p2 = Dl[2] > 0.f;
  const float i0 = Dl[0] != 0.f ? 1.0f / Dl[0] : 0.f;
  const float i1 = Dl[1] != 0.f ? 1.0f / Dl[1] : 0.f;
  const float i2 = Dl[2] != 0.f ? 1.0f / Dl[2] : 0.f;
  const Idx d0 = (Idx)s0, d1 = (Idx)s1 * sy, d2 = (Idx)s2 * sz;
  int r0 = 0, r1 = 0, r2 = 0;  // cells stepped from the entry cell
  float tm0 = Dl[0] != 0.f ? ((float)p0 - Q[0]) * i0 : INF;
  float tm1 = Dl[1] != 0.f ? ((float)p1 - Q[1]) * i1 : INF;
  float tm2 = Dl[2] != 0.f ? ((float)p2 - Q[2]) * i2 : INF;
  Idx idx = (Idx)lz * sz + (Idx)ly * sy + (Idx)lx;
  float rh;
  uint32_t xv;
  load_cell(cells, bc.fmt, idx, rh, xv);
  float tl = 0.f;
  for (;;) {
    const float tn = fminf(fminf(tm0, tm1), fminf(tm2, tend));
    const float ds = tn - tl;
    bool more = tn < tend;
    float rh_n = 0.f;
    uint32_t xv_n = 0u;
    if (more) {
      if (tm0 <= tm1 && tm0 <= tm2) {
        r0 += s0;
        more = (unsigned)(lx + r0) < (unsigned)nx;
        idx += d0;
        tm0 = ((float)(r0 + p0) - Q[0]) * i0;
      } else if (tm1 <= tm2) {
        r1 += s1;
        more = (unsigned)(ly + r1) < (unsigned)ny;
        idx += d1;
        tm1 = ((float)(r1 + p1) - Q[1]) * i1;
      } else {
        r2 += s2;
        more = (unsigned)(lz + r2) < (unsigned)nz;
        idx += d2;
        tm2 = ((float)(r2 + p2) - Q[2]) * i2;
      }
      if (more) load_cell(cells, bc.fmt, idx, rh_n, xv_n);
    }
    if (ds > 0.f) rt_cell<NBT>(r, rh, xv, ds, bc, br);
    if (!more) break;  // left the block (through its far face, or by rounding)
    rh = rh_n;
    xv = xv_n;
    tl = tn;
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
                                          int j, double O[3], double &t0) {
  const double pix = rg.pix0 * exp2_neg(L);
  const double uc = fma((double)i + 0.5, pix, -rg.H);
  const double vc = fma((double)j + 0.5, pix, -rg.H);
  t0 = -DBL_MAX;
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
      t0 = fmax(t0, ta);
      t1 = fmin(t1, tb);
    }
  }
  return hit && t0 < t1;
}

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

template <int NBT>
__device__ void march_uniform(RTState<NBT> &r, const GridView &g, const double O[3],
                              const double D[3], double t0, const BandCtx &bc,
                              const BandRegs<NBT> &br) {
  float Q[3], Dl[3];
  int lc[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double F = O[a] + t0 * D[a];
    lc[a] = clampi((int)floor(F), 0, g.nf[a] - 1);
    Q[a] = (float)(F - (double)lc[a]);
    Dl[a] = (float)D[a];
  }
  // the ray leaves through a face of the grid: no end parameter needed
  march_block<NBT, int64_t>(r, Q, Dl, FLT_MAX, lc[0], lc[1], lc[2], g.nf[0], g.nf[1], g.nf[2],
                            (int64_t)g.nf[0], (int64_t)g.nf[0] * g.nf[1], g.cells, bc, br);
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

// Per-launch constants (direction, its inverse and its double-float split)
// are read from the kernel-parameter bank, not held per thread.
template <int NBT>
__device__ void march_amr(RTState<NBT> &r, const GridView &g, const double O[3],
                          const RayGeom &rg, double t0, int fp64_level, const BandCtx &bc,
                          const BandRegs<NBT> &br) {
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
  const int s0 = lb + Lm;
  for (int it = 0; it < max_iter; ++it) {
    // leaf brick holding finest cell c
    int code = __ldg(g.base + ((int64_t)(c[2] >> s0) * g.nb0[1] + (c[1] >> s0)) * g.nb0[0] + (c[0] >> s0));
    int lev = 0;
    while (code < 0) {
      ++lev;
      const int sh = s0 - lev;
      const int oc = ((c[0] >> sh) & 1) | (((c[1] >> sh) & 1) << 1) | (((c[2] >> sh) & 1) << 2);
      code = __ldg(g.oct + (int64_t)(-code - 1) * 8 + oc);
    }
    const int4 bi = __ldg(g.binfo + code);
    r.maxlev = max(r.maxlev, bi.w);
    const int bo[3] = {bi.x, bi.y, bi.z};
    const int shift = Lm - bi.w;
    const int S = B << shift;
    const float scale = 1.0f / (float)(1 << shift);
    int lc[3], anchor[3];
    float Q[3], Dl[3], inv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lc[a] = (c[a] - bo[a]) >> shift;
      anchor[a] = bo[a] + (lc[a] << shift);
      Dl[a] = rg.Dhi[a] * scale;
      inv[a] = Dl[a] != 0.f ? 1.0f / Dl[a] : 0.f;
    }
    const bool deep = bi.w >= fp64_level;
    // entry point relative to the entry cell, and the exit face: smallest
    // parameter over the axes, measured from the entry
    float tend = FLT_MAX;
    int ax = -1;
    double te = 0.0;
    if (deep) {
      const double td = (double)t.hi + (double)t.lo;
      double tmin = DBL_MAX;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Q[a] = (float)(fma(td, D[a], O[a] - (double)anchor[a]) * (double)scale);
        if (D[a] != 0.0) {
          const double face = (double)(D[a] > 0.0 ? bo[a] + S : bo[a]);
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
    const int64_t boff = (int64_t)code << (3 * lb);
    const void *cb = g.cell_fmt == kCellRho ? (const void *)((const float *)g.cells + boff)
                                            : (const void *)((const uint2 *)g.cells + boff);
    march_block<NBT, int>(r, Q, Dl, tend, lc[0], lc[1], lc[2], B, B, B, B, B * B, cb, bc, br);
    if (ax < 0) break;
    // advance to the exit point
    if (deep) t = f2_from(te);
    else t = f2_add_f(t, tend);
    // finest cell just across the exit face; the other coordinates, from the
    // exit point in this brick's frame, stay in this brick's range
    bool out = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == ax) {
        c[a] = D[a] > 0.0 ? bo[a] + S : bo[a] - 1;
        out = c[a] < 0 || c[a] >= g.nf[a];
      } else {
        const float e = fmaf(tend, Dl[a], Q[a]);  // local cells from the entry cell
        const int f = anchor[a] + (int)floorf(e * (float)(1 << shift));
        c[a] = clampi(f, bo[a], bo[a] + S - 1);
      }
    }
    if (out) break;
  }
}

// One ray (pixel (L, i, j)) through the grid, bands [b0, b0 + NBT) of bc/br.
template <int NBT, bool AMR>
__device__ __forceinline__ void trace_ray(RTState<NBT> &st, const GridView &g, const RayGeom &rg,
                                          int L, int i, int j, int fp64_level, const BandCtx &bc,
                                          const BandRegs<NBT> &br) {
  rt_init<NBT>(st);
  double O[3], t0;
  if (ray_setup(g, rg, L, i, j, O, t0)) {
    if (AMR)
      march_amr<NBT>(st, g, O, rg, t0, fp64_level, bc, br);
    else
      march_uniform<NBT>(st, g, O, rg.D, t0, bc, br);
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
    rg.Dlo[a] = (float)(rg.D[a] - (double)rg.Dhi[a]);
  }
  rg.H = cam.H;
  rg.pix0 = (2.0 * cam.H) / (double)n0;
  return rg;
}

}  // namespace air
