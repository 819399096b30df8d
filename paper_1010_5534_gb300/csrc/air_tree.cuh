// air_tree.cuh -- image-quadtree device functions shared by the single-view
// and the batched refinement (Parkin 2010, Section 2 steps iii-iv; Eq. 2).
#pragma once
#include "air_refine.cuh"

namespace air {

// Node holding level-L pixel (i, j): descend from the base pixel through the
// child links; stops at the deepest existing node (level <= L). base0 is the
// index of the view's base pixel (0, 0).
__device__ __forceinline__ int descend(const TreeView &t, int base0, int L, int i, int j) {
  int k = base0 + (j >> L) * t.n0 + (i >> L);
  for (int l = 1; l <= L; ++l) {
    const int c = t.child[k];
    if (c < 0) break;
    const int s = L - l;
    k = c + ((((j >> s) & 1) << 1) | ((i >> s) & 1));
  }
  return k;
}

// Level maps of a single-view tree: for every level 1 <= l < Lm a dense
// (n0 2^l)^2 array of node indices (-1 where no node exists), written when
// the node is created; level 0 is implicit (node j n0 + i). The deepest node
// at a level <= L covering level-L pixel (i, j) is then found by at most L
// independent loads (one, or two next to a coarser neighbour, in a balanced
// tree) instead of a chain of L dependent child-link hops.
__device__ __forceinline__ int map_deepest(const TreeView &t, const int32_t *__restrict__ lmap, int L,
                                           int i, int j) {
  for (int l = L; l >= 1; --l) {
    const int s = L - l;
    const int64_t nl = (int64_t)t.n0 << l;
    const int q = __ldg(lmap + level_map_offset(t.n0, l) + (int64_t)(j >> s) * nl + (i >> s));
    if (q >= 0) return q;
  }
  return (j >> L) * t.n0 + (i >> L);
}

// The deepest node at a level <= L covering level-L pixel (i, j): through the
// level maps when the tree has them, else by descent from the base pixel.
struct NodeLookup {
  int base0;              // index of the view's base pixel (0, 0)
  const int32_t *lmap;   // level maps (single view, base0 = 0), or NULL
  __device__ __forceinline__ int operator()(const TreeView &t, int L, int i, int j) const {
    return lmap ? map_deepest(t, lmap, L, i, j) : descend(t, base0, L, i, j);
  }
};

// Numerator and denominator of Eq. 2 (squared) on the 3x3 stencil
// s[3*(dj+1) + (di+1)], FP64 with every operation rounded separately (no
// fused multiply-add), in a fixed order.
__device__ __forceinline__ void xi_terms(const double s[9], int xi_norm, double &num, double &den) {
  const double c = s[4], xm = s[3], xp = s[5], ym = s[1], yp = s[7];
  const double mm = s[0], pm = s[2], mp = s[6], pp = s[8];
  const double c2 = __dmul_rn(2.0, c);
  const double d2u = __dadd_rn(__dsub_rn(xp, c2), xm);
  const double d2v = __dadd_rn(__dsub_rn(yp, c2), ym);
  const double duv = __dmul_rn(__dadd_rn(__dsub_rn(__dsub_rn(pp, pm), mp), mm), 0.25);
  num = __dadd_rn(__dadd_rn(__dmul_rn(d2u, d2u), __dmul_rn(d2v, d2v)),
                  __dmul_rn(2.0, __dmul_rn(duv, duv)));
  const double au = __dadd_rn(fabs(__dsub_rn(xp, c)), fabs(__dsub_rn(c, xm)));
  const double av = __dadd_rn(fabs(__dsub_rn(yp, c)), fabs(__dsub_rn(c, ym)));
  den = __dadd_rn(__dmul_rn(au, au), __dmul_rn(av, av));
  if (xi_norm == 1) den = __dmul_rn(2.0, den);
}

// xi of Eq. 2: 0 where the numerator vanishes, 1 where only the denominator
// does, sqrt(num / den) (correctly rounded quotient and root) clamped to 1.
__device__ __forceinline__ double xi_eq2(const double s[9], int xi_norm) {
  double num, den;
  xi_terms(s, xi_norm, num, den);
  if (num == 0.0) return 0.0;
  if (den == 0.0) return 1.0;
  const double x = __dsqrt_rn(__ddiv_rn(num, den));
  return x > 1.0 ? 1.0 : x;
}

// xi_eq2(s) >= xi_crit, decided without the quotient and root where num is
// clearly above or below den xi_crit^2: the margin 2^-40 exceeds the rounding
// of the products and of the quotient and root by a factor of about 2^12,
// so every decision equals the comparison of the rounded xi. Inside the
// margin the rounded xi is computed and compared.
__device__ __forceinline__ bool xi_at_least(const double s[9], int xi_norm, double xi_crit) {
  if (!(xi_crit > 0.0)) return true;
  if (xi_crit > 1.0) return false;
  double num, den;
  xi_terms(s, xi_norm, num, den);
  if (num == 0.0) return false;
  if (den == 0.0) return true;
  const double c2 = __dmul_rn(xi_crit, xi_crit);
  const double m = 9.094947017729282e-13;  // 2^-40
  if (num >= __dmul_rn(den, __dmul_rn(c2, 1.0 + m))) return true;
  if (num <= __dmul_rn(den, __dmul_rn(c2, 1.0 - m))) return false;
  const double x = __dsqrt_rn(__ddiv_rn(num, den));
  return (x > 1.0 ? 1.0 : x) >= xi_crit;
}

// xi_at_least decided in FP32 where the answer is clear: 1 (xi >= xi_crit),
// 0 (xi < xi_crit) or -1 (too close to call: take the FP64 path). FP64 runs
// at a small fraction of the FP32 rate on this GPU, and most stencils are far
// from the threshold.
//
// With A = max |f_m| and u = 2^-24, each FP32 operation of the numerator and
// denominator below rounds with relative error <= u, and a first-order count
// over the operations (second differences <= 4A, first differences <= 2A,
// squares <= 16A^2, sums <= 34A^2) bounds |num32 - num| <= 221 u A^2 and
// |den32 - den| <= 192 u A^2 (twice that with xi_norm = 1); E = 512 u A^2 is
// used for both. The answer is 1 when num32 - E > (den32 + E) xi_crit^2
// (1 + 2^-9) and 0 when num32 + E < (den32 - E) xi_crit^2 (1 - 2^-9): then the
// exact num and den satisfy the strict inequality with margin 2^-11, which
// exceeds the FP64 path's rounding (about 2^-44 A^2 absolute, against num or
// den of at least E xi_crit^2 >= 2^-23 A^2 when xi_crit >= 1/16) by orders of
// magnitude, so the FP64 path returns the same. Outside 1/16 <= xi_crit <= 1
// the answer is -1 (the FP64 path's own rules for xi_crit <= 0 and > 1 then
// apply); A = 0 (all nine values zero) is 0, as the FP64 path's num == 0 rule
// gives; with A outside [2^-50, 2^60] (squares and bounds must stay normal
// FP32 numbers) the answer is -1.
__device__ __forceinline__ int xi_at_least_f32(const float f[9], int xi_norm, double xi_crit) {
  if (!(xi_crit >= 0.0625 && xi_crit <= 1.0)) return -1;
  float A = 0.f;
#pragma unroll
  for (int m = 0; m < 9; ++m) A = fmaxf(A, fabsf(f[m]));
  if (A == 0.f) return 0;
  if (!(A >= 0x1p-50f && A <= 0x1p60f)) return -1;
  const float c = f[4], xm = f[3], xp = f[5], ym = f[1], yp = f[7];
  const float mm = f[0], pm = f[2], mp = f[6], pp = f[8];
  const float c2 = 2.f * c;
  const float d2u = __fadd_rn(__fsub_rn(xp, c2), xm);
  const float d2v = __fadd_rn(__fsub_rn(yp, c2), ym);
  const float duv = __fmul_rn(__fadd_rn(__fsub_rn(__fsub_rn(pp, pm), mp), mm), 0.25f);
  const float num = __fadd_rn(__fadd_rn(__fmul_rn(d2u, d2u), __fmul_rn(d2v, d2v)),
                              __fmul_rn(2.f, __fmul_rn(duv, duv)));
  const float au = __fadd_rn(fabsf(__fsub_rn(xp, c)), fabsf(__fsub_rn(c, xm)));
  const float av = __fadd_rn(fabsf(__fsub_rn(yp, c)), fabsf(__fsub_rn(c, ym)));
  float den = __fadd_rn(__fmul_rn(au, au), __fmul_rn(av, av));
  float E = __fmul_rn(0x1p-15f, __fmul_rn(A, A));  // 512 u A^2
  if (xi_norm == 1) {
    den = 2.f * den;
  }
  const float Ed = xi_norm == 1 ? 2.f * E : E;
  const float x2 = (float)(xi_crit * xi_crit);
  const float c_hi = x2 * (1.f + 0x1p-9f), c_lo = x2 * (1.f - 0x1p-9f);
  if (__fsub_rn(num, E) > __fmul_rn(__fadd_rn(den, Ed), c_hi)) return 1;
  if (__fadd_rn(num, E) < __fmul_rn(__fsub_rn(den, Ed), c_lo)) return 0;
  return -1;
}

// Step iii for node k: 1 if it is a leaf below max_level with xi >= xi_crit.
__device__ __forceinline__ uint32_t xi_flag(const TreeView &t, NodeLookup look, int64_t k,
                                            double xi_crit, int xi_norm, int refine_on) {
  const int L = t.lvl[k];
  if (t.child[k] >= 0 || L >= t.Lm) return 0u;
  const int i = t.pi[k], j = t.pj[k];
  const int nl = t.n0 << L;
  int q[9];
  if (look.lmap && L >= 1) {
    // level maps: the eight level-L entries are independent loads, issued
    // together; a neighbour missing at level L (a coarser leaf covers it, at
    // most one level up in a balanced tree) is looked up level by level
    const int32_t *mL = look.lmap + level_map_offset(t.n0, L);
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const int ii = min(max(i + di, 0), nl - 1), jj = min(max(j + dj, 0), nl - 1);
        q[3 * (dj + 1) + (di + 1)] = (di == 0 && dj == 0) ? (int)k : __ldg(mL + (int64_t)jj * nl + ii);
      }
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const int m = 3 * (dj + 1) + (di + 1);
        if (q[m] < 0) {
          const int ii = min(max(i + di, 0), nl - 1), jj = min(max(j + dj, 0), nl - 1);
          q[m] = map_deepest(t, look.lmap, L - 1, ii >> 1, jj >> 1);
        }
      }
  } else {
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const int ii = min(max(i + di, 0), nl - 1), jj = min(max(j + dj, 0), nl - 1);
        q[3 * (dj + 1) + (di + 1)] = (di == 0 && dj == 0) ? (int)k : look(t, L, ii, jj);
      }
  }
  uint32_t f = 0;
  float v[9];
  double s[9];
  if (refine_on == 0 || refine_on == 2) {
#pragma unroll
    for (int m = 0; m < 9; ++m) v[m] = t.p[q[m]];
    int d = xi_at_least_f32(v, xi_norm, xi_crit);
    if (d < 0) {
#pragma unroll
      for (int m = 0; m < 9; ++m) s[m] = (double)v[m];
      d = xi_at_least(s, xi_norm, xi_crit);
    }
    f |= (uint32_t)d;
  }
  if (f == 0 && (refine_on == 1 || refine_on == 2)) {
#pragma unroll
    for (int m = 0; m < 9; ++m) v[m] = t.N[q[m]];
    int d = xi_at_least_f32(v, xi_norm, xi_crit);
    if (d < 0) {
#pragma unroll
      for (int m = 0; m < 9; ++m) s[m] = (double)v[m];
      d = xi_at_least(s, xi_norm, xi_crit);
    }
    f |= (uint32_t)d;
  }
  return f;
}

// Step iii, balance: a flagged leaf at level L forces every leaf at a level
// < L that covers one of its 8 same-level neighbours, and so on down the
// levels. Each newly set flag is expanded by the thread that set it.
//
// With level maps (single-view trees) a neighbour needs one load: the maps
// of levels below the top level are complete, so a level-L entry that exists
// is a level-L node (nothing to force) and an entry of -1 means no level-L
// node covers that pixel, so the deepest node covering it is a leaf at a
// level below L: it is forced without reading it. The eight entries are
// loaded together; only the missing ones are looked up one level up.
__device__ __forceinline__ void balance_from_maps(const TreeView &t, const int32_t *__restrict__ lmap,
                                                  int k0, uint32_t *__restrict__ flag,
                                                  uint32_t *__restrict__ err,
                                                  int (&stack)[kBalanceStack]) {
  int sp = 0;
  int q = k0;
  for (;;) {
    const int L = t.lvl[q], i = t.pi[q], j = t.pj[q];
    if (L >= 1) {  // level-0 neighbours always exist
      const int nl = t.n0 << L;
      const int32_t *mL = lmap + level_map_offset(t.n0, L);
      int e[8];
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        const int dd = d < 4 ? d : d + 1;  // skip the centre of the 3x3 stencil
        const int ii = i + dd % 3 - 1, jj = j + dd / 3 - 1;
        const bool in = ii >= 0 && jj >= 0 && ii < nl && jj < nl;
        e[d] = in ? __ldg(mL + (int64_t)jj * nl + ii) : 0;
      }
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        if (e[d] >= 0) continue;
        const int dd = d < 4 ? d : d + 1;
        const int ii = i + dd % 3 - 1, jj = j + dd / 3 - 1;
        const int m = map_deepest(t, lmap, L - 1, ii >> 1, jj >> 1);
        if (atomicExch(flag + m, 1u) == 0u) {
          if (sp < kBalanceStack) stack[sp++] = m;
          else atomicOr(err, 1u);
        }
      }
    }
    if (sp == 0) break;
    q = stack[--sp];
  }
}

__device__ __forceinline__ void balance_from(const TreeView &t, NodeLookup look, int k0,
                                             uint32_t *__restrict__ flag,
                                             uint32_t *__restrict__ err) {
  int stack[kBalanceStack];
  if (look.lmap) {
    balance_from_maps(t, look.lmap, k0, flag, err, stack);
    return;
  }
  int sp = 0;
  stack[sp++] = k0;
  while (sp > 0) {
    const int q = stack[--sp];
    const int L = t.lvl[q], i = t.pi[q], j = t.pj[q];
    const int nl = t.n0 << L;
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        if (!di && !dj) continue;
        const int ii = i + di, jj = j + dj;
        if (ii < 0 || jj < 0 || ii >= nl || jj >= nl) continue;
        const int m = look(t, L, ii, jj);
        if (t.child[m] < 0 && t.lvl[m] < L) {
          if (atomicExch(flag + m, 1u) == 0u) {
            if (sp < kBalanceStack) stack[sp++] = m;
            else atomicOr(err, 1u);
          }
        }
      }
  }
}

}  // namespace air
