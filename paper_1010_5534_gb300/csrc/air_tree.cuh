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

// Step iii for node k: 1 if it is a leaf below max_level with xi >= xi_crit.
__device__ __forceinline__ uint32_t xi_flag(const TreeView &t, int base0, int64_t k,
                                            double xi_crit, int xi_norm, int refine_on) {
  const int L = t.lvl[k];
  if (t.child[k] >= 0 || L >= t.Lm) return 0u;
  const int i = t.pi[k], j = t.pj[k];
  const int nl = t.n0 << L;
  int q[9];
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const int ii = min(max(i + di, 0), nl - 1), jj = min(max(j + dj, 0), nl - 1);
      q[3 * (dj + 1) + (di + 1)] = (di == 0 && dj == 0) ? (int)k : descend(t, base0, L, ii, jj);
    }
  uint32_t f = 0;
  double s[9];
  if (refine_on == 0 || refine_on == 2) {
#pragma unroll
    for (int m = 0; m < 9; ++m) s[m] = (double)t.p[q[m]];
    f |= xi_at_least(s, xi_norm, xi_crit);
  }
  if (refine_on == 1 || refine_on == 2) {
#pragma unroll
    for (int m = 0; m < 9; ++m) s[m] = (double)t.N[q[m]];
    f |= xi_at_least(s, xi_norm, xi_crit);
  }
  return f;
}

// Step iii, balance: a flagged leaf at level L forces every leaf at a level
// < L that covers one of its 8 same-level neighbours, and so on down the
// levels. Each newly set flag is expanded by the thread that set it.
__device__ __forceinline__ void balance_from(const TreeView &t, int base0, int k0,
                                             uint32_t *__restrict__ flag,
                                             uint32_t *__restrict__ err) {
  int stack[kBalanceStack];
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
        const int m = descend(t, base0, L, ii, jj);
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
