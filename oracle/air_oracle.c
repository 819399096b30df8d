/* air_oracle.c -- plain FP64 CPU oracle for adaptive image ray-tracing (AIR).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's
 * CPU-baseline leg to check the CUDA library. The library never links it and
 * the two share no code.
 *
 * What it computes (E. R. Parkin 2010, "Adaptive image ray-tracing for
 * astrophysical simulations"):
 *   - Section 1 and Section 2 step (ii): one ray per pixel through the
 *     simulation grid, summing the column density and solving the equation of
 *     radiative transfer for the emergent intensity. Fields are piecewise
 *     constant per cell, so the exact solution is a sum over the cells the ray
 *     crosses: N = sum rho_k ds_k and, front to back,
 *     I_b = sum_k (j_k/alpha_k)(1 - exp(-dtau_k)) exp(-tau_<k)  (alpha = 0: j_k ds_k).
 *     The ray is split at EVERY plane of the finest grid level (a superset of
 *     all cell faces); each piece is assigned to the cell containing its
 *     midpoint; consecutive pieces in one cell are merged into that cell's chord.
 *   - Section 2 steps (iii)-(v): truncation-error scan (Eq. 2, with Eq. 1 as
 *     its 1-D case), 2:1 level balance between adjacent pixels, quadtree
 *     refinement of flagged pixels, repeated until nothing is flagged.
 *   - Section 2 step (vi): the final image is the list of leaf pixels.
 *
 * Readings where the paper is silent (all of them also hold for the CUDA path):
 *   cells are half-open [x_k, x_k+1): a ray lying on a face samples the higher
 *   cell; Eq. 2's denominator sums over the axis u only (xi_norm 0), or over
 *   u and v literally (xi_norm 1); xi = 0 when the numerator is 0, xi = 1 when
 *   only the denominator is 0, xi clamped to <= 1; flag when xi >= xi_crit;
 *   stencil neighbours outside the image are clamped to the edge; a missing
 *   neighbour at level L takes the value of the deepest existing node at a
 *   level <= L covering it; balance is over the 8 neighbours; every leaf below
 *   the maximum level is rescanned in every sweep.
 *
 * Parity pins: the closed-form, brute-force and invariant tests under tests/.
 */
#include "air_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_ctx {
  orc_scene s;
  int64_t nf[3];   /* finest-level cells per axis */
  double hf[3];    /* finest-level cell size per axis */
  int64_t md[ORC_MAX_LEVELS][3];
  int32_t *map[ORC_MAX_LEVELS]; /* AMR: leaf brick id at (level, brick coords), -1 if none */
};

/* ------------------------------------------------------------------ setup */

void orc_release(orc_ctx *c) {
  if (!c) return;
  for (int l = 0; l < ORC_MAX_LEVELS; ++l) free(c->map[l]);
  free(c);
}

/* Cell value id of a field stored as double or float (a float widens exactly). */
static double field_at(const orc_scene *s, const void *f, int64_t id) {
  return s->field_f32 ? (double)((const float *)f)[id] : ((const double *)f)[id];
}

orc_ctx *orc_prepare(const orc_scene *s, int32_t *err) {
  *err = ORC_ERR_ARG;
  if (!s || !s->rho || s->n_bands < 1 || s->n_bands > ORC_MAX_BANDS || !s->kappa) return NULL;
  if (s->emis_mode == 1 && (!s->temp || !s->lambda_table || s->n_tbins < 2)) return NULL;
  for (int a = 0; a < 3; ++a)
    if (s->n[a] < 1 || !(s->hi[a] > s->lo[a])) return NULL;
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  if (!c) { *err = ORC_ERR_OOM; return NULL; }
  c->s = *s;
  if (s->kind == 0) {
    for (int a = 0; a < 3; ++a) {
      c->nf[a] = s->n[a];
      c->hf[a] = (s->hi[a] - s->lo[a]) / (double)s->n[a];
    }
    *err = ORC_OK;
    return c;
  }
  if (s->kind != 1 || s->brick < 1 || s->max_level < 0 || s->max_level >= ORC_MAX_LEVELS ||
      s->n_bricks < 1 || !s->brick_level || !s->brick_origin) {
    orc_release(c);
    return NULL;
  }
  const int Lm = s->max_level, B = s->brick;
  for (int a = 0; a < 3; ++a) {
    if (s->n[a] % B) { orc_release(c); return NULL; }
    c->nf[a] = (int64_t)s->n[a] << Lm;
    c->hf[a] = (s->hi[a] - s->lo[a]) / (double)c->nf[a];
  }
  for (int l = 0; l <= Lm; ++l) {
    int64_t S = (int64_t)B << (Lm - l), cnt = 1;
    for (int a = 0; a < 3; ++a) { c->md[l][a] = c->nf[a] / S; cnt *= c->md[l][a]; }
    c->map[l] = (int32_t *)malloc(sizeof(int32_t) * cnt);
    if (!c->map[l]) { orc_release(c); *err = ORC_ERR_OOM; return NULL; }
    for (int64_t k = 0; k < cnt; ++k) c->map[l][k] = -1;
  }
  /* place every leaf brick in its level's map */
  double covered = 0.0, total = (double)c->nf[0] * (double)c->nf[1] * (double)c->nf[2];
  for (int b = 0; b < s->n_bricks; ++b) {
    int l = s->brick_level[b];
    if (l < 0 || l > Lm) { orc_release(c); return NULL; }
    int64_t S = (int64_t)B << (Lm - l), bc[3];
    for (int a = 0; a < 3; ++a) {
      int64_t o = s->brick_origin[3 * b + a];
      if (o < 0 || o % S || o + S > c->nf[a]) { orc_release(c); return NULL; }
      bc[a] = o / S;
    }
    int64_t idx = (bc[2] * c->md[l][1] + bc[1]) * c->md[l][0] + bc[0];
    if (c->map[l][idx] != -1) { orc_release(c); return NULL; }
    c->map[l][idx] = b;
    covered += (double)S * (double)S * (double)S;
  }
  /* no leaf brick may lie inside another leaf brick; together they must fill the box */
  for (int b = 0; b < s->n_bricks; ++b) {
    int l = s->brick_level[b];
    for (int lc = 0; lc < l; ++lc) {
      int64_t S = (int64_t)B << (Lm - lc), bc[3];
      for (int a = 0; a < 3; ++a) bc[a] = s->brick_origin[3 * b + a] / S;
      if (c->map[lc][(bc[2] * c->md[lc][1] + bc[1]) * c->md[lc][0] + bc[0]] != -1) {
        orc_release(c);
        return NULL;
      }
    }
  }
  if (covered != total) { orc_release(c); return NULL; }
  *err = ORC_OK;
  return c;
}

/* ------------------------------------------------------------ emissivity */

double orc_lambda(const orc_ctx *c, int32_t band, double T) {
  const orc_scene *s = &c->s;
  int nt = s->n_tbins;
  double x = (log10(T) - s->logT_lo) / (s->logT_hi - s->logT_lo) * (double)(nt - 1);
  if (!(x > 0.0)) x = 0.0;
  if (x > (double)(nt - 1)) x = (double)(nt - 1);
  int k = (int)floor(x);
  if (k > nt - 2) k = nt - 2;
  double w = x - (double)k;
  const double *tab = s->lambda_table + (int64_t)band * nt;
  return (1.0 - w) * tab[k] + w * tab[k + 1];
}

/* ------------------------------------------------------------------ march */

/* Leaf cell holding the point at ray parameter t: the finest-level cell index
 * of the point (half-open cells), then the leaf brick containing it. */
static int64_t cell_at(const orc_ctx *c, const double *o, const double *d, double t) {
  int64_t f[3];
  for (int a = 0; a < 3; ++a) {
    double x = o[a] + t * d[a];
    int64_t k = (int64_t)floor((x - c->s.lo[a]) / c->hf[a]);
    if (k < 0) k = 0;
    if (k > c->nf[a] - 1) k = c->nf[a] - 1;
    f[a] = k;
  }
  if (c->s.kind == 0) return (f[2] * c->nf[1] + f[1]) * c->nf[0] + f[0];
  const int Lm = c->s.max_level, B = c->s.brick;
  for (int l = 0; l <= Lm; ++l) {
    int64_t S = (int64_t)B << (Lm - l);
    int64_t idx = ((f[2] / S) * c->md[l][1] + f[1] / S) * c->md[l][0] + f[0] / S;
    int32_t b = c->map[l][idx];
    if (b >= 0) {
      const int32_t *org = c->s.brick_origin + 3 * (int64_t)b;
      int sh = Lm - l;
      int64_t lx = (f[0] - org[0]) >> sh, ly = (f[1] - org[1]) >> sh, lz = (f[2] - org[2]) >> sh;
      return (int64_t)b * B * B * B + (lz * B + ly) * B + lx;
    }
  }
  return -1; /* unreachable for a validated tiling */
}

typedef struct {
  double col;
  double tau[ORC_MAX_BANDS];
  double *inten;
  int64_t steps;
} ray_acc;

/* One cell chord of length ds: column density and the per-cell formal solution
 * of the transfer equation with constant source function j/alpha. */
static void add_chord(const orc_ctx *c, ray_acc *r, int64_t id, double ds) {
  const orc_scene *s = &c->s;
  double rho = field_at(s, s->rho, id);
  r->col += rho * ds;
  r->steps += 1;
  for (int b = 0; b < s->n_bands; ++b) {
    double alpha = s->kappa[b] * rho;
    double dtau = alpha * ds;
    double j = rho * rho;
    if (s->emis_mode == 1) j *= orc_lambda(c, b, field_at(s, s->temp, id));
    double att = exp(-r->tau[b]);
    double term = (alpha > 0.0) ? (j / alpha) * (-expm1(-dtau)) * att : j * ds * att;
    r->inten[b] += term;
    r->tau[b] += dtau;
  }
}

static double plane_t(const orc_ctx *c, int a, int64_t k, const double *o, const double *d) {
  return (c->s.lo[a] + (double)k * c->hf[a] - o[a]) / d[a];
}

static void trace_segment(const orc_ctx *c, const double *o, const double *d, double t0, double t1,
                          double *col, double *inten, int64_t *steps) {
  ray_acc r;
  memset(&r, 0, sizeof(r));
  r.inten = inten;
  for (int b = 0; b < c->s.n_bands; ++b) inten[b] = 0.0;
  /* next interior finest-level plane crossed along each axis, k in [1, nf-1] */
  int64_t k[3];
  int has[3], sg[3];
  double tk[3];
  for (int a = 0; a < 3; ++a) {
    has[a] = 0;
    if (d[a] == 0.0) continue;
    int64_t nf = c->nf[a];
    double xs = (o[a] + t0 * d[a] - c->s.lo[a]) / c->hf[a];
    if (d[a] > 0) {
      sg[a] = 1;
      int64_t kk = (int64_t)floor(xs) + 1;
      if (kk < 1) kk = 1;
      if (kk > nf) kk = nf;
      while (kk > 1 && plane_t(c, a, kk - 1, o, d) > t0) --kk;
      while (kk <= nf - 1 && plane_t(c, a, kk, o, d) <= t0) ++kk;
      if (kk <= nf - 1) { has[a] = 1; k[a] = kk; }
    } else {
      sg[a] = -1;
      int64_t kk = (int64_t)ceil(xs) - 1;
      if (kk > nf - 1) kk = nf - 1;
      if (kk < 0) kk = 0;
      while (kk < nf - 1 && plane_t(c, a, kk + 1, o, d) > t0) ++kk;
      while (kk >= 1 && plane_t(c, a, kk, o, d) <= t0) --kk;
      if (kk >= 1) { has[a] = 1; k[a] = kk; }
    }
    if (has[a]) tk[a] = plane_t(c, a, k[a], o, d);
  }
  int64_t cur = -1;
  double run_a = t0, run_b = t0, t = t0;
  while (t < t1) {
    double tn = t1;
    for (int a = 0; a < 3; ++a)
      if (has[a] && tk[a] < tn) tn = tk[a];
    if (tn > t) {
      int64_t id = cell_at(c, o, d, 0.5 * (t + tn));
      if (id != cur) {
        if (cur >= 0) add_chord(c, &r, cur, run_b - run_a);
        cur = id;
        run_a = t;
      }
      run_b = tn;
    }
    for (int a = 0; a < 3; ++a) {
      if (has[a] && tk[a] == tn) {
        k[a] += sg[a];
        if (k[a] < 1 || k[a] > c->nf[a] - 1) has[a] = 0;
        else tk[a] = plane_t(c, a, k[a], o, d);
      }
    }
    t = tn;
  }
  if (cur >= 0) add_chord(c, &r, cur, run_b - run_a);
  *col = r.col;
  *steps = r.steps;
}

typedef struct {
  double d[3], u[3], v[3];
} basis_t;

static int make_basis(const orc_view *v, basis_t *b) {
  double n = sqrt(v->dir[0] * v->dir[0] + v->dir[1] * v->dir[1] + v->dir[2] * v->dir[2]);
  if (!(n > 0.0) || !(v->half_extent > 0.0)) return 0;
  for (int a = 0; a < 3; ++a) b->d[a] = v->dir[a] / n;
  /* u = normalize(up x d), v = d x u */
  double ux = v->up[1] * b->d[2] - v->up[2] * b->d[1];
  double uy = v->up[2] * b->d[0] - v->up[0] * b->d[2];
  double uz = v->up[0] * b->d[1] - v->up[1] * b->d[0];
  double un = sqrt(ux * ux + uy * uy + uz * uz);
  if (!(un > 0.0)) return 0;
  b->u[0] = ux / un; b->u[1] = uy / un; b->u[2] = uz / un;
  b->v[0] = b->d[1] * b->u[2] - b->d[2] * b->u[1];
  b->v[1] = b->d[2] * b->u[0] - b->d[0] * b->u[2];
  b->v[2] = b->d[0] * b->u[1] - b->d[1] * b->u[0];
  return 1;
}

/* Pixel (L, i, j) of an n0 x n0 base image: centre u = -H + (i + 1/2) * (2H / (n0 2^L)). */
static void trace_pixel(const orc_ctx *c, const orc_view *v, const basis_t *bs, int n0, int L,
                        int i, int j, double *col, double *inten, int64_t *steps) {
  double H = v->half_extent;
  double nL = ldexp((double)n0, L);
  double pix = (2.0 * H) / nL;
  double uc = -H + ((double)i + 0.5) * pix;
  double vc = -H + ((double)j + 0.5) * pix;
  double o[3];
  for (int a = 0; a < 3; ++a) o[a] = v->center[a] + uc * bs->u[a] + vc * bs->v[a];
  double t0 = -INFINITY, t1 = INFINITY;
  int miss = 0;
  for (int a = 0; a < 3; ++a) {
    if (bs->d[a] == 0.0) {
      if (o[a] < c->s.lo[a] || o[a] >= c->s.hi[a]) miss = 1;
    } else {
      double ta = (c->s.lo[a] - o[a]) / bs->d[a], tb = (c->s.hi[a] - o[a]) / bs->d[a];
      if (ta > tb) { double x = ta; ta = tb; tb = x; }
      if (ta > t0) t0 = ta;
      if (tb < t1) t1 = tb;
    }
  }
  if (miss || !(t0 < t1)) {
    *col = 0.0;
    *steps = 0;
    for (int b = 0; b < c->s.n_bands; ++b) inten[b] = 0.0;
    return;
  }
  trace_segment(c, o, bs->d, t0, t1, col, inten, steps);
}

int32_t orc_trace(const orc_ctx *c, const orc_view *v, int32_t n0, int64_t n_rays,
                  const int32_t *L, const int32_t *I, const int32_t *J, double *col,
                  double *inten, int64_t *steps) {
  basis_t bs;
  if (!c || !v || n0 < 1 || !make_basis(v, &bs)) return ORC_ERR_ARG;
  const int nb = c->s.n_bands;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < n_rays; ++k)
    trace_pixel(c, v, &bs, n0, L[k], I[k], J[k], &col[k], &inten[k * nb], &steps[k]);
  return ORC_OK;
}

/* ------------------------------------------------------- refinement (Eq. 2) */

double orc_xi(const double *s, int32_t xi_norm) {
  double c = s[4];
  double xm = s[3], xp = s[5], ym = s[1], yp = s[7];
  double mm = s[0], pm = s[2], mp = s[6], pp = s[8];
  /* second differences (d2p/dx_u dx_v) dx_u dx_v at the pixel centre */
  double d2u = (xp - 2.0 * c) + xm;
  double d2v = (yp - 2.0 * c) + ym;
  double duv = (((pp - pm) - mp) + mm) * 0.25;
  double num = (d2u * d2u + d2v * d2v) + 2.0 * (duv * duv);
  /* first differences at i+1/2 and i-1/2 along each axis */
  double au = fabs(xp - c) + fabs(c - xm);
  double av = fabs(yp - c) + fabs(c - ym);
  double den = au * au + av * av;
  if (xi_norm == 1) den = 2.0 * den;
  if (num == 0.0) return 0.0;
  if (den == 0.0) return 1.0;
  double xi = sqrt(num / den);
  return xi > 1.0 ? 1.0 : xi;
}

typedef struct {
  int n0, Lm;
  int32_t *map[ORC_MAX_LEVELS]; /* node index at (level, i, j), -1 if no node */
} node_maps;

static int32_t deepest(const node_maps *m, int L, int64_t i, int64_t j) {
  for (int l = L; l >= 0; --l) {
    int sh = L - l;
    int64_t nl = (int64_t)m->n0 << l;
    int32_t k = m->map[l][(j >> sh) * nl + (i >> sh)];
    if (k >= 0) return k;
  }
  return -1;
}

/* Stencil of node k (Eq. 2 at level L): the node whose value each of the nine
 * positions takes, indexed [dj+1][di+1]. Positions outside the image are
 * clamped to its edge; a position with no node at level L takes the deepest
 * existing node at a level <= L covering it. */
static void stencil_nodes(const orc_tree *t, const node_maps *m, int64_t k, int32_t q[9]) {
  int L = t->level[k];
  int64_t nl = (int64_t)m->n0 << L;
  for (int dj = -1; dj <= 1; ++dj)
    for (int di = -1; di <= 1; ++di) {
      int64_t ii = (int64_t)t->i[k] + di, jj = (int64_t)t->j[k] + dj;
      if (ii < 0) ii = 0;
      if (ii > nl - 1) ii = nl - 1;
      if (jj < 0) jj = 0;
      if (jj > nl - 1) jj = nl - 1;
      q[3 * (dj + 1) + (di + 1)] = deepest(m, L, ii, jj);
    }
}

typedef struct {
  int64_t *idx[ORC_MAX_LEVELS];
} replay_maps;

/* First-order bound of how far xi can move when each stencil value s_k moves
 * by up to rtol |s_k| (the tolerance the GPU's pixel values are held to): the
 * sum over the nine positions of the larger one-sided change of xi. One-sided
 * changes (not a central difference) keep the larger slope at the kinks of
 * the |.| terms of the denominator. */
static double xi_margin(const double s[9], int xi_norm, double rtol) {
  const double x0 = orc_xi(s, xi_norm);
  double w[9], d = 0.0;
  memcpy(w, s, sizeof(w));
  for (int k = 0; k < 9; ++k) {
    const double tol = rtol * fabs(s[k]);
    if (tol == 0.0) continue;
    w[k] = s[k] + tol;
    const double a = fabs(orc_xi(w, xi_norm) - x0);
    w[k] = s[k] - tol;
    const double b = fabs(orc_xi(w, xi_norm) - x0);
    w[k] = s[k];
    d += a > b ? a : b;
  }
  return d;
}

/* One flag decision of the scan for parameter `which` (0 intensity, 1 column
 * density) of node k. Plain mode (h NULL): xi >= xi_crit on this tree's
 * values. Hybrid mode: the same, unless |xi - xi_crit| <= margin x the
 * first-order bound above ("undecided": within the value tolerance either
 * answer is correct); an undecided decision is taken from the other side's
 * values of the same nine stencil nodes, looked up by (level, i, j), when all
 * nine are there. */
static int decide(const orc_tree *t, const node_maps *m, int64_t k, int which,
                  const orc_params *p, const orc_replay *other, const replay_maps *om,
                  orc_hybrid *h) {
  int32_t q[9];
  double s[9];
  stencil_nodes(t, m, k, q);
  for (int x = 0; x < 9; ++x) s[x] = which ? t->col[q[x]] : t->p_int[q[x]];
  const double xi = orc_xi(s, p->xi_norm);
  const int own = xi >= p->xi_crit;
  if (!h) return own;
  h->n_decisions += 1;
  const double d = h->margin * xi_margin(s, p->xi_norm, h->rtol);
  if (fabs(xi - p->xi_crit) > d) return own;
  h->n_undecided += 1;
  double so[9];
  for (int x = 0; x < 9; ++x) {
    const int32_t n = q[x];
    const int L = t->level[n];
    const int64_t nl = (int64_t)m->n0 << L;
    const int64_t r = om->idx[L][(int64_t)t->j[n] * nl + t->i[n]];
    if (r < 0) {
      h->n_unresolved += 1;
      return own;
    }
    so[x] = which ? other->p_col[r] : other->p_int[r];
  }
  const int oth = orc_xi(so, p->xi_norm) >= p->xi_crit;
  if (oth != own) h->n_taken_from_other += 1;
  return oth;
}

static int32_t fill_nodes(const orc_ctx *c, const orc_view *v, int n0, orc_tree *t, int64_t a,
                          int64_t b, const orc_replay *rp, const replay_maps *rm) {
  const int nb = c->s.n_bands;
  if (rp) {
    for (int64_t k = a; k < b; ++k) {
      int L = t->level[k];
      int64_t nl = (int64_t)n0 << L;
      int64_t r = rm->idx[L][(int64_t)t->j[k] * nl + t->i[k]];
      if (r < 0) return ORC_ERR_REPLAY_MISSING;
      t->p_int[k] = rp->p_int[r];
      t->col[k] = rp->p_col[r];
      for (int bb = 0; bb < nb; ++bb) t->inten[k * nb + bb] = 0.0;
      t->steps[k] = 0;
    }
    return ORC_OK;
  }
  int32_t e = orc_trace(c, v, n0, b - a, t->level + a, t->i + a, t->j + a, t->col + a,
                        t->inten + a * nb, t->steps + a);
  if (e) return e;
  for (int64_t k = a; k < b; ++k) {
    double s = 0.0;
    for (int bb = 0; bb < nb; ++bb) s += t->inten[k * nb + bb];
    t->p_int[k] = s;
  }
  return ORC_OK;
}

/* The AIR sweep loop. rp: pixel values come from this table instead of
 * tracing (replay). other + h: hybrid decisions (see decide); values are
 * traced. */
static int32_t air_loop(const orc_ctx *c, const orc_view *v, const orc_params *p, orc_tree *t,
                        const orc_replay *rp, const orc_replay *other, orc_hybrid *h) {
  if (!c || !v || !p || !t) return ORC_ERR_ARG;
  if ((other != NULL) != (h != NULL) || (other && rp)) return ORC_ERR_ARG;
  const orc_replay *tab = rp ? rp : other; /* the table the maps index */
  const int n0 = p->base_res, Lm = p->max_level;
  if (n0 < 1 || Lm < 0 || Lm >= ORC_MAX_LEVELS || !(p->xi_crit >= 0.0) || p->refine_on < 0 ||
      p->refine_on > 2 || (p->xi_norm != 0 && p->xi_norm != 1))
    return ORC_ERR_ARG;
  if ((int64_t)n0 * n0 > t->capacity) return ORC_ERR_CAPACITY;
  int32_t err = ORC_OK;
  node_maps m;
  replay_maps rm;
  memset(&m, 0, sizeof(m));
  memset(&rm, 0, sizeof(rm));
  uint8_t *flag = (uint8_t *)calloc((size_t)t->capacity, 1);
  m.n0 = n0;
  m.Lm = Lm;
  if (!flag) return ORC_ERR_OOM;
  for (int l = 0; l <= Lm; ++l) {
    int64_t nl = (int64_t)n0 << l;
    m.map[l] = (int32_t *)malloc(sizeof(int32_t) * nl * nl);
    if (!m.map[l]) { err = ORC_ERR_OOM; goto done; }
    for (int64_t q = 0; q < nl * nl; ++q) m.map[l][q] = -1;
    if (tab) {
      rm.idx[l] = (int64_t *)malloc(sizeof(int64_t) * nl * nl);
      if (!rm.idx[l]) { err = ORC_ERR_OOM; goto done; }
      for (int64_t q = 0; q < nl * nl; ++q) rm.idx[l][q] = -1;
    }
  }
  if (tab) {
    for (int64_t r = 0; r < tab->n; ++r) {
      int L = tab->level[r];
      if (L < 0 || L > Lm) continue;
      int64_t nl = (int64_t)n0 << L;
      if (tab->i[r] < 0 || tab->i[r] >= nl || tab->j[r] < 0 || tab->j[r] >= nl) continue;
      rm.idx[L][(int64_t)tab->j[r] * nl + tab->i[r]] = r;
    }
  }
  if (h) h->n_decisions = h->n_undecided = h->n_taken_from_other = h->n_unresolved = 0;
  /* step (i): base image, row-major */
  int64_t n = 0;
  for (int j = 0; j < n0; ++j)
    for (int i = 0; i < n0; ++i) {
      t->level[n] = 0; t->i[n] = i; t->j[n] = j; t->leaf[n] = 1; t->parent[n] = -1;
      m.map[0][(int64_t)j * n0 + i] = (int32_t)n;
      ++n;
    }
  /* step (ii) */
  err = fill_nodes(c, v, n0, t, 0, n, rp, &rm);
  if (err) goto done;
  t->n_sweeps = 0;
  t->n_refined = 0;
  for (;;) {
    /* step (iii): truncation-error scan of every leaf below the maximum level */
    for (int64_t k = 0; k < n; ++k) {
      flag[k] = 0;
      if (!t->leaf[k] || t->level[k] >= Lm) continue;
      int f = 0;
      if (p->refine_on == 0 || p->refine_on == 2) f |= decide(t, &m, k, 0, p, other, &rm, h);
      if (p->refine_on == 1 || p->refine_on == 2) f |= decide(t, &m, k, 1, p, other, &rm, h);
      flag[k] = (uint8_t)f;
    }
    /* step (iii): adjacent pixels may differ by at most one level after refinement */
    for (int changed = 1; changed;) {
      changed = 0;
      for (int64_t k = 0; k < n; ++k) {
        if (!flag[k]) continue;
        int L = t->level[k];
        int64_t nl = (int64_t)n0 << L;
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            if (!di && !dj) continue;
            int64_t ii = (int64_t)t->i[k] + di, jj = (int64_t)t->j[k] + dj;
            if (ii < 0 || jj < 0 || ii >= nl || jj >= nl) continue;
            int32_t q = deepest(&m, L, ii, jj);
            if (t->leaf[q] && t->level[q] < L && !flag[q]) {
              flag[q] = 1;
              changed = 1;
            }
          }
      }
    }
    int64_t nflag = 0;
    for (int64_t k = 0; k < n; ++k) nflag += flag[k];
    if (nflag == 0) break;
    if (n + 4 * nflag > t->capacity) { err = ORC_ERR_CAPACITY; t->n_nodes = n + 4 * nflag; goto done; }
    /* step (iv): four children per flagged leaf, in node order, child c = 2*dj + di */
    int64_t n_old = n;
    for (int64_t k = 0; k < n_old; ++k) {
      if (!flag[k]) continue;
      int L = t->level[k] + 1;
      int64_t nl = (int64_t)n0 << L;
      for (int ch = 0; ch < 4; ++ch) {
        t->level[n] = L;
        t->i[n] = 2 * t->i[k] + (ch & 1);
        t->j[n] = 2 * t->j[k] + (ch >> 1);
        t->leaf[n] = 1;
        t->parent[n] = (int32_t)k;
        m.map[L][(int64_t)t->j[n] * nl + t->i[n]] = (int32_t)n;
        ++n;
      }
      t->leaf[k] = 0;
    }
    t->n_refined += nflag;
    t->n_sweeps += 1;
    /* step (ii) for the new pixels, then loop (step v) */
    err = fill_nodes(c, v, n0, t, n_old, n, rp, &rm);
    if (err) goto done;
  }
  t->n_nodes = n;
  t->n_leaves = 0;
  t->n_steps = 0;
  for (int64_t k = 0; k < n; ++k) {
    t->n_leaves += t->leaf[k];
    t->n_steps += t->steps[k];
  }
done:
  for (int l = 0; l < ORC_MAX_LEVELS; ++l) {
    free(m.map[l]);
    free(rm.idx[l]);
  }
  free(flag);
  return err;
}

int32_t orc_air(const orc_ctx *c, const orc_view *v, const orc_params *p, orc_tree *out,
                const orc_replay *replay) {
  return air_loop(c, v, p, out, replay, NULL, NULL);
}

int32_t orc_air_hybrid(const orc_ctx *c, const orc_view *v, const orc_params *p, orc_tree *out,
                       const orc_replay *other, orc_hybrid *h) {
  if (!other || !h || !(h->rtol >= 0.0) || !(h->margin >= 0.0)) return ORC_ERR_ARG;
  return air_loop(c, v, p, out, NULL, other, h);
}
