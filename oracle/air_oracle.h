/* air_oracle.h -- plain FP64 CPU oracle for adaptive image ray-tracing (AIR).
 *
 * TEST INFRASTRUCTURE ONLY. This header and air_oracle.c are the slow,
 * obviously-correct reference that the tests, the smoke check and the
 * benchmark's CPU-baseline leg compare the CUDA library against. The product
 * library never includes, links or calls it, and it shares no code with it.
 *
 * Method: E. R. Parkin (2010), "Adaptive image ray-tracing for astrophysical
 * simulations", MNRAS Letters. Section 2 steps (i)-(vi), Eq. 1 and Eq. 2.
 */
#ifndef AIR_ORACLE_H
#define AIR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_LEVELS 16
#define ORC_MAX_BANDS 64

enum {
  ORC_OK = 0,
  ORC_ERR_ARG = 1,
  ORC_ERR_OOM = 2,
  ORC_ERR_CAPACITY = 4,
  ORC_ERR_REPLAY_MISSING = 7
};

/* Simulation grid. Uniform: n[0]*n[1]*n[2] cells, fields [n2][n1][n0] (x fastest).
 * Block AMR: n[] base cells per axis, bricks of brick^3 cells, leaf bricks only,
 * brick b at level brick_level[b] with origin brick_origin[3b..3b+2] in units of
 * the finest-level cell; fields [n_bricks][brick][brick][brick] (x fastest). */
typedef struct {
  int32_t kind; /* 0 uniform, 1 block-AMR */
  int32_t n[3];
  double lo[3], hi[3];
  int32_t brick, max_level, n_bricks;
  const int32_t *brick_level;
  const int32_t *brick_origin;
  const void *rho;             /* double, or float when field_f32 (read exactly as double) */
  const void *temp;            /* NULL allowed when emis_mode == 0 */
  int32_t n_bands, emis_mode;  /* emis_mode 0: j = rho^2 ; 1: j = rho^2 Lambda_b(T) */
  const double *lambda_table;  /* [n_bands][n_tbins] */
  int32_t n_tbins;
  double logT_lo, logT_hi;
  const double *kappa;         /* [n_bands], opacity per unit density */
  int32_t field_f32;           /* 1: rho and temp are float arrays */
} orc_scene;

typedef struct {
  double dir[3], up[3], center[3];
  double half_extent;
} orc_view;

typedef struct {
  int32_t base_res, max_level;
  double xi_crit;
  int32_t xi_norm;   /* 0: axis-sum denominator, 1: literal sum over u,v */
  int32_t refine_on; /* 0: band-summed intensity, 1: column density, 2: either */
} orc_params;

/* Externally supplied per-node values (replay): the refinement loop looks up the
 * parameter values of node (level, i, j) here instead of tracing its ray. */
typedef struct {
  int64_t n;
  const int32_t *level, *i, *j;
  const double *p_int;  /* band-summed intensity */
  const double *p_col;  /* column density */
} orc_replay;

typedef struct {
  int64_t capacity; /* entries available in every per-node array */
  int64_t n_nodes, n_leaves, n_refined, n_sweeps, n_steps; /* out */
  int32_t *level, *i, *j, *leaf, *parent; /* [capacity] */
  double *col;   /* [capacity] column density */
  double *inten; /* [capacity][n_bands] */
  double *p_int; /* [capacity] band-summed intensity */
  int64_t *steps;/* [capacity] cell segments crossed by the node's ray */
} orc_tree;

typedef struct orc_ctx orc_ctx;

orc_ctx *orc_prepare(const orc_scene *s, int32_t *err);
void orc_release(orc_ctx *c);

/* Trace n_rays rays of pixels (L[k], I[k], J[k]) of a base image n0 x n0. */
int32_t orc_trace(const orc_ctx *c, const orc_view *v, int32_t n0, int64_t n_rays,
                  const int32_t *L, const int32_t *I, const int32_t *J, double *col,
                  double *inten /* [n_rays][n_bands] */, int64_t *steps);

/* The AIR sweep loop, Section 2 (ii)-(v). replay may be NULL. */
int32_t orc_air(const orc_ctx *c, const orc_view *v, const orc_params *p, orc_tree *out,
                const orc_replay *replay);

/* Tree comparison where decisions sit within the value tolerance of the
 * threshold. The sweep loop traces its own values, but a flag decision whose
 * |xi - xi_crit| is within margin x (first-order bound of the change of xi
 * when each stencil value moves by rtol of itself) is "undecided" and is
 * taken from `other`'s values of the same stencil nodes (looked up by
 * level, i, j). A tree built this way equals the other side's tree exactly
 * when the two differ only in undecided decisions. */
typedef struct {
  double rtol, margin;          /* in */
  int64_t n_decisions;          /* out: xi evaluations of the scan */
  int64_t n_undecided;          /* out: of those, within the margin */
  int64_t n_taken_from_other;   /* out: undecided ones where other's answer differed */
  int64_t n_unresolved;         /* out: undecided ones with a stencil node missing in other */
} orc_hybrid;

int32_t orc_air_hybrid(const orc_ctx *c, const orc_view *v, const orc_params *p, orc_tree *out,
                       const orc_replay *other, orc_hybrid *h);

/* Eq. 2 on a 3x3 stencil s[dj+1][di+1] (pixel (i+di, j+dj)). */
double orc_xi(const double *s9, int32_t xi_norm);

/* Lambda_b(T) by the table interpolation the oracle uses. */
double orc_lambda(const orc_ctx *c, int32_t band, double T);

#ifdef __cplusplus
}
#endif
#endif
