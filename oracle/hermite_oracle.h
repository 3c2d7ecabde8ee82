/*
 * FP64 CPU oracle for the list-driven 4th-order Hermite force evaluation of
 * Fukushige & Kawai, "Hierarchical Tree Algorithm for Collisional N-body
 * Simulations on GRAPE" (arXiv:1602.02832).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code: only the tests, the package entry point's smoke check and
 * the benchmark's CPU-baseline leg use it.  It shares no source with the CUDA
 * path.
 *
 * Layout: every 3-vector array is array-of-structures, double[n][3].
 * Indices: after a tree build, particles are numbered 0..n-1 in Morton order
 * and tree cells n..n+n_cells-1 in pre-order (the root is cell 0, index n).
 */
#ifndef HERMITE_ORACLE_H
#define HERMITE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Plummer-softened force, jerk and potential from all other particles
 * (direct N^2 sum, the force step of the original GRAPE-6 Hermite loop). */
void hho_direct_force(int n, const double *x, const double *v, const double *m,
                      double eps2, double *acc, double *jerk, double *pot);

/* Same sum restricted to the i-particles listed in i_idx (targets inside the
 * j set given by x, v, m).  Used for sampled checks at large n. */
void hho_direct_force_subset(int n, const double *x, const double *v, const double *m,
                             double eps2, int n_i, const int32_t *i_idx,
                             double *acc, double *jerk, double *pot);

/* Force on active i from the entries of its group's interaction list (step 5
 * of the tree loop).  xj/vj/mj: predicted j entries (particles then nodes),
 * n_j of them.  gid[k]: list (group) index for active particle i_idx[k].
 * The entry equal to the i-particle's own index is skipped. */
void hho_list_force(int n_j, const double *xj, const double *vj, const double *mj,
                    int n_act, const int32_t *i_idx, const int32_t *gid,
                    const int64_t *list_off, const int32_t *list_idx, double eps2,
                    double *acc, double *jerk, double *pot);

/* 3rd-order Taylor predictor for n entries with their own times t0[k]. */
void hho_predict(int n, const double *x, const double *v, const double *a, const double *jk,
                 const double *t0, double t, double *xp, double *vp);

/* 4th-order Hermite corrector for one particle over a step of length dt.
 * On entry xp/vp are the predicted values; a0/j0 the old and a1/j1 the new
 * force and jerk.  Writes corrected x1/v1 and the 2nd/3rd derivatives of the
 * acceleration at the END of the step (a2_end, a3). */
void hho_correct_one(double dt, const double xp[3], const double vp[3],
                     const double a0[3], const double j0[3],
                     const double a1[3], const double j1[3],
                     double x1[3], double v1[3], double a2_end[3], double a3[3]);

/* Aarseth timestep criterion (unquantised). */
double hho_aarseth_dt(double eta, const double a[3], const double j[3],
                      const double a2[3], const double a3[3]);

/* Power-of-two block quantisation of a new step (see the .c file). */
double hho_block_dt(double dt_want, double dt_old, double t_new, double dt_min, double dt_max);

/* Initial step eta_s |a| / |j|, quantised. */
double hho_initial_dt(double eta_s, const double a[3], const double j[3],
                      double dt_min, double dt_max);

/* ---- Octree (Morton or Peano-Hilbert order), groups and interaction lists ---- */
typedef struct hho_tree hho_tree;

/* 3-bits-per-level keys of grid cell (ix, iy, iz): Morton (bit interleaving,
 * x highest) and Peano-Hilbert (Section 2; Skilling 2004) on a 2^bits grid. */
uint64_t hho_morton_key(uint32_t ix, uint32_t iy, uint32_t iz);
uint64_t hho_hilbert_key(uint32_t ix, uint32_t iy, uint32_t iz, int bits);

/* order 0: Morton (hho_tree_build), 1: Peano-Hilbert.  The octree and the
 * groups are the same in both orders; only the order of children, and so of
 * particles, nodes and list entries, differs. */
hho_tree *hho_tree_build(int n, const double *x, const double *v, const double *a,
                         const double *jk, const double *m,
                         int leaf, int n_crit, double theta);
hho_tree *hho_tree_build_ordered(int n, const double *x, const double *v, const double *a,
                                 const double *jk, const double *m,
                                 int leaf, int n_crit, double theta, int order);
void     hho_tree_free(hho_tree *t);
int      hho_tree_n_cells(const hho_tree *t);
int      hho_tree_n_groups(const hho_tree *t);
int64_t  hho_tree_list_len(const hho_tree *t);
/* perm[k] = input index of the particle at Morton position k */
void     hho_tree_perm(const hho_tree *t, int32_t *perm);
void     hho_tree_keys(const hho_tree *t, uint64_t *keys);
/* node records: x, v, a, jk [n_cells][3], mass [n_cells] */
void     hho_tree_nodes(const hho_tree *t, double *x, double *v, double *a, double *jk, double *m);
/* per cell: begin, end (Morton particle range), depth, side */
void     hho_tree_cells(const hho_tree *t, int32_t *begin, int32_t *end, int32_t *depth, double *side);
/* per group: cell id, begin, end; per particle (Morton order): group id */
void     hho_tree_groups(const hho_tree *t, int32_t *g_cell, int32_t *g_begin, int32_t *g_end,
                         int32_t *group_of);
/* CSR lists: off[n_groups+1], idx[list_len] (ascending within each list) */
void     hho_tree_lists(const hho_tree *t, int64_t *off, int32_t *idx);

/* ---- Whole Hermite block-step run (the tree loop of Section 2) ---- */
typedef struct {
    double eps2, eta, eta_s, dt_min, dt_max, dt_tree, theta;
    int leaf, n_crit;
    int use_tree;      /* 0: direct N^2 force (the original Hermite loop) */
} hho_params;

typedef struct {
    int64_t block_steps, particle_steps, interactions, rebuilds;
} hho_stats;

/* Integrates n particles (x, v updated in place, input order kept) from t=0
 * to t_end.  a/jk/t/dt (may be NULL) receive the final derivatives, times and
 * steps. */
int hho_run(int n, double *x, double *v, const double *m, double t_end,
            const hho_params *p, double *a, double *jk, double *t, double *dt,
            hho_stats *stats);

/* hho_run continued from a synchronised state at t0, a multiple of dt_tree:
 * every particle at t0 with its forces a, jk there and its block step dt.
 * The tree is rebuilt from that state (Section 2, step 1) and block steps
 * follow until t_end; x, v, a, jk, dt are updated in place.  Resuming the
 * state hho_run reached at t0 gives the same result as one hho_run. */
int hho_resume(int n, double *x, double *v, double *a, double *jk, double *dt, const double *m, double t0,
               double t_end, const hho_params *p, hho_stats *stats);

/* Total energy: kinetic plus the direct-summation softened potential energy. */
double hho_energy(int n, const double *x, const double *v, const double *m, double eps2);

/* Threads the OpenMP loops use (for reporting). */
int hho_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
