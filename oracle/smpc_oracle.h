/*
 * FP64 CPU oracle of one sampling-based MPC (SMPC) iteration (ParaMaP,
 * arXiv 2512.22575, Sec. IV and Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * definition the CUDA path is checked against.  It shares no code, header,
 * table or constant with the CUDA path.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it.
 *
 * Layout conventions (shared with the inputs, not with the CUDA code):
 *   joint arrays are indexed j = 0..n-1 for joint i = j+1;
 *   U, eps are row-major [H][n];
 *   the distance grid is float32 [nz][ny][nx] (x fastest);
 *   poses are 4x4 homogeneous, row-major.
 */
#ifndef SMPC_ORACLE_H
#define SMPC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_J 8
#define OR_MAX_S 64
#define OR_MAX_P 2048

typedef struct {
    int n_joints;
    double a[OR_MAX_J];            /* a_{i-1} */
    double d[OR_MAX_J];            /* d_i */
    double alpha[OR_MAX_J];        /* alpha_{i-1} */
    double theta_offset[OR_MAX_J];
    double flange_d;
    double q_min[OR_MAX_J], q_max[OR_MAX_J];
    double qd_max[OR_MAX_J], qdd_max[OR_MAX_J];
    int n_spheres;
    int sphere_link[OR_MAX_S];     /* frame index 1..n */
    double sphere_offset[OR_MAX_S][3];
    double sphere_radius[OR_MAX_S];
    int n_pairs;
    int pairs[OR_MAX_P][2];
} or_robot;

typedef struct {
    int nx, ny, nz;
    double res;
    double origin[3];
    const float *phi;
} or_grid;

typedef struct {
    double Q[6], QH[6];            /* diagonals acting on xi = [v; omega] */
    double w_env, d_act, w_self;
    double w_q, w_qd, w_qdd, margin_frac;
    double w_s, w_ns;
    double q_ref[OR_MAX_J];
} or_cost;

/* Per-step cost columns written by or_rollout when trace != NULL. */
enum { OR_T_POSE = 0, OR_T_ENV, OR_T_SELF, OR_T_LIM_Q, OR_T_LIM_QD,
       OR_T_LIM_QDD, OR_T_SMOOTH, OR_T_NS, OR_T_COLS };

void   or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_word_to_uniform(uint32_t x);
void   or_normals(uint64_t seed, uint32_t iter, uint32_t m, uint32_t k, double z[8]);
void   or_fk(const or_robot *rb, const double *q, double T[][4][4]);
void   or_sphere_centres(const or_robot *rb, const double T[][4][4], double p[][3]);
double or_phi(const or_grid *g, const double p[3]);
void   or_se3_log(const double T[4][4], double xi[6]);
void   or_pose_error(const double Tg[4][4], const double Tee[4][4], double xi[6]);
void   or_integrate(int n, int H, double dt, const double *q0, const double *qd0,
                    const double *u, double *q, double *qd);
double or_rollout(const or_robot *rb, const or_grid *g, const or_cost *c,
                  const double *q0, const double *qd0, const double Tg[4][4],
                  const double *u, int H, double dt, double *trace);
int    or_smpc_iterate(const or_robot *rb, const or_grid *g, const or_cost *c,
                       const double *q0, const double *qd0, const double Tg[4][4],
                       double *U, int K, int H, double dt, double lambda,
                       const double *sigma, uint64_t seed, uint32_t iter_index,
                       double *costs, double *weights, int n_threads);
int    or_replan(const or_robot *rb, const or_grid *g, const or_cost *c,
                 double *q, double *qd, const double Tg[4][4], double *U,
                 int K, int H, double dt, double lambda, const double *sigma,
                 uint64_t seed, uint32_t replan_index, int n_iters,
                 double *u0_out, double *best_cost, int n_threads);
void   or_edt_bruteforce(const uint8_t *occ, int nx, int ny, int nz, int64_t *D);
void   or_eps_range(uint64_t seed, uint32_t iter, uint32_t m0, int count, int H, int n, const double *sigma,
                    double *eps);
void   or_pose_metrics(const or_robot *rb, const double *q, const double *Tg, double out[2]);
void   or_robot_mask(const or_robot *rb, const double *q, int nx, int ny, int nz, double res,
                     const double *origin, double inflate, uint8_t *occ);

#ifdef __cplusplus
}
#endif
#endif
