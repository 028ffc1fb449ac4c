/*
 * FP64 CPU oracle of one SMPC iteration (ParaMaP, arXiv 2512.22575).
 *
 * TEST INFRASTRUCTURE ONLY: the reference definition that the CUDA path is
 * checked against.  It is deliberately plain: straight loops in the order of
 * Algorithm 1 and of the cost definitions in Sec. IV-B, 4x4 matrix products
 * for the kinematics, no blocking, no fusion.  It shares no code with the
 * CUDA path.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it.
 *
 * Readings of the paper that this file fixes (the paper is silent on them):
 *  - Sampling distribution D (Alg. 1, Eq. 27): independent Gaussians with
 *    per-joint standard deviation sigma_j, drawn from Philox4x32-10 (Salmon
 *    et al., SC'11) with key = (seed lo, seed hi) and counter
 *    (m, k, b, iter); block b = 0 gives joints 0-3, b = 1 joints 4-7.
 *    Words map to uniforms u = ((x >> 9) + 0.5) 2^-23 (23 random bits; the
 *    value is exact in FP32 as well as FP64, so both precisions draw the
 *    same uniform) and pairs of uniforms to normals by Box-Muller.
 *  - Dynamics (Eq. 7 with u = joint acceleration): semi-implicit Euler,
 *    qd_{k+1} = qd_k + dt u_k, q_{k+1} = q_k + dt qd_{k+1}, qdd_k = u_k.
 *    The process noise of Eq. 7 is read as the sampling perturbation.
 *  - Forward kinematics (Eq. 6): modified (Craig) DH,
 *    T_i = T_{i-1} RotX(alpha_{i-1}) TransX(a_{i-1}) RotZ(q_i) TransZ(d_i),
 *    and the end effector is the flange, T_n TransZ(flange_d).
 *  - phi in the collision cost (Eq. 17) is the unsigned distance field,
 *    sampled by trilinear interpolation between voxel centres, clamped to
 *    the grid (edge replication outside).
 *  - Q_k and Q_H (Eqs. 16, 25) are diagonal.
 */
#include "smpc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ Philox */
/* Philox4x32 round and key schedule as defined in Salmon, Moraes, Dror and
 * Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11): two 32x32->64
 * multiplications per round, key bumped by the Weyl constants. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double or_word_to_uniform(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Normals for rollout m, step k: z[0..7] (sampling step of Algorithm 1, Eq. 27). */
void or_normals(uint64_t seed, uint32_t iter, uint32_t m, uint32_t k, double z[8])
{
    const uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    for (uint32_t b = 0; b < 2; ++b) {
        const uint32_t ctr[4] = { m, k, b, iter };
        uint32_t w[4];
        or_philox4x32_10(ctr, key, w);
        for (int p = 0; p < 2; ++p) {
            double u0 = or_word_to_uniform(w[2 * p]);
            double u1 = or_word_to_uniform(w[2 * p + 1]);
            double r = sqrt(-2.0 * log(u0));
            z[4 * b + 2 * p]     = r * cos(2.0 * M_PI * u1);
            z[4 * b + 2 * p + 1] = r * sin(2.0 * M_PI * u1);
        }
    }
}

/* ------------------------------------------------------------ kinematics */
static void mat4_identity(double M[4][4])
{
    memset(M, 0, 16 * sizeof(double));
    M[0][0] = M[1][1] = M[2][2] = M[3][3] = 1.0;
}

static void mat4_mul(const double A[4][4], const double B[4][4], double C[4][4])
{
    double tmp[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int l = 0; l < 4; ++l) s += A[i][l] * B[l][j];
            tmp[i][j] = s;
        }
    memcpy(C, tmp, sizeof(tmp));
}

static void rot_x(double a, double M[4][4])
{
    mat4_identity(M);
    M[1][1] = cos(a); M[1][2] = -sin(a);
    M[2][1] = sin(a); M[2][2] = cos(a);
}

static void rot_z(double a, double M[4][4])
{
    mat4_identity(M);
    M[0][0] = cos(a); M[0][1] = -sin(a);
    M[1][0] = sin(a); M[1][1] = cos(a);
}

static void trans(double x, double y, double z, double M[4][4])
{
    mat4_identity(M);
    M[0][3] = x; M[1][3] = y; M[2][3] = z;
}

/* Link poses T^0..T^n and the flange T^{n+1} (Eq. 6, Sec. IV-A). */
void or_fk(const or_robot *rb, const double *q, double T[][4][4])
{
    const int n = rb->n_joints;
    mat4_identity(T[0]);
    for (int j = 0; j < n; ++j) {
        double A[4][4], B[4][4];
        rot_x(rb->alpha[j], A);
        trans(rb->a[j], 0.0, 0.0, B);   mat4_mul(A, B, A);
        rot_z(q[j] + rb->theta_offset[j], B); mat4_mul(A, B, A);
        trans(0.0, 0.0, rb->d[j], B);   mat4_mul(A, B, A);
        mat4_mul(T[j], A, T[j + 1]);
    }
    double F[4][4];
    trans(0.0, 0.0, rb->flange_d, F);
    mat4_mul(T[n], F, T[n + 1]);
}

/* p_i = R^{link(i)} o_i + t^{link(i)} (sphere model, Sec. IV-B-2). */
void or_sphere_centres(const or_robot *rb, const double T[][4][4], double p[][3])
{
    for (int s = 0; s < rb->n_spheres; ++s) {
        const int L = rb->sphere_link[s];
        for (int r = 0; r < 3; ++r) {
            p[s][r] = T[L][r][3];
            for (int c = 0; c < 3; ++c) p[s][r] += T[L][r][c] * rb->sphere_offset[s][c];
        }
    }
}

/* ------------------------------------------------------------- distance */
static double grid_at(const or_grid *g, int i, int j, int l)
{
    return (double)g->phi[((size_t)l * g->ny + j) * g->nx + i];
}

static void cell_coord(double p, double origin, double res, int n, int *i0, double *f)
{
    double x = (p - origin) / res - 0.5;
    if (x < 0.0) x = 0.0;
    if (x > (double)(n - 1)) x = (double)(n - 1);
    int i = (int)floor(x);
    if (i > n - 2) i = n - 2;
    *i0 = i;
    *f = x - (double)i;
}

/* phi(p): trilinear interpolation of the voxel-centre samples (Eq. 17). */
double or_phi(const or_grid *g, const double p[3])
{
    int i, j, l;
    double fx, fy, fz;
    cell_coord(p[0], g->origin[0], g->res, g->nx, &i, &fx);
    cell_coord(p[1], g->origin[1], g->res, g->ny, &j, &fy);
    cell_coord(p[2], g->origin[2], g->res, g->nz, &l, &fz);
    double c00 = grid_at(g, i, j, l)         * (1 - fx) + grid_at(g, i + 1, j, l)         * fx;
    double c10 = grid_at(g, i, j + 1, l)     * (1 - fx) + grid_at(g, i + 1, j + 1, l)     * fx;
    double c01 = grid_at(g, i, j, l + 1)     * (1 - fx) + grid_at(g, i + 1, j, l + 1)     * fx;
    double c11 = grid_at(g, i, j + 1, l + 1) * (1 - fx) + grid_at(g, i + 1, j + 1, l + 1) * fx;
    double c0 = c00 * (1 - fy) + c10 * fy;
    double c1 = c01 * (1 - fy) + c11 * fy;
    return c0 * (1 - fz) + c1 * fz;
}

/* ---------------------------------------------------------------- SE(3) */
/* omega with R = exp([omega]x), the principal logarithm (Eq. 12). */
static void so3_log(const double R[3][3], double w[3])
{
    double vee[3] = { R[2][1] - R[1][2], R[0][2] - R[2][0], R[1][0] - R[0][1] };
    double s = 0.5 * sqrt(vee[0] * vee[0] + vee[1] * vee[1] + vee[2] * vee[2]);
    double c = 0.5 * (R[0][0] + R[1][1] + R[2][2] - 1.0);
    double th = atan2(s, c);
    if (th < 1e-6) {
        double f = 0.5 + th * th / 12.0;
        for (int i = 0; i < 3; ++i) w[i] = f * vee[i];
    } else if (th < M_PI - 1e-6) {
        double f = th / (2.0 * sin(th));
        for (int i = 0; i < 3; ++i) w[i] = f * vee[i];
    } else {
        /* (R + R^T)/2 = cos(th) I + (1 - cos(th)) a a^T: take the axis from
         * the column with the largest diagonal. */
        double B[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                B[i][j] = (0.5 * (R[i][j] + R[j][i]) - (i == j ? c : 0.0)) / (1.0 - c);
        int im = 0;
        for (int i = 1; i < 3; ++i) if (B[i][i] > B[im][im]) im = i;
        double a[3], an = sqrt(B[im][im]);
        for (int i = 0; i < 3; ++i) a[i] = B[i][im] / an;
        double nrm = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int i = 0; i < 3; ++i) a[i] /= nrm;
        double dot = a[0] * vee[0] + a[1] * vee[1] + a[2] * vee[2];
        int big = 0;
        for (int i = 1; i < 3; ++i) if (fabs(a[i]) > fabs(a[big])) big = i;
        double sgn = (dot != 0.0) ? (dot > 0 ? 1.0 : -1.0) : (a[big] >= 0 ? 1.0 : -1.0);
        for (int i = 0; i < 3; ++i) w[i] = sgn * th * a[i];
    }
}

static double det3(const double M[3][3])
{
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
         - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
         + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* xi = [v; omega] = log(T) (Eqs. 12-15): omega = log R, and v solves
 * t = V(theta) v with V(theta) = I + (1-cos)/th^2 [w]x + (th-sin)/th^3 [w]x^2,
 * solved by Cramer's rule. */
void or_se3_log(const double T[4][4], double xi[6])
{
    double R[3][3], t[3], w[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) R[i][j] = T[i][j];
        t[i] = T[i][3];
    }
    so3_log(R, w);
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double A, B;
    if (th < 1e-3) {
        double t2 = th * th;
        A = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        B = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
    } else {
        A = (1.0 - cos(th)) / (th * th);
        B = (th - sin(th)) / (th * th * th);
    }
    double W[3][3] = { { 0, -w[2], w[1] }, { w[2], 0, -w[0] }, { -w[1], w[0], 0 } };
    double W2[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int l = 0; l < 3; ++l) s += W[i][l] * W[l][j];
            W2[i][j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            V[i][j] = (i == j ? 1.0 : 0.0) + A * W[i][j] + B * W2[i][j];
    double dV = det3(V);
    for (int col = 0; col < 3; ++col) {
        double M[3][3];
        memcpy(M, V, sizeof(M));
        for (int i = 0; i < 3; ++i) M[i][col] = t[i];
        xi[col] = det3(M) / dV;
    }
    xi[3] = w[0]; xi[4] = w[1]; xi[5] = w[2];
}

/* Delta T = T_g^{-1} T_ee (Eq. 11), then xi = log(Delta T). */
void or_pose_error(const double Tg[4][4], const double Tee[4][4], double xi[6])
{
    double D[4][4];
    mat4_identity(D);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int l = 0; l < 3; ++l) s += Tg[l][i] * Tee[l][j];   /* R_g^T R */
            D[i][j] = s;
        }
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += Tg[l][i] * (Tee[l][3] - Tg[l][3]); /* R_g^T (t - t_g) */
        D[i][3] = s;
    }
    or_se3_log(D, xi);
}

/* --------------------------------------------------------------- costs */
static double pose_cost(const double Q[6], const double xi[6])
{
    double s = 0.0;
    for (int i = 0; i < 6; ++i) s += Q[i] * xi[i] * xi[i];
    return 0.5 * s;
}

/* delta_i(x) of Eq. 21 on the tightened box [lo + eps, hi - eps]. */
static double limit_violation(double x, double lo, double hi, double margin_frac)
{
    double e = margin_frac * (hi - lo);
    double up = x - (hi - e), dn = x - (lo + e);
    return (up > 0.0 ? up : 0.0) + (dn < 0.0 ? dn : 0.0);
}

/* Semi-implicit Euler roll-out of Eq. 7: q, qd of size (H+1) x n. */
void or_integrate(int n, int H, double dt, const double *q0, const double *qd0,
                  const double *u, double *q, double *qd)
{
    for (int j = 0; j < n; ++j) { q[j] = q0[j]; qd[j] = qd0[j]; }
    for (int k = 0; k < H; ++k)
        for (int j = 0; j < n; ++j) {
            qd[(k + 1) * n + j] = qd[k * n + j] + dt * u[k * n + j];
            q[(k + 1) * n + j]  = q[k * n + j] + dt * qd[(k + 1) * n + j];
        }
}

/* S^{(m)} of Eq. 28 for one control sequence u [H][n]: running costs
 * (Eqs. 16, 19-20, 22, 23, 24) at k = 0..H-1 plus the terminal cost (Eq. 25)
 * at k = H.  If trace != NULL it receives (H+1) x OR_T_COLS per-step terms
 * (the terminal cost in row H, column OR_T_POSE). */
double or_rollout(const or_robot *rb, const or_grid *g, const or_cost *c,
                  const double *q0, const double *qd0, const double Tg[4][4],
                  const double *u, int H, double dt, double *trace)
{
    const int n = rb->n_joints;
    double *q = (double *)malloc(sizeof(double) * (size_t)(H + 1) * n);
    double *qd = (double *)malloc(sizeof(double) * (size_t)(H + 1) * n);
    or_integrate(n, H, dt, q0, qd0, u, q, qd);

    double T[OR_MAX_J + 2][4][4];
    double p[OR_MAX_S][3];
    double S = 0.0;
    for (int k = 0; k <= H; ++k) {
        const double *qk = q + (size_t)k * n;
        or_fk(rb, qk, T);
        double xi[6];
        or_pose_error(Tg, T[n + 1], xi);
        double term[OR_T_COLS] = { 0 };
        if (k == H) {
            term[OR_T_POSE] = pose_cost(c->QH, xi);
        } else {
            const double *qdk = qd + (size_t)k * n;
            const double *uk = u + (size_t)k * n;
            term[OR_T_POSE] = pose_cost(c->Q, xi);
            or_sphere_centres(rb, T, p);
            for (int s = 0; s < rb->n_spheres; ++s) {
                double d_env = or_phi(g, p[s]) - rb->sphere_radius[s];
                double del = c->d_act - d_env;
                if (del < 0.0) del = 0.0;
                term[OR_T_ENV] += c->w_env * del * del;
            }
            for (int pr = 0; pr < rb->n_pairs; ++pr) {
                int a = rb->pairs[pr][0], b = rb->pairs[pr][1];
                double dx = p[a][0] - p[b][0], dy = p[a][1] - p[b][1], dz = p[a][2] - p[b][2];
                double d_self = sqrt(dx * dx + dy * dy + dz * dz)
                              - (rb->sphere_radius[a] + rb->sphere_radius[b]);
                double del = -d_self;
                if (del < 0.0) del = 0.0;
                term[OR_T_SELF] += c->w_self * del * del;
            }
            for (int j = 0; j < n; ++j) {
                double dq = limit_violation(qk[j], rb->q_min[j], rb->q_max[j], c->margin_frac);
                double dqd = limit_violation(qdk[j], -rb->qd_max[j], rb->qd_max[j], c->margin_frac);
                double dqdd = limit_violation(uk[j], -rb->qdd_max[j], rb->qdd_max[j], c->margin_frac);
                term[OR_T_LIM_Q] += c->w_q * dq * dq;
                term[OR_T_LIM_QD] += c->w_qd * dqd * dqd;
                term[OR_T_LIM_QDD] += c->w_qdd * dqdd * dqdd;
                term[OR_T_SMOOTH] += c->w_s * uk[j] * uk[j];
                double e = qk[j] - c->q_ref[j];
                term[OR_T_NS] += c->w_ns * e * e;
            }
        }
        for (int t = 0; t < OR_T_COLS; ++t) {
            S += term[t];
            if (trace) trace[(size_t)k * OR_T_COLS + t] = term[t];
        }
    }
    free(q);
    free(qd);
    return S;
}

/* ------------------------------------------------------------ Algorithm 1 */
/* One SMPC iteration.  U [H][n] holds the nominal sequence on entry and the
 * update U* of Eq. 30 on return.  costs/weights (length K) may be NULL. */
int or_smpc_iterate(const or_robot *rb, const or_grid *g, const or_cost *c,
                    const double *q0, const double *qd0, const double Tg[4][4],
                    double *U, int K, int H, double dt, double lambda,
                    const double *sigma, uint64_t seed, uint32_t iter_index,
                    double *costs, double *weights, int n_threads)
{
    const int n = rb->n_joints;
    if (K < 1 || H < 1 || n < 1 || n > OR_MAX_J || !(lambda > 0.0)) return -1;
    double *eps = (double *)malloc(sizeof(double) * (size_t)K * H * n);
    double *S = (double *)malloc(sizeof(double) * (size_t)K);
    double *w = (double *)malloc(sizeof(double) * (size_t)K);
    if (!eps || !S || !w) { free(eps); free(S); free(w); return -2; }

#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 8)
#endif
    for (int m = 0; m < K; ++m) {
        double *e = eps + (size_t)m * H * n;
        double *um = (double *)malloc(sizeof(double) * (size_t)H * n);
        for (int k = 0; k < H; ++k) {                       /* sample eps */
            double z[8];
            or_normals(seed, iter_index, (uint32_t)m, (uint32_t)k, z);
            for (int j = 0; j < n; ++j) {
                e[k * n + j] = sigma[j] * z[j];
                um[k * n + j] = U[k * n + j] + e[k * n + j];  /* perturb */
            }
        }
        S[m] = or_rollout(rb, g, c, q0, qd0, Tg, um, H, dt, NULL);  /* roll out, FK, cost */
        free(um);
    }
    (void)n_threads;

    double Smin = S[0];                                      /* minimum cost */
    for (int m = 1; m < K; ++m) if (S[m] < Smin) Smin = S[m];
    double Z = 0.0;                                          /* weights, Eq. 29 */
    for (int m = 0; m < K; ++m) { w[m] = exp(-(S[m] - Smin) / lambda); Z += w[m]; }
    for (int m = 0; m < K; ++m) w[m] /= Z;
    for (int k = 0; k < H; ++k)                              /* update, Eq. 30 */
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int m = 0; m < K; ++m) acc += w[m] * eps[((size_t)m * H + k) * n + j];
            U[k * n + j] += acc;
        }
    if (costs) memcpy(costs, S, sizeof(double) * (size_t)K);
    if (weights) memcpy(weights, w, sizeof(double) * (size_t)K);
    free(eps); free(S); free(w);
    return 0;
}

/* One receding-horizon replan (Sec. IV-C, last paragraph): n_iters SMPC
 * iterations with iter_index = replan_index * n_iters + it, then u0* is
 * executed for one step of the same integrator and the sequence is shifted
 * by one step (last row repeated) as the next warm start.  q, qd are
 * advanced in place; U [H][n] receives the shifted sequence. */
int or_replan(const or_robot *rb, const or_grid *g, const or_cost *c,
              double *q, double *qd, const double Tg[4][4], double *U,
              int K, int H, double dt, double lambda, const double *sigma,
              uint64_t seed, uint32_t replan_index, int n_iters,
              double *u0_out, double *best_cost, int n_threads)
{
    const int n = rb->n_joints;
    double *S = (double *)malloc(sizeof(double) * (size_t)K);
    if (!S) return -2;
    for (int it = 0; it < n_iters; ++it) {
        int rc = or_smpc_iterate(rb, g, c, q, qd, Tg, U, K, H, dt, lambda, sigma, seed,
                                 replan_index * (uint32_t)n_iters + (uint32_t)it, S, NULL,
                                 n_threads);
        if (rc) { free(S); return rc; }
    }
    if (best_cost) {
        double b = S[0];
        for (int m = 1; m < K; ++m) if (S[m] < b) b = S[m];
        *best_cost = b;
    }
    free(S);
    for (int j = 0; j < n; ++j) {
        if (u0_out) u0_out[j] = U[j];
        qd[j] = qd[j] + dt * U[j];
        q[j] = q[j] + dt * qd[j];
    }
    for (int k = 0; k + 1 < H; ++k)
        for (int j = 0; j < n; ++j) U[k * n + j] = U[(k + 1) * n + j];
    return 0;
}

/* ------------------------------------------------------------ brute EDT */
/* Exact squared distance (voxel units) from every voxel to the nearest
 * occupied voxel, by exhaustive search over occupied voxels that have a free
 * 6-neighbour inside the grid (the nearest occupied voxel of a free voxel is
 * always such a voxel).  D = 0 on occupied voxels, -1 everywhere if the grid
 * holds no occupied voxel. */
void or_edt_bruteforce(const uint8_t *occ, int nx, int ny, int nz, int64_t *D)
{
    const size_t N = (size_t)nx * ny * nz;
    int *sx = (int *)malloc(sizeof(int) * N), *sy = (int *)malloc(sizeof(int) * N),
        *sz = (int *)malloc(sizeof(int) * N);
    size_t ns = 0;
    for (int l = 0; l < nz; ++l)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t id = ((size_t)l * ny + j) * nx + i;
                if (!occ[id]) continue;
                static const int nb[6][3] = { {1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1} };
                int surf = 0;
                for (int t = 0; t < 6 && !surf; ++t) {
                    int a = i + nb[t][0], b = j + nb[t][1], e = l + nb[t][2];
                    if (a < 0 || b < 0 || e < 0 || a >= nx || b >= ny || e >= nz) continue;
                    if (!occ[((size_t)e * ny + b) * nx + a]) surf = 1;
                }
                if (surf) { sx[ns] = i; sy[ns] = j; sz[ns] = l; ++ns; }
            }
    int any = 0;
    for (size_t id = 0; id < N; ++id) if (occ[id]) { any = 1; break; }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int l = 0; l < nz; ++l)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t id = ((size_t)l * ny + j) * nx + i;
                if (!any) { D[id] = -1; continue; }
                if (occ[id]) { D[id] = 0; continue; }
                int64_t best = INT64_MAX;
                for (size_t s = 0; s < ns; ++s) {
                    int64_t dx = i - sx[s], dy = j - sy[s], dz = l - sz[s];
                    int64_t d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 < best) best = d2;
                }
                D[id] = best;
            }
    free(sx); free(sy); free(sz);
}

/* Robot-masked occupancy reset (Sec. IV-B-2, Remark 2): every voxel whose
 * centre origin + (i + 1/2, j + 1/2, l + 1/2) res lies within a sphere of the
 * model at configuration q (radius + inflate, closed ball) is set to 0 in
 * occ [nz][ny][nx]; other voxels are left as they are. */
void or_robot_mask(const or_robot *rb, const double *q, int nx, int ny, int nz, double res,
                   const double *origin, double inflate, uint8_t *occ)
{
    double T[OR_MAX_J + 2][4][4];
    double p[OR_MAX_S][3];
    or_fk(rb, q, T);
    or_sphere_centres(rb, T, p);
    for (int l = 0; l < nz; ++l)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const double c[3] = { origin[0] + (i + 0.5) * res, origin[1] + (j + 0.5) * res,
                                      origin[2] + (l + 0.5) * res };
                for (int s = 0; s < rb->n_spheres; ++s) {
                    const double dx = c[0] - p[s][0], dy = c[1] - p[s][1], dz = c[2] - p[s][2];
                    const double r = rb->sphere_radius[s] + inflate;
                    if (dx * dx + dy * dy + dz * dz <= r * r) {
                        occ[((size_t)l * ny + j) * nx + i] = 0;
                        break;
                    }
                }
            }
}

/* Unit quaternion (w, x, y, z) of a rotation matrix (Shepperd's method:
 * the largest of 1 + tr, 1 + 2 R_ii - tr picks the stable formula). */
static void rot_to_quat(const double R[3][3], double q[4])
{
    const double tr = R[0][0] + R[1][1] + R[2][2];
    if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) {
        const double w = 0.5 * sqrt(1.0 + tr);
        q[0] = w;
        q[1] = (R[2][1] - R[1][2]) / (4.0 * w);
        q[2] = (R[0][2] - R[2][0]) / (4.0 * w);
        q[3] = (R[1][0] - R[0][1]) / (4.0 * w);
    } else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) {
        const double x = 0.5 * sqrt(1.0 + 2.0 * R[0][0] - tr);
        q[1] = x;
        q[0] = (R[2][1] - R[1][2]) / (4.0 * x);
        q[2] = (R[0][1] + R[1][0]) / (4.0 * x);
        q[3] = (R[0][2] + R[2][0]) / (4.0 * x);
    } else if (R[1][1] >= R[2][2]) {
        const double y = 0.5 * sqrt(1.0 + 2.0 * R[1][1] - tr);
        q[2] = y;
        q[0] = (R[0][2] - R[2][0]) / (4.0 * y);
        q[1] = (R[0][1] + R[1][0]) / (4.0 * y);
        q[3] = (R[1][2] + R[2][1]) / (4.0 * y);
    } else {
        const double z = 0.5 * sqrt(1.0 + 2.0 * R[2][2] - tr);
        q[3] = z;
        q[0] = (R[1][0] - R[0][1]) / (4.0 * z);
        q[1] = (R[0][2] + R[2][0]) / (4.0 * z);
        q[2] = (R[1][2] + R[2][1]) / (4.0 * z);
    }
}

/* Final pose error of configuration q against the goal Tg (row-major 4x4),
 * as the evaluation defines it (Sec. V-A, pose error metrics):
 * e_pos = |p_g - p|, e_ori = 2 arccos |q_g . q| with unit quaternions. */
void or_pose_metrics(const or_robot *rb, const double *q, const double *Tg, double out[2])
{
    double T[OR_MAX_J + 2][4][4];
    or_fk(rb, q, T);
    const int n = rb->n_joints;
    double dx = T[n + 1][0][3] - Tg[3], dy = T[n + 1][1][3] - Tg[7], dz = T[n + 1][2][3] - Tg[11];
    out[0] = sqrt(dx * dx + dy * dy + dz * dz);
    double Ra[3][3], Rb[3][3], qa[4], qb[4];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { Ra[i][j] = Tg[4 * i + j]; Rb[i][j] = T[n + 1][i][j]; }
    rot_to_quat(Ra, qa);
    rot_to_quat(Rb, qb);
    double na = 0.0, nb = 0.0, d = 0.0;
    for (int k = 0; k < 4; ++k) { na += qa[k] * qa[k]; nb += qb[k] * qb[k]; d += qa[k] * qb[k]; }
    d = fabs(d) / sqrt(na * nb);
    out[1] = 2.0 * acos(d > 1.0 ? 1.0 : d);
}

/* eps[i][k][j] = sigma_j z_j(m0 + i, k) for i < count, k < H, j < n (the
 * sampling step of Algorithm 1 over a range of roll-outs; OpenMP). */
void or_eps_range(uint64_t seed, uint32_t iter, uint32_t m0, int count, int H, int n, const double *sigma,
                  double *eps)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int i = 0; i < count; ++i) {
        double z[8];
        for (int k = 0; k < H; ++k) {
            or_normals(seed, iter, m0 + (uint32_t)i, (uint32_t)k, z);
            for (int j = 0; j < n; ++j) eps[((size_t)i * H + k) * n + j] = sigma[j] * z[j];
        }
    }
}

