/*
 * ms_oracle.c -- plain FP64 CPU definition of the explicit mass-spring step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product path never does.  It shares
 * no code, header or table with the GPU library.
 *
 * What it computes (Cronos paper, section "Method"):
 *   eq. 1-3   m_i a_i = f_i,  f_i = m_i g + f_ext_i + sum_j k_ij (|l_ij| - L_ij) l_ij/|l_ij|,
 *             l_ij = x_j - x_i, integrated as d/dt [x; v] = [v; f/m].
 *   Readings of points the paper leaves open (each listed with its reason in
 *   the design notes):
 *     R1  default scheme = symplectic (semi-implicit) Euler: v' = v + dt f/m,
 *         x' = x + dt v'.  Forward Euler (eq. 4), position Verlet (eq. 5-6)
 *         and classical RK4 (eq. 7-8 with the dt factors restored, R17) are
 *         selectable.
 *     R2  each spring also carries an axial dashpot c ((v_j - v_i).u) u;
 *         optional global velocity damping v' *= (1 - d).
 *     R3  actuated rest length L = L0 (1 + A sin(2 pi f t_n + phi)), t_n = n dt.
 *     R4  ground plane z = 0: penalty normal force k_c max(0, -z) when z < 0
 *         strictly, then Coulomb friction as an impulse clamp on the
 *         tangential velocity: stick if |v_t| <= mu Fn dt / m, else reduce
 *         |v_t| by that amount.
 *     R5  anchored masses keep x, have v = 0, and still pull on neighbours.
 *     R7  a spring of zero length exerts no force.
 *
 * Springs are summed in spring-index order; all state is FP64.  No blocking,
 * fusion or reordering beyond the definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double dt;
    double g[3];
    double k_c;          /* ground penalty stiffness [N/m] */
    double mu;           /* Coulomb friction coefficient */
    double vel_damping;  /* global per-step velocity damping d */
    double freq;         /* actuation frequency [Hz] */
    int32_t contact_on;
    int32_t integrator;  /* 0 symplectic Euler, 1 forward Euler, 2 Verlet, 3 RK4 */
} ora_params;

enum { ORA_OK = 0, ORA_ERR_ARG = 1, ORA_ERR_UNSUPPORTED = 2, ORA_ERR_OOM = 3 };

typedef struct {
    int64_t N, S;
    const double *m;
    const uint8_t *fixed;
    const double *fext;      /* N*3 or NULL */
    const int32_t *ij;       /* S*2 */
    const double *k, *c, *L0;
    const double *A, *phi;   /* S each, or NULL (passive) */
} ora_system;

static const double ORA_PI = 3.14159265358979323846;

/* Spring e at time t for state (x, v): the Hooke term of eq. 2 with the R3
 * rest length plus the R2 dashpot, as a signed magnitude fs along the unit
 * vector u from x_i to x_j (mass i receives +fs u, mass j -fs u).  Returns 0
 * for a spring of zero length, which exerts nothing (R7). */
static int ora_spring(const ora_params *p, const ora_system *s, int64_t e,
                      const double *x, const double *v, double t, double *fs, double u[3])
{
    const int64_t i = s->ij[2 * e], j = s->ij[2 * e + 1];
    double d[3], dv[3];
    for (int a = 0; a < 3; ++a) {
        d[a] = x[3 * j + a] - x[3 * i + a];
        dv[a] = v[3 * j + a] - v[3 * i + a];
    }
    const double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (l == 0.0) return 0;                                       /* R7 */
    for (int a = 0; a < 3; ++a) u[a] = d[a] / l;
    double L = s->L0[e];
    if (s->A) L = s->L0[e] * (1.0 + s->A[e] * sin(2.0 * ORA_PI * p->freq * t + s->phi[e]));
    *fs = s->k[e] * (l - L) + s->c[e] * (dv[0] * u[0] + dv[1] * u[1] + dv[2] * u[2]);
    return 1;
}

/* Gravity and external force of eq. 2 and the R4 penalty normal force on
 * mass i, added to its spring sum; pen[i] records whether it penetrates the
 * ground (z < 0), which the friction clamp needs. */
static void ora_body_force(const ora_params *p, const ora_system *s, int64_t i,
                           const double *x, double *F, uint8_t *pen)
{
    for (int a = 0; a < 3; ++a) {
        F[3 * i + a] += s->m[i] * p->g[a];
        if (s->fext) F[3 * i + a] += s->fext[3 * i + a];
    }
    pen[i] = 0;
    if (p->contact_on && x[3 * i + 2] < 0.0) {
        pen[i] = 1;
        F[3 * i + 2] += -p->k_c * x[3 * i + 2];
    }
}

/* Total force on every mass at time t for state (x, v): the spring terms in
 * spring-index order, then each mass's gravity, external and ground force. */
static void ora_total_force(const ora_params *p, const ora_system *s,
                            const double *x, const double *v, double t,
                            double *F, uint8_t *pen)
{
    const int64_t N = s->N, S = s->S;
    memset(F, 0, sizeof(double) * 3 * (size_t)N);
    for (int64_t e = 0; e < S; ++e) {
        const int64_t i = s->ij[2 * e], j = s->ij[2 * e + 1];
        double fs, u[3];
        if (!ora_spring(p, s, e, x, v, t, &fs, u)) continue;
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] += fs * u[a];
            F[3 * j + a] -= fs * u[a];
        }
    }
    for (int64_t i = 0; i < N; ++i) ora_body_force(p, s, i, x, F, pen);
}

/* R4 Coulomb clamp on the tangential (x, y) part of a velocity. */
static void ora_friction(const ora_params *p, double mass, double z, double *vnew)
{
    const double Fn = -p->k_c * z;
    const double D = p->mu * Fn * p->dt / mass;
    const double vt = sqrt(vnew[0] * vnew[0] + vnew[1] * vnew[1]);
    if (vt <= D) {
        vnew[0] = 0.0; vnew[1] = 0.0;
    } else {
        vnew[0] -= D * vnew[0] / vt;
        vnew[1] -= D * vnew[1] / vt;
    }
}

/* Symplectic Euler (R1) update of mass i from its total force: v' = v + dt f/m,
 * the R4 friction clamp, the R2 global damping, then x' = x + dt v'.  Anchored
 * masses (R5) keep x and have v = 0. */
static void ora_se_update(const ora_params *p, const ora_system *s, int64_t i, double *x, double *v,
                          const double *F, const uint8_t *pen)
{
    if (s->fixed[i]) { v[3 * i] = v[3 * i + 1] = v[3 * i + 2] = 0.0; return; }
    double vn[3];
    for (int a = 0; a < 3; ++a) vn[a] = v[3 * i + a] + p->dt * F[3 * i + a] / s->m[i];
    if (pen[i] && p->mu > 0.0) ora_friction(p, s->m[i], x[3 * i + 2], vn);
    for (int a = 0; a < 3; ++a) {
        vn[a] *= (1.0 - p->vel_damping);
        x[3 * i + a] += p->dt * vn[a];
        v[3 * i + a] = vn[a];
    }
}

static int ora_symplectic_euler(const ora_params *p, const ora_system *s, double *x, double *v,
                                int64_t n0, int64_t nsteps, double *F, uint8_t *pen)
{
    for (int64_t n = n0; n < n0 + nsteps; ++n) {
        const double t = (double)n * p->dt;
        ora_total_force(p, s, x, v, t, F, pen);
        for (int64_t i = 0; i < s->N; ++i) ora_se_update(p, s, i, x, v, F, pen);
    }
    return ORA_OK;
}

/* eq. 4: both updates use the state at t_n. */
static int ora_forward_euler(const ora_params *p, const ora_system *s, double *x, double *v,
                             int64_t n0, int64_t nsteps, double *F, uint8_t *pen)
{
    for (int64_t n = n0; n < n0 + nsteps; ++n) {
        const double t = (double)n * p->dt;
        ora_total_force(p, s, x, v, t, F, pen);
        for (int64_t i = 0; i < s->N; ++i) {
            if (s->fixed[i]) { v[3 * i] = v[3 * i + 1] = v[3 * i + 2] = 0.0; continue; }
            double vn[3];
            for (int a = 0; a < 3; ++a) vn[a] = v[3 * i + a] + p->dt * F[3 * i + a] / s->m[i];
            if (pen[i] && p->mu > 0.0) ora_friction(p, s->m[i], x[3 * i + 2], vn);
            for (int a = 0; a < 3; ++a) {
                vn[a] *= (1.0 - p->vel_damping);
                x[3 * i + a] += p->dt * v[3 * i + a];
                v[3 * i + a] = vn[a];
            }
        }
    }
    return ORA_OK;
}

/* eq. 5-6, position form.  The velocity that the dashpots see at step n is
 * the backward difference (x_n - x_{n-1}) / dt (the given v_0 at n = n0). */
static int ora_verlet(const ora_params *p, const ora_system *s, double *x, double *v,
                      int64_t n0, int64_t nsteps, double *F, uint8_t *pen)
{
    const int64_t N = s->N;
    double *xprev = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    if (!xprev) return ORA_ERR_OOM;
    for (int64_t n = n0; n < n0 + nsteps; ++n) {
        const double t = (double)n * p->dt;
        ora_total_force(p, s, x, v, t, F, pen);
        for (int64_t i = 0; i < N; ++i) {
            for (int a = 0; a < 3; ++a) {
                const double xn = x[3 * i + a];
                double xnext;
                if (s->fixed[i]) xnext = xn;
                else if (n == n0)      /* eq. 5 */
                    xnext = xn + p->dt * v[3 * i + a] + p->dt * p->dt / (2.0 * s->m[i]) * F[3 * i + a];
                else                   /* eq. 6 */
                    xnext = 2.0 * xn - xprev[3 * i + a] + p->dt * p->dt / s->m[i] * F[3 * i + a];
                xprev[3 * i + a] = xn;
                x[3 * i + a] = xnext;
                v[3 * i + a] = s->fixed[i] ? 0.0 : (xnext - xn) / p->dt;
            }
        }
    }
    free(xprev);
    return ORA_OK;
}

/* Classical fourth-order Runge-Kutta on eq. 3 (the paper's eq. 7-8 with the
 * dt factors of the stages restored). */
static int ora_rk4(const ora_params *p, const ora_system *s, double *x, double *v,
                   int64_t n0, int64_t nsteps, double *F, uint8_t *pen)
{
    const int64_t N = s->N;
    const size_t nb = sizeof(double) * 3 * (size_t)N;
    double *xs = (double *)malloc(nb), *vs = (double *)malloc(nb);
    double *kx[4], *kv[4];
    int ok = xs && vs;
    for (int q = 0; q < 4; ++q) { kx[q] = (double *)malloc(nb); kv[q] = (double *)malloc(nb); ok = ok && kx[q] && kv[q]; }
    if (!ok) {
        free(xs); free(vs);
        for (int q = 0; q < 4; ++q) { free(kx[q]); free(kv[q]); }
        return ORA_ERR_OOM;
    }
    const double h = p->dt;
    const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    for (int64_t n = n0; n < n0 + nsteps; ++n) {
        const double t = (double)n * h;
        for (int q = 0; q < 4; ++q) {
            for (int64_t e = 0; e < 3 * N; ++e) {
                xs[e] = x[e] + (q ? cst[q] * h * kx[q - 1][e] : 0.0);
                vs[e] = v[e] + (q ? cst[q] * h * kv[q - 1][e] : 0.0);
            }
            ora_total_force(p, s, xs, vs, t + cst[q] * h, F, pen);
            for (int64_t i = 0; i < N; ++i)
                for (int a = 0; a < 3; ++a) {
                    kx[q][3 * i + a] = s->fixed[i] ? 0.0 : vs[3 * i + a];
                    kv[q][3 * i + a] = s->fixed[i] ? 0.0 : F[3 * i + a] / s->m[i];
                }
        }
        for (int64_t i = 0; i < N; ++i)
            for (int a = 0; a < 3; ++a) {
                const int64_t e = 3 * i + a;
                if (s->fixed[i]) { v[e] = 0.0; continue; }
                x[e] += h / 6.0 * (kx[0][e] + 2.0 * kx[1][e] + 2.0 * kx[2][e] + kx[3][e]);
                v[e] += h / 6.0 * (kv[0][e] + 2.0 * kv[1][e] + 2.0 * kv[2][e] + kv[3][e]);
            }
    }
    free(xs); free(vs);
    for (int q = 0; q < 4; ++q) { free(kx[q]); free(kv[q]); }
    return ORA_OK;
}

/* Advance (x, v) in place by nsteps steps, the first at t = n0 * dt. */
int ora_run(const ora_params *p, int64_t N, double *x, double *v, const double *m,
            const uint8_t *fixed, const double *fext, int64_t S, const int32_t *ij,
            const double *k, const double *c, const double *L0, const double *A,
            const double *phi, int64_t n0, int64_t nsteps)
{
    if (!p || N < 0 || S < 0 || nsteps < 0 || (N > 0 && (!x || !v || !m || !fixed)) ||
        (S > 0 && (!ij || !k || !c || !L0)) || ((A == NULL) != (phi == NULL)))
        return ORA_ERR_ARG;
    for (int64_t e = 0; e < S; ++e)
        if (ij[2 * e] < 0 || ij[2 * e] >= N || ij[2 * e + 1] < 0 || ij[2 * e + 1] >= N) return ORA_ERR_ARG;
    if (p->integrator >= 2 && (p->mu > 0.0 || p->vel_damping != 0.0)) return ORA_ERR_UNSUPPORTED;
    ora_system s = {N, S, m, fixed, fext, ij, k, c, L0, A, phi};
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    uint8_t *pen = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    if (!F || !pen) { free(F); free(pen); return ORA_ERR_OOM; }
    int rc;
    switch (p->integrator) {
        case 0: rc = ora_symplectic_euler(p, &s, x, v, n0, nsteps, F, pen); break;
        case 1: rc = ora_forward_euler(p, &s, x, v, n0, nsteps, F, pen); break;
        case 2: rc = ora_verlet(p, &s, x, v, n0, nsteps, F, pen); break;
        case 3: rc = ora_rk4(p, &s, x, v, n0, nsteps, F, pen); break;
        default: rc = ORA_ERR_ARG;
    }
    free(F); free(pen);
    return rc;
}

/* The same symplectic Euler run (integrator 0) on several host threads, for
 * timing the oracle on all cores.  Masses are cut into contiguous blocks, one
 * per thread; each thread walks, in spring-index order, the springs that
 * touch its block and adds their terms to its own masses only, so every
 * mass's force is summed in exactly the serial order and the result is
 * bit-identical to ora_run.  A barrier separates the force pass (which reads
 * every mass at t_n) from the update pass.  *threads_used receives the
 * number of threads that ran (1 without OpenMP). */
int ora_run_threads(const ora_params *p, int64_t N, double *x, double *v, const double *m,
                    const uint8_t *fixed, const double *fext, int64_t S, const int32_t *ij,
                    const double *k, const double *c, const double *L0, const double *A,
                    const double *phi, int64_t n0, int64_t nsteps, int32_t nthreads,
                    int32_t *threads_used)
{
    if (!p || N < 1 || S < 0 || nsteps < 0 || nthreads < 1 || !x || !v || !m || !fixed ||
        (S > 0 && (!ij || !k || !c || !L0)) || ((A == NULL) != (phi == NULL)))
        return ORA_ERR_ARG;
    if (p->integrator != 0) return ORA_ERR_UNSUPPORTED;
    for (int64_t e = 0; e < S; ++e)
        if (ij[2 * e] < 0 || ij[2 * e] >= N || ij[2 * e + 1] < 0 || ij[2 * e + 1] >= N) return ORA_ERR_ARG;
#ifndef _OPENMP
    nthreads = 1;
#endif
    if ((int64_t)nthreads > N) nthreads = (int32_t)N;
    ora_system s = {N, S, m, fixed, fext, ij, k, c, L0, A, phi};
    const int64_t T = nthreads;
    /* springs touching each block, in index order (a spring is listed by both
     * blocks when its endpoints lie in different ones) */
    int64_t *cnt = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    uint8_t *pen = (uint8_t *)malloc((size_t)N);
    if (!cnt || !F || !pen) { free(cnt); free(F); free(pen); return ORA_ERR_OOM; }
#define ORA_BLOCK(i) ((int64_t)(((i) * T) / N))
    for (int64_t e = 0; e < S; ++e) {
        const int64_t bi = ORA_BLOCK((int64_t)ij[2 * e]), bj = ORA_BLOCK((int64_t)ij[2 * e + 1]);
        cnt[bi + 1]++;
        if (bj != bi) cnt[bj + 1]++;
    }
    for (int64_t b = 0; b < T; ++b) cnt[b + 1] += cnt[b];
    int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt[T] > 0 ? cnt[T] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)T);
    if (!list || !fill) { free(cnt); free(F); free(pen); free(list); free(fill); return ORA_ERR_OOM; }
    for (int64_t b = 0; b < T; ++b) fill[b] = cnt[b];
    for (int64_t e = 0; e < S; ++e) {
        const int64_t bi = ORA_BLOCK((int64_t)ij[2 * e]), bj = ORA_BLOCK((int64_t)ij[2 * e + 1]);
        list[fill[bi]++] = e;
        if (bj != bi) list[fill[bj]++] = e;
    }
    int32_t used = 1;
#pragma omp parallel num_threads(nthreads)
    {
        int64_t b = 0;
#ifdef _OPENMP
        b = omp_get_thread_num();
#pragma omp single
        used = (int32_t)omp_get_num_threads();
#endif
        /* block b holds the masses i with floor(i T / N) == b */
        const int64_t lo = (b * N + T - 1) / T, hi = ((b + 1) * N + T - 1) / T;
        for (int64_t n = n0; n < n0 + nsteps; ++n) {
            const double t = (double)n * p->dt;
            memset(F + 3 * lo, 0, sizeof(double) * 3 * (size_t)(hi - lo));
            for (int64_t q = cnt[b]; q < cnt[b + 1]; ++q) {
                const int64_t e = list[q];
                const int64_t i = ij[2 * e], j = ij[2 * e + 1];
                double fs, u[3];
                if (!ora_spring(p, &s, e, x, v, t, &fs, u)) continue;
                if (i >= lo && i < hi)
                    for (int a = 0; a < 3; ++a) F[3 * i + a] += fs * u[a];
                if (j >= lo && j < hi)
                    for (int a = 0; a < 3; ++a) F[3 * j + a] -= fs * u[a];
            }
            for (int64_t i = lo; i < hi; ++i) ora_body_force(p, &s, i, x, F, pen);
#pragma omp barrier
            for (int64_t i = lo; i < hi; ++i) ora_se_update(p, &s, i, x, v, F, pen);
#pragma omp barrier
        }
    }
#undef ORA_BLOCK
    if (threads_used) *threads_used = used;
    free(cnt); free(F); free(pen); free(list); free(fill);
    return ORA_OK;
}
