/*
 * FP64 CPU oracle for the direct-summation Hermite hot path.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference the CUDA
 * path is checked against. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never links,
 * calls or falls back to it, and it shares no code with the CUDA sources.
 *
 * What it computes (paper: Portegies Zwart & Bedorf, "Computational
 * Gravitational Dynamics with Modern Numerical Accelerators"):
 *   - the force that a j-set exerts on an i-set, by direct summation over
 *     every (i, j) pair (Sect. III.A: i particles receive, j particles exert,
 *     the two sets may coincide or be disjoint; cost N_i * N_j);
 *   - the pair interaction is Newton's softened gravity (Sect. II), with the
 *     acceleration, its time derivative (the jerk) and the potential that a
 *     4th-order Hermite integrator needs (Sect. II: >= 4th-order integrators
 *     with individual steps for direct codes; Sect. VI: ph4, a 4th-order
 *     Hermite predictor-corrector);
 *   - the prediction of the j particles to the current time (Sect. III.A,
 *     the optional prediction step on the j particles);
 *   - the Hermite corrector and the individual block time steps, where only
 *     the particles that are due at time t are advanced (Sect. III and
 *     III.A: individual/block time steps, N_i << N_j).
 * The paper prints none of these formulas; they are the textbook forms it
 * names (Makino & Aarseth 1992 Hermite scheme, Aarseth's step criterion),
 * written out here plainly. Readings of the paper are listed in the design
 * notes at the repository root.
 *
 * Arithmetic: IEEE binary64, round to nearest, compiled without FMA
 * contraction (-ffp-contract=off) and without fast-math, so x86 and Arm hosts
 * give the same bits. Force sums are plain j-ascending loops accumulated with
 * Neumaier's compensated summation, so that the oracle's own rounding error
 * (~1e-16 relative) is far below every tolerance it is used to check.
 *
 * Layout: positions, velocities, accelerations and jerks are row-major
 * (n, 3) arrays of doubles; masses, potentials, times and steps are length-n
 * arrays.
 *
 * Parity pins (tests/test_oracle_*.py): closed-form two-body values, exact
 * symmetric configurations, Newton's third law (sum m a = sum m jerk = 0),
 * finite-difference checks that acc = -grad(pot) and jerk = d(acc)/dt,
 * brute force in 50-digit arithmetic on tiny N, Kepler's equation and the
 * softened circular orbit for the integrator, 4th-order convergence and
 * energy conservation.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- compensated (Neumaier) summation ---------------------------------- */

typedef struct {
    double s; /* running sum */
    double c; /* accumulated rounding error */
} ksum;

static void ks_add(ksum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x))
        k->c += (k->s - t) + x;
    else
        k->c += (x - t) + k->s;
    k->s = t;
}

static double ks_val(const ksum *k) { return k->s + k->c; }

/* ---- pair interaction (Sect. II: Newtonian gravity, softened) ----------- */

/*
 * Contribution of particle j (mass mj, position xj, velocity vj) to particle
 * i (position xi, velocity vi). With r = xj - xi, v = vj - vi and
 * s2 = |r|^2 + eps2:
 *   acc  = mj r / s2^(3/2)
 *   jerk = mj [ v / s2^(3/2) - 3 (r.v) r / s2^(5/2) ]     (d acc / dt)
 *   pot  = -mj / s2^(1/2)
 */
static void pair_terms(double mj, const double *xj, const double *vj,
                       const double *xi, const double *vi, double eps2,
                       double acc[3], double jerk[3], double *pot)
{
    double r[3], v[3];
    for (int c = 0; c < 3; c++) {
        r[c] = xj[c] - xi[c];
        v[c] = vj[c] - vi[c];
    }
    double s2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2;
    double s = sqrt(s2);
    double inv_s3 = 1.0 / (s2 * s);
    double rv = r[0] * v[0] + r[1] * v[1] + r[2] * v[2];
    for (int c = 0; c < 3; c++) {
        acc[c] = mj * r[c] * inv_s3;
        jerk[c] = mj * (v[c] * inv_s3 - 3.0 * rv * r[c] * inv_s3 / s2);
    }
    *pot = -mj / s;
}

/* Sum over all j of the pair terms on one i-particle; j == skip is left out
 * (skip < 0 means none is left out). */
static void sum_over_j(int nj, const double *m, const double *pos,
                       const double *vel, const double *xi, const double *vi,
                       double eps2, int skip, double acc[3], double jerk[3],
                       double *pot)
{
    ksum ka[3] = {{0, 0}, {0, 0}, {0, 0}};
    ksum kj[3] = {{0, 0}, {0, 0}, {0, 0}};
    ksum kp = {0, 0};
    for (int j = 0; j < nj; j++) {
        if (j == skip)
            continue;
        double a[3], jk[3], p;
        pair_terms(m[j], pos + 3 * (size_t)j, vel + 3 * (size_t)j, xi, vi,
                   eps2, a, jk, &p);
        for (int c = 0; c < 3; c++) {
            ks_add(&ka[c], a[c]);
            ks_add(&kj[c], jk[c]);
        }
        ks_add(&kp, p);
    }
    for (int c = 0; c < 3; c++) {
        acc[c] = ks_val(&ka[c]);
        jerk[c] = ks_val(&kj[c]);
    }
    *pot = ks_val(&kp);
}

/*
 * Force on i-particles that are members of the j-set (Sect. III.A, same-set
 * case): i = idx[k] (idx == NULL means i = k for k < ni), summing over every
 * j != i. Outputs are indexed by k.
 */
void orc_force_idx(int nj, const double *m, const double *pos,
                   const double *vel, double eps2, int ni, const int *idx,
                   double *acc, double *jerk, double *pot)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < ni; k++) {
        int i = idx ? idx[k] : k;
        sum_over_j(nj, m, pos, vel, pos + 3 * (size_t)i, vel + 3 * (size_t)i,
                   eps2, i, acc + 3 * (size_t)k, jerk + 3 * (size_t)k,
                   pot + k);
    }
}

/*
 * Force on an external i-set, disjoint from the j-set (Sect. III.A,
 * different-set case): no pair is left out.
 */
void orc_force_ext(int nj, const double *m, const double *pos,
                   const double *vel, double eps2, int ni, const double *ipos,
                   const double *ivel, double *acc, double *jerk, double *pot)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < ni; k++)
        sum_over_j(nj, m, pos, vel, ipos + 3 * (size_t)k,
                   ivel + 3 * (size_t)k, eps2, -1, acc + 3 * (size_t)k,
                   jerk + 3 * (size_t)k, pot + k);
}

/* ---- predictor (Sect. III.A: prediction of the j particles) ------------- */

/*
 * Taylor prediction of every particle from its own time tj[i] to time t:
 *   xp = x + v d + a d^2/2 + jerk d^3/6,   vp = v + a d + jerk d^2/2,
 * with d = t - tj[i].
 */
void orc_predict(int n, double t, const double *tj, const double *pos,
                 const double *vel, const double *acc, const double *jerk,
                 double *pos_p, double *vel_p)
{
    for (int i = 0; i < n; i++) {
        double d = t - tj[i];
        for (int c = 0; c < 3; c++) {
            size_t q = 3 * (size_t)i + c;
            pos_p[q] = pos[q] + vel[q] * d + acc[q] * d * d / 2.0 +
                       jerk[q] * d * d * d / 6.0;
            vel_p[q] = vel[q] + acc[q] * d + jerk[q] * d * d / 2.0;
        }
    }
}

/* ---- corrector (4th-order Hermite, Sect. II and VI) --------------------- */

/*
 * Hermite corrector for one particle over a step of length dt, from the
 * predicted state (xp, vp), the start-of-step acc/jerk (a0, j0) and the
 * end-of-step acc/jerk (a1, j1). The 2nd and 3rd derivatives of the
 * acceleration at the start of the step follow from the cubic Hermite
 * interpolant through (a0, j0) and (a1, j1):
 *   a2 = (-6 (a0 - a1) - dt (4 j0 + 2 j1)) / dt^2
 *   a3 = (12 (a0 - a1) + 6 dt (j0 + j1)) / dt^3
 *   x1 = xp + a2 dt^4/24 + a3 dt^5/120,   v1 = vp + a2 dt^3/6 + a3 dt^4/24.
 * Returns a2 and a3 moved to the end of the step (a2 + dt a3, a3), which the
 * step criterion uses.
 */
void orc_correct_one(double dt, const double xp[3], const double vp[3],
                     const double a0[3], const double j0[3],
                     const double a1[3], const double j1[3], double x1[3],
                     double v1[3], double a2_end[3], double a3_end[3])
{
    for (int c = 0; c < 3; c++) {
        double a2 = (-6.0 * (a0[c] - a1[c]) - dt * (4.0 * j0[c] + 2.0 * j1[c])) /
                    (dt * dt);
        double a3 = (12.0 * (a0[c] - a1[c]) + 6.0 * dt * (j0[c] + j1[c])) /
                    (dt * dt * dt);
        x1[c] = xp[c] + a2 * dt * dt * dt * dt / 24.0 +
                a3 * dt * dt * dt * dt * dt / 120.0;
        v1[c] = vp[c] + a2 * dt * dt * dt / 6.0 + a3 * dt * dt * dt * dt / 24.0;
        a2_end[c] = a2 + dt * a3;
        a3_end[c] = a3;
    }
}

/* ---- time steps (Sect. III, III.A: individual and block steps) ---------- */

static double norm3(const double *u)
{
    return sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

/*
 * Aarseth's step criterion:
 *   dt = sqrt( eta (|a| |a2| + |j|^2) / (|j| |a3| + |a2|^2) ).
 * A zero denominator (no higher derivatives, e.g. an isolated particle)
 * gives +inf, which the quantizer turns into dt_max.
 */
double orc_aarseth_dt(const double a[3], const double j[3], const double a2[3],
                      const double a3[3], double eta)
{
    double na = norm3(a), nj = norm3(j), n2 = norm3(a2), n3 = norm3(a3);
    double num = na * n2 + nj * nj;
    double den = nj * n3 + n2 * n2;
    if (den == 0.0)
        return INFINITY;
    return sqrt(eta * num / den);
}

/* Initial step without higher derivatives: dt0 = eta_s |a| / |j|. */
double orc_initial_dt(const double a[3], const double j[3], double eta_s)
{
    double nj = norm3(j);
    if (nj == 0.0)
        return INFINITY;
    return eta_s * norm3(a) / nj;
}

/*
 * Block quantization of a raw step into a power of two:
 *   - the largest power of two <= dt_raw (dt_max when dt_raw is +inf);
 *   - at most twice the previous step (dt_old > 0), i.e. growth by one level;
 *   - clamped to [dt_min, dt_max];
 *   - halved until it divides the particle's new time t_new, so block times
 *     stay commensurate (exact in binary64 for dyadic times).
 */
double orc_quantize(double dt_raw, double dt_old, double t_new, double dt_min,
                    double dt_max)
{
    double d;
    if (!(dt_raw < dt_max)) {
        d = dt_max;
    } else {
        int e;
        frexp(dt_raw, &e); /* dt_raw = f 2^e, f in [0.5, 1) */
        d = ldexp(1.0, e - 1);
    }
    if (dt_old > 0.0 && d > 2.0 * dt_old)
        d = 2.0 * dt_old;
    if (d > dt_max)
        d = dt_max;
    if (d < dt_min)
        d = dt_min;
    while (d > dt_min && fmod(t_new, d) != 0.0)
        d = d / 2.0;
    return d;
}

/* ---- integrator state ---------------------------------------------------- */

/*
 * Full state of a system: mass, position, velocity, acceleration, jerk, own
 * time and own step per particle. The force and correction steps act on the
 * 'active' particles (all of them in shared-step mode).
 */
typedef struct {
    int n;
    double eps2;
    double *m, *pos, *vel, *acc, *jerk, *t, *dt;
} orc_state;

/* Evaluate acc and jerk of all particles at their current (synchronous)
 * positions and assign the initial block step. */
static void initialise(orc_state *s, double eta_s, double dt_min,
                       double dt_max, double dt_shared, double *pot_scratch)
{
    orc_force_idx(s->n, s->m, s->pos, s->vel, s->eps2, s->n, NULL, s->acc,
                  s->jerk, pot_scratch);
    for (int i = 0; i < s->n; i++) {
        if (dt_shared > 0.0) {
            s->dt[i] = dt_shared;
        } else {
            double raw = orc_initial_dt(s->acc + 3 * (size_t)i,
                                        s->jerk + 3 * (size_t)i, eta_s);
            s->dt[i] = orc_quantize(raw, 0.0, s->t[i], dt_min, dt_max);
        }
    }
}

/*
 * One block step (shared-step mode is the special case where all particles
 * share one dt and all are due together):
 *   1. t_next = min_i (t_i + dt_i); active = {i : t_i + dt_i == t_next}, in
 *      ascending index order;
 *   2. predict every particle to t_next;
 *   3. evaluate acc/jerk on the active particles from the predicted set;
 *   4. correct the active particles; with n_corr > 1 (the iterated Hermite
 *      corrector, P(EC)^n) the corrected positions and velocities of the
 *      active particles replace their predicted ones in the j-set, their
 *      acc/jerk are evaluated again and the corrector is applied again to the
 *      same predicted values and start-of-step acc/jerk, n_corr times in all;
 *   5. give the active particles a new step from the last evaluation.
 * Returns the number of active particles, sets *t_out = t_next.
 * Scratch: pp, vp (n,3); a1, j1, p1, xs, vs, x1, v1 (n,3) for the active set.
 */
static int block_step(orc_state *s, double eta, double dt_min, double dt_max,
                      double dt_shared, int n_corr, int *active, double *pp,
                      double *vp, double *a1, double *j1, double *p1, double *xs,
                      double *vs, double *x1, double *v1, double *t_out)
{
    int n = s->n;
    double t_next = INFINITY;
    for (int i = 0; i < n; i++)
        if (s->t[i] + s->dt[i] < t_next)
            t_next = s->t[i] + s->dt[i];
    int na = 0;
    for (int i = 0; i < n; i++)
        if (s->t[i] + s->dt[i] == t_next)
            active[na++] = i;

    orc_predict(n, t_next, s->t, s->pos, s->vel, s->acc, s->jerk, pp, vp);
    for (int k = 0; k < na; k++) {
        size_t q = 3 * (size_t)active[k], r = 3 * (size_t)k;
        for (int c = 0; c < 3; c++) {
            xs[r + c] = pp[q + c];
            vs[r + c] = vp[q + c];
        }
    }
    orc_force_idx(n, s->m, pp, vp, s->eps2, na, active, a1, j1, p1);
    for (int it = 1; it < n_corr; it++) {
        for (int k = 0; k < na; k++) {
            int i = active[k];
            size_t q = 3 * (size_t)i, r = 3 * (size_t)k;
            double a2[3], a3[3];
            orc_correct_one(t_next - s->t[i], xs + r, vs + r, s->acc + q,
                            s->jerk + q, a1 + r, j1 + r, x1 + r, v1 + r, a2, a3);
        }
        for (int k = 0; k < na; k++) {
            size_t q = 3 * (size_t)active[k], r = 3 * (size_t)k;
            for (int c = 0; c < 3; c++) {
                pp[q + c] = x1[r + c];
                vp[q + c] = v1[r + c];
            }
        }
        orc_force_idx(n, s->m, pp, vp, s->eps2, na, active, a1, j1, p1);
    }

    for (int k = 0; k < na; k++) {
        int i = active[k];
        size_t q = 3 * (size_t)i, r = 3 * (size_t)k;
        double dt = t_next - s->t[i];
        double xn[3], vn[3], a2[3], a3[3];
        orc_correct_one(dt, xs + r, vs + r, s->acc + q, s->jerk + q, a1 + r,
                        j1 + r, xn, vn, a2, a3);
        double dt_new;
        if (dt_shared > 0.0) {
            dt_new = dt_shared;
        } else {
            double raw = orc_aarseth_dt(a1 + r, j1 + r, a2, a3, eta);
            dt_new = orc_quantize(raw, dt, t_next, dt_min, dt_max);
        }
        for (int c = 0; c < 3; c++) {
            s->pos[q + c] = xn[c];
            s->vel[q + c] = vn[c];
            s->acc[q + c] = a1[r + c];
            s->jerk[q + c] = j1[r + c];
        }
        s->t[i] = t_next;
        s->dt[i] = dt_new;
    }
    *t_out = t_next;
    return na;
}

/*
 * Integrate a system with 4th-order Hermite and block (or shared) steps
 * until every particle reaches t_end, or until max_steps block steps have
 * been taken (max_steps <= 0: no limit).
 *
 * In/out arrays: pos, vel (n,3); acc, jerk (n,3); t, dt (n). When init != 0
 * the acc/jerk are evaluated at the start and dt is assigned (t must then be
 * the same for all particles); otherwise acc, jerk, t and dt are taken as
 * given (a resumed run).
 * dt_shared > 0 selects shared-step mode with that step; n_corr >= 1 is the
 * number of force evaluations and corrections per step (1: PEC).
 * Counters: *n_block_steps, *n_interactions (sum over steps of
 * n_corr * N_active * N, the initial evaluation included when init != 0).
 * Returns 0, or -1 if a scratch allocation failed.
 */
int orc_hermite_run(int n, const double *m, double *pos, double *vel,
                    double *acc, double *jerk, double *t, double *dt,
                    double eps2, double eta, double eta_s, double dt_min,
                    double dt_max, double dt_shared, double t_end,
                    long max_steps, int init, int n_corr, long *n_block_steps,
                    double *n_interactions)
{
    orc_state s = {n, eps2, (double *)m, pos, vel, acc, jerk, t, dt};
    int *active = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double *buf = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * 27);
    if (!active || !buf) {
        free(active);
        free(buf);
        return -1;
    }
    if (n_corr < 1)
        n_corr = 1;
    double *pp = buf, *vp = buf + 3 * (size_t)n, *a1 = buf + 6 * (size_t)n;
    double *j1 = buf + 9 * (size_t)n, *p1 = buf + 12 * (size_t)n;
    double *xs = buf + 15 * (size_t)n, *vs = buf + 18 * (size_t)n;
    double *x1 = buf + 21 * (size_t)n, *v1 = buf + 24 * (size_t)n;
    long steps = 0;
    double inter = 0.0;
    if (init && n > 0) {
        initialise(&s, eta_s, dt_min, dt_max, dt_shared, p1);
        inter += (double)n * (double)n;
    }
    while (n > 0 && (max_steps <= 0 || steps < max_steps)) {
        double t_next = INFINITY;
        for (int i = 0; i < n; i++)
            if (t[i] + dt[i] < t_next)
                t_next = t[i] + dt[i];
        if (t_next > t_end)
            break;
        double tn;
        int na = block_step(&s, eta, dt_min, dt_max, dt_shared, n_corr, active,
                            pp, vp, a1, j1, p1, xs, vs, x1, v1, &tn);
        inter += (double)n_corr * (double)na * (double)n;
        steps++;
    }
    *n_block_steps = steps;
    *n_interactions = inter;
    free(active);
    free(buf);
    return 0;
}

/* ---- energy diagnostic -------------------------------------------------- */

/*
 * Kinetic and softened potential energy of a synchronised system:
 *   K = sum_i m_i |v_i|^2 / 2,   W = -sum_{i<j} m_i m_j / sqrt(r_ij^2 + eps2),
 * the potential written as the sum over distinct pairs (not through the
 * per-particle potential), so it also cross-checks the force routine's pot.
 */
void orc_energy(int n, const double *m, const double *pos, const double *vel,
                double eps2, double *kin, double *wpot)
{
    ksum kk = {0, 0}, kw = {0, 0};
    for (int i = 0; i < n; i++) {
        const double *v = vel + 3 * (size_t)i;
        ks_add(&kk, 0.5 * m[i] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    }
    double *rowsum = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < n; i++) {
        ksum kr = {0, 0};
        for (int j = i + 1; j < n; j++) {
            double r2 = eps2;
            for (int c = 0; c < 3; c++) {
                double d = pos[3 * (size_t)j + c] - pos[3 * (size_t)i + c];
                r2 += d * d;
            }
            ks_add(&kr, -m[i] * m[j] / sqrt(r2));
        }
        rowsum[i] = ks_val(&kr);
    }
    for (int i = 0; i < n; i++)
        ks_add(&kw, rowsum[i]);
    free(rowsum);
    *kin = ks_val(&kk);
    *wpot = ks_val(&kw);
}

/* Number of threads the force loops run on. */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- 6th-order Hermite (Sect. II: direct codes pair with >= 4th-order
 * integrators and individual steps; the reference cited there is Nitadori &
 * Makino's 6th- and 8th-order Hermite schemes) ----------------------------- */

/*
 * Contribution of particle j to particle i with the second time derivative of
 * the acceleration (the snap). With dx = xj - xi, dv = vj - vi, da = aj - ai
 * (the particles' own accelerations) and q2 = |dx|^2 + eps2, differentiate
 * A = mj dx q2^(-3/2) twice along the motion:
 *   alpha = (dx.dv) / q2,   beta = (|dv|^2 + dx.da) / q2 + alpha^2
 *   A = mj dx / q2^(3/2)
 *   J = mj dv / q2^(3/2) - 3 alpha A                        (dA/dt)
 *   S = mj da / q2^(3/2) - 6 alpha J - 3 beta A             (d^2A/dt^2)
 *   pot = -mj / q2^(1/2)
 */
static void pair_terms6(double mj, const double *xj, const double *vj,
                        const double *aj, const double *xi, const double *vi,
                        const double *ai, double eps2, double acc[3],
                        double jerk[3], double snap[3], double *pot)
{
    double dx[3], dv[3], da[3];
    for (int c = 0; c < 3; c++) {
        dx[c] = xj[c] - xi[c];
        dv[c] = vj[c] - vi[c];
        da[c] = aj[c] - ai[c];
    }
    double q2 = eps2 + dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    double q = sqrt(q2);
    double inv_q3 = 1.0 / (q * q2);
    double alpha = (dx[0] * dv[0] + dx[1] * dv[1] + dx[2] * dv[2]) / q2;
    double beta = (dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2] + dx[0] * da[0] +
                   dx[1] * da[1] + dx[2] * da[2]) / q2 + alpha * alpha;
    for (int c = 0; c < 3; c++) {
        acc[c] = mj * dx[c] * inv_q3;
        jerk[c] = mj * dv[c] * inv_q3 - 3.0 * alpha * acc[c];
        snap[c] = mj * da[c] * inv_q3 - 6.0 * alpha * jerk[c] - 3.0 * beta * acc[c];
    }
    *pot = -mj / q;
}

static void sum_over_j6(int nj, const double *m, const double *pos,
                        const double *vel, const double *acc_j,
                        const double *xi, const double *vi, const double *ai,
                        double eps2, int skip, double acc[3], double jerk[3],
                        double snap[3], double *pot)
{
    ksum ka[3] = {{0, 0}, {0, 0}, {0, 0}};
    ksum kj[3] = {{0, 0}, {0, 0}, {0, 0}};
    ksum ks[3] = {{0, 0}, {0, 0}, {0, 0}};
    ksum kp = {0, 0};
    for (int j = 0; j < nj; j++) {
        if (skip == j)
            continue;
        double a[3], jk[3], sn[3], p;
        pair_terms6(m[j], pos + 3 * (size_t)j, vel + 3 * (size_t)j,
                    acc_j + 3 * (size_t)j, xi, vi, ai, eps2, a, jk, sn, &p);
        for (int c = 0; c < 3; c++) {
            ks_add(&ka[c], a[c]);
            ks_add(&kj[c], jk[c]);
            ks_add(&ks[c], sn[c]);
        }
        ks_add(&kp, p);
    }
    for (int c = 0; c < 3; c++) {
        acc[c] = ks_val(&ka[c]);
        jerk[c] = ks_val(&kj[c]);
        snap[c] = ks_val(&ks[c]);
    }
    *pot = ks_val(&kp);
}

/*
 * acc, jerk, snap and pot of the members i = idx[k] (idx == NULL: i = k) from
 * every j != i, given each particle's position, velocity and acceleration
 * (acc_j: the accelerations the snap term differentiates along).
 */
void orc_force6_idx(int nj, const double *m, const double *pos,
                    const double *vel, const double *acc_j, double eps2,
                    int ni, const int *idx, double *acc, double *jerk,
                    double *snap, double *pot)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < ni; k++) {
        int i = idx ? idx[k] : k;
        sum_over_j6(nj, m, pos, vel, acc_j, pos + 3 * (size_t)i,
                    vel + 3 * (size_t)i, acc_j + 3 * (size_t)i, eps2, i,
                    acc + 3 * (size_t)k, jerk + 3 * (size_t)k,
                    snap + 3 * (size_t)k, pot + k);
    }
}

/*
 * Taylor prediction to time t through the crackle term, d = t - tj[i]:
 *   xp = x + v d + a d^2/2 + j d^3/6 + s d^4/24 + c d^5/120
 *   vp = v + a d + j d^2/2 + s d^3/6 + c d^4/24
 *   ap = a + j d + s d^2/2 + c d^3/6
 */
void orc_predict6(int n, double t, const double *tj, const double *pos,
                  const double *vel, const double *acc, const double *jerk,
                  const double *snap, const double *crackle, double *pos_p,
                  double *vel_p, double *acc_p)
{
    for (int i = 0; i < n; i++) {
        double d = t - tj[i];
        double d2 = d * d, d3 = d2 * d, d4 = d3 * d, d5 = d4 * d;
        for (int c = 0; c < 3; c++) {
            size_t q = 3 * (size_t)i + c;
            pos_p[q] = pos[q] + vel[q] * d + acc[q] * d2 / 2.0 + jerk[q] * d3 / 6.0 +
                       snap[q] * d4 / 24.0 + crackle[q] * d5 / 120.0;
            vel_p[q] = vel[q] + acc[q] * d + jerk[q] * d2 / 2.0 + snap[q] * d3 / 6.0 +
                       crackle[q] * d4 / 24.0;
            acc_p[q] = acc[q] + jerk[q] * d + snap[q] * d2 / 2.0 + crackle[q] * d3 / 6.0;
        }
    }
}

/*
 * 6th-order Hermite corrector of one particle over a step dt, from the
 * start-of-step x0, v0, a0, j0, s0 and the end-of-step a1, j1, s1 (evaluated
 * at the predicted state). The two-point Hermite quadrature that is exact
 * when the acceleration is a polynomial of degree <= 5 in time:
 *   v1 = v0 + dt/2 (a0 + a1) - dt^2/10 (j1 - j0) + dt^3/120 (s0 + s1)
 *   x1 = x0 + dt/2 (v0 + v1) - dt^2/10 (a1 - a0) + dt^3/120 (j0 + j1)
 * The 3rd, 4th and 5th derivatives of the acceleration at the end of the
 * step (for the step criterion and the next prediction) come from that
 * quintic. Expanding it about the mid-point with T = dt/2, c_k its k-th
 * derivative there, and the half sums / half differences
 *   Am = (a1 - a0)/2, Jp = (j1 + j0)/2, Jm = (j1 - j0)/2,
 *   Sp = (s1 + s0)/2, Sm = (s1 - s0)/2,
 * the odd and even parts give
 *   c5 = (45 Am - 45 T Jp + 15 T^2 Sm) / T^5
 *   c3 = (15 (T Jp - Am) - 3 T^2 Sm) / (2 T^3)
 *   c4 = 3 (T Sp - Jm) / T^3
 * and at t1 = mid + T: a3 = c3 + c4 T + c5 T^2/2, a4 = c4 + c5 T, a5 = c5.
 * The k-th derivative carries the force's rounding error divided by T^k. The
 * block steps' default criterion takes a, jerk, snap (evaluated) and the
 * crackle a3 only (Aarseth's form, orc_aarseth_dt with a2 = snap, a3 =
 * crackle); the published order-6 criterion on a3, a4 and a5
 * (orc_aarseth6_dt) is the alternative. With forces rounded at ~1e-7 of |a|
 * (FP32 pair arithmetic), a4 and a5 are mostly noise at small T and that
 * criterion drives the steps down to dt_min (shown with perturb_forces).
 */
void orc_correct6_one(double dt, const double x0[3], const double v0[3],
                      const double a0[3], const double j0[3],
                      const double s0[3], const double a1[3],
                      const double j1[3], const double s1[3], double x1[3],
                      double v1[3], double a3_end[3], double a4_end[3],
                      double a5_end[3])
{
    double T = dt / 2.0;
    for (int c = 0; c < 3; c++) {
        v1[c] = v0[c] + dt / 2.0 * (a0[c] + a1[c]) - dt * dt / 10.0 * (j1[c] - j0[c]) +
                dt * dt * dt / 120.0 * (s0[c] + s1[c]);
        x1[c] = x0[c] + dt / 2.0 * (v0[c] + v1[c]) - dt * dt / 10.0 * (a1[c] - a0[c]) +
                dt * dt * dt / 120.0 * (j0[c] + j1[c]);
        double Am = (a1[c] - a0[c]) / 2.0;
        double Jp = (j1[c] + j0[c]) / 2.0, Jm = (j1[c] - j0[c]) / 2.0;
        double Sp = (s1[c] + s0[c]) / 2.0, Sm = (s1[c] - s0[c]) / 2.0;
        double c5 = (45.0 * Am - 45.0 * T * Jp + 15.0 * T * T * Sm) / (T * T * T * T * T);
        double c3 = (15.0 * (T * Jp - Am) - 3.0 * T * T * Sm) / (2.0 * T * T * T);
        double c4 = 3.0 * (T * Sp - Jm) / (T * T * T);
        a3_end[c] = c3 + c4 * T + c5 * T * T / 2.0;
        a4_end[c] = c4 + c5 * T;
        a5_end[c] = c5;
    }
}

/*
 * The step criterion that Nitadori & Makino publish for their order-p Hermite
 * schemes (Aarseth's form generalised to higher derivatives), for p = 6:
 *   dt = eta ( (sqrt(|a| |a2|) + |a1|) / (sqrt(|a3| |a5|) + |a4|) )^(1/3),
 * with a1 = jerk, a2 = snap and a3, a4, a5 the end-of-step crackle, pop and
 * 5th derivative from the corrector (orc_correct6_one). A zero denominator
 * gives +inf (dt_max after quantization).
 */
double orc_aarseth6_dt(const double a[3], const double a1[3],
                       const double a2[3], const double a3[3],
                       const double a4[3], const double a5[3], double eta)
{
    double num = sqrt(norm3(a) * norm3(a2)) + norm3(a1);
    double den = sqrt(norm3(a3) * norm3(a5)) + norm3(a4);
    if (den == 0.0)
        return INFINITY;
    return eta * cbrt(num / den);
}

/* Step criteria of the 6th-order block steps (orc_hermite6_run's crit). */
enum { ORC_CRIT_AARSETH_CRACKLE = 0, ORC_CRIT_GENERALISED = 1 };

/*
 * Force noise for the criterion study (orc_hermite6_run's perturb): a value
 * uniform in [-1, 1) that is a pure function of (seed, step, particle, slot),
 * from SplitMix64's output function (Steele, Lea & Flood 2014) applied to the
 * chained keys. It models the rounding of reduced-precision forces; the
 * oracle's own forces are exact to ~1e-16 and take no noise unless asked.
 */
static unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double noise_unit(unsigned long long seed, long step, int i, int slot)
{
    unsigned long long h = splitmix64(seed);
    h = splitmix64(h ^ (unsigned long long)step);
    h = splitmix64(h ^ (((unsigned long long)(unsigned)i << 4) | (unsigned)slot));
    return (double)(h >> 11) * 0x1.0p-52 - 1.0;
}

/* a, jerk, snap of the na active particles each change by perturb times their
 * own magnitude times noise_unit, per component. */
static void perturb_forces(int na, const int *active, long step,
                           unsigned long long seed, double perturb, double *a1,
                           double *j1, double *s1)
{
    for (int k = 0; k < na; k++) {
        size_t r = 3 * (size_t)k;
        double na1 = norm3(a1 + r), nj1 = norm3(j1 + r), ns1 = norm3(s1 + r);
        for (int c = 0; c < 3; c++) {
            a1[r + c] += perturb * na1 * noise_unit(seed, step, active[k], c);
            j1[r + c] += perturb * nj1 * noise_unit(seed, step, active[k], 3 + c);
            s1[r + c] += perturb * ns1 * noise_unit(seed, step, active[k], 6 + c);
        }
    }
}

typedef struct {
    int n;
    double eps2;
    double *m, *pos, *vel, *acc, *jerk, *snap, *crk, *t, *dt;
} orc_state6;

/* acc, jerk and snap of all particles at their common time: a first pass
 * gives acc and jerk (which do not depend on the accelerations), a second
 * pass with those accelerations gives the snap; crackle starts at zero and
 * the initial step is eta_s |a| / |jerk| (quantized). Scratch: 4n doubles. */
static void initialise6(orc_state6 *s, double eta_s, double dt_min,
                        double dt_max, double dt_shared, double *scratch)
{
    int n = s->n;
    double *aj = scratch, *pot = scratch + 3 * (size_t)n;
    memset(aj, 0, sizeof(double) * 3 * (size_t)n);
    orc_force6_idx(n, s->m, s->pos, s->vel, aj, s->eps2, n, NULL, s->acc,
                   s->jerk, s->snap, pot);
    memcpy(aj, s->acc, sizeof(double) * 3 * (size_t)n);
    orc_force6_idx(n, s->m, s->pos, s->vel, aj, s->eps2, n, NULL, s->acc,
                   s->jerk, s->snap, pot);
    memset(s->crk, 0, sizeof(double) * 3 * (size_t)n);
    for (int i = 0; i < n; i++) {
        if (dt_shared > 0.0) {
            s->dt[i] = dt_shared;
        } else {
            double raw = orc_initial_dt(s->acc + 3 * (size_t)i,
                                        s->jerk + 3 * (size_t)i, eta_s);
            s->dt[i] = orc_quantize(raw, 0.0, s->t[i], dt_min, dt_max);
        }
    }
}

/*
 * One block step of the 6th-order scheme (PEC):
 *   1. t_next = min_i (t_i + dt_i); active = {i : t_i + dt_i == t_next};
 *   2. predict every particle's x, v, a to t_next (orc_predict6);
 *   3. evaluate acc, jerk, snap of the active particles from the predicted
 *      positions, velocities and accelerations;
 *   4. correct them (orc_correct6_one) and give each a new step from the
 *      end-of-step a, jerk, snap and crackle (orc_aarseth_dt, quantized; or
 *      with crit = ORC_CRIT_GENERALISED from a .. a5, orc_aarseth6_dt), or
 *      dt_shared.
 * perturb > 0: the evaluated a, jerk, snap first take seeded relative noise.
 * Scratch: pp, vp, ap (n,3); a1, j1, s1 (n,3) and p1 (n) for the active set.
 */
static int block_step6(orc_state6 *s, double eta, double noise, int crit,
                       double perturb, unsigned long long seed, long step,
                       double dt_min, double dt_max, double dt_shared,
                       int *active, double *pp, double *vp, double *ap,
                       double *a1, double *j1, double *s1, double *p1,
                       double *t_out)
{
    int n = s->n;
    double t_next = INFINITY;
    for (int i = 0; i < n; i++)
        t_next = fmin(t_next, s->t[i] + s->dt[i]);
    int na = 0;
    for (int i = 0; i < n; i++) {
        double due = s->t[i] + s->dt[i];
        if (due == t_next)
            active[na++] = i;
    }

    orc_predict6(n, t_next, s->t, s->pos, s->vel, s->acc, s->jerk, s->snap,
                 s->crk, pp, vp, ap);
    orc_force6_idx(n, s->m, pp, vp, ap, s->eps2, na, active, a1, j1, s1, p1);
    if (perturb > 0.0)
        perturb_forces(na, active, step, seed, perturb, a1, j1, s1);
    for (int k = 0; k < na; k++) {
        int i = active[k];
        size_t q = 3 * (size_t)i, r = 3 * (size_t)k;
        double dt = t_next - s->t[i];
        double xn[3], vn[3], a3[3], a4[3], a5[3];
        orc_correct6_one(dt, s->pos + q, s->vel + q, s->acc + q, s->jerk + q,
                         s->snap + q, a1 + r, j1 + r, s1 + r, xn, vn, a3, a4, a5);
        double dt_new;
        if (dt_shared > 0.0) {
            dt_new = dt_shared;
        } else if (crit == ORC_CRIT_GENERALISED) {
            double raw = orc_aarseth6_dt(a1 + r, j1 + r, s1 + r, a3, a4, a5, eta);
            dt_new = orc_quantize(raw, dt, t_next, dt_min, dt_max);
        } else {
            /* Aarseth's criterion with the evaluated snap as a2 and the
             * interpolated crackle as a3 (the 5th and 4th derivatives stay
             * out: see orc_correct6_one). The crackle's magnitude is reduced
             * by its rounding floor 30 noise |a| / T^3 (T = dt/2; the force's
             * relative rounding noise enters a3 through (a1 - a0) / T^3 with
             * coefficients 7.5 + 22.5): a crackle below the floor carries no
             * information and counts as zero. noise = 0: no floor. */
            double T = dt / 2.0;
            double cfl = 30.0 * noise * norm3(a1 + r) / (T * T * T);
            double cn = norm3(a3), ce[3] = {0.0, 0.0, 0.0};
            if (cn > cfl)
                for (int c = 0; c < 3; c++)
                    ce[c] = a3[c] * ((cn - cfl) / cn);
            double raw = orc_aarseth_dt(a1 + r, j1 + r, s1 + r, ce, eta);
            dt_new = orc_quantize(raw, dt, t_next, dt_min, dt_max);
        }
        for (int c = 0; c < 3; c++) {
            s->pos[q + c] = xn[c];
            s->vel[q + c] = vn[c];
            s->acc[q + c] = a1[r + c];
            s->jerk[q + c] = j1[r + c];
            s->snap[q + c] = s1[r + c];
            s->crk[q + c] = a3[c];
        }
        s->t[i] = t_next;
        s->dt[i] = dt_new;
    }
    *t_out = t_next;
    return na;
}

/*
 * Integrate with the 6th-order Hermite scheme and block (or shared) steps
 * until every particle reaches t_end or max_steps block steps were taken
 * (max_steps <= 0: no limit). In/out (n,3) arrays: pos, vel, acc, jerk, snap,
 * crackle; (n) arrays t, dt. init != 0 evaluates acc, jerk, snap at the
 * common start time, zeroes the crackle and assigns the steps; otherwise the
 * given derivatives, times and steps are used (a resumed run).
 * noise >= 0 is the relative rounding noise of the forces for the crackle's
 * floor in the step criterion (block_step6); 0 for exact forces.
 * crit: ORC_CRIT_AARSETH_CRACKLE (Aarseth's form on a, jerk, snap and the
 * crackle above its floor; the default) or ORC_CRIT_GENERALISED (the
 * published order-6 criterion, orc_aarseth6_dt; noise is not used).
 * perturb > 0 adds seeded relative noise of that size to every evaluated
 * a, jerk and snap of the block steps (perturb_forces; for the study of the
 * criteria under reduced-precision forces), 0 leaves the forces exact.
 * Counters as orc_hermite_run (the initial evaluation counts twice: it takes
 * two passes). Returns 0, or -1 if a scratch allocation failed.
 */
int orc_hermite6_run(int n, const double *m, double *pos, double *vel,
                     double *acc, double *jerk, double *snap, double *crackle,
                     double *t, double *dt, double eps2, double eta,
                     double eta_s, double dt_min, double dt_max,
                     double dt_shared, double noise, int crit, double perturb,
                     unsigned long long seed, double t_end, long max_steps,
                     int init, long *n_block_steps, double *n_interactions)
{
    orc_state6 s = {n, eps2, (double *)m, pos, vel, acc, jerk, snap, crackle, t, dt};
    int *active = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double *buf = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * 19);
    if (!active || !buf) {
        free(active);
        free(buf);
        return -1;
    }
    double *pp = buf, *vp = buf + 3 * (size_t)n, *ap = buf + 6 * (size_t)n;
    double *a1 = buf + 9 * (size_t)n, *j1 = buf + 12 * (size_t)n;
    double *s1 = buf + 15 * (size_t)n, *p1 = buf + 18 * (size_t)n;
    long steps = 0;
    double inter = 0.0;
    if (init && n > 0) {
        initialise6(&s, eta_s, dt_min, dt_max, dt_shared, buf);
        inter += 2.0 * (double)n * (double)n;
    }
    while (n > 0 && (max_steps <= 0 || steps < max_steps)) {
        double t_next = INFINITY;
        for (int i = 0; i < n; i++)
            if (t[i] + dt[i] < t_next)
                t_next = t[i] + dt[i];
        if (!(t_next <= t_end)) /* also ends a run whose times became NaN */
            break;
        double tn;
        int na = block_step6(&s, eta, noise, crit, perturb, seed, steps, dt_min,
                             dt_max, dt_shared, active, pp, vp, ap, a1, j1, s1,
                             p1, &tn);
        inter += (double)na * (double)n;
        steps++;
    }
    *n_block_steps = steps;
    *n_interactions = inter;
    free(active);
    free(buf);
    return 0;
}
