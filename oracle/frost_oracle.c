/*
 * Plain FP64 CPU oracle for the HHS-FSI hot path (Rantala, Naab & Springel 2021, "FROST").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU-baseline
 * leg may load this library.  It shares no code, header, table or constant generator with
 * the CUDA path; it is written from the paper's equations and algorithms:
 *
 *   or_acc             Eq. acc-newton (Sec. 2.3), inter-level form Eq. force-newton-inter (Sec. 3.3)
 *   or_grad            Eq. acc-gradient-g / acc-gradient (Sec. 2.3),
 *                      inter-level forms Eqs. force-gradient-inter-1/2 (Sec. 3.3)
 *   or_accel_gradient  a and a~ = a + eps^2 g / 48 for an intra-set or a cross (S x F) pass
 *   or_pair_timescales Eqs. dt-freefall, dt-flyby and their derivatives
 *                      (Eqs. dt-freefall-derivative, dt-flyby-derivative, two-body form)
 *   or_sym_harmonic    harmonic symmetrisation factor, Eq. time-step-factor (Sec. 4.2)
 *   or_sym_arithmetic  arithmetic symmetrisation factor, Eq. time-step-factor (Sec. 4.2)
 *   or_timesteps       tau_i = min_j of the symmetrised pair timescales (Sec. 4.3);
 *                      or_timesteps_ex adds the exact fly-by derivative variant
 *   or_steps_hold      the second-order HOLD integrator (Eq. hhs2), for comparison
 *   or_partition       slow/fast split by the pivot step (Sec. 3.1)
 *   or_kick, or_drift  kick / drift (Sec. 5.3)
 *   or_fsi             Algorithm fsi (Eq. fsi)
 *   or_hhs_fsi         Algorithm hhs-fsi (Eq. time-evolution-operator-hhs-fsi)
 *   or_steps           main loop of Algorithm frost, n top-level steps of size dt
 *   or_energy          E = T + U (Sec. 2.3), total momentum and angular momentum
 *
 * Conventions: positions/velocities are [n][3] row-major doubles, index lists are int32
 * particle indices into the global arrays.  x_ji = x_j - x_i, r_ji = |x_ji|.
 * Plummer softening (Sec. 2.3, last paragraph) replaces r^2 by r^2 + eps_P^2 in the
 * Newtonian and gradient sums (including the r^2 inside the gradient bracket); the
 * time-step criteria use the unsoftened two-body separation.
 *
 * Readings where the paper is silent (all listed in the design notes):
 *  - the i = j term is skipped by index equality; two distinct particles at the same
 *    position with zero softening are an error (OR_ECOINCIDENT);
 *  - for a cross pass the a_j entering a_ji are the sources' accelerations due to the
 *    active set (the inter-level accelerations of Eq. force-newton-inter);
 *  - eps in a~ is the step of the operator holding the 2/3 kick: dt in fsi, tau_pivot in
 *    hhs_fsi;
 *  - d = eta * dt_ij/dt enters the symmetrisation factor; the harmonic factor is evaluated
 *    in two forms algebraically identical to the printed one that are finite at d = 0 and
 *    free of cancellation (see or_sym_harmonic);
 *  - v_ij = 0 gives an infinite fly-by time; a set of one particle has tau = +inf;
 *  - a particle with tau_i == tau_pivot is slow; partitions keep the input order;
 *  - hhs_fsi calls below depth max_depth with a non-empty set fail with OR_EDEPTH.
 *
 * The i-loops may run under OpenMP; every per-particle sum runs serially over the source
 * list in its given order, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_ENONFINITE 4
#define OR_ECOINCIDENT 5
#define OR_EDEPTH 6

/* flag or-ed into the symmetrisation selector: exact fly-by derivative (Eq.
 * dt-flyby-derivative, first line) instead of its two-body approximation */
#define OR_FLYBY_EXACT 4

/* passes with fewer pair evaluations than this run on one thread (a parallel region per
 * few-body pass would cost more than the pass) */
#define OR_PAR_MIN 262144

/* ---- counters (pair evaluations), read by the tests and the CPU baseline ---- */
static int64_t or_count_acc = 0;
static int64_t or_count_grad = 0;
static int64_t or_count_tstep = 0;
static int or_max_depth_seen = 0;

void or_get_counters(int64_t out[4])
{
    out[0] = or_count_acc;
    out[1] = or_count_grad;
    out[2] = or_count_tstep;
    out[3] = or_max_depth_seen;
}

void or_reset_counters(void)
{
    or_count_acc = or_count_grad = or_count_tstep = 0;
    or_max_depth_seen = 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

/*
 * Newtonian acceleration of every active particle i in A due to the sources j in B:
 *   a_i = G sum_{j in B, j != i} m_j x_ji / r_ji^3                 (Eq. acc-newton)
 * With A = S and B = F this is the first line of Eq. force-newton-inter, with A = F and
 * B = S its second line.
 */
int or_acc(const double *m, const double *x, const int32_t *A, int64_t nA,
           const int32_t *B, int64_t nB, double G, double eps2, double *a)
{
    int err = OR_OK;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : err) if (nA * nB > OR_PAR_MIN)
    for (int64_t ia = 0; ia < nA; ++ia) {
        const int32_t i = A[ia];
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t jb = 0; jb < nB; ++jb) {
            const int32_t j = B[jb];
            if (j == i) continue;
            const double dx = x[3 * j + 0] - x[3 * i + 0];
            const double dy = x[3 * j + 1] - x[3 * i + 1];
            const double dz = x[3 * j + 2] - x[3 * i + 2];
            const double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) { err = OR_ECOINCIDENT; continue; }
            const double r = sqrt(r2);
            const double w = m[j] / (r2 * r);
            sx += w * dx;
            sy += w * dy;
            sz += w * dz;
        }
        a[3 * ia + 0] = G * sx;
        a[3 * ia + 1] = G * sy;
        a[3 * ia + 2] = G * sz;
    }
    or_count_acc += nA * nB;
    return err;
}

/*
 * Gradient acceleration of every active particle i in A due to the sources j in B:
 *   g_i = 2 G sum_{j != i} m_j / r_ji^5 ( r_ji^2 a_ji - 3 (x_ji . a_ji) x_ji ),
 *   a_ji = a_j - a_i                                       (Eq. acc-gradient-g)
 * aA[ia] is the acceleration of A[ia] and aB[jb] that of B[jb] (Newtonian accelerations
 * of the same pass).
 */
int or_grad(const double *m, const double *x, const int32_t *A, int64_t nA, const double *aA,
            const int32_t *B, int64_t nB, const double *aB, double G, double eps2, double *g)
{
    int err = OR_OK;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : err) if (nA * nB > OR_PAR_MIN)
    for (int64_t ia = 0; ia < nA; ++ia) {
        const int32_t i = A[ia];
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t jb = 0; jb < nB; ++jb) {
            const int32_t j = B[jb];
            if (j == i) continue;
            const double dx = x[3 * j + 0] - x[3 * i + 0];
            const double dy = x[3 * j + 1] - x[3 * i + 1];
            const double dz = x[3 * j + 2] - x[3 * i + 2];
            const double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) { err = OR_ECOINCIDENT; continue; }
            const double ax = aB[3 * jb + 0] - aA[3 * ia + 0];
            const double ay = aB[3 * jb + 1] - aA[3 * ia + 1];
            const double az = aB[3 * jb + 2] - aA[3 * ia + 2];
            const double xa = dx * ax + dy * ay + dz * az;
            const double r = sqrt(r2);
            const double r5 = r2 * r2 * r;
            const double w = m[j] / r5;
            sx += w * (r2 * ax - 3.0 * xa * dx);
            sy += w * (r2 * ay - 3.0 * xa * dy);
            sz += w * (r2 * az - 3.0 * xa * dz);
        }
        g[3 * ia + 0] = 2.0 * G * sx;
        g[3 * ia + 1] = 2.0 * G * sy;
        g[3 * ia + 2] = 2.0 * G * sz;
    }
    or_count_grad += nA * nB;
    return err;
}

/* Relation of two index lists: 0 = the same set, 1 = disjoint, -1 = partial overlap or a
 * repeated index.  n_tot bounds the indices. */
static int list_relation(int64_t n_tot, const int32_t *A, int64_t nA, const int32_t *B, int64_t nB)
{
    unsigned char *mark = (unsigned char *)calloc((size_t)(n_tot > 0 ? n_tot : 1), 1);
    if (!mark) return -2;
    for (int64_t k = 0; k < nB; ++k) {
        if (B[k] < 0 || B[k] >= n_tot || mark[B[k]]) { free(mark); return -1; }
        mark[B[k]] = 1;
    }
    int64_t common = 0;
    for (int64_t k = 0; k < nA; ++k) {
        if (A[k] < 0 || A[k] >= n_tot || (mark[A[k]] & 2)) { free(mark); return -1; }
        if (mark[A[k]] & 1) ++common;
        mark[A[k]] |= 2;
    }
    free(mark);
    if (common == 0) return 1;
    if (common == nA && nA == nB) return 0;
    return -1;
}

/*
 * a_i and a~_i = a_i + eps^2 g_i / 48 for every active particle (Eq. acc-gradient,
 * Eqs. force-gradient-inter-1/2).  Intra-set pass if A and B are the same set; cross pass
 * if they are disjoint, in which case the accelerations entering a_ji are the inter-level
 * ones (A due to B, and B due to A).  acc / acc_tilde are [nA][3]; either may be NULL.
 */
int or_accel_gradient(int64_t n_tot, const double *m, const double *x, const int32_t *A,
                      int64_t nA, const int32_t *B, int64_t nB, double G, double eps2,
                      double eps_grad, double *acc, double *acc_tilde)
{
    const int rel = list_relation(n_tot, A, nA, B, nB);
    if (rel == -2) return OR_ENOMEM;
    if (rel < 0) return OR_EINVAL;
    double *aA = (double *)malloc(sizeof(double) * 3 * (size_t)(nA > 0 ? nA : 1));
    double *aB = NULL;
    double *g = (double *)malloc(sizeof(double) * 3 * (size_t)(nA > 0 ? nA : 1));
    int err = OR_OK;
    if (!aA || !g) { err = OR_ENOMEM; goto done; }
    err = or_acc(m, x, A, nA, B, nB, G, eps2, aA);
    if (err) goto done;
    if (acc_tilde) {
        /* a_j of every source: for the same set, its acceleration due to that set (the
         * pass already made, recomputed in B's order); for a cross pass, its acceleration
         * due to the active set (Eq. force-newton-inter, second line). */
        aB = (double *)malloc(sizeof(double) * 3 * (size_t)(nB > 0 ? nB : 1));
        if (!aB) { err = OR_ENOMEM; goto done; }
        err = or_acc(m, x, B, nB, A, nA, G, eps2, aB);
        if (err) goto done;
        err = or_grad(m, x, A, nA, aA, B, nB, aB, G, eps2, g);
        if (err) goto done;
        const double c = eps_grad * eps_grad / 48.0;
        for (int64_t k = 0; k < 3 * nA; ++k) acc_tilde[k] = aA[k] + c * g[k];
    }
    if (acc) memcpy(acc, aA, sizeof(double) * 3 * (size_t)nA);
done:
    free(aA);
    free(aB);
    free(g);
    return err;
}

/*
 * Two-body timescales of the pair (i, j) and their time derivatives:
 *   t_ff = ( r^3 / (G (m_i + m_j)) )^(1/2)                         (Eq. dt-freefall)
 *   t_fb = r / |v_ij|                                               (Eq. dt-flyby)
 *   dt_ff/dt = 3/2 (r . v / r^2) t_ff                               (Eq. dt-freefall-derivative)
 *   dt_fb/dt = (r . v / r^2) (1 + G (m_i + m_j) / (|v|^2 r)) t_fb   (Eq. dt-flyby-derivative,
 *                                                                    two-body approximation)
 * out = {t_ff, dt_ff/dt, t_fb, dt_fb/dt}; t_fb = +inf and dt_fb/dt = 0 when v_ij = 0.
 */
void or_pair_timescales(const double *xi, const double *vi, double mi, const double *xj,
                        const double *vj, double mj, double G, double *out)
{
    const double rx = xi[0] - xj[0], ry = xi[1] - xj[1], rz = xi[2] - xj[2];
    const double ux = vi[0] - vj[0], uy = vi[1] - vj[1], uz = vi[2] - vj[2];
    const double r2 = rx * rx + ry * ry + rz * rz;
    const double v2 = ux * ux + uy * uy + uz * uz;
    const double rv = rx * ux + ry * uy + rz * uz;
    const double r = sqrt(r2);
    const double gm = G * (mi + mj);
    const double tff = sqrt(r2 * r / gm);
    out[0] = tff;
    out[1] = 1.5 * (rv / r2) * tff;
    if (v2 > 0.0) {
        const double tfb = r / sqrt(v2);
        out[2] = tfb;
        out[3] = (rv / r2) * (1.0 + gm / (v2 * r)) * tfb;
    } else {
        out[2] = INFINITY;
        out[3] = 0.0;
    }
}

/* The same with the exact fly-by derivative (first line of Eq. dt-flyby-derivative):
 * d t_fb / dt = [ r.v / r^2 - v.a / v^2 ] t_fb with the relative acceleration a = a_i - a_j
 * (instead of its two-body approximation -G (m_i + m_j) r / r^3). */
void or_pair_timescales_exact(const double *xi, const double *vi, const double *ai, double mi,
                              const double *xj, const double *vj, const double *aj, double mj, double G,
                              double *out)
{
    or_pair_timescales(xi, vi, mi, xj, vj, mj, G, out);
    const double rx = xi[0] - xj[0], ry = xi[1] - xj[1], rz = xi[2] - xj[2];
    const double ux = vi[0] - vj[0], uy = vi[1] - vj[1], uz = vi[2] - vj[2];
    const double wx = ai[0] - aj[0], wy = ai[1] - aj[1], wz = ai[2] - aj[2];
    const double r2 = rx * rx + ry * ry + rz * rz;
    const double v2 = ux * ux + uy * uy + uz * uz;
    if (v2 > 0.0) {
        const double rv = rx * ux + ry * uy + rz * uz;
        const double va = ux * wx + uy * wy + uz * wz;
        out[3] = (rv / r2 - va / v2) * out[2];
    }
}

/* tau_sym / tau for the harmonic mean, with d = d tau / dt (Eq. time-step-factor, second
 * line).  With q = 1 + sqrt(1 + d^2) the printed factor (d + sqrt(1 + d^2) - 1) / d equals
 * (q + d) / q and also 2 / (q - d); each is free of cancellation on one side of d = 0 and
 * both are finite at d = 0. */
double or_sym_harmonic(double d)
{
    const double q = 1.0 + sqrt(1.0 + d * d);
    return d >= 0.0 ? (q + d) / q : 2.0 / (q - d);
}

/* tau_sym / tau for the arithmetic mean (Eq. time-step-factor, first line), valid for
 * d < 2.  For d >= 2 the paper lowers the step until its derivative is below 2 (Sec. 4.2);
 * reading: the step is first scaled by 1/d (its derivative becomes 1), then symmetrised,
 * which gives the factor (1/d) / (1 - 1/2) = 2/d. */
double or_sym_arithmetic(double d)
{
    return d < 2.0 ? 1.0 / (1.0 - 0.5 * d) : 2.0 / d;
}

/*
 * tau_i = min_{j in P, j != i} min( s(eta dt_ff/dt) eta t_ff, s(eta dt_fb/dt) eta t_fb )
 * for every i of the set P (Sec. 4.3: the pair timescales are symmetrised first, then the
 * minimum is taken).  sym & 3 = 0: harmonic factor, 1: arithmetic factor, 2: none (s = 1).
 * sym & OR_FLYBY_EXACT: the exact fly-by derivative, with the accelerations of the set P due
 * to P (reading: the level's own interactions, the same set the minimum runs over), softened
 * by eps2 like the dynamics; otherwise its two-body approximation (no accelerations).
 */
int or_timesteps_ex(const double *m, const double *x, const double *v, const int32_t *A, int64_t nA,
                    const int32_t *P, int64_t nP, double G, double eta, double eps2, int sym,
                    double *tau);

int or_timesteps(const double *m, const double *x, const double *v, const int32_t *P, int64_t nP,
                 double G, double eta, int sym, double *tau)
{
    return or_timesteps_ex(m, x, v, P, nP, P, nP, G, eta, 0.0, sym, tau);
}

/* tau of the particles A, the minimum taken over the set P (A may be a sample of P). */
int or_timesteps_of(const double *m, const double *x, const double *v, const int32_t *A, int64_t nA,
                    const int32_t *P, int64_t nP, double G, double eta, int sym, double *tau)
{
    return or_timesteps_ex(m, x, v, A, nA, P, nP, G, eta, 0.0, sym, tau);
}

int or_timesteps_ex(const double *m, const double *x, const double *v, const int32_t *A, int64_t nA,
                    const int32_t *P, int64_t nP, double G, double eta, double eps2, int sym,
                    double *tau)
{
    int err = OR_OK;
    const int exact = (sym & OR_FLYBY_EXACT) != 0;
    sym &= 3;
    double *aA = NULL, *aP = NULL;
    if (exact) {
        aA = (double *)malloc(sizeof(double) * 3 * (size_t)(nA > 0 ? nA : 1));
        aP = (double *)malloc(sizeof(double) * 3 * (size_t)(nP > 0 ? nP : 1));
        if (!aA || !aP) {
            free(aA);
            free(aP);
            return OR_ENOMEM;
        }
        if ((err = or_acc(m, x, A, nA, P, nP, G, eps2, aA)) || (err = or_acc(m, x, P, nP, P, nP, G, eps2, aP))) {
            free(aA);
            free(aP);
            return err;
        }
    }
#pragma omp parallel for schedule(dynamic, 16) reduction(max : err) if (nA * nP > OR_PAR_MIN)
    for (int64_t ia = 0; ia < nA; ++ia) {
        const int32_t i = A[ia];
        double best = INFINITY;
        for (int64_t jb = 0; jb < nP; ++jb) {
            const int32_t j = P[jb];
            if (j == i) continue;
            double t[4];
            if (exact)
                or_pair_timescales_exact(&x[3 * i], &v[3 * i], &aA[3 * ia], m[i], &x[3 * j], &v[3 * j], &aP[3 * jb],
                                         m[j], G, t);
            else
                or_pair_timescales(&x[3 * i], &v[3 * i], m[i], &x[3 * j], &v[3 * j], m[j], G, t);
            if (!(t[0] > 0.0)) { err = OR_ECOINCIDENT; continue; }
            for (int c = 0; c < 2; ++c) {
                const double tc = t[2 * c];
                if (isinf(tc)) continue;
                const double d = eta * t[2 * c + 1];
                double s = 1.0;
                if (sym == 0) s = or_sym_harmonic(d);
                else if (sym == 1) s = or_sym_arithmetic(d);
                const double ts = s * eta * tc;
                if (ts < best) best = ts;
            }
        }
        tau[ia] = best;
    }
    or_count_tstep += nA * nP;
    free(aA);
    free(aP);
    return err;
}

/* S = {i in P : tau_i >= tau_pivot}, F = the rest, both in the order of P (Sec. 3.1). */
void or_partition(const int32_t *P, int64_t nP, const double *tau, double tau_pivot, int32_t *S,
                  int64_t *nS, int32_t *F, int64_t *nF)
{
    int64_t s = 0, f = 0;
    for (int64_t k = 0; k < nP; ++k) {
        if (tau[k] >= tau_pivot) S[s++] = P[k];
        else F[f++] = P[k];
    }
    *nS = s;
    *nF = f;
}

/* v_i <- v_i + dt a_i for i in I (a indexed by list position) (Sec. 5.3, kick). */
void or_kick(const int32_t *I, int64_t n, double *v, const double *a, double dt)
{
    for (int64_t k = 0; k < n; ++k)
        for (int c = 0; c < 3; ++c) v[3 * I[k] + c] += dt * a[3 * k + c];
}

/* x_i <- x_i + dt v_i for i in I (Sec. 5.3, drift). */
void or_drift(const int32_t *I, int64_t n, double *x, const double *v, double dt)
{
    for (int64_t k = 0; k < n; ++k)
        for (int c = 0; c < 3; ++c) x[3 * I[k] + c] += dt * v[3 * I[k] + c];
}

typedef struct {
    int64_t n;
    const double *m;
    double *x, *v;
    double G, eta, eps2;
    int max_depth, sym;
} or_sys;

/* Algorithm fsi: kick 1/6, drift 1/2, kick 2/3 with a~ (eps = dt), drift 1/2, kick 1/6. */
static int fsi(or_sys *s, const int32_t *S, int64_t nS, double dt)
{
    if (nS == 0) return OR_OK;
    double *a = (double *)malloc(sizeof(double) * 3 * (size_t)nS);
    if (!a) return OR_ENOMEM;
    int err = or_accel_gradient(s->n, s->m, s->x, S, nS, S, nS, s->G, s->eps2, 0.0, a, NULL);
    if (err) goto done;
    or_kick(S, nS, s->v, a, dt / 6.0);
    or_drift(S, nS, s->x, s->v, 0.5 * dt);
    err = or_accel_gradient(s->n, s->m, s->x, S, nS, S, nS, s->G, s->eps2, dt, NULL, a);
    if (err) goto done;
    or_kick(S, nS, s->v, a, 2.0 * dt / 3.0);
    or_drift(S, nS, s->x, s->v, 0.5 * dt);
    err = or_accel_gradient(s->n, s->m, s->x, S, nS, S, nS, s->G, s->eps2, 0.0, a, NULL);
    if (err) goto done;
    or_kick(S, nS, s->v, a, dt / 6.0);
done:
    free(a);
    return err;
}

int or_fsi(int64_t n, const double *m, double *x, double *v, const int32_t *S, int64_t nS,
           double dt, double G, double eps2)
{
    or_sys s = {n, m, x, v, G, 0.0, eps2, 0, 0};
    return fsi(&s, S, nS, dt);
}

/* Inter-level kick (kick_sf): S kicked by its accelerations due to F and F by its
 * accelerations due to S, both computed before either kick.  grad = 0: Newtonian
 * (acc_sf_newton), grad = 1: gradient accelerations with eps = tau (acc_sf_gradient). */
static int kick_sf(or_sys *s, const int32_t *S, int64_t nS, const int32_t *F, int64_t nF,
                   double c_dt, int grad, double tau)
{
    if (nS == 0 || nF == 0) return OR_OK;
    double *aS = (double *)malloc(sizeof(double) * 3 * (size_t)nS);
    double *aF = (double *)malloc(sizeof(double) * 3 * (size_t)nF);
    int err = OR_OK;
    if (!aS || !aF) { err = OR_ENOMEM; goto done; }
    if (grad) {
        err = or_accel_gradient(s->n, s->m, s->x, S, nS, F, nF, s->G, s->eps2, tau, NULL, aS);
        if (!err) err = or_accel_gradient(s->n, s->m, s->x, F, nF, S, nS, s->G, s->eps2, tau, NULL, aF);
    } else {
        err = or_acc(s->m, s->x, S, nS, F, nF, s->G, s->eps2, aS);
        if (!err) err = or_acc(s->m, s->x, F, nF, S, nS, s->G, s->eps2, aF);
    }
    if (err) goto done;
    or_kick(S, nS, s->v, aS, c_dt);
    or_kick(F, nF, s->v, aF, c_dt);
done:
    free(aS);
    free(aF);
    return err;
}

/* Algorithm hhs-fsi on the set P with pivot step tau at recursion depth `depth`. */
static int hhs_fsi(or_sys *s, const int32_t *P, int64_t nP, double tau, int depth)
{
    if (nP == 0) return OR_OK;
    if (depth > s->max_depth) return OR_EDEPTH;
    if (depth > or_max_depth_seen) or_max_depth_seen = depth;
    int err = OR_OK;
    double *t = (double *)malloc(sizeof(double) * (size_t)nP);
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)nP);
    int32_t *F = (int32_t *)malloc(sizeof(int32_t) * (size_t)nP);
    int64_t nS = 0, nF = 0;
    if (!t || !S || !F) { err = OR_ENOMEM; goto done; }
    err = or_timesteps_ex(s->m, s->x, s->v, P, nP, P, nP, s->G, s->eta, s->eps2, s->sym, t);
    if (err) goto done;
    or_partition(P, nP, t, tau, S, &nS, F, &nF);
    if ((err = kick_sf(s, S, nS, F, nF, tau / 6.0, 0, tau))) goto done;
    if ((err = fsi(s, S, nS, 0.5 * tau))) goto done;
    if ((err = hhs_fsi(s, F, nF, 0.5 * tau, depth + 1))) goto done;
    if ((err = kick_sf(s, S, nS, F, nF, 2.0 * tau / 3.0, 1, tau))) goto done;
    if ((err = hhs_fsi(s, F, nF, 0.5 * tau, depth + 1))) goto done;
    if ((err = fsi(s, S, nS, 0.5 * tau))) goto done;
    err = kick_sf(s, S, nS, F, nF, tau / 6.0, 0, tau);
done:
    free(t);
    free(S);
    free(F);
    return err;
}

int or_hhs_fsi(int64_t n, const double *m, double *x, double *v, const int32_t *P, int64_t nP,
               double tau_pivot, double G, double eta, double eps2, int max_depth, int sym)
{
    or_sys s = {n, m, x, v, G, eta, eps2, max_depth, sym};
    return hhs_fsi(&s, P, nP, tau_pivot, 0);
}

/* Main loop of Algorithm frost: n_steps calls hhs_fsi(all particles, dt). */
/*
 * Second-order HOLD integrator (Eq. hhs2, Sec. 3.1), the comparison integrator of the paper:
 *   e^{eps H} ~ e^{eps/2 H_F} e^{eps/2 H_S} e^{eps U_FS} e^{eps/2 H_S} e^{eps/2 H_F}
 * with e^{h H_S} the leapfrog kick(h/2) drift(h) kick(h/2) of the slow set under its own
 * forces (the equation that follows Eq. hhs2), e^{eps U_FS} one pairwise kick of S and F
 * with their mutual accelerations, and e^{eps/2 H_F} the same operator recursively on the
 * fast set with the pivot halved.
 */
static int leapfrog(or_sys *s, const int32_t *S, int64_t nS, double h)
{
    if (nS == 0) return OR_OK;
    double *a = (double *)malloc(sizeof(double) * 3 * (size_t)nS);
    if (!a) return OR_ENOMEM;
    int err = or_acc(s->m, s->x, S, nS, S, nS, s->G, s->eps2, a);
    if (!err) {
        or_kick(S, nS, s->v, a, 0.5 * h);
        or_drift(S, nS, s->x, s->v, h);
        err = or_acc(s->m, s->x, S, nS, S, nS, s->G, s->eps2, a);
    }
    if (!err) or_kick(S, nS, s->v, a, 0.5 * h);
    free(a);
    return err;
}

static int hold2(or_sys *s, const int32_t *P, int64_t nP, double tau, int depth)
{
    if (nP == 0) return OR_OK;
    if (depth > s->max_depth) return OR_EDEPTH;
    if (depth > or_max_depth_seen) or_max_depth_seen = depth;
    int err = OR_OK;
    double *t = (double *)malloc(sizeof(double) * (size_t)nP);
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)nP);
    int32_t *F = (int32_t *)malloc(sizeof(int32_t) * (size_t)nP);
    int64_t nS = 0, nF = 0;
    if (!t || !S || !F) { err = OR_ENOMEM; goto done; }
    err = or_timesteps_ex(s->m, s->x, s->v, P, nP, P, nP, s->G, s->eta, s->eps2, s->sym, t);
    if (err) goto done;
    or_partition(P, nP, t, tau, S, &nS, F, &nF);
    if ((err = hold2(s, F, nF, 0.5 * tau, depth + 1))) goto done;
    if ((err = leapfrog(s, S, nS, 0.5 * tau))) goto done;
    if ((err = kick_sf(s, S, nS, F, nF, tau, 0, tau))) goto done;
    if ((err = leapfrog(s, S, nS, 0.5 * tau))) goto done;
    err = hold2(s, F, nF, 0.5 * tau, depth + 1);
done:
    free(t);
    free(S);
    free(F);
    return err;
}

/* n_steps top-level steps of the second-order HOLD integrator over all particles. */
int or_steps_hold(int64_t n, const double *m, double *x, double *v, double dt, int64_t n_steps,
                  double G, double eta, double eps2, int max_depth, int sym)
{
    int32_t *all = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!all) return OR_ENOMEM;
    for (int64_t k = 0; k < n; ++k) all[k] = (int32_t)k;
    or_sys s = {n, m, x, v, G, eta, eps2, max_depth, sym};
    int err = OR_OK;
    for (int64_t k = 0; k < n_steps && !err; ++k) err = hold2(&s, all, n, dt, 0);
    free(all);
    return err;
}

int or_steps(int64_t n, const double *m, double *x, double *v, double dt, int64_t n_steps,
             double G, double eta, double eps2, int max_depth, int sym)
{
    int32_t *all = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!all) return OR_ENOMEM;
    for (int64_t k = 0; k < n; ++k) all[k] = (int32_t)k;
    or_sys s = {n, m, x, v, G, eta, eps2, max_depth, sym};
    int err = OR_OK;
    for (int64_t k = 0; k < n_steps && !err; ++k) err = hhs_fsi(&s, all, n, dt, 0);
    free(all);
    return err;
}

/*
 * Kinetic energy T = 1/2 sum m v^2, potential U = -G sum_{i<j} m_i m_j / r_ij (Sec. 2.3,
 * softened r -> (r^2 + eps^2)^(1/2)), momentum P = sum m v, angular momentum
 * L = sum m x cross v.  out = {T, U, Px, Py, Pz, Lx, Ly, Lz}.
 */
int or_energy(int64_t n, const double *m, const double *x, const double *v, double G,
              double eps2, double *out)
{
    double *e = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!e) return OR_ENOMEM;
    int err = OR_OK;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : err) if (n * n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            const double dx = x[3 * j + 0] - x[3 * i + 0];
            const double dy = x[3 * j + 1] - x[3 * i + 1];
            const double dz = x[3 * j + 2] - x[3 * i + 2];
            const double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) { err = OR_ECOINCIDENT; continue; }
            s += m[j] / sqrt(r2);
        }
        e[i] = s;
    }
    double T = 0.0, U = 0.0, P[3] = {0, 0, 0}, L[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        const double *xi = &x[3 * i], *vi = &v[3 * i];
        T += 0.5 * m[i] * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]);
        U += m[i] * e[i];
        for (int c = 0; c < 3; ++c) P[c] += m[i] * vi[c];
        L[0] += m[i] * (xi[1] * vi[2] - xi[2] * vi[1]);
        L[1] += m[i] * (xi[2] * vi[0] - xi[0] * vi[2]);
        L[2] += m[i] * (xi[0] * vi[1] - xi[1] * vi[0]);
    }
    free(e);
    out[0] = T;
    out[1] = -G * U;
    for (int c = 0; c < 3; ++c) {
        out[2 + c] = P[c];
        out[5 + c] = L[c];
    }
    return err;
}
