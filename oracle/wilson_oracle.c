/*
 * FP64 CPU oracle for the Wilson multi-mass solve of Alexandru, Pelissier,
 * Gamari & Lee, "Multi-mass solvers for lattice QCD on GPUs" (arXiv:1103.5103).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the library
 * never calls it and shares no code with it.
 *
 * Everything is FP64, scalar loops, C99 complex arithmetic.  The per-site
 * loops of the hop and of the sampled-site operator may run on several
 * threads (an OpenMP parallel-for when built with -fopenmp): every output
 * site is computed by the same code from the same inputs, so the result is
 * bit-identical for any thread count.  Reductions stay sequential.
 * Fields use the canonical layouts:
 *   spinor psi[n][s][c]      (site n lexicographic, spin s = 0..3, colour c = 0..2)
 *   links  U[mu][n][a][b]    (mu = 0..3 <-> x, y, z, t = the paper's gamma_1..gamma_4)
 * with n = x + X*(y + Y*(z + Z*t)).  Site parity = (x+y+z+t) mod 2.
 *
 * Operators (Section 2, Eq. 3 and Eq. 4):
 *   (D psi)_n = sum_mu [ U_mu(n) psi_{n+mu} (1 - gamma_mu)
 *                       + U_mu(n-mu)^dag psi_{n-mu} (1 + gamma_mu) ]
 *   with psi_n read as a 3x4 matrix (colour rows, spin columns) and the spin
 *   matrix multiplying from the right, exactly as Eq. 4 writes it.  Hops that
 *   cross the time boundary carry a factor -1 when the lattice is
 *   antiperiodic in time (the paper is silent on boundaries; this is the
 *   standard fermion boundary condition the workloads use).
 *   M_p(m) = (m+4) - D/2                      (Eq. 3, the paper's form)
 *   M_k    = 1 - kappa D,  kappa = 1/(2m+8)   (so M_p = (m+4) M_k)
 *   M_prec = 1 - kappa^2 D_eo D_oe            (kappa form of Eqs. eo2-eo4)
 *
 * Parity is unpinned for nothing in this file: every function is pinned by
 * a CPU test (free-field closed form, constant-abelian closed form, gauge
 * covariance, gamma5-hermiticity, dense LU solves, finite differences).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { OR_OP_HOP = 0, OR_OP_MK = 1, OR_OP_MP = 2, OR_OP_MPREC = 3 };
enum { OR_OK = 0, OR_NOCONV = 1, OR_ERR = 2 };

/* Operator descriptor handed in from Python. */
typedef struct {
    int kind;            /* OR_OP_* */
    int dims[4];         /* X, Y, Z, T */
    int antiperiodic_t;  /* 1: -1 on hops across the t boundary */
    int dagger;          /* 1: apply the adjoint */
    double param;        /* kappa for MK/MPREC, bare mass m for MP */
    const cplx *U;       /* links [4][V][3][3] */
} or_op;

typedef struct {
    int iterations;      /* Krylov iterations */
    int matvecs;         /* applications of the operator */
    int restarts;        /* restarts after an iterated/true residual gap or breakdown */
    double true_relres;  /* ||b - A x|| / bref at exit */
} or_stats;

/* Threads for the per-site loops: n > 0 sets the count; returns the count
 * in use (1 when built without OpenMP). */
int or_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---------------------------------------------------------------- gamma -- */

/* gamma_i = [[0, i sigma_i], [-i sigma_i, 0]], gamma_4 = [[0, -1], [-1, 0]]
 * (Section 2, the gamma-matrix definition after Eq. 4). */
static void or_gammas(cplx g[4][4][4])
{
    cplx sig[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(g, 0, sizeof(cplx) * 64);
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                g[i][a][2 + b] = I * sig[i][a][b];
                g[i][2 + a][b] = -I * sig[i][a][b];
            }
    g[3][0][2] = g[3][1][3] = g[3][2][0] = g[3][3][1] = -1;
}

/* Export gamma_1..gamma_4 and gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4. */
void or_gamma_matrices(cplx *g_out /* [5][4][4] */)
{
    cplx g[4][4][4];
    or_gammas(g);
    memcpy(g_out, g, sizeof(g));
    cplx t1[4][4], t2[4][4];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += g[0][a][k] * g[1][k][b];
            t1[a][b] = s;
        }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += t1[a][k] * g[2][k][b];
            t2[a][b] = s;
        }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += t2[a][k] * g[3][k][b];
            g_out[64 + 4 * a + b] = s;
        }
}

/* ------------------------------------------------------------- geometry -- */

static long or_volume(const int d[4]) { return (long)d[0] * d[1] * d[2] * d[3]; }

static void or_coords(const int d[4], long n, int x[4])
{
    x[0] = (int)(n % d[0]); n /= d[0];
    x[1] = (int)(n % d[1]); n /= d[1];
    x[2] = (int)(n % d[2]); n /= d[2];
    x[3] = (int)n;
}

static long or_lex(const int d[4], const int x[4])
{
    return x[0] + (long)d[0] * (x[1] + (long)d[1] * (x[2] + (long)d[2] * x[3]));
}

/* Neighbour n +- mu with periodic wrap; *sign = -1 when the hop crosses the
 * time boundary of an antiperiodic lattice. */
static long or_neighbour(const int d[4], int ap, long n, int mu, int dir, double *sign)
{
    int x[4];
    or_coords(d, n, x);
    int v = x[mu] + dir;
    *sign = 1.0;
    if (v >= d[mu]) { v -= d[mu]; if (mu == 3 && ap) *sign = -1.0; }
    if (v < 0) { v += d[mu]; if (mu == 3 && ap) *sign = -1.0; }
    x[mu] = v;
    return or_lex(d, x);
}

int or_site_parity(const int d[4], long n)
{
    int x[4];
    or_coords(d, n, x);
    return (x[0] + x[1] + x[2] + x[3]) & 1;
}

/* ------------------------------------------------------------------ hop -- */

/* out = D in on the whole lattice (Eq. 4 summed over the eight directions).
 * psi_n is the 3x4 matrix psi[c][s] = in[12 n + 3 s + c]. */
void or_hop(const int d[4], int ap, const cplx *U, const cplx *in, cplx *out)
{
    cplx g[4][4][4];
    or_gammas(g);
    cplx Pm[4][4][4], Pp[4][4][4]; /* 1 - gamma_mu, 1 + gamma_mu */
    for (int mu = 0; mu < 4; ++mu)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                cplx id = (a == b) ? 1.0 : 0.0;
                Pm[mu][a][b] = id - g[mu][a][b];
                Pp[mu][a][b] = id + g[mu][a][b];
            }
    const long V = or_volume(d);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < V; ++n) {
        cplx acc[3][4] = {{0}};
        for (int mu = 0; mu < 4; ++mu) {
            for (int dir = +1; dir >= -1; dir -= 2) {
                double sign;
                long m = or_neighbour(d, ap, n, mu, dir, &sign);
                /* link: U_mu(n) forward, U_mu(n - mu)^dagger backward */
                cplx L[3][3];
                const cplx *u = U + ((long)mu * V + (dir > 0 ? n : m)) * 9;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        L[a][b] = dir > 0 ? u[3 * a + b] : conj(u[3 * b + a]);
                /* colour: tmp = L psi_m (3x3 times 3x4) */
                cplx tmp[3][4];
                for (int a = 0; a < 3; ++a)
                    for (int s = 0; s < 4; ++s) {
                        cplx t = 0;
                        for (int b = 0; b < 3; ++b) t += L[a][b] * in[12 * m + 3 * s + b];
                        tmp[a][s] = t;
                    }
                /* spin: acc += sign * tmp (1 -/+ gamma_mu), matrix on the right */
                cplx (*P)[4] = dir > 0 ? Pm[mu] : Pp[mu];
                for (int a = 0; a < 3; ++a)
                    for (int s = 0; s < 4; ++s) {
                        cplx t = 0;
                        for (int k = 0; k < 4; ++k) t += tmp[a][k] * P[k][s];
                        acc[a][s] += sign * t;
                    }
            }
        }
        for (int a = 0; a < 3; ++a)
            for (int s = 0; s < 4; ++s) out[12 * n + 3 * s + a] = acc[a][s];
    }
}

/* (M_k psi)_n = psi_n - kappa (D psi)_n at the listed sites only (Eq. 4 per
 * site), for checking large solutions at a sample of sites.  out[j] holds
 * the 12 complex entries of site sites[j]. */
void or_apply_mk_sites(const int d[4], int ap, const cplx *U, const cplx *in, double kappa, const long *sites,
                       long nsites, cplx *out)
{
    cplx g[4][4][4];
    or_gammas(g);
    const long V = or_volume(d);
#pragma omp parallel for schedule(static)
    for (long j = 0; j < nsites; ++j) {
        const long n = sites[j];
        cplx acc[3][4] = {{0}};
        for (int mu = 0; mu < 4; ++mu) {
            for (int dir = +1; dir >= -1; dir -= 2) {
                double sign;
                long m = or_neighbour(d, ap, n, mu, dir, &sign);
                cplx L[3][3];
                const cplx *u = U + ((long)mu * V + (dir > 0 ? n : m)) * 9;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) L[a][b] = dir > 0 ? u[3 * a + b] : conj(u[3 * b + a]);
                cplx tmp[3][4];
                for (int a = 0; a < 3; ++a)
                    for (int s = 0; s < 4; ++s) {
                        cplx t = 0;
                        for (int b = 0; b < 3; ++b) t += L[a][b] * in[12 * m + 3 * s + b];
                        tmp[a][s] = t;
                    }
                for (int a = 0; a < 3; ++a)
                    for (int s = 0; s < 4; ++s) {
                        cplx t = 0;
                        for (int k = 0; k < 4; ++k)
                            t += tmp[a][k] * ((k == s ? 1.0 : 0.0) + (dir > 0 ? -1.0 : 1.0) * g[mu][k][s]);
                        acc[a][s] += sign * t;
                    }
            }
        }
        for (int a = 0; a < 3; ++a)
            for (int s = 0; s < 4; ++s) out[12 * j + 3 * s + a] = in[12 * n + 3 * s + a] - kappa * acc[a][s];
    }
}

/* psi -> psi gamma_5 (gamma_5 = diag(1, 1, -1, -1) acting on the spin index). */
void or_gamma5(const int d[4], const cplx *in, cplx *out)
{
    cplx g[5][4][4];
    or_gamma_matrices(&g[0][0][0]);
    const long V = or_volume(d);
    for (long n = 0; n < V; ++n)
        for (int c = 0; c < 3; ++c)
            for (int s = 0; s < 4; ++s) {
                cplx t = 0;
                for (int k = 0; k < 4; ++k) t += in[12 * n + 3 * k + c] * g[4][k][s];
                out[12 * n + 3 * s + c] = t;
            }
}

/* Zero the sites of the given parity. */
static void or_mask_parity(const int d[4], cplx *v, int parity)
{
    const long V = or_volume(d);
    for (long n = 0; n < V; ++n)
        if (or_site_parity(d, n) == parity)
            for (int k = 0; k < 12; ++k) v[12 * n + k] = 0;
}

/* D or D^dagger = gamma5 D gamma5 on a full-lattice vector. */
static void or_hop_dag(const or_op *A, const cplx *in, cplx *out, cplx *w)
{
    const long n12 = or_volume(A->dims) * 12;
    if (!A->dagger) { or_hop(A->dims, A->antiperiodic_t, A->U, in, out); return; }
    or_gamma5(A->dims, in, w);
    or_hop(A->dims, A->antiperiodic_t, A->U, w, out);
    memcpy(w, out, sizeof(cplx) * n12);
    or_gamma5(A->dims, w, out);
}

/* out = A in for the four operator kinds.  MPREC acts on vectors whose odd
 * sites are zero and returns a vector whose odd sites are zero. */
void or_apply(const or_op *A, const cplx *in, cplx *out)
{
    const long n12 = or_volume(A->dims) * 12;
    cplx *w = (cplx *)malloc(sizeof(cplx) * n12);
    if (A->kind == OR_OP_HOP) {
        or_hop_dag(A, in, out, w);
    } else if (A->kind == OR_OP_MK) {
        or_hop_dag(A, in, out, w);
        for (long i = 0; i < n12; ++i) out[i] = in[i] - A->param * out[i];
    } else if (A->kind == OR_OP_MP) {
        or_hop_dag(A, in, out, w);
        for (long i = 0; i < n12; ++i) out[i] = (A->param + 4.0) * in[i] - 0.5 * out[i];
    } else { /* OR_OP_MPREC: x - kappa^2 D_eo D_oe x on even sites */
        cplx *e = (cplx *)malloc(sizeof(cplx) * n12);
        cplx *o = (cplx *)malloc(sizeof(cplx) * n12);
        memcpy(e, in, sizeof(cplx) * n12);
        or_mask_parity(A->dims, e, 1);          /* x_e */
        or_hop_dag(A, e, o, w);
        or_mask_parity(A->dims, o, 0);          /* D_oe x_e */
        or_hop_dag(A, o, out, w);
        or_mask_parity(A->dims, out, 1);        /* D_eo D_oe x_e */
        const double k2 = A->param * A->param;
        for (long i = 0; i < n12; ++i) out[i] = e[i] - k2 * out[i];
        free(e);
        free(o);
    }
    free(w);
}

/* ----------------------------------------------------------------- BLAS -- */

static cplx or_dot(long n, const cplx *a, const cplx *b)
{
    cplx s = 0;
    for (long i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

static double or_norm(long n, const cplx *a) { return sqrt(creal(or_dot(n, a, a))); }

double or_norm2(long n, const cplx *a) { return creal(or_dot(n, a, a)); }

void or_dot_export(long n, const cplx *a, const cplx *b, cplx *out) { *out = or_dot(n, a, b); }

/* ------------------------------------------------------------- BiCGstab -- */

/* van der Vorst BiCGstab (the single-mass inverter the paper cites in
 * Section 6; it does not print it), <a,b> = sum conj(a) b:
 *   r = b - A x, rhat = r, p = r, rho = <rhat, r>
 *   loop: v = A p; alpha = rho / <rhat, v>; s = r - alpha v
 *         t = A s; omega = <t, s> / <t, t>
 *         x += alpha p + omega s; r = s - omega t
 *         rho' = <rhat, r>; beta = (rho'/rho)(alpha/omega); p = r + beta (p - omega v)
 * Stops when the true residual ||b - A x|| <= tol * bref.  When the
 * iterated residual reaches the target but the true one does not, or when a
 * denominator vanishes, the recursion restarts from the current x with
 * r = rhat = p = b - A x.  Returns OR_OK or OR_NOCONV (x = last iterate). */
int or_bicgstab(const or_op *A, const cplx *b, cplx *x, double tol, double bref,
                int maxiter, or_stats *st)
{
    const long n = or_volume(A->dims) * 12;
    cplx *r = malloc(sizeof(cplx) * n), *rh = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *v = malloc(sizeof(cplx) * n);
    cplx *s = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    int it = 0, mv = 0, restarts = 0, status = OR_NOCONV;
    const double target = tol * bref;

    for (;;) { /* (re)start */
        or_apply(A, x, r); ++mv;
        for (long i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double rn = or_norm(n, r);
        if (rn <= target) { status = OR_OK; break; }
        if (it >= maxiter) break;
        memcpy(rh, r, sizeof(cplx) * n);
        memcpy(p, r, sizeof(cplx) * n);
        cplx rho = or_dot(n, rh, r);
        int restart = 0;
        while (it < maxiter) {
            or_apply(A, p, v); ++mv;
            cplx rv = or_dot(n, rh, v);
            if (rv == 0) { restart = 1; break; }
            cplx alpha = rho / rv;
            for (long i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
            or_apply(A, s, t); ++mv;
            double tt = creal(or_dot(n, t, t));
            cplx omega = tt > 0 ? or_dot(n, t, s) / tt : 0;
            for (long i = 0; i < n; ++i) x[i] += alpha * p[i] + omega * s[i];
            for (long i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
            ++it;
            rn = or_norm(n, r);
            if (rn <= target) break;               /* check the true residual */
            cplx rho1 = or_dot(n, rh, r);
            if (omega == 0 || rho1 == 0) { restart = 1; break; }
            cplx beta = (rho1 / rho) * (alpha / omega);
            rho = rho1;
            for (long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        }
        (void)restart;
        ++restarts;
    }
    if (st) {
        st->iterations = it;
        st->matvecs = mv;
        st->restarts = restarts - 1 > 0 ? restarts - 1 : 0;
        or_apply(A, x, r);
        for (long i = 0; i < n; ++i) r[i] = b[i] - r[i];
        st->true_relres = or_norm(n, r) / bref;
    }
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return status;
}

/* ----------------------------------------------------------- BiCGstab-M -- */

/* Multi-shift BiCGstab (Section 6.1; the paper cites Jegerlehner and does
 * not print the recurrences).  Unshifted system A = M_p(m_s) with
 * m_s = min m_i, zero initial guess, shifts sigma_i = m_i - m_s, so that
 * (A + sigma_i) psi_i = b.  Per shift, with pi_{-1} = pi_0 = 1, lambda_0 = 1,
 * alpha_{-1} = 1, beta_{-1} = 0, x^s = 0, p^s = b, after alpha_n, omega_n:
 *   c = alpha_n beta_{n-1} / alpha_{n-1}
 *   pi_{n+1} = (1 + c + alpha_n sigma) pi_n - c pi_{n-1}
 *   alpha^s = alpha_n pi_n / pi_{n+1},   omega^s = omega_n / (1 + omega_n sigma)
 *   r^s = r_n / (pi_n lambda_n),          s^s = s_n / (pi_{n+1} lambda_n)
 *   x^s += alpha^s p^s + omega^s s^s
 * and after r_{n+1}, beta_n:
 *   lambda_{n+1} = lambda_n (1 + omega_n sigma),  beta^s = beta_n (pi_n/pi_{n+1})^2
 *   p^s = r_{n+1}/(pi_{n+1} lambda_{n+1}) + beta^s (p^s - (omega^s/alpha^s)(r^s - s^s))
 * The shifted residual is r_{n+1} / (pi_{n+1} lambda_{n+1}); a shift whose
 * residual norm is below tol*||b|| is frozen (Section 6.1).  The loop stops
 * when the unshifted iterated residual is below tol*||b||.
 * Outputs psi_i in the paper's normalisation, one per entry of masses
 * (x_out[i] has V*12 entries).  Returns OR_OK or OR_NOCONV. */
int or_bicgstab_m(const int d[4], int ap, const cplx *U, const double *masses, int nm,
                  const cplx *b, const cplx *rhat0 /* shadow residual, NULL: b */, cplx **x_out,
                  double tol, int maxiter, int *iters_out /* per mass: iteration at which it froze */)
{
    const long n = or_volume(d) * 12;
    int is = 0;
    for (int i = 1; i < nm; ++i) if (masses[i] < masses[is]) is = i;
    or_op A = {OR_OP_MP, {d[0], d[1], d[2], d[3]}, ap, 0, masses[is], U};

    cplx *r = malloc(sizeof(cplx) * n), *rh = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *v = malloc(sizeof(cplx) * n);
    cplx *s = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    cplx *rold = malloc(sizeof(cplx) * n);
    cplx **ps = malloc(sizeof(cplx *) * nm);
    cplx *pi_prev = malloc(sizeof(cplx) * nm), *pi = malloc(sizeof(cplx) * nm);
    cplx *lam = malloc(sizeof(cplx) * nm), *pin = malloc(sizeof(cplx) * nm);
    cplx *als = malloc(sizeof(cplx) * nm), *oms = malloc(sizeof(cplx) * nm);
    int *active = malloc(sizeof(int) * nm);
    double *sig = malloc(sizeof(double) * nm);

    const double bn = or_norm(n, b), target = tol * bn;
    memcpy(r, b, sizeof(cplx) * n);
    memcpy(rh, rhat0 ? rhat0 : b, sizeof(cplx) * n);
    memcpy(p, b, sizeof(cplx) * n);
    for (int i = 0; i < nm; ++i) {
        sig[i] = masses[i] - masses[is];
        memset(x_out[i], 0, sizeof(cplx) * n);
        active[i] = 1;
        ps[i] = NULL;
        if (i != is) { ps[i] = malloc(sizeof(cplx) * n); memcpy(ps[i], b, sizeof(cplx) * n); }
        pi_prev[i] = pi[i] = lam[i] = 1;
        iters_out[i] = 0;
    }
    cplx *x = x_out[is];
    cplx rho = or_dot(n, rh, r), alpha_prev = 1, beta_prev = 0;
    const double rhn = or_norm(n, rh);
    double rn_cur = bn;
    int it = 0, status = OR_NOCONV;
    if (bn == 0) status = OR_OK;
    while (status == OR_NOCONV && it < maxiter) {
        or_apply(&A, p, v);
        /* Breakdown: rho = <rhat, r> or <rhat, v> vanishes to rounding
         * (below 1e-12 of the Cauchy-Schwarz bound), and the recurrences are
         * driven by noise from then on.  With rhat = b a point source, rho
         * vanishes exactly after one iteration in exact arithmetic: r_1 at
         * the source site comes from closed two-hop paths, all backtracks on
         * extents >= 4, and (1 - gamma_mu)(1 + gamma_mu) = 0. */
        const cplx rv = or_dot(n, rh, v);
        if (!(cabs(rho) > 1e-12 * rhn * rn_cur) || !(cabs(rv) > 1e-12 * rhn * or_norm(n, v))) {
            status = OR_ERR;
            break;
        }
        cplx alpha = rho / rv;
        for (long k = 0; k < n; ++k) s[k] = r[k] - alpha * v[k];
        or_apply(&A, s, t);
        cplx omega = or_dot(n, t, s) / or_dot(n, t, t);
        for (int i = 0; i < nm; ++i) {
            if (i == is || !active[i]) continue;
            cplx c = alpha * beta_prev / alpha_prev;
            pin[i] = (1.0 + c + alpha * sig[i]) * pi[i] - c * pi_prev[i];
            als[i] = alpha * pi[i] / pin[i];
            oms[i] = omega / (1.0 + omega * sig[i]);
            cplx *xs = x_out[i];
            for (long k = 0; k < n; ++k)
                xs[k] += als[i] * ps[i][k] + oms[i] * s[k] / (pin[i] * lam[i]);
        }
        for (long k = 0; k < n; ++k) x[k] += alpha * p[k] + omega * s[k];
        memcpy(rold, r, sizeof(cplx) * n);
        for (long k = 0; k < n; ++k) r[k] = s[k] - omega * t[k];
        ++it;
        cplx rho1 = or_dot(n, rh, r);
        cplx beta = (rho1 / rho) * (alpha / omega);
        const double rn = or_norm(n, r);
        rn_cur = rn;
        for (int i = 0; i < nm; ++i) {
            if (i == is || !active[i]) continue;
            cplx lamn = lam[i] * (1.0 + omega * sig[i]);
            cplx bes = beta * (pi[i] / pin[i]) * (pi[i] / pin[i]);
            cplx f = oms[i] / als[i];
            for (long k = 0; k < n; ++k) {
                cplx rs = rold[k] / (pi[i] * lam[i]);
                cplx ss = s[k] / (pin[i] * lam[i]);
                ps[i][k] = r[k] / (pin[i] * lamn) + bes * (ps[i][k] - f * (rs - ss));
            }
            pi_prev[i] = pi[i];
            pi[i] = pin[i];
            lam[i] = lamn;
            if (rn / cabs(pi[i] * lam[i]) < target) { active[i] = 0; iters_out[i] = it; }
        }
        for (long k = 0; k < n; ++k) p[k] = r[k] + beta * (p[k] - omega * v[k]);
        alpha_prev = alpha;
        beta_prev = beta;
        rho = rho1;
        if (rn < target) status = OR_OK;
    }
    for (int i = 0; i < nm; ++i) if (active[i] || i == is) iters_out[i] = it;
    for (int i = 0; i < nm; ++i) free(ps[i]);
    free(ps); free(r); free(rh); free(p); free(v); free(s); free(t); free(rold);
    free(pi_prev); free(pi); free(lam); free(pin); free(als); free(oms); free(active); free(sig);
    return status;
}

/* ----------------------------------------------------------- link force -- */

/* Derivative of a real loss through M_k x = b with respect to the links.
 * Given the solution x and the adjoint solution lam = M_k^{-dag} g, where g
 * is the loss gradient dL/d(Re x) + i dL/d(Im x), perturb
 * U_mu(n) -> exp(i h T) U_mu(n) with T Hermitian traceless.  Then
 *   dL/dh = -Re<lam, (dM/dh) x> = -kappa * Im tr(T W_mu(n)),
 *   W_mu(n) = sign * [ U_mu(n) x_{n+mu} (1 - gamma_mu) lam_n^dag
 *                      - x_n (1 + gamma_mu) lam_{n+mu}^dag U_mu(n)^dag ],
 * a 3x3 colour matrix (3x4 . 4x4 . 4x3).  The output is the component along
 * each generator T_a = lambda_a / 2, accumulated into force[mu][n][a]
 * (8 reals per link): force += -coef * Im tr(T_a W).  coef = kappa for M_k.
 * gm holds the eight Gell-Mann matrices [8][3][3]. */
void or_link_force(const int d[4], int ap, const cplx *U, const cplx *x, const cplx *lam,
                   double coef, const cplx *gm, double *force)
{
    cplx g[4][4][4];
    or_gammas(g);
    const long V = or_volume(d);
    for (int mu = 0; mu < 4; ++mu)
        for (long n = 0; n < V; ++n) {
            double sign;
            long m = or_neighbour(d, ap, n, mu, +1, &sign);
            const cplx *u = U + ((long)mu * V + n) * 9;
            cplx A[3][4], B[3][4];   /* A = U x_m (1 - g), B = x_n (1 + g) */
            cplx Ux[3][4];
            for (int a = 0; a < 3; ++a)
                for (int s = 0; s < 4; ++s) {
                    cplx t = 0;
                    for (int b = 0; b < 3; ++b) t += u[3 * a + b] * x[12 * m + 3 * s + b];
                    Ux[a][s] = t;
                }
            for (int a = 0; a < 3; ++a)
                for (int s = 0; s < 4; ++s) {
                    cplx ta = 0, tb = 0;
                    for (int k = 0; k < 4; ++k) {
                        cplx pm = (k == s ? 1.0 : 0.0) - g[mu][k][s];
                        cplx pp = (k == s ? 1.0 : 0.0) + g[mu][k][s];
                        ta += Ux[a][k] * pm;
                        tb += x[12 * n + 3 * k + a] * pp;
                    }
                    A[a][s] = ta;
                    B[a][s] = tb;
                }
            /* W = A lam_n^dag - B lam_m^dag U^dag */
            cplx W[3][3], BL[3][3];
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    cplx t1 = 0, t2 = 0;
                    for (int s = 0; s < 4; ++s) {
                        t1 += A[a][s] * conj(lam[12 * n + 3 * s + c]);
                        t2 += B[a][s] * conj(lam[12 * m + 3 * s + c]);
                    }
                    W[a][c] = t1;
                    BL[a][c] = t2;
                }
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    cplx t = 0;
                    for (int b = 0; b < 3; ++b) t += BL[a][b] * conj(u[3 * c + b]);
                    W[a][c] = sign * (W[a][c] - t);
                }
            for (int k = 0; k < 8; ++k) {
                cplx tr = 0; /* tr(T_k W), T_k = gm_k / 2 */
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) tr += 0.5 * gm[9 * k + 3 * a + c] * W[c][a];
                force[((long)mu * V + n) * 8 + k] += -coef * cimag(tr);
            }
        }
}
