/*
 * lee_oracle.c -- plain FP64 CPU restatement of the BGK lattice Boltzmann schemes for the
 * Linearized Euler Equations without background velocity (Otte & Frank, arXiv:1601.08103).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is checked against.
 * Only the test suite, the smoke check and the CPU-baseline leg of the benchmark load it.  It
 * shares no code, header, table or constant with the CUDA library: the velocity sets below are
 * built here from the paper's formulas, independently of the GPU tables.
 *
 * Everything is FP64, loops are plain, and the update is written in the paper's order:
 *   moments (Sec. 4, discrete moments; Sec. 5, polyatomic temperature)
 *   -> equilibrium (Sec. 4 eq. "equilibrium" for monoatomic sets, Sec. 5 general form otherwise)
 *   -> BGK relaxation and streaming (Sec. 6, eqs. "LBE" / "LBE update scheme"), in PUSH form:
 *      g_i(t+1, x + c_i) = (1 - 1/tau) g_i(t, x) + (1/tau) g_i^eq(t, x).
 * The array g always holds the paper's g(t, .), i.e. the populations BEFORE collision.
 *
 * Layout: structure of arrays, g[i * cells + cell], cell = x + nx * (y + ny * z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_QMAX 27

/* Velocity-set identifiers (own numbering; the tests map them by name). */
enum {
    OR_D1Q3 = 0,
    OR_D2Q5 = 1,
    OR_D2Q5_DI = 2,
    OR_D3Q7 = 3,
    OR_D3Q9 = 4,
    OR_D3Q13 = 5,
    OR_D3Q19 = 6,
    OR_D3Q7_DI = 7,
    OR_NSETS = 8
};

/* Boundary handling. */
enum { OR_BC_PERIODIC = 0, OR_BC_OPEN_ZERO = 1, OR_BC_OPEN_SPONGE = 2, OR_BC_OPEN_GHOST = 3 };

typedef struct {
    int D, q;
    int mono;                  /* 1: monoatomic (Sec. 4 formulas), 0: polyatomic (Sec. 5) */
    double rho0, theta0, gamma;
    double a1, a2, b, c1, c2;  /* Sec. 5 general-equilibrium coefficients */
    int c[OR_QMAX][3];
    double f[OR_QMAX];         /* f*_i */
    double beta[OR_QMAX];      /* additional energies beta_i (0 for monoatomic) */
} or_set;

static int g_threads = 1;

void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int or_get_threads(void) { return g_threads; }

/* Monoatomic sets in general-form coefficients: eq. "equilibrium" (Sec. 4) expands to
 * a1 = 1/rho0, b = 1/theta0, a2 = -D/(2 theta0), c1 = 0, c2 = 1/theta0^2, beta = 0, and the
 * adiabatic exponent of a gas with M = D degrees of freedom is gamma = (M+2)/M (Sec. 5). */
static void mono_coeffs(or_set *s) {
    s->mono = 1;
    s->a1 = 1.0 / s->rho0;
    s->b = 1.0 / s->theta0;
    s->a2 = -(double)s->D / (2.0 * s->theta0);
    s->c1 = 0.0;
    s->c2 = 1.0 / (s->theta0 * s->theta0);
    s->gamma = ((double)s->D + 2.0) / (double)s->D;
    for (int i = 0; i < s->q; ++i) s->beta[i] = 0.0;
}

/* 3D monoatomic family on the D3Q27 stencil (Sec. 8.3.1): the weight of a velocity depends on
 * its shell (0: rest, 1: face, 2: edge, 3: corner) through rho0, theta0 and alpha.  Velocities
 * whose weight vanishes are dropped, which yields D3Q7, D3Q9, D3Q13 and D3Q19. */
static double family3d_weight(int shell, double rho0, double th, double alpha) {
    switch (shell) {
    case 0: return 0.5 * rho0 * th * (15.0 * th - 9.0) + rho0 - 8.0 * alpha;
    case 1: return 0.5 * rho0 * th * (2.0 - 5.0 * th) + 4.0 * alpha;
    case 2: return 0.125 * rho0 * th * (5.0 * th - 1.0) - 2.0 * alpha;
    default: return alpha;
    }
}

static void build_family3d(or_set *s, double theta0, double alpha) {
    s->D = 3;
    s->rho0 = 1.0;
    s->theta0 = theta0;
    s->q = 0;
    /* enumerate shells in order rest, faces, edges, corners */
    for (int shell = 0; shell <= 3; ++shell) {
        for (int z = -1; z <= 1; ++z)
            for (int y = -1; y <= 1; ++y)
                for (int x = -1; x <= 1; ++x) {
                    int sh = abs(x) + abs(y) + abs(z);
                    if (sh != shell) continue;
                    double w = family3d_weight(shell, s->rho0, theta0, alpha);
                    if (fabs(w) < 1e-14) continue;
                    s->c[s->q][0] = x;
                    s->c[s->q][1] = y;
                    s->c[s->q][2] = z;
                    s->f[s->q] = w;
                    s->q++;
                }
    }
    mono_coeffs(s);
}

static void set_vel(or_set *s, int i, int x, int y, int z) {
    s->c[i][0] = x;
    s->c[i][1] = y;
    s->c[i][2] = z;
}

/* Builds velocity set `id`.  Returns 0 on success, -1 for an unknown id. */
static int build_set(int id, or_set *s) {
    memset(s, 0, sizeof(*s));
    switch (id) {
    case OR_D1Q3: /* Sec. 8.1: rho0 = 1, theta0 = 1/3 */
        s->D = 1; s->q = 3; s->rho0 = 1.0; s->theta0 = 1.0 / 3.0;
        set_vel(s, 0, 0, 0, 0); set_vel(s, 1, -1, 0, 0); set_vel(s, 2, 1, 0, 0);
        s->f[0] = 2.0 / 3.0; s->f[1] = 1.0 / 6.0; s->f[2] = 1.0 / 6.0;
        mono_coeffs(s);
        return 0;
    case OR_D2Q5: /* Sec. 8.2.1: rho0 = 1, theta0 = 1/4 */
        s->D = 2; s->q = 5; s->rho0 = 1.0; s->theta0 = 0.25;
        set_vel(s, 0, 0, 0, 0); set_vel(s, 1, -1, 0, 0); set_vel(s, 2, 1, 0, 0);
        set_vel(s, 3, 0, -1, 0); set_vel(s, 4, 0, 1, 0);
        s->f[0] = 0.5;
        for (int i = 1; i < 5; ++i) s->f[i] = 0.125;
        mono_coeffs(s);
        return 0;
    case OR_D2Q5_DI: /* Sec. 8.2.2: rho0 = 20/3, theta0 = 3/10, diatomic (M = 2D-1 = 3) */
        s->D = 2; s->q = 5; s->rho0 = 20.0 / 3.0; s->theta0 = 0.3;
        set_vel(s, 0, 0, 0, 0); set_vel(s, 1, -1, 0, 0); set_vel(s, 2, 1, 0, 0);
        set_vel(s, 3, 0, -1, 0); set_vel(s, 4, 0, 1, 0);
        s->f[0] = 8.0 / 3.0; s->beta[0] = 0.0;
        for (int i = 1; i < 5; ++i) { s->f[i] = 1.0; s->beta[i] = 0.5; }
        s->mono = 0;
        s->a1 = 1.0 / s->rho0; s->a2 = -5.0; s->b = 1.0 / s->theta0; s->c1 = 0.0;
        s->c2 = 5.0 / s->theta0;
        s->gamma = (3.0 + 2.0) / 3.0;
        return 0;
    case OR_D3Q7: build_family3d(s, 0.2, 0.0); return 0;           /* theta0 = 1/5, alpha = 0 */
    case OR_D3Q9: build_family3d(s, 0.6, 3.0 / 40.0); return 0;    /* theta0 = 3/5, alpha = 3/40 */
    case OR_D3Q13: build_family3d(s, 0.4, 0.0); return 0;          /* theta0 = 2/5, alpha = 0 */
    case OR_D3Q19: build_family3d(s, 0.3, 0.0); return 0;          /* theta0 = 3/10, alpha = 0 */
    case OR_D3Q7_DI: { /* Sec. 8.3.2: f1 = 5/42 family member, diatomic (M = 2D-1 = 5) */
        const double f1 = 5.0 / 42.0;
        s->D = 3; s->q = 7; s->rho0 = 42.0 / 5.0 * f1; s->theta0 = 5.0 / 21.0;
        set_vel(s, 0, 0, 0, 0);
        set_vel(s, 1, -1, 0, 0); set_vel(s, 2, 1, 0, 0);
        set_vel(s, 3, 0, -1, 0); set_vel(s, 4, 0, 1, 0);
        set_vel(s, 5, 0, 0, -1); set_vel(s, 6, 0, 0, 1);
        s->f[0] = 12.0 / 5.0 * f1; s->beta[0] = 0.0;
        for (int i = 1; i < 7; ++i) { s->f[i] = f1; s->beta[i] = 2.0 / 3.0; }
        s->mono = 0;
        s->a1 = 1.0 / s->rho0; s->a2 = -21.0 / 2.0; s->b = 21.0 / 5.0; s->c1 = 0.0;
        s->c2 = 147.0 / 5.0;
        s->gamma = (5.0 + 2.0) / 5.0;
        return 0;
    }
    default:
        return -1;
    }
}

/* Exported description of a set.  consts = {rho0, theta0, gamma, a1, a2, b, c1, c2, mono}. */
int or_set_info(int id, int *D, int *q, double *consts, int *c, double *f, double *beta) {
    or_set s;
    if (build_set(id, &s) != 0) return -1;
    *D = s.D;
    *q = s.q;
    consts[0] = s.rho0; consts[1] = s.theta0; consts[2] = s.gamma;
    consts[3] = s.a1; consts[4] = s.a2; consts[5] = s.b; consts[6] = s.c1; consts[7] = s.c2;
    consts[8] = (double)s.mono;
    for (int i = 0; i < s.q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = s.c[i][a];
        f[i] = s.f[i];
        beta[i] = s.beta[i];
    }
    return 0;
}

/* ---- per-cell building blocks ------------------------------------------------------------ */

static int csq(const or_set *s, int i) {
    return s->c[i][0] * s->c[i][0] + s->c[i][1] * s->c[i][1] + s->c[i][2] * s->c[i][2];
}

/* Discrete moments of one cell's populations.
 * rho' = <g>_S, u' = <v g>_S / rho0 (Sec. 4), and
 *   monoatomic:  theta' = ( <|v|^2 g>_S / D - theta0 <g>_S ) / rho0         (Sec. 4)
 *   polyatomic:  theta' = ( (gamma-1) <(|v|^2 + beta) g / 2>_S - theta0 rho' ) / rho0  (Sec. 5) */
static void cell_moments(const or_set *s, const double *gc, double *rho, double u[3], double *theta) {
    double r = 0.0, j[3] = {0.0, 0.0, 0.0}, e2 = 0.0, en = 0.0;
    for (int i = 0; i < s->q; ++i) {
        r += gc[i];
        for (int a = 0; a < 3; ++a) j[a] += s->c[i][a] * gc[i];
        e2 += csq(s, i) * gc[i];
        en += 0.5 * (csq(s, i) + s->beta[i]) * gc[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = j[a] / s->rho0;
    if (s->mono)
        *theta = (e2 / s->D - s->theta0 * r) / s->rho0;
    else
        *theta = ((s->gamma - 1.0) * en - s->theta0 * r) / s->rho0;
}

/* Equilibrium of one cell.
 *   monoatomic (Sec. 4, eq. "equilibrium"):
 *     g_i^eq = ( rho'/rho0 + c_i.u'/theta0 + theta' (|c_i|^2/(2 theta0^2) - D/(2 theta0)) ) f*_i
 *   polyatomic (Sec. 5):
 *     g_i^eq = ( a1 rho' + a2 theta' + b c_i.u' + |c_i|^2 (c1 rho' + c2 theta') / 2 ) f*_i */
static void cell_equilibrium(const or_set *s, double rho, const double u[3], double theta, double *geq) {
    for (int i = 0; i < s->q; ++i) {
        double cu = s->c[i][0] * u[0] + s->c[i][1] * u[1] + s->c[i][2] * u[2];
        double c2 = (double)csq(s, i);
        double bracket;
        if (s->mono)
            bracket = rho / s->rho0 + cu / s->theta0 +
                      theta * (c2 / (2.0 * s->theta0 * s->theta0) - s->D / (2.0 * s->theta0));
        else
            bracket = s->a1 * rho + s->a2 * theta + s->b * cu + 0.5 * c2 * (s->c1 * rho + s->c2 * theta);
        geq[i] = bracket * s->f[i];
    }
}

/* ---- field-level entry points ------------------------------------------------------------ */

/* Initial condition of Sec. 7: g_i(0, x) = g_i^eq(rho'(0,x), u'(0,x), theta'(0,x)). */
int or_equilibrium_fields(int id, int64_t cells, const double *rho, const double *u, const double *theta,
                          double *g) {
    or_set s;
    if (build_set(id, &s) != 0) return -1;
    for (int64_t x = 0; x < cells; ++x) {
        double uu[3] = {0.0, 0.0, 0.0}, geq[OR_QMAX];
        for (int a = 0; a < s.D; ++a) uu[a] = u[a * cells + x];
        cell_equilibrium(&s, rho[x], uu, theta[x], geq);
        for (int i = 0; i < s.q; ++i) g[i * cells + x] = geq[i];
    }
    return 0;
}

/* Per-cell macroscopic fluctuations (rho', u'[D], theta') of a population field. */
int or_moments_fields(int id, int64_t cells, const double *g, double *rho, double *u, double *theta) {
    or_set s;
    if (build_set(id, &s) != 0) return -1;
    for (int64_t x = 0; x < cells; ++x) {
        double gc[OR_QMAX], r, uu[3], th;
        for (int i = 0; i < s.q; ++i) gc[i] = g[i * cells + x];
        cell_moments(&s, gc, &r, uu, &th);
        rho[x] = r;
        for (int a = 0; a < s.D; ++a) u[a * cells + x] = uu[a];
        theta[x] = th;
    }
    return 0;
}

/* BGK relaxation alone (no streaming): gout = (1 - 1/tau) g + (1/tau) g^eq(g), per cell.
 * This maps the paper's pre-collision state to the post-collision state. */
int or_collide(int id, int64_t cells, double tau, const double *g, double *gout) {
    or_set s;
    if (build_set(id, &s) != 0) return -1;
    for (int64_t x = 0; x < cells; ++x) {
        double gc[OR_QMAX], geq[OR_QMAX], r, uu[3], th;
        for (int i = 0; i < s.q; ++i) gc[i] = g[i * cells + x];
        cell_moments(&s, gc, &r, uu, &th);
        cell_equilibrium(&s, r, uu, th, geq);
        for (int i = 0; i < s.q; ++i) gout[i * cells + x] = (1.0 - 1.0 / tau) * gc[i] + (1.0 / tau) * geq[i];
    }
    return 0;
}

/* Sponge damping factor of a frame cell: sigma(d) = smax (d / W)^2, d = how many cells deep the
 * cell lies inside the W-cell frame (1 at the innermost frame cell, W at the outer edge), taken as
 * the maximum over the non-trivial axes; d = 0 (no damping) in the interior. */
static double sponge_sigma(int64_t x, int64_t y, int64_t z, const int64_t n[3], int D, int w, double smax) {
    int64_t p[3] = {x, y, z};
    int64_t d = 0;
    for (int a = 0; a < D; ++a) {
        int64_t lo = w - p[a];                  /* depth from the low side  */
        int64_t hi = p[a] - (n[a] - 1 - w);     /* depth from the high side */
        if (lo > d) d = lo;
        if (hi > d) d = hi;
    }
    if (d <= 0) return 0.0;
    double r = (double)d / (double)w;
    return smax * r * r;
}

/* n time steps of the LBE update scheme (Sec. 6) in push form.
 *
 * bc = OR_BC_PERIODIC: x + c_i wraps around every axis (Sec. 2.2 restricts the paper to periodic
 *      domains).
 * bc = OR_BC_OPEN_ZERO: a population pushed across the outer edge leaves the domain, and a
 *      population that would enter from outside is the rest state, g = 0.
 * bc = OR_BC_OPEN_SPONGE: as OPEN_ZERO, and the post-collision populations of the cells in a
 *      frame of width sponge_w are multiplied by 1 - sigma(d) (sponge_sigma above).
 * bc = OR_BC_OPEN_GHOST: as OPEN_ZERO, except that on a 2D grid with the five-velocity stencil
 *      the entering population of each edge cell is read from `ghost` (one step only):
 *      ghost[0*L + y] for x = 0 (entering c = (+1,0)), ghost[1*L + y] for x = nx-1 (c = (-1,0)),
 *      ghost[2*L + x] for y = 0 (c = (0,+1)), ghost[3*L + x] for y = ny-1 (c = (0,-1)),
 *      with L = max(nx, ny).
 * Returns 0 on success, a negative value on a bad argument. */
int or_step(int id, int64_t nx, int64_t ny, int64_t nz, double tau, int bc, int sponge_w, double sponge_smax,
            double *g, int64_t nsteps, const double *ghost) {
    or_set s;
    if (build_set(id, &s) != 0) return -1;
    if (nx < 1 || ny < 1 || nz < 1) return -2;
    if (s.D < 3 && nz != 1) return -2;
    if (s.D < 2 && ny != 1) return -2;
    if (bc == OR_BC_OPEN_GHOST && (s.D != 2 || s.q != 5 || ghost == NULL || nsteps != 1)) return -3;
    if (bc == OR_BC_OPEN_SPONGE && (sponge_w < 1)) return -4;
    const int64_t cells = nx * ny * nz;
    const int64_t n[3] = {nx, ny, nz};
    double *gn = (double *)malloc(sizeof(double) * (size_t)s.q * (size_t)cells);
    if (!gn) return -5;

    for (int64_t step = 0; step < nsteps; ++step) {
        if (bc != OR_BC_PERIODIC) memset(gn, 0, sizeof(double) * (size_t)s.q * (size_t)cells);
#pragma omp parallel for num_threads(g_threads) schedule(static)
        for (int64_t cell = 0; cell < cells; ++cell) {
            int64_t x = cell % nx, y = (cell / nx) % ny, z = cell / (nx * ny);
            double gc[OR_QMAX], geq[OR_QMAX], r, uu[3], th;
            for (int i = 0; i < s.q; ++i) gc[i] = g[i * cells + cell];
            cell_moments(&s, gc, &r, uu, &th);
            cell_equilibrium(&s, r, uu, th, geq);
            double damp = 1.0;
            if (bc == OR_BC_OPEN_SPONGE) damp = 1.0 - sponge_sigma(x, y, z, n, s.D, sponge_w, sponge_smax);
            for (int i = 0; i < s.q; ++i) {
                double post = (1.0 - 1.0 / tau) * gc[i] + (1.0 / tau) * geq[i];
                post *= damp;
                int64_t t[3] = {x + s.c[i][0], y + s.c[i][1], z + s.c[i][2]};
                int inside = 1;
                for (int a = 0; a < 3; ++a) {
                    if (t[a] < 0 || t[a] >= n[a]) {
                        if (bc == OR_BC_PERIODIC)
                            t[a] = (t[a] + n[a]) % n[a];
                        else
                            inside = 0;
                    }
                }
                if (inside) gn[i * cells + t[0] + nx * (t[1] + ny * t[2])] = post;
            }
        }
        if (bc == OR_BC_OPEN_GHOST) {
            const int64_t L = nx > ny ? nx : ny;
            for (int i = 0; i < s.q; ++i) {
                int cx = s.c[i][0], cy = s.c[i][1];
                if (cx == 1 && cy == 0)
                    for (int64_t y = 0; y < ny; ++y) gn[i * cells + 0 + nx * y] = ghost[0 * L + y];
                if (cx == -1 && cy == 0)
                    for (int64_t y = 0; y < ny; ++y) gn[i * cells + (nx - 1) + nx * y] = ghost[1 * L + y];
                if (cx == 0 && cy == 1)
                    for (int64_t x = 0; x < nx; ++x) gn[i * cells + x] = ghost[2 * L + x];
                if (cx == 0 && cy == -1)
                    for (int64_t x = 0; x < nx; ++x) gn[i * cells + x + nx * (ny - 1)] = ghost[3 * L + x];
            }
        }
        memcpy(g, gn, sizeof(double) * (size_t)s.q * (size_t)cells);
    }
    free(gn);
    return 0;
}

/* Post-collision state of a field: (1 - 1/tau) g + (1/tau) g^eq(g) per cell, multiplied inside a
 * sponge frame (bc = OR_BC_OPEN_SPONGE) by the same 1 - sigma(d) that or_step applies before
 * streaming.  This is the state that one push step streams, i.e. the populations "in flight". */
int or_post_state(int id, int64_t nx, int64_t ny, int64_t nz, double tau, int bc, int sponge_w, double sponge_smax,
                  const double *g, double *out) {
    or_set s;
    if (build_set(id, &s) != 0) return -1;
    const int64_t cells = nx * ny * nz;
    const int64_t n[3] = {nx, ny, nz};
    int rc = or_collide(id, cells, tau, g, out);
    if (rc != 0) return rc;
    if (bc == OR_BC_OPEN_SPONGE) {
        for (int64_t cell = 0; cell < cells; ++cell) {
            int64_t x = cell % nx, y = (cell / nx) % ny, z = cell / (nx * ny);
            double damp = 1.0 - sponge_sigma(x, y, z, n, s.D, sponge_w, sponge_smax);
            for (int i = 0; i < s.q; ++i) out[i * cells + cell] *= damp;
        }
    }
    return 0;
}

/* Global sums of a population field, in FP64 with Kahan compensation:
 *   out[0]       = sum_x rho'                       (zeroth moment, conserved on periodic grids)
 *   out[1..D]    = sum_x <c_a g>_S = rho0 sum_x u'_a (momentum, conserved)
 *   out[D+1]     = sum_x <(|c|^2 + beta) g / 2>_S   (energy moment of Sec. 5, conserved)
 *   out[D+2]     = sum_x sum_i g_i^2 / f*_i          (weighted energy; the diagonal weight
 *                                                     A0 ~ diag(1/f*) of Sec. 8.3.1)
 *   out[D+3]     = number of non-finite populations */
int or_reduce(int id, int64_t cells, const double *g, double *out) {
    or_set s;
    if (build_set(id, &s) != 0) return -1;
    const int nout = s.D + 4;
    double sum[8] = {0}, comp[8] = {0};
    int64_t nonfinite = 0;
    for (int64_t x = 0; x < cells; ++x) {
        double term[8] = {0};
        for (int i = 0; i < s.q; ++i) {
            double v = g[i * cells + x];
            if (!isfinite(v)) { nonfinite++; continue; }
            term[0] += v;
            for (int a = 0; a < s.D; ++a) term[1 + a] += s.c[i][a] * v;
            term[s.D + 1] += 0.5 * (csq(&s, i) + s.beta[i]) * v;
            term[s.D + 2] += v * v / s.f[i];
        }
        for (int k = 0; k < s.D + 3; ++k) {
            double yk = term[k] - comp[k];
            double tk = sum[k] + yk;
            comp[k] = (tk - sum[k]) - yk;
            sum[k] = tk;
        }
    }
    for (int k = 0; k < s.D + 3; ++k) out[k] = sum[k];
    out[nout - 1] = (double)nonfinite;
    return 0;
}
