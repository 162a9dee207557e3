/*
 * bsq_oracle.c -- plain, slow FP64 CPU oracle for the adaptive-AB3 extended
 * Boussinesq time step (Tavakkol, Son & Lynett, arXiv 1909.04153).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it; the library never does.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Everything is double precision, single threaded, written as plain loops in
 * the order the paper states the method.  Build with -O2 -ffp-contract=off.
 *
 * What each part follows:
 *   model ............ Eqs. 1-5 (Sec. 2) in the Wei-Kirby form Eqs. 6-15 (Sec. 3.1)
 *   hyperbolic part .. Kurganov-Petrova 2007 central-upwind scheme, cited in Sec. 3
 *                      and 3.1 (bed at cell corners, generalized minmod,
 *                      positivity fix, desingularised velocities, well-balanced
 *                      bed source); minmod dissipation is the breaking model (Sec. 3.4)
 *   dispersive part .. second-order central differences (Sec. 3.1)
 *   implicit part .... tridiagonal systems Eqs. 19-21, plain Thomas per line
 *   time step ........ CFL of Eq. 22 (Sec. 3.2.2), lazy EMA of Eq. 47 (Sec. 3.2.2.4)
 *   AB3 weights ...... Eq. 42 (= Eq. 30), Euler start (Sec. 3.2.1)
 *   time derivative . variable-step differences Eqs. 44-46 plugged into Eq. 43
 *   boundaries ....... two ghost layers (Sec. 3.3): wall, sponge, wave maker
 *   wet/dry .......... no flags; every cell is wet, h >= 0 (Sec. 3.5)
 *
 * Readings of silent or garbled passages (the same readings the library takes):
 *   - F's third component is PQ/(w-b) and S carries g (Eq. 5 is garbled).
 *   - Eq. 15 defines G*(P) (its right-hand side uses P).
 *   - eta = h - d with h = max(w-b,0), d = max(w_s-b,0).
 *   - Euler start: steps 0 and 1 use w += dt E, U* += dt F + (F*^n - F*^{n-1}),
 *     with the F* term zero on step 0.
 *   - The positivity of h under AB3 is enforced by clamping w >= b after the
 *     update; the clamps are counted.
 *   - Tridiagonal boundary rows: wall = odd mirror of the normal flux;
 *     wave maker = prescribed ghost value moved to the right-hand side.
 *   - Sponge: gamma(r) = 1/2 + 1/2 cos(pi (1 - r/L)), r from the outer edge,
 *     product over sponge sides; eta, P, Q scaled by gamma once per step,
 *     Q right after its solve, eta and P after the P solve.
 *   - cross_mode 1 (default): the y-lines are solved first and F* is taken
 *     at the new level from Q^{n+1}; cross_mode 0 extrapolates F* and G* as
 *     printed in Eqs. 17-18 / 43.
 *   - Wave maker: linear components eta = r(t) sum a cos(k.x - w t + phi),
 *     flux = (omega/k) eta along the direction of travel,
 *     r(t) = tanh(3 t / ramp_time), k from the linearised dispersion relation.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

#define ORC_WALL 0
#define ORC_SPONGE 1
#define ORC_MAKER 2

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_UNSTABLE 5

typedef struct {
    int nx, ny;
    double dx, dy;
    double g;          /* gravity */
    double Bd;         /* dispersion coefficient B of Eqs. 2-3 */
    double cfl;        /* target CFL of Eq. 22 */
    double ema_alpha;  /* alpha of Eq. 47 */
    double dt_init;    /* <= 0: from Eq. 22 */
    double dt_min;
    double dt_max;     /* <= 0: none */
    double friction;   /* quadratic friction factor f */
    double theta;      /* generalized minmod parameter (1 = minmod) */
    double eps;        /* desingularisation epsilon, <= 0: max(dx,dy)^4 */
    double w_s;        /* still water elevation from the datum */
    double ramp_time;  /* wave maker ramp (s), <= 0: none */
    int cross_mode;    /* 0: F*, G* both extrapolated (Eq. 43); 1: Q first, F* at the new level */
    int bc[4];         /* W, E, S, N */
    double sponge_width[4];
} orc_params;

typedef struct {
    orc_params p;
    int nx, ny, sx, sy;        /* sx = nx+4, sy = ny+4 */
    int cx;                    /* corner row length nx+5 */
    double *w, *P, *Q;         /* cells with 2 ghost layers */
    double *corner;            /* bed at corners, extended by mirroring, (nx+5)(ny+5) */
    double *bxf;               /* bed at x-faces (nx+5) x (ny+4) */
    double *byf;               /* bed at y-faces (nx+4) x (ny+5) */
    double *b, *d, *ddx, *ddy; /* cell centre bed, still depth, its gradients */
    double *eta;               /* scratch: eta of current state */
    double *sponge;            /* per-cell sponge factor (1 outside bands) */
    double *hist[5][3];        /* E, F, G, F*, G* : ring of 3 time levels */
    double *Hx[3], *Hy[3];     /* face fluxes */
    double *Us, *Vs;           /* U*, V* of Eqs. 9-10 */
    double *ta, *tb, *tc, *tr, *tx; /* line work arrays */
    int ncomp;
    double *amp, *om, *kw, *ph, *dir;
    long long n;               /* steps taken */
    int slot;                  /* ring slot of level n */
    double t, dtm1, dtm2;
    double last_dt, last_rate;
    double beta[3], gam[3];
    long long clamps;
} orc_dom;

/* ------------------------------------------------------------------ */
/* indexing                                                            */

static inline int CI(const orc_dom *D, int i, int j) { return (i + 2) + (j + 2) * D->sx; }
static inline int KI(const orc_dom *D, int i, int j) { return (i + 2) + (j + 2) * D->cx; }
static inline int XF(const orc_dom *D, int i, int j) { return (i + 2) + (j + 2) * (D->nx + 5); }
static inline int YF(const orc_dom *D, int i, int j) { return (i + 2) + (j + 2) * D->sx; }

/* ------------------------------------------------------------------ */
/* time-stepping coefficients                                          */

/* Eq. 42 (= Eq. 30): weights of X_t^n, X_t^{n-1}, X_t^{n-2}, including dt_n/6.
 * a = dt_n, b = dt_{n-1}, c = dt_{n-2}. */
void orc_ab3_weights(double a, double b, double c, double out[3])
{
    out[0] = a / 6.0 * (a / b * (2.0 * a + 6.0 * b + 3.0 * c) / (b + c) + 6.0);
    out[1] = -a / 6.0 * (a / b * (2.0 * a + 3.0 * b + 3.0 * c) / c);
    out[2] = a / 6.0 * (a / c * (2.0 * a + 3.0 * b) / (b + c));
}

/* Eqs. 35, 38, 41 (= 44-46): row r gives Y_t at level n-r as weights of
 * Y^n, Y^{n-1}, Y^{n-2}.  b = dt_{n-1}, c = dt_{n-2}.  out is row-major 3x3. */
void orc_fd_weights(double b, double c, double out[9])
{
    /* Eq. 35: backward, at t_n */
    out[0] = (2.0 * b + c) / (b * (b + c));
    out[1] = -(b + c) / (b * c);
    out[2] = b / (c * (b + c));
    /* Eq. 38: central, at t_{n-1} */
    out[3] = c / (b * (b + c));
    out[4] = (b - c) / (b * c);
    out[5] = -b / (c * (b + c));
    /* Eq. 41: forward, at t_{n-2} */
    out[6] = -c / (b * (b + c));
    out[7] = (b + c) / (b * c);
    out[8] = -(b + 2.0 * c) / (c * (b + c));
}

/* Eq. 43 with Eqs. 44-46 plugged in: the weights of F*^n, F*^{n-1}, F*^{n-2}
 * in the U* update, i.e. sum_k beta_k (F*^{n-k})_t. */
void orc_dstar_weights(double a, double b, double c, double out[3])
{
    double beta[3], D[9];
    orc_ab3_weights(a, b, c, beta);
    orc_fd_weights(b, c, D);
    for (int m = 0; m < 3; m++)
        out[m] = beta[0] * D[0 * 3 + m] + beta[1] * D[1 * 3 + m] + beta[2] * D[2 * 3 + m];
}

/* ------------------------------------------------------------------ */
/* small helpers                                                       */

static double minmod3(double a, double b, double c)
{
    if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
    if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
    return 0.0;
}

/* generalized minmod slope of q across (qm, q0, qp), per cell width */
static double gslope(double qm, double q0, double qp, double theta)
{
    return minmod3(theta * (q0 - qm), 0.5 * (qp - qm), theta * (qp - q0));
}

/* desingularised velocity of KP07: sqrt(2) h m / sqrt(h^4 + max(h^4, eps)) */
static double desing(double h, double m, double eps)
{
    double h4 = h * h * h * h;
    return sqrt(2.0) * h * m / sqrt(h4 + fmax(h4, eps));
}

/* Thomas algorithm for a_i x_{i-1} + b_i x_i + c_i x_{i+1} = r_i, a_0 = c_{n-1} = 0.
 * Textbook elimination without pivoting (the systems are diagonally dominant). */
void orc_thomas(int n, const double *a, const double *b, const double *c,
                const double *r, double *x)
{
    double *cp = (double *)malloc(sizeof(double) * (size_t)n);
    double *dp = (double *)malloc(sizeof(double) * (size_t)n);
    cp[0] = c[0] / b[0];
    dp[0] = r[0] / b[0];
    for (int i = 1; i < n; i++) {
        double den = b[i] - a[i] * cp[i - 1];
        cp[i] = c[i] / den;
        dp[i] = (r[i] - a[i] * dp[i - 1]) / den;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; i--) x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp);
    free(dp);
}

/* Linearised dispersion relation of Eqs. 1-3 on a flat bed of depth d:
 * omega^2 = g d k^2 (1 + B (kd)^2) / (1 + (B + 1/3)(kd)^2).  Newton for k. */
double orc_wavenumber(double omega, double d, double g, double Bd)
{
    if (omega <= 0.0 || d <= 0.0) return 0.0;
    double k = omega / sqrt(g * d);
    for (int it = 0; it < 100; it++) {
        double kd = k * d;
        double num = 1.0 + Bd * kd * kd, den = 1.0 + (Bd + 1.0 / 3.0) * kd * kd;
        double f = g * d * k * k * num / den - omega * omega;
        /* derivative of g d k^2 num/den in k */
        double dnum = 2.0 * Bd * kd * d, dden = 2.0 * (Bd + 1.0 / 3.0) * kd * d;
        double df = g * d * (2.0 * k * num / den + k * k * (dnum * den - num * dden) / (den * den));
        double step = f / df;
        k -= step;
        if (fabs(step) <= 1e-15 * fabs(k)) break;
    }
    return k;
}

/* ------------------------------------------------------------------ */
/* creation                                                            */

static double *zalloc(size_t n) { return (double *)calloc(n, sizeof(double)); }

void orc_destroy(orc_dom *D)
{
    if (!D) return;
    free(D->w); free(D->P); free(D->Q);
    free(D->corner); free(D->bxf); free(D->byf);
    free(D->b); free(D->d); free(D->ddx); free(D->ddy);
    free(D->eta); free(D->sponge);
    for (int f = 0; f < 5; f++)
        for (int s = 0; s < 3; s++) free(D->hist[f][s]);
    for (int c = 0; c < 3; c++) { free(D->Hx[c]); free(D->Hy[c]); }
    free(D->Us); free(D->Vs);
    free(D->ta); free(D->tb); free(D->tc); free(D->tr); free(D->tx);
    free(D->amp); free(D->om); free(D->kw); free(D->ph); free(D->dir);
    free(D);
}

static double sponge_gamma(double r, double L)
{
    if (L <= 0.0 || r >= L) return 1.0;
    if (r < 0.0) r = 0.0;
    return 0.5 + 0.5 * cos(ORC_PI * (1.0 - r / L));
}

/* bed_corners: (nx+1)(ny+1) row-major, x fastest, corner (i,j) at (i dx, j dy).
 * comps: ncomp rows of (amplitude m, frequency Hz, phase rad, direction rad).
 * eta0, P0, Q0: nx*ny row-major or NULL (zero). */
orc_dom *orc_create(const orc_params *prm, const double *bed_corners,
                    int ncomp, const double *comps,
                    const double *eta0, const double *P0, const double *Q0)
{
    if (!prm || prm->nx < 3 || prm->ny < 3 || !(prm->dx > 0) || !(prm->dy > 0) || !bed_corners)
        return NULL;
    orc_dom *D = (orc_dom *)calloc(1, sizeof(orc_dom));
    if (!D) return NULL;
    D->p = *prm;
    if (D->p.eps <= 0.0) {
        double m = fmax(D->p.dx, D->p.dy);
        D->p.eps = m * m * m * m;
    }
    if (D->p.theta <= 0.0) D->p.theta = 1.0;
    int nx = prm->nx, ny = prm->ny;
    D->nx = nx; D->ny = ny; D->sx = nx + 4; D->sy = ny + 4; D->cx = nx + 5;
    size_t nc = (size_t)D->sx * D->sy;
    D->w = zalloc(nc); D->P = zalloc(nc); D->Q = zalloc(nc);
    D->corner = zalloc((size_t)(nx + 5) * (ny + 5));
    D->bxf = zalloc((size_t)(nx + 5) * (ny + 4));
    D->byf = zalloc((size_t)(nx + 4) * (ny + 5));
    D->b = zalloc(nc); D->d = zalloc(nc); D->ddx = zalloc(nc); D->ddy = zalloc(nc);
    D->eta = zalloc(nc); D->sponge = zalloc(nc);
    for (int f = 0; f < 5; f++)
        for (int s = 0; s < 3; s++) D->hist[f][s] = zalloc(nc);
    for (int c = 0; c < 3; c++) {
        D->Hx[c] = zalloc((size_t)(nx + 5) * (ny + 4));
        D->Hy[c] = zalloc((size_t)(nx + 4) * (ny + 5));
    }
    D->Us = zalloc(nc); D->Vs = zalloc(nc);
    int L = (nx > ny ? nx : ny) + 4;
    D->ta = zalloc(L); D->tb = zalloc(L); D->tc = zalloc(L); D->tr = zalloc(L); D->tx = zalloc(L);
    D->ncomp = ncomp > 0 ? ncomp : 0;
    int nk = D->ncomp > 0 ? D->ncomp : 1;
    D->amp = zalloc(nk); D->om = zalloc(nk); D->kw = zalloc(nk); D->ph = zalloc(nk); D->dir = zalloc(nk);
    if (!D->w || !D->tx || !D->dir) { orc_destroy(D); return NULL; }

    /* bed at corners, extended two layers outward by mirroring about the edge */
    for (int j = -2; j <= ny + 2; j++) {
        int js = j < 0 ? -j : (j > ny ? 2 * ny - j : j);
        for (int i = -2; i <= nx + 2; i++) {
            int is = i < 0 ? -i : (i > nx ? 2 * nx - i : i);
            D->corner[KI(D, i, j)] = bed_corners[is + js * (nx + 1)];
        }
    }
    /* KP07: face value = mean of its two corners; centre value = mean of 4 faces */
    for (int j = -2; j <= ny + 1; j++)
        for (int i = -2; i <= nx + 2; i++)
            D->bxf[XF(D, i, j)] = 0.5 * (D->corner[KI(D, i, j)] + D->corner[KI(D, i, j + 1)]);
    for (int j = -2; j <= ny + 2; j++)
        for (int i = -2; i <= nx + 1; i++)
            D->byf[YF(D, i, j)] = 0.5 * (D->corner[KI(D, i, j)] + D->corner[KI(D, i + 1, j)]);
    for (int j = -2; j <= ny + 1; j++)
        for (int i = -2; i <= nx + 1; i++) {
            double bc = 0.25 * (D->bxf[XF(D, i, j)] + D->bxf[XF(D, i + 1, j)] +
                                D->byf[YF(D, i, j)] + D->byf[YF(D, i, j + 1)]);
            D->b[CI(D, i, j)] = bc;
            D->d[CI(D, i, j)] = fmax(D->p.w_s - bc, 0.0);
        }
    for (int j = -1; j <= ny; j++)
        for (int i = -1; i <= nx; i++) {
            D->ddx[CI(D, i, j)] = (D->d[CI(D, i + 1, j)] - D->d[CI(D, i - 1, j)]) / (2.0 * D->p.dx);
            D->ddy[CI(D, i, j)] = (D->d[CI(D, i, j + 1)] - D->d[CI(D, i, j - 1)]) / (2.0 * D->p.dy);
        }

    /* sponge factor per cell: product over sponge sides */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double gmm = 1.0;
            if (prm->bc[0] == ORC_SPONGE) gmm *= sponge_gamma((i + 0.5) * prm->dx, prm->sponge_width[0]);
            if (prm->bc[1] == ORC_SPONGE) gmm *= sponge_gamma((nx - i - 0.5) * prm->dx, prm->sponge_width[1]);
            if (prm->bc[2] == ORC_SPONGE) gmm *= sponge_gamma((j + 0.5) * prm->dy, prm->sponge_width[2]);
            if (prm->bc[3] == ORC_SPONGE) gmm *= sponge_gamma((ny - j - 0.5) * prm->dy, prm->sponge_width[3]);
            D->sponge[CI(D, i, j)] = gmm;
        }

    /* wave-maker components; k from the dispersion relation at the maker depth.
     * The maker depth is the still depth of the first maker side's ghost cells. */
    double dmk = 0.0;
    int found = 0;
    for (int s = 0; s < 4 && !found; s++) {
        if (prm->bc[s] != ORC_MAKER) continue;
        int i = s == 0 ? -1 : (s == 1 ? nx : nx / 2);
        int j = s == 2 ? -1 : (s == 3 ? ny : ny / 2);
        dmk = D->d[CI(D, i, j)];
        found = 1;
    }
    for (int k = 0; k < D->ncomp; k++) {
        D->amp[k] = comps[4 * k + 0];
        D->om[k] = 2.0 * ORC_PI * comps[4 * k + 1];
        D->ph[k] = comps[4 * k + 2];
        D->dir[k] = comps[4 * k + 3];
        D->kw[k] = orc_wavenumber(D->om[k], dmk, prm->g, prm->Bd);
    }

    /* initial state: h = max(d + eta, 0), w = b + h */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = CI(D, i, j), k = i + j * nx;
            double e = eta0 ? eta0[k] : 0.0;
            double h = fmax(D->d[c] + e, 0.0);
            D->w[c] = D->b[c] + h;
            D->P[c] = P0 ? P0[k] : 0.0;
            D->Q[c] = Q0 ? Q0[k] : 0.0;
        }
    D->n = 0; D->slot = 0; D->t = 0.0; D->dtm1 = 0.0; D->dtm2 = 0.0;
    return D;
}

/* ------------------------------------------------------------------ */
/* boundary conditions (Sec. 3.3)                                      */

/* linear wave-maker state at a point: eta, P, Q */
static void maker_state(const orc_dom *D, double x, double y, double t,
                        double *eta, double *P, double *Q)
{
    double r = D->p.ramp_time > 0.0 ? tanh(3.0 * t / D->p.ramp_time) : 1.0;
    double e = 0.0, p = 0.0, q = 0.0;
    for (int k = 0; k < D->ncomp; k++) {
        double kx = D->kw[k] * cos(D->dir[k]), ky = D->kw[k] * sin(D->dir[k]);
        double ek = D->amp[k] * cos(kx * x + ky * y - D->om[k] * t + D->ph[k]);
        double c = D->kw[k] > 0.0 ? D->om[k] / D->kw[k] : 0.0;
        e += ek;
        p += c * cos(D->dir[k]) * ek;
        q += c * sin(D->dir[k]) * ek;
    }
    *eta = r * e; *P = r * p; *Q = r * q;
}

static void set_maker_cell(orc_dom *D, int i, int j, double t)
{
    double e, p, q;
    maker_state(D, (i + 0.5) * D->p.dx, (j + 0.5) * D->p.dy, t, &e, &p, &q);
    int c = CI(D, i, j);
    double h = fmax(D->d[c] + e, 0.0);
    D->w[c] = D->b[c] + h;
    D->P[c] = p;
    D->Q[c] = q;
}

/* Fill the two ghost layers: first the W/E columns of the interior rows,
 * then the S/N rows over all columns (so corners come from the columns). */
void orc_fill_ghosts(orc_dom *D, double t)
{
    int nx = D->nx, ny = D->ny;
    for (int j = 0; j < ny; j++) {
        for (int g = 1; g <= 2; g++) {
            /* west: ghost -g mirrors interior g-1 */
            int gi = -g, si = g - 1;
            if (D->p.bc[0] == ORC_MAKER) set_maker_cell(D, gi, j, t);
            else {
                D->w[CI(D, gi, j)] = D->w[CI(D, si, j)];
                D->P[CI(D, gi, j)] = -D->P[CI(D, si, j)];
                D->Q[CI(D, gi, j)] = D->Q[CI(D, si, j)];
            }
            /* east: ghost nx-1+g mirrors nx-g */
            gi = nx - 1 + g; si = nx - g;
            if (D->p.bc[1] == ORC_MAKER) set_maker_cell(D, gi, j, t);
            else {
                D->w[CI(D, gi, j)] = D->w[CI(D, si, j)];
                D->P[CI(D, gi, j)] = -D->P[CI(D, si, j)];
                D->Q[CI(D, gi, j)] = D->Q[CI(D, si, j)];
            }
        }
    }
    for (int i = -2; i <= nx + 1; i++) {
        for (int g = 1; g <= 2; g++) {
            int gj = -g, sj = g - 1;
            if (D->p.bc[2] == ORC_MAKER) set_maker_cell(D, i, gj, t);
            else {
                D->w[CI(D, i, gj)] = D->w[CI(D, i, sj)];
                D->P[CI(D, i, gj)] = D->P[CI(D, i, sj)];
                D->Q[CI(D, i, gj)] = -D->Q[CI(D, i, sj)];
            }
            gj = ny - 1 + g; sj = ny - g;
            if (D->p.bc[3] == ORC_MAKER) set_maker_cell(D, i, gj, t);
            else {
                D->w[CI(D, i, gj)] = D->w[CI(D, i, sj)];
                D->P[CI(D, i, gj)] = D->P[CI(D, i, sj)];
                D->Q[CI(D, i, gj)] = -D->Q[CI(D, i, sj)];
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* right-hand side: E, F, G (Eqs. 11-13) and F*, G* (Eqs. 14-15)         */

/* KP07 face states of cell (i,j) in one direction.  dir 0: x (E/W faces),
 * dir 1: y (N/S faces).  Returns w at the low face and the high face after
 * the positivity correction, and the reconstructed P, Q there. */
static void reconstruct(const orc_dom *D, int i, int j, int dir,
                        double *wlo, double *whi, double *Plo, double *Phi,
                        double *Qlo, double *Qhi)
{
    int cm = dir == 0 ? CI(D, i - 1, j) : CI(D, i, j - 1);
    int c0 = CI(D, i, j);
    int cp = dir == 0 ? CI(D, i + 1, j) : CI(D, i, j + 1);
    double th = D->p.theta;
    double sw = gslope(D->w[cm], D->w[c0], D->w[cp], th);
    double sP = gslope(D->P[cm], D->P[c0], D->P[cp], th);
    double sQ = gslope(D->Q[cm], D->Q[c0], D->Q[cp], th);
    double blo = dir == 0 ? D->bxf[XF(D, i, j)] : D->byf[YF(D, i, j)];
    double bhi = dir == 0 ? D->bxf[XF(D, i + 1, j)] : D->byf[YF(D, i, j + 1)];
    double w0 = D->w[c0];
    double wh = w0 + 0.5 * sw, wl = w0 - 0.5 * sw;
    /* positivity: keep the face water level above the face bed */
    if (wh < bhi) { wh = bhi; wl = 2.0 * w0 - bhi; }
    else if (wl < blo) { wl = blo; wh = 2.0 * w0 - blo; }
    *wlo = wl; *whi = wh;
    *Plo = D->P[c0] - 0.5 * sP; *Phi = D->P[c0] + 0.5 * sP;
    *Qlo = D->Q[c0] - 0.5 * sQ; *Qhi = D->Q[c0] + 0.5 * sQ;
}

/* central-upwind numerical flux across one face (Eq. 5 fluxes, KP07 form).
 * dir 0: x-face (normal discharge P), dir 1: y-face (normal discharge Q).
 * Left/right states are (w - b_face, P, Q) on each side. */
static void cu_flux(const orc_dom *D, int dir, double bface,
                    double wL, double PL, double QL, double wR, double PR, double QR,
                    double H[3])
{
    double g = D->p.g, eps = D->p.eps;
    double hL = fmax(wL - bface, 0.0), hR = fmax(wR - bface, 0.0);
    double uL = desing(hL, PL, eps), vL = desing(hL, QL, eps);
    double uR = desing(hR, PR, eps), vR = desing(hR, QR, eps);
    /* discharges recomputed from the desingularised velocities */
    double pL = hL * uL, qL = hL * vL, pR = hR * uR, qR = hR * vR;
    double cL = sqrt(g * hL), cR = sqrt(g * hR);
    double unL = dir == 0 ? uL : vL, unR = dir == 0 ? uR : vR;
    double ap = fmax(fmax(unL + cL, unR + cR), 0.0);
    double am = fmin(fmin(unL - cL, unR - cR), 0.0);
    double FL[3], FR[3], UL[3], UR[3];
    if (dir == 0) {
        FL[0] = pL; FL[1] = pL * uL + 0.5 * g * hL * hL; FL[2] = qL * uL;
        FR[0] = pR; FR[1] = pR * uR + 0.5 * g * hR * hR; FR[2] = qR * uR;
    } else {
        FL[0] = qL; FL[1] = pL * vL; FL[2] = qL * vL + 0.5 * g * hL * hL;
        FR[0] = qR; FR[1] = pR * vR; FR[2] = qR * vR + 0.5 * g * hR * hR;
    }
    UL[0] = hL; UL[1] = pL; UL[2] = qL;
    UR[0] = hR; UR[1] = pR; UR[2] = qR;
    double den = ap - am;
    for (int m = 0; m < 3; m++) {
        if (den > 0.0)
            H[m] = (ap * FL[m] - am * FR[m]) / den + ap * am / den * (UR[m] - UL[m]);
        else
            H[m] = 0.0;
    }
}

/* Evaluate E, F, G, F*, G* of the current (ghost-filled) state into ring slot s. */
static void compute_rhs(orc_dom *D, int s)
{
    int nx = D->nx, ny = D->ny;
    double dx = D->p.dx, dy = D->p.dy, g = D->p.g, Bd = D->p.Bd;

    /* x-faces i = 0..nx between cells i-1 and i, rows 0..ny-1 */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i <= nx; i++) {
            double a1, a2, b1, b2, c1, c2; /* left cell high face */
            double e1, e2, f1, f2, g1, g2; /* right cell low face */
            reconstruct(D, i - 1, j, 0, &a1, &a2, &b1, &b2, &c1, &c2);
            reconstruct(D, i, j, 0, &e1, &e2, &f1, &f2, &g1, &g2);
            double H[3];
            cu_flux(D, 0, D->bxf[XF(D, i, j)], a2, b2, c2, e1, f1, g1, H);
            for (int m = 0; m < 3; m++) D->Hx[m][XF(D, i, j)] = H[m];
        }
    /* y-faces j = 0..ny between cells j-1 and j */
    for (int j = 0; j <= ny; j++)
        for (int i = 0; i < nx; i++) {
            double a1, a2, b1, b2, c1, c2, e1, e2, f1, f2, g1, g2;
            reconstruct(D, i, j - 1, 1, &a1, &a2, &b1, &b2, &c1, &c2);
            reconstruct(D, i, j, 1, &e1, &e2, &f1, &f2, &g1, &g2);
            double H[3];
            cu_flux(D, 1, D->byf[YF(D, i, j)], a2, b2, c2, e1, f1, g1, H);
            for (int m = 0; m < 3; m++) D->Hy[m][YF(D, i, j)] = H[m];
        }

    /* eta = h - d on every cell (ghosts included) for the dispersive terms */
    for (int j = -2; j <= ny + 1; j++)
        for (int i = -2; i <= nx + 1; i++) {
            int c = CI(D, i, j);
            D->eta[c] = fmax(D->w[c] - D->b[c], 0.0) - D->d[c];
        }

    double *E = D->hist[0][s], *F = D->hist[1][s], *G = D->hist[2][s];
    double *Fs = D->hist[3][s], *Gs = D->hist[4][s];
    const double *et = D->eta, *P = D->P, *Q = D->Q;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = CI(D, i, j);
            /* Eq. 11 and the flux-divergence parts of Eqs. 12-13 */
            double divx[3], divy[3];
            for (int m = 0; m < 3; m++) {
                divx[m] = (D->Hx[m][XF(D, i + 1, j)] - D->Hx[m][XF(D, i, j)]) / dx;
                divy[m] = (D->Hy[m][YF(D, i, j + 1)] - D->Hy[m][YF(D, i, j)]) / dy;
            }
            /* well-balanced bed-slope source (KP07): -g (b_E - b_W)/dx * (mean face depth) */
            double bE = D->bxf[XF(D, i + 1, j)], bW = D->bxf[XF(D, i, j)];
            double bN = D->byf[YF(D, i, j + 1)], bS = D->byf[YF(D, i, j)];
            double w0 = D->w[c];
            double srcx = -g * (bE - bW) / dx * (w0 - 0.5 * (bE + bW));
            double srcy = -g * (bN - bS) / dy * (w0 - 0.5 * (bN + bS));
            /* quadratic bottom friction with desingularised cell velocities */
            double h = fmax(w0 - D->b[c], 0.0);
            double u = desing(h, P[c], D->p.eps), v = desing(h, Q[c], D->p.eps);
            double sp = sqrt(u * u + v * v);
            double fr1 = D->p.friction * u * sp, fr2 = D->p.friction * v * sp;
            /* central differences of eta (Eqs. 12-13), P and Q (Eqs. 14-15) */
            double d = D->d[c], dxd = D->ddx[c], dyd = D->ddy[c];
            double e_xx = (et[CI(D, i + 1, j)] - 2.0 * et[c] + et[CI(D, i - 1, j)]) / (dx * dx);
            double e_yy = (et[CI(D, i, j + 1)] - 2.0 * et[c] + et[CI(D, i, j - 1)]) / (dy * dy);
            double e_xy = (et[CI(D, i + 1, j + 1)] - et[CI(D, i + 1, j - 1)]
                           - et[CI(D, i - 1, j + 1)] + et[CI(D, i - 1, j - 1)]) / (4.0 * dx * dy);
            double e_xxx = (et[CI(D, i + 2, j)] - 2.0 * et[CI(D, i + 1, j)]
                            + 2.0 * et[CI(D, i - 1, j)] - et[CI(D, i - 2, j)]) / (2.0 * dx * dx * dx);
            double e_yyy = (et[CI(D, i, j + 2)] - 2.0 * et[CI(D, i, j + 1)]
                            + 2.0 * et[CI(D, i, j - 1)] - et[CI(D, i, j - 2)]) / (2.0 * dy * dy * dy);
            /* eta_xyy = d/dx of eta_yy ; eta_xxy = d/dy of eta_xx */
            double eyy_p = (et[CI(D, i + 1, j + 1)] - 2.0 * et[CI(D, i + 1, j)] + et[CI(D, i + 1, j - 1)]) / (dy * dy);
            double eyy_m = (et[CI(D, i - 1, j + 1)] - 2.0 * et[CI(D, i - 1, j)] + et[CI(D, i - 1, j - 1)]) / (dy * dy);
            double e_xyy = (eyy_p - eyy_m) / (2.0 * dx);
            double exx_p = (et[CI(D, i + 1, j + 1)] - 2.0 * et[CI(D, i, j + 1)] + et[CI(D, i - 1, j + 1)]) / (dx * dx);
            double exx_m = (et[CI(D, i + 1, j - 1)] - 2.0 * et[CI(D, i, j - 1)] + et[CI(D, i - 1, j - 1)]) / (dx * dx);
            double e_xxy = (exx_p - exx_m) / (2.0 * dy);
            double dispx = Bd * g * d * d * d * (e_xxx + e_xyy)
                         + Bd * g * d * d * (dxd * (2.0 * e_xx + e_yy) + dyd * e_xy);
            double dispy = Bd * g * d * d * d * (e_yyy + e_xxy)
                         + Bd * g * d * d * (dyd * (2.0 * e_yy + e_xx) + dxd * e_xy);

            E[c] = -divx[0] - divy[0];
            F[c] = -divx[1] - divy[1] + srcx - fr1 + dispx;
            G[c] = -divx[2] - divy[2] + srcy - fr2 + dispy;

            double Q_x = (Q[CI(D, i + 1, j)] - Q[CI(D, i - 1, j)]) / (2.0 * dx);
            double Q_y = (Q[CI(D, i, j + 1)] - Q[CI(D, i, j - 1)]) / (2.0 * dy);
            double Q_xy = (Q[CI(D, i + 1, j + 1)] - Q[CI(D, i + 1, j - 1)]
                           - Q[CI(D, i - 1, j + 1)] + Q[CI(D, i - 1, j - 1)]) / (4.0 * dx * dy);
            double P_x = (P[CI(D, i + 1, j)] - P[CI(D, i - 1, j)]) / (2.0 * dx);
            double P_y = (P[CI(D, i, j + 1)] - P[CI(D, i, j - 1)]) / (2.0 * dy);
            double P_xy = (P[CI(D, i + 1, j + 1)] - P[CI(D, i + 1, j - 1)]
                           - P[CI(D, i - 1, j + 1)] + P[CI(D, i - 1, j - 1)]) / (4.0 * dx * dy);
            Fs[c] = d * dxd * Q_y / 6.0 + d * dyd * Q_x / 6.0 + (Bd + 1.0 / 3.0) * d * d * Q_xy;
            Gs[c] = d * dxd * P_y / 6.0 + d * dyd * P_x / 6.0 + (Bd + 1.0 / 3.0) * d * d * P_xy;
        }
}

/* Eq. 22: max over the interior of (|u| + c)/dx and (|v| + c)/dy */
static double cfl_rate(const orc_dom *D)
{
    double m = 0.0;
    for (int j = 0; j < D->ny; j++)
        for (int i = 0; i < D->nx; i++) {
            int c = CI(D, i, j);
            double h = fmax(D->w[c] - D->b[c], 0.0);
            double u = desing(h, D->P[c], D->p.eps), v = desing(h, D->Q[c], D->p.eps);
            double cc = sqrt(D->p.g * h);
            double rx = (fabs(u) + cc) / D->p.dx, ry = (fabs(v) + cc) / D->p.dy;
            double r = fmax(rx, ry);
            if (r > m) m = r;
        }
    return m;
}

/* ------------------------------------------------------------------ */
/* tridiagonal coefficients, Eq. 21                                     */

static void coef_x(const orc_dom *D, int i, int j, double *A, double *B, double *C)
{
    int c = CI(D, i, j);
    double d = D->d[c], dd = D->ddx[c], dx = D->p.dx, k = D->p.Bd + 1.0 / 3.0;
    *A = d * dd / (6.0 * dx) - k * d * d / (dx * dx);
    *B = 1.0 + 2.0 * k * d * d / (dx * dx);
    *C = -d * dd / (6.0 * dx) - k * d * d / (dx * dx);
}

static void coef_y(const orc_dom *D, int i, int j, double *A, double *B, double *C)
{
    int c = CI(D, i, j);
    double d = D->d[c], dd = D->ddy[c], dy = D->p.dy, k = D->p.Bd + 1.0 / 3.0;
    *A = d * dd / (6.0 * dy) - k * d * d / (dy * dy);
    *B = 1.0 + 2.0 * k * d * d / (dy * dy);
    *C = -d * dd / (6.0 * dy) - k * d * d / (dy * dy);
}

/* 1 if every row of both line systems (with boundary closure) is strictly
 * diagonally dominant, else 0. */
int orc_diag_dominant(const orc_dom *D)
{
    for (int j = 0; j < D->ny; j++)
        for (int i = 0; i < D->nx; i++) {
            double A, B, C;
            coef_x(D, i, j, &A, &B, &C);
            if (i == 0) { if (D->p.bc[0] != ORC_MAKER) B -= A; A = 0.0; }
            if (i == D->nx - 1) { if (D->p.bc[1] != ORC_MAKER) B -= C; C = 0.0; }
            if (!(fabs(B) > fabs(A) + fabs(C))) return 0;
            coef_y(D, i, j, &A, &B, &C);
            if (j == 0) { if (D->p.bc[2] != ORC_MAKER) B -= A; A = 0.0; }
            if (j == D->ny - 1) { if (D->p.bc[3] != ORC_MAKER) B -= C; C = 0.0; }
            if (!(fabs(B) > fabs(A) + fabs(C))) return 0;
        }
    return 1;
}

/* ------------------------------------------------------------------ */
/* one time step                                                        */

/* dt_replay > 0: take that step.  Otherwise choose dt from Eq. 22 and the
 * lazy EMA of Eq. 47, clamp to dt_max and to t_end - t. */
int orc_step(orc_dom *D, double dt_replay, double t_end)
{
    int nx = D->nx, ny = D->ny;
    int s0 = D->slot, s1 = (D->slot + 2) % 3, s2 = (D->slot + 1) % 3; /* n, n-1, n-2 */

    orc_fill_ghosts(D, D->t);
    compute_rhs(D, s0);
    double rate = cfl_rate(D);
    D->last_rate = rate;

    double dt;
    if (dt_replay > 0.0) {
        dt = dt_replay;
    } else {
        double dtc;
        if (rate > 0.0) dtc = D->p.cfl / rate;
        else if (D->p.dt_max > 0.0) dtc = D->p.dt_max;
        else return ORC_ERR_UNSTABLE;
        if (D->n == 0 && D->p.dt_init > 0.0) dt = D->p.dt_init;
        else dt = dtc;
        /* Eq. 47: may drop at once, rises only gradually (off during the Euler start) */
        if (D->n >= 2 && dt > D->dtm1) dt = D->p.ema_alpha * dt + (1.0 - D->p.ema_alpha) * D->dtm1;
        if (D->p.dt_max > 0.0 && dt > D->p.dt_max) dt = D->p.dt_max;
        if (dt < D->p.dt_min) return ORC_ERR_UNSTABLE;
        double rem = t_end - D->t;
        if (dt > rem) dt = rem;
    }
    if (!(dt > 0.0)) return ORC_ERR_ARG;

    /* weights of the RHS levels n, n-1, n-2 (beta) and of F*, G* (gamma) */
    double beta[3] = {0, 0, 0}, gam[3] = {0, 0, 0};
    if (D->n == 0) {
        beta[0] = dt;                      /* forward Euler, no F* history yet */
    } else if (D->n == 1) {
        beta[0] = dt;                      /* forward Euler */
        gam[0] = 1.0; gam[1] = -1.0;       /* F*^n - F*^{n-1} */
    } else {
        orc_ab3_weights(dt, D->dtm1, D->dtm2, beta);
        orc_dstar_weights(dt, D->dtm1, D->dtm2, gam);
    }
    for (int k = 0; k < 3; k++) { D->beta[k] = beta[k]; D->gam[k] = gam[k]; }
    int sl[3] = {s0, s1, s2};

    /* U*^n and V*^n from Eqs. 9-10 on the current (ghost-filled) P, Q */
    double *Us = D->Us, *Vs = D->Vs;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double A, B, C;
            coef_x(D, i, j, &A, &B, &C);
            Us[CI(D, i, j)] = A * D->P[CI(D, i - 1, j)] + B * D->P[CI(D, i, j)] + C * D->P[CI(D, i + 1, j)];
            coef_y(D, i, j, &A, &B, &C);
            Vs[CI(D, i, j)] = A * D->Q[CI(D, i, j - 1)] + B * D->Q[CI(D, i, j)] + C * D->Q[CI(D, i, j + 1)];
        }

    /* prediction equations: Eq. 42 for w, Eq. 43 (+ Eqs. 44-46) for U*, V*.
     * cross_mode 1 leaves the F* term of U* out here and adds the exact
     * difference F*(Q^{n+1}) - F*^n once Q^{n+1} is known. */
    int nlev = D->n >= 2 ? 3 : 2;
    int fs_extrap = D->p.cross_mode == 0;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = CI(D, i, j);
            double dw = 0.0, dU = 0.0, dV = 0.0;
            for (int k = 0; k < nlev; k++) {
                dw += beta[k] * D->hist[0][sl[k]][c];
                dU += beta[k] * D->hist[1][sl[k]][c];
                if (fs_extrap) dU += gam[k] * D->hist[3][sl[k]][c];
                dV += beta[k] * D->hist[2][sl[k]][c] + gam[k] * D->hist[4][sl[k]][c];
            }
            double wn = D->w[c] + dw;
            if (wn < D->b[c]) { wn = D->b[c]; D->clamps++; }
            D->w[c] = wn;
            Us[c] += dU;
            Vs[c] += dV;
        }

    double t1 = D->t + dt;
    /* Eq. 20 on y-lines for Q^{n+1} */
    for (int i = 0; i < nx; i++) {
        for (int j = 0; j < ny; j++) {
            double A, B, C;
            coef_y(D, i, j, &A, &B, &C);
            D->ta[j] = A; D->tb[j] = B; D->tc[j] = C; D->tr[j] = Vs[CI(D, i, j)];
        }
        if (D->p.bc[2] == ORC_MAKER) {
            double e, p, q;
            maker_state(D, (i + 0.5) * D->p.dx, -0.5 * D->p.dy, t1, &e, &p, &q);
            D->tr[0] -= D->ta[0] * q;
        } else {
            D->tb[0] -= D->ta[0];
        }
        D->ta[0] = 0.0;
        if (D->p.bc[3] == ORC_MAKER) {
            double e, p, q;
            maker_state(D, (i + 0.5) * D->p.dx, (ny + 0.5) * D->p.dy, t1, &e, &p, &q);
            D->tr[ny - 1] -= D->tc[ny - 1] * q;
        } else {
            D->tb[ny - 1] -= D->tc[ny - 1];
        }
        D->tc[ny - 1] = 0.0;
        orc_thomas(ny, D->ta, D->tb, D->tc, D->tr, D->tx);
        for (int j = 0; j < ny; j++) D->Q[CI(D, i, j)] = D->tx[j];
    }
    /* sponge on Q (Sec. 3.3): Q scaled by gamma as soon as Q^{n+1} exists */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double gm = D->sponge[CI(D, i, j)];
            if (gm < 1.0) D->Q[CI(D, i, j)] *= gm;
        }

    if (!fs_extrap) {
        /* F* of Eq. 14 at the new level from Q^{n+1} (ghosts at t_{n+1}) */
        orc_fill_ghosts(D, t1);
        const double *Q = D->Q;
        double dx = D->p.dx, dy = D->p.dy, kB = D->p.Bd + 1.0 / 3.0;
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int c = CI(D, i, j);
                double d = D->d[c];
                double Q_x = (Q[CI(D, i + 1, j)] - Q[CI(D, i - 1, j)]) / (2.0 * dx);
                double Q_y = (Q[CI(D, i, j + 1)] - Q[CI(D, i, j - 1)]) / (2.0 * dy);
                double Q_xy = (Q[CI(D, i + 1, j + 1)] - Q[CI(D, i + 1, j - 1)]
                               - Q[CI(D, i - 1, j + 1)] + Q[CI(D, i - 1, j - 1)]) / (4.0 * dx * dy);
                double fs1 = d * D->ddx[c] * Q_y / 6.0 + d * D->ddy[c] * Q_x / 6.0 + kB * d * d * Q_xy;
                Us[c] += fs1 - D->hist[3][s0][c];
            }
    }

    /* Eq. 19 on x-lines for P^{n+1} */
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            double A, B, C;
            coef_x(D, i, j, &A, &B, &C);
            D->ta[i] = A; D->tb[i] = B; D->tc[i] = C; D->tr[i] = Us[CI(D, i, j)];
        }
        if (D->p.bc[0] == ORC_MAKER) {
            double e, p, q;
            maker_state(D, -0.5 * D->p.dx, (j + 0.5) * D->p.dy, t1, &e, &p, &q);
            D->tr[0] -= D->ta[0] * p;
        } else {
            D->tb[0] -= D->ta[0];
        }
        D->ta[0] = 0.0;
        if (D->p.bc[1] == ORC_MAKER) {
            double e, p, q;
            maker_state(D, (nx + 0.5) * D->p.dx, (j + 0.5) * D->p.dy, t1, &e, &p, &q);
            D->tr[nx - 1] -= D->tc[nx - 1] * p;
        } else {
            D->tb[nx - 1] -= D->tc[nx - 1];
        }
        D->tc[nx - 1] = 0.0;
        orc_thomas(nx, D->ta, D->tb, D->tc, D->tr, D->tx);
        for (int i = 0; i < nx; i++) D->P[CI(D, i, j)] = D->tx[i];
    }

    /* sponge on eta and P once P^{n+1} exists */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = CI(D, i, j);
            double gm = D->sponge[c];
            if (gm < 1.0) {
                double h = fmax(D->w[c] - D->b[c], 0.0), d = D->d[c];
                D->w[c] = D->b[c] + (d + gm * (h - d));
                D->P[c] *= gm;
            }
        }

    /* history bookkeeping */
    D->dtm2 = D->dtm1;
    D->dtm1 = dt;
    D->last_dt = dt;
    D->t = t1;
    D->n++;
    D->slot = (D->slot + 1) % 3;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* accessors                                                            */

/* field: 0 eta (= h - d), 1 P, 2 Q, 3 h, 4 w, 5 b (centre), 6 d,
 * 7 the per-cell sponge factor gamma (1 outside every band) */
int orc_get(const orc_dom *D, int field, double *out)
{
    for (int j = 0; j < D->ny; j++)
        for (int i = 0; i < D->nx; i++) {
            int c = CI(D, i, j);
            double h = fmax(D->w[c] - D->b[c], 0.0), v;
            switch (field) {
            case 0: v = h - D->d[c]; break;
            case 1: v = D->P[c]; break;
            case 2: v = D->Q[c]; break;
            case 3: v = h; break;
            case 4: v = D->w[c]; break;
            case 5: v = D->b[c]; break;
            case 6: v = D->d[c]; break;
            case 7: v = D->sponge[c]; break;
            default: return ORC_ERR_ARG;
            }
            out[i + j * D->nx] = v;
        }
    return ORC_OK;
}

/* The raw state w, P or Q (field 0, 1, 2) with its two ghost layers,
 * (nx+4)*(ny+4) values, x fastest, cell (i, j) at (i+2) + (j+2)(nx+4). */
int orc_get_padded(const orc_dom *D, int field, double *out)
{
    const double *src = field == 0 ? D->w : field == 1 ? D->P : field == 2 ? D->Q : NULL;
    if (!src) return ORC_ERR_ARG;
    for (int k = 0; k < D->sx * D->sy; k++) out[k] = src[k];
    return ORC_OK;
}

/* Overwrite the interior state from eta, P, Q (nx*ny each, NULL keeps). */
int orc_set_state(orc_dom *D, const double *eta, const double *P, const double *Q)
{
    for (int j = 0; j < D->ny; j++)
        for (int i = 0; i < D->nx; i++) {
            int c = CI(D, i, j), k = i + j * D->nx;
            if (eta) D->w[c] = D->b[c] + fmax(D->d[c] + eta[k], 0.0);
            if (P) D->P[c] = P[k];
            if (Q) D->Q[c] = Q[k];
        }
    return ORC_OK;
}

/* info: t, n, last dt, last CFL rate, mass sum(h) dx dy, clamp count */
void orc_info(const orc_dom *D, double *t, long long *n, double *last_dt,
              double *last_rate, double *mass, long long *clamps)
{
    double m = 0.0;
    for (int j = 0; j < D->ny; j++)
        for (int i = 0; i < D->nx; i++) {
            int c = CI(D, i, j);
            m += fmax(D->w[c] - D->b[c], 0.0);
        }
    if (t) *t = D->t;
    if (n) *n = D->n;
    if (last_dt) *last_dt = D->last_dt;
    if (last_rate) *last_rate = D->last_rate;
    if (mass) *mass = m * D->p.dx * D->p.dy;
    if (clamps) *clamps = D->clamps;
}

/* Ghost-fill the current state and evaluate the right-hand side without
 * stepping.  Outputs (nx*ny each, any may be NULL): E, F, G, F*, G*,
 * and the current CFL rate of Eq. 22. */
int orc_rhs(orc_dom *D, double *E, double *F, double *G, double *Fs, double *Gs, double *rate)
{
    orc_fill_ghosts(D, D->t);
    int s = D->slot;
    compute_rhs(D, s);
    double *outs[5] = {E, F, G, Fs, Gs};
    for (int f = 0; f < 5; f++) {
        if (!outs[f]) continue;
        for (int j = 0; j < D->ny; j++)
            for (int i = 0; i < D->nx; i++) outs[f][i + j * D->nx] = D->hist[f][s][CI(D, i, j)];
    }
    if (rate) *rate = cfl_rate(D);
    return ORC_OK;
}

/* Dispersive parts alone: the eta terms of Eqs. 12-13 (dispx, dispy) and
 * F*, G* of Eqs. 14-15, from the current ghost-filled state. */
int orc_dispersive(orc_dom *D, double *dispx, double *dispy, double *Fs, double *Gs)
{
    orc_fill_ghosts(D, D->t);
    int s = D->slot;
    compute_rhs(D, s); /* fills eta of the current state and F*, G* */
    int nx = D->nx, ny = D->ny;
    double dx = D->p.dx, dy = D->p.dy, g = D->p.g, Bd = D->p.Bd;
    const double *et = D->eta;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = CI(D, i, j), k = i + j * nx;
            double d = D->d[c], dxd = D->ddx[c], dyd = D->ddy[c];
            double e_xx = (et[CI(D, i + 1, j)] - 2.0 * et[c] + et[CI(D, i - 1, j)]) / (dx * dx);
            double e_yy = (et[CI(D, i, j + 1)] - 2.0 * et[c] + et[CI(D, i, j - 1)]) / (dy * dy);
            double e_xy = (et[CI(D, i + 1, j + 1)] - et[CI(D, i + 1, j - 1)]
                           - et[CI(D, i - 1, j + 1)] + et[CI(D, i - 1, j - 1)]) / (4.0 * dx * dy);
            double e_xxx = (et[CI(D, i + 2, j)] - 2.0 * et[CI(D, i + 1, j)]
                            + 2.0 * et[CI(D, i - 1, j)] - et[CI(D, i - 2, j)]) / (2.0 * dx * dx * dx);
            double e_yyy = (et[CI(D, i, j + 2)] - 2.0 * et[CI(D, i, j + 1)]
                            + 2.0 * et[CI(D, i, j - 1)] - et[CI(D, i, j - 2)]) / (2.0 * dy * dy * dy);
            double eyy_p = (et[CI(D, i + 1, j + 1)] - 2.0 * et[CI(D, i + 1, j)] + et[CI(D, i + 1, j - 1)]) / (dy * dy);
            double eyy_m = (et[CI(D, i - 1, j + 1)] - 2.0 * et[CI(D, i - 1, j)] + et[CI(D, i - 1, j - 1)]) / (dy * dy);
            double exx_p = (et[CI(D, i + 1, j + 1)] - 2.0 * et[CI(D, i, j + 1)] + et[CI(D, i - 1, j + 1)]) / (dx * dx);
            double exx_m = (et[CI(D, i + 1, j - 1)] - 2.0 * et[CI(D, i, j - 1)] + et[CI(D, i - 1, j - 1)]) / (dx * dx);
            double e_xyy = (eyy_p - eyy_m) / (2.0 * dx), e_xxy = (exx_p - exx_m) / (2.0 * dy);
            if (dispx) dispx[k] = Bd * g * d * d * d * (e_xxx + e_xyy)
                                + Bd * g * d * d * (dxd * (2.0 * e_xx + e_yy) + dyd * e_xy);
            if (dispy) dispy[k] = Bd * g * d * d * d * (e_yyy + e_xxy)
                                + Bd * g * d * d * (dyd * (2.0 * e_yy + e_xx) + dxd * e_xy);
            if (Fs) Fs[k] = D->hist[3][s][c];
            if (Gs) Gs[k] = D->hist[4][s][c];
        }
    return ORC_OK;
}

/* Apply the x-line operator of Eq. 9 (the left-hand side of Eq. 19 with the
 * ghost-filled neighbours) to the current P: out = U*.  And the y-line
 * operator of Eq. 10 to Q: out = V*. */
int orc_apply_T(orc_dom *D, double *Ustar, double *Vstar)
{
    orc_fill_ghosts(D, D->t);
    for (int j = 0; j < D->ny; j++)
        for (int i = 0; i < D->nx; i++) {
            double A, B, C;
            int k = i + j * D->nx;
            coef_x(D, i, j, &A, &B, &C);
            if (Ustar) Ustar[k] = A * D->P[CI(D, i - 1, j)] + B * D->P[CI(D, i, j)] + C * D->P[CI(D, i + 1, j)];
            coef_y(D, i, j, &A, &B, &C);
            if (Vstar) Vstar[k] = A * D->Q[CI(D, i, j - 1)] + B * D->Q[CI(D, i, j)] + C * D->Q[CI(D, i, j + 1)];
        }
    return ORC_OK;
}

/* Last step's weights: beta[3], gamma[3]. */
void orc_last_weights(const orc_dom *D, double *beta, double *gam)
{
    for (int k = 0; k < 3; k++) { beta[k] = D->beta[k]; gam[k] = D->gam[k]; }
}

/* Wave-maker state at a point and time (eta, P, Q), for checks. */
void orc_maker_state(const orc_dom *D, double x, double y, double t, double out[3])
{
    maker_state(D, x, y, t, &out[0], &out[1], &out[2]);
}

double orc_component_k(const orc_dom *D, int k) { return (k >= 0 && k < D->ncomp) ? D->kw[k] : 0.0; }
