/* btdf_oracle.c - plain FP64 CPU oracle of the BTDF-IB / D2Q9 LBM step.
 *
 * TEST INFRASTRUCTURE: loaded only by the tests, the smoke check and the CPU
 * baseline of the benchmark.  Slow and literal on purpose.  Every function
 * cites the passage of Jiang & Liu (arXiv 1806.09403) it follows.
 *
 * One time step (NF forcing passes, the paper's Algorithm 1), starting from
 * the post-streaming populations f^n:
 *   1. rho and u* at every node (Eqs. 9, 10).
 *   2. For k = 1..NF (Algorithm 1, step 3):
 *        interpolate u* and rho to every marker (Eqs. 12, 14),
 *        dF_b = 2 rho_l (U_b - D_I u*) (Eq. 20, also Eq. 29),
 *        df = D_E dF_b with the thickened shell drs (Eqs. 13, 15),
 *        F_b += dF_b, f += df, u* += df / (2 rho) (Eq. 11).
 *   3. Force on each body F_p = -sum_l F_b,l ds drs (Eq. 27; minus sign: F_b
 *      acts on the fluid).
 *   4. u = u*_0 + (f + g) / (2 rho) (Eq. 11), f_eq (Eq. 6), Guo term (Eq. 7),
 *      BGK collision (Eq. 5).
 *   5. Push streaming (left side of Eq. 5), then boundary rules in the order
 *      walls, inlet column, outlet column.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - rho in Eq. 20 is the interpolated density D_I rho.
 *   - Delta arguments are (x_e - X_l)/dh, dh = 1; D_E carries drs*ds/dh^2.
 *   - Support of a marker: the w nodes per axis with |x_e - X| < w/2
 *     (w = 2, 3, 4); nodes outside a non-periodic lattice are dropped,
 *     periodic axes wrap.
 *   - Boundaries of the cylinder channel (Sec. 5.2 gives only their physical
 *     meaning): inlet x = 0 by non-equilibrium extrapolation from column 1
 *     with u = (u_in, 0); outlet x = nx-1 copies column nx-2 (bc_x = 1) or
 *     follows the convective condition d f / dt + U d f / dx = 0 with
 *     U = u_in, implicit upwind in time and space (bc_x = 2); free-slip walls
 *     by half-way specular reflection; no-slip walls by half-way bounce-back.
 *   - Taylor-Green box (Sec. 5.1, bc_x = 3): every outer node by
 *     non-equilibrium extrapolation from its nearest interior node (the
 *     diagonal one at a corner) to the prescribed boundary velocity.
 *
 * Parity pins (tests/test_oracle_*.py): delta identities, equilibrium and
 * Guo-term moments, exact momentum budget, dense-operator brute force,
 * Eq. 27's two sides, flat-wall thickness closed form, circle thickness
 * against Sec. 4.4, Poiseuille and Taylor-Green closed forms, uniform-flow
 * invariance of every boundary rule, and BTDF slip below DF slip (Sec. 5.2).
 */
#include "btdf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D2Q9 lattice, Eq. 8 and the weights stated below Eq. 7. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

typedef struct {
    int n;
    double ds, drs;
    double *X, *Y, *Ubx, *Uby;
    double *Usx, *Usy, *Fx, *Fy, *Ux, *Uy, *rho;
    double *hx, *hy;
    int64_t hlen, hcap;
} ora_body;

struct ora_sim {
    int nx, ny, bcx, bcy, delta, nf;
    double *outlet_old;      /* [ny][9] outlet column before the last streaming (bc_x = 2) */
    double *box_ux, *box_uy; /* perimeter velocities of the prescribed-velocity box (bc_x = 3) */
    double tau, u_in, gx, gy;
    double *f, *fpost;          /* [ny][nx][9] */
    double *rho, *ux, *uy;      /* moments; ux, uy are u* (updated by passes) */
    double *fx, *fy;            /* IB force density of the current step */
    double *dfx, *dfy;          /* one pass's spread increment */
    int nb;
    ora_body *b;
    int64_t step;
};

static int g_threads = 1;
void oracle_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int oracle_get_threads(void) { return g_threads; }

/* ---- regularized delta functions, Sec. 4.3 -------------------------------- */

double oracle_delta(int kind, double r)
{
    double a = fabs(r);
    switch (kind) {
    case 2: /* Eq. 37 */
        return a <= 1.0 ? 1.0 - a : 0.0;
    case 3: /* Eq. 38 */
        if (a > 1.5) return 0.0;
        if (a > 0.5) return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))) / 6.0;
        return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
    case 4: /* Eq. 39 */
        if (a >= 2.0) return 0.0;
        if (a >= 1.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
        return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    case 5: /* 4-point cosine kernel (not printed in the paper) */
        return a < 2.0 ? 0.25 * (1.0 + cos(M_PI * a / 2.0)) : 0.0;
    default:
        return 0.0;
    }
}

int oracle_support_width(int kind)
{
    switch (kind) {
    case 2: return 2;
    case 3: return 3;
    case 4: case 5: return 4;
    default: return 0;
    }
}

/* Thickness of the solid forcing shell suggested in Sec. 4.4 for the 2-, 3-
 * and 4-point functions; the cosine kernel shares the 4-point support and
 * takes the 4-point value. */
double oracle_drs_paper(int kind)
{
    switch (kind) {
    case 2: return 1.4;
    case 3: return 1.9;
    case 4: case 5: return 2.6;
    default: return 1.0;
    }
}

/* ---- equilibrium and forcing, Eqs. 6 and 7 --------------------------------- */

void oracle_feq(double rho, double ux, double uy, double *out)
{
    double usq = ux * ux + uy * uy;
    for (int a = 0; a < 9; a++) {
        double eu = EX[a] * ux + EY[a] * uy;
        out[a] = WT[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
    }
}

void oracle_guo(double tau, double ux, double uy, double fx, double fy, double *out)
{
    double pre = 1.0 - 1.0 / (2.0 * tau);
    for (int a = 0; a < 9; a++) {
        double eu = EX[a] * ux + EY[a] * uy;
        double t = 3.0 * ((EX[a] - ux) * fx + (EY[a] - uy) * fy)
                 + 9.0 * eu * (EX[a] * fx + EY[a] * fy);
        out[a] = pre * WT[a] * t;
    }
}

/* ---- lattice --------------------------------------------------------------- */

ora_sim *oracle_create(int nx, int ny, double tau, double u_in, int bc_x, int bc_y,
                       double gx, double gy, int delta, int nf)
{
    if (nx < 3 || ny < 3 || !(tau > 0.5) || oracle_support_width(delta) == 0 || nf < 1 ||
        bc_x < 0 || bc_x > 3)
        return NULL;
    ora_sim *s = (ora_sim *)calloc(1, sizeof(ora_sim));
    size_t nn = (size_t)nx * ny;
    s->nx = nx; s->ny = ny; s->tau = tau; s->u_in = u_in;
    s->bcx = bc_x; s->bcy = bc_y; s->gx = gx; s->gy = gy;
    s->delta = delta; s->nf = nf;
    s->f = (double *)calloc(nn * 9, sizeof(double));
    s->fpost = (double *)calloc(nn * 9, sizeof(double));
    s->outlet_old = (double *)calloc((size_t)ny * 9, sizeof(double));
    s->box_ux = (double *)calloc((size_t)(2 * nx + 2 * (ny - 2)), sizeof(double));
    s->box_uy = (double *)calloc((size_t)(2 * nx + 2 * (ny - 2)), sizeof(double));
    s->rho = (double *)calloc(nn, sizeof(double));
    s->ux = (double *)calloc(nn, sizeof(double));
    s->uy = (double *)calloc(nn, sizeof(double));
    s->fx = (double *)calloc(nn, sizeof(double));
    s->fy = (double *)calloc(nn, sizeof(double));
    s->dfx = (double *)calloc(nn, sizeof(double));
    s->dfy = (double *)calloc(nn, sizeof(double));
    return s;
}

static void free_body(ora_body *b)
{
    free(b->X); free(b->Y); free(b->Ubx); free(b->Uby);
    free(b->Usx); free(b->Usy); free(b->Fx); free(b->Fy);
    free(b->Ux); free(b->Uy); free(b->rho); free(b->hx); free(b->hy);
}

void oracle_destroy(ora_sim *s)
{
    if (!s) return;
    for (int i = 0; i < s->nb; i++) free_body(&s->b[i]);
    free(s->b);
    free(s->f); free(s->fpost); free(s->rho); free(s->ux); free(s->uy); free(s->outlet_old); free(s->box_ux); free(s->box_uy);
    free(s->fx); free(s->fy); free(s->dfx); free(s->dfy);
    free(s);
}

void oracle_init_fields(ora_sim *s, const double *rho, const double *ux, const double *uy)
{
    size_t nn = (size_t)s->nx * s->ny;
    for (size_t n = 0; n < nn; n++) oracle_feq(rho[n], ux[n], uy[n], &s->f[n * 9]);
    s->step = 0;
}

void oracle_get_pops(const ora_sim *s, double *out)
{
    memcpy(out, s->f, sizeof(double) * 9 * (size_t)s->nx * s->ny);
}

void oracle_set_pops(ora_sim *s, const double *in)
{
    memcpy(s->f, in, sizeof(double) * 9 * (size_t)s->nx * s->ny);
}

static double *dup(const double *p, int n)
{
    double *q = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    if (p) memcpy(q, p, sizeof(double) * n); else memset(q, 0, sizeof(double) * n);
    return q;
}

int oracle_add_body(ora_sim *s, int n, const double *X, const double *Y,
                    const double *Ubx, const double *Uby, double ds, double drs)
{
    s->b = (ora_body *)realloc(s->b, sizeof(ora_body) * (s->nb + 1));
    ora_body *b = &s->b[s->nb];
    memset(b, 0, sizeof(*b));
    b->n = n; b->ds = ds;
    b->drs = drs > 0.0 ? drs : oracle_drs_paper(s->delta);
    b->X = dup(X, n); b->Y = dup(Y, n); b->Ubx = dup(Ubx, n); b->Uby = dup(Uby, n);
    b->Usx = dup(NULL, n); b->Usy = dup(NULL, n); b->Fx = dup(NULL, n); b->Fy = dup(NULL, n);
    b->Ux = dup(NULL, n); b->Uy = dup(NULL, n); b->rho = dup(NULL, n);
    return s->nb++;
}

void oracle_set_marker_velocity(ora_sim *s, int body, const double *Ubx, const double *Uby)
{
    ora_body *b = &s->b[body];
    memcpy(b->Ubx, Ubx, sizeof(double) * b->n);
    memcpy(b->Uby, Uby, sizeof(double) * b->n);
}

double oracle_body_drs(const ora_sim *s, int body) { return s->b[body].drs; }

/* ---- support of a marker and the operators D_I, D_E, Eqs. 12-15 ----------- */

/* Maps a node coordinate onto the lattice: wraps periodic axes, returns -1
 * for a node outside a bounded axis. */
static int map_axis(int i, int n, int periodic)
{
    if (periodic) return ((i % n) + n) % n;
    return (i < 0 || i >= n) ? -1 : i;
}

int oracle_support(const ora_sim *s, double X, double Y, int64_t *nodes, double *w)
{
    int wd = oracle_support_width(s->delta);
    int i0 = (int)floor(X - 0.5 * wd) + 1;   /* first node with x > X - w/2 */
    int j0 = (int)floor(Y - 0.5 * wd) + 1;
    int cnt = 0;
    for (int j = j0; j < j0 + wd; j++) {
        int yy = map_axis(j, s->ny, s->bcy == 0);
        if (yy < 0) continue;
        double wy = oracle_delta(s->delta, (double)j - Y);
        for (int i = i0; i < i0 + wd; i++) {
            int xx = map_axis(i, s->nx, s->bcx == 0);
            if (xx < 0) continue;
            double wx = oracle_delta(s->delta, (double)i - X);
            nodes[cnt] = (int64_t)yy * s->nx + xx;
            w[cnt] = wx * wy;             /* Eq. 14 with dh = 1 */
            cnt++;
        }
    }
    return cnt;
}

void oracle_interp(const ora_sim *s, int body, const double *fx, const double *fy,
                   double *Ux, double *Uy)
{
    const ora_body *b = &s->b[body];
    int64_t nodes[16];
    double w[16];
    for (int l = 0; l < b->n; l++) {
        int c = oracle_support(s, b->X[l], b->Y[l], nodes, w);
        double ax = 0.0, ay = 0.0;
        for (int k = 0; k < c; k++) {
            ax += w[k] * fx[nodes[k]];
            ay += w[k] * fy[nodes[k]];
        }
        Ux[l] = ax;
        Uy[l] = ay;
    }
}

void oracle_spread(const ora_sim *s, int body, const double *Fx, const double *Fy,
                   double *fx, double *fy)
{
    const ora_body *b = &s->b[body];
    int64_t nodes[16];
    double w[16];
    for (int l = 0; l < b->n; l++) {
        int c = oracle_support(s, b->X[l], b->Y[l], nodes, w);
        for (int k = 0; k < c; k++) {
            /* Eq. 15 with dh = 1: weight * drs * ds */
            fx[nodes[k]] += w[k] * b->drs * b->ds * Fx[l];
            fy[nodes[k]] += w[k] * b->drs * b->ds * Fy[l];
        }
    }
}

/* Eq. 22 with dh = 1: A_ij = sum_k W_ik W_jk ds, then Eq. 24-25:
 * A drs = 1.  Dense Gaussian elimination with partial pivoting. */
int oracle_drs_local(const ora_sim *s, int body, double *drs_out)
{
    const ora_body *b = &s->b[body];
    int n = b->n;
    size_t nn = (size_t)s->nx * s->ny;
    double *A = (double *)calloc((size_t)n * (n + 1), sizeof(double));
    double *col = (double *)calloc(nn, sizeof(double));
    int64_t ni[16], nj[16];
    double wi[16], wj[16];
    for (int i = 0; i < n; i++) {
        int ci = oracle_support(s, b->X[i], b->Y[i], ni, wi);
        for (int k = 0; k < ci; k++) col[ni[k]] = wi[k];
        for (int j = 0; j < n; j++) {
            int cj = oracle_support(s, b->X[j], b->Y[j], nj, wj);
            double acc = 0.0;
            for (int k = 0; k < cj; k++) acc += col[nj[k]] * wj[k];
            A[(size_t)i * (n + 1) + j] = acc * b->ds;
        }
        for (int k = 0; k < ci; k++) col[ni[k]] = 0.0;
        A[(size_t)i * (n + 1) + n] = 1.0;
    }
    int rc = 0;
    for (int c = 0; c < n && rc == 0; c++) {
        int p = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(A[(size_t)r * (n + 1) + c]) > fabs(A[(size_t)p * (n + 1) + c])) p = r;
        if (fabs(A[(size_t)p * (n + 1) + c]) < 1e-300) { rc = -1; break; }
        if (p != c)
            for (int k = 0; k <= n; k++) {
                double t = A[(size_t)c * (n + 1) + k];
                A[(size_t)c * (n + 1) + k] = A[(size_t)p * (n + 1) + k];
                A[(size_t)p * (n + 1) + k] = t;
            }
        for (int r = c + 1; r < n; r++) {
            double m = A[(size_t)r * (n + 1) + c] / A[(size_t)c * (n + 1) + c];
            for (int k = c; k <= n; k++) A[(size_t)r * (n + 1) + k] -= m * A[(size_t)c * (n + 1) + k];
        }
    }
    if (rc == 0)
        for (int r = n - 1; r >= 0; r--) {
            double acc = A[(size_t)r * (n + 1) + n];
            for (int k = r + 1; k < n; k++) acc -= A[(size_t)r * (n + 1) + k] * drs_out[k];
            drs_out[r] = acc / A[(size_t)r * (n + 1) + r];
        }
    free(A);
    free(col);
    return rc;
}

/* ---- the time step, Algorithm 1 ------------------------------------------- */

/* Eqs. 9-10: density and unforced velocity of node n. */
static void node_moments(const double *fn, double *rho, double *ux, double *uy)
{
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; a++) {
        r += fn[a];
        jx += EX[a] * fn[a];
        jy += EY[a] * fn[a];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

static void ensure_hist(ora_body *b)
{
    if (b->hlen == b->hcap) {
        b->hcap = b->hcap ? 2 * b->hcap : 1024;
        b->hx = (double *)realloc(b->hx, sizeof(double) * b->hcap);
        b->hy = (double *)realloc(b->hy, sizeof(double) * b->hcap);
    }
}

/* Algorithm 1, step 3: NF forcing passes. */
static void ib_stage(ora_sim *s)
{
    size_t nn = (size_t)s->nx * s->ny;
    memset(s->fx, 0, sizeof(double) * nn);
    memset(s->fy, 0, sizeof(double) * nn);
    for (int bi = 0; bi < s->nb; bi++) {
        ora_body *b = &s->b[bi];
        memset(b->Fx, 0, sizeof(double) * b->n);
        memset(b->Fy, 0, sizeof(double) * b->n);
    }
    if (s->nb == 0) return;
    int64_t nodes[16];
    double w[16];
    for (int k = 1; k <= s->nf; k++) {
        /* (a) Eq. 20 for the increment, with u* of this pass, for all markers */
        double **dFx = (double **)malloc(sizeof(double *) * s->nb);
        double **dFy = (double **)malloc(sizeof(double *) * s->nb);
        for (int bi = 0; bi < s->nb; bi++) {
            ora_body *b = &s->b[bi];
            dFx[bi] = (double *)malloc(sizeof(double) * b->n);
            dFy[bi] = (double *)malloc(sizeof(double) * b->n);
            for (int l = 0; l < b->n; l++) {
                int c = oracle_support(s, b->X[l], b->Y[l], nodes, w);
                double Ux = 0.0, Uy = 0.0, rl = 0.0;
                for (int q = 0; q < c; q++) {           /* Eq. 14 */
                    Ux += w[q] * s->ux[nodes[q]];
                    Uy += w[q] * s->uy[nodes[q]];
                    rl += w[q] * s->rho[nodes[q]];
                }
                if (k == 1) { b->Usx[l] = Ux; b->Usy[l] = Uy; b->rho[l] = rl; }
                dFx[bi][l] = 2.0 * rl * (b->Ubx[l] - Ux);   /* Eq. 20, dt = 1 */
                dFy[bi][l] = 2.0 * rl * (b->Uby[l] - Uy);
                b->Fx[l] += dFx[bi][l];                     /* step 3(c) */
                b->Fy[l] += dFy[bi][l];
            }
        }
        /* (b) spread with Eq. 15 */
        memset(s->dfx, 0, sizeof(double) * nn);
        memset(s->dfy, 0, sizeof(double) * nn);
        for (int bi = 0; bi < s->nb; bi++) oracle_spread(s, bi, dFx[bi], dFy[bi], s->dfx, s->dfy);
        /* (d), (e): u* += df / (2 rho) (Eq. 11), f += df */
        for (size_t n = 0; n < nn; n++) {
            s->fx[n] += s->dfx[n];
            s->fy[n] += s->dfy[n];
            s->ux[n] += s->dfx[n] / (2.0 * s->rho[n]);
            s->uy[n] += s->dfy[n] / (2.0 * s->rho[n]);
        }
        for (int bi = 0; bi < s->nb; bi++) { free(dFx[bi]); free(dFy[bi]); }
        free(dFx);
        free(dFy);
    }
    /* Diagnostics: D_I of the corrected velocity (boundary slip, Eq. 45). */
    for (int bi = 0; bi < s->nb; bi++) oracle_interp(s, bi, s->ux, s->uy, s->b[bi].Ux, s->b[bi].Uy);
    /* Algorithm 1 step 4, Eq. 27: force on the body is minus the force on the fluid. */
    for (int bi = 0; bi < s->nb; bi++) {
        ora_body *b = &s->b[bi];
        double sx = 0.0, sy = 0.0;
        for (int l = 0; l < b->n; l++) {
            sx += b->Fx[l] * b->ds * b->drs;
            sy += b->Fy[l] * b->ds * b->drs;
        }
        ensure_hist(b);
        b->hx[b->hlen] = -sx;
        b->hy[b->hlen] = -sy;
        b->hlen++;
    }
}

/* Source node of a pull along one axis; -1 when it lies off a bounded axis. */
static int src_axis(int i, int n, int periodic) { return map_axis(i, n, periodic); }

/* Inlet x = 0 by non-equilibrium extrapolation from column 1 of the
 * post-streaming populations: f(0) = f_eq(rho_1, (u_in, 0)) + f(1) - f_eq(rho_1, u_1). */
static void inlet_column(ora_sim *s)
{
    const int nx = s->nx, ny = s->ny;
    double *fn = s->f;
    for (int y = 0; y < ny; y++) {
        double r1, u1x, u1y, e_in[9], e_1[9];
        const double *f1 = &fn[((size_t)y * nx + 1) * 9];
        double *f0 = &fn[((size_t)y * nx) * 9];
        node_moments(f1, &r1, &u1x, &u1y);
        oracle_feq(r1, s->u_in, 0.0, e_in);
        oracle_feq(r1, u1x, u1y, e_1);
        for (int a = 0; a < 9; a++) f0[a] = e_in[a] + f1[a] - e_1[a];
    }
}

/* Position of outer node (x, y) in the perimeter order: row 0, row ny-1,
 * column 0 without its corners, column nx-1 without its corners. */
static int perimeter(const ora_sim *s, int x, int y)
{
    if (y == 0) return x;
    if (y == s->ny - 1) return s->nx + x;
    if (x == 0) return 2 * s->nx + (y - 1);
    return 2 * s->nx + (s->ny - 2) + (y - 1);
}

/* Prescribed-velocity box (Sec. 5.1): every outer node by non-equilibrium
 * extrapolation from its nearest interior node (the diagonal one at a
 * corner), f = f_eq(rho_n, u_b) + f_n - f_eq(rho_n, u_n). */
static void box_nodes(ora_sim *s)
{
    const int nx = s->nx, ny = s->ny;
    double *fn = s->f;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            if (x != 0 && x != nx - 1 && y != 0 && y != ny - 1) continue;
            const int xn = x < 1 ? 1 : (x > nx - 2 ? nx - 2 : x);
            const int yn = y < 1 ? 1 : (y > ny - 2 ? ny - 2 : y);
            const double *f1 = &fn[((size_t)yn * nx + xn) * 9];
            double *f0 = &fn[((size_t)y * nx + x) * 9];
            double r1, u1x, u1y, e_b[9], e_1[9];
            const int k = perimeter(s, x, y);
            node_moments(f1, &r1, &u1x, &u1y);
            oracle_feq(r1, s->box_ux[k], s->box_uy[k], e_b);
            oracle_feq(r1, u1x, u1y, e_1);
            for (int a = 0; a < 9; a++) f0[a] = e_b[a] + f1[a] - e_1[a];
        }
}

void oracle_set_boundary_velocity(ora_sim *s, const double *ubx, const double *uby)
{
    const size_t np = (size_t)(2 * s->nx + 2 * (s->ny - 2));
    memcpy(s->box_ux, ubx, sizeof(double) * np);
    memcpy(s->box_uy, uby, sizeof(double) * np);
}

void oracle_apply_inlet(ora_sim *s)
{
    if (s->bcx == 1 || s->bcx == 2) inlet_column(s);
}

static void stream_and_bc(ora_sim *s)
{
    const int nx = s->nx, ny = s->ny;
    /* the box overrides every outer node afterwards: stream periodically */
    const int px = s->bcx == 0 || s->bcx == 3, py = s->bcy == 0 || s->bcx == 3;
    double *fn = s->f;
    /* the outlet column before this streaming (convective outlet) */
    if (s->bcx == 2)
        for (int y = 0; y < ny; y++)
            for (int a = 0; a < 9; a++) s->outlet_old[y * 9 + a] = fn[((size_t)y * nx + nx - 1) * 9 + a];
    /* Every entry is overwritten below; NaN marks any that is not. */
    for (size_t q = 0; q < (size_t)nx * ny * 9; q++) fn[q] = NAN;
    /* Push streaming: f(x + e_a, t + 1) = f_post(x, t). */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++)
            for (int a = 0; a < 9; a++) {
                int tx = map_axis(x + EX[a], nx, px);
                int ty = map_axis(y + EY[a], ny, py);
                if (tx < 0 || ty < 0) continue;
                fn[((size_t)ty * nx + tx) * 9 + a] = s->fpost[((size_t)y * nx + x) * 9 + a];
            }
    const double *fp = s->fpost;
#define FP(xx, yy, a) fp[((size_t)(yy) * nx + (xx)) * 9 + (a)]
#define FN(xx, yy, a) fn[((size_t)(yy) * nx + (xx)) * 9 + (a)]
    if (!py) {
        int top = ny - 1;
        for (int x = 0; x < nx; x++) {
            FN(x, 0, 2) = FP(x, 0, 4);
            FN(x, top, 4) = FP(x, top, 2);
            if (s->bcy == 2) {            /* half-way bounce-back */
                FN(x, 0, 5) = FP(x, 0, 7);
                FN(x, 0, 6) = FP(x, 0, 8);
                FN(x, top, 7) = FP(x, top, 5);
                FN(x, top, 8) = FP(x, top, 6);
            } else {                      /* half-way specular reflection */
                int xm = src_axis(x - 1, nx, px), xp = src_axis(x + 1, nx, px);
                if (xm >= 0) { FN(x, 0, 5) = FP(xm, 0, 8); FN(x, top, 8) = FP(xm, top, 5); }
                if (xp >= 0) { FN(x, 0, 6) = FP(xp, 0, 7); FN(x, top, 7) = FP(xp, top, 6); }
            }
        }
    }
    if (s->bcx == 1) {
        inlet_column(s);
        for (int y = 0; y < ny; y++)          /* outlet: zero gradient */
            for (int a = 0; a < 9; a++) FN(nx - 1, y, a) = FN(nx - 2, y, a);
    } else if (s->bcx == 3) {
        box_nodes(s);
    } else if (s->bcx == 2) {
        inlet_column(s);
        /* convective outlet, d f / dt + U d f / dx = 0 with U = u_in,
         * implicit upwind: f(N, t+1) = (f(N, t) + U f(N-1, t+1)) / (1 + U) */
        const double U = s->u_in;
        for (int y = 0; y < ny; y++)
            for (int a = 0; a < 9; a++)
                FN(nx - 1, y, a) = (s->outlet_old[y * 9 + a] + U * FN(nx - 2, y, a)) / (1.0 + U);
    }
#undef FP
#undef FN
}

static void step_once(ora_sim *s)
{
    const size_t nn = (size_t)s->nx * s->ny;
    /* Algorithm 1 step 1: Eqs. 9-10 */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (size_t n = 0; n < nn; n++) node_moments(&s->f[n * 9], &s->rho[n], &s->ux[n], &s->uy[n]);
    /* steps 2-4 */
    ib_stage(s);
    /* steps 5-6: Eqs. 11, 6, 7, 5 */
    const double tau = s->tau;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (size_t n = 0; n < nn; n++) {
        const double *fn = &s->f[n * 9];
        double rho, u0x, u0y, feq[9], guo[9];
        node_moments(fn, &rho, &u0x, &u0y);
        double Fx = s->fx[n] + s->gx, Fy = s->fy[n] + s->gy;
        double ux = u0x + Fx / (2.0 * rho);
        double uy = u0y + Fy / (2.0 * rho);
        oracle_feq(rho, ux, uy, feq);
        oracle_guo(tau, ux, uy, Fx, Fy, guo);
        for (int a = 0; a < 9; a++) s->fpost[n * 9 + a] = fn[a] - (fn[a] - feq[a]) / tau + guo[a];
    }
    /* step 7 */
    stream_and_bc(s);
    s->step++;
}

void oracle_step(ora_sim *s, int64_t nsteps)
{
    for (int64_t i = 0; i < nsteps; i++) step_once(s);
}

int64_t oracle_step_count(const ora_sim *s) { return s->step; }

void oracle_moments(const ora_sim *s, double *rho, double *ux, double *uy)
{
    size_t nn = (size_t)s->nx * s->ny;
    for (size_t n = 0; n < nn; n++) node_moments(&s->f[n * 9], &rho[n], &ux[n], &uy[n]);
}

void oracle_force_field(const ora_sim *s, double *fx, double *fy)
{
    size_t nn = (size_t)s->nx * s->ny;
    memcpy(fx, s->fx, sizeof(double) * nn);
    memcpy(fy, s->fy, sizeof(double) * nn);
}

int64_t oracle_history(const ora_sim *s, int body, int64_t first, int64_t n, double *Fx, double *Fy)
{
    const ora_body *b = &s->b[body];
    int64_t c = 0;
    for (int64_t i = first; i < first + n && i < b->hlen; i++, c++) {
        Fx[c] = b->hx[i];
        Fy[c] = b->hy[i];
    }
    return c;
}

void oracle_marker_diag(const ora_sim *s, int body, double *Usx, double *Usy,
                        double *Fbx, double *Fby, double *Ux, double *Uy, double *rho_l)
{
    const ora_body *b = &s->b[body];
    size_t sz = sizeof(double) * b->n;
    if (Usx) memcpy(Usx, b->Usx, sz);
    if (Usy) memcpy(Usy, b->Usy, sz);
    if (Fbx) memcpy(Fbx, b->Fx, sz);
    if (Fby) memcpy(Fby, b->Fy, sz);
    if (Ux) memcpy(Ux, b->Ux, sz);
    if (Uy) memcpy(Uy, b->Uy, sz);
    if (rho_l) memcpy(rho_l, b->rho, sz);
}
