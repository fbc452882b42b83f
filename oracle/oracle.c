/*
 * oracle.c -- plain FP64 CPU oracle of the nonlocal hydrodynamic FDTD method
 * of arXiv 2005.06997.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Slow on purpose: full-grid FP64 arrays for every quantity, one function call
 * per neighbour read, no blocking or fusion.  The loops over z-planes may run
 * on several OpenMP threads; that does not change any arithmetic.
 *
 * Grid: nx*ny*nz cells, arrays [nz][ny][nx].  Positions (Table Yee):
 *   E_x(i,j,k) at (i+1/2, j, k)    H_x(i,j,k) at (i, j+1/2, k+1/2)
 *   E_y(i,j,k) at (i, j+1/2, k)    H_y(i,j,k) at (i+1/2, j, k+1/2)
 *   E_z(i,j,k) at (i, j, k+1/2)    H_z(i,j,k) at (i+1/2, j+1/2, k)
 * P_f and P_CP are collocated with E (Sec. III).  On a PEC (or CPML-backed)
 * axis the walls are at 0 and N cells; tangential E on index 0 is held at
 * zero and anything at index N or -1 reads as zero.  A periodic axis wraps.
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define EPS0 8.8541878128e-12
#define MU0  1.25663706212e-6

static char g_err[256];
const char* orc_error(void) { return g_err; }

typedef struct { double re, im; } cplx;

struct orc_sim {
    orc_grid g;
    double dt, c0, eta0;
    size_t ncell;
    int nmat;
    orc_material mat[256];
    uint8_t* map[3];            /* material id per E-site, 0 = background */

    double *E[3], *Eprev[3], *Enew[3];
    double *H[3];
    double *P[3], *Pprev[3], *Pnew[3];
    double *GD[3], *GD1[3], *GD2[3];
    double *Pcp[4][3], *Pcpprev[4][3], *Pcpnew[4][3];
    int max_poles;
    /* CPML auxiliaries, full grid: psiE[c][a] for component c, derivative axis a */
    double *psiE[3][3], *psiH[3][3];

    orc_source src;
    int inc_len, inc_off, inc_pml;
    double *Einc, *Hinc, *psiEinc, *psiHinc;

    orc_monitors mon;
    double* omega;
    int nrec;
    int* rec;                   /* 10 ints per record */
    double* coef;
    double* accE;               /* [(nrec+1)][nf][2] */
    double* accH;
    int inc_node;               /* 1D node of the centre plane */

    /* single-frequency plane maps */
    orc_plane pl;
    double* pl_omega;
    double* pl_acc;             /* [4][nf][n1][n2][2]: E_x, E_y, E_z, div P_f */

    long long n;                /* time index: E^n, H^{n-1/2} are current */

    /* filled once at creation from the formulas below */
    struct coefs_s* ctab;       /* [nmat + 1], index = material id */
    double* pml_b[3];           /* [2 n_axis + 2], index = half-cell position */
    double* pml_c[3];
};

/* ------------------------------------------------------------------ indexing */

static size_t at(const orc_sim* s, int i, int j, int k)
{
    return ((size_t)k * s->g.ny + (size_t)j) * s->g.nx + (size_t)i;
}

/* Map an index along an axis into the array; returns 0 if it lies outside a
 * non-periodic axis (the field there is zero). */
static int fix_index(const orc_sim* s, int axis, int* v)
{
    int n = axis == 0 ? s->g.nx : axis == 1 ? s->g.ny : s->g.nz;
    if (*v >= 0 && *v < n) return 1;
    if (s->g.bc[axis] == ORC_BC_PERIODIC) {
        *v = ((*v % n) + n) % n;
        return 1;
    }
    return 0;
}

static double rd(const orc_sim* s, const double* a, int i, int j, int k)
{
    if (!fix_index(s, 0, &i) || !fix_index(s, 1, &j) || !fix_index(s, 2, &k)) return 0.0;
    return a[at(s, i, j, k)];
}

/* Half-cell offsets of the Yee positions. */
static const int E_OFF[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
static const int H_OFF[3][3] = {{0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

/* ------------------------------------------------------------------ geometry */

static long long sq(long long v) { return v * v; }

/* Is the half-cell point p inside shape sh?  Pure integer arithmetic. */
static int shape_contains(const orc_shape* sh, const long long p[3])
{
    long long d[3] = {p[0] - sh->c[0], p[1] - sh->c[1], p[2] - sh->c[2]};
    if (sh->kind == ORC_SHAPE_SPHERE) {
        return sq(d[0]) + sq(d[1]) + sq(d[2]) <= sq(sh->radius);
    }
    if (sh->kind == ORC_SHAPE_BOX) {
        return llabs(d[0]) <= sh->half[0] && llabs(d[1]) <= sh->half[1] && llabs(d[2]) <= sh->half[2];
    }
    if (sh->kind == ORC_SHAPE_CUBE_TIPS) {
        long long A = sh->side / 2, B = sh->tip_base / 2, h = sh->tip_height;
        if (llabs(d[0]) <= A && llabs(d[1]) <= A && llabs(d[2]) <= A) return 1;
        /* six tips, one on each face centre, pointing along +-x, +-y, +-z */
        for (int ax = 0; ax < 3; ++ax) {
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                long long t = sgn * d[ax];
                long long v = llabs(d[(ax + 1) % 3]);
                long long w = llabs(d[(ax + 2) % 3]);
                /* rounding sphere on the tip axis */
                long long dc = t - sh->tip_center;
                if (sq(dc) + sq(v) + sq(w) <= sq(sh->tip_radius)) return 1;
                /* square pyramid: base 2B on the face t = A, apex at t = A + h,
                 * kept up to the cut plane */
                if (t >= A && t <= sh->tip_cut &&
                    h * v <= B * (A + h - t) && h * w <= B * (A + h - t))
                    return 1;
            }
        }
        return 0;
    }
    return 0;
}

static void voxelise(orc_sim* s, const orc_shape* shapes, int nshapes)
{
    for (int c = 0; c < 3; ++c) {
        for (int k = 0; k < s->g.nz; ++k)
            for (int j = 0; j < s->g.ny; ++j)
                for (int i = 0; i < s->g.nx; ++i) {
                    long long p[3] = {2LL * i + E_OFF[c][0], 2LL * j + E_OFF[c][1], 2LL * k + E_OFF[c][2]};
                    uint8_t id = 0;
                    for (int q = 0; q < nshapes; ++q) {
                        if (shape_contains(&shapes[q], p)) { id = (uint8_t)shapes[q].material; break; }
                    }
                    s->map[c][at(s, i, j, k)] = id;
                }
    }
}

/* ------------------------------------------------------------- coefficients */

typedef struct coefs_s {
    int plasmonic, npoles;
    double eps_inf;
    double Dd, D1, D2, D3, DNL, DG1, DG2;
    double Cp[4], C1[4], C2[4], C3[4], C4[4], C5[4];
} coefs;

/* Eqs. d1-dd, the GNOR coefficients D_G1, D_G2, and the critical-points
 * coefficients C_1p..C_5p, C_p of Sec. III, with reading 2 for the sin(phi)
 * terms of C_3p and C_5p. */
static coefs material_coefs(const orc_sim* s, int id)
{
    coefs k;
    memset(&k, 0, sizeof k);
    double dt = s->dt;
    if (id == 0) { k.eps_inf = s->g.eps_b; return k; }
    const orc_material* m = &s->mat[id - 1];
    k.eps_inf = m->eps_inf;
    k.plasmonic = m->wp > 0.0;
    if (k.plasmonic) {
        k.Dd = m->gamma / (2.0 * dt) + 1.0 / (dt * dt);
        k.D1 = 2.0 / (k.Dd * dt * dt);
        k.D2 = (m->gamma / (2.0 * dt) - 1.0 / (dt * dt)) / k.Dd;
        k.D3 = EPS0 * m->wp * m->wp / (4.0 * k.Dd);
        k.DNL = m->beta * m->beta / k.Dd;
        double eta = m->beta * m->beta + m->diff * m->gamma;
        k.DG1 = eta / k.Dd;
        k.DG2 = m->diff / (2.0 * dt * k.Dd);
    }
    k.npoles = m->n_poles;
    for (int p = 0; p < m->n_poles; ++p) {
        double A = m->A[p], Om = m->Om[p], Ga = m->Ga[p], ph = m->phi[p];
        double W2 = Om * Om + Ga * Ga;
        k.Cp[p] = Ga / dt + 1.0 / (dt * dt) + W2 / 4.0;
        k.C1[p] = (2.0 / (dt * dt) - W2 / 2.0) / k.Cp[p];
        k.C2[p] = (Ga / dt - 1.0 / (dt * dt) - W2 / 4.0) / k.Cp[p];
        k.C4[p] = EPS0 * A * Om * (Om * cos(ph) - Ga * sin(ph)) / k.Cp[p];
        k.C3[p] = k.C4[p] / 2.0 - EPS0 * A * Om * sin(ph) / (dt * k.Cp[p]);
        k.C5[p] = k.C4[p] / 2.0 + EPS0 * A * Om * sin(ph) / (dt * k.Cp[p]);
    }
    return k;
}

void orc_coefficients(const orc_sim* s, int material, double* out_d, double* out_c)
{
    coefs k = material_coefs(s, material);
    double d[7] = {k.Dd, k.D1, k.D2, k.D3, k.DNL, k.DG1, k.DG2};
    memcpy(out_d, d, sizeof d);
    for (int p = 0; p < k.npoles; ++p) {
        double c[6] = {k.Cp[p], k.C1[p], k.C2[p], k.C3[p], k.C4[p], k.C5[p]};
        memcpy(out_c + 6 * p, c, sizeof c);
    }
}

/* -------------------------------------------------------------------- CPML */

/* Depth into the CPML of a position x (cells, may be half-integer) on an axis
 * of n cells with a layer of L cells at each end, normalised to [0,1]. */
static double pml_depth(double x, int n, int L)
{
    if (L <= 0) return 0.0;
    double r = 0.0;
    if (x < L) r = (L - x) / L;
    else if (x > n - L) r = (x - (n - L)) / L;
    if (r < 0.0) r = 0.0;
    if (r > 1.0) r = 1.0;
    return r;
}

/* Reading 7: b = exp(-(sigma/kappa + alpha) dt/eps0), c = sigma (b-1)/(sigma kappa + kappa^2 alpha), kappa = 1. */
static void pml_bc(const orc_sim* s, double rho, double* b, double* c)
{
    const double m = 3.0;
    double sig_max = 0.8 * (m + 1.0) / (s->eta0 * s->g.dx * sqrt(s->g.eps_b));
    double sig = sig_max * pow(rho, m);
    double alpha = rho > 0.0 ? 0.05 * (1.0 - rho) : 0.0;
    *b = exp(-(sig + alpha) * s->dt / EPS0);
    *c = (sig + alpha) > 0.0 ? sig * (*b - 1.0) / (sig + alpha) : 0.0;
}

static int axis_n(const orc_sim* s, int a) { return a == 0 ? s->g.nx : a == 1 ? s->g.ny : s->g.nz; }

/* b,c for a field at half-cell coordinate hp along axis a. */
static void pml_axis_compute(const orc_sim* s, int a, long long hp, double* b, double* c)
{
    if (s->g.bc[a] != ORC_BC_CPML) { *b = 1.0; *c = 0.0; return; }
    pml_bc(s, pml_depth(0.5 * (double)hp, axis_n(s, a), s->g.pml), b, c);
}

static void pml_axis(const orc_sim* s, int a, long long hp, double* b, double* c)
{
    long long n2 = 2LL * axis_n(s, a) + 1;
    if (hp < 0 || hp > n2) { pml_axis_compute(s, a, hp, b, c); return; }
    *b = s->pml_b[a][hp];
    *c = s->pml_c[a][hp];
}

/* ------------------------------------------------------------------- TF/SF */

static int in_tf(const orc_sim* s, const long long p[3])
{
    if (!s->src.enabled) return 0;
    for (int a = 0; a < 3; ++a)
        if (p[a] < 2LL * s->src.tf_lo[a] || p[a] > 2LL * s->src.tf_hi[a]) return 0;
    return 1;
}

/* Incident plane wave: E_x and H_y only, functions of the z index. */
static double inc_E(const orc_sim* s, int comp, int k)
{
    if (!s->src.enabled || comp != 0) return 0.0;
    int m = k - s->inc_off;
    return (m >= 0 && m < s->inc_len) ? s->Einc[m] : 0.0;
}
static double inc_H(const orc_sim* s, int comp, int k)
{
    if (!s->src.enabled || comp != 1) return 0.0;
    int m = k - s->inc_off;
    return (m >= 0 && m < s->inc_len) ? s->Hinc[m] : 0.0;
}

/* Neighbour E (component c at i,j,k) as seen by an update at half-cell point
 * self: total and scattered fields are converted across the TF/SF surface. */
static double seen_E(const orc_sim* s, int c, int i, int j, int k, const long long self[3])
{
    double v = rd(s, s->E[c], i, j, k);
    long long p[3] = {2LL * i + E_OFF[c][0], 2LL * j + E_OFF[c][1], 2LL * k + E_OFF[c][2]};
    int d = in_tf(s, self) - in_tf(s, p);
    if (d != 0) v += d * inc_E(s, c, k);
    return v;
}
static double seen_H(const orc_sim* s, int c, int i, int j, int k, const long long self[3])
{
    double v = rd(s, s->H[c], i, j, k);
    long long p[3] = {2LL * i + H_OFF[c][0], 2LL * j + H_OFF[c][1], 2LL * k + H_OFF[c][2]};
    int d = in_tf(s, self) - in_tf(s, p);
    if (d != 0) v += d * inc_H(s, c, k);
    return v;
}

static double waveform(const orc_sim* s, double t)
{
    const orc_source* q = &s->src;
    if (q->waveform == ORC_WAVE_GAUSSIAN) {
        double u = (t - q->t0) / q->tau;
        return q->amp * exp(-u * u) * sin(q->w0 * (t - q->t0));
    }
    if (q->waveform == ORC_WAVE_RAISED_COS) {
        if (t < 0.0 || t > 2.0 * M_PI / q->w0) return 0.0;
        double r = (1.0 - cos(q->w0 * t)) / 2.0;
        return q->amp * r * r * r;
    }
    return 0.0;
}

/* 1D auxiliary grid: E_inc(m) at z = m, H_inc(m) at z = m + 1/2 (cells), a
 * CPML of inc_pml cells at the far end and a hard source at m = 0. */
static void inc_pml_bc(const orc_sim* s, double x, double* b, double* c)
{
    int start = s->inc_len - s->inc_pml;
    double rho = x > start ? (x - start) / s->inc_pml : 0.0;
    if (rho > 1.0) rho = 1.0;
    pml_bc(s, rho, b, c);
}

static void inc_update_H(orc_sim* s)
{
    double ch = s->dt / (MU0 * s->g.dx);
    for (int m = 0; m < s->inc_len; ++m) {
        double e1 = m + 1 < s->inc_len ? s->Einc[m + 1] : 0.0;
        double dE = e1 - s->Einc[m];
        double b, c;
        inc_pml_bc(s, m + 0.5, &b, &c);
        s->psiHinc[m] = b * s->psiHinc[m] + c * dE;
        s->Hinc[m] -= ch * (dE + s->psiHinc[m]);
    }
}

static void inc_update_E(orc_sim* s, double t_next)
{
    double ce = s->dt / (EPS0 * s->g.eps_b * s->g.dx);
    for (int m = 1; m < s->inc_len; ++m) {
        double dH = s->Hinc[m] - s->Hinc[m - 1];
        double b, c;
        inc_pml_bc(s, (double)m, &b, &c);
        s->psiEinc[m] = b * s->psiEinc[m] + c * dH;
        s->Einc[m] -= ce * (dH + s->psiEinc[m]);
    }
    s->Einc[0] = waveform(s, t_next);
}

/* ------------------------------------------------------------- f1: H update */

/* One H component at (i,j,k):  H^{n+1/2} = H^{n-1/2} - (dt/mu0) curl E^n,
 * with CPML on each derivative and TF/SF conversion of the E neighbours. */
static void update_H_site(orc_sim* s, int c, int i, int j, int k)
{
    long long self[3] = {2LL * i + H_OFF[c][0], 2LL * j + H_OFF[c][1], 2LL * k + H_OFF[c][2]};
    /* curl component c = d_b E_q - d_q E_b with (c, b, q) cyclic:
     * (curl E)_c = dE_{c+2}/dx_{c+1} - dE_{c+1}/dx_{c+2} */
    int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
    /* term 1: d E_{a2} / d x_{a1} */
    int n1[3] = {i, j, k};
    n1[a1] += 1;
    double t1 = seen_E(s, a2, n1[0], n1[1], n1[2], self) - seen_E(s, a2, i, j, k, self);
    /* term 2: d E_{a1} / d x_{a2} */
    int n2[3] = {i, j, k};
    n2[a2] += 1;
    double t2 = seen_E(s, a1, n2[0], n2[1], n2[2], self) - seen_E(s, a1, i, j, k, self);
    double b, cc;
    size_t q = at(s, i, j, k);
    pml_axis(s, a1, self[a1], &b, &cc);
    s->psiH[c][a1][q] = b * s->psiH[c][a1][q] + cc * t1;
    t1 += s->psiH[c][a1][q];
    pml_axis(s, a2, self[a2], &b, &cc);
    s->psiH[c][a2][q] = b * s->psiH[c][a2][q] + cc * t2;
    t2 += s->psiH[c][a2][q];
    s->H[c][q] -= s->dt / (MU0 * s->g.dx) * (t1 - t2);
}

static void update_H(orc_sim* s)
{
    for (int c = 0; c < 3; ++c) {
#pragma omp parallel for schedule(static)
        for (int k = 0; k < s->g.nz; ++k)
            for (int j = 0; j < s->g.ny; ++j)
                for (int i = 0; i < s->g.nx; ++i) update_H_site(s, c, i, j, k);
    }
}

/* ------------------------------------------------ Eq. GradDiv (expanded) */

static double rdP(const orc_sim* s, const double* const* P, int c, int i, int j, int k)
{
    return rd(s, P[c], i, j, k);
}

/* grad(div P) at the site of component c, (i,j,k), Eq. GradDiv (a)-(c):
 * the three-point second difference of P_c plus the two four-point cross
 * differences of the other components. */
static double graddiv_site(const orc_sim* s, const double* const* P, int c, int i, int j, int k)
{
    double h2 = s->g.dx * s->g.dx;
    int u[3] = {0, 0, 0};
    u[c] = 1;
    /* second difference along c */
    double v = rdP(s, P, c, i + u[0], j + u[1], k + u[2]) - 2.0 * rdP(s, P, c, i, j, k) +
               rdP(s, P, c, i - u[0], j - u[1], k - u[2]);
    for (int b = 0; b < 3; ++b) {
        if (b == c) continue;
        int w[3] = {0, 0, 0};
        w[b] = 1;
        /* P_b at (site + e_c) +- e_b/2 and at site +- e_b/2 (in index form:
         * P_b(idx + e_c), P_b(idx + e_c - e_b), P_b(idx), P_b(idx - e_b)) */
        v += rdP(s, P, b, i + u[0], j + u[1], k + u[2]) -
             rdP(s, P, b, i + u[0] - w[0], j + u[1] - w[1], k + u[2] - w[2]) -
             rdP(s, P, b, i, j, k) + rdP(s, P, b, i - w[0], j - w[1], k - w[2]);
    }
    return v / h2;
}

static int site_plasmonic(const orc_sim* s, int c, size_t q)
{
    uint8_t id = s->map[c][q];
    return id != 0 && s->mat[id - 1].wp > 0.0;
}

void orc_graddiv(const orc_sim* s, const double* const* P, double* const* out)
{
    for (int c = 0; c < 3; ++c) {
#pragma omp parallel for schedule(static)
        for (int k = 0; k < s->g.nz; ++k)
            for (int j = 0; j < s->g.ny; ++j)
                for (int i = 0; i < s->g.nx; ++i) {
                    size_t q = at(s, i, j, k);
                    out[c][q] = site_plasmonic(s, c, q) ? graddiv_site(s, P, c, i, j, k) : 0.0;
                }
    }
}

/* ------------------------------------------------- f2, f3, f4 (E, P_CP, P_f) */

/* Is cell (i, j, k) inside a CPML slab (index < L or >= n - L along a CPML
 * axis)?  Sec. III keeps the nonlocal response out of the PML: a nonlocal
 * material that reaches into it (a substrate, say) is updated there with the
 * local (LRA) Drude model, beta = D = 0. */
static int in_cpml_cell(const orc_sim* s, int i, int j, int k)
{
    const int ix[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        if (s->g.bc[a] != ORC_BC_CPML) continue;
        if (ix[a] < s->g.pml || ix[a] >= axis_n(s, a) - s->g.pml) return 1;
    }
    return 0;
}

/* Tangential E on index 0 of a non-periodic axis is the PEC wall. */
static int E_updated(const orc_sim* s, int c, int i, int j, int k)
{
    int ix[3] = {i, j, k};
    for (int a = 0; a < 3; ++a)
        if (a != c && s->g.bc[a] != ORC_BC_PERIODIC && ix[a] == 0) return 0;
    return 1;
}

/* (curl H^{n+1/2})_c at E-site (c,i,j,k), times dx, with CPML and TF/SF. */
static double curl_H_site(orc_sim* s, int c, int i, int j, int k)
{
    long long self[3] = {2LL * i + E_OFF[c][0], 2LL * j + E_OFF[c][1], 2LL * k + E_OFF[c][2]};
    int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
    /* (curl H)_c = dH_{a2}/dx_{a1} - dH_{a1}/dx_{a2}; H sits half a cell
     * above the E point along the derivative axis, so the difference is
     * H(idx) - H(idx - e_axis). */
    int n1[3] = {i, j, k};
    n1[a1] -= 1;
    double t1 = seen_H(s, a2, i, j, k, self) - seen_H(s, a2, n1[0], n1[1], n1[2], self);
    int n2[3] = {i, j, k};
    n2[a2] -= 1;
    double t2 = seen_H(s, a1, i, j, k, self) - seen_H(s, a1, n2[0], n2[1], n2[2], self);
    double b, cc;
    size_t q = at(s, i, j, k);
    pml_axis(s, a1, self[a1], &b, &cc);
    s->psiE[c][a1][q] = b * s->psiE[c][a1][q] + cc * t1;
    t1 += s->psiE[c][a1][q];
    pml_axis(s, a2, self[a2], &b, &cc);
    s->psiE[c][a2][q] = b * s->psiE[c][a2][q] + cc * t2;
    t2 += s->psiE[c][a2][q];
    return t1 - t2;
}

static void update_E_P(orc_sim* s)
{
    double dt = s->dt;
    for (int c = 0; c < 3; ++c) {
#pragma omp parallel for schedule(static)
        for (int k = 0; k < s->g.nz; ++k)
            for (int j = 0; j < s->g.ny; ++j)
                for (int i = 0; i < s->g.nx; ++i) {
                    size_t q = at(s, i, j, k);
                    uint8_t id = s->map[c][q];
                    coefs m = s->ctab[id];
                    if (m.plasmonic && in_cpml_cell(s, i, j, k)) {
                        /* local Drude inside the CPML (Sec. III): no pressure or diffusion term */
                        m.DNL = 0.0;
                        m.DG1 = 0.0;
                        m.DG2 = 0.0;
                    }
                    double En = s->E[c][q], Em = s->Eprev[c][q];
                    if (!E_updated(s, c, i, j, k)) {
                        s->Enew[c][q] = En;
                        s->Pnew[c][q] = s->P[c][q];
                        for (int p = 0; p < s->max_poles; ++p) s->Pcpnew[p][c][q] = s->Pcp[p][c][q];
                        continue;
                    }
                    double curl = curl_H_site(s, c, i, j, k) / s->g.dx;
                    double Enext;
                    if (!m.plasmonic && m.npoles == 0) {
                        /* LRA dielectric: eps0 eps (E^{n+1}-E^n)/dt = curl H */
                        Enext = En + dt * curl / (EPS0 * m.eps_inf);
                    } else {
                        /* f2: Eq. discreteamperes with f3 and f4 substituted (reading 1: -sum C4p) */
                        double den = EPS0 * m.eps_inf + m.D3;
                        double num = dt * curl + (EPS0 * m.eps_inf - 2.0 * m.D3) * En - m.D3 * Em;
                        if (m.plasmonic) {
                            double gd = s->GD[c][q];
                            num -= (m.D1 - 1.0) * s->P[c][q] + m.D2 * s->Pprev[c][q];
                            if (s->mat[id - 1].diff == 0.0) {
                                num -= m.DNL * gd;
                            } else {
                                num -= m.DG1 * gd + m.DG2 * (3.0 * gd - 4.0 * s->GD1[c][q] + s->GD2[c][q]);
                            }
                        }
                        for (int p = 0; p < m.npoles; ++p) {
                            den += m.C3[p];
                            num -= m.C4[p] * En;
                            num -= m.C5[p] * Em;
                            num -= (m.C1[p] - 1.0) * s->Pcp[p][c][q] + m.C2[p] * s->Pcpprev[p][c][q];
                        }
                        Enext = num / den;
                    }
                    s->Enew[c][q] = Enext;
                    /* f3: Eq. critpointupdate */
                    for (int p = 0; p < s->max_poles; ++p) {
                        if (p < m.npoles)
                            s->Pcpnew[p][c][q] = m.C1[p] * s->Pcp[p][c][q] + m.C2[p] * s->Pcpprev[p][c][q] +
                                                 m.C3[p] * Enext + m.C4[p] * En + m.C5[p] * Em;
                        else
                            s->Pcpnew[p][c][q] = 0.0;
                    }
                    /* f4: Eq. NonlocalUpdate / Eq. GNORUpdate; Pekar: P_f = 0 off the metal */
                    if (m.plasmonic) {
                        double gd = s->GD[c][q];
                        double Pn = m.D1 * s->P[c][q] + m.D2 * s->Pprev[c][q] + m.D3 * (Em + 2.0 * En + Enext);
                        if (s->mat[id - 1].diff == 0.0)
                            Pn += m.DNL * gd;
                        else
                            Pn += m.DG1 * gd + m.DG2 * (3.0 * gd - 4.0 * s->GD1[c][q] + s->GD2[c][q]);
                        s->Pnew[c][q] = Pn;
                    } else {
                        s->Pnew[c][q] = 0.0;
                    }
                }
    }
}

/* --------------------------------------------------------------- monitors */

/* Face records of a flux box [lo,hi] (node indices).  For the face with
 * normal axis a at plane p, with (a, b, c) cyclic, S_a = E_b H_c - E_c H_b:
 *   term +E_b H_c: E_b at b-index t_b in [lo_b, hi_b-1], c-index t_c in
 *     [lo_c, hi_c]; H_c averaged over a-index p-1 and p; weight 1/2 on the
 *     edges t_c = lo_c, hi_c;
 *   term -E_c H_b: E_c at t_c in [lo_c, hi_c-1], t_b in [lo_b, hi_b]; H_b
 *     averaged likewise; weight 1/2 on t_b = lo_b, hi_b.
 * coef = (outward sign) * (term sign) * weight / 2.  Loop order: box, a,
 * low face then high face, term, slower in-plane axis outer, faster inner. */
static int build_box(int box, const int lo[3], const int hi[3], int* rec, double* coef)
{
    int n = 0;
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        int slow = b > c ? b : c, fast = b > c ? c : b;
        for (int side = 0; side < 2; ++side) {
            int p = side == 0 ? lo[a] : hi[a];
            double outward = side == 0 ? -1.0 : 1.0;
            for (int term = 0; term < 2; ++term) {
                int ecomp = term == 0 ? b : c;
                int hcomp = term == 0 ? c : b;
                double tsign = term == 0 ? 1.0 : -1.0;
                int lo_s = lo[slow], hi_s = ecomp == slow ? hi[slow] - 1 : hi[slow];
                int lo_f = lo[fast], hi_f = ecomp == fast ? hi[fast] - 1 : hi[fast];
                for (int ts = lo_s; ts <= hi_s; ++ts)
                    for (int tf = lo_f; tf <= hi_f; ++tf) {
                        int idx[3];
                        idx[a] = p;
                        idx[slow] = ts;
                        idx[fast] = tf;
                        /* the in-plane axis other than ecomp carries the trapezoid weight */
                        int other = ecomp == b ? c : b;
                        double w = (idx[other] == lo[other] || idx[other] == hi[other]) ? 0.5 : 1.0;
                        if (rec) {
                            int* r = rec + 10 * n;
                            r[0] = box; r[1] = a; r[2] = ecomp;
                            r[3] = idx[0]; r[4] = idx[1]; r[5] = idx[2];
                            r[6] = hcomp;
                            int h[3] = {idx[0], idx[1], idx[2]};
                            h[a] = p - 1;
                            r[7] = h[0]; r[8] = h[1]; r[9] = h[2];
                            coef[n] = outward * tsign * w * 0.5;
                        }
                        ++n;
                    }
            }
        }
    }
    return n;
}

static void build_records(orc_sim* s)
{
    int n0 = build_box(0, s->mon.abs_lo, s->mon.abs_hi, NULL, NULL);
    int n1 = build_box(1, s->mon.sca_lo, s->mon.sca_hi, NULL, NULL);
    s->nrec = n0 + n1;
    s->rec = (int*)malloc(sizeof(int) * 10 * (size_t)s->nrec);
    s->coef = (double*)malloc(sizeof(double) * (size_t)s->nrec);
    build_box(0, s->mon.abs_lo, s->mon.abs_hi, s->rec, s->coef);
    build_box(1, s->mon.sca_lo, s->mon.sca_hi, s->rec + 10 * n0, s->coef + n0);
    size_t na = (size_t)(s->nrec + 1) * s->mon.nf * 2;
    s->accE = (double*)calloc(na, sizeof(double));
    s->accH = (double*)calloc(na, sizeof(double));
    int kc = (s->mon.abs_lo[2] + s->mon.abs_hi[2]) / 2;
    s->inc_node = kc - s->inc_off;
}

/* div P_f at node (i, j, k): P_a lives at the E_a site half a cell up the
 * a axis, so the divergence at the node takes P_a(node) - P_a(node - e_a)
 * over dx for each axis (outside the grid P_f is zero). */
static double density_at(const orc_sim* s, int i, int j, int k)
{
    double d = rd(s, s->P[0], i, j, k) - rd(s, s->P[0], i - 1, j, k);
    d += rd(s, s->P[1], i, j, k) - rd(s, s->P[1], i, j - 1, k);
    d += rd(s, s->P[2], i, j, k) - rd(s, s->P[2], i, j, k - 1);
    return d / s->g.dx;
}

void orc_density(const orc_sim* s, double* out)
{
    for (int k = 0; k < s->g.nz; ++k)
        for (int j = 0; j < s->g.ny; ++j)
            for (int i = 0; i < s->g.nx; ++i) out[at(s, i, j, k)] = density_at(s, i, j, k);
}

static void plane_extents(const orc_sim* s, int* n1, int* n2)
{
    const int n3[3] = {s->g.nx, s->g.ny, s->g.nz};
    const int a = s->pl.axis;
    const int slow = a == 2 ? 1 : 2, fast = a == 0 ? 1 : 0;
    *n1 = n3[slow];
    *n2 = n3[fast];
}

int orc_set_plane(orc_sim* s, const orc_plane* p)
{
    const int n3[3] = {s->g.nx, s->g.ny, s->g.nz};
    if (p->axis < 0 || p->axis > 2 || p->index < 0 || p->index >= n3[p->axis] || p->nf < 1 || p->K < 1 || s->n != 0)
        return -1;
    s->pl = *p;
    s->pl_omega = (double*)malloc(sizeof(double) * (size_t)p->nf);
    memcpy(s->pl_omega, p->omega, sizeof(double) * (size_t)p->nf);
    s->pl.omega = s->pl_omega;
    int n1, n2;
    plane_extents(s, &n1, &n2);
    s->pl_acc = (double*)calloc((size_t)4 * p->nf * n1 * n2 * 2, sizeof(double));
    return 0;
}

/* Plane maps (rectangle rule, reading 11): F(w) += f * exp(+i w n dt) * K dt. */
static void plane_accumulate(orc_sim* s)
{
    int n1, n2;
    plane_extents(s, &n1, &n2);
    const int a = s->pl.axis, nf = s->pl.nf;
    const int slow = a == 2 ? 1 : 2, fast = a == 0 ? 1 : 0;
    const double t = s->n * s->dt, scale = s->pl.K * s->dt;
    const size_t per = (size_t)nf * n1 * n2 * 2;
#pragma omp parallel for schedule(static)
    for (int u = 0; u < n1; ++u)
        for (int v = 0; v < n2; ++v) {
            int idx[3];
            idx[a] = s->pl.index;
            idx[slow] = u;
            idx[fast] = v;
            double val[4];
            for (int c = 0; c < 3; ++c) val[c] = s->E[c][at(s, idx[0], idx[1], idx[2])];
            val[3] = density_at(s, idx[0], idx[1], idx[2]);
            for (int f = 0; f < nf; ++f) {
                const double w = s->pl.omega[f];
                const double cr = cos(w * t) * scale, ci = sin(w * t) * scale;
                for (int q = 0; q < 4; ++q) {
                    double* o = s->pl_acc + q * per + (((size_t)f * n1 + u) * n2 + v) * 2;
                    o[0] += val[q] * cr;
                    o[1] += val[q] * ci;
                }
            }
        }
}

void orc_plane_dft(const orc_sim* s, int which, double* out)
{
    int n1, n2;
    if (!s->pl_acc || which < 0 || which > 3) return;
    plane_extents(s, &n1, &n2);
    const size_t per = (size_t)s->pl.nf * n1 * n2 * 2;
    memcpy(out, s->pl_acc + which * per, per * sizeof(double));
}

/* Running DFT (reading 11): called when n is a multiple of K, with E^n and
 * H^{n-1/2} current.  F(w) += f * exp(+i w t) * K dt. */
static void dft_accumulate(orc_sim* s)
{
    int nf = s->mon.nf;
    double scale = s->mon.K * s->dt;
    double tE = s->n * s->dt, tH = (s->n - 0.5) * s->dt;
#pragma omp parallel for schedule(static)
    for (int r = 0; r <= s->nrec; ++r) {
        double e, h;
        if (r < s->nrec) {
            const int* q = s->rec + 10 * r;
            e = s->E[q[2]][at(s, q[3], q[4], q[5])];
            int h2[3] = {q[7], q[8], q[9]};
            h2[q[1]] += 1;
            h = 0.5 * (rd(s, s->H[q[6]], q[7], q[8], q[9]) + rd(s, s->H[q[6]], h2[0], h2[1], h2[2]));
        } else {
            int m = s->inc_node;
            e = s->Einc[m];
            h = 0.5 * (s->Hinc[m - 1] + s->Hinc[m]);
        }
        for (int f = 0; f < nf; ++f) {
            double w = s->omega[f];
            double* aE = s->accE + ((size_t)r * nf + f) * 2;
            double* aH = s->accH + ((size_t)r * nf + f) * 2;
            aE[0] += e * cos(w * tE) * scale;
            aE[1] += e * sin(w * tE) * scale;
            aH[0] += h * cos(w * tH) * scale;
            aH[1] += h * sin(w * tH) * scale;
        }
    }
}

int orc_num_records(const orc_sim* s) { return s->nrec; }

void orc_records(const orc_sim* s, int* rec, double* coef)
{
    memcpy(rec, s->rec, sizeof(int) * 10 * (size_t)s->nrec);
    memcpy(coef, s->coef, sizeof(double) * (size_t)s->nrec);
}

void orc_dft(const orc_sim* s, double* accE, double* accH)
{
    size_t na = (size_t)(s->nrec + 1) * s->mon.nf * 2;
    memcpy(accE, s->accE, na * sizeof(double));
    memcpy(accH, s->accH, na * sizeof(double));
}

/* sigma_abs = -(1/I) sum_abs coef Re(E H*) dA,  sigma_sca = +(1/I) sum_sca ...,
 * I = Re(E_inc H_inc*)/2, sigma_ext = sigma_abs + sigma_sca (reading of
 * Sec. V's absorption cross-sections). */
void orc_spectra(const orc_sim* s, double* s_ext, double* s_abs, double* s_sca, double* inc)
{
    int nf = s->mon.nf;
    double dA = s->g.dx * s->g.dx;
    for (int f = 0; f < nf; ++f) {
        double sum[2] = {0.0, 0.0};
        for (int r = 0; r < s->nrec; ++r) {
            const double* e = s->accE + ((size_t)r * nf + f) * 2;
            const double* h = s->accH + ((size_t)r * nf + f) * 2;
            double re = e[0] * h[0] + e[1] * h[1];
            sum[s->rec[10 * r]] += s->coef[r] * re;
        }
        const double* e = s->accE + ((size_t)s->nrec * nf + f) * 2;
        const double* h = s->accH + ((size_t)s->nrec * nf + f) * 2;
        double I = 0.5 * (e[0] * h[0] + e[1] * h[1]);
        double sa = -sum[0] * dA / I, ss = sum[1] * dA / I;
        if (s_abs) s_abs[f] = sa;
        if (s_sca) s_sca[f] = ss;
        if (s_ext) s_ext[f] = sa + ss;
        if (inc) inc[f] = I;
    }
}

/* -------------------------------------------------------------- lifecycle */

static double* zalloc(size_t n)
{
    double* p = (double*)calloc(n, sizeof(double));
    return p;
}

orc_sim* orc_create(const orc_grid* g, const orc_material* mats, int nmat,
                    const orc_shape* shapes, int nshapes, const uint8_t* map,
                    const orc_source* src, const orc_monitors* mon)
{
    g_err[0] = 0;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->dx <= 0.0 || nmat < 0 || nmat > 255) {
        snprintf(g_err, sizeof g_err, "bad grid or material count");
        return NULL;
    }
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->g = *g;
    s->c0 = 1.0 / sqrt(EPS0 * MU0);
    s->eta0 = sqrt(MU0 / EPS0);
    s->dt = g->courant * g->dx / s->c0;
    s->ncell = (size_t)g->nx * g->ny * g->nz;
    s->nmat = nmat;
    for (int m = 0; m < nmat; ++m) {
        s->mat[m] = mats[m];
        if (mats[m].n_poles > s->max_poles) s->max_poles = mats[m].n_poles;
    }
    for (int c = 0; c < 3; ++c) {
        s->map[c] = (uint8_t*)calloc(s->ncell, 1);
        s->E[c] = zalloc(s->ncell); s->Eprev[c] = zalloc(s->ncell); s->Enew[c] = zalloc(s->ncell);
        s->H[c] = zalloc(s->ncell);
        s->P[c] = zalloc(s->ncell); s->Pprev[c] = zalloc(s->ncell); s->Pnew[c] = zalloc(s->ncell);
        s->GD[c] = zalloc(s->ncell); s->GD1[c] = zalloc(s->ncell); s->GD2[c] = zalloc(s->ncell);
        for (int p = 0; p < s->max_poles; ++p) {
            s->Pcp[p][c] = zalloc(s->ncell); s->Pcpprev[p][c] = zalloc(s->ncell); s->Pcpnew[p][c] = zalloc(s->ncell);
        }
        for (int a = 0; a < 3; ++a) {
            if (a == c) continue;
            s->psiE[c][a] = zalloc(s->ncell);
            s->psiH[c][a] = zalloc(s->ncell);
        }
    }
    if (map) {
        for (int c = 0; c < 3; ++c) memcpy(s->map[c], map + (size_t)c * s->ncell, s->ncell);
    } else {
        voxelise(s, shapes, nshapes);
    }
    s->ctab = (coefs*)calloc((size_t)nmat + 1, sizeof(coefs));
    for (int m = 0; m <= nmat; ++m) s->ctab[m] = material_coefs(s, m);
    for (int a = 0; a < 3; ++a) {
        int n2 = 2 * axis_n(s, a) + 2;
        s->pml_b[a] = zalloc((size_t)n2);
        s->pml_c[a] = zalloc((size_t)n2);
        for (int hp = 0; hp < n2; ++hp) pml_axis_compute(s, a, hp, &s->pml_b[a][hp], &s->pml_c[a][hp]);
    }
    if (src && src->enabled) {
        s->src = *src;
        s->inc_off = src->tf_lo[2] - 3;
        s->inc_pml = 40;
        s->inc_len = (src->tf_hi[2] - s->inc_off + 1) + 10 + s->inc_pml;
        s->Einc = zalloc((size_t)s->inc_len); s->Hinc = zalloc((size_t)s->inc_len);
        s->psiEinc = zalloc((size_t)s->inc_len); s->psiHinc = zalloc((size_t)s->inc_len);
    }
    if (mon && mon->nf > 0) {
        if (!(src && src->enabled)) {
            snprintf(g_err, sizeof g_err, "monitors need a source");
            orc_destroy(s);
            return NULL;
        }
        s->mon = *mon;
        s->omega = (double*)malloc(sizeof(double) * (size_t)mon->nf);
        memcpy(s->omega, mon->omega, sizeof(double) * (size_t)mon->nf);
        s->mon.omega = s->omega;
        build_records(s);
    }
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    for (int c = 0; c < 3; ++c) {
        free(s->map[c]); free(s->E[c]); free(s->Eprev[c]); free(s->Enew[c]); free(s->H[c]);
        free(s->P[c]); free(s->Pprev[c]); free(s->Pnew[c]);
        free(s->GD[c]); free(s->GD1[c]); free(s->GD2[c]);
        for (int p = 0; p < 4; ++p) { free(s->Pcp[p][c]); free(s->Pcpprev[p][c]); free(s->Pcpnew[p][c]); }
        for (int a = 0; a < 3; ++a) { free(s->psiE[c][a]); free(s->psiH[c][a]); }
    }
    free(s->Einc); free(s->Hinc); free(s->psiEinc); free(s->psiHinc);
    free(s->omega); free(s->rec); free(s->coef); free(s->accE); free(s->accH);
    free(s->ctab);
    free(s->pl_omega);
    free(s->pl_acc);
    for (int a = 0; a < 3; ++a) { free(s->pml_b[a]); free(s->pml_c[a]); }
    free(s);
}

static void swap(double** a, double** b) { double* t = *a; *a = *b; *b = t; }

/* One time step n -> n+1 in the order of Sec. III: f1, f2, f3, f4. */
static void one_step(orc_sim* s)
{
    update_H(s);                                   /* H^{n+1/2} (uses E_inc^n) */
    if (s->src.enabled) inc_update_H(s);           /* H_inc^{n+1/2} */
    orc_graddiv(s, (const double* const*)s->P, s->GD);   /* GD^n */
    update_E_P(s);                                 /* E^{n+1}, P_CP^{n+1}, P_f^{n+1} */
    if (s->src.enabled) inc_update_E(s, (s->n + 1) * s->dt);
    for (int c = 0; c < 3; ++c) {
        /* E^{n-1} <- E^n <- E^{n+1}; P likewise; GD^{n-2} <- GD^{n-1} <- GD^n */
        swap(&s->Eprev[c], &s->E[c]);
        swap(&s->E[c], &s->Enew[c]);
        swap(&s->Pprev[c], &s->P[c]);
        swap(&s->P[c], &s->Pnew[c]);
        swap(&s->GD2[c], &s->GD1[c]);
        swap(&s->GD1[c], &s->GD[c]);
        for (int p = 0; p < s->max_poles; ++p) {
            swap(&s->Pcpprev[p][c], &s->Pcp[p][c]);
            swap(&s->Pcp[p][c], &s->Pcpnew[p][c]);
        }
    }
    s->n += 1;
    if (s->nrec > 0 && s->n % s->mon.K == 0) dft_accumulate(s);
    if (s->pl_acc && s->n % s->pl.K == 0) plane_accumulate(s);
}

void orc_step(orc_sim* s, long long nsteps)
{
    for (long long t = 0; t < nsteps; ++t) one_step(s);
}

long long orc_time_index(const orc_sim* s) { return s->n; }
double orc_dt(const orc_sim* s) { return s->dt; }

double* orc_array(orc_sim* s, int which)
{
    int c = which % 3;
    switch (which / 3) {
    case 0: return s->E[c];
    case 1: return s->H[c];
    case 2: return s->P[c];
    case 3: return s->Eprev[c];
    case 4: return s->Pprev[c];
    case 5: return s->max_poles > 0 ? s->Pcp[0][c] : NULL;
    case 6: return s->max_poles > 0 ? s->Pcpprev[0][c] : NULL;
    case 7: return s->GD1[c];
    case 8: return s->GD2[c];
    }
    return NULL;
}

uint8_t* orc_material_map(orc_sim* s, int comp) { return s->map[comp]; }

double* orc_inc_array(orc_sim* s, int which, int* len)
{
    *len = s->inc_len;
    return which == 0 ? s->Einc : s->Hinc;
}

int orc_inc_offset(const orc_sim* s) { return s->inc_off; }
