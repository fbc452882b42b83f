/*
 * oracle.h -- plain FP64 CPU oracle of the nonlocal hydrodynamic FDTD method
 * (Baxter, Cala Lesina, Ramunno, "Parallel FDTD modelling of nonlocality in
 * plasmonics", arXiv 2005.06997).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library: every formula here is written again from the paper.
 *
 * The oracle follows the paper's printed forms literally:
 *   - f1 (H update, Sec. III step (1), vacuum Faraday law),
 *   - Eq. GradDiv in its expanded three-term form per component,
 *   - f2 (E update) in the form obtained by substituting Eq. NonlocalUpdate /
 *     Eq. GNORUpdate and Eq. critpointupdate into Eq. discreteamperes,
 *   - f3 (Eq. critpointupdate) with P_CP^{n-1},
 *   - f4 (Eq. NonlocalUpdate or Eq. GNORUpdate) with P^{n-1}, and the stored
 *     grad-div histories GD^{n-1}, GD^{n-2} of Sec. III (GNOR memory note),
 *   - Pekar ABC: P_f is kept at zero outside the plasmonic material.
 * Units are SI throughout (E in V/m, H in A/m, P in C/m^2).
 *
 * Readings of points the paper leaves open (each is listed in the design
 * notes of the repository):
 *   1. sign of sum C4p in the E update: substituting f3 into Ampere's law
 *      gives -C4p (the printed +C4p contradicts Eq. critpointupdate);
 *   2. the sin(phi) terms of C3p/C5p carry 1/(dt*Cp), the central difference
 *      of the d/dt E term of Eq. CritPoint (the printed 1/(2 dt Cp) is not
 *      consistent with the continuous model);
 *   3. time convention exp(-i w t) (from the Drude form in Sec. II), so the
 *      running DFT uses exp(+i w t);
 *   7. CPML: polynomial grading m=3, sigma_max = 0.8 (m+1)/(eta0 dx sqrt(eps_b)),
 *      kappa = 1, alpha linear from 0.05 S/m at the inner edge to 0 at the outer
 *      edge, PEC behind it;
 *   8. TF/SF plane wave propagating +z, polarised along x, fed by a 1D
 *      auxiliary grid with the same dx, dt and a hard source;
 *  10. material of an E-site = first shape that contains its point (integer
 *      half-cell geometry, ties count as inside);
 *  11. DFT: rectangle rule every K steps, E at n*dt, H at (n-1/2)*dt;
 *      flux boxes with trapezoid edge weights; incident intensity from the 1D
 *      grid at the centre plane of the absorption box.
 */
#ifndef NLF_ORACLE_H
#define NLF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PEC = 0, ORC_BC_CPML = 1, ORC_BC_PERIODIC = 2 };
enum { ORC_SHAPE_SPHERE = 1, ORC_SHAPE_BOX = 2, ORC_SHAPE_CUBE_TIPS = 3 };
enum { ORC_WAVE_GAUSSIAN = 1, ORC_WAVE_RAISED_COS = 2 };

typedef struct {
    int nx, ny, nz;
    double dx;          /* m, uniform cubic cells */
    double courant;     /* S = c dt / dx */
    int pml;            /* CPML thickness in cells (axes with bc == CPML) */
    int bc[3];
    double eps_b;       /* background relative permittivity */
} orc_grid;

typedef struct {
    double eps_inf;     /* epsilon_infinity */
    double wp, gamma;   /* rad/s */
    double beta;        /* m/s */
    double diff;        /* m^2/s (GNOR diffusion D); 0 selects nonlocal Drude */
    int n_poles;        /* critical points, <= 4 */
    double A[4], Om[4], Ga[4], phi[4];
} orc_material;

/* Geometry in integer half-cell units: a point (2i+ox, 2j+oy, 2k+oz). */
typedef struct {
    int kind;
    int material;       /* 1-based index into the material table */
    int c[3];           /* centre */
    int radius;         /* sphere radius */
    int half[3];        /* box half extents */
    int side;           /* cube side (even) */
    int tip_base;       /* pyramid base width (even) */
    int tip_height;     /* pyramid height above the cube face */
    int tip_radius;     /* rounding sphere radius */
    int tip_center;     /* distance cube centre -> rounding sphere centre */
    int tip_cut;        /* pyramid kept only up to this distance from the centre */
} orc_shape;

typedef struct {
    int enabled;
    int tf_lo[3], tf_hi[3];  /* node indices of the total-field box */
    int waveform;
    double w0, tau, t0, amp; /* rad/s, s, s, V/m */
} orc_source;

typedef struct {
    int nf;
    const double* omega;     /* rad/s, nf values */
    int abs_lo[3], abs_hi[3];
    int sca_lo[3], sca_hi[3];
    int K;                   /* DFT decimation */
} orc_monitors;

typedef struct orc_sim orc_sim;

orc_sim* orc_create(const orc_grid* g, const orc_material* mats, int nmat,
                    const orc_shape* shapes, int nshapes, const uint8_t* map,
                    const orc_source* src, const orc_monitors* mon);
void     orc_destroy(orc_sim* s);
const char* orc_error(void);

void     orc_step(orc_sim* s, long long nsteps);
long long orc_time_index(const orc_sim* s);
double   orc_dt(const orc_sim* s);

/* Arrays owned by the simulation (x fastest: [nz][ny][nx]).
 * which: 0..2 E, 3..5 H, 6..8 P_f, 9..11 E^{n-1}, 12..14 P_f^{n-1},
 *        15..17 P_CP (pole 0), 18..20 P_CP^{n-1} (pole 0), 21..23 GD^{n-1},
 *        24..26 GD^{n-2}. */
double*  orc_array(orc_sim* s, int which);
uint8_t* orc_material_map(orc_sim* s, int comp);
/* 1D incident grid: which 0 = E_inc, 1 = H_inc; *len receives its length. */
double*  orc_inc_array(orc_sim* s, int which, int* len);
int      orc_inc_offset(const orc_sim* s);

/* Eq. GradDiv (expanded) applied to arbitrary P (3 arrays), masked to the
 * plasmonic sites of the simulation: out = grad(div P). */
void     orc_graddiv(const orc_sim* s, const double* const* P, double* const* out);

/* Coefficients exactly as used by the updates (SI). out_d: Dd,D1,D2,D3,DNL,DG1,DG2;
 * out_c (per pole, 6 values): Cp,C1,C2,C3,C4,C5. */
void     orc_coefficients(const orc_sim* s, int material, double* out_d, double* out_c);

/* Monitors. */
int      orc_num_records(const orc_sim* s);
/* rec: per record 10 ints: box (0 absorption, 1 scattering), normal axis a,
 * E component, E index (i,j,k), H component, first H index (i,j,k); the
 * second H point is the first shifted by +1 along axis a.  coef: double. */
void     orc_records(const orc_sim* s, int* rec, double* coef);
/* accumulators, complex, [nrec+1][nf][2] for E and H; the last record is the
 * incident field at the centre plane. */
void     orc_dft(const orc_sim* s, double* accE, double* accH);
void     orc_spectra(const orc_sim* s, double* s_ext, double* s_abs, double* s_sca, double* inc);

/* Single-frequency maps on one lattice plane (the near-field and
 * free-electron density maps of Sec. V): plane normal to `axis` (0, 1, 2) at
 * node index `index`; every K steps (at t = n dt, E^n and P_f^n current) the
 * running DFT, rectangle rule as for the flux monitors, of E_x, E_y, E_z at
 * the E-sites (i, j, k) of the plane and of the free-electron charge density
 * div P_f (C/m^3; Eq. Nsol gives n - n0 = div P_f / e) at its nodes, by the
 * backward differences of the Yee grid.  Set before the first step. */
typedef struct {
    int axis, index;
    int nf;
    const double* omega;     /* rad/s */
    int K;
} orc_plane;
int      orc_set_plane(orc_sim* s, const orc_plane* p);
/* which: 0..2 E_x..E_z, 3 density; out: [nf][n1][n2][2] where (n1, n2) are
 * the plane's extents along its two other axes, slow then fast, in axis
 * order (axis 0: [nz][ny], axis 1: [nz][nx], axis 2: [ny][nx]). */
void     orc_plane_dft(const orc_sim* s, int which, double* out);
/* div P_f^n at every node (C/m^3), [nz][ny][nx]. */
void     orc_density(const orc_sim* s, double* out);

#ifdef __cplusplus
}
#endif
#endif
