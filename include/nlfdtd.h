/*
 * nlfdtd.h -- C ABI of the GB300 (sm_103a) nonlocal hydrodynamic FDTD library.
 *
 * The library advances the 3D Yee FDTD scheme with the linear hydrodynamic
 * free-electron response of Baxter, Cala Lesina and Ramunno, "Parallel FDTD
 * modelling of nonlocality in plasmonics" (arXiv 2005.06997):
 *   - Sec. III, update order f1 (H), f2 (E), f3 (P_CP), f4 (P_f), Table Yee;
 *   - Eq. NonlocalUpdate (nonlocal Drude) and Eq. GNORUpdate (GNOR), with the
 *     grad(div P) stencil of Eq. GradDiv, the Pekar condition P_f = 0 outside
 *     the metal, nonlocal metal only inside the total-field region;
 *   - Eq. critpointupdate (critical-points bound-electron poles);
 *   - Eq. discreteamperes for the E update;
 *   - CPML absorbing boundaries, a TF/SF plane-wave source and running-DFT
 *     flux monitors for the absorption / scattering / extinction cross
 *     sections of Sec. V.
 * One context holds one grid on one GPU.  All functions are plain C; pointers
 * are host pointers unless the argument says "device".  Every function that
 * returns int returns NLF_OK (0) or a negative NLF_E_* code; the text of the
 * last error of a context is available from nlf_last_error().
 *
 * Units at the boundary are SI: metres, seconds, rad/s, V/m (E), A/m (H),
 * C/m^2 (P).  Geometry is given in integer half-cell units: a point with
 * half-cell coordinates (p0, p1, p2) sits at (p0, p1, p2) * dx / 2.
 *
 * Field arrays are [nz][ny][nx] with x fastest.  E_x(i,j,k) sits at
 * (i+1/2, j, k) dx, E_y at (i, j+1/2, k), E_z at (i, j, k+1/2); H_x at
 * (i, j+1/2, k+1/2), H_y at (i+1/2, j, k+1/2), H_z at (i+1/2, j+1/2, k)
 * (Table Yee).  The outer wall of every axis is a PEC at 0 and n cells:
 * tangential E on index 0 stays zero.
 *
 * Thread safety: a context may be used by one host thread at a time;
 * contexts share nothing.
 */
#ifndef NLFDTD_H
#define NLFDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NLF_OK             0
#define NLF_E_ARG         (-1)  /* bad argument or inconsistent sizes */
#define NLF_E_CFL         (-2)  /* S > 1/sqrt(3), or beta dt sqrt(3)/dx > 1 */
#define NLF_E_GEOMETRY    (-3)  /* metal near a wall or the TF surface, bad boxes */
#define NLF_E_OOM         (-4)  /* device allocation failed or bound buffer too small */
#define NLF_E_CUDA        (-5)  /* a CUDA call failed */
#define NLF_E_UNSTABLE    (-6)  /* a non-finite field was detected */
#define NLF_E_TIMEOUT     (-7)  /* nlf_sync gave up waiting */
#define NLF_E_STATE       (-8)  /* call made in the wrong order */
#define NLF_E_UNSUPPORTED (-9)  /* valid request outside what this build implements */

/* Boundary of each axis: a PEC wall, or a CPML of pml_cells in front of it
 * (the absorbing boundary of Sec. V, with the coefficients of the
 * convolutional PML; the paper gives the thickness only). */
#define NLF_BC_PEC       0
#define NLF_BC_CPML      1      /* CPML of pml_cells, PEC behind it */

#define NLF_SHAPE_SPHERE     1
#define NLF_SHAPE_BOX        2
#define NLF_SHAPE_CUBE_TIPS  3

#define NLF_WAVE_GAUSSIAN    1  /* amplitude exp(-((t-t0)/tau)^2) sin(w0 (t-t0)) */
#define NLF_WAVE_RAISED_COS  2  /* amplitude [(1-cos(w0 t))/2]^3 for 0 <= t <= 2 pi/w0 (Sec. V) */

#define NLF_FIELD_EX 0
#define NLF_FIELD_EY 1
#define NLF_FIELD_EZ 2
#define NLF_FIELD_HX 3
#define NLF_FIELD_HY 4
#define NLF_FIELD_HZ 5
#define NLF_FIELD_PX 6          /* free-electron polarisation P_f (Sec. III) */
#define NLF_FIELD_PY 7
#define NLF_FIELD_PZ 8
#define NLF_FIELD_DENSITY 9     /* free-electron charge density div P_f at the nodes (Eq. Nsol), C/m^3 */

#define NLF_MAX_POLES      4
#define NLF_MAX_MATERIALS  32
#define NLF_MAX_SHAPES     16

/* Grid (Sec. III, Sec. IV): uniform cubic cells dx, time step dt = S dx / c. */
typedef struct {
    int nx, ny, nz;           /* cells, each >= 8 */
    double dx;                /* m */
    double courant;           /* S = c dt / dx, 0 < S <= 1/sqrt(3) */
    int pml_cells;            /* CPML thickness on CPML axes */
    int boundary[3];          /* NLF_BC_* per axis */
    double eps_background;    /* relative permittivity of the background */
} nlf_grid;

/* Material (Sec. II): eps_inf, free electrons (Eq. NonlocDrude / Eq. GNOR)
 * and critical points (Eq. CritPoint).  wp = 0 means no free electrons;
 * beta = diff = 0 gives the local Drude model; diff > 0 selects GNOR. */
typedef struct {
    double eps_inf;
    double wp, gamma;         /* rad/s */
    double beta;              /* m/s */
    double diff;              /* m^2/s */
    int n_poles;              /* 0..NLF_MAX_POLES */
    double A[NLF_MAX_POLES], Omega[NLF_MAX_POLES], Gamma[NLF_MAX_POLES], phi[NLF_MAX_POLES];
} nlf_material;

/* Shape, integer half-cell units.  The material of an E-site is that of the
 * first shape (lowest index) containing its point; ties count as inside.
 *   SPHERE:    |p - center|^2 <= radius^2
 *   BOX:       |p_a - center_a| <= half[a] for all a
 *   CUBE_TIPS: cube |p_a - c_a| <= side/2, plus on each of its six face centres
 *              a square pyramid of base tip_base (even) and height tip_height,
 *              kept up to tip_cut from the centre, united with a sphere of
 *              radius tip_radius centred tip_center from the centre on the
 *              tip axis (the rounded apex). */
typedef struct {
    int kind;
    int material;             /* 1-based index into the material table */
    int center[3];
    int radius;
    int half[3];
    int side;
    int tip_base, tip_height, tip_radius, tip_center, tip_cut;
} nlf_shape;

/* TF/SF plane-wave source (Sec. III: nonlocal metal only in the TF region).
 * Propagation +z (axis_prop = 2), polarisation x (axis_pol = 0).  The TF box
 * is given in node indices: E_x(i,j,k) is a total field iff
 * tf_lo[0] <= i < tf_hi[0], tf_lo[1] <= j <= tf_hi[1], tf_lo[2] <= k <= tf_hi[2]
 * (in general: its point lies in [2 tf_lo, 2 tf_hi] in half cells). */
typedef struct {
    int axis_prop, axis_pol;
    int tf_lo[3], tf_hi[3];
    int waveform;             /* NLF_WAVE_* */
    double w0, tau, t0, amplitude;   /* rad/s, s, s, V/m */
} nlf_source;

/* Running-DFT monitors: flux boxes in node indices, the absorption box inside
 * the TF box (one cell clear of its surface), the scattering box outside it
 * (in the scattered-field region, clear of the CPML).  Samples every
 * decimate_k steps (E at n dt, H at (n - 1/2) dt), FP64 accumulators. */
typedef struct {
    int nf;
    const double* omega;      /* nf values, rad/s; copied */
    int abs_lo[3], abs_hi[3];
    int sca_lo[3], sca_hi[3];
    int decimate_k;           /* >= 1 */
    int block_b;              /* samples buffered before accumulation: rounded up to 8, 16 or 32 (0 = 32) */
} nlf_monitors;

/* Sizes and algorithmic traffic of a configured context. */
typedef struct {
    long long cells;              /* nx ny nz */
    long long metal_sites;        /* plasmonic E-sites */
    long long pole_sites;         /* E-sites with critical-point poles (per pole) */
    long long bbox_cells;         /* cells of the metal bounding box (with margin) */
    long long pml_slab_cells;     /* sum over CPML axes of slab cells */
    long long dft_records;        /* flux-face samples (without the incident record) */
    double step_bytes;            /* algorithmic HBM bytes of one time step, the sum of the two below */
    double step_kernel_bytes;     /* EM step kernels: 48 cells + 32 pml_slab_cells (E and H read
                                   * and written once, per slab cell and axis two psi_E read and
                                   * written, two psi_H read and written); when the metal tiles
                                   * update their material sites inside the z march (a metal box
                                   * of at least a quarter of the grid), also 1 per such site (its
                                   * material id) + 8 (2 + gnor) + 16 n_poles per such plasmonic
                                   * or pole site (P_f, a_f, the GNOR history, P_CP and a_CP read
                                   * and written) */
    double metal_kernel_bytes;    /* site-list material update (every material site, or with the
                                   * fused form only those of CPML tiles): 21 per site (site entry
                                   * and cell offset 8, id 1, E read and written 8, H 4) + 8 (2 +
                                   * gnor) per plasmonic site + 16 n_poles per pole site */
    long long material_sites;     /* E-sites holding any material (entries of the site list) */
    double dt;                    /* s */
    int gnor, n_poles;
    long long h2d_bytes;          /* bytes copied host -> device by this context so far */
    long long d2h_bytes;          /* bytes copied device -> host by this context so far */
} nlf_info;

typedef struct nlf_ctx nlf_ctx;

/* Create a context for one grid: the Yee lattice of Table Yee with uniform
 * cells and dt = S dx / c (Sec. III; the Courant bound S <= 1/sqrt(3) of the
 * scheme).  Validates S and sizes; allocates nothing on the device.  *out
 * receives the context, to be released by nlf_destroy.
 * Errors: NLF_E_ARG (sizes, or a boundary other than PEC / CPML), NLF_E_CFL. */
int nlf_create(const nlf_grid* grid, nlf_ctx** out);

/* Material table (copied), n <= NLF_MAX_MATERIALS.  Coefficients D_1..D_d,
 * D_G1, D_G2 (Eqs. d1-dd, GNOR) and C_1p..C_p (Eq. critpointupdate) are
 * formed in FP64 and stored in FP32.  Errors: NLF_E_ARG, NLF_E_CFL
 * (hydrodynamic stability beta dt sqrt(3) / dx > 1). */
int nlf_set_materials(nlf_ctx* ctx, const nlf_material* mats, int n);

/* Shapes (copied), voxelised on the device at the first run (integer,
 * bit-exact): each E-site of Table Yee takes the material of the shape
 * containing its point, with no sub-cell averaging (the staircased surfaces
 * Sec. V discusses); P_f is carried only on those sites (the Pekar condition
 * of Sec. III).  Replaces any material map.  Errors: NLF_E_ARG.
 *
 * Geometry rules (checked at the first run, NLF_E_GEOMETRY): metal stays two
 * cells clear of the outer walls.  With a TF/SF source it lies at least two
 * cells inside the TF box (nonlocal metal only in the total-field region,
 * Sec. III).  Without a source it may reach into a CPML slab (a substrate,
 * say): the E-sites of CPML cells then follow the local Drude model, the
 * material's beta and D taken as zero there, as Sec. III prescribes for a
 * nonlocal structure that has to extend through the PML. */
int nlf_set_shapes(nlf_ctx* ctx, const nlf_shape* shapes, int n);

/* Alternative to shapes: a material id per E-site of Table Yee (0 =
 * background), uint8 [3][nz][ny][nx] (component-major), copied at the call:
 * from host memory, or from device memory if on_device (then the call
 * synchronises the device).  Errors: NLF_E_ARG, NLF_E_STATE (after the first
 * run), NLF_E_CUDA (device copy). */
int nlf_set_material_map(nlf_ctx* ctx, const uint8_t* ids3, int on_device);

/* Source (copied): the TF/SF plane wave of Sec. V, propagating along +z and
 * polarised along x, fed by a 1D auxiliary grid; waveform per NLF_WAVE_*.
 * Errors: NLF_E_ARG, NLF_E_UNSUPPORTED (other axes). */
int nlf_set_source(nlf_ctx* ctx, const nlf_source* src);

/* Monitors (copied, including omega): running DFTs on the faces of the two
 * flux boxes, from which the absorption, scattering and extinction cross
 * sections of Sec. V are formed (the paper does not say how it computes
 * them; nlf_get_spectra states the reading).  Requires a source.
 * Errors: NLF_E_ARG, NLF_E_GEOMETRY. */
int nlf_set_monitors(nlf_ctx* ctx, const nlf_monitors* mon);

/* Single-frequency maps on one lattice plane (Sec. V: the near-field
 * amplitude and free-electron density maps; Eq. Nsol gives the density as
 * n - n0 = div P_f / e).  Every decimate_k steps, at t = n dt, the running
 * DFT (rectangle rule, K dt per sample, exp(+i w t)) of E_x, E_y, E_z at the
 * E-sites (i, j, k) of the plane normal to `axis` at node `index`, and of the
 * charge density div P_f (C/m^3) at its nodes, by the backward differences
 * of the Yee grid.  nf <= NLF_PLANE_MAX_NF; with flux monitors set,
 * decimate_k must equal theirs.  Set before the first run; a context with a
 * plane monitor is not accepted by nlf_batch_run.  Copied.  Errors: NLF_E_ARG,
 * NLF_E_STATE. */
#define NLF_PLANE_MAX_NF 16
typedef struct {
    int axis;                 /* 0, 1, 2: the plane's normal */
    int index;                /* node index along axis */
    int nf;
    const double* omega;      /* rad/s */
    int decimate_k;
} nlf_plane_monitor;
int nlf_set_plane_monitor(nlf_ctx* ctx, const nlf_plane_monitor* mon);

/* Bytes of device state the context needs (for admission by HBM budget).
 * Valid after materials, shapes/map, source and monitors are set; 0 on error.
 * The paper has no counterpart (its memory remark of Sec. III is about the
 * extra grad-div history arrays GNOR needs, which this count includes). */
size_t nlf_state_bytes(const nlf_ctx* ctx);

/* Use caller-owned device memory (e.g. a torch tensor) for the whole state
 * instead of a library allocation (no counterpart in the paper).  dev_ptr
 * must be 256-byte aligned and stay valid until nlf_destroy.  The memory is cleared on first use.
 * Errors: NLF_E_ARG, NLF_E_OOM (bytes < nlf_state_bytes), NLF_E_STATE
 * (state already allocated). */
int nlf_bind_state(nlf_ctx* ctx, void* dev_ptr, size_t bytes);

/* Advance `steps` time steps on `cuda_stream` (a cudaStream_t; NULL = the
 * legacy default stream): each step is f1 (H), f2 (E), f3 (P_CP), f4 (P_f) of
 * Sec. III in that order, with the CPML, the TF/SF corrections and, every
 * decimate_k steps, the running DFT.  Asynchronous; the first call validates
 * the geometry (nonlocal metal only inside the total-field region, Sec. III),
 * allocates (unless bound), voxelises and uploads.  Runs are
 * resumable: run(a) then run(b) equals run(a+b) bit for bit.  The calls
 * that read results, save, destroy or wait (nlf_get_*, nlf_save_state,
 * nlf_sync, nlf_destroy) order themselves after the context's last stream;
 * a caller that moves one context to another stream orders the two streams
 * itself (an event between them, or a synchronisation).
 * Errors: NLF_E_STATE, NLF_E_GEOMETRY, NLF_E_OOM, NLF_E_CUDA. */
int nlf_run(nlf_ctx* ctx, long long steps, void* cuda_stream);

/* Return the context to time index 0 on `cuda_stream` without reallocating
 * (no counterpart in the paper): every field, polarisation, CPML and DFT
 * array is cleared, the tables are uploaded again and the shapes voxelised
 * again (the first call allocates, like nlf_run).  Errors: as nlf_run. */
int nlf_reset(nlf_ctx* ctx, void* cuda_stream);

/* Wait for the work queued by nlf_run, polling for at most timeout_ms
 * (< 0: no limit; no counterpart in the paper).  Checks the device error word: the non-finite watchdog
 * (NLF_E_UNSTABLE) and the step kernel's bounded waits for its tensor-memory
 * copies (NLF_E_CUDA if one gave up; the kernel then skipped the rest of that
 * tile).  Errors: NLF_E_TIMEOUT (work still running; nothing is lost),
 * NLF_E_UNSTABLE, NLF_E_CUDA. */
int nlf_sync(nlf_ctx* ctx, int timeout_ms);

/* Copy one field (NLF_FIELD_*) in SI units, FP32, [nz][ny][nx], to dst
 * (device memory if dst_on_device, else host): E^n, H^{n-1/2}, P_f^n at
 * their Table Yee positions, or the charge density div P_f^n at the nodes
 * (Eq. Nsol: the free-electron density change is it divided by e; backward
 * differences P_a(node) - P_a(node - e_a) over dx).  Synchronises the
 * context's stream.  P outside the metal bounding box is zero.
 * Errors: NLF_E_ARG, NLF_E_STATE (no run yet), NLF_E_CUDA. */
int nlf_get_field(nlf_ctx* ctx, int which, void* dst, int dst_on_device);

/* Set E^n (NLF_FIELD_EX .. EZ, V/m) or H^{n-1/2} (NLF_FIELD_HX .. HZ, A/m) of
 * the current time index from src, FP32 [nz][ny][nx], in device memory if
 * src_on_device, else host: an initial field for a source-free problem (the
 * first call allocates and initialises the state like nlf_run).  The
 * polarisation histories keep their values: at time index 0 the problem then
 * starts from rest with this field (E^{-1} = P^0 = P^{-1} = 0).  Tangential E
 * on a PEC wall must be zero.  A device source is read once every stream's
 * work has finished (the call synchronises the device); the field is on the
 * device when the call returns, so a run launched next on any stream starts
 * from it.  No counterpart in the paper.
 * Errors: NLF_E_ARG, NLF_E_CUDA, and those of the first run's set-up. */
int nlf_set_field(nlf_ctx* ctx, int which, const void* src, int src_on_device);

/* Copy the voxelised material ids, uint8 [3][nz][ny][nx], to host dst (the
 * material of every E-site of Table Yee; 0 = background).  Errors: NLF_E_ARG,
 * and those of the first run's set-up. */
int nlf_get_voxels(nlf_ctx* ctx, uint8_t* dst);

/* Cross sections in m^2 (FP64, nf values each; any pointer may be NULL): the
 * absorption / scattering / extinction cross sections of Sec. V (the paper
 * plots them but does not say how it computes them; this is the flux-box
 * reading), computed on the device from the FP64 accumulators:
 *   sigma_abs = -(1/I) sum_abs-box (1/2) Re(E x H*).n dA,
 *   sigma_sca = +(1/I) sum_sca-box (1/2) Re(E x H*).n dA,
 *   sigma_ext = sigma_abs + sigma_sca, I = (1/2) Re(E_inc H_inc*) at the
 *   centre plane of the absorption box.  Uses library scratch in the state. */
int nlf_get_spectra(nlf_ctx* ctx, double* s_ext, double* s_abs, double* s_sca);

/* Raw accumulators of the running DFT behind the cross sections of Sec. V
 * (the e^{-i w t} convention of the Drude permittivity of Sec. II makes the
 * kernel exp(+i w t)), host dst of 2 * (n_records + 1) * nf * 2 doubles:
 * [E | H][record][frequency][re, im], SI units, including the K dt factor.
 * Records are ordered box (absorption, scattering), normal axis a = x, y, z,
 * low face then high face, term (+E_b H_c, then -E_c H_b with (a,b,c)
 * cyclic), slower in-plane axis outer; the last record is the incident field. */
int nlf_get_dft(nlf_ctx* ctx, double* dst);

/* One plane map (the single-wavelength near-field and density maps of
 * Sec. V; set with nlf_set_plane_monitor): which = NLF_FIELD_EX .. EZ or
 * NLF_MAP_DENSITY; host dst of nf * n1 * n2 * 2 doubles [f][n1][n2][re, im],
 * (n1, n2) the plane's extents along its other two axes, slower first
 * (axis 0: nz, ny; axis 1: nz, nx; axis 2: ny, nx).  E in V/m s, density
 * in C/m^3 s.  Errors: NLF_E_ARG, NLF_E_STATE (no plane monitor or no run),
 * NLF_E_CUDA. */
#define NLF_MAP_DENSITY 9
int nlf_get_plane_map(nlf_ctx* ctx, int which, double* dst);

/* Number of flux-face records of a context with monitors (-1 otherwise). */
long long nlf_num_records(const nlf_ctx* ctx);

/* Checkpoint: copy the whole device state (nlf_state_bytes bytes, including
 * the step counter and pending DFT samples) to / from host memory.  Both
 * allocate and initialise the state first if no run has done so, wait for
 * the context's stream and return once the copy has completed (a run
 * launched after nlf_load_state on any stream starts from the loaded
 * state).  The paper has no counterpart (its runs of 3e5 and 4e5
 * iterations, Sec. V and VI, are the case for one).  Errors: NLF_E_ARG, NLF_E_CUDA. */
int nlf_save_state(nlf_ctx* ctx, void* host);
int nlf_load_state(nlf_ctx* ctx, const void* host);

/* Advance n independent contexts, steps[i] each, on `cuda_stream`: contexts
 * on the same DFT period advance together, every kernel of a time step
 * launched once over the concatenated work of all of them (one launch per
 * kernel per time step, replayed from a captured CUDA graph per DFT period);
 * contexts left with the same number of steps short of a period advance
 * together too (launched directly; the samples of that partial period stay
 * buffered, as after nlf_run, until the next flush or nlf_get_spectra), and
 * the rest one context at a time.  status_out[i] receives each context's
 * status (NLF_OK or NLF_E_*).  All contexts must be configured; contexts with
 * a plane monitor are refused (NLF_E_ARG).  A set of contexts met for the
 * first time gets its launch descriptors copied on `cuda_stream`, and the
 * call waits for that stream there (any stream, blocking or not, is safe).  The paper has no counterpart
 * (it runs one problem per MPI job). */
int nlf_batch_run(nlf_ctx** ctxs, int n, const long long* steps, void* cuda_stream, int* status_out);

/* Cross sections from running-DFT accumulators that the caller holds in its
 * own device memory, computed without allocating anything.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc -- device
 * memory owned by another allocator under a fixed budget, or a loop that must
 * not take cudaMalloc / cudaFree and the device synchronisation they imply.
 * The flux partial sums live in a file-scope device array of
 * NLF_FLUX_STATIC_PAIRS pairs of doubles (2.4 MB) that every GPU loading the
 * library holds until exit.  All pointers are device pointers:
 *   acc_e, acc_h  [(n_records + 1)][nf][re, im] doubles, laid out as returned
 *                 by nlf_get_dft (any common scale factor cancels); the last
 *                 record is the incident field at the centre plane;
 *   coef          n_records doubles, the signed face weights of the records
 *                 (outward sign x term sign x trapezoid weight / 2), in the
 *                 record order of nlf_get_dft, absorption box records first;
 *   n_abs         number of absorption-box records;
 *   dA            face area of one cell, dx^2 (m^2);
 *   out           4 nf doubles: sigma_ext, sigma_abs, sigma_sca (m^2), I.
 * The per-record weights and n_abs of a configured context are available
 * from nlf_get_flux_weights.  Asynchronous on cuda_stream.  The first call on
 * a device looks up the array's device address once for that device (make it
 * before any stream capture); that address is not valid across a
 * cudaDeviceReset of the device in the same process.  Every call shares the
 * array, which keeps the last call's partial sums (all are rewritten by each
 * call, none needs clearing); calls that overlap on the GPU race on it.
 * Errors: NLF_E_ARG (nf > NLF_FLUX_STATIC_PAIRS, null pointers, bad sizes),
 * NLF_E_CUDA (also when an earlier CUDA error is still pending on the thread:
 * it is left pending and nothing is launched). */
#define NLF_FLUX_STATIC_PAIRS 155648
int nlf_flux_spectra_static(const double* acc_e, const double* acc_h, const double* coef, long long n_abs,
                            long long n_records, int nf, double dA, double* out, void* cuda_stream);

/* The signed face weights of the flux records of a configured context (the
 * record order of nlf_get_dft): host coef receives nlf_num_records doubles,
 * each (outward sign of the face) x (sign of the term in S_a = E_b H_c -
 * E_c H_b) x (trapezoid weight: 1/2 on the records at the face's edges
 * along the in-plane axis other than the E component, else 1) / 2, the last
 * factor being the 1/2 of the time-averaged Poynting vector; *n_abs receives
 * the number of absorption-box records (they come first).  This is the flux
 * sum of the extinction method (the cross sections of Sec. V) that
 * nlf_get_spectra evaluates.  Host-side; no device work.  Errors: NLF_E_ARG,
 * NLF_E_STATE (no monitors), the geometry errors of planning. */
int nlf_get_flux_weights(nlf_ctx* ctx, double* coef, long long* n_abs);

/* Time index n (E^n, H^{n-1/2} current), sizes, and number of kernels this
 * context has launched (graph replays count each kernel node).  No
 * counterpart in the paper. */
long long nlf_time_index(const nlf_ctx* ctx);
int nlf_get_info(nlf_ctx* ctx, nlf_info* info);

/* Measurement: advance `steps` time steps with CUDA events recorded around
 * each kernel (the steps are captured and replayed once as a CUDA graph on
 * cuda_stream, as nlf_run executes them), wait, and return the summed device
 * durations in ms: ms_out[0] EM step kernels, ms_out[1] material update and
 * TF/SF corrections, ms_out[2] running-DFT kernels.  The solution advances
 * exactly as with nlf_run.  The paper has no counterpart.
 * Errors: NLF_E_ARG (steps < 1 or > 65536, null ms_out), NLF_E_CUDA. */
int nlf_time_kernels(nlf_ctx* ctx, long long steps, void* cuda_stream, double* ms_out);

/* Kernels this context has launched so far (graph replays count each kernel
 * node).  No counterpart in the paper. */
long long nlf_kernel_launches(const nlf_ctx* ctx);

/* Text of the context's last error, and release of a context (waits for its
 * stream, frees library-owned device memory).  No counterpart in the paper. */
const char* nlf_last_error(const nlf_ctx* ctx);
void nlf_destroy(nlf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
