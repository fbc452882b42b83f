// nlf_internal.h -- device-side data layout of the nonlocal FDTD library.
//
// Internal units are normalised so that every curl coefficient is the Courant
// number S = c dt / dx:  E as is, Ht = eta0 H, Pt = P / eps0.  Then
//   Ht^{n+1/2} = Ht^{n-1/2} - S diff(E^n)                      (f1)
//   eps_inf dE + dPt_f + sum dPt_CP = S diff(Ht^{n+1/2})        (Eq. discreteamperes)
// with diff() the plain difference of neighbouring Yee samples.
//
// All fields are FP32, structure of arrays, [nz][ny][nx], x fastest.
// E and H are double buffered (the fused step reads generation n and writes
// generation n+1 without read/write races between neighbouring threads).
#pragma once

#include <cstdint>

#ifndef NLF_MAX_POLES
#define NLF_MAX_POLES 4
#endif
#define NLF_MAX_MAT 32
// TMA boxes of the background step kernel: x0-4 .. x0+35 along x, the tile's
// 8 rows plus halo rows along y (E: y0-1 .. y0+8, H: y0-1 .. y0+7), one z
// plane, three components
#define NLF_TMA_BOX_X 40
#define NLF_TMA_BOX_EY 10
#define NLF_TMA_BOX_HY 9
#define NLF_MAX_SHP 16
// Material site list entries: component << 30 | flag | box offset
#define NLF_SITE_IN_CPML (1u << 29)          // the site's cell lies in a CPML slab
#define NLF_SITE_OFFSET_MASK ((1u << 29) - 1u)
// Tiles of the EM z-march: BX x BY columns of cells, marched along z in
// chunks (zchunk_range)
#define NLF_TILE_BX 32
#define NLF_TILE_BY 8
#define NLF_INC_PML 40          // CPML cells at the far end of the 1D incident grid
#define NLF_INC_MARGIN 10       // vacuum cells between the TF box and that CPML
#define NLF_MAX_BATCH 256       // instances in one batched launch
#define NLF_BATCH_RCH 32        // records per chunk of the batched accumulation
#define NLF_BATCH_GROUP 8       // chunks per block of the batched accumulation

namespace nlf {

// Bounds-checked build (-DNLF_BOUNDS_CHECK): the non-TMA global accesses of
// the step, material, TF/SF and DFT kernels are checked against the size of
// their array; a violation raises bit 3 of the error word, the first one is
// recorded (the access site's code, the index and the limit), and the access
// is skipped (a load reads zero).  The product build compiles the checks out.
struct BoundsRecord {
    int code;
    int hits;
    long long idx, lim;
};

#ifdef NLF_BOUNDS_CHECK
__device__ __forceinline__ bool nlf_in_bounds(int* err, BoundsRecord* rec, int code, long long idx, long long lim)
{
    if (idx >= 0 && idx < lim) return true;
    if (err) atomicOr(err, 8);
    if (rec && atomicCAS(&rec->code, 0, code) == 0) {
        rec->idx = idx;
        rec->lim = lim;
    }
    if (rec) atomicAdd(&rec->hits, 1);
    return false;
}
#define NLF_IN(P, CODE, IDX, LIM) ::nlf::nlf_in_bounds((P).err, (P).chk, (CODE), (long long)(IDX), (long long)(LIM))
// The state these parameters point into still belongs to the context they
// were made for (its header holds that context's id): a mismatch (a plan, a
// graph or a parameter block that outlived its context, or whose memory went
// to another one) is recorded as access site 30 and the work is skipped.
__device__ __forceinline__ bool nlf_ctx_ok(int* err, BoundsRecord* rec, const long long* hdr_id, long long ctx_id)
{
    const long long held = *hdr_id;
    if (held == ctx_id) return true;
    if (err) atomicOr(err, 8);
    if (rec && atomicCAS(&rec->code, 0, 30) == 0) {
        rec->idx = held;
        rec->lim = ctx_id;
    }
    if (rec) atomicAdd(&rec->hits, 1);
    return false;
}
#define NLF_CTX(P) ::nlf::nlf_ctx_ok((P).err, (P).chk, (P).hdr_id, (P).ctx_id)
#else
#define NLF_IN(P, CODE, IDX, LIM) true
#define NLF_CTX(P) true
#endif

// The CPML slab axes that the cell box [lo, hi] (inclusive) reaches, bit a
// for axis a (0: clear of every slab).
__host__ __device__ __forceinline__ int pml_axes_of_box(const int n3[3], const int cpml[3], int pml, const int lo[3],
                                                         const int hi[3])
{
    int m = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (cpml[a] && (lo[a] < pml || hi[a] >= n3[a] - pml)) m |= 1 << a;
    return m;
}

// The z chunks of the EM z-march.  Without a CPML along z: chunks of kz
// planes from plane 0.  With one (and room between the slabs): the bottom
// chunk holds the slab and one plane more, [0, pml + 1), the top chunk
// likewise [nz - pml - 1, nz), and the planes between are cut into chunks of
// kz (the last may be shorter).  The interior chunks' halo planes (k0 - 1
// below, k1 above) then lie outside the slabs, so only the two end chunks
// run the CPML code along z.
__host__ __device__ __forceinline__ bool zchunk_aligned(int nz, int cpml_z, int pml)
{
    return cpml_z && nz - 2 * (pml + 1) >= 1;
}

__host__ __device__ __forceinline__ int zchunk_count(int nz, int cpml_z, int pml, int kz)
{
    if (!zchunk_aligned(nz, cpml_z, pml)) return (nz + kz - 1) / kz;
    return 2 + (nz - 2 * (pml + 1) + kz - 1) / kz;
}

// Planes [k0, k1) of chunk c (0 <= c < zchunk_count).
__host__ __device__ __forceinline__ void zchunk_range(int nz, int cpml_z, int pml, int kz, int c, int& k0, int& k1)
{
    if (!zchunk_aligned(nz, cpml_z, pml)) {
        k0 = c * kz;
        k1 = k0 + kz < nz ? k0 + kz : nz;
        return;
    }
    const int zl = pml + 1, zh = nz - pml - 1;
    if (c == 0) {
        k0 = 0;
        k1 = zl;
    } else if (c == zchunk_count(nz, cpml_z, pml, kz) - 1) {
        k0 = zh;
        k1 = nz;
    } else {
        k0 = zl + (c - 1) * kz;
        k1 = k0 + kz < zh ? k0 + kz : zh;
    }
}

// The chunk that holds plane k.
__host__ __device__ __forceinline__ int zchunk_of(int nz, int cpml_z, int pml, int kz, int k)
{
    if (!zchunk_aligned(nz, cpml_z, pml)) return k / kz;
    const int zl = pml + 1, zh = nz - pml - 1;
    if (k < zl) return 0;
    if (k >= zh) return zchunk_count(nz, cpml_z, pml, kz) - 1;
    return 1 + (k - zl) / kz;
}

// Does the tile holding cell (i, j, k) reach a CPML slab (its one-cell halo
// included)?  Tiles are NLF_TILE_BX x NLF_TILE_BY x (a z chunk).
__host__ __device__ __forceinline__ bool cell_in_pml_tile(const int n3[3], const int cpml[3], int pml, int kz, int i,
                                                          int j, int k)
{
    const int x0 = i / NLF_TILE_BX * NLF_TILE_BX, y0 = j / NLF_TILE_BY * NLF_TILE_BY;
    int k0 = 0, k1 = 0;
    zchunk_range(n3[2], cpml[2], pml, kz, zchunk_of(n3[2], cpml[2], pml, kz, k), k0, k1);
    const int lo[3] = {x0 - 1, y0 - 1, k0 - 1};
    const int hi[3] = {x0 + NLF_TILE_BX, y0 + NLF_TILE_BY, k1};
    return pml_axes_of_box(n3, cpml, pml, lo, hi) != 0;
}

// Per-material FP32 coefficients of the increment form of f2/f3/f4.
struct MatCoef {
    float inv_den;      // 1 / (eps_inf + D3 + sum C3)
    float cE;           // 3 D3 + sum (C3 + C4)
    float G;            // (D_G1 + 3 D_G2) / dx^2  (D_NL / dx^2 for the nonlocal Drude model)
    // g2 = 1 + D2 and c2g = 1 + C2, formed without cancellation in FP64
    // (gamma dt / (1 + gamma dt / 2) and its pole analogue): D2 and C2 lie
    // within gamma dt of -1, so as FP32 numbers they would carry the damping
    // with only a few significant digits
    float g2, D3, DG2;  // 1 + D2; D3/eps0; D_G2/dx^2
    float c2g[NLF_MAX_POLES], C3[NLF_MAX_POLES], C4[NLF_MAX_POLES], C5[NLF_MAX_POLES],
        kap[NLF_MAX_POLES];   // 1 + C2; C3..C5 / eps0; kap = (Om^2 + Ga^2) / Cp
    int free_e;         // has free electrons (P_f is updated)
    int gnor;           // D > 0: GD history used
    int npoles;
    int pad;
};

struct Shape {
    int kind, material;
    int c[3];
    int radius;
    int half[3];
    int side, tip_base, tip_height, tip_radius, tip_center, tip_cut;
};

// The 128 opaque bytes of a CUDA tensor map (the layout of CUtensorMap).
struct alignas(64) TensorMapBytes {
    unsigned long long w[16];
};

// Everything the fused time step needs.  Pointers are device pointers.
struct StepParams {
    int nx, ny, nz;
    int px;             // row pitch of the field arrays (nx rounded up to 8): cell (i, j, k) at (k ny + j) px + i
    const void* tmE;    // tensor maps (device memory, 64-byte aligned) of E^n and H^{n-1/2} as 4D
    const void* tmH;    // [3][nz][ny][px] arrays, boxes of NLF_TMA_BOX_X x (EY | HY) x 1 x 3 floats
    float S;            // H curl coefficient
    float Sb;           // S / eps_b, background E curl coefficient
    const float* E0[3];
    const float* H0[3];
    float* E1[3];
    float* H1[3];

    // CPML: profiles b, c at integer (E) and half-integer (H) positions of
    // each axis; psi in slabs of 2*pml cells per CPML axis.
    int pml;
    int cpml[3];
    const float* bE[3];
    const float* cE[3];
    const float* bH[3];
    const float* cH[3];
    float* psiE[3][2];          // [derivative axis][slot]: slot 0 = component a+1, 1 = a+2 (mod 3)
    const float* psiH0[3][2];
    float* psiH1[3][2];

    // TF/SF: incident E_x(z index k) = e_inc[k - inc_off], H_y(k) = h_inc[k - inc_off]
    int tfsf;
    int tf_lo[3], tf_hi[3];
    int inc_off, inc_len;
    const float* e_inc0;        // E_inc^n
    const float* h_inc0;        // H_inc^{n-1/2}
    float* e_inc1;              // written by block 0: E_inc^{n+1}
    float* h_inc1;              //                     H_inc^{n+1/2}
    float* psi_e_inc;           // 1D CPML auxiliaries (in place, block 0 only)
    float* psi_h_inc;
    const float* b_e_inc;
    const float* c_e_inc;
    const float* b_h_inc;
    const float* c_h_inc;
    int waveform;
    double w0, tau, t0, amp, dt;

    // metal bounding box (cells [bb_lo, bb_lo + bb_n)) with its hydrodynamic state
    int has_metal;
    int bb_lo[3], bb_n[3];
    const uint8_t* mat[3];
    const uint32_t* sites;      // material E-sites of the box: (component << 30) | CPML flag | box offset
    const uint32_t* site_q;     // their cell offsets in the field arrays
    const MatCoef* coef;        // [n_materials + 1], index 0 unused
    const float* P0[3];
    float* P1[3];
    float* auxf[3];
    float* gdp[3];
    float* pcp[NLF_MAX_POLES][3];
    float* auxcp[NLF_MAX_POLES][3];
    int any_gnor;
    int max_poles;
    // material update fused into the EM z-march: tile column (bx, by) holds
    // material E-sites on cell planes [nz - tile_kr.x, tile_kr.y - 1] (both 0:
    // none); its tiles run k_step_metal.  Sites of CPML tiles keep the
    // site-list update (psites, n_psites entries).
    int fuse_metal;
    int tiles_x;
    const int2* tile_kr;
    const uint32_t* psites;
    const uint32_t* psite_q;

    // step counters: step0 holds n, block 0 writes n+1 into step1
    const long long* step0;
    long long* step1;
    int* err;
    // array sizes for the bounds-checked build: floats per field component,
    // per psi slot of each CPML axis, cells of the metal box, tile columns
    long long nfield;
    long long psi_n[3];
    long long nbb;
    int ntiles_xy;
    BoundsRecord* chk;
    const long long* hdr_id;    // the context id in the state's header, and the id these parameters
    long long ctx_id;           // were made for (compared by the bounds-checked build's kernels)
    // copies of the maps tmE and tmH point to; with map_in_params set (the
    // single-grid kernels, whose parameter block is a grid constant) the
    // copies read them from the kernel parameter, else (a block's copy of
    // the parameters in shared memory, the batched kernels) from tmE / tmH
    TensorMapBytes mapE, mapH;
    int map_in_params;
};

struct VoxParams {
    int nshape;
    Shape shp[NLF_MAX_SHP];
    int bb_lo[3], bb_n[3];
    uint8_t* mat[3];
    unsigned long long* counts;   // [3] plasmonic E-sites per component (atomic)
    const int* free_e;            // [NLF_MAX_MAT + 1] material has free electrons
};

// Single-frequency plane maps: running DFT of E_x, E_y, E_z and of div P_f on
// one lattice plane.
#define NLF_PLANE_MAX_NF_DEV 16
struct PlaneParams {
    int axis, index;
    int nx, ny, nz, px;
    int n1, n2;                 // plane extents along its other axes, slow then fast
    int nf;
    const double* omega;        // [nf] rad/s
    double dt, scale;           // scale = K dt (rectangle rule)
    double eps0_dx;             // eps0 / dx: P/eps0 difference units -> C/m^3
    int has_metal;
    int bb_lo[3], bb_n[3];
    double2* acc;               // [4][nf][n1][n2]
};

// Density output: div P_f over the whole grid from the metal box's P_f.
struct DensityParams {
    int nx, ny, nz;
    int bb_lo[3], bb_n[3];
    const float* P[3];          // P_f / eps0, [bb_n2][bb_n1][bb_n0]
    double eps0_dx;             // eps0 / dx
};

// Where the metal box sits in the field arrays (for the site list), and the
// tiling that decides which sites the fused EM kernel updates: with
// only_pml set, the list keeps only the sites whose tile (BX x BY x kz, its
// one-cell halo included) reaches a CPML slab; tile_kr receives the z range
// of material sites of every tile column.
struct SiteGeom {
    int bb_lo[3], bb_n[3];
    int nx, ny, nz, px;
    int only_pml;
    int kz, pml;
    int cpml[3];
    int tiles_x;
    int2* tile_kr;
    const int* free_e;          // [NLF_MAX_MAT + 1]
};

struct DftParams {
    long long nrec;             // face records; the incident record is nrec
    int nf, B;
    const uint32_t* rec_e;      // offset into the E component space (comp * ncell + cell)
    const uint32_t* rec_h;      // offset of the first H point
    const uint32_t* rec_hs;     // stride to the second H point
    float* sE;                  // [B][nrec + 1]
    float* sH;
    long long* sample_step;     // [B]
    float4* phase;              // [B][nf]: cos, sin at n dt and at (n - 1/2) dt
    double2* accE;              // [nrec + 1][nf]
    double2* accH;
    const double* omega;
    double dt;
    int inc_node;
    long long nfield3;          // floats of the three components of E (and of H): bounds-checked build
    int* err;
    BoundsRecord* chk;
    const long long* hdr_id;    // as in StepParams
    long long ctx_id;
};

// Batched stepping: instance q uses params[2 q + (base_par ^ launch parity)].
struct BatchInst {
    int tiles_x, tiles_y, chunks, kz;
    int base_par;
    int pad;
};

struct BatchStep {
    const StepParams* params;   // [2 n]
    const BatchInst* inst;      // [n]
    const long long* item_end;  // [n] inclusive prefix sums of work items
    const long long* met_end;   // [n] inclusive prefix sums of material sites
    const long long* tf_end;    // [n] inclusive prefix sums of TF/SF correction items
    int n;
    int launch_par;
};

struct BatchDftInst {
    DftParams d;
    const float* E[2];
    const float* H[2];
    const float* e_inc[2];
    const float* h_inc[2];
    const long long* step[2];
    int* err;
    int base_par;
    int pad;
};

struct BatchDft {
    const BatchDftInst* inst;   // [n]
    const long long* rec_end;   // [n] prefix sums of (records + 1)
    const long long* ph_end;    // [n] prefix sums of B * nf
    const long long* chunk_end; // [n] prefix sums of record groups (NLF_BATCH_GROUP chunks of NLF_BATCH_RCH)
    int n;
    int cur_par;                // generation parity of the fields just written
};

}  // namespace nlf
