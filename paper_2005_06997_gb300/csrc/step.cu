// step.cu -- one time step of the nonlocal hydrodynamic FDTD scheme.
//
// Two kernels advance (H^{n-1/2}, E^n, P^n) to (H^{n+1/2}, E^{n+1}, P^{n+1})
// in the order of Sec. III: f1 (H), f2 (E), f3 (P_CP), f4 (P_f).
//
// The EM step (k_step, k_step_pml, or k_step_batch over many grids): a
// thread block owns a BX x BY column tile and marches through a chunk of z
// planes.  For plane k it holds E^n of planes k and k+1 (tile plus a one-cell
// halo) in shared memory, computes H^{n+1/2} of the tile plus the -x / -y
// halo (the halo H is the only recomputed work), keeps H of plane k-1 in
// registers, and then updates the background E of the tile.  Planes arrive
// ahead of use by TMA into a ring of shared-memory stages, the CPML psi
// operands by cp.async.  E, H and psi_H are double buffered (generation n
// read, n+1 written), so tiles need no grid-wide barrier; every field crosses
// HBM once per step apart from halos.  Tiles are classified once per block:
// clear of the CPML slabs they run plain Yee arithmetic with no per-cell
// tests; CPML tiles run in their own kernel (more shared memory: the psi
// staging area) concurrently with the others.  The TF/SF connection is a
// set of additive corrections on the TF surface applied after the step.
//
// The material update: one thread per material E-site of a compact list
// rewrites E^{n+1} there from the H^{n+1/2} just written and advances P_CP
// and P_f.  With a source and a material present, one kernel (k_post) runs
// both the corrections and the material update; otherwise k_tfsf or
// k_metal runs alone.
//
// f2/f3/f4 are applied in increment form, algebraically identical to the
// paper's printed recurrences (Eq. NonlocalUpdate, Eq. GNORUpdate,
// Eq. critpointupdate substituted into Eq. discreteamperes) but free of the
// cancellation of D1 P^n + D2 P^{n-1} (D1 ~ 2, D2 ~ -1) in FP32.  With
// dP^{n+1} = P^{n+1} - P^n and D1 + D2 = 1:
//   dP_f^{n+1}  = a_f^n + D3 (2 E^n + E^{n+1}) + (D_G1 + 3 D_G2) GD^n
//   a_f^{n+1}   = -D2 dP_f^{n+1} + D3 E^n + D_G2 (GD^{n-1} - 4 GD^n)
//   dP_CP^{n+1} = a_c^n + C3 E^{n+1} + C4 E^n
//   a_c^{n+1}   = -kap P_CP^{n+1} - C2 dP_CP^{n+1} + C5 E^n,  kap = (Om^2+Ga^2)/Cp
//   E^{n+1} = E^n + delta,
//   delta (eps_inf + D3 + C3) = S curl Ht - a_f - a_c - (D_G1 + 3 D_G2) GD - (3 D3 + C3 + C4) E^n
// (the last line carries the -C4 of substituting f3 into Ampere's law).
// D2 and C2 enter as -D2 dP = dP - (1 + D2) dP with 1 + D2 (and 1 + C2)
// stored in FP32 to full relative precision, so the damping they carry is
// not rounded away.
// GD^n = grad(div P_f^n) is evaluated as the difference of node divergences,
// which equals Eq. GradDiv term by term.
//
// Offsets are 32-bit: the library rejects grids with 3 px ny nz >= 2^32.
#include <cuda_runtime.h>

#include <type_traits>

#include "nlf_internal.h"

namespace nlf {

constexpr int BX = NLF_TILE_BX, BY = NLF_TILE_BY;
static_assert(NLF_TMA_BOX_X == BX + 8 && NLF_TMA_BOX_EY == BY + 2 && NLF_TMA_BOX_HY == BY + 1,
              "tensor-map boxes must match the tile");

// Half-cell offsets of the Yee positions (Table Yee).
__device__ __forceinline__ int eoff(int c, int a) { return c == a ? 1 : 0; }
__device__ __forceinline__ int hoff(int c, int a) { return c == a ? 0 : 1; }

__device__ __forceinline__ bool tf_point(const StepParams& p, int h0, int h1, int h2)
{
    return h0 >= 2 * p.tf_lo[0] && h0 <= 2 * p.tf_hi[0] && h1 >= 2 * p.tf_lo[1] && h1 <= 2 * p.tf_hi[1] &&
           h2 >= 2 * p.tf_lo[2] && h2 <= 2 * p.tf_hi[2];
}

__device__ __forceinline__ float e_inc(const StepParams& p, int k)
{
    int m = k - p.inc_off;
    return (m >= 0 && m < p.inc_len) ? __ldg(p.e_inc0 + m) : 0.f;
}

// Ht_inc^{n+1/2} at the H_y z-index k, from the 1D grid's generation n.
__device__ __forceinline__ float h_inc_next(const StepParams& p, int k)
{
    int m = k - p.inc_off;
    if (m < 0 || m + 1 >= p.inc_len) return 0.f;
    float e0 = __ldg(p.e_inc0 + m), e1 = __ldg(p.e_inc0 + m + 1);
    return __ldg(p.h_inc0 + m) - p.S * (e1 - e0);
}

// Local index of v inside the CPML slabs of axis a, or -1.
__device__ __forceinline__ int slab_local(const StepParams& p, int a, int v)
{
    const int n = a == 0 ? p.nx : (a == 1 ? p.ny : p.nz);
    if (!p.cpml[a]) return -1;
    if (v < p.pml) return v;
    if (v >= n - p.pml) return v - (n - p.pml) + p.pml;
    return -1;
}

// One cell as the update functions see it: its indices, its 32-bit offset and,
// on CPML tiles, its slab position along each axis (-1: not in that slab) and
// its offset in that axis' psi arrays.
struct Cell {
    int i, j, k;
    uint32_t q;
    int l[3];
    uint32_t s[3];
    int wm = 7;         // bit a: some lane of the warp has its cell in the slab of axis a (else its psi work is skipped)
};

__device__ __forceinline__ void cell_slabs(const StepParams& p, Cell& c)
{
    const uint32_t two = 2u * (uint32_t)p.pml;
    c.s[0] = c.l[0] >= 0 ? ((uint32_t)c.k * p.ny + c.j) * two + c.l[0] : 0u;
    c.s[1] = c.l[1] >= 0 ? ((uint32_t)c.k * two + c.l[1]) * p.nx + c.i : 0u;
    c.s[2] = c.l[2] >= 0 ? ((uint32_t)c.l[2] * p.ny + c.j) * p.nx + c.i : 0u;
}

__device__ __forceinline__ Cell make_cell(const StepParams& p, int i, int j, int k, bool pml)
{
    Cell c;
    c.i = i;
    c.j = j;
    c.k = k;
    c.q = ((uint32_t)k * p.ny + j) * p.px + i;
    c.l[0] = c.l[1] = c.l[2] = -1;
    if (pml) {
        c.l[0] = slab_local(p, 0, i);
        c.l[1] = slab_local(p, 1, j);
        c.l[2] = slab_local(p, 2, k);
        cell_slabs(p, c);
    }
    return c;
}

// H_C^{n+1/2} at cell c from H^{n-1/2} = h0 and the E^n values of its curl
// ((curl E)_C = dE_{A2}/dx_{A1} - dE_{A1}/dx_{A2}, (C, A1, A2) cyclic):
// a_here, a_next = E_{A2} at idx and idx + e_A1, b_here, b_next = E_{A1} at idx
// and idx + e_A2 (zero beyond the wall).  psA1, psA2: psi_H^{n-1/2} of the
// two derivatives and pr1, pr2 the (b, c) CPML coefficients of their axes at
// the cell (used only inside the slab of that axis).  If own, store it and
// its psi.
//
template <int C, bool PML, int AX = 7>
__device__ __forceinline__ float h_cell(const StepParams& p, const Cell& c, float h0, float a_here, float a_next,
                                        float b_here, float b_next, bool own, float psA1 = 0.f, float psA2 = 0.f,
                                        float2 pr1 = {}, float2 pr2 = {})
{
    constexpr int A1 = (C + 1) % 3, A2 = (C + 2) % 3;
    float t1 = a_next - a_here;
    float t2 = b_next - b_here;
    if (PML) {
        // pr = (b, c) of the derivative's axis at the cell; selects, not
        // branches: lanes in and out of a slab take one path
        // AX: the slab axes the tile touches (compile time); others have no psi here
        if ((AX >> A1 & 1) && (c.wm >> A1 & 1)) {
            const float psi1 = c.l[A1] >= 0 ? pr1.x * psA1 + pr1.y * t1 : 0.f;
            if (own && c.l[A1] >= 0 && NLF_IN(p, 3, c.s[A1], p.psi_n[A1])) p.psiH1[A1][1][c.s[A1]] = psi1;
            t1 += psi1;
        }
        if ((AX >> A2 & 1) && (c.wm >> A2 & 1)) {
            const float psi2 = c.l[A2] >= 0 ? pr2.x * psA2 + pr2.y * t2 : 0.f;
            if (own && c.l[A2] >= 0 && NLF_IN(p, 3, c.s[A2], p.psi_n[A2])) p.psiH1[A2][0][c.s[A2]] = psi2;
            t2 += psi2;
        }
    }
    const float h = h0 - p.S * (t1 - t2);
    if (own && NLF_IN(p, 2, c.q, p.nfield)) p.H1[C][c.q] = h;
    return h;
}

// E_C^{n+1} of the background at cell c from E^n = En and H^{n+1/2}:
// hA2 = H_{A2}(idx), hA2m = H_{A2}(idx - e_A1), hA1 = H_{A1}(idx), hA1m = H_{A1}(idx - e_A2);
// peA1, peA2: psi_E^n of the two derivatives, pr1, pr2 the (b, c) of their
// axes (used only inside the slab).
// Sites that hold a material are rewritten afterwards by k_metal.
template <int C, bool PML, int AX = 7>
__device__ __forceinline__ void e_cell(const StepParams& p, const Cell& c, float En, float hA2, float hA2m, float hA1,
                                       float hA1m, float peA1 = 0.f, float peA2 = 0.f, float2 pr1 = {},
                                       float2 pr2 = {})
{
    constexpr int A1 = (C + 1) % 3, A2 = (C + 2) % 3;
    float t1 = hA2 - hA2m;
    float t2 = hA1 - hA1m;
    if (PML) {
        if ((AX >> A1 & 1) && (c.wm >> A1 & 1)) {
            const float psi1 = c.l[A1] >= 0 ? pr1.x * peA1 + pr1.y * t1 : 0.f;
            if (c.l[A1] >= 0 && NLF_IN(p, 4, c.s[A1], p.psi_n[A1])) p.psiE[A1][1][c.s[A1]] = psi1;
            t1 += psi1;
        }
        if ((AX >> A2 & 1) && (c.wm >> A2 & 1)) {
            const float psi2 = c.l[A2] >= 0 ? pr2.x * peA2 + pr2.y * t2 : 0.f;
            if (c.l[A2] >= 0 && NLF_IN(p, 4, c.s[A2], p.psi_n[A2])) p.psiE[A2][0][c.s[A2]] = psi2;
            t2 += psi2;
        }
    }
    if (NLF_IN(p, 5, c.q, p.nfield)) p.E1[C][c.q] = En + p.Sb * (t1 - t2);
}

// Node divergence of P_f^n (difference units) at bbox-local offset b.
__device__ __forceinline__ float node_div(const StepParams& p, uint32_t b, uint32_t sy, uint32_t sz)
{
    return (__ldg(p.P0[0] + b) - __ldg(p.P0[0] + b - 1)) + (__ldg(p.P0[1] + b) - __ldg(p.P0[1] + b - sy)) +
           (__ldg(p.P0[2] + b) - __ldg(p.P0[2] + b - sz));
}

// The material update of E-site (C, box offset b) of material id: E^{n+1}
// from Eq. discreteamperes with f3 and f4 substituted (increment form), then
// P_CP^{n+1} and P_f^{n+1}.  curl = the plain difference curl of H^{n+1/2} at
// the site, gd_raw = the difference of the node divergences of P_f^n,
// p_old, af_raw, g1, pc, ac the site's P_f^n, a_f^n, GD^{n-1}, P_CP^n and
// a_CP^n (arrays a material does not use are read and ignored: gd_raw and
// af_raw for a material without free electrons, poles past its own count).
// Returns E^{n+1}; writes the site's hydrodynamic and pole state.
template <int C, int NPMAX>
__device__ __forceinline__ float site_update(const StepParams& p, uint32_t b, int id, float En, float curl,
                                             float gd_raw, float p_old, float af_raw, float g1, float (&pc)[NPMAX],
                                             float (&ac)[NPMAX], bool local = false)
{
    const MatCoef& m = p.coef[id];
    // local: a site of a CPML cell, where the metal follows the local Drude
    // model (no pressure or diffusion term: G = D_G2 = 0), Sec. III
    const float mG = local ? 0.f : m.G, mDG2 = local ? 0.f : m.DG2;
    const float gd = m.free_e ? gd_raw : 0.f;
    const float af = m.free_e ? af_raw : 0.f;
    float acs = 0.f;
#pragma unroll
    for (int pp = 0; pp < NPMAX; ++pp) {
        if (pp >= m.npoles) ac[pp] = 0.f;
        acs += ac[pp];
    }
    const float delta = (p.S * curl - af - acs - mG * gd - m.cE * En) * m.inv_den;
    if (!NLF_IN(p, 11, b, p.nbb)) return En + delta;
    if (m.free_e) {
        const float dP = af + m.D3 * (3.f * En + delta) + mG * gd;
        p.P1[C][b] = p_old + dP;
        float a_new = fmaf(-m.g2, dP, dP) + m.D3 * En;      // -D2 dP + D3 E^n
        if (m.gnor) {
            a_new += mDG2 * (g1 - 4.f * gd);
            p.gdp[C][b] = gd;
        }
        p.auxf[C][b] = a_new;
    }
#pragma unroll
    for (int pp = 0; pp < NPMAX; ++pp) {
        if (pp >= m.npoles) break;
        const float dPc = ac[pp] + m.C3[pp] * (En + delta) + m.C4[pp] * En;
        const float pcn = pc[pp] + dPc;
        p.pcp[pp][C][b] = pcn;
        p.auxcp[pp][C][b] = -m.kap[pp] * pcn + fmaf(-m.c2g[pp], dPc, dPc) + m.C5[pp] * En;
    }
    return En + delta;
}

// Material update of E-site (C, box offset b) after the EM step, from the
// site list (sites of tiles that the fused z-march does not update): the
// curl uses H^{n+1/2} just written by the step (material sites lie at least
// two cells inside the TF box and outside the CPML, so neither correction
// applies there).  Every operand is loaded before the material's
// coefficients are consulted, so one memory round trip serves the whole site.
template <int C, bool PMLS = false>
__device__ __forceinline__ void metal_site(const StepParams& p, uint32_t b, uint32_t q)
{
    constexpr int A1 = (C + 1) % 3, A2 = (C + 2) % 3;
    const uint32_t sy = (uint32_t)p.bb_n[0], sz = (uint32_t)p.bb_n[0] * (uint32_t)p.bb_n[1];
    const uint32_t st[3] = {1u, (uint32_t)p.px, (uint32_t)p.px * (uint32_t)p.ny};
    const uint32_t stb = C == 0 ? 1u : (C == 1 ? sy : sz);
    if (!(NLF_IN(p, 13, q, p.nfield) && NLF_IN(p, 13, (long long)q - st[A1], p.nfield) &&
          NLF_IN(p, 13, (long long)q - st[A2], p.nfield) && NLF_IN(p, 14, b + stb, p.nbb) &&
          NLF_IN(p, 14, (long long)b - sz, p.nbb)))
        return;
    const int id = __ldg(p.mat[C] + b);
    const float h2 = p.H1[A2][q], h2m = p.H1[A2][q - st[A1]];
    const float h1 = p.H1[A1][q], h1m = p.H1[A1][q - st[A2]];
    const float En = __ldg(p.E0[C] + q);
    const float gd_raw = node_div(p, b + stb, sy, sz) - node_div(p, b, sy, sz);
    const float p_old = __ldg(p.P0[C] + b);
    const float af_raw = p.auxf[C][b];
    const float g1 = p.any_gnor ? p.gdp[C][b] : 0.f;
    float ac[NLF_MAX_POLES], pc[NLF_MAX_POLES];
#pragma unroll
    for (int pp = 0; pp < NLF_MAX_POLES; ++pp) {
        ac[pp] = pp < p.max_poles ? p.auxcp[pp][C][b] : 0.f;
        pc[pp] = pp < p.max_poles ? p.pcp[pp][C][b] : 0.f;
    }
    float t1 = h2 - h2m, t2 = h1 - h1m;
    if constexpr (PMLS) {
        // a site of a CPML cell: the step kernel has already advanced the
        // site's psi_E of each derivative whose slab holds the cell; the
        // curl takes them as the background update does
        const uint32_t bi = b % (uint32_t)p.bb_n[0], r = b / (uint32_t)p.bb_n[0];
        const uint32_t bj = r % (uint32_t)p.bb_n[1], bk = r / (uint32_t)p.bb_n[1];
        Cell c = make_cell(p, p.bb_lo[0] + (int)bi, p.bb_lo[1] + (int)bj, p.bb_lo[2] + (int)bk, true);
        if (c.l[A1] >= 0 && NLF_IN(p, 15, c.s[A1], p.psi_n[A1])) t1 += p.psiE[A1][1][c.s[A1]];
        if (c.l[A2] >= 0 && NLF_IN(p, 15, c.s[A2], p.psi_n[A2])) t2 += p.psiE[A2][0][c.s[A2]];
    }
    const float curl = t1 - t2;
    p.E1[C][q] = site_update<C, NLF_MAX_POLES>(p, b, id, En, curl, gd_raw, p_old, af_raw, g1, pc, ac, PMLS);
}

// Entry t of the material site list (box entry e: component << 30, bit 29
// set for a site of a CPML cell, box offset below; cell offset q).
__device__ __forceinline__ void metal_entry(const StepParams& p, long long t)
{
    if (!NLF_CTX(p)) return;
    const uint32_t e = __ldg(p.sites + t), q = __ldg(p.site_q + t);
    const uint32_t c = e >> 30, b = e & NLF_SITE_OFFSET_MASK;
    if (e & NLF_SITE_IN_CPML) {
        if (c == 0)
            metal_site<0, true>(p, b, q);
        else if (c == 1)
            metal_site<1, true>(p, b, q);
        else
            metal_site<2, true>(p, b, q);
        return;
    }
    if (c == 0)
        metal_site<0>(p, b, q);
    else if (c == 1)
        metal_site<1>(p, b, q);
    else
        metal_site<2>(p, b, q);
}

__global__ void __launch_bounds__(256, 6) k_metal(const StepParams p, long long n_sites)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_sites) metal_entry(p, t);
}

__device__ double source_value(const StepParams& p, double t)
{
    if (p.waveform == 1) {
        double u = (t - p.t0) / p.tau;
        return p.amp * exp(-u * u) * sin(p.w0 * (t - p.t0));
    }
    if (p.waveform == 2) {
        if (t < 0.0 || t > 2.0 * 3.14159265358979323846 / p.w0) return 0.0;
        double r = 0.5 * (1.0 - cos(p.w0 * t));
        return p.amp * r * r * r;
    }
    return 0.0;
}

// 1D incident grid step (one block): H_inc^{n+1/2}, then E_inc^{n+1}, hard
// source at node 0, CPML at the far end.
__device__ void inc_step(const StepParams& p, int tid, int nt)
{
    const int L = p.inc_len;
    for (int m = tid; m < L; m += nt) {
        float e1 = m + 1 < L ? p.e_inc0[m + 1] : 0.f;
        float dE = e1 - p.e_inc0[m];
        float psi = p.b_h_inc[m] * p.psi_h_inc[m] + p.c_h_inc[m] * dE;
        p.psi_h_inc[m] = psi;
        p.h_inc1[m] = p.h_inc0[m] - p.S * (dE + psi);
    }
    __syncthreads();
    for (int m = 1 + tid; m < L; m += nt) {
        float dH = p.h_inc1[m] - p.h_inc1[m - 1];
        float psi = p.b_e_inc[m] * p.psi_e_inc[m] + p.c_e_inc[m] * dH;
        p.psi_e_inc[m] = psi;
        p.e_inc1[m] = p.e_inc0[m] - p.Sb * (dH + psi);
    }
    if (tid == 0) {
        long long n = *p.step0;
        p.e_inc1[0] = (float)source_value(p, (double)(n + 1) * p.dt);
    }
}

// ------------------------------------------------------------------ tiles

// CPML tiles stage the psi values of plane k+1 in shared memory with
// asynchronous copies issued during plane k, so the slab's extra operands
// arrive off the critical path.  Per thread (own cell), by component C:
// slot 2C / 2C+1 = psi_H^{n-1/2} of the A1 / A2 derivative, 6+2C / 7+2C the
// same for psi_E^n; per halo thread, its two H components' A1 / A2 psi_H.
// The tile's CPML coefficients (b_E, c_E, b_H, c_H) along x (x0-1 .. x0+BX-1)
// and y (y0-1 .. y0+BY-1) sit beside them; those along z are uniform per
// plane and read per plane.
struct PsiShared {
    float own[2][12][BX * BY];
    float halo[2][4][BX + BY];
    float cx[4][BX + 1];
    float cy[4][BY + 1];
};

// (b_E, c_E, b_H, c_H) of plane k along z.
struct ZCoef {
    float bE, cE, bH, cH;
};

__device__ __forceinline__ ZCoef zcoef(const StepParams& p, int k)
{
    const int kk = min(max(k, 0), p.nz - 1);
    return ZCoef{__ldg(p.bE[2] + kk), __ldg(p.cE[2] + kk), __ldg(p.bH[2] + kk), __ldg(p.cH[2] + kk)};
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// 4-byte asynchronous copy; when !valid nothing is read and zero is written.
__device__ __forceinline__ void cp_async4z(float* dst, const float* src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

// Slab geometry of one column (i, j) of a CPML tile, constant along z: the
// slab positions along x and y and the z-independent parts of the psi
// offsets (psi_x at ((k ny + j) 2L + l0), psi_y at ((k 2L + l1) nx + i),
// psi_z at ((l2 ny + j) nx + i) for an L-cell CPML).
struct PmlCol {
    int l0, l1;
    uint32_t s0b, s1b, s2b;
};

__device__ __forceinline__ PmlCol pml_col(const StepParams& p, int i, int j)
{
    PmlCol q;
    q.l0 = slab_local(p, 0, i);
    q.l1 = slab_local(p, 1, j);
    const uint32_t two = 2u * (uint32_t)p.pml;
    q.s0b = (uint32_t)j * two + (uint32_t)(q.l0 >= 0 ? q.l0 : 0);
    q.s1b = (uint32_t)(q.l1 >= 0 ? q.l1 : 0) * (uint32_t)p.nx + (uint32_t)i;
    q.s2b = (uint32_t)j * (uint32_t)p.nx + (uint32_t)i;
    return q;
}

// Slab positions and psi offsets of cell (c.i, c.j, c.k) from its column;
// the offset of an axis whose slab does not hold the cell is 0 (a valid
// element that is never used).
__device__ __forceinline__ void pml_cell(const StepParams& p, const PmlCol& q, Cell& c)
{
    const uint32_t two = 2u * (uint32_t)p.pml;
    c.l[0] = q.l0;
    c.l[1] = q.l1;
    c.l[2] = slab_local(p, 2, c.k);
    c.s[0] = q.l0 >= 0 ? q.s0b + (uint32_t)c.k * (uint32_t)p.ny * two : 0u;
    c.s[1] = q.l1 >= 0 ? q.s1b + (uint32_t)c.k * two * (uint32_t)p.nx : 0u;
    c.s[2] = c.l[2] >= 0 ? (uint32_t)c.l[2] * (uint32_t)p.ny * (uint32_t)p.nx + q.s2b : 0u;
}

// Queue the psi operands of component C at cell c: psi_H (d1, d2) and, if
// e1, psi_E (e1, e2); zero for a derivative whose slab does not hold the cell.
template <int C, int AX>
__device__ __forceinline__ void psi_fetch(const StepParams& p, const Cell& c, float* d1, float* d2, float* e1,
                                          float* e2)
{
    constexpr int A1 = (C + 1) % 3, A2 = (C + 2) % 3;
    // an axis whose slab no lane of the warp reaches is skipped: its
    // consumers skip it too (Cell::wm), so the stale slots are never read
    if ((AX >> A1 & 1) && (c.wm >> A1 & 1) && p.cpml[A1]) {
        const bool v = c.l[A1] >= 0 && NLF_IN(p, 7, c.s[A1], p.psi_n[A1]);
        cp_async4z(d1, p.psiH0[A1][1] + c.s[A1], v);
        if (e1) cp_async4z(e1, p.psiE[A1][1] + c.s[A1], v);
    }
    if ((AX >> A2 & 1) && (c.wm >> A2 & 1) && p.cpml[A2]) {
        const bool v = c.l[A2] >= 0 && NLF_IN(p, 7, c.s[A2], p.psi_n[A2]);
        cp_async4z(d2, p.psiH0[A2][0] + c.s[A2], v);
        if (e2) cp_async4z(e2, p.psiE[A2][0] + c.s[A2], v);
    }
}

// Queue every psi operand of plane kk into buffer b: own cell (i, j, kk) and,
// for the halo threads, their halo H cell (column geometry qh).
template <int AX>
__device__ __forceinline__ void psi_plane(const StepParams& p, PsiShared& ps, int b, int kk, int x0, int y0, int i,
                                          int j, bool in, const PmlCol& qo, const PmlCol& qh, int tid, int wm_xy)
{
    if (in) {
        Cell c;
        c.i = i;
        c.j = j;
        c.k = kk;
        pml_cell(p, qo, c);
        c.wm = wm_xy | (c.l[2] >= 0 ? 4 : 0);
        float(*o)[BX * BY] = ps.own[b];
        psi_fetch<0, AX>(p, c, &o[0][tid], &o[1][tid], &o[6][tid], &o[7][tid]);
        psi_fetch<1, AX>(p, c, &o[2][tid], &o[3][tid], &o[8][tid], &o[9][tid]);
        psi_fetch<2, AX>(p, c, &o[4][tid], &o[5][tid], &o[10][tid], &o[11][tid]);
    }
    float(*h)[BX + BY] = ps.halo[b];
    if (tid < BY) {
        const int jh = y0 + tid;
        if (x0 > 0 && jh < p.ny) {
            Cell c;
            c.i = x0 - 1;
            c.j = jh;
            c.k = kk;
            pml_cell(p, qh, c);
            psi_fetch<1, AX>(p, c, &h[0][tid], &h[1][tid], nullptr, nullptr);
            psi_fetch<2, AX>(p, c, &h[2][tid], &h[3][tid], nullptr, nullptr);
        }
    } else if (tid < BY + BX) {
        const int ih = x0 + tid - BY;
        if (y0 > 0 && ih < p.nx) {
            Cell c;
            c.i = ih;
            c.j = y0 - 1;
            c.k = kk;
            pml_cell(p, qh, c);
            psi_fetch<0, AX>(p, c, &h[0][tid], &h[1][tid], nullptr, nullptr);
            psi_fetch<2, AX>(p, c, &h[2][tid], &h[3][tid], nullptr, nullptr);
        }
    }
    cp_async_commit();
}

// (b, c) of axis a at a tile position: w = 0 for E, 2 for H; ux, uy the
// offsets from (x0-1, y0-1); z from the plane's coefficients.
template <int a>
__device__ __forceinline__ float2 cpml_coef(const PsiShared& ps, int w, int ux, int uy, const ZCoef& z)
{
    if (a == 0) return make_float2(ps.cx[w][ux], ps.cx[w + 1][ux]);
    if (a == 1) return make_float2(ps.cy[w][uy], ps.cy[w + 1][uy]);
    return w == 0 ? make_float2(z.bE, z.cE) : make_float2(z.bH, z.cH);
}

// Fill the tile's coefficient tables (every thread of the block; a barrier
// must follow before use).
__device__ __forceinline__ void cpml_tables(const StepParams& p, PsiShared& ps, int x0, int y0, int tid)
{
    // the profile arrays are named member by member (no address of the
    // parameter block is taken, which would move it to local memory)
    auto tab = [&](int w, int a) -> const float* {
        const float* e = w == 0 ? p.bE[a] : p.cE[a];
        const float* h = w == 2 ? p.bH[a] : p.cH[a];
        return w < 2 ? e : h;
    };
    for (int t = tid; t < 4 * (BX + 1); t += BX * BY) {
        const int w = t / (BX + 1), u = t - w * (BX + 1);
        ps.cx[w][u] = __ldg(tab(w, 0) + min(max(x0 - 1 + u, 0), p.nx - 1));
    }
    for (int t = tid; t < 4 * (BY + 1); t += BX * BY) {
        const int w = t / (BY + 1), u = t - w * (BY + 1);
        ps.cy[w][u] = __ldg(tab(w, 1) + min(max(y0 - 1 + u, 0), p.ny - 1));
    }
}

// ------------------------------------------------------- TMA-fed z march
//
// The background tiles (no CPML) take their E^n and H^{n-1/2} planes from
// the tensor memory accelerator instead of per-thread loads: one thread
// issues a 4D tiled copy per plane (all three components, the tile with its
// halo, out-of-grid cells zero-filled) into a ring of shared-memory stages,
// each with an mbarrier that completes when the bytes have landed.  E planes
// k+2 and k+3 and H planes k+1 and k+2 are in flight while plane k is
// computed; a stage is refilled right after the block barrier that ends its
// last reader.  Boxes start at x0 - 4 so that the innermost coordinate stays
// a multiple of 16 bytes.

constexpr int TMA_EX = BX + 8;                 // 40 floats per row (x0-4 .. x0+35)
constexpr int TMA_EY = BY + 2;                 // rows y0-1 .. y0+BY
constexpr int TMA_HY = BY + 1;                 // rows y0-1 .. y0+BY-1
constexpr int TMA_E_FLOATS = 3 * TMA_EY * TMA_EX;
constexpr int TMA_H_FLOATS = 3 * TMA_HY * TMA_EX;
constexpr int TMA_E_STAGE = (TMA_E_FLOATS * 4 + 127) / 128 * 32;   // floats, 128-byte multiple
constexpr int TMA_H_STAGE = (TMA_H_FLOATS * 4 + 127) / 128 * 32;
constexpr int NE_STAGE = 4, NH_STAGE = 3;      // background tiles
constexpr int NE_PML = 3, NH_PML = 2, PML_BLOCKS = 4;   // CPML tiles (also stage psi): 4 blocks per SM
#ifdef NLF_TEST_TMA_STALL
// test-only build: the first E stage of every k_step block expects more
// bytes than its copy delivers, so its (shortened) bounded wait runs out
constexpr long long TMA_SPIN = 1LL << 10;
constexpr unsigned TMA_TEST_EXTRA = 16;
#else
constexpr long long TMA_SPIN = 1LL << 21;      // bounded mbarrier wait (~2 s at the hint below)
constexpr unsigned TMA_TEST_EXTRA = 0;
#endif

struct NoPsi {};

// CPML tiles skip the psi work of an axis in warps none of whose cells lies
// in that axis' slab, and map the threads of x-slab tiles so that half of
// their warps are clear of the slab (build option NLF_PML_NO_WARP_SKIP: every
// warp does all of its tile's psi work, lanes along x)
#ifdef NLF_PML_NO_WARP_SKIP
constexpr bool kWarpSkip = false;
#else
constexpr bool kWarpSkip = true;
#endif

// Metal tiles: node divergences of P_f^n (difference units) on three planes,
// plane q in slot q mod 3 (at plane k the z march reads planes k and k+1 and
// writes k+1; with one block barrier per plane a slot is rewritten only after
// every thread has left the last plane that read it), for the tile's own
// nodes and one node past it along +x and +y.
struct MetShared {
    float d[3][BY + 1][BX + 1];
};

template <int NE, int NH, bool PML, bool MET = false>
struct TileSharedTMA {
    static constexpr int kNE = NE, kNH = NH;
    static constexpr bool kPoisonFree = PML || MET;     // only the background kernel's tiles in the stall test
    alignas(128) float sE[NE][TMA_E_STAGE];
    alignas(128) float sHo[NH][TMA_H_STAGE];
    float sH[2][3][BY + 1][BX + 1];
    unsigned long long barE[NE];
    unsigned long long barH[NH];
    typename std::conditional<PML, PsiShared, NoPsi>::type ps;
    typename std::conditional<MET, MetShared, NoPsi>::type met;
};

__device__ __forceinline__ unsigned smem_u32(const void* ptr) { return (unsigned)__cvta_generic_to_shared(ptr); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Wait for phase `parity` of the barrier, giving up after TMA_SPIN tries
// (false: the copy did not land in time).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity)
{
    const unsigned a = smem_u32(bar);
    for (long long it = 0; it < TMA_SPIN; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, 1000;\n"
            " selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// One plane (all three components) of a [3][nz][ny][px] field: box origin
// (x, y, z, 0), completion on bar.
__device__ __forceinline__ void tma_plane(float* dst, const void* map, int x, int y, int z, unsigned long long* bar,
                                          unsigned bytes)
{
    mbar_expect(bar, bytes);
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

// The ring of one block's z march: issue (thread 0) and wait (every thread)
// by plane index.  Thread 0 also records which stages hold a copy not yet
// waited for, so that after a timed-out wait it can let the copies in flight
// land before the block exits.
template <class SM>
struct TmaRing {
    static constexpr int NE = SM::kNE, NH = SM::kNH;
    SM& sm;
    const StepParams& p;
    int k0, x0, y0;
    unsigned pendE = 0, parE = 0, pendH = 0, parH = 0;
    bool bad = false;
    // E plane pl lives in stage (pl - k0 + 1) mod NE, H plane pl in (pl - k0) mod NH;
    // the parity is that of the stage's use count
    __device__ int eslot(int pl) const { return (pl - k0 + 1) % NE; }
    __device__ unsigned epar(int pl) const { return (unsigned)(((pl - k0 + 1) / NE) & 1); }
    __device__ int hslot(int pl) const { return (pl - k0) % NH; }
    __device__ unsigned hpar(int pl) const { return (unsigned)(((pl - k0) / NH) & 1); }
    __device__ void issue_e(int pl)
    {
        const int q = eslot(pl);
        // (TMA_TEST_EXTRA: 0 except in the stall test build, which poisons
        // the first E stage of the background kernel's blocks)
        const unsigned extra = (TMA_TEST_EXTRA && !SM::kPoisonFree && pl == k0 - 1) ? TMA_TEST_EXTRA : 0u;
        tma_plane(sm.sE[q], p.map_in_params ? static_cast<const void*>(&p.mapE) : p.tmE, x0 - 4, y0 - 1, pl,
                  &sm.barE[q], TMA_E_FLOATS * 4 + extra);
        pendE |= 1u << q;
        parE = (parE & ~(1u << q)) | (epar(pl) << q);
    }
    __device__ void issue_h(int pl)
    {
        const int q = hslot(pl);
        tma_plane(sm.sHo[q], p.map_in_params ? static_cast<const void*>(&p.mapH) : p.tmH, x0 - 4, y0 - 1, pl,
                  &sm.barH[q], TMA_H_FLOATS * 4);
        pendH |= 1u << q;
        parH = (parH & ~(1u << q)) | (hpar(pl) << q);
    }
    __device__ void wait_e(int pl)
    {
        if (bad) return;
        if (mbar_wait(&sm.barE[eslot(pl)], epar(pl)))
            pendE &= ~(1u << eslot(pl));
        else
            bad = true;
    }
    __device__ void wait_h(int pl)
    {
        if (bad) return;
        if (mbar_wait(&sm.barH[hslot(pl)], hpar(pl)))
            pendH &= ~(1u << hslot(pl));
        else
            bad = true;
    }
    __device__ float e(int pl, int c, int y, int x) const { return sm.sE[eslot(pl)][(c * TMA_EY + y) * TMA_EX + x]; }
    __device__ float h(int pl, int c, int y, int x) const { return sm.sHo[hslot(pl)][(c * TMA_HY + y) * TMA_EX + x]; }
    // thread 0, after a block-wide failure: wait (bounded) for what is in flight
    __device__ void drain()
    {
        for (int q = 0; q < NE; ++q)
            if (pendE >> q & 1u) mbar_wait(&sm.barE[q], parE >> q & 1u);
        for (int q = 0; q < NH; ++q)
            if (pendH >> q & 1u) mbar_wait(&sm.barH[q], parH >> q & 1u);
    }
};

// (b, c) pairs of the A1 and A2 derivatives of component C (w = 0: E, 2: H).
template <int C>
__device__ __forceinline__ void cpml_pair(const PsiShared& ps, int w, int ux, int uy, const ZCoef& z, float2& pr1,
                                          float2& pr2)
{
    pr1 = cpml_coef<(C + 1) % 3>(ps, w, ux, uy, z);
    pr2 = cpml_coef<(C + 2) % 3>(ps, w, ux, uy, z);
}

// ------------------------------------------------- fused material update
//
// Metal tiles update their material E-sites inside the z march: E^{n+1} from
// Eq. discreteamperes with f3 and f4 substituted, P_CP and P_f (site_update),
// with GD^n = grad(div P_f^n) as the difference of node divergences staged in
// shared memory (MetShared).

// Material ids of the three E-sites of cell (i, j, k) (one byte each), 0
// outside the metal box; bi, bj are the cell's box-local column.
__device__ __forceinline__ uint32_t site_ids(const StepParams& p, bool in, int bi, int bj, int k)
{
    const int bk = k - p.bb_lo[2];
    if (!in || bi < 0 || bj < 0 || bk < 0 || bi >= p.bb_n[0] || bj >= p.bb_n[1] || bk >= p.bb_n[2]) return 0u;
    const uint32_t b = ((uint32_t)bk * (uint32_t)p.bb_n[1] + (uint32_t)bj) * (uint32_t)p.bb_n[0] + (uint32_t)bi;
    if (!NLF_IN(p, 8, b, p.nbb)) return 0u;
    return (uint32_t)__ldg(p.mat[0] + b) | ((uint32_t)__ldg(p.mat[1] + b) << 8) |
           ((uint32_t)__ldg(p.mat[2] + b) << 16);
}

// The six P_f^n values of the node divergence at node (i, j, k): P_x at the
// node and one cell down x, P_y likewise along y, P_z along z; zero unless
// the node lies at least one cell inside the metal box (no material site
// reads the divergence anywhere else).
__device__ __forceinline__ void div_load(const StepParams& p, int i, int j, int k, float (&v)[6])
{
    const int bi = i - p.bb_lo[0], bj = j - p.bb_lo[1], bk = k - p.bb_lo[2];
    if (bi < 1 || bj < 1 || bk < 1 || bi >= p.bb_n[0] || bj >= p.bb_n[1] || bk >= p.bb_n[2]) {
#pragma unroll
        for (int q = 0; q < 6; ++q) v[q] = 0.f;
        return;
    }
    const uint32_t sy = (uint32_t)p.bb_n[0], sz = (uint32_t)p.bb_n[0] * (uint32_t)p.bb_n[1];
    const uint32_t b = (uint32_t)bk * sz + (uint32_t)bj * sy + (uint32_t)bi;
    if (!(NLF_IN(p, 9, b, p.nbb) && NLF_IN(p, 9, (long long)b - sz, p.nbb))) {
#pragma unroll
        for (int q = 0; q < 6; ++q) v[q] = 0.f;
        return;
    }
    v[0] = __ldg(p.P0[0] + b);
    v[1] = __ldg(p.P0[0] + b - 1);
    v[2] = __ldg(p.P0[1] + b);
    v[3] = __ldg(p.P0[1] + b - sy);
    v[4] = __ldg(p.P0[2] + b);
    v[5] = __ldg(p.P0[2] + b - sz);
}

// The divergence from the six values, in the order of node_div.
__device__ __forceinline__ float div_sum(const float (&v)[6]) { return (v[0] - v[1]) + (v[2] - v[3]) + (v[4] - v[5]); }

// Node (x, y) of the tile's divergence plane that thread tid fills besides
// its own: the node past the tile along +x (tid < BY) or +y (BY <= tid <
// BY + BX); false for the other threads.
__device__ __forceinline__ bool div_extra(int tid, int& x, int& y)
{
    if (tid < BY) {
        x = BX;
        y = tid;
        return true;
    }
    if (tid < BY + BX) {
        x = tid - BY;
        y = BY;
        return true;
    }
    return false;
}

// The z march of one tile over planes [k0, k1).  PML (uniform per block):
// the tile or its halo reaches a CPML slab (psi arithmetic, psi staged by
// cp.async).  MP >= 0: a metal tile whose material sites (with at most MP
// critical-point poles) are updated in the march.
template <bool PML, int AX, class SM, int MP = -1>
__device__ __forceinline__ void march_tma(const StepParams& p, int x0, int y0, int k0, int k1, SM& sm)
{
    constexpr bool MET = MP >= 0;
    constexpr int NE = SM::kNE, NH = SM::kNH;
    // own cell of the thread: lanes along x, rows along y; in CPML tiles that
    // reach an x slab each warp covers 16 columns of two rows instead, so
    // that the warps of the half tile clear of the slab skip its psi work
    constexpr bool XR = PML && (AX & 1) && kWarpSkip;
    const int tid = threadIdx.y * BX + threadIdx.x;
    const int tx = XR ? ((tid & 15) + 16 * ((tid >> 5) & 1)) : (int)threadIdx.x;
    const int ty = XR ? (2 * (tid >> 6) + ((tid >> 4) & 1)) : (int)threadIdx.y;
    const int i = x0 + tx, j = y0 + ty;
    const bool in = i < p.nx && j < p.ny;
    const int lx = tx + 4, ly = ty + 1;               // own cell in an E or H stage
    // CPML geometry of the own column and of the halo column (constant along z)
    PmlCol qo{}, qh{};
    int wm_xy = 3;                                    // the warp's own cells reach the x (bit 0) / y (bit 1) slab
    if constexpr (PML) {
        qo = pml_col(p, i, j);
        if (tid < BY)
            qh = pml_col(p, x0 - 1, y0 + tid);
        else if (tid < BY + BX)
            qh = pml_col(p, x0 + tid - BY, y0 - 1);
        cpml_tables(p, sm.ps, x0, y0, tid);
        if (kWarpSkip)
            wm_xy = (__any_sync(0xffffffffu, in && qo.l0 >= 0) ? 1 : 0) |
                    (__any_sync(0xffffffffu, in && qo.l1 >= 0) ? 2 : 0);
    }
    const int wm_z = kWarpSkip ? 0 : 4;               // without the skip every axis is always on
    TmaRing<SM> r{sm, p, k0, x0, y0};
    if (tid == 0) {
        for (int q = 0; q < NE; ++q) mbar_init(&sm.barE[q]);
        for (int q = 0; q < NH; ++q) mbar_init(&sm.barH[q]);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        // maps read from the state were written to device memory by a copy
        // from the host, not by this proxy: the acquire takes system scope
        // (maps in the kernel parameter need no fence)
        if (!p.map_in_params) {
            asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;\n" ::"l"(p.tmE) : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;\n" ::"l"(p.tmH) : "memory");
        }
    }
    __syncthreads();
    // E planes k0-1 .. k0+NE-2 and H planes k0 .. k0+NH-1 (E is needed up to plane k1, H up to k1-1)
    if (tid == 0) {
        for (int pl = k0 - 1; pl <= k0 + NE - 2 && pl <= k1; ++pl) r.issue_e(pl);
        for (int pl = k0; pl <= k0 + NH - 1 && pl < k1; ++pl) r.issue_h(pl);
    }
    // H_x, H_y of plane k0-1 (own column) for the first E update
    float hx_prev = 0.f, hy_prev = 0.f;
    r.wait_e(k0 - 1);
    r.wait_e(k0);
    if (!r.bad && k0 > 0 && in) {
        Cell c = make_cell(p, i, j, k0 - 1, false);
        const int pm = k0 - 1;
        // psi_H of H_x (A1 = y, A2 = z) and H_y (A1 = z, A2 = x) at plane k0-1
        float px1 = 0.f, px2 = 0.f, py1 = 0.f, py2 = 0.f;
        float2 cx1{}, cx2{}, cy1{}, cy2{};
        if constexpr (PML) {
            pml_cell(p, qo, c);
            c.wm = wm_xy | wm_z | (c.l[2] >= 0 ? 4 : 0);
            if (c.l[1] >= 0 && NLF_IN(p, 6, c.s[1], p.psi_n[1])) px1 = __ldg(p.psiH0[1][1] + c.s[1]);
            if (c.l[2] >= 0 && NLF_IN(p, 6, c.s[2], p.psi_n[2])) px2 = __ldg(p.psiH0[2][0] + c.s[2]);
            if (c.l[2] >= 0 && NLF_IN(p, 6, c.s[2], p.psi_n[2])) py1 = __ldg(p.psiH0[2][1] + c.s[2]);
            if (c.l[0] >= 0 && NLF_IN(p, 6, c.s[0], p.psi_n[0])) py2 = __ldg(p.psiH0[0][0] + c.s[0]);
            const ZCoef zp = zcoef(p, k0 - 1);
            cpml_pair<0>(sm.ps, 2, tx + 1, ty + 1, zp, cx1, cx2);
            cpml_pair<1>(sm.ps, 2, tx + 1, ty + 1, zp, cy1, cy2);
        }
        const bool qok = NLF_IN(p, 1, c.q, p.nfield);
        hx_prev = h_cell<0, PML, AX>(p, c, qok ? __ldg(p.H0[0] + c.q) : 0.f, r.e(pm, 2, ly, lx), r.e(pm, 2, ly + 1, lx),
                                 r.e(pm, 1, ly, lx), r.e(k0, 1, ly, lx), false, px1, px2, cx1, cx2);
        hy_prev = h_cell<1, PML, AX>(p, c, qok ? __ldg(p.H0[1] + c.q) : 0.f, r.e(pm, 0, ly, lx), r.e(k0, 0, ly, lx),
                                 r.e(pm, 2, ly, lx), r.e(pm, 2, ly, lx + 1), false, py1, py2, cy1, cy2);
    }
    if constexpr (PML) psi_plane<AX>(p, sm.ps, 0, k0, x0, y0, i, j, in, qo, qh, tid, wm_xy | wm_z);
    bool fail = __syncthreads_or(r.bad);
    if (!fail && tid == 0 && k0 + NE - 1 <= k1) r.issue_e(k0 + NE - 1);
    // metal tile: the planes of this chunk that hold material sites of the
    // tile column, the own cell's box column, and the material ids of the
    // next plane (loaded a plane ahead)
    int kmin = 1, kmax = 0, mbi = 0, mbj = 0;
    uint32_t idn = 0;
    bool prev_mp = false;
    if constexpr (MET) {
        const int tix = (y0 / BY) * p.tiles_x + x0 / BX;
        const int2 kr = NLF_IN(p, 12, tix, p.ntiles_xy) ? p.tile_kr[tix] : make_int2(0, 0);
        kmin = max(p.nz - kr.x, k0);
        kmax = min(kr.y - 1, k1 - 1);
        mbi = i - p.bb_lo[0];
        mbj = j - p.bb_lo[1];
        if (kmin == k0 && kmin <= kmax) idn = site_ids(p, in, mbi, mbj, k0);
    }
    int hb = 0, pb = 0;
    for (int k = k0; k < k1 && !fail; ++k) {
        float (*sH)[BY + 1][BX + 1] = sm.sH[hb];
        const bool more = k + 1 < k1;
        // metal plane: operands of the material sites and of the node
        // divergences of plane k+1, issued before the plane's H work so that
        // their latency overlaps it
        const bool mp = MET && k >= kmin && k <= kmax;
        uint32_t ids = 0, bsite = 0;
        float so_p[3] = {}, so_a[3] = {}, so_g[3] = {}, so_c[3][1] = {}, so_q[3][1] = {};
        float dv_own[6] = {}, dv_ext[6] = {};
        int ex_x = 0, ex_y = 0;
        bool has_ext = false;
        if constexpr (MET) {
            if (mp) {
                has_ext = div_extra(tid, ex_x, ex_y);
                if (!prev_mp) {
                    // entering the metal: divergences of plane k itself
                    float v[6];
                    div_load(p, i, j, k, v);
                    sm.met.d[k % 3][ty][tx] = div_sum(v);
                    if (has_ext) {
                        div_load(p, x0 + ex_x, y0 + ex_y, k, v);
                        sm.met.d[k % 3][ex_y][ex_x] = div_sum(v);
                    }
                }
                div_load(p, i, j, k + 1, dv_own);
                if (has_ext) div_load(p, x0 + ex_x, y0 + ex_y, k + 1, dv_ext);
                ids = idn;
                if (ids) {
                    const int bk = k - p.bb_lo[2];
                    bsite = ((uint32_t)bk * (uint32_t)p.bb_n[1] + (uint32_t)mbj) * (uint32_t)p.bb_n[0] + (uint32_t)mbi;
                    if (!NLF_IN(p, 10, bsite, p.nbb)) ids = 0u;
#pragma unroll
                    for (int C = 0; C < 3; ++C) {
                        if (!((ids >> (8 * C)) & 0xffu)) continue;
                        so_p[C] = __ldg(p.P0[C] + bsite);
                        so_a[C] = p.auxf[C][bsite];
                        so_g[C] = p.any_gnor ? p.gdp[C][bsite] : 0.f;
                        if constexpr (MP >= 1) {
                            so_c[C][0] = p.pcp[0][C][bsite];
                            so_q[C][0] = p.auxcp[0][C][bsite];
                        }
                    }
                }
            }
            idn = (k + 1 >= kmin && k + 1 <= kmax) ? site_ids(p, in, mbi, mbj, k + 1) : 0u;
            prev_mp = mp;
        }
        r.wait_e(k + 1);
        r.wait_h(k);
        // this plane's stages: E^n of planes k and k+1, H^{n-1/2} of plane k
        const float* e0 = sm.sE[r.eslot(k)];
        const float* e1 = sm.sE[r.eslot(k + 1)];
        const float* h0 = sm.sHo[r.hslot(k)];
        auto E0 = [&](int c, int y, int x) { return e0[(c * TMA_EY + y) * TMA_EX + x]; };
        auto E1 = [&](int c, int y, int x) { return e1[(c * TMA_EY + y) * TMA_EX + x]; };
        auto H0 = [&](int c, int y, int x) { return h0[(c * TMA_HY + y) * TMA_EX + x]; };
        const float* po = nullptr;
        const float* ph = nullptr;
        if constexpr (PML) {
            // psi of plane k+1 on its way while plane k is computed
            if (more) {
                psi_plane<AX>(p, sm.ps, pb ^ 1, k + 1, x0, y0, i, j, in, qo, qh, tid, wm_xy | wm_z);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            po = &sm.ps.own[pb][0][tid];
            ph = &sm.ps.halo[pb][0][tid < BY + BX ? tid : 0];
        }
        Cell c;
        c.i = i;
        c.j = j;
        c.k = k;
        c.q = ((uint32_t)k * p.ny + j) * p.px + i;
        c.l[0] = c.l[1] = c.l[2] = -1;
        if constexpr (PML) {
            pml_cell(p, qo, c);
            c.wm = wm_xy | wm_z | (c.l[2] >= 0 ? 4 : 0);
        }
        ZCoef uz{};
        if constexpr (PML) uz = zcoef(p, k);      // plane k's coefficients along z
        float hx = 0.f, hy = 0.f, hz = 0.f;
        float ex = 0.f, ey = 0.f, ez = 0.f;
        // f1: own H^{n+1/2}
        if (in) {
            constexpr int S = BX * BY;
            float2 c1{}, c2{}, d1{}, d2{}, e1{}, e2{};
            if constexpr (PML) {
                cpml_pair<0>(sm.ps, 2, tx + 1, ty + 1, uz, c1, c2);
                cpml_pair<1>(sm.ps, 2, tx + 1, ty + 1, uz, d1, d2);
                cpml_pair<2>(sm.ps, 2, tx + 1, ty + 1, uz, e1, e2);
            }
            ex = E0(0, ly, lx);
            ey = E0(1, ly, lx);
            ez = E0(2, ly, lx);
            hx = h_cell<0, PML, AX>(p, c, H0(0, ly, lx), ez, E0(2, ly + 1, lx), ey, E1(1, ly, lx), true,
                                PML ? po[0 * S] : 0.f, PML ? po[1 * S] : 0.f, c1, c2);
            hy = h_cell<1, PML, AX>(p, c, H0(1, ly, lx), ex, E1(0, ly, lx), ez, E0(2, ly, lx + 1), true,
                                PML ? po[2 * S] : 0.f, PML ? po[3 * S] : 0.f, d1, d2);
            hz = h_cell<2, PML, AX>(p, c, H0(2, ly, lx), ey, E0(1, ly, lx + 1), ex, E0(0, ly + 1, lx), true,
                                PML ? po[4 * S] : 0.f, PML ? po[5 * S] : 0.f, e1, e2);
            sH[0][ly][tx + 1] = hx;
            sH[1][ly][tx + 1] = hy;
            sH[2][ly][tx + 1] = hz;
        }
        // halo H on two warps: H_y, H_z at x0-1 (threads 0..BY-1), H_x, H_z at y0-1 (BY..BY+BX-1)
        {
            constexpr int S = BX + BY;
            if (tid < BY) {
                const int jh = y0 + tid, sy = tid + 1;
                if (x0 > 0 && jh < p.ny) {
                    Cell h = make_cell(p, x0 - 1, jh, k, false);
                    float2 c1{}, c2{}, d1{}, d2{};
                    if constexpr (PML) {
                        pml_cell(p, qh, h);
                        cpml_pair<1>(sm.ps, 2, 0, sy, uz, c1, c2);
                        cpml_pair<2>(sm.ps, 2, 0, sy, uz, d1, d2);
                    }
                    sH[1][sy][0] = h_cell<1, PML, AX>(p, h, H0(1, sy, 3), E0(0, sy, 3), E1(0, sy, 3), E0(2, sy, 3),
                                                  E0(2, sy, 4), false, PML ? ph[0 * S] : 0.f,
                                                  PML ? ph[1 * S] : 0.f, c1, c2);
                    sH[2][sy][0] = h_cell<2, PML, AX>(p, h, H0(2, sy, 3), E0(1, sy, 3), E0(1, sy, 4), E0(0, sy, 3),
                                                  E0(0, sy + 1, 3), false, PML ? ph[2 * S] : 0.f,
                                                  PML ? ph[3 * S] : 0.f, d1, d2);
                }
            } else if (tid < BY + BX) {
                const int s0 = tid - BY, ih = x0 + s0, sx = s0 + 4;
                if (y0 > 0 && ih < p.nx) {
                    Cell h = make_cell(p, ih, y0 - 1, k, false);
                    float2 c1{}, c2{}, d1{}, d2{};
                    if constexpr (PML) {
                        pml_cell(p, qh, h);
                        cpml_pair<0>(sm.ps, 2, s0 + 1, 0, uz, c1, c2);
                        cpml_pair<2>(sm.ps, 2, s0 + 1, 0, uz, d1, d2);
                    }
                    sH[0][0][s0 + 1] = h_cell<0, PML, AX>(p, h, H0(0, 0, sx), E0(2, 0, sx), E0(2, 1, sx),
                                                      E0(1, 0, sx), E1(1, 0, sx), false, PML ? ph[0 * S] : 0.f,
                                                      PML ? ph[1 * S] : 0.f, c1, c2);
                    sH[2][0][s0 + 1] = h_cell<2, PML, AX>(p, h, H0(2, 0, sx), E0(1, 0, sx), E0(1, 0, sx + 1),
                                                      E0(0, 0, sx), E0(0, 1, sx), false, PML ? ph[2 * S] : 0.f,
                                                      PML ? ph[3 * S] : 0.f, d1, d2);
                }
            }
        }
        if constexpr (MET) {
            if (mp) {
                sm.met.d[(k + 1) % 3][ty][tx] = div_sum(dv_own);
                if (has_ext) sm.met.d[(k + 1) % 3][ex_y][ex_x] = div_sum(dv_ext);
            }
        }
        fail = __syncthreads_or(r.bad);
        if (fail) break;
        // E plane k and H plane k have had their last reader: refill their stages
        if (tid == 0) {
            if (k + NE <= k1) r.issue_e(k + NE);
            if (k + NH < k1) r.issue_h(k + NH);
        }
        // f2 on the tile (reads only sH and registers); tangential E on the walls stays zero
        if (in) {
            const int ox = tx + 1;
            const float hzm = sH[2][ly - 1][ox], hzi = sH[2][ly][ox - 1];
            const float hyi = sH[1][ly][ox - 1], hxm = sH[0][ly - 1][ox];
            if (PML) {
                constexpr int S = BX * BY;
                float2 c1{}, c2{}, d1{}, d2{}, e1{}, e2{};
                if constexpr (PML) {
                    cpml_pair<0>(sm.ps, 0, tx + 1, ty + 1, uz, c1, c2);
                    cpml_pair<1>(sm.ps, 0, tx + 1, ty + 1, uz, d1, d2);
                    cpml_pair<2>(sm.ps, 0, tx + 1, ty + 1, uz, e1, e2);
                }
                if (j >= 1 && k >= 1)
                    e_cell<0, PML, AX>(p, c, ex, hz, hzm, hy, hy_prev, PML ? po[6 * S] : 0.f, PML ? po[7 * S] : 0.f,
                                   c1, c2);
                else if (NLF_IN(p, 5, c.q, p.nfield))
                    p.E1[0][c.q] = 0.f;
                if (i >= 1 && k >= 1)
                    e_cell<1, PML, AX>(p, c, ey, hx, hx_prev, hz, hzi, PML ? po[8 * S] : 0.f, PML ? po[9 * S] : 0.f,
                                   d1, d2);
                else if (NLF_IN(p, 5, c.q, p.nfield))
                    p.E1[1][c.q] = 0.f;
                if (i >= 1 && j >= 1)
                    e_cell<2, PML, AX>(p, c, ez, hy, hyi, hx, hxm, PML ? po[10 * S] : 0.f, PML ? po[11 * S] : 0.f,
                                   e1, e2);
                else if (NLF_IN(p, 5, c.q, p.nfield))
                    p.E1[2][c.q] = 0.f;
            } else {
                const float cx = (hz - hzm) - (hy - hy_prev);
                const float cy = (hx - hx_prev) - (hz - hzi);
                const float cz = (hy - hyi) - (hx - hxm);
                float nx = (j >= 1 && k >= 1) ? ex + p.Sb * cx : 0.f;
                float ny = (i >= 1 && k >= 1) ? ey + p.Sb * cy : 0.f;
                float nz = (i >= 1 && j >= 1) ? ez + p.Sb * cz : 0.f;
                if constexpr (MET) {
                    if (ids) {
                        // material sites (never on a wall): GD from the staged divergences
                        const float (*dk)[BX + 1] = sm.met.d[k % 3];
                        const float (*dk1)[BX + 1] = sm.met.d[(k + 1) % 3];
                        const float d0 = dk[ty][tx];
                        const uint32_t idx = ids & 0xffu, idy = (ids >> 8) & 0xffu, idz = (ids >> 16) & 0xffu;
                        if (idx)
                            nx = site_update<0, 1>(p, bsite, idx, ex, cx, dk[ty][tx + 1] - d0, so_p[0], so_a[0],
                                                   so_g[0], so_c[0], so_q[0]);
                        if (idy)
                            ny = site_update<1, 1>(p, bsite, idy, ey, cy, dk[ty + 1][tx] - d0, so_p[1], so_a[1],
                                                   so_g[1], so_c[1], so_q[1]);
                        if (idz)
                            nz = site_update<2, 1>(p, bsite, idz, ez, cz, dk1[ty][tx] - d0, so_p[2], so_a[2],
                                                   so_g[2], so_c[2], so_q[2]);
                    }
                }
                if (NLF_IN(p, 5, c.q, p.nfield)) {
                    p.E1[0][c.q] = nx;
                    p.E1[1][c.q] = ny;
                    p.E1[2][c.q] = nz;
                }
            }
        }
        hx_prev = hx;
        hy_prev = hy;
        hb ^= 1;
        pb ^= 1;
    }
    if (fail && tid == 0) {
        atomicOr(p.err, 4);
        r.drain();
    }
    if constexpr (PML) cp_async_wait<0>();
}

// The CPML slab axes the box [lo, hi] (cells, inclusive) touches, bit a for
// axis a (0: a background tile).
__device__ __forceinline__ int tile_pml_axes(const StepParams& p, const int lo[3], const int hi[3])
{
    // the parameter block's members are copied, not addressed (an address
    // would move the block to local memory)
    const int n3[3] = {p.nx, p.ny, p.nz};
    const int cp[3] = {p.cpml[0], p.cpml[1], p.cpml[2]};
    return pml_axes_of_box(n3, cp, p.pml, lo, hi);
}


// The single-grid step runs as up to three kernels over the same grid of
// tiles: k_step_pml takes the CPML tiles, k_step_metal the tiles that hold
// material sites (with the material update fused), k_step the others, each
// block leaving at once if its tile belongs to another kernel.  k_step and
// k_step_pml run concurrently on two streams, k_step_metal after them.
// Without CPML or metal tiles k_step alone runs.
// Separate kernels let the background tiles run TMA-fed with fewer registers
// and without the psi staging area or the divergence ring: 5 blocks per SM.
enum { TILE_BG = 0, TILE_PML = 1, TILE_MET = 2 };

// Does tile (bx, by) with chunk [k0, k1) hold material sites that the fused
// march updates?
__device__ __forceinline__ bool metal_tile(const StepParams& p, int bx, int by, int k0, int k1)
{
    if (!p.fuse_metal) return false;
    const int tix = by * p.tiles_x + bx;
    if (!NLF_IN(p, 12, tix, p.ntiles_xy)) return false;
    const int2 kr = p.tile_kr[tix];
    return p.nz - kr.x < k1 && kr.y - 1 >= k0;
}

// The metal kernel marches the planes that k_step leaves to it (the chunks
// that hold material sites of the tile column) in sub-chunks of kzm planes
// (kzm divides kz, so kz / kzm sub-chunks cover an interior chunk): more,
// shorter marches for its heavier planes.  Returns false if sub-chunk bzm of
// tile (bx, by) is not one of them; [c0, c1) is the chunk that holds it.
__device__ __forceinline__ bool metal_subchunk(const StepParams& p, int bx, int by, int bzm, int kz, int kzm, int& k0,
                                               int& k1, int& c0, int& c1)
{
    const int per = kz / kzm;
    zchunk_range(p.nz, p.cpml[2], p.pml, kz, bzm / per, c0, c1);
    k0 = c0 + (bzm % per) * kzm;
    k1 = min(k0 + kzm, c1);
    return k0 < c1 && metal_tile(p, bx, by, c0, c1);
}

template <int KIND, int MP, class SM>
__device__ __forceinline__ void step_tile_of(const StepParams& p, int bx, int by, int bz, int kz, SM& sm, int kzm = 0)
{
    if (!NLF_CTX(p)) return;        // (uniform over the block)
    const int x0 = bx * BX, y0 = by * BY;
    int k0 = 0, k1 = 0, c0 = 0, c1 = 0;
    if constexpr (KIND == TILE_MET) {
        if (!metal_subchunk(p, bx, by, bz, kz, kzm, k0, k1, c0, c1)) return;
    } else {
        zchunk_range(p.nz, p.cpml[2], p.pml, kz, bz, k0, k1);
    }
    const int lo[3] = {x0 - 1, y0 - 1, k0 - 1};
    const int hi[3] = {x0 + BX, y0 + BY, k1};
    const int ax = tile_pml_axes(p, lo, hi);
    if constexpr (KIND == TILE_PML) {
        // tiles touching one slab axis run code with that axis' psi only
        if (ax == 1)
            march_tma<true, 1>(p, x0, y0, k0, k1, sm);
        else if (ax == 2)
            march_tma<true, 2>(p, x0, y0, k0, k1, sm);
        else if (ax == 4)
            march_tma<true, 4>(p, x0, y0, k0, k1, sm);
        else if (ax != 0)
            march_tma<true, 7>(p, x0, y0, k0, k1, sm);
    } else if constexpr (KIND == TILE_MET) {
        // the chunk's PML class is that of k_step's chunk, which holds the sub-chunk
        const int clo[3] = {x0 - 1, y0 - 1, c0 - 1};
        const int chi[3] = {x0 + BX, y0 + BY, c1};
        if (tile_pml_axes(p, clo, chi) == 0) march_tma<false, 0, SM, MP>(p, x0, y0, k0, k1, sm);
    } else {
        if (ax == 0 && !metal_tile(p, bx, by, k0, k1)) march_tma<false, 0>(p, x0, y0, k0, k1, sm);
    }
    // the 1D incident grid and the step counter: block (0,0,0) of k_step
    if (KIND == TILE_BG && bx == 0 && by == 0 && bz == 0) {
        const int tid = threadIdx.y * BX + threadIdx.x;
        if (p.tfsf) inc_step(p, tid, BX * BY);
        if (tid == 0) *p.step1 = *p.step0 + 1;
    }
}

using SharedBG = TileSharedTMA<NE_STAGE, NH_STAGE, false>;
using SharedPML = TileSharedTMA<NE_PML, NH_PML, true>;
using SharedMET = TileSharedTMA<NE_STAGE, NH_STAGE, false, true>;
// PML_BLOCKS blocks of the CPML kernel (plus the 1 KB the SM reserves per
// block) must fit the SM's 228 KB of shared memory
static_assert(PML_BLOCKS * (sizeof(SharedPML) + 128 + 1024) <= 228 * 1024, "CPML tile blocks do not fit an SM");
static_assert(sizeof(SharedMET) <= 48 * 1024, "metal tile shared memory exceeds the static limit");

__global__ void __launch_bounds__(BX * BY, 5) k_step(const __grid_constant__ StepParams p, int kz)
{
    __shared__ SharedBG sm;
    step_tile_of<TILE_BG, -1>(p, blockIdx.x, blockIdx.y, blockIdx.z, kz, sm);
}

// Metal tiles, MP critical-point poles at most.  Resident blocks per SM
// (4: 64 registers per thread) and the sub-chunk of the metal march
// (kz / NLF_METAL_KZ_DIV planes, at least 4) are build-time choices.  With
// the metal kernel beside the other two, whole chunks are the faster march
// (512^3 cube: 1.794 against 1.813 ms per step with halves of chunks).
#ifndef NLF_METAL_BLOCKS
#define NLF_METAL_BLOCKS 4
#endif
#ifndef NLF_METAL_KZ_DIV
#define NLF_METAL_KZ_DIV 1
#endif
template <int MP>
__global__ void __launch_bounds__(BX * BY, NLF_METAL_BLOCKS) k_step_metal(const __grid_constant__ StepParams p, int kz,
                                                                          int kzm)
{
    __shared__ SharedMET sm;
    step_tile_of<TILE_MET, MP>(p, blockIdx.x, blockIdx.y, blockIdx.z, kz, sm, kzm);
}

// CPML tiles: TMA rings plus the psi staging area exceed the 48 KB of static
// shared memory, so the block's area is dynamic (aligned here to 128 bytes).
__global__ void __launch_bounds__(BX * BY, PML_BLOCKS) k_step_pml(const __grid_constant__ StepParams p, int kz)
{
    extern __shared__ unsigned char nlf_dyn_smem[];
    const unsigned mis = smem_u32(nlf_dyn_smem) & 127u;
    SharedPML& sm = *reinterpret_cast<SharedPML*>(nlf_dyn_smem + ((128u - mis) & 127u));
    // z chunks in the order 0, n-1, 1, n-2, ...: the first and last chunks,
    // CPML tiles only, start first, and the blocks left at the end are the
    // few CPML tiles of middle chunks, which share the SMs with background
    // tiles instead of running as an under-filled tail
    const int zb = (int)blockIdx.z, nzb = (int)gridDim.z;
    step_tile_of<TILE_PML, -1>(p, blockIdx.x, blockIdx.y, (zb & 1) ? nzb - 1 - (zb >> 1) : (zb >> 1), kz, sm);
}

// ---------------------------------------------------------------- batched

// Find the instance of work item w: the first q with end[q] > w.
__device__ __forceinline__ int find_inst(const long long* end, int n, long long w)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (end[mid] > w)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// ------------------------------------------------------------- TF/SF
//
// The total-field / scattered-field connection, applied after the EM step as
// additive corrections.  The step kernels update every cell as if the grid
// held one field; the TF/SF surface then needs H_y on the planes
// k = lo_z - 1 and k = hi_z and H_z on the planes j = lo_y - 1 and j = hi_y
// (scattered-field cells whose curl reads a total-field E_x) corrected by the
// incident E_inc^n, and E_x on k = lo_z, hi_z and E_z on i = lo_x, hi_x
// (total-field cells whose curl reads a scattered-field H) corrected by the
// incident H_inc^{n+1/2}.  The update is linear, so E^{n+1} of every cell whose
// curl reads a corrected H also receives Sb curl(dH); the cells so touched
// are gathered here, each with its whole correction.  TF/SF cells lie outside
// the CPML and the metal, so only the background coefficient Sb appears.
//
// Item sets (i in [lo_x, hi_x) unless stated, j/k ranges inclusive):
//   0  E_x, j in [lo_y, hi_y], k in {lo_z-1, lo_z, hi_z, hi_z+1}
//   1  E_x, j in {lo_y-1, lo_y, hi_y, hi_y+1}, k in [lo_z, hi_z] (not in set 0)
//   2  E_y, i in {lo_x, hi_x}, j in {lo_y-1, hi_y}, k in [lo_z, hi_z]
//   3  E_z, i in {lo_x, hi_x}, j in [lo_y, hi_y], k in [lo_z-1, hi_z]
//   4  H_y, j in [lo_y, hi_y], k in {lo_z-1, hi_z}
//   5  H_z, j in {lo_y-1, hi_y}, k in [lo_z, hi_z]
// Sizes of the six item sets, in order.
__host__ __device__ __forceinline__ void tfsf_sizes(const StepParams& p, long long n[6])
{
    const long long nx = p.tf_hi[0] - p.tf_lo[0], ny = p.tf_hi[1] - p.tf_lo[1] + 1,
                    nz = p.tf_hi[2] - p.tf_lo[2] + 1;
    n[0] = nx * ny * 4;
    n[1] = nx * 4 * nz;
    n[2] = 4 * nz;
    n[3] = 2 * ny * (nz + 1);
    n[4] = nx * ny * 2;
    n[5] = nx * 2 * nz;
}

__host__ __device__ __forceinline__ long long tfsf_count(const StepParams& p)
{
    if (!p.tfsf) return 0;
    long long n[6];
    tfsf_sizes(p, n);
    return n[0] + n[1] + n[2] + n[3] + n[4] + n[5];
}

__device__ __forceinline__ void tfsf_item(const StepParams& p, long long t)
{
    if (!NLF_CTX(p)) return;
    const int l0 = p.tf_lo[0], h0 = p.tf_hi[0], l1 = p.tf_lo[1], h1 = p.tf_hi[1], l2 = p.tf_lo[2],
              h2 = p.tf_hi[2];
    const int nx = h0 - l0, ny = h1 - l1 + 1;
    long long n[6];
    tfsf_sizes(p, n);
    int set = 0;
    long long r = t;
    while (set < 6 && r >= n[set]) r -= n[set++];
    if (set == 6) return;
    const float S = p.S, Sb = p.Sb;
    // dH_y on k = lo_z - 1, hi_z and dH_z on j = lo_y - 1, hi_y (plane k)
    const float dy_lo = S * e_inc(p, l2), dy_hi = -S * e_inc(p, h2);
    auto dz = [&](int jh, int k) { return (jh == l1 - 1 ? -S : S) * e_inc(p, k); };
    int i, j, k, comp;
    float v = 0.f;
    bool isH = false;
    if (set == 0 || set == 1) {
        comp = 0;
        i = l0 + (int)(r % nx);
        r /= nx;
        if (set == 0) {
            j = l1 + (int)(r % ny);
            const int kk[4] = {l2 - 1, l2, h2, h2 + 1};
            k = kk[r / ny];
        } else {
            const int jj[4] = {l1 - 1, l1, h1, h1 + 1};
            j = jj[r % 4];
            k = l2 + (int)(r / 4);
            if ((j == l1 || j == h1) && (k == l2 || k == h2)) return;   // in set 0
        }
        if (j >= l1 && j <= h1) {
            if (k == l2 - 1) v -= Sb * dy_lo;
            if (k == l2) v += Sb * dy_lo + Sb * h_inc_next(p, l2 - 1);
            if (k == h2) v -= Sb * dy_hi + Sb * h_inc_next(p, h2);
            if (k == h2 + 1) v += Sb * dy_hi;
        }
        if (k >= l2 && k <= h2) {
            if (j == l1 - 1 || j == h1) v += Sb * dz(j, k);
            if (j == l1) v -= Sb * dz(l1 - 1, k);
            if (j == h1 + 1) v -= Sb * dz(h1, k);
        }
    } else if (set == 2) {
        comp = 1;
        i = (r & 1) ? h0 : l0;
        j = (r & 2) ? h1 : l1 - 1;
        k = l2 + (int)(r >> 2);
        v = (i == l0 ? -Sb : Sb) * dz(j, k);
    } else if (set == 3) {
        comp = 2;
        i = (r & 1) ? h0 : l0;
        r >>= 1;
        j = l1 + (int)(r % ny);
        k = l2 - 1 + (int)(r / ny);
        const float sg = i == l0 ? 1.f : -1.f;
        if (k == l2 - 1) v += sg * Sb * dy_lo;
        if (k == h2) v += sg * Sb * dy_hi;
        if (k >= l2 && k < h2) v -= sg * Sb * h_inc_next(p, k);
    } else if (set == 4) {
        comp = 1;
        isH = true;
        i = l0 + (int)(r % nx);
        r /= nx;
        j = l1 + (int)(r % ny);
        k = (r / ny) ? h2 : l2 - 1;
        v = k == h2 ? dy_hi : dy_lo;
    } else {
        comp = 2;
        isH = true;
        i = l0 + (int)(r % nx);
        r /= nx;
        j = (r & 1) ? h1 : l1 - 1;
        k = l2 + (int)(r >> 1);
        v = dz(j, k);
    }
    // a TF surface one cell from a wall: tangential E on index 0 is the wall
    // (held at zero) and index n lies beyond it, so neither is corrected
    if (!isH && ((comp != 0 && i == 0) || (comp != 1 && j == 0) || (comp != 2 && k == 0) || i >= p.nx ||
                 j >= p.ny || k >= p.nz))
        return;
    const uint32_t q = ((uint32_t)k * p.ny + j) * p.px + i;
    float* f = isH ? p.H1[comp] : p.E1[comp];
    if (NLF_IN(p, 16, q, p.nfield)) f[q] += v;
}

__global__ void __launch_bounds__(256) k_tfsf(const StepParams p, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) tfsf_item(p, t);
}

// The material update and the TF/SF corrections in one launch: blocks below
// nb_metal take material sites, the rest TF/SF items.  The two touch disjoint
// cells (material sites lie at least two cells inside the TF surface), so no
// order between them is needed, and the short TF/SF blocks fill the SMs the
// material blocks leave at the end of the launch.
__global__ void __launch_bounds__(256, 8) k_post(const StepParams p, long long n_sites, long long nb_metal, long long n_tf)
{
    const long long bx = blockIdx.x;
    if (bx < nb_metal) {
        const long long t = bx * blockDim.x + threadIdx.x;
        if (t < n_sites) metal_entry(p, t);
    } else {
        const long long t = (bx - nb_metal) * blockDim.x + threadIdx.x;
        if (t < n_tf) tfsf_item(p, t);
    }
}

// Batched grids: one block per work item (instance, tile, z chunk) of the
// concatenated list of every instance.  As for a single grid, two kernels
// take the list concurrently, k_step_batch the background tiles
// (TMA-fed) and k_step_batch_pml the CPML tiles, each block leaving at once if
// its tile belongs to the other kernel.  A block stages its instance's
// parameters in shared memory first (for the CPML blocks this leaves room
// for three blocks per SM, not four; read from the descriptor array instead,
// the 64 batched instances ran at 32.7 against 36.3 Gcell-updates/s).
template <bool PMLK, class SM>
__device__ __forceinline__ void batch_item(const BatchStep& a, SM& sm, StepParams& sp)
{
    const int tid = threadIdx.y * BX + threadIdx.x;
    const long long w = blockIdx.x;
    const int q = find_inst(a.item_end, a.n, w);
    const BatchInst& I = a.inst[q];
    const int par = I.base_par ^ a.launch_par;
    const int* src = reinterpret_cast<const int*>(&a.params[2 * q + par]);
    int* dst = reinterpret_cast<int*>(&sp);
    for (int t = tid; t < (int)(sizeof(StepParams) / sizeof(int)); t += BX * BY) dst[t] = src[t];
    __syncthreads();
    const long long r = w - (q > 0 ? a.item_end[q - 1] : 0);
    const long long per_plane = (long long)I.tiles_x * I.tiles_y;
    const int bz = (int)(r / per_plane);
    const long long rem = r - bz * per_plane;
    const int by = (int)(rem / I.tiles_x);
    const int bx = (int)(rem - (long long)by * I.tiles_x);
    step_tile_of<PMLK ? TILE_PML : TILE_BG, -1>(sp, bx, by, bz, I.kz, sm);
}

__global__ void __launch_bounds__(BX * BY, 5) k_step_batch(const BatchStep a)
{
    __shared__ SharedBG sm;
    __shared__ StepParams sp;
    batch_item<false>(a, sm, sp);
}

constexpr size_t kPmlSpOff = (sizeof(SharedPML) + 127) / 128 * 128;

__global__ void __launch_bounds__(BX * BY, PML_BLOCKS) k_step_batch_pml(const BatchStep a)
{
    extern __shared__ unsigned char nlf_dyn_smem[];
    const unsigned mis = smem_u32(nlf_dyn_smem) & 127u;
    unsigned char* base = nlf_dyn_smem + ((128u - mis) & 127u);
    SharedPML& sm = *reinterpret_cast<SharedPML*>(base);
    StepParams& sp = *reinterpret_cast<StepParams*>(base + kPmlSpOff);
    batch_item<true>(a, sm, sp);
}

// Dynamic shared memory above 48 KB must be granted per kernel and device.
template <class K>
void grant_smem(K kernel, size_t bytes, bool* granted)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !granted[dev]) {
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess &&
            dev >= 0 && dev < 64)
            granted[dev] = true;
    }
}

void launch_step_batch(const BatchStep& a, long long total_items, cudaStream_t st)
{
    if (total_items <= 0) return;
    k_step_batch<<<(unsigned)total_items, dim3(BX, BY, 1), 0, st>>>(a);
}

void launch_step_batch_pml(const BatchStep& a, long long total_items, cudaStream_t st)
{
    if (total_items <= 0) return;
    constexpr size_t smem = kPmlSpOff + sizeof(StepParams) + 128;
    static bool granted[64] = {};
    grant_smem(k_step_batch_pml, smem, granted);
    k_step_batch_pml<<<(unsigned)total_items, dim3(BX, BY, 1), smem, st>>>(a);
}

// Batched post-step work: the material sites of every instance (prefix sums
// met_end), then the TF/SF correction items of every instance (prefix sums
// tf_end), one per thread over the concatenated list; the two touch
// disjoint cells of each instance, so one launch takes both.
__global__ void __launch_bounds__(256) k_post_batch(const BatchStep a)
{
    __shared__ long long s_met[NLF_MAX_BATCH], s_tf[NLF_MAX_BATCH];
    for (int q = threadIdx.x; q < a.n; q += blockDim.x) {
        s_met[q] = a.met_end[q];
        s_tf[q] = a.tf_end[q];
    }
    __syncthreads();
    const long long n_met = s_met[a.n - 1], total = n_met + s_tf[a.n - 1];
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= total) return;
    if (w < n_met) {
        const int q = find_inst(s_met, a.n, w);
        const StepParams& p = a.params[2 * q + (a.inst[q].base_par ^ a.launch_par)];
        metal_entry(p, w - (q > 0 ? s_met[q - 1] : 0));
    } else {
        const long long t = w - n_met;
        const int q = find_inst(s_tf, a.n, t);
        const StepParams& p = a.params[2 * q + (a.inst[q].base_par ^ a.launch_par)];
        tfsf_item(p, t - (q > 0 ? s_tf[q - 1] : 0));
    }
}

void launch_metal(const StepParams& p, long long n_sites, cudaStream_t st)
{
    if (n_sites <= 0) return;
    k_metal<<<(unsigned)((n_sites + 255) / 256), 256, 0, st>>>(p, n_sites);
}

// One site or item per thread: the material update is a chain of dependent
// loads, and more threads in flight hide it better than a resident
// grid-stride loop (64 batched instances: 36.1 against 35.7 Gcell-updates/s
// with the grid held to 8 blocks per SM, before the TF/SF items joined).
void launch_post_batch(const BatchStep& a, long long total_sites, long long total_tf, cudaStream_t st)
{
    const long long g = (total_sites + total_tf + 255) / 256;
    if (g > 0) k_post_batch<<<(unsigned)g, 256, 0, st>>>(a);
}

int step_chunks(const StepParams& p, int kz) { return zchunk_count(p.nz, p.cpml[2], p.pml, kz); }

int step_kz(const StepParams& p)
{
    // z chunk: enough blocks for several waves over 152 SMs, few chunk prologues
    const long long tiles = (long long)((p.nx + BX - 1) / BX) * ((p.ny + BY - 1) / BY);
    int kz = 32;
    while (kz > 8 && tiles * step_chunks(p, kz) < 4 * 152 * 4) kz /= 2;
    return kz;
}

bool step_has_pml(const StepParams& p) { return p.cpml[0] || p.cpml[1] || p.cpml[2]; }

long long tfsf_items(const StepParams& p) { return tfsf_count(p); }

void launch_tfsf(const StepParams& p, cudaStream_t st)
{
    const long long n = tfsf_count(p);
    if (n > 0) k_tfsf<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, n);
}

void launch_post(const StepParams& p, long long n_sites, cudaStream_t st)
{
    const long long n_tf = tfsf_count(p);
    const long long nb_m = (n_sites + 255) / 256, nb_t = (n_tf + 255) / 256;
    if (nb_m + nb_t > 0) k_post<<<(unsigned)(nb_m + nb_t), 256, 0, st>>>(p, n_sites, nb_m, n_tf);
}

void launch_step(const StepParams& p, cudaStream_t st)
{
    const int kz = step_kz(p);
    dim3 blk(BX, BY, 1);
    dim3 grd((p.nx + BX - 1) / BX, (p.ny + BY - 1) / BY, step_chunks(p, kz));
    k_step<<<grd, blk, 0, st>>>(p, kz);
}

void launch_step_metal(const StepParams& p, cudaStream_t st)
{
    const int kz = step_kz(p);
    const int kzm = max(min(4, kz), kz / NLF_METAL_KZ_DIV);
    dim3 blk(BX, BY, 1);
    dim3 grd((p.nx + BX - 1) / BX, (p.ny + BY - 1) / BY, step_chunks(p, kz) * (kz / kzm));
    if (p.max_poles >= 1)
        k_step_metal<1><<<grd, blk, 0, st>>>(p, kz, kzm);
    else
        k_step_metal<0><<<grd, blk, 0, st>>>(p, kz, kzm);
}

void launch_step_pml(const StepParams& p, cudaStream_t st)
{
    const int kz = step_kz(p);
    constexpr size_t smem = sizeof(SharedPML) + 128;
    static bool granted[64] = {};
    grant_smem(k_step_pml, smem, granted);
    dim3 blk(BX, BY, 1);
    dim3 grd((p.nx + BX - 1) / BX, (p.ny + BY - 1) / BY, step_chunks(p, kz));
    k_step_pml<<<grd, blk, smem, st>>>(p, kz);
}

}  // namespace nlf
