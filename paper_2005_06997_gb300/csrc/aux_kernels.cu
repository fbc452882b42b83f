// aux_kernels.cu -- voxeliser, running DFT and flux reduction kernels.
#include <cuda_runtime.h>

#include "nlf_internal.h"
#include "dft_accum.cuh"

namespace nlf {

// ---------------------------------------------------------------- voxeliser
// Integer containment tests in half-cell units (bit-exact with any correct
// implementation of the same definitions).

__device__ __forceinline__ long long sq(long long v) { return v * v; }

__device__ bool contains(const Shape& s, long long p0, long long p1, long long p2)
{
    const long long d[3] = {p0 - s.c[0], p1 - s.c[1], p2 - s.c[2]};
    if (s.kind == 1) return sq(d[0]) + sq(d[1]) + sq(d[2]) <= sq(s.radius);
    if (s.kind == 2) return llabs(d[0]) <= s.half[0] && llabs(d[1]) <= s.half[1] && llabs(d[2]) <= s.half[2];
    if (s.kind == 3) {
        const long long A = s.side / 2, B = s.tip_base / 2, h = s.tip_height;
        if (llabs(d[0]) <= A && llabs(d[1]) <= A && llabs(d[2]) <= A) return true;
        for (int ax = 0; ax < 3; ++ax) {
            const long long v = llabs(d[(ax + 1) % 3]), w = llabs(d[(ax + 2) % 3]);
            for (int sg = -1; sg <= 1; sg += 2) {
                const long long t = sg * d[ax];
                if (sq(t - s.tip_center) + sq(v) + sq(w) <= sq(s.tip_radius)) return true;
                if (t >= A && t <= s.tip_cut && h * v <= B * (A + h - t) && h * w <= B * (A + h - t)) return true;
            }
        }
    }
    return false;
}

__global__ void k_voxelise(const VoxParams v)
{
    const long long nb = (long long)v.bb_n[0] * v.bb_n[1] * v.bb_n[2];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nb) return;
    const int c = (int)(t / nb);
    const long long r = t - c * nb;
    const int bi = (int)(r % v.bb_n[0]);
    const int bj = (int)((r / v.bb_n[0]) % v.bb_n[1]);
    const int bk = (int)(r / ((long long)v.bb_n[0] * v.bb_n[1]));
    const long long p0 = 2LL * (bi + v.bb_lo[0]) + (c == 0);
    const long long p1 = 2LL * (bj + v.bb_lo[1]) + (c == 1);
    const long long p2 = 2LL * (bk + v.bb_lo[2]) + (c == 2);
    int id = 0;
    for (int q = 0; q < v.nshape; ++q) {
        if (contains(v.shp[q], p0, p1, p2)) {
            id = v.shp[q].material;
            break;
        }
    }
    v.mat[c][r] = (uint8_t)id;
    if (id != 0 && v.free_e[id]) atomicAdd(&v.counts[c], 1ULL);
}

// Compact list of the E-sites of the metal box that hold a material, entry
// (component << 30) | box offset.  Each warp reserves its run with one atomic,
// so runs land in any order while each run keeps box order; the material
// update is independent per site, so the order does not change any result.
// With g.only_pml the list keeps the sites of tiles that reach a CPML slab
// (the EM kernel updates the others in its z-march); with g.tile_kr every
// material site also widens the z range of its tile column.  count[0]
// receives the entries, count[1] those with free electrons.
__global__ void k_site_list(const uint8_t* __restrict__ mat, long long n3, uint32_t* sites, uint32_t* site_q,
                            long long nb, SiteGeom g, unsigned long long* count)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const uint8_t id = t < n3 ? mat[t] : 0;
    bool has = id != 0;
    uint32_t c = 0, b = 0;
    int i = 0, j = 0, k = 0;
    if (has) {
        c = (uint32_t)(t / nb);
        b = (uint32_t)(t - (long long)c * nb);
        const uint32_t bi = b % (uint32_t)g.bb_n[0], r = b / (uint32_t)g.bb_n[0];
        const uint32_t bj = r % (uint32_t)g.bb_n[1], bk = r / (uint32_t)g.bb_n[1];
        i = g.bb_lo[0] + (int)bi;
        j = g.bb_lo[1] + (int)bj;
        k = g.bb_lo[2] + (int)bk;
        if (g.tile_kr) {
            int2* kr = g.tile_kr + (j / NLF_TILE_BY) * g.tiles_x + i / NLF_TILE_BX;
            atomicMax(&kr->x, g.nz - k);
            atomicMax(&kr->y, k + 1);
        }
        if (g.only_pml) {
            const int n3g[3] = {g.nx, g.ny, g.nz};
            has = cell_in_pml_tile(n3g, g.cpml, g.pml, g.kz, i, j, k);
        }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, has);
    if (mask == 0u) return;
    const unsigned pmask = __ballot_sync(0xffffffffu, has && g.free_e[id]);
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) {
        base = atomicAdd(&count[0], (unsigned long long)__popc(mask));
        atomicAdd(&count[1], (unsigned long long)__popc(pmask));
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (has) {
        const unsigned long long w = base + __popc(mask & ((1u << lane) - 1u));
        // a site of a CPML cell is flagged: the metal is local Drude there
        const int ix[3] = {i, j, k}, n3g[3] = {g.nx, g.ny, g.nz};
        bool in_cpml = false;
        for (int a = 0; a < 3; ++a)
            if (g.cpml[a] && (ix[a] < g.pml || ix[a] >= n3g[a] - g.pml)) in_cpml = true;
        sites[w] = (c << 30) | (in_cpml ? NLF_SITE_IN_CPML : 0u) | b;
        site_q[w] = ((uint32_t)k * (uint32_t)g.ny + (uint32_t)j) * (uint32_t)g.px + (uint32_t)i;
    }
}

void launch_site_list(const uint8_t* mat, long long nb, uint32_t* sites, uint32_t* site_q, const SiteGeom& g,
                      unsigned long long* count, cudaStream_t st)
{
    const long long n = 3 * nb;
    k_site_list<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mat, n, sites, site_q, nb, g, count);
}

// Non-finite watchdog over the whole grid: every value of E^n (three
// components, padding cells included, which stay zero).  A non-finite value
// anywhere in the state reaches E within a step or two, so checking E once
// per period covers the grid; it raises bit 0 of the error word.
__global__ void __launch_bounds__(256) k_watch(const float4* __restrict__ E, long long n4, int* err)
{
    bool bad = false;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
        const float4 v = __ldg(E + q);
        bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, 1);
}

void launch_watch(const float* E, long long nfloats, int* err, cudaStream_t st)
{
    const long long n4 = nfloats / 4;
    long long g = (n4 + 255) / 256;
    if (g > 152LL * 8) g = 152LL * 8;
    k_watch<<<(unsigned)g, 256, 0, st>>>(reinterpret_cast<const float4*>(E), n4, err);
}

void launch_voxelise(const VoxParams& v, cudaStream_t st)
{
    const long long nb = (long long)v.bb_n[0] * v.bb_n[1] * v.bb_n[2];
    const long long n = 3 * nb;
    k_voxelise<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v);
}

// ------------------------------------------------------------- running DFT

// Store one FP32 sample of every flux record (E at n dt, H averaged over the
// two half cells around the face, at (n - 1/2) dt) into slot `slot`.  A
// non-finite sample raises bit 0 of the error word (the instability watchdog).
__global__ void k_dft_gather(const DftParams d, const float* __restrict__ E, const float* __restrict__ H,
                             const float* __restrict__ e_inc, const float* __restrict__ h_inc, int slot,
                             const long long* __restrict__ step, int* err)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > d.nrec || !NLF_CTX(d)) return;
    float e, h;
    if (r < d.nrec) {
        const uint32_t oe = d.rec_e[r], o = d.rec_h[r], hs = d.rec_hs[r];
        if (!(NLF_IN(d, 17, oe, d.nfield3) && NLF_IN(d, 18, (long long)o + hs, d.nfield3))) return;
        e = __ldg(E + oe);
        h = 0.5f * (__ldg(H + o) + __ldg(H + o + hs));
    } else {
        e = e_inc[d.inc_node];
        h = 0.5f * (h_inc[d.inc_node - 1] + h_inc[d.inc_node]);
        d.sample_step[slot] = *step;
    }
    const long long w = (long long)slot * (d.nrec + 1) + r;
    if (!NLF_IN(d, 19, w, (long long)d.B * (d.nrec + 1))) return;
    d.sE[w] = e;
    d.sH[w] = h;
    if (!isfinite(e) || !isfinite(h)) atomicOr(err, 1);
}

// Phase table: cos/sin(w_f n dt) and cos/sin(w_f (n - 1/2) dt) per filled
// slot, from the integer step index in FP64; zeros for unfilled slots.
__global__ void k_dft_phase(const DftParams d, int count)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d.B * d.nf || !NLF_CTX(d)) return;
    const int s = t / d.nf, f = t - s * d.nf;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < count) {
        const double n = (double)d.sample_step[s];
        const double w = d.omega[f];
        double se, ce, sh, ch;
        sincos(w * n * d.dt, &se, &ce);
        sincos(w * (n - 0.5) * d.dt, &sh, &ch);
        v = make_float4((float)ce, (float)se, (float)ch, (float)sh);
    }
    d.phase[t] = v;
}

// One flush of the running DFT: block = ACC_NT frequencies x ACC_NCH chunks
// of RCH records (accum_block).
template <int B, int RCH>
__global__ void __launch_bounds__(ACC_NT, 4) k_dft_accum(const DftParams d)
{
    __shared__ AccShared<B, RCH> sm;
    accum_block<B, RCH>(d, (long long)blockIdx.x * RCH * ACC_NCH, ACC_NCH, blockIdx.y * ACC_NT, sm);
}

void launch_dft_gather(const DftParams& d, const float* E, const float* H, const float* e_inc, const float* h_inc,
                       int slot, const long long* step, int* err, cudaStream_t st)
{
    const long long n = d.nrec + 1;
    k_dft_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, E, H, e_inc, h_inc, slot, step, err);
}

void launch_dft_flush(const DftParams& d, int count, cudaStream_t st)
{
    const int np = d.B * d.nf;
    k_dft_phase<<<(np + 255) / 256, 256, 0, st>>>(d, count);
    constexpr int RCH = 32;
    constexpr long long per = (long long)RCH * ACC_NCH;
    dim3 grd((unsigned)((d.nrec + 1 + per - 1) / per), (unsigned)((d.nf + ACC_NT - 1) / ACC_NT));
    if (d.B <= 8)
        k_dft_accum<8, RCH><<<grd, ACC_NT, 0, st>>>(d);
    else if (d.B <= 16)
        k_dft_accum<16, RCH><<<grd, ACC_NT, 0, st>>>(d);
    else
        k_dft_accum<32, RCH><<<grd, ACC_NT, 0, st>>>(d);
}

// ----------------------------------------------------------------- fluxes

// partial[g][f] = (sum over records r = g, g+G, ... of the absorption box,
// same for the scattering box) of coef_r Re(E_r H_r^*), FP64.
__global__ void k_flux_partial(const double2* __restrict__ accE, const double2* __restrict__ accH,
                               const double* __restrict__ coef, long long n_abs, long long nrec, int nf,
                               double2* __restrict__ partial)
{
    const int f = blockIdx.y * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int G = gridDim.x;
    double sa = 0.0, ss = 0.0;
    for (long long r = blockIdx.x; r < nrec; r += G) {
        const double2 e = accE[r * nf + f], h = accH[r * nf + f];
        const double v = __ldg(coef + r) * (e.x * h.x + e.y * h.y);
        if (r < n_abs)
            sa += v;
        else
            ss += v;
    }
    partial[(long long)blockIdx.x * nf + f] = make_double2(sa, ss);
}

// sigma_abs = -dA S_abs / I, sigma_sca = dA S_sca / I, I = Re(E_inc H_inc^*) / 2.
__global__ void k_flux_final(const double2* __restrict__ accE, const double2* __restrict__ accH, long long nrec,
                             int nf, const double2* __restrict__ partial, int G, double dA, double* out)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    double sa = 0.0, ss = 0.0;
    for (int g = 0; g < G; ++g) {
        const double2 v = partial[(long long)g * nf + f];
        sa += v.x;
        ss += v.y;
    }
    const double2 e = accE[nrec * nf + f], h = accH[nrec * nf + f];
    const double I = 0.5 * (e.x * h.x + e.y * h.y);
    const double s_abs = -sa * dA / I, s_sca = ss * dA / I;
    out[f] = s_abs + s_sca;
    out[nf + f] = s_abs;
    out[2 * nf + f] = s_sca;
    out[3 * nf + f] = I;
}

void launch_flux(const double2* accE, const double2* accH, const double* coef, long long n_abs, long long nrec,
                 int nf, double2* partial, int G, double dA, double* out, cudaStream_t st)
{
    dim3 grd(G, (nf + 127) / 128);
    k_flux_partial<<<grd, 128, 0, st>>>(accE, accH, coef, n_abs, nrec, nf, partial);
    k_flux_final<<<(nf + 127) / 128, 128, 0, st>>>(accE, accH, nrec, nf, partial, G, dA, out);
}

}  // namespace nlf

namespace nlf {

// P_f component c (P/eps0) at node (i, j, k); zero outside the metal box.
__device__ __forceinline__ float plane_p(const PlaneParams& m, const float* const* P, int c, int i, int j, int k)
{
    const int bi = i - m.bb_lo[0], bj = j - m.bb_lo[1], bk = k - m.bb_lo[2];
    if (!m.has_metal || bi < 0 || bj < 0 || bk < 0 || bi >= m.bb_n[0] || bj >= m.bb_n[1] || bk >= m.bb_n[2])
        return 0.f;
    return __ldg(P[c] + ((size_t)bk * m.bb_n[1] + bj) * m.bb_n[0] + bi);
}

// One sample of the plane maps at time index n (read from the device step
// counter, so that a replayed graph samples the right time): E^n at the
// plane's E-sites and div P_f^n (backward differences, C/m^3) at its nodes,
// added with exp(+i w n dt) K dt.  The block stages the nf phases (FP64).
__global__ void __launch_bounds__(256) k_plane_dft(const PlaneParams m, const float* E0, const float* E1,
                                                   const float* E2, const float* P0, const float* P1, const float* P2,
                                                   const long long* step)
{
    __shared__ double2 ph[NLF_PLANE_MAX_NF_DEV];
    if (threadIdx.x < m.nf) {
        double s, c;
        sincos(m.omega[threadIdx.x] * (double)(*step) * m.dt, &s, &c);
        ph[threadIdx.x] = make_double2(c * m.scale, s * m.scale);
    }
    __syncthreads();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long np = (long long)m.n1 * m.n2;
    if (t >= np) return;
    const int u = (int)(t / m.n2), v = (int)(t - (long long)u * m.n2);
    int idx[3];
    const int slow = m.axis == 2 ? 1 : 2, fast = m.axis == 0 ? 1 : 0;
    idx[m.axis] = m.index;
    idx[slow] = u;
    idx[fast] = v;
    const int i = idx[0], j = idx[1], k = idx[2];
    const size_t q = ((size_t)k * m.ny + j) * m.px + i;
    const float* P[3] = {P0, P1, P2};
    float val[4];
    val[0] = __ldg(E0 + q);
    val[1] = __ldg(E1 + q);
    val[2] = __ldg(E2 + q);
    val[3] = 0.f;
    if (m.has_metal) {
        const float d = (plane_p(m, P, 0, i, j, k) - plane_p(m, P, 0, i - 1, j, k)) +
                        (plane_p(m, P, 1, i, j, k) - plane_p(m, P, 1, i, j - 1, k)) +
                        (plane_p(m, P, 2, i, j, k) - plane_p(m, P, 2, i, j, k - 1));
        val[3] = (float)(d * m.eps0_dx);
    }
    for (int f = 0; f < m.nf; ++f) {
        const double2 p = ph[f];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            double2* a = m.acc + ((size_t)w * m.nf + f) * np + t;
            double2 x = *a;
            x.x += (double)val[w] * p.x;
            x.y += (double)val[w] * p.y;
            *a = x;
        }
    }
}

void launch_plane_dft(const PlaneParams& m, const float* const* E, const float* const* P, const long long* step,
                      cudaStream_t st)
{
    const long long np = (long long)m.n1 * m.n2;
    k_plane_dft<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(m, E[0], E[1], E[2], P ? P[0] : nullptr,
                                                              P ? P[1] : nullptr, P ? P[2] : nullptr, step);
}

// Copy one field component out of the padded layout (rows of px floats, nx
// used) into a dense [nz][ny][nx] array, scaled.
__global__ void k_field_out(const float* __restrict__ src, float* __restrict__ dst, int nx, int px, long long n,
                            float scale)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const long long row = q / nx;
    const int i = (int)(q - row * nx);
    dst[q] = src[row * px + i] * scale;
}

void launch_field_out(const float* src, float* dst, int nx, int px, long long rows, float scale, cudaStream_t st)
{
    const long long n = rows * nx;
    k_field_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, nx, px, n, scale);
}

// Free-electron charge density div P_f (C/m^3) at every node (i, j, k) of the
// grid (Eq. Nsol: n - n0 = div P_f / e), dense [nz][ny][nx]: P_a lives at the
// E_a site half a cell up the a axis, so the node takes the backward
// difference P_a(node) - P_a(node - e_a) along each axis over dx.  P_f is
// stored as P/eps0 inside the metal box and is zero outside it.
__global__ void k_density_out(const DensityParams d, float* __restrict__ dst)
{
    const long long n = (long long)d.nx * d.ny * d.nz;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const long long row = q / d.nx;
    const int i = (int)(q - row * d.nx), j = (int)(row % d.ny), k = (int)(row / d.ny);
    auto P = [&](int c, int ii, int jj, int kk) -> float {
        const int bi = ii - d.bb_lo[0], bj = jj - d.bb_lo[1], bk = kk - d.bb_lo[2];
        if (bi < 0 || bj < 0 || bk < 0 || bi >= d.bb_n[0] || bj >= d.bb_n[1] || bk >= d.bb_n[2]) return 0.f;
        return __ldg(d.P[c] + ((long long)bk * d.bb_n[1] + bj) * d.bb_n[0] + bi);
    };
    const float v = (P(0, i, j, k) - P(0, i - 1, j, k)) + (P(1, i, j, k) - P(1, i, j - 1, k)) +
                    (P(2, i, j, k) - P(2, i, j, k - 1));
    dst[q] = (float)((double)v * d.eps0_dx);
}

void launch_density_out(const DensityParams& d, float* dst, cudaStream_t st)
{
    const long long n = (long long)d.nx * d.ny * d.nz;
    k_density_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, dst);
}

}  // namespace nlf
