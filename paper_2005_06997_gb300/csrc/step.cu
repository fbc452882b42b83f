// step.cu -- one fused time step of the nonlocal hydrodynamic FDTD scheme.
//
// One launch advances (H^{n-1/2}, E^n, P^n) to (H^{n+1/2}, E^{n+1}, P^{n+1})
// in the order of Sec. III: f1 (H), f2 (E), f3 (P_CP), f4 (P_f).  Every
// thread owns one cell (i,j,k): it writes H^{n+1/2} and E^{n+1} of that cell.
// The E update needs H^{n+1/2} of the cells at i-1, j-1, k-1, which another
// thread owns; instead of a grid-wide barrier the thread recomputes those H
// values from generation n (E, H and psi_H are double buffered), so the whole
// step is one launch and each field is read once from HBM per step (the
// neighbour reads hit L1/L2).
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
// GD^n = grad(div P_f^n) is evaluated as the difference of node divergences,
// which equals Eq. GradDiv term by term.
#include <cuda_runtime.h>

#include "nlf_internal.h"

namespace nlf {

__device__ __forceinline__ float ldg(const float* p, long long i) { return __ldg(p + i); }

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
__device__ __forceinline__ int slab_local(const StepParams& p, int a, int v, int n)
{
    if (!p.cpml[a]) return -1;
    if (v < p.pml) return v;
    if (v >= n - p.pml) return v - (n - p.pml) + p.pml;
    return -1;
}

__device__ __forceinline__ long long slab_index(const StepParams& p, int a, int l, int i, int j, int k)
{
    int two = 2 * p.pml;
    if (a == 0) return ((long long)k * p.ny + j) * two + l;
    if (a == 1) return ((long long)k * two + l) * p.nx + i;
    return ((long long)l * p.ny + j) * p.nx + i;
}

// H_C^{n+1/2} at cell (i,j,k); if own, also store it and its psi.
// (curl E)_C = dE_{A2}/dx_{A1} - dE_{A1}/dx_{A2}, (C, A1, A2) cyclic.
template <int C>
__device__ __forceinline__ float h_next(const StepParams& p, int i, int j, int k, bool own)
{
    constexpr int A1 = (C + 1) % 3, A2 = (C + 2) % 3;
    const int n3[3] = {p.nx, p.ny, p.nz};
    const int ix[3] = {i, j, k};
    const long long st[3] = {1, (long long)p.nx, (long long)p.nx * p.ny};
    const long long q = (long long)k * st[2] + (long long)j * st[1] + i;
    float a_here = ldg(p.E0[A2], q);
    float a_next = (ix[A1] + 1 < n3[A1]) ? ldg(p.E0[A2], q + st[A1]) : 0.f;
    float b_here = ldg(p.E0[A1], q);
    float b_next = (ix[A2] + 1 < n3[A2]) ? ldg(p.E0[A1], q + st[A2]) : 0.f;
    if (p.tfsf && (A1 == 0 || A2 == 0)) {
        // only E_x carries an incident field; convert it across the TF/SF surface
        const int self = tf_point(p, 2 * i + hoff(C, 0), 2 * j + hoff(C, 1), 2 * k + hoff(C, 2));
        if (A2 == 0) {   // a_* are E_x at idx and idx + e_A1
            int t0 = tf_point(p, 2 * i + 1, 2 * j, 2 * k);
            int t1 = tf_point(p, 2 * i + 1 + 2 * (A1 == 0), 2 * j + 2 * (A1 == 1), 2 * k + 2 * (A1 == 2));
            if (self != t0) a_here += (self - t0) * e_inc(p, k);
            if (self != t1) a_next += (self - t1) * e_inc(p, k + (A1 == 2));
        } else {         // b_* are E_x at idx and idx + e_A2
            int t0 = tf_point(p, 2 * i + 1, 2 * j, 2 * k);
            int t1 = tf_point(p, 2 * i + 1 + 2 * (A2 == 0), 2 * j + 2 * (A2 == 1), 2 * k + 2 * (A2 == 2));
            if (self != t0) b_here += (self - t0) * e_inc(p, k);
            if (self != t1) b_next += (self - t1) * e_inc(p, k + (A2 == 2));
        }
    }
    float t1 = a_next - a_here;
    float t2 = b_next - b_here;
    int l1 = slab_local(p, A1, ix[A1], n3[A1]);
    if (l1 >= 0) {
        long long s = slab_index(p, A1, l1, i, j, k);
        float psi = __ldg(p.bH[A1] + ix[A1]) * __ldg(p.psiH0[A1][1] + s) + __ldg(p.cH[A1] + ix[A1]) * t1;
        if (own) p.psiH1[A1][1][s] = psi;
        t1 += psi;
    }
    int l2 = slab_local(p, A2, ix[A2], n3[A2]);
    if (l2 >= 0) {
        long long s = slab_index(p, A2, l2, i, j, k);
        float psi = __ldg(p.bH[A2] + ix[A2]) * __ldg(p.psiH0[A2][0] + s) + __ldg(p.cH[A2] + ix[A2]) * t2;
        if (own) p.psiH1[A2][0][s] = psi;
        t2 += psi;
    }
    float h = ldg(p.H0[C], q) - p.S * (t1 - t2);
    if (own) p.H1[C][q] = h;
    return h;
}

// Node divergence of P_f^n (difference units) at bbox-local linear index b.
__device__ __forceinline__ float node_div(const StepParams& p, long long b, long long sy, long long sz)
{
    return (ldg(p.P0[0], b) - ldg(p.P0[0], b - 1)) + (ldg(p.P0[1], b) - ldg(p.P0[1], b - sy)) +
           (ldg(p.P0[2], b) - ldg(p.P0[2], b - sz));
}

// E_C^{n+1} at cell (i,j,k) from H^{n+1/2}: hA2 = H_{A2}(idx), hA2m = H_{A2}(idx - e_A1),
// hA1 = H_{A1}(idx), hA1m = H_{A1}(idx - e_A2).
template <int C>
__device__ __forceinline__ void e_next(const StepParams& p, int i, int j, int k, float hA2, float hA2m, float hA1,
                                       float hA1m, float& d_here, bool& d_valid)
{
    constexpr int A1 = (C + 1) % 3, A2 = (C + 2) % 3;
    const int n3[3] = {p.nx, p.ny, p.nz};
    const int ix[3] = {i, j, k};
    const long long q = ((long long)k * p.ny + j) * p.nx + i;
    if (p.tfsf && (A1 == 1 || A2 == 1)) {
        // only H_y carries an incident field
        const int self = tf_point(p, 2 * i + eoff(C, 0), 2 * j + eoff(C, 1), 2 * k + eoff(C, 2));
        if (A2 == 1) {   // hA2 = H_y(idx), hA2m = H_y(idx - e_A1)
            int t0 = tf_point(p, 2 * i + 1, 2 * j, 2 * k + 1);
            int t1 = tf_point(p, 2 * i + 1 - 2 * (A1 == 0), 2 * j - 2 * (A1 == 1), 2 * k + 1 - 2 * (A1 == 2));
            if (self != t0) hA2 += (self - t0) * h_inc_next(p, k);
            if (self != t1) hA2m += (self - t1) * h_inc_next(p, k - (A1 == 2));
        } else {         // hA1 = H_y(idx), hA1m = H_y(idx - e_A2)
            int t0 = tf_point(p, 2 * i + 1, 2 * j, 2 * k + 1);
            int t1 = tf_point(p, 2 * i + 1 - 2 * (A2 == 0), 2 * j - 2 * (A2 == 1), 2 * k + 1 - 2 * (A2 == 2));
            if (self != t0) hA1 += (self - t0) * h_inc_next(p, k);
            if (self != t1) hA1m += (self - t1) * h_inc_next(p, k - (A2 == 2));
        }
    }
    float t1 = hA2 - hA2m;
    float t2 = hA1 - hA1m;
    int l1 = slab_local(p, A1, ix[A1], n3[A1]);
    if (l1 >= 0) {
        long long s = slab_index(p, A1, l1, i, j, k);
        float psi = __ldg(p.bE[A1] + ix[A1]) * p.psiE[A1][1][s] + __ldg(p.cE[A1] + ix[A1]) * t1;
        p.psiE[A1][1][s] = psi;
        t1 += psi;
    }
    int l2 = slab_local(p, A2, ix[A2], n3[A2]);
    if (l2 >= 0) {
        long long s = slab_index(p, A2, l2, i, j, k);
        float psi = __ldg(p.bE[A2] + ix[A2]) * p.psiE[A2][0][s] + __ldg(p.cE[A2] + ix[A2]) * t2;
        p.psiE[A2][0][s] = psi;
        t2 += psi;
    }
    const float curl = t1 - t2;
    const float En = ldg(p.E0[C], q);
    int id = 0;
    long long b = 0, sy = 0, sz = 0;
    if (p.has_metal) {
        int bi = i - p.bb_lo[0], bj = j - p.bb_lo[1], bk = k - p.bb_lo[2];
        if (bi >= 0 && bj >= 0 && bk >= 0 && bi < p.bb_n[0] && bj < p.bb_n[1] && bk < p.bb_n[2]) {
            sy = p.bb_n[0];
            sz = (long long)p.bb_n[0] * p.bb_n[1];
            b = (long long)bk * sz + (long long)bj * sy + bi;
            id = p.mat[C][b];
        }
    }
    if (id == 0) {
        p.E1[C][q] = En + p.Sb * curl;
        return;
    }
    const MatCoef& m = p.coef[id];
    float gd = 0.f, af = 0.f;
    if (m.free_e) {
        if (!d_valid) {
            d_here = node_div(p, b, sy, sz);
            d_valid = true;
        }
        const long long stb = C == 0 ? 1 : (C == 1 ? sy : sz);
        gd = node_div(p, b + stb, sy, sz) - d_here;
        af = p.auxf[C][b];
    }
    float ac[NLF_MAX_POLES];
    float acs = 0.f;
#pragma unroll
    for (int pp = 0; pp < NLF_MAX_POLES; ++pp) {
        ac[pp] = pp < m.npoles ? p.auxcp[pp][C][b] : 0.f;
        acs += ac[pp];
    }
    const float delta = (p.S * curl - af - acs - m.G * gd - m.cE * En) * m.inv_den;
    p.E1[C][q] = En + delta;
    if (m.free_e) {
        const float dP = af + m.D3 * (3.f * En + delta) + m.G * gd;
        p.P1[C][b] = ldg(p.P0[C], b) + dP;
        float a_new = -m.D2 * dP + m.D3 * En;
        if (m.gnor) {
            const float g1 = p.gdp[C][b];
            a_new += m.DG2 * (g1 - 4.f * gd);
            p.gdp[C][b] = gd;
        }
        p.auxf[C][b] = a_new;
    }
#pragma unroll
    for (int pp = 0; pp < NLF_MAX_POLES; ++pp) {
        if (pp >= m.npoles) break;
        const float dPc = ac[pp] + m.C3[pp] * (En + delta) + m.C4[pp] * En;
        const float pc = p.pcp[pp][C][b] + dPc;
        p.pcp[pp][C][b] = pc;
        p.auxcp[pp][C][b] = -m.kap[pp] * pc - m.C2[pp] * dPc + m.C5[pp] * En;
    }
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

__global__ void __launch_bounds__(256) k_step(const StepParams p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i < p.nx && j < p.ny && k < p.nz) {
        // own H^{n+1/2}
        const float hx = h_next<0>(p, i, j, k, true);
        const float hy = h_next<1>(p, i, j, k, true);
        const float hz = h_next<2>(p, i, j, k, true);
        float d_here = 0.f;
        bool d_valid = false;
        // E_x: needs H_z(j-1), H_y(k-1); updated for j >= 1, k >= 1
        if (j >= 1 && k >= 1) {
            e_next<0>(p, i, j, k, hz, h_next<2>(p, i, j - 1, k, false), hy, h_next<1>(p, i, j, k - 1, false),
                      d_here, d_valid);
        } else {
            p.E1[0][((long long)k * p.ny + j) * p.nx + i] = 0.f;
        }
        // E_y: needs H_x(k-1), H_z(i-1); updated for i >= 1, k >= 1
        if (i >= 1 && k >= 1) {
            e_next<1>(p, i, j, k, hx, h_next<0>(p, i, j, k - 1, false), hz, h_next<2>(p, i - 1, j, k, false),
                      d_here, d_valid);
        } else {
            p.E1[1][((long long)k * p.ny + j) * p.nx + i] = 0.f;
        }
        // E_z: needs H_y(i-1), H_x(j-1); updated for i >= 1, j >= 1
        if (i >= 1 && j >= 1) {
            e_next<2>(p, i, j, k, hy, h_next<1>(p, i - 1, j, k, false), hx, h_next<0>(p, i, j - 1, k, false),
                      d_here, d_valid);
        } else {
            p.E1[2][((long long)k * p.ny + j) * p.nx + i] = 0.f;
        }
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
        const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
        const int nt = blockDim.x * blockDim.y * blockDim.z;
        if (p.tfsf) inc_step(p, tid, nt);
        if (tid == 0) *p.step1 = *p.step0 + 1;
    }
}

void launch_step(const StepParams& p, cudaStream_t st)
{
    dim3 blk(32, 4, 2);
    dim3 grd((p.nx + 31) / 32, (p.ny + 3) / 4, (p.nz + 1) / 2);
    k_step<<<grd, blk, 0, st>>>(p);
}

}  // namespace nlf
