// capi.cu -- host side of the nlf_* C ABI (include/nlfdtd.h).
//
// A context owns one state buffer on the device (library-allocated or bound
// by the caller) that holds every array of the method; nothing else lives on
// the device.  Time steps are launched eagerly or replayed from a CUDA graph
// that holds a whole DFT period (K * B steps): the step kernel, the sample
// gathers and the accumulation.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <unordered_set>
#include <string>
#include <thread>
#include <vector>

#include "../../include/nlfdtd.h"
#include "nlf_internal.h"

namespace nlf {
void launch_step(const StepParams& p, cudaStream_t st);
void launch_step_pml(const StepParams& p, cudaStream_t st);
void launch_step_metal(const StepParams& p, cudaStream_t st);
bool step_has_pml(const StepParams& p);
long long tfsf_items(const StepParams& p);
void launch_tfsf(const StepParams& p, cudaStream_t st);
void launch_metal(const StepParams& p, long long n_sites, cudaStream_t st);
void launch_post(const StepParams& p, long long n_sites, cudaStream_t st);
void launch_site_list(const uint8_t* mat, long long nb, uint32_t* sites, uint32_t* site_q, const SiteGeom& g,
                      unsigned long long* count, cudaStream_t st);
void launch_voxelise(const VoxParams& v, cudaStream_t st);
void launch_dft_gather(const DftParams& d, const float* E, const float* H, const float* e_inc, const float* h_inc,
                       int slot, const long long* step, int* err, cudaStream_t st);
void launch_dft_flush(const DftParams& d, int count, cudaStream_t st);
void launch_flux(const double2* accE, const double2* accH, const double* coef, long long n_abs, long long nrec,
                 int nf, double2* partial, int G, double dA, double* out, cudaStream_t st);
void launch_plane_dft(const PlaneParams& m, const float* const* E, const float* const* P, const long long* step,
                      cudaStream_t st);
void launch_field_out(const float* src, float* dst, int nx, int px, long long rows, float scale, cudaStream_t st);
void launch_watch(const float* E, long long nfloats, int* err, cudaStream_t st);
void launch_density_out(const DensityParams& d, float* dst, cudaStream_t st);
void launch_step_batch(const BatchStep& a, long long total_items, cudaStream_t st);
void launch_step_batch_pml(const BatchStep& a, long long total_items, cudaStream_t st);
void launch_post_batch(const BatchStep& a, long long total_sites, long long total_tf, cudaStream_t st);
void launch_gather_batch(const BatchDft& a, long long total_records, int slot, cudaStream_t st);
void launch_flush_batch(const BatchDft& a, long long total_phase, long long total_chunks, int max_nf, int B,
                        int count, cudaStream_t st);
int step_kz(const StepParams& p);
int step_chunks(const StepParams& p, int kz);
}  // namespace nlf

namespace {

constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.25663706212e-6;

struct Header {            // first bytes of the state buffer
    long long step[2];     // step counters, ping-pong by parity
    int err;               // bit 0: non-finite value; bit 2: a TMA wait gave up; bit 3: bounds (checked build)
    int cnt;               // pending DFT samples (host mirror, written before a save)
    long long n;           // time index (host mirror, written before a save)
    nlf::BoundsRecord chk; // first out-of-bounds access of the bounds-checked build
    long long ctx_id;      // the id of the context that owns this state
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct nlf_ctx {
    long long id = 0;               // unique per context of the process (also in the state's header)
    nlf_grid g{};
    double dt = 0, c0 = 0, eta0 = 0;
    long long ncell = 0;
    int px = 0;                     // row pitch of the field arrays: nx rounded up to 8 (32-byte rows)
    CUtensorMap tmaps[4];           // E gen 0, E gen 1, H gen 0, H gen 1 (host copy of the device tables)
    size_t off_tmap = 0;
    long long nfield = 0;           // floats per field component: px ny nz
    std::vector<nlf_material> mats;
    std::vector<nlf_shape> shapes;
    std::vector<uint8_t> map;      // full [3][nz][ny][nx] map if given
    bool use_map = false;
    bool have_src = false;
    nlf_source src{};
    bool have_mon = false;
    bool have_plane = false;
    nlf_plane_monitor plane{};
    std::vector<double> plane_omega;
    size_t off_pacc = 0, off_pomega = 0;
    nlf::PlaneParams pp{};
    nlf_monitors mon{};
    std::vector<double> omega;
    std::string err;

    // derived geometry
    bool has_metal = false;
    int bb_lo[3] = {0, 0, 0}, bb_n[3] = {0, 0, 0};
    long long nbb = 0;
    long long n_msites = 0;     // E-sites of the metal box that hold a material
    // material update fused into the EM z-march (metal tiles): sites of CPML
    // tiles stay on the site-list kernel (n_psites of them, n_ppl with free
    // electrons); fuse is off with more than one critical-point pole
    bool fuse = false;
    int tiles_x = 0, tiles_y = 0;
    long long n_psites = 0, n_ppl = 0;
    int inc_off = 0, inc_len = 0, inc_node = 0;
    int K = 1, B = 16, U = 128;
    long long nrec = 0, n_abs = 0;
    int G = 1;
    int max_poles = 0;
    bool any_gnor = false;
    long long pml_slab[3] = {0, 0, 0};
    bool planned = false;

    // state
    size_t bytes = 0;
    char* base = nullptr;
    bool owned = false;
    bool ready = false;
    size_t off_hdr = 0, off_E[2] = {0, 0}, off_H[2] = {0, 0};
    size_t off_psiE[3] = {0, 0, 0}, off_psiH[2][3] = {{0, 0, 0}, {0, 0, 0}};
    size_t off_prof[3] = {0, 0, 0};
    size_t off_inc = 0;
    size_t off_sites = 0, off_siteq = 0, off_psites = 0, off_psiteq = 0, off_tilekr = 0;
    size_t off_mat = 0, off_P[2] = {0, 0}, off_auxf = 0, off_gdp = 0, off_pcp = 0, off_auxcp = 0, off_coef = 0,
           off_free = 0, off_counts = 0;
    size_t off_rec = 0, off_dcoef = 0, off_omega = 0, off_samples = 0, off_sstep = 0, off_phase = 0, off_acc = 0,
           off_partial = 0, off_out = 0;

    nlf::StepParams sp[2];
    nlf::DftParams dp{};
    cudaStream_t stream = nullptr;      // stream of the last run
    cudaEvent_t done = nullptr;
    cudaStream_t cap = nullptr;         // private stream for graph capture
    cudaStream_t aux = nullptr;         // second stream of the step: the CPML tiles
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaStream_t aux2 = nullptr;        // third stream of the step: the metal tiles
    cudaEvent_t join2 = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long gnodes = 0;
    long long n = 0;                    // time index
    int cnt = 0;                        // pending DFT samples
    long long launches = 0;
    long long h2d = 0, d2h = 0;         // bytes moved between host and device
    nlf_info info{};
};

namespace {

int fail(nlf_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(c, NLF_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
T* at(nlf_ctx* c, size_t off) { return reinterpret_cast<T*>(c->base + off); }

// ---------------------------------------------------------------- geometry

// Conservative cell range of E-sites that may lie in shape s (inclusive).
void shape_cells(const nlf_shape& s, int lo[3], int hi[3])
{
    for (int a = 0; a < 3; ++a) {
        long long r = 0;
        if (s.kind == NLF_SHAPE_SPHERE) r = s.radius;
        if (s.kind == NLF_SHAPE_BOX) r = s.half[a];
        if (s.kind == NLF_SHAPE_CUBE_TIPS)
            r = std::max<long long>((long long)s.side / 2 + s.tip_height, (long long)s.tip_center + s.tip_radius);
        // E-sites sit at half-cell coordinate 2 i or 2 i + 1: the first index with
        // 2 i + 1 >= p0 and the last with 2 i <= p1
        long long p0 = s.center[a] - r, p1 = s.center[a] + r;
        lo[a] = (int)std::ceil((p0 - 1) / 2.0);
        hi[a] = (int)std::floor(p1 / 2.0);
    }
}

// Depth-graded CPML coefficients: sigma = sigma_max rho^3, sigma_max =
// 0.8 (m+1) / (eta0 dx sqrt(eps_b)), alpha = 0.05 S/m (1 - rho), kappa = 1,
// b = exp(-(sigma + alpha) dt / eps0), c = sigma (b - 1) / (sigma + alpha).
void cpml_bc(const nlf_ctx* c, double rho, float* b, float* cc)
{
    const double m = 3.0;
    const double smax = 0.8 * (m + 1.0) / (c->eta0 * c->g.dx * std::sqrt(c->g.eps_background));
    const double sig = smax * std::pow(rho, m);
    const double alpha = rho > 0.0 ? 0.05 * (1.0 - rho) : 0.0;
    const double bb = std::exp(-(sig + alpha) * c->dt / kEps0);
    *b = (float)bb;
    *cc = (float)((sig + alpha) > 0.0 ? sig * (bb - 1.0) / (sig + alpha) : 0.0);
}

double axis_depth(double x, int n, int L)
{
    double r = 0.0;
    if (x < L) r = (L - x) / L;
    else if (x > n - L) r = (x - (n - L)) / L;
    return std::min(1.0, std::max(0.0, r));
}

// FP64 coefficients of Sec. III (Eqs. d1-dd, GNOR D_G1, D_G2, critical points
// C_1p..C_p with the sin(phi) terms of C3p/C5p over dt Cp), normalised
// (P/eps0, grad-div in difference units) and rounded to FP32.
nlf::MatCoef make_coef(const nlf_ctx* c, const nlf_material& m)
{
    nlf::MatCoef k{};
    const double dt = c->dt, dx2 = c->g.dx * c->g.dx;
    double den = m.eps_inf, cE = 0.0;
    if (m.wp > 0.0) {
        const double Dd = m.gamma / (2.0 * dt) + 1.0 / (dt * dt);
        const double g2 = (m.gamma / dt) / Dd;                          // 1 + D2
        const double D3 = m.wp * m.wp / (4.0 * Dd);                    // D3 / eps0
        const double eta = m.beta * m.beta + m.diff * m.gamma;
        const double DG1 = eta / Dd, DG2 = m.diff / (2.0 * dt * Dd);
        k.free_e = 1;
        k.gnor = m.diff > 0.0;
        k.g2 = (float)g2;
        k.D3 = (float)D3;
        k.DG2 = (float)(DG2 / dx2);
        k.G = (float)((DG1 + 3.0 * DG2) / dx2);
        den += D3;
        cE += 3.0 * D3;
    }
    k.npoles = m.n_poles;
    for (int p = 0; p < m.n_poles; ++p) {
        const double A = m.A[p], Om = m.Omega[p], Ga = m.Gamma[p], ph = m.phi[p];
        const double W2 = Om * Om + Ga * Ga;
        const double Cp = Ga / dt + 1.0 / (dt * dt) + W2 / 4.0;
        const double c2g = (2.0 * Ga / dt) / Cp;                        // 1 + C2
        const double C4 = A * Om * (Om * std::cos(ph) - Ga * std::sin(ph)) / Cp;
        const double C3 = C4 / 2.0 - A * Om * std::sin(ph) / (dt * Cp);
        const double C5 = C4 / 2.0 + A * Om * std::sin(ph) / (dt * Cp);
        k.c2g[p] = (float)c2g;
        k.C3[p] = (float)C3;
        k.C4[p] = (float)C4;
        k.C5[p] = (float)C5;
        k.kap[p] = (float)(W2 / Cp);
        den += C3;
        cE += C3 + C4;
    }
    k.inv_den = (float)(1.0 / den);
    k.cE = (float)cE;
    return k;
}

// Flux-face records of one box, in the order documented in nlfdtd.h.
void box_records(const nlf_ctx* c, const int lo[3], const int hi[3], std::vector<uint32_t>& re,
                 std::vector<uint32_t>& rh, std::vector<uint32_t>& rs, std::vector<double>& co)
{
    const long long st[3] = {1, c->px, (long long)c->px * c->g.ny};
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, cc = (a + 2) % 3;
        const int slow = std::max(b, cc), fast = std::min(b, cc);
        for (int side = 0; side < 2; ++side) {
            const int p = side == 0 ? lo[a] : hi[a];
            const double outward = side == 0 ? -1.0 : 1.0;
            for (int term = 0; term < 2; ++term) {
                const int ec = term == 0 ? b : cc;       // tangential E component
                const int hc = term == 0 ? cc : b;       // paired H component
                const int other = ec == b ? cc : b;      // in-plane axis with node positions
                const double tsign = term == 0 ? 1.0 : -1.0;
                const int hs = ec == slow ? hi[slow] - 1 : hi[slow];
                const int hf = ec == fast ? hi[fast] - 1 : hi[fast];
                for (int ts = lo[slow]; ts <= hs; ++ts)
                    for (int tf = lo[fast]; tf <= hf; ++tf) {
                        int idx[3];
                        idx[a] = p;
                        idx[slow] = ts;
                        idx[fast] = tf;
                        const double w = (idx[other] == lo[other] || idx[other] == hi[other]) ? 0.5 : 1.0;
                        const long long cell = idx[0] * st[0] + idx[1] * st[1] + idx[2] * st[2];
                        re.push_back((uint32_t)(ec * c->nfield + cell));
                        rh.push_back((uint32_t)(hc * c->nfield + cell - st[a]));
                        rs.push_back((uint32_t)st[a]);
                        co.push_back(outward * tsign * w * 0.5);
                    }
            }
        }
    }
}

int check_boxes(nlf_ctx* c)
{
    const nlf_source& s = c->src;
    const int n3[3] = {c->g.nx, c->g.ny, c->g.nz};
    for (int a = 0; a < 3; ++a) {
        int lo_lim = c->g.boundary[a] == NLF_BC_CPML ? c->g.pml_cells + 1 : 1;
        int hi_lim = c->g.boundary[a] == NLF_BC_CPML ? n3[a] - c->g.pml_cells - 1 : n3[a] - 1;
        if (s.tf_lo[a] < lo_lim || s.tf_hi[a] > hi_lim || s.tf_hi[a] - s.tf_lo[a] < 2)
            return fail(c, NLF_E_GEOMETRY, "TF box axis %d [%d,%d] must lie in [%d,%d]", a, s.tf_lo[a], s.tf_hi[a],
                        lo_lim, hi_lim);
        if (c->has_metal) {
            int mlo = c->bb_lo[a] + 2, mhi = c->bb_lo[a] + c->bb_n[a] - 3;
            if (mlo < s.tf_lo[a] + 2 || mhi > s.tf_hi[a] - 2)
                return fail(c, NLF_E_GEOMETRY, "metal on axis %d (cells %d..%d) closer than 2 cells to the TF surface",
                            a, mlo, mhi);
        }
        if (c->have_mon) {
            const nlf_monitors& m = c->mon;
            if (m.abs_lo[a] < s.tf_lo[a] + 1 || m.abs_hi[a] > s.tf_hi[a] - 1 || m.abs_hi[a] <= m.abs_lo[a])
                return fail(c, NLF_E_GEOMETRY, "absorption box axis %d must lie one cell inside the TF box", a);
            if (c->has_metal && (m.abs_lo[a] > c->bb_lo[a] + 2 || m.abs_hi[a] < c->bb_lo[a] + c->bb_n[a] - 2))
                return fail(c, NLF_E_GEOMETRY, "absorption box axis %d does not enclose the metal", a);
            if (m.sca_lo[a] > s.tf_lo[a] - 1 || m.sca_hi[a] < s.tf_hi[a] + 1 || m.sca_lo[a] < lo_lim ||
                m.sca_hi[a] > hi_lim)
                return fail(c, NLF_E_GEOMETRY, "scattering box axis %d must lie between the TF box and the CPML", a);
        }
    }
    return NLF_OK;
}

// Decide the metal bounding box, DFT layout and the state buffer layout.
int plan(nlf_ctx* c)
{
    if (c->planned) return NLF_OK;
    const int n3[3] = {c->g.nx, c->g.ny, c->g.nz};
    // metal bounding box
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
    bool any = false;
    if (c->use_map) {
        for (int cc = 0; cc < 3; ++cc)
            for (int k = 0; k < n3[2]; ++k)
                for (int j = 0; j < n3[1]; ++j)
                    for (int i = 0; i < n3[0]; ++i) {
                        const uint8_t id = c->map[(size_t)cc * c->ncell + ((size_t)k * n3[1] + j) * n3[0] + i];
                        if (!id) continue;
                        if (id > c->mats.size())
                            return fail(c, NLF_E_ARG, "material map id %d exceeds the %zu materials", id,
                                        c->mats.size());
                        any = true;
                        const int v[3] = {i, j, k};
                        for (int a = 0; a < 3; ++a) {
                            lo[a] = std::min(lo[a], v[a]);
                            hi[a] = std::max(hi[a], v[a]);
                        }
                    }
    } else {
        for (const nlf_shape& s : c->shapes) {
            if (s.material < 1 || s.material > (int)c->mats.size())
                return fail(c, NLF_E_ARG, "shape material %d out of range", s.material);
            int l[3], h[3];
            shape_cells(s, l, h);
            any = true;
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], l[a]);
                hi[a] = std::max(hi[a], h[a]);
            }
        }
    }
    c->has_metal = any;
    if (any) {
        // the metal box (material extent and two cells around it) must lie in
        // the grid: metal stays two cells clear of the outer walls.  It may
        // reach into a CPML slab, where it follows the local Drude model
        // (Sec. III); with a TF/SF source it must lie inside the TF box
        // (check_boxes), which keeps it out of the CPML.
        for (int a = 0; a < 3; ++a) {
            c->bb_lo[a] = lo[a] - 2;
            c->bb_n[a] = hi[a] - lo[a] + 5;
            if (c->bb_lo[a] < 0 || c->bb_lo[a] + c->bb_n[a] > n3[a])
                return fail(c, NLF_E_GEOMETRY, "metal closer than two cells to the wall on axis %d", a);
        }
        c->nbb = (long long)c->bb_n[0] * c->bb_n[1] * c->bb_n[2];
        if (c->nbb > (long long)NLF_SITE_OFFSET_MASK)
            return fail(c, NLF_E_GEOMETRY, "metal bounding box of %lld cells exceeds 2^29", c->nbb);
    }
    if (c->have_src) {
        int rc = check_boxes(c);
        if (rc) return rc;
        c->inc_off = c->src.tf_lo[2] - 3;
        c->inc_len = (c->src.tf_hi[2] - c->inc_off + 1) + NLF_INC_MARGIN + NLF_INC_PML;
    }
    c->max_poles = 0;
    c->any_gnor = false;
    for (const nlf_material& m : c->mats) {
        c->max_poles = std::max(c->max_poles, m.n_poles);
        if (m.wp > 0.0 && m.diff > 0.0) c->any_gnor = true;
    }
    if (c->have_mon) {
        c->K = c->mon.decimate_k;
        // the accumulation kernel is instantiated for 8, 16 and 32 buffered samples
        const int bb = c->mon.block_b > 0 ? c->mon.block_b : 32;
        c->B = bb <= 8 ? 8 : (bb <= 16 ? 16 : 32);
        std::vector<uint32_t> re, rh, rs;
        std::vector<double> co;
        box_records(c, c->mon.abs_lo, c->mon.abs_hi, re, rh, rs, co);
        c->n_abs = (long long)re.size();
        box_records(c, c->mon.sca_lo, c->mon.sca_hi, re, rh, rs, co);
        c->nrec = (long long)re.size();
        c->inc_node = (c->mon.abs_lo[2] + c->mon.abs_hi[2]) / 2 - c->inc_off;
        c->G = (int)std::min<long long>(608, std::max<long long>(1, c->nrec / 64));
        long long kb = (long long)c->K * c->B;
        c->U = (int)(kb % 2 == 0 ? kb : 2 * kb);
    } else {
        c->U = 128;
    }
    // a captured period must hold a whole number of plane samples
    if (c->have_plane && !c->have_mon) {
        const long long kp = 16LL * c->plane.decimate_k;
        c->U = (int)(kp % 2 == 0 ? kp : 2 * kp);
    }
    // layout
    size_t o = 0;
    auto take = [&](size_t nbytes) {
        size_t r = o;
        o = align_up(o + nbytes, 256);
        return r;
    };
    const size_t f3 = 3 * (size_t)c->nfield * sizeof(float);
    c->off_hdr = take(sizeof(Header));
    c->off_tmap = take(4 * sizeof(CUtensorMap));
    for (int gI = 0; gI < 2; ++gI) c->off_E[gI] = take(f3);
    for (int gI = 0; gI < 2; ++gI) c->off_H[gI] = take(f3);
    for (int a = 0; a < 3; ++a) {
        c->pml_slab[a] = 0;
        if (c->g.boundary[a] != NLF_BC_CPML) continue;
        long long other = c->ncell / n3[a];
        c->pml_slab[a] = 2LL * c->g.pml_cells * other;
        c->off_psiE[a] = take(2 * c->pml_slab[a] * sizeof(float));
        for (int gI = 0; gI < 2; ++gI) c->off_psiH[gI][a] = take(2 * c->pml_slab[a] * sizeof(float));
    }
    for (int a = 0; a < 3; ++a) c->off_prof[a] = take(4 * (size_t)n3[a] * sizeof(float));
    if (c->have_src) c->off_inc = take(10 * (size_t)c->inc_len * sizeof(float));
    c->off_coef = take((NLF_MAX_MAT + 1) * sizeof(nlf::MatCoef));
    c->off_free = take((NLF_MAX_MAT + 1) * sizeof(int));
    c->off_counts = take(8 * sizeof(unsigned long long));
    c->tiles_x = (c->g.nx + NLF_TILE_BX - 1) / NLF_TILE_BX;
    c->tiles_y = (c->g.ny + NLF_TILE_BY - 1) / NLF_TILE_BY;
#ifdef NLF_NO_FUSE
    c->fuse = false;                  // build option: every material site on the site-list kernel
#else
    // fused when the metal box is a quarter of the grid or more (build option
    // NLF_FUSE_FRAC: fused when FRAC x box cells >= grid cells): a smaller
    // particle gives the metal kernel too few tiles to fill the GPU, and the
    // site-list kernel is then faster (224^3 sphere, 10 % of the cells in its
    // box: 0.181 against 0.190 ms per step fused; 512^3 cube, 25 %: 2.10
    // against 1.83); contexts with more than one critical-point pole are not
    // fused
#ifndef NLF_FUSE_FRAC
#define NLF_FUSE_FRAC 4
#endif
    c->fuse = c->has_metal && c->max_poles <= 1 && (long long)NLF_FUSE_FRAC * c->nbb >= c->ncell;
#endif
    if (c->has_metal) {
        const size_t nb = (size_t)c->nbb;
        c->off_mat = take(3 * nb);
        c->off_sites = take(3 * nb * sizeof(uint32_t));
        c->off_siteq = take(3 * nb * sizeof(uint32_t));
        if (c->fuse) {
            c->off_psites = take(3 * nb * sizeof(uint32_t));
            c->off_psiteq = take(3 * nb * sizeof(uint32_t));
            c->off_tilekr = take((size_t)c->tiles_x * c->tiles_y * sizeof(int2));
        }
        c->off_P[0] = take(3 * nb * sizeof(float));
        c->off_P[1] = take(3 * nb * sizeof(float));
        c->off_auxf = take(3 * nb * sizeof(float));
        if (c->any_gnor) c->off_gdp = take(3 * nb * sizeof(float));
        if (c->max_poles > 0) {
            c->off_pcp = take((size_t)c->max_poles * 3 * nb * sizeof(float));
            c->off_auxcp = take((size_t)c->max_poles * 3 * nb * sizeof(float));
        }
    }
    if (c->have_mon) {
        const size_t nr = (size_t)c->nrec, nr1 = nr + 1, nf = (size_t)c->mon.nf;
        c->off_rec = take(3 * nr * sizeof(uint32_t) + 64);
        c->off_dcoef = take(nr * sizeof(double));
        c->off_omega = take(nf * sizeof(double));
        c->off_samples = take(2 * (size_t)c->B * nr1 * sizeof(float));
        c->off_sstep = take((size_t)c->B * sizeof(long long));
        c->off_phase = take((size_t)c->B * nf * sizeof(float4));
        c->off_acc = take(2 * nr1 * nf * sizeof(double2));
        c->off_partial = take((size_t)c->G * nf * sizeof(double2));
        c->off_out = take(4 * nf * sizeof(double));
    }
    if (c->have_plane) {
        const long long n3[3] = {c->g.nx, c->g.ny, c->g.nz};
        const int a = c->plane.axis, slow = a == 2 ? 1 : 2, fast = a == 0 ? 1 : 0;
        c->pp.n1 = (int)n3[slow];
        c->pp.n2 = (int)n3[fast];
        c->off_pomega = take((size_t)c->plane.nf * sizeof(double));
        c->off_pacc = take((size_t)4 * c->plane.nf * c->pp.n1 * c->pp.n2 * sizeof(double2));
    }
    c->bytes = o;
    c->planned = true;
    return NLF_OK;
}

// L2 promotion of the tensor-map loads (build option NLF_TMA_L2_PROMO = 0,
// 64, 128 or 256 bytes).  A tile row of the z march starts 16 bytes before
// a 128-byte line (the box starts at x0 - 4 floats) and spans 160 bytes:
// promoted to 128-byte lines it pulls three lines, to 64-byte granules
// four granules (256 bytes).  Measured on the 512^3 cube (ms per step):
// none 1.944, 64 B 1.841, 128 B 1.943, 256 B 1.958.
#ifndef NLF_TMA_L2_PROMO
#define NLF_TMA_L2_PROMO 64
#endif
constexpr CUtensorMapL2promotion kTmaPromotion =
    NLF_TMA_L2_PROMO == 0 ? CU_TENSOR_MAP_L2_PROMOTION_NONE
    : NLF_TMA_L2_PROMO == 64 ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B
    : NLF_TMA_L2_PROMO == 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
                              : CU_TENSOR_MAP_L2_PROMOTION_L2_128B;

// Tensor maps of the four field arrays for the TMA-fed step kernel: 4D
// [3][nz][ny][px] floats, globally nx x ny x nz x 3 (cells past nx, below 0
// or past the grid read as zero), boxes of NLF_TMA_BOX_X x (EY | HY) x 1 x 3.
int encode_maps(nlf_ctx* c)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!encode) {
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q{};
            cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
                return fail(c, NLF_E_CUDA, "cuTensorMapEncodeTiled not available");
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
    }
    const cuuint64_t dims[4] = {(cuuint64_t)c->g.nx, (cuuint64_t)c->g.ny, (cuuint64_t)c->g.nz, 3};
    const cuuint64_t strides[3] = {(cuuint64_t)c->px * 4, (cuuint64_t)c->px * c->g.ny * 4, (cuuint64_t)c->nfield * 4};
    const cuuint32_t elem[4] = {1, 1, 1, 1};
    for (int m = 0; m < 4; ++m) {
        const bool isE = m < 2;
        const cuuint32_t box[4] = {NLF_TMA_BOX_X, (cuuint32_t)(isE ? NLF_TMA_BOX_EY : NLF_TMA_BOX_HY), 1, 3};
        void* base = c->base + (isE ? c->off_E[m & 1] : c->off_H[m & 1]);
        CUresult r = encode(&c->tmaps[m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, elem,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, kTmaPromotion,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(c, NLF_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    return NLF_OK;
}

void fill_params(nlf_ctx* c)
{
    const int n3[3] = {c->g.nx, c->g.ny, c->g.nz};
    for (int par = 0; par < 2; ++par) {
        nlf::StepParams& p = c->sp[par];
        memset(&p, 0, sizeof p);
        const int r = par, w = 1 - par;
        p.nx = c->g.nx;
        p.px = c->px;
        p.tmE = c->base + c->off_tmap + (size_t)r * sizeof(CUtensorMap);
        p.tmH = c->base + c->off_tmap + (size_t)(2 + r) * sizeof(CUtensorMap);
        static_assert(sizeof(nlf::TensorMapBytes) == sizeof(CUtensorMap), "tensor map size");
        memcpy(&p.mapE, &c->tmaps[r], sizeof(CUtensorMap));
        memcpy(&p.mapH, &c->tmaps[2 + r], sizeof(CUtensorMap));
#ifdef NLF_TMAP_GLOBAL
        p.map_in_params = 0;            // build option: the maps from the state in global memory
#else
        p.map_in_params = 1;
#endif
        p.ny = c->g.ny;
        p.nz = c->g.nz;
        p.S = (float)c->g.courant;
        p.Sb = (float)(c->g.courant / c->g.eps_background);
        for (int k = 0; k < 3; ++k) {
            p.E0[k] = at<float>(c, c->off_E[r]) + k * c->nfield;
            p.H0[k] = at<float>(c, c->off_H[r]) + k * c->nfield;
            p.E1[k] = at<float>(c, c->off_E[w]) + k * c->nfield;
            p.H1[k] = at<float>(c, c->off_H[w]) + k * c->nfield;
        }
        p.pml = c->g.pml_cells;
        for (int a = 0; a < 3; ++a) {
            p.cpml[a] = c->g.boundary[a] == NLF_BC_CPML;
            float* pr = at<float>(c, c->off_prof[a]);
            p.bE[a] = pr;
            p.cE[a] = pr + n3[a];
            p.bH[a] = pr + 2 * n3[a];
            p.cH[a] = pr + 3 * n3[a];
            if (p.cpml[a]) {
                for (int s = 0; s < 2; ++s) {
                    p.psiE[a][s] = at<float>(c, c->off_psiE[a]) + s * c->pml_slab[a];
                    p.psiH0[a][s] = at<float>(c, c->off_psiH[r][a]) + s * c->pml_slab[a];
                    p.psiH1[a][s] = at<float>(c, c->off_psiH[w][a]) + s * c->pml_slab[a];
                }
            }
        }
        p.tfsf = c->have_src;
        if (c->have_src) {
            for (int a = 0; a < 3; ++a) {
                p.tf_lo[a] = c->src.tf_lo[a];
                p.tf_hi[a] = c->src.tf_hi[a];
            }
            p.inc_off = c->inc_off;
            p.inc_len = c->inc_len;
            float* inc = at<float>(c, c->off_inc);
            const int L = c->inc_len;
            // [e0 e1 h0 h1 psie psih be ce bh ch]
            p.e_inc0 = inc + r * L;
            p.e_inc1 = inc + w * L;
            p.h_inc0 = inc + (2 + r) * L;
            p.h_inc1 = inc + (2 + w) * L;
            p.psi_e_inc = inc + 4 * L;
            p.psi_h_inc = inc + 5 * L;
            p.b_e_inc = inc + 6 * L;
            p.c_e_inc = inc + 7 * L;
            p.b_h_inc = inc + 8 * L;
            p.c_h_inc = inc + 9 * L;
            p.waveform = c->src.waveform;
            p.w0 = c->src.w0;
            p.tau = c->src.tau;
            p.t0 = c->src.t0;
            p.amp = c->src.amplitude;
            p.dt = c->dt;
        }
        p.has_metal = c->has_metal;
        p.coef = at<nlf::MatCoef>(c, c->off_coef);
        p.any_gnor = c->any_gnor;
        p.max_poles = c->max_poles;
        if (c->has_metal) {
            const size_t nb = (size_t)c->nbb;
            for (int a = 0; a < 3; ++a) {
                p.bb_lo[a] = c->bb_lo[a];
                p.bb_n[a] = c->bb_n[a];
            }
            p.fuse_metal = c->fuse;
            p.tiles_x = c->tiles_x;
            if (c->fuse) {
                p.tile_kr = at<int2>(c, c->off_tilekr);
                p.psites = at<uint32_t>(c, c->off_psites);
                p.psite_q = at<uint32_t>(c, c->off_psiteq);
            }
            // the site list the post-step kernel walks: the CPML tiles' sites
            // when the z march updates the others, else every material site
            p.sites = at<uint32_t>(c, c->fuse ? c->off_psites : c->off_sites);
            p.site_q = at<uint32_t>(c, c->fuse ? c->off_psiteq : c->off_siteq);
            for (int k = 0; k < 3; ++k) {
                p.mat[k] = at<uint8_t>(c, c->off_mat) + k * nb;
                p.P0[k] = at<float>(c, c->off_P[r]) + k * nb;
                p.P1[k] = at<float>(c, c->off_P[w]) + k * nb;
                p.auxf[k] = at<float>(c, c->off_auxf) + k * nb;
                if (c->any_gnor) p.gdp[k] = at<float>(c, c->off_gdp) + k * nb;
                for (int q = 0; q < c->max_poles; ++q) {
                    p.pcp[q][k] = at<float>(c, c->off_pcp) + ((size_t)q * 3 + k) * nb;
                    p.auxcp[q][k] = at<float>(c, c->off_auxcp) + ((size_t)q * 3 + k) * nb;
                }
            }
        }
        Header* h = at<Header>(c, c->off_hdr);
        p.step0 = &h->step[r];
        p.step1 = &h->step[w];
        p.err = &h->err;
        p.chk = &h->chk;
        p.hdr_id = &h->ctx_id;
        p.ctx_id = c->id;
        p.nfield = c->nfield;
        for (int a = 0; a < 3; ++a) p.psi_n[a] = c->pml_slab[a];
        p.nbb = c->nbb;
        p.ntiles_xy = c->tiles_x * c->tiles_y;
    }
    if (c->have_plane) {
        nlf::PlaneParams& m = c->pp;
        m.axis = c->plane.axis;
        m.index = c->plane.index;
        m.nx = c->g.nx;
        m.ny = c->g.ny;
        m.nz = c->g.nz;
        m.px = c->px;
        m.nf = c->plane.nf;
        m.omega = at<double>(c, c->off_pomega);
        m.dt = c->dt;
        m.scale = c->plane.decimate_k * c->dt;
        m.eps0_dx = kEps0 / c->g.dx;
        m.has_metal = c->has_metal;
        for (int a2 = 0; a2 < 3; ++a2) {
            m.bb_lo[a2] = c->bb_lo[a2];
            m.bb_n[a2] = c->bb_n[a2];
        }
        m.acc = at<double2>(c, c->off_pacc);
    }
    if (c->have_mon) {
        nlf::DftParams& d = c->dp;
        const size_t nr1 = (size_t)c->nrec + 1, nf = (size_t)c->mon.nf;
        d.nrec = c->nrec;
        d.nf = c->mon.nf;
        d.B = c->B;
        uint32_t* rec = at<uint32_t>(c, c->off_rec);
        d.rec_e = rec;
        d.rec_h = rec + c->nrec;
        d.rec_hs = rec + 2 * c->nrec;
        d.sE = at<float>(c, c->off_samples);
        d.sH = d.sE + (size_t)c->B * nr1;
        d.sample_step = at<long long>(c, c->off_sstep);
        d.phase = at<float4>(c, c->off_phase);
        d.accE = at<double2>(c, c->off_acc);
        d.accH = d.accE + nr1 * nf;
        d.omega = at<double>(c, c->off_omega);
        d.dt = c->dt;
        d.inc_node = c->inc_node;
        d.nfield3 = 3 * c->nfield;
        d.err = &at<Header>(c, c->off_hdr)->err;
        d.chk = &at<Header>(c, c->off_hdr)->chk;
        d.hdr_id = &at<Header>(c, c->off_hdr)->ctx_id;
        d.ctx_id = c->id;
    }
}

// Clear the state, upload tables and voxelise.
int initialise(nlf_ctx* c, cudaStream_t st)
{
    const int n3[3] = {c->g.nx, c->g.ny, c->g.nz};
    CK(cudaMemsetAsync(c->base, 0, c->bytes, st));
    std::vector<char> tmp;
    auto put = [&](size_t off, const void* src, size_t nbytes) -> int {
        c->h2d += (long long)nbytes;
        CK(cudaMemcpyAsync(c->base + off, src, nbytes, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));   // host staging buffers are reused
        return NLF_OK;
    };
    int rc;
    if ((rc = put(c->off_hdr + offsetof(Header, ctx_id), &c->id, sizeof c->id))) return rc;
    if ((rc = encode_maps(c))) return rc;
    if ((rc = put(c->off_tmap, c->tmaps, sizeof c->tmaps))) return rc;
    for (int a = 0; a < 3; ++a) {
        std::vector<float> pr(4 * (size_t)n3[a], 0.f);
        for (int v = 0; v < n3[a]; ++v) {
            pr[v] = 1.f;
            pr[2 * n3[a] + v] = 1.f;
            if (c->g.boundary[a] != NLF_BC_CPML) continue;
            cpml_bc(c, axis_depth((double)v, n3[a], c->g.pml_cells), &pr[v], &pr[n3[a] + v]);
            cpml_bc(c, axis_depth(v + 0.5, n3[a], c->g.pml_cells), &pr[2 * n3[a] + v], &pr[3 * n3[a] + v]);
        }
        if ((rc = put(c->off_prof[a], pr.data(), pr.size() * sizeof(float)))) return rc;
    }
    if (c->have_src) {
        const int L = c->inc_len, start = L - NLF_INC_PML;
        std::vector<float> v(10 * (size_t)L, 0.f);
        for (int m = 0; m < L; ++m) {
            double xe = m, xh = m + 0.5;
            double re = xe > start ? std::min(1.0, (xe - start) / NLF_INC_PML) : 0.0;
            double rh = xh > start ? std::min(1.0, (xh - start) / NLF_INC_PML) : 0.0;
            cpml_bc(c, re, &v[6 * (size_t)L + m], &v[7 * (size_t)L + m]);
            cpml_bc(c, rh, &v[8 * (size_t)L + m], &v[9 * (size_t)L + m]);
        }
        if ((rc = put(c->off_inc, v.data(), v.size() * sizeof(float)))) return rc;
    }
    std::vector<nlf::MatCoef> coef(NLF_MAX_MAT + 1);
    std::vector<int> fe(NLF_MAX_MAT + 1, 0);
    for (size_t m = 0; m < c->mats.size(); ++m) {
        coef[m + 1] = make_coef(c, c->mats[m]);
        fe[m + 1] = coef[m + 1].free_e;
    }
    if ((rc = put(c->off_coef, coef.data(), coef.size() * sizeof(nlf::MatCoef)))) return rc;
    if ((rc = put(c->off_free, fe.data(), fe.size() * sizeof(int)))) return rc;
    if (c->has_metal) {
        if (c->use_map) {
            const size_t nb = (size_t)c->nbb;
            std::vector<uint8_t> sub(3 * nb);
            for (int cc = 0; cc < 3; ++cc)
                for (int bk = 0; bk < c->bb_n[2]; ++bk)
                    for (int bj = 0; bj < c->bb_n[1]; ++bj)
                        for (int bi = 0; bi < c->bb_n[0]; ++bi) {
                            size_t src = (size_t)cc * c->ncell +
                                         ((size_t)(bk + c->bb_lo[2]) * n3[1] + (bj + c->bb_lo[1])) * n3[0] +
                                         (bi + c->bb_lo[0]);
                            sub[cc * nb + ((size_t)bk * c->bb_n[1] + bj) * c->bb_n[0] + bi] = c->map[src];
                        }
            if ((rc = put(c->off_mat, sub.data(), sub.size()))) return rc;
            unsigned long long cnts[3] = {0, 0, 0};
            for (int cc = 0; cc < 3; ++cc)
                for (size_t q = 0; q < nb; ++q)
                    if (sub[cc * nb + q] && fe[sub[cc * nb + q]]) ++cnts[cc];
            if ((rc = put(c->off_counts, cnts, sizeof cnts))) return rc;
        } else {
            nlf::VoxParams v{};
            v.nshape = (int)c->shapes.size();
            for (int q = 0; q < v.nshape; ++q) {
                const nlf_shape& s = c->shapes[q];
                nlf::Shape& d = v.shp[q];
                d.kind = s.kind;
                d.material = s.material;
                for (int a = 0; a < 3; ++a) {
                    d.c[a] = s.center[a];
                    d.half[a] = s.half[a];
                }
                d.radius = s.radius;
                d.side = s.side;
                d.tip_base = s.tip_base;
                d.tip_height = s.tip_height;
                d.tip_radius = s.tip_radius;
                d.tip_center = s.tip_center;
                d.tip_cut = s.tip_cut;
            }
            for (int a = 0; a < 3; ++a) {
                v.bb_lo[a] = c->bb_lo[a];
                v.bb_n[a] = c->bb_n[a];
            }
            for (int k = 0; k < 3; ++k) v.mat[k] = at<uint8_t>(c, c->off_mat) + (size_t)k * c->nbb;
            v.counts = at<unsigned long long>(c, c->off_counts);
            v.free_e = at<int>(c, c->off_free);
            nlf::launch_voxelise(v, st);
            CK(cudaGetLastError());
            c->launches += 1;
        }
    }
    if (c->have_mon) {
        std::vector<uint32_t> re, rh, rs;
        std::vector<double> co;
        box_records(c, c->mon.abs_lo, c->mon.abs_hi, re, rh, rs, co);
        box_records(c, c->mon.sca_lo, c->mon.sca_hi, re, rh, rs, co);
        std::vector<uint32_t> all;
        all.reserve(3 * re.size());
        all.insert(all.end(), re.begin(), re.end());
        all.insert(all.end(), rh.begin(), rh.end());
        all.insert(all.end(), rs.begin(), rs.end());
        if ((rc = put(c->off_rec, all.data(), all.size() * sizeof(uint32_t)))) return rc;
        if ((rc = put(c->off_dcoef, co.data(), co.size() * sizeof(double)))) return rc;
        if ((rc = put(c->off_omega, c->omega.data(), c->omega.size() * sizeof(double)))) return rc;
    }
    if (c->have_plane &&
        (rc = put(c->off_pomega, c->plane_omega.data(), c->plane_omega.size() * sizeof(double))))
        return rc;
    if (c->has_metal) {
        nlf::SiteGeom sg{};
        for (int a = 0; a < 3; ++a) {
            sg.bb_lo[a] = c->bb_lo[a];
            sg.bb_n[a] = c->bb_n[a];
            sg.cpml[a] = c->g.boundary[a] == NLF_BC_CPML;
        }
        sg.nx = c->g.nx;
        sg.ny = c->g.ny;
        sg.nz = c->g.nz;
        sg.px = c->px;
        sg.pml = c->g.pml_cells;
        sg.tiles_x = c->tiles_x;
        sg.free_e = at<int>(c, c->off_free);
        // every material site (the batched update walks this list), and the
        // z range of material sites per tile column
        sg.tile_kr = c->fuse ? at<int2>(c, c->off_tilekr) : nullptr;
        nlf::launch_site_list(at<uint8_t>(c, c->off_mat), c->nbb, at<uint32_t>(c, c->off_sites),
                              at<uint32_t>(c, c->off_siteq), sg,
                              at<unsigned long long>(c, c->off_counts) + 3, st);
        CK(cudaGetLastError());
        c->launches += 1;
        if (c->fuse) {
            // the sites of CPML tiles, for the post-step kernel (the tiling
            // of the single-grid step)
            nlf::StepParams tmp{};
            tmp.nx = c->g.nx;
            tmp.ny = c->g.ny;
            tmp.nz = c->g.nz;
            for (int a = 0; a < 3; ++a) tmp.cpml[a] = sg.cpml[a];
            tmp.pml = sg.pml;
            sg.tile_kr = nullptr;
            sg.only_pml = 1;
            sg.kz = nlf::step_kz(tmp);
            nlf::launch_site_list(at<uint8_t>(c, c->off_mat), c->nbb, at<uint32_t>(c, c->off_psites),
                                  at<uint32_t>(c, c->off_psiteq), sg,
                                  at<unsigned long long>(c, c->off_counts) + 5, st);
            CK(cudaGetLastError());
            c->launches += 1;
        }
    }
    fill_params(c);
    // info
    unsigned long long cnts[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(cnts, c->base + c->off_counts, sizeof cnts, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    c->d2h += (long long)sizeof cnts;
    nlf_info& in = c->info;
    in.cells = c->ncell;
    in.metal_sites = (long long)(cnts[0] + cnts[1] + cnts[2]);
    c->n_msites = (long long)cnts[3];
    c->n_psites = c->fuse ? (long long)cnts[5] : c->n_msites;
    c->n_ppl = c->fuse ? (long long)cnts[6] : in.metal_sites;
    in.pole_sites = c->max_poles > 0 ? in.metal_sites : 0;
    in.bbox_cells = c->nbb;
    in.pml_slab_cells = c->pml_slab[0] + c->pml_slab[1] + c->pml_slab[2];
    in.dft_records = c->nrec;
    in.dt = c->dt;
    in.gnor = c->any_gnor;
    in.n_poles = c->max_poles;
    in.material_sites = c->n_msites;
    // the EM kernels: E and H once, CPML psi, and the material update of the
    // sites they update in their march (material id, P_f, a_f, the GNOR
    // history, P_CP and a_CP read and written); the post-step kernel: the
    // site-list update of the CPML tiles' sites (entry and cell offset, id,
    // E read and written, H, and the same hydrodynamic state)
    const double hydro = 8.0 * (2 + (c->any_gnor ? 1 : 0));
    const double pole = 16.0 * c->max_poles;
    const long long f_sites = c->n_msites - c->n_psites, f_pl = in.metal_sites - c->n_ppl;
    in.step_kernel_bytes = 48.0 * c->ncell + 32.0 * in.pml_slab_cells + 1.0 * f_sites + hydro * f_pl +
                           (c->max_poles ? pole * f_pl : 0.0);
    in.metal_kernel_bytes = 21.0 * c->n_psites + hydro * c->n_ppl + (c->max_poles ? pole * c->n_ppl : 0.0);
    in.step_bytes = in.step_kernel_bytes + in.metal_kernel_bytes;
    c->ready = true;
    return NLF_OK;
}

int ensure_ready(nlf_ctx* c, cudaStream_t st)
{
    if (c->ready) return NLF_OK;
    int rc = plan(c);
    if (rc) return rc;
    if (!c->base) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, c->bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, NLF_E_OOM, "cudaMalloc(%zu): %s", c->bytes, cudaGetErrorString(e));
        }
        c->base = (char*)p;
        c->owned = true;
    }
    if (!c->done) CK(cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming));
    if (!c->aux) CK(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
    if (!c->fork) CK(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    if (!c->join) CK(cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming));
    if (!c->aux2) CK(cudaStreamCreateWithFlags(&c->aux2, cudaStreamNonBlocking));
    if (!c->join2) CK(cudaEventCreateWithFlags(&c->join2, cudaEventDisableTiming));
    return initialise(c, st);
}

void monitor_work(nlf_ctx* c, cudaStream_t st);

// The EM step of time step n on st: with CPML tiles, their kernel runs on the
// context's second stream and, with fused metal tiles, the metal kernel on
// its third, concurrently with the other tiles' kernel, forked from and
// joined back into st (a fork / join inside a captured graph too).
void launch_em(nlf_ctx* c, cudaStream_t st)
{
    const nlf::StepParams& sp = c->sp[c->n & 1];
    const bool pml = nlf::step_has_pml(sp);
    const bool met = c->fuse && c->n_msites > c->n_psites;
#ifndef NLF_METAL_AFTER
    // the metal tiles on a third stream beside the others (512^3 cube: 1.833
    // against 1.859 ms per step with the metal kernel after them)
    if (met) {
        cudaEventRecord(c->fork, st);
        cudaStreamWaitEvent(c->aux2, c->fork, 0);
        nlf::launch_step_metal(sp, c->aux2);
        cudaEventRecord(c->join2, c->aux2);
        c->launches += 1;
    }
#endif
    if (pml) {
        cudaEventRecord(c->fork, st);
        cudaStreamWaitEvent(c->aux, c->fork, 0);
        nlf::launch_step_pml(sp, c->aux);
        nlf::launch_step(sp, st);
        cudaEventRecord(c->join, c->aux);
        cudaStreamWaitEvent(st, c->join, 0);
        c->launches += 2;
    } else {
        nlf::launch_step(sp, st);
        c->launches += 1;
    }
#ifndef NLF_METAL_AFTER
    if (met) cudaStreamWaitEvent(st, c->join2, 0);
#else
    // build option: the metal tiles after the others
    if (met) {
        nlf::launch_step_metal(sp, st);
        c->launches += 1;
    }
#endif
}

// The work after the EM step of time step n: the TF/SF corrections and the
// material update touch disjoint cells (material sites lie two cells inside
// the TF surface), so with both present one kernel does both.
void launch_post(nlf_ctx* c, cudaStream_t st)
{
    const nlf::StepParams& sp = c->sp[c->n & 1];
    const bool tf = nlf::tfsf_items(sp) > 0, met = c->n_psites > 0;
    if (tf && met) {
        nlf::launch_post(sp, c->n_psites, st);
        c->launches += 1;
    } else if (tf) {
        nlf::launch_tfsf(sp, st);
        c->launches += 1;
    } else if (met) {
        nlf::launch_metal(sp, c->n_psites, st);
        c->launches += 1;
    }
}

// One time step and its monitor work, launched on st; at the end of every
// period (U steps, one captured graph) the whole-grid non-finite watchdog.
void step_once(nlf_ctx* c, cudaStream_t st)
{
    launch_em(c, st);
    launch_post(c, st);
    c->n += 1;
    monitor_work(c, st);
    if (c->n % c->U == 0) {
        const int cur = (int)(c->n & 1);
        nlf::launch_watch(at<float>(c, c->off_E[cur]), 3 * c->nfield, &at<Header>(c, c->off_hdr)->err, st);
        c->launches += 1;
    }
}

// The running-DFT work due after time step n (c->n already advanced).
void monitor_work(nlf_ctx* c, cudaStream_t st)
{
    if (c->have_plane && c->n % c->plane.decimate_k == 0) {
        const int cur = (int)(c->n & 1);
        const float* E[3];
        const float* P[3];
        for (int q = 0; q < 3; ++q) {
            E[q] = at<float>(c, c->off_E[cur]) + (size_t)q * c->nfield;
            P[q] = c->has_metal ? at<float>(c, c->off_P[cur]) + (size_t)q * c->nbb : nullptr;
        }
        nlf::launch_plane_dft(c->pp, E, c->has_metal ? P : nullptr, &at<Header>(c, c->off_hdr)->step[cur], st);
        c->launches += 1;
    }
    if (c->have_mon && c->n % c->K == 0) {
        const int cur = (int)(c->n & 1);
        Header* h = at<Header>(c, c->off_hdr);
        const float* inc = c->have_src ? at<float>(c, c->off_inc) : nullptr;
        nlf::launch_dft_gather(c->dp, at<float>(c, c->off_E[cur]), at<float>(c, c->off_H[cur]),
                               inc + cur * c->inc_len, inc + (2 + cur) * c->inc_len, c->cnt, &h->step[cur], &h->err,
                               st);
        c->launches += 1;
        c->cnt += 1;
        if (c->cnt == c->B) {
            nlf::launch_dft_flush(c->dp, c->B, st);
            c->launches += 2;
            c->cnt = 0;
        }
    }
}

int build_graph(nlf_ctx* c)
{
    if (c->gexec) return NLF_OK;
    if (!c->cap) CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    // the graph is captured from the aligned state n % U == 0, cnt == 0
    const long long n_save = c->n, l_save = c->launches;
    const int cnt_save = c->cnt;
    c->n = 0;
    c->cnt = 0;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    for (int s = 0; s < c->U; ++s) step_once(c, c->cap);
    cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    c->gnodes = c->launches - l_save;
    c->n = n_save;
    c->cnt = cnt_save;
    c->launches = l_save;
    if (e != cudaSuccess) return fail(c, NLF_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, NLF_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return NLF_OK;
}

int flush_pending(nlf_ctx* c, cudaStream_t st)
{
    if (c->have_mon && c->cnt > 0) {
        nlf::launch_dft_flush(c->dp, c->cnt, st);
        c->launches += 2;
        c->cnt = 0;
        CK(cudaGetLastError());
    }
    return NLF_OK;
}

// ------------------------------------------------------------- batching

// A batched segment plan: the device descriptors of one ordered set of
// instances (and their parities) and the CUDA graph of one DFT period.
struct BatchPlan {
    std::vector<nlf_ctx*> ctxs;       // heaviest first
    std::vector<int> par;             // base parity of each instance
    char* dev = nullptr;              // descriptors (device)
    nlf::BatchStep bs{};
    nlf::BatchDft bd{};
    long long items = 0, met_sites = 0, tf_items = 0, recs = 0, phases = 0, chunks = 0;
    int max_nf = 0, K = 1, B = 8, U = 128;
    bool mon = false;
    int kz = 0;                       // z chunk used for every instance (0: per-instance heuristic)
    std::vector<int> tried;           // autotuner: candidate z chunks tried so far
    std::vector<float> tried_ms;
    long long uses = 0;               // segments run with this plan
    cudaGraphExec_t gexec = nullptr;
    long long gnodes = 0;
    cudaStream_t cap = nullptr;
    bool any_pml = false;             // some instance has CPML tiles: second kernel on aux
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    ~BatchPlan()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (cap) cudaStreamDestroy(cap);
        if (aux) cudaStreamDestroy(aux);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (dev) cudaFree(dev);
    }
};

std::mutex g_batch_mu;
std::vector<std::unique_ptr<BatchPlan>> g_plans;
// Contexts created and not yet destroyed (guarded by g_batch_mu): a batched
// plan is launched only while every context it holds is among them.
std::unordered_set<const nlf_ctx*> g_live;

// NLF_OK if every context of plan P is alive and has its state, else the
// error recorded on the plan's first context.
int plan_alive(BatchPlan* P)
{
    for (nlf_ctx* x : P->ctxs)
        if (!g_live.count(x) || !x->ready || !x->base)
            return fail(P->ctxs[0], NLF_E_STATE, "batched plan holds a context that was released or not initialised");
    return NLF_OK;
}
const int kTuneKz[] = {8, 16, 32};

// Build the device descriptors of a plan for z chunk kz (0: heuristic),
// copied on st, the stream its launches go to.
int plan_descriptors(BatchPlan* P, int kz, cudaStream_t st)
{
    nlf_ctx* c = P->ctxs[0];
    const int n = (int)P->ctxs.size();
    std::vector<nlf::StepParams> params(2 * n);
    std::vector<nlf::BatchInst> inst(n);
    std::vector<long long> item_end(n), met_end(n), tf_end(n), rec_end(n), ph_end(n), chunk_end(n);
    std::vector<nlf::BatchDftInst> dinst(n);
    long long it = 0, ms = 0, tf = 0, rc = 0, ph = 0, ch = 0;
    P->max_nf = 0;
    for (int q = 0; q < n; ++q) {
        nlf_ctx* x = P->ctxs[q];
        params[2 * q] = x->sp[0];
        params[2 * q + 1] = x->sp[1];
        // a block stages its instance's parameters in shared memory, where a
        // tensor map cannot be read from: the maps come from the state
        params[2 * q].map_in_params = 0;
        params[2 * q + 1].map_in_params = 0;
        for (int g2 = 0; g2 < 2 && x->has_metal; ++g2) {
            // batched steps update every material site from the full list
            params[2 * q + g2].fuse_metal = 0;
            params[2 * q + g2].sites = at<uint32_t>(x, x->off_sites);
            params[2 * q + g2].site_q = at<uint32_t>(x, x->off_siteq);
        }
        nlf::BatchInst& b = inst[q];
        b.tiles_x = (x->g.nx + 31) / 32;
        b.tiles_y = (x->g.ny + 7) / 8;
        b.kz = kz > 0 ? kz : nlf::step_kz(x->sp[0]);
        b.chunks = nlf::step_chunks(x->sp[0], b.kz);
        b.base_par = P->par[q];
        it += (long long)b.tiles_x * b.tiles_y * b.chunks;
        item_end[q] = it;
        if (x->has_metal) ms += x->n_msites;
        met_end[q] = ms;
        tf += nlf::tfsf_items(x->sp[0]);
        tf_end[q] = tf;
        if (P->mon) {
            nlf::BatchDftInst& d = dinst[q];
            d.d = x->dp;
            for (int g2 = 0; g2 < 2; ++g2) {
                d.E[g2] = at<float>(x, x->off_E[g2]);
                d.H[g2] = at<float>(x, x->off_H[g2]);
                const float* inc = at<float>(x, x->off_inc);
                d.e_inc[g2] = inc + g2 * x->inc_len;
                d.h_inc[g2] = inc + (2 + g2) * x->inc_len;
                d.step[g2] = &at<Header>(x, x->off_hdr)->step[g2];
            }
            d.err = &at<Header>(x, x->off_hdr)->err;
            d.base_par = P->par[q];
            rc += x->nrec + 1;
            ph += (long long)x->B * x->mon.nf;
            ch += (x->nrec + 1 + NLF_BATCH_RCH * NLF_BATCH_GROUP - 1) / (NLF_BATCH_RCH * NLF_BATCH_GROUP);
            P->max_nf = std::max(P->max_nf, x->mon.nf);
        }
        rec_end[q] = rc;
        ph_end[q] = ph;
        chunk_end[q] = ch;
    }
    P->items = it;
    P->met_sites = ms;
    P->tf_items = tf;
    P->recs = rc;
    P->phases = ph;
    P->chunks = ch;
    size_t o = 0;
    auto take = [&](size_t nb) {
        size_t r = o;
        o = align_up(o + nb, 256);
        return r;
    };
    const size_t o_par = take(params.size() * sizeof(nlf::StepParams));
    const size_t o_inst = take(inst.size() * sizeof(nlf::BatchInst));
    const size_t o_item = take(n * sizeof(long long));
    const size_t o_met = take(n * sizeof(long long));
    const size_t o_tf = take(n * sizeof(long long));
    const size_t o_dinst = take(dinst.size() * sizeof(nlf::BatchDftInst));
    const size_t o_rec = take(n * sizeof(long long));
    const size_t o_ph = take(n * sizeof(long long));
    const size_t o_ch = take(n * sizeof(long long));
    if (!P->dev) {
        cudaError_t e = cudaMalloc(&P->dev, o);
        if (e != cudaSuccess) return fail(c, NLF_E_OOM, "batch descriptors: %s", cudaGetErrorString(e));
    }
    std::vector<char> h(o, 0);
    memcpy(h.data() + o_par, params.data(), params.size() * sizeof(nlf::StepParams));
    memcpy(h.data() + o_inst, inst.data(), inst.size() * sizeof(nlf::BatchInst));
    memcpy(h.data() + o_item, item_end.data(), n * sizeof(long long));
    memcpy(h.data() + o_met, met_end.data(), n * sizeof(long long));
    memcpy(h.data() + o_tf, tf_end.data(), n * sizeof(long long));
    memcpy(h.data() + o_dinst, dinst.data(), dinst.size() * sizeof(nlf::BatchDftInst));
    memcpy(h.data() + o_rec, rec_end.data(), n * sizeof(long long));
    memcpy(h.data() + o_ph, ph_end.data(), n * sizeof(long long));
    memcpy(h.data() + o_ch, chunk_end.data(), n * sizeof(long long));
    // a plain cudaMemcpy from pageable memory goes to the legacy stream and may
    // return before its DMA lands, unordered with launches on a non-blocking
    // stream: copy on st and wait, so that no launch can read the descriptors
    // of an earlier plan that this allocation reuses
    CK(cudaMemcpyAsync(P->dev, h.data(), o, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    P->bs.params = reinterpret_cast<const nlf::StepParams*>(P->dev + o_par);
    P->bs.inst = reinterpret_cast<const nlf::BatchInst*>(P->dev + o_inst);
    P->bs.item_end = reinterpret_cast<const long long*>(P->dev + o_item);
    P->bs.met_end = reinterpret_cast<const long long*>(P->dev + o_met);
    P->bs.tf_end = reinterpret_cast<const long long*>(P->dev + o_tf);
    P->bs.n = n;
    P->bd.inst = reinterpret_cast<const nlf::BatchDftInst*>(P->dev + o_dinst);
    P->bd.rec_end = reinterpret_cast<const long long*>(P->dev + o_rec);
    P->bd.ph_end = reinterpret_cast<const long long*>(P->dev + o_ph);
    P->bd.chunk_end = reinterpret_cast<const long long*>(P->dev + o_ch);
    P->bd.n = n;
    P->kz = kz;
    return NLF_OK;
}

// Launch one DFT period of batched work (step, gathers, flushes) on st, or
// its first `steps` time steps (steps < U: no flush, the samples stay in
// their slots); returns the number of kernel launches.
long long plan_launch(BatchPlan* P, cudaStream_t st, int steps = 0)
{
    long long nodes = 0;
    int slot = 0;
    const int S = steps > 0 ? steps : P->U;
    for (int s = 0; s < S; ++s) {
        nlf::BatchStep bs = P->bs;
        bs.launch_par = s & 1;
        if (P->any_pml) {
            // CPML tiles on the plan's second stream, forked from and joined into st
            cudaEventRecord(P->fork, st);
            cudaStreamWaitEvent(P->aux, P->fork, 0);
            nlf::launch_step_batch_pml(bs, P->items, P->aux);
            nlf::launch_step_batch(bs, P->items, st);
            cudaEventRecord(P->join, P->aux);
            cudaStreamWaitEvent(st, P->join, 0);
            nodes += 2;
        } else {
            nlf::launch_step_batch(bs, P->items, st);
            ++nodes;
        }
        if (P->met_sites + P->tf_items > 0) {
            // material sites and TF/SF items of every instance in one launch
            nlf::launch_post_batch(bs, P->met_sites, P->tf_items, st);
            ++nodes;
        }
        if (s + 1 == S) {
            // the whole-grid non-finite watchdog of every instance
            for (size_t q = 0; q < P->ctxs.size(); ++q) {
                nlf_ctx* x = P->ctxs[q];
                const int cur = (P->par[q] + S) & 1;
                nlf::launch_watch(at<float>(x, x->off_E[cur]), 3 * x->nfield, &at<Header>(x, x->off_hdr)->err, st);
                ++nodes;
            }
        }
        if (P->mon && (s + 1) % P->K == 0) {
            nlf::BatchDft bd = P->bd;
            bd.cur_par = (s + 1) & 1;
            nlf::launch_gather_batch(bd, P->recs, slot, st);
            ++nodes;
            if (++slot == P->B) {
                nlf::launch_flush_batch(bd, P->phases, P->chunks, P->max_nf, P->B, P->B, st);
                nodes += 2;
                slot = 0;
            }
        }
    }
    return nodes;
}

// Capture one DFT period of batched launches in a CUDA graph.
int plan_graph(BatchPlan* P)
{
    nlf_ctx* c = P->ctxs[0];
    if (P->gexec) {
        cudaGraphExecDestroy(P->gexec);
        P->gexec = nullptr;
    }
    if (!P->cap) CK(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
    const long long nodes = plan_launch(P, P->cap);
    cudaError_t e = cudaStreamEndCapture(P->cap, &g);
    if (e != cudaSuccess) return fail(c, NLF_E_CUDA, "batch graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&P->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, NLF_E_CUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    P->gnodes = nodes;
    return NLF_OK;
}

double inst_cost(const nlf_ctx* c)
{
    return (double)c->ncell + 2.0 * (double)c->nbb;   // metal box cells cost about three times a vacuum cell
}

int g_kz_best = 0;                    // z chunk chosen by the autotuner (0: not tuned yet)

BatchPlan* find_plan(std::vector<nlf_ctx*> act, cudaStream_t st, int* rcode)
{
    std::stable_sort(act.begin(), act.end(),
                     [](const nlf_ctx* a, const nlf_ctx* b) { return inst_cost(a) > inst_cost(b); });
    std::vector<int> par(act.size());
    for (size_t q = 0; q < act.size(); ++q) par[q] = (int)(act[q]->n & 1);
    for (auto& P : g_plans)
        if (P->ctxs == act && P->par == par) return P.get();
    std::unique_ptr<BatchPlan> P(new BatchPlan());
    P->ctxs = act;
    P->par = par;
    P->mon = act[0]->have_mon;
    P->K = act[0]->K;
    P->B = act[0]->B;
    P->U = act[0]->U;
    for (nlf_ctx* x : act) {
        if (nlf::step_has_pml(x->sp[0])) P->any_pml = true;
    }
    if (P->any_pml) {
        if (cudaStreamCreateWithFlags(&P->aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->join, cudaEventDisableTiming) != cudaSuccess) {
            *rcode = fail(act[0], NLF_E_CUDA, "batch plan streams");
            return nullptr;
        }
    }
    *rcode = plan_descriptors(P.get(), g_kz_best, st);
    if (*rcode) return nullptr;
    g_plans.push_back(std::move(P));
    return g_plans.back().get();
}

// Advance every instance of `act` by one DFT period in batched launches.
// Until the autotuner has chosen a z chunk, successive segments run with each
// candidate (every candidate computes the same update; only the work split
// differs) timed with events, and the fastest is kept for every later plan.
// A plan's first segment is launched directly; a plan that comes back is
// captured once and replayed as a CUDA graph.
int batch_segment(const std::vector<nlf_ctx*>& act, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    int rcode = NLF_OK;
    BatchPlan* P = find_plan(act, st, &rcode);
    if (!P) return rcode;
    if ((rcode = plan_alive(P))) return rcode;
    nlf_ctx* c = P->ctxs[0];
    const int ncand = (int)(sizeof(kTuneKz) / sizeof(kTuneKz[0]));
    if (g_kz_best == 0) {
        const int kz = kTuneKz[P->tried.size() % ncand];
        if ((rcode = plan_descriptors(P, kz, st))) return rcode;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, st));
        c->launches += plan_launch(P, st);
        CK(cudaGetLastError());
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        P->tried.push_back(kz);
        P->tried_ms.push_back(ms);
        if ((int)P->tried.size() == ncand) {
            size_t best = 0;
            for (size_t q = 1; q < P->tried.size(); ++q)
                if (P->tried_ms[q] < P->tried_ms[best]) best = q;
            g_kz_best = P->tried[best];
            if ((rcode = plan_descriptors(P, g_kz_best, st))) return rcode;
        }
    } else if (P->uses == 0) {
        c->launches += plan_launch(P, st);
        CK(cudaGetLastError());
    } else {
        if (!P->gexec && (rcode = plan_graph(P))) return rcode;
        CK(cudaGraphLaunch(P->gexec, st));
        c->launches += P->gnodes;
    }
    P->uses += 1;
    for (nlf_ctx* x : P->ctxs) x->n += P->U;
    return NLF_OK;
}

// Advance every instance of `act` (on a DFT period boundary, nothing
// buffered) by `steps` < U time steps in batched launches, launched directly:
// the samples of the partial period stay in their slots (cnt of each
// context), to be accumulated by the next flush of the single-grid path.
int batch_tail(const std::vector<nlf_ctx*>& act, int steps, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    int rcode = NLF_OK;
    BatchPlan* P = find_plan(act, st, &rcode);
    if (!P) return rcode;
    if ((rcode = plan_alive(P))) return rcode;
    if (steps <= 0 || steps >= P->U) return NLF_E_ARG;
    nlf_ctx* c = P->ctxs[0];
    c->launches += plan_launch(P, st, steps);
    CK(cudaGetLastError());
    for (nlf_ctx* x : P->ctxs) {
        x->n += steps;
        if (P->mon) x->cnt = (steps / P->K) % P->B;   // a period of 2 K B steps flushes once within
    }
    return NLF_OK;
}

void register_ctx(const nlf_ctx* x)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_live.insert(x);
}

void drop_plans(const nlf_ctx* x)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_live.erase(x);
    for (size_t q = 0; q < g_plans.size();) {
        if (std::find(g_plans[q]->ctxs.begin(), g_plans[q]->ctxs.end(), x) != g_plans[q]->ctxs.end())
            g_plans.erase(g_plans.begin() + q);
        else
            ++q;
    }
}

}  // namespace

// ===================================================================== ABI

extern "C" {

int nlf_create(const nlf_grid* grid, nlf_ctx** out)
{
    if (!grid || !out) return NLF_E_ARG;
    *out = nullptr;
    const nlf_grid& g = *grid;
    if (g.nx < 8 || g.ny < 8 || g.nz < 8 || !(g.dx > 0.0) || !(g.courant > 0.0) || !(g.eps_background >= 1.0 - 1e-12))
        return NLF_E_ARG;
    if ((long long)((g.nx + 7) & ~7) * g.ny * g.nz * 3 >= (1LL << 32)) return NLF_E_ARG;
    if (g.courant > 1.0 / std::sqrt(3.0) + 1e-12) return NLF_E_CFL;
    for (int a = 0; a < 3; ++a) {
        if (g.boundary[a] != NLF_BC_PEC && g.boundary[a] != NLF_BC_CPML) return NLF_E_ARG;
        const int n = a == 0 ? g.nx : a == 1 ? g.ny : g.nz;
        if (g.boundary[a] == NLF_BC_CPML && (g.pml_cells < 1 || 2 * g.pml_cells + 4 > n)) return NLF_E_ARG;
    }
    static std::atomic<long long> next_id{0};
    nlf_ctx* c = new nlf_ctx();
    c->id = ++next_id;
    c->g = g;
    c->c0 = 1.0 / std::sqrt(kEps0 * kMu0);
    c->eta0 = std::sqrt(kMu0 / kEps0);
    c->dt = g.courant * g.dx / c->c0;
    c->ncell = (long long)g.nx * g.ny * g.nz;
    c->px = (g.nx + 7) & ~7;
    c->nfield = (long long)c->px * g.ny * g.nz;
    register_ctx(c);
    *out = c;
    return NLF_OK;
}

int nlf_set_materials(nlf_ctx* c, const nlf_material* mats, int n)
{
    if (!c || n < 0 || n > NLF_MAX_MATERIALS || (n > 0 && !mats)) return NLF_E_ARG;
    if (c->ready) return fail(c, NLF_E_STATE, "materials are fixed after the first run");
    for (int q = 0; q < n; ++q) {
        const nlf_material& m = mats[q];
        if (m.n_poles < 0 || m.n_poles > NLF_MAX_POLES || m.eps_inf < 1e-6 || m.wp < 0 || m.gamma < 0 ||
            m.beta < 0 || m.diff < 0)
            return fail(c, NLF_E_ARG, "material %d: bad parameters", q + 1);
        const double eta = m.beta * m.beta + m.diff * m.gamma;
        if (std::sqrt(eta) * c->dt * std::sqrt(3.0) / c->g.dx > 1.0)
            return fail(c, NLF_E_CFL, "material %d: hydrodynamic term unstable (beta dt sqrt3/dx > 1)", q + 1);
    }
    c->mats.assign(mats, mats + n);
    c->planned = false;
    return NLF_OK;
}

int nlf_set_shapes(nlf_ctx* c, const nlf_shape* shapes, int n)
{
    if (!c || n < 0 || n > NLF_MAX_SHAPES || (n > 0 && !shapes)) return NLF_E_ARG;
    if (c->ready) return fail(c, NLF_E_STATE, "geometry is fixed after the first run");
    for (int q = 0; q < n; ++q) {
        const nlf_shape& s = shapes[q];
        if (s.kind < NLF_SHAPE_SPHERE || s.kind > NLF_SHAPE_CUBE_TIPS || s.material < 1 ||
            s.material > NLF_MAX_MATERIALS)
            return fail(c, NLF_E_ARG, "shape %d: bad kind or material", q);
        if (s.kind == NLF_SHAPE_CUBE_TIPS && (s.side % 2 || s.tip_base % 2 || s.tip_height <= 0))
            return fail(c, NLF_E_ARG, "shape %d: cube side and tip base must be even, tip height > 0", q);
    }
    c->shapes.assign(shapes, shapes + n);
    c->use_map = false;
    c->map.clear();
    c->planned = false;
    return NLF_OK;
}

int nlf_set_material_map(nlf_ctx* c, const uint8_t* ids3, int on_device)
{
    if (!c || !ids3) return NLF_E_ARG;
    if (c->ready) return fail(c, NLF_E_STATE, "geometry is fixed after the first run");
    if (on_device) {
        // the map is planned on the host (bounding box, id checks): copy it
        // over once every stream's work has finished (the caller may have
        // written it on a stream that a legacy-stream copy does not wait for)
        std::vector<uint8_t> h(3 * (size_t)c->ncell);
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(h.data(), ids3, h.size(), cudaMemcpyDeviceToHost));
        c->d2h += (long long)h.size();
        c->map.swap(h);
    } else {
        c->map.assign(ids3, ids3 + 3 * (size_t)c->ncell);
    }
    c->use_map = true;
    c->shapes.clear();
    c->planned = false;
    return NLF_OK;
}

int nlf_set_source(nlf_ctx* c, const nlf_source* s)
{
    if (!c || !s) return NLF_E_ARG;
    if (c->ready) return fail(c, NLF_E_STATE, "source is fixed after the first run");
    if (s->axis_prop != 2 || s->axis_pol != 0)
        return fail(c, NLF_E_UNSUPPORTED, "only +z propagation with x polarisation is implemented");
    if (s->waveform != NLF_WAVE_GAUSSIAN && s->waveform != NLF_WAVE_RAISED_COS) return NLF_E_ARG;
    if (s->waveform == NLF_WAVE_GAUSSIAN && !(s->tau > 0.0)) return NLF_E_ARG;
    if (!(s->w0 > 0.0)) return NLF_E_ARG;
    c->src = *s;
    c->have_src = true;
    c->planned = false;
    return NLF_OK;
}

int nlf_set_monitors(nlf_ctx* c, const nlf_monitors* m)
{
    if (!c || !m || m->nf < 1 || !m->omega || m->decimate_k < 1 || m->block_b < 0 || m->block_b > 32)
        return NLF_E_ARG;
    if (c->ready) return fail(c, NLF_E_STATE, "monitors are fixed after the first run");
    if (!c->have_src) return fail(c, NLF_E_STATE, "set the source before the monitors");
    if (c->have_plane && m->decimate_k != c->plane.decimate_k)
        return fail(c, NLF_E_ARG, "monitor decimate_k must equal the plane monitor's");
    c->mon = *m;
    c->omega.assign(m->omega, m->omega + m->nf);
    c->mon.omega = c->omega.data();
    c->have_mon = true;
    c->planned = false;
    return NLF_OK;
}

int nlf_set_plane_monitor(nlf_ctx* c, const nlf_plane_monitor* m)
{
    if (!c || !m || m->axis < 0 || m->axis > 2 || m->nf < 1 || m->nf > NLF_PLANE_MAX_NF || !m->omega ||
        m->decimate_k < 1)
        return NLF_E_ARG;
    const int n3[3] = {c->g.nx, c->g.ny, c->g.nz};
    if (m->index < 0 || m->index >= n3[m->axis]) return fail(c, NLF_E_ARG, "plane index outside the grid");
    if (c->ready) return fail(c, NLF_E_STATE, "the plane monitor is fixed after the first run");
    if (c->have_mon && m->decimate_k != c->mon.decimate_k)
        return fail(c, NLF_E_ARG, "plane decimate_k must equal the flux monitors'");
    c->plane = *m;
    c->plane_omega.assign(m->omega, m->omega + m->nf);
    c->plane.omega = c->plane_omega.data();
    c->have_plane = true;
    c->planned = false;
    return NLF_OK;
}

int nlf_get_plane_map(nlf_ctx* c, int which, double* dst)
{
    if (!c || !dst || !((which >= NLF_FIELD_EX && which <= NLF_FIELD_EZ) || which == NLF_MAP_DENSITY))
        return NLF_E_ARG;
    if (!c->have_plane || !c->ready) return fail(c, NLF_E_STATE, "no plane monitor or no run yet");
    CK(cudaStreamSynchronize(c->stream));
    const int w = which == NLF_MAP_DENSITY ? 3 : which;
    const size_t per = (size_t)c->plane.nf * c->pp.n1 * c->pp.n2;
    CK(cudaMemcpy(dst, c->base + c->off_pacc + (size_t)w * per * sizeof(double2), per * sizeof(double2),
                  cudaMemcpyDeviceToHost));
    c->d2h += (long long)(per * sizeof(double2));
    return NLF_OK;
}

size_t nlf_state_bytes(const nlf_ctx* cc)
{
    nlf_ctx* c = const_cast<nlf_ctx*>(cc);
    if (!c) return 0;
    if (plan(c)) return 0;
    return c->bytes;
}

int nlf_bind_state(nlf_ctx* c, void* dev_ptr, size_t bytes)
{
    if (!c || !dev_ptr || ((uintptr_t)dev_ptr & 255)) return NLF_E_ARG;
    if (c->base) return fail(c, NLF_E_STATE, "state already allocated");
    int rc = plan(c);
    if (rc) return rc;
    if (bytes < c->bytes) return fail(c, NLF_E_OOM, "bound buffer %zu < %zu bytes", bytes, c->bytes);
    c->base = (char*)dev_ptr;
    c->owned = false;
    return NLF_OK;
}

int nlf_run(nlf_ctx* c, long long steps, void* stream)
{
    if (!c || steps < 0) return NLF_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_ready(c, st);
    if (rc) return rc;
    c->stream = st;
    bool graph_tried = false;
    while (steps > 0) {
        const bool aligned = c->cnt == 0 && (c->n % 2 == 0) && (!c->have_mon || c->n % c->K == 0);
        if (aligned && steps >= c->U) {
            if (!graph_tried) {
                graph_tried = true;
                if ((rc = build_graph(c))) return rc;
            }
            CK(cudaGraphLaunch(c->gexec, st));
            c->n += c->U;
            c->launches += c->gnodes;
            steps -= c->U;
        } else {
            step_once(c, st);
            steps -= 1;
        }
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(c->done, st));
    return NLF_OK;
}

int nlf_time_kernels(nlf_ctx* c, long long steps, void* stream, double* ms_out)
{
    if (!c || !ms_out || steps < 1 || steps > 65536) return NLF_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_ready(c, st);
    if (rc) return rc;
    c->stream = st;
    // four events per step: before the step kernel, after it, after the
    // material update, after the monitor kernels
    std::vector<cudaEvent_t> ev((size_t)(4 * steps), nullptr);
    auto release = [&]() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    };
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            release();
            return fail(c, NLF_E_CUDA, "event creation failed");
        }
    // the instrumented steps are captured and replayed once as a graph, the
    // way nlf_run executes steps, so that launch overheads of eager launches
    // (and of the fork / join of the CPML kernel) do not enter the figures; the timing events are recorded as external event nodes (a plain record
    // inside a capture only orders streams)
    if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
        release();
        return fail(c, NLF_E_CUDA, "capture stream");
    }
    cudaError_t err = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) {
        release();
        return fail(c, NLF_E_CUDA, "kernel timing capture: %s", cudaGetErrorString(err));
    }
    for (long long s = 0; s < steps; ++s) {
        cudaEvent_t* e = &ev[(size_t)(4 * s)];
        cudaEventRecordWithFlags(e[0], c->cap, cudaEventRecordExternal);
        launch_em(c, c->cap);
        cudaEventRecordWithFlags(e[1], c->cap, cudaEventRecordExternal);
        launch_post(c, c->cap);
        cudaEventRecordWithFlags(e[2], c->cap, cudaEventRecordExternal);
        c->n += 1;
        monitor_work(c, c->cap);
        cudaEventRecordWithFlags(e[3], c->cap, cudaEventRecordExternal);
    }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    err = cudaStreamEndCapture(c->cap, &g);
    if (err == cudaSuccess) err = cudaGraphInstantiate(&x, g, 0);
    if (err == cudaSuccess) err = cudaGraphLaunch(x, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long s = 0; s < steps && err == cudaSuccess; ++s) {
        cudaEvent_t* e = &ev[(size_t)(4 * s)];
        for (int q = 0; q < 3; ++q) {
            float ms = 0.f;
            err = cudaEventElapsedTime(&ms, e[q], e[q + 1]);
            if (err != cudaSuccess) break;
            acc[q] += ms;
        }
    }
    release();
    if (err != cudaSuccess) return fail(c, NLF_E_CUDA, "kernel timing: %s", cudaGetErrorString(err));
    for (int q = 0; q < 3; ++q) ms_out[q] = acc[q];
    CK(cudaEventRecord(c->done, st));
    return NLF_OK;
}

int nlf_reset(nlf_ctx* c, void* stream)
{
    if (!c) return NLF_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    c->stream = st;
    if (!c->ready) return ensure_ready(c, st);
    c->ready = false;
    c->n = 0;
    c->cnt = 0;
    return initialise(c, st);
}

int nlf_sync(nlf_ctx* c, int timeout_ms)
{
    if (!c) return NLF_E_ARG;
    if (!c->ready) return NLF_OK;
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(c->done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return fail(c, NLF_E_CUDA, "event query: %s", cudaGetErrorString(e));
        if (timeout_ms >= 0 &&
            std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
            return fail(c, NLF_E_TIMEOUT, "work still running after %d ms", timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    Header h{};
    CK(cudaMemcpy(&h, c->base + c->off_hdr, sizeof h, cudaMemcpyDeviceToHost));
    if (h.err & 8 && h.chk.code == 30)
        return fail(c, NLF_E_CUDA, "context check: parameters made for context %lld ran on the state of context %lld "
                    "(this context: %lld; %d launches' work skipped)", h.chk.lim, h.chk.idx, c->id, h.chk.hits);
    if (h.err & 8)
        return fail(c, NLF_E_CUDA, "bounds check: access site %d index %lld outside [0, %lld) (%d accesses skipped)",
                    h.chk.code, h.chk.idx, h.chk.lim, h.chk.hits);
    if (h.err & 1) return fail(c, NLF_E_UNSTABLE, "non-finite field sample at time index %lld", c->n);
    if (h.err & 4) return fail(c, NLF_E_CUDA, "a tensor-memory copy of the step kernel did not complete in time");
    return NLF_OK;
}

int nlf_get_field(nlf_ctx* c, int which, void* dst, int on_device)
{
    if (!c || !dst || which < 0 || which > NLF_FIELD_DENSITY) return NLF_E_ARG;
    if (!c->ready) return fail(c, NLF_E_STATE, "no state yet");
    cudaStream_t st = c->stream;
    CK(cudaStreamSynchronize(st));
    const int cur = (int)(c->n & 1);
    const int comp = which % 3;
    const size_t n = (size_t)c->ncell;
    if (which <= NLF_FIELD_HZ) {
        const float* src = at<float>(c, which < 3 ? c->off_E[cur] : c->off_H[cur]) + comp * (size_t)c->nfield;
        const float scale = which < 3 ? 1.f : (float)(1.0 / c->eta0);
        const long long rows = (long long)c->g.ny * c->g.nz;
        if (on_device) {
            nlf::launch_field_out(src, (float*)dst, c->g.nx, c->px, rows, scale, st);
            c->launches += 1;
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(st));
        } else {
            // drop the row padding: nx floats of every px-float row
            CK(cudaMemcpy2D(dst, (size_t)c->g.nx * sizeof(float), src, (size_t)c->px * sizeof(float),
                            (size_t)c->g.nx * sizeof(float), (size_t)rows, cudaMemcpyDeviceToHost));
            c->d2h += (long long)(n * sizeof(float));
            if (scale != 1.f)
                for (size_t q = 0; q < n; ++q) ((float*)dst)[q] *= scale;
        }
        return NLF_OK;
    }
    if (which == NLF_FIELD_DENSITY) {
        // div P_f at every node, computed on the device into dst or into a
        // staging area of the state (the sample buffer is not large enough
        // in general, so a host destination goes through a temporary)
        nlf::DensityParams d{};
        d.nx = c->g.nx;
        d.ny = c->g.ny;
        d.nz = c->g.nz;
        d.eps0_dx = kEps0 / c->g.dx;
        for (int a = 0; a < 3; ++a) {
            d.bb_lo[a] = c->bb_lo[a];
            d.bb_n[a] = c->has_metal ? c->bb_n[a] : 0;
            d.P[a] = c->has_metal ? at<float>(c, c->off_P[cur]) + (size_t)a * c->nbb : nullptr;
        }
        float* out = (float*)dst;
        float* tmp = nullptr;
        if (!on_device) {
            CK(cudaMallocAsync((void**)&tmp, n * sizeof(float), st));
            out = tmp;
        }
        nlf::launch_density_out(d, out, st);
        c->launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && tmp) {
            e = cudaMemcpyAsync(dst, tmp, n * sizeof(float), cudaMemcpyDeviceToHost, st);
            c->d2h += (long long)(n * sizeof(float));
        }
        if (tmp) cudaFreeAsync(tmp, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(c, NLF_E_CUDA, "density output: %s", cudaGetErrorString(e));
        return NLF_OK;
    }
    std::vector<float> full(n, 0.f);
    if (c->has_metal) {
        const size_t nb = (size_t)c->nbb;
        std::vector<float> sub(nb);
        CK(cudaMemcpy(sub.data(), at<float>(c, c->off_P[cur]) + comp * nb, nb * sizeof(float),
                      cudaMemcpyDeviceToHost));
        for (int bk = 0; bk < c->bb_n[2]; ++bk)
            for (int bj = 0; bj < c->bb_n[1]; ++bj)
                for (int bi = 0; bi < c->bb_n[0]; ++bi)
                    full[((size_t)(bk + c->bb_lo[2]) * c->g.ny + (bj + c->bb_lo[1])) * c->g.nx + bi + c->bb_lo[0]] =
                        (float)(kEps0 * sub[((size_t)bk * c->bb_n[1] + bj) * c->bb_n[0] + bi]);
    }
    if (on_device) {
        CK(cudaMemcpyAsync(dst, full.data(), n * sizeof(float), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    } else {
        memcpy(dst, full.data(), n * sizeof(float));
    }
    return NLF_OK;
}

int nlf_set_field(nlf_ctx* c, int which, const void* src, int src_on_device)
{
    if (!c || !src || which < NLF_FIELD_EX || which > NLF_FIELD_HZ) return NLF_E_ARG;
    int rc = ensure_ready(c, c->stream);
    if (rc) return rc;
    cudaStream_t st = c->stream;
    CK(cudaStreamSynchronize(st));
    const int cur = (int)(c->n & 1);
    const int comp = which % 3;
    float* dst = at<float>(c, which < 3 ? c->off_E[cur] : c->off_H[cur]) + comp * (size_t)c->nfield;
    const long long rows = (long long)c->g.ny * c->g.nz;
    const size_t n = (size_t)c->ncell;
    // into the padded rows; H is held as eta0 H
    std::vector<float> h;
    const float* from = static_cast<const float*>(src);
    if (src_on_device) {
        // the source may have been written on any stream (see
        // nlf_set_material_map)
        h.resize(n);
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(h.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost));
        from = h.data();
    }
    if (which >= 3) {
        if (h.empty()) h.assign(from, from + n);
        for (size_t q = 0; q < n; ++q) h[q] = (float)(h[q] * c->eta0);
        from = h.data();
    }
    // on the context's stream, waited for (see nlf_load_state)
    CK(cudaMemcpy2DAsync(dst, (size_t)c->px * sizeof(float), from, (size_t)c->g.nx * sizeof(float),
                         (size_t)c->g.nx * sizeof(float), (size_t)rows, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    c->h2d += (long long)(n * sizeof(float));
    return NLF_OK;
}

int nlf_get_voxels(nlf_ctx* c, uint8_t* dst)
{
    if (!c || !dst) return NLF_E_ARG;
    int rc = ensure_ready(c, c->stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    const size_t n = (size_t)c->ncell;
    memset(dst, 0, 3 * n);
    if (!c->has_metal) return NLF_OK;
    const size_t nb = (size_t)c->nbb;
    std::vector<uint8_t> sub(3 * nb);
    CK(cudaMemcpy(sub.data(), c->base + c->off_mat, 3 * nb, cudaMemcpyDeviceToHost));
    for (int cc = 0; cc < 3; ++cc)
        for (int bk = 0; bk < c->bb_n[2]; ++bk)
            for (int bj = 0; bj < c->bb_n[1]; ++bj)
                for (int bi = 0; bi < c->bb_n[0]; ++bi)
                    dst[cc * n + ((size_t)(bk + c->bb_lo[2]) * c->g.ny + (bj + c->bb_lo[1])) * c->g.nx + bi +
                        c->bb_lo[0]] = sub[cc * nb + ((size_t)bk * c->bb_n[1] + bj) * c->bb_n[0] + bi];
    return NLF_OK;
}

int nlf_get_spectra(nlf_ctx* c, double* s_ext, double* s_abs, double* s_sca)
{
    if (!c) return NLF_E_ARG;
    if (!c->ready || !c->have_mon) return fail(c, NLF_E_STATE, "no monitors or no run yet");
    cudaStream_t st = c->stream;
    int rc = flush_pending(c, st);
    if (rc) return rc;
    const int nf = c->mon.nf;
    double* out = at<double>(c, c->off_out);
    nlf::launch_flux(c->dp.accE, c->dp.accH, at<double>(c, c->off_dcoef), c->n_abs, c->nrec, nf,
                     at<double2>(c, c->off_partial), c->G, c->g.dx * c->g.dx, out, st);
    c->launches += 2;
    CK(cudaGetLastError());
    std::vector<double> h(4 * (size_t)nf);
    CK(cudaMemcpyAsync(h.data(), out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    c->d2h += (long long)(h.size() * sizeof(double));
    if (s_ext) memcpy(s_ext, h.data(), nf * sizeof(double));
    if (s_abs) memcpy(s_abs, h.data() + nf, nf * sizeof(double));
    if (s_sca) memcpy(s_sca, h.data() + 2 * nf, nf * sizeof(double));
    return NLF_OK;
}

long long nlf_num_records(const nlf_ctx* cc)
{
    nlf_ctx* c = const_cast<nlf_ctx*>(cc);
    if (!c || !c->have_mon || plan(c)) return -1;
    return c->nrec;
}

int nlf_get_flux_weights(nlf_ctx* c, double* coef, long long* n_abs)
{
    if (!c || !coef || !n_abs) return NLF_E_ARG;
    if (!c->have_mon) return fail(c, NLF_E_STATE, "no monitors");
    int rc = plan(c);
    if (rc) return rc;
    std::vector<uint32_t> re, rh, rs;
    std::vector<double> co;
    box_records(c, c->mon.abs_lo, c->mon.abs_hi, re, rh, rs, co);
    box_records(c, c->mon.sca_lo, c->mon.sca_hi, re, rh, rs, co);
    memcpy(coef, co.data(), co.size() * sizeof(double));
    *n_abs = c->n_abs;
    return NLF_OK;
}

int nlf_get_dft(nlf_ctx* c, double* dst)
{
    if (!c || !dst) return NLF_E_ARG;
    if (!c->ready || !c->have_mon) return fail(c, NLF_E_STATE, "no monitors or no run yet");
    cudaStream_t st = c->stream;
    int rc = flush_pending(c, st);
    if (rc) return rc;
    const size_t n = ((size_t)c->nrec + 1) * c->mon.nf * 2;
    CK(cudaMemcpyAsync(dst, c->dp.accE, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    c->d2h += (long long)(2 * n * sizeof(double));
    const double se = c->K * c->dt, sh = c->K * c->dt / c->eta0;
    for (size_t q = 0; q < n; ++q) dst[q] *= se;
    for (size_t q = 0; q < n; ++q) dst[n + q] *= sh;
    return NLF_OK;
}

int nlf_save_state(nlf_ctx* c, void* host)
{
    if (!c || !host) return NLF_E_ARG;
    int rc = ensure_ready(c, c->stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    Header h{};
    CK(cudaMemcpy(&h, c->base + c->off_hdr, sizeof h, cudaMemcpyDeviceToHost));
    h.n = c->n;
    h.cnt = c->cnt;
    CK(cudaMemcpy(c->base + c->off_hdr, &h, sizeof h, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(host, c->base, c->bytes, cudaMemcpyDeviceToHost));
    return NLF_OK;
}

int nlf_load_state(nlf_ctx* c, const void* host)
{
    if (!c || !host) return NLF_E_ARG;
    int rc = ensure_ready(c, c->stream);
    if (rc) return rc;
    // copies on the context's stream, waited for: later launches on any
    // stream read the loaded state (a plain cudaMemcpy from pageable memory
    // may return before its DMA lands)
    cudaStream_t st = c->stream;
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpyAsync(c->base, host, c->bytes, cudaMemcpyHostToDevice, st));
    // the tensor maps hold this buffer's addresses, not the saved state's,
    // and the header this context's id
    CK(cudaMemcpyAsync(c->base + c->off_tmap, c->tmaps, sizeof c->tmaps, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->base + c->off_hdr + offsetof(Header, ctx_id), &c->id, sizeof c->id,
                       cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    Header h{};
    memcpy(&h, host, sizeof h);
    c->n = h.n;
    c->cnt = h.cnt;
    return NLF_OK;
}

int nlf_batch_run(nlf_ctx** ctxs, int n, const long long* steps, void* stream, int* status_out)
{
    if (!ctxs || n < 0 || n > NLF_MAX_BATCH || !steps) return NLF_E_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> rc(n, NLF_OK);
    std::vector<long long> rem(n, 0);
    std::vector<int> batchable;
    for (int q = 0; q < n; ++q) {
        nlf_ctx* c = ctxs[q];
        if (!c || steps[q] < 0 || c->have_plane) {   // plane maps are single-grid only
            rc[q] = NLF_E_ARG;
            continue;
        }
        rc[q] = ensure_ready(c, st);
        if (rc[q]) continue;
        rem[q] = steps[q];
        batchable.push_back(q);
    }
    // instances join a batched segment when they sit on a DFT period boundary
    // with the same period as the first one; the others run on their own
    int K = 0, B = 0, U = 0;
    bool mon = false;
    std::vector<int> members;
    for (int q : batchable) {
        nlf_ctx* c = ctxs[q];
        if (members.empty()) {
            K = c->K;
            B = c->B;
            U = c->U;
            mon = c->have_mon;
        }
        const bool fits = c->have_mon == mon && c->K == K && c->B == B && c->U == U && c->cnt == 0 &&
                          (!mon || c->n % K == 0);
        if (fits) members.push_back(q);
    }
    for (;;) {
        std::vector<nlf_ctx*> act;
        for (int q : members)
            if (rc[q] == NLF_OK && rem[q] >= U) act.push_back(ctxs[q]);
        if (act.empty()) break;
        int r = batch_segment(act, st);
        for (int q : members) {
            if (rc[q] != NLF_OK || rem[q] < U) continue;
            if (r) {
                rc[q] = r;
                continue;
            }
            rem[q] -= U;
        }
        if (r) break;
    }
    // members left with the same number of steps short of a period advance
    // batched too, one group per remainder
    std::vector<long long> tails;
    for (int q : members)
        if (rc[q] == NLF_OK && rem[q] > 0 && rem[q] < U &&
            std::find(tails.begin(), tails.end(), rem[q]) == tails.end())
            tails.push_back(rem[q]);
    for (long long r : tails) {
        std::vector<nlf_ctx*> act;
        for (int q : members)
            if (rc[q] == NLF_OK && rem[q] == r) act.push_back(ctxs[q]);
        if (act.size() < 2) continue;
        const int e = batch_tail(act, (int)r, st);
        for (int q : members)
            if (rc[q] == NLF_OK && rem[q] == r) {
                if (e)
                    rc[q] = e;
                else
                    rem[q] = 0;
            }
    }
    for (int q : batchable) {
        if (rc[q] == NLF_OK && rem[q] > 0) rc[q] = nlf_run(ctxs[q], rem[q], stream);
        if (rc[q] == NLF_OK) {
            nlf_ctx* c = ctxs[q];
            c->stream = st;
            cudaError_t e = cudaEventRecord(c->done, st);
            if (e != cudaSuccess) rc[q] = fail(c, NLF_E_CUDA, "event record: %s", cudaGetErrorString(e));
        }
    }
    int worst = NLF_OK;
    for (int q = 0; q < n; ++q) {
        if (status_out) status_out[q] = rc[q];
        if (rc[q] && worst == NLF_OK) worst = rc[q];
    }
    return worst;
}

long long nlf_time_index(const nlf_ctx* c) { return c ? c->n : -1; }

int nlf_get_info(nlf_ctx* c, nlf_info* info)
{
    if (!c || !info) return NLF_E_ARG;
    int rc = ensure_ready(c, c->stream);
    if (rc) return rc;
    *info = c->info;
    info->h2d_bytes = c->h2d;
    info->d2h_bytes = c->d2h;
    return NLF_OK;
}

long long nlf_kernel_launches(const nlf_ctx* c) { return c ? c->launches : -1; }

const char* nlf_last_error(const nlf_ctx* c) { return c ? c->err.c_str() : "null context"; }

void nlf_destroy(nlf_ctx* c)
{
    if (!c) return;
    if (c->stream || c->ready) cudaStreamSynchronize(c->stream);
    drop_plans(c);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->done) cudaEventDestroy(c->done);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    if (c->aux2) cudaStreamDestroy(c->aux2);
    if (c->join2) cudaEventDestroy(c->join2);
    if (c->owned && c->base) cudaFree(c->base);
    delete c;
}

}  // extern "C"
