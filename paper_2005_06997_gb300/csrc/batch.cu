// batch.cu -- many independent grids advanced together.
//
// A batch step is one launch per kernel over the concatenated work of every
// active instance: the step kernels take one block per (instance, tile, z
// chunk) item of the joint work list (heaviest instances first) and run the
// same tile code as the single-grid step; the material sites and the TF/SF
// items of all instances are one thread each over their joint lists.  The
// monitor work of all instances is
// batched the same way (one gather launch per sample, one phase and one
// accumulation launch per block of samples).  The host captures a whole DFT
// period of these launches in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>

#include "nlf_internal.h"
#include "dft_accum.cuh"

namespace nlf {

// The first q with end[q] > w (end: inclusive prefix sums).
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

// One FP32 sample of every record of every instance into slot `slot`.
__global__ void k_gather_batch(const BatchDft a, int slot)
{
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = a.rec_end[a.n - 1];
    if (w >= total) return;
    const int q = find_inst(a.rec_end, a.n, w);
    const BatchDftInst& I = a.inst[q];
    const long long r = w - (q > 0 ? a.rec_end[q - 1] : 0);
    const int cur = I.base_par ^ a.cur_par;
    const DftParams& d = I.d;
    if (!NLF_CTX(d)) return;
    float e, h;
    if (r < d.nrec) {
        const uint32_t oe = d.rec_e[r], o = d.rec_h[r], hs = d.rec_hs[r];
        if (!(NLF_IN(d, 17, oe, d.nfield3) && NLF_IN(d, 18, (long long)o + hs, d.nfield3))) return;
        e = __ldg(I.E[cur] + oe);
        h = 0.5f * (__ldg(I.H[cur] + o) + __ldg(I.H[cur] + o + hs));
    } else {
        e = I.e_inc[cur][d.inc_node];
        h = 0.5f * (I.h_inc[cur][d.inc_node - 1] + I.h_inc[cur][d.inc_node]);
        d.sample_step[slot] = *I.step[cur];
    }
    const long long o = (long long)slot * (d.nrec + 1) + r;
    if (!NLF_IN(d, 19, o, (long long)d.B * (d.nrec + 1))) return;
    d.sE[o] = e;
    d.sH[o] = h;
    if (!isfinite(e) || !isfinite(h)) atomicOr(I.err, 1);
}

__global__ void k_phase_batch(const BatchDft a, int count)
{
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = a.ph_end[a.n - 1];
    if (w >= total) return;
    const int q = find_inst(a.ph_end, a.n, w);
    const DftParams& d = a.inst[q].d;
    if (!NLF_CTX(d)) return;
    const long long t = w - (q > 0 ? a.ph_end[q - 1] : 0);
    const int s = (int)(t / d.nf), f = (int)(t - (long long)s * d.nf);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < count) {
        const double n = (double)d.sample_step[s];
        const double om = d.omega[f];
        double se, ce, sh, ch;
        sincos(om * n * d.dt, &se, &ce);
        sincos(om * (n - 0.5) * d.dt, &sh, &ch);
        v = make_float4((float)ce, (float)se, (float)ch, (float)sh);
    }
    d.phase[t] = v;
}

// Same arithmetic as the single-grid accumulation: per group of
// NLF_BATCH_GROUP record chunks and per frequency chunk, FP32 sums over the
// B samples added into FP64; the phases a block stages serve the whole group.
template <int B, int RCH>
__global__ void __launch_bounds__(ACC_NT) k_accum_batch(const BatchDft a)
{
    __shared__ AccShared<B, RCH> sm;
    const long long w = blockIdx.x;
    const int q = find_inst(a.chunk_end, a.n, w);
    const DftParams& d = a.inst[q].d;
    const int f0 = blockIdx.y * ACC_NT;
    if (f0 >= d.nf) return;
    accum_block<B, RCH>(d, (w - (q > 0 ? a.chunk_end[q - 1] : 0)) * RCH * NLF_BATCH_GROUP, NLF_BATCH_GROUP, f0, sm);
}

void launch_gather_batch(const BatchDft& a, long long total_records, int slot, cudaStream_t st)
{
    k_gather_batch<<<(unsigned)((total_records + 255) / 256), 256, 0, st>>>(a, slot);
}

void launch_flush_batch(const BatchDft& a, long long total_phase, long long total_chunks, int max_nf, int B,
                        int count, cudaStream_t st)
{
    k_phase_batch<<<(unsigned)((total_phase + 255) / 256), 256, 0, st>>>(a, count);
    dim3 grd((unsigned)total_chunks, (max_nf + ACC_NT - 1) / ACC_NT);
    if (B <= 8)
        k_accum_batch<8, NLF_BATCH_RCH><<<grd, ACC_NT, 0, st>>>(a);
    else if (B <= 16)
        k_accum_batch<16, NLF_BATCH_RCH><<<grd, ACC_NT, 0, st>>>(a);
    else
        k_accum_batch<32, NLF_BATCH_RCH><<<grd, ACC_NT, 0, st>>>(a);
}

}  // namespace nlf
