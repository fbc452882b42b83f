// dft_accum.cuh -- the accumulation step of the running DFT, shared by the
// single-grid and the batched flush kernels.
//
// acc[r][f] += sum_s sample[s][r] exp(i phase[s][f]) for the buffered samples
// of RCH records at the block's ACC_NT frequencies: FP32 products within one
// block of samples, FP64 accumulation.  The block stages the samples and the
// E phases (cos, sin of w n dt) in shared memory; the H sum, whose phase is
// w (n - 1/2) dt, is taken with the E phases and turned by exp(-i w dt / 2)
// once per record.  On this part FP64 runs at a small fraction of the FP32
// rate and bounds the flush, so FP64 is kept to the accumulator additions.
// The FP64 accumulators are read for G records before any is written back,
// so that G read-modify-writes are in flight per thread.  The sample rows
// (RCH floats per sample) start on 16-byte boundaries.
#pragma once

#include "nlf_internal.h"

namespace nlf {

constexpr int ACC_NT = 128;   // frequencies (threads) per block
constexpr int ACC_NCH = 8;    // record chunks per block of a single grid

template <int B, int RCH>
struct alignas(16) AccShared {
    float sE[B][RCH];
    float sH[B][RCH];
    float2 ph[B][ACC_NT];
};

// G = 4 records at a time of one chunk at frequency f (thread t of the
// block).  The sample loop is outside the record loop, so each phase is read
// from shared memory once per G records, and the G records' samples arrive
// as broadcast float4 loads; every record still sums its samples in order
// s = 0 .. B-1.  Records past the chunk's end hold zero samples and are not
// stored.
template <int B, int RCH>
__device__ __forceinline__ void accum_chunk(const DftParams& d, long long r0, int f, int t, float cr, float sr,
                                            const AccShared<B, RCH>& sm)
{
    constexpr int G = 4;
    static_assert(RCH % G == 0, "record chunk must hold whole groups");
    const int rmax = (int)min((long long)RCH, d.nrec + 1 - r0);
    for (int g = 0; g < rmax; g += G) {
        double2 ae[G], ah[G];
#pragma unroll
        for (int u = 0; u < G; ++u) {
            ae[u] = ah[u] = make_double2(0.0, 0.0);
            if (g + u < rmax) {
                const long long o = (r0 + g + u) * d.nf + f;
                if (NLF_IN(d, 20, o, (d.nrec + 1) * d.nf)) {
                    ae[u] = d.accE[o];
                    ah[u] = d.accH[o];
                }
            }
        }
        float er[G], ei[G], hr[G], hi[G];
#pragma unroll
        for (int u = 0; u < G; ++u) er[u] = ei[u] = hr[u] = hi[u] = 0.f;
#pragma unroll 8
        for (int s = 0; s < B; ++s) {
            const float2 p = sm.ph[s][t];
            const float4 e4 = *reinterpret_cast<const float4*>(&sm.sE[s][g]);
            const float4 h4 = *reinterpret_cast<const float4*>(&sm.sH[s][g]);
            const float e[G] = {e4.x, e4.y, e4.z, e4.w}, h[G] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
            for (int u = 0; u < G; ++u) {
                er[u] = fmaf(e[u], p.x, er[u]);
                ei[u] = fmaf(e[u], p.y, ei[u]);
                hr[u] = fmaf(h[u], p.x, hr[u]);
                hi[u] = fmaf(h[u], p.y, hi[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < G; ++u) {
            if (g + u < rmax && NLF_IN(d, 20, (r0 + g + u) * d.nf + f, (d.nrec + 1) * d.nf)) {
                const long long o = (r0 + g + u) * d.nf + f;
                ae[u].x += (double)er[u];
                ae[u].y += (double)ei[u];
                // the turn by exp(-i w dt / 2) acts on the FP32 block sum in FP32
                // (its rounding is that of the sum itself); only the two
                // additions to the accumulator are FP64, the slow pipe here
                ah[u].x += (double)fmaf(cr, hr[u], sr * hi[u]);
                ah[u].y += (double)fmaf(cr, hi[u], -sr * hr[u]);
                d.accE[o] = ae[u];
                d.accH[o] = ah[u];
            }
        }
    }
}

// Records rb .. rb + nchunk RCH - 1 (in chunks of RCH), frequencies
// f0 .. f0+ACC_NT-1 of one context.  The phases are staged once per block,
// the samples once per chunk.
template <int B, int RCH>
__device__ __forceinline__ void accum_block(const DftParams& d, long long rb, int nchunk, int f0,
                                            AccShared<B, RCH>& sm)
{
    if (!NLF_CTX(d)) return;        // (uniform over the block)
    const int t = threadIdx.x;
    for (int q = t; q < B * ACC_NT; q += blockDim.x) {
        const int s = q / ACC_NT, u = q - s * ACC_NT;
        float2 v = make_float2(0.f, 0.f);
        if (f0 + u < d.nf && NLF_IN(d, 21, (long long)s * d.nf + f0 + u, (long long)d.B * d.nf)) {
            const float4 w = d.phase[s * d.nf + f0 + u];
            v = make_float2(w.x, w.y);
        }
        sm.ph[s][u] = v;
    }
    const int f = f0 + t;
    double sr = 0.0, cr = 1.0;
    if (f < d.nf) sincos(0.5 * d.omega[f] * d.dt, &sr, &cr);
    const float crf = (float)cr, srf = (float)sr;
    const long long nr = d.nrec + 1;
    for (int ch = 0; ch < nchunk; ++ch) {
        const long long r0 = rb + (long long)ch * RCH;
        if (r0 >= nr) break;
        __syncthreads();   // the previous chunk's samples are no longer read
        for (int q = t; q < B * RCH; q += blockDim.x) {
            const int s = q / RCH, rr = q - s * RCH;
            const long long r = r0 + rr;
            const bool ok = r < nr && NLF_IN(d, 21, (long long)s * nr + r, (long long)d.B * nr);
            sm.sE[s][rr] = ok ? d.sE[(long long)s * nr + r] : 0.f;
            sm.sH[s][rr] = ok ? d.sH[(long long)s * nr + r] : 0.f;
        }
        __syncthreads();
        if (f < d.nf) accum_chunk<B, RCH>(d, r0, f, t, crf, srf, sm);
    }
}
}  // namespace nlf
