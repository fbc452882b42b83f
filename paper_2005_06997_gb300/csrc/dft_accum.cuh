// dft_accum.cuh -- the accumulation step of the running DFT, shared by the
// single-grid and the batched flush kernels.
//
// acc[r][f] += sum_s sample[s][r] exp(i phase[s][f]) for the buffered samples
// of RCH records at the block's ACC_NT frequencies: FP32 products within one
// block of samples, FP64 accumulation.  The block stages the samples and the
// E phases (cos, sin of w n dt) in shared memory; the H sum, whose phase is
// w (n - 1/2) dt, is taken with the E phases and turned by exp(-i w dt / 2)
// once per record.  The FP64 accumulators are read for G records before any
// is written back, so that G read-modify-writes are in flight per thread.
#pragma once

#include "nlf_internal.h"

namespace nlf {

constexpr int ACC_NT = 128;   // frequencies (threads) per block
constexpr int ACC_NCH = 8;    // record chunks per block of a single grid

template <int B, int RCH>
struct AccShared {
    float sE[B][RCH];
    float sH[B][RCH];
    float2 ph[B][ACC_NT];
};

// G records at a time of one chunk at frequency f (thread t of the block).
template <int B, int RCH>
__device__ __forceinline__ void accum_chunk(const DftParams& d, long long r0, int f, int t, double cr, double sr,
                                            const AccShared<B, RCH>& sm)
{
    constexpr int G = 8;
    const int rmax = (int)min((long long)RCH, d.nrec + 1 - r0);
    for (int g = 0; g < rmax; g += G) {
        double2 ae[G], ah[G];
#pragma unroll
        for (int u = 0; u < G; ++u) {
            if (g + u < rmax) {
                const long long o = (r0 + g + u) * d.nf + f;
                ae[u] = d.accE[o];
                ah[u] = d.accH[o];
            }
        }
#pragma unroll
        for (int u = 0; u < G; ++u) {
            if (g + u < rmax) {
                const int rr = g + u;
                float er = 0.f, ei = 0.f, hr = 0.f, hi = 0.f;
#pragma unroll
                for (int s = 0; s < B; ++s) {
                    const float2 p = sm.ph[s][t];
                    const float e = sm.sE[s][rr], h = sm.sH[s][rr];
                    er = fmaf(e, p.x, er);
                    ei = fmaf(e, p.y, ei);
                    hr = fmaf(h, p.x, hr);
                    hi = fmaf(h, p.y, hi);
                }
                const long long o = (r0 + rr) * d.nf + f;
                ae[u].x += (double)er;
                ae[u].y += (double)ei;
                ah[u].x += cr * (double)hr + sr * (double)hi;
                ah[u].y += cr * (double)hi - sr * (double)hr;
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
    const int t = threadIdx.x;
    for (int q = t; q < B * ACC_NT; q += blockDim.x) {
        const int s = q / ACC_NT, u = q - s * ACC_NT;
        float2 v = make_float2(0.f, 0.f);
        if (f0 + u < d.nf) {
            const float4 w = d.phase[s * d.nf + f0 + u];
            v = make_float2(w.x, w.y);
        }
        sm.ph[s][u] = v;
    }
    const int f = f0 + t;
    double sr = 0.0, cr = 1.0;
    if (f < d.nf) sincos(0.5 * d.omega[f] * d.dt, &sr, &cr);
    const long long nr = d.nrec + 1;
    for (int ch = 0; ch < nchunk; ++ch) {
        const long long r0 = rb + (long long)ch * RCH;
        if (r0 >= nr) break;
        __syncthreads();   // the previous chunk's samples are no longer read
        for (int q = t; q < B * RCH; q += blockDim.x) {
            const int s = q / RCH, rr = q - s * RCH;
            const long long r = r0 + rr;
            sm.sE[s][rr] = r < nr ? d.sE[(long long)s * nr + r] : 0.f;
            sm.sH[s][rr] = r < nr ? d.sH[(long long)s * nr + r] : 0.f;
        }
        __syncthreads();
        if (f < d.nf) accum_chunk<B, RCH>(d, r0, f, t, cr, sr, sm);
    }
}
}  // namespace nlf
