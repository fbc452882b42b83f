// dft_accum.cuh -- the accumulation step of the running DFT, shared by the
// single-grid and the batched flush kernels.
//
// acc[r][f] += sum_s sample[s][r] exp(i phase[s][f]) for the buffered samples
// of RCH records (staged in shared memory by the caller) at frequency f:
// FP32 products within one block of samples, FP64 accumulation.  The FP64
// accumulators are read for G records before any is written back, so that G
// read-modify-writes are in flight per thread instead of one.
#pragma once

#include "nlf_internal.h"

namespace nlf {

template <int B, int RCH>
__device__ __forceinline__ void accum_records(const DftParams& d, long long r0, int f, const float (*sE)[RCH],
                                              const float (*sH)[RCH])
{
    constexpr int G = B <= 16 ? 8 : 4;
    const long long nr = d.nrec + 1;
    float ce[B], se[B], ch[B], sh[B];
#pragma unroll
    for (int s = 0; s < B; ++s) {
        const float4 v = d.phase[s * d.nf + f];
        ce[s] = v.x;
        se[s] = v.y;
        ch[s] = v.z;
        sh[s] = v.w;
    }
    const int rmax = (int)min((long long)RCH, nr - r0);
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
                    const float e = sE[s][rr], h = sH[s][rr];
                    er = fmaf(e, ce[s], er);
                    ei = fmaf(e, se[s], ei);
                    hr = fmaf(h, ch[s], hr);
                    hi = fmaf(h, sh[s], hi);
                }
                const long long o = (r0 + rr) * d.nf + f;
                ae[u].x += (double)er;
                ae[u].y += (double)ei;
                ah[u].x += (double)hr;
                ah[u].y += (double)hi;
                d.accE[o] = ae[u];
                d.accH[o] = ah[u];
            }
        }
    }
}

}  // namespace nlf
