// apx_spectra.cu -- the FP32 kernel spectrum of the FFT core (Section IV
// "Initialization": the kernel is prepared once per request).
//
// H[k] = FFT_n(taps)[k] / (4m), k in [0, m], n = W_block = 2m real points, as a
// direct DFT split over many CTAs: each CTA owns a few frequencies, each thread
// a strided subset of the taps (twiddles advanced by a complex recurrence from
// the table), partial sums combined by a tree reduction.  With N taps this is
// N (m+1) complex multiply-adds spread over the whole GPU, which finishes well
// before the block kernel (launched as its programmatic dependent) needs it.
#include "apx_block.cuh"
#include "apx_launch.h"

namespace apx {

constexpr int kSpecThreads = 256;

__global__ void __launch_bounds__(kSpecThreads) k_spec(const Params p) {
    __shared__ float2 part[kSpecThreads / 32][kSpecFreqs];
    pdl_trigger();
    const int m = p.Wb / 2, n = p.Wb;
    const int k0 = blockIdx.x * kSpecFreqs;
    float2 acc[kSpecFreqs], w[kSpecFreqs], st[kSpecFreqs];
    const int t0 = threadIdx.x;
    const float h0 = ktap(p, t0);  // t0 < N handled by ktap (zero past N)
#pragma unroll
    for (int f = 0; f < kSpecFreqs; ++f) {
        const int k = min(k0 + f, m);
        w[f] = __ldg(&p.tw32[(int)(((long long)t0 * k) & (n - 1))]);               // W^(t0 k)
        st[f] = __ldg(&p.tw32[(int)(((long long)kSpecThreads * k) & (n - 1))]);    // W^(NT k)
        acc[f] = make_float2(0.f, 0.f);
    }
    float h = h0;
    for (int t = t0; t < p.N; t += kSpecThreads) {
        const float hn = ktap(p, t + kSpecThreads);
#pragma unroll
        for (int f = 0; f < kSpecFreqs; ++f) {
            acc[f].x = fmaf(h, w[f].x, acc[f].x);
            acc[f].y = fmaf(h, w[f].y, acc[f].y);
            w[f] = cmul(w[f], st[f]);
        }
        h = hn;
    }
    // tree reduction over the CTA
#pragma unroll
    for (int f = 0; f < kSpecFreqs; ++f) {
        float x = acc[f].x, y = acc[f].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5][f] = make_float2(x, y);
    }
    __syncthreads();
    if (threadIdx.x < kSpecFreqs && k0 + threadIdx.x <= m) {
        float x = 0.f, y = 0.f;
#pragma unroll
        for (int wi = 0; wi < kSpecThreads / 32; ++wi) { x += part[wi][threadIdx.x].x; y += part[wi][threadIdx.x].y; }
        const float scale = 1.f / (float)(4 * m);
        p.Hfull[k0 + threadIdx.x] = make_float2(x * scale, y * scale);
    }
}

cudaError_t launch_spec(const Params& p, cudaStream_t st) {
    const int m = p.Wb / 2;
    const int grid = (m + 1 + kSpecFreqs - 1) / kSpecFreqs;
    return launch_k(k_spec, dim3(grid), dim3(kSpecThreads), 0, st, false, p);
}

}  // namespace apx
