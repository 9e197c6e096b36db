// apx_spectra.cu -- kernel preparation of the FFT core (Section IV
// "Initialization": the kernel is prepared once per request).
//
// CTAs 0..G-1: the FP32 spectrum H[k] = FFT_n(taps)[k] / (4m), k in [0, m],
// n = W_block = 2m, as a direct DFT split over the GPU: each CTA owns a few
// frequencies, each thread a strided subset of the taps (held in registers;
// twiddles advanced by a complex recurrence from the table), partial sums
// combined by a tree reduction.
// CTA G: the kernel statistics (||k||_inf, second moment) and the exact
// ||kbar||_1 of every packing candidate, for the selection in the block kernel.
// The block kernel is this launch's programmatic dependent.
#include "apx_block.cuh"
#include "apx_launch.h"

namespace apx {

constexpr int kSpecThreads = 256;
constexpr int kSpecChunk = 16;  // taps per thread loaded together

__global__ void __launch_bounds__(kSpecThreads) k_spec(const Params p) {
    __shared__ float2 part[kSpecThreads / 32][kSpecFreqs];
    __shared__ Shared sh;
    pdl_trigger();
    const int m = p.Wb / 2, n = p.Wb;
    const int nfreq_ctas = (m + 1 + kSpecFreqs - 1) / kSpecFreqs;
    if ((int)blockIdx.x == nfreq_ctas) {
        const KStats ks = kernel_stats(p, sh);
        double l1s[kMaxCand] = {0.0, 0.0, 0.0};
        const bool ok = !ks.bad && ks.Mk > 0.f;
        for (int c = 0; c < p.ncand; ++c)
            if (ok) l1s[c] = (double)kbar_l1(p, p.cand[c], compand_factor(p.cand[c].K, ks.Mk), sh);
        if (threadIdx.x == 0) {
            KInfo o;
            o.Mk = ks.Mk;
            o.bad = ks.bad;
            o.sig2k = ks.sig2k;
            for (int c = 0; c < kMaxCand; ++c) o.l1[c] = l1s[c];
            *p.ki = o;
        }
        return;
    }
    const int k0 = blockIdx.x * kSpecFreqs;
    float2 acc[kSpecFreqs], w[kSpecFreqs], st[kSpecFreqs];
#pragma unroll
    for (int f = 0; f < kSpecFreqs; ++f) {
        const int k = min(k0 + f, m);
        w[f] = __ldg(&p.tw32[(int)(((long long)threadIdx.x * k) & (n - 1))]);      // W^(t k)
        st[f] = __ldg(&p.tw32[(int)(((long long)kSpecThreads * k) & (n - 1))]);    // W^(NT k)
        acc[f] = make_float2(0.f, 0.f);
    }
    for (int u0 = 0; u0 * kSpecThreads < p.N; u0 += kSpecChunk) {
        float h[kSpecChunk];
#pragma unroll
        for (int u = 0; u < kSpecChunk; ++u) h[u] = ktap(p, threadIdx.x + (u0 + u) * kSpecThreads);
#pragma unroll
        for (int u = 0; u < kSpecChunk; ++u) {
#pragma unroll
            for (int f = 0; f < kSpecFreqs; ++f) {
                acc[f].x = fmaf(h[u], w[f].x, acc[f].x);
                acc[f].y = fmaf(h[u], w[f].y, acc[f].y);
                w[f] = cmul(w[f], st[f]);
            }
        }
    }
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
    if (threadIdx.x < kSpecFreqs && k0 + (int)threadIdx.x <= m) {
        float x = 0.f, y = 0.f;
#pragma unroll
        for (int wi = 0; wi < kSpecThreads / 32; ++wi) { x += part[wi][threadIdx.x].x; y += part[wi][threadIdx.x].y; }
        const float scale = 1.f / (float)(4 * m);
        p.Hfull[k0 + threadIdx.x] = make_float2(x * scale, y * scale);
    }
}

cudaError_t launch_spec(const Params& p, cudaStream_t st) {
    const int m = p.Wb / 2;
    const int grid = (m + 1 + kSpecFreqs - 1) / kSpecFreqs + 1;
    return launch_k(k_spec, dim3(grid), dim3(kSpecThreads), 0, st, false, p);
}

}  // namespace apx
