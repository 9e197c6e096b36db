// apx_spectra.cu -- kernel preparation of the FFT core (Section IV
// "Initialization": the kernel is prepared once per request).
//
// The FP32 spectrum H[k] = FFT_n(taps)[k] / (4m), k in [0, m], n = W_block = 2m,
// in two small launches that run ahead of the block kernel:
//   k_spec:   CTA r < R1 transforms the decimated taps h[r], h[r+R1], ... (n/R1
//             points) in shared memory: Y_r = FFT_{n/R1}(h[r::R1]);
//             CTA R1 publishes the kernel statistics (||k||_inf, second moment)
//             and the exact ||kbar||_1 of every packing candidate.
//   k_combine: H[k] = sum_{r < R1} W_n^(r k) Y_r[k mod n/R1]  (the last
//             decimation-in-time stage), one thread per frequency.
// Each launch is the programmatic dependent of the one before it; the block
// kernel waits for k_combine only where it multiplies by H.
#include "apx_block.cuh"
#include "apx_launch.h"

namespace apx {

template <bool BATCH>
__global__ void __launch_bounds__(kSpecThreads) k_spec(const Params p0, const BatchTab bt) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ Params sp;
    pdl_trigger();
    const int cta = BATCH ? (int)batch_enter(bt, sp) : (int)blockIdx.x;
    const Params& p = BATCH ? sp : p0;
    const int n = p.Wb, R1 = spec_r1(n), ns = n / R1;
    if (cta == R1) {
        const KStats ks = kernel_stats(p, sh);
        double l1s[kMaxCand] = {0.0, 0.0, 0.0};
        const bool ok = !ks.bad && ks.Mk > 0.f;
        for (int c = 0; c < p.ncand; ++c) {
            // Under per-block selection a candidate whose model SNR misses the target even for
            // the best window (second moment = squared maximum; the model depends on the window
            // only through that ratio) is never chosen: skip its norm (1 % margin for rounding).
            const bool reachable = !p.autosel || snr_feasible(1.0, 1.f, ks.sig2k, ks.Mk, p.cand[c].S, p.cand[c].K,
                                                              __dmul_rn(p.thr, 1.01));
            if (ok && reachable) l1s[c] = (double)kbar_l1(p, p.cand[c], compand_factor(p.cand[c].K, ks.Mk), sh);
        }
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
    const int r = cta;
    float2* Z = reinterpret_cast<float2*>(smem);
    for (int j = threadIdx.x; j < ns; j += blockDim.x) Z[pad16(j)] = make_float2(ktap(p, r + j * R1), 0.f);
    __syncthreads();
    fft_smem<float2, false>(Z, ns, p.tw32, p.ntab, p.status);
    for (int k = threadIdx.x; k < ns; k += blockDim.x) p.Ysub[r * ns + k] = Z[pad16(fft_perm<float2>(k, ns))];
}

template <bool BATCH>
__global__ void __launch_bounds__(256) k_combine(const Params p0, const BatchTab bt) {
    __shared__ Params sp;
    pdl_trigger();
    const int cta = BATCH ? (int)batch_enter(bt, sp) : (int)blockIdx.x;
    const Params& p = BATCH ? sp : p0;
    pdl_wait();  // the decimated sub-spectra
    const int n = p.Wb, m = n / 2, R1 = spec_r1(n), ns = n / R1;
    const int k = cta * blockDim.x + threadIdx.x;
    if (k > m) return;
    float2 acc = make_float2(0.f, 0.f);
    const int kk = k & (ns - 1);
    float2 y[16], w[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        if (r < R1) {
            y[r] = __ldcg(&p.Ysub[r * ns + kk]);
            w[r] = __ldg(&p.tw32[(r * k * (p.ntab / n)) & (p.ntab - 1)]);
        }
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        if (r < R1) {
            acc.x = fmaf(y[r].x, w[r].x, fmaf(-y[r].y, w[r].y, acc.x));
            acc.y = fmaf(y[r].x, w[r].y, fmaf(y[r].y, w[r].x, acc.y));
        }
    }
    const float scale = 1.f / (float)(4 * m);
    p.Hfull[k] = make_float2(acc.x * scale, acc.y * scale);
}

cudaError_t launch_spec(const Params& p, cudaStream_t st) {
    const int n = p.Wb, R1 = spec_r1(n);
    const size_t smem = sizeof(float2) * padded_len(n / R1);
    const BatchTab none = {nullptr, nullptr, 0};
    return launch_k(k_spec<false>, dim3(R1 + 1), dim3(kSpecThreads), smem, st, false, p, none);
}

cudaError_t launch_spec_combine(const Params& p, cudaStream_t st) {
    const int m = p.Wb / 2;
    const BatchTab none = {nullptr, nullptr, 0};
    return launch_k(k_combine<false>, dim3((m + 1 + 255) / 256), dim3(256), 0, st, true, p, none);
}

int spec_ctas(int Wb) { return spec_r1(Wb) + 1; }
int combine_ctas(int Wb) { return (Wb / 2 + 1 + 255) / 256; }

cudaError_t launch_spec_batch(const Params& any, const BatchTab& bt, int ctas, cudaStream_t st, bool pdl) {
    const int n = any.Wb, R1 = spec_r1(n);
    const size_t smem = sizeof(float2) * padded_len(n / R1);
    return launch_k(k_spec<true>, dim3(ctas), dim3(kSpecThreads), smem, st, pdl, any, bt);
}

cudaError_t launch_combine_batch(const Params& any, const BatchTab& bt, int ctas, cudaStream_t st) {
    return launch_k(k_combine<true>, dim3(ctas), dim3(256), 0, st, true, any, bt);
}

}  // namespace apx
