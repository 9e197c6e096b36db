// apx_spectra.cu -- kernel preparation of the FFT core (Section IV
// "Initialization": the kernel is prepared once per request).
//
// CTA 0: the FP32 spectrum H[k] = FFT_n(taps)[k] / (4m), k in [0, m],
// n = W_block = 2m, through the shared-memory FFT on 1024 threads (radix-4 or
// radix-8 passes, one butterfly per thread).
// CTA 1: the kernel statistics (||k||_inf, second moment) and the exact
// ||kbar||_1 of every packing candidate, for the selection in the block kernel.
// Two SMs busy; the block kernel, launched as this launch's programmatic
// dependent, fills the rest of the GPU meanwhile.
#include "apx_block.cuh"
#include "apx_launch.h"

namespace apx {

__global__ void __launch_bounds__(kSpecThreads) k_spec(const Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    pdl_trigger();
    if (blockIdx.x == 1) {
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
    auto tap = [&](int n) -> float { return ktap(p, n); };
    spectrum_of<float>(tap, p.Wb, p.Wb, p.tw32, p.Hfull, reinterpret_cast<float2*>(smem));
}

cudaError_t launch_spec(const Params& p, cudaStream_t st) {
    static int attr_dev = -1;
    int dev;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_spec, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const size_t smem = sizeof(float2) * padded_len(p.Wb / 2);
    return launch_k(k_spec, dim3(2), dim3(kSpecThreads), smem, st, false, p);
}

}  // namespace apx
