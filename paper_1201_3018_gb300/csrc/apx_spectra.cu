// apx_spectra.cu -- kernel spectra of the FFT core (Section IV "Initialization":
// the kernel is prepared once per request).
//
// CTA 0 transforms the FP32 taps (reversed for cross-correlation); it needs
// nothing from the selection pass and runs while that pass is still working.
// CTA 1 + c transforms the packed taps of candidate c (Eq. 5 with the pair
// order k~[2n+1] + eps^-1 k~[2n], or k~ for asymmetric packing), and only if
// some block selected candidate c.  Every CTA waits for the selection pass
// before it exits, so this grid's completion implies that pass's.
#include "apx_block.cuh"
#include "apx_launch.h"

namespace apx {

// H = FFT_n(taps) / (4m), k in [0, m], natural order; tap(j) gives tap j.
template <typename R, typename C, typename F>
__device__ void spectrum_of(F tap, int Wb, int n, const C* __restrict__ tw, C* H, C* Z) {
    const int m = n / 2;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        C v;
        v.x = tap(2 * j);
        v.y = tap(2 * j + 1);
        Z[pad16(j)] = v;
    }
    __syncthreads();
    fft_smem<C, false>(Z, m, tw, Wb);
    const R scale = (R)1 / (R)(8 * m);
    for (int k = threadIdx.x; k <= m; k += blockDim.x) {
        C X;
        if (k == 0 || k == m) {
            const C z0 = Z[0];
            X.x = 2 * (k == 0 ? z0.x + z0.y : z0.x - z0.y);
            X.y = 0;
        } else {
            C Xmk;
            real_post(Z[pad16(fft_perm(k, m))], Z[pad16(fft_perm(m - k, m))], __ldg(&tw[k * (Wb / n)]), X, Xmk);
        }
        X.x *= scale; X.y *= scale;
        H[k] = X;
    }
}

__global__ void __launch_bounds__(512) k_spectra(const Params p, float2* Hfull, double2* H0, double2* H1,
                                                 double2* H2) {
    extern __shared__ __align__(16) unsigned char smem[];
    pdl_trigger();
    const int job = blockIdx.x;
    if (job == 0) {
        auto tap = [&](int n) -> float { return ktap(p, n); };
        spectrum_of<float>(tap, p.Wb, p.Wb, p.tw32, Hfull, reinterpret_cast<float2*>(smem));
        if (threadIdx.x == 0) *p.used_next = 0u;
        pdl_wait();
        return;
    }
    pdl_wait();  // selection complete: `used` and the published kernel statistics are final
    const int c = job - 1;
    if (c >= p.ncand || !(*p.used & (1u << c))) return;
    const Cand& cd = p.cand[c];
    const float ck = compand_factor(cd.K, p.ki->Mk);
    auto tap = [&](int n) -> double { return (double)kbar_int(p, cd, ck, n); };
    double2* Hc = c == 0 ? H0 : (c == 1 ? H1 : H2);
    const int n = cd.blk == APX_BLK_SYM ? p.Wb / 2 : p.Wb;
    spectrum_of<double>(tap, p.Wb, n, p.tw64, Hc, reinterpret_cast<double2*>(smem));
}

cudaError_t launch_spectra(const Params& p, float2* Hfull, double2* Hc[kMaxCand], cudaStream_t st) {
    static int attr_dev = -1;
    int dev;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const size_t smem = sizeof(double2) * padded_len(p.Wb / 2);
    return launch_k(k_spectra, dim3(1 + p.ncand), dim3(fft_threads(p.Wb)), smem, st, true, p, Hfull, Hc[0], Hc[1],
                    Hc[2]);
}

}  // namespace apx
