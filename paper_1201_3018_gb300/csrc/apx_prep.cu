// apx_prep.cu -- per-request kernel preparation (Section IV "Initialization"):
// ||k||_inf, the kernel's second moment, the FP32 taps (reversed for
// cross-correlation, padded), and for every packing candidate the companded
// (Eq. 2) and packed (Eq. 5, kernel pair order k~[2n+1] + eps^-1 k~[2n]) taps
// with their exact l1 norm.  The FFT core also needs kernel spectra; those are
// computed only for the candidates that some block actually selected.
#include "apx_block.cuh"
#include "apx_launch.h"

namespace apx {

__global__ void __launch_bounds__(kPrepThreads) k_prep(const Params p, const float* __restrict__ k, int xcorr,
                                                       KInfo* ki, float* kfull, double* kb0, double* kb1,
                                                       double* kb2) {
    __shared__ Shared sh;
    if (threadIdx.x == 0 && p.used) *p.used = 0u;
    const int N = p.N, Nodd = p.Nodd;
    auto kr = [&](int n) -> float { return n < N ? __ldg(&k[xcorr ? N - 1 - n : n]) : 0.f; };

    float m = 0.f;
    int bad = 0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        float a = fabsf(kr(n));
        if (!(a <= 3.402823466e38f)) bad = 1;
        m = fmaxf(m, a);
    }
    m = block_reduce<float, true>(m, sh.redf);
    bad = block_reduce<int, true>(bad, sh.redi);

    const int nkp32 = (Nodd + 7) / 8 * 8;
    for (int n = threadIdx.x; n < nkp32; n += blockDim.x) kfull[n] = kr(n);

    double sig2 = 0.0;
    const bool ok = !bad && m > 0.f;
    if (ok) {
        int e;
        (void)frexpf(m, &e);
        const int shf = 24 - e;
        long long acc = 0;
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            long long q = __float2ll_rz(ldexpf(kr(n), shf));
            acc += q * q;
        }
        acc = block_reduce<long long, false>(acc, sh.redl);
        sig2 = __ddiv_rn(ldexp(__ll2double_rn(acc), -2 * shf), (double)N);
    }

    double* kbs[kMaxCand] = {kb0, kb1, kb2};
    float cks[kMaxCand] = {0.f, 0.f, 0.f};
    double l1s[kMaxCand] = {0.0, 0.0, 0.0};
    for (int c = 0; c < p.ncand; ++c) {
        const Cand& cd = p.cand[c];
        const float ck = ok ? compand_factor(cd.K, m) : 0.f;          // Eq. (2)
        auto kq = [&](int n) -> long long { return (ok && n < N) ? (long long)compand(ck, kr(n)) : 0ll; };
        const int nkp = (cd.nk + 3) / 4 * 4;
        long long l1 = 0;
        for (int t = threadIdx.x; t < nkp; t += blockDim.x) {
            long long v = 0;
            if (t < cd.nk) {
                if (cd.blk == APX_BLK_SYM) v = kq(2 * t + 1) + (kq(2 * t) << cd.b);  // Eq. (5), reading c2
                else v = kq(t);
            }
            kbs[c][t] = (double)v;
            l1 += v < 0 ? -v : v;
        }
        l1 = block_reduce<long long, false>(l1, sh.redl);
        cks[c] = ck;
        l1s[c] = (double)l1;
    }
    if (threadIdx.x == 0) {
        KInfo o;
        o.Mk = m;
        o.nonfinite = bad;
        o.sig2k = sig2;
        for (int c = 0; c < kMaxCand; ++c) { o.ck[c] = cks[c]; o.l1[c] = l1s[c]; }
        o.pad_ = 0.f;
        *ki = o;
    }
}

// Kernel spectra for the FFT core: H = FFT_n(taps) / (4m) for k in [0, m].
// CTA 0: FP32 taps (full precision); CTA 1 + c: packed taps of candidate c.
// A spectrum nobody selected is skipped.
template <typename R, typename C, int MAXB>
__device__ void spectrum_of(const R* taps, int ntaps, int Wb, int n, const C* __restrict__ tw, C* H, C* z) {
    const int m = n / 2;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        C v;
        v.x = 2 * j < ntaps ? taps[2 * j] : (R)0;
        v.y = 2 * j + 1 < ntaps ? taps[2 * j + 1] : (R)0;
        z[j] = v;
    }
    __syncthreads();
    fft_smem<C, false, MAXB>(z, m, tw, Wb / m);
    const R scale = (R)1 / (R)(8 * m);
    for (int k = threadIdx.x; k <= m; k += blockDim.x) {
        C X;
        if (k == 0) { X.x = 2 * (z[0].x + z[0].y); X.y = 0; }
        else if (k == m) { X.x = 2 * (z[0].x - z[0].y); X.y = 0; }
        else {
            C Xmk;
            real_post(z[k], z[m - k], __ldg(&tw[k * (Wb / n)]), X, Xmk);
        }
        X.x *= scale; X.y *= scale;
        H[k] = X;
    }
}

template <int MAXB>
__global__ void __launch_bounds__(kFftThreads) k_spectra(const Params p, float2* Hfull, double2* H0, double2* H1,
                                                         double2* H2) {
    extern __shared__ __align__(16) unsigned char smem[];
    const unsigned used = *p.used;
    const int job = blockIdx.x;
    if (job == 0) {
        if (!(used & 8u)) return;
        spectrum_of<float, float2, MAXB>(p.kfull, p.Nodd, p.Wb, p.Wb, p.tw32, Hfull, reinterpret_cast<float2*>(smem));
        return;
    }
    const int c = job - 1;
    if (c >= p.ncand || !(used & (1u << c))) return;
    const Cand& cd = p.cand[c];
    double2* Hs[kMaxCand] = {H0, H1, H2};
    const int n = cd.blk == APX_BLK_SYM ? p.Wb / 2 : p.Wb;
    spectrum_of<double, double2, MAXB>(cd.kbar, cd.nk, p.Wb, n, p.tw64, Hs[c], reinterpret_cast<double2*>(smem));
}

cudaError_t launch_prep(const Params& p, const float* k, int xcorr, double* kbar_out[kMaxCand], KInfo* ki,
                        float* kfull, cudaStream_t st) {
    k_prep<<<1, kPrepThreads, 0, st>>>(p, k, xcorr, ki, kfull, kbar_out[0], kbar_out[1], kbar_out[2]);
    return cudaGetLastError();
}

int fft_maxb(int Wb) {
    int need = (Wb / 2) / (8 * kFftThreads);
    return need <= 1 ? 1 : (need <= 2 ? 2 : 4);
}

template <int MAXB>
static cudaError_t spectra_t(const Params& p, float2* Hfull, double2* Hc[kMaxCand], cudaStream_t st) {
    size_t smem = (size_t)8 * p.Wb;  // complex FP64 of length W_block/2
    static int attr_dev = -1;
    int dev;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_spectra<MAXB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    k_spectra<MAXB><<<1 + p.ncand, kFftThreads, smem, st>>>(p, Hfull, Hc[0], Hc[1], Hc[2]);
    return cudaGetLastError();
}

cudaError_t launch_spectra(const Params& p, float2* Hfull, double2* Hc[kMaxCand], cudaStream_t st) {
    switch (fft_maxb(p.Wb)) {
        case 1: return spectra_t<1>(p, Hfull, Hc, st);
        case 2: return spectra_t<2>(p, Hfull, Hc, st);
        default: return spectra_t<4>(p, Hfull, Hc, st);
    }
}

}  // namespace apx
