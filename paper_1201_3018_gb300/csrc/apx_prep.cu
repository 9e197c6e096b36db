// apx_prep.cu -- per-request kernel preparation (Section IV "Initialization"):
// ||k||_inf, the kernel's second moment, the FP32 taps (reversed for
// cross-correlation, zero-padded), and for every packing candidate the
// companded (Eq. 2) and packed taps (Eq. 5 with the pair order
// k~[2n+1] + eps^-1 k~[2n]) with their exact l1 norm.  The FFT core also needs
// kernel spectra; those are computed only for the candidates that some block
// actually selected.
#include "apx_block.cuh"
#include "apx_launch.h"

namespace apx {

constexpr int kPrepPairs = 8;  // tap pairs per thread: 2 * 8 * 1024 >= 16384 taps

__global__ void __launch_bounds__(kPrepThreads) k_prep(const Params p, const float* __restrict__ k, int xcorr,
                                                       KInfo* ki, float* kfull, double* kb0, double* kb1,
                                                       double* kb2) {
    __shared__ Shared sh;
    pdl_trigger();
    if (threadIdx.x == 0 && p.used) *p.used = 0u;
    const int N = p.N, Nodd = p.Nodd;
    const int nkp32 = (Nodd + 7) / 8 * 8;
    // thread t holds taps 2(t + i NT) and 2(t + i NT) + 1 of the (reversed) kernel
    float kv[2 * kPrepPairs];
#pragma unroll
    for (int i = 0; i < kPrepPairs; ++i) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n = 2 * (threadIdx.x + i * blockDim.x) + h;
            kv[2 * i + h] = n < N ? __ldg(&k[xcorr ? N - 1 - n : n]) : 0.f;
            if (n < nkp32) kfull[n] = kv[2 * i + h];
        }
    }
    float m = 0.f;
    int bad = 0;
#pragma unroll
    for (int v = 0; v < 2 * kPrepPairs; ++v) {
        const float a = fabsf(kv[v]);
        if (!(a <= 3.402823466e38f)) bad = 1;
        m = fmaxf(m, a);
    }
    m = block_reduce<float, true>(m, sh.redf);
    bad = block_reduce<int, true>(bad, sh.redi);

    const bool ok = !bad && m > 0.f;
    double sig2 = 0.0;
    if (ok) {
        int e;
        (void)frexpf(m, &e);
        const int sh2 = 24 - e, a = sh2 / 2, b = sh2 - a;
        const float fa = __int_as_float((a + 127) << 23), fb = __int_as_float((b + 127) << 23);
        long long acc = 0;
#pragma unroll
        for (int v = 0; v < 2 * kPrepPairs; ++v) {
            const long long q = __float2int_rz(__fmul_rn(__fmul_rn(kv[v], fa), fb));
            acc += q * q;
        }
        acc = block_reduce<long long, false>(acc, sh.redl);
        sig2 = __ddiv_rn(ldexp(__ll2double_rn(acc), -2 * sh2), (double)N);
    }

    float cks[kMaxCand] = {0.f, 0.f, 0.f};
    double l1s[kMaxCand] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < kMaxCand; ++c) {
        if (c >= p.ncand) break;
        const Cand& cd = p.cand[c];
        double* kb = c == 0 ? kb0 : (c == 1 ? kb1 : kb2);
        const float ck = ok ? compand_factor(cd.K, m) : 0.f;            // Eq. (2)
        const int nkp = (cd.nk + 3) / 4 * 4;
        long long l1 = 0;
#pragma unroll
        for (int i = 0; i < kPrepPairs; ++i) {
            const int pr = threadIdx.x + i * blockDim.x;                  // pair index
            const long long q0 = ok ? (long long)compand(ck, kv[2 * i]) : 0ll;
            const long long q1 = ok ? (long long)compand(ck, kv[2 * i + 1]) : 0ll;
            if (cd.blk == APX_BLK_SYM) {
                if (pr < nkp) {
                    const long long v = pr < cd.nk ? q1 + (q0 << cd.b) : 0ll;  // Eq. (5), reading c2
                    kb[pr] = (double)v;
                    l1 += v < 0 ? -v : v;
                }
            } else {
                if (2 * pr < nkp) { kb[2 * pr] = (double)q0; l1 += q0 < 0 ? -q0 : q0; }
                if (2 * pr + 1 < nkp) { kb[2 * pr + 1] = (double)q1; l1 += q1 < 0 ? -q1 : q1; }
            }
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

// Kernel spectrum H = FFT_n(taps) / (4m), k in [0, m], natural order.
template <typename R, typename C>
__device__ void spectrum_of(const R* taps, int ntaps, int Wb, int n, const C* __restrict__ tw, C* H, C* Z) {
    const int m = n / 2;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        C v;
        v.x = 2 * j < ntaps ? taps[2 * j] : (R)0;
        v.y = 2 * j + 1 < ntaps ? taps[2 * j + 1] : (R)0;
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

// CTA 0: FP32 taps (full precision); CTA 1 + c: packed taps of candidate c.
// A spectrum nobody selected is skipped.
__global__ void __launch_bounds__(512) k_spectra(const Params p, float2* Hfull, double2* H0, double2* H1,
                                                 double2* H2) {
    extern __shared__ __align__(16) unsigned char smem[];
    pdl_trigger();
    pdl_wait();  // selection complete: `used` and the packed taps are final
    const unsigned used = *p.used;
    const int job = blockIdx.x;
    if (job == 0) {
        if (!(used & 8u)) return;
        spectrum_of<float, float2>(p.kfull, p.Nodd, p.Wb, p.Wb, p.tw32, Hfull, reinterpret_cast<float2*>(smem));
        return;
    }
    const int c = job - 1;
    if (c >= p.ncand || !(used & (1u << c))) return;
    const Cand& cd = p.cand[c];
    double2* Hc = c == 0 ? H0 : (c == 1 ? H1 : H2);
    const int n = cd.blk == APX_BLK_SYM ? p.Wb / 2 : p.Wb;
    spectrum_of<double, double2>(cd.kbar, cd.nk, p.Wb, n, p.tw64, Hc, reinterpret_cast<double2*>(smem));
}

cudaError_t launch_prep(const Params& p, const float* k, int xcorr, double* kbar_out[kMaxCand], KInfo* ki,
                        float* kfull, cudaStream_t st) {
    return launch_k(k_prep, dim3(1), dim3(kPrepThreads), 0, st, false, p, k, xcorr, ki, kfull, kbar_out[0],
                    kbar_out[1], kbar_out[2]);
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
