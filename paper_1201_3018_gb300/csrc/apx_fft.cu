// apx_fft.cu -- the frequency-domain (FFT) core.
//
// Pass 1 (k_select): one CTA per block computes the block statistics and runs
// the Section IV.D selection; for a packing candidate it also companded the
// block and checks the FFT error bound (reading c7) with the exact integer
// norm sum(s~^2), so the packed digits are recovered by rounding.
// Pass 2 (k_spectra, apx_prep.cu): kernel spectra of the candidates in use.
// Pass 3 (k_fft): one CTA per block: compand + pack into a complex buffer
// (two real samples per complex word), forward real FFT, product with the
// kernel spectrum, inverse FFT, digit extraction, inverse companding, store.
#include "apx_block.cuh"
#include "apx_launch.h"

namespace apx {

__global__ void __launch_bounds__(kFftThreads) k_select(const Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    const long long i = blockIdx.x;
    const BlockGeom g = block_geom(p, i);
    float* xs = reinterpret_cast<float*>(smem);
    load_window(p, g, xs);
    const Pro pr = block_prologue(p, xs, sh);
    Sel s;
    s.cs = 0.f; s.Ms = pr.Ms; s.sig2 = pr.sig2; s.ferr = 0.0; s.pad_ = 0;
    if (pr.kind != 0) {
        s.ci = pr.kind == 3 ? -3 : -2;
        if (threadIdx.x == 0) p.sel[i] = s;
        return;
    }
    const KInfo& ki = *p.ki;
    s.ci = -1;
    for (int c = 0; c < p.ncand; ++c) {
        const Cand& cd = p.cand[c];
        if (p.autosel && !snr_feasible(pr.sig2, pr.Ms, ki.sig2k, ki.Mk, cd.S, cd.K, p.thr)) continue;
        const float cs = compand_factor(cd.S, pr.Ms);
        long long ss = 0;
        for (int t = threadIdx.x; t < p.Wb; t += blockDim.x) {
            long long q = compand(cs, xs[t]);
            ss += q * q;
        }
        ss = block_reduce<long long, false>(ss, sh.redl);
        const double eps = ldexp(1.0, -cd.b);
        const double grow = cd.blk == APX_BLK_SYM ? __dadd_rn(1.0, eps) : __dadd_rn(1.0, __dmul_rn(2.0, eps));
        const double l2 = __dmul_rn(__dsqrt_rn(__ll2double_rn(ss)), grow);
        const double E = ldexp(__dmul_rn(__dmul_rn(cd.fftc, ki.l1[c]), l2), cd.sc);
        if (E < 0.25) {
            s.ci = c; s.cs = cs; s.ferr = E;
            break;
        }
    }
    if (threadIdx.x == 0) {
        p.sel[i] = s;
        atomicOr(p.used, s.ci >= 0 ? (1u << s.ci) : 8u);
    }
}

template <int MAXB>
__global__ void __launch_bounds__(kFftThreads) k_fft(const Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const long long i = blockIdx.x;
    const BlockGeom g = block_geom(p, i);
    const Sel s = p.sel[i];
    if (s.ci <= -2) {
        Pro pr;
        pr.kind = s.ci == -3 ? 3 : 2;
        pr.Ms = s.Ms;
        pr.sig2 = 0.0;
        handle_trivial(p, i, g, pr);
        return;
    }
    float* xs = reinterpret_cast<float*>(smem);
    unsigned char* cbuf = smem + (size_t)4 * p.Wb;
    load_window(p, g, xs);

    if (s.ci < 0) {
        // Full precision: real FFT of length W_block in FP32.
        const int m = p.Wb / 2;
        float2* z = reinterpret_cast<float2*>(cbuf);
        for (int j = threadIdx.x; j < m; j += blockDim.x) z[j] = make_float2(xs[2 * j], xs[2 * j + 1]);
        __syncthreads();
        fft_smem<float2, false, MAXB>(z, m, p.tw32, 2);
        spectral_multiply(z, m, p.Hfull, p.tw32, 1);
        fft_smem<float2, true, MAXB>(z, m, p.tw32, 2);
        const float* y = reinterpret_cast<const float*>(z);
        for (int j = g.lo + threadIdx.x; j < g.hi; j += blockDim.x) {
            const long long o = g.start + j;
            if (o < 0 || o >= p.out_len) continue;
            p.r[o] = y[j];
            if (p.rq) p.rq[o] = 0;
        }
        write_stats(p, i, APX_BLK_FULL, nullptr, 0.f, s.Ms, s.sig2, __longlong_as_double(0x7ff0000000000000ll), 0.0);
        return;
    }

    const Cand& c = p.cand[s.ci];
    const float cs = s.cs;
    const double eps = ldexp(1.0, -c.b);
    double2* z = reinterpret_cast<double2*>(cbuf);
    double* zr = reinterpret_cast<double*>(cbuf);  // packed real words, two per complex entry
    int n, Ls = 0, nr = 0;
    if (c.blk == APX_BLK_SYM) {
        n = p.Wb / 2;
        for (int m = threadIdx.x; m < n; m += blockDim.x) {              // Eq. (4)
            const double e = (double)compand(cs, xs[2 * m]);
            const double o = (double)compand(cs, xs[2 * m + 1]);
            zr[m] = __dadd_rn(e, __dmul_rn(eps, o));
        }
    } else {
        n = p.Wb;
        Ls = (p.Wb + c.M - 1) / c.M;
        nr = Ls + p.Nodd - 1;
        for (int m = threadIdx.x; m < n; m += blockDim.x) {              // Eq. (7), zero past Ls
            double acc = 0.0, ep = 1.0;
            if (m < Ls) {
                for (int q = 0; q < c.M; ++q) {
                    const int t = m + q * Ls;
                    if (t < p.Wb) acc = __dadd_rn(acc, __dmul_rn(ep, (double)compand(cs, xs[t])));
                    ep = __dmul_rn(ep, eps);
                }
            }
            zr[m] = acc;
        }
    }
    __syncthreads();
    const int m = n / 2;
    fft_smem<double2, false, MAXB>(z, m, p.tw64, p.Wb / m);
    spectral_multiply(z, m, c.H, p.tw64, p.Wb / n);
    fft_smem<double2, true, MAXB>(z, m, p.tw64, p.Wb / m);

    const KInfo& ki = *p.ki;
    const float inv = (float)(1.0 / ((double)cs * (double)ki.ck[s.ci]));
    auto Tat = [&](int idx) { return scaled(zr[idx], c.sc); };
    for (int j = g.lo + threadIdx.x; j < g.hi; j += blockDim.x) {
        const long long o = g.start + j;
        if (o < 0 || o >= p.out_len) continue;
        long long rt = c.blk == APX_BLK_SYM ? unpack_sym(c, j, g.wstart, Tat) : unpack_asym(c, j, Ls, nr, Tat);
        p.r[o] = __fmul_rn(__ll2float_rn(rt), inv);
        if (p.rq) p.rq[o] = (int)rt;
    }
    if (threadIdx.x == 0)
        write_stats(p, i, c.blk, &c, cs, s.Ms, s.sig2, snr_model_db(s.sig2, s.Ms, ki.sig2k, ki.Mk, c.S, c.K), s.ferr);
}

cudaError_t launch_select(const Params& p, cudaStream_t st) {
    static int attr_dev = -1;
    int dev;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    if (p.P <= 0) return cudaSuccess;
    k_select<<<(unsigned)p.P, kFftThreads, (size_t)4 * p.Wb, st>>>(p);
    return cudaGetLastError();
}

template <int MAXB>
static cudaError_t fft_t(const Params& p, size_t smem, cudaStream_t st) {
    static int attr_dev = -1;
    int dev;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_fft<MAXB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    k_fft<MAXB><<<(unsigned)p.P, kFftThreads, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fft(const Params& p, size_t smem, cudaStream_t st) {
    if (p.P <= 0) return cudaSuccess;
    switch (fft_maxb(p.Wb)) {
        case 1: return fft_t<1>(p, smem, st);
        case 2: return fft_t<2>(p, smem, st);
        default: return fft_t<4>(p, smem, st);
    }
}

}  // namespace apx
