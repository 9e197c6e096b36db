// apx_fft.cu -- the frequency-domain (FFT) core.
//
// k_select (one CTA per block): kernel and window statistics and the Section
// IV.D selection; for a packing candidate it also companded the block and
// checks the FFT error bound (reading c7) with the exact integer norms
// sum(s~^2) and ||kbar||_1, so that rounding recovers the packed digits.
// k_spectra (apx_spectra.cu): kernel spectra; the FP32 one runs concurrently
// with k_select, the packed ones only for candidates some block selected.
// k_fft (one CTA per block): compand + pack into a complex buffer (two real
// words per complex entry), forward real FFT, product with the kernel
// spectrum, inverse FFT, digit extraction, inverse companding, store.
//
// k_spectra and k_fft are programmatic dependents of the kernel before them:
// k_fft fetches its window into registers before griddepcontrol.wait, so the
// load overlaps the spectra.
#include "apx_block.cuh"
#include "apx_launch.h"

namespace apx {

constexpr int kVals = 32;  // window samples per thread (W_block / threads)

// Thread t holds window samples 2(t + i NT) and 2(t + i NT) + 1 (pair t + i NT)
// for pairs below W_block/2; other slots hold zeros, which leave the maximum,
// the second moment and the companded norm unchanged.
__device__ __forceinline__ bool pair_ok(const Params& p, int i) { return threadIdx.x + i * blockDim.x < p.Wb / 2; }

__device__ __forceinline__ void load_window_regs(const Params& p, long long start, float (&xv)[kVals]) {
    const bool aligned = ((reinterpret_cast<uintptr_t>(p.s + start) & 7u) == 0);
#pragma unroll
    for (int i = 0; i < kVals / 2; ++i) {
        xv[2 * i] = 0.f;
        xv[2 * i + 1] = 0.f;
        if (pair_ok(p, i)) {
            const long long gi = start + 2ll * (threadIdx.x + i * blockDim.x);
            float2 v;
            if (aligned && gi >= 0 && gi + 1 < p.L) {
                v = __ldg(reinterpret_cast<const float2*>(p.s + gi));
            } else {
                v.x = (gi >= 0 && gi < p.L) ? __ldg(p.s + gi) : 0.f;
                v.y = (gi + 1 >= 0 && gi + 1 < p.L) ? __ldg(p.s + gi + 1) : 0.f;
            }
            xv[2 * i] = v.x;
            xv[2 * i + 1] = v.y;
        }
    }
}

__global__ void __launch_bounds__(512, 1) k_select(const Params p) {
    __shared__ Shared sh;
    __shared__ int s_go;
    pdl_trigger();  // the spectrum of the FP32 taps needs nothing from this pass
    const long long i = blockIdx.x;
    const BlockGeom g = block_geom(p, i);
    float xv[kVals];
    load_window_regs(p, g.start, xv);

    // ||s||_inf and the fixed-point second moment, from registers
    float m = 0.f;
    int bad = 0;
#pragma unroll
    for (int v = 0; v < kVals; ++v) {
        float a = fabsf(xv[v]);
        if (a != a) bad = 1;
        m = fmaxf(m, a);
    }
    m = block_reduce<float, true>(m, sh.redf);
    bad = block_reduce<int, true>(bad, sh.redi);
    const bool finite = !bad && m <= 3.402823466e38f;
    double sig2 = 0.0;
    if (finite && m > 0.f) {
        const FxScale f = fx_scale(m);
        long long acc = 0;
#pragma unroll
        for (int v = 0; v < kVals; ++v) acc += fx_sq(f, xv[v]);
        acc = block_reduce<long long, false>(acc, sh.redl);
        sig2 = fx_moment(acc, f, p.Wb, sh);
    }
    // Kernel initialisation of Section IV, from the raw taps in every CTA.
    const KStats ks = kernel_stats(p, sh);
    if (i == 0 && threadIdx.x == 0) {
        KInfo o;
        o.Mk = ks.Mk;
        o.nonfinite = ks.bad;
        o.sig2k = ks.sig2k;
        *p.ki = o;
    }

    Sel s;
    s.cs = 0.f; s.Ms = bad ? __int_as_float(0x7fc00000) : m; s.inv = 0.f;
    s.sig2 = sig2; s.ferr = 0.0; s.snr_db = __longlong_as_double(0x7ff0000000000000ll);
    if (!finite || ks.bad) s.ci = -3;
    else if (m == 0.f || ks.Mk == 0.f) s.ci = -2;
    else {
        s.ci = -1;
        for (int c = 0; c < p.ncand; ++c) {
            const Cand& cd = p.cand[c];
            if (threadIdx.x == 0)
                s_go = !p.autosel || snr_feasible(sig2, m, ks.sig2k, ks.Mk, cd.S, cd.K, p.thr);
            __syncthreads();
            const int go = s_go;
            __syncthreads();
            if (!go) continue;
            // FFT exactness (reading c7) with the exact norms of this block and kernel
            const float cs = compand_factor(cd.S, m);
            const float ck = compand_factor(cd.K, ks.Mk);
            long long ss = 0;
#pragma unroll
            for (int v = 0; v < kVals; ++v) {
                const long long q = compand(cs, xv[v]);
                ss += q * q;
            }
            ss = block_reduce<long long, false>(ss, sh.redl);
            const long long l1 = kbar_l1(p, cd, ck, sh);
            if (threadIdx.x == 0) {
                const double eps = ldexp(1.0, -cd.b);
                const double grow = cd.blk == APX_BLK_SYM ? __dadd_rn(1.0, eps) : __dadd_rn(1.0, __dmul_rn(2.0, eps));
                const double l2 = __dmul_rn(__dsqrt_rn(__ll2double_rn(ss)), grow);
                const double E = ldexp(__dmul_rn(__dmul_rn(cd.fftc, __ll2double_rn(l1)), l2), cd.sc);
                sh.bcast[1] = E;
                sh.bcast[2] = 1.0 / ((double)cs * (double)ck);
            }
            __syncthreads();
            const double E = sh.bcast[1];
            if (E < 0.25) {
                s.ci = c; s.cs = cs; s.ferr = E; s.inv = (float)sh.bcast[2];
                if (threadIdx.x == 0) s.snr_db = snr_model_db(sig2, m, ks.sig2k, ks.Mk, cd.S, cd.K);
                break;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        p.sel[i] = s;
        if (s.ci >= -1) atomicOr(p.used, s.ci >= 0 ? (1u << s.ci) : 8u);
    }
}

// real word w of a padded complex buffer
template <typename R, typename C>
__device__ __forceinline__ R& word(C* Z, int w) {
    return reinterpret_cast<R*>(Z)[2 * pad16(w >> 1) + (w & 1)];
}

__global__ void __launch_bounds__(512) k_fft(const Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const long long i = blockIdx.x;
    const BlockGeom g = block_geom(p, i);
    float xv[kVals];
    load_window_regs(p, g.start, xv);

    pdl_wait();  // spectra (and, through it, the selection) complete
    const Sel s = p.sel[i];
    if (s.ci <= -2) {
        Pro pr;
        pr.kind = s.ci == -3 ? 3 : 2;
        pr.Ms = s.Ms;
        pr.sig2 = 0.0;
        handle_trivial(p, i, g, pr);
        return;
    }

    if (s.ci < 0) {
        // Full precision: real FFT of length W_block in FP32.
        const int m = p.Wb / 2;
        float2* Z = reinterpret_cast<float2*>(smem);
#pragma unroll
        for (int v = 0; v < kVals / 2; ++v)
            if (pair_ok(p, v)) Z[pad16(threadIdx.x + v * blockDim.x)] = make_float2(xv[2 * v], xv[2 * v + 1]);
        __syncthreads();
        fft_smem<float2, false>(Z, m, p.tw32, p.Wb);
        spectral_multiply(Z, m, p.Hfull, p.tw32, 1);
        fft_smem<float2, true>(Z, m, p.tw32, p.Wb);
        for (int j = g.lo + threadIdx.x; j < g.hi; j += blockDim.x) {
            const long long o = g.start + j;
            if (o < 0 || o >= p.out_len) continue;
            p.r[o] = word<float>(Z, j);
            if (p.rq) p.rq[o] = 0;
        }
        write_stats(p, i, APX_BLK_FULL, nullptr, 0.f, s.Ms, s.sig2, __longlong_as_double(0x7ff0000000000000ll), 0.0);
        return;
    }

    const Cand& c = p.cand[s.ci];
    const float cs = s.cs;
    const double eps = ldexp(1.0, -c.b);
    double2* Z = reinterpret_cast<double2*>(smem);
    int n, Ls = 0, nr = 0;
    if (c.blk == APX_BLK_SYM) {
        // Eq. (4): word w = s~[2w] + eps s~[2w+1]; this thread holds pair w
        n = p.Wb / 2;
#pragma unroll
        for (int v = 0; v < kVals / 2; ++v)
            if (pair_ok(p, v)) {
                const int w = threadIdx.x + v * blockDim.x;
                word<double>(Z, w) = __dadd_rn((double)compand(cs, xv[2 * v]),
                                               __dmul_rn(eps, (double)compand(cs, xv[2 * v + 1])));
            }
    } else {
        // Eq. (7): word w = sum_q eps^q s~[w + q Ls], zero past Ls
        n = p.Wb;
        Ls = (p.Wb + c.M - 1) / c.M;
        nr = Ls + p.Nodd - 1;
        int* sq = reinterpret_cast<int*>(smem + sizeof(double2) * padded_len(p.Wb / 2));
#pragma unroll
        for (int v = 0; v < kVals / 2; ++v)
            if (pair_ok(p, v)) {
                const int e = 2 * (threadIdx.x + v * blockDim.x);
                sq[e] = compand(cs, xv[2 * v]);
                sq[e + 1] = compand(cs, xv[2 * v + 1]);
            }
        __syncthreads();
        for (int w = threadIdx.x; w < n; w += blockDim.x) {
            double acc = 0.0, ep = 1.0;
            if (w < Ls) {
                for (int q = 0; q < c.M; ++q) {
                    const int t = w + q * Ls;
                    if (t < p.Wb) acc = __dadd_rn(acc, __dmul_rn(ep, (double)sq[t]));
                    ep = __dmul_rn(ep, eps);
                }
            }
            word<double>(Z, w) = acc;
        }
    }
    __syncthreads();
    const int m = n / 2;
    fft_smem<double2, false>(Z, m, p.tw64, p.Wb);
    spectral_multiply(Z, m, c.H, p.tw64, p.Wb / n);
    fft_smem<double2, true>(Z, m, p.tw64, p.Wb);

    const float inv = s.inv;
    auto Tat = [&](int idx) { return scaled(word<double>(Z, idx), c.sc); };
    for (int j = g.lo + threadIdx.x; j < g.hi; j += blockDim.x) {
        const long long o = g.start + j;
        if (o < 0 || o >= p.out_len) continue;
        long long rt = c.blk == APX_BLK_SYM ? unpack_sym(c, j, g.wstart, Tat) : unpack_asym(c, j, Ls, nr, Tat);
        p.r[o] = __fmul_rn(__ll2float_rn(rt), inv);
        if (p.rq) p.rq[o] = (int)rt;
    }
    if (threadIdx.x == 0)
        write_stats(p, i, c.blk, &c, cs, s.Ms, s.sig2, s.snr_db, s.ferr);
}

cudaError_t launch_select(const Params& p, cudaStream_t st) {
    if (p.P <= 0) return cudaSuccess;
    return launch_k(k_select, dim3((unsigned)p.P), dim3(fft_threads(p.Wb)), 0, st, false, p);
}

size_t fft_smem_bytes(const Params& p) {
    bool asym = false, packed = p.ncand > 0;
    for (int j = 0; j < p.ncand; ++j) asym |= p.cand[j].blk != APX_BLK_SYM;
    size_t z32 = sizeof(float2) * padded_len(p.Wb / 2);
    size_t z64 = packed ? sizeof(double2) * padded_len(asym ? p.Wb / 2 : p.Wb / 4) : 0;
    size_t sq = asym ? sizeof(int) * (size_t)p.Wb : 0;
    return (z32 > z64 + sq ? z32 : z64 + sq);
}

cudaError_t launch_fft(const Params& p, size_t smem, cudaStream_t st) {
    if (p.P <= 0) return cudaSuccess;
    static int attr_dev = -1;
    int dev;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    return launch_k(k_fft, dim3((unsigned)p.P), dim3(fft_threads(p.Wb)), smem, st, true, p);
}

}  // namespace apx
