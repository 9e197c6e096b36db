// apx_fft.cu -- the frequency-domain (FFT) core.
//
// k_select (one CTA per block): window statistics and the Section IV.D
// selection; for a packing candidate it also companded the block and checks
// the FFT error bound (reading c7) with the exact integer norm sum(s~^2), so
// that rounding recovers the packed digits exactly.
// k_spectra (apx_prep.cu): kernel spectra of the candidates in use.
// k_fft (one CTA per block): compand + pack into a complex buffer (two real
// words per complex entry), forward real FFT, product with the kernel
// spectrum, inverse FFT, digit extraction, inverse companding, store.
//
// Each kernel is launched as a programmatic dependent of the previous one: the
// window is fetched into registers before griddepcontrol.wait, so the load
// overlaps the tail of the previous kernel.
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

__global__ void __launch_bounds__(512) k_select(const Params p) {
    __shared__ Shared sh;
    pdl_trigger();
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
    Sel s;
    s.cs = 0.f; s.Ms = bad ? __int_as_float(0x7fc00000) : m; s.sig2 = 0.0; s.ferr = 0.0; s.pad_ = 0;
    const bool finite = !bad && m <= 3.402823466e38f;
    double sig2 = 0.0;
    if (finite && m > 0.f) {
        int e;
        (void)frexpf(m, &e);
        const int sh2 = 24 - e, a = sh2 / 2, b = sh2 - a;
        const float fa = __int_as_float((a + 127) << 23), fb = __int_as_float((b + 127) << 23);
        long long acc = 0;
#pragma unroll
        for (int v = 0; v < kVals; ++v) {
            const long long q = __float2int_rz(__fmul_rn(__fmul_rn(xv[v], fa), fb));
            acc += q * q;
        }
        acc = block_reduce<long long, false>(acc, sh.redl);
        sig2 = __ddiv_rn(ldexp(__ll2double_rn(acc), -2 * sh2), (double)p.Wb);
    }
    s.sig2 = sig2;

    pdl_wait();  // kernel statistics from the preparation launch
    const KInfo& ki = *p.ki;
    if (!finite || ki.nonfinite) s.ci = -3;
    else if (m == 0.f || ki.Mk == 0.f) s.ci = -2;
    else {
        s.ci = -1;
        for (int c = 0; c < p.ncand; ++c) {
            const Cand& cd = p.cand[c];
            if (p.autosel && !snr_feasible(sig2, m, ki.sig2k, ki.Mk, cd.S, cd.K, p.thr)) continue;
            const float cs = compand_factor(cd.S, m);
            long long ss = 0;
#pragma unroll
            for (int v = 0; v < kVals; ++v) {
                const long long q = compand(cs, xv[v]);
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

    const KInfo& ki = *p.ki;
    const float inv = (float)(1.0 / ((double)cs * (double)ki.ck[s.ci]));
    auto Tat = [&](int idx) { return scaled(word<double>(Z, idx), c.sc); };
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
    if (p.P <= 0) return cudaSuccess;
    return launch_k(k_select, dim3((unsigned)p.P), dim3(fft_threads(p.Wb)), 0, st, true, p);
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
