// apx_fft_body.cuh -- one overlap-save block of the FFT core on a whole CTA
// (the body of the general block kernel k_fft, and of the serving engine's
// persistent CTAs).  See apx_fft.cu for the steps.
#pragma once

#include <type_traits>

#include "apx_prep.cuh"

namespace apx {

constexpr long long kSpinCycles = kPrepSpinCycles;

// Thread t holds window samples 2(t + i NT) and 2(t + i NT) + 1 (pair t + i NT)
// for pairs below W_block/2; other slots hold zeros, which leave the maximum,
// the second moment and the companded norm unchanged.
__device__ __forceinline__ bool pair_ok(const Params& p, int i) { return threadIdx.x + i * blockDim.x < p.Wb / 2; }

template <int kVals>
__device__ __forceinline__ void load_window_regs(const Params& p, long long start, float (&xv)[kVals]) {
    static_assert(kVals % 4 == 0, "runs in couples");
    const bool aligned = ((reinterpret_cast<uintptr_t>(p.s + start) & 7u) == 0);
    const int nt = (int)blockDim.x, t = (int)threadIdx.x;
    auto pair_at = [&](int i) {  // pair t + i nt, one thread alone
        float2 v = make_float2(0.f, 0.f);
        if (pair_ok(p, i)) {
            const long long gi = start + 2ll * (t + i * nt);
            if (aligned && gi >= 0 && gi + 1 < p.L) {
                v = APX_LD_IN(reinterpret_cast<const float2*>(p.s + gi));
            } else {
                v.x = (gi >= 0 && gi < p.L) ? APX_LD_IN(p.s + gi) : 0.f;
                v.y = (gi + 1 >= 0 && gi + 1 < p.L) ? APX_LD_IN(p.s + gi + 1) : 0.f;
            }
        }
        return v;
    };
    // 16-byte loads when every run of the warp starts on a 16-byte boundary of
    // the signal and lies inside the window and the signal (warp-uniform):
    // lanes 2c and 2c + 1 form a couple; of runs 2a and 2a + 1, the even lane
    // loads run 2a for both, the odd lane run 2a + 1, and each passes the
    // other its half by a shuffle.  Runs 8 bytes off a boundary take 8-byte
    // loads, which cover them in as few instructions.
    constexpr int kRuns = kVals / 2;
    const int lane = t & 31, pw = t - lane;
    const long long gw = start + 2ll * pw;
    const bool vec = ((reinterpret_cast<uintptr_t>(p.s + gw) & 15u) == 0) && pw + 31 + (kRuns - 1) * nt < p.Wb / 2 &&
                     gw >= 0 && gw + 2ll * (kRuns - 1) * nt + 63 < p.L;
    if (vec) {
        const bool even = (lane & 1) == 0;
        const float* b = p.s + start + 2ll * t;  // this thread's pair of run 0
#pragma unroll
        for (int a = 0; a < kRuns / 2; ++a) {
            const float4 w = APX_LD_IN(reinterpret_cast<const float4*>(even ? b + 4 * a * nt
                                                                             : b + 2 * (2 * a + 1) * nt - 2));
            const float2 mine = even ? make_float2(w.x, w.y) : make_float2(w.z, w.w);
            const float2 other = even ? make_float2(w.z, w.w) : make_float2(w.x, w.y);
            float2 got;
            got.x = __shfl_xor_sync(0xffffffffu, other.x, 1);
            got.y = __shfl_xor_sync(0xffffffffu, other.y, 1);
            const float2 v0 = even ? mine : got, v1 = even ? got : mine;
            xv[4 * a] = v0.x;
            xv[4 * a + 1] = v0.y;
            xv[4 * a + 2] = v1.x;
            xv[4 * a + 3] = v1.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kRuns; ++i) {
            const float2 v = pair_at(i);
            xv[2 * i] = v.x;
            xv[2 * i + 1] = v.y;
        }
    }
}

// How a block waits for its call's kernel preparation: the preparation
// launches it is the programmatic dependent of; jobs 0 .. nj-1 of the call run
// by other CTAs of the same launch (bounded wait); or nothing (the preparation
// is resident: a prepared kernel).
constexpr int kWaitLaunch = 0, kWaitJobs = 1, kWaitNone = 2;

// Overlap-save block i of the call p on the whole CTA (the general block
// kernel's body; also run by the serving engine's persistent CTAs).
template <int kVals>
__device__ __forceinline__ void fft_block_body(const Params& p, long long i, int nj, int wait, unsigned char* smem,
                                               Shared& sh, int& s_flag, unsigned& s_feas, int& s_job) {
    const BlockGeom g = block_geom(p, i);
    float xv[kVals];
    load_window_regs(p, g.start, xv);

    // ||s||_inf and the fixed-point second moment, from registers
    // one integer reduction gives the maximum and whether a NaN (bits above
    // +inf) is present
    int mb = 0;
#pragma unroll
    for (int v = 0; v < kVals; ++v) mb = max(mb, __float_as_int(xv[v]) & 0x7fffffff);
    mb = block_reduce<int, true>(mb, sh.redi);
    const int bad = mb > 0x7f800000;
    const float m = bad ? 0.f : __int_as_float(mb);
    const bool finite = !bad && m <= 3.402823466e38f;
    // the second moment as its exact fixed-point sum (pro_sig2 rounds it to
    // FP64 where a thread needs it; s2s_f feeds the model's FP32 screen)
    Pro pr;
    pr.kind = 0;
    pr.Ms = m;
    pr.acc = 0;
    pr.fsh = 0;
    pr.s2s_f = 0.f;
    if (finite && m > 0.f) {
        const FxScale f = fx_scale(m);
        long long acc = 0;
#pragma unroll
        for (int v = 0; v < kVals; ++v) acc += fx_sq(f, xv[v]);
        pr.acc = block_reduce<long long, false>(acc, sh.redl);
        pr.fsh = f.sh;
        pr.s2s_f = fx_moment_f32(pr.acc, f.sh, p.Wb);
    }

    // Full precision is every block's fallback: start its forward FFT (FP32)
    // while the kernel preparation may still be running.
    const int mf = p.Wb / 2;
    float2* Zf = reinterpret_cast<float2*>(smem);
    const bool live = finite && m > 0.f;
    if (live) {
#pragma unroll
        for (int v = 0; v < kVals / 2; ++v)
            if (pair_ok(p, v)) Zf[pad16(threadIdx.x + v * blockDim.x)] = make_float2(xv[2 * v], xv[2 * v + 1]);
        __syncthreads();
        fft_smem<float2, false>(Zf, mf, p.tw32, p.ntab, p.status);
    }

    // kernel statistics and FP32 kernel spectrum: from the preparation launches,
    // or from the preparation jobs of this launch
    if (wait == kWaitLaunch) {
        pdl_wait();
    } else if (wait == kWaitJobs && !wait_jobs(p, 0, nj, &s_job)) {
        store_constant(p, g, __int_as_float(0x7fc00000));
        return;
    }
    const float Mk = __ldcg(&p.ki->Mk);
    const int kbad = __ldcg(&p.ki->bad);
    const double sig2k = __ldcg(&p.ki->sig2k);
    const float Ms = bad ? __int_as_float(0x7fc00000) : m;
    if (!finite || kbad || m == 0.f || Mk == 0.f) {
        pr.kind = (!finite || kbad) ? 3 : 2;
        pr.Ms = Ms;
        handle_trivial(p, i, g, pr);
        return;
    }

    // Section IV.D selection (first admissible candidate in the Table 1 order).
    int ci = -1;
    float cs = 0.f, ck = 0.f;
    double ferr = 0.0;
    bool have_window = false;
    KStats ks;
    ks.Mk = Mk;
    ks.bad = kbad;
    ks.sig2k = sig2k;
    ks.sig2k_f = threadIdx.x < 32 ? (float)sig2k : 0.f;  // FP64 conversions in the deciding warp only
    ks.thr_f = threadIdx.x < 32 ? (float)p.thr : 0.f;
    const unsigned feas = feasible_mask_pro(p, pr, ks, &s_feas);
    for (int c = 0; c < p.ncand; ++c) {
        if (!((feas >> c) & 1u)) continue;
        const Cand& cd = p.cand[c];
        if (!have_window) { load_window_regs(p, g.start, xv); have_window = true; }
        const float cs_c = compand_factor(cd.S, m);
        const float ck_c = compand_factor(cd.K, Mk);
        long long ss = 0;
#pragma unroll
        for (int v = 0; v < kVals; ++v) {
            const long long q = compand(cs_c, xv[v]);
            ss += q * q;
        }
        ss = block_reduce<long long, false>(ss, sh.redl);
        if (threadIdx.x == 0) {
            const double eps = ldexp(1.0, -cd.b);
            const double grow = cd.blk == APX_BLK_SYM ? __dadd_rn(1.0, eps) : __dadd_rn(1.0, __dmul_rn(2.0, eps));
            const double l2 = __dmul_rn(__dsqrt_rn(__ll2double_rn(ss)), grow);
            // a nonzero kernel has ||kbar||_1 >= 1 (its largest tap companded to +-K_q);
            // 0 means the preparation skipped this candidate: never admit it on that
            const double l1 = __ldcg(&p.ki->l1[c]);
            sh.bcast[1] = l1 > 0.0 ? ldexp(__dmul_rn(__dmul_rn(cd.fftc, l1), l2), cd.sc) : 1.0;
        }
        __syncthreads();
        const double E = sh.bcast[1];
        __syncthreads();
        if (E < 0.25) {
            ci = c; cs = cs_c; ck = ck_c; ferr = E;
            break;
        }
    }

    if (ci < 0) {
        // Full precision: finish the FP32 real-FFT convolution.
        spectral_multiply(Zf, mf, static_cast<const float2*>(p.Hfull), p.tw32, p.ntab / p.Wb, true, p.status);
        fft_smem<float2, true>(Zf, mf, p.tw32, p.ntab, p.status);
        store_kept(p, g, [&](int j, int& iv) {
            iv = 0;
            return APX_IN_BOUNDS(j >= 0 && j < p.Wb, p.status) ? word<float>(Zf, j) : 0.f;
        });
        if (p.st && threadIdx.x == 0)
            write_stats(p, i, APX_BLK_FULL, nullptr, 0.f, Ms, pro_sig2(pr, p.Wb),
                        __longlong_as_double(0x7ff0000000000000ll), 0.0);
        return;
    }

    const Cand& c = p.cand[ci];
    const double eps = ldexp(1.0, -c.b);
    double2* Z = reinterpret_cast<double2*>(smem);
    const int n = c.blk == APX_BLK_SYM ? p.Wb / 2 : p.Wb;
    const int mm = n / 2;

    // The packed kernel spectrum, built once per call by the first CTA to claim it.
    if (threadIdx.x == 0) {
        int st = 0;  // 0 ready, 1 build it here, 2 wait for another CTA
        if (ld_acquire(&p.ready[ci]) != p.epoch) st = atomicExch(&p.claim[ci], p.epoch) != p.epoch ? 1 : 2;
        s_flag = st;
    }
    __syncthreads();
    const int role = s_flag;
    __syncthreads();  // (also: every thread is done with the speculative FP32 buffer)
    if (role == 1) {
        auto tap = [&](int t) -> double { return (double)kbar_int(p, c, ck, t); };  // Eq. (5) / k~
        spectrum_of<double>(tap, p.ntab, n, p.tw64, c.H, Z);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release(&p.ready[ci], p.epoch);
    }

    int Ls = 0, nr = 0;
    if (c.blk == APX_BLK_SYM) {
        // Eq. (4): word w = s~[2w] + eps s~[2w+1]; this thread holds pair w
#pragma unroll
        for (int v = 0; v < kVals / 2; ++v)
            if (pair_ok(p, v)) {
                const int w = threadIdx.x + v * blockDim.x;
                word<double>(Z, w) = __dadd_rn((double)compand(cs, xv[2 * v]),
                                               __dmul_rn(eps, (double)compand(cs, xv[2 * v + 1])));
            }
    } else {
        // Eq. (7): word w = sum_q eps^q s~[w + q Ls], zero past Ls
        Ls = (p.Wb + c.M - 1) / c.M;
        nr = Ls + p.Nodd - 1;
        // the companded block, in the narrowest integer type that holds +-S_q
        unsigned char* sqb = smem + sizeof(double2) * padded_len(p.Wb / 2);
        auto pack = [&](auto* sq) {
            using T = typename std::remove_pointer<decltype(sq)>::type;
#pragma unroll
            for (int v = 0; v < kVals / 2; ++v)
                if (pair_ok(p, v)) {
                    const int e = 2 * (threadIdx.x + v * blockDim.x);
                    sq[e] = (T)compand(cs, xv[2 * v]);
                    sq[e + 1] = (T)compand(cs, xv[2 * v + 1]);
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
        };
        const int esz = companded_bytes(p);
        if (esz == 1) pack(reinterpret_cast<signed char*>(sqb));
        else if (esz == 2) pack(reinterpret_cast<short*>(sqb));
        else pack(reinterpret_cast<int*>(sqb));
    }
    __syncthreads();
    fft_smem<double2, false>(Z, mm, p.tw64, p.ntab, p.status);

    if (role == 2) {
        if (threadIdx.x == 0) {
            int ok = 0;
            const long long t0 = clock64();
            while (true) {
                if (ld_acquire(&p.ready[ci]) == p.epoch) { ok = 1; break; }
                if (clock64() - t0 > kSpinCycles) break;
                __nanosleep(256);
            }
            if (!ok) atomicOr(p.status, 2u);
            s_flag = ok;
        }
        __syncthreads();
        if (!s_flag) {
            store_constant(p, g, __int_as_float(0x7fc00000));
            return;
        }
    }
    spectral_multiply(Z, mm, static_cast<const double2*>(c.H), p.tw64, p.ntab / n, true, p.status);
    fft_smem<double2, true>(Z, mm, p.tw64, p.ntab, p.status);

    if (threadIdx.x == 0) sh.bcast[2] = 1.0 / ((double)cs * (double)ck);
    __syncthreads();
    const float inv = (float)sh.bcast[2];
    auto Tat = [&](int idx) { return scaled(word<double>(Z, idx), c.sc); };
    store_kept<true>(p, g, [&](int j, int& iv) {
        const long long rt = c.blk == APX_BLK_SYM ? unpack_sym(c, j, g.wstart, Tat) : unpack_asym(c, j, Ls, nr, Tat);
        iv = (int)rt;
        return __fmul_rn(__ll2float_rn(rt), inv);
    });
    if (p.st && threadIdx.x == 0)
        write_stats(p, i, c.blk, &c, cs, Ms, pro_sig2(pr, p.Wb), snr_model_db(pro_sig2(pr, p.Wb), m, sig2k, Mk, c.S, c.K),
                    ferr);
}

}  // namespace apx
