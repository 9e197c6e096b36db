// apx_prep.cuh -- kernel preparation of the FFT core (Section IV
// "Initialization": the kernel is prepared once per request), as pieces that
// either the spectrum launches (k_spec, k_combine: batched calls and small
// single calls) or the first CTAs of the block kernel's own launch (single
// calls with enough blocks) run.  Whoever runs them, the pieces are the same code, so every path
// produces the same bits.
//
// The FP32 spectrum H[k] = FFT_n(taps)[k] / (4m), k in [0, m], n = W_block = 2m:
//   spec_subfft(r)   Y_r = FFT_{n/R1}(h[r], h[r+R1], ...) into Ysub, r < R1
//                    (decimation in time; the transform takes the radix of a
//                    kSpecRadixNt-thread CTA whatever the caller's size: radix
//                    8 at 512 points, three passes)
//   spec_combine(k)  H[k] = sum_{r < R1} W_n^(r k) Y_r[k mod n/R1] (the last
//                    decimation stage, one frequency)
//   spec_stats()     ||k||_inf, the second moment and the exact ||kbar||_1 of
//                    every reachable packing candidate into KInfo
#pragma once

#include "apx_block.cuh"
#include "apx_launch.h"

namespace apx {

constexpr long long kPrepSpinCycles = 2000000000LL;  // about one second at the maximum SM clock
// the thread count the sub-transforms' radix is chosen for (their CTAs have
// more threads; the surplus waits at the passes' barriers)
constexpr int kSpecRadixNt = 64;

// Y_r into Ysub[r * ns ..], Z: shared scratch of padded_len(ns) entries.
__device__ inline void spec_subfft(const Params& p, int r, float2* Z) {
    const int n = p.Wb, R1 = spec_r1(n), ns = n / R1;
    for (int j = threadIdx.x; j < ns; j += blockDim.x) Z[pad16(j)] = make_float2(ktap(p, r + j * R1), 0.f);
    __syncthreads();
    fft_smem_nt<float2, false>(Z, ns, kSpecRadixNt, p.tw32, p.ntab, p.status);
    for (int k = threadIdx.x; k < ns; k += blockDim.x)
        p.Ysub[r * ns + k] = Z[pad16(fft_perm_nt<float2>(k, ns, kSpecRadixNt))];
    __syncthreads();  // Z is free again
}

// H[k] for one k <= m from y[r] = Y_r[k mod n/R1], r < R1 (the last
// decimation stage), into Hfull and, when the call runs the two-CTA block
// kernel, its staging-order table.
__device__ inline void spec_combine_y(const Params& p, int k, const float2 (&y)[16]) {
    const int n = p.Wb, m = n / 2, R1 = spec_r1(n);
    float2 acc = make_float2(0.f, 0.f);
    float2 w[16];
#pragma unroll
    for (int r = 0; r < 16; ++r)
        if (r < R1) w[r] = __ldg(&p.tw32[(r * k * (p.ntab / n)) & (p.ntab - 1)]);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        if (r < R1) {
            acc.x = fmaf(y[r].x, w[r].x, fmaf(-y[r].y, w[r].y, acc.x));
            acc.y = fmaf(y[r].x, w[r].y, fmaf(y[r].y, w[r].x, acc.y));
        }
    }
    const float scale = 1.f / (float)(4 * m);
    const float2 h = make_float2(acc.x * scale, acc.y * scale);
    p.Hfull[k] = h;
    if (p.Hpair) {
        // the same values in the two-CTA kernel's staging order: H[k] (a = 0) and
        // W^k (a = 2) under frequency k <= m/2, H[m-k] (a = 1) under m - k
        const int nt = m / 16, kk = k <= m / 2 ? k : m - k;
        int rank, u, t;
        pair_entry(kk, m, &rank, &u, &t);
        float2* e = p.Hpair + rank * 15 * nt + 3 * u * nt + t;
        if (k <= m / 2) {
            e[0] = h;
            e[2 * nt] = p.tw32[k * (p.ntab / n)];
        }
        if (k >= m / 2) e[nt] = h;
    }
}

// H[k] for one k <= m, from the sub-spectra (read around L1: written during this call).
__device__ inline void spec_combine(const Params& p, int k) {
    const int n = p.Wb, R1 = spec_r1(n), ns = n / R1;
    const int kk = k & (ns - 1);
    float2 y[16];
#pragma unroll
    for (int r = 0; r < 16; ++r)
        if (r < R1) y[r] = __ldcg(&p.Ysub[r * ns + kk]);
    spec_combine_y(p, k, y);
}

// Kernel statistics and candidate norms into *p.ki (the whole CTA).
__device__ inline void spec_stats(const Params& p, Shared& sh) {
    const KStats ks = kernel_stats(p, sh);
    double l1s[kMaxCand] = {0.0, 0.0, 0.0};
    const bool ok = !ks.bad && ks.Mk > 0.f;
    // Under per-block selection a candidate whose model SNR misses the target even for the
    // best window is never chosen: skip its norm.  The model grows with the window's ratio
    // sigma^2 / ||s||_inf^2 <= 1, so the best window has ratio 1; the check is made 1 % below
    // the target, so that rounding can only keep a norm that is not needed, never drop one
    // that is.  Lane c of warp 0 checks candidate c (one FP64 chain for all of them).
    if (threadIdx.x < 32) {
        const int c = threadIdx.x;
        const bool reach = c < p.ncand && (!p.autosel || snr_feasible(1.0, 1.f, ks.sig2k, ks.Mk, p.cand[c].S,
                                                                      p.cand[c].K, __dmul_rn(p.thr, 0.99)));
        const unsigned m = __ballot_sync(0xffffffffu, reach);
        if (c == 0) sh.redi[0] = (int)m;
    }
    __syncthreads();
    const unsigned reach = (unsigned)sh.redi[0];
    __syncthreads();
    for (int c = 0; c < p.ncand; ++c)
        if (ok && ((reach >> c) & 1u)) l1s[c] = (double)kbar_l1(p, p.cand[c], compand_factor(p.cand[c].K, ks.Mk), sh);
    if (threadIdx.x == 0) {
        KInfo o;
        o.Mk = ks.Mk;
        o.bad = ks.bad;
        o.sig2k = ks.sig2k;
        for (int c = 0; c < kMaxCand; ++c) o.l1[c] = l1s[c];
        *p.ki = o;
    }
}

// ---- the preparation inside the block kernel (fused single calls)
// Jobs (prep_jobs_count): 0 .. R1-1 the sub-transforms, R1 .. R1+C-1 the
// combine slices of blockDim.x frequencies, R1+C the statistics.  Every CTA of
// the launch first takes a ticket from a counter that only grows (the host
// passes the counter's value before the launch, so tickets of a call start at
// 0): tickets below nj are preparation jobs, the others are blocks.  A CTA
// only ever waits for jobs with smaller tickets, which CTAs that have already
// started hold, so the waits end in whatever order the CTAs are scheduled.
// A finished job sets its ready word to the call's epoch.

// This CTA's ticket (thread 0 takes it; the CTA gets it).
__device__ __forceinline__ long long prep_ticket(const Params& p, long long* slot) {
    if (threadIdx.x == 0) *slot = (long long)(atomicAdd(p.ticket, 1ull) - p.ticket_base);
    __syncthreads();
    return *slot;
}

// Wait (warp 0, bounded) until jobs [j0, j1) of this call are complete; false
// after about a second, with the timeout bit set.  The whole CTA returns the
// same answer and may then read the jobs' results around L1.
__device__ __forceinline__ bool wait_jobs(const Params& p, int j0, int j1, int* flag) {
    if (threadIdx.x < 32) {
        const long long t0 = clock64();
        int ok = 1;
        while (true) {
            bool mine = true;
            for (int j = j0 + (int)threadIdx.x; j < j1; j += 32) mine &= ld_acquire(&p.jobready[j]) == p.epoch;
            if (__all_sync(0xffffffffu, mine)) break;
            if (__shfl_sync(0xffffffffu, (int)(clock64() - t0 > kPrepSpinCycles), 0)) {
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        if (threadIdx.x == 0) {
            *flag = ok;
            if (!ok) atomicOr(p.status, 2u);
        }
    }
    __syncthreads();
    const int ok = *flag;
    __syncthreads();
    return ok != 0;
}

// Run preparation job j (Z: the CTA's free FFT buffer) and mark it complete.
__device__ inline void prep_job(const Params& p, int j, float2* Z, Shared& sh, int* flag) {
    const int R1 = spec_r1(p.Wb), nt = blockDim.x, m = p.Wb / 2;
    const int C = (m + 1 + nt - 1) / nt;
    if (j < R1) {
        spec_subfft(p, j, Z);
    } else if (j < R1 + C) {
        if (wait_jobs(p, 0, R1, flag)) {
            const int k = (j - R1) * nt + (int)threadIdx.x;
            if (k <= m) spec_combine(p, k);
        }
    } else {
        spec_stats(p, sh);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release(&p.jobready[j], p.epoch);
}

}  // namespace apx
