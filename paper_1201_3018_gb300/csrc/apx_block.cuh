// apx_block.cuh -- per-block prologue and epilogue shared by the direct and
// FFT cores: window load, block statistics (a3), the Section IV.D selector
// (a4), integer digit extraction (Eqs. 11-15 and the asymmetric "successive
// iterations"), inverse companding (Eq. 16) and output placement (Eq. 17).
#pragma once

#include "apx_internal.cuh"

namespace apx {

struct BlockGeom {
    long long start;  // input index of window element 0
    int lo, hi;       // local outputs kept: [lo, hi)
    int wstart;       // W_start of Eq. (10)
};

// Section III / Eq. (17): block origin and kept outputs.  Direct core: block 0
// starts at 0 and keeps [0, W+N'-1); block w >= 1 starts at wW-2 and keeps
// [N'+1, W_block).  FFT core: `head` leading blocks, all of the second kind.
__device__ __forceinline__ BlockGeom block_geom(const Params& p, long long i) {
    BlockGeom g;
    if (p.fft) {
        g.start = (i - p.head) * (long long)p.W - 2;
        g.lo = p.Nodd + 1; g.hi = p.Wb; g.wstart = (p.Nodd - 1) / 2;
    } else if (i == 0) {
        g.start = 0; g.lo = 0; g.hi = p.Wb - 2; g.wstart = 0;
    } else {
        g.start = i * (long long)p.W - 2;
        g.lo = p.Nodd + 1; g.hi = p.Wb; g.wstart = (p.Nodd - 1) / 2;
    }
    return g;
}

// Elements from a up to its next 16-byte boundary (FP32 and int32 arrays are
// 4-byte aligned).
__device__ __forceinline__ int head16(const void* a) {
    return (int)((4u - ((uint32_t)reinterpret_cast<uintptr_t>(a) >> 2)) & 3u);
}

// Coalesced window load into shared memory (xs 16-byte aligned), zeros
// outside [0, L).  Where the window starts on an even sample of the signal
// (W_block and the block origins are even), 16-byte loads between the
// signal's 16-byte boundaries: with the boundary h = 0 samples in, 16-byte
// shared-memory stores; with h = 2 (a block origin wW - 2 with W a multiple of
// 4), two 8-byte stores, lanes 8 .. 15 and 24 .. 31 of a warp storing their
// halves in the other order so that each store hits every bank at most twice
// (256 bytes in two wavefronts); the samples before the first boundary and
// after the last one one at a time.  Otherwise single samples.
__device__ __forceinline__ void load_window(const Params& p, const BlockGeom& g, float* xs) {
    const float* __restrict__ s = p.s;
    const int h = head16(s + g.start);
    if ((h & 1) == 0) {
        const int nq = (p.Wb - h) >> 2, tail = h + 4 * nq;
        const bool swap = (threadIdx.x & 8) != 0;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            const int t = h + 4 * q;
            const long long gi = g.start + t;
            float4 v;
            if (gi >= 0 && gi + 3 < p.L) {
                v = APX_LD_IN(reinterpret_cast<const float4*>(s + gi));
            } else {
                v.x = (gi >= 0 && gi < p.L) ? APX_LD_IN(&s[gi]) : 0.f;
                v.y = (gi + 1 >= 0 && gi + 1 < p.L) ? APX_LD_IN(&s[gi + 1]) : 0.f;
                v.z = (gi + 2 >= 0 && gi + 2 < p.L) ? APX_LD_IN(&s[gi + 2]) : 0.f;
                v.w = (gi + 3 >= 0 && gi + 3 < p.L) ? APX_LD_IN(&s[gi + 3]) : 0.f;
            }
            if (h == 0) {
                *reinterpret_cast<float4*>(xs + t) = v;
            } else {
                const float2 a = make_float2(v.x, v.y), b = make_float2(v.z, v.w);
                *reinterpret_cast<float2*>(xs + t + (swap ? 2 : 0)) = swap ? b : a;
                *reinterpret_cast<float2*>(xs + t + (swap ? 0 : 2)) = swap ? a : b;
            }
        }
        if ((int)threadIdx.x < h + (p.Wb - tail)) {  // at most 2 + 3 samples
            const int t = (int)threadIdx.x < h ? (int)threadIdx.x : tail + ((int)threadIdx.x - h);
            const long long gi = g.start + t;
            xs[t] = (gi >= 0 && gi < p.L) ? APX_LD_IN(&s[gi]) : 0.f;
        }
    } else {
        for (int t = threadIdx.x; t < p.Wb; t += blockDim.x) {
            const long long gi = g.start + t;
            xs[t] = (gi >= 0 && gi < p.L) ? APX_LD_IN(&s[gi]) : 0.f;
        }
    }
    __syncthreads();
}

// Eq. (17) on a whole CTA: output j of the block, kept where g.lo <= j < g.hi
// and 0 <= g.start + j < out_len, is out(j, rq_j) (rq_j: its integer, where
// integers are asked for).  The kept outputs go out as 16-byte stores between
// the 16-byte boundaries of r, one by one at the ragged ends.  ONE: a single
// inlined copy of out (a long unpacking) in a loop over the four outputs.
template <bool ONE = false, class F>
__device__ __forceinline__ void store_kept(const Params& p, const BlockGeom& g, F out) {
    const long long olo = g.start + g.lo > 0 ? g.start + g.lo : 0;
    const long long ohi = g.start + g.hi < p.out_len ? g.start + g.hi : p.out_len;
    if (olo >= ohi) return;
    const long long oa = olo + head16(p.r + olo) < ohi ? olo + head16(p.r + olo) : ohi;
    const int nq = (int)((ohi - oa) >> 2);
    const long long ot = oa + 4ll * nq;
    const bool rq4 = p.rq && head16(p.rq + oa) == 0;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const long long o = oa + 4ll * q;
        const int j = (int)(o - g.start);
        float4 v;
        int4 iv;
        if (ONE) {
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                int ic;
                const float x = out(j + c, ic);
                v.x = c == 0 ? x : v.x; iv.x = c == 0 ? ic : iv.x;
                v.y = c == 1 ? x : v.y; iv.y = c == 1 ? ic : iv.y;
                v.z = c == 2 ? x : v.z; iv.z = c == 2 ? ic : iv.z;
                v.w = c == 3 ? x : v.w; iv.w = c == 3 ? ic : iv.w;
            }
        } else {
            v.x = out(j, iv.x);
            v.y = out(j + 1, iv.y);
            v.z = out(j + 2, iv.z);
            v.w = out(j + 3, iv.w);
        }
        *reinterpret_cast<float4*>(p.r + o) = v;
        if (rq4) {
            *reinterpret_cast<int4*>(p.rq + o) = iv;
        } else if (p.rq) {
            p.rq[o] = iv.x; p.rq[o + 1] = iv.y; p.rq[o + 2] = iv.z; p.rq[o + 3] = iv.w;
        }
    }
    const int nh = (int)(oa - olo), nt = (int)(ohi - ot);
    if ((int)threadIdx.x < nh + nt) {  // at most 3 + 3 outputs
        const long long o = (int)threadIdx.x < nh ? olo + threadIdx.x : ot + ((int)threadIdx.x - nh);
        int iv;
        const float v = out((int)(o - g.start), iv);
        p.r[o] = v;
        if (p.rq) p.rq[o] = iv;
    }
}

struct Shared {
    float redf[32];
    int redi[32];
    long long redl[32];
    double bcast[3];
};

// Tap n of the convolution kernel: reversed for cross-correlation
// (xcorr(s, t) = conv(s, reverse(t)); the paper only names Matlab's xcorr),
// zero past N (the odd-length pad of Section III).
__device__ __forceinline__ float ktap(const Params& p, int n) {
    return n < p.N ? APX_LD_IN(&p.k[p.xcorr ? p.N - 1 - n : n]) : 0.f;
}

// Fixed-point second-moment sum: q = trunc(x 2^sh) with ||x||_inf 2^sh in
// [2^23, 2^24); 2^sh is applied as two exact power-of-two products.
struct FxScale {
    int sh;
    float fa, fb;
};
__device__ __forceinline__ FxScale fx_scale(float maxabs) {
    int e;
    (void)frexpf(maxabs, &e);
    FxScale f;
    f.sh = 24 - e;
    const int a = f.sh / 2, b = f.sh - a;
    f.fa = __int_as_float((a + 127) << 23);
    f.fb = __int_as_float((b + 127) << 23);
    return f;
}
__device__ __forceinline__ long long fx_sq(const FxScale& f, float x) {
    const long long q = __float2int_rz(__fmul_rn(__fmul_rn(x, f.fa), f.fb));
    return q * q;
}
// sum q^2 * 2^(-2 sh) / n, one thread, broadcast through shared memory
__device__ __forceinline__ double fx_moment(long long sum, const FxScale& f, int n, Shared& sh) {
    if (threadIdx.x == 0) {
        const double v = ldexp(__ll2double_rn(sum), -2 * f.sh);
        // dividing by a power of two is exact: the same bits without the FP64 divide
        sh.bcast[0] = (n & (n - 1)) == 0 ? ldexp(v, -(31 - __clz(n))) : __ddiv_rn(v, (double)n);
    }
    __syncthreads();
    const double v = sh.bcast[0];
    __syncthreads();
    return v;
}

struct KStats {
    float Mk;
    int bad;
    double sig2k;
    float sig2k_f, thr_f;  // sig2k and the call's SNR threshold rounded to FP32 (the model's FP32 screen)
};

// ||k||_inf and, when a packing candidate needs it, the kernel's second moment
// over its N taps (block-wide); taps are fetched 8 per thread at a time so the
// loads overlap.
constexpr int kTapBatch = 8;
__device__ inline KStats kernel_stats(const Params& p, Shared& sh) {
    float m = 0.f;
    int bad = 0;
    const int step = kTapBatch * blockDim.x;
    for (int n0 = threadIdx.x; n0 < p.N; n0 += step) {
        float v[kTapBatch];
#pragma unroll
        for (int u = 0; u < kTapBatch; ++u) v[u] = ktap(p, n0 + u * blockDim.x);
#pragma unroll
        for (int u = 0; u < kTapBatch; ++u) {
            const float a = fabsf(v[u]);
            if (!(a <= 3.402823466e38f)) bad = 1;
            m = fmaxf(m, a);
        }
    }
    KStats k;
    k.Mk = block_reduce<float, true>(m, sh.redf);
    k.bad = block_reduce<int, true>(bad, sh.redi);
    k.sig2k = 0.0;
    if (!k.bad && k.Mk > 0.f && p.ncand > 0) {  // the moment feeds only the packing candidates' model
        const FxScale f = fx_scale(k.Mk);
        long long acc = 0;
        for (int n0 = threadIdx.x; n0 < p.N; n0 += step) {
            float v[kTapBatch];
#pragma unroll
            for (int u = 0; u < kTapBatch; ++u) v[u] = ktap(p, n0 + u * blockDim.x);
#pragma unroll
            for (int u = 0; u < kTapBatch; ++u) acc += fx_sq(f, v[u]);
        }
        acc = block_reduce<long long, false>(acc, sh.redl);
        k.sig2k = fx_moment(acc, f, p.N, sh);
    }
    k.sig2k_f = (float)k.sig2k;
    k.thr_f = (float)p.thr;
    return k;
}

// Companded tap k~[n] = rint(c_k k[n]) (Eq. 2); zero past N.
__device__ __forceinline__ long long kq(const Params& p, float ck, int n) {
    return n < p.N ? (long long)compand(ck, ktap(p, n)) : 0ll;
}
// Packed tap n of candidate c as an exact integer: symmetric (Eq. 5, reading
// c2) k~[2n+1] + 2^b k~[2n]; asymmetric k~[n].
__device__ __forceinline__ long long kbar_int(const Params& p, const Cand& c, float ck, int n) {
    if (n >= c.nk) return 0ll;
    if (c.blk == APX_BLK_SYM) return kq(p, ck, 2 * n + 1) + (kq(p, ck, 2 * n) << c.b);
    return kq(p, ck, n);
}
// ||kbar||_1, exact (block-wide), packed taps fetched in batches.
__device__ inline long long kbar_l1(const Params& p, const Cand& c, float ck, Shared& sh) {
    long long l1 = 0;
    const int step = kTapBatch * blockDim.x;
    for (int n0 = threadIdx.x; n0 < c.nk; n0 += step) {
        long long v[kTapBatch];
#pragma unroll
        for (int u = 0; u < kTapBatch; ++u) v[u] = kbar_int(p, c, ck, n0 + u * blockDim.x);
#pragma unroll
        for (int u = 0; u < kTapBatch; ++u) l1 += v[u] < 0 ? -v[u] : v[u];
    }
    return block_reduce<long long, false>(l1, sh.redl);
}

// Fill every kept output of the block with `v` (zero block or non-finite).
__device__ __forceinline__ void store_constant(const Params& p, const BlockGeom& g, float v) {
    store_kept(p, g, [v](int, int& iv) { iv = 0; return v; });
}

__device__ __forceinline__ void write_stats(const Params& p, long long i, int mode, const Cand* c, float cs,
                                            float Ms, double sig2, double snr_db, double ferr) {
    if (!p.st || threadIdx.x != 0) return;
    apx_block_stats s;
    s.mode = mode;
    s.Sq = c ? c->S : 0;
    s.Kq = c ? c->K : 0;
    s.b = c ? c->b : 0;
    s.cs = cs;
    s.maxabs = Ms;
    s.sigma2 = sig2;
    s.snr_pred_db = snr_db;
    s.fft_err = ferr;
    p.st[i] = s;
}

// Prologue result.
// A block's maximum and second moment.  The moment stays the exact
// fixed-point sum acc (scale 2^fsh) in every thread; pro_sig2 gives the FP64
// value (as fx_moment rounds it) where a thread needs it, and s2s_f its FP32
// approximation for the model's FP32 screen.
struct Pro {
    int kind;     // 0 full / packed decided later, 2 zero, 3 non-finite
    float Ms;
    long long acc;
    int fsh;
    float s2s_f;
};

// The FP32 approximation of sum q^2 * 2^(-2 sh) / n (sum >= 0): within 2^-22
// relative where the result is a normal number.
__device__ __forceinline__ float fx_moment_f32(long long sum, int sh, int n) {
    const float hi = (float)(int)(sum >> 32), lo = (float)(unsigned)(sum & 0xffffffffll);
    return __fdiv_rn(ldexpf(fmaf(hi, 4294967296.f, lo), -2 * sh), (float)n);
}

// The block's second moment in FP64, the same bits as fx_moment.
__device__ __forceinline__ double pro_sig2(const Pro& r, int n) {
    if (r.kind != 0) return 0.0;
    const double v = ldexp(__ll2double_rn(r.acc), -2 * r.fsh);
    return (n & (n - 1)) == 0 ? ldexp(v, -(31 - __clz(n))) : __ddiv_rn(v, (double)n);
}

__device__ __forceinline__ Pro block_prologue(const Params& p, const float* xs, const KStats& ks, Shared& sh) {
    Pro r;
    r.Ms = block_maxabs(xs, p.Wb, sh.redf, sh.redi);
    r.acc = 0;
    r.fsh = 0;
    r.s2s_f = 0.f;
    if (!(r.Ms <= 3.402823466e38f) || ks.bad) { r.kind = 3; return r; }  // NaN or inf
    if (r.Ms == 0.f || ks.Mk == 0.f) { r.kind = 2; return r; }
    const FxScale f = fx_scale(r.Ms);
    long long acc = 0;
    for (int t = threadIdx.x; t < p.Wb; t += blockDim.x) acc += fx_sq(f, xs[t]);
    r.acc = block_reduce<long long, false>(acc, sh.redl);
    r.fsh = f.sh;
    r.s2s_f = fx_moment_f32(r.acc, f.sh, p.Wb);
    r.kind = 0;
    return r;
}

// feasible_mask for a block of the direct cores: lane c of warp 0 decides
// candidate c by the FP32 screen and evaluates the FP64 model only where the
// screen leaves it open, so that the FP64 chain (a slow pipe on this part)
// rarely runs; the decisions are snr_feasible's, bit for bit.
__device__ inline unsigned feasible_mask_pro(const Params& p, const Pro& pr, const KStats& ks, unsigned* slot) {
    if (threadIdx.x < 32) {
        const int c = threadIdx.x;
        bool ok = false;
        if (c < p.ncand) {
            if (!p.autosel) {
                ok = true;
            } else {
                const int S = p.cand[c].S, K = p.cand[c].K;
                const int sc = snr_screen(pr.s2s_f, pr.Ms, ks.sig2k_f, ks.Mk, S, K, ks.thr_f);
                ok = sc > 0 || (sc == 0 && snr_feasible(pro_sig2(pr, p.Wb), pr.Ms, ks.sig2k, ks.Mk, S, K, p.thr));
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (c == 0) *slot = m;
    }
    __syncthreads();
    return *slot;
}

__device__ __forceinline__ void handle_trivial(const Params& p, long long i, const BlockGeom& g, const Pro& pr) {
    if (pr.kind == 3) {
        store_constant(p, g, __int_as_float(0x7fc00000));
        if (threadIdx.x == 0) atomicOr(p.status, 1u);
        write_stats(p, i, APX_BLK_NONFINITE, nullptr, 0.f, pr.Ms, 0.0, __longlong_as_double(0x7ff8000000000000ll), 0.0);
    } else {
        store_constant(p, g, 0.f);
        write_stats(p, i, APX_BLK_ZERO, nullptr, 0.f, pr.Ms, 0.0, __longlong_as_double(0x7ff0000000000000ll), 0.0);
    }
}

// ------------------------------------------------------------------ digit extraction
// Finest-digit scaled packed output T = rbar * 2^sc as an integer.  Exact for
// the direct core; nearest for the FFT core (error bound below 1/4 digit).
__device__ __forceinline__ long long scaled(double rbar, int sc) { return __double2ll_rn(ldexp(rbar, sc)); }

// Eqs. (11)-(15) for output j of a symmetric-packed block, on u scaled by 2^b:
//   U = T + R_max (2^2b + 2^b + 1)                     (11)
//   side_eps^-1 = U >> 2b                                 (13)
//   side_eps    = R_max (m = W_start) or U[m-1] mod 2^b   (12)
//   r~[2m]   = side_eps^-1 + side_eps - 2 R_max          (14)
//   r~[2m+1] = (U >> b) - 2^b side_eps^-1 - R_max         (15)
template <typename F>
__device__ __forceinline__ long long unpack_sym(const Cand& c, int j, int wstart, F Tat) {
    const int m = j >> 1;
    const long long one = 1;
    const long long Rs = c.Rmax * ((one << (2 * c.b)) + (one << c.b) + 1);
    const long long U = Tat(m) + Rs;
    const long long sinv = U >> (2 * c.b);
    if (j & 1) return (U >> c.b) - (sinv << c.b) - c.Rmax;
    const long long se = (m == wstart) ? c.Rmax : ((Tat(m - 1) + Rs) & ((one << c.b) - 1));
    return sinv + se - 2 * c.Rmax;
}

// The paper's own form (APX_LITERAL): eps = (2 R_max)^-1 (Eq. 6) and Eqs.
// (11)-(15) in FP64 on the packed outputs rbar, with R_safe = R_max (eps + 1 +
// eps^-1) + u_sys eps^-1 and u_sys = 3.1193e-11 (Section IV).  Every operation
// is one correctly rounded FP64 step in the order the equations give them
// (no contraction), so the result is a function of rbar alone; rounding can
// move a digit, which is what the paper's SNR measurements include.
constexpr double kUsys = 3.1193e-11;
__device__ __forceinline__ long long unpack_sym_literal(const Cand& c, int j, int wstart, const double* rbar) {
    const int m = j >> 1;
    const double R = (double)c.Rmax, eps = c.eps_l, einv = __ddiv_rn(1.0, eps);
    const double Rsafe = __dadd_rn(__dmul_rn(R, __dadd_rn(__dadd_rn(eps, 1.0), einv)), __dmul_rn(kUsys, einv));
    const double u = __dadd_rn(rbar[m], Rsafe);                                  // (11)
    const double sinv = floor(__dmul_rn(eps, u));                                 // (13)
    if (j & 1) return (long long)floor(__dsub_rn(__dsub_rn(floor(u), __dmul_rn(einv, sinv)), R));  // (15)
    double se = R;                                                                // (12)
    if (m != wstart) {
        const double up = __dadd_rn(rbar[m - 1], Rsafe);
        se = __dmul_rn(einv, __dsub_rn(up, floor(up)));
    }
    return (long long)floor(__dsub_rn(__dadd_rn(sinv, se), __dmul_rn(2.0, R)));   // (14)
}
// Eq. (5) with the paper's eps^-1 = 2 R_max (pair order as in kbar_int): an
// exact integer in FP64.
__device__ __forceinline__ double kbar_literal(const Params& p, const Cand& c, float ck, int n) {
    if (n >= c.nk) return 0.0;
    return __dadd_rn((double)kq(p, ck, 2 * n + 1), __dmul_rn(__dmul_rn(2.0, (double)c.Rmax), (double)kq(p, ck, 2 * n)));
}

// Asymmetric unpacking: digit q of T[i] offset by R_max, overlap-added over the
// M segments: r~[j] = sum_q c_q[j - q Ls], with packed outputs i < nr.
template <typename F>
__device__ __forceinline__ long long unpack_asym(const Cand& c, int j, int Ls, int nr, F Tat) {
    const long long one = 1;
    const long long mask = (one << c.b) - 1;
    long long off = 0;
    for (int q = 0; q < c.M; ++q) off += c.Rmax << (c.b * q);
    long long acc = 0;
    for (int q = 0; q < c.M; ++q) {
        const int i = j - q * Ls;
        if (i < 0 || i >= nr) continue;
        const long long U = Tat(i) + off;
        acc += ((U >> (c.b * (c.M - 1 - q))) & mask) - c.Rmax;
    }
    return acc;
}

// real word w of a padded complex buffer
template <typename R, typename C>
__device__ __forceinline__ R& word(C* Z, int w) {
    return reinterpret_cast<R*>(Z)[2 * pad16(w >> 1) + (w & 1)];
}

// H = FFT_n(taps) / (4m), k in [0, m], natural order, through the block FFT;
// tap(j) gives tap j; tw holds exp(-2 pi i t / ntab).  Z is scratch of
// padded_len(n/2) entries.
template <typename R, typename C, typename F>
__device__ void spectrum_of(F tap, int ntab, int n, const C* __restrict__ tw, C* H, C* Z) {
    const int m = n / 2;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        C v;
        v.x = tap(2 * j);
        v.y = tap(2 * j + 1);
        Z[pad16(j)] = v;
    }
    __syncthreads();
    fft_smem<C, false>(Z, m, tw, ntab);
    const R scale = (R)1 / (R)(8 * m);
    for (int k = threadIdx.x; k <= m; k += blockDim.x) {
        C X;
        if (k == 0 || k == m) {
            const C z0 = Z[0];
            X.x = 2 * (k == 0 ? z0.x + z0.y : z0.x - z0.y);
            X.y = 0;
        } else {
            C Xmk;
            real_post(Z[pad16(fft_perm<C>(k, m))], Z[pad16(fft_perm<C>(m - k, m))], __ldg(&tw[k * (ntab / n)]), X, Xmk);
        }
        X.x *= scale; X.y *= scale;
        H[k] = X;
    }
    __syncthreads();
}

}  // namespace apx
