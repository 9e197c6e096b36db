// apx_internal.cuh -- device-side building blocks of libapx (sm_103a).
//
// Block statistics, the per-block selector arithmetic, companding, packing,
// digit extraction and an in-shared-memory radix-8/4/2 Stockham FFT.  Every
// floating-point decision that selects an integer (a quantised code, a mode)
// is taken with one IEEE operation at a time (__fmul_rn, __dmul_rn, ...) so
// that it does not depend on contraction or summation order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/apx.h"


// Device-side bounds checks of builds with -DAPX_CHECKED: a failed check sets
// bit 2 of the status word (APX_ERR_CHECK from apx_sync) and the guarded
// access is skipped.  Other builds compile the checks away.
#ifdef APX_CHECKED
#define APX_IN_BOUNDS(cond, status) ((cond) ? true : ((status) ? (atomicOr((status), 4u), false) : false))
#else
#define APX_IN_BOUNDS(cond, status) true
#endif

// Loads of a call's input samples and taps: through the read-only data cache,
// except in the serving engine's persistent kernel, whose requests may reuse
// an input buffer with new contents during its lifetime; its translation unit
// defines APX_INPUT_COHERENT, and its loads stay inside the memory model
// (plain loads, ordered after the acquire that published the request).
#ifdef APX_INPUT_COHERENT
#define APX_LD_IN(ptr) (*(ptr))
#else
#define APX_LD_IN(ptr) __ldg(ptr)
#endif

namespace apx {

constexpr int kMaxWblock = 16384;
constexpr int kMaxCand = 3;

// One packing candidate (set by the host from N' and W_block).
struct Cand {
    int blk;          // APX_BLK_SYM / ASYM2 / ASYM3, or APX_BLK_TC (the direct core's tensor-core candidate)
    int M;            // 1 for symmetric, 2 or 3 for asymmetric
    int S, K, b;      // companding ranges and eps = 2^-b
    int sc;           // exponent of the finest digit: b (sym, asym2) or 2b (asym3)
    long long Rmax;   // N' S K (Eq. 3)
    int nk;           // packed taps: (N'+1)/2 (sym) or N' (asym)
    int log2n;        // FFT core: log2 of the real transform length
    double fftc;      // FFT core: (3 phi + 16 u) for log2n (error-bound constant)
    double2* H;       // FFT core: kernel spectrum FFT_n(kbar) / (4m), m+1 entries (built on demand)
    int literal;      // APX_LITERAL: eps = eps_l = (2 R_max)^-1, FP64 unpacking with u_sys
    double eps_l;
};

// Kernel statistics published by the FFT core's spectrum launch.
struct KInfo {
    float Mk;             // ||k||_inf
    int bad;              // kernel has NaN/Inf
    double sig2k;         // second moment of the kernel (24-bit fixed point)
    double l1[kMaxCand];  // ||kbar||_1 of each candidate, exact integer
};

// Shared-memory layout of the direct kernel (byte offsets; element pads).
struct DirectLayout {
    int padF;         // zero floats in front of the window
    int offK;         // FP32 taps: byte offset (nkp32 floats)
    int offS, padS;   // packed-signal buffer: byte offset, zero doubles in front
    int nS;           // packed-signal buffer length in doubles (pads included)
    int offT;         // packed-output buffer: byte offset
    int offKb;        // packed taps: byte offset
};

struct Params {
    const float* s;       // input, L samples
    long long L;
    const float* k;       // kernel taps as given (the template for cross-correlation)
    int N, Nodd, Wb, W, head, fft, xcorr;
    int pf;               // FFT core, single call with the spectrum launches: k_spec prefetches the signal into L2
    long long P, out_len;
    float* r;             // output, out_len
    int* rq;              // integer-domain output or null
    apx_block_stats* st;  // per-block stats or null
    float2* Hfull;        // FFT core: FP32 spectrum FFT_n(k) / (4m), m+1 entries
    float2* Ysub;         // FFT core: spectra of the R1 decimated tap sequences (n entries)
    float2* Hpair;        // FFT core, two-CTA kernel: H and the real-step twiddles in the order its
                          // CTAs stage them (2 x 15 x W_block/32 entries), or null
    KInfo* ki;            // FFT core: kernel statistics from the spectrum launch
    const double2* tw64;  // twiddles exp(-2 pi i t / ntab), t in [0, ntab)
    const float2* tw32;
    int ntab;             // twiddle table length: a power of two >= W_block
    unsigned* status;     // bit 0: non-finite input seen; bit 1: a bounded wait gave up
    unsigned* claim;      // FFT core, per candidate: last call that claimed building its spectrum
    unsigned* ready;      // FFT core, per candidate: last call whose spectrum is complete
    unsigned epoch;       // FFT core: this call's number (never 0)
    int fused;            // FFT core, single call: the block kernel's first CTAs run the kernel preparation
    unsigned long long* ticket;     // fused: CTA ticket counter (only grows)
    unsigned long long ticket_base; // fused: its value before this launch
    unsigned* jobready;   // fused, per preparation job: last call in which it completed
    int autosel;          // 1: per-block selection under thr
    int full64;           // direct core, no packing: full precision in FP64
    int ncand;
    unsigned claim_init;  // FFT core, three-launch single call: value k_spec writes to the claim words
                          // (0; the call's epoch when a test stalls the builders)
    double thr;           // 10^(target/10)
    Cand cand[kMaxCand];
    DirectLayout dl;      // direct core
};

// Two-CTA form of the FP32 block kernel (apx_fft_pair.cu): with radix-8
// passes the first forward pass sends output digit r to the class of slots
// [r S, r S + S), S = m/8; CTA 0 holds classes {0, 1, 4, 7}, CTA 1 classes
// {2, 3, 5, 6} (each set closed under r -> -r mod 8, so frequencies k and m-k
// meet in one CTA).  pair_owner(r): the CTA holding class r; pair_local(r):
// its position among that CTA's four classes (ascending class order).
constexpr unsigned kPairMask1 = 0x6Cu;  // the classes of CTA 1
__host__ __device__ __forceinline__ int pair_owner(int r) { return (int)((kPairMask1 >> r) & 1u); }
__host__ __device__ __forceinline__ int pair_local(int r) {
    const unsigned mine = pair_owner(r) ? kPairMask1 : (~kPairMask1 & 0xFFu);
    unsigned below = mine & ((1u << r) - 1u), c = 0;
    while (below) { c += below & 1u; below >>= 1; }
    return (int)c;
}
// Entry of the pair-ordered spectrum table for frequency k <= m/2: CTA `rank`,
// thread t, item u (k = 8 t + c_u, or u = 4 for k = m/2 in CTA 0, thread 0).
// Item u of thread t holds H[k], H[m-k], W^k at (3u + a) nt + t, a = 0, 1, 2,
// after rank * 15 nt; nt = m/16 threads per CTA.
__host__ __device__ __forceinline__ void pair_entry(int k, int m, int* rank, int* u, int* t) {
    if (k == m / 2) { *rank = 0; *u = 4; *t = 0; return; }
    const int c = k & 7;
    *rank = pair_owner(c); *u = pair_local(c); *t = k >> 3;
}

// The direct core's tensor-core candidate (APX_CORE_TC): a block's outputs as
// rows of kTcbRow phases (at most 128 rows, one MMA tile), its companded
// window as rows of kTcbRow samples behind a shift of KN = kTcbRow
// ceil((N'-1) / kTcbRow) zeros, the Toeplitz band of its taps in K slices of
// kTcbRow (KN / kTcbRow + 1 slices).  Exact while |s~|, |k~| <= 2048 (FP16)
// and N' S_q K_q <= 2^24 (FP32 sums of integers).
constexpr int kTcbRow = 64;
constexpr int kTcbMaxSlices = 8;
constexpr int kTcbQMax = 2048;
constexpr long long kTcbSumMax = 1LL << 24;
__host__ __device__ constexpr int tcb_kshift(int Nodd) { return (Nodd - 1 + kTcbRow - 1) / kTcbRow * kTcbRow; }
__host__ __device__ constexpr int tcb_kslices(int Nodd) { return tcb_kshift(Nodd) / kTcbRow + 1; }
// blocks per CTA of the tensor-core kernel (its setup is shared by them)
constexpr int kTcbBlocks = 12;
__host__ __device__ constexpr long long tcb_ctas(long long P) { return (P + kTcbBlocks - 1) / kTcbBlocks; }

// Several requests in one launch: request r owns CTAs [cta_start[r], cta_start[r+1]).
struct BatchTab {
    const Params* reqs;
    const int* cta_start;
    int nreq;
};

// The request of this CTA (binary search) and the CTA's index within it; the
// request's parameters are copied into shared memory `sp`.
__device__ __forceinline__ long long batch_enter(const BatchTab& t, Params& sp) {
    int lo = 0, hi = t.nreq;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&t.cta_start[mid]) <= (int)blockIdx.x) lo = mid; else hi = mid;
    }
    const int* src = reinterpret_cast<const int*>(&t.reqs[lo]);
    int* dst = reinterpret_cast<int*>(&sp);
    for (int w = threadIdx.x; w < (int)(sizeof(Params) / sizeof(int)); w += blockDim.x) dst[w] = __ldg(&src[w]);
    __syncthreads();
    return (long long)blockIdx.x - __ldg(&t.cta_start[lo]);
}

// ------------------------------------------------------------------ reductions
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide reduction; `red` is shared scratch of >= 32 elements of T.
// Every warp reduces the per-warp partials itself (the same values in the
// same shuffle order, so every thread gets the same bits), which takes two
// barriers: the partials written, then read by everyone before any thread
// writes `red` again.  Other users of the scratch end with a barrier after
// their last read, so none is needed before the partials are written.
template <typename T, bool IS_MAX>
__device__ T block_reduce(T v, T* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = IS_MAX ? warp_max(v) : warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T t = lane < nw ? red[lane] : (IS_MAX ? red[0] : T(0));
    t = IS_MAX ? warp_max(t) : warp_sum(t);
    __syncthreads();
    return t;
}

// ||x||_inf over n samples in shared memory; returns NaN if any sample is NaN
// and +inf if any is infinite.
// One integer reduction: the bit patterns of non-negative floats order as the
// values, and every NaN pattern lies above +inf (0x7f800000).
__device__ inline float block_maxabs(const float* x, int n, float* redf, int* redi) {
    (void)redf;
    int mb = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mb = max(mb, __float_as_int(x[i]) & 0x7fffffff);
    mb = block_reduce<int, true>(mb, redi);
    return mb > 0x7f800000 ? __int_as_float(0x7fc00000) : __int_as_float(mb);
}

// Table 1 model (derived from Eqs. 18-19), one IEEE operation at a time:
//   144 s2s s2k S^2 K^2 >= thr (12 (s2s S^2 Mk^2 + s2k K^2 Ms^2) + Ms^2 Mk^2)
__device__ inline bool snr_feasible(double s2s, float Ms, double s2k, float Mk, int S, int K, double thr) {
    double S2 = __dmul_rn((double)S, (double)S), K2 = __dmul_rn((double)K, (double)K);
    double Ms2 = __dmul_rn((double)Ms, (double)Ms), Mk2 = __dmul_rn((double)Mk, (double)Mk);
    double num = __dmul_rn(__dmul_rn(144.0, __dmul_rn(s2s, s2k)), __dmul_rn(S2, K2));
    double a = __dmul_rn(__dmul_rn(s2s, S2), Mk2);
    double c = __dmul_rn(__dmul_rn(s2k, K2), Ms2);
    double den = __dadd_rn(__dmul_rn(12.0, __dadd_rn(a, c)), __dmul_rn(Ms2, Mk2));
    return num >= __dmul_rn(thr, den);
}

// The same comparison in FP32, as a screen: +1 feasible, -1 not, 0 undecided
// (left to snr_feasible).  With every operand and intermediate in [1e-30,
// 1e30] (normal, finite) each FP32 value is within 2^-20 relative of its FP64
// counterpart (inputs rounded once, a few products of non-negative terms), so
// a decision with a margin of 2^-14 between the two sides is the one the FP64
// comparison takes.
__device__ inline int snr_screen(float s2s, float Ms, float s2k, float Mk, int S, int K, float thr) {
    const float S2 = (float)S * (float)S, K2 = (float)K * (float)K;
    const float Ms2 = Ms * Ms, Mk2 = Mk * Mk;
    const float ss = s2s * s2k, SK = S2 * K2, t144 = 144.f * ss;
    const float num = t144 * SK;
    const float sa = s2s * S2, a = sa * Mk2;
    const float kc = s2k * K2, c = kc * Ms2;
    const float mm = Ms2 * Mk2, den = 12.f * (a + c) + mm;
    const float rhs = thr * den;
    const float lo = fminf(fminf(fminf(fminf(s2s, s2k), fminf(Ms2, Mk2)), fminf(fminf(ss, SK), fminf(t144, num))),
                           fminf(fminf(fminf(sa, a), fminf(kc, c)), fminf(fminf(mm, den), fminf(rhs, thr))));
    const float hi = fmaxf(fmaxf(fmaxf(fmaxf(s2s, s2k), fmaxf(Ms2, Mk2)), fmaxf(fmaxf(ss, SK), fmaxf(t144, num))),
                           fmaxf(fmaxf(fmaxf(sa, a), fmaxf(kc, c)), fmaxf(fmaxf(mm, den), fmaxf(rhs, thr))));
    if (!(lo >= 1e-30f && hi <= 1e30f)) return 0;
    const float marg = 1.f + 0x1p-14f;
    if (num >= rhs * marg) return 1;
    if (num * marg <= rhs) return -1;
    return 0;
}

__device__ inline double snr_model_db(double s2s, float Ms, double s2k, float Mk, int S, int K) {
    double S2 = (double)S * S, K2 = (double)K * K, Ms2 = (double)Ms * Ms, Mk2 = (double)Mk * Mk;
    double num = 144.0 * (s2s * s2k) * (S2 * K2);
    double den = 12.0 * (s2s * S2 * Mk2 + s2k * K2 * Ms2) + Ms2 * Mk2;
    return 10.0 * log10(num / den);
}

// Section IV.D model check of every candidate at once: bit c of the result is
// set when candidate c's model SNR meets the target (every candidate when
// selection is off).  Lane c of warp 0 evaluates candidate c, so the FP64
// chain (a slow pipe on this part) runs once per block, not once per
// candidate; the same decisions, bit for bit.  `slot` is a shared word that no
// thread writes again before every thread has returned.
__device__ inline unsigned feasible_mask(const Params& p, double s2s, float Ms, double s2k, float Mk,
                                         unsigned* slot) {
    if (threadIdx.x < 32) {
        const int c = threadIdx.x;
        bool ok = false;
        if (c < p.ncand) ok = !p.autosel || snr_feasible(s2s, Ms, s2k, Mk, p.cand[c].S, p.cand[c].K, p.thr);
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (c == 0) *slot = m;
    }
    __syncthreads();
    return *slot;
}

// Bytes per companded sample the FFT core's asymmetric packing stages in
// shared memory: |s~| <= S_q of every candidate (Eq. 2 rounds c x with
// |c x| <= S_q), so one byte while every S_q <= 127, two up to 32767.
__host__ __device__ inline int companded_bytes(const Params& p) {
    int smax = 0;
    for (int j = 0; j < p.ncand; ++j) smax = p.cand[j].S > smax ? p.cand[j].S : smax;
    return smax <= 127 ? 1 : (smax <= 32767 ? 2 : 4);
}

// Eq. (2): c = Q / ||x||_inf (correctly rounded FP32) and x~ = rint(c x).
__device__ __forceinline__ float compand_factor(int Q, float m) { return __fdiv_rn((float)Q, m); }
__device__ __forceinline__ int compand(float c, float x) { return __float2int_rn(__fmul_rn(c, x)); }

// ------------------------------------------------------------------ complex helpers
template <typename R> struct cpx;
template <> struct cpx<float> { using T = float2; };
template <> struct cpx<double> { using T = double2; };

// Products are written out (one fused multiply-add and one rounded product per
// component, rounded products elsewhere): the device compiler would otherwise
// fuse multiplies into later additions as its schedule allows, and the block
// kernels (general, full-precision-only, two-CTA, batched) could then differ
// in the last bit.  Written this way every kernel performs the same operations.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = rfma(a.x, b.x, -rmul(a.y, b.y));
    r.y = rfma(a.x, b.y, rmul(a.y, b.x));
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// multiply by -i (forward) or +i (inverse): exact
template <typename C, bool INV> __device__ __forceinline__ C mul_mi(C a) {
    C r;
    if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}
template <typename C, bool INV> __device__ __forceinline__ C mul_w8(C a) {  // exp(-+ i pi/4)
    using R = decltype(a.x);
    const R h = (R)0.70710678118654752440;
    C r;
    if (INV) { r.x = rmul(a.x - a.y, h); r.y = rmul(a.x + a.y, h); }
    else     { r.x = rmul(a.x + a.y, h); r.y = rmul(a.y - a.x, h); }
    return r;
}
template <typename C, bool INV> __device__ __forceinline__ C mul_w83(C a) {  // exp(-+ 3 i pi/4)
    using R = decltype(a.x);
    const R h = (R)0.70710678118654752440;
    C r;
    if (INV) { r.x = rmul(-a.x - a.y, h); r.y = rmul(a.x - a.y, h); }
    else     { r.x = rmul(a.y - a.x, h); r.y = rmul(-a.x - a.y, h); }
    return r;
}

// In-register DFTs (natural order in, natural order out), built from radix-2
// butterflies so the standard radix-2 error analysis applies.
template <typename C, bool INV> __device__ __forceinline__ void dft2(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
}
template <typename C, bool INV> __device__ __forceinline__ void dft4(C* v) {
    C e0 = cadd(v[0], v[2]), e1 = csub(v[0], v[2]);
    C o0 = cadd(v[1], v[3]), o1 = mul_mi<C, INV>(csub(v[1], v[3]));
    v[0] = cadd(e0, o0); v[2] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[3] = csub(e1, o1);
}
template <typename C, bool INV> __device__ __forceinline__ void dft8(C* v) {
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4<C, INV>(e);
    dft4<C, INV>(o);
    o[1] = mul_w8<C, INV>(o[1]);
    o[2] = mul_mi<C, INV>(o[2]);
    o[3] = mul_w83<C, INV>(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) { v[k] = cadd(e[k], o[k]); v[k + 4] = csub(e[k], o[k]); }
}
// exp(-+ 2 pi i e / 16) for the exponents that occur inside a 4x4 DFT16
template <typename C, bool INV> __device__ __forceinline__ C mul_w16(C a, int e) {
    using R = decltype(a.x);
    const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173, h = (R)0.70710678118654752440;
    R wr, wi;  // forward value cos - i sin
    switch (e) {
        case 1: wr = c1; wi = -s1; break;
        case 2: wr = h; wi = -h; break;
        case 3: wr = s1; wi = -c1; break;
        case 4: return mul_mi<C, INV>(a);
        case 6: wr = -h; wi = -h; break;
        default: wr = -c1; wi = s1; break;  // e = 9
    }
    if (INV) wi = -wi;
    C r;
    r.x = rfma(a.x, wr, -rmul(a.y, wi));
    r.y = rfma(a.x, wi, rmul(a.y, wr));
    return r;
}
// DFT16 as 4 x 4: X[b + 4d] = sum_a W4^(ad) W16^(ab) sum_c x[a + 4c] W4^(cb)
template <typename C, bool INV> __device__ __forceinline__ void dft16(C* v) {
    C t[16];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        C u[4] = {v[a], v[a + 4], v[a + 8], v[a + 12]};
        dft4<C, INV>(u);
#pragma unroll
        for (int b = 0; b < 4; ++b) t[4 * a + b] = (a && b) ? mul_w16<C, INV>(u[b], a * b) : u[b];
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        C u[4] = {t[b], t[4 + b], t[8 + b], t[12 + b]};
        dft4<C, INV>(u);
#pragma unroll
        for (int d = 0; d < 4; ++d) v[b + 4 * d] = u[d];
    }
}
template <int RAD, typename C, bool INV> __device__ __forceinline__ void dft_small(C* v) {
    if constexpr (RAD == 16) dft16<C, INV>(v);
    else if constexpr (RAD == 8) dft8<C, INV>(v);
    else if constexpr (RAD == 4) dft4<C, INV>(v);
    else dft2<C, INV>(v);
}

// Shared-memory slot of complex element i: one pad element per 16 and one more
// per 256.  The passes below (strides 1, 16, 256 across a warp) and the
// spectral product (digit-reversed slots, lanes 256 elements apart) then all
// use the minimum number of shared-memory wavefronts; with the per-16 pad
// alone the digit-reversed access put 16 lanes on one bank.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4) + (i >> 8); }
__host__ __device__ constexpr int padded_len(int m) { return m + (m >> 4) + (m >> 8) + 1; }

// Twiddles w[r] = W_M^(r j), r < RAD, from a table of exp(-2 pi i t / ntab).
// FP32: one table load and products (at most four deep); FP64: one load each,
// so that every twiddle carries only the table's rounding (the FFT error bound
// assumes that).
template <typename C, int RAD, bool INV>
__device__ __forceinline__ void twiddles(C (&w)[RAD], const C* __restrict__ tw, int step) {
    using R = decltype(w[0].x);
    w[0].x = (R)1; w[0].y = (R)0;
    // plain loads: the table is in global memory or, for the FP32 passes of
    // some kernels, a copy of the bases in shared memory
    if constexpr (sizeof(R) == 8) {
#pragma unroll
        for (int r = 1; r < RAD; ++r) w[r] = tw[r * step];
    } else {
        if constexpr (RAD > 1) w[1] = tw[step];
        if constexpr (RAD > 2) { w[2] = cmul(w[1], w[1]); w[3] = cmul(w[2], w[1]); }
        if constexpr (RAD > 4) {
            w[4] = cmul(w[2], w[2]);
#pragma unroll
            for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
        }
        if constexpr (RAD > 8) {
            w[8] = cmul(w[4], w[4]);
#pragma unroll
            for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
        }
    }
    if (INV) {
#pragma unroll
        for (int r = 1; r < RAD; ++r) w[r].y = -w[r].y;
    }
}

// Radix of the main passes of a length-m transform on nt threads: the largest
// of 16, 8, 4 that still gives every thread a butterfly; FP64 transforms
// always use radix 4 (their time is set by the FP64 rate, and the small
// butterfly keeps the register count low).
// Largest radix of the FP32 passes.  8: every block kernel (the general one,
// the full-precision-only one at twice the threads, the two-CTA form) then
// takes the same radix at each length, so they give the same bits; radix-16
// butterflies measured no faster (the kernels wait on instruction fetch and
// latency, and the smaller butterfly keeps their code and registers small).
#ifndef APX_FFT_RMAX
#define APX_FFT_RMAX 8
#endif
template <typename C>
__host__ __device__ constexpr int fft_radix(int m, int nt) {
    return sizeof(C) == 16 ? 4
                           : ((APX_FFT_RMAX >= 16 && m >= 16 * nt) ? 16 : ((APX_FFT_RMAX >= 8 && m >= 8 * nt) ? 8 : 4));
}

// One in-place pass over sub-transforms of length M with radix RAD (stride
// S = M/RAD).  Forward (decimation in frequency): DFT then twiddle W_M^(r j).
// Inverse (decimation in time, the exact reverse): conjugate twiddle then
// inverse DFT.  Each butterfly reads and writes the same slots, so a pass needs
// no barrier inside; callers separate passes with __syncthreads().
//
// Slot addresses: for base = g M + j with j < S (all powers of two),
// pad16(base + q S) = pad16(base) + pad16(q S): the i >> 4 and i >> 8 terms of
// base + q S split into those of base and of q S, because base's aligned part
// g M is a multiple of 16 (of 256) whenever the run from base to base + (RAD-1)
// S crosses a multiple of 16 (of 256).  So a butterfly's slots are one pad16
// and per-q offsets, constants where S is.
template <typename C, int RAD, bool INV>
__device__ __forceinline__ void fft_pass(C* Z, int m, int M, const C* __restrict__ tw, int ntab, unsigned* st) {
    const int S = M / RAD, nbf = m / RAD;
    const int tstep = ntab / M;
    const int lS = 31 - __clz(S);  // S is a power of two: sub-transform and offset by shift and mask
    int off[RAD];
#pragma unroll
    for (int q = 0; q < RAD; ++q) off[q] = pad16(q * S);
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
        const int g = b >> lS, j = b & (S - 1);
        const int base = g * M + j;
        C v[RAD], w[RAD];
        if (!APX_IN_BOUNDS(base + (RAD - 1) * S < m, st)) continue;
        int slot[RAD];
        const int p0 = pad16(base);
#pragma unroll
        for (int q = 0; q < RAD; ++q) slot[q] = p0 + off[q];
#pragma unroll
        for (int q = 0; q < RAD; ++q) v[q] = Z[slot[q]];
        if (S > 1) twiddles<C, RAD, INV>(w, tw, j * tstep);
        if (!INV) {
            dft_small<RAD, C, false>(v);
            if (S > 1) {
#pragma unroll
                for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], w[r]);
            }
        } else {
            if (S > 1) {
#pragma unroll
                for (int r = 1; r < RAD; ++r) v[r] = cmul(v[r], w[r]);
            }
            dft_small<RAD, C, true>(v);
        }
#pragma unroll
        for (int q = 0; q < RAD; ++q) Z[slot[q]] = v[q];
    }
}

template <typename C, int R, bool INV>
__device__ __forceinline__ void fft_passes(C* Z, int m, const C* __restrict__ tw, int ntab, unsigned* st) {
    int a = 0, t = m;
    while (t >= R) { t /= R; ++a; }   // m = R^a * t, t < R
    if (!INV) {
        int M = m;
        for (int s = 0; s < a; ++s) { fft_pass<C, R, false>(Z, m, M, tw, ntab, st); __syncthreads(); M /= R; }
        if (t == 8) fft_pass<C, 8, false>(Z, m, 8, tw, ntab, st);
        else if (t == 4) fft_pass<C, 4, false>(Z, m, 4, tw, ntab, st);
        else if (t == 2) fft_pass<C, 2, false>(Z, m, 2, tw, ntab, st);
        if (t > 1) __syncthreads();
    } else {
        if (t == 8) fft_pass<C, 8, true>(Z, m, 8, tw, ntab, st);
        else if (t == 4) fft_pass<C, 4, true>(Z, m, 4, tw, ntab, st);
        else if (t == 2) fft_pass<C, 2, true>(Z, m, 2, tw, ntab, st);
        if (t > 1) __syncthreads();
        int M = t * R;
        for (int s = 0; s < a; ++s) { fft_pass<C, R, true>(Z, m, M, tw, ntab, st); __syncthreads(); M *= R; }
    }
}

// Length-m (power of two) complex FFT of the padded buffer Z by the whole
// CTA, with the radix a CTA of nt threads would use (the result depends on
// the radix, not on the CTA size).  Forward: natural order in, digit-reversed
// order out (see fft_perm).  Inverse: that order in, natural order out,
// unnormalised.
template <typename C, bool INV>
__device__ void fft_smem_nt(C* Z, int m, int nt, const C* __restrict__ tw, int ntab, unsigned* st = nullptr) {
    const int R = fft_radix<C>(m, nt);
    if (sizeof(C) == 8 && R == 16) fft_passes<C, 16, INV>(Z, m, tw, ntab, st);
    else if (sizeof(C) == 8 && R == 8) fft_passes<C, 8, INV>(Z, m, tw, ntab, st);
    else fft_passes<C, 4, INV>(Z, m, tw, ntab, st);
}
template <typename C, bool INV>
__device__ __forceinline__ void fft_smem(C* Z, int m, const C* __restrict__ tw, int ntab, unsigned* st = nullptr) {
    fft_smem_nt<C, INV>(Z, m, blockDim.x, tw, ntab, st);
}

// Slot of frequency k after the forward FFT: k = r1 + R1 r2 + R1 R2 r3 + ...
// (r_s the output digit of pass s) sits at r1 S1 + r2 S2 + ..., S_s the
// stride of pass s.
template <typename C>
__device__ __forceinline__ int fft_perm_nt(int k, int m, int nt) {
    const int R = fft_radix<C>(m, nt);
    int pos = 0, S = m;
    while (S >= R) { S /= R; pos += (k % R) * S; k /= R; }
    if (S > 1) pos += k % S;   // last pass: stride 1
    return pos;
}
template <typename C>
__device__ __forceinline__ int fft_perm(int k, int m) {
    return fft_perm_nt<C>(k, m, blockDim.x);
}

// Real-signal step.  Z holds FFT_m of z[j] = x[2j] + i x[2j+1] (n = 2m real
// samples) in fft_perm order.  With W = exp(-2 pi i / n):
//   X2[k] = (Z[k] + conj Z[m-k]) - i W^k (Z[k] - conj Z[m-k]) = 2 X[k].
template <typename C>
__device__ __forceinline__ void real_post(C a, C b, C w, C& Xk, C& Xmk) {
    // a = Z[k], b = Z[m-k], w = W^k;  W^(m-k) = -conj(w)
    C cb = cconj(b), ca = cconj(a);
    C d1 = csub(a, cb), d2 = csub(b, ca);
    Xk = cadd(cadd(a, cb), mul_mi<C, false>(cmul(w, d1)));
    C wm = w; wm.x = -w.x;  // -conj(w)
    Xmk = cadd(cadd(b, ca), mul_mi<C, false>(cmul(wm, d2)));
}
// Inverse: from Y (spectrum of the real result) build
//   Z'[k] = (Y[k] + conj Y[m-k]) + i conj(W^k) (Y[k] - conj Y[m-k])
template <typename C>
__device__ __forceinline__ void real_pre(C yk, C ymk, C w, C& Zk, C& Zmk) {
    C cym = cconj(ymk), cyk = cconj(yk);
    C wc = cconj(w);
    C wmc; wmc.x = -w.x; wmc.y = -w.y;  // conj(W^(m-k)) = conj(-conj(w)) = -w
    Zk = cadd(cadd(yk, cym), mul_mi<C, true>(cmul(wc, csub(yk, cym))));
    Zmk = cadd(cadd(ymk, cyk), mul_mi<C, true>(cmul(wmc, csub(ymk, cyk))));
}

// Z (forward FFT of the packed real block, fft_perm order) -> Z' ready for the
// inverse FFT, multiplying by the kernel spectrum H = FFT_n(k) / (4m) (m+1
// entries, natural order).  The factor 2 of X2, the missing 1/2 of the inverse
// step and the 1/m of the inverse FFT fold into that power-of-two scale.
template <typename C>
__device__ __forceinline__ C load_h(const C* H, int k, bool coherent) {
    return coherent ? __ldcg(&H[k]) : __ldg(&H[k]);
}
// fft_perm for a transform whose main passes have radix R (a compile-time
// constant: the digit arithmetic becomes shifts and masks).
template <int R>
__device__ __forceinline__ int fft_perm_r(int k, int m) {
    int pos = 0, S = m;
    while (S >= R) { S /= R; pos += (k & (R - 1)) * S; k /= R; }
    if (S > 1) pos += k & (S - 1);   // last pass: stride 1
    return pos;
}
// ... and for a length known at compile time (MM > 0; 0: the runtime m)
template <int R, int MM>
__device__ __forceinline__ int fft_perm_rc(int k, int m) {
    if constexpr (MM == 0) {
        return fft_perm_r<R>(k, m);
    } else {
        int pos = 0, S = MM;
#pragma unroll
        for (int it = 0; it < 32 && S >= R; ++it) { S /= R; pos += (k & (R - 1)) * S; k /= R; }
        if (S > 1) pos += k & (S - 1);
        return pos;
    }
}

// One thread's frequencies k = t, t + nt, ... in rounds of B: every load of a
// round (both spectrum entries and the twiddle) is issued before any is used,
// so a round costs one memory latency.
template <typename C, int R, int B, int MM = 0>
__device__ __forceinline__ void spectral_multiply_r(C* Z, int m_rt, const C* H, const C* __restrict__ tw, int twn,
                                                    bool coherent, unsigned* st) {
    const int m = MM > 0 ? MM : m_rt;
    const int half = m / 2, nt = blockDim.x;
    for (int k0 = threadIdx.x; k0 <= half; k0 += B * nt) {
        C hk[B], hmk[B], w[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int k = k0 + u * nt;
            if (k <= half) {
                hk[u] = load_h(H, k, coherent);
                hmk[u] = load_h(H, m - k, coherent);
                w[u] = __ldg(&tw[k * twn]);
            }
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int k = k0 + u * nt;
            if (k > half) break;
            if (k == 0) {
                C z0 = Z[0];
                C X0, Xm;
                X0.x = 2 * (z0.x + z0.y); X0.y = 0;
                Xm.x = 2 * (z0.x - z0.y); Xm.y = 0;
                C Y0 = cmul(X0, hk[u]), Ym = cmul(Xm, hmk[u]);
                C cym = cconj(Ym);
                Z[0] = cadd(cadd(Y0, cym), mul_mi<C, true>(csub(Y0, cym)));
            } else {
                const int qk = fft_perm_rc<R, MM>(k, m), qmk = fft_perm_rc<R, MM>(m - k, m);
                if (!APX_IN_BOUNDS(qk < m && qmk < m, st)) continue;
                const int pk = pad16(qk), pmk = pad16(qmk);
                C a = Z[pk], b = Z[pmk];
                C Xk, Xmk;
                real_post(a, b, w[u], Xk, Xmk);
                C Yk = cmul(Xk, hk[u]);
                C Ymk = cmul(Xmk, hmk[u]);
                C Zk, Zmk;
                real_pre(Yk, Ymk, w[u], Zk, Zmk);
                Z[pk] = Zk;
                if (k != m - k) Z[pmk] = Zmk;
            }
        }
    }
    __syncthreads();
}

// `coherent`: H was written during this kernel (read around L1).
template <typename C>
__device__ void spectral_multiply(C* Z, int m, const C* H, const C* __restrict__ tw, int twn, bool coherent,
                                  unsigned* st = nullptr) {
    constexpr int B = sizeof(C) == 8 ? 5 : 3;
    const int R = fft_radix<C>(m, blockDim.x);
    if (R == 16) {
        switch (m) {  // the lengths with compile-time FFT passes
            case 1024: spectral_multiply_r<C, 16, B, 1024>(Z, m, H, tw, twn, coherent, st); return;
            case 2048: spectral_multiply_r<C, 16, B, 2048>(Z, m, H, tw, twn, coherent, st); return;
            case 4096: spectral_multiply_r<C, 16, B, 4096>(Z, m, H, tw, twn, coherent, st); return;
            case 8192: spectral_multiply_r<C, 16, B, 8192>(Z, m, H, tw, twn, coherent, st); return;
            default: spectral_multiply_r<C, 16, B>(Z, m, H, tw, twn, coherent, st); return;
        }
    }
    else if (R == 8) spectral_multiply_r<C, 8, B>(Z, m, H, tw, twn, coherent, st);
    else spectral_multiply_r<C, 4, B>(Z, m, H, tw, twn, coherent, st);
}

// Programmatic dependent launch: let the next kernel in the stream start, and
// wait for the previous one's results.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Cluster barrier in two halves (every thread of every CTA of the cluster).
// arrive.relaxed orders nothing (it only says that this CTA has started, so
// that the others may access its shared memory after their wait); arrive
// (release) makes this thread's earlier memory accesses, those to other CTAs'
// shared memory included, visible to the threads past the matching wait
// (acquire).  Work placed between the halves overlaps the barrier.
__device__ __forceinline__ void cl_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* a) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* a, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

}  // namespace apx
