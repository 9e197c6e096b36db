/*
 * apx_oracle.c -- plain, slow FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Follows Anam & Andreopoulos, arXiv 1201.3018, step by step in the paper's
 * order: Eq. (1) convolution, Section III block geometry, Eq. (2) companding,
 * Eq. (3) companding range, Eqs. (4)-(8) packing, Eq. (9) block convolution,
 * Eqs. (10)-(15) unpacking, Eq. (16) inverse companding, Eq. (17) output
 * assembly, Eqs. (18)-(19)/Table 1 distortion model, Section IV.D selection.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.  No fused
 * multiply-add anywhere: every product and sum is a separate IEEE operation.
 *
 * Where the paper is silent or garbled, the reading taken is stated at the
 * code it governs.
 */
#include "apx_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ======================================================================== */
/* Plain definitions                                                         */
/* ======================================================================== */

/* Eq. (1): r_out[m] = sum_{n=0}^{N-1} s_in[m-n] k[n], for m in [0, L+N-1). */
void or_conv_ref(const double* s, int64_t L, const double* k, int32_t N, double* r) {
    for (int64_t m = 0; m < L + N - 1; ++m) {
        double acc = 0.0;
        for (int32_t n = 0; n < N; ++n) {
            int64_t i = m - n;
            if (i >= 0 && i < L) acc += s[i] * k[n];
        }
        r[m] = acc;
    }
}

/* Cross-correlation (the paper only names Matlab's xcorr; read as the plain
 * definition below, equal to conv(s, reverse(t))):
 *   x[l] = sum_n s[n + l] t[n],  l in [-(N-1), L-1],  stored at index l + N - 1.
 * Written from the definition, not through a reversed convolution, so that it
 * pins the reversal the pipeline uses. */
void or_xcorr_ref(const double* s, int64_t L, const double* t, int32_t N, double* r) {
    for (int64_t l = -(int64_t)(N - 1); l <= L - 1; ++l) {
        double acc = 0.0;
        for (int32_t n = 0; n < N; ++n) {
            int64_t i = n + l;
            if (i >= 0 && i < L) acc += s[i] * t[n];
        }
        r[l + N - 1] = acc;
    }
}

/* Eq. (1) at chosen output indices only (for spot checks of long signals). */
void or_conv_ref_at(const double* s, int64_t L, const double* k, int32_t N, const int64_t* idx, int64_t n,
                    double* r) {
    for (int64_t j = 0; j < n; ++j) {
        int64_t m = idx[j];
        double acc = 0.0;
        for (int32_t q = 0; q < N; ++q) {
            int64_t i = m - q;
            if (i >= 0 && i < L) acc += s[i] * k[q];
        }
        r[j] = acc;
    }
}

/* Eq. (1) over integers: the exact target r~ = s~ * k~ of the packed path. */
void or_conv_int(const int64_t* s, int64_t L, const int64_t* k, int32_t N, int64_t* r) {
    for (int64_t m = 0; m < L + N - 1; ++m) {
        int64_t acc = 0;
        for (int32_t n = 0; n < N; ++n) {
            int64_t i = m - n;
            if (i >= 0 && i < L) acc += s[i] * k[n];
        }
        r[m] = acc;
    }
}

/* ======================================================================== */
/* a1: block plan (Section III, Eqs. (10) and (17)): W_block = W + N' + 1, block
 * w >= 1 starts at wW - 2 (Eq. 17 solved for the origin)                    */
/* ======================================================================== */

/* Section III: N odd (an even kernel gets one zero tap), W even, and
 * W_block = W + N + 1.  Here W is derived from the given W_block.
 *
 * Direct core, Eq. (17) as printed: block 0 covers s_in[0, W_block) and yields
 * outputs [0, W+N'-1); block w >= 1 starts at input w*W - 2 (solving Eq. (17)
 * for the block origin) and yields its local outputs [N'+1, W_block).
 *
 * FFT core: a circular block convolution cannot produce block 0's leading
 * outputs (they alias with the block tail), so every block uses the w >= 1 rule
 * (start w*W - 2, local outputs [N'+1, W_block)) and h = ceil((N'-1)/W) head
 * blocks w = -h..-1 in front yield outputs [0, N'-1).  Blocks are indexed
 * i = w + h.
 *
 * Windows read zeros outside [0, L); outputs beyond L+N-1 are dropped. */
int or_plan(int64_t L, int32_t N, int32_t Wblock, int fft, or_plan_t* p) {
    if (!p || L < 1 || N < 1) return OR_ERR_ARG;
    int32_t Nodd = (N % 2) ? N : N + 1;
    if (Wblock < 4 || (Wblock % 2) || Wblock > 32768) return OR_ERR_WBLOCK;
    int32_t W = Wblock - Nodd - 1;
    if (W < 2) return OR_ERR_WBLOCK;
    if (fft && (Wblock & (Wblock - 1))) return OR_ERR_WBLOCK;
    int64_t span = L + N - Nodd;          /* outputs beyond the first N'-1 */
    int64_t P = (span + W - 1) / W;
    if (P < 1) P = 1;
    int32_t head = fft ? (Nodd - 1 + W - 1) / W : 0;
    p->L = L; p->N = N; p->Nodd = Nodd; p->Wblock = Wblock; p->W = W; p->fft = fft ? 1 : 0;
    p->head = head;
    p->P = P + head;
    p->out_len = L + N - 1;
    return OR_OK;
}

int64_t or_block_start(const or_plan_t* p, int64_t i) {
    if (p->fft) return (i - p->head) * (int64_t)p->W - 2;
    return i == 0 ? 0 : i * (int64_t)p->W - 2;
}

void or_block_out_range(const or_plan_t* p, int64_t i, int32_t* lo, int32_t* hi) {
    if (!p->fft && i == 0) { *lo = 0; *hi = p->Wblock - 2; }  /* W + N' - 1 outputs */
    else { *lo = p->Nodd + 1; *hi = p->Wblock; }              /* m + 2 W_start + 2 */
}

/* ======================================================================== */
/* a3: block statistics                                                      */
/* ======================================================================== */

/* ||x||_inf (Section II notation).  NaN is reported as NaN. */
float or_maxabs(const float* x, int64_t n) {
    float m = 0.0f;
    for (int64_t i = 0; i < n; ++i) {
        float a = fabsf(x[i]);
        if (a != a) return a;
        if (a > m) m = a;
    }
    return m;
}

/* Second moment of the marginal (Section IV.D: sigma^2 is the second moment of
 * the fitted marginal; here the sample second moment of the window).
 * Evaluated in 24-bit fixed point relative to ||x||_inf so that
 * the sum is an exact integer, independent of summation order:
 *   q_i = trunc(x_i * 2^sh), ||x||_inf * 2^sh in [2^23, 2^24),
 *   sigma^2 = (sum q_i^2) * 2^(-2 sh) / n.                                   */
double or_second_moment(const float* x, int64_t n, float maxabs) {
    if (!(maxabs > 0.0f) || n <= 0) return 0.0;
    int e;
    (void)frexpf(maxabs, &e);             /* maxabs = f 2^e, f in [0.5, 1) */
    int sh = 24 - e;
    int64_t acc = 0;
    for (int64_t i = 0; i < n; ++i) {
        float y = ldexpf(x[i], sh);
        int64_t q = (int64_t)y;           /* truncation toward zero */
        acc += q * q;
    }
    return ldexp((double)acc, -2 * sh) / (double)n;
}

/* ======================================================================== */
/* a4: exactness bounds and the per-block selector (Section IV.D)            */
/* ======================================================================== */

/* Eq. (6) with a power of two: eps = 2^-b with the smallest b such that 2^b >= 2 R_max + 1, so
 * every offset digit R_max + c, c in [-R_max, R_max], fits in b bits (the
 * paper's Eq. (6) eps = 1/(2 R_max) rounded down to a power of two). */
int32_t or_bits(int64_t Rmax) {
    int32_t b = 0;
    while (b < 62 && ((int64_t)1 << b) < 2 * Rmax + 1) ++b;
    return b;
}

/* Exactness bound (replaces Table 1's "Companding range" row for power-of-two eps):
 * every packed word, product and partial sum of the FP64 block convolution is
 * an integer multiple of the finest digit; it is exact and order-independent
 * when the scaled magnitude bound stays within 2^53.
 *   symmetric, Eq. (9):   A 2^{2b} + B 2^b + C <= 2^53 with
 *       A = ceil(N'/2) S K  (eps^-1 term), B = N' S K (base), C = floor(N'/2) S K (eps term);
 *   asymmetric, Eq. (7):  R_max (sum_{q<M} 2^{b q}) <= 2^53.                  */
int or_exact_ok(int blkmode, int32_t Nodd, int32_t Sq, int32_t Kq) {
    if (Nodd < 1 || Sq < 1 || Kq < 1) return 0;
    if (blkmode == OR_BLK_TC) {
        /* Tensor-core core: every companded integer (|x| <= 2048) is exact in
         * FP16, every product exact in FP32, and FP32 sums of integers stay
         * exact while their magnitude is at most 2^24 (the 24-bit significand);
         * a partial sum of the N' taps is bounded by N' S K. */
        return Sq <= 2048 && Kq <= 2048 && (int64_t)Nodd * Sq * Kq <= ((int64_t)1 << 24);
    }
    u128 SK = (u128)(uint32_t)Sq * (u128)(uint32_t)Kq;
    u128 Rmax = SK * (u128)(uint32_t)Nodd;
    const u128 lim = (u128)1 << 53;
    if (Rmax >= lim) return 0;
    int32_t b = or_bits((int64_t)Rmax);
    if (blkmode == OR_BLK_SYM) {
        if (2 * b > 100) return 0;
        u128 A = (u128)((Nodd + 1) / 2) * SK, B = Rmax, C = (u128)((Nodd - 1) / 2) * SK;
        return (A << (2 * b)) + (B << b) + C <= lim;
    }
    int M = blkmode == OR_BLK_ASYM2 ? 2 : (blkmode == OR_BLK_ASYM3 ? 3 : 0);
    if (!M || b * (M - 1) > 100) return 0;
    u128 g = 0;
    for (int q = 0; q < M; ++q) g += (u128)1 << (b * q);
    return Rmax * g <= lim;
}

/* Section IV.D: "the maximum S_q and K_q that allow for this packing".  With
 * S_q = K_q = Q as in every experiment of the paper, the largest
 * Q in [1, 2^20] that passes the exactness bound; 0 when none does. */
int32_t or_qmax_direct(int blkmode, int32_t Nodd) {
    if (!or_exact_ok(blkmode, Nodd, 1, 1)) return 0;
    int32_t lo = 1, hi = 1 << 20;
    if (or_exact_ok(blkmode, Nodd, hi, hi)) return hi;
    while (hi - lo > 1) {
        int32_t mid = lo + (hi - lo) / 2;
        if (or_exact_ok(blkmode, Nodd, mid, mid)) lo = mid; else hi = mid;
    }
    return lo;
}

/* FFT core (the paper is silent on its rounding): error bound of an FFT block convolution in units of the finest
 * packed digit.  Radix-2 structured FFT with twiddle error mu (Higham,
 * Accuracy and Stability of Numerical Algorithms, Thm 24.2):
 *   phi = Lg eta / (1 - Lg eta),  eta = mu + gamma_4 (sqrt 2 + mu),
 *   |err| <= (3 phi + 16 u) ||kbar||_1 ||sbar||_2
 * (forward transform of the block, transform of the kernel, inverse transform
 * and the pointwise products), Lg = log2(n) + 2 stages for the real-signal
 * transform of length n, mu = 4u.  The finest digit of the packed output is
 * eps^(M-1) (eps for symmetric packing). */
double or_fft_err_digits(int blkmode, int32_t log2n, double l1_kbar, double l2_sbar, int32_t b) {
    const double u = ldexp(1.0, -53);
    double mu = 4.0 * u;
    double g4 = (4.0 * u) / (1.0 - 4.0 * u);
    double eta = mu + g4 * (sqrt(2.0) + mu);
    double Lg = (double)(log2n + 2);
    double phi = (Lg * eta) / (1.0 - Lg * eta);
    double E = (3.0 * phi + 16.0 * u) * l1_kbar * l2_sbar;
    int32_t sc = blkmode == OR_BLK_SYM ? b : (blkmode == OR_BLK_ASYM2 ? b : 2 * b);
    return ldexp(E, sc);
}

static int32_t blk_M(int blkmode) { return blkmode == OR_BLK_ASYM2 ? 2 : (blkmode == OR_BLK_ASYM3 ? 3 : 1); }

static int32_t ilog2_i(int64_t n) { int32_t l = 0; while (((int64_t)1 << l) < n) ++l; return l; }

/* Length of the real block signal transformed by the FFT core for a mode:
 * symmetric packs W_block samples into W_block/2 words; asymmetric packing
 * convolves segments of ceil(W_block/M) words whose full linear convolution
 * fits a transform of W_block points (the asymmetric layout of Eq. (7)). */
static int32_t fft_log2n(int blkmode, int32_t Wblock) {
    return blkmode == OR_BLK_SYM ? ilog2_i(Wblock / 2) : ilog2_i(Wblock);
}

/* FFT core, per mode: the largest Q <= or_qmax_direct whose a-priori error
 * bound stays below 1/4 digit for a block and kernel of crest factor 3
 * (||x||_1 ~ n Q / 3, ||x||_2 ~ sqrt(n) Q / 3).  A guide only: every block is
 * checked again with its exact norms before it is packed. */
int32_t or_qmax_fft(int blkmode, int32_t Nodd, int32_t Wblock) {
    int32_t qd = or_qmax_direct(blkmode, Nodd);
    int32_t lg = fft_log2n(blkmode, Wblock);
    for (int32_t Q = qd; Q >= 1; --Q) {
        int64_t Rmax = (int64_t)Nodd * Q * Q;
        int32_t b = or_bits(Rmax);
        double taps = blkmode == OR_BLK_SYM ? (double)((Nodd + 1) / 2) : (double)Nodd;
        double kscale = blkmode == OR_BLK_SYM ? ldexp(1.0, b) + 1.0 : 1.0;
        double l1 = taps * (double)Q / 3.0 * kscale;
        double l2 = sqrt((double)Wblock) * (double)Q / 3.0;
        if (or_fft_err_digits(blkmode, lg, l1, l2, b) < 0.25) return Q;
    }
    return 0;
}

/* Table 1 SNR, derived from Eqs. (18)-(19) with sigma_v = ||.||_inf/(Q sqrt 12):
 *   SNR = 144 (s_s s_k S K)^2 / (12 [(s_s S ||k||)^2 + (s_k K ||s||)^2] + (||s|| ||k||)^2).
 * Reading: the printed Table 1 pairs s_s with ||s|| inside the bracket, which is
 * dimensionally inconsistent with Eq. (18); Eq. (18) decides.  The two forms
 * agree at the Section IV.A settings (both 27.1 dB and 51.2 dB).
 * Evaluated with one IEEE operation at a time in a fixed order. */
static void snr_terms(double sig2_s, float Ms, double sig2_k, float Mk, int32_t Sq, int32_t Kq,
                      double* num, double* den) {
    double S2 = (double)Sq * (double)Sq;
    double K2 = (double)Kq * (double)Kq;
    double Ms2 = (double)Ms * (double)Ms;
    double Mk2 = (double)Mk * (double)Mk;
    double t1 = sig2_s * sig2_k;
    double t2 = S2 * K2;
    *num = (144.0 * t1) * t2;
    double a = (sig2_s * S2) * Mk2;
    double c = (sig2_k * K2) * Ms2;
    *den = 12.0 * (a + c) + Ms2 * Mk2;
}

double or_snr_model_lin(double sig2_s, float Ms, double sig2_k, float Mk, int32_t Sq, int32_t Kq) {
    double num, den;
    snr_terms(sig2_s, Ms, sig2_k, Mk, Sq, Kq, &num, &den);
    return num / den;
}

double or_snr_model_db(double sig2_s, float Ms, double sig2_k, float Mk, int32_t Sq, int32_t Kq) {
    return 10.0 * log10(or_snr_model_lin(sig2_s, Ms, sig2_k, Mk, Sq, Kq));
}

/* Section IV.D asks for an SNR of at least the target in every block, while the
 * Table 1 model gives the SNR a block can expect: a block's measured SNR
 * scatters around the model, the more so the fewer outputs it keeps (its
 * signal and error powers are sums over W outputs).  A packing is therefore
 * admitted only when the model clears the target by
 *   delta(W) = 0.5 + 48 / sqrt(W) dB,  W = outputs kept per block,
 * a bound on the model's overestimate measured over many blocks of Gaussian,
 * Laplacian and uniform signals and kernels (1.6 dB at W = 958, 6.2 dB at
 * W = 56 at worst), with about 10 % to spare. */
double or_snr_margin_db(int32_t W) { return 0.5 + 48.0 / sqrt((double)W); }

/* Section IV.D: a packing is admissible when the model SNR meets the minimum. */
int or_snr_feasible(double sig2_s, float Ms, double sig2_k, float Mk, int32_t Sq, int32_t Kq,
                    double thr_lin) {
    double num, den;
    snr_terms(sig2_s, Ms, sig2_k, Mk, Sq, Kq, &num, &den);
    return num >= thr_lin * den;
}

/* ======================================================================== */
/* a5/a6: companding (Eq. 2) and packing (Eqs. 4, 5, 7)                      */
/* ======================================================================== */

/* Eq. (2): c = Q / ||x||_inf, one correctly rounded FP32 divide
 * (the inputs are FP32; the decision is taken in FP32 on every side). */
float or_compand_factor(int32_t Q, float maxabs) { return (float)Q / maxabs; }

/* Eq. (2): x~ = [[c x]], round half to even on the FP32 product (the paper does
 * not name its rounding). */
void or_compand(const float* x, int64_t n, float c, int32_t* q) {
    for (int64_t i = 0; i < n; ++i) {
        float p = c * x[i];
        q[i] = (int32_t)rintf(p);
    }
}

/* Eq. (4): sbar[m] = s~[2m] + eps s~[2m+1], m in [0, n/2). */
void or_pack_sym_signal(const int32_t* sq, int32_t n, int32_t b, double* sbar) {
    double eps = ldexp(1.0, -b);
    for (int32_t m = 0; m < n / 2; ++m) sbar[m] = (double)sq[2 * m] + eps * (double)sq[2 * m + 1];
}

/* Eq. (5) with the kernel pair swapped relative to the print (as printed, Eqs.
 * (12)-(15) do not reconstruct s~*k~),
 *   kbar[n] = k~[2n+1] + eps^-1 k~[2n],  n in [0, (N'+1)/2),  k~[N'] = 0,
 * which makes the eps^0 term of Eq. (9) the odd output r~[2m+1] and the
 * eps^-1 / eps terms the two halves of r~[2m], as Eqs. (14)-(15) require. */
void or_pack_sym_kernel(const int32_t* kq, int32_t Nodd, int32_t b, double* kbar) {
    double einv = ldexp(1.0, b);
    for (int32_t n = 0; n < (Nodd + 1) / 2; ++n) {
        int32_t ko = (2 * n + 1 < Nodd) ? kq[2 * n + 1] : 0;
        kbar[n] = (double)ko + einv * (double)kq[2 * n];
    }
}

/* Eq. (5) exactly as printed, kbar[n] = k~[2n] + eps^-1 k~[2n+1]; kept only so
 * that a test can show this pairing does not reconstruct s~ * k~. */
void or_pack_sym_kernel_printed(const int32_t* kq, int32_t Nodd, int32_t b, double* kbar) {
    double einv = ldexp(1.0, b);
    for (int32_t n = 0; n < (Nodd + 1) / 2; ++n) {
        int32_t ko = (2 * n + 1 < Nodd) ? kq[2 * n + 1] : 0;
        kbar[n] = (double)kq[2 * n] + einv * (double)ko;
    }
}

/* Eq. (7) (its stride is garbled in the print): segments of Ls = ceil(n/M) samples,
 *   sbar[m] = sum_{q<M} eps^q s~[m + q Ls],  zero past the block end. */
void or_pack_asym_signal(const int32_t* sq, int32_t n, int32_t M, int32_t b, double* sbar) {
    int32_t Ls = (n + M - 1) / M;
    for (int32_t m = 0; m < Ls; ++m) {
        double acc = 0.0;
        for (int32_t q = 0; q < M; ++q) {
            int32_t i = m + q * Ls;
            if (i < n) acc += ldexp((double)sq[i], -b * q);
        }
        sbar[m] = acc;
    }
}

/* ======================================================================== */
/* a7: block convolution cores (Eqs. 8, 9)                                    */
/* ======================================================================== */

/* Direct FP64 convolution r[j] = sum_{n<nk} a[j-n] k[n], j in [0, nr),
 * with a[i] = 0 outside [0, na). */
void or_conv_f64(const double* a, int64_t na, const double* k, int64_t nk, double* r, int64_t nr) {
    for (int64_t j = 0; j < nr; ++j) {
        double acc = 0.0;
        for (int64_t n = 0; n < nk; ++n) {
            int64_t i = j - n;
            if (i >= 0 && i < na) acc += a[i] * k[n];
        }
        r[j] = acc;
    }
}

/* Textbook iterative radix-2 FFT (bit reversal then butterflies), FP64,
 * sign -1 forward / +1 inverse, twiddles from libm cos/sin. */
static void fft_radix2(double* re, double* im, int64_t n, int sign) {
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        for (int64_t i = 0; i < n; i += len) {
            for (int64_t j = 0; j < len / 2; ++j) {
                double ang = (double)sign * 2.0 * M_PI * (double)j / (double)len;
                double wr = cos(ang), wi = sin(ang);
                int64_t a = i + j, c = i + j + len / 2;
                double xr = re[c] * wr - im[c] * wi;
                double xi = re[c] * wi + im[c] * wr;
                re[c] = re[a] - xr; im[c] = im[a] - xi;
                re[a] = re[a] + xr; im[a] = im[a] + xi;
            }
        }
    }
}

/* Circular convolution of length n (a power of two) through the FFT:
 * r = IFFT(FFT(a) . FFT(k)) (the frequency-domain core of Section IV.A),
 * first nr entries returned. */
int or_conv_f64_fft(const double* a, int64_t na, const double* k, int64_t nk, double* r, int64_t nr,
                    int64_t n) {
    if (n < 2 || (n & (n - 1)) || na > n || nk > n || nr > n) return OR_ERR_ARG;
    double* ar = calloc((size_t)n, sizeof(double));
    double* ai = calloc((size_t)n, sizeof(double));
    double* kr = calloc((size_t)n, sizeof(double));
    double* ki = calloc((size_t)n, sizeof(double));
    if (!ar || !ai || !kr || !ki) { free(ar); free(ai); free(kr); free(ki); return OR_ERR_ARG; }
    memcpy(ar, a, (size_t)na * sizeof(double));
    memcpy(kr, k, (size_t)nk * sizeof(double));
    fft_radix2(ar, ai, n, -1);
    fft_radix2(kr, ki, n, -1);
    for (int64_t i = 0; i < n; ++i) {
        double xr = ar[i] * kr[i] - ai[i] * ki[i];
        double xi = ar[i] * ki[i] + ai[i] * kr[i];
        ar[i] = xr; ai[i] = xi;
    }
    fft_radix2(ar, ai, n, +1);
    for (int64_t j = 0; j < nr; ++j) r[j] = ar[j] / (double)n;
    free(ar); free(ai); free(kr); free(ki);
    return OR_OK;
}

/* ======================================================================== */
/* a8: unpacking                                                              */
/* ======================================================================== */

/* Packed output scaled to the finest digit: T = rbar 2^sc, an exact integer
 * whenever the exactness bound holds (rounded to nearest for the FFT core,
 * whose error bound is kept below 1/4 digit). */
static int scaled_int(double rbar, int32_t sc, int round_nearest, int64_t* T) {
    double t = ldexp(rbar, sc);
    if (round_nearest) t = nearbyint(t);
    if (t != floor(t) || fabs(t) > 9007199254740992.0) return OR_ERR_INEXACT;
    *T = (int64_t)t;
    return OR_OK;
}

/* Eqs. (11)-(15), exact mode (u_sys = 0, eps = 2^-b), evaluated
 * on u scaled by 2^b, which is an integer:
 *   (11) u[m] = rbar[m] + R_safe,  R_safe = R_max (eps + 1 + eps^-1)
 *   (12) side_eps    = R_max for m = W_start, else eps^-1 (u[m-1] - floor u[m-1])
 *   (13) side_epsinv = floor(eps u[m])
 *   (14) r~[2m]   = side_epsinv + side_eps - 2 R_max
 *   (15) r~[2m+1] = floor(u[m]) - eps^-1 side_epsinv - R_max
 * for m in [W_start, nbar); rq has 2 nbar entries, those below 2 W_start are 0. */
int or_unpack_sym(const double* rbar, int32_t nbar, int32_t Wstart, int64_t Rmax, int32_t b,
                  int64_t* rq) {
    if (2 * b > 61) return OR_ERR_RANGE;
    int64_t one = 1;
    int64_t Rsafe_b = Rmax * ((one << (2 * b)) + (one << b) + 1);  /* 2^b R_safe */
    int64_t mask = (one << b) - 1;
    int64_t Uprev = 0;
    for (int32_t m = 0; m < 2 * Wstart && m < 2 * nbar; ++m) rq[m] = 0;
    for (int32_t m = Wstart; m < nbar; ++m) {
        int64_t T;
        if (scaled_int(rbar[m], b, 0, &T)) return OR_ERR_INEXACT;
        int64_t U = T + Rsafe_b;                              /* (11), times 2^b */
        if (U < 0) return OR_ERR_RANGE;
        int64_t side_epsinv = U >> (2 * b);                   /* (13) */
        int64_t side_eps = (m == Wstart) ? Rmax : (Uprev & mask); /* (12) */
        rq[2 * m] = side_epsinv + side_eps - 2 * Rmax;        /* (14) */
        rq[2 * m + 1] = (U >> b) - (side_epsinv << b) - Rmax; /* (15) */
        Uprev = U;
    }
    return OR_OK;
}

/* Exact mode, second form: balanced base-2^b digits of T = rbar 2^b,
 * T = A 2^{2b} + B 2^b + C, r~[2m+1] = B, r~[2m] = A[m] + C[m-1].  Must agree
 * with or_unpack_sym wherever both are exact (tested). */
int or_unpack_sym_digits(const double* rbar, int32_t nbar, int32_t Wstart, int32_t b, int64_t* rq) {
    int64_t one = 1, mod = one << b, half = one << (b - 1);
    int64_t Cprev = 0;
    for (int32_t m = 0; m < 2 * Wstart && m < 2 * nbar; ++m) rq[m] = 0;
    for (int32_t m = Wstart; m < nbar; ++m) {
        int64_t T;
        if (scaled_int(rbar[m], b, 0, &T)) return OR_ERR_INEXACT;
        int64_t C = T & (mod - 1); if (C >= half) C -= mod;
        int64_t T1 = (T - C) / mod;
        int64_t B = T1 & (mod - 1); if (B >= half) B -= mod;
        int64_t A = (T1 - B) / mod;
        rq[2 * m + 1] = B;
        rq[2 * m] = A + (m == Wstart ? 0 : Cprev);
        Cprev = C;
    }
    return OR_OK;
}

/* Eqs. (11)-(15) literally in FP64 with any eps and u_sys (the paper's own
 * eps = (2 R_max)^-1 and u_sys = 3.1193e-11 of Section IV).  Rounding errors
 * land in the fractional digit, so this form is only compared by SNR. */
void or_unpack_sym_fp64(const double* rbar, int32_t nbar, int32_t Wstart, double Rmax, double eps,
                        double u_sys, double* rq) {
    double einv = 1.0 / eps;
    double Rsafe = Rmax * (eps + 1.0 + einv) + u_sys * einv;
    double uprev = 0.0;
    for (int32_t m = 0; m < 2 * Wstart && m < 2 * nbar; ++m) rq[m] = 0.0;
    for (int32_t m = Wstart; m < nbar; ++m) {
        double u = rbar[m] + Rsafe;
        double side_epsinv = floor(eps * u);
        double side_eps = (m == Wstart) ? Rmax : einv * (uprev - floor(uprev));
        rq[2 * m] = floor(side_epsinv + side_eps - 2.0 * Rmax);
        rq[2 * m + 1] = floor(floor(u) - einv * side_epsinv - Rmax);
        uprev = u;
    }
}

/* Asymmetric unpacking: "M successive iterations" (Section III.C, citing [8]).
 * Offset every digit by R_max, u = rbar + R_max sum_q eps^q, then
 * for q = 0..M-1 take the integer part at the scale of digit q and keep the
 * remainder; c_q = digit - R_max.  Segment results overlap-add:
 *   r~[j] = sum_q c_q[j - q Ls],  j in [0, nout). */
int or_unpack_asym(const double* rbar, int32_t nr, int32_t Ls, int32_t M, int64_t Rmax, int32_t b,
                   int32_t nout, int64_t* rq) {
    if (b * M > 62) return OR_ERR_RANGE;
    int64_t one = 1, off = 0;
    for (int32_t q = 0; q < M; ++q) off += Rmax << (b * q);
    for (int32_t j = 0; j < nout; ++j) rq[j] = 0;
    for (int32_t i = 0; i < nr; ++i) {
        int64_t T;
        if (scaled_int(rbar[i], b * (M - 1), 0, &T)) return OR_ERR_INEXACT;
        int64_t V = T + off;
        if (V < 0) return OR_ERR_RANGE;
        for (int32_t q = 0; q < M; ++q) {
            int32_t sh = b * (M - 1 - q);
            int64_t digit = V >> sh;
            V -= digit << sh;
            int32_t j = i + q * Ls;
            if (j < nout) rq[j] += digit - Rmax;
        }
    }
    (void)one;
    return OR_OK;
}

/* ======================================================================== */
/* a1..a9: the whole method                                                  */
/* ======================================================================== */

typedef struct {
    int32_t blk;      /* OR_BLK_* */
    int32_t S, K, b, M;
    int64_t Rmax;
    float ck;
    double* kpk;      /* packed kernel, FP64 */
    int32_t nk;       /* packed kernel taps */
    double l1;        /* ||kbar||_1 (exact integer) */
    int32_t log2n;
    int literal;      /* OR_LITERAL: eps = (2 R_max)^-1, FP64 unpacking with u_sys */
} mode_t_;

static int prep_mode(mode_t_* md, int blk, int32_t S, int32_t K, const float* kr, int32_t N,
                     int32_t Nodd, float Mk, int32_t Wblock, int literal) {
    md->blk = blk; md->S = S; md->K = K; md->M = blk_M(blk);
    md->literal = literal;
    md->Rmax = (int64_t)Nodd * S * K;                                 /* Eq. (3) */
    md->b = or_bits(md->Rmax);                                        /* Eq. (6), eps = 2^-b */
    md->ck = or_compand_factor(K, Mk);                                /* Eq. (2) */
    int32_t* kq = calloc((size_t)Nodd + 1, sizeof(int32_t));
    if (!kq) return OR_ERR_ARG;
    or_compand(kr, N, md->ck, kq);                                    /* k~[N..N'] = 0 */
    if (blk == OR_BLK_SYM && literal) {
        /* Eq. (5) with the paper's eps^-1 = 2 R_max (the swapped pair order above):
         * kbar[n] = k~[2n+1] + eps^-1 k~[2n], an exact integer in FP64 */
        md->nk = (Nodd + 1) / 2;
        md->kpk = malloc(sizeof(double) * (size_t)md->nk);
        if (md->kpk) {
            double einv = 2.0 * (double)md->Rmax;
            for (int32_t n = 0; n < md->nk; ++n) {
                double ko = (2 * n + 1 < Nodd) ? (double)kq[2 * n + 1] : 0.0;
                md->kpk[n] = ko + einv * (double)kq[2 * n];
            }
        }
        md->l1 = 0.0;
    } else if (blk == OR_BLK_SYM) {
        md->nk = (Nodd + 1) / 2;
        md->kpk = malloc(sizeof(double) * (size_t)md->nk);
        or_pack_sym_kernel(kq, Nodd, md->b, md->kpk);                 /* Eq. (5), the pair swapped */
        int64_t l1 = 0;
        for (int32_t n = 0; n < md->nk; ++n) {
            int64_t ko = (2 * n + 1 < Nodd) ? kq[2 * n + 1] : 0;
            int64_t v = ko + ((int64_t)kq[2 * n] << md->b);
            l1 += v < 0 ? -v : v;
        }
        md->l1 = (double)l1;
    } else {
        md->nk = Nodd;
        md->kpk = malloc(sizeof(double) * (size_t)md->nk);
        int64_t l1 = 0;
        for (int32_t n = 0; n < Nodd; ++n) { md->kpk[n] = (double)kq[n]; l1 += kq[n] < 0 ? -kq[n] : kq[n]; }
        md->l1 = (double)l1;
    }
    md->log2n = fft_log2n(blk, Wblock);
    free(kq);
    return md->kpk ? OR_OK : OR_ERR_ARG;
}

/* One block in one packed mode.  Returns 1 if the mode was applied, 0 if the
 * FFT exactness check rejected it. */
static int run_packed_block(const mode_t_* md, const or_plan_t* p, int64_t i, const float* x, float Ms,
                            int fft, int64_t* rq_blk, int32_t* q, double* sbar, double* rbar,
                            or_block_stats_t* st) {
    int32_t Wb = p->Wblock, Nodd = p->Nodd;
    float cs = or_compand_factor(md->S, Ms);                          /* Eq. (2) */
    or_compand(x, Wb, cs, q);
    double eps = ldexp(1.0, -md->b);
    double ferr = 0.0;
    if (fft) {
        int64_t ss = 0;
        for (int32_t t = 0; t < Wb; ++t) ss += (int64_t)q[t] * q[t];
        double grow = md->blk == OR_BLK_SYM ? 1.0 + eps : 1.0 + 2.0 * eps;
        double l2 = sqrt((double)ss) * grow;
        ferr = or_fft_err_digits(md->blk, md->log2n, md->l1, l2, md->b);
        if (!(ferr < 0.25)) return 0;
    }
    int32_t Wstart = (!fft && i == 0) ? 0 : (Nodd - 1) / 2;          /* Eq. (10) */
    if (md->blk == OR_BLK_TC) {
        /* the exact integer convolution of the block, Eq. (1) on s~ and k~ */
        for (int32_t j = 0; j < Wb; ++j) {
            int64_t acc = 0;
            for (int32_t n = 0; n < Nodd && n <= j; ++n) acc += (int64_t)q[j - n] * (int64_t)md->kpk[n];
            rq_blk[j] = acc;
        }
        st->mode = OR_BLK_TC; st->Sq = md->S; st->Kq = md->K; st->b = 0; st->cs = cs;
        st->fft_err = 0.0;
        return 1;
    }
    if (md->literal) {
        /* the paper's own form: eps of Eq. (6), Eq. (4) and Eq. (9) in FP64,
         * Eqs. (11)-(15) in FP64 with u_sys; rounding may move a digit */
        int32_t nbar = Wb / 2;
        double eps_l = 1.0 / (2.0 * (double)md->Rmax);
        for (int32_t m = 0; m < nbar; ++m) sbar[m] = (double)q[2 * m] + eps_l * (double)q[2 * m + 1];
        or_conv_f64(sbar, nbar, md->kpk, md->nk, rbar, nbar);
        double* rqd = rbar + nbar;                                    /* spare room after rbar */
        or_unpack_sym_fp64(rbar, nbar, Wstart, (double)md->Rmax, eps_l, OR_U_SYS, rqd);
        for (int32_t j = 0; j < 2 * nbar; ++j) rq_blk[j] = (int64_t)rqd[j];
    } else if (md->blk == OR_BLK_SYM) {
        int32_t nbar = Wb / 2;
        or_pack_sym_signal(q, Wb, md->b, sbar);                       /* Eq. (4) */
        or_conv_f64(sbar, nbar, md->kpk, md->nk, rbar, nbar);         /* Eq. (9) */
        if (or_unpack_sym(rbar, nbar, Wstart, md->Rmax, md->b, rq_blk)) return -1; /* (11)-(15) */
    } else {
        int32_t Ls = (Wb + md->M - 1) / md->M;
        int32_t nr = Ls + Nodd - 1;
        or_pack_asym_signal(q, Wb, md->M, md->b, sbar);               /* Eq. (7) */
        or_conv_f64(sbar, Ls, md->kpk, md->nk, rbar, nr);             /* Eq. (8) */
        if (or_unpack_asym(rbar, nr, Ls, md->M, md->Rmax, md->b, Wb, rq_blk)) return -1;
    }
    st->mode = md->blk; st->Sq = md->S; st->Kq = md->K; st->b = md->b; st->cs = cs;
    st->fft_err = ferr;
    return 1;
}

int or_apx_conv(const float* s, int64_t L, const float* k, int32_t N, int32_t Wblock, uint32_t mode,
                double snr_db, int32_t Sq_fixed, int32_t Kq_fixed,
                float* r_out, int64_t* rq_out, or_block_stats_t* stats, int nthreads,
                const uint8_t* want) {
    if (!s || !k || !r_out) return OR_ERR_ARG;
    uint32_t op = mode & OR_OP_MASK, core = mode & OR_CORE_MASK, pack = mode & OR_PACK_MASK;
    if (op > OR_OP_XCORR || (core != OR_CORE_DIRECT && core != OR_CORE_FFT && core != OR_CORE_TC) ||
        pack > OR_PACK_ASYM3)
        return OR_ERR_ARG;
    int fft = core == OR_CORE_FFT;
    /* the tensor-core core: the direct core's blocks, one candidate (OR_BLK_TC at
     * the largest S_q = K_q its bound admits) or full precision */
    int tc = core == OR_CORE_TC;
    if (tc && pack != OR_PACK_AUTO && pack != OR_PACK_NONE) return OR_ERR_ARG;
    /* the paper-literal form: symmetric packing, direct core, fixed quantiser */
    int literal = (mode & OR_LITERAL) != 0;
    if (literal && (fft || pack != OR_PACK_SYM)) return OR_ERR_ARG;
    or_plan_t p;
    int rc = or_plan(L, N, Wblock, fft, &p);
    if (rc) return rc;
    int32_t Nodd = p.Nodd, Wb = Wblock;

    /* Section II: xcorr(s, t) = conv(s, reverse(t)). */
    float* kr = calloc((size_t)Nodd, sizeof(float));
    if (!kr) return OR_ERR_ARG;
    for (int32_t n = 0; n < N; ++n) kr[n] = op == OR_OP_XCORR ? k[N - 1 - n] : k[n];
    float Mk = or_maxabs(kr, N);
    double sig2_k = or_second_moment(kr, N, Mk);
    int kfinite = isfinite(Mk);

    /* Kernel initialisation of Section IV: compand and pack once per mode. */
    mode_t_ modes[3];
    int nmodes = 0;
    int order[3] = {OR_BLK_SYM, OR_BLK_ASYM3, OR_BLK_ASYM2};  /* Table 1 ranking */
    if (kfinite && Mk > 0.0f) {
        if (pack == OR_PACK_AUTO && tc) {
            int32_t Q = or_qmax_direct(OR_BLK_TC, Nodd);
            if (Q >= 1) {
                if (prep_mode(&modes[0], OR_BLK_TC, Q, Q, kr, N, Nodd, Mk, Wb, 0)) rc = OR_ERR_ARG;
                else nmodes = 1;
            }
        } else if (pack == OR_PACK_AUTO) {
            for (int j = 0; j < 3; ++j) {
                int32_t Q = fft ? or_qmax_fft(order[j], Nodd, Wb) : or_qmax_direct(order[j], Nodd);
                if (Q < 1) continue;
                if (prep_mode(&modes[nmodes], order[j], Q, Q, kr, N, Nodd, Mk, Wb, 0)) { rc = OR_ERR_ARG; break; }
                ++nmodes;
            }
        } else if (pack != OR_PACK_NONE) {
            int blk = pack == OR_PACK_SYM ? OR_BLK_SYM : (pack == OR_PACK_ASYM2 ? OR_BLK_ASYM2 : OR_BLK_ASYM3);
            if (Sq_fixed < 1 || Kq_fixed < 1 || Sq_fixed > (1 << 20) || Kq_fixed > (1 << 20)) rc = OR_ERR_ARG;
            else if (literal && (int64_t)Nodd * Sq_fixed * Kq_fixed > ((int64_t)1 << 31)) rc = OR_ERR_RANGE;
            else if (!literal && !or_exact_ok(blk, Nodd, Sq_fixed, Kq_fixed)) rc = OR_ERR_RANGE;
            else if (prep_mode(&modes[0], blk, Sq_fixed, Kq_fixed, kr, N, Nodd, Mk, Wb, literal)) rc = OR_ERR_ARG;
            else nmodes = 1;
        }
    }
    if (rc) { for (int j = 0; j < nmodes; ++j) free(modes[j].kpk); free(kr); return rc; }
    double thr = pow(10.0, (snr_db + or_snr_margin_db(p.W)) / 10.0);  /* Section IV.D minimum */

    for (int64_t g = 0; g < p.out_len; ++g) { r_out[g] = 0.0f; if (rq_out) rq_out[g] = 0; }

    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    (void)nthreads;
    int err = 0;
#pragma omp parallel num_threads(nt)
    {
        float* x = malloc(sizeof(float) * (size_t)Wb);
        int32_t* q = malloc(sizeof(int32_t) * (size_t)Wb);
        double* sbar = malloc(sizeof(double) * (size_t)Wb);
        double* rbar = malloc(sizeof(double) * (size_t)(2 * Wb + Nodd));
        int64_t* rqb = malloc(sizeof(int64_t) * (size_t)Wb);
        if (!x || !q || !sbar || !rbar || !rqb) {
#pragma omp atomic write
            err = OR_ERR_ARG;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < p.P; ++i) {
            if (err) continue;
            int64_t st0 = or_block_start(&p, i);
            for (int32_t t = 0; t < Wb; ++t) {
                int64_t gi = st0 + t;
                x[t] = (gi >= 0 && gi < L) ? s[gi] : 0.0f;
            }
            int32_t lo, hi;
            or_block_out_range(&p, i, &lo, &hi);
            or_block_stats_t st;
            memset(&st, 0, sizeof st);
            float Ms = or_maxabs(x, Wb);                              /* ||s||_inf */
            st.maxabs = Ms;
            int kind;  /* 0 full, 1 packed, 2 zero, 3 nonfinite */
            const mode_t_* used = NULL;
            if (!isfinite(Ms) || !kfinite) kind = 3;
            else if (Ms == 0.0f || Mk == 0.0f) kind = 2;
            else {
                st.sigma2 = or_second_moment(x, Wb, Ms);
                kind = 0;
                for (int j = 0; j < nmodes && kind == 0; ++j) {
                    const mode_t_* md = &modes[j];
                    if (pack == OR_PACK_AUTO &&
                        !or_snr_feasible(st.sigma2, Ms, sig2_k, Mk, md->S, md->K, thr))
                        continue;                                     /* Section IV.D */
                    int ok = run_packed_block(md, &p, i, x, Ms, fft, rqb, q, sbar, rbar, &st);
                    if (ok < 0) {
#pragma omp atomic write
                        err = OR_ERR_INEXACT;
                    }
                    if (ok == 1) {
                        kind = 1;
                        used = md;
                        st.snr_pred_db = or_snr_model_db(st.sigma2, Ms, sig2_k, Mk, md->S, md->K);
                    }
                }
            }
            for (int32_t j = lo; j < hi; ++j) {
                int64_t g = st0 + j;                                  /* Eq. (17) */
                if (g < 0 || g >= p.out_len) continue;
                if (kind == 1) {
                    /* Eq. (16): r = (c_s c_k)^-1 r~ */
                    double sc = (double)st.cs * (double)used->ck;
                    r_out[g] = (float)((double)rqb[j] / sc);
                    if (rq_out) rq_out[g] = rqb[j];
                } else if (kind == 0) {
                    /* no admissible packing: full precision, Eq. (1) over the window
                     * (only where the caller asked for it: want[g] != 0 or want NULL) */
                    if (want && !want[g]) continue;
                    double acc = 0.0;
                    for (int32_t n = 0; n < N; ++n) {
                        int32_t t = j - n;
                        if (t >= 0) acc += (double)x[t] * (double)kr[n];
                    }
                    r_out[g] = (float)acc;
                } else if (kind == 3) {
                    r_out[g] = NAN;
                }
            }
            if (kind == 0) { st.mode = OR_BLK_FULL; st.snr_pred_db = INFINITY; }
            if (kind == 2) { st.mode = OR_BLK_ZERO; st.snr_pred_db = INFINITY; }
            if (kind == 3) { st.mode = OR_BLK_NONFINITE; st.snr_pred_db = NAN; }
            if (stats) stats[i] = st;
        }
        free(x); free(q); free(sbar); free(rbar); free(rqb);
    }
    for (int j = 0; j < nmodes; ++j) free(modes[j].kpk);
    free(kr);
    return err;
}

/* ---- filterbank on exact small integers ------------------------------------
 * The same three steps as the packed path, Eq. (2) companding per block,
 * an exact integer convolution (here plain int64 sums, Eq. (1) on the
 * quantized values), Eq. (16) inverse companding, for F kernels sharing one
 * input.  The block is the set of T consecutive outputs, and its window is
 * every input sample those outputs touch. */
int or_filterbank(const float* s, int64_t L, const float* kbank, int32_t F, int32_t N, int32_t T,
                  int32_t Sq, int32_t Kq, int64_t b0, int64_t b1, float* y, int64_t ldy, int64_t* yq,
                  float* block_cs, int nthreads) {
    if (!s || !kbank || !y || L < 1 || F < 1 || N < 1 || T < 1 || Sq < 1 || Kq < 1) return OR_ERR_ARG;
    const int64_t out_len = L + N - 1;
    const int64_t nb = (out_len + T - 1) / T;
    if (ldy < out_len || b0 < 0 || b1 > nb || b0 > b1) return OR_ERR_ARG;
    for (int64_t i = 0; i < L; ++i) if (!isfinite(s[i])) return OR_ERR_RANGE;
    for (int64_t i = 0; i < (int64_t)F * N; ++i) if (!isfinite(kbank[i])) return OR_ERR_RANGE;

    /* Eq. (2) on each filter, once */
    int32_t* kq = malloc(sizeof(int32_t) * (size_t)F * (size_t)N);
    float* ck = malloc(sizeof(float) * (size_t)F);
    if (!kq || !ck) { free(kq); free(ck); return OR_ERR_ARG; }
    for (int32_t f = 0; f < F; ++f) {
        const float* kf = kbank + (int64_t)f * N;
        float Mk = or_maxabs(kf, N);
        ck[f] = Mk > 0.0f ? or_compand_factor(Kq, Mk) : 0.0f;
        if (Mk > 0.0f) or_compand(kf, N, ck[f], kq + (int64_t)f * N);
        else for (int32_t n = 0; n < N; ++n) kq[(int64_t)f * N + n] = 0;
    }
    const int64_t nw = (int64_t)T + N - 1;
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    (void)nthreads;
    int err = 0;
#pragma omp parallel num_threads(nt)
    {
        float* w = malloc(sizeof(float) * (size_t)nw);
        int32_t* q = malloc(sizeof(int32_t) * (size_t)nw);
        if (!w || !q) {
#pragma omp atomic write
            err = OR_ERR_ARG;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = b0; i < b1; ++i) {
            if (err) continue;
            const int64_t t0 = i * T;
            for (int64_t u = 0; u < nw; ++u) {
                int64_t g = t0 - N + 1 + u;
                w[u] = (g >= 0 && g < L) ? s[g] : 0.0f;
            }
            const float Ms = or_maxabs(w, nw);
            const float cs = Ms > 0.0f ? or_compand_factor(Sq, Ms) : 0.0f;   /* Eq. (2) */
            if (block_cs) block_cs[i] = cs;
            if (Ms > 0.0f) or_compand(w, nw, cs, q);
            const int64_t t1 = t0 + T < out_len ? t0 + T : out_len;
            for (int32_t f = 0; f < F; ++f) {
                const int32_t* kf = kq + (int64_t)f * N;
                for (int64_t t = t0; t < t1; ++t) {
                    int64_t acc = 0;
                    if (Ms > 0.0f && ck[f] > 0.0f)
                        for (int32_t n = 0; n < N; ++n)                          /* Eq. (1) */
                            acc += (int64_t)q[t - t0 + N - 1 - n] * (int64_t)kf[n];
                    double sc = (double)cs * (double)ck[f];
                    y[(int64_t)f * ldy + t] = acc == 0 ? 0.0f : (float)((double)acc / sc);  /* Eq. (16) */
                    if (yq) yq[(int64_t)f * ldy + t] = acc;
                }
            }
        }
        free(w);
        free(q);
    }
    free(kq);
    free(ck);
    return err;
}
