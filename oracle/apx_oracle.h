/*
 * apx_oracle.h -- plain, slow FP64 CPU oracle for approximate overlap-save
 * convolution with companding and tight packing (Anam & Andreopoulos,
 * "Throughput Scaling Of Convolution For Error-Tolerant Multimedia
 * Applications", arXiv 1201.3018).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares nothing with
 * the CUDA library: its own header, its own constants, its own arithmetic.
 *
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent, ambiguous or garbled the reading taken is stated beside the code:
 * the block geometry, the kernel-pair order of symmetric packing, a
 * power-of-two epsilon, the u_sys term, the exactness bounds, the asymmetric
 * layout, FFT exactness, rounding, cross-correlation, the per-block selector
 * and SNR measurement.
 */
#ifndef APX_ORACLE_H
#define APX_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* mode word: op | core | pack (same bit layout as the public ABI) */
#define OR_OP_CONV      0x0u
#define OR_OP_XCORR     0x1u
#define OR_OP_MASK      0xFu
#define OR_CORE_DIRECT  0x00u
#define OR_CORE_FFT     0x10u
#define OR_CORE_TC      0x30u   /* time-domain core on the tensor cores: FP16 integers, FP32 sums */
#define OR_CORE_MASK    0xF0u
#define OR_PACK_AUTO    0x000u
#define OR_PACK_NONE    0x100u
#define OR_PACK_SYM     0x200u
#define OR_PACK_ASYM2   0x300u
#define OR_PACK_ASYM3   0x400u
#define OR_PACK_MASK    0xF00u
/* with OR_PACK_SYM on the direct core and a fixed quantiser: the paper's own
 * packing coefficient eps = (2 R_max)^-1 (Eq. 6) and Eqs. (11)-(15) in FP64
 * with u_sys (Section IV) instead of the exact power-of-two form */
#define OR_LITERAL      0x2000u
#define OR_U_SYS        3.1193e-11  /* Section IV, from the machine-precision measurement the paper cites */

/* per-block mode codes (what a block actually ran) */
#define OR_BLK_FULL  0
#define OR_BLK_SYM   1
#define OR_BLK_ASYM2 2
#define OR_BLK_ASYM3 3
#define OR_BLK_ZERO  4   /* ||s||_inf == 0 or ||k||_inf == 0: output is exactly 0 */
#define OR_BLK_NONFINITE 5
#define OR_BLK_TC    6   /* the block's companded integers convolved exactly in FP16 x FP16 -> FP32 */

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_WBLOCK (-2)
#define OR_ERR_RANGE (-3)
#define OR_ERR_INEXACT (-4)

typedef struct {
    int64_t L;        /* input length */
    int32_t N;        /* kernel length as given */
    int32_t Nodd;     /* N' = N rounded up to odd (Section III, one zero tap) */
    int32_t Wblock;   /* samples per block */
    int32_t W;        /* outputs per block: W = Wblock - N' - 1 (Section III) */
    int32_t fft;      /* 1: FFT-core geometry (leading head blocks), 0: Eq. (17) as printed */
    int32_t head;     /* FFT core: number of head blocks in front, ceil((N'-1)/W) */
    int64_t P;        /* number of blocks */
    int64_t out_len;  /* L + N - 1 */
} or_plan_t;

typedef struct {
    int32_t mode;      /* OR_BLK_* */
    int32_t Sq, Kq;    /* companding ranges used */
    int32_t b;         /* epsilon = 2^-b */
    float   cs;        /* c_s of Eq. (2) */
    float   maxabs;    /* ||s||_inf over the block window */
    double  sigma2;    /* fixed-point second moment of the window */
    double  snr_pred_db;  /* Table 1 model (derived from Eqs. 18-19) for the chosen mode; inf for full */
    double  fft_err;   /* FFT error bound in units of the finest digit (0 for the direct core) */
} or_block_stats_t;

/* ---- plain definitions --------------------------------------------------- */
void or_conv_ref(const double* s, int64_t L, const double* k, int32_t N, double* r);
void or_xcorr_ref(const double* s, int64_t L, const double* t, int32_t N, double* r);
void or_conv_int(const int64_t* s, int64_t L, const int64_t* k, int32_t N, int64_t* r);
void or_conv_ref_at(const double* s, int64_t L, const double* k, int32_t N, const int64_t* idx, int64_t n,
                    double* r);

/* ---- a1: block plan ------------------------------------------------------ */
int     or_plan(int64_t L, int32_t N, int32_t Wblock, int fft, or_plan_t* p);
int64_t or_block_start(const or_plan_t* p, int64_t i);
void    or_block_out_range(const or_plan_t* p, int64_t i, int32_t* lo, int32_t* hi);

/* ---- a3: statistics ------------------------------------------------------ */
float  or_maxabs(const float* x, int64_t n);
double or_second_moment(const float* x, int64_t n, float maxabs);

/* ---- a4: exactness bounds and selection ----------------------------------- */
int32_t or_bits(int64_t Rmax);
int     or_exact_ok(int blkmode, int32_t Nodd, int32_t Sq, int32_t Kq);
int32_t or_qmax_direct(int blkmode, int32_t Nodd);
int32_t or_qmax_fft(int blkmode, int32_t Nodd, int32_t Wblock);
double  or_snr_model_lin(double sig2_s, float Ms, double sig2_k, float Mk, int32_t Sq, int32_t Kq);
double  or_snr_model_db(double sig2_s, float Ms, double sig2_k, float Mk, int32_t Sq, int32_t Kq);
int     or_snr_feasible(double sig2_s, float Ms, double sig2_k, float Mk, int32_t Sq, int32_t Kq, double thr_lin);
/* margin in dB by which the model must clear the target (W = outputs kept per block) */
double  or_snr_margin_db(int32_t W);
double  or_fft_err_digits(int blkmode, int32_t log2n, double l1_kbar, double l2_sbar, int32_t b);

/* ---- a5/a6: compand and pack --------------------------------------------- */
float or_compand_factor(int32_t Q, float maxabs);
void  or_compand(const float* x, int64_t n, float c, int32_t* q);
void  or_pack_sym_signal(const int32_t* sq, int32_t n, int32_t b, double* sbar);
void  or_pack_sym_kernel(const int32_t* kq, int32_t Nodd, int32_t b, double* kbar);
void  or_pack_sym_kernel_printed(const int32_t* kq, int32_t Nodd, int32_t b, double* kbar);
void  or_pack_asym_signal(const int32_t* sq, int32_t n, int32_t M, int32_t b, double* sbar);

/* ---- a7: block convolution cores ----------------------------------------- */
void or_conv_f64(const double* a, int64_t na, const double* k, int64_t nk, double* r, int64_t nr);
int  or_conv_f64_fft(const double* a, int64_t na, const double* k, int64_t nk, double* r, int64_t nr, int64_t n);

/* ---- a8: unpack ---------------------------------------------------------- */
int  or_unpack_sym(const double* rbar, int32_t nbar, int32_t Wstart, int64_t Rmax, int32_t b, int64_t* rq);
int  or_unpack_sym_digits(const double* rbar, int32_t nbar, int32_t Wstart, int32_t b, int64_t* rq);
void or_unpack_sym_fp64(const double* rbar, int32_t nbar, int32_t Wstart, double Rmax, double eps,
                        double u_sys, double* rq);
int  or_unpack_asym(const double* rbar, int32_t nr, int32_t Ls, int32_t M, int64_t Rmax, int32_t b,
                    int32_t nout, int64_t* rq);

/* ---- a1..a9: whole pipeline ---------------------------------------------- */
int or_apx_conv(const float* s, int64_t L, const float* k, int32_t N, int32_t Wblock, uint32_t mode,
                double snr_db, int32_t Sq_fixed, int32_t Kq_fixed,
                float* r_out, int64_t* rq_out, or_block_stats_t* stats, int nthreads,
                const uint8_t* want);

/* ---- filterbank on exact small integers (time-domain Toeplitz reading) ---
 * Eq. (1) for F kernels at once with the companding of Eq. (2) applied per
 * block of T consecutive outputs and the inverse companding of Eq. (16).
 * Block i quantizes the input window its outputs depend on,
 * s[iT-N+1 .. iT+T-1] (zero outside [0, L)), with c_s = S_q / ||window||_inf;
 * filter f is quantized once with c_k = K_q / ||k_f||_inf.  The integer
 * convolution is exact (int64) and y = r~ / (c_s c_k) (Eq. 16) rounded once
 * to FP32.  An all-zero window or an all-zero filter gives exact zeros.
 * Only blocks [b0, b1) are written (y, yq: F rows of ldy entries; yq and
 * block_cs may be NULL).  Returns OR_ERR_RANGE for a non-finite sample. */
int or_filterbank(const float* s, int64_t L, const float* kbank, int32_t F, int32_t N, int32_t T,
                  int32_t Sq, int32_t Kq, int64_t b0, int64_t b1, float* y, int64_t ldy, int64_t* yq,
                  float* block_cs, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
