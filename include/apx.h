/*
 * apx.h -- C ABI of libapx.so: GB300 (sm_103a) approximate overlap-save
 * convolution and cross-correlation with per-block companding and tight
 * packing, after Anam & Andreopoulos, "Throughput Scaling Of Convolution For
 * Error-Tolerant Multimedia Applications" (arXiv 1201.3018).
 *
 * The problem (Section II, Eq. 1): r_out[m] = sum_{n<N} s_in[m-n] k[n] for
 * m in [0, L+N-1).  Overlap-save splits s_in into P blocks of W_block samples
 * (Section III).  Per block the middle layer compands the block (Eq. 2),
 * packs pairs or triples of small integers into one FP64 word (symmetric
 * packing, Eqs. 4-5; asymmetric packing, Eq. 7), convolves the packed words
 * with a direct or FFT core (Eqs. 8-9), unpacks (Eqs. 11-15), inverts the
 * companding (Eq. 16) and places the block's W outputs (Eq. 17).  Under an SNR target the
 * packing and companding range are chosen per block from the block's marginal
 * statistics (Table 1 model, Section IV.D); when no packing meets the target
 * the block runs in full precision (FP32).
 *
 * Conventions for every call below:
 *  - Pointers named s_in, k, r_out, rq_out and stats are DEVICE pointers on the
 *    context's device unless a call says "host".  The caller owns them.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL
 *    = legacy default stream).  Argument errors are returned immediately;
 *    data-dependent errors (non-finite input) are recorded in the context and
 *    returned by apx_sync().
 *  - Layouts: all arrays are dense, contiguous, element 0 first.
 *  - Return value: APX_OK (0) or a negative APX_ERR_* code; apx_strerror()
 *    names it.  No call aborts the process.
 *  - A context is not thread-safe: one host thread issues its calls.
 */
#ifndef APX_H
#define APX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define APX_OK              0
#define APX_ERR_ARG        (-1)  /* null pointer, bad length, bad mode bits   */
#define APX_ERR_WBLOCK     (-2)  /* W_block odd, < N'+3, too large, or not a power of two (FFT core) */
#define APX_ERR_RANGE      (-3)  /* fixed S_q/K_q beyond the packing's exactness bound */
#define APX_ERR_NONFINITE  (-4)  /* NaN/Inf in the input or kernel (outputs of the affected blocks are NaN) */
#define APX_ERR_OOM        (-5)  /* device allocation failed                   */
#define APX_ERR_BUDGET     (-6)  /* request needs more workspace than the context's budget */
#define APX_ERR_CUDA       (-7)  /* a CUDA runtime call failed                  */
#define APX_ERR_TIMEOUT    (-8)  /* a bounded device wait gave up               */
#define APX_ERR_CHECK      (-9)  /* a device bounds check failed (builds with
                                    APX_CHECKED only; the access was skipped)  */

/* ---- mode word: op | core | pack ------------------------------------- */
#define APX_OP_CONV      0x000u  /* Eq. (1)                                   */
#define APX_OP_XCORR     0x001u  /* x[l+N-1] = sum_n s[n+l] t[n], l in [-(N-1), L-1] */
#define APX_CORE_DIRECT  0x000u  /* time-domain block convolution             */
#define APX_CORE_FFT     0x010u  /* frequency-domain block convolution (W_block a power of two) */
#define APX_CORE_AUTO    0x020u  /* batched calls only: the library picks the core */
#define APX_CORE_TC      0x030u  /* time-domain blocks on the tensor cores: one
                                    candidate, the block's companded integers in
                                    FP16 at the largest S_q = K_q with
                                    N' S_q K_q <= 2^24 (and <= 2048), summed
                                    exactly in FP32 (Eq. 2 range, Eq. 3); blocks
                                    the Section IV.D model does not admit run
                                    full precision.  W_block a multiple of 64 up
                                    to 8192, N' <= 449; APX_PACK_AUTO or
                                    APX_PACK_NONE */
#define APX_PACK_AUTO    0x000u  /* per-block choice under snr_target_db (Section IV.D) */
#define APX_PACK_NONE    0x100u  /* full precision, FP32                        */
#define APX_PACK_SYM     0x200u  /* symmetric packing, Eqs. (4)-(5)            */
#define APX_PACK_ASYM2   0x300u  /* asymmetric packing, M = 2, Eq. (7)         */
#define APX_PACK_ASYM3   0x400u  /* asymmetric packing, M = 3, Eq. (7)         */
#define APX_FULL_FP64    0x1000u /* with APX_PACK_NONE and the direct core: the
                                    full-precision convolution in FP64 (the
                                    paper's full-precision baseline runs in FP64),
                                    rounded once to FP32 on output              */
#define APX_LITERAL      0x2000u /* with APX_PACK_SYM, the direct core and a fixed
                                    quantiser (apx_conv_fixed): the paper's own
                                    eps = (2 R_max)^-1 (Eq. 6) and Eqs. (11)-(15)
                                    in FP64 with u_sys = 3.1193e-11 (Section IV)
                                    instead of the exact power-of-two form.
                                    Rounding can move a digit (the paper measures
                                    the result by SNR); R_max = N' S_q K_q up to
                                    2^31, beyond the exact form's bound.  The
                                    packed block convolution runs without fused
                                    multiply-adds, as the equations are written.
                                    Single calls only (batched calls reject it). */

/* ---- per-block modes reported in apx_block_stats.mode ----------------- */
#define APX_BLK_FULL      0
#define APX_BLK_SYM       1
#define APX_BLK_ASYM2     2
#define APX_BLK_ASYM3     3
#define APX_BLK_ZERO      4      /* ||s||_inf = 0 or ||k||_inf = 0: exact zeros   */
#define APX_BLK_NONFINITE 5
#define APX_BLK_TC        6      /* companded integers convolved on the tensor cores (APX_CORE_TC) */

/* What one block did.  48 bytes, naturally aligned. */
typedef struct {
    int32_t mode;         /* APX_BLK_*                                         */
    int32_t Sq, Kq;       /* companding ranges of Eq. (2) (0 for full)          */
    int32_t b;            /* packing coefficient eps = 2^-b (Eq. 6, power of two) */
    float   cs;           /* c_s = S_q / ||s||_inf of the block                 */
    float   maxabs;       /* ||s||_inf over the block's W_block window          */
    double  sigma2;       /* second moment of the window (24-bit fixed point)   */
    double  snr_pred_db;  /* Table 1 model SNR of the chosen packing (inf: full) */
    double  fft_err;      /* FFT core: error bound in units of the finest digit */
} apx_block_stats;

typedef struct apx_ctx apx_ctx;

/* Create a context on CUDA device `device`.  It owns a device workspace for
 * prepared kernels (companded/packed taps, kernel spectra, twiddles), grown on
 * demand up to mem_budget_bytes (0 = 4 GiB).  *out receives the handle.
 * Errors: APX_ERR_ARG (out NULL, bad device), APX_ERR_CUDA. */
int apx_create(apx_ctx** out, int device, size_t mem_budget_bytes);

/* Free the context and its workspace (synchronises its device).  NULL is a no-op. */
void apx_destroy(apx_ctx* ctx);

/* Host-only block plan (Section III, Eq. 17).  For length-L input, length-N
 * kernel and W_block samples per block: *W = W_block - N' - 1 outputs per
 * block (N' = N rounded up to odd) and *P blocks.  The FFT core adds
 * ceil((N'-1)/W) head blocks in front (a circular block convolution cannot
 * produce the first block's leading outputs).  Either out pointer may be NULL.
 * Errors: APX_ERR_ARG, APX_ERR_WBLOCK. */
int apx_plan_blocks(int64_t L, int32_t N, int32_t W_block, uint32_t mode, int64_t* P, int32_t* W);

/* Host-only: the packing candidates that apx_conv (or apx_conv_host,
 * apx_conv_batch) with this mode and target gives its blocks, in the order a
 * block tries them (Table 1: symmetric, asymmetric M = 3, asymmetric M = 2).
 * With APX_PACK_AUTO every packing at the largest S_q = K_q = Q for which the
 * FP64 packed convolution stays exact (every packed word, product and partial
 * sum an integer multiple of the finest digit 2^-b below 2^53; the FFT core
 * also keeps its a-priori rounding-error bound below a quarter digit), less
 * those whose Section IV.D model misses the target plus its margin even at
 * ratios sigma^2 / ||.||_inf^2 = 1 for block and kernel (checked 1 % below):
 * no block could pick them.  The margin is 0.5 + 48 / sqrt(W) dB, W =
 * W_block - N' - 1 the outputs kept per block: the model gives the SNR a
 * block can expect, and a packing is admitted only where every block's
 * measured SNR stays at or above the target.  A single packing bit gives that
 * packing alone, APX_PACK_NONE none.
 * Writes up to 3 entries: blk[i] (APX_BLK_*), q[i] = S_q = K_q, b[i] (eps =
 * 2^-b); any output pointer may be NULL.  Returns the count (0 to 3), or
 * APX_ERR_ARG, APX_ERR_WBLOCK, APX_ERR_RANGE as apx_conv would. */
int apx_plan_candidates(int64_t L, int32_t N, int32_t W_block, uint32_t mode, double snr_target_db, int32_t* blk,
                        int32_t* q, int32_t* b);

/* Approximate convolution / cross-correlation under a per-block SNR target
 * (pack bits APX_PACK_AUTO; Section IV.D), or with a forced packing whose
 * S_q = K_q is the largest the packing's exactness bound admits.
 *   s_in   : device, L FP32 samples
 *   k      : device, N FP32 taps (the template t for APX_OP_XCORR)
 *   r_out  : device, L+N-1 FP32 outputs
 *   rq_out : device or NULL, L+N-1 int32: the exact integer-domain result
 *            r~ = s~ * k~ of Eqs. (11)-(15) for outputs of packed blocks, 0 elsewhere
 *   stats  : device or NULL, P entries (apx_plan_blocks with the same mode)
 * Errors: APX_ERR_ARG, APX_ERR_WBLOCK, APX_ERR_BUDGET, APX_ERR_OOM, APX_ERR_CUDA. */
int apx_conv(apx_ctx* ctx, const float* s_in, int64_t L, const float* k, int32_t N, int32_t W_block,
             uint32_t mode, double snr_target_db, float* r_out, int32_t* rq_out,
             apx_block_stats* stats, void* stream);

/* As apx_conv with a fixed companding range (S_q, K_q in [1, 2^20]) for every
 * block and the packing given by the pack bits (SYM, ASYM2 or ASYM3).  Errors
 * as apx_conv, plus APX_ERR_RANGE when N' S_q K_q exceeds the packing's
 * exactness bound.  With the FFT core a block whose error bound exceeds 1/4
 * digit runs in full precision instead (its stats say so). */
int apx_conv_fixed(apx_ctx* ctx, const float* s_in, int64_t L, const float* k, int32_t N,
                   int32_t W_block, uint32_t mode, int32_t S_q, int32_t K_q, float* r_out,
                   int32_t* rq_out, apx_block_stats* stats, void* stream);

/* Full-precision twin (no companding, no packing): FP32 overlap-save with the
 * same block geometry and core.  Pack bits are ignored. */
int apx_conv_full(apx_ctx* ctx, const float* s_in, int64_t L, const float* k, int32_t N,
                  int32_t W_block, uint32_t mode, float* r_out, void* stream);

/* End-to-end variant for callers holding HOST data: s_in (host, L), k (host,
 * N) in, r_out (host, L+N-1) out, apx_conv (S_q = K_q = 0) or apx_conv_fixed
 * on `stream`, which is then synchronised.  When all three buffers are
 * page-locked and addressable by the device (cudaHostAlloc or registered),
 * the kernels read and write them in place over the host link, overlapping
 * the transfers with the computation; otherwise s_in and k are copied to
 * device staging buffers from the context workspace and r_out is copied back.
 * The results are the same either way.  Returns the apx_sync() status. */
int apx_conv_host(apx_ctx* ctx, const float* s_in_host, int64_t L, const float* k_host, int32_t N,
                  int32_t W_block, uint32_t mode, double snr_target_db, int32_t S_q, int32_t K_q,
                  float* r_out_host, void* stream);

/* Wait for `stream` and return the data-dependent status of the calls issued
 * since the previous apx_sync (APX_OK, APX_ERR_NONFINITE, APX_ERR_TIMEOUT when
 * a bounded device-side wait gave up, or APX_ERR_CHECK when a bounds check of
 * a checked build failed), then clear it. */
int apx_sync(apx_ctx* ctx, void* stream);

/* Number of CUDA kernel launches this context has issued since creation. */
int64_t apx_launch_count(const apx_ctx* ctx);

/* ---- tracing: per-kernel device time ------------------------------------
 * With profiling enabled the context records a CUDA event pair on the
 * launching stream around every kernel it launches.  apx_profile_read waits
 * for the recorded events, writes the summed milliseconds and the launch count
 * per kernel kind (APX_PHASE_*) into ms[APX_NPHASES] and n[APX_NPHASES] (either
 * may be NULL), and clears the record.  Errors: APX_ERR_ARG, APX_ERR_CUDA. */
#define APX_PHASE_DIRECT  0   /* direct core: the single fused block kernel        */
#define APX_PHASE_SPECTRA 1   /* FFT core: FP32 kernel spectrum (direct DFT)       */
#define APX_PHASE_FFT     2   /* FFT core: block kernel (packed spectra on demand) */
#define APX_PHASE_TC_PREP 3   /* filterbank: block companding and Toeplitz columns */
#define APX_PHASE_TC_MMA  4   /* filterbank: tensor-core GEMM and inverse companding */
#define APX_NPHASES       5
int apx_profile(apx_ctx* ctx, int enable);
int apx_profile_read(apx_ctx* ctx, double* ms, int64_t* n);

/* Test hook for the failure path (the paper has no counterpart).  The next
 * FFT-core call of this context finds every packed kernel spectrum claimed by
 * a builder that never publishes it, so each block that selects a packing
 * waits in its bounded spin, gives up after about one second of SM clock,
 * writes NaN for its outputs and sets the timeout bit: apx_sync then returns
 * APX_ERR_TIMEOUT, and the context stays usable for the next call.  Nothing
 * faults or hangs.  Errors: APX_ERR_ARG. */
int apx_test_stall_next(apx_ctx* ctx);

/* Test hook for the one-launch FFT core's ticket check (no counterpart in the
 * paper).  Moves the context's count of CTA tickets handed out by n without
 * launching anything, as a bookkeeping fault would.  The next one-launch call
 * finds its tickets out of range in every CTA, touches no output, and apx_sync
 * returns APX_ERR_CHECK; apx_sync then reads the device counter back, so the
 * call after that is correct again.  Errors: APX_ERR_ARG. */
int apx_test_skew_tickets(apx_ctx* ctx, int64_t n);

/* Static string naming a status code. */
const char* apx_strerror(int status);

/* ---- batched calls ---------------------------------------------------------
 * Many independent signals in one call (Section II: overlap-save blocks are
 * independent, so the blocks of all requests share each launch).  Requests are
 * grouped by core, W_block and whether any packing candidate remains for them
 * (apx_plan_candidates: the candidates' FP64 buffers set a group's shared
 * memory); each group is one launch of the direct kernel or three of the FFT
 * core (spectrum, combine, block kernel).  Each request's result equals that
 * of the corresponding single call. */
typedef struct {
    const float* s_in;      /* device, L samples                                  */
    int64_t L;
    const float* k;         /* device, N taps (template for cross-correlation)    */
    int32_t N;
    float* r_out;           /* device, L+N-1 outputs                              */
    int32_t W_block;        /* 0: the library's default for the core and N        */
    uint32_t mode;          /* op | core (APX_CORE_AUTO allowed) | pack           */
    double snr_target_db;   /* APX_PACK_AUTO: per-block target (Section IV.D)     */
    int32_t S_q, K_q;       /* > 0 with SYM / ASYM2 / ASYM3: fixed quantiser      */
    int32_t* rq_out;        /* device or NULL: L+N-1 integer-domain outputs, as apx_conv's rq_out */
    apx_block_stats* stats; /* device or NULL: one record per block, as apx_conv's stats */
} apx_request;

/* Enqueue all requests on `stream`.  Errors: any single-call error of a request
 * (the whole batch is rejected before anything is enqueued), APX_ERR_OOM,
 * APX_ERR_BUDGET, APX_ERR_CUDA.  The context's batch workspace is reused by the
 * next batched call: calls on different streams must not overlap. */
int apx_conv_batch(apx_ctx* ctx, const apx_request* reqs, int32_t n, void* stream);

/* The same from HOST buffers: s_in, k and r_out of every request are host
 * pointers (rq_out and stats must be NULL: APX_ERR_ARG otherwise).  A request whose three buffers are page-locked and addressable by
 * the device runs on them in place (the kernels read and write them over the
 * host link).  For the others `stream` gets one host-to-device copy per input
 * into device copies and one device-to-host copy per output after the batched
 * launches (pageable memory makes those copies synchronous).  The outputs are
 * valid once the stream has reached the end of the call, and the host buffers
 * must stay valid until then.  The device copies live in the context (grown on
 * demand, budget-checked) and are reused by the next call on any stream.
 * Errors: as apx_conv_batch (nothing is enqueued for an invalid batch). */
int apx_conv_batch_host(apx_ctx* ctx, const apx_request* reqs, int32_t n, void* stream);

/* A batch captured once into a CUDA graph and replayed: apx_graph_create plans
 * the requests, gives the graph its own workspace (device memory allocated
 * here, not from the context budget), and captures the launches; every
 * apx_graph_launch recomputes everything from the current contents of the
 * requests' inputs into their outputs (the pointers are fixed at creation).
 * The context must outlive the graph (its status word reports non-finite
 * input through apx_sync). */
typedef struct apx_graph apx_graph;
int apx_graph_create(apx_ctx* ctx, const apx_request* reqs, int32_t n, void* stream, apx_graph** out);
int apx_graph_launch(apx_graph* graph, void* stream);
int64_t apx_graph_launch_count(const apx_graph* graph);  /* kernel launches per replay */
void apx_graph_destroy(apx_graph* graph);

/* ---- filterbank on the tensor cores ---------------------------------------
 * F kernels applied to one input, y_f = s * k_f (Eq. 1), through the paper's
 * companding layer: every block of T consecutive outputs quantizes the input
 * window those outputs depend on, s[bT-N+1 .. bT+T-1], with its own factor
 * c_s = S_q / ||window||_inf; kernel f is quantized once with
 * c_k = K_q / ||k_f||_inf (Eq. 2, round half to even on the FP32 product); the
 * integer convolution is exact; y = r~ / (c_s c_k) (Eq. 16).  The exact
 * integer arithmetic runs on the tensor cores (FP16 integers, or FP8 E4M3
 * integers when S_q, K_q <= 16, with FP32 accumulation), which is exact because
 * every companded integer is exact in the operand type and N * S_q * K_q <=
 * 2^24; it replaces the FP64 packing of Section III, whose gain does not carry
 * over to a GPU whose FP64 rate is a small fraction of its FP32 and tensor
 * rates.
 *   s_in     : device, L samples (FP32)
 *   k_bank   : device, F x N taps, row-major (FP32)
 *   S_q, K_q : 1 .. 2048 with N * S_q * K_q <= 2^24, else APX_ERR_RANGE
 *   y_out    : device, F rows of ldy floats, y_f[t] at y_out[f * ldy + t] for
 *              t < L+N-1; ldy >= L+N-1, a multiple of 4, y_out 16-byte aligned
 *   yq_out   : NULL or device int32 like y_out: the integer outputs r~
 *   block_cs : NULL or device, one float per block: c_s (0 for an all-zero window)
 * T = 128 * P outputs per block with P = 256 (F = 1), 128 (F = 2) or 64 (F >= 3)
 * for FP16 operands and P = 256 (F = 1) or 128 (F >= 2) for FP8 operands; the
 * number of blocks is ceil((L+N-1) / T).  Limits: F <= 1024, N <= 16384
 * (APX_ERR_ARG beyond).  A window holding a non-finite sample gives zero
 * outputs for its block and APX_ERR_NONFINITE from the next apx_sync.  The
 * context's filterbank workspace (about 2.3 bytes per output of one kernel in
 * FP16, half that in FP8, plus the Toeplitz columns and one float per block and
 * kernel) is reused by the next call on any stream.
 * Errors: APX_ERR_ARG, APX_ERR_RANGE, APX_ERR_OOM, APX_ERR_BUDGET, APX_ERR_CUDA. */
int apx_filterbank(apx_ctx* ctx, const float* s_in, int64_t L, const float* k_bank, int32_t F, int32_t N,
                   int32_t S_q, int32_t K_q, float* y_out, int64_t ldy, int32_t* yq_out, float* block_cs,
                   void* stream);

/* Host-only: the block geometry apx_filterbank uses for these sizes and
 * companding ranges: *T outputs per block (T = 128 P, the phases P per row as
 * above) and *nb blocks, ceil((L+N-1) / T).  Either pointer may be NULL.
 * Errors: APX_ERR_ARG (sizes beyond the limits above), APX_ERR_RANGE. */
int apx_filterbank_blocks(int64_t L, int32_t F, int32_t N, int32_t S_q, int32_t K_q, int32_t* T, int64_t* nb);

/* ---- prepared kernels (resident across calls) ----------------------------
 * Section IV prepares the kernel once per request; a caller that convolves
 * many signals with the same kernel (template matching against a stream of
 * inputs, a filter applied block after block) can prepare it once instead.
 * apx_kernel_create copies the N taps into the handle's own device memory and
 * computes there the kernel statistics, the exact packed-kernel norms and the
 * FP32 spectrum (FFT core); the FP64 packed spectra are built by the first
 * call whose blocks select each packing and kept.  Everything stays resident
 * until apx_kernel_destroy (the handle's memory is its own, outside the
 * context budget; the caller's tap buffer may be reused once `stream` has
 * passed the creation).
 *   mode : op | APX_CORE_FFT | APX_PACK_AUTO or APX_PACK_NONE
 * apx_conv_prepared then runs one call: the same as apx_conv (APX_PACK_AUTO,
 * per-block selection under snr_target_db) or apx_conv_full (APX_PACK_NONE)
 * with this kernel, as one launch of the block kernel, with the same results
 * bit for bit.  Calls with one handle on different streams may overlap (the
 * on-demand spectra are built once either way); the handle must outlive them.
 * Errors: APX_ERR_ARG (other cores or packings), as apx_conv otherwise. */
typedef struct apx_kernel apx_kernel;
int apx_kernel_create(apx_ctx* ctx, const float* k, int32_t N, int32_t W_block, uint32_t mode, void* stream,
                      apx_kernel** out);
int apx_conv_prepared(apx_ctx* ctx, const apx_kernel* kp, const float* s_in, int64_t L, double snr_target_db,
                      float* r_out, int32_t* rq_out, apx_block_stats* stats, void* stream);
void apx_kernel_destroy(apx_kernel* kp);

/* ---- serving engine (persistent kernel) ------------------------------------
 * Section IV.D adapts each block to a per-block SNR minimum; a server that
 * receives such requests continuously keeps one persistent kernel on the GPU
 * instead of launching per request.  Requests are appended to a queue in
 * page-locked, device-mapped memory; the kernel's CTAs claim their work items
 * (a template's preparation jobs, then the request's overlap-save blocks) in
 * order and signal each request's completion through a host-mapped word.
 * Templates (kernel buffer, N, W_block, op and packing bits) stay resident:
 * the first request with a template prepares its statistics and spectra, and
 * later requests with the same template only run their blocks, until the
 * template's entry is taken for another one (least recently used first).
 *
 * apx_server_create: slots = requests in flight at most, templates = resident
 * entries (about 300 KB of device memory each, outside the context budget),
 * ctas = persistent CTAs (0: two per SM), idle_ms = how long a CTA waits for
 * work before it leaves (the next submit relaunches the kernel).  The context
 * provides the device and must outlive the server; the server runs on a
 * stream of its own.  Errors: APX_ERR_ARG, APX_ERR_OOM, APX_ERR_CUDA.
 *
 * apx_server_submit: one request (apx_request; FFT core or APX_CORE_AUTO,
 * APX_PACK_AUTO or APX_PACK_NONE, W_block <= 8192 or 0 for the default;
 * rq_out and stats NULL).  s_in, k and r_out are device pointers or
 * page-locked host buffers (read and written in place); the kernel buffer is
 * the template's identity, so its contents must not change while it is
 * resident.  Writes the request's sequence number (never 0).  Errors:
 * APX_ERR_ARG, APX_ERR_WBLOCK, APX_ERR_BUDGET (every slot or template entry is
 * in use: poll and retry), APX_ERR_CUDA.
 *
 * apx_server_poll: 1 when request seq is complete (its outputs are then
 * visible to the host; *status receives APX_OK, APX_ERR_NONFINITE, or
 * APX_ERR_TIMEOUT when a block gave up waiting for its template's preparation,
 * its outputs NaN), 0 while it is in flight; a request is reported complete
 * once.  Errors: APX_ERR_ARG (unknown sequence number), APX_ERR_CUDA.
 *
 * apx_server_destroy: asks the CTAs to leave, waits for the kernel, frees the
 * server (requests still in flight complete first).  NULL is a no-op.
 *
 * apx_server_test_stall_next (no counterpart in the paper; a failure-path
 * test hook): the next submitted request prepares its template afresh but
 * drops the preparation jobs, so each of its blocks waits in its bounded spin,
 * gives up after about a second and writes NaN; the request completes with
 * APX_ERR_TIMEOUT and the template is prepared anew by the next request.
 * Nothing faults or hangs.  apx_server_launch_count: persistent-kernel
 * launches so far. */
typedef struct apx_server apx_server;
int apx_server_create(apx_ctx* ctx, int32_t slots, int32_t templates, int32_t ctas, double idle_ms,
                      apx_server** out);
int apx_server_submit(apx_server* srv, const apx_request* req, int64_t* seq);
int apx_server_poll(apx_server* srv, int64_t seq, int32_t* status);
void apx_server_destroy(apx_server* srv);
int apx_server_test_stall_next(apx_server* srv);
int64_t apx_server_launch_count(const apx_server* srv);

/* ---- allocation-free FFT core ---------------------------------------------
 * The paper has no counterpart: this is a deployment variant of apx_conv with
 * the FFT core for callers that may not allocate device memory once they are
 * running -- a real-time audio callback, a plug-in inside a host application
 * whose allocator owns the GPU, code that runs while another library holds the
 * device's memory pool.  It takes no context and calls no cudaMalloc, cudaFree
 * or other allocating routine: all of its scratch (twiddle tables, kernel
 * spectra, kernel statistics, claim, ready and ticket words) lives in one fixed device array of
 * about 550 KB that every GPU loading the library keeps until the process
 * exits.
 *   s_in, k, r_out : device pointers as for apx_conv (L, N and L+N-1 floats)
 *   mode           : op | APX_CORE_FFT | pack bits (APX_PACK_AUTO uses
 *                    snr_target_db); the direct core is rejected (APX_ERR_ARG)
 *   W_block        : a power of two up to 8192; larger -> APX_ERR_WBLOCK
 * Results equal apx_conv's for the same arguments: the same per-block
 * decisions, and outputs of packed blocks bit for bit (the same integers
 * times the same FP32 factor); outputs of full-precision blocks within FP32
 * rounding (this entry point builds its twiddle tables on the device with
 * sincospi, apx_conv on the host in long double, and the two can differ in the
 * last bit).  Non-finite input yields NaN outputs for the affected blocks;
 * there is no status word to read back (the array's status bits are set as in
 * apx_conv but nothing reads or clears them, which affects no later call).
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress); the first call on a device also clears the array's
 * flag words and fills its twiddle tables (once, for every W_block up to the
 * maximum), enqueued on `stream`: make that first call before any stream
 * capture.  A device reset (cudaDeviceReset) while the process runs is not
 * supported by this entry point.  Every call shares the array and leaves its
 * contents for the next: calls that overlap on the GPU (different streams, or
 * several host threads) race and must be serialised by the caller.
 * Errors: APX_ERR_ARG (null pointer, not the FFT core, mode bits the FFT core
 * rejects such as APX_FULL_FP64 or APX_LITERAL), APX_ERR_WBLOCK, APX_ERR_RANGE,
 * APX_ERR_CUDA. */
int apx_conv_fft_static(const float* s_in, int64_t L, const float* k, int32_t N, int32_t W_block, uint32_t mode,
                        double snr_target_db, float* r_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
