// apx_api.cu -- host side of libapx: the C ABI declared in include/apx.h.
//
// Per call: validate, plan the blocks (Section III, Eq. 17), choose the packing
// candidates (largest S_q = K_q for which the FP64 packed convolution stays
// exact; Section IV.D), then enqueue the kernel preparation and the block kernels
// on the caller's stream.  Nothing here touches sample data on the host.
#include <nvtx3/nvToolsExt.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "apx_launch.h"
#include "apx_serve.h"
#include "apx_tc.h"

using namespace apx;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

// status, claim[3], ready[3], (pad), ticket counter (64-bit, words 8-9), job ready[kMaxJobs]
constexpr int kMaxJobs = 40;
constexpr int kFlagWords = 10 + kMaxJobs;
// A single FFT-core call runs the kernel preparation inside the block kernel
// when it has at least this many blocks (fewer CTAs would take the jobs one
// after another); below, the two preparation launches run ahead of it.
constexpr long long kFuseMinBlocks = 64;
static_assert(kFlagWords * sizeof(unsigned) <= 512, "the static scratch holds 512 bytes of flag words");

// Flag-word pointers of a call (ctx->flags or the static scratch).
void set_flag_ptrs(Params& p, unsigned* flags) {
    p.status = flags;
    p.claim = flags + 1;
    p.ready = flags + 1 + kMaxCand;
    p.ticket = reinterpret_cast<unsigned long long*>(flags + 8);
    p.jobready = flags + 10;
}
// Not while the stream is being captured into a graph: the launch's ticket
// base is fixed at capture, so replays would find the counter moved on.
bool use_fused(const Params& p, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    // A call that needs full precision only runs the two-CTA block kernel, whose
    // launch follows the two preparation launches as their programmatic
    // dependent (measured faster than the one-launch form with the one-CTA kernel).
    if (fft_full_only(p)) return false;
    return cs == cudaStreamCaptureStatusNone && p.fft && p.P >= kFuseMinBlocks &&
           prep_jobs_count(p.Wb, fft_threads(p.Wb)) <= kMaxJobs;
}

struct apx_ctx {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;
    int64_t launches = 0;
    DevBuf flags, ki, Hfull, Ysub, Hpair, Hc[kMaxCand], tw64, tw32, hs, hk, hr;
    DevBuf barena, bparams, btab;       // batched calls: per-request workspace, parameters, CTA tables
    DevBuf tc_seg, tc_b, tc_cs, tc_inv;  // filterbank: block segments, Toeplitz B, c_s per block, 1/(c_s c_k) per block and kernel
    DevBuf bhost;                       // batched calls from host buffers: device copies of inputs and outputs
    cudaStream_t hp_in = nullptr;       // calls from host buffers: the signal's copy stream
    std::vector<cudaEvent_t> hp_ev;     // and its events
    void* hstage = nullptr;             // pinned staging for batch parameters
    size_t hstage_bytes = 0;
    cudaEvent_t stage_ev = nullptr;     // last upload from hstage
    int tw_wb = 0;          // W_block the twiddle tables were built for
    const void* res_ptr = nullptr;  // the pointer device_resident last classified
    bool res_dev = false;
    unsigned epoch = 0;     // FFT-core call number (claims of on-demand spectra)
    unsigned long long tickets = 0;  // CTA tickets handed out by fused launches (the device counter's value)
    int stall_next = 0;     // test hook: pre-claim the next call's packed spectra
    std::vector<void*> retired;       // device buffers replaced by larger ones (freed with the context)
    std::vector<void*> retired_host;  // page-locked staging buffers replaced likewise
    // tracing
    bool profiling = false;
    std::vector<cudaEvent_t> ev;          // event pool, pairs
    std::vector<int> ev_phase;            // phase of each recorded pair
    size_t ev_used = 0;                   // pairs recorded since the last read
};

namespace {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return APX_OK;
    return e == cudaErrorMemoryAllocation ? APX_ERR_OOM : APX_ERR_CUDA;
}

// Grow a workspace buffer to at least `bytes` (256-byte aligned by cudaMalloc).
// The buffer it replaces is retired, not freed: cudaFree waits for the whole
// device, which would stall this host thread behind every kernel in flight (a
// running serving kernel among them); retired buffers are freed with the
// context.
int ensure(apx_ctx* c, DevBuf& b, size_t bytes) {
    if (b.bytes >= bytes) return APX_OK;
    size_t want = bytes < 256 ? 256 : bytes;
    if (c->in_use - b.bytes + want > c->budget) return APX_ERR_BUDGET;
    if (b.p) {
        c->retired.push_back(b.p);
        c->in_use -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) { b.p = nullptr; return cuda_status(e); }
    b.bytes = want;
    c->in_use += want;
    return APX_OK;
}

void release(apx_ctx* c, DevBuf& b) {
    if (b.p) cudaFree(b.p);
    c->in_use -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

// ------------------------------------------------------------------ host arithmetic of the selector
// eps = 2^-b, smallest b with 2^b >= 2 R_max + 1 (the paper's eps = (2 R_max)^-1,
// Eq. 6, rounded to a power of two so that every packed value is an exact multiple
// of the finest digit).
int bits_for(long long Rmax) {
    int b = 0;
    while (b < 62 && (1ll << b) < 2 * Rmax + 1) ++b;
    return b;
}

typedef unsigned __int128 u128;

// Exactness of the FP64 packed convolution with eps = 2^-b: every packed word,
// product and partial sum, scaled by the finest digit, stays <= 2^53 (this
// replaces Table 1's companding-range row for a power-of-two eps).
bool exact_ok(int blk, int Nodd, int S, int K) {
    if (Nodd < 1 || S < 1 || K < 1) return false;
    if (blk == APX_BLK_TC)  // FP16 operands (every integer up to 2048), FP32 sums of integers up to 2^24
        return S <= kTcbQMax && K <= kTcbQMax && (long long)Nodd * S * K <= kTcbSumMax;
    u128 SK = (u128)(unsigned)S * (unsigned)K;
    u128 R = SK * (unsigned)Nodd;
    const u128 lim = (u128)1 << 53;
    if (R >= lim) return false;
    int b = bits_for((long long)R);
    if (blk == APX_BLK_SYM) {
        if (2 * b > 100) return false;
        u128 A = (u128)((Nodd + 1) / 2) * SK, C = (u128)((Nodd - 1) / 2) * SK;
        return (A << (2 * b)) + (R << b) + C <= lim;
    }
    int M = blk == APX_BLK_ASYM2 ? 2 : 3;
    if (b * (M - 1) > 100) return false;
    u128 gsum = 0;
    for (int q = 0; q < M; ++q) gsum += (u128)1 << (b * q);
    return R * gsum <= lim;
}

// Largest Q = S_q = K_q in [1, 2^20] within the exactness bound, 0 if none.
int qmax_direct(int blk, int Nodd) {
    if (!exact_ok(blk, Nodd, 1, 1)) return 0;
    int lo = 1, hi = 1 << 20;
    if (exact_ok(blk, Nodd, hi, hi)) return hi;
    while (hi - lo > 1) {
        int mid = lo + (hi - lo) / 2;
        if (exact_ok(blk, Nodd, mid, mid)) lo = mid; else hi = mid;
    }
    return lo;
}

// FFT-core error bound constant (the FFT round-off must stay below a quarter of
// the finest digit so that rounding recovers the digits): (3 phi + 16 u) with phi = Lg eta / (1 - Lg eta), eta = mu + gamma_4 (sqrt 2 + mu),
// mu = 4u, Lg = log2(n) + 2 (Higham, Thm 24.2, for radix-2 structured FFTs).
double fft_const(int log2n) {
    const double u = ldexp(1.0, -53);
    double mu = 4.0 * u;
    double g4 = (4.0 * u) / (1.0 - 4.0 * u);
    double eta = mu + g4 * (sqrt(2.0) + mu);
    double Lg = (double)(log2n + 2);
    double phi = (Lg * eta) / (1.0 - Lg * eta);
    return 3.0 * phi + 16.0 * u;
}

int digit_shift(int blk, int b) { return blk == APX_BLK_ASYM3 ? 2 * b : b; }

int ilog2i(long long n) { int l = 0; while ((1ll << l) < n) ++l; return l; }

int fft_log2n(int blk, int Wb) { return blk == APX_BLK_SYM ? ilog2i(Wb / 2) : ilog2i(Wb); }

// FFT core guide: largest Q <= qmax_direct whose a-priori bound (crest factor 3
// for block and kernel) stays below 1/4 digit.  Every block is checked again
// with its exact norm on the device.
int qmax_fft(int blk, int Nodd, int Wb) {
    int qd = qmax_direct(blk, Nodd);
    int lg = fft_log2n(blk, Wb);
    double C = fft_const(lg);
    for (int Q = qd; Q >= 1; --Q) {
        long long Rmax = (long long)Nodd * Q * Q;
        int b = bits_for(Rmax);
        double taps = blk == APX_BLK_SYM ? (double)((Nodd + 1) / 2) : (double)Nodd;
        double kscale = blk == APX_BLK_SYM ? ldexp(1.0, b) + 1.0 : 1.0;
        double l1 = taps * (double)Q / 3.0 * kscale;
        double l2 = sqrt((double)Wb) * (double)Q / 3.0;
        double E = C * l1 * l2;
        if (ldexp(E, digit_shift(blk, b)) < 0.25) return Q;
    }
    return 0;
}

Cand make_cand(int blk, int S, int K, int Nodd, int Wb) {
    Cand c;
    memset(&c, 0, sizeof c);
    c.blk = blk;
    c.M = blk == APX_BLK_SYM ? 1 : (blk == APX_BLK_ASYM2 ? 2 : 3);
    c.S = S; c.K = K;
    c.Rmax = (long long)Nodd * S * K;
    c.b = bits_for(c.Rmax);
    c.sc = digit_shift(blk, c.b);
    c.nk = blk == APX_BLK_SYM ? (Nodd + 1) / 2 : Nodd;
    c.log2n = fft_log2n(blk, Wb);
    c.fftc = fft_const(c.log2n);
    return c;
}

struct Plan {
    int Nodd, W, head, fft;
    long long P;
};

int plan(int64_t L, int32_t N, int32_t Wb, uint32_t mode, Plan* p) {
    if (L < 1 || N < 1) return APX_ERR_ARG;
    const uint32_t core = mode & 0xF0u;
    if ((mode & 0xFu) > APX_OP_XCORR || (core != APX_CORE_DIRECT && core != APX_CORE_FFT && core != APX_CORE_TC) ||
        ((mode >> 8) & 0xFu) > 4u ||
        (mode & ~(0xFFFu | APX_FULL_FP64 | APX_LITERAL)))
        return APX_ERR_ARG;
    if ((mode & APX_FULL_FP64) && ((mode & 0xF00u) != APX_PACK_NONE || (mode & 0xF0u) != APX_CORE_DIRECT))
        return APX_ERR_ARG;
    if ((mode & APX_LITERAL) && ((mode & 0xF00u) != APX_PACK_SYM || (mode & 0xF0u) != APX_CORE_DIRECT))
        return APX_ERR_ARG;
    int fft = (mode & 0xF0u) == APX_CORE_FFT;
    int Nodd = (N % 2) ? N : N + 1;
    if (Wb < 4 || (Wb % 2) || Wb > kMaxWblock) return APX_ERR_WBLOCK;
    int W = Wb - Nodd - 1;
    if (W < 2) return APX_ERR_WBLOCK;
    if (fft && (Wb & (Wb - 1))) return APX_ERR_WBLOCK;
    if (core == APX_CORE_TC) {  // the tensor-core block: 64-sample rows, at most one 128-row MMA tile
        if (Wb % kTcbRow || Wb > 128 * kTcbRow) return APX_ERR_WBLOCK;
        if (tcb_kslices(Nodd) > kTcbMaxSlices) return APX_ERR_ARG;
        const uint32_t pack = mode & 0xF00u;
        if (pack != APX_PACK_AUTO && pack != APX_PACK_NONE) return APX_ERR_ARG;
    }
    long long span = L + N - Nodd;
    long long P = (span + W - 1) / W;
    if (P < 1) P = 1;
    p->Nodd = Nodd; p->W = W; p->fft = fft;
    p->head = fft ? (Nodd - 1 + W - 1) / W : 0;
    p->P = P + p->head;
    if (p->P > 0x7fffffffll) return APX_ERR_ARG;
    return APX_OK;
}

int round_up(int a, int m) { return (a + m - 1) / m * m; }

// Direct core shared-memory layout for the candidate set.  Full precision:
// the FP32 window behind a zero pad of N' samples, then one chunk of FP32
// taps.  Packed blocks: the packed signal in a region of its own; the packed
// outputs and one chunk of packed taps overlay the FP32 window (packing is the
// last step to read it).  Taps are staged a chunk at a time (kDirectTapChunk*),
// so every packing fits one CTA up to the largest W_block at any kernel length.
size_t direct_layout(const Cand* c, int nc, int Wb, int Nodd, DirectLayout* dl, bool full64 = false) {
    auto al16 = [](size_t b) { return (b + 15) / 16 * 16; };
    dl->padF = round_up(Nodd, 8);
    dl->offK = (int)al16((size_t)4 * (dl->padF + Wb + 8));
    const int kcf = round_up(Nodd, 8) < kDirectTapChunkF ? round_up(Nodd, 8) : kDirectTapChunkF;
    const size_t full_end = (size_t)dl->offK + (size_t)4 * kcf;
    if (nc == 1 && c[0].blk == APX_BLK_TC) {
        // the tensor-core candidate (tc_block): 1024 bytes of alignment slack, the
        // segment of 128 + slices - 1 rows of 128 bytes (rounded up to 1024), the
        // tap slices of 64 rows of 128 bytes; the FP32 window and tap chunk stay
        // in front for the blocks that run full precision
        const int ns = tcb_kslices(Nodd);
        dl->padS = tcb_kshift(Nodd);
        dl->nS = ns;
        dl->offS = (int)al16(full_end);
        dl->offT = dl->offKb = 0;
        return (size_t)dl->offS + 1024 + (size_t)round_up((128 + ns - 1) * 128, 1024) + (size_t)ns * 8192;
    }
    if (full64) {  // the window and every tap as FP64, behind the FP32 region
        const int nkb = round_up(Nodd, 4);
        dl->offS = (int)al16(full_end);
        dl->padS = nkb;
        dl->nS = nkb + Wb + 4;
        dl->offT = (int)al16((size_t)dl->offS + (size_t)8 * dl->nS);
        dl->offKb = dl->offT;
        return (size_t)dl->offKb + (size_t)8 * nkb;
    }
    int body = 0, nT = 0, kcd = 0;
    for (int i = 0; i < nc; ++i) {
        const int nkp = round_up(c[i].nk, 4);
        const int kc = nkp < kDirectTapChunkD ? nkp : kDirectTapChunkD;
        if (kc > kcd) kcd = kc;
        if (c[i].blk == APX_BLK_SYM) {
            body = body > Wb / 2 ? body : Wb / 2;
            nT = nT > Wb / 2 ? nT : Wb / 2;
        } else {
            const int Ls = (Wb + c[i].M - 1) / c[i].M;
            body = body > Ls ? body : Ls;
            const int t = Ls + Nodd - 1 < Wb ? Ls + Nodd - 1 : Wb;
            nT = nT > t ? nT : t;
        }
    }
    dl->padS = 0;
    dl->nS = body;
    dl->offT = 0;
    dl->offKb = (int)al16((size_t)8 * nT);
    const size_t over = (size_t)dl->offKb + (size_t)8 * kcd;
    dl->offS = (int)al16(full_end > over ? full_end : over);
    return nc ? (size_t)dl->offS + (size_t)8 * body : full_end;
}

// exp(-2 pi i t / Wb), t in [0, Wb), from long double arithmetic.  One table
// for the largest W_block seen; smaller transforms index it with a stride.
int ensure_twiddles(apx_ctx* c, int Wb, cudaStream_t st) {
    if (c->tw_wb >= Wb) return APX_OK;
    int rc = ensure(c, c->tw64, sizeof(double2) * Wb);
    if (!rc) rc = ensure(c, c->tw32, sizeof(float2) * Wb);
    if (rc) return rc;
    std::vector<double2> t64(Wb);
    std::vector<float2> t32(Wb);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int t = 0; t < Wb; ++t) {
        long double a = two_pi * (long double)t / (long double)Wb;
        t64[t].x = (double)cosl(a);
        t64[t].y = (double)-sinl(a);
        t32[t].x = (float)t64[t].x;
        t32[t].y = (float)t64[t].y;
    }
    cudaError_t e = cudaMemcpyAsync(c->tw64.p, t64.data(), sizeof(double2) * Wb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->tw32.p, t32.data(), sizeof(float2) * Wb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    c->tw_wb = Wb;
    return APX_OK;
}

// Record an event pair around one launch when profiling is on.
// Host-side NVTX range (visible to Nsight tools when one is attached; a few
// nanoseconds otherwise).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

const char* const kPhaseName[APX_NPHASES] = {"apx.direct", "apx.spectra", "apx.fft", "apx.tc_prep", "apx.tc_mma"};

// One phase: an NVTX range and, while profiling is on, a pair of CUDA events on
// the launching stream.
struct Trace {
    apx_ctx* c;
    cudaStream_t st;
    size_t pair = (size_t)-1;
    Range range;
    Trace(apx_ctx* c_, cudaStream_t st_, int phase) : c(c_), st(st_), range(kPhaseName[phase]) {
        if (!c->profiling) return;
        if (2 * (c->ev_used + 1) > c->ev.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess) return;
            if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
            c->ev.push_back(a);
            c->ev.push_back(b);
            c->ev_phase.push_back(phase);
        }
        pair = c->ev_used++;
        c->ev_phase[pair] = phase;
        cudaEventRecord(c->ev[2 * pair], st);
    }
    ~Trace() {
        if (pair != (size_t)-1) cudaEventRecord(c->ev[2 * pair + 1], st);
    }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Every device pointer a launch dereferences must be set before it launches.
bool device_pointers_set(const Params& p) {
    if (!p.s || !p.k || !p.r || !p.status) return false;
    if (!p.fft) return true;
    if (!p.Hfull || !p.Ysub || !p.ki || !p.tw64 || !p.tw32 || !p.claim || !p.ready) return false;
    for (int j = 0; j < p.ncand; ++j)
        if (!p.cand[j].H) return false;
    return true;
}

// Section IV.D asks for at least the target SNR in every block, while the
// Table 1 model gives the SNR a block can expect; a block's measured SNR
// scatters around the model, the more so the fewer outputs W it keeps.  A
// packing is admitted only when the model clears the target by
// 0.5 + 48 / sqrt(W) dB (the model's overestimate over many blocks of
// Gaussian, Laplacian and uniform data stays below this: 1.6 dB at W = 958,
// 6.2 dB at W = 56), so the measured SNR of every packed block is at least
// the target.
double snr_margin_db(int W) { return 0.5 + 48.0 / sqrt((double)W); }
double target_thr(double snr_db, int W) { return pow(10.0, (snr_db + snr_margin_db(W)) / 10.0); }

// Table 1 model check on the host (the device's inequality, without its
// operation-by-operation rounding; callers leave a margin).
bool snr_feasible_host(double s2s, double Ms, double s2k, double Mk, int S, int K, double thr) {
    const double S2 = (double)S * S, K2 = (double)K * K, Ms2 = Ms * Ms, Mk2 = Mk * Mk;
    const double num = 144.0 * (s2s * s2k) * (S2 * K2);
    const double den = 12.0 * (s2s * S2 * Mk2 + s2k * K2 * Ms2) + Ms2 * Mk2;
    return num >= thr * den;
}

// The model grows with sigma_s^2 / ||s||_inf^2 and sigma_k^2 / ||k||_inf^2,
// both at most 1: a candidate below the target there (checked 1 % below it,
// far beyond the device's rounding) fails every block's check for every
// kernel.  Such candidates are left out (the others keep their order), so the
// block kernel holds no buffers for them; the same decisions, bit for bit.
int prune_unreachable(Cand* c, int nc, double thr) {
    int m = 0;
    for (int j = 0; j < nc; ++j)
        if (snr_feasible_host(1.0, 1.0, 1.0, 1.0, c[j].S, c[j].K, thr * 0.99)) c[m++] = c[j];
    return m;
}

// Host half of a call: validate, plan (Section III, Eq. 17), choose the
// packing candidates and the block kernel's shared memory.  Pointers to the
// workspace are filled in by the caller.
int make_params(const float* s, int64_t L, const float* k, int32_t N, int32_t Wb, uint32_t mode,
                int sel_kind /*0 auto, 1 fixed, 2 none*/, double snr_db, int S, int K, float* r, int32_t* rq,
                apx_block_stats* st, Params* out, size_t* smem_out, bool prune = true) {
    if (!s || !k || !r) return APX_ERR_ARG;
    Plan pl;
    int rc = plan(L, N, Wb, mode, &pl);
    if (rc) return rc;
    const uint32_t pack = mode & 0xF00u;
    if (sel_kind == 0 && pack == APX_PACK_NONE) sel_kind = 2;
    if (sel_kind == 1 && (pack == APX_PACK_AUTO || pack == APX_PACK_NONE)) return APX_ERR_ARG;
    if (sel_kind == 0 && pack != APX_PACK_AUTO) {
        // forced packing, largest S_q = K_q its exactness bound admits
        int blk = pack == APX_PACK_SYM ? APX_BLK_SYM : (pack == APX_PACK_ASYM2 ? APX_BLK_ASYM2 : APX_BLK_ASYM3);
        int Q = pl.fft ? qmax_fft(blk, pl.Nodd, Wb) : qmax_direct(blk, pl.Nodd);
        if (Q < 1) return APX_ERR_RANGE;
        S = K = Q;
        sel_kind = 1;
    }
    Params& p = *out;
    memset(&p, 0, sizeof p);
    p.s = s; p.L = L; p.k = k; p.N = N; p.Nodd = pl.Nodd; p.Wb = Wb; p.W = pl.W; p.head = pl.head; p.fft = pl.fft;
    p.xcorr = (mode & 0xFu) == APX_OP_XCORR;
    p.P = pl.P; p.out_len = L + N - 1;
    p.r = r; p.rq = rq; p.st = st;
    p.autosel = sel_kind == 0;
    p.full64 = (mode & APX_FULL_FP64) ? 1 : 0;
    p.thr = target_thr(snr_db, pl.W);  // Section IV.D minimum with the model margin
    int nc = 0;
    if (sel_kind == 0 && (mode & 0xF0u) == APX_CORE_TC) {
        // the tensor-core candidate at the largest S_q = K_q its bound admits
        const int Q = qmax_direct(APX_BLK_TC, pl.Nodd);
        if (Q >= 1) {
            Cand c = make_cand(APX_BLK_TC, Q, Q, pl.Nodd, Wb);
            c.M = 1;
            c.b = 0;  // no packing: integers, not digits
            c.sc = 0;
            p.cand[nc++] = c;
        }
        if (prune) nc = prune_unreachable(p.cand, nc, p.thr);
    } else if (sel_kind == 0) {
        const int order[3] = {APX_BLK_SYM, APX_BLK_ASYM3, APX_BLK_ASYM2};  // Table 1 ranking
        for (int j = 0; j < 3; ++j) {
            int Q = pl.fft ? qmax_fft(order[j], pl.Nodd, Wb) : qmax_direct(order[j], pl.Nodd);
            if (Q >= 1) p.cand[nc++] = make_cand(order[j], Q, Q, pl.Nodd, Wb);
        }
        if (prune) nc = prune_unreachable(p.cand, nc, p.thr);
    } else if (sel_kind == 1) {
        int blk = pack == APX_PACK_SYM ? APX_BLK_SYM : (pack == APX_PACK_ASYM2 ? APX_BLK_ASYM2 : APX_BLK_ASYM3);
        if (S < 1 || K < 1 || S > (1 << 20) || K > (1 << 20)) return APX_ERR_ARG;
        const bool literal = (mode & APX_LITERAL) != 0;
        if (literal ? (long long)pl.Nodd * S * K > (1LL << 31) : !exact_ok(blk, pl.Nodd, S, K)) return APX_ERR_RANGE;
        Cand c = make_cand(blk, S, K, pl.Nodd, Wb);
        if (literal) {  // Eq. (6) as printed
            c.literal = 1;
            c.eps_l = 1.0 / (2.0 * (double)c.Rmax);
        }
        p.cand[nc++] = c;
    }

    // Shared memory of the block kernel for this candidate set.
    size_t smem = 0;
    if (!pl.fft) {
        smem = direct_layout(p.cand, nc, Wb, pl.Nodd, &p.dl, p.full64 != 0);
        while (smem > (size_t)kMaxSmem && nc > 0 && sel_kind == 0) {
            // drop the widest asymmetric candidate that does not fit
            int drop = -1;
            for (int j = 0; j < nc; ++j) if (p.cand[j].blk != APX_BLK_SYM) drop = j;
            if (drop < 0) drop = nc - 1;
            for (int j = drop; j + 1 < nc; ++j) p.cand[j] = p.cand[j + 1];
            --nc;
            smem = direct_layout(p.cand, nc, Wb, pl.Nodd, &p.dl, p.full64 != 0);
        }
        if (smem > (size_t)kMaxSmem) return APX_ERR_WBLOCK;
    }
    p.ncand = nc;
    if (pl.fft) smem = fft_smem_bytes(p);
    *smem_out = smem;
    return APX_OK;
}

// A call from host buffers: the signal's host-to-device copy runs on a copy
// stream while the caller's stream copies the kernel and (three-launch FFT
// core) prepares its spectrum; the block kernel then waits for the signal copy
// (a one-launch call waits before its first CTA).
cudaError_t copy_stream_begin(apx_ctx* ctx, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (!ctx->hp_in) e = cudaStreamCreateWithFlags(&ctx->hp_in, cudaStreamNonBlocking);
    while (e == cudaSuccess && ctx->hp_ev.size() < 2) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) ctx->hp_ev.push_back(ev);
    }
    // the device buffers may still be read by earlier work on the caller's stream
    if (e == cudaSuccess) e = cudaEventRecord(ctx->hp_ev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->hp_in, ctx->hp_ev[0], 0);
    return e;
}

// Shared body of apx_conv / apx_conv_fixed / apx_conv_full.
// Whether p is device memory of the context's device (the last answer is kept
// per pointer: the query costs host time on every call).
bool device_resident(apx_ctx* ctx, const void* ptr) {
    if (ptr == ctx->res_ptr) return ctx->res_dev;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    ctx->res_ptr = ptr;
    ctx->res_dev = a.type == cudaMemoryTypeDevice && a.device == ctx->device;
    return ctx->res_dev;
}

int run(apx_ctx* ctx, const float* s, int64_t L, const float* k, int32_t N, int32_t Wb, uint32_t mode,
        int sel_kind /*0 auto, 1 fixed, 2 none*/, double snr_db, int S, int K, float* r, int32_t* rq,
        apx_block_stats* st, cudaStream_t stream, cudaEvent_t before_blocks = nullptr) {
    if (!ctx) return APX_ERR_ARG;
    Range range(sel_kind == 2 ? "apx_conv_full" : (sel_kind == 1 ? "apx_conv_fixed" : "apx_conv"));
    Params p;
    size_t smem = 0;
    int rc = make_params(s, L, k, N, Wb, mode, sel_kind, snr_db, S, K, r, rq, st, &p, &smem);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    const int nc = p.ncand;
    struct { int fft; } pl = {p.fft};

    // Workspace: status word, per-candidate claim and ready words, spectra, twiddles.
    rc = ensure(ctx, ctx->flags, kFlagWords * sizeof(unsigned));
    if (!rc && pl.fft) {
        const size_t m1 = (size_t)Wb / 2 + 1;
        rc = ensure(ctx, ctx->Hfull, sizeof(float2) * m1);
        if (!rc) rc = ensure(ctx, ctx->ki, sizeof(KInfo));
        if (!rc) rc = ensure(ctx, ctx->Ysub, sizeof(float2) * (size_t)Wb);
        for (int j = 0; j < nc && !rc; ++j) rc = ensure(ctx, ctx->Hc[j], sizeof(double2) * m1);
        if (!rc) rc = ensure_twiddles(ctx, Wb, stream);
    }
    if (rc) return rc;

    for (int j = 0; j < nc; ++j) p.cand[j].H = (double2*)ctx->Hc[j].p;
    set_flag_ptrs(p, (unsigned*)ctx->flags.p);
    p.fused = use_fused(p, stream);
    // the spectrum launch prefetches a device-resident signal into L2 (not one
    // still being copied in: its copy is waited for only before the blocks)
    p.pf = pl.fft && !p.fused && !before_blocks && device_resident(ctx, s);
    if (pl.fft && !p.fused && fft_full_only(p)) {  // the two-CTA block kernel: its staging-order spectrum
        rc = ensure(ctx, ctx->Hpair, pair_table_bytes(Wb));
        if (rc) return rc;
        p.Hpair = (float2*)ctx->Hpair.p;
    }
    p.ticket_base = ctx->tickets;
    p.Hfull = (float2*)ctx->Hfull.p;
    p.ki = (KInfo*)ctx->ki.p;
    p.Ysub = (float2*)ctx->Ysub.p;
    p.tw64 = (const double2*)ctx->tw64.p;
    p.tw32 = (const float2*)ctx->tw32.p;
    p.ntab = ctx->tw_wb;
    if (!device_pointers_set(p)) return APX_ERR_CUDA;

    cudaError_t e;
    if (!pl.fft) {
        Trace t(ctx, stream, APX_PHASE_DIRECT);
        e = before_blocks ? cudaStreamWaitEvent(stream, before_blocks, 0) : cudaSuccess;
        if (e == cudaSuccess) e = launch_direct(p, smem, stream);
        ctx->launches += 1;
    } else {
        if (++ctx->epoch == 0) ctx->epoch = 1;  // 0 marks "never"
        p.epoch = ctx->epoch;
        if (ctx->stall_next) {  // claimed by no one who will build them: blocks that pick a packing time out
            ctx->stall_next = 0;
            if (p.fused) {
                const unsigned ep[kMaxCand] = {p.epoch, p.epoch, p.epoch};
                cudaError_t e0 = cudaMemcpyAsync(p.claim, ep, sizeof ep, cudaMemcpyHostToDevice, stream);
                if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(stream);  // the host array goes out of scope
                if (e0 != cudaSuccess) return cuda_status(e0);
            } else {
                p.claim_init = p.epoch;  // the spectrum launch claims them
            }
        }
        e = cudaSuccess;
        if (!p.fused) {
            Trace t(ctx, stream, APX_PHASE_SPECTRA);
            e = launch_spec(p, stream);
            if (e == cudaSuccess) e = launch_spec_combine(p, stream);
            ctx->launches += 2;
        }
        if (e == cudaSuccess) {
            Trace t(ctx, stream, APX_PHASE_FFT);
            if (before_blocks) e = cudaStreamWaitEvent(stream, before_blocks, 0);
            if (e == cudaSuccess) e = p.fused ? launch_fft_fused(p, smem, stream) : launch_fft(p, smem, stream);
            if (e == cudaSuccess && p.fused) ctx->tickets += fused_grid(p);
            ctx->launches += 1;
        }
    }
    return cuda_status(e);
}


// ------------------------------------------------------------------ batched calls
// Library defaults when a request leaves the core or W_block open (the
// autotuner in tune.py measures and passes explicit choices): the FFT core
// above 64 taps, W_block the power of two at or above 4 N' (at least 1024).
int default_core_fft(int Nodd) { return Nodd > 64; }
int default_wblock(int Nodd) {
    int w = 1024;
    while (w < 4 * Nodd && w < kMaxWblock) w <<= 1;
    while (w - Nodd - 1 < 2 && w < kMaxWblock) w <<= 1;
    return w;
}

struct BatchPlan {
    std::vector<Params> prm;
    std::vector<size_t> smem;
    struct Group {
        int fft, Wb;
        int packed;  // whether its requests keep packing candidates (their buffers set the shared memory)
        int tc;      // tensor-core candidate (a kernel instantiation of its own)
        std::vector<int> reqs;
        size_t smem = 0;
        std::vector<int> start_blk, start_spec, start_comb;  // CTA offsets, nreq + 1 each
        int off_blk = 0, off_spec = 0, off_comb = 0;         // offsets of those tables in the int table
    };
    std::vector<Group> groups;
    std::vector<size_t> arena_off;  // per request
    size_t arena_bytes = 0;
    size_t flags_bytes = 0;         // leading part of the arena: claim/ready words of every request
    int max_wb = 0;
    std::vector<int> table;         // all CTA tables
};

size_t al256b(size_t b) { return (b + 255) / 256 * 256; }

// Per-request arena: claim[3], ready[3] | KInfo | Hfull | Ysub | Hc[ncand]
size_t arena_need(const Params& p) {
    if (!p.fft) return 0;
    const size_t m1 = (size_t)p.Wb / 2 + 1;
    return al256b(sizeof(KInfo)) + al256b(sizeof(float2) * m1) + al256b(sizeof(float2) * (size_t)p.Wb) +
           (size_t)p.ncand * al256b(sizeof(double2) * m1);
}

int plan_batch(const apx_request* reqs, int n, BatchPlan* bp) {
    if (!reqs || n < 1) return APX_ERR_ARG;
    bp->prm.resize(n);
    bp->smem.resize(n);
    for (int r = 0; r < n; ++r) {
        const apx_request& q = reqs[r];
        if (q.N < 1) return APX_ERR_ARG;
        const int Nodd = (q.N % 2) ? q.N : q.N + 1;
        uint32_t mode = q.mode;
        if (mode & APX_LITERAL) return APX_ERR_ARG;  // the paper-literal form: single calls only
        uint32_t core = mode & 0xF0u;
        if (core == APX_CORE_AUTO) core = default_core_fft(Nodd) ? APX_CORE_FFT : APX_CORE_DIRECT;
        mode = (mode & ~0xF0u) | core;
        const int Wb = q.W_block > 0 ? q.W_block : default_wblock(Nodd);
        const uint32_t pack = mode & 0xF00u;
        int sel = 0;
        if (pack == APX_PACK_NONE) sel = 2;
        else if (pack != APX_PACK_AUTO && q.S_q > 0 && q.K_q > 0) sel = 1;
        int rc = make_params(q.s_in, q.L, q.k, q.N, Wb, mode, sel, q.snr_target_db, q.S_q, q.K_q, q.r_out, q.rq_out,
                             q.stats, &bp->prm[r], &bp->smem[r]);
        if (rc) return rc;
    }
    // group by core and W_block, and apart the requests without packing candidates
    // (full precision, or no candidate can reach the target): a group launches with the
    // largest shared memory of its requests, and the candidates' FP64 buffers would
    // take L1 cache from the others
    for (int r = 0; r < n; ++r) {
        const Params& p = bp->prm[r];
        const int packed = p.ncand > 0;
        const int tc = p.ncand == 1 && p.cand[0].blk == APX_BLK_TC;
        int g = -1;
        for (size_t j = 0; j < bp->groups.size(); ++j)
            if (bp->groups[j].fft == p.fft && bp->groups[j].Wb == p.Wb && bp->groups[j].packed == packed &&
                bp->groups[j].tc == tc)
                g = (int)j;
        if (g < 0) {
            bp->groups.emplace_back();
            bp->groups.back().fft = p.fft;
            bp->groups.back().Wb = p.Wb;
            bp->groups.back().packed = packed;
            bp->groups.back().tc = tc;
            g = (int)bp->groups.size() - 1;
        }
        bp->groups[g].reqs.push_back(r);
        if (bp->smem[r] > bp->groups[g].smem) bp->groups[g].smem = bp->smem[r];
        if (p.fft && p.Wb > bp->max_wb) bp->max_wb = p.Wb;
    }
    // arena: flags for every request first, then each FFT request's buffers
    bp->flags_bytes = al256b(sizeof(unsigned) * 2 * kMaxCand * (size_t)n);
    size_t off = bp->flags_bytes;
    bp->arena_off.resize(n);
    for (int r = 0; r < n; ++r) {
        bp->arena_off[r] = off;
        off += arena_need(bp->prm[r]);
    }
    bp->arena_bytes = off;
    // CTA tables
    for (auto& G : bp->groups) {
        int a = 0, b = 0, c = 0;
        G.start_blk.push_back(0);
        G.start_spec.push_back(0);
        G.start_comb.push_back(0);
        for (int r : G.reqs) {
            const Params& p = bp->prm[r];
            const long long nctas = G.tc ? tcb_ctas(p.P) : p.P;  // the tensor-core kernel takes several blocks per CTA
            if (nctas > 0x7fffffffLL - a) return APX_ERR_ARG;  // one launch's grid: fewer than 2^31 CTAs
            a += (int)nctas;
            G.start_blk.push_back(a);
            if (G.fft) {
                b += spec_ctas(p.Wb);
                c += combine_ctas(p.Wb);
            }
            G.start_spec.push_back(b);
            G.start_comb.push_back(c);
        }
        G.off_blk = (int)bp->table.size();
        bp->table.insert(bp->table.end(), G.start_blk.begin(), G.start_blk.end());
        G.off_spec = (int)bp->table.size();
        bp->table.insert(bp->table.end(), G.start_spec.begin(), G.start_spec.end());
        G.off_comb = (int)bp->table.size();
        bp->table.insert(bp->table.end(), G.start_comb.begin(), G.start_comb.end());
    }
    return APX_OK;
}

// Point every request at its workspace (arena base, twiddles, status word).
void bind_batch(BatchPlan* bp, unsigned char* arena, const double2* tw64, const float2* tw32, int ntab,
                unsigned* status, unsigned epoch) {
    const int n = (int)bp->prm.size();
    for (int r = 0; r < n; ++r) {
        Params& p = bp->prm[r];
        p.status = status;
        p.claim = reinterpret_cast<unsigned*>(arena) + 2 * kMaxCand * r;
        p.ready = p.claim + kMaxCand;
        p.epoch = epoch;
        p.tw64 = tw64;
        p.tw32 = tw32;
        p.ntab = ntab;
        if (!p.fft) continue;
        unsigned char* b = arena + bp->arena_off[r];
        const size_t m1 = (size_t)p.Wb / 2 + 1;
        p.ki = (KInfo*)b;
        b += al256b(sizeof(KInfo));
        p.Hfull = (float2*)b;
        b += al256b(sizeof(float2) * m1);
        p.Ysub = (float2*)b;
        b += al256b(sizeof(float2) * (size_t)p.Wb);
        for (int j = 0; j < p.ncand; ++j) {
            p.cand[j].H = (double2*)b;
            b += al256b(sizeof(double2) * m1);
        }
    }
}

// The launches of a planned batch, groups one after another on `st`.
cudaError_t launch_batch(const BatchPlan& bp, const Params* dprm, const int* dtab, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    size_t base = 0;  // the device parameter array holds the requests group by group
    for (const auto& G : bp.groups) {
        const int nr = (int)G.reqs.size();
        const Params* gp = dprm + base;
        const Params& any = bp.prm[G.reqs[0]];
        BatchTab tb = {gp, dtab + G.off_blk, nr};
        if (!G.fft) {
            e = launch_direct_batch(any, tb, G.start_blk[nr], G.smem, st);
        } else {
            BatchTab ts = {gp, dtab + G.off_spec, nr};
            BatchTab tc = {gp, dtab + G.off_comb, nr};
            e = launch_spec_batch(any, ts, G.start_spec[nr], st, false);
            if (e == cudaSuccess) e = launch_combine_batch(any, tc, G.start_comb[nr], st);
            if (e == cudaSuccess) e = launch_fft_batch(any, tb, G.start_blk[nr], G.smem, st);
        }
        if (e != cudaSuccess) return e;
        base += nr;
    }
    return e;
}

// Parameters in group order (the device array is indexed per group).
std::vector<Params> grouped_params(const BatchPlan& bp) {
    std::vector<Params> v;
    v.reserve(bp.prm.size());
    for (const auto& G : bp.groups)
        for (int r : G.reqs) v.push_back(bp.prm[r]);
    return v;
}

int stage_upload(apx_ctx* c, const void* src1, size_t n1, void* dst1, const void* src2, size_t n2, void* dst2,
                 cudaStream_t st) {
    const size_t need = n1 + n2;
    if (c->stage_ev) {
        cudaError_t e = cudaEventSynchronize(c->stage_ev);
        if (e != cudaSuccess) return cuda_status(e);
    } else if (cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming) != cudaSuccess) {
        return APX_ERR_CUDA;
    }
    if (c->hstage_bytes < need) {
        if (c->hstage) c->retired_host.push_back(c->hstage);  // freed with the context (cudaFreeHost waits for the device)
        c->hstage = nullptr;
        c->hstage_bytes = 0;
        if (cudaMallocHost(&c->hstage, need) != cudaSuccess) { c->hstage = nullptr; return APX_ERR_OOM; }
        c->hstage_bytes = need;
    }
    memcpy(c->hstage, src1, n1);
    memcpy((char*)c->hstage + n1, src2, n2);
    cudaError_t e = cudaMemcpyAsync(dst1, c->hstage, n1, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst2, (char*)c->hstage + n1, n2, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(c->stage_ev, st);
    return cuda_status(e);
}

}  // namespace

extern "C" {

int apx_create(apx_ctx** out, int device, size_t mem_budget_bytes) {
    if (!out) return APX_ERR_ARG;
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_status(e);
    if (device < 0 || device >= n) return APX_ERR_ARG;
    apx_ctx* c = new apx_ctx();
    c->device = device;
    c->budget = mem_budget_bytes ? mem_budget_bytes : ((size_t)4 << 30);
    DeviceGuard dg(device);
    int rc = ensure(c, c->flags, kFlagWords * sizeof(unsigned));
    if (!rc) rc = cuda_status(cudaMemset(c->flags.p, 0, kFlagWords * sizeof(unsigned)));
    if (rc) { apx_destroy(c); return rc; }
    *out = c;
    return APX_OK;
}

void apx_destroy(apx_ctx* c) {
    if (!c) return;
    {
        DeviceGuard dg(c->device);
        cudaDeviceSynchronize();
        DevBuf* all[] = {&c->flags, &c->ki, &c->Hfull, &c->Ysub, &c->Hpair, &c->Hc[0], &c->Hc[1], &c->Hc[2], &c->tw64,
                         &c->tw32, &c->hs, &c->hk, &c->hr, &c->barena, &c->bparams, &c->btab,
                         &c->tc_seg, &c->tc_b, &c->tc_cs, &c->tc_inv, &c->bhost};
        for (DevBuf* b : all) release(c, *b);
        for (void* p : c->retired) cudaFree(p);
        for (void* p : c->retired_host) cudaFreeHost(p);
        if (c->hstage) cudaFreeHost(c->hstage);
        if (c->hp_in) cudaStreamDestroy(c->hp_in);
        for (cudaEvent_t e : c->hp_ev) cudaEventDestroy(e);
        if (c->stage_ev) cudaEventDestroy(c->stage_ev);
        for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    }
    delete c;
}

int apx_plan_blocks(int64_t L, int32_t N, int32_t W_block, uint32_t mode, int64_t* P, int32_t* W) {
    Plan p;
    int rc = plan(L, N, W_block, mode, &p);
    if (rc) return rc;
    if (P) *P = p.P;
    if (W) *W = p.W;
    return APX_OK;
}

int apx_plan_candidates(int64_t L, int32_t N, int32_t W_block, uint32_t mode, double snr_target_db, int32_t* blk,
                        int32_t* q, int32_t* b) {
    // the plan of a call reads no sample: any non-null addresses do
    static float none;
    Params p;
    size_t smem = 0;
    const int sel = (mode & 0xF00u) == APX_PACK_NONE ? 2 : 0;
    int rc = make_params(&none, L, &none, N, W_block, mode, sel, snr_target_db, 0, 0, &none, nullptr, nullptr, &p,
                         &smem);
    if (rc) return rc;
    for (int j = 0; j < p.ncand; ++j) {
        if (blk) blk[j] = p.cand[j].blk;
        if (q) q[j] = p.cand[j].S;
        if (b) b[j] = p.cand[j].b;
    }
    return p.ncand;
}

int apx_conv(apx_ctx* ctx, const float* s_in, int64_t L, const float* k, int32_t N, int32_t W_block,
             uint32_t mode, double snr_target_db, float* r_out, int32_t* rq_out, apx_block_stats* stats,
             void* stream) {
    return run(ctx, s_in, L, k, N, W_block, mode, 0, snr_target_db, 0, 0, r_out, rq_out, stats,
               (cudaStream_t)stream);
}

int apx_conv_fixed(apx_ctx* ctx, const float* s_in, int64_t L, const float* k, int32_t N, int32_t W_block,
                   uint32_t mode, int32_t S_q, int32_t K_q, float* r_out, int32_t* rq_out,
                   apx_block_stats* stats, void* stream) {
    return run(ctx, s_in, L, k, N, W_block, mode, 1, 0.0, S_q, K_q, r_out, rq_out, stats, (cudaStream_t)stream);
}

int apx_conv_full(apx_ctx* ctx, const float* s_in, int64_t L, const float* k, int32_t N, int32_t W_block,
                  uint32_t mode, float* r_out, void* stream) {
    return run(ctx, s_in, L, k, N, W_block, (mode & (0xFFu | APX_FULL_FP64)) | APX_PACK_NONE, 2, 0.0, 0, 0, r_out,
               nullptr, nullptr, (cudaStream_t)stream);
}

int apx_sync(apx_ctx* ctx, void* stream) {
    if (!ctx) return APX_ERR_ARG;
    DeviceGuard dg(ctx->device);
    unsigned h = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->flags.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && h) e = cudaMemsetAsync(ctx->flags.p, 0, sizeof(unsigned), st);
    if (e == cudaSuccess && (h & 4u)) {
        // a failed check may be a ticket count out of step: take the device's
        unsigned long long t = 0;
        e = cudaMemcpyAsync(&t, (unsigned*)ctx->flags.p + 8, sizeof t, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) ctx->tickets = t;
    }
    if (e == cudaSuccess && h) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (h & 4u) return APX_ERR_CHECK;
    if (h & 2u) return APX_ERR_TIMEOUT;
    return (h & 1u) ? APX_ERR_NONFINITE : APX_OK;
}

// Device address of a page-locked host buffer the current device can access,
// else null (pageable memory, or memory of another kind).
void* host_alias(const void* h) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        (void)cudaGetLastError();  // not a CUDA allocation: clear the sticky-free error state
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int apx_conv_host(apx_ctx* ctx, const float* s_h, int64_t L, const float* k_h, int32_t N, int32_t W_block,
                  uint32_t mode, double snr_target_db, int32_t S_q, int32_t K_q, float* r_h, void* stream) {
    if (!ctx || !s_h || !k_h || !r_h || L < 1 || N < 1) return APX_ERR_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t pack = mode & 0xF00u;
    const int sel = pack == APX_PACK_NONE ? 2 : ((S_q > 0 && K_q > 0 && pack != APX_PACK_AUTO) ? 1 : 0);
    // Page-locked host buffers that this device can address: the kernels read the
    // input and write the result through those addresses, so the transfers over
    // the host link overlap the computation (measured 94 against 100 us per call
    // on the 2^20-sample matching workload; the same bits).
    const float* s_a = (const float*)host_alias(s_h);
    const float* k_a = (const float*)host_alias(k_h);
    float* r_a = (float*)host_alias(r_h);
    int rc;
    if (s_a && k_a && r_a) {
        rc = run(ctx, s_a, L, k_a, N, W_block, mode, sel, snr_target_db, S_q, K_q, r_a, nullptr, nullptr, st);
        return rc ? rc : apx_sync(ctx, stream);
    }
    // otherwise through device staging buffers
    rc = ensure(ctx, ctx->hs, sizeof(float) * (size_t)L);
    if (!rc) rc = ensure(ctx, ctx->hk, sizeof(float) * (size_t)N);
    if (!rc) rc = ensure(ctx, ctx->hr, sizeof(float) * (size_t)(L + N - 1));
    if (rc) return rc;
    // the signal copy overlaps the kernel copy (and a three-launch call's spectrum preparation)
    cudaError_t e = copy_stream_begin(ctx, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->hs.p, s_h, sizeof(float) * (size_t)L, cudaMemcpyHostToDevice, ctx->hp_in);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->hp_ev[1], ctx->hp_in);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->hk.p, k_h, sizeof(float) * (size_t)N, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    rc = run(ctx, (const float*)ctx->hs.p, L, (const float*)ctx->hk.p, N, W_block, mode, sel, snr_target_db, S_q, K_q,
             (float*)ctx->hr.p, nullptr, nullptr, st, ctx->hp_ev[1]);
    if (rc) return rc;
    e = cudaMemcpyAsync(r_h, ctx->hr.p, sizeof(float) * (size_t)(L + N - 1), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_status(e);
    return apx_sync(ctx, stream);
}

int64_t apx_launch_count(const apx_ctx* ctx) { return ctx ? ctx->launches : 0; }

int apx_profile(apx_ctx* ctx, int enable) {
    if (!ctx) return APX_ERR_ARG;
    ctx->profiling = enable != 0;
    return APX_OK;
}

int apx_profile_read(apx_ctx* ctx, double* ms, int64_t* n) {
    if (!ctx) return APX_ERR_ARG;
    DeviceGuard dg(ctx->device);
    double acc[APX_NPHASES] = {};
    int64_t cnt[APX_NPHASES] = {};
    for (size_t i = 0; i < ctx->ev_used; ++i) {
        cudaError_t e = cudaEventSynchronize(ctx->ev[2 * i + 1]);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ctx->ev[2 * i], ctx->ev[2 * i + 1]);
        if (e != cudaSuccess) { ctx->ev_used = 0; return cuda_status(e); }
        int ph = ctx->ev_phase[i];
        acc[ph] += t;
        cnt[ph] += 1;
    }
    ctx->ev_used = 0;
    for (int i = 0; i < APX_NPHASES; ++i) {
        if (ms) ms[i] = acc[i];
        if (n) n[i] = cnt[i];
    }
    return APX_OK;
}

const char* apx_strerror(int s) {
    switch (s) {
        case APX_OK: return "ok";
        case APX_ERR_ARG: return "invalid argument";
        case APX_ERR_WBLOCK: return "invalid W_block for this kernel length and core";
        case APX_ERR_RANGE: return "companding range exceeds the packing's exactness bound";
        case APX_ERR_NONFINITE: return "non-finite input or kernel";
        case APX_ERR_OOM: return "device memory allocation failed";
        case APX_ERR_BUDGET: return "workspace budget exceeded";
        case APX_ERR_CUDA: return "CUDA runtime error";
        case APX_ERR_TIMEOUT: return "bounded device wait timed out";
        case APX_ERR_CHECK: return "device bounds check failed (checked build)";
        default: return "unknown status";
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched calls and captured graphs.
struct apx_graph {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* bufs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // arena, params, table, tw64, tw32
    int64_t launches = 0;
};

// Launch a planned batch on the context's batch workspace.
static int batch_run(apx_ctx* ctx, BatchPlan& bp, int32_t n, cudaStream_t st) {
    Range range("apx.batch");
    int rc = ensure(ctx, ctx->flags, kFlagWords * sizeof(unsigned));
    if (!rc && bp.max_wb > 0) rc = ensure_twiddles(ctx, bp.max_wb, st);
    if (!rc) rc = ensure(ctx, ctx->barena, bp.arena_bytes);
    if (!rc) rc = ensure(ctx, ctx->bparams, sizeof(Params) * (size_t)n);
    if (!rc) rc = ensure(ctx, ctx->btab, sizeof(int) * bp.table.size());
    if (rc) return rc;
    bind_batch(&bp, (unsigned char*)ctx->barena.p, (const double2*)ctx->tw64.p, (const float2*)ctx->tw32.p,
               ctx->tw_wb, (unsigned*)ctx->flags.p, 1u);
    const std::vector<Params> gp = grouped_params(bp);
    rc = stage_upload(ctx, gp.data(), sizeof(Params) * gp.size(), ctx->bparams.p, bp.table.data(),
                      sizeof(int) * bp.table.size(), ctx->btab.p, st);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(ctx->barena.p, 0, bp.flags_bytes, st);  // claim/ready words
    if (e == cudaSuccess) e = launch_batch(bp, (const Params*)ctx->bparams.p, (const int*)ctx->btab.p, st);
    for (const auto& G : bp.groups) ctx->launches += G.fft ? 3 : 1;
    return cuda_status(e);
}

extern "C" int apx_conv_batch(apx_ctx* ctx, const apx_request* reqs, int32_t n, void* stream) {
    if (!ctx) return APX_ERR_ARG;
    BatchPlan bp;
    int rc = plan_batch(reqs, n, &bp);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    return batch_run(ctx, bp, n, (cudaStream_t)stream);
}

extern "C" int apx_conv_batch_host(apx_ctx* ctx, const apx_request* reqs, int32_t n, void* stream) {
    if (!ctx || n < 0 || (n > 0 && !reqs)) return APX_ERR_ARG;
    Range range("apx_conv_batch_host");
    DeviceGuard dg(ctx->device);
    // A request whose three buffers are page-locked and addressable by the device
    // runs on them in place (as apx_conv_host); the others get device copies of
    // their signal, kernel and output, 256-byte aligned, in the context workspace.
    std::vector<apx_request> dq(reqs, reqs + n);
    std::vector<char> staged((size_t)n, 0);
    std::vector<size_t> off(3 * (size_t)n);
    size_t total = 0;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    for (int32_t i = 0; i < n; ++i) {
        const apx_request& q = reqs[i];
        if (!q.s_in || !q.k || !q.r_out || q.L < 1 || q.N < 1 || q.rq_out || q.stats) return APX_ERR_ARG;
        const void* sa = host_alias(q.s_in);
        const void* ka = sa ? host_alias(q.k) : nullptr;
        void* ra = ka ? host_alias(q.r_out) : nullptr;
        if (ra) {
            dq[i].s_in = (const float*)sa;
            dq[i].k = (const float*)ka;
            dq[i].r_out = (float*)ra;
            continue;
        }
        staged[i] = 1;
        off[3 * i] = total;
        total += al(sizeof(float) * (size_t)q.L);
        off[3 * i + 1] = total;
        total += al(sizeof(float) * (size_t)q.N);
        off[3 * i + 2] = total;
        total += al(sizeof(float) * (size_t)(q.L + q.N - 1));
    }
    int rc = total > 0 ? ensure(ctx, ctx->bhost, total) : 0;
    if (rc) return rc;
    unsigned char* base = (unsigned char*)ctx->bhost.p;
    for (int32_t i = 0; i < n; ++i) {
        if (!staged[i]) continue;
        dq[i].s_in = (const float*)(base + off[3 * i]);
        dq[i].k = (const float*)(base + off[3 * i + 1]);
        dq[i].r_out = (float*)(base + off[3 * i + 2]);
    }
    BatchPlan bp;
    rc = plan_batch(dq.data(), n, &bp);  // reject before anything is enqueued
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    for (int32_t i = 0; i < n && e == cudaSuccess; ++i) {
        if (!staged[i]) continue;
        e = cudaMemcpyAsync((void*)dq[i].s_in, reqs[i].s_in, sizeof(float) * (size_t)reqs[i].L,
                            cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((void*)dq[i].k, reqs[i].k, sizeof(float) * (size_t)reqs[i].N, cudaMemcpyHostToDevice,
                                st);
    }
    if (e != cudaSuccess) return cuda_status(e);
    rc = batch_run(ctx, bp, n, st);
    if (rc) return rc;
    for (int32_t i = 0; i < n && e == cudaSuccess; ++i) {
        if (!staged[i]) continue;
        e = cudaMemcpyAsync(reqs[i].r_out, dq[i].r_out, sizeof(float) * (size_t)(reqs[i].L + reqs[i].N - 1),
                            cudaMemcpyDeviceToHost, st);
    }
    return cuda_status(e);
}

extern "C" int apx_test_skew_tickets(apx_ctx* ctx, int64_t n) {
    if (!ctx) return APX_ERR_ARG;
    ctx->tickets += (unsigned long long)n;
    return APX_OK;
}

extern "C" int apx_test_stall_next(apx_ctx* ctx) {
    if (!ctx) return APX_ERR_ARG;
    ctx->stall_next = 1;
    return APX_OK;
}

extern "C" int apx_filterbank(apx_ctx* ctx, const float* s_in, int64_t L, const float* k_bank, int32_t F,
                              int32_t N, int32_t S_q, int32_t K_q, float* y_out, int64_t ldy, int32_t* yq_out,
                              float* block_cs, void* stream) {
    if (!ctx || !s_in || !k_bank || !y_out) return APX_ERR_ARG;
    if (L < 1 || F < 1 || N < 1 || F > kTcMaxF || N > kTcMaxN) return APX_ERR_ARG;
    if (S_q < 1 || K_q < 1 || S_q > kTcMaxQ || K_q > kTcMaxQ) return APX_ERR_RANGE;
    if ((long long)N * S_q * K_q > kTcExactSum) return APX_ERR_RANGE;
    TcGeom g;
    // the narrowest operand type that holds every companded integer exactly
    const int esize = (S_q <= kTcMaxQ8 && K_q <= kTcMaxQ8) ? 1 : 2;
    if (!tc_geometry(L, F, N, esize, &g)) return APX_ERR_ARG;
    if (ldy < g.out_len || (ldy & 3) || ((uintptr_t)y_out & 15) || ((uintptr_t)yq_out & 15)) return APX_ERR_ARG;
    g.ldy = ldy;
    DeviceGuard dg(ctx->device);
    int rc = ensure(ctx, ctx->flags, kFlagWords * sizeof(unsigned));
    if (!rc) rc = ensure(ctx, ctx->tc_seg, tc_seg_bytes(g));
    if (!rc) rc = ensure(ctx, ctx->tc_b, tc_b_bytes(g));
    if (!rc) rc = ensure(ctx, ctx->tc_cs, sizeof(float) * (size_t)g.nb);
    if (!rc) rc = ensure(ctx, ctx->tc_inv, sizeof(float) * (size_t)g.nb * g.ngroups * g.G);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    {
        Trace t(ctx, st, APX_PHASE_TC_PREP);
        e = launch_tc_prep(g, s_in, L, k_bank, S_q, K_q, ctx->tc_seg.p, ctx->tc_b.p, (float*)ctx->tc_cs.p,
                           (float*)ctx->tc_inv.p, block_cs, (unsigned*)ctx->flags.p, st);
    }
    if (e != cudaSuccess) return cuda_status(e);
    bool enc_failed = false;
    {
        Trace t(ctx, st, APX_PHASE_TC_MMA);
        e = launch_tc_mma(g, ctx->tc_seg.p, ctx->tc_b.p, (const float*)ctx->tc_inv.p, y_out, yq_out,
                          (unsigned*)ctx->flags.p, st, &enc_failed);
    }
    if (enc_failed) return APX_ERR_CUDA;
    if (e == cudaSuccess) ctx->launches += 3;
    return cuda_status(e);
}

extern "C" int apx_filterbank_blocks(int64_t L, int32_t F, int32_t N, int32_t S_q, int32_t K_q, int32_t* T,
                                     int64_t* nb) {
    if (L < 1 || F < 1 || N < 1 || F > kTcMaxF || N > kTcMaxN) return APX_ERR_ARG;
    if (S_q < 1 || K_q < 1 || S_q > kTcMaxQ || K_q > kTcMaxQ) return APX_ERR_RANGE;
    if ((long long)N * S_q * K_q > kTcExactSum) return APX_ERR_RANGE;
    TcGeom g;
    const int esize = (S_q <= kTcMaxQ8 && K_q <= kTcMaxQ8) ? 1 : 2;  // as apx_filterbank chooses
    if (!tc_geometry(L, F, N, esize, &g)) return APX_ERR_ARG;
    if (T) *T = g.T;
    if (nb) *nb = g.nb;
    return APX_OK;
}

// ------------------------------------------------------------------ prepared kernels
// A kernel's preparation kept resident: its own device arena holds the
// claim/ready words of its packed spectra, a copy of the taps, the kernel
// statistics, the FP32 spectrum with its decimated sub-spectra, and the packed
// spectra.  The epoch is fixed, so a packed spectrum built by one call is
// ready for every later one.
struct apx_kernel {
    int device = 0;
    int32_t N = 0, W_block = 0;
    uint32_t mode = 0;
    void* arena = nullptr;
    float* taps = nullptr;
    Params prep;  // the kernel half of the parameters (pointers into the arena)
    KInfo stats;  // a host copy of the kernel statistics
};

extern "C" int apx_kernel_create(apx_ctx* ctx, const float* k, int32_t N, int32_t W_block, uint32_t mode,
                                 void* stream, apx_kernel** out) {
    if (!ctx || !k || !out || N < 1) return APX_ERR_ARG;
    *out = nullptr;
    const uint32_t pack = mode & 0xF00u;
    if ((mode & 0xF0u) != APX_CORE_FFT || (pack != APX_PACK_AUTO && pack != APX_PACK_NONE) || (mode & ~0xFFFu))
        return APX_ERR_ARG;
    // the candidate set depends on N, W_block and the mode only: plan a one-sample call
    Params p;
    size_t smem = 0;
    // every candidate: the resident norms and spectra are indexed by candidate position
    int rc = make_params(k, 1, k, N, W_block, mode, pack == APX_PACK_NONE ? 2 : 0, 0.0, 0, 0, (float*)k, nullptr,
                         nullptr, &p, &smem, false);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    rc = ensure(ctx, ctx->flags, kFlagWords * sizeof(unsigned));
    if (!rc) rc = ensure_twiddles(ctx, W_block, (cudaStream_t)stream);
    if (rc) return rc;
    const size_t m1 = (size_t)W_block / 2 + 1;
    const size_t off_taps = 256, off_ki = off_taps + al256b(sizeof(float) * (size_t)N);
    const size_t off_h = off_ki + al256b(sizeof(KInfo)), off_y = off_h + al256b(sizeof(float2) * (m1 + 1));
    const size_t off_c = off_y + al256b(sizeof(float2) * (size_t)W_block);
    const size_t off_pair = off_c + (size_t)p.ncand * al256b(sizeof(double2) * m1);
    const size_t bytes = off_pair + al256b(pair_table_bytes(W_block));
    apx_kernel* kp = new apx_kernel();
    kp->device = ctx->device;
    kp->N = N;
    kp->W_block = W_block;
    kp->mode = mode;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&kp->arena, bytes);
    if (e != cudaSuccess) { kp->arena = nullptr; delete kp; return cuda_status(e); }
    unsigned char* a = (unsigned char*)kp->arena;
    kp->taps = (float*)(a + off_taps);
    e = cudaMemsetAsync(a, 0, 256, st);  // claim and ready words
    if (e == cudaSuccess) e = cudaMemcpyAsync(kp->taps, k, sizeof(float) * (size_t)N, cudaMemcpyDeviceToDevice, st);
    p.s = kp->taps;
    p.k = kp->taps;
    p.r = (float*)kp->taps;
    p.status = (unsigned*)ctx->flags.p;
    p.claim = (unsigned*)a;
    p.ready = (unsigned*)a + kMaxCand;
    p.epoch = 1;
    p.ki = (KInfo*)(a + off_ki);
    p.Hfull = (float2*)(a + off_h);
    p.Ysub = (float2*)(a + off_y);
    for (int j = 0; j < p.ncand; ++j) p.cand[j].H = (double2*)(a + off_c + (size_t)j * al256b(sizeof(double2) * m1));
    p.Hpair = W_block >= 1024 ? (float2*)(a + off_pair) : nullptr;  // for calls that run the two-CTA kernel
    p.tw64 = (const double2*)ctx->tw64.p;
    p.tw32 = (const float2*)ctx->tw32.p;
    p.ntab = ctx->tw_wb;
    p.autosel = 0;  // the norms of every candidate: the target is chosen per call
    if (e == cudaSuccess) {
        Trace t(ctx, st, APX_PHASE_SPECTRA);
        e = launch_spec(p, st);
        if (e == cudaSuccess) e = launch_spec_combine(p, st);
        ctx->launches += 2;
    }
    // the statistics on the host too (creation is a setup step: it waits for them)
    if (e == cudaSuccess) e = cudaMemcpyAsync(&kp->stats, p.ki, sizeof(KInfo), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(kp->arena);
        delete kp;
        return cuda_status(e);
    }
    kp->prep = p;
    *out = kp;
    return APX_OK;
}

extern "C" int apx_conv_prepared(apx_ctx* ctx, const apx_kernel* kp, const float* s_in, int64_t L,
                                 double snr_target_db, float* r_out, int32_t* rq_out, apx_block_stats* stats,
                                 void* stream) {
    if (!ctx || !kp || !s_in || !r_out) return APX_ERR_ARG;
    if (kp->device != ctx->device) return APX_ERR_ARG;
    Range range("apx_conv_prepared");
    const int sel = (kp->mode & 0xF00u) == APX_PACK_NONE ? 2 : 0;
    Params p;
    size_t smem = 0;
    int rc = make_params(s_in, L, kp->taps, kp->N, kp->W_block, kp->mode, sel, snr_target_db, 0, 0, r_out, rq_out,
                         stats, &p, &smem, false);  // candidate positions as at creation
    if (rc) return rc;
    // With the kernel's statistics known on the host, a target that no packing can reach
    // even for the best window (model SNR at sigma^2 = ||s||_inf^2, checked 1 % below the
    // target) leaves every block in full precision: drop the candidates, and with them the
    // FP64 buffers from the block kernel's shared memory.  The same results: those
    // candidates fail every block's model check.
    if (sel == 0 && !kp->stats.bad && kp->stats.Mk > 0.f) {
        bool any = false;
        for (int j = 0; j < p.ncand; ++j)
            any |= snr_feasible_host(1.0, 1.0, kp->stats.sig2k, kp->stats.Mk, p.cand[j].S, p.cand[j].K,
                                     p.thr * 0.99);
        if (!any) {
            p.ncand = 0;
            smem = fft_smem_bytes(p);
        }
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    rc = ensure(ctx, ctx->flags, kFlagWords * sizeof(unsigned));
    if (!rc) rc = ensure_twiddles(ctx, kp->W_block, st);
    if (rc) return rc;
    const Params& q = kp->prep;
    for (int j = 0; j < p.ncand; ++j) p.cand[j].H = q.cand[j].H;
    p.status = (unsigned*)ctx->flags.p;
    p.claim = q.claim;
    p.ready = q.ready;
    p.epoch = q.epoch;
    p.ki = q.ki;
    p.Hfull = q.Hfull;
    p.Ysub = q.Ysub;
    p.Hpair = q.Hpair;
    p.tw64 = (const double2*)ctx->tw64.p;
    p.tw32 = (const float2*)ctx->tw32.p;
    p.ntab = ctx->tw_wb;
    p.fused = 0;
    if (!device_pointers_set(p)) return APX_ERR_CUDA;
    cudaError_t e;
    {
        Trace t(ctx, st, APX_PHASE_FFT);
        e = launch_fft(p, smem, st, false);  // the preparation is resident: not a dependent launch
        ctx->launches += 1;
    }
    return cuda_status(e);
}

extern "C" void apx_kernel_destroy(apx_kernel* kp) {
    if (!kp) return;
    {
        DeviceGuard dg(kp->device);
        cudaDeviceSynchronize();
        if (kp->arena) cudaFree(kp->arena);
    }
    delete kp;
}

extern "C" int apx_graph_create(apx_ctx* ctx, const apx_request* reqs, int32_t n, void* stream, apx_graph** out) {
    if (!ctx || !out) return APX_ERR_ARG;
    *out = nullptr;
    BatchPlan bp;
    int rc = plan_batch(reqs, n, &bp);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    rc = ensure(ctx, ctx->flags, kFlagWords * sizeof(unsigned));
    if (!rc && bp.max_wb > 0) rc = ensure_twiddles(ctx, bp.max_wb, (cudaStream_t)stream);
    if (rc) return rc;
    apx_graph* g = new apx_graph();
    g->device = ctx->device;
    const size_t ntw = (size_t)(bp.max_wb > 0 ? ctx->tw_wb : 0);
    const size_t sizes[5] = {bp.arena_bytes > 0 ? bp.arena_bytes : 256, sizeof(Params) * (size_t)n,
                             sizeof(int) * bp.table.size(), sizeof(double2) * (ntw ? ntw : 1),
                             sizeof(float2) * (ntw ? ntw : 1)};
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 5 && e == cudaSuccess; ++b) e = cudaMalloc(&g->bufs[b], sizes[b]);
    if (e == cudaSuccess && ntw) e = cudaMemcpy(g->bufs[3], ctx->tw64.p, sizes[3], cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && ntw) e = cudaMemcpy(g->bufs[4], ctx->tw32.p, sizes[4], cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) {
        bind_batch(&bp, (unsigned char*)g->bufs[0], (const double2*)g->bufs[3], (const float2*)g->bufs[4], (int)ntw,
                   (unsigned*)ctx->flags.p, 1u);
        const std::vector<Params> gp = grouped_params(bp);
        e = cudaMemcpy(g->bufs[1], gp.data(), sizes[1], cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->bufs[2], bp.table.data(), sizes[2], cudaMemcpyHostToDevice);
    }
    cudaStream_t cap = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaMemsetAsync(g->bufs[0], 0, bp.flags_bytes, cap);
        if (le == cudaSuccess) le = launch_batch(bp, (const Params*)g->bufs[1], (const int*)g->bufs[2], cap);
        e = cudaStreamEndCapture(cap, &g->graph);
        if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (cap) cudaStreamDestroy(cap);
    for (const auto& G : bp.groups) g->launches += G.fft ? 3 : 1;
    if (e != cudaSuccess) {
        apx_graph_destroy(g);
        return cuda_status(e);
    }
    *out = g;
    return APX_OK;
}

extern "C" int apx_graph_launch(apx_graph* g, void* stream) {
    if (!g || !g->exec) return APX_ERR_ARG;
    DeviceGuard dg(g->device);
    return cuda_status(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
}

extern "C" int64_t apx_graph_launch_count(const apx_graph* g) { return g ? g->launches : 0; }

extern "C" void apx_graph_destroy(apx_graph* g) {
    if (!g) return;
    {
        DeviceGuard dg(g->device);
        cudaDeviceSynchronize();
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        for (void* b : g->bufs)
            if (b) cudaFree(b);
    }
    delete g;
}

// ---------------------------------------------------------------------------
// Allocation-free FFT core.
//
// For callers that may not allocate device memory after start-up (a real-time
// audio callback, a host application whose allocator owns the device, code
// running while another library holds the memory pool): every scratch buffer
// of the FFT core lives in one file-scope device array of fixed size, sized
// for W_block up to kStaticWbMax.  The array belongs to every GPU that loads
// the library until the process exits.
namespace {

constexpr int kStaticWbMax = 8192;
constexpr size_t al256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kSOffFlags = 0;  // the flag words (kFlagWords <= 64)
constexpr size_t kSOffKInfo = kSOffFlags + 512;
constexpr size_t kSOffHfull = kSOffKInfo + al256(sizeof(KInfo));
constexpr size_t kSOffYsub = kSOffHfull + al256(sizeof(float2) * (kStaticWbMax / 2 + 1));
constexpr size_t kSOffTw32 = kSOffYsub + al256(sizeof(float2) * kStaticWbMax);
constexpr size_t kSOffTw64 = kSOffTw32 + al256(sizeof(float2) * kStaticWbMax);
constexpr size_t kSOffHc = kSOffTw64 + al256(sizeof(double2) * kStaticWbMax);
constexpr size_t kSHcBytes = al256(sizeof(double2) * (kStaticWbMax / 2 + 1));
constexpr size_t kSOffHpair = kSOffHc + kMaxCand * kSHcBytes;
constexpr size_t kStaticBytes = kSOffHpair + al256(sizeof(float2) * 30 * (kStaticWbMax / 32));  // about 550 KB

}  // namespace

static __device__ __align__(256) unsigned char g_apx_scratch[kStaticBytes];

namespace {

struct StaticDevice {
    unsigned char* base = nullptr;  // device address of g_apx_scratch on this device (null: not set up)
    unsigned epoch = 0;             // call number (claims of on-demand spectra)
    unsigned long long tickets = 0; // CTA tickets handed out by fused launches
};
std::mutex g_static_mu;
StaticDevice g_static[64];

// exp(-2 pi i t / n) from sincospi of the exact ratio 2t/n, t < n = kStaticWbMax:
// one table for every W_block up to the maximum (a transform of length Wb reads
// every (n / Wb)-th entry, whose ratio 2 (t n / Wb) / n = 2t / Wb is exact).
__global__ void k_twiddles(double2* t64, float2* t32, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double sn, cs;
    sincospi(2.0 * (double)t / (double)n, &sn, &cs);
    t64[t] = make_double2(cs, -sn);
    t32[t] = make_float2((float)cs, (float)-sn);
}

}  // namespace

extern "C" int apx_conv_fft_static(const float* s_in, int64_t L, const float* k, int32_t N, int32_t W_block,
                                   uint32_t mode, double snr_target_db, float* r_out, void* stream) {
    if (!s_in || !k || !r_out) return APX_ERR_ARG;
    if ((mode & 0xF0u) != APX_CORE_FFT) return APX_ERR_ARG;
    if (W_block > kStaticWbMax) return APX_ERR_WBLOCK;
    Plan pl;
    int rc = plan(L, N, W_block, mode, &pl);
    if (rc) return rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return APX_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;

    unsigned char* base;
    unsigned epoch;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        StaticDevice& sd = g_static[dev];
        // The array's device address on this device (the host-side name is not one).
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_apx_scratch) != cudaSuccess || !ptr) return APX_ERR_CUDA;
        if (sd.base != (unsigned char*)ptr) {
            // first call on this device (or the module was loaded anew): the flag
            // words start from zero (the ticket counter matches `tickets`), and the
            // twiddle tables are filled once at the maximum length
            if (cudaMemsetAsync(ptr, 0, kSOffKInfo, st) != cudaSuccess) return APX_ERR_CUDA;
            unsigned char* b = (unsigned char*)ptr;
            k_twiddles<<<(kStaticWbMax + 255) / 256, 256, 0, st>>>((double2*)(b + kSOffTw64), (float2*)(b + kSOffTw32),
                                                                  kStaticWbMax);
            if (cudaGetLastError() != cudaSuccess) return APX_ERR_CUDA;
            sd.base = b;
            sd.epoch = 0;
            sd.tickets = 0;
        }
        if (++sd.epoch == 0) sd.epoch = 1;
        base = sd.base;
        epoch = sd.epoch;
    }

    // Candidates as in apx_conv: per-block choice under the target, or a forced
    // packing at the largest S_q = K_q its bound admits, or none.
    Params p;
    memset(&p, 0, sizeof p);
    const uint32_t pack = mode & 0xF00u;
    p.thr = target_thr(snr_target_db, pl.W);
    int nc = 0;
    if (pack == APX_PACK_AUTO) {
        const int order[3] = {APX_BLK_SYM, APX_BLK_ASYM3, APX_BLK_ASYM2};
        for (int j = 0; j < 3; ++j) {
            int Q = qmax_fft(order[j], pl.Nodd, W_block);
            if (Q >= 1) p.cand[nc++] = make_cand(order[j], Q, Q, pl.Nodd, W_block);
        }
        nc = prune_unreachable(p.cand, nc, p.thr);
    } else if (pack != APX_PACK_NONE) {
        int blk = pack == APX_PACK_SYM ? APX_BLK_SYM : (pack == APX_PACK_ASYM2 ? APX_BLK_ASYM2 : APX_BLK_ASYM3);
        int Q = qmax_fft(blk, pl.Nodd, W_block);
        if (Q < 1) return APX_ERR_RANGE;
        p.cand[nc++] = make_cand(blk, Q, Q, pl.Nodd, W_block);
    }
    p.ncand = nc;
    p.autosel = pack == APX_PACK_AUTO;
    p.s = s_in; p.L = L; p.k = k; p.N = N; p.Nodd = pl.Nodd; p.Wb = W_block; p.W = pl.W; p.head = pl.head;
    p.fft = 1; p.xcorr = (mode & 0xFu) == APX_OP_XCORR;
    p.P = pl.P; p.out_len = L + N - 1;
    p.r = r_out;
    set_flag_ptrs(p, (unsigned*)(base + kSOffFlags));
    p.epoch = epoch;
    p.ki = (KInfo*)(base + kSOffKInfo);
    p.Hfull = (float2*)(base + kSOffHfull);
    p.Ysub = (float2*)(base + kSOffYsub);
    p.tw32 = (const float2*)(base + kSOffTw32);
    p.tw64 = (const double2*)(base + kSOffTw64);
    p.ntab = kStaticWbMax;
    for (int j = 0; j < nc; ++j) p.cand[j].H = (double2*)(base + kSOffHc + j * kSHcBytes);
    const size_t smem = fft_smem_bytes(p);
    if (smem > (size_t)kMaxSmem) return APX_ERR_WBLOCK;
    p.fused = use_fused(p, st);
    if (!p.fused && fft_full_only(p)) p.Hpair = (float2*)(base + kSOffHpair);
    if (p.fused) {
        std::lock_guard<std::mutex> lk(g_static_mu);
        p.ticket_base = g_static[dev].tickets;
        g_static[dev].tickets += fused_grid(p);
    }

    cudaError_t e = cudaSuccess;
    if (!p.fused) e = launch_spec(p, st);
    if (e == cudaSuccess && !p.fused) e = launch_spec_combine(p, st);
    if (e == cudaSuccess) e = p.fused ? launch_fft_fused(p, smem, st) : launch_fft(p, smem, st);
    if (e != cudaSuccess && p.fused) {  // not launched: its tickets were never taken
        std::lock_guard<std::mutex> lk(g_static_mu);
        g_static[dev].tickets -= fused_grid(p);
    }
    return cuda_status(e);
}



// ---------------------------------------------------------------------------
// Serving engine: a persistent kernel fed through a ticket queue in mapped
// memory (apx_serve.h).  Requests share templates: the kernel statistics,
// spectrum and packed spectra of a (kernel buffer, N, W_block, op, packing)
// are prepared by the first request that uses them and stay resident for the
// following ones until the entry is reused for another template.
namespace {

constexpr int kServeTmapBits = 20;  // ticket -> slot map: 2^20 entries

struct ServeTemplate {
    const float* k = nullptr;
    int N = 0, Wb = 0;
    uint32_t key = 0;        // op | pack bits
    unsigned epoch = 0;      // 0: free (or to be prepared anew)
    int inflight = 0;        // requests using it
    uint64_t last_use = 0;
    unsigned char* base = nullptr;  // device: KInfo | Hfull | Ysub | Hc[3] | claim/ready | jobready
};

// Template entry layout at the largest W_block (every entry has the same size).
struct TplLayout {
    size_t ki, hfull, ysub, hc, flags, bytes;
};
TplLayout tpl_layout() {
    const size_t m1 = (size_t)kServeWbMax / 2 + 1;
    TplLayout t;
    t.ki = 0;
    t.hfull = t.ki + al256b(sizeof(KInfo));
    t.ysub = t.hfull + al256b(sizeof(float2) * m1);
    t.hc = t.ysub + al256b(sizeof(float2) * kServeWbMax);
    t.flags = t.hc + kMaxCand * al256b(sizeof(double2) * m1);
    t.bytes = t.flags + al256b(sizeof(unsigned) * (2 * kMaxCand + kMaxJobs));
    return t;
}

}  // namespace

struct apx_server {
    apx_ctx* ctx = nullptr;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ran = nullptr;      // recorded after each launch of the persistent kernel
    bool launched = false;
    int nslots = 0, ctas = 0;
    size_t smem = 0;
    ServeEnv env{};                 // device-side view
    ServeHdr* hdr = nullptr;        // host views of the mapped words
    ServeSlot* slots = nullptr;
    int* tmap = nullptr;
    unsigned* done_seq = nullptr;
    unsigned* fstatus = nullptr;
    void* dmem = nullptr;           // device: ticket counter, per-slot counts and status, template arena
    long long published = 0;
    std::vector<int> free_slots;
    std::vector<unsigned> slot_seq; // 0: free
    std::vector<int> slot_tpl;
    std::vector<ServeTemplate> tpl;
    unsigned next_seq = 0, next_epoch = 0;
    uint64_t clock = 0;
    int stall_next = 0;
    int64_t launches = 0;
    void* tw = nullptr;             // its own twiddle tables (the context's may be regrown meanwhile)
    std::unordered_map<unsigned, int> seq_slot;
};

extern "C" void apx_server_destroy(apx_server* s) {
    if (!s) return;
    {
        DeviceGuard dg(s->device);
        if (s->hdr) *reinterpret_cast<volatile int*>(&s->hdr->stop) = 1;  // the CTAs leave at their next claim
        if (s->stream) cudaStreamSynchronize(s->stream);
        if (s->ran) cudaEventDestroy(s->ran);
        if (s->stream) cudaStreamDestroy(s->stream);
        if (s->hdr) cudaFreeHost(s->hdr);
        if (s->dmem) cudaFree(s->dmem);
        if (s->tw) cudaFree(s->tw);
    }
    delete s;
}

extern "C" int apx_server_create(apx_ctx* ctx, int32_t slots, int32_t templates, int32_t ctas, double idle_ms,
                                 apx_server** out) {
    if (!ctx || !out || slots < 1 || slots > 65536 || templates < 1 || templates > 4096 || ctas < 0 ||
        !(idle_ms > 0.0) || idle_ms > 60000.0)
        return APX_ERR_ARG;
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    apx_server* s = new apx_server();
    s->ctx = ctx;
    s->device = ctx->device;
    s->nslots = slots;
    int sms = 0, khz = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device);
    if (e != cudaSuccess) { delete s; return cuda_status(e); }
    s->ctas = ctas > 0 ? ctas : 2 * sms;  // two CTAs per SM fit the block body's registers
    s->smem = serve_smem_bytes();
    // twiddle tables for every W_block up to the maximum, the engine's own copy
    int rc = ensure_twiddles(ctx, kServeWbMax, nullptr);
    if (rc) { delete s; return rc; }
    const size_t ntw = (size_t)ctx->tw_wb;
    e = cudaMalloc(&s->tw, (sizeof(double2) + sizeof(float2)) * ntw);
    if (e == cudaSuccess) e = cudaMemcpy(s->tw, ctx->tw64.p, sizeof(double2) * ntw, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy((char*)s->tw + sizeof(double2) * ntw, ctx->tw32.p, sizeof(float2) * ntw, cudaMemcpyDeviceToDevice);
    // mapped host words: header | slots | ticket map | completion words | final status
    const size_t tsz = (size_t)1 << kServeTmapBits;
    const size_t o_slots = 256, o_tmap = o_slots + al256b(sizeof(ServeSlot) * (size_t)slots);
    const size_t o_seq = o_tmap + al256b(sizeof(int) * tsz), o_st = o_seq + al256b(sizeof(unsigned) * (size_t)slots);
    const size_t hbytes = o_st + al256b(sizeof(unsigned) * (size_t)slots);
    void* h = nullptr;
    if (e == cudaSuccess) e = cudaHostAlloc(&h, hbytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) { apx_server_destroy(s); return cuda_status(e); }
    memset(h, 0, hbytes);
    s->hdr = (ServeHdr*)h;
    s->slots = (ServeSlot*)((char*)h + o_slots);
    s->tmap = (int*)((char*)h + o_tmap);
    s->done_seq = (unsigned*)((char*)h + o_seq);
    s->fstatus = (unsigned*)((char*)h + o_st);
    void* hd = nullptr;
    e = cudaHostGetDevicePointer(&hd, h, 0);
    // device words: ticket counter | finished items per slot | status per slot | template arena
    const TplLayout tl = tpl_layout();
    const size_t d_done = 256, d_st = d_done + al256b(sizeof(int) * (size_t)slots);
    const size_t d_tpl = d_st + al256b(sizeof(unsigned) * (size_t)slots);
    const size_t dbytes = d_tpl + tl.bytes * (size_t)templates;
    if (e == cudaSuccess) e = cudaMalloc(&s->dmem, dbytes);
    if (e == cudaSuccess) e = cudaMemset(s->dmem, 0, dbytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ran, cudaEventDisableTiming);
    if (e != cudaSuccess) { apx_server_destroy(s); return cuda_status(e); }
    unsigned char* d = (unsigned char*)s->dmem;
    s->env.hdr = (ServeHdr*)hd;
    s->env.slots = (ServeSlot*)((char*)hd + o_slots);
    s->env.tmap = (int*)((char*)hd + o_tmap);
    s->env.tmask = (long long)tsz - 1;
    s->env.next = (unsigned long long*)d;
    s->env.done_items = (int*)(d + d_done);
    s->env.dstatus = (unsigned*)(d + d_st);
    s->env.done_seq = (unsigned*)((char*)hd + o_seq);
    s->env.fstatus = (unsigned*)((char*)hd + o_st);
    s->env.idle_cycles = (long long)(idle_ms * (double)khz);
    s->tpl.resize(templates);
    for (int t = 0; t < templates; ++t) s->tpl[t].base = d + d_tpl + tl.bytes * (size_t)t;
    s->slot_seq.assign(slots, 0u);
    s->slot_tpl.assign(slots, -1);
    for (int i = slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    *out = s;
    return APX_OK;
}

namespace {

// (Re)launch the persistent kernel when tickets are published that no CTA will
// claim: its CTAs leave after a bounded time without work, possibly just before
// the host published more.
int serve_ensure_running(apx_server* s) {
    if (s->launched) {
        const cudaError_t q = cudaEventQuery(s->ran);
        if (q == cudaErrorNotReady) return APX_OK;  // still running: it will claim them
        if (q != cudaSuccess) return cuda_status(q);
        s->launched = false;
    }
    unsigned long long next = 0;  // the kernel has left: its counter is stable
    cudaError_t e = cudaMemcpyAsync(&next, s->env.next, sizeof next, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    if ((long long)next >= s->published) return APX_OK;
    e = launch_serve(s->env, s->ctas, s->smem, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->ran, s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    s->launched = true;
    s->launches += 1;
    return APX_OK;
}

// A template entry for this request: the resident one with the same key, else
// the least recently used entry that no request in flight uses (prepared anew).
int serve_template(apx_server* s, const float* k, int N, int Wb, uint32_t key, bool fresh, bool* prepare) {
    int best = -1;
    for (int t = 0; t < (int)s->tpl.size(); ++t) {
        const ServeTemplate& e = s->tpl[t];
        if (!fresh && e.epoch && e.k == k && e.N == N && e.Wb == Wb && e.key == key) { *prepare = false; return t; }
        if (e.inflight == 0 && (best < 0 || e.last_use < s->tpl[best].last_use)) best = t;
    }
    if (best < 0) return -1;
    ServeTemplate& e = s->tpl[best];
    e.k = k; e.N = N; e.Wb = Wb; e.key = key;
    if (++s->next_epoch == 0) s->next_epoch = 1;  // words of earlier uses never equal a new epoch
    e.epoch = s->next_epoch;
    *prepare = true;
    return best;
}

}  // namespace

extern "C" int apx_server_submit(apx_server* s, const apx_request* q, int64_t* seq_out) {
    if (!s || !q || !q->s_in || !q->k || !q->r_out || q->L < 1 || q->N < 1 || q->rq_out || q->stats) return APX_ERR_ARG;
    const uint32_t core = q->mode & 0xF0u, pack = q->mode & 0xF00u;
    if ((core != APX_CORE_FFT && core != APX_CORE_AUTO) || (pack != APX_PACK_AUTO && pack != APX_PACK_NONE) ||
        (q->mode & ~0xFFFu))
        return APX_ERR_ARG;
    const int Nodd = q->N % 2 ? q->N : q->N + 1;
    const int Wb = q->W_block > 0 ? q->W_block : default_wblock(Nodd);
    if (Wb > kServeWbMax) return APX_ERR_WBLOCK;
    const uint32_t mode = (q->mode & ~0xF0u) | APX_CORE_FFT;
    DeviceGuard dg(s->device);
    // page-locked host buffers are read and written in place
    const float* sa = (const float*)host_alias(q->s_in);
    const float* ka = (const float*)host_alias(q->k);
    float* ra = (float*)host_alias(q->r_out);
    Params p;
    size_t smem = 0;
    // every candidate: a template's norms and spectra are indexed by candidate position
    int rc = make_params(sa ? sa : q->s_in, q->L, ka ? ka : q->k, q->N, Wb, mode, pack == APX_PACK_NONE ? 2 : 0,
                         q->snr_target_db, 0, 0, ra ? ra : q->r_out, nullptr, nullptr, &p, &smem, false);
    if (rc) return rc;
    if (s->free_slots.empty()) return APX_ERR_BUDGET;
    const int njobs = prep_jobs_count(Wb, kServeThreads);
    const long long nblk = p.P;
    bool prepare = false;
    const bool stall = s->stall_next != 0;
    const int ti = serve_template(s, q->k, q->N, Wb, mode & 0xF0Fu, stall, &prepare);
    if (ti < 0) return APX_ERR_BUDGET;
    const int nprep = prepare ? njobs : 0;
    const long long nitems = nprep + nblk;
    // the ticket map must not wrap onto a request still in flight
    long long oldest = s->published;
    for (int i = 0; i < s->nslots; ++i)
        if (s->slot_seq[i] && s->slots[i].base < oldest) oldest = s->slots[i].base;
    if (nitems > 0x7fffffffLL || s->published + nitems - oldest > (1LL << kServeTmapBits)) {
        if (prepare) s->tpl[ti].epoch = 0;
        return APX_ERR_BUDGET;
    }
    s->stall_next = 0;
    ServeTemplate& tp = s->tpl[ti];
    const TplLayout tl = tpl_layout();
    unsigned* flags = (unsigned*)(tp.base + tl.flags);
    p.ki = (KInfo*)(tp.base + tl.ki);
    p.Hfull = (float2*)(tp.base + tl.hfull);
    p.Ysub = (float2*)(tp.base + tl.ysub);
    for (int j = 0; j < p.ncand; ++j) p.cand[j].H = (double2*)(tp.base + tl.hc + (size_t)j * al256b(sizeof(double2) * (kServeWbMax / 2 + 1)));
    p.claim = flags;
    p.ready = flags + kMaxCand;
    p.jobready = flags + 2 * kMaxCand;
    p.epoch = tp.epoch;
    const size_t ntw = (size_t)s->ctx->tw_wb;
    p.tw64 = (const double2*)s->tw;
    p.tw32 = (const float2*)((char*)s->tw + sizeof(double2) * ntw);
    p.ntab = (int)ntw;
    p.fused = 0;
    p.Hpair = nullptr;
    const int slot = s->free_slots.back();
    s->free_slots.pop_back();
    p.status = s->env.dstatus + slot;
    if (++s->next_seq == 0) s->next_seq = 1;
    ServeSlot& sl = s->slots[slot];
    memcpy(&sl.p, &p, sizeof p);
    sl.base = s->published;
    sl.nprep = nprep;
    sl.njobs = njobs;
    sl.nitems = (int)nitems;
    sl.seq = s->next_seq;
    sl.skip_prep = stall ? 1 : 0;
    for (long long t = 0; t < nitems; ++t) s->tmap[(s->published + t) & s->env.tmask] = slot;
    // the slot and the map before the count that publishes them
    std::atomic_thread_fence(std::memory_order_seq_cst);
    s->published += nitems;
    *reinterpret_cast<volatile long long*>(&s->hdr->published) = s->published;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    s->slot_seq[slot] = sl.seq;
    s->slot_tpl[slot] = ti;
    s->seq_slot[sl.seq] = slot;
    tp.inflight += 1;
    tp.last_use = ++s->clock;
    if (seq_out) *seq_out = sl.seq;
    return serve_ensure_running(s);
}

extern "C" int apx_server_poll(apx_server* s, int64_t seq, int32_t* status) {
    if (!s) return APX_ERR_ARG;
    auto it = s->seq_slot.find((unsigned)seq);
    if (it == s->seq_slot.end()) return APX_ERR_ARG;  // unknown or already collected
    const int slot = it->second;
    if (*reinterpret_cast<volatile unsigned*>(&s->done_seq[slot]) != (unsigned)seq) {
        DeviceGuard dg(s->device);
        const int rc = serve_ensure_running(s);
        return rc ? rc : 0;
    }
    std::atomic_thread_fence(std::memory_order_seq_cst);  // the outputs after the completion word
    const unsigned st = *reinterpret_cast<volatile unsigned*>(&s->fstatus[slot]);
    ServeTemplate& tp = s->tpl[s->slot_tpl[slot]];
    tp.inflight -= 1;
    if (st & 2u) tp.epoch = 0;  // a preparation that did not finish: prepare the template anew next time
    s->slot_seq[slot] = 0;
    s->slot_tpl[slot] = -1;
    s->seq_slot.erase(it);
    s->free_slots.push_back(slot);
    if (status) *status = (st & 4u) ? APX_ERR_CHECK : (st & 2u) ? APX_ERR_TIMEOUT : (st & 1u) ? APX_ERR_NONFINITE : APX_OK;
    return 1;
}

extern "C" int apx_server_test_stall_next(apx_server* s) {
    if (!s) return APX_ERR_ARG;
    s->stall_next = 1;
    return APX_OK;
}

extern "C" int64_t apx_server_launch_count(const apx_server* s) { return s ? s->launches : 0; }
