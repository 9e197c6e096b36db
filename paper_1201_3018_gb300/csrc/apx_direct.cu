// apx_direct.cu -- fused per-block kernel of the time-domain (direct) core.
//
// One launch per call, one CTA per overlap-save block: load the W_block window,
// kernel and block statistics, Section IV.D selection, companding (Eq. 2) and
// packing (Eqs. 4, 5, 7) of block and taps into shared memory, the packed FP64
// convolution (Eqs. 8-9) with a register sliding window, digit extraction
// (Eqs. 11-15), inverse companding (Eq. 16) and the Eq. (17) store.  Blocks
// without an admissible packing run the FP32 full-precision convolution in the
// same CTA.  With APX_CORE_TC the candidate is the block's companded integers
// convolved on the tensor cores instead (tc_block below).
#include <cuda_fp16.h>

#include "apx_block.cuh"
#include "apx_launch.h"
#include "apx_umma.cuh"

namespace apx {

constexpr int kRf = 8;  // FP32 outputs per thread (taps padded to a multiple of 8)
constexpr int kRd = 4;  // FP64 outputs per thread (taps padded to a multiple of 4)

// Taps are staged in shared memory a chunk at a time, so that neither the
// kernel length nor the block length limits which packings a CTA can run.
// The chunked forms continue the sums the previous chunk left in acc, in the
// same order as one pass over all taps would take.
constexpr int kKcF = kDirectTapChunkF;  // FP32 taps per chunk (8 KB)
constexpr int kKcD = kDirectTapChunkD;  // packed FP64 taps per chunk (8 KB)

// acc[r] += sum_{n0 <= n < n1} sig[j0 + r - n] taps[n - n0], n1 - n0 a multiple
// of R; sig is zero-padded by >= n1 in front.  Register ring: slot (t mod R)
// holds sig[j0 + t - n].
template <int R>
__device__ __forceinline__ void conv_f32(const float* sig, const float* taps, int n0, int n1, int j0,
                                         float (&acc)[R]) {
    float w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = sig[j0 + r - n0];
    for (int n = n0; n < n1; n += R) {
        float t[R];
#pragma unroll
        for (int v = 0; v < R; v += 4) {
            float4 q = *reinterpret_cast<const float4*>(taps + (n - n0) + v);
            t[v] = q.x; t[v + 1] = q.y; t[v + 2] = q.z; t[v + 3] = q.w;
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fmaf(w[(r - u + R) % R], t[u], acc[r]);
            w[R - 1 - u] = sig[j0 - n - u - 1];
        }
    }
}

// The packed FP64 form over the nsig packed words, zero outside [0, nsig)
// (the block's history and tail; a predicated read costs nothing beside an
// FP64 multiply-add).  NOFMA: separate correctly rounded products and sums in
// the same order (the paper-literal form, the oracle's arithmetic step for
// step).
template <int R, bool NOFMA>
__device__ __forceinline__ void conv_f64(const double* sig, int nsig, const double* taps, int n0, int n1, int j0,
                                         double (&acc)[R]) {
    auto at = [&](int i) { return (unsigned)i < (unsigned)nsig ? sig[i] : 0.0; };
    double w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = at(j0 + r - n0);
    for (int n = n0; n < n1; n += R) {
        double t[R];
#pragma unroll
        for (int v = 0; v < R; v += 2) {
            double2 q = *reinterpret_cast<const double2*>(taps + (n - n0) + v);
            t[v] = q.x; t[v + 1] = q.y;
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                acc[r] = NOFMA ? __dadd_rn(acc[r], __dmul_rn(w[(r - u + R) % R], t[u]))
                               : fma(w[(r - u + R) % R], t[u], acc[r]);
            w[R - 1 - u] = at(j0 - n - u - 1);
        }
    }
}

// The FP64 full-precision form (APX_FULL_FP64): every tap resident, the
// window zero-padded by >= nkp in front.
template <int R>
__device__ __forceinline__ void conv_f64_full(const double* sig, const double* taps, int nkp, int j0,
                                              double (&acc)[R]) {
    double w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { acc[r] = 0.0; w[r] = sig[j0 + r]; }
    for (int n = 0; n < nkp; n += R) {
        double t[R];
#pragma unroll
        for (int v = 0; v < R; v += 2) {
            double2 q = *reinterpret_cast<const double2*>(taps + n + v);
            t[v] = q.x; t[v + 1] = q.y;
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fma(w[(r - u + R) % R], t[u], acc[r]);
            w[R - 1 - u] = sig[j0 - n - u - 1];
        }
    }
}

__device__ __forceinline__ int round_up(int a, int m) { return (a + m - 1) / m * m; }

// A thread's run of R outputs j0 .. j0+R-1 (R a multiple of 4) goes out as
// 16-byte stores when it is kept whole and starts on a 16-byte boundary of r.
template <int R>
__device__ __forceinline__ bool run_vec(const Params& p, const BlockGeom& g, int j0) {
    const long long o = g.start + j0;
    return j0 + R <= g.hi && o >= 0 && o + R <= p.out_len && head16(p.r + o) == 0;
}
template <int R>
__device__ __forceinline__ void store_run(const Params& p, long long o, const float (&v)[R], bool zero_rq) {
#pragma unroll
    for (int r = 0; r < R; r += 4)
        *reinterpret_cast<float4*>(p.r + o + r) = make_float4(v[r], v[r + 1], v[r + 2], v[r + 3]);
    if (zero_rq) {
        if (head16(p.rq + o) == 0) {
#pragma unroll
            for (int r = 0; r < R; r += 4) *reinterpret_cast<int4*>(p.rq + o + r) = make_int4(0, 0, 0, 0);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) p.rq[o + r] = 0;
        }
    }
}

// Full precision (FP32), Eq. (1) over the window, taps staged in shared memory
// a chunk at a time; a later chunk continues the sums the thread stored for
// its outputs.  xs: the window behind a zero pad of dl.padF samples.
__device__ void full_block_f32(const Params& p, long long i, const BlockGeom& g, const Pro& pr, const float* xs,
                               unsigned char* smem) {
    const DirectLayout& dl = p.dl;
    const int nkp = round_up(p.Nodd, kRf);
    float* kf = reinterpret_cast<float*>(smem + dl.offK);
    const int nout = g.hi - g.lo;
    for (int n0 = 0; n0 < nkp; n0 += kKcF) {
        const int n1 = min(nkp, n0 + kKcF);
        if (n0 > 0) __syncthreads();  // every thread is done with the previous chunk
        for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x) kf[n - n0] = ktap(p, n);
        __syncthreads();
        for (int ch = threadIdx.x; ch * kRf < nout; ch += blockDim.x) {
            const int j0 = g.lo + ch * kRf;
            if (!APX_IN_BOUNDS(j0 - n1 >= -dl.padF && j0 + kRf <= p.Wb + 8, p.status)) continue;
            const bool vec = run_vec<kRf>(p, g, j0);
            float acc[kRf];
            if (vec) {
#pragma unroll
                for (int r = 0; r < kRf; r += 4) {
                    const float4 a = n0 > 0 ? *reinterpret_cast<const float4*>(p.r + g.start + j0 + r)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
                    acc[r] = a.x; acc[r + 1] = a.y; acc[r + 2] = a.z; acc[r + 3] = a.w;
                }
            } else {
#pragma unroll
                for (int r = 0; r < kRf; ++r) {
                    const long long o = g.start + j0 + r;
                    acc[r] = (n0 > 0 && j0 + r < g.hi && o >= 0 && o < p.out_len) ? p.r[o] : 0.f;
                }
            }
            conv_f32<kRf>(xs, kf, n0, n1, j0, acc);
            if (vec) {
                store_run<kRf>(p, g.start + j0, acc, p.rq && n1 == nkp);
            } else {
#pragma unroll
                for (int r = 0; r < kRf; ++r) {
                    const int j = j0 + r;
                    const long long o = g.start + j;
                    if (j < g.hi && o >= 0 && o < p.out_len) {
                        p.r[o] = acc[r];
                        if (p.rq && n1 == nkp) p.rq[o] = 0;
                    }
                }
            }
        }
    }
    if (p.st && threadIdx.x == 0)
        write_stats(p, i, APX_BLK_FULL, nullptr, 0.f, pr.Ms, pro_sig2(pr, p.Wb),
                    __longlong_as_double(0x7ff0000000000000ll), 0.0);
}

// ---- the tensor-core candidate (APX_CORE_TC)
// Eq. (1) on the block's companded integers (Eq. 2) as a product on the
// tensor cores.  Output j = q R + p of the block (R = kTcbRow phases, q < RB =
// W_block / R rows) is
//   r~[j] = sum_x A[q][x] B[p][x],  A[q][x] = s~[q R + x - KN],  B[p][x] = k~[p + KN - x],
// x < KN + R (s~ zero outside the window, k~ zero outside [0, N')).  Every row
// of A is a row of one segment S[r][x'] = s~[r R + x' - KN] (x' < R): K slice
// kt of A is rows kt .. kt+127 of S, so S is written once and each slice's
// descriptor starts kt rows further in; rows past the block's own are read
// by the MMA but never read back.  FP16 holds every |s~|, |k~| <= 2048, their
// products are exact in FP32, and so is every partial sum (N' S_q K_q <= 2^24):
// the integers are exact, as the packed FP64 forms' are.
// Column of accumulator element (q, x) in the staging rows of 64 FP32 values:
// the 32 lanes of a warp writing one row each (q = lane, x fixed) hit 32
// different banks, and the 32 lanes reading four consecutive outputs each
// (x = 4 lane + c over two rows) at most two to a bank, none when the warp's
// first output starts a row.  x ^ (q mod 32) spreads the rows; bit 5 of x,
// moved to bit 1, separates x from x + 32 within a row.
__device__ __forceinline__ int tc_stage_col(int q, int x) { return x ^ (q & 31) ^ ((x >> 4) & 2); }

__device__ __forceinline__ uint32_t pack_h2(int a, int b) {
    return (uint32_t)__half_as_ushort(__int2half_rn(a)) | ((uint32_t)__half_as_ushort(__int2half_rn(b)) << 16);
}

// Operand buffers of a CTA (1024-byte aligned, in the 128-byte swizzle): the
// segment (128 + NS - 1 rows of 128 bytes), then NS tap slices of 64 rows.
struct TcBufs {
    uint32_t abase, bbase;  // shared-memory addresses
    unsigned char *abuf, *bbuf;
};
__device__ __forceinline__ TcBufs tc_bufs(const Params& p, unsigned char* smem) {
    const DirectLayout& dl = p.dl;
    TcBufs t;
    const uint32_t raw = smem_u32(smem + dl.offS);
    t.abase = (raw + 1023u) & ~1023u;
    const uint32_t aspan = ((uint32_t)(128 + dl.nS - 1) * 128u + 1023u) & ~1023u;
    t.bbase = t.abase + aspan;
    t.abuf = smem + dl.offS + (t.abase - raw);
    t.bbuf = t.abuf + aspan;
    return t;
}

// The kernel's Toeplitz slices B[p][x] = k~[p + KN - x] (Eq. 2 on the taps),
// once per CTA.  The companded taps are staged in the FP32 tap chunk's space.
__device__ void tc_prepare_taps(const Params& p, const TcBufs& tb, float ck, unsigned char* smem) {
    const DirectLayout& dl = p.dl;
    const int KN = dl.padS, NS = dl.nS, t = threadIdx.x;
    short* kh = reinterpret_cast<short*>(smem + dl.offK);
    for (int n = t; n < p.Nodd; n += blockDim.x) kh[n] = (short)kq(p, ck, n);
    __syncthreads();
    for (int ch = t; ch < NS * 512; ch += blockDim.x) {
        const int kt = ch >> 9, ph = (ch >> 3) & 63, c16 = ch & 7;
        const int n0 = ph + KN - kt * kTcbRow - c16 * 8;  // element x of the chunk is tap n0 - x
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int na = n0 - 2 * h, nb = na - 1;
            w[h] = pack_h2((na >= 0 && na < p.Nodd) ? kh[na] : 0, (nb >= 0 && nb < p.Nodd) ? kh[nb] : 0);
        }
        *reinterpret_cast<uint4*>(tb.bbuf + kt * 8192 + ph * 128 + ((c16 ^ (ph & 7)) << 4)) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();  // the tap chunk's space is free again (a full-precision block may use it)
}

// One block on the tensor cores: the segment of its companded window, the
// MMAs (completion on bar, phase `parity`), the rows back from tensor memory,
// Eq. (16) and Eq. (17).
__device__ void tc_block_body(const Params& p, long long i, const BlockGeom& g, const Cand& c, const KStats& ks,
                              const Pro& pr, float ck, float* xs, const TcBufs& tb, uint32_t tmem, uint32_t bar,
                              uint32_t parity, Shared& sh) {
    const DirectLayout& dl = p.dl;
    const int KN = dl.padS, NS = dl.nS, RB = p.Wb / kTcbRow, t = threadIdx.x;
    const float cs = compand_factor(c.S, pr.Ms);  // Eq. (2)
    // the Eq. (16) factor (an FP64 division, slow on this part) from the last
    // thread, which takes no part in the MMA issue, while the operands are built
    if (t == blockDim.x - 1) sh.bcast[0] = 1.0 / ((double)cs * (double)ck);
    for (int ch = t; ch < (RB + NS - 1) * 8; ch += blockDim.x) {
        const int r = ch >> 3, c16 = ch & 7, t0 = r * kTcbRow + c16 * 8 - KN;
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int ta = t0 + 2 * h, tb2 = ta + 1;
            w[h] = pack_h2((ta >= 0 && ta < p.Wb) ? compand(cs, xs[ta]) : 0,
                           (tb2 >= 0 && tb2 < p.Wb) ? compand(cs, xs[tb2]) : 0);
        }
        *reinterpret_cast<uint4*>(tb.abuf + r * 128 + ((c16 ^ (r & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the operands, visible to the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (t == 0) {
        for (int kt = 0; kt < NS; ++kt)
#pragma unroll
            for (int k = 0; k < 4; ++k)  // four K = 16 steps of 32 bytes per 128-byte row
                umma_f16_id(tmem, sdesc_sw128(tb.abase + (uint32_t)kt * 128u + 32u * k),
                            sdesc_sw128(tb.bbase + (uint32_t)kt * 8192u + 32u * k), umma_idesc_f16(128, kTcbRow),
                            (kt | k) != 0);
        umma_commit(bar);
        // the issuing thread alone waits (bounded: false after about two
        // seconds); the others wait at the barrier instead of polling
        sh.redi[0] = mbar_wait(bar, parity, true) ? 1 : 0;
    }
    __syncthreads();
    tc_fence_after();
    const bool ok = sh.redi[0] != 0;
    // Accumulator row q (tensor-memory lane q) into the FP32 window's space, now
    // dead, at the columns tc_stage_col gives.
    float* stage = xs;
    const int warp = t >> 5, lane = t & 31;
    if (warp < 4 && warp * 32 < RB) {
        const int q = warp * 32 + lane;
        const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int hx = 0; hx < 2; ++hx) {
            uint32_t v[32];
            tmem_ld32_nowait(tw + 32u * hx, v);
            tmem_wait_ld(v);
            if (q < RB) {
#pragma unroll
                for (int x = 0; x < 32; ++x) stage[q * kTcbRow + tc_stage_col(q, hx * 32 + x)] = __uint_as_float(v[x]);
            }
        }
    }
    tc_fence_before();
    if (!ok && t == 0) atomicOr(p.status, 2u);  // timed out: the block's outputs are not valid
    __syncthreads();
    const float inv = (float)sh.bcast[0];
    // Inverse compand (Eq. 16), place (Eq. 17).  The integers are exact in FP32
    // (|r~| <= 2^24): no 64-bit conversion, whose FP64 pipe is slow on this part.
    store_kept(p, g, [&](int j, int& iv) {
        const int q = j / kTcbRow;
        const float v = stage[q * kTcbRow + tc_stage_col(q, j % kTcbRow)];
        iv = __float2int_rn(v);
        return __fmul_rn(v, inv);
    });
    if (p.st && t == 0)  // (the model's FP64 log10 only where a record is written)
        write_stats(p, i, APX_BLK_TC, &c, cs, pr.Ms, pro_sig2(pr, p.Wb),
                    snr_model_db(pro_sig2(pr, p.Wb), pr.Ms, ks.sig2k, ks.Mk, c.S, c.K),
                    0.0);
}

// The FP64 full-precision form over the block's kept outputs, R per thread,
// rounded once to FP32 (16-byte stores for runs of 4 kept whole and aligned).
template <int R>
__device__ __forceinline__ void full64_pass(const Params& p, const BlockGeom& g, const double* sd, const double* kd,
                                            int nkp) {
    const int nout = g.hi - g.lo;
    for (int ch = threadIdx.x; ch * R < nout; ch += blockDim.x) {
        const int j0 = g.lo + ch * R;
        double acc[R];
        conv_f64_full<R>(sd, kd, nkp, j0, acc);
        float accf[R];
#pragma unroll
        for (int r = 0; r < R; ++r) accf[r] = __double2float_rn(acc[r]);
        if constexpr (R % 4 == 0) {
            if (run_vec<R>(p, g, j0)) {
                store_run<R>(p, g.start + j0, accf, p.rq != nullptr);
                continue;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = j0 + r;
            const long long o = g.start + j;
            if (j < g.hi && o >= 0 && o < p.out_len) {
                p.r[o] = accf[r];
                if (p.rq) p.rq[o] = 0;
            }
        }
    }
}

// One tap chunk [n0, n1) of the packed FP64 convolution over outputs [olo,
// ohi), R per thread, continuing the partial sums in tb.
template <int R, bool LIT>
__device__ __forceinline__ void packed_conv_pass(const double* sb, int nsb, const double* kb, double* tb, int n0,
                                                 int n1, int olo, int ohi) {
    for (int ch = threadIdx.x; olo + ch * R < ohi; ch += blockDim.x) {
        const int j0 = olo + ch * R;
        double acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = (n0 > 0 && j0 + r < ohi) ? tb[j0 + r] : 0.0;
        conv_f64<R, LIT>(sb, nsb, kb, n0, n1, j0, acc);
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (j0 + r < ohi) tb[j0 + r] = acc[r];
    }
}

// LIT: the paper-literal symmetric form (APX_LITERAL, single calls only) in
// an instantiation of its own, so that the other kernels are compiled as if
// it did not exist.
template <bool BATCH, bool LIT>
__global__ void __launch_bounds__(kDirectThreads, 4) k_direct(const Params p0, const BatchTab bt) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ unsigned s_feas;
    __shared__ Params sp;
    const long long i = BATCH ? batch_enter(bt, sp) : (long long)blockIdx.x;
    const Params& p = BATCH ? sp : p0;
    const BlockGeom g = block_geom(p, i);
    const DirectLayout& dl = p.dl;

    float* xs = reinterpret_cast<float*>(smem) + dl.padF;
    for (int t = threadIdx.x; t < dl.padF; t += blockDim.x) xs[t - dl.padF] = 0.f;
    for (int t = threadIdx.x; t < kRf; t += blockDim.x) xs[p.Wb + t] = 0.f;
    load_window(p, g, xs);

    // Kernel initialisation of Section IV, done by every CTA from the raw taps.
    const KStats ks = kernel_stats(p, sh);
    const Pro pr = block_prologue(p, xs, ks, sh);
    if (pr.kind != 0) { handle_trivial(p, i, g, pr); return; }

    // Section IV.D: first candidate (in the Table 1 order) whose model SNR meets
    // the target; with a fixed quantiser the single candidate is taken.
    const unsigned feas = feasible_mask_pro(p, pr, ks, &s_feas);
    const int ci = feas ? __ffs(feas) - 1 : -1;

    if (ci < 0 && p.full64) {
        // Full precision in FP64, Eq. (1) over the window, rounded once to FP32.
        double* sd = reinterpret_cast<double*>(smem + dl.offS) + dl.padS;
        double* kd = reinterpret_cast<double*>(smem + dl.offKb);
        const int nkp = round_up(p.Nodd, kRd);
        for (int t = threadIdx.x; t < dl.padS; t += blockDim.x) sd[t - dl.padS] = 0.0;
        for (int t = threadIdx.x; t < dl.nS - dl.padS; t += blockDim.x) sd[t] = t < p.Wb ? (double)xs[t] : 0.0;
        for (int n = threadIdx.x; n < nkp; n += blockDim.x) kd[n] = (double)ktap(p, n);
        __syncthreads();
        // two outputs per thread when four would leave most threads idle, as the
        // packed form does (the same sums either way)
        if (g.hi - g.lo < 4 * (int)blockDim.x) full64_pass<2>(p, g, sd, kd, nkp);
        else full64_pass<kRd>(p, g, sd, kd, nkp);
        if (p.st && threadIdx.x == 0)
            write_stats(p, i, APX_BLK_FULL, nullptr, 0.f, pr.Ms, pro_sig2(pr, p.Wb),
                        __longlong_as_double(0x7ff0000000000000ll), 0.0);
        return;
    }
    if (ci < 0) {
        full_block_f32(p, i, g, pr, xs, smem);
        return;
    }

    const Cand& c = p.cand[ci];
    const float cs = compand_factor(c.S, pr.Ms);                        // Eq. (2)
    const float ck = compand_factor(c.K, ks.Mk);
    const double eps = LIT ? c.eps_l : ldexp(1.0, -c.b);
    // packed signal (its own region); packed outputs and the packed-tap chunk
    // overlay the FP32 window, which packing is the last to read
    double* sb = reinterpret_cast<double*>(smem + dl.offS);
    double* tb = reinterpret_cast<double*>(smem + dl.offT);
    double* kb = reinterpret_cast<double*>(smem + dl.offKb);
    const int nkp = round_up(c.nk, kRd);
    int nsb, Ls = 0;
    if (c.blk == APX_BLK_SYM) {
        nsb = p.Wb / 2;
        for (int m = threadIdx.x; m < nsb; m += blockDim.x) {          // Eq. (4)
            const double e = (double)compand(cs, xs[2 * m]);
            const double o = (double)compand(cs, xs[2 * m + 1]);
            sb[m] = __dadd_rn(e, __dmul_rn(eps, o));
        }
    } else {
        Ls = (p.Wb + c.M - 1) / c.M;
        nsb = Ls;
        for (int m = threadIdx.x; m < Ls; m += blockDim.x) {            // Eq. (7)
            double acc = 0.0, ep = 1.0;
            for (int q = 0; q < c.M; ++q) {
                const int t = m + q * Ls;
                if (t < p.Wb) acc = __dadd_rn(acc, __dmul_rn(ep, (double)compand(cs, xs[t])));
                ep = __dmul_rn(ep, eps);
            }
            sb[m] = acc;
        }
    }
    __syncthreads();  // the FP32 window is free from here on

    // Packed FP64 block convolution (Eq. 9 / Eq. 8): exact, since S_q, K_q keep
    // every scaled partial sum below 2^53,
    // taps staged a chunk at a time, partial sums kept in the output buffer.
    int olo, ohi, nr = 0;
    if (c.blk == APX_BLK_SYM) {
        olo = g.wstart; ohi = g.hi / 2;
    } else {
        nr = Ls + p.Nodd - 1;
        olo = max(0, g.lo - (c.M - 1) * Ls);
        ohi = min(g.hi, nr);
    }
    for (int n0 = 0; n0 < nkp; n0 += kKcD) {
        const int n1 = min(nkp, n0 + kKcD);
        if (n0 > 0) __syncthreads();  // every thread is done with the previous chunk
        for (int n = n0 + threadIdx.x; n < n1; n += blockDim.x)  // Eq. (5) / k~
            kb[n - n0] = LIT ? kbar_literal(p, c, ck, n) : (double)kbar_int(p, c, ck, n);
        __syncthreads();
        // two outputs per thread when four would leave most threads idle (a
        // W_block of 1024 has about 580 packed outputs): the FP64 pipe then sees
        // twice the warps; each output's sum runs in the same order either way
        if (ohi - olo < 4 * (int)blockDim.x) packed_conv_pass<2, LIT>(sb, nsb, kb, tb, n0, n1, olo, ohi);
        else packed_conv_pass<kRd, LIT>(sb, nsb, kb, tb, n0, n1, olo, ohi);
    }
    __syncthreads();

    // Unpack, inverse compand (Eq. 16), place (Eq. 17).
    if (threadIdx.x == 0) sh.bcast[0] = 1.0 / ((double)cs * (double)ck);
    __syncthreads();
    const float inv = (float)sh.bcast[0];
    auto Tat = [&](int m) { return scaled(tb[m], c.sc); };
    store_kept<false>(p, g, [&](int j, int& iv) {
        const long long rt = LIT                    ? unpack_sym_literal(c, j, g.wstart, tb)
                             : c.blk == APX_BLK_SYM ? unpack_sym(c, j, g.wstart, Tat)
                                                    : unpack_asym(c, j, Ls, nr, Tat);
        iv = (int)rt;
        return __fmul_rn(__ll2float_rn(rt), inv);
    });
    if (p.st && threadIdx.x == 0)
        write_stats(p, i, c.blk, &c, cs, pr.Ms, pro_sig2(pr, p.Wb),
                    snr_model_db(pro_sig2(pr, p.Wb), pr.Ms, ks.sig2k, ks.Mk, c.S, c.K), 0.0);
}

// The tensor-core candidate's kernel (APX_CORE_TC): each CTA takes kTcbBlocks
// consecutive blocks of one request, so that the kernel statistics, the tap
// slices and the tensor memory are set up once for all of them; every block
// then runs as in k_direct (window, statistics, Section IV.D selection), on
// the tensor cores when its candidate is admitted, else in FP32.
template <bool BATCH>
__global__ void __launch_bounds__(kDirectThreads, 4) k_direct_tc(const Params p0, const BatchTab bt) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ unsigned s_feas;
    __shared__ Params sp;
    __shared__ __align__(8) unsigned long long s_bar;  // completion of a block's MMAs
    __shared__ uint32_t s_tmem;
    const long long c0 = BATCH ? batch_enter(bt, sp) : (long long)blockIdx.x;
    const Params& p = BATCH ? sp : p0;
    const DirectLayout& dl = p.dl;
    float* xs = reinterpret_cast<float*>(smem) + dl.padF;
    for (int t = threadIdx.x; t < dl.padF; t += blockDim.x) xs[t - dl.padF] = 0.f;
    for (int t = threadIdx.x; t < kRf; t += blockDim.x) xs[p.Wb + t] = 0.f;
    const KStats ks = kernel_stats(p, sh);  // Section IV kernel initialisation, once for the CTA's blocks
    const TcBufs tb = tc_bufs(p, smem);
    const bool live_k = !ks.bad && ks.Mk > 0.f;
    const float ck = live_k ? compand_factor(p.cand[0].K, ks.Mk) : 0.f;
    if (live_k) tc_prepare_taps(p, tb, ck, smem);
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&s_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) tmem_alloc(&s_tmem, 64);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    uint32_t phase = 0;
    for (int u = 0; u < kTcbBlocks; ++u) {
        const long long i = c0 * kTcbBlocks + u;
        if (i >= p.P) break;  // the same for the whole CTA
        const BlockGeom g = block_geom(p, i);
        load_window(p, g, xs);
        const Pro pr = block_prologue(p, xs, ks, sh);
        if (pr.kind != 0) {
            handle_trivial(p, i, g, pr);
        } else if (!feasible_mask_pro(p, pr, ks, &s_feas)) {
            full_block_f32(p, i, g, pr, xs, smem);
        } else {
            tc_block_body(p, i, g, p.cand[0], ks, pr, ck, xs, tb, tmem, smem_u32(&s_bar), phase, sh);
            phase ^= 1u;
        }
        __syncthreads();  // the window's space is read before the next block's window lands
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_free(tmem, 64);
}

template <typename K>
static cudaError_t set_smem_attr(K kern, int* attr_dev) {
    int dev;
    cudaGetDevice(&dev);
    if (*attr_dev == dev) return cudaSuccess;
    // the largest dynamic shared memory beside this kernel's static shared memory
    // (227 KB per CTA in all; layouts never ask for more than kMaxSmem)
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    const int dyn = 227 * 1024 - (int)fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn < kMaxSmem ? dyn : kMaxSmem);
    if (e == cudaSuccess) *attr_dev = dev;
    return e;
}
template <bool BATCH, bool LIT>
static cudaError_t direct_attrs() {
    static int attr_dev = -1;
    return set_smem_attr(k_direct<BATCH, LIT>, &attr_dev);
}
template <bool BATCH>
static cudaError_t direct_tc_attrs() {
    static int attr_dev = -1;
    return set_smem_attr(k_direct_tc<BATCH>, &attr_dev);
}

// the tensor-core kernel when the call's one candidate is the tensor-core one
static bool tc_call(const Params& p) { return p.ncand == 1 && p.cand[0].blk == APX_BLK_TC; }

cudaError_t launch_direct(const Params& p, size_t smem, cudaStream_t st) {
    const bool lit = p.ncand == 1 && p.cand[0].literal, tc = tc_call(p);
    cudaError_t e = lit ? direct_attrs<false, true>() : (tc ? direct_tc_attrs<false>() : direct_attrs<false, false>());
    if (e != cudaSuccess) return e;
    if (p.P <= 0) return cudaSuccess;
    const BatchTab none = {nullptr, nullptr, 0};
    const dim3 block(kDirectThreads);
    if (lit) return launch_k(k_direct<false, true>, dim3((unsigned)p.P), block, smem, st, false, p, none);
    if (tc) return launch_k(k_direct_tc<false>, dim3((unsigned)tcb_ctas(p.P)), block, smem, st, false, p, none);
    return launch_k(k_direct<false, false>, dim3((unsigned)p.P), block, smem, st, false, p, none);
}

// Batched groups keep tensor-core requests apart from the others; their CTA
// table counts tcb_ctas(P) CTAs per request.
cudaError_t launch_direct_batch(const Params& any, const BatchTab& bt, int ctas, size_t smem, cudaStream_t st) {
    const bool tc = tc_call(any);
    cudaError_t e = tc ? direct_tc_attrs<true>() : direct_attrs<true, false>();
    if (e != cudaSuccess) return e;
    if (ctas <= 0) return cudaSuccess;
    if (tc) return launch_k(k_direct_tc<true>, dim3(ctas), dim3(kDirectThreads), smem, st, false, any, bt);
    return launch_k(k_direct<true, false>, dim3(ctas), dim3(kDirectThreads), smem, st, false, any, bt);
}

}  // namespace apx
