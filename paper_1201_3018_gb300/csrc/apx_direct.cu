// apx_direct.cu -- fused per-block kernel of the time-domain (direct) core.
//
// One launch per call, one CTA per overlap-save block: load the W_block window,
// kernel and block statistics, Section IV.D selection, companding (Eq. 2) and
// packing (Eqs. 4, 5, 7) of block and taps into shared memory, the packed FP64
// convolution (Eqs. 8-9) with a register sliding window, digit extraction
// (Eqs. 11-15), inverse companding (Eq. 16) and the Eq. (17) store.  Blocks
// without an admissible packing run the FP32 full-precision convolution in the
// same CTA.
#include "apx_block.cuh"
#include "apx_launch.h"

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

// LIT: the paper-literal symmetric form (APX_LITERAL, single calls only) in
// an instantiation of its own, so that the other kernels are compiled as if
// it did not exist.
template <bool BATCH, bool LIT>
__global__ void __launch_bounds__(kDirectThreads) k_direct(const Params p0, const BatchTab bt) {
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
    const unsigned feas = feasible_mask(p, pr.sig2, pr.Ms, ks.sig2k, ks.Mk, &s_feas);
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
        const int nout = g.hi - g.lo;
        for (int ch = threadIdx.x; ch * kRd < nout; ch += blockDim.x) {
            const int j0 = g.lo + ch * kRd;
            double acc[kRd];
            conv_f64_full<kRd>(sd, kd, nkp, j0, acc);
#pragma unroll
            for (int r = 0; r < kRd; ++r) {
                const int j = j0 + r;
                const long long o = g.start + j;
                if (j < g.hi && o >= 0 && o < p.out_len) {
                    p.r[o] = __double2float_rn(acc[r]);
                    if (p.rq) p.rq[o] = 0;
                }
            }
        }
        write_stats(p, i, APX_BLK_FULL, nullptr, 0.f, pr.Ms, pr.sig2, __longlong_as_double(0x7ff0000000000000ll), 0.0);
        return;
    }
    if (ci < 0) {
        // Full precision (FP32), Eq. (1) over the window, taps staged in
        // shared memory a chunk at a time; a later chunk continues the sums
        // the thread stored for its outputs.
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
                float acc[kRf];
#pragma unroll
                for (int r = 0; r < kRf; ++r) {
                    const long long o = g.start + j0 + r;
                    acc[r] = (n0 > 0 && j0 + r < g.hi && o >= 0 && o < p.out_len) ? p.r[o] : 0.f;
                }
                conv_f32<kRf>(xs, kf, n0, n1, j0, acc);
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
        write_stats(p, i, APX_BLK_FULL, nullptr, 0.f, pr.Ms, pr.sig2, __longlong_as_double(0x7ff0000000000000ll), 0.0);
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
        for (int ch = threadIdx.x; olo + ch * kRd < ohi; ch += blockDim.x) {
            const int j0 = olo + ch * kRd;
            double acc[kRd];
#pragma unroll
            for (int r = 0; r < kRd; ++r) acc[r] = (n0 > 0 && j0 + r < ohi) ? tb[j0 + r] : 0.0;
            if (LIT) conv_f64<kRd, true>(sb, nsb, kb, n0, n1, j0, acc);
            else conv_f64<kRd, false>(sb, nsb, kb, n0, n1, j0, acc);
#pragma unroll
            for (int r = 0; r < kRd; ++r)
                if (j0 + r < ohi) tb[j0 + r] = acc[r];
        }
    }
    __syncthreads();

    // Unpack, inverse compand (Eq. 16), place (Eq. 17).
    if (threadIdx.x == 0) sh.bcast[0] = 1.0 / ((double)cs * (double)ck);
    __syncthreads();
    const float inv = (float)sh.bcast[0];
    auto Tat = [&](int m) { return scaled(tb[m], c.sc); };
    for (int j = g.lo + threadIdx.x; j < g.hi; j += blockDim.x) {
        const long long o = g.start + j;
        if (o < 0 || o >= p.out_len) continue;
        long long rt = LIT                      ? unpack_sym_literal(c, j, g.wstart, tb)
                       : c.blk == APX_BLK_SYM ? unpack_sym(c, j, g.wstart, Tat)
                                              : unpack_asym(c, j, Ls, nr, Tat);
        p.r[o] = __fmul_rn(__ll2float_rn(rt), inv);
        if (p.rq) p.rq[o] = (int)rt;
    }
    if (threadIdx.x == 0)
        write_stats(p, i, c.blk, &c, cs, pr.Ms, pr.sig2, snr_model_db(pr.sig2, pr.Ms, ks.sig2k, ks.Mk, c.S, c.K), 0.0);
}

template <bool BATCH, bool LIT>
static cudaError_t direct_attrs() {
    static int attr_dev = -1;
    int dev;
    cudaGetDevice(&dev);
    if (attr_dev == dev) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_direct<BATCH, LIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e == cudaSuccess) attr_dev = dev;
    return e;
}

cudaError_t launch_direct(const Params& p, size_t smem, cudaStream_t st) {
    const bool lit = p.ncand == 1 && p.cand[0].literal;
    cudaError_t e = lit ? direct_attrs<false, true>() : direct_attrs<false, false>();
    if (e != cudaSuccess) return e;
    if (p.P <= 0) return cudaSuccess;
    const BatchTab none = {nullptr, nullptr, 0};
    if (lit) return launch_k(k_direct<false, true>, dim3((unsigned)p.P), dim3(kDirectThreads), smem, st, false, p, none);
    return launch_k(k_direct<false, false>, dim3((unsigned)p.P), dim3(kDirectThreads), smem, st, false, p, none);
}

cudaError_t launch_direct_batch(const Params& any, const BatchTab& bt, int ctas, size_t smem, cudaStream_t st) {
    cudaError_t e = direct_attrs<true, false>();
    if (e != cudaSuccess) return e;
    if (ctas <= 0) return cudaSuccess;
    return launch_k(k_direct<true, false>, dim3(ctas), dim3(kDirectThreads), smem, st, false, any, bt);
}

}  // namespace apx
