// apx_tc.cu -- time-domain convolution core on the tensor cores, for a bank of
// kernels sharing one input (the filterbank).
//
// The paper's layer around the core is kept: each block of outputs quantizes
// the input window it depends on with its own companding factor (Eq. 2), the
// kernels are companded once, the convolution of the small integers is exact,
// and the result is scaled back (Eq. 16).  What replaces the FP64 packing is
// the arithmetic: the integers (|q| <= 2048) are exact in FP16, their products
// exact in FP32, and FP32 accumulation stays exact while every partial sum is
// at most 2^24 in magnitude, which N * S_q * K_q <= 2^24 guarantees.
//
// Eq. (1) as a matrix product.  With P output phases per row,
//   y_f[t0 + q P + p] = sum_j A[q][j] B[j][(f, p)],
//   A[q][j]      = s~[t0 - N + 1 + q P + j]          (Toeplitz in q, j)
//   B[j][(f, p)] = k~_f[p + N - 1 - j]  (zero outside [0, N)),
// j in [0, K), K = N + P - 1.  Rows q are time (M = 128 per tile), columns are
// G = 256 / P kernels times P phases (N_gemm = 256).
//
// The Toeplitz operand without expansion: the quantized window of each block
// is stored as a matrix with rows of P samples, S[r][c] = seg[r P + c]; then
// A[q][j] = S[q + j / P][j % P], so the 64-wide K slice j0..j0+63 (P a
// multiple of 64) is the plain 128 x 64 box of S at (row j0 / P, column j0 % P),
// one TMA load.
//
// Kernels:
//   k_tc_quant  one CTA per block: ||window||_inf, c_s, companding into the
//               block's FP16 segment (Eq. 2), c_s to the block table.
//   k_tc_kern   one CTA per kernel: c_k, companding, the Toeplitz columns of B
//               (K-major, FP16 or FP8), and the Eq. (16) factors
//               fl32(1 / (c_s c_k)) of the kernel for every block.
//   k_tc_mma    persistent, one CTA per SM over the (block, kernel group)
//               tiles: warp 0 streams operands with TMA into a shared-memory
//               ring, warp 1 issues tcgen05.mma (M 128, N 256, K 16 in FP16
//               or 32 in FP8, FP32 accumulators in tensor memory,
//               double-buffered), warps 2-5 read the accumulators back with
//               tcgen05.ld, scale them (Eq. 16) and write them out with TMA
//               tensor stores.
//
// With P = 64 a row of S is exactly one 128-byte swizzle row, and the A slice
// of K step kt is rows kt .. kt+127 of S: the whole A operand of a tile (its
// 128 + ktiles - 1 rows) is loaded once, and each K step's descriptor starts
// kt rows further in (the swizzle phase goes in the descriptor's base-offset
// field).  Only B streams through the ring.  For P = 128 or 256 both operands
// stream, one 128 x 64 A box per K step.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstdint>

#include "apx_tc.h"
#include "apx_umma.cuh"

namespace apx {

namespace {

constexpr int kTcEpiWarps = 4;   // one per tensor-memory lane quarter (warp % 4 selects the quarter)
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;  // warp 0 TMA, warp 1 MMA, warps 2.. epilogue
constexpr uint32_t kTcABytes = kTcM * 128;  // a K slice: one 128-byte row per operand row
constexpr uint32_t kTcBBytes = kTcN * 128;
constexpr uint32_t kTcTmemCols = kTcN;
// Output staging per epilogue warp: kTcStgBufs buffers of kTcStgChunks 4 KB
// chunks (32 rows x 32 FP32 outputs); a buffer's chunks are written back by one
// bulk tensor store, and a warp refills a buffer while its other buffers'
// stores are still reading.
#ifndef APX_TC_STG_BUFS
#define APX_TC_STG_BUFS 1
#endif
#ifndef APX_TC_STG_CHUNKS
#define APX_TC_STG_CHUNKS 2
#endif
constexpr int kTcStgBufs = APX_TC_STG_BUFS;
constexpr int kTcStgChunks = APX_TC_STG_CHUNKS;
static_assert(kTcStgChunks == 1 || kTcStgChunks == 2 || kTcStgChunks == 4, "chunks per store divide P / 32");
constexpr uint32_t kTcStgWarp = (uint32_t)(kTcStgBufs * kTcStgChunks) * 4096u;
constexpr uint32_t kTcStageOut = kTcEpiWarps * kTcStgWarp;
constexpr int kTcABoxRows = 64;                     // resident A: TMA box rows
constexpr uint32_t kTcABoxBytes = kTcABoxRows * 128;
constexpr uint32_t kTcIdesc = umma_idesc_f16(kTcM, kTcN);  // FP16 operands, FP32 accumulators, M 128, N 256

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    umma_f16_id(d_tmem, adesc, bdesc, kTcIdesc, accum);
}

// The same with FP8 E4M3 operands (kind::f8f6f4: format code 0 = E4M3 in the same
// descriptor fields, K = 32 per instruction, still 32 bytes of each row).
__device__ __forceinline__ void umma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accum)
        : "memory");
}

// Bulk tensor store of a staged shared-memory box (one bulk group per call).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, uint32_t src, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n\t"
        "cp.async.bulk.commit_group;" ::"l"(reinterpret_cast<uint64_t>(map)),
        "r"(x), "r"(y), "r"(z), "r"(src)
        : "memory");
}
// The same through the 4-D map of whole rows: box (32 phases, 32 rows, chunks, 1).
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, uint32_t src, int x, int y, int z, int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n\t"
        "cp.async.bulk.commit_group;" ::"l"(reinterpret_cast<uint64_t>(map)),
        "r"(x), "r"(y), "r"(z), "r"(w), "r"(src)
        : "memory");
}
// The bulk stores of this thread, all but the N most recent, have finished
// reading shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// ... and their writes are performed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ float block_max_abs(const float* x, int64_t lo, int64_t hi, int64_t L, bool* bad,
                                               float* red) {
    float m = 0.f;
    bool nf = false;
    for (int64_t g = lo + threadIdx.x; g < hi; g += blockDim.x) {
        if (g < 0 || g >= L) continue;
        const float v = fabsf(x[g]);
        if (!(v <= 3.402823466e38f)) nf = true;  // NaN or Inf
        else m = fmaxf(m, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        nf |= __shfl_xor_sync(0xffffffffu, (int)nf, o) != 0;
    }
    __shared__ int nfs;
    if (threadIdx.x == 0) nfs = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = m;
        if (nf) nfs = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
        red[0] = t;
    }
    __syncthreads();
    const float r = red[0];
    *bad = nfs != 0;
    __syncthreads();
    return r;
}

// Operand element types: FP16, or FP8 E4M3 when S_q, K_q <= 16 (every
// companded integer is then exact in E4M3, and the tensor core takes twice the
// K per instruction).  from_int converts an exact small integer.
template <typename E> struct TcElem;
template <> struct TcElem<__half> {
    static __device__ __forceinline__ __half from_int(float q) { return __float2half_rn(q); }
};
template <> struct TcElem<uint8_t> {
    static __device__ __forceinline__ uint8_t from_int(float q) {
        return (uint8_t)__nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
    }
};

// Eq. (2) on the block's window, written as the block's segment (FP16 or FP8)
// seg[u] = s~[t0 - N + 1 + u]; entries past the window (u >= T + N - 1) are 0.
// One coalesced pass stages the window in shared memory and finds its
// maximum (one integer reduction of the magnitude bits: NaN lies above inf);
// the companding then reads shared memory and writes 8-element vectors.
constexpr int kRun = 8;
template <typename E>
__global__ void __launch_bounds__(256) k_tc_quant(const float* __restrict__ s, int64_t L, TcGeom g, int Sq,
                                                  E* __restrict__ seg, float* __restrict__ cs_tab,
                                                  float* __restrict__ cs_out, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) float win[];  // nwin window samples, padded to a multiple of kRun
    __shared__ int red[8];
    const int64_t b = blockIdx.x;
    const int64_t lo = b * g.T - g.N + 1;
    const int nwin = g.T + g.N - 1;
    const int64_t nseg = g.seg_rows * g.P;
    int mb = 0;
    for (int u0 = threadIdx.x; u0 < nwin; u0 += kRun * blockDim.x) {
        float v[kRun];
#pragma unroll
        for (int i = 0; i < kRun; ++i) {
            const int u = u0 + i * blockDim.x;
            const int64_t gi = lo + u;
            v[i] = (u < nwin && gi >= 0 && gi < L) ? __ldg(s + gi) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < kRun; ++i) {
            const int u = u0 + i * blockDim.x;
            if (u < nwin) win[u] = v[i];
            mb = max(mb, __float_as_int(v[i]) & 0x7fffffff);
        }
    }
    for (int u = nwin + threadIdx.x; u < (nwin + kRun - 1) / kRun * kRun; u += blockDim.x) win[u] = 0.f;
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mb;
    __syncthreads();
    int M = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) M = max(M, red[w]);
    const bool bad = M > 0x7f800000;  // a NaN
    const float Mf = __int_as_float(M);
    float c = 0.f;
    if (bad || Mf > 3.402823466e38f) c = __int_as_float(0x7fc00000);
    else if (Mf > 0.f) c = __fdiv_rn((float)Sq, Mf);
    const bool live = Mf > 0.f && Mf <= 3.402823466e38f && !bad;
    E* out = seg + b * nseg;
    for (int64_t u0 = (int64_t)threadIdx.x * kRun; u0 < nseg; u0 += (int64_t)blockDim.x * kRun) {
        __align__(16) E h[kRun];
        if (live && u0 < nwin) {
            const float4 p = *reinterpret_cast<const float4*>(win + u0);
            const float4 q = *reinterpret_cast<const float4*>(win + u0 + 4);
            const float v[kRun] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w};
#pragma unroll
            for (int i = 0; i < kRun; ++i)
                h[i] = TcElem<E>::from_int(u0 + i < nwin ? rintf(__fmul_rn(c, v[i])) : 0.f);
        } else {
#pragma unroll
            for (int i = 0; i < kRun; ++i) h[i] = TcElem<E>::from_int(0.f);
        }
        // nseg % 8 == 0: one 16-byte (FP16) or 8-byte (FP8) store
        if (sizeof(E) == 2) *reinterpret_cast<uint4*>(out + u0) = *reinterpret_cast<const uint4*>(h);
        else *reinterpret_cast<uint2*>(out + u0) = *reinterpret_cast<const uint2*>(h);
    }
    if (threadIdx.x == 0) {
        if (bad || Mf > 3.402823466e38f) atomicOr(status, 1u);
        cs_tab[b] = c;
        if (cs_out) cs_out[b] = c;
    }
}

// Eq. (2) on kernel f and its Toeplitz columns: row n = group * 256 + fl * P + p
// of the K-major B operand holds k~_f[p + N - 1 - j] at column j.  CTA
// (f, y) writes the rows of phases p = y, y + gridDim.y, ...
//
// CTA (f, 0) also writes fl32(1 / (c_s c_k)) of kernel f for every block b to
// inv_tab[b * ngroups * G + f] (0 for an all-zero or non-finite window or
// kernel, and for the zero columns past F): the epilogue's Eq. (16) factor,
// computed once here in FP64 (c_s c_k is exact in FP64) instead of per tile.
// The block table cs_tab is complete: k_tc_quant runs before on the stream.
template <typename E>
__global__ void __launch_bounds__(256) k_tc_kern(const float* __restrict__ kb, TcGeom g, int Kq,
                                                 E* __restrict__ bt, const float* __restrict__ cs_tab,
                                                 float* __restrict__ inv_tab, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char tc_kern_smem[];
    E* kq = reinterpret_cast<E*>(tc_kern_smem);  // kq[n + 64] = k~[n], zero outside [0, N)
    __shared__ float red[8];
    const int f = blockIdx.x;  // 0 .. ngroups * G - 1 (past F: zero columns)
    const int kpadded = g.N + 128;
    float c = 0.f;
    bool bad = false;
    if (f < g.F) {
        const float* k = kb + (int64_t)f * g.N;
        const float M = block_max_abs(k, 0, g.N, g.N, &bad, red);
        if (!bad && M > 0.f) c = __fdiv_rn((float)Kq, M);
        for (int n = threadIdx.x; n < kpadded; n += blockDim.x) {
            const int t = n - 64;
            kq[n] = TcElem<E>::from_int((c > 0.f && t >= 0 && t < g.N) ? rintf(__fmul_rn(c, k[t])) : 0.f);
        }
        if (threadIdx.x == 0 && blockIdx.y == 0 && bad) atomicOr(status, 1u);
    } else {
        for (int n = threadIdx.x; n < kpadded; n += blockDim.x) kq[n] = TcElem<E>::from_int(0.f);
    }
    if (blockIdx.y == 0) {
        const int64_t gs = (int64_t)g.ngroups * g.G;
        for (int64_t b = threadIdx.x; b < g.nb; b += blockDim.x) {
            const float cs = cs_tab[b];
            inv_tab[b * gs + f] = (cs > 0.f && c > 0.f && !bad) ? (float)(1.0 / ((double)cs * (double)c)) : 0.f;
        }
    }
    __syncthreads();
    const int grp = f / g.G, fl = f % g.G;
    E* rows = bt + ((int64_t)grp * kTcN + (int64_t)fl * g.P) * g.Kpad;
    const int half_row = g.Kpad / 2;
    for (int p = blockIdx.y; p < g.P; p += gridDim.y) {
        E* row = rows + (int64_t)p * g.Kpad;
        for (int jj = threadIdx.x; jj < half_row; jj += blockDim.x) {
            const int j = 2 * jj;
            // taps n = p + N - 1 - j and n - 1; past the band they read the zero pad
            int n0 = p + g.N - 1 - j;
            n0 = n0 < -64 ? -64 : (n0 > g.N + 63 ? g.N + 63 : n0);
            const int n1 = n0 - 1 < -64 ? -64 : n0 - 1;
            row[j] = kq[n0 + 64];
            row[j + 1] = kq[n1 + 64];
        }
    }
}

// Epilogue of one tile for one warp (TMEM lane quarter lq): read the warp's
// 32 accumulator rows in 32-column chunks (chunk ch is columns 32 ch .. 32 ch
// + 31, kernel fl = ch / (P / 32)), the load of the next chunk in flight while
// this one is processed; scale by the block's and kernel's (c_s c_k)^-1
// (Eq. 16); stage the 32 x 32 chunk in shared memory in the 128-byte swizzled
// layout (16-byte slot i of row r at r * 128 + ((i ^ (r & 7)) * 16):
// conflict-free writes).  g.stg_ch consecutive chunks of one kernel fill a
// staging buffer, written by one TMA store of the box (g.stg_ch = 1: columns c
// .. c + 31 of P, time rows row0 .. row0 + 31, kernel f, through the 3-D map;
// otherwise the 4-D map's sub-rows of 32 phases, so that 2 or 4 chunks make
// whole 256- or 512-byte rows).  The warp's kTcStgBufs buffers rotate (sg
// counts the warp's stores).  The maps cover the out_len / P whole rows of each
// kernel, so TMA drops rows past them; the one partial row at the end (out_len
// % P outputs) is written by its lane with plain stores.
__device__ __forceinline__ void epilogue_tile(const TcGeom& g, const CUtensorMap* tmY, int64_t blk, int grp,
                                              uint32_t acc0, uint32_t stg, int lane, int lq,
                                              const float* __restrict__ inv_tab, float* __restrict__ y,
                                              int32_t* __restrict__ yq, unsigned* status, int& sg) {
    const int64_t row0 = blk * kTcM + lq * 32;  // first time row of this warp's quarter
    const int64_t rows_full = g.out_len / g.P;  // rows the output map covers
    const int64_t tail_row = (g.out_len % g.P) ? rows_full : -1;
    const bool stores = row0 < rows_full;       // the same for every tile after the first that has none
    const uint32_t acc = acc0 + ((uint32_t)(lq * 32) << 16);
    const int nf = g.F - grp * g.G < g.G ? g.F - grp * g.G : g.G;  // kernels of this group
    const float inv_l = lane < nf ? inv_tab[blk * (int64_t)(g.ngroups * g.G) + grp * g.G + lane] : 0.f;
    const int cpk = g.P / 32;  // chunks per kernel
    const int chg = g.stg_ch;  // chunks per store (divides cpk)
    const int nchunks = nf * cpk;
    uint32_t rn[32];
    if (!APX_IN_BOUNDS(nchunks * 32 <= kTcN && chg <= kTcStgChunks && cpk % chg == 0, status)) return;
    tmem_ld32_nowait(acc, rn);
    for (int ch = 0; ch < nchunks; ++ch) {
        const int fl = ch / cpk, c = (ch - fl * cpk) * 32;
        const int f = grp * g.G + fl;
        const int sub = (ch - fl * cpk) % chg;  // position of the chunk in its store
        uint32_t r[32];
        tmem_wait_ld(rn);
#pragma unroll
        for (int i = 0; i < 32; ++i) r[i] = rn[i];
        if (ch + 1 < nchunks) tmem_ld32_nowait(acc + (uint32_t)(32 * (ch + 1)), rn);
        const float inv = __shfl_sync(0xffffffffu, inv_l, fl);
        const uint32_t buf = stg + (uint32_t)(sg % kTcStgBufs) * (uint32_t)(kTcStgChunks * 4096);
        if (sub == 0) {
            // this buffer's previous store has read it (with no store in this
            // tile, wait for every store: the rotation no longer counts)
            if (lane == 0) {
                if (stores) bulk_wait_read<kTcStgBufs - 1>();
                else bulk_wait_read<0>();
            }
            __syncwarp();
        }
        const uint32_t cb = buf + (uint32_t)sub * 4096u;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = __fmul_rn(__uint_as_float(r[4 * i + e]), inv);
            asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(
                             cb + (uint32_t)lane * 128u + (uint32_t)((i ^ (lane & 7)) * 16)),
                         "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3])
                         : "memory");
        }
        if (sub == chg - 1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the bulk copy
            __syncwarp();
            if (lane == 0 && stores) {
                if (chg == 1) tma_store_3d(tmY, buf, c, (int)row0, f);
                else tma_store_4d(tmY, buf, 0, (int)row0, c / 32 - (chg - 1), f);
            }
            ++sg;
        }
        const int64_t t0 = (row0 + lane) * g.P + c;  // this lane's first output
        if (row0 + lane == tail_row) {
            float* yf = y + (int64_t)f * g.ldy;
            for (int i = 0; i < 32 && t0 + i < g.out_len; ++i) yf[t0 + i] = __fmul_rn(__uint_as_float(r[i]), inv);
        }
        if (yq && t0 < g.out_len) {
            // integer outputs (a test aid): straight from the row
            int32_t* qf = yq + (int64_t)f * g.ldy;
            for (int i = 0; i < 32 && t0 + i < g.out_len; ++i) qf[t0 + i] = __float2int_rn(__uint_as_float(r[i]));
        }
    }
}

// Persistent: CTA c takes tiles u = c, c + gridDim.x, ...; tile u is block
// u / ngroups, kernel group u % ngroups (the groups of one block run side by
// side, so a block's segment comes from DRAM once).  The shared-memory ring
// runs across tiles; the accumulator is double-buffered in tensor memory
// (2 x 256 columns) so that the epilogue of one tile overlaps the MMAs of the
// next.
template <bool RESIDENT_A, bool F8>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_mma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             const __grid_constant__ CUtensorMap tmY, const TcGeom g, const float* __restrict__ inv_tab,
             float* __restrict__ y, int32_t* __restrict__ yq, unsigned* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kTcMaxStages], empty_bar[kTcMaxStages], accf_bar[2], acce_bar[2],
        afull_bar[2], aempty_bar[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh, issued_sh;
    const uint32_t base = (smem_u32(tc_smem_raw) + 1023u) & ~1023u;
    // [output staging, kTcStgWarp per epilogue warp][A buffer 0][A buffer 1][B stages] (RESIDENT_A)
    // [output staging][B stage, A stage] x stages (otherwise)
    const uint32_t abuf0 = base + kTcStageOut;
    const uint32_t ring = RESIDENT_A ? abuf0 + 2u * (uint32_t)g.abuf_bytes : abuf0;
    const uint32_t stage_bytes = RESIDENT_A ? kTcBBytes : kTcABytes + kTcBBytes;
    const int S = g.stages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nsets = g.nb * g.ngroups;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&accf_bar[a]), 1);
            mbar_init(smem_u32(&acce_bar[a]), kTcEpiWarps);  // one arrival per epilogue warp
            mbar_init(smem_u32(&afull_bar[a]), 1);
            mbar_init(smem_u32(&aempty_bar[a]), 1);
        }
        abort_sh = 0;
        issued_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(2 * kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int it = 0, local = 0;
            for (int64_t u = blockIdx.x; u < nsets && !*(volatile int*)&abort_sh; u += gridDim.x, ++local) {
                const int64_t blk = u / g.ngroups;
                const int grp = (int)(u % g.ngroups);
                const int arow0 = (int)(blk * g.seg_rows);
                if (RESIDENT_A) {
                    const int ab = local & 1;
                    if (local >= 2 &&
                        !mbar_wait(smem_u32(&aempty_bar[ab]), (uint32_t)((local >> 1) - 1) & 1u, false)) {
                        atomicOr(status, 2u);
                        abort_sh = 1;
                        break;
                    }
                    const uint32_t afb = smem_u32(&afull_bar[ab]);
                    const uint32_t abase = abuf0 + (uint32_t)ab * (uint32_t)g.abuf_bytes;
                    mbar_expect_tx(afb, (uint32_t)g.abuf_bytes);
                    for (int r = 0; r < g.a_loads; ++r)
                        tma_load_2d(abase + (uint32_t)r * kTcABoxBytes, &tmA, 0, arow0 + r * kTcABoxRows, afb);
                }
                for (int kt = 0; kt < g.ktiles; ++kt, ++it) {
                    const int s = it % S;
                    const uint32_t ph = (uint32_t)(it / S) & 1u;
                    if (it >= S && !mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, false)) {
                        atomicOr(status, 2u);
                        abort_sh = 1;
                        break;
                    }
                    if (*(volatile int*)&abort_sh) break;
                    const uint32_t st = ring + (uint32_t)s * stage_bytes;
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    const int j0 = kt * g.ktile;
                    mbar_expect_tx(fb, stage_bytes);
                    if (!RESIDENT_A) tma_load_2d(st + kTcBBytes, &tmA, j0 % g.P, arow0 + j0 / g.P, fb);
                    tma_load_2d(st, &tmB, j0, grp * kTcN, fb);
                    issued_sh = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int it = 0, local = 0;
            for (int64_t u = blockIdx.x; u < nsets; u += gridDim.x, ++local) {
                const int a = local & 1;
                const uint32_t acc = tmem + (uint32_t)(a * kTcTmemCols);
                if (local >= 2 &&
                    (!mbar_wait(smem_u32(&acce_bar[a]), (uint32_t)((local >> 1) - 1) & 1u, false) ||
                     *(volatile int*)&abort_sh)) {
                    atomicOr(status, 2u);
                    abort_sh = 1;
                    break;
                }
                if (RESIDENT_A && !mbar_wait(smem_u32(&afull_bar[a]), (uint32_t)(local >> 1) & 1u, false)) {
                    atomicOr(status, 2u);
                    abort_sh = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t abase = abuf0 + (uint32_t)a * (uint32_t)g.abuf_bytes;
                bool ok = true;
                for (int kt = 0; kt < g.ktiles; ++kt, ++it) {
                    const int s = it % S;
                    const uint32_t ph = (uint32_t)(it / S) & 1u;
                    if (!mbar_wait(smem_u32(&full_bar[s]), ph, false) || *(volatile int*)&abort_sh) {
                        atomicOr(status, 2u);
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sb = ring + (uint32_t)s * stage_bytes;
                    const uint32_t sa = RESIDENT_A ? abase + (uint32_t)kt * 128u : sb + kTcBBytes;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {  // four 32-byte K steps per 128-byte row
                        if (F8) umma_f8(acc, sdesc_sw128(sa + 32u * k), sdesc_sw128(sb + 32u * k), (kt | k) != 0);
                        else umma_f16(acc, sdesc_sw128(sa + 32u * k), sdesc_sw128(sb + 32u * k), (kt | k) != 0);
                    }
                    umma_commit(smem_u32(&empty_bar[s]));
                }
                umma_commit(smem_u32(&accf_bar[a]));  // this tile's MMAs done
                if (RESIDENT_A) umma_commit(smem_u32(&aempty_bar[a]));
                if (!ok) break;
            }
        }
    } else {  // epilogue: warps 2-5, tensor-memory lane quarter warp % 4
        const int lq = warp & 3;
        int local = 0, sg = 0;
        for (int64_t u = blockIdx.x; u < nsets; u += gridDim.x, ++local) {
            const int a = local & 1;
            const bool ok = mbar_wait(smem_u32(&accf_bar[a]), (uint32_t)(local >> 1) & 1u, true);
            tc_fence_after();
            __syncwarp();
            if (!ok || *(volatile int*)&abort_sh) {
                if (lane == 0) atomicOr(status, ok ? 0u : 2u);
                break;
            }
            const int64_t blk = u / g.ngroups;
            const int grp = (int)(u % g.ngroups);
            epilogue_tile(g, &tmY, blk, grp, tmem + (uint32_t)(a * kTcTmemCols), base + (uint32_t)(warp - 2) * kTcStgWarp,
                          lane, lq, inv_tab, y, yq, status, sg);
            // every tcgen05.ld of this buffer has completed (wait::ld): hand it back
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[a]))
                                        : "memory");
        }
        if (lane == 0) bulk_wait_all();  // the output stores are done before the CTA exits
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0 && lane == 0 && abort_sh) {
        // TMA loads issued but never consumed: let them land before the CTA exits
        for (int i = issued_sh - S; i < issued_sh; ++i)
            if (i >= 0) (void)mbar_wait(smem_u32(&full_bar[i % S]), (uint32_t)(i / S) & 1u, true);
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTcTmemCols)
                     : "memory");
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D FP16 map: inner extent `inner` (contiguous), `rows` rows `pitch` bytes
// apart, box 64 x box_rows, 128-byte swizzle.
bool encode_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t pitch, uint32_t box_rows,
               int esize) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {pitch};
    const cuuint32_t box[2] = {(cuuint32_t)(128 / esize), box_rows};  // one 128-byte row
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The FP32 outputs as a map for the epilogue's stores, 128-byte swizzle.  One
// chunk per store: 3-D, P phases (inner), the out_len / P whole rows of a
// kernel (row pitch P floats), F kernels (pitch ldy floats); box 32 x 32 x 1.
// Several: 4-D, 32 phases (inner), rows (pitch P floats), P / 32 sub-rows
// (pitch 32 floats), F kernels; box 32 x 32 x stg_ch x 1, so that the staged
// chunks of a store are [sub-row][row][32 phases] in shared memory and each
// 128-byte line keeps the swizzle phase of its row.  With fewer than P outputs
// there is no whole row: the map gets one row and the epilogue stores nothing
// through it.
bool encode_out(CUtensorMap* m, float* y, const TcGeom& g) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const int64_t rows = g.out_len / g.P;
    const cuuint64_t nrows = (cuuint64_t)(rows > 0 ? rows : 1);
    if (g.stg_ch == 1) {
        const cuuint64_t dims[3] = {(cuuint64_t)g.P, nrows, (cuuint64_t)g.F};
        const cuuint64_t strides[2] = {(cuuint64_t)g.P * 4u, (cuuint64_t)g.ldy * 4u};
        const cuuint32_t box[3] = {32, 32, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, y, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const cuuint64_t dims[4] = {32, nrows, (cuuint64_t)(g.P / 32), (cuuint64_t)g.F};
    const cuuint64_t strides[3] = {(cuuint64_t)g.P * 4u, 128u, (cuuint64_t)g.ldy * 4u};
    const cuuint32_t box[4] = {32, 32, (cuuint32_t)g.stg_ch, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, y, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tc_geometry(int64_t L, int F, int N, int esize, TcGeom* g) {
    if (L < 1 || F < 1 || N < 1 || N > kTcMaxN || F > kTcMaxF || (esize != 1 && esize != 2)) return false;
    g->esize = esize;
    g->ktile = 128 / esize;  // a K slice is one 128-byte row
    // P phases per row: 128-byte rows (P = 64 FP16 or 128 FP8 samples) keep the
    // whole Toeplitz operand resident; one or two kernels use longer rows
    const int prow = 128 / esize;
    g->P = F == 1 ? 256 : (F == 2 ? (prow > 128 ? prow : 128) : prow);
    g->G = kTcN / g->P;
    g->F = F;
    g->N = N;
    g->ngroups = (F + g->G - 1) / g->G;
    g->Kpad = ((N + g->P - 1) + g->ktile - 1) / g->ktile * g->ktile;
    g->ktiles = g->Kpad / g->ktile;
    g->T = kTcM * g->P;
    g->out_len = L + N - 1;
    g->nb = (g->out_len + g->T - 1) / g->T;
    g->seg_rows = ((int64_t)g->T + g->Kpad + g->P - 1) / g->P;
    g->ldy = g->out_len;
    g->stg_ch = kTcStgChunks < g->P / 32 ? kTcStgChunks : g->P / 32;
    const int budget = kTcSmemCap - 1024;  // data bytes after the 1024-byte alignment slack
    if (g->P * esize == 128) {
        g->a_loads = (kTcM - 1 + g->ktiles + kTcABoxRows - 1) / kTcABoxRows;
        g->abuf_bytes = g->a_loads * (int)kTcABoxBytes;
        g->stages = (budget - (int)kTcStageOut - 2 * g->abuf_bytes) / (int)kTcBBytes;
    } else {
        g->a_loads = 0;
        g->abuf_bytes = 0;
        g->stages = (budget - (int)kTcStageOut) / (int)(kTcABytes + kTcBBytes);
    }
    if (g->stages > kTcMaxStages) g->stages = kTcMaxStages;
    if (g->stages < 2) return false;
    g->smem_bytes = (int)kTcStageOut +
                    (g->P * esize == 128 ? 2 * g->abuf_bytes + g->stages * (int)kTcBBytes
                                         : g->stages * (int)(kTcABytes + kTcBBytes)) + 1024;
    return true;
}

size_t tc_seg_bytes(const TcGeom& g) { return (size_t)g.esize * (size_t)(g.nb * g.seg_rows * g.P); }
size_t tc_b_bytes(const TcGeom& g) { return (size_t)g.esize * (size_t)g.ngroups * kTcN * (size_t)g.Kpad; }

template <typename E>
static cudaError_t launch_prep_e(const TcGeom& g, const float* s, int64_t L, const float* kb, int Sq, int Kq,
                                 void* seg, void* bt, float* cs_tab, float* inv_tab, float* cs_out, unsigned* status,
                                 cudaStream_t st) {
    const size_t wsm = sizeof(float) * (size_t)((g.T + g.N - 1 + kRun - 1) / kRun * kRun);
    static int wsm_dev = -1;  // the device whose copy of the kernel has the raised cap
    if (wsm > 48 * 1024) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (wsm_dev != dev) {
            cudaError_t e =
                cudaFuncSetAttribute(k_tc_quant<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemCap);
            if (e != cudaSuccess) return e;
            wsm_dev = dev;
        }
    }
    k_tc_quant<E><<<(unsigned)g.nb, 256, wsm, st>>>(s, L, g, Sq, (E*)seg, cs_tab, cs_out, status);
    k_tc_kern<E><<<dim3((unsigned)(g.ngroups * g.G), (unsigned)(g.P / 8)), 256, sizeof(E) * (size_t)(g.N + 128), st>>>(
        kb, g, Kq, (E*)bt, cs_tab, inv_tab, status);
    return cudaGetLastError();
}

cudaError_t launch_tc_prep(const TcGeom& g, const float* s, int64_t L, const float* kb, int Sq, int Kq, void* seg,
                           void* bt, float* cs_tab, float* inv_tab, float* cs_out, unsigned* status, cudaStream_t st) {
    if (g.esize == 1) return launch_prep_e<uint8_t>(g, s, L, kb, Sq, Kq, seg, bt, cs_tab, inv_tab, cs_out, status, st);
    return launch_prep_e<__half>(g, s, L, kb, Sq, Kq, seg, bt, cs_tab, inv_tab, cs_out, status, st);
}

template <bool RA, bool F8>
static void launch_mma_e(unsigned grid, const TcGeom& g, const CUtensorMap& ma, const CUtensorMap& mb,
                         const CUtensorMap& my, const float* inv_tab, float* y, int32_t* yq, unsigned* status,
                         cudaStream_t st) {
    k_tc_mma<RA, F8><<<grid, kTcThreads, (size_t)g.smem_bytes, st>>>(ma, mb, my, g, inv_tab, y, yq, status);
}

cudaError_t launch_tc_mma(const TcGeom& g, const void* seg, const void* bt, const float* inv_tab,
                          float* y, int32_t* yq, unsigned* status, cudaStream_t st, bool* encode_failed) {
    *encode_failed = false;
    const bool resident = g.P * g.esize == 128;
    CUtensorMap ma, mb, my;
    if (!encode_2d(&ma, seg, (uint64_t)g.P, (uint64_t)(g.nb * g.seg_rows), (uint64_t)g.P * g.esize,
                   resident ? kTcABoxRows : kTcM, g.esize) ||
        !encode_2d(&mb, bt, (uint64_t)g.Kpad, (uint64_t)g.ngroups * kTcN, (uint64_t)g.Kpad * g.esize, kTcN, g.esize) ||
        !encode_out(&my, y, g)) {
        *encode_failed = true;
        return cudaErrorInvalidValue;
    }
    // function attributes and the SM count belong to a device: redo them when it changes
    static int attr_dev = -1;
    static int sms = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaSuccess;
        void (*ks[4])(CUtensorMap, CUtensorMap, CUtensorMap, TcGeom, const float*, float*, int32_t*, unsigned*) = {
            k_tc_mma<true, false>, k_tc_mma<false, false>, k_tc_mma<true, true>, k_tc_mma<false, true>};
        for (int i = 0; i < 4 && e == cudaSuccess; ++i)
            e = cudaFuncSetAttribute(ks[i], cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemCap);
        if (e != cudaSuccess) return e;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        attr_dev = dev;
    }
    const int64_t nsets = g.nb * g.ngroups;
    const unsigned grid = (unsigned)(nsets < sms ? nsets : sms);
    if (g.esize == 1) {
        if (resident) launch_mma_e<true, true>(grid, g, ma, mb, my, inv_tab, y, yq, status, st);
        else launch_mma_e<false, true>(grid, g, ma, mb, my, inv_tab, y, yq, status, st);
    } else {
        if (resident) launch_mma_e<true, false>(grid, g, ma, mb, my, inv_tab, y, yq, status, st);
        else launch_mma_e<false, false>(grid, g, ma, mb, my, inv_tab, y, yq, status, st);
    }
    return cudaGetLastError();
}

}  // namespace apx
