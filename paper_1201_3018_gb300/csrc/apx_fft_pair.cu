// apx_fft_pair.cu -- the full-precision FFT block kernel on a cluster of CTAs.
//
// The block kernel is latency bound: one CTA per W_block block leaves most of
// an SM's warp slots empty (a 2^20-sample call has fewer than two blocks per
// SM), and each CTA's transform is a long chain of dependent passes.  Here a
// thread-block cluster of two CTAs computes one block, each CTA half the
// points with half the registers, so that an SM holds twice the warps and
// each chain is half as long.  The two CTAs exchange data through distributed
// shared memory twice per block, and nowhere else:
//
// With radix-8 passes (decimation in frequency), the first forward pass of a
// length-m transform (M = m, stride S = m/8) sends the output digit r of
// butterfly j to slot r S + j; every later pass works inside one of the eight
// ranges [r S, r S + S) ("class" r).  The real-signal step pairs frequency k
// with m - k, whose class is -r mod 8, so the classes split into two sets
// closed under that pairing: CTA 0 holds classes {0, 1, 4, 7}, CTA 1 holds
// {2, 3, 5, 6}.  The first forward pass (butterflies split between the CTAs,
// inputs straight from the window) writes each output to the CTA that holds
// its class; the forward inner passes, the spectral product and the inverse
// inner passes stay inside a CTA; the last inverse pass (M = m) reads the
// partner's four classes and writes the block's outputs (Eq. 17).
//
// The kernel is compiled for each W_block (m = 2^LM), so that the passes'
// strides, slot arithmetic and digit reversals are constants (measured 17 %
// faster than one kernel for every W_block; clusters of four CTAs, each two
// classes, measured no faster at W_block 8192 and slower at 4096).  Every butterfly
// and every spectral-product term is the single-CTA kernels' arithmetic in the
// same order, so the results are the same bits.  Full precision only (no
// packing candidate, no per-block records), W_block >= 1024.
#include <cooperative_groups.h>

#include "apx_prep.cuh"

namespace apx {

namespace cg = cooperative_groups;

namespace {

// Class of position u < 4 of CTA `rank` (ascending class order).
__device__ __forceinline__ int class_of(int rank, int u) {
    const int c0[4] = {0, 1, 4, 7}, c1[4] = {2, 3, 5, 6};
    return rank ? c1[u] : c0[u];
}
// Position of class -c mod 8 in the same CTA, for its u-th class c != 0.
__device__ __forceinline__ int partner_local(int rank, int u) { return (rank == 0 ? 4 : 3) - u; }

// Radix-8 passes inside the local classes (m/2 points, four sub-transforms of
// S = m/8 points): forward M = S, S/8, ... then the tail radix-T pass (m = 8^A
// T); inverse in the reverse order.  Table: W_m^u, u < S (length-m indexing).
template <int LM, bool INV>
__device__ __forceinline__ void pair_inner_passes(float2* Z, const float2* __restrict__ tw, unsigned* st) {
    constexpr int m = 1 << LM, A = LM / 3, T = 1 << (LM % 3), ML = m / 2;
    if constexpr (!INV) {
#pragma unroll
        for (int s = 1; s < A; ++s) {
            fft_pass<float2, 8, false>(Z, ML, m >> (3 * s), tw, m, st);
            __syncthreads();
        }
        if constexpr (T == 4) fft_pass<float2, 4, false>(Z, ML, 4, tw, m, st);
        if constexpr (T == 2) fft_pass<float2, 2, false>(Z, ML, 2, tw, m, st);
        if constexpr (T > 1) __syncthreads();
    } else {
        if constexpr (T == 4) fft_pass<float2, 4, true>(Z, ML, 4, tw, m, st);
        if constexpr (T == 2) fft_pass<float2, 2, true>(Z, ML, 2, tw, m, st);
        if constexpr (T > 1) __syncthreads();
#pragma unroll
        for (int s = A - 1; s >= 1; --s) {
            fft_pass<float2, 8, true>(Z, ML, m >> (3 * s), tw, m, st);
            __syncthreads();
        }
    }
}

// 8-byte asynchronous copy global -> shared (cached in L1: the source is not
// written during this launch once the preparation it depends on is complete).
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// threads per CTA (m = 2^LM, W_block = 2m) and the CTAs per SM the register
// budget is set for (64 registers per thread)
constexpr int pair_threads(int LM) { return (1 << LM) / 16; }
constexpr int pair_min_ctas(int nt) { return 1024 / nt > 16 ? 16 : 1024 / nt; }

}  // namespace

// One block per cluster of two CTAs (cluster rank = blockIdx.x & 1), S/2 =
// W_block/32 threads each.  Not a batched form: single calls that run
// their kernel preparation in launches ahead of it, and prepared kernels.
template <int LM>
__global__ void __launch_bounds__(pair_threads(LM), pair_min_ctas(pair_threads(LM))) k_fft_pair(const Params p) {
    constexpr int Q = 2, m = 1 << LM, S = m / 8, nt = S / Q, ML = m / Q;
    constexpr int NW = nt / 32;  // warps per CTA
    static_assert(nt >= 32 && nt % 32 == 0, "whole warps");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_wf[Q * NW];  // every warp's input flags, cluster-wide: bit 0 non-finite, bit 1 non-zero
    if (!APX_IN_BOUNDS(blockDim.x == nt, p.status)) return;  // every CTA alike: none reaches a barrier
    cl_arrive_relaxed();  // this CTA has started: the others write its shared memory only after their wait
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const long long i = (long long)(blockIdx.x / Q);
    const BlockGeom g = block_geom(p, i);
    const int t = threadIdx.x;
    float2* Z = reinterpret_cast<float2*>(smem);

    // The twiddle bases of every pass, W_m^u for u < m/8 (FP32 passes load only
    // W^j and form its powers by products), copied into shared memory while the
    // window loads are in flight: table entry u is tw[u ntab / m], read by the
    // passes as a table of length m.  Thread t copies u = t and t + nt.
    float2* tws = Z + padded_len(ML);
#pragma unroll
    for (int e = 0; e < Q; ++e) cp_async8(&tws[t + e * nt], &p.tw32[(t + e * nt) * (p.ntab / m)]);
    cp_async_commit();

    // First forward pass (M = m): butterfly j takes z[j + S q] = x[2e] + i x[2e+1],
    // e = j + S q, straight from the window, and sends output r to its class.
    const int j = rank * nt + t;
    float2 v[8];
    const bool al8 = ((reinterpret_cast<uintptr_t>(p.s + g.start) & 7u) == 0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long long gi = g.start + 2ll * (j + q * S);
        if (al8 && gi >= 0 && gi + 1 < p.L) {
            v[q] = __ldg(reinterpret_cast<const float2*>(p.s + gi));
        } else {
            v[q].x = (gi >= 0 && gi < p.L) ? __ldg(p.s + gi) : 0.f;
            v[q].y = (gi + 1 >= 0 && gi + 1 < p.L) ? __ldg(p.s + gi + 1) : 0.f;
        }
    }
    bool bad = false, nz = false;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        bad |= (__float_as_uint(v[q].x) & 0x7f800000u) == 0x7f800000u;
        bad |= (__float_as_uint(v[q].y) & 0x7f800000u) == 0x7f800000u;
        nz |= (v[q].x != 0.f) | (v[q].y != 0.f);
    }
    const unsigned wbits = (__any_sync(0xffffffffu, bad) ? 1u : 0u) | (__any_sync(0xffffffffu, nz) ? 2u : 0u);
    cp_async_wait_all();  // this thread's copies: the first pass reads tws[j], j = t + rank nt, one of them
    {
        float2 w[8];
        twiddles<float2, 8, false>(w, tws, j);
        dft8<float2, false>(v);
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], w[r]);
    }
    cl_wait();  // every CTA of the cluster has started
    {
        float2* dst[Q];
        unsigned* wf[Q];
#pragma unroll
        for (int o = 0; o < Q; ++o) {
            dst[o] = o == rank ? Z : cl.map_shared_rank(Z, o);
            wf[o] = o == rank ? s_wf : cl.map_shared_rank(s_wf, o);
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) dst[pair_owner(r)][pad16(pair_local(r) * S + j)] = v[r];
        if ((t & 31) == 0) {
#pragma unroll
            for (int o = 0; o < Q; ++o) wf[o][rank * NW + (t >> 5)] = wbits;
        }
    }
    cl_arrive();  // release: this thread's writes into the cluster's shared memory
    cl_wait();    // every CTA's first-pass outputs, flags and twiddle copies are in place
    unsigned fl = 0;
#pragma unroll
    for (int w = 0; w < Q * NW; ++w) fl |= s_wf[w];
    const bool any_bad = (fl & 1u) != 0;
    const bool live = (fl & 2u) != 0 && !any_bad;

    pair_inner_passes<LM, false>(Z, tws, p.status);

    // The kernel's statistics and FP32 spectrum come from the preparation
    // launches, which this launch overlaps up to here.  This thread's entries
    // H[k], H[m-k] and W^k, 15 per thread in this order (pair_entry), so that
    // each load instruction of a warp is contiguous; read around L1.
    pdl_wait();
    const float2* src = p.Hpair + rank * 15 * nt + t;
    float2 hs[15];
#pragma unroll
    for (int a = 0; a < 12; ++a) hs[a] = __ldcg(src + a * nt);
    if (rank == 0 && t == 0) {
#pragma unroll
        for (int a = 12; a < 15; ++a) hs[a] = __ldcg(src + a * nt);
    }
    const float Mk = __ldcg(&p.ki->Mk);
    const int kbad = __ldcg(&p.ki->bad);
    if (any_bad || kbad || !live || Mk == 0.f) {
        // the same for every CTA of the cluster: NaN for a non-finite block or
        // kernel, zeros for a silent one; no access to another CTA's shared
        // memory after the barrier above
        const float c = (any_bad || kbad) ? __int_as_float(0x7fc00000) : 0.f;
        for (int jj = g.lo + rank * nt + t; jj < g.hi; jj += Q * nt) {
            const long long o = g.start + jj;
            if (o < 0 || o >= p.out_len) continue;
            p.r[o] = c;
            if (p.rq) p.rq[o] = 0;
        }
        if ((any_bad || kbad) && rank == 0 && t == 0) atomicOr(p.status, 1u);
        return;
    }

    // Spectral product of the real-signal step on this CTA's classes: thread t
    // takes k = 8 t + c_u for its four classes (u = position of class c_u; CTA 0
    // also k = m/2); the partner m - k lies in the same CTA.  Frequency k's slot
    // is c S + rev(k / 8), rev the sub-transforms' digit reversal; rev(S - 1 -
    // x) = S - 1 - rev(x) (every digit complemented).
    {
#pragma unroll
        for (int u = 0; u < 5; ++u) {
            if (u == 4 && (rank != 0 || t != 0)) continue;
            const int c = u < 4 ? class_of(rank, u) : 0;
            const int k = u < 4 ? 8 * t + c : m / 2;
            const float2 hk = hs[3 * u], hmk = hs[3 * u + 1], w = hs[3 * u + 2];
            if (k == 0) {
                const float2 z0 = Z[0];
                float2 X0, Xm;
                X0.x = 2 * (z0.x + z0.y); X0.y = 0;
                Xm.x = 2 * (z0.x - z0.y); Xm.y = 0;
                const float2 Y0 = cmul(X0, hk), Ym = cmul(Xm, hmk);
                const float2 cym = cconj(Ym);
                Z[0] = cadd(cadd(Y0, cym), mul_mi<float2, true>(csub(Y0, cym)));
            } else {
                int pk, pmk;
                if (u == 4) {
                    pk = pmk = pad16(fft_perm_rc<8, S>(S / 2, S));
                } else {
                    const int rt = fft_perm_rc<8, S>(t, S);
                    if (c == 0) {
                        pk = pad16(rt);
                        pmk = pad16(fft_perm_rc<8, S>(S - t, S));
                    } else {
                        pk = pad16(u * S + rt);
                        pmk = pad16(partner_local(rank, u) * S + (S - 1 - rt));
                    }
                }
                const float2 a = Z[pk], b = Z[pmk];
                float2 Xk, Xmk, Zk, Zmk;
                real_post(a, b, w, Xk, Xmk);
                const float2 Yk = cmul(Xk, hk), Ymk = cmul(Xmk, hmk);
                real_pre(Yk, Ymk, w, Zk, Zmk);
                Z[pk] = Zk;
                if (k != m - k) Z[pmk] = Zmk;
            }
        }
    }
    __syncthreads();
    pair_inner_passes<LM, true>(Z, tws, p.status);
    cl_arrive();  // release: this CTA's classes are complete

    // Last inverse pass (M = m): butterfly j reads its eight slots r S + j (the
    // other CTAs' classes among them) and yields the natural-order points
    // z[j + S q].  Its twiddles come first, while the barrier completes.
    float2 w[8];
    twiddles<float2, 8, true>(w, tws, j);
    cl_wait();
    {
        const float2* srcq[Q];
#pragma unroll
        for (int o = 0; o < Q; ++o) srcq[o] = o == rank ? Z : cl.map_shared_rank(Z, o);
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = srcq[pair_owner(r)][pad16(pair_local(r) * S + j)];
    }
#pragma unroll
    for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], w[r]);
    dft8<float2, true>(v);
    cl_arrive();  // this thread's reads of other CTAs' shared memory are complete (their values are used)

    // Eq. (17): point e = j + S q holds outputs 2e and 2e+1 of the block.
    const bool oal8 = ((reinterpret_cast<uintptr_t>(p.r) & 7u) == 0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int jj = 2 * (j + q * S);
        if (jj < g.lo || jj >= g.hi) continue;
        const long long o = g.start + jj;
        if (oal8 && o >= 0 && o + 1 < p.out_len) {
            *reinterpret_cast<float2*>(p.r + o) = v[q];
            if (p.rq) *reinterpret_cast<int2*>(p.rq + o) = make_int2(0, 0);
        } else {
            if (o >= 0 && o < p.out_len) { p.r[o] = v[q].x; if (p.rq) p.rq[o] = 0; }
            if (o + 1 >= 0 && o + 1 < p.out_len) { p.r[o + 1] = v[q].y; if (p.rq) p.rq[o + 1] = 0; }
        }
    }
    cl_wait();  // no CTA leaves while another still reads its shared memory
}

// the CTA's classes and the twiddle bases (m/8 = W_block/16 entries)
size_t fft_pair_smem_bytes(int Wb) { return sizeof(float2) * (padded_len(Wb / 4) + Wb / 16); }

namespace {

template <int LM>
cudaError_t launch_pair(const Params& p, cudaStream_t st, bool pdl) {
    static int attr_dev = -1;  // device whose attribute is set (per W_block)
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t smem = fft_pair_smem_bytes(2 << LM);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_fft_pair<LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * p.P));
    cfg.blockDim = dim3((unsigned)pair_threads(LM));  // S / 2 butterflies of the outer passes per CTA
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_fft_pair<LM>, p);
}

}  // namespace

cudaError_t launch_fft_pair(const Params& p, cudaStream_t st, bool pdl) {
    if (p.P <= 0) return cudaSuccess;
    switch (p.Wb) {
        case 1024: return launch_pair<9>(p, st, pdl);
        case 2048: return launch_pair<10>(p, st, pdl);
        case 4096: return launch_pair<11>(p, st, pdl);
        case 8192: return launch_pair<12>(p, st, pdl);
        case 16384: return launch_pair<13>(p, st, pdl);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace apx
