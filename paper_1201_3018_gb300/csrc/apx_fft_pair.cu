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
// inner passes stay inside a CTA; for the last inverse pass (M = m) each CTA
// sends the partner the values of its four classes that the partner's
// butterflies take, and writes the block's outputs (Eq. 17).
//
// The exchanges are asynchronous remote stores (st.async) that count their
// bytes on the receiving CTA's transaction barrier (mbarrier): the sender
// waits for nothing, the receiver waits for its barrier's phase, and no CTA
// ever reads another's shared memory, so only one cluster-wide barrier remains
// (at the start, so that both CTAs and their barriers exist before any remote
// store).  Every wait is bounded (about a second; then the status word's
// timeout bit is set and the CTA leaves).
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

// Shared-memory addresses in the cluster window and the transaction barrier.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// the same variable in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cluster_addr(unsigned a, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_init(unsigned long long* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
}
// the barrier inits, visible to the cluster before its next barrier wait
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// the phase's only arrival, expecting `bytes` of remote stores
__device__ __forceinline__ void mbar_expect(unsigned long long* b, unsigned bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
                     smem_addr(b)),
                 "r"(bytes)
                 : "memory");
}
// Wait (bounded) for phase 0 of the barrier: the remote stores it counts are
// then visible to this thread.  False after about a second.
__device__ __forceinline__ bool mbar_wait0(unsigned long long* b) {
    const unsigned a = smem_addr(b);
    const long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kPrepSpinCycles) return false;
    }
}
// 8 and 4 bytes into another CTA's shared memory, counted on its barrier
__device__ __forceinline__ void st_async(unsigned raddr, float2 v, unsigned rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "f"(v.x), "f"(v.y), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void st_async(unsigned raddr, unsigned v, unsigned rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(raddr), "r"(v),
                 "r"(rbar)
                 : "memory");
}

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
    // bytes each CTA receives: the partner's first-pass outputs of this CTA's four
    // classes and its warps' flags; then the partner's classes at this CTA's
    // last-pass butterflies
    constexpr unsigned kBytesA = 32u * nt + 4u * NW, kBytesB = 32u * nt;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_wf[Q * NW];  // every warp's input flags, cluster-wide: bit 0 non-finite, bit 1 non-zero
    __shared__ __align__(8) unsigned long long s_bar[2];  // the two exchanges' transaction barriers
    if (!APX_IN_BOUNDS(blockDim.x == nt, p.status)) return;  // every CTA alike: none reaches a barrier
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0]);
        mbar_init(&s_bar[1]);
        mbar_init_fence();
        mbar_expect(&s_bar[0], kBytesA);
        mbar_expect(&s_bar[1], kBytesB);
    }
    cl_arrive_relaxed();  // this CTA and its barriers exist: the partner stores into it only after its wait
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
    const long long g0 = g.start + 2ll * j;
    if (al8 && g0 >= 0 && g0 + 14ll * S + 1 < p.L) {  // all eight pairs inside the signal
        const float2* src = reinterpret_cast<const float2*>(p.s + g0);
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __ldg(src + q * S);
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long long gi = g0 + 2ll * q * S;
            if (al8 && gi >= 0 && gi + 1 < p.L) {
                v[q] = __ldg(reinterpret_cast<const float2*>(p.s + gi));
            } else {
                v[q].x = (gi >= 0 && gi < p.L) ? __ldg(p.s + gi) : 0.f;
                v[q].y = (gi + 1 >= 0 && gi + 1 < p.L) ? __ldg(p.s + gi + 1) : 0.f;
            }
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
    cl_wait();  // the partner has started and its barriers are initialised
    const unsigned prank = (unsigned)(rank ^ 1);
    {
        const unsigned zr = cluster_addr(smem_addr(Z), prank), br = cluster_addr(smem_addr(&s_bar[0]), prank);
        const int pj = pad16(j);  // slot of class position u: pj + pad16(u S), as j < S
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int sl = pj + pad16(pair_local(r) * S);
            if (pair_owner(r) == rank) Z[sl] = v[r];
            else st_async(zr + (unsigned)sizeof(float2) * sl, v[r], br);
        }
        if ((t & 31) == 0) {
            unsigned* f = &s_wf[rank * NW + (t >> 5)];
            *f = wbits;
            st_async(cluster_addr(smem_addr(f), prank), wbits, br);
        }
    }
    // this CTA's own outputs and flags (barrier), the partner's (transaction
    // barrier: it counts kBytesA); on a timeout the status says so and the
    // block's outputs are not valid
    const bool got_a = mbar_wait0(&s_bar[0]);
    __syncthreads();
    if (!got_a) atomicOr(p.status, 2u);
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
        // kernel, zeros for a silent one; neither CTA sends the second
        // exchange, and the first has been received
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
                    } else {  // pad16(a S + x) = pad16(a S) + pad16(x) for x < S
                        pk = pad16(u * S) + pad16(rt);
                        pmk = pad16(partner_local(rank, u) * S) + pad16(S - 1 - rt);
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
    pair_inner_passes<LM, true>(Z, tws, p.status);  // (ends with a barrier: the classes are complete)

    // Last inverse pass (M = m): butterfly j takes its eight slots r S + j and
    // yields the natural-order points z[j + S q].  Each thread first sends the
    // partner's thread t (butterfly prank nt + t) this CTA's four values of it,
    // into the partner's receive buffer at u nt + t (u: class position).
    float2* Rb = tws + S;  // the partner's four classes at this CTA's butterflies
    {
        const unsigned rr = cluster_addr(smem_addr(Rb), prank), br = cluster_addr(smem_addr(&s_bar[1]), prank);
        const int pjp = pad16((int)prank * nt + t);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            st_async(rr + (unsigned)sizeof(float2) * (u * nt + t), Z[pjp + pad16(u * S)], br);
    }
    float2 w[8];
    twiddles<float2, 8, true>(w, tws, j);
    if (!mbar_wait0(&s_bar[1])) atomicOr(p.status, 2u);
    {
        const int pj = pad16(j);
#pragma unroll
        for (int r = 0; r < 8; ++r)
            v[r] = pair_owner(r) == rank ? Z[pj + pad16(pair_local(r) * S)] : Rb[pair_local(r) * nt + t];
    }
#pragma unroll
    for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], w[r]);
    dft8<float2, true>(v);

    // Eq. (17): point e = j + S q holds outputs 2e and 2e+1 of the block.
    const bool oal8 = ((reinterpret_cast<uintptr_t>(p.r) & 7u) == 0);
    const long long o0 = g.start + 2ll * j;
    const bool oin = oal8 && o0 >= 0 && o0 + 14ll * S + 1 < p.out_len;  // every pair inside the output
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int jj = 2 * (j + q * S);
        if (jj < g.lo || jj >= g.hi) continue;
        const long long o = g.start + jj;
        if (oin || (oal8 && o >= 0 && o + 1 < p.out_len)) {
            *reinterpret_cast<float2*>(p.r + o) = v[q];
            if (p.rq) *reinterpret_cast<int2*>(p.rq + o) = make_int2(0, 0);
        } else {
            if (o >= 0 && o < p.out_len) { p.r[o] = v[q].x; if (p.rq) p.rq[o] = 0; }
            if (o + 1 >= 0 && o + 1 < p.out_len) { p.r[o + 1] = v[q].y; if (p.rq) p.rq[o + 1] = 0; }
        }
    }
    // Leaving needs no cluster barrier: no CTA reads another's shared memory,
    // and each CTA has received all the partner's stores into it (its waits).
}

// the CTA's classes, the twiddle bases (m/8 = W_block/16 entries), the receive
// buffer of the last pass (4 W_block/32 entries)
size_t fft_pair_smem_bytes(int Wb) { return sizeof(float2) * (padded_len(Wb / 4) + Wb / 16 + Wb / 8); }

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
