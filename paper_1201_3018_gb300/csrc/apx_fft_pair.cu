// apx_fft_pair.cu -- the full-precision FFT block kernel on a pair of CTAs.
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
// Every butterfly and every spectral-product term is the single-CTA kernels'
// arithmetic in the same order, so the results are the same bits.  Full
// precision only (no packing candidate, no per-block records), W_block >= 1024.
#include <cooperative_groups.h>

#include "apx_prep.cuh"

namespace apx {

namespace cg = cooperative_groups;

namespace {

__device__ __forceinline__ int class_owner(int r) { return pair_owner(r); }
__device__ __forceinline__ int class_local(int r) { return pair_local(r); }
// the four classes of CTA `rank`, in local order
__device__ __forceinline__ int class_of(int rank, int u) {
    const int c0[4] = {0, 1, 4, 7}, c1[4] = {2, 3, 5, 6};
    return rank ? c1[u] : c0[u];
}

// Radix-8 passes inside the local classes (mloc = m/2 points, four
// sub-transforms of S = m/8 points): forward M = S, S/8, ... then the tail
// radix-t pass (m = 8^a t); inverse in the reverse order.
template <bool INV>
__device__ __forceinline__ void pair_inner_passes(float2* Z, int m, const float2* __restrict__ tw, int ntab,
                                                  unsigned* st) {
    int a = 0, t = m;
    while (t >= 8) { t /= 8; ++a; }
    const int mloc = m / 2;
    if (!INV) {
        int M = m / 8;
        for (int s = 1; s < a; ++s) { fft_pass<float2, 8, false>(Z, mloc, M, tw, ntab, st); __syncthreads(); M /= 8; }
        if (t == 4) fft_pass<float2, 4, false>(Z, mloc, 4, tw, ntab, st);
        else if (t == 2) fft_pass<float2, 2, false>(Z, mloc, 2, tw, ntab, st);
        if (t > 1) __syncthreads();
    } else {
        if (t == 4) fft_pass<float2, 4, true>(Z, mloc, 4, tw, ntab, st);
        else if (t == 2) fft_pass<float2, 2, true>(Z, mloc, 2, tw, ntab, st);
        if (t > 1) __syncthreads();
        int M = t * 8;
        for (int s = 1; s < a; ++s) { fft_pass<float2, 8, true>(Z, mloc, M, tw, ntab, st); __syncthreads(); M *= 8; }
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


}  // namespace

// One block per cluster of two CTAs (cluster rank = blockIdx.x & 1), S/2 =
// W_block/32 threads each.  Not a batched form: single calls that run their
// kernel preparation in launches ahead of it, and prepared kernels.
__global__ void __launch_bounds__(512, 2) k_fft_pair(const Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_peer[2];  // the partner's block flags: non-finite, non-zero
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const long long i = (long long)(blockIdx.x >> 1);
    const BlockGeom g = block_geom(p, i);
    const int m = p.Wb / 2, S = m / 8, nt = blockDim.x, t = threadIdx.x;
    float2* Z = reinterpret_cast<float2*>(smem);
    float2* Zp = cl.map_shared_rank(Z, rank ^ 1);
    const bool shape_ok = APX_IN_BOUNDS(2 * nt == S, p.status);

    // The twiddle bases of every pass, W_m^u for u < m/8 (FP32 passes load only
    // W^j and form its powers by products), copied into shared memory while the
    // window loads are in flight: table entry u is tw[u ntab / m], read by the
    // passes as a table of length m.
    float2* tws = Z + padded_len(m / 2) + 15 * nt;
    for (int u = t; u < S; u += nt) cp_async8(&tws[u], &p.tw32[u * (p.ntab / m)]);
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
    const unsigned my_bad = __syncthreads_or(bad) ? 1u : 0u;
    const unsigned my_nz = __syncthreads_or(nz) ? 1u : 0u;
    cp_async_wait_all();
    __syncthreads();  // every thread's part of the table
    {
        float2 w[8];
        twiddles<float2, 8, false>(w, tws, j);
        dft8<float2, false>(v);
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], w[r]);
        if (shape_ok) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                float2* dst = class_owner(r) == rank ? Z : Zp;
                dst[pad16(class_local(r) * S + j)] = v[r];
            }
        }
    }
    if (t == 0) {  // the block's flags to the partner (read after the cluster barrier)
        unsigned* peer = cl.map_shared_rank(s_peer, rank ^ 1);
        peer[0] = my_bad;
        peer[1] = my_nz;
    }
    cl.sync();  // remote writes of both CTAs visible
    const bool any_bad = (my_bad | s_peer[0]) != 0;
    const bool live = (my_nz | s_peer[1]) != 0 && !any_bad;

    // The kernel's statistics and FP32 spectrum (from the preparation launches,
    // which this launch may overlap): this thread's spectrum entries H[k],
    // H[m-k] and twiddles W^k are copied asynchronously into shared memory
    // while the forward passes run, so the spectral product waits for no load.
    pdl_wait();
    // 15 entries per thread: (u, {H[k], H[m-k], W^k}) x nt, prepared in this
    // order (pair_entry), so that each copy instruction of a warp is contiguous
    float2* stage = Z + padded_len(m / 2);
    const float2* src = p.Hpair + rank * 15 * nt;
#pragma unroll
    for (int a = 0; a < 15; ++a) cp_async8(&stage[a * nt + t], &src[a * nt + t]);
    cp_async_commit();
    const float Mk = __ldcg(&p.ki->Mk);
    const int kbad = __ldcg(&p.ki->bad);
    pair_inner_passes<false>(Z, m, tws, m, p.status);
    if (any_bad || kbad || !live || Mk == 0.f) {
        // the same for both CTAs: NaN for a non-finite block or kernel, zeros
        // for a silent one; no remote access after the barrier above
        const float c = (any_bad || kbad) ? __int_as_float(0x7fc00000) : 0.f;
        for (int jj = g.lo + rank * nt + t; jj < g.hi; jj += 2 * nt) {
            const long long o = g.start + jj;
            if (o < 0 || o >= p.out_len) continue;
            p.r[o] = c;
            if (p.rq) p.rq[o] = 0;
        }
        if ((any_bad || kbad) && rank == 0 && t == 0) atomicOr(p.status, 1u);
        cp_async_wait_all();  // no copy into this CTA's shared memory outlives it
        return;
    }

    // Spectral product of the real-signal step on this CTA's classes: thread t
    // takes k = 8 t + c_u for its four classes (u = position of class c_u; CTA 0
    // also k = m/2); the partner m - k lies in the same CTA.  Frequency k's slot
    // is c S + rev(k / 8), rev the sub-transforms' digit reversal, so the
    // thread's slots follow from rev(t), rev(S - 1 - t) and rev(S - t).
    {
        const int rt = fft_perm_r<8>(t, S), rt1 = fft_perm_r<8>(S - 1 - t, S);
        const int rt0 = t > 0 ? fft_perm_r<8>(S - t, S) : 0, rhalf = fft_perm_r<8>(S / 2, S);
        cp_async_wait_all();  // this thread's staged entries (it reads only its own)
#pragma unroll
        for (int u = 0; u < 5; ++u) {
            if (u == 4 && (rank != 0 || t != 0)) continue;
            const int c = u < 4 ? class_of(rank, u) : 0;
            const int k = u < 4 ? 8 * t + c : m / 2;
            const float2 hk = stage[(3 * u + 0) * nt + t], hmk = stage[(3 * u + 1) * nt + t];
            const float2 w = stage[(3 * u + 2) * nt + t];
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
                    pk = pmk = pad16(rhalf);
                } else if (c == 0) {
                    pk = pad16(rt);
                    pmk = pad16(rt0);
                } else {
                    pk = pad16(u * S + rt);
                    pmk = pad16(class_local(8 - c) * S + rt1);
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
    pair_inner_passes<true>(Z, m, tws, m, p.status);
    cl.sync();  // both CTAs' inner passes done: the partner's classes can be read

    // Last inverse pass (M = m): butterfly j reads its eight slots r S + j (four
    // of them the partner's) and yields the natural-order points z[j + S q].
    {
        float2 w[8];
        if (shape_ok) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float2* src = class_owner(r) == rank ? Z : Zp;
                v[r] = src[pad16(class_local(r) * S + j)];
            }
        }
        twiddles<float2, 8, true>(w, tws, j);
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], w[r]);
        dft8<float2, true>(v);
    }
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
    cl.sync();  // the partner has read this CTA's classes before either exits
}

// the CTA's classes, the spectral-product staging (15 entries per thread), the
// twiddle bases (m/8 = W_block/16 entries)
size_t fft_pair_smem_bytes(int Wb) { return sizeof(float2) * (padded_len(Wb / 4) + 15 * (Wb / 32) + Wb / 16); }

cudaError_t launch_fft_pair(const Params& p, cudaStream_t st, bool pdl) {
    if (p.P <= 0) return cudaSuccess;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t smem = fft_pair_smem_bytes(p.Wb);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_fft_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * p.P));
    cfg.blockDim = dim3((unsigned)(p.Wb / 32));  // S / 2 butterflies of the outer passes per CTA
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
    return cudaLaunchKernelEx(&cfg, k_fft_pair, p);
}

}  // namespace apx
