// apx_spectra.cu -- kernel preparation of the FFT core (Section IV
// "Initialization": the kernel is prepared once per request) as two small
// launches ahead of the block kernel, for batched calls and for single calls
// with few blocks (single calls with many blocks run the same pieces inside
// the block kernel, see apx_prep.cuh):
//   k_spec:   CTA r < R1 runs spec_subfft(r); CTA R1 runs spec_stats; a
//             single call's CTA 0 also resets the claim and ready words of
//             its packed spectra.
//   k_combine: spec_combine, one thread per frequency.
// Each launch is the programmatic dependent of the one before it; the block
// kernel waits for k_combine only where it multiplies by H.
#include "apx_prep.cuh"

namespace apx {

// The signal's bytes, a slice per CTA, into L2 while the kernel preparation
// runs (the block kernel reads every sample, most of them twice): the first
// warp issues bulk L2 prefetches of up to 64 KB between the slice's 16-byte
// boundaries, inside the signal.  Nothing waits for them.
__device__ __forceinline__ void prefetch_signal(const Params& p) {
    if (threadIdx.x >= 32) return;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p.s), e = a + 4ull * (uintptr_t)p.L;
    const uintptr_t lo = (a + 15u) & ~(uintptr_t)15u, hi = e & ~(uintptr_t)15u;
    if (hi <= lo) return;
    const uintptr_t per = (((hi - lo) + gridDim.x - 1) / gridDim.x + 15u) & ~(uintptr_t)15u;
    const uintptr_t s0 = lo + per * blockIdx.x, s1 = s0 + per < hi ? s0 + per : hi;
    constexpr uintptr_t kPiece = 64u * 1024u;
    for (uintptr_t q = s0 + kPiece * threadIdx.x; q < s1; q += kPiece * 32u) {
        const uint32_t n = (uint32_t)(s1 - q < kPiece ? s1 - q : kPiece);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(
                         reinterpret_cast<const void*>(q))),
                     "r"(n)
                     : "memory");
    }
}

template <bool BATCH>
__global__ void __launch_bounds__(kSpecThreads) k_spec(const Params p0, const BatchTab bt) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ Params sp;
    pdl_trigger();
    const int cta = BATCH ? (int)batch_enter(bt, sp) : (int)blockIdx.x;
    const Params& p = BATCH ? sp : p0;
    if (!BATCH && cta == 0 && threadIdx.x < kMaxCand) {
        // A single call's packed spectra are built anew: a call captured into a
        // graph replays with the same epoch, and its kernel taps may have
        // changed since the last replay.  The block kernel claims them only
        // after the combine launch, which waits for this one.
        p0.claim[threadIdx.x] = p0.claim_init;
        p0.ready[threadIdx.x] = 0u;
    }
    if (!BATCH && p0.pf) prefetch_signal(p0);
    if (cta == spec_r1(p.Wb)) spec_stats(p, sh);
    else spec_subfft(p, cta, reinterpret_cast<float2*>(smem));
}

template <bool BATCH>
__global__ void __launch_bounds__(256) k_combine(const Params p0, const BatchTab bt) {
    __shared__ Params sp;
    pdl_trigger();
    const int cta = BATCH ? (int)batch_enter(bt, sp) : (int)blockIdx.x;
    const Params& p = BATCH ? sp : p0;
    pdl_wait();  // the decimated sub-spectra
    const int k = cta * blockDim.x + threadIdx.x;
    if (k <= p.Wb / 2) spec_combine(p, k);
}

cudaError_t launch_spec(const Params& p, cudaStream_t st) {
    const int n = p.Wb, R1 = spec_r1(n);
    const size_t smem = sizeof(float2) * padded_len(n / R1);
    const BatchTab none = {nullptr, nullptr, 0};
    return launch_k(k_spec<false>, dim3(R1 + 1), dim3(kSpecThreads), smem, st, false, p, none);
}

cudaError_t launch_spec_combine(const Params& p, cudaStream_t st) {
    const int m = p.Wb / 2;
    const BatchTab none = {nullptr, nullptr, 0};
    return launch_k(k_combine<false>, dim3((m + 1 + 255) / 256), dim3(256), 0, st, true, p, none);
}

int spec_ctas(int Wb) { return spec_r1(Wb) + 1; }
int combine_ctas(int Wb) { return (Wb / 2 + 1 + 255) / 256; }

cudaError_t launch_spec_batch(const Params& any, const BatchTab& bt, int ctas, cudaStream_t st, bool pdl) {
    const int n = any.Wb, R1 = spec_r1(n);
    const size_t smem = sizeof(float2) * padded_len(n / R1);
    return launch_k(k_spec<true>, dim3(ctas), dim3(kSpecThreads), smem, st, pdl, any, bt);
}

cudaError_t launch_combine_batch(const Params& any, const BatchTab& bt, int ctas, cudaStream_t st) {
    return launch_k(k_combine<true>, dim3(ctas), dim3(256), 0, st, true, any, bt);
}

}  // namespace apx
