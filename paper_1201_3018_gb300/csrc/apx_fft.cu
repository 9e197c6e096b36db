// apx_fft.cu -- the frequency-domain (FFT) block kernel.
//
// One CTA per overlap-save block.  The kernel preparation (kernel statistics
// and the FP32 kernel spectrum, apx_prep.cuh) either ran in the launches
// before (batched calls and single calls with few blocks: this kernel is their
// programmatic dependent) or runs here: in a fused single call each CTA first
// claims preparation jobs until none is left, so the preparation is spread
// over the first CTAs to start and no launch waits for another.  Each CTA:
//   1. fetches its W_block window into registers and computes the block
//      statistics,
//   2. starts the FP32 forward real FFT of the window (full precision is every
//      block's fallback) before it waits for the preparation,
//   3. runs the Section IV.D selection; for a packing candidate it companded
//      the block and checks the FFT error bound (the round-off of the FP64
//      transforms below a quarter of the finest digit) with the exact
//      integer norms sum(s~^2) and ||kbar||_1, so rounding recovers the digits,
//   4. full precision: multiplies by the spectrum and inverts; packed:
//      companded and packs (Eqs. 2, 4, 7) into an FP64 complex buffer (two
//      real words per complex entry), forward FFT, product, inverse FFT, digit
//      extraction (Eqs. 11-15), inverse companding (Eq. 16),
//   5. stores its W outputs (Eq. 17).
// A packed candidate's FP64 spectrum is built on demand by the first CTA that
// selects it; later CTAs wait for it with a bounded spin and report a timeout
// in the status word instead of hanging.
#include <type_traits>

#include "apx_fft_body.cuh"

namespace apx {

// kVals: window samples per thread (W_block / threads: 16, or 32 at the largest W_block)
template <int kVals, bool BATCH>
__global__ void __launch_bounds__(512) k_fft(const Params p0, const BatchTab bt) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ int s_flag;
    __shared__ unsigned s_feas;
    __shared__ int s_job;
    __shared__ long long s_ticket;
    __shared__ Params sp;
    // fused single call: tickets below nj are preparation jobs, the rest blocks
    const int nj = (!BATCH && p0.fused) ? prep_jobs_count(p0.Wb, blockDim.x) : 0;
    long long i;
    if (BATCH) {
        i = batch_enter(bt, sp);
    } else if (nj) {
        // a programmatic dependent of whatever ran before on the stream: its
        // launch is prepared early, and nothing is read before that work is done
        pdl_wait();
        const long long t = prep_ticket(p0, &s_ticket);
        if (t < 0 || t >= nj + p0.P) {  // the host's count of tickets is off: touch nothing
            if (threadIdx.x == 0) atomicOr(p0.status, 4u);
            return;
        }
        if (t < nj) {
            prep_job(p0, (int)t, reinterpret_cast<float2*>(smem), sh, &s_job);
            return;
        }
        i = t - nj;
    } else {
        i = blockIdx.x;
    }
    const Params& p = BATCH ? sp : p0;
    fft_block_body<kVals>(p, i, nj, (BATCH || !p0.fused) ? kWaitLaunch : kWaitJobs, smem, sh, s_flag, s_feas, s_job);
}

size_t fft_smem_bytes(const Params& p) {
    bool asym = false;
    for (int j = 0; j < p.ncand; ++j) asym |= p.cand[j].blk != APX_BLK_SYM;
    const size_t z32 = sizeof(float2) * padded_len(p.Wb / 2);
    // a symmetric candidate transforms W_block/2 real words (W_block/4 complex),
    // an asymmetric one W_block real words plus the companded block (the
    // smaller the buffer, the more of the SM's unified memory stays L1 cache)
    size_t z64 = 0;
    if (p.ncand > 0) z64 = sizeof(double2) * padded_len(asym ? p.Wb / 2 : p.Wb / 4);
    if (asym) z64 += (size_t)companded_bytes(p) * (size_t)p.Wb;
    return z32 > z64 ? z32 : z64;
}

template <bool BATCH>
static cudaError_t fft_attrs() {
    static int attr_dev = -1;
    int dev;
    cudaGetDevice(&dev);
    if (attr_dev == dev) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_fft<16, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft<32, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e == cudaSuccess) attr_dev = dev;
    return e;
}

// A call with no packing candidate and no per-block records, at W_block >= 1024,
// can run the two-CTA full-precision kernel (apx_fft_pair.cu) when it is not a
// one-launch call.
bool fft_full_only(const Params& p) { return p.ncand == 0 && !p.st && p.Wb >= 1024; }

// pdl: the programmatic dependent of the preparation launches just before it;
// false when the kernel's preparation is already resident (a prepared kernel).
cudaError_t launch_fft(const Params& p, size_t smem, cudaStream_t st, bool pdl) {
    if (p.P <= 0) return cudaSuccess;
    cudaError_t e = fft_attrs<false>();
    if (e != cudaSuccess) return e;
    const BatchTab none = {nullptr, nullptr, 0};
    if (fft_full_only(p) && p.Hpair) return launch_fft_pair(p, st, pdl);
    if (p.Wb / fft_threads(p.Wb) > 16)
        return launch_k(k_fft<32, false>, dim3((unsigned)p.P), dim3(fft_threads(p.Wb)), smem, st, pdl, p, none);
    return launch_k(k_fft<16, false>, dim3((unsigned)p.P), dim3(fft_threads(p.Wb)), smem, st, pdl, p, none);
}

// Fused single call: nj preparation CTAs ahead of the P block CTAs in one
// launch, a programmatic dependent of the stream's previous work (the kernel
// waits for it before reading anything).  Every CTA takes one ticket: the
// caller advances its copy of the counter by the grid size.
unsigned fused_grid(const Params& p) { return (unsigned)(p.P + prep_jobs_count(p.Wb, fft_threads(p.Wb))); }

cudaError_t launch_fft_fused(const Params& p, size_t smem, cudaStream_t st) {
    if (p.P <= 0) return cudaSuccess;
    cudaError_t e = fft_attrs<false>();
    if (e != cudaSuccess) return e;
    const int nt = fft_threads(p.Wb);
    const BatchTab none = {nullptr, nullptr, 0};
    if (p.Wb / nt > 16) return launch_k(k_fft<32, false>, dim3(fused_grid(p)), dim3(nt), smem, st, true, p, none);
    return launch_k(k_fft<16, false>, dim3(fused_grid(p)), dim3(nt), smem, st, true, p, none);
}

cudaError_t launch_fft_batch(const Params& any, const BatchTab& bt, int ctas, size_t smem, cudaStream_t st) {
    if (ctas <= 0) return cudaSuccess;
    cudaError_t e = fft_attrs<true>();
    if (e != cudaSuccess) return e;
    if (any.Wb / fft_threads(any.Wb) > 16)
        return launch_k(k_fft<32, true>, dim3((unsigned)ctas), dim3(fft_threads(any.Wb)), smem, st, true, any, bt);
    return launch_k(k_fft<16, true>, dim3((unsigned)ctas), dim3(fft_threads(any.Wb)), smem, st, true, any, bt);
}

// A batched launch's static shared memory (the block scratch, the request's
// parameters and two flags) has to fit beside the dynamic cap: a larger Params
// or Shared makes setting that cap fail.
static_assert(sizeof(Shared) + sizeof(Params) + 2 * sizeof(int) <= 227 * 1024 - kMaxSmem,
              "k_fft's static shared memory exceeds the room the dynamic cap leaves");

}  // namespace apx
