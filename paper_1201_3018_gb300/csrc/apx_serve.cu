// apx_serve.cu -- the serving engine's persistent kernel.
//
// Persistent CTAs of kServeThreads threads claim published tickets one at a
// time (apx_serve.h).  A ticket is a preparation job of a request's template
// (the kernel statistics, the 16 decimated sub-transforms of its spectrum, the
// combine slices: the same device functions the other FFT-core forms run) or
// one overlap-save block of the request (the general FFT block body, which
// waits, bounded, for its template's jobs).  The CTA that completes a
// request's last item publishes its status and sequence number to host-mapped
// words.  Every wait is bounded: a CTA leaves after idle_cycles without work
// (the host relaunches the kernel when it publishes more), and the block body
// gives up on a missing preparation after about a second (timeout status).
#define APX_INPUT_COHERENT  // requests may reuse input buffers during the kernel's lifetime
#include "apx_fft_body.cuh"
#include "apx_serve.h"

namespace apx {

namespace {

__device__ __forceinline__ long long ld_acquire_sys64(const long long* a) {
    long long v;
    asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_i(const int* a) { return *reinterpret_cast<const volatile int*>(a); }
__device__ __forceinline__ void st_release_sys(unsigned* a, unsigned v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// The next published ticket (thread 0), or -1 when the host asks the CTAs to
// leave or after idle_cycles without one.  A ticket is taken only below the
// published count, so a CTA that leaves strands none.
__device__ long long serve_claim(const ServeEnv& env) {
    const long long t0 = clock64();
    unsigned nap = 500;  // ns between looks at the host's count, doubling to 8 us while idle
    while (true) {
        if (ld_volatile_i(&env.hdr->stop)) return -1;
        const long long pub = ld_acquire_sys64(&env.hdr->published);
        const unsigned long long n = *reinterpret_cast<volatile unsigned long long*>(env.next);
        if ((long long)n < pub) {
            if (atomicCAS(env.next, n, n + 1ull) == n) return (long long)n;
            continue;  // another CTA took it
        }
        if (clock64() - t0 > env.idle_cycles) return -1;
        __nanosleep(nap);
        if (nap < 8000) nap *= 2;
    }
}

}  // namespace

__global__ void __launch_bounds__(kServeThreads, 2) k_serve(const ServeEnv env) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ int s_flag, s_job;
    __shared__ unsigned s_feas;
    __shared__ ServeSlot sq;  // the request of the current ticket
    __shared__ long long s_t;
    __shared__ int s_slot;
    Params& sp = sq.p;
    while (true) {
        if (threadIdx.x == 0) {
            const long long t = serve_claim(env);
            s_t = t;
            // the request of ticket t (written before the count that published t)
            if (t >= 0) s_slot = ld_volatile_i(&env.tmap[t & env.tmask]);
        }
        __syncthreads();
        const long long t = s_t;
        if (t < 0) break;
        {  // the whole slot into shared memory, one word per thread: one trip over the host link
            const volatile int* src = reinterpret_cast<const volatile int*>(&env.slots[s_slot]);
            int* dst = reinterpret_cast<int*>(&sq);
            for (int w = threadIdx.x; w < (int)(sizeof(ServeSlot) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
        }
        __syncthreads();
        const long long s_base = sq.base;
        const int s_nprep = sq.nprep, s_njobs = sq.njobs, s_nitems = sq.nitems, s_skip = sq.skip_prep;
        const unsigned s_seq = sq.seq;
        const long long li = t - s_base;
        if (li < s_nprep) {
            // A preparation job of the template: the norms of every candidate
            // (blocks of any target read them by candidate position).
            if (threadIdx.x == 0) sp.autosel = 0;
            __syncthreads();
            if (!s_skip) prep_job(sp, (int)li, reinterpret_cast<float2*>(smem), sh, &s_job);
        } else {
            fft_block_body<32>(sp, li - s_nprep, s_njobs, s_njobs ? kWaitJobs : kWaitNone, smem, sh, s_flag, s_feas,
                               s_job);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence_system();  // this item's outputs before its count
            const int slot = s_slot;
            if (atomicAdd(&env.done_items[slot], 1) + 1 == s_nitems) {
                __threadfence_system();
                env.done_items[slot] = 0;
                const unsigned st = atomicExch(&env.dstatus[slot], 0u);
                *reinterpret_cast<volatile unsigned*>(&env.fstatus[slot]) = st;
                __threadfence_system();
                st_release_sys(&env.done_seq[slot], s_seq);
            }
        }
        __syncthreads();  // the request's shared state is rewritten for the next ticket
    }
}

// The block body's largest shared memory at W_block <= 8192: the FP64 packed
// transform of an asymmetric candidate with the companded block in 4-byte
// integers (the FP32 transform and the preparation jobs need less).
size_t serve_smem_bytes() {
    const size_t z64 = sizeof(double2) * padded_len(kServeWbMax / 2) + 4 * (size_t)kServeWbMax;
    const size_t z32 = sizeof(float2) * padded_len(kServeWbMax / 2);
    return z64 > z32 ? z64 : z32;
}

cudaError_t launch_serve(const ServeEnv& env, int ctas, size_t smem, cudaStream_t st) {
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {  // exactly what it uses (its static shared memory needs the rest)
        cudaError_t e = cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)serve_smem_bytes());
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    k_serve<<<(unsigned)ctas, kServeThreads, smem, st>>>(env);
    return cudaGetLastError();
}

}  // namespace apx
