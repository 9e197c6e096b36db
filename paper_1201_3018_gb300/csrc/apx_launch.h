// apx_launch.h -- launch configuration shared by the host API and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "apx_internal.cuh"

namespace apx {

constexpr int kDirectThreads = 256;
// Direct core: taps staged in shared memory per chunk (FP32 taps for full
// precision, packed FP64 taps for packed blocks).
constexpr int kDirectTapChunkF = 2048;
constexpr int kDirectTapChunkD = 1024;
constexpr int kMaxSmem = 227 * 1024 - 1024;  // dynamic shared memory cap (static shared memory needs the rest)

// FFT core block kernel: one thread per 16 complex points of the largest
// transform (W_block/2), at least 32.
__host__ __device__ constexpr int fft_threads(int Wb) { return Wb / 32 > 32 ? Wb / 32 : 32; }
// FFT core kernel spectrum: R1 decimated sub-transforms of n / R1 points.
__host__ __device__ constexpr int spec_r1(int n) { return n / 2 < 16 ? n / 2 : 16; }
constexpr int kSpecThreads = 256;
// Preparation jobs of a fused single call (apx_prep.cuh) for a block kernel of
// nt threads: R1 sub-transforms, the combine in slices of nt frequencies, the
// kernel statistics.
__host__ __device__ constexpr int prep_jobs_count(int Wb, int nt) {
    return spec_r1(Wb) + (Wb / 2 + 1 + nt - 1) / nt + 1;
}

// Launch through cudaLaunchKernelEx; `pdl` marks the launch as a programmatic
// dependent of the previous kernel in the stream (the kernel calls
// griddepcontrol.wait before it reads that kernel's results).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_spec(const Params& p, cudaStream_t st);
cudaError_t launch_spec_combine(const Params& p, cudaStream_t st);
cudaError_t launch_direct(const Params& p, size_t smem, cudaStream_t st);
cudaError_t launch_fft(const Params& p, size_t smem, cudaStream_t st, bool pdl = true);
cudaError_t launch_fft_fused(const Params& p, size_t smem, cudaStream_t st);
unsigned fused_grid(const Params& p);
size_t fft_smem_bytes(const Params& p);

// Batched launches: `any` is one request's parameters (for the launch shape and
// as the unused parameter-space copy); the kernels read every request's own
// parameters through the table.
int spec_ctas(int Wb);
int combine_ctas(int Wb);
cudaError_t launch_direct_batch(const Params& any, const BatchTab& bt, int ctas, size_t smem, cudaStream_t st);
cudaError_t launch_spec_batch(const Params& any, const BatchTab& bt, int ctas, cudaStream_t st, bool pdl);
cudaError_t launch_combine_batch(const Params& any, const BatchTab& bt, int ctas, cudaStream_t st);
cudaError_t launch_fft_batch(const Params& any, const BatchTab& bt, int ctas, size_t smem, cudaStream_t st);
bool fft_full_only(const Params& p);
// Full precision only, outside a fused launch: one block per cluster of two CTAs.
cudaError_t launch_fft_pair(const Params& p, cudaStream_t st, bool pdl);
// bytes of its staging-order spectrum table (2 CTAs x 15 entries x W_block/32 threads)
inline size_t pair_table_bytes(int Wb) { return sizeof(float2) * 30 * (size_t)(Wb / 32); }
size_t fft_pair_smem_bytes(int Wb);

}  // namespace apx
