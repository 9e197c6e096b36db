// apx_launch.h -- launch configuration shared by the host API and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "apx_internal.cuh"

namespace apx {

constexpr int kDirectThreads = 256;
constexpr int kFftThreads = 256;
constexpr int kPrepThreads = 1024;
constexpr int kMaxSmem = 227 * 1024 - 1024;  // dynamic shared memory cap (static shared memory needs the rest)

cudaError_t launch_prep(const Params& p, const float* k, int xcorr, double* kbar_out[kMaxCand], KInfo* ki,
                        float* kfull, cudaStream_t st);
cudaError_t launch_select(const Params& p, cudaStream_t st);
cudaError_t launch_spectra(const Params& p, float2* Hfull, double2* Hc[kMaxCand], cudaStream_t st);
cudaError_t launch_direct(const Params& p, size_t smem, cudaStream_t st);
cudaError_t launch_fft(const Params& p, size_t smem, cudaStream_t st);

int fft_maxb(int Wb);

}  // namespace apx
