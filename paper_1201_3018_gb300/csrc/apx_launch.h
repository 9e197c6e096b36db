// apx_launch.h -- launch configuration shared by the host API and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "apx_internal.cuh"

namespace apx {

constexpr int kDirectThreads = 256;
constexpr int kMaxSmem = 227 * 1024 - 1024;  // dynamic shared memory cap (static shared memory needs the rest)

// FFT core block kernel: one thread per 16 complex points of the largest
// transform (W_block/2), at least 32.
__host__ __device__ constexpr int fft_threads(int Wb) { return Wb / 32 > 32 ? Wb / 32 : 32; }
// FFT core kernel spectrum: R1 decimated sub-transforms of n / R1 points.
__host__ __device__ constexpr int spec_r1(int n) { return n / 2 < 16 ? n / 2 : 16; }
constexpr int kSpecThreads = 256;

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
cudaError_t launch_fft(const Params& p, size_t smem, cudaStream_t st);
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

// Tensor-core time-domain core (filterbank).  A tile is kTcM rows of P output
// phases by kTcN = G kernels x P phases; K runs over the Toeplitz band in
// slices of kTcK.
constexpr int kTcM = 128;
constexpr int kTcN = 256;
constexpr int kTcK = 64;
constexpr int kTcMaxStages = 8;
constexpr int kTcMaxN = 16384;
constexpr int kTcMaxF = 1024;
constexpr int kTcMaxQ = 2048;              // |q| <= 2048 is exact in FP16
constexpr long long kTcExactSum = 1LL << 24;  // FP32 holds every integer up to 2^24

struct TcGeom {
    int P;            // output phases per row (64, 128 or 256)
    int G;            // kernels per column group, kTcN / P
    int F;            // kernels
    int N;            // taps per kernel
    int ngroups;      // ceil(F / G)
    int Kpad;         // N + P - 1 rounded up to kTcK
    int ktiles;       // Kpad / kTcK
    int T;            // outputs per block, kTcM * P
    int64_t out_len;  // L + N - 1
    int64_t ldy;      // row pitch of the outputs (elements)
    int64_t nb;       // blocks, ceil(out_len / T)
    int64_t seg_rows; // rows of P samples in a block's segment
    int stages;       // shared-memory ring depth
    int a_loads;      // P = 64: 128-row TMA boxes that make up a tile's whole A operand
    int abuf_bytes;   // P = 64: bytes of one A buffer (a_loads x 16 KB)
    int smem_bytes;   // dynamic shared memory of the GEMM kernel
};

bool tc_geometry(int64_t L, int F, int N, TcGeom* g);
size_t tc_seg_bytes(const TcGeom& g);
size_t tc_b_bytes(const TcGeom& g);
// Block companding into FP16 segments and the kernels' Toeplitz columns.
cudaError_t launch_tc_prep(const TcGeom& g, const float* s, int64_t L, const float* kb, int Sq, int Kq, void* seg,
                           void* bt, float* cs_tab, float* ck_tab, float* cs_out, unsigned* status, cudaStream_t st);
// The persistent tensor-core GEMM with the Eq. (16) epilogue.
cudaError_t launch_tc_mma(const TcGeom& g, const void* seg, const void* bt, const float* cs_tab, const float* ck_tab,
                          float* y, int32_t* yq, unsigned* status, cudaStream_t st, bool* encode_failed);

}  // namespace apx
