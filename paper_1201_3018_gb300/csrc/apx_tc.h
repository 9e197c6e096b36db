// apx_tc.h -- launch interface of the tensor-core time-domain core (filterbank).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>


// Device-side bounds checks of builds with -DAPX_CHECKED: a failed check sets
// bit 2 of the status word (APX_ERR_CHECK from apx_sync) and the guarded
// access is skipped.  Other builds compile the checks away.
#ifdef APX_CHECKED
#define APX_IN_BOUNDS(cond, status) ((cond) ? true : ((status) ? (atomicOr((status), 4u), false) : false))
#else
#define APX_IN_BOUNDS(cond, status) true
#endif

namespace apx {

// Tensor-core time-domain core (filterbank).  A tile is kTcM rows of P output
// phases by kTcN = G kernels x P phases; K runs over the Toeplitz band in
// slices of one 128-byte row (64 FP16 or 128 FP8 elements).
constexpr int kTcSmemCap = 227 * 1024 - 1024;  // dynamic shared memory cap (static needs the rest)
constexpr int kTcM = 128;
constexpr int kTcN = 256;
constexpr int kTcMaxStages = 8;
constexpr int kTcMaxN = 16384;
constexpr int kTcMaxF = 1024;
constexpr int kTcMaxQ = 2048;              // |q| <= 2048 is exact in FP16
constexpr int kTcMaxQ8 = 16;               // |q| <= 16 is exact in FP8 E4M3
constexpr long long kTcExactSum = 1LL << 24;  // FP32 holds every integer up to 2^24

struct TcGeom {
    int P;            // output phases per row (64, 128 or 256)
    int G;            // kernels per column group, kTcN / P
    int F;            // kernels
    int N;            // taps per kernel
    int ngroups;      // ceil(F / G)
    int esize;        // operand bytes: 2 (FP16) or 1 (FP8 E4M3, S_q and K_q <= 16)
    int ktile;        // elements per K slice, 128 / esize
    int Kpad;         // N + P - 1 rounded up to ktile
    int ktiles;       // Kpad / ktile
    int T;            // outputs per block, kTcM * P
    int64_t out_len;  // L + N - 1
    int64_t ldy;      // row pitch of the outputs (elements)
    int64_t nb;       // blocks, ceil(out_len / T)
    int64_t seg_rows; // rows of P samples in a block's segment
    int stages;       // shared-memory ring depth
    int a_loads;      // P = 64: 128-row TMA boxes that make up a tile's whole A operand
    int abuf_bytes;   // P = 64: bytes of one A buffer (a_loads x 16 KB)
    int smem_bytes;   // dynamic shared memory of the GEMM kernel
    int stg_ch;       // output chunks (32 rows x 32 phases) per bulk store of the epilogue
};

bool tc_geometry(int64_t L, int F, int N, int esize, TcGeom* g);
size_t tc_seg_bytes(const TcGeom& g);
size_t tc_b_bytes(const TcGeom& g);
// Block companding into FP16 segments and the kernels' Toeplitz columns.
// cs_tab: c_s per block; inv_tab: fl32(1 / (c_s c_k)) per block and kernel
// slot (nb x ngroups * G floats).
cudaError_t launch_tc_prep(const TcGeom& g, const float* s, int64_t L, const float* kb, int Sq, int Kq, void* seg,
                           void* bt, float* cs_tab, float* inv_tab, float* cs_out, unsigned* status, cudaStream_t st);
// The persistent tensor-core GEMM with the Eq. (16) epilogue.
cudaError_t launch_tc_mma(const TcGeom& g, const void* seg, const void* bt, const float* inv_tab, float* y,
                          int32_t* yq, unsigned* status, cudaStream_t st, bool* encode_failed);

}  // namespace apx
