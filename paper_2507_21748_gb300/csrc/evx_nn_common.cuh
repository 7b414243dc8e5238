// Definitions shared by the surrogate's convolution kernels (mma.sync and
// tcgen05 engines): tile geometry of the mma.sync path, the GELU pair, the
// convolution arguments, and the tcgen05 entry points.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace evxnn {

constexpr int TZ = 64;            // output voxels per tile row (along z)
constexpr int TY = 2;             // tile rows (along y): a tile is 2 x 64 voxels
constexpr int NTHR = 256;         // 8 warps x 16 voxels
constexpr int HR = 3 * (TY + 2);  // halo rows: x - 1 .. x + 1, y0 - 1 .. y0 + TY

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
// d gelu / dx = Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

struct ConvArgs {
    const __nv_bfloat16* in;     // [B][X][Y][Z][CIN]
    const __nv_bfloat16* w;      // [27][COUT][CIN]
    const float* bias;           // [COUT] or null
    void* out;                   // bf16 [..][COUT] or f32 field
    __nv_bfloat16* pre;          // GELU: pre-activation out; GELU_BWD: pre-activation in
    const __nv_bfloat16* res;    // RESID: residual [..][COUT]
    int B, X, Y, Z;
    int ntiles;
};

// tile index -> (b, x, y0, z0)
__device__ __forceinline__ void tile_coords(int tile, int X, int Y, int Z, int& b, int& x, int& y0, int& z0) {
    const int zt = Z / TZ, yt = Y / TY;
    int r = tile;
    z0 = (r % zt) * TZ;
    r /= zt;
    y0 = (r % yt) * TY;
    r /= yt;
    x = r % X;
    b = r / X;
}

// tcgen05 engine for 32 -> 32 convolutions (Z a multiple of 64; any epilogue
// but the FP32 field). Returns the launch status.
cudaError_t conv32_tc(const ConvArgs& a, int epilogue, cudaStream_t st, int sms);
// reads and clears the tcgen05 kernels' timeout flag (synchronous)
cudaError_t tc_take_timeout(int* flag);

}  // namespace evxnn
