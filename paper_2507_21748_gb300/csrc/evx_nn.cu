// Kernels of the learned surrogate: a 3D residual CNN that advances the
// Cahn-Hilliard field by a block of solver steps. Periodic 3x3x3
// convolutions as implicit GEMMs on the tensor cores (BF16 operands, FP32
// accumulation, mma.sync m16n8k16), their data and weight gradients, and the
// element-wise and reduction kernels of training (GELU, zero-mean output
// correction, mean-squared loss, Adam) with FP64 reductions.
//
// Activations are BF16, channels-last: [B][X][Y][Z][C], C = 16 or 32.
// Conv weights are [27][Cout][Cin] (tap t = 9 (dx+1) + 3 (dy+1) + (dz+1)),
// Cin fastest; biases FP32 [Cout]. out(v, co) = b(co) + sum_t sum_ci
// W[t][co][ci] in(v + off_t, ci) with periodic wrap.
#include <cuda_bf16.h>

#include <atomic>
#include <cstdlib>
#include <cstdint>

#include "../../include/evx_nn.h"
#include "evx_nn_common.cuh"

namespace evxnn {

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}


__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t& r0, uint32_t& r1, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(smem_addr(p)));
}


// load the halo rows (x+dx, y0-1 .. y0+TY) x (z0-1 .. z0+TZ), periodic, into
// s[HR][TZ+2][C+8] (pitch C+8 halves: conflict-free fragment loads); halo
// row index (dx+1) * (TY+2) + (y - y0 + 1)
template <int C>
__device__ __forceinline__ void load_halo(__nv_bfloat16* s, const __nv_bfloat16* g, int b, int x, int y0, int z0,
                                          int X, int Y, int Z, int nthreads) {
    constexpr int P = C + 8, V16 = C / 8;  // 16-byte pieces per voxel
    const int n = HR * (TZ + 2) * V16;
    for (int e = threadIdx.x; e < n; e += nthreads) {
        const int q = e % V16, rem = e / V16, zi = rem % (TZ + 2), nb = rem / (TZ + 2);
        const int dx = nb / (TY + 2) - 1, yi = nb % (TY + 2) - 1;
        const int xx = (x + dx + X) % X, yy = (y0 + yi + Y) % Y, zz = (z0 + zi - 1 + Z) % Z;
        const long long vox = (((long long)b * X + xx) * Y + yy) * Z + zz;
        const uint4 val = *reinterpret_cast<const uint4*>(g + vox * C + q * 8);
        *reinterpret_cast<uint4*>(s + (nb * (TZ + 2) + zi) * P + q * 8) = val;
    }
}


template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(NTHR) conv_fwd_kernel(ConvArgs a) {
    constexpr int PI = CIN + 8, PW = CIN + 8, NT = COUT / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(smem_raw);   // [27][COUT][PW]
    __nv_bfloat16* sin = sw + 27 * COUT * PW;                          // [HR][TZ+2][PI]
    for (int e = threadIdx.x; e < 27 * COUT * (CIN / 8); e += NTHR) {
        const int q = e % (CIN / 8), row = e / (CIN / 8);
        *reinterpret_cast<uint4*>(sw + row * PW + q * 8) = *reinterpret_cast<const uint4*>(a.w + row * CIN + q * 8);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
    const int yl = warp >> 2, zs = (warp & 3) * 16;  // warp's 16 voxels: row y0 + yl, z0 + zs ..
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        int b, x, y0, z0;
        tile_coords(tile, a.X, a.Y, a.Z, b, x, y0, z0);
        __syncthreads();  // previous tile done with sin (and weights loaded)
        load_halo<CIN>(sin, a.in, b, x, y0, z0, a.X, a.Y, a.Z, NTHR);
        __syncthreads();
        float acc[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
        const int zl = zs + g;
#pragma unroll 1
        for (int t = 0; t < 27; ++t) {
            const int dx = t / 9, dy = (t / 3) % 3, dz = t % 3 - 1;
            const int nb = dx * (TY + 2) + yl + dy;  // (dx+1)(TY+2) + (yl + (dy-1) + 1)
            const __nv_bfloat16* r0 = sin + (nb * (TZ + 2) + zl + dz + 1) * PI;
            const __nv_bfloat16* r1 = r0 + 8 * PI;
            const __nv_bfloat16* wt = sw + t * COUT * PW;
#pragma unroll
            for (int ks = 0; ks < CIN / 16; ++ks) {
                uint32_t af[4];
                af[0] = *reinterpret_cast<const uint32_t*>(r0 + ks * 16 + 2 * tig);
                af[1] = *reinterpret_cast<const uint32_t*>(r1 + ks * 16 + 2 * tig);
                af[2] = *reinterpret_cast<const uint32_t*>(r0 + ks * 16 + 2 * tig + 8);
                af[3] = *reinterpret_cast<const uint32_t*>(r1 + ks * 16 + 2 * tig + 8);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const __nv_bfloat16* wr = wt + (nt * 8 + g) * PW + ks * 16 + 2 * tig;
                    mma_bf16(acc[nt], af, *reinterpret_cast<const uint32_t*>(wr),
                             *reinterpret_cast<const uint32_t*>(wr + 8));
                }
            }
        }
        // epilogue: rows g, g+8 of the warp's 16 voxels; columns co = nt*8 + 2 tig (+1)
        const long long vbase = (((long long)b * a.X + x) * a.Y + y0 + yl) * a.Z + z0 + zs;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long vox = vbase + g + 8 * h;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int co = nt * 8 + 2 * tig;
                float v0 = acc[nt][2 * h], v1 = acc[nt][2 * h + 1];
                if (a.bias) {
                    v0 += a.bias[co];
                    v1 += a.bias[co + 1];
                }
                const long long o = vox * COUT + co;
                if (EPI == EVX_NN_EPI_FIELD) {
                    if (co == 0) reinterpret_cast<float*>(a.out)[vox] = v0;
                    continue;
                }
                if (EPI == EVX_NN_EPI_GELU) {
                    if (a.pre) *reinterpret_cast<__nv_bfloat162*>(a.pre + o) = __floats2bfloat162_rn(v0, v1);
                    v0 = gelu(v0);
                    v1 = gelu(v1);
                } else if (EPI == EVX_NN_EPI_GELU_BWD) {
                    const float2 p = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(a.pre + o));
                    v0 *= gelu_grad(p.x);
                    v1 *= gelu_grad(p.y);
                } else if (EPI == EVX_NN_EPI_RESID) {
                    const float2 q = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(a.res + o));
                    v0 += q.x;
                    v1 += q.y;
                } else if (EPI == EVX_NN_EPI_RESID32) {  // FP32 stream in a.pre, updated in place
                    float2* sp = reinterpret_cast<float2*>(reinterpret_cast<float*>(a.pre) + o);
                    const float2 q = *sp;
                    v0 += q.x;
                    v1 += q.y;
                    *sp = make_float2(v0, v1);
                }
                *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(a.out) + o) =
                    __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}


// ----------------------------------------------------------- weight gradient
// dW[t][co][ci] = sum_v dY(v, co) X(v + off_t, ci): per tap a (COUT x CIN) GEMM
// over the voxels. Warp w owns accumulator tiles j = w, w + 4, ... of the
// 27 * (COUT/16) * (CIN/8) m16n8 tiles; each CTA walks its voxel tiles and
// writes its partial sums, reduced in a fixed order afterwards.
struct WgradArgs {
    const __nv_bfloat16* dy;   // [..][COUT]
    const __nv_bfloat16* x;    // [..][CIN]
    float* partials;           // [grid][27][COUT][CIN]
    int B, X, Y, Z, ntiles;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(NTHR) conv_wgrad_kernel(WgradArgs a) {
    constexpr int PI = CIN + 8, PD = COUT + 8, TPT = (COUT / 16) * (CIN / 8), NTOT = 27 * TPT;
    constexpr int NW = NTHR / 32, MAXJ = (NTOT + NW - 1) / NW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* sx = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // [HR][TZ+2][PI]
    __nv_bfloat16* sdy = sx + HR * (TZ + 2) * PI;                     // [TY * TZ][PD]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
    float acc[MAXJ][4];
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        int b, x, y0, z0;
        tile_coords(tile, a.X, a.Y, a.Z, b, x, y0, z0);
        __syncthreads();
        load_halo<CIN>(sx, a.x, b, x, y0, z0, a.X, a.Y, a.Z, NTHR);
        for (int e = threadIdx.x; e < TY * TZ * (COUT / 8); e += NTHR) {
            const int q = e % (COUT / 8), v = e / (COUT / 8), yl = v / TZ, z = v % TZ;
            const long long vox = (((long long)b * a.X + x) * a.Y + y0 + yl) * a.Z + z0 + z;
            *reinterpret_cast<uint4*>(sdy + v * PD + q * 8) =
                *reinterpret_cast<const uint4*>(a.dy + vox * COUT + q * 8);
        }
        __syncthreads();
#pragma unroll 1
        for (int k0 = 0; k0 < TY * TZ; k0 += 16) {
            const int yl = k0 / TZ, zk = k0 % TZ;  // the 16 voxels share a row
#pragma unroll
            for (int jj = 0; jj < MAXJ; ++jj) {
                const int j = warp + NW * jj;
                if (j < NTOT) {
                    const int t = j / TPT, tile_ = j % TPT;
                    const int mt = tile_ / (CIN / 8), nt = tile_ % (CIN / 8);
                    // A = dY^T (co x v): 8x8 blocks (v 0-7 | 8-15) x (co 0-7 | 8-15), transposed
                    uint32_t af[4];
                    const int va = k0 + (lane & 7) + ((lane >> 4) << 3);
                    ldsm_x4_trans(af, sdy + va * PD + mt * 16 + ((lane >> 3) & 1) * 8);
                    // B = X shifted by tap t (v x ci): blocks v 0-7 and 8-15 of columns nt*8..+8
                    const int dx = t / 9, dy = (t / 3) % 3, dz = t % 3 - 1;
                    const int nb = dx * (TY + 2) + yl + dy;
                    const int vb = zk + (lane & 7) + ((lane >> 3) & 1) * 8;
                    uint32_t b0, b1;
                    ldsm_x2_trans(b0, b1, sx + (nb * (TZ + 2) + vb + dz + 1) * PI + nt * 8);
                    mma_bf16(acc[jj], af, b0, b1);
                }
            }
        }
    }
    // write this CTA's partial dW (c0,c1: row g; c2,c3: row g+8; cols 2 tig, 2 tig + 1)
    float* P = a.partials + (long long)blockIdx.x * 27 * COUT * CIN;
#pragma unroll
    for (int jj = 0; jj < MAXJ; ++jj) {
        const int j = warp + NW * jj;
        if (j < NTOT) {
            const int t = j / TPT, tile_ = j % TPT;
            const int mt = tile_ / (CIN / 8), nt = tile_ % (CIN / 8);
            const int co = mt * 16 + g, ci = nt * 8 + 2 * tig;
            float* p = P + ((long long)t * COUT + co) * CIN + ci;
            p[0] = acc[jj][0];
            p[1] = acc[jj][1];
            p[8 * CIN] = acc[jj][2];
            p[8 * CIN + 1] = acc[jj][3];
        }
    }
}

// out[i] = sum_b partials[b * n + i] in order b = 0, 1, ... (deterministic)
__global__ void reduce_partials_f32(const float* partials, int nparts, int n, float* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += partials[(long long)b * n + i];
        out[i] = (float)s;
    }
}

// ---------------------------------------------------------- element-wise
// bias gradient: db[co] = sum_v dy(v, co); per-block FP64 partials
__global__ void bias_grad_kernel(const __nv_bfloat16* dy, long long nvox, int C, double* partials) {
    __shared__ double ws[256];
    for (int co = 0; co < C; ++co) {
        double s = 0.0;
        for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
             v += (long long)gridDim.x * blockDim.x)
            s += (double)__bfloat162float(dy[v * C + co]);
        ws[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) ws[threadIdx.x] += ws[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * C + co] = ws[0];
        __syncthreads();
    }
}
// One pass for all channels (C = 16 or 32): C / 8 threads per voxel, each summing
// 8 channels from 16-byte loads (four voxels in flight), FP32 over 32 voxels at a
// time and FP64 beyond;
// the CTA then adds its threads' sums per channel in a fixed order.
template <int C>
__global__ void __launch_bounds__(256) bias_grad_vec_kernel(const __nv_bfloat16* __restrict__ dy, long long nvox,
                                                             double* partials) {
    constexpr int TPV = C / 8;
    __shared__ double red[256][9];  // padded rows
    const int piece = threadIdx.x % TPV;
    const long long stride = (long long)gridDim.x * blockDim.x / TPV;
    double acc[8];
    float part[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.0, part[k] = 0.f;
    // four voxels in flight per thread per round; FP32 over 8 rounds, then FP64
    int cnt = 0;
    for (long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / TPV; v < nvox; v += 4 * stride) {
        uint4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long vu = v + u * stride;
            q[u] = vu < nvox ? *reinterpret_cast<const uint4*>(dy + vu * C + 8 * piece) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q[u]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 f = __bfloat1622float2(h[j]);
                part[2 * j] += f.x;
                part[2 * j + 1] += f.y;
            }
        }
        if (++cnt == 8) {
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += part[k], part[k] = 0.f;
            cnt = 0;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) red[threadIdx.x][k] = acc[k] + part[k];
    __syncthreads();
    if (threadIdx.x < C) {
        const int pc = threadIdx.x / 8, j = threadIdx.x % 8;
        double s = 0.0;
        for (int t = pc; t < (int)blockDim.x; t += TPV) s += red[t][j];
        partials[(long long)blockIdx.x * C + threadIdx.x] = s;
    }
}

__global__ void bias_grad_finish(const double* partials, int nparts, int C, float* db) {
    const int co = threadIdx.x;
    if (co < C) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += partials[b * C + co];
        db[co] = (float)s;
    }
}

// field (FP32, one value per voxel) -> activation with C channels, channel 0 = field * scale
__global__ void field_to_act_kernel(const float* f, long long nvox, int C, float scale, __nv_bfloat16* act) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < C; ++c) act[v * C + c] = __float2bfloat16_rn(c == 0 ? f[v] * scale : 0.f);
    }
}

// per-sample FP64 sums of a field: partials[s * nb + blk]
__global__ void sample_sum_kernel(const float* f, long long V, double* partials, int nb) {
    __shared__ double ws[256];
    const int s = blockIdx.y;
    double acc = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x)
        acc += (double)f[s * V + v];
    ws[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) ws[threadIdx.x] += ws[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[s * nb + blockIdx.x] = ws[0];
}

// out = base + (d - mean_s(d)) per sample (base may be null: out = d - mean)
__global__ void zero_mean_add_kernel(const float* base, const float* d, const double* partials, int nb, long long V,
                                     float* out, const double* scale) {
    const int s = blockIdx.y;
    double m = 0.0;
    for (int b = 0; b < nb; ++b) m += partials[s * nb + b];
    const float mean = (float)(m / (double)V);
    const float f = scale ? (float)scale[s] : 1.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        const float x = f * (d[s * V + v] - mean);
        out[s * V + v] = base ? base[s * V + v] + x : x;
    }
}

// Per sample s and block b: with the sample's FP64 mean m (from the partial sums
// pm), partial FP64 sums of d^2 and N^2, d = x - m, N = d^2 (3 m + d) (the
// nonlinear remainder of c^3 - c about the mean): out[(s * 2 + 0|1) * nb + b].
__global__ void nl_moments_kernel(const float* x, long long V, const double* pm, int nb, double* out) {
    __shared__ double ws[2][256];
    const int s = blockIdx.y;
    double m = 0.0;
    for (int b = 0; b < nb; ++b) m += pm[s * nb + b];
    m /= (double)V;
    double a2 = 0.0, n2 = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const double d = (double)x[s * V + v] - m;
        const double N = d * d * (3.0 * m + d);
        a2 += d * d;
        n2 += N * N;
    }
    ws[0][threadIdx.x] = a2;
    ws[1][threadIdx.x] = n2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ws[0][threadIdx.x] += ws[0][threadIdx.x + o];
            ws[1][threadIdx.x] += ws[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[(s * 2 + 0) * nb + blockIdx.x] = ws[0][0];
        out[(s * 2 + 1) * nb + blockIdx.x] = ws[1][0];
    }
}
// scale[s] = min(1, sqrt(sum N^2 / sum d^2)) (0 for a uniform sample), fixed order
__global__ void nl_scale_kernel(const double* mom, int nb, int nsamples, double* scale) {
    const int s = threadIdx.x;
    if (s >= nsamples || blockIdx.x != 0) return;
    double a2 = 0.0, n2 = 0.0;
    for (int b = 0; b < nb; ++b) {
        a2 += mom[(s * 2 + 0) * nb + b];
        n2 += mom[(s * 2 + 1) * nb + b];
    }
    scale[s] = a2 > 0.0 ? fmin(1.0, sqrt(n2 / a2)) : 0.0;
}

// squared error: partials of sum (p - t)^2 (FP64); grad = scale (p - t)
__global__ void mse_kernel(const float* p, const float* t, long long n, float scale, float* grad, double* partials) {
    __shared__ double ws[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float d = p[i] - t[i];
        acc += (double)d * d;
        if (grad) grad[i] = scale * d;
    }
    ws[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) ws[threadIdx.x] += ws[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = ws[0];
}
// partials[b] = FP64 sum of |x| over a grid-stride share of the n values
__global__ void abs_sum_kernel(const float* x, long long n, double* partials) {
    __shared__ double ws[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += fabs((double)x[i]);
    ws[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) ws[threadIdx.x] += ws[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = ws[0];
}
__global__ void sum_partials_kernel(const double* partials, int n, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += partials[i];
        *out = s;
    }
}

// dgrad weights: Wt[26 - t][ci][co] = W[t][co][ci] (BF16)
__global__ void flip_weights_kernel(const __nv_bfloat16* w, int cout, int cin, __nv_bfloat16* wt) {
    const int n = 27 * cout * cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % cin, co = (i / cin) % cout, t = i / (cin * cout);
        wt[((26 - t) * cin + ci) * cout + co] = w[i];
    }
}

// Adam on FP32 master parameters, BF16 copy refreshed (bf16 may be null)
__global__ void adam_kernel(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2, __nv_bfloat16* wbf) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        w[i] = wi;
        if (wbf) wbf[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void f32_to_bf16_kernel(const float* a, int n, __nv_bfloat16* b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

// ------------------------------------------- direct lift and projection
// The network's first and last convolutions touch one field: the lift reads
// only channel 0 of its (zero-padded) input, the projection writes only
// channel 0. As tensor-core GEMMs they would spend 15/16 of the work on
// zeros; here they are direct 3x3x3 sums on the CUDA cores, one voxel per
// thread (864 FMAs), weights broadcast from shared memory, neighbour loads
// coalesced along z (a warp covers 32 consecutive voxels of a row).
__device__ __forceinline__ void vox_coords(long long v, int X, int Y, int Z, int& b, int& x, int& y, int& z) {
    z = (int)(v % Z);
    long long r = v / Z;
    y = (int)(r % Y);
    r /= Y;
    x = (int)(r % X);
    b = (int)(r / X);
}

// out(v, co) = bias(co) + sum_t w[t][co][0] BF16(scale f(v + off_t)), co < 32
// F32: the FP32-stream variant (the field enters unrounded; out32 receives the FP32 sums)
template <bool F32>
__global__ void __launch_bounds__(256) lift_direct_kernel(const float* __restrict__ f, float scale,
                                                           const __nv_bfloat16* __restrict__ w, int wcin,
                                                           const float* __restrict__ bias, __nv_bfloat16* out,
                                                           float* __restrict__ out32, int B, int X, int Y, int Z) {
    __shared__ float4 ws[27][8];  // w[t][co][0], co = 4 q .. 4 q + 3
    __shared__ float bs[32];
    for (int i = threadIdx.x; i < 27 * 32; i += blockDim.x) {
        const int t = i >> 5, co = i & 31;
        reinterpret_cast<float*>(&ws[t][0])[co] = __bfloat162float(w[(t * 32 + co) * wcin]);
    }
    if (threadIdx.x < 32) bs[threadIdx.x] = bias ? bias[threadIdx.x] : 0.f;
    __syncthreads();
    const long long nvox = (long long)B * X * Y * Z;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        int b, x, y, z;
        vox_coords(v, X, Y, Z, b, x, y, z);
        float acc[32];
#pragma unroll
        for (int co = 0; co < 32; ++co) acc[co] = bs[co];
#pragma unroll 1
        for (int t = 0; t < 27; ++t) {
            const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
            const int xx = x + dx < 0 ? X - 1 : (x + dx == X ? 0 : x + dx);
            const int yy = y + dy < 0 ? Y - 1 : (y + dy == Y ? 0 : y + dy);
            const int zz = z + dz < 0 ? Z - 1 : (z + dz == Z ? 0 : z + dz);
            const float fv = scale * f[(((long long)b * X + xx) * Y + yy) * Z + zz];
            const float val = F32 ? fv : __bfloat162float(__float2bfloat16_rn(fv));
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 wq = ws[t][q];
                acc[4 * q] = fmaf(wq.x, val, acc[4 * q]);
                acc[4 * q + 1] = fmaf(wq.y, val, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(wq.z, val, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(wq.w, val, acc[4 * q + 3]);
            }
        }
        uint4* o = reinterpret_cast<uint4*>(out + v * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint4 pk;
            __nv_bfloat162* pp = reinterpret_cast<__nv_bfloat162*>(&pk);
#pragma unroll
            for (int j = 0; j < 4; ++j) pp[j] = __floats2bfloat162_rn(acc[8 * q + 2 * j], acc[8 * q + 2 * j + 1]);
            o[q] = pk;
        }
        if (F32) {
            float4* o32 = reinterpret_cast<float4*>(out32 + v * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q) o32[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
    }
}

// out(v) = bias(0) + sum_t sum_ci w[t][0][ci] h(v + off_t, ci), ci < 32, FP32 field;
// w is [27][wcout][32] (row 0 of each tap used)
// F32: reads the FP32 residual stream h32 instead of the BF16 activations h
template <bool F32>
__global__ void __launch_bounds__(256) project_direct_kernel(const __nv_bfloat16* __restrict__ h,
                                                              const float* __restrict__ h32,
                                                              const __nv_bfloat16* __restrict__ w, int wcout,
                                                              const float* __restrict__ bias, float* out, int B,
                                                              int X, int Y, int Z) {
    __shared__ float4 ws[27][8];  // w[t][0][ci], ci = 4 q .. 4 q + 3
    for (int i = threadIdx.x; i < 27 * 32; i += blockDim.x) {
        const int t = i >> 5, ci = i & 31;
        reinterpret_cast<float*>(&ws[t][0])[ci] = __bfloat162float(w[(long long)t * wcout * 32 + ci]);
    }
    __syncthreads();
    const float b0 = bias ? bias[0] : 0.f;
    const long long nvox = (long long)B * X * Y * Z;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        int b, x, y, z;
        vox_coords(v, X, Y, Z, b, x, y, z);
        float acc = b0;
#pragma unroll 1
        for (int t = 0; t < 27; ++t) {
            const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
            const int xx = x + dx < 0 ? X - 1 : (x + dx == X ? 0 : x + dx);
            const int yy = y + dy < 0 ? Y - 1 : (y + dy == Y ? 0 : y + dy);
            const int zz = z + dz < 0 ? Z - 1 : (z + dz == Z ? 0 : z + dz);
            const long long vi = (((long long)b * X + xx) * Y + yy) * Z + zz;
            if (F32) {
                const float4* hp = reinterpret_cast<const float4*>(h32 + vi * 32);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 hv = hp[q], wq = ws[t][q];
                    acc = fmaf(wq.x, hv.x, acc);
                    acc = fmaf(wq.y, hv.y, acc);
                    acc = fmaf(wq.z, hv.z, acc);
                    acc = fmaf(wq.w, hv.w, acc);
                }
                continue;
            }
            const uint4* hp = reinterpret_cast<const uint4*>(h + vi * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 hv = hp[q];
                const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&hv);
                const float4 wa = ws[t][2 * q], wb = ws[t][2 * q + 1];
                const float2 h0 = __bfloat1622float2(h2[0]), h1 = __bfloat1622float2(h2[1]);
                const float2 h2f = __bfloat1622float2(h2[2]), h3 = __bfloat1622float2(h2[3]);
                acc = fmaf(wa.x, h0.x, acc);
                acc = fmaf(wa.y, h0.y, acc);
                acc = fmaf(wa.z, h1.x, acc);
                acc = fmaf(wa.w, h1.y, acc);
                acc = fmaf(wb.x, h2f.x, acc);
                acc = fmaf(wb.y, h2f.y, acc);
                acc = fmaf(wb.z, h3.x, acc);
                acc = fmaf(wb.w, h3.y, acc);
            }
        }
        out[v] = acc;
    }
}

// ---------------------------------------------------------------------------
// Lift and projection with one warp per RY x 32 outputs of a (b, x) plane
// (rows y0 .. y0 + RY - 1, z0 .. z0 + 31) and lane = channel: every global access
// of a voxel is one coalesced row of its 32 channels, and each input row segment
// is read once per warp for all the outputs it feeds (3 dz taps along z, up to
// 3 dy taps across the RY rows). Needs Z % 32 = 0 and Y % RY = 0.
__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// lane l ends with the lane sum of v[l] (a butterfly that halves the values per step)
__device__ __forceinline__ float lane_sum_transpose(float (&v)[32], int lane) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = lane & off;
#pragma unroll
        for (int k = 0; k < off; ++k) {
            const float send = upper ? v[k] : v[k + off];
            const float keep = upper ? v[k + off] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0];
}

template <int RY>
__device__ __forceinline__ bool lane_unit(long long u, int X, int Y, int Z, int& b, int& x, int& y0, int& z0) {
    const int nzr = Z >> 5, nyr = Y / RY;
    z0 = (int)(u % nzr) << 5;
    long long r = u / nzr;
    y0 = (int)(r % nyr) * RY;
    r /= nyr;
    x = (int)(r % X);
    b = (int)(r / X);
    return true;
}

// out(v) = bias(0) + sum_t sum_ci w[t][0][ci] h(v + off_t, ci); lane = ci
template <bool F32, int RY, int MINB>
__global__ void __launch_bounds__(256, MINB) project_lane_kernel(const __nv_bfloat16* __restrict__ h,
                                                            const float* __restrict__ h32,
                                                            const __nv_bfloat16* __restrict__ w, int wcout,
                                                            const float* __restrict__ bias, float* out, int B,
                                                            int X, int Y, int Z) {
    __shared__ float ws[27][32];  // w[t][0][ci]
    for (int i = threadIdx.x; i < 27 * 32; i += blockDim.x)
        ws[i >> 5][i & 31] = __bfloat162float(w[(long long)(i >> 5) * wcout * 32 + (i & 31)]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float b0 = bias ? bias[0] : 0.f;
    const long long units = (long long)B * X * (Y / RY) * (Z >> 5);
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += nw) {
        int b, x, y0, z0;
        lane_unit<RY>(u, X, Y, Z, b, x, y0, z0);
        float acc[RY][32];
#pragma unroll
        for (int r = 0; r < RY; ++r)
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[r][j] = 0.f;
        const int zl = wrapi(z0 - 1, Z), zh = wrapi(z0 + 32, Z);
#pragma unroll 1
        for (int dx = 0; dx < 3; ++dx) {
            const int xx = wrapi(x + dx - 1, X);
#pragma unroll 1
            for (int yy = 0; yy < RY + 2; ++yy) {
                const long long row = (((long long)b * X + xx) * Y + wrapi(y0 + yy - 1, Y)) * Z;
                float hv[34];
                if (F32) {
                    const float* rp = h32 + (row + z0) * 32 + lane;  // z0 + j - 1 at rp[(j - 1) 32]
                    hv[0] = __ldg(h32 + (row + zl) * 32 + lane);
#pragma unroll
                    for (int j = 1; j < 33; ++j) hv[j] = __ldg(rp + (j - 1) * 32);
                    hv[33] = __ldg(h32 + (row + zh) * 32 + lane);
                } else {
                    const __nv_bfloat16* rp = h + (row + z0) * 32 + lane;
                    hv[0] = __bfloat162float(h[(row + zl) * 32 + lane]);
#pragma unroll
                    for (int j = 1; j < 33; ++j) hv[j] = __bfloat162float(rp[(j - 1) * 32]);
                    hv[33] = __bfloat162float(h[(row + zh) * 32 + lane]);
                }
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    const int dy = yy - r;  // tap 9 dx + 3 dy + dz  // input row y0 + yy - 1 = output row y0 + r + dy - 1
                    if (dy < 0 || dy > 2) continue;
#pragma unroll
                    for (int dz = 0; dz < 3; ++dz) {
                        const float wt = ws[9 * dx + 3 * dy + dz][lane];
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[r][j] = fmaf(wt, hv[j + dz], acc[r][j]);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const float sum = lane_sum_transpose(acc[r], lane);
            out[(((long long)b * X + x) * Y + y0 + r) * Z + z0 + lane] = sum + b0;
        }
    }
}

// out(v, co) = bias(co) + sum_t w[t][co][0] val(f(v + off_t)), val = scale f (F32) or its
// BF16 rounding; lane = co. F32 also writes the FP32 copy out32.
template <bool F32, int RY, int MINB>
__global__ void __launch_bounds__(256, MINB) lift_lane_kernel(const float* __restrict__ f, float scale,
                                                         const __nv_bfloat16* __restrict__ w, int wcin,
                                                         const float* __restrict__ bias, __nv_bfloat16* out,
                                                         float* __restrict__ out32, int B, int X, int Y, int Z) {
    __shared__ float ws[27][32];  // w[t][co][0]
    for (int i = threadIdx.x; i < 27 * 32; i += blockDim.x) ws[i >> 5][i & 31] = __bfloat162float(w[i * wcin]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float bl = bias ? bias[lane] : 0.f;
    const long long units = (long long)B * X * (Y / RY) * (Z >> 5);
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += nw) {
        int b, x, y0, z0;
        lane_unit<RY>(u, X, Y, Z, b, x, y0, z0);
        float acc[RY][32];
#pragma unroll
        for (int r = 0; r < RY; ++r)
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[r][j] = bl;
#pragma unroll 1
        for (int dx = 0; dx < 3; ++dx) {
            const int xx = wrapi(x + dx - 1, X);
#pragma unroll 1
            for (int yy = 0; yy < RY + 2; ++yy) {
                const long long row = (((long long)b * X + xx) * Y + wrapi(y0 + yy - 1, Y)) * Z;
                // lane l holds z0 - 1 + l; lanes 0, 1 also z0 + 31, z0 + 32
                float f0 = scale * f[row + wrapi(z0 - 1 + lane, Z)];
                float f1 = lane < 2 ? scale * f[row + wrapi(z0 + 31 + lane, Z)] : 0.f;
                if (!F32) {
                    f0 = __bfloat162float(__float2bfloat16_rn(f0));
                    f1 = __bfloat162float(__float2bfloat16_rn(f1));
                }
                float hv[34];
#pragma unroll
                for (int j = 0; j < 34; ++j)
                    hv[j] = j < 32 ? __shfl_sync(0xffffffffu, f0, j) : __shfl_sync(0xffffffffu, f1, j - 32);
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    const int dy = yy - r;  // tap 9 dx + 3 dy + dz
                    if (dy < 0 || dy > 2) continue;
#pragma unroll
                    for (int dz = 0; dz < 3; ++dz) {
                        const float wt = ws[9 * dx + 3 * dy + dz][lane];
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[r][j] = fmaf(wt, hv[j + dz], acc[r][j]);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const long long v0 = (((long long)b * X + x) * Y + y0 + r) * Z + z0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                out[(v0 + j) * 32 + lane] = __float2bfloat16_rn(acc[r][j]);
                if (F32) out32[(v0 + j) * 32 + lane] = acc[r][j];
            }
        }
    }
}

}  // namespace evxnn

// ===================================================================== C-ABI
using namespace evxnn;

namespace {
thread_local const char* g_nn_err = "";
int g_nn_sms = 0;
int nn_sms() {
    if (!g_nn_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_nn_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_nn_sms <= 0) g_nn_sms = 1;
    }
    return g_nn_sms;
}
evx_status nn_fail(evx_status s, const char* m) {
    g_nn_err = m;
    return s;
}
evx_status nn_cuda(cudaError_t e) {
    if (e == cudaSuccess) return EVX_OK;
    g_nn_err = cudaGetErrorString(e);
    return EVX_ERR_CUDA;
}
bool dims_ok(int B, int X, int Y, int Z) {
    return B > 0 && X > 0 && Y > 0 && Z > 0 && Z % TZ == 0 && Y % TY == 0;
}

std::atomic<int> g_engine{EVX_NN_ENGINE_TCGEN05};
bool use_tcgen05() { return g_engine.load() == EVX_NN_ENGINE_TCGEN05; }

template <int CIN, int COUT, int EPI>
evx_status launch_conv(const ConvArgs& a0, cudaStream_t st) {
    if (CIN == 32 && COUT == 32 && EPI != EVX_NN_EPI_FIELD && use_tcgen05()) return nn_cuda(conv32_tc(a0, EPI, st, nn_sms()));
    ConvArgs a = a0;
    a.ntiles = a.B * a.X * (a.Y / TY) * (a.Z / TZ);
    const size_t smem = sizeof(__nv_bfloat16) * (27 * COUT * (CIN + 8) + HR * (TZ + 2) * (CIN + 8));
    cudaError_t e = cudaFuncSetAttribute(conv_fwd_kernel<CIN, COUT, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return nn_cuda(e);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, conv_fwd_kernel<CIN, COUT, EPI>, NTHR, smem);
    const int grid = std::min(a.ntiles, std::max(per, 1) * nn_sms());
    conv_fwd_kernel<CIN, COUT, EPI><<<grid, NTHR, smem, st>>>(a);
    return nn_cuda(cudaGetLastError());
}

template <int CIN, int COUT>
evx_status conv_epi(int epi, const ConvArgs& a, cudaStream_t st) {
    switch (epi) {
        case EVX_NN_EPI_PLAIN: return launch_conv<CIN, COUT, EVX_NN_EPI_PLAIN>(a, st);
        case EVX_NN_EPI_GELU: return launch_conv<CIN, COUT, EVX_NN_EPI_GELU>(a, st);
        case EVX_NN_EPI_RESID: return launch_conv<CIN, COUT, EVX_NN_EPI_RESID>(a, st);
        case EVX_NN_EPI_RESID32: return launch_conv<CIN, COUT, EVX_NN_EPI_RESID32>(a, st);
        case EVX_NN_EPI_GELU_BWD: return launch_conv<CIN, COUT, EVX_NN_EPI_GELU_BWD>(a, st);
        case EVX_NN_EPI_FIELD: return launch_conv<CIN, COUT, EVX_NN_EPI_FIELD>(a, st);
    }
    return nn_fail(EVX_ERR_ARG, "unknown epilogue");
}

template <int CIN, int COUT>
evx_status launch_wgrad(const WgradArgs& a0, float* dw, float* partials, size_t partial_floats,
                        cudaStream_t st) {
    WgradArgs a = a0;
    a.ntiles = a.B * a.X * (a.Y / TY) * (a.Z / TZ);
    const size_t smem = sizeof(__nv_bfloat16) * (HR * (TZ + 2) * (CIN + 8) + TY * TZ * (COUT + 8));
    cudaError_t e = cudaFuncSetAttribute(conv_wgrad_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return nn_cuda(e);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, conv_wgrad_kernel<CIN, COUT>, NTHR, smem);
    const size_t per_cta = (size_t)27 * COUT * CIN;
    int grid = std::min(a.ntiles, std::max(per, 1) * nn_sms());
    grid = std::max(1, std::min(grid, (int)(partial_floats / per_cta)));
    a.partials = partials;
    conv_wgrad_kernel<CIN, COUT><<<grid, NTHR, smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return nn_cuda(e);
    reduce_partials_f32<<<(int)((per_cta + 255) / 256), 256, 0, st>>>(partials, grid, (int)per_cta, dw);
    return nn_cuda(cudaGetLastError());
}

}  // namespace

extern "C" {

const char* evx_nn_last_error(void) { return g_nn_err; }

evx_status evx_nn_set_conv_engine(int engine) {
    if (engine != EVX_NN_ENGINE_TCGEN05 && engine != EVX_NN_ENGINE_MMA_SYNC)
        return nn_fail(EVX_ERR_ARG, "unknown convolution engine");
    g_engine.store(engine);
    return EVX_OK;
}

int evx_nn_conv_engine(void) { return g_engine.load(); }

evx_status evx_nn_check(void) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return nn_cuda(e);
    int flag = 0;
    if ((e = tc_take_timeout(&flag)) != cudaSuccess) return nn_cuda(e);
    if (!flag) return EVX_OK;
    return nn_fail(EVX_ERR_CUDA, "tensor-core convolution: a pipeline wait timed out (outputs invalid)");
}

evx_status evx_nn_conv3d(const void* in, const void* w, const float* bias, void* out, void* pre, const void* res,
                         int B, int X, int Y, int Z, int cin, int cout, int epilogue, void* stream) {
    if (!in || !w || !out) return nn_fail(EVX_ERR_ARG, "NULL pointer");
    if (!dims_ok(B, X, Y, Z)) return nn_fail(EVX_ERR_SIZE, "need Y even and Z a multiple of 64");
    if (epilogue == EVX_NN_EPI_GELU_BWD && !pre)
        return nn_fail(EVX_ERR_ARG, "the GELU-backward epilogue needs the pre-activation buffer");
    if (epilogue == EVX_NN_EPI_RESID && !res) return nn_fail(EVX_ERR_ARG, "residual epilogue needs res");
    if (epilogue == EVX_NN_EPI_RESID32 && (!pre || cout != 32))
        return nn_fail(EVX_ERR_ARG, "the FP32-stream epilogue needs the stream in pre and cout = 32");
    ConvArgs a{};
    a.in = (const __nv_bfloat16*)in;
    a.w = (const __nv_bfloat16*)w;
    a.bias = bias;
    a.out = out;
    a.pre = (__nv_bfloat16*)pre;
    a.res = (const __nv_bfloat16*)res;
    a.B = B;
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    cudaStream_t st = (cudaStream_t)stream;
    if (cin == 32 && cout == 32) return conv_epi<32, 32>(epilogue, a, st);
    if (cin == 16 && cout == 32) return conv_epi<16, 32>(epilogue, a, st);
    if (cin == 32 && cout == 16) return conv_epi<32, 16>(epilogue, a, st);
    if (cin == 16 && cout == 16) return conv_epi<16, 16>(epilogue, a, st);
    return nn_fail(EVX_ERR_ARG, "supported channel pairs: 16/32 -> 16/32");
}

// the lane-per-channel lift and projection: RY = 2 rows x 32 z per warp, two
// 256-thread CTAs per SM (measured at 8 x 256^3: projection 10.6 ms against 13.2 for
// one row per warp and 16.1 with one CTA per SM; lift 10.4 against 12.6 for one row)
constexpr int LANE_RY = 2;
static bool lane_path(int Y, int Z) { return Z % 32 == 0 && Y % LANE_RY == 0; }
static int lane_grid(int B, int X, int Y, int Z) {
    const long long warps = (long long)B * X * (Y / LANE_RY) * (Z / 32);
    return (int)std::min<long long>((warps + 7) / 8, 16LL * nn_sms());
}

evx_status evx_nn_lift(const float* f, float scale, const void* w, int cin, int cout, const float* bias, void* out,
                       int B, int X, int Y, int Z, void* stream) {
    if (!f || !w || !out) return nn_fail(EVX_ERR_ARG, "NULL pointer");
    if (B <= 0 || X <= 0 || Y <= 0 || Z <= 0) return nn_fail(EVX_ERR_SIZE, "empty grid");
    if (cout != 32 || cin < 1) return nn_fail(EVX_ERR_ARG, "lift: cout must be 32, cin >= 1");
    if (lane_path(Y, Z))
        lift_lane_kernel<false, LANE_RY, 2><<<lane_grid(B, X, Y, Z), 256, 0, (cudaStream_t)stream>>>(
            f, scale, (const __nv_bfloat16*)w, cin, bias, (__nv_bfloat16*)out, nullptr, B, X, Y, Z);
    else
        lift_direct_kernel<false><<<8 * nn_sms(), 256, 0, (cudaStream_t)stream>>>(
            f, scale, (const __nv_bfloat16*)w, cin, bias, (__nv_bfloat16*)out, nullptr, B, X, Y, Z);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_lift32(const float* f, float scale, const void* w, int cin, int cout, const float* bias, void* out,
                         float* out32, int B, int X, int Y, int Z, void* stream) {
    if (!f || !w || !out || !out32) return nn_fail(EVX_ERR_ARG, "NULL pointer");
    if (B <= 0 || X <= 0 || Y <= 0 || Z <= 0) return nn_fail(EVX_ERR_SIZE, "empty grid");
    if (cout != 32 || cin < 1) return nn_fail(EVX_ERR_ARG, "lift: cout must be 32, cin >= 1");
    if (lane_path(Y, Z))
        lift_lane_kernel<true, LANE_RY, 2><<<lane_grid(B, X, Y, Z), 256, 0, (cudaStream_t)stream>>>(
            f, scale, (const __nv_bfloat16*)w, cin, bias, (__nv_bfloat16*)out, out32, B, X, Y, Z);
    else
        lift_direct_kernel<true><<<8 * nn_sms(), 256, 0, (cudaStream_t)stream>>>(
            f, scale, (const __nv_bfloat16*)w, cin, bias, (__nv_bfloat16*)out, out32, B, X, Y, Z);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_project(const void* h, const void* w, int cin, int cout, const float* bias, float* out, int B,
                          int X, int Y, int Z, void* stream) {
    if (!h || !w || !out) return nn_fail(EVX_ERR_ARG, "NULL pointer");
    if (B <= 0 || X <= 0 || Y <= 0 || Z <= 0) return nn_fail(EVX_ERR_SIZE, "empty grid");
    if (cin != 32 || cout < 1) return nn_fail(EVX_ERR_ARG, "project: cin must be 32, cout >= 1");
    if (lane_path(Y, Z))
        project_lane_kernel<false, LANE_RY, 2><<<lane_grid(B, X, Y, Z), 256, 0, (cudaStream_t)stream>>>(
            (const __nv_bfloat16*)h, nullptr, (const __nv_bfloat16*)w, cout, bias, out, B, X, Y, Z);
    else
        project_direct_kernel<false><<<8 * nn_sms(), 256, 0, (cudaStream_t)stream>>>(
            (const __nv_bfloat16*)h, nullptr, (const __nv_bfloat16*)w, cout, bias, out, B, X, Y, Z);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_project32(const float* h32, const void* w, int cin, int cout, const float* bias, float* out, int B,
                            int X, int Y, int Z, void* stream) {
    if (!h32 || !w || !out) return nn_fail(EVX_ERR_ARG, "NULL pointer");
    if (B <= 0 || X <= 0 || Y <= 0 || Z <= 0) return nn_fail(EVX_ERR_SIZE, "empty grid");
    if (cin != 32 || cout < 1) return nn_fail(EVX_ERR_ARG, "project: cin must be 32, cout >= 1");
    if (lane_path(Y, Z))
        project_lane_kernel<true, LANE_RY, 2><<<lane_grid(B, X, Y, Z), 256, 0, (cudaStream_t)stream>>>(
            nullptr, h32, (const __nv_bfloat16*)w, cout, bias, out, B, X, Y, Z);
    else
        project_direct_kernel<true><<<8 * nn_sms(), 256, 0, (cudaStream_t)stream>>>(
            nullptr, h32, (const __nv_bfloat16*)w, cout, bias, out, B, X, Y, Z);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_conv3d_wgrad(const void* dy, const void* x, float* dw, float* partials, size_t partial_floats,
                               int B, int X, int Y, int Z, int cin, int cout, void* stream) {
    if (!dy || !x || !dw || !partials) return nn_fail(EVX_ERR_ARG, "NULL pointer");
    if (!dims_ok(B, X, Y, Z)) return nn_fail(EVX_ERR_SIZE, "need Y even and Z a multiple of 64");
    if (partial_floats < (size_t)27 * cin * cout) return nn_fail(EVX_ERR_ARG, "partials too small");
    WgradArgs a{};
    a.dy = (const __nv_bfloat16*)dy;
    a.x = (const __nv_bfloat16*)x;
    a.B = B;
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    cudaStream_t st = (cudaStream_t)stream;
    if (cin == 32 && cout == 32) return launch_wgrad<32, 32>(a, dw, partials, partial_floats, st);
    if (cin == 16 && cout == 32) return launch_wgrad<16, 32>(a, dw, partials, partial_floats, st);
    if (cin == 32 && cout == 16) return launch_wgrad<32, 16>(a, dw, partials, partial_floats, st);
    if (cin == 16 && cout == 16) return launch_wgrad<16, 16>(a, dw, partials, partial_floats, st);
    return nn_fail(EVX_ERR_ARG, "supported channel pairs: 16/32 -> 16/32");
}

evx_status evx_nn_bias_grad(const void* dy, long long nvox, int c, double* partials, int nparts, float* db,
                            void* stream) {
    if (!dy || !partials || !db || c <= 0 || c > 256 || nparts <= 0) return nn_fail(EVX_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const bool al16 = ((uintptr_t)dy & 15) == 0;  // the one-pass kernel reads 16-byte pieces
    if (c == 32 && al16)
        bias_grad_vec_kernel<32><<<nparts, 256, 0, st>>>((const __nv_bfloat16*)dy, nvox, partials);
    else if (c == 16 && al16)
        bias_grad_vec_kernel<16><<<nparts, 256, 0, st>>>((const __nv_bfloat16*)dy, nvox, partials);
    else
        bias_grad_kernel<<<nparts, 256, 0, st>>>((const __nv_bfloat16*)dy, nvox, c, partials);
    bias_grad_finish<<<1, 256, 0, st>>>(partials, nparts, c, db);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_flip_weights(const void* w, int cout, int cin, void* wt, void* stream) {
    if (!w || !wt) return nn_fail(EVX_ERR_ARG, "NULL pointer");
    flip_weights_kernel<<<64, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)w, cout, cin,
                                                               (__nv_bfloat16*)wt);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_field_to_act(const float* f, long long nvox, int c, float scale, void* act, void* stream) {
    if (!f || !act || c <= 0) return nn_fail(EVX_ERR_ARG, "bad argument");
    field_to_act_kernel<<<4 * nn_sms(), 256, 0, (cudaStream_t)stream>>>(f, nvox, c, scale, (__nv_bfloat16*)act);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_zero_mean_add(const float* base, const float* d, int nsamples, long long V, double* partials,
                                int nparts, float* out, void* stream) {
    if (!d || !out || !partials || nsamples <= 0 || nparts <= 0 || nparts > 4096)
        return nn_fail(EVX_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    sample_sum_kernel<<<dim3(nparts, nsamples), 256, 0, st>>>(d, V, partials, nparts);
    zero_mean_add_kernel<<<dim3(nparts, nsamples), 256, 0, st>>>(base, d, partials, nparts, V, out, nullptr);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_zero_mean_add_scaled(const float* base, const float* d, const double* scale, int nsamples, long long V,
                                       double* partials, int nparts, float* out, void* stream) {
    if (!d || !out || !partials || !scale || nsamples <= 0 || nparts <= 0 || nparts > 4096)
        return nn_fail(EVX_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    sample_sum_kernel<<<dim3(nparts, nsamples), 256, 0, st>>>(d, V, partials, nparts);
    zero_mean_add_kernel<<<dim3(nparts, nsamples), 256, 0, st>>>(base, d, partials, nparts, V, out, scale);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_nl_scale(const float* c, int nsamples, long long V, double* partials, int nparts, double* scale,
                           void* stream) {
    if (!c || !partials || !scale || nsamples <= 0 || nsamples > 32 || V <= 0 || nparts <= 0 || nparts > 4096)
        return nn_fail(EVX_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    sample_sum_kernel<<<dim3(nparts, nsamples), 256, 0, st>>>(c, V, partials, nparts);
    nl_moments_kernel<<<dim3(nparts, nsamples), 256, 0, st>>>(c, V, partials, nparts, partials + (long long)nsamples * nparts);
    nl_scale_kernel<<<1, 32, 0, st>>>(partials + (long long)nsamples * nparts, nparts, nsamples, scale);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_mse(const float* p, const float* t, long long n, float grad_scale, float* grad, double* partials,
                      int nparts, double* d_sum, void* stream) {
    if (!p || !t || !partials || !d_sum || nparts <= 0) return nn_fail(EVX_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    mse_kernel<<<nparts, 256, 0, st>>>(p, t, n, grad_scale, grad, partials);
    sum_partials_kernel<<<1, 32, 0, st>>>(partials, nparts, d_sum);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_abs_sum(const float* x, long long n, double* partials, int nparts, double* d_sum, void* stream) {
    if (!x || n <= 0 || !partials || !d_sum || nparts <= 0) return nn_fail(EVX_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    abs_sum_kernel<<<nparts, 256, 0, st>>>(x, n, partials);
    sum_partials_kernel<<<1, 32, 0, st>>>(partials, nparts, d_sum);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       int step, void* wbf, void* stream) {
    if (!w || !g || !m || !v || n <= 0 || step < 1) return nn_fail(EVX_ERR_ARG, "bad argument");
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<std::min(4 * nn_sms(), (n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        w, g, m, v, n, lr, b1, b2, eps, bc1, bc2, (__nv_bfloat16*)wbf);
    return nn_cuda(cudaGetLastError());
}

evx_status evx_nn_f32_to_bf16(const float* a, int n, void* b, void* stream) {
    if (!a || !b || n <= 0) return nn_fail(EVX_ERR_ARG, "bad argument");
    f32_to_bf16_kernel<<<std::min(4 * nn_sms(), (n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        a, n, (__nv_bfloat16*)b);
    return nn_cuda(cudaGetLastError());
}

}  // extern "C"
