// Fast paths of the four step passes for lengths L = R1 * TP: R1 = 32 with TP a
// power of two 2 .. 32 (L = 64 .. 1024), and R1 = 20 with TP = 20 (L = 400) or
// TP = 10 (the z pass of nz = 400, M = 200); the z pass works on M = nz/2.
//
// Four-step FFT of a length-L pencil, n = n2 + TP n1 (n2 < TP, n1 < R1):
//   pass A:  Y[n2][k1] = sum_{n1} x[n2 + TP n1] w_R1^{n1 k1}        (DFT-R1 in registers)
//   twiddle: Y[n2][k1] *= w_L^{n2 k1}
//   pass B:  X[k1 + R1 k2] = sum_{n2} Y[n2][k1] w_TP^{n2 k2}         (R1/TP DFT-TP per thread)
// Thread n2 of a pencil owns the R1 values x[n2 + TP n1] ("n2 ownership"); after
// the one shared-memory transpose thread j owns X[k1 + R1 k2] for
// k1 in [j R1/TP, (j+1) R1/TP), all k2 ("block ownership"). The inverse walks the
// same way back. Global loads and stores go straight from/to registers in
// both ownerships (each warp touches whole 64-byte row segments) for the z
// pass, whose next tile is prefetched with cp.async; the x and y passes move
// whole tiles with TMA (below). CTAs are persistent (one wave).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "evx_fast_dev.cuh"

namespace evx {
namespace fast {
// ------------------------------------------------ z pass: C2R, c^3 - c, R2C
template <int R1, int TP, int NTZ, bool GS, bool ADJ>
__global__ void __launch_bounds__(NTZ, 512 / NTZ) fzstep_kernel(ZPassArgs a, int ntiles) {
    // GS (Allen-Cahn): also sum g(c) - g(cbar) over the grid, FP32 per thread and
    // tile, FP64 across tiles, one FP64 partial per CTA in a.gsum[blockIdx.x].
    // ADJ (the adjoint's z pass): the pointwise stage multiplies the real field by
    // g'(c_n) = 3 c_n^2 - 1, c_n read from the real rows a.cn (memory row order)
    constexpr int M = R1 * TP, NB = R1 / TP, RPC = NTZ / TP, ZPAD = zpad(R1, TP), RS = M + TP * ZPAD;
    extern __shared__ float4 smem4[];
    const int Zp = a.Zp, Zh = a.Zp / 2;
    // row stride of the shared tile: >= Zp and RS, and = TP (mod 16) so that the
    // rows a warp spans fall on different banks
    const int BS = TP + (((Zp > RS ? Zp : RS) - TP + 15) & ~15);
    // One tile buffer serves as cp.async destination (rows of Zp), transpose
    // space (rows of RS) and is refilled for the next tile as soon as the last
    // transpose has been read: 46 KB per CTA at M = 512, four CTAs per SM.
    float2* buf = reinterpret_cast<float2*>(smem4);  // [RPC][BS]
    float2* tA = buf + RPC * BS;                      // [M] complex FFT twiddles (n2 ownership)
    float2* tB = tA + M;                              // [M] (block ownership)
    float2* rtws = tB + M;                            // [M + 1] real-transform twiddles
    float2* xz = rtws + M + 1;                        // [RPC][zxs(M, TP)] R2C partner rows (R1 != 32)
    const int n2 = threadIdx.x % TP, r = threadIdx.x / TP;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    fill_twiddles<R1, TP>(tA, tB, a.tw, NTZ);
    for (int i = threadIdx.x; i <= M; i += NTZ) rtws[i] = a.rtw[i];
    // rows to warps, 16-byte pieces of a row to lanes (no division by the runtime pitch)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto issue = [&](int tl) {
        const long long row0 = (long long)tl * RPC;
        for (int rr = warp; rr < RPC; rr += NTZ / 32) {
            const bool ok = row0 + rr < a.nrows;
            const float2* src = a.in + (ok ? (row0 + rr) * Zp : 0);
            for (int q = lane; q < Zh; q += 32) cp_async16(buf + rr * BS + 2 * q, ok ? src + 2 * q : a.in, ok ? 16 : 0);
        }
        cp_commit();
    };
    issue(tile);
    const double cbd = a.cbar ? *a.cbar : 0.0;
    const float cb = (float)cbd;
    const float cbl = (float)(cbd - (double)cb);
    // g'(cbar); 0 with a.nl_only: the pass then forms the nonlinear remainder
    // N = d^2 (3 cbar + d) alone (the block propagator's input)
    const float gp = a.nl_only ? 0.f : (float)(3.0 * cbd * cbd - 1.0);
    const float c3 = (float)(3.0 * cbd);
    const float s = a.scale;
    auto slot = [&](int rr, int nn, int aa) { return rr * BS + aa * TP + nn + aa / NB * ZPAD; };
    double gacc = 0.0;
    for (; tile < ntiles; tile += gridDim.x) {
        const long long row0 = (long long)tile * RPC;
        cp_wait<0>();
        __syncthreads();
        // C2R pre-processing: Z[k] = (X_k + conj X_{M-k}) + i e^{+2 pi i k/nz} (X_k - conj X_{M-k})
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
            const int k = n2 + TP * n1;
            float2 xk = buf[r * BS + k], xm = buf[r * BS + (M - k)];
            if (k == 0) {
                xk.y = 0.f;
                xm.y = 0.f;
            }
            v[n1] = c2r_pre(xk, xm, rtws[k]);
        }
        __syncthreads();  // tile read: buf becomes transpose space
        // inverse complex FFT of length M
        Dft<R1, 1>::run(v);
        twiddle_a<R1, TP, 1>(v, n2, tA);
#pragma unroll
        for (int aa = 0; aa < R1; ++aa) buf[slot(r, n2, aa)] = v[aa];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) v[i * TP + c] = buf[slot(r, c, n2 * NB + i)];
        pass_b<R1, TP, 1>(v);
        // real-space samples z[m] = c[2m] + i c[2m+1], m = k1 + 32 k2
        const long long row = row0 + r;
        const bool rowok = row < a.nrows;
        float gtile = 0.f;  // rows past the end were loaded as zeros: d = 0 adds nothing
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) {
                const float2 z = v[i * TP + c];
                const float d0 = z.x * s, d1 = z.y * s;  // c - cbar (the state has no k = 0 mode)
                if (ADJ) {  // lambda-side field times g'(c_n)
                    const float2 cn = rowok ? reinterpret_cast<const float2*>(a.cn + row * a.cnpitch)[n2 * NB + i + R1 * c]
                                            : make_float2(0.f, 0.f);
                    v[i * TP + c] = make_float2(d0 * fmaf(3.f * cn.x, cn.x, -1.f), d1 * fmaf(3.f * cn.y, cn.y, -1.f));
                    continue;
                }
                if (a.rout && rowok)
                    reinterpret_cast<float2*>(a.rout + row * a.rpitch)[n2 * NB + i + R1 * c] =
                        make_float2(fmaf(z.x, s, cbl) + cb, fmaf(z.y, s, cbl) + cb);
                // g(c) - g(cbar) = d (g'(cbar) + d (3 cbar + d)); the constant g(cbar) only
                // feeds the k = 0 mode, which the update multiplies by b(0) = 0
                v[i * TP + c] = make_float2(d0 * fmaf(d0, c3 + d0, gp), d1 * fmaf(d1, c3 + d1, gp));
                if (GS) gtile += v[i * TP + c].x + v[i * TP + c].y;
            }
        if (GS) gacc += (double)gtile;
        // forward complex FFT of length M from block ownership (m = a + 32 b)
        pass_b<R1, TP, -1>(v);
        twiddle_b<R1, TP, -1>(v, n2, tB);
        __syncthreads();  // block-ownership reads of the first transpose done
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) buf[slot(r, c, n2 * NB + i)] = v[i * TP + c];
        __syncthreads();
#pragma unroll
        for (int aa = 0; aa < R1; ++aa) v[aa] = buf[slot(r, n2, aa)];
        __syncthreads();  // buf free: fetch the next tile while this one finishes
        if (tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x);
        Dft<R1, -1>::run(v);
        // R2C post-processing (partner exchange by warp shuffle or the shared row xz)
        r2c_store<R1, TP>(v, n2, xz + r * zxs(M, TP), a.out + row * Zp, rowok, rtws);
    }
    if (GS) {  // fixed-order CTA reduction of the FP64 sums
        __shared__ double red[NTZ / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gacc += __shfl_down_sync(0xffffffffu, gacc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gacc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < NTZ / 32; ++w) t += red[w];
            a.gsum[blockIdx.x] = t;
        }
    }
}

// ----------------------------------------- z transforms alone (R2C, C2R)
// The two halves of fzstep_kernel as kernels of their own, for the field
// I/O of the spectral models and for the variable-mobility step: same tile
// (RPC rows of M = nz/2 complex samples per CTA, one shared buffer for the
// rows and the transpose), same four-step FFT and real-transform twiddles.
// Real rows are the caller's C-order rows when a.map_rows (row r of the
// y-blocked spectrum is caller row user_row(r)), pitch a.rpitch floats.

// R2C: real rows (minus the FP64 mean when a.cbar) -> complex rows a.out
template <int R1, int TP, int NTZ>
__global__ void __launch_bounds__(NTZ, 512 / NTZ) fr2c_kernel(ZPassArgs a, int ntiles) {
    constexpr int M = R1 * TP, NB = R1 / TP, RPC = NTZ / TP, ZPAD = zpad(R1, TP), RS = M + TP * ZPAD;
    extern __shared__ float4 smem4[];
    const int Zp = a.Zp;
    const int BS = TP + (((Zp > RS ? Zp : RS) - TP + 15) & ~15);
    float2* buf = reinterpret_cast<float2*>(smem4);  // [RPC][BS]
    float2* tA = buf + RPC * BS;
    float2* tB = tA + M;
    float2* rtws = tB + M;
    float2* xz = rtws + M + 1;  // [RPC][zxs(M, TP)] R2C partner rows (R1 != 32)
    const int n2 = threadIdx.x % TP, r = threadIdx.x / TP;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    fill_twiddles<R1, TP>(tA, tB, a.tw, NTZ);
    for (int i = threadIdx.x; i <= M; i += NTZ) rtws[i] = a.rtw[i];
    // rows to warps (the caller's row once per row), 16-byte chunks of 4 floats to lanes
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto issue = [&](int tl) {
        const long long row0 = (long long)tl * RPC;
        for (int rr = warp; rr < RPC; rr += NTZ / 32) {
            const long long row = row0 + rr;
            const bool ok = row < a.nrows;
            const long long ur = ok ? (a.map_rows ? user_row(row, a.YB, a.nxr, a.nyr) : row) : 0;
            const float* src = a.rin + ur * a.rpitch;
            for (int q = lane; q < M / 2; q += 32) cp_async16(buf + rr * BS + 2 * q, ok ? src + 4 * q : a.rin, ok ? 16 : 0);
        }
        cp_commit();
    };
    issue(tile);
    const double cbd = a.cbar ? *a.cbar : 0.0;
    const float hi = (float)cbd, lo = (float)(cbd - (double)hi);
    const bool sub = a.cbar != nullptr;
    auto slot = [&](int rr, int nn, int aa) { return rr * BS + aa * TP + nn + aa / NB * ZPAD; };
    for (; tile < ntiles; tile += gridDim.x) {
        const long long row0 = (long long)tile * RPC;
        cp_wait<0>();
        __syncthreads();
        // samples z[m] = c[2m] + i c[2m+1] in block ownership (m = n2 NB + i + 32 c)
        float2 v[R1];
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) {
                float2 z = buf[r * BS + n2 * NB + i + R1 * c];
                if (sub) {  // (x - hi) - lo: x - hi is exact for x within a factor 2 of hi
                    z.x = (z.x - hi) - lo;
                    z.y = (z.y - hi) - lo;
                }
                v[i * TP + c] = z;
            }
        __syncthreads();  // rows read: buf becomes transpose space
        pass_b<R1, TP, -1>(v);
        twiddle_b<R1, TP, -1>(v, n2, tB);
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) buf[slot(r, c, n2 * NB + i)] = v[i * TP + c];
        __syncthreads();
#pragma unroll
        for (int aa = 0; aa < R1; ++aa) v[aa] = buf[slot(r, n2, aa)];
        __syncthreads();  // buf free: fetch the next tile while this one finishes
        if (tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x);
        Dft<R1, -1>::run(v);
        // R2C post-processing (as in the z step)
        const long long row = row0 + r;
        const bool rowok = row < a.nrows;
        r2c_store<R1, TP>(v, n2, xz + r * zxs(M, TP), a.out + row * Zp, rowok, rtws);
    }
}

// C2R: complex rows a.in -> real rows c = z / (ny nz) + cbar; ACC adds to the
// rows instead; PART: FP64 partial per CTA of sum (c^2 - 1)^2 in a.partials
template <int R1, int TP, int NTZ, bool ACC, bool PART>
__global__ void __launch_bounds__(NTZ, 512 / NTZ) fc2r_kernel(ZPassArgs a, int ntiles) {
    constexpr int M = R1 * TP, NB = R1 / TP, RPC = NTZ / TP, ZPAD = zpad(R1, TP), RS = M + TP * ZPAD;
    extern __shared__ float4 smem4[];
    const int Zp = a.Zp, Zh = a.Zp / 2;
    const int BS = TP + (((Zp > RS ? Zp : RS) - TP + 15) & ~15);
    float2* buf = reinterpret_cast<float2*>(smem4);  // [RPC][BS]
    float2* tA = buf + RPC * BS;
    float2* tB = tA + M;
    float2* rtws = tB + M;
    const int n2 = threadIdx.x % TP, r = threadIdx.x / TP;
    int tile = blockIdx.x;
    double acc = 0.0;
    if (tile < ntiles) {
        fill_twiddles<R1, TP>(tA, tB, a.tw, NTZ);
        for (int i = threadIdx.x; i <= M; i += NTZ) rtws[i] = a.rtw[i];
    }
    // rows to warps, 16-byte pieces of a row to lanes (no division by the runtime pitch)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto issue = [&](int tl) {
        const long long row0 = (long long)tl * RPC;
        for (int rr = warp; rr < RPC; rr += NTZ / 32) {
            const bool ok = row0 + rr < a.nrows;
            const float2* src = a.in + (ok ? (row0 + rr) * Zp : 0);
            for (int q = lane; q < Zh; q += 32) cp_async16(buf + rr * BS + 2 * q, ok ? src + 2 * q : a.in, ok ? 16 : 0);
        }
        cp_commit();
    };
    if (tile < ntiles) issue(tile);
    const double cbd = a.cbar ? *a.cbar : 0.0;
    const float cb = (float)cbd, cbl = (float)(cbd - (double)cb);
    const float s = a.scale;
    auto slot = [&](int rr, int nn, int aa) { return rr * BS + aa * TP + nn + aa / NB * ZPAD; };
    for (; tile < ntiles; tile += gridDim.x) {
        const long long row0 = (long long)tile * RPC;
        cp_wait<0>();
        __syncthreads();
        // C2R pre-processing: Z[k] = (X_k + conj X_{M-k}) + i e^{+2 pi i k/nz} (X_k - conj X_{M-k})
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
            const int k = n2 + TP * n1;
            float2 xk = buf[r * BS + k], xm = buf[r * BS + (M - k)];
            if (k == 0) {
                xk.y = 0.f;
                xm.y = 0.f;
            }
            v[n1] = c2r_pre(xk, xm, rtws[k]);
        }
        __syncthreads();  // tile read: buf becomes transpose space
        Dft<R1, 1>::run(v);
        twiddle_a<R1, TP, 1>(v, n2, tA);
#pragma unroll
        for (int aa = 0; aa < R1; ++aa) buf[slot(r, n2, aa)] = v[aa];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) v[i * TP + c] = buf[slot(r, c, n2 * NB + i)];
        pass_b<R1, TP, 1>(v);
        __syncthreads();  // transpose reads done: buf stages the real rows in natural order
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) {
                const float2 z = v[i * TP + c];
                buf[r * BS + n2 * NB + i + R1 * c] = make_float2(fmaf(z.x, s, cbl) + cb, fmaf(z.y, s, cbl) + cb);
            }
        __syncthreads();
        for (int rr = warp; rr < RPC; rr += NTZ / 32) {  // rows to warps, coalesced 16-byte stores by lanes
            const long long row = row0 + rr;
            if (row >= a.nrows) continue;
            const long long ur = a.map_rows ? user_row(row, a.YB, a.nxr, a.nyr) : row;
            float4* drow = reinterpret_cast<float4*>(a.rout + ur * a.rpitch);
            for (int q = lane; q < M / 2; q += 32) {
                float4* dst = drow + q;
                float4 val = *reinterpret_cast<const float4*>(buf + rr * BS + 2 * q);
                if (ACC) {
                    const float4 prev = *dst;
                    val.x += prev.x;
                    val.y += prev.y;
                    val.z += prev.z;
                    val.w += prev.w;
                }
                *dst = val;
                if (PART) {
                    const double q0 = (double)val.x * val.x - 1.0, q1 = (double)val.y * val.y - 1.0;
                    const double q2 = (double)val.z * val.z - 1.0, q3 = (double)val.w * val.w - 1.0;
                    acc += q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3;
                }
            }
        }
        __syncthreads();  // staged rows stored: buf free for the next tile
        if (tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x);
    }
    if (PART) {  // fixed-order CTA reduction
        __shared__ double red[NTZ / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < NTZ / 32; ++w) t += red[w];
            a.partials[blockIdx.x] = t;
        }
    }
}

// ------------------------------------------------------------ TMA helpers
// Tile loads and stores of the strided passes go through the tensor memory
// accelerator: one thread issues cp.async.bulk.tensor boxes of up to 256 rows
// of 8 complex values (64 bytes); loads complete on an mbarrier, stores are
// bulk groups read out of a shared-memory staging tile. Every wait is bounded:
// on timeout the kernel records it in g_timeout (mbar_wait_or_abort).
__device__ int g_timeout;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// wait for the phase of the given parity; false after about 2^32 cycles (~2 s)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > (1LL << 32)) return false;
    }
}

// bounded wait that gives up at once when another thread of the CTA already has:
// the first thread to run out of time sets *abort_flag and g_timeout. Callers do
// not leave their tile loop on failure (every thread keeps the same barrier
// sequence, so no vote is needed); the remaining tiles are processed from stale
// buffers without waiting and the host reports the flag.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > (1LL << 32)) {
            *abort_flag = 1;
            atomicExch(&g_timeout, 1);
            return false;
        }
    }
}
// 4D tensor {kz, y within block, x, y block} of a y-blocked half spectrum
__device__ __forceinline__ void tma_load4(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store4(const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                           const void* src) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// y pass with TMA: boxes {8, 32 (y in block), 1 (x), BOX/32 (y blocks)} cover
// BOX consecutive y rows of one x line (y blocks of 32 rows). NBUF tile buffers
// take the loads: with two (L = 1024, one CTA per SM) the tile after next is
// already on its way while a tile is transformed.
template <int R1, int TP, int DIR, int NBUF>
__global__ void __launch_bounds__(8 * TP) fspass_tma_kernel(SPassArgs a, int ntiles,
                                                            const __grid_constant__ CUtensorMap min,
                                                            const __grid_constant__ CUtensorMap mout) {
    constexpr int L = R1 * TP, NB = R1 / TP, XB = (L + TP) * 8, BOX = ybox(R1, L), NBOX = L / BOX;
    extern __shared__ __align__(1024) float4 smem4[];
    float2* bufs = reinterpret_cast<float2*>(smem4);  // [NBUF][L][8] TMA destinations
    float2* xb = bufs + NBUF * L * 8;                 // transpose, then store staging
    float2* tA = xb + XB;                             // [L] twiddles (n2 ownership)
    float2* tB = tA + L;                              // [L] twiddles (block ownership)
    uint64_t* bar = reinterpret_cast<uint64_t*>(tB + L);  // [NBUF]
    const int p = threadIdx.x & 7, n2 = threadIdx.x >> 3;
    const int nchunks = a.nchunks;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    fill_twiddles<R1, TP>(tA, tB, a.tw, 8 * TP);
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(bar + b, 1);
        s_abort = 0;
    }
    __syncthreads();
    auto issue = [&](int tl, int b) {
        const int outer = tl / nchunks, chunk = tl - outer * nchunks;
        fence_async_smem();
        mbar_expect_tx(bar + b, L * 8 * sizeof(float2));
#pragma unroll
        for (int q = 0; q < NBOX; ++q)
            tma_load4(bufs + (b * L + q * BOX) * 8, &min, chunk * 8, 0, outer, q * BOX / a.YB, bar + b);
    };
    if (threadIdx.x == 0)
        for (int b = 0; b < NBUF && tile + b * (int)gridDim.x < ntiles; ++b) issue(tile + b * gridDim.x, b);
    uint32_t parity = 0;
    for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
        const int b = NBUF == 1 ? 0 : it % NBUF;
        float2* buf = bufs + b * L * 8;
        mbar_wait_or_abort(bar + b, parity, &s_abort);
        if (b == NBUF - 1) parity ^= 1;
        float2 v[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[n1] = buf[(n2 + TP * n1) * 8 + p];
        if (threadIdx.x == 0) bulk_wait_read0();  // previous store has left the staging tile
        __syncthreads();
        const int next = tile + NBUF * gridDim.x;
        if (threadIdx.x == 0 && next < ntiles) issue(next, b);
        Dft<R1, DIR>::run(v);
        twiddle_a<R1, TP, DIR>(v, n2, tA);
        t1_s<R1, TP, 8>(v, xb, n2, p);
        pass_b<R1, TP, DIR>(v);
        __syncthreads();  // transpose reads done: xb becomes the store staging tile
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) xb[(n2 * NB + i + R1 * c) * 8 + p] = v[i * TP + c];
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int outer = tile / nchunks, chunk = tile - outer * nchunks;
#pragma unroll
            for (int q = 0; q < NBOX; ++q)
                tma_store4(&mout, chunk * 8, 0, outer, q * BOX / a.YB, xb + q * BOX * 8);
            bulk_commit();
        }
    }
    if (threadIdx.x == 0) bulk_wait0();
}

// x pass + update with TMA: boxes {8, 1, BOX (x), 1} of 8 columns. MODE 0:
// Cahn-Hilliard, 1: Allen-Cahn, 2: preconditioner only (S' = F_x^-1 (dt / (1 +
// dt M0 kappa |k|^4) F_x W), S not read; the variable-mobility model's spectral step),
// 3: Cahn-Hilliard block propagator (evx_ch_block).
// Two tile buffers, (L + TP) x 8 each, receive W and S by TMA. SEP (L = 1024):
// a third buffer of the same size takes the transposes and stages the result,
// and each field's next tile is loaded as soon as the current one is in
// registers (one 256-thread CTA per SM). Otherwise each tile buffer, once read,
// is that FFT's transpose space and the S buffer stages the result. The next W
// is then loaded after the W transposes, the next S once the store has read the
// staging tile (the next tile's W phase covers that load). Without the third
// buffer, three CTAs fit on an SM for L <= 512 and L = 400.
template <int R1, int TP, int MODE, bool SEP>
__global__ void __launch_bounds__(8 * TP, SEP ? 1 : (8 * TP >= 128 ? 3 : 1))
    fxupd_tma_kernel(XUpdArgs a, int ntiles, const __grid_constant__ CUtensorMap mW,
                     const __grid_constant__ CUtensorMap mS, const __grid_constant__ CUtensorMap mO) {
    constexpr int P = 8, L = R1 * TP, NB = R1 / TP, XB = (L + TP) * P, BOX = xbox(L), NBOX = L / BOX, NT = P * TP;
    constexpr int FWD_UNROLL = SEP ? 1 : 2;  // see the forward loop below
    static_assert(L % BOX == 0 && BOX <= 256, "x-pass TMA box");
    extern __shared__ __align__(1024) float4 smem4[];
    float2* bufW = reinterpret_cast<float2*>(smem4);  // [XB] W tile (then its transposes unless SEP)
    float2* bufS = bufW + XB;                          // [XB] S tile (then transposes and staging unless SEP)
    float2* xb = bufS + XB;                            // [XB] transposes and staging (SEP only)
    float2* tA = SEP ? xb + XB : xb;                   // [L] twiddles (n2 ownership)
    float2* tB = NB == 1 ? tA : tA + L;                // [L] block ownership (the same table when TP = R1)
    float* k2xs = reinterpret_cast<float*>(tA + (NB == 1 ? L : 2 * L));  // [L] |k_x|^2 (SEP only)
    uint64_t* bars = reinterpret_cast<uint64_t*>(k2xs + (SEP ? L : 0));  // [0] W, [1] S
    const float* k2x = SEP ? k2xs : a.k2x;             // read through L1 otherwise
    float2* const xW = SEP ? xb : bufW;                // transpose space of F_x W
    float2* const xS = SEP ? xb : bufS;                // of F_x S, F_x^-1 and the store staging
    const int p = threadIdx.x % P, n2 = threadIdx.x / P;
    const int nchunks = a.nchunks;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    fill_twiddles<R1, TP>(tA, tB, a.tw, NT);
    if (SEP)
        for (int i = threadIdx.x; i < L; i += NT) k2xs[i] = a.k2x[i];
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        mbar_init(bars + 0, 1);
        mbar_init(bars + 1, 1);
        s_abort = 0;
    }
    __syncthreads();
    const int YB = a.YB;
    auto issue = [&](const CUtensorMap* m, float2* buf, uint64_t* bar, int tl) {
        const int ky = tl / nchunks, chunk = tl - ky * nchunks;
        fence_async_smem();
        mbar_expect_tx(bar, L * P * sizeof(float2));
#pragma unroll
        for (int b = 0; b < NBOX; ++b)
            tma_load4(buf + b * BOX * P, m, chunk * P, ky % YB, b * BOX, ky / YB, bar);
    };
    constexpr bool AC = MODE == 1, PRE = MODE == 2, BLK = MODE == 3;
    // MODE 3 (block of a.nblk steps, linear part exact, nonlinear remainder frozen):
    // L = (1 - dt M |k|^2 g'(cbar)) / D, c_hat' = L^n c_hat + B (sum_{j<n} L^j) N_hat
    const float gpb = BLK ? (float)(3.0 * (*a.cbar) * (*a.cbar) - 1.0) : 0.f;
    auto blk = [&](float k2, float& Pn, float& BS) {
        const float Dinv = rcp_approx(fmaf(a.dtMk, k2 * k2, 1.f));
        const float Lk = fmaf(-a.dtM * k2, gpb, 1.f) * Dinv;
        float P = 1.f, S = 0.f;
        for (int j = 0; j < a.nblk; ++j) {
            S += P;
            P *= Lk;
        }
        Pn = P;
        BS = -a.dtM * k2 * Dinv * S;
    };
    if (threadIdx.x == 0) {
        issue(&mW, bufW, bars + 0, tile);
        if (!PRE) issue(&mS, bufS, bars + 1, tile);
    }
    uint32_t parity = 0;
    const float ndtM = -a.dtM;
    for (; tile < ntiles; tile += gridDim.x) {
        const int ky = tile / nchunks, chunk = tile - ky * nchunks;
        const int next = tile + gridDim.x;
        // ---- f = 0: g_hat = F_x W, kept as G = -dt M |k|^2 g_hat (Allen-Cahn: -dt L g_hat);
        //      f = 1: c_hat = F_x S and the update. With SEP (L = 1024) the loop is not
        //      unrolled: both fields run through one copy of the forward FFT, which cut the
        //      instruction-fetch stalls of this large kernel (x pass 3.15 -> 3.04 ms at 1024^3).
        const int kz = chunk * P + p;
        const bool valid = kz < a.ncols;
        const float k2yz = a.k2y[ky] + (valid ? a.k2z[kz] : 0.f);
        float2 v[R1], G[R1];
#pragma unroll FWD_UNROLL
        for (int f = 0; f < (PRE ? 1 : 2); ++f) {
            float2* const buf = f ? bufS : bufW;
            mbar_wait_or_abort(bars + f, parity, &s_abort);
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) v[n1] = buf[(n2 + TP * n1) * P + p];
            if (SEP && f == 0 && threadIdx.x == 0) bulk_wait_read0();
            __syncthreads();
            if (SEP && threadIdx.x == 0 && next < ntiles) issue(f ? &mS : &mW, buf, bars + f, next);
            Dft<R1, -1>::run(v);
            twiddle_a<R1, TP, -1>(v, n2, tA);
            t1_s<R1, TP, P>(v, f ? xS : xW, n2, p);
            pass_b<R1, TP, -1>(v);
            if (f == 0) {
                if (!SEP) {
                    __syncthreads();
                    if (threadIdx.x == 0 && next < ntiles) issue(&mW, bufW, bars + 0, next);
                }
#pragma unroll
                for (int i = 0; i < NB; ++i)
#pragma unroll
                    for (int c = 0; c < TP; ++c) {
                        const float k2g = (SEP ? k2x[n2 * NB + i + R1 * c] : __ldg(k2x + n2 * NB + i + R1 * c)) + k2yz;
                        float fa;
                        if (BLK) {
                            float Pn;
                            blk(k2g, Pn, fa);
                            fa *= a.invL;
                        } else {
                            fa = PRE  ? a.dtM * a.invL * rcp_approx(fmaf(a.dtMk, k2g * k2g, 1.f))
                                 : AC ? ndtM
                                      : ndtM * k2g;
                        }
                        G[i * TP + c] = cscale(v[i * TP + c], fa);
                    }
            } else {
#pragma unroll
                for (int i = 0; i < NB; ++i)
#pragma unroll
                    for (int c = 0; c < TP; ++c) {
                        const float k2 = (SEP ? k2x[n2 * NB + i + R1 * c] : __ldg(k2x + n2 * NB + i + R1 * c)) + k2yz;
                        if (BLK) {
                            float Pn, BS;
                            blk(k2, Pn, BS);
                            v[i * TP + c] = cadd(cscale(v[i * TP + c], Pn * a.invL), G[i * TP + c]);
                        } else {
                            const float fa = a.invL * rcp_approx(fmaf(a.dtMk, AC ? k2 : k2 * k2, 1.f));
                            v[i * TP + c] = cscale(cadd(v[i * TP + c], G[i * TP + c]), fa);
                        }
                    }
            }
        }
        parity ^= 1;
        if (PRE) {
#pragma unroll
            for (int q = 0; q < R1; ++q) v[q] = G[q];
        }
        if (ky == 0 && kz == 0 && n2 == 0) v[0] = make_float2(0.f, 0.f);
        // ---- S' = F_x^-1 c_hat'
        pass_b<R1, TP, 1>(v);
        twiddle_b<R1, TP, 1>(v, n2, tB);
        __syncthreads();  // earlier transpose reads of xS done
        t2_s<R1, TP, P>(v, xS, n2, p);
        Dft<R1, 1>::run(v);
        __syncthreads();  // transpose reads done: xS becomes the store staging tile
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) xS[(n2 + TP * n1) * P + p] = v[n1];
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int b = 0; b < NBOX; ++b)
                tma_store4(&mO, chunk * P, ky % YB, b * BOX, ky / YB, xS + b * BOX * P);
            bulk_commit();
            if (!SEP) {
                bulk_wait_read0();  // the store has read the staging tile: bufS takes the next S
                if (!PRE && next < ntiles) issue(&mS, bufS, bars + 1, next);
            }
        }
    }
    if (threadIdx.x == 0) bulk_wait0();
}

// ------------------------------------------------------ adjoint x pass
// One tile = 8 columns (kz) of one ky line, all nx rows; 8 TP threads, thread
// (p, n2) owns column p and rows n2 + TP n1 (loads and stores go straight
// between global memory and registers; 64-byte row segments per 8 threads).
// lambda_hat = F_x Lambda stays in registers while F_x S_{n+1} and F_x G_n pass
// through for the parameter-gradient partials; then P = F_x^-1(a lambda_hat)/nx
// and T = F_x^-1(b lambda_hat)/nx, a = 1/D, b = -dt M |k|^2 / D, D = 1 + dt M kappa |k|^4.
// Partials (FP32 per thread, FP64 per CTA):
//   kappa: w Re(conj(lambda_hat) c_hat) (-dt M |k|^4 / D)
//   M:     w Re(conj(lambda_hat) c_hat) (-dt kappa |k|^4 / D) + w Re(conj(lambda_hat) g_hat) (-dt |k|^2 / D)
// with w = 1 for kz = 0 or M and 2 otherwise (Hermitian half spectrum).
template <int R1, int TP>
__global__ void __launch_bounds__(8 * TP) fxadj_kernel(XAdjArgs a) {
    constexpr int P = 8, L = R1 * TP, NB = R1 / TP, NT = P * TP;
    extern __shared__ __align__(1024) float4 smem4[];
    float2* xb = reinterpret_cast<float2*>(smem4);  // [(L + TP) P] transposes
    float2* tA = xb + (L + TP) * P;
    float2* tB = NB == 1 ? tA : tA + L;
    fill_twiddles<R1, TP>(tA, tB, a.tw, NT);
    __shared__ double red[2][NT / 32 + 1];
    const int p = threadIdx.x % P, n2 = threadIdx.x / P;
    const int chunk = blockIdx.x, ky = blockIdx.y;
    const int kz = chunk * P + p;
    const bool valid = kz < a.ncols;
    const long long base = split_off(ky, a.YB, a.os, a.os2) + (long long)chunk * P + p;
    const float k2yz = a.k2y[ky] + (valid ? a.k2z[kz] : 0.f);
    const float w = (kz == 0 || kz == a.M) ? 1.f : 2.f;
    __syncthreads();
    auto forward = [&](const float2* f, float2 (&v)[R1]) {
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1)
            v[n1] = valid ? f[base + (long long)(n2 + TP * n1) * a.rs] : make_float2(0.f, 0.f);
        Dft<R1, -1>::run(v);
        twiddle_a<R1, TP, -1>(v, n2, tA);
        __syncthreads();  // earlier reads of xb done
        t1_s<R1, TP, P>(v, xb, n2, p);
        pass_b<R1, TP, -1>(v);
    };
    auto inverse_store = [&](float2 (&v)[R1], float2* out) {
        pass_b<R1, TP, 1>(v);
        twiddle_b<R1, TP, 1>(v, n2, tB);
        __syncthreads();
        t2_s<R1, TP, P>(v, xb, n2, p);
        Dft<R1, 1>::run(v);
        if (valid)
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) out[base + (long long)(n2 + TP * n1) * a.rs] = v[n1];
    };
    float2 lam[R1], v[R1];
    forward(a.Lam, lam);
    float acck = 0.f, accm = 0.f;
    forward(a.Sn1, v);
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) {
            const float k2 = a.k2x[n2 * NB + i + R1 * c] + k2yz, k4 = k2 * k2;
            const float Dinv = rcp_approx(fmaf(a.dtMk, k4, 1.f));
            const float2 l = lam[i * TP + c], ch = v[i * TP + c];
            const float re = valid ? w * fmaf(l.x, ch.x, l.y * ch.y) : 0.f;
            acck = fmaf(re, -a.dtM * k4 * Dinv, acck);
            accm = fmaf(re, -a.dtk * k4 * Dinv, accm);
        }
    forward(a.Gn, v);
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) {
            const float k2 = a.k2x[n2 * NB + i + R1 * c] + k2yz;
            const float Dinv = rcp_approx(fmaf(a.dtMk, k2 * k2, 1.f));
            const float2 l = lam[i * TP + c], gh = v[i * TP + c];
            const float re = valid ? w * fmaf(l.x, gh.x, l.y * gh.y) : 0.f;
            accm = fmaf(re, -a.dt * k2 * Dinv, accm);
        }
    // P = F_x^-1 (a lambda_hat) / nx
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) {
            const float k2 = a.k2x[n2 * NB + i + R1 * c] + k2yz;
            v[i * TP + c] = cscale(lam[i * TP + c], a.invL * rcp_approx(fmaf(a.dtMk, k2 * k2, 1.f)));
        }
    inverse_store(v, a.P);
    // T = F_x^-1 (b lambda_hat) / nx
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) {
            const float k2 = a.k2x[n2 * NB + i + R1 * c] + k2yz;
            v[i * TP + c] = cscale(lam[i * TP + c], -a.dtM * k2 * a.invL * rcp_approx(fmaf(a.dtMk, k2 * k2, 1.f)));
        }
    inverse_store(v, a.T);
    // per-CTA FP64 partials, fixed order
    double dk = acck, dm = accm;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dk += __shfl_down_sync(0xffffffffu, dk, o);
        dm += __shfl_down_sync(0xffffffffu, dm, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = dk;
        red[1][threadIdx.x >> 5] = dm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sk = 0.0, sm = 0.0;
        for (int q = 0; q < (NT + 31) / 32; ++q) {
            sk += red[0][q];
            sm += red[1][q];
        }
        const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
        const long long nblk = (long long)gridDim.x * gridDim.y;
        a.partials[blk] = sk;
        a.partials[nblk + blk] = sm;
    }
}

}  // namespace fast

// --------------------------------------------------------------- dispatch
static int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// set the kernel's shared-memory limit and return its resident CTAs per SM
// (cached per kernel and smem size; kernels of one signature share a type, so
// the cache is keyed by the function address)
struct PrepEntry {
    const void* fn;
    int dev;
    size_t smem;
    int nb;
};
template <typename K>
static cudaError_t prep(K kernel, size_t smem, int threads, int* grid_per_sm) {
    static PrepEntry cache[64];
    static int ncache = 0;
    static std::mutex mu;  // grids may be driven from several host threads
    std::lock_guard<std::mutex> lock(mu);
    const void* key = (const void*)kernel;
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < ncache; ++i)
        if (cache[i].fn == key && cache[i].dev == dev && cache[i].smem == smem) {
            *grid_per_sm = cache[i].nb;
            return cudaSuccess;
        }
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    nb = nb > 0 ? nb : 1;
    if (ncache < 64) cache[ncache++] = PrepEntry{key, dev, smem, nb};
    *grid_per_sm = nb;
    return cudaSuccess;
}

// ------------------------------------------------------- tensor maps (host)
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
        else
            cudaGetLastError();
    }
    return fn;
}

// 4D map of a y-blocked half-spectrum buffer: dims {ncols, YB, nx, ny / YB}
// (complex64 as 8-byte elements), box {b0, b1, b2, b3} (b0 columns: 4 or 8, 32 or 64 bytes)
static bool make_map(CUtensorMap* m, const void* base, int ncols, int YB, int nx, int ny, long long Zp, int b0,
                     int b1, int b2, int b3) {
    auto fn = encode_fn();
    if (!fn || ((uintptr_t)base & 15) || (ny % YB)) return false;
    cuuint64_t dims[4] = {(cuuint64_t)ncols, (cuuint64_t)YB, (cuuint64_t)nx, (cuuint64_t)(ny / YB)};
    cuuint64_t strides[3] = {(cuuint64_t)(Zp * 8), (cuuint64_t)(YB * Zp * 8), (cuuint64_t)((long long)nx * YB * Zp * 8)};
    cuuint32_t box[4] = {(cuuint32_t)b0, (cuuint32_t)b1, (cuuint32_t)b2, (cuuint32_t)b3};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_INT64, 4, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool fast_timeout_flag(int* flag, bool clear) {
    int h = 0;
    if (cudaMemcpyFromSymbol(&h, fast::g_timeout, sizeof(int)) != cudaSuccess) return false;
    if (clear && h) {
        int z = 0;
        cudaMemcpyToSymbol(fast::g_timeout, &z, sizeof(int));
    }
    *flag = h;
    return true;
}

template <int R1, int TP, int DIR>
static bool run_fspass_tma(const SPassArgs& a, cudaStream_t st, cudaError_t* err) {
    constexpr int L = R1 * TP, BOX = fast::ybox(R1, L);
    // y pass geometry: rows y split in blocks of YB (rs = Zp), lines x (os = YB Zp);
    // a box covers YB rows of BOX / YB consecutive blocks
    if (a.rs * a.YB != a.os || a.YB > 256 || BOX % a.YB || BOX / a.YB > 256) return false;
    const long long Zp = a.rs;
    CUtensorMap mi, mo;
    if (!make_map(&mi, a.in, a.ncols, a.YB, a.nouter, a.L, Zp, 8, a.YB, 1, BOX / a.YB) ||
        !make_map(&mo, a.out, a.ncols, a.YB, a.nouter, a.L, Zp, 8, a.YB, 1, BOX / a.YB))
        return false;
    constexpr int NBUF = L == 1024 ? 2 : 1;  // one CTA per SM at 1024 either way
    const size_t smem = sizeof(float2) * (NBUF * L * 8 + (L + TP) * 8 + 2 * L) + 8 * NBUF;
    int per = 0;
    cudaError_t e = prep(fast::fspass_tma_kernel<R1, TP, DIR, NBUF>, smem, 8 * TP, &per);
    if (e != cudaSuccess) {
        *err = e;
        return true;
    }
    const int ntiles = a.nchunks * a.nouter;
    const int grid = std::min(ntiles, per * num_sms());
    fast::fspass_tma_kernel<R1, TP, DIR, NBUF><<<grid, 8 * TP, smem, st>>>(a, ntiles, mi, mo);
    *err = cudaGetLastError();
    return true;
}

template <int R1, int TP>
static bool run_fxupd_tma(const XUpdArgs& a, cudaStream_t st, cudaError_t* err) {
    constexpr int L = R1 * TP, BOX = fast::xbox(L);
    constexpr bool SEP = L == 1024;  // separate transpose/staging buffer (see fxupd_tma_kernel)
    // x pass geometry: rows x (rs = YB Zp), lines y split in blocks of YB (os = Zp)
    if (a.os * a.YB != a.rs) return false;
    const long long Zp = a.os;
    CUtensorMap mw, ms, mo;
    if (!make_map(&mw, a.W, a.ncols, a.YB, a.L, a.ny, Zp, 8, 1, BOX, 1) ||
        !make_map(&ms, a.S, a.ncols, a.YB, a.L, a.ny, Zp, 8, 1, BOX, 1) ||
        !make_map(&mo, a.S_out, a.ncols, a.YB, a.L, a.ny, Zp, 8, 1, BOX, 1))
        return false;
    const size_t smem =
        sizeof(float2) * ((SEP ? 3 : 2) * (size_t)(L + TP) * 8 + (R1 == TP ? 1 : 2) * (size_t)L) +
        (SEP ? sizeof(float) * L : 0) + 16;
    int per = 0;
    auto kern = a.model == 3   ? fast::fxupd_tma_kernel<R1, TP, 3, SEP>
                : a.model == 2 ? fast::fxupd_tma_kernel<R1, TP, 2, SEP>
                : a.model == 1 ? fast::fxupd_tma_kernel<R1, TP, 1, SEP>
                               : fast::fxupd_tma_kernel<R1, TP, 0, SEP>;
    cudaError_t e = prep(kern, smem, 8 * TP, &per);
    if (e != cudaSuccess) {
        *err = e;
        return true;
    }
    const int ntiles = a.nchunks * a.ny;
    const int grid = std::min(ntiles, per * num_sms());
    kern<<<grid, 8 * TP, smem, st>>>(a, ntiles, mw, ms, mo);
    *err = cudaGetLastError();
    return true;
}

bool fast_spass(const SPassArgs& a, int dir, cudaStream_t st, cudaError_t* err) {
#define CASE(L, R, T)                                                                       \
    case L:                                                                                 \
        return dir < 0 ? run_fspass_tma<R, T, -1>(a, st, err) : run_fspass_tma<R, T, 1>(a, st, err);
    switch (a.L) {
        CASE(64, 32, 2) CASE(128, 32, 4) CASE(256, 32, 8) CASE(512, 32, 16) CASE(1024, 32, 32) CASE(400, 20, 20)
    }
#undef CASE
    return false;
}

bool fast_xupdate(const XUpdArgs& a, cudaStream_t st, cudaError_t* err) {
    if (a.W == nullptr) return false;
    switch (a.L) {
        case 64: return run_fxupd_tma<32, 2>(a, st, err);
        case 128: return run_fxupd_tma<32, 4>(a, st, err);
        case 256: return run_fxupd_tma<32, 8>(a, st, err);
        case 512: return run_fxupd_tma<32, 16>(a, st, err);
        case 1024: return run_fxupd_tma<32, 32>(a, st, err);
        case 400: return run_fxupd_tma<20, 20>(a, st, err);
    }
    return false;
}

// threads of a z-pass CTA: 128 for R1 = 32, 160 (16 rows of 10 threads) for R1 = 20
template <int R1, int TP>
constexpr int ntz_of() {
    return R1 == 32 ? 128 : 160;
}
// shared memory of a z-pass CTA: the row tile, three twiddle tables and, for
// R1 != 32, the R2C partner rows (as laid out in the kernels)
template <int R1, int TP>
static size_t zpass_smem(int Zp) {
    constexpr int NTZ = ntz_of<R1, TP>(), RPC = NTZ / TP, M = R1 * TP, RS = M + TP * fast::zpad(R1, TP);
    const int BS = TP + (((Zp > RS ? Zp : RS) - TP + 15) & ~15);
    return sizeof(float2) * ((size_t)RPC * BS + 3 * M + 1 + (R1 != 32 ? (size_t)RPC * fast::zxs(M, TP) : 0));
}

template <int R1, int TP>
static cudaError_t run_fzstep(const ZPassArgs& a, cudaStream_t st, int* grid_used, bool adj = false) {
    constexpr int NTZ = ntz_of<R1, TP>(), RPC = NTZ / TP;
    const size_t smem = zpass_smem<R1, TP>(a.Zp);
    int per = 0;
    auto kern = adj       ? fast::fzstep_kernel<R1, TP, NTZ, false, true>
                : a.gsum ? fast::fzstep_kernel<R1, TP, NTZ, true, false>
                         : fast::fzstep_kernel<R1, TP, NTZ, false, false>;
    cudaError_t e = prep(kern, smem, NTZ, &per);
    if (e != cudaSuccess) return e;
    const int ntiles = (int)((a.nrows + RPC - 1) / RPC);
    const int grid = std::min(ntiles, per * num_sms());
    if (grid_used) *grid_used = grid;
    kern<<<grid, NTZ, smem, st>>>(a, ntiles);
    return cudaGetLastError();
}

template <int R1, int TP>
static cudaError_t run_fzconv(const ZPassArgs& a, int dir, cudaStream_t st, int* grid_used) {
    constexpr int NTZ = ntz_of<R1, TP>(), RPC = NTZ / TP;
    const size_t smem = zpass_smem<R1, TP>(a.Zp);
    const int ntiles = (int)((a.nrows + RPC - 1) / RPC);
    void (*kern)(ZPassArgs, int);
    if (dir < 0)
        kern = fast::fr2c_kernel<R1, TP, NTZ>;
    else if (a.accumulate)
        kern = a.partials ? fast::fc2r_kernel<R1, TP, NTZ, true, true> : fast::fc2r_kernel<R1, TP, NTZ, true, false>;
    else
        kern = a.partials ? fast::fc2r_kernel<R1, TP, NTZ, false, true> : fast::fc2r_kernel<R1, TP, NTZ, false, false>;
    int per = 0;
    cudaError_t e = prep(kern, smem, NTZ, &per);
    if (e != cudaSuccess) return e;
    const int grid = std::min(ntiles, per * num_sms());
    if (grid_used) *grid_used = grid;
    kern<<<grid, NTZ, smem, st>>>(a, ntiles);
    return cudaGetLastError();
}

// z R2C (dir < 0) or C2R (dir > 0) alone; false when the fast kernels do not apply
bool fast_zconv(const ZPassArgs& a, int dir, cudaStream_t st, cudaError_t* err, int* grid_used) {
    const float* real = dir < 0 ? a.rin : a.rout;
    if (!real || ((uintptr_t)real & 15) || (a.rpitch & 3)) return false;
    switch (a.M) {
        case 64: *err = run_fzconv<32, 2>(a, dir, st, grid_used); return true;
        case 128: *err = run_fzconv<32, 4>(a, dir, st, grid_used); return true;
        case 256: *err = run_fzconv<32, 8>(a, dir, st, grid_used); return true;
        case 512: *err = run_fzconv<32, 16>(a, dir, st, grid_used); return true;
        case 200: *err = run_fzconv<20, 10>(a, dir, st, grid_used); return true;
    }
    return false;
}

template <int R1, int TP>
static cudaError_t run_fxadj(const XAdjArgs& a, cudaStream_t st) {
    constexpr int L = R1 * TP;
    const size_t smem = sizeof(float2) * ((size_t)(L + TP) * 8 + (R1 == TP ? 1 : 2) * (size_t)L);
    int per = 0;
    cudaError_t e = prep(fast::fxadj_kernel<R1, TP>, smem, 8 * TP, &per);
    if (e != cudaSuccess) return e;
    fast::fxadj_kernel<R1, TP><<<dim3(a.nchunks, a.ny), 8 * TP, smem, st>>>(a);
    return cudaGetLastError();
}

bool fast_xadj(const XAdjArgs& a, cudaStream_t st, cudaError_t* err) {
    if (!fast_paths_enabled() || a.os * a.YB != a.rs) return false;
    switch (a.L) {
        case 64: *err = run_fxadj<32, 2>(a, st); return true;
        case 128: *err = run_fxadj<32, 4>(a, st); return true;
        case 256: *err = run_fxadj<32, 8>(a, st); return true;
        case 512: *err = run_fxadj<32, 16>(a, st); return true;
        case 1024: *err = run_fxadj<32, 32>(a, st); return true;
        case 400: *err = run_fxadj<20, 20>(a, st); return true;
    }
    return false;
}

bool fast_zstep(const ZPassArgs& a, cudaStream_t st, cudaError_t* err, int* grid_used, bool adj) {
    if (adj && (!a.cn || (a.cnpitch & 1) || ((uintptr_t)a.cn & 7))) return false;
    switch (a.M) {
        case 64: *err = run_fzstep<32, 2>(a, st, grid_used, adj); return true;
        case 128: *err = run_fzstep<32, 4>(a, st, grid_used, adj); return true;
        case 256: *err = run_fzstep<32, 8>(a, st, grid_used, adj); return true;
        case 512: *err = run_fzstep<32, 16>(a, st, grid_used, adj); return true;
        case 200: *err = run_fzstep<20, 10>(a, st, grid_used, adj); return true;
    }
    return false;
}

}  // namespace evx
