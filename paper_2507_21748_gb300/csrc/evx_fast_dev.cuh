// Device building blocks of the four-step fast passes (shared by the
// per-axis kernels and the fused y-z-y pass): cp.async helpers, the
// re-indexed twiddle tables, the twiddle multiplies of both ownerships, the
// padded shared-memory transposes, the R2C post-processing of a row and the
// shared-memory padding rules. See evx_fast.cu for the transform they make up.
#pragma once
#include <cstdint>

#include "evx_internal.h"

namespace evx {
namespace fast {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Twiddles of the four-step transform, re-indexed in shared memory so that
// the threads of a warp read consecutive entries (no bank conflicts):
//   tA[a * TP + n2]           = w_L^{n2 a}     (n2 ownership, a < R1)
//   tB[(c * NB + i) * TP + j] = w_L^{a c}, a = j NB + i  (block ownership)
// both filled from the L-entry table tw[m] = w_L^m at kernel start.
template <int R1, int TP>
__device__ __forceinline__ void fill_twiddles(float2* tA, float2* tB, const float2* __restrict__ tw, int nthreads) {
    constexpr int NB = R1 / TP, L = R1 * TP;
    for (int idx = threadIdx.x; idx < L; idx += nthreads) {
        const int a = idx / TP, n2 = idx % TP;
        tA[idx] = tw[n2 * a];
        const int c = idx / R1, rem = idx % R1, i = rem / TP, j = rem % TP;
        tB[idx] = tw[(j * NB + i) * c];
    }
}

// v[a] *= w_L^{+-n2 a}  (n2 ownership)
template <int R1, int TP, int DIR>
__device__ __forceinline__ void twiddle_a(float2 (&v)[R1], int n2, const float2* tA) {
#pragma unroll
    for (int a = 1; a < R1; ++a) {
        float2 w = tA[a * TP + n2];
        if (DIR > 0) w.y = -w.y;
        v[a] = cmul(v[a], w);
    }
}

// v[i TP + c] *= w_L^{+-a c}, a = j NB + i  (block ownership)
template <int R1, int TP, int DIR>
__device__ __forceinline__ void twiddle_b(float2 (&v)[R1], int j, const float2* tB) {
    constexpr int NB = R1 / TP;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
#pragma unroll
        for (int c = 1; c < TP; ++c) {
            float2 w = tB[(c * NB + i) * TP + j];
            if (DIR > 0) w.y = -w.y;
            v[i * TP + c] = cmul(v[i * TP + c], w);
        }
    }
}

template <int R1, int TP, int DIR>
__device__ __forceinline__ void pass_b(float2 (&v)[R1]) {
#pragma unroll
    for (int i = 0; i < R1 / TP; ++i) Dft<TP, DIR>::run(v + i * TP);
}

// ---- shared-memory slots of the transposes
// Column tiles (P pencils adjacent, p fastest): group G = a TP + n2 of P
// complex, padded by one group per block a / (R1/TP). For R1 = 32,
// block-ownership accesses of one warp then fall 33 groups apart (bank
// offsets 8 or 16 words) and n2-ownership accesses are contiguous: both
// conflict-free, and every address is a per-thread base plus a compile-time
// offset.
template <int R1, int TP, int P>
__device__ __forceinline__ int slot_s(int n2, int a, int p) {
    constexpr int NB = R1 / TP;
    return (a * TP + n2 + a / NB) * P + p;
}
template <int R1, int TP, int P>
__device__ __forceinline__ void t1_s(float2 (&v)[R1], float2* xb, int n2, int p) {
    constexpr int NB = R1 / TP;
#pragma unroll
    for (int a = 0; a < R1; ++a) xb[slot_s<R1, TP, P>(n2, a, p)] = v[a];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) v[i * TP + c] = xb[slot_s<R1, TP, P>(c, n2 * NB + i, p)];
}
template <int R1, int TP, int P>
__device__ __forceinline__ void t2_s(float2 (&v)[R1], float2* xb, int n2, int p) {
    constexpr int NB = R1 / TP;
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) xb[slot_s<R1, TP, P>(c, n2 * NB + i, p)] = v[i * TP + c];
    __syncthreads();
#pragma unroll
    for (int a = 0; a < R1; ++a) v[a] = xb[slot_s<R1, TP, P>(n2, a, p)];
}

// R2C post-processing of one row: thread n2 holds Z[n2 + TP d] (d < R1) of the
// length-M complex transform Z of the packed real row; it writes, for its k,
//   X_k = (Z_k + conj Z_{M-k})/2 - i e^{-2 pi i k/nz} (Z_k - conj Z_{M-k})/2
// and thread 0 also X_M = Re Z_0 - Im Z_0. With R1 = 32 (TP a power of two
// dividing 32) the partner Z[M - k] of k = n2 + TP d sits in thread TP - n2 of
// the same warp at index 31 - d (thread 0: its own index 32 - d) and is
// fetched by warp shuffle; otherwise the row passes through the M-entry shared
// row xz. Every thread of the CTA calls this (it may synchronise the CTA).
// Real-transform pre- and post-processing of one pair (k, M - k) of a length-2M
// real row held as M complex values, w = exp(-2 pi i k / 2M); P and Q are the
// pair's sum and difference, the twiddle product is taken into FMAs.
// C2R: Z_k = P + i conj(w) Q with P = X_k + conj X_{M-k}, Q = X_k - conj X_{M-k}
__device__ __forceinline__ float2 c2r_pre(float2 xk, float2 xm, float2 w) {
    const float px = xk.x + xm.x, py = xk.y - xm.y, qx = xk.x - xm.x, qy = xk.y + xm.y;
    return make_float2(fmaf(-w.x, qy, fmaf(w.y, qx, px)), fmaf(w.x, qx, fmaf(w.y, qy, py)));
}
// R2C: X_k = (P - i w Q) / 2 with P = Z_k + conj Z_{M-k}, Q = Z_k - conj Z_{M-k}
__device__ __forceinline__ float2 r2c_post(float2 zk, float2 zm, float2 w) {
    const float px = zk.x + zm.x, py = zk.y - zm.y, qx = zk.x - zm.x, qy = zk.y + zm.y;
    return make_float2(0.5f * fmaf(w.x, qy, fmaf(w.y, qx, px)), 0.5f * fmaf(-w.x, qx, fmaf(w.y, qy, py)));
}

template <int R1, int TP>
__device__ __forceinline__ void r2c_store(const float2 (&v)[R1], int n2, float2* xz, float2* out, bool rowok,
                                          const float2* rtws) {
    constexpr int M = R1 * TP;
    if constexpr (R1 == 32) {
        const int lane = threadIdx.x & 31;
        const int src = (lane & ~(TP - 1)) | ((TP - n2) & (TP - 1));
#pragma unroll
        for (int d = 0; d < 32; ++d) {
            float2 zm;
            zm.x = __shfl_sync(0xffffffffu, v[31 - d].x, src);
            zm.y = __shfl_sync(0xffffffffu, v[31 - d].y, src);
            if (n2 == 0) zm = v[(32 - d) & 31];
            const int k = n2 + TP * d;
            if (rowok) out[k] = r2c_post(v[d], zm, rtws[k]);
        }
    } else {
#pragma unroll
        for (int d = 0; d < R1; ++d) xz[n2 + TP * d] = v[d];
        __syncthreads();
#pragma unroll
        for (int d = 0; d < R1; ++d) {
            const int k = n2 + TP * d;
            const float2 zm = xz[k == 0 ? 0 : M - k];
            if (rowok) out[k] = r2c_post(v[d], zm, rtws[k]);
        }
    }
    if (rowok && n2 == 0) out[M] = make_float2(v[0].x - v[0].y, 0.f);  // X_M = Re Z_0 - Im Z_0
}

// rows of the y-pass TMA box: up to 256 for R1 = 32 (y blocks of 32 rows), the
// whole line otherwise (y blocks of 16, at most 256 of them); x-pass box: the
// largest of L, 256 or L / 2 that divides L and is at most 256
__host__ __device__ constexpr int ybox(int R1, int L) { return R1 == 32 ? (L < 256 ? L : 256) : L; }
__host__ __device__ constexpr int xbox(int L) { return L <= 256 ? L : (L % 256 == 0 ? 256 : L / 2); }

// z-pass transposes: a tile row (one pencil, r = thread / TP) holds slot
// aa TP + n2 + (aa / NB) ZPAD, the rows BS = TP (mod 16) apart. With the group
// stride s = R1 + ZPAD odd and (s - 1) TP = 0 (mod 16), thread t = TP r + n2
// addresses bank pair t (n2 ownership) or s t (block ownership) mod 16: no two
// threads of a half-warp share a bank. ZPAD = 1 for R1 = 32 (s = 33), 5 for
// R1 = 20, TP = 10 (s = 25).
__host__ __device__ constexpr int zpad(int R1, int TP) {
    for (int d = 1; d < 16; ++d)
        if (((R1 + d) & 1) && ((R1 + d - 1) * TP) % 16 == 0) return d;
    return 1;
}
// stride of the R2C partner rows xz: M rounded up to = TP (mod 16), so the row
// writes are conflict-free like the n2-ownership slots
__host__ __device__ constexpr int zxs(int M, int TP) { return M + (((TP - M) % 16) + 16) % 16; }

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}


}  // namespace fast
}  // namespace evx
