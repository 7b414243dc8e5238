// Fast paths of the four step passes for power-of-two lengths L = 32 * TP
// (TP = 2 .. 32, i.e. L = 64 .. 1024; the z pass works on M = nz/2).
//
// Four-step FFT of a length-L pencil, n = n2 + TP n1 (n2 < TP, n1 < 32):
//   pass A:  Y[n2][k1] = sum_{n1} x[n2 + TP n1] w_32^{n1 k1}        (DFT-32 in registers)
//   twiddle: Y[n2][k1] *= w_L^{n2 k1}
//   pass B:  X[k1 + 32 k2] = sum_{n2} Y[n2][k1] w_TP^{n2 k2}         (32/TP DFT-TP per thread)
// Thread n2 of a pencil owns the 32 values x[n2 + TP n1] ("n2 ownership"); after
// the one shared-memory transpose thread j owns X[k1 + 32 k2] for
// k1 in [j 32/TP, (j+1) 32/TP), all k2 ("block ownership"). The inverse walks the
// same way back. Global loads and stores go straight from/to registers in
// both ownerships (each warp touches whole 64-byte row segments), the next
// tile is prefetched into shared memory with cp.async while the current one
// is computed, and the CTAs are persistent (one wave).
#include <algorithm>

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

// v[a] *= w_L^{+-n2 a}  (n2 ownership); tw is the shared-memory copy of the table
template <int DIR>
__device__ __forceinline__ void twiddle_a(float2 (&v)[32], int n2, const float2* tw) {
#pragma unroll
    for (int a = 1; a < 32; ++a) {
        float2 w = tw[n2 * a];
        if (DIR > 0) w.y = -w.y;
        v[a] = cmul(v[a], w);
    }
}

// v[i TP + c] *= w_L^{+-a c}, a = j NB + i  (block ownership)
template <int TP, int DIR>
__device__ __forceinline__ void twiddle_b(float2 (&v)[32], int j, const float2* tw) {
    constexpr int NB = 32 / TP;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int a = j * NB + i;
#pragma unroll
        for (int c = 1; c < TP; ++c) {
            float2 w = tw[a * c];
            if (DIR > 0) w.y = -w.y;
            v[i * TP + c] = cmul(v[i * TP + c], w);
        }
    }
}

template <int TP, int DIR>
__device__ __forceinline__ void pass_b(float2 (&v)[32]) {
#pragma unroll
    for (int i = 0; i < 32 / TP; ++i) Dft<TP, DIR>::run(v + i * TP);
}

// ---- shared-memory slots of the transposes
// Column tiles (P pencils adjacent, p fastest): group G = a TP + n2 of P
// complex, padded by one group per block a / (32/TP). Block-ownership
// accesses of one warp then fall 33 groups apart (bank offsets 8 or 16
// words) and n2-ownership accesses are contiguous: both conflict-free, and
// every address is a per-thread base plus a compile-time offset.
template <int TP, int P>
__device__ __forceinline__ int slot_s(int n2, int a, int p) {
    constexpr int NB = 32 / TP;
    return (a * TP + n2 + a / NB) * P + p;
}
// Row tiles (one pencil per row r, row stride RS = M + TP): the same one-slot
// padding per block of a staggers block-ownership accesses by 33 slots.
template <int TP>
__device__ __forceinline__ int slot_z(int r, int n2, int a) {
    constexpr int NB = 32 / TP, RS = 32 * TP + TP;
    return r * RS + a * TP + n2 + a / NB;
}

template <int TP, int P>
__device__ __forceinline__ void t1_s(float2 (&v)[32], float2* xb, int n2, int p) {
    constexpr int NB = 32 / TP;
#pragma unroll
    for (int a = 0; a < 32; ++a) xb[slot_s<TP, P>(n2, a, p)] = v[a];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) v[i * TP + c] = xb[slot_s<TP, P>(c, n2 * NB + i, p)];
}
template <int TP, int P>
__device__ __forceinline__ void t2_s(float2 (&v)[32], float2* xb, int n2, int p) {
    constexpr int NB = 32 / TP;
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) xb[slot_s<TP, P>(c, n2 * NB + i, p)] = v[i * TP + c];
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = xb[slot_s<TP, P>(n2, a, p)];
}
template <int TP>
__device__ __forceinline__ void t1_z(float2 (&v)[32], float2* xb, int n2, int r) {
    constexpr int NB = 32 / TP;
#pragma unroll
    for (int a = 0; a < 32; ++a) xb[slot_z<TP>(r, n2, a)] = v[a];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) v[i * TP + c] = xb[slot_z<TP>(r, c, n2 * NB + i)];
}
template <int TP>
__device__ __forceinline__ void t2_z(float2 (&v)[32], float2* xb, int n2, int r) {
    constexpr int NB = 32 / TP;
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) xb[slot_z<TP>(r, c, n2 * NB + i)] = v[i * TP + c];
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = xb[slot_z<TP>(r, n2, a)];
}

// prefetch one [L][P] column tile (rows rs apart) into buf as 16-byte
// pieces; invalid columns are zero-filled
template <int TP, int P>
__device__ __forceinline__ void issue_tile(float2* buf, const float2* g, long long base, long long rs,
                                           int col0, int ncols) {
    constexpr int NT_ = P * TP, PR = P / 2;  // threads, pieces per row
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int e = threadIdx.x + k * NT_;
        const int row = e / PR, q = e % PR;
        const int nv = min(max(ncols - (col0 + 2 * q), 0), 2);
        const float2* src = g + base + (long long)row * rs + 2 * q;
        cp_async16(buf + row * P + 2 * q, nv ? src : g, nv * 8);
    }
    cp_commit();
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------- y pass (strided)
template <int TP, int P, int DIR>
__global__ void __launch_bounds__(P * TP) fspass_kernel(SPassArgs a, int ntiles) {
    constexpr int L = 32 * TP, NB = 32 / TP, XB = (L + TP) * P;
    extern __shared__ float4 smem4[];
    float2* buf = reinterpret_cast<float2*>(smem4);  // [L][P]
    float2* xb = buf + L * P;                         // transpose
    float2* tws = xb + XB;                            // [L] twiddles
    const int p = threadIdx.x % P, n2 = threadIdx.x / P;
    const int nchunks = a.nchunks;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    for (int i = threadIdx.x; i < L; i += P * TP) tws[i] = a.tw[i];
    {
        const int outer = tile / nchunks, chunk = tile - outer * nchunks;
        issue_tile<TP, P>(buf, a.in, (long long)outer * a.os + chunk * P, a.rs, chunk * P, a.ncols);
    }
    for (; tile < ntiles; tile += gridDim.x) {
        cp_wait<0>();
        __syncthreads();
        float2 v[32];
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) v[n1] = buf[(n2 + TP * n1) * P + p];
        __syncthreads();
        const int next = tile + gridDim.x;
        if (next < ntiles) {
            const int outer = next / nchunks, chunk = next - outer * nchunks;
            issue_tile<TP, P>(buf, a.in, (long long)outer * a.os + chunk * P, a.rs, chunk * P, a.ncols);
        }
        Dft<32, DIR>::run(v);
        twiddle_a<DIR>(v, n2, tws);
        t1_s<TP, P>(v, xb, n2, p);
        pass_b<TP, DIR>(v);
        const int outer = tile / nchunks, chunk = tile - outer * nchunks;
        if (chunk * P + p < a.ncols) {
            float2* out = a.out + (long long)outer * a.os + chunk * P + p;
#pragma unroll
            for (int i = 0; i < NB; ++i)
#pragma unroll
                for (int c = 0; c < TP; ++c) out[(long long)(n2 * NB + i + 32 * c) * a.rs] = v[i * TP + c];
        }
    }
}

// ------------------------------------------------- x pass + k-space update
template <int TP, int P>
__global__ void __launch_bounds__(P * TP, 8 / P) fxupd_kernel(XUpdArgs a, int ntiles) {
    constexpr int L = 32 * TP, NB = 32 / TP, XB = (L + TP) * P;
    extern __shared__ float4 smem4[];
    float2* bufW = reinterpret_cast<float2*>(smem4);
    float2* bufS = bufW + L * P;
    float2* xb = bufS + L * P;
    float2* tws = xb + XB;                               // [L] twiddles
    float* k2xs = reinterpret_cast<float*>(tws + L);     // [L] |k_x|^2
    const int p = threadIdx.x % P, n2 = threadIdx.x / P;
    const int nchunks = a.nchunks;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    for (int i = threadIdx.x; i < L; i += P * TP) {
        tws[i] = a.tw[i];
        k2xs[i] = a.k2x[i];
    }
    {
        const int ky = tile / nchunks, chunk = tile - ky * nchunks;
        const long long base = (long long)ky * a.os + chunk * P;
        issue_tile<TP, P>(bufW, a.W, base, a.rs, chunk * P, a.ncols);
        issue_tile<TP, P>(bufS, a.S, base, a.rs, chunk * P, a.ncols);
    }
    const float ndtM = -a.dtM;
    for (; tile < ntiles; tile += gridDim.x) {
        const int ky = tile / nchunks, chunk = tile - ky * nchunks;
        const int next = tile + gridDim.x;
        long long nbase = 0;
        int nchunk = 0;
        if (next < ntiles) {
            const int nky = next / nchunks;
            nchunk = next - nky * nchunks;
            nbase = (long long)nky * a.os + nchunk * P;
        }
        // ---- g_hat = F_x W, kept as G = -dt M |k|^2 g_hat
        cp_wait<1>();
        __syncthreads();
        float2 v[32];
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) v[n1] = bufW[(n2 + TP * n1) * P + p];
        __syncthreads();
        if (next < ntiles) issue_tile<TP, P>(bufW, a.W, nbase, a.rs, nchunk * P, a.ncols);
        Dft<32, -1>::run(v);
        twiddle_a<-1>(v, n2, tws);
        t1_s<TP, P>(v, xb, n2, p);
        pass_b<TP, -1>(v);
        const int kz = chunk * P + p;
        const bool valid = kz < a.ncols;
        const float k2yz = a.k2y[ky] + (valid ? a.k2z[kz] : 0.f);
        float2 G[32];
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) {
                const float f = ndtM * (k2xs[n2 * NB + i + 32 * c] + k2yz);
                G[i * TP + c] = cscale(v[i * TP + c], f);
            }
        // ---- c_hat = F_x S
        if (next < ntiles) cp_wait<1>(); else cp_wait<0>();
        __syncthreads();
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) v[n1] = bufS[(n2 + TP * n1) * P + p];
        __syncthreads();
        if (next < ntiles) issue_tile<TP, P>(bufS, a.S, nbase, a.rs, nchunk * P, a.ncols);
        Dft<32, -1>::run(v);
        twiddle_a<-1>(v, n2, tws);
        t1_s<TP, P>(v, xb, n2, p);
        pass_b<TP, -1>(v);
        // ---- c_hat' = (c_hat - dt M |k|^2 g_hat) / (1 + dt M kappa |k|^4) / L;
        //      the k = 0 mode stays out (the mean is carried in FP64)
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) {
                const float k2 = k2xs[n2 * NB + i + 32 * c] + k2yz;
                const float f = a.invL * rcp_approx(fmaf(a.dtMk, k2 * k2, 1.f));
                const float2 r = cadd(v[i * TP + c], G[i * TP + c]);
                v[i * TP + c] = cscale(r, f);
            }
        if (ky == 0 && kz == 0 && n2 == 0) v[0] = make_float2(0.f, 0.f);
        // ---- S' = F_x^-1 c_hat'
        pass_b<TP, 1>(v);
        twiddle_b<TP, 1>(v, n2, tws);
        __syncthreads();  // transpose buffer reads of the forward done
        t2_s<TP, P>(v, xb, n2, p);
        Dft<32, 1>::run(v);
        if (valid) {
            float2* out = a.S_out + (long long)ky * a.os + chunk * P + p;
#pragma unroll
            for (int n1 = 0; n1 < 32; ++n1) out[(long long)(n2 + TP * n1) * a.rs] = v[n1];
        }
    }
}

// ------------------------------------------------ z pass: C2R, c^3 - c, R2C
template <int TP, int NTZ>
__global__ void __launch_bounds__(NTZ, 256 / NTZ) fzstep_kernel(ZPassArgs a, int ntiles) {
    constexpr int M = 32 * TP, NB = 32 / TP, RPC = NTZ / TP, RS = M + TP, H = M / 2 + 1;
    extern __shared__ float4 smem4[];
    const int Zp = a.Zp, Zh = a.Zp / 2;
    float2* bin = reinterpret_cast<float2*>(smem4);  // [RPC][Zp]
    float2* xb = bin + RPC * Zp;                      // [RPC][RS]
    float2* tws = xb + RPC * RS;                      // [M] complex FFT twiddles
    float2* rtws = tws + M;                           // [M + 1] real-transform twiddles
    const int n2 = threadIdx.x % TP, r = threadIdx.x / TP;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    for (int i = threadIdx.x; i < M; i += NTZ) tws[i] = a.tw[i];
    for (int i = threadIdx.x; i <= M; i += NTZ) rtws[i] = a.rtw[i];
    auto issue = [&](int tl) {
        const long long row0 = (long long)tl * RPC;
        for (int e = threadIdx.x; e < RPC * Zh; e += NTZ) {
            const int rr = e / Zh, q = e - rr * Zh;
            const bool ok = row0 + rr < a.nrows;
            const float2* src = a.in + (row0 + rr) * Zp + 2 * q;
            cp_async16(bin + rr * Zp + 2 * q, ok ? src : a.in, ok ? 16 : 0);
        }
        cp_commit();
    };
    issue(tile);
    const double cbd = a.cbar ? *a.cbar : 0.0;
    const float cb = (float)cbd;
    const float cbl = (float)(cbd - (double)cb);
    const float gp = (float)(3.0 * cbd * cbd - 1.0);  // g'(cbar)
    const float c3 = (float)(3.0 * cbd);
    const float s = a.scale;
    for (; tile < ntiles; tile += gridDim.x) {
        const long long row0 = (long long)tile * RPC;
        cp_wait<0>();
        __syncthreads();
        // C2R pre-processing: Z[k] = (X_k + conj X_{M-k}) + i e^{+2 pi i k/nz} (X_k - conj X_{M-k})
        float2 v[32];
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) {
            const int k = n2 + TP * n1;
            float2 xk = bin[r * Zp + k], xm = bin[r * Zp + (M - k)];
            if (k == 0) {
                xk.y = 0.f;
                xm.y = 0.f;
            }
            const float2 A = make_float2(xk.x + xm.x, xk.y - xm.y);
            const float2 B = make_float2(xk.x - xm.x, xk.y + xm.y);
            v[n1] = cadd(A, mul_i<1>(cmul(cconj(rtws[k]), B)));
        }
        __syncthreads();
        if (tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x);
        // inverse complex FFT of length M
        Dft<32, 1>::run(v);
        twiddle_a<1>(v, n2, tws);
        t1_z<TP>(v, xb, n2, r);
        pass_b<TP, 1>(v);
        // real-space samples z[m] = c[2m] + i c[2m+1], m = k1 + 32 k2
        const long long row = row0 + r;
        const bool rowok = row < a.nrows;
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) {
                const float2 z = v[i * TP + c];
                const float d0 = z.x * s, d1 = z.y * s;  // c - cbar (the state has no k = 0 mode)
                if (a.rout && rowok)
                    reinterpret_cast<float2*>(a.rout + row * a.rpitch)[n2 * NB + i + 32 * c] =
                        make_float2(fmaf(z.x, s, cbl) + cb, fmaf(z.y, s, cbl) + cb);
                // g(c) - g(cbar) = d (g'(cbar) + d (3 cbar + d)); the constant g(cbar) only
                // feeds the k = 0 mode, which the update multiplies by b(0) = 0
                v[i * TP + c] = make_float2(d0 * fmaf(d0, c3 + d0, gp), d1 * fmaf(d1, c3 + d1, gp));
            }
        // forward complex FFT of length M from block ownership (m = a + 32 b)
        pass_b<TP, -1>(v);
        twiddle_b<TP, -1>(v, n2, tws);
        __syncthreads();
        t2_z<TP>(v, xb, n2, r);
        Dft<32, -1>::run(v);
        // natural-order staging, then R2C post-processing in pairs (k, M - k)
        __syncthreads();
#pragma unroll
        for (int d = 0; d < 32; ++d) xb[r * RS + n2 + TP * d] = v[d];
        __syncthreads();
        for (int e = threadIdx.x; e < RPC * H; e += NTZ) {
            const int rr = e / H, k = e - rr * H;
            const long long orow = row0 + rr;
            if (orow >= a.nrows) continue;
            const int m = M - k;
            const float2 zk = xb[rr * RS + k], zm = xb[rr * RS + (m == M ? 0 : m)];
            const float2 A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            const float2 B = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y + zm.y));
            float2* out = a.out + orow * Zp;
            out[k] = cadd(A, mul_i<-1>(cmul(rtws[k], B)));
            if (m != k) {
                const float2 A2 = make_float2(A.x, -A.y);
                const float2 B2 = make_float2(-B.x, B.y);
                out[m] = cadd(A2, mul_i<-1>(cmul(rtws[m], B2)));
            }
        }
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

static int tp_of(int L) {
    switch (L) {
        case 64: return 2;
        case 128: return 4;
        case 256: return 8;
        case 512: return 16;
        case 1024: return 32;
        default: return 0;
    }
}

// pencils per column tile: 8, i.e. 64-byte row segments. (Four pencils, 32-byte
// halves taken by different tiles, measured about 30% DRAM over-fetch.)
template <int TP>
struct Cols {
    static constexpr int P = 8;
};

template <int TP, int DIR>
static cudaError_t run_fspass(const SPassArgs& a0, cudaStream_t st) {
    constexpr int P = Cols<TP>::P, L = 32 * TP;
    SPassArgs a = a0;
    a.nchunks = a0.nchunks * 8 / P;  // chunks of P columns
    const size_t smem = sizeof(float2) * (L * P + (L + TP) * P + L);
    int per = 0;
    cudaError_t e = prep(fast::fspass_kernel<TP, P, DIR>, smem, P * TP, &per);
    if (e != cudaSuccess) return e;
    const int ntiles = a.nchunks * a.nouter;
    const int grid = std::min(ntiles, per * num_sms());
    fast::fspass_kernel<TP, P, DIR><<<grid, P * TP, smem, st>>>(a, ntiles);
    return cudaGetLastError();
}

bool fast_spass(const SPassArgs& a, int dir, cudaStream_t st, cudaError_t* err) {
    const int TP = tp_of(a.L);
    if (!TP) return false;
#define CASE(T)                                                                       \
    case T:                                                                           \
        *err = dir < 0 ? run_fspass<T, -1>(a, st) : run_fspass<T, 1>(a, st);          \
        return true;
    switch (TP) {
        CASE(2) CASE(4) CASE(8) CASE(16) CASE(32)
    }
#undef CASE
    return false;
}

template <int TP>
static cudaError_t run_fxupd(const XUpdArgs& a0, cudaStream_t st) {
    constexpr int P = Cols<TP>::P, L = 32 * TP;
    XUpdArgs a = a0;
    a.nchunks = a0.nchunks * 8 / P;
    const size_t smem = sizeof(float2) * (2 * L * P + (L + TP) * P + L) + sizeof(float) * L;
    int per = 0;
    cudaError_t e = prep(fast::fxupd_kernel<TP, P>, smem, P * TP, &per);
    if (e != cudaSuccess) return e;
    const int ntiles = a.nchunks * a.ny;
    const int grid = std::min(ntiles, per * num_sms());
    fast::fxupd_kernel<TP, P><<<grid, P * TP, smem, st>>>(a, ntiles);
    return cudaGetLastError();
}

bool fast_xupdate(const XUpdArgs& a, cudaStream_t st, cudaError_t* err) {
    const int TP = tp_of(a.L);
    if (!TP || a.W == nullptr) return false;
    switch (TP) {
        case 2: *err = run_fxupd<2>(a, st); return true;
        case 4: *err = run_fxupd<4>(a, st); return true;
        case 8: *err = run_fxupd<8>(a, st); return true;
        case 16: *err = run_fxupd<16>(a, st); return true;
        case 32: *err = run_fxupd<32>(a, st); return true;
    }
    return false;
}

template <int TP>
static cudaError_t run_fzstep(const ZPassArgs& a, cudaStream_t st) {
    constexpr int NTZ = 128, RPC = NTZ / TP;
    const size_t smem =
        sizeof(float2) * ((size_t)RPC * a.Zp + (size_t)RPC * (32 * TP + TP) + 32 * TP + 32 * TP + 1);
    int per = 0;
    cudaError_t e = prep(fast::fzstep_kernel<TP, NTZ>, smem, NTZ, &per);
    if (e != cudaSuccess) return e;
    const int ntiles = (int)((a.nrows + RPC - 1) / RPC);
    const int grid = std::min(ntiles, per * num_sms());
    fast::fzstep_kernel<TP, NTZ><<<grid, NTZ, smem, st>>>(a, ntiles);
    return cudaGetLastError();
}

bool fast_zstep(const ZPassArgs& a, cudaStream_t st, cudaError_t* err) {
    const int TP = tp_of(a.M);
    if (TP < 2 || TP > 16) return false;
    switch (TP) {
        case 2: *err = run_fzstep<2>(a, st); return true;
        case 4: *err = run_fzstep<4>(a, st); return true;
        case 8: *err = run_fzstep<8>(a, st); return true;
        case 16: *err = run_fzstep<16>(a, st); return true;
    }
    return false;
}

}  // namespace evx
