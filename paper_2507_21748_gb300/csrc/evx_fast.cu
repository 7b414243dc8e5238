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

// v[a] *= w_L^{+-n2 a}  (n2 ownership)
template <int DIR>
__device__ __forceinline__ void twiddle_a(float2 (&v)[32], int n2, const float2* __restrict__ tw) {
#pragma unroll
    for (int a = 1; a < 32; ++a) {
        float2 w = __ldg(tw + n2 * a);
        if (DIR > 0) w.y = -w.y;
        v[a] = cmul(v[a], w);
    }
}

// v[i TP + c] *= w_L^{+-a c}, a = j NB + i  (block ownership)
template <int TP, int DIR>
__device__ __forceinline__ void twiddle_b(float2 (&v)[32], int j, const float2* __restrict__ tw) {
    constexpr int NB = 32 / TP;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int a = j * NB + i;
#pragma unroll
        for (int c = 1; c < TP; ++c) {
            float2 w = __ldg(tw + a * c);
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
// strided tiles: 8 pencils p fastest; 64-byte group G = a TP + n2, bank half
// flipped by bit 5 of G so that both ownerships access it conflict-free
template <int TP>
__device__ __forceinline__ int slot_s(int n2, int a, int p) {
    const int G = a * TP + n2;
    return ((G ^ ((G >> 5) & 1)) << 3) + p;
}
// row tiles: row r, row stride RS = M + TP; n2 xor-swizzled by the block of a
template <int TP>
__device__ __forceinline__ int slot_z(int r, int n2, int a) {
    constexpr int NB = 32 / TP, RS = 32 * TP + TP;
    return r * RS + a * TP + (n2 ^ (a / NB));
}

template <int TP>
__device__ __forceinline__ void t1_s(float2 (&v)[32], float2* xb, int n2, int p) {
    constexpr int NB = 32 / TP;
#pragma unroll
    for (int a = 0; a < 32; ++a) xb[slot_s<TP>(n2, a, p)] = v[a];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) v[i * TP + c] = xb[slot_s<TP>(c, n2 * NB + i, p)];
}
template <int TP>
__device__ __forceinline__ void t2_s(float2 (&v)[32], float2* xb, int n2, int p) {
    constexpr int NB = 32 / TP;
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) xb[slot_s<TP>(c, n2 * NB + i, p)] = v[i * TP + c];
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = xb[slot_s<TP>(n2, a, p)];
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

// prefetch one [L][8] column tile (rows rs apart) into buf; invalid columns zero-filled
template <int TP>
__device__ __forceinline__ void issue_tile(float2* buf, const float2* g, long long base, long long rs,
                                           int col0, int ncols) {
    constexpr int NT_ = 8 * TP;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int e = threadIdx.x + k * NT_;
        const int row = e >> 2, q = e & 3;
        const int nv = min(max(ncols - (col0 + 2 * q), 0), 2);
        const float2* src = g + base + (long long)row * rs + 2 * q;
        cp_async16(buf + row * 8 + 2 * q, nv ? src : g, nv * 8);
    }
    cp_commit();
}

// ---------------------------------------------------------- y pass (strided)
template <int TP, int DIR>
__global__ void __launch_bounds__(8 * TP) fspass_kernel(SPassArgs a, int ntiles) {
    constexpr int L = 32 * TP, NB = 32 / TP;
    extern __shared__ float4 smem4[];
    float2* buf = reinterpret_cast<float2*>(smem4);  // [L][8]
    float2* xb = buf + L * 8;                         // [L * 8] transpose
    const int p = threadIdx.x & 7, n2 = threadIdx.x >> 3;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    {
        const int outer = tile / a.nchunks, chunk = tile - outer * a.nchunks;
        issue_tile<TP>(buf, a.in, (long long)outer * a.os + chunk * 8, a.rs, chunk * 8, a.ncols);
    }
    for (; tile < ntiles; tile += gridDim.x) {
        cp_wait<0>();
        __syncthreads();
        float2 v[32];
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) v[n1] = buf[(n2 + TP * n1) * 8 + p];
        __syncthreads();
        const int next = tile + gridDim.x;
        if (next < ntiles) {
            const int outer = next / a.nchunks, chunk = next - outer * a.nchunks;
            issue_tile<TP>(buf, a.in, (long long)outer * a.os + chunk * 8, a.rs, chunk * 8, a.ncols);
        }
        Dft<32, DIR>::run(v);
        twiddle_a<DIR>(v, n2, a.tw);
        t1_s<TP>(v, xb, n2, p);
        pass_b<TP, DIR>(v);
        const int outer = tile / a.nchunks, chunk = tile - outer * a.nchunks;
        if (chunk * 8 + p < a.ncols) {
            float2* out = a.out + (long long)outer * a.os + chunk * 8 + p;
#pragma unroll
            for (int i = 0; i < NB; ++i)
#pragma unroll
                for (int c = 0; c < TP; ++c) out[(long long)(n2 * NB + i + 32 * c) * a.rs] = v[i * TP + c];
        }
    }
}

// ------------------------------------------------- x pass + k-space update
template <int TP>
__global__ void __launch_bounds__(8 * TP, 1) fxupd_kernel(XUpdArgs a, int ntiles) {
    constexpr int L = 32 * TP, NB = 32 / TP;
    extern __shared__ float4 smem4[];
    float2* bufW = reinterpret_cast<float2*>(smem4);
    float2* bufS = bufW + L * 8;
    float2* xb = bufS + L * 8;
    const int p = threadIdx.x & 7, n2 = threadIdx.x >> 3;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    {
        const int ky = tile / a.nchunks, chunk = tile - ky * a.nchunks;
        const long long base = (long long)ky * a.os + chunk * 8;
        issue_tile<TP>(bufW, a.W, base, a.rs, chunk * 8, a.ncols);
        issue_tile<TP>(bufS, a.S, base, a.rs, chunk * 8, a.ncols);
    }
    for (; tile < ntiles; tile += gridDim.x) {
        const int ky = tile / a.nchunks, chunk = tile - ky * a.nchunks;
        const int next = tile + gridDim.x;
        long long nbase = 0;
        int nchunk = 0;
        if (next < ntiles) {
            const int nky = next / a.nchunks;
            nchunk = next - nky * a.nchunks;
            nbase = (long long)nky * a.os + nchunk * 8;
        }
        // ---- g_hat = F_x W
        cp_wait<1>();
        __syncthreads();
        float2 v[32];
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) v[n1] = bufW[(n2 + TP * n1) * 8 + p];
        __syncthreads();
        if (next < ntiles) issue_tile<TP>(bufW, a.W, nbase, a.rs, nchunk * 8, a.ncols);
        Dft<32, -1>::run(v);
        twiddle_a<-1>(v, n2, a.tw);
        t1_s<TP>(v, xb, n2, p);
        pass_b<TP, -1>(v);
        const int kz = chunk * 8 + p;
        const bool valid = kz < a.ncols;
        const float k2yz = a.k2y[ky] + (valid ? a.k2z[kz] : 0.f);
        float2 G[32];
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) {
                const float k2 = __ldg(a.k2x + n2 * NB + i + 32 * c) + k2yz;
                const float ainv = a.invL / fmaf(a.dtMk, k2 * k2, 1.f);
                const float b = -a.dtM * k2 * ainv;
                G[i * TP + c] = cscale(v[i * TP + c], b);
            }
        // ---- c_hat = F_x S
        if (next < ntiles) cp_wait<1>(); else cp_wait<0>();
        __syncthreads();
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) v[n1] = bufS[(n2 + TP * n1) * 8 + p];
        __syncthreads();
        if (next < ntiles) issue_tile<TP>(bufS, a.S, nbase, a.rs, nchunk * 8, a.ncols);
        Dft<32, -1>::run(v);
        twiddle_a<-1>(v, n2, a.tw);
        t1_s<TP>(v, xb, n2, p);
        pass_b<TP, -1>(v);
        // ---- c_hat' = a c_hat + b g_hat  (1/L folded in); k = 0 kept out (FP64 mean)
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int c = 0; c < TP; ++c) {
                const float k2 = __ldg(a.k2x + n2 * NB + i + 32 * c) + k2yz;
                const float ainv = a.invL / fmaf(a.dtMk, k2 * k2, 1.f);
                float2 r = v[i * TP + c];
                r.x = fmaf(ainv, r.x, G[i * TP + c].x);
                r.y = fmaf(ainv, r.y, G[i * TP + c].y);
                v[i * TP + c] = r;
            }
        if (ky == 0 && kz == 0 && n2 == 0) v[0] = make_float2(0.f, 0.f);
        // ---- S' = F_x^-1 c_hat'
        pass_b<TP, 1>(v);
        twiddle_b<TP, 1>(v, n2, a.tw);
        __syncthreads();  // transpose buffer reads of the forward done
        t2_s<TP>(v, xb, n2, p);
        Dft<32, 1>::run(v);
        if (valid) {
            float2* out = a.S_out + (long long)ky * a.os + chunk * 8 + p;
#pragma unroll
            for (int n1 = 0; n1 < 32; ++n1) out[(long long)(n2 + TP * n1) * a.rs] = v[n1];
        }
    }
}

// ------------------------------------------------ z pass: C2R, c^3 - c, R2C
template <int TP>
__global__ void __launch_bounds__(256, 1) fzstep_kernel(ZPassArgs a, int ntiles) {
    constexpr int M = 32 * TP, NB = 32 / TP, RPC = 256 / TP, RS = M + TP, H = M / 2 + 1;
    extern __shared__ float4 smem4[];
    const int Zp = a.Zp, Zh = a.Zp / 2;
    float2* bin = reinterpret_cast<float2*>(smem4);  // [RPC][Zp]
    float2* xb = bin + RPC * Zp;                      // [RPC][RS]
    const int n2 = threadIdx.x % TP, r = threadIdx.x / TP;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    auto issue = [&](int tl) {
        const long long row0 = (long long)tl * RPC;
        for (int e = threadIdx.x; e < RPC * Zh; e += 256) {
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
            v[n1] = cadd(A, mul_i<1>(cmul(cconj(__ldg(a.rtw + k)), B)));
        }
        __syncthreads();
        if (tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x);
        // inverse complex FFT of length M
        Dft<32, 1>::run(v);
        twiddle_a<1>(v, n2, a.tw);
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
                const float c0 = fmaf(z.x, s, cbl) + cb, c1 = fmaf(z.y, s, cbl) + cb;
                if (a.rout && rowok)
                    reinterpret_cast<float2*>(a.rout + row * a.rpitch)[n2 * NB + i + 32 * c] =
                        make_float2(c0, c1);
                v[i * TP + c] = make_float2(c0 * fmaf(c0, c0, -1.f), c1 * fmaf(c1, c1, -1.f));
            }
        // forward complex FFT of length M from block ownership (m = a + 32 b)
        pass_b<TP, -1>(v);
        twiddle_b<TP, -1>(v, n2, a.tw);
        __syncthreads();
        t2_z<TP>(v, xb, n2, r);
        Dft<32, -1>::run(v);
        // natural-order staging, then R2C post-processing in pairs (k, M - k)
        __syncthreads();
#pragma unroll
        for (int d = 0; d < 32; ++d) xb[r * RS + n2 + TP * d] = v[d];
        __syncthreads();
        for (int e = threadIdx.x; e < RPC * H; e += 256) {
            const int rr = e / H, k = e - rr * H;
            const long long orow = row0 + rr;
            if (orow >= a.nrows) continue;
            const int m = M - k;
            const float2 zk = xb[rr * RS + k], zm = xb[rr * RS + (m == M ? 0 : m)];
            const float2 A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            const float2 B = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y + zm.y));
            float2* out = a.out + orow * Zp;
            out[k] = cadd(A, mul_i<-1>(cmul(__ldg(a.rtw + k), B)));
            if (m != k) {
                const float2 A2 = make_float2(A.x, -A.y);
                const float2 B2 = make_float2(-B.x, B.y);
                out[m] = cadd(A2, mul_i<-1>(cmul(__ldg(a.rtw + m), B2)));
            }
        }
    }
}

}  // namespace fast

// --------------------------------------------------------------- dispatch
static int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// set the kernel's shared-memory limit and return its resident CTAs per SM
// (cached per kernel and smem size; kernels of one signature share a type, so
// the cache is keyed by the function address)
struct PrepEntry {
    const void* fn;
    size_t smem;
    int nb;
};
template <typename K>
static cudaError_t prep(K kernel, size_t smem, int threads, int* grid_per_sm) {
    static PrepEntry cache[64];
    static int ncache = 0;
    const void* key = (const void*)kernel;
    for (int i = 0; i < ncache; ++i)
        if (cache[i].fn == key && cache[i].smem == smem) {
            *grid_per_sm = cache[i].nb;
            return cudaSuccess;
        }
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    nb = nb > 0 ? nb : 1;
    if (ncache < 64) cache[ncache++] = PrepEntry{key, smem, nb};
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

template <int TP, int DIR>
static cudaError_t run_fspass(const SPassArgs& a, cudaStream_t st) {
    const size_t smem = sizeof(float2) * 2 * 32 * TP * 8;
    int per = 0;
    cudaError_t e = prep(fast::fspass_kernel<TP, DIR>, smem, 8 * TP, &per);
    if (e != cudaSuccess) return e;
    const int ntiles = a.nchunks * a.nouter;
    const int grid = std::min(ntiles, per * num_sms());
    fast::fspass_kernel<TP, DIR><<<grid, 8 * TP, smem, st>>>(a, ntiles);
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
static cudaError_t run_fxupd(const XUpdArgs& a, cudaStream_t st) {
    const size_t smem = sizeof(float2) * 3 * 32 * TP * 8;
    int per = 0;
    cudaError_t e = prep(fast::fxupd_kernel<TP>, smem, 8 * TP, &per);
    if (e != cudaSuccess) return e;
    const int ntiles = a.nchunks * a.ny;
    const int grid = std::min(ntiles, per * num_sms());
    fast::fxupd_kernel<TP><<<grid, 8 * TP, smem, st>>>(a, ntiles);
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
    constexpr int RPC = 256 / TP;
    const size_t smem = sizeof(float2) * ((size_t)RPC * a.Zp + (size_t)RPC * (32 * TP + TP));
    int per = 0;
    cudaError_t e = prep(fast::fzstep_kernel<TP>, smem, 256, &per);
    if (e != cudaSuccess) return e;
    const int ntiles = (int)((a.nrows + RPC - 1) / RPC);
    const int grid = std::min(ntiles, per * num_sms());
    fast::fzstep_kernel<TP><<<grid, 256, smem, st>>>(a, ntiles);
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
