// Fused y-z-y pass of the spectral step: the y inverse, the z C2R -> c^3 - c
// -> z R2C and the y forward transform in one persistent kernel, scheduled so
// that each x slab's work buffer stays in L2 between its three stages.
//
// The state between two steps is S = F_y F_z c (real in x). The pass turns it
// into W = F_y F_z (g(c) - g(cbar)) (the k = 0 constant g(cbar) is dropped: the
// update multiplies that mode by b(0) = 0), exactly what the three separate
// passes compute, with the same four-step transforms (evx_fast_dev.cuh). Per x
// slab (ny rows of Zp complex, 4.3 MB at 1024^3) there are three kinds of work
// item:
//   Yinv(x, chunk)  8 columns of all ny rows: S -> y inverse -> W
//   Z(x, q)         16 consecutive rows: W -> z C2R, g, z R2C -> W
//   Yfwd(x, chunk)  8 columns of all ny rows: W -> y forward -> W
// A Z item of slab x needs every Yinv item of x, a Yfwd item every Z item of x.
// Items are handed out in ticket order (one atomic counter): phase p issues
// the Yinv items of slab p, the Z items of slab p - lag and the Yfwd items of
// slab p - 2 lag. Every dependency therefore points to a lower ticket, so the
// lowest unfinished item never waits and the kernel always makes progress
// (whether or not all CTAs are resident). Between the Yinv and Yfwd items of a
// slab about 2 lag + 1 slabs of W are live, a few tens of MB, so the slab's
// intermediate reads and writes are served by L2: the pass moves about 2F of
// DRAM traffic (read S, write W) instead of the 6F of three separate passes.
//
// Synchronisation follows the grid-barrier pattern: a producer's threads store
// with plain global stores, the CTA synchronises, thread 0 fences at gpu scope
// and bumps the slab's counter; a consumer's thread 0 waits for the count with
// acquire loads, the CTA synchronises, then every thread loads with cp.async.cg
// (L2, not L1). Every wait is bounded (about 2 s of clock64); one that runs out
// sets the launch's abort word (every other wait then returns at once) and the
// device flag that the runtime checks at synchronisation points.
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "evx_fast_dev.cuh"

namespace evx {
namespace fused {

__device__ int g_fused_timeout;

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// thread 0: wait until *cnt >= target; false if the wait ran out or another CTA gave up
__device__ bool wait_count(const int* cnt, int target, int* abort_word) {
    const long long t0 = clock64();
    while (true) {
        if (ld_acquire(cnt) >= target) return true;
        if (ld_acquire(abort_word)) return false;
        if (clock64() - t0 > (1LL << 32)) {
            atomicExch(abort_word, 1);
            atomicExch(&g_fused_timeout, 1);
            return false;
        }
        __nanosleep(100);
    }
}

// shared memory of the fused kernel, in float2 units: one tile buffer that
// holds either a y tile ((L + TPy) x 8, transposes included) or a z tile
// (RPC rows of pitch BS, plus the R2C partner rows when R1z != 32), then the
// y twiddles (one table when R1y = TPy), the two z twiddle tables and the
// real-transform twiddles
template <int R1y, int TPy, int R1z, int TPz>
struct FusedGeom {
    static constexpr int L = R1y * TPy, NT = 8 * TPy, M = R1z * TPz, RPC = NT / TPz;
    static constexpr int RS = M + TPz * fast::zpad(R1z, TPz);
    static constexpr int YT = (L + TPy) * 8;
    static constexpr int YTW = R1y == TPy ? L : 2 * L;
    __host__ __device__ static int bs(int Zp) { return TPz + (((Zp > RS ? Zp : RS) - TPz + 15) & ~15); }
    __host__ __device__ static int zt(int Zp) { return RPC * bs(Zp) + (R1z != 32 ? RPC * fast::zxs(M, TPz) : 0); }
    __host__ __device__ static int tile(int Zp) { return YT > zt(Zp) ? YT : zt(Zp); }
    __host__ __device__ static int floats2(int Zp) { return tile(Zp) + YTW + 3 * M + 1; }
};

// One y item: 8 columns (chunk) of all L rows of slab x, in -> 1D DFT along y -> out.
// Element (x, y, kz) sits at base_x + (y / YB) os2 + (y % YB) Zp + kz (YB = a.YB,
// a compile-time constant here: 32 for power-of-two edges, 16 for 400).
template <int R1, int TP, int YB, int DIR>
__device__ __forceinline__ void y_item(const float2* in, float2* out, long long base_x,
                                       const YZYArgs& a, int chunk, float2* buf, const float2* tA, const float2* tB) {
    constexpr int L = R1 * TP, NB = R1 / TP, NT = 8 * TP;
    const int p = threadIdx.x & 7, n2 = threadIdx.x >> 3;
    const int kz0 = chunk * 8;
    // 16-byte pieces: 4 per row; thread t moves piece q = t % 4 (columns kz0 + 2q, +1;
    // columns past ncols are zero-filled) of rows t / 4, t / 4 + NT / 4, ...
    const int q = threadIdx.x & 3, kz = kz0 + 2 * q;
    const int nval = min(max(a.ncols - kz, 0), 2);
    for (int y = threadIdx.x >> 2; y < L; y += NT / 4) {
        const long long off = base_x + (long long)(y / YB) * a.os2 + (y % YB) * a.Zp + kz;
        fast::cp_async16(buf + y * 8 + 2 * q, nval ? in + off : in, nval * 8);
    }
    fast::cp_commit();
    fast::cp_wait<0>();
    __syncthreads();
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = buf[(n2 + TP * n1) * 8 + p];
    __syncthreads();  // tile read: buf becomes transpose space
    Dft<R1, DIR>::run(v);
    fast::twiddle_a<R1, TP, DIR>(v, n2, tA);
    fast::t1_s<R1, TP, 8>(v, buf, n2, p);
    fast::pass_b<R1, TP, DIR>(v);
    __syncthreads();  // transpose reads done: buf stages the result in row order
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) buf[(n2 * NB + i + R1 * c) * 8 + p] = v[i * TP + c];
    __syncthreads();
    for (int y = threadIdx.x >> 2; y < L; y += NT / 4) {
        const long long off = base_x + (long long)(y / YB) * a.os2 + (y % YB) * a.Zp + kz;
        const float2* src = buf + y * 8 + 2 * q;
        if (nval == 2)
            *reinterpret_cast<float4*>(out + off) = *reinterpret_cast<const float4*>(src);
        else if (nval == 1)
            out[off] = src[0];
    }
}

// One z item: RPC consecutive memory rows r0 .. r0 + RPC - 1 of W, in place:
// C2R (scale 1/(ny nz), about the FP64 mean), d (g'(cbar) + d (3 cbar + d)) with
// d = c - cbar, R2C. The same arithmetic as the separate z pass.
template <int R1, int TP, int NT, bool GS>
__device__ __forceinline__ void z_item(float2* W, long long r0, const YZYArgs& a, float2* buf, const float2* tA,
                                       const float2* tB, const float2* rtws, float gp, float c3, double& gacc) {
    constexpr int M = R1 * TP, NB = R1 / TP, RPC = NT / TP, ZPAD = fast::zpad(R1, TP), RS = M + TP * ZPAD;
    const int Zp = a.Zp, Zh = a.Zp / 2;
    const int BS = TP + (((Zp > RS ? Zp : RS) - TP + 15) & ~15);
    float2* xz = buf + RPC * BS;  // [RPC][zxs(M, TP)] R2C partner rows (R1 != 32)
    const int n2 = threadIdx.x % TP, r = threadIdx.x / TP;
    // rows to warps, 16-byte pieces of a row to lanes
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int rr = warp; rr < RPC; rr += NT / 32) {
        const float2* src = W + (r0 + rr) * Zp;
        for (int q = lane; q < Zh; q += 32) fast::cp_async16(buf + rr * BS + 2 * q, src + 2 * q, 16);
    }
    fast::cp_commit();
    fast::cp_wait<0>();
    __syncthreads();
    auto slot = [&](int rr, int nn, int aa) { return rr * BS + aa * TP + nn + aa / NB * ZPAD; };
    const float s = a.scale;
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
        v[n1] = fast::c2r_pre(xk, xm, rtws[k]);
    }
    __syncthreads();  // tile read: buf becomes transpose space
    Dft<R1, 1>::run(v);
    fast::twiddle_a<R1, TP, 1>(v, n2, tA);
#pragma unroll
    for (int aa = 0; aa < R1; ++aa) buf[slot(r, n2, aa)] = v[aa];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) v[i * TP + c] = buf[slot(r, c, n2 * NB + i)];
    fast::pass_b<R1, TP, 1>(v);
    float gtile = 0.f;
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) {
            const float2 z = v[i * TP + c];
            const float d0 = z.x * s, d1 = z.y * s;  // c - cbar (the state has no k = 0 mode)
            v[i * TP + c] = make_float2(d0 * fmaf(d0, c3 + d0, gp), d1 * fmaf(d1, c3 + d1, gp));
            if (GS) gtile += v[i * TP + c].x + v[i * TP + c].y;
        }
    if (GS) gacc += (double)gtile;
    fast::pass_b<R1, TP, -1>(v);
    fast::twiddle_b<R1, TP, -1>(v, n2, tB);
    __syncthreads();  // block-ownership reads of the first transpose done
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int c = 0; c < TP; ++c) buf[slot(r, c, n2 * NB + i)] = v[i * TP + c];
    __syncthreads();
#pragma unroll
    for (int aa = 0; aa < R1; ++aa) v[aa] = buf[slot(r, n2, aa)];
    Dft<R1, -1>::run(v);
    fast::r2c_store<R1, TP>(v, n2, xz + r * fast::zxs(M, TP), W + (r0 + r) * Zp, true, rtws);
}

template <int R1y, int TPy, int R1z, int TPz, bool GS>
__global__ void __launch_bounds__(8 * TPy, (512 / (8 * TPy)) > 0 ? 512 / (8 * TPy) : 1)
    fyzy_kernel(YZYArgs a) {
    using G = FusedGeom<R1y, TPy, R1z, TPz>;
    constexpr int L = G::L, NT = G::NT, M = G::M, RPC = G::RPC;
    constexpr int YBc = R1y == 20 ? 16 : 32;  // the y block of the layout (fused_yzy_shape checks a.YB)
    static_assert(NT % TPz == 0 && RPC >= 1, "z rows per item");
    extern __shared__ __align__(16) float4 smem4[];
    float2* buf = reinterpret_cast<float2*>(smem4);
    float2* tAy = buf + G::tile(a.Zp);
    float2* tBy = R1y == TPy ? tAy : tAy + L;
    float2* tAz = tAy + G::YTW;
    float2* tBz = tAz + M;
    float2* rtws = tBz + M;
    __shared__ int s_ticket;
    __shared__ int s_abort;
    fast::fill_twiddles<R1y, TPy>(tAy, tBy, a.twy, NT);
    fast::fill_twiddles<R1z, TPz>(tAz, tBz, a.twz, NT);
    for (int i = threadIdx.x; i <= M; i += NT) rtws[i] = a.rtw[i];
    if (threadIdx.x == 0) s_abort = 0;
    const double cbd = a.cbar ? *a.cbar : 0.0;
    const float gp = (float)(3.0 * cbd * cbd - 1.0);  // g'(cbar)
    const float c3 = (float)(3.0 * cbd);
    const int nyi = a.nchunks, nzi = a.ny / RPC, per = 2 * nyi + nzi;
    const int total = (a.nx + 2 * a.lag) * per;
    int* const abort_word = a.ctl + 1;
    int* const cnt_y = a.ctl + 2;
    int* const cnt_z = a.ctl + 2 + a.nx;
    const long long xs = (long long)a.YB * a.Zp;  // x stride of the y-blocked layout
    double gacc = 0.0;
    while (true) {
        __syncthreads();  // previous item done with s_ticket and the tile buffer
        if (threadIdx.x == 0) s_ticket = atomicAdd(a.ctl, 1);
        __syncthreads();
        const int t = s_ticket;
        if (t >= total) break;
        const int ph = t / per, o = t - ph * per;
        int kind, x, idx;
        if (o < nyi) {
            kind = 0, x = ph, idx = o;
        } else if (o < nyi + nzi) {
            kind = 1, x = ph - a.lag, idx = o - nyi;
        } else {
            kind = 2, x = ph - 2 * a.lag, idx = o - nyi - nzi;
        }
        if (x < 0 || x >= a.nx) continue;  // the pipeline's fill and drain phases
        if (kind > 0) {  // wait for the slab's previous stage
            if (threadIdx.x == 0 && !s_abort) {
                const bool ok = kind == 1 ? wait_count(cnt_y + x, nyi, abort_word)
                                          : wait_count(cnt_z + x, nzi, abort_word);
                if (!ok) s_abort = 1;
                __threadfence();
            }
            __syncthreads();
        }
        if (kind == 0) {
            y_item<R1y, TPy, YBc, 1>(a.S, a.W, x * xs, a, idx, buf, tAy, tBy);
        } else if (kind == 1) {
            // rows y = RPC idx .. RPC idx + RPC - 1 of slab x (inside one y block)
            const int y0 = RPC * idx;
            const long long r0 = ((long long)(y0 / a.YB) * a.nx + x) * a.YB + y0 % a.YB;
            z_item<R1z, TPz, NT, GS>(a.W, r0, a, buf, tAz, tBz, rtws, gp, c3, gacc);
        } else {
            y_item<R1y, TPy, YBc, -1>(a.W, a.W, x * xs, a, idx, buf, tAy, tBy);
        }
        if (kind < 2) {  // publish the item to the slab's next stage
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(kind == 0 ? cnt_y + x : cnt_z + x, 1);
            }
        }
    }
    if (GS) {  // fixed-order CTA reduction of the Allen-Cahn sums
        __shared__ double red[NT / 32 + 1];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gacc += __shfl_down_sync(0xffffffffu, gacc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gacc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (NT + 31) / 32; ++w) t += red[w];
            a.gsum[blockIdx.x] = t;
        }
    }
}

}  // namespace fused

// ------------------------------------------------------------------ host
namespace {
int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

struct OccEntry {
    const void* fn;
    int dev;
    size_t smem;
    int nb;
};

template <typename K>
cudaError_t occupancy(K kernel, size_t smem, int threads, int* per_sm) {
    static OccEntry cache[32];
    static int ncache = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < ncache; ++i)
        if (cache[i].fn == (const void*)kernel && cache[i].dev == dev && cache[i].smem == smem) {
            *per_sm = cache[i].nb;
            return cudaSuccess;
        }
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    nb = nb > 0 ? nb : 1;
    if (ncache < 32) cache[ncache++] = OccEntry{(const void*)kernel, dev, smem, nb};
    *per_sm = nb;
    return cudaSuccess;
}

template <int R1y, int TPy, int R1z, int TPz>
cudaError_t run_fyzy(const YZYArgs& a, cudaStream_t st, int* grid_used) {
    using G = fused::FusedGeom<R1y, TPy, R1z, TPz>;
    const size_t smem = sizeof(float2) * (size_t)G::floats2(a.Zp);
    auto kern = a.gsum ? fused::fyzy_kernel<R1y, TPy, R1z, TPz, true> : fused::fyzy_kernel<R1y, TPy, R1z, TPz, false>;
    int per = 0;
    cudaError_t e = occupancy(kern, smem, G::NT, &per);
    if (e != cudaSuccess) return e;
    const int nyi = a.nchunks, nzi = a.ny / G::RPC;
    const long long total = (long long)(a.nx + 2 * a.lag) * (2 * nyi + nzi);
    const int grid = (int)std::min<long long>(total, (long long)per * sm_count());
    if (grid_used) *grid_used = grid;
    // every CTA resident at once (cooperative launch); the ticket order alone
    // already rules out a deadlock, residency keeps waiting CTAs off the tail
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(G::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}
}  // namespace

int fused_yzy_shape(int ny, int M, int YB) {
    // (ny, M) pairs with kernels: the fast y and z transforms of equal edges;
    // a z item's 16 rows must sit inside one y block
    if (YB != choose_yblock(ny, true) || YB != (ny == 400 ? 16 : 32) || ny % 16) return 0;
    if ((ny == 1024 && M == 512) || (ny == 512 && M == 256) || (ny == 256 && M == 128) || (ny == 400 && M == 200))
        return 1;
    return 0;
}

bool fused_yzy_enabled() {
    // opt-in, read when a grid is created: the fused pass moves 5 instead of 9
    // sweeps per step but is slower than the three separate passes on GB300
    // (it is issue- and barrier-bound, not bandwidth-bound)
    const char* e = std::getenv("EVX_FUSE");
    return e && e[0] == '1' && fast_paths_enabled();
}

size_t fused_ctl_ints(int nx) { return 2 + 2 * (size_t)nx; }

cudaError_t launch_fused_yzy(const YZYArgs& a, cudaStream_t st, int* grid_used) {
    cudaError_t e = cudaMemsetAsync(a.ctl, 0, sizeof(int) * fused_ctl_ints(a.nx), st);
    if (e != cudaSuccess) return e;
    switch (a.ny) {
        case 1024: return run_fyzy<32, 32, 32, 16>(a, st, grid_used);
        case 512: return run_fyzy<32, 16, 32, 8>(a, st, grid_used);
        case 256: return run_fyzy<32, 8, 32, 4>(a, st, grid_used);
        case 400: return run_fyzy<20, 20, 20, 10>(a, st, grid_used);
    }
    return cudaErrorInvalidValue;
}

int fused_yzy_grid(const YZYArgs& a) {
    // upper bound of the CTAs a launch uses (for sizing the per-CTA partials)
    int per = 0, nt = 0;
    cudaError_t e = cudaSuccess;
    switch (a.ny) {
        case 1024: {
            using G = fused::FusedGeom<32, 32, 32, 16>;
            nt = G::NT;
            e = occupancy(fused::fyzy_kernel<32, 32, 32, 16, true>, sizeof(float2) * (size_t)G::floats2(a.Zp), nt, &per);
            break;
        }
        case 512: {
            using G = fused::FusedGeom<32, 16, 32, 8>;
            nt = G::NT;
            e = occupancy(fused::fyzy_kernel<32, 16, 32, 8, true>, sizeof(float2) * (size_t)G::floats2(a.Zp), nt, &per);
            break;
        }
        case 256: {
            using G = fused::FusedGeom<32, 8, 32, 4>;
            nt = G::NT;
            e = occupancy(fused::fyzy_kernel<32, 8, 32, 4, true>, sizeof(float2) * (size_t)G::floats2(a.Zp), nt, &per);
            break;
        }
        case 400: {
            using G = fused::FusedGeom<20, 20, 20, 10>;
            nt = G::NT;
            e = occupancy(fused::fyzy_kernel<20, 20, 20, 10, true>, sizeof(float2) * (size_t)G::floats2(a.Zp), nt, &per);
            break;
        }
        default: return 0;
    }
    if (e != cudaSuccess) return 0;
    return per * sm_count();
}

bool fused_timeout_flag(int* flag, bool clear) {
    int h = 0;
    if (cudaMemcpyFromSymbol(&h, fused::g_fused_timeout, sizeof(int)) != cudaSuccess) return false;
    if (clear && h) {
        int z = 0;
        cudaMemcpyToSymbol(fused::g_fused_timeout, &z, sizeof(int));
    }
    *flag = h;
    return true;
}

}  // namespace evx
