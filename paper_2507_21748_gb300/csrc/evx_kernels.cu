// CUDA kernels of the semi-implicit Fourier-spectral Cahn-Hilliard step
// (paper: Appendix "Semi-implicit timestepping"; update
//   c_hat <- (c_hat - dt M |k|^2 F{c^3 - c}) / (1 + dt M kappa |k|^4) ).
//
// Spectral buffers hold the half spectrum of a real nx*ny*nz field as
// complex64 in layout [x or kx][y or ky][kz], kz = 0..M (M = nz/2) padded to
// Zp columns. The state S holds F_y F_z c (transformed along y and z, real
// space along x) with the k = 0 mode removed; the mean of c is carried in
// FP64 beside it. One step is four passes over HBM:
//   y pass inverse     S -> W
//   z pass             W -> W : C2R along z, c = W/(ny nz) + cbar, g = c^3 - c, R2C
//   y pass forward     W -> W       (W = F_y F_z g)
//   x pass + update    W, S -> S : F_x both, c_hat' = a c_hat + b g_hat, F_x^-1 / nx
// with a = 1/(1 + dt M kappa |k|^4), b = -dt M |k|^2 a.
#include <cstdint>
#include <cstdlib>

#include <algorithm>

#include "evx_internal.h"

namespace evx {

// ------------------------------------------------------------ reductions
__device__ __forceinline__ double block_sum_double(double v, double* ws) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (warp == 0) {
        v = lane < nw ? ws[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;  // valid in thread 0
}

// ------------------------------------------------------------ strided pass
// Transform SP adjacent columns (pencils) of a [L][pitch] tile along L, in
// groups of pencils small enough for one fft_tile call.
template <int DIR>
__device__ __forceinline__ void fft_cols(float2* tile, int L, int pitch, const Plan& plan,
                                         const float2* tws) {
    const int g = max(1, min(SP, TILE_CAP / L));
    for (int p0 = 0; p0 < SP; p0 += g) fft_tile<DIR, true>(Tile{tile + p0, L, min(g, SP - p0), pitch, 1}, plan, tws);
}

template <int DIR>
__global__ void __launch_bounds__(NT, 2) spass_kernel(SPassArgs a) {
    extern __shared__ float2 smem[];
    float2* tile = smem;                 // [L][SP]
    float2* tws = smem + a.L * SP;       // [L]
    for (int i = threadIdx.x; i < a.L; i += NT) tws[i] = a.tw[i];
    const int chunk = blockIdx.x, outer = blockIdx.y;
    const long long base = (long long)outer * a.os + (long long)chunk * SP;
    const int col0 = chunk * SP;
    const bool full = col0 + SP <= a.ncols;
    const long long nbuf = (long long)(a.L / a.YB) * a.os2;  // complex elements of in / out
    if (full) {
        for (int e = threadIdx.x; e < a.L * (SP / 2); e += NT) {
            const int i = e / (SP / 2), q = e % (SP / 2);
            const long long idx = base + split_off(i, a.YB, a.rs, a.os2) + 2 * q;
            const float4 v = EVX_IN(idx + 1, nbuf) ? *reinterpret_cast<const float4*>(a.in + idx)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<float4*>(tile)[e] = v;
        }
    } else {
        for (int e = threadIdx.x; e < a.L * SP; e += NT) {
            const int i = e / SP, p = e % SP;
            const long long idx = base + split_off(i, a.YB, a.rs, a.os2) + p;
            tile[e] = (col0 + p < a.ncols && EVX_IN(idx, nbuf)) ? a.in[idx] : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    fft_cols<DIR>(tile, a.L, SP, a.plan, tws);
    if (full) {
        for (int e = threadIdx.x; e < a.L * (SP / 2); e += NT) {
            const int i = e / (SP / 2), q = e % (SP / 2);
            const long long idx = base + split_off(i, a.YB, a.rs, a.os2) + 2 * q;
            if (EVX_IN(idx + 1, nbuf)) *reinterpret_cast<float4*>(a.out + idx) = reinterpret_cast<const float4*>(tile)[e];
        }
    } else {
        for (int e = threadIdx.x; e < a.L * SP; e += NT) {
            const int i = e / SP, p = e % SP;
            const long long idx = base + split_off(i, a.YB, a.rs, a.os2) + p;
            if (col0 + p < a.ncols && EVX_IN(idx, nbuf)) a.out[idx] = tile[e];
        }
    }
}

// load SP columns of an x line into tile columns [c0, c0+SP) of a [L][2SP] tile
__device__ __forceinline__ void load_x_cols(float2* tile, int c0, const float2* g, long long base,
                                            long long rs, int L, int col0, int ncols, long long nbuf) {
    if (col0 + SP <= ncols) {
        for (int e = threadIdx.x; e < L * (SP / 2); e += NT) {
            const int i = e / (SP / 2), q = e % (SP / 2);
            const long long idx = base + i * rs + 2 * q;
            const float4 v = EVX_IN(idx + 1, nbuf) ? *reinterpret_cast<const float4*>(g + idx)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(tile + i * (2 * SP) + c0 + 2 * q) = v;
        }
    } else {
        for (int e = threadIdx.x; e < L * SP; e += NT) {
            const int i = e / SP, p = e % SP;
            const long long idx = base + i * rs + p;
            tile[i * (2 * SP) + c0 + p] = (col0 + p < ncols && EVX_IN(idx, nbuf)) ? g[idx] : make_float2(0.f, 0.f);
        }
    }
}

// ------------------------------------------------------ x pass + update
__global__ void __launch_bounds__(NT, 1) xupdate_kernel(XUpdArgs a) {
    extern __shared__ float2 smem[];
    const int L = a.L;
    float2* tile = smem;                 // [L][2 SP]: W in cols [0,SP), S in [SP, 2SP)
    float2* tws = smem + L * 2 * SP;     // [L]
    for (int i = threadIdx.x; i < L; i += NT) tws[i] = a.tw[i];
    const int chunk = blockIdx.x, ky = blockIdx.y;
    const int col0 = chunk * SP;
    const long long base = split_off(ky, a.YB, a.os, a.os2) + col0;
    const bool haveW = a.W != nullptr;
    const bool pre = a.model == 2;  // preconditioner only: S' = F_x^-1 (dt / (1 + dt M0 kappa |k|^4)) F_x W
    const bool blk = a.model == 3;  // block propagator: L^n c_hat + B (sum_{j<n} L^j) N_hat
    const float gpb = blk ? (float)(3.0 * (*a.cbar) * (*a.cbar) - 1.0) : 0.f;
    const long long nbuf = (long long)(a.ny / a.YB) * a.os2;  // complex elements of W, S, S_out
    if (haveW) load_x_cols(tile, 0, a.W, base, a.rs, L, col0, a.ncols, nbuf);
    if (!pre) load_x_cols(tile, SP, a.S, base, a.rs, L, col0, a.ncols, nbuf);
    __syncthreads();
    if (haveW) fft_cols<-1>(tile, L, 2 * SP, a.plan, tws);
    if (!pre) fft_cols<-1>(tile + SP, L, 2 * SP, a.plan, tws);
    const float k2y = a.k2y[ky];
    for (int e = threadIdx.x; e < L * SP; e += NT) {
        const int i = e / SP, p = e % SP;
        const int kz = col0 + p;
        if (kz < a.ncols) {
            const float k2 = a.k2x[i] + k2y + a.k2z[kz];
            // Cahn-Hilliard: a = 1/D, b = -dt M |k|^2 / D, D = 1 + dt M kappa |k|^4;
            // Allen-Cahn:   a = 1/D, b = -dt L / D,       D = 1 + dt L kappa |k|^2
            const float ainv = a.invL / fmaf(a.dtMk, a.model == 1 ? k2 : k2 * k2, 1.f);
            const float b = -a.dtM * (a.model == 1 ? 1.f : k2) * ainv;
            const float2 c = pre ? make_float2(0.f, 0.f) : tile[i * (2 * SP) + SP + p];
            float2 r = make_float2(ainv * c.x, ainv * c.y);
            if (blk) {  // L = (1 - dt M |k|^2 g'(cbar)) / D; ainv = invL / D
                const float Lk = fmaf(-a.dtM * k2, gpb, 1.f) * ainv * (float)L;
                float P = 1.f, S = 0.f;
                for (int j = 0; j < a.nblk; ++j) {
                    S += P;
                    P *= Lk;
                }
                const float2 gh = tile[i * (2 * SP) + p];
                const float bs = -a.dtM * k2 * ainv * S;
                r = make_float2(fmaf(bs, gh.x, P * a.invL * c.x), fmaf(bs, gh.y, P * a.invL * c.y));
            } else if (pre) {  // dtM holds dt here: r = dt / (1 + dt M0 kappa |k|^4) g_hat / L
                const float2 gh = tile[i * (2 * SP) + p];
                r = make_float2(a.dtM * ainv * gh.x, a.dtM * ainv * gh.y);
            } else if (haveW) {
                const float2 gh = tile[i * (2 * SP) + p];
                r.x = fmaf(b, gh.x, r.x);
                r.y = fmaf(b, gh.y, r.y);
            }
            if (i == 0 && ky == 0 && kz == 0) r = make_float2(0.f, 0.f);  // mean carried in FP64
            tile[i * (2 * SP) + SP + p] = r;
        }
    }
    __syncthreads();
    fft_cols<1>(tile + SP, L, 2 * SP, a.plan, tws);
    if (col0 + SP <= a.ncols) {
        for (int e = threadIdx.x; e < L * (SP / 2); e += NT) {
            const int i = e / (SP / 2), q = e % (SP / 2);
            const long long idx = base + i * a.rs + 2 * q;
            if (EVX_IN(idx + 1, nbuf))
                *reinterpret_cast<float4*>(a.S_out + idx) = *reinterpret_cast<const float4*>(tile + i * (2 * SP) + SP + 2 * q);
        }
    } else {
        for (int e = threadIdx.x; e < L * SP; e += NT) {
            const int i = e / SP, p = e % SP;
            const long long idx = base + i * a.rs + p;
            if (col0 + p < a.ncols && EVX_IN(idx, nbuf)) a.S_out[idx] = tile[i * (2 * SP) + SP + p];
        }
    }
}

// ------------------------------------------- energy: gradient term (x pass)
__global__ void __launch_bounds__(NT, 1) xenergy_kernel(XEnergyArgs a) {
    extern __shared__ float2 smem[];
    __shared__ double ws[NT / 32];
    const int L = a.L;
    float2* tile = smem;                 // [L][2 SP], S in cols [SP, 2SP)
    float2* tws = smem + L * 2 * SP;
    for (int i = threadIdx.x; i < L; i += NT) tws[i] = a.tw[i];
    const int chunk = blockIdx.x, ky = blockIdx.y;
    const int col0 = chunk * SP;
    const long long base = split_off(ky, a.YB, a.os, a.os2) + col0;
    load_x_cols(tile, SP, a.S, base, a.rs, L, col0, a.ncols, (long long)(a.ny / a.YB) * a.os2);
    __syncthreads();
    fft_cols<-1>(tile + SP, L, 2 * SP, a.plan, tws);
    const double k2y = a.k2y[ky];
    double acc = 0.0;
    for (int e = threadIdx.x; e < L * SP; e += NT) {
        const int i = e / SP, p = e % SP;
        const int kz = col0 + p;
        if (kz < a.ncols) {
            const double k2 = (double)a.k2x[i] + k2y + (double)a.k2z[kz];
            const float2 c = tile[i * (2 * SP) + SP + p];
            const double w = (kz == 0 || kz == a.M) ? 1.0 : 2.0;  // Hermitian half spectrum
            acc += w * k2 * ((double)c.x * c.x + (double)c.y * c.y);
        }
    }
    acc = block_sum_double(acc, ws);
    if (threadIdx.x == 0) a.partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// ------------------------------------------------------------- z pass
template <int MODE>
__global__ void __launch_bounds__(NT, 2) zpass_kernel(ZPassArgs a) {
    extern __shared__ float2 smem[];
    __shared__ double ws[NT / 32];
    const int M = a.M, PZ = a.PZ, rows = a.rows_per_cta;
    float2* tile = smem;                  // [rows][PZ]
    float2* tws = smem + rows * PZ;       // [M]
    float2* rtws = tws + M;               // [M + 1]
    for (int i = threadIdx.x; i < M; i += NT) tws[i] = a.tw[i];
    for (int i = threadIdx.x; i <= M; i += NT) rtws[i] = a.rtw[i];
    const long long row0 = (long long)blockIdx.x * rows;
    const int nr = (int)min((long long)rows, a.nrows - row0);
    const int H = M / 2 + 1;  // pairs (k, M - k), k = 0 .. M/2

    if (MODE == Z_R2C) {
        // real row of nz = 2M floats read as M complex z[n] = x[2n] + i x[2n+1].
        // With a.cbar set, the FP64 mean is subtracted first ((x - hi) - lo; x - hi
        // is exact for x within a factor 2 of hi): the transforms then never carry
        // the large k = 0 sums whose FP32 roundoff would spill into the other modes.
        const double cbd = a.cbar ? *a.cbar : 0.0;
        const float cb = (float)cbd;
        const float cbl = (float)(cbd - (double)cb);
        for (int e = threadIdx.x; e < rows * M; e += NT) {
            const int r = e / M, n = e - r * M;
            float2 x = make_float2(0.f, 0.f);
            if (r < nr) {
                const long long rr = a.map_rows ? user_row(row0 + r, a.YB, a.nxr, a.nyr) : row0 + r;
                if (EVX_IN(rr * a.rpitch + 2 * n + 1, a.nrows * a.rpitch))
                    x = reinterpret_cast<const float2*>(a.rin + rr * a.rpitch)[n];
                x = make_float2((x.x - cb) - cbl, (x.y - cb) - cbl);
            }
            tile[r * PZ + n] = x;
        }
        __syncthreads();
    } else {
        for (int e = threadIdx.x; e < rows * (M + 1); e += NT) {
            const int r = e / (M + 1), i = e - r * (M + 1);
            const long long idx = (row0 + r) * a.Zp + i;
            tile[r * PZ + i] = (r < nr && EVX_IN(idx, a.nrows * a.Zp)) ? a.in[idx] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // C2R pre-processing: Z[k] = (X_k + conj X_{M-k}) + i e^{+2 pi i k/nz} (X_k - conj X_{M-k});
        // imaginary parts of X_0 and X_M are dropped (real field).
        for (int e = threadIdx.x; e < rows * H; e += NT) {
            const int r = e / H, k = e - r * H;
            float2* row = tile + r * PZ;
            if (k == 0) {
                const float2 x0 = row[0], xm = row[M];
                row[0] = make_float2(x0.x + xm.x, x0.x - xm.x);
            } else {
                const int m = M - k;
                const float2 xk = row[k], xm = row[m];
                const float2 A = make_float2(xk.x + xm.x, xk.y - xm.y);
                const float2 B = make_float2(xk.x - xm.x, xk.y + xm.y);
                const float2 zk = cadd(A, mul_i<1>(cmul(cconj(rtws[k]), B)));
                const float2 A2 = make_float2(xm.x + xk.x, xm.y - xk.y);
                const float2 B2 = make_float2(xm.x - xk.x, xm.y + xk.y);
                const float2 zm = cadd(A2, mul_i<1>(cmul(cconj(rtws[m]), B2)));
                row[k] = zk;
                if (m != k) row[m] = zm;
            }
        }
        __syncthreads();
        fft_tile<1, false>(Tile{tile, M, rows, 1, PZ}, a.plan, tws);
        // mean split into FP32 hi + lo parts: c = (z s + lo) + hi rounds once at
        // the scale of c without a common bias (adding (float)cbar alone would
        // shift every voxel by the same rounding error of cbar)
        const double cbd = a.cbar ? *a.cbar : 0.0;
        const float cb = (float)cbd;
        const float cbl = (float)(cbd - (double)cb);
        const float gp = a.nl_only ? 0.f : (float)(3.0 * cbd * cbd - 1.0);  // g'(cbar); 0: remainder N only
        const float c3 = (float)(3.0 * cbd);
        const float s = a.scale;
        double acc = 0.0;
        for (int e = threadIdx.x; e < nr * M; e += NT) {
            const int r = e / M, n = e - r * M;
            const float2 z = tile[r * PZ + n];
            if (MODE == Z_ADJ) {
                const float2 cn = EVX_IN((row0 + r) * a.cnpitch + 2 * n + 1, a.nrows * a.cnpitch)
                                      ? reinterpret_cast<const float2*>(a.cn + (row0 + r) * a.cnpitch)[n]
                                      : make_float2(0.f, 0.f);
                const float d0 = fmaf(3.f * cn.x, cn.x, -1.f), d1 = fmaf(3.f * cn.y, cn.y, -1.f);
                tile[r * PZ + n] = make_float2(z.x * s * d0, z.y * s * d1);
            } else {
                const float c0 = fmaf(z.x, s, cbl) + cb, c1 = fmaf(z.y, s, cbl) + cb;
                if (MODE == Z_STEP) {
                    if (a.rout && EVX_IN((row0 + r) * a.rpitch + 2 * n + 1, a.nrows * a.rpitch))
                        reinterpret_cast<float2*>(a.rout + (row0 + r) * a.rpitch)[n] = make_float2(c0, c1);
                    // g(c) - g(cbar) from d = c - cbar (see the fast z pass)
                    const float d0 = z.x * s, d1 = z.y * s;
                    const float2 gv = make_float2(d0 * fmaf(d0, c3 + d0, gp), d1 * fmaf(d1, c3 + d1, gp));
                    tile[r * PZ + n] = gv;
                    if (a.gsum) acc += (double)gv.x + (double)gv.y;
                } else {  // Z_C2R
                    const long long rr = a.map_rows ? user_row(row0 + r, a.YB, a.nxr, a.nyr) : row0 + r;
                    if (a.rout && EVX_IN(rr * a.rpitch + 2 * n + 1, a.nrows * a.rpitch)) {
                        float2* o = reinterpret_cast<float2*>(a.rout + rr * a.rpitch) + n;
                        if (a.accumulate) {  // the variable-mobility step adds its increment
                            const float2 prev = *o;
                            *o = make_float2(prev.x + c0, prev.y + c1);
                        } else {
                            *o = make_float2(c0, c1);
                        }
                    }
                    if (a.partials) {
                        const double q0 = (double)c0 * c0 - 1.0, q1 = (double)c1 * c1 - 1.0;
                        acc += q0 * q0 + q1 * q1;
                    }
                }
            }
        }
        if (MODE == Z_C2R) {
            if (a.partials) {
                acc = block_sum_double(acc, ws);
                if (threadIdx.x == 0) a.partials[blockIdx.x] = acc;
            }
            return;
        }
        if (MODE == Z_STEP && a.gsum) {  // uniform: every thread of the CTA takes it
            acc = block_sum_double(acc, ws);
            if (threadIdx.x == 0) a.gsum[blockIdx.x] = acc;
        }
        __syncthreads();
    }
    fft_tile<-1, false>(Tile{tile, M, rows, 1, PZ}, a.plan, tws);
    // R2C post-processing: X_k = (Z_k + conj Z_{M-k})/2 - i e^{-2 pi i k/nz} (Z_k - conj Z_{M-k})/2
    for (int e = threadIdx.x; e < rows * H; e += NT) {
        const int r = e / H, k = e - r * H;
        float2* row = tile + r * PZ;
        if (k == 0) {
            const float2 z0 = row[0];
            row[0] = make_float2(z0.x + z0.y, 0.f);
            row[M] = make_float2(z0.x - z0.y, 0.f);
        } else {
            const int m = M - k;
            const float2 zk = row[k], zm = row[m];
            const float2 A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            const float2 B = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y + zm.y));
            const float2 xk = cadd(A, mul_i<-1>(cmul(rtws[k], B)));
            const float2 A2 = make_float2(0.5f * (zm.x + zk.x), 0.5f * (zm.y - zk.y));
            const float2 B2 = make_float2(0.5f * (zm.x - zk.x), 0.5f * (zm.y + zk.y));
            const float2 xm = cadd(A2, mul_i<-1>(cmul(rtws[m], B2)));
            row[k] = xk;
            if (m != k) row[m] = xm;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * (M + 1); e += NT) {
        const int r = e / (M + 1), i = e - r * (M + 1);
        const long long idx = (row0 + r) * a.Zp + i;
        if (EVX_IN(idx, a.nrows * a.Zp)) a.out[idx] = tile[r * PZ + i];
    }
}

// --------------------------------------------------- FP64 sums of a field
// partials[b] = sum over rows b, b + nblocks, ... of sum_z c[row * pitch + z]
__global__ void __launch_bounds__(NT) sum_rows_kernel(const float* c, long long nrows, int rowlen,
                                                      long long pitch, double* partials) {
    __shared__ double ws[NT / 32];
    double acc = 0.0;
    for (long long r = blockIdx.x; r < nrows; r += gridDim.x) {
        const float* row = c + r * pitch;
        for (int z = threadIdx.x; z < rowlen; z += NT)
            if (EVX_IN(r * pitch + z, nrows * pitch)) acc += (double)row[z];
    }
    acc = block_sum_double(acc, ws);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// FP64 row sums with 16-byte loads (rowlen and pitch multiples of 4, c 16-byte
// aligned): rows to warps, a lane takes every 32nd float4 of its warp's row. Each
// lane adds up to 32 floats exactly in FP32 as a rounded sum s and the sum e of the
// TwoSum error terms (Knuth), and passes s + e to its FP64 accumulator: the FP64
// work (the slow pipe on this GPU) falls to 2 operations per 32 elements, and the
// result is the FP64 sum to within the FP64 rounding of the old kernel.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x) {
    const float t = s + x, bp = t - s;
    e += (s - (t - bp)) + (x - bp);
    s = t;
}
__global__ void __launch_bounds__(NT) sum_rows_vec_kernel(const float* c, long long nrows, int rowlen,
                                                          long long pitch, double* partials) {
    __shared__ double ws[NT / 32];
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * NT) >> 5;
    double acc = 0.0;
    for (long long r = ((long long)blockIdx.x * NT + threadIdx.x) >> 5; r < nrows; r += nw) {
        const float4* row = reinterpret_cast<const float4*>(c + r * pitch);
        float s = 0.f, e = 0.f;
        int k = 0;
        for (int q = lane; q < rowlen / 4; q += 32) {
            const float4 v = EVX_IN(r * pitch + 4 * q + 3, nrows * pitch) ? row[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            two_sum_acc(s, e, v.x);
            two_sum_acc(s, e, v.y);
            two_sum_acc(s, e, v.z);
            two_sum_acc(s, e, v.w);
            if (++k == 8) {
                acc += (double)s + (double)e;
                s = e = 0.f;
                k = 0;
            }
        }
        acc += (double)s + (double)e;
    }
    acc = block_sum_double(acc, ws);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// The k = 0 mode of a state that is spectral in y and z and real in x is the
// x-sum of its (ky = 0, kz = 0) line: removing it subtracts the line's mean
// from each of its n elements (stride apart). One block, FP64 sum.
__global__ void __launch_bounds__(1024) remove_k0_kernel(float2* line, int n, long long stride) {
    __shared__ double ws[32];
    __shared__ double mre, mim;
    double sr = 0.0, si = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) {
        const float2 v = line[(long long)i * stride];
        sr += (double)v.x;
        si += (double)v.y;
    }
    sr = block_sum_double(sr, ws);
    __syncthreads();
    si = block_sum_double(si, ws);
    if (threadIdx.x == 0) {
        mre = sr / n;
        mim = si / n;
    }
    __syncthreads();
    const float fr = (float)mre, fi = (float)mim;
    for (int i = threadIdx.x; i < n; i += 1024) {
        float2 v = line[(long long)i * stride];
        v.x -= fr;
        v.y -= fi;
        line[(long long)i * stride] = v;
    }
}

__global__ void __launch_bounds__(1024) reduce_partials_kernel(const double* partials, int n,
                                                                double* out, double scale) {
    __shared__ double ws[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) acc += partials[i];
    acc = block_sum_double(acc, ws);
    if (threadIdx.x == 0) *out = acc * scale;
}

// ------------------------------------------- variable-mobility FD stencils
// Real C-order fields (x, y, z), z fastest, periodic. A CTA walks (x, y) rows
// (grid-stride); its threads run along z, so every neighbour row is read
// coalesced. Rows r and r + 1 (y neighbours) and r +- ny (x neighbours) are
// processed by CTAs running at the same time, so the re-reads hit L2.
struct VmRow {
    long long base, xp, xm, yp, ym;
};
__device__ __forceinline__ VmRow vm_row(long long row, int nx, int ny, int nz) {
    const int x = (int)(row / ny), y = (int)(row - (long long)x * ny);
    VmRow r;
    r.base = row * nz;
    r.xp = ((long long)(x + 1 == nx ? 0 : x + 1) * ny + y) * nz;
    r.xm = ((long long)(x == 0 ? nx - 1 : x - 1) * ny + y) * nz;
    r.yp = ((long long)x * ny + (y + 1 == ny ? 0 : y + 1)) * nz;
    r.ym = ((long long)x * ny + (y == 0 ? ny - 1 : y - 1)) * nz;
    return r;
}

// checked load of a real field of n values (the bounds-checked build tests i)
__device__ __forceinline__ float ldf(const float* __restrict__ p, long long i, long long n) {
    return EVX_IN(i, n) ? p[i] : 0.f;
}

// mu = c^3 - c - (kappa / h^2) (sum of the 6 neighbours - 6 c)
__global__ void __launch_bounds__(256) vm_mu_kernel(const float* __restrict__ c, float* __restrict__ mu, int nx,
                                                     int ny, int nz, float kh2) {
    const long long nrows = (long long)nx * ny;
    for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
        const VmRow r = vm_row(row, nx, ny, nz);
        for (int z = threadIdx.x; z < nz; z += blockDim.x) {
            const int zp = z + 1 == nz ? 0 : z + 1, zm = z == 0 ? nz - 1 : z - 1;
            const long long V = nrows * nz;
            const float v = ldf(c, r.base + z, V);
            const float nb = ((ldf(c, r.xp + z, V) + ldf(c, r.xm + z, V)) + (ldf(c, r.yp + z, V) + ldf(c, r.ym + z, V))) +
                             (ldf(c, r.base + zp, V) + ldf(c, r.base + zm, V));
            if (EVX_IN(r.base + z, V)) mu[r.base + z] = v * (v * v - 1.f) - kh2 * fmaf(-6.f, v, nb);
        }
    }
}

// rhs = (1 / h^2) sum_j (M_i + M_j)/2 (mu_j - mu_i), M = M0 max(1 - c^2, 0)
__global__ void __launch_bounds__(256) vm_rhs_kernel(const float* __restrict__ c, const float* __restrict__ mu,
                                                      float* __restrict__ rhs, int nx, int ny, int nz, float M0,
                                                      float ih2) {
    const long long nrows = (long long)nx * ny;
    auto mob = [&](float v) { return M0 * fmaxf(1.f - v * v, 0.f); };
    for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
        const VmRow r = vm_row(row, nx, ny, nz);
        for (int z = threadIdx.x; z < nz; z += blockDim.x) {
            const int zp = z + 1 == nz ? 0 : z + 1, zm = z == 0 ? nz - 1 : z - 1;
            const long long idx[6] = {r.xp + z, r.xm + z, r.yp + z, r.ym + z, r.base + zp, r.base + zm};
            const long long V = nrows * nz;
            const float mi = mob(ldf(c, r.base + z, V)), ui = ldf(mu, r.base + z, V);
            float acc = 0.f;
#pragma unroll
            for (int q = 0; q < 6; ++q) acc = fmaf(0.5f * (mi + mob(ldf(c, idx[q], V))), ldf(mu, idx[q], V) - ui, acc);
            if (EVX_IN(r.base + z, V)) rhs[r.base + z] = acc * ih2;
        }
    }
}

// Both stencils in one pass (rhs straight from c, mu never stored): a CTA owns
// TY x TZ columns (y, z) and marches along x through XC planes, with c in a ring
// of 8 planes (2-halo in y and z), and mu and the mobility M(c) in rings of 4
// planes (1-halo) in shared memory. Plane x + 3 is copied in with cp.async while
// plane x is computed; each thread's shared and global offsets are the same on
// every plane and are computed once. Each c value is read from HBM once (its
// halo copies mostly from L2) and rhs written once: 8 B per voxel against 20 B
// for the two separate kernels. The arithmetic and its grouping are those of
// vm_mu_kernel and vm_rhs_kernel (same results to the bit).
constexpr int VM_TY = 8, VM_TZ = 64, VM_XC = 64, VM_CS = 8, VM_NT = 256;
constexpr int VM_CY = VM_TY + 4, VM_CZ = VM_TZ + 4, VM_MY = VM_TY + 2, VM_MZ = VM_TZ + 2;
constexpr int VM_CP = VM_CY * VM_CZ, VM_MP = VM_MY * VM_MZ;  // floats per c / mu plane
constexpr int VM_NL = (VM_CP + VM_NT - 1) / VM_NT, VM_NM = (VM_MP + VM_NT - 1) / VM_NT, VM_NR = VM_TY * VM_TZ / VM_NT;
__device__ __forceinline__ int vm_wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__global__ void __launch_bounds__(VM_NT) vm_fd_kernel(const float* __restrict__ c, float* __restrict__ rhs, int nx,
                                                       int ny, int nz, float kh2, float M0, float ih2) {
    static_assert(VM_TY * VM_TZ % VM_NT == 0, "rhs points per thread");
    extern __shared__ float vm_smem[];
    float* cs = vm_smem;                  // [VM_CS][VM_CY][VM_CZ]
    float* ms = cs + VM_CS * VM_CP;       // [4][VM_MY][VM_MZ] mu
    float* mbs = ms + 4 * VM_MP;          // [4][VM_MY][VM_MZ] M(c)
    const int y0 = blockIdx.x * VM_TY, z0 = blockIdx.y * VM_TZ, x0 = blockIdx.z * VM_XC;
    const int xe = min(x0 + VM_XC, nx);
    const long long V = (long long)nx * ny * nz;
    const int tid = threadIdx.x;
    // this thread's points: c loads (plane offset in c, index in a c plane), mu / M
    // points (index in a mu plane, centre index in a c plane), rhs points (likewise)
    int lg[VM_NL], ls[VM_NL], mi_[VM_NM], mc[VM_NM], rm[VM_NR], ro[VM_NR];
#pragma unroll
    for (int k = 0; k < VM_NL; ++k) {
        const int i = tid + k * VM_NT, r = i / VM_CZ, q = i - r * VM_CZ;
        lg[k] = i < VM_CP ? vm_wrap(y0 + r - 2, ny) * nz + vm_wrap(z0 + q - 2, nz) : -1;
        ls[k] = i;
    }
#pragma unroll
    for (int k = 0; k < VM_NM; ++k) {
        const int i = tid + k * VM_NT, r = i / VM_MZ, q = i - r * VM_MZ;
        mi_[k] = i < VM_MP ? i : -1;
        mc[k] = (r + 1) * VM_CZ + q + 1;
    }
#pragma unroll
    for (int k = 0; k < VM_NR; ++k) {
        const int i = tid + k * VM_NT, r = i / VM_TZ, q = i - r * VM_TZ;
        rm[k] = (r + 1) * VM_MZ + q + 1;
        ro[k] = (y0 + r) * nz + z0 + q;
    }
    auto load_c = [&](int xp) {  // plane xp (x0 - 2 <= xp <= xe + 1) into slot (xp + 8) % 8, one commit group
        float* dst = cs + ((xp + VM_CS) % VM_CS) * VM_CP;
        const long long pb = (long long)vm_wrap(xp, nx) * ny * nz;
#pragma unroll
        for (int k = 0; k < VM_NL; ++k)
            if (lg[k] >= 0) {
                const long long g = pb + lg[k];
                cp_async4(dst + ls[k], c + (EVX_IN(g, V) ? g : 0), EVX_IN(g, V));
            }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto mu_plane = [&](int xp) {  // mu and M of plane xp, rows y0 - 1 .., columns z0 - 1 ..
        const float* c0 = cs + ((xp + VM_CS) % VM_CS) * VM_CP;
        const float* cm = cs + ((xp + VM_CS - 1) % VM_CS) * VM_CP;
        const float* cp = cs + ((xp + 1) % VM_CS) * VM_CP;
        float* mo = ms + ((xp + 4) & 3) * VM_MP;
        float* bo = mbs + ((xp + 4) & 3) * VM_MP;
#pragma unroll
        for (int k = 0; k < VM_NM; ++k)
            if (mi_[k] >= 0) {
                const int e = mc[k];
                const float v = c0[e];
                const float nb = ((cp[e] + cm[e]) + (c0[e + VM_CZ] + c0[e - VM_CZ])) + (c0[e + 1] + c0[e - 1]);
                mo[mi_[k]] = v * (v * v - 1.f) - kh2 * fmaf(-6.f, v, nb);
                bo[mi_[k]] = M0 * fmaxf(1.f - v * v, 0.f);
            }
    };
    for (int xp = x0 - 2; xp <= x0 + 2; ++xp) load_c(xp);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    mu_plane(x0 - 1);
    mu_plane(x0);
    for (int x = x0; x < xe; ++x) {
        // planes x - 1 .. x + 2 are in; plane x + 3 takes the slot of plane x - 5
        if (x + 3 <= xe + 1)
            load_c(x + 3);
        else
            asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // all but the newest group: plane x + 2
        __syncthreads();
        mu_plane(x + 1);  // the mu and M slots of plane x - 3
        __syncthreads();
        const float* u0 = ms + ((x + 4) & 3) * VM_MP;
        const float* um = ms + ((x + 3) & 3) * VM_MP;
        const float* up = ms + ((x + 5) & 3) * VM_MP;
        const float* b0 = mbs + ((x + 4) & 3) * VM_MP;
        const float* bm = mbs + ((x + 3) & 3) * VM_MP;
        const float* bp = mbs + ((x + 5) & 3) * VM_MP;
        const long long pb = (long long)x * ny * nz;
#pragma unroll
        for (int k = 0; k < VM_NR; ++k) {
            const int e = rm[k];
            const float mi = b0[e], ui = u0[e];
            // neighbours in the order x+, x-, y+, y-, z+, z-
            float acc = 0.f;
            acc = fmaf(0.5f * (mi + bp[e]), up[e] - ui, acc);
            acc = fmaf(0.5f * (mi + bm[e]), um[e] - ui, acc);
            acc = fmaf(0.5f * (mi + b0[e + VM_MZ]), u0[e + VM_MZ] - ui, acc);
            acc = fmaf(0.5f * (mi + b0[e - VM_MZ]), u0[e - VM_MZ] - ui, acc);
            acc = fmaf(0.5f * (mi + b0[e + 1]), u0[e + 1] - ui, acc);
            acc = fmaf(0.5f * (mi + b0[e - 1]), u0[e - 1] - ui, acc);
            const long long o = pb + ro[k];
            if (EVX_IN(o, V)) rhs[o] = acc * ih2;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// FD energy partials: (c^2 - 1)^2 / 4 + (kappa / 2h^2) sum_d (c_{i+e_d} - c_i)^2 per voxel, FP64
__global__ void __launch_bounds__(256) vm_energy_kernel(const float* __restrict__ c, int nx, int ny, int nz,
                                                         double k2h2, double* partials) {
    __shared__ double ws[32];
    const long long nrows = (long long)nx * ny;
    double acc = 0.0;
    for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
        const VmRow r = vm_row(row, nx, ny, nz);
        for (int z = threadIdx.x; z < nz; z += blockDim.x) {
            const int zp = z + 1 == nz ? 0 : z + 1;
            const long long V = nrows * nz;
            const double v = ldf(c, r.base + z, V);
            const double q = v * v - 1.0;
            const double dx = ldf(c, r.xp + z, V) - v, dy = ldf(c, r.yp + z, V) - v, dz = ldf(c, r.base + zp, V) - v;
            acc += 0.25 * q * q + k2h2 * (dx * dx + dy * dy + dz * dz);
        }
    }
    acc = block_sum_double(acc, ws);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Allen-Cahn: the k = 0 mode of the update has D = 1, so the FP64 mean moves by
// cbar' = cbar - dt L mean(g(c)), mean(g(c)) = g(cbar) + sum(g(c) - g(cbar)) / V
__global__ void __launch_bounds__(1024) ac_mean_kernel(const double* gsum, int n, double* cbar, double dtL,
                                                        double invV) {
    __shared__ double ws[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) acc += gsum[i];
    acc = block_sum_double(acc, ws);
    if (threadIdx.x == 0) {
        const double c = *cbar;
        *cbar = c - dtL * (c * c * c - c + acc * invV);
    }
}

__global__ void cadd_kernel(const float2* a, const float2* b, float2* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = cadd(a[i], b[i]);
}

// ------------------------------------------------------------- launchers
size_t spass_smem(int L) { return sizeof(float2) * ((size_t)L * SP + L); }
size_t xupdate_smem(int L) { return sizeof(float2) * ((size_t)L * 2 * SP + L); }
size_t zpass_smem(int M, int PZ, int rows) {
    return sizeof(float2) * ((size_t)rows * PZ + M + M + 1);
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int bounds_line_kernels(bool clear) {
#ifdef EVX_BOUNDS_CHECK
    int h = 0;
    if (cudaMemcpyFromSymbol(&h, g_bounds_line, sizeof(int)) != cudaSuccess) return -1;
    if (clear && h) {
        const int z = 0;
        cudaMemcpyToSymbol(g_bounds_line, &z, sizeof(int));
    }
    return h;
#else
    (void)clear;
    return 0;
#endif
}

bool fast_paths_enabled() {
    static int on = -1;
    if (on < 0) {
        const char* e = getenv("EVX_GENERIC");
        on = (e && e[0] == '1') ? 0 : 1;
    }
    return on == 1;
}

cudaError_t launch_spass(const SPassArgs& a, int dir, cudaStream_t st) {
    cudaError_t fe;
    if (!a.generic && fast_paths_enabled() && fast_spass(a, dir, st, &fe)) return fe;
    const size_t sm = spass_smem(a.L);
    dim3 grid(a.nchunks, a.nouter);
    cudaError_t e;
    if (dir < 0) {
        if ((e = set_smem(spass_kernel<-1>, sm)) != cudaSuccess) return e;
        spass_kernel<-1><<<grid, NT, sm, st>>>(a);
    } else {
        if ((e = set_smem(spass_kernel<1>, sm)) != cudaSuccess) return e;
        spass_kernel<1><<<grid, NT, sm, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_xupdate(const XUpdArgs& a, cudaStream_t st) {
    cudaError_t fe;
    if (!a.generic && fast_paths_enabled() && fast_xupdate(a, st, &fe)) return fe;
    const size_t sm = xupdate_smem(a.L);
    cudaError_t e;
    if ((e = set_smem(xupdate_kernel, sm)) != cudaSuccess) return e;
    xupdate_kernel<<<dim3(a.nchunks, a.ny), NT, sm, st>>>(a);
    return cudaGetLastError();
}

int xenergy_grid(const XEnergyArgs& a) { return a.nchunks * a.ny; }

cudaError_t launch_xenergy(const XEnergyArgs& a, cudaStream_t st) {
    const size_t sm = xupdate_smem(a.L);
    cudaError_t e;
    if ((e = set_smem(xenergy_kernel, sm)) != cudaSuccess) return e;
    xenergy_kernel<<<dim3(a.nchunks, a.ny), NT, sm, st>>>(a);
    return cudaGetLastError();
}

int zpass_grid(const ZPassArgs& a) {
    return (int)((a.nrows + a.rows_per_cta - 1) / a.rows_per_cta);
}

cudaError_t launch_zpass(const ZPassArgs& a, int mode, cudaStream_t st, int* grid_used) {
    cudaError_t fe;
    if ((mode == Z_STEP || mode == Z_ADJ) && !a.generic && fast_paths_enabled() &&
        fast_zstep(a, st, &fe, grid_used, mode == Z_ADJ))
        return fe;
    if ((mode == Z_R2C || mode == Z_C2R) && a.fast_ok && !a.generic && fast_paths_enabled() &&
        fast_zconv(a, mode == Z_R2C ? -1 : 1, st, &fe, grid_used))
        return fe;
    const size_t sm = zpass_smem(a.M, a.PZ, a.rows_per_cta);
    const int grid = zpass_grid(a);
    if (grid_used) *grid_used = grid;
    cudaError_t e = cudaSuccess;
    switch (mode) {
        case Z_STEP:
            if ((e = set_smem(zpass_kernel<Z_STEP>, sm)) != cudaSuccess) return e;
            zpass_kernel<Z_STEP><<<grid, NT, sm, st>>>(a);
            break;
        case Z_ADJ:
            if ((e = set_smem(zpass_kernel<Z_ADJ>, sm)) != cudaSuccess) return e;
            zpass_kernel<Z_ADJ><<<grid, NT, sm, st>>>(a);
            break;
        case Z_R2C:
            if ((e = set_smem(zpass_kernel<Z_R2C>, sm)) != cudaSuccess) return e;
            zpass_kernel<Z_R2C><<<grid, NT, sm, st>>>(a);
            break;
        case Z_C2R:
            if ((e = set_smem(zpass_kernel<Z_C2R>, sm)) != cudaSuccess) return e;
            zpass_kernel<Z_C2R><<<grid, NT, sm, st>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_sum_field(const float* c, long long nrows, int rowlen, long long pitch,
                             double* partials, int nblocks, cudaStream_t st) {
    if (rowlen % 4 == 0 && pitch % 4 == 0 && ((uintptr_t)c & 15) == 0)
        sum_rows_vec_kernel<<<nblocks, NT, 0, st>>>(c, nrows, rowlen, pitch, partials);
    else
        sum_rows_kernel<<<nblocks, NT, 0, st>>>(c, nrows, rowlen, pitch, partials);
    return cudaGetLastError();
}

static int vm_grid(int nx, int ny) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const long long nrows = (long long)nx * ny;
    return (int)std::min<long long>(nrows, 8LL * sms);
}

cudaError_t launch_vm_mu(const float* c, float* mu, int nx, int ny, int nz, float kappa_h2, cudaStream_t st) {
    vm_mu_kernel<<<vm_grid(nx, ny), 256, 0, st>>>(c, mu, nx, ny, nz, kappa_h2);
    return cudaGetLastError();
}

bool vm_fd_fused_ok(int nx, int ny, int nz) { return ny % VM_TY == 0 && nz % VM_TZ == 0 && nx >= 8; }

cudaError_t launch_vm_fd(const float* c, float* rhs, int nx, int ny, int nz, float kappa_h2, float M0, float inv_h2,
                         cudaStream_t st) {
    if (!vm_fd_fused_ok(nx, ny, nz)) return cudaErrorInvalidValue;
    constexpr size_t smem = sizeof(float) * (VM_CS * VM_CP + 8 * VM_MP);  // 47,232 bytes
    vm_fd_kernel<<<dim3(ny / VM_TY, nz / VM_TZ, (nx + VM_XC - 1) / VM_XC), VM_NT, smem, st>>>(c, rhs, nx, ny, nz,
                                                                                           kappa_h2, M0, inv_h2);
    return cudaGetLastError();
}

cudaError_t launch_vm_rhs(const float* c, const float* mu, float* rhs, int nx, int ny, int nz, float M0,
                          float inv_h2, cudaStream_t st) {
    vm_rhs_kernel<<<vm_grid(nx, ny), 256, 0, st>>>(c, mu, rhs, nx, ny, nz, M0, inv_h2);
    return cudaGetLastError();
}

cudaError_t launch_vm_energy(const float* c, int nx, int ny, int nz, double kappa_2h2, double* partials, int nparts,
                             cudaStream_t st) {
    const int grid = std::min(vm_grid(nx, ny), nparts);
    vm_energy_kernel<<<grid, 256, 0, st>>>(c, nx, ny, nz, kappa_2h2, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return grid > 0 ? cudaSuccess : cudaErrorInvalidValue;
}

int vm_energy_grid(int nx, int ny, int nparts) { return std::min(vm_grid(nx, ny), nparts); }

cudaError_t launch_ac_mean(const double* gsum, int n, double* cbar, double dtL, double invV, cudaStream_t st) {
    ac_mean_kernel<<<1, 1024, 0, st>>>(gsum, n, cbar, dtL, invV);
    return cudaGetLastError();
}

cudaError_t launch_remove_k0(float2* line, int n, long long stride, cudaStream_t st) {
    remove_k0_kernel<<<1, 1024, 0, st>>>(line, n, stride);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partials, int n, double* out, double scale,
                                   cudaStream_t st) {
    reduce_partials_kernel<<<1, 1024, 0, st>>>(partials, n, out, scale);
    return cudaGetLastError();
}

cudaError_t launch_cadd(const float2* a, const float2* b, float2* out, long long n,
                        cudaStream_t st) {
    cadd_kernel<<<SUM_BLOCKS, NT, 0, st>>>(a, b, out, n);
    return cudaGetLastError();
}

}  // namespace evx
