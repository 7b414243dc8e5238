// Discrete adjoint of the semi-implicit spectral Cahn-Hilliard scheme
// (gradients with respect to the initial field, kappa and M), with
// checkpoint-every-k recomputation.
//
// The scheme (Appendix "Semi-implicit timestepping", S = -M kappa |k|^4) is
//   c_{n+1} = A c_n + B g(c_n),  g(c) = c^3 - c,
// A, B the real symmetric convolutions with symbols a = 1/D,
// b = -dt M |k|^2 / D, D = 1 + dt M kappa |k|^4. Its adjoint is
//   lambda_n = A lambda_{n+1} + g'(c_n) (B lambda_{n+1}),  g'(c) = 3 c^2 - 1,
// and, since d/dkappa (a c_hat_n + b g_hat_n) = -(dt M |k|^4 / D) c_hat_{n+1} and
// d/dM (a c_hat_n + b g_hat_n) = -(dt kappa |k|^4 / D) c_hat_{n+1} - (dt |k|^2 / D) g_hat_n,
//   dL/dkappa = sum_n (1/V) sum_k Re[conj(lambda_hat_{n+1}) (-(dt M k^4/D) c_hat_{n+1})]
//   dL/dM     = sum_n (1/V) sum_k Re[conj(lambda_hat_{n+1}) (-(dt kappa k^4/D) c_hat_{n+1}
//                                                            - (dt k^2/D) g_hat_n)].
//
// The adjoint state lives in the same "x-real, y/z-spectral" form as the
// forward state (F_x Lambda = lambda_hat). One adjoint step is
//   x pass   Lambda_{n+1}, S_{n+1}, G_n -> P = B_x(a lambda_hat)/nx, T = B_x(b lambda_hat)/nx
//            (+ FP64 partial sums of the two parameter gradients)
//   y pass inverse   T -> W
//   z pass           W -> F_z[ g'(c_n) * C2R_z(W)/(ny nz) ]
//   y pass forward   W -> W
//   Lambda_n = P + W
// The forward states c_n (real), G_n = F_y F_z g(c_n) and S_{n+1} of one
// segment are recomputed from the segment's checkpoint before its adjoint
// steps run.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "evx_grid_impl.h"

using namespace evx;

namespace evx {

__device__ __forceinline__ double block_sum_d(double v, double* ws) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (NT / 32) ? ws[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

__device__ __forceinline__ void load_cols(float2* tile, int c0, const float2* g, long long base,
                                          long long rs, int L, int col0, int ncols, long long nbuf) {
    for (int e = threadIdx.x; e < L * SP; e += NT) {
        const int i = e / SP, p = e % SP;
        const long long idx = base + i * rs + p;
        tile[i * (2 * SP) + c0 + p] = (col0 + p < ncols && EVX_IN(idx, nbuf)) ? g[idx] : make_float2(0.f, 0.f);
    }
}

__device__ __forceinline__ void store_cols(float2* g, const float2* tile, int c0, long long base,
                                           long long rs, int L, int col0, int ncols, long long nbuf) {
    for (int e = threadIdx.x; e < L * SP; e += NT) {
        const int i = e / SP, p = e % SP;
        const long long idx = base + i * rs + p;
        if (col0 + p < ncols && EVX_IN(idx, nbuf)) g[idx] = tile[i * (2 * SP) + c0 + p];
    }
}

template <int DIR>
__device__ __forceinline__ void fft_cols2(float2* tile, int L, const Plan& plan, const float2* tws) {
    const int g = max(1, min(SP, TILE_CAP / L));
    for (int p0 = 0; p0 < SP; p0 += g)
        fft_tile<DIR, true>(Tile{tile + p0, L, min(g, SP - p0), 2 * SP, 1}, plan, tws);
}

__global__ void __launch_bounds__(NT, 1) xadj_kernel(XAdjArgs a) {
    extern __shared__ float2 smem[];
    __shared__ double ws[NT / 32];
    const int L = a.L;
    float2* tile = smem;               // [L][2 SP]: lambda_hat in [0, SP), work in [SP, 2 SP)
    float2* tws = smem + L * 2 * SP;
    for (int i = threadIdx.x; i < L; i += NT) tws[i] = a.tw[i];
    const int chunk = blockIdx.x, ky = blockIdx.y;
    const int col0 = chunk * SP;
    const long long base = split_off(ky, a.YB, a.os, a.os2) + col0;
    const long long nbuf = (long long)(a.ny / a.YB) * a.os2;  // complex elements of each field
    load_cols(tile, 0, a.Lam, base, a.rs, L, col0, a.ncols, nbuf);
    load_cols(tile, SP, a.Sn1, base, a.rs, L, col0, a.ncols, nbuf);
    __syncthreads();
    fft_cols2<-1>(tile, L, a.plan, tws);
    fft_cols2<-1>(tile + SP, L, a.plan, tws);
    const float k2y = a.k2y[ky];
    double acc_k = 0.0, acc_m = 0.0;
    for (int e = threadIdx.x; e < L * SP; e += NT) {
        const int i = e / SP, p = e % SP;
        const int kz = col0 + p;
        if (kz < a.ncols) {
            const float k2 = a.k2x[i] + k2y + a.k2z[kz];
            const double k4 = (double)k2 * k2;
            const double D = 1.0 + (double)a.dtMk * k4;
            const float2 lh = tile[i * (2 * SP) + p], ch = tile[i * (2 * SP) + SP + p];
            const double re = (double)lh.x * ch.x + (double)lh.y * ch.y;
            const double w = (kz == 0 || kz == a.M) ? 1.0 : 2.0;
            acc_k += w * re * (-(double)a.dtM * k4 / D);
            acc_m += w * re * (-(double)a.dtk * k4 / D);
        }
    }
    __syncthreads();
    load_cols(tile, SP, a.Gn, base, a.rs, L, col0, a.ncols, nbuf);
    __syncthreads();
    fft_cols2<-1>(tile + SP, L, a.plan, tws);
    for (int e = threadIdx.x; e < L * SP; e += NT) {
        const int i = e / SP, p = e % SP;
        const int kz = col0 + p;
        if (kz < a.ncols) {
            const float k2 = a.k2x[i] + k2y + a.k2z[kz];
            const float Df = fmaf(a.dtMk, k2 * k2, 1.f);
            const float2 lh = tile[i * (2 * SP) + p], gh = tile[i * (2 * SP) + SP + p];
            const double re = (double)lh.x * gh.x + (double)lh.y * gh.y;
            const double w = (kz == 0 || kz == a.M) ? 1.0 : 2.0;
            acc_m += w * re * (-(double)a.dt * k2 / (1.0 + (double)a.dtMk * (double)k2 * k2));
            const float av = a.invL / Df;
            const float bv = -a.dtM * k2 * av;
            tile[i * (2 * SP) + p] = make_float2(av * lh.x, av * lh.y);
            tile[i * (2 * SP) + SP + p] = make_float2(bv * lh.x, bv * lh.y);
        }
    }
    __syncthreads();
    fft_cols2<1>(tile, L, a.plan, tws);
    fft_cols2<1>(tile + SP, L, a.plan, tws);
    store_cols(a.P, tile, 0, base, a.rs, L, col0, a.ncols, nbuf);
    store_cols(a.T, tile, SP, base, a.rs, L, col0, a.ncols, nbuf);
    const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    const long long nblk = (long long)gridDim.x * gridDim.y;
    acc_k = block_sum_d(acc_k, ws);
    if (threadIdx.x == 0) a.partials[blk] = acc_k;
    acc_m = block_sum_d(acc_m, ws);
    if (threadIdx.x == 0) a.partials[nblk + blk] = acc_m;
}

// out[0] += scale * sum(partials[0..n)), deterministic order
__global__ void __launch_bounds__(1024) accum_partials_kernel(const double* partials, int n,
                                                               double* out, double scale) {
    __shared__ double ws[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) acc += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = ws[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) *out += acc * scale;
    }
}

int bounds_line_adjoint(bool clear) {
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

}  // namespace evx

struct AdjStore {
    int K = 0;          // checkpoint interval the store was sized for
    int nseg = 0;       // checkpoints allocated
    std::vector<float2*> ck;   // checkpoints of S at segment starts
    std::vector<float*> cs;    // c_j (real) for j < K
    std::vector<float2*> G;    // G_j for j < K
    std::vector<float2*> Sn;   // S_{j+1} for j < K
    float2* Lam = nullptr;
    float2* P = nullptr;
    float2* seg0 = nullptr;    // start state of the segment being replayed (the captured graph's input)
    double* part = nullptr;
    double* d_acc = nullptr;   // [0] dL/dkappa, [1] dL/dM
    size_t bytes = 0;
};

namespace evxrt {

void adjoint_free(evx_grid* g) {
    AdjStore* s = g->adj;
    if (!s) return;
    for (auto p : s->ck) cudaFree(p);
    for (auto p : s->cs) cudaFree(p);
    for (auto p : s->G) cudaFree(p);
    for (auto p : s->Sn) cudaFree(p);
    if (s->Lam) cudaFree(s->Lam);
    if (s->P) cudaFree(s->P);
    if (s->seg0) cudaFree(s->seg0);
    if (s->part) cudaFree(s->part);
    if (s->d_acc) cudaFree(s->d_acc);
    g->bytes -= s->bytes;
    delete s;
    g->adj = nullptr;
}

}  // namespace evxrt

using namespace evxrt;

#define CKA(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            std::string m_ = std::string(#call) + " failed: " + cudaGetErrorString(e_);   \
            return set_error(g, EVX_ERR_CUDA, m_.c_str());                                \
        }                                                                                 \
    } while (0)

static evx_status adj_alloc(evx_grid* g, int K, int nseg) {
    if (g->adj && g->adj->K >= K && g->adj->nseg >= nseg) return EVX_OK;
    adjoint_free(g);
    AdjStore* s = new AdjStore();
    g->adj = s;
    s->K = K;
    s->nseg = nseg;
    const size_t fspec = (size_t)g->nx * g->ny * g->Zp * sizeof(float2);
    const size_t freal = (size_t)g->nx * g->ny * g->nz * sizeof(float);
    const int xg = (g->Zp / SP) * g->ny;
    begin_alloc_call(g);
    auto get = [&](void** p, size_t b) -> bool {
        if (!device_alloc(g, p, b)) return false;
        s->bytes += b;
        return true;
    };
    bool ok = true;
    s->ck.assign(nseg, nullptr);
    s->cs.assign(K, nullptr);
    s->G.assign(K, nullptr);
    s->Sn.assign(K, nullptr);
    for (int i = 0; i < nseg && ok; ++i) ok = get((void**)&s->ck[i], fspec);
    for (int i = 0; i < K && ok; ++i)
        ok = get((void**)&s->cs[i], freal) && get((void**)&s->G[i], fspec) &&
             get((void**)&s->Sn[i], fspec);
    ok = ok && get((void**)&s->Lam, fspec) && get((void**)&s->P, fspec) && get((void**)&s->seg0, fspec) &&
         get((void**)&s->part, sizeof(double) * 2 * xg) && get((void**)&s->d_acc, 2 * sizeof(double));
    g->bytes += s->bytes;
    if (!ok) {
        adjoint_free(g);
        return set_error(g, EVX_ERR_OOM, "adjoint store allocation failed (reduce ckpt_every)");
    }
    return EVX_OK;
}

// one forward step S_in -> S_out, keeping c (real rows) and G = F_y F_z g
static evx_status fwd_step_store(evx_grid* g, const float2* S_in, float* c_out, float2* G_out,
                                 float2* S_out, cudaStream_t st) {
    CKA(launch_spass(y_args(g, S_in, g->W), +1, st));
    ZPassArgs z = z_args(g);
    z.in = g->W;
    z.out = g->W;
    z.cbar = g->d_scal;
    z.rout = c_out;
    z.rpitch = g->nz;
    CKA(launch_zpass(z, Z_STEP, st));
    CKA(launch_spass(y_args(g, g->W, G_out), -1, st));
    CKA(launch_xupdate(x_args(g, G_out, (float2*)S_in, S_out, g->p.dt, g->p.M, g->p.kappa), st));
    return EVX_OK;
}

extern "C" evx_status evx_ch_adjoint(evx_grid* g, const float* d_c0, int n_steps, int ckpt_every,
                                     const float* d_dLdcN, float* d_dLdc0, double* dLdkappa,
                                     double* dLdM) {
    if (!g || !d_c0 || !d_dLdcN || !d_dLdc0) return set_error(g, EVX_ERR_ARG, "NULL argument");
    nvtxRangePushA("evx_ch_adjoint");
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop_;
    if (g->model != EVX_MODEL_CH)
        return set_error(g, EVX_ERR_STATE, "the adjoint is implemented for the Cahn-Hilliard model only");
    if (n_steps < 0 || ckpt_every < 1) return set_error(g, EVX_ERR_ARG, "bad n_steps / ckpt_every");
    if ((((uintptr_t)d_c0) | ((uintptr_t)d_dLdcN) | ((uintptr_t)d_dLdc0)) & 7u)
        return set_error(g, EVX_ERR_ARG, "field pointers must be 8-byte aligned");
    const int K = std::min(ckpt_every, std::max(n_steps, 1));
    const int nseg = (n_steps + K - 1) / K;
    evx_status s = adj_alloc(g, K, std::max(nseg, 1));
    if (s != EVX_OK) return s;
    AdjStore* A = g->adj;
    cudaStream_t st = g->st;
    s = evx_set_field(g, d_c0);
    if (s != EVX_OK) return s;
    const size_t fspec = (size_t)g->nx * g->ny * g->Zp * sizeof(float2);
    // forward sweep, checkpoint S at every segment start
    for (int seg = 0; seg < nseg; ++seg) {
        CKA(cudaMemcpyAsync(A->ck[seg], g->S, fspec, cudaMemcpyDeviceToDevice, st));
        const int n = std::min(K, n_steps - seg * K);
        s = evx_ch_step(g, n);
        if (s != EVX_OK) return s;
    }
    // Lambda_N = F_y F_z dL/dc_N (the k = 0 mode is kept: lambda has a mean)
    {
        ZPassArgs z = z_args(g);
        z.rin = d_dLdcN;
        z.rpitch = g->nz;
        z.map_rows = 1;
        z.out = g->W;
        CKA(launch_zpass(z, Z_R2C, st));
        CKA(launch_spass(y_args(g, g->W, A->Lam), -1, st));
    }
    CKA(cudaMemsetAsync(A->d_acc, 0, 2 * sizeof(double), st));
    const double V = (double)g->nx * g->ny * g->nz;
    XAdjArgs xa{};
    xa.L = g->nx;
    xa.rs = (long long)g->YB * g->Zp;
    xa.os = g->Zp;
    xa.YB = g->YB;
    xa.os2 = (long long)g->nx * g->YB * g->Zp;
    xa.ny = g->ny;
    xa.ncols = g->M + 1;
    xa.nchunks = g->Zp / SP;
    xa.M = g->M;
    xa.plan = g->px;
    xa.tw = g->twx;
    xa.k2x = g->k2x;
    xa.k2y = g->k2y;
    xa.k2z = g->k2z;
    xa.dt = (float)g->p.dt;
    xa.dtM = (float)(g->p.dt * g->p.M);
    xa.dtMk = (float)(g->p.dt * g->p.M * g->p.kappa);
    xa.dtk = (float)(g->p.dt * g->p.kappa);
    xa.invL = (float)(1.0 / g->nx);
    xa.partials = A->part;
    const int xg = xa.nchunks * xa.ny;
    const size_t xsm = xupdate_smem(g->nx);
    if (xsm > 48 * 1024)
        CKA(cudaFuncSetAttribute(xadj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm));
    const long long nspec = (long long)g->nx * g->ny * g->Zp;
    // one segment from S_start: recompute its n forward states, then its n adjoint steps
    auto segment = [&](const float2* S_start, int n, cudaStream_t sst) -> evx_status {
        for (int j = 0; j < n; ++j) {
            const float2* S_in = j == 0 ? S_start : A->Sn[j - 1];
            evx_status r = fwd_step_store(g, S_in, A->cs[j], A->G[j], A->Sn[j], sst);
            if (r != EVX_OK) return r;
        }
        for (int j = n - 1; j >= 0; --j) {
            XAdjArgs x = xa;
            x.Lam = A->Lam;
            x.Sn1 = A->Sn[j];
            x.Gn = A->G[j];
            x.P = A->P;
            x.T = g->W;
            cudaError_t fe = cudaSuccess;
            if (!fast_xadj(x, sst, &fe)) {
                xadj_kernel<<<dim3(x.nchunks, x.ny), NT, xsm, sst>>>(x);
                fe = cudaGetLastError();
            }
            CKA(fe);
            accum_partials_kernel<<<1, 1024, 0, sst>>>(A->part, xg, A->d_acc + 0, 1.0 / V);
            accum_partials_kernel<<<1, 1024, 0, sst>>>(A->part + xg, xg, A->d_acc + 1, 1.0 / V);
            CKA(cudaGetLastError());
            CKA(launch_spass(y_args(g, g->W, g->W), +1, sst));
            ZPassArgs z = z_args(g);
            z.in = g->W;
            z.out = g->W;
            z.cn = A->cs[j];
            z.cnpitch = g->nz;
            CKA(launch_zpass(z, Z_ADJ, sst));
            CKA(launch_spass(y_args(g, g->W, g->W), -1, sst));
            CKA(launch_cadd(A->P, g->W, A->Lam, nspec, sst));
        }
        return EVX_OK;
    };
    // full segments replay one captured graph (about 11 launches per step) whose
    // input is the seg0 buffer; a shorter last segment runs eagerly
    cudaGraphExec_t gexec = nullptr;
    if (n_steps >= K && nseg > (n_steps % K ? 1 : 0)) {
        cudaGraph_t graph = nullptr;
        CKA(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
        evx_status r = segment(A->seg0, K, g->cap);
        cudaError_t e2 = cudaStreamEndCapture(g->cap, &graph);
        if (r != EVX_OK || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (r != EVX_OK) return r;
            return set_error(g, EVX_ERR_CUDA, "adjoint segment capture failed");
        }
        cudaError_t e3 = cudaGraphInstantiate(&gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) return set_error(g, EVX_ERR_CUDA, "adjoint segment graph instantiation failed");
    }
    struct ExecGuard {
        cudaGraphExec_t* e;
        ~ExecGuard() {
            if (*e) cudaGraphExecDestroy(*e);
        }
    } eg_{&gexec};
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int n0 = seg * K;
        const int n = std::min(K, n_steps - n0);
        if (n == K && gexec) {
            CKA(cudaMemcpyAsync(A->seg0, A->ck[seg], fspec, cudaMemcpyDeviceToDevice, st));
            CKA(cudaGraphLaunch(gexec, st));
        } else {
            s = segment(A->ck[seg], n, st);
            if (s != EVX_OK) return s;
        }
    }
    // dL/dc_0 = lambda_0 in real space
    {
        CKA(launch_spass(y_args(g, A->Lam, g->W), +1, st));
        ZPassArgs z = z_args(g);
        z.in = g->W;
        z.rout = d_dLdc0;
        z.rpitch = g->nz;
        z.map_rows = 1;
        z.cbar = nullptr;
        CKA(launch_zpass(z, Z_C2R, st));
    }
    double acc[2];
    CKA(cudaMemcpyAsync(acc, A->d_acc, sizeof acc, cudaMemcpyDeviceToHost, st));
    CKA(cudaStreamSynchronize(st));
    if (dLdkappa) *dLdkappa = acc[0];
    if (dLdM) *dLdM = acc[1];
    return EVX_OK;
}
