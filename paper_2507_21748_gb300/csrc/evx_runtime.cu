// Host runtime of the evx C-ABI (include/evx.h): grid plans, tables,
// buffers, pass sequencing, CUDA graphs and error state.
#include <cmath>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "evx_grid_impl.h"
#include "evx_tables.h"

using namespace evx;

static const int GRAPH_CHUNK = 16;

// NVTX range for the duration of a scope (a no-op unless a profiler is attached);
// the public calls and, in profiling mode, each pass of a step carry one
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
static thread_local std::string tl_err;

static evx_status fail(evx_grid* g, evx_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (g) g->err = buf;
    tl_err = buf;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(g, EVX_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

using evxrt::k2table;
using evxrt::make_plan;
using evxrt::smooth235;
using evxrt::twiddles;

static evx_status check_params(evx_grid* g, const evx_params& p) {
    if (!(p.dt >= 0) || !(p.M >= 0) || !(p.kappa >= 0) || !(p.h > 0) || !std::isfinite(p.dt) ||
        !std::isfinite(p.M) || !std::isfinite(p.kappa) || !std::isfinite(p.h))
        return fail(g, EVX_ERR_ARG, "invalid parameters dt=%g M=%g kappa=%g h=%g", p.dt, p.M,
                    p.kappa, p.h);
    return EVX_OK;
}

static void drop_graphs(evx_grid* g) {
    if (g->g1) cudaGraphExecDestroy(g->g1);
    if (g->gN) cudaGraphExecDestroy(g->gN);
    g->g1 = g->gN = nullptr;
}

namespace evxrt {
void begin_alloc_call(evx_grid* g) { g->call_allocs = 0; }

bool device_alloc(evx_grid* g, void** p, size_t bytes) {
    *p = nullptr;
    const int k = ++g->call_allocs;
    if (const char* env = std::getenv("EVX_FAIL_ALLOC")) {
        const int at = std::atoi(env);
        if (at >= 1 && k >= at) return false;  // injected failure: cudaMalloc is not called
    }
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}
}  // namespace evxrt

template <typename T>
static evx_status dmalloc(evx_grid* g, T** ptr, size_t bytes) {
    if (!evxrt::device_alloc(g, (void**)ptr, bytes))
        return fail(g, EVX_ERR_OOM, "device allocation of %zu bytes failed (allocation %d of the call)", bytes,
                    g->call_allocs);
    g->bytes += bytes;
    return EVX_OK;
}

template <typename T>
static evx_status upload(evx_grid* g, T** ptr, const std::vector<T>& v) {
    evx_status s = dmalloc(g, ptr, sizeof(T) * v.size());
    if (s != EVX_OK) return s;
    CK(cudaMemcpy(*ptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return EVX_OK;
}

static evx_status upload_k2(evx_grid* g) {
    std::vector<float> kx = k2table(g->nx, g->p.h, g->nx), ky = k2table(g->ny, g->p.h, g->ny),
                       kz = k2table(g->nz, g->p.h, g->M + 1);
    CK(cudaMemcpy(g->k2x, kx.data(), sizeof(float) * kx.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(g->k2y, ky.data(), sizeof(float) * ky.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(g->k2z, kz.data(), sizeof(float) * kz.size(), cudaMemcpyHostToDevice));
    return EVX_OK;
}

// ------------------------------------------------------------ pass args
namespace evxrt {

SPassArgs y_args(const evx_grid* g, const float2* in, float2* out) {
    SPassArgs a{};
    a.in = in;
    a.out = out;
    a.L = g->ny;
    a.rs = g->Zp;
    a.os = (long long)g->YB * g->Zp;
    a.YB = g->YB;
    a.os2 = (long long)g->nx * g->YB * g->Zp;
    a.nouter = g->nx;
    a.ncols = g->M + 1;
    a.nchunks = g->Zp / SP;
    a.plan = g->py;
    a.tw = g->twy;
    return a;
}

XUpdArgs x_args(const evx_grid* g, const float2* W, float2* S, float2* S_out, double dt, double M,
                double kappa) {
    XUpdArgs a{};
    a.W = W;
    a.S = S;
    a.S_out = S_out;
    a.L = g->nx;
    a.rs = (long long)g->YB * g->Zp;
    a.os = g->Zp;
    a.YB = g->YB;
    a.os2 = (long long)g->nx * g->YB * g->Zp;
    a.ny = g->ny;
    a.ncols = g->M + 1;
    a.nchunks = g->Zp / SP;
    a.plan = g->px;
    a.tw = g->twx;
    a.k2x = g->k2x;
    a.k2y = g->k2y;
    a.k2z = g->k2z;
    a.dtM = (float)(dt * M);
    a.dtMk = (float)(dt * M * kappa);
    a.invL = (float)(1.0 / g->nx);
    a.model = g->model == EVX_MODEL_AC ? 1 : 0;
    return a;
}

ZPassArgs z_args(const evx_grid* g) {
    ZPassArgs a{};
    a.nrows = (long long)g->nx * g->ny;
    a.M = g->M;
    a.Zp = g->Zp;
    a.PZ = g->PZ;
    a.rows_per_cta = g->zrows;
    a.plan = g->pz;
    a.tw = g->twz;
    a.rtw = g->rtw;
    a.scale = (float)(1.0 / ((double)g->ny * g->nz));
    a.YB = g->YB;
    a.nxr = g->nx;
    a.nyr = g->ny;
    return a;
}

YZYArgs yzy_args(const evx_grid* g) {
    YZYArgs a{};
    a.S = g->S;
    a.W = g->W;
    a.nx = g->nx;
    a.ny = g->ny;
    a.Zp = g->Zp;
    a.YB = g->YB;
    a.os2 = (long long)g->nx * g->YB * g->Zp;
    a.ncols = g->M + 1;
    a.nchunks = g->Zp / SP;
    a.twy = g->twy;
    a.twz = g->twz;
    a.rtw = g->rtw;
    a.scale = (float)(1.0 / ((double)g->ny * g->nz));
    a.cbar = g->d_scal;
    a.ctl = g->ctl;
    a.lag = g->lag;
    return a;
}

evx_status set_error(evx_grid* g, evx_status s, const char* msg) { return fail(g, s, "%s", msg); }

}  // namespace evxrt
using namespace evxrt;

// --------------------------------------------------------- step sequence
// profiling mode: record event k of a step and move the NVTX range on to the
// pass that follows it (next = nullptr after the last pass)
static void mark(cudaEvent_t* ev, int k, cudaStream_t st, const char* next) {
    if (!ev) return;
    cudaEventRecord(ev[k], st);
    if (k > 0) nvtxRangePop();
    if (next) nvtxRangePushA(next);
}

// ev: null, or 5 events recorded around the four passes
// variable mobility: c (real, in S) <- c + F^-1{ dt / (1 + dt M kappa |k|^4) F{div(M(c) grad mu)} }
// events: [FD stencils] [z R2C] [y forward] [x preconditioner + y inverse + z C2R-add]
static cudaError_t issue_vm_step(evx_grid* g, cudaStream_t st, cudaEvent_t* ev) {
    cudaError_t e;
    float* c = reinterpret_cast<float*>(g->S);
    float* mu = reinterpret_cast<float*>(g->W);
    const double ih2 = 1.0 / (g->p.h * g->p.h);
    mark(ev, 0, st, "FD stencils");
    if (vm_fd_fused_ok(g->nx, g->ny, g->nz)) {  // both stencils in one pass (mu not stored)
        if ((e = launch_vm_fd(c, g->R, g->nx, g->ny, g->nz, (float)(g->p.kappa * ih2), (float)g->p.M, (float)ih2,
                              st)) != cudaSuccess)
            return e;
    } else {
        if ((e = launch_vm_mu(c, mu, g->nx, g->ny, g->nz, (float)(g->p.kappa * ih2), st)) != cudaSuccess) return e;
        if ((e = launch_vm_rhs(c, mu, g->R, g->nx, g->ny, g->nz, (float)g->p.M, (float)ih2, st)) != cudaSuccess)
            return e;
    }
    mark(ev, 1, st, "z R2C");
    ZPassArgs z = z_args(g);
    z.rin = g->R;
    z.rpitch = g->nz;
    z.map_rows = 1;
    z.out = g->W;
    z.fast_ok = 1;
    if ((e = launch_zpass(z, Z_R2C, st)) != cudaSuccess) return e;
    mark(ev, 2, st, "y forward");
    if ((e = launch_spass(y_args(g, g->W, g->W), -1, st)) != cudaSuccess) return e;
    mark(ev, 3, st, "x preconditioner, y inverse, z C2R-add");
    XUpdArgs xa = x_args(g, g->W, g->W, g->W, g->p.dt, g->p.M, g->p.kappa);
    xa.model = 2;
    xa.dtM = (float)g->p.dt;  // preconditioner numerator
    if ((e = launch_xupdate(xa, st)) != cudaSuccess) return e;
    if ((e = launch_spass(y_args(g, g->W, g->W), +1, st)) != cudaSuccess) return e;
    ZPassArgs z2 = z_args(g);
    z2.in = g->W;
    z2.rout = c;
    z2.rpitch = g->nz;
    z2.map_rows = 1;
    z2.accumulate = 1;
    z2.fast_ok = 1;
    if ((e = launch_zpass(z2, Z_C2R, st)) != cudaSuccess) return e;
    mark(ev, 4, st, nullptr);
    return cudaSuccess;
}

static cudaError_t issue_step(evx_grid* g, cudaStream_t st, cudaEvent_t* ev) {
    if (g->model == EVX_MODEL_VM) return issue_vm_step(g, st, ev);
    cudaError_t e;
    mark(ev, 0, st, g->fused ? "fused y-z-y pass" : "y inverse");
    if (g->fused) {  // y inverse + z step + y forward in one pass (its time is reported as pass 1)
        YZYArgs y = yzy_args(g);
        const bool ac = g->model == EVX_MODEL_AC;
        if (ac) y.gsum = g->d_part;
        int grid = 0;
        if ((e = launch_fused_yzy(y, st, &grid)) != cudaSuccess) return e;
        if (ac) {
            const double V = (double)g->nx * g->ny * g->nz;
            if (grid <= 0 || grid > g->npart) return cudaErrorInvalidValue;
            if ((e = launch_ac_mean(g->d_part, grid, g->d_scal, g->p.dt * g->p.M, 1.0 / V, st)) != cudaSuccess)
                return e;
        }
        if (ev) {
            mark(ev, 1, st, "(in the fused pass)");
            mark(ev, 2, st, "(in the fused pass)");
            mark(ev, 3, st, "x pass + update");
        }
        if ((e = launch_xupdate(x_args(g, g->W, g->S, g->S, g->p.dt, g->p.M, g->p.kappa), st)) != cudaSuccess)
            return e;
        mark(ev, 4, st, nullptr);
        return cudaSuccess;
    }
    if ((e = launch_spass(y_args(g, g->S, g->W), +1, st)) != cudaSuccess) return e;
    mark(ev, 1, st, "z C2R, c^3 - c, R2C");
    ZPassArgs z = z_args(g);
    z.in = g->W;
    z.out = g->W;
    z.cbar = g->d_scal;
    const bool ac = g->model == EVX_MODEL_AC;
    if (ac) z.gsum = g->d_part;  // Allen-Cahn: the mean moves by -dt L mean(g(c))
    int zgrid = 0;
    if ((e = launch_zpass(z, Z_STEP, st, &zgrid)) != cudaSuccess) return e;
    if (ac) {
        const double V = (double)g->nx * g->ny * g->nz;
        if (zgrid <= 0 || zgrid > g->npart) return cudaErrorInvalidValue;
        if ((e = launch_ac_mean(g->d_part, zgrid, g->d_scal, g->p.dt * g->p.M, 1.0 / V, st)) != cudaSuccess)
            return e;
    }
    mark(ev, 2, st, "y forward");
    if ((e = launch_spass(y_args(g, g->W, g->W), -1, st)) != cudaSuccess) return e;
    mark(ev, 3, st, "x pass + update");
    if ((e = launch_xupdate(x_args(g, g->W, g->S, g->S, g->p.dt, g->p.M, g->p.kappa), st)) !=
        cudaSuccess)
        return e;
    mark(ev, 4, st, nullptr);
    return cudaSuccess;
}

// add the recorded event intervals to the per-pass totals (synchronises)
static evx_status drain_events(evx_grid* g) {
    if (g->ev_used == 0) return EVX_OK;
    CK(cudaEventSynchronize(g->evpool[g->ev_used - 1]));
    for (int s = 0; s < g->ev_used; s += 5) {
        float ms[4];
        for (int k = 0; k < 4; ++k)
            CK(cudaEventElapsedTime(&ms[k], g->evpool[s + k], g->evpool[s + k + 1]));
        // event order: y inverse, z, y forward, x + update  ->  pass ids 1, 2, 3, 0
        g->pass_ms[1] += ms[0];
        g->pass_ms[2] += ms[1];
        g->pass_ms[3] += ms[2];
        g->pass_ms[0] += ms[3];
        for (int k = 0; k < 4; ++k) g->pass_cnt[k] += 1;
    }
    g->ev_used = 0;
    return EVX_OK;
}

// after a synchronisation: report a bounded wait that gave up in a fast kernel
static evx_status check_timeouts(evx_grid* g) {
    int f = 0;
    if (fast_timeout_flag(&f, true) && f)
        return fail(g, EVX_ERR_CUDA, "a bounded TMA wait timed out in a fast kernel; results are invalid");
    if (fused_timeout_flag(&f, true) && f)
        return fail(g, EVX_ERR_CUDA, "a bounded wait timed out in the fused y-z-y pass; results are invalid");
    return EVX_OK;
}

static evx_status build_graph(evx_grid* g, int nsteps, cudaGraphExec_t* out) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nsteps && e == cudaSuccess; ++i) e = issue_step(g, g->cap, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(g->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(g, EVX_ERR_CUDA, "graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(g, EVX_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return EVX_OK;
}

// ================================================================ C-ABI
extern "C" {

const char* evx_last_error(const evx_grid* g) { return g ? g->err.c_str() : tl_err.c_str(); }

evx_status evx_grid_destroy(evx_grid* g);

evx_status evx_grid_create(int nx, int ny, int nz, evx_params p, void* cuda_stream, evx_grid** out) {
    evx_grid* g = nullptr;
    if (!out) return fail(g, EVX_ERR_ARG, "out is NULL");
    *out = nullptr;
    const int dims[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        const int n = dims[d];
        if (n < 8 || n > 1024 || (n & 1) || !smooth235(n))
            return fail(g, EVX_ERR_SIZE,
                        "grid size %d x %d x %d unsupported: each edge must be even, 8..1024, "
                        "with prime factors 2, 3, 5 only",
                        nx, ny, nz);
    }
    if (check_params(nullptr, p) != EVX_OK) return EVX_ERR_ARG;
    g = new evx_grid();
    evxrt::begin_alloc_call(g);
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->M = nz / 2;
    g->YB = choose_yblock(ny, fast_paths_enabled());
    g->Zp = ((g->M + 1 + SP - 1) / SP) * SP;
    g->PZ = (g->M + 2) & ~1;
    g->zrows = TILE_CAP / g->PZ;
    if (g->zrows < 1) g->zrows = 1;
    g->p = p;
    g->st = (cudaStream_t)cuda_stream;
    g->px = make_plan(nx);
    g->py = make_plan(ny);
    g->pz = make_plan(g->M);
    evx_status s;
    const size_t nspec = (size_t)nx * ny * g->Zp;
#define TRY(x)                       \
    do {                             \
        s = (x);                     \
        if (s != EVX_OK) goto bad;   \
    } while (0)
    {
        TRY(dmalloc(g, &g->S, nspec * sizeof(float2)));
        TRY(dmalloc(g, &g->W, nspec * sizeof(float2)));
        TRY(dmalloc(g, &g->d_scal, 8 * sizeof(double)));
        ZPassArgs z = z_args(g);
        const int zg = zpass_grid(z);
        const int xg = (g->Zp / SP) * ny;
        g->npart = std::max(std::max(zg, xg), SUM_BLOCKS);
        if (fused_yzy_enabled() && fused_yzy_shape(ny, g->M, g->YB)) {
            g->fused = true;
            if (const char* lg = std::getenv("EVX_FUSE_LAG")) g->lag = std::min(16, std::max(1, std::atoi(lg)));
            TRY(dmalloc(g, &g->ctl, sizeof(int) * fused_ctl_ints(nx)));
            g->npart = std::max(g->npart, fused_yzy_grid(yzy_args(g)));
        }
        TRY(dmalloc(g, &g->d_part, (size_t)g->npart * sizeof(double)));
        TRY(upload(g, &g->twx, twiddles(nx)));
        TRY(upload(g, &g->twy, twiddles(ny)));
        TRY(upload(g, &g->twz, twiddles(g->M)));
        TRY(upload(g, &g->rtw, twiddles(nz, g->M + 1)));  // exp(-2 pi i k / nz), k <= M
        TRY(dmalloc(g, &g->k2x, sizeof(float) * nx));
        TRY(dmalloc(g, &g->k2y, sizeof(float) * ny));
        TRY(dmalloc(g, &g->k2z, sizeof(float) * (g->M + 1)));
        TRY(upload_k2(g));
        cudaError_t e = cudaMemset(g->d_scal, 0, 8 * sizeof(double));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            s = fail(g, EVX_ERR_CUDA, "create: %s", cudaGetErrorString(e));
            goto bad;
        }
    }
#undef TRY
    *out = g;
    return EVX_OK;
bad:
    tl_err = g->err;
    evx_grid_destroy(g);
    return s;
}

evx_status evx_grid_destroy(evx_grid* g) {
    if (!g) return EVX_OK;
    if (g->st || g->S) cudaStreamSynchronize(g->st);
    evxrt::adjoint_free(g);
    drop_graphs(g);
    for (auto ptr : {(void*)g->S, (void*)g->W, (void*)g->R, (void*)g->ctl, (void*)g->d_scal, (void*)g->d_part, (void*)g->twx,
                     (void*)g->twy, (void*)g->twz, (void*)g->rtw, (void*)g->k2x, (void*)g->k2y,
                     (void*)g->k2z})
        if (ptr) cudaFree(ptr);
    for (auto e : g->evpool) cudaEventDestroy(e);
    if (g->cap) cudaStreamDestroy(g->cap);
    delete g;
    return EVX_OK;
}

evx_status evx_set_params(evx_grid* g, evx_params p) {
    if (!g) return fail(g, EVX_ERR_ARG, "grid is NULL");
    if (check_params(g, p) != EVX_OK) return EVX_ERR_ARG;
    const bool hchg = p.h != g->p.h;
    g->p = p;
    drop_graphs(g);
    if (hchg) {
        CK(cudaStreamSynchronize(g->st));
        return upload_k2(g);
    }
    return EVX_OK;
}

evx_status evx_get_params(const evx_grid* g, evx_params* p) {
    if (!g || !p) return fail(nullptr, EVX_ERR_ARG, "NULL argument");
    *p = g->p;
    return EVX_OK;
}

evx_status evx_set_stream(evx_grid* g, void* cuda_stream) {
    if (!g) return fail(g, EVX_ERR_ARG, "grid is NULL");
    g->st = (cudaStream_t)cuda_stream;
    return EVX_OK;
}

static bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

// real rows (pitch floats apart) -> spectral state S, FP64 mean -> d_scal[0].
// map: rows are the caller's C-order field (else memory order of the spectrum)
static evx_status load_real(evx_grid* g, const float* rows, long long pitch, int map) {
    const long long nrows = (long long)g->nx * g->ny;
    const double V = (double)nrows * g->nz;
    CK(launch_sum_field(rows, nrows, g->nz, pitch, g->d_part, SUM_BLOCKS, g->st));
    CK(launch_reduce_partials(g->d_part, SUM_BLOCKS, g->d_scal + 0, 1.0 / V, g->st));
    ZPassArgs z = z_args(g);
    z.rin = rows;
    z.rpitch = pitch;
    z.map_rows = map;
    z.out = g->S;
    z.cbar = g->d_scal;  // transform c - cbar
    z.fast_ok = 1;
    CK(launch_zpass(z, Z_R2C, g->st));
    CK(launch_spass(y_args(g, g->S, g->S), -1, g->st));
    // remove the k = 0 mode (carried in FP64): the mean of the (ky = 0, kz = 0) x line
    CK(launch_remove_k0(g->S, g->nx, (long long)g->YB * g->Zp, g->st));
    g->has_field = true;
    g->steps = 0;
    return EVX_OK;
}

static size_t field_bytes(const evx_grid* g) { return sizeof(float) * (size_t)g->nx * g->ny * g->nz; }

evx_status evx_set_field(evx_grid* g, const float* d_c) {
    NvtxRange nvtx_("evx_set_field");
    if (!g || !d_c) return fail(g, EVX_ERR_ARG, "NULL argument");
    if (!aligned8(d_c)) return fail(g, EVX_ERR_ARG, "field pointer must be 8-byte aligned");
    if (g->model == EVX_MODEL_VM) {  // the variable-mobility state is the real field itself
        CK(cudaMemcpyAsync(g->S, d_c, field_bytes(g), cudaMemcpyDeviceToDevice, g->st));
        g->has_field = true;
        g->steps = 0;
        return EVX_OK;
    }
    return load_real(g, d_c, g->nz, 1);
}

// copies between a caller's C-order real field (host) and real rows staged
// in W's row slots (pitch 2 Zp floats) in the spectrum's memory row order:
// one 3D copy per y block (rows (x, yi) of block yb)
static evx_status host_rows_copy(evx_grid* g, float* host, bool to_device) {
    const int nyb = g->ny / g->YB;
    for (int yb = 0; yb < nyb; ++yb) {
        cudaMemcpy3DParms c = {};
        cudaPitchedPtr hp = make_cudaPitchedPtr(host + (size_t)yb * g->YB * g->nz, sizeof(float) * g->nz,
                                                g->nz, g->ny);
        cudaPitchedPtr dp = make_cudaPitchedPtr((float*)g->W + (size_t)yb * g->nx * g->YB * 2 * g->Zp,
                                                sizeof(float) * 2 * g->Zp, g->nz, g->YB);
        c.srcPtr = to_device ? hp : dp;
        c.dstPtr = to_device ? dp : hp;
        c.extent = make_cudaExtent(sizeof(float) * g->nz, g->YB, g->nx);
        c.kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
        CK(cudaMemcpy3DAsync(&c, g->st));
    }
    return EVX_OK;
}

evx_status evx_set_field_host(evx_grid* g, const float* h_c) {
    NvtxRange nvtx_("evx_set_field_host");
    if (!g || !h_c) return fail(g, EVX_ERR_ARG, "NULL argument");
    if (g->model == EVX_MODEL_VM) {
        CK(cudaMemcpyAsync(g->S, h_c, field_bytes(g), cudaMemcpyHostToDevice, g->st));
        CK(cudaStreamSynchronize(g->st));
        g->has_field = true;
        g->steps = 0;
        return EVX_OK;
    }
    // one contiguous copy into W's memory (the R2C reads the caller-order rows from
    // there and writes the state S), then the caller-order row map
    CK(cudaMemcpyAsync(g->W, h_c, field_bytes(g), cudaMemcpyHostToDevice, g->st));
    evx_status s = load_real(g, reinterpret_cast<const float*>(g->W), g->nz, 1);
    if (s != EVX_OK) return s;
    CK(cudaStreamSynchronize(g->st));
    return EVX_OK;
}

// state -> real rows (pitch floats apart), optional bulk-energy partials;
// map as in load_real
static evx_status store_real(evx_grid* g, float* rows, long long pitch, double* partials, int map,
                             int* grid_used = nullptr) {
    CK(launch_spass(y_args(g, g->S, g->W), +1, g->st));
    ZPassArgs z = z_args(g);
    z.in = g->W;
    z.rout = rows;
    z.rpitch = pitch;
    z.map_rows = map;
    z.cbar = g->d_scal;
    z.partials = partials;
    z.fast_ok = 1;
    int zg = zpass_grid(z);
    CK(launch_zpass(z, Z_C2R, g->st, &zg));
    if (grid_used) *grid_used = zg;
    return EVX_OK;
}

evx_status evx_get_field(evx_grid* g, float* d_out) {
    NvtxRange nvtx_("evx_get_field");
    if (!g || !d_out) return fail(g, EVX_ERR_ARG, "NULL argument");
    if (!g->has_field) return fail(g, EVX_ERR_STATE, "no field set");
    if (!aligned8(d_out)) return fail(g, EVX_ERR_ARG, "output pointer must be 8-byte aligned");
    if (g->model == EVX_MODEL_VM) {
        CK(cudaMemcpyAsync(d_out, g->S, field_bytes(g), cudaMemcpyDeviceToDevice, g->st));
        return EVX_OK;
    }
    return store_real(g, d_out, g->nz, nullptr, 1);
}

evx_status evx_get_field_host(evx_grid* g, float* h_out) {
    NvtxRange nvtx_("evx_get_field_host");
    if (!g || !h_out) return fail(g, EVX_ERR_ARG, "NULL argument");
    if (!g->has_field) return fail(g, EVX_ERR_STATE, "no field set");
    if (g->model == EVX_MODEL_VM) {
        CK(cudaMemcpyAsync(h_out, g->S, field_bytes(g), cudaMemcpyDeviceToHost, g->st));
        CK(cudaStreamSynchronize(g->st));
        return check_timeouts(g);
    }
    // pinned host memory that the device can address (page-locked and mapped, as
    // cudaHostAlloc / torch pin_memory give under unified addressing): the C2R
    // writes the caller-order rows straight into it, with no staging copy
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h_out) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer &&
        ((uintptr_t)at.devicePointer & 15) == 0) {
        evx_status s = store_real(g, (float*)at.devicePointer, g->nz, nullptr, 1);
        if (s != EVX_OK) return s;
        CK(cudaStreamSynchronize(g->st));
        return check_timeouts(g);
    }
    cudaGetLastError();  // pageable memory: the attribute query may leave an error behind
    evx_status s = store_real(g, (float*)g->W, 2LL * g->Zp, nullptr, 0);
    if (s != EVX_OK) return s;
    s = host_rows_copy(g, h_out, false);
    if (s != EVX_OK) return s;
    CK(cudaStreamSynchronize(g->st));
    return check_timeouts(g);
}

evx_status evx_set_model(evx_grid* g, int model) {
    if (!g) return fail(g, EVX_ERR_ARG, "grid is NULL");
    if (model != EVX_MODEL_CH && model != EVX_MODEL_AC && model != EVX_MODEL_VM)
        return fail(g, EVX_ERR_ARG, "unknown model %d", model);
    if (model != g->model) {
        CK(cudaStreamSynchronize(g->st));
        drop_graphs(g);
        if (model == EVX_MODEL_VM && !g->R) {
            evxrt::begin_alloc_call(g);
            evx_status s = dmalloc(g, &g->R, field_bytes(g));
            if (s != EVX_OK) return s;
        }
        // CH and AC share the spectral state; the variable-mobility state is the real field
        if (model == EVX_MODEL_VM || g->model == EVX_MODEL_VM) g->has_field = false;
        g->model = model;
    }
    return EVX_OK;
}

int evx_get_model(const evx_grid* g) { return g ? g->model : -1; }

evx_status evx_ch_step(evx_grid* g, int n_steps) {
    if (g && g->model != EVX_MODEL_CH)
        return fail(g, EVX_ERR_STATE, "evx_ch_step on a grid set to another model (use evx_step)");
    return evx_step(g, n_steps);
}

evx_status evx_step(evx_grid* g, int n_steps) {
    NvtxRange nvtx_("evx_step");
    if (!g) return fail(g, EVX_ERR_ARG, "grid is NULL");
    if (n_steps < 0) return fail(g, EVX_ERR_ARG, "n_steps < 0");
    if (!g->has_field) return fail(g, EVX_ERR_STATE, "no field set");
    if (n_steps == 0) return EVX_OK;
    g->steps += n_steps;
    if (g->prof) {
        for (int i = 0; i < n_steps; ++i) {
            if ((size_t)g->ev_used + 5 > g->evpool.size()) {
                if (g->evpool.size() >= 5 * 4096) {
                    evx_status s = drain_events(g);
                    if (s != EVX_OK) return s;
                } else {
                    for (int k = 0; k < 5; ++k) {
                        cudaEvent_t e;
                        CK(cudaEventCreate(&e));
                        g->evpool.push_back(e);
                    }
                }
            }
            {
                NvtxRange r_("step (profiled: one launch per pass)");
                CK(issue_step(g, g->st, &g->evpool[g->ev_used]));
            }
            g->ev_used += 5;
        }
        return EVX_OK;
    }
    if (!g->g1) {
        evx_status s = build_graph(g, 1, &g->g1);
        if (s != EVX_OK) return s;
    }
    if (n_steps >= GRAPH_CHUNK && !g->gN) {
        evx_status s = build_graph(g, GRAPH_CHUNK, &g->gN);
        if (s != EVX_OK) return s;
    }
    int left = n_steps;
    while (left >= GRAPH_CHUNK) {
        CK(cudaGraphLaunch(g->gN, g->st));
        left -= GRAPH_CHUNK;
    }
    while (left-- > 0) CK(cudaGraphLaunch(g->g1, g->st));
    return EVX_OK;
}

evx_status evx_ch_block(evx_grid* g, int n_steps) {
    NvtxRange nvtx_("evx_ch_block");
    if (!g) return fail(g, EVX_ERR_ARG, "grid is NULL");
    if (g->model != EVX_MODEL_CH) return fail(g, EVX_ERR_STATE, "evx_ch_block is defined for the Cahn-Hilliard model");
    if (n_steps < 1 || n_steps > 4096) return fail(g, EVX_ERR_ARG, "n_steps must be 1..4096");
    if (!g->has_field) return fail(g, EVX_ERR_STATE, "no field set");
    // y inverse, z pass forming N only, y forward, x pass with the block symbols
    // (the separate passes, also on a grid created with the fused y-z-y pass)
    CK(launch_spass(y_args(g, g->S, g->W), +1, g->st));
    ZPassArgs z = z_args(g);
    z.in = g->W;
    z.out = g->W;
    z.cbar = g->d_scal;
    z.nl_only = 1;
    CK(launch_zpass(z, Z_STEP, g->st));
    CK(launch_spass(y_args(g, g->W, g->W), -1, g->st));
    XUpdArgs xa = x_args(g, g->W, g->S, g->S, g->p.dt, g->p.M, g->p.kappa);
    xa.model = 3;
    xa.nblk = n_steps;
    xa.cbar = g->d_scal;
    CK(launch_xupdate(xa, g->st));
    g->steps += n_steps;
    return EVX_OK;
}

// variable mobility: FP64 mean of the real field -> d_scal[0]
static cudaError_t vm_sum(evx_grid* g) {
    const long long nrows = (long long)g->nx * g->ny;
    const double V = (double)nrows * g->nz;
    cudaError_t e = launch_sum_field(reinterpret_cast<const float*>(g->S), nrows, g->nz, g->nz, g->d_part,
                                     SUM_BLOCKS, g->st);
    if (e != cudaSuccess) return e;
    return launch_reduce_partials(g->d_part, SUM_BLOCKS, g->d_scal + 0, 1.0 / V, g->st);
}

evx_status evx_energy(evx_grid* g, double* E, double* mass) {
    NvtxRange nvtx_("evx_energy");
    if (!g) return fail(g, EVX_ERR_ARG, "grid is NULL");
    if (!g->has_field) return fail(g, EVX_ERR_STATE, "no field set");
    const double h3 = g->p.h * g->p.h * g->p.h;
    const double V = (double)g->nx * g->ny * g->nz;
    if (g->model == EVX_MODEL_VM) {  // FD energy of the real field, h^3 sum (...)
        const float* c = reinterpret_cast<const float*>(g->S);
        const double k2h2 = 0.5 * g->p.kappa / (g->p.h * g->p.h);
        CK(launch_vm_energy(c, g->nx, g->ny, g->nz, k2h2, g->d_part, g->npart, g->st));
        CK(launch_reduce_partials(g->d_part, vm_energy_grid(g->nx, g->ny, g->npart), g->d_scal + 1, h3, g->st));
        CK(vm_sum(g));
        double host[2];
        CK(cudaMemcpyAsync(host, g->d_scal, sizeof host, cudaMemcpyDeviceToHost, g->st));
        CK(cudaStreamSynchronize(g->st));
        if (!std::isfinite(host[1]) || !std::isfinite(host[0]))
            return fail(g, EVX_ERR_NONFINITE, "field holds NaN or Inf (energy %g, mean %g)", host[1], host[0]);
        if (E) *E = host[1];
        if (mass) *mass = h3 * V * host[0];
        return check_timeouts(g);
    }
    // bulk: h^3/4 sum (c^2-1)^2 over the real field (written into W's row slots, discarded)
    int zg = 0;
    evx_status s = store_real(g, (float*)g->W, 2LL * g->Zp, g->d_part, 0, &zg);
    if (s != EVX_OK) return s;
    CK(launch_reduce_partials(g->d_part, zg, g->d_scal + 1, 0.25 * h3, g->st));
    // gradient: h^3 (kappa/2)(1/V) sum_k |k|^2 |c_hat|^2
    XEnergyArgs xa{};
    xa.S = g->S;
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
    xa.partials = g->d_part;
    CK(launch_xenergy(xa, g->st));
    CK(launch_reduce_partials(g->d_part, xenergy_grid(xa), g->d_scal + 2,
                              0.5 * g->p.kappa * h3 / V, g->st));
    double host[3];
    CK(cudaMemcpyAsync(host, g->d_scal, sizeof host, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    s = check_timeouts(g);
    if (s != EVX_OK) return s;
    const double e = host[1] + host[2];
    if (!std::isfinite(e) || !std::isfinite(host[0]))
        return fail(g, EVX_ERR_NONFINITE, "field holds NaN or Inf (energy %g, mean %g)", e, host[0]);
    if (E) *E = e;
    if (mass) *mass = h3 * V * host[0];
    return EVX_OK;
}

evx_status evx_mean(evx_grid* g, double* cbar) {
    if (!g || !cbar) return fail(g, EVX_ERR_ARG, "NULL argument");
    if (!g->has_field) return fail(g, EVX_ERR_STATE, "no field set");
    if (g->model == EVX_MODEL_VM) CK(vm_sum(g));  // the real field's FP64 mean (not carried)
    CK(cudaMemcpyAsync(cbar, g->d_scal, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    return check_timeouts(g);
}

evx_status evx_footprint(const evx_grid* g, size_t* bytes) {
    if (!g || !bytes) return fail(nullptr, EVX_ERR_ARG, "NULL argument");
    *bytes = g->bytes;
    return EVX_OK;
}

evx_status evx_set_profiling(evx_grid* g, int on) {
    if (!g) return fail(g, EVX_ERR_ARG, "grid is NULL");
    if (!on) {
        evx_status s = drain_events(g);
        if (s != EVX_OK) return s;
    }
    g->prof = on != 0;
    return EVX_OK;
}

evx_status evx_pass_times(evx_grid* g, double* ms, long long* counts, int reset) {
    if (!g) return fail(g, EVX_ERR_ARG, "grid is NULL");
    CK(cudaStreamSynchronize(g->st));
    evx_status s = drain_events(g);
    if (s != EVX_OK) return s;
    s = check_timeouts(g);
    if (s != EVX_OK) return s;
    for (int k = 0; k < 4; ++k) {
        if (ms) ms[k] = g->pass_ms[k];
        if (counts) counts[k] = g->pass_cnt[k];
        if (reset) {
            g->pass_ms[k] = 0;
            g->pass_cnt[k] = 0;
        }
    }
    return EVX_OK;
}

evx_status evx_pass_bytes(const evx_grid* g, int pass, double* bytes) {
    if (!g || !bytes || pass < 0 || pass > 3) return fail(nullptr, EVX_ERR_ARG, "bad argument");
    // one half-spectrum field: nx * ny * (M + 1) complex64 elements
    const double F = (double)g->nx * g->ny * (g->M + 1) * sizeof(float2);
    // pass 0 reads W and S, writes S; passes 1..3 read one field and write one.
    // With the fused y-z-y pass, pass 1 is that pass (read S, write W; the
    // intermediate sweeps stay in L2) and passes 2 and 3 are empty.
    if (g->fused && g->model != EVX_MODEL_VM)
        *bytes = pass == 0 ? 3.0 * F : pass == 1 ? 2.0 * F : 0.0;
    else
        *bytes = pass == 0 ? 3.0 * F : 2.0 * F;
    return EVX_OK;
}

evx_status evx_debug_bounds(int* enabled, int* line) {
#ifdef EVX_BOUNDS_CHECK
    const int on = 1;
#else
    const int on = 0;
#endif
    if (enabled) *enabled = on;
    if (line) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return fail(nullptr, EVX_ERR_CUDA, "synchronise: %s", cudaGetErrorString(e));
        const int a = bounds_line_kernels(true), b = bounds_line_adjoint(true);
        *line = a ? a : b;
    }
    return EVX_OK;
}

evx_status evx_step_count(const evx_grid* g, long long* steps) {
    if (!g || !steps) return fail(nullptr, EVX_ERR_ARG, "NULL argument");
    *steps = g->steps;
    return EVX_OK;
}

}  // extern "C"

// ------------------------------------------------------ checkpoint / resume
// File: a fixed header, then the payload (the state buffer exactly as the grid
// holds it), little-endian as both host architectures store it.
namespace {
struct CkptHeader {
    char magic[8];              // "EVXCKPT1"
    uint32_t version, header_bytes;
    int32_t nx, ny, nz, model, YB, Zp;
    double dt, M, kappa, h;
    double cbar;                // FP64 mean (the k = 0 mode)
    int64_t steps;
    uint64_t payload_bytes, payload_fnv;
};
const char CKPT_MAGIC[8] = {'E', 'V', 'X', 'C', 'K', 'P', 'T', '1'};
constexpr size_t CKPT_CHUNK = 64u << 20;  // host staging per copy

uint64_t fnv1a(uint64_t h, const unsigned char* p, size_t n) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ULL;
    }
    return h;
}

// the state buffer and its size: the spectral state (CH, AC) or the real field (VM)
size_t state_bytes(const evx_grid* g) {
    return g->model == EVX_MODEL_VM ? sizeof(float) * (size_t)g->nx * g->ny * g->nz
                                    : sizeof(float2) * (size_t)g->nx * g->ny * g->Zp;
}
}  // namespace

extern "C" {

evx_status evx_save(evx_grid* g, const char* path) {
    NvtxRange nvtx_("evx_save");
    if (!g || !path) return fail(g, EVX_ERR_ARG, "NULL argument");
    if (!g->has_field) return fail(g, EVX_ERR_STATE, "no field set");
    CK(cudaStreamSynchronize(g->st));
    evx_status s = check_timeouts(g);
    if (s != EVX_OK) return s;
    CkptHeader hd{};
    std::memcpy(hd.magic, CKPT_MAGIC, 8);
    hd.version = 1;
    hd.header_bytes = sizeof(CkptHeader);
    hd.nx = g->nx;
    hd.ny = g->ny;
    hd.nz = g->nz;
    hd.model = g->model;
    hd.YB = g->YB;
    hd.Zp = g->Zp;
    hd.dt = g->p.dt;
    hd.M = g->p.M;
    hd.kappa = g->p.kappa;
    hd.h = g->p.h;
    hd.steps = g->steps;
    if (g->model != EVX_MODEL_VM) CK(cudaMemcpy(&hd.cbar, g->d_scal, sizeof(double), cudaMemcpyDeviceToHost));
    const size_t total = state_bytes(g);
    hd.payload_bytes = total;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(g, EVX_ERR_IO, "cannot open %s for writing", path);
    std::vector<unsigned char> buf(std::min(total, CKPT_CHUNK));
    bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1;
    uint64_t h = 0xcbf29ce484222325ULL;
    const unsigned char* src = reinterpret_cast<const unsigned char*>(g->S);
    for (size_t off = 0; ok && off < total; off += buf.size()) {
        const size_t n = std::min(buf.size(), total - off);
        if (cudaMemcpy(buf.data(), src + off, n, cudaMemcpyDeviceToHost) != cudaSuccess) {
            std::fclose(f);
            return fail(g, EVX_ERR_CUDA, "state copy failed: %s", cudaGetErrorString(cudaGetLastError()));
        }
        h = fnv1a(h, buf.data(), n);
        ok = std::fwrite(buf.data(), 1, n, f) == n;
    }
    hd.payload_fnv = h;  // the checksum goes into the header once the payload is written
    ok = ok && std::fseek(f, 0, SEEK_SET) == 0 && std::fwrite(&hd, sizeof hd, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(g, EVX_ERR_IO, "write to %s failed", path);
    return EVX_OK;
}

evx_status evx_load(evx_grid* g, const char* path) {
    NvtxRange nvtx_("evx_load");
    if (!g || !path) return fail(g, EVX_ERR_ARG, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(g, EVX_ERR_IO, "cannot open %s", path);
    CkptHeader hd{};
    if (std::fread(&hd, sizeof hd, 1, f) != 1 || std::memcmp(hd.magic, CKPT_MAGIC, 8) != 0 || hd.version != 1 ||
        hd.header_bytes != sizeof(CkptHeader)) {
        std::fclose(f);
        return fail(g, EVX_ERR_IO, "%s is not an evx checkpoint", path);
    }
    if (hd.nx != g->nx || hd.ny != g->ny || hd.nz != g->nz) {
        std::fclose(f);
        return fail(g, EVX_ERR_STATE, "checkpoint grid %d x %d x %d differs from this grid %d x %d x %d", hd.nx,
                    hd.ny, hd.nz, g->nx, g->ny, g->nz);
    }
    if (hd.model != g->model) {
        std::fclose(f);
        return fail(g, EVX_ERR_STATE, "checkpoint holds model %d, the grid is set to model %d (evx_set_model first)",
                    hd.model, g->model);
    }
    if (hd.YB != g->YB || hd.Zp != g->Zp || hd.payload_bytes != state_bytes(g)) {
        std::fclose(f);
        return fail(g, EVX_ERR_STATE, "checkpoint layout (y block %d, row pitch %d) differs from this grid's (%d, %d)",
                    hd.YB, hd.Zp, g->YB, g->Zp);
    }
    const evx_params p{hd.dt, hd.M, hd.kappa, hd.h};
    if (check_params(g, p) != EVX_OK) {
        std::fclose(f);
        return EVX_ERR_IO;
    }
    // read and verify the whole payload before the grid's state is touched
    const size_t total = hd.payload_bytes;
    std::vector<unsigned char> data(total);
    const bool rd = std::fread(data.data(), 1, total, f) == total;
    std::fclose(f);
    if (!rd) return fail(g, EVX_ERR_IO, "%s is truncated", path);
    if (fnv1a(0xcbf29ce484222325ULL, data.data(), total) != hd.payload_fnv)
        return fail(g, EVX_ERR_IO, "%s: payload checksum mismatch", path);
    evx_status s = evx_set_params(g, p);
    if (s != EVX_OK) return s;
    CK(cudaStreamSynchronize(g->st));
    CK(cudaMemcpy(g->S, data.data(), total, cudaMemcpyHostToDevice));
    if (g->model != EVX_MODEL_VM) CK(cudaMemcpy(g->d_scal, &hd.cbar, sizeof(double), cudaMemcpyHostToDevice));
    g->has_field = true;
    g->steps = hd.steps;
    return EVX_OK;
}

}  // extern "C"

