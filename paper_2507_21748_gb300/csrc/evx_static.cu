// Allocation-free variant of the Cahn-Hilliard step for callers that cannot
// call cudaMalloc (for example code that runs under a host-side memory
// budget fixed at start-up, inside another framework's allocator-free
// callbacks, or in a process whose device allocations are owned by someone
// else). Every scratch buffer the step needs - the half-spectrum state and
// work buffer, the FP64 scalars and reduction partials, the twiddle and
// wave-number tables - lives in one file-scope static device array whose size
// is fixed at compile time; the caller passes only the input and output
// fields. The path runs the mixed-radix kernels in the plain [x][y][kz]
// layout: they have no bounded waits, so nothing is left on the device for a
// later call to report.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "evx_grid_impl.h"
#include "evx_tables.h"

using namespace evx;

namespace {

// 8 MiB: enough for any valid grid of at most 64^3 voxels (two half spectra of
// at most 2 * (V/2 + 8 V/8) complex64 values plus tables and partials).
constexpr size_t STATIC_BYTES = 8u << 20;
constexpr long long STATIC_MAX_VOXELS = 64LL * 64 * 64;

__device__ __align__(256) unsigned char g_static_scratch[STATIC_BYTES];

constexpr int MAX_DEVICES = 64;
void* g_static_addr[MAX_DEVICES] = {nullptr};
std::mutex g_static_mutex;

// message readable through evx_last_error(NULL)
evx_status static_fail(evx_status s, const std::string& m) { return evxrt::set_error(nullptr, s, m.c_str()); }

// device address of the static array for the current device (host code only
// holds a stand-in for the symbol; the address must be queried per device)
evx_status static_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(EVX_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return static_fail(EVX_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_static_mutex);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return static_fail(EVX_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return EVX_OK;
}

// bump allocator over the static array (256-byte aligned pieces)
struct Carve {
    unsigned char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

}  // namespace

// pass arguments of the static path: always the mixed-radix kernels
static SPassArgs ys(const evx_grid* g, const float2* in, float2* out) {
    SPassArgs a = evxrt::y_args(g, in, out);
    a.generic = 1;
    return a;
}
static XUpdArgs xs(const evx_grid* g, const float2* W, float2* S, float2* S_out, double dt, double M, double kappa) {
    XUpdArgs a = evxrt::x_args(g, W, S, S_out, dt, M, kappa);
    a.generic = 1;
    return a;
}
static ZPassArgs zs(const evx_grid* g) {
    ZPassArgs a = evxrt::z_args(g);
    a.generic = 1;
    return a;
}

#define CKS(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return static_fail(EVX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" evx_status evx_ch_step_static(const float* d_c_in, float* d_c_out, int nx, int ny, int nz,
                                         evx_params p, int n_steps, void* cuda_stream) {
    if (!d_c_in || !d_c_out) return static_fail(EVX_ERR_ARG, "NULL field pointer");
    if ((((uintptr_t)d_c_in) | ((uintptr_t)d_c_out)) & 7u)
        return static_fail(EVX_ERR_ARG, "field pointers must be 8-byte aligned");
    if (n_steps < 0) return static_fail(EVX_ERR_ARG, "n_steps < 0");
    if (!(p.dt >= 0) || !(p.M >= 0) || !(p.kappa >= 0) || !(p.h > 0) || !std::isfinite(p.dt) ||
        !std::isfinite(p.M) || !std::isfinite(p.kappa) || !std::isfinite(p.h))
        return static_fail(EVX_ERR_ARG, "invalid parameters");
    for (int n : {nx, ny, nz})
        if (n < 8 || n > 1024 || (n & 1) || !evxrt::smooth235(n))
            return static_fail(EVX_ERR_SIZE, "each edge must be even, 8..1024, prime factors 2, 3, 5");
    const long long V = (long long)nx * ny * nz;
    if (V > STATIC_MAX_VOXELS)
        return static_fail(EVX_ERR_SIZE, "evx_ch_step_static handles at most 64^3 = 262144 voxels");

    void* addr = nullptr;
    evx_status s = static_address(&addr);
    if (s != EVX_OK) return s;

    // a grid description whose buffers all point into the static array
    evx_grid g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.M = nz / 2;
    // plain [x][y][kz] layout and the mixed-radix kernels only: they have no
    // bounded waits, so a call has no device-side timeout flag left to report
    g.YB = choose_yblock(ny, false);
    g.Zp = ((g.M + 1 + SP - 1) / SP) * SP;
    g.PZ = (g.M + 2) & ~1;
    g.zrows = std::max(1, TILE_CAP / g.PZ);
    g.p = p;
    g.st = (cudaStream_t)cuda_stream;
    g.px = evxrt::make_plan(nx);
    g.py = evxrt::make_plan(ny);
    g.pz = evxrt::make_plan(g.M);
    const size_t nspec = (size_t)nx * ny * g.Zp;
    Carve cv{reinterpret_cast<unsigned char*>(addr)};
    g.S = cv.take<float2>(nspec);
    g.W = cv.take<float2>(nspec);
    g.d_scal = cv.take<double>(8);
    {
        ZPassArgs z = evxrt::z_args(&g);
        const int zg = zpass_grid(z), xg = (g.Zp / SP) * ny;
        g.npart = std::max(std::max(zg, xg), SUM_BLOCKS);
    }
    g.d_part = cv.take<double>(g.npart);
    g.twx = cv.take<float2>(nx);
    g.twy = cv.take<float2>(ny);
    g.twz = cv.take<float2>(g.M);
    g.rtw = cv.take<float2>(g.M + 1);
    g.k2x = cv.take<float>(nx);
    g.k2y = cv.take<float>(ny);
    g.k2z = cv.take<float>(g.M + 1);
    if (cv.off > STATIC_BYTES) return static_fail(EVX_ERR_SIZE, "grid does not fit the static scratch");

    // tables (host FP64, rounded to FP32; the same functions as the grid path),
    // copied into the static array
    const std::vector<float2> tx = evxrt::twiddles(nx), ty = evxrt::twiddles(ny), tz = evxrt::twiddles(g.M),
                              r = evxrt::twiddles(nz, g.M + 1);
    const std::vector<float> kx = evxrt::k2table(nx, p.h, nx), ky = evxrt::k2table(ny, p.h, ny),
                             kz = evxrt::k2table(nz, p.h, g.M + 1);
    cudaStream_t st = g.st;
    // pageable sources: each copy has read its host buffer when the call returns
    CKS(cudaMemcpyAsync(g.twx, tx.data(), sizeof(float2) * nx, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(g.twy, ty.data(), sizeof(float2) * ny, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(g.twz, tz.data(), sizeof(float2) * g.M, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(g.rtw, r.data(), sizeof(float2) * (g.M + 1), cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(g.k2x, kx.data(), sizeof(float) * nx, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(g.k2y, ky.data(), sizeof(float) * ny, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(g.k2z, kz.data(), sizeof(float) * (g.M + 1), cudaMemcpyHostToDevice, st));
    // the array keeps the previous call's contents: clear the scalars
    CKS(cudaMemsetAsync(g.d_scal, 0, 8 * sizeof(double), st));

    // initial field -> state (FP64 mean, transform of c - mean, k = 0 removed)
    const long long nrows = (long long)nx * ny;
    CKS(launch_sum_field(d_c_in, nrows, nz, nz, g.d_part, SUM_BLOCKS, st));
    CKS(launch_reduce_partials(g.d_part, SUM_BLOCKS, g.d_scal, 1.0 / (double)V, st));
    {
        ZPassArgs z = zs(&g);
        z.rin = d_c_in;
        z.rpitch = nz;
        z.map_rows = 1;
        z.out = g.W;
        z.cbar = g.d_scal;
        CKS(launch_zpass(z, Z_R2C, st));
        CKS(launch_spass(ys(&g, g.W, g.W), -1, st));
        CKS(launch_xupdate(xs(&g, nullptr, g.W, g.S, 0.0, 0.0, 0.0), st));
    }
    // n_steps semi-implicit steps
    for (int i = 0; i < n_steps; ++i) {
        CKS(launch_spass(ys(&g, g.S, g.W), +1, st));
        ZPassArgs z = zs(&g);
        z.in = g.W;
        z.out = g.W;
        z.cbar = g.d_scal;
        CKS(launch_zpass(z, Z_STEP, st));
        CKS(launch_spass(ys(&g, g.W, g.W), -1, st));
        CKS(launch_xupdate(xs(&g, g.W, g.S, g.S, p.dt, p.M, p.kappa), st));
    }
    // state -> output field
    CKS(launch_spass(ys(&g, g.S, g.W), +1, st));
    {
        ZPassArgs z = zs(&g);
        z.in = g.W;
        z.rout = d_c_out;
        z.rpitch = nz;
        z.map_rows = 1;
        z.cbar = g.d_scal;
        CKS(launch_zpass(z, Z_C2R, st));
    }
    return EVX_OK;
}
