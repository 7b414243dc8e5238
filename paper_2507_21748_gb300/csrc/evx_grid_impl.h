// Private definition of the evx grid handle, shared by the runtime files.
#pragma once
#include <string>
#include <vector>

#include "../../include/evx.h"
#include "evx_internal.h"

using evx::Plan;

struct AdjStore;  // adjoint segment store (evx_adjoint.cu)

struct evx_grid {
    int nx = 0, ny = 0, nz = 0, M = 0, Zp = 0, PZ = 0, zrows = 0;
    int YB = 0;                  // y block of the spectral layout (choose_yblock)
    evx_params p{};
    int model = EVX_MODEL_CH;    // evx_set_model
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only for graph capture
    float2* S = nullptr;
    float2* W = nullptr;
    float* R = nullptr;          // variable-mobility model: real right-hand side (V floats)
    double* d_scal = nullptr;    // [0] cbar, [1] bulk energy, [2] gradient energy, [3..7] scratch
    double* d_part = nullptr;
    int npart = 0;
    float2 *twx = nullptr, *twy = nullptr, *twz = nullptr, *rtw = nullptr;
    float *k2x = nullptr, *k2y = nullptr, *k2z = nullptr;
    Plan px{}, py{}, pz{};
    bool has_field = false;
    std::string err;
    cudaGraphExec_t g1 = nullptr, gN = nullptr;
    bool prof = false;
    std::vector<cudaEvent_t> evpool;  // profiling: 5 events per recorded step
    int ev_used = 0;                  // events of steps not yet accumulated
    double pass_ms[4] = {0, 0, 0, 0};
    long long pass_cnt[4] = {0, 0, 0, 0};
    size_t bytes = 0;
    AdjStore* adj = nullptr;
    int* ctl = nullptr;          // fused y-z-y pass: ticket, abort word, per-slab counters
    bool fused = false;          // the step runs the fused y-z-y pass (evx_fused.cu)
    int lag = 3;                 // its slab lag
    long long steps = 0;         // steps taken since the field was set (saved by evx_save)
    int call_allocs = 0;         // device allocations made in the current public call
};


namespace evxrt {
evx::SPassArgs y_args(const evx_grid* g, const float2* in, float2* out);
evx::XUpdArgs x_args(const evx_grid* g, const float2* W, float2* S, float2* S_out, double dt,
                     double M, double kappa);
evx::ZPassArgs z_args(const evx_grid* g);
evx::YZYArgs yzy_args(const evx_grid* g);
evx_status set_error(evx_grid* g, evx_status s, const char* msg);
// Every device allocation a grid makes goes through device_alloc. Test hook
// (host-side fault injection): when the environment sets EVX_FAIL_ALLOC=k
// (k >= 1), the k-th and every later allocation of one public call report
// failure without calling cudaMalloc. begin_alloc_call starts the count.
void begin_alloc_call(evx_grid* g);
bool device_alloc(evx_grid* g, void** p, size_t bytes);
void adjoint_free(evx_grid* g);  // evx_adjoint.cu
}  // namespace evxrt
