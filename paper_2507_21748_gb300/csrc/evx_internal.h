// Internal interface between the evx runtime (C-ABI) and its CUDA kernels.
#pragma once
#include <cuda_runtime.h>

#include "evx_fft.cuh"

namespace evx {

// Bounds-checked debug build (-DEVX_BOUNDS_CHECK, libevx_bounds.so): the global
// loads and stores of the mixed-radix, adjoint, reduction and variable-mobility
// kernels test their index against the buffer's extent. An access outside it is
// skipped (a load yields zero) and the first offending source line is kept in a
// device word of the translation unit, reported by evx_debug_bounds(). There is
// no trap: the kernel completes and the context stays usable. In the normal
// build the predicate is the constant true.
#ifdef EVX_BOUNDS_CHECK
static __device__ int g_bounds_line;
__device__ __forceinline__ bool evx_in_bounds(long long i, long long n, int line) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&g_bounds_line, 0, line);
    return false;
}
#define EVX_IN(i, n) ::evx::evx_in_bounds((long long)(i), (long long)(n), __LINE__)
#else
#define EVX_IN(i, n) true
#endif
int bounds_line_kernels(bool clear);   // evx_kernels.cu (0 in the normal build)
int bounds_line_adjoint(bool clear);   // evx_adjoint.cu

// Spectral buffers are y-blocked: element (x, y, kz) of a half spectrum sits at
//   ((y / YB * nx + x) * YB + y % YB) * Zp + kz      (complex64 units)
// with YB = 32 when the y pass has a fast path (ny a power of two >= 64) and
// YB = ny otherwise (plain [x][y][kz]). The x stride is then YB * Zp (at most
// 133 KB at nz = 1024), so the 1024 rows of an x tile share a few 2 MB pages.
inline int choose_yblock(int ny, bool fast) {
    if (fast && ny >= 64 && ny <= 1024 && (ny & (ny - 1)) == 0) return 32;
    if (fast && ny == 400) return 16;  // the y pass moves a whole line as one box of 25 blocks
    return ny;
}
// offset of index i along an axis split into blocks of YB: i % YB steps of
// s_in, i / YB steps of s_out
__host__ __device__ inline long long split_off(long long i, int YB, long long s_in, long long s_out) {
    return (i / YB) * s_out + (i % YB) * s_in;
}

// Strided pass: 1D transforms along y; a tile covers P adjacent columns (kz)
// of one x line.
struct SPassArgs {
    const float2* in;
    float2* out;        // may equal in
    int L;              // transform length
    long long rs;       // stride between consecutive elements within a block (complex)
    long long os;       // stride between consecutive outer lines (complex)
    int YB;             // element i at split_off(i, YB, rs, os2)
    long long os2;      // stride between element blocks
    int nouter;         // number of outer lines
    int ncols;          // valid columns (kz = 0 .. M)
    int nchunks;        // column chunks of P
    Plan plan;
    const float2* tw;   // L-entry table exp(-2 pi i m / L)
    int generic;        // 1: mixed-radix kernel only (no fast path, no bounded waits)
};

// x pass fused with the k-space update (one step of the scheme).
struct XUpdArgs {
    const float2* W;    // y,z-transformed g = c^3 - c   (F_y F_z g)
    float2* S;          // state: F_y F_z c (without the k = 0 mode), updated in place
    float2* S_out;      // where the new state goes (== S for a plain step)
    int L;              // nx
    long long rs;       // stride between consecutive x (YB * Zp)
    long long os;       // stride between consecutive y within a block (Zp)
    int YB;             // line ky starts at split_off(ky, YB, os, os2)
    long long os2;      // stride between y blocks (nx * YB * Zp)
    int ny, ncols, nchunks;
    Plan plan;
    const float2* tw;
    const float* k2x;   // |k_x|^2 per index (nx)
    const float* k2y;   // (ny)
    const float* k2z;   // (M + 1)
    float dtM, dtMk, invL;
    int model;          // 0 Cahn-Hilliard: b = -dt M |k|^2, D = 1 + dt M kappa |k|^4
                        // 1 Allen-Cahn:    b = -dt L,       D = 1 + dt L kappa |k|^2
                        // 2 preconditioner: S_out = F_x^-1 dt / (1 + dtMk |k|^4) F_x W / L,
                        //   S not read (dtM holds dt)
                        // 3 Cahn-Hilliard block of nblk steps (evx_ch_block): with
                        //   L = (1 - dt M |k|^2 g'(cbar)) / D, B = -dt M |k|^2 / D,
                        //   S' = F_x^-1 [L^n F_x S + B sum_{j<n} L^j F_x W] / L_x (W: F_y F_z N)
    int generic;        // 1: mixed-radix kernel only (no fast path, no bounded waits)
    int nblk;           // model 3: steps per block
    const double* cbar; // model 3: FP64 mean (for g'(cbar))
};

// Adjoint x pass (evx_adjoint.cu, fast variant in evx_fast.cu): from
// Lambda_{n+1}, S_{n+1} and G_n, P = F_x^-1(a lambda_hat)/nx, T = F_x^-1(b lambda_hat)/nx
// and per-CTA FP64 partials of the two parameter gradients.
struct XAdjArgs {
    const float2* Lam;   // Lambda_{n+1}
    const float2* Sn1;   // S_{n+1}
    const float2* Gn;    // G_n
    float2* P;
    float2* T;
    int L;
    long long rs, os;
    int YB;
    long long os2;
    int ny, ncols, nchunks, M;
    Plan plan;
    const float2* tw;
    const float* k2x;
    const float* k2y;
    const float* k2z;
    float dt, dtM, dtMk, dtk, invL;
    double* partials;    // [2 * nblocks]: kappa partials, then M partials
};

// Energy: gradient term sum_k w(kz) |k|^2 |c_hat|^2 from the state S.
struct XEnergyArgs {
    const float2* S;
    int L;
    long long rs, os;
    int YB;
    long long os2;
    int ny, ncols, nchunks, M;
    Plan plan;
    const float2* tw;
    const float* k2x;
    const float* k2y;
    const float* k2z;
    double* partials;   // one per CTA
};

enum ZMode { Z_STEP = 0, Z_ADJ = 1, Z_R2C = 2, Z_C2R = 3 };

// z pass: real-to-complex / complex-to-real transforms of rows of nz reals
// (half spectrum of M + 1 = nz/2 + 1 complex, row pitch Zp).
struct ZPassArgs {
    const float2* in;       // complex rows (Z_STEP, Z_ADJ, Z_C2R)
    float2* out;            // complex rows (Z_STEP, Z_ADJ, Z_R2C)
    const float* rin;       // real rows (Z_R2C)
    float* rout;            // real rows (Z_C2R; optional side store of c in Z_STEP)
    long long rpitch;       // floats between real rows
    const float* cn;        // real rows of c_n (Z_ADJ)
    long long cnpitch;
    long long nrows;        // nx * ny
    int M, Zp, PZ, rows_per_cta;
    Plan plan;
    const float2* tw;       // M-entry table exp(-2 pi i m / M)
    const float2* rtw;      // (M + 1)-entry table exp(-2 pi i k / nz)
    float scale;            // 1 / (ny nz)
    const double* cbar;     // FP64 mean (Z_STEP, Z_C2R); may be null (0)
    double* partials;       // bulk energy partial per CTA (Z_C2R) or null
    double* gsum;           // Z_STEP, Allen-Cahn: per-CTA FP64 sums of g(c) - g(cbar), or null
    int accumulate;         // Z_C2R: rout += value instead of rout = value
    int fast_ok;            // Z_R2C / Z_C2R: the fast power-of-two kernels may run (grid then reported)
    // map_rows = 1: real rows rin / rout are a caller's C-order field; memory
    // row r of the y-blocked spectrum is caller row x * ny + y
    int map_rows, YB, nxr, nyr;
    int generic;            // 1: mixed-radix kernel only (no fast path)
    int nl_only;            // Z_STEP: form N = d^2 (3 cbar + d) instead of g(c) - g(cbar)
};
__host__ __device__ inline long long user_row(long long r, int YB, int nx, int ny) {
    const long long x = (r / YB) % nx, yb = r / ((long long)YB * nx), yi = r % YB;
    return x * ny + yb * YB + yi;
}

// Fused y inverse + z step + y forward (evx_fused.cu): S (state, F_y F_z c)
// -> W (F_y F_z (g(c) - g(cbar))), per x slab in L2 (see the file's header).
struct YZYArgs {
    const float2* S;
    float2* W;
    int nx, ny, Zp, YB;
    long long os2;          // stride between y blocks (nx * YB * Zp)
    int ncols, nchunks;     // valid columns (M + 1), column chunks of 8
    const float2* twy;      // ny-entry table exp(-2 pi i m / ny)
    const float2* twz;      // M-entry table
    const float2* rtw;      // (M + 1)-entry table exp(-2 pi i k / nz)
    float scale;            // 1 / (ny nz)
    const double* cbar;     // FP64 mean
    double* gsum;           // Allen-Cahn: per-CTA FP64 sums of g(c) - g(cbar), or null
    int* ctl;               // fused_ctl_ints(nx) ints: ticket, abort word, per-slab counters (cleared per launch)
    int lag;                // slabs between a slab's stages in the ticket order
};
int fused_yzy_shape(int ny, int M, int YB);  // 1 if a fused kernel exists for this y / z geometry
bool fused_yzy_enabled();                    // true under EVX_FUSE=1 (read at grid creation), unless EVX_GENERIC=1
size_t fused_ctl_ints(int nx);
cudaError_t launch_fused_yzy(const YZYArgs& a, cudaStream_t st, int* grid_used);
int fused_yzy_grid(const YZYArgs& a);        // CTAs a launch may use (partials it may write)
bool fused_timeout_flag(int* flag, bool clear);

// launchers (evx_kernels.cu)
cudaError_t launch_spass(const SPassArgs& a, int dir, cudaStream_t st);
cudaError_t launch_xupdate(const XUpdArgs& a, cudaStream_t st);
cudaError_t launch_xenergy(const XEnergyArgs& a, cudaStream_t st);
cudaError_t launch_zpass(const ZPassArgs& a, int mode, cudaStream_t st, int* grid_used = nullptr);
// variable-mobility model (real C-order fields, z fastest; periodic)
//   mu  = c^3 - c - (kappa / h^2) lap1 c                    (lap1: 7-point stencil, h = 1)
//   rhs = (1 / h^2) sum over the 6 neighbours j of (M_i + M_j)/2 (mu_j - mu_i), M = M0 max(1 - c^2, 0)
//   partials[b] = sum over the CTA's voxels of (c^2 - 1)^2 / 4 + (kappa / 2h^2) sum_d (c_{i+e_d} - c_i)^2
cudaError_t launch_vm_mu(const float* c, float* mu, int nx, int ny, int nz, float kappa_h2, cudaStream_t st);
// both stencils in one pass (ny a multiple of 8, nz of 64; vm_fd_fused_ok): rhs from c, mu not stored
bool vm_fd_fused_ok(int nx, int ny, int nz);
cudaError_t launch_vm_fd(const float* c, float* rhs, int nx, int ny, int nz, float kappa_h2, float M0, float inv_h2,
                         cudaStream_t st);
cudaError_t launch_vm_rhs(const float* c, const float* mu, float* rhs, int nx, int ny, int nz, float M0,
                          float inv_h2, cudaStream_t st);
cudaError_t launch_vm_energy(const float* c, int nx, int ny, int nz, double kappa_2h2, double* partials, int nparts,
                             cudaStream_t st);
int vm_energy_grid(int nx, int ny, int nparts);  // partials the energy launch writes
// Allen-Cahn mean: cbar <- cbar - dtL (g(cbar) + sum(gsum[0..n)) / V), one block, fixed order
cudaError_t launch_ac_mean(const double* gsum, int n, double* cbar, double dtL, double invV, cudaStream_t st);
int zpass_grid(const ZPassArgs& a);
int xenergy_grid(const XEnergyArgs& a);
// deterministic FP64 sums
// partials[b] (b < nblocks) = FP64 sums over rows of rowlen floats, pitch floats apart
cudaError_t launch_sum_field(const float* c, long long nrows, int rowlen, long long pitch,
                             double* partials, int nblocks, cudaStream_t st);
cudaError_t launch_reduce_partials(const double* partials, int n, double* out, double scale,
                                   cudaStream_t st);
// subtract the mean of n complex values stride apart from each (one block, FP64 sum)
cudaError_t launch_remove_k0(float2* line, int n, long long stride, cudaStream_t st);
// out = a + b (complex arrays of n elements)
cudaError_t launch_cadd(const float2* a, const float2* b, float2* out, long long n,
                        cudaStream_t st);
constexpr int SUM_BLOCKS = 1216;  // 8 x 152 SMs

// fast paths for power-of-two lengths (evx_fast.cu); return false if not applicable
bool fast_spass(const SPassArgs& a, int dir, cudaStream_t st, cudaError_t* err);
bool fast_xupdate(const XUpdArgs& a, cudaStream_t st, cudaError_t* err);
bool fast_zstep(const ZPassArgs& a, cudaStream_t st, cudaError_t* err, int* grid_used, bool adj = false);
// adjoint x pass with the four-step transforms; false if the length has no fast kernel
bool fast_xadj(const XAdjArgs& a, cudaStream_t st, cudaError_t* err);
bool fast_zconv(const ZPassArgs& a, int dir, cudaStream_t st, cudaError_t* err, int* grid_used);
bool fast_paths_enabled();  // false when the environment sets EVX_GENERIC=1
// reads (and optionally clears) the flag a bounded TMA wait sets when it gives up
bool fast_timeout_flag(int* flag, bool clear);

size_t spass_smem(int L);
size_t xupdate_smem(int L);
size_t zpass_smem(int M, int PZ, int rows);

constexpr int SP = 8;  // columns per strided tile (8 complex = 64 B contiguous)

}  // namespace evx
