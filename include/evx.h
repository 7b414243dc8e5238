/*
 * evx.h - C-ABI of the GB300 (sm_103a) semi-implicit Fourier-spectral
 * Cahn-Hilliard solver (the evoxels method, arXiv 2507.21748).
 *
 * The method (paper, Appendix "Microstructure modelling"):
 *   Eq. (cahn-hilliard)  c_t = div(M grad mu), mu = f'(c) - kappa lap c, here
 *   with constant mobility M, f'(c) = c^3 - c and kappa the gradient
 *   coefficient (the paper's 2 gamma0 eps).
 *   Subsection "Semi-implicit timestepping": the stiff linear operator is
 *   treated implicitly in Fourier space with the prefactor dt / (1 - dt S),
 *   S its symbol (S = -M kappa |k|^4), which for the spectral right-hand side
 *   gives, per step,
 *       c_hat <- (c_hat - dt M |k|^2 F{c^3 - c}) / (1 + dt M kappa |k|^4).
 *   Grid: periodic nx*ny*nz voxels of edge h; k_d = 2 pi m / (n_d h) with m the
 *   signed index.
 *
 * Conventions for every entry point
 *   - Every call returns an evx_status; no exception or abort crosses the ABI.
 *     On failure the message is available from evx_last_error(g).
 *   - "device pointer" arguments are CUDA device addresses on the device that
 *     was current when the grid was created; the caller owns them and keeps
 *     them alive until the work on the grid's stream that uses them has
 *     finished. "host pointer" arguments are ordinary (ideally pinned) host
 *     memory; calls taking host pointers return only after the copy is done.
 *   - Real fields are float32, C order (x slowest, z fastest), nx*ny*nz values,
 *     contiguous.
 *   - A grid owns all of its internal buffers (allocated in evx_grid_create,
 *     except the adjoint's segment store, allocated by the first
 *     evx_ch_adjoint call and kept until destroy). One grid is used by one
 *     host thread at a time.
 *   - Work is issued on the grid's CUDA stream and is asynchronous unless the
 *     entry point says it synchronises.
 *   - Sizes: nx, ny, nz each even, 8 <= n <= 1024, with no prime factor other
 *     than 2, 3 and 5; otherwise EVX_ERR_SIZE. Every such size runs the same
 *     arithmetic. Each pass picks its kernel by its own length: nx, ny in
 *     {64, ..., 1024 powers of two, 400} and nz in {128, ..., 1024 powers of
 *     two, 400} take the tuned four-step kernels; other lengths take the
 *     mixed-radix ones (same results to FP32 rounding, several times slower).
 */
#ifndef EVX_H
#define EVX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct evx_grid evx_grid; /* opaque */

typedef enum {
    EVX_OK = 0,
    EVX_ERR_ARG = 1,       /* null pointer, non-positive count, bad parameter */
    EVX_ERR_SIZE = 2,      /* grid size outside the supported set */
    EVX_ERR_OOM = 3,       /* device allocation failed */
    EVX_ERR_CUDA = 4,      /* a CUDA runtime call or kernel launch failed */
    EVX_ERR_NONFINITE = 5, /* a reduction found NaN or Inf in the field */
    EVX_ERR_STATE = 6,     /* call made in the wrong state (e.g. no field set) */
    EVX_ERR_IO = 7         /* checkpoint file cannot be opened, read or written, or is corrupt */
} evx_status;

/* Scheme parameters: time step dt, mobility M (>= 0), gradient coefficient
 * kappa (>= 0), voxel edge h (> 0). Appendix "Semi-implicit timestepping". */
typedef struct {
    double dt;
    double M;
    double kappa;
    double h;
} evx_params;

/* Create a grid: validates sizes, allocates the two half-spectrum FP32
 * buffers (state S and work W, each nx*ny*Zp complex64 with
 * Zp = roundup(nz/2 + 1, 8)), FP64 scalars, reduction scratch and the
 * twiddle and wave-number tables. cuda_stream: a cudaStream_t (NULL = the
 * legacy default stream). *out receives the handle. The grid holds no field
 * until evx_set_field. On EVX_ERR_OOM every buffer the call allocated has been
 * freed. Test hook for the allocation-failure paths (host side, no GPU fault):
 * with EVX_FAIL_ALLOC=k in the environment, the k-th and every later device
 * allocation within one call (evx_grid_create, evx_set_model, evx_ch_adjoint)
 * reports failure without calling cudaMalloc. */
evx_status evx_grid_create(int nx, int ny, int nz, evx_params p, void *cuda_stream,
                           evx_grid **out);

/* Synchronise the grid's stream and free everything the grid owns. NULL is
 * accepted (no-op). */
evx_status evx_grid_destroy(evx_grid *g);

/* Replace dt, M, kappa, h (validated as above). Takes effect for work issued
 * after the call. */
evx_status evx_set_params(evx_grid *g, evx_params p);

/* Current parameters of g (after evx_load: the checkpoint's). */
evx_status evx_get_params(const evx_grid *g, evx_params *p);

/* Change the stream later work is issued on (the caller orders it against
 * earlier work). */
evx_status evx_set_stream(evx_grid *g, void *cuda_stream);

/* Load the initial field from a device pointer d_c (nx*ny*nz float32). The
 * library forms the spectral state (3D real-to-complex transform of c) and
 * carries the mean of c separately in FP64 (sum in FP64 of the FP32 input):
 * the k = 0 Fourier mode never enters an FP32 buffer, so the scheme's mass
 * (paper: "conserved") is kept exactly. Asynchronous. */
evx_status evx_set_field(evx_grid *g, const float *d_c);

/* Same from a host pointer; returns after the host buffer has been read. */
evx_status evx_set_field_host(evx_grid *g, const float *h_c);

/* Write the current real field c(x) (inverse transform + FP64 mean) to the
 * caller's device buffer d_out (nx*ny*nz float32). Asynchronous. */
evx_status evx_get_field(evx_grid *g, float *d_out);

/* Same into host memory; synchronises the stream. When h_out is page-locked
 * host memory mapped into the device's address space (cudaHostAlloc or
 * cudaMallocHost under unified addressing), the inverse transform writes the
 * field straight into it; other host memory is filled through a device
 * staging buffer and copies. */
evx_status evx_get_field_host(evx_grid *g, float *h_out);

/* Advance the state by n_steps >= 0 semi-implicit Cahn-Hilliard steps
 * (update above). Asynchronous: the steps are issued on the grid's stream (as
 * CUDA-graph launches when profiling is off). EVX_ERR_STATE if the grid is set
 * to another model. */
evx_status evx_ch_step(evx_grid *g, int n_steps);

/* Models the step engine runs (default EVX_MODEL_CH).
 *
 * EVX_MODEL_AC: the Allen-Cahn equation for a non-conserved order parameter
 * (paper: Eq. (allen-cahn) of subsection "Phase transformations of first and
 * second order"), under the same readings as above (gamma0 = 1, kappa =
 * 2 gamma0 eps, f'(c) = c^3 - c) with the kinetic coefficient L = p.M:
 *   c_t = -L (c^3 - c - kappa lap c).
 * Subsection "Semi-implicit timestepping" with S = -L kappa |k|^2 gives
 *   c_hat' = (c_hat - dt L F{c^3 - c}) / (1 + dt L kappa |k|^2).
 * The k = 0 mode is not conserved: the FP64 mean moves by
 *   cbar' = cbar - dt L mean(c^3 - c)
 * with the mean of the nonlinearity summed in FP64 from per-CTA partials.
 * Same four passes (plus a one-block mean update), same sizes, energy and
 * field calls; evx_ch_adjoint and evx_ch_step_static are Cahn-Hilliard only.
 * Changing the model drops the captured step graphs (synchronises). */
/*
 * EVX_MODEL_VM: Cahn-Hilliard with the variable mobility of Eq.
 * (cahn-hilliard), M(phi) = D0 phi (1 - phi), read in the c form as
 * M(c) = p.M max(1 - c^2, 0), in the general form of subsection
 * "Semi-implicit timestepping": the right-hand side is a finite-difference
 * approximation in real space and only the preconditioner is spectral,
 *   c' = c + F^-1{ dt / (1 + dt M kappa |k|^4) F{div(M(c) grad mu)} },
 *   mu = c^3 - c - kappa lap_h c,
 * with second-order central differences in conservative form (7-point
 * Laplacian; face mobility (M_i + M_j)/2). The state is the real FP32 field;
 * per step two FD stencil kernels, a z R2C, the y and x passes (x pass in its
 * preconditioner-only mode), the y inverse and a z C2R that adds the increment
 * (7 launches). Switching to or from EVX_MODEL_VM drops the field (set it
 * again); it allocates one more real field for the right-hand side. Its
 * energy is the FD form h^3 sum (c^2-1)^2/4 + h^3 (kappa/2) sum_d |D_d c|^2
 * and evx_mean sums the field in FP64 on each call. Per-pass times in this
 * model: 0 x preconditioner + y inverse + z C2R-add, 1 FD stencils,
 * 2 z R2C, 3 y forward.
 */
typedef enum { EVX_MODEL_CH = 0, EVX_MODEL_AC = 1, EVX_MODEL_VM = 2 } evx_model;
evx_status evx_set_model(evx_grid *g, int model);
int evx_get_model(const evx_grid *g); /* -1 for NULL */

/* Advance the state by n_steps >= 0 steps of the grid's model (either one);
 * asynchronous, as evx_ch_step. */
evx_status evx_step(evx_grid *g, int n_steps);

/* One block of n_steps (1..4096) Cahn-Hilliard steps at the cost of one step:
 * the scheme's stiff linear part is applied exactly over the block and its
 * nonlinear remainder is frozen at the block's start. With d = c - cbar and
 * g(c) = g(cbar) + g'(cbar) d + N(d), N = d^2 (3 cbar + d), the scheme above
 * reads c_hat' = L c_hat + B N_hat (k != 0), L = (1 - dt M |k|^2 g'(cbar)) / D,
 * B = -dt M |k|^2 / D; holding N_hat fixed,
 *   c_hat_n = L^n c_hat_0 + B (sum_{j<n} L^j) N_hat_0,
 * and the FP64 mean is unchanged. n_steps = 1 is one step of the scheme. This
 * propagator is not the paper's: it is the base that the learned surrogate
 * corrects (include/evx_nn.h). Four passes on the grid's stream, not captured
 * in a graph; the step count advances by n_steps. EVX_ERR_STATE for another
 * model or no field. */
evx_status evx_ch_block(evx_grid *g, int n_steps);

/* Ginzburg-Landau energy and mass of the current field, in FP64 (paper:
 * F_int of subsection "Phase transformations", in the c in [-1, 1] form):
 *   E    = h^3 sum_x (c^2 - 1)^2 / 4 + h^3 (kappa/2) (1/V) sum_k |k|^2 |c_hat(k)|^2
 *   mass = h^3 V cbar   (cbar the FP64 mean carried since evx_set_field).
 * Either output pointer may be NULL. Host outputs; synchronises the stream.
 * Returns EVX_ERR_NONFINITE if the field holds NaN or Inf. */
evx_status evx_energy(evx_grid *g, double *E, double *mass);

/* FP64 mean of the field (the carried cbar); host output; synchronises. */
evx_status evx_mean(evx_grid *g, double *cbar);

/* Discrete adjoint of n_steps steps of the scheme started from d_c0 (device,
 * nx*ny*nz float32), with the current parameters. Given d_dLdcN = dL/dc_N
 * (device, same layout) it writes dL/dc_0 to d_dLdc0 (device, caller-owned)
 * and, if non-NULL, dL/dkappa and dL/dM to host doubles. The forward states
 * are recomputed from checkpoints taken every ckpt_every steps (>= 1); memory
 * grows with ckpt_every (about 3 fields per step of a segment). The grid's
 * own state is overwritten (it holds c_N of the replayed trajectory
 * afterwards). Synchronises. Recursion:
 *   lambda_N = dL/dc_N,
 *   lambda_n = A lambda_{n+1} + (3 c_n^2 - 1) (B lambda_{n+1}),
 * A, B the convolutions of symbols a = 1/D, b = -dt M |k|^2 / D,
 * D = 1 + dt M kappa |k|^4; parameter gradients accumulate
 * <lambda_{n+1}, (dA/dtheta) c_n + (dB/dtheta) g(c_n)> in FP64. */
evx_status evx_ch_adjoint(evx_grid *g, const float *d_c0, int n_steps, int ckpt_every,
                          const float *d_dLdcN, float *d_dLdc0, double *dLdkappa,
                          double *dLdM);

/* Device memory the grid holds, in bytes (buffers + tables + scratch). */
evx_status evx_footprint(const evx_grid *g, size_t *bytes);

/* Per-pass timing. With profiling on, evx_step / evx_ch_step issue their kernels
 * without CUDA graphs and records a CUDA event pair around every pass on the
 * grid's stream; evx_pass_times (synchronises) returns, for each of the four
 * step passes (0: x pass + update, 1: y inverse, 2: z C2R + c^3-c + R2C,
 * 3: y forward), the summed milliseconds and launch counts since the last
 * reset. ms and counts each hold 4 entries. */
evx_status evx_set_profiling(evx_grid *g, int on);
evx_status evx_pass_times(evx_grid *g, double *ms, long long *counts, int reset);

/* Algorithmic bytes one launch of a step pass reads plus writes (each input
 * and output element once): pass index as in evx_pass_times. */
evx_status evx_pass_bytes(const evx_grid *g, int pass, double *bytes);

/* Allocation-free variant of evx_set_field + evx_ch_step + evx_get_field for
 * callers that cannot allocate device memory (a process whose device memory
 * is owned by another runtime, code that must not grow its footprint after
 * start-up, callbacks that may not call cudaMalloc). The paper has no
 * counterpart; it is a deployment convenience around the same kernels.
 * Reads d_c_in (device, nx*ny*nz float32), advances n_steps steps with p and
 * writes d_c_out (device, same layout; may equal d_c_in). All scratch - the
 * two half-spectrum buffers, FP64 scalars, reduction partials, tables - lives
 * in one static device array of 8 MiB that every GPU loading the library
 * holds until the process exits; grids above 64^3 = 262144 voxels return
 * EVX_ERR_SIZE (size rules otherwise as above). No cudaMalloc/cudaFree or
 * allocating library call is made. It always runs the Cahn-Hilliard model, on
 * the mixed-radix kernels (they have no bounded waits, so a call leaves no
 * device-side flag to report). The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture begins. Work is issued asynchronously on cuda_stream. Every call
 * shares the array (its contents persist between calls; the call clears what
 * must start at zero), so calls that overlap on the GPU - e.g. on two streams
 * - race and must be serialised by the caller. Errors: EVX_ERR_ARG,
 * EVX_ERR_SIZE, EVX_ERR_CUDA; message via evx_last_error(NULL). */
evx_status evx_ch_step_static(const float *d_c_in, float *d_c_out, int nx, int ny, int nz,
                              evx_params p, int n_steps, void *cuda_stream);

/* Steps taken since the field was last set (evx_set_field*, evx_load restores
 * the saved count, evx_ch_adjoint leaves n_steps). Host output. */
evx_status evx_step_count(const evx_grid *g, long long *steps);

/* Checkpoint and resume of a run. The paper has no checkpoint format of its
 * own; this serves long runs of the scheme above (subsection "Semi-implicit
 * timestepping") that must survive a restart.
 * evx_save synchronises the grid's stream and writes to the file at path: a
 * header (magic "EVXCKPT1", version 1, nx, ny, nz, model, y block and row pitch
 * of the state layout, dt, M, kappa, h, the FP64 mean, the step count, the
 * payload size and its FNV-1a 64-bit checksum) followed by the state buffer as
 * the grid holds it (the half-spectrum state S of the spectral models, or the
 * real FP32 field of EVX_MODEL_VM). evx_load reads such a file into a grid of
 * the same size, model and layout, restores the parameters, the FP64 mean and
 * the step count, and synchronises; stepping on from it gives bit-for-bit the
 * fields of an uninterrupted run. The payload is read and checked before the
 * grid's state changes. Errors: EVX_ERR_ARG (NULL), EVX_ERR_STATE (no field to
 * save; size, model or layout mismatch), EVX_ERR_IO (open, read, write,
 * truncated or checksum mismatch), EVX_ERR_CUDA. The host buffer used is
 * allocated and freed inside the call (the state's size, or 64 MiB chunks on
 * save). */
evx_status evx_save(evx_grid *g, const char *path);
evx_status evx_load(evx_grid *g, const char *path);

/* Bounds-checked debug build (libevx_bounds.so, compiled with
 * -DEVX_BOUNDS_CHECK; a test facility, not part of the method): *enabled (may
 * be NULL) is 1 in that build, 0 in the normal one. *line (may be NULL)
 * receives the source line of the first global access that the mixed-radix,
 * adjoint, reduction or variable-mobility kernels found outside its buffer
 * since the last call (0 if none; the access was skipped, nothing trapped),
 * and the record is cleared. With line non-NULL the call synchronises the
 * device. The normal build has no checks and always reports 0. */
evx_status evx_debug_bounds(int *enabled, int *line);

/* Last error message of g (or of the calling thread when g is NULL). */
const char *evx_last_error(const evx_grid *g);

#ifdef __cplusplus
}
#endif

#endif /* EVX_H */
