/*
 * pfgpu — explicit forward-Euler time step of phase-field (Allen-Cahn "Model A",
 * Cahn-Hilliard "Model B") and reaction-diffusion (Gray-Scott) models on periodic
 * 2D/3D grids, computed by hand-written CUDA kernels for sm_103a (GB300).
 *
 * The method (arxiv 2109.02598, SymPhas):
 *   - grid: a row-major array with x fastest (Sec. 2.2.1 "Uniform Grid"), periodic on
 *     every side (driver example, Fig. "driver_implementation", Sec. 2.4);
 *   - derivatives: the second-order central Laplacian, 5 points in 2D and 7 in 3D
 *     (Sec. 2.2.2); Model B applies it twice (the 13-point bilaplacian of Sec. 2.2.2);
 *   - equations of motion (Sec. 3):  Model A  dphi/dt = lap phi + c1 phi - c2 phi^3;
 *     Model B  dphi/dt = M lap(c2 phi^3 - c1 phi - lap phi);  Gray-Scott (named in
 *     Sec. 1, standard two-species form)  du/dt = Du lap u - u v^2 + F (1 - u),
 *     dv/dt = Dv lap v + u v^2 - (F + k) v;
 *   - solver: forward Euler (Sec. 2.4.1), x^{n+1} = x^n + dt f(x^n) with every field
 *     read from x^n — the paper's equation()/step() pair (Sec. 2.2.4) fused into one
 *     kernel per step (or per k steps with temporal blocking).
 *
 * Conventions for every call:
 *   - returns PF_OK (0) or a negative PF_ERR_* code; pf_last_error() then gives a
 *     message (thread-local, valid until the next failing call on that thread);
 *   - field arrays exchanged with the caller are dense float32, C order
 *     [nz][ny][nx] (3D) or [ny][nx] (2D), x fastest; the library copies them into its
 *     own padded layout (row pitch rounded up to a multiple of 4 floats);
 *   - pointers passed in are borrowed: the library never frees or retains them past the
 *     call, except that device-to-device copies are enqueued on the grid's stream and
 *     read the source when that stream reaches them;
 *   - handles (pf_grid_t, pf_batch_t) and the device memory behind them are owned by
 *     the library and released by pf_destroy / pf_batch_destroy;
 *   - all device work is enqueued on the CUDA stream given at creation (NULL = the
 *     legacy default stream); calls that hand data to host memory synchronize it.
 *   No call traps, aborts or waits without bound; bad arguments are rejected with
 *   PF_ERR_INVALID_ARG before any device work is enqueued.
 */
#ifndef PFGPU_H
#define PFGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define PF_OK 0
#define PF_ERR_INVALID_ARG (-1) /* bad handle, size, index, model or coefficient count */
#define PF_ERR_OOM (-2)         /* device or pinned-host allocation failed */
#define PF_ERR_CUDA (-3)        /* a CUDA runtime/driver call failed (message has the name) */
#define PF_ERR_UNSTABLE_DT (-4) /* dt beyond the linear forward-Euler stability bound */
#define PF_ERR_NONFINITE (-5)   /* a reduction found NaN/Inf: the state blew up */
#define PF_ERR_STATE (-6)       /* call out of order (no model set, no forward pass, ...) */
#define PF_ERR_TIMEOUT (-7)     /* a bounded wait inside a kernel ran out; the kernel stopped
                                   early and the state is invalid (reported by the next
                                   synchronising call) */

/* ---------------------------------------------------------------- models */
#define PF_MODEL_AC 1 /* Allen-Cahn, 1 field, coeffs {c1, c2}          (Sec. 3, Model A) */
#define PF_MODEL_CH 2 /* Cahn-Hilliard, 1 field, coeffs {c1, c2, M}    (Sec. 3, Model B) */
#define PF_MODEL_GS 3 /* Gray-Scott, 2 fields (u, v), coeffs {Du, Dv, F, k}   (Sec. 1) */
#define PF_MODEL_C 4  /* Model C (eutectic), 2 fields (psi, m), coeffs {c1, c2, c3, c4, c5}:
                         dpsi/dt = lap psi + c1 psi - c2 psi^3 + 2 c5 psi m,
                         dm/dt = -lap^2 m - lap(c3 m - c4 m^3 + c5 psi^2)   (Sec. 3) */
#define PF_MODEL_RD 5 /* N coupled species of reaction-diffusion type, N = the grid's field
                         count (1..4; the coupled equations of motion of Sec. 2.3, of which
                         Gray-Scott, Sec. 1, is the two-species case):
                           du_i/dt = D_i lap u_i + sum_m K[i][m] prod_j u_j^E[m][j]
                         coeffs {D_0 .. D_{N-1}, M, E[0][0..N-1] .. E[M-1][..],
                                 K[0][0..M-1] .. K[N-1][..]}: M <= 8 monomials, exponents
                         integers in [0, 3], D_i >= 0; N + 1 + 2 N M values. 5-/7-point
                         stencil, one kernel, k = 1; the stability check covers the
                         diffusion terms (dt max D 4d/h^2 <= 2) */

/* ---------------------------------------------------------------- Laplacian stencils */
#define PF_STENCIL_STD 0 /* second order: 5-point (2D), 7-point (3D); the default      */
#define PF_STENCIL_ISO 1 /* second order, isotropic leading error: 9-point (2D) with
                            weights (4 axial, 1 diagonal, -20)/6h^2; 19-point (3D) with
                            (2 faces, 1 edges, -24)/6h^2                     (Sec. 2.2.2) */
#define PF_STENCIL_4TH 2 /* fourth order, 9-point (2D only): per axis
                            (-1, 16, -30, 16, -1)/12h^2                     (Sec. 2.2.2) */
#define PF_STENCIL_ISO27 3 /* second order, isotropic leading error, 27-point (3D only):
                              (14 faces, 3 edges, 1 corners, -128)/30h^2   (Sec. 2.2.2) */

/* ---------------------------------------------------------------- reductions */
#define PF_REDUCE_MASS 1   /* h^d * sum_x phi_x of one field                         */
#define PF_REDUCE_ENERGY 2 /* discrete free energy (AC, CH: of field 0; Model C: of both):
                              h^d sum_x [1/2 sum_i ((phi_{x+e_i}-phi_x)/h)^2
                                         - c1/2 phi^2 + c2/4 phi^4]; Model C adds
                              1/2 |grad m|^2 - c3/2 m^2 + c4/4 m^4 - c5 psi^2 m     */

typedef struct pf_grid_s* pf_grid_t;
typedef struct pf_batch_s* pf_batch_t;

/* Library version (major*10000 + minor*100 + patch). */
int pf_version(void);

/* Message of the last failing call on this thread ("" if none). Owned by the library. */
const char* pf_last_error(void);

/* ----------------------------------------------------------------- single grid */

/* Create a periodic grid (the paper's Grid/System, Sec. 2.2.1 and 2.2.5).
 *   dim      2 or 3;
 *   n        n[0] = nx, n[1] = ny, n[2] = nz (ignored for dim 2); each in [1, 2^30];
 *   n_fields 1 .. 4 (Models A and B take 1, Gray-Scott and Model C 2, PF_MODEL_RD any);
 *   h        grid spacing, > 0;
 *   stream   cudaStream_t to enqueue all work on (NULL = legacy default stream);
 *   out      receives the handle.
 * Allocates two device copies of every field (ping-pong), zero-filled.
 * Errors: PF_ERR_INVALID_ARG, PF_ERR_OOM, PF_ERR_CUDA. */
int pf_create_grid(int dim, const int64_t* n, int n_fields, double h, void* stream,
                   pf_grid_t* out);

/* Release the grid and its device memory (synchronizes its stream first). NULL is a no-op. */
void pf_destroy(pf_grid_t g);

/* Choose the equation of motion and its coefficients (Sec. 3; see PF_MODEL_*).
 *   coeffs/n_coeffs  AC {c1, c2}, CH {c1, c2, M}, GS {Du, Dv, F, k},
 *                    C {c1, c2, c3, c4, c5}, RD as at PF_MODEL_RD (exact count);
 *   dt               time step, > 0;
 *   force            0: reject dt beyond the linear stability bound of forward Euler
 *                    (PF_ERR_UNSTABLE_DT, nothing changed); 1: accept it.
 * The kernels use the coefficients rounded once to float32.
 * Errors: PF_ERR_INVALID_ARG (model, count, field count, non-finite), PF_ERR_UNSTABLE_DT. */
int pf_set_model(pf_grid_t g, int model, const double* coeffs, int n_coeffs, double dt,
                 int force);

/* Copy field `field` in from `src` (host memory if src_on_device == 0, else device memory):
 * a dense float32 array [nz][ny][nx], x fastest, the row-major uniform grid of Sec. 2.2.1
 * ("Uniform Grid"); the library copies it into its padded rows. Host copies complete before
 * return; device copies are enqueued on the grid's stream.
 * Errors: PF_ERR_INVALID_ARG, PF_ERR_CUDA. */
int pf_write_field(pf_grid_t g, int field, const float* src, int src_on_device);

/* Copy field `field` out to `dst`: a dense float32 array [nz][ny][nx], x fastest (the
 * layout of Sec. 2.2.1, as pf_write_field). Host destinations are complete on return (the
 * stream is synchronized); device destinations are enqueued.
 * Errors: PF_ERR_INVALID_ARG, PF_ERR_CUDA. */
int pf_read_field(pf_grid_t g, int field, float* dst, int dst_on_device);

/* Host copies that do not wait: the copy of a dense float32 host array into field `field`
 * (write) or of field `field` out to one (read) is enqueued on the grid's stream after the
 * work already there, and the call returns. A caller that pipelines jobs (uploading the next
 * job's fields and downloading the last one's results while a step runs, e.g. on two grids
 * with two streams) uses these; the host array must be page-locked (pinned) for the copy to
 * overlap other work, and must stay valid and untouched until the stream has passed the
 * copy (pf_synchronize). A read sees the field as the preceding pf_step calls leave it.
 * Errors: PF_ERR_INVALID_ARG, PF_ERR_CUDA; a timed-out kernel wait is reported by the next
 * pf_synchronize. */
int pf_write_field_host_async(pf_grid_t g, int field, const float* src);
int pf_read_field_host_async(pf_grid_t g, int field, float* dst);

/* Advance the state by n_steps forward-Euler steps (Sec. 2.4.1), asynchronously on the
 * grid's stream. Uses temporal blocking of depth k (pf_set_tuning) where the model and
 * dimension support it; the result is bitwise the same for every k and tile shape.
 * n_steps == 0 is a no-op. Errors: PF_ERR_STATE (no model), PF_ERR_INVALID_ARG (n < 0),
 * PF_ERR_CUDA. */
int pf_step(pf_grid_t g, int64_t n_steps);

/* Deterministic reduction of the current state into *out (see PF_REDUCE_*): warp
 * shuffles to per-block partial sums in FP64, then one fixed-order FP64 sum.
 *   PF_REDUCE_MASS    h^d sum_x phi_x of field `field` (the conserved quantity of Model B,
 *                     Sec. 3, and of Model C's m);
 *   PF_REDUCE_ENERGY  the discrete free energy (the paper does not write one out; the reading
 *                     used is the functional whose gradient is Model A's right-hand side,
 *                     with forward differences: see PF_REDUCE_ENERGY above), of field 0 for
 *                     AC/CH, of both fields for Model C; `field` is ignored.
 * Synchronizes the stream. Errors: PF_ERR_INVALID_ARG, PF_ERR_STATE (energy without an
 * AC, CH or Model C model), PF_ERR_CUDA, PF_ERR_NONFINITE (*out is still written). */
int pf_reduce(pf_grid_t g, int what, int field, double* out);

/* Choose the Laplacian stencil of the step (PF_STENCIL_*; Sec. 2.2.2 lists these among the
 * stencil families). Model B and Model C apply it twice. The tuning returns to the default
 * for the stencil. The isotropic and fourth-order stencils run with 2D tiles 64x16 or
 * 128x32 (k <= 2) and with the general 3D kernel (k = 1); the isotropic 9-point stencil also
 * runs on the 2D strip kernel for Allen-Cahn and Gray-Scott (k = 1, 2 or 4); the batch and
 * the adjoint use the standard stencil. Errors: PF_ERR_INVALID_ARG (unknown stencil; fourth order in 3D;
 * 27-point in 2D),
 * PF_ERR_UNSTABLE_DT (the current dt exceeds the bound for the new stencil; nothing changed). */
int pf_set_stencil(pf_grid_t g, int stencil);

/* Kernel tuning: tile_x, tile_y (2D tile, or xy tile of the 3D z-streaming kernel) and
 * k_steps (temporal-blocking depth, 2D only). 0 for any value = library default.
 * Unsupported combinations are rejected with PF_ERR_INVALID_ARG.
 * Supported: 2D tiles 64x16, 128x16, 32x32, 128x32; k in {1, 2, 4} (CH, C: {1, 2});
 * 3D tiles 32x16, 64x8 (general kernel, every model and size) and 64x16, 128x8, 128x16
 * (TMA-staged kernel: AC and GS with nx % tile_x == 0 and ny % tile_y == 0); k = 1;
 * 3D k = 2 with tile nx x 8 (nx = 128 or 256; AC and GS).
 * 3D tile 32x8 selects the box kernel (Models B and C, k = 1 or 2, nx % 4 == 0, any ny and
 * nz): a CTA stages a whole 32 x 8 x 8 box with a halo of 2 k and runs k steps on regions that
 * shrink to the box (the chemical potential one site wider than each step's result); for
 * small grids (64^3), where the z-streaming kernels' plane-by-plane walk is the step's time.
 * 2D tile nx x (ny / CS) selects the on-chip cluster kernel (standard stencil, nx % 4 == 0,
 * ny % CS == 0, the grid in CS CTAs' shared memory; CS = 16 where the device allows clusters
 * of 16, else 8; k in {1, 2, 4, 8} for AC and GS, {1, 2} for CH and C, with k R <= ny / CS):
 * one thread-block cluster holds the whole grid, exchanges k-row halos between its CTAs
 * through distributed shared memory, and runs all steps of a pf_step call in one launch.
 * 2D tile nx x PF_TILE_BANDS selects the band kernel (Allen-Cahn and Cahn-Hilliard, the
 * standard stencil, k = 1, nx % 4 == 0 with 64 <= nx <= 4096, and a band of ceil(ny / P)
 * full rows plus halos in each SM's shared memory, P = min(SMs, ny / (2R)) >= 2 CTAs, R = 1
 * for Allen-Cahn and 2 for Cahn-Hilliard; Cahn-Hilliard 2048^2 takes 14 rows per SM): the
 * grid stays in the shared memory of all SMs for a whole pf_step call (one cooperative
 * launch), and neighbouring bands exchange their edge rows through global memory every step
 * (as 64-bit words tagged with their step, so no flag or fence is needed).
 * It needs all P CTAs resident at once: if the device cannot host them (other work, a
 * restricted context), pf_step fails with PF_ERR_CUDA. Its exchange buffers (4 R nx 8-byte
 * words per CTA) are allocated at its first launch.
 * 2D tile 128 x PF_TILE_STRIPS or 64 x PF_TILE_STRIPS selects the strip kernel (any grid
 * size; k in {1, 2, 4} for Allen-Cahn and Gray-Scott with the 5-point or the isotropic
 * 9-point stencil, {1, 2} for Models B and C with the 5-point stencil): one warp per strip of
 * 128 (or 64) columns walks down its rows with the k steps pipelined in registers, the row
 * neighbours across lanes taken by warp shuffle; the outer k R columns (rounded up to 4, or
 * 2; R = 1 for Allen-Cahn and Gray-Scott, 2 for Models B and C) on each side are recomputed
 * halo, and no shared memory is used.
 * Results are bitwise identical to the tiled kernels. */
#define PF_TILE_BANDS (-1) /* tile_y of the band kernel (with tile_x = nx) */
#define PF_TILE_STRIPS (-2) /* tile_y of the strip kernel (with tile_x = 128 or 64) */
int pf_set_tuning(pf_grid_t g, int tile_x, int tile_y, int k_steps);

/* The tuning in effect (after defaults are resolved). */
int pf_get_tuning(pf_grid_t g, int* tile_x, int* tile_y, int* k_steps);

/* Time every supported (tile, k) for this grid and model (CUDA events), keep the fastest
 * and report it: tiled kernels as a replayed CUDA graph of max(probe_launches, 8) launches
 * (as pf_step runs them), the cluster and band kernels as one launch of 16 k probe_launches
 * steps. A cluster or band candidate whose CTAs the device cannot host at once (the launch
 * reports it) is skipped.
 * The state is not changed: probe launches read the current buffer and write the spare one.
 * Errors: PF_ERR_STATE (no model), PF_ERR_CUDA. */
int pf_autotune(pf_grid_t g, int probe_launches, int* tile_x, int* tile_y, int* k_steps);

/* Block until all work enqueued on the grid's stream is done. */
int pf_synchronize(pf_grid_t g);

/* Copy `count` consecutive planes along the slowest axis (z-planes of ny x nx floats in 3D,
 * rows of nx floats in 2D), from plane `first`, of field `field`'s current state to a dense
 * float32 buffer (to_buf = 1) or from one into it (to_buf = 0): the boundary layers that a
 * domain split along that axis exchanges between neighbours (the paper's boundary layers of
 * Sec. 2.2.1, here between the slabs of one grid). Host buffers synchronize the stream
 * before return; device buffers are enqueued on it.
 * Errors: PF_ERR_INVALID_ARG (range outside the grid, NULL buf), PF_ERR_CUDA. */
int pf_copy_planes(pf_grid_t g, int field, int64_t first, int64_t count, float* buf,
                   int to_buf, int buf_on_device);

/* Current device addresses of field `field` in the padded layout, and that layout:
 * row pitch and plane stride in floats. For zero-copy interop only; the addresses
 * change after every pf_step (ping-pong). */
int pf_field_view(pf_grid_t g, int field, float** dev_ptr, int64_t* pitch, int64_t* plane);

/* ----------------------------------------------------------------- batched runner */

/* One independent periodic 2D Gray-Scott instance of a batch: its size and coefficients. */
typedef struct {
  int64_t nx, ny;       /* grid sides, each in [1, 2^20] */
  double Du, Dv, F, k;  /* Gray-Scott coefficients (Sec. 1 names the model; standard form) */
} pf_gs2d_spec;

/* Create a batch of n independent 2D Gray-Scott grids of uneven sizes and coefficients
 * that advance together: the GPU form of the paper's driver that runs a list of models
 * (Sec. 2.4, the "simultaneous-configs" example). All instances share dt and h.
 * Allocates one device buffer holding every instance twice (ping-pong), zero-filled.
 * Errors: PF_ERR_INVALID_ARG, PF_ERR_UNSTABLE_DT (any instance), PF_ERR_OOM, PF_ERR_CUDA. */
int pf_batch_create(int n, const pf_gs2d_spec* specs, double dt, double h, void* stream,
                    pf_batch_t* out);

/* Release the batch (synchronizes its stream). NULL is a no-op. */
void pf_batch_destroy(pf_batch_t b);

/* Copy field `field` (0 = u, 1 = v) of instance `inst` in / out; dense float32 [ny][nx].
 * Host transfers complete before return; device transfers are enqueued on the stream. */
int pf_batch_write_field(pf_batch_t b, int inst, int field, const float* src, int on_device);
int pf_batch_read_field(pf_batch_t b, int inst, int field, float* dst, int on_device);

/* Tile (one of the 2D tiles of pf_set_tuning, or 128 or 64 x PF_TILE_STRIPS for the strip
 * kernel) and temporal depth k in {1, 2, 4} for every instance; 0 keeps the current value.
 * With the strip kernel each instance's width is split evenly over the fewest strips of 128
 * (or 64) columns that cover it, their output boundaries multiples of 4, and cut into tasks
 * of one height for the whole batch (at least 6 k rows), chosen by playing the task list
 * through the device's in-order dispatch onto its resident warps. Other tile_x values with
 * PF_TILE_STRIPS return PF_ERR_INVALID_ARG. */
int pf_batch_set_tuning(pf_batch_t b, int tile_x, int tile_y, int k_steps);
int pf_batch_get_tuning(pf_batch_t b, int* tile_x, int* tile_y, int* k_steps);

/* Time every (tile, k) on this batch (probe launches read the current state and write the
 * spare copy, so the state is unchanged) and keep the fastest. */
int pf_batch_autotune(pf_batch_t b, int probe_launches, int* tile_x, int* tile_y,
                      int* k_steps);

/* Advance every instance by n_steps forward-Euler steps in one CUDA-graph launch on the
 * batch's stream (one kernel node per k steps, each over all instances' tiles). The graph
 * is recorded on first use for a given (n_steps, tuning, starting buffer) and replayed
 * afterwards. Each instance's result is bitwise the same as pf_step on a single grid. */
int pf_batch_run(pf_batch_t b, int64_t n_steps);

/* Block until the batch's stream is idle. */
int pf_batch_synchronize(pf_batch_t b);

/* Total lattice sites of all instances, and bytes of one state copy (with padding). */
int pf_batch_info(pf_batch_t b, int64_t* sites, int64_t* bytes_per_copy);

/* -------------------------------------- adjoint (2D Gray-Scott, Model A, Model B) */

/* Forward pass that records checkpoints for pf_adj_backward: advances the grid's current
 * state (2D grid; Gray-Scott, Allen-Cahn or Cahn-Hilliard model) by n_steps forward-Euler
 * steps exactly like
 * pf_step, storing the state every ckpt_interval steps (0 = ceil(sqrt(n_steps))), i.e.
 * sqrt(N) checkpointing of the time loop of Sec. 2.4.1. Allocates the checkpoints
 * (ceil(N/C) states), one segment of C-1 states and the adjoint buffers on first use.
 * Errors: PF_ERR_STATE (no Gray-Scott model), PF_ERR_INVALID_ARG (3D grid, n < 1),
 * PF_ERR_OOM, PF_ERR_CUDA. */
int pf_adj_forward(pf_grid_t g, int64_t n_steps, int64_t ckpt_interval);

/* Reverse pass of the recorded forward pass (discrete adjoint of the forward-Euler map):
 * given dL/dx_N (dense float32 [ny][nx]: dLdu_N for field 0, dLdv_N for field 1 of
 * Gray-Scott, NULL for one-field models) of any loss of the final state, writes dL/dx_0
 * (dLdu0, dLdv0; either may be NULL) and dtheta = dL/dcoeffs in pf_set_model order
 * (host doubles, may be NULL): Gray-Scott 4 values (Du, Dv, F, k), Model A 2 (c1, c2),
 * Model B 3 (c1, c2, M). Arrays are device memory if on_device, else host memory.
 * Recomputes each segment from its checkpoint with the forward kernel (bitwise the same
 * states), then applies lambda^n = lambda^{n+1} + dt J(x^n)^T lambda^{n+1} per step;
 * parameter terms are summed in FP64 in a fixed order. The grid's state is not changed.
 * Synchronizes the stream. Errors: PF_ERR_STATE (no forward pass), PF_ERR_INVALID_ARG,
 * PF_ERR_CUDA. */
int pf_adj_backward(pf_grid_t g, const float* dLdu_N, const float* dLdv_N, int on_device,
                    float* dLdu0, float* dLdv0, double* dtheta);

/* -------------------------------------------- semi-implicit Fourier spectral solver */

/* The paper's second solver (Sec. 2.4.2). Each field's equation of motion is split into a
 * linear part L(k) and a nonlinear part N(k) f_hat(psi) in Fourier space; one step is
 *     psi_hat^{n+1}(k) = A(k) psi_hat^n(k) + B(k) N(k) f_hat(psi^n)(k),
 *     A = exp(L dt),  B = (exp(L dt) - 1) / L   (B = dt where L = 0),
 * with A and B N computed once, before the first step (Sec. 2.4.2). The splits, with
 * |k|^2 the wavenumber of the periodic grid of spacing h:
 *     Model A   L = -|k|^2 + c1,            N = 1,        f = -c2 psi^3;
 *     Model B   L = M(-|k|^4 + c1 |k|^2),   N = -M |k|^2, f = c2 psi^3;
 *     Model C   psi: L = -|k|^2 + c1,       N = 1,        f = -c2 psi^3 + 2 c5 psi m;
 *               m:   L = -|k|^4 + c3 |k|^2, N = -|k|^2,   f = c4 m^3 - c5 psi^2.
 * Fourier transforms are cuFFT's (loaded at the first call; PF_ERR_CUDA names it if it is
 * missing); the nonlinear terms, the k-space update and the tables are this library's
 * kernels. Arithmetic is float32; the tables are computed in float64 and rounded once.
 * The state lives in Fourier space on the device; fields cross the boundary in real space
 * as dense float32 arrays in the layout of pf_write_field. */
typedef struct pf_spectral_s* pf_spectral_t;

/* Create a spectral solver.
 *   dim, n    as in pf_create_grid, with nx >= 2 and nx * ny * nz <= 2^30;
 *   h         grid spacing, > 0;
 *   model     PF_MODEL_AC, PF_MODEL_CH or PF_MODEL_C (coefficients as for pf_set_model);
 *   dt        time step, > 0 (the scheme has no stability check: the nonlinear part is
 *             explicit, and too large a dt blows up as it would on the CPU);
 *   stream    cudaStream_t for all work (NULL = legacy default stream);
 *   out       receives the handle. Fields start at zero.
 * Errors: PF_ERR_INVALID_ARG, PF_ERR_OOM, PF_ERR_CUDA. */
int pf_spectral_create(int dim, const int64_t* n, double h, int model, const double* coeffs,
                       int n_coeffs, double dt, void* stream, pf_spectral_t* out);
void pf_spectral_destroy(pf_spectral_t s);

/* Replace field `field` (0 = psi or phi, 1 = m for Model C) by a dense float32 array,
 * host or device. Host copies complete before the call returns; device copies are
 * enqueued. Errors: PF_ERR_INVALID_ARG, PF_ERR_CUDA. */
int pf_spectral_write_field(pf_spectral_t s, int field, const float* src, int src_on_device);

/* Real-space value of field `field` (an inverse transform of the state) into a dense
 * float32 array; host destinations synchronize the stream. Errors as above. */
int pf_spectral_read_field(pf_spectral_t s, int field, float* dst, int dst_on_device);

/* Advance n_steps >= 0 steps (asynchronous). The cuFFT engine replays a recorded CUDA graph
 * per 32 steps; the fused engine runs all n_steps in one cooperative launch.
 * Errors: PF_ERR_INVALID_ARG, PF_ERR_CUDA. */
int pf_spectral_step(pf_spectral_t s, int64_t n_steps);

/* Wait for the solver's stream. Errors: PF_ERR_CUDA; PF_ERR_TIMEOUT if a grid-barrier wait
 * of the fused engine ran out (its kernel then stopped early and the state is invalid; the
 * barrier is reset for the next launch). Host reads report the same. */
int pf_spectral_synchronize(pf_spectral_t s);

/* Engines of pf_spectral_step; both compute the same scheme (float32, to rounding):
 *   PF_SPECTRAL_ENGINE_CUFFT  cuFFT transforms with this library's kernels between them;
 *   PF_SPECTRAL_ENGINE_FUSED  power-of-two sides, nx in [4, 1024], in 2D ny <= 1024 and in 3D
 *                             a (y, z) slab that fits one CTA's shared memory (64 x 64 and
 *                             the like): the whole run in one cooperative launch, two phases
 *                             per step (x-rows: inverse x transform, nonlinear terms, forward
 *                             x transform; per kx, the (y, z) slab: forward transform, update,
 *                             inverse transform) with this library's shared-memory FFTs and a
 *                             bounded grid barrier;
 *   PF_SPECTRAL_ENGINE_AUTO   (default) fused wherever it takes the grid, except two-field
 *                             (Model C) 2D grids with a 1024 side, where cuFFT was measured
 *                             faster; else cuFFT. */
#define PF_SPECTRAL_ENGINE_AUTO 0
#define PF_SPECTRAL_ENGINE_CUFFT 1
#define PF_SPECTRAL_ENGINE_FUSED 2
/* Errors: PF_ERR_INVALID_ARG (unknown engine; fused on a grid it does not take). */
int pf_spectral_set_engine(pf_spectral_t s, int engine);
/* The engine pf_spectral_step uses now (CUFFT or FUSED). */
int pf_spectral_get_engine(pf_spectral_t s, int* engine);

/* ----------------------------------------------------------------- structure factor */

/* Radially averaged structure factor of the phase indicator rho = 1 where psi > 0, else 0,
 * the analysis of the phase-separated systems of Sec. 3:
 *     S(k) = |rho_hat(k)|^2 / N over the full spectrum (N = nx ny nz sites), binned by |k|
 *     in (0, k_max], k_max = (pi / h) sqrt(dim), into n_bins bins of equal width; bin
 *     b = min(floor(|k| / k_max * n_bins), n_bins - 1); k = 0 is left out.
 *   dim, n, pitch  as in pf_reduce_noalloc (psi: float32 [nz][ny][pitch] on the device),
 *                  with nx >= 2 and nx * ny * nz <= 2^30;
 *   h              grid spacing, > 0;
 *   n_bins         in [1, 1024];
 *   centres, mean  host arrays of n_bins doubles: bin centres (b + 1/2) k_max / n_bins and the
 *                  mean of S over the modes in the bin (0 for an empty bin);
 *   counts         host array of n_bins int64: modes per bin (a mode and its mirror -k count
 *                  separately, as in the full spectrum);
 *   stream         cudaStream_t (NULL = legacy default stream); synchronized on return.
 * The transform is a float64 cuFFT; |k| and the bin index are float64 in a fixed order of
 * correctly rounded operations; the per-bin sums are in a fixed order, so the result is the
 * same on every run. Scratch (about 16 bytes per site) is allocated and freed by the call.
 * Errors: PF_ERR_INVALID_ARG, PF_ERR_OOM, PF_ERR_CUDA. */
int pf_structure_factor(int dim, const int64_t* n, int64_t pitch, const float* psi, double h,
                        int n_bins, double* centres, double* mean, int64_t* counts,
                        void* stream);

/* Porod-law check (Sec. 3, Porod's law S ~ (L k^(d+1))^-1): the least-squares line
 *     log S = slope * log k + intercept
 * through the bins of a pf_structure_factor result whose centre lies in [k_lo, k_hi], whose
 * count is > 0 and whose mean S is > 0 (slope near -(d+1) in the scaling regime).
 *   n_bins, centres, mean, counts  host arrays as pf_structure_factor returns them;
 *   slope, intercept, n_used       receive the fit and the number of bins it used.
 * Host arithmetic in float64 only (no device work): sums in bin order, then
 * slope = sum (x - xbar)(y - ybar) / sum (x - xbar)^2.
 * Errors: PF_ERR_INVALID_ARG (NULL pointer, n_bins < 1, k_lo >= k_hi, fewer than two usable
 * bins). */
int pf_porod_fit(int n_bins, const double* centres, const double* mean, const int64_t* counts,
                 double k_lo, double k_hi, double* slope, double* intercept, int* n_used);

/* ------------------------------------------------------------------- self-test */

/* Self-test of the bounded waits inside the kernels: launches one CTA that waits on an
 * mbarrier phase nothing completes (the TMA kernels' wait), then on tagged words nothing
 * writes (the band kernel's wait for its neighbours' edge rows), each with a budget of
 * budget_cycles SM clocks (in [1, 4e9]); both waits give up, the kernel records it and the
 * call returns PF_ERR_TIMEOUT, which is the expected result. Any other status means a path
 * is broken. The GPU stays usable. */
int pf_selftest_wait_timeout(int64_t budget_cycles, void* stream);

/* ------------------------------------------------------- reduction without allocation */

/* Mass or free energy (PF_REDUCE_*) of one caller-owned device field, written to a
 * caller-owned device double, with no memory allocated by the call.
 * The paper has no counterpart: this entry point exists for callers that cannot allocate
 * device memory, such as a host framework that has reserved the whole device for its own
 * allocator, or a latency-critical loop that cannot take cudaMalloc's implicit
 * device-wide synchronisation.
 *   what     PF_REDUCE_MASS or PF_REDUCE_ENERGY (energy uses c1, c2; mass ignores them);
 *   dim, n   as in pf_create_grid; pitch = floats per row (>= nx); the field is float32
 *            [nz][ny][pitch] on the current device, x fastest; entries beyond nx unread;
 *   h        grid spacing (> 0);
 *   out_dev  device address of one double that receives the result;
 *   stream   cudaStream_t (NULL = legacy default stream); the call is asynchronous.
 * Scratch: a fixed 4 KiB device array (512 FP64 partial sums) inside the library, which every
 * GPU that loads the library holds until the process exits; the partial count does not grow
 * with the grid, so every grid within the size limits below fits. The first call on a device
 * looks up the array's device address (make that call before any stream capture). Under
 * CUDA's lazy module loading (the default) that first call also loads the library's modules
 * on the device, which allocates device memory for their code and the array and may
 * synchronise: make one warm-up call before handing the device to an allocator that must
 * own all of it. The address is cached per device for the process; after cudaDeviceReset
 * it is stale, so do not call this entry point again after a reset. All calls share the
 * array and each overwrites all of it before reading it; calls that overlap on the GPU race
 * and may return wrong sums.
 * Errors: PF_ERR_INVALID_ARG (NULL pointers, sides outside [1, 2^30], pitch < nx, more than
 * 2^36 floats, h not finite or <= 0), PF_ERR_CUDA. After the first call on a device it calls
 * no cudaMalloc, cudaFree or other allocating routine. */
int pf_reduce_noalloc(int what, int dim, const int64_t* n, int64_t pitch, const float* field,
                      double h, double c1, double c2, double* out_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PFGPU_H */
