/*
 * fdtd.h -- C ABI of the GB300 Yee + embedded reduced-order-model library.
 *
 * Method: Zhang, Bekmambetova, Triverio, "A Stable FDTD Method with Embedded
 * Reduced-Order Models" (arXiv:1609.07114).  A 2D TEz Yee leapfrog (Ex, Ey,
 * Hz) runs on a coarse mesh with perfect-electric-conductor walls
 * (Sec. II-A, Eqs. (3), (5)); fine-mesh regions are replaced by passive
 * reduced models (Sec. III, Eq. (11)) coupled to the coarse interface edges
 * (Sec. IV, Eq. (23)) and stepped every time step.
 *
 * Conventions shared by every call
 *   - All calls return int status: FDTD_OK (0) or a negative FDTD_E* code.
 *     A failing call leaves its outputs untouched and records a message,
 *     read with fdtd_last_error(ctx) (or fdtd_last_error(NULL) for calls
 *     without a context).
 *   - Host input arrays are copied during the call; the caller keeps them.
 *   - Device pointers passed in (waveforms, probe outputs) are owned by the
 *     caller and must stay valid until the work queued on the context's
 *     stream has finished.  Device work is queued on the stream given to
 *     fdtd_create (NULL = legacy default stream); calls that return host
 *     data synchronise that stream.
 *   - Grid indexing (0-based): coarse cell (i, j), i < nx, j < ny; Hz[j][i];
 *     Ex[j][i] on the x-edge from node (i, j) to (i+1, j), j <= ny;
 *     Ey[j][i] on the y-edge from node (i, j) to (i, j+1), i <= nx.
 *     Host field buffers are dense row-major: Ex (ny+1) x nx,
 *     Ey ny x (nx+1), Hz ny x nx.
 *   - Units: SI (m, s, S/m, A/m^2); relative permittivity is dimensionless.
 */
#ifndef FDTD_ROM_H
#define FDTD_ROM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FDTD_OK = 0,
  FDTD_EINVAL = -1,       /* malformed argument or descriptor */
  FDTD_ENOMEM = -2,       /* host or device allocation failed */
  FDTD_ECFL = -3,         /* dt not below the coarse CFL limit, Eq. (1) */
  FDTD_ENOTPASSIVE = -4,  /* reduced model violates Eq. (26a)-(26c) at this dt */
  FDTD_ESINGULAR = -5,    /* coupling system of Eq. (19) inconsistent or degenerate */
  FDTD_EUNSTABLE = -6,    /* non-finite field value detected */
  FDTD_ETIMEOUT = -7,     /* a bounded device wait gave up */
  FDTD_ECUDA = -8         /* a CUDA runtime call failed */
};

/* Interpolation rule between coarse interface and fine boundary. */
enum {
  FDTD_RULE_DUAL = 0,  /* y = (1/r) T^T y_hat, u_hat = T U (lossless; any order) */
  FDTD_RULE_PAPER = 1  /* y_hat = T y, U = (1/r) T^T u_hat, Eqs. (15)-(16) */
};

enum { FDTD_SRC_JX = 0, FDTD_SRC_JY = 1 };

typedef struct fdtd_ctx fdtd_ctx;
typedef struct rom_model rom_model;

/* ------------------------------------------------------------------ grids */

/* One independent coarse simulation.  eps_r, sigma: host [ny][nx] per-cell
 * relative permittivity (> 0) and conductivity (>= 0, S/m).  Edge values
 * are the mean of the two adjacent cells (Sec. II-A, text below Eq. (3)). */
typedef struct {
  int nx, ny;
  const double* eps_r;
  const double* sigma;
} fdtd_sim_desc;

/* A batch of simulations sharing cell size and time step.  Grid sizes may
 * differ between simulations; all of them advance together in fdtd_run. */
typedef struct {
  double dx, dy, dt;
  int nsim;
  const fdtd_sim_desc* sims;
} fdtd_grid_desc;

/* Creates a context, allocates all device state (fields zeroed) on the
 * current CUDA device.  Checks dt < 1/(c0 sqrt(1/dx^2+1/dy^2)) (Eq. (1));
 * FDTD_ECFL otherwise.  cuda_stream: a cudaStream_t or NULL. */
int fdtd_create(const fdtd_grid_desc* grid, void* cuda_stream, fdtd_ctx** out);
void fdtd_destroy(fdtd_ctx* ctx);

/* Eq. (1): the 2D vacuum CFL limit of a dx x dy mesh (seconds). */
int fdtd_cfl_limit(double dx, double dy, double* out);

/* --------------------------------------------------------- reduced models */

/* A fine-mesh region of a x b coarse cells refined r times (Sec. II):
 * fine cells (r*a) x (r*b) of size dx/r x dy/r; eps_r, sigma host
 * [r*b][r*a].  q: reduced order q_E + q_H of the SPRIM projection
 * (Sec. III); 0 keeps the full fine model (V = I).  dt: the time step the
 * model will run at (must equal the context's).  f0: frequency (Hz) of the
 * real Krylov expansion point psi0 = tan(pi f0 dt_b).  gamma: CFL-extension
 * margin of Sec. V-E (singular values of Eq. (27) above gamma*2/dt are
 * clamped to it); gamma <= 0 disables the extension.  defl_tol: relative
 * deflation tolerance of the block Arnoldi process (0 selects 1e-12). */
typedef struct {
  int a, b, r;
  double dx, dy, dt;
  const double* eps_r;
  const double* sigma;
  int q;
  int rule;
  double f0;
  double gamma;
  double defl_tol;
} rom_desc;

typedef struct {
  int qE, qH;              /* achieved block orders of V1, V2 (Eq. (9)) */
  int n_inputs;            /* Krylov start-block width: n_u (paper) or n_y (dual) */
  int n_clamped;           /* singular values clamped by the CFL extension */
  double smax_before;      /* max s_k * dt/2 of Eq. (27) before the extension */
  double smax_after;       /* ... and after it (< 1 means Eq. (26a) holds) */
  double min_eig_R;        /* smallest eigenvalue of R~ / largest (Eq. (26a)) */
  double cond3_residual;   /* ||B~ - L~ S_hat|| / ||B~|| (Eq. (26c)) */
  double seconds;          /* host wall time of the build */
} rom_build_report;

/* Builds a reduced model on the host in FP64: fine-system assembly
 * (Sec. II), block-Krylov SPRIM projection (Sec. III), passivity check and
 * optional CFL extension (Sec. V).  rep may be NULL.  The model is
 * independent of any context and may be embedded many times. */
int rom_build(const rom_desc* desc, rom_model** out, rom_build_report* rep);
void rom_free(rom_model* model);

/* Achieved orders and port count of a built model. */
int rom_get_info(const rom_model* model, int* qE, int* qH, int* n_u);

/* Copies the reduced blocks (row-major, FP64, caller-owned host buffers):
 * R11 qE x qE (= V1^T D_eps V1), R22 qH x qH (= V2^T D_mu V2),
 * Kt qE x qH (= V1^T K V2, after any CFL extension), Sig qE x qE
 * (= V1^T D_sigma V1), LE qE x n_u (= V1^T L_E).  Eq. (12):
 * R~ = [[R11/dt, -Kt/2], [-Kt^T/2, R22/dt]], F~ = [[Sig/2, -Kt/2],
 * [Kt^T/2, 0]], B~ = [LE S_hat; 0].  Any pointer may be NULL. */
int rom_get_blocks(const rom_model* model, double* R11, double* R22, double* Kt,
                   double* Sig, double* LE);

/* rom_build with the block Krylov basis, its orthonormalisation and the
 * congruences of Eq. (12) computed on the GPU in FP64 (stream cuda_stream;
 * the banded factorisation, small eigenproblems and Eq. (27) stay on the
 * host).  Orthonormalisation goes through Gram matrices in two stages (the
 * second on what the first leaves), which resolve singular values down to
 * the same deflation tolerance as rom_build, so both builds give the same
 * reduced space to rounding.  Same outputs, ownership and errors as
 * rom_build, plus FDTD_ECUDA on a device failure.  Synchronises the
 * stream. */
int rom_build_gpu(const rom_desc* desc, void* cuda_stream, rom_model** model,
                  rom_build_report* report);

/* Projection bases of a model (Sec. III: x_hat ~ V x~, V = blkdiag(V1, V2)),
 * row-major FP64: V1 is nE x qE over the fine E unknowns, V2 nH x qH over the
 * fine Hz unknowns, in the fine state order (all Ex [r b + 1][r a], then all
 * Ey [r b][r a + 1], each row-major; Hz [r b][r a]).  Sizes through nE, nH;
 * any pointer may be NULL (query the sizes first). */
int rom_get_basis(const rom_model* model, int* nE, int* nH, double* V1, double* V2);

/* Places a model into simulation `sim` with its lower-left coarse cell at
 * (i0, j0); the region is [i0, i0+a) x [j0, j0+b).  The region must keep
 * one coarse cell from the walls and from every other region.  Precomputes
 * in FP64 the run-time map of Eq. (23),
 *     [y; x~]^{n+1} = P [y; x~]^n + Q h^{n+1/2},
 * with the coarse half-cell materials of the cells just outside
 * (Eq. (13)), uploads P and Q in FP32, and zeroes the fields inside.
 * Returns the instance index through inst (may be NULL).
 * FDTD_ENOTPASSIVE if R~ is not positive definite at the context's dt;
 * FDTD_ESINGULAR if the coupling system is inconsistent or (paper rule)
 * leaves the interface unable to carry any field. */
int rom_embed(fdtd_ctx* ctx, const rom_model* model, int sim, int i0, int j0, int* inst);

/* Host-only form of the coupling done by rom_embed: the FP64 run-time map
 * of Eq. (23) for a model whose interface edges (ordered S, N, W, E; n_y =
 * 2(a+b)) see coarse half cells of relative permittivity ring_eps_r[k] and
 * conductivity ring_sigma[k] (Eq. (13)).  P (n_y+q)^2 and Q (n_y+q) x n_y,
 * row-major, caller-owned.  No device work. */
int rom_couple(const rom_model* model, const double* ring_eps_r, const double* ring_sigma,
               double* P, double* Q);

/* The FP64 run-time map of an embedded instance: n = n_y + q.  P n x n,
 * Q n x n_y row-major host buffers (either may be NULL to query sizes). */
int fdtd_get_rom_map(const fdtd_ctx* ctx, int inst, int* n, int* n_y, double* P, double* Q);

/* ---------------------------------------------------------- time marching */

/* An electric current density J (A/m^2) on `len` consecutive edges of one
 * component, starting at edge (i, j) and running along the edge direction
 * (Jx: i, i+1, ...; Jy: j, j+1, ...).  It enters Eq. (3) as the term
 * -dx dy J on the right-hand side.  wave: samples J(t^{n+1/2}) for the
 * n = 0 .. nsteps-1 steps of this run (device FP32 for fdtd_run, host FP32
 * for fdtd_run_host).  Edges must be updated coarse edges (not PEC, not on
 * or inside a region). */
typedef struct {
  int sim;
  int comp;
  int i, j;
  int len;
  const float* wave;
} fdtd_source;

/* Records Hz^{n+1/2} of coarse cell (i, j) of simulation sim every step. */
typedef struct {
  int sim, i, j;
} fdtd_probe;

/* Advances every simulation of the context by nsteps (Sec. IV-C: coarse
 * H, coarse E with sources, then Eq. (23) for every embedded model).
 * probe_out: device FP32 [nsteps][nprobe] (may be NULL when nprobe = 0).
 * Asynchronous on the context's stream. */
int fdtd_run(fdtd_ctx* ctx, long long nsteps, const fdtd_source* src, int nsrc,
             const fdtd_probe* probes, int nprobe, float* probe_out);

/* Same as fdtd_run with host buffers: copies the source waveforms to the
 * device, runs, copies the probe samples back, and synchronises.  Returns
 * FDTD_EUNSTABLE if a probe sample is not finite. */
int fdtd_run_host(fdtd_ctx* ctx, long long nsteps, const fdtd_source* src, int nsrc,
                  const fdtd_probe* probes, int nprobe, float* probe_out_host);

/* Gradient of the probe energy J = sum_n sum_p (Hz^{n+1/2}(p))^2 over the
 * next nsteps steps, by the exact discrete adjoint of the time loop
 * (transposed Eqs. (3), (5) and (23), run backwards).  Not in the paper; the
 * reverse sweep recomputes the forward pass segment by segment from
 * checkpoints taken every ckpt_every steps (the E fields of one segment are
 * held in device memory).  Outputs (device, caller-owned, overwritten):
 *   dJ_deps   FP32, per simulation [ny][nx] concatenated: dJ/d eps_r of each
 *             coarse cell (0 for cells covered by a model; the coarse half
 *             cells of interface edges include their effect through A1, A2
 *             of Eq. (19));
 *   dJ_dsigma FP32, same layout: dJ/d sigma (S/m);
 *   dJ_dsrc   FP32 [nsrc][nsteps]: dJ/dJ^n for each source sample;
 * any of them may be NULL.  J_out: host double (may be NULL).  The context
 * ends in the state reached by the forward pass (as after fdtd_run).
 * Ring-cell gradients assume a nonsingular coupling (dual rule, or the paper
 * rule with a full-order model).  The recomputation and the reverse sweep
 * take two steps per launch where the context does; the reverse sweep then
 * adds the model, probe and source terms of its second step afterwards as
 * local corrections (FDTD_ADJ_TB2=0: one reverse step per launch), which
 * changes the FP32 rounding at the cells beside the models and at the probes
 * only; additions that meet in one cell or edge are atomic, so the last bit
 * there can vary between calls.  Synchronises. */
int fdtd_grad(fdtd_ctx* ctx, long long nsteps, const fdtd_source* src, int nsrc,
              const fdtd_probe* probes, int nprobe, int ckpt_every, float* dJ_deps,
              float* dJ_dsigma, float* dJ_dsrc, double* J_out);

/* Vector-Jacobian product of the probe series (not in the paper): with the
 * probe samples o[n][p] = Hz^{n+1/2}(probe p) of the next nsteps steps and a
 * cotangent c = dL_dprobe (device FP32 [nsteps][nprobe], caller-owned),
 * the gradient of L = sum_n sum_p c[n][p] o[n][p] by the same exact discrete
 * adjoint as fdtd_grad (whose J is the case c = 2 o).  It runs the forward
 * pass with checkpoints every ckpt_every steps and the reverse sweep seeded
 * with c.  Outputs as for fdtd_grad (dL_deps, dL_dsigma per simulation
 * [ny][nx] concatenated, dL_dsrc [nsrc][nsteps]; any may be NULL; device,
 * caller-owned, overwritten); probe_out (device FP32 [nsteps][nprobe], may be
 * NULL) receives the forward pass's probe samples.  The context ends in the
 * state reached by the forward pass.  FDTD_EINVAL when nprobe > 0 and
 * dL_dprobe is NULL.  Synchronises. */
int fdtd_vjp(fdtd_ctx* ctx, long long nsteps, const fdtd_source* src, int nsrc,
             const fdtd_probe* probes, int nprobe, int ckpt_every, const float* dL_dprobe,
             float* dL_deps, float* dL_dsigma, float* dL_dsrc, float* probe_out);

/* ---------------------------------------------------------- open boundaries */

/* Convolutional PML layers (complex-frequency-shifted CPML of Roden and
 * Gedney) inside the PEC walls of one simulation; the paper terminates its
 * open structures with PML layers of a few coarse cells (Sec. VI) without
 * stating the formulation.  Every spatial difference of Eqs. (3), (5) in a
 * layer becomes (1/kappa) d + psi with psi^n = b psi^{n-1} + a d^n,
 * b = exp(-(sigma/kappa + alpha) dt/eps0),
 * a = sigma (b - 1) / (sigma kappa + kappa^2 alpha); at depth rho in [0, 1]
 * (0 at the layer's inner face, 1 at the wall) sigma = sigma_max rho^m,
 * kappa = 1 + (kappa_max - 1) rho^m, alpha = alpha_max (1 - rho), each sampled
 * where its difference is taken.  Outside the layers the update is unchanged. */
enum { FDTD_PML_W = 1, FDTD_PML_E = 2, FDTD_PML_S = 4, FDTD_PML_N = 8 };
typedef struct {
  int sides;          /* FDTD_PML_* bits (x = 0, x = nx, y = 0, y = ny); 0 = none */
  int ncells;         /* layer thickness in coarse cells (>= 1 when sides != 0) */
  double m;           /* grading order, > 0 (3 is usual) */
  double sigma_max;   /* S/m at the wall; <= 0 selects 0.8 (m + 1) / (eta0 h) */
  double kappa_max;   /* >= 1 */
  double alpha_max;   /* S/m, >= 0 */
} fdtd_pml_desc;

/* Sets (or with sides = 0 removes) the layers of simulation `sim` and
 * zeroes the auxiliary fields of every simulation's layers.  Layers must
 * leave at least two interior cells in each direction and keep two coarse
 * cells from every embedded region (rom_embed checks the same later);
 * sources may not drive an edge next to a layer cell.  The storage function
 * (fdtd_energy) does not include the auxiliaries; fdtd_grad rejects a
 * context with layers.  fdtd_save_state / fdtd_load_state carry the
 * auxiliaries.  Host data is copied; synchronises the context's stream.
 * FDTD_EINVAL on a bad descriptor or placement. */
int fdtd_set_pml(fdtd_ctx* ctx, int sim, const fdtd_pml_desc* pml);

/* -------------------------------------------------------- frequency response */

/* Running DFT monitors of Hz (the paper reports its results as frequency
 * responses and reflected power, Sec. VI).  Sets nmon monitor cells
 * (fdtd_probe: sim, coarse cell i, j) and nfreq frequencies (Hz, finite,
 * >= 0) and sets the accumulators to acc_init ([nmon][nfreq][2] doubles
 * {Re, Im} as returned by fdtd_dft_get; NULL = zeros).  From then on every
 * time step n the context takes (fdtd_run, fdtd_run_host and the forward
 * pass of fdtd_grad; n counted from creation, as fdtd_get_step) adds
 *     X_m(f) += Hz^{n+1/2}(m) exp(-i 2 pi f (n + 1/2) dt) dt
 * in FP64 (fused into the probe step on the device).  nmon = 0 removes the
 * monitors.  Host arrays are copied.  FDTD_EINVAL for a monitor outside its
 * grid, a bad frequency or more than 2^24 monitor-frequency pairs.
 * Synchronises the context's stream.  While monitors are set the
 * two-steps-per-launch path is not used. */
int fdtd_dft_set(fdtd_ctx* ctx, const fdtd_probe* mons, int nmon, const double* freqs,
                 int nfreq, const double* acc_init);
/* Host copy of the accumulators: out[m][f] = {Re X_m(f), Im X_m(f)}
 * (2 nmon nfreq doubles; nothing is written when no monitors are set).
 * Synchronises the context's stream. */
int fdtd_dft_get(fdtd_ctx* ctx, double* out);

/* Fine-region fields of an embedded instance rebuilt from its state
 * (x_hat ~ V x~, Sec. III; output only, not part of the time march).
 * `model` must be the model the instance was embedded with (FDTD_EINVAL
 * otherwise).  Writes Ex [r b + 1][r a], Ey [r b][r a + 1], Hz [r b][r a]
 * (FP32, row-major, fine cell (0, 0) at the region's lower-left corner) to
 * caller-owned DEVICE buffers, on the context's stream, at the time levels of
 * the coarse fields (E^n, Hz^{n-1/2}).  The first call for a model keeps an
 * FP32 copy of its bases on the device (4 (nE qE + nH qH) bytes) until
 * fdtd_destroy. */
int fdtd_fine_fields(fdtd_ctx* ctx, int inst, const rom_model* model, float* Ex, float* Ey,
                     float* Hz);

/* ------------------------------------------------------------------ state */

/* Self-test of failure detection (no counterpart in the paper): launches a
 * kernel whose bounded wait on a barrier that nothing arrives at gives up
 * after a short limit and reports through the context's status word, the
 * same path the bulk-copy stencil uses; returns FDTD_ETIMEOUT when the path
 * works (FDTD_OK would mean the wait did not give up), and the context stays
 * usable.  Synchronises. */
int fdtd_selftest_timeout(fdtd_ctx* ctx);

/* Host copies of the current fields of one simulation (E^n, Hz^{n-1/2}). */
int fdtd_get_fields(fdtd_ctx* ctx, int sim, float* Ex, float* Ey, float* Hz);
/* Overwrites the fields; values on PEC walls and inside regions are
 * ignored (held at 0); interface values become each model's y. */
int fdtd_set_fields(fdtd_ctx* ctx, int sim, const float* Ex, const float* Ey,
                    const float* Hz);
/* Reduced state x~ (length q) of an embedded instance. */
int fdtd_get_rom_state(fdtd_ctx* ctx, int inst, float* x);
int fdtd_set_rom_state(fdtd_ctx* ctx, int inst, const float* x);
/* Number of steps taken since creation. */
int fdtd_get_step(const fdtd_ctx* ctx, long long* n);

/* Checkpoint / resume: the complete time-marching state (fields of every
 * simulation, every model's [y; x~], the step counter) as one host buffer.
 * fdtd_save_state with buf = NULL stores the required size in *size; with a
 * buffer of *size bytes it fills it.  fdtd_load_state restores a buffer saved
 * from a context with the same grids and embeddings (FDTD_EINVAL otherwise).
 * Continuing after save + load gives bit-identical results. */
int fdtd_save_state(fdtd_ctx* ctx, void* buf, size_t* size);
int fdtd_load_state(fdtd_ctx* ctx, const void* buf, size_t size);

/* Discrete storage function (Sec. V, Appendix A) of every simulation at the
 * current step, x = [E^n; Hz^{n-1/2}]:
 *   W = 1/2 E^T D_eps E + 1/2 H^T D_mu H - dt/2 E^T K H      (coarse system,
 *       interface edges on their coarse half cell, Eqs. (13)-(14))
 *     + dt/2 x~^T R~ x~                                      (each model, Eq. (12)).
 * Lossless and source-free, W is constant; with losses it does not
 * increase.  FP32 state, FP64 accumulation.  out: host double[nsim].
 * Returns FDTD_EUNSTABLE (after filling out) if some W is not finite.
 * Uses a device scratch buffer owned by the context (allocated on first
 * use).  Synchronises the context's stream. */
int fdtd_energy(fdtd_ctx* ctx, double* out);

/* fdtd_energy without any device allocation.  No counterpart in the paper:
 * this is a convenience for callers that must not allocate GPU memory at
 * this point -- for example code that runs while another framework's caching
 * allocator has reserved the free device memory, code that must not pay the
 * implicit synchronisation of cudaMalloc/cudaFree inside a time-critical
 * loop, or code that is about to record work into a CUDA graph.  The
 * per-block partial sums go to a fixed array in the library's device memory
 * (FDTD_ENERGY_STATIC_MAX doubles, 256 KB on every GPU that loads the
 * library, kept until the process exits) instead of a buffer owned by the
 * context; the result is the same as fdtd_energy's.
 *   - Capacity: the context's stencil tiles + embedded models + simulations
 *     must not exceed FDTD_ENERGY_STATIC_MAX; larger contexts get
 *     FDTD_EINVAL (use fdtd_energy).
 *   - The first call on a device looks up the array's device address once
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - The array is chosen by the CUDA device current when the call is made,
 *     so the context's device must be current (as for every call of this
 *     library, whose kernels run on the current device).
 *   - All calls in the process share the one array: calls whose GPU work
 *     overlaps (different contexts on different streams) race.  Every entry
 *     used is written before it is read, so nothing needs clearing.
 *   - out: host double[nsim].  Synchronises the context's stream. */
#define FDTD_ENERGY_STATIC_MAX 32768
int fdtd_energy_noalloc(fdtd_ctx* ctx, double* out);

/* ------------------------------------------------------------ measurement */

/* When on, fdtd_run launches every step directly (no CUDA graph) and records
 * CUDA events around each kernel on the context's stream; the device time of
 * the stencil kernel and of the reduced-model/probe kernel accumulates until
 * timing is switched on again (which resets it). */
int fdtd_set_timing(fdtd_ctx* ctx, int on);
/* Accumulated device time (ms) and launch counts; synchronises the stream.
 * On the two-steps-per-launch path (fdtd_steps_per_launch = 2) yee_ms is the
 * time of each two-step launch (the row-marching kernel with the model tiles
 * beside it, Eq. (5), Eq. (3) and Eq. (23) twice) and yee_launches counts
 * those launches; a trailing odd step is a one-step launch (stencil only, its
 * model step counted in post_ms). */
int fdtd_get_kernel_times(fdtd_ctx* ctx, double* yee_ms, long long* yee_launches,
                          double* post_ms, long long* post_launches);

/* Device time (ms) of one launch of the context's stencil kernel alone, for
 * roofline figures without per-kernel instrumentation: a CUDA graph of
 * `launches` back-to-back launches of the kernel fdtd_run uses for the
 * coarse update (the row-marching kernel when the context steps in pairs,
 * else the one-step kernel), without sources, probes or reduced models, is
 * replayed `reps` times between two CUDA events on the context's stream
 * (after one untimed replay); *ms_per_launch = elapsed / (reps * launches).
 * Every launch reads the current fields and writes the other copy of the
 * ping-pong pair, so the current state and the step counter are unchanged
 * (the other copy is overwritten by the next step anyway).  Synchronises.
 * FDTD_EINVAL for a bad argument or while fdtd_set_timing is on. */
int fdtd_time_stencil(fdtd_ctx* ctx, int launches, int reps, double* ms_per_launch);

/* Launch configuration chosen by fdtd_autotune. */
typedef struct {
  int steps_per_launch;    /* 1, or 2 (two steps per pass over the fields) */
  int tile_rows;           /* tile height of the one-step stencil */
  int march_rows;          /* tile height of the row-marching two-step kernel (0: unused) */
  int march_ring;          /* rows it stages ahead through shared memory (0: loads to registers) */
  int march_prefetch;      /* register loads: rows prefetched ahead, < 0 into L1, > 0 into L2 */
  int gemm_min;            /* simulations sharing a map from which it steps as a GEMM (0: fixed rule, 20) */
  int gemm_rows_per_warp;  /* GEMM CTA shape, 1 or 2 (0: fixed rule) */
  int chain;               /* two-step path, maps outside the zone tiles: 1 every model, 0 none,
                              -1 the maps shared by a GEMM group */
  int chained_models;      /* models stepped that way in the chosen plan */
  int candidates;          /* configurations timed (0: taken from the cache file) */
  double ms_default;       /* device ms per time step of the fixed rule */
  double ms_best;          /* ... and of the chosen configuration */
  int march_ctas;          /* resident CTAs per SM the row-marching kernel is built for, 4 or 3 (0: unused) */
} fdtd_tune_report;

/* Autotuner of the launch configuration (no counterpart in the paper): times
 * candidate configurations on the context itself and keeps the fastest for
 * the context's life.  The candidates are the choices that leave every
 * result bit-identical: one or two steps per launch, the tile heights of the
 * one-step and two-step kernels, the two-step kernel's resident CTAs per SM
 * (4 or 3) and how many rows it stages ahead or prefetches, where the
 * models' maps run on the two-step path, and from how many
 * sharing simulations (and with which CTA shape) a map runs as a GEMM.  Search: one pass of coordinate descent from the fixed
 * rule, each candidate marched from the current state with the source and
 * probe positions of the context's most recent fdtd_run / fdtd_run_host (the
 * sources at zero amplitude, the probe samples into a scratch buffer; none
 * before the first run), a few ms of steps timed with CUDA events on the
 * context's stream; a
 * candidate wins only if more than 1% faster.  The marching state (fields,
 * model states, step count, PML auxiliaries, DFT sums) is restored after
 * every candidate, so the context continues where it was.  cache_path (NULL:
 * the FDTD_TUNE_CACHE environment variable; neither: no cache) names a text
 * file holding one line per tuned problem, keyed by the device (name, SM
 * count, clock), the grids and the embedded models: a key found there is
 * applied without timing, a new result is appended.  report may be NULL.
 * Synchronises.  Call it again after embedding more models or setting
 * layers or monitors (those re-plan with the kept choices). */
int fdtd_autotune(fdtd_ctx* ctx, const char* cache_path, fdtd_tune_report* report);

/* The context's current launch configuration in the same form (candidates,
 * ms_default and ms_best are 0); no device work. */
int fdtd_get_plan(const fdtd_ctx* ctx, fdtd_tune_report* report);

/* Time steps one stencil launch of fdtd_run advances: 2 when the context
 * steps in pairs (temporal blocking: two steps of Eq. (5), Eq. (3) per pass
 * over the fields, each model's Eq. (23) evaluated between them in its own
 * tile; bit-identical to single steps), else 1.  Contexts with CPML layers
 * and runs with DFT monitors step singly.  FDTD_TB=0 / 1 in the environment
 * at context creation (kept for the context's life) forces one or the other
 * where the pair form applies; unset, pairs are used unless the slowest
 * model tile outlasts the pass over the cells or most strip rows hold only
 * the background material (re-decided whenever a model is embedded).
 * Returns FDTD_EINVAL for a null context. */
int fdtd_steps_per_launch(const fdtd_ctx* ctx);

const char* fdtd_last_error(const fdtd_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FDTD_ROM_H */
