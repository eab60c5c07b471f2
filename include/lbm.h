/*
 * lbm.h -- C ABI of the GB300 library for the compressible Navier-Stokes-Fourier
 * lattice Boltzmann scheme of Bukreev, Kummerlaender and Krause ("Lattice
 * Boltzmann Method for Compressible Navier-Stokes-Fourier Equations").
 *
 * One time step (lbm_step) updates every cell of a 3-D grid with
 *   - the zeroth moments Q_k of 14 D3Q7 population sets, one per component of
 *     Q = (rho, rho u, E, tau, q)                                     (Eq. 2, Sec. 2.2)
 *   - the closure p = (gamma-1)(E - rho|u|^2/2), T = p/rho and Sutherland's law
 *                                                                     (Sec. 2.1, Listing 1)
 *   - the cell-local shock sensor: dilatation from the cell's own moments,
 *     s = max(0, -div u)/c_s, chi, omega_h = omega - chi (omega - omega_min),
 *     omega = 1/tau_base, tau_base = 1/2 + 4 f_mu (mu/rho) dt/dx^2  (Sec. 2.3, Eqs. 3-6)
 *   - BGK collision toward the linear equilibrium feq_{k,i} = w_i (Q_k + c_i.Phi_k/c_s^2)
 *     with the source projected on the weights                       (Sec. 2.2)
 *   - streaming along the lattice characteristics, in place           (Sec. 1, Sec. 2.2)
 *
 * Conventions shared by every entry point:
 *   - Every call returns an lbm_status; no exception or abort crosses the ABI.
 *     On failure lbm_last_error() returns a message for the calling thread.
 *   - Fields are numbered k = 0 rho, 1-3 rho u, 4 E, 5-10 tau (xx yy zz xy xz yz),
 *     11-13 q; directions i = 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z.
 *   - Cell index = x + nx (y + ny z). Per-cell arrays are [field][z][y][x];
 *     population arrays are [k][i][z][y][x] in canonical order: the pre-collision
 *     populations of the current time step, independent of the in-place storage.
 *   - "dst_on_device"/"src_on_device" = 1: the pointer is device memory on the
 *     handle's device; 0: host memory (pageable or pinned). lbm_init_fields,
 *     lbm_init_state, lbm_moments and lbm_sensor read or write page-locked host
 *     memory (cudaHostAlloc, cudaHostRegister; element-aligned) directly from their
 *     kernels over the CPU-GPU link; pageable memory goes through a device staging
 *     buffer. The caller owns every buffer it passes in; the library owns the device
 *     memory it allocates.
 *   - Work is issued on the handle's CUDA stream (borrowed from the caller, or the
 *     legacy default stream when none is given). Calls that return data to the
 *     host synchronise that stream; lbm_step does not.
 *   - A handle is used by one host thread at a time.
 */
#ifndef LBM_H_
#define LBM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_handle lbm_handle;  /* one domain; opaque */
typedef struct lbm_batch lbm_batch;    /* many independent domains; opaque */

typedef enum {
  LBM_OK = 0,
  LBM_E_INVAL = 1,      /* bad argument or parameter */
  LBM_E_NOMEM = 2,      /* device or host allocation failed */
  LBM_E_CUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error), or
                           the handle's device could not be made current */
  LBM_E_NONFINITE = 4,  /* a non-finite moment was detected; sticky until re-init */
  LBM_E_STATE = 5,      /* call not valid in the current state (e.g. step before init) */
  LBM_E_IO = 6,         /* checkpoint file could not be read or written, or is corrupt */
  LBM_E_TIMEOUT = 7     /* a bounded wait inside a kernel ran out (a staged step's wait for its
                           own bulk copy): the state is incomplete; sticky until re-init */
} lbm_status;

/* Population storage. All arithmetic is FP32 in every mode.
 * F32: f - w_i Q_ref,k stored as float (the reference-shifted form of Sec. 2.2).
 * F16 / BF16: (f - w_i Q_ref,k) / s_k stored as IEEE half / bfloat16, rounded to
 * nearest even or stochastically (lbm_params.stochastic_round); s_k is fixed per
 * field at init (see lbm_info). */
typedef enum { LBM_STORE_F32 = 0, LBM_STORE_F16 = 1, LBM_STORE_BF16 = 2 } lbm_store;

/* Element types of data exchanged with the caller. NATIVE = the stored bits
 * (4 bytes for F32 storage, 2 bytes otherwise), in canonical order. */
typedef enum { LBM_DT_F32 = 0, LBM_DT_F64 = 1, LBM_DT_NATIVE = 2 } lbm_dtype;

/* Selector of lbm_moments. */
typedef enum {
  LBM_MOM_Q = 0,     /* the 14 zeroth moments Q_k */
  LBM_MOM_PRIM = 1   /* rho, u_x, u_y, u_z, T, p */
} lbm_moment_set;

/* Parameters of one domain (Table 1 and Sec. 2.1-2.3 of the paper). */
typedef struct {
  int nx, ny, nz;        /* cells per axis, each >= 1; nx*ny*nz < 2^31 */
  int bc_x;              /* 0: periodic in x; 1: x ends held at the initial state
                            (ghost layers keep the initial populations of the boundary
                            cells; only their inward populations enter). y, z periodic. */
  double dx;             /* lattice spacing, > 0 */
  double dt;             /* > 0: time step; <= 0: dt = cfl * dx / (2 lambda_ref), i.e. the
                            acoustic Courant number taken against c_s = c/2 (Table 1) */
  double cfl;            /* acoustic Courant number (Table 1) */
  double lambda_ref;     /* largest signal speed |u| + a of the problem, > 0 if dt <= 0 */
  double gamma;          /* adiabatic index, > 1 */
  double mu, kappa;      /* viscosity and conductivity (reference values if Sutherland) */
  double tau_R, tau_q;   /* relaxation times of tau and q (Eq. 2), > 0 */
  double T_ref;          /* Sutherland reference temperature, > 0 */
  int relax_in_dt;       /* 1: tau_R, tau_q are given in units of dt (Sec. 3.1) */
  int sutherland;        /* 1: mu_T = mu (1 + T_S) t^{3/2} / (t + T_S), t = T/T_ref,
                            T_S = 0.4042, kappa_T = kappa mu_T/mu (Listing 1); 0: constant */
  int source_mode;       /* 0: w_i dt S_k (explicit); 1: w_i (exp(-dt/tau) - 1) Q_k */
  double f_mu;           /* background dissipation factor of Eq. 6, >= 0 */
  double C_sigma;        /* sensor slope (Eq. 4), >= 0 */
  double J_min;          /* sensor threshold on s (Eq. 4), >= 0 */
  double omega_min;      /* floor of the blended rate (Eq. 5), in (0, 2] */
  int sensor_mode;       /* 0: div u = (div(rho u) - u.grad rho)/rho from the cell's
                            non-equilibrium moments; 1: div(rho u)/rho only */
  int collide;           /* 1: collide and stream; 0: stream only (tests) */
  int store;             /* lbm_store */
  int stochastic_round;  /* 16-bit storage only: 1 rounds every stored population up or
                            down at random with the probabilities that make the rounding
                            unbiased (random bits from the cell's index and state, so the
                            result is reproducible); 0 rounds to nearest (default). The
                            staged kernel forms round to nearest only; a batch takes one
                            mode for all its domains */
  int use_graphs;        /* 1: lbm_step replays captured CUDA graphs of whole step pairs */
  int streaming;         /* in-place form of the streaming along the lattice links (Sec. 1,
                            Sec. 2.2), one population buffer either way (no counterpart in
                            the paper, which leaves the memory layout open):
                            0: AA pattern (default): even steps read and write the cell's
                               own slots, odd steps the slots of its six neighbours;
                            1: esoteric twist: the slots of the -x, -y, -z directions are
                               stored with the cell one step along +x, +y, +z, so every
                               step reads and writes the own cell and one slot of each of
                               the neighbours x + e_x, x + e_y, x + e_z. The stored buffer
                               is a fixed permutation of the AA buffer and every result
                               (populations in canonical order, moments, diagnostics,
                               checkpoints) is the same bit for bit. The staged variants
                               and lbm_plane_get/set return LBM_E_INVAL under it; a batch
                               takes one map for all its domains. */
  void* cuda_stream;     /* cudaStream_t to issue work on (borrowed), or NULL */
  void* pop_buffer;      /* optional device buffer of lbm_population_bytes() bytes,
                            256-byte aligned, borrowed for the handle's lifetime; NULL:
                            the library allocates it */
} lbm_params;

/* Read-only facts of a handle. */
typedef struct {
  double dt, c;             /* time step and lattice speed dx/dt */
  double tau_R, tau_q;      /* relaxation times in use (after relax_in_dt) */
  double rho_ref, E_ref;    /* reference shift Q_ref (other components 0) */
  double scale[14];         /* per-field storage scale s_k (1 for F32/BF16) */
  long long step;           /* steps taken since the last init */
  long long ncell;
  size_t population_bytes;  /* bytes of the population buffer */
  int store;
  int block_x;              /* threads per block of the step kernel */
  int variant;              /* form of the step kernel: 0 = plain loads, 3 blocks of 128
                               threads per SM (<= 170 registers); 1 = plain loads, 4 blocks
                               (<= 128 registers); 2, 3, 4 = reads staged through shared
                               memory by bulk asynchronous copies, a persistent grid of
                               4-warp blocks: 2 stages per warp with <= 170 registers (2),
                               2 stages with <= 128 (3), 3 stages with <= 170 (4) */
  int prefetch_tiles;       /* L2 prefetch distance of variants 0 and 1 on whole-tile rows
                               (see lbm_set_prefetch); 0 = off */
  int device;               /* CUDA device ordinal the handle is bound to (see lbm_create) */
} lbm_info_t;

/* Diagnostics (Sec. 3.2, Eq. 7). Sums and extrema in FP64 over all cells.
 * Velocity gradients by second-order central differences (periodic; one-sided
 * at held x ends); mu_local follows the domain's viscosity law. */
typedef struct {
  double step, time;
  double sum_rho, sum_mx, sum_my, sum_mz, sum_E;  /* sum over cells of Q_k */
  double ek_mean;       /* <rho |u|^2 / 2> */
  double eps_s_raw;     /* <mu_local |curl u|^2>; eps_s of Eq. 7 = eps_s_raw / rho_ref */
  double eps_d_raw;     /* 4/3 <mu_local (div u)^2>; eps_d = eps_d_raw / rho_ref */
  double max_mach;      /* max |u| / sqrt(gamma T) */
  double max_cfl;       /* max over cells and axes of (|u_a| + a) dt / dx */
  double min_rho, min_T;
  double nonfinite;     /* cells with a non-finite zeroth moment */
} lbm_diag_t;

/* Kernel configuration chosen by the autotuner. */
typedef struct {
  int block_x;          /* threads per block of the step kernel */
  int variant;          /* register budget (see lbm_info_t) */
  float ms_per_step;    /* measured time of one step with that configuration */
  int candidates;       /* configurations timed */
  int prefetch_tiles;   /* L2 prefetch distance chosen (0 = off) */
} lbm_tune_t;

/* ---- lifecycle -------------------------------------------------------------- */

/* Bytes of the population buffer for these parameters: ceil(cells / 32) tiles of
 * 98 x 32 elements of the storage type (tiled SoA: a tile holds the 98 arrays
 * (field, direction) of 32 consecutive cells). Returns 0 if the sizes are invalid. */
size_t lbm_population_bytes(const lbm_params* p);

/* Validates *p (LBM_E_INVAL with the reason), derives dt and the relaxation
 * times, allocates the device state on the current CUDA device (LBM_E_NOMEM if it
 * does not fit) and returns an uninitialised handle in *out. The state is one
 * population buffer updated in place; nothing of size O(cells) is allocated
 * besides it until lbm_diag is first called. The handle is bound to that device
 * (lbm_info_t.device): every later call on it makes the device current while it
 * runs and restores the caller's current device before returning, so one thread can
 * drive handles on several GPUs. cuda_stream and pop_buffer must belong to it. */
lbm_status lbm_create(const lbm_params* p, lbm_handle** out);

/* Releases everything the handle allocated (not borrowed buffers or streams).
 * Waits for the handle's pending work. NULL is accepted. */
lbm_status lbm_destroy(lbm_handle* h);

/* Message of the last failed call made by this thread ("" if none). */
const char* lbm_last_error(void);

/* Name of a status code. */
const char* lbm_status_string(lbm_status s);

lbm_status lbm_get_info(const lbm_handle* h, lbm_info_t* out);

/* ---- initial states (Sec. 3) --------------------------------------------------
 * Each sets every cell's populations to the linear equilibrium of its state with
 * zero stress and heat flux (tau = q = 0), resets the step counter and the
 * non-finite flag, records the held-x ghost populations, and fixes the storage
 * reference Q_ref and (F16) the per-field scales s_k = max|f - w Q_ref| / 1024.
 * A state that is not finite in some cell gives LBM_E_INVAL and leaves the handle
 * uninitialised. */

/* Supersonic Taylor-Green vortex of Sec. 3.2 on a box of side nx*dx = 2 pi L:
 * u = U0 sin x cos y cos z, v = -U0 cos x sin y cos z, w = 0,
 * p = p0 + rho0 U0^2/16 (cos 2x + cos 2y)(cos 2z + 2), p0 = rho0 U0^2/(gamma M0^2),
 * uniform T0 = p0/rho0, rho = p/T0. Node (x,y,z) of cell (i,j,l) = (i,j,l) dx.
 * Q_ref = (rho0, 0, 0, 0, p0/(gamma-1)). */
lbm_status lbm_init_tgv(lbm_handle* h, double U0, double M0, double rho0);

/* Riemann problem along `axis` (0,1,2): cells with index < i_split take
 * left = (rho, u_axis, p), the others right. Q_ref = right state. */
lbm_status lbm_init_riemann(lbm_handle* h, int axis, int i_split, const double left[3],
                            const double right[3]);

/* Equilibrium from caller fields [5][cells] = rho, u_x, u_y, u_z, p in `dtype`
 * (LBM_DT_F32 or LBM_DT_F64) on the host or the device. Q_ref = (mean rho, 0, 0, 0,
 * mean of p/(gamma-1) + rho|u|^2/2), the means taken over every cell of domains of up
 * to 2^20 cells and, for larger ones, over a fixed sample of about 2^20 cells (every
 * s-th run of 32 consecutive cells, s = floor(runs / 2^15)): the storage only needs a
 * reference near the data, and the sample saves a second full read of the fields. */
lbm_status lbm_init_fields(lbm_handle* h, const void* fields, int src_on_device, int dtype);

/* Equilibrium from caller zeroth moments [14][cells] (rho, rho u, E, tau, q; the
 * field order above) in `dtype` on the host or the device, e.g. a state whose stress
 * and heat flux start at their Newtonian and Fourier values (Becker's shock,
 * Sec. 3.1). Q_ref = (mean rho, 0, 0, 0, mean E), means as for lbm_init_fields. */
lbm_status lbm_init_state(lbm_handle* h, const void* Q, int src_on_device, int dtype);

/* ---- the hot path ------------------------------------------------------------ */

/* Advances n >= 0 time steps: per step one fused kernel reads each cell's 98
 * populations (AA pattern: own slots on even steps, the neighbours' slots on odd
 * steps; esoteric twist: own slots and one slot of each of the +x, +y, +z
 * neighbours on every step; lbm_params.streaming), computes moments, closure,
 * sensor and collision in FP32 and writes the 98 post-collision populations back
 * in place, so that streaming happens through the index maps. Asynchronous on the handle's stream. Returns LBM_E_STATE before
 * an init, LBM_E_NONFINITE if an earlier synchronising call saw non-finite
 * moments (no work is issued then). */
lbm_status lbm_step(lbm_handle* h, int n);

/* Waits for the handle's stream; then reports LBM_E_NONFINITE if any step since
 * the last init produced a non-finite moment (the flag is sticky). */
lbm_status lbm_synchronize(lbm_handle* h);

/* ---- outputs ------------------------------------------------------------------- */

/* Per-cell moments of the current (pre-collision) state: `which` = LBM_MOM_Q
 * (14 fields) or LBM_MOM_PRIM (6 fields: rho, u_x, u_y, u_z, T, p), as
 * [field][z][y][x] in `dtype` (LBM_DT_F32 or LBM_DT_F64), into dst on the host or
 * device. Populations are decoded in FP32 as the step decodes them; Q is a
 * float-float sum (about 48 significant bits) of the seven populations and the
 * reference; the primitives are exactly the step's own (its FP32 sums and closure).
 * Synchronises when dst is on the host (through a device staging buffer the handle
 * keeps, 256 MB, allocated on first use). */
lbm_status lbm_moments(lbm_handle* h, int which, void* dst, int dst_on_device, int dtype);

/* Sensor of the current state, [3][z][y][x]: theta = div u (physical units),
 * chi (Eq. 4) and omega_h (Eq. 5), exactly as the next step computes them (FP32
 * arithmetic), written in `dtype` (F32 or F64). */
lbm_status lbm_sensor(lbm_handle* h, void* dst, int dst_on_device, int dtype);

/* FP64 reductions of Eq. 7 and conservation sums into *out (host). Allocates
 * O(cells) device scratch on first use (kept until destroy). Synchronises. Also
 * latches LBM_E_NONFINITE for later lbm_step calls when a non-finite moment is
 * found (returned by this call as well, after *out is filled). */
lbm_status lbm_diag(lbm_handle* h, lbm_diag_t* out);

/* Advances n >= 1 time steps like lbm_step, and the first of them also computes
 * the diagnostics of the state it starts from (Sec. 3.2, Eq. 7; the values lbm_diag
 * would return just before this call, with the same per-cell arithmetic) inside the
 * step kernel, from the registers that hold the cell's moments, instead of a
 * separate pass over the populations. Besides the populations, that step writes u
 * and mu_local (16 bytes per cell) and one record per warp (13 doubles per 32 cells);
 * a short reduction follows. Allocates the same scratch as lbm_diag plus the
 * records on first use. Blocks the calling thread until the diagnostics are in
 * *out (host); the other n - 1 steps stay queued, asynchronous, as with lbm_step.
 * Sums may differ from lbm_diag's in the last bits (another summation order);
 * extrema, counts and the dissipation integrals are identical. Errors as lbm_step;
 * also returns LBM_E_NONFINITE (after filling *out) when the state had non-finite
 * moments, and latches it. */
lbm_status lbm_step_diag(lbm_handle* h, int n, lbm_diag_t* out);

/* lbm_diag without any memory allocation (no counterpart in the paper; a service
 * for callers that cannot allocate device memory when they sample diagnostics,
 * for example because a memory pool already holds the free device memory or
 * because cudaMalloc's device-wide synchronisation is not acceptable there).
 * Same results as lbm_diag. Its scratch is a fixed device array inside the
 * library (about 4.2 MiB on every device that loads the library, kept until the
 * process exits), so it handles domains of at most 262144 cells (64^3) and returns
 * LBM_E_INVAL for larger ones. The first call on a device looks up the array's
 * device address (with the handle's device made current) and keeps it; make that
 * first call before any stream capture (the kept address does not survive
 * cudaDeviceReset). Calls share the array: two calls whose kernels overlap on the
 * GPU race, so serialise them. Synchronises the handle's stream. */
lbm_status lbm_diag_static(lbm_handle* h, lbm_diag_t* out);

/* Canonical populations [k][i][z][y][x] in `dtype`: F64/F32 = the physical f
 * (decoded), NATIVE = the stored bits. */
lbm_status lbm_populations_get(lbm_handle* h, void* dst, int dst_on_device, int dtype);

/* Replaces the state with canonical populations in `dtype` (F64/F32 are encoded
 * into the storage type; NATIVE is copied bit for bit). With held x ends the
 * inward populations of the boundary cells stay those of the ghost layer. Marks
 * the handle initialised; the step counter is kept. A handle never initialised
 * gets Q_ref = 0 and s_k = 1. */
lbm_status lbm_populations_set(lbm_handle* h, const void* src, int src_on_device, int dtype);

/* ---- checkpoint ---------------------------------------------------------------- */

/* Writes the parameters, step counter, storage reference and scales, ghost
 * layers and the raw population buffer (canonical order) to `path` with a CRC-32;
 * lbm_load restores them into a handle with the same sizes and storage
 * (LBM_E_INVAL otherwise, LBM_E_IO on a bad file). Resuming is bit-identical, also
 * from a handle with the other streaming map (the file holds canonical order). */
lbm_status lbm_save(lbm_handle* h, const char* path);
lbm_status lbm_load(lbm_handle* h, const char* path);

/* ---- tuning ------------------------------------------------------------------- */

/* Times the step kernel for each candidate form (variants 0 and 1 at blocks of 64
 * and 128 threads, each with L2 prefetch distances 0, 512, 1024 and 2048 tiles on
 * whole-tile rows: at most 16 candidates; the staged variants 2-4, measured slower
 * everywhere, only through lbm_set_kernel_config) on whole step pairs with CUDA events
 * on the handle's stream, and keeps the fastest in the handle; returns it in *out if
 * out != NULL. Needs an initialised state
 * (LBM_E_STATE otherwise); each candidate runs on the live state, so the state
 * advances by an even number of steps: re-init before the run you keep. */
lbm_status lbm_autotune(lbm_handle* h, int pairs_per_trial, lbm_tune_t* out);

/* Fixes the step kernel's form (variant 0-4, see lbm_info_t) and, for variants 0 and
 * 1, its block size (32, 64, 96 or 128 threads; ignored by the staged variants)
 * instead of the defaults or the autotuner's choice. The staged variants need a
 * periodic x axis, nx a multiple of 32 (whole 32-cell tiles per row), rounding to
 * nearest and the AA maps (streaming 0) (LBM_E_INVAL otherwise). All forms compute
 * bit-identical populations. A staged step whose wait
 * for a copy runs out (bounded; it does not happen in normal operation) stops,
 * reports LBM_E_TIMEOUT from the next synchronising call and refuses further steps
 * until a re-init. */
lbm_status lbm_set_kernel_config(lbm_handle* h, int block_x, int variant);

/* Sets the L2 prefetch distance of the plain step kernel (variants 0 and 1) on
 * domains of whole 32-cell tile rows (periodic x, nx a multiple of 32): the warp
 * updating tile t first asks L2, with one bulk prefetch per slot run, for the slot
 * blocks that the warp on tile t + tiles will read, so that warp's loads meet L2
 * instead of DRAM (an implementation choice; the paper has no counterpart). 0 turns
 * it off; held-x domains, other row lengths and the staged and batched forms ignore
 * it. The default is 1024 tiles for 16-bit storage and 0 for FP32; lbm_autotune
 * chooses among 0, 512, 1024 and 2048. Populations are bit-identical with any
 * distance. LBM_E_INVAL for tiles < 0 or > 2^20 or a NULL handle. */
lbm_status lbm_set_prefetch(lbm_handle* h, int tiles);

/* Failure-detection test hook (no counterpart in the paper). With a staged kernel form
 * (variant 2-4), the next step does not issue the bulk copy of the first tile of one
 * warp (block 0, warp 0), so that warp's bounded wait for it runs out after about a
 * second; nothing faults or hangs. The step then ends early and the next
 * synchronising call (lbm_synchronize, lbm_diag) returns LBM_E_TIMEOUT, after which
 * lbm_step refuses to run until a re-init. LBM_E_INVAL for a plain form. */
lbm_status lbm_test_skip_copy(lbm_handle* h);

/* Memory-safety test hook (no counterpart in the paper; a stand-in for a GPU memory
 * checker). A build compiled with LBM_CHECKED tests every population tile and ghost
 * address its kernels form against the buffer before using it; an address outside
 * adds 1 to a per-handle (per-batch) count and the access is dropped (a load reads
 * zero) instead of faulting. These calls return that count, accumulated since
 * create, in *count (synchronising the stream). Other builds set *count = 0 and return
 * LBM_E_STATE. LBM_E_INVAL for a NULL argument. */
lbm_status lbm_check_count(const lbm_handle* h, unsigned long long* count);
lbm_status lbm_batch_check_count(const lbm_batch* b, unsigned long long* count);

/* Codec test hook: the 16-bit store conversion of the step kernels (the encoding of the
 * reference-shifted deviations of Sec. 2.2 into FP16 or BF16; no counterpart in the
 * paper, which stores FP32) applied at unit scale to npair pairs of floats:
 * in[2j] -> low half and in[2j+1] -> high half of out[j]. stochastic_round 0 rounds to
 * nearest even; 1 rounds stochastically with the random word rbits[j] (its low 16 bits
 * serve in[2j], its high 16 bits in[2j+1]; as in the kernels). store: LBM_STORE_F16 or
 * LBM_STORE_BF16. in (2*npair floats), rbits (npair words; unused and may be NULL when
 * rounding to nearest) and out (npair words) are DEVICE pointers owned by the caller;
 * the work is queued on cuda_stream (a cudaStream_t, NULL for the default stream) and
 * the call does not wait for it. LBM_E_INVAL for another store, a stochastic_round
 * other than 0 or 1, npair outside 0..2^30 or a NULL buffer (checked before any CUDA
 * call); LBM_E_CUDA if the launch fails. */
lbm_status lbm_test_encode(int store, int stochastic_round, const float* in,
                           const unsigned* rbits, unsigned* out, long long npair,
                           void* cuda_stream);

/* ---- z-slab decomposition ------------------------------------------------------ */

/* One domain split into z-slabs, one handle per slab (no counterpart in the paper,
 * which runs one domain). Each slab handle is periodic in z on its own; D3Q7 moves
 * populations only along the axes, so neighbouring slabs couple through the two
 * z-moving populations of their boundary planes alone. These two calls move the raw
 * stored values (element bits, no decoding) of storage slot `slot` (0 rest, 1 +x,
 * 2 -x, 3 +y, 4 -y, 5 +z, 6 -z) of all 14 fields on plane z, as [k][y][x]: 14 * nx * ny
 * elements of 4 bytes (F32) or 2 bytes (F16, BF16), to or from `buf` on the host or
 * the device. Slots are those of the AA layout (after an even number of steps slot i
 * of cell x holds f_i(x)). paper_2608_13437_gb300/slab.py holds the exchanges, before
 * and after each odd step, that make a ring of slab handles step exactly like the
 * whole domain; the handles must share Q_ref and the storage scales. Asynchronous on
 * the handle's stream for device buffers, synchronous for host buffers.
 * LBM_E_INVAL for z outside [0, nz), slot outside [0, 7), a NULL buffer or a handle
 * under the esoteric twist (streaming 1). */
lbm_status lbm_plane_get(lbm_handle* h, int z, int slot, void* dst, int dst_on_device);
lbm_status lbm_plane_set(lbm_handle* h, int z, int slot, const void* src, int src_on_device);

/* ---- many independent domains (batched mode) -------------------------------------
 * n periodic domains with their own sizes and parameters (one storage type for all,
 * F32, F16 or BF16), stored in one buffer on the device current at lbm_batch_create,
 * to which the batch is bound as a handle is (see lbm_create). lbm_batch_step advances all of them by one step per persistent launch
 * (grid = the resident blocks of the GPU; each warp takes items of consecutive
 * 32-cell tiles across all domains and keeps the constants of the domain it works on
 * in a slot of shared memory of its own),
 * replayed from a CUDA graph; lbm_batch_step_sequential issues one plain launch per
 * domain per step instead. Both give bit-identical populations. Items per warp,
 * block size and register budget come from lbm_batch_autotune. At most 65535
 * domains per batch, and each domain's nx at most 65535 (the per-tile records hold
 * 16-bit domain indices and coordinates); LBM_E_INVAL otherwise, before any CUDA
 * call. */
lbm_status lbm_batch_create(int n, const lbm_params* params, lbm_batch** out);
lbm_status lbm_batch_destroy(lbm_batch* b);
/* Per-domain TGV parameters, arrays of n values (host). */
lbm_status lbm_batch_init_tgv(lbm_batch* b, const double* U0, const double* M0,
                              const double* rho0);
lbm_status lbm_batch_step(lbm_batch* b, int n);
lbm_status lbm_batch_step_sequential(lbm_batch* b, int n);
lbm_status lbm_batch_synchronize(lbm_batch* b);
/* lbm_moments of one domain. */
lbm_status lbm_batch_moments(lbm_batch* b, int domain, int which, void* dst, int dst_on_device,
                             int dtype);
/* lbm_diag of one domain of the batch (the same FP64 reductions of Eq. 7 and the
 * conservation sums, from the same kernels). Allocates O(cells of the largest domain)
 * of device scratch on first use (kept until destroy). Synchronises. LBM_E_INVAL for a
 * bad domain index, LBM_E_STATE before an init, LBM_E_NONFINITE (after filling *out)
 * when a non-finite moment was found; it then latches for lbm_batch_step. */
lbm_status lbm_batch_diag(lbm_batch* b, int domain, lbm_diag_t* out);
/* Total cells of all domains; time step of one domain. */
lbm_status lbm_batch_info(const lbm_batch* b, long long* total_cells, int domain, double* dt);
/* Times items per warp (1, 2, 4, 8, 16, 32 tiles of 32 cells) x block sizes x register
 * budgets of the persistent kernel at the current L2 prefetch distance, then the
 * distances 0, 512, 1024 and 2048 tiles for the fastest of those, and keeps the
 * fastest; reports the cells per item, the block size, the time per step and the
 * prefetch distance (each pointer may be NULL). Advances the state like lbm_autotune. */
lbm_status lbm_batch_autotune(lbm_batch* b, int steps_per_trial, int* tile_cells,
                              int* block_threads, float* ms_per_step, int* prefetch_tiles);
/* L2 prefetch distance of the persistent kernel, in tiles (an implementation choice;
 * the paper has no counterpart): a warp starting an item asks L2 for the slot blocks
 * of the item that many tiles ahead in the claim order, in the pattern of
 * lbm_set_prefetch. 0 turns it off; the default is 1024 for 16-bit storage and 0 for
 * FP32. Populations are bit-identical with any distance. LBM_E_INVAL for tiles < 0 or
 * > 2^20 or a NULL batch. */
lbm_status lbm_batch_set_prefetch(lbm_batch* b, int tiles);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H_ */
