/*
 * lesbgk.h -- C ABI of the GB300 lattice ES-BGK solver (liblesbgk.so).
 *
 * The method is the lattice ellipsoidal-statistical BGK model of Meng, Zhang,
 * Hadjiconstantinou, Radtke & Shan (arXiv 1209.6548):
 *
 *   f_a(n+1) = f_a - (c_ax dt/dx)[F_{i+1/2} - F_{i-1/2}]
 *                  - (c_ay dt/dy)[F_{j+1/2} - F_{j-1/2}]
 *                  + (dt/tau)(f_ES,a - f_a) + dt g_a                 (Sec. 3.1)
 *
 * on a tensor-product Gauss-Hermite velocity set (Sec. 2.2, Eq. weight), with
 * f_ES the Hermite expansion of the anisotropic Gaussian (Eq. cfeq, a_ES^(n)
 * of Sec. 2.2) to order N, tau = (Kn/Pr) mu/p with Pr = 1/(1-b) and
 * mu = T^varpi (Sec. 2.1-2.2), second-order TVD fluxes with the minmod
 * limiter (Sec. 3.1), the projected body force (Sec. 2.2) and fully diffuse
 * walls (Sec. 3.2, Eq. feq0).
 *
 * Conventions (non-dimensional units of Sec. 2.2: R = T0 = rho0 = L = 1):
 *   - D = 2 (the lattice dimension) in T, in Eq. (feq0) and in Pr.
 *   - Velocity index a = ix*nroots + iy, c_a = (c_ix, c_iy), the 1D roots of
 *     He_nroots sorted ascending.
 *   - Grid nx x ny nodes, x periodic.  bc_y = LESBGK_PERIODIC, or
 *     LESBGK_DIFFUSE with walls on nodes j = 0 (bottom, inward normal +y) and
 *     j = ny-1 (top); ghost rows beyond a wall hold the wall node's values.
 *   - Spacing: periodic y: dx = 1/nx, dy = 1/ny; walls: dy = 1/(ny-1), dx = dy.
 *   - Populations are stored as deviations f_a - w_a (w_a the quadrature
 *     weight, i.e. the rest equilibrium at rho0 = 1, T0 = 1), layout
 *     [a][j][i] (a-major, then row j, then column i), float32.
 *
 * Memory: the caller owns every device buffer.  lesbgk_workspace_size tells
 * how many bytes of device memory one solve needs; the caller allocates them
 * (e.g. a torch uint8 tensor) and passes the pointer to lesbgk_create, and
 * keeps them alive until lesbgk_destroy.  The library allocates no device
 * memory.  Every call is asynchronous on the given CUDA stream (a
 * cudaStream_t passed as void*; NULL = legacy default stream) except where
 * a host output is written, which synchronises that stream.
 *
 * Errors: every function returns 0 on success or a negative LESBGK_E* code;
 * lesbgk_last_error() returns a thread-local message for the last failure.
 * The library never aborts and has no CPU fallback.
 */
#ifndef LESBGK_H
#define LESBGK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LESBGK_OK 0
#define LESBGK_EINVAL (-1)    /* invalid argument */
#define LESBGK_EUNSTABLE (-2) /* CFL > 1, or explicit dt with dt/tau_ref >= 2 */
#define LESBGK_ESPACE (-3)    /* workspace too small or misaligned */
#define LESBGK_ECUDA (-4)     /* CUDA error (message in lesbgk_last_error) */
#define LESBGK_EDIVERGED (-5) /* NaN/Inf found in the moments */

#define LESBGK_PERIODIC 0
#define LESBGK_DIFFUSE 1

/* Population storage (compute is always FP32).  LESBGK_F32 stores the
 * deviation f_a - w_a; LESBGK_F16 and LESBGK_BF16 store the relative deviation
 * (f_a - w_a)/w_a (times 2^10 in FP16, to stay in its normal range), halving
 * the bytes per lattice update.  Each step's stores round stochastically
 * (the hardware's unbiased stochastic rounding, fed random words from a
 * counter-based hash of the step, the row and the population group -- not the
 * column, so a flow uniform in x stays uniform -- hence reproducible and
 * independent of the launch shape); initial and set populations round to
 * nearest.  16-bit storage is
 * built for the default orders (D2Q16 N = 3, D2Q36 N = 4) and D3Q64. */
#define LESBGK_F32 0
#define LESBGK_F16 1
#define LESBGK_BF16 2
/* Compensated FP32 storage (not in the paper; FP32 compute): each deviation
 * f_a - w_a is held as hi + lo, hi in FP32 and lo, the remainder FP32 cannot
 * hold, in FP16 (stored as lo 2^24 / w_a), 6 bytes per value.  Every step
 * adds its increment to hi + lo exactly (an error-free two-sum) and the TVD
 * differences take both parts, so the storage rounding per step falls from
 * half an FP32 ulp to 2^-11 of it: a solve of many small steps (dt/tau ~ 1e-3,
 * where the relaxation barely damps accumulated rounding) keeps its stress
 * and heat flux to the precision FP32 arithmetic gives one step.  1.5 times
 * the bytes of FP32 storage.  Built for D2Q16 and D3Q64 (order 3) with
 * periodic or fully diffuse steady or heated y-walls. */
#define LESBGK_F32C 3

/* Advection schemes.  LESBGK_UNSPLIT is the update of Sec. 3.1 as printed:
 * both flux differences are taken from f^n.  For flows that vary in both x
 * and y that sum of two one-dimensional second-order operators has an
 * amplification factor above 1 at every Courant number (the paper only runs
 * flows uniform in x, where it is exact); LESBGK_SPLIT takes the y-sweep
 * first, f* = f^n - (c_y dt/dy)[F_{j+1/2} - F_{j-1/2}](f^n), then the x-fluxes
 * of f*, with collision and force from f^n.  For flows uniform in x the two
 * give the same update. */
#define LESBGK_UNSPLIT 0
#define LESBGK_SPLIT 1

typedef struct lesbgk_params {
  uint32_t struct_size; /* sizeof(lesbgk_params), checked */
  int32_t nroots;       /* Gauss-Hermite roots per axis: 4 (D2Q16, D3Q64) or 6 (D2Q36, D3Q216) */
  int32_t order;        /* Hermite order N of f_ES (3 or 4); 0 = 3 for D2Q16, 4 for D2Q36 */
  int32_t nx, ny;       /* nodes; nx >= 1; ny >= 1 (>= 2 with walls); nx ny < 2^31 */
  int32_t bc_y;         /* LESBGK_PERIODIC or LESBGK_DIFFUSE (walls on rows j = 0 and ny-1) */
  int32_t storage;      /* LESBGK_F32, LESBGK_F16, LESBGK_BF16 or LESBGK_F32C */
  int32_t scheme;       /* LESBGK_UNSPLIT (default) or LESBGK_SPLIT */
  double kn;            /* Knudsen number of Sec. 2.2, > 0 */
  double b;             /* ES parameter, -1/2 <= b < 1 (b = 1 gives tau = 0) */
  double visc_exp;      /* varpi in mu = T^varpi (0.5 hard sphere, 1 Maxwell) */
  double cfl;           /* used when dt == 0: dt = min(cfl min(dx,dy)/c_max, tau_ref) */
  double dt;            /* explicit time step, or 0 */
  double wall_T[2];     /* wall temperatures, [0] = bottom (j=0), [1] = top */
  double wall_ux[2];    /* wall x-velocities (walls do not move in y) */
  double g[2];          /* body force (g_x, g_y) */
  double wall_specular; /* Maxwell wall model (Sec. 3.2): fraction 1 - gamma of the outgoing half
                           re-emitted specularly; 0 = fully diffuse (the paper's runs) */
  double wall_T_amp;    /* wall heating (Sec. 4.2): T_w(t) = wall_T + wall_T_amp sin(wall_T_freq t) */
  double wall_T_freq;   /* (St in the units of Sec. 2.2); amp 0 = steady walls.  The wall
                           tables are FP64 polynomials in the heating, evaluated for each
                           step's time (the same bits on the host for lesbgk_step and on
                           the device in the batched solver).  Specular fractions need
                           FP32 storage; heating takes any storage. */
  int32_t dim;          /* dimension D of the velocity set: 0 or 2 = the 2D sets above;
                           3 = D3Q64 (nroots 4, order 3; any storage) or D3Q216 (nroots 6,
                           order 4, the paper's 11th-order set; FP32, FP16 or BF16), on the same 2D grid: the
                           paper's D = 3 thermodynamics (C_p = 5/2; Sec. 2.1, Sec. 4).
                           Nothing varies in z and walls and forces have no z part, so the
                           state stays even in c_z: the library stores the c_z > 0 half
                           (Q = nroots^3/2 values per node, population
                           a = (iz*nroots + ix)*nroots + iy, c_z = c[nroots/2 + iz]), each
                           value standing for +c_z and -c_z.  T = tr P/(3 rho) and sigma is
                           trace-free in 3D in the moments.  */
  int32_t bc_x;         /* LESBGK_PERIODIC (default) or LESBGK_DIFFUSE: fully diffuse walls at rest
                           on columns i = 0 and nx-1 (not in the paper, whose flows are uniform
                           in x), at temperatures wall_Tx; ghost columns hold the wall node.
                           With walls in y as well the domain is a cavity (the unit square,
                           dx = 1/(nx-1), dy = 1/(ny-1)) whose lid is the top wall (wall_ux[1]);
                           a corner node belongs to both walls: the populations arriving
                           towards both walls are kept, the others re-emitted as rho_W S(T_wx,
                           u = 0) with zero net mass flux along n_x + n_y.  With walls in x only,
                           dy = dx = 1/(nx-1).  FP32, FP16 or BF16 storage, fully diffuse y-walls. */
  double wall_Tx[2];    /* x-wall temperatures, [0] = left (i = 0), [1] = right (i = nx-1) */
  double dx, dy;        /* grid spacing; 0, 0 = derived from the grid and walls as described above.
                           Explicit values (both > 0) serve a y-slab of a larger domain, which
                           runs as a solver of its own on the slab's rows plus halo rows and
                           keeps the whole domain's spacing (pass the whole domain's dt too). */
  int32_t row_offset;   /* global index of this grid's row 0 (a y-slab's place in the whole
                           domain, negative where its halo wraps around a periodic domain; 0
                           otherwise) */
  int32_t row_period;   /* the whole domain's ny where it is periodic in y, else 0: the 16-bit
                           stochastic rounding is keyed by the global row, (row + row_offset)
                           mod row_period, so a slab -- halo rows that wrap around included --
                           rounds exactly as the whole domain does */
} lesbgk_params;

/* Read-only facts about a created solver. */
typedef struct lesbgk_info {
  double dt, dx, dy;  /* time step and spacing in use */
  double c_max;       /* largest |root| of He_nroots */
  double cfl;         /* effective Courant number c_max dt / min(dx,dy) */
  double tau_ref;     /* (Kn/Pr) T_max^(varpi-1) / rho_max at set-up */
  int64_t steps_done; /* time steps taken since create */
  int32_t q, order;   /* values stored per node (velocities; 32 for D3Q64), Hermite order */
  int32_t cells_per_thread, rows_per_segment; /* launch shape of the step kernel */
} lesbgk_info;

typedef struct lesbgk lesbgk;

/* Bytes of device workspace one solve with these parameters needs
 * (two population buffers of Q*nx*ny floats each, the second also large enough
 * to stage the initial fields and the nine moment fields, plus 4 KiB of
 * reduction scratch per 1024 blocks).  Returns LESBGK_EINVAL on bad params. */
int lesbgk_workspace_size(const lesbgk_params *p, size_t *bytes);

/* Validate p, build the quadrature and Hermite tables in FP64 on the host
 * (Sec. 2.2), pick dt, and write the initial populations
 * f = rho S(T,u) (Eq. feq0 at order N), followed once by the wall rule.
 *   d_workspace: device memory of >= lesbgk_workspace_size bytes, 256-byte
 *                aligned, owned by the caller.
 *   h_init:      HOST array double[4][ny][nx] = rho, u_x, u_y, T per node, or
 *                NULL for rest (rho = 1, u = 0, T = 1).  It is copied before
 *                the call returns.
 *   out:         receives the handle (host memory owned by the library until
 *                lesbgk_destroy). */
int lesbgk_create(const lesbgk_params *p, void *d_workspace, size_t bytes, const double *h_init,
                  void *stream, lesbgk **out);

/* Re-initialise the populations in place from DEVICE fields d_fields,
 * double[4][ny][nx] = rho, u_x, u_y, T (or NULL for rest): f = rho S(T,u)
 * then the wall rule, exactly as lesbgk_create does; the step counter restarts
 * at 0.  dt and the tables chosen at creation are kept.  d_fields must not
 * overlap the workspace. */
int lesbgk_reinit(lesbgk *h, const double *d_fields, void *stream);

/* Take nsteps >= 0 time steps: each is one launch of the fused kernel
 * (moments -> tau -> lambda -> a_ES -> force -> Hermite evaluation -> TVD
 * advection -> update -> diffuse walls), ping-ponging the two buffers. */
int lesbgk_step(lesbgk *h, int64_t nsteps, void *stream);

/* Moments of Eq. (mac) per node into DEVICE memory d_out, float[9][ny][nx]:
 * rho, u_x, u_y, T, sigma_xx, sigma_xy, sigma_yy, q_x, q_y
 * (sigma trace-free, q_i = 1/2 sum f C_i C^2, D = 2).
 * If h_sums is not NULL it receives, in HOST memory, double[4]: total mass,
 * x- and y-momentum and energy (sum over nodes of sum_a f_a {1, c_x, c_y,
 * c^2/2}): per-node sums in FP32, summed in FP32 over runs of 16 nodes, the
 * runs in FP64, in a fixed order (bitwise reproducible); this
 * synchronises the stream, and returns LESBGK_EDIVERGED if any is not
 * finite. */
int lesbgk_moments(lesbgk *h, float *d_out, double *h_sums, void *stream);

/* As lesbgk_moments, but into HOST memory h_out (float[9][ny][nx]); the
 * moments are staged in the workspace and copied back before returning. */
int lesbgk_moments_host(lesbgk *h, float *h_out, double *h_sums, void *stream);

/* Steady-state residual of the solve since a snapshot (not in the paper; the
 * test a serving loop applies):
 *   r = max over nodes of (|d rho| + |d u_x| + |d u_y| + |d T|) / (steps dt),
 * d the change of the node's fields since the snapshot, steps the time steps
 * taken since it; a node whose change is not finite makes r = +Inf.
 *   d_snap:  DEVICE float[4][ny][nx] (rho, u_x, u_y, T), caller-owned; read as
 *            the previous snapshot and overwritten with the current fields.
 *   steps:   time steps since the snapshot; <= 0 only takes the snapshot and
 *            returns r = NaN.
 *   h_r:     HOST double, receives r.
 *   h_mass:  HOST double receiving the total mass sum over nodes of rho (the
 *            per-node values in FP32, summed in FP64 in a fixed order), or
 *            NULL.  With diffuse walls at a temperature other than the gas's
 *            the wall rule exchanges a constant amount of mass per step, and
 *            the mass history tells that drift apart from a transient.
 * Synchronises the stream.  Errors: LESBGK_EINVAL (NULL arguments),
 * LESBGK_ECUDA. */
int lesbgk_residual(lesbgk *h, float *d_snap, int64_t steps, double *h_r, double *h_mass, void *stream);

/* Copy the current populations (deviations f_a - w_a, float[Q][ny][nx]) into
 * DEVICE memory d_out; with lesbgk_set_populations this is a checkpoint. */
int lesbgk_get_populations(lesbgk *h, float *d_out, void *stream);

/* Overwrite the current populations from DEVICE memory d_in (same layout);
 * the step counter is set to steps_done. */
int lesbgk_set_populations(lesbgk *h, const float *d_in, int64_t steps_done, void *stream);

/* Rows of the populations in the library's internal grouped layout, for the
 * halo exchange of a y-slab decomposition (not in the paper: one large solve
 * split over several solvers, each holding a slab of rows plus halo rows that
 * its neighbours refill; the TVD stencil of Sec. 3.1 reaches two rows, so a
 * halo of 2k rows carries k steps).
 *   lesbgk_rows_bytes: bytes of nrows packed rows.
 *   lesbgk_get_rows:   copy rows [j0, j0 + nrows) of the current populations
 *                      into DEVICE d_out (packed: for each population group,
 *                      its nrows x nx vectors; the stored type, any storage).
 *   lesbgk_set_rows:   overwrite rows [j0, j0 + nrows) from DEVICE d_in in the
 *                      same packing.
 * Both are one asynchronous 2D copy on the stream.  Errors: LESBGK_EINVAL for
 * rows outside [0, ny) or NULL pointers. */
int lesbgk_rows_bytes(const lesbgk *h, int32_t nrows, size_t *bytes);
int lesbgk_get_rows(lesbgk *h, int32_t j0, int32_t nrows, void *d_out, void *stream);
int lesbgk_set_rows(lesbgk *h, int32_t j0, int32_t nrows, const void *d_in, void *stream);

/* As lesbgk_moments, over rows [j0, j0 + nrows) only (a slab's own rows,
 * without its halo): d_out (DEVICE, or NULL) is float[9][nrows][nx], h_sums
 * (HOST, or NULL) the FP64 totals of those rows. */
int lesbgk_moments_rows(lesbgk *h, int32_t j0, int32_t nrows, float *d_out, double *h_sums, void *stream);

/* Choose the launch shape of the step kernel: cells_per_thread (x-nodes per
 * lane: 1, the only shape built; any other value is refused) and
 * rows_per_segment (rows one warp marches through, >= 1).  0 keeps the current
 * value.  Results do not depend on the shape (bitwise). */
int lesbgk_set_launch(lesbgk *h, int32_t cells_per_thread, int32_t rows_per_segment);

/* Fill *out with the solver's time step, spacing and launch shape. */
int lesbgk_get_info(const lesbgk *h, lesbgk_info *out);

/* Release the handle (not the caller's workspace).  NULL is a no-op. */
int lesbgk_destroy(lesbgk *h);

/* ------------------------------------------------------------------------
 * Batched solver: many independent narrow solves advanced together.
 *
 * A batch holds up to `capacity` instances ("slots"), all with the same nx, a
 * power of two <= 32 (the 1D-in-y flows of the paper's Sec. 4 run on nx = 4),
 * each with its own ny, Kn, b, walls (diffuse, Maxwell, steady or heated),
 * force and time step, on D2Q16 (order 3), D2Q36 (order 4) or D3Q64 (order 3, dim 3)
 * in FP32, FP16 or BF16 storage,
 * periodic in x.  Every lesbgk_batch_step advances every slot by the same
 * number of steps: per step one launch per class (velocity set, storage, wall
 * heating) over a work list of
 * (slot, row segment) items; steps in multiples of 64 replay a CUDA graph.
 * Each slot's arithmetic is that of lesbgk_step on the same problem (results
 * are bitwise equal), so a solve gives the same answer alone or in a batch.
 *
 * Memory: one caller-owned device workspace of lesbgk_batch_workspace_size
 * bytes: fixed tables for `capacity` slots, then a pool of pool_bytes from
 * which lesbgk_batch_add carves each slot's buffers
 * (lesbgk_batch_slot_bytes); a full pool makes lesbgk_batch_add return
 * LESBGK_ESPACE, which a caller can use as its admission test.
 * ---------------------------------------------------------------------- */
typedef struct lesbgk_batch lesbgk_batch;

int lesbgk_batch_workspace_size(int32_t capacity, size_t pool_bytes, size_t *bytes);
/* Pool bytes one slot with these parameters takes. */
int lesbgk_batch_slot_bytes(const lesbgk_params *p, size_t *bytes);
int lesbgk_batch_create(int32_t capacity, int32_t nx, void *d_workspace, size_t bytes, void *stream,
                        lesbgk_batch **out);
/* Admit a solve: tables, dt and the initial populations exactly as
 * lesbgk_create (h_init: HOST double[4][ny][nx] or NULL, copied before the
 * call returns); *slot receives its slot index.  The initialisation is queued
 * on the stream; the work list is rebuilt at the next step. */
int lesbgk_batch_add(lesbgk_batch *b, const lesbgk_params *p, const double *h_init, void *stream,
                     int32_t *slot);
/* Admit n solves at once (ps[i], h_inits[i] as in lesbgk_batch_add; h_inits
 * may be NULL for all at rest, or hold NULL entries): their descriptors go to
 * the device in one copy and their initial populations are written by one
 * launch per class, with the arithmetic of lesbgk_batch_add (bitwise
 * the same populations).  slots_out (HOST int32[n]) receives the slots.  All
 * or nothing: if one solve cannot be admitted (LESBGK_ESPACE when the pool or
 * the slots run out), none is, and the error is returned.  Synchronises the
 * stream. */
int lesbgk_batch_add_many(lesbgk_batch *b, int32_t n, const lesbgk_params *ps, const double *const *h_inits,
                          void *stream, int32_t *slots_out);
/* Retire a slot and return its buffers to the pool (synchronises the stream
 * first, so no queued step still reads them). */
int lesbgk_batch_remove(lesbgk_batch *b, int32_t slot, void *stream);
int lesbgk_batch_step(lesbgk_batch *b, int64_t nsteps, void *stream);
/* Steady-state residual of every slot since the previous call:
 * r = max over nodes of (|d rho| + |d u_x| + |d u_y| + |d T|) / (steps * dt),
 * into HOST double[capacity]; NaN for empty slots and for a slot's first call,
 * +Inf for a slot with a non-finite change (a diverged solve).  h_mass, if not
 * NULL, receives HOST double[capacity]: each slot's total mass (as
 * lesbgk_residual; NaN for empty slots).  Synchronises the stream. */
int lesbgk_batch_residuals(lesbgk_batch *b, double *h_res, double *h_mass, void *stream);
/* As lesbgk_moments / lesbgk_get_populations / lesbgk_get_info, per slot. */
int lesbgk_batch_moments(lesbgk_batch *b, int32_t slot, float *d_out, double *h_sums, void *stream);
int lesbgk_batch_get_populations(lesbgk_batch *b, int32_t slot, float *d_out, void *stream);
/* The moment fields of n slots in one launch per class: d_outs (HOST
 * array of n DEVICE pointers) receives slot slots[i]'s float[9][ny][nx], with
 * the per-node arithmetic of lesbgk_batch_moments (bitwise the same fields;
 * no totals).  The pointer list is staged in the batch's workspace: calls on
 * one batch must not overlap on the GPU. */
int lesbgk_batch_moments_many(lesbgk_batch *b, int32_t n, const int32_t *slots, float *const *d_outs,
                              void *stream);
int lesbgk_batch_get_info(const lesbgk_batch *b, int32_t slot, lesbgk_info *out);
/* Checkpoint and resume of one slot, bitwise for every storage: the slot's
 * current population buffer as stored (grouped layout, FP32 or 16-bit,
 * lesbgk_batch_raw_bytes bytes) copied to or from DEVICE memory.
 * lesbgk_batch_set_raw also sets the slot's step count to steps_done (its
 * clock: the heated walls' time and the 16-bit rounding keys), so a slot
 * admitted with the same parameters and given a checkpoint taken after n
 * steps continues exactly as the original would; it synchronises the stream
 * and invalidates the slot's residual snapshot (the next
 * lesbgk_batch_residuals reports NaN for it). */
int lesbgk_batch_raw_bytes(const lesbgk_batch *b, int32_t slot, size_t *bytes);
int lesbgk_batch_get_raw(lesbgk_batch *b, int32_t slot, void *d_out, void *stream);
int lesbgk_batch_set_raw(lesbgk_batch *b, int32_t slot, const void *d_in, int64_t steps_done, void *stream);
/* Rows per work item (default 32); results do not depend on it. */
int lesbgk_batch_set_rows(lesbgk_batch *b, int32_t rows, void *stream);
/* Resident kernel (on by default): D2Q16 FP32 instances of at most max_ny rows
 * (0 keeps the current limit, 128 by default) whose two population buffers
 * fit in one block's shared memory (454 rows at nx = 4 on GB300) are each held
 * (steady walls) by one block for steps_per_launch time steps (an even divisor of 64; 0
 * keeps the current, 64 by default), reading and writing device memory once
 * per launch, while the other instances take one launch per step; in the
 * 64-step graphs the two run side by side.  A resident instance is one
 * block's serial work, so tall ones are better left to the per-step kernel.
 * Results do not depend on the choice (bitwise). */
int lesbgk_batch_set_resident(lesbgk_batch *b, int32_t on, int32_t steps_per_launch, int32_t max_ny, void *stream);
/* The launch configuration in use (any pointer may be NULL). */
int lesbgk_batch_get_launch(const lesbgk_batch *b, int32_t *rows, int32_t *resident, int32_t *steps_per_launch,
                            int32_t *resident_max_ny);
/* Autotuner: time a 64-step chunk of the current slots for each candidate
 * rows per work item, each with the resident kernel off, and on at 16 and 64
 * steps per launch for instances of at most 64, 128, 256 rows or as many as
 * fit (the state is left unchanged: every timed launch writes the spare
 * buffers), and keep the fastest; *chosen receives its rows per item
 * (lesbgk_batch_get_launch gives the rest). */
int lesbgk_batch_autotune(lesbgk_batch *b, const int32_t *candidates, int32_t n, int32_t *chosen, void *stream);
/* Largest free block and total free bytes of the pool. */
int lesbgk_batch_pool_free(const lesbgk_batch *b, size_t *largest, size_t *total);
/* Guard words (a check for writes outside a slot's memory; the paper has no
 * counterpart): each slot's pool block ends in 256 bytes set to 0xA5 at
 * admission, which no kernel writes.  lesbgk_batch_check_guards compares
 * them on the device and sets h_bad[slot] (HOST int32[capacity]) to 1 for
 * every admitted slot whose guard changed, 0 otherwise; it synchronises the
 * stream.  lesbgk_batch_debug_poison overwrites 4 bytes of one slot's guard,
 * for testing the check.  Both use the workspace's moment-output and
 * admission scratch: they must not overlap lesbgk_batch_moments_many or
 * lesbgk_batch_add_many on the GPU. */
int lesbgk_batch_check_guards(lesbgk_batch *b, int32_t *h_bad, void *stream);
int lesbgk_batch_debug_poison(lesbgk_batch *b, int32_t slot, void *stream);
int lesbgk_batch_destroy(lesbgk_batch *b);

/* Moments without any allocation (the paper has no counterpart: this is a
 * service to embedding code).  Some callers cannot allocate device memory at
 * all -- their device memory belongs to another allocator, they run under a
 * fixed memory budget, or they cannot afford the device-wide synchronisation
 * of cudaMalloc -- and so cannot provide the scratch that lesbgk_moments finds
 * in the solver's workspace.  This entry point computes the same nine fields
 * and FP64 totals as lesbgk_moments from populations the caller already holds
 * and calls no cudaMalloc, cudaFree or allocating library routine.
 *   p:             the solver parameters (grid and velocity set are used).
 *   d_populations: DEVICE float[Q][ny][nx], deviations f_a - w_a in the layout
 *                  lesbgk_get_populations returns.
 *   d_out:         DEVICE float[9][ny][nx] as in lesbgk_moments, or NULL.
 *   h_sums:        HOST double[4] as in lesbgk_moments, or NULL (if given, the
 *                  stream is synchronised).
 * Limit: nx*ny <= 2^24 nodes (4096 x 4096); larger grids return LESBGK_EINVAL.
 * Its scratch is a fixed 256 KiB + 32 B array inside the library that every GPU which
 * loads the library keeps until the process exits.  The first call in a CUDA
 * context looks up that array's device address in the current context (the
 * device's primary context unless the caller made another one current) and
 * remembers it for that context's unique ID; make that first call before any
 * stream capture.  The address belongs to the context: after a device reset,
 * or in a context of the caller's own, the next call looks it up again (it is
 * then again a first call).  All calls share the array: each call writes
 * every scratch slot it reads, so nothing carries over, but calls that
 * overlap on the GPU (other streams, other host threads) race on it and must
 * be serialised by the caller. */
int lesbgk_moments_noalloc(const lesbgk_params *p, const float *d_populations, float *d_out, double *h_sums,
                           void *stream);

/* Thread-local message of the last error ("" if none). */
const char *lesbgk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LESBGK_H */
