/*
 * tdse.h -- C ABI of libtdse: the FDTD leapfrog for the 3-D time-dependent
 * Schrodinger equation on one GB300 (sm_103a).
 *
 * Method: Nagaya, Omatsu, Packwood, "Fast generation of quantum dynamics data
 * using a GPU implementation of the time-dependent Schrodinger equation",
 * arXiv 2401.07416.  psi = psi_R + i psi_I on a uniform grid (Sec. 2.1, Eqs. 5-7);
 * psi_R lives at integer and psi_I at half-integer time levels and they are
 * advanced in turn by Eq. 9 (psi_I += A psi_R) and Eq. 8 (psi_R -= A psi_I), where
 *   A f = c_x (f[i+1] - 2 f + f[i-1]) + c_y (...) + c_z (...) - c_v V f,
 *   c_a = hbar dt / (2 m h_a^2),  c_v = dt / hbar          (Sec. 2.1 after Eq. 9).
 * Periodic axes wrap neighbours as in Eqs. 13-14; a walled axis reads zero
 * outside [0, n).  Eq. 10's absorbing potential is replaced by a per-plane
 * factor M_k = cos^2(eta (pi/2) d / W) on W-cell layers at the z ends (d = 1..W,
 * the depth into the layer), applied to both parts after every step.  The
 * detector (Eq. 15 stores the density on a plane) records here the probability
 * flux through the face between planes det_k and det_k+1,
 *   j = hbar / (m h_z) * (R[det_k] I[det_k+1] - R[det_k+1] I[det_k]),
 * with R at step n and I at step n+1/2, and its time integral F = sum_n j dt.
 *
 * Conventions for every function:
 *   - Arrays are [nz][ny][nx] with x fastest, unpadded, FP64, unless stated.
 *   - Every call returns a tdse_status; nothing throws across the ABI.  On an
 *     error, tdse_last_error() describes it; the context stays usable unless
 *     the status is TDSE_ECUDA, TDSE_EUNSTABLE or TDSE_ETIMEOUT.  After the last
 *     two its state is not a result of the scheme: tdse_step, tdse_adjoint,
 *     tdse_autotune and tdse_save_state then return TDSE_ESTATE, while the
 *     calls that read the state still work (for inspection).
 *   - The context owns all device memory it allocates (through the allocator
 *     callbacks, cudaMalloc/cudaFree by default) and frees it in tdse_destroy.
 *     Caller pointers are borrowed for the duration of the call only.
 *   - `on_device` != 0 means a pointer is CUDA device memory on the current
 *     device; otherwise it is host memory.
 *   - All GPU work is issued on the stream given to tdse_set_stream (default:
 *     the legacy default stream).  Functions that return host data synchronise
 *     that stream.
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - There is no CPU fallback: every computation runs in this library's CUDA
 *     kernels, and a missing GPU is reported as TDSE_ECUDA.
 */
#ifndef TDSE_H
#define TDSE_H

#include <stddef.h>

#if defined(__GNUC__)
#define TDSE_API __attribute__((visibility("default")))
#else
#define TDSE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TDSE_OK = 0,
    TDSE_EINVAL = -1,    /* bad argument: shape, NULL pointer, dt above the stability bound ... */
    TDSE_ENOMEM = -2,    /* the allocator returned NULL */
    TDSE_ECUDA = -3,     /* a CUDA runtime/driver call failed */
    TDSE_EUNSTABLE = -4, /* non-finite values or growth of the invariant Q by > 1e-3 */
    TDSE_ETIMEOUT = -5,  /* a bounded wait inside a kernel expired */
    TDSE_ESTATE = -6     /* call out of order (e.g. step before set_wavepacket) */
} tdse_status;

enum { TDSE_BC_PERIODIC = 0, TDSE_BC_DIRICHLET = 1 };

/* Storage and arithmetic of psi and of the potential term:
 *   TDSE_FP64        FP64 fields and FP64 arithmetic;
 *   TDSE_FP32        FP32 fields, FP32 stencil arithmetic;
 *   TDSE_FP32_KAHAN  FP32 fields plus FP32 compensation terms of the Kahan
 *                    (compensated) sum f += increment, persisted between calls.
 * Reductions (norm, energy, flux) are FP64 in every mode. */
enum { TDSE_FP64 = 0, TDSE_FP32 = 1, TDSE_FP32_KAHAN = 2 };

typedef struct tdse_params {
    int nx, ny, nz;          /* nodes per axis; nx must be a multiple of 4, ny, nz >= 1 */
    double hx, hy, hz;       /* spacings (Sec. 2.1: r = (i hx, j hy, k hz), i, j, k >= 0) */
    double dt;               /* time step; <= 0 selects Eq. 11, dt = m min(h)^2 / (5 hbar) */
    double hbar, mass;       /* <= 0 selects 1 (atomic units) */
    int bc[3];               /* TDSE_BC_* per axis x, y, z */
    int mask_lo, mask_hi;    /* absorbing cells at the z = 0 and z = nz-1 ends (0: none) */
    double mask_eta;         /* absorbing strength: TDSE_MASK_COS2: eta (M at the outermost cell =
                                cos^2(eta pi/2)); TDSE_MASK_CAP: W at the outermost cell (energy) */
    int det_k;               /* detector face between planes det_k, det_k+1; -1: no detector */
    int obs_every;           /* norm/energy reduction every obs_every steps (<= 0: 20, Sec. 2.3) */
    int ckpt_every;          /* > 0: keep FP64 checkpoints every ckpt_every steps for tdse_adjoint */
    int precision;           /* TDSE_FP64 / TDSE_FP32 / TDSE_FP32_KAHAN (same for all members) */
    int tblock;              /* steps fused per kernel launch (temporal blocking), 1..TDSE_MAX_TBLOCK
                                among the depths with kernel variants (tdse_variant_count: FP64
                                fuses 1, FP32 and FP32_KAHAN 1 to 4); 0: automatic */
    int mask_kind;           /* TDSE_MASK_COS2 (0) or TDSE_MASK_CAP (1), see below */
    int reserved[5];         /* must be zero */
} tdse_params;

/* Absorbing layers (mask_lo planes at z = 0, mask_hi at z = nz-1; depth d = 1..W
 * from the layer's inner edge, d = W the outermost plane).  After every step both
 * parts of psi are multiplied by a per-plane factor M(d):
 *   TDSE_MASK_COS2  M = cos^2(eta (pi/2) d / W)
 *   TDSE_MASK_CAP   M = exp(-W(d) dt / hbar), W(d) = mask_eta (d / W)^2: Eq. 10's
 *                   absorbing potential -i W (quadratic in the depth into the layer),
 *                   applied by operator splitting (exp(-W dt/hbar) is the exact
 *                   action of that term alone over one step).  The paper's set-up is
 *                   one layer (mask_lo only) on an appended bottom region. */
enum { TDSE_MASK_COS2 = 0, TDSE_MASK_CAP = 1 };

typedef struct tdse_obs {
    double Q;                /* h^3 sum (R^n R^n + I^{n+1/2} I^{n-1/2}), exactly conserved by the
                                scheme for real V without absorbing layer */
    double norm_paper;       /* h^3 sum (R^n^2 + I^{n-1/2}^2), the density of Sec. 2.1 */
    double energy;           /* (R.H R + I^{n+1/2}.H I^{n-1/2}) / (R.R + I^{n+1/2}.I^{n-1/2}) */
    double flux;             /* hx hy sum_yx j^{n-1}: detector flux of the last step */
    double flux_integrated;  /* hx hy sum_yx F: probability that crossed the face so far */
    double t;                /* time n dt */
    long long step;          /* n */
} tdse_obs;

typedef struct tdse_ctx tdse_ctx;

typedef void *(*tdse_alloc_fn)(size_t bytes, void *user);
typedef void (*tdse_free_fn)(void *ptr, void *user);

/* Create a context for `batch` simulations; p[m] describes member m (Sec. 2.1,
 * Eqs. 6-11).  Members may differ in shape, spacing, dt and boundaries, but
 * share precision, tblock, obs_every and ckpt_every.  Validates everything
 * (EINVAL: shape, spacing, dt above the leapfrog stability bound of the free
 * part, nx not a multiple of 4, periodic axis shorter than 8, det_k outside
 * [0, nz-2], an xy plane above 2^30 nodes with its ghost zones); allocates no
 * device memory.  *out receives the context. */
TDSE_API tdse_status tdse_create(const tdse_params *p, int batch, tdse_ctx **out);

/* Route device allocations through (alloc, free, user), e.g. a framework's
 * caching allocator.  Allowed only before the first allocation (ESTATE). */
TDSE_API tdse_status tdse_set_allocator(tdse_ctx *ctx, tdse_alloc_fn alloc, tdse_free_fn free_fn,
                               void *user);

/* Issue all work on `cuda_stream` (a cudaStream_t; NULL: legacy default stream). */
TDSE_API tdse_status tdse_set_stream(tdse_ctx *ctx, void *cuda_stream);

/* Potential V[nz][ny][nx] (FP64) of member m, Eq. 2's V(r) on the grid
 * (Sec. 2.3 interpolates a DFT potential; any gridded V is accepted).  V is a host
 * pointer (on_device = 0) or a device pointer (on_device = 1); it is copied into the
 * member's resident FP64 copy, from which the step's diagonal d = -2 (cx + cy + cz)
 * - cv V is built.  Page-locked host memory (cudaHostAlloc, cudaHostRegister, a
 * pinned torch tensor) is read directly by the kernel that builds d; pageable host
 * memory is copied first.  A host buffer may be reused when the call returns (it
 * waits for the transfer); a device buffer once the stream has passed this call.  A
 * failed transfer (ECUDA) leaves the member's potential undefined until the next
 * successful call. */
TDSE_API tdse_status tdse_set_potential(tdse_ctx *ctx, int member, const double *V, int on_device);

/* Potential of member m interpolated from one periodic cell (Sec. 2.3: the
 * electrostatic potential of a unit cell, expanded and interpolated onto the
 * mesh, the step the paper found dominant).  Vc[cnz][cny][cnx] holds the cell's
 * potential at origin + (i Lx/cnx, j Ly/cny, k Lz/cnz), cell = (Lx, Ly, Lz); the
 * cell repeats in every axis.  V at node (i hx, j hy, k hz) is the trilinear
 * interpolation of that periodic lattice, computed in FP64 on the GPU, then used
 * exactly like tdse_set_potential.  EINVAL: NULL pointer, cnx/cny/cnz < 1, a
 * cell length <= 0, or a non-finite cell length or origin. */
TDSE_API tdse_status tdse_set_potential_grid(tdse_ctx *ctx, int member, const double *Vc, int cnx,
                                             int cny, int cnz, const double cell[3],
                                             const double origin[3], int on_device);

/* Build V on the GPU from n atoms, xyzZ[n][4] = (x, y, z, Z):
 * V(r) = -sum_a Z_a phi(|r - r_a|), phi = 1/sqrt(r^2 + a^2) minus its second-order
 * Taylor polynomial in r^2 about r_cut for r < r_cut, 0 beyond; minimum-image
 * distances along periodic axes.  soft_a2 = a^2; r_cut <= 0 selects half the
 * shortest periodic length (no cut-off if no axis is periodic).  The atoms are
 * kept for the chain rule of tdse_adjoint. */
TDSE_API tdse_status tdse_set_atoms(tdse_ctx *ctx, int member, int n, const double *xyzZ,
                           double soft_a2, double r_cut);

/* Copy the potential V[nz][ny][nx] (FP64) of member m out (ESTATE if none was set). */
TDSE_API tdse_status tdse_get_potential(tdse_ctx *ctx, int member, double *V, int on_device);

/* Initial packet (Eq. 3 with a vector wave number): psi0 = prod_a g_a exp(i k0.(r - r0)),
 * g_a = exp(-(r_a - r0_a)^2 / (2 sigma_a^2)), sigma_a <= 0 meaning no Gaussian factor
 * along a; normalised so that h^3 sum |psi0|^2 = 1.  Sets R^0 = Re psi0 and
 * I^{-1/2} = Im psi0 - A[Re psi0] / 2 (second-order start of the staggered scheme),
 * resets the flux integral, observation history and checkpoints.  Without a
 * potential, V = 0 is used. */
TDSE_API tdse_status tdse_set_wavepacket(tdse_ctx *ctx, int member, const double r0[3],
                                const double sigma[3], const double k0[3]);

/* Set the state directly: R = psi_R^n, I = psi_I^{n-1/2} (FP64 [nz][ny][nx]). */
TDSE_API tdse_status tdse_set_state(tdse_ctx *ctx, int member, const double *R, const double *I,
                           int on_device);

/* Advance every member by nsteps leapfrog steps (Eqs. 8-9 + absorbing layer),
 * accumulating the detector flux, reducing Q and E every obs_every steps and
 * recording checkpoints every ckpt_every steps.  Returns EUNSTABLE if a
 * reduction saw non-finite values or, when the first value Q0 is positive, Q
 * above (1 + 1e-3) Q0,
 * and ETIMEOUT if a step kernel's bounded wait for a tile's data expired (see
 * tdse_set_wait_limit).  Each observation point copies the kernels' status word
 * to the host without stalling the GPU; the host reads these copies as they
 * complete, so a failure ends the call at most two observation intervals after
 * the observation point that recorded it (the message names that step), with
 * the issued work finished and the step counter at the last step run. */
TDSE_API tdse_status tdse_step(tdse_ctx *ctx, long long nsteps);

/* Observables of member m at the current step (computed now, FP64). */
TDSE_API tdse_status tdse_observables(tdse_ctx *ctx, int member, tdse_obs *out);

/* History of the periodic reductions of member m: up to `cap` records of
 * (step, Q, norm_paper, energy) into out[4*i..4*i+3]; *count receives the
 * number available. */
TDSE_API tdse_status tdse_get_obs_history(tdse_ctx *ctx, int member, double *out, int cap, int *count);

/* Copy the state out as FP64: R = psi_R^n, I = psi_I^{n-1/2} (Kahan mode: value
 * plus compensation).  Either pointer may be NULL. */
TDSE_API tdse_status tdse_get_state(tdse_ctx *ctx, int member, double *R, double *I, int on_device);

/* Time-integrated detector flux F[ny][nx] = sum_n j^n dt (FP64). */
TDSE_API tdse_status tdse_get_flux_map(tdse_ctx *ctx, int member, double *F, int on_device);

/* Detector-plane density frames (Sec. 2.3, Eq. 15): rho[y][x] = R^n^2 + I^{n-1/2}^2
 * on plane det_k (the paper's density of Sec. 2.1 restricted to the detector
 * plane D), FP64, recorded into a device buffer of `capacity` frames per member
 * at the start of a run (tdse_set_wavepacket / tdse_set_state) and at every
 * observation point (every obs_every steps).  Recording stops when the buffer is
 * full.  Setting a capacity (0 frees the buffer) discards recorded frames.
 * EINVAL: member has no detector plane (det_k < 0) or capacity < 0. */
TDSE_API tdse_status tdse_set_frame_capacity(tdse_ctx *ctx, int member, int capacity);

/* Copy up to `cap` recorded frames of member m into frames[cap][ny][nx] and their
 * step numbers into steps[cap] (either may be NULL); *count receives the number
 * recorded. */
TDSE_API tdse_status tdse_get_frames(tdse_ctx *ctx, int member, double *frames, long long *steps,
                                     int cap, int *count, int on_device);

/* Eq. 16 dissimilarity of K detector-density trajectories:
 *   d_kj = 1/(t1 - t0) * integral_{t0}^{t1} ( integral_D (rho_k - rho_j)^2 dA )^{1/2} dt,
 * discretised over the frames whose time lies in [t0, t1]: the inner integral is
 * dA * sum over the P pixels, the outer one the trapezoidal rule on those frame
 * times (a single frame in the window counts for the whole window).
 *   frames  [K][M][P] FP64, trajectory k's M frames of P pixels (same times t[M],
 *           increasing, for every trajectory)
 *   d       [K][K] FP64 output; symmetric, zero diagonal
 * Both arrays are on the device if on_device != 0, else on the host.  The work
 * (K (K+1)/2 pairs x frames x pixels in FP64, then the time sums) runs on
 * `stream` (a cudaStream_t; NULL: legacy default stream), which is synchronised
 * before returning; scratch memory comes from cudaMallocAsync on that stream.
 * EINVAL: NULL pointer, K < 1, M < 1, P < 1, dA <= 0, t1 <= t0 or no frame time
 * in [t0, t1]; ENOMEM / ECUDA: a CUDA allocation or call failed.  Stateless: no
 * context is involved. */
TDSE_API tdse_status tdse_dissimilarity(const double *frames, int K, int M, long long P,
                                        const double *t, double t0, double t1, double dA,
                                        double *d, int on_device, void *stream);

/* Reverse-mode gradient of a loss L(F) of the time-integrated flux of member m,
 * over all steps since tdse_set_wavepacket (requires ckpt_every > 0).
 * dL_dF[ny][nx] is dL/dF; outputs (each may be NULL): dL_dV[nz][ny][nx] and,
 * if the potential came from tdse_set_atoms, dL_datoms[n][4] = dL/d(x, y, z, Z).
 * The leapfrog is run backward in time from the latest state (the map is
 * invertible: R^n = R~ + A I~, I^{n-1/2} = I~ - A R^n with R~ = R^{n+1}/M,
 * I~ = I^{n+1/2}/M), re-anchored at every FP64 checkpoint; the adjoint
 * recursion is the transpose of the forward step.  The forward state is left
 * unchanged.  ESTATE: no state, no checkpoints, or dL_datoms without atoms;
 * EINVAL: dL_dF NULL, or an absorbing factor M that is 0 in the step's number format
 * (a CAP with W dt / hbar beyond about 745 in FP64 or 103 in FP32 underflows), which
 * the backward steps cannot divide out.  A small M is accepted, but the reversal
 * amplifies rounding by up to (1 / M_min)^ckpt_every between checkpoints. */
TDSE_API tdse_status tdse_adjoint(tdse_ctx *ctx, int member, const double *dL_dF, double *dL_dV,
                         double *dL_datoms, int on_device);

/* Form of tdse_adjoint's backward step: 0 (the default) runs three passes in
 * place; enable != 0 runs each step as one z-march over tiles that reads the
 * reconstructed state and its adjoint from one set of buffers and writes the next
 * into a second set (four more arrays of the grid's size; it moves each field once
 * per step, but measured slower than the three passes on GB300).  Both give the
 * same numbers, bit for bit (the per-cell arithmetic is shared). */
TDSE_API tdse_status tdse_set_adjoint_fused(tdse_ctx *ctx, int enable);

/* Save / restore the whole context state to / from a binary file: for every
 * member its parameters, the raw state fields (R, I and, in Kahan mode, their
 * compensation terms, each stored exactly as FP64), V, the flux integral and last flux,
 * the observation history, the atoms and the adjoint checkpoints; plus the step
 * counter.  load_state needs a context created with the same batch and grid
 * parameters (EINVAL otherwise) and replaces its potential and state. */
TDSE_API tdse_status tdse_save_state(tdse_ctx *ctx, const char *path);
TDSE_API tdse_status tdse_load_state(tdse_ctx *ctx, const char *path);

/* Largest number of time steps fused into one kernel launch (temporal blocking). */
#define TDSE_MAX_TBLOCK 4

/* Kernel timing, for benchmarks.  While enabled, the fused-step launches are
 * timed with CUDA events on the context's stream: a step sequence between two
 * reductions whose launches all fuse the same number of steps is replayed from
 * its CUDA graph (when graphs are on) and timed as a whole, its time divided
 * evenly over its launches; any other sequence is issued as direct launches,
 * each bracketed by its own events.  tdse_get_profile returns, since the last
 * reset, the launches and device milliseconds of the step kernels (in total and
 * per fused depth T) and of the reduction kernels, the grid nodes per step
 * launch (all members), and the backward steps of tdse_adjoint with their device
 * time (each checkpoint segment timed as a whole). */
typedef struct tdse_profile {
    long long step_launches;        /* fused-step launches, every depth */
    double step_ms;                 /* their device time */
    long long reduce_launches;
    double reduce_ms;
    long long cells_per_launch;     /* grid nodes updated by one step launch */
    int steps_per_launch;           /* fused depth of the last step launch */
    int reserved;
    long long launches_at_depth[TDSE_MAX_TBLOCK + 1];   /* [T]: launches fusing T steps */
    double ms_at_depth[TDSE_MAX_TBLOCK + 1];            /* [T]: their device time */
    long long adjoint_steps;        /* backward steps of tdse_adjoint */
    double adjoint_ms;              /* their device time (checkpoint reloads excluded) */
} tdse_profile;
TDSE_API tdse_status tdse_set_profiling(tdse_ctx *ctx, int enable);
TDSE_API tdse_status tdse_get_profile(tdse_ctx *ctx, tdse_profile *out);

/* Kernel variants and fused depth.  The fused step exists in several variants
 * (tile shape, planes loaded ahead, CTAs per SM) for each precision and number
 * of steps per launch T (tdse_variant_count(precision, T) of them; a depth
 * without variants is not available for that precision).  tdse_autotune times
 * every variant on this context's own grids (`launches` launches each, after one
 * warm-up) at z-chunks of 1, 0.7, 0.5, 0.35 and 0.2 of the makespan model's
 * length for it (only the fixed one if tdse_set_chunk fixed one), then the
 * fastest pair at 0.85, 0.9, 0.95, 1.05, 1.1 and 1.15 of its chunk; the four fastest pairs
 * are then timed twice more in turn, each keeping its best time, and the fastest
 * is kept for each depth.  If the context was created with tblock = 0, it picks the depth
 * with the lowest time per step.  The state, flux integral and step counter are
 * saved before and restored after the trials.
 * Step sequences between two reductions are replayed from captured CUDA graphs
 * unless tdse_set_graphs(ctx, 0) was called (with profiling on, only sequences
 * whose launches all have one depth are replayed). */
typedef struct tdse_tuning {
    int tblock;                                 /* steps fused per launch in use */
    int variant[TDSE_MAX_TBLOCK + 1];           /* [T]: variant index for T fused steps ([0] unused) */
    double ms_per_step[TDSE_MAX_TBLOCK + 1];    /* [T]: measured by tdse_autotune, 0 if not measured */
    char name[TDSE_MAX_TBLOCK + 1][48];         /* [T]: variant names ("" without variants) */
    int chunk[TDSE_MAX_TBLOCK + 1];             /* [T]: z-planes per work item of the longest member */
} tdse_tuning;
TDSE_API int tdse_variant_count(int precision, int tsteps);
TDSE_API tdse_status tdse_set_variant(tdse_ctx *ctx, int tsteps, int variant);
TDSE_API tdse_status tdse_autotune(tdse_ctx *ctx, int launches);
TDSE_API tdse_status tdse_get_tuning(tdse_ctx *ctx, tdse_tuning *out);
TDSE_API tdse_status tdse_set_graphs(tdse_ctx *ctx, int enable);

/* z-planes per work item of the fused step with `tsteps` steps per launch (planes
 * <= 0: the makespan model's choice, the default; members shorter than that take
 * one item per tile).  A work item also loads and computes the 2 tsteps planes on
 * each side that its pipeline needs, so shorter items cost more arithmetic; they
 * finish sooner, and neighbouring tiles then read their shared halos while they are
 * still in L2.  EINVAL: no variants for that depth, planes < 0. */
TDSE_API tdse_status tdse_set_chunk(tdse_ctx *ctx, int tsteps, int planes);

/* Limit, in nanoseconds, of each wait of a step kernel for a tile's data to land
 * in shared memory (default 2e9 = 2 s; no correct launch comes near it).  When a
 * wait expires, the CTA sets the status word, waits (bounded, 2 s) for its own
 * loads still in flight, releases its tensor memory and leaves; tdse_step
 * returns ETIMEOUT and the context is failed.  ns = 0 makes every wait test its
 * data once without waiting, so any wait whose data is still in flight expires:
 * a way to exercise that path with every load valid.  EINVAL: ns < 0. */
TDSE_API tdse_status tdse_set_wait_limit(tdse_ctx *ctx, long long ns);

/* Description of the last error on this context (static storage, never NULL). */
TDSE_API const char *tdse_last_error(const tdse_ctx *ctx);

/* Q, paper norm and energy (out[0..2], as in tdse_obs) of an FP64 state
 * R = psi_R^n, I = psi_I^{n-1/2} and potential V (each [nz][ny][nx], device memory;
 * V may be NULL for V = 0) on the grid described by *p (spacings, dt, hbar, mass,
 * boundaries; precision, absorbing layers and detector are ignored), without
 * allocating any device memory.  The paper has no counterpart: this exists for
 * callers that cannot allocate, such as a host program whose device memory is
 * owned by another allocator (a framework pool or a fixed arena it must not
 * bypass), or code where a cudaMalloc would implicitly synchronise the device.
 * The reduction's scratch is a static device array of 8193 x 4 doubles
 * (256 KiB) that every GPU loading this library keeps until the process exits;
 * the first call on a device looks up its address, so make that first call
 * before any stream capture.  Each call overwrites the nz per-plane sums it
 * reads and the result slot, so nothing has to be cleared between calls, but
 * calls on the same device share the array: calls that overlap on the GPU
 * (other streams, other host threads) race.  The call is synchronous: its two
 * kernels run on `stream` (a cudaStream_t; NULL: legacy default stream), the
 * results are copied into the caller's host array out, and the stream is
 * synchronised before the call returns.  R, I and V must each hold nx ny nz
 * doubles on the current device (not checked here: a shorter array is read out
 * of bounds).  EINVAL: NULL pointer, bad spacing, a boundary flag other than
 * TDSE_BC_PERIODIC / TDSE_BC_DIRICHLET, nz above 8192 (one scratch slot per z
 * plane), or an xy plane above 2^30 nodes; ECUDA: a CUDA call failed (its own
 * launches or copies; an error left by earlier, unrelated work is not reported). */
TDSE_API tdse_status tdse_observables_static(const tdse_params *p, const double *R,
                                             const double *I, const double *V, double out[3],
                                             void *stream);

/* Library version string. */
TDSE_API const char *tdse_version(void);

/* Free every device allocation and the context (NULL is accepted). */
TDSE_API tdse_status tdse_destroy(tdse_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* TDSE_H */
