/*
 * lbm.h - C ABI of the GB300 (sm_103a) D3V15 finite-difference lattice
 * Boltzmann solver for the 3D compressible Euler equations of Chen, Xu,
 * Zhang & Li, "Three-Dimensional Lattice Boltzmann Model for High-Speed
 * Compressible Flows" (arXiv:1010.4135).
 *
 * One time step (lbm_step) is the paper's update of the 15 distribution
 * functions f_i (Sec. 2 velocity set and equilibrium, Sec. 3 NND convection,
 * extra dissipation term, BGK relaxation, forward Euler) with the boundary
 * layers of Sec. 4(2).  All arithmetic of the step runs in CUDA kernels.
 *
 * Conventions shared by every entry point
 *   - Velocity index i = 0..14 is the paper's i = 1..15: 0 rest; 1..6 = c1
 *     along +x,-x,+y,-y,+z,-z; 7..14 = c2/sqrt(3) (sx,sy,sz) with the sign
 *     triples in the order +++,++-,+-+,+--,-++,-+-,--+,---.
 *   - Dense field arrays are x-fastest over interior cells only:
 *     rho[z][y][x], T[z][y][x], u[3][z][y][x], f[15][z][y][x].
 *   - Macroscopic tuples are (rho, u1, u2, u3, T) with R = 1 (p = rho T).
 *   - Pointers flagged on_device = 1 are device pointers on the device that
 *     owns the sim; on_device = 0 means ordinary (pageable or pinned) host
 *     memory, and the call then returns only after the copy has completed.
 *   - Every call returns an lbm_status (0 = success).  Kernel launches are
 *     asynchronous on the sim's stream; a fault inside a kernel is reported
 *     by the next call that synchronises (lbm_sync, lbm_moments, lbm_get_f,
 *     lbm_conserved, lbm_health, host-pointer lbm_init/lbm_set_f).  A CUDA
 *     error is sticky: every later call on that sim returns LBM_ESTATE.
 *   - No kernel traps or spins without bound.
 *
 * Ownership: the caller allocates the device workspace (lbm_workspace_bytes)
 * and the CUDA stream; both must outlive the sim.  The sim owns only a small
 * host-side descriptor.  The library allocates no device memory.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,      /* invalid argument (sizes, constants, boundary kinds, pointers) */
  LBM_ENOMEM = -2,      /* workspace smaller than lbm_workspace_bytes() */
  LBM_ECUDA = -3,       /* a CUDA call failed; the sim is then in LBM_ESTATE */
  LBM_ENONFINITE = -4,  /* the health flag saw rho <= 0, T <= 0 or a non-finite value */
  LBM_ETIMEOUT = -5,    /* a bounded device wait ran out */
  LBM_ESTATE = -6       /* the sim failed earlier; only lbm_destroy is meaningful */
} lbm_status;

/* Boundary kinds of the two node layers outside a face (Sec. 4(2)). */
enum {
  LBM_BC_PERIODIC = 0,    /* wrap; both faces of the axis must be periodic */
  LBM_BC_FIXED = 1,       /* both layers hold the given (rho,u1,u2,u3,T) */
  LBM_BC_EXTRAPOLATE = 2, /* g1 = 2 m0 - m1, g2 = 2 g1 - m0 on rho, u, T (needs >= 2 cells) */
  LBM_BC_REFLECT = 3,     /* wall layer: (rho,T,u_t) of the last cell, u_n = 0;
                             outer layer: the last cell with u_n negated */
  LBM_BC_EXTERNAL = 4     /* x faces only (needs >= 2 cells): the two layers hold the
                             neighbouring slab's two columns, written by the caller
                             (lbm_set_halo) before every step; see lbm_set_halo */
};

/* Storage and arithmetic precision of f. */
enum { LBM_FP64 = 0, LBM_FP32 = 1 };

/* Convection scheme: the paper's NND (Sec. 3), the second-order upwind scheme
 * of the original Kataoka-Tsutahara model it is compared with (Sec. 3, Fig. 6),
 * and first-order upwind (the linearisation alpha~ = beta~ = 0 of Sec. 3). */
enum { LBM_SCHEME_NND = 0, LBM_SCHEME_UPWIND2 = 1, LBM_SCHEME_UPWIND1 = 2 };

/* Health flag bits (lbm_health). */
enum { LBM_HEALTH_NONFINITE = 1u, LBM_HEALTH_RHO = 2u, LBM_HEALTH_T = 4u, LBM_HEALTH_TIMEOUT = 8u };

/* Step kernel variants of the FP32 path (lbm_set_launch): TILED = TMA plane
 * tiles of 32 x 8 cells in a four-plane ring (two CTAs of 4 warps per SM),
 * two x-adjacent cells per thread in packed f32x2 arithmetic (default); the
 * step kernel also writes the periodic images and the extrapolated /
 * reflected x-face layers of the state it produces, so no fill launch is
 * needed between steps; TILED64 = the same on 64 x 8 tiles (one CTA of 8
 * warps per SM, run as two halves of 4 warps with their own barriers);
 * TILED_FILL = the TILED kernel with all boundary layers left to a fill
 * launch before each step; TILED_SINGLE = 32 x 8 tiles, one cell per thread;
 * PLAIN = one thread per cell reading global memory; TILED_SPLIT = the TILED
 * tiles and ring with two warp groups per tile, one updating f_0..f_8 and the
 * other f_9..f_14 of every cell pair (both form the moments), so each thread
 * holds half the z-marching state and two CTAs of 8 warps fit on an SM; it
 * writes the same boundary layers as TILED, and TILED, TILED64, TILED_FILL
 * and TILED_SPLIT give bitwise the same results.  lbm_step_batch takes
 * TILED, TILED64 or TILED_SPLIT sims (all the same). */
enum {
  LBM_VARIANT_TILED = 0,
  LBM_VARIANT_PLAIN = 1,
  LBM_VARIANT_TILED_SINGLE = 2,
  LBM_VARIANT_TILED_FILL = 3,
  LBM_VARIANT_TILED64 = 4,
  LBM_VARIANT_TILED_SPLIT = 5
};

/* Grid of nx*ny*nz interior cells of edge dx and the boundary kind of each
 * face; fixed_lo/fixed_hi give (rho,u1,u2,u3,T) for FIXED faces (axis 0=x). */
typedef struct lbm_grid {
  int32_t nx, ny, nz;
  int32_t bc_lo[3], bc_hi[3];
  double fixed_lo[3][5], fixed_hi[3][5];
} lbm_grid;

/* The discrete-velocity constants c1 != c2, eta0 > 0 (Sec. 2) and the
 * specific-heat ratio gamma > 1 (b = 2/(gamma-1), Eq. 2). */
typedef struct lbm_vset {
  double c1, c2, eta0, gamma;
} lbm_vset;

typedef struct lbm_sim lbm_sim;

/* Bytes of device workspace a sim of this grid and precision needs (two
 * padded f buffers, reduction scratch and status words), 0 if the grid is
 * invalid.  Lets a caller admit work by HBM footprint before allocating. */
LBM_API size_t lbm_workspace_bytes(const lbm_grid* grid, int32_t precision);

/* Create a sim on the current CUDA device.  tau is the BGK relaxation time
 * (Eq. 1), dt the time step, dx = dy = dz the cell edge.  d_workspace must be
 * a device allocation of at least lbm_workspace_bytes() bytes, 256-byte
 * aligned; cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * The f state is undefined until lbm_init or lbm_set_f.  Errors: LBM_EINVAL
 * (sizes < 1, c1 == c2, eta0 <= 0, tau/dt/dx <= 0, gamma <= 1, unpaired
 * periodic faces, EXTRAPOLATE with fewer than 2 cells, a padded field of
 * 2^32 or more cells, NULL pointers),
 * LBM_ENOMEM (workspace too small), LBM_ECUDA. */
LBM_API int lbm_create(const lbm_grid* grid, const lbm_vset* vset, double tau, double dt, double dx,
               int32_t precision, void* d_workspace, size_t ws_bytes, void* cuda_stream, lbm_sim** out);

/* Select the convection scheme (LBM_SCHEME_*) and switch the extra
 * dissipation term lambda_i Laplacian(f_i) (Eq. "lp") on (1, default) or off (0). */
LBM_API int lbm_set_scheme(lbm_sim* sim, int32_t scheme, int32_t dissipation);

/* Launch configuration of the FP32 step kernel (the autotuner's knobs):
 * a LBM_VARIANT_* value; zchunk = z planes per CTA (one unit of work) of the
 * tiled kernels, 0 = automatic (chunk and tail chosen from the grid and the
 * SM count; ztail is then ignored); ztail (pair kernels: TILED, TILED_FILL,
 * TILED64 and lbm_step_batch) = 0 for equal chunks, or a length below zchunk:
 * the first floor((nz - ztail) / zchunk) chunks of each tile column have
 * zchunk planes and the rest of the column is split into chunks of ztail
 * planes, launched last, so that the SMs run out of work together.  All
 * variants and chunkings compute the same update (the pair kernels bitwise;
 * the others to float rounding); FP64 sims always use the plain kernel.
 * LBM_EINVAL for an unknown variant or a negative zchunk or ztail. */
LBM_API int lbm_set_launch(lbm_sim* sim, int32_t variant, int32_t zchunk, int32_t ztail);

/* FP64 temperature recovery of the FP32 tiled step (LBM_VARIANT_TILED and
 * lbm_step_batch).  The FP32 T = (E/rho - u^2)/b of Sec. 2 subtracts large
 * terms when c1^2 >> T (the equilibrium's axis and diagonal populations are
 * then large and of opposite sign); its relative rounding error is about
 * 2^-24 kappa with kappa = 1 + (6 c1^2 |A_axis| + 8 c2^2 |A_diag| + u^2)/(b T).
 * Cells with kappa > kappa_max, or with T <= 0 in FP32, recompute rho, u and
 * T from their 15 values in FP64.  kappa_max = 0 turns it off; otherwise
 * kappa_max >= 1 (LBM_EINVAL else).  The paper has no counterpart: it fixes
 * no precision. */
LBM_API int lbm_set_t_recovery(lbm_sim* sim, double kappa_max);

/* Polls the tiled step kernels make on a shared-memory copy barrier before
 * giving up (default 2^22, seconds of waiting).  On giving up a kernel sets
 * LBM_HEALTH_TIMEOUT, lets its copies in flight finish (with the default
 * limit) and returns; lbm_health then reports LBM_ETIMEOUT and the device
 * stays usable.  A small value exercises that path (0 gives up at once). */
LBM_API int lbm_set_wait_limit(lbm_sim* sim, uint32_t polls);

/* f = f^eq(rho, u, T) at every interior cell (Eq. "eq").  Resets the step
 * counter and the health flags.  rho, T > 0 is not checked here; the first
 * step's health flag reports it. */
LBM_API int lbm_init(lbm_sim* sim, const double* rho, const double* u, const double* T, int32_t on_device);

/* Advance n >= 0 time steps: per step one boundary-fill kernel and one fused
 * step kernel on the sim's stream; returns without waiting. */
LBM_API int lbm_step(lbm_sim* sim, int64_t n);

/* (rho, u, T) of every interior cell in double precision (relations e1-e3,
 * T = (E/rho - u^2)/b).  Synchronises the stream. */
LBM_API int lbm_moments(lbm_sim* sim, double* rho, double* u, double* T, int32_t on_device);

/* Copy the interior f out / in, dense [15][nz][ny][nx], in the sim's storage
 * precision (double for LBM_FP64, float for LBM_FP32). */
LBM_API int lbm_get_f(lbm_sim* sim, void* f, int32_t on_device);
LBM_API int lbm_set_f(lbm_sim* sim, const void* f, int32_t on_device);

/* Global (mass, momentum x/y/z, energy) summed over interior cells in double
 * precision by a deterministic reduction (the invariants of relations e1-e3);
 * out is a host array of 5.  Synchronises; returns LBM_ENONFINITE if the
 * health flag is set (out is still written). */
LBM_API int lbm_conserved(lbm_sim* sim, double out[5]);

/* Global (mass, momentum x/y/z, energy) of a dense device array
 * f[15][nz][ny][nx] (the layout lbm_get_f writes, float or double per
 * precision) for callers that cannot allocate device memory: code running
 * while a stream is captured into a CUDA graph, hosts whose allocator owns all
 * of device memory, and monitoring hooks that must not change the device's
 * memory footprint.  The paper has no counterpart; this is a deployment
 * convenience.  No workspace and no allocation: the per-block partial sums
 * live in one static 256 KiB device array that every GPU loading this library
 * keeps until exit.  At most 33,554,432 cells (4096 blocks of 8192 cells);
 * larger grids return LBM_EINVAL.  The first call on a device looks up the
 * array's address, so make it before any stream capture; the address is kept
 * with the id of the device's CUDA context, and after a context reset
 * (cudaDeviceReset) the next call looks it up again.  All calls share the
 * array: calls that overlap on the same GPU race and give wrong sums.  out is
 * 5 doubles, in device memory (out_on_device = 1; asynchronous on
 * cuda_stream) or host memory (the call synchronises cuda_stream; on a stream
 * under capture, which cannot be synchronised, LBM_EINVAL before anything is
 * queued). */
LBM_API int lbm_conserved_noalloc(const void* f, int32_t precision, int32_t nx, int32_t ny, int32_t nz,
                                  const lbm_vset* vset, double* out, int32_t out_on_device, void* cuda_stream);

/* Slab decomposition along x.  A grid cut into x-slabs (one sim per slab,
 * on one or several GPUs) advances exactly as the whole grid when, before
 * every step, each cut face's two outside layers hold the neighbouring
 * slab's two boundary columns: the stencil of Sec. 3 reaches two cells along
 * each axis and no further.  Faces at cuts are LBM_BC_EXTERNAL.
 *   lbm_get_halo_source: the two interior columns next to x face `side`
 *     (0 = lo: x = 0, 1; 1 = hi: x = nx-2, nx-1) of the current state, into
 *     buf, dense [15][nz][ny][2] (x order) in the storage precision
 *     (15 * ny * nz * 2 * 4 or 8 bytes).
 *   lbm_set_halo: writes the two layers outside x face `side` (lo: x = -2,
 *     -1; hi: x = nx, nx+1) from buf, same layout; the face must be
 *     LBM_BC_EXTERNAL.  The lo neighbour's hi source is this slab's lo halo,
 *     the hi neighbour's lo source its hi halo.
 * With on_device = 1 both are asynchronous on the sim's stream (buf a device
 * pointer, valid once the stream reaches the call); with on_device = 0 they
 * stage through the spare f buffer and synchronise.  A sim with EXTERNAL
 * faces steps one step per lbm_step call, after lbm_set_halo on each of its
 * EXTERNAL faces since its previous step (LBM_EINVAL otherwise), and is not
 * taken by lbm_step_batch or lbm_graph_capture.  Errors: LBM_EINVAL (side
 * not 0 / 1, NULL buf, face not EXTERNAL), LBM_ECUDA. */
LBM_API int lbm_get_halo_source(lbm_sim* sim, int32_t side, void* buf, int32_t on_device);
LBM_API int lbm_set_halo(lbm_sim* sim, int32_t side, const void* buf, int32_t on_device);

/* Von Neumann stability (Sec. 3): for each parameter set p, out[p] = the
 * largest spectral radius max |omega| of the amplification matrix G(k) of one
 * step (the paper's G with alpha~ = beta~ = 0: first-order upwind phases,
 * BGK relaxation, the extra dissipation term when dissipation = 1, and the
 * equilibrium Jacobian by the chain rule through rho, u and T) over the
 * uniform states, the wave-vector directions and the wave numbers
 * |k| dx = pi q / nk, q = 1..nk.  states: nstates x (rho, u1, u2, u3, T);
 * params: nparams x (c1, c2, eta0, gamma, dt, tau, dx); dirs: ndirs x 3
 * (normalised here); out: nparams doubles.  All four are device pointers;
 * asynchronous on cuda_stream.  A matrix whose eigenvalue iteration does not
 * converge, or that holds non-finite values, gives +inf.  The paper accepts
 * a scheme when max |omega| <= 1.  Errors: LBM_EINVAL (NULL pointers, counts
 * < 1, more than 2^30 matrices), LBM_ECUDA. */
LBM_API int lbm_vn_max_growth(const double* states, int32_t nstates, const double* params, int32_t nparams,
                              const double* dirs, int32_t ndirs, int32_t nk, int32_t dissipation, double* out,
                              void* cuda_stream);

/* Diagnostic: y[j] = 1/x[j] for n floats as the FP32 step kernels form the
 * inverse density (the hardware approximation rcp.approx.ftz.f32 refined by
 * one Newton-Raphson step): |y x - 1| <= 2^-24 + 2^-40 for 2^-100 <= |x| <=
 * 2^100 and <= 2^-23 for 2^-125 <= |x| <= 2^125 (beyond 2^100 the Newton
 * correction is subnormal), not always the nearest float, never more than
 * one float from it; NaN for x = 0, +-inf, NaN and
 * subnormal x (flushed to zero), 0 for |x| >= 2^127 (a subnormal 1/x is
 * flushed to zero).  d_x, d_y: device arrays
 * (they may be the same array); asynchronous on cuda_stream.  Errors:
 * LBM_EINVAL (n < 0, NULL pointers with n > 0), LBM_ECUDA. */
LBM_API int lbm_reciprocal_fp32(const float* d_x, float* d_y, int64_t n, void* cuda_stream);

/* Synchronise and read the health flag bits (LBM_HEALTH_*) accumulated since
 * lbm_init; returns LBM_ETIMEOUT when a bounded device wait ran out
 * (LBM_HEALTH_TIMEOUT), else LBM_ENONFINITE when any other bit is set. */
LBM_API int lbm_health(lbm_sim* sim, uint32_t* flags);

/* Stream-ordered forms for callers that keep the GPU busy (a serving loop):
 * nothing synchronises; completion is observed with an event recorded on
 * the sim's stream after the call.  lbm_moments_async writes rho, u, T
 * ([nz][ny][nx], u as 3 such planes, FP64) to device memory; lbm_health_async
 * copies the health bits to `flags` (device memory or page-locked host
 * memory; valid once the stream reaches this point).  The paper has no
 * counterpart.  Errors: LBM_EINVAL (NULL pointers), LBM_ECUDA. */
LBM_API int lbm_moments_async(lbm_sim* sim, double* rho, double* u, double* T);
LBM_API int lbm_health_async(lbm_sim* sim, uint32_t* flags);

/* Wait for the sim's stream; reports asynchronous kernel faults. */
LBM_API int lbm_sync(lbm_sim* sim);

/* Steps taken since lbm_init / lbm_set_f. */
LBM_API int64_t lbm_steps_done(const lbm_sim* sim);

/* Most grids one batched step can carry. */
#define LBM_MAX_BATCH 48

/* Advance n sims by `steps` time steps together.  Per step, one launch of the
 * persistent FP32 tile kernel walks a descriptor table holding every grid's
 * tiles (uneven grids, different constants and boundaries are fine), plus a
 * fill launch only for boundary layers that kernel does not write itself.
 * All sims must be FP32 with the default tiled variant and the same scheme,
 * live on the current device and share one stream (sims[0]'s); 1 <= n <=
 * LBM_MAX_BATCH.  Each sim's result is bitwise the one lbm_step gives it
 * alone.  Returns without waiting; LBM_EINVAL on a mismatch. */
LBM_API int lbm_step_batch(lbm_sim* const* sims, int32_t n, int64_t steps);

/* A CUDA graph of `steps` (even, >= 2) time steps of one sim (n = 1, any
 * precision or variant) or of a batch (the lbm_step_batch rules).  Capture
 * launches nothing; each lbm_graph_launch replays all the steps with one
 * graph launch on the sims' stream and advances their step counters.  A
 * replay is refused (LBM_ESTATE) if a sim was stepped an odd number of times
 * outside the graph since the capture (its buffers would be swapped).
 * Graph instantiation allocates driver resources; destroy releases them. */
typedef struct lbm_graph lbm_graph;
LBM_API int lbm_graph_capture(lbm_sim* const* sims, int32_t n, int64_t steps, lbm_graph** out);
LBM_API int lbm_graph_launch(lbm_graph* graph);
LBM_API void lbm_graph_destroy(lbm_graph* graph);

/* Kernel classes of the launch and time accounting below. */
enum { LBM_KERNEL_FILL = 0, LBM_KERNEL_STEP = 1, LBM_KERNEL_REDUCE = 2, LBM_KERNEL_OTHER = 3, LBM_NKERNEL = 4 };

/* Device-time accounting of this sim's kernels: with enable = 1 every launch
 * is bracketed by a pair of CUDA events on the sim's stream (a ring of event
 * pairs, drained as it fills); enable = 0 stops recording.  Launch counts are
 * kept whether or not timing is on.  Creating the events is the only
 * allocation this makes (host-side CUDA event objects). */
LBM_API int lbm_set_timing(lbm_sim* sim, int32_t enable);

/* Synchronise, then report per kernel class (LBM_KERNEL_*) the summed device
 * milliseconds of timed launches and the number of launches since creation
 * or the last reset (reset = 1 clears both after reading).  ms and launches
 * are host arrays of LBM_NKERNEL entries; either may be NULL. */
LBM_API int lbm_get_timing(lbm_sim* sim, double* ms, int64_t* launches, int32_t reset);

/* Human-readable name of a status code (static string). */
LBM_API const char* lbm_status_str(int status);

/* Release the descriptor (not the caller's workspace or stream). NULL is ignored. */
LBM_API void lbm_destroy(lbm_sim* sim);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
