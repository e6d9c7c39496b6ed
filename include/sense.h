/*
 * sense.h -- C ABI of the GB300 non-Fourier SENSE library (libsense.so).
 *
 * The library applies the encoding operator of non-Fourier (higher-order) SENSE and
 * solves its normal equations by conjugate gradients, with the encoding matrix generated
 * on the fly on the GPU and never stored.
 *
 *   Eq. 4     P = e^{o i K R},  E m == P (S o (m 1^T))           (s = E m, [K][C])
 *   Eq. 5     E^H sigma == (S* o (P^H Sigma)) 1                   (m = E^H s, [L])
 *   Fig. 2, Alg. 1: S <- S o j, CG on E^H E rho = E^H sigma from rho = 0,
 *             rho <- rho o j.
 *
 * Notation (variable table of Fig. 2): L voxels, K samples, C (Gamma) coils, P1 = P + 1
 * rows of the spatial basis R / columns of the temporal basis K.
 *
 * Conventions for every entry point:
 *  - Return value: SENSE_OK (0) or a negative SENSE_E* code; nothing aborts or throws.
 *    sense_strerror() names a code; sense_last_error() gives the message of the last
 *    failing call on the calling thread.
 *  - Complex arrays are interleaved single precision (re, im) pairs ("complex64").
 *  - Vector arguments (m, s, x, out) may be DEVICE pointers (the fast path: the call is
 *    asynchronous on `stream`) or HOST pointers (pageable or pinned: the call stages them
 *    through plan-owned device buffers and returns after the results are back in host
 *    memory). The caller owns every buffer it passes; nothing is freed or retained.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - A plan is bound to the device that was current at sense_plan_create(); calls must be
 *    made with that device current. Calls on one plan must not overlap (they share the
 *    plan's workspace); different plans are independent.
 */
#ifndef SENSE_H
#define SENSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SENSE_OK 0
#define SENSE_EINVAL (-1)       /* bad argument: null pointer, size, layout, option  */
#define SENSE_ENOMEM (-2)       /* device or host allocation failed                  */
#define SENSE_ECUDA (-3)        /* a CUDA runtime call failed (see sense_last_error) */
#define SENSE_ENONFINITE (-4)   /* non-finite input, or CG produced a non-finite value */
#define SENSE_EBREAKDOWN (-5)   /* CG breakdown: p^H E^H E p == 0                    */
#define SENSE_EUNSUPPORTED (-6) /* valid but unsupported size (e.g. C > 64 coils)    */
#define SENSE_ENODEVICE (-7)    /* no usable sm_103 device                           */
#define SENSE_ETIMEOUT (-8)     /* a tensor-core kernel gave up waiting (bounded wait) */

typedef struct sense_plan_s* sense_plan;

/* Arithmetic used for the two contractions of E and E^H (the phase is always evaluated
 * the same way, see sense_plan_create). */
typedef enum {
  SENSE_PREC_FP32 = 0,     /* FP32 CUDA cores ("explicit" path)                        */
  SENSE_PREC_TC_FP16 = 1,  /* tcgen05 tensor cores, operands single FP16, FP32 accumulate */
  SENSE_PREC_TC_SPLIT = 2  /* tcgen05, operands split hi+lo FP16 (3 products), FP32 acc. */
} sense_precision;

/* Problem definition (Fig. 2 inputs). All pointers are HOST pointers read during
 * sense_plan_create() only.
 *   Kmat [K][P1] float64  temporal basis: Kmat[k][0] = t_k (s), Kmat[k][p+1] = k_p(t_k)
 *   Rmat [P1][L] float64  spatial basis:  Rmat[0][l] = B0(r_l) as angular frequency
 *                         (rad/s), Rmat[p+1][l] = h_p(r_l); phi = Kmat x Rmat (radians)
 *   S    [L][C]  complex64 coil sensitivities
 *   j    [L]     float32 intensity correction, or NULL for all ones                      */
typedef struct {
  int64_t L;
  int64_t K;
  int32_t C;
  int32_t P1;
  const double* Kmat;
  const double* Rmat;
  const float* S;
  const float* j;
} sense_problem;

/* Create a plan: validates the problem, orders voxels into spatially compact blocks of
 * 128, derives the per-block phase anchors (FP64 on the device) and uploads S o j.
 * Phase evaluation: phi/2pi = A(sample block, l) + B(voxel block, k) + sum_q dK(k,q)
 * dR(l,q), with A and B computed in FP64 and reduced mod 1, and the local bilinear part
 * in FP32 over the rows of K R that vary inside a block.
 * Errors: EINVAL (null pointers, L<1, K<1, C<1, P1<1), EUNSUPPORTED (C > 64, more than 20
 * varying basis rows), ENONFINITE (non-finite Kmat/Rmat/S/j), ENOMEM, ECUDA, ENODEVICE.
 * On success *out owns device memory until sense_plan_destroy().                        */
int sense_plan_create(const sense_problem* prob, sense_plan* out);

/* Release every resource of the plan. NULL is accepted. Returns SENSE_OK or ECUDA. */
int sense_plan_destroy(sense_plan plan);

/* Replace row 0 of R (the B0 map, rad/s, [L] host float64, user voxel order) and rebuild
 * the phase anchors; used when the B0 map itself is optimised. Errors: EINVAL,
 * ENONFINITE, ECUDA. Stream-ordered on `stream`. */
int sense_plan_set_b0(sense_plan plan, const double* omega, void* stream);

/* Wait for the plan's work on `stream` and report a device-side failure recorded since the
 * last check (SENSE_ETIMEOUT when a tensor-core kernel gave up waiting; its outputs are
 * then invalid). Device-pointer calls are asynchronous and report such failures only here
 * or in a later synchronising call. Errors: EINVAL, ECUDA, ETIMEOUT. */
int sense_plan_sync(sense_plan plan, void* stream);

/* Plan dimensions: out[0]=L, out[1]=K, out[2]=C, out[3]=P1, out[4]=number of basis rows
 * kept in the FP32 bilinear part, out[5]=padded L, out[6]=padded K, out[7]=padded C. */
int sense_plan_info(sense_plan plan, int64_t out[8]);

/* s = E m (Eq. 4). m: [L] complex64, s: [K][C] complex64 (device or host, see above). */
int sense_encode(sense_plan plan, int prec, const float* m, float* s, void* stream);

/* m = E^H s (Eq. 5). s: [K][C] complex64, m: [L] complex64. */
int sense_adjoint(sense_plan plan, int prec, const float* s, float* m, void* stream);

/* out = E^H E m (the normal operator of Alg. 1, Fig. 2). m, out: [L] complex64; may alias. */
int sense_normal_op(sense_plan plan, int prec, const float* m, float* out, void* stream);

/* CG options. Stopping: the paper's fixed iteration count N_It (max_iter), optionally
 * also ||r_n|| <= rel_tol ||E^H s|| (the residual of rho = 0). */
typedef struct {
  int32_t max_iter;     /* N_It >= 0                                                   */
  int32_t prec;         /* sense_precision of E^H E inside the iterations              */
  double rel_tol;       /* 0 disables the residual stop                                */
  int32_t refine_every; /* tensor-core modes: replace the recursive residual by
                           b - E^H E x with the FP32 operator every this many
                           iterations (0 = never)                                      */
  int32_t apply_j;      /* nonzero: multiply the result by j (as Alg. 1 ends)          */
  int32_t use_x0;       /* nonzero: x holds the start rho_0 on input (sense_cg_solve and
                           sense_cg_solve_iterates; a solve resumed from an earlier result
                           passes that result computed with apply_j = 0)               */
} sense_cg_opts;

typedef struct {
  int32_t iters;        /* iterations run                                              */
  int32_t status;       /* SENSE_OK, SENSE_EBREAKDOWN or SENSE_ENONFINITE              */
  double rr0;           /* r_0^H r_0                                                   */
  double rr_final;      /* r_n^H r_n at exit                                           */
} sense_cg_info;

/* rho = CG(E^H E, E^H s) (the CG loop of Alg. 1, Fig. 2), starting from rho = 0 or, with
 * opts->use_x0, from the rho_0 given in x (then r_0 = E^H s - E^H E rho_0 and p_0 = r_0, with
 * E^H E in the iteration precision, or FP32 when refine_every > 0). A zero residual at the
 * start (E^H s = 0, or a start that solves the system exactly) ends the solve after 0
 * iterations with SENSE_OK.
 *   s        [K][C] complex64 coil data Sigma (device or host)
 *   x        [L] complex64 output rho (device or host); input rho_0 too with use_x0
 *   history  NULL or HOST double[(max_iter+1)*3]: for n = 0..iters the row
 *            (||r_n||, ||rho_n||, ||E rho_n - s||) -- the L-curve coordinates; the data
 *            residual uses ||E x - s||^2 = ||s||^2 - Re<x,b> - Re<x,r> (r = b - E^H E x)
 *   info     NULL or HOST output
 * Returns SENSE_OK when the loop ran (a CG breakdown is reported in info->status, with
 * rho left at the last finite iterate), or an error code. Synchronises the stream when
 * history, info or a host x is given. */
int sense_cg_solve(sense_plan plan, const float* s, float* x, const sense_cg_opts* opts,
                   double* history, sense_cg_info* info, void* stream);

/* sense_cg_solve that also records every iterate: iterates is DEVICE memory of
 * (max_iter + 1) x L complex64, row n = rho_n in user voxel order (multiplied by j when
 * apply_j, like the result); row 0 is zero (with use_x0: the start rho_0, read from row 0 on
 * input and rewritten times j when apply_j) and rows after a tolerance stop repeat the final
 * iterate; the result itself is row max_iter. Used to study stopping rules against a known
 * image (the paper compares the L-curve corner with SSIM over the iterations). Errors as
 * sense_cg_solve, plus EINVAL for host memory. */
int sense_cg_solve_iterates(sense_plan plan, const float* s, float* iterates,
                            const sense_cg_opts* opts, double* history, sense_cg_info* info,
                            void* stream);

/* Maximum-curvature (L-curve corner) iteration of a CG history of n rows (format of
 * sense_cg_solve; "assessment of the number of CG iterations" in the paper's methods): the
 * curve's points are (log ||E x_i - s||, log ||x_i||) for the iterates i = 1..n-1 (row 0, the
 * start x_0 = 0, is not a point and is never read); curvature by central differences in i,
 * signed positive for the clockwise turn at the corner; candidates i = 2..n-2, first maximum
 * wins. Host-only. *corner = -1 when n < 4 (fewer than three points). Errors: EINVAL. */
int sense_lcurve_corner(const double* history, int32_t n, int32_t* corner);

/* Differentiation ----------------------------------------------------------------------
 * (no counterpart in the paper, which only solves; these serve B0-map refinement and
 * training through the reconstruction)
 * Gradients follow the convention dL/dRe(v) + i dL/dIm(v) of a real loss L.
 *
 * B0 gradient primitive. Row 0 of R is the B0 map omega (rad/s) and column 0 of K the
 * sample time t, so d phi / d omega(l) = t_kappa (Eq. 4). This call computes
 *     grad_omega(l) = Im( conj(a(l)) * (E^H (t o y))(l) )      [L] float, user voxel order
 * and, when z is not NULL, z = E^H y ([L] complex64). It is the backward of both operators:
 *   y_out = E m   with upstream g:  a = m, y = g  ->  dL/domega, and z = dL/dm;
 *   x_out = E^H y with upstream h:  a = h, y = y  ->  dL/domega (dL/dy = E h: sense_encode).
 * a [L] complex64, y [K][C] complex64; host or device pointers. The gradient is that of the
 * operator the plan holds (its current B0 map). Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
int sense_grad_b0(sense_plan plan, int32_t prec, const float* a, const float* y, float* z,
                  float* grad_omega, void* stream);

/* Checkpointed CG solve for reverse-mode differentiation. Runs exactly sense_cg_solve
 * (refine_every must be 0) and writes into ckpt (caller-owned device memory, 16-byte
 * aligned, at least sense_cg_ckpt_bytes() bytes) the residual, search direction and
 * scalars before every ckpt_every-th iteration plus the final scalars, so that
 * sense_cg_backward can replay one segment of ckpt_every iterations at a time: memory is
 * O(max_iter / ckpt_every) vectors for the checkpoints plus ckpt_every vectors (and
 * ckpt_every E p products) held by the plan during the backward.
 * sense_cg_ckpt_bytes returns the size, or a negative error code (EINVAL). */
int64_t sense_cg_ckpt_bytes(sense_plan plan, int32_t max_iter, int32_t ckpt_every);
int sense_cg_solve_ckpt(sense_plan plan, const float* s, float* x, const sense_cg_opts* opts,
                        int32_t ckpt_every, void* ckpt, int64_t ckpt_bytes,
                        sense_cg_info* info, void* stream);

/* Reverse mode through the solve recorded in ckpt: given xbar = dL/dx ([L] complex64) for
 * the returned x, writes sbar = dL/ds ([K][C] complex64) and/or omega_bar = dL/domega
 * ([L] float, user voxel order); either output may be NULL, not both. s must be the data
 * of that solve and the plan must hold the same B0 map. The step lengths are differentiated
 * (the iterate is a nonlinear function of s and omega); the stopping decision is not.
 * Synchronises the stream to read the checkpoint header. Errors: EINVAL (ckpt not written
 * by sense_cg_solve_ckpt on this plan), ENOMEM, ECUDA, ETIMEOUT. */
int sense_cg_backward(sense_plan plan, const float* s, const void* ckpt, int64_t ckpt_bytes,
                      const float* xbar, float* sbar, float* omega_bar, void* stream);

/* s = E m for callers that cannot allocate device memory (the paper has no counterpart).
 * Hosts that reserve all GPU memory at start-up and forbid later allocation, and callers
 * whose device memory is owned by another framework's allocator, can neither create a plan
 * nor let a call allocate. This entry point takes the problem directly and allocates
 * nothing: its only scratch (the partial sums of the voxel-split FP32 encode) is a fixed
 * 16 MiB array inside the library. Phases are evaluated per pair in FP64 (no plan, no
 * anchors), the rest as in the FP32 path.
 *   Kmat [K][P1] float64, Rmat [P1][L] float64, S [L][C] complex64, j [L] float32 or NULL,
 *   m [L] complex64: DEVICE inputs; s [K][C] complex64: DEVICE output (caller-owned).
 * Limits: C <= 64, P1 <= 24, K x (C rounded up to 8/16/32/64) <= 2^21; larger sizes are
 * rejected with SENSE_EINVAL and a message.
 * First call on a device: CUDA loads the library's device code lazily, so the 16 MiB array
 * comes into existence on a device only when this entry point first runs there, and that
 * first call also looks up the array's device address (with that device current) and caches
 * it for the life of the process. A caller that reserves the GPU's memory up front should
 * therefore make one call (any valid size) before reserving, and before any stream capture;
 * from then on the array stays resident on that device until the process exits. The cached
 * address does not survive cudaDeviceReset(): do not call this entry point on a device after
 * resetting it. All calls share the array, which keeps the last call's partial sums; calls
 * that overlap on the GPU (other streams, other host threads) race on it.
 * Asynchronous on `stream`. Errors: EINVAL, EUNSUPPORTED, ECUDA. */
int sense_encode_noalloc(int64_t L, int64_t K, int32_t C, int32_t P1, const double* Kmat,
                         const double* Rmat, const float* S, const float* j, const float* m,
                         float* s, void* stream);

/* k-space filter (the filtering that ends Alg. 1, Fig. 2: rho = IFFT(FFT(rho) o f)) ---------
 * sense_kspace_filter_mask (host only): f for an nx x ny grid of spacing dx, dy (m): 1 for the
 *   Cartesian k-space points k = 2 pi (u - n/2) / (n d) inside (or on) the convex hull of the
 *   K first-order coefficients (kx, ky) (rad/m) of the samples, else 0; mask [ny][nx] host
 *   float. Errors: EINVAL, ENONFINITE.
 * sense_kspace_filter: image [nz][ny][nx] complex64 (DEVICE, raster order = the user voxel
 *   order of a full-grid problem) filtered in place with mask [nz][ny][nx] float (DEVICE),
 *   using the signal model's sign: F(k_u) = sum_x rho(x) e^{+i k_u r_x}, r_x = (x - n/2) d,
 *   then rho(x) = (1/n) sum_u F(k_u) f(u) e^{-i k_u r_x} along every axis of length > 1
 *   (any length up to 4096; a mask of ones returns the image). Synchronises the stream.
 *   Errors: EINVAL, ENOMEM, ECUDA. */
int sense_kspace_filter_mask(int32_t nx, int32_t ny, double dx, double dy, const double* kx,
                             const double* ky, int64_t K, float* mask);
/* 3D: the same for an nx x ny x nz grid (mask [nz][ny][nx]) and samples (kx, ky, kz) that lie on
 * at most 4096 kz planes (stacks of planar trajectories): the hull's cross-section at each grid
 * kz is the 2D convex hull of (1 - t) H_i + t H_j over the plane pairs bracketing it (H_i the 2D
 * hull of plane i), so only 2D geometry is needed. Errors: EINVAL, ENONFINITE, EUNSUPPORTED. */
int sense_kspace_filter_mask3d(int32_t nx, int32_t ny, int32_t nz, double dx, double dy,
                               double dz, const double* kx, const double* ky, const double* kz,
                               int64_t K, float* mask);
int sense_kspace_filter(int32_t nx, int32_t ny, int32_t nz, const float* mask, float* image,
                        void* stream);

/* Map smoothing and extrapolation (Eq. 1: sensitivity maps; Eq. 3: the B0 map) -------------
 * Solves, on an nx x ny x nz grid (raster order, x fastest), the least-squares system of the
 * two equations, A x = [w0 o xhat; 0; 0; 0] with A = [diag(w0); sqrt(alpha) diag(wd) D_x;
 * sqrt(alpha) diag(wd) D_y; sqrt(alpha) diag(wd) D_z], D the second difference (order 2, Eq. 1:
 * w0 = trusted mask M_T, wd = reconstruction mask M_R) or the first difference (order 1, Eq. 3:
 * w0 = 1, wd = the standard error of the phase fit), through its normal equations by CG from
 * x = xhat. Second-difference rows exist at interior voxels, first-difference rows where the
 * next voxel exists; a row is weighted by wd at its voxel; axes of length 1 have none.
 * n_fields right-hand sides share w0 and wd and are solved together, each with its own CG
 * scalars and stop test: xhat, x are [n_fields][n] complex64 (real maps: zero imaginary parts),
 * w0, wd [n] float, all DEVICE memory; x may equal xhat. Voxels that no equation constrains
 * (w0 = 0 and no weighted derivative row touches them) keep xhat. precond selects plain CG or CG
 * preconditioned by one symmetric multigrid V-cycle (Galerkin coarse operators of linear
 * interpolation, Chebyshev smoothing on the diagonal; built on the device at every call; the
 * paper's incomplete-Cholesky choice is sequential and is not offered). info (nullable):
 * [n_fields] host entries, iterations run and the final relative residual of the normal
 * equations per field. Workspace (about 10 field-sized vectors plus the hierarchy) comes from a
 * stream-ordered memory pool the library keeps per device, which retains up to 1 GiB of freed
 * blocks between calls. Synchronises the stream. Errors: EINVAL, ENOMEM, ECUDA. */
#define SENSE_SMOOTH_PLAIN 0
#define SENSE_SMOOTH_MULTIGRID 1
typedef struct {
  int32_t nx, ny, nz;
  int32_t order;      /* 1 or 2                                                         */
  double alpha;       /* smoothness weight (alpha_B or alpha_S)                         */
  int32_t max_iter;
  double rel_tol;     /* stop when ||r|| <= rel_tol ||diag(w0^2) xhat||                 */
  int32_t precond;    /* SENSE_SMOOTH_PLAIN or SENSE_SMOOTH_MULTIGRID                   */
  int32_t n_fields;   /* right-hand sides, 1..65535                                     */
} sense_smooth_opts;

typedef struct {
  int32_t iters;
  double rel_residual;
} sense_smooth_info;

int sense_smooth_map(const sense_smooth_opts* opts, const float* w0, const float* wd,
                     const float* xhat, float* x, sense_smooth_info* info, void* stream);

/* Sensitivity maps as the paper processes them with Eq. 1 (section on sensitivity maps): for
 * every coil the magnitude |S_hat| and the magnitude-normalised map S_hat / |S_hat| (0 where
 * S_hat = 0) are smoothed separately, then recombined as S = m u / |u| (m the smoothed
 * magnitude, u the smoothed normalised map; 0 where u = 0). All 2 C fields are solved in one
 * call of the solver above (opts->n_fields is ignored). S_hat, S: [L][C] complex64 (coil
 * fastest, L = nx ny nz raster order), DEVICE memory, may alias. info (nullable): [2 C] host
 * entries, magnitudes first. Synchronises the stream. Errors: EINVAL, ENOMEM, ECUDA. */
int sense_smooth_sensitivities(const sense_smooth_opts* opts, int32_t C, const float* w0,
                               const float* wd, const float* S_hat, float* S,
                               sense_smooth_info* info, void* stream);

/* Batched reconstruction -----------------------------------------------------------------
 * (no counterpart in the paper, which reconstructs one slice or volume at a time)
 * A batch holds n independent problems of uneven size (voxels, samples, coils, basis rows)
 * and solves them together: each E and E^H of a batch iteration is one persistent launch
 * whose CTAs claim (instance, row block, chunk) work items from a device queue, skipping
 * instances whose CG has stopped; one CG iteration of the whole batch is captured once in a
 * CUDA graph and replayed. All instances share the batch-wide padded coil count and delta
 * row count (zero padding), so the batch costs at most what its largest member's layout
 * costs per (sample, voxel) pair. Tensor-core precisions only (TC_FP16, TC_SPLIT).
 *
 * sense_batch_create: probs[n] as for sense_plan_create (host arrays, copied). The batch
 *   owns one plan per instance; sense_batch_plan returns it (borrowed: do not destroy) for
 *   single-instance calls; after sense_plan_set_b0 on a member plan the next batch call
 *   rebuilds the batch's descriptors. Errors as sense_plan_create, EINVAL for n < 1.
 * sense_batch_info: out = {n, padded coils, delta rows, chunk}.
 * sense_batch_normal_op: out[b] = E_b^H E_b m[b] for every b ([L_b] complex64, device).
 * sense_batch_cg_solve: sense_cg_solve for every instance with the same options (history
 *   not recorded, refine_every must be 0); s[b] [K_b][C_b] and x[b] [L_b] device pointers,
 *   info[n] (nullable; when given the call synchronises and reports ETIMEOUT). Instances
 *   stop individually (rel_tol or max_iter). The first call per precision captures the
 *   iteration graph; concurrent solves on one batch race.
 * sense_batch_set_tuning: streamed blocks per work item (chunk, 1..4096) and accumulator
 *   segment length (1..64); defaults 16 and 4.
 * sense_batch_autotune: times the batched E^H E for chunk in {8,16,32,64} x seg_len in
 *   {2,4} and keeps the fastest; returns it and its time (ms) through the non-null outputs.
 */
typedef struct sense_batch_s* sense_batch;
int sense_batch_create(const sense_problem* probs, int32_t n, sense_batch* out);
int sense_batch_destroy(sense_batch batch);
int sense_batch_plan(sense_batch batch, int32_t i, sense_plan* out);
int sense_batch_info(sense_batch batch, int32_t out[4]);
int sense_batch_normal_op(sense_batch batch, int32_t prec, const float* const* m,
                          float* const* out, void* stream);
int sense_batch_cg_solve(sense_batch batch, const float* const* s, float* const* x,
                         const sense_cg_opts* opts, sense_cg_info* info, void* stream);
int sense_batch_set_tuning(sense_batch batch, int32_t chunk, int32_t seg_len);
int sense_batch_autotune(sense_batch batch, int32_t prec, int32_t* chunk, int32_t* seg_len,
                         double* ms);

/* Stored-P mode (the paper's Alg. 1 choice, offered as a comparison to on-the-fly generation).
 * enable != 0: compute the phase tiles of both passes once (FP16 hi and lo, 8 bytes per
 * (sample, voxel) pair and pass: 2 x 8 x L_p x K_p bytes, 37.6 GB at 256 x 256 and 35750 samples)
 * and from then on stream them from HBM in the tensor-core passes instead of generating them;
 * results are bit-identical in TC_SPLIT mode (TC_FP16 uses the split's hi part). enable == 0
 * frees them. sense_plan_set_b0 regenerates them. Synchronises the stream. Errors: EINVAL,
 * ENOMEM (the tiles do not fit), ECUDA. */
int sense_plan_store_p(sense_plan plan, int32_t enable, void* stream);

/* Tuning ------------------------------------------------------------------------------
 * (no counterpart in the paper: execution parameters of the tensor-core kernels)
 *   seg_len  the tensor-core passes accumulate at most this many 128 x 128 (sample, voxel)
 *            blocks in one FP32 tensor-memory accumulator before adding it to a running
 *            sum; shorter = more accurate, longer = fewer drains. 1..64, or 0 = by precision
 *            (default): 4 for TC_SPLIT, 16 for TC_FP16 (whose FP16 rounding dominates).
 *   grid     persistent CTAs of a tensor-core pass; 0 = one per SM (default).
 *   wait_limit_us  every wait inside a tensor-core pass gives up after this long (measured
 *            in SM clock cycles at the maximum clock); the CTA then records the failure,
 *            completes what it issued, frees its tensor memory and returns, and the next
 *            synchronising call (or sense_plan_sync) reports SENSE_ETIMEOUT. 0 = about 2 s
 *            (default); at most 6e7.
 *   test_hold_stage  for tests of that time-out path only: when > 0, the loader warp of CTA 0
 *            never signals the arrival of its stage number test_hold_stage (counted from 1),
 *            so the waits on it run out; 0 = off (default).
 *   inner_chunk  streamed 128-blocks per chunk of the single-problem schedule: chunk by
 *            chunk, every CTA takes an equal share of the chunk's (row block, streamed block)
 *            pairs, so that the CTAs read the same streamed-side images at about the same time
 *            and find them in L2. 0 = automatic (default): one chunk unless the streamed-side
 *            images of all blocks exceed 32 MiB. A forced value may lower the number of CTAs
 *            (each CTA needs a pair in every chunk). Results are the same up to summation order.
 *            At least 0. */
typedef struct {
  int32_t seg_len;
  int32_t grid;
  int32_t wait_limit_us;
  int32_t test_hold_stage;
  int32_t inner_chunk;
  int32_t reserved[3];
} sense_tuning;

int sense_plan_get_tuning(sense_plan plan, sense_tuning* out);
/* Errors: EINVAL (out-of-range value; the plan is left unchanged), ENOMEM, ECUDA. */
int sense_plan_set_tuning(sense_plan plan, const sense_tuning* t);

/* Diagnostics -------------------------------------------------------------------------
 * (no counterpart in the paper: measurement support for the kernels above)
 * Kernel classes: 0 = tensor-core E pass, 1 = tensor-core E^H pass, 2 = FP32 E kernel,
 * 3 = FP32 E^H kernel. */
typedef struct {
  int64_t launches;      /* kernels this plan launched since the last sense_plan_profile() */
  int64_t timed[4];      /* launches of each class timed with CUDA events (profiling on)   */
  double ms[4];          /* summed event durations of those launches (ms)                 */
} sense_stats;

/* Reset the statistics and switch per-launch event timing of the four kernel classes on
 * (enable != 0) or off. Events are recorded on the stream of each launch. */
int sense_plan_profile(sense_plan plan, int enable);

/* Read the statistics; waits for the recorded events. Errors: EINVAL, ECUDA. */
int sense_plan_stats(sense_plan plan, sense_stats* out);

/* Measured sincos throughput of the current device: a kernel that keeps every SM's
 * special-function unit busy with __sincosf chains; *per_s = sincos evaluations per
 * second over `ms_budget` milliseconds of work (approximately). Errors: EINVAL, ECUDA. */
int sense_diag_sincos_rate(double ms_budget, double* per_s);

/* Host-only views of the single-problem schedule of the tensor-core passes (no device use).
 * sense_diag_chunk_width: the streamed 128-blocks per stream-K chunk that a pass over n_outer
 *   row blocks x n_inner streamed blocks with cp padded coils uses on g CTAs (automatic width:
 *   n_inner unless the streamed-side images exceed 32 MiB). *width out. Errors: EINVAL.
 * sense_diag_stream_k_layout: for chunks of `chunk` streamed blocks, chunk by chunk CTA i takes
 *   the pairs [i W / g, (i + 1) W / g) of the chunk's (row block, streamed block) space (W =
 *   n_outer x chunk width); the partial slot of (chunk c, row block o, CTA i) is
 *   slot_base[c * n_outer + o] + i. Writes slot_base [ceil(n_inner / chunk)][n_outer], nslot
 *   [n_outer] (slots per row block) and *max_slots. Every chunk must give each CTA a pair
 *   (n_outer x narrowest chunk >= g), else EINVAL. */
int sense_diag_chunk_width(int64_t n_outer, int64_t n_inner, int32_t cp, int32_t g,
                           int64_t* width);
int sense_diag_stream_k_layout(int64_t n_outer, int64_t n_inner, int64_t chunk, int32_t g,
                               int32_t* slot_base, int32_t* nslot, int32_t* max_slots);

const char* sense_strerror(int code);
const char* sense_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SENSE_H */
