/*
 * lbm.h -- C ABI of the GB300 D3Q27 colour-fluid lattice Boltzmann library.
 *
 * The library advances the two-colour (red r / blue b) lattice Boltzmann model
 * of Saito, Abe & Koyama (arXiv 1705.03141), Sec. II: D3Q27 velocities
 * (Eq. velSet), MRT collision with the moment set of Eq. (momentSet) and the
 * relaxation matrix K, the enhanced equilibrium Eq. (EES) with phi_i^k
 * (Eq. varphi_ik) and Phi_i^k (Eq. Phi), MRT body forcing Eqs. (ketF)-(ketFd),
 * the generalised perturbation operator Eq. (perturb), recolouring (Sec. II),
 * streaming (Eq. LBE) and the jet boundaries of Sec. IV.A (circular
 * equilibrium inlet, free-slip walls, convective outflow).
 *
 * Conventions for every call:
 *  - Every call returns an lbm_status and never aborts the process.  NULL
 *    handles or pointers, bad sizes or bad parameters give LBM_EINVAL; the
 *    text of the last error is available from lbm_last_error().
 *  - Scalar fields are SoA arrays of N = nx*ny*nz doubles with x fastest:
 *    idx = x + nx*(y + ny*z).  Vector fields are three such arrays back to
 *    back (u_x, then u_y, then u_z).
 *  - Population arrays are [2][27][nz][ny][nx] doubles: colour (0 red,
 *    1 blue), then the direction i = 1..27 in the paper's order (the order of
 *    rows 2-4 of the printed M, App. A), then the node.  They hold the
 *    post-streaming populations f_i^k(x, t) at the handle's current time t.
 *  - Every buffer a caller passes is caller-owned; the library never frees it
 *    and never keeps a pointer to it after the call returns.  Such a buffer
 *    may be host memory or device memory of the handle's device; the library
 *    detects which.
 *  - Device work is enqueued on the handle's CUDA stream (lbm_params.cuda_stream,
 *    or the legacy default stream when NULL).  lbm_step() only enqueues;
 *    calls that return data (lbm_macro, lbm_diag, lbm_get_populations) and
 *    lbm_synchronize() wait for that stream.
 *  - One handle is used by one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#if defined(__GNUC__)
#define LBM_EXPORT __attribute__((visibility("default")))
#else
#define LBM_EXPORT
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,    /* invalid argument, size or parameter */
  LBM_ENOMEM = -2,    /* device or host allocation failed, or workspace too small */
  LBM_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
  LBM_EUNSTABLE = -4, /* the watchdog saw a non-finite or non-positive density */
  LBM_ETIMEOUT = -5,  /* a bounded device-side wait ran out (the TMA-pipelined pass 1 of compact storage) */
  LBM_ESTATE = -6     /* call not valid in the handle's current state */
} lbm_status;

/* How populations are held in device memory.  All collision arithmetic is
 * FP32 except in LBM_STORE_F64, which computes in FP64 and is the mode that
 * matches the FP64 CPU oracle.  LBM_STORE_F16 / LBM_STORE_BF16 keep, per
 * direction and node, the total population as a deviation from its
 * rest-state value in half / bfloat16 plus the red fraction f^r/f as an
 * unsigned 16-bit fixed-point number (4 bytes per direction and node).
 * LBM_STORE_F16C / LBM_STORE_BF16C (compact) keep the total population of
 * each moving direction as a half / bfloat16 deviation from its rest value
 * (2 bytes), the rest direction's total in FP32, and one FP32 record per node
 * (frac, m) from which the recolouring of Sec. II fixes the colour split of
 * everything the node emitted: f^r_i = frac f_i + (w_i/|c_i|) c_i.m (72 bytes
 * per node in all).  Compact storage runs collide-stream variant 1 only and
 * has no z-slab exchange; after lbm_init_fields or lbm_set_populations its
 * per-colour populations are available again (lbm_get_populations) after the
 * first step. */
typedef enum {
  LBM_STORE_F64 = 0,
  LBM_STORE_F32 = 1,
  LBM_STORE_F16 = 2,
  LBM_STORE_BF16 = 3,
  LBM_STORE_F16C = 4,
  LBM_STORE_BF16C = 5
} lbm_storage;

/* Face conditions, faces ordered (-x, +x, -y, +y, -z, +z).
 *  PERIODIC    both faces of an axis must be periodic.
 *  NOSLIP      halfway bounce-back (Sec. III.C walls).
 *  FREESLIP    specular reflection of the wall-normal velocity component
 *              (Sec. IV.A wall boundary).
 *  INFLOW_WALL a free-slip wall whose plane carries the circular inlet set by
 *              lbm_set_inflow(); only allowed on -z.
 *  OUTFLOW     convective outflow of Sec. IV.A; only allowed on +z.
 *  HALO        the z face joins the box to a neighbouring z-slab of a larger
 *              domain held by another handle (spatial decomposition along z,
 *              possibly on another GPU or process); only allowed on -z / +z.
 *              Populations crossing the face and the densities the gradient
 *              stencil reads across it come from the neighbour through the
 *              halo exchange below; such a handle steps with lbm_step_pass.
 * Gradients next to a non-periodic face use a mirror ghost value (zero
 * normal gradient). */
typedef enum {
  LBM_BC_PERIODIC = 0,
  LBM_BC_NOSLIP = 1,
  LBM_BC_FREESLIP = 2,
  LBM_BC_INFLOW_WALL = 3,
  LBM_BC_OUTFLOW = 4,
  LBM_BC_HALO = 5
} lbm_bc;

/* Body force F(x, t) used in Eq. (Momentum) and Eq. (ketFd).
 *  NONE       F = 0.
 *  BUOYANCY   F = (rho - (rho_r0 + rho_b0)/2) g  (Rayleigh-Taylor, Sec. III.C;
 *             gravity acts on the density excess over the mean initial density).
 *  DISPERSED  F = (rho - rho_b0) g  (jet, Eq. bodyForceJet).
 *  UNIFORM    F = g  (a constant force density). */
typedef enum {
  LBM_FORCE_NONE = 0,
  LBM_FORCE_BUOYANCY = 1,
  LBM_FORCE_DISPERSED = 2,
  LBM_FORCE_UNIFORM = 3
} lbm_force;

typedef struct {
  double rho_r0, rho_b0; /* initial phase densities; gamma = rho_r0/rho_b0 sets
                            alpha_r = 1 - (1 - alpha_b)/gamma with alpha_b = 8/27
                            (Grunau relation and the choice of alpha_b, Sec. II) */
  double nu_r, nu_b;     /* kinematic viscosities; per node
                            nu_bar = (1+phi)/2 nu_r + (1-phi)/2 nu_b and
                            s6 = s8 = 1/(3 nu_bar + 1/2) (Eq. shear) */
  double A, beta;        /* perturbation strength of Eq. (perturb) (A_r = A_b = A)
                            and recolouring parameter beta */
  double s[27];          /* relaxation rate of each moment of Eq. (momentSet), in
                            moment order; the entries of the s6 and s8 slots
                            (moments 6-10) are ignored and replaced by the local
                            shear rate; all rates must lie in [0, 2) */
  double g[3];           /* gravity / force vector of the force mode */
  int force_mode;        /* lbm_force */
  int bc[6];             /* lbm_bc per face (-x,+x,-y,+y,-z,+z) */
  int storage;           /* lbm_storage */
  unsigned long long seed; /* seed of the inlet velocity noise */
  void* cuda_stream;     /* cudaStream_t to enqueue on; NULL = legacy default stream */
  void* workspace;       /* optional caller-owned device memory for all device
                            state (populations, density field, buffers); must
                            hold lbm_workspace_size() bytes, be 256-byte
                            aligned and outlive the handle.  NULL: the library
                            allocates (cudaMalloc) and frees it itself. */
  size_t workspace_bytes;
  int variant;           /* collide-stream kernel: 0 = library's choice (3 for F32
                            storage with nx a multiple of 32, 5 for F16/BF16
                            storage, 1 otherwise: the measured faster ones),
                            1 = one node per thread, 2 = two x-adjacent nodes per
                            thread with packed FP32x2 arithmetic (needs F32/F16/BF16
                            storage and an even nx), 3 = one node per thread with
                            the fused density pass: the collide-stream kernel also
                            accumulates the next step's densities, so the separate
                            density pass is skipped (needs F32/F16/BF16 storage),
                            4 = one node per thread, software-pipelined: persistent
                            blocks copy the next tile's populations into shared
                            memory while computing the current one (needs F16/BF16
                            storage), 5 = the interior tiles (every row away from
                            the y and z faces) by persistent blocks of 8 consumer
                            warps and one producer warp that stages each tile's
                            population words and (rho, phi) halo in shared memory
                            with TMA copies, the remaining tiles by variant 1
                            (needs F16/BF16 storage; where an x face is periodic or
                            no-slip, nx is odd or the box has no interior tile,
                            variant 5 runs variant 1 throughout, with the same
                            results).  Variants 1 and 5 give bitwise the same
                            fields.  All variants compute the same update; they
                            differ in FP32 rounding (variant 3 also rounds the
                            densities that enter the gradients to fixed point), and
                            each is bitwise reproducible.  F32/F16/BF16 storage needs
                            rho_r0, rho_b0 <= 64. */
  int block;             /* thread-block shape of the one-node density and
                            collide-stream kernels (variants 1 and 3, FP32
                            arithmetic): 0 = library's choice (32x2x4 for variant 3
                            in F32 storage, else 32x4x2: the measured faster ones),
                            1 = 32x4x2 nodes, 2 = 32x2x4, 3 = 32x8x1 (a warp is one
                            32-node x-row in each).  Variant 1 computes the same
                            update bitwise in every shape; variant 3 differs by FP32
                            rounding (how the next step's densities are grouped
                            before their exact fixed-point sum).  FP64 storage
                            always runs 32x4x2.  Compact storage (F16C/BF16C) runs
                            32x4x2 tiles with one of two density passes: 1 = one
                            block per tile, 4 = persistent blocks of 8 consumer
                            warps and one producer warp that streams each tile's
                            totals and colour records into a 3-stage shared-memory
                            ring with TMA copies (needs x faces that are neither
                            periodic nor no-slip; the library's choice there, and
                            bitwise the same densities as 1).  Any other storage
                            with block 4, or compact storage with 2 or 3, gives
                            LBM_EINVAL. */
} lbm_params;

typedef struct lbm lbm; /* opaque handle; owns all device state it allocated */

/* Bytes of device workspace a handle of this size and storage needs. */
LBM_EXPORT lbm_status lbm_workspace_size(int nx, int ny, int nz, const lbm_params* p, size_t* bytes);

/* Create a handle for an nx x ny x nz box (each >= 3) on the current CUDA
 * device.  Validates and copies *p, derives alpha_r, sets the populations to
 * the rest state of pure blue fluid (rho_b = rho_b0) and the time to 0.  The
 * handle must be released with lbm_free(). */
LBM_EXPORT lbm_status lbm_create(int nx, int ny, int nz, const lbm_params* p, lbm** out);

/* Initial state (t = 0): f^k = f^{k(e)}(rho_k, u, alpha_k) of Eq. (EES) with
 * Phi = 0.  rhoR, rhoB: N doubles each; u: 3N doubles or NULL for rest.
 * Host or device pointers.  Resets the outflow plane history. */
LBM_EXPORT lbm_status lbm_init_fields(lbm* h, const double* rhoR, const double* rhoB, const double* u);

/* Circular equilibrium inlet of Sec. IV.A on the z = 0 plane: the nodes with
 * (x-xc)^2 + (y-yc)^2 < (D/2)^2 emit f^r = f^{r(e)}(rho_r0, u_in, alpha_r)
 * (Phi = 0) and f^b = 0 every step, u_in = (0, 0, u_j0) plus, per node, step
 * and component, u_j0 * noise_frac * xi with xi uniform in [-1, 1) from
 * SplitMix64 keyed by (seed, step, node index, component).  Requires
 * bc[4] == LBM_BC_INFLOW_WALL.  D <= 0 removes the inlet. */
LBM_EXPORT lbm_status lbm_set_inflow(lbm* h, double xc, double yc, double D, double u_j0, double noise_frac);

/* Enqueue n >= 0 time steps: per step a density/phase-field pass, the fused
 * collide-perturb-recolour-stream pass (in place, AA pattern) and, with an
 * outflow face, the convective outflow update.  Asynchronous: returns after
 * enqueueing.  Returns LBM_EUNSTABLE if a watchdog flag raised by earlier
 * steps has already been observed by a synchronising call.  Runs of 16 steps
 * replay a captured CUDA graph; with the environment variable LBM_NO_GRAPHS
 * set (read once per process) every step is launched directly instead (the
 * same kernels and results, for tools that do not follow graphs).  The
 * collide-stream pass of the two-pass FP32-arithmetic kernels stages each
 * block's (rho, phi) halo tile with one TMA copy; with LBM_NO_TMA set when a
 * step is launched or captured, the tiles are loaded thread by thread (the
 * same values, bitwise the same results). */
LBM_EXPORT lbm_status lbm_step(lbm* h, int n);

/* Macroscopic fields at the current time: rho_r, rho_b (N each) and
 * u = (sum_i sum_k f_i^k c_i + F/2)/rho (3N), Eq. (Momentum).  Any output
 * pointer may be NULL.  Host or device pointers.  Synchronises. */
LBM_EXPORT lbm_status lbm_macro(lbm* h, double* rhoR, double* rhoB, double* u);

/* Diagnostics at the current time, reduced on the device in FP64 with a
 * fixed summation order (bitwise reproducible):
 *   mass_rb[2]       sum of rho_r and of rho_b over all nodes;
 *   z_leading_edge   the jet's leading edge (Sec. IV.B): largest z of a node
 *                    with phi > 0, refined by linear interpolation of the
 *                    phi = 0 crossing towards z+1 (-1 if no node has phi > 0);
 *   dp_laplace       the Laplace pressure jump of Sec. III.A (Eq. lap): mean
 *                    pressure over nodes with phi > 0.99 minus mean over
 *                    nodes with phi < -0.99, p = sum_k rho_k 9(1-alpha_k)/19
 *                    (Eq. press); 0 if either set is empty.
 * Host pointers; any may be NULL.  Synchronises. */
LBM_EXPORT lbm_status lbm_diag(lbm* h, double* mass_rb, double* z_leading_edge, double* dp_laplace);

/* Copy out / in the post-streaming populations ([2][27][nz][ny][nx], see the
 * conventions above).  lbm_set_populations also sets the time to t >= 0 and
 * the outflow plane history to the given top plane.  Host or device
 * pointers.  In F16/BF16 storage the values are decoded / encoded. */
LBM_EXPORT lbm_status lbm_get_populations(lbm* h, double* f);
LBM_EXPORT lbm_status lbm_set_populations(lbm* h, const double* f, long long t);

/* Take n >= 1 steps with direct kernel launches, timing each launch with CUDA
 * events recorded on the handle's stream (the stream the kernels run on).
 * ms_out[0..2] receive the mean device time per launch, in milliseconds, of
 * the density pass, the collide-stream pass and the outflow pass (0 when the
 * box has no outflow face).  Synchronises; advances the time by n. */
LBM_EXPORT lbm_status lbm_profile_step(lbm* h, int n, double* ms_out);

/* Switch the stream later calls enqueue on (NULL = legacy default stream). */
LBM_EXPORT lbm_status lbm_set_stream(lbm* h, void* cuda_stream);

/* Wait for the handle's stream; reports LBM_EUNSTABLE if the watchdog fired. */
LBM_EXPORT lbm_status lbm_synchronize(lbm* h);

/* Current time step index t (number of steps taken since initialisation). */
LBM_EXPORT long long lbm_time(const lbm* h);

/* Number of kernel launches one lbm_step(h, 1) enqueues (the fused density
 * pass also enqueues one memset per step, not counted; longer runs launch the
 * outflow kernel once per run: lbm_launch_count counts exactly). */
LBM_EXPORT int lbm_kernels_per_step(const lbm* h);

/* Kernel launches the handle's stepping calls (lbm_step, lbm_autotune, lbm_batch_step) have
 * enqueued since lbm_create: each CUDA-graph replay counts the kernels the graph holds.  The
 * fused density pass's memset is not a kernel and is not counted.  Runs of two-pass steps with
 * an outflow face launch the outflow kernel once, after their last step (the outflow of each
 * earlier step runs at the start of the next step's density pass).  -1 for NULL. */
LBM_EXPORT long long lbm_launch_count(const lbm* h);

/* The collide-stream kernel variant the handle runs (1 to 5; see
 * lbm_params.variant and lbm_autotune); -1 for NULL. */
LBM_EXPORT int lbm_kernel_variant(const lbm* h);

/* The block shape the handle's one-node kernels run (1 = 32x4x2, 2 = 32x2x4,
 * 3 = 32x8x1, 4 = 32x4x2 tiles with the TMA-pipelined compact density pass:
 * lbm_params.block, the library's choice, or the one lbm_autotune chose); -1
 * for NULL. */
LBM_EXPORT int lbm_kernel_block(const lbm* h);

/* Last error message of this handle ("" if none); valid until the next call. */
LBM_EXPORT const char* lbm_last_error(const lbm* h);

/* Name of a status code. */
LBM_EXPORT const char* lbm_status_string(lbm_status s);

/* The 27x27 transformation matrix M the kernels apply (row-major; row j is
 * moment j+1 of Eq. momentSet, column i is the paper's direction i+1), for
 * checking against App. A.  Host-only: needs no GPU. */
LBM_EXPORT lbm_status lbm_moment_matrix(double* M);

/* Check the library's own lattice tables on the host (moment basis against
 * Eq. momentSet, orthogonality, weights, velocity order).  Needs no GPU.
 * Returns LBM_OK or LBM_EINVAL with a message in *msg (static storage). */
LBM_EXPORT lbm_status lbm_selfcheck(const char** msg);

/* Pick the fastest collide-stream kernel for this handle by measurement: take
 * `steps` steps (>= 1) with each available variant (1; 2 where the storage and
 * nx allow; 3 for F32/F16/BF16 storage; 4 and 5 for F16/BF16 storage), variants 1
 * and 3 in each of the three block shapes of lbm_params.block (FP32-arithmetic
 * storages other than compact; compact storage: block 1 and, where its x faces
 * allow, block 4), timed with CUDA events on the handle's stream,
 * keep the fastest (variant, shape) for later steps and report the variant in
 * *chosen (1 to 5; may be NULL; lbm_kernel_block gives the shape).  The tuning
 * steps are ordinary time steps of the same update, so the time advances by
 * steps times the number of candidates tried.  Synchronises. */
LBM_EXPORT lbm_status lbm_autotune(lbm* h, int steps, int* chosen);

/* Batched stepping of several independent boxes (e.g. the jets of a regime
 * sweep): one CUDA graph holds, per handle, its own chain of kernels as an
 * independent branch, so one graph launch advances every box and boxes of
 * different sizes run concurrently.  The handles stay owned by the caller and
 * must outlive the batch; they must all be at the same step parity (t mod 2)
 * whenever lbm_batch_step is called (LBM_ESTATE otherwise).  Work goes on
 * cuda_stream (NULL = legacy default stream), ordered after the work already
 * queued on each handle's own stream, and each handle's stream is made to
 * wait for it, so per-handle calls before and after a batch step stay in
 * stream order.  The graph records each handle's kernel choice when first
 * launched: autotune before stepping. */
typedef struct lbm_batch lbm_batch;
LBM_EXPORT lbm_status lbm_batch_create(lbm* const* handles, int n, void* cuda_stream, lbm_batch** out);
/* Advance every handle by n >= 0 steps (graph launches of 16 steps, then
 * single steps).  Asynchronous. */
LBM_EXPORT lbm_status lbm_batch_step(lbm_batch* b, int n);
/* Wait for the batch's stream; LBM_EUNSTABLE if any handle's watchdog fired. */
LBM_EXPORT lbm_status lbm_batch_synchronize(lbm_batch* b);
/* Release the batch (not the handles).  NULL is a no-op. */
LBM_EXPORT void lbm_batch_free(lbm_batch* b);

/* Measured FP32 CUDA-core throughput of the current device (a measurement
 * utility; the paper has no counterpart): the ALU roof of the stepping
 * kernels, whose arithmetic is FP32 FMA/ADD/MUL.  Runs 8 independent FMA
 * chains per thread on 8 blocks of 256 threads per SM (packed != 0: the same
 * FLOPs as packed FP32x2 FMAs), best of three timed launches on cuda_stream
 * (NULL = legacy default stream), and writes TFLOP/s (2 per FMA) to *tflops.
 * Allocates and frees a small device buffer; synchronises. */
LBM_EXPORT lbm_status lbm_measure_fp32_peak(void* cuda_stream, int packed, double* tflops);

/* Self-test of the primitives of the TMA-pipelined density pass (a utility; the
 * paper has no counterpart).  One block issues a tiled TMA copy of a 16 x 16
 * box of a 32 x 32 FP32 tensor into shared memory, completing on one mbarrier
 * with its byte count, and arms a second mbarrier for 16 bytes that no copy
 * delivers.  *copy_ok = 1 if the copy completed with the expected values;
 * *timed_out = 1 if the bounded wait on the second barrier gave up after
 * wait_cycles SM clock cycles (1 .. 2e9) instead of spinning: the mechanism
 * behind LBM_ETIMEOUT.  Runs on cuda_stream (NULL = legacy default stream),
 * allocates and frees two small device buffers, synchronises.  LBM_EINVAL for
 * NULL outputs or wait_cycles out of range; LBM_ECUDA if the driver offers no
 * tensor-map encoder or a CUDA call fails. */
LBM_EXPORT lbm_status lbm_selftest_tma(void* cuda_stream, long long wait_cycles, int* copy_ok, int* timed_out);

/* Allocation-free diagnostics; the paper has no counterpart (it is an
 * interface for callers, not part of the method).  Reduces caller-owned device
 * fields rhoR, rhoB (N = nx*ny*nz doubles each, x fastest, e.g. filled by
 * lbm_macro into device buffers) to out[0..3] = {mass_r, mass_b,
 * z_leading_edge, dp_laplace}, defined exactly as in lbm_diag; rho_r0/rho_b0
 * give alpha_r as in lbm_create and must satisfy the same range (density
 * ratio >= 19/27), else LBM_EINVAL.
 * It exists for callers that cannot allocate device memory: code whose host
 * framework owns every device allocation through its own pool, or loops that
 * forbid cudaMalloc and the synchronisation it implies.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.  Its only scratch, the
 * per-block partial sums, is a static device array of 3.7 MB that every GPU
 * loading this library holds until the process exits; boxes above 16,777,216
 * nodes (65536 blocks of 256) are rejected with LBM_EINVAL.  The first call
 * on a device looks up that array's device address (set-up): make that first
 * call before any stream capture.  All calls share the array and leave their
 * contents in it; every slot a call reads is written by the same call first,
 * so nothing needs clearing, but calls that overlap on the GPU (several
 * streams or host threads at once) race on it.  rhoR and rhoB must be device
 * (or managed) memory of the current device, else LBM_EINVAL; the host cannot
 * check that they hold N doubles.  Work goes on cuda_stream (NULL = legacy
 * default stream) of the current device; out may be device memory of that
 * device, or host memory, in which case the call synchronises the stream: a
 * host out is refused with LBM_EINVAL while cuda_stream is being captured, so
 * under capture out must be device memory.  *err (may be NULL) receives a
 * static message. */
LBM_EXPORT lbm_status lbm_diag_fields_static(const double* rhoR, const double* rhoB, int nx, int ny, int nz,
                                             double rho_r0, double rho_b0, double* out, void* cuda_stream,
                                             const char** err);

/* ---- Spatial decomposition along z (z-slabs) -------------------------
 * A domain of nx x ny x NZ nodes can be split into slabs nx x ny x nz_k, one
 * handle each (same nx, ny, storage and parameters; faces between slabs are
 * LBM_BC_HALO, the outer z faces keep the domain's conditions, or are HALO
 * both ways round for a domain periodic in z).  The split run computes
 * exactly the single-domain update (Eq. LBE with the collision of Sec. II is
 * local except for the 26-neighbour gradient stencil and the streaming to
 * neighbours, both one node deep): each node gets the same inputs, so FP64
 * and FP32 results are bitwise those of one handle over the whole domain.
 *
 * Slab handles do not accept lbm_step, lbm_profile_step, lbm_autotune or a
 * batch (LBM_ESTATE); they use the fused-density variant 3 nowhere (the
 * default becomes 1; asking for 3 gives LBM_EINVAL).  One time step of the
 * decomposed domain, with the exchange of a phase meaning: for every pair of
 * adjacent slabs (lower L, upper U), pack(L, +z) -> unpack(U, -z) and
 * pack(U, -z) -> unpack(L, +z) through a buffer of lbm_halo_bytes:
 *     lbm_step_pass(h, 1) on every slab        (density / phase field)
 *     exchange LBM_HALO_DENS                   (the (rho, phi) planes next to each face)
 *     lbm_step_pass(h, 2) on every slab        (collide-stream (+ outflow); t advances)
 *     exchange LBM_HALO_POP_IN  if the step just taken was even (t now odd)
 *     exchange LBM_HALO_POP_OUT if it was odd (t now even)
 * With the in-place AA pattern an even step writes only a node's own slots,
 * and the odd step that follows reads and writes the slots of its
 * neighbours: POP_IN hands each slab a copy of the slots its odd step reads
 * across a face (those of the neighbour's boundary plane holding the
 * populations that move across the face, 9 directions per colour, into
 * this slab's ghost plane), and POP_OUT returns what the odd step wrote into
 * the ghost plane to the neighbour's boundary plane.  After each step the slabs' states are complete: fields,
 * populations and diagnostics of each slab are those of its part of the
 * domain (lbm_diag's leading edge and pressure means are per slab).
 *
 * Buffers are device memory of the handle's device (for another device or
 * process, copy them there: a plain byte buffer).  Pack and unpack are
 * stream-ordered copies on the handle's stream; unpack must not start before
 * the matching pack has completed (same stream, an event, or a
 * synchronisation in between). */
typedef enum {
  LBM_HALO_DENS = 0,     /* pack: the (rho, phi) plane next to the face; unpack: into the halo plane */
  LBM_HALO_POP_IN = 1,   /* pack: boundary plane, populations leaving through the face; unpack: into the ghost plane */
  LBM_HALO_POP_OUT = 2   /* pack: ghost plane, populations leaving through the face; unpack: into the boundary plane */
} lbm_halo_phase;
/* Bytes of one face's message of a phase (the same for both faces). */
LBM_EXPORT lbm_status lbm_halo_bytes(const lbm* h, int phase, size_t* bytes);
/* face: 4 = -z, 5 = +z (must be LBM_BC_HALO).  buf: device memory of
 * lbm_halo_bytes(phase) bytes.  Asynchronous on the handle's stream. */
LBM_EXPORT lbm_status lbm_halo_pack(lbm* h, int face, int phase, void* buf);
LBM_EXPORT lbm_status lbm_halo_unpack(lbm* h, int face, int phase, const void* buf);
/* One pass of one time step: pass 1 = density / phase-field pass, pass 2 =
 * collide-stream pass (+ outflow; advances the time).  Passes alternate 1, 2,
 * 1, 2, ... (LBM_ESTATE otherwise).  Asynchronous.  Allowed on any handle. */
LBM_EXPORT lbm_status lbm_step_pass(lbm* h, int pass);

/* Release the handle and all device memory it allocated (not a caller
 * workspace).  NULL is a no-op. */
LBM_EXPORT void lbm_free(lbm* h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
