/*
 * pppm.h -- C ABI of a single-GPU (sm_103a) PPPM solver for the long-range
 * Gaussian-charge electrostatics of Deep Potential Long-Range (DPLR).
 *
 * What is computed (arXiv 2504.15508, Section 2.1):
 *   E_Gt = 1/(2 pi V) sum_{m != 0} exp(-pi^2 m^2 / beta^2) / m^2 |S(m)|^2   (Eq. DPLR:EGt)
 *   S(m) = sum_sites q_j exp(-2 pi i m . r_j)                               (Eq. DPLR:Sm)
 * over ionic sites and Wannier centroids alike (Eq. DPLR:Wn gives the WC
 * positions; to this library every site is a plain charged point), together
 * with the forces -dE_Gt/dr_j (the E_Gt terms of Eq. DPLR:F_inter) and the
 * virial.  The solver is PPPM with ik differentiation ("Poisson-ik", Section
 * 3.1: one forward and three inverse 3D FFTs): order-p B-spline charge
 * assignment, a real-to-complex 3D FFT, a multiply by the optimal influence
 * function with energy and virial reduction, ik-differentiated inverse FFTs,
 * and B-spline interpolation of the field back to every site.
 *
 * Units and conventions
 *   Lengths in Angstrom, charges in e.  beta is the splitting parameter (an
 *   inverse length): a pair of sites interacts as erf(beta r) / r.  E is in
 *   q^2/Angstrom times `prefactor` (default 1; 14.399645 gives eV).  The box is
 *   orthorhombic with edges box[0..2]; the k = 0 term is dropped and the
 *   boundary is conducting.  Virial order: xx, yy, zz, xy, xz, yz, with
 *   Pi_ab = -dE/d(eps_ab) under affine strain.
 *   Positions are AoS n x 3 (x, y, z of site 0, then site 1, ...); they need
 *   not lie inside the box.  Forces are AoS n x 3 in the caller's site order.
 *
 * Memory and streams
 *   Unless an entry point says "host", every array argument is a DEVICE
 *   pointer, owned by the caller, on the device that was current when the
 *   plan was created.  The plan owns its workspace (meshes, influence table,
 *   sort buffers).  Compute calls are asynchronous on the given stream
 *   (a cudaStream_t passed as void*, NULL = legacy default stream) and write
 *   energy and virial to device memory, so a call can be captured in a CUDA
 *   graph once the plan's site capacity covers n (pppm_reserve).
 *   A plan is not thread-safe: one compute at a time per plan.  Its calls
 *   share the workspace, so calls on different streams must be ordered by
 *   the caller (a synchronization or an event wait between them).
 *
 * Errors
 *   Every call returns PPPM_OK (0) or a negative PPPM_ERR_* code; nothing
 *   aborts or traps.  Invalid positions (NaN, Inf, or farther than ~10^6 box
 *   lengths from the origin) are detected on the device: the affected sites
 *   are placed at the origin so that every access stays in bounds, and the
 *   plan's status word records PPPM_ERR_NONFINITE; pppm_status() reads and
 *   clears it (it synchronizes the stream).  The gather's wait for its tile
 *   copies is bounded: one that runs out records PPPM_ERR_TIMEOUT instead,
 *   and that call's forces are invalid.
 */
#ifndef PPPM_H
#define PPPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PPPM_OK = 0,
    PPPM_ERR_INVALID_ARG = -1,  /* NULL pointer, n < 0, beta <= 0, bad precision */
    PPPM_ERR_BAD_MESH = -2,     /* a mesh edge is not 2^a 3^b 5^c, is < order, or > 2048 */
    PPPM_ERR_BAD_ORDER = -3,    /* order outside [2, 7] */
    PPPM_ERR_BAD_BOX = -4,      /* an edge <= 0 or not finite */
    PPPM_ERR_CUDA = -5,         /* a CUDA runtime call failed (no device, out of memory, ...) */
    PPPM_ERR_TIMEOUT = -6,      /* a bounded device-side wait ran out */
    PPPM_ERR_NONFINITE = -7,    /* non-finite or far-away positions were seen */
    PPPM_ERR_TOO_LARGE = -8     /* n or the mesh exceeds what the entry point supports */
};

enum { PPPM_FP32 = 1, PPPM_FP64 = 2 };

typedef struct pppm_plan pppm_plan;

typedef struct {
    double prefactor;   /* multiplies E, forces and virial (default 1.0) */
    int alias;          /* alias range a of the influence-function numerator, n in [-a,a]^3 (default 2) */
    int tile;           /* edge of the spread/gather tiles in mesh cells, 0 = automatic (default 0) */
} pppm_options;

/* Default options. */
int pppm_default_options(pppm_options *opt);

/*
 * Create a plan for one orthorhombic box.
 *   box[3]    edge lengths (Angstrom), host array
 *   mesh[3]   mesh points per edge, each 2^a 3^b 5^c, >= order, <= 2048
 *   order     B-spline assignment order p in [2, 7] (p^3 stencil points)
 *   beta      splitting parameter of Eq. DPLR:EGt (inverse Angstrom), > 0
 *   precision PPPM_FP32 (spread/FFT/gather in FP32; energy and virial terms
 *             summed per thread in FP32, the partials combined with
 *             compensated FP32 pairs and an FP64 final sum) or PPPM_FP64
 * The influence function (computed in FP64 on the device) and the FFT twiddles
 * are built here.  The current CUDA device is used and recorded.
 */
int pppm_create(const double box[3], const int mesh[3], int order, double beta,
                int precision, pppm_plan **out);
int pppm_set_options(pppm_plan *plan, const pppm_options *opt); /* rebuilds G if alias changed */
int pppm_get_options(const pppm_plan *plan, pppm_options *opt);
/* Grow the per-site workspace to at least n sites (compute calls grow it on demand). */
int pppm_reserve(pppm_plan *plan, int64_t n);
void pppm_destroy(pppm_plan *plan);
const char *pppm_strerror(int code);
/* Text of the last CUDA failure behind a PPPM_ERR_CUDA on the calling thread
 * (static thread-local buffer, "" if none). */
const char *pppm_last_error(void);
/* Read and clear the device status word (synchronizes the plan's last stream). */
int pppm_status(pppm_plan *plan);

/*
 * One force evaluation (Eqs. DPLR:EGt, DPLR:Sm and the E_Gt part of
 * DPLR:F_inter) over n sites, asynchronous on `stream`.
 *   pos     n x 3 positions        (device; double for pppm_compute, float for _f32)
 *   q       n charges              (device; same type as pos)
 *   energy  1 double               (device)
 *   forces  n x 3                  (device; same type as pos; overwritten)
 *   virial  6 doubles              (device)
 * Works with plans of either precision; the plan's precision sets the
 * arithmetic.  n = 0 gives zero energy and virial.
 */
int pppm_compute(pppm_plan *plan, void *stream, const double *pos, const double *q, int64_t n,
                 double *energy, double *forces, double *virial);
int pppm_compute_f32(pppm_plan *plan, void *stream, const float *pos, const float *q, int64_t n,
                     double *energy, float *forces, double *virial);

/*
 * The same evaluation from HOST arrays (pinned or pageable), synchronous:
 * energy, forces and virial are in the host arrays on return.  pos and q are
 * copied to plan-owned device buffers (at full copy-engine speed from pinned
 * memory), the forces come back by one copy.  From the second call with the
 * same n and plan state the device part is a replay of a graph captured by
 * the first.  Returns the
 * device status too (PPPM_ERR_NONFINITE if bad positions were seen,
 * PPPM_ERR_TIMEOUT if a bounded device-side wait ran out).
 */
int pppm_compute_host(pppm_plan *plan, const double *pos, const double *q, int64_t n,
                      double *energy, double *forces, double *virial);
int pppm_compute_host_f32(pppm_plan *plan, const float *pos, const float *q, int64_t n,
                          double *energy, float *forces, double *virial);

/*
 * Stages of the path, exposed for testing each one on its own.  Mesh arrays
 * are in the plan's precision (float or double), row-major with z fastest:
 * real meshes Nx x Ny x Nz, complex half spectra Nx x Ny x (Nz/2+1) of
 * interleaved (re, im) pairs.
 *
 * pppm_spread     charge density rho_p = sum_i q_i W W W / (hx hy hz)
 *                 (order-p B-spline assignment, periodic) into rho.
 * pppm_fft_r2c    unnormalised forward 3D DFT of a real mesh: out(k) = sum_p in_p e^{-i k.x_p}.
 * pppm_fft_c2r    unnormalised inverse 3D DFT of a Hermitian half spectrum
 *                 (imaginary parts of the kz = 0 and kz = Nz/2 planes are ignored).
 * pppm_influence  copy the optimal influence function G (half spectrum,
 *                 Nx x Ny x (Nz/2+1) doubles, FP64 as computed) to `G`.
 * pppm_fields     the three field meshes E_x, E_y, E_z (3 consecutive real
 *                 meshes) that the force interpolation reads.
 */
int pppm_spread(pppm_plan *plan, void *stream, const double *pos, const double *q, int64_t n, void *rho);
int pppm_fft_r2c(pppm_plan *plan, void *stream, const void *in, void *out);
int pppm_fft_c2r(pppm_plan *plan, void *stream, const void *in, void *out);
int pppm_influence(pppm_plan *plan, double *G);
int pppm_fields(pppm_plan *plan, void *stream, const double *pos, const double *q, int64_t n, void *fields);

/*
 * Batched form: many independent orthorhombic boxes (e.g. water boxes of
 * uneven size) evaluated by ONE persistent kernel launch, recorded in a CUDA
 * graph and replayed on later calls with the same pointers.  FP32 arithmetic
 * as in PPPM_FP32 plans.  The paper evaluates one box per run; batching is this
 * library's own form, not a method of the paper.
 *
 * pppm_batch_create
 *   nbox           number of boxes, 1..65535
 *   boxes          nbox x 3 edge lengths (host)
 *   meshes         nbox x 3 mesh sizes (host), or NULL: per axis the smallest
 *                  2^a 3^b 5^c >= L / 1.2 (spacing <= 1.2 Angstrom); every size
 *                  must be 2^a 3^b 5^c in [order + 3, 512]; the tile edge 8
 *                  needs every axis of every box >= order + 7, else the batch
 *                  runs with tile edge 4 (forcing 8 then gives PPPM_ERR_BAD_MESH)
 *   order          3, 5 or 7
 *   beta           as in pppm_create
 * pppm_compute_batched
 *   pos, q         all boxes' sites concatenated (float, device), box b owning
 *                  sites offsets[b] .. offsets[b+1]-1
 *   offsets        nbox + 1 int64 (DEVICE); read back to the host on each call
 *                  (a synchronization point) to detect a change of layout
 *   energies       nbox doubles (device); virials nbox x 6 doubles (device)
 *   forces         n x 3 floats (device), in the concatenated site order
 *   The first call (and every call after the offsets change) times both tile
 *   edges (4 and 8 mesh cells) and keeps the faster: the autotuner.  Unless the
 *   stream is capturing or is the legacy stream, the work is recorded into a
 *   CUDA graph, re-recorded when any pointer changes.
 *   Stage dependencies inside the kernel are bounded waits; a wait that runs
 *   out sets PPPM_ERR_TIMEOUT in the batch status (pppm_batch_status).
 * pppm_batch_set       prefactor, tile edge (0 = autotune, 4, 8) and the spin
 *                      limit of the bounded waits.
 * pppm_batch_set_dft   lines of length <= max_len (0..18; default 0 = off)
 *                      are transformed as a DFT matrix product on the tensor
 *                      cores (mma.sync TF32 with split operands, FP32
 *                      accuracy) instead of by the FFT: the small boxes'
 *                      meshes (X = F_N x per axis, as in the paper's DFT
 *                      formulation of its distributed FFT, Section
 *                      "Hardware-offloaded 3D FFT").
 * pppm_batch_set_quantized
 *                      group > 0 (1..18; default 0 = off): every line whose
 *                      length is <= 18 and a multiple of group is transformed
 *                      as the paper's int32-quantised distributed DFT
 *                      (Section "Hardware-offloaded 3D FFT", its quantisation
 *                      panel): the line is split into nodes of group
 *                      consecutive points, each node's partial sum for every
 *                      output is computed in FP32, multiplied by scale (the
 *                      paper's 10^7; 1 .. 1e15), rounded to the nearest
 *                      integer and clamped to int32, and the nodes' integers
 *                      are added exactly before dividing by scale.  What is
 *                      transformed: the charge per mesh point (sum of q W)
 *                      forward, the field spectra divided by N h^3 backward.
 *                      It takes precedence over pppm_batch_set_dft.  An
 *                      accuracy ablation, not a fast path, built for order 5
 *                      only (another order: PPPM_ERR_INVALID_ARG): a clamped
 *                      partial sum makes pppm_batch_status return
 *                      PPPM_ERR_TOO_LARGE.
 * pppm_batch_meshes    copy the nbox x 3 meshes in use to a host array.
 * pppm_batch_tile      tile edge in use (0 before the first call).
 */
typedef struct pppm_batch pppm_batch;
int pppm_batch_create(int nbox, const double *boxes, const int *meshes, int order, double beta,
                      pppm_batch **out);
int pppm_batch_set(pppm_batch *batch, double prefactor, int tile, long long spin_limit);
int pppm_batch_set_dft(pppm_batch *batch, int max_len);
int pppm_batch_set_quantized(pppm_batch *batch, int group, double scale);
/* pppm_batch_set_launch: the launch form.  PPPM_BATCH_PERSISTENT runs every
 * stage of every box in the one persistent launch described above;
 * PPPM_BATCH_STAGED runs one kernel per stage over that stage's work items of
 * all boxes (ten launches, recorded in the same graph), stream order taking
 * the place of the in-kernel waits, so each stage gets its own register and
 * shared-memory budget; PPPM_BATCH_AUTO (default) lets the autotuner time
 * both with the tile edges and keep the fastest.  The two forms run the same
 * stage code but are compiled separately, so results agree to rounding, not
 * bit for bit; each form is deterministic.  The wait probe and the spin limit
 * apply to the persistent form only.  Another mode: PPPM_ERR_INVALID_ARG.
 * pppm_batch_launch: the form in use (the requested one before the first
 * call).  The paper has no counterpart. */
enum { PPPM_BATCH_PERSISTENT = 0, PPPM_BATCH_STAGED = 1, PPPM_BATCH_AUTO = 2 };
int pppm_batch_set_launch(pppm_batch *batch, int mode);
int pppm_batch_launch(const pppm_batch *batch);
/* pppm_batch_set_wait_probe: when on (nonzero), the scan stage of box 0 waits
 * for one binning item more than the box has, so that bounded wait must run
 * out after the spin limit: the launch ends, pppm_batch_status returns
 * PPPM_ERR_TIMEOUT and box 0's results are not written.  A test of the
 * timeout path without any fault; off by default. */
int pppm_batch_set_wait_probe(pppm_batch *batch, int on);
int pppm_batch_meshes(const pppm_batch *batch, int *meshes);
int pppm_batch_tile(const pppm_batch *batch);
int pppm_compute_batched(pppm_batch *batch, void *stream, const float *pos, const float *q,
                         const int64_t *offsets, double *energies, float *forces, double *virials);
int pppm_batch_status(pppm_batch *batch);
void pppm_batch_destroy(pppm_batch *batch);

/*
 * pppm_spread_noalloc -- the charge spread of pppm_spread (FP32 arithmetic,
 * float density rho, same layout and scaling) for callers that cannot
 * allocate device memory: code running inside a host callback or an allocator
 * hook, in a process whose device memory is owned by another framework's
 * pool, or in a plugin that must not grow its footprint at run time.  The
 * paper has no counterpart; this is a deployment convenience.
 *   box, mesh, order  as in pppm_create (host arrays); no plan is needed
 *   stream            cudaStream_t as void*
 *   pos, q            n x 3 positions and n charges, double, device
 *   rho               Nx x Ny x Nz floats, device, written
 * It calls no cudaMalloc/cudaFree: its scratch is one file-scope device array
 * of 32 MiB that every GPU loading this library holds until the process exits.
 * Inputs needing more scratch than that (about 52 B per site plus
 * 4 B x (T+p-1)^3 per tile of T^3 mesh cells, T = 8 or 4) return
 * PPPM_ERR_TOO_LARGE.  All calls share the array and it keeps the last call's
 * contents (the per-tile counters are cleared by each call); calls whose work
 * overlaps on the GPU (other streams or threads) race on it and must be
 * serialized.  The first call on a device looks up the array's device address
 * and uploads the B-spline coefficients, so make it before any stream
 * capture.  Every call puts only memsets and kernel launches on the stream
 * (the fold's cover lists are built on the device, in the scratch array); no
 * host memory is read after the call returns.  Non-finite positions are
 * placed at the origin without a status.
 */
int pppm_spread_noalloc(const double box[3], const int mesh[3], int order, void *stream,
                        const double *pos, const double *q, int64_t n, float *rho);

/*
 * pppm_set_potential -- when on (nonzero), every later compute call of an FP32
 * plan also writes the mesh potential phi (the inverse FFT of G(k) rho_hat(k),
 * Eq. DPLR:EGt's reciprocal-space potential, same scaling as the field meshes)
 * into a padded mesh of the plan's own workspace (allocated by the first call
 * with on; PPPM_ERR_CUDA if that fails); it costs one more inverse z
 * transform.  Used by the correction network below.  Off by default.
 */
int pppm_set_potential(pppm_plan *plan, int on);

/*
 * pppm_set_dependent_launch -- when on (nonzero, the default), the kernels of
 * one evaluation are launched with programmatic dependent launch: each may be
 * scheduled while its predecessor's last blocks run and waits on the device
 * for the predecessor to complete before touching memory.  That removes the
 * gaps between kernels of a plan running alone; when other work shares the
 * GPU concurrently (another stream), the early-scheduled blocks hold SM
 * resources that work could use, and off may overlap better.  Results are
 * identical either way.  A graph captured before the change no longer
 * matches the plan (pppm_graph_launch refuses it).
 */
int pppm_set_dependent_launch(pppm_plan *plan, int on);

/*
 * pppm_set_wait_limit -- polls of the gather's bounded wait for each tile's
 * field copy (default 2^26).  A wait that runs out records PPPM_ERR_TIMEOUT
 * in the plan's status word and the tile's forces are not written; the block
 * then waits once more (bounded) so that its copy lands before it exits.
 * 0 makes every first wait run out: a way to test the timeout path without
 * any fault.  spins < 0: PPPM_ERR_INVALID_ARG.  A graph captured before the
 * change no longer matches the plan.  The paper has no counterpart.
 */
int pppm_set_wait_limit(pppm_plan *plan, long long spins);

/*
 * Learned coarse-mesh correction.  A coarse-mesh FP32 PPPM is corrected per
 * site by a small network over local features of the coarse mesh potential;
 * the network is trained on forces of a fine-mesh PPPM of the same
 * configurations.  The paper's accuracy table (Section "Evaluation",
 * Table "Error of the energy and force") shows coarse FFT meshes keeping the
 * force error of the fine one, which motivates a cheaper coarse solve; the
 * network itself has no counterpart in the paper.
 *
 *   features x_i (n_in BF16 values per site, row-major n x n_in), n_in = 32
 *   for the stated feature set (PPPM_CORR_STATED: local potential samples and
 *   site type) and 48 for the cell set (PPPM_CORR_CELL, the default: the same
 *   and the site's offset inside its mesh cell):
 *     x_i[9 a + 3 b + c] = s_in * phi(r_i + h * (a-1, b-1, c-1)), a, b, c in
 *     {0, 1, 2}, phi interpolated from the coarse potential mesh with the
 *     plan's order-p B-spline weights (h = box / mesh per axis);
 *     x_i[27 + t] = 1 for the site type t in {0, 1, 2}, 0 otherwise;
 *     stated set: x_i[30..31] = 0;
 *     cell set: x_i[30 + 2 d] = sin(2 pi u_d), x_i[31 + 2 d] = cos(2 pi u_d),
 *     d = x, y, z, with u_d = x_d N_d / L_d (the site's offset inside its
 *     mesh cell); x_i[36..47] = 0.
 *   network  h1 = tanh(W1 x + b1) (64), h2 = tanh(W2 h1 + b2) (64),
 *            y = W3 h2 + b3 (3).  Parameters: one FP32 vector of
 *            pppm_corr_param_count() values [W1 64 x n_in row-major, b1, W2
 *            64x64, b2, W3 3x64, b3]: 7491 for the cell set, 6467 for the
 *            stated set.  Inference and training use them rounded to BF16;
 *            accumulation is FP32.
 *   forces   F_i = F_coarse,i + q_i * s_out * y_i.
 *   training target t_i = (F_fine,i - F_coarse,i) / (q_i * s_out) (n x 3
 *            FP32); loss = (1/nb) sum over the nb sites of |y_i - t_i|^2;
 *            Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master weights.
 *
 * pppm_corr_create      borrow an FP32 coarse plan (it must outlive the
 *                       corrector; its potential output is switched on);
 *                       parameters start at zero, s_in = s_out = 1; the cell
 *                       feature set.
 * pppm_corr_create_features
 *                       the same with the feature set chosen (PPPM_CORR_CELL
 *                       or PPPM_CORR_STATED; another value:
 *                       PPPM_ERR_INVALID_ARG).
 * pppm_corr_nparams     7491 (the parameter count of the cell set).
 * pppm_corr_param_count parameters of this corrector (7491 or 6467).
 * pppm_corr_feature_width
 *                       n_in of this corrector (48 or 32).
 * pppm_corr_set_weights host FP32 parameters and the scales s_in, s_out (> 0);
 *                       resets the Adam moments and step count.
 * pppm_corr_get_weights host copy of the FP32 master parameters and scales
 *                       (s_in, s_out may be NULL).
 * pppm_corr_features    run the coarse PPPM on (pos, q) (device, FP32, n x 3
 *                       and n), write its forces to forces (device n x 3) and
 *                       the features to feat (device, n x n_in BF16, 96 or
 *                       64 B per row, 16-byte aligned); types is a device
 *                       array of n signed chars.
 * pppm_corr_calibrate   choose the scales from one configuration: runs the
 *                       coarse PPPM and the features with s_in = 1, then sets
 *                       s_in = 1 / rms of the 27 potential samples and
 *                       s_out = rms over sites and axes of
 *                       (F_fine - F_coarse) / q (f_fine: device n x 3, the
 *                       fine-mesh forces of the same sites).  Synchronizes
 *                       the stream; PPPM_ERR_NONFINITE if a scale is 0 or
 *                       not finite.  Does not touch the parameters.
 * pppm_corr_get_scales  current s_in, s_out.
 * pppm_corr_targets     training targets t_i = (f_fine,i - f_coarse,i) /
 *                       (q_i s_out), 0 where q_i = 0 (device n x 3 FP32).
 * pppm_corr_forward     y = network(feat) for n feature rows -> out (device
 *                       n x 3 FP32); feat must be 4-byte aligned
 *                       (PPPM_ERR_INVALID_ARG otherwise, nothing launched).
 * pppm_corr_set_forward the kernel that runs the network forward (in
 *                       pppm_corr_forward and pppm_corr_apply):
 *                       PPPM_FORWARD_MMA_SYNC (the default) runs the
 *                       warp-level mma.sync kernel, 16 sites a warp, the
 *                       layers chained in registers; PPPM_FORWARD_TCGEN05
 *                       runs each layer as tcgen05.mma instructions, 128
 *                       sites a tile, with the accumulators in tensor memory
 *                       (a feature pointer that is not 16-byte aligned runs
 *                       the mma.sync kernel).  Both take BF16 weights and
 *                       activations and accumulate in FP32; their results
 *                       agree to rounding (on the workloads, bitwise).
 * pppm_corr_set_wait_limit polls of the tcgen05 forward's wait for each MMA
 *                       completion (default 2^26).  A wait that runs out
 *                       sets PPPM_ERR_TIMEOUT in the coarse plan's status
 *                       word (pppm_status); the CTA then waits once more
 *                       (bounded) for the MMA in flight, frees its tensor
 *                       memory and ends without writing its remaining rows.
 *                       0 makes every first wait run out: a way to test the
 *                       timeout path without any fault.  spins < 0:
 *                       PPPM_ERR_INVALID_ARG.
 * pppm_corr_apply       corrected PPPM: coarse compute (energy, virial:
 *                       device doubles, uncorrected) and forces + q s_out y.
 * pppm_corr_grad        loss and its gradient w.r.t. the parameters over the
 *                       nb rows idx[0..nb) of the nrows-row tables feat /
 *                       target (idx device int32, NULL = rows 0..nb, then
 *                       nb <= nrows; an index outside [0, nrows) counts as a
 *                       row that contributes nothing); grad: device, 7491
 *                       floats; loss: device float (may be NULL).
 *                       Deterministic: fixed-order sums, no atomics.
 * pppm_corr_train_step  the same gradient, then one Adam step with learning
 *                       rate lr (> 0); the BF16 copies are refreshed.
 * pppm_corr_save/load   binary checkpoint: "PPPMCORR", version 1, parameter
 *                       count, s_in, s_out, Adam step, master parameters and
 *                       both Adam moments.  Resuming from it continues
 *                       training bit for bit.
 * All calls are asynchronous on the given stream except set/get/save/load,
 * which synchronize the device.  Errors: PPPM_ERR_INVALID_ARG for null or
 * inconsistent arguments or an unreadable checkpoint, PPPM_ERR_CUDA.
 */
typedef struct pppm_corr pppm_corr;
enum { PPPM_CORR_CELL = 0, PPPM_CORR_STATED = 1 };
enum { PPPM_FORWARD_TCGEN05 = 0, PPPM_FORWARD_MMA_SYNC = 1 };
int pppm_corr_create(pppm_plan *coarse, pppm_corr **out);
int pppm_corr_create_features(pppm_plan *coarse, int features, pppm_corr **out);
int pppm_corr_nparams(void);
int pppm_corr_param_count(const pppm_corr *corr);
int pppm_corr_feature_width(const pppm_corr *corr);
int pppm_corr_set_weights(pppm_corr *corr, const float *params, double s_in, double s_out);
int pppm_corr_get_weights(const pppm_corr *corr, float *params, double *s_in, double *s_out);
int pppm_corr_features(pppm_corr *corr, void *stream, const float *pos, const float *q,
                       const signed char *types, int64_t n, void *feat, float *forces);
int pppm_corr_calibrate(pppm_corr *corr, void *stream, const float *pos, const float *q,
                        const signed char *types, int64_t n, const float *f_fine);
int pppm_corr_get_scales(const pppm_corr *corr, double *s_in, double *s_out);
int pppm_corr_targets(pppm_corr *corr, void *stream, const float *f_fine, const float *f_coarse,
                      const float *q, int64_t n, float *target);
int pppm_corr_set_forward(pppm_corr *corr, int kind);
int pppm_corr_set_wait_limit(pppm_corr *corr, long long spins);
int pppm_corr_forward(pppm_corr *corr, void *stream, const void *feat, int64_t n, float *out);
int pppm_corr_apply(pppm_corr *corr, void *stream, const float *pos, const float *q,
                    const signed char *types, int64_t n, double *energy, float *forces,
                    double *virial);
int pppm_corr_grad(pppm_corr *corr, void *stream, const void *feat, const float *target,
                   int64_t nrows, const int *idx, int64_t nb, float *grad, float *loss);
int pppm_corr_train_step(pppm_corr *corr, void *stream, const void *feat, const float *target,
                         int64_t nrows, const int *idx, int64_t nb, float lr, float *loss);
int pppm_corr_save(const pppm_corr *corr, const char *path);
int pppm_corr_load(pppm_corr *corr, const char *path);
void pppm_corr_destroy(pppm_corr *corr);

/*
 * pppm_wc_fold -- long-range force on atoms from the site forces, the fold of
 * Eq. DPLR:F_final.  A Wannier centroid sits at W_n = R_host(n) + Delta_n(R)
 * (Eq. DPLR:Wn); by the chain rule of Eq. DPLR:F_inter the force on atom j is
 *   F_j = F_site[j] + sum over the WCs n hosted by j of F_site[n_atoms + n]
 *         + sum over the blocks (n, J) of row j of J^T F_site[n_atoms + n],
 * with J = dDelta_n/dR_j (3 x 3, row-major: J[a][b] = dDelta_{n,a}/dR_{j,b}),
 * supplied by the caller (in DPLR, by the Deep Wannier model).
 *   f_sites        (n_atoms + n_wc) x 3, device: the PPPM forces of the atoms
 *                  (sites 0..n_atoms-1) then of the WCs, e.g. pppm_compute's
 *                  output when the sites are ordered that way
 *   host_ptr/wc    compressed rows (n_atoms + 1 offsets, device int32): the
 *                  WCs each atom hosts; NULL for none
 *   jac_ptr/wc/jac compressed rows (n_atoms + 1 offsets, device int64; WC
 *                  index per block, device int32; 9 values per block, device):
 *                  the blocks of the WCs whose displacement depends on each
 *                  atom; NULL for none
 *   f_atoms        n_atoms x 3, device, written
 *   status         device int or NULL: bit 0 is set (atomically) if a WC
 *                  index was outside [0, n_wc); that entry is skipped
 * Row offsets must be non-decreasing and inside the arrays (not checked).
 * Asynchronous on the stream; each atom's sum has a fixed order, so the
 * result is bitwise reproducible.  The paper computes this in its MD code;
 * here it is one warp per atom streaming the Jacobian once.
 */
int pppm_wc_fold(void *stream, int64_t n_atoms, int64_t n_wc, const double *f_sites,
                 const int *host_ptr, const int *host_wc, const int64_t *jac_ptr,
                 const int *jac_wc, const double *jac, double *f_atoms, int *status);
int pppm_wc_fold_f32(void *stream, int64_t n_atoms, int64_t n_wc, const float *f_sites,
                     const int *host_ptr, const int *host_wc, const int64_t *jac_ptr,
                     const int *jac_wc, const float *jac, float *f_atoms, int *status);

/*
 * Captured steps.  pppm_graph_create runs one ordinary compute call on the
 * stream (so that every buffer is allocated), then captures a second one as a
 * CUDA graph.  pppm_graph_launch replays it on a stream; pos and q may be new
 * device pointers (NULL: keep the previous ones), which are patched into the
 * one kernel that reads them, so a run can hand a different resident frame to
 * every step without a copy.  The site count, the outputs (energy, forces,
 * virial) and the plan's options are those of the capture: to change them,
 * destroy the graph and create a new one.  The stream must not be the legacy
 * default stream, and per-kernel timing (pppm_profile_enable) must be off.
 * Replays of one graph must not overlap each other or other calls on the same
 * plan (they share its workspace).  Destroy the graph before the plan.
 * A launch fails with PPPM_ERR_INVALID_ARG once the plan has changed since
 * the capture (an option, the potential output, or a workspace reallocation
 * by a compute call with more sites or another tile size); create a new graph.
 * Errors: PPPM_ERR_INVALID_ARG (null or empty arguments, profiling on, input
 * precision differing from the capture's, plan changed), PPPM_ERR_CUDA.
 */
typedef struct pppm_graph pppm_graph;
int pppm_graph_create(pppm_plan *plan, void *stream, const double *pos, const double *q, int64_t n,
                      double *energy, double *forces, double *virial, pppm_graph **out);
int pppm_graph_create_f32(pppm_plan *plan, void *stream, const float *pos, const float *q, int64_t n,
                          double *energy, float *forces, double *virial, pppm_graph **out);
int pppm_graph_launch(pppm_graph *graph, void *stream, const double *pos, const double *q);
int pppm_graph_launch_f32(pppm_graph *graph, void *stream, const float *pos, const float *q);
void pppm_graph_destroy(pppm_graph *graph);

/*
 * Per-kernel timing (for benchmarks).  While enabled, every kernel launch of a
 * compute call is bracketed by CUDA events on the compute stream.
 * pppm_profile_read synchronizes, writes for each kernel slot i < cap the
 * accumulated milliseconds ms[i] and launch count calls[i] (host arrays, may
 * be NULL), resets the accumulators and returns the number of slots.
 * pppm_profile_name(i) names slot i (static string, "" if out of range).
 */
int pppm_profile_enable(pppm_plan *plan, int on);
int pppm_profile_read(pppm_plan *plan, double *ms, int64_t *calls, int cap);
const char *pppm_profile_name(int slot);

#ifdef __cplusplus
}
#endif

#endif /* PPPM_H */
