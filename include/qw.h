/*
 * qw.h -- C ABI of the GB300 Dirac quantum-walk library (libqw.so).
 *
 * The walk is the Dirac quantum walk of D'Ariano, Mosco, Perinotti, Tosini,
 * "Discrete Time Dirac Quantum Walk in 3+1 Dimensions" (Entropy 2016):
 * a 2-component spinor field on the periodic chain (Sec. 3.2, decoupled 1D
 * walk) or a 4-component field on the periodic square lattice (Eq. weyl2d) or
 * BCC lattice (Eqs. bcc-vecs, weyl3d), coupled by the mass m with n^2 + m^2 = 1
 * (Sec. 3.2).  One step is the update rule of Eq. upd-rule,
 *     psi'(x) = sum_{h in S + {0}} U_h psi(x - h),
 * whose Fourier symbol is D_k = sum_h exp(-i k.h) U_h (Eq. walk-K).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Field layout ("device layout"), complex values interleaved (re, im):
 *   dim 1: [s=2][x]          N sites
 *   dim 2: [s=4][y][x]       N x N sites, lattice coordinates (x, y) = (a, b)
 *                            along h1 = (1,0), h2 = (0,1)
 *   dim 3: [c=2][s=4][z][y][x], M = N/2 cells per axis.  Coset c holds the BCC
 *                            site with physical coordinates 2*(x,y,z) + c*(1,1,1)
 *                            of the periodic box [0,N)^3 (Sec. 4, the vertex set
 *                            2Z^3 u (2Z^3 + t)); N must be even.
 * Element type: QW_C64 = two float32 (8 bytes), QW_C128 = two float64 (16 bytes).
 * Field pointers are DEVICE pointers (cudaMalloc / torch CUDA tensors) unless a
 * name says _host; they must be aligned to the element size and hold
 * qw_plan_field_elems(plan) elements.  The caller owns them.  Kernels that move
 * 16-byte vectors (the VEC/TMA/TMA2 stencils, paired projections) run only on
 * 16-byte aligned fields; a complex64 field that is merely 8-byte aligned gets
 * the scalar kernels (same results).
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls are asynchronous on that stream unless stated otherwise.
 * Errors: every call returns a qw_status and never aborts; a failed CUDA call
 * gives QW_ECUDA.  qw_last_error() returns the message of the calling thread's
 * last failure.  Plans are not thread-safe: one host thread per plan at a time.
 */
#ifndef QW_H
#define QW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QW_OK = 0,
  QW_EINVAL = 1,    /* bad argument (dimension, size, mass, null pointer, ...) */
  QW_ENOMEM = 2,    /* device or host allocation failed                     */
  QW_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed           */
  QW_ETIMEOUT = 4,  /* a bounded device- or host-side wait gave up           */
  QW_EAGAIN = 5,    /* not admitted now (budget / queue full); try later     */
  QW_EBUSY = 6,     /* object in use                                         */
  QW_ENOTFOUND = 7  /* unknown ticket                                        */
} qw_status;

typedef enum { QW_C64 = 0, QW_C128 = 1 } qw_dtype;

/* Kernel used by qw_step.  All variants compute the same update; they differ in
 * data movement.  PLAIN: any geometry and dtype, one thread per site.  VEC: BCC,
 * complex64, N/2 % 64 == 0; two cells per thread, 16-byte loads.  TMA: BCC,
 * complex64, N/2 % 64 == 0; z-marching CTAs with TMA-staged shared-memory tiles.
 * TMA2: as TMA with two steps fused per pass over HBM (temporal fusion; an odd
 * remaining step runs as TMA).  FUSED: any lattice and size, complex64; box
 * tiles of the field with a halo loaded into shared memory, `depth` steps per
 * launch (temporal fusion of depth 2..4, tile box and depth set by
 * qw_plan_set_fusion or the autotuner).  AUTO restores the default, the
 * fastest measured on GB300: TMA2 where supported, FUSED for complex64 chains,
 * else TMA > VEC > PLAIN; qw_plan_autotune measures every variant (FUSED with
 * several depths and boxes) and keeps the fastest. */
typedef enum {
  QW_STENCIL_AUTO = 0,
  QW_STENCIL_PLAIN = 1,
  QW_STENCIL_VEC = 2,
  QW_STENCIL_TMA = 3,
  QW_STENCIL_TMA2 = 4,
  QW_STENCIL_FUSED = 5
} qw_stencil_variant;

typedef struct qw_plan_s* qw_plan;

/* Observables of one field (Sec. 5.2): the norm sum_x |psi(x)|^2; the mean
 * position <x_i> = sum_x x_i |psi(x)|^2 / norm per axis in the fixed window
 * [0, N) of the periodic box (physical coordinates in 3D, lattice coordinates
 * in 2D; unused axes are 0); the weights of the positive- and negative-
 * frequency parts (eigenvalue exp(-+i omega_k) of D_k, Eq. eigen-D), i.e.
 * sum_k psi^_k^dag (I +- G_k/sin(omega_k))/2 psi^_k / sum_k |psi^_k|^2 where
 * D_k = cos(omega_k) I - i G_k; at sin(omega_k) = 0 both halves share. */
typedef struct {
  double norm;
  double x_mean[3];
  double w_particle;
  double w_antiparticle;
} qw_obs;

/* Last error message of the calling thread ("" if none).  Never NULL. */
const char* qw_last_error(void);

/* Library version string. */
const char* qw_version(void);

/* Create a plan for the walk of dimension `dim` (1, 2 or 3) on the periodic box
 * of side N (N >= 2; even for dim 3), mass m in [0, 1] (n = sqrt(1 - m^2),
 * Sec. 3.2) and element type `dtype`.  Allocates on the current CUDA device a
 * scratch field of the same size (ping-pong buffer) and small reduction
 * buffers; the plan owns them.  *out receives the plan.
 * Errors: QW_EINVAL (bad dim/N/m/dtype, null out), QW_ENOMEM, QW_ECUDA. */
qw_status qw_plan_create(int dim, int64_t N, double mass, qw_dtype dtype, qw_plan* out);

/* Release a plan and its device memory (synchronises the device first). */
qw_status qw_plan_destroy(qw_plan plan);

/* Number of complex elements of one field in the device layout
 * (s * sites: 2N, 4N^2, or 2*4*(N/2)^3); -1 for a null plan. */
int64_t qw_plan_field_elems(qw_plan plan);

/* Number of lattice sites (N, N^2, or N^3/4 for the BCC box); -1 for null. */
int64_t qw_plan_sites(qw_plan plan);

/* Select the stencil kernel of qw_step (QW_STENCIL_AUTO restores the default).
 * Errors: QW_EINVAL if the variant does not support this plan's geometry/dtype. */
qw_status qw_plan_set_stencil(qw_plan plan, int variant);

/* The stencil variant qw_step currently uses (never QW_STENCIL_AUTO); -1 for null. */
int qw_plan_get_stencil(qw_plan plan);

/* Debug poison, process-wide: while on != 0, the scratch and partner buffers of
 * plans (qw_step, qw_observables), batches (each launch; a batch's CUDA graph
 * holds the fills if it is captured while this is on) and qw_step_static are
 * filled with NaN before every call that must write them before reading them,
 * so that a read of memory a kernel did not write shows as NaN in the results.
 * Costs one device fill per call; off by default.  Never fails (QW_OK). */
qw_status qw_set_debug_poison(int on);

/* Autotune cache, process-wide: while `path` is set, qw_plan_autotune and
 * qw_batch_autotune first look in that text file for a choice measured on the
 * same GPU model for the same problem (plan: dim, N, dtype; batch: the walks'
 * (dim, N, t) and rounds_cap) and apply it without measuring; otherwise they
 * measure and append a line "<kind> <GPU model> <problem> | <values>".  The last
 * matching line wins; delete the file to re-measure.  NULL or "" turns the
 * cache off (the default).  Never fails (QW_OK). */
qw_status qw_set_autotune_cache(const char* path);

/* Temporal fusion of the FUSED variant: `depth` (2..4) steps per launch on tiles
 * of box[0..dim) cells (x, y, z; on the BCC lattice both cosets of the cells),
 * read with a halo of depth cells per side (depth/2 rounded up on the BCC
 * lattice).  Defaults: depth 4 with 2048 cells (chain) or 64x16 (square
 * lattice), depth 2 with 8x8x6 (BCC).
 * Errors: QW_EINVAL (null argument, complex128 plan, depth outside 2..4, or a
 * tile that with its halo needs more than 227 KB of shared memory). */
qw_status qw_plan_set_fusion(qw_plan plan, int depth, const int* box);
/* The FUSED variant's depth and box (either pointer may be NULL; box: 3 ints). */
qw_status qw_plan_get_fusion(qw_plan plan, int* depth, int* box);

/* Autotuner of the stencil: times every variant that supports the plan (data
 * movement PLAIN / VEC / TMA, fusion depth 2 with TMA2, and FUSED with depth 2,
 * 3, 4 on three tile boxes per lattice) for 8 steps on a temporary
 * field (allocated and freed here; the caller's fields are not touched) and keeps
 * the fastest; *best_rate (optional) receives its site-steps/s.  Synchronous.
 * Errors: QW_EINVAL, QW_ENOMEM, QW_ECUDA, QW_ETIMEOUT. */
qw_status qw_plan_autotune(qw_plan plan, void* stream, double* best_rate);

/* Advance psi_dev in place by `nsteps` >= 0 applications of the update rule
 * (Eq. upd-rule; the plain position-space form of Sec. 4) with the plan's
 * stencil variant.  Ping-pongs through the plan's scratch field (an odd step
 * count ends with one device copy).  Asynchronous on `stream`; a bounded
 * device-side wait that gave up is reported by the next qw_sync/qw_observables.
 * Errors: QW_EINVAL (null plan/pointer, nsteps < 0), QW_ECUDA. */
qw_status qw_step(qw_plan plan, void* psi_dev, int64_t nsteps, void* stream);

/* Build the spectral-path state of the plan: FFT pass plans and twiddle
 * tables, and the table of omega_k = atan2(sin omega_k, n u_k) (Sec. 3.2,
 * cos omega_k = n u_k) for every stored wave vector (one per site in 1D/2D; on
 * the BCC lattice one per cell, the wave vector q0 of its pair, since
 * omega_q1 = pi - omega_q0): complex128 plans hold omega_k as a double-double
 * (16 bytes per entry, ~1e-31 accurate, so that the phase omega_k t keeps ~1e-16
 * at any t), complex64 plans omega_k / 2 pi as a pair of FP32 numbers (8 bytes
 * per entry).  Synchronous; done
 * implicitly by the first qw_evolve_spectral / qw_observables call.
 * Needs every axis length (N, or N/2 for dim 3) of the form 2^a 3^b.
 * Errors: QW_EINVAL (axis length not 2^a 3^b), QW_ENOMEM, QW_ECUDA. */
qw_status qw_plan_prepare_spectral(qw_plan plan);

/* Evolve psi_dev in place to time t >= 0 in the Fourier form of Sec. 4:
 * forward DFT of every component plane (hand-written batched FFT), the
 * per-wave-vector product with D_k^t = cos(omega_k t) I - i sin(omega_k t) G_k/sin(omega_k)
 * (D_k = cos(omega_k) I - i G_k, Sec. 3.2), with the BCC two-coset reduction of
 * Eqs. bcc-dft / bcc-idft, and the inverse DFT.  omega_k t is reduced modulo
 * 2 pi (complex128: from the double-double omega_k, so the phase keeps
 * ~1e-16 at any t); the cost does not depend on t.  Asynchronous on `stream`
 * (after the first call's synchronous preparation).  Same result as t calls
 * of the update rule, up to rounding.
 * Errors: QW_EINVAL (null plan/pointer, t < 0, axis length not 2^a 3^b),
 * QW_ENOMEM, QW_ECUDA. */
qw_status qw_evolve_spectral(qw_plan plan, void* psi_dev, int64_t t, void* stream);

/* Wait for the plan's work on `stream`, then check its device error word.
 * Errors: QW_ETIMEOUT (a kernel's bounded wait gave up; the word is cleared),
 * QW_ECUDA. */
qw_status qw_sync(qw_plan plan, void* stream);

/* Compute the observables of psi_dev (see qw_obs).  Blocks the host until the
 * reductions on `stream` are done, then fills *out.  The particle weights come
 * from a forward DFT of a copy in the plan's scratch field; for boxes whose
 * axis lengths are not 2^a 3^b they are NaN.
 * Errors: QW_EINVAL, QW_ECUDA, QW_ETIMEOUT (as qw_sync). */
qw_status qw_observables(qw_plan plan, const void* psi_dev, qw_obs* out, void* stream);

/* Foldy-Wouthuysen field (the Remark on the Newton-Wigner position, Eqs. fw, NW):
 * the coefficients phi_r(k) = u_r(k)^dag psi^(k) of psi_dev on the paper's
 * eigenvectors of D_k (Eq. evecs-D; 1D: u_+ = (cos th/2, -sin th/2),
 * u_- = (sin th/2, cos th/2), th = atan2(m, n sin k)), taken back to position
 * space, written to out_dev (DEVICE, caller-owned, the field's size and layout,
 * component r in place of spinor component s, r = (s, p) in the order (+,+),
 * (+,-), (-,+), (-,-); 1D: +, -).  Its mean position (qw_position_moments or
 * qw_observables on out_dev) is the Newton-Wigner position, which moves by
 * t <grad omega> on the positive and -t <grad omega> on the negative part and
 * does not jitter.  out_dev may equal psi_dev (in place).  Needs the spectral
 * sizes of qw_plan_prepare_spectral.  Asynchronous on `stream`.
 * Errors: QW_EINVAL (null argument, axis length not 2^a 3^b), QW_ENOMEM, QW_ECUDA. */
qw_status qw_fw_transform(qw_plan plan, const void* psi_dev, void* out_dev, void* stream);

/* Position moments up to second order (the mean and covariance that the drift
 * v = grad omega and diffusion D = grad grad omega of Sec. 5.1's particle states
 * move and spread).  out (HOST, 10 doubles, caller-owned): norm, the mean
 * position (x, y, z) and the central second moments (xx, yy, zz, xy, xz, yz)
 * of the normalised density, on the window and coordinates of qw_observables'
 * mean position; entries of axes at or above dim are 0.  Sums in FP64 (site
 * densities in the field's precision).  Blocks the host until `stream` is done.
 * Errors: QW_EINVAL (null argument), QW_ECUDA, QW_ETIMEOUT (as qw_sync). */
qw_status qw_position_moments(qw_plan plan, const void* psi_dev, double* out, void* stream);

/* Probability projections (Sec. 5.2: the distribution of a localised state
 * projected onto axes and planes).  The density rho(x) = sum_s |psi_s(x)|^2 of
 * psi_dev, summed over the axes NOT named in `keep` (bit 0 = x, bit 1 = y,
 * bit 2 = z; only axes below dim; at least one), on the physical grid of the
 * box with the coordinates of qw_observables' mean position: lattice
 * coordinates (a, b) in 2D, physical BCC coordinates 2 (x, y, z) + c (1, 1, 1)
 * in 3D, each in [0, N).
 * out_dev: caller-owned DEVICE array of qw_projection_elems(plan, keep) =
 * N^(number of kept axes) doubles, indexed with x fastest, then y, then z among
 * the kept axes.  On the BCC lattice, kept-coordinate tuples that are not sites
 * (mixed parity, two or more kept axes) hold 0.  keep = all axes gives the
 * density itself.  Sums are FP64 in a fixed order (site densities in the
 * field's precision): the result is deterministic.  Asynchronous on `stream`;
 * the first call needing chunk partials allocates them in the plan (a few MB).
 * Errors: QW_EINVAL (null argument, bad keep), QW_ENOMEM, QW_ECUDA. */
qw_status qw_projection(qw_plan plan, const void* psi_dev, int keep, double* out_dev, void* stream);

/* Number of doubles qw_projection writes for `keep`, or -1 for a bad plan/mask. */
int64_t qw_projection_elems(qw_plan plan, int keep);

/* End-to-end runs on HOST fields.  For j = 0 .. count-1: copy the field
 * psi_host[j] (host memory, device layout, qw_plan_field_elems elements;
 * page-locked memory copies fastest and overlaps) to the device, advance it by
 * nsteps applications of the update rule (as qw_step) and compute its
 * observables into out[j] (as qw_observables).  If psi_out_host is not NULL,
 * psi_out_host[j] (host memory, same size; may equal psi_host[j]) receives the
 * evolved field.  The fields pass through three device buffers owned by the
 * plan (allocated by the first call, freed with the plan): the copy of field
 * j + 2 starts on the plan's copy stream once field j - 1's observables are done
 * and runs while field j is advanced on `stream`, so a transfer has two steps to
 * land; the read-back of field j on the copy stream overlaps field j + 1.  Synchronous:
 * returns when every result is on the host.  count = 0 does nothing.
 * Errors: QW_EINVAL (null plan, count < 0, nsteps < 0, null psi_host / out or a
 * null entry), QW_ENOMEM (device buffers), QW_ECUDA, QW_ETIMEOUT (as qw_sync). */
qw_status qw_run_host(qw_plan plan, const void* const* psi_host, void* const* psi_out_host, int count,
                      int64_t nsteps, qw_obs* out, void* stream);

/* Per-field timing of qw_run_host, to measure how well the host-to-device copies
 * overlap the computation.  on != 0: later qw_run_host calls record CUDA events
 * (timing enabled) at the start and end of each field's copy in (copy stream),
 * the start and end of its steps and the end of its observables (compute
 * stream); on = 0 stops recording.  Errors: QW_EINVAL (null plan). */
qw_status qw_plan_set_host_timing(qw_plan plan, int on);

/* For the first `count` fields of the last timed qw_run_host call, writes 5
 * doubles per field (HOST array of 5 * count): copy start, copy end, step start,
 * step end, observables end, in ms from the first field's copy start.
 * Synchronises with those events.  Errors: QW_EINVAL (null argument, or count
 * not in 1 .. the fields of the last timed run), QW_ECUDA. */
qw_status qw_plan_host_timing(qw_plan plan, double* out, int count);

/* ---------------------------------------------------------------- batches
 * Many independent walks of uneven size advanced together by one persistent
 * kernel launch, replayed from a CUDA graph (complex64 only).  Each walk is the
 * update rule (Eq. upd-rule) applied t times to its own field, with the same
 * per-site arithmetic as qw_step's PLAIN kernel (bit-identical results, fused
 * or not). */
typedef struct {
  int dim;          /* 1, 2 or 3 */
  int64_t N;        /* box side (even for dim 3) */
  double mass;      /* m in [0, 1] */
  int64_t t;        /* steps per qw_batch_run, 0 <= t < 2^30 */
  void* psi_dev;    /* the walk's complex64 field (device layout), caller-owned */
} qw_walk;

typedef struct qw_batch_s* qw_batch;

/* Create a batch over n walks (descriptors copied).  Allocates a partner
 * field per walk, the schedule tables and counters on the current device.
 * Default tiling: depth 1 on every lattice with 2048-site tiles, one group
 * (16 GiB), the autotuner's choice for a mix of 256 square-lattice and BCC walks
 * on GB300; boxes for fused rounds 1024, 32x16 and 8x8x4 cells.  qw_batch_autotune
 * measures the mix at hand.
 * Errors: QW_EINVAL (bad descriptor, a walk of 2^31 complex values or more),
 * QW_ENOMEM, QW_ECUDA. */
qw_status qw_batch_create(const qw_walk* walks, int n, qw_batch* out);
qw_status qw_batch_destroy(qw_batch batch);

/* How a batch cuts its walks into work items.  A round advances one tile of a walk
 * by `depth` steps (its fusion depth, per lattice dimension):
 *   depth 1: every site updated from global memory; tiles are whole x rows (x
 *            segments on the chain) of about tile_sites sites;
 *   depth 2..4: temporal fusion; the tile is a box of box[dim-1] = (x, y, z)
 *            cells (both cosets on the BCC lattice; unused axes ignored), which
 *            is read with a halo of `depth` cells per side (depth/2 rounded up on
 *            the BCC lattice) into shared memory, advanced there by `depth`
 *            steps and written once: one read and one write of the field per
 *            `depth` steps instead of per step.
 * Walks whose two buffers fit l2_budget_bytes together form a group; groups
 * run one after the other (small budgets keep a group's walks in L2). */
typedef struct {
  int64_t tile_sites;       /* depth-1 walks: sites per tile, 32 .. 4M */
  int64_t l2_budget_bytes;  /* footprint of one group of walks, >= 1 MiB */
  int depth[3];             /* fusion depth of 1D, 2D and BCC walks: 1 .. 4 */
  int box[3][3];            /* fused tiles of 1D, 2D and BCC walks: (x, y, z) extents in cells */
} qw_batch_tiling;

/* Set the tiling (rebuilds the schedule and drops the captured graph).
 * Errors: QW_EINVAL (value out of range, or a walk whose fused tile, the box
 * clipped to the walk plus its halo, needs more than 227 KB of shared memory for
 * its two buffers), QW_ENOMEM, QW_ECUDA. */
qw_status qw_batch_set_tiling(qw_batch batch, const qw_batch_tiling* tiling);

/* The current tiling and the number of work items of one run (either may be NULL). */
qw_status qw_batch_get_tiling(qw_batch batch, qw_batch_tiling* tiling, int64_t* items);

/* Autotuner of the batched kernel: times one launch of the batch per candidate
 * tiling on stand-in fields of the same sizes (zero-filled scratch, allocated and
 * freed here; the walks' fields are not touched), with the step counts scaled so
 * that the longest walk runs rounds_cap steps (the mix keeps its shape), and keeps
 * the fastest.  Candidates: depth 1 with tile_sites in {1K, 2K, 4K, 8K}; fusion
 * depth {2, 4} for 1D/2D walks with 2D boxes {32x16, 64x8, 32x32, 64x16} and depth
 * {1, 2} for BCC walks with boxes {8x8x4, 8x8x6, 16x8x4, 8x8x8}; then the group
 * budget in {48, 96, 192 MiB, 1 GiB} against one group (16 GiB).  Optional
 * outputs: the chosen tiling and its measured site-steps/s.  Synchronous.
 * Errors: QW_EINVAL, QW_ENOMEM, QW_ECUDA. */
qw_status qw_batch_autotune(qw_batch batch, int64_t rounds_cap, void* stream, qw_batch_tiling* best,
                            double* best_rate);

/* Fault injection for tests of the bounded dependency waits.  walk >= 0: the
 * first tile of that walk (caller's order) never publishes the rounds it
 * completes, so the rounds that depend on it wait, give up after spin_limit
 * polls (about 100 ns each), and qw_batch_sync returns QW_ETIMEOUT; the launch
 * ends early and the walks' fields hold partial results.  walk < 0 restores
 * normal operation (spin_limit ignored).  Drops the captured graph.
 * Errors: QW_EINVAL (walk >= n, or spin_limit < 1 with walk >= 0). */
qw_status qw_batch_debug_stall(qw_batch batch, int walk, int64_t spin_limit);

/* Advance every walk by its t steps, in place, in one persistent launch
 * (captured into a CUDA graph on the first call, replayed afterwards).
 * Asynchronous on `stream`.  Dependency waits inside the kernel are bounded;
 * a wait that gives up is reported by qw_batch_sync.  Errors: QW_EINVAL, QW_ECUDA. */
qw_status qw_batch_run(qw_batch batch, void* stream);

/* Wait for the batch's work on `stream`; QW_ETIMEOUT if a dependency wait gave up. */
qw_status qw_batch_sync(qw_batch batch, void* stream);

/* Norm and <x> of every walk (out[i] for walk i, original order); particle
 * weights are NaN here (use a plan's qw_observables).  Synchronous. */
qw_status qw_batch_observables(qw_batch batch, qw_obs* out, void* stream);

/* Fill psi_dev with the Gaussian packet
 *     psi(x) = exp(-|d|^2 / (4 sigma^2)) exp(i k0.d) chi,   d = minimum-image (x - x0),
 * on the plan's box (physical coordinates on the BCC lattice, lattice
 * coordinates (a, b) in 2D): the position-space shape of the particle states of
 * Sec. 5 (Definition 1).  chi: s complex values as (re, im) pairs (s = 2 in 1D,
 * 4 otherwise; 8 doubles are read).  Not normalised.  Asynchronous.
 * Errors: QW_EINVAL (null pointer, sigma <= 0), QW_ECUDA. */
qw_status qw_prepare_packet(qw_plan plan, void* psi_dev, const double* x0, double sigma, const double* k0,
                            const double* chi, void* stream);

/* ---------------------------------------------------------------- serving
 * Walk requests evolved in the Fourier form (Sec. 4, complex64 fields, FP64
 * phase and reductions) by one scheduler thread with continuous batching:
 * requests wait in a FIFO, the head is admitted when one of `slots` CUDA
 * streams is free and its field (8 B per complex value) fits in the device pool
 * of `hbm_budget_bytes` (allocated once at creation); finished requests return their slot and memory, so requests that
 * arrived meanwhile start while others are still running, and requests in
 * different slots overlap on the device.  The initial state is normalised. */
typedef struct {
  int dim;                 /* 1, 2 or 3 */
  int64_t N;               /* box side; every axis length (N, or N/2 in 3D) 2^a 3^b */
  double mass;             /* m in [0, 1] */
  int64_t t;               /* time, >= 0 */
  const void* psi0_host;   /* complex64 initial field (device layout), copied at submit; or NULL ... */
  double x0[3];            /* ... for the packet of qw_prepare_packet with these parameters */
  double sigma;
  double k0[3];
  double chi[8];
} qw_request;

typedef struct qw_server_s* qw_server;

typedef struct {
  int64_t pending, running, admitted, completed;
  int64_t bytes_in_use, peak_bytes, budget_bytes;
} qw_server_stats_t;

/* Start a server on the current device with a device pool of hbm_budget_bytes,
 * `slots` concurrent streams (1..64) and at most max_pending queued requests.
 * Errors: QW_EINVAL, QW_ENOMEM, QW_ECUDA. */
qw_status qw_server_create(size_t hbm_budget_bytes, int slots, int max_pending, qw_server* out);

/* Queue a request; *ticket identifies it.  Does not block on the GPU.
 * Errors: QW_EINVAL (bad request, axis not 2^a 3^b, larger than the whole
 * budget), QW_EAGAIN (pending queue full: retry later). */
qw_status qw_submit(qw_server server, const qw_request* req, uint64_t* ticket);

/* Non-blocking: *done = 0 while the request waits or runs; once done, *done = 1,
 * *out holds its norm, <x> and particle weights, *latency_s the time from
 * qw_submit to completion, and the ticket is retired.
 * Errors: QW_ENOTFOUND (unknown or retired ticket), QW_ECUDA (the request failed). */
qw_status qw_poll(qw_server server, uint64_t ticket, qw_obs* out, int* done, double* latency_s);

/* Queue and pool occupancy counters. */
qw_status qw_server_stats(qw_server server, qw_server_stats_t* out);

/* Stop the scheduler (queued requests are dropped, running ones finish) and free everything. */
qw_status qw_server_destroy(qw_server server);

/* qw_step without any device allocation, for callers that cannot call
 * cudaMalloc where they step a walk: code whose device memory is owned and
 * budgeted by another allocator (for example a framework's caching pool that
 * already holds the GPU), or a latency-critical loop that must not pay for
 * cudaMalloc's implicit device synchronisation.  The paper has no counterpart;
 * this is a library-interface variant of qw_step.
 * Same update and arguments as qw_plan_create + qw_step (dim, N, mass, dtype,
 * psi_dev of qw_plan_field_elems elements, nsteps >= 0, stream), but the
 * ping-pong partner field is a file-scope static device array of 64 MiB that
 * every GPU loading libqw.so holds until the process exits; the kernel is the
 * VEC variant where it applies, else PLAIN (never the TMA variant).
 * The first call on a device looks up that array's device address (with the
 * device current) and caches it for the process; make that first call before
 * any stream capture.  The cached address does not survive cudaDeviceReset:
 * after a reset of a device, do not call qw_step_static on it again in the
 * same process.  The device that is current, the stream's device and the
 * field's device must be the same one (a stream of another device: QW_EINVAL).
 * All calls on a device share the one array, and it keeps the last call's
 * contents: calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller.
 * Errors: QW_EINVAL (bad arguments, a stream of another device, or a field
 * larger than 64 MiB -- use a plan for those), QW_ECUDA. */
qw_status qw_step_static(int dim, int64_t N, double mass, qw_dtype dtype, void* psi_dev, int64_t nsteps,
                         void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QW_H */
