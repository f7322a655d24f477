/*
 * soc.h -- C-ABI of libsoc, a GB300 (sm_103a) implementation of the Monte Carlo
 * photon-package transport and equilibrium dust-temperature update of SOC
 * (M. Juvela, "SOC program for dust continuum radiative transfer",
 * A&A 2019, arXiv:1812.06632).
 *
 * Conventions
 *  - Every function returns soc_status (SOC_OK == 0, errors < 0) and never
 *    throws.  soc_last_error() gives a message for the last failing call on
 *    a context.
 *  - "host" pointers are read during the call only; the caller keeps
 *    ownership.  "device" pointers are caller-owned device memory on the
 *    context's device (e.g. torch tensors); the library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls taking a stream are asynchronous on it unless stated.
 *  - Fixed point: one photon package starts with SOC_W_UNIT = 2^31 weight
 *    units; absorption counters ("tallies") are int64 sums of weight units.
 *  - Lengths: the kernels work in root-cell units; physical sizes (cm)
 *    enter only through the root-cell side of each grid.
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef SOC_H
#define SOC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int soc_status;
#define SOC_OK              0
#define SOC_ERR_ARG        -1   /* bad argument (null pointer, size, index)          */
#define SOC_ERR_GRID       -2   /* malformed grid (link out of range, NaN, rho < 0)  */
#define SOC_ERR_CUDA       -3   /* a CUDA runtime call failed                        */
#define SOC_ERR_STEP_LIMIT -4   /* packages were ended by the step cap               */
#define SOC_ERR_STATE      -5   /* call order: e.g. simulation before soc_dust_upload */
#define SOC_ERR_NOMEM      -6   /* device or host allocation failed                  */
#define SOC_ERR_TIMEOUT    -7   /* the abort flag was set (soc_abort, or the watchdog
                                   of soc_set_timeout): the call stopped early       */

#define SOC_SRC_BACKGROUND 0
#define SOC_SRC_POINT      1
#define SOC_SRC_DUST       2

#define SOC_W_UNIT   2147483648ull      /* 2^31 */
#define SOC_MAX_LEVELS 16

typedef struct soc_ctx soc_ctx;

/* Create a context on CUDA device `device` with the Monte Carlo seed `seed`
 * (the Philox key of every package stream).  *out receives the context. */
soc_status soc_create(soc_ctx **out, int device, uint64_t seed);
/* Free every device buffer the context owns.  NULL is accepted. */
void soc_destroy(soc_ctx *ctx);
/* Message of the last failing call on ctx (never NULL). */
const char *soc_last_error(const soc_ctx *ctx);

/* ------------------------------------------------------------------------
 * soc_grid_upload -- hierarchical density grid (paper Sect. 2.1.1).
 * The root grid is nx*ny*nz cubic cells (x fastest: c = i + nx*(j + ny*k)).
 * Octree refinement splits a cell into an octet of 8 equal cells.  The cell
 * vector is level ordered: root cells, then every cell of level 2, then of
 * level 3, ...; each octet is contiguous, its cells ordered by octant
 * ox + 2*oy + 4*oz, so cell c >= n_root belongs to octet (c - n_root)/8.
 *   rho[n_cells]      host, FP32: density of every leaf (>= 0, finite).  With
 *                     first_child == NULL, refined cells carry the paper's
 *                     encoding: minus the index of their first child (exact
 *                     only below 2^24 cells).
 *   first_child       host [n_cells] int32 or NULL: first child index of a
 *                     refined cell, -1 for a leaf (overrides rho's encoding).
 *   parent            host [(n_cells - n_root)/8] int32 or NULL: parent cell of
 *                     each octet (reverse links); derived when NULL, checked
 *                     when given.
 *   cells_per_level   host [n_levels].
 *   root_cell_size    root-cell side in cm (> 0).
 * The grid is validated on the host (SOC_ERR_GRID on any inconsistency),
 * converted to tagged 32-bit cell words (bit 31 set: first-child index in
 * bits 0..30; else the FP32 density) and copied to the device.  Returns the
 * new cloud id in *cloud_id (0, 1, 2, ... in call order).  Synchronous.
 * ------------------------------------------------------------------------ */
typedef struct soc_grid_desc {
    int32_t nx, ny, nz;
    int32_t n_levels;
    const int64_t *cells_per_level;
    const float *rho;
    const int32_t *first_child;
    const int32_t *parent;
    double root_cell_size;
} soc_grid_desc;

soc_status soc_grid_upload(soc_ctx *ctx, const soc_grid_desc *desc, int *cloud_id);

/* Release the device memory of an uploaded grid (and of its sources and
 * iteration buffers).  The id is not reused; later calls naming it fail with
 * SOC_ERR_ARG.  Synchronous: waits for the device to finish using it. */
soc_status soc_grid_free(soc_ctx *ctx, int cloud_id);

/* Host-only check of a grid description with the rules of soc_grid_upload
 * (needs no device and no context).  SOC_OK or SOC_ERR_ARG / SOC_ERR_GRID;
 * msg (host, msg_len bytes, may be NULL) receives the reason. */
soc_status soc_grid_validate(const soc_grid_desc *desc, char *msg, int msg_len);

/* ------------------------------------------------------------------------
 * soc_dust_upload -- dust properties on the fixed frequency grid (paper
 * Sect. 2.1.1: cross sections for absorption and scattering and the
 * scattering function against frequency; Sect. 2.2: fixed frequency grid).
 *   nu[n_freq]        host, Hz, strictly increasing.
 *   kabs, ksca        host [n_freq]: cross sections per density unit (cm^2):
 *                     rho*kappa is an inverse length in 1/cm.
 *   g                 host [n_freq]: Henyey-Greenstein asymmetry, |g| < 1.
 * Also builds the FP64 emission table E(T) = 4 pi sum_nu w_nu kabs B_nu(T)
 * on 4096 log-spaced T in [2.7, 3000] K (w_nu = trapezoid weights).  Must be
 * called once, before any simulation.  Synchronous.
 * ------------------------------------------------------------------------ */
soc_status soc_dust_upload(soc_ctx *ctx, int n_freq, const double *nu, const double *kabs,
                           const double *ksca, const double *g);

/* ------------------------------------------------------------------------
 * soc_sources_upload -- radiation sources of one cloud (paper Sect. 2.2:
 * isotropic external background and blackbody point sources).
 *   bg_I_nu           host [n_freq] or NULL: background intensity
 *                     (erg/s/cm^2/Hz/sr) outside the box.
 *   n_ps              number of point sources (0 allowed).
 *   ps_pos            host [3*n_ps]: positions in root-cell units, strictly
 *                     inside the root grid.
 *   ps_L_nu           host [n_ps*n_freq] (source-major): luminosity erg/s/Hz.
 * A point-source package picks its source with probability proportional to
 * L_nu, so all packages of a frequency carry the same energy.  Synchronous.
 * ------------------------------------------------------------------------ */
soc_status soc_sources_upload(soc_ctx *ctx, int cloud_id, const double *bg_I_nu, int n_ps,
                              const double *ps_pos, const double *ps_L_nu);

/* ------------------------------------------------------------------------
 * soc_simulate_frequency_batch -- trace photon packages (paper Sect. 2.1.1:
 * package creation, cell-to-cell stepping with partial traversal of the
 * hierarchy, absorption counters per cell and frequency).  Every item is one
 * (cloud, frequency, source class) with its own package-id range; all items
 * run in ONE persistent kernel launch.
 *   items[n_items]    host array (copied during the call):
 *     cloud, freq     indices of an uploaded grid and of the frequency grid;
 *     source          SOC_SRC_BACKGROUND / SOC_SRC_POINT / SOC_SRC_DUST;
 *     iteration       RNG stream selector (key word 1 gets iteration << 16);
 *     pid_offset      first package id (packages pid_offset .. +n_packages-1);
 *     n_packages      number of packages (< 2^32 - pid_offset);
 *     w0              initial weight of background / point packages (1..2^31);
 *     tally_offset    element offset in d_tally of this item's cell 0: the
 *                     item adds its deposits to d_tally[tally_offset + cell];
 *     d_dust_w        device [n_leaf] uint64: initial weight of the packages
 *                     of each leaf (leaves in cell order, each <= SOC_W_UNIT;
 *                     larger values are not checked), SOC_SRC_DUST only;
 *     n_per_cell      dust packages per leaf (n_packages = n_leaf*n_per_cell).
 *     reserved        flags: SOC_ITEM_WEIGHTED (dust) = emission-weighted
 *                     sampling: d_dust_w holds [n_leaf] weights followed by
 *                     the [n_leaf + 1] uint64 prefix of packages per leaf
 *                     (as written by soc_dust_weighted); package pid comes
 *                     from the leaf li with prefix[li] <= pid < prefix[li+1];
 *                     n_packages = prefix[n_leaf].
 *   d_tally           device int64, accumulated into (caller zeroes it).
 *   d_stats           device int64 [n_items][4], accumulated into:
 *                     {escaped weight, capped packages, photon-cell steps,
 *                      emitted weight}.  Energy is conserved exactly:
 *                     sum(tally of the item) + escaped == emitted.
 *   d_pkg_steps       device uint32 [sum of n_packages] or NULL: steps of each
 *                     package, in item order then package order.
 * Deterministic: results depend only on inputs and the seed, not on launch
 * shape.  Asynchronous on `stream`.  The item table is copied from host
 * memory, so the call cannot be captured into a CUDA graph: on a capturing
 * stream it returns SOC_ERR_STATE (capture soc_batch_launch instead).
 * ------------------------------------------------------------------------ */
#define SOC_ITEM_WEIGHTED 1u   /* soc_batch_item.reserved flag: weighted dust sampling */

typedef struct soc_batch_item {
    int32_t cloud;
    int32_t freq;
    int32_t source;
    int32_t iteration;
    uint64_t pid_offset;
    uint64_t n_packages;
    uint64_t w0;
    int64_t tally_offset;
    const uint64_t *d_dust_w;
    uint32_t n_per_cell;
    uint32_t reserved;
} soc_batch_item;

soc_status soc_simulate_frequency_batch(soc_ctx *ctx, const soc_batch_item *items, int n_items,
                                        int64_t *d_tally, int64_t *d_stats,
                                        uint32_t *d_pkg_steps, void *stream);

/* The same, with a second counter array d_self (device int64, same layout
 * and offsets as d_tally, accumulated; NULL = none): for dust items it
 * receives the deposits a package makes in its emission cell before it
 * first leaves that cell -- the local re-absorption used by the accelerated
 * (ALI, paper Sect. 2.1.2 / 3.3) temperature update. */
soc_status soc_simulate_frequency_batch_ex(soc_ctx *ctx, const soc_batch_item *items, int n_items,
                                           int64_t *d_tally, int64_t *d_self, int64_t *d_stats,
                                           uint32_t *d_pkg_steps, void *stream);

/* ------------------------------------------------------------------------
 * soc_simulate_frequency_batch_noalloc -- the same call, arguments, results
 * and determinism as soc_simulate_frequency_batch, for callers that must not
 * allocate device memory while they run (code inside a framework's caching
 * allocator or memory budget, real-time loops where cudaMalloc/cudaFree would
 * synchronise the device, embedders that only hand out fixed buffers).  The
 * paper has no counterpart: this is an interface variant, not a step of the
 * method.
 *   Scratch (work counter, item table, prefix sums, grid table) lives in one
 *   fixed device array inside the library, about 74 KB, which every GPU that
 *   loads the library keeps until the process exits.  No cudaMalloc, cudaFree
 *   or allocating library routine is called.
 *   Limits: n_items <= SOC_NOALLOC_MAX_ITEMS and at most
 *   SOC_NOALLOC_MAX_CLOUDS grids uploaded on the context (freed grids still
 *   count); larger requests fail with SOC_ERR_ARG.
 *   The first call on a device looks up the array's device address (set-up
 *   for that device; threads that race on it store the same address).
 *   Like soc_simulate_frequency_batch it copies its tables from host memory,
 *   so it cannot be captured into a CUDA graph: on a capturing stream it
 *   returns SOC_ERR_STATE (graphs use soc_batch_create / soc_batch_launch).
 *   All calls share the one array: calls that overlap on the GPU (other
 *   streams, other contexts on the same device) race and must be ordered by
 *   the caller.
 * ------------------------------------------------------------------------ */
#define SOC_NOALLOC_MAX_ITEMS  1024
#define SOC_NOALLOC_MAX_CLOUDS 64
soc_status soc_simulate_frequency_batch_noalloc(soc_ctx *ctx, const soc_batch_item *items, int n_items,
                                                int64_t *d_tally, int64_t *d_stats,
                                                uint32_t *d_pkg_steps, void *stream);

/* ------------------------------------------------------------------------
 * Prepared batches and CUDA graphs: many frequencies and clouds in one
 * persistent launch, replayed without host work.
 * soc_batch_create checks the items as soc_simulate_frequency_batch does and
 * copies them once into library-owned device memory (synchronous); returns
 * *batch_id.  soc_batch_launch zeroes d_tally[0, tally_len) (tally_len 0:
 * no zeroing) and the batch's d_stats rows, resets the batch's work counter
 * and launches the tracer on `stream`: no host-to-device copy, so it can be
 * captured.  soc_capture_begin / soc_capture_end capture every library call
 * issued on `stream` in between (soc_batch_launch, soc_absorbed_power,
 * soc_update_temperature, soc_dust_emission; NOT soc_simulate_frequency_batch,
 * which copies from host memory) into an executable CUDA graph *graph_id;
 * soc_graph_launch replays it.  `stream` must not be the legacy default
 * stream.  Grids, dust and sources must not be re-uploaded or freed while a
 * batch or graph that uses them is alive.
 * ------------------------------------------------------------------------ */
soc_status soc_batch_create(soc_ctx *ctx, const soc_batch_item *items, int n_items, int *batch_id);
soc_status soc_batch_launch(soc_ctx *ctx, int batch_id, int64_t *d_tally, int64_t tally_len,
                            int64_t *d_stats, uint32_t *d_pkg_steps, void *stream);
soc_status soc_batch_destroy(soc_ctx *ctx, int batch_id);
soc_status soc_capture_begin(soc_ctx *ctx, void *stream);
soc_status soc_capture_end(soc_ctx *ctx, void *stream, int *graph_id);
soc_status soc_graph_launch(soc_ctx *ctx, int graph_id, void *stream);
soc_status soc_graph_destroy(soc_ctx *ctx, int graph_id);

/* Per-package energy of background / point-source packages (paper Sect. 2.2
 * sources): the energy in erg/s/Hz carried by one weight unit when
 * n_packages packages of weight 2^31 are launched at every frequency.
 *   background: pi I_nu S / n_packages / 2^31 (S = box surface, cm^2);
 *   point:      sum_k L_nu,k / n_packages / 2^31.
 * e_unit: host [n_freq].  Synchronous (host only). */
soc_status soc_package_energy(soc_ctx *ctx, int cloud_id, int source, uint64_t n_packages,
                              double *e_unit);

/* ------------------------------------------------------------------------
 * soc_dust_emission -- weights of dust re-emission packages (paper Sect. 3.2:
 * the same number of packages from every cell, random position and direction
 * inside the cell).  For every leaf c and frequency index f in
 * [freq_lo, freq_lo + n_freq):
 *   L_c = 4 pi rho_c V_c kabs(nu) B_nu(T_c)   (FP64),
 *   d_w[(f - freq_lo)*n_leaf + leaf(c)] = rint(2^31 L_c / max_c L_c),
 *   d_e_unit[f - freq_lo] = max_c L_c / n_per_cell / 2^31.
 *   d_T               device float [n_cells] (leaf temperatures; parents ignored).
 *   d_w               device uint64 [n_freq][n_leaf].
 *   d_e_unit          device double [n_freq].
 * Asynchronous on `stream`.
 * ------------------------------------------------------------------------ */
soc_status soc_dust_emission(soc_ctx *ctx, int cloud_id, const float *d_T, int freq_lo, int n_freq,
                             uint32_t n_per_cell, uint64_t *d_w, double *d_e_unit, void *stream);

/* ------------------------------------------------------------------------
 * soc_dust_weighted -- emission-weighted dust sampling (paper Sect. 3.2:
 * packages per cell in proportion to the cell's luminosity, with a cap on
 * any single cell).  From the uniform weights u = rint(2^31 L / max L) of
 * soc_dust_emission (n_per_cell = 1) and its d_e_unit, per frequency:
 *   S = sum u;  n_c = u_c ? min(cap, ceil(N u_c / S)) : 0;
 *   E_ref = max(S / N, 2^31 / cap);  W_c = rint((u_c / n_c) / E_ref 2^31);
 *   e_unit = e_unit_uniform E_ref / 2^31  (energy of one weight unit).
 *   d_u               device uint64 [n_freq][n_leaf].
 *   d_out             device uint64 [n_freq][2 n_leaf + 1]: W then the
 *                     exclusive prefix of n (last entry = packages to trace).
 *   d_e_unit          device double [n_freq].
 * Integer sums and a fixed operation order: deterministic.  Asynchronous.
 * ------------------------------------------------------------------------ */
soc_status soc_dust_weighted(soc_ctx *ctx, int cloud_id, const uint64_t *d_u, const double *d_e_unit_uniform,
                             int n_freq, uint64_t n_total, uint32_t cap, uint64_t *d_out, double *d_e_unit,
                             void *stream);

/* ------------------------------------------------------------------------
 * soc_dust_reweight -- new weights for an existing allocation (the prefix
 * half of d_inout, as written by soc_dust_weighted, is read and kept), from
 * new uniform weights u of soc_dust_emission (n_per_cell = 1):
 *   n_c = prefix[c+1] - prefix[c];  E_ref = max over n_c > 0 of u_c / n_c;
 *   W_c = n_c ? rint((u_c / n_c) / E_ref 2^31) : 0;
 *   e_unit = e_unit_uniform E_ref / 2^31.
 * Keeping the counts keeps every package's id -> cell map between dust
 * iterations, so frozen random numbers (paper Sect. 3.2) give the same paths
 * and the iteration converges like the uniform one.
 *   d_u               device uint64 [n_freq][n_leaf].
 *   d_inout           device uint64 [n_freq][2 n_leaf + 1]: W overwritten,
 *                     prefix read.
 *   d_e_unit          device double [n_freq], written.
 * Deterministic.  Asynchronous on `stream`.
 * ------------------------------------------------------------------------ */
soc_status soc_dust_reweight(soc_ctx *ctx, int cloud_id, const uint64_t *d_u, const double *d_e_unit_uniform,
                             int n_freq, uint64_t *d_inout, double *d_e_unit, void *stream);

/* ------------------------------------------------------------------------
 * Reference-field building blocks (paper Sect. 2.1.2: a simulation estimates
 * only a correction to the mean radiation field of the earlier iterations,
 * storing the absorption of that reference field; Sects. 3.4, 3.6 and 4.1:
 * package counts growing over the iterations, earlier iterations weighted
 * less).  Arrays over (frequency, leaf) are frequency-major [n_freq][n_leaf],
 * leaves in the order of the cloud's leaf list.  All asynchronous on
 * `stream`; SOC_ERR_ARG for null pointers or n_freq < 1.
 *
 * soc_dust_luminosity: d_L (device double) = 4 pi rho V kabs B_nu(T) of every
 *   leaf at frequencies freq_lo .. freq_lo + n_freq - 1 (erg/s/Hz).
 *
 * soc_reference_delta: per frequency, d = L - L_ref, m = max |d|,
 *   d_u (device uint64) = rint(|d| / m 2^31), d_neg (device uint8) = d < 0,
 *   d_e_unit_uniform (device double [n_freq]) = m / 2^31 (energy of one
 *   unit of u with one package per cell: the input of soc_dust_weighted),
 *   and L_ref (device double, in/out) += w d.
 *
 * soc_dust_split: splits allocations [n_freq][2 n_leaf + 1] (W then prefix,
 *   from soc_dust_weighted) by d_neg: d_alloc keeps the weights of leaves
 *   with d >= 0 (others 0), d_alloc_neg gets those of leaves with d < 0 and
 *   a copy of the prefix; d_e_unit_neg = -d_e_unit, so that
 *   soc_absorbed_power with it subtracts the falling cells' part.
 *
 * soc_reference_update: over the cloud's n_cells, d_A_ref (in/out) +=
 *   w (d_A_d - d_A_ref); d_A_out (may be NULL) = d_A_const + X with
 *   X = the updated d_A_ref if out_mean, else d_A_d (d_A_const may be NULL:
 *   then X).
 * ------------------------------------------------------------------------ */
soc_status soc_dust_luminosity(soc_ctx *ctx, int cloud_id, const float *d_T, int freq_lo, int n_freq, double *d_L,
                               void *stream);
soc_status soc_reference_delta(soc_ctx *ctx, int cloud_id, int n_freq, const double *d_L, double *d_L_ref,
                               double w, uint64_t *d_u, uint8_t *d_neg, double *d_e_unit_uniform, void *stream);
soc_status soc_dust_split(soc_ctx *ctx, int cloud_id, int n_freq, const uint8_t *d_neg, uint64_t *d_alloc,
                          uint64_t *d_alloc_neg, const double *d_e_unit, double *d_e_unit_neg, void *stream);
soc_status soc_reference_update(soc_ctx *ctx, int cloud_id, double *d_A_ref, const double *d_A_d, double w,
                                const double *d_A_const, double *d_A_out, int out_mean, void *stream);

/* ------------------------------------------------------------------------
 * soc_absorbed_power -- frequency integral of the absorption counters (paper
 * Sect. 2.1.1: for equilibrium dust the integral of absorbed energy over
 * frequency is gathered on the device):
 *   d_A_out[c] = d_A_in[c] + sum_f w_f e_unit_f d_tally[f*tally_stride + c] / (rho_c V_c)
 * for every leaf with rho > 0 (others: d_A_in[c], or 0), in FP64, summed in
 * frequency order.  w_f = trapezoid weights of the uploaded frequency grid.
 *   d_tally           device int64 [n_freq][tally_stride] (cell 0 at offset 0).
 *   d_e_unit          device double [n_freq].
 *   d_A_in            device double [n_cells] or NULL; may equal d_A_out.
 *   d_A_out           device double [n_cells].
 * Asynchronous on `stream`.
 * ------------------------------------------------------------------------ */
soc_status soc_absorbed_power(soc_ctx *ctx, int cloud_id, const int64_t *d_tally, int64_t tally_stride,
                              const double *d_e_unit, const double *d_A_in, double *d_A_out,
                              void *stream);

/* ------------------------------------------------------------------------
 * soc_update_temperature -- equilibrium dust temperature (paper Sect. 2.1.1:
 * a separate kernel solves the temperatures from the absorbed energy).  For
 * every leaf: T solves 4 pi sum_nu w_nu kabs B_nu(T) = A by FP64 table
 * inversion: ln A is bracketed in ln E(T_k) (4096 log-spaced T_k) and ln T
 * interpolated linearly (error < 2e-7 relative on a 64-point grid).
 * A >= E(3000 K) gives 3000 K.
 * The temperature update of an iteration is two calls: soc_absorbed_power
 * (once per counter array, accumulating into A) and this one.  They stand in
 * for one call taking the constant-source and the dust counters together, so
 * that counters of different energy units (background, point-source and dust
 * packages) are combined into A without a second copy of either.
 *   d_A               device double [n_cells].
 *   d_T               device float [n_cells], in/out: holds T_prev on entry.
 *   d_max_dT          device double [1] or NULL: receives max |T - T_prev|
 *                     over leaves (overwritten, not accumulated).
 * Asynchronous on `stream`.
 * ------------------------------------------------------------------------ */
soc_status soc_update_temperature(soc_ctx *ctx, int cloud_id, const double *d_A, float *d_T,
                                  double *d_max_dT, void *stream);

/* Accelerated lambda iteration with the diagonal operator (paper Sect. 2.1.2:
 * ALI solves explicitly for the photons absorbed within the emitting cell;
 * Sect. 3.3 tests it): with A_self the absorbed power per unit rho V that a
 * leaf re-absorbed from its own emission in this iteration (from the d_self
 * counters of soc_simulate_frequency_batch_ex through soc_absorbed_power),
 * beta = A_self / E(T_prev) (clamped to [0, 0.99], E from the table) and T
 * solves E(T) (1 - beta) = A - A_self.  Same arguments otherwise as
 * soc_update_temperature.  Asynchronous on `stream`. */
soc_status soc_update_temperature_ali(soc_ctx *ctx, int cloud_id, const double *d_A, const double *d_A_self,
                                      float *d_T, double *d_max_dT, void *stream);

/* ------------------------------------------------------------------------
 * soc_map -- surface-brightness map (paper Sect. 2.1.1: after the
 * temperatures are solved, a mapping kernel makes maps for chosen
 * frequencies and directions).  Rays travel along `dir` (the observer looks
 * back along it); the map plane has axes e1 = up x dir and e2 = dir x e1
 * (normalised); pixel (px, py) is centred at
 *   center + ((px + 0.5) - npx/2) pix_size e1 + ((py + 0.5) - npy/2) pix_size e2
 * (root-cell units).  Along each leaf segment of extinction optical depth
 * dtau (kext = kabs + ksca of frequency `freq`) the intensity gains
 * (kabs/kext) B_nu(T) (1 - e^-dtau) e^-tau_front; I_bg (erg/s/cm^2/Hz/sr)
 * enters from behind attenuated by the total optical depth.
 *   d_T     device float [n_cells];  d_map  device float [npy][npx].
 * FP32 cell-local traversal and segment optical depths as in the tracer;
 * the source function per cell and the accumulation along the ray in FP64.
 * Uses a per-context scratch of n_cells doubles (calls on one context must
 * not overlap on the GPU).  Asynchronous.
 * ------------------------------------------------------------------------ */
soc_status soc_map(soc_ctx *ctx, int cloud_id, const float *d_T, int freq, const double *dir, const double *up,
                   int npx, int npy, double pix_size, const double *center, double I_bg, float *d_map,
                   void *stream);

/* ------------------------------------------------------------------------
 * soc_iterate -- the iteration of paper Sect. 2.1.2 / 3.3: iteration 0
 * simulates the constant sources (background, point sources) once and keeps
 * their absorbed power; iterations k >= 1 re-simulate only dust re-emission
 * from T_{k-1} (with the same random numbers every iteration), add the
 * constant part and update T, until max |T_k - T_{k-1}| < dT_tol or
 * max_iter iterations.  Synchronises once per iteration (reads max |dT|).
 * With a reference field, iteration k uses n_k dust packages per frequency
 * (n_dust_first .. n_dust_last, or n_weighted), the reference step
 * w_k = n_k / (n_1 + .. + n_k) and random-number iteration key k; mode 1
 * traces the full emission (soc_dust_emission, soc_dust_weighted) and
 * averages, mode 2 traces the change (soc_dust_luminosity ..
 * soc_reference_update).
 *   d_T_seed          device float [n_cells] or NULL: initial temperatures
 *                     (e.g. a learned prediction); NULL uses T from the
 *                     constant sources alone.
 *   d_T_out           device float [n_cells]: final temperatures.
 *   res               host, out (may be NULL).
 *   dT_history        host double [max_iter] or NULL: max |dT| per iteration.
 * ------------------------------------------------------------------------ */
typedef struct soc_iterate_params {
    uint64_t n_background;     /* background packages per frequency (0: none)  */
    uint64_t n_point;          /* point-source packages per frequency (0: none) */
    uint32_t n_per_cell;       /* dust packages per leaf and frequency          */
    int32_t max_iter;          /* dust iterations after iteration 0 (>= 0)      */
    double dT_tol;             /* stop when max |dT| < dT_tol (K)               */
    int32_t reuse_constant;    /* 1: skip iteration 0 and reuse the constant-
                                  source absorption kept by the previous
                                  soc_iterate call on this cloud               */
    int32_t ali;               /* 1: accelerated update (diagonal operator,
                                  soc_update_temperature_ali)                  */
    uint64_t n_weighted;       /* > 0: emission-weighted dust sampling with about
                                  this many packages per frequency (replaces
                                  n_per_cell), see soc_dust_weighted; the
                                  allocation is made at the first dust
                                  iteration and kept (soc_dust_reweight)       */
    uint32_t weighted_cap;     /* packages per cell at most (weighted sampling) */
    int32_t reference_field;   /* reference field (paper Sect. 2.1.2), fresh
                                  random numbers per dust iteration, emission-
                                  weighted sampling, not with ali.
                                  1 (mean): every dust iteration traces the
                                  full dust emission; A_ref = package-weighted
                                  mean of the estimates; T from A_const + A_ref.
                                  2 (difference): traces only the change of
                                  the emission against the running mean of the
                                  earlier emissions; T from A_const + A_ref +
                                  the traced change (the noise of the first
                                  estimate stays in A_ref).                    */
    uint64_t n_dust_first;     /* reference field: dust packages per frequency
                                  of the first dust iteration (0: n_weighted
                                  for every iteration)                         */
    uint64_t n_dust_last;      /* ... and of iteration max_iter; log n grows
                                  linearly in between (paper Sect. 3.6)       */
} soc_iterate_params;

typedef struct soc_iterate_result {
    int32_t iterations;        /* dust iterations done                          */
    int32_t converged;         /* 1 if max |dT| < dT_tol was reached            */
    double final_max_dT;
    int64_t steps;             /* photon-cell steps over all iterations          */
    int64_t capped;            /* packages ended by the step cap                */
} soc_iterate_result;

soc_status soc_iterate(soc_ctx *ctx, int cloud_id, const soc_iterate_params *params,
                       const float *d_T_seed, float *d_T_out, soc_iterate_result *res,
                       double *dT_history, void *stream);

/* ------------------------------------------------------------------------
 * soc_iterate_batch -- soc_iterate for n_clouds clouds at once: iteration 0
 * traces the background and point sources of every cloud in one tracer
 * launch, and each dust iteration traces the re-emission of every cloud not
 * yet converged in one launch (paper Sect. 4.2: many work items interleaved
 * in one kernel), then updates each cloud's T.  A cloud leaves the batch once
 * its max |dT| < dT_tol.  Each cloud's results (T, iterations, steps) are
 * bit-identical to soc_iterate on that cloud alone (the packages, their
 * random numbers and their integer counters do not depend on the launch).
 * Synchronises once per iteration.
 *   cloud_ids         host int [n_clouds], distinct uploaded clouds.
 *   params            as soc_iterate; n_weighted and reference_field must
 *                     be 0 (SOC_ERR_ARG), ali is supported.
 *   d_T_seed          host array [n_clouds] of device float pointers, or
 *                     NULL; a NULL entry starts that cloud from the constant
 *                     sources' T.
 *   d_T_out           host array [n_clouds] of device float [n_cells].
 *   res               host [n_clouds] or NULL.
 *   dT_history        host double [n_clouds][max_iter] or NULL.
 * Scratch: counters for every item of one launch (library-owned, kept for
 * the next call).  Abort flag and watchdog as soc_iterate.
 * ------------------------------------------------------------------------ */
soc_status soc_iterate_batch(soc_ctx *ctx, int n_clouds, const int *cloud_ids, const soc_iterate_params *params,
                             const float *const *d_T_seed, float *const *d_T_out, soc_iterate_result *res,
                             double *dT_history, void *stream);

/* ------------------------------------------------------------------------
 * soc_nn_error_flag -- 1 if a tensor-core convolution block gave up waiting
 * for its matrix multiplies (each wait is bounded; the block then frees its
 * tensor memory and returns without writing its outputs), else 0; the flag
 * of the current device is cleared.  Synchronous with the device.
 * ------------------------------------------------------------------------ */
soc_status soc_nn_error_flag(int *flag);

/* ------------------------------------------------------------------------
 * Learned temperature seed (not a step of the paper's method: a 3D U-Net that
 * maps the first, noisy temperature field and the log density to the
 * converged temperature and seeds soc_iterate; the Monte Carlo iterations
 * then check the seed and remain its fallback).  Channels-last (N, side,
 * side, side, C) tensors; BF16 activations and weights on the tcgen05 tensor
 * cores with FP32 accumulation in tensor memory (convolutions, input and
 * weight gradients); FP32 master weights, gradients and Adam moments.  Architecture: 4 levels with
 * 16-32-64-128 channels, two 3x3x3 convolutions (ReLU) per level, 2x2x2 max
 * pooling, nearest 2x upsampling, skip concatenation [upsampled, skip], a
 * 3x3x3 output convolution (channel 0 = prediction).  side % 8 == 0.
 * Parameters are packed layer by layer (15 layers in forward order), each as
 * w[Cout][27][Cin] then b[Cout], FP32; soc_unet_param_count() floats.
 *   soc_unet_create     device buffers for a batch size, cube side and number
 *                       of input channels n_inputs (1..16; the first layer
 *                       always has 16 input channels, the ones beyond
 *                       n_inputs read zeros).
 *   soc_unet_forward    d_input (N,S,S,S,n_inputs) FP32 device -> d_pred (N,S,S,S).
 *   soc_unet_backward   forward, MSE loss against d_target (N,S,S,S), and
 *                       the gradients of every parameter (kept in the net);
 *                       d_pred / d_loss (device double) optional.
 *   soc_unet_adam       one Adam step (beta 0.9, 0.999, eps 1e-8) with lr.
 *   soc_unet_get_params host copy of the parameters (grads = 0) or of their
 *                       gradients (grads = 1).  Synchronous.
 * ------------------------------------------------------------------------ */
soc_status soc_unet_create(int device, int batch, int side, int n_inputs, int *net_id);
soc_status soc_unet_destroy(int net_id);
int64_t soc_unet_param_count(void);
soc_status soc_unet_set_params(int net_id, const float *host_params);
soc_status soc_unet_get_params(int net_id, float *host_params, int grads);
soc_status soc_unet_forward(int net_id, const float *d_input, float *d_pred, void *stream);
soc_status soc_unet_backward(int net_id, const float *d_input, const float *d_target, float *d_pred,
                             double *d_loss, void *stream);
soc_status soc_unet_adam(int net_id, float lr, void *stream);

/* Single network operations (channels-last BF16, Cin and Cout multiples of
 * 16), the building blocks of the U-Net:
 *   soc_nn_conv3d        y = relu?(conv3x3x3(x, w) + bias) into y_bf16 or y_f32;
 *   soc_nn_conv3d_dgrad  gx (FP32) = transposed convolution of gy with w
 *                        (w_scratch: device BF16 [Cout*27*Cin]);
 *   soc_nn_conv3d_wgrad  gw[Cout][27][Cin] += sum_v gy[v] x[v + tap] and
 *                        gb[Cout] += sum_v gy[v] (FP32, accumulated).  The
 *                        voxels are split over blocks whose partial sums go
 *                        to a library-owned workspace of the device (grown
 *                        on demand with cudaMalloc) and are added in a fixed
 *                        order: bit-reproducible.  Calls on one device share
 *                        the workspace and must not overlap on the GPU.
 *   soc_nn_adam          one Adam step (Kingma & Ba 2015) at step t >= 1 on
 *                        n FP32 parameters d_w with moments d_m, d_v (device,
 *                        in/out) and gradients d_g: beta1 0.9, beta2 0.999,
 *                        eps 1e-8 (FP32 constants), bias corrections
 *                        1 - beta^t; d_w_bf16 (device BF16 [n] or NULL)
 *                        receives the rounded weights.  The U-Net's
 *                        soc_unet_adam runs the same kernel. */
soc_status soc_nn_conv3d(const void *x, int N, int D, int H, int W, int Cin, const void *w, const float *bias,
                         int Cout, int relu, void *y_bf16, float *y_f32, void *stream);
soc_status soc_nn_conv3d_dgrad(const void *gy, int N, int D, int H, int W, int Cout, const void *w, int Cin,
                               void *w_scratch, float *gx, void *stream);
soc_status soc_nn_conv3d_wgrad(const void *gy, const void *x, int N, int D, int H, int W, int Cin, int Cout,
                               float *gw, float *gb, void *stream);
soc_status soc_nn_adam(float *d_w, float *d_m, float *d_v, const float *d_g, int64_t n, float lr, int32_t t,
                       void *d_w_bf16, void *stream);

/* soc_nn_scale_add: d_y[i] = fma(a, d_x[i], d_y[i]) for i < n (device FP32,
 * d_y in/out, one rounding per element), in the order of the calls on the
 * stream.  The learned seed averages the predictions of an ensemble of
 * networks with it (a = 1/K per member, members in a fixed order, so the
 * mean is bit-reproducible).  SOC_ERR_ARG for null pointers, n < 1 or a NaN. */
soc_status soc_nn_scale_add(float *d_y, const float *d_x, int64_t n, float a, void *stream);

/* ------------------------------------------------------------------------
 * Seeding transform of the learned temperature seed (not a step of the
 * paper's method), per cell of an uploaded regular grid, in FP64:
 *   soc_seed_features   network input d_x (device float [n_cells][n_features],
 *                       the channels-last (side, side, side, n_features)
 *                       layout of one sample), n_features 2, 3 or 4:
 *                       x[c][0] = (ln clamp(T[c], 2.7, 3000) - norm[0]) / norm[1],
 *                       x[c][1] = (ln max(rho_c, 1e-30) - norm[2]) / norm[3],
 *                       x[c][2] = (ln clamp(T[c]) - ln clamp(T_prev[c]) -
 *                                  norm[4]) / norm[5]   (n_features >= 3:
 *                       the last iteration's change; d_T_prev required),
 *                       x[c][3] = (ln clamp(T_prev[c]) - ln clamp(T_prev2[c]) -
 *                                  norm[6]) / norm[7]   (n_features = 4:
 *                       the change one iteration earlier; d_T_prev2
 *                       required; NULL otherwise),
 *                       each feature clipped to [-6, 6] after the
 *                       standardisation; rho from the uploaded grid.  norm:
 *                       host double [2 n_features], {mean, width} of each
 *                       feature over the training set (widths > 0).  The grid must be a
 *                       regular cube whose side is a multiple of 8
 *                       (SOC_ERR_ARG otherwise).
 *   soc_seed_transform  for every cell (the network predicts the normalised
 *                       y = ln T - ln T1):
 *                         y = shrink (pred[c] y_std + y_mean);
 *                         with an envelope (n_bins > 0): bin b of ln T1
 *                         (n_bins equal bins over [lnT1_lo, lnT1_hi), the
 *                         end bins extended), y = min(max(y, y_lo[b]), y_hi[b]);
 *                         d_T_seed[c] = clamp(T1[c] exp(y), 2.7, 3000).
 *                       map: host soc_seed_map (copied into the launch).
 *                       d_T1, d_pred, d_T_seed: device float [n_cells].
 *   soc_nn_seed_features  the features of soc_seed_features from caller
 *                       arrays (no context): d_T, d_T_prev, d_T_prev2, d_rho
 *                       device float [n], d_x device float [n][n_features] (e.g. a
 *                       training set kept after its clouds were freed).
 * All asynchronous on `stream`; d_T_seed may be passed as the seed of
 * soc_iterate or soc_iterate_batch.
 * ------------------------------------------------------------------------ */
soc_status soc_seed_features(soc_ctx *ctx, int cloud_id, const float *d_T, const float *d_T_prev,
                             const float *d_T_prev2, const double *norm, int n_features, float *d_x, void *stream);
#define SOC_SEED_MAX_BINS 64
typedef struct soc_seed_map {
    double y_mean, y_std;      /* de-normalisation of the prediction            */
    double shrink;             /* factor on the de-normalised prediction (> 0) */
    int32_t n_bins;            /* 0: no envelope; else 1..SOC_SEED_MAX_BINS     */
    int32_t reserved;
    double lnT1_lo, lnT1_hi;   /* the bins' range of ln T1 (lo < hi)            */
    double y_lo[SOC_SEED_MAX_BINS], y_hi[SOC_SEED_MAX_BINS];   /* per-bin bounds */
} soc_seed_map;
soc_status soc_seed_transform(soc_ctx *ctx, int cloud_id, const float *d_T1, const float *d_pred,
                              const soc_seed_map *map, float *d_T_seed, void *stream);
soc_status soc_nn_seed_features(const float *d_T, const float *d_T_prev, const float *d_T_prev2, const float *d_rho,
                                int64_t n, const double *norm, int n_features, float *d_x, void *stream);

/* ------------------------------------------------------------------------
 * Launch configuration of the tracer (autotuner hook).  threads_per_block in
 * {32, 64, ..., 256}; blocks_per_sm >= 1 (0 = occupancy maximum of the
 * default build; 4 or more selects the build limited to 64 registers per
 * thread, which keeps 4 blocks of 256 threads resident per SM); chunk in
 * [1, 1024] = packages per lane that a warp takes from the global work
 * counter at a time.
 * Results do not depend on these settings.
 * ------------------------------------------------------------------------ */
soc_status soc_set_launch(soc_ctx *ctx, int threads_per_block, int blocks_per_sm, int chunk);
/* A warp refills its idle lanes with new packages once at least
 * min_idle_lanes (1..32) of its 32 lanes are idle (or all are): emission then
 * runs for several lanes together instead of one lane at a time.  Results do
 * not depend on it. */
soc_status soc_set_refill(soc_ctx *ctx, int min_idle_lanes);
/* A lane whose package has to scatter waits until min_lanes (1..32) lanes of
 * its warp wait too (or every active lane does); the warp then draws their
 * new directions together instead of diverging on every scattering.  Each
 * package's draws and operations keep their order: results do not depend
 * on it. */
soc_status soc_set_scatter_batch(soc_ctx *ctx, int min_lanes);
/* Step cap per package (default 10^7); packages beyond it are ended with
 * their weight deposited and counted in stats[1]. */
soc_status soc_set_max_steps(soc_ctx *ctx, uint32_t max_steps);

/* ------------------------------------------------------------------------
 * Abort flag and watchdog (failure handling; the paper has no counterpart).
 * Every context owns a flag in host-mapped pinned memory.  Each tracer
 * launch (direct, allocation-free, prepared batch or graph replay) reads it
 * whenever a warp takes a new chunk of work: once it is set, warps take no
 * more work and the launch ends after the packages already in flight (each
 * bounded by the step cap).  The counters and statistics then hold exactly
 * the packages that were traced: per item, sum(tally) + escaped == emitted
 * still holds, with emitted below the full count.
 *   soc_abort         sets the flag; callable from any host thread at any
 *                     time (a plain store, no CUDA call).  The flag stays
 *                     set, and every later launch traces nothing, until
 *                     soc_abort_clear.
 *   soc_abort_clear   clears the flag and the "cut" record.  Call it when no
 *                     launch of the context is in flight.
 *   soc_abort_status  *requested = the flag, *cut = 1 if a launch since the
 *                     last clear left work untraced (read it after the
 *                     launches have finished, e.g. after a stream sync).
 *                     Either pointer may be NULL.
 *   soc_set_timeout   seconds > 0: each soc_iterate call starts a host
 *                     watchdog thread that sets the flag when the call has
 *                     run that long; 0 (default) = none.
 * soc_iterate checks the flag before each tracer launch and after each
 * iteration's synchronisation; when it is set it returns SOC_ERR_TIMEOUT
 * with *res describing the iterations completed.  The flag stays set.
 * ------------------------------------------------------------------------ */
soc_status soc_abort(soc_ctx *ctx);
soc_status soc_abort_clear(soc_ctx *ctx);
soc_status soc_abort_status(soc_ctx *ctx, int *requested, int *cut);
soc_status soc_set_timeout(soc_ctx *ctx, double seconds);

/* ------------------------------------------------------------------------
 * soc_probe_read -- measurement helper for the tracer's roofline (not part
 * of the method): one launch that reads the device buffer d_buf of `bytes`
 * bytes `reps` times over with 16-byte loads that bypass L1, on `stream`
 * (cudaStream_t or NULL).  A buffer that fits in L2 is read from L2 after
 * the first pass, so (bytes x reps) / launch time is the L2 read bandwidth;
 * a larger one measures HBM.  The caller times it (CUDA events on the same
 * stream).  d_buf: device pointer, 16-byte aligned; bytes: a positive
 * multiple of 16; reps >= 1; otherwise SOC_ERR_ARG.  The contents are not
 * changed.
 * ------------------------------------------------------------------------ */
soc_status soc_probe_read(soc_ctx *ctx, const void *d_buf, uint64_t bytes, int32_t reps, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SOC_H */
