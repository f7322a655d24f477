// soc_internal.h -- device-side data layout shared by the libsoc translation
// units (not part of the public C-ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/soc.h"

namespace soc {

constexpr uint32_t kLinkBit = 0x80000000u;   // cell word: bit 31 = refined
constexpr double kWUnit = 2147483648.0;      // fixed-point units of one full package (SOC_W_UNIT)
constexpr int kTableN = 4096;                // T grid of the emission table
constexpr double kTMin = 2.7, kTMax = 3000.0;

// One uploaded grid as the kernels see it (lives in device memory, in an
// array indexed by cloud id).  Cell words: FP32 density, or kLinkBit | first
// child.  Octet k (cells n_root + 8k .. +7) has parent parent[k].
struct DevCloud {
    const uint32_t *cell;        // [n_cells]
    const int32_t *parent;       // [n_octets]
    const int32_t *leaf;         // [n_leaf] leaf cells in increasing order
    const float *rho;            // [n_cells] FP32 density (0 for refined cells)
    const double *volume;        // [n_cells] cm^3
    const float2 *kappa;         // [n_freq] (kabs * ell, ksca * ell) per root-cell length
    const float *ps_pos;         // [3 n_ps] root-cell units
    const float *ps_cdf;         // [n_freq][n_ps] cumulative luminosity fraction
    int32_t nx, ny, nz, n_levels;
    int32_t n_ps, pad_;
    int64_t n_cells, n_root, n_leaf;
    int64_t level_start[SOC_MAX_LEVELS + 1];
};

// Batch item after preparation on the host.
constexpr uint32_t kItemWeighted = 1u;   // dust weights followed by the package prefix

struct DevItem {
    int32_t cloud, freq, source, iteration;
    uint32_t pid_offset, n_per_cell;
    uint32_t flags, pad_;
    uint64_t w0;
    int64_t tally_offset;
    const uint64_t *dust_w;
};

// The cloud fields the tracer's step reads (see TraceParams::hot).
struct HotCloud {
    const uint32_t *cell;
    const int32_t *parent;
    int32_t nx, ny, nz, n_root;
};

struct TraceParams {
    const DevCloud *clouds;
    const DevItem *items;
    const uint64_t *prefix;      // [n_items + 1] exclusive prefix of n_packages
    const float *g_hg;           // [n_freq]
    unsigned long long *tally;
    unsigned long long *self;    // nullable: same layout as tally; deposits of dust
                                 // packages in their emission cell before they leave it
    unsigned long long *stats;   // [n_items][4]
    uint32_t *pkg_steps;         // nullable
    unsigned long long *counter; // global work counter
    uint64_t total;
    uint64_t seed;
    int32_t n_items;
    uint32_t max_steps;
    int32_t chunk;
    int32_t refill_min;          // refill a warp's idle lanes once this many are idle
    int32_t scatter_min;         // scatter a warp's waiting lanes once this many wait
    const int *abort_flag;       // host-mapped: nonzero = take no more work (soc_abort)
    int *cut;                    // host-mapped: set to 1 when work was left untraced
    HotCloud hot;                // cell != nullptr: every item uses this one cloud
    int32_t regular;             // every item's cloud is a regular grid (selects the
                                 // tracer build without octree traversal, two steps
                                 // per pass)
};

// variant: 3 or 4 = minimum resident 256-thread blocks per SM the kernel is
// compiled for (register budget 80 or 64 per thread)
cudaError_t launch_trace(const TraceParams &p, int grid, int block, int variant, cudaStream_t s);
int trace_block_limit(int block, int variant, bool regular);   // max resident blocks/SM

// Surface-brightness map of one frequency seen along direction d (rays
// travel along d); pixel (px, py) centre = c + ((px+0.5) - npx/2) pix e1 +
// ((py+0.5) - npy/2) pix e2, all in root-cell units.
struct MapParams {
    const DevCloud *cloud;
    const float *T;               // [n_cells]
    double *S;                    // [n_cells] scratch: (kabs/kext) B_nu(T) per cell
    float *map;                   // [npy][npx]
    double d[3], e1[3], e2[3], c[3];
    double pix, nu, kext_root, kabs_over_kext, I_bg;
    int32_t npx, npy;
    uint32_t max_cells;
};

// source-function pass over the n_cells cells into m.S, then one thread per pixel
cudaError_t launch_map(const MapParams &m, int64_t n_cells, int sms, cudaStream_t s);

struct TempTables {
    int n_freq;
    const double *w_kabs;        // [n_freq] 4 pi w_nu kabs(nu)
    const double *w;             // [n_freq] trapezoid weights
    const double *nu;            // [n_freq]
    const double *kabs;          // [n_freq] physical cross sections
    const double *lnE;           // [kTableN]
    const double *lnT;           // [kTableN]
};

cudaError_t launch_absorbed_power(const DevCloud *dcl, int64_t n_cells, const int64_t *tally,
                                  int64_t stride, const double *e_unit, const double *w, int n_freq,
                                  const double *A_in, double *A_out, cudaStream_t s);
cudaError_t launch_update_temperature(const DevCloud *dcl, int64_t n_cells, const TempTables &tt,
                                      const double *A, float *T, double *max_dT, cudaStream_t s);
cudaError_t launch_dust_weighted(int64_t n_leaf, int n_freq, const uint64_t *u, const double *e_uni, uint64_t n_total,
                                 uint32_t cap, uint64_t *out, double *e_unit, unsigned long long *scratch,
                                 cudaStream_t s);
cudaError_t launch_dust_reweight(int64_t n_leaf, int n_freq, const uint64_t *u, const double *e_uni, uint64_t *out,
                                 double *e_unit, unsigned long long *scratch, cudaStream_t s);
cudaError_t launch_dust_luminosity(const DevCloud *dcl, int64_t n_leaf, const TempTables &tt, const float *T,
                                   int freq_lo, int n_freq, double *L, cudaStream_t s);
cudaError_t launch_reference_delta(int64_t n_leaf, int n_freq, const double *L, double *L_ref, double w, uint64_t *u,
                                   uint8_t *neg, double *e_uni, unsigned long long *scratch, cudaStream_t s);
cudaError_t launch_dust_split(int64_t n_leaf, int n_freq, const uint8_t *neg, uint64_t *alloc, uint64_t *alloc_neg,
                              const double *e, double *e_neg, cudaStream_t s);
cudaError_t launch_reference_update(int64_t n, double *A_ref, const double *A_d, double w, const double *A_const,
                                    double *A_out, int out_mean, cudaStream_t s);
cudaError_t launch_cell_init(const uint32_t *word, int64_t n, const int64_t *start, int n_levels, double ell3,
                             float *rho, double *vol, cudaStream_t s);
cudaError_t launch_update_temperature_ali(const DevCloud *dcl, int64_t n_cells, const TempTables &tt,
                                          const double *A, const double *A_self, float *T, double *max_dT,
                                          cudaStream_t s);
cudaError_t launch_dust_emission(const DevCloud *dcl, int64_t n_leaf, const TempTables &tt, const float *T,
                                 int freq_lo, int n_freq, uint32_t n_per_cell, uint64_t *w,
                                 double *e_unit, unsigned long long *scratch_max, cudaStream_t s);

// Learned seed: network features of a cloud's cells and the seeding transform
// (soc_nn.cu).  norm: {mean, width} of each feature (2, 3 or 4 features).
struct SeedNorm { double v[8]; };
cudaError_t launch_seed_features(const float *T, const float *T_prev, const float *T_prev2, const float *rho,
                                 int64_t n, int n_features, const double *norm, float *x, cudaStream_t s);
cudaError_t launch_seed_transform(const float *T1, const float *pred, int64_t n, const soc_seed_map &map,
                                  float *T_seed, cudaStream_t s);

}  // namespace soc
