/*
 * soc_oracle.c -- plain, slow, single-threaded CPU oracle for the Monte Carlo
 * photon-package tracer of SOC (Juvela 2019, arXiv:1812.06632).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / --impl reference legs use it.  It shares no code, header or
 * constant table with the CUDA library; both sides implement, separately, the
 * same FP32 contract (stated operation by operation in the comments below).
 *
 * What it follows in the paper (Sect. 2.1.1, "Basic program"):
 *   - a regular root grid of cubic cells refined by octrees into octets of
 *     eight equal sub-cells, stored as one level-ordered cell vector with each
 *     octet contiguous, a link from every refined cell to its first child and
 *     a reverse link from every octet to its parent;
 *   - on every cell change the package climbs the hierarchy only as far as
 *     the common ancestor and then descends to the leaf it enters (no
 *     neighbour lists);
 *   - packages are simulated one frequency at a time and every cell keeps a
 *     counter of the energy absorbed in it.
 * The paper gives no transport formulas.  The readings used here: absorption
 * as continuous attenuation of the package weight, free paths drawn in
 * scattering optical depth, Henyey-Greenstein scattering, cosine-weighted
 * background entry through the six faces, isotropic point sources, uniform
 * in-cell dust emission, and uint64 fixed-point counters (2^31 units per
 * package) so that energy is conserved exactly.
 *
 * Arithmetic: IEEE binary32, round-to-nearest-even, one rounding per written
 * operation (compiled with -ffp-contract=off and without fast-math); the
 * fused multiply-adds the contract names are explicit fmaf calls.  1 - exp
 * and log are the project's own polynomials (Cody-Waite reduction + Taylor
 * series; atanh series), not libm.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random       */
/* numbers: as easy as 1, 2, 3").  Multipliers and Weyl key increments are   */
/* the published ones.                                                       */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One package's stream of draws.  Key = (seed_lo, seed_hi ^ iter<<16 ^ freq),
 * counter = (package id, block index, cloud, source class); draw n is word
 * n%4 of block n/4. */
typedef struct {
    uint32_t key[2];
    uint32_t pid, cloud, cls;
    uint32_t n;        /* draws consumed */
    uint32_t buf[4];
} rng_t;

static void rng_init(rng_t *r, uint64_t seed, uint32_t iteration, uint32_t freq,
                     uint32_t pid, uint32_t cloud, uint32_t cls)
{
    r->key[0] = (uint32_t)seed;
    r->key[1] = (uint32_t)(seed >> 32) ^ (iteration << 16) ^ freq;
    r->pid = pid; r->cloud = cloud; r->cls = cls; r->n = 0;
}

static uint32_t rng_next(rng_t *r)
{
    if ((r->n & 3u) == 0) {
        uint32_t ctr[4] = { r->pid, r->n >> 2, r->cloud, r->cls };
        oracle_philox4x32_10(ctr, r->key, r->buf);
    }
    uint32_t v = r->buf[r->n & 3u];
    r->n++;
    return v;
}

/* u = ((x >> 8) | 1) * 2^-24 : odd multiples of 2^-24, never 0 or 1. */
float oracle_u01(uint32_t x) { return (float)((x >> 8) | 1u) * 0x1p-24f; }

static float rng_u(rng_t *r) { return oracle_u01(rng_next(r)); }

/* ------------------------------------------------------------------------- */
/* Elementary functions of the contract.                                      */
/* ------------------------------------------------------------------------- */
static const float LN2_HI = 0x1.62e4p-1f;        /* 45426 / 65536, exact with 16 bits */
static const float LN2_LO = 0x1.7f7d1cp-20f;     /* RN(ln 2 - LN2_HI)                */
static const float LOG2E  = 0x1.715476p+0f;      /* RN(1 / ln 2)                     */
static const float SQRT2F = 0x1.6a09e6p+0f;      /* RN(sqrt 2)                       */

static float bits_to_float(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t float_to_bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* 1 - exp(-tau), tau >= 0, with full relative accuracy at every tau and no
 * branch on tau: x = max(-tau, -87) = k ln2 + r (Cody-Waite: k = rint(x / ln2),
 * r = x - k LN2_HI - k LN2_LO by two fused multiply-adds, |r| <= ln2/2);
 * e^r - 1 = r P(r), P the Taylor series of (e^r - 1)/r to degree 6 with
 * coefficients RN(1/n!), in Horner form with fused multiply-adds; then
 * 1 - e^x = (1 - 2^k) - 2^k (e^r - 1) as one fused multiply-add.  For tau
 * below ln2/2 (k = 0) the result is -(e^r - 1) itself, so thin cells keep
 * full relative accuracy.  tau <= 0 (or NaN) gives 0.  fmaf is the C99
 * fused multiply-add, rounded once (the CUDA side uses __fmaf_rn). */
float oracle_one_minus_exp(float tau)
{
    const float x = fmaxf(-tau, -87.0f);
    const float t = rintf(x * LOG2E);           /* k as an integral float, in [-126, 0] */
    const int k = (int)t;
    float r = fmaf(-t, LN2_HI, x);
    r = fmaf(-t, LN2_LO, r);
    float p = 0x1.a01a02p-13f;                  /* 1/7! */
    p = fmaf(p, r, 0x1.6c16c2p-10f);            /* 1/6! */
    p = fmaf(p, r, 0x1.111112p-7f);             /* 1/5! */
    p = fmaf(p, r, 0x1.555556p-5f);             /* 1/4! */
    p = fmaf(p, r, 0x1.555556p-3f);             /* 1/3! */
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    const float em1 = r * p;                    /* e^r - 1 */
    const float scale = bits_to_float((uint32_t)(k + 127) << 23);      /* 2^k */
    const float q = fmaf(-scale, em1, 1.0f - scale);
    return (tau > 0.0f) ? q : 0.0f;
}

/* ln(u) for u in (0,1) (any positive normal u works).  u = m 2^e with
 * m in (sqrt(1/2), sqrt 2]; ln m = 2 atanh(s), s = (m-1)/(m+1):
 * ln m = 2s + 2s z (1/3 + z/5 + z^2/7 + z^3/9), z = s^2. */
float oracle_log(float u)
{
    uint32_t b = float_to_bits(u);
    int e = (int)(b >> 23) - 127;
    float m = bits_to_float((b & 0x007fffffu) | 0x3f800000u);
    if (m > SQRT2F) { m = m * 0.5f; e = e + 1; }
    float f = m - 1.0f;
    float s = f / (m + 1.0f);
    float z = s * s;
    float q = 0x1.c71c72p-4f;                   /* 1/9 */
    q = q * z + 0x1.24924ap-3f;                 /* 1/7 */
    q = q * z + 0x1.99999ap-3f;                 /* 1/5 */
    q = q * z + 0x1.555556p-2f;                 /* 1/3 */
    float s2 = s + s;
    float lm = s2 + (s2 * z) * q;               /* leading term kept apart */
    float t = (float)e;
    return (t * LN2_LO + lm) + t * LN2_HI;
}

/* ------------------------------------------------------------------------- */
/* Grid, tables and work description (plain structs, filled from Python).   */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t nx, ny, nz;          /* root grid                                       */
    int32_t n_levels;
    int64_t n_cells;
    const int64_t *level_start;  /* [n_levels+1]                                    */
    const float *rho;            /* [n_cells] density of leaves (parents: ignored)  */
    const int32_t *child;        /* [n_cells] first child index, -1 for a leaf      */
    const int32_t *parent;       /* [(n_cells - n_root)/8] parent of each octet     */
} oracle_grid;

enum { SRC_BACKGROUND = 0, SRC_POINT = 1, SRC_DUST = 2 };

typedef struct {
    int32_t source;              /* SRC_*                                           */
    int32_t freq;                /* frequency index (enters the RNG key)             */
    int32_t iteration;           /* RNG stream selector                              */
    int32_t cloud;               /* enters the RNG counter                           */
    uint64_t seed;
    float kabs, ksca, g;         /* per root-cell length and unit density; HG g     */
    uint64_t w0;                 /* initial weight (background / point sources)     */
    uint32_t max_steps;
    /* point sources */
    int32_t n_ps;
    const float *ps_pos;         /* [3 n_ps], root-cell units                       */
    const float *ps_cdf;         /* [n_ps] cumulative luminosity fraction (last = 1) */
    /* dust emission */
    uint32_t n_per_cell;
    int64_t n_leaf;
    const int32_t *leaf;         /* [n_leaf] leaf cell indices, increasing          */
    const uint64_t *dust_w;      /* [n_leaf] initial weight of each cell's packages */
    const uint64_t *dust_prefix; /* [n_leaf+1] or NULL: package ids of leaf li are
                                    prefix[li] .. prefix[li+1]-1 (weighted sampling) */
} oracle_item;

typedef struct {
    int64_t escaped;             /* sum of W leaving the root grid                  */
    int64_t capped;              /* packages ended by the step cap                  */
    int64_t steps;               /* photon-cell steps                               */
    int64_t emitted;             /* sum of initial W                                */
} oracle_stats;

/* Package state in the cell-local frame of its current leaf. */
typedef struct {
    int32_t cell;
    float h;                     /* cell side in root-cell units (power of two)     */
    float x[3];                  /* position in [0,1]^3 of the cell                  */
    float d[3];                  /* direction                                        */
    float inv[3];                /* 1/d per axis (unused where d == 0)               */
    uint64_t W;
} pkg_t;

static float clamp01(float v) { return fminf(fmaxf(v, 0.0f), 1.0f); }

static int64_t n_root_of(const oracle_grid *G) { return (int64_t)G->nx * G->ny * G->nz; }

static void set_inverse(pkg_t *p)
{
    for (int i = 0; i < 3; ++i) p->inv[i] = (p->d[i] != 0.0f) ? 1.0f / p->d[i] : 0.0f;
}

/* Leaf lookup from a root cell: follow child links; the child octant on each
 * axis is the upper one when 2x >= 1 (x on the mid plane goes up). */
static void descend(const oracle_grid *G, pkg_t *p)
{
    while (G->child[p->cell] >= 0) {
        int oct = 0;
        for (int i = 0; i < 3; ++i) {
            float x2 = 2.0f * p->x[i];
            int b = (x2 >= 1.0f) ? 1 : 0;
            p->x[i] = x2 - (float)b;
            oct |= b << i;
        }
        p->h = p->h * 0.5f;
        p->cell = G->child[p->cell] + oct;
    }
}

/* Unit-disk rejection sample -> (cos phi, sin phi), no trigonometry.  At
 * most 64 tries (all rejected with probability < 1e-42); then azimuth 0. */
static void disk_azimuth(rng_t *r, float *c, float *s)
{
    float a = 1.0f, b = 0.0f, r2 = 1.0f;
    for (int tries = 0; tries < 64; ++tries) {
        float ta = 2.0f * rng_u(r) - 1.0f;
        float tb = 2.0f * rng_u(r) - 1.0f;
        float t2 = ta * ta + tb * tb;
        if (t2 <= 1.0f && t2 > 0.0f) { a = ta; b = tb; r2 = t2; break; }
    }
    float rr = sqrtf(r2);
    *c = a / rr;
    *s = b / rr;
}

/* Isotropic direction: mu = 2u - 1, azimuth from the disk sampler. */
static void isotropic_direction(rng_t *r, float d[3])
{
    float mu = 2.0f * rng_u(r) - 1.0f;
    float c, s;
    disk_azimuth(r, &c, &s);
    float sint = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
    d[0] = sint * c;
    d[1] = sint * s;
    d[2] = mu;
}

/* Henyey-Greenstein scattering of direction d with asymmetry g.
 *   cos(theta) = (1 + g^2 - ((1 - g^2) / (1 - g + 2 g u))^2) / (2 g),
 *   isotropic (2u - 1) when |g| < 1e-4;
 * azimuth from the disk sampler; the new direction by the usual rotation
 * about the old one, then renormalised. */
static void hg_scatter(rng_t *r, float g, float d[3])
{
    float u = rng_u(r);
    float mu;
    if (fabsf(g) < 1e-4f) {
        mu = 2.0f * u - 1.0f;
    } else {
        float g2 = g * g;
        float den = (1.0f - g) + (g + g) * u;
        float tmp = (1.0f - g2) / den;
        mu = ((1.0f + g2) - tmp * tmp) / (g + g);
        mu = fminf(fmaxf(mu, -1.0f), 1.0f);
    }
    float c, s;
    disk_azimuth(r, &c, &s);
    float sint = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
    float dx = d[0], dy = d[1], dz = d[2];
    float nx, ny, nz;
    if (fabsf(dz) > 0.99999f) {
        nx = sint * c;
        ny = sint * s;
        nz = (dz > 0.0f) ? mu : -mu;
    } else {
        float t = sqrtf(1.0f - dz * dz);
        nx = (sint * ((dx * dz) * c - dy * s)) / t + dx * mu;
        ny = (sint * ((dy * dz) * c + dx * s)) / t + dy * mu;
        nz = dz * mu - (sint * c) * t;
    }
    float nrm = sqrtf((nx * nx + ny * ny) + nz * nz);
    d[0] = nx / nrm;
    d[1] = ny / nrm;
    d[2] = nz / nrm;
}

/* Root cell containing root-unit coordinate v along an axis of n cells, and
 * the cell-local coordinate v - i. */
static int root_index(float v, int n, float *local)
{
    int i = (int)v;
    if (i < 0) i = 0;
    if (i > n - 1) i = n - 1;
    *local = clamp01(v - (float)i);
    return i;
}

/* Emission of package pid of an item.  Returns 0 for a package with zero
 * initial weight (dust cells that emit nothing). */
static int emit(const oracle_grid *G, const oracle_item *it, rng_t *r, uint32_t pid, pkg_t *p)
{
    const int nr[3] = { G->nx, G->ny, G->nz };
    int idx[3] = { 0, 0, 0 };
    p->h = 1.0f;
    if (it->source == SRC_BACKGROUND) {
        /* Face chosen with probability proportional to its area; faces are
         * ordered -x,+x,-y,+y,-z,+z (entering at x=0 means moving along +x). */
        float ax = (float)G->ny * (float)G->nz, ay = (float)G->nx * (float)G->nz,
              az = (float)G->nx * (float)G->ny;
        float cum[6];
        cum[0] = ax; cum[1] = cum[0] + ax; cum[2] = cum[1] + ay;
        cum[3] = cum[2] + ay; cum[4] = cum[3] + az; cum[5] = cum[4] + az;
        float t = rng_u(r) * cum[5];
        int f = 0;
        while (f < 5 && !(t < cum[f])) ++f;
        int a = f >> 1, low = ((f & 1) == 0);
        int t1 = (a == 0) ? 1 : 0, t2 = (a == 2) ? 1 : 2;
        float p1 = rng_u(r) * (float)nr[t1];
        float p2 = rng_u(r) * (float)nr[t2];
        idx[t1] = root_index(p1, nr[t1], &p->x[t1]);
        idx[t2] = root_index(p2, nr[t2], &p->x[t2]);
        idx[a] = low ? 0 : nr[a] - 1;
        p->x[a] = low ? 0.0f : 1.0f;
        float u = rng_u(r);
        float mu = sqrtf(u);                 /* cosine-weighted inward angle */
        float sint = sqrtf(1.0f - u);
        float c, s;
        disk_azimuth(r, &c, &s);
        p->d[a] = low ? mu : -mu;
        p->d[t1] = sint * c;
        p->d[t2] = sint * s;
        p->W = it->w0;
        p->cell = idx[0] + G->nx * (idx[1] + G->ny * idx[2]);
        descend(G, p);
        return 1;
    }
    if (it->source == SRC_POINT) {
        float t = rng_u(r);
        int k = 0;
        while (k < it->n_ps - 1 && !(t < it->ps_cdf[k])) ++k;
        for (int i = 0; i < 3; ++i) idx[i] = root_index(it->ps_pos[3 * k + i], nr[i], &p->x[i]);
        isotropic_direction(r, p->d);
        p->W = it->w0;
        p->cell = idx[0] + G->nx * (idx[1] + G->ny * idx[2]);
        descend(G, p);
        return 1;
    }
    /* Dust: n_per_cell packages from every leaf, or (weighted sampling) the
     * leaf whose range of package ids holds pid; uniform in the cell. */
    int64_t li;
    if (it->dust_prefix) {
        int64_t lo = 0, hi = it->n_leaf;          /* prefix[lo] <= pid < prefix[hi] */
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            if (it->dust_prefix[mid] <= (uint64_t)pid) lo = mid; else hi = mid;
        }
        li = lo;
    } else {
        li = (int64_t)(pid / it->n_per_cell);
    }
    p->cell = it->leaf[li];
    p->W = it->dust_w[li];
    if (p->W == 0) return 0;
    int L = 0;
    while (L + 1 < G->n_levels && (int64_t)p->cell >= G->level_start[L + 1]) ++L;
    p->h = ldexpf(1.0f, -L);
    for (int i = 0; i < 3; ++i) p->x[i] = rng_u(r);
    isotropic_direction(r, p->d);
    return 1;
}

/* Move across the face on axis `a` (the package already sits on it).  Climb
 * while the neighbour lies outside the current octet, step into the sibling
 * or the neighbouring root cell, then descend to the leaf.  Returns 0 when
 * the package leaves the root grid. */
static int cross_face(const oracle_grid *G, pkg_t *p, int a)
{
    const int64_t n_root = n_root_of(G);
    const int up = p->d[a] > 0.0f;
    while ((int64_t)p->cell >= n_root) {
        int oct = (int)((p->cell - n_root) & 7);
        int b = (oct >> a) & 1;
        if (up && b == 0) { p->cell += 1 << a; p->x[a] = 0.0f; descend(G, p); return 1; }
        if (!up && b == 1) { p->cell -= 1 << a; p->x[a] = 1.0f; descend(G, p); return 1; }
        for (int i = 0; i < 3; ++i) p->x[i] = (p->x[i] + (float)((oct >> i) & 1)) * 0.5f;
        p->h = p->h * 2.0f;
        p->cell = G->parent[(p->cell - n_root) >> 3];
    }
    int idx[3];
    idx[0] = (int)(p->cell % G->nx);
    idx[1] = (int)((p->cell / G->nx) % G->ny);
    idx[2] = (int)(p->cell / ((int64_t)G->nx * G->ny));
    const int nr[3] = { G->nx, G->ny, G->nz };
    idx[a] += up ? 1 : -1;
    if (idx[a] < 0 || idx[a] >= nr[a]) return 0;
    p->cell = idx[0] + G->nx * (idx[1] + G->ny * idx[2]);
    p->x[a] = up ? 0.0f : 1.0f;
    descend(G, p);
    return 1;
}

/* Follow one emitted package to its end.  Per photon-cell step (one segment
 * inside one leaf cell):
 *   s      = min over axes with d_i != 0 of (face_i - x_i) * (1/d_i), ties to
 *            the lowest axis (x, y, z);
 *   ksh    = (rho * ksca) * h,  dtau = ksh * s;
 *   if ksh > 0 and dtau >= tau_f: the package scatters inside the cell after
 *            s' = min(tau_f / ksh, s), else s' = s;
 *   q      = 1 - exp(-((rho * kabs) * h) * s'),
 *            dep = min(W, rint(float(W) * q)), W -= dep (exact in integers);
 *   W < max(W0 / 2^20, 1) (W0 = initial weight; 2^11 for a full package)
 *            ends the package with W deposited in the cell;
 *   a scattering moves x by d s', draws a new HG direction and a new tau_f;
 *   a face crossing subtracts dtau from tau_f, flushes the cell's merged
 *            deposits, places x exactly on the face and finds the neighbour.
 * Deposits made in one cell between two crossings are merged before they are
 * added to tally[cell]. */
static uint32_t propagate(const oracle_grid *G, const oracle_item *it, rng_t *r, pkg_t *pp,
                          int64_t *tally, int64_t *self_tally, oracle_stats *st)
{
    pkg_t p = *pp;
    /* a dust package is "at home" until it first leaves its emission cell;
       deposits made at home are also added to self_tally (the local
       re-absorption used by the accelerated temperature update) */
    int home = (it->source == SRC_DUST) && self_tally != 0;
    st->emitted += (int64_t)p.W;
    /* packages end once attenuated below 2^-20 of their initial weight */
    const uint64_t w_min = (p.W >> 20) > 0 ? (p.W >> 20) : 1;
    set_inverse(&p);
    float tauf = -oracle_log(rng_u(r));
    uint64_t pend = 0;
    uint32_t steps = 0;
    for (;;) {
        if (steps >= it->max_steps) {          /* safety cap: end here, keep energy */
            pend += p.W; p.W = 0; st->capped++;
            break;
        }
        ++steps;
        const float rho = G->rho[p.cell];
        float s = INFINITY;
        int axis = -1;
        for (int i = 0; i < 3; ++i) {
            if (p.d[i] != 0.0f) {
                float face = (p.d[i] > 0.0f) ? 1.0f : 0.0f;
                float si = (face - p.x[i]) * p.inv[i];
                if (si < s) { s = si; axis = i; }
            }
        }
        if (axis < 0) {                        /* no finite exit face: end here */
            pend += p.W; p.W = 0; st->capped++;
            break;
        }
        const float ksh = (rho * it->ksca) * p.h;
        const float dtau = ksh * s;
        float sp = s;
        int scatter = 0;
        if (ksh > 0.0f && dtau >= tauf) {
            sp = tauf / ksh;
            if (sp > s) sp = s;
            scatter = 1;
        }
        const float tau_abs = ((rho * it->kabs) * p.h) * sp;
        if (tau_abs > 0.0f) {
            float q = oracle_one_minus_exp(tau_abs);
            uint64_t dep = (uint64_t)rintf((float)p.W * q);
            if (dep > p.W) dep = p.W;
            p.W -= dep;
            pend += dep;
        }
        if (p.W < w_min) { pend += p.W; p.W = 0; break; }
        if (scatter) {
            for (int i = 0; i < 3; ++i) p.x[i] = clamp01(p.x[i] + p.d[i] * sp);
            hg_scatter(r, it->g, p.d);
            set_inverse(&p);
            tauf = -oracle_log(rng_u(r));
            continue;
        }
        tauf = tauf - dtau;
        if (pend) {
            tally[p.cell] += (int64_t)pend;
            if (home) self_tally[p.cell] += (int64_t)pend;
            pend = 0;
        }
        home = 0;
        for (int i = 0; i < 3; ++i)
            p.x[i] = (i == axis) ? ((p.d[i] > 0.0f) ? 1.0f : 0.0f) : clamp01(p.x[i] + p.d[i] * s);
        if (!cross_face(G, &p, axis)) {
            st->escaped += (int64_t)p.W;
            p.W = 0;
            break;
        }
    }
    if (pend) {
        tally[p.cell] += (int64_t)pend;
        if (home) self_tally[p.cell] += (int64_t)pend;
    }
    st->steps += steps;
    *pp = p;
    return steps;
}

/* Emit and trace package pid of an item; returns its step count. */
static uint32_t trace_one(const oracle_grid *G, const oracle_item *it, uint32_t pid,
                          int64_t *tally, int64_t *self_tally, oracle_stats *st)
{
    rng_t r;
    rng_init(&r, it->seed, (uint32_t)it->iteration, (uint32_t)it->freq, pid,
             (uint32_t)it->cloud, (uint32_t)it->source);
    pkg_t p;
    if (!emit(G, it, &r, pid, &p)) return 0;
    return propagate(G, it, &r, &p, tally, self_tally, st);
}

/* Trace packages pid_lo .. pid_hi-1 of one item.  tally[] (n_cells, int64)
 * and *st are accumulated into; pkg_steps (nullable) receives each package's
 * step count at index pid - pid_lo; self_tally (nullable, n_cells) receives
 * the deposits dust packages make in their emission cell before they first
 * leave it. */
void oracle_trace(const oracle_grid *G, const oracle_item *it, uint32_t pid_lo, uint32_t pid_hi,
                  int64_t *tally, oracle_stats *st, uint32_t *pkg_steps, int64_t *self_tally)
{
    for (uint32_t pid = pid_lo; pid < pid_hi; ++pid) {
        uint32_t n = trace_one(G, it, pid, tally, self_tally, st);
        if (pkg_steps) pkg_steps[pid - pid_lo] = n;
    }
}

/* Elementwise wrappers used by the tests that pin the elementary functions. */
void oracle_one_minus_exp_v(const float *x, float *y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = oracle_one_minus_exp(x[i]); }
void oracle_log_v(const float *x, float *y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = oracle_log(x[i]); }

/* Draw n HG scatterings of direction d0 with asymmetry g from the stream of
 * (seed, pid); returns the cosines between successive directions in cosv and
 * the new directions in dout[3n].  Used by the phase-function pins. */
void oracle_hg_samples(float g, const float d0[3], uint64_t seed, int64_t n, float *cosv, float *dout)
{
    for (int64_t i = 0; i < n; ++i) {
        rng_t r;
        rng_init(&r, seed, 0, 0, (uint32_t)i, 0, 7);
        float d[3] = { d0[0], d0[1], d0[2] };
        hg_scatter(&r, g, d);
        cosv[i] = d[0] * d0[0] + d[1] * d0[1] + d[2] * d0[2];
        dout[3 * i] = d[0]; dout[3 * i + 1] = d[1]; dout[3 * i + 2] = d[2];
    }
}

/* Pencil beam (test pin only): one package started at root-unit position pos
 * with direction dir and weight it->w0, then traced like any other package.
 * Draws come from the stream of package pid.  Returns its step count. */
uint32_t oracle_trace_pencil(const oracle_grid *G, const oracle_item *it, const float pos[3],
                             const float dir[3], uint32_t pid, int64_t *tally, oracle_stats *st)
{
    const int nr[3] = { G->nx, G->ny, G->nz };
    int idx[3];
    pkg_t p;
    p.h = 1.0f;
    for (int i = 0; i < 3; ++i) {
        idx[i] = root_index(pos[i], nr[i], &p.x[i]);
        p.d[i] = dir[i];
    }
    p.W = it->w0;
    p.cell = idx[0] + G->nx * (idx[1] + G->ny * idx[2]);
    descend(G, &p);
    rng_t r;
    rng_init(&r, it->seed, (uint32_t)it->iteration, (uint32_t)it->freq, pid,
             (uint32_t)it->cloud, (uint32_t)it->source);
    return propagate(G, it, &r, &p, tally, 0, st);
}
