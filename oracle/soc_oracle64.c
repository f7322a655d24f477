/*
 * soc_oracle64.c -- FP64 Monte Carlo oracle for the photon-package tracer of
 * SOC (Juvela 2019, arXiv:1812.06632).
 *
 * TEST INFRASTRUCTURE ONLY, like soc_oracle.c (the FP32-contract oracle it is
 * compiled with): only tests/ and bench.py's CPU legs may use it.  It shares
 * no code with the CUDA library.
 *
 * It runs the same method as soc_oracle.c -- emission (Sect. 2.2 background
 * and point sources, Sect. 3.2 dust), cell-to-cell stepping through the
 * level-ordered octree with climbs to the common ancestor and descents to the
 * entered leaf (Sect. 2.1.1), free paths in scattering optical depth,
 * Henyey-Greenstein scattering, absorption as continuous attenuation of the
 * package weight -- and consumes the same random numbers in the same order,
 * but in double precision throughout: positions, directions and optical
 * depths are doubles, exp and log are libm's, and the weight is a real
 * number (in the same units as the FP32 oracle's integer weight, 2^31 per
 * full package) that loses W (1 - e^-tau) per segment.  Counters are doubles.
 *
 * Its purpose: state how far the FP32 contract's results (the GPU's, bit for
 * bit) are from the same Monte Carlo done in FP64.  Where a rounding flips a
 * decision (which face is nearer, whether the package scatters in this
 * cell, whether a disk sample is accepted) the two runs of a package part
 * ways; everywhere else they differ by rounding only.
 *
 * The grid and item structures below have the layout of soc_oracle.c's (the
 * Python side passes the same ctypes structures to both).
 */
#include <stdint.h>
#include <math.h>

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);
float oracle_u01(uint32_t x);

typedef struct {
    int32_t nx, ny, nz;
    int32_t n_levels;
    int64_t n_cells;
    const int64_t *level_start;
    const float *rho;
    const int32_t *child;
    const int32_t *parent;
} grid64;

typedef struct {
    int32_t source;
    int32_t freq;
    int32_t iteration;
    int32_t cloud;
    uint64_t seed;
    float kabs, ksca, g;
    uint64_t w0;
    uint32_t max_steps;
    int32_t n_ps;
    const float *ps_pos;
    const float *ps_cdf;
    uint32_t n_per_cell;
    int64_t n_leaf;
    const int32_t *leaf;
    const uint64_t *dust_w;
    const uint64_t *dust_prefix;
} item64;

typedef struct {
    double escaped;              /* weight leaving the root grid                    */
    int64_t capped;
    int64_t steps;
    double emitted;
} stats64;

enum { BG = 0, PS = 1, DUST = 2 };

/* The package's stream of uniform draws: Philox4x32-10 with key
 * (seed_lo, seed_hi ^ iteration<<16 ^ freq) and counter (package id, block,
 * cloud, source class); draw n is word n%4 of block n/4, mapped to (0,1). */
typedef struct {
    uint32_t key[2], ctr[4], buf[4];
    uint32_t n;
} stream64;

static void stream_init(stream64 *s, const item64 *it, uint32_t pid)
{
    s->key[0] = (uint32_t)it->seed;
    s->key[1] = (uint32_t)(it->seed >> 32) ^ ((uint32_t)it->iteration << 16) ^ (uint32_t)it->freq;
    s->ctr[0] = pid; s->ctr[1] = 0; s->ctr[2] = (uint32_t)it->cloud; s->ctr[3] = (uint32_t)it->source;
    s->n = 0;
}

static double draw(stream64 *s)
{
    if (s->n % 4 == 0) {
        s->ctr[1] = s->n / 4;
        oracle_philox4x32_10(s->ctr, s->key, s->buf);
    }
    return (double)oracle_u01(s->buf[s->n++ % 4]);
}

typedef struct {
    int64_t cell;
    double h, x[3], d[3], W;
} pkg64;

static double clamp_unit(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

static void to_leaf(const grid64 *G, pkg64 *p)
{
    while (G->child[p->cell] >= 0) {
        int oct = 0;
        for (int i = 0; i < 3; ++i) {
            int b = 2.0 * p->x[i] >= 1.0;
            p->x[i] = 2.0 * p->x[i] - b;
            oct |= b << i;
        }
        p->h *= 0.5;
        p->cell = G->child[p->cell] + oct;
    }
}

/* (cos phi, sin phi) of a point drawn uniformly in the unit disk (at most 64
 * tries, then phi = 0). */
static void azimuth(stream64 *s, double *c, double *sn)
{
    double a = 1.0, b = 0.0, r2 = 1.0;
    for (int k = 0; k < 64; ++k) {
        double ta = 2.0 * draw(s) - 1.0, tb = 2.0 * draw(s) - 1.0;
        double t2 = ta * ta + tb * tb;
        if (t2 <= 1.0 && t2 > 0.0) { a = ta; b = tb; r2 = t2; break; }
    }
    *c = a / sqrt(r2);
    *sn = b / sqrt(r2);
}

static void isotropic(stream64 *s, double d[3])
{
    double mu = 2.0 * draw(s) - 1.0, c, sn;
    azimuth(s, &c, &sn);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    d[0] = st * c; d[1] = st * sn; d[2] = mu;
}

/* Henyey-Greenstein: cos theta from the inverse of its cumulative
 * distribution (uniform for |g| < 1e-4), azimuth from the disk sample, and
 * the new direction rotated from the old one. */
static void scatter_hg(stream64 *s, double g, double d[3])
{
    double u = draw(s), mu;
    if (fabs(g) < 1e-4) {
        mu = 2.0 * u - 1.0;
    } else {
        double q = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
        mu = fmin(1.0, fmax(-1.0, (1.0 + g * g - q * q) / (2.0 * g)));
    }
    double c, sn;
    azimuth(s, &c, &sn);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double n[3];
    if (fabs(d[2]) > 0.99999) {
        n[0] = st * c; n[1] = st * sn; n[2] = d[2] > 0.0 ? mu : -mu;
    } else {
        double t = sqrt(1.0 - d[2] * d[2]);
        n[0] = st * (d[0] * d[2] * c - d[1] * sn) / t + d[0] * mu;
        n[1] = st * (d[1] * d[2] * c + d[0] * sn) / t + d[1] * mu;
        n[2] = d[2] * mu - st * c * t;
    }
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int i = 0; i < 3; ++i) d[i] = n[i] / nn;
}

static int root_cell_of(double v, int n, double *local)
{
    int i = (int)v;
    if (i < 0) i = 0;
    if (i > n - 1) i = n - 1;
    *local = clamp_unit(v - i);
    return i;
}

static int emit64(const grid64 *G, const item64 *it, stream64 *s, uint32_t pid, pkg64 *p)
{
    const int nr[3] = { G->nx, G->ny, G->nz };
    int idx[3] = { 0, 0, 0 };
    p->h = 1.0;
    if (it->source == BG) {
        /* a face with probability proportional to its area (-x,+x,-y,+y,-z,+z),
         * a uniform point on it, a cosine-weighted inward direction */
        double area[3] = { (double)nr[1] * nr[2], (double)nr[0] * nr[2], (double)nr[0] * nr[1] };
        double t = draw(s) * 2.0 * (area[0] + area[1] + area[2]), cum = 0.0;
        int f = 0;
        for (; f < 5; ++f) {
            cum += area[f >> 1];
            if (t < cum) break;
        }
        int a = f >> 1, low = (f & 1) == 0;
        int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
        idx[t1] = root_cell_of(draw(s) * nr[t1], nr[t1], &p->x[t1]);
        idx[t2] = root_cell_of(draw(s) * nr[t2], nr[t2], &p->x[t2]);
        idx[a] = low ? 0 : nr[a] - 1;
        p->x[a] = low ? 0.0 : 1.0;
        double u = draw(s), c, sn;
        azimuth(s, &c, &sn);
        p->d[a] = low ? sqrt(u) : -sqrt(u);
        p->d[t1] = sqrt(1.0 - u) * c;
        p->d[t2] = sqrt(1.0 - u) * sn;
        p->W = (double)it->w0;
    } else if (it->source == PS) {
        double t = draw(s);
        int k = 0;
        while (k < it->n_ps - 1 && !(t < it->ps_cdf[k])) ++k;
        for (int i = 0; i < 3; ++i) idx[i] = root_cell_of(it->ps_pos[3 * k + i], nr[i], &p->x[i]);
        isotropic(s, p->d);
        p->W = (double)it->w0;
    } else {
        int64_t li;
        if (it->dust_prefix) {
            int64_t lo = 0, hi = it->n_leaf;
            while (hi - lo > 1) {
                int64_t mid = (lo + hi) / 2;
                if (it->dust_prefix[mid] <= (uint64_t)pid) lo = mid; else hi = mid;
            }
            li = lo;
        } else {
            li = pid / it->n_per_cell;
        }
        p->cell = it->leaf[li];
        if (it->dust_w[li] == 0) return 0;
        p->W = (double)it->dust_w[li];
        int L = 0;
        while (L + 1 < G->n_levels && p->cell >= G->level_start[L + 1]) ++L;
        p->h = ldexp(1.0, -L);
        for (int i = 0; i < 3; ++i) p->x[i] = draw(s);
        isotropic(s, p->d);
        return 1;
    }
    p->cell = idx[0] + (int64_t)G->nx * (idx[1] + (int64_t)G->ny * idx[2]);
    to_leaf(G, p);
    return 1;
}

/* Into the neighbour across the face on axis a: up to the first ancestor
 * whose octet holds the neighbour (or the root grid), across, down to the
 * leaf.  0 when the package leaves the root grid. */
static int next_cell(const grid64 *G, pkg64 *p, int a)
{
    const int64_t n_root = (int64_t)G->nx * G->ny * G->nz;
    const int up = p->d[a] > 0.0;
    while (p->cell >= n_root) {
        int oct = (int)((p->cell - n_root) % 8);
        int side = (oct >> a) & 1;
        if (up != side) {                      /* the neighbour is a sibling */
            p->cell += up ? (1 << a) : -(1 << a);
            p->x[a] = up ? 0.0 : 1.0;
            to_leaf(G, p);
            return 1;
        }
        for (int i = 0; i < 3; ++i) p->x[i] = 0.5 * (p->x[i] + ((oct >> i) & 1));
        p->h *= 2.0;
        p->cell = G->parent[(p->cell - n_root) / 8];
    }
    int64_t i = p->cell % G->nx, j = (p->cell / G->nx) % G->ny, k = p->cell / ((int64_t)G->nx * G->ny);
    int64_t ijk[3] = { i, j, k };
    const int nr[3] = { G->nx, G->ny, G->nz };
    ijk[a] += up ? 1 : -1;
    if (ijk[a] < 0 || ijk[a] >= nr[a]) return 0;
    p->cell = ijk[0] + (int64_t)G->nx * (ijk[1] + (int64_t)G->ny * ijk[2]);
    p->x[a] = up ? 0.0 : 1.0;
    to_leaf(G, p);
    return 1;
}

static uint32_t follow(const grid64 *G, const item64 *it, stream64 *s, pkg64 *p, double *tally, stats64 *st)
{
    st->emitted += p->W;
    const double w_min = fmax(floor(p->W / 1048576.0), 1.0);   /* 2^-20 of the start */
    double tauf = -log(draw(s));
    uint32_t steps = 0;
    for (;;) {
        if (steps >= it->max_steps) { tally[p->cell] += p->W; st->capped++; break; }
        ++steps;
        double s_exit = INFINITY;
        int axis = -1;
        for (int i = 0; i < 3; ++i) {
            if (p->d[i] == 0.0) continue;
            double si = ((p->d[i] > 0.0 ? 1.0 : 0.0) - p->x[i]) / p->d[i];
            if (si < s_exit) { s_exit = si; axis = i; }
        }
        if (axis < 0) { tally[p->cell] += p->W; st->capped++; break; }
        const double rho = G->rho[p->cell];
        const double ksh = rho * it->ksca * p->h;
        double seg = s_exit;
        int scat = 0;
        if (ksh > 0.0 && ksh * s_exit >= tauf) {
            seg = fmin(tauf / ksh, s_exit);
            scat = 1;
        }
        const double dep = p->W * -expm1(-rho * it->kabs * p->h * seg);
        p->W -= dep;
        tally[p->cell] += dep;
        if (p->W < w_min) { tally[p->cell] += p->W; break; }
        if (scat) {
            for (int i = 0; i < 3; ++i) p->x[i] = clamp_unit(p->x[i] + p->d[i] * seg);
            scatter_hg(s, it->g, p->d);
            tauf = -log(draw(s));
            continue;
        }
        tauf -= ksh * s_exit;
        for (int i = 0; i < 3; ++i)
            p->x[i] = i == axis ? (p->d[i] > 0.0 ? 1.0 : 0.0) : clamp_unit(p->x[i] + p->d[i] * s_exit);
        if (!next_cell(G, p, axis)) { st->escaped += p->W; break; }
    }
    st->steps += steps;
    return steps;
}

/* Trace packages pid_lo .. pid_hi-1 of one item in FP64; tally (doubles,
 * n_cells) and *st are accumulated into; pkg_steps (nullable) receives each
 * package's step count. */
void oracle64_trace(const grid64 *G, const item64 *it, uint32_t pid_lo, uint32_t pid_hi, double *tally,
                    stats64 *st, uint32_t *pkg_steps)
{
    for (uint32_t pid = pid_lo; pid < pid_hi; ++pid) {
        stream64 s;
        stream_init(&s, it, pid);
        pkg64 p;
        uint32_t n = emit64(G, it, &s, pid, &p) ? follow(G, it, &s, &p, tally, st) : 0;
        if (pkg_steps) pkg_steps[pid - pid_lo] = n;
    }
}
