// soc_trace.cu -- persistent photon-package tracer (paper Sect. 2.1.1: package
// creation, cell-to-cell stepping through the hierarchical grid with partial
// traversal up to the common ancestor and down to the new leaf, per-cell
// absorption counters; Sect. 2.2 sources; Sect. 3.2 uniform dust emission).
//
// Scheduling: one package per lane.  A warp takes chunk*32 consecutive work
// indices at a time from a global counter; lanes whose packages ended take
// the next indices of the warp's chunk once refill_min of them are idle
// (per-lane refill in batches, the interleaving of creation and tracking
// suggested in Sect. 4.2).  Each pass of the warp's loop then runs, for the
// lanes waiting on them, the scattering phase and (octrees) the descent
// phase, and steps the other lanes: two steps on regular grids, one on
// octrees.  One launch covers every (cloud, frequency, source) item of a
// batch.
//
// Arithmetic: the FP32 sequence of soc_fp32.cuh; deposits are fixed point
// (2^31 units per package, so a package's weight and its pending deposits
// fit 32-bit registers) and are merged per cell before one 64-bit
// atomic add, so the counters are exact and independent of scheduling.
// A host-set abort flag, read when a warp takes a new chunk of work, stops the
// launch early (paper-independent failure handling: a watchdog's deadline).
// Compiled with -fmad=false.
#include <cuda_runtime.h>
#include <cstdint>
#include "soc_internal.h"
#include "soc_fp32.cuh"

namespace soc {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// One package's random stream: key (seed, iteration, frequency), counter
// (package id, block, cloud, source class); draw n = word n%4 of block n/4.
struct Rng {
    uint32_t k0, k1, pid, cloud, cls, n;
    uint32_t b0, b1, b2, b3;

    __device__ __forceinline__ void init(uint64_t seed, uint32_t iteration, uint32_t freq,
                                         uint32_t pid_, uint32_t cloud_, uint32_t cls_)
    {
        k0 = (uint32_t)seed;
        k1 = (uint32_t)(seed >> 32) ^ (iteration << 16) ^ freq;
        pid = pid_; cloud = cloud_; cls = cls_; n = 0;
    }
    __device__ __forceinline__ uint32_t next()
    {
        const uint32_t j = n & 3u;
        if (j == 0) {
            const U4 v = philox10(pid, n >> 2, cloud, cls, k0, k1);
            b0 = v.a; b1 = v.b; b2 = v.c; b3 = v.d;
        }
        ++n;
        return j == 0 ? b0 : (j == 1 ? b1 : (j == 2 ? b2 : b3));
    }
    __device__ __forceinline__ float u() { return u01(next()); }
};

struct Pkg {
    int32_t cell;                 // current leaf
    int32_t ri, rj, rk;           // root-grid coordinates of its root ancestor
    float h;                      // cell side in root-cell units
    float x, y, z;                // position in [0,1]^3 of the cell
    float dx, dy, dz;             // direction
    float ix, iy, iz;             // 1/d (unused where d == 0)
    float rho;                    // density of the current leaf
    float tauf;                   // remaining scattering optical depth
    uint32_t W;                   // weight (fixed point, <= 2^31)
    uint32_t pend;                // deposits in the current cell not yet added (<= W0)
    uint32_t wf;                  // bits 0..12: weight floor max(W0 / 2^20, 1) (<= 2^11);
                                  // kHomeBit: dust package still in its emission cell
    uint32_t steps;
    bool scat;                    // waiting for its scattering (new direction, new free path)
};

constexpr uint32_t kFloorMask = 0x1fffu;
constexpr uint32_t kHomeBit = 1u << 31;

// 1/d per axis; +inf for a zero component (either sign of zero).  With the
// face taken as 1 for d >= 0, such an axis gives (1 - x) * inf = +inf or
// NaN, which never wins the strict comparison for the nearest face: the same
// choice as skipping the axis, without a test per axis and step.
__device__ __forceinline__ void set_inverse(Pkg &p)
{
    const float inf = __int_as_float(0x7f800000);
    p.ix = (p.dx != 0.0f) ? __fdiv_rn(1.0f, p.dx) : inf;
    p.iy = (p.dy != 0.0f) ? __fdiv_rn(1.0f, p.dy) : inf;
    p.iz = (p.dz != 0.0f) ? __fdiv_rn(1.0f, p.dz) : inf;
}

// The fields of a cloud that every step reads.  When every item of a launch
// uses one cloud they travel in the kernel parameters (TraceParams::hot), so
// the compiler takes them as constant operands; otherwise each lane reads
// them through its own DevCloud pointer (GlobalCloud).
struct ParamCloud {
    const HotCloud &h;
    __device__ const uint32_t *cell() const { return h.cell; }
    __device__ const int32_t *parent() const { return h.parent; }
    __device__ int32_t nx() const { return h.nx; }
    __device__ int32_t ny() const { return h.ny; }
    __device__ int32_t nz() const { return h.nz; }
    __device__ int32_t n_root() const { return h.n_root; }
};

struct GlobalCloud {
    const DevCloud &C;
    __device__ const uint32_t *cell() const { return C.cell; }
    __device__ const int32_t *parent() const { return C.parent; }
    __device__ int32_t nx() const { return C.nx; }
    __device__ int32_t ny() const { return C.ny; }
    __device__ int32_t nz() const { return C.nz; }
    __device__ int32_t n_root() const { return (int32_t)C.n_root; }
};

// The ancestors of a lane's current cell (entry L: the index of the
// ancestor at level L), in dynamic shared memory, kAncRows words per thread
// (an odd count, so lanes reading the same level hit distinct banks): an
// octree climb reads its parent from here (tens of cycles) rather than
// following the parent link in global memory (an L2 round trip that the next
// step waits on).  Levels 0 .. SOC_MAX_LEVELS-2 are enough, since only cells
// above the deepest level have children.
constexpr int kAncRows = SOC_MAX_LEVELS - 1;
// lanes that wait for a descent before the warp runs the descent phase
constexpr int kDescendMin = 4;

// Level of a cell from its side h = 2^-L (h only ever halves or doubles).
__device__ __forceinline__ int level_of(float h)
{
    return 127 - (int)(__float_as_uint(h) >> 23);
}

// Follow child links to the leaf that contains the position; the upper child
// is taken on an axis when 2x >= 1.  kStack: push every cell left on the way
// down onto the lane's ancestor rows.
template <bool kStack = false>
__device__ __forceinline__ void descend(const uint32_t *__restrict__ cells, Pkg &p, int32_t *anc = nullptr)
{
    uint32_t w = __ldg(cells + p.cell);
    int L = kStack ? level_of(p.h) : 0;
    while (w & kLinkBit) {
        if (kStack) anc[L++] = p.cell;
        const float x2 = __fmul_rn(2.0f, p.x), y2 = __fmul_rn(2.0f, p.y), z2 = __fmul_rn(2.0f, p.z);
        const int bx = x2 >= 1.0f, by = y2 >= 1.0f, bz = z2 >= 1.0f;
        p.x = __fsub_rn(x2, (float)bx);
        p.y = __fsub_rn(y2, (float)by);
        p.z = __fsub_rn(z2, (float)bz);
        p.h = __fmul_rn(p.h, 0.5f);
        p.cell = (int32_t)(w & ~kLinkBit) + (bx | (by << 1) | (bz << 2));
        w = __ldg(cells + p.cell);
    }
    p.rho = __uint_as_float(w);
}

// (cos phi, sin phi) from a point drawn uniformly in the unit disk.  After 64
// rejections (probability < 1e-42) the azimuth 0 is used, so the loop is bounded.
__device__ __forceinline__ void disk(Rng &r, float &c, float &s)
{
    float a = 1.0f, b = 0.0f, r2 = 1.0f;
    for (int tries = 0; tries < 64; ++tries) {
        const float ta = __fsub_rn(__fmul_rn(2.0f, r.u()), 1.0f);
        const float tb = __fsub_rn(__fmul_rn(2.0f, r.u()), 1.0f);
        const float t2 = __fadd_rn(__fmul_rn(ta, ta), __fmul_rn(tb, tb));
        if (t2 <= 1.0f && t2 > 0.0f) { a = ta; b = tb; r2 = t2; break; }
    }
    const float rr = __fsqrt_rn(r2);
    c = __fdiv_rn(a, rr);
    s = __fdiv_rn(b, rr);
}

__device__ __forceinline__ void isotropic(Rng &r, Pkg &p)
{
    const float mu = __fsub_rn(__fmul_rn(2.0f, r.u()), 1.0f);
    float c, s;
    disk(r, c, s);
    const float st = __fsqrt_rn(fmaxf(0.0f, __fsub_rn(1.0f, __fmul_rn(mu, mu))));
    p.dx = __fmul_rn(st, c);
    p.dy = __fmul_rn(st, s);
    p.dz = mu;
}

// Henyey-Greenstein deflection of the direction by the angle with
// cos = (1 + g^2 - ((1 - g^2)/(1 - g + 2 g u))^2) / (2 g); rotation about the
// old direction by the azimuth from the disk sampler; renormalised.
__device__ __forceinline__ void hg_scatter(Rng &r, float g, Pkg &p)
{
    const float u = r.u();
    float mu;
    if (fabsf(g) < 1e-4f) {
        mu = __fsub_rn(__fmul_rn(2.0f, u), 1.0f);
    } else {
        const float g2 = __fmul_rn(g, g);
        const float den = __fadd_rn(__fsub_rn(1.0f, g), __fmul_rn(__fadd_rn(g, g), u));
        const float tmp = __fdiv_rn(__fsub_rn(1.0f, g2), den);
        mu = __fdiv_rn(__fsub_rn(__fadd_rn(1.0f, g2), __fmul_rn(tmp, tmp)), __fadd_rn(g, g));
        mu = fminf(fmaxf(mu, -1.0f), 1.0f);
    }
    float c, s;
    disk(r, c, s);
    const float st = __fsqrt_rn(fmaxf(0.0f, __fsub_rn(1.0f, __fmul_rn(mu, mu))));
    const float dx = p.dx, dy = p.dy, dz = p.dz;
    float nx, ny, nz;
    if (fabsf(dz) > 0.99999f) {
        nx = __fmul_rn(st, c);
        ny = __fmul_rn(st, s);
        nz = (dz > 0.0f) ? mu : -mu;
    } else {
        const float t = __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(dz, dz)));
        const float ax = __fsub_rn(__fmul_rn(__fmul_rn(dx, dz), c), __fmul_rn(dy, s));
        const float ay = __fadd_rn(__fmul_rn(__fmul_rn(dy, dz), c), __fmul_rn(dx, s));
        nx = __fadd_rn(__fdiv_rn(__fmul_rn(st, ax), t), __fmul_rn(dx, mu));
        ny = __fadd_rn(__fdiv_rn(__fmul_rn(st, ay), t), __fmul_rn(dy, mu));
        nz = __fsub_rn(__fmul_rn(dz, mu), __fmul_rn(__fmul_rn(st, c), t));
    }
    const float nrm = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(nx, nx), __fmul_rn(ny, ny)),
                                           __fmul_rn(nz, nz)));
    p.dx = __fdiv_rn(nx, nrm);
    p.dy = __fdiv_rn(ny, nrm);
    p.dz = __fdiv_rn(nz, nrm);
}

// Root cell index along an axis of n cells for root-unit coordinate v, and
// the local coordinate v - i.
__device__ __forceinline__ int root_axis(float v, int n, float &local)
{
    int i = __float2int_rz(v);
    i = max(0, min(i, n - 1));
    local = clamp01(__fsub_rn(v, __int2float_rn(i)));
    return i;
}

__device__ __forceinline__ int32_t root_cell(const DevCloud &C, int i, int j, int k)
{
    return i + C.nx * (j + C.ny * k);
}

// Emission (Sect. 2.2 background and point sources, Sect. 3.2 dust).  Returns
// false for a dust package of zero weight (nothing to trace).  kStack: also
// fill the lane's ancestor rows for the cell it starts in.
template <bool kStack>
__device__ bool emit(const DevCloud &C, const DevItem &it, uint32_t pid, Rng &r, Pkg &p, int32_t *anc)
{
    p.h = 1.0f;
    if (it.source == SOC_SRC_BACKGROUND) {
        const float fx = __int2float_rn(C.nx), fy = __int2float_rn(C.ny), fz = __int2float_rn(C.nz);
        const float ax = __fmul_rn(fy, fz), ay = __fmul_rn(fx, fz), az = __fmul_rn(fx, fy);
        const float c0 = ax, c1 = __fadd_rn(c0, ax), c2 = __fadd_rn(c1, ay);
        const float c3 = __fadd_rn(c2, ay), c4 = __fadd_rn(c3, az), c5 = __fadd_rn(c4, az);
        const float t = __fmul_rn(r.u(), c5);
        const int f = (t < c0) ? 0 : (t < c1) ? 1 : (t < c2) ? 2 : (t < c3) ? 3 : (t < c4) ? 4 : 5;
        const int a = f >> 1;
        const bool low = (f & 1) == 0;
        // tangential axes t1 < t2
        const int n1 = (a == 0) ? C.ny : C.nx;
        const int n2 = (a == 2) ? C.ny : C.nz;
        const int na = (a == 0) ? C.nx : (a == 1) ? C.ny : C.nz;
        float l1, l2;
        const int i1 = root_axis(__fmul_rn(r.u(), __int2float_rn(n1)), n1, l1);
        const int i2 = root_axis(__fmul_rn(r.u(), __int2float_rn(n2)), n2, l2);
        const int ia = low ? 0 : na - 1;
        const float la = low ? 0.0f : 1.0f;
        const float u = r.u();
        const float mu = __fsqrt_rn(u);                 // cosine-weighted inward
        const float st = __fsqrt_rn(__fsub_rn(1.0f, u));
        float c, s;
        disk(r, c, s);
        const float da = low ? mu : -mu, d1 = __fmul_rn(st, c), d2 = __fmul_rn(st, s);
        p.x = (a == 0) ? la : l1;
        p.y = (a == 0) ? l1 : (a == 1) ? la : l2;
        p.z = (a == 2) ? la : l2;
        p.ri = (a == 0) ? ia : i1;
        p.rj = (a == 0) ? i1 : (a == 1) ? ia : i2;
        p.rk = (a == 2) ? ia : i2;
        p.dx = (a == 0) ? da : d1;
        p.dy = (a == 0) ? d1 : (a == 1) ? da : d2;
        p.dz = (a == 2) ? da : d2;
        p.W = (uint32_t)it.w0;
        p.cell = root_cell(C, p.ri, p.rj, p.rk);
        descend<kStack>(C.cell, p, anc);
        return true;
    }
    if (it.source == SOC_SRC_POINT) {
        const float t = r.u();
        const float *cdf = C.ps_cdf + (int64_t)it.freq * C.n_ps;
        int k = 0;
        while (k < C.n_ps - 1 && !(t < __ldg(cdf + k))) ++k;
        p.ri = root_axis(__ldg(C.ps_pos + 3 * k + 0), C.nx, p.x);
        p.rj = root_axis(__ldg(C.ps_pos + 3 * k + 1), C.ny, p.y);
        p.rk = root_axis(__ldg(C.ps_pos + 3 * k + 2), C.nz, p.z);
        isotropic(r, p);
        p.W = (uint32_t)it.w0;
        p.cell = root_cell(C, p.ri, p.rj, p.rk);
        descend<kStack>(C.cell, p, anc);
        return true;
    }
    // dust: n_per_cell packages from every leaf, or (weighted sampling) the
    // leaf whose package-id range [prefix[li], prefix[li+1]) holds pid;
    // uniform inside the cell
    int32_t li;
    if (it.flags & kItemWeighted) {
        const unsigned long long *pre = reinterpret_cast<const unsigned long long *>(it.dust_w) + C.n_leaf;
        int32_t lo = 0, hi = (int32_t)C.n_leaf;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (__ldg(pre + mid) <= (unsigned long long)pid) lo = mid; else hi = mid;
        }
        li = lo;
    } else {
        li = (int32_t)(pid / it.n_per_cell);
    }
    p.cell = __ldg(C.leaf + li);
    p.W = (uint32_t)__ldg(reinterpret_cast<const unsigned long long *>(it.dust_w) + li);
    if (p.W == 0) return false;
    int L = 0;
    while (L + 1 < C.n_levels && (int64_t)p.cell >= C.level_start[L + 1]) ++L;
    p.h = __uint_as_float((uint32_t)(127 - L) << 23);        // 2^-L
    int32_t a = p.cell;
    while ((int64_t)a >= C.n_root) {
        a = __ldg(C.parent + ((a - C.n_root) >> 3));
        if (kStack) anc[--L] = a;
    }
    const int32_t root = a;
    p.ri = root % C.nx;
    p.rj = (root / C.nx) % C.ny;
    p.rk = root / (C.nx * C.ny);
    p.rho = __uint_as_float(__ldg(C.cell + p.cell));
    p.x = r.u();
    p.y = r.u();
    p.z = r.u();
    isotropic(r, p);
    return true;
}

// Entered cell of an octree crossing in the tracer: a leaf gives its
// density; a refined cell leaves rho = -1, "descent pending", and the warp
// runs the descent in a phase of its own (trace_kernel) instead of here.
__device__ __forceinline__ void enter_cell(const uint32_t *__restrict__ cells, Pkg &p)
{
    const uint32_t w = __ldg(cells + p.cell);
    p.rho = (w & kLinkBit) ? -1.0f : __uint_as_float(w);
}

// Cross the face on axis `ax`: the package sits on it in the current frame.
// Returns false when it leaves the root grid.  kRegular: every cell is a
// root leaf (a one-level grid), so there is nothing to climb or descend.
// kStack (the tracer's octree builds): climbs pop the lane's ancestor rows,
// and the descent into a refined neighbour is left pending (enter_cell);
// otherwise (maps) the parent links are followed and the descent is done here.
template <bool kRegular = false, bool kStack = false, class CC>
__device__ bool cross_face(const CC &C, Pkg &p, int ax, bool up, int32_t *anc = nullptr)
{
    const int32_t n_root = C.n_root();
    int L = kStack ? level_of(p.h) : 0;
    while (!kRegular && p.cell >= n_root) {
        const int o = (p.cell - n_root) & 7;
        const int b = (o >> ax) & 1;
        if (up ? (b == 0) : (b == 1)) {
            p.cell += up ? (1 << ax) : -(1 << ax);
            const float v = up ? 0.0f : 1.0f;
            p.x = (ax == 0) ? v : p.x;
            p.y = (ax == 1) ? v : p.y;
            p.z = (ax == 2) ? v : p.z;
            if (kStack) enter_cell(C.cell(), p);
            else descend(C.cell(), p);
            return true;
        }
        p.x = __fmul_rn(__fadd_rn(p.x, (float)(o & 1)), 0.5f);
        p.y = __fmul_rn(__fadd_rn(p.y, (float)((o >> 1) & 1)), 0.5f);
        p.z = __fmul_rn(__fadd_rn(p.z, (float)((o >> 2) & 1)), 0.5f);
        p.h = __fmul_rn(p.h, 2.0f);
        p.cell = kStack ? anc[--L] : __ldg(C.parent() + ((p.cell - n_root) >> 3));
    }
    const int step = up ? 1 : -1;
    const int ri = p.ri + ((ax == 0) ? step : 0);
    const int rj = p.rj + ((ax == 1) ? step : 0);
    const int rk = p.rk + ((ax == 2) ? step : 0);
    // one unsigned compare per axis tests both ends of the root grid
    const int32_t nx = C.nx(), ny = C.ny();
    if ((unsigned)ri >= (unsigned)nx || (unsigned)rj >= (unsigned)ny || (unsigned)rk >= (unsigned)C.nz())
        return false;
    p.ri = ri; p.rj = rj; p.rk = rk;
    p.cell = ri + nx * (rj + ny * rk);
    if (!kRegular) {            // (regular grids: the step already put it there)
        const float v = up ? 0.0f : 1.0f;
        p.x = (ax == 0) ? v : p.x;
        p.y = (ax == 1) ? v : p.y;
        p.z = (ax == 2) ? v : p.z;
    }
    if (kRegular) p.rho = __uint_as_float(__ldg(C.cell() + p.cell));
    else if (kStack) enter_cell(C.cell(), p);
    else descend(C.cell(), p);
    return true;
}

enum StepResult { kContinue = 0, kAbsorbed = 1, kEscaped = 2, kCapped = 3 };

// float(W) with round-to-nearest (W <= 2^31).
__device__ __forceinline__ float w_to_float(uint32_t W)
{
    return __uint2float_rn(W);
}

// rint(v) as an integer for 0 <= v <= 2^31 (v = float(W) * q, q <= 1).
__device__ __forceinline__ uint32_t float_to_w(float v)
{
    return __float2uint_rn(v);
}

// One photon-cell step (one segment inside one leaf).
template <bool kSelf, bool kRegular, class CC>
__device__ __forceinline__ int step(const CC &C, Pkg &p, float kabs, float ksca,
                                    unsigned long long *tally, const TraceParams &P, int32_t *anc)
{
    if (p.steps >= P.max_steps) { p.pend += p.W; p.W = 0; return kCapped; }
    ++p.steps;
    float s = __int_as_float(0x7f800000);     // +inf
    int ax = -1;
    {   // axes with d = 0 carry 1/d = +inf (set_inverse) and never win
        const float si = __fmul_rn(__fsub_rn(p.dx < 0.0f ? 0.0f : 1.0f, p.x), p.ix);
        if (si < s) { s = si; ax = 0; }
    }
    {
        const float si = __fmul_rn(__fsub_rn(p.dy < 0.0f ? 0.0f : 1.0f, p.y), p.iy);
        if (si < s) { s = si; ax = 1; }
    }
    {
        const float si = __fmul_rn(__fsub_rn(p.dz < 0.0f ? 0.0f : 1.0f, p.z), p.iz);
        if (si < s) { s = si; ax = 2; }
    }
    if (ax < 0) { p.pend += p.W; p.W = 0; return kCapped; }     // no exit face: end safely
    // on regular grids h = 1 and the multiplications by h are exact: left out
    const float ksh = kRegular ? __fmul_rn(p.rho, ksca) : __fmul_rn(__fmul_rn(p.rho, ksca), p.h);
    const float dtau = __fmul_rn(ksh, s);
    float sp = s;
    bool scatter = false;
    if (ksh > 0.0f && dtau >= p.tauf) {
        sp = fminf(__fdiv_rn(p.tauf, ksh), s);
        scatter = true;
    }
    const float tau_abs = kRegular ? __fmul_rn(__fmul_rn(p.rho, kabs), sp)
                                   : __fmul_rn(__fmul_rn(__fmul_rn(p.rho, kabs), p.h), sp);
    if (tau_abs > 0.0f) {
        const float q = one_minus_exp(tau_abs);
        const float prod = __fmul_rn(w_to_float(p.W), q);
        uint32_t dep = float_to_w(prod);
        dep = dep > p.W ? p.W : dep;
        p.W -= dep;
        p.pend += dep;
    }
    if (p.W < (kSelf ? (p.wf & kFloorMask) : p.wf)) { p.pend += p.W; p.W = 0; return kAbsorbed; }
    if (scatter) {
        p.x = clamp01(__fadd_rn(p.x, __fmul_rn(p.dx, sp)));
        p.y = clamp01(__fadd_rn(p.y, __fmul_rn(p.dy, sp)));
        p.z = clamp01(__fadd_rn(p.z, __fmul_rn(p.dz, sp)));
        p.scat = true;            // the new direction is drawn in the warp's scattering phase
        return kContinue;
    }
    p.tauf = __fsub_rn(p.tauf, dtau);
    if (p.pend) {
        atomicAdd(tally + p.cell, (unsigned long long)p.pend);
        if (kSelf && (p.wf & kHomeBit))      // self counters: same offset as the item's counters
            atomicAdd(P.self + (tally - P.tally) + p.cell, (unsigned long long)p.pend);
        p.pend = 0;
    }
    if (kSelf) p.wf &= ~kHomeBit;            // it leaves the cell it was emitted in
    // move to the exit face: the exit coordinate exactly on the face, the
    // others advanced (selects, so lanes leaving through different faces
    // stay converged)
    const float da = (ax == 0) ? p.dx : (ax == 1) ? p.dy : p.dz;
    const bool up = da > 0.0f;
    // regular grids: the exit coordinate goes straight to the neighbour's
    // entry face (0 when moving up, 1 when moving down), which is where the
    // crossing puts it; octrees place it on the exit face first (a climb
    // rescales it)
    const float face = (up != kRegular) ? 1.0f : 0.0f;
    const float mx = clamp01(__fadd_rn(p.x, __fmul_rn(p.dx, s)));
    const float my = clamp01(__fadd_rn(p.y, __fmul_rn(p.dy, s)));
    const float mz = clamp01(__fadd_rn(p.z, __fmul_rn(p.dz, s)));
    p.x = (ax == 0) ? face : mx;
    p.y = (ax == 1) ? face : my;
    p.z = (ax == 2) ? face : mz;
    if (!cross_face<kRegular, !kRegular>(C, p, ax, up, anc)) return kEscaped;
    return kContinue;
}

__device__ __forceinline__ int find_item(const uint64_t *__restrict__ prefix, int n_items, uint64_t g)
{
    int lo = 0, hi = n_items;              // prefix[lo] <= g < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(reinterpret_cast<const unsigned long long *>(prefix) + mid) <= g) lo = mid; else hi = mid;
    }
    return lo;
}

template <int kMinBlocks, bool kSelf, bool kOneCloud, bool kRegular>
__global__ void __launch_bounds__(256, kMinBlocks) trace_kernel(const TraceParams P)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint64_t span = (uint64_t)P.chunk * 32u;
    // the warp's current chunk of work indices [q_next, q_end), kept in shared
    // memory (read only when lanes refill) to spare registers
    __shared__ unsigned long long s_q[8][2];
    unsigned long long *const q = s_q[threadIdx.x >> 5];
    if (lane == 0) { q[0] = 0; q[1] = 0; }
    __syncwarp();
    bool exhausted = false;

    Pkg p;
    Rng r;
    p.steps = 0; p.W = 0; p.pend = 0; p.wf = 0; p.scat = false;
    bool active = false;
    int item = -1;
    float kabs = 0.f, ksca = 0.f, g = 0.f;
    unsigned long long *tally = nullptr;
    uint64_t gidx = 0;
    // per-lane statistics, flushed when the lane moves to another item; the
    // sums live in shared memory (touched once per package) to spare registers
    __shared__ unsigned long long s_acc[256][3];     // escaped, steps, emitted
    unsigned long long *const acc = s_acc[threadIdx.x];
    acc[0] = acc[1] = acc[2] = 0;
    // octree launches: the lane's ancestors (regular-grid launches get no
    // dynamic shared memory and never touch them)
    extern __shared__ int32_t s_anc[];
    int32_t *const anc = s_anc + kAncRows * threadIdx.x;
    const DevCloud *C = P.clouds;             // the lane's cloud (used when !kOneCloud)
    int acc_item = -1;
    unsigned acc_cap = 0;

    for (;;) {
        unsigned idle = __ballot_sync(kFull, !active);
        // refill once at least refill_min lanes are idle (emission runs for
        // several lanes together), or when the whole warp is idle
        if (__popc(idle) < P.refill_min && idle != kFull) idle = 0;
        while (idle && !exhausted) {
            uint64_t q_next = q[0], q_end = q[1];
            if (q_next >= q_end) {
                unsigned long long base = 0;
                if (lane == 0) {
                    base = atomicAdd(P.counter, (unsigned long long)span);
                    // host abort (soc_abort, a watchdog): the chunk is dropped
                    // and the warp takes no more work; packages in flight end
                    // normally, so the counters of what was traced conserve
                    // energy exactly.  One read of host-mapped memory per chunk.
                    if (base < P.total && *reinterpret_cast<const volatile int *>(P.abort_flag)) {
                        *reinterpret_cast<volatile int *>(P.cut) = 1;
                        base = P.total;
                    }
                }
                base = __shfl_sync(kFull, base, 0);
                if (base >= P.total) { exhausted = true; break; }
                q_next = base;
                q_end = min((uint64_t)base + span, P.total);
            }
            const int n_idle = __popc(idle);
            const uint64_t avail = q_end - q_next;
            const int take = avail < (uint64_t)n_idle ? (int)avail : n_idle;
            const int rank = __popc(idle & lt_mask);
            if (!active && rank < take) {
                gidx = q_next + rank;
                const int it_idx = find_item(P.prefix, P.n_items, gidx);
                if (it_idx != item) {
                    item = it_idx;
                    const DevItem &IT = P.items[item];
                    C = P.clouds + IT.cloud;
                    const float2 kap = __ldg(C->kappa + IT.freq);
                    kabs = kap.x; ksca = kap.y;
                    g = __ldg(P.g_hg + IT.freq);
                    tally = P.tally + IT.tally_offset;
                }
                const DevItem &IT = P.items[item];
                const uint32_t pid = IT.pid_offset + (uint32_t)(gidx - P.prefix[item]);
                r.init(P.seed, (uint32_t)IT.iteration, (uint32_t)IT.freq, pid, (uint32_t)IT.cloud,
                       (uint32_t)IT.source);
                p.steps = 0; p.pend = 0; p.scat = false;
                if (emit<!kRegular>(*C, IT, pid, r, p, anc)) {
                    p.wf = ((p.W >> 20) ? (p.W >> 20) : 1u) |
                           ((kSelf && IT.source == SOC_SRC_DUST) ? kHomeBit : 0u);
                    set_inverse(p);
                    p.tauf = -log_pos(r.u());
                    if (acc_item != item) {
                        if (acc_item >= 0) {
                            unsigned long long *st = P.stats + 4 * acc_item;
                            if (acc[0]) atomicAdd(st + 0, acc[0]);
                            if (acc_cap) atomicAdd(st + 1, (unsigned long long)acc_cap);
                            if (acc[1]) atomicAdd(st + 2, acc[1]);
                            if (acc[2]) atomicAdd(st + 3, acc[2]);
                        }
                        acc_item = item; acc_cap = 0;
                        acc[0] = acc[1] = acc[2] = 0;
                    }
                    acc[2] += p.W;
                    active = true;
                } else if (P.pkg_steps) {
                    P.pkg_steps[gidx] = 0;
                }
            }
            __syncwarp();
            if (lane == 0) { q[0] = q_next + (uint64_t)take; q[1] = q_end; }
            __syncwarp();
            idle = __ballot_sync(kFull, !active);
        }
        if (!__any_sync(kFull, active)) {
            if (exhausted) break;
            continue;
        }
        // scattering phase: run the Henyey-Greenstein draw for the waiting
        // lanes together once scatter_min of them wait (or no active lane can
        // step); a package's draws and operations keep their order.
        // Descent phase (octrees): lanes that crossed into a refined cell
        // descend to the leaf together, once kDescendMin of them wait (or no
        // lane can step), rather than each inside its own step while the
        // rest of the warp waits.  Timed on GB300 (4.4e6-cell octree, 64 nu):
        // 213.5 ms against 241.7 ms with the descent inside the step, counters
        // unchanged; thresholds 1 to 6 lie within 1 %.
        {
            const unsigned act = __ballot_sync(kFull, active);
            const unsigned sc = __ballot_sync(kFull, active && p.scat);
            const unsigned dn = kRegular ? 0u : __ballot_sync(kFull, active && p.rho < 0.0f);
            const bool stuck = kRegular ? (sc == act) : ((act & ~(sc | dn)) == 0u);
            if (sc && (__popc(sc) >= P.scatter_min || stuck) && active && p.scat) {
                hg_scatter(r, g, p);
                set_inverse(p);
                p.tauf = -log_pos(r.u());
                p.scat = false;
            }
            if (!kRegular && dn && (__popc(dn) >= kDescendMin || stuck) && active && p.rho < 0.0f)
                descend<true>(kOneCloud ? P.hot.cell : C->cell, p, anc);
        }
        if (active && !p.scat && (kRegular || !(p.rho < 0.0f))) {
            // On regular grids (kRegular: no octree climbs or descents in a
            // step) two steps before the warp looks at refills and
            // scatterings again: half the passes of the scheduling code per
            // step.  Timed on GB300 (128^3, 64 nu): 71.5 ms against
            // 77.0 ms for one step, and slower with three or four steps or
            // with the two written as a loop.  Octree steps, whose climbs and
            // descents vary in length, are faster one at a time (78 against
            // 99 ms on the 4.4e6-cell octree).
            int res;
            if (kOneCloud) {
                const ParamCloud pc{P.hot};
                res = step<kSelf, kRegular>(pc, p, kabs, ksca, tally, P, anc);
                if (kRegular && res == kContinue && !p.scat) res = step<kSelf, kRegular>(pc, p, kabs, ksca, tally, P, anc);
            } else {
                const GlobalCloud gc{*C};
                res = step<kSelf, kRegular>(gc, p, kabs, ksca, tally, P, anc);
                if (kRegular && res == kContinue && !p.scat) res = step<kSelf, kRegular>(gc, p, kabs, ksca, tally, P, anc);
            }
            if (res != kContinue) {
                if (p.pend) {
                    atomicAdd(tally + p.cell, (unsigned long long)p.pend);
                    if (kSelf && (p.wf & kHomeBit))
                        atomicAdd(P.self + (tally - P.tally) + p.cell, (unsigned long long)p.pend);
                }
                p.pend = 0;
                if (res == kEscaped) acc[0] += p.W;
                if (res == kCapped) acc_cap += 1;
                acc[1] += p.steps;
                if (P.pkg_steps) P.pkg_steps[gidx] = p.steps;
                active = false;
            }
        }
    }
    if (acc_item >= 0) {
        unsigned long long *st = P.stats + 4 * acc_item;
        if (acc[0]) atomicAdd(st + 0, acc[0]);
        if (acc_cap) atomicAdd(st + 1, (unsigned long long)acc_cap);
        if (acc[1]) atomicAdd(st + 2, acc[1]);
        if (acc[2]) atomicAdd(st + 3, acc[2]);
    }
}

// ---------------------------------------------------------------------------
// Surface-brightness maps (paper Sect. 2.1.1: a separate kernel makes maps at
// chosen frequencies and directions from the solved temperatures).  One
// thread per pixel: the ray enters the root box (FP64 slab test), then walks
// the leaves with the tracer's FP32 cell-local traversal; along each segment
// of optical depth dtau = rho kext_root h s (FP32) the intensity gains
// S (1 - e^-dtau) e^-tau_front, with S = (kabs / kext) B_nu(T_cell) computed
// once per cell in FP64 (map_source_kernel) and the intensity and the
// transmission e^-tau_front accumulated in FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double planck_d(double nu, double T)
{
    const double h = 6.62607015e-27, k = 1.380649e-16, c = 2.99792458e10;
    return (2.0 * h * nu * nu * nu / (c * c)) / expm1(h * nu / (k * T));
}

// Source function of every cell at the map's frequency, (kabs/kext) B_nu(T),
// in FP64: one Planck evaluation per cell instead of one per ray segment.
__global__ void map_source_kernel(const float *__restrict__ T, int64_t n, double nu, double ratio,
                                  double *__restrict__ S)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        S[c] = ratio * planck_d(nu, (double)T[c]);
}

__global__ void map_kernel(const MapParams M)
{
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= M.npx || py >= M.npy) return;
    const DevCloud &C = *M.cloud;
    const double ox = M.c[0] + ((px + 0.5) - 0.5 * M.npx) * M.pix * M.e1[0] + ((py + 0.5) - 0.5 * M.npy) * M.pix * M.e2[0];
    const double oy = M.c[1] + ((px + 0.5) - 0.5 * M.npx) * M.pix * M.e1[1] + ((py + 0.5) - 0.5 * M.npy) * M.pix * M.e2[1];
    const double oz = M.c[2] + ((px + 0.5) - 0.5 * M.npx) * M.pix * M.e1[2] + ((py + 0.5) - 0.5 * M.npy) * M.pix * M.e2[2];
    const double o[3] = {ox, oy, oz};
    const double n[3] = {(double)C.nx, (double)C.ny, (double)C.nz};
    double t0 = -1e300, t1 = 1e300;
    int ea = -1;
    for (int a = 0; a < 3; ++a) {
        const double da = M.d[a];
        if (da == 0.0) {
            if (o[a] < 0.0 || o[a] > n[a]) { t0 = 1.0; t1 = 0.0; }
            continue;
        }
        double ta = (0.0 - o[a]) / da, tb = (n[a] - o[a]) / da;
        if (ta > tb) { const double tt = ta; ta = tb; tb = tt; }
        if (ta > t0) { t0 = ta; ea = a; }
        if (tb < t1) t1 = tb;
    }
    double I = 0.0, trans = 1.0;
    if (ea >= 0 && t0 < t1) {
        Pkg p;
        p.h = 1.0f;
        p.dx = (float)M.d[0]; p.dy = (float)M.d[1]; p.dz = (float)M.d[2];
        set_inverse(p);
        const double q[3] = {o[0] + t0 * M.d[0], o[1] + t0 * M.d[1], o[2] + t0 * M.d[2]};
        float lx, ly, lz;
        p.ri = root_axis((float)q[0], C.nx, lx);
        p.rj = root_axis((float)q[1], C.ny, ly);
        p.rk = root_axis((float)q[2], C.nz, lz);
        // the entry coordinate exactly on the face the ray enters through
        const bool up = M.d[ea] > 0.0;
        if (ea == 0) { p.ri = up ? 0 : C.nx - 1; lx = up ? 0.f : 1.f; }
        if (ea == 1) { p.rj = up ? 0 : C.ny - 1; ly = up ? 0.f : 1.f; }
        if (ea == 2) { p.rk = up ? 0 : C.nz - 1; lz = up ? 0.f : 1.f; }
        p.x = lx; p.y = ly; p.z = lz;
        p.cell = root_cell(C, p.ri, p.rj, p.rk);
        descend(C.cell, p);
        const float kext = (float)M.kext_root;
        for (uint32_t it = 0; it < M.max_cells; ++it) {
            float s = __int_as_float(0x7f800000);
            int ax = -1;
            if (p.dx != 0.0f) { const float si = __fmul_rn(__fsub_rn(p.dx > 0.0f ? 1.0f : 0.0f, p.x), p.ix); if (si < s) { s = si; ax = 0; } }
            if (p.dy != 0.0f) { const float si = __fmul_rn(__fsub_rn(p.dy > 0.0f ? 1.0f : 0.0f, p.y), p.iy); if (si < s) { s = si; ax = 1; } }
            if (p.dz != 0.0f) { const float si = __fmul_rn(__fsub_rn(p.dz > 0.0f ? 1.0f : 0.0f, p.z), p.iz); if (si < s) { s = si; ax = 2; } }
            if (ax < 0) break;
            const float dtau = __fmul_rn(__fmul_rn(__fmul_rn(p.rho, kext), p.h), s);
            if (dtau > 0.0f) {
                // the segment emits S (1 - e^-dtau), seen through the
                // transmission of everything in front of it.  The segment's
                // optical depth and factors are FP32, as in the tracer
                // (relative error ~1e-7 each, no cancellation: 1 - e^-x by
                // expm1f, e^-x by 1 - q below 0.5 and by expf above); the
                // running intensity and transmission stay FP64 (the FP64
                // pipe bounds this kernel: four FP64 operations a segment).
                const float q = -expm1f(-dtau);
                I = fma(__ldg(M.S + p.cell), (double)q * trans, I);
                trans *= (double)((dtau < 0.5f) ? __fsub_rn(1.0f, q) : expf(-dtau));
            }
            const float da = (ax == 0) ? p.dx : (ax == 1) ? p.dy : p.dz;
            const bool upx = da > 0.0f;
            const float face = upx ? 1.0f : 0.0f;
            const float mx = clamp01(__fadd_rn(p.x, __fmul_rn(p.dx, s)));
            const float my = clamp01(__fadd_rn(p.y, __fmul_rn(p.dy, s)));
            const float mz = clamp01(__fadd_rn(p.z, __fmul_rn(p.dz, s)));
            p.x = (ax == 0) ? face : mx;
            p.y = (ax == 1) ? face : my;
            p.z = (ax == 2) ? face : mz;
            if (!cross_face(GlobalCloud{C}, p, ax, upx)) break;
        }
    }
    M.map[(int64_t)py * M.npx + px] = (float)(I + M.I_bg * trans);
}

}  // namespace

cudaError_t launch_map(const MapParams &m, int64_t n_cells, int sms, cudaStream_t s)
{
    map_source_kernel<<<sms * 4, 256, 0, s>>>(m.T, n_cells, m.nu, m.kabs_over_kext, m.S);
    dim3 block(16, 16);
    dim3 grid((m.npx + 15) / 16, (m.npy + 15) / 16);
    map_kernel<<<grid, block, 0, s>>>(m);
    return cudaGetLastError();
}

// Dynamic shared memory of a tracer launch: the ancestor rows of octree launches.
static size_t trace_smem(int block, bool regular)
{
    return regular ? 0 : (size_t)block * kAncRows * sizeof(int32_t);
}

template <int kMinBlocks, bool kRegular>
static void launch_variant(const TraceParams &p, int grid, int block, cudaStream_t s)
{
    // the self-counter logic (ALI) is compiled only into the variants that need it
    const bool one = p.hot.cell != nullptr;
    const size_t sm = trace_smem(block, kRegular);
    if (p.self) {
        if (one) trace_kernel<kMinBlocks, true, true, kRegular><<<grid, block, sm, s>>>(p);
        else trace_kernel<kMinBlocks, true, false, kRegular><<<grid, block, sm, s>>>(p);
    } else {
        if (one) trace_kernel<kMinBlocks, false, true, kRegular><<<grid, block, sm, s>>>(p);
        else trace_kernel<kMinBlocks, false, false, kRegular><<<grid, block, sm, s>>>(p);
    }
}

cudaError_t launch_trace(const TraceParams &p, int grid, int block, int variant, cudaStream_t s)
{
    if (p.regular) {
        if (variant == 4) launch_variant<4, true>(p, grid, block, s);
        else launch_variant<3, true>(p, grid, block, s);
    } else {
        if (variant == 4) launch_variant<4, false>(p, grid, block, s);
        else launch_variant<3, false>(p, grid, block, s);
    }
    return cudaGetLastError();
}

int trace_block_limit(int block, int variant, bool regular)
{
    int n = 0;
    const size_t sm = trace_smem(block, regular);
    cudaError_t e;
    if (regular)
        e = (variant == 4)
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace_kernel<4, false, false, true>, block, sm)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace_kernel<3, false, false, true>, block, sm);
    else
        e = (variant == 4)
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace_kernel<4, false, false, false>, block, sm)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace_kernel<3, false, false, false>, block, sm);
    if (e != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace soc
