// soc_nn.cu -- the learned temperature seed: a 3D U-Net trained and run by
// this library's own kernels (tensor cores in BF16 with FP32 accumulation).
//
// The method itself has no network; the seed replaces the first, most
// expensive iterations of the temperature solution (paper Sect. 3.3-3.4
// discuss cutting the cost of the early iterations).  Layout: channels-last
// (N, D, H, W, C), BF16 activations, FP32 master weights, gradients and Adam
// moments.
//
// Convolutions (3x3x3, stride 1, zero padding 1) are implicit GEMMs:
//   forward:  M = voxels, N = C_out, K = 27 C_in (tap-major, channel-minor),
//             on the tcgen05 tensor cores with the accumulator in tensor
//             memory, operands staged by the Tensor Memory Accelerator;
//   dgrad:    the forward kernel with the weights flipped in space and
//             transposed in channels;
//   wgrad:    M = C_out, N = C_in per tap, K = voxels (split over blocks
//             that write partial sums, reduced in a fixed order), on the
//             tcgen05 tensor cores as well.
// BF16 inputs, FP32 accumulation throughout.  Every reduction (weight and
// bias gradients, the loss) sums per-block partials in a fixed order, so a
// training run is bit-reproducible.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>
#include "soc_internal.h"

namespace soc {
namespace nn {

using bf16 = __nv_bfloat16;

struct ConvArgs {
    const bf16 *in;
    int in_stride, in_off;          // elements per voxel, first channel
    const bf16 *w;                  // [Cout][27][Cin]
    const float *bias;              // [Cout] or null
    bf16 *out;                      // BF16 output (when out_f32 is null)
    float *out_f32;                 // FP32 output (optional)
    int out_stride, out_off;
    int N, D, H, W, Cin, Cout;
    int relu, accumulate;           // accumulate: FP32 output += result
};

// ---------------------------------------------------------------------------
// Helpers of the tensor-core kernels (tcgen05.mma with the accumulator in
// tensor memory; shared-memory operand descriptors; bounded mbarrier waits).
// Every wait is bounded: on a timeout a block raises the error flag, frees
// its tensor memory and returns.
// ---------------------------------------------------------------------------
__device__ int g_tc_error;                    // set by a block whose wait timed out

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start, leading and stride byte offsets
// (all >> 4), descriptor version 1, no swizzling.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t mma_idesc(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(addr), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// 16-byte asynchronous copy global -> shared through L1 (the 27 taps of a
// tile re-read most of its input); src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// ---------------------------------------------------------------------------
// Forward (and dgrad) convolution with operands staged by the Tensor Memory
// Accelerator.  A block computes a box of 128 output voxels (bx x by x bz x
// bn over W, H, D, N; accumulator row r = voxel ((n bz + z) by + y) bx + x of
// the box) x n_tile output channels.  For every tap and chunk of KC input
// channels, one TMA load brings the input box shifted by the tap's offset --
// coordinates outside the volume read zeros, which is the convolution's
// padding -- and a second one the weights (n_tile rows x KC), both with
// rows of KC * 2 bytes in the hardware's 32/64/128-byte swizzle, which the
// MMA's shared-memory descriptors name.  One thread issues the loads
// (mbarrier with the expected byte count per stage), another the MMAs
// (committed to the stage's "empty" mbarrier), n_stages stages deep; every
// wait is bounded (on a timeout the block raises the error flag, waits for
// its loads and MMAs in flight, frees its tensor memory and returns).
// ---------------------------------------------------------------------------
// Output of a convolution: bias, ReLU, then BF16 or FP32 (optionally added
// to what is there) at out[v * out_stride + out_off + co].
struct ConvOut {
    bf16 *out;
    float *out_f32;
    const float *bias;
    int out_stride, out_off, relu, accumulate;
};

struct TmaConvArgs {
    int N, D, H, W, Cin, Cout;
    int bx, by, bz, bn;              // output box (bx by bz bn <= 128)
    int tiles_x, tiles_y, tiles_z;
    ConvOut o;
};

// 16 consecutive accumulator columns of the warp's 32 tensor-memory lanes
__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&rr)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                   "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
                   "=r"(rr[14]), "=r"(rr[15])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Output channels co .. co + 15 of voxel v from their FP32 accumulators
__device__ __forceinline__ void store_row16(const ConvOut &o, long long v, int co, const uint32_t (&rr)[16])
{
    float val[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        float t = __uint_as_float(rr[j]);
        if (o.bias) t += o.bias[co + j];
        if (o.relu) t = fmaxf(t, 0.f);
        val[j] = t;
    }
    const long long off = v * o.out_stride + o.out_off + co;
    if (o.out_f32) {
        float4 *dst = reinterpret_cast<float4 *>(o.out_f32 + off);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
            float4 w4 = make_float4(val[4 * q4], val[4 * q4 + 1], val[4 * q4 + 2], val[4 * q4 + 3]);
            if (o.accumulate) {
                const float4 old = dst[q4];
                w4.x += old.x; w4.y += old.y; w4.z += old.z; w4.w += old.w;
            }
            dst[q4] = w4;
        }
    } else {
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(val[2 * j], val[2 * j + 1]);
            pk[j] = *reinterpret_cast<const uint32_t *>(&h2);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(o.out + off);
        dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
}

// Shared-memory descriptor of a K-major operand whose rows are `row_bytes`
// (32, 64 or 128) long in the matching swizzle: 8-row groups row_bytes * 8
// apart (stride offset), layout type 6 / 4 / 2.
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t addr, int row_bytes)
{
    const uint64_t layout = row_bytes == 32 ? 6ull : (row_bytes == 64 ? 4ull : 2ull);
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) |
           ((uint64_t)(((uint32_t)row_bytes * 8u >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (layout << 61);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
                    "r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar) : "memory");
}

// Bookkeeping of a persistent convolution block, in shared memory after its
// n_stages operand stages: full/empty per stage (TMA bytes arrived / MMAs
// done with it), acc_full/acc_empty per accumulator buffer (MMAs of a box
// done / epilogue done), the drain barrier (all MMAs done, after a failure),
// the tensor-memory slot and the failure flag.
struct ConvBlock {
    uint64_t *full, *empty, *acc_full, *acc_empty, *drain;
    int *s_fail;
    uint32_t tmem;
};

// Carve the bookkeeping after the stages, allocate tmem_cols columns of
// tensor memory (warp 5) and initialise the barriers (thread 0).  Every
// thread of the block calls it.
__device__ __forceinline__ ConvBlock conv_block_begin(uint8_t *after_stages, int n_stages, uint32_t tmem_cols)
{
    ConvBlock c;
    c.full = reinterpret_cast<uint64_t *>(after_stages);
    c.empty = c.full + n_stages;
    c.acc_full = c.empty + n_stages;
    c.acc_empty = c.acc_full + 2;
    c.drain = c.acc_empty + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(c.drain + 1);
    c.s_fail = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < n_stages; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&c.full[k])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&c.empty[k])) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&c.acc_full[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" :: "r"(smem_u32(&c.acc_empty[b])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(c.drain)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *c.s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    c.tmem = *tslot;
    return c;
}

// The producer's last stages (issued: its copies so far, into stages
// h mod n_stages): after a failure the copies in flight land, else the MMAs'
// releases of them arrive, before the block leaves.  Bounded waits.
__device__ __forceinline__ void conv_producer_tail(const ConvBlock &c, int n_stages, int issued)
{
    const bool failed = *reinterpret_cast<volatile int *>(c.s_fail);
    for (int h = (issued > n_stages ? issued - n_stages : 0); h < issued; ++h)
        mbar_wait(smem_u32(failed ? &c.full[h % n_stages] : &c.empty[h % n_stages]), (uint32_t)(h / n_stages) & 1u);
}

// End of a block: every MMA has completed before the tensor memory is freed
// (the epilogue waited for the last box's accumulator, or, after a failure,
// the MMA thread waits, bounded, for all it issued); a failure raises the
// error flag.  Every thread calls it.
__device__ __forceinline__ void conv_block_end(const ConvBlock &c, uint32_t tmem_cols)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const bool ok = __syncthreads_and(!*reinterpret_cast<volatile int *>(c.s_fail));
    if (!ok) {
        if (tid == 0) atomicExch(&g_tc_error, 1);
        if (warp == 5 && lane == 0) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(c.drain)) : "memory");
            mbar_wait(smem_u32(c.drain), 0);
        }
    }
    __syncthreads();
    if (warp == 5) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(c.tmem), "r"(tmem_cols) : "memory");
    }
}

// Persistent and warp-specialised: a block of 6 warps walks the output
// boxes blockIdx.x, blockIdx.x + gridDim.x, ...  Warp 4 (lane 0) issues the
// TMA loads into n_stages shared-memory stages, warp 5 (lane 0) the MMAs into
// one of two accumulators in tensor memory (2 x n_tile columns), and warps
// 0-3 (tensor-memory lanes 32w .. 32w + 31) drain the other accumulator:
// loads of the next box, MMAs and the epilogue of the previous one overlap.
// Barriers: full/empty per stage (TMA bytes arrived / MMAs done with it),
// acc_full/acc_empty per accumulator (MMAs of a box done / epilogue done).
constexpr int kConvThreads = 192;

template <int KC>
__global__ void __launch_bounds__(kConvThreads) conv3d_tma_kernel(const __grid_constant__ CUtensorMap map_in,
                                                                  const __grid_constant__ CUtensorMap map_w,
                                                                  const TmaConvArgs a, int n_tile, uint32_t tmem_cols,
                                                                  int n_stages)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // stages start on 1024-byte boundaries (the swizzle pattern repeats every
    // 8 rows of up to 128 bytes)
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int kRow = KC * 2;                       // bytes per operand row
    const int a_bytes = 128 * kRow, b_bytes = n_tile * kRow;
    const int stage_bytes = a_bytes + b_bytes;         // multiple of 1024
    const ConvBlock cb = conv_block_begin(smem + n_stages * stage_bytes, n_stages, tmem_cols);
    uint64_t *const full = cb.full, *const empty = cb.empty, *const acc_full = cb.acc_full;
    uint64_t *const acc_empty = cb.acc_empty;
    int *const s_fail = cb.s_fail;
    volatile int *fail = s_fail;
    const uint32_t tmem = cb.tmem;
    const uint32_t smem0 = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.y * n_tile;
    const int n_chunks = a.Cin / KC;
    const int steps = 27 * n_chunks;                   // per box
    const int n_boxes = a.tiles_x * a.tiles_y * a.tiles_z * ((a.N + a.bn - 1) / a.bn);
    const uint32_t tx_bytes = (uint32_t)(a.bx * a.by * a.bz * a.bn) * kRow + (uint32_t)b_bytes;


    if (warp == 4) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&map_in)) : "memory");
            asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&map_w)) : "memory");
            // producer: step g = (box, tap, chunk) into stage st = g mod
            // n_stages, in round ph = floor(g / n_stages) mod 2, once the MMAs
            // of step g - n_stages have released it
            int st = 0, issued = 0;
            uint32_t ph = 0;
            for (int box = blockIdx.x; box < n_boxes && !*fail; box += gridDim.x) {
                int q = box;
                const int tx = q % a.tiles_x; q /= a.tiles_x;
                const int ty = q % a.tiles_y; q /= a.tiles_y;
                const int tz = q % a.tiles_z;
                const int tn = q / a.tiles_z;
                const int x0 = tx * a.bx - 1, y0 = ty * a.by - 1, z0 = tz * a.bz - 1, nb0 = tn * a.bn;
                bool stop = false;
                for (int tap = 0, dx = 0, dy = 0, dz = 0; tap < 27 && !stop; ++tap) {
                    for (int c0 = 0; c0 < a.Cin; c0 += KC) {
                        if (issued >= n_stages && !mbar_wait(smem_u32(&empty[st]), ph ^ 1u)) {
                            atomicExch(s_fail, 1);
                            stop = true;
                            break;
                        }
                        if (*fail) { stop = true; break; }
                        const uint32_t dst = smem0 + (uint32_t)(st * stage_bytes);
                        const uint32_t bar = smem_u32(&full[st]);
                        mbar_expect_tx(bar, tx_bytes);
                        tma_load_5d(dst, &map_in, c0, x0 + dx, y0 + dy, z0 + dz, nb0, bar);
                        tma_load_2d(dst + (uint32_t)a_bytes, &map_w, tap * a.Cin + c0, n0, bar);
                        ++issued;
                        if (++st == n_stages) { st = 0; ph ^= 1u; }
                    }
                    // tap = 9 dz + 3 dy + dx
                    if (++dx == 3) { dx = 0; if (++dy == 3) { dy = 0; ++dz; } }
                }
                if (stop) break;
            }
            conv_producer_tail(cb, n_stages, issued);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer: box i into accumulator i % 2, once the epilogue has
            // drained box i - 2 from it
            const uint32_t idesc = mma_idesc(128, n_tile);
            int st = 0, i = 0;
            uint32_t ph = 0;
            for (int box = blockIdx.x; box < n_boxes && !*fail; box += gridDim.x, ++i) {
                const int b = i & 1;
                if (i >= 2 && !mbar_wait(smem_u32(&acc_empty[b]), (uint32_t)((i >> 1) - 1) & 1u)) {
                    atomicExch(s_fail, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc_addr = tmem + (uint32_t)(b * n_tile);
                for (int t = 0; t < steps; ++t) {
                    if (!mbar_wait(smem_u32(&full[st]), ph)) {
                        atomicExch(s_fail, 1);
                        break;
                    }
                    if (*fail) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem0 + (uint32_t)(st * stage_bytes), b0 = a0 + (uint32_t)a_bytes;
#pragma unroll
                    for (int j = 0; j < KC / 16; ++j) {
                        const uint64_t ad = smem_desc_sw(a0 + j * 32, kRow);
                        const uint64_t bd = smem_desc_sw(b0 + j * 32, kRow);
                        const uint32_t acc = (t > 0 || j > 0) ? 1u : 0u;
                        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                     :: "r"(acc_addr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(smem_u32(&empty[st])) : "memory");
                    if (++st == n_stages) { st = 0; ph ^= 1u; }
                }
                // the box's accumulator is complete once its MMAs are
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(smem_u32(&acc_full[b])) : "memory");
            }
        }
    } else {
        // epilogue: warps 0-3, accumulator row tid = voxel of the box
        int i = 0;
        for (int box = blockIdx.x; box < n_boxes; box += gridDim.x, ++i) {
            const int b = i & 1;
            const bool ready = mbar_wait(smem_u32(&acc_full[b]), (uint32_t)(i >> 1) & 1u);
            if (__any_sync(0xffffffffu, !ready || *fail)) { atomicExch(s_fail, 1); break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int q = box;
            const int tx = q % a.tiles_x; q /= a.tiles_x;
            const int ty = q % a.tiles_y; q /= a.tiles_y;
            const int tz = q % a.tiles_z;
            const int tn = q / a.tiles_z;
            int r = tid;
            const int x = tx * a.bx + r % a.bx; r /= a.bx;
            const int y = ty * a.by + r % a.by; r /= a.by;
            const int z = tz * a.bz + r % a.bz;
            const int nn = tn * a.bn + r / a.bz;
            const bool vin = tid < a.bx * a.by * a.bz * a.bn && x < a.W && y < a.H && z < a.D && nn < a.N;
            const long long v = vin ? (((long long)nn * a.D + z) * a.H + y) * a.W + x : 0;
            const uint32_t row_addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * n_tile);
            for (int c = 0; c < n_tile; c += 16) {
                uint32_t rr[16];
                tmem_ld16(row_addr + (uint32_t)c, rr);
                if (vin) store_row16(a.o, v, n0 + c, rr);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&acc_empty[b])) : "memory");
        }
    }
    conv_block_end(cb, tmem_cols);
}

// ---------------------------------------------------------------------------
// Slab-fed convolution, for volumes whose rows hold W = 8 .. 128 voxels with
// W dividing 128.  An output box is bx = W by by x bz voxels of one sample,
// n_acc groups of 128 voxels (g = 128 / W consecutive rows each, gyn groups
// along y, bz along z).  For every chunk of KC input channels and x offset
// dx, TMA loads (one per row) bring the slab of voxels x + dx - 1 (x = 0 ..
// W - 1), y0 - 1 .. y0 + by, z0 - 1 .. z0 + bz (out-of-volume voxels read
// zero), and nine loads the weights of the taps (dx, dy, dz).  The A operand of tap
// (dy, dz) and group (gy, gz) is the 128 consecutive slab rows from
// ((gz + dz)(by + 2) + g gy + dy) W on: a multiple of 8 rows, so the swizzle
// atoms stay aligned.  Every input voxel is then read from L2 3 (by + 2)
// (bz + 2) / (by bz) times per chunk instead of 27.  Block organisation,
// barriers and the bounded waits are those of conv3d_tma_kernel; the
// accumulators of box i are the n_acc x n_tile columns of buffer i mod 2.
// ---------------------------------------------------------------------------
struct SlabArgs {
    int N, D, H, W, Cin, Cout;
    int by, bz, g, gyn, n_acc, tiles_y, tiles_z;
    ConvOut o;
};

template <int KC, int NACC>
__global__ void __launch_bounds__(kConvThreads, 1) conv3d_slab_kernel(const __grid_constant__ CUtensorMap map_in,
                                                                   const __grid_constant__ CUtensorMap map_w,
                                                                   const SlabArgs a, int n_tile, uint32_t tmem_cols,
                                                                   int n_stages, int slab_bytes, int stage_bytes)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int kRow = KC * 2;
    const int bx = a.W;
    const int rows_s = bx * (a.by + 2) * (a.bz + 2);
    const int tap_bytes = n_tile * kRow;
    const ConvBlock cb = conv_block_begin(smem + n_stages * stage_bytes, n_stages, tmem_cols);
    uint64_t *const full = cb.full, *const empty = cb.empty, *const acc_full = cb.acc_full;
    uint64_t *const acc_empty = cb.acc_empty;
    int *const s_fail = cb.s_fail;
    volatile int *fail = s_fail;
    const uint32_t tmem = cb.tmem;
    const uint32_t smem0 = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.y * n_tile;
    const int n_boxes = a.tiles_y * a.tiles_z * a.N;
    const uint32_t tx_bytes = (uint32_t)rows_s * kRow + 9u * (uint32_t)tap_bytes;


    if (warp == 4) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&map_in)) : "memory");
            asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&map_w)) : "memory");
            const int n_rows = (a.by + 2) * (a.bz + 2), row_bytes = bx * kRow;
            int st = 0, issued = 0;
            uint32_t ph = 0;
            bool stop = false;
            for (int box = blockIdx.x; box < n_boxes && !stop && !*fail; box += gridDim.x) {
                const int ty = box % a.tiles_y, q = box / a.tiles_y;
                const int tz = q % a.tiles_z, nn = q / a.tiles_z;
                const int y0 = ty * a.by - 1, z0 = tz * a.bz - 1;
                for (int c0 = 0; c0 < a.Cin && !stop; c0 += KC) {
                    for (int dx = 0; dx < 3; ++dx) {
                        if (issued >= n_stages && !mbar_wait(smem_u32(&empty[st]), ph ^ 1u)) {
                            atomicExch(s_fail, 1);
                            stop = true;
                            break;
                        }
                        if (*fail) { stop = true; break; }
                        const uint32_t dst = smem0 + (uint32_t)(st * stage_bytes);
                        const uint32_t bar = smem_u32(&full[st]);
                        mbar_expect_tx(bar, tx_bytes);
                        // the slab one row (y, z) at a time: many short
                        // copies in flight keep the copy engine busier
                        // than one large box
                        for (int r = 0, ry = 0, rz = 0; r < n_rows; ++r) {
                            tma_load_5d(dst + (uint32_t)(r * row_bytes), &map_in, c0, dx - 1, y0 + ry, z0 + rz, nn,
                                        bar);
                            if (++ry == a.by + 2) { ry = 0; ++rz; }
                        }
                        // weights of taps 9 dz + 3 dy + dx, block 3 dz + dy
                        for (int t9 = 0; t9 < 9; ++t9)
                            tma_load_2d(dst + (uint32_t)(slab_bytes + t9 * tap_bytes), &map_w,
                                        (3 * t9 + dx) * a.Cin + c0, n0, bar);
                        ++issued;
                        if (++st == n_stages) { st = 0; ph ^= 1u; }
                    }
                }
            }
            conv_producer_tail(cb, n_stages, issued);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            const uint32_t idesc = mma_idesc(128, n_tile);
            const int steps = 3 * (a.Cin / KC);
            // descriptor start-address offsets (16-byte units): A rows of
            // group q at dy = dz = 0, one row of the slab in y and in z, one
            // tap's weights (a descriptor plus an offset names the shifted
            // operand: smem addresses stay below 2^18, the 14-bit field
            // does not overflow)
            uint32_t q_off[NACC];
#pragma unroll
            for (int q = 0; q < NACC; ++q) {
                const int gz = q / a.gyn, gy = q - gz * a.gyn;
                q_off[q] = (uint32_t)((gz * (a.by + 2) + gy * a.g) * bx * kRow) >> 4;
            }
            const uint32_t dy_off = (uint32_t)(bx * kRow) >> 4, dz_off = (uint32_t)((a.by + 2) * bx * kRow) >> 4;
            const uint32_t tap_off = (uint32_t)tap_bytes >> 4;
            int st = 0, i = 0;
            uint32_t ph = 0;
            for (int box = blockIdx.x; box < n_boxes && !*fail; box += gridDim.x, ++i) {
                const int b = i & 1;
                if (i >= 2 && !mbar_wait(smem_u32(&acc_empty[b]), (uint32_t)((i >> 1) - 1) & 1u)) {
                    atomicExch(s_fail, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc0 = tmem + (uint32_t)(b * NACC * n_tile);
                for (int s = 0; s < steps; ++s) {
                    if (!mbar_wait(smem_u32(&full[st]), ph)) {
                        atomicExch(s_fail, 1);
                        break;
                    }
                    if (*fail) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem0 + (uint32_t)(st * stage_bytes);
                    const uint64_t da = smem_desc_sw(a0, kRow), db = smem_desc_sw(a0 + (uint32_t)slab_bytes, kRow);
#pragma unroll
                    for (int t9 = 0; t9 < 9; ++t9) {
                        const uint32_t rt = (uint32_t)(t9 / 3) * dz_off + (uint32_t)(t9 % 3) * dy_off;
#pragma unroll
                        for (int q = 0; q < NACC; ++q) {
#pragma unroll
                            for (int j = 0; j < KC / 16; ++j) {
                                const uint64_t ad = da + (q_off[q] + rt + 2u * j);
                                const uint64_t bd = db + ((uint32_t)t9 * tap_off + 2u * j);
                                const uint32_t acc = (s > 0 || t9 > 0 || j > 0) ? 1u : 0u;
                                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                             :: "r"(acc0 + (uint32_t)(q * n_tile)), "l"(ad), "l"(bd), "r"(idesc),
                                                "r"(acc) : "memory");
                            }
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(smem_u32(&empty[st])) : "memory");
                    if (++st == n_stages) { st = 0; ph ^= 1u; }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(smem_u32(&acc_full[b])) : "memory");
            }
        }
    } else {
        // epilogue: warps 0-3; accumulator row tid of group q = voxel
        // (x, y) = (tid mod W, y0 + g gy + tid / W), z = z0 + gz
        int i = 0;
        for (int box = blockIdx.x; box < n_boxes; box += gridDim.x, ++i) {
            const int b = i & 1;
            const bool ready = mbar_wait(smem_u32(&acc_full[b]), (uint32_t)(i >> 1) & 1u);
            if (__any_sync(0xffffffffu, !ready || *fail)) { atomicExch(s_fail, 1); break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int ty = box % a.tiles_y, qq = box / a.tiles_y;
            const int tz = qq % a.tiles_z, nn = qq / a.tiles_z;
            const int x = tid % bx;
#pragma unroll
            for (int q = 0; q < NACC; ++q) {
                const int gz = q / a.gyn, gy = q - gz * a.gyn;
                const int y = ty * a.by + gy * a.g + tid / bx, z = tz * a.bz + gz;
                const bool vin = y < a.H && z < a.D;
                const long long v = vin ? (((long long)nn * a.D + z) * a.H + y) * a.W + x : 0;
                const uint32_t row_addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((b * NACC + q) * n_tile);
                for (int c = 0; c < n_tile; c += 16) {
                    uint32_t rr[16];
                    tmem_ld16(row_addr + (uint32_t)c, rr);
                    if (vin) store_row16(a.o, v, n0 + c, rr);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&acc_empty[b])) : "memory");
        }
    }
    conv_block_end(cb, tmem_cols);
}

// Wt[ci][t][co] = W[co][26 - t][ci]: weights of the transposed convolution.
__global__ void flip_weights_kernel(const bf16 *W, int Cout, int Cin, bf16 *Wt)
{
    const long long n = (long long)Cout * 27 * Cin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(i % Cout);
        const int t = (int)((i / Cout) % 27);
        const int ci = (int)(i / (27LL * Cout));
        Wt[i] = W[((long long)co * 27 + (26 - t)) * Cin + ci];
    }
}

struct WgradArgs {
    const bf16 *gy;
    int gy_stride, gy_off;
    const bf16 *x;
    int x_stride, x_off;
    float *part;                     // [gridDim.x][Cout][27][Cin]: each block's partial sums
    int N, D, H, W, Cin, Cout;
    long long vox_per_block;
};

// ---------------------------------------------------------------------------
// Weight gradient on the tcgen05 tensor cores:
//   gw[co][tap][ci] += sum_v x[v + off(tap)][ci] gy[v][co]
// The M = 128 rows of the accumulator are (tap, input channel) pairs: a
// block takes TT = 128 / ci_tile consecutive taps of ci_tile input channels
// (8 taps of 16 channels, 4 of 32, 2 of 64, 1 of 128), N = n_tile output
// channels, K = voxels (split over blocks along x; block x writes its sums to
// partial slice x, and reduce_partials_kernel adds the slices in order, so
// the result does not depend on block scheduling).  Both operands are
// staged MN-major: one 16-byte global row (8 channels of one voxel) is one
// row of a core matrix (8 K-rows of 8 consecutive M or N elements, 128
// bytes).  Core (mn, k) of A sits at (k * 16 + mn) * 128 bytes, of B at
// (k * n_tile / 8 + mn) * 128: the stride between cores along M/N (the
// descriptor's stride offset) is 128 B, along K (its leading offset)
// 16 * 128 or n_tile / 8 * 128 B.  A step covers kWgKV = 128 voxels (eight
// MMAs with K = 16); two threads of the block's 256 share a voxel, and warps
// 0-3 read the accumulator out.
// ---------------------------------------------------------------------------
constexpr int kWgKV = 128;
constexpr int kWgThreads = 2 * kWgKV;         // two threads per voxel of a step

__host__ __device__ constexpr uint32_t mma_idesc_mn(int m, int n)
{
    return mma_idesc(m, n) | (1u << 15) | (1u << 16);       // A and B MN-major
}

__global__ void __launch_bounds__(kWgThreads) conv3d_wgrad_tc_kernel(const WgradArgs a, int ci_tile, int n_tile,
                                                             uint32_t tmem_cols, int n_stages)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int a_bytes = 128 * kWgKV * 2, b_bytes = n_tile * kWgKV * 2;
    const int stage_bytes = a_bytes + b_bytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + n_stages * stage_bytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + n_stages * stage_bytes + 8 * n_stages);
    const uint32_t smem0 = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long V = (long long)a.N * a.D * a.H * a.W;
    const int TT = 128 / ci_tile;                         // taps per block
    const int n_co_tiles = a.Cout / n_tile;
    const int tap0 = blockIdx.y * TT;
    const int ci0 = (blockIdx.z / n_co_tiles) * ci_tile;
    const int co0 = (blockIdx.z % n_co_tiles) * n_tile;
    const long long vb = (long long)blockIdx.x * a.vox_per_block;
    const long long ve = vb + a.vox_per_block < V ? vb + a.vox_per_block : V;
    const int total = (int)((ve - vb + kWgKV - 1) / kWgKV);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < n_stages; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[k])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    const int NC = n_tile / 8, CP = ci_tile / 8;           // 16-byte pieces per voxel of B and per tap of A
    const uint32_t a_lbo = 16 * 128, b_lbo = (uint32_t)NC * 128;      // stride between cores along K
    const uint32_t idesc = mma_idesc_mn(128, n_tile);
    const int kv = tid & (kWgKV - 1), half = tid / kWgKV;              // this thread's voxel and half

    // this thread's 8 pieces of A: piece pc = half * 8 + i is tap tap0 +
    // pc / CP of the block (offsets tdx, tdy, tdz), channels tco
    int tdx[8], tdy[8], tdz[8], tco[8];
    bool tin[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int pc = half * 8 + i, tl = pc / CP, tap = tap0 + tl;
        tin[i] = tap < 27;
        tdz[i] = tap / 9 - 1;
        tdy[i] = (tap / 3) % 3 - 1;
        tdx[i] = tap % 3 - 1;
        tco[i] = a.x_off + ci0 + (pc - tl * CP) * 8;
    }
    // the voxel of the next step, advanced by kWgKV per step
    long long cv = vb + kv;
    int cx = 0, cy = 0, cz = 0;
    long long cn = 0;
    {
        long long q = cv < V ? cv : 0;
        cx = (int)(q % a.W); q /= a.W;
        cy = (int)(q % a.H); q /= a.H;
        cz = (int)(q % a.D); cn = q / a.D;
    }

    auto issue = [&](int t) {
        if (t < total) {
            const uint32_t st = smem0 + (uint32_t)((t % n_stages) * stage_bytes);
            const long long v = cv;
            const bool vin = v < ve;
            // A: the 16 pieces of this voxel's row of cores
            const uint32_t arow = st + (uint32_t)(((kv >> 3) * 16) * 128 + (kv & 7) * 16);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int zz = cz + tdz[i], yy = cy + tdy[i], xx = cx + tdx[i];
                const bool ok = vin && tin[i] && (unsigned)zz < (unsigned)a.D && (unsigned)yy < (unsigned)a.H &&
                                (unsigned)xx < (unsigned)a.W;
                const long long sv = ok ? ((cn * a.D + zz) * a.H + yy) * a.W + xx : 0;
                cp_async16(arow + (half * 8 + i) * 128, a.x + sv * a.x_stride + tco[i], ok ? 16u : 0u);
            }
            // B: gy[v][co0 .. co0 + n_tile - 1], half of the NC pieces
            const uint32_t brow = st + (uint32_t)a_bytes + (uint32_t)(((kv >> 3) * NC) * 128 + (kv & 7) * 16);
            for (int nc = half * (NC / 2); nc < (half + 1) * (NC / 2); ++nc)
                cp_async16(brow + nc * 128, a.gy + (vin ? v * a.gy_stride : 0) + a.gy_off + co0 + nc * 8,
                           vin ? 16u : 0u);
            // next step's voxel: kWgKV further along x, carried into y, z, n
            cv += kWgKV;
            cx += kWgKV;
            while (cx >= a.W) {
                cx -= a.W;
                if (++cy == a.H) {
                    cy = 0;
                    if (++cz == a.D) { cz = 0; ++cn; }
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    bool ok_run = true;
    int last = -1;
    const int ahead = n_stages - 2;
    for (int t = 0; t < ahead; ++t) issue(t);
    for (int step = 0; step < total; ++step) {
        const int s = step % n_stages;
        const int nxt = step + ahead;
        bool waited = true;
        if (step >= 2 && nxt < total) {
            const int prev = step - 2;
            waited = mbar_wait(smem_u32(&mbar[prev % n_stages]), (uint32_t)(prev / n_stages) & 1u);
        }
        if (waited) issue(nxt);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        // this step's copies have landed once at most `ahead` later groups
        // are pending (the count is an immediate)
        switch (ahead) {
        case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
        case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (!__syncthreads_and(waited)) { ok_run = false; break; }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem0 + (uint32_t)(s * stage_bytes), b0 = a0 + (uint32_t)a_bytes;
#pragma unroll
            for (int j = 0; j < kWgKV / 16; ++j) {
                const uint64_t ad = smem_desc(a0 + j * 2 * a_lbo, a_lbo, 128);
                const uint64_t bd = smem_desc(b0 + j * 2 * b_lbo, b_lbo, 128);
                const uint32_t acc = (step > 0 || j > 0) ? 1u : 0u;
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&mbar[s])) : "memory");
        }
        last = step;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    {
        bool done = true;
        if (last >= 0) done = mbar_wait(smem_u32(&mbar[last % n_stages]), (uint32_t)(last / n_stages) & 1u);
        ok_run = __syncthreads_and(ok_run && done);
    }
    if (!ok_run) {
        if (tid == 0) atomicExch(&g_tc_error, 1);
    } else if (warp < 4) {
        // warps 0-3 read the 128 accumulator lanes (warp w: lanes 32w ..)
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t row_addr = tmem + ((uint32_t)(warp * 32) << 16);
        const int tap = tap0 + tid / ci_tile, ci = ci0 + tid % ci_tile;   // accumulator lane = (tap, ci)
        float *const slice = a.part + (long long)blockIdx.x * a.Cout * 27 * a.Cin;
        for (int c = 0; c < n_tile; c += 16) {
            uint32_t r[16];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15])
                         : "r"(row_addr + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (tap >= 27) continue;
            float *dst = slice + ((long long)(co0 + c) * 27 + tap) * a.Cin + ci;
#pragma unroll
            for (int j = 0; j < 16; ++j) dst[(long long)j * 27 * a.Cin] = last >= 0 ? __uint_as_float(r[j]) : 0.f;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// out[i] += sum_{k < n_parts} part[k * n + i], k in increasing order (the
// fixed-order reduction of per-block partial sums).
__global__ void reduce_partials_kernel(const float *part, int n_parts, long long n, float *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < n_parts; ++k) s += part[(long long)k * n + i];
        out[i] += s;
    }
}

// Bias gradient, per block: part[blockIdx.x][c] = sum over the block's voxels
// of gy[v][c] (BF16 gradient, dense C channels), 256 / C voxel lanes of C
// channels each; bias_reduce_kernel adds the blocks' sums in a fixed order.
__global__ void bias_grad_kernel(const bf16 *gy, int C, long long V, long long vox_per_block, float *part)
{
    __shared__ float s_part[256];
    const long long vb = (long long)blockIdx.x * vox_per_block;
    const long long ve = vb + vox_per_block < V ? vb + vox_per_block : V;
    const int c = threadIdx.x % C, lane_v = threadIdx.x / C, nv = blockDim.x / C;
    float s = 0.f;
    if (lane_v < nv)
        for (long long v = vb + lane_v; v < ve; v += nv) s += __bfloat162float(gy[v * C + c]);
    s_part[threadIdx.x] = (lane_v < nv) ? s : 0.f;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.f;
        for (int k = 0; k < nv; ++k) t += s_part[k * C + threadIdx.x];
        part[(long long)blockIdx.x * C + threadIdx.x] = t;
    }
}

// gb[c] += sum over k of part[k][c], block c: thread t takes k = t, t + 256,
// ... in order, then a fixed tree over the 256 threads (the same order on
// every run).
__global__ void bias_reduce_kernel(const float *part, int n_parts, int C, float *gb)
{
    __shared__ float s_sum[256];
    const int c = blockIdx.x;
    float t = 0.f;
    for (int k = threadIdx.x; k < n_parts; k += blockDim.x) t += part[(long long)k * C + c];
    s_sum[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_sum[threadIdx.x] += s_sum[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[c] += s_sum[0];
}

// out_bf16[v][c] = (mask == null || mask[v][c] > 0) ? bf16(g[v][c]) : 0;
// one voxel per thread, 8 channels at a time (C, the strides and offsets
// multiples of 8, of 4 for g).
__global__ void mask_to_bf16_kernel(const float *g, int g_stride, int g_off, const bf16 *mask, int m_stride, int m_off,
                                    int C, long long V, bf16 *out)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= V) return;
    const float *gv = g + v * g_stride + g_off;
    for (int c = 0; c < C; c += 8) {
        const float4 a = *reinterpret_cast<const float4 *>(gv + c);
        const float4 b = *reinterpret_cast<const float4 *>(gv + c + 4);
        float val[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        if (mask) {
            const uint4 m = *reinterpret_cast<const uint4 *>(mask + v * m_stride + m_off + c);
            const __nv_bfloat16 *mh = reinterpret_cast<const __nv_bfloat16 *>(&m);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (!(__bfloat162float(mh[j]) > 0.f)) val[j] = 0.f;
        }
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(val[2 * j], val[2 * j + 1]);
            pk[j] = *reinterpret_cast<const uint32_t *>(&h2);
        }
        *reinterpret_cast<uint4 *>(out + v * C + c) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// Kernels over the voxels of a volume N x D x H x W: blockIdx.y (strided by
// gridDim.y) walks the rows (n, z, y), threads the row's voxels x times
// channel groups of 8 (BF16) or 4 (FP32).

// 2x2x2 max pooling of a strided BF16 view into a dense output; arg = index
// of the first maximum in octant order ox + 2 oy + 4 oz.  Coarse rows.
__global__ void maxpool_kernel(const bf16 *in, int in_stride, int in_off, int N, int D, int H, int W, int C, bf16 *out,
                               uint8_t *arg)
{
    const int d2 = D / 2, h2 = H / 2, w2 = W / 2, ng = C / 8;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= w2 * ng) return;
    const int x = t / ng, c = (t - x * ng) * 8;
    const int rows = N * d2 * h2;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int y = row % h2, q = row / h2, z = q % d2, n = q / d2;
        float best[8];
        uint32_t bi[8];
        for (int o = 0; o < 8; ++o) {
            const int zz = 2 * z + (o >> 2), yy = 2 * y + ((o >> 1) & 1), xx = 2 * x + (o & 1);
            const uint4 u = *reinterpret_cast<const uint4 *>(
                in + ((((long long)n * D + zz) * H + yy) * W + xx) * in_stride + in_off + c);
            const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&u);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float val = __bfloat162float(h[j]);
                if (o == 0 || val > best[j]) { best[j] = val; bi[j] = (uint32_t)o; }
            }
        }
        const long long ov = (long long)row * w2 + x;
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __nv_bfloat162 h2v = __floats2bfloat162_rn(best[2 * j], best[2 * j + 1]);
            pk[j] = *reinterpret_cast<const uint32_t *>(&h2v);
        }
        *reinterpret_cast<uint4 *>(out + ov * C + c) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint2 *>(arg + ov * C + c) =
            make_uint2(bi[0] | bi[1] << 8 | bi[2] << 16 | bi[3] << 24, bi[4] | bi[5] << 8 | bi[6] << 16 | bi[7] << 24);
    }
}

// g_in[argmax] += g_out (FP32; g_in strided view of the fine grid).  Coarse
// rows; the 8 voxels of an octant belong to one coarse voxel, so no two
// threads write one element.
__global__ void maxpool_bwd_kernel(const float *g_out, const uint8_t *arg, int N, int D, int H, int W, int C, float *g_in,
                                   int in_stride, int in_off)
{
    const int d2 = D / 2, h2 = H / 2, w2 = W / 2, ng = C / 8;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= w2 * ng) return;
    const int x = t / ng, c = (t - x * ng) * 8;
    const int rows = N * d2 * h2;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int y = row % h2, q = row / h2, z = q % d2, n = q / d2;
        const long long ov = (long long)row * w2 + x;
        const uint2 a = *reinterpret_cast<const uint2 *>(arg + ov * C + c);
        const float4 g0 = *reinterpret_cast<const float4 *>(g_out + ov * C + c);
        const float4 g1 = *reinterpret_cast<const float4 *>(g_out + ov * C + c + 4);
        const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int o = (int)(((j < 4 ? a.x : a.y) >> (8 * (j & 3))) & 0xFFu);
            const int zz = 2 * z + (o >> 2), yy = 2 * y + ((o >> 1) & 1), xx = 2 * x + (o & 1);
            g_in[((((long long)n * D + zz) * H + yy) * W + xx) * in_stride + in_off + c + j] += gv[j];
        }
    }
}

// Nearest 2x upsampling of a dense coarse BF16 tensor into a strided fine
// view.  Fine rows.
__global__ void upsample_kernel(const bf16 *in, int N, int d2, int h2, int w2, int C, bf16 *out, int out_stride, int out_off)
{
    const int D = 2 * d2, H = 2 * h2, W = 2 * w2, ng = C / 8;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W * ng) return;
    const int x = t / ng, c = (t - x * ng) * 8;
    const int rows = N * D * H;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int y = row % H, q = row / H, z = q % D, n = q / D;
        const uint4 u = *reinterpret_cast<const uint4 *>(
            in + ((((long long)n * d2 + z / 2) * h2 + y / 2) * w2 + x / 2) * C + c);
        *reinterpret_cast<uint4 *>(out + ((long long)row * W + x) * out_stride + out_off + c) = u;
    }
}

// g_in[coarse] = sum over the 8 fine voxels, in octant order, of g_out
// (strided FP32 view).  Coarse rows, 4 channels per thread.
__global__ void upsample_bwd_kernel(const float *g_out, int out_stride, int out_off, int N, int d2, int h2, int w2, int C,
                                    float *g_in)
{
    const int D = 2 * d2, H = 2 * h2, W = 2 * w2, ng = C / 4;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= w2 * ng) return;
    const int x = t / ng, c = (t - x * ng) * 4;
    const int rows = N * d2 * h2;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int y = row % h2, q = row / h2, z = q % d2, n = q / d2;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int o = 0; o < 8; ++o) {
            const int zz = 2 * z + (o >> 2), yy = 2 * y + ((o >> 1) & 1), xx = 2 * x + (o & 1);
            const float4 g = *reinterpret_cast<const float4 *>(
                g_out + ((((long long)n * D + zz) * H + yy) * W + xx) * out_stride + out_off + c);
            s.x += g.x; s.y += g.y; s.z += g.z; s.w += g.w;
        }
        *reinterpret_cast<float4 *>(g_in + ((long long)row * w2 + x) * C + c) = s;
    }
}

// Network input: x16[v][0..n_in-1] = bf16(in[v][0..n_in-1]), the other
// channels of the 16 zero; one voxel per thread.
__global__ void input_kernel(const float *in, long long V, int n_in, bf16 *x16)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= V) return;
    float val[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) val[c] = c < n_in ? in[v * n_in + c] : 0.f;
    uint32_t pk[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(val[2 * j], val[2 * j + 1]);
        pk[j] = *reinterpret_cast<const uint32_t *>(&h2);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(x16 + v * 16);
    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

// Prediction = head channel 0; MSE loss and its gradient into head channel 0.
// loss_part[blockIdx.x] = the block's share of the loss (sum_loss_kernel
// adds the shares in order).
__global__ void mse_kernel(const float *head, const float *target, long long V, float *pred, float *ghead,
                           double *loss_part)
{
    __shared__ double part[256];
    double s = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const float p = head[v * 16];
        if (pred) pred[v] = p;
        if (target) {
            const float d = p - target[v];
            s += (double)d * d;
            if (ghead) ghead[v * 16] = 2.0f * d / (float)V;
        }
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss_part && target) loss_part[blockIdx.x] = part[0] / (double)V;
}

// loss = sum of the blocks' shares: thread t takes k = t, t + 256, ... in
// order, then a fixed tree (one block of 256 threads).
__global__ void sum_loss_kernel(const double *loss_part, int n, double *loss)
{
    __shared__ double s_sum[256];
    double t = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) t += loss_part[k];
    s_sum[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_sum[threadIdx.x] += s_sum[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = s_sum[0];
}

// Adam on FP32 master weights; writes the BF16 copy used by the kernels.
__global__ void adam_kernel(float *w, float *m, float *v, const float *g, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2, bf16 *w16)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (w16) w16[i] = __float2bfloat16_rn(wi);
    }
}

// y[i] = fma(a, x[i], y[i]): one rounding per element (the mean of an
// ensemble's predictions, summed member by member in a fixed order).
__global__ void scale_add_kernel(float *y, const float *x, long long n, float a)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __fmaf_rn(a, x[i], y[i]);
}

__global__ void to_bf16_kernel(const float *src, long long n, bf16 *dst)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

// Seeding transform of the learned temperature seed, in FP64 per cell.
// Features (nf = 2 or 3 per cell), each standardised and then clipped to
// [-6, 6] (rare cells far outside the training distribution, e.g. next to
// a source, would otherwise dominate the first layer):
//   x[c][0] = (ln clamp(T, 2.7, 3000) - norm[0]) / norm[1],
//   x[c][1] = (ln max(rho, 1e-30) - norm[2]) / norm[3],
//   x[c][2] = (ln clamp(T) - ln clamp(T_prev) - norm[4]) / norm[5]  (nf = 3).
constexpr double kFeatureClip = 6.0;

__device__ __forceinline__ float clip_feature(double v)
{
    return (float)fmin(fmax(v, -kFeatureClip), kFeatureClip);
}

__global__ void seed_features_kernel(const float *T, const float *T_prev, const float *T_prev2, const float *rho,
                                     long long n, int nf, const SeedNorm nm, float *x)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double lt = log(fmin(fmax((double)T[c], kTMin), kTMax));
        const double r = fmax((double)rho[c], 1e-30);
        x[nf * c] = clip_feature((lt - nm.v[0]) / nm.v[1]);
        x[nf * c + 1] = clip_feature((log(r) - nm.v[2]) / nm.v[3]);
        if (nf >= 3) {
            const double lp = log(fmin(fmax((double)T_prev[c], kTMin), kTMax));
            x[nf * c + 2] = clip_feature((lt - lp - nm.v[4]) / nm.v[5]);
            if (nf == 4) {
                const double lpp = log(fmin(fmax((double)T_prev2[c], kTMin), kTMax));
                x[nf * c + 3] = clip_feature((lp - lpp - nm.v[6]) / nm.v[7]);
            }
        }
    }
}

// T_seed = clamp(T1 exp(y), 2.7, 3000) with y = shrink (pred y_std + y_mean)
// (the network predicts the normalised ln T - ln T1), bounded by the
// envelope of its bin of ln T1 when the map has one.
__global__ void seed_transform_kernel(const float *T1, const float *pred, long long n, const soc_seed_map m,
                                      float *T_seed)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double t1 = (double)T1[c];
        double y = m.shrink * ((double)pred[c] * m.y_std + m.y_mean);
        if (m.n_bins > 0) {
            const double lt = log(fmin(fmax(t1, kTMin), kTMax));
            int b = (int)floor((lt - m.lnT1_lo) / (m.lnT1_hi - m.lnT1_lo) * m.n_bins);
            b = b < 0 ? 0 : (b >= m.n_bins ? m.n_bins - 1 : b);
            y = fmin(fmax(y, m.y_lo[b]), m.y_hi[b]);
        }
        T_seed[c] = (float)fmin(fmax(t1 * exp(y), kTMin), kTMax);
    }
}

inline int grid_1d(long long n, int block = 256)
{
    long long g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

// One thread per element (no grid-stride loop)
inline unsigned grid_all(long long n, int block = 256) { return (unsigned)((n + block - 1) / block); }

// Grid of the row kernels: threads over row_threads, blockIdx.y over the
// rows, at most about 8 blocks per SM's worth in all (the kernels stride by
// gridDim.y, so each block takes several rows)
inline dim3 grid_rows(int row_threads, long long rows)
{
    const long long gx = (row_threads + 127) / 128;
    long long gy = std::max(1LL, 1216 / gx);
    gy = std::min(gy, std::max(1LL, rows));
    return dim3((unsigned)gx, (unsigned)gy);
}


// Output channels per block of the tensor-core convolution: a multiple of
// 16 dividing C_out, at most 256, narrowed (down to 16) while the blocks
// would cover fewer than half the SMs (narrow tiles re-read A, so they only
// pay on the smallest grids).
inline int tc_n_tile(int Cout, long long v_tiles, int sms)
{
    int t = 256;
    while (t > 16 && (t > Cout || Cout % t)) t -= 16;
    while (t > 16 && 2 * v_tiles * (Cout / t) < (long long)sms) {
        int u = t - 16;
        while (u > 16 && Cout % u) u -= 16;
        t = u;
    }
    return t;
}

// cuTensorMapEncodeTiled from the driver, looked up once (no link against
// libcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// The TMA-fed convolution: tensor maps over the input view (channels,
// W, H, D, N; channels c0 .. c0 + KC of a voxel, voxel stride in_stride) and
// the weights ([Cout][27 Cin]), boxes of KC channels x the output box and
// KC x n_tile, the swizzle of KC * 2-byte rows.
template <int KC>
cudaError_t tma_launch(const ConvArgs &a, cudaStream_t s)
{
    auto encode = encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    const uintptr_t in_addr = reinterpret_cast<uintptr_t>(a.in + a.in_off);
    if ((in_addr & 15u) || (a.in_stride % 8) || (reinterpret_cast<uintptr_t>(a.w) & 15u)) return cudaErrorInvalidValue;
    int dev = 0, sms = 148, sm_smem = 0, blk_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&blk_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    TmaConvArgs t{};
    t.N = a.N; t.D = a.D; t.H = a.H; t.W = a.W; t.Cin = a.Cin; t.Cout = a.Cout;
    t.bx = std::min(a.W, 128);
    t.by = std::min(a.H, 128 / t.bx);
    t.bz = std::min(a.D, 128 / (t.bx * t.by));
    t.bn = std::min(a.N, 128 / (t.bx * t.by * t.bz));
    t.tiles_x = (a.W + t.bx - 1) / t.bx;
    t.tiles_y = (a.H + t.by - 1) / t.by;
    t.tiles_z = (a.D + t.bz - 1) / t.bz;
    const long long tiles = (long long)t.tiles_x * t.tiles_y * t.tiles_z * ((a.N + t.bn - 1) / t.bn);
    t.o = ConvOut{a.out, a.out_f32, a.bias, a.out_stride, a.out_off, a.relu, a.accumulate};
    const int n_tile = tc_n_tile(a.Cout, tiles, sms);
    constexpr CUtensorMapSwizzle sw = KC == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                                    : (KC == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
    CUtensorMap map_in, map_w;
    {
        const cuuint64_t dims[5] = {(cuuint64_t)a.Cin, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.D,
                                    (cuuint64_t)a.N};
        const cuuint64_t vb = (cuuint64_t)a.in_stride * 2;
        const cuuint64_t strides[4] = {vb, vb * a.W, vb * a.W * a.H, vb * a.W * a.H * a.D};
        const cuuint32_t box[5] = {(cuuint32_t)KC, (cuuint32_t)t.bx, (cuuint32_t)t.by, (cuuint32_t)t.bz,
                                   (cuuint32_t)t.bn};
        const cuuint32_t es[5] = {1, 1, 1, 1, 1};
        if (encode(&map_in, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, reinterpret_cast<void *>(in_addr), dims, strides, box,
                   es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)27 * a.Cin, (cuuint64_t)a.Cout};
        const cuuint64_t strides[1] = {(cuuint64_t)27 * a.Cin * 2};
        const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)n_tile};
        const cuuint32_t es[2] = {1, 1};
        if (encode(&map_w, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(a.w), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    // two accumulators of n_tile columns
    uint32_t cols = 32;
    while ((int)cols < 2 * n_tile) cols <<= 1;
    if (cols > 512) return cudaErrorInvalidValue;
    // blocks per SM: at most what 512 columns of tensor memory hold, and 8;
    // the rest of the SM's shared memory split among them as stages, 2 to 8
    const int per_sm = std::min(8, std::min(512 / (int)cols, 2048 / kConvThreads));
    const int stage_bytes = (128 + n_tile) * KC * 2;
    const int fixed = 1024 + 8 * (2 * 8 + 5) + 8;     // alignment, barriers, slot and flag
    int stages = (sm_smem / per_sm - 1024 - fixed) / stage_bytes;
    stages = stages < 2 ? 2 : (stages > 8 ? 8 : stages);
    const int need = 1024 + stages * stage_bytes + 8 * (2 * stages + 5) + 8;
    if (need > blk_max) return cudaErrorInvalidValue;
    // padded so that no more than per_sm blocks are resident on an SM
    const int pad = sm_smem / (per_sm + 1) + 1024;
    int bytes = need > pad ? need : pad;
    if (bytes > blk_max) bytes = blk_max;
    cudaError_t e = cudaFuncSetAttribute(conv3d_tma_kernel<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    // all of the SM's unified memory as shared memory, so that per_sm blocks fit
    e = cudaFuncSetAttribute(conv3d_tma_kernel<KC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // blocks an SM holds, from the kernel's registers (the runtime's occupancy
    // query answers 1 for any kernel that allocates tensor memory); more
    // blocks than the SMs hold only run later, each still walking its boxes
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, conv3d_tma_kernel<KC>);
    if (e != cudaSuccess) return e;
    const int warp_regs = ((fa.numRegs + 7) / 8) * 8 * 32;
    const int reg_blocks = 65536 / (warp_regs * (kConvThreads / 32));
    const int occ = std::max(1, std::min(per_sm, reg_blocks));
    const int grid_y = a.Cout / n_tile;
    // persistent: each block walks boxes gridDim.x apart
    const long long slots = std::max(1LL, (long long)sms * occ / grid_y);
    dim3 grid((unsigned)std::min(tiles, slots), (unsigned)grid_y);
    conv3d_tma_kernel<KC><<<grid, kConvThreads, bytes, s>>>(map_in, map_w, t, n_tile, cols, stages);
    return cudaGetLastError();
}

// Plan of the slab-fed kernel, or false where it does not apply (rows that
// do not divide 128 voxels, a 128-voxel group taller than the volume,
// channel counts not multiples of 16).  Output boxes are tried from the most
// input reuse down (4, then 2, then 1 groups of 128 voxels) and taken with
// the widest channel tile that still gives every SM a block; K chunks of 32
// or 16 channels, 32 where two blocks still fit an SM.
struct SlabPlan {
    int kc, by, bz, gyn, n_acc, n_tile, stages, slab_bytes, stage_bytes, bytes, per_sm;
};

bool slab_plan(const ConvArgs &a, int sms, int sm_smem, int blk_max, SlabPlan &p)
{
    if (a.W < 8 || 128 % a.W || a.Cin % 16 || a.Cout % 16 || a.in_stride % 8) return false;
    const int g = 128 / a.W;
    if (g > a.H) return false;
    static const int cand[6][2] = {{2, 2}, {4, 1}, {1, 4}, {1, 2}, {2, 1}, {1, 1}};
    const int fixed = 1024 + 8 * (2 * 8 + 5) + 8;
    for (const auto &c : cand) {
        const int gyn = c[0], bz = c[1], by = gyn * g, n_acc = gyn * bz;
        if ((gyn > 1 && by > a.H) || (bz > 1 && bz > a.D)) continue;
        const long long boxes = (long long)((a.H + by - 1) / by) * ((a.D + bz - 1) / bz) * a.N;
        int n_tile = 256 / n_acc;
        while (n_tile > 16 && a.Cout % n_tile) n_tile -= 16;
        while (n_tile > 16 && boxes * (a.Cout / n_tile) < sms) {
            int u = n_tile - 16;
            while (u > 16 && a.Cout % u) u -= 16;
            n_tile = u;
        }
        if (a.Cout % n_tile || boxes * (a.Cout / n_tile) < sms) continue;
        uint32_t cols = 32;
        while ((int)cols < 2 * n_acc * n_tile) cols <<= 1;
        if (cols > 512) continue;
        bool found = false;
        for (int kc = 32; kc >= 16; kc >>= 1) {
            if (a.Cin % kc) continue;
            const int rows_s = a.W * (by + 2) * (bz + 2);
            const int slab = (rows_s * kc * 2 + 1023) / 1024 * 1024;
            const int stage = (slab + 9 * n_tile * kc * 2 + 1023) / 1024 * 1024;
            if (2 * stage + fixed > blk_max) continue;
            const int per_sm = std::min(std::min(512 / (int)cols, 2048 / kConvThreads),
                                        sm_smem / (2 * stage + fixed + 1024));
            if (per_sm < 1) continue;
            if (!found || (p.per_sm < 2 && per_sm >= 2)) {
                p = SlabPlan{kc, by, bz, gyn, n_acc, n_tile, 0, slab, stage, 0, per_sm};
                found = true;
            }
            if (per_sm >= 2) break;
        }
        if (!found) continue;
        int stages = (sm_smem / p.per_sm - 1024 - fixed) / p.stage_bytes;
        p.stages = stages < 2 ? 2 : (stages > 8 ? 8 : stages);
        const int need = 1024 + p.stages * p.stage_bytes + 8 * (2 * p.stages + 5) + 8;
        const int pad = sm_smem / (p.per_sm + 1) + 1024;
        p.bytes = std::min(std::max(need, pad), blk_max);
        return need <= blk_max;
    }
    return false;
}

template <int KC, int NACC>
cudaError_t slab_launch(const ConvArgs &a, const SlabPlan &p, int sms, cudaStream_t s)
{
    auto encode = encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    const uintptr_t in_addr = reinterpret_cast<uintptr_t>(a.in + a.in_off);
    if ((in_addr & 15u) || (reinterpret_cast<uintptr_t>(a.w) & 15u)) return cudaErrorInvalidValue;
    SlabArgs t{};
    t.N = a.N; t.D = a.D; t.H = a.H; t.W = a.W; t.Cin = a.Cin; t.Cout = a.Cout;
    t.by = p.by; t.bz = p.bz; t.g = 128 / a.W; t.gyn = p.gyn; t.n_acc = p.n_acc;
    t.tiles_y = (a.H + p.by - 1) / p.by;
    t.tiles_z = (a.D + p.bz - 1) / p.bz;
    t.o = ConvOut{a.out, a.out_f32, a.bias, a.out_stride, a.out_off, a.relu, a.accumulate};
    constexpr CUtensorMapSwizzle sw = KC == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                                    : (KC == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
    CUtensorMap map_in, map_w;
    {
        const cuuint64_t dims[5] = {(cuuint64_t)a.Cin, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.D,
                                    (cuuint64_t)a.N};
        const cuuint64_t vb = (cuuint64_t)a.in_stride * 2;
        const cuuint64_t strides[4] = {vb, vb * a.W, vb * a.W * a.H, vb * a.W * a.H * a.D};
        const cuuint32_t box[5] = {(cuuint32_t)KC, (cuuint32_t)a.W, 1, 1, 1};       // one row of the slab
        const cuuint32_t es[5] = {1, 1, 1, 1, 1};
        if (encode(&map_in, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, reinterpret_cast<void *>(in_addr), dims, strides, box,
                   es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)27 * a.Cin, (cuuint64_t)a.Cout};
        const cuuint64_t strides[1] = {(cuuint64_t)27 * a.Cin * 2};
        const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)p.n_tile};
        const cuuint32_t es[2] = {1, 1};
        if (encode(&map_w, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(a.w), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    uint32_t cols = 32;
    while ((int)cols < 2 * p.n_acc * p.n_tile) cols <<= 1;
    cudaError_t e = cudaFuncSetAttribute(conv3d_slab_kernel<KC, NACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(conv3d_slab_kernel<KC, NACC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, conv3d_slab_kernel<KC, NACC>);
    if (e != cudaSuccess) return e;
    const int warp_regs = ((fa.numRegs + 7) / 8) * 8 * 32;
    const int occ = std::max(1, std::min(p.per_sm, 65536 / (warp_regs * (kConvThreads / 32))));
    const int grid_y = a.Cout / p.n_tile;
    const long long n_boxes = (long long)t.tiles_y * t.tiles_z * a.N;
    const long long slots = std::max(1LL, (long long)sms * occ / grid_y);
    dim3 grid((unsigned)std::min(n_boxes, slots), (unsigned)grid_y);
    conv3d_slab_kernel<KC, NACC><<<grid, kConvThreads, p.bytes, s>>>(map_in, map_w, t, p.n_tile, cols, p.stages,
                                                               p.slab_bytes, p.stage_bytes);
    return cudaGetLastError();
}

// The slab-fed kernel where its plan applies, else the per-tap kernel with K
// chunks of 64, 32 or 16 input channels (the largest dividing C_in).
cudaError_t conv_launch(const ConvArgs &a, cudaStream_t s)
{
    int dev = 0, sms = 148, sm_smem = 0, blk_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&blk_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    SlabPlan p{};
    if (slab_plan(a, sms, sm_smem, blk_max, p)) {
        if (p.kc == 32)
            return p.n_acc == 4 ? slab_launch<32, 4>(a, p, sms, s)
                                : (p.n_acc == 2 ? slab_launch<32, 2>(a, p, sms, s) : slab_launch<32, 1>(a, p, sms, s));
        return p.n_acc == 4 ? slab_launch<16, 4>(a, p, sms, s)
                            : (p.n_acc == 2 ? slab_launch<16, 2>(a, p, sms, s) : slab_launch<16, 1>(a, p, sms, s));
    }
    if (a.Cin % 64 == 0) return tma_launch<64>(a, s);
    if (a.Cin % 32 == 0) return tma_launch<32>(a, s);
    return tma_launch<16>(a, s);
}

// Launch plan of the weight gradient: tiles and the split of the voxels into
// `chunks` blocks along x (about 4 blocks per SM).
struct WgradPlan {
    int ci_tile = 0, n_tile = 0, tap_groups = 0;
    long long per = 0, chunks = 0;
};

// Stages of a weight-gradient block and blocks per SM: as many stages as
// leave room for two blocks (3 to 8), so that every block of the grid is
// resident at once.
inline void wgrad_stages(int n_tile, int sm_smem, int *stages, int *per_sm)
{
    const int stage_bytes = (128 + n_tile) * kWgKV * 2;
    int st = (sm_smem / 2 - 2048) / stage_bytes;
    st = st < 3 ? 3 : (st > 8 ? 8 : st);
    *stages = st;
    *per_sm = std::max(1, sm_smem / (st * stage_bytes + 8 * st + 16 + 1024));
}

inline WgradPlan wgrad_plan(long long V, int Cin, int Cout, int sms, int sm_smem = 233472)
{
    WgradPlan p;
    // input-channel tile: 16, 32, 64 or 128 (dividing C_in), 128 / tile taps
    // per block; output-channel tile: a multiple of 16, at most 128
    p.ci_tile = 128;
    while (p.ci_tile > 16 && Cin % p.ci_tile) p.ci_tile >>= 1;
    p.n_tile = 128;          // at most 128: three stages of kWgKV voxels fit a block
    while (p.n_tile > 16 && (p.n_tile > Cout || Cout % p.n_tile)) p.n_tile -= 16;
    const int TT = 128 / p.ci_tile;
    p.tap_groups = (27 + TT - 1) / TT;
    const long long tiles = (long long)p.tap_groups * (Cin / p.ci_tile) * (Cout / p.n_tile);
    // one wave: the voxels split into as many chunks as the SMs hold blocks
    // of every tile
    int stages = 0, per_sm = 0;
    wgrad_stages(p.n_tile, sm_smem, &stages, &per_sm);
    long long chunks = std::max(1LL, (long long)per_sm * sms / tiles);
    long long per = (V + chunks - 1) / chunks;
    per = (per + kWgKV - 1) / kWgKV * kWgKV;
    if (per < kWgKV) per = kWgKV;
    p.per = per;
    p.chunks = (V + per - 1) / per;
    return p;
}

inline int device_sms()
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Floats of partial sums a weight gradient of this shape needs.
inline long long wgrad_part_floats(long long V, int Cin, int Cout, int sms)
{
    int dev = 0, sm_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    return wgrad_plan(V, Cin, Cout, sms, sm_smem).chunks * Cout * 27LL * Cin;
}

// gw[Cout][27][Cin] += sum_v gy[v] x[v + tap]: partial sums per voxel chunk
// into part (part_floats available), then their ordered sum into gw.
cudaError_t wgrad_launch(const WgradArgs &a0, float *gw, long long part_floats, cudaStream_t s)
{
    WgradArgs a = a0;
    const long long V = (long long)a.N * a.D * a.H * a.W;
    int dev = 0, sm_smem = 0, blk_max = 0;
    cudaGetDevice(&dev);
    const int sms = device_sms();
    cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&blk_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const WgradPlan p = wgrad_plan(V, a.Cin, a.Cout, sms, sm_smem);
    if (a.Cin % p.ci_tile) return cudaErrorInvalidValue;
    const long long n_w = (long long)a.Cout * 27 * a.Cin;
    if (p.chunks * n_w > part_floats) return cudaErrorInvalidValue;
    a.vox_per_block = p.per;
    uint32_t cols = 32;
    while ((int)cols < p.n_tile) cols <<= 1;
    const int stage_bytes = (128 + p.n_tile) * kWgKV * 2;
    int stages = 0, per_sm = 0;
    wgrad_stages(p.n_tile, sm_smem, &stages, &per_sm);
    const int need = stages * stage_bytes + 8 * stages + 16;
    const int max_blocks = 512 / (int)cols;
    const int pad = sm_smem / (max_blocks + 1) + 1024;
    int bytes = need > pad ? need : pad;
    if (need > blk_max) return cudaErrorInvalidValue;
    if (bytes > blk_max) bytes = blk_max;
    cudaError_t e = cudaFuncSetAttribute(conv3d_wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)p.chunks, (unsigned)p.tap_groups, (unsigned)((a.Cin / p.ci_tile) * (a.Cout / p.n_tile)));
    conv3d_wgrad_tc_kernel<<<grid, kWgThreads, bytes, s>>>(a, p.ci_tile, p.n_tile, cols, stages);
    reduce_partials_kernel<<<grid_1d(n_w), 256, 0, s>>>(a.part, (int)p.chunks, n_w, gw);
    return cudaGetLastError();
}

// Voxels per block of the bias gradient: 16 per voxel lane of its 256 threads
inline long long bias_vox(int C) { return 16LL * (256 / (C < 1 ? 1 : C)); }

inline long long bias_part_floats(long long V, int C) { return (V + bias_vox(C) - 1) / bias_vox(C) * C; }

// gb[C] += sum_v gy[v]: per-block sums into part, then their sum in a fixed
// order.
cudaError_t bias_grad_launch(const bf16 *gy, int C, long long V, float *gb, float *part, long long part_floats,
                             cudaStream_t s)
{
    if (C < 1 || C > 256) return cudaErrorInvalidValue;
    const long long blocks = (V + bias_vox(C) - 1) / bias_vox(C);
    if (blocks * C > part_floats || blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
    bias_grad_kernel<<<(unsigned)blocks, 256, 0, s>>>(gy, C, V, bias_vox(C), part);
    bias_reduce_kernel<<<C, 256, 0, s>>>(part, (int)blocks, C, gb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The U-Net
// ---------------------------------------------------------------------------
constexpr int kLayers = 15;
struct LayerSpec { int cin, cout, relu; };
constexpr LayerSpec kSpec[kLayers] = {
    {16, 16, 1}, {16, 16, 1}, {16, 32, 1}, {32, 32, 1}, {32, 64, 1}, {64, 64, 1}, {64, 128, 1}, {128, 128, 1},
    {192, 64, 1}, {64, 64, 1}, {96, 32, 1}, {32, 32, 1}, {48, 16, 1}, {16, 16, 1}, {16, 16, 0}};

template <class T>
struct Buf {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count)
    {
        n = count;
        return cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    }
    void release() { if (p) cudaFree(p); p = nullptr; n = 0; }
};

struct Net {
    int device = 0;
    int batch = 0, S = 0, n_in = 2;              // n_in: real input channels (of the 16)
    long long V0 = 0, V1 = 0, V2 = 0, V3 = 0;     // voxels per level (all samples)
    // parameters
    Buf<float> w32[kLayers], b32[kLayers], gw[kLayers], gb[kLayers], mw[kLayers], vw[kLayers], mb[kLayers], vb[kLayers];
    Buf<bf16> w16[kLayers], wt[kLayers];
    long long adam_t = 0;
    // activations (BF16)
    Buf<bf16> x16, e0a, cat0, p0, e1a, cat1, p1, e2a, cat2, p2, b_a, b_b, d2a, d2b, d1a, d1b, d0a, d0b;
    Buf<uint8_t> arg0, arg1, arg2;
    Buf<float> head;
    // gradients (FP32) and a BF16 staging buffer
    Buf<float> g_head, g_d0b, g_d0a, g_cat0, g_d1b, g_d1a, g_cat1, g_d2b, g_d2a, g_cat2, g_bb, g_ba, g_p2, g_e2a, g_p1,
        g_e1a, g_p0, g_e0a;
    Buf<bf16> gstage;
    Buf<double> loss, loss_part;
    Buf<float> part;              // per-block partial sums of the weight and bias gradients

    template <class F>
    void each(F f)
    {
        for (int l = 0; l < kLayers; ++l) {
            f(w32[l]); f(b32[l]); f(gw[l]); f(gb[l]); f(mw[l]); f(vw[l]); f(mb[l]); f(vb[l]);
        }
        f(head); f(g_head); f(g_d0b); f(g_d0a); f(g_cat0); f(g_d1b); f(g_d1a); f(g_cat1); f(g_d2b); f(g_d2a);
        f(g_cat2); f(g_bb); f(g_ba); f(g_p2); f(g_e2a); f(g_p1); f(g_e1a); f(g_p0); f(g_e0a); f(part);
    }
    template <class F>
    void each16(F f)
    {
        for (int l = 0; l < kLayers; ++l) { f(w16[l]); f(wt[l]); }
        f(x16); f(e0a); f(cat0); f(p0); f(e1a); f(cat1); f(p1); f(e2a); f(cat2); f(p2); f(b_a); f(b_b); f(d2a);
        f(d2b); f(d1a); f(d1b); f(d0a); f(d0b); f(gstage);
    }
    void release()
    {
        each([](Buf<float> &b) { b.release(); });
        each16([](Buf<bf16> &b) { b.release(); });
        arg0.release(); arg1.release(); arg2.release(); loss.release(); loss_part.release();
    }
};

}  // namespace nn

cudaError_t launch_seed_features(const float *T, const float *T_prev, const float *T_prev2, const float *rho,
                                 int64_t n, int n_features, const double *norm, float *x, cudaStream_t s)
{
    SeedNorm nm{};
    for (int k = 0; k < 2 * n_features; ++k) nm.v[k] = norm[k];
    nn::seed_features_kernel<<<nn::grid_1d(n), 256, 0, s>>>(T, T_prev, T_prev2, rho, n, n_features, nm, x);
    return cudaGetLastError();
}

cudaError_t launch_seed_transform(const float *T1, const float *pred, int64_t n, const soc_seed_map &map,
                                  float *T_seed, cudaStream_t s)
{
    nn::seed_transform_kernel<<<nn::grid_1d(n), 256, 0, s>>>(T1, pred, n, map, T_seed);
    return cudaGetLastError();
}

}  // namespace soc

using namespace soc::nn;

namespace {

// Networks by id.  The table is shared by all host threads; the mutex guards
// its entries (a network itself is used by one thread at a time).
struct NetRegistry {
    std::mutex m;
    std::vector<Net *> nets;
};
NetRegistry g_nets;

Net *net_of(int id)
{
    Net *n = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_nets.m);
        if (id < 0 || id >= (int)g_nets.nets.size() || !g_nets.nets[id]) return nullptr;
        n = g_nets.nets[id];
    }
    if (cudaSetDevice(n->device) != cudaSuccess) return nullptr;
    return n;
}

#define NNCK(expr)                                        \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return SOC_ERR_CUDA;       \
    } while (0)

ConvArgs conv_args(const bf16 *in, int in_stride, int in_off, const bf16 *w, const float *bias, int N, int S, int Cin,
                   int Cout, int relu)
{
    ConvArgs a;
    memset(&a, 0, sizeof a);
    a.in = in; a.in_stride = in_stride; a.in_off = in_off; a.w = w; a.bias = bias;
    a.N = N; a.D = S; a.H = S; a.W = S; a.Cin = Cin; a.Cout = Cout; a.relu = relu;
    return a;
}

// forward of one layer into a BF16 view
soc_status fwd(Net &n, int l, const bf16 *in, int in_stride, int in_off, int S, bf16 *out, int out_stride, int out_off,
               cudaStream_t s)
{
    ConvArgs a = conv_args(in, in_stride, in_off, n.w16[l].p, n.b32[l].p, n.batch, S, kSpec[l].cin, kSpec[l].cout,
                           kSpec[l].relu);
    a.out = out; a.out_stride = out_stride; a.out_off = out_off;
    NNCK(conv_launch(a, s));
    return SOC_OK;
}

// backward of one layer: gy (FP32 view, masked by the layer's output y when it
// has a ReLU) -> gw, gb, and (if gx) gx (FP32 view, accumulate or overwrite)
soc_status bwd(Net &n, int l, const float *gy, int gy_stride, int gy_off, const bf16 *y, int y_stride, int y_off,
               const bf16 *x, int x_stride, int x_off, int S, float *gx, int gx_stride, int gx_off, int accumulate,
               cudaStream_t s)
{
    const int Cin = kSpec[l].cin, Cout = kSpec[l].cout;
    const long long V = (long long)n.batch * S * S * S;
    mask_to_bf16_kernel<<<grid_all(V), 256, 0, s>>>(gy, gy_stride, gy_off, kSpec[l].relu ? y : nullptr, y_stride,
                                                         y_off, Cout, V, n.gstage.p);
    NNCK(cudaGetLastError());
    WgradArgs wa;
    memset(&wa, 0, sizeof wa);
    wa.gy = n.gstage.p; wa.gy_stride = Cout; wa.gy_off = 0; wa.x = x; wa.x_stride = x_stride; wa.x_off = x_off;
    wa.part = n.part.p; wa.N = n.batch; wa.D = S; wa.H = S; wa.W = S; wa.Cin = Cin; wa.Cout = Cout;
    NNCK(wgrad_launch(wa, n.gw[l].p, (long long)n.part.n, s));
    NNCK(bias_grad_launch(n.gstage.p, Cout, V, n.gb[l].p, n.part.p, (long long)n.part.n, s));
    if (gx) {
        ConvArgs a = conv_args(n.gstage.p, Cout, 0, n.wt[l].p, nullptr, n.batch, S, Cout, Cin, 0);
        a.out_f32 = gx; a.out_stride = gx_stride; a.out_off = gx_off; a.accumulate = accumulate;
        NNCK(conv_launch(a, s));
    }
    return SOC_OK;
}

soc_status forward(Net &n, const float *d_in, cudaStream_t s)
{
    const int S0 = n.S, S1 = S0 / 2, S2 = S0 / 4, S3 = S0 / 8;
    soc_status st;
    input_kernel<<<grid_all(n.V0), 256, 0, s>>>(d_in, n.V0, n.n_in, n.x16.p);
    NNCK(cudaGetLastError());
    if ((st = fwd(n, 0, n.x16.p, 16, 0, S0, n.e0a.p, 16, 0, s))) return st;
    if ((st = fwd(n, 1, n.e0a.p, 16, 0, S0, n.cat0.p, 48, 32, s))) return st;
    maxpool_kernel<<<grid_rows(S1 * 2, (long long)n.batch * S1 * S1), 128, 0, s>>>(n.cat0.p, 48, 32, n.batch, S0, S0, S0, 16, n.p0.p, n.arg0.p);
    if ((st = fwd(n, 2, n.p0.p, 16, 0, S1, n.e1a.p, 32, 0, s))) return st;
    if ((st = fwd(n, 3, n.e1a.p, 32, 0, S1, n.cat1.p, 96, 64, s))) return st;
    maxpool_kernel<<<grid_rows(S2 * 4, (long long)n.batch * S2 * S2), 128, 0, s>>>(n.cat1.p, 96, 64, n.batch, S1, S1, S1, 32, n.p1.p, n.arg1.p);
    if ((st = fwd(n, 4, n.p1.p, 32, 0, S2, n.e2a.p, 64, 0, s))) return st;
    if ((st = fwd(n, 5, n.e2a.p, 64, 0, S2, n.cat2.p, 192, 128, s))) return st;
    maxpool_kernel<<<grid_rows(S3 * 8, (long long)n.batch * S3 * S3), 128, 0, s>>>(n.cat2.p, 192, 128, n.batch, S2, S2, S2, 64, n.p2.p, n.arg2.p);
    if ((st = fwd(n, 6, n.p2.p, 64, 0, S3, n.b_a.p, 128, 0, s))) return st;
    if ((st = fwd(n, 7, n.b_a.p, 128, 0, S3, n.b_b.p, 128, 0, s))) return st;
    upsample_kernel<<<grid_rows(S2 * 16, (long long)n.batch * S2 * S2), 128, 0, s>>>(n.b_b.p, n.batch, S3, S3, S3, 128, n.cat2.p, 192, 0);
    if ((st = fwd(n, 8, n.cat2.p, 192, 0, S2, n.d2a.p, 64, 0, s))) return st;
    if ((st = fwd(n, 9, n.d2a.p, 64, 0, S2, n.d2b.p, 64, 0, s))) return st;
    upsample_kernel<<<grid_rows(S1 * 8, (long long)n.batch * S1 * S1), 128, 0, s>>>(n.d2b.p, n.batch, S2, S2, S2, 64, n.cat1.p, 96, 0);
    if ((st = fwd(n, 10, n.cat1.p, 96, 0, S1, n.d1a.p, 32, 0, s))) return st;
    if ((st = fwd(n, 11, n.d1a.p, 32, 0, S1, n.d1b.p, 32, 0, s))) return st;
    upsample_kernel<<<grid_rows(S0 * 4, (long long)n.batch * S0 * S0), 128, 0, s>>>(n.d1b.p, n.batch, S1, S1, S1, 32, n.cat0.p, 48, 0);
    if ((st = fwd(n, 12, n.cat0.p, 48, 0, S0, n.d0a.p, 16, 0, s))) return st;
    if ((st = fwd(n, 13, n.d0a.p, 16, 0, S0, n.d0b.p, 16, 0, s))) return st;
    ConvArgs a = conv_args(n.d0b.p, 16, 0, n.w16[14].p, n.b32[14].p, n.batch, S0, 16, 16, 0);
    a.out_f32 = n.head.p; a.out_stride = 16; a.out_off = 0;
    NNCK(conv_launch(a, s));
    return SOC_OK;
}

soc_status backward(Net &n, const float *d_target, cudaStream_t s)
{
    const int S0 = n.S, S1 = S0 / 2, S2 = S0 / 4, S3 = S0 / 8;
    soc_status st;
    for (int l = 0; l < kLayers; ++l) {
        NNCK(cudaMemsetAsync(n.gw[l].p, 0, n.gw[l].n * 4, s));
        NNCK(cudaMemsetAsync(n.gb[l].p, 0, n.gb[l].n * 4, s));
        flip_weights_kernel<<<grid_1d((long long)kSpec[l].cout * 27 * kSpec[l].cin), 256, 0, s>>>(
            n.w16[l].p, kSpec[l].cout, kSpec[l].cin, n.wt[l].p);
    }
    NNCK(cudaMemsetAsync(n.g_head.p, 0, n.g_head.n * 4, s));
    mse_kernel<<<grid_1d(n.V0), 256, 0, s>>>(n.head.p, d_target, n.V0, nullptr, n.g_head.p, n.loss_part.p);
    sum_loss_kernel<<<1, 256, 0, s>>>(n.loss_part.p, grid_1d(n.V0), n.loss.p);
    NNCK(cudaGetLastError());
    // decoder level 0
    if ((st = bwd(n, 14, n.g_head.p, 16, 0, nullptr, 0, 0, n.d0b.p, 16, 0, S0, n.g_d0b.p, 16, 0, 0, s))) return st;
    if ((st = bwd(n, 13, n.g_d0b.p, 16, 0, n.d0b.p, 16, 0, n.d0a.p, 16, 0, S0, n.g_d0a.p, 16, 0, 0, s))) return st;
    if ((st = bwd(n, 12, n.g_d0a.p, 16, 0, n.d0a.p, 16, 0, n.cat0.p, 48, 0, S0, n.g_cat0.p, 48, 0, 0, s))) return st;
    upsample_bwd_kernel<<<grid_rows(S1 * 8, (long long)n.batch * S1 * S1), 128, 0, s>>>(n.g_cat0.p, 48, 0, n.batch, S1, S1, S1, 32, n.g_d1b.p);
    // decoder level 1
    if ((st = bwd(n, 11, n.g_d1b.p, 32, 0, n.d1b.p, 32, 0, n.d1a.p, 32, 0, S1, n.g_d1a.p, 32, 0, 0, s))) return st;
    if ((st = bwd(n, 10, n.g_d1a.p, 32, 0, n.d1a.p, 32, 0, n.cat1.p, 96, 0, S1, n.g_cat1.p, 96, 0, 0, s))) return st;
    upsample_bwd_kernel<<<grid_rows(S2 * 16, (long long)n.batch * S2 * S2), 128, 0, s>>>(n.g_cat1.p, 96, 0, n.batch, S2, S2, S2, 64, n.g_d2b.p);
    // decoder level 2
    if ((st = bwd(n, 9, n.g_d2b.p, 64, 0, n.d2b.p, 64, 0, n.d2a.p, 64, 0, S2, n.g_d2a.p, 64, 0, 0, s))) return st;
    if ((st = bwd(n, 8, n.g_d2a.p, 64, 0, n.d2a.p, 64, 0, n.cat2.p, 192, 0, S2, n.g_cat2.p, 192, 0, 0, s))) return st;
    upsample_bwd_kernel<<<grid_rows(S3 * 32, (long long)n.batch * S3 * S3), 128, 0, s>>>(n.g_cat2.p, 192, 0, n.batch, S3, S3, S3, 128, n.g_bb.p);
    // bottleneck
    if ((st = bwd(n, 7, n.g_bb.p, 128, 0, n.b_b.p, 128, 0, n.b_a.p, 128, 0, S3, n.g_ba.p, 128, 0, 0, s))) return st;
    if ((st = bwd(n, 6, n.g_ba.p, 128, 0, n.b_a.p, 128, 0, n.p2.p, 64, 0, S3, n.g_p2.p, 64, 0, 0, s))) return st;
    maxpool_bwd_kernel<<<grid_rows(S3 * 8, (long long)n.batch * S3 * S3), 128, 0, s>>>(n.g_p2.p, n.arg2.p, n.batch, S2, S2, S2, 64, n.g_cat2.p, 192,
                                                          128);
    // encoder level 2 (its output is the skip slice of cat2)
    if ((st = bwd(n, 5, n.g_cat2.p, 192, 128, n.cat2.p, 192, 128, n.e2a.p, 64, 0, S2, n.g_e2a.p, 64, 0, 0, s))) return st;
    if ((st = bwd(n, 4, n.g_e2a.p, 64, 0, n.e2a.p, 64, 0, n.p1.p, 32, 0, S2, n.g_p1.p, 32, 0, 0, s))) return st;
    maxpool_bwd_kernel<<<grid_rows(S2 * 4, (long long)n.batch * S2 * S2), 128, 0, s>>>(n.g_p1.p, n.arg1.p, n.batch, S1, S1, S1, 32, n.g_cat1.p, 96, 64);
    if ((st = bwd(n, 3, n.g_cat1.p, 96, 64, n.cat1.p, 96, 64, n.e1a.p, 32, 0, S1, n.g_e1a.p, 32, 0, 0, s))) return st;
    if ((st = bwd(n, 2, n.g_e1a.p, 32, 0, n.e1a.p, 32, 0, n.p0.p, 16, 0, S1, n.g_p0.p, 16, 0, 0, s))) return st;
    maxpool_bwd_kernel<<<grid_rows(S1 * 2, (long long)n.batch * S1 * S1), 128, 0, s>>>(n.g_p0.p, n.arg0.p, n.batch, S0, S0, S0, 16, n.g_cat0.p, 48, 32);
    if ((st = bwd(n, 1, n.g_cat0.p, 48, 32, n.cat0.p, 48, 32, n.e0a.p, 16, 0, S0, n.g_e0a.p, 16, 0, 0, s))) return st;
    if ((st = bwd(n, 0, n.g_e0a.p, 16, 0, n.e0a.p, 16, 0, n.x16.p, 16, 0, S0, nullptr, 0, 0, 0, s))) return st;
    NNCK(cudaGetLastError());
    return SOC_OK;
}

}  // namespace

extern "C" {

soc_status soc_unet_create(int device, int batch, int side, int n_inputs, int *net_id)
{
    if (!net_id || batch < 1 || side < 8 || side % 8 != 0 || n_inputs < 1 || n_inputs > 16) return SOC_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return SOC_ERR_CUDA;
    Net *n = new (std::nothrow) Net();
    if (!n) return SOC_ERR_NOMEM;
    n->device = device;
    n->batch = batch;
    n->S = side;
    n->n_in = n_inputs;
    n->V0 = (long long)batch * side * side * side;
    n->V1 = n->V0 / 8; n->V2 = n->V1 / 8; n->V3 = n->V2 / 8;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto &b, size_t cnt) { if (e == cudaSuccess) e = b.alloc(cnt); };
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = (size_t)kSpec[l].cout * 27 * kSpec[l].cin, nb = kSpec[l].cout;
        A(n->w32[l], nw); A(n->gw[l], nw); A(n->mw[l], nw); A(n->vw[l], nw); A(n->w16[l], nw); A(n->wt[l], nw);
        A(n->b32[l], nb); A(n->gb[l], nb); A(n->mb[l], nb); A(n->vb[l], nb);
    }
    A(n->x16, n->V0 * 16); A(n->e0a, n->V0 * 16); A(n->cat0, n->V0 * 48); A(n->p0, n->V1 * 16);
    A(n->e1a, n->V1 * 32); A(n->cat1, n->V1 * 96); A(n->p1, n->V2 * 32); A(n->e2a, n->V2 * 64);
    A(n->cat2, n->V2 * 192); A(n->p2, n->V3 * 64); A(n->b_a, n->V3 * 128); A(n->b_b, n->V3 * 128);
    A(n->d2a, n->V2 * 64); A(n->d2b, n->V2 * 64); A(n->d1a, n->V1 * 32); A(n->d1b, n->V1 * 32);
    A(n->d0a, n->V0 * 16); A(n->d0b, n->V0 * 16); A(n->head, n->V0 * 16);
    A(n->arg0, n->V1 * 16); A(n->arg1, n->V2 * 32); A(n->arg2, n->V3 * 64);
    A(n->g_head, n->V0 * 16); A(n->g_d0b, n->V0 * 16); A(n->g_d0a, n->V0 * 16); A(n->g_cat0, n->V0 * 48);
    A(n->g_d1b, n->V1 * 32); A(n->g_d1a, n->V1 * 32); A(n->g_cat1, n->V1 * 96); A(n->g_d2b, n->V2 * 64);
    A(n->g_d2a, n->V2 * 64); A(n->g_cat2, n->V2 * 192); A(n->g_bb, n->V3 * 128); A(n->g_ba, n->V3 * 128);
    A(n->g_p2, n->V3 * 64); A(n->g_e2a, n->V2 * 64); A(n->g_p1, n->V2 * 32); A(n->g_e1a, n->V1 * 32);
    A(n->g_p0, n->V1 * 16); A(n->g_e0a, n->V0 * 16); A(n->gstage, n->V0 * 48); A(n->loss, 1);
    A(n->loss_part, (size_t)grid_1d(n->V0));
    {   // partial sums: the largest weight (or bias) gradient of any layer
        const int sms = device_sms();
        long long need = 0;
        for (int l = 0; l < kLayers; ++l) {
            const int lev = l < 2 ? 0 : l < 4 ? 1 : l < 6 ? 2 : l < 8 ? 3 : l < 10 ? 2 : l < 12 ? 1 : 0;
            const long long V = n->V0 >> (3 * lev);
            need = std::max(need, wgrad_part_floats(V, kSpec[l].cin, kSpec[l].cout, sms));
            need = std::max(need, bias_part_floats(V, kSpec[l].cout));
        }
        A(n->part, (size_t)need);
    }
    if (e != cudaSuccess) { n->release(); delete n; return SOC_ERR_NOMEM; }
    for (int l = 0; l < kLayers; ++l) {
        cudaMemset(n->mw[l].p, 0, n->mw[l].n * 4); cudaMemset(n->vw[l].p, 0, n->vw[l].n * 4);
        cudaMemset(n->mb[l].p, 0, n->mb[l].n * 4); cudaMemset(n->vb[l].p, 0, n->vb[l].n * 4);
        cudaMemset(n->w32[l].p, 0, n->w32[l].n * 4); cudaMemset(n->b32[l].p, 0, n->b32[l].n * 4);
        cudaMemset(n->w16[l].p, 0, n->w16[l].n * 2);
    }
    try {                                  // no exception crosses the C ABI
        std::lock_guard<std::mutex> lock(g_nets.m);
        g_nets.nets.push_back(n);
        *net_id = (int)g_nets.nets.size() - 1;
    } catch (...) {
        n->release();
        delete n;
        return SOC_ERR_NOMEM;
    }
    return SOC_OK;
}

soc_status soc_unet_destroy(int net_id)
{
    Net *n = net_of(net_id);
    if (!n) return SOC_ERR_ARG;
    {
        std::lock_guard<std::mutex> lock(g_nets.m);
        g_nets.nets[net_id] = nullptr;
    }
    cudaDeviceSynchronize();
    n->release();
    delete n;
    return SOC_OK;
}

int64_t soc_unet_param_count(void)
{
    int64_t c = 0;
    for (int l = 0; l < kLayers; ++l) c += (int64_t)kSpec[l].cout * 27 * kSpec[l].cin + kSpec[l].cout;
    return c;
}

soc_status soc_unet_set_params(int net_id, const float *host)
{
    Net *n = net_of(net_id);
    if (!n || !host) return SOC_ERR_ARG;
    const float *p = host;
    for (int l = 0; l < kLayers; ++l) {
        NNCK(cudaMemcpy(n->w32[l].p, p, n->w32[l].n * 4, cudaMemcpyHostToDevice));
        p += n->w32[l].n;
        NNCK(cudaMemcpy(n->b32[l].p, p, n->b32[l].n * 4, cudaMemcpyHostToDevice));
        p += n->b32[l].n;
        to_bf16_kernel<<<grid_1d((long long)n->w32[l].n), 256>>>(n->w32[l].p, (long long)n->w32[l].n, n->w16[l].p);
        NNCK(cudaGetLastError());
    }
    NNCK(cudaDeviceSynchronize());
    n->adam_t = 0;
    return SOC_OK;
}

soc_status soc_unet_get_params(int net_id, float *host, int grads)
{
    Net *n = net_of(net_id);
    if (!n || !host) return SOC_ERR_ARG;
    NNCK(cudaDeviceSynchronize());
    float *p = host;
    for (int l = 0; l < kLayers; ++l) {
        NNCK(cudaMemcpy(p, grads ? n->gw[l].p : n->w32[l].p, n->w32[l].n * 4, cudaMemcpyDeviceToHost));
        p += n->w32[l].n;
        NNCK(cudaMemcpy(p, grads ? n->gb[l].p : n->b32[l].p, n->b32[l].n * 4, cudaMemcpyDeviceToHost));
        p += n->b32[l].n;
    }
    return SOC_OK;
}

soc_status soc_unet_forward(int net_id, const float *d_input, float *d_pred, void *stream)
{
    Net *n = net_of(net_id);
    if (!n || !d_input || !d_pred) return SOC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    soc_status st = forward(*n, d_input, s);
    if (st) return st;
    mse_kernel<<<grid_1d(n->V0), 256, 0, s>>>(n->head.p, nullptr, n->V0, d_pred, nullptr, nullptr);
    NNCK(cudaGetLastError());
    return SOC_OK;
}

soc_status soc_unet_backward(int net_id, const float *d_input, const float *d_target, float *d_pred, double *d_loss,
                             void *stream)
{
    Net *n = net_of(net_id);
    if (!n || !d_input || !d_target) return SOC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    soc_status st = forward(*n, d_input, s);
    if (st) return st;
    if (d_pred) {
        mse_kernel<<<grid_1d(n->V0), 256, 0, s>>>(n->head.p, nullptr, n->V0, d_pred, nullptr, nullptr);
        NNCK(cudaGetLastError());
    }
    if ((st = backward(*n, d_target, s))) return st;
    if (d_loss) NNCK(cudaMemcpyAsync(d_loss, n->loss.p, 8, cudaMemcpyDeviceToDevice, s));
    return SOC_OK;
}

soc_status soc_unet_adam(int net_id, float lr, void *stream)
{
    Net *n = net_of(net_id);
    if (!n || !(lr >= 0.f)) return SOC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    n->adam_t += 1;
    // bias corrections 1 - beta^t in double (in FP32, 1 - 0.999^t cancels:
    // 7e-6 relative error at t = 2), then rounded once
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)n->adam_t));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)n->adam_t));
    for (int l = 0; l < kLayers; ++l) {
        adam_kernel<<<grid_1d((long long)n->w32[l].n), 256, 0, s>>>(n->w32[l].p, n->mw[l].p, n->vw[l].p, n->gw[l].p,
                                                                   (long long)n->w32[l].n, lr, b1, b2, eps, c1, c2,
                                                                   n->w16[l].p);
        adam_kernel<<<grid_1d((long long)n->b32[l].n), 256, 0, s>>>(n->b32[l].p, n->mb[l].p, n->vb[l].p, n->gb[l].p,
                                                                   (long long)n->b32[l].n, lr, b1, b2, eps, c1, c2,
                                                                   nullptr);
    }
    NNCK(cudaGetLastError());
    return SOC_OK;
}

// --- single-operation entry points (for parity tests and reuse) -----------
soc_status soc_nn_error_flag(int *flag)
{
    if (!flag) return SOC_ERR_ARG;
    int zero = 0;
    if (cudaMemcpyFromSymbol(flag, g_tc_error, sizeof(int)) != cudaSuccess) return SOC_ERR_CUDA;
    if (cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int)) != cudaSuccess) return SOC_ERR_CUDA;
    return SOC_OK;
}

soc_status soc_nn_conv3d(const void *x, int N, int D, int H, int W, int Cin, const void *w, const float *bias, int Cout,
                         int relu, void *y_bf16, float *y_f32, void *stream)
{
    if (!x || !w || (!y_bf16 && !y_f32) || Cin % 16 || Cout % 16 || N < 1 || D < 1 || H < 1 || W < 1) return SOC_ERR_ARG;
    ConvArgs a;
    memset(&a, 0, sizeof a);
    a.in = (const bf16 *)x; a.in_stride = Cin; a.w = (const bf16 *)w; a.bias = bias;
    a.out = (bf16 *)y_bf16; a.out_f32 = y_f32; a.out_stride = Cout;
    a.N = N; a.D = D; a.H = H; a.W = W; a.Cin = Cin; a.Cout = Cout; a.relu = relu;
    NNCK(conv_launch(a, (cudaStream_t)stream));
    return SOC_OK;
}

soc_status soc_nn_conv3d_dgrad(const void *gy, int N, int D, int H, int W, int Cout, const void *w, int Cin, void *w_scratch,
                               float *gx, void *stream)
{
    if (!gy || !w || !w_scratch || !gx || Cin % 16 || Cout % 16) return SOC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    flip_weights_kernel<<<grid_1d((long long)Cout * 27 * Cin), 256, 0, s>>>((const bf16 *)w, Cout, Cin, (bf16 *)w_scratch);
    NNCK(cudaGetLastError());
    ConvArgs a;
    memset(&a, 0, sizeof a);
    a.in = (const bf16 *)gy; a.in_stride = Cout; a.w = (const bf16 *)w_scratch;
    a.out_f32 = gx; a.out_stride = Cin; a.N = N; a.D = D; a.H = H; a.W = W; a.Cin = Cout; a.Cout = Cin;
    NNCK(conv_launch(a, s));
    return SOC_OK;
}

soc_status soc_nn_conv3d_wgrad(const void *gy, const void *x, int N, int D, int H, int W, int Cin, int Cout, float *gw,
                               float *gb, void *stream)
{
    if (!gy || !x || !gw || Cin % 16 || Cout % 16 || N < 1 || D < 1 || H < 1 || W < 1) return SOC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const long long V = (long long)N * D * H * W;
    const long long need = std::max(wgrad_part_floats(V, Cin, Cout, device_sms()), bias_part_floats(V, Cout));
    // partial sums in a library-owned workspace of this device (grown on
    // demand; calls on one device share it and are ordered by the caller)
    static std::mutex ws_mutex;
    static std::vector<Buf<float>> ws;
    std::lock_guard<std::mutex> lock(ws_mutex);
    int dev = 0;
    NNCK(cudaGetDevice(&dev));
    try {
        if ((int)ws.size() <= dev) ws.resize(dev + 1);
    } catch (...) {
        return SOC_ERR_NOMEM;
    }
    Buf<float> &w = ws[dev];
    if ((long long)w.n < need) {
        NNCK(cudaStreamSynchronize(s));          // the old workspace may still be in use on this stream
        w.release();
        if (w.alloc((size_t)need) != cudaSuccess) { w.p = nullptr; w.n = 0; return SOC_ERR_NOMEM; }
    }
    WgradArgs wa;
    memset(&wa, 0, sizeof wa);
    wa.gy = (const bf16 *)gy; wa.gy_stride = Cout; wa.x = (const bf16 *)x; wa.x_stride = Cin; wa.part = w.p;
    wa.N = N; wa.D = D; wa.H = H; wa.W = W; wa.Cin = Cin; wa.Cout = Cout;
    NNCK(wgrad_launch(wa, gw, (long long)w.n, s));
    if (gb) NNCK(bias_grad_launch((const bf16 *)gy, Cout, V, gb, w.p, (long long)w.n, s));
    return SOC_OK;
}

soc_status soc_nn_seed_features(const float *d_T, const float *d_T_prev, const float *d_T_prev2, const float *d_rho,
                                int64_t n, const double *norm, int n_features, float *d_x, void *stream)
{
    if (!d_T || !d_rho || !norm || !d_x || n < 1 || n_features < 2 || n_features > 4 ||
        (n_features >= 3 && !d_T_prev) || (n_features == 4 && !d_T_prev2))
        return SOC_ERR_ARG;
    for (int k = 1; k < 2 * n_features; k += 2)
        if (!(norm[k] > 0.0)) return SOC_ERR_ARG;
    NNCK(soc::launch_seed_features(d_T, d_T_prev, d_T_prev2, d_rho, n, n_features, norm, d_x, (cudaStream_t)stream));
    return SOC_OK;
}

soc_status soc_nn_adam(float *d_w, float *d_m, float *d_v, const float *d_g, int64_t n, float lr, int32_t t,
                       void *d_w_bf16, void *stream)
{
    if (!d_w || !d_m || !d_v || !d_g || n < 1 || t < 1 || !(lr >= 0.f)) return SOC_ERR_ARG;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)t));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)t));
    adam_kernel<<<grid_1d(n), 256, 0, (cudaStream_t)stream>>>(d_w, d_m, d_v, d_g, n, lr, b1, b2, eps, c1, c2,
                                                              (bf16 *)d_w_bf16);
    NNCK(cudaGetLastError());
    return SOC_OK;
}

soc_status soc_nn_scale_add(float *d_y, const float *d_x, int64_t n, float a, void *stream)
{
    if (!d_y || !d_x || n < 1 || !(a == a)) return SOC_ERR_ARG;
    scale_add_kernel<<<grid_1d(n), 256, 0, (cudaStream_t)stream>>>(d_y, d_x, n, a);
    NNCK(cudaGetLastError());
    return SOC_OK;
}

}  // extern "C"
