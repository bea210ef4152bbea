// ocmc_unet_tc.cu -- 3x3x3 convolutions of the denoiser on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory, operands staged by TMA).
//
// Output tile: 8 (x) x 16 (y) x TZ (z) voxels. For one z-slice the 128 voxels are the M = 128
// rows of an MMA (row m = x + 8 y). The block loads, per 16-channel input chunk, the halo
// of its tile, 10 x 18 x (TZ + 2) voxels, as two planes of 8 channels (16 bytes per voxel) in
// the order z, y, x: TMA writes exactly that from a 5-D view of the channels-last activation
// (8 channels, channel group, x, y, z) and zero-fills outside the grid, which is the
// convolution's padding. Because every halo row of 10 voxels is contiguous, the A operand of
// tap (dx, dy, dz) for slice s is a no-swizzle K-major matrix starting at halo voxel
// (dx, dy, s + dz): 8 rows 16 bytes apart (x), next 8-row group 160 bytes on (y), second
// 8 channels one plane on (K). No data is copied per tap.
// Output channels are split into slices of NSL (NSL = cout for up to 32 input channels; 32 or
// 16 for the 64- and 128-channel layers, whose whole weights would not fit): blockIdx.y is the
// slice, and the slice's weights stay in shared memory for the whole kernel, packed [tap]
// [channel group][out channel][8 channels] so that B (N = NSL out channels, K = 16 input
// channels) is K-major too. Each (tap, z-slice) is one MMA of M = 128, N = NSL, K = 16,
// accumulating in FP32 in tensor memory; two accumulator sets let the epilogue of one tile
// overlap the MMAs of the next. Blocks of different channel slices read the same halo tiles,
// which L2 serves.
// With 16 or 32 output channels per slice the kernel stacks the z-taps instead: the window of
// halo plane zi at shift (dx, dy) feeds output slices zi - 2, zi - 1 and zi through z-taps 2, 1
// and 0, so one MMA of N = 3 NSL (weights packed [dx, dy][channel group][dz = 2, 1, 0][out
// channel][8]) writes three consecutive slices of an accumulator set that carries two spare
// slices at each end. The tensor core's operand reads from shared memory, which bound the
// one-tap form at these widths, drop by 1.4-2x.
//
// Warp roles of the 3x3x3 kernel (192 threads): warp 0 issues the TMA copies, warp 1 owns tensor memory and one of
// its lanes issues the MMAs, warps 2-5 read the accumulators (each warp its 32-lane quarter of
// tensor memory), add bias / previous value, apply ReLU and mask, and store BF16. Every wait
// gives up after two seconds, sets the error flag, lets its copies in flight land and frees
// tensor memory before the block exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "ocmc_umma.cuh"
#include "ocmc_unet_kernels.cuh"
#include "ocmc_unet_tc.h"

namespace ocmc {
namespace unet {
namespace {

using namespace ocmc::umma;

constexpr int TX = 8, TY = 16, HX = TX + 2, HY = TY + 2;
constexpr int TC_THREADS = 192;
constexpr uint64_t WAIT_NS = 2000000000ull;

// test hook of the bounded waits (process-wide; off by default)
int g_stall_tile = -1;
uint64_t g_stall_ns = 0;

struct TcArgs {
    Grid3 g;
    Grid3 gfine;                 // UP: the fine output grid; DOWN: the fine input grid
    Slice out;
    const __nv_bfloat16* wpack;
    const float* bias;
    int relu, accumulate;
    const __nv_bfloat16* mask;
    int mask_stride, mask_c0;
    int tiles_x, tiles_y, ntiles;
    int* err;
    // test hook: at its block-local tile number stall_tile (>= 0) the MMA thread waits stall_ns
    // on a barrier that nothing completes, so that this wait runs out like a real timeout
    int stall_tile;
    uint64_t stall_ns;
};

template <int CIN, int NSL, int TZ, int NS_>
struct Cfg {
    static constexpr int NS = NS_;                                       // halo stages
    static constexpr int G = CIN / 8;
    static constexpr int CHUNKS = CIN / 16;
    // z-stacked taps for 16- and 32-channel slices: the three z-taps of one (dx, dy) are the
    // N = 3 NSL columns of one MMA (see the kernel), so that each A window is read once instead
    // of three times; an accumulator set then spans TZ + 4 slices (two spare slices at each end),
    // which for NSL = 32 fits tensor memory twice only with TZ <= 4
    static constexpr bool ZS = NSL == 16 || (NSL == 32 && TZ <= 4);
    static constexpr int ASLICES = ZS ? TZ + 4 : TZ;                     // slices per accumulator set
    static constexpr uint32_t W_BYTES = 27u * CIN * NSL * 2;             // one channel slice
    static constexpr uint32_t PLANE = (uint32_t)(TZ + 2) * HY * HX * 16;
    static constexpr uint32_t STAGE = 2 * PLANE;
    static constexpr uint32_t BAR_OFF = W_BYTES + NS * STAGE;
    static constexpr uint32_t BIAS_OFF = BAR_OFF + 256;
    static constexpr uint32_t ZERO_OFF = (BIAS_OFF + NSL * 4 + 127) / 128 * 128;
    static constexpr uint32_t ZERO_BYTES = ZS ? 2u * ASLICES * NSL * 16 : 0u;   // zero B operand, both K halves
    static constexpr uint32_t SMEM = ZERO_OFF + ZERO_BYTES;
    static constexpr uint32_t COLS = 2 * ASLICES * NSL;
    static constexpr uint32_t NCOLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
    static_assert(COLS <= 512, "tensor memory holds 512 columns");
    static_assert(CIN % 16 == 0 && NSL % 16 == 0 && NSL <= 256, "MMA shape");
    static_assert(W_BYTES % 128 == 0 && PLANE % 128 == 0, "TMA destinations 128-byte aligned");
    static_assert(SMEM <= 232448, "shared memory per block");
    static_assert(!ZS || ASLICES * NSL <= 256, "the zeroing MMA covers a whole accumulator set");
};

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity)
{
    int dummy = 0;
    return mbar_wait(bar, parity, &dummy, WAIT_NS);
}

template <int CIN, int NSL, int TZ, int NS_>
__global__ void __launch_bounds__(TC_THREADS, 1) k_conv3_tc(const __grid_constant__ CUtensorMap tmap, const TcArgs a)
{
    using C = Cfg<CIN, NSL, TZ, NS_>;
    constexpr int NS = C::NS;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sw = smem;
    uint8_t* sh = smem + C::W_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
    uint64_t* w_full = bars;
    uint64_t* h_full = bars + 1;
    uint64_t* h_empty = bars + 1 + NS;
    uint64_t* t_full = bars + 1 + 2 * NS;
    uint64_t* t_empty = bars + 3 + 2 * NS;
    uint64_t* drain = bars + 5 + 2 * NS;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 6 + 2 * NS);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* sbias = reinterpret_cast<float*>(smem + C::BIAS_OFF);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.y * NSL;                  // this block's output channels n0 .. n0 + NSL - 1
    for (int i = threadIdx.x; i < NSL; i += TC_THREADS) sbias[i] = a.bias ? a.bias[n0 + i] : 0.f;
    if constexpr (C::ZS)
        for (uint32_t i = threadIdx.x; i < C::ZERO_BYTES / 16; i += TC_THREADS)
            reinterpret_cast<uint4*>(smem + C::ZERO_OFF)[i] = make_uint4(0u, 0u, 0u, 0u);

    if (threadIdx.x == 0) {
        mbar_init(w_full, 1);
        for (int i = 0; i < NS; ++i) {
            mbar_init(&h_full[i], 1);
            mbar_init(&h_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&t_full[i], 1);
            mbar_init(&t_empty[i], 4);
        }
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, C::NCOLS);
    if constexpr (C::ZS) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- producer: weights once, then one halo chunk per (tile, chunk) ----
        if (lane == 0) {
            mbar_expect_tx(w_full, C::W_BYTES);
            const uint8_t* wsrc = reinterpret_cast<const uint8_t*>(a.wpack) + (size_t)blockIdx.y * C::W_BYTES;
            for (uint32_t off = 0; off < C::W_BYTES; off += 32768u)
                bulk_load(sw + off, wsrc + off, min(32768u, C::W_BYTES - off), w_full);
            int it = 0;
            int last[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) last[i] = -1;
            for (int tile = blockIdx.x; tile < a.ntiles && !*abort; tile += gridDim.x) {
                const int tx = tile % a.tiles_x, r = tile / a.tiles_x;
                const int x0 = tx * TX, y0 = (r % a.tiles_y) * TY, z0 = (r / a.tiles_y) * TZ;
                for (int c = 0; c < C::CHUNKS; ++c, ++it) {
                    const int st = it % NS, u = it / NS;
                    if (!mbar_wait(&h_empty[st], (u & 1) ^ 1, abort, WAIT_NS)) break;
                    uint8_t* dst = sh + st * C::STAGE;
                    mbar_expect_tx(&h_full[st], C::STAGE);
                    tma_load_5d(dst, &tmap, 0, 2 * c, x0 - 1, y0 - 1, z0 - 1, &h_full[st]);
                    tma_load_5d(dst + C::PLANE, &tmap, 0, 2 * c + 1, x0 - 1, y0 - 1, z0 - 1, &h_full[st]);
                    last[st] = u;
                }
            }
            if (*abort) {   // copies in flight must land before the block exits
                wait_bounded(w_full, 0);
                for (int i = 0; i < NS; ++i)
                    if (last[i] >= 0) wait_bounded(&h_full[i], last[i] & 1);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue ----
        if (lane == 0) {
            bool issued = false;
            if (mbar_wait(w_full, 0, abort, WAIT_NS)) {
                fence_after_sync();
                constexpr uint32_t idesc = idesc_bf16_f32(128, NSL);
                const uint32_t sw_addr = saddr(sw), sh_addr = saddr(sh);
                int it = 0, lt = 0;
                for (int tile = blockIdx.x; tile < a.ntiles && !*abort; tile += gridDim.x, ++lt) {
                    const int acc = lt & 1, ua = lt >> 1;
                    if (lt == a.stall_tile) {   // drain's phase 0 completes only in the abort path below
                        mbar_wait(drain, 0, abort, a.stall_ns);
                        break;
                    }
                    if (!mbar_wait(&t_empty[acc], (ua & 1) ^ 1, abort, WAIT_NS)) break;
                    fence_after_sync();
                    const uint32_t d0 = tmem + (uint32_t)(acc * C::ASLICES * NSL);
                    for (int c = 0; c < C::CHUNKS; ++c, ++it) {
                        const int st = it % NS, u = it / NS;
                        if (!mbar_wait(&h_full[st], u & 1, abort, WAIT_NS)) break;
                        fence_after_sync();
                        // descriptors are built once per chunk; a tap or slice only moves the start
                        // address, which is the descriptor's low field in 16-byte units
                        const uint64_t a0 = sdesc(sh_addr + (uint32_t)st * C::STAGE, C::PLANE, HX * 16);
                        if constexpr (C::ZS) {
                            // Input z-plane zi of the halo (0 .. TZ + 1) with shift (dx, dy) feeds output
                            // slices zi - 2 + k through z-tap dz = 2 - k, k = 0, 1, 2: the weights hold the
                            // z-taps of one (dx, dy) as N blocks k (dz = 2, 1, 0), and the MMA writes
                            // accumulator slices zi .. zi + 2 of a set whose slice j is output slice j - 2.
                            // Every MMA accumulates; the set is zeroed first by an MMA with a zero B.
                            constexpr uint32_t idesc3 = idesc_bf16_f32(128, 3 * NSL);
                            if (c == 0) {
                                constexpr uint32_t idesc0 = idesc_bf16_f32(128, C::ASLICES * NSL);
                                mma_f16(d0, a0, sdesc(saddr(smem + C::ZERO_OFF), C::ASLICES * NSL * 16, 128), idesc0, 0u);
                            }
                            const uint64_t b0 = sdesc(sw_addr + (uint32_t)(2 * c) * 3 * NSL * 16, 3 * NSL * 16, 128);
#pragma unroll
                            for (int zi = 0; zi < TZ + 2; ++zi)
#pragma unroll
                                for (int t9 = 0; t9 < 9; ++t9) {
                                    const int dx = t9 % 3, dy = t9 / 3;
                                    mma_f16(d0 + (uint32_t)(zi * NSL), a0 + (uint64_t)((zi * HY + dy) * HX + dx),
                                            b0 + (uint64_t)(t9 * C::G * 3 * NSL), idesc3, 1u);
                                }
                        } else {
                            const uint64_t b0 = sdesc(sw_addr + (uint32_t)(2 * c) * NSL * 16, NSL * 16, 128);
#pragma unroll
                            for (int t = 0; t < 27; ++t) {
                                const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;
                                const uint64_t bd = b0 + (uint64_t)(t * C::G * NSL);
#pragma unroll
                                for (int s = 0; s < TZ; ++s)
                                    mma_f16(d0 + (uint32_t)(s * NSL), a0 + (uint64_t)(((s + dz) * HY + dy) * HX + dx),
                                            bd, idesc, (t != 0 || c != 0) ? 1u : 0u);
                            }
                        }
                        mma_commit(&h_empty[st]);
                        issued = true;
                    }
                    if (*abort) break;
                    mma_commit(&t_full[acc]);
                }
            }
            if (*abort && issued) {   // MMAs in flight must finish before tensor memory is freed
                mma_commit(drain);
                wait_bounded(drain, 0);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: tensor memory -> bias / accumulate / ReLU / mask -> BF16 ----
        const int q = warp & 3;                       // the tensor-memory lane quarter of this warp
        const int row = 32 * q + lane;
        int lt = 0;
        for (int tile = blockIdx.x; tile < a.ntiles && !*abort; tile += gridDim.x, ++lt) {
            const int acc = lt & 1, ua = lt >> 1;
            if (!mbar_wait(&t_full[acc], ua & 1, abort, WAIT_NS)) break;
            fence_after_sync();
            const int tx = tile % a.tiles_x, r = tile / a.tiles_x;
            const int x = tx * TX + (row & 7), y = (r % a.tiles_y) * TY + (row >> 3), z0 = (r / a.tiles_y) * TZ;
            // (with z-stacked taps output slice s is accumulator slice s + 2)
            const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * C::ASLICES * NSL) +
                                   (uint32_t)(C::ZS ? 2 * NSL : 0);
#pragma unroll 1
            for (int s = 0; s < TZ; ++s) {
                float v[NSL];
#pragma unroll
                for (int j = 0; j < NSL / 16; ++j) tmem_ld16(tbase + (uint32_t)(s * NSL + 16 * j), v + 16 * j);
                const int z = z0 + s;
                if (x < a.g.nx && y < a.g.ny && z < a.g.nz) {
                    const long long vox = x + (long long)a.g.nx * (y + (long long)a.g.ny * z);
                    __nv_bfloat16* o = a.out.ptr + vox * a.out.stride + a.out.c0 + n0;
                    const __nv_bfloat16* mk = a.mask ? a.mask + vox * a.mask_stride + a.mask_c0 + n0 : nullptr;
#pragma unroll
                    for (int j = 0; j < NSL / 8; ++j) {
                        float f[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) f[e] = v[8 * j + e] + sbias[8 * j + e];
                        if (a.accumulate) {
                            uint4 old = *reinterpret_cast<const uint4*>(o + 8 * j);
                            const __nv_bfloat162* ob = reinterpret_cast<const __nv_bfloat162*>(&old);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                float2 p = __bfloat1622float2(ob[e]);
                                f[2 * e] += p.x;
                                f[2 * e + 1] += p.y;
                            }
                        }
                        if (a.relu) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) f[e] = fmaxf(f[e], 0.f);
                        }
                        if (mk) {
                            uint4 mv = *reinterpret_cast<const uint4*>(mk + 8 * j);
                            const __nv_bfloat162* mb = reinterpret_cast<const __nv_bfloat162*>(&mv);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                float2 p = __bfloat1622float2(mb[e]);
                                if (!(p.x > 0.f)) f[2 * e] = 0.f;
                                if (!(p.y > 0.f)) f[2 * e + 1] = 0.f;
                            }
                        }
                        uint4 w;
                        __nv_bfloat162* wb2 = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
                        for (int e = 0; e < 4; ++e) wb2[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
                        *reinterpret_cast<uint4*>(o + 8 * j) = w;
                    }
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&t_empty[acc]);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, C::NCOLS);
    }
    if (threadIdx.x == 0 && *abort && a.err) atomicExch(a.err, 1);
}

// [27][K][N] (tap t = dx + 3 dy + 9 dz) -> one contiguous block per output-channel slice:
// [N / NSL][27][K/8][NSL][8], or with z-stacked taps (zs) [N / NSL][9 (dx + 3 dy)][K/8][3][NSL][8]
// with the z-taps in the order dz = 2, 1, 0
__global__ void k_pack_tc(const __nv_bfloat16* src, int K, int N, int nsl, int zs, __nv_bfloat16* dst)
{
    long long total = 27LL * K * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        int kk = (int)(i & 7);
        long long q = i >> 3;
        int nn = (int)(q % nsl);
        q /= nsl;
        int t, g, sl;
        if (zs) {
            const int k3 = (int)(q % 3);
            q /= 3;
            g = (int)(q % (K / 8));
            q /= K / 8;
            t = 9 * (2 - k3) + (int)(q % 9);
            sl = (int)(q / 9);
        } else {
            g = (int)(q % (K / 8));
            q /= K / 8;
            t = (int)(q % 27);
            sl = (int)(q / 27);
        }
        dst[i] = src[((long long)t * K + 8 * g + kk) * N + sl * nsl + nn];
    }
}

// ---- transposed 2x2x2 convolution (UP: coarse -> fine) on tcgen05 ----------------------------
// Rows are coarse voxels: a tile is 8 (x) x 16 (y) voxels of one z-plane, the M = 128 rows of
// an MMA (row m = x + 8 y), loaded by TMA as one plane of 8 channels per channel group (the same
// 5-D view as the 3x3x3 kernel's, without a halo). Columns are the eight output parities times
// the output channels, N = 8 COUT (j = p COUT + n), so one chain of CIN / 16 MMAs (two per K
// step when N = 512) gives every output of the tile; the weights [p][cin][cout] stay in shared
// memory packed [cin/8][N][8] (K-major B). Output voxel of row (x, y, z) and parity p =
// (px, py, pz): (2x + px, 2y + py, 2z + pz). The data gradient of a DOWN layer is this same
// operation with the transposed weights.
constexpr int UP_THREADS = 320;   // producer warp, MMA warp, 8 epilogue warps (two per lane quarter)

template <int CIN, int COUT>
struct UpCfg {
    static constexpr int G = CIN / 8;
    static constexpr int N = 8 * COUT;
    static constexpr int NMMA = N > 256 ? 2 : 1;                     // MMAs per K step (N <= 256 each)
    static constexpr int NACC = 2 * N <= 512 ? 2 : 1;                // accumulator sets in tensor memory
    static constexpr int NS = CIN * N * 2 > 65536 ? 2 : 4;           // input stages
    static constexpr uint32_t W_BYTES = (uint32_t)N * CIN * 2;
    static constexpr uint32_t PLANE = 128 * 16;                      // one channel group of a tile
    static constexpr uint32_t STAGE = G * PLANE;
    static constexpr uint32_t BAR_OFF = W_BYTES + NS * STAGE;
    static constexpr uint32_t BIAS_OFF = BAR_OFF + 256;
    static constexpr uint32_t SMEM = BIAS_OFF + COUT * 4;
    static constexpr uint32_t COLS = NACC * N;
    static constexpr uint32_t NCOLS = COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COLS <= 512, "UP tile shape");
    static_assert(W_BYTES % 128 == 0 && SMEM <= 232448, "shared memory per block");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(UP_THREADS, 1) k_up_tc(const __grid_constant__ CUtensorMap tmap, const TcArgs a)
{
    using C = UpCfg<CIN, COUT>;
    constexpr int NS = C::NS, N = C::N;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sw = smem;
    uint8_t* sh = smem + C::W_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
    uint64_t* w_full = bars;
    uint64_t* h_full = bars + 1;
    uint64_t* h_empty = bars + 1 + NS;
    uint64_t* t_full = bars + 1 + 2 * NS;
    uint64_t* t_empty = bars + 3 + 2 * NS;
    uint64_t* drain = bars + 5 + 2 * NS;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 6 + 2 * NS);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* sbias = reinterpret_cast<float*>(smem + C::BIAS_OFF);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < COUT; i += UP_THREADS) sbias[i] = a.bias ? a.bias[i] : 0.f;
    if (threadIdx.x == 0) {
        mbar_init(w_full, 1);
        for (int i = 0; i < NS; ++i) {
            mbar_init(&h_full[i], 1);
            mbar_init(&h_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&t_full[i], 1);
            mbar_init(&t_empty[i], 8);
        }
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, C::NCOLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- producer: weights once, then every channel group of one tile per stage ----
        if (lane == 0) {
            mbar_expect_tx(w_full, C::W_BYTES);
            const uint8_t* wsrc = reinterpret_cast<const uint8_t*>(a.wpack);
            for (uint32_t off = 0; off < C::W_BYTES; off += 32768u)
                bulk_load(sw + off, wsrc + off, min(32768u, C::W_BYTES - off), w_full);
            int it = 0;
            int last[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) last[i] = -1;
            for (int tile = blockIdx.x; tile < a.ntiles && !*abort; tile += gridDim.x, ++it) {
                const int tx = tile % a.tiles_x, r = tile / a.tiles_x;
                const int x0 = tx * TX, y0 = (r % a.tiles_y) * TY, z = r / a.tiles_y;
                const int st = it % NS, u = it / NS;
                if (!mbar_wait(&h_empty[st], (u & 1) ^ 1, abort, WAIT_NS)) break;
                uint8_t* dst = sh + st * C::STAGE;
                mbar_expect_tx(&h_full[st], C::STAGE);
                for (int g = 0; g < C::G; ++g) tma_load_5d(dst + g * C::PLANE, &tmap, 0, g, x0, y0, z, &h_full[st]);
                last[st] = u;
            }
            if (*abort) {   // copies in flight must land before the block exits
                wait_bounded(w_full, 0);
                for (int i = 0; i < NS; ++i)
                    if (last[i] >= 0) wait_bounded(&h_full[i], last[i] & 1);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue: D[128 x N] = A[128 x CIN] W[CIN x N] per tile ----
        if (lane == 0) {
            bool issued = false;
            if (mbar_wait(w_full, 0, abort, WAIT_NS)) {
                fence_after_sync();
                constexpr uint32_t idesc = idesc_bf16_f32(128, N / C::NMMA);
                const uint32_t sw_addr = saddr(sw), sh_addr = saddr(sh);
                const uint64_t b0 = sdesc(sw_addr, N * 16, 128);
                int it = 0;
                for (int tile = blockIdx.x; tile < a.ntiles && !*abort; tile += gridDim.x, ++it) {
                    const int acc = it % C::NACC, ua = it / C::NACC;
                    if (!mbar_wait(&t_empty[acc], (ua & 1) ^ 1, abort, WAIT_NS)) break;
                    fence_after_sync();
                    const int st = it % NS, u = it / NS;
                    if (!mbar_wait(&h_full[st], u & 1, abort, WAIT_NS)) break;
                    fence_after_sync();
                    const uint32_t d0 = tmem + (uint32_t)(acc * N);
                    // rows 16 bytes apart, 8-row groups 128 bytes apart, channel groups one plane apart
                    const uint64_t a0 = sdesc(sh_addr + (uint32_t)st * C::STAGE, C::PLANE, 128);
#pragma unroll
                    for (int k = 0; k < CIN / 16; ++k)
#pragma unroll
                        for (int h = 0; h < C::NMMA; ++h)
                            mma_f16(d0 + (uint32_t)(h * 256), a0 + (uint64_t)(2 * k * C::PLANE / 16),
                                    b0 + (uint64_t)((2 * k * N * 16 + h * 256 * 16) / 16), idesc, k ? 1u : 0u);
                    mma_commit(&h_empty[st]);
                    mma_commit(&t_full[acc]);
                    issued = true;
                }
            }
            if (*abort && issued) {   // MMAs in flight must finish before tensor memory is freed
                mma_commit(drain);
                wait_bounded(drain, 0);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: tensor memory -> bias / accumulate / ReLU / mask -> BF16 ----
        // warps 2-9: two per tensor-memory lane quarter, each taking four of the eight parities
        const int q = warp & 3;                       // the tensor-memory lane quarter of this warp
        const int p0 = ((warp - 2) >> 2) * 4;
        const int row = 32 * q + lane;
        int it = 0;
        for (int tile = blockIdx.x; tile < a.ntiles && !*abort; tile += gridDim.x, ++it) {
            const int acc = it % C::NACC, ua = it / C::NACC;
            if (!mbar_wait(&t_full[acc], ua & 1, abort, WAIT_NS)) break;
            fence_after_sync();
            const int tx = tile % a.tiles_x, r = tile / a.tiles_x;
            const int x = tx * TX + (row & 7), y = (r % a.tiles_y) * TY + (row >> 3), z = r / a.tiles_y;
            const bool inside = x < a.g.nx && y < a.g.ny;
            const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * N);
#pragma unroll 1
            for (int p = p0; p < p0 + 4; ++p) {
                const int ox = 2 * x + (p & 1), oy = 2 * y + ((p >> 1) & 1), oz = 2 * z + (p >> 2);
                const bool ok = inside && ox < a.gfine.nx && oy < a.gfine.ny && oz < a.gfine.nz;
                const long long vox = ox + (long long)a.gfine.nx * (oy + (long long)a.gfine.ny * oz);
#pragma unroll
                for (int j = 0; j < COUT / 16; ++j) {
                    float v[16];
                    tmem_ld16(tbase + (uint32_t)(p * COUT + 16 * j), v);   // every lane: the load is warp-wide
                    if (!ok) continue;
                    __nv_bfloat16* o = a.out.ptr + vox * a.out.stride + a.out.c0 + 16 * j;
                    const __nv_bfloat16* mk = a.mask ? a.mask + vox * a.mask_stride + a.mask_c0 + 16 * j : nullptr;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float f[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) f[e] = v[8 * h + e] + sbias[16 * j + 8 * h + e];
                        if (a.accumulate) {
                            uint4 old = *reinterpret_cast<const uint4*>(o + 8 * h);
                            const __nv_bfloat162* ob = reinterpret_cast<const __nv_bfloat162*>(&old);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                float2 t2 = __bfloat1622float2(ob[e]);
                                f[2 * e] += t2.x;
                                f[2 * e + 1] += t2.y;
                            }
                        }
                        if (a.relu) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) f[e] = fmaxf(f[e], 0.f);
                        }
                        if (mk) {
                            uint4 mv = *reinterpret_cast<const uint4*>(mk + 8 * h);
                            const __nv_bfloat162* mb = reinterpret_cast<const __nv_bfloat162*>(&mv);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                float2 t2 = __bfloat1622float2(mb[e]);
                                if (!(t2.x > 0.f)) f[2 * e] = 0.f;
                                if (!(t2.y > 0.f)) f[2 * e + 1] = 0.f;
                            }
                        }
                        uint4 w;
                        __nv_bfloat162* wb2 = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
                        for (int e = 0; e < 4; ++e) wb2[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
                        *reinterpret_cast<uint4*>(o + 8 * h) = w;
                    }
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&t_empty[acc]);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, C::NCOLS);
    }
    if (threadIdx.x == 0 && *abort && a.err) atomicExch(a.err, 1);
}

// [8][K][COUT] (parity p, input channel, output channel) -> [K/8][8 COUT][8]: K-major B with
// column j = p COUT + n
__global__ void k_pack_up_tc(const __nv_bfloat16* src, int K, int cout, __nv_bfloat16* dst)
{
    const int N = 8 * cout;
    long long total = (long long)K * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int kk = (int)(i & 7);
        const long long q = i >> 3;
        const int n = (int)(q % N), g = (int)(q / N);
        const int p = n / cout, co = n - p * cout;
        dst[i] = src[((long long)p * K + 8 * g + kk) * cout + co];
    }
}

// ---- stride-2 2x2x2 convolution (DOWN: fine -> coarse) on tcgen05 -----------------------------
// Rows are coarse output voxels, a tile of 8 (x) x 16 (y) voxels of one z-plane (row m = x + 8 y).
// Input voxel of row (x, y, z) and parity p = (px, py, pz): (2x + px, 2y + py, 2z + pz) -- every
// other voxel along each axis, which a TMA box cannot hand to a K-major descriptor, so eight
// producer warps gather them: two threads per row m load the 16-byte channel runs of the row for
// four parities each and every channel group and writes them to plane (p, g) of the stage, row m (16 bytes per
// row, 2 KB per plane), then fences them for the tensor core and arrives on the stage's barrier.
// One MMA chain of 8 CIN / 16 steps (K = parity x input channel, N = COUT) per tile; weights
// [p][cin][cout] packed [p][cin/8][cout][8] stay in shared memory. The data gradient of an UP
// layer is this same operation with the transposed weights.
constexpr int DOWN_THREADS = 416;   // MMA warp, eight producer warps, four epilogue warps

template <int CIN, int COUT>
struct DownCfg {
    static constexpr int G = CIN / 8;
    static constexpr int NS = CIN <= 16 ? 4 : 2;                     // input stages (64 KB each for 32 channels)
    static constexpr uint32_t W_BYTES = 8u * CIN * COUT * 2;
    static constexpr uint32_t PLANE = 128 * 16;
    static constexpr uint32_t STAGE = 8 * G * PLANE;                 // eight parities x channel groups
    static constexpr uint32_t BAR_OFF = W_BYTES + NS * STAGE;
    static constexpr uint32_t BIAS_OFF = BAR_OFF + 256;
    static constexpr uint32_t SMEM = BIAS_OFF + COUT * 4;
    static constexpr uint32_t COLS = 2 * COUT;
    static constexpr uint32_t NCOLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : 256;
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 128, "DOWN tile shape");
    static_assert(W_BYTES % 128 == 0 && SMEM <= 232448, "shared memory per block");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(DOWN_THREADS, 1) k_down_tc(const TcArgs a, const __nv_bfloat16* __restrict__ in,
                                                             int in_stride)
{
    using C = DownCfg<CIN, COUT>;
    constexpr int NS = C::NS, G = C::G;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sw = smem;
    uint8_t* sh = smem + C::W_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
    uint64_t* w_full = bars;
    uint64_t* h_full = bars + 1;
    uint64_t* h_empty = bars + 1 + NS;
    uint64_t* t_full = bars + 1 + 2 * NS;
    uint64_t* t_empty = bars + 3 + 2 * NS;
    uint64_t* drain = bars + 5 + 2 * NS;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 6 + 2 * NS);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* sbias = reinterpret_cast<float*>(smem + C::BIAS_OFF);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < COUT; i += DOWN_THREADS) sbias[i] = a.bias ? a.bias[i] : 0.f;
    if (threadIdx.x == 0) {
        mbar_init(w_full, 1);
        for (int i = 0; i < NS; ++i) {
            mbar_init(&h_full[i], 256);             // every producer thread arrives
            mbar_init(&h_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&t_full[i], 1);
            mbar_init(&t_empty[i], 4);
        }
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, C::NCOLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- weights, then MMA issue: D[128 x COUT] = sum over parities of A_p[128 x CIN] W_p ----
        if (lane == 0) {
            mbar_expect_tx(w_full, C::W_BYTES);
            const uint8_t* wsrc = reinterpret_cast<const uint8_t*>(a.wpack);
            for (uint32_t off = 0; off < C::W_BYTES; off += 32768u)
                bulk_load(sw + off, wsrc + off, min(32768u, C::W_BYTES - off), w_full);
            bool issued = false, weights = mbar_wait(w_full, 0, abort, WAIT_NS);
            if (weights) {
                fence_after_sync();
                constexpr uint32_t idesc = idesc_bf16_f32(128, COUT);
                const uint32_t sw_addr = saddr(sw), sh_addr = saddr(sh);
                int it = 0;
                for (int tile = blockIdx.x; tile < a.ntiles && !*abort; tile += gridDim.x, ++it) {
                    const int acc = it & 1, ua = it >> 1;
                    if (!mbar_wait(&t_empty[acc], (ua & 1) ^ 1, abort, WAIT_NS)) break;
                    fence_after_sync();
                    const int st = it % NS, u = it / NS;
                    if (!mbar_wait(&h_full[st], u & 1, abort, WAIT_NS)) break;
                    fence_after_sync();
                    const uint32_t d0 = tmem + (uint32_t)(acc * COUT);
                    const uint32_t stage = sh_addr + (uint32_t)st * C::STAGE;
#pragma unroll
                    for (int p = 0; p < 8; ++p)
#pragma unroll
                        for (int k = 0; k < CIN / 16; ++k) {
                            const uint32_t pg = (uint32_t)(p * G + 2 * k);
                            mma_f16(d0, sdesc(stage + pg * C::PLANE, C::PLANE, 128),
                                    sdesc(sw_addr + pg * COUT * 16, COUT * 16, 128), idesc, (p | k) ? 1u : 0u);
                        }
                    mma_commit(&h_empty[st]);
                    mma_commit(&t_full[acc]);
                    issued = true;
                }
            } else {
                wait_bounded(w_full, 0);               // the weight copy must land before the block exits
            }
            if (*abort && issued) {   // MMAs in flight must finish before tensor memory is freed
                mma_commit(drain);
                wait_bounded(drain, 0);
            }
        }
        __syncwarp();
    } else if (warp <= 8) {
        // ---- producers: threads m and m + 128 gather row m of the (parity, channel group) planes
        // of parities 0-3 and 4-7 ----
        const int m = (threadIdx.x - 32) & 127, p_lo = ((threadIdx.x - 32) >> 7) * 4;
        constexpr int PB = G <= 2 ? 4 : 2;           // parities per batch of loads in flight
        int it = 0;
        for (int tile = blockIdx.x; tile < a.ntiles && !*abort; tile += gridDim.x, ++it) {
            const int st = it % NS, u = it / NS;
            if (!mbar_wait(&h_empty[st], (u & 1) ^ 1, abort, WAIT_NS)) break;
            const int tx = tile % a.tiles_x, r = tile / a.tiles_x;
            const int x = tx * TX + (m & 7), y = (r % a.tiles_y) * TY + (m >> 3), z = r / a.tiles_y;
            const bool rowin = x < a.g.nx && y < a.g.ny;
            uint8_t* dst = sh + st * C::STAGE + m * 16;
#pragma unroll
            for (int p0 = p_lo; p0 < p_lo + 4; p0 += PB) {
                uint4 v[PB][G];
#pragma unroll
                for (int q = 0; q < PB; ++q) {
                    const int p = p0 + q;
                    const int ix = 2 * x + (p & 1), iy = 2 * y + ((p >> 1) & 1), iz = 2 * z + (p >> 2);
                    const bool ok = rowin && ix < a.gfine.nx && iy < a.gfine.ny && iz < a.gfine.nz;
                    const long long vox = ok ? ix + (long long)a.gfine.nx * (iy + (long long)a.gfine.ny * iz) : 0;
                    const uint4* src = reinterpret_cast<const uint4*>(in + vox * in_stride);
#pragma unroll
                    for (int g = 0; g < G; ++g) v[q][g] = ok ? __ldg(src + g) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int q = 0; q < PB; ++q)
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        *reinterpret_cast<uint4*>(dst + ((p0 + q) * G + g) * C::PLANE) = v[q][g];
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
            mbar_arrive(&h_full[st]);
        }
    } else {
        // ---- epilogue (warps 9-12): tensor memory -> bias / accumulate / ReLU / mask -> BF16 ----
        const int q = warp & 3;                       // the tensor-memory lane quarter of this warp
        const int row = 32 * q + lane;
        int it = 0;
        for (int tile = blockIdx.x; tile < a.ntiles && !*abort; tile += gridDim.x, ++it) {
            const int acc = it & 1, ua = it >> 1;
            if (!mbar_wait(&t_full[acc], ua & 1, abort, WAIT_NS)) break;
            fence_after_sync();
            const int tx = tile % a.tiles_x, r = tile / a.tiles_x;
            const int x = tx * TX + (row & 7), y = (r % a.tiles_y) * TY + (row >> 3), z = r / a.tiles_y;
            const bool ok = x < a.g.nx && y < a.g.ny;
            const long long vox = x + (long long)a.g.nx * (y + (long long)a.g.ny * z);
            const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * COUT);
#pragma unroll
            for (int j = 0; j < COUT / 16; ++j) {
                float v[16];
                tmem_ld16(tbase + (uint32_t)(16 * j), v);   // every lane: the load is warp-wide
                if (!ok) continue;
                __nv_bfloat16* o = a.out.ptr + vox * a.out.stride + a.out.c0 + 16 * j;
                const __nv_bfloat16* mk = a.mask ? a.mask + vox * a.mask_stride + a.mask_c0 + 16 * j : nullptr;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float f[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) f[e] = v[8 * h + e] + sbias[16 * j + 8 * h + e];
                    if (a.accumulate) {
                        uint4 old = *reinterpret_cast<const uint4*>(o + 8 * h);
                        const __nv_bfloat162* ob = reinterpret_cast<const __nv_bfloat162*>(&old);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            float2 t2 = __bfloat1622float2(ob[e]);
                            f[2 * e] += t2.x;
                            f[2 * e + 1] += t2.y;
                        }
                    }
                    if (a.relu) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) f[e] = fmaxf(f[e], 0.f);
                    }
                    if (mk) {
                        uint4 mv = *reinterpret_cast<const uint4*>(mk + 8 * h);
                        const __nv_bfloat162* mb = reinterpret_cast<const __nv_bfloat162*>(&mv);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            float2 t2 = __bfloat1622float2(mb[e]);
                            if (!(t2.x > 0.f)) f[2 * e] = 0.f;
                            if (!(t2.y > 0.f)) f[2 * e + 1] = 0.f;
                        }
                    }
                    uint4 w;
                    __nv_bfloat162* wb2 = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
                    for (int e = 0; e < 4; ++e) wb2[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
                    *reinterpret_cast<uint4*>(o + 8 * h) = w;
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&t_empty[acc]);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(tmem, C::NCOLS);
    }
    if (threadIdx.x == 0 && *abort && a.err) atomicExch(a.err, 1);
}

// [8][K][N] -> [8][K/8][N][8]: per parity a K-major B of N = cout rows
__global__ void k_pack_down_tc(const __nv_bfloat16* src, int K, int N, __nv_bfloat16* dst)
{
    long long total = 8LL * K * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int kk = (int)(i & 7);
        long long q = i >> 3;
        const int n = (int)(q % N);
        q /= N;
        const int g = (int)(q % (K / 8)), p = (int)(q / (K / 8));
        dst[i] = src[((long long)p * K + 8 * g + kk) * N + n];
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

template <int CIN, int NSL, int TZ, int NS>
cudaError_t launch_cfg(const ConvArgs& a, const __nv_bfloat16* wpack, int* err, cudaStream_t s)
{
    using C = Cfg<CIN, NSL, TZ, NS>;
    static_assert(C::ZS == (NSL <= 32), "pack_conv3_tc stacks the z-taps exactly for slices of up to 32 channels");
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_conv3_tc<CIN, NSL, TZ, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    });
    if (attr != cudaSuccess) return attr;
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const Grid3 g = a.gin;
    CUtensorMap m;
    cuuint64_t dims[5] = {8, (cuuint64_t)(CIN / 8), (cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t vb = (cuuint64_t)a.in.stride * 2;
    cuuint64_t strides[4] = {16, vb, vb * g.nx, vb * g.nx * g.ny};
    cuuint32_t box[5] = {8, 1, HX, HY, (cuuint32_t)(TZ + 2)};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)(a.in.ptr + a.in.c0), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    TcArgs t;
    t.g = g;
    t.out = a.out;
    t.wpack = wpack;
    t.bias = a.bias;
    t.relu = a.relu;
    t.accumulate = a.accumulate;
    t.mask = a.mask;
    t.mask_stride = a.mask_stride;
    t.mask_c0 = a.mask_c0;
    t.tiles_x = (g.nx + TX - 1) / TX;
    t.tiles_y = (g.ny + TY - 1) / TY;
    const int tiles_z = (g.nz + TZ - 1) / TZ;
    t.ntiles = t.tiles_x * t.tiles_y * tiles_z;
    t.err = err;
    t.stall_tile = g_stall_tile;
    t.stall_ns = g_stall_ns;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int slices = a.cout / NSL;
    const dim3 blocks((unsigned)std::max(1, std::min(t.ntiles, sms / slices)), (unsigned)slices);
    k_conv3_tc<CIN, NSL, TZ, NS><<<blocks, TC_THREADS, C::SMEM, s>>>(m, t);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t launch_up_cfg(const ConvArgs& a, const __nv_bfloat16* wpack, int* err, cudaStream_t s)
{
    using C = UpCfg<CIN, COUT>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_up_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    });
    if (attr != cudaSuccess) return attr;
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const Grid3 g = a.gin;
    CUtensorMap m;
    cuuint64_t dims[5] = {8, (cuuint64_t)(CIN / 8), (cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t vb = (cuuint64_t)a.in.stride * 2;
    cuuint64_t strides[4] = {16, vb, vb * g.nx, vb * g.nx * g.ny};
    cuuint32_t box[5] = {8, 1, TX, TY, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)(a.in.ptr + a.in.c0), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    TcArgs t;
    std::memset(&t, 0, sizeof(t));
    t.g = g;
    t.gfine = a.gout;
    t.out = a.out;
    t.wpack = wpack;
    t.bias = a.bias;
    t.relu = a.relu;
    t.accumulate = a.accumulate;
    t.mask = a.mask;
    t.mask_stride = a.mask_stride;
    t.mask_c0 = a.mask_c0;
    t.tiles_x = (g.nx + TX - 1) / TX;
    t.tiles_y = (g.ny + TY - 1) / TY;
    t.ntiles = t.tiles_x * t.tiles_y * g.nz;
    t.err = err;
    t.stall_tile = -1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_up_tc<CIN, COUT><<<(unsigned)std::max(1, std::min(t.ntiles, sms)), UP_THREADS, C::SMEM, s>>>(m, t);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t launch_down_cfg(const ConvArgs& a, const __nv_bfloat16* wpack, int* err, cudaStream_t s)
{
    using C = DownCfg<CIN, COUT>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_down_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    });
    if (attr != cudaSuccess) return attr;
    TcArgs t;
    std::memset(&t, 0, sizeof(t));
    t.g = a.gout;                    // tiles over the coarse output grid
    t.gfine = a.gin;
    t.out = a.out;
    t.wpack = wpack;
    t.bias = a.bias;
    t.relu = a.relu;
    t.accumulate = a.accumulate;
    t.mask = a.mask;
    t.mask_stride = a.mask_stride;
    t.mask_c0 = a.mask_c0;
    t.tiles_x = (t.g.nx + TX - 1) / TX;
    t.tiles_y = (t.g.ny + TY - 1) / TY;
    t.ntiles = t.tiles_x * t.tiles_y * t.g.nz;
    t.err = err;
    t.stall_tile = -1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_down_tc<CIN, COUT><<<(unsigned)std::max(1, std::min(t.ntiles, sms)), DOWN_THREADS, C::SMEM, s>>>(
        t, a.in.ptr + a.in.c0, a.in.stride);
    return cudaGetLastError();
}

// Output channels per block: the whole layer where its weights fit next to the halo stages,
// else slices of 32 (64 input channels) or 16 (128 input channels).
int slice_width(int cin, int cout)
{
    if (cin <= 32) return cout;
    if (cin == 64) return cout <= 32 ? cout : 32;
    return 16;
}

// Tiles of 8 x 16 x tz voxels over the grid, times the channel slices.
long long tc_blocks(Grid3 g, int tz, int slices)
{
    return (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY) * ((g.nz + tz - 1) / tz) * slices;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

void conv3_tc_test_stall(int tile, uint64_t ns)
{
    g_stall_tile = tile;
    g_stall_ns = std::min<uint64_t>(ns, WAIT_NS);
}

bool conv3_tc_supported(int cin, int cout)
{
    return (cin == 16 && (cout == 16 || cout == 32)) || (cin == 32 && (cout == 16 || cout == 32 || cout == 64)) ||
           (cin == 64 && (cout == 32 || cout == 64 || cout == 128)) || (cin == 128 && (cout == 64 || cout == 128));
}

cudaError_t pack_conv3_tc(const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* wpack, cudaStream_t s)
{
    long long n = 27LL * cin * cout;
    const int nsl = slice_width(cin, cout);
    k_pack_tc<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(w, cin, cout, nsl, nsl <= 32 ? 1 : 0,
                                                                                  wpack);
    return cudaGetLastError();
}

bool up_tc_supported(int cin, int cout)
{
    // (128, 64) runs on the 16^3 level: 32 tiles, each block would load 128 KB of weights for
    // one tile, and the implicit-GEMM kernel is faster there (measured)
    return (cin == 32 && cout == 16) || (cin == 64 && cout == 32);
}

cudaError_t pack_up_tc(const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* wpack, cudaStream_t s)
{
    long long n = 8LL * cin * cout;
    k_pack_up_tc<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(w, cin, cout, wpack);
    return cudaGetLastError();
}

cudaError_t launch_up_tc(const ConvArgs& a, const __nv_bfloat16* wpack, int* err, cudaStream_t s)
{
    if (a.mode != UP || a.in.c0 % 8 || a.in.stride % 8 || a.out.c0 % 8 || a.out.stride % 8 ||
        (a.mask && (a.mask_c0 % 8 || a.mask_stride % 8)) || !up_tc_supported(a.cin, a.cout))
        return cudaErrorInvalidValue;
    if (a.cin == 32) return launch_up_cfg<32, 16>(a, wpack, err, s);
    return launch_up_cfg<64, 32>(a, wpack, err, s);
}

bool down_tc_supported(int cin, int cout)
{
    // measured against the implicit-GEMM kernel on GB300: (32, 64) over 64^3 -> 32^3 15.4 us
    // instead of 19.0; (16, 32) over 128^3 -> 64^3 37.6 us instead of 36.0 (its 2 KB channel runs per
    // voxel keep the gathering warps latency-bound), and (64, 128) on the 16^3 level has 32 tiles:
    // those two stay on the implicit-GEMM kernel
    return cin == 32 && cout == 64;
}

cudaError_t pack_down_tc(const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* wpack, cudaStream_t s)
{
    long long n = 8LL * cin * cout;
    k_pack_down_tc<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(w, cin, cout, wpack);
    return cudaGetLastError();
}

cudaError_t launch_down_tc(const ConvArgs& a, const __nv_bfloat16* wpack, int* err, cudaStream_t s)
{
    if (a.mode != DOWN || a.in.c0 % 8 || a.in.stride % 8 || a.out.c0 % 8 || a.out.stride % 8 ||
        (a.mask && (a.mask_c0 % 8 || a.mask_stride % 8)) || !down_tc_supported(a.cin, a.cout))
        return cudaErrorInvalidValue;
    return launch_down_cfg<32, 64>(a, wpack, err, s);
}

cudaError_t launch_conv3_tc(const ConvArgs& a, const __nv_bfloat16* wpack, int* err, cudaStream_t s)
{
    if (a.mode != CONV3 || a.in.c0 % 8 || a.in.stride % 8 || a.out.c0 % 8 || a.out.stride % 8 ||
        (a.mask && (a.mask_c0 % 8 || a.mask_stride % 8)) || !conv3_tc_supported(a.cin, a.cout))
        return cudaErrorInvalidValue;
    if (a.cin == 16 && a.cout == 16) return launch_cfg<16, 16, 8, 3>(a, wpack, err, s);
    if (a.cin == 16 && a.cout == 32) return launch_cfg<16, 32, 4, 3>(a, wpack, err, s);
    if (a.cin == 32 && a.cout == 16) return launch_cfg<32, 16, 8, 3>(a, wpack, err, s);
    if (a.cin == 32 && a.cout == 32) return launch_cfg<32, 32, 4, 3>(a, wpack, err, s);
    if (a.cin == 32 && a.cout == 64) return launch_cfg<32, 64, 4, 3>(a, wpack, err, s);
    if (a.cin == 64 && a.cout == 32) return launch_cfg<64, 32, 4, 3>(a, wpack, err, s);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int slices = a.cout / slice_width(a.cin, a.cout);
    // thin z-tiles where 4-deep ones would leave half the SMs idle (the 16^3 level); otherwise
    // 4-deep tiles, which re-read less halo for the same number of rounds
    const bool thin = 2 * tc_blocks(a.gin, 4, slices) < sms;
    if (a.cin == 64) return thin ? launch_cfg<64, 32, 2, 4>(a, wpack, err, s) : launch_cfg<64, 32, 4, 3>(a, wpack, err, s);
    return thin ? launch_cfg<128, 16, 2, 4>(a, wpack, err, s) : launch_cfg<128, 16, 4, 3>(a, wpack, err, s);
}

}  // namespace unet
}  // namespace ocmc
