// ocmc_unet_wgrad_tc.cu -- weight gradients of the denoiser's 3x3x3 convolutions on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory, operands staged by TMA).
//
// dW[t][c][n] = sum over output voxels v of x[v + d_t][c] dy[v][n], t = dx + 3 dy + 9 dz, x zero
// outside the grid. The sum over voxels is the MMA's K; input channels are its M, output channels
// its N.
//
// A block walks lines of output voxels along x (the whole line, nx <= 128, at fixed (y, z)). With
// P = L + 16 (L = nx rounded up to 16) it stages by TMA
//   - the nine input lines j = dy + 3 dz at (y + dy - 1, z + dz - 1), voxels -1 .. P - 2: one plane
//     per j of P voxels x CIN channels (position p holds input voxel p - 1), zero-filled outside
//     the grid (the convolution's padding);
//   - the dy line three times, shifted: plane dx holds at position p the dy of output voxel p - dx
//     (zero outside the grid).
// Then dW_dx = sum_p x_plane[p] dy_dx[p] over p in [0, P): every output voxel i meets its input
// voxel i + dx - 1 exactly once, at p = i + dx, and every other product has a zero factor.
// A plane row (one voxel, all its channels: 32, 64 or 128 bytes) is one TMA swizzle span (32B,
// 64B or 128B swizzle), so TMA moves whole voxels and the plane is the canonical swizzled MN-major
// layout of the MMA: M (or N) runs along a row's channels, K along the voxels; K-groups of 8 voxels
// are 8 rows apart (the descriptor's stride offset) and rows of the next plane one plane apart (its
// leading offset). Every operand starts at a plane or at a multiple of 16 voxels in it, i.e. on a
// swizzle-pattern boundary. Row m = 8 g + c of the M dimension, g = j H + h (H = CIN / 8), is input
// channel 8 h + c at line offset j; one MMA (M = 128) covers a window of 16 consecutive channel
// groups (16 / H planes). Its N = 3 COUT columns are (dx, output channel), so each A window is read
// once for all three x-taps. With 9 H groups the windows start at groups 0, 16, ..., and the last
// one at 9 H - 16, overlapping the one before it; its rows that the earlier window covers are not
// written.
// Each window accumulates into its own FP32 accumulator of 3 COUT columns in tensor memory over
// all lines of the block; at the end the block writes its partial dW [27][CIN][COUT], and the
// caller sums the partials of all blocks in a fixed order.
//
// Warp roles (192 threads): warp 0 issues the TMA copies (its lanes share each row's copies), warp 1
// owns tensor memory and one of its lanes issues the MMAs, warps 2-5 read the accumulators out at
// the end (each warp its 32-lane quarter of tensor memory). Every wait gives up after two seconds,
// sets the error flag, lets the copies and MMAs in flight finish and frees tensor memory before the
// block exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "ocmc_umma.cuh"
#include "ocmc_unet_tc.h"

namespace ocmc {
namespace unet {
namespace {

using namespace ocmc::umma;

constexpr int WG_THREADS = 192;
constexpr uint64_t WG_WAIT_NS = 2000000000ull;
constexpr uint32_t WG_STAGE_BUDGET = 222u * 1024u;   // bytes for the line stages
constexpr uint32_t WG_TAIL = 256u + 4096u;           // barriers, then a guard band
constexpr uint32_t WG_MIN_SMEM = 120u * 1024u;       // one block per SM: its tensor memory is never contended
constexpr int WG_MAX_STAGES = 4;

struct WgArgs {
    Grid3 g;
    int P;                       // plane positions: nx rounded up to 16, plus 16
    long long rows;              // lines: ny * nz
    uint32_t pa, pb, stage;      // input plane, dy plane (2 CIN P, 2 COUT P bytes rounded up to 1 KB), stage bytes
    int ns;                      // stages
    float* partial;              // [gridDim.x][27][CIN][COUT]
    int* err;
};

template <int CIN, int COUT>
struct WgCfg {
    static constexpr int H = CIN / 8, G = 9 * H;
    static constexpr int W = (G + 15) / 16;                   // windows of 16 input planes (M = 128)
    static constexpr uint32_t COLS = 3u * W * COUT;           // one accumulator of 3 COUT columns per window
    static constexpr uint32_t NCOLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
    static_assert(G >= 16 && COLS <= 512, "accumulators fit tensor memory");
    static_assert(COUT % 16 == 0 && 3 * COUT <= 256 && CIN % 8 == 0, "MMA shape");
    __host__ __device__ static constexpr int wstart(int w) { return w < W - 1 ? 16 * w : G - 16; }
    // swizzle span = one voxel's channels; descriptor layout codes: 6 = 32B, 4 = 64B, 2 = 128B
    static constexpr uint64_t swz(int bytes) { return bytes == 32 ? 6ull : bytes == 64 ? 4ull : 2ull; }
    static constexpr uint64_t A_LAYOUT = swz(2 * CIN) << 61, B_LAYOUT = swz(2 * COUT) << 61;
    static_assert(CIN == 16 || CIN == 32 || CIN == 64, "one voxel of input channels is one swizzle span");
    static_assert(COUT == 16 || COUT == 32 || COUT == 64, "one voxel of output channels is one swizzle span");
};

__device__ __forceinline__ bool wg_wait_bounded(uint64_t* bar, uint32_t parity)
{
    int dummy = 0;
    return mbar_wait(bar, parity, &dummy, WG_WAIT_NS);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_THREADS, 1)
    k_wgrad3_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dymap, const WgArgs a)
{
    using C = WgCfg<CIN, COUT>;
    extern __shared__ __align__(1024) uint8_t smem[];
    const int NS = a.ns;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)NS * a.stage);
    uint64_t* full = bars;                      // [WG_MAX_STAGES]
    uint64_t* empty = bars + WG_MAX_STAGES;     // [WG_MAX_STAGES]
    uint64_t* done = bars + 2 * WG_MAX_STAGES;
    uint64_t* drain = done + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this block's rows: blockIdx.x, blockIdx.x + gridDim.x, ...
    const long long nrows = a.rows > (long long)blockIdx.x ? (a.rows - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(done, 1);
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, C::NCOLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t in_bytes = 9u * a.pa;

    if (warp == 0) {
        // ---- producer: the nine input lines and the three shifted dy lines of each line of the block ----
        const uint32_t row_bytes = (uint32_t)a.P * 2u * (9u * CIN + 3u * COUT);   // what the twelve copies deliver
        int last[WG_MAX_STAGES];
#pragma unroll
        for (int i = 0; i < WG_MAX_STAGES; ++i) last[i] = -1;
        for (long long i = 0; i < nrows; ++i) {
            const int st = (int)(i % NS), u = (int)(i / NS);
            int ok = 1;
            if (lane == 0) {
                ok = mbar_wait(&empty[st], (u & 1) ^ 1, abort, WG_WAIT_NS) ? 1 : 0;
                if (ok) mbar_expect_tx(&full[st], row_bytes);
            }
            ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
            if (!ok) break;
            last[st] = u;
            const long long r = blockIdx.x + i * (long long)gridDim.x;
            const int y = (int)(r % a.g.ny), z = (int)(r / a.g.ny);
            uint8_t* sa = smem + (size_t)st * a.stage;
            uint8_t* sb = sa + in_bytes;
            if (lane < 9)
                tma_load_4d(sa + (size_t)lane * a.pa, &xmap, 0, -1, y + lane % 3 - 1, z + lane / 3 - 1, &full[st]);
            else if (lane < 12)
                tma_load_4d(sb + (size_t)(lane - 9) * a.pb, &dymap, 0, 9 - lane, y, z, &full[st]);
            __syncwarp();
        }
        if (*abort && lane == 0) {   // copies in flight must land before the block exits
            for (int i = 0; i < NS; ++i)
                if (last[i] >= 0) wg_wait_bounded(&full[i], last[i] & 1);
        }
    } else if (warp == 1) {
        // ---- MMA issue ----
        if (lane == 0) {
            bool issued = false;
            // kind::f16, BF16 A and B, FP32 D, A and B MN-major (bits 15 and 16), N = (dx, output channel)
            constexpr uint32_t idesc = idesc_bf16_f32(128, 3 * COUT) | (1u << 15) | (1u << 16);
            const uint32_t s0 = saddr(smem);
            for (long long i = 0; i < nrows && !*abort; ++i) {
                const int st = (int)(i % NS), u = (int)(i / NS);
                if (!mbar_wait(&full[st], u & 1, abort, WG_WAIT_NS)) break;
                fence_after_sync();
                const uint32_t sa = s0 + (uint32_t)st * a.stage, sb = sa + in_bytes;
                for (int k = 0; k < a.P / 16; ++k) {
                    // K step k: plane positions 16 k .. 16 k + 15; K-groups of 8 voxels are 8 rows apart
                    // (stride offset), the next plane's rows one plane apart (leading offset)
                    const uint64_t bd = sdesc(sb + (uint32_t)k * 32u * COUT, a.pb, 16u * COUT) | C::B_LAYOUT;
#pragma unroll
                    for (int w = 0; w < C::W; ++w) {
                        // window w starts at channel group wstart(w): plane wstart(w) / H
                        const uint64_t ad = sdesc(sa + (uint32_t)(C::wstart(w) / C::H) * a.pa + (uint32_t)k * 32u * CIN,
                                                  a.pa, 16u * CIN) | C::A_LAYOUT;
                        mma_f16(tmem + (uint32_t)(3 * w * COUT), ad, bd, idesc, (i > 0 || k > 0) ? 1u : 0u);
                    }
                }
                mma_commit(&empty[st]);
                issued = true;
            }
            if (!*abort) {
                mma_commit(done);        // arrives once every MMA above has completed
            } else if (issued) {         // MMAs in flight must finish before tensor memory is freed
                mma_commit(drain);
                wg_wait_bounded(drain, 0);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: accumulators -> this block's partial dW ----
        const int q = warp & 3;                       // the tensor-memory lane quarter of this warp
        const int m = 32 * q + lane;
        if (mbar_wait(done, 0, abort, WG_WAIT_NS)) {
            fence_after_sync();
            float* P = a.partial + (size_t)blockIdx.x * 27 * CIN * COUT;
#pragma unroll 1
            for (int w = 0; w < C::W; ++w) {
                const int gp = C::wstart(w) + (m >> 3);
                const bool mine = gp >= 16 * w;            // rows of an earlier window are written there
                const int j = gp / C::H, h = gp - (gp / C::H) * C::H;
                const int c = 8 * h + (m & 7);
#pragma unroll 1
                for (int dx = 0; dx < 3; ++dx) {
                    const int t = dx + 3 * (j % 3) + 9 * (j / 3);
                    float4* o = reinterpret_cast<float4*>(P + ((size_t)t * CIN + c) * COUT);
#pragma unroll
                    for (int n16 = 0; n16 < COUT / 16; ++n16) {
                        float v[16];
                        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((3 * w + dx) * COUT + 16 * n16), v);
                        if (mine) {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                o[4 * n16 + e] = nrows ? make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3])
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
                }
            }
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

template <int CIN, int COUT>
cudaError_t launch_wg_cfg(Grid3 g, Slice x, Slice dy, float* part, size_t part_cap, int* err, cudaStream_t s,
                          int* parts)
{
    using C = WgCfg<CIN, COUT>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_wgrad3_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    });
    if (attr != cudaSuccess) return attr;
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    if (!wgrad3_tc_fits(CIN, COUT, g.nx)) return cudaErrorNotSupported;
    WgArgs a;
    a.g = g;
    a.P = (g.nx + 15) / 16 * 16 + 16;
    a.rows = (long long)g.ny * g.nz;
    // plane strides rounded up to 1024 bytes: every TMA destination and operand start sits on a
    // boundary of the largest (128B) swizzle pattern
    a.pa = (uint32_t)(a.P * 2 * CIN + 1023) / 1024u * 1024u;
    a.pb = (uint32_t)(a.P * 2 * COUT + 1023) / 1024u * 1024u;
    a.stage = 9u * a.pa + 3u * a.pb;
    a.ns = (int)std::min<uint32_t>(WG_MAX_STAGES, WG_STAGE_BUDGET / a.stage);
    a.err = err;
    a.partial = part;
    const long long m = 27LL * CIN * COUT;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long blocks = std::min<long long>({a.rows, (long long)std::max(1, sms), (long long)(part_cap / m)});
    if (blocks < 1) return cudaErrorMemoryAllocation;

    CUtensorMap mx, md;
    cuuint32_t estr[4] = {1, 1, 1, 1};
    auto swz = [](int bytes) {
        return bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    };
    {
        // whole voxels (CIN channels, one swizzle span) along x, one line per copy
        cuuint64_t dims[4] = {(cuuint64_t)CIN, (cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
        const cuuint64_t vb = (cuuint64_t)x.stride * 2;
        cuuint64_t strides[3] = {vb, vb * g.nx, vb * g.nx * g.ny};
        cuuint32_t box[4] = {(cuuint32_t)CIN, (cuuint32_t)a.P, 1, 1};
        if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)(x.ptr + x.c0), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swz(2 * CIN), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        cuuint64_t dims[4] = {(cuuint64_t)COUT, (cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
        const cuuint64_t vb = (cuuint64_t)dy.stride * 2;
        cuuint64_t strides[3] = {vb, vb * g.nx, vb * g.nx * g.ny};
        cuuint32_t box[4] = {(cuuint32_t)COUT, (cuuint32_t)a.P, 1, 1};
        if (enc(&md, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)(dy.ptr + dy.c0), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swz(2 * COUT), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const uint32_t smem = std::max<uint32_t>(WG_MIN_SMEM, (uint32_t)a.ns * a.stage + WG_TAIL);
    k_wgrad3_tc<CIN, COUT><<<(unsigned)blocks, WG_THREADS, smem, s>>>(mx, md, a);
    *parts = (int)blocks;
    return cudaGetLastError();
}

}  // namespace

bool wgrad3_tc_supported(int cin, int cout)
{
    return (cout == 16 && (cin == 16 || cin == 32)) || (cout == 32 && (cin == 16 || cin == 32 || cin == 64));
}

bool wgrad3_tc_fits(int cin, int cout, int nx)
{
    if (!wgrad3_tc_supported(cin, cout) || nx < 1 || nx > 128) return false;
    const uint32_t P = (uint32_t)(nx + 15) / 16 * 16 + 16;
    const uint32_t pa = (P * 2u * cin + 1023u) / 1024u * 1024u, pb = (P * 2u * cout + 1023u) / 1024u * 1024u;
    const uint32_t stage = 9u * pa + 3u * pb;
    return 2u * stage <= WG_STAGE_BUDGET;
}

cudaError_t launch_wgrad3_tc(Grid3 g, Slice x, Slice dy, int cin, int cout, float* part, size_t part_cap, int* err,
                             cudaStream_t s, int* parts)
{
    if (!wgrad3_tc_fits(cin, cout, g.nx) || x.c0 % 8 || x.stride % 8 || dy.c0 % 8 || dy.stride % 8 || g.ny < 1 ||
        g.nz < 1)
        return cudaErrorInvalidValue;
    if (cout == 16) return cin == 16 ? launch_wg_cfg<16, 16>(g, x, dy, part, part_cap, err, s, parts)
                                     : launch_wg_cfg<32, 16>(g, x, dy, part, part_cap, err, s, parts);
    if (cin == 16) return launch_wg_cfg<16, 32>(g, x, dy, part, part_cap, err, s, parts);
    if (cin == 32) return launch_wg_cfg<32, 32>(g, x, dy, part, part_cap, err, s, parts);
    return launch_wg_cfg<64, 32>(g, x, dy, part, part_cap, err, s, parts);
}

}  // namespace unet
}  // namespace ocmc
