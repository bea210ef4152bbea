// ocmc_unet_wgrad_tc.cu -- weight gradients of the denoiser's 3x3x3 convolutions on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory, operands staged by TMA).
//
// dW[t][c][n] = sum over output voxels v of x[v + d_t][c] dy[v][n], t = dx + 3 dy + 9 dz, x zero
// outside the grid. The sum over voxels is the MMA's K; input channels are its M, output channels
// its N.
//
// A block walks lines of output voxels along x (the whole line, nx <= 128, at fixed (y, z)) for
// one slice of NSL output channels (blockIdx.y; the accumulators of all output channels of the
// wider layers would not fit tensor memory). With P = L + 16 (L = nx rounded up to 16) it stages
// by TMA
//   - the nine input lines j = dy + 3 dz at (y + dy - 1, z + dz - 1), voxels -1 .. P - 2 (position p
//     holds input voxel p - 1), zero-filled outside the grid (the convolution's padding);
//   - the slice's dy line three times, shifted: copy dx holds at position p the dy of output voxel
//     p - dx (zero outside the grid).
// Then dW_dx = sum_p x_line[p] dy_dx[p] over p in [0, P): every output voxel i meets its input
// voxel i + dx - 1 exactly once, at p = i + dx, and every other product has a zero factor.
// A line is stored as atoms of up to 64 channels (one atom for 16-64 channels, two for 128): an
// atom row (one voxel's channels of that atom: 32, 64 or 128 bytes) is one TMA swizzle span (32B,
// 64B or 128B swizzle), so TMA moves whole voxels and the atom is the canonical swizzled MN-major
// layout of the MMA: M (or N) runs along a row's channels, K along the voxels; K-groups of 8 voxels
// are 8 rows apart (the descriptor's stride offset) and the rows of the next atom one atom apart
// (its leading offset). Every operand starts at an atom or at a multiple of 16 voxels in it, i.e.
// on a swizzle-pattern boundary. Row m = 8 g + c of the M dimension, g = j CIN/8 + h, is input
// channel 8 h + c at line offset j; one MMA (M = 128) covers a window of 16 consecutive channel
// groups. Its N = 3 NSL columns are (dx, output channel of the slice), so each A window is read
// once for all three x-taps. With 9 CIN/8 groups the windows start at groups 0, 16, ..., and the
// last one at 9 CIN/8 - 16, overlapping the one before it where 16 does not divide the count; its
// rows that the earlier window covers are not written.
// Each window accumulates into its own FP32 accumulator of 3 NSL columns in tensor memory over all
// lines of the block; at the end the block writes its slice of the partial dW [27][CIN][cout] of
// its column blockIdx.x, and the caller sums the partials in a fixed order.
//
// Warp roles (192 threads): warp 0 issues the TMA copies (its lanes share each line's copies), warp
// 1 owns tensor memory and one of its lanes issues the MMAs, warps 2-5 read the accumulators out at
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
    int P;                       // line positions: nx rounded up to 16, plus 16
    int cout;                    // output channels of the layer (NSL per block)
    long long rows;              // lines: ny * nz
    uint32_t pa, pb, stage;      // input atom, dy copy (P rows each, rounded up to 1 KB), stage bytes
    int ns;                      // stages
    float* partial;              // [gridDim.x][27][CIN][cout]
    int* err;
};

template <int CIN, int NSL>
struct WgCfg {
    static constexpr int SPAN_A = 2 * CIN < 128 ? 2 * CIN : 128;        // bytes of one atom row
    static constexpr int AT = 2 * CIN / SPAN_A;                         // atoms per line
    static constexpr int GA = SPAN_A / 16;                              // channel groups per atom
    static constexpr int G = 9 * CIN / 8;                               // channel groups of the nine lines
    static constexpr int W = (G + 15) / 16;                             // windows of 16 groups (M = 128)
    static constexpr int SPAN_B = 2 * NSL;
    static constexpr uint32_t COLS = 3u * W * NSL;                      // one accumulator of 3 NSL columns per window
    static constexpr uint32_t NCOLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
    static_assert(G >= 16 && COLS <= 512, "accumulators fit tensor memory");
    static_assert((NSL == 16 || NSL == 32) && (CIN == 16 || CIN == 32 || CIN == 64 || CIN == 128), "shapes");
    __host__ __device__ static constexpr int wstart(int w) { return w < W - 1 ? 16 * w : G - 16; }
    static_assert(wstart(W - 1) % GA == 0, "every window starts at an atom");
    // descriptor layout codes: 6 = 32B, 4 = 64B, 2 = 128B swizzle
    static constexpr uint64_t swz(int bytes) { return bytes == 32 ? 6ull : bytes == 64 ? 4ull : 2ull; }
    static constexpr uint64_t A_LAYOUT = swz(SPAN_A) << 61, B_LAYOUT = swz(SPAN_B) << 61;
};

__device__ __forceinline__ bool wg_wait_bounded(uint64_t* bar, uint32_t parity)
{
    int dummy = 0;
    return mbar_wait(bar, parity, &dummy, WG_WAIT_NS);
}

template <int CIN, int NSL>
__global__ void __launch_bounds__(WG_THREADS, 1)
    k_wgrad3_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dymap, const WgArgs a)
{
    using C = WgCfg<CIN, NSL>;
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
    const int n0 = blockIdx.y * NSL;            // this block's output channels n0 .. n0 + NSL - 1
    // this block's lines: blockIdx.x, blockIdx.x + gridDim.x, ...
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
    const uint32_t in_bytes = 9u * C::AT * a.pa;

    if (warp == 0) {
        // ---- producer: the nine input lines and the three shifted dy lines of each line of the block ----
        const uint32_t row_bytes = (uint32_t)a.P * 2u * (9u * CIN + 3u * NSL);   // what the copies deliver
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
            if (lane < 9 * C::AT) {                 // atom q of input line j, stored as atom j AT + q
                const int j = lane / C::AT, q = lane - j * C::AT;
                tma_load_4d(sa + (size_t)lane * a.pa, &xmap, q * (C::SPAN_A / 2), -1, y + j % 3 - 1, z + j / 3 - 1,
                            &full[st]);
            } else if (lane < 9 * C::AT + 3) {      // dy copy dx, shifted by dx voxels
                const int dx = lane - 9 * C::AT;
                tma_load_4d(sb + (size_t)dx * a.pb, &dymap, n0, -dx, y, z, &full[st]);
            }
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
            constexpr uint32_t idesc = idesc_bf16_f32(128, 3 * NSL) | (1u << 15) | (1u << 16);
            const uint32_t s0 = saddr(smem);
            for (long long i = 0; i < nrows && !*abort; ++i) {
                const int st = (int)(i % NS), u = (int)(i / NS);
                if (!mbar_wait(&full[st], u & 1, abort, WG_WAIT_NS)) break;
                fence_after_sync();
                const uint32_t sa = s0 + (uint32_t)st * a.stage, sb = sa + in_bytes;
                for (int k = 0; k < a.P / 16; ++k) {
                    // K step k: line positions 16 k .. 16 k + 15; K-groups of 8 voxels are 8 rows apart
                    // (stride offset), the next atom's rows one atom apart (leading offset)
                    const uint64_t bd = sdesc(sb + (uint32_t)k * 16u * C::SPAN_B, a.pb, 8u * C::SPAN_B) | C::B_LAYOUT;
#pragma unroll
                    for (int w = 0; w < C::W; ++w) {
                        // window w starts at channel group wstart(w), the first group of atom wstart(w) / GA
                        const uint64_t ad = sdesc(sa + (uint32_t)(C::wstart(w) / C::GA) * a.pa + (uint32_t)k * 16u * C::SPAN_A,
                                                  a.pa, 8u * C::SPAN_A) | C::A_LAYOUT;
                        mma_f16(tmem + (uint32_t)(3 * w * NSL), ad, bd, idesc, (i > 0 || k > 0) ? 1u : 0u);
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
        // ---- epilogue: accumulators -> this block's slice of its partial dW ----
        const int q = warp & 3;                       // the tensor-memory lane quarter of this warp
        const int m = 32 * q + lane;
        if (mbar_wait(done, 0, abort, WG_WAIT_NS)) {
            fence_after_sync();
            float* P = a.partial + (size_t)blockIdx.x * 27 * CIN * a.cout;
#pragma unroll 1
            for (int w = 0; w < C::W; ++w) {
                const int gp = C::wstart(w) + (m >> 3);
                const bool mine = gp >= 16 * w;            // rows of an earlier window are written there
                const int j = gp / (CIN / 8), h = gp - j * (CIN / 8);
                const int c = 8 * h + (m & 7);
#pragma unroll 1
                for (int dx = 0; dx < 3; ++dx) {
                    const int t = dx + 3 * (j % 3) + 9 * (j / 3);
                    float4* o = reinterpret_cast<float4*>(P + ((size_t)t * CIN + c) * a.cout + n0);
#pragma unroll
                    for (int n16 = 0; n16 < NSL / 16; ++n16) {
                        float v[16];
                        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((3 * w + dx) * NSL + 16 * n16), v);
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

uint32_t round1k(uint32_t b) { return (b + 1023u) / 1024u * 1024u; }

// output channels per block: 32 where three accumulators of 32 columns per window fit tensor
// memory, else 16
int wg_slice(int cin, int cout)
{
    const int w = (9 * cin / 8 + 15) / 16;
    return cout % 32 == 0 && 3 * w * 32 <= 512 ? 32 : 16;
}

uint32_t wg_stage_bytes(int cin, int nsl, int P)
{
    const uint32_t span_a = (uint32_t)std::min(2 * cin, 128), at = (uint32_t)(2 * cin) / span_a;
    return 9u * at * round1k((uint32_t)P * span_a) + 3u * round1k((uint32_t)P * 2u * (uint32_t)nsl);
}

template <int CIN, int NSL>
cudaError_t launch_wg_cfg(Grid3 g, Slice x, Slice dy, int cout, float* part, size_t part_cap, int* err,
                          cudaStream_t s, int* parts)
{
    using C = WgCfg<CIN, NSL>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_wgrad3_tc<CIN, NSL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    });
    if (attr != cudaSuccess) return attr;
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    if (!wgrad3_tc_fits(CIN, cout, g.nx) || cout % NSL) return cudaErrorNotSupported;
    WgArgs a;
    a.g = g;
    a.P = (g.nx + 15) / 16 * 16 + 16;
    a.cout = cout;
    a.rows = (long long)g.ny * g.nz;
    // atom and copy strides rounded up to 1024 bytes: every TMA destination and operand start sits
    // on a boundary of the largest (128B) swizzle pattern
    a.pa = round1k((uint32_t)a.P * C::SPAN_A);
    a.pb = round1k((uint32_t)a.P * C::SPAN_B);
    a.stage = 9u * C::AT * a.pa + 3u * a.pb;
    a.ns = (int)std::min<uint32_t>(WG_MAX_STAGES, WG_STAGE_BUDGET / a.stage);
    a.err = err;
    a.partial = part;
    if (a.ns < 1) return cudaErrorNotSupported;
    const int slices = cout / NSL;
    const long long m = 27LL * CIN * cout;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long blocks =
        std::min<long long>({a.rows, (long long)std::max(1, sms / slices), (long long)(part_cap / m)});
    if (blocks < 1) return cudaErrorMemoryAllocation;

    CUtensorMap mx, md;
    cuuint32_t estr[4] = {1, 1, 1, 1};
    auto swz = [](int bytes) {
        return bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    };
    {
        // whole voxels of one atom (SPAN_A bytes, one swizzle span) along x, one line per copy
        cuuint64_t dims[4] = {(cuuint64_t)CIN, (cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
        const cuuint64_t vb = (cuuint64_t)x.stride * 2;
        cuuint64_t strides[3] = {vb, vb * g.nx, vb * g.nx * g.ny};
        cuuint32_t box[4] = {(cuuint32_t)(C::SPAN_A / 2), (cuuint32_t)a.P, 1, 1};
        if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)(x.ptr + x.c0), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swz(C::SPAN_A), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        // one slice of NSL output channels (SPAN_B bytes, one swizzle span) along x
        cuuint64_t dims[4] = {(cuuint64_t)cout, (cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
        const cuuint64_t vb = (cuuint64_t)dy.stride * 2;
        cuuint64_t strides[3] = {vb, vb * g.nx, vb * g.nx * g.ny};
        cuuint32_t box[4] = {(cuuint32_t)NSL, (cuuint32_t)a.P, 1, 1};
        if (enc(&md, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)(dy.ptr + dy.c0), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swz(C::SPAN_B), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const uint32_t smem = std::max<uint32_t>(WG_MIN_SMEM, (uint32_t)a.ns * a.stage + WG_TAIL);
    k_wgrad3_tc<CIN, NSL><<<dim3((unsigned)blocks, (unsigned)slices), WG_THREADS, smem, s>>>(mx, md, a);
    *parts = (int)blocks;
    return cudaGetLastError();
}

}  // namespace

bool wgrad3_tc_supported(int cin, int cout)
{
    return (cin == 16 || cin == 32 || cin == 64 || cin == 128) && (cout == 16 || cout == 32 || cout == 64 || cout == 128);
}

bool wgrad3_tc_fits(int cin, int cout, int nx)
{
    if (!wgrad3_tc_supported(cin, cout) || nx < 1 || nx > 128) return false;
    const int P = (nx + 15) / 16 * 16 + 16;
    return wg_stage_bytes(cin, wg_slice(cin, cout), P) <= WG_STAGE_BUDGET;
}

cudaError_t launch_wgrad3_tc(Grid3 g, Slice x, Slice dy, int cin, int cout, float* part, size_t part_cap, int* err,
                             cudaStream_t s, int* parts)
{
    if (!wgrad3_tc_fits(cin, cout, g.nx) || x.c0 % 8 || x.stride % 8 || dy.c0 % 8 || dy.stride % 8 || g.ny < 1 ||
        g.nz < 1)
        return cudaErrorInvalidValue;
    const int nsl = wg_slice(cin, cout);
    if (cin == 16) return nsl == 32 ? launch_wg_cfg<16, 32>(g, x, dy, cout, part, part_cap, err, s, parts)
                                    : launch_wg_cfg<16, 16>(g, x, dy, cout, part, part_cap, err, s, parts);
    if (cin == 32) return nsl == 32 ? launch_wg_cfg<32, 32>(g, x, dy, cout, part, part_cap, err, s, parts)
                                    : launch_wg_cfg<32, 16>(g, x, dy, cout, part, part_cap, err, s, parts);
    if (cin == 64) return nsl == 32 ? launch_wg_cfg<64, 32>(g, x, dy, cout, part, part_cap, err, s, parts)
                                    : launch_wg_cfg<64, 16>(g, x, dy, cout, part, part_cap, err, s, parts);
    return launch_wg_cfg<128, 16>(g, x, dy, cout, part, part_cap, err, s, parts);
}

}  // namespace unet
}  // namespace ocmc
