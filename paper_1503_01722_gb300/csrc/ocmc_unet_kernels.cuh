// ocmc_unet_kernels.cuh -- tensor-core kernels of the 3D U-Net dose denoiser.
//
// Activations are BF16, channels-last (NDHWC with x fastest among voxels), stored
// with a per-voxel channel stride so that convolutions read and write channel
// slices (the U-Net's concatenations need no copies). Weights are BF16 copies of
// FP32 master weights, laid out [tap][in channel][out channel]. Every product runs
// on the tensor cores (mma.sync m16n8k16, BF16 inputs, FP32 accumulation).
//
// One implicit-GEMM kernel covers the forward pass and the data gradients of all
// layer kinds: each output row (voxel) gathers its input voxels per tap:
//   CONV3 : 3x3x3, stride 1, zero padding 1      (27 taps, src = v + d - 1)
//   DOWN  : 2x2x2, stride 2 (fine -> coarse)      (8 taps,  src = 2v + d)
//   UP    : 2x2x2 transposed, stride 2 (coarse -> fine), all eight output parities in one
//           launch: row = coarse voxel u, column j = p * cout + n (N = 8 cout, K = cin),
//           out voxel 2u + p, channel n.
// Data gradients use the same kernel with transposed (and, for CONV3, flipped)
// weights: dgrad(CONV3) = CONV3, dgrad(DOWN) = UP, dgrad(UP) = DOWN.
// The weight gradient is a second kernel: dW[tap][c][n] = sum over rows of
// in[src(row, tap)][c] * dy[row][n], split over row chunks into FP32 partials that
// a third kernel sums in a fixed order (deterministic).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ocmc {
namespace unet {

enum Mode { CONV3 = 0, DOWN = 1, UP = 2 };

struct Grid3 {
    int nx, ny, nz;
    __host__ __device__ long long n() const { return (long long)nx * ny * nz; }
};

// Channel slice of an activation buffer: element (v, c) at ptr[v * stride + c0 + c].
struct Slice {
    __nv_bfloat16* ptr;
    int stride, c0;
};

struct ConvArgs {
    Mode mode;
    Grid3 gin, gout;             // input and output grids (output = rows, except UP: rows = input grid)
    Slice in, out;
    int cin, cout;               // channels read / written
    const __nv_bfloat16* w;      // [taps][cin][cout]
    const float* bias;           // [cout] or null
    int relu;                    // apply max(0, .) to the result
    int accumulate;              // out = out + result
    const __nv_bfloat16* mask;   // multiply by (mask(v, c) > 0), mask is a Slice-like buffer
    int mask_stride, mask_c0;
    const __nv_bfloat16* wtc;    // CONV3 / UP: weights packed for the tensor-memory kernel, or null
    int* err;                    // device error flag for the tensor-memory kernel (may be null)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid)
{
    uint32_t s = smem_u32(smem);
    int sz = valid ? 16 : 0;                    // 0 source bytes: the 16 destination bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x2_t(uint32_t& r0, uint32_t& r1, const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(smem_u32(p)));
}

// D = A (16x16, row) * B (16x8, col) + D, BF16 in, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int num_taps(Mode m) { return m == CONV3 ? 27 : (m == DOWN ? 8 : 1); }

// Input voxel for tap t of the output row at (x, y, z) (-1: zero padding). For UP the row is
// the coarse voxel (x, y, z) itself and there is one tap.
__device__ __forceinline__ long long src_of(const ConvArgs& a, int x, int y, int z, int t)
{
    int sx, sy, sz;
    if (a.mode == CONV3) {
        sx = x + (t % 3) - 1;
        sy = y + (t / 3) % 3 - 1;
        sz = z + t / 9 - 1;
    } else if (a.mode == DOWN) {
        sx = 2 * x + (t & 1);
        sy = 2 * y + ((t >> 1) & 1);
        sz = 2 * z + (t >> 2);
    } else {
        sx = x;
        sy = y;
        sz = z;
    }
    const Grid3& gi = a.gin;
    if (sx < 0 || sy < 0 || sz < 0 || sx >= gi.nx || sy >= gi.ny || sz >= gi.nz) return -1;
    return sx + (long long)gi.nx * (sy + (long long)gi.ny * sz);
}

constexpr int BM = 128;        // rows per block
constexpr int THREADS = 256;   // 8 warps, 16 rows each
constexpr int NSTAGE = 4;      // cp.async pipeline depth (K chunks in flight)

// Shared memory of k_conv<BK, BN>: NSTAGE stages of an A tile (BM x BK) and a B tile (BK x BN),
// rows padded by 16 bytes against bank conflicts; reused for the epilogue's FP32 output tile.
__host__ __device__ constexpr int conv_smem_bytes(int bk, int bn)
{
    // the pipeline stages, or the FP32 output tile staged by the epilogue, whichever is larger
    return NSTAGE * (BM * (bk + 8) + bk * (bn + 8)) * 2 > BM * (bn + 5) * 4 ? NSTAGE * (BM * (bk + 8) + bk * (bn + 8)) * 2
                                                                             : BM * (bn + 5) * 4;
}

// Implicit-GEMM convolution. BK: input channels per K chunk (16 or 32); BN: output columns per
// block (16, 32, 64 or 128; gridDim.y covers the columns: cout, or 8 cout for UP).
template <int BK, int BN>
__global__ void __launch_bounds__(THREADS) k_conv(const ConvArgs a)
{
    constexpr int AST = BK + 8;        // smem row strides (bf16)
    constexpr int BST = BN + 8;
    extern __shared__ __align__(16) unsigned char conv_smem[];
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(conv_smem);                  // [NSTAGE][BM * AST]
    __nv_bfloat16* sB = sA + NSTAGE * BM * AST;                                        // [NSTAGE][BK * BST]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long rows = a.mode == UP ? a.gin.n() : a.gout.n();
    const long long r0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int T = num_taps(a.mode);
    const int KC = a.cin / BK;                    // chunks per tap
    const int steps = T * KC;

    // A rows this thread copies (the same rows for every K chunk): their grid coordinates are
    // worked out once, so the per-chunk gathers need no divisions
    constexpr int CH_A = BK / 8;                 // 16-byte chunks per A row
    constexpr int RPT = BM * CH_A / THREADS;     // rows per thread
    const int ach = tid % CH_A;
    int rx[RPT], ry[RPT], rz[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const long long row = r0 + tid / CH_A + k * (THREADS / CH_A);
        const Grid3& gr = a.mode == UP ? a.gin : a.gout;
        if (row < rows) {
            rx[k] = (int)(row % gr.nx);
            const long long q = row / gr.nx;
            ry[k] = (int)(q % gr.ny);
            rz[k] = (int)(q / gr.ny);
        } else {
            rx[k] = -1 << 20;                    // far outside: every tap reads zeros
            ry[k] = rz[k] = 0;
        }
    }

    auto load = [&](int step, int buf) {
        const int t = step / KC;
        const int c0 = (step % KC) * BK;
        __nv_bfloat16* dA = sA + buf * BM * AST;
        __nv_bfloat16* dB = sB + buf * BK * BST;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = tid / CH_A + k * (THREADS / CH_A);
            const long long s = src_of(a, rx[k], ry[k], rz[k], t);
            const __nv_bfloat16* g = a.in.ptr + (s >= 0 ? s : 0) * a.in.stride + a.in.c0 + c0 + ach * 8;
            cp_async16(&dA[r * AST + ach * 8], g, s >= 0);
        }
        constexpr int CH_B = BN / 8;
        for (int i = tid; i < BK * CH_B; i += THREADS) {
            int k = i / CH_B, ch = i % CH_B;
            const int col = n0 + ch * 8;
            // UP: column p * cout + n reads parity p's weights [p][cin][cout] (cout is a multiple
            // of 8, so a 16-byte chunk never straddles two parities)
            const int wt = a.mode == UP ? col / a.cout : t;
            const int n = a.mode == UP ? col % a.cout : col;
            const __nv_bfloat16* g = a.w + ((long long)wt * a.cin + c0 + k) * a.cout + n;
            cp_async16(&dB[k * BST + ch * 8], g, true);
        }
    };

    float acc[BN / 8][4];
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

    // NSTAGE - 1 chunks in flight ahead of the one being multiplied; one commit group per
    // chunk (empty past the end), so wait_group<NSTAGE - 2> means "chunk s has landed"
#pragma unroll
    for (int st = 0; st < NSTAGE - 1; ++st) {
        if (st < steps) load(st, st);
        cp_async_commit();
    }
    for (int s = 0; s < steps; ++s) {
        const int buf = s % NSTAGE;
        cp_async_wait<NSTAGE - 2>();
        __syncthreads();   // chunk s visible to all; buffer (s - 1) % NSTAGE free again
        if (s + NSTAGE - 1 < steps) load(s + NSTAGE - 1, (s + NSTAGE - 1) % NSTAGE);
        cp_async_commit();
        const __nv_bfloat16* cA = sA + buf * BM * AST;
        const __nv_bfloat16* cB = sB + buf * BK * BST;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a0, a1, a2, a3;
            {
                int row = warp * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
                int col = kk + 8 * (lane >> 4);
                ldsm_x4(a0, a1, a2, a3, &cA[row * AST + col]);
            }
#pragma unroll
            for (int j = 0; j < BN / 8; j += 2) {
                if (j + 1 < BN / 8) {
                    uint32_t b0, b1, b2, b3;
                    int k = kk + (lane & 7) + 8 * ((lane >> 3) & 1);
                    int n = j * 8 + 8 * (lane >> 4);
                    ldsm_x4_t(b0, b1, b2, b3, &cB[k * BST + n]);
                    mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
                    mma_bf16(acc[j + 1], a0, a1, a2, a3, b2, b3);
                } else {
                    uint32_t b0, b1;
                    int k = kk + (lane & 7) + 8 * ((lane >> 3) & 1);
                    ldsm_x2_t(b0, b1, &cB[k * BST + j * 8]);
                    mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
                }
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();                             // the pipeline buffers are free: stage the tile
    // epilogue, in two passes through shared memory so that every store is 16 bytes: the FP32
    // fragments (rows g and g+8 of the warp's 16, columns 2t, 2t+1 of each n-tile) go to a
    // [BM][BN] staging tile; then each thread finishes 8 consecutive columns of one row (bias,
    // accumulate, ReLU, mask, BF16) and stores them at once. UP column p * cout + n: cout is a
    // power of two in the network, so p and n come from a shift and a mask.
    constexpr int CST = BN + 4;
    float* sC = reinterpret_cast<float*>(conv_smem);
    unsigned* sRow = reinterpret_cast<unsigned*>(sC + BM * CST);   // UP: coarse (x, y, z) of each row, 10 bits each
    if (a.mode == UP && tid < BM) {
        const unsigned row = (unsigned)(r0 + tid), nx = (unsigned)a.gin.nx, ny = (unsigned)a.gin.ny;
        const unsigned q = row / nx;                                 // grids hold fewer than 2^31 voxels, sides <= 512
        sRow[tid] = (row - q * nx) | ((q % ny) << 10) | ((q / ny) << 20);
    }
    {
        const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float* rowp = sC + (warp * 16 + g + 8 * h) * CST + 2 * t4;
#pragma unroll
            for (int j = 0; j < BN / 8; ++j) *reinterpret_cast<float2*>(rowp + j * 8) = make_float2(acc[j][2 * h], acc[j][2 * h + 1]);
        }
    }
    __syncthreads();
    const bool pow2 = (a.cout & (a.cout - 1)) == 0;
    const int csh = 31 - __clz(a.cout);
    constexpr int NCH = BN / 8;
    for (int q = tid; q < BM * NCH; q += THREADS) {
        const int r = q / NCH, cc = q % NCH;
        const long long row = r0 + r;
        if (row >= rows) continue;
        const int col = n0 + cc * 8;
        int n = col;
        long long v = row;
        if (a.mode == UP) {
            const int p = pow2 ? col >> csh : col / a.cout;
            n = col - p * a.cout;
            const unsigned c3 = sRow[r];
            const int ux = (int)(c3 & 1023u), uy = (int)((c3 >> 10) & 1023u), uz = (int)(c3 >> 20);
            const int ox = 2 * ux + (p & 1), oy = 2 * uy + ((p >> 1) & 1), oz = 2 * uz + (p >> 2);
            if (ox >= a.gout.nx || oy >= a.gout.ny || oz >= a.gout.nz) continue;
            v = ox + (long long)a.gout.nx * (oy + (long long)a.gout.ny * oz);
        }
        float f[8];
        const float4 lo = *reinterpret_cast<const float4*>(sC + r * CST + cc * 8);
        const float4 hi = *reinterpret_cast<const float4*>(sC + r * CST + cc * 8 + 4);
        f[0] = lo.x; f[1] = lo.y; f[2] = lo.z; f[3] = lo.w; f[4] = hi.x; f[5] = hi.y; f[6] = hi.z; f[7] = hi.w;
        if (a.bias) {
#pragma unroll
            for (int e = 0; e < 8; ++e) f[e] += a.bias[n + e];
        }
        uint4* o = reinterpret_cast<uint4*>(a.out.ptr + v * a.out.stride + a.out.c0 + n);
        if (a.accumulate) {
            const uint4 old = *o;
            const __nv_bfloat162* ob = reinterpret_cast<const __nv_bfloat162*>(&old);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 t = __bfloat1622float2(ob[e]);
                f[2 * e] += t.x;
                f[2 * e + 1] += t.y;
            }
        }
        if (a.relu) {
#pragma unroll
            for (int e = 0; e < 8; ++e) f[e] = fmaxf(f[e], 0.f);
        }
        if (a.mask) {
            const uint4 mv = *reinterpret_cast<const uint4*>(a.mask + v * a.mask_stride + a.mask_c0 + n);
            const __nv_bfloat162* mb = reinterpret_cast<const __nv_bfloat162*>(&mv);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 t = __bfloat1622float2(mb[e]);
                if (!(t.x > 0.f)) f[2 * e] = 0.f;
                if (!(t.y > 0.f)) f[2 * e + 1] = 0.f;
            }
        }
        uint4 w;
        __nv_bfloat162* wb = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
        for (int e = 0; e < 4; ++e) wb[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
        *o = w;
    }
}

struct WgradArgs {
    Mode mode;
    Grid3 gin, gout;
    Slice in;                    // layer input x
    Slice dy;                    // gradient of the layer output (rows = output voxels; UP: fine grid)
    int cin, cout;
    long long rows_per_chunk;
    float* partial;              // [chunks][taps][cin][cout]
};

// Row r's input voxel for the weight gradient: for UP the rows are output (fine)
// voxels whose single source is their coarse parent, and the tap is their parity.
// Grids hold fewer than 2^31 voxels (at most 512^3), so 32-bit division suffices.
__device__ __forceinline__ long long wsrc(const WgradArgs& a, long long r, int t)
{
    const Grid3& go = a.gout;
    const unsigned ur = (unsigned)r, unx = (unsigned)go.nx, q = ur / unx;
    int x = (int)(ur - q * unx);
    int y = (int)(q % (unsigned)go.ny);
    int z = (int)(q / (unsigned)go.ny);
    int sx, sy, sz;
    if (a.mode == CONV3) {
        sx = x + (t % 3) - 1; sy = y + (t / 3) % 3 - 1; sz = z + t / 9 - 1;
    } else if (a.mode == DOWN) {
        sx = 2 * x + (t & 1); sy = 2 * y + ((t >> 1) & 1); sz = 2 * z + (t >> 2);
    } else {
        int p = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
        if (p != t) return -1;
        sx = x >> 1; sy = y >> 1; sz = z >> 1;
    }
    const Grid3& gi = a.gin;
    if (sx < 0 || sy < 0 || sz < 0 || sx >= gi.nx || sy >= gi.ny || sz >= gi.nz) return -1;
    return sx + (long long)gi.nx * (sy + (long long)gi.ny * sz);
}

// Weight-gradient partials: block (chunk, tap) computes the [BC x BN] tile
// sum_{rows in chunk} x[src(row, tap)][c] * dy[row][n]; rows are the GEMM's K.
// gridDim.z covers (cin / BC) x (cout / BN) tiles.
template <int BC, int BN>
__global__ void __launch_bounds__(THREADS) k_wgrad(const WgradArgs a)
{
    constexpr int KR = 32;                 // rows per K step
    constexpr int XST = BC + 8, YST = BN + 8;
    __shared__ __align__(16) __nv_bfloat16 sX[2][KR * XST];
    __shared__ __align__(16) __nv_bfloat16 sY[2][KR * YST];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = blockIdx.y;
    const int tiles_n = a.cout / BN;
    const int c0 = (blockIdx.z / tiles_n) * BC, n0 = (blockIdx.z % tiles_n) * BN;
    const long long rows = a.gout.n();
    const long long rb = (long long)blockIdx.x * a.rows_per_chunk;
    const long long re = rb + a.rows_per_chunk < rows ? rb + a.rows_per_chunk : rows;
    const int steps = (int)((re - rb + KR - 1) / KR);
    constexpr int MT = BC / 16, NT = BN / 8, TILES = MT * NT;
    constexpr int PER_WARP = (TILES + 7) / 8;
    float acc[PER_WARP][4];
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;

    auto load = [&](int s, int buf) {
        long long base = rb + (long long)s * KR;
        for (int i = tid; i < KR * (BC / 8); i += THREADS) {
            int r = i / (BC / 8), ch = i % (BC / 8);
            long long row = base + r;
            long long sv = row < re ? wsrc(a, row, t) : -1;
            const __nv_bfloat16* g = a.in.ptr + (sv >= 0 ? sv : 0) * a.in.stride + a.in.c0 + c0 + ch * 8;
            cp_async16(&sX[buf][r * XST + ch * 8], g, sv >= 0);
        }
        for (int i = tid; i < KR * (BN / 8); i += THREADS) {
            int r = i / (BN / 8), ch = i % (BN / 8);
            long long row = base + r;
            bool ok = row < re;
            const __nv_bfloat16* g = a.dy.ptr + (ok ? row : 0) * a.dy.stride + a.dy.c0 + n0 + ch * 8;
            cp_async16(&sY[buf][r * YST + ch * 8], g, ok);
        }
        cp_async_commit();
    };

    if (steps > 0) load(0, 0);
    for (int s = 0; s < steps; ++s) {
        const int buf = s & 1;
        cp_async_wait_all();
        __syncthreads();
        if (s + 1 < steps) load(s + 1, buf ^ 1);
#pragma unroll
        for (int kk = 0; kk < KR; kk += 16) {
#pragma unroll
            for (int i = 0; i < PER_WARP; ++i) {
                int tile = warp + 8 * i;
                if (tile >= TILES) break;
                int mt = tile / NT, nt = tile % NT;
                // A (M = channel, K = row) from sX[row][c]: transposed 8x8 loads
                uint32_t a0, a1, a2, a3;
                {
                    int j = lane >> 3;
                    int row = kk + (lane & 7) + 8 * (j >> 1);
                    int col = mt * 16 + 8 * (j & 1);
                    ldsm_x4_t(a0, a1, a2, a3, &sX[buf][row * XST + col]);
                }
                uint32_t b0, b1;
                {
                    int row = kk + (lane & 7) + 8 * ((lane >> 3) & 1);
                    ldsm_x2_t(b0, b1, &sY[buf][row * YST + nt * 8]);
                }
                mma_bf16(acc[i], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    const int g = lane >> 2, t4 = lane & 3;
    const int taps = a.mode == CONV3 ? 27 : 8;
    float* P = a.partial + ((long long)blockIdx.x * taps + t) * a.cin * a.cout;
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) {
        int tile = warp + 8 * i;
        if (tile >= TILES) break;
        int mt = tile / NT, nt = tile % NT;
        int c = c0 + mt * 16 + g, n = n0 + nt * 8 + 2 * t4;
        P[(long long)c * a.cout + n] = acc[i][0];
        P[(long long)c * a.cout + n + 1] = acc[i][1];
        P[(long long)(c + 8) * a.cout + n] = acc[i][2];
        P[(long long)(c + 8) * a.cout + n + 1] = acc[i][3];
    }
}

// Weight gradient of a 3x3x3 convolution, all nine taps of one z-offset per block:
// dW[t][c][n] = sum over output voxels v of x[v + d_t][c] dy[v][n] (zero outside the grid).
// The K dimension runs over segments of WSEG = 32 voxels along x. For a segment at (x0, y, z)
// the block stages dy[x0 .. x0+31, y, z] and, for dy' = -1, 0, 1, the input run
// x[x0-1 .. x0+32, y+dy', z+dz] (zero-filled where it leaves the grid); tap (dx, dy') then
// reads its A operand from that run shifted by dx rows, so one staged segment feeds nine taps
// (the per-tap kernel above re-reads both operands for every tap). blockIdx = (segment chunk,
// z-offset, channel tile); a block walks its contiguous segments with running coordinates.
// Partials [chunk][27][cin][cout] are summed in a fixed order.
constexpr int WSEG = 32;

struct Wgrad3Args {
    Grid3 g;
    Slice in, dy;
    int cin, cout;
    int seg_x;                   // segments per x line
    long long nseg, seg_per_chunk;
    float* partial;
};

template <int BC, int BN>
__global__ void __launch_bounds__(THREADS, 4) k_wgrad3(const Wgrad3Args a)
{
    constexpr int RUN = WSEG + 2, NST = 4;
    constexpr int XST = BC + 8, YST = BN + 8;
    constexpr int XS = 3 * RUN * XST, YS = WSEG * YST;
    constexpr int CX = BC / 8, CY = BN / 8;
    __shared__ __align__(16) __nv_bfloat16 sX[NST][XS];
    __shared__ __align__(16) __nv_bfloat16 sY[NST][YS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dz = blockIdx.y;
    const int tiles_n = a.cout / BN;
    const int c0 = (blockIdx.z / tiles_n) * BC, n0 = (blockIdx.z % tiles_n) * BN;
    const long long sb = (long long)blockIdx.x * a.seg_per_chunk;
    const long long se = sb + a.seg_per_chunk < a.nseg ? sb + a.seg_per_chunk : a.nseg;
    const int steps = se > sb ? (int)(se - sb) : 0;
    constexpr int MT = BC / 16, NT = BN / 8, TILES = 9 * MT * NT;
    constexpr int PER_WARP = (TILES + 7) / 8;
    const Grid3 g = a.g;
    float acc[PER_WARP][4];
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;

    // coordinates of the next segment to stage (segments are loaded strictly in order)
    int lx0, ly, lz;
    {
        const unsigned sg = (unsigned)sb;                 // grids hold fewer than 2^31 voxels
        const unsigned q = sg / (unsigned)a.seg_x;
        lx0 = (int)(sg - q * (unsigned)a.seg_x) * WSEG;
        ly = (int)(q % (unsigned)g.ny);
        lz = (int)(q / (unsigned)g.ny);
    }
    auto load = [&](int buf) {
        const int zz = lz + dz - 1;
        const bool zok = zz >= 0 && zz < g.nz;
        for (int i = tid; i < 3 * RUN * CX; i += THREADS) {
            const int ch = i % CX, pos = (i / CX) % RUN, r = i / (CX * RUN);
            const int xx = lx0 - 1 + pos, yy = ly + r - 1;
            const bool ok = zok && xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny;
            const int v = ok ? xx + g.nx * (yy + g.ny * zz) : 0;
            cp_async16(&sX[buf][(r * RUN + pos) * XST + ch * 8], a.in.ptr + (long long)v * a.in.stride + a.in.c0 + c0 + ch * 8,
                       ok);
        }
        for (int i = tid; i < WSEG * CY; i += THREADS) {
            const int ch = i % CY, k = i / CY;
            const int xx = lx0 + k;
            const bool ok = xx < g.nx;
            const int v = ok ? xx + g.nx * (ly + g.ny * lz) : 0;
            cp_async16(&sY[buf][k * YST + ch * 8], a.dy.ptr + (long long)v * a.dy.stride + a.dy.c0 + n0 + ch * 8, ok);
        }
        lx0 += WSEG;
        if (lx0 >= a.seg_x * WSEG) {
            lx0 = 0;
            if (++ly == g.ny) { ly = 0; ++lz; }
        }
    };

#pragma unroll
    for (int st = 0; st < NST - 1; ++st) {
        if (st < steps) load(st);
        cp_async_commit();
    }
    for (int s = 0; s < steps; ++s) {
        const int buf = s % NST;
        cp_async_wait<NST - 2>();
        __syncthreads();
        if (s + NST - 1 < steps) load((s + NST - 1) % NST);
        cp_async_commit();
#pragma unroll
        for (int kk = 0; kk < WSEG; kk += 16) {
            uint32_t bfr[NT][2];                          // dy fragments, shared by the nine taps
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int row = kk + (lane & 7) + 8 * ((lane >> 3) & 1);
                ldsm_x2_t(bfr[nt][0], bfr[nt][1], &sY[buf][row * YST + nt * 8]);
            }
#pragma unroll
            for (int i = 0; i < PER_WARP; ++i) {
                const int tile = warp + 8 * i;
                if (tile >= TILES) break;
                const int t9 = tile / (MT * NT), rem = tile % (MT * NT);
                const int mt = rem / NT, nt = rem % NT;
                const int ddx = t9 % 3, ddy = t9 / 3;
                uint32_t a0, a1, a2, a3;
                // A (M = channel, K = position) from the run of row offset ddy, shifted by ddx
                const int j = lane >> 3;
                const int row = ddy * RUN + ddx + kk + (lane & 7) + 8 * (j >> 1);
                const int col = mt * 16 + 8 * (j & 1);
                ldsm_x4_t(a0, a1, a2, a3, &sX[buf][row * XST + col]);
                uint32_t b0 = bfr[0][0], b1 = bfr[0][1];
#pragma unroll
                for (int q = 1; q < NT; ++q)              // select, not an indexed (local-memory) read
                    if (q == nt) { b0 = bfr[q][0]; b1 = bfr[q][1]; }
                mma_bf16(acc[i], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    cp_async_wait<0>();
    const int gq = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) {
        const int tile = warp + 8 * i;
        if (tile >= TILES) break;
        const int t9 = tile / (MT * NT), rem = tile % (MT * NT);
        const int mt = rem / NT, nt = rem % NT;
        const int t = 9 * dz + t9;                       // tap index dx + 3 dy + 9 dz
        float* P = a.partial + ((long long)blockIdx.x * 27 + t) * a.cin * a.cout;
        const int c = c0 + mt * 16 + gq, n = n0 + nt * 8 + 2 * t4;
        P[(long long)c * a.cout + n] = acc[i][0];
        P[(long long)c * a.cout + n + 1] = acc[i][1];
        P[(long long)(c + 8) * a.cout + n] = acc[i][2];
        P[(long long)(c + 8) * a.cout + n + 1] = acc[i][3];
    }
}

}  // namespace unet
}  // namespace ocmc
