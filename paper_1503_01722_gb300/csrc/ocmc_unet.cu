// ocmc_unet.cu -- 3D U-Net dose denoiser: network, training step, inference and the
// uncertainty-flagged fallback to plain Monte Carlo.
//
// Architecture (4 levels, 16-32-64-128 channels): per level two 3x3x3 convolutions
// with ReLU, 2x2x2 stride-2 convolutions down, 2x2x2 stride-2 transposed convolutions
// up, skip connections by channel concatenation, and a 1x1x1 head that predicts a
// correction added to the normalised noisy dose. Input channels: noisy dose / s and
// density (s = the noisy dose maximum); loss: mean squared error of (out - target/s)
// over voxels of density >= 0.1 g/cm^3; Adam on FP32 master weights with BF16 copies.
#include "ocmc_ctx.h"
#include "ocmc_unet_kernels.cuh"
#include "ocmc_unet_tc.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace ocmc;
using namespace ocmc::unet;

namespace {

constexpr int LEVELS = 4;
constexpr int CH[LEVELS] = {16, 32, 64, 128};
constexpr int NLAYERS = 20;

// ---- small kernels ------------------------------------------------------------------------
__global__ void k_max_reduce(const float* x, long long n, unsigned int* out)
{
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, x[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));   // non-negative floats
}

// x0 = dose / s, x1 = density, x2 = sigma / s (0 without sigma). Channels 3-15 of the input
// activation are zeroed when the network is created and never written, so each voxel needs one
// 8-byte store (channels 0-3).
__global__ void k_pack_input(const float* dose, const float* dens, const float* sigma, long long n,
                             const unsigned int* smax, __nv_bfloat16* x, float* x0f)
{
    float s = __uint_as_float(*smax);
    float inv = s > 0.f ? 1.f / s : 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        float d = dose[v] * inv;
        x0f[v] = d;
        float sg = sigma ? sigma[v] * inv : 0.f;
        __nv_bfloat162 lo = __floats2bfloat162_rn(d, dens[v]), hi = __floats2bfloat162_rn(sg, 0.f);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t*>(&lo);
        w.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(x + v * 16) = w;
    }
}

// out = x0 + sum_c h[v][c] w[c] + b
__global__ void k_head_fwd(const __nv_bfloat16* h, const float* w, const float* b, const float* x0, long long n,
                           float* out)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        float s = b[0] + x0[v];
        const __nv_bfloat16* p = h + v * 16;
#pragma unroll
        for (int c = 0; c < 16; ++c) s += __bfloat162float(p[c]) * w[c];
        out[v] = s;
    }
}

// masked MSE of out against target/s; gout = d loss / d out; loss sum into *acc[0], mask count *acc[1]
__global__ void k_loss(const float* out, const float* target, const float* dens, long long n, const unsigned int* smax,
                       float* gout, double* acc)
{
    float s = __uint_as_float(*smax);
    float inv = s > 0.f ? 1.f / s : 0.f;
    double l = 0.0, cnt = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        bool m = dens[v] >= 0.1f;
        float e = m ? out[v] - target[v] * inv : 0.f;
        gout[v] = e;                    // scaled by 2 / count in k_scale_gout
        l += (double)e * e;
        cnt += m ? 1.0 : 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_down_sync(0xFFFFFFFFu, l, o);
        cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, l);
        atomicAdd(acc + 1, cnt);
    }
}

__global__ void k_scale_gout(float* g, long long n, const double* acc)
{
    float sc = acc[1] > 0.0 ? (float)(2.0 / acc[1]) : 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        g[v] *= sc;
}

// head backward: gh[v][c] = gout[v] w[c] (h > 0); partial sums of gout*h and gout per block
__global__ void k_head_bwd(const __nv_bfloat16* h, const float* w, const float* gout, long long n, __nv_bfloat16* gh,
                           float* part /* [gridDim.x][17] */)
{
    float sw[17];
#pragma unroll
    for (int c = 0; c < 17; ++c) sw[c] = 0.f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        float g = gout[v];
        const __nv_bfloat16* p = h + v * 16;
        __nv_bfloat16* q = gh + v * 16;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float hv = __bfloat162float(p[c]);
            sw[c] += g * hv;
            q[c] = __float2bfloat16_rn(hv > 0.f ? g * w[c] : 0.f);
        }
        sw[16] += g;
    }
    __shared__ float red[17][8];
#pragma unroll
    for (int c = 0; c < 17; ++c) {
        float x = sw[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 17) {
        float x = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) x += red[threadIdx.x][i];
        part[blockIdx.x * 17 + threadIdx.x] = x;
    }
}

// Sum of `parts` rows of length m in a fixed order: thread (x, y) of a 32 x 32 block adds rows
// [y L, (y + 1) L) of column j in order (loads unrolled, so many are in flight), then the 32
// partial sums of the column are added in order of y.
__global__ void __launch_bounds__(1024) k_sum_rows(const float* part, int parts, int m, float* out)
{
    __shared__ float sh[32][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int L = (parts + 31) / 32;
    const int i0 = threadIdx.y * L, i1 = min(parts, i0 + L);
    float s = 0.f;
    if (j < m) {
#pragma unroll 8
        for (int i = i0; i < i1; ++i) s += part[(long long)i * m + j];
    }
    sh[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && j < m) {
        float t = 0.f;
        for (int y = 0; y < 32; ++y) t += sh[y][threadIdx.x];
        out[j] = t;
    }
}

// The same sums for wide rows, four columns per thread (the block-per-32-columns form above would
// launch m / 32 blocks of mostly idle threads): identical order of additions (parts in 32
// consecutive groups, each group summed from zero, the group sums added in order from zero).
__global__ void k_sum_rows4(const float4* part, int parts, long long m4, float4* out)
{
    const int L = (parts + 31) / 32;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m4; j += (long long)gridDim.x * blockDim.x) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int y = 0; y < 32; ++y) {
            const int i0 = y * L, i1 = min(parts, i0 + L);
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = i0; i < i1; ++i) {
                const float4 v = part[(long long)i * m4 + j];
                s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
            }
            t.x += s.x; t.y += s.y; t.z += s.z; t.w += s.w;
        }
        out[j] = t;
    }
}

int sm_count();

void sum_rows(const float* part, int parts, long long m, float* out, cudaStream_t s)
{
    // wide rows with few parts, or rows wide enough for a thread per four columns to keep the GPU
    // busy; otherwise (narrow rows of many parts) the block form
    if (m % 4 == 0 && m >= 8192 && (parts <= 32 || m >= 131072)) {
        const long long m4 = m / 4;
        k_sum_rows4<<<(unsigned)std::min<long long>((m4 + 255) / 256, 8LL * sm_count()), 256, 0, s>>>(
            reinterpret_cast<const float4*>(part), parts, m4, reinterpret_cast<float4*>(out));
        return;
    }
    k_sum_rows<<<(unsigned)((m + 31) / 32), dim3(32, 32), 0, s>>>(part, parts, (int)m, out);
}

// bias gradient partials: per block sums of dy[v][n] over its voxels, in a fixed order (thread
// (r, g) of the block sums channels 8 g .. 8 g + 7 over voxels r, r + R, ... with 16-byte loads;
// then the R partial sums of each channel are added in order), so that gradients are
// bit-reproducible. cout / 8 divides blockDim.x (at most 256 threads); stride and c0 are
// multiples of 8.
__global__ void k_bias_part(const __nv_bfloat16* dy, int stride, int c0, int cout, long long n, float* part)
{
    __shared__ float sh[256 * 8];
    const int G = cout / 8, rpp = blockDim.x / G;
    const int g = threadIdx.x % G, r = threadIdx.x / G;
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0.f;
    if (r < rpp)
        for (long long v = (long long)blockIdx.x * rpp + r; v < n; v += (long long)gridDim.x * rpp) {
            const uint4 q = *reinterpret_cast<const uint4*>(dy + v * stride + c0 + 8 * g);
            const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(b[e]);
                acc[2 * e] += f.x;
                acc[2 * e + 1] += f.y;
            }
        }
#pragma unroll
    for (int e = 0; e < 8; ++e) sh[threadIdx.x * 8 + e] = acc[e];
    __syncthreads();
    if (threadIdx.x < cout) {
        const int gg = threadIdx.x / 8, e = threadIdx.x % 8;
        float sum = 0.f;
        for (int i = 0; i < rpp; ++i) sum += sh[(i * G + gg) * 8 + e];
        part[blockIdx.x * cout + threadIdx.x] = sum;
    }
}

// BF16 copies of the FP32 weights: forward layout W[t][c][n] and the data-gradient layout
// W'[t'][n][c] (t' = 26 - t for 3x3x3 kernels, t' = t for 2x2x2)
__global__ void k_weights_bf16(const float* w, int taps, int cin, int cout, int flip, __nv_bfloat16* wf,
                               __nv_bfloat16* wt)
{
    long long total = (long long)taps * cin * cout;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        int n = (int)(i % cout);
        long long q = i / cout;
        int c = (int)(q % cin);
        int t = (int)(q / cin);
        __nv_bfloat16 b = __float2bfloat16_rn(w[i]);
        wf[i] = b;
        int t2 = flip ? taps - 1 - t : t;
        wt[((long long)t2 * cout + n) * cin + c] = b;
    }
}

__global__ void k_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// He-normal initial weights from Philox (Box-Muller), biases zero
__global__ void k_init(float* w, long long n, float stddev, uint32_t k0, uint32_t k1, uint32_t stream)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        uint32_t c0 = (uint32_t)i, c1 = (uint32_t)(i >> 32), c2 = stream, c3 = 0x0D15EA5Eu;
        uint32_t a0 = k0, a1 = k1;
        for (int r = 0; r < 10; ++r) {
            uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
            uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
            uint32_t n0 = hi1 ^ c1 ^ a0, n2 = hi0 ^ c3 ^ a1;
            c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
            a0 += 0x9E3779B9u; a1 += 0xBB67AE85u;
        }
        float u1 = ((c0 >> 8) + 1u) * 5.9604644775390625e-08f, u2 = ((c1 >> 8) + 1u) * 5.9604644775390625e-08f;
        w[i] = stddev * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
    }
}

// ---- network ------------------------------------------------------------------------------
struct Act {
    __nv_bfloat16* x = nullptr;     // activation
    __nv_bfloat16* g = nullptr;     // its gradient
    int ch = 0;
    int level = 0;
};

struct Layer {
    Mode mode;
    int cin, cout, taps;
    int in_act, in_c0, out_act, out_c0;
    int lin, lout;                  // levels of input and output
    size_t woff, boff;              // offsets in the flat parameter vector
    __nv_bfloat16* wf = nullptr;    // forward BF16 weights
    __nv_bfloat16* wt = nullptr;    // transposed / flipped BF16 weights
    __nv_bfloat16* wtc_f = nullptr; // wf packed for the tensor-memory convolution (CONV3), or null
    __nv_bfloat16* wtc_t = nullptr; // wt packed likewise, for the data gradient
    bool grad_accumulate = false;   // the input's gradient slice was already written
};

}  // namespace

struct ocmc_unet {
    int device = 0;
    Grid3 g[LEVELS];
    long long nvox = 0;
    std::vector<Act> acts;
    std::vector<Layer> layers;
    size_t nparams = 0;
    size_t head_w = 0, head_b = 0;
    float* params = nullptr;        // FP32 master weights (flat)
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    long long step = 0;
    float* part = nullptr;          // weight-gradient partials
    size_t part_n = 0;
    float* tmpw = nullptr;          // UP weight gradient before transposition, [8][cout][cin]
    float* bpart = nullptr;         // bias / head gradient partials
    float* x0f = nullptr;           // normalised noisy dose (FP32)
    float* outf = nullptr;          // network output (normalised)
    float* gout = nullptr;
    unsigned int* smax = nullptr;
    double* lacc = nullptr;
    float* fb = nullptr;            // denoise scratch: plain dose, sigma, output, flags (4 x nvox)
    int* kerr = nullptr;            // device flag: a tensor-memory kernel timed out
    bool tc = true;                 // 3x3x3 convolutions on tcgen05 where the kernel covers them
    std::string err;
};

namespace {

ocmc_status ufail(ocmc_unet* u, ocmc_status s, const std::string& m)
{
    if (u) u->err = m;
    return s;
}

#define UCK(call, where)                                                                          \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return ufail(u, e_ == cudaErrorMemoryAllocation ? OCMC_ERR_OOM : OCMC_ERR_CUDA,       \
                         std::string(where) + ": " + cudaGetErrorString(e_));                     \
    } while (0)

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 16)); }

// A tensor-memory kernel that timed out has set u->kerr; report it once and clear it.
ocmc_status take_kernel_flag(ocmc_unet* u, cudaStream_t s)
{
    int f = 0;
    UCK(cudaMemcpyAsync(&f, u->kerr, sizeof(int), cudaMemcpyDeviceToHost, s), "flag");
    UCK(cudaStreamSynchronize(s), "sync");
    if (!f) return OCMC_OK;
    UCK(cudaMemsetAsync(u->kerr, 0, sizeof(int), s), "flag");
    return ufail(u, OCMC_ERR_TIMEOUT, "a tensor-memory convolution timed out waiting for its data");
}

template <int BK, int BN>
cudaError_t launch_conv_tile(const ConvArgs& a, dim3 grid, cudaStream_t s)
{
    constexpr int smem = conv_smem_bytes(BK, BN);
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_conv<BK, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    if (attr != cudaSuccess) return attr;
    k_conv<BK, BN><<<grid, THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Column tile: the widest of 128 / 64 / 32 / 16 that still gives about two blocks per SM (small
// grids at the coarse levels would otherwise leave most SMs idle).
template <int BK>
cudaError_t launch_conv_bk(const ConvArgs& a, cudaStream_t s)
{
    const long long rows = a.mode == UP ? a.gin.n() : a.gout.n();
    const int cols = a.mode == UP ? 8 * a.cout : a.cout;
    const long long rb = (rows + BM - 1) / BM;
    int bn = std::min(cols, 128);
    const long long want = 2LL * sm_count();
    while (bn > 16 && rb * (cols / bn) < want) bn /= 2;
    dim3 grid((unsigned)rb, (unsigned)(cols / bn));
    switch (bn) {
    case 16: return launch_conv_tile<BK, 16>(a, grid, s);
    case 32: return launch_conv_tile<BK, 32>(a, grid, s);
    case 64: return launch_conv_tile<BK, 64>(a, grid, s);
    default: return launch_conv_tile<BK, 128>(a, grid, s);
    }
}

// The data gradient of a layer kind: 3x3x3 stays 3x3x3, DOWN and UP swap.
Mode dgrad_mode(Mode m) { return m == DOWN ? UP : (m == UP ? DOWN : CONV3); }

// Whether a convolution of kind m with (cin, cout) has a tensor-memory kernel, and its weight packing.
bool tc_supported(Mode m, int cin, int cout)
{
    return m == CONV3 ? conv3_tc_supported(cin, cout) : (m == UP ? up_tc_supported(cin, cout) : down_tc_supported(cin, cout));
}

cudaError_t pack_tc(Mode m, const __nv_bfloat16* w, int cin, int cout, __nv_bfloat16* wpack, cudaStream_t s)
{
    return m == CONV3 ? pack_conv3_tc(w, cin, cout, wpack, s)
                      : (m == UP ? pack_up_tc(w, cin, cout, wpack, s) : pack_down_tc(w, cin, cout, wpack, s));
}

cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s)
{
    // 16-byte copies and stores: channel offsets and strides in multiples of 8 (BF16)
    if (a.in.c0 % 8 || a.in.stride % 8 || a.out.c0 % 8 || a.out.stride % 8 || a.cin % 16 || a.cout % 16 ||
        (a.mask && (a.mask_c0 % 8 || a.mask_stride % 8)))
        return cudaErrorInvalidValue;
    if (a.mode == CONV3 && a.wtc && conv3_tc_supported(a.cin, a.cout)) return launch_conv3_tc(a, a.wtc, a.err, s);
    if (a.mode == UP && a.wtc && up_tc_supported(a.cin, a.cout)) return launch_up_tc(a, a.wtc, a.err, s);
    if (a.mode == DOWN && a.wtc && down_tc_supported(a.cin, a.cout)) return launch_down_tc(a, a.wtc, a.err, s);
    return a.cin % 32 == 0 ? launch_conv_bk<32>(a, s) : launch_conv_bk<16>(a, s);
}

__global__ void k_transpose_pnc(const float* src, int taps, int n, int c, float* dst)
{
    long long total = (long long)taps * n * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        int ci = (int)(i % c);
        long long q = i / c;
        int ni = (int)(q % n);
        int t = (int)(q / n);
        dst[((long long)t * c + ci) * n + ni] = src[i];
    }
}

// Weight gradient of a 3x3x3 convolution over grid g (input and output) into dW [27][cin][cout]:
// on tcgen05 where that kernel covers the channel counts (tc), else on mma.sync.
cudaError_t launch_wgrad3(Grid3 g, Slice x, Slice dy, int cin, int cout, float* part, size_t part_cap, float* dW,
                          bool tc, int* err, cudaStream_t s)
{
    if (tc && wgrad3_tc_fits(cin, cout, g.nx) && x.c0 % 8 == 0 && x.stride % 8 == 0 && dy.c0 % 8 == 0 &&
        dy.stride % 8 == 0) {
        int parts = 0;
        cudaError_t e = launch_wgrad3_tc(g, x, dy, cin, cout, part, part_cap, err, s, &parts);
        if (e != cudaSuccess) return e;
        sum_rows(part, parts, 27LL * cin * cout, dW, s);
        return cudaGetLastError();
    }
    Wgrad3Args a;
    a.g = g;
    a.in = x;
    a.dy = dy;
    a.cin = cin;
    a.cout = cout;
    a.seg_x = (g.nx + WSEG - 1) / WSEG;
    a.nseg = (long long)a.seg_x * g.ny * g.nz;
    const int bc = std::min(cin, 32), bn = std::min(cout, 32);
    const int tiles = (cin / bc) * (cout / bn);
    const long long m = 27LL * cin * cout;
    // one wave of four blocks per SM (the kernel's registers allow four) over (chunks, 3
    // z-offsets, channel tiles)
    long long chunks = std::max<long long>(1, std::min<long long>(a.nseg, (4LL * sm_count() + 3 * tiles - 1) / (3 * tiles)));
    while (chunks > 1 && (size_t)(chunks * m) > part_cap) chunks /= 2;
    if ((size_t)(chunks * m) > part_cap) return cudaErrorMemoryAllocation;
    a.seg_per_chunk = (a.nseg + chunks - 1) / chunks;
    chunks = (a.nseg + a.seg_per_chunk - 1) / a.seg_per_chunk;
    a.partial = part;
    dim3 grid((unsigned)chunks, 3, (unsigned)tiles);
    if (bc == 16 && bn == 16) k_wgrad3<16, 16><<<grid, THREADS, 0, s>>>(a);
    else if (bc == 16) k_wgrad3<16, 32><<<grid, THREADS, 0, s>>>(a);
    else if (bn == 16) k_wgrad3<32, 16><<<grid, THREADS, 0, s>>>(a);
    else k_wgrad3<32, 32><<<grid, THREADS, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_rows(part, (int)chunks, m, dW, s);
    return cudaGetLastError();
}

// Weight gradient of one layer into dW (FP32, [taps][cin][cout]).
cudaError_t launch_wgrad(Mode mode, Grid3 gin, Grid3 gout, Slice x, Slice dy, int cin, int cout, float* part,
                         size_t part_cap, float* dW, bool tc, int* err, cudaStream_t s)
{
    // UP layers are handled as DOWN over (dy, x) with the roles of the grids swapped:
    // dW[p][c][n] = sum_u x[u][c] dy[2u+p][n]  ==  sum_u (DOWN gather of dy)[u][n] x[u][c]
    WgradArgs a;
    a.mode = mode;
    a.gin = gin;
    a.gout = gout;
    a.in = x;
    a.dy = dy;
    a.cin = cin;
    a.cout = cout;
    if (mode == CONV3) return launch_wgrad3(gout, x, dy, cin, cout, part, part_cap, dW, tc, err, s);
    const int taps = 8;
    long long rows = gout.n();
    int bc = std::min(cin, 64), bn = std::min(cout, 64);
    int tiles = (cin / bc) * (cout / bn);
    long long chunks = std::max<long long>(1, std::min<long long>(64, (rows + 2047) / 2048));
    while (chunks > 1 && (size_t)chunks * taps * cin * cout > part_cap) chunks /= 2;
    if ((size_t)chunks * taps * cin * cout > part_cap) return cudaErrorMemoryAllocation;
    a.rows_per_chunk = (rows + chunks - 1) / chunks;
    a.partial = part;
    dim3 grid((unsigned)chunks, (unsigned)taps, (unsigned)tiles);
#define WG(BC, BN) k_wgrad<BC, BN><<<grid, THREADS, 0, s>>>(a)
    if (bc == 16) { if (bn == 16) WG(16, 16); else if (bn == 32) WG(16, 32); else WG(16, 64); }
    else if (bc == 32) { if (bn == 16) WG(32, 16); else if (bn == 32) WG(32, 32); else WG(32, 64); }
    else { if (bn == 16) WG(64, 16); else if (bn == 32) WG(64, 32); else WG(64, 64); }
#undef WG
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long m = (long long)taps * cin * cout;
    sum_rows(part, (int)chunks, m, dW, s);
    return cudaGetLastError();
}

Slice slice_of(const ocmc_unet* u, int act, int c0, bool grad)
{
    const Act& A = u->acts[act];
    return Slice{grad ? A.g : A.x, A.ch, c0};
}

// forward of layer L
cudaError_t layer_fwd(ocmc_unet* u, const Layer& L, cudaStream_t s)
{
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.mode = L.mode;
    a.gin = u->g[L.lin];
    a.gout = u->g[L.lout];
    a.in = slice_of(u, L.in_act, L.in_c0, false);
    a.out = slice_of(u, L.out_act, L.out_c0, false);
    a.cin = L.cin;
    a.cout = L.cout;
    a.bias = u->params + L.boff;
    a.relu = 1;
    a.err = u->kerr;
    a.w = L.wf;
    a.wtc = u->tc ? L.wtc_f : nullptr;     // CONV3 and UP layers have packed weights
    return launch_conv(a, s);
}

// backward of layer L: weight and bias gradients, then the data gradient into the
// gradient slice of its input (masked by that input's ReLU, accumulated for skips)
cudaError_t layer_bwd(ocmc_unet* u, const Layer& L, bool need_dx, cudaStream_t s)
{
    Slice dy = slice_of(u, L.out_act, L.out_c0, true);
    Slice x = slice_of(u, L.in_act, L.in_c0, false);
    cudaError_t e;
    if (L.mode == UP) {
        // dW[p][c][n] = sum_u x[u][c] dy[2u+p][n]: a DOWN-gather weight gradient over the coarse
        // grid with operands (dy as gathered input, x as rows), computed into [p][n][c], then transposed
        e = launch_wgrad(DOWN, u->g[L.lout], u->g[L.lin], dy, x, L.cout, L.cin, u->part, u->part_n, u->tmpw, u->tc,
                         u->kerr, s);
        if (e != cudaSuccess) return e;
        long long m = 8LL * L.cin * L.cout;          // [p][n][c] -> grads [p][c][n]
        k_transpose_pnc<<<grid_for(m), 256, 0, s>>>(u->tmpw, 8, L.cout, L.cin, u->grads + L.woff);
    } else {
        e = launch_wgrad(L.mode, u->g[L.lin], u->g[L.lout], x, dy, L.cin, L.cout, u->part, u->part_n,
                         u->grads + L.woff, u->tc, u->kerr, s);
        if (e != cudaSuccess) return e;
    }
    long long nout = u->g[L.lout].n();
    // four blocks per SM stream dy once; few partials keep their fixed-order sum short
    int blocks = (int)std::min<long long>(grid_for(nout * L.cout), 4LL * sm_count());
    k_bias_part<<<blocks, 256, 0, s>>>(dy.ptr, dy.stride, dy.c0, L.cout, nout, u->bpart);
    sum_rows(u->bpart, blocks, L.cout, u->grads + L.boff, s);
    e = cudaGetLastError();
    if (e != cudaSuccess || !need_dx) return e;
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in = dy;
    a.out = slice_of(u, L.in_act, L.in_c0, true);
    a.cin = L.cout;
    a.cout = L.cin;
    a.accumulate = L.grad_accumulate ? 1 : 0;
    a.mask = u->acts[L.in_act].x;
    a.mask_stride = u->acts[L.in_act].ch;
    a.mask_c0 = L.in_c0;
    if (L.mode == CONV3) {
        a.mode = CONV3;
        a.gin = u->g[L.lout];
        a.gout = u->g[L.lin];
        a.w = L.wt;
        a.wtc = u->tc ? L.wtc_t : nullptr;
        a.err = u->kerr;
        return launch_conv(a, s);
    }
    if (L.mode == DOWN) {           // fine <- coarse: UP (all parities) with W'[p][n][c]
        a.mode = UP;
        a.gin = u->g[L.lout];
        a.gout = u->g[L.lin];
        a.w = L.wt;
        a.wtc = u->tc ? L.wtc_t : nullptr;
        a.err = u->kerr;
        return launch_conv(a, s);
    }
    a.mode = DOWN;                  // UP layer: coarse <- fine, DOWN gather with W'[p][n][c]
    a.gin = u->g[L.lout];
    a.gout = u->g[L.lin];
    a.w = L.wt;
    a.wtc = u->tc ? L.wtc_t : nullptr;
    a.err = u->kerr;
    return launch_conv(a, s);
}

cudaError_t refresh_bf16(ocmc_unet* u, cudaStream_t s)
{
    for (Layer& L : u->layers) {
        long long m = (long long)L.taps * L.cin * L.cout;
        k_weights_bf16<<<grid_for(m), 256, 0, s>>>(u->params + L.woff, L.taps, L.cin, L.cout, L.mode == CONV3,
                                                   L.wf, L.wt);
        cudaError_t e = cudaSuccess;
        if (L.wtc_f) e = pack_tc(L.mode, L.wf, L.cin, L.cout, L.wtc_f, s);
        if (e == cudaSuccess && L.wtc_t) e = pack_tc(dgrad_mode(L.mode), L.wt, L.cout, L.cin, L.wtc_t, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

ocmc_status forward(ocmc_unet* u, const float* dose, const float* sigma, const float* dens, cudaStream_t s)
{
    long long n = u->nvox;
    UCK(cudaMemsetAsync(u->smax, 0, sizeof(unsigned int), s), "memset");
    k_max_reduce<<<grid_for(n), 256, 0, s>>>(dose, n, u->smax);
    k_pack_input<<<grid_for(n), 256, 0, s>>>(dose, dens, sigma, n, u->smax, u->acts[0].x, u->x0f);
    UCK(cudaGetLastError(), "input");
    for (const Layer& L : u->layers) UCK(layer_fwd(u, L, s), "layer forward");
    const Act& last = u->acts[u->layers.back().out_act];
    k_head_fwd<<<grid_for(n), 256, 0, s>>>(last.x, u->params + u->head_w, u->params + u->head_b, u->x0f, n, u->outf);
    UCK(cudaGetLastError(), "head");
    return OCMC_OK;
}

__global__ void k_denorm(const float* out, const unsigned int* smax, long long n, float* dst)
{
    float sc = __uint_as_float(*smax);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        dst[v] = out[v] * sc;
}

// Fallback to plain Monte Carlo where the network's change exceeds k sigma of the plain
// estimate: out = flag ? plain : denoised. sigma is the batch standard error pooled over the
// voxel's 3x3x3 neighbourhood (root of the mean of the neighbours' variances, clipped at the
// grid's faces): with few batches the per-voxel estimate is itself noisy, and it is exactly
// zero wherever no batch deposited anything, which would make any denoised value there fail.
__global__ void k_fallback(const float* plain, const float* sigma, float* den, float* flag, float k, int nx, int ny,
                           int nz)
{
    const long long n = (long long)nx * ny * nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
        float s2 = 0.f;
        int cnt = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xx = x + dx, yy = y + dy, zz = z + dz;
                    if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
                    const float sg = sigma[xx + (long long)nx * (yy + (long long)ny * zz)];
                    s2 = __fadd_rn(s2, __fmul_rn(sg, sg));     // no contraction: reproducible on the host
                    ++cnt;
                }
        const bool f = fabsf(__fsub_rn(den[v], plain[v])) > __fmul_rn(k, sqrtf(__fdiv_rn(s2, (float)cnt)));
        if (flag) flag[v] = f ? 1.f : 0.f;
        if (f) den[v] = plain[v];
    }
}

}  // namespace

extern "C" {

ocmc_status ocmc_unet_create(ocmc_unet** out, int device, int nx, int ny, int nz, uint64_t seed)
{
    if (!out) return OCMC_ERR_ARG;
    *out = nullptr;
    if (nx < 8 || ny < 8 || nz < 8 || nx % 8 || ny % 8 || nz % 8 || nx > 512 || ny > 512 || nz > 512)
        return OCMC_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return OCMC_ERR_CUDA;
    ocmc_unet* u = new ocmc_unet();
    u->device = device;
    for (int l = 0; l < LEVELS; ++l) u->g[l] = Grid3{nx >> l, ny >> l, nz >> l};
    u->nvox = u->g[0].n();
    // activations: 0 input(16), per level: E_a(C), CAT(2C) [0,C) up / [C,2C) skip, D (down out, level l+1),
    // F_a(C), F_b(C); bottleneck E3a, E3b
    auto add = [&](int ch, int level) { u->acts.push_back(Act{nullptr, nullptr, ch, level}); return (int)u->acts.size() - 1; };
    int X0 = add(16, 0);
    int Ea[LEVELS], CAT[LEVELS], D[LEVELS], Fa[LEVELS], Fb[LEVELS];
    for (int l = 0; l < LEVELS; ++l) {
        Ea[l] = add(CH[l], l);
        CAT[l] = l < LEVELS - 1 ? add(2 * CH[l], l) : add(CH[l], l);   // bottleneck: E3b
        D[l] = l < LEVELS - 1 ? add(CH[l + 1], l + 1) : -1;
        Fa[l] = l < LEVELS - 1 ? add(CH[l], l) : -1;
        Fb[l] = l < LEVELS - 1 ? add(CH[l], l) : -1;
    }
    auto conv = [&](Mode m, int cin, int cout, int ia, int ic0, int oa, int oc0, int lin, int lout, bool acc) {
        Layer L;
        L.mode = m; L.cin = cin; L.cout = cout; L.taps = m == CONV3 ? 27 : 8;
        L.in_act = ia; L.in_c0 = ic0; L.out_act = oa; L.out_c0 = oc0; L.lin = lin; L.lout = lout;
        L.grad_accumulate = acc;
        u->layers.push_back(L);
    };
    // encoder
    int in_act = X0, in_c0 = 0, in_ch = 16;
    for (int l = 0; l < LEVELS; ++l) {
        const int C = CH[l];
        bool last = l == LEVELS - 1;
        conv(CONV3, in_ch, C, in_act, in_c0, Ea[l], 0, l, l, false);
        conv(CONV3, C, C, Ea[l], 0, CAT[l], last ? 0 : C, l, l, false);
        if (!last) {
            // the skip slice's gradient is first written by the decoder's concat convolution
            conv(DOWN, C, CH[l + 1], CAT[l], C, D[l], 0, l, l + 1, true);
            in_act = D[l]; in_c0 = 0; in_ch = CH[l + 1];
        }
    }
    // decoder
    int prev = CAT[LEVELS - 1], prev_ch = CH[LEVELS - 1];
    for (int l = LEVELS - 2; l >= 0; --l) {
        const int C = CH[l];
        conv(UP, prev_ch, C, prev, 0, CAT[l], 0, l + 1, l, false);
        conv(CONV3, 2 * C, C, CAT[l], 0, Fa[l], 0, l, l, false);
        conv(CONV3, C, C, Fa[l], 0, Fb[l], 0, l, l, false);
        prev = Fb[l]; prev_ch = C;
    }
    size_t off = 0;
    for (Layer& L : u->layers) {
        L.woff = off; off += (size_t)L.taps * L.cin * L.cout;
        L.boff = off; off += L.cout;
    }
    u->head_w = off; off += 16;
    u->head_b = off; off += 1;
    u->nparams = off;
    cudaError_t e = cudaSuccess;
    for (Act& A : u->acts) {
        size_t bytes = (size_t)u->g[A.level].n() * A.ch * sizeof(__nv_bfloat16);
        if (e == cudaSuccess) e = cudaMalloc(&A.x, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&A.g, bytes);
        if (e == cudaSuccess) e = cudaMemset(A.x, 0, bytes);
        if (e == cudaSuccess) e = cudaMemset(A.g, 0, bytes);
    }
    for (Layer& L : u->layers) {
        size_t m = (size_t)L.taps * L.cin * L.cout * sizeof(__nv_bfloat16);
        if (e == cudaSuccess) e = cudaMalloc(&L.wf, m);
        if (e == cudaSuccess) e = cudaMalloc(&L.wt, m);
        // packed weights for the tensor-memory kernels, forward and data gradient (the data
        // gradient of a DOWN layer is an UP convolution and vice versa)
        if (L.mode == CONV3 && conv3_tc_supported(L.cin, L.cout) && e == cudaSuccess) e = cudaMalloc(&L.wtc_f, m);
        if (L.mode == CONV3 && conv3_tc_supported(L.cout, L.cin) && e == cudaSuccess) e = cudaMalloc(&L.wtc_t, m);
        if (L.mode != CONV3 && tc_supported(L.mode, L.cin, L.cout) && e == cudaSuccess) e = cudaMalloc(&L.wtc_f, m);
        if (L.mode != CONV3 && tc_supported(dgrad_mode(L.mode), L.cout, L.cin) && e == cudaSuccess)
            e = cudaMalloc(&L.wtc_t, m);
    }
    if (e == cudaSuccess) e = cudaMalloc(&u->kerr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(u->kerr, 0, sizeof(int));
    {
        const char* k = std::getenv("OCMC_UNET_KERNELS");
        u->tc = !(k && std::strcmp(k, "mma") == 0);
    }
    size_t pbytes = u->nparams * sizeof(float);
    if (e == cudaSuccess) e = cudaMalloc(&u->params, pbytes);
    if (e == cudaSuccess) e = cudaMalloc(&u->grads, pbytes);
    if (e == cudaSuccess) e = cudaMalloc(&u->adam_m, pbytes);
    if (e == cudaSuccess) e = cudaMalloc(&u->adam_v, pbytes);
    u->part_n = (size_t)8 << 20;
    if (e == cudaSuccess) e = cudaMalloc(&u->part, u->part_n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&u->tmpw, (size_t)8 * 128 * 128 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&u->bpart, (size_t)152 * 16 * 128 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&u->x0f, u->nvox * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&u->outf, u->nvox * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&u->gout, u->nvox * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&u->smax, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&u->lacc, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(u->params, 0, pbytes);
    if (e == cudaSuccess) e = cudaMemset(u->grads, 0, pbytes);
    if (e == cudaSuccess) e = cudaMemset(u->adam_m, 0, pbytes);
    if (e == cudaSuccess) e = cudaMemset(u->adam_v, 0, pbytes);
    if (e != cudaSuccess) {
        ocmc_unet_destroy(u);
        return e == cudaErrorMemoryAllocation ? OCMC_ERR_OOM : OCMC_ERR_CUDA;
    }
    uint32_t stream = 1;
    for (Layer& L : u->layers) {
        long long m = (long long)L.taps * L.cin * L.cout;
        float fan_in = (float)(L.mode == UP ? L.cin : L.taps * L.cin);
        k_init<<<grid_for(m), 256>>>(u->params + L.woff, m, sqrtf(2.f / fan_in), (uint32_t)seed,
                                     (uint32_t)(seed >> 32), stream++);
    }
    k_init<<<1, 32>>>(u->params + u->head_w, 16, 1e-3f, (uint32_t)seed, (uint32_t)(seed >> 32), stream++);
    e = refresh_bf16(u, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        ocmc_unet_destroy(u);
        return OCMC_ERR_CUDA;
    }
    *out = u;
    return OCMC_OK;
}

void ocmc_unet_destroy(ocmc_unet* u)
{
    if (!u) return;
    cudaSetDevice(u->device);
    cudaDeviceSynchronize();
    for (Act& A : u->acts) { cudaFree(A.x); cudaFree(A.g); }
    for (Layer& L : u->layers) { cudaFree(L.wf); cudaFree(L.wt); cudaFree(L.wtc_f); cudaFree(L.wtc_t); }
    cudaFree(u->params); cudaFree(u->grads); cudaFree(u->adam_m); cudaFree(u->adam_v); cudaFree(u->part);
    cudaFree(u->tmpw); cudaFree(u->bpart);
    cudaFree(u->x0f); cudaFree(u->outf); cudaFree(u->gout); cudaFree(u->smax); cudaFree(u->lacc);
    cudaFree(u->fb); cudaFree(u->kerr);
    delete u;
}

const char* ocmc_unet_last_error(ocmc_unet* u) { return u ? u->err.c_str() : ""; }

ocmc_status ocmc_unet_num_params(ocmc_unet* u, int64_t* n)
{
    if (!u || !n) return OCMC_ERR_ARG;
    *n = (int64_t)u->nparams;
    return OCMC_OK;
}

ocmc_status ocmc_unet_get_params(ocmc_unet* u, float* host, int grads)
{
    if (!u || !host) return OCMC_ERR_ARG;
    UCK(cudaSetDevice(u->device), "device");
    UCK(cudaMemcpy(host, grads ? u->grads : u->params, u->nparams * sizeof(float), cudaMemcpyDeviceToHost), "copy");
    return OCMC_OK;
}

ocmc_status ocmc_unet_set_params(ocmc_unet* u, const float* host)
{
    if (!u || !host) return OCMC_ERR_ARG;
    UCK(cudaSetDevice(u->device), "device");
    UCK(cudaMemcpy(u->params, host, u->nparams * sizeof(float), cudaMemcpyHostToDevice), "copy");
    UCK(cudaMemset(u->adam_m, 0, u->nparams * sizeof(float)), "adam");
    UCK(cudaMemset(u->adam_v, 0, u->nparams * sizeof(float)), "adam");
    u->step = 0;
    UCK(refresh_bf16(u, nullptr), "weights");
    UCK(cudaDeviceSynchronize(), "sync");
    return OCMC_OK;
}

ocmc_status ocmc_unet_forward(ocmc_unet* u, const float* dose, const float* sigma, const float* dens, float* out,
                              void* stream)
{
    if (!u || !dose || !dens || !out) return ufail(u, OCMC_ERR_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    UCK(cudaSetDevice(u->device), "device");
    ocmc_status st = forward(u, dose, sigma, dens, s);
    if (st != OCMC_OK) return st;
    k_denorm<<<grid_for(u->nvox), 256, 0, s>>>(u->outf, u->smax, u->nvox, out);
    UCK(cudaGetLastError(), "output");
    return OCMC_OK;
}

// One training step: forward, masked MSE loss, backward, Adam (lr; betas 0.9/0.999).
// lr <= 0 computes the gradients without updating the weights.
ocmc_status ocmc_unet_train_step(ocmc_unet* u, const float* dose, const float* sigma, const float* dens,
                                 const float* target, float lr,
                                 float* loss_host, void* stream)
{
    if (!u || !dose || !dens || !target) return ufail(u, OCMC_ERR_ARG, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    UCK(cudaSetDevice(u->device), "device");
    ocmc_status st = forward(u, dose, sigma, dens, s);
    if (st != OCMC_OK) return st;
    long long n = u->nvox;
    UCK(cudaMemsetAsync(u->lacc, 0, 2 * sizeof(double), s), "memset");
    k_loss<<<grid_for(n), 256, 0, s>>>(u->outf, target, dens, n, u->smax, u->gout, u->lacc);
    k_scale_gout<<<grid_for(n), 256, 0, s>>>(u->gout, n, u->lacc);
    // head
    const Layer& lastL = u->layers.back();
    const Act& last = u->acts[lastL.out_act];
    int hb = grid_for(n);
    k_head_bwd<<<hb, 256, 0, s>>>(last.x, u->params + u->head_w, u->gout, n, last.g, u->bpart);
    sum_rows(u->bpart, hb, 17, u->grads + u->head_w, s);
    UCK(cudaGetLastError(), "head backward");
    // layers in reverse; UP weight gradients come out as [p][n][c] and are transposed
    for (int i = (int)u->layers.size() - 1; i >= 0; --i) {
        const Layer& L = u->layers[i];
        UCK(layer_bwd(u, L, i > 0, s), "layer backward");
    }
    if (lr > 0.f) {
        u->step++;
        const float b1 = 0.9f, b2 = 0.999f;
        float c1 = 1.f - powf(b1, (float)u->step), c2 = 1.f - powf(b2, (float)u->step);
        k_adam<<<grid_for((long long)u->nparams), 256, 0, s>>>(u->params, u->grads, u->adam_m, u->adam_v,
                                                              (long long)u->nparams, lr, b1, b2, 1e-8f, c1, c2);
        UCK(refresh_bf16(u, s), "weights");
    }
    if (loss_host) {
        ocmc_status fs = take_kernel_flag(u, s);
        if (fs != OCMC_OK) return fs;
        double acc[2];
        UCK(cudaMemcpyAsync(acc, u->lacc, sizeof(acc), cudaMemcpyDeviceToHost, s), "loss");
        UCK(cudaStreamSynchronize(s), "sync");
        *loss_host = acc[1] > 0 ? (float)(acc[0] / acc[1]) : 0.f;
    }
    return OCMC_OK;
}

// Forward pass with a CUDA event pair around every layer: ms_out[i] = mean time of layer i over
// `repeats` passes (stream order, so each layer's time is its own launches only).
ocmc_status ocmc_unet_layer_times(ocmc_unet* u, const float* dose, const float* sigma, const float* dens, int repeats,
                                  float* ms_out,
                                  int* n_layers)
{
    if (!u || !dose || !dens || repeats < 1) return ufail(u, OCMC_ERR_ARG, "bad argument");
    const int L = (int)u->layers.size();
    if (n_layers) *n_layers = L;
    if (!ms_out) return OCMC_OK;
    UCK(cudaSetDevice(u->device), "device");
    std::vector<cudaEvent_t> ev(L + 1);
    for (auto& e : ev) UCK(cudaEventCreate(&e), "event");
    std::vector<double> acc(L, 0.0);
    ocmc_status st = OCMC_OK;
    for (int r = 0; r < repeats && st == OCMC_OK; ++r) {
        long long n = u->nvox;
        cudaMemsetAsync(u->smax, 0, sizeof(unsigned int), nullptr);
        k_max_reduce<<<grid_for(n), 256>>>(dose, n, u->smax);
        k_pack_input<<<grid_for(n), 256>>>(dose, dens, sigma, n, u->smax, u->acts[0].x, u->x0f);
        cudaEventRecord(ev[0], nullptr);
        for (int i = 0; i < L; ++i) {
            if (layer_fwd(u, u->layers[i], nullptr) != cudaSuccess) { st = ufail(u, OCMC_ERR_CUDA, "layer"); break; }
            cudaEventRecord(ev[i + 1], nullptr);
        }
        if (cudaEventSynchronize(ev[L]) != cudaSuccess) st = ufail(u, OCMC_ERR_CUDA, "sync");
        for (int i = 0; i < L && st == OCMC_OK; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            acc[i] += ms;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (st != OCMC_OK) return st;
    ocmc_status fs = take_kernel_flag(u, nullptr);
    if (fs != OCMC_OK) return fs;
    for (int i = 0; i < L; ++i) ms_out[i] = (float)(acc[i] / repeats);
    return OCMC_OK;
}

ocmc_status ocmc_unet_test_stall(int tile, uint64_t wait_ns)
{
    if (tile < -1) return OCMC_ERR_ARG;
    conv3_tc_test_stall(tile, wait_ns);
    return OCMC_OK;
}

// Single layer through the network's kernels, for the gradient tests: x (input grid,
// cin channels), w [taps][cin][cout], dy (output grid, cout) host arrays in FP32 (rounded
// to BF16); y = layer(x) without bias/ReLU, dx, dw (FP32) out.
ocmc_status ocmc_unet_test_layer(int device, int mode, int nx, int ny, int nz, int cin, int cout, const float* x,
                                 const float* w, const float* dy, float* y, float* dx, float* dw)
{
    if (mode < 0 || mode > 2 || cin % 16 || cout % 16 || cin > 256 || cout > 256 || nx % 2 || ny % 2 || nz % 2 ||
        nx < 2 || ny < 2 || nz < 2 || nx > 512 || ny > 512 || nz > 512)
        return OCMC_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return OCMC_ERR_CUDA;
    Grid3 fine{nx, ny, nz}, coarse{nx / 2, ny / 2, nz / 2};
    Mode m = (Mode)mode;
    Grid3 gi = m == UP ? coarse : fine, go = m == DOWN ? coarse : (m == UP ? fine : fine);
    const int taps = m == CONV3 ? 27 : 8;
    long long ni = gi.n(), no = go.n(), nw = (long long)taps * cin * cout;
    std::vector<__nv_bfloat16> hx(ni * cin), hdy(no * cout);
    for (long long i = 0; i < ni * cin; ++i) hx[i] = __float2bfloat16_rn(x[i]);
    for (long long i = 0; i < no * cout; ++i) hdy[i] = __float2bfloat16_rn(dy[i]);
    __nv_bfloat16 *dX = nullptr, *dY = nullptr, *dDY = nullptr, *dDX = nullptr, *wf = nullptr, *wt = nullptr;
    float *w32 = nullptr, *part = nullptr, *dW = nullptr, *dW2 = nullptr;
    size_t part_n = (size_t)64 * 27 * 256 * 256;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
    A((void**)&dX, ni * cin * 2); A((void**)&dY, no * cout * 2); A((void**)&dDY, no * cout * 2);
    A((void**)&dDX, ni * cin * 2); A((void**)&wf, nw * 2); A((void**)&wt, nw * 2); A((void**)&w32, nw * 4);
    A((void**)&part, part_n * 4); A((void**)&dW, nw * 4); A((void**)&dW2, nw * 4);
    __nv_bfloat16 *pf = nullptr, *pt = nullptr;
    int* kerr = nullptr;
    const bool tcf = tc_supported(m, cin, cout), tct = tc_supported(dgrad_mode(m), cout, cin);
    if (tcf) A((void**)&pf, nw * 2);
    if (tct) A((void**)&pt, nw * 2);
    A((void**)&kerr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(kerr, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dX, hx.data(), ni * cin * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dDY, hdy.data(), no * cout * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w32, w, nw * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_weights_bf16<<<grid_for(nw), 256>>>(w32, taps, cin, cout, m == CONV3, wf, wt);
        if (tcf) e = pack_tc(m, wf, cin, cout, pf, nullptr);
        if (tct && e == cudaSuccess) e = pack_tc(dgrad_mode(m), wt, cout, cin, pt, nullptr);
        ConvArgs a;
        std::memset(&a, 0, sizeof(a));
        a.mode = m; a.gin = gi; a.gout = go; a.in = Slice{dX, cin, 0}; a.out = Slice{dY, cout, 0};
        a.cin = cin; a.cout = cout;
        a.wtc = pf; a.err = kerr;
        a.w = wf;
        if (e == cudaSuccess) e = launch_conv(a, nullptr);
    }
    if (e == cudaSuccess) {
        ConvArgs a;
        std::memset(&a, 0, sizeof(a));
        a.in = Slice{dDY, cout, 0}; a.out = Slice{dDX, cin, 0}; a.cin = cout; a.cout = cin;
        a.gin = go; a.gout = gi;
        a.wtc = pt; a.err = kerr;
        if (m == CONV3) { a.mode = CONV3; a.w = wt; e = launch_conv(a, nullptr); }
        else if (m == DOWN) { a.mode = UP; a.w = wt; e = launch_conv(a, nullptr); }
        else { a.mode = DOWN; a.w = wt; e = launch_conv(a, nullptr); }
    }
    if (e == cudaSuccess) {
        if (m == UP) {
            e = launch_wgrad(DOWN, go, gi, Slice{dDY, cout, 0}, Slice{dX, cin, 0}, cout, cin, part, part_n, dW2, true,
                             kerr, nullptr);
            if (e == cudaSuccess) {
                k_transpose_pnc<<<grid_for(nw), 256>>>(dW2, 8, cout, cin, dW);
                e = cudaGetLastError();
            }
        } else {
            e = launch_wgrad(m, gi, go, Slice{dX, cin, 0}, Slice{dDY, cout, 0}, cin, cout, part, part_n, dW, true, kerr,
                             nullptr);
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, kerr, sizeof(int), cudaMemcpyDeviceToHost);
    std::vector<__nv_bfloat16> hy(no * cout), hdx(ni * cin);
    if (e == cudaSuccess) e = cudaMemcpy(hy.data(), dY, no * cout * 2, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hdx.data(), dDX, ni * cin * 2, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(dw, dW, nw * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        for (long long i = 0; i < no * cout; ++i) y[i] = __bfloat162float(hy[i]);
        for (long long i = 0; i < ni * cin; ++i) dx[i] = __bfloat162float(hdx[i]);
    }
    cudaFree(dX); cudaFree(dY); cudaFree(dDY); cudaFree(dDX); cudaFree(wf); cudaFree(wt); cudaFree(w32);
    cudaFree(part); cudaFree(dW); cudaFree(dW2); cudaFree(pf); cudaFree(pt); cudaFree(kerr);
    if (e != cudaSuccess) return OCMC_ERR_CUDA;
    return flag ? OCMC_ERR_TIMEOUT : OCMC_OK;
}

// Denoise the context's current dose: the network maps (dose, density) to a converged
// dose; where the change exceeds k_sigma times the plain dose's batch sigma the plain
// Monte Carlo value is kept (flag = 1). Outputs nx*ny*nz floats.
ocmc_status ocmc_denoise(ocmc_ctx* c, ocmc_unet* u, float k_sigma, float* dose_out, float* flag_out, int on_device)
{
    if (!c || !u || !dose_out) return ctx_fail(c, OCMC_ERR_ARG, "NULL argument");
    if (!c->have_phantom || c->nvox != u->nvox) return ctx_fail(c, OCMC_ERR_ARG, "network grid differs from phantom");
    if (!(k_sigma > 0.f)) return ctx_fail(c, OCMC_ERR_ARG, "k_sigma must be > 0");
    cudaError_t e = cudaSetDevice(c->device);
    long long n = c->nvox;
    if (e == cudaSuccess && !u->fb) e = cudaMalloc(&u->fb, 4 * n * sizeof(float));
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "allocation");
    float *dd = u->fb, *ds = dd + n, *dout = ds + n, *dflag = dout + n;
    if (on_device) {
        dout = dose_out;
        if (flag_out) dflag = flag_out;
    }
    ocmc_status st = ocmc_get_dose(c, dd, ds, 1);
    if (st == OCMC_OK || st == OCMC_ERR_OVERFLOW || st == OCMC_ERR_TIMEOUT) {
        ocmc_status s2 = ocmc_unet_forward(u, dd, ds, c->d_density, dout, nullptr);
        if (s2 == OCMC_OK) {
            k_fallback<<<grid_for(n), 256>>>(dd, ds, dout, dflag, k_sigma, u->g[0].nx, u->g[0].ny, u->g[0].nz);
            e = cudaGetLastError();
            if (e == cudaSuccess && !on_device) e = cudaMemcpy(dose_out, dout, n * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && !on_device && flag_out) e = cudaMemcpy(flag_out, dflag, n * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) st = ctx_cuda_fail(c, e, "denoise");
            else if (take_kernel_flag(u, nullptr) != OCMC_OK) st = ctx_fail(c, OCMC_ERR_TIMEOUT, u->err);
        } else {
            st = ctx_fail(c, s2, std::string("network: ") + u->err);
        }
    }
    return st;
}

}  // extern "C"
