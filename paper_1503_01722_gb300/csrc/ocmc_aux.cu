// ocmc_aux.cu -- dose finalisation and the test kernels that expose the transport
// kernel's building blocks (RNG, source, samplers, tables) to the test suite.
#include "ocmc_device.cuh"

#include <algorithm>

namespace ocmc {

namespace {

// int64 -> float without a 64-bit conversion (which runs on GB300's narrow FP64 pipe): the high
// and low words convert exactly or to nearest, so the result is within 2 ulp of the exact value.
__device__ __forceinline__ float i64_to_f32(long long x)
{
    const int hi = (int)(x >> 32);
    const unsigned lo = (unsigned)x;
    return fmaf(__int2float_rn(hi), 4294967296.f, __uint2float_rn(lo));
}

// D_v = sum_b tally / (2^28 rho_v V N) in MeV/g per source particle (Sec. 2.2 "Materials");
// sigma_D by the batch method (Sec. 3.1): sqrt(sum_b (D_b - D)^2 / (B (B - 1))) with the batch
// means D_b = tally_b / (2^28 rho_v V n_b). Grid-stride over voxels. The integer sum is exact; the
// rest is FP32, like the outputs (FP64 here made this kernel 13x slower than its memory traffic on
// GB300's narrow FP64 pipe).
__global__ void k_finalize(const long long* __restrict__ tally, const float* __restrict__ density, int B, long long nvox,
                           float voxel_volume, const float* __restrict__ w_nb, float inv_n, float* dose,
                           float* sigma)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        const float rho = density[v];
        if (!(rho > 0.f)) {
            dose[v] = 0.f;
            if (sigma) sigma[v] = 0.f;
            continue;
        }
        const float scale = inv_n / (rho * voxel_volume * 268435456.f);   // MeV/g per history per unit
        long long tot = 0;
        for (int b = 0; b < B; ++b) tot += tally[(long long)b * nvox + v];
        const float tf = i64_to_f32(tot);
        dose[v] = tf * scale;
        if (sigma) {
            // batch b's mean relative to the whole: tally_b * (N / n_b) - tot, in units of 2^32 tally
            // units so that the squares stay in FP32's range for any int64 tally
            float ss = 0.f;
            if (B > 1) {
                for (int b = 0; b < B; ++b) {
                    const float d = fmaf(i64_to_f32(tally[(long long)b * nvox + v]), w_nb[b], -tf) * 2.3283064365386963e-10f;
                    ss = fmaf(d, d, ss);
                }
                ss /= (float)B * (float)(B - 1);
            }
            sigma[v] = sqrtf(ss) * 4294967296.f * scale;
        }
    }
}

__global__ void k_test_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t first,
                              uint32_t n, uint32_t* out)
{
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint4 r = philox4x32_10(make_uint4(first + j, c1, c2, c3), k0, k1);
    out[4 * j] = r.x;
    out[4 * j + 1] = r.y;
    out[4 * j + 2] = r.z;
    out[4 * j + 3] = r.w;
}

__global__ void k_test_rotate(const float* dir, const float* mu, const float* xi, int n, float* out)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float u = dir[3 * j], v = dir[3 * j + 1], w = dir[3 * j + 2];
    rotate(u, v, w, mu[j], xi[j]);
    out[3 * j] = u;
    out[3 * j + 1] = v;
    out[3 * j + 2] = w;
}

__global__ void k_test_source(const TransportArgs a, unsigned long long first, unsigned long long count, float* out)
{
    unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (j >= count) return;
    Lane p;
    bool in = a.ps ? init_phase_space(a, first + j, p) : init_primary(a, first + j, p);
    float* o = out + 8 * j;
    o[0] = in ? p.x : 0.f; o[1] = in ? p.y : 0.f; o[2] = in ? p.z : 0.f;
    o[3] = in ? p.u : 0.f; o[4] = in ? p.v : 0.f; o[5] = in ? p.w : 0.f;
    o[6] = p.E;
    o[7] = in ? 1.f : 0.f;
}

__global__ void k_test_sample(const TransportArgs a, int kind, int m, float E, float aux, unsigned long long n,
                              float* out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemTables T = stage_tables(a.t, smem);
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        Rng r;
        r.h0 = (uint32_t)j; r.h1 = (uint32_t)(j >> 32); r.sub = 0x5A5Au + (uint32_t)kind; r.n = 0; r.blk = 0xFFFFFFFFu;
        bool ok = true;
        float v = 0.f, eps;
        if (kind == 0) v = sample_compton(E, r, a.key0, a.key1, &eps, &ok);
        else if (kind == 1) v = sample_moller(E, a.pp.w_cc, r, a.key0, a.key1, &ok);
        else if (kind == 2) v = sample_brems(E, a.pp.w_cb, T.msc[m * MS1], T.msc[m * MS1 + 1], r, a.key0, a.key1, &ok);
        else if (kind == 3) v = sample_ms(T, aux, r, a.key0, a.key1);
        out[j] = ok ? v : __int_as_float(0x7FC00000);
    }
}

__global__ void k_test_tables(const TransportArgs a, int m, const float* E, int n, float* out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemTables T = stage_tables(a.t, smem);
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    EIdx ei = e_index(E[j]);
    const int mb = m * MS4;
    float4 pa = T.ph[mb + ei.i], pb = T.ph[mb + ei.i + 1];
    float mt = __expf(lerp1(pa.x, pb.x, ei.f));
    float4 A = T.el[mb + ei.i], B = T.el[mb + ei.i + 1];
    float* o = out + 8 * j;
    o[0] = mt;
    o[1] = mt * lerp1(pa.y, pb.y, ei.f);
    o[2] = mt * lerp1(pa.z, pb.z, ei.f);
    o[3] = __expf(lerp1(A.x, B.x, ei.f));
    o[4] = lerp1(A.y, B.y, ei.f);
    o[5] = lerp1(A.z, B.z, ei.f);
    o[6] = lerp1(A.w, B.w, ei.f);
    o[7] = T.el2[m * MS2 + ei.i].y;
}

__global__ void k_test_csda(const TransportArgs a, int m, const float* Tk, const float* X, int n, float* out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemTables T = stage_tables(a.t, smem);
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    EIdx ei = e_index(Tk[j]);
    float lnR = lerp1(T.el[m * MS4 + ei.i].x, T.el[m * MS4 + ei.i + 1].x, ei.f);
    out[j] = csda_end(T, m, Tk[j], lnR, X[j]);
}

__global__ void k_add_tally(long long* t, const long long* in, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        t[i] += in[i];
}

__global__ void k_sum_tally(const long long* t, long long n, unsigned long long* out)
{
    __shared__ long long red[32];
    long long s = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += t[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
        if (threadIdx.x == 0) atomicAdd(out, (unsigned long long)s);
    }
}

// ---- batched-beamlet tables ------------------------------------------------------------------
__global__ void k_bl_count(const unsigned int* keys, const unsigned long long* offs, const unsigned int* caps,
                           unsigned long long* nnz)
{
    const int b = blockIdx.x;
    const unsigned int* k = keys + offs[b];
    unsigned long long c = 0;
    for (unsigned int i = threadIdx.x; i < caps[b]; i += blockDim.x) c += k[i] != BL_EMPTY;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(nnz + b, c);
}

__global__ void k_bl_scatter(const unsigned int* keys, const unsigned long long* vals, unsigned long long cap,
                             long long* dense)
{
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < cap;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned int k = keys[i];
        if (k != BL_EMPTY) dense[k] = (long long)vals[i];   // keys are unique within a table
    }
}

constexpr int CHUNK = 1024;   // voxels per compaction block (= threads per block)

__global__ void k_chunk_count(const long long* dense, long long nvox, unsigned int* counts)
{
    long long v = blockIdx.x * (long long)CHUNK + threadIdx.x;
    int nz = v < nvox && dense[v] != 0;
    int c = __syncthreads_count(nz);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// exclusive scan of n counts in place (one block); total to *nnz
__global__ void k_scan_counts(unsigned int* counts, int n, unsigned long long* nnz)
{
    __shared__ unsigned int part[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(n, b0 + per);
    unsigned int s = 0;
    for (int i = b0; i < b1; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        unsigned int v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned int run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int i = b0; i < b1; ++i) {
        unsigned int c = counts[i];
        counts[i] = run;
        run += c;
    }
    if (threadIdx.x == blockDim.x - 1) *nnz = part[threadIdx.x];
}

__global__ void k_compact(const long long* dense, long long nvox, const unsigned int* offsets, int* idx,
                          long long* raw, float* dose, const float* density, double scale)
{
    __shared__ unsigned int warp_base[CHUNK / 32];
    long long v = blockIdx.x * (long long)CHUNK + threadIdx.x;
    long long q = v < nvox ? dense[v] : 0;
    bool nz = q != 0;
    unsigned int bal = __ballot_sync(0xFFFFFFFFu, nz);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_base[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int r = 0;
        for (int i = 0; i < CHUNK / 32; ++i) { unsigned int c = warp_base[i]; warp_base[i] = r; r += c; }
    }
    __syncthreads();
    if (nz) {
        unsigned int pos = offsets[blockIdx.x] + warp_base[w] + __popc(bal & ((1u << lane) - 1u));
        if (idx) idx[pos] = (int)v;
        if (raw) raw[pos] = q;
        if (dose) {
            float rho = density[v];
            dose[pos] = rho > 0.f ? (float)((double)q * scale / rho) : 0.f;
        }
    }
}

}  // namespace

// Count phase-space records that cannot be transported: unknown type, energy not in
// (0, 1e4) MeV, non-finite position, zero or non-finite direction.
__global__ void k_ps_validate(const PsRec* ps, unsigned long long n, unsigned long long* bad)
{
    unsigned long long nb = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const PsRec r = ps[i];
        const float d2 = r.u * r.u + r.v * r.v + r.w * r.w;
        const bool ok = r.type >= 0 && r.type <= 2 && r.E > 0.f && r.E < 1e4f && isfinite(r.x) && isfinite(r.y) &&
                        isfinite(r.z) && d2 > 0.f && isfinite(d2);
        nb += ok ? 0 : 1;
    }
    if (nb) atomicAdd(bad, nb);
}

cudaError_t launch_ps_validate(const PsRec* ps, unsigned long long n, unsigned long long* bad, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    unsigned blocks = (unsigned)std::min<unsigned long long>((n + 255) / 256, 4096);
    k_ps_validate<<<blocks, 256, 0, s>>>(ps, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_bl_count(const unsigned int* keys, const unsigned long long* offs, const unsigned int* caps, int n,
                            unsigned long long* nnz, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(nnz, 0, sizeof(unsigned long long) * n, s);
    if (e != cudaSuccess) return e;
    k_bl_count<<<n, 256, 0, s>>>(keys, offs, caps, nnz);
    return cudaGetLastError();
}

// Entries of one beamlet table in increasing voxel order (deterministic whatever the
// slot order): scatter into a dense scratch, count per 1024-voxel chunk, scan, compact.
cudaError_t launch_bl_extract(const unsigned int* keys, const unsigned long long* vals, unsigned long long cap,
                              long long nvox, long long* dense, unsigned int* block_counts, int* idx_out,
                              long long* raw_out, float* dose_out, const float* density, double scale,
                              unsigned long long* nnz_out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(dense, 0, sizeof(long long) * nvox, s);
    if (e != cudaSuccess) return e;
    int sb = (int)std::min<unsigned long long>((cap + 255) / 256, 152 * 8);
    k_bl_scatter<<<sb > 0 ? sb : 1, 256, 0, s>>>(keys, vals, cap, dense);
    int nchunks = (int)((nvox + CHUNK - 1) / CHUNK);
    k_chunk_count<<<nchunks, CHUNK, 0, s>>>(dense, nvox, block_counts);
    k_scan_counts<<<1, 1024, 0, s>>>(block_counts, nchunks, nnz_out);
    if (idx_out || raw_out || dose_out)
        k_compact<<<nchunks, CHUNK, 0, s>>>(dense, nvox, block_counts, idx_out, raw_out, dose_out, density, scale);
    return cudaGetLastError();
}

cudaError_t launch_add_tally(long long* tally, const long long* in, long long n, cudaStream_t s)
{
    k_add_tally<<<1024, 256, 0, s>>>(tally, in, n);
    return cudaGetLastError();
}

cudaError_t launch_sum_tally(const long long* tally, long long n, unsigned long long* out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_sum_tally<<<1024, 256, 0, s>>>(tally, n, out);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const long long* tally, const float* density, int B, long long nvox, double voxel_volume,
                            const float* w_nb, double inv_n, float* dose, float* sigma, cudaStream_t s)
{
    int blocks = (int)std::min<long long>((nvox + 255) / 256, 152 * 16);
    k_finalize<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(tally, density, B, nvox, (float)voxel_volume, w_nb,
                                                       (float)inv_n, dose, sigma);
    return cudaGetLastError();
}

cudaError_t launch_test_philox(uint32_t key0, uint32_t key1, uint32_t c1, uint32_t c2, uint32_t c3,
                               uint32_t first_block, uint32_t n_blocks, uint32_t* out, cudaStream_t s)
{
    k_test_philox<<<(n_blocks + 255) / 256, 256, 0, s>>>(key0, key1, c1, c2, c3, first_block, n_blocks, out);
    return cudaGetLastError();
}

cudaError_t launch_test_rotate(const float* dir, const float* mu, const float* xi, int n, float* out, cudaStream_t s)
{
    k_test_rotate<<<(n + 255) / 256, 256, 0, s>>>(dir, mu, xi, n, out);
    return cudaGetLastError();
}

cudaError_t launch_test_source(const TransportArgs& a, unsigned long long n_total, unsigned long long first,
                               unsigned long long count, float* out, cudaStream_t s)
{
    (void)n_total;
    k_test_source<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(a, first, count, out);
    return cudaGetLastError();
}

cudaError_t launch_test_sample(const TransportArgs& a, int kind, int m, float E, float aux, unsigned long long n,
                               float* out, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_test_sample, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_table_bytes(a.t.n_mat));
    if (e != cudaSuccess) return e;
    k_test_sample<<<152 * 2, 256, smem_table_bytes(a.t.n_mat), s>>>(a, kind, m, E, aux, n, out);
    return cudaGetLastError();
}

cudaError_t launch_test_tables(const TransportArgs& a, int m, const float* E, int n, float* out, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_test_tables, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_table_bytes(a.t.n_mat));
    if (e != cudaSuccess) return e;
    k_test_tables<<<(n + 255) / 256, 256, smem_table_bytes(a.t.n_mat), s>>>(a, m, E, n, out);
    return cudaGetLastError();
}

cudaError_t launch_test_csda(const TransportArgs& a, int m, const float* T, const float* X, int n, float* out,
                             cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_test_csda, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_table_bytes(a.t.n_mat));
    if (e != cudaSuccess) return e;
    k_test_csda<<<(n + 255) / 256, 256, smem_table_bytes(a.t.n_mat), s>>>(a, m, T, X, n, out);
    return cudaGetLastError();
}

}  // namespace ocmc
