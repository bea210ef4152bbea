// ocmc_device.cuh -- device building blocks of the transport kernel: the
// counter-based RNG, table lookups from shared memory, interaction samplers
// and voxel geometry. The test kernels use the same functions.
#pragma once
#include "ocmc_internal.h"

namespace ocmc {

// ---- Philox4x32-10 (Salmon et al. 2011) -----------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// A particle's random stream: counter (n/4, history lo, history hi, sub-stream),
// key = the run's seed. Draw n is word n mod 4 of that block, mapped to
// ((x >> 8) + 1) 2^-24 in (0, 1]. The stream depends only on the particle, never
// on the thread that transports it, so the dose is independent of scheduling.
struct Rng {
    uint32_t h0, h1, sub, n, blk;
    uint4 buf;
};

// One out-of-line copy of the generator for draws beyond a step's first block:
// call sites stay small, so the transport kernel's code fits the instruction cache.
static __device__ __noinline__ uint4 philox_block(uint32_t b, uint32_t h0, uint32_t h1, uint32_t sub, uint32_t k0, uint32_t k1)
{
    return philox4x32_10(make_uint4(b, h0, h1, sub), k0, k1);
}

// Every transport step starts on a fresh block: n is rounded up to a multiple of 4
// and that block is generated by all lanes of the warp together (no divergence for
// the first four draws of a step). The rounding depends only on the particle's own
// step sequence, so streams stay independent of scheduling.
__device__ __forceinline__ void rng_step_start(Rng& r, uint32_t k0, uint32_t k1)
{
    r.n = (r.n + 3u) & ~3u;
    r.blk = r.n >> 2;
    r.buf = philox4x32_10(make_uint4(r.blk, r.h0, r.h1, r.sub), k0, k1);
}

__device__ __forceinline__ float rng_u(Rng& r, uint32_t k0, uint32_t k1)
{
    uint32_t b = r.n >> 2;
    if (b != r.blk) {
        r.buf = philox_block(b, r.h0, r.h1, r.sub, k0, k1);
        r.blk = b;
    }
    uint32_t i = r.n & 3u;
    r.n++;
    uint32_t x = i == 0 ? r.buf.x : (i == 1 ? r.buf.y : (i == 2 ? r.buf.z : r.buf.w));
    return (float)((x >> 8) + 1u) * 5.9604644775390625e-08f;
}

__device__ __forceinline__ uint32_t child_sub(uint32_t parent, uint32_t n, uint32_t slot)
{
    uint32_t h = parent * 0x9E3779B1u ^ (n + 0x7F4A7C15u) * 0x85EBCA77u ^ (slot + 1u) * 0xC2B2AE3Du;
    h ^= h >> 16; h *= 0x85EBCA6Bu; h ^= h >> 13; h *= 0xC2B2AE35u; h ^= h >> 16;
    return h == 0u ? 1u : h;
}

// ---- tables in shared memory ---------------------------------------------------------------
// Pointers to material 0's rows of the shared-memory tables; material m's row is m * MS4
// (float4), m * MS2 (float2) or m * MS1 (float) further on.
struct SmemTables {
    float4* ph;     // [m * MS4 + i], i < NE
    float4* el;     // [m * MS4 + i]
    float2* el2;    // [m * MS2 + i]
    float* phmaj;   // NE
    float* rinv;    // [m * MS1 + j], j < NR
    float* msA;     // NG
    float* rmeta;   // [m * MS1 + 0/1]
    float* msc;     // [m * MS1 + 0/1]
};

constexpr float LN_E_LO = -6.907755278982137f;              // ln(1e-3)
constexpr float INV_DLNE = (float)((NE - 1) / 10.373491181781864);   // (NE-1) / ln(E_HI/E_LO)
constexpr float LN_G_LO = -27.631021115928547f;             // ln(1e-12)
constexpr float INV_DLNG = (float)((NG - 1) / (2.70805020110221 + 27.631021115928547));

struct EIdx {
    int i;
    float f;
};

__device__ __forceinline__ EIdx e_index(float E)
{
    float x = (__logf(E) - LN_E_LO) * INV_DLNE;
    x = fminf(fmaxf(x, 0.f), (float)(NE - 1) - 1e-3f);
    EIdx r;
    r.i = (int)x;
    r.f = x - (float)r.i;
    return r;
}

__device__ __forceinline__ float lerp1(float a, float b, float f) { return fmaf(f, b - a, a); }

// ln E at ln R for material m (range-table inversion)
__device__ __forceinline__ float range_to_lnE(const SmemTables& T, int m, float lnR)
{
    float x = (lnR - T.rmeta[m * MS1]) * T.rmeta[m * MS1 + 1];
    x = fminf(fmaxf(x, 0.f), (float)(NR - 1) - 1e-3f);
    int j = (int)x;
    float f = x - (float)j;
    const float* r = T.rinv + m * MS1;
    return lerp1(r[j], r[j + 1], f);
}

// Energy after CSDA slowing over mass thickness X (g/cm^2) from energy E, with
// R = R(E) and g0 = g(ln R): E_end = E exp(g(ln(R - X)) - g0), g the inverse range
// table; exact at X = 0 and monotone in X.
__device__ __forceinline__ float csda_end2(const SmemTables& T, int m, float E, float R, float g0, float X)
{
    float R1 = R - X;
    if (!(R1 > 0.f)) return 0.f;
    float g1 = range_to_lnE(T, m, __logf(R1));
    return fminf(E, E * __expf(g1 - g0));
}

__device__ __forceinline__ float csda_end(const SmemTables& T, int m, float E, float lnR, float X)
{
    return csda_end2(T, m, E, __expf(lnR), range_to_lnE(T, m, lnR), X);
}

// ---- interaction samplers -------------------------------------------------------------------
constexpr int SAMPLE_LIMIT = 10000;
constexpr float MC2F = 0.51099895f;

// Compton scattering: eps = E'/E from the Klein-Nishina cross section by the
// Butcher-Messel decomposition (1/eps and eps envelopes with the rejection
// factor 1 - eps sin^2 / (1 + eps^2)). Returns cos(theta); *eps_out = E'/E.
__device__ __forceinline__ float sample_compton(float E, Rng& r, uint32_t k0, uint32_t k1, float* eps_out, bool* ok)
{
    float k = E / MC2F;
    float e0 = 1.f / (1.f + 2.f * k);
    float a1 = __logf(1.f + 2.f * k);
    float a2 = 0.5f * (1.f - e0 * e0);
    float eps = 1.f, t = 0.f;
    for (int it = 0; it < SAMPLE_LIMIT; ++it) {
        float r1 = rng_u(r, k0, k1), r2 = rng_u(r, k0, k1), r3 = rng_u(r, k0, k1);
        if (r1 * (a1 + a2) < a1) eps = __expf(-a1 * r2);
        else eps = sqrtf(e0 * e0 + (1.f - e0 * e0) * r2);
        eps = fminf(fmaxf(eps, e0), 1.f);
        t = (1.f - eps) / (k * eps);
        float s2 = t * (2.f - t);
        float g = 1.f - eps * s2 / (1.f + eps * eps);
        if (r3 <= g) {
            *eps_out = eps;
            return fmaxf(-1.f, 1.f - t);
        }
    }
    *ok = false;
    *eps_out = 1.f;
    return 1.f;
}

// Moller: eps = W/T on [w_cc/T, 1/2] from the 1/eps^2 envelope, accepted with
// g(eps) / (2 + c/4), g = 1 + (eps/(1-eps))^2 + c eps^2 - d eps/(1-eps).
__device__ __forceinline__ float sample_moller(float T, float wcc, Rng& r, uint32_t k0, uint32_t k1, bool* ok)
{
    float tau = T / MC2F, g = tau + 1.f;
    float c = (tau / g) * (tau / g), d = (2.f * tau + 1.f) / (g * g);
    float e0 = wcc / T, gmax = 2.f + 0.25f * c;
    for (int it = 0; it < SAMPLE_LIMIT; ++it) {
        float r1 = rng_u(r, k0, k1), r2 = rng_u(r, k0, k1);
        float eps = e0 / (1.f - r1 * (1.f - 2.f * e0));
        eps = fminf(fmaxf(eps, e0), 0.5f);
        float q = eps / (1.f - eps);
        float gv = 1.f + q * q + c * eps * eps - d * q;
        if (r2 * gmax <= gv) return eps;
    }
    *ok = false;
    return e0;
}

// Bremsstrahlung photon energy on [w_cb, T] from the 1/k envelope, accepted with
// [(4/3 - 4/3 y + y^2) S1 + (1 - y) S2] / (4/3 S1 + S2), y = k / (T + mc^2).
__device__ __forceinline__ float sample_brems(float T, float wcb, float S1, float S2, Rng& r, uint32_t k0, uint32_t k1,
                                              bool* ok)
{
    float E = T + MC2F, lr = __logf(T / wcb);
    float gmax = (4.f / 3.f) * S1 + S2;
    for (int it = 0; it < SAMPLE_LIMIT; ++it) {
        float r1 = rng_u(r, k0, k1), r2 = rng_u(r, k0, k1);
        float k = fminf(wcb * __expf(r1 * lr), T);
        float y = k / E;
        float gv = (4.f / 3.f - (4.f / 3.f) * y + y * y) * S1 + (1.f - y) * S2;
        if (r2 * gmax <= gv) return fmaxf(k, wcb);
    }
    *ok = false;
    return wcb;
}

// Multiple-scattering cos(theta) for G1 = s / lambda_1: Wentzel distribution with
// screening A chosen so that <1 - cos> = 1 - exp(-G1) (table of ln A at ln G1).
__device__ __forceinline__ float sample_ms(const SmemTables& T, float G1, Rng& r, uint32_t k0, uint32_t k1)
{
    if (!(G1 >= 1e-12f)) return 1.f;
    float xi = rng_u(r, k0, k1);
    if (G1 >= 15.f) return 2.f * xi - 1.f;
    float x = (__logf(G1) - LN_G_LO) * INV_DLNG;
    x = fminf(fmaxf(x, 0.f), (float)(NG - 1) - 1e-3f);
    int j = (int)x;
    float A = __expf(lerp1(T.msA[j], T.msA[j + 1], x - (float)j));
    float q = 1.f - xi;                              // [0, 1)
    float u = 2.f * A * q / (1.f + A - q);
    return fmaxf(-1.f, 1.f - u);
}

// The GPU's global nanosecond timer (consistent across SMs).
__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Rotate unit direction (u,v,w) by polar cosine mu and azimuth phi = 2 pi xi.
__device__ __forceinline__ void rotate(float& u, float& v, float& w, float mu, float xi)
{
    float st = sqrtf(fmaxf(0.f, 1.f - mu * mu));
    float sp, cp;
    __sincosf(6.283185307179586f * xi, &sp, &cp);
    // sin of the polar angle of (u, v, w) from its own components: 1 - w^2 would cancel near
    // the poles and give the frame a wrong scale there. Explicitly rounded products and an
    // explicit reciprocal square root: the compiler may not contract or rewrite them differently
    // in different instantiations of the transport kernel, which keeps the tally bit-identical
    // across launch shapes.
    const float s2 = __fmaf_rn(u, u, __fmul_rn(v, v));
    const float is = rsqrtf(s2), s = __fmul_rn(s2, is);
    float nu, nv, nw;
    if (s2 > 1e-20f) {
        nu = u * mu + st * (u * w * cp - v * sp) * is;
        nv = v * mu + st * (v * w * cp + u * sp) * is;
        nw = w * mu - s * st * cp;
    } else {
        float sg = w >= 0.f ? 1.f : -1.f;
        nu = st * cp;
        nv = st * sp;
        nw = sg * mu;
    }
    float inv = rsqrtf(nu * nu + nv * nv + nw * nw);
    u = nu * inv;
    v = nv * inv;
    w = nw * inv;
}

// ---- voxel geometry -----------------------------------------------------------------------
// Distance from (x,y,z) along (u,v,w) to the faces of voxel (ix,iy,iz);
// *face = axis*2 + (direction > 0).
__device__ __forceinline__ float dist_to_face(float x, float y, float z, float u, float v, float w, int ix, int iy,
                                              int iz, float dx, float dy, float dz, int* face)
{
    float best = 3.0e38f;
    int f = 0;
    if (u != 0.f) {
        float t = fmaxf(__fdividef((u > 0.f ? (float)(ix + 1) : (float)ix) * dx - x, u), 0.f);
        if (t < best) { best = t; f = u > 0.f ? 1 : 0; }
    }
    if (v != 0.f) {
        float t = fmaxf(__fdividef((v > 0.f ? (float)(iy + 1) : (float)iy) * dy - y, v), 0.f);
        if (t < best) { best = t; f = v > 0.f ? 3 : 2; }
    }
    if (w != 0.f) {
        float t = fmaxf(__fdividef((w > 0.f ? (float)(iz + 1) : (float)iz) * dz - z, w), 0.f);
        if (t < best) { best = t; f = w > 0.f ? 5 : 4; }
    }
    *face = f;
    return best;
}

}  // namespace ocmc

namespace ocmc {

// ---- shared-memory staging of the tables ------------------------------------------------
__device__ __forceinline__ SmemTables carve_tables(unsigned char* smem)
{
    SmemTables T;
    T.phmaj = reinterpret_cast<float*>(smem);
    T.msA = T.phmaj + NE;
    T.ph = reinterpret_cast<float4*>(smem + SM_SHARED_BYTES);
    T.el = T.ph + NE;
    T.el2 = reinterpret_cast<float2*>(T.el + NE);
    T.rinv = reinterpret_cast<float*>(T.el2 + NE);
    T.rmeta = T.rinv + NR;
    T.msc = T.rmeta + 2;
    return T;
}

__device__ __forceinline__ SmemTables stage_tables(const Tables& t, unsigned char* smem)
{
    SmemTables T = carve_tables(smem);
    const int nm = t.n_mat;
    for (int i = threadIdx.x; i < nm * NE; i += blockDim.x) {
        const int m = i / NE, k = i - m * NE;
        T.ph[m * MS4 + k] = t.ph[i];
        T.el[m * MS4 + k] = t.el[i];
        T.el2[m * MS2 + k] = t.el2[i];
    }
    for (int i = threadIdx.x; i < NE; i += blockDim.x) T.phmaj[i] = t.phmaj[i];
    for (int i = threadIdx.x; i < nm * NR; i += blockDim.x) {
        const int m = i / NR, k = i - m * NR;
        T.rinv[m * MS1 + k] = t.rinv[i];
    }
    for (int i = threadIdx.x; i < NG; i += blockDim.x) T.msA[i] = t.msA[i];
    if (threadIdx.x < 2 * nm) {
        const int m = threadIdx.x >> 1, k = threadIdx.x & 1;
        T.rmeta[m * MS1 + k] = t.rmeta[threadIdx.x];
        T.msc[m * MS1 + k] = t.msc[threadIdx.x];
    }
    __syncthreads();
    return T;
}

// ---- particle state in registers ------------------------------------------------------------
enum { PHOTON = 0, ELECTRON = 1, POSITRON = 2 };

struct Lane {
    float x, y, z, u, v, w, E;
    int ix, iy, iz, type, batch, steps;
    Rng r;
};

__device__ __forceinline__ int batch_of(uint32_t h0, uint32_t h1, int B)
{
    if (h1 == 0u) return (int)(h0 % (uint32_t)B);          // 32-bit path for ids below 2^32
    unsigned long long h = ((unsigned long long)h1 << 32) | h0;
    return (int)(h % (unsigned long long)B);
}

// Move a particle starting at O with unit direction d (line parameter t >= tmin) through
// vacuum to the phantom box; sets position, direction and voxel. False if it misses.
__device__ __forceinline__ bool enter_box(const TransportArgs& a, const float* O, const float* d, float tmin, Lane& p)
{
    const float Lb[3] = {a.nx * a.dx, a.ny * a.dy, a.nz * a.dz};
    float tmax = 3.0e38f;
    int ent = -1;
    for (int k = 0; k < 3; ++k) {
        if (fabsf(d[k]) < 1e-30f) {
            if (O[k] < 0.f || O[k] > Lb[k]) return false;
            continue;
        }
        float t1 = (0.f - O[k]) / d[k], t2 = (Lb[k] - O[k]) / d[k];
        float tn = fminf(t1, t2), tx = fmaxf(t1, t2);
        if (tn > tmin) { tmin = tn; ent = k * 2 + (t1 < t2 ? 0 : 1); }
        tmax = fminf(tmax, tx);
    }
    if (!(tmax > tmin)) return false;
    p.x = O[0] + tmin * d[0];
    p.y = O[1] + tmin * d[1];
    p.z = O[2] + tmin * d[2];
    if (ent >= 0) {                              // put the entry point exactly on its face
        float f = (ent & 1) ? Lb[ent >> 1] : 0.f;
        if ((ent >> 1) == 0) p.x = f; else if ((ent >> 1) == 1) p.y = f; else p.z = f;
    }
    p.u = d[0]; p.v = d[1]; p.w = d[2];
    p.ix = min(max((int)floorf(p.x / a.dx), 0), a.nx - 1);
    p.iy = min(max((int)floorf(p.y / a.dy), 0), a.ny - 1);
    p.iz = min(max((int)floorf(p.z / a.dz), 0), a.nz - 1);
    return true;
}


// Source particle of history h of a beam with geometry g (Sec. 2.2 "Materials": point
// source at SSD with the field defined at the surface, or a parallel beam; energy
// bins in decreasing energy, Sec. 2.2.1). Draws: energy within the bin, then the
// two field coordinates. Returns false if the ray misses the phantom; p.E is set
// either way. The stream is (history lo, history hi ^ h1_tag, sub-stream 0).
template <class G>
__device__ __forceinline__ bool init_source(const TransportArgs& a, const G& g, const unsigned long long* bound,
                                            unsigned long long h, uint32_t h1_tag, Lane& p)
{
    const SourceDev& s = a.src;
    p.r.h0 = (uint32_t)h;
    p.r.h1 = (uint32_t)(h >> 32) ^ h1_tag;
    p.r.sub = 0u;
    p.r.n = 0u;
    p.r.blk = 0xFFFFFFFFu;
    p.type = s.particle == 0 ? PHOTON : ELECTRON;
    p.steps = 0;
    int lo = 0, hi = s.n_bins - 1;               // last q with bound[q] <= h
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (bound[mid] <= h) lo = mid; else hi = mid - 1;
    }
    int bin = s.order[lo];
    float e0 = s.lo[bin], e1 = s.hi[bin];
    p.E = e0 + rng_u(p.r, a.key0, a.key1) * (e1 - e0);
    float fa = rng_u(p.r, a.key0, a.key1) - 0.5f, fb = rng_u(p.r, a.key0, a.key1) - 0.5f;
    float P[3], O[3], d[3];
    for (int k = 0; k < 3; ++k) P[k] = g.iso[k] + fa * g.fx * g.e1[k] + fb * g.fy * g.e2[k];
    float tmin;
    if (g.ssd > 0.f) {
        for (int k = 0; k < 3; ++k) { O[k] = g.iso[k] - g.ssd * g.dir[k]; d[k] = P[k] - O[k]; }
        float inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int k = 0; k < 3; ++k) d[k] *= inv;
        tmin = 0.f;
    } else {
        for (int k = 0; k < 3; ++k) { O[k] = P[k]; d[k] = g.dir[k]; }
        tmin = -3.0e38f;
    }
    return enter_box(a, O, d, tmin, p);
}

// Single-beam source: history h of the run, batch = h mod B.
__device__ __forceinline__ bool init_primary(const TransportArgs& a, unsigned long long h, Lane& p)
{
    p.batch = batch_of((uint32_t)h, (uint32_t)(h >> 32), a.pp.n_batches);
    return init_source(a, a.src, a.src.bound, h, a.stream_tag, p);
}

// Phase-space source: history h starts from record h mod ps_n, moved forward through vacuum to
// the phantom (a record inside starts where it is); no random number is drawn before the first
// transport step. Stream (history lo, history hi ^ stream tag, sub-stream 0), batch h mod B.
__device__ __forceinline__ bool init_phase_space(const TransportArgs& a, unsigned long long h, Lane& p)
{
    const PsRec r = a.ps[h % a.ps_n];
    p.batch = batch_of((uint32_t)h, (uint32_t)(h >> 32), a.pp.n_batches);
    p.r.h0 = (uint32_t)h;
    p.r.h1 = (uint32_t)(h >> 32) ^ a.stream_tag;
    p.r.sub = 0u;
    p.r.n = 0u;
    p.r.blk = 0xFFFFFFFFu;
    p.type = r.type == 0 ? PHOTON : (r.type == 1 ? ELECTRON : POSITRON);
    p.steps = 0;
    p.E = r.E;
    float O[3] = {r.x, r.y, r.z}, d[3] = {r.u, r.v, r.w};
    const float inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) d[k] *= inv;
    return enter_box(a, O, d, 0.f, p);
}

// Batched beamlets: global history g -> (beamlet b, its history h); stream high word
// tagged with 0x80000000 | b, which also tells the tally which beamlet a particle
// belongs to.
__device__ __forceinline__ bool init_beamlet(const TransportArgs& a, unsigned long long g, Lane& p)
{
    int lo = 0, hi = a.n_beamlets - 1;           // last b with prefix[b] <= g
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a.bl_prefix[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const BeamletDev& B = a.beamlets[lo];
    p.batch = 0;
    return init_source(a, B, B.bound, g - a.bl_prefix[lo], BL_TAG | (uint32_t)lo, p);
}

}  // namespace ocmc
