// ocmc_transport.cu -- persistent coupled photon-electron transport kernel.
//
// Method (Tian et al., Sec. 2.1): photons fly by Woodcock tracking against a
// phantom-wide majorant and interact by Compton scattering, photoelectric
// absorption or pair production; electrons and positrons take Class II
// condensed-history steps d = min(d_vox, d_maxs, d_maxe, d_event), each inside
// one voxel, with a random-hinge multiple-scattering deflection, CSDA energy
// loss deposited in the step's voxel, and discrete Moller / bremsstrahlung
// events sampled by Woodcock tracking in energy; positrons annihilate into two
// photons at the end of their track.
//
// Scheduling (Sec. 2.2.1, Table 1): the paper launches batches of up to M
// particles of one type, taken from the photon stack, the electron stack or
// the source. Here every warp runs that loop by itself inside one persistent
// launch: its 32 lanes always hold particles of one kind (warp mode: photons,
// or charged particles, which wait on two stacks split by energy class); once
// enough lanes are free they refill from the warp's own stack of that kind,
// then from the source (energy-sorted history ids from a global counter); the
// warp moves to the fullest other stack when its lanes run dry or that stack
// grows large. Secondaries are pushed to the warp's stacks. A warp ends when
// the source is exhausted and its stacks are empty; no warp ever waits on
// another.
//
// Dose tally (Sec. 2.2.2): 64-bit fixed-point integer atomics (2^-28 MeV
// units) into the tally of batch (history id mod B). Integer addition is
// associative and every particle's random stream is keyed by its lineage, so
// the tally is bit-identical for any launch configuration and timing.
#include "ocmc_device.cuh"

namespace ocmc {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int MAX_WARPS = 32;
constexpr int STEP_LIMIT = 1 << 22;

// BL: batched-beamlet mode (sparse hash tallies) or single-beam mode (dense tally);
// a compile-time flag so the single-beam kernel carries no beamlet code.
template <bool BL>
struct CtxT {
    static constexpr bool beamlets = BL;
    const TransportArgs& a;
    const SmemTables& T;
    PRec* stk;                   // warp's stacks: [0, cap) photons, [cap, 2cap) charged, [2cap, 3cap) slow charged
    int* top;                    // shared: top[0] photons, top[1] charged, top[2] charged below e_split
    unsigned long long* st;      // shared block statistics
    float inv_dx, inv_dy, inv_dz, Lx, Ly, Lz;
    bool ok;
};

template <class C>
__device__ __forceinline__ void stat_add(C& c, int k, unsigned long long v) { atomicAdd(c.st + k, v); }

// Checks build: a lane whose voxel index lies outside the grid flags ERR_BOUNDS (and its
// particle is ended by the caller before any access). Always false in the normal build.
template <class C>
__device__ __forceinline__ bool vox_bad(const C& c, const Lane& p)
{
    if constexpr (OCMC_CHECKS) {
        if (p.ix < 0 || p.iy < 0 || p.iz < 0 || p.ix >= c.a.nx || p.iy >= c.a.ny || p.iz >= c.a.nz) {
            atomicOr(c.a.err, ERR_BOUNDS);
            return true;
        }
    }
    return false;
}

// Stack of a waiting charged particle: 1, or 2 below the energy-class boundary (e_split is 0
// when the warps keep a single charged stack, so that everything then goes to stack 1).
__device__ __forceinline__ int charged_stack(const TransportArgs& a, float E) { return E < a.e_split ? 2 : 1; }

// fixed-point energy (round to nearest even) with 32-bit conversions only: below 2^32 units
// (16 MeV) directly; above, q is a float >= 2^32 and therefore a multiple of 2^9, so q / 2^8 is
// an integer below 2^32 for any energy under 4 GeV and the result is exact (no 64-bit
// float-to-integer conversion, which would occupy the FP64 pipe)
__device__ __forceinline__ unsigned long long fx(float e)
{
    float q = e * TALLY_SCALE;
    return q < 4294967040.f ? (unsigned long long)__float2uint_rn(q)
                            : (unsigned long long)__float2uint_rn(q * 0.00390625f) << 8;
}

// Batched-beamlet tally: add q to voxel v of beamlet b's open-addressing table
// (linear probing, key claimed by compare-and-swap). A full table sets the
// beamlet's overflow flag; the host then enlarges that table and runs again.
__device__ __forceinline__ void hash_add(const TransportArgs& a, uint32_t b, uint32_t v, unsigned long long q)
{
    const BeamletDev& B = a.beamlets[b];
    unsigned int* keys = a.bl_keys + B.table_off;
    unsigned long long* vals = a.bl_vals + B.table_off;
    const uint32_t mask = B.cap_mask;
    uint32_t h = v * 0x9E3779B1u;
    uint32_t s = (h ^ (h >> 15)) & mask;
    for (int probe = 0; probe <= (int)min(mask, 4095u); ++probe) {
        uint32_t k = *((volatile unsigned int*)(keys + s));
        if (k == BL_EMPTY) k = atomicCAS(keys + s, BL_EMPTY, v);
        if (k == BL_EMPTY || k == v) {
            atomicAdd(vals + s, q);
            return;
        }
        s = (s + 1u) & mask;
    }
    atomicOr(a.bl_overflow + b, 1u);
}

template <class C>
__device__ __forceinline__ void deposit(C& c, const Lane& p, int ix, int iy, int iz, float dE)
{
    if (dE > 0.f) {
        const int v = ix + c.a.nx * (iy + c.a.ny * iz);     // grids have at most 1024^3 voxels
        if constexpr (OCMC_CHECKS) {
            if (ix < 0 || iy < 0 || iz < 0 || ix >= c.a.nx || iy >= c.a.ny || iz >= c.a.nz ||
                (!C::beamlets && (p.batch < 0 || p.batch >= c.a.pp.n_batches))) {
                atomicOr(c.a.err, ERR_BOUNDS);
                return;
            }
        }
        if constexpr (C::beamlets) hash_add(c.a, p.r.h1 & ~BL_TAG, (uint32_t)v, fx(dE));
        else atomicAdd(c.a.tally + (long long)p.batch * c.a.nvox + v, fx(dE));
    }
}

template <class C>
__device__ __forceinline__ void push(C& c, int t, float x, float y, float z, float E, float u, float v, float w, int ix,
                                     int iy, int iz, int type, uint32_t h0, uint32_t h1, uint32_t sub)
{
    int slot = atomicAdd(c.top + t, 1);
    if (slot >= c.a.cap) {
        atomicOr(c.a.err, ERR_OVERFLOW);
        stat_add(c, ST_DROPPED, 1);
        stat_add(c, ST_E_DROPPED, fx(E));
        return;
    }
    PRec* r = c.stk + (size_t)t * c.a.cap + slot;
    uint32_t vt = (uint32_t)ix | ((uint32_t)iy << 10) | ((uint32_t)iz << 20) | ((uint32_t)type << 30);
    uint4* q = reinterpret_cast<uint4*>(r);
    q[0] = make_uint4(__float_as_uint(x), __float_as_uint(y), __float_as_uint(z), __float_as_uint(E));
    q[1] = make_uint4(__float_as_uint(u), __float_as_uint(v), __float_as_uint(w), vt);
    q[2] = make_uint4(h0, h1, sub, 0u);
}

template <class C>
__device__ __forceinline__ void push_lane(C& c, int t, const Lane& p)
{
    int slot = atomicAdd(c.top + t, 1);
    if (slot >= c.a.cap) {
        atomicOr(c.a.err, ERR_OVERFLOW);
        stat_add(c, ST_DROPPED, 1);
        stat_add(c, ST_E_DROPPED, fx(p.E));
        return;
    }
    PRec* r = c.stk + (size_t)t * c.a.cap + slot;
    uint32_t vt = (uint32_t)p.ix | ((uint32_t)p.iy << 10) | ((uint32_t)p.iz << 20) | ((uint32_t)p.type << 30);
    uint4* q = reinterpret_cast<uint4*>(r);
    q[0] = make_uint4(__float_as_uint(p.x), __float_as_uint(p.y), __float_as_uint(p.z), __float_as_uint(p.E));
    q[1] = make_uint4(__float_as_uint(p.u), __float_as_uint(p.v), __float_as_uint(p.w), vt);
    q[2] = make_uint4(p.r.h0, p.r.h1, p.r.sub, p.r.n);
}

template <class C>
__device__ __forceinline__ void pop_lane(const C& c, int t, int slot, Lane& p)
{
    if constexpr (OCMC_CHECKS) {
        if (slot < 0 || slot >= c.a.cap || t < 0 || t >= c.a.nstk) {
            atomicOr(c.a.err, ERR_BOUNDS);
            slot = 0;
            t = 0;
        }
    }
    const uint4* q = reinterpret_cast<const uint4*>(c.stk + (size_t)t * c.a.cap + slot);
    uint4 a = q[0], b = q[1], d = q[2];
    p.x = __uint_as_float(a.x); p.y = __uint_as_float(a.y); p.z = __uint_as_float(a.z); p.E = __uint_as_float(a.w);
    p.u = __uint_as_float(b.x); p.v = __uint_as_float(b.y); p.w = __uint_as_float(b.z);
    p.ix = b.w & 1023u; p.iy = (b.w >> 10) & 1023u; p.iz = (b.w >> 20) & 1023u; p.type = b.w >> 30;
    p.r.h0 = d.x; p.r.h1 = d.y; p.r.sub = d.z; p.r.n = d.w; p.r.blk = 0xFFFFFFFFu;
    if constexpr (C::beamlets) p.batch = 0;
    else p.batch = batch_of(d.x, d.y ^ c.a.stream_tag, c.a.pp.n_batches);
    p.steps = 0;
}

template <class C>
__device__ __forceinline__ void escape(C& c, const Lane& p)
{
    stat_add(c, ST_ESCAPED, 1);
    stat_add(c, ST_E_ESC, fx(p.E));
}

// e-/e+ created at p's position with energy E and direction d: pushed if above the
// absorption energy, otherwise deposited (a positron then annihilates).
template <class C>
__device__ void emit_charged(C& c, const Lane& p, int type, float E, float du, float dv, float dw, uint32_t slot);

// Two photons of mc^2, back to back and isotropic, from a positron with stream r.
template <class C>
__device__ __forceinline__ void annihilate(C& c, const Lane& p, Rng& r)
{
    float wc = 2.f * rng_u(r, c.a.key0, c.a.key1) - 1.f, xi = rng_u(r, c.a.key0, c.a.key1);
    float st = sqrtf(fmaxf(0.f, 1.f - wc * wc)), sp, cp;
    __sincosf(6.283185307179586f * xi, &sp, &cp);
    stat_add(c, ST_ANNIH, 1);
    if (MC2F >= c.a.pp.e_abs_g) {
        push(c, 0, p.x, p.y, p.z, MC2F, st * cp, st * sp, wc, p.ix, p.iy, p.iz, PHOTON, r.h0, r.h1,
             child_sub(r.sub, r.n, 0));
        push(c, 0, p.x, p.y, p.z, MC2F, -st * cp, -st * sp, -wc, p.ix, p.iy, p.iz, PHOTON, r.h0, r.h1,
             child_sub(r.sub, r.n, 1));
    } else {
        deposit(c, p, p.ix, p.iy, p.iz, 2.f * MC2F);
    }
}

template <class C>
__device__ void emit_charged(C& c, const Lane& p, int type, float E, float du, float dv, float dw, uint32_t slot)
{
    uint32_t sub = child_sub(p.r.sub, p.r.n, slot);
    if (E >= c.a.pp.e_abs_e && !(c.a.pp.flags & 8)) {
        push(c, charged_stack(c.a, E), p.x, p.y, p.z, E, du, dv, dw, p.ix, p.iy, p.iz, type, p.r.h0, p.r.h1, sub);
        return;
    }
    deposit(c, p, p.ix, p.iy, p.iz, E);
    if (type == POSITRON) {
        Rng r;
        r.h0 = p.r.h0; r.h1 = p.r.h1; r.sub = sub; r.n = 0; r.blk = 0xFFFFFFFFu;
        annihilate(c, p, r);
    }
}

// Pair production: e- and e+ along the photon, sharing E - 2 mc^2 uniformly.
template <class C>
__device__ __forceinline__ void pair_event(C& c, Lane& p)
{
    stat_add(c, ST_PAIR, 1);
    float avail = p.E - 2.f * MC2F;
    float Tm = rng_u(p.r, c.a.key0, c.a.key1) * avail, Tp = avail - Tm;
    emit_charged(c, p, ELECTRON, Tm, p.u, p.v, p.w, 0);
    emit_charged(c, p, POSITRON, Tp, p.u, p.v, p.w, 1);
}

// One Woodcock flight and, if real, the interaction. Returns false when the photon ends.
template <class C>
__device__ __forceinline__ bool photon_step(C& c, Lane& p, unsigned& n_fict)
{
    const TransportArgs& a = c.a;
    const SmemTables& T = c.T;
    const uint32_t k0 = a.key0, k1 = a.key1;
    rng_step_start(p.r, k0, k1);
    EIdx ei = e_index(p.E);
    float lnmaj = lerp1(T.phmaj[ei.i], T.phmaj[ei.i + 1], ei.f);
    if (lnmaj < -1e29f) { escape(c, p); return false; }
    float mumax = __expf(lnmaj);
    float s = -__logf(rng_u(p.r, k0, k1)) / mumax;
    p.x = fmaf(s, p.u, p.x);
    p.y = fmaf(s, p.v, p.y);
    p.z = fmaf(s, p.w, p.z);
    if (!(p.x >= 0.f && p.y >= 0.f && p.z >= 0.f && p.x <= c.Lx && p.y <= c.Ly && p.z <= c.Lz)) {
        if ((a.pp.flags & 4) && p.z > c.Lz) {
            stat_add(c, ST_TRANSMITTED, 1);
            stat_add(c, ST_E_TRANS, fx(p.E));
        }
        escape(c, p);
        return false;
    }
    p.ix = min((int)(p.x * c.inv_dx), a.nx - 1);
    p.iy = min((int)(p.y * c.inv_dy), a.ny - 1);
    p.iz = min((int)(p.z * c.inv_dz), a.nz - 1);
    const int vox = p.ix + a.nx * (p.iy + a.ny * p.iz);
    float rho = __ldg(a.density + vox);
    int m = __ldg(a.material + vox);
    float4 pa = T.ph[m * MS4 + ei.i], pb = T.ph[m * MS4 + ei.i + 1];
    float mu = rho * __expf(lerp1(pa.x, pb.x, ei.f));
    if (mu > mumax * 1.00001f) stat_add(c, ST_VIOL, 1);
    if (rng_u(p.r, k0, k1) * mumax >= mu) { n_fict++; return true; }
    if (a.pp.flags & 4) { stat_add(c, ST_E_KILLED, fx(p.E)); return false; }
    float fC = lerp1(pa.y, pb.y, ei.f), fP = lerp1(pa.z, pb.z, ei.f);
    float xi = rng_u(p.r, k0, k1);
    if (xi >= fC && xi < fC + fP) {
        stat_add(c, ST_PHOTO, 1);
        deposit(c, p, p.ix, p.iy, p.iz, p.E);
        return false;
    }
    if (xi >= fC + fP && p.E > 2.f * MC2F) {
        pair_event(c, p);
        return false;
    }
    // Compton scattering (also the rare pair selection below threshold from table interpolation)
    stat_add(c, ST_COMPTON, 1);
    float eps;
    float cth = sample_compton(p.E, p.r, k0, k1, &eps, &c.ok);
    float xphi = rng_u(p.r, k0, k1);
    float E0 = p.E, E1 = eps * E0, Te = E0 - E1;
    float u0 = p.u, v0 = p.v, w0 = p.w;
    rotate(p.u, p.v, p.w, cth, xphi);
    if (Te > 0.f) {
        float qu = E0 * u0 - E1 * p.u, qv = E0 * v0 - E1 * p.v, qw = E0 * w0 - E1 * p.w;
        float inv = rsqrtf(fmaxf(qu * qu + qv * qv + qw * qw, 1e-30f));
        emit_charged(c, p, ELECTRON, Te, qu * inv, qv * inv, qw * inv, 0);
    }
    p.E = E1;
    if (p.E < a.pp.e_abs_g) {
        deposit(c, p, p.ix, p.iy, p.iz, p.E);
        return false;
    }
    return true;
}

template <class C>
__device__ __forceinline__ bool cross_face(const C& c, Lane& p, int face)
{
    int ax = face >> 1;
    bool up = face & 1;
    if (ax == 0) { p.ix += up ? 1 : -1; p.x = (float)(up ? p.ix : p.ix + 1) * c.a.dx; }
    else if (ax == 1) { p.iy += up ? 1 : -1; p.y = (float)(up ? p.iy : p.iy + 1) * c.a.dy; }
    else { p.iz += up ? 1 : -1; p.z = (float)(up ? p.iz : p.iz + 1) * c.a.dz; }
    return p.ix >= 0 && p.iy >= 0 && p.iz >= 0 && p.ix < c.a.nx && p.iy < c.a.ny && p.iz < c.a.nz;
}

// Discrete hard event at the end of a step: Moller (probability sM / tot) or bremsstrahlung.
template <class C>
__device__ __forceinline__ void hard_event(C& c, Lane& p, int m, float sM, float tot)
{
    const SmemTables& T = c.T;
    if (rng_u(p.r, c.a.key0, c.a.key1) * tot < sM) {
        stat_add(c, ST_MOLLER, 1);
        float Tk = p.E;
        float eps = sample_moller(Tk, c.a.pp.w_cc, p.r, c.a.key0, c.a.key1, &c.ok);
        float W = eps * Tk, T1 = Tk - W;
        float xphi = rng_u(p.r, c.a.key0, c.a.key1);
        float mu1 = sqrtf(fminf(1.f, T1 * (Tk + 2.f * MC2F) / (Tk * (T1 + 2.f * MC2F))));
        float mu2 = sqrtf(fminf(1.f, W * (Tk + 2.f * MC2F) / (Tk * (W + 2.f * MC2F))));
        float su = p.u, sv2 = p.v, sw = p.w;
        rotate(su, sv2, sw, mu2, xphi + 0.5f);
        emit_charged(c, p, ELECTRON, W, su, sv2, sw, 2);
        rotate(p.u, p.v, p.w, mu1, xphi);
        p.E = T1;
    } else {
        stat_add(c, ST_BREMS, 1);
        float Tk = p.E;
        float k = sample_brems(Tk, c.a.pp.w_cb, T.msc[m * MS1], T.msc[m * MS1 + 1], p.r, c.a.key0, c.a.key1, &c.ok);
        float th = MC2F / (Tk + MC2F);
        float xphi = rng_u(p.r, c.a.key0, c.a.key1);
        float gu = p.u, gv = p.v, gw = p.w;
        rotate(gu, gv, gw, __cosf(th), xphi);
        if (k >= c.a.pp.e_abs_g)
            push(c, 0, p.x, p.y, p.z, k, gu, gv, gw, p.ix, p.iy, p.iz, PHOTON, p.r.h0, p.r.h1,
                 child_sub(p.r.sub, p.r.n, 3));
        else
            deposit(c, p, p.ix, p.iy, p.iz, k);
        p.E = Tk - k;
    }
}

// A charged particle that fell below its absorption energy.
template <class C>
__device__ __forceinline__ void absorb_charged(C& c, Lane& p)
{
    deposit(c, p, p.ix, p.iy, p.iz, p.E);
    if (p.type == POSITRON) annihilate(c, p, p.r);
}

// One condensed-history step. Returns false when the particle ends.
template <class C>
__device__ __forceinline__ bool charged_step(C& c, Lane& p, unsigned& n_hfict)
{
    const TransportArgs& a = c.a;
    const SmemTables& T = c.T;
    const uint32_t k0 = a.key0, k1 = a.key1;
    if (vox_bad(c, p)) return false;
    const int vox = p.ix + a.nx * (p.iy + a.ny * p.iz);
    float rho = __ldg(a.density + vox);
    int m = __ldg(a.material + vox);
    int face;
    float sv = dist_to_face(p.x, p.y, p.z, p.u, p.v, p.w, p.ix, p.iy, p.iz, a.dx, a.dy, a.dz, &face);
    if (!(rho > 0.f) || sv < a.pp.s_min) {
        // nothing to interact with, or a boundary closer than s_min: cross geometrically
        p.x = fmaf(sv, p.u, p.x);
        p.y = fmaf(sv, p.v, p.y);
        p.z = fmaf(sv, p.w, p.z);
        stat_add(c, ST_GEO, 1);
        if (!cross_face(c, p, face)) { escape(c, p); return false; }
        return true;
    }
    rng_step_start(p.r, k0, k1);
    EIdx ei = e_index(p.E);
    const int mb = m * MS4, mb2 = m * MS2;
    float4 A = T.el[mb + ei.i], B = T.el[mb + ei.i + 1];
    float2 C2 = T.el2[mb2 + ei.i], D2 = T.el2[mb2 + ei.i + 1];
    float lnR = lerp1(A.x, B.x, ei.f);
    float s_maxe = lerp1(C2.x, D2.x, ei.f) / rho;
    float sighat = (a.pp.flags & 1) ? 0.f : C2.y;
    float d_ev = sighat > 0.f ? -__logf(rng_u(p.r, k0, k1)) / (rho * sighat) : 3.0e38f;
    float s = sv;
    int lim = 0;
    if (a.pp.d_maxs < s) { s = a.pp.d_maxs; lim = 1; }
    if (s_maxe < s) { s = s_maxe; lim = 2; }
    if (d_ev < s) { s = d_ev; lim = 3; }
    // random hinge: s1 straight, deflect, then the rest (clipped to this voxel)
    float s1 = rng_u(p.r, k0, k1) * s;
    float hx = fmaf(s1, p.u, p.x), hy = fmaf(s1, p.v, p.y), hz = fmaf(s1, p.w, p.z);
    float E0 = p.E;
    const float R0 = __expf(lnR), g0 = range_to_lnE(T, m, lnR);
    float Efull = csda_end2(T, m, E0, R0, g0, rho * s);
    if (!(a.pp.flags & 2)) {
        EIdx em = e_index(0.5f * (E0 + Efull));
        float l1 = lerp1(T.el[mb + em.i].y, T.el[mb + em.i + 1].y, em.f);
        float cth = sample_ms(T, rho * s * l1, p.r, k0, k1);
        float xphi = rng_u(p.r, k0, k1);
        rotate(p.u, p.v, p.w, cth, xphi);
    }
    int face2;
    float tex = dist_to_face(hx, hy, hz, p.u, p.v, p.w, p.ix, p.iy, p.iz, a.dx, a.dy, a.dz, &face2);
    float rem = s - s1, Eend;
    bool crossed;
    if (rem < tex) {
        p.x = fmaf(rem, p.u, hx);
        p.y = fmaf(rem, p.v, hy);
        p.z = fmaf(rem, p.w, hz);
        Eend = Efull;
        crossed = false;
    } else {
        p.x = fmaf(tex, p.u, hx);
        p.y = fmaf(tex, p.v, hy);
        p.z = fmaf(tex, p.w, hz);
        Eend = csda_end2(T, m, E0, R0, g0, rho * (s1 + tex));
        crossed = true;
    }
    deposit(c, p, p.ix, p.iy, p.iz, E0 - Eend);
    p.E = Eend;
    if (crossed && !cross_face(c, p, face2)) { escape(c, p); return false; }
    if (p.E < a.pp.e_abs_e) { absorb_charged(c, p); return false; }
    if (lim == 3 && !crossed) {
        EIdx e2 = e_index(p.E);
        float4 A2 = T.el[mb + e2.i], B2 = T.el[mb + e2.i + 1];
        float sM = p.E > 2.f * a.pp.w_cc ? lerp1(A2.z, B2.z, e2.f) : 0.f;
        float sB = p.E > a.pp.w_cb ? lerp1(A2.w, B2.w, e2.f) : 0.f;
        float tot = sM + sB;
        if (tot > sighat * 1.00001f) stat_add(c, ST_VIOL, 1);
        if (rng_u(p.r, k0, k1) * sighat < tot) {
            hard_event(c, p, m, sM, tot);
            if (p.E < a.pp.e_abs_e) { absorb_charged(c, p); return false; }
        } else {
            n_hfict++;
        }
    }
    return true;
}

// ---- voxel-crossing (fixed-step) electron steps ------------------------------------------
// The stepping scheme the paper contrasts with its own (Sec. 4): a step is not stopped at voxel
// faces. s = min(d_maxs, d_maxe, d_event) with d_maxe from the step's first voxel and d_event
// sampled against the phantom-wide majorant of rho * sigma_hard (so a candidate may fall in any
// voxel); random hinge at xi s with the multiple-scattering angle of the whole step in the first
// voxel's medium; along both straight parts the CSDA loss of each traversed voxel's own
// material and density is deposited there; the step ends early where the energy reaches
// E (1 - f_maxe) (before the hinge: deflected there, for the path travelled); a candidate at the
// end of an event-limited step is real with probability rho sigma_hard(E) / majorant in the
// voxel where it ends.
enum { SEG_DONE = 0, SEG_FLOOR, SEG_OUT };   // SEG_OUT: the particle escaped or was absorbed

__device__ __forceinline__ float range_R(const SmemTables& T, int m, float E)
{
    const EIdx ei = e_index(E);
    return __expf(lerp1(T.el[m * MS4 + ei.i].x, T.el[m * MS4 + ei.i + 1].x, ei.f));
}

// Moves p a path length L along its direction through the voxels, losing and depositing the
// CSDA energy of each voxel it crosses; stops early at the energy floor Ef, on absorption or on
// escape. *done receives the path length travelled.
template <class C>
__device__ __forceinline__ int cross_segment(C& c, Lane& p, float L, float Ef, float* done)
{
    const TransportArgs& a = c.a;
    const SmemTables& T = c.T;
    float left = L, moved = 0.f;
    for (int guard = 0; left > 0.f; ++guard) {
        if (guard > 4 * (a.nx + a.ny + a.nz)) { c.ok = false; break; }   // cannot happen: bounded crossings
        if (vox_bad(c, p)) { *done = moved; return SEG_OUT; }
        const int vox = p.ix + a.nx * (p.iy + a.ny * p.iz);
        const float rho = __ldg(a.density + vox);
        const int m = __ldg(a.material + vox);
        int face;
        const float sv = dist_to_face(p.x, p.y, p.z, p.u, p.v, p.w, p.ix, p.iy, p.iz, a.dx, a.dy, a.dz, &face);
        float l = left, Eend = p.E;
        bool cross = false, flo = false;
        if (sv < l) { l = sv; cross = true; }
        if (rho > 0.f) {
            const EIdx ei = e_index(p.E);
            const float lnR = lerp1(T.el[m * MS4 + ei.i].x, T.el[m * MS4 + ei.i + 1].x, ei.f);
            const float R = __expf(lnR);
            const float lf = (R - range_R(T, m, Ef)) / rho;
            if (lf <= l) { l = fmaxf(lf, 0.f); cross = false; flo = true; Eend = Ef; }
            else Eend = csda_end2(T, m, p.E, R, range_to_lnE(T, m, lnR), rho * l);
        }
        p.x = fmaf(l, p.u, p.x);
        p.y = fmaf(l, p.v, p.y);
        p.z = fmaf(l, p.w, p.z);
        deposit(c, p, p.ix, p.iy, p.iz, p.E - Eend);
        p.E = Eend;
        left -= l;
        moved += l;
        if (p.E < a.pp.e_abs_e) { absorb_charged(c, p); *done = moved; return SEG_OUT; }
        if (flo) { *done = moved; return SEG_FLOOR; }
        if (cross && !cross_face(c, p, face)) { escape(c, p); *done = moved; return SEG_OUT; }
    }
    *done = moved;
    return SEG_DONE;
}

template <class C>
__device__ __forceinline__ bool charged_step_cross(C& c, Lane& p, unsigned& n_hfict)
{
    const TransportArgs& a = c.a;
    const SmemTables& T = c.T;
    const uint32_t k0 = a.key0, k1 = a.key1;
    if (vox_bad(c, p)) return false;
    const int vox = p.ix + a.nx * (p.iy + a.ny * p.iz);
    const float rho0 = __ldg(a.density + vox);
    const int m0 = __ldg(a.material + vox);
    if (!(rho0 > 0.f)) {                       // no matter here: fly to the next voxel
        int face;
        float sv = dist_to_face(p.x, p.y, p.z, p.u, p.v, p.w, p.ix, p.iy, p.iz, a.dx, a.dy, a.dz, &face);
        p.x = fmaf(sv, p.u, p.x);
        p.y = fmaf(sv, p.v, p.y);
        p.z = fmaf(sv, p.w, p.z);
        stat_add(c, ST_GEO, 1);
        if (!cross_face(c, p, face)) { escape(c, p); return false; }
        return true;
    }
    rng_step_start(p.r, k0, k1);
    const float E0 = p.E;
    const EIdx ei = e_index(E0);
    const int mb = m0 * MS4, mb2 = m0 * MS2;
    const float lnR = lerp1(T.el[mb + ei.i].x, T.el[mb + ei.i + 1].x, ei.f);
    const float s_maxe = lerp1(T.el2[mb2 + ei.i].x, T.el2[mb2 + ei.i + 1].x, ei.f) / rho0;
    const float maj = (a.pp.flags & 1) ? 0.f : __ldg(a.t.elmaj + ei.i);
    const float d_ev = maj > 0.f ? -__logf(rng_u(p.r, k0, k1)) / maj : 3.0e38f;
    float s = a.pp.d_maxs;
    int lim = 1;
    if (s_maxe < s) { s = s_maxe; lim = 2; }
    if (d_ev < s) { s = d_ev; lim = 3; }
    const float s1 = rng_u(p.r, k0, k1) * s;
    const float Ef = E0 * (1.f - a.pp.f_maxe);
    const float Efull = csda_end2(T, m0, E0, __expf(lnR), range_to_lnE(T, m0, lnR), rho0 * s);
    float done;
    int r = cross_segment(c, p, s1, Ef, &done);
    if (r == SEG_OUT) return false;
    if (!(a.pp.flags & 2)) {
        EIdx em = e_index(0.5f * (E0 + Efull));
        float l1 = lerp1(T.el[mb + em.i].y, T.el[mb + em.i + 1].y, em.f);
        float cth = sample_ms(T, rho0 * (r == SEG_FLOOR ? done : s) * l1, p.r, k0, k1);
        float xphi = rng_u(p.r, k0, k1);
        rotate(p.u, p.v, p.w, cth, xphi);
    }
    if (r == SEG_FLOOR) return true;
    r = cross_segment(c, p, s - s1, Ef, &done);
    if (r == SEG_OUT) return false;
    if (r == SEG_FLOOR || lim != 3) return true;
    // candidate hard event where the step ended
    if (vox_bad(c, p)) return false;
    const int v2 = p.ix + a.nx * (p.iy + a.ny * p.iz);
    const float rho = __ldg(a.density + v2);
    const int m = __ldg(a.material + v2);
    const EIdx e2 = e_index(p.E);
    const float4 A2 = T.el[m * MS4 + e2.i], B2 = T.el[m * MS4 + e2.i + 1];
    const float sM = p.E > 2.f * a.pp.w_cc ? rho * lerp1(A2.z, B2.z, e2.f) : 0.f;
    const float sB = p.E > a.pp.w_cb ? rho * lerp1(A2.w, B2.w, e2.f) : 0.f;
    const float tot = sM + sB;
    if (tot > maj * 1.00001f) stat_add(c, ST_VIOL, 1);
    if (rng_u(p.r, k0, k1) * maj < tot) {
        hard_event(c, p, m, sM, tot);
        if (p.E < a.pp.e_abs_e) { absorb_charged(c, p); return false; }
    } else {
        n_hfict++;
    }
    return true;
}

// NREG: register cap per thread. More registers spill less; fewer registers let more
// warps share an SM (80: 3 x 256 threads, 64: 2 x 512, 56: 3 x 384 on GB300).
// PS: the source is a phase space (per-history records of mixed particle types); a separate
// instantiation, so that the analytic-source kernel carries none of its code.
// XV: electron steps cross voxel faces (the fixed-step variant); a separate instantiation of the
// analytic-source kernel, so the voxel-limited kernels carry none of its code.
template <bool BL, bool PS, int NREG, bool XV = false>
__global__ void __maxnreg__(NREG) k_transport(const __grid_constant__ TransportArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_top[MAX_WARPS][3];
    __shared__ unsigned long long s_st[ST_COUNT];
    __shared__ unsigned long long s_time[MAX_WARPS][2];   // per warp: start, source seen exhausted
    __shared__ unsigned long long s_wc[MAX_WARPS][3];     // per warp: iterations, photon / charged lane-steps
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x) s_st[i] = 0ull;
    if (lane == 0) { s_top[wib][0] = 0; s_top[wib][1] = 0; s_top[wib][2] = 0; }
    SmemTables T = stage_tables(a.t, smem);   // ends with __syncthreads()
    if (lane == 0) { s_time[wib][0] = globaltimer_ns(); s_time[wib][1] = 0ull; }

    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
    CtxT<BL> c{a, T, a.stacks + (size_t)gw * a.nstk * a.cap, s_top[wib], s_st,
          1.f / a.dx, 1.f / a.dy, 1.f / a.dz, a.nx * a.dx, a.ny * a.dy, a.nz * a.dz, true};
    const unsigned lt = (1u << lane) - 1u;
    const int src_mode = a.src.particle == 0 ? 0 : 1;
    // a phase-space source mixes particle types: warps of either type draw from it, and a
    // primary of the other type goes to that type's stack like a secondary
    constexpr bool ps_src = PS && !BL;
    int mode = src_mode;
    bool src_done = a.count == 0;
    // with switch_high >= cap, switching on stack size is off (stacks may then overflow, which
    // is reported); otherwise a warp also switches when another stack nears its capacity
    const int emergency = a.switch_high < a.cap ? a.cap - 128 : 0x7FFFFFFF;
    bool active = false, just_switched = false;
    Lane p;
    unsigned n_fict = 0, n_hfict = 0;
    // per-warp scheduler counters live in shared memory (iterations, photon and charged lane-steps),
    // and per-history counts go straight to the block's statistics: none of them takes a register
    // under the register cap
    unsigned long long* wc = s_wc[wib];
    if (lane == 0) { wc[0] = 0ull; wc[1] = 0ull; wc[2] = 0ull; }

    // modes (= stacks): 0 photons, 1 charged particles (at or above e_split when there are
    // three stacks), 2 charged particles below e_split
    for (;;) {
        __syncwarp();
        int top0 = min(c.top[0], a.cap), top1 = min(c.top[1], a.cap), top2 = a.nstk == 3 ? min(c.top[2], a.cap) : 0;
        unsigned act = __ballot_sync(FULL, active);
        int nfree = 32 - __popc(act);
        // refill when enough lanes are free: the refill code runs on the free lanes only,
        // so waiting for several of them spreads its cost
        if (nfree >= a.refill_min || nfree == 32) {
            int topm = mode == 0 ? top0 : (mode == 1 ? top1 : top2);
            int rank = __popc(~act & lt);
            int take = min(nfree, topm);
            if (!active && rank < take) {
                pop_lane(c, mode, topm - 1 - rank, p);
                active = true;
            }
            int want = nfree - take;
            if (want > 0 && (ps_src || mode == src_mode) && !src_done) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(a.hist_counter, (unsigned long long)want);
                base = __shfl_sync(FULL, base, 0);
                if (base + want >= a.count) {
                    src_done = true;
                    if (lane == 0) s_time[wib][1] = globaltimer_ns();
                }
                int r2 = rank - take;
                if (!active && r2 >= 0 && r2 < want && base + r2 < a.count) {
                    stat_add(c, ST_HISTORIES, 1);
                    bool in;
                    if constexpr (BL) in = init_beamlet(a, base + r2, p);
                    else if constexpr (ps_src) in = init_phase_space(a, a.first + base + r2, p);
                    else in = init_primary(a, a.first + base + r2, p);
                    float ecut = p.type == PHOTON ? a.pp.e_abs_g : a.pp.e_abs_e;
                    if (!in) {
                        stat_add(c, ST_MISSED, 1);
                        stat_add(c, ST_E_MISS, fx(p.E));
                    } else if constexpr (ps_src) {
                        stat_add(c, ST_E_IN, fx(p.E));
                        const bool charged = p.type != PHOTON;
                        if (p.E >= ecut && !(charged && (a.pp.flags & 8))) {
                            const int target = charged ? charged_stack(a, p.E) : 0;
                            if (target == mode) active = true;
                            else push_lane(c, target, p);
                        } else if (charged) {
                            absorb_charged(c, p);       // positrons annihilate
                        } else {
                            deposit(c, p, p.ix, p.iy, p.iz, p.E);
                        }
                    } else {
                        stat_add(c, ST_E_IN, fx(p.E));
                        if (p.E >= ecut && !(p.type != PHOTON && (a.pp.flags & 8))) active = true;
                        else deposit(c, p, p.ix, p.iy, p.iz, p.E);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) c.top[mode] = topm - take;
            __syncwarp();
            if (mode == 0) top0 = topm - take; else if (mode == 1) top1 = topm - take; else top2 = topm - take;
            act = __ballot_sync(FULL, active);
        }
        int nact = __popc(act);
        const int topm = mode == 0 ? top0 : (mode == 1 ? top1 : top2);
        bool m_avail = topm > 0 || ((ps_src || mode == src_mode) && !src_done);
        // the other mode: the fullest other stack that has work (or that the source feeds)
        int other = -1, topo = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int tk = k == 0 ? top0 : (k == 1 ? top1 : top2);
            if (k != mode && k < a.nstk && (tk > 0 || ((ps_src || k == src_mode) && !src_done)) &&
                (other < 0 || tk > topo)) {
                other = k;
                topo = tk;
            }
        }
        const bool o_avail = other >= 0;
        if (nact == 0) {
            if (m_avail) continue;
            if (o_avail) { mode = other; continue; }
            break;
        }
        bool sw = false;
        if (o_avail && !just_switched) {     // at most one switch between two steps
            // the other group must be strictly larger (or the source), so a switch is never undone at once
            if (!m_avail && nact <= a.switch_low && (topo > nact || (!ps_src && other == src_mode && !src_done)))
                sw = true;
            else if (topo >= a.switch_high && topo >= 2 * (nact + topm)) sw = true;
            // the other stack is within one iteration's pushes (32 lanes x 3 secondaries, plus
            // 32 refilled primaries) of its capacity: switch before it can overflow
            else if (topo >= emergency && topo > topm) sw = true;
        }
        if (sw) {
            if (active) { push_lane(c, mode ? charged_stack(a, p.E) : 0, p); active = false; }
            mode = other;
            just_switched = true;
            continue;
        }
        just_switched = false;
        if (lane == 0) {
            wc[0] += 1ull;
            wc[mode ? 2 : 1] += (unsigned long long)nact;
        }
        if (active) {
            if constexpr (XV) active = mode ? charged_step_cross(c, p, n_hfict) : photon_step(c, p, n_fict);
            else active = mode ? charged_step(c, p, n_hfict) : photon_step(c, p, n_fict);
            if (active && ++p.steps > STEP_LIMIT) {
                atomicOr(a.err, ERR_LIMIT);
                stat_add(c, ST_DROPPED, 1);
                stat_add(c, ST_E_DROPPED, fx(p.E));
                active = false;
            }
            if (!c.ok) {
                atomicOr(a.err, ERR_LIMIT);
                c.ok = true;
            }
        }
    }
    // per-warp and per-lane statistics
    atomicAdd(s_st + ST_FICT, (unsigned long long)n_fict);
    atomicAdd(s_st + ST_HARD_FICT, (unsigned long long)n_hfict);
    if (lane == 0) {
        atomicAdd(s_st + ST_WARP_ITERS, wc[0]);
        atomicAdd(s_st + ST_LANES_PHOTON, wc[1]);
        atomicAdd(s_st + ST_LANES_CHARGED, wc[2]);
        // tail: how long this warp ran on its own stacks after the source ran dry
        const unsigned long long t_end = globaltimer_ns(), t0 = s_time[wib][0];
        const unsigned long long ts = s_time[wib][1] ? s_time[wib][1] : t0;
        atomicAdd(s_st + ST_WARP_NS, t_end - t0);
        atomicAdd(s_st + ST_WARPS, 1ull);
        atomicAdd(s_st + ST_TAIL_NS, t_end - ts);
        atomicMax(a.stats + ST_T_START_INV, ~t0);
        atomicMax(a.stats + ST_T_SRC_INV, ~ts);
        atomicMax(a.stats + ST_T_END, t_end);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x)
        if (s_st[i]) atomicAdd(a.stats + i, s_st[i]);
}

}  // namespace

size_t transport_smem_bytes(int n_mat) { return smem_table_bytes(n_mat); }

namespace {
template <bool BL, bool PS, int R, bool XV = false>
cudaError_t launch_variant(const TransportArgs& a, int blocks, int threads, size_t smem, cudaStream_t s)
{
    cudaError_t e =
        cudaFuncSetAttribute(k_transport<BL, PS, R, XV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_transport<BL, PS, R, XV><<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <bool BL, bool PS, int R>
int occupancy(int threads, size_t smem)
{
    cudaFuncSetAttribute(k_transport<BL, PS, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_transport<BL, PS, R>, threads, smem) != cudaSuccess)
        return 0;
    return n;
}

template <bool BL, bool PS>
cudaError_t launch_source(const TransportArgs& a, int blocks, int threads, size_t smem, cudaStream_t s, int nreg)
{
    if (nreg == 56) return launch_variant<BL, PS, 56>(a, blocks, threads, smem, s);
    if (nreg == 64) return launch_variant<BL, PS, 64>(a, blocks, threads, smem, s);
    return launch_variant<BL, PS, 80>(a, blocks, threads, smem, s);
}
}  // namespace

bool transport_nreg_supported(int nreg) { return nreg == 56 || nreg == 64 || nreg == 80; }

int transport_max_blocks_per_sm(int threads, size_t smem, int nreg)
{
    occupancy<true, false, 56>(threads, smem);   // sets the shared-memory attribute of every variant
    occupancy<true, false, 64>(threads, smem);
    occupancy<true, false, 80>(threads, smem);
    occupancy<false, true, 56>(threads, smem);
    occupancy<false, true, 64>(threads, smem);
    occupancy<false, true, 80>(threads, smem);
    cudaFuncSetAttribute(k_transport<false, false, 56, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_transport<false, false, 64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_transport<false, false, 80, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (nreg == 56) return occupancy<false, false, 56>(threads, smem);
    if (nreg == 64) return occupancy<false, false, 64>(threads, smem);
    return occupancy<false, false, 80>(threads, smem);
}

cudaError_t launch_transport(const TransportArgs& a, int blocks, int threads, size_t smem, cudaStream_t s, int nreg)
{
    if (a.pp.flags & FLAG_CROSS_VOXELS) {
        // voxel-crossing electron steps: analytic single-beam source only (callers check)
        if (a.beamlets || a.ps) return cudaErrorInvalidValue;
        if (nreg == 56) return launch_variant<false, false, 56, true>(a, blocks, threads, smem, s);
        if (nreg == 64) return launch_variant<false, false, 64, true>(a, blocks, threads, smem, s);
        return launch_variant<false, false, 80, true>(a, blocks, threads, smem, s);
    }
    if (a.beamlets) return launch_source<true, false>(a, blocks, threads, smem, s, nreg);
    if (a.ps) return launch_source<false, true>(a, blocks, threads, smem, s, nreg);
    return launch_source<false, false>(a, blocks, threads, smem, s, nreg);
}

}  // namespace ocmc
