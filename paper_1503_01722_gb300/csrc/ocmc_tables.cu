// ocmc_tables.cu -- physics tables of the transport kernel, built on the GPU in
// double precision from closed-form models, then stored as FP32.
//
// The paper stores per-material photon attenuation per channel, restricted
// stopping powers and macroscopic cross sections as 2D images indexed by
// energy and material (Sec. 2.1, Sec. 2.2.2). Here the same quantities come
// from published closed forms (one table row per material, uniform in ln E):
//   photons  : Klein-Nishina (free electrons), K-shell Born photoelectric,
//              Maximon's pair expansions with Z(Z+1);
//   electrons: ICRU-37 restricted collision stopping power with the
//              Sternheimer-Peierls density effect, complete-screening
//              Bethe-Heitler bremsstrahlung with Z(Z+1), Moller cross section,
//              screened-Rutherford transport cross section (Moliere screening).
// The CSDA range R(E) is the integral of 1/L (8-point Gauss-Legendre per
// table interval), inverted on a uniform ln R grid by bisection.
#include "ocmc_internal.h"

#include <cmath>

namespace ocmc {

namespace {


constexpr double RE = 2.8179403262e-13;
constexpr double ALPHA = 1.0 / 137.035999084;
constexpr double NAV = 6.02214076e23;
constexpr double PI = 3.14159265358979323846;

struct MC {
    double ne, photo, pairZ, S1, S2, I, dC, dX0, dX1, dA;
};

__device__ MC mconst(const MatDef& d)
{
    MC c;
    double ws = 0.0;
    for (int i = 0; i < d.n; ++i) ws += d.w[i];
    c.ne = c.photo = c.pairZ = c.S1 = c.S2 = 0.0;
    for (int i = 0; i < d.n; ++i) {
        double Z = d.Z[i], n = NAV * d.w[i] / ws / d.A[i];
        c.ne += n * Z;
        c.photo += n * Z * Z * Z * Z * Z;
        c.pairZ += n * Z * (Z + 1.0);
        c.S1 += n * Z * (Z + 1.0) * log(183.0 / cbrt(Z));
        c.S2 += n * Z * (Z + 1.0) / 9.0;
    }
    c.I = d.I_eV;
    double hw = 28.816 * sqrt(d.rho0 * c.ne / NAV);
    double C = 2.0 * log(d.I_eV / hw) + 1.0;
    double x0, x1;
    if (d.I_eV < 100.0) { x1 = 2.0; x0 = C < 3.681 ? 0.2 : 0.326 * C - 1.0; }
    else                { x1 = 3.0; x0 = C < 5.215 ? 0.2 : 0.326 * C - 1.5; }
    c.dC = C; c.dX0 = x0; c.dX1 = x1;
    double span = x1 - x0;
    c.dA = (C - 2.0 * log(10.0) * x0) / (span * span * span);
    return c;
}

__device__ double kn_total(double E)
{
    double k = E / MC2, a = 1.0 + 2.0 * k, l = log(a);
    return 2.0 * PI * RE * RE *
           ((1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k) + l / (2.0 * k) - (1.0 + 3.0 * k) / (a * a));
}

__device__ double pair_phi(double E)
{
    double k = E / MC2;
    if (k <= 2.0) return 0.0;
    double v;
    if (k <= 4.0) {
        double e = (2.0 * k - 4.0) / (2.0 + k + 2.0 * sqrt(2.0 * k));
        double r = 1.0 - 2.0 / k;
        v = (2.0 * PI / 3.0) * r * r * r *
            (1.0 + e * (0.5 + e * (23.0 / 40.0 + e * (11.0 / 60.0 + e * 29.0 / 960.0))));
    } else {
        double L = log(2.0 * k), q2 = 4.0 / (k * k);
        const double zeta3 = 1.2020569031595942;
        v = 28.0 / 9.0 * L - 218.0 / 27.0 +
            q2 * (6.0 * L - 3.5 + (2.0 / 3.0) * L * L * L - L * L - (PI * PI / 3.0) * L + 2.0 * zeta3 +
                  PI * PI / 6.0) -
            q2 * q2 * (3.0 / 16.0 * L + 0.125) -
            q2 * q2 * q2 * (29.0 / 2304.0 * L - 77.0 / 13824.0);
    }
    return v > 0.0 ? v : 0.0;
}

// 0 total, 1 Compton, 2 photoelectric, 3 pair  (cm^2/g)
__device__ double mu_channel(const MC& c, double E, int ch)
{
    double sC = c.ne * kn_total(E);
    double sigT = 8.0 * PI / 3.0 * RE * RE;
    double sP = c.photo * 4.0 * sqrt(2.0) * ALPHA * ALPHA * ALPHA * ALPHA * sigT * pow(MC2 / E, 3.5);
    double sQ = c.pairZ * ALPHA * RE * RE * pair_phi(E);
    return ch == 1 ? sC : ch == 2 ? sP : ch == 3 ? sQ : sC + sP + sQ;
}

__device__ double density_delta(const MC& c, double T)
{
    double tau = T / MC2;
    double x = 0.5 * log10(tau * (tau + 2.0));
    if (x < c.dX0) return 0.0;
    double r = 2.0 * log(10.0) * x - c.dC;
    if (x < c.dX1) {
        double y = c.dX1 - x;
        r += c.dA * y * y * y;
    }
    return r;
}

__device__ double L_col(const MC& c, double T, double wcc)
{
    double tau = T / MC2, g = tau + 1.0, b2 = 1.0 - 1.0 / (g * g);
    double d = fmin(wcc, 0.5 * T) / MC2;
    double I = c.I * 1e-6 / MC2;
    double F = -1.0 - b2 + log((tau - d) * d) + tau / (tau - d) +
               (0.5 * d * d + (2.0 * tau + 1.0) * log(1.0 - d / tau)) / (g * g);
    return 2.0 * PI * RE * RE * MC2 * c.ne / b2 * (log(2.0 * (tau + 2.0) / (I * I)) + F - density_delta(c, T));
}

__device__ double L_rad(const MC& c, double T, double wcb)
{
    double E = T + MC2, k = fmin(wcb, T);
    double a = c.S1 * (4.0 / 3.0 * k - 2.0 / 3.0 * k * k / E + k * k * k / (3.0 * E * E));
    double b = c.S2 * (k - 0.5 * k * k / E);
    return 4.0 * ALPHA * RE * RE * (a + b);
}

__device__ double L_tot(const MC& c, double T, const PhysParams& pp)
{
    T = fmax(T, 1e-3);
    return L_col(c, T, pp.w_cc) + L_rad(c, T, pp.w_cb);
}

__device__ double sig_moller(const MC& c, double T, double wcc)
{
    if (T <= 2.0 * wcc) return 0.0;
    double tau = T / MC2, g = tau + 1.0, b2 = 1.0 - 1.0 / (g * g);
    double cc = (tau / g) * (tau / g), dd = (2.0 * tau + 1.0) / (g * g), e0 = wcc / T;
    // integral over eps in [e0, 1/2] of 1/e^2 + 1/(1-e)^2 + cc - dd/(e(1-e))
    double I = (1.0 / e0 - 2.0) + (2.0 - 1.0 / (1.0 - e0)) + cc * (0.5 - e0) - dd * log((1.0 - e0) / e0);
    return 2.0 * PI * RE * RE * MC2 * c.ne / (b2 * T) * I;
}

__device__ double sig_brems(const MC& c, double T, double wcb)
{
    if (T <= wcb) return 0.0;
    double E = T + MC2, l = log(T / wcb), dk = T - wcb;
    double a = c.S1 * (4.0 / 3.0 * l - 4.0 / 3.0 * dk / E + (T * T - wcb * wcb) / (2.0 * E * E));
    double b = c.S2 * (l - dk / E);
    return 4.0 * ALPHA * RE * RE * (a + b);
}

__device__ double lambda1_inv(const MatDef& d, double T)
{
    double ws = 0.0;
    for (int i = 0; i < d.n; ++i) ws += d.w[i];
    double pc = sqrt(T * (T + 2.0 * MC2)), beta = pc / (T + MC2), q = MC2 / (pc * beta);
    double s = 0.0;
    for (int i = 0; i < d.n; ++i) {
        double Z = d.Z[i];
        double a = ALPHA * cbrt(Z) * MC2 / (0.885 * pc);
        double az = ALPHA * Z / beta;
        double eta = 0.25 * a * a * (1.13 + 3.76 * az * az);
        s += NAV * d.w[i] / ws / d.A[i] * 2.0 * PI * Z * (Z + 1.0) * RE * RE * q * q *
             (log1p(1.0 / eta) - 1.0 / (1.0 + eta));
    }
    return s;
}

__device__ double wentzel_mean(double A)
{
    if (A > 1e3) {
        double x = 1.0 / A;
        return 1.0 - x * (1.0 / 3.0 - x * (1.0 / 6.0 - x / 10.0));
    }
    return 2.0 * A * ((1.0 + A) * log1p(1.0 / A) - 1.0);
}

__device__ double wentzel_solve(double G1)
{
    double target = -expm1(-G1), lo = log(1e-40), hi = log(1e15);
    for (int it = 0; it < 100; ++it) {
        double mid = 0.5 * (lo + hi);
        if (wentzel_mean(exp(mid)) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// integral of dT / L(T) over [a, b], 8-point Gauss-Legendre
__device__ double inv_L_integral(const MC& c, double a, double b, const PhysParams& pp)
{
    const double x[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    const double w[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    double mid = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int k = 0; k < 4; ++k)
        s += w[k] * (1.0 / L_tot(c, mid + h * x[k], pp) + 1.0 / L_tot(c, mid - h * x[k], pp));
    return s * h;
}

__device__ __forceinline__ double node_E(int i)
{
    double d = log(E_HI / E_LO) / (NE - 1);
    return exp(log(E_LO) + d * i);
}

__global__ void k_nodes(Tables t, PhysParams pp)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= t.n_mat * NE) return;
    int m = idx / NE, i = idx % NE;
    MC c = mconst(t.mats[m]);
    double E = node_E(i);
    double mt = mu_channel(c, E, 0), mC = mu_channel(c, E, 1), mP = mu_channel(c, E, 2);
    t.ph[idx] = make_float4((float)log(mt), (float)(mC / mt), (float)(mP / mt), (float)mt);
    double sM = sig_moller(c, E, pp.w_cc), sB = sig_brems(c, E, pp.w_cb);
    t.el[idx] = make_float4(0.f, (float)lambda1_inv(t.mats[m], E), (float)sM, (float)sB);
    // step limit d_maxe (mass thickness) and the hard-event majorant on [E_i, E_i+1),
    // covering the energies a step starting there can reach (down to E (1 - f_maxe)).
    double dRf = inv_L_integral(c, E * (1.0 - pp.f_maxe), E, pp);
    double Ehi = node_E(i) * exp(log(E_HI / E_LO) / (NE - 1));
    double Elo = E * (1.0 - pp.f_maxe) * 0.99, mx = 0.0;
    for (int k = 0; k <= 32; ++k) {
        double e = Elo + (Ehi - Elo) * k / 32.0;
        mx = fmax(mx, sig_moller(c, e, pp.w_cc) + sig_brems(c, e, pp.w_cb));
    }
    t.el2[idx] = make_float2((float)dRf, (float)(1.02 * mx));
    if (i == 0) {
        t.msc[2 * m] = (float)c.S1;
        t.msc[2 * m + 1] = (float)c.S2;
    }
    t.scratch[idx] = (i == 0) ? E / L_tot(c, E, pp) : inv_L_integral(c, node_E(i - 1), E, pp);
}

__global__ void k_range_scan(Tables t)
{
    int m = threadIdx.x;
    if (m >= t.n_mat) return;
    double R = 0.0;
    for (int i = 0; i < NE; ++i) {
        R += t.scratch[m * NE + i];
        t.scratch[m * NE + i] = R;                 // cumulative range at node i
        t.el[m * NE + i].x = (float)log(R);
    }
    double lo = log(t.scratch[m * NE]), hi = log(t.scratch[m * NE + NE - 1]);
    t.rmeta[2 * m] = (float)lo;
    t.rmeta[2 * m + 1] = (float)((NR - 1) / (hi - lo));
}

__global__ void k_range_inverse(Tables t, PhysParams pp)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= t.n_mat * NR) return;
    int m = idx / NR, j = idx % NR;
    MC c = mconst(t.mats[m]);
    const double* R = t.scratch + m * NE;
    double lo = log(R[0]), hi = log(R[NE - 1]);
    double Rt = exp(lo + (hi - lo) * j / (NR - 1));
    int a = 0, b = NE - 1;                          // R[a] <= Rt <= R[b]
    while (b - a > 1) {
        int mid = (a + b) / 2;
        if (R[mid] <= Rt) a = mid; else b = mid;
    }
    double E;
    if (j == 0) E = node_E(0);
    else if (j == NR - 1) E = node_E(NE - 1);
    else {
        double e0 = node_E(a), el = e0, eh = node_E(b);
        for (int it = 0; it < 60; ++it) {
            double em = 0.5 * (el + eh);
            if (R[a] + inv_L_integral(c, e0, em, pp) < Rt) el = em; else eh = em;
        }
        E = 0.5 * (el + eh);
    }
    t.rinv[idx] = (float)log(E);
}

__global__ void k_ms_table(Tables t)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NG) return;
    double lg = log(G1_LO) + (log(G1_ISO) - log(G1_LO)) * j / (NG - 1);
    t.msA[j] = (float)wentzel_solve(exp(lg));
}

// Per-material maximum density and the validity check. Maxima are gathered in shared memory
// first (one global atomic per material and block): with every voxel's atomic going to the same
// few global words the scan took 1.3 ms on a 128^3 phantom.
__global__ void k_phantom_scan(const float* density, const uint8_t* material, long long nvox, int n_mat,
                               unsigned int* rho_max, int* err)
{
    __shared__ unsigned int s_max[MAX_STAGED];
    __shared__ int s_bad;
    for (int m = threadIdx.x; m < MAX_STAGED; m += blockDim.x) s_max[m] = 0u;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    bool bad = false;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        float r = density[v];
        int m = material[v];
        const bool ok = m < n_mat && r >= 0.f && r <= 30.f;
        bad |= !ok;
        // lanes of one material take their maximum together; one shared atomic per material
        const unsigned key = ok ? (unsigned)m : 0xFFu;
        const unsigned grp = __match_any_sync(__activemask(), key);
        const unsigned mx = __reduce_max_sync(grp, ok && r > 0.f ? __float_as_uint(r) : 0u);   // non-negative floats order as their bits
        if (ok && mx && (threadIdx.x & 31) == __ffs(grp) - 1) atomicMax(s_max + m, mx);
    }
    if (bad) s_bad = 1;
    __syncthreads();
    for (int m = threadIdx.x; m < n_mat; m += blockDim.x)
        if (s_max[m]) atomicMax(rho_max + m, s_max[m]);
    if (threadIdx.x == 0 && s_bad) atomicOr(err, ERR_PHANTOM);
}

__global__ void k_photon_majorant(Tables t)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NE) return;
    float best = -1e30f;
    for (int m = 0; m < t.n_mat; ++m) {
        float r = __uint_as_float(t.rho_max[m]);
        if (r > 0.f) best = fmaxf(best, (float)log((double)r) + t.ph[m * NE + i].x);
    }
    t.phmaj[i] = best > -1e29f ? best + 1e-6f : best;   // small margin over FP32 rounding
    // voxel-crossing electron steps: max over materials of rho_max * (hard-event majorant of a
    // step starting in [E_i, E_i+1)), so a step's candidate events may fall in any voxel
    float hm = 0.f;
    for (int m = 0; m < t.n_mat; ++m) hm = fmaxf(hm, __uint_as_float(t.rho_max[m]) * t.el2[m * NE + i].y);
    t.elmaj[i] = hm * 1.00001f;
}

}  // namespace

void material_defs(MatDef out[NMAT_DEFAULT])
{
    // mass fractions: water H2O; cortical bone (ICRP); lung (ICRP)
    MatDef water = {2, {1, 8}, {1.008, 15.999}, {0.111894, 0.888106}, 75.0, 1.0};
    MatDef bone = {9, {1, 6, 7, 8, 12, 15, 16, 20, 30},
                   {1.008, 12.011, 14.007, 15.999, 24.305, 30.974, 32.06, 40.078, 65.38},
                   {0.047234, 0.144330, 0.041990, 0.446096, 0.002200, 0.104970, 0.003150, 0.209930, 0.000100},
                   106.4, 1.85};
    MatDef lung = {13, {1, 6, 7, 8, 11, 12, 15, 16, 17, 19, 20, 26, 30},
                   {1.008, 12.011, 14.007, 15.999, 22.990, 24.305, 30.974, 32.06, 35.45, 39.098, 40.078, 55.845, 65.38},
                   {0.101278, 0.102310, 0.028650, 0.757072, 0.001840, 0.000730, 0.000800, 0.002250, 0.002660,
                    0.001940, 0.000090, 0.000370, 0.000010},
                   75.3, 0.26};
    out[0] = water;
    out[1] = bone;
    out[2] = lung;
}

// Material tables for the t.n_mat staged materials defs[0 .. n_mat) (table row m = defs[m]):
// they depend on the compositions and the physics parameters only, not on the phantom.
cudaError_t build_material_tables(const Tables& t, const PhysParams& pp, const MatDef* defs, cudaStream_t s)
{
    if (t.n_mat < 1 || t.n_mat > MAX_STAGED) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyAsync(t.mats, defs, sizeof(MatDef) * t.n_mat, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_nodes<<<(t.n_mat * NE + 127) / 128, 128, 0, s>>>(t, pp);
    k_range_scan<<<1, 32, 0, s>>>(t);
    k_range_inverse<<<(t.n_mat * NR + 127) / 128, 128, 0, s>>>(t, pp);
    k_ms_table<<<(NG + 127) / 128, 128, 0, s>>>(t);
    return cudaGetLastError();
}

// Phantom-dependent part: per-material maximum density (with the phantom's validity check) and
// the photon majorant built from it.
cudaError_t build_phantom_tables(const Tables& t, const float* density, const uint8_t* material, long long nvox,
                                 int* d_err, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(t.rho_max, 0, t.n_mat * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    k_phantom_scan<<<1024, 256, 0, s>>>(density, material, nvox, t.n_mat, t.rho_max, d_err);
    k_photon_majorant<<<(NE + 127) / 128, 128, 0, s>>>(t);
    return cudaGetLastError();
}

cudaError_t build_tables(const Tables& t, const PhysParams& pp, const float* density, const uint8_t* material,
                         long long nvox, int* d_err, const MatDef* defs, cudaStream_t s)
{
    cudaError_t e = build_material_tables(t, pp, defs, s);
    return e != cudaSuccess ? e : build_phantom_tables(t, density, material, nvox, d_err, s);
}

}  // namespace ocmc
