/*
 * ocmc_oracle.c -- TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).
 *
 * A plain, slow, double-precision CPU implementation of the coupled
 * photon-electron Monte Carlo dose method of Tian et al. ("oclMC"):
 *   - photons: analogue transport with Woodcock (delta) tracking; Compton,
 *     photoelectric and pair events (Sec. 2.1, photon paragraph);
 *   - electrons/positrons: Class II condensed history, step
 *     d = min(d_vox, d_maxs, d_maxe, d_event) confined to one voxel, hard
 *     event distance sampled with Woodcock in energy, discrete Moller and
 *     bremsstrahlung events, random-hinge multiple scattering, CSDA loss
 *     deposited in the step's voxel, positron annihilation into two photons
 *     (Sec. 2.1, electron paragraph);
 *   - dose tally per statistical batch; output MeV/g per source particle
 *     (Sec. 2.2 "Materials", last paragraph).
 * Physics quantities are evaluated from their closed forms at every use; no
 * tables. Sampling uses the most direct correct methods (rejection from the
 * definition, or bisection on a closed-form cumulative distribution).
 * Random numbers: Philox4x32-10 (Salmon et al. 2011), keyed by the seed, with
 * the counter carrying (draw block, history id, particle sub-stream).
 *
 * Model choices where the paper gives only a name (each is a published
 * closed form): Klein-Nishina on free electrons; K-shell Born photoelectric
 * cross section; Maximon's pair cross-section expansions with Z(Z+1);
 * ICRU-37 restricted collision stopping power with the Sternheimer-Peierls
 * density effect; complete-screening Bethe-Heitler bremsstrahlung with
 * Z(Z+1); Moller cross section; screened-Rutherford (Moliere screening)
 * transport cross section with a modified-Wentzel angular distribution that
 * reproduces <cos theta> = exp(-s/lambda_1).
 */
#include "ocmc_oracle.h"
#include <math.h>
#include <string.h>
#include <stdlib.h>

/* ---- physical constants (CODATA 2018) ---------------------------------- */
static const double MC2   = 0.51099895000;        /* MeV            */
static const double RE    = 2.8179403262e-13;     /* cm             */
static const double ALPHA = 1.0 / 137.035999084;
static const double NAV   = 6.02214076e23;        /* 1/mol          */
static const double PI    = 3.14159265358979323846;
static const double ZETA3 = 1.2020569031595942;
static const double TALLY_SCALE = 268435456.0;    /* 2^28 units per MeV */

/* ---- materials: element mass fractions (ICRU/ICRP compositions) --------- */
typedef struct { int Z; double A; double w; } elem;
typedef struct {
    const char* name; double I_eV; double rho0; int n; elem e[ORC_MAX_ELEM];
    /* derived per-gram constants (computed once by orc_init) */
    double n_e, photo, pairZ, S1, S2;
    double dC, dX0, dX1, dA;    /* Sternheimer-Peierls density-effect parameters */
} material;

static material MAT[ORC_MAX_MAT] = {
    { "water", 75.0, 1.0, 2, { {1, 1.008, 0.111894}, {8, 15.999, 0.888106} } },
    { "bone_cortical_icrp", 106.4, 1.85, 9, {
        {1, 1.008, 0.047234}, {6, 12.011, 0.144330}, {7, 14.007, 0.041990},
        {8, 15.999, 0.446096}, {12, 24.305, 0.002200}, {15, 30.974, 0.104970},
        {16, 32.06, 0.003150}, {20, 40.078, 0.209930}, {30, 65.38, 0.000100} } },
    { "lung_icrp", 75.3, 0.26, 13, {
        {1, 1.008, 0.101278}, {6, 12.011, 0.102310}, {7, 14.007, 0.028650},
        {8, 15.999, 0.757072}, {11, 22.990, 0.001840}, {12, 24.305, 0.000730},
        {15, 30.974, 0.000800}, {16, 32.06, 0.002250}, {17, 35.45, 0.002660},
        {19, 39.098, 0.001940}, {20, 40.078, 0.000090}, {26, 55.845, 0.000370},
        {30, 65.38, 0.000010} } },
};

static int N_MAT = 3;
static material DEFAULT_MAT[3];

/* Per-gram constants of material M from its composition (the atoms of each element per gram
 * are N_A w_i / A_i). */
static void derive_material(material* M)
{
    double wsum = 0.0;
    for (int i = 0; i < M->n; ++i) wsum += M->e[i].w;
    M->n_e = M->photo = M->pairZ = M->S1 = M->S2 = 0.0;
    for (int i = 0; i < M->n; ++i) {
        double Z = M->e[i].Z, atoms = NAV * (M->e[i].w / wsum) / M->e[i].A; /* per g */
        M->n_e   += atoms * Z;
        M->photo += atoms * pow(Z, 5.0);
        M->pairZ += atoms * Z * (Z + 1.0);
        M->S1    += atoms * Z * (Z + 1.0) * log(183.0 * pow(Z, -1.0 / 3.0));
        M->S2    += atoms * Z * (Z + 1.0) / 9.0;
    }
    /* Sternheimer & Peierls (1971) general density-effect parameters for
       condensed media, evaluated at the material's nominal density. */
    double hw = 28.816 * sqrt(M->rho0 * M->n_e / NAV);      /* eV */
    double C = 2.0 * log(M->I_eV / hw) + 1.0, x0, x1;
    if (M->I_eV < 100.0) { x1 = 2.0; x0 = (C < 3.681) ? 0.2 : 0.326 * C - 1.0; }
    else                 { x1 = 3.0; x0 = (C < 5.215) ? 0.2 : 0.326 * C - 1.5; }
    M->dC = C; M->dX0 = x0; M->dX1 = x1;
    M->dA = (C - 2.0 * log(10.0) * x0) / pow(x1 - x0, 3.0);
}

void orc_init(void)
{
    static int done = 0;
    if (done) return;
    done = 1;
    for (int m = 0; m < 3; ++m) {
        derive_material(&MAT[m]);
        DEFAULT_MAT[m] = MAT[m];
    }
    N_MAT = 3;
}

int orc_set_materials(int n, const orc_material* defs)
{
    orc_init();
    if (n < 1 || n > ORC_MAX_MAT || !defs) return -1;
    for (int m = 0; m < n; ++m) {
        const orc_material* d = defs + m;
        double wsum = 0.0;
        if (d->n_elements < 1 || d->n_elements > ORC_MAX_ELEM || !(d->I_eV > 0.0) || !(d->density > 0.0)) return -1;
        for (int i = 0; i < d->n_elements; ++i) {
            if (d->Z[i] < 1 || d->Z[i] > 100 || !(d->A[i] > 0.0) || !(d->mass_fraction[i] >= 0.0)) return -1;
            wsum += d->mass_fraction[i];
        }
        if (!(wsum > 0.0)) return -1;
    }
    for (int m = 0; m < n; ++m) {
        const orc_material* d = defs + m;
        material* M = &MAT[m];
        memset(M, 0, sizeof(*M));
        M->name = "user";
        M->I_eV = d->I_eV;
        M->rho0 = d->density;
        M->n = d->n_elements;
        for (int i = 0; i < d->n_elements; ++i) {
            M->e[i].Z = d->Z[i]; M->e[i].A = d->A[i]; M->e[i].w = d->mass_fraction[i];
        }
        derive_material(M);
    }
    N_MAT = n;
    return 0;
}

void orc_reset_materials(void)
{
    orc_init();
    for (int m = 0; m < 3; ++m) MAT[m] = DEFAULT_MAT[m];
    N_MAT = 3;
}

int orc_n_materials(void) { return N_MAT; }

double orc_material_const(int m, int which)
{
    const material* M = &MAT[m];
    switch (which) {
    case 0: return M->n_e;  case 1: return M->photo; case 2: return M->pairZ;
    case 3: return M->S1;   case 4: return M->S2;    case 5: return M->I_eV;
    case 6: return M->rho0; case 7: return M->dC;    case 8: return M->dX0;
    case 9: return M->dX1;  case 10: return M->dA;
    }
    return NAN;
}

/* ---- photon cross sections ---------------------------------------------- */
/* Klein-Nishina total cross section per free electron (cm^2). */
double orc_sigma_kn(double E)
{
    double k = E / MC2, l = log(1.0 + 2.0 * k);
    double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / (1.0 + 2.0 * k) - l / k);
    double t2 = l / (2.0 * k);
    double t3 = (1.0 + 3.0 * k) / ((1.0 + 2.0 * k) * (1.0 + 2.0 * k));
    return 2.0 * PI * RE * RE * (t1 + t2 - t3);
}

/* K-shell Born photoelectric cross section 4 sqrt2 alpha^4 Z^5 sigma_T (mc^2/E)^(7/2). */
static double photo_per_Z5(double E)
{
    double sigT = 8.0 * PI / 3.0 * RE * RE;
    return 4.0 * sqrt(2.0) * pow(ALPHA, 4.0) * sigT * pow(MC2 / E, 3.5);
}

/* Pair production in the nuclear field, per alpha r_e^2 Z(Z+1): Maximon's
   near-threshold expansion for k <= 4 mc^2, Maximon's high-energy expansion
   above; zero at and below 2 mc^2. */
static double pair_shape(double E)
{
    double k = E / MC2;
    if (k <= 2.0) return 0.0;
    double f;
    if (k <= 4.0) {
        double e = (2.0 * k - 4.0) / (2.0 + k + 2.0 * sqrt(2.0 * k));
        double r = (k - 2.0) / k;
        f = 2.0 * PI / 3.0 * r * r * r *
            (1.0 + e / 2.0 + 23.0 * e * e / 40.0 + 11.0 * e * e * e / 60.0 + 29.0 * e * e * e * e / 960.0);
    } else {
        double L = log(2.0 * k), q = 2.0 / k, q2 = q * q;
        f = 28.0 / 9.0 * L - 218.0 / 27.0
          + q2 * (6.0 * L - 3.5 + 2.0 / 3.0 * L * L * L - L * L - PI * PI / 3.0 * L + 2.0 * ZETA3 + PI * PI / 6.0)
          - q2 * q2 * (3.0 / 16.0 * L + 1.0 / 8.0)
          - q2 * q2 * q2 * (29.0 / (9.0 * 256.0) * L - 77.0 / (27.0 * 512.0));
    }
    return f > 0.0 ? f : 0.0;
}

double orc_mu(int m, double E, int channel)
{
    const material* M = &MAT[m];
    double c = M->n_e * orc_sigma_kn(E);
    double p = M->photo * photo_per_Z5(E);
    double q = M->pairZ * ALPHA * RE * RE * pair_shape(E);
    switch (channel) {
    case 1: return c; case 2: return p; case 3: return q;
    }
    return c + p + q;
}

/* ---- electron stopping powers and cross sections ----------------------- */
double orc_density_effect(int m, double T)
{
    const material* M = &MAT[m];
    double tau = T / MC2;
    double x = log10(sqrt(tau * (tau + 2.0)));              /* log10(beta*gamma) */
    double ln10 = log(10.0);
    if (x < M->dX0) return 0.0;
    if (x < M->dX1) return 2.0 * ln10 * x - M->dC + M->dA * pow(M->dX1 - x, 3.0);
    return 2.0 * ln10 * x - M->dC;
}

/* ICRU-37 restricted collision stopping power (soft Moller losses W < w_cc). */
double orc_L_col(int m, double T, double w_cc)
{
    const material* M = &MAT[m];
    double tau = T / MC2, g = tau + 1.0, b2 = 1.0 - 1.0 / (g * g);
    double d = fmin(w_cc, 0.5 * T) / MC2;
    double Ir = M->I_eV * 1e-6 / MC2;
    double F = -1.0 - b2 + log((tau - d) * d) + tau / (tau - d)
             + (0.5 * d * d + (2.0 * tau + 1.0) * log(1.0 - d / tau)) / (g * g);
    double K = 2.0 * PI * RE * RE * MC2 * M->n_e;
    return K / b2 * (log(2.0 * (tau + 2.0) / (Ir * Ir)) + F - orc_density_effect(m, T));
}

/* Restricted radiative stopping power: integral of k dsigma/dk over k < w_cb
   for the complete-screening Bethe-Heitler spectrum
   dsigma/dk = 4 alpha r_e^2 / k [ (4/3 - 4/3 y + y^2) S1 + (1 - y) S2 ], y = k/E. */
double orc_L_rad(int m, double T, double w_cb)
{
    const material* M = &MAT[m];
    double E = T + MC2, k1 = fmin(w_cb, T);
    double a = M->S1 * (4.0 / 3.0 * k1 - 2.0 / 3.0 * k1 * k1 / E + k1 * k1 * k1 / (3.0 * E * E));
    double b = M->S2 * (k1 - 0.5 * k1 * k1 / E);
    return 4.0 * ALPHA * RE * RE * (a + b);
}

static double brems_cdf_unnorm(const material* M, double k, double E)
{
    return M->S1 * (4.0 / 3.0 * log(k) - 4.0 / 3.0 * k / E + k * k / (2.0 * E * E))
         + M->S2 * (log(k) - k / E);
}

double orc_sigma_brems(int m, double T, double w_cb)
{
    if (T <= w_cb) return 0.0;
    const material* M = &MAT[m];
    double E = T + MC2;
    return 4.0 * ALPHA * RE * RE * (brems_cdf_unnorm(M, T, E) - brems_cdf_unnorm(M, w_cb, E));
}

/* Moller integrand antiderivative in eps = W/T (without the common factor). */
static double moller_F(double e, double c, double d)
{
    return -1.0 / e + 1.0 / (1.0 - e) + c * e - d * log(e / (1.0 - e));
}

double orc_sigma_moller(int m, double T, double w_cc)
{
    if (T <= 2.0 * w_cc) return 0.0;
    const material* M = &MAT[m];
    double tau = T / MC2, g = tau + 1.0, b2 = 1.0 - 1.0 / (g * g);
    double c = (tau / g) * (tau / g), d = (2.0 * tau + 1.0) / (g * g);
    double e0 = w_cc / T;
    double K = 2.0 * PI * RE * RE * MC2 * M->n_e;
    return K / (b2 * T) * (moller_F(0.5, c, d) - moller_F(e0, c, d));
}

static double orc_sigma_hard(int m, double T, const orc_params* p)
{
    if (p->flags & ORC_NO_HARD) return 0.0;
    return orc_sigma_moller(m, T, p->w_cc) + orc_sigma_brems(m, T, p->w_cb);
}

static double L_total(int m, double T, const orc_params* p)
{
    if (T < 1e-3) T = 1e-3;
    return orc_L_col(m, T, p->w_cc) + orc_L_rad(m, T, p->w_cb);
}

/* First transport cross section of the screened Rutherford (Wentzel) model
   with Moliere screening, summed over elements: 1/lambda_1 in cm^2/g. */
double orc_lambda1_inv(int m, double T)
{
    const material* M = &MAT[m];
    double wsum = 0.0;
    for (int i = 0; i < M->n; ++i) wsum += M->e[i].w;
    double pc2 = T * (T + 2.0 * MC2), pc = sqrt(pc2), b = pc / (T + MC2);
    double pbc = pc * b, s = 0.0;
    for (int i = 0; i < M->n; ++i) {
        double Z = M->e[i].Z, atoms = NAV * (M->e[i].w / wsum) / M->e[i].A;
        double a = ALPHA * cbrt(Z) * MC2 / (0.885 * pc);
        double eta = 0.25 * a * a * (1.13 + 3.76 * (ALPHA * Z / b) * (ALPHA * Z / b));
        double sig1 = 2.0 * PI * Z * (Z + 1.0) * RE * RE * (MC2 / pbc) * (MC2 / pbc)
                    * (log1p(1.0 / eta) - 1.0 / (1.0 + eta));
        s += atoms * sig1;
    }
    return s;
}

/* Mean of u = 1 - cos(theta) for the Wentzel distribution p(u) ~ (u + 2A)^-2 on [0,2]. */
double orc_ms_mean_u(double A)
{
    if (A > 1e3) { double x = 1.0 / A; return 1.0 - x / 3.0 + x * x / 6.0 - x * x * x / 10.0; }
    return 2.0 * A * ((1.0 + A) * log1p(1.0 / A) - 1.0);
}

/* Screening parameter A with <u>(A) = 1 - exp(-G1), by bisection in ln A. */
double orc_ms_solve_A(double G1)
{
    double target = -expm1(-G1);
    double lo = log(1e-40), hi = log(1e15);
    for (int it = 0; it < 90; ++it) {
        double mid = 0.5 * (lo + hi);
        if (orc_ms_mean_u(exp(mid)) < target) lo = mid; else hi = mid;
    }
    return exp(0.5 * (lo + hi));
}

/* Above this G1 the deflection is taken as isotropic. */
static const double MS_G1_ISO = 15.0;
static const double MS_G1_NONE = 1e-12;

/* CSDA energy after a mass thickness X (g/cm^2): RK4 on dT/dX = -L(T), 32 substeps. */
double orc_csda_loss(int m, double T, double X, const orc_params* p)
{
    double h = X / 32.0, E = T;
    for (int i = 0; i < 32; ++i) {
        double k1 = L_total(m, E, p);
        double k2 = L_total(m, E - 0.5 * h * k1, p);
        double k3 = L_total(m, E - 0.5 * h * k2, p);
        double k4 = L_total(m, E - h * k3, p);
        E -= h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
        if (E <= 0.0) return 0.0;
    }
    return E;
}

/* 8-point Gauss-Legendre nodes and weights on [-1,1]. */
static const double GLX[4] = { 0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363 };
static const double GLW[4] = { 0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763 };

/* Mass thickness needed to slow from T to Tlo: integral of dT / L(T). */
static double range_between(int m, double Tlo, double T, const orc_params* p)
{
    double c = 0.5 * (T + Tlo), h = 0.5 * (T - Tlo), s = 0.0;
    for (int i = 0; i < 4; ++i)
        s += GLW[i] * (1.0 / L_total(m, c + h * GLX[i], p) + 1.0 / L_total(m, c - h * GLX[i], p));
    return s * h;
}

/* ---- Philox4x32-10 -------------------------------------------------------- */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0; c1 = (uint32_t)p1; c2 = n2; c3 = (uint32_t)p0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A particle's random stream: counter = (draw block, history lo, history hi, sub).
   Draw n is word n mod 4 of block n/4; a word x maps to ((x >> 8) + 1) 2^-24. */
typedef struct { uint32_t key[2]; uint64_t hist; uint32_t sub; uint32_t n; } stream;

static double rnd(stream* s)
{
    uint32_t ctr[4] = { s->n >> 2, (uint32_t)s->hist, (uint32_t)(s->hist >> 32), s->sub };
    uint32_t out[4];
    orc_philox(ctr, s->key, out);
    uint32_t x = out[s->n & 3u];
    s->n++;
    return (double)((x >> 8) + 1u) * (1.0 / 16777216.0);   /* (0, 1] on a 2^-24 grid */
}

static uint32_t child_sub(uint32_t parent, uint32_t n, uint32_t slot)
{
    uint32_t h = parent * 0x9E3779B1u ^ (n + 0x7F4A7C15u) * 0x85EBCA77u ^ (slot + 1u) * 0xC2B2AE3Du;
    h ^= h >> 16; h *= 0x85EBCA6Bu; h ^= h >> 13; h *= 0xC2B2AE35u; h ^= h >> 16;
    return h == 0u ? 1u : h;
}

/* ---- sampling ------------------------------------------------------------ */
/* Compton: cos(theta) by rejection from the Klein-Nishina d sigma / d Omega,
   whose maximum over angle is 2 pi r_e^2 at theta = 0. */
static double sample_kn_mu(double E, stream* s)
{
    double k = E / MC2;
    for (;;) {
        double mu = 2.0 * rnd(s) - 1.0;
        double e = 1.0 / (1.0 + k * (1.0 - mu));
        double f = e * e * e + e - e * e * (1.0 - mu * mu);
        if (2.0 * rnd(s) <= f) return mu;
    }
}

/* Moller: eps = W/T on [w_cc/T, 1/2] by bisection on the closed-form CDF. */
static double sample_moller_eps(double T, double w_cc, stream* s)
{
    double tau = T / MC2, g = tau + 1.0;
    double c = (tau / g) * (tau / g), d = (2.0 * tau + 1.0) / (g * g);
    double e0 = w_cc / T, F0 = moller_F(e0, c, d), F1 = moller_F(0.5, c, d);
    double target = F0 + rnd(s) * (F1 - F0), lo = e0, hi = 0.5;
    for (int it = 0; it < 64; ++it) {
        double mid = 0.5 * (lo + hi);
        if (moller_F(mid, c, d) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Bremsstrahlung: photon energy k on [w_cb, T] by bisection on the CDF. */
static double sample_brems_k(int m, double T, double w_cb, stream* s)
{
    const material* M = &MAT[m];
    double E = T + MC2, G0 = brems_cdf_unnorm(M, w_cb, E), G1 = brems_cdf_unnorm(M, T, E);
    double target = G0 + rnd(s) * (G1 - G0), lo = log(w_cb), hi = log(T);
    for (int it = 0; it < 64; ++it) {
        double mid = 0.5 * (lo + hi);
        if (brems_cdf_unnorm(M, exp(mid), E) < target) lo = mid; else hi = mid;
    }
    return exp(0.5 * (lo + hi));
}

/* Multiple-scattering polar cosine for a path with G1 = s / lambda_1. */
static double sample_ms_mu(double G1, stream* s)
{
    if (G1 < MS_G1_NONE) { (void)rnd(s); return 1.0; }
    if (G1 >= MS_G1_ISO) return 2.0 * rnd(s) - 1.0;
    double A = orc_ms_solve_A(G1), xi = 1.0 - rnd(s);          /* xi in [0, 1) */
    double u = 2.0 * A * xi / (1.0 + A - xi);
    double mu = 1.0 - u;
    return mu < -1.0 ? -1.0 : (mu > 1.0 ? 1.0 : mu);
}

/* ---- geometry helpers --------------------------------------------------- */
static void normalize3(double* a)
{
    double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= n; a[1] /= n; a[2] /= n;
}

/* Rotate unit vector d by polar cosine mu and azimuth phi about itself. */
static void rotate(double* d, double mu, double phi)
{
    double st = sqrt(fmax(0.0, 1.0 - mu * mu)), cp = cos(phi), sp = sin(phi);
    double u = d[0], v = d[1], w = d[2], s = sqrt(u * u + v * v);   /* not sqrt(1 - w^2): no cancellation near the poles */
    if (s > 1e-10) {
        d[0] = u * mu + st * (u * w * cp - v * sp) / s;
        d[1] = v * mu + st * (v * w * cp + u * sp) / s;
        d[2] = w * mu - s * st * cp;
    } else {
        double sg = w >= 0.0 ? 1.0 : -1.0;
        d[0] = st * cp; d[1] = st * sp; d[2] = sg * mu;
    }
    normalize3(d);
}

/* ---- event kinematics (Sec. 2.1) ------------------------------------------ */
/* Each function draws its random numbers from the particle's stream in a fixed order and
   returns the outgoing energies and unit directions; d0 is the incoming unit direction. */

/* Compton scattering of a photon of energy E0: polar cosine mu from Klein-Nishina, uniform
   azimuth; the scattered photon energy follows from mu, and the recoil electron carries the
   kinetic energy T = E0 - E1 along the momentum balance E0 d0 - E1 d1 (units MeV/c). */
static void compton_event(double E0, const double* d0, stream* rs,
                          double* E1, double* d1, double* T, double* de)
{
    double mu = sample_kn_mu(E0, rs), phi = 2.0 * PI * rnd(rs);
    *E1 = E0 / (1.0 + E0 / MC2 * (1.0 - mu));
    *T = E0 - *E1;
    d1[0] = d0[0]; d1[1] = d0[1]; d1[2] = d0[2];
    rotate(d1, mu, phi);
    de[0] = E0 * d0[0] - *E1 * d1[0];
    de[1] = E0 * d0[1] - *E1 * d1[1];
    de[2] = E0 * d0[2] - *E1 * d1[2];
    if (*T > 0.0) normalize3(de);
}

/* Moller event of an electron of kinetic energy T0 above the threshold w_cc: energy fraction
   eps of the knock-on electron, uniform azimuth; both polar cosines follow from energy and
   momentum conservation for a free electron at rest, and the two outgoing electrons lie in one
   plane with the incoming direction, on opposite sides of it. */
static void moller_event(double T0, double w_cc, const double* d0, stream* rs,
                         double* T1, double* d1, double* W, double* d2)
{
    double eps = sample_moller_eps(T0, w_cc, rs), phi = 2.0 * PI * rnd(rs);
    *W = eps * T0;
    *T1 = T0 - *W;
    double mu1 = sqrt(fmin(1.0, *T1 * (T0 + 2.0 * MC2) / (T0 * (*T1 + 2.0 * MC2))));
    double mu2 = sqrt(fmin(1.0, *W * (T0 + 2.0 * MC2) / (T0 * (*W + 2.0 * MC2))));
    d2[0] = d0[0]; d2[1] = d0[1]; d2[2] = d0[2];
    rotate(d2, mu2, phi + PI);
    d1[0] = d0[0]; d1[1] = d0[1]; d1[2] = d0[2];
    rotate(d1, mu1, phi);
}

/* Bremsstrahlung event of an electron of kinetic energy T0 in material m: photon energy k
   on [w_cb, T0]; the photon leaves at the fixed polar angle mc^2 / (T0 + mc^2) with uniform
   azimuth, and the electron keeps its direction. */
static void brems_event(int m, double T0, double w_cb, const double* d0, stream* rs,
                        double* k, double* dg)
{
    *k = sample_brems_k(m, T0, w_cb, rs);
    double th = MC2 / (T0 + MC2), phi = 2.0 * PI * rnd(rs);
    dg[0] = d0[0]; dg[1] = d0[1]; dg[2] = d0[2];
    rotate(dg, cos(th), phi);
}

/* Annihilation of a positron at rest: two photons of mc^2 back to back, the first one's
   direction isotropic (uniform polar cosine and azimuth). */
static void annihilation_event(stream* rs, double* d1, double* d2)
{
    double w = 2.0 * rnd(rs) - 1.0, phi = 2.0 * PI * rnd(rs), st = sqrt(fmax(0.0, 1.0 - w * w));
    d1[0] = st * cos(phi); d1[1] = st * sin(phi); d1[2] = w;
    d2[0] = -d1[0]; d2[1] = -d1[1]; d2[2] = -d1[2];
}

/* ---- transport ----------------------------------------------------------- */
enum { PHOTON = 0, ELECTRON = 1, POSITRON = 2 };
typedef struct { double r[3], d[3], E; int i[3]; int type; stream rs; } particle;

#define STACK_MAX 4096
typedef struct {
    const orc_phantom* ph; const orc_params* p;
    int64_t* tally; double* ledger; uint64_t* cnt;
    uint64_t hist; int64_t nvox; double L[3]; double dd[3]; int nn[3];
    double rho_max[ORC_MAX_MAT]; int present[ORC_MAX_MAT];
    particle stack[STACK_MAX]; int top;
} run_ctx;

static void deposit(run_ctx* c, const int* i, double dE)
{
    if (dE <= 0.0) return;
    int64_t v = i[0] + (int64_t)c->nn[0] * (i[1] + (int64_t)c->nn[1] * i[2]);
    int64_t b = (int64_t)(c->hist % (uint64_t)c->p->n_batches);
    c->tally[b * c->nvox + v] += llrint(dE * TALLY_SCALE);
    c->ledger[ORC_L_EDEP] += dE;
}

static void push(run_ctx* c, const particle* q)
{
    if (c->top >= STACK_MAX) { c->cnt[ORC_C_STACK_OVERFLOW]++; return; }
    c->stack[c->top++] = *q;
}

static int inside_index(const run_ctx* c, const int* i)
{
    return i[0] >= 0 && i[0] < c->nn[0] && i[1] >= 0 && i[1] < c->nn[1] && i[2] >= 0 && i[2] < c->nn[2];
}

static void index_of(const run_ctx* c, const double* r, int* i)
{
    for (int a = 0; a < 3; ++a) {
        int k = (int)floor(r[a] / c->dd[a]);
        i[a] = k < 0 ? 0 : (k >= c->nn[a] ? c->nn[a] - 1 : k);
    }
}

static double voxel_rho(const run_ctx* c, const int* i, int* m)
{
    int64_t v = i[0] + (int64_t)c->nn[0] * (i[1] + (int64_t)c->nn[1] * i[2]);
    *m = c->ph->material[v];
    return (double)c->ph->density[v];
}

/* Distance from r along d to the faces of voxel i; returns the face as
   axis*2 + (d>0). */
static double dist_to_face(const run_ctx* c, const double* r, const double* d, const int* i, int* face)
{
    double best = INFINITY; int f = -1;
    for (int a = 0; a < 3; ++a) {
        double t;
        if (d[a] > 0.0)      t = ((i[a] + 1) * c->dd[a] - r[a]) / d[a];
        else if (d[a] < 0.0) t = (i[a] * c->dd[a] - r[a]) / d[a];
        else continue;
        if (t < 0.0) t = 0.0;
        if (t < best) { best = t; f = a * 2 + (d[a] > 0.0 ? 1 : 0); }
    }
    *face = f;
    return best;
}

static void cross_face(const run_ctx* c, particle* q, int face)
{
    int a = face >> 1;
    if (face & 1) { q->r[a] = (q->i[a] + 1) * c->dd[a]; q->i[a] += 1; }
    else          { q->r[a] = q->i[a] * c->dd[a];       q->i[a] -= 1; }
}

static double photon_majorant(const run_ctx* c, double E)
{
    double mx = 0.0;
    for (int m = 0; m < N_MAT; ++m)
        if (c->present[m]) mx = fmax(mx, c->rho_max[m] * orc_mu(m, E, 0));
    return mx;
}

static void escape(run_ctx* c, const particle* q)
{
    c->ledger[ORC_L_EESC] += q->E;
    c->cnt[ORC_C_ESCAPED]++;
}

static particle make_child(const particle* parent, uint32_t slot, int type, double E, const double* d)
{
    particle q = *parent;
    q.type = type; q.E = E;
    q.d[0] = d[0]; q.d[1] = d[1]; q.d[2] = d[2];
    q.rs.sub = child_sub(parent->rs.sub, parent->rs.n, slot);
    q.rs.n = 0;
    return q;
}

/* Positron at rest: two photons of mc^2, back to back, isotropic. */
static void annihilate(run_ctx* c, particle* q)
{
    double d1[3], d2[3];
    annihilation_event(&q->rs, d1, d2);
    c->cnt[ORC_C_ANNIH]++;
    c->ledger[ORC_L_ANNIHMASS] += 2.0 * MC2;
    if (MC2 >= c->p->e_abs_g) {
        particle a = make_child(q, 0, PHOTON, MC2, d1); push(c, &a);
        particle b = make_child(q, 1, PHOTON, MC2, d2); push(c, &b);
    } else {
        deposit(c, q->i, 2.0 * MC2);
    }
}

/* A charged particle that has fallen below its absorption energy. */
static void absorb_charged(run_ctx* c, particle* q)
{
    deposit(c, q->i, q->E);
    if (q->type == POSITRON) annihilate(c, q);
}

/* A newly created e-/e+ at q's position: transported if above cutoff. */
static void emit_charged(run_ctx* c, particle* q)
{
    if (q->E >= c->p->e_abs_e && !(c->p->flags & ORC_KERMA)) { push(c, q); return; }
    absorb_charged(c, q);
}

static void transport_photon(run_ctx* c, particle* q)
{
    const orc_params* p = c->p;
    int killed_mode = (p->flags & ORC_KILL_FIRST_REAL) != 0;
    for (;;) {
        double mx = photon_majorant(c, q->E);
        double s = mx > 0.0 ? -log(rnd(&q->rs)) / mx : INFINITY;
        int out = 0;
        if (isinf(s)) out = 1;
        else {
            for (int a = 0; a < 3; ++a) q->r[a] += s * q->d[a];
            for (int a = 0; a < 3; ++a) if (q->r[a] < 0.0 || q->r[a] > c->L[a]) out = 1;
        }
        c->cnt[ORC_C_FLIGHTS]++;
        if (out) {
            if (killed_mode && !isinf(s) && q->r[2] > c->L[2]) {
                c->cnt[ORC_C_TRANSMITTED]++;
                c->ledger[ORC_L_ETRANS] += q->E;
            }
            escape(c, q);
            return;
        }
        index_of(c, q->r, q->i);
        int m; double rho = voxel_rho(c, q->i, &m);
        double mut = rho * orc_mu(m, q->E, 0);
        if (mut > mx * (1.0 + 1e-12)) c->cnt[ORC_C_VIOL_PHOTON]++;
        if (rnd(&q->rs) * mx >= mut) { c->cnt[ORC_C_FICTITIOUS]++; continue; }
        if (killed_mode) { c->ledger[ORC_L_EKILLED] += q->E; return; }
        double muC = orc_mu(m, q->E, 1), muP = orc_mu(m, q->E, 2), muQ = orc_mu(m, q->E, 3);
        double x = rnd(&q->rs) * (muC + muP + muQ);
        if (x < muC) {
            c->cnt[ORC_C_COMPTON]++;
            double E1, T, d1[3], pe[3];
            compton_event(q->E, q->d, &q->rs, &E1, d1, &T, pe);
            q->d[0] = d1[0]; q->d[1] = d1[1]; q->d[2] = d1[2];
            if (T > 0.0) {
                particle e = make_child(q, 0, ELECTRON, T, pe);
                emit_charged(c, &e);
            }
            q->E = E1;
            if (q->E < p->e_abs_g) { deposit(c, q->i, q->E); return; }
        } else if (x < muC + muP) {
            c->cnt[ORC_C_PHOTO]++;
            deposit(c, q->i, q->E);
            return;
        } else {
            c->cnt[ORC_C_PAIR]++;
            c->ledger[ORC_L_PAIRMASS] += 2.0 * MC2;
            double avail = q->E - 2.0 * MC2, Tm = rnd(&q->rs) * avail, Tp = avail - Tm;
            particle e = make_child(q, 0, ELECTRON, Tm, q->d);
            particle f = make_child(q, 1, POSITRON, Tp, q->d);
            emit_charged(c, &e);
            emit_charged(c, &f);
            return;
        }
    }
}

/* An accepted hard event of a charged particle in material m: Moller with probability
   sM / tot, else bremsstrahlung (Sec. 2.1); secondaries are emitted or absorbed. */
static void hard_event(run_ctx* c, particle* q, int m, double sM, double tot)
{
    const orc_params* p = c->p;
    if (rnd(&q->rs) * tot < sM) {
        c->cnt[ORC_C_MOLLER]++;
        double T1, W, d1[3], d2[3];
        moller_event(q->E, p->w_cc, q->d, &q->rs, &T1, d1, &W, d2);
        particle e = make_child(q, 2, ELECTRON, W, d2);
        q->d[0] = d1[0]; q->d[1] = d1[1]; q->d[2] = d1[2];
        q->E = T1;
        emit_charged(c, &e);
    } else {
        c->cnt[ORC_C_BREMS]++;
        double T0 = q->E, k, dg[3];
        brems_event(m, T0, p->w_cb, q->d, &q->rs, &k, dg);
        particle g = make_child(q, 3, PHOTON, k, dg);
        q->E = T0 - k;
        if (k >= p->e_abs_g) push(c, &g); else deposit(c, q->i, k);
    }
}

static void transport_charged(run_ctx* c, particle* q)
{
    const orc_params* p = c->p;
    enum { LIM_VOX, LIM_MAXS, LIM_MAXE, LIM_EVENT };
    for (;;) {
        int m, face;
        double rho = voxel_rho(c, q->i, &m);
        double sv = dist_to_face(c, q->r, q->d, q->i, &face);
        if (rho <= 0.0 || sv < p->s_min) {
            /* no matter to interact with, or a boundary closer than s_min:
               cross geometrically */
            for (int a = 0; a < 3; ++a) q->r[a] += sv * q->d[a];
            cross_face(c, q, face);
            c->cnt[ORC_C_GEO_CROSS]++;
            if (!inside_index(c, q->i)) { escape(c, q); return; }
            continue;
        }
        double T = q->E, Tlo = T * (1.0 - p->f_maxe);
        double s_maxe = range_between(m, Tlo, T, p) / rho;
        double sig_hat = 0.0;
        if (!(p->flags & ORC_NO_HARD)) {
            for (int j = 0; j <= 16; ++j)
                sig_hat = fmax(sig_hat, orc_sigma_hard(m, Tlo + (T - Tlo) * j / 16.0, p));
            sig_hat *= 1.02;
        }
        double d_ev = sig_hat > 0.0 ? -log(rnd(&q->rs)) / (rho * sig_hat) : INFINITY;
        double s = sv; int lim = LIM_VOX;
        if (p->d_maxs < s) { s = p->d_maxs; lim = LIM_MAXS; }
        if (s_maxe < s)    { s = s_maxe;    lim = LIM_MAXE; }
        if (d_ev < s)      { s = d_ev;      lim = LIM_EVENT; }

        /* random hinge: straight s1 = xi*s, deflect, then the rest, clipped to the voxel */
        double s1 = rnd(&q->rs) * s;
        double H[3] = { q->r[0] + s1 * q->d[0], q->r[1] + s1 * q->d[1], q->r[2] + s1 * q->d[2] };
        double T_full = orc_csda_loss(m, T, rho * s, p);
        if (!(p->flags & ORC_NO_MS)) {
            double G1 = rho * s * orc_lambda1_inv(m, 0.5 * (T + T_full));
            double mu = sample_ms_mu(G1, &q->rs), phi = 2.0 * PI * rnd(&q->rs);
            rotate(q->d, mu, phi);
        }
        int face2;
        double t_exit = dist_to_face(c, H, q->d, q->i, &face2);
        double rem = s - s1, s_tr, T_end;
        int crossed;
        if (rem < t_exit) {
            for (int a = 0; a < 3; ++a) q->r[a] = H[a] + rem * q->d[a];
            s_tr = s; T_end = T_full; crossed = 0;
        } else {
            for (int a = 0; a < 3; ++a) q->r[a] = H[a] + t_exit * q->d[a];
            s_tr = s1 + t_exit; T_end = orc_csda_loss(m, T, rho * s_tr, p); crossed = 1;
        }
        c->cnt[ORC_C_ESTEPS]++;
        c->ledger[ORC_L_EPATH] += s_tr;
        deposit(c, q->i, T - T_end);
        q->E = T_end;
        if (crossed) {
            cross_face(c, q, face2);
            if (!inside_index(c, q->i)) { escape(c, q); return; }
        }
        if (q->E < p->e_abs_e) { absorb_charged(c, q); return; }
        if (lim == LIM_EVENT && !crossed) {
            double sM = p->flags & ORC_NO_HARD ? 0.0 : orc_sigma_moller(m, q->E, p->w_cc);
            double sB = p->flags & ORC_NO_HARD ? 0.0 : orc_sigma_brems(m, q->E, p->w_cb);
            double tot = sM + sB;
            if (tot > sig_hat * (1.0 + 1e-12)) c->cnt[ORC_C_VIOL_ELECTRON]++;
            if (rnd(&q->rs) * sig_hat < tot) {
                hard_event(c, q, m, sM, tot);
                if (q->E < p->e_abs_e) { absorb_charged(c, q); return; }
            } else {
                c->cnt[ORC_C_HARD_FICT]++;
            }
        }
    }
}

/* ---- voxel-crossing (fixed-step) electron transport ------------------------------------
   The stepping scheme the paper contrasts with its own in the Discussion (Sec. 4): an electron
   step is not stopped at voxel faces, so it crosses as many voxels as its length takes it
   through. Reading implemented here (the same on the GPU):
   - step length s = min(d_maxs, d_maxe, d_event): d_maxe is the path in the step's first voxel
     over which the CSDA energy falls by the fraction f_maxe; d_event is sampled by Woodcock
     tracking against the phantom-wide majorant max_m rho_max(m) sigma_hard,m over the step's
     energy interval, so a candidate event may fall in any voxel;
   - random hinge at xi s; the multiple-scattering angle is that of the whole step in the
     medium of its first voxel (the scaling assumption of fixed-step schemes);
   - along both straight parts the energy loss is the CSDA loss in each traversed voxel's own
     material and density, deposited there; if the energy reaches T (1 - f_maxe) before the
     end (denser voxels on the way), the step ends there (before the hinge: deflected there,
     with the angle of the path travelled);
   - at the end of an event-limited step the candidate is real with probability
     rho sigma_hard(E) / majorant in the voxel where it ends. */
enum { SEG_DONE, SEG_FLOOR, SEG_ESCAPED, SEG_ABSORBED };

/* Move q a path length L along its direction through the voxels with CSDA loss deposited in
   each; stops early at the energy floor Tfloor, on absorption or on escape. *done: path moved. */
static int cross_segment(run_ctx* c, particle* q, double L, double Tfloor, double* done)
{
    const orc_params* p = c->p;
    double left = L;
    *done = 0.0;
    while (left > 0.0) {
        int m, face;
        double rho = voxel_rho(c, q->i, &m);
        double sv = dist_to_face(c, q->r, q->d, q->i, &face);
        double l = left, T_end = q->E;
        int cross = 0, floor_hit = 0;
        if (sv < l) { l = sv; cross = 1; }
        if (rho > 0.0) {
            double lf = range_between(m, Tfloor, q->E, p) / rho;
            if (lf <= l) { l = lf; cross = 0; floor_hit = 1; T_end = Tfloor; }
            else T_end = orc_csda_loss(m, q->E, rho * l, p);
        }
        for (int a = 0; a < 3; ++a) q->r[a] += l * q->d[a];
        deposit(c, q->i, q->E - T_end);
        q->E = T_end;
        c->ledger[ORC_L_EPATH] += l;
        left -= l;
        *done += l;
        if (q->E < p->e_abs_e) { absorb_charged(c, q); return SEG_ABSORBED; }
        if (floor_hit) return SEG_FLOOR;
        if (cross) {
            cross_face(c, q, face);
            if (!inside_index(c, q->i)) { escape(c, q); return SEG_ESCAPED; }
        }
    }
    return SEG_DONE;
}

static void transport_charged_cross(run_ctx* c, particle* q)
{
    const orc_params* p = c->p;
    enum { LIM_MAXS, LIM_MAXE, LIM_EVENT };
    for (;;) {
        int m0, face;
        double rho0 = voxel_rho(c, q->i, &m0);
        if (rho0 <= 0.0) {                     /* no matter here: fly to the next voxel */
            double sv = dist_to_face(c, q->r, q->d, q->i, &face);
            for (int a = 0; a < 3; ++a) q->r[a] += sv * q->d[a];
            cross_face(c, q, face);
            c->cnt[ORC_C_GEO_CROSS]++;
            if (!inside_index(c, q->i)) { escape(c, q); return; }
            continue;
        }
        double T = q->E, Tlo = T * (1.0 - p->f_maxe);
        double s_maxe = range_between(m0, Tlo, T, p) / rho0;
        double maj = 0.0;
        if (!(p->flags & ORC_NO_HARD)) {
            for (int m = 0; m < N_MAT; ++m) {
                if (!c->present[m]) continue;
                for (int j = 0; j <= 16; ++j)
                    maj = fmax(maj, c->rho_max[m] * orc_sigma_hard(m, Tlo + (T - Tlo) * j / 16.0, p));
            }
            maj *= 1.02;
        }
        double d_ev = maj > 0.0 ? -log(rnd(&q->rs)) / maj : INFINITY;
        double s = p->d_maxs;
        int lim = LIM_MAXS;
        if (s_maxe < s) { s = s_maxe; lim = LIM_MAXE; }
        if (d_ev < s)   { s = d_ev;   lim = LIM_EVENT; }
        double s1 = rnd(&q->rs) * s, done;
        double T_full = orc_csda_loss(m0, T, rho0 * s, p);
        c->cnt[ORC_C_ESTEPS]++;
        int r = cross_segment(c, q, s1, Tlo, &done);
        if (r == SEG_ESCAPED || r == SEG_ABSORBED) return;
        if (!(p->flags & ORC_NO_MS)) {
            double G1 = rho0 * (r == SEG_FLOOR ? done : s) * orc_lambda1_inv(m0, 0.5 * (T + T_full));
            double mu = sample_ms_mu(G1, &q->rs), phi = 2.0 * PI * rnd(&q->rs);
            rotate(q->d, mu, phi);
        }
        if (r == SEG_FLOOR) continue;
        r = cross_segment(c, q, s - s1, Tlo, &done);
        if (r == SEG_ESCAPED || r == SEG_ABSORBED) return;
        if (r == SEG_FLOOR || lim != LIM_EVENT) continue;
        int m;
        double rho = voxel_rho(c, q->i, &m);
        double sM = rho * orc_sigma_moller(m, q->E, p->w_cc), sB = rho * orc_sigma_brems(m, q->E, p->w_cb);
        double tot = sM + sB;
        if (tot > maj * (1.0 + 1e-12)) c->cnt[ORC_C_VIOL_ELECTRON]++;
        if (rnd(&q->rs) * maj < tot) {
            hard_event(c, q, m, sM, tot);
            if (q->E < p->e_abs_e) { absorb_charged(c, q); return; }
        } else {
            c->cnt[ORC_C_HARD_FICT]++;
        }
    }
}

/* ---- source --------------------------------------------------------------- */
int orc_stratify(int n_bins, const float* edges, const float* weights,
                 uint64_t n_total, uint64_t* bounds, int32_t* order)
{
    /* bins processed in order of decreasing lower edge (ties: lower index first) */
    for (int i = 0; i < n_bins; ++i) order[i] = i;
    for (int i = 1; i < n_bins; ++i) {
        int32_t v = order[i]; int j = i - 1;
        while (j >= 0 && (edges[order[j]] < edges[v] || (edges[order[j]] == edges[v] && order[j] > v))) {
            order[j + 1] = order[j]; --j;
        }
        order[j + 1] = v;
    }
    double W = 0.0;
    for (int q = 0; q < n_bins; ++q) W += (double)weights[order[q]];
    if (!(W > 0.0)) return -1;
    double cum = 0.0;
    bounds[0] = 0;
    for (int q = 1; q < n_bins; ++q) {
        cum += (double)weights[order[q - 1]];
        double b = floor((double)n_total * cum / W);
        bounds[q] = (uint64_t)b;
        if (bounds[q] > n_total) bounds[q] = n_total;
        if (bounds[q] < bounds[q - 1]) bounds[q] = bounds[q - 1];
    }
    bounds[n_bins] = n_total;
    return 0;
}

typedef struct { double e1[3], e2[3], u[3]; } frame;

static void beam_frame(const orc_source* s, frame* f)
{
    double d[3] = { s->dir[0], s->dir[1], s->dir[2] };
    normalize3(d);
    double a[3] = { d[2], 0.0, -d[0] };                  /* y x d */
    if (sqrt(a[0] * a[0] + a[2] * a[2]) < 1e-6) { a[0] = 0.0; a[1] = -d[2]; a[2] = d[1]; }  /* x x d */
    normalize3(a);
    f->e1[0] = a[0]; f->e1[1] = a[1]; f->e1[2] = a[2];
    f->e2[0] = d[1] * a[2] - d[2] * a[1];
    f->e2[1] = d[2] * a[0] - d[0] * a[2];
    f->e2[2] = d[0] * a[1] - d[1] * a[0];
    f->u[0] = d[0]; f->u[1] = d[1]; f->u[2] = d[2];
}

/* Source particle for history h. Returns 1 if it enters the phantom. */
static int make_primary(const run_ctx* c, const orc_source* src, const frame* f,
                        const uint64_t* bounds, const int32_t* order, uint64_t seed,
                        uint64_t h, particle* q)
{
    memset(q, 0, sizeof(*q));
    q->rs.key[0] = (uint32_t)seed; q->rs.key[1] = (uint32_t)(seed >> 32);
    q->rs.hist = h; q->rs.sub = 0; q->rs.n = 0;
    q->type = src->particle == 0 ? PHOTON : ELECTRON;
    int qb = 0;
    while (qb + 1 < src->n_bins && h >= bounds[qb + 1]) ++qb;
    int bin = order[qb];
    double lo = src->edges[bin], hi = src->edges[bin + 1];
    q->E = lo + rnd(&q->rs) * (hi - lo);
    double a = rnd(&q->rs) - 0.5, b = rnd(&q->rs) - 0.5, P[3], O[3], d[3];
    for (int k = 0; k < 3; ++k) P[k] = src->iso[k] + a * src->field_x * f->e1[k] + b * src->field_y * f->e2[k];
    double tmin;
    if (src->ssd > 0.0) {
        for (int k = 0; k < 3; ++k) { O[k] = src->iso[k] - src->ssd * f->u[k]; d[k] = P[k] - O[k]; }
        normalize3(d);
        tmin = 0.0;
    } else {
        for (int k = 0; k < 3; ++k) { O[k] = P[k]; d[k] = f->u[k]; }
        tmin = -INFINITY;
    }
    double tmax = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (fabs(d[k]) < 1e-300) {
            if (O[k] < 0.0 || O[k] > c->L[k]) return 0;
            continue;
        }
        double t1 = (0.0 - O[k]) / d[k], t2 = (c->L[k] - O[k]) / d[k];
        tmin = fmax(tmin, fmin(t1, t2));
        tmax = fmin(tmax, fmax(t1, t2));
    }
    if (!(tmax > tmin)) return 0;
    for (int k = 0; k < 3; ++k) { q->r[k] = O[k] + tmin * d[k]; q->d[k] = d[k]; }
    index_of(c, q->r, q->i);
    return 1;
}

static int setup_ctx(run_ctx* c, const orc_phantom* ph, const orc_params* p)
{
    c->ph = ph; c->p = p;
    c->nn[0] = ph->nx; c->nn[1] = ph->ny; c->nn[2] = ph->nz;
    c->dd[0] = ph->dx; c->dd[1] = ph->dy; c->dd[2] = ph->dz;
    for (int a = 0; a < 3; ++a) c->L[a] = c->nn[a] * c->dd[a];
    c->nvox = (int64_t)ph->nx * ph->ny * ph->nz;
    for (int m = 0; m < ORC_MAX_MAT; ++m) { c->rho_max[m] = 0.0; c->present[m] = 0; }
    for (int64_t v = 0; v < c->nvox; ++v) {
        int m = ph->material[v];
        if (m >= N_MAT) return -1;
        double r = ph->density[v];
        if (!(r >= 0.0)) return -1;
        c->present[m] = 1;
        if (r > c->rho_max[m]) c->rho_max[m] = r;
    }
    c->top = 0;
    return 0;
}

int orc_source_sample(const orc_phantom* ph, const orc_source* src, uint64_t seed,
                      uint64_t n_total, uint64_t first, uint64_t count, double* out)
{
    static const orc_params dummy = { 0.2, 0.01, 0.2, 0.01, 0.5, 0.05, 1e-4, 1, 0 };
    run_ctx* c = (run_ctx*)calloc(1, sizeof(run_ctx));
    if (!c || setup_ctx(c, ph, &dummy) != 0 || src->n_bins < 1 || src->n_bins > 4096) { free(c); return -1; }
    uint64_t* bounds = (uint64_t*)malloc(sizeof(uint64_t) * (src->n_bins + 1));
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * src->n_bins);
    if (orc_stratify(src->n_bins, src->edges, src->weights, n_total, bounds, order) != 0) {
        free(bounds); free(order); free(c); return -1;
    }
    frame f; beam_frame(src, &f);
    for (uint64_t j = 0; j < count; ++j) {
        particle q;
        int hit = make_primary(c, src, &f, bounds, order, seed, first + j, &q);
        double* o = out + 8 * j;
        o[0] = q.r[0]; o[1] = q.r[1]; o[2] = q.r[2];
        o[3] = q.d[0]; o[4] = q.d[1]; o[5] = q.d[2];
        o[6] = q.E; o[7] = hit;
    }
    free(bounds); free(order); free(c);
    return 0;
}

int orc_run(const orc_phantom* ph, const orc_source* src, const orc_params* p,
            uint64_t seed, uint64_t n_total, uint64_t first, uint64_t count,
            int64_t* tally, double* ledger, uint64_t* counters)
{
    if (p->n_batches < 1 || src->n_bins < 1 || src->n_bins > 4096) return -1;
    run_ctx* c = (run_ctx*)calloc(1, sizeof(run_ctx));
    if (!c) return -2;
    if (setup_ctx(c, ph, p) != 0) { free(c); return -1; }
    c->tally = tally; c->ledger = ledger; c->cnt = counters;
    uint64_t* bounds = (uint64_t*)malloc(sizeof(uint64_t) * (src->n_bins + 1));
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * src->n_bins);
    if (orc_stratify(src->n_bins, src->edges, src->weights, n_total, bounds, order) != 0) {
        free(bounds); free(order); free(c); return -1;
    }
    frame f; beam_frame(src, &f);
    for (uint64_t j = 0; j < count; ++j) {
        uint64_t h = first + j;
        c->hist = h;
        particle q;
        if (!make_primary(c, src, &f, bounds, order, seed, h, &q)) {
            c->ledger[ORC_L_EMISS] += q.E;
            c->cnt[ORC_C_MISSED]++;
            continue;
        }
        c->ledger[ORC_L_EIN] += q.E;
        if (q.type == PHOTON) {
            if (q.E >= p->e_abs_g) push(c, &q); else deposit(c, q.i, q.E);
        } else {
            emit_charged(c, &q);
        }
        while (c->top > 0) {
            particle r = c->stack[--c->top];
            if (r.type == PHOTON) transport_photon(c, &r);
            else if (p->flags & ORC_CROSS_VOXELS) transport_charged_cross(c, &r);
            else transport_charged(c, &r);
        }
    }
    free(bounds); free(order); free(c);
    return 0;
}

/* Phase-space primary of history h: record h mod n_ps, moved along its direction through
 * vacuum to the phantom box (t >= 0, so a particle inside starts where it is). Returns 1 if
 * it enters. No random numbers are drawn here. */
static int make_primary_ps(const run_ctx* c, const orc_ps_particle* ps, uint64_t n_ps, uint64_t seed,
                           uint64_t h, particle* q)
{
    const orc_ps_particle* rec = ps + (h % n_ps);
    memset(q, 0, sizeof(*q));
    q->rs.key[0] = (uint32_t)seed; q->rs.key[1] = (uint32_t)(seed >> 32);
    q->rs.hist = h; q->rs.sub = 0; q->rs.n = 0;
    q->type = rec->type == 0 ? PHOTON : (rec->type == 1 ? ELECTRON : POSITRON);
    q->E = rec->E;
    double O[3] = { rec->x, rec->y, rec->z }, d[3] = { rec->u, rec->v, rec->w };
    normalize3(d);
    double tmin = 0.0, tmax = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (fabs(d[k]) < 1e-300) {
            if (O[k] < 0.0 || O[k] > c->L[k]) return 0;
            continue;
        }
        double t1 = (0.0 - O[k]) / d[k], t2 = (c->L[k] - O[k]) / d[k];
        tmin = fmax(tmin, fmin(t1, t2));
        tmax = fmin(tmax, fmax(t1, t2));
    }
    if (!(tmax > tmin)) return 0;
    for (int k = 0; k < 3; ++k) { q->r[k] = O[k] + tmin * d[k]; q->d[k] = d[k]; }
    index_of(c, q->r, q->i);
    return 1;
}

static int ps_valid(const orc_ps_particle* ps, uint64_t n_ps)
{
    if (n_ps == 0) return 0;
    for (uint64_t i = 0; i < n_ps; ++i) {
        const orc_ps_particle* r = ps + i;
        double n2 = (double)r->u * r->u + (double)r->v * r->v + (double)r->w * r->w;
        if (r->type < 0 || r->type > 2 || !(r->E > 0.0) || !(n2 > 0.0) || !isfinite(r->E) ||
            !isfinite(r->x) || !isfinite(r->y) || !isfinite(r->z))
            return 0;
    }
    return 1;
}

int orc_ps_sample(const orc_phantom* ph, const orc_ps_particle* ps, uint64_t n_ps,
                  uint64_t first, uint64_t count, double* out)
{
    static const orc_params dummy = { 0.2, 0.01, 0.2, 0.01, 0.5, 0.05, 1e-4, 1, 0 };
    if (!ps_valid(ps, n_ps)) return -1;
    run_ctx* c = (run_ctx*)calloc(1, sizeof(run_ctx));
    if (!c || setup_ctx(c, ph, &dummy) != 0) { free(c); return -1; }
    for (uint64_t j = 0; j < count; ++j) {
        particle q;
        int hit = make_primary_ps(c, ps, n_ps, 0, first + j, &q);
        double* o = out + 8 * j;
        o[0] = q.r[0]; o[1] = q.r[1]; o[2] = q.r[2];
        o[3] = q.d[0]; o[4] = q.d[1]; o[5] = q.d[2];
        o[6] = q.E; o[7] = hit;
    }
    free(c);
    return 0;
}

int orc_run_ps(const orc_phantom* ph, const orc_ps_particle* ps, uint64_t n_ps,
               const orc_params* p, uint64_t seed, uint64_t first, uint64_t count,
               int64_t* tally, double* ledger, uint64_t* counters)
{
    if (p->n_batches < 1 || !ps_valid(ps, n_ps)) return -1;
    run_ctx* c = (run_ctx*)calloc(1, sizeof(run_ctx));
    if (!c) return -2;
    if (setup_ctx(c, ph, p) != 0) { free(c); return -1; }
    c->tally = tally; c->ledger = ledger; c->cnt = counters;
    for (uint64_t j = 0; j < count; ++j) {
        uint64_t h = first + j;
        c->hist = h;
        particle q;
        if (!make_primary_ps(c, ps, n_ps, seed, h, &q)) {
            c->ledger[ORC_L_EMISS] += q.E;
            c->cnt[ORC_C_MISSED]++;
            continue;
        }
        c->ledger[ORC_L_EIN] += q.E;
        if (q.type == PHOTON) {
            if (q.E >= p->e_abs_g) push(c, &q); else deposit(c, q.i, q.E);
        } else {
            emit_charged(c, &q);
        }
        while (c->top > 0) {
            particle r = c->stack[--c->top];
            if (r.type == PHOTON) transport_photon(c, &r);
            else if (p->flags & ORC_CROSS_VOXELS) transport_charged_cross(c, &r);
            else transport_charged(c, &r);
        }
    }
    free(c);
    return 0;
}

/* ---- sampler access for distribution tests ------------------------------ */
int orc_sample(int kind, int m, double E, double aux, uint64_t n, uint64_t seed,
               const orc_params* p, double* out)
{
    for (uint64_t j = 0; j < n; ++j) {
        stream s = { { (uint32_t)seed, (uint32_t)(seed >> 32) }, j, 0x5A5Au + (uint32_t)kind, 0 };
        switch (kind) {
        case 0: out[j] = sample_kn_mu(E, &s); break;
        case 1: out[j] = sample_moller_eps(E, p->w_cc, &s); break;
        case 2: out[j] = sample_brems_k(m, E, p->w_cb, &s); break;
        case 3: out[j] = sample_ms_mu(aux, &s); break;
        default: return -1;
        }
    }
    return 0;
}

/* ---- event kinematics access for conservation and angle tests ------------- */
/* n events of one kind from the incoming unit direction d0 (normalised here), each on its own
   random stream. out holds 8 doubles per event: energy and unit direction of the first and of
   the second outgoing particle --
     kind 0 Compton:      scattered photon (E1, d1), recoil electron (T, de);  E = photon energy
     kind 1 Moller:       primary electron (T1, d1), knock-on electron (W, d2); E = kinetic energy
     kind 2 brems:        electron (E - k, unchanged direction), photon (k, dg); E = kinetic energy
     kind 3 annihilation: two photons (mc^2, d1), (mc^2, d2)
     kind 4 rotation:     (aux, d0 rotated by polar cosine aux), (azimuth, d0) */
int orc_event(int kind, int m, double E, double aux, const double* d_in, uint64_t n, uint64_t seed,
              const orc_params* p, double* out)
{
    double d0[3] = { d_in[0], d_in[1], d_in[2] };
    double nn = sqrt(d0[0] * d0[0] + d0[1] * d0[1] + d0[2] * d0[2]);
    if (!(nn > 0.0) || kind < 0 || kind > 4) return -1;
    d0[0] /= nn; d0[1] /= nn; d0[2] /= nn;
    for (uint64_t j = 0; j < n; ++j) {
        stream s = { { (uint32_t)seed, (uint32_t)(seed >> 32) }, j, 0xE7E7u + (uint32_t)kind, 0 };
        double* o = out + 8 * j;
        double a = 0.0, b = 0.0, da[3] = { d0[0], d0[1], d0[2] }, db[3] = { d0[0], d0[1], d0[2] };
        switch (kind) {
        case 0: compton_event(E, d0, &s, &a, da, &b, db); break;
        case 1: moller_event(E, p->w_cc, d0, &s, &a, da, &b, db); break;
        case 2: brems_event(m, E, p->w_cb, d0, &s, &b, db); a = E - b; break;
        case 3: annihilation_event(&s, da, db); a = b = MC2; break;
        case 4: b = 2.0 * PI * rnd(&s); a = aux; rotate(da, aux, b); break;
        }
        o[0] = a; o[1] = da[0]; o[2] = da[1]; o[3] = da[2];
        o[4] = b; o[5] = db[0]; o[6] = db[1]; o[7] = db[2];
    }
    return 0;
}

/* The rotation itself, for direction-by-direction comparisons: d (normalised here) turned by
   polar cosine mu and azimuth phi. */
void orc_rotate(const double* d, double mu, double phi, double* out)
{
    double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    out[0] = d[0] / nn; out[1] = d[1] / nn; out[2] = d[2] / nn;
    rotate(out, mu, phi);
}
