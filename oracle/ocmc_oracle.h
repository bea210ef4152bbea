/*
 * ocmc_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, double-precision CPU oracle for coupled photon-electron Monte
 * Carlo dose calculation in a voxel phantom (Tian et al., "oclMC", Sec. 2.1).
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it. It shares no source with the CUDA engine and neither side
 * includes the other.
 *
 * Parity of every function here is pinned by tests/test_oracle_*.py against
 * closed forms, numerical quadrature of the differential cross sections,
 * published reference values and a third-party Philox implementation.
 */
#ifndef OCMC_ORACLE_H
#define OCMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* run flags (test modes) */
#define ORC_NO_HARD          1  /* no discrete Moller / bremsstrahlung events      */
#define ORC_NO_MS            2  /* no multiple-scattering deflection               */
#define ORC_KILL_FIRST_REAL  4  /* photons removed at their first real interaction */
#define ORC_KERMA            8  /* e-/e+ deposit their kinetic energy at creation  */
#define ORC_CROSS_VOXELS    16  /* electron steps cross voxel faces (fixed-step variant, Sec. 4) */

typedef struct {
    double e_abs_e;   /* MeV, electron/positron absorption energy              */
    double e_abs_g;   /* MeV, photon absorption energy                         */
    double w_cc;      /* MeV, Moller hard-collision threshold                  */
    double w_cb;      /* MeV, bremsstrahlung hard-emission threshold           */
    double d_maxs;    /* cm, maximum electron step                             */
    double f_maxe;    /* maximum fractional CSDA energy loss per step          */
    double s_min;     /* cm, a boundary closer than this is crossed geometrically */
    int32_t n_batches;/* statistical batches, batch = history id mod n_batches */
    int32_t flags;    /* ORC_* test modes                                      */
} orc_params;

/* Materials (Sec. 2.1: the per-voxel material type selects the cross-section data; the
 * paper's database has 16 materials). By default 0 water, 1 ICRP cortical bone, 2 ICRP lung;
 * orc_set_materials replaces them with up to ORC_MAX_MAT compositions: elements (Z, atomic
 * mass A in g/mol, mass fraction, normalised over the elements), mean excitation energy and the
 * nominal density that fixes the density-effect parameters. Process-wide; set before runs. */
#define ORC_MAX_MAT  16
#define ORC_MAX_ELEM 16
typedef struct {
    int32_t n_elements;
    int32_t Z[ORC_MAX_ELEM];
    double A[ORC_MAX_ELEM];
    double mass_fraction[ORC_MAX_ELEM];
    double I_eV;
    double density;
} orc_material;

int  orc_set_materials(int n, const orc_material* defs);   /* 0, or -1 on a bad definition */
void orc_reset_materials(void);
int  orc_n_materials(void);

typedef struct {
    int32_t nx, ny, nz;      /* voxels, x fastest                       */
    double dx, dy, dz;       /* cm                                      */
    const float* density;    /* g/cm^3, nx*ny*nz                        */
    const uint8_t* material; /* index into the materials (default 0 water, 1 bone, 2 lung) */
} orc_phantom;

typedef struct {
    int32_t particle;        /* 0 photon, 1 electron                    */
    int32_t n_bins;
    const float* edges;      /* n_bins+1, MeV                           */
    const float* weights;    /* n_bins                                  */
    double field_x, field_y; /* cm, in the plane through iso normal to dir */
    double ssd;              /* cm, >0 point source at iso - ssd*dir, else parallel */
    double iso[3], dir[3];
} orc_source;

/* One source particle of a phase-space source (Sec. 2.2 "Materials": source particles may be
 * loaded from a phase-space file or made by a user's own source model). Position in the
 * phantom frame (cm, origin at the outer corner of voxel (0,0,0)), direction (any length > 0),
 * kinetic energy (MeV), type 0 photon, 1 electron, 2 positron. */
typedef struct {
    float x, y, z, u, v, w, E;
    int32_t type;
} orc_ps_particle;

/* counters[] layout (uint64) */
enum {
    ORC_C_FLIGHTS = 0, ORC_C_FICTITIOUS, ORC_C_COMPTON, ORC_C_PHOTO, ORC_C_PAIR,
    ORC_C_ESTEPS, ORC_C_MOLLER, ORC_C_BREMS, ORC_C_HARD_FICT, ORC_C_ESCAPED,
    ORC_C_VIOL_PHOTON, ORC_C_VIOL_ELECTRON, ORC_C_STACK_OVERFLOW,
    ORC_C_TRANSMITTED, ORC_C_GEO_CROSS, ORC_C_ANNIH, ORC_C_MISSED,
    ORC_N_COUNTERS = 24
};
/* ledger[] layout (double, MeV) */
enum {
    ORC_L_EIN = 0,   /* kinetic energy of source particles entering the phantom */
    ORC_L_EDEP,      /* deposited energy, exact fp64 sum                        */
    ORC_L_EESC,      /* kinetic energy leaving the phantom                      */
    ORC_L_EMISS,     /* source energy that missed the phantom                   */
    ORC_L_PAIRMASS,  /* 2 mc^2 per pair production                              */
    ORC_L_ANNIHMASS, /* 2 mc^2 per positron annihilation                        */
    ORC_L_EKILLED,   /* energy removed by ORC_KILL_FIRST_REAL                   */
    ORC_L_EPATH,     /* summed electron path length (cm)                        */
    ORC_L_ETRANS,    /* energy of photons leaving through z=Lz unscattered      */
    ORC_N_LEDGER = 12
};

void   orc_init(void);
/* mass coefficients (cm^2/g) and stopping powers (MeV cm^2/g) at unit density */
double orc_mu(int m, double E, int channel); /* 0 total 1 Compton 2 photo 3 pair */
double orc_sigma_kn(double E);               /* cm^2 per electron */
double orc_L_col(int m, double T, double w_cc);
double orc_L_rad(int m, double T, double w_cb);
double orc_sigma_moller(int m, double T, double w_cc);
double orc_sigma_brems(int m, double T, double w_cb);
double orc_lambda1_inv(int m, double T);
double orc_density_effect(int m, double T);
double orc_material_const(int m, int which);  /* 0 n_e 1 photo 2 pairZ 3 S1 4 S2 5 I 6 rho0 */
double orc_ms_mean_u(double A);
double orc_ms_solve_A(double G1);
double orc_csda_loss(int m, double T, double mass_thickness, const orc_params* p);

void   orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int    orc_sample(int kind, int m, double E, double aux, uint64_t n, uint64_t seed,
                  const orc_params* p, double* out);
/* One interaction's outgoing energies and directions (tests of the kinematics; layout in the
   source file): kind 0 Compton, 1 Moller, 2 bremsstrahlung, 3 annihilation, 4 rotation. */
int    orc_event(int kind, int m, double E, double aux, const double* d0, uint64_t n, uint64_t seed,
                 const orc_params* p, double* out);
void   orc_rotate(const double* d, double mu, double phi, double* out);
int    orc_stratify(int n_bins, const float* edges, const float* weights,
                    uint64_t n_total, uint64_t* bounds, int32_t* order);
int    orc_source_sample(const orc_phantom* ph, const orc_source* src, uint64_t seed,
                         uint64_t n_total, uint64_t first, uint64_t count, double* out);
int    orc_run(const orc_phantom* ph, const orc_source* src, const orc_params* p,
               uint64_t seed, uint64_t n_total, uint64_t first, uint64_t count,
               int64_t* tally, double* ledger, uint64_t* counters);
/* Phase-space source: history h starts from record h mod n_ps, moved forward in vacuum to
 * the phantom (or starting where it is when inside); it draws no random numbers before its
 * first transport step. */
int    orc_ps_sample(const orc_phantom* ph, const orc_ps_particle* ps, uint64_t n_ps,
                     uint64_t first, uint64_t count, double* out);
int    orc_run_ps(const orc_phantom* ph, const orc_ps_particle* ps, uint64_t n_ps,
                  const orc_params* p, uint64_t seed, uint64_t first, uint64_t count,
                  int64_t* tally, double* ledger, uint64_t* counters);

#ifdef __cplusplus
}
#endif
#endif
