// ocmc_internal.h -- definitions shared by the engine's translation units.
//
// Physics tables: per material (0 water, 1 cortical bone, 2 lung), NE nodes
// uniform in ln E on [E_LO, E_HI], quantities per unit density (g/cm^3):
//   ph[m][i]  = { ln mu_total, mu_C / mu_total, mu_pe / mu_total, mu_total }   (cm^2/g)
//   el[m][i]  = { ln R, 1/lambda_1, sigma_Moller, sigma_brems }                (R in g/cm^2)
//   el2[m][i] = { R(E_i) - R(E_i (1 - f_maxe)), hard-event majorant on [E_i, E_i+1) }
//   rinv[m][j] = ln E at ln R = lnR0[m] + j dlnR[m], j < NR
//   msA[j]     = ln A (Wentzel screening) at ln G1 = ln G1_LO + j dlnG
//   phmaj[i]   = ln mu_max(E_i): photon Woodcock majorant over the phantom (1/cm)
//   msc[m]     = { S1, S2 }: bremsstrahlung spectrum constants (per gram)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ocmc {

constexpr int NE = 512;
constexpr int NR = 512;
constexpr int NG = 512;
constexpr int NMAT_DEFAULT = 3;   // built-in materials: water, ICRP cortical bone, ICRP lung
constexpr int MAX_MAT = 16;       // user-defined materials (the paper's database has 16)
constexpr int MAX_STAGED = 10;    // materials whose tables one transport block holds in shared memory
constexpr int MAX_ELEM = 16;      // elements per material
constexpr int MAX_BINS = 256;
constexpr double E_LO = 1.0e-3;   // MeV
constexpr double E_HI = 32.0;     // MeV
constexpr double G1_LO = 1.0e-12; // below: no deflection
constexpr double G1_ISO = 15.0;   // at and above: isotropic deflection
constexpr double MC2 = 0.51099895000;
constexpr float TALLY_SCALE = 268435456.0f;   // 2^28 fixed-point units per MeV
constexpr int MAX_DIM = 1024;
constexpr unsigned long long RUN_CHUNK = 100000000ull;   // histories per transport launch of a run

// transport flags (ocmc_params.flags)
constexpr int FLAG_CROSS_VOXELS = 16;   // electron steps cross voxel faces (fixed-step variant)

// error bits written by kernels
constexpr int ERR_OVERFLOW = 1;
constexpr int ERR_LIMIT = 2;
constexpr int ERR_PHANTOM = 4;
constexpr int ERR_BOUNDS = 8;     // a bounds check of the checks build failed (the access was skipped)

// Checks build (-DOCMC_CHECKS=1): voxel indices, tally addresses and stack slots are checked
// before use; a failure sets ERR_BOUNDS and the access is skipped. Off in the normal build.
#ifndef OCMC_CHECKS
#define OCMC_CHECKS 0
#endif

// run statistics slots (uint64, device)
enum Stat {
    ST_FICT = 0, ST_COMPTON, ST_PHOTO, ST_PAIR, ST_MOLLER, ST_BREMS, ST_HARD_FICT,
    ST_ANNIH, ST_ESCAPED, ST_MISSED, ST_GEO, ST_VIOL, ST_DROPPED, ST_TRANSMITTED,
    ST_WARP_ITERS, ST_LANES_PHOTON, ST_LANES_CHARGED, ST_HISTORIES,
    // fixed-point energies (2^28 units per MeV)
    ST_E_IN, ST_E_ESC, ST_E_MISS, ST_E_KILLED, ST_E_TRANS, ST_E_DROPPED,
    // transport-kernel timing from %globaltimer (ns): summed warp lifetimes, summed warp time
    // after the warp saw the source exhausted, and (max-reduced, written directly) the bitwise
    // complement of the earliest warp start and of the earliest source exhaustion, and the
    // latest warp end
    ST_WARP_NS, ST_TAIL_NS, ST_T_START_INV, ST_T_SRC_INV, ST_T_END, ST_WARPS,
    ST_COUNT
};

// Tables in global memory, one row per staged material m < n_mat (capacity MAX_STAGED).
struct MatDef;
struct Tables {
    int n_mat;      // staged materials (table rows)
    MatDef* mats;   // their definitions (device, MAX_STAGED)
    float4* ph;     // n_mat*NE
    float* phmaj;   // NE
    float* elmaj;   // NE: phantom-wide majorant of rho * sigma_hard over a step (voxel-crossing steps)
    float4* el;     // n_mat*NE
    float2* el2;    // n_mat*NE
    float* rinv;    // n_mat*NR
    float* msA;     // NG
    float* rmeta;   // n_mat*2: lnR0, 1/dlnR
    float* msc;     // n_mat*2: bremsstrahlung screening sums S1, S2 (per gram)
    double* scratch;        // n_mat*NE interval ranges
    unsigned int* rho_max;  // n_mat, float bits of the max density per material
};

// Per-material composition for the table builder: elements (Z, atomic mass A in g/mol, mass
// fraction), mean excitation energy, nominal density.
struct MatDef {
    int n;
    int Z[MAX_ELEM];
    double A[MAX_ELEM];
    double w[MAX_ELEM];
    double I_eV;
    double rho0;
};

// Shared-memory image of the tables in a transport block: the material-independent photon
// majorant (NE floats) and Wentzel screening table (NG floats), then one block per staged
// material, SM_MAT_BYTES apart: ph (NE float4), el (NE float4), el2 (NE float2), rinv (NR
// floats), rmeta[2], msc[2]. A material's row is at a compile-time stride, so table addressing
// costs the same for any number of materials.
constexpr size_t SM_SHARED_BYTES = (size_t)(NE + NG) * sizeof(float);
constexpr size_t SM_MAT_BYTES = (size_t)NE * (2 * sizeof(float4) + sizeof(float2)) + (size_t)NR * sizeof(float) +
                                4 * sizeof(float);
static_assert(SM_SHARED_BYTES % 16 == 0 && SM_MAT_BYTES % 16 == 0, "16-byte aligned table rows");
constexpr int MS4 = (int)(SM_MAT_BYTES / 16);   // material stride in float4
constexpr int MS2 = (int)(SM_MAT_BYTES / 8);    // in float2
constexpr int MS1 = (int)(SM_MAT_BYTES / 4);    // in float
__host__ __device__ constexpr size_t smem_table_bytes(int n_mat) { return SM_SHARED_BYTES + n_mat * SM_MAT_BYTES; }

struct PhysParams {
    float e_abs_e, e_abs_g, w_cc, w_cb, d_maxs, f_maxe, s_min;
    int flags;
    int n_batches;
};

// 48-byte particle record of the secondary stacks.
struct __align__(16) PRec {
    float x, y, z, E;
    float u, v, w;
    uint32_t vt;     // ix | iy << 10 | iz << 20 | type << 30
    uint32_t h0, h1, sub, n;
};

struct SourceDev {
    int particle;            // 0 photon, 1 electron
    int n_bins;
    float fx, fy, ssd;
    float iso[3], e1[3], e2[3], dir[3];
    unsigned long long bound[MAX_BINS + 1];   // stratification bounds (history ids)
    int order[MAX_BINS];                      // bin processed at position q
    float lo[MAX_BINS], hi[MAX_BINS];         // bin edges
};

// Batched beamlets: each beamlet is an independent beam with its own histories,
// random streams (history counter high word = 0x80000000 | beamlet) and sparse
// tally (open-addressing hash: uint32 voxel key, int64 value).
constexpr int MAX_BL_BINS = 32;
constexpr unsigned int BL_EMPTY = 0xFFFFFFFFu;
constexpr unsigned int BL_TAG = 0x80000000u;

struct BeamletDev {
    float fx, fy, ssd, pad0;
    float iso[3], e1[3], e2[3], dir[3];
    unsigned long long table_off;              // first slot of this beamlet's table
    unsigned int cap_mask;                     // table capacity - 1 (power of two)
    unsigned int pad1;
    unsigned long long n;                      // histories
    unsigned long long bound[MAX_BL_BINS + 1]; // energy-bin stratification of its histories
};

// Phase-space source record (Sec. 2.2 "Materials": particles from a phase-space file or a
// user's source model); the same 32-byte layout as ocmc_ps_particle of the C ABI.
struct PsRec {
    float x, y, z, u, v, w, E;
    int type;                            // 0 photon, 1 electron, 2 positron
};

struct TransportArgs {
    // geometry
    int nx, ny, nz;
    float dx, dy, dz;
    const float* density;
    const uint8_t* material;
    long long nvox;
    // tables
    Tables t;
    PhysParams pp;
    // run
    unsigned long long first, count, n_total;
    uint32_t key0, key1;
    unsigned long long* tally;
    // scratch
    PRec* stacks;               // per warp: nstk stacks of `cap` records
    int cap;
    int nstk;                   // 2 (photons, charged) or 3 (photons, charged >= e_split, charged < e_split)
    float e_split;              // MeV; energy-class boundary of the charged stacks when nstk == 3
    int switch_high, switch_low;
    int refill_min;                      // free lanes needed before a warp refills (>= 1)
    unsigned long long* hist_counter;
    unsigned long long* stats;  // ST_COUNT
    int* err;
    SourceDev src;
    uint32_t stream_tag;                 // XORed into the high history word (single-beam mode)
    const PsRec* ps;                     // phase-space source (null: the analytic source src)
    unsigned long long ps_n;             // its records; history h starts from record h mod ps_n
    // batched beamlets (beamlets == nullptr: single-beam mode with the dense tally)
    const BeamletDev* beamlets;
    const unsigned long long* bl_prefix; // n_beamlets + 1 prefix sums of histories
    int n_beamlets;
    unsigned int* bl_keys;
    unsigned long long* bl_vals;
    unsigned int* bl_overflow;           // per-beamlet table-full flags
};

// kernels / launchers (defined in the .cu files)
cudaError_t build_tables(const Tables& t, const PhysParams& pp, const float* density, const uint8_t* material,
                         long long nvox, int* d_err, const MatDef* defs, cudaStream_t s);
cudaError_t build_material_tables(const Tables& t, const PhysParams& pp, const MatDef* defs, cudaStream_t s);
cudaError_t build_phantom_tables(const Tables& t, const float* density, const uint8_t* material, long long nvox,
                                 int* d_err, cudaStream_t s);
cudaError_t launch_transport(const TransportArgs& a, int blocks, int threads, size_t smem, cudaStream_t s,
                             int nreg);
size_t transport_smem_bytes(int n_mat);
int transport_max_blocks_per_sm(int threads, size_t smem, int nreg);
bool transport_nreg_supported(int nreg);
cudaError_t launch_finalize(const long long* tally, const float* density, int B, long long nvox, double voxel_volume,
                            const float* w_nb, double inv_n, float* dose, float* sigma, cudaStream_t s);
// (w_nb[b] = N / n_b: the whole run's histories over batch b's, 0 for an empty batch)
cudaError_t launch_test_philox(uint32_t key0, uint32_t key1, uint32_t c1, uint32_t c2, uint32_t c3,
                               uint32_t first_block, uint32_t n_blocks, uint32_t* out, cudaStream_t s);
cudaError_t launch_test_rotate(const float* dir, const float* mu, const float* xi, int n, float* out, cudaStream_t s);
cudaError_t launch_test_source(const TransportArgs& a, unsigned long long n_total, unsigned long long first,
                               unsigned long long count, float* out, cudaStream_t s);
cudaError_t launch_test_sample(const TransportArgs& a, int kind, int m, float E, float aux, unsigned long long n,
                               float* out, cudaStream_t s);
cudaError_t launch_test_tables(const TransportArgs& a, int m, const float* E, int n, float* out, cudaStream_t s);
cudaError_t launch_test_csda(const TransportArgs& a, int m, const float* T, const float* X, int n, float* out,
                             cudaStream_t s);
void material_defs(MatDef out[NMAT_DEFAULT]);
cudaError_t launch_ps_validate(const PsRec* ps, unsigned long long n, unsigned long long* bad, cudaStream_t s);
cudaError_t launch_bl_count(const unsigned int* keys, const unsigned long long* offs, const unsigned int* caps, int n,
                            unsigned long long* nnz, cudaStream_t s);
cudaError_t launch_bl_extract(const unsigned int* keys, const unsigned long long* vals, unsigned long long cap,
                              long long nvox, long long* dense, unsigned int* block_counts, int* idx_out,
                              long long* raw_out, float* dose_out, const float* density, double scale,
                              unsigned long long* nnz_out, cudaStream_t s);

}  // namespace ocmc
