/*
 * ocmc.h -- C ABI of the GB300 coupled photon-electron Monte Carlo dose engine.
 *
 * The engine computes the method of Tian et al., "An OpenCL-based Monte Carlo
 * dose calculation engine (oclMC) for coupled photon-electron transport":
 * analogue photon transport with Woodcock tracking (Compton, photoelectric,
 * pair production) and Class II condensed-history electron/positron transport
 * (continuous restricted energy loss, random-hinge multiple scattering,
 * discrete Moller and bremsstrahlung events) through a voxel phantom, with
 * the deposited energy tallied per voxel (Sec. 2.1). Results are reported in
 * MeV/g per source particle (Sec. 2.2 "Materials").
 *
 * Conventions for every call:
 *  - Each call returns an ocmc_status; on failure a message is kept per
 *    context and returned by ocmc_last_error().
 *  - The library owns the context and all device memory it allocates.
 *    Input arrays are copied; the caller keeps ownership of its buffers.
 *  - A context is not thread-safe; one host thread drives it at a time.
 *  - All pointers named *_host are host memory; where a call takes an
 *    `on_device` flag, 1 means the pointer is CUDA device memory on the
 *    context's device and 0 means host memory.
 *  - Arrays over the voxel grid are x-fastest: v = ix + nx*(iy + ny*iz).
 */
#ifndef OCMC_H
#define OCMC_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ocmc_ctx ocmc_ctx;

typedef enum {
    OCMC_OK = 0,
    OCMC_ERR_ARG = 1,       /* invalid argument; nothing changed                  */
    OCMC_ERR_CUDA = 2,      /* a CUDA runtime call failed (no device, launch...)  */
    OCMC_ERR_OOM = 3,       /* device allocation failed                           */
    OCMC_ERR_OVERFLOW = 4,  /* a secondary-particle stack overflowed; the run's   */
                            /* tally misses the dropped particles                 */
    OCMC_ERR_TIMEOUT = 5,   /* a particle exceeded the step limit or a sampling   */
                            /* loop its iteration limit; that particle was dropped*/
    OCMC_ERR_STATE = 6,     /* call out of order (no phantom, no source, ...)     */
    OCMC_ERR_BOUNDS = 7     /* checks build only (libocmc_checks.so, built with   */
                            /* -DOCMC_CHECKS=1): a voxel index, tally address or  */
                            /* stack slot was out of range; the access was skipped*/
} ocmc_status;

/* Test modes of ocmc_params.flags (used by the physics tests, 0 in production). */
#define OCMC_FLAG_NO_HARD          1  /* no discrete Moller/bremsstrahlung events   */
#define OCMC_FLAG_NO_MS            2  /* no multiple-scattering deflection          */
#define OCMC_FLAG_KILL_FIRST_REAL  4  /* photons removed at first real interaction  */
#define OCMC_FLAG_KERMA            8  /* e-/e+ deposit their energy where created   */
/* Stepping variant (Sec. 4 Discussion): electron steps are not stopped at voxel faces but
 * cross as many voxels as their length d = min(d_maxs, d_maxe, d_event) takes them through,
 * depositing each voxel's own CSDA loss there; hard events are sampled against the
 * phantom-wide majorant so that a candidate may fall in any voxel; the multiple-scattering
 * angle of a step is that of its first voxel's medium; a step also ends where its energy has
 * fallen by the fraction f_maxe. Analytic single-beam source only (ocmc_run_range returns
 * OCMC_ERR_ARG with a phase-space source, ocmc_run_beamlets with beamlets). */
#define OCMC_FLAG_CROSS_VOXELS    16

/* Transport and execution parameters (Sec. 2.1: absorption energies, hard-event
 * cutoffs and the user-defined step limits d_maxs, d_maxe; Sec. 2.2.1: the
 * number of concurrently transported particles). Execution fields change speed
 * only: the dose is bit-identical for any value of them. */
typedef struct {
    float e_abs_e;          /* MeV, electron/positron absorption energy (0.2)      */
    float e_abs_g;          /* MeV, photon absorption energy (0.01)                */
    float w_cc;             /* MeV, Moller hard-collision threshold (= e_abs_e)    */
    float w_cb;             /* MeV, bremsstrahlung hard threshold (= e_abs_g)      */
    float d_maxs;           /* cm, maximum electron step (0.5)                     */
    float f_maxe;           /* maximum fractional CSDA loss per step (0.05)        */
    float s_min;            /* cm, boundaries closer than this are crossed without */
                            /* physics (1e-4)                                      */
    int32_t n_batches;      /* statistical batches B; batch = history id mod B (10)*/
    int32_t flags;          /* OCMC_FLAG_* test modes (0)                          */
    /* execution (tuning) parameters, 0 = automatic */
    int32_t block_threads;  /* threads per block of the transport kernel           */
    int32_t blocks_per_sm;  /* resident transport blocks per SM                    */
    int32_t stack_capacity; /* per-warp capacity of each secondary stack (8192)   */
    int32_t switch_high;    /* size of another stack that makes a warp move to it  */
                            /* (15/16 of the capacity); at or above the capacity   */
                            /* it disables switching on stack size                 */
    int32_t switch_low;     /* active lanes at or below which a warp whose own     */
                            /* stack and source are empty moves to another stack   */
    uint32_t stream_tag;    /* XORed into the high word of every history's random  */
                            /* stream (0); 0x80000000|b reproduces beamlet b       */
    float beamlet_capacity_scale; /* scales the pilot estimate of beamlet table    */
                            /* sizes (0 = 1); tables that fill up are enlarged and */
                            /* the run repeated, so any value gives the same dose  */
    int32_t refill_min;     /* free lanes a warp waits for before refilling (0=6)  */
    int32_t max_registers;  /* register cap of the transport kernel: 56, 64 or 80; */
                            /* 0 = 64 (with 1024-thread blocks)                    */
    float e_class_split;    /* MeV; > 0: charged particles waiting below this      */
                            /* energy go to a third per-warp stack, so that a warp */
                            /* steps electrons of one energy class at a time       */
                            /* (2.0; 0 = one charged stack)                        */
} ocmc_params;

/* Run statistics accumulated since the last ocmc_reset_tally(). */
typedef struct {
    uint64_t histories;        /* histories transported                           */
    uint64_t photon_flights;   /* Woodcock flights (real + fictitious)            */
    uint64_t fictitious;       /* fictitious photon events                         */
    uint64_t compton, photo, pair;
    uint64_t electron_steps;   /* condensed-history steps of e-/e+                 */
    uint64_t moller, brems;    /* accepted hard events                              */
    uint64_t hard_fictitious;  /* rejected hard-event candidates (energy Woodcock)  */
    uint64_t annihilations;
    uint64_t escaped;          /* particles leaving the phantom                     */
    uint64_t missed;           /* source particles that miss the phantom            */
    uint64_t geo_crossings;    /* boundary crossings without physics                */
    uint64_t majorant_violations; /* must stay 0                                     */
    uint64_t dropped;          /* particles dropped (overflow/limits); must stay 0  */
    uint64_t transmitted;      /* KILL_FIRST_REAL mode: photons out at z = Lz       */
    uint64_t warp_iterations;  /* warp-level scheduler iterations                   */
    uint64_t lane_steps;       /* lane-steps executed (active lanes summed)         */
    double e_in, e_dep, e_esc, e_miss, pair_mass, annih_mass, e_killed, e_trans, e_dropped; /* MeV */
    double last_run_ms;        /* device time of the last ocmc_run (CUDA events)   */
    /* transport-kernel timing (device timer): warp lifetimes summed over warps; the part
     * of them after each warp found the source exhausted (work from its own stacks only);
     * for the transport launches since the last reset, first warp start to last warp end,
     * and the earliest source exhaustion seen by a warp to the last warp end. With `warps`
     * (warps launched), 1 - warp_ms / (warps * span_ms) is the share of warp slots left idle
     * by warps that finished before the last one (the end-of-launch imbalance). */
    double warp_ms, tail_warp_ms, span_ms, tail_span_ms;
    uint64_t warps;
} ocmc_stats;

/* Fill p with the defaults listed above. */
void ocmc_default_params(ocmc_params* p);

/* Create a context on CUDA device `device` (Sec. 2.2.1 "Initialize"). p may be
 * NULL for defaults. Errors: OCMC_ERR_ARG (bad parameter values),
 * OCMC_ERR_CUDA (no such device / no driver), OCMC_ERR_OOM. On failure *out is
 * set to NULL. */
ocmc_status ocmc_init(ocmc_ctx** out, int device, const ocmc_params* p);

/* Replace the transport parameters (the tally is kept). Same errors as init. */
ocmc_status ocmc_set_params(ocmc_ctx* ctx, const ocmc_params* p);

/* ---- materials ----------------------------------------------------------------------
 * Sec. 2.1: each voxel has a density and a material type that selects the cross-section
 * and stopping-power data (the paper's database has 16 materials). By default material 0 is
 * water, 1 ICRP cortical bone (nominal 1.85 g/cm^3), 2 ICRP lung (0.26 g/cm^3). A material is a
 * composition: elements (atomic number Z, atomic mass A in g/mol, mass fraction; the fractions
 * are normalised), its mean excitation energy I (eV) and the nominal density that fixes its
 * density-effect parameters; every table is built from the closed-form models for it. */
typedef struct {
    int32_t n_elements;          /* 1..16 */
    int32_t Z[16];               /* 1..100 */
    double A[16];                /* g/mol */
    double mass_fraction[16];    /* >= 0, sum > 0 */
    double I_eV;                 /* (1, 1e4) */
    double density;              /* nominal g/cm^3, (0, 30] */
} ocmc_material;

/* Define n (1..16) materials; voxel material m of later phantoms is defs[m]. The definitions
 * are copied. The current phantom is dropped (its indices referred to the old set): call
 * ocmc_create_phantom again. A transport block holds the tables of at most 10 materials in
 * shared memory: with more than 10 defined, a phantom may use at most 10 distinct ones. */
ocmc_status ocmc_set_materials(ocmc_ctx* ctx, int n, const ocmc_material* defs);

/* The voxel phantom (Sec. 2.1: each voxel has a density and a material type).
 * density_host: nx*ny*nz float, g/cm^3, finite and in [0, 30];
 * material_host: nx*ny*nz uint8, an index into the defined materials (by default 0 water,
 *   1 cortical bone (ICRP), 2 lung (ICRP); see ocmc_set_materials);
 * dx, dy, dz: voxel size in cm. The phantom occupies [0,nx*dx] x [0,ny*dy] x
 * [0,nz*dz]. 1 <= nx, ny, nz <= 1024. Copies the data (host pointers) and
 * resets the tally. Errors: OCMC_ERR_ARG for bad sizes or values. */
ocmc_status ocmc_create_phantom(ocmc_ctx* ctx, int nx, int ny, int nz,
                                const float* density_host, const uint8_t* material_host,
                                float dx, float dy, float dz);

/* The beam (Sec. 2.2 "Materials": point source at an SSD with a field defined
 * at the surface, 15 MeV mono-energetic electrons or a 6 MV photon spectrum;
 * Sec. 2.2.1: source particles are simulated bin by bin in energy).
 * particle: 0 photon, 1 electron. bin_edges_host: n_bins+1 floats in MeV
 * (ascending per bin; a mono-energetic beam is n_bins=1 with equal edges);
 * weights_host: n_bins non-negative floats, not all zero; 1 <= n_bins <= 256.
 * Histories are stratified over the bins: of N histories, bin order q (bins by
 * decreasing energy) receives ids [floor(N c_q / W), floor(N c_{q+1} / W)),
 * c_q the partial weight sums, W the total. Energies are uniform in the bin.
 * field_x, field_y: cm, rectangle in the plane through iso normal to dir,
 * with in-plane axes e1 = normalize(y_hat x dir), e2 = dir x e1.
 * ssd > 0: point source at iso - ssd*dir; ssd <= 0: parallel beam along dir.
 * Particles travel in vacuum to the phantom surface. */
ocmc_status ocmc_set_source(ocmc_ctx* ctx, int particle, int n_bins,
                            const float* bin_edges_host, const float* weights_host,
                            float field_x, float field_y, float ssd,
                            const float iso[3], const float dir[3]);

/* ---- phase-space source ---------------------------------------------------------
 * Sec. 2.2 "Materials" leaves source generation open: source particles may come from a
 * phase-space file or from a user's own CPU/GPU source model. A record is one source
 * particle: position (cm, phantom frame: origin at the outer corner of voxel (0,0,0)),
 * direction (any non-zero length; normalised by the engine), kinetic energy (MeV) and type
 * (0 photon, 1 electron, 2 positron). History h of a run starts from record h mod n and moves
 * forward in vacuum to the phantom (a record inside the phantom starts where it is); records
 * are thus recycled when a run has more histories than records, each use with its own random
 * stream. The dose stays per source history (MeV/g per history). */
typedef struct {
    float x, y, z;
    float u, v, w;
    float E;
    int32_t type;
} ocmc_ps_particle;

/* Use n records (host memory, or device memory of the context's GPU if on_device) as the
 * source until the next ocmc_set_source / ocmc_set_phase_space. The records are copied.
 * OCMC_ERR_ARG if any record has another type, E outside (0, 1e4) MeV, a non-finite
 * position or a zero direction (the previous source is then unset). */
ocmc_status ocmc_set_phase_space(ocmc_ctx* ctx, const ocmc_ps_particle* records, uint64_t n, int on_device);

/* The same from a file: 8 bytes "OCMCPS01", uint64 record count (little endian), then the
 * 32-byte records above (little endian). OCMC_ERR_ARG on a missing, short or foreign file. */
ocmc_status ocmc_load_phase_space(ocmc_ctx* ctx, const char* path);

/* Transport histories 0..n_histories-1 with the Philox key `seed` and add the
 * deposited energy to the tally (Sec. 2.2.1, Table 1 loop). Asynchronous on
 * cuda_stream (a cudaStream_t, NULL = the legacy default stream); the call
 * returns after the launch. Repeated calls accumulate; use different seeds.
 * Errors: OCMC_ERR_STATE without phantom or source, OCMC_ERR_ARG if n is 0. */
ocmc_status ocmc_run(ocmc_ctx* ctx, uint64_t n_histories, uint64_t seed, void* cuda_stream);

/* Transport histories [first, first+count) of a run of n_total histories
 * (sharding over GPUs or resuming a run). The union of disjoint ranges with
 * the same n_total and seed gives the tally of one ocmc_run(n_total, seed),
 * bit for bit. A range of more than 1e8 histories is transported in launches of
 * 1e8 (on GB300 one launch of 1e9 histories ran 15 % slower per history than ten
 * of 1e8); by the same composition rule the tally does not change. */
ocmc_status ocmc_run_range(ocmc_ctx* ctx, uint64_t first, uint64_t count, uint64_t n_total,
                           uint64_t seed, void* cuda_stream);

/* Dose in MeV/g per source particle, D_v = sum_b E_bv / (rho_v V N), and its
 * batch standard error sigma_v = sqrt(sum_b (D_bv - D_v)^2 / (B (B-1)))
 * (Sec. 3.1). dose_out: nx*ny*nz floats; sigma_out may be NULL. Voxels of
 * zero density report 0. Synchronises with the last run. Errors:
 * OCMC_ERR_STATE before any run; OCMC_ERR_OVERFLOW / OCMC_ERR_TIMEOUT if the
 * runs dropped particles (the dose is still written). */
ocmc_status ocmc_get_dose(ocmc_ctx* ctx, float* dose_out, float* sigma_out, int on_device);

/* Raw int64 tally, B x nvox, in units of 2^-28 MeV (round to nearest even per
 * deposit). Integer sums make it bit-identical for any scheduling. */
ocmc_status ocmc_get_raw_tally(ocmc_ctx* ctx, int64_t* out, int on_device);

/* Add a raw tally (same layout) from another context or rank, together with
 * the number of histories it represents; used after a cross-GPU sum. */
ocmc_status ocmc_add_raw_tally(ocmc_ctx* ctx, const int64_t* in, int on_device,
                               uint64_t first, uint64_t count);

/* Zero the tally, the history count and the statistics. */
ocmc_status ocmc_reset_tally(ocmc_ctx* ctx);

/* Statistics of the runs since the last reset (synchronises); after ocmc_run_beamlets, of that
 * beamlet run alone (a beamlet run replaces its tallies). */
ocmc_status ocmc_get_stats(ocmc_ctx* ctx, ocmc_stats* out);

/* Number of voxels and batches of the current phantom/parameters. */
ocmc_status ocmc_get_shape(ocmc_ctx* ctx, int64_t* nvox, int32_t* n_batches);

/* Message of the last failed call on ctx ("" if none; valid until the next
 * call). ctx may be NULL for failures of ocmc_init. */
const char* ocmc_last_error(ocmc_ctx* ctx);

/* Release the context and its device memory. NULL is ignored. */
void ocmc_destroy(ocmc_ctx* ctx);

/* ---- batched beamlets --------------------------------------------------------
 * Many small beams transported together in one persistent launch, captured once in
 * a CUDA graph and replayed, each beamlet with its own sparse tally (an open-
 * addressing hash of voxel -> int64 energy). Extends the paper's per-source loop
 * (Sec. 2.2.1, Table 1) to a queue of sources; the per-history physics is the same.
 * Beamlet b's histories use random streams whose history high word is
 * 0x80000000 | b, so a single-beam run with stream_tag = 0x80000000 | b, the same
 * source, seed and n_histories gives beamlet b's tally densely, bit for bit. */
typedef struct {
    float field_x, field_y;  /* cm, rectangle in the plane through iso normal to dir */
    float ssd;               /* cm; > 0 point source at iso - ssd*dir, <= 0 parallel  */
    float iso[3];            /* cm, field centre                                      */
    float dir[3];            /* beam axis (normalised by the library)                 */
    uint64_t n_histories;    /* 1 .. 2^32 - 1                                         */
} ocmc_beamlet;

/* Define the beamlets (all share particle type and energy spectrum, as in
 * ocmc_set_source, with n_bins <= 32). 1 <= n_beamlets <= 65536. Host arrays,
 * copied. Invalidates table sizes and the captured graph. */
ocmc_status ocmc_set_beamlets(ocmc_ctx* ctx, int particle, int n_bins, const float* bin_edges_host,
                              const float* weights_host, int n_beamlets, const ocmc_beamlet* beamlets_host);

/* Transport every beamlet's histories with Philox key `seed` (replacing the
 * previous beamlet tallies). The first call after ocmc_set_beamlets sizes each
 * table from two pilot runs (distinct-voxel footprint at two history counts,
 * extrapolated as a power law) and captures the launch in a CUDA graph; later
 * calls replay it. A table that fills up is enlarged and the run repeated.
 * Synchronises cuda_stream. */
ocmc_status ocmc_run_beamlets(ocmc_ctx* ctx, uint64_t seed, void* cuda_stream);

/* Beamlet b's non-zero voxels in increasing voxel order: idx_host (int32 voxel
 * index), dose_host (MeV/g per history of that beamlet), raw_host (int64, 2^-28
 * MeV); any of the three may be NULL. At most `capacity` entries are written;
 * *nnz receives the number of non-zero voxels. */
ocmc_status ocmc_get_beamlet_dose(ocmc_ctx* ctx, int beamlet, int32_t* idx_host, float* dose_host,
                                  int64_t* raw_host, int64_t capacity, int64_t* nnz);

/* Autotuner: times the transport of `pilot_histories` histories of the current
 * source for a set of launch shapes (threads per block, type-switch thresholds,
 * stack capacity) and keeps the fastest in the context's parameters (copied to
 * *chosen if not NULL). Resets the tally. The dose does not depend on the choice. */
ocmc_status ocmc_autotune(ocmc_ctx* ctx, uint64_t pilot_histories, ocmc_params* chosen);

/* ---- learned dose denoiser ----------------------------------------------------
 * The paper has no learned component; this is a systems extension. A 3D U-Net
 * (4 levels, 16/32/64/128 channels, 3x3x3 convolutions with ReLU, 2x2x2 stride-2
 * down and transposed-up convolutions, concatenated skips, 1x1x1 head adding a
 * correction to the normalised input) maps a low-history dose plus density to a
 * converged dose. BF16 activations and weights, FP32 accumulation on the tensor
 * cores, FP32 master weights trained with Adam. Grid sizes must be multiples of 8
 * (at most 512). Dose arrays are nx*ny*nz floats on the network's device. */
typedef struct ocmc_unet ocmc_unet;

/* Create a network with He-normal initial weights drawn from Philox(seed). */
ocmc_status ocmc_unet_create(ocmc_unet** out, int device, int nx, int ny, int nz, uint64_t seed);
void ocmc_unet_destroy(ocmc_unet* net);
const char* ocmc_unet_last_error(ocmc_unet* net);
/* Number of FP32 parameters; get/set all of them (grads = 1: the last gradients).
 * Setting the parameters also restarts Adam (zero moments, step count 0). */
ocmc_status ocmc_unet_num_params(ocmc_unet* net, int64_t* n);
ocmc_status ocmc_unet_get_params(ocmc_unet* net, float* host, int grads);
ocmc_status ocmc_unet_set_params(ocmc_unet* net, const float* host);
/* Denoised dose (same units as dose_dev) from (dose_dev, sigma_dev, density_dev), device
 * arrays of nx*ny*nz floats: the Monte Carlo dose, its statistical uncertainty (batch standard
 * error, same units; may be NULL, read as zero) and the density in g/cm^3. The network sees
 * dose / s, density and sigma / s, s the maximum of dose_dev. */
ocmc_status ocmc_unet_forward(ocmc_unet* net, const float* dose_dev, const float* sigma_dev, const float* density_dev,
                              float* out_dev, void* cuda_stream);
/* One Adam step (learning rate lr; lr <= 0: gradients only) on the mean squared error
 * between output and target_dev / s over voxels with density >= 0.1 g/cm^3, s the
 * maximum of dose_dev. *loss_host (may be NULL) receives the loss (synchronises). */
ocmc_status ocmc_unet_train_step(ocmc_unet* net, const float* dose_dev, const float* sigma_dev,
                                 const float* density_dev, const float* target_dev, float lr, float* loss_host,
                                 void* cuda_stream);
/* Timing: forward passes with a CUDA event pair around every layer (20 layers, in the order
 * encoder level 0..3, then decoder level 2..0); ms_out[i] (may be NULL to query *n_layers) is
 * the mean duration of layer i over `repeats` passes. Synchronises. */
ocmc_status ocmc_unet_layer_times(ocmc_unet* net, const float* dose_dev, const float* sigma_dev,
                                  const float* density_dev, int repeats, float* ms_out, int* n_layers);
/* One layer through the network's own kernels (for the gradient tests): mode 0 3x3x3
 * convolution, 1 2x2x2 stride-2 convolution, 2 its transposed form; (nx,ny,nz) is the
 * fine grid (even sides of 2 to 512); cin, cout multiples of 16 up to 256; x, dy, y, dx
 * channels-last FP32 host arrays (inputs rounded to BF16); w [taps][cin][cout];
 * y = layer(x) without bias or ReLU; dx, dw the gradients for dy. OCMC_ERR_ARG otherwise. */
ocmc_status ocmc_unet_test_layer(int device, int mode, int nx, int ny, int nz, int cin, int cout,
                                 const float* x_host, const float* w_host, const float* dy_host, float* y_host,
                                 float* dx_host, float* dw_host);
/* Test hook of the tensor-memory convolution's bounded waits (no counterpart in the paper;
 * process-wide, off by default): with tile >= 0, every later launch's MMA-issuing thread waits,
 * at its block-local tile number `tile`, up to `wait_ns` nanoseconds (at most the normal 2 s
 * limit) on a barrier that nothing completes; the wait runs out, the block stops issuing, lets
 * its copies and MMAs in flight finish, frees its tensor memory and sets the network's error
 * flag, so the call returns OCMC_ERR_TIMEOUT. tile = -1 turns the hook off. */
ocmc_status ocmc_unet_test_stall(int tile, uint64_t wait_ns);
/* Denoise the context's current dose (and its batch sigma, the network's third input) with the
 * network; where the denoised value
 * differs from the plain Monte Carlo value by more than k_sigma times the plain dose's
 * batch standard error (pooled over the voxel's 3x3x3 neighbourhood: root of the mean
 * variance) the plain value is kept and flag_out (may be NULL) is 1. dose_out and
 * flag_out hold nx*ny*nz floats, on the device if on_device, else in host memory. */
ocmc_status ocmc_denoise(ocmc_ctx* ctx, ocmc_unet* net, float k_sigma, float* dose_out, float* flag_out,
                         int on_device);

/* ---- test access to the engine's building blocks ---------------------------
 * These run the same device functions the transport kernel uses, so the
 * tests can compare each building block with the CPU oracle. */

/* Philox4x32-10 (Salmon et al. 2011) on the device: for block j in
 * [0, n_blocks), out_host[4j..4j+3] = Philox(counter = (first_block + j,
 * c1, c2, c3), key = (key0, key1)). */
ocmc_status ocmc_test_philox(int device, uint32_t key0, uint32_t key1, uint32_t c1, uint32_t c2,
                             uint32_t c3, uint32_t first_block, uint32_t n_blocks,
                             uint32_t* out_host);

/* The transport kernel's rotation of a direction (Sec. 2.1: new directions after Compton,
 * Moller and bremsstrahlung events and multiple scattering): for j in [0, n), the unit vector
 * dir_host[3j..3j+2] turned by polar cosine mu_host[j] and azimuth 2 pi xi_host[j] about
 * itself, written to out_host[3j..3j+2]. Host arrays; OCMC_ERR_ARG on NULL or n <= 0. */
ocmc_status ocmc_test_rotate(int device, const float* dir_host, const float* mu_host,
                             const float* xi_host, int n, float* out_host);

/* Source particles of histories [first, first+count) of a run of n_total:
 * out_host[8j..8j+7] = x, y, z, u, v, w, E, entered (1/0). */
ocmc_status ocmc_test_source(ocmc_ctx* ctx, uint64_t n_total, uint64_t first, uint64_t count,
                             uint64_t seed, float* out_host);

/* Samples of one interaction model at energy E (MeV) in material m:
 * kind 0: Compton cos(theta); 1: Moller W/T; 2: bremsstrahlung photon energy
 * (MeV); 3: multiple-scattering cos(theta) for G1 = aux (path / lambda_1).
 * Sample j uses the Philox stream (history j, sub-stream 0x5A5A + kind). */
ocmc_status ocmc_test_sample(ocmc_ctx* ctx, int kind, int material, float E, float aux,
                             uint64_t n, uint64_t seed, float* out_host);

/* Engine tables interpolated at energies E_host[0..n) for material m:
 * out_host[8j..8j+7] = mu_total, mu_compton, mu_photo (cm^2/g), restricted
 * CSDA range R (g/cm^2, offset: R at the table's lowest energy is the
 * first-interval estimate), 1/lambda_1 (cm^2/g), sigma_moller, sigma_brems
 * (cm^2/g), hard-event majorant (cm^2/g). Builds the tables if needed (a
 * phantom must be set). */
ocmc_status ocmc_test_tables(ocmc_ctx* ctx, int material, const float* E_host, int n,
                             float* out_host);

/* End energy of a CSDA step of mass thickness X (g/cm^2) from energy T in
 * material m, as the transport kernel computes it (range-table inversion). */
ocmc_status ocmc_test_csda(ocmc_ctx* ctx, int material, const float* T_host, const float* X_host,
                           int n, float* out_host);

/* ---- allocation-free transport -----------------------------------------------
 * The paper has no counterpart to this call. It is for callers that cannot
 * allocate device memory: code running under another framework's allocator or
 * memory pool (which must own every device allocation), treatment-planning hosts
 * that forbid allocation after start-up, and plug-ins handed only device
 * pointers. It transports histories [first, first+count) of a run of n_total,
 * exactly as ocmc_run_range does on a context with the same phantom, source,
 * parameters and seed (the same tally, bit for bit), and ADDS the deposited
 * energy into tally_dev (int64, n_batches x nx*ny*nz, units 2^-28 MeV; zero it
 * first for a fresh run). It calls no cudaMalloc, cudaFree or allocating routine.
 *
 * All scratch memory (physics tables, secondary-particle stacks, history counter,
 * statistics, error flag) is one static device array of
 * OCMC_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds until
 * the process exits. Each call clears the counter, statistics and error flag and
 * rebuilds the tables; the array otherwise keeps the last call's contents. Calls
 * that overlap on the GPU (other streams, other host threads) share the array and
 * race: serialise them. The first call on a device looks up the array's address
 * with that device current and caches it: make it before any stream capture.
 *
 * density_dev, material_dev: device arrays as in ocmc_create_phantom, with the built-in
 * materials 0 water, 1 cortical bone, 2 lung (values are checked on the device after the
 * table build and before any transport; bad values give OCMC_ERR_ARG and leave the tally
 * untouched). Source arguments as in ocmc_set_source (host arrays). params: NULL for
 * defaults (256-record stacks, 256-thread blocks; the type-switch threshold defaults to
 * capacity - capacity/16 as in ocmc_run_range); a launch shape (block_threads,
 * blocks_per_sm, stack_capacity) whose stacks do not fit in the static array is rejected
 * with OCMC_ERR_ARG. Runs on cuda_stream and waits for it twice before returning (after the
 * table build and after the transport, to read the error flag). The caller's current device
 * is restored on return. err_msg (host, may be NULL) receives a message of at most err_len
 * bytes on failure. */
#define OCMC_NOALLOC_SCRATCH_BYTES (64ull * 1024ull * 1024ull)
ocmc_status ocmc_run_noalloc(int device, int nx, int ny, int nz, const float* density_dev,
                             const uint8_t* material_dev, float dx, float dy, float dz, int particle,
                             int n_bins, const float* bin_edges_host, const float* weights_host,
                             float field_x, float field_y, float ssd, const float iso[3], const float dir[3],
                             const ocmc_params* params, uint64_t first, uint64_t count, uint64_t n_total,
                             uint64_t seed, int64_t* tally_dev, void* cuda_stream, char* err_msg,
                             size_t err_len);

#ifdef __cplusplus
}
#endif
#endif
