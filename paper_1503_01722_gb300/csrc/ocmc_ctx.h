// ocmc_ctx.h -- the engine context (private to the library's host code).
#pragma once
#include "ocmc.h"
#include "ocmc_internal.h"

#include <string>
#include <vector>

struct ocmc_ctx {
    int device = 0;
    int sms = 0;
    // blocks per SM of the last launch shape asked for (the occupancy query costs host time on
    // every run otherwise)
    mutable int occ_threads = -1, occ_nreg = -1, occ_bps = 0;
    mutable size_t occ_smem = 0;
    ocmc_params p{};
    std::string err;
    // phantom
    int nx = 0, ny = 0, nz = 0;
    float dx = 0.f, dy = 0.f, dz = 0.f;
    long long nvox = 0;
    float* d_density = nullptr;
    uint8_t* d_material = nullptr;
    bool have_phantom = false;
    // source
    bool have_source = false;
    int particle = 0, n_bins = 0;
    std::vector<float> edges, weights;
    float fx = 0.f, fy = 0.f, ssd = 0.f, iso[3] = {0, 0, 0}, dir[3] = {0, 0, 1}, e1[3], e2[3];
    int src_kind = 0;                        // 0 analytic beam (ocmc_set_source), 1 phase space
    ocmc::PsRec* d_ps = nullptr;             // phase-space records on the device
    unsigned long long ps_n = 0, ps_cap = 0;
    // materials: defined (default water, ICRP cortical bone, ICRP lung) and the ones whose
    // tables are built (staged): all defined ones when at most MAX_STAGED, else the phantom's
    // own, whose indices are compacted when the phantom is uploaded
    std::vector<ocmc::MatDef> mats;
    std::vector<ocmc::MatDef> staged;
    std::vector<int> slot_of;                // defined index -> staged slot, -1 if not staged
    // tables
    ocmc::Tables t{};
    bool tables_valid = false;               // material and phantom parts both current
    bool mat_tables_valid = false;           // material part current (kept across phantoms of the same staged set)
    // tally and its history counts per batch
    long long* d_tally = nullptr;
    int tally_B = 0;
    std::vector<double> nb;
    // run scratch
    unsigned long long* d_stats = nullptr;
    unsigned long long* d_counter = nullptr;
    unsigned long long* d_sum = nullptr;
    int* d_err = nullptr;
    ocmc::PRec* d_stacks = nullptr;
    size_t stack_records = 0;
    // outputs
    float* d_dose = nullptr;
    float* d_sigma = nullptr;
    float* d_invnb = nullptr;       // N / n_b per batch (k_finalize)
    int invnb_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timed = false;
    cudaStream_t last_stream = nullptr;
    bool ran = false;
    // batched beamlets
    int bl_n = 0, bl_particle = 0, bl_bins = 0;
    std::vector<float> bl_edges, bl_weights;
    std::vector<ocmc_beamlet> bl_list;
    std::vector<unsigned long long> bl_cap;     // table capacity per beamlet (power of two)
    bool bl_sized = false, bl_ran = false;
    ocmc::BeamletDev* d_bl = nullptr;
    unsigned long long* d_bl_prefix = nullptr;
    unsigned long long* d_bl_offs = nullptr;
    unsigned int* d_bl_caps = nullptr;
    unsigned long long* d_bl_nnz = nullptr;
    unsigned int* d_bl_over = nullptr;
    unsigned int* d_bl_keys = nullptr;
    unsigned long long* d_bl_vals = nullptr;
    size_t bl_slots = 0;
    cudaStream_t bl_capture = nullptr;
    cudaGraphExec_t bl_exec = nullptr;
    bool bl_graph_valid = false;
    unsigned long long bl_graph_seed = 0;
    long long* d_dense = nullptr;
    unsigned int* d_chunks = nullptr;
    int* d_oidx = nullptr;
    float* d_odose = nullptr;
    long long* d_oraw = nullptr;
    long long out_cap = 0;
};

namespace ocmc {
// shared host helpers (ocmc_api.cu)
ocmc_status ctx_fail(ocmc_ctx* c, ocmc_status s, const std::string& msg);
ocmc_status ctx_cuda_fail(ocmc_ctx* c, cudaError_t e, const char* where);
ocmc_status ctx_ensure_tables(ocmc_ctx* c, cudaStream_t s);
void ctx_fill_args(const ocmc_ctx* c, TransportArgs& a);
void ctx_launch_shape(const ocmc_ctx* c, int* threads, int* blocks, int* cap, int* nreg);
ocmc_status ctx_ensure_stacks(ocmc_ctx* c, size_t records);
void stratify_bins(const float* edges, const float* weights, int n_bins, unsigned long long N, int* order,
                   unsigned long long* bound);
void beam_frame(const float dir[3], float d[3], float e1[3], float e2[3]);
}  // namespace ocmc
