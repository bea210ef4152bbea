// ocmc_api.cu -- the C ABI (include/ocmc.h): context, validation, memory and launches.
#include "ocmc_ctx.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace ocmc;

namespace ocmc {
cudaError_t launch_add_tally(long long* tally, const long long* in, long long n, cudaStream_t s);
cudaError_t launch_sum_tally(const long long* tally, long long n, unsigned long long* out, cudaStream_t s);
}


namespace {

thread_local std::string g_init_err;

ocmc_status fail(ocmc_ctx* c, ocmc_status s, const std::string& msg)
{
    if (c) c->err = msg; else g_init_err = msg;
    return s;
}

ocmc_status cuda_fail(ocmc_ctx* c, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? OCMC_ERR_OOM : OCMC_ERR_CUDA, m);
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t n)
{
    if (*p) { cudaFree(*p); *p = nullptr; }
    return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T) > 0 ? n * sizeof(T) : 1);
}

template <class T>
void dfree(T** p)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
}

const char* check_params(const ocmc_params* p)
{
    if (!(p->e_abs_e >= 1e-3f && p->e_abs_e <= 10.f)) return "e_abs_e must be in [0.001, 10] MeV";
    if (!(p->e_abs_g >= 1e-3f && p->e_abs_g <= 10.f)) return "e_abs_g must be in [0.001, 10] MeV";
    if (!(p->w_cc >= 1e-3f && p->w_cc <= 10.f)) return "w_cc must be in [0.001, 10] MeV";
    if (!(p->w_cb >= 1e-3f && p->w_cb <= 10.f)) return "w_cb must be in [0.001, 10] MeV";
    if (!(p->d_maxs > 0.f && p->d_maxs <= 1e3f)) return "d_maxs must be in (0, 1000] cm";
    if (!(p->f_maxe > 0.f && p->f_maxe <= 0.5f)) return "f_maxe must be in (0, 0.5]";
    if (!(p->s_min >= 0.f && p->s_min <= 0.01f)) return "s_min must be in [0, 0.01] cm";
    if (p->n_batches < 1 || p->n_batches > 1000) return "n_batches must be in [1, 1000]";
    if (p->flags < 0 || p->flags > 31) return "unknown flags";
    if (p->block_threads != 0 && (p->block_threads < 32 || p->block_threads > 1024 || p->block_threads % 32))
        return "block_threads must be 0 or a multiple of 32 in [32, 1024]";
    if (p->blocks_per_sm < 0 || p->blocks_per_sm > 32) return "blocks_per_sm must be in [0, 32]";
    if (p->stack_capacity != 0 && (p->stack_capacity < 64 || p->stack_capacity > (1 << 20)))
        return "stack_capacity must be 0 or in [64, 2^20]";
    if (p->switch_high < 0 || p->switch_low < 0 || p->switch_low > 32) return "bad switch thresholds";
    if (p->refill_min < 0 || p->refill_min > 32) return "refill_min must be in [0, 32]";
    if (p->max_registers != 0 && !transport_nreg_supported(p->max_registers))
        return "max_registers must be 0, 56, 64 or 80";
    if (!(p->beamlet_capacity_scale >= 0.f && p->beamlet_capacity_scale <= 1e6f))
        return "beamlet_capacity_scale must be in [0, 1e6]";
    if (!(p->e_class_split >= 0.f && p->e_class_split <= 30.f)) return "e_class_split must be in [0, 30] MeV";
    return nullptr;
}

unsigned long long batch_count(unsigned long long N, int b, int B)
{
    return N > (unsigned long long)b ? (N - b - 1) / B + 1 : 0ull;
}

void add_histories(ocmc_ctx* c, unsigned long long first, unsigned long long count)
{
    for (int b = 0; b < c->tally_B; ++b)
        c->nb[b] += (double)(batch_count(first + count, b, c->tally_B) - batch_count(first, b, c->tally_B));
}

// Stratification of histories over energy bins: bins in order of decreasing lower
// edge (ties by index); bin at position q gets [floor(N c_q / W), floor(N c_{q+1} / W)).
void stratify(const ocmc_ctx* c, unsigned long long N, SourceDev& s)
{
    int nb = c->n_bins;
    for (int i = 0; i < nb; ++i) s.order[i] = i;
    for (int i = 1; i < nb; ++i) {
        int v = s.order[i], j = i - 1;
        while (j >= 0 && (c->edges[s.order[j]] < c->edges[v] || (c->edges[s.order[j]] == c->edges[v] && s.order[j] > v))) {
            s.order[j + 1] = s.order[j];
            --j;
        }
        s.order[j + 1] = v;
    }
    double W = 0.0;
    for (int q = 0; q < nb; ++q) W += (double)c->weights[s.order[q]];
    double cum = 0.0;
    s.bound[0] = 0;
    for (int q = 1; q < nb; ++q) {
        cum += (double)c->weights[s.order[q - 1]];
        double b = std::floor((double)N * cum / W);
        unsigned long long u = (unsigned long long)b;
        if (u > N) u = N;
        if (u < s.bound[q - 1]) u = s.bound[q - 1];
        s.bound[q] = u;
    }
    s.bound[nb] = N;
    for (int i = 0; i < nb; ++i) {
        s.lo[i] = c->edges[i];
        s.hi[i] = c->edges[i + 1];
    }
}

void fill_args(const ocmc_ctx* c, TransportArgs& a)
{
    memset(&a, 0, sizeof(a));
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
    a.dx = c->dx; a.dy = c->dy; a.dz = c->dz;
    a.density = c->d_density;
    a.material = c->d_material;
    a.nvox = c->nvox;
    a.t = c->t;
    a.pp.e_abs_e = c->p.e_abs_e; a.pp.e_abs_g = c->p.e_abs_g;
    a.pp.w_cc = c->p.w_cc; a.pp.w_cb = c->p.w_cb;
    a.pp.d_maxs = c->p.d_maxs; a.pp.f_maxe = c->p.f_maxe; a.pp.s_min = c->p.s_min;
    a.pp.flags = c->p.flags;
    a.pp.n_batches = c->p.n_batches;
    a.stream_tag = c->p.stream_tag;
    a.tally = reinterpret_cast<unsigned long long*>(c->d_tally);
    a.stats = c->d_stats;
    a.err = c->d_err;
    a.hist_counter = c->d_counter;
    a.src.particle = c->src_kind == 1 ? 0 : c->particle;
    a.src.n_bins = c->n_bins;
    a.ps = c->src_kind == 1 ? c->d_ps : nullptr;
    a.ps_n = c->src_kind == 1 ? c->ps_n : 0;
    a.src.fx = c->fx; a.src.fy = c->fy; a.src.ssd = c->ssd;
    for (int k = 0; k < 3; ++k) {
        a.src.iso[k] = c->iso[k]; a.src.e1[k] = c->e1[k]; a.src.e2[k] = c->e2[k]; a.src.dir[k] = c->dir[k];
    }
}

bool same_defs(const std::vector<MatDef>& a, const std::vector<MatDef>& b)
{
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i) {
        const MatDef &x = a[i], &y = b[i];
        if (x.n != y.n || x.I_eV != y.I_eV || x.rho0 != y.rho0) return false;
        for (int k = 0; k < x.n; ++k)
            if (x.Z[k] != y.Z[k] || x.A[k] != y.A[k] || x.w[k] != y.w[k]) return false;
    }
    return true;
}

ocmc_status ensure_tables(ocmc_ctx* c, cudaStream_t s)
{
    if (c->tables_valid) return OCMC_OK;
    if (!c->mat_tables_valid) {
        PhysParams pp{c->p.e_abs_e, c->p.e_abs_g, c->p.w_cc, c->p.w_cb, c->p.d_maxs, c->p.f_maxe, c->p.s_min,
                      c->p.flags, c->p.n_batches};
        CK(build_material_tables(c->t, pp, c->staged.data(), s), "table build");
        c->mat_tables_valid = true;
    }
    CK(build_phantom_tables(c->t, c->d_density, c->d_material, c->nvox, c->d_err, s), "table build");
    c->tables_valid = true;
    return OCMC_OK;
}

ocmc_status ensure_tally(ocmc_ctx* c)
{
    if (c->d_tally && c->tally_B == c->p.n_batches) return OCMC_OK;
    CK(dalloc(&c->d_tally, (size_t)c->p.n_batches * c->nvox), "tally allocation");
    CK(cudaMemset(c->d_tally, 0, sizeof(long long) * (size_t)c->p.n_batches * c->nvox), "tally reset");
    c->tally_B = c->p.n_batches;
    c->nb.assign(c->tally_B, 0.0);
    c->ran = false;
    return OCMC_OK;
}

void launch_shape(const ocmc_ctx* c, int* threads, int* blocks, int* cap, int* nreg)
{
    *nreg = c->p.max_registers ? c->p.max_registers : 64;
    *threads = c->p.block_threads ? c->p.block_threads : (*nreg == 64 ? 1024 : *nreg == 56 ? 384 : 256);
    size_t smem = transport_smem_bytes(c->t.n_mat);
    int bps = c->p.blocks_per_sm;
    if (!bps) {
        if (c->occ_threads != *threads || c->occ_nreg != *nreg || c->occ_smem != smem) {
            c->occ_bps = transport_max_blocks_per_sm(*threads, smem, *nreg);
            c->occ_threads = *threads;
            c->occ_nreg = *nreg;
            c->occ_smem = smem;
        }
        bps = c->occ_bps;
    }
    if (bps < 1) bps = 1;
    *blocks = c->sms * bps;
    *cap = c->p.stack_capacity ? c->p.stack_capacity : 8192;
}

}  // namespace

namespace ocmc {
ocmc_status ctx_fail(ocmc_ctx* c, ocmc_status s, const std::string& msg) { return fail(c, s, msg); }
ocmc_status ctx_cuda_fail(ocmc_ctx* c, cudaError_t e, const char* where) { return cuda_fail(c, e, where); }
ocmc_status ctx_ensure_tables(ocmc_ctx* c, cudaStream_t s) { return ensure_tables(c, s); }
void ctx_fill_args(const ocmc_ctx* c, TransportArgs& a) { fill_args(c, a); }
void ctx_launch_shape(const ocmc_ctx* c, int* threads, int* blocks, int* cap, int* nreg)
{
    launch_shape(c, threads, blocks, cap, nreg);
}

ocmc_status ctx_ensure_stacks(ocmc_ctx* c, size_t need)
{
    if (need > c->stack_records) {
        if (c->ran || c->last_stream) cudaDeviceSynchronize();
        CK(dalloc(&c->d_stacks, need), "stack allocation");
        c->stack_records = need;
    }
    return OCMC_OK;
}

void stratify_bins(const float* edges, const float* weights, int nb, unsigned long long N, int* order,
                   unsigned long long* bound)
{
    for (int i = 0; i < nb; ++i) order[i] = i;
    for (int i = 1; i < nb; ++i) {
        int v = order[i], j = i - 1;
        while (j >= 0 && (edges[order[j]] < edges[v] || (edges[order[j]] == edges[v] && order[j] > v))) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = v;
    }
    double W = 0.0, cum = 0.0;
    for (int q = 0; q < nb; ++q) W += (double)weights[order[q]];
    bound[0] = 0;
    for (int q = 1; q < nb; ++q) {
        cum += (double)weights[order[q - 1]];
        unsigned long long u = (unsigned long long)std::floor((double)N * cum / W);
        if (u > N) u = N;
        if (u < bound[q - 1]) u = bound[q - 1];
        bound[q] = u;
    }
    bound[nb] = N;
}

void beam_frame(const float dir[3], float d[3], float e1[3], float e2[3])
{
    double v[3] = {dir[0], dir[1], dir[2]};
    double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int k = 0; k < 3; ++k) v[k] /= n;
    double a[3] = {v[2], 0.0, -v[0]};   // y_hat x dir
    if (std::sqrt(a[0] * a[0] + a[2] * a[2]) < 1e-6) { a[0] = 0.0; a[1] = -v[2]; a[2] = v[1]; }   // x_hat x dir
    double na = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    for (int k = 0; k < 3; ++k) a[k] /= na;
    double b[3] = {v[1] * a[2] - v[2] * a[1], v[2] * a[0] - v[0] * a[2], v[0] * a[1] - v[1] * a[0]};
    for (int k = 0; k < 3; ++k) { d[k] = (float)v[k]; e1[k] = (float)a[k]; e2[k] = (float)b[k]; }
}
}  // namespace ocmc

extern "C" {

void ocmc_default_params(ocmc_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->e_abs_e = 0.2f;
    p->e_abs_g = 0.01f;
    p->w_cc = 0.2f;
    p->w_cb = 0.01f;
    p->d_maxs = 0.5f;
    p->f_maxe = 0.05f;
    p->s_min = 1e-4f;
    p->n_batches = 10;
    p->e_class_split = 2.0f;
}

ocmc_status ocmc_init(ocmc_ctx** out, int device, const ocmc_params* p)
{
    if (!out) return fail(nullptr, OCMC_ERR_ARG, "out is NULL");
    *out = nullptr;
    ocmc_params q;
    ocmc_default_params(&q);
    if (p) q = *p;
    if (const char* m = check_params(&q)) return fail(nullptr, OCMC_ERR_ARG, m);
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return fail(nullptr, OCMC_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    if (device < 0 || device >= n) return fail(nullptr, OCMC_ERR_ARG, "device index out of range");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, OCMC_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    ocmc_ctx* c = new ocmc_ctx();
    c->device = device;
    c->p = q;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t r = cudaSuccess;
    if (r == cudaSuccess) r = dalloc(&c->t.ph, MAX_STAGED * NE * 4);
    if (r == cudaSuccess) r = dalloc(&c->t.el, MAX_STAGED * NE * 4);
    if (r == cudaSuccess) r = dalloc(&c->t.el2, MAX_STAGED * NE * 2);
    if (r == cudaSuccess) r = dalloc(&c->t.phmaj, NE);
    if (r == cudaSuccess) r = dalloc(&c->t.elmaj, NE);
    if (r == cudaSuccess) r = dalloc(&c->t.rinv, MAX_STAGED * NR);
    if (r == cudaSuccess) r = dalloc(&c->t.msA, NG);
    if (r == cudaSuccess) r = dalloc(&c->t.rmeta, 2 * MAX_STAGED);
    if (r == cudaSuccess) r = dalloc(&c->t.msc, 2 * MAX_STAGED);
    if (r == cudaSuccess) r = dalloc(&c->t.scratch, MAX_STAGED * NE);
    if (r == cudaSuccess) r = dalloc(&c->t.rho_max, MAX_STAGED);
    if (r == cudaSuccess) r = dalloc(&c->t.mats, MAX_STAGED);
    {
        MatDef d[NMAT_DEFAULT];
        material_defs(d);
        c->mats.assign(d, d + NMAT_DEFAULT);
        c->staged = c->mats;
        c->slot_of = {0, 1, 2};
        c->t.n_mat = NMAT_DEFAULT;
    }
    if (r == cudaSuccess) r = dalloc(&c->d_stats, ST_COUNT);
    if (r == cudaSuccess) r = dalloc(&c->d_counter, 1);
    if (r == cudaSuccess) r = dalloc(&c->d_sum, 1);
    if (r == cudaSuccess) r = dalloc(&c->d_err, 1);
    if (r == cudaSuccess) r = cudaMemset(c->d_stats, 0, ST_COUNT * sizeof(unsigned long long));
    if (r == cudaSuccess) r = cudaMemset(c->d_err, 0, sizeof(int));
    if (r == cudaSuccess) r = cudaEventCreate(&c->ev0);
    if (r == cudaSuccess) r = cudaEventCreate(&c->ev1);
    if (r != cudaSuccess) {
        ocmc_status s = cuda_fail(nullptr, r, "ocmc_init");
        ocmc_destroy(c);
        return s;
    }
    *out = c;
    return OCMC_OK;
}

ocmc_status ocmc_set_params(ocmc_ctx* c, const ocmc_params* p)
{
    if (!c || !p) return fail(c, OCMC_ERR_ARG, "NULL argument");
    if (const char* m = check_params(p)) return fail(c, OCMC_ERR_ARG, m);
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    bool phys = memcmp(&c->p, p, offsetof(ocmc_params, block_threads)) != 0;
    c->p = *p;
    if (phys) c->tables_valid = c->mat_tables_valid = false;
    if (c->have_phantom && c->tally_B != p->n_batches) return ensure_tally(c);
    return OCMC_OK;
}

ocmc_status ocmc_set_materials(ocmc_ctx* c, int n, const ocmc_material* defs)
{
    if (!c) return fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (n < 1 || n > MAX_MAT || !defs) return fail(c, OCMC_ERR_ARG, "need 1 to 16 materials");
    std::vector<MatDef> mats((size_t)n);
    for (int m = 0; m < n; ++m) {
        const ocmc_material& d = defs[m];
        if (d.n_elements < 1 || d.n_elements > MAX_ELEM)
            return fail(c, OCMC_ERR_ARG, "material " + std::to_string(m) + ": 1 to 16 elements");
        if (!(d.I_eV > 1.0 && d.I_eV < 1e4) || !(d.density > 0.0 && d.density <= 30.0))
            return fail(c, OCMC_ERR_ARG, "material " + std::to_string(m) + ": need 1 < I < 1e4 eV, 0 < density <= 30");
        double ws = 0.0;
        MatDef& o = mats[m];
        std::memset(&o, 0, sizeof(o));
        o.n = d.n_elements;
        for (int i = 0; i < d.n_elements; ++i) {
            if (d.Z[i] < 1 || d.Z[i] > 100 || !(d.A[i] > 0.5 && d.A[i] < 300.0) ||
                !(d.mass_fraction[i] >= 0.0 && std::isfinite(d.mass_fraction[i])))
                return fail(c, OCMC_ERR_ARG, "material " + std::to_string(m) + ": bad element");
            o.Z[i] = d.Z[i];
            o.A[i] = d.A[i];
            o.w[i] = d.mass_fraction[i];
            ws += d.mass_fraction[i];
        }
        if (!(ws > 0.0)) return fail(c, OCMC_ERR_ARG, "material " + std::to_string(m) + ": mass fractions sum to 0");
        o.I_eV = d.I_eV;
        o.rho0 = d.density;
    }
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    if (c->last_stream || c->ran) cudaDeviceSynchronize();
    c->mats = mats;
    c->have_phantom = false;       // the phantom's material indices refer to the old set
    c->tables_valid = c->mat_tables_valid = false;
    return OCMC_OK;
}

ocmc_status ocmc_create_phantom(ocmc_ctx* c, int nx, int ny, int nz, const float* density, const uint8_t* material,
                                float dx, float dy, float dz)
{
    if (!c) return fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (!density || !material) return fail(c, OCMC_ERR_ARG, "density/material is NULL");
    if (nx < 1 || ny < 1 || nz < 1 || nx > MAX_DIM || ny > MAX_DIM || nz > MAX_DIM)
        return fail(c, OCMC_ERR_ARG, "grid dimensions must be in [1, 1024]");
    if (!(dx > 0.f && dy > 0.f && dz > 0.f && dx < 100.f && dy < 100.f && dz < 100.f))
        return fail(c, OCMC_ERR_ARG, "voxel sizes must be in (0, 100) cm");
    long long n = (long long)nx * ny * nz;
    const int nd = (int)c->mats.size();
    bool used[MAX_MAT] = {false};
    for (long long v = 0; v < n; ++v) {
        if (material[v] >= nd)
            return fail(c, OCMC_ERR_ARG, "material index must be below the number of defined materials (" +
                                             std::to_string(nd) + ")");
        if (!(density[v] >= 0.f && density[v] <= 30.f)) return fail(c, OCMC_ERR_ARG, "density must be in [0, 30] g/cm^3");
        used[material[v]] = true;
    }
    // staging: every defined material when they fit in a block's shared memory, else the
    // phantom's own materials in increasing index order (the uploaded indices are compacted)
    std::vector<int> slot(nd, -1);
    std::vector<MatDef> staged;
    if (nd <= MAX_STAGED) {
        for (int m = 0; m < nd; ++m) slot[m] = m;
        staged = c->mats;
    } else {
        for (int m = 0; m < nd; ++m)
            if (used[m]) {
                slot[m] = (int)staged.size();
                staged.push_back(c->mats[m]);
            }
        if ((int)staged.size() > MAX_STAGED)
            return fail(c, OCMC_ERR_ARG, "a phantom may use at most " + std::to_string(MAX_STAGED) +
                                             " distinct materials (their tables share a block's shared memory)");
    }
    std::vector<uint8_t> remapped;
    if (nd > MAX_STAGED) {
        remapped.resize((size_t)n);
        for (long long v = 0; v < n; ++v) remapped[v] = (uint8_t)slot[material[v]];
        material = remapped.data();
    }
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    if (c->last_stream || c->ran) cudaDeviceSynchronize();
    if (n != c->nvox) {
        CK(dalloc(&c->d_density, n), "phantom allocation");
        CK(dalloc(&c->d_material, n), "phantom allocation");
        CK(dalloc(&c->d_dose, n), "dose allocation");
        CK(dalloc(&c->d_sigma, n), "dose allocation");
        dfree(&c->d_tally);
    }
    c->nx = nx; c->ny = ny; c->nz = nz; c->nvox = n;
    c->dx = dx; c->dy = dy; c->dz = dz;
    CK(cudaMemcpy(c->d_density, density, n * sizeof(float), cudaMemcpyHostToDevice), "phantom upload");
    CK(cudaMemcpy(c->d_material, material, n, cudaMemcpyHostToDevice), "phantom upload");
    if (!same_defs(staged, c->staged)) c->mat_tables_valid = false;   // else only the phantom part is rebuilt
    c->staged = staged;
    c->slot_of = slot;
    c->t.n_mat = (int)staged.size();
    c->have_phantom = true;
    c->tables_valid = false;
    if (c->d_tally && c->tally_B == c->p.n_batches) {
        CK(cudaMemset(c->d_tally, 0, sizeof(long long) * (size_t)c->tally_B * n), "tally reset");
        c->nb.assign(c->tally_B, 0.0);
        c->ran = false;
        CK(cudaMemset(c->d_stats, 0, ST_COUNT * sizeof(unsigned long long)), "stats reset");
        CK(cudaMemset(c->d_err, 0, sizeof(int)), "stats reset");
        return OCMC_OK;
    }
    CK(cudaMemset(c->d_stats, 0, ST_COUNT * sizeof(unsigned long long)), "stats reset");
    CK(cudaMemset(c->d_err, 0, sizeof(int)), "stats reset");
    return ensure_tally(c);
}

ocmc_status ocmc_set_source(ocmc_ctx* c, int particle, int n_bins, const float* edges, const float* weights, float fx,
                            float fy, float ssd, const float iso[3], const float dir[3])
{
    if (!c) return fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (particle != 0 && particle != 1) return fail(c, OCMC_ERR_ARG, "particle must be 0 (photon) or 1 (electron)");
    if (n_bins < 1 || n_bins > MAX_BINS) return fail(c, OCMC_ERR_ARG, "n_bins must be in [1, 256]");
    if (!edges || !weights || !iso || !dir) return fail(c, OCMC_ERR_ARG, "NULL array");
    double W = 0.0;
    for (int i = 0; i < n_bins; ++i) {
        if (!(edges[i] >= 1e-3f && edges[i + 1] <= 30.f && edges[i + 1] >= edges[i]))
            return fail(c, OCMC_ERR_ARG, "bin edges must satisfy 0.001 <= lo <= hi <= 30 MeV");
        if (!(weights[i] >= 0.f && std::isfinite(weights[i]))) return fail(c, OCMC_ERR_ARG, "weights must be >= 0");
        W += weights[i];
    }
    if (!(W > 0.0)) return fail(c, OCMC_ERR_ARG, "weights sum to zero");
    if (!(fx >= 0.f && fy >= 0.f && fx < 1e4f && fy < 1e4f)) return fail(c, OCMC_ERR_ARG, "bad field size");
    if (!std::isfinite(ssd) || std::fabs(ssd) > 1e5f) return fail(c, OCMC_ERR_ARG, "bad ssd");
    double d[3] = {dir[0], dir[1], dir[2]};
    double nd = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(nd > 1e-6) || !std::isfinite(nd)) return fail(c, OCMC_ERR_ARG, "dir must be a non-zero vector");
    for (int k = 0; k < 3; ++k) {
        if (!std::isfinite(iso[k])) return fail(c, OCMC_ERR_ARG, "iso must be finite");
        d[k] /= nd;
    }
    double a[3] = {d[2], 0.0, -d[0]};   // y_hat x dir
    if (std::sqrt(a[0] * a[0] + a[2] * a[2]) < 1e-6) { a[0] = 0.0; a[1] = -d[2]; a[2] = d[1]; }   // x_hat x dir
    double na = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    for (int k = 0; k < 3; ++k) a[k] /= na;
    double b[3] = {d[1] * a[2] - d[2] * a[1], d[2] * a[0] - d[0] * a[2], d[0] * a[1] - d[1] * a[0]};
    c->particle = particle;
    c->n_bins = n_bins;
    c->edges.assign(edges, edges + n_bins + 1);
    c->weights.assign(weights, weights + n_bins);
    c->fx = fx; c->fy = fy; c->ssd = ssd;
    for (int k = 0; k < 3; ++k) {
        c->iso[k] = iso[k];
        c->dir[k] = (float)d[k];
        c->e1[k] = (float)a[k];
        c->e2[k] = (float)b[k];
    }
    c->have_source = true;
    c->src_kind = 0;
    return OCMC_OK;
}

ocmc_status ocmc_set_phase_space(ocmc_ctx* c, const ocmc_ps_particle* records, uint64_t n, int on_device)
{
    if (!c) return fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (!records || n == 0) return fail(c, OCMC_ERR_ARG, "need at least one record");
    static_assert(sizeof(ocmc_ps_particle) == sizeof(PsRec), "record layout");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    if (n > c->ps_cap) {
        cudaDeviceSynchronize();
        CK(dalloc(&c->d_ps, (size_t)n), "phase-space allocation");
        c->ps_cap = n;
    }
    CK(cudaMemcpy(c->d_ps, records, sizeof(PsRec) * (size_t)n, on_device ? cudaMemcpyDeviceToDevice
                                                                           : cudaMemcpyHostToDevice),
       "phase-space copy");
    CK(launch_ps_validate(c->d_ps, n, c->d_sum, nullptr), "phase-space check");
    unsigned long long bad = 0;
    CK(cudaMemcpy(&bad, c->d_sum, sizeof(bad), cudaMemcpyDeviceToHost), "phase-space check");
    if (bad) {
        if (c->src_kind == 1) c->have_source = false;
        return fail(c, OCMC_ERR_ARG, std::to_string(bad) + " phase-space record(s) invalid (type 0/1/2, 0 < E < "
                                     "1e4 MeV, finite position, non-zero direction)");
    }
    c->ps_n = n;
    c->src_kind = 1;
    c->have_source = true;
    return OCMC_OK;
}

ocmc_status ocmc_load_phase_space(ocmc_ctx* c, const char* path)
{
    if (!c) return fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (!path) return fail(c, OCMC_ERR_ARG, "path is NULL");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(c, OCMC_ERR_ARG, std::string("cannot open ") + path);
    unsigned char hdr[16];
    if (std::fread(hdr, 1, 16, f) != 16 || std::memcmp(hdr, "OCMCPS01", 8) != 0) {
        std::fclose(f);
        return fail(c, OCMC_ERR_ARG, "not a phase-space file (magic OCMCPS01)");
    }
    uint64_t n = 0;
    for (int i = 0; i < 8; ++i) n |= (uint64_t)hdr[8 + i] << (8 * i);      // little endian
    if (n == 0 || n > (1ull << 36)) {
        std::fclose(f);
        return fail(c, OCMC_ERR_ARG, "bad record count");
    }
    std::vector<ocmc_ps_particle> recs;
    try {
        recs.resize((size_t)n);
    } catch (...) {
        std::fclose(f);
        return fail(c, OCMC_ERR_OOM, "host memory for the phase space");
    }
    size_t got = std::fread(recs.data(), sizeof(ocmc_ps_particle), (size_t)n, f);
    std::fclose(f);
    if (got != (size_t)n) return fail(c, OCMC_ERR_ARG, "phase-space file shorter than its record count");
    return ocmc_set_phase_space(c, recs.data(), n, 0);
}

ocmc_status ocmc_run_range(ocmc_ctx* c, uint64_t first, uint64_t count, uint64_t n_total, uint64_t seed,
                           void* stream)
{
    if (!c) return fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (!c->have_phantom) return fail(c, OCMC_ERR_STATE, "no phantom (call ocmc_create_phantom)");
    if (!c->have_source) return fail(c, OCMC_ERR_STATE, "no source (call ocmc_set_source)");
    if (count == 0 || n_total == 0 || first + count > n_total || first + count < first)
        return fail(c, OCMC_ERR_ARG, "need 0 < count and first + count <= n_total");
    if ((c->p.flags & FLAG_CROSS_VOXELS) && c->src_kind == 1)
        return fail(c, OCMC_ERR_ARG, "voxel-crossing electron steps need the analytic source (not a phase space)");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    ocmc_status st = ensure_tally(c);
    if (st != OCMC_OK) return st;
    st = ensure_tables(c, s);
    if (st != OCMC_OK) return st;
    int threads, blocks, cap, nreg;
    launch_shape(c, &threads, &blocks, &cap, &nreg);
    const int nstk = c->p.e_class_split > 0.f ? 3 : 2;
    size_t need = (size_t)blocks * (threads / 32) * nstk * cap;
    if (need > c->stack_records) {
        if (c->ran || c->last_stream) cudaDeviceSynchronize();
        CK(dalloc(&c->d_stacks, need), "stack allocation");
        c->stack_records = need;
    }
    TransportArgs a;
    fill_args(c, a);
    if (c->src_kind == 0) stratify(c, n_total, a.src);
    a.first = first;
    a.count = count;
    a.n_total = n_total;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.stacks = c->d_stacks;
    a.cap = cap;
    a.nstk = nstk;
    a.e_split = c->p.e_class_split;
    a.switch_high = c->p.switch_high ? c->p.switch_high : cap - cap / 16;
    a.switch_low = c->p.switch_low ? c->p.switch_low : 8;
    a.refill_min = c->p.refill_min ? c->p.refill_min : 6;
    CK(cudaEventRecord(c->ev0, s), "event");
    // A range is transported in launches of at most RUN_CHUNK histories: on GB300 a single launch
    // of 1e9 histories ran 15 % slower per history than ten launches of 1e8 (measured). Ranges
    // compose, so the tally is the same bit for bit.
    for (uint64_t done = 0; done < count; done += RUN_CHUNK) {
        a.first = first + done;
        a.count = std::min<uint64_t>(RUN_CHUNK, count - done);
        CK(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), s), "counter reset");
        CK(launch_transport(a, blocks, threads, transport_smem_bytes(c->t.n_mat), s, nreg), "transport launch");
    }
    CK(cudaEventRecord(c->ev1, s), "event");
    c->timed = true;
    c->last_stream = s;
    c->ran = true;
    add_histories(c, first, count);
    return OCMC_OK;
}

ocmc_status ocmc_run(ocmc_ctx* c, uint64_t n, uint64_t seed, void* stream)
{
    if (!c) return fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (n == 0) return fail(c, OCMC_ERR_ARG, "n_histories must be > 0");
    return ocmc_run_range(c, 0, n, n, seed, stream);
}

static ocmc_status check_err_flag(ocmc_ctx* c)
{
    int e = 0;
    CK(cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error flag");
    if (e & ERR_PHANTOM) return fail(c, OCMC_ERR_ARG, "phantom contains invalid values");
    if (e & ERR_BOUNDS) return fail(c, OCMC_ERR_BOUNDS, "a bounds check failed (checks build); the access was skipped");
    if (e & ERR_OVERFLOW) return fail(c, OCMC_ERR_OVERFLOW, "a secondary stack overflowed; particles were dropped");
    if (e & ERR_LIMIT) return fail(c, OCMC_ERR_TIMEOUT, "a particle hit the step or sampling iteration limit");
    return OCMC_OK;
}

ocmc_status ocmc_get_dose(ocmc_ctx* c, float* dose, float* sigma, int on_device)
{
    if (!c || !dose) return fail(c, OCMC_ERR_ARG, "NULL argument");
    if (!c->have_phantom || !c->d_tally) return fail(c, OCMC_ERR_STATE, "no phantom/tally");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    double n = 0.0;
    for (double v : c->nb) n += v;
    if (!(n > 0.0)) return fail(c, OCMC_ERR_STATE, "no histories have been run");
    cudaStream_t s = c->last_stream;
    if (c->invnb_cap < c->tally_B) {
        CK(dalloc(&c->d_invnb, c->tally_B), "allocation");
        c->invnb_cap = c->tally_B;
    }
    std::vector<float> inv(c->tally_B);
    for (int b = 0; b < c->tally_B; ++b) inv[b] = c->nb[b] > 0 ? (float)(n / c->nb[b]) : 0.f;
    CK(cudaMemcpyAsync(c->d_invnb, inv.data(), sizeof(float) * c->tally_B, cudaMemcpyHostToDevice, s), "upload");
    // device outputs are written in place; host outputs go through the context's buffers
    float* dd = on_device ? dose : c->d_dose;
    float* ds = sigma ? (on_device ? sigma : c->d_sigma) : nullptr;
    CK(launch_finalize(c->d_tally, c->d_density, c->tally_B, c->nvox, (double)c->dx * c->dy * c->dz, c->d_invnb,
                       1.0 / n, dd, ds, s),
       "finalize launch");
    if (!on_device) {
        CK(cudaMemcpyAsync(dose, c->d_dose, sizeof(float) * c->nvox, cudaMemcpyDeviceToHost, s), "dose copy");
        if (sigma) CK(cudaMemcpyAsync(sigma, c->d_sigma, sizeof(float) * c->nvox, cudaMemcpyDeviceToHost, s), "sigma copy");
    }
    CK(cudaStreamSynchronize(s), "synchronize");
    return check_err_flag(c);
}

ocmc_status ocmc_get_raw_tally(ocmc_ctx* c, int64_t* out, int on_device)
{
    if (!c || !out) return fail(c, OCMC_ERR_ARG, "NULL argument");
    if (!c->d_tally) return fail(c, OCMC_ERR_STATE, "no tally");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(c->last_stream), "synchronize");
    CK(cudaMemcpy(out, c->d_tally, sizeof(long long) * (size_t)c->tally_B * c->nvox,
                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost),
       "tally copy");
    return check_err_flag(c);
}

ocmc_status ocmc_add_raw_tally(ocmc_ctx* c, const int64_t* in, int on_device, uint64_t first, uint64_t count)
{
    if (!c || !in) return fail(c, OCMC_ERR_ARG, "NULL argument");
    if (!c->have_phantom) return fail(c, OCMC_ERR_STATE, "no phantom");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    ocmc_status st = ensure_tally(c);
    if (st != OCMC_OK) return st;
    long long n = (long long)c->tally_B * c->nvox;
    const long long* src = reinterpret_cast<const long long*>(in);
    long long* tmp = nullptr;
    if (!on_device) {
        CK(cudaMalloc(&tmp, sizeof(long long) * n), "allocation");
        cudaError_t e = cudaMemcpy(tmp, in, sizeof(long long) * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(tmp); return cuda_fail(c, e, "tally upload"); }
        src = tmp;
    }
    cudaError_t e = launch_add_tally(c->d_tally, src, n, c->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->last_stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "tally add");
    add_histories(c, first, count);
    c->ran = true;
    return OCMC_OK;
}

ocmc_status ocmc_reset_tally(ocmc_ctx* c)
{
    if (!c) return fail(c, OCMC_ERR_ARG, "ctx is NULL");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    if (c->last_stream || c->ran) CK(cudaStreamSynchronize(c->last_stream), "synchronize");
    if (c->d_tally) CK(cudaMemset(c->d_tally, 0, sizeof(long long) * (size_t)c->tally_B * c->nvox), "tally reset");
    c->nb.assign(c->tally_B, 0.0);
    CK(cudaMemset(c->d_stats, 0, ST_COUNT * sizeof(unsigned long long)), "stats reset");
    CK(cudaMemset(c->d_err, 0, sizeof(int)), "stats reset");
    c->ran = false;
    c->timed = false;
    return OCMC_OK;
}

ocmc_status ocmc_get_stats(ocmc_ctx* c, ocmc_stats* out)
{
    if (!c || !out) return fail(c, OCMC_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(c->last_stream), "synchronize");
    unsigned long long st[ST_COUNT];
    CK(cudaMemcpy(st, c->d_stats, sizeof(st), cudaMemcpyDeviceToHost), "stats copy");
    memset(out, 0, sizeof(*out));
    const double S = 1.0 / 268435456.0;
    out->histories = st[ST_HISTORIES];
    out->photon_flights = st[ST_LANES_PHOTON];
    out->fictitious = st[ST_FICT];
    out->compton = st[ST_COMPTON];
    out->photo = st[ST_PHOTO];
    out->pair = st[ST_PAIR];
    out->electron_steps = st[ST_LANES_CHARGED] - st[ST_GEO];
    out->moller = st[ST_MOLLER];
    out->brems = st[ST_BREMS];
    out->hard_fictitious = st[ST_HARD_FICT];
    out->annihilations = st[ST_ANNIH];
    out->escaped = st[ST_ESCAPED];
    out->missed = st[ST_MISSED];
    out->geo_crossings = st[ST_GEO];
    out->majorant_violations = st[ST_VIOL];
    out->dropped = st[ST_DROPPED];
    out->transmitted = st[ST_TRANSMITTED];
    out->warp_iterations = st[ST_WARP_ITERS];
    out->lane_steps = st[ST_LANES_PHOTON] + st[ST_LANES_CHARGED];
    out->e_in = st[ST_E_IN] * S;
    out->e_esc = st[ST_E_ESC] * S;
    out->e_miss = st[ST_E_MISS] * S;
    out->e_killed = st[ST_E_KILLED] * S;
    out->e_trans = st[ST_E_TRANS] * S;
    out->e_dropped = st[ST_E_DROPPED] * S;
    out->warp_ms = st[ST_WARP_NS] * 1e-6;
    out->warps = st[ST_WARPS];
    out->tail_warp_ms = st[ST_TAIL_NS] * 1e-6;
    if (st[ST_T_END]) {
        const unsigned long long t0 = ~st[ST_T_START_INV], ts = ~st[ST_T_SRC_INV];
        out->span_ms = (st[ST_T_END] - t0) * 1e-6;
        out->tail_span_ms = (st[ST_T_END] - ts) * 1e-6;
    }
    out->pair_mass = 2.0 * MC2 * (double)st[ST_PAIR];
    out->annih_mass = 2.0 * MC2 * (double)st[ST_ANNIH];
    if (c->d_tally) {
        CK(launch_sum_tally(c->d_tally, (long long)c->tally_B * c->nvox, c->d_sum, c->last_stream), "tally sum");
        unsigned long long sum = 0;
        CK(cudaMemcpy(&sum, c->d_sum, sizeof(sum), cudaMemcpyDeviceToHost), "tally sum");
        out->e_dep = (double)(long long)sum * S;
    }
    if (c->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) out->last_run_ms = ms;
    }
    return OCMC_OK;
}

ocmc_status ocmc_get_shape(ocmc_ctx* c, int64_t* nvox, int32_t* nb)
{
    if (!c) return fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (nvox) *nvox = c->nvox;
    if (nb) *nb = c->p.n_batches;
    return OCMC_OK;
}

const char* ocmc_last_error(ocmc_ctx* c) { return c ? c->err.c_str() : g_init_err.c_str(); }

void ocmc_destroy(ocmc_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    dfree(&c->d_density); dfree(&c->d_material); dfree(&c->d_tally); dfree(&c->d_stats);
    dfree(&c->d_counter); dfree(&c->d_sum); dfree(&c->d_err); dfree(&c->d_stacks); dfree(&c->d_dose);
    dfree(&c->d_sigma); dfree(&c->d_invnb);
    dfree(&c->t.ph); dfree(&c->t.el); dfree(&c->t.el2); dfree(&c->t.phmaj); dfree(&c->t.elmaj); dfree(&c->t.rinv); dfree(&c->t.msA);
    dfree(&c->t.rmeta); dfree(&c->t.msc); dfree(&c->t.scratch); dfree(&c->t.rho_max);
    dfree(&c->d_bl); dfree(&c->d_bl_prefix); dfree(&c->d_bl_offs); dfree(&c->d_bl_caps); dfree(&c->d_bl_nnz);
    dfree(&c->d_bl_over); dfree(&c->d_bl_keys); dfree(&c->d_bl_vals); dfree(&c->d_dense); dfree(&c->d_chunks);
    dfree(&c->d_oidx); dfree(&c->d_odose); dfree(&c->d_oraw); dfree(&c->d_ps);
    if (c->bl_exec) cudaGraphExecDestroy(c->bl_exec);
    if (c->bl_capture) cudaStreamDestroy(c->bl_capture);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

// ---- test access ------------------------------------------------------------------------------
ocmc_status ocmc_test_philox(int device, uint32_t key0, uint32_t key1, uint32_t c1, uint32_t c2, uint32_t c3,
                             uint32_t first_block, uint32_t n_blocks, uint32_t* out)
{
    ocmc_ctx* c = nullptr;
    if (!out || n_blocks == 0) return fail(nullptr, OCMC_ERR_ARG, "bad arguments");
    CK(cudaSetDevice(device), "cudaSetDevice");
    uint32_t* d = nullptr;
    CK(cudaMalloc(&d, sizeof(uint32_t) * 4 * (size_t)n_blocks), "allocation");
    cudaError_t e = launch_test_philox(key0, key1, c1, c2, c3, first_block, n_blocks, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(uint32_t) * 4 * (size_t)n_blocks, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "philox test");
    return OCMC_OK;
}

ocmc_status ocmc_test_rotate(int device, const float* dir, const float* mu, const float* xi, int n, float* out)
{
    ocmc_ctx* c = nullptr;
    if (!dir || !mu || !xi || !out || n <= 0) return fail(nullptr, OCMC_ERR_ARG, "bad arguments");
    CK(cudaSetDevice(device), "cudaSetDevice");
    float* d = nullptr;
    const size_t nb = sizeof(float) * (size_t)n;
    CK(cudaMalloc(&d, 8 * nb), "allocation");   // dir (3n), mu (n), xi (n), out (3n)
    cudaError_t e = cudaMemcpy(d, dir, 3 * nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + 3 * (size_t)n, mu, nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + 4 * (size_t)n, xi, nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_test_rotate(d, d + 3 * (size_t)n, d + 4 * (size_t)n, n, d + 5 * (size_t)n, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d + 5 * (size_t)n, 3 * nb, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "rotation test");
    return OCMC_OK;
}

ocmc_status ocmc_test_source(ocmc_ctx* c, uint64_t n_total, uint64_t first, uint64_t count, uint64_t seed, float* out)
{
    if (!c || !out || count == 0 || first + count > n_total) return fail(c, OCMC_ERR_ARG, "bad arguments");
    if (!c->have_phantom || !c->have_source) return fail(c, OCMC_ERR_STATE, "need phantom and source");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    TransportArgs a;
    fill_args(c, a);
    if (c->src_kind == 0) stratify(c, n_total, a.src);
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    float* d = nullptr;
    CK(cudaMalloc(&d, sizeof(float) * 8 * count), "allocation");
    cudaError_t e = launch_test_source(a, n_total, first, count, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(float) * 8 * count, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(c, e, "source test");
    return OCMC_OK;
}

ocmc_status ocmc_test_sample(ocmc_ctx* c, int kind, int m, float E, float aux, uint64_t n, uint64_t seed, float* out)
{
    if (!c || !out || n == 0 || kind < 0 || kind > 3 || m < 0 || m >= (int)c->slot_of.size() || !(E > 0.f))
        return fail(c, OCMC_ERR_ARG, "bad arguments");
    if (c->slot_of[m] < 0) return fail(c, OCMC_ERR_ARG, "material not in the phantom's tables");
    m = c->slot_of[m];
    if (!c->have_phantom) return fail(c, OCMC_ERR_STATE, "need a phantom");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    ocmc_status st = ensure_tables(c, nullptr);
    if (st != OCMC_OK) return st;
    TransportArgs a;
    fill_args(c, a);
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    float* d = nullptr;
    CK(cudaMalloc(&d, sizeof(float) * n), "allocation");
    cudaError_t e = launch_test_sample(a, kind, m, E, aux, n, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(float) * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(c, e, "sample test");
    return OCMC_OK;
}

ocmc_status ocmc_test_tables(ocmc_ctx* c, int m, const float* E, int n, float* out)
{
    if (!c || !E || !out || n <= 0 || m < 0 || m >= (int)c->slot_of.size()) return fail(c, OCMC_ERR_ARG, "bad arguments");
    if (c->slot_of[m] < 0) return fail(c, OCMC_ERR_ARG, "material not in the phantom's tables");
    m = c->slot_of[m];
    if (!c->have_phantom) return fail(c, OCMC_ERR_STATE, "need a phantom");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    ocmc_status st = ensure_tables(c, nullptr);
    if (st != OCMC_OK) return st;
    TransportArgs a;
    fill_args(c, a);
    float *dE = nullptr, *d = nullptr;
    CK(cudaMalloc(&dE, sizeof(float) * n), "allocation");
    cudaError_t e = cudaMalloc(&d, sizeof(float) * 8 * n);
    if (e == cudaSuccess) e = cudaMemcpy(dE, E, sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_test_tables(a, m, dE, n, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(float) * 8 * n, cudaMemcpyDeviceToHost);
    cudaFree(dE);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(c, e, "table test");
    return OCMC_OK;
}

ocmc_status ocmc_test_csda(ocmc_ctx* c, int m, const float* T, const float* X, int n, float* out)
{
    if (!c || !T || !X || !out || n <= 0 || m < 0 || m >= (int)c->slot_of.size()) return fail(c, OCMC_ERR_ARG, "bad arguments");
    if (c->slot_of[m] < 0) return fail(c, OCMC_ERR_ARG, "material not in the phantom's tables");
    m = c->slot_of[m];
    if (!c->have_phantom) return fail(c, OCMC_ERR_STATE, "need a phantom");
    CK(cudaSetDevice(c->device), "cudaSetDevice");
    ocmc_status st = ensure_tables(c, nullptr);
    if (st != OCMC_OK) return st;
    TransportArgs a;
    fill_args(c, a);
    float *dT = nullptr, *dX = nullptr, *d = nullptr;
    cudaError_t e = cudaMalloc(&dT, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dX, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dT, T, sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dX, X, sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_test_csda(a, m, dT, dX, n, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(float) * n, cudaMemcpyDeviceToHost);
    cudaFree(dT);
    cudaFree(dX);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(c, e, "csda test");
    return OCMC_OK;
}

}  // extern "C"
