// ocmc_noalloc.cu -- allocation-free transport entry point.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator (which must own every device
// allocation), real-time or certified treatment-planning hosts that forbid
// allocation after start-up, and plug-ins that get only device pointers from
// their host. ocmc_run_noalloc serves them: the caller passes the phantom on the
// device and the tally to add into, and all scratch memory the transport needs
// (physics tables, per-warp secondary stacks, the history counter, statistics
// and the error flag) lives in one file-scope static device array of fixed size.
//
// The array is created when the library is loaded on a device and stays until
// the process exits. Every call shares it and it keeps the last call's contents:
// each call rebuilds the tables and clears the counter, statistics and error
// flag itself. Calls that overlap on the GPU (on different streams, or from
// different host threads) race on the array and give wrong results; serialise
// them. The first call on a device looks up the array's device address (with
// that device current) and caches it; make that first call before any stream
// capture. Every call waits for its stream before it returns (it reads the
// error flag back), and it leaves the caller's current device as it found it.
#include "ocmc.h"
#include "ocmc_internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

using namespace ocmc;

namespace {

constexpr size_t NOALLOC_BYTES = OCMC_NOALLOC_SCRATCH_BYTES;
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_CAP = 256;        // records per stack (two or three stacks per warp)
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_scratch[NOALLOC_BYTES];

std::mutex g_mutex;
void* g_scratch_dev[MAX_DEVICES] = {};

struct Msg {
    char* buf;
    size_t len;
    ocmc_status fail(ocmc_status s, const char* msg) const
    {
        if (buf && len) std::snprintf(buf, len, "%s", msg);
        return s;
    }
    ocmc_status cuda(cudaError_t e, const char* where) const
    {
        if (buf && len) std::snprintf(buf, len, "%s: %s", where, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? OCMC_ERR_OOM : OCMC_ERR_CUDA;
    }
};

// Host code may not use g_scratch's name as a device address; look the address up
// once per device with that device current.
cudaError_t scratch_address(int device, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[device] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_dev[device]);
    return cudaSuccess;
}

// Bump allocator over the static array (256-byte aligned pieces).
struct Carver {
    unsigned char* base;
    size_t used;
    template <class T>
    T* take(size_t n)
    {
        size_t bytes = (n * sizeof(T) + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return p;
    }
};

// Puts the caller's current device back when the call returns.
struct DeviceGuard {
    int prev = -1;
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" ocmc_status ocmc_run_noalloc(int device, int nx, int ny, int nz, const float* density_dev,
                                        const uint8_t* material_dev, float dx, float dy, float dz, int particle,
                                        int n_bins, const float* edges, const float* weights, float field_x,
                                        float field_y, float ssd, const float iso[3], const float dir[3],
                                        const ocmc_params* params, uint64_t first, uint64_t count, uint64_t n_total,
                                        uint64_t seed, int64_t* tally_dev, void* cuda_stream, char* err_msg,
                                        size_t err_len)
{
    const Msg M{err_msg, err_len};
    if (err_msg && err_len) err_msg[0] = 0;
    ocmc_params p;
    ocmc_default_params(&p);
    if (params) p = *params;
    if (!density_dev || !material_dev || !tally_dev || !edges || !weights || !iso || !dir)
        return M.fail(OCMC_ERR_ARG, "NULL argument");
    if (device < 0 || device >= MAX_DEVICES) return M.fail(OCMC_ERR_ARG, "device index out of range");
    if (nx < 1 || ny < 1 || nz < 1 || nx > MAX_DIM || ny > MAX_DIM || nz > MAX_DIM)
        return M.fail(OCMC_ERR_ARG, "grid dimensions must be in [1, 1024]");
    if (!(dx > 0.f && dy > 0.f && dz > 0.f && dx < 100.f && dy < 100.f && dz < 100.f))
        return M.fail(OCMC_ERR_ARG, "voxel sizes must be in (0, 100) cm");
    if (particle != 0 && particle != 1) return M.fail(OCMC_ERR_ARG, "particle must be 0 or 1");
    if (n_bins < 1 || n_bins > MAX_BINS) return M.fail(OCMC_ERR_ARG, "n_bins must be in [1, 256]");
    if (count == 0 || n_total == 0 || first + count > n_total || first + count < first)
        return M.fail(OCMC_ERR_ARG, "need 0 < count and first + count <= n_total");
    if (!(p.e_abs_e >= 1e-3f && p.e_abs_e <= 10.f && p.e_abs_g >= 1e-3f && p.e_abs_g <= 10.f &&
          p.w_cc >= 1e-3f && p.w_cc <= 10.f && p.w_cb >= 1e-3f && p.w_cb <= 10.f && p.d_maxs > 0.f &&
          p.f_maxe > 0.f && p.f_maxe <= 0.5f && p.s_min >= 0.f && p.s_min <= 0.01f && p.n_batches >= 1 &&
          p.n_batches <= 1000 && p.flags >= 0 && p.flags <= 15))
        return M.fail(OCMC_ERR_ARG, "invalid transport parameters");
    if ((p.block_threads != 0 && (p.block_threads < 32 || p.block_threads > 1024 || p.block_threads % 32)) ||
        p.blocks_per_sm < 0 || p.blocks_per_sm > 32 ||
        (p.stack_capacity != 0 && (p.stack_capacity < 64 || p.stack_capacity > (1 << 20))) || p.switch_high < 0 ||
        p.switch_low < 0 || p.switch_low > 32 || p.refill_min < 0 || p.refill_min > 32 ||
        (p.max_registers != 0 && !transport_nreg_supported(p.max_registers)) ||
        !(p.e_class_split >= 0.f && p.e_class_split <= 30.f))
        return M.fail(OCMC_ERR_ARG, "invalid execution parameters");
    double W = 0.0;
    for (int i = 0; i < n_bins; ++i) {
        if (!(edges[i] >= 1e-3f && edges[i + 1] <= 30.f && edges[i + 1] >= edges[i]))
            return M.fail(OCMC_ERR_ARG, "bin edges must satisfy 0.001 <= lo <= hi <= 30 MeV");
        if (!(weights[i] >= 0.f)) return M.fail(OCMC_ERR_ARG, "weights must be >= 0");
        W += weights[i];
    }
    if (!(W > 0.0)) return M.fail(OCMC_ERR_ARG, "weights sum to zero");
    double d[3] = {dir[0], dir[1], dir[2]};
    double nd = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(nd > 1e-6) || !std::isfinite(nd)) return M.fail(OCMC_ERR_ARG, "dir must be a non-zero vector");

    DeviceGuard guard;
    cudaError_t e = cudaGetDevice(&guard.prev);
    if (e != cudaSuccess) return M.cuda(e, "cudaGetDevice");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return M.cuda(e, "cudaSetDevice");
    unsigned char* base = nullptr;
    e = scratch_address(device, &base);
    if (e != cudaSuccess) return M.cuda(e, "cudaGetSymbolAddress");

    // scratch layout: tables, then run counters, then the per-warp stacks
    Carver cv{base, 0};
    Tables t;
    t.n_mat = NMAT_DEFAULT;                    // the built-in materials: water, cortical bone, lung
    t.ph = cv.take<float4>(NMAT_DEFAULT * NE);
    t.el = cv.take<float4>(NMAT_DEFAULT * NE);
    t.el2 = cv.take<float2>(NMAT_DEFAULT * NE);
    t.phmaj = cv.take<float>(NE);
    t.elmaj = cv.take<float>(NE);
    t.rinv = cv.take<float>(NMAT_DEFAULT * NR);
    t.msA = cv.take<float>(NG);
    t.rmeta = cv.take<float>(2 * NMAT_DEFAULT);
    t.msc = cv.take<float>(2 * NMAT_DEFAULT);
    t.scratch = cv.take<double>(NMAT_DEFAULT * NE);
    t.rho_max = cv.take<unsigned int>(NMAT_DEFAULT);
    t.mats = cv.take<MatDef>(NMAT_DEFAULT);
    MatDef defs[NMAT_DEFAULT];
    material_defs(defs);
    unsigned long long* stats = cv.take<unsigned long long>(ST_COUNT);
    unsigned long long* counter = cv.take<unsigned long long>(1);
    int* err = cv.take<int>(1);
    size_t counters_end = cv.used;

    int threads = p.block_threads ? p.block_threads : NOALLOC_THREADS;
    int cap = p.stack_capacity ? p.stack_capacity : NOALLOC_CAP;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return M.cuda(e, "device attribute");
    size_t smem = transport_smem_bytes(NMAT_DEFAULT);
    const int nreg = p.max_registers ? p.max_registers : 80;
    int bps = p.blocks_per_sm ? p.blocks_per_sm : transport_max_blocks_per_sm(threads, smem, nreg);
    if (bps < 1) bps = 1;
    const int nstk = p.e_class_split > 0.f ? 3 : 2;
    size_t per_block = (size_t)(threads / 32) * nstk * cap * sizeof(PRec);
    size_t room = NOALLOC_BYTES - cv.used;
    long long blocks = (long long)sms * bps;
    if (!p.blocks_per_sm && (size_t)blocks * per_block > room) blocks = (long long)(room / per_block);
    if (blocks < 1 || (size_t)blocks * per_block > room)
        return M.fail(OCMC_ERR_ARG, "launch shape needs more secondary-stack scratch than the 64 MiB static array "
                                   "(lower stack_capacity, block_threads or blocks_per_sm)");
    PRec* stacks = cv.take<PRec>((size_t)blocks * (threads / 32) * nstk * cap);

    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    size_t stats_off = (size_t)(reinterpret_cast<unsigned char*>(stats) - base);
    e = cudaMemsetAsync(stats, 0, counters_end - stats_off, s);   // counter, statistics, error flag start at 0
    if (e != cudaSuccess) return M.cuda(e, "clearing counters");
    PhysParams pp{p.e_abs_e, p.e_abs_g, p.w_cc, p.w_cb, p.d_maxs, p.f_maxe, p.s_min, p.flags, p.n_batches};
    long long nvox = (long long)nx * ny * nz;
    e = build_tables(t, pp, density_dev, material_dev, nvox, err, defs, s);
    if (e != cudaSuccess) return M.cuda(e, "table build");
    // The phantom lives on the device, so its values are checked there (by the table build's
    // scan); the transport kernel indexes tables by material, so it must not start on a bad one.
    int flag = 0;
    e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return M.cuda(e, "table build");
    if (flag & ERR_PHANTOM)
        return M.fail(OCMC_ERR_ARG, "phantom contains invalid values (material >= 3 or density outside [0, 30])");

    TransportArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nx = nx; a.ny = ny; a.nz = nz;
    a.dx = dx; a.dy = dy; a.dz = dz;
    a.density = density_dev;
    a.material = material_dev;
    a.nvox = nvox;
    a.t = t;
    a.pp = pp;
    a.first = first;
    a.count = count;
    a.n_total = n_total;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.tally = reinterpret_cast<unsigned long long*>(tally_dev);
    a.stacks = stacks;
    a.cap = cap;
    a.nstk = nstk;
    a.e_split = p.e_class_split;
    a.switch_high = p.switch_high ? p.switch_high : cap - cap / 16;   // below the capacity: switching stays on
    a.switch_low = p.switch_low ? p.switch_low : 8;
    a.refill_min = p.refill_min ? p.refill_min : 6;
    a.hist_counter = counter;
    a.stats = stats;
    a.err = err;
    // source: beam frame and energy-bin stratification (same definitions as ocmc_set_source/ocmc_run)
    for (int k = 0; k < 3; ++k) d[k] /= nd;
    double ax[3] = {d[2], 0.0, -d[0]};
    if (std::sqrt(ax[0] * ax[0] + ax[2] * ax[2]) < 1e-6) { ax[0] = 0.0; ax[1] = -d[2]; ax[2] = d[1]; }
    double na = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
    for (int k = 0; k < 3; ++k) ax[k] /= na;
    double bx[3] = {d[1] * ax[2] - d[2] * ax[1], d[2] * ax[0] - d[0] * ax[2], d[0] * ax[1] - d[1] * ax[0]};
    SourceDev& sd = a.src;
    sd.particle = particle;
    sd.n_bins = n_bins;
    sd.fx = field_x; sd.fy = field_y; sd.ssd = ssd;
    for (int k = 0; k < 3; ++k) {
        sd.iso[k] = iso[k]; sd.dir[k] = (float)d[k]; sd.e1[k] = (float)ax[k]; sd.e2[k] = (float)bx[k];
    }
    for (int i = 0; i < n_bins; ++i) sd.order[i] = i;
    for (int i = 1; i < n_bins; ++i) {
        int v = sd.order[i], j = i - 1;
        while (j >= 0 && (edges[sd.order[j]] < edges[v] || (edges[sd.order[j]] == edges[v] && sd.order[j] > v))) {
            sd.order[j + 1] = sd.order[j];
            --j;
        }
        sd.order[j + 1] = v;
    }
    double Wq = 0.0, cum = 0.0;
    for (int q = 0; q < n_bins; ++q) Wq += (double)weights[sd.order[q]];
    sd.bound[0] = 0;
    for (int q = 1; q < n_bins; ++q) {
        cum += (double)weights[sd.order[q - 1]];
        unsigned long long u = (unsigned long long)std::floor((double)n_total * cum / Wq);
        if (u > n_total) u = n_total;
        if (u < sd.bound[q - 1]) u = sd.bound[q - 1];
        sd.bound[q] = u;
    }
    sd.bound[n_bins] = n_total;
    for (int i = 0; i < n_bins; ++i) { sd.lo[i] = edges[i]; sd.hi[i] = edges[i + 1]; }

    e = launch_transport(a, (int)blocks, threads, smem, s, nreg);
    if (e != cudaSuccess) return M.cuda(e, "transport launch");
    e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return M.cuda(e, "transport");
    if (flag & ERR_PHANTOM) return M.fail(OCMC_ERR_ARG, "phantom contains invalid values");
    if (flag & ERR_BOUNDS) return M.fail(OCMC_ERR_BOUNDS, "a bounds check failed (checks build)");
    if (flag & ERR_OVERFLOW) return M.fail(OCMC_ERR_OVERFLOW, "a secondary stack overflowed; particles were dropped");
    if (flag & ERR_LIMIT) return M.fail(OCMC_ERR_TIMEOUT, "a particle hit the step or sampling iteration limit");
    return OCMC_OK;
}
