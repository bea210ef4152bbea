// ocmc_beamlets.cu -- batched beamlets (one persistent, graph-captured launch over a
// queue of sources with per-beamlet sparse tallies) and the launch-shape autotuner.
#include "ocmc_ctx.h"

#include <algorithm>
#include <cmath>
#include <cstring>

using namespace ocmc;

namespace {

#define BCK(call, where)                                          \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ctx_cuda_fail(c, e_, where); \
    } while (0)

unsigned long long next_pow2(unsigned long long x)
{
    unsigned long long p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <class T>
cudaError_t realloc_dev(T** p, size_t n)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
}

// Per-beamlet device records for the given history counts and table capacities.
ocmc_status upload_beamlets(ocmc_ctx* c, const std::vector<unsigned long long>& counts,
                            const std::vector<unsigned long long>& caps, unsigned long long* total_hist,
                            size_t* total_slots)
{
    const int n = c->bl_n;
    std::vector<BeamletDev> dev(n);
    std::vector<unsigned long long> prefix(n + 1), offs(n);
    std::vector<unsigned int> capv(n);
    unsigned long long off = 0, pre = 0;
    int order[MAX_BL_BINS];
    for (int b = 0; b < n; ++b) {
        const ocmc_beamlet& B = c->bl_list[b];
        BeamletDev& d = dev[b];
        std::memset(&d, 0, sizeof(d));
        d.fx = B.field_x;
        d.fy = B.field_y;
        d.ssd = B.ssd;
        beam_frame(B.dir, d.dir, d.e1, d.e2);
        for (int k = 0; k < 3; ++k) d.iso[k] = B.iso[k];
        d.table_off = off;
        d.cap_mask = (unsigned int)(caps[b] - 1);
        d.n = counts[b];
        stratify_bins(c->bl_edges.data(), c->bl_weights.data(), c->bl_bins, counts[b], order, d.bound);
        prefix[b] = pre;
        offs[b] = off;
        capv[b] = (unsigned int)caps[b];
        pre += counts[b];
        off += caps[b];
    }
    prefix[n] = pre;
    BCK(cudaMemcpy(c->d_bl, dev.data(), sizeof(BeamletDev) * n, cudaMemcpyHostToDevice), "beamlet upload");
    BCK(cudaMemcpy(c->d_bl_prefix, prefix.data(), sizeof(unsigned long long) * (n + 1), cudaMemcpyHostToDevice),
        "beamlet upload");
    BCK(cudaMemcpy(c->d_bl_offs, offs.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice), "upload");
    BCK(cudaMemcpy(c->d_bl_caps, capv.data(), sizeof(unsigned int) * n, cudaMemcpyHostToDevice), "upload");
    if (off > c->bl_slots) {
        BCK(realloc_dev(&c->d_bl_keys, off), "beamlet table allocation");
        BCK(realloc_dev(&c->d_bl_vals, off), "beamlet table allocation");
        c->bl_slots = off;
    }
    *total_hist = pre;
    *total_slots = off;
    return OCMC_OK;
}

// Transport arguments of a beamlet launch (tables cleared by the caller's memsets).
ocmc_status beamlet_args(ocmc_ctx* c, unsigned long long total, uint64_t seed, TransportArgs& a, int* threads,
                         int* blocks, int* nreg)
{
    ctx_fill_args(c, a);
    a.src.particle = c->bl_particle;
    a.src.n_bins = c->bl_bins;
    std::vector<unsigned long long> dummy(c->bl_bins + 1);
    stratify_bins(c->bl_edges.data(), c->bl_weights.data(), c->bl_bins, 1, a.src.order, dummy.data());
    for (int i = 0; i < c->bl_bins; ++i) {
        a.src.lo[i] = c->bl_edges[i];
        a.src.hi[i] = c->bl_edges[i + 1];
    }
    a.first = 0;
    a.count = total;
    a.n_total = total;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.stream_tag = 0;
    a.beamlets = c->d_bl;
    a.bl_prefix = c->d_bl_prefix;
    a.n_beamlets = c->bl_n;
    a.bl_keys = c->d_bl_keys;
    a.bl_vals = c->d_bl_vals;
    a.bl_overflow = c->d_bl_over;
    int cap;
    ctx_launch_shape(c, threads, blocks, &cap, nreg);
    const int nstk = c->p.e_class_split > 0.f ? 3 : 2;
    ocmc_status st = ctx_ensure_stacks(c, (size_t)*blocks * (*threads / 32) * nstk * cap);
    if (st != OCMC_OK) return st;
    a.stacks = c->d_stacks;
    a.cap = cap;
    a.nstk = nstk;
    a.e_split = c->p.e_class_split;
    a.switch_high = c->p.switch_high ? c->p.switch_high : cap - cap / 16;
    a.switch_low = c->p.switch_low ? c->p.switch_low : 8;
    a.refill_min = c->p.refill_min ? c->p.refill_min : 6;
    return OCMC_OK;
}

// Clears the tables, flags and counter, then launches the transport (all on stream s).
cudaError_t enqueue_beamlets(ocmc_ctx* c, const TransportArgs& a, size_t slots, int threads, int blocks, int nreg,
                             cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(c->d_bl_keys, 0xFF, sizeof(unsigned int) * slots, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_bl_vals, 0, sizeof(unsigned long long) * slots, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_bl_over, 0, sizeof(unsigned int) * c->bl_n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), s);
    // a beamlet run replaces its tallies, so its statistics describe that run alone
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * ST_COUNT, s);
    if (e == cudaSuccess) e = launch_transport(a, blocks, threads, transport_smem_bytes(c->t.n_mat), s, nreg);
    return e;
}

ocmc_status read_overflow(ocmc_ctx* c, std::vector<unsigned int>& over)
{
    over.resize(c->bl_n);
    BCK(cudaMemcpy(over.data(), c->d_bl_over, sizeof(unsigned int) * c->bl_n, cudaMemcpyDeviceToHost), "flags");
    return OCMC_OK;
}

// Table sizes from two pilot runs: the distinct-voxel footprint at p2 and p1 = 4 p2
// histories per beamlet, extrapolated to n as a power law (exponent clamped to
// [0.2, 1]), with a 1.2 margin, a load factor of at most BL_LOAD and the global cap.
// Target load factor of a beamlet's table at its estimated footprint: linear probing pays for
// every occupied slot it passes, and on GB300 the 512-beamlet CT run took 219.8 ms at 0.7,
// 183.9 ms at 0.35 and 180.7 ms at 0.175 (measured), at twice and four times the table memory.
constexpr double BL_LOAD = 0.35;

ocmc_status size_tables(ocmc_ctx* c, uint64_t seed, cudaStream_t s)
{
    const int n = c->bl_n;
    const unsigned long long cap_max = next_pow2((unsigned long long)std::ceil(c->nvox / 0.7) + 1);
    std::vector<unsigned long long> p1(n), p2(n), nnz1(n), nnz2(n), caps(n);
    for (int b = 0; b < n; ++b) {
        unsigned long long nb = c->bl_list[b].n_histories;
        p1[b] = std::max<unsigned long long>(std::min<unsigned long long>(nb, 256), nb / 64);
        p2[b] = std::max<unsigned long long>(1, p1[b] / 4);
    }
    unsigned long long saved[ST_COUNT];
    BCK(cudaMemcpy(saved, c->d_stats, sizeof(saved), cudaMemcpyDeviceToHost), "stats");
    for (int pass = 0; pass < 2; ++pass) {
        const std::vector<unsigned long long>& cnt = pass == 0 ? p2 : p1;
        for (int b = 0; b < n; ++b)
            caps[b] = std::min(cap_max, next_pow2(std::max<unsigned long long>(1024, 48 * cnt[b])));
        for (int attempt = 0;; ++attempt) {
            unsigned long long total;
            size_t slots;
            ocmc_status st = upload_beamlets(c, cnt, caps, &total, &slots);
            if (st != OCMC_OK) return st;
            TransportArgs a;
            int threads, blocks, nreg;
            st = beamlet_args(c, total, seed ^ 0x5EEDF00Dull, a, &threads, &blocks, &nreg);
            if (st != OCMC_OK) return st;
            BCK(enqueue_beamlets(c, a, slots, threads, blocks, nreg, s), "pilot launch");
            BCK(cudaStreamSynchronize(s), "pilot");
            std::vector<unsigned int> over;
            st = read_overflow(c, over);
            if (st != OCMC_OK) return st;
            bool any = false;
            for (int b = 0; b < n; ++b)
                if (over[b]) { any = true; caps[b] = std::min(cap_max, caps[b] * 4); }
            if (!any) break;
            if (attempt >= 8) return ctx_fail(c, OCMC_ERR_OVERFLOW, "beamlet pilot tables keep overflowing");
        }
        BCK(launch_bl_count(c->d_bl_keys, c->d_bl_offs, c->d_bl_caps, n, c->d_bl_nnz, s), "footprint count");
        BCK(cudaMemcpy(pass == 0 ? nnz2.data() : nnz1.data(), c->d_bl_nnz, sizeof(unsigned long long) * n,
                       cudaMemcpyDeviceToHost), "footprint count");
    }
    BCK(cudaMemcpy(c->d_stats, saved, sizeof(saved), cudaMemcpyHostToDevice), "stats");
    BCK(cudaMemset(c->d_err, 0, sizeof(int)), "flags");
    const double scale = c->p.beamlet_capacity_scale > 0.f ? c->p.beamlet_capacity_scale : 1.0;
    c->bl_cap.resize(n);
    for (int b = 0; b < n; ++b) {
        double nb = (double)c->bl_list[b].n_histories, a = 1.0;
        if (nnz1[b] > nnz2[b] && nnz2[b] > 0 && p1[b] > p2[b])
            a = std::log((double)nnz1[b] / nnz2[b]) / std::log((double)p1[b] / p2[b]);
        a = std::min(1.0, std::max(0.2, a));
        double est = std::min((double)c->nvox, std::max(1.0, (double)nnz1[b]) * std::pow(nb / p1[b], a)) * 1.2 * scale;
        c->bl_cap[b] = std::min(cap_max, next_pow2(std::max<unsigned long long>(1024, (unsigned long long)(est / BL_LOAD))));
    }
    c->bl_sized = true;
    c->bl_graph_valid = false;
    return OCMC_OK;
}

// Capture {clear tables, clear flags, reset counter, transport} as one CUDA graph.
ocmc_status capture_graph(ocmc_ctx* c, uint64_t seed)
{
    std::vector<unsigned long long> counts(c->bl_n);
    for (int b = 0; b < c->bl_n; ++b) counts[b] = c->bl_list[b].n_histories;
    unsigned long long total;
    size_t slots;
    ocmc_status st = upload_beamlets(c, counts, c->bl_cap, &total, &slots);
    if (st != OCMC_OK) return st;
    TransportArgs a;
    int threads, blocks, nreg;
    st = beamlet_args(c, total, seed, a, &threads, &blocks, &nreg);
    if (st != OCMC_OK) return st;
    if (!c->bl_capture) BCK(cudaStreamCreateWithFlags(&c->bl_capture, cudaStreamNonBlocking), "stream");
    transport_max_blocks_per_sm(threads, transport_smem_bytes(c->t.n_mat), nreg);   // sets the kernels' smem attribute
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(c->bl_capture, cudaStreamCaptureModeRelaxed), "graph capture");
    cudaError_t e = enqueue_beamlets(c, a, slots, threads, blocks, nreg, c->bl_capture);
    cudaError_t e2 = cudaStreamEndCapture(c->bl_capture, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return ctx_cuda_fail(c, e != cudaSuccess ? e : e2, "graph capture");
    }
    if (c->bl_exec) cudaGraphExecDestroy(c->bl_exec);
    c->bl_exec = nullptr;
    e = cudaGraphInstantiate(&c->bl_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return ctx_cuda_fail(c, e, "graph instantiate");
    c->bl_graph_valid = true;
    c->bl_graph_seed = seed;
    return OCMC_OK;
}

}  // namespace

extern "C" {

ocmc_status ocmc_set_beamlets(ocmc_ctx* c, int particle, int n_bins, const float* edges, const float* weights,
                              int n_beamlets, const ocmc_beamlet* list)
{
    if (!c) return ctx_fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (particle != 0 && particle != 1) return ctx_fail(c, OCMC_ERR_ARG, "particle must be 0 or 1");
    if (n_bins < 1 || n_bins > MAX_BL_BINS) return ctx_fail(c, OCMC_ERR_ARG, "n_bins must be in [1, 32]");
    if (n_beamlets < 1 || n_beamlets > 65536) return ctx_fail(c, OCMC_ERR_ARG, "n_beamlets must be in [1, 65536]");
    if (!edges || !weights || !list) return ctx_fail(c, OCMC_ERR_ARG, "NULL array");
    double W = 0.0;
    for (int i = 0; i < n_bins; ++i) {
        if (!(edges[i] >= 1e-3f && edges[i + 1] <= 30.f && edges[i + 1] >= edges[i]))
            return ctx_fail(c, OCMC_ERR_ARG, "bin edges must satisfy 0.001 <= lo <= hi <= 30 MeV");
        if (!(weights[i] >= 0.f && std::isfinite(weights[i]))) return ctx_fail(c, OCMC_ERR_ARG, "weights must be >= 0");
        W += weights[i];
    }
    if (!(W > 0.0)) return ctx_fail(c, OCMC_ERR_ARG, "weights sum to zero");
    for (int b = 0; b < n_beamlets; ++b) {
        const ocmc_beamlet& B = list[b];
        if (B.n_histories < 1 || B.n_histories >= (1ull << 32))
            return ctx_fail(c, OCMC_ERR_ARG, "beamlet histories must be in [1, 2^32)");
        double nd = std::sqrt((double)B.dir[0] * B.dir[0] + (double)B.dir[1] * B.dir[1] + (double)B.dir[2] * B.dir[2]);
        if (!(nd > 1e-6) || !std::isfinite(nd)) return ctx_fail(c, OCMC_ERR_ARG, "beamlet dir must be non-zero");
        if (!(B.field_x >= 0.f && B.field_y >= 0.f && std::isfinite(B.ssd) && std::isfinite(B.iso[0]) &&
              std::isfinite(B.iso[1]) && std::isfinite(B.iso[2])))
            return ctx_fail(c, OCMC_ERR_ARG, "bad beamlet geometry");
    }
    BCK(cudaSetDevice(c->device), "cudaSetDevice");
    if (c->ran || c->bl_ran) cudaDeviceSynchronize();
    if (n_beamlets != c->bl_n) {
        BCK(realloc_dev(&c->d_bl, n_beamlets), "allocation");
        BCK(realloc_dev(&c->d_bl_prefix, n_beamlets + 1), "allocation");
        BCK(realloc_dev(&c->d_bl_offs, n_beamlets), "allocation");
        BCK(realloc_dev(&c->d_bl_caps, n_beamlets), "allocation");
        BCK(realloc_dev(&c->d_bl_nnz, n_beamlets), "allocation");
        BCK(realloc_dev(&c->d_bl_over, n_beamlets), "allocation");
    }
    c->bl_n = n_beamlets;
    c->bl_particle = particle;
    c->bl_bins = n_bins;
    c->bl_edges.assign(edges, edges + n_bins + 1);
    c->bl_weights.assign(weights, weights + n_bins);
    c->bl_list.assign(list, list + n_beamlets);
    c->bl_sized = false;
    c->bl_graph_valid = false;
    c->bl_ran = false;
    return OCMC_OK;
}

ocmc_status ocmc_run_beamlets(ocmc_ctx* c, uint64_t seed, void* stream)
{
    if (!c) return ctx_fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (!c->have_phantom) return ctx_fail(c, OCMC_ERR_STATE, "no phantom (call ocmc_create_phantom)");
    if (c->bl_n < 1) return ctx_fail(c, OCMC_ERR_STATE, "no beamlets (call ocmc_set_beamlets)");
    if (c->p.flags & FLAG_CROSS_VOXELS)
        return ctx_fail(c, OCMC_ERR_ARG, "voxel-crossing electron steps are not available for beamlets");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BCK(cudaSetDevice(c->device), "cudaSetDevice");
    ocmc_status st = ctx_ensure_tables(c, s);
    if (st != OCMC_OK) return st;
    if (!c->bl_sized) {
        st = size_tables(c, seed, s);
        if (st != OCMC_OK) return st;
    }
    for (int attempt = 0;; ++attempt) {
        if (!c->bl_graph_valid || c->bl_graph_seed != seed) {
            st = capture_graph(c, seed);
            if (st != OCMC_OK) return st;
        }
        BCK(cudaEventRecord(c->ev0, s), "event");
        BCK(cudaGraphLaunch(c->bl_exec, s), "graph launch");
        BCK(cudaEventRecord(c->ev1, s), "event");
        BCK(cudaStreamSynchronize(s), "synchronize");
        c->timed = true;
        c->last_stream = s;
        std::vector<unsigned int> over;
        st = read_overflow(c, over);
        if (st != OCMC_OK) return st;
        bool any = false;
        const unsigned long long cap_max = next_pow2((unsigned long long)std::ceil(c->nvox / 0.7) + 1);
        for (int b = 0; b < c->bl_n; ++b)
            if (over[b]) {
                any = true;
                c->bl_cap[b] = std::min(cap_max, c->bl_cap[b] * 4);
            }
        if (!any) break;
        c->bl_graph_valid = false;      // enlarge the full tables and run again (same result)
        if (attempt >= 8) return ctx_fail(c, OCMC_ERR_OVERFLOW, "beamlet tables keep overflowing");
    }
    c->bl_ran = true;
    int e = 0;
    BCK(cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error flag");
    if (e & ERR_BOUNDS) return ctx_fail(c, OCMC_ERR_BOUNDS, "a bounds check failed (checks build)");
    if (e & ERR_OVERFLOW) return ctx_fail(c, OCMC_ERR_OVERFLOW, "a secondary stack overflowed");
    if (e & ERR_LIMIT) return ctx_fail(c, OCMC_ERR_TIMEOUT, "a particle hit the step or sampling limit");
    return OCMC_OK;
}

ocmc_status ocmc_get_beamlet_dose(ocmc_ctx* c, int b, int32_t* idx, float* dose, int64_t* raw, int64_t capacity,
                                  int64_t* nnz)
{
    if (!c || !nnz) return ctx_fail(c, OCMC_ERR_ARG, "NULL argument");
    if (!c->bl_ran) return ctx_fail(c, OCMC_ERR_STATE, "no beamlet run");
    if (b < 0 || b >= c->bl_n) return ctx_fail(c, OCMC_ERR_ARG, "beamlet index out of range");
    if (capacity < 0) return ctx_fail(c, OCMC_ERR_ARG, "capacity must be >= 0");
    BCK(cudaSetDevice(c->device), "cudaSetDevice");
    if (c->out_cap < c->nvox) {
        BCK(realloc_dev(&c->d_dense, c->nvox), "allocation");
        BCK(realloc_dev(&c->d_chunks, (c->nvox + 1023) / 1024 + 1), "allocation");
        BCK(realloc_dev(&c->d_oidx, c->nvox), "allocation");
        BCK(realloc_dev(&c->d_odose, c->nvox), "allocation");
        BCK(realloc_dev(&c->d_oraw, c->nvox), "allocation");
        c->out_cap = c->nvox;
    }
    unsigned long long off = 0;
    for (int i = 0; i < b; ++i) off += c->bl_cap[i];
    cudaStream_t s = c->last_stream;
    const double scale = 1.0 / (268435456.0 * (double)c->dx * c->dy * c->dz * (double)c->bl_list[b].n_histories);
    BCK(launch_bl_extract(c->d_bl_keys + off, c->d_bl_vals + off, c->bl_cap[b], c->nvox, c->d_dense, c->d_chunks,
                          c->d_oidx, c->d_oraw, c->d_odose, c->d_density, scale, c->d_sum, s),
        "beamlet extraction");
    unsigned long long n = 0;
    BCK(cudaMemcpyAsync(&n, c->d_sum, sizeof(n), cudaMemcpyDeviceToHost, s), "copy");
    BCK(cudaStreamSynchronize(s), "synchronize");
    *nnz = (int64_t)n;
    size_t m = (size_t)std::min<long long>((long long)n, capacity);
    if (m) {
        if (idx) BCK(cudaMemcpy(idx, c->d_oidx, sizeof(int) * m, cudaMemcpyDeviceToHost), "copy");
        if (dose) BCK(cudaMemcpy(dose, c->d_odose, sizeof(float) * m, cudaMemcpyDeviceToHost), "copy");
        if (raw) BCK(cudaMemcpy(raw, c->d_oraw, sizeof(long long) * m, cudaMemcpyDeviceToHost), "copy");
    }
    return OCMC_OK;
}

ocmc_status ocmc_autotune(ocmc_ctx* c, uint64_t pilot, ocmc_params* chosen)
{
    if (!c) return ctx_fail(c, OCMC_ERR_ARG, "ctx is NULL");
    if (!c->have_phantom || !c->have_source) return ctx_fail(c, OCMC_ERR_STATE, "need a phantom and a source");
    if (pilot < 1) return ctx_fail(c, OCMC_ERR_ARG, "pilot_histories must be > 0");
    // (register cap, threads per block) pairs that fill an SM, x type-switch thresholds, x
    // energy classes of the charged stacks (one stack, or a second below 2 MeV)
    const int shape_c[][2] = {{64, 1024}, {64, 512}, {80, 256}, {56, 384}};
    const int high_c[] = {2048, 4096, 7680};   // of the default 8192-record stacks
    const int low_c[] = {8, 16};
    const float split_c[] = {0.f, 2.f};
    ocmc_params base = c->p, best = c->p;
    float best_ms = 3.0e38f;
    for (const auto& sh : shape_c)
        for (int hi : high_c)
            for (int lo : low_c)
                for (float sp : split_c) {
                    ocmc_params q = base;
                    q.max_registers = sh[0];
                    q.block_threads = sh[1];
                    q.blocks_per_sm = 0;
                    q.switch_high = hi;
                    q.switch_low = lo;
                    q.e_class_split = sp;
                    ocmc_status st = ocmc_set_params(c, &q);
                    if (st != OCMC_OK) return st;
                    float ms_min = 3.0e38f;
                    for (int rep = 0; rep < 3; ++rep) {
                        st = ocmc_reset_tally(c);
                        if (st == OCMC_OK) st = ocmc_run_range(c, 0, pilot, pilot, 1, nullptr);
                        if (st != OCMC_OK) return st;
                        BCK(cudaEventSynchronize(c->ev1), "synchronize");
                        float ms = 0.f;
                        BCK(cudaEventElapsedTime(&ms, c->ev0, c->ev1), "timing");
                        if (rep > 0) ms_min = std::min(ms_min, ms);
                    }
                    if (ms_min < best_ms) {
                        best_ms = ms_min;
                        best = q;
                    }
                }
    ocmc_status st = ocmc_set_params(c, &best);
    if (st == OCMC_OK) st = ocmc_reset_tally(c);
    if (st == OCMC_OK && chosen) *chosen = best;
    return st;
}

}  // extern "C"
