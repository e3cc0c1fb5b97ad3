// tcm_api.cu -- host runtime and C ABI of libtcm (see include/tcm.h).
//
// The runtime is a batch engine: one box pool, one brick-table space split
// into per-simulation ranges, one simulation table and one active list, all
// resident in HBM.  Every step is one cooperative launch of the step kernel
// over all live simulations; the host only launches, and reads a status
// word per call.  tcm_create makes a batch holding exactly one simulation.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <thread>
#include <vector>

#include "../../include/tcm.h"
#include "tcm_internal.cuh"

using namespace tcm;

namespace {

constexpr double INV_SQRT3 = 0.57735026918962576451;

struct HostSrc {
    int brick, local;
    long long start;
    std::vector<float> w;
};

struct HostSim {
    bool used = false;     // this table entry holds a simulation
    bool primed = false;   // its initial bricks are boxed
    bool live = false;     // steps with the batch
    bool paused = false;   // kept with its boxes, not stepping (tcm_batch_pause)
    long long nx = 0, ny = 0, nz = 0;
    int mx = 0, my = 0, mz = 0;
    long long n_bricks = 0, range_len = 0, brick_base = 0;
    int dense = 0;
    float *kslabs = nullptr;
    long long n_kslabs = 0;
    std::vector<HostSrc> sources;
    std::vector<float> init_now, init_prev;
    bool have_field = false;
    long long step = 0;
    long long target = -1;   // freeze after this many steps (-1: never)
    double dx = 1, dt = 1;
    float c_max = 0.f;
    float *lpf_a = nullptr;    // Eq. 7 filter operator (device)
    SimDev dev{};
};

struct Range {
    long long base, len;
};

}  // namespace

struct tcm_sim {
    tcm_batch *b = nullptr;
    int id = 0;
    bool owns_batch = false;
};

struct tcm_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    int grid = 0;
    Engine E{};
    long long cap_bricks = 0, n_words = 0;
    int max_sims = 0;
    int n_slots = 0;
    void *pool = nullptr;
    bool own_pool = false;
    std::vector<void *> allocs;
    std::vector<HostSim> sims;
    std::vector<tcm_sim *> handles;
    std::vector<Range> free_ranges;
    SrcDev *d_src = nullptr;
    float *d_wave = nullptr;
    unsigned *h_err = nullptr;  // pinned
    bool poisoned = false;
    tcm_status sticky = TCM_OK;
    long long launches = 0;
    int list_parity = 0;
    bool dirty_list = false;   // the active list must be rebuilt before the next step
    int lpf_grid = 0;          // grid of the Eq. 7 kernel (0 until a sim uses it)
    // Captured CUDA graphs of launch sequences, keyed by their launch
    // arguments; valid for the Engine they were captured with.
    bool use_graphs = true;
    cudaStream_t cap_stream = nullptr;   // private stream to capture on (the user's may be the legacy one)
    struct Graph {
        std::vector<int> key;
        cudaGraphExec_t exec;
        unsigned long long last_use;
    };
    std::vector<Graph> graphs;
    Engine graph_engine{};
    unsigned long long graph_clock = 0;
    long long graph_launches = 0;   // launches issued through graphs
    // scratch of tcm_batch_headroom (allocated by its first call)
    unsigned char *reach_a = nullptr, *reach_b = nullptr;
    unsigned long long *reach_count = nullptr;
    // device scratch of the read and count calls (grown as needed, kept)
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
};

namespace {

tcm_status dev_err(cudaError_t e)
{
    if (e == cudaSuccess) return TCM_OK;
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return TCM_ENOMEM;
    return TCM_EDEVICE;
}

#define TRY(expr)                                          \
    do {                                                   \
        tcm_status _s = dev_err(expr);                     \
        if (_s != TCM_OK) return _s;                       \
    } while (0)

#define TRYS(expr)                                         \
    do {                                                   \
        tcm_status _s = (expr);                            \
        if (_s != TCM_OK) return _s;                       \
    } while (0)

template <typename T>
tcm_status dalloc(tcm_batch *b, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TCM_ENOMEM : TCM_EDEVICE;
    }
    b->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return TCM_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Device scratch of at least `bytes` for a read or count call: one buffer per
// batch, grown when a call needs more (the old one freed after the batch's
// stream has drained) and kept until the batch is destroyed, so that the
// calls neither allocate nor free (and so synchronise the device) each time.
tcm_status scratch(tcm_batch *b, size_t bytes, void **out)
{
    bytes = std::max<size_t>(bytes, 256);
    if (b->scratch_bytes < bytes) {
        if (b->scratch) {
            cudaStreamSynchronize(b->stream);
            cudaFree(b->scratch);
            b->scratch = nullptr;
            b->scratch_bytes = 0;
        }
        if (cudaMalloc(&b->scratch, bytes) != cudaSuccess) {
            cudaGetLastError();
            b->scratch = nullptr;
            return TCM_ENOMEM;
        }
        b->scratch_bytes = bytes;
    }
    *out = b->scratch;
    return TCM_OK;
}

tcm_status poison(tcm_batch *b, tcm_status s)
{
    b->poisoned = true;
    if (b->sticky == TCM_OK) b->sticky = s;
    return s;
}

tcm_status sync_status(tcm_batch *b)
{
    cudaError_t e = cudaMemcpyAsync(b->h_err, &b->E.st->err, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return poison(b, TCM_EDEVICE);
    }
    const unsigned err = *b->h_err;
    if (err & ERR_TIMEOUT) return poison(b, TCM_ETIMEOUT);
    if (err & ERR_BOUNDS) return poison(b, TCM_EDEVICE);   // checked build only
    if (err & ERR_NOMEM) return poison(b, TCM_ENOMEM);
    return TCM_OK;
}

// Immutable part of a SimDev (everything before the device-owned counters).
tcm_status upload_sim_header(tcm_batch *b, int id)
{
    TRY(cudaMemcpyAsync(b->E.sims + id, &b->sims[id].dev, offsetof(SimDev, step), cudaMemcpyHostToDevice,
                        b->stream));
    return TCM_OK;
}

// Concatenate the sources of every simulation into the device table.
tcm_status upload_sources(tcm_batch *b)
{
    std::vector<SrcDev> src;
    std::vector<float> wave;
    for (int id = 0; id < (int)b->sims.size(); ++id) {
        HostSim &h = b->sims[id];
        if (!h.used) continue;
        h.dev.src_begin = (int)src.size();
        for (const auto &q : h.sources) {
            SrcDev d{};
            d.sim = id;
            d.brick = q.brick;
            d.local = q.local;
            d.start = q.start;
            d.len = (long long)q.w.size();
            d.w_off = (long long)wave.size();
            wave.insert(wave.end(), q.w.begin(), q.w.end());
            src.push_back(d);
        }
        h.dev.src_end = (int)src.size();
    }
    TRY(cudaStreamSynchronize(b->stream));
    if (b->d_src) cudaFree(b->d_src);
    if (b->d_wave) cudaFree(b->d_wave);
    b->d_src = nullptr;
    b->d_wave = nullptr;
    TRY(cudaMalloc(&b->d_src, std::max<size_t>(src.size(), 1) * sizeof(SrcDev)));
    TRY(cudaMalloc(&b->d_wave, std::max<size_t>(wave.size(), 1) * sizeof(float)));
    if (!src.empty())
        TRY(cudaMemcpyAsync(b->d_src, src.data(), src.size() * sizeof(SrcDev), cudaMemcpyHostToDevice, b->stream));
    if (!wave.empty())
        TRY(cudaMemcpyAsync(b->d_wave, wave.data(), wave.size() * sizeof(float), cudaMemcpyHostToDevice,
                            b->stream));
    b->E.src = b->d_src;
    b->E.n_src = (int)src.size();
    b->E.wave = b->d_wave;
    for (int id = 0; id < (int)b->sims.size(); ++id)
        if (b->sims[id].used) TRYS(upload_sim_header(b, id));
    return TCM_OK;
}

long long range_alloc(tcm_batch *b, long long len)
{
    for (size_t i = 0; i < b->free_ranges.size(); ++i) {
        Range &r = b->free_ranges[i];
        if (r.len >= len) {
            const long long base = r.base;
            r.base += len;
            r.len -= len;
            if (r.len == 0) b->free_ranges.erase(b->free_ranges.begin() + (long)i);
            return base;
        }
    }
    return -1;
}

void range_free(tcm_batch *b, long long base, long long len)
{
    b->free_ranges.push_back({base, len});
    std::sort(b->free_ranges.begin(), b->free_ranges.end(),
              [](const Range &x, const Range &y) { return x.base < y.base; });
    std::vector<Range> merged;
    for (const Range &r : b->free_ranges) {
        if (!merged.empty() && merged.back().base + merged.back().len == r.base) merged.back().len += r.len;
        else merged.push_back(r);
    }
    b->free_ranges.swap(merged);
}

// Largest value of c[0..n) and whether any is negative, NaN or infinite, in
// four-wide vectors (GCC vector extensions: SIMD on any host) with eight
// independent running maxima; the comparisons are IEEE ones, so a NaN fails
// x >= 0 and is flagged, and a maximum does not depend on the order it is
// taken in.
void scan_c(const float *c, long long n, float *cmax, bool *bad)
{
    typedef float v4f __attribute__((vector_size(16)));
    typedef int v4i __attribute__((vector_size(16)));
    const v4f zero = {0.f, 0.f, 0.f, 0.f};
    const v4f inf = {INFINITY, INFINITY, INFINITY, INFINITY};
    v4f m0 = zero, m1 = zero;
    v4i f = {0, 0, 0, 0};
    long long i = 0;
    for (; i + 8 <= n; i += 8) {
        v4f a, b;
        std::memcpy(&a, c + i, sizeof(a));
        std::memcpy(&b, c + i + 4, sizeof(b));
        m0 = a > m0 ? a : m0;
        m1 = b > m1 ? b : m1;
        f |= ~(a >= zero) | (a == inf) | ~(b >= zero) | (b == inf);
    }
    float m = 0.f;
    unsigned flag = 0;
    for (int k = 0; k < 4; ++k) {
        m = m0[k] > m ? m0[k] : m;
        m = m1[k] > m ? m1[k] : m;
        flag |= f[k] != 0;
    }
    for (; i < n; ++i) {
        const float x = c[i];
        m = x > m ? x : m;
        flag |= (unsigned)!(x >= 0.f) | (unsigned)(x == INFINITY);
    }
    *cmax = m;
    *bad = flag != 0;
}

float model_c_max(const tcm_domain *d, const tcm_velocity_model *v, bool *bad)
{
    *bad = false;
    float cmax = 0.f;
    if (v->kind == TCM_MEDIA_DENSE) {
        // A dense model can hold 1e8+ values: the scan is split over host
        // threads (max and "any bad" do not depend on the split).
        const long long n = d->nx * d->ny * d->nz;
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nt = (int)std::min<long long>(std::min(hw, 16u), std::max(1LL, n >> 22));
        std::vector<float> part_max((size_t)nt, 0.f);
        std::vector<char> part_bad((size_t)nt, 0);
        std::vector<std::thread> pool;
        const long long chunk = (n + nt - 1) / nt;
        for (int t = 0; t < nt; ++t) {
            const long long i0 = std::min(n, (long long)t * chunk), i1 = std::min(n, i0 + chunk);
            auto job = [=, &part_max, &part_bad]() {
                bool b = false;
                scan_c(v->c + i0, i1 - i0, &part_max[(size_t)t], &b);
                part_bad[(size_t)t] = b;
            };
            if (t + 1 < nt) {
                try {
                    pool.emplace_back(job);
                    continue;
                } catch (...) {
                }
            }
            job();   // the last chunk (or one no thread could be started for)
        }
        for (auto &th : pool) th.join();
        for (int t = 0; t < nt; ++t) {
            cmax = std::max(cmax, part_max[(size_t)t]);
            if (part_bad[(size_t)t]) *bad = true;
        }
        return cmax;
    }
    cmax = v->c_background;
    if (!(v->c_background >= 0.f)) *bad = true;
    for (int m = 0; m < v->n_layers; ++m) {
        if (!(v->layer_c[m] >= 0.f)) *bad = true;
        cmax = std::max(cmax, v->layer_c[m]);
    }
    for (int q = 0; q < v->n_spheres; ++q) {
        if (!(v->sphere_c[q] >= 0.f)) *bad = true;
        cmax = std::max(cmax, v->sphere_c[q]);
    }
    if (std::isinf(cmax)) *bad = true;
    return cmax;
}

// Argument checks shared by tcm_create and tcm_batch_add, before any GPU work.
tcm_status check_sim_args(const tcm_domain *domain, const tcm_velocity_model *velocity, double dx, double dt,
                          double threshold, tcm_brick brick, int storage, int threshold_mode, int decay_steps,
                          float *c_max_out)
{
    if (!domain || !velocity) return TCM_EINVAL;
    if (domain->nx < 1 || domain->ny < 1 || domain->nz < 1) return TCM_EINVAL;
    if (domain->nx > (1LL << 30) || domain->ny > (1LL << 30) || domain->nz > (1LL << 30)) return TCM_EINVAL;
    if (!(dx > 0) || !(dt > 0) || !(threshold >= 0) || std::isinf(threshold)) return TCM_EINVAL;
    size_t slot_bytes = 0;
    if (tcm_slot_bytes(brick, storage, &slot_bytes) != TCM_OK) return TCM_EINVAL;
    if (threshold_mode != TCM_THR_ABSOLUTE && threshold_mode != TCM_THR_RELATIVE) return TCM_EINVAL;
    if (decay_steps < 0 || decay_steps > (int)SD_MASK) return TCM_EINVAL;
    if (velocity->kind == TCM_MEDIA_DENSE) {
        if (!velocity->c) return TCM_EINVAL;
    } else if (velocity->kind == TCM_MEDIA_RULES) {
        if (velocity->n_layers < 0 || velocity->n_spheres < 0) return TCM_EINVAL;
        if (velocity->n_layers > 0 && (!velocity->layer_z || !velocity->layer_c)) return TCM_EINVAL;
        if (velocity->n_spheres > 0 && (!velocity->sphere_xyzr || !velocity->sphere_c)) return TCM_EINVAL;
    } else {
        return TCM_EINVAL;
    }
    const long long mx = (domain->nx + BX - 1) / BX, my = (domain->ny + BY - 1) / BY,
                    mz = (domain->nz + BZ - 1) / BZ;
    if (mx * my * mz > (1LL << 31) - 64) return TCM_EINVAL;
    // Eq. 4 with the largest velocity of the model.
    bool bad = false;
    const float cmax = model_c_max(domain, velocity, &bad);
    if (bad) return TCM_EINVAL;
    if ((double)cmax * dt / dx > INV_SQRT3) return TCM_ECFL;
    *c_max_out = cmax;
    return TCM_OK;
}

tcm_status batch_new(int device, cudaStream_t stream, void *pool_ptr, size_t pool_bytes, int storage,
                     long long max_bricks, int max_sims, tcm_batch **out)
{
    *out = nullptr;
    if (storage != TCM_STORAGE_F32 && storage != TCM_STORAGE_BF16 && storage != TCM_STORAGE_F16 &&
        storage != TCM_STORAGE_MIXED)
        return TCM_EINVAL;
    const size_t slot_bytes = storage == TCM_STORAGE_MIXED ? (size_t)slot_elems(ST_F32) * storage_bytes(ST_F32)
                                                           : (size_t)slot_elems(storage) * storage_bytes(storage);
    const long long n_slots_ll = (long long)(pool_bytes / slot_bytes);
    if (n_slots_ll < 1 || max_bricks < 1 || max_sims < 1 || max_sims > 65535) return TCM_EINVAL;
    if (pool_ptr && reinterpret_cast<uintptr_t>(pool_ptr) % 16 != 0) return TCM_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return TCM_EDEVICE;
    }
    DeviceGuard guard(device);
    tcm_batch *b = new (std::nothrow) tcm_batch();
    if (!b) return TCM_ENOMEM;
    auto fail = [&](tcm_status e) {
        tcm_batch_destroy(b);
        return e;
    };
    b->device = device;
    b->stream = stream;
    b->n_slots = (int)std::min<long long>(n_slots_ll, (1LL << 31) - 64);
    b->cap_bricks = (max_bricks + 31) / 32 * 32;
    b->n_words = b->cap_bricks / 32;
    b->max_sims = max_sims;
    b->grid = step_grid_size(device);
    if (b->grid <= 0) return fail(TCM_EDEVICE);
    if (cudaMallocHost(&b->h_err, sizeof(unsigned)) != cudaSuccess) return fail(TCM_EDEVICE);
    if (pool_ptr) {
        b->pool = pool_ptr;
    } else {
        if (cudaMalloc(&b->pool, (size_t)b->n_slots * slot_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(TCM_ENOMEM);
        }
        b->own_pool = true;
    }
    Engine &E = b->E;
    E.phi = b->pool;
    E.storage = storage;
    E.slot_bytes = (int)slot_bytes;
    E.n_slots = b->n_slots;
    E.n_words = b->n_words;
    E.words_per_block = (int)std::max<long long>(1, (b->n_words + b->grid - 1) / b->grid);
    tcm_status st;
    float *kscal = nullptr;
    int *kslab_of_brick = nullptr;
    if ((st = dalloc(b, &E.slot_of_brick, b->cap_bricks)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &kscal, b->cap_bricks)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &kslab_of_brick, b->cap_bricks)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.sd_of_brick, b->cap_bricks)) != TCM_OK) return fail(st);
    E.kscal = kscal;
    E.kslab_of_brick = kslab_of_brick;
    if ((st = dalloc(b, &E.bitmap, b->n_words)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.sim_of_word, b->n_words)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.blocktot, b->grid)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.meta, b->n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.rec, (size_t)b->n_slots * 8)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.items0, b->n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.items1, b->n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.listids, b->n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.free_stack, b->n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.retired, b->n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.newslots, b->n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.sims, max_sims)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.st, 1)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.claim_step, b->n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.lpf_mark, b->n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.lpf_q, b->n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(b, &E.lpf_aff, b->n_slots)) != TCM_OK) return fail(st);
    E.n_sims = max_sims;
    E.prefetch = 1;
    b->sims.resize(max_sims);
    b->handles.assign(max_sims, nullptr);
    b->free_ranges.push_back({0, b->cap_bricks});
    cudaStream_t q = b->stream;
    EngineState es{};
    es.free_top = b->n_slots;
    if (cudaMemsetAsync(E.slot_of_brick, 0xff, b->cap_bricks * sizeof(int), q) != cudaSuccess ||
        cudaMemsetAsync(E.sd_of_brick, 0, b->cap_bricks * sizeof(unsigned short), q) != cudaSuccess ||
        cudaMemsetAsync(E.bitmap, 0, b->n_words * sizeof(unsigned), q) != cudaSuccess ||
        cudaMemsetAsync(E.sim_of_word, 0, b->n_words * sizeof(unsigned short), q) != cudaSuccess ||
        cudaMemsetAsync(E.blocktot, 0, b->grid * sizeof(int), q) != cudaSuccess ||
        cudaMemsetAsync(E.sims, 0, max_sims * sizeof(SimDev), q) != cudaSuccess ||
        cudaMemsetAsync(E.claim_step, 0xff, b->n_slots * sizeof(int), q) != cudaSuccess ||
        cudaMemsetAsync(E.lpf_mark, 0, b->n_slots * sizeof(int), q) != cudaSuccess ||
        // records stamped with launch 0xffffffff: never taken for a current one
        cudaMemsetAsync(E.rec, 0xff, (size_t)b->n_slots * 8 * sizeof(float), q) != cudaSuccess ||
        cudaMemcpyAsync(E.st, &es, sizeof(es), cudaMemcpyHostToDevice, q) != cudaSuccess ||
        launch_iota_desc(E.free_stack, b->n_slots, b->n_slots - 1, q) != cudaSuccess ||
        cudaStreamSynchronize(q) != cudaSuccess)
        return fail(TCM_EDEVICE);
    // an empty source table, so kernels always see valid pointers
    if ((st = upload_sources(b)) != TCM_OK) return fail(st);
    if (cudaStreamSynchronize(q) != cudaSuccess) return fail(TCM_EDEVICE);
    *out = b;
    return TCM_OK;
}

// Heterogenic Bulking of one simulation into its brick range (Media).
tcm_status bulk_sim(tcm_batch *b, HostSim &h, const tcm_velocity_model *velocity, double dx, double dt)
{
    cudaStream_t q = b->stream;
    MediaDev md{};
    md.kind = velocity->kind == TCM_MEDIA_DENSE ? MEDIA_DENSE : MEDIA_RULES;
    std::vector<void *> tmp;
    auto tmp_alloc = [&](void **p, size_t bytes) -> bool {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        tmp.push_back(*p);
        return true;
    };
    struct Cleanup {
        std::vector<void *> &t;
        ~Cleanup()
        {
            for (void *p : t) cudaFree(p);
        }
    } cleanup{tmp};
    int *d_cnt = nullptr;
    bool ok = tmp_alloc((void **)&d_cnt, sizeof(int));
    const size_t n_nodes = (size_t)(h.nx * h.ny * h.nz);
    if (ok && md.kind == MEDIA_DENSE) {
        // page-locked host memory the device can address is read in place by
        // the bulking kernels; other memory is copied to the device first
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, velocity->c) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer) {
            md.c = static_cast<const float *>(pa.devicePointer);
        } else {
            cudaGetLastError();
            float *d_c = nullptr;
            ok = tmp_alloc((void **)&d_c, n_nodes * sizeof(float)) &&
                 cudaMemcpyAsync(d_c, velocity->c, n_nodes * sizeof(float), cudaMemcpyHostToDevice, q) ==
                     cudaSuccess;
            md.c = d_c;
        }
    } else if (ok) {
        double *d_lz = nullptr, *d_sph = nullptr;
        float *d_lc = nullptr, *d_sc = nullptr;
        md.c_bg = velocity->c_background;
        md.n_layers = velocity->n_layers;
        md.n_spheres = velocity->n_spheres;
        ok = tmp_alloc((void **)&d_lz, sizeof(double) * velocity->n_layers) &&
             tmp_alloc((void **)&d_lc, sizeof(float) * velocity->n_layers) &&
             tmp_alloc((void **)&d_sph, sizeof(double) * 4 * velocity->n_spheres) &&
             tmp_alloc((void **)&d_sc, sizeof(float) * velocity->n_spheres);
        if (ok && velocity->n_layers > 0)
            ok = cudaMemcpyAsync(d_lz, velocity->layer_z, sizeof(double) * velocity->n_layers,
                                 cudaMemcpyHostToDevice, q) == cudaSuccess &&
                 cudaMemcpyAsync(d_lc, velocity->layer_c, sizeof(float) * velocity->n_layers,
                                 cudaMemcpyHostToDevice, q) == cudaSuccess;
        if (ok && velocity->n_spheres > 0)
            ok = cudaMemcpyAsync(d_sph, velocity->sphere_xyzr, sizeof(double) * 4 * velocity->n_spheres,
                                 cudaMemcpyHostToDevice, q) == cudaSuccess &&
                 cudaMemcpyAsync(d_sc, velocity->sphere_c, sizeof(float) * velocity->n_spheres,
                                 cudaMemcpyHostToDevice, q) == cudaSuccess;
        md.layer_z = d_lz;
        md.layer_c = d_lc;
        md.sph = d_sph;
        md.sph_c = d_sc;
    }
    if (!ok) return TCM_ENOMEM;
    float *kscal = const_cast<float *>(b->E.kscal);
    int *kslab_of_brick = const_cast<int *>(b->E.kslab_of_brick);
    TRY(cudaMemsetAsync(d_cnt, 0, sizeof(int), q));
    TRY(launch_bulk_classify(md, (int)h.nx, (int)h.ny, (int)h.nz, h.mx, h.my, h.mz, dt, dx, h.brick_base, kscal,
                             kslab_of_brick, d_cnt, q));
    int n_kslabs = 0;
    TRY(cudaMemcpyAsync(b->h_err, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, q));
    TRY(cudaStreamSynchronize(q));
    std::memcpy(&n_kslabs, b->h_err, sizeof(int));
    h.n_kslabs = n_kslabs;
    TRY(cudaMalloc(&h.kslabs, std::max<size_t>((size_t)n_kslabs * BVOL, 1) * sizeof(float)));
    if (n_kslabs > 0)
        TRY(launch_bulk_fill(md, (int)h.nx, (int)h.ny, (int)h.nz, h.mx, h.my, h.mz, dt, dx, h.brick_base,
                             kslab_of_brick, h.kslabs, q));
    TRY(cudaStreamSynchronize(q));
    return TCM_OK;
}

tcm_status sim_add(tcm_batch *b, const tcm_domain *domain, const tcm_velocity_model *velocity, double dx, double dt,
                   float c_max, double threshold, int thr_mode, float alpha, int decay_steps, int dense,
                   long long n_steps, int *out_id)
{
    int id = -1;
    for (int i = 0; i < b->max_sims; ++i)
        if (!b->sims[i].used) {
            id = i;
            break;
        }
    if (id < 0) return TCM_ENOMEM;
    HostSim h;
    h.nx = domain->nx;
    h.ny = domain->ny;
    h.nz = domain->nz;
    h.mx = (int)((h.nx + BX - 1) / BX);
    h.my = (int)((h.ny + BY - 1) / BY);
    h.mz = (int)((h.nz + BZ - 1) / BZ);
    h.n_bricks = (long long)h.mx * h.my * h.mz;
    h.range_len = (h.n_bricks + 31) / 32 * 32;
    h.dense = dense;
    h.target = n_steps > 0 ? n_steps : -1;
    if (dense && h.n_bricks > b->n_slots) return TCM_ENOMEM;
    h.brick_base = range_alloc(b, h.range_len);
    if (h.brick_base < 0) return TCM_ENOMEM;
    tcm_status st = bulk_sim(b, h, velocity, dx, dt);
    if (st != TCM_OK) {
        if (h.kslabs) cudaFree(h.kslabs);
        range_free(b, h.brick_base, h.range_len);
        return st;
    }
    SimDev &S = h.dev;
    S = SimDev{};
    S.nx = (int)h.nx;
    S.ny = (int)h.ny;
    S.nz = (int)h.nz;
    S.mx = h.mx;
    S.my = h.my;
    S.mz = h.mz;
    S.brick_base = h.brick_base;
    S.n_bricks = h.n_bricks;
    S.thr_mode = thr_mode;
    S.dense = dense;
    S.tau = threshold;
    S.alpha = alpha;
    S.decay_steps = decay_steps;
    S.kslabs = h.kslabs;
    S.live = 0;
    S.scale = 1.f;
    S.inv_scale = 1.f;
    S.interval = 1;
    S.neighbours = 6;
    S.storage = b->E.storage == ST_MIXED ? ST_F32 : b->E.storage;
    h.c_max = c_max;
    h.dx = dx;
    h.dt = dt;
    h.used = true;
    // the brick range's words now belong to this sim
    {
        std::vector<unsigned short> owner((size_t)(h.range_len / 32), (unsigned short)id);
        cudaError_t e = cudaMemcpyAsync(b->E.sim_of_word + h.brick_base / 32, owner.data(),
                                        owner.size() * sizeof(unsigned short), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h.kslabs);
            range_free(b, h.brick_base, h.range_len);
            return TCM_EDEVICE;
        }
    }
    b->sims[id] = std::move(h);
    // full upload: counters start at zero
    TRY(cudaMemcpyAsync(b->E.sims + id, &b->sims[id].dev, sizeof(SimDev), cudaMemcpyHostToDevice, b->stream));
    TRY(cudaStreamSynchronize(b->stream));
    *out_id = id;
    return TCM_OK;
}

// The update procedure run on the initial state (before step 0), over the
// initially boxed bricks `mark`: returns the bricks it triggers.  Level from
// the initial phi^0 (relative: tau x max |phi^0|, FP64).  6-neighbour set:
// the brick across each face whose max |phi^0| is above the level.
// 26-neighbour set: all 26 neighbours of a brick whose max(|phi^0|,
// |phi^-1|) is above the level or that a source feeds in steps
// 0 .. interval-1.
std::vector<long long> initial_triggers(const HostSim &h, const std::vector<char> &mark)
{
    std::vector<long long> out;
    const long long nb = h.n_bricks;
    std::vector<float> mc, fm;
    double G = 0.0;
    if (h.have_field) {
        mc.assign((size_t)nb, 0.f);
        fm.assign((size_t)nb * 6, 0.f);
        for (long long z = 0; z < h.nz; ++z)
            for (long long y = 0; y < h.ny; ++y)
                for (long long x = 0; x < h.nx; ++x) {
                    const size_t i = (size_t)((z * h.ny + y) * h.nx + x);
                    const float a = std::fabs(h.init_now[i]), p = std::fabs(h.init_prev[i]);
                    if (a == 0.f && p == 0.f) continue;
                    const size_t b = (size_t)(((z / BZ) * h.my + (y / BY)) * h.mx + (x / BX));
                    G = std::max(G, (double)a);
                    mc[b] = std::max(mc[b], std::max(a, p));
                    const long long lx = x % BX, ly = y % BY, lz = z % BZ;
                    if (lx == 0) fm[b * 6 + 0] = std::max(fm[b * 6 + 0], a);
                    if (lx == BX - 1) fm[b * 6 + 1] = std::max(fm[b * 6 + 1], a);
                    if (ly == 0) fm[b * 6 + 2] = std::max(fm[b * 6 + 2], a);
                    if (ly == BY - 1) fm[b * 6 + 3] = std::max(fm[b * 6 + 3], a);
                    if (lz == 0) fm[b * 6 + 4] = std::max(fm[b * 6 + 4], a);
                    if (lz == BZ - 1) fm[b * 6 + 5] = std::max(fm[b * 6 + 5], a);
                }
    }
    const double thr = h.dev.thr_mode == TCM_THR_RELATIVE ? h.dev.tau * G : h.dev.tau;
    std::vector<char> src((size_t)nb, 0);
    for (const auto &q : h.sources)
        if (!q.w.empty() && q.start <= h.step + h.dev.interval - 1) src[(size_t)q.brick] = 1;
    for (long long b = 0; b < nb; ++b) {
        if (!mark[(size_t)b]) continue;
        const int cx = (int)(b % h.mx), cy = (int)((b / h.mx) % h.my), cz = (int)(b / ((long long)h.mx * h.my));
        if (h.dev.neighbours == 26) {
            const bool hot = src[(size_t)b] || (h.have_field && (double)mc[(size_t)b] > thr);
            if (!hot) continue;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int ax = cx + dx, ay = cy + dy, az = cz + dz;
                        if ((!dx && !dy && !dz) || ax < 0 || ay < 0 || az < 0 || ax >= h.mx || ay >= h.my ||
                            az >= h.mz)
                            continue;
                        out.push_back(((long long)az * h.my + ay) * h.mx + ax);
                    }
        } else if (h.have_field) {
            for (int f = 0; f < 6; ++f) {
                if (!((double)fm[(size_t)b * 6 + f] > thr)) continue;
                const int ax = cx + (f == 0 ? -1 : f == 1 ? 1 : 0);
                const int ay = cy + (f == 2 ? -1 : f == 3 ? 1 : 0);
                const int az = cz + (f == 4 ? -1 : f == 5 ? 1 : 0);
                if (ax < 0 || ay < 0 || az < 0 || ax >= h.mx || ay >= h.my || az >= h.mz) continue;
                out.push_back(((long long)az * h.my + ay) * h.mx + ax);
            }
        }
    }
    return out;
}

// Box a simulation's initial bricks (source bricks, bricks with initial
// values, or every brick of a dense simulation, plus the bricks the update
// procedure triggers from that state) and start it stepping.
tcm_status sim_prime(tcm_batch *b, int id)
{
    HostSim &h = b->sims[id];
    if (h.primed) return TCM_OK;
    cudaStream_t q = b->stream;
    if (h.dev.storage == ST_F16) {
        // binary16 holds phi / scale: the largest initial value or source
        // sample maps to [128, 256), leaving 2^8 of headroom below 65504.
        float peak = 0.f;
        for (const auto &src : h.sources)
            for (float v : src.w) peak = std::max(peak, std::fabs(v));
        for (float v : h.init_now) peak = std::max(peak, std::fabs(v));
        for (float v : h.init_prev) peak = std::max(peak, std::fabs(v));
        int e = 0;
        if (peak > 0.f && std::isfinite(peak)) {
            std::frexp(peak, &e);   // peak = f * 2^e, f in [0.5, 1)
            e -= 8;
        }
        e = std::max(-100, std::min(100, e));
        h.dev.scale = std::ldexp(1.f, e);
        h.dev.inv_scale = std::ldexp(1.f, -e);
    }
    TRYS(upload_sim_header(b, id));
    TRYS(upload_sources(b));
    for (const auto &src : h.sources) {
        const unsigned short bit = (unsigned short)FLAG_HAS_SRC;
        TRY(cudaMemcpyAsync(b->E.sd_of_brick + h.brick_base + src.brick, &bit, sizeof(bit), cudaMemcpyHostToDevice,
                            q));
        TRY(cudaStreamSynchronize(q));
    }
    std::vector<long long> init;
    long long n_init = 0;
    if (h.dense) {
        n_init = h.n_bricks;
    } else if (!h.have_field) {
        // Source cells only (and, with the 26-neighbour set, the neighbourhood
        // of each source fed before the first update): the same set the pass
        // below finds, without a pass over the whole brick table (the virtual
        // 4096^3 domain has 1.3e8 bricks).
        for (const auto &src : h.sources) {
            if (src.w.empty()) continue;
            init.push_back(src.brick);
            if (h.dev.neighbours != 26 || src.start > h.step + h.dev.interval - 1) continue;
            const int cx = src.brick % h.mx, cy = (src.brick / h.mx) % h.my, cz = src.brick / (h.mx * h.my);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int ax = cx + dx, ay = cy + dy, az = cz + dz;
                        if (ax < 0 || ay < 0 || az < 0 || ax >= h.mx || ay >= h.my || az >= h.mz) continue;
                        init.push_back(((long long)az * h.my + ay) * h.mx + ax);
                    }
        }
        std::sort(init.begin(), init.end());
        init.erase(std::unique(init.begin(), init.end()), init.end());
        n_init = (long long)init.size();
    } else {
        std::vector<char> mark((size_t)h.n_bricks, 0);
        for (const auto &src : h.sources)
            if (!src.w.empty()) mark[(size_t)src.brick] = 1;
        if (h.have_field) {
            for (long long z = 0; z < h.nz; ++z)
                for (long long y = 0; y < h.ny; ++y)
                    for (long long x = 0; x < h.nx; ++x) {
                        const size_t i = (size_t)((z * h.ny + y) * h.nx + x);
                        if (h.init_now[i] != 0.f || h.init_prev[i] != 0.f)
                            mark[(size_t)(((z / BZ) * h.my + (y / BY)) * h.mx + (x / BX))] = 1;
                    }
        }
        // The update procedure before the first step: triggers from the
        // initial fields, and (26-neighbour set) the neighbourhoods of
        // source bricks.
        const std::vector<long long> extra = initial_triggers(h, mark);
        for (long long e : extra) mark[(size_t)e] = 1;
        for (long long i = 0; i < h.n_bricks; ++i)
            if (mark[(size_t)i]) init.push_back(i);
        n_init = (long long)init.size();
    }
    long long *d_init = nullptr;
    if (!h.dense && n_init > 0) {
        TRY(cudaMalloc(&d_init, n_init * sizeof(long long)));
        TRY(cudaMemcpyAsync(d_init, init.data(), n_init * sizeof(long long), cudaMemcpyHostToDevice, q));
    }
    tcm_status st = dev_err(launch_settle(b->E, q));
    if (st == TCM_OK) st = dev_err(launch_admit(b->E, id, d_init, n_init, q));
    if (st == TCM_OK && h.have_field && n_init > 0) {
        const long long bvol = BVOL;
        std::vector<float> packed((size_t)(n_init * 2 * bvol), 0.f);
        std::vector<long long> gids((size_t)n_init);
        for (long long i = 0; i < n_init; ++i) {
            const long long brick = h.dense ? i : init[(size_t)i];
            gids[(size_t)i] = h.brick_base + brick;
            const long long cx = brick % h.mx, cy = (brick / h.mx) % h.my, cz = brick / ((long long)h.mx * h.my);
            for (int e = 0; e < BVOL; ++e) {
                const long long x = cx * BX + e % BX, y = cy * BY + (e / BX) % BY, z = cz * BZ + e / (BX * BY);
                if (x >= h.nx || y >= h.ny || z >= h.nz) continue;
                const size_t i0 = (size_t)((z * h.ny + y) * h.nx + x);
                packed[(size_t)(i * 2 * bvol + e)] = h.init_now[i0];
                // binary32: phi^{-1}; velocity form (16-bit): v^0 = phi^0 - phi^{-1}
                packed[(size_t)(i * 2 * bvol + bvol + e)] =
                    h.dev.storage == ST_F32 ? h.init_prev[i0] : h.init_now[i0] - h.init_prev[i0];
            }
        }
        float *d_packed = nullptr;
        long long *d_gids = nullptr;
        st = dev_err(cudaMalloc(&d_packed, packed.size() * sizeof(float)));
        if (st == TCM_OK) st = dev_err(cudaMalloc(&d_gids, gids.size() * sizeof(long long)));
        if (st == TCM_OK)
            st = dev_err(cudaMemcpyAsync(d_packed, packed.data(), packed.size() * sizeof(float),
                                         cudaMemcpyHostToDevice, q));
        if (st == TCM_OK)
            st = dev_err(cudaMemcpyAsync(d_gids, gids.data(), gids.size() * sizeof(long long),
                                         cudaMemcpyHostToDevice, q));
        if (st == TCM_OK) st = dev_err(launch_scatter_field(b->E, d_packed, d_gids, n_init, (int)(h.step & 1), q));
        if (st == TCM_OK) st = dev_err(cudaStreamSynchronize(q));
        if (d_packed) cudaFree(d_packed);
        if (d_gids) cudaFree(d_gids);
    }
    if (st == TCM_OK) st = dev_err(cudaStreamSynchronize(q));
    if (d_init) cudaFree(d_init);
    if (st != TCM_OK) return poison(b, st);
    std::vector<float>().swap(h.init_now);
    std::vector<float>().swap(h.init_prev);
    h.primed = true;
    h.live = h.target != 0;
    h.dev.live = h.live ? 1 : 0;
    TRYS(upload_sim_header(b, id));
    b->dirty_list = true;
    // a pool too small for the initial bricks
    return sync_status(b);
}

tcm_status prime_all(tcm_batch *b)
{
    for (int id = 0; id < b->max_sims; ++id)
        if (b->sims[id].used && !b->sims[id].primed) TRYS(sim_prime(b, id));
    return TCM_OK;
}

tcm_status ensure_list(tcm_batch *b)
{
    if (!b->dirty_list) return TCM_OK;
    TRY(launch_compact(b->E, b->grid, b->list_parity, b->stream));
    b->dirty_list = false;
    return TCM_OK;
}

tcm_status freeze_sim(tcm_batch *b, int id)
{
    HostSim &h = b->sims[id];
    TRY(launch_freeze(b->E, id, h.brick_base / 32, h.range_len / 32, b->stream));
    h.live = false;
    h.dev.live = 0;
    b->dirty_list = true;
    return TCM_OK;
}

void drop_graphs(tcm_batch *b)
{
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
}

// Launch arguments of the next m steps: per launch (list parity, whether any
// sim runs the update procedure, whether any of those uses Eq. 7), from the
// host copy of every sim's step counter.
std::vector<int> step_args(const tcm_batch *b, long long m)
{
    std::vector<int> key;
    key.reserve((size_t)(3 * m + 1));
    key.push_back((int)m);
    int parity = b->list_parity;
    for (long long j = 0; j < m; ++j) {
        int manage = 0, lpf = 0;
        for (int id = 0; id < b->max_sims; ++id) {
            const HostSim &h = b->sims[id];
            if (h.used && h.live && !h.dense && (h.step + j + 1) % h.dev.interval == 0) {
                manage = 1;
                lpf |= h.dev.lpf;
            }
        }
        key.push_back(parity);
        key.push_back(manage);
        key.push_back(lpf);
        if (manage) parity ^= 1;
    }
    return key;
}

// Issue the launches described by `key` as one CUDA graph (captured on first
// use and kept, up to 32 graphs).  Returns false if capture is unavailable;
// nothing has been launched then.
bool launch_graph(tcm_batch *b, const std::vector<int> &key)
{
    if (std::memcmp(&b->graph_engine, &b->E, sizeof(Engine)) != 0) {
        drop_graphs(b);
        std::memcpy(&b->graph_engine, &b->E, sizeof(Engine));
    }
    tcm_batch::Graph *hit = nullptr;
    for (auto &g : b->graphs)
        if (g.key == key) hit = &g;
    if (!hit) {
        cudaGraph_t graph = nullptr;
        if (!b->cap_stream && cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            b->cap_stream = nullptr;
            b->use_graphs = false;
            return false;
        }
        if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            b->use_graphs = false;
            return false;
        }
        cudaError_t e = cudaSuccess;
        const long long m = key[0];
        for (long long j = 0; j < m && e == cudaSuccess; ++j) {
            e = launch_step(b->E, b->grid, key[1 + 3 * j], key[2 + 3 * j], b->cap_stream);
            if (e == cudaSuccess && key[3 + 3 * j]) e = launch_lpf(b->E, b->lpf_grid, b->cap_stream);
        }
        const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess && e2 == cudaSuccess && graph)
            e = cudaGraphInstantiate(&exec, graph, 0);
        else
            e = e != cudaSuccess ? e : e2;
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess || !exec) {
            cudaGetLastError();
            b->use_graphs = false;   // capture not available: launch directly from now on
            return false;
        }
        if (b->graphs.size() >= 32) {
            size_t old = 0;
            for (size_t i = 1; i < b->graphs.size(); ++i)
                if (b->graphs[i].last_use < b->graphs[old].last_use) old = i;
            cudaGraphExecDestroy(b->graphs[old].exec);
            b->graphs.erase(b->graphs.begin() + (long)old);
        }
        b->graphs.push_back({key, exec, 0});
        hit = &b->graphs.back();
    }
    hit->last_use = ++b->graph_clock;
    if (cudaGraphLaunch(hit->exec, b->stream) != cudaSuccess) {
        cudaGetLastError();
        b->use_graphs = false;
        return false;
    }
    return true;
}

tcm_status batch_step_async(tcm_batch *b, long long n)
{
    if (b->poisoned) return TCM_ESTATE;
    DeviceGuard g(b->device);
    TRYS(prime_all(b));
    for (long long i = 0; i < n;) {
        TRYS(ensure_list(b));
        // Launches up to the next freeze (a sim reaching its step count)
        // form one graph.
        long long m = std::min<long long>(n - i, 64);
        for (int id = 0; id < b->max_sims; ++id) {
            const HostSim &h = b->sims[id];
            if (h.used && h.live && h.target > 0) m = std::min(m, h.target - h.step);
        }
        if (b->use_graphs && m >= 2) {
            const std::vector<int> key = step_args(b, m);
            if (launch_graph(b, key)) {
                b->launches += m;
                b->graph_launches += m;
                for (long long j = 0; j < m; ++j)
                    if (key[2 + 3 * j]) b->list_parity ^= 1;
                for (int id = 0; id < b->max_sims; ++id) {
                    HostSim &h = b->sims[id];
                    if (!h.used || !h.live) continue;
                    h.step += m;
                    if (h.target > 0 && h.step >= h.target) TRYS(freeze_sim(b, id));
                }
                i += m;
                continue;
            }
        }
        TRYS(ensure_list(b));
        // Does any simulation run the update procedure after this step (and
        // with the Eq. 7 shut-down)?
        int manage = 0, lpf = 0;
        for (int id = 0; id < b->max_sims; ++id) {
            const HostSim &h = b->sims[id];
            if (h.used && h.live && !h.dense && (h.step + 1) % h.dev.interval == 0) {
                manage = 1;
                lpf |= h.dev.lpf;
            }
        }
        cudaError_t e = launch_step(b->E, b->grid, b->list_parity, manage, b->stream);
        if (e == cudaSuccess && lpf) e = launch_lpf(b->E, b->lpf_grid, b->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return poison(b, TCM_EDEVICE);
        }
        b->launches += 1;
        if (manage) b->list_parity ^= 1;
        for (int id = 0; id < b->max_sims; ++id) {
            HostSim &h = b->sims[id];
            if (!h.used || !h.live) continue;
            h.step += 1;
            if (h.target > 0 && h.step >= h.target) TRYS(freeze_sim(b, id));
        }
        ++i;
    }
    return TCM_OK;
}

tcm_status sim_release(tcm_batch *b, int id)
{
    DeviceGuard g(b->device);
    HostSim &h = b->sims[id];
    if (!h.used) return TCM_EINVAL;
    if (h.primed) {
        TRY(launch_settle(b->E, b->stream));
        TRY(launch_release(b->E, id, h.brick_base, h.n_bricks, b->stream));
    }
    TRY(cudaStreamSynchronize(b->stream));
    if (h.kslabs) cudaFree(h.kslabs);
    if (h.lpf_a) cudaFree(h.lpf_a);
    range_free(b, h.brick_base, h.range_len);
    // the released entry stops stepping; clear it on the device
    SimDev zero{};
    TRY(cudaMemcpyAsync(b->E.sims + id, &zero, sizeof(SimDev), cudaMemcpyHostToDevice, b->stream));
    b->sims[id] = HostSim{};
    TRYS(upload_sources(b));
    TRY(cudaStreamSynchronize(b->stream));
    b->dirty_list = true;
    return TCM_OK;
}

HostSim *sim_of(const tcm_sim *s)
{
    if (!s || !s->b || s->id < 0 || s->id >= s->b->max_sims || !s->b->sims[s->id].used) return nullptr;
    return &s->b->sims[s->id];
}

// Make sure the simulation's initial state is on the device and the active
// list matches the current state (reads and diagnostics).
tcm_status ready_for_read(tcm_batch *b, int id)
{
    if (!b->sims[id].primed) TRYS(sim_prime(b, id));
    TRYS(ensure_list(b));
    return TCM_OK;
}

}  // namespace

bool tcm_internal_view(const tcm_sim *s, SimView *v, bool refresh_list)
{
    HostSim *h = sim_of(s);
    if (!h || !v) return false;
    tcm_batch *b = s->b;
    v->E = &b->E;
    v->device = b->device;
    v->stream = b->stream;
    v->started = h->primed;
    v->list_ok = !b->dirty_list;
    if (refresh_list && h->primed && b->dirty_list) {
        // an admission or removal since the last step: rebuild the active
        // list (one compaction launch on the batch's stream; no allocation)
        DeviceGuard g(b->device);
        v->list_ok = ensure_list(b) == TCM_OK;
    }
    v->step = h->step;
    v->list_parity = b->list_parity;
    v->sim = s->id;
    return true;
}

extern "C" {

tcm_status tcm_barrier_selftest(int device, int skew, double timeout_s, unsigned *err_out)
{
    if (!err_out || (skew != 0 && skew != 1) || !(timeout_s > 0.0) || timeout_s > 1.0) return TCM_EINVAL;
    *err_out = 0;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return TCM_EDEVICE;
    }
    DeviceGuard guard(device);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return TCM_EDEVICE;
    EngineState *st = nullptr;
    unsigned long long *ctr = nullptr;
    cudaStream_t q = nullptr;
    tcm_status rc = TCM_OK;
    const unsigned long long start = (unsigned long long)skew;
    unsigned err = 0;
    if (cudaMalloc(&st, sizeof(EngineState)) != cudaSuccess || cudaMalloc(&ctr, sizeof(*ctr)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemsetAsync(st, 0, sizeof(EngineState), q) != cudaSuccess ||
        cudaMemcpyAsync(ctr, &start, sizeof(start), cudaMemcpyHostToDevice, q) != cudaSuccess ||
        launch_barrier_selftest(st, ctr, sms, (unsigned long long)(timeout_s * 1e9), q) != cudaSuccess ||
        cudaMemcpyAsync(&err, &st->err, sizeof(err), cudaMemcpyDeviceToHost, q) != cudaSuccess ||
        cudaStreamSynchronize(q) != cudaSuccess)
        rc = TCM_EDEVICE;
    if (q) cudaStreamDestroy(q);
    if (ctr) cudaFree(ctr);
    if (st) cudaFree(st);
    if (rc != TCM_OK) {
        cudaGetLastError();
        return rc;
    }
    *err_out = err;
    return (err & ERR_TIMEOUT) ? TCM_ETIMEOUT : TCM_OK;
}

tcm_status tcm_slot_bytes(tcm_brick brick, int storage, size_t *out)
{
    if (!out || brick.bx != BX || brick.by != BY || brick.bz != BZ) return TCM_EINVAL;
    if (storage == TCM_STORAGE_MIXED) storage = TCM_STORAGE_F32;   // boxes sized for the widest
    if (storage != TCM_STORAGE_F32 && storage != TCM_STORAGE_BF16 && storage != TCM_STORAGE_F16) return TCM_EINVAL;
    *out = (size_t)slot_elems(storage) * storage_bytes(storage);
    return TCM_OK;
}

tcm_status tcm_create(const tcm_domain *domain, const tcm_velocity_model *velocity, double dx, double dt,
                      double threshold, tcm_brick brick, const tcm_options *options, tcm_sim **out)
{
    if (!out) return TCM_EINVAL;
    *out = nullptr;
    if (!options || options->storage == TCM_STORAGE_MIXED) return TCM_EINVAL;
    float c_max = 0.f;
    TRYS(check_sim_args(domain, velocity, dx, dt, threshold, brick, options->storage, options->threshold_mode,
                        options->decay_steps, &c_max));
    const long long n_bricks = ((domain->nx + BX - 1) / BX) * ((domain->ny + BY - 1) / BY) *
                               ((domain->nz + BZ - 1) / BZ);
    size_t slot_bytes = 0;
    tcm_slot_bytes(brick, options->storage, &slot_bytes);
    const size_t pool_bytes = options->pool_bytes ? options->pool_bytes
                                                  : (options->dense ? (size_t)n_bricks * slot_bytes : 0);
    if (pool_bytes / slot_bytes < 1) return TCM_EINVAL;
    if (options->dense && (long long)(pool_bytes / slot_bytes) < n_bricks) return TCM_ENOMEM;
    tcm_batch *b = nullptr;
    TRYS(batch_new(options->device, (cudaStream_t)options->stream, options->pool_ptr, pool_bytes, options->storage,
                   n_bricks, 1, &b));
    b->use_graphs = !options->no_graphs;
    b->E.prefetch = options->no_prefetch ? 0 : 1;
    DeviceGuard g(b->device);
    int id = -1;
    tcm_status st = sim_add(b, domain, velocity, dx, dt, c_max, threshold, options->threshold_mode,
                            options->decay_alpha, options->decay_steps, options->dense ? 1 : 0, -1, &id);
    if (st != TCM_OK) {
        tcm_batch_destroy(b);
        return st;
    }
    tcm_sim *s = new (std::nothrow) tcm_sim();
    if (!s) {
        tcm_batch_destroy(b);
        return TCM_ENOMEM;
    }
    s->b = b;
    s->id = id;
    s->owns_batch = true;
    b->handles[id] = s;
    *out = s;
    return TCM_OK;
}

tcm_status tcm_add_source(tcm_sim *s, int64_t x, int64_t y, int64_t z, const float *wavelet, int64_t n)
{
    HostSim *h = sim_of(s);
    if (!h || n < 0 || (n > 0 && !wavelet)) return TCM_EINVAL;
    if (x < 0 || y < 0 || z < 0 || x >= h->nx || y >= h->ny || z >= h->nz) return TCM_EINVAL;
    if (h->primed) return TCM_ESTATE;
    HostSrc q;
    q.brick = (int)(((z / BZ) * h->my + (y / BY)) * h->mx + (x / BX));
    q.local = (int)(((z % BZ) * BY + (y % BY)) * BX + (x % BX));
    q.start = h->step;
    q.w.assign(wavelet, wavelet + n);
    h->sources.push_back(std::move(q));
    return TCM_OK;
}

tcm_status tcm_set_schedule(tcm_sim *s, int interval, int neighbours)
{
    HostSim *h = sim_of(s);
    if (!h || interval < 0 || (neighbours != 6 && neighbours != 26)) return TCM_EINVAL;
    if (h->primed) return TCM_ESTATE;
    if (interval == 0) {
        // Eq. 5: n = dx * (cell length) / (2 c dt), cell length = the
        // shortest brick edge in nodes
        const int edge = std::min(BX, std::min(BY, BZ));
        const double n = h->c_max > 0.f ? h->dx * edge / (2.0 * (double)h->c_max * h->dt) : 1.0;
        interval = (int)std::max(1.0, std::min(std::floor(n), 1e6));
    }
    h->dev.interval = interval;
    h->dev.neighbours = neighbours;
    return TCM_OK;
}

tcm_status tcm_set_lpf_shutdown(tcm_sim *s, double pass, double stop)
{
    HostSim *h = sim_of(s);
    if (!h || !(pass > 0) || !(stop > pass) || !(stop <= 1)) return TCM_EINVAL;
    if (BX != BY || BX != BZ) return TCM_EINVAL;   // the filter region is a cube of bricks
    if (h->primed) return TCM_ESTATE;
    tcm_batch *b = s->b;
    DeviceGuard g(b->device);
    if (!b->lpf_grid) {
        b->lpf_grid = lpf_grid_size(b->device);
        if (b->lpf_grid <= 0) return TCM_EDEVICE;
    }
    if (!b->E.lpf_out) {
        const int cap = (int)std::min<long long>(b->n_slots, 65536);
        TRYS(dalloc(b, &b->E.lpf_out, (size_t)cap * 2 * BVOL));
        b->E.lpf_cap = cap;
    }
    // Centre rows of the 1-D operator P^T F^-1 diag(H) F P (zero-padding P of
    // LPF_L nodes to LPF_M, DFT F): A[i][j] = (1/M) sum_k H(k) cos(2 pi k
    // (i + C - j) / M) -- real because H(k) = H(M - k).  Summed in FP64 and
    // rounded once to binary32, the precision the filter runs in.
    std::vector<float> A((size_t)LPF_C * LPF_L);
    for (int i = 0; i < LPF_C; ++i)
        for (int j = 0; j < LPF_L; ++j) {
            double acc = 0.0;
            for (int k = 0; k < LPF_M; ++k) {
                const int kk = std::min(k, LPF_M - k);
                const double nu = kk / (LPF_M / 2.0);
                const double hk = nu <= pass ? 1.0 : nu >= stop ? 0.0 : 0.5 * (1.0 + std::cos(M_PI * (nu - pass) / (stop - pass)));
                acc += hk * std::cos(2.0 * M_PI * (double)k * (double)(i + LPF_C - j) / LPF_M);
            }
            A[(size_t)i * LPF_L + j] = (float)(acc / LPF_M);
        }
    if (!h->lpf_a) {
        if (cudaMalloc(&h->lpf_a, A.size() * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return TCM_ENOMEM;
        }
    }
    TRY(cudaMemcpyAsync(h->lpf_a, A.data(), A.size() * sizeof(float), cudaMemcpyHostToDevice, b->stream));
    TRY(cudaStreamSynchronize(b->stream));
    h->dev.lpf = 1;
    h->dev.lpf_a = h->lpf_a;
    TRYS(upload_sim_header(b, s->id));
    return TCM_OK;
}

tcm_status tcm_schedule(const tcm_sim *s, int *interval, int *neighbours)
{
    HostSim *h = sim_of(s);
    if (!h || !interval || !neighbours) return TCM_EINVAL;
    *interval = h->dev.interval;
    *neighbours = h->dev.neighbours;
    return TCM_OK;
}

tcm_status tcm_set_field(tcm_sim *s, const float *now, const float *prev)
{
    HostSim *h = sim_of(s);
    if (!h || !now || !prev) return TCM_EINVAL;
    if (h->primed) return TCM_ESTATE;
    const size_t n = (size_t)(h->nx * h->ny * h->nz);
    h->init_now.assign(now, now + n);
    h->init_prev.assign(prev, prev + n);
    h->have_field = true;
    return TCM_OK;
}

tcm_status tcm_step_async(tcm_sim *s, int64_t n)
{
    if (!sim_of(s) || n < 0) return TCM_EINVAL;
    if (!s->owns_batch) return TCM_ESTATE;
    return batch_step_async(s->b, n);
}

tcm_status tcm_sync(tcm_sim *s)
{
    if (!sim_of(s)) return TCM_EINVAL;
    return tcm_batch_sync(s->b);
}

tcm_status tcm_step(tcm_sim *s, int64_t n)
{
    tcm_status st = tcm_step_async(s, n);
    if (st != TCM_OK) return st;
    return tcm_sync(s);
}

tcm_status tcm_read_field_device(const tcm_sim *cs, int which, int64_t x0, int64_t y0, int64_t z0, int64_t wx,
                                 int64_t wy, int64_t wz, float *device_out)
{
    HostSim *h = sim_of(cs);
    if (!h || (which != 0 && which != 1) || wx < 0 || wy < 0 || wz < 0 || (!device_out && wx * wy * wz > 0))
        return TCM_EINVAL;
    tcm_batch *b = cs->b;
    DeviceGuard g(b->device);
    TRYS(ready_for_read(b, cs->id));
    TRY(launch_read_window(b->E, cs->id, (int)(h->step & 1), which, x0, y0, z0, wx, wy, wz, device_out,
                           b->stream));
    return TCM_OK;
}

tcm_status tcm_read_field(const tcm_sim *cs, int which, int64_t x0, int64_t y0, int64_t z0, int64_t wx,
                          int64_t wy, int64_t wz, float *host_out)
{
    HostSim *h = sim_of(cs);
    if (!h || (which != 0 && which != 1) || wx < 0 || wy < 0 || wz < 0 || (!host_out && wx * wy * wz > 0))
        return TCM_EINVAL;
    const long long n = wx * wy * wz;
    if (n == 0) return TCM_OK;
    tcm_batch *b = cs->b;
    DeviceGuard g(b->device);
    // page-locked host memory the device can address: the gather kernel
    // writes it directly
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, host_out) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer) {
        tcm_status st = tcm_read_field_device(cs, which, x0, y0, z0, wx, wy, wz, static_cast<float *>(pa.devicePointer));
        if (st == TCM_OK) st = dev_err(cudaStreamSynchronize(b->stream));
        return st;
    }
    cudaGetLastError();
    void *d = nullptr;
    TRYS(scratch(b, (size_t)n * sizeof(float), &d));
    tcm_status st = tcm_read_field_device(cs, which, x0, y0, z0, wx, wy, wz, static_cast<float *>(d));
    if (st == TCM_OK) {
        cudaError_t e = cudaMemcpyAsync(host_out, d, n * sizeof(float), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        st = dev_err(e);
    }
    return st;
}

tcm_status tcm_active_count(const tcm_sim *cs, int64_t *bricks, int64_t *cells)
{
    HostSim *h = sim_of(cs);
    if (!h) return TCM_EINVAL;
    tcm_batch *b = cs->b;
    DeviceGuard g(b->device);
    TRYS(ready_for_read(b, cs->id));
    void *sp = nullptr;
    TRYS(scratch(b, 2 * sizeof(unsigned long long), &sp));
    unsigned long long *d = static_cast<unsigned long long *>(sp);
    unsigned long long hc[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), b->stream);
    if (e == cudaSuccess) e = launch_active_bricks(b->E, cs->id, b->list_parity, nullptr, d, d + 1, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, d, sizeof(hc), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    TRY(e);
    if (bricks) *bricks = (int64_t)hc[0];
    if (cells) *cells = (int64_t)hc[1];
    return TCM_OK;
}

tcm_status tcm_active_bricks(const tcm_sim *cs, int64_t *ids, int64_t cap, int64_t *n)
{
    HostSim *h = sim_of(cs);
    if (!h || cap < 0 || (cap > 0 && !ids)) return TCM_EINVAL;
    tcm_batch *b = cs->b;
    DeviceGuard g(b->device);
    TRYS(ready_for_read(b, cs->id));
    const long long upper = h->n_bricks;
    void *sp = nullptr;
    TRYS(scratch(b, (size_t)(std::max<long long>(upper, 1) + 1) * sizeof(long long), &sp));
    unsigned long long *dn = static_cast<unsigned long long *>(sp);   // the count, then the ids
    long long *d = static_cast<long long *>(sp) + 1;
    unsigned long long hn = 0;
    cudaError_t e = cudaMemsetAsync(dn, 0, sizeof(unsigned long long), b->stream);
    if (e == cudaSuccess) e = launch_active_bricks(b->E, cs->id, b->list_parity, d, dn, nullptr, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hn, dn, sizeof(hn), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    std::vector<long long> hv((size_t)hn);
    if (e == cudaSuccess && hn > 0)
        e = cudaMemcpy(hv.data(), d, hn * sizeof(long long), cudaMemcpyDeviceToHost);
    TRY(e);
    std::sort(hv.begin(), hv.end());
    if (n) *n = (int64_t)hn;
    for (long long i = 0; i < (long long)hn && i < cap; ++i) ids[i] = hv[(size_t)i];
    return TCM_OK;
}

tcm_status tcm_updates(const tcm_sim *cs, int64_t *cell_updates)
{
    HostSim *h = sim_of(cs);
    if (!h || !cell_updates) return TCM_EINVAL;
    tcm_batch *b = cs->b;
    DeviceGuard g(b->device);
    unsigned long long u = 0;
    TRY(cudaMemcpyAsync(&u, &b->E.sims[cs->id].updates, sizeof(u), cudaMemcpyDeviceToHost, b->stream));
    TRY(cudaStreamSynchronize(b->stream));
    *cell_updates = (int64_t)u;
    return TCM_OK;
}

tcm_status tcm_energy(const tcm_sim *cs, double *e_out)
{
    HostSim *h = sim_of(cs);
    if (!h || !e_out) return TCM_EINVAL;
    tcm_batch *b = cs->b;
    DeviceGuard g(b->device);
    TRYS(ready_for_read(b, cs->id));
    void *sp = nullptr;
    TRYS(scratch(b, sizeof(double), &sp));
    double *d = static_cast<double *>(sp);
    double hv = 0.0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(double), b->stream);
    if (e == cudaSuccess) e = launch_energy(b->E, cs->id, (int)(h->step & 1), b->list_parity, d, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hv, d, sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    TRY(e);
    *e_out = hv;
    return TCM_OK;
}

tcm_status tcm_brick_media(const tcm_sim *cs, int64_t bi, int *kind, float *k)
{
    HostSim *h = sim_of(cs);
    if (!h || bi < 0 || bi >= h->n_bricks || !kind) return TCM_EINVAL;
    tcm_batch *b = cs->b;
    DeviceGuard g(b->device);
    int ks = 0;
    float kv = 0.f;
    TRY(cudaMemcpyAsync(&ks, b->E.kslab_of_brick + h->brick_base + bi, sizeof(int), cudaMemcpyDeviceToHost,
                        b->stream));
    TRY(cudaMemcpyAsync(&kv, b->E.kscal + h->brick_base + bi, sizeof(float), cudaMemcpyDeviceToHost, b->stream));
    TRY(cudaStreamSynchronize(b->stream));
    *kind = ks >= 0 ? 2 : 1;
    if (k) *k = ks >= 0 ? 0.f : kv;
    return TCM_OK;
}

tcm_status tcm_pool_info(const tcm_sim *cs, int64_t *slots, int64_t *free_slots)
{
    if (!sim_of(cs)) return TCM_EINVAL;
    return tcm_batch_info(cs->b, slots, free_slots, nullptr);
}

tcm_status tcm_phase_ns(const tcm_sim *cs, int64_t *stepping, int64_t *update, int64_t *compaction)
{
    if (!sim_of(cs)) return TCM_EINVAL;
    tcm_batch *b = cs->b;
    DeviceGuard g(b->device);
    EngineState es{};
    TRY(cudaMemcpyAsync(&es, b->E.st, sizeof(es), cudaMemcpyDeviceToHost, b->stream));
    TRY(cudaStreamSynchronize(b->stream));
    if (stepping) *stepping = (int64_t)es.phase_ns[0];
    if (update) *update = (int64_t)es.phase_ns[1];
    if (compaction) *compaction = (int64_t)es.phase_ns[2];
    return TCM_OK;
}

tcm_status tcm_lpf_info(const tcm_sim *cs, int64_t *ns, int64_t *bricks, int64_t *fma_per_brick)
{
    if (!sim_of(cs)) return TCM_EINVAL;
    tcm_batch *b = cs->b;
    DeviceGuard g(b->device);
    EngineState es{};
    TRY(cudaMemcpyAsync(&es, b->E.st, sizeof(es), cudaMemcpyDeviceToHost, b->stream));
    TRY(cudaStreamSynchronize(b->stream));
    if (ns) *ns = (int64_t)es.lpf_ns;
    if (bricks) *bricks = (int64_t)es.lpf_bricks;
    if (fma_per_brick) *fma_per_brick = (BX == BY && BX == BZ) ? LPF_FMA_PER_BRICK : 0;
    return TCM_OK;
}

int64_t tcm_launch_count(const tcm_sim *s) { return sim_of(s) ? s->b->launches : -1; }

int64_t tcm_graph_launch_count(const tcm_sim *s) { return sim_of(s) ? s->b->graph_launches : -1; }

int64_t tcm_step_index(const tcm_sim *s)
{
    HostSim *h = sim_of(s);
    return h ? h->step : -1;
}

const char *tcm_status_string(tcm_status st)
{
    switch (st) {
    case TCM_OK: return "ok";
    case TCM_EINVAL: return "invalid argument";
    case TCM_ECFL: return "CFL condition violated (Eq. 4)";
    case TCM_ENOMEM: return "out of memory (box pool exhausted or allocation failed)";
    case TCM_EDEVICE: return "CUDA error";
    case TCM_ETIMEOUT: return "device barrier timed out";
    case TCM_ESTATE: return "operation not allowed in this state";
    }
    return "unknown status";
}

void tcm_destroy(tcm_sim *s)
{
    if (!s) return;
    if (s->owns_batch) {
        tcm_batch_destroy(s->b);   // also deletes s
        return;
    }
    tcm_batch_remove(s->b, s);
}

// ---- batches --------------------------------------------------------------

tcm_status tcm_batch_create(const tcm_batch_options *o, tcm_batch **out)
{
    if (!out) return TCM_EINVAL;
    *out = nullptr;
    if (!o) return TCM_EINVAL;
    const tcm_status st = batch_new(o->device, (cudaStream_t)o->stream, o->pool_ptr, o->pool_bytes, o->storage,
                                    o->max_bricks, o->max_sims, out);
    if (st == TCM_OK) {
        (*out)->use_graphs = !o->no_graphs;
        (*out)->E.prefetch = o->no_prefetch ? 0 : 1;
    }
    return st;
}

tcm_status tcm_batch_add(tcm_batch *b, const tcm_domain *domain, const tcm_velocity_model *velocity, double dx,
                         double dt, double threshold, tcm_brick brick, int threshold_mode, float decay_alpha,
                         int decay_steps, int dense, int64_t n_steps, tcm_sim **out)
{
    if (!b || !out) return TCM_EINVAL;
    *out = nullptr;
    float c_max = 0.f;
    TRYS(check_sim_args(domain, velocity, dx, dt, threshold, brick, b->E.storage, threshold_mode, decay_steps,
                        &c_max));
    if (b->poisoned) return TCM_ESTATE;
    DeviceGuard g(b->device);
    int id = -1;
    TRYS(sim_add(b, domain, velocity, dx, dt, c_max, threshold, threshold_mode, decay_alpha, decay_steps,
                 dense ? 1 : 0, n_steps, &id));
    tcm_sim *s = new (std::nothrow) tcm_sim();
    if (!s) {
        sim_release(b, id);
        return TCM_ENOMEM;
    }
    s->b = b;
    s->id = id;
    s->owns_batch = false;
    b->handles[id] = s;
    *out = s;
    return TCM_OK;
}

tcm_status tcm_batch_step_async(tcm_batch *b, int64_t n)
{
    if (!b || n < 0) return TCM_EINVAL;
    return batch_step_async(b, n);
}

tcm_status tcm_batch_sync(tcm_batch *b)
{
    if (!b) return TCM_EINVAL;
    DeviceGuard g(b->device);
    if (b->poisoned && b->sticky != TCM_OK) return b->sticky;
    return sync_status(b);
}

tcm_status tcm_batch_step(tcm_batch *b, int64_t n)
{
    tcm_status st = tcm_batch_step_async(b, n);
    if (st != TCM_OK) return st;
    return tcm_batch_sync(b);
}

tcm_status tcm_sim_done(const tcm_sim *s, int *done)
{
    HostSim *h = sim_of(s);
    if (!h || !done) return TCM_EINVAL;
    *done = (h->target > 0 && h->step >= h->target) ? 1 : 0;
    return TCM_OK;
}

tcm_status tcm_batch_remove(tcm_batch *b, tcm_sim *s)
{
    if (!b || !s || s->b != b || !sim_of(s)) return TCM_EINVAL;
    const int id = s->id;
    tcm_status st = sim_release(b, id);
    b->handles[id] = nullptr;
    if (!s->owns_batch) delete s;
    return st;
}

tcm_status tcm_set_storage(tcm_sim *s, int storage)
{
    HostSim *h = sim_of(s);
    if (!h) return TCM_EINVAL;
    if (storage != TCM_STORAGE_F32 && storage != TCM_STORAGE_BF16 && storage != TCM_STORAGE_F16) return TCM_EINVAL;
    if (s->b->E.storage != ST_MIXED) return storage == s->b->E.storage ? TCM_OK : TCM_EINVAL;
    if (h->primed) return TCM_ESTATE;
    h->dev.storage = storage;
    return TCM_OK;
}

tcm_status tcm_batch_pause(tcm_sim *s)
{
    HostSim *h = sim_of(s);
    if (!h || s->owns_batch) return TCM_EINVAL;
    tcm_batch *b = s->b;
    if (b->poisoned) return TCM_ESTATE;
    if (h->paused || (h->target > 0 && h->step >= h->target)) return TCM_OK;   // nothing to do
    DeviceGuard g(b->device);
    TRYS(sim_prime(b, s->id));
    TRYS(freeze_sim(b, s->id));
    h->paused = true;
    return TCM_OK;
}

tcm_status tcm_batch_resume(tcm_sim *s)
{
    HostSim *h = sim_of(s);
    if (!h || s->owns_batch) return TCM_EINVAL;
    if (!h->paused) return TCM_OK;
    tcm_batch *b = s->b;
    if (b->poisoned) return TCM_ESTATE;
    DeviceGuard g(b->device);
    TRY(launch_thaw(b->E, s->id, h->brick_base / 32, h->range_len / 32, h->brick_base, h->n_bricks, b->stream));
    h->paused = false;
    h->live = true;
    h->dev.live = 1;
    b->dirty_list = true;
    return TCM_OK;
}

tcm_status tcm_batch_headroom(tcm_batch *b, int64_t steps, int64_t *boxes)
{
    if (!b || !boxes || steps < 0) return TCM_EINVAL;
    *boxes = 0;
    if (b->poisoned) return TCM_ESTATE;
    DeviceGuard g(b->device);
    TRYS(prime_all(b));
    bool any = false;
    for (const auto &h : b->sims) any = any || (h.used && h.live);
    if (!any || steps == 0) return TCM_OK;
    if (!b->reach_a) {
        TRYS(dalloc(b, &b->reach_a, (size_t)b->cap_bricks));
        TRYS(dalloc(b, &b->reach_b, (size_t)b->cap_bricks));
        TRYS(dalloc(b, &b->reach_count, 1));
    }
    // values move at most one node per step (Eq. 3 couples face neighbours
    // only), so in `steps` steps they reach cells within ceil(steps / L) cells
    // of a boxed cell, L the shortest cell edge; the update boxes at most the
    // neighbours of such cells
    const int L = std::min(BX, std::min(BY, BZ));
    const long long r = (steps + L - 1) / L + 1;
    const int rr = (int)std::min<long long>(r, 1 << 20);
    unsigned long long count = 0;
    TRY(cudaMemsetAsync(b->reach_count, 0, sizeof(unsigned long long), b->stream));
    TRY(launch_reach(b->E, rr, b->reach_a, b->reach_b, b->reach_count, b->stream));
    TRY(cudaMemcpyAsync(&count, b->reach_count, sizeof(count), cudaMemcpyDeviceToHost, b->stream));
    TRY(cudaStreamSynchronize(b->stream));
    *boxes = (int64_t)count;
    return TCM_OK;
}

tcm_status tcm_batch_info(const tcm_batch *cb, int64_t *slots, int64_t *free_slots, int *sims)
{
    tcm_batch *b = const_cast<tcm_batch *>(cb);
    if (!b) return TCM_EINVAL;
    DeviceGuard g(b->device);
    if (slots) *slots = b->n_slots;
    if (sims) {
        int n = 0;
        for (const auto &h : b->sims) n += h.used ? 1 : 0;
        *sims = n;
    }
    if (free_slots) {
        EngineState es{};
        TRY(cudaMemcpyAsync(&es, b->E.st, sizeof(es), cudaMemcpyDeviceToHost, b->stream));
        TRY(cudaStreamSynchronize(b->stream));
        *free_slots = std::max(es.free_top, 0) + es.n_retired;
    }
    return TCM_OK;
}

void tcm_batch_destroy(tcm_batch *b)
{
    if (!b) return;
    DeviceGuard g(b->device);
    cudaStreamSynchronize(b->stream);
    for (auto &h : b->sims) {
        if (h.kslabs) cudaFree(h.kslabs);
        if (h.lpf_a) cudaFree(h.lpf_a);
    }
    for (tcm_sim *s : b->handles) delete s;
    drop_graphs(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void *p : b->allocs) cudaFree(p);
    if (b->d_src) cudaFree(b->d_src);
    if (b->d_wave) cudaFree(b->d_wave);
    if (b->own_pool && b->pool) cudaFree(b->pool);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->scratch) cudaFree(b->scratch);
    delete b;
}

}  // extern "C"
