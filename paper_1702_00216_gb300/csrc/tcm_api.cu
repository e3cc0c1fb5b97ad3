// tcm_api.cu -- host runtime and C ABI of libtcm (see include/tcm.h).
//
// One tcm_sim owns one engine: the brick tables of its domain, the per-box
// metadata, the active lists and the step state, all resident in HBM; the
// boxes themselves live in the caller's pool (or one the library allocates).
// Everything a step needs stays on the device between calls; the host only
// launches one cooperative kernel per step and reads a status word per call.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "../../include/tcm.h"
#include "tcm_internal.cuh"

using namespace tcm;

struct tcm_sim {
    int device = 0;
    cudaStream_t stream = nullptr;
    Engine E{};
    SimDev simh{};
    long long nx = 0, ny = 0, nz = 0;
    int mx = 0, my = 0, mz = 0;
    long long n_bricks = 0, n_words = 0;
    int n_slots = 0;
    int grid = 0;
    bool own_pool = false;
    void *pool = nullptr;
    std::vector<void *> allocs;
    long long n_kslabs = 0;
    struct Source {
        int brick, local;
        long long start;
        std::vector<float> w;
    };
    std::vector<Source> sources;
    std::vector<float> init_now, init_prev;
    bool have_field = false;
    bool started = false;
    bool poisoned = false;
    tcm_status sticky = TCM_OK;
    long long step = 0;
    long long launches = 0;
    int list_parity = 0;
    unsigned *h_err = nullptr;  // pinned
};

namespace {

constexpr double INV_SQRT3 = 0.57735026918962576451;

tcm_status dev_err(cudaError_t e)
{
    if (e == cudaSuccess) return TCM_OK;
    if (e == cudaErrorMemoryAllocation) return TCM_ENOMEM;
    return TCM_EDEVICE;
}

#define TRY(expr)                                          \
    do {                                                   \
        tcm_status _s = dev_err(expr);                     \
        if (_s != TCM_OK) return _s;                       \
    } while (0)

template <typename T>
tcm_status dalloc(tcm_sim *s, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TCM_ENOMEM : TCM_EDEVICE;
    }
    s->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return TCM_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(d);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

tcm_status sync_status(tcm_sim *s)
{
    cudaError_t e = cudaMemcpyAsync(s->h_err, &s->E.st->err, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                    s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        s->poisoned = true;
        s->sticky = TCM_EDEVICE;
        return TCM_EDEVICE;
    }
    const unsigned err = *s->h_err;
    if (err & ERR_TIMEOUT) {
        s->poisoned = true;
        s->sticky = TCM_ETIMEOUT;
        return TCM_ETIMEOUT;
    }
    if (err & ERR_NOMEM) {
        s->poisoned = true;
        s->sticky = TCM_ENOMEM;
        return TCM_ENOMEM;
    }
    return TCM_OK;
}

// Box the initial bricks (source bricks and bricks holding initial values),
// in brick order, and hand every other box to the free stack.
tcm_status start(tcm_sim *s)
{
    if (s->started) return TCM_OK;
    DeviceGuard g(s->device);
    // sources -> device
    std::vector<SrcDev> src;
    std::vector<float> wave;
    for (const auto &q : s->sources) {
        SrcDev d{};
        d.sim = 0;
        d.brick = q.brick;
        d.local = q.local;
        d.start = q.start;
        d.len = (long long)q.w.size();
        d.w_off = (long long)wave.size();
        wave.insert(wave.end(), q.w.begin(), q.w.end());
        src.push_back(d);
    }
    SrcDev *d_src = nullptr;
    float *d_wave = nullptr;
    tcm_status st;
    if ((st = dalloc(s, &d_src, src.size())) != TCM_OK) return st;
    if ((st = dalloc(s, &d_wave, wave.size())) != TCM_OK) return st;
    if (!src.empty())
        TRY(cudaMemcpyAsync(d_src, src.data(), src.size() * sizeof(SrcDev), cudaMemcpyHostToDevice, s->stream));
    if (!wave.empty())
        TRY(cudaMemcpyAsync(d_wave, wave.data(), wave.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    // mark the source bricks in the per-brick state word
    for (const auto &q : s->sources) {
        const unsigned short bit = (unsigned short)FLAG_HAS_SRC;
        TRY(cudaMemcpyAsync(s->E.sd_of_brick + s->simh.brick_base + q.brick, &bit, sizeof(bit),
                            cudaMemcpyHostToDevice, s->stream));
        TRY(cudaStreamSynchronize(s->stream));
    }
    s->E.src = d_src;
    s->E.n_src = (int)src.size();
    s->E.wave = d_wave;
    s->simh.src_begin = 0;
    s->simh.src_end = (int)src.size();
    TRY(cudaMemcpyAsync(s->E.sims, &s->simh, sizeof(SimDev), cudaMemcpyHostToDevice, s->stream));

    // initial active set
    std::vector<long long> init;
    long long n_init = 0;
    const long long bvol = BVOL;
    if (s->simh.dense) {
        n_init = s->n_bricks;
    } else {
        std::vector<char> mark((size_t)s->n_bricks, 0);
        for (const auto &q : s->sources)
            if (!q.w.empty()) mark[(size_t)q.brick] = 1;
        if (s->have_field) {
            for (long long z = 0; z < s->nz; ++z)
                for (long long y = 0; y < s->ny; ++y)
                    for (long long x = 0; x < s->nx; ++x) {
                        const size_t id = (size_t)((z * s->ny + y) * s->nx + x);
                        if (s->init_now[id] != 0.f || s->init_prev[id] != 0.f)
                            mark[(size_t)(((z / BZ) * s->my + (y / BY)) * s->mx + (x / BX))] = 1;
                    }
        }
        for (long long b = 0; b < s->n_bricks; ++b)
            if (mark[(size_t)b]) init.push_back(b);
        n_init = (long long)init.size();
    }
    if (n_init > s->n_slots) {
        s->poisoned = true;
        s->sticky = TCM_ENOMEM;
        return TCM_ENOMEM;
    }
    long long *d_init = nullptr;
    if (!s->simh.dense && n_init > 0) {
        TRY(cudaMalloc(&d_init, n_init * sizeof(long long)));
        TRY(cudaMemcpyAsync(d_init, init.data(), n_init * sizeof(long long), cudaMemcpyHostToDevice, s->stream));
    }
    TRY(launch_prime(s->E, 0, d_init, n_init, 0, s->stream));
    TRY(launch_zero_slots(s->E, 0, n_init, s->stream));
    if (s->have_field && n_init > 0) {
        // pack the initial values of the boxed bricks
        std::vector<float> packed((size_t)(n_init * 2 * bvol), 0.f);
        for (long long i = 0; i < n_init; ++i) {
            const long long b = s->simh.dense ? i : init[(size_t)i];
            const long long cx = b % s->mx, cy = (b / s->mx) % s->my, cz = b / ((long long)s->mx * s->my);
            for (int e = 0; e < BVOL; ++e) {
                const long long x = cx * BX + e % BX, y = cy * BY + (e / BX) % BY, z = cz * BZ + e / (BX * BY);
                if (x >= s->nx || y >= s->ny || z >= s->nz) continue;
                const size_t id = (size_t)((z * s->ny + y) * s->nx + x);
                packed[(size_t)(i * 2 * bvol + e)] = s->init_now[id];
                packed[(size_t)(i * 2 * bvol + bvol + e)] = s->init_prev[id];
            }
        }
        float *d_packed = nullptr;
        TRY(cudaMalloc(&d_packed, packed.size() * sizeof(float)));
        TRY(cudaMemcpyAsync(d_packed, packed.data(), packed.size() * sizeof(float), cudaMemcpyHostToDevice,
                            s->stream));
        TRY(launch_scatter_field(s->E, d_packed, n_init, 0, (int)(s->step & 1), s->stream));
        TRY(cudaStreamSynchronize(s->stream));
        cudaFree(d_packed);
        std::vector<float>().swap(s->init_now);
        std::vector<float>().swap(s->init_prev);
    }
    // free stack: boxes n_init .. n_slots-1, lowest on top
    const int n_free = s->n_slots - (int)n_init;
    TRY(launch_iota_desc(s->E.free_stack, n_free, s->n_slots - 1, s->stream));
    EngineState es{};
    es.free_top = n_free;
    es.list_parity = 0;
    es.n_active[0] = (int)n_init;
    TRY(cudaMemcpyAsync(s->E.st, &es, sizeof(es), cudaMemcpyHostToDevice, s->stream));
    TRY(launch_compact(s->E, s->grid, 0, s->stream));
    TRY(cudaStreamSynchronize(s->stream));
    if (d_init) cudaFree(d_init);
    s->list_parity = 0;
    s->started = true;
    return TCM_OK;
}

float model_c_max(const tcm_domain *d, const tcm_velocity_model *v, bool *bad)
{
    *bad = false;
    float cmax = 0.f;
    if (v->kind == TCM_MEDIA_DENSE) {
        const long long n = d->nx * d->ny * d->nz;
        for (long long i = 0; i < n; ++i) {
            const float c = v->c[i];
            if (!(c >= 0.f) || std::isinf(c)) *bad = true;
            cmax = std::max(cmax, c);
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

}  // namespace

bool tcm_internal_view(const tcm_sim *s, SimView *v)
{
    if (!s || !v) return false;
    v->E = &s->E;
    v->device = s->device;
    v->stream = s->stream;
    v->started = s->started;
    v->step = s->step;
    v->list_parity = s->list_parity;
    return true;
}

extern "C" {

tcm_status tcm_slot_bytes(tcm_brick brick, int storage, size_t *out)
{
    if (!out || brick.bx != BX || brick.by != BY || brick.bz != BZ || storage != TCM_STORAGE_F32)
        return TCM_EINVAL;
    *out = (size_t)2 * BVOL * sizeof(float);
    return TCM_OK;
}

tcm_status tcm_create(const tcm_domain *domain, const tcm_velocity_model *velocity, double dx, double dt,
                      double threshold, tcm_brick brick, const tcm_options *options, tcm_sim **out)
{
    if (!out) return TCM_EINVAL;
    *out = nullptr;
    if (!domain || !velocity || !options) return TCM_EINVAL;
    if (domain->nx < 1 || domain->ny < 1 || domain->nz < 1) return TCM_EINVAL;
    if (domain->nx > (1LL << 30) || domain->ny > (1LL << 30) || domain->nz > (1LL << 30)) return TCM_EINVAL;
    if (!(dx > 0) || !(dt > 0) || !(threshold >= 0) || std::isinf(threshold)) return TCM_EINVAL;
    size_t slot_bytes = 0;
    if (tcm_slot_bytes(brick, options->storage, &slot_bytes) != TCM_OK) return TCM_EINVAL;
    if (options->threshold_mode != TCM_THR_ABSOLUTE && options->threshold_mode != TCM_THR_RELATIVE)
        return TCM_EINVAL;
    if (options->decay_steps < 0 || options->decay_steps > (int)SD_MASK) return TCM_EINVAL;
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
    const long long n_bricks = mx * my * mz;
    if (n_bricks > (1LL << 31) - 64) return TCM_EINVAL;
    // Eq. 4 with the largest velocity of the model.
    bool bad = false;
    const float cmax = model_c_max(domain, velocity, &bad);
    if (bad) return TCM_EINVAL;
    if ((double)cmax * dt / dx > INV_SQRT3) return TCM_ECFL;
    if (options->dense && options->pool_ptr == nullptr && options->pool_bytes == 0) {
        // default pool for the dense comparator: one box per brick
    }
    const size_t pool_bytes = options->pool_bytes ? options->pool_bytes
                                                  : (options->dense ? (size_t)n_bricks * slot_bytes : 0);
    const long long n_slots_ll = (long long)(pool_bytes / slot_bytes);
    if (n_slots_ll < 1) return TCM_EINVAL;
    const int n_slots = (int)std::min<long long>(n_slots_ll, (1LL << 31) - 64);
    if (options->dense && n_slots < n_bricks) return TCM_ENOMEM;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || options->device < 0 || options->device >= ndev) {
        cudaGetLastError();
        return TCM_EDEVICE;
    }
    DeviceGuard guard(options->device);
    tcm_sim *s = new (std::nothrow) tcm_sim();
    if (!s) return TCM_ENOMEM;
    s->device = options->device;
    s->stream = (cudaStream_t)options->stream;
    s->nx = domain->nx;
    s->ny = domain->ny;
    s->nz = domain->nz;
    s->mx = (int)mx;
    s->my = (int)my;
    s->mz = (int)mz;
    s->n_bricks = n_bricks;
    s->n_words = (n_bricks + 31) / 32;
    s->n_slots = n_slots;
    s->grid = step_grid_size(s->device);
    tcm_status st = TCM_OK;
    auto fail = [&](tcm_status e) {
        tcm_destroy(s);
        return e;
    };
    if (s->grid <= 0) return fail(TCM_EDEVICE);
    if (cudaMallocHost(&s->h_err, sizeof(unsigned)) != cudaSuccess) return fail(TCM_EDEVICE);

    // pool
    if (options->pool_ptr) {
        if (reinterpret_cast<uintptr_t>(options->pool_ptr) % 16 != 0) return fail(TCM_EINVAL);
        s->pool = options->pool_ptr;
    } else {
        if (cudaMalloc(&s->pool, (size_t)n_slots * slot_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(TCM_ENOMEM);
        }
        s->own_pool = true;
    }
    Engine &E = s->E;
    E.phi = static_cast<float *>(s->pool);
    E.n_slots = n_slots;
    E.n_words = s->n_words;
    E.words_per_block = (int)((s->n_words + s->grid - 1) / s->grid);
    if (E.words_per_block < 1) E.words_per_block = 1;
    const long long nb_pad = s->n_words * 32;
    float *kscal = nullptr;
    int *kslab_of_brick = nullptr;
    if ((st = dalloc(s, &E.slot_of_brick, nb_pad)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &kscal, nb_pad)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &kslab_of_brick, nb_pad)) != TCM_OK) return fail(st);
    E.kscal = kscal;
    E.kslab_of_brick = kslab_of_brick;
    if ((st = dalloc(s, &E.sd_of_brick, nb_pad)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.bitmap, s->n_words)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.blocktot, s->grid)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.meta, n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.rec, (size_t)n_slots * 8)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.items0, n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.items1, n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.listids, n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.free_stack, n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.retired, n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.newslots, n_slots)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.sims, 1)) != TCM_OK) return fail(st);
    if ((st = dalloc(s, &E.st, 1)) != TCM_OK) return fail(st);
    E.n_sims = 1;
    cudaStream_t q = s->stream;
    if (cudaMemsetAsync(E.slot_of_brick, 0xff, nb_pad * sizeof(int), q) != cudaSuccess ||
        cudaMemsetAsync(E.bitmap, 0, s->n_words * sizeof(unsigned), q) != cudaSuccess ||
        cudaMemsetAsync(E.sd_of_brick, 0, nb_pad * sizeof(unsigned short), q) != cudaSuccess ||
        cudaMemsetAsync(E.blocktot, 0, s->grid * sizeof(int), q) != cudaSuccess ||
        cudaMemsetAsync(E.st, 0, sizeof(EngineState), q) != cudaSuccess)
        return fail(TCM_EDEVICE);

    // Heterogenic Bulking, once (Media).
    MediaDev md{};
    md.kind = velocity->kind == TCM_MEDIA_DENSE ? MEDIA_DENSE : MEDIA_RULES;
    float *d_c = nullptr;
    double *d_lz = nullptr, *d_sph = nullptr;
    float *d_lc = nullptr, *d_sc = nullptr;
    int *d_cnt = nullptr;
    std::vector<void *> tmp;
    auto tmp_alloc = [&](void **p, size_t bytes) -> bool {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        tmp.push_back(*p);
        return true;
    };
    auto free_tmp = [&]() {
        for (void *p : tmp) cudaFree(p);
        tmp.clear();
    };
    const size_t n_nodes = (size_t)(domain->nx * domain->ny * domain->nz);
    bool ok = tmp_alloc((void **)&d_cnt, sizeof(int));
    if (ok && md.kind == MEDIA_DENSE) {
        ok = tmp_alloc((void **)&d_c, n_nodes * sizeof(float)) &&
             cudaMemcpyAsync(d_c, velocity->c, n_nodes * sizeof(float), cudaMemcpyHostToDevice, q) == cudaSuccess;
        md.c = d_c;
    } else if (ok) {
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
    if (!ok) {
        free_tmp();
        return fail(TCM_ENOMEM);
    }
    int n_kslabs = 0;
    if (cudaMemsetAsync(d_cnt, 0, sizeof(int), q) != cudaSuccess ||
        launch_bulk_classify(md, (int)s->nx, (int)s->ny, (int)s->nz, s->mx, s->my, s->mz, dt, dx, kscal,
                             kslab_of_brick, d_cnt, q) != cudaSuccess ||
        cudaMemcpyAsync(s->h_err, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, q) != cudaSuccess ||
        cudaStreamSynchronize(q) != cudaSuccess) {
        free_tmp();
        return fail(TCM_EDEVICE);
    }
    std::memcpy(&n_kslabs, s->h_err, sizeof(int));
    s->n_kslabs = n_kslabs;
    float *kslabs = nullptr;
    if ((st = dalloc(s, &kslabs, (size_t)n_kslabs * BVOL)) != TCM_OK) {
        free_tmp();
        return fail(st);
    }
    E.kslabs = kslabs;
    if (n_kslabs > 0 &&
        (launch_bulk_fill(md, (int)s->nx, (int)s->ny, (int)s->nz, s->mx, s->my, s->mz, dt, dx, kslab_of_brick,
                          kslabs, q) != cudaSuccess ||
         cudaStreamSynchronize(q) != cudaSuccess)) {
        free_tmp();
        return fail(TCM_EDEVICE);
    }
    cudaStreamSynchronize(q);
    free_tmp();

    SimDev &S = s->simh;
    S.nx = (int)s->nx;
    S.ny = (int)s->ny;
    S.nz = (int)s->nz;
    S.mx = s->mx;
    S.my = s->my;
    S.mz = s->mz;
    S.brick_base = 0;
    S.n_bricks = n_bricks;
    S.thr_mode = options->threshold_mode;
    S.dense = options->dense ? 1 : 0;
    S.tau = threshold;
    S.alpha = options->decay_alpha;
    S.decay_steps = options->decay_steps;
    S.step = 0;
    if (cudaMemcpyAsync(E.sims, &S, sizeof(SimDev), cudaMemcpyHostToDevice, q) != cudaSuccess ||
        cudaStreamSynchronize(q) != cudaSuccess)
        return fail(TCM_EDEVICE);
    *out = s;
    return TCM_OK;
}

tcm_status tcm_add_source(tcm_sim *s, int64_t x, int64_t y, int64_t z, const float *wavelet, int64_t n)
{
    if (!s || n < 0 || (n > 0 && !wavelet)) return TCM_EINVAL;
    if (x < 0 || y < 0 || z < 0 || x >= s->nx || y >= s->ny || z >= s->nz) return TCM_EINVAL;
    if (s->started) return TCM_ESTATE;
    tcm_sim::Source q;
    q.brick = (int)(((z / BZ) * s->my + (y / BY)) * s->mx + (x / BX));
    q.local = (int)(((z % BZ) * BY + (y % BY)) * BX + (x % BX));
    q.start = s->step;
    q.w.assign(wavelet, wavelet + n);
    s->sources.push_back(std::move(q));
    return TCM_OK;
}

tcm_status tcm_set_field(tcm_sim *s, const float *now, const float *prev)
{
    if (!s || !now || !prev) return TCM_EINVAL;
    if (s->started) return TCM_ESTATE;
    const size_t n = (size_t)(s->nx * s->ny * s->nz);
    s->init_now.assign(now, now + n);
    s->init_prev.assign(prev, prev + n);
    s->have_field = true;
    return TCM_OK;
}

tcm_status tcm_step_async(tcm_sim *s, int64_t n)
{
    if (!s || n < 0) return TCM_EINVAL;
    if (s->poisoned) return TCM_ESTATE;
    DeviceGuard g(s->device);
    tcm_status st = start(s);
    if (st != TCM_OK) return st;
    for (int64_t i = 0; i < n; ++i) {
        cudaError_t e = launch_step(s->E, s->grid, s->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->poisoned = true;
            s->sticky = TCM_EDEVICE;
            return TCM_EDEVICE;
        }
        s->step += 1;
        s->launches += 1;
        s->list_parity ^= 1;
    }
    return TCM_OK;
}

tcm_status tcm_sync(tcm_sim *s)
{
    if (!s) return TCM_EINVAL;
    DeviceGuard g(s->device);
    if (s->poisoned && s->sticky != TCM_OK) return s->sticky;
    return sync_status(s);
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
    tcm_sim *s = const_cast<tcm_sim *>(cs);
    if (!s || (which != 0 && which != 1) || wx < 0 || wy < 0 || wz < 0 || (!device_out && wx * wy * wz > 0))
        return TCM_EINVAL;
    DeviceGuard g(s->device);
    tcm_status st = start(s);
    if (st != TCM_OK) return st;
    const int half = which == 0 ? (int)(s->step & 1) : (int)((s->step + 1) & 1);
    TRY(launch_read_window(s->E, 0, half, x0, y0, z0, wx, wy, wz, device_out, s->stream));
    return TCM_OK;
}

tcm_status tcm_read_field(const tcm_sim *cs, int which, int64_t x0, int64_t y0, int64_t z0, int64_t wx,
                          int64_t wy, int64_t wz, float *host_out)
{
    tcm_sim *s = const_cast<tcm_sim *>(cs);
    if (!s || (which != 0 && which != 1) || wx < 0 || wy < 0 || wz < 0 || (!host_out && wx * wy * wz > 0))
        return TCM_EINVAL;
    const long long n = wx * wy * wz;
    if (n == 0) return TCM_OK;
    DeviceGuard g(s->device);
    float *d = nullptr;
    if (cudaMalloc(&d, n * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return TCM_ENOMEM;
    }
    tcm_status st = tcm_read_field_device(s, which, x0, y0, z0, wx, wy, wz, d);
    if (st == TCM_OK) {
        cudaError_t e = cudaMemcpyAsync(host_out, d, n * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        st = dev_err(e);
    }
    cudaFree(d);
    return st;
}

tcm_status tcm_active_count(const tcm_sim *cs, int64_t *bricks, int64_t *cells)
{
    tcm_sim *s = const_cast<tcm_sim *>(cs);
    if (!s) return TCM_EINVAL;
    DeviceGuard g(s->device);
    tcm_status st = start(s);
    if (st != TCM_OK) return st;
    unsigned long long *d = nullptr;
    TRY(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
    EngineState es{};
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), s->stream);
    if (e == cudaSuccess) e = launch_active_bricks(s->E, s->list_parity, nullptr, d, s->stream);
    unsigned long long hc = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, d, sizeof(hc), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&es, s->E.st, sizeof(es), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(d);
    TRY(e);
    if (bricks) *bricks = es.n_active[s->list_parity];
    if (cells) *cells = (int64_t)hc;
    return TCM_OK;
}

tcm_status tcm_active_bricks(const tcm_sim *cs, int64_t *ids, int64_t cap, int64_t *n)
{
    tcm_sim *s = const_cast<tcm_sim *>(cs);
    if (!s || cap < 0 || (cap > 0 && !ids)) return TCM_EINVAL;
    DeviceGuard g(s->device);
    tcm_status st = start(s);
    if (st != TCM_OK) return st;
    EngineState es{};
    TRY(cudaMemcpyAsync(&es, s->E.st, sizeof(es), cudaMemcpyDeviceToHost, s->stream));
    TRY(cudaStreamSynchronize(s->stream));
    const long long na = es.n_active[s->list_parity];
    if (n) *n = na;
    if (na == 0 || cap == 0) return TCM_OK;
    long long *d = nullptr;
    TRY(cudaMalloc(&d, na * sizeof(long long)));
    std::vector<long long> h((size_t)na);
    cudaError_t e = launch_active_bricks(s->E, s->list_parity, d, nullptr, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, na * sizeof(long long), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(d);
    TRY(e);
    std::sort(h.begin(), h.end());
    for (long long i = 0; i < na && i < cap; ++i) ids[i] = h[(size_t)i];
    return TCM_OK;
}

tcm_status tcm_updates(const tcm_sim *cs, int64_t *cell_updates)
{
    tcm_sim *s = const_cast<tcm_sim *>(cs);
    if (!s || !cell_updates) return TCM_EINVAL;
    DeviceGuard g(s->device);
    if (!s->started) {
        *cell_updates = 0;
        return TCM_OK;
    }
    EngineState es{};
    TRY(cudaMemcpyAsync(&es, s->E.st, sizeof(es), cudaMemcpyDeviceToHost, s->stream));
    TRY(cudaStreamSynchronize(s->stream));
    *cell_updates = (int64_t)es.updates;
    return TCM_OK;
}

tcm_status tcm_energy(const tcm_sim *cs, double *e_out)
{
    tcm_sim *s = const_cast<tcm_sim *>(cs);
    if (!s || !e_out) return TCM_EINVAL;
    DeviceGuard g(s->device);
    tcm_status st = start(s);
    if (st != TCM_OK) return st;
    double *d = nullptr;
    TRY(cudaMalloc(&d, sizeof(double)));
    double h = 0.0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(double), s->stream);
    if (e == cudaSuccess) e = launch_energy(s->E, 0, (int)(s->step & 1), s->list_parity, d, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(d);
    TRY(e);
    *e_out = h;
    return TCM_OK;
}

tcm_status tcm_brick_media(const tcm_sim *cs, int64_t b, int *kind, float *k)
{
    tcm_sim *s = const_cast<tcm_sim *>(cs);
    if (!s || b < 0 || b >= s->n_bricks || !kind) return TCM_EINVAL;
    DeviceGuard g(s->device);
    int ks = 0;
    float kv = 0.f;
    TRY(cudaMemcpyAsync(&ks, s->E.kslab_of_brick + b, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    TRY(cudaMemcpyAsync(&kv, s->E.kscal + b, sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    TRY(cudaStreamSynchronize(s->stream));
    *kind = ks >= 0 ? 2 : 1;
    if (k) *k = ks >= 0 ? 0.f : kv;
    return TCM_OK;
}

tcm_status tcm_pool_info(const tcm_sim *cs, int64_t *slots, int64_t *free_slots)
{
    tcm_sim *s = const_cast<tcm_sim *>(cs);
    if (!s) return TCM_EINVAL;
    DeviceGuard g(s->device);
    if (slots) *slots = s->n_slots;
    if (!free_slots) return TCM_OK;
    if (!s->started) {
        *free_slots = s->n_slots;
        return TCM_OK;
    }
    EngineState es{};
    TRY(cudaMemcpyAsync(&es, s->E.st, sizeof(es), cudaMemcpyDeviceToHost, s->stream));
    TRY(cudaStreamSynchronize(s->stream));
    *free_slots = std::max(es.free_top, 0) + es.n_retired;
    return TCM_OK;
}

tcm_status tcm_phase_ns(const tcm_sim *cs, int64_t *stepping, int64_t *update, int64_t *compaction)
{
    tcm_sim *s = const_cast<tcm_sim *>(cs);
    if (!s) return TCM_EINVAL;
    int64_t v[3] = {0, 0, 0};
    if (s->started) {
        DeviceGuard g(s->device);
        EngineState es{};
        TRY(cudaMemcpyAsync(&es, s->E.st, sizeof(es), cudaMemcpyDeviceToHost, s->stream));
        TRY(cudaStreamSynchronize(s->stream));
        for (int i = 0; i < 3; ++i) v[i] = (int64_t)es.phase_ns[i];
    }
    if (stepping) *stepping = v[0];
    if (update) *update = v[1];
    if (compaction) *compaction = v[2];
    return TCM_OK;
}

int64_t tcm_launch_count(const tcm_sim *s) { return s ? s->launches : -1; }

int64_t tcm_step_index(const tcm_sim *s) { return s ? s->step : -1; }

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
    DeviceGuard g(s->device);
    if (s->stream || true) cudaStreamSynchronize(s->stream);
    for (void *p : s->allocs) cudaFree(p);
    if (s->own_pool && s->pool) cudaFree(s->pool);
    if (s->h_err) cudaFreeHost(s->h_err);
    delete s;
}

}  // extern "C"
