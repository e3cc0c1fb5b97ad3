// tcm_dispatch.cpp -- the public C ABI of libtcm (include/tcm.h).
//
// The runtime and kernels are compiled once per supported brick shape, with
// every entry point renamed tcm_<shape>_<name> (4x4x4: b444, 8x8x8: b888,
// 16x8x8: b1688).  This file defines the public tcm_* functions: a
// simulation or batch handle records its shape and the handle of that
// shape's build, and every call goes to that build.
#include <cstdint>
#include <new>
#include <vector>
#include <algorithm>

#include "../../include/tcm.h"

struct tcm_sim {
    int shape;
    void *impl;
    tcm_batch *owner;   // batch that owns it, or null (tcm_create)
};

struct tcm_batch {
    int shape;
    void *impl;
    std::vector<tcm_sim *> sims;
};

#define DECL3(ret, name, params)             \
    extern "C" ret tcm_b444_##name params;   \
    extern "C" ret tcm_b888_##name params;   \
    extern "C" ret tcm_b1688_##name params;  \
    extern "C" ret tcm_b888w4_##name params; \
    extern "C" ret tcm_b888w12_##name params;

DECL3(tcm_status, slot_bytes, (tcm_brick, int, size_t *))
DECL3(tcm_status, create, (const tcm_domain *, const tcm_velocity_model *, double, double, double, tcm_brick,
                           const tcm_options *, void **))
DECL3(tcm_status, add_source, (void *, int64_t, int64_t, int64_t, const float *, int64_t))
DECL3(tcm_status, set_field, (void *, const float *, const float *))
DECL3(tcm_status, set_schedule, (void *, int, int))
DECL3(tcm_status, set_lpf_shutdown, (void *, double, double))
DECL3(tcm_status, schedule, (const void *, int *, int *))
DECL3(tcm_status, step, (void *, int64_t))
DECL3(tcm_status, step_async, (void *, int64_t))
DECL3(tcm_status, sync, (void *))
DECL3(tcm_status, read_field, (const void *, int, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, float *))
DECL3(tcm_status, read_field_device,
      (const void *, int, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, float *))
DECL3(tcm_status, active_count, (const void *, int64_t *, int64_t *))
DECL3(tcm_status, active_bricks, (const void *, int64_t *, int64_t, int64_t *))
DECL3(tcm_status, updates, (const void *, int64_t *))
DECL3(tcm_status, energy, (const void *, double *))
DECL3(tcm_status, energy_noalloc, (const void *, double *))
DECL3(tcm_status, brick_media, (const void *, int64_t, int *, float *))
DECL3(tcm_status, pool_info, (const void *, int64_t *, int64_t *))
DECL3(tcm_status, phase_ns, (const void *, int64_t *, int64_t *, int64_t *))
DECL3(int64_t, launch_count, (const void *))
DECL3(int64_t, graph_launch_count, (const void *))
DECL3(int64_t, step_index, (const void *))
DECL3(const char *, status_string, (tcm_status))
DECL3(tcm_status, barrier_selftest, (int, int, double, unsigned *))
DECL3(void, destroy, (void *))
DECL3(tcm_status, batch_create, (const tcm_batch_options *, void **))
DECL3(tcm_status, batch_add, (void *, const tcm_domain *, const tcm_velocity_model *, double, double, double,
                              tcm_brick, int, float, int, int, int64_t, void **))
DECL3(tcm_status, batch_step, (void *, int64_t))
DECL3(tcm_status, batch_step_async, (void *, int64_t))
DECL3(tcm_status, batch_sync, (void *))
DECL3(tcm_status, sim_done, (const void *, int *))
DECL3(tcm_status, batch_remove, (void *, void *))
DECL3(tcm_status, batch_info, (const void *, int64_t *, int64_t *, int *))
DECL3(void, batch_destroy, (void *))
DECL3(tcm_status, set_storage, (void *, int))
DECL3(tcm_status, batch_pause, (void *))
DECL3(tcm_status, batch_resume, (void *))
DECL3(tcm_status, batch_headroom, (void *, int64_t, int64_t *))
DECL3(tcm_status, lpf_info, (const void *, int64_t *, int64_t *, int64_t *))

// Call the build of `shape` (0 4x4x4, 1 8x8x8, 2 16x8x8, 3 8x8x8 with 4 warps
// per CTA, 4 8x8x8 with 12 warps per CTA).
#define SHAPE_CALL(shape, name, ...)                                                           \
    ((shape) == 0   ? tcm_b444_##name(__VA_ARGS__)                                              \
     : (shape) == 1 ? tcm_b888_##name(__VA_ARGS__)                                              \
     : (shape) == 2 ? tcm_b1688_##name(__VA_ARGS__)                                             \
     : (shape) == 3 ? tcm_b888w4_##name(__VA_ARGS__)                                            \
                    : tcm_b888w12_##name(__VA_ARGS__))

namespace {

// Build index of a brick shape and CTA blocking (warps per CTA of the step
// kernel), -1 if unsupported.  warps = 0 takes the default: 8, except 12 for
// 8x8x8 bricks with a 16-bit storage (measured fastest for those: the 16-bit
// time stepping is bound by instruction issue, and 12 warps keep more of it
// in flight).
int shape_of(tcm_brick b, int warps = 0, int storage = TCM_STORAGE_F32)
{
    const bool cube8 = b.bx == 8 && b.by == 8 && b.bz == 8;
    if (warps == 0) warps = cube8 && (storage == TCM_STORAGE_BF16 || storage == TCM_STORAGE_F16) ? 12 : 8;
    if (b.bx == 4 && b.by == 4 && b.bz == 4) return warps == 8 ? 0 : -1;
    if (cube8) return warps == 8 ? 1 : warps == 4 ? 3 : warps == 12 ? 4 : -1;
    if (b.bx == 16 && b.by == 8 && b.bz == 8) return warps == 8 ? 2 : -1;
    return -1;
}

// The blocking of a build (for adding to a batch: any shape index of the
// brick is the batch's if the brick matches).
bool same_brick(int shape, tcm_brick b)
{
    const int s = shape_of(b);
    return s >= 0 && (s == shape || (s == 1 && (shape == 3 || shape == 4)));
}

tcm_sim *wrap_sim(int shape, void *impl, tcm_batch *owner)
{
    tcm_sim *s = new (std::nothrow) tcm_sim();
    if (!s) return nullptr;
    s->shape = shape;
    s->impl = impl;
    s->owner = owner;
    return s;
}

void forget(tcm_sim *s)
{
    if (s->owner) {
        auto &v = s->owner->sims;
        v.erase(std::remove(v.begin(), v.end(), s), v.end());
    }
    delete s;
}

}  // namespace

#define SIM_OK(s) \
    if (!(s)) return TCM_EINVAL

extern "C" {

tcm_status tcm_slot_bytes(tcm_brick brick, int storage, size_t *out)
{
    const int sh = shape_of(brick);
    if (sh < 0) return TCM_EINVAL;
    return SHAPE_CALL(sh, slot_bytes, brick, storage, out);
}

tcm_status tcm_create(const tcm_domain *domain, const tcm_velocity_model *velocity, double dx, double dt,
                      double threshold, tcm_brick brick, const tcm_options *options, tcm_sim **out)
{
    if (!out) return TCM_EINVAL;
    *out = nullptr;
    if (!options) return TCM_EINVAL;
    const int sh = shape_of(brick, options->cta_warps, options->storage);
    if (sh < 0) return TCM_EINVAL;
    void *impl = nullptr;
    const tcm_status st = SHAPE_CALL(sh, create, domain, velocity, dx, dt, threshold, brick, options, &impl);
    if (st != TCM_OK) return st;
    tcm_sim *s = wrap_sim(sh, impl, nullptr);
    if (!s) {
        SHAPE_CALL(sh, destroy, impl);
        return TCM_ENOMEM;
    }
    *out = s;
    return TCM_OK;
}

tcm_status tcm_add_source(tcm_sim *s, int64_t x, int64_t y, int64_t z, const float *w, int64_t n)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, add_source, s->impl, x, y, z, w, n);
}

tcm_status tcm_set_field(tcm_sim *s, const float *now, const float *prev)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, set_field, s->impl, now, prev);
}

tcm_status tcm_set_schedule(tcm_sim *s, int interval, int neighbours)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, set_schedule, s->impl, interval, neighbours);
}

tcm_status tcm_set_lpf_shutdown(tcm_sim *s, double pass, double stop)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, set_lpf_shutdown, s->impl, pass, stop);
}

tcm_status tcm_schedule(const tcm_sim *s, int *interval, int *neighbours)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, schedule, s->impl, interval, neighbours);
}

tcm_status tcm_step(tcm_sim *s, int64_t n)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, step, s->impl, n);
}

tcm_status tcm_step_async(tcm_sim *s, int64_t n)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, step_async, s->impl, n);
}

tcm_status tcm_sync(tcm_sim *s)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, sync, s->impl);
}

tcm_status tcm_read_field(const tcm_sim *s, int which, int64_t x0, int64_t y0, int64_t z0, int64_t wx, int64_t wy,
                          int64_t wz, float *out)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, read_field, s->impl, which, x0, y0, z0, wx, wy, wz, out);
}

tcm_status tcm_read_field_device(const tcm_sim *s, int which, int64_t x0, int64_t y0, int64_t z0, int64_t wx,
                                 int64_t wy, int64_t wz, float *out)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, read_field_device, s->impl, which, x0, y0, z0, wx, wy, wz, out);
}

tcm_status tcm_active_count(const tcm_sim *s, int64_t *bricks, int64_t *cells)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, active_count, s->impl, bricks, cells);
}

tcm_status tcm_active_bricks(const tcm_sim *s, int64_t *ids, int64_t cap, int64_t *n)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, active_bricks, s->impl, ids, cap, n);
}

tcm_status tcm_updates(const tcm_sim *s, int64_t *u)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, updates, s->impl, u);
}

tcm_status tcm_energy(const tcm_sim *s, double *e)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, energy, s->impl, e);
}

tcm_status tcm_energy_noalloc(const tcm_sim *s, double *device_out)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, energy_noalloc, s->impl, device_out);
}

tcm_status tcm_brick_media(const tcm_sim *s, int64_t b, int *kind, float *k)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, brick_media, s->impl, b, kind, k);
}

tcm_status tcm_pool_info(const tcm_sim *s, int64_t *slots, int64_t *free_slots)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, pool_info, s->impl, slots, free_slots);
}

tcm_status tcm_phase_ns(const tcm_sim *s, int64_t *a, int64_t *b, int64_t *c)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, phase_ns, s->impl, a, b, c);
}

tcm_status tcm_lpf_info(const tcm_sim *s, int64_t *ns, int64_t *bricks, int64_t *fma_per_brick)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, lpf_info, s->impl, ns, bricks, fma_per_brick);
}

int64_t tcm_launch_count(const tcm_sim *s) { return s ? SHAPE_CALL(s->shape, launch_count, s->impl) : -1; }

int64_t tcm_graph_launch_count(const tcm_sim *s)
{
    return s ? SHAPE_CALL(s->shape, graph_launch_count, s->impl) : -1;
}

int64_t tcm_step_index(const tcm_sim *s) { return s ? SHAPE_CALL(s->shape, step_index, s->impl) : -1; }

const char *tcm_status_string(tcm_status st) { return tcm_b888_status_string(st); }

// The barrier does not depend on the brick shape: the 8x8x8 build runs it.
tcm_status tcm_barrier_selftest(int device, int skew, double timeout_s, unsigned *err_out)
{
    return tcm_b888_barrier_selftest(device, skew, timeout_s, err_out);
}

void tcm_destroy(tcm_sim *s)
{
    if (!s) return;
    SHAPE_CALL(s->shape, destroy, s->impl);
    forget(s);
}

tcm_status tcm_batch_create(const tcm_batch_options *o, tcm_batch **out)
{
    if (!out) return TCM_EINVAL;
    *out = nullptr;
    if (!o) return TCM_EINVAL;
    tcm_brick br = o->brick;
    if (br.bx == 0 && br.by == 0 && br.bz == 0) br = tcm_brick{8, 8, 8};
    const int sh = shape_of(br, o->cta_warps, o->storage);
    if (sh < 0) return TCM_EINVAL;
    void *impl = nullptr;
    const tcm_status st = SHAPE_CALL(sh, batch_create, o, &impl);
    if (st != TCM_OK) return st;
    tcm_batch *b = new (std::nothrow) tcm_batch();
    if (!b) {
        SHAPE_CALL(sh, batch_destroy, impl);
        return TCM_ENOMEM;
    }
    b->shape = sh;
    b->impl = impl;
    *out = b;
    return TCM_OK;
}

tcm_status tcm_batch_add(tcm_batch *b, const tcm_domain *domain, const tcm_velocity_model *velocity, double dx,
                         double dt, double threshold, tcm_brick brick, int threshold_mode, float decay_alpha,
                         int decay_steps, int dense, int64_t n_steps, tcm_sim **out)
{
    if (!b || !out) return TCM_EINVAL;
    *out = nullptr;
    if (!same_brick(b->shape, brick)) return TCM_EINVAL;
    void *impl = nullptr;
    const tcm_status st = SHAPE_CALL(b->shape, batch_add, b->impl, domain, velocity, dx, dt, threshold, brick,
                                     threshold_mode, decay_alpha, decay_steps, dense, n_steps, &impl);
    if (st != TCM_OK) return st;
    tcm_sim *s = wrap_sim(b->shape, impl, b);
    if (!s) {
        SHAPE_CALL(b->shape, batch_remove, b->impl, impl);
        return TCM_ENOMEM;
    }
    b->sims.push_back(s);
    *out = s;
    return TCM_OK;
}

tcm_status tcm_batch_step(tcm_batch *b, int64_t n)
{
    if (!b) return TCM_EINVAL;
    return SHAPE_CALL(b->shape, batch_step, b->impl, n);
}

tcm_status tcm_batch_step_async(tcm_batch *b, int64_t n)
{
    if (!b) return TCM_EINVAL;
    return SHAPE_CALL(b->shape, batch_step_async, b->impl, n);
}

tcm_status tcm_batch_sync(tcm_batch *b)
{
    if (!b) return TCM_EINVAL;
    return SHAPE_CALL(b->shape, batch_sync, b->impl);
}

tcm_status tcm_sim_done(const tcm_sim *s, int *done)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, sim_done, s->impl, done);
}

tcm_status tcm_batch_remove(tcm_batch *b, tcm_sim *s)
{
    if (!b || !s || s->owner != b) return TCM_EINVAL;
    // the build releases its handle whatever the status
    const tcm_status st = SHAPE_CALL(b->shape, batch_remove, b->impl, s->impl);
    forget(s);
    return st;
}

tcm_status tcm_set_storage(tcm_sim *s, int storage)
{
    SIM_OK(s);
    return SHAPE_CALL(s->shape, set_storage, s->impl, storage);
}

tcm_status tcm_batch_pause(tcm_sim *s)
{
    SIM_OK(s);
    if (!s->owner) return TCM_EINVAL;
    return SHAPE_CALL(s->shape, batch_pause, s->impl);
}

tcm_status tcm_batch_resume(tcm_sim *s)
{
    SIM_OK(s);
    if (!s->owner) return TCM_EINVAL;
    return SHAPE_CALL(s->shape, batch_resume, s->impl);
}

tcm_status tcm_batch_headroom(tcm_batch *b, int64_t steps, int64_t *boxes)
{
    if (!b) return TCM_EINVAL;
    return SHAPE_CALL(b->shape, batch_headroom, b->impl, steps, boxes);
}

tcm_status tcm_batch_info(const tcm_batch *b, int64_t *slots, int64_t *free_slots, int *sims)
{
    if (!b) return TCM_EINVAL;
    return SHAPE_CALL(b->shape, batch_info, b->impl, slots, free_slots, sims);
}

void tcm_batch_destroy(tcm_batch *b)
{
    if (!b) return;
    SHAPE_CALL(b->shape, batch_destroy, b->impl);
    for (tcm_sim *s : b->sims) delete s;
    delete b;
}

}  // extern "C"
