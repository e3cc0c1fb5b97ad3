/*
 * tcm.h -- C ABI of the GB300 Triggered Cells Method library (libtcm.so).
 *
 * Method: Naeh, "Handling massive spatial volumes in time domain simulations
 * using Triggered Cells Method", arXiv:1702.00216.  One time step advances the
 * 3D scalar wave equation (Eq. 1) with the second-order central-difference
 * update of Eq. 3,
 *     phi^{n+1} = 2 phi^n - phi^{n-1} + k (sum of 6 neighbours - 6 phi^n),
 *     k = (c dt / dx)^2,
 * but only on the triggered cells ("bricks"), each held in a box ("slot") of
 * an on-device pool (Boxes, Fig. 1), with the media bulked once (Heterogenic
 * Bulking Method, Media), sources inserted into forced-active cells (Source
 * insertion), the trigger/retire procedure run every step (Updating active
 * cells, Fig. 3a) and an optional time-domain shut-down (Eq. 6).
 *
 * Conventions
 *  - All field and velocity arrays are x fastest: index = (z*ny + y)*nx + x.
 *  - Every function returns a tcm_status; no exception, abort or device trap
 *    crosses this interface.  After an error the simulation stays readable.
 *  - Host pointers are read (or written) only during the call; the library
 *    keeps its own copies.  Device memory passed in tcm_options.pool_ptr stays
 *    owned by the caller and must outlive the simulation.
 *  - Work is issued on tcm_options.stream (a cudaStream_t; NULL = the legacy
 *    default stream) of device tcm_options.device.
 *  - Arithmetic: binary32 round-to-nearest, no contraction into FMA, no
 *    flush-to-zero, one fixed grouping of Eq. 3:
 *        s = ((((xm + xp) + ym) + yp) + zm) + zp;  lap = s - 6 p;
 *        q = (2 p - pm) + k lap;   then + source sample;  then * alpha in shut-down.
 *    Results are bit-for-bit reproducible and independent of scheduling.
 *  - Nodes outside the domain read as zero (zero Dirichlet boundary); the
 *    domain need not be a multiple of the brick size.
 */
#ifndef TCM_H
#define TCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tcm_sim tcm_sim; /* opaque, library-owned */

typedef enum {
    TCM_OK = 0,
    TCM_EINVAL = 1,   /* bad argument (sizes, pointers, brick shape, source outside) */
    TCM_ECFL = 2,     /* max(c) dt / dx > 1/sqrt(3): violates Eq. 4 */
    TCM_ENOMEM = 3,   /* pool exhausted (or a device allocation failed) */
    TCM_EDEVICE = 4,  /* a CUDA call failed */
    TCM_ETIMEOUT = 5, /* a device-wide barrier gave up waiting (bounded spin) */
    TCM_ESTATE = 6    /* call not allowed in this state (e.g. after ENOMEM) */
} tcm_status;

enum { TCM_MEDIA_DENSE = 0, TCM_MEDIA_RULES = 1 };
enum { TCM_THR_ABSOLUTE = 0, TCM_THR_RELATIVE = 1 };
/* Field storage in the pool.  F32: binary32, a box holds phi^n and phi^{n-1}.
 * BF16 / F16: bfloat16 or IEEE binary16 holding value / s, with s a power of
 * two per simulation (1 for BF16; for F16 chosen when the simulation starts
 * so that its largest source sample or initial value is stored in
 * [128, 256)); a box holds phi^n, the phi^{n+1} being written and
 * v^n = phi^n - phi^{n-1} (the velocity form of Eq. 3: v' = v + k lap,
 * phi^{n+1} = phi^n + v', so rounding a stored phi does not act on the
 * velocity).  Every storage computes in binary32 with binary32 k; values are
 * rounded to nearest-even on store.  With 16-bit storage, reading phi^{n-1}
 * returns phi^n - v^n (binary32). */
enum { TCM_STORAGE_F32 = 0, TCM_STORAGE_BF16 = 1, TCM_STORAGE_F16 = 2 };
/* Batches only (tcm_batch_options.storage): every simulation of the batch has
 * its own storage, chosen with tcm_set_storage (F32 by default), and all of
 * them step in the same launches.  Boxes are sized for binary32 (the widest:
 * 8 bytes per node), so a 16-bit simulation leaves a quarter of its boxes
 * unused. */
enum { TCM_STORAGE_MIXED = 3 };

typedef struct {
    int64_t nx, ny, nz; /* nodes */
} tcm_domain;

/* Velocity model (Media).  DENSE: c is a host array of nx*ny*nz floats.
 * RULES: c = c_background; then for each layer m in order c = layer_c[m]
 * where z >= layer_z[m]; then for each sphere s in order c = sphere_c[s] where
 * (x-X)^2 + (y-Y)^2 + (z-Z)^2 <= R^2 with sphere_xyzr[4s..4s+3] = X,Y,Z,R
 * (node-index units, FP64).  Rules are evaluated once, at tcm_create. */
typedef struct {
    int kind;
    const float *c;
    float c_background;
    int n_layers;
    const double *layer_z;
    const float *layer_c;
    int n_spheres;
    const double *sphere_xyzr;
    const float *sphere_c;
} tcm_velocity_model;

/* Brick ("cell") shape in nodes.  Supported: 4x4x4, 8x8x8 and 16x8x8
 * (bx x by x bz); a batch holds one shape.  The library is built once per
 * shape; a simulation or batch runs on the build of its shape. */
typedef struct {
    int bx, by, bz;
} tcm_brick;

typedef struct {
    int threshold_mode; /* TCM_THR_ABSOLUTE: level = threshold;
                           TCM_THR_RELATIVE: level = threshold * max|phi^{n+1}| (FP64) */
    float decay_alpha;  /* Eq. 6 factor per shut-down step */
    int decay_steps;    /* Eq. 6 n; 0 = release a quiet brick at once */
    void *pool_ptr;     /* device memory for the boxes, or NULL: library allocates */
    size_t pool_bytes;  /* size of the pool (caps the number of boxes) */
    void *stream;       /* cudaStream_t */
    int storage;        /* TCM_STORAGE_F32 / _BF16 / _F16 */
    int dense;          /* 1: box every brick and never release (dense comparator) */
    int device;         /* CUDA device ordinal */
    int no_graphs;      /* 1: issue every step launch directly; 0: runs of launches up to
                           the next change of the batch are captured once as a CUDA graph
                           and replayed (same kernels, same results) */
    int no_prefetch;    /* 1: no L2 prefetch in the time stepping; 0: while a warp steps a
                           brick pair it asks L2 for the next pair's field arrays and
                           per-node k (bricks with per-node k only).  Same results
                           either way */
    int cta_warps;      /* warps per CTA of the step kernel: 8 (every brick shape), 4 or
                           12 (8x8x8 only); 0: 8, except 12 for 8x8x8 bricks with a
                           16-bit storage.  Same results, different blocking
                           (TCM_EINVAL otherwise) */
} tcm_options;

/* Bytes of pool one box takes for this brick shape and storage (binary32:
 * two field arrays of 4 B per node; 16-bit: three arrays of 2 B per node).
 * TCM_EINVAL for unsupported shapes or storages. */
tcm_status tcm_slot_bytes(tcm_brick brick, int storage, size_t *out);

/* Create a simulation (Cells construction, Media / HBM bulking, Boxes).
 * dx, dt > 0; threshold >= 0.  Checks Eq. 4 on the largest velocity of the
 * model (TCM_ECFL) before touching the GPU.  Allocates the brick tables
 * (about 12 bytes per brick of the whole domain), per-box metadata, and the
 * bulked coefficient arrays of heterogeneous bricks.  *out is NULL on error. */
tcm_status tcm_create(const tcm_domain *domain, const tcm_velocity_model *velocity, double dx,
                      double dt, double threshold, tcm_brick brick, const tcm_options *options,
                      tcm_sim **out);

/* Add a point source at node (x,y,z) (Source insertion): sample i of the
 * wavelet is added to phi^{s+i+1} at that node, s = the step index at the time
 * of the call, and the source's brick is forced active while samples remain.
 * Only before the first tcm_step.  The wavelet is copied. */
tcm_status tcm_add_source(tcm_sim *sim, int64_t x, int64_t y, int64_t z, const float *wavelet,
                          int64_t n_samples);

/* Initial fields phi^0 and phi^{-1} (host arrays, nx*ny*nz).  Bricks holding a
 * non-zero value in either become active, and the update procedure runs once
 * on this state before the first step (bricks across a face whose max |phi^0|
 * is above the level become active too; with the 26-neighbour set, all
 * neighbours of a brick above the level).  Only before the first tcm_step. */
tcm_status tcm_set_field(tcm_sim *sim, const float *phi_now, const float *phi_prev);

/* Schedule of the update procedure (Simulation section, Eq. 5, Fig. 3).
 * interval >= 1: the procedure runs after every interval-th step of this
 * simulation (after step n when (n+1) % interval == 0); launches in between
 * only step the active bricks.  interval = 0: Eq. 5, n = dx * L / (2 c_max
 * dt) rounded down (at least 1), L = the shortest brick edge in nodes (8 for
 * 8^3 bricks).  A run covers
 * the steps up to the next one: a source brick fed in any of them is kept or
 * boxed, and a shut-down count (in time steps) drops by interval.
 * neighbours = 6 (default): a brick stays if its maximum or the touching face
 * of a boxed face neighbour is above the level; each face above the level
 * boxes the brick across it.  neighbours = 26: a brick is triggered if its
 * maximum is above the level or a source feeds it; it stays if it or a boxed
 * one of its 26 neighbours is triggered by its maximum; a triggered brick
 * boxes all 26 neighbours (the paper's nearest and diagonal cells) -- with
 * interval <= L and threshold 0 this equals the dense grid exactly.
 * Default interval 1, neighbours 6.  Only before the first step (TCM_ESTATE
 * after); TCM_EINVAL for interval < 0 or another neighbour count. */
tcm_status tcm_set_schedule(tcm_sim *sim, int interval, int neighbours);
/* Frequency-domain shut-down (Eq. 7) instead of the time-domain decay of
 * Eq. 6: at a run of the update procedure a brick that is not kept is
 * released at once, and every boxed brick that stays (not claimed by this
 * run) with such a released brick among its 26 neighbours -- one that held a
 * non-zero value -- gets both time levels replaced by
 * Phi~ = F^-1[F(Phi) LPF] evaluated on its 3x3x3-brick block (L = 3 brick
 * edges per axis, e.g. 24^3 nodes for 8^3 bricks; released, unboxed and
 * outside bricks read zero) zero-padded to M^3, M the power of two >= 2 L
 * (spatial oversampling; 64 for 8^3 bricks), LPF = H(kx) H(ky) H(kz), H = 1 up to `pass`, 0
 * from `stop` (fractions of the Nyquist frequency), raised cosine between;
 * the centre brick of the result is kept.  The filter is applied as the
 * separable operator equal to that transform (its centre rows, computed in
 * FP64 and rounded once to binary32) in binary32 FMA arithmetic, x, y, z in
 * turn, each output summed over the taps in increasing order; against exact
 * arithmetic the result is within 3 (L + 1) 2^-24 |A|^3 max|Phi| per
 * application, |A| the largest absolute row sum of the 1-D operator (about
 * 1.5 at pass 0.25, stop 0.5), then rounded to the storage.  All filtered values come from the state before any is
 * written.  decay_alpha / decay_steps are then unused.  0 < pass < stop <= 1
 * and cubic bricks (TCM_EINVAL otherwise); only before the first step
 * (TCM_ESTATE).  At most
 * 65536 bricks are filtered per run (beyond that the batch reports
 * TCM_ENOMEM). */
tcm_status tcm_set_lpf_shutdown(tcm_sim *sim, double pass, double stop);

/* The schedule in use (interval resolved when 0 was given). */
tcm_status tcm_schedule(const tcm_sim *sim, int *interval, int *neighbours);

/* Advance n steps; returns when they are done (or failed).  TCM_ENOMEM: the
 * pool ran out, the step completed without the bricks that found no box and
 * the simulation is poisoned (later steps return TCM_ESTATE). */
tcm_status tcm_step(tcm_sim *sim, int64_t n);

/* Enqueue n steps on the stream and return at once; tcm_sync reports the
 * status of everything enqueued. */
tcm_status tcm_step_async(tcm_sim *sim, int64_t n);
tcm_status tcm_sync(tcm_sim *sim);

/* Copy a window of phi^n (which = 0) or phi^{n-1} (which = 1) into host_out
 * (wx*wy*wz floats, x fastest).  Zeros where a brick is inactive or the window
 * leaves the domain.  The _device variant writes device memory on the stream.
 * Page-locked host memory the device can address is written directly by the
 * device; other host memory goes through a device staging buffer that the
 * batch keeps (grown to the largest window read so far, freed with the
 * batch), as do the small buffers of tcm_active_count, tcm_active_bricks and
 * tcm_energy: these calls allocate device memory only when their need grows. */
tcm_status tcm_read_field(const tcm_sim *sim, int which, int64_t x0, int64_t y0, int64_t z0,
                          int64_t wx, int64_t wy, int64_t wz, float *host_out);
tcm_status tcm_read_field_device(const tcm_sim *sim, int which, int64_t x0, int64_t y0,
                                 int64_t z0, int64_t wx, int64_t wy, int64_t wz,
                                 float *device_out);

/* Active (boxed) bricks for the next step, and the in-domain nodes they
 * hold; a frozen batch simulation reports the set it ended with. */
tcm_status tcm_active_count(const tcm_sim *sim, int64_t *bricks, int64_t *cells);

/* Sorted ids (z*my*mx + y*mx + x over the brick grid) of the active bricks;
 * *n = how many there are, at most cap are written. */
tcm_status tcm_active_bricks(const tcm_sim *sim, int64_t *ids, int64_t cap, int64_t *n);

/* Cumulative node updates (sum over steps of active in-domain nodes). */
tcm_status tcm_updates(const tcm_sim *sim, int64_t *cell_updates);

/* Discrete leapfrog energy between phi^n and phi^{n-1}:
 *   E = sum (phi^n - phi^{n-1})^2 / k + sum phi^n (6 phi^{n-1} - sum of 6 neighbours of phi^{n-1})
 * over active bricks, accumulated in FP64 on the device.  Constant once the
 * sources have stopped while no brick is released (threshold 0). */
tcm_status tcm_energy(const tcm_sim *sim, double *e);

/* The same energy as tcm_energy, written to device memory (*device_out, one
 * double) on the simulation's stream, without allocating any device memory.
 * The paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc/cudaFree while the simulation runs -- programs whose device
 * memory belongs to another allocator with a fixed budget, and code on a
 * latency-critical path that must not synchronise the device (freeing memory
 * does).  Its scratch is a static 512 KiB device array (one partial sum per
 * entry of the active list) that every GPU loading the library holds until
 * exit.  The active list is the batch's: it holds the active bricks of every
 * simulation of the batch (a simulation made by tcm_create is a batch of
 * one), so the limit of 65536 entries counts them all -- a longer list
 * returns TCM_EINVAL, even for a small simulation in a busy batch.  The first
 * call on a device looks up the array's device address; make that first call
 * before any stream capture.  The array is shared by all calls and keeps the
 * last call's partial sums (each call overwrites what it reads), so calls
 * whose work overlaps on the GPU race: serialise them.  Only after the
 * simulation has started, i.e. after its first step or read (TCM_ESTATE
 * before); if simulations were added to or removed from its batch since the
 * last step, the active list is rebuilt first (one kernel launch, no
 * allocation).  Blocks for one 4-byte read of the list length; the sum is in
 * a fixed order (deterministic). */
tcm_status tcm_energy_noalloc(const tcm_sim *sim, double *device_out);

/* Heterogenic bulking result of brick b: *kind = 1 homogenic (*k = its
 * coefficient) or 2 bulked (per-node coefficients). */
tcm_status tcm_brick_media(const tcm_sim *sim, int64_t b, int *kind, float *k);

/* Boxes: total in the pool, and currently free. */
tcm_status tcm_pool_info(const tcm_sim *sim, int64_t *slots, int64_t *free_slots);

/* Cumulative device time (ns, from the GPU's global timer) of the three
 * phases of every step so far: time stepping (Eq. 3 on the active bricks),
 * the update procedure (trigger/keep/release/claim), and box recycling plus
 * compaction of the active list -- the per-operation split the paper reports
 * for its step (Results, Fig. 11). */
tcm_status tcm_phase_ns(const tcm_sim *sim, int64_t *stepping, int64_t *update, int64_t *compaction);

/* The Eq. 7 filter's work so far: device time of its working launches (ns,
 * from the GPU's global timer), bricks filtered, and binary32 multiply-adds
 * per filtered brick (two time levels through the separable operator: 319488
 * for 8^3 cells; 0 for shapes the filter does not support).  Not in the
 * paper: the numbers behind the filter's roofline. */
tcm_status tcm_lpf_info(const tcm_sim *sim, int64_t *ns, int64_t *bricks, int64_t *fma_per_brick);

/* Kernel launches issued so far (one per step). */
int64_t tcm_launch_count(const tcm_sim *sim);
/* How many of those launches were replayed from captured CUDA graphs. */
int64_t tcm_graph_launch_count(const tcm_sim *sim);

/* Step index n of phi^n. */
int64_t tcm_step_index(const tcm_sim *sim);

const char *tcm_status_string(tcm_status s);

/* Self-test of the bounded device-wide barrier that the step and filter
 * kernels use between their phases (the library's own failure detection;
 * the paper has no counterpart).  One cooperative launch of one CTA per SM on
 * device `device`; every CTA arrives once.  skew = 0: the barrier completes,
 * TCM_OK.  skew = 1: the arrival counter starts one ahead, so the CTA that
 * arrives last waits for a round no CTA completes; it gives up after
 * timeout_s seconds (0 < timeout_s <= 1) and records the timeout, every CTA
 * returns, the device stays usable, and the call returns TCM_ETIMEOUT.
 * *err_out receives the device error bits (2 = barrier timeout).  Allocates
 * and frees a few bytes of device memory; blocks until done.  TCM_EINVAL for
 * bad arguments, TCM_EDEVICE if a CUDA call fails. */
tcm_status tcm_barrier_selftest(int device, int skew, double timeout_s, unsigned *err_out);

/* Destroy a simulation made by tcm_create (and its device memory).  On a
 * simulation of a batch it is tcm_batch_remove. */
void tcm_destroy(tcm_sim *sim);

/* ---- Batches: many simulations stepped by one launch per step -----------
 * A batch owns one box pool and one brick-table space shared by its
 * simulations (each gets a contiguous range of brick slots).  Every launch
 * steps all live simulations of the batch by one step; each keeps its own
 * step counter, media, sources, threshold and shut-down settings, so results
 * are bit-for-bit those of the same simulation run alone.  Simulations may
 * be added and removed between steps (continuous batching); a simulation
 * with n_steps > 0 stops stepping (is frozen, its fields kept) when it has
 * done them.  Simulation handles from tcm_batch_add are owned by the batch:
 * the per-simulation functions above (add_source, set_field, read_field,
 * active_count, active_bricks, updates, energy, brick_media, step_index)
 * accept them; tcm_step / tcm_step_async on them return TCM_ESTATE. */
typedef struct tcm_batch tcm_batch;

typedef struct {
    void *pool_ptr;     /* device memory for the boxes, or NULL: library allocates */
    size_t pool_bytes;  /* pool size (number of boxes = pool_bytes / tcm_slot_bytes) */
    void *stream;       /* cudaStream_t */
    int device;         /* CUDA device ordinal */
    int storage;        /* TCM_STORAGE_F32 / _BF16 / _F16 */
    int64_t max_bricks; /* brick-table capacity summed over simulations (12 B per brick) */
    int max_sims;       /* simulation-table capacity */
    int no_graphs;      /* as in tcm_options */
    tcm_brick brick;    /* brick shape of every simulation of the batch ({0,0,0}: 8x8x8) */
    int no_prefetch;    /* as in tcm_options */
    int cta_warps;      /* as in tcm_options */
} tcm_batch_options;

tcm_status tcm_batch_create(const tcm_batch_options *options, tcm_batch **out);

/* Add a simulation (arguments as tcm_create, dense = 1 boxes every brick).
 * TCM_ENOMEM when the brick-table space or the simulation table is full.
 * Sources and initial fields may be added until the next step. */
tcm_status tcm_batch_add(tcm_batch *batch, const tcm_domain *domain, const tcm_velocity_model *velocity,
                         double dx, double dt, double threshold, tcm_brick brick, int threshold_mode,
                         float decay_alpha, int decay_steps, int dense, int64_t n_steps, tcm_sim **out);

/* Step every live simulation n times (tcm_batch_step waits and reports the
 * status; _async only enqueues, tcm_batch_sync reports). */
tcm_status tcm_batch_step(tcm_batch *batch, int64_t n);
tcm_status tcm_batch_step_async(tcm_batch *batch, int64_t n);
tcm_status tcm_batch_sync(tcm_batch *batch);

/* Whether a simulation has done its n_steps (and no longer steps). */
tcm_status tcm_sim_done(const tcm_sim *sim, int *done);

/* Remove a simulation: its boxes return to the pool, its brick range and
 * table entry are reused; the handle is invalid afterwards. */
tcm_status tcm_batch_remove(tcm_batch *batch, tcm_sim *sim);

/* Boxes in the pool and free now; simulations alive. */
tcm_status tcm_batch_info(const tcm_batch *batch, int64_t *slots, int64_t *free_slots, int *sims);

/* Field storage of a simulation of a TCM_STORAGE_MIXED batch (TCM_STORAGE_F32,
 * _BF16 or _F16; see the storage enum).  Only before the simulation's first
 * step (TCM_ESTATE after).  In a batch of one storage only that storage is
 * accepted (TCM_OK, nothing changes); any other gives TCM_EINVAL.  Not in the
 * paper: it lets requests of both precisions share one launch per step. */
tcm_status tcm_set_storage(tcm_sim *sim, int storage);

/* Pause / resume a simulation of a batch (not in the paper; a serving loop
 * uses it to keep the pool from running out).  A paused simulation keeps its
 * boxes, fields, shut-down counts and step index but is not stepped, so it
 * claims no boxes; resumed, it continues exactly where it stopped (its
 * results equal those of an uninterrupted run bit for bit).  Pausing a
 * simulation that has done its n_steps, or one already paused, does nothing;
 * so does resuming one that is not paused.  Takes effect at the next step
 * call.  TCM_EINVAL for a simulation made by tcm_create; TCM_ESTATE after the
 * batch failed. */
tcm_status tcm_batch_pause(tcm_sim *sim);
tcm_status tcm_batch_resume(tcm_sim *sim);

/* An upper bound on the boxes the batch's stepping (not paused, not done)
 * simulations can claim during the next `steps` steps: the unboxed cells of
 * each simulation that lie within ceil(steps / L) + 1 cells (Chebyshev
 * distance, L the shortest cell edge in nodes) of one of its boxed cells.
 * It holds because Eq. 3 moves values at most one node per step and the
 * update procedure only boxes neighbours of cells that hold values (update
 * steps 4-5, Fig. 3).  Simulations added since the last step are started
 * first (their initial cells boxed).  If the free boxes (tcm_batch_info) are
 * at least this bound, the next `steps` steps cannot exhaust the pool.  One
 * pass over the brick tables on the device; the first call allocates
 * 2 bytes of scratch per brick of the batch's capacity; blocks until done.
 * Not in the paper: admission control for the serving form. */
tcm_status tcm_batch_headroom(tcm_batch *batch, int64_t steps, int64_t *boxes);

void tcm_batch_destroy(tcm_batch *batch);

#ifdef __cplusplus
}
#endif
#endif /* TCM_H */
