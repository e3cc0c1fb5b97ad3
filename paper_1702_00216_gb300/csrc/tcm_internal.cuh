// tcm_internal.cuh -- device-side data layout shared by the kernels and the host
// runtime of libtcm (Triggered Cells Method, Naeh, arXiv:1702.00216).
//
// HBM layout of one engine (a set of simulations stepped by one launch):
//   pool      phi[slot][half][z][y][x]   two binary32 halves of one brick per box
//                                        (Boxes section, Fig. 1)
//   per brick slot_of_brick[g]  int32    Cell2box (-1 inactive, -2 claim in flight)
//             kscal[g]          float    homogenic coefficient (HBM)
//             kslab_of_brick[g] int32    index of the bulked coefficient brick, -1 if homogenic
//             sd_of_brick[g]    uint16   Shutdown_log: shut-down steps left (bits 0-14) and
//                                        "holds a source" (bit 15)
//             bitmap[g/32]      bit      active for the next step (drives the compaction)
//             sim_of_word[g/32] uint16   simulation owning those 32 bricks
//   per box   meta[slot]        16 B     Box2cell brick id, bulk index, scalar k, sim/sd flags
//             rec[slot][8]      float    6 face maxima, cell maximum, launch that wrote it
//   lists     items[2][n_slots] 48 B     active bricks in brick order (double-buffered): box,
//                                        brick, k, flags and the boxes of the 6 face neighbours
//             listids, free_stack, retired, newslots  int32 per box
// Global brick index g = sim.brick_base + local brick id; every sim's range
// starts on a 32-brick boundary so bitmap words never straddle two sims.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace tcm {

// Brick shape of this build of the library (one build per supported shape;
// the public entry points dispatch on the shape a simulation was created with).
#ifndef TCM_BX
#define TCM_BX 8
#define TCM_BY 8
#define TCM_BZ 8
#endif
constexpr int BX = TCM_BX, BY = TCM_BY, BZ = TCM_BZ;
constexpr int BVOL = BX * BY * BZ;          // nodes per brick
constexpr int XQ = BX / 4;                  // float4 columns per brick row
constexpr int TPB = XQ * BY;                // threads per brick (one float4 column, all z)
#ifndef TCM_P1_WARPS
#define TCM_P1_WARPS 8
#endif
constexpr int P1_WARPS = TCM_P1_WARPS;      // warps per CTA of the step kernel
constexpr int BLOCK = 32 * P1_WARPS;        // threads per CTA of the step kernel
constexpr int BRICKS_PER_WARP = 32 / TPB;
static_assert(BX % 4 == 0 && TPB <= 32 && 32 % TPB == 0, "a brick's float4 columns must tile a warp");
static_assert(BRICKS_PER_WARP == 1 || XQ <= 2, "pair exchange lane mapping needs XQ <= 2");

constexpr unsigned ERR_NOMEM = 1u;
constexpr unsigned ERR_TIMEOUT = 2u;
constexpr unsigned ERR_BOUNDS = 4u;   // the checked build found an index out of range

constexpr unsigned FLAG_HAS_SRC = 1u << 15;
constexpr unsigned SD_MASK = 0x7fffu;

enum { MEDIA_DENSE = 0, MEDIA_RULES = 1 };
// Field storage of the boxes: binary32, or bfloat16 / binary16 holding
// phi / scale (scale a power of two per simulation; compute is binary32).
enum { ST_F32 = 0, ST_BF16 = 1, ST_F16 = 2 };
// A batch whose simulations each choose one of the three storages; its boxes
// are sized for binary32 (the widest).
constexpr int ST_MIXED = 3;
__host__ __device__ constexpr int storage_bytes(int st) { return st == ST_F32 ? 4 : 2; }
// Elements per box: the two field halves (phi^n, phi^{n-1}) in binary32; with
// a 16-bit storage the velocity form keeps the two phi halves (phi^n and the
// phi^{n+1} being written) plus v^n = phi^n - phi^{n-1} as a third array.
__host__ __device__ constexpr int slot_elems(int st) { return st == ST_F32 ? 2 * BVOL : 3 * BVOL; }
constexpr int V_HALF = 2;   // index of the v array in a 16-bit box

struct __align__(16) SlotMeta {
    int brick;       // local brick id within its sim (Box2cell)
    int kslab;       // bulked coefficient brick, or -1
    float kscal;     // homogenic coefficient
    unsigned flags;  // sim << 16 | has_src << 15 | shut-down steps left
};

// One active brick of the list (built by the compaction phase).
struct __align__(16) WorkItem {
    int slot;
    int brick;
    unsigned long long kp;   // bulked: address of the brick's k values; homogenic: KP_SCALAR | k bits
    unsigned flags;
    int nb[6];       // boxes of the face neighbours x-, x+, y-, y+, z-, z+ (-1 none, -3 outside)
    int nh;          // field half holding phi^n for the step that processes this item
};
static_assert(sizeof(WorkItem) == 48, "work item layout");
constexpr unsigned long long KP_SCALAR = 1ull << 63;

struct SimDev {
    // immutable after create
    int nx, ny, nz;
    int mx, my, mz;
    long long brick_base;
    long long n_bricks;
    int thr_mode;
    int dense;
    double tau;
    float alpha;
    int decay_steps;
    int src_begin, src_end;
    const float *kslabs;   // this sim's bulked coefficient bricks
    int live;              // 1 while the sim steps (0: frozen or released)
    float scale;           // stored field value = phi / scale (power of two)
    float inv_scale;
    int interval;          // the update procedure runs after every interval-th step
    int neighbours;        // 6: activation across hot faces; 26: all neighbours of a hot cell
    int lpf;               // 1: frequency-domain shut-down (Eq. 7) instead of the decay
    const float *lpf_a;    // LPF_C x LPF_L centre rows of the 1-D filter operator (binary32)
    int storage;           // field storage of this sim's boxes (ST_F32 / ST_BF16 / ST_F16)
    int pad_storage;
    // mutable (device-owned)
    long long step;        // n of phi^n
    unsigned gmax[2];      // max |phi^{n+1}| of step n in gmax[n & 1] (float bits)
    unsigned poisoned;
    unsigned pad;
    unsigned long long updates;   // cumulative node updates of this sim
};

struct SrcDev {
    int sim;
    int brick;           // local brick id
    int local;           // node index within the brick
    int pad;
    long long start;     // first step that adds a sample
    long long len;
    long long w_off;     // offset into the concatenated wavelets
};

struct EngineState {
    int free_top;          // entries on the free stack
    int n_retired;         // boxes released this step (pushed by the compaction phase)
    int n_new;             // boxes claimed this step (zeroed by the compaction phase)
    int list_parity;       // which list holds the current active boxes
    int n_active[2];
    unsigned err;
    unsigned long long bar_count;      // step kernel's grid barrier: arrivals so far (only grows)
    unsigned long long bar_count_lpf;  // the same for the Eq. 7 kernel
    unsigned p3_done;      // blocks finished with the compaction phase this launch
    unsigned long long updates;   // cumulative node updates
    unsigned long long launches;
    unsigned long long t_start, t_p1, t_p2;   // globaltimer stamps of the current launch
    unsigned long long phase_ns[3];           // cumulative: time stepping, update, compaction
    int list_age;          // launches since the active list was built (phase of its nh)
    int n_lpf_q;           // bricks released this update that held values (Eq. 7 sources)
    int n_lpf_aff;         // boxed bricks the Eq. 7 filter rewrites this update
    unsigned lpf_done;     // blocks finished with the Eq. 7 kernel this launch
    unsigned long long t_lpf;          // globaltimer at the start of the Eq. 7 kernel
    unsigned long long lpf_ns;         // cumulative: time of the Eq. 7 kernel's working launches
    unsigned long long lpf_bricks;     // cumulative: bricks it filtered
};

// Eq. 7 region: the 3x3x3-brick block around a brick (LPF_L nodes per axis),
// zero-padded to LPF_M per axis; the filter keeps the centre LPF_C nodes.
constexpr int LPF_C = BX;   // cubic bricks only
constexpr int LPF_L = 3 * LPF_C;
constexpr int lpf_pow2(int v) { return v <= 1 ? 1 : 2 * lpf_pow2((v + 1) / 2); }
constexpr int LPF_M = lpf_pow2(2 * LPF_L);   // at least 2x oversampling

struct Engine {
    void *phi;             // pool: slot_bytes per box
    int storage;           // ST_F32 / ST_BF16 / ST_F16, or ST_MIXED (per simulation)
    int slot_bytes;        // bytes per box
    int n_slots;
    int *slot_of_brick;
    const float *kscal;
    const int *kslab_of_brick;
    unsigned short *sd_of_brick;
    unsigned *bitmap;
    unsigned short *sim_of_word;   // owning sim of each 32-brick bitmap word
    long long n_words;
    int *blocktot;
    int words_per_block;
    SlotMeta *meta;
    float *rec;
    WorkItem *items0, *items1;
    int *listids;
    int *free_stack, *retired, *newslots;
    SimDev *sims;
    int n_sims;
    const SrcDev *src;
    int n_src;
    const float *wave;
    EngineState *st;
    // Eq. 7 shut-down (per slot: claim step, mark; lists; filtered values)
    int *claim_step;       // step index of the update that claimed the box
    int *lpf_mark;         // 1 while the box is on the affected list
    long long *lpf_q;      // released bricks (global ids) that held values
    long long *lpf_aff;    // affected bricks (global ids)
    float *lpf_out;        // filtered values, 2 * BVOL per affected brick
    int lpf_cap;           // capacity of lpf_out in bricks
    int prefetch;          // 1: L2 prefetch of the next brick pair's arrays in the time stepping
};

struct MediaDev {
    int kind;
    const float *c;        // dense: device memory, or page-locked host memory the device addresses
    float c_bg;
    int n_layers;
    const double *layer_z;
    const float *layer_c;
    int n_spheres;
    const double *sph;
    const float *sph_c;
};

// Bounds checks of the checked build (compiled with -DTCM_CHECKED): every
// box, brick, free-stack, list and claim index is checked before the access
// it guards; an index out of range sets ERR_BOUNDS and the access is
// skipped (no trap).  In the normal build the checks compile to `true`.
#ifdef TCM_CHECKED
__device__ __forceinline__ bool in_range(EngineState *st, long long i, long long n)
{
    if (i >= 0 && i < n) return true;
    atomicOr(&st->err, ERR_BOUNDS);
    return false;
}
#define TCM_IN(E, i, n) ::tcm::in_range((E).st, (long long)(i), (long long)(n))
#else
#define TCM_IN(E, i, n) true
#endif
// the brick tables hold n_words * 32 entries
#define TCM_BRICK_OK(E, g) TCM_IN(E, g, (E).n_words * 32)
#define TCM_SLOT_OK(E, s) TCM_IN(E, s, (E).n_slots)

// Field storage of simulation S's boxes.
__host__ __device__ __forceinline__ int sim_storage(const Engine &E, const SimDev *S)
{
    return E.storage == ST_MIXED ? S->storage : E.storage;
}

// First byte of box `slot`.
__device__ __forceinline__ unsigned char *box_base(const Engine &E, int slot)
{
    return static_cast<unsigned char *>(E.phi) + (size_t)slot * (size_t)E.slot_bytes;
}

// Element e of box array (slot, half) -- half 0/1 a field half, V_HALF the
// velocity (16-bit storages) -- of a box in storage st, as a physical value
// (x scale).
__device__ __forceinline__ float load_phys(const Engine &E, int st, int slot, int half, int e, float scale)
{
    const unsigned char *base = box_base(E, slot);
    const size_t i = (size_t)half * BVOL + e;
    if (st == ST_F32) return reinterpret_cast<const float *>(base)[i] * scale;
    const unsigned short bits = reinterpret_cast<const unsigned short *>(base)[i];
    if (st == ST_BF16) return __uint_as_float((unsigned)bits << 16) * scale;
    return __half2float(__ushort_as_half(bits)) * scale;
}

// Store a physical value v into element e of box half (slot, half).
__device__ __forceinline__ void store_phys(const Engine &E, int st, int slot, int half, int e, float v,
                                           float inv_scale)
{
    unsigned char *base = box_base(E, slot);
    const size_t i = (size_t)half * BVOL + e;
    const float s = v * inv_scale;
    if (st == ST_F32) reinterpret_cast<float *>(base)[i] = s;
    else if (st == ST_BF16) reinterpret_cast<__nv_bfloat16 *>(base)[i] = __float2bfloat16_rn(s);
    else reinterpret_cast<__half *>(base)[i] = __float2half_rn(s);
}

// phi^{n-1} at element e of a box whose phi^n is in half now_half: the other
// half in binary32; phi^n - v^n (binary32 subtraction) in the velocity form.
__device__ __forceinline__ float load_prev_phys(const Engine &E, int st, int slot, int now_half, int e, float scale)
{
    if (st == ST_F32) return load_phys(E, st, slot, now_half ^ 1, e, scale);
    return __fsub_rn(load_phys(E, st, slot, now_half, e, scale), load_phys(E, st, slot, V_HALF, e, scale));
}

// ---- launchers (tcm_kernels.cu) -------------------------------------------
// Every launcher returns the cudaError_t of its launch.
cudaError_t launch_barrier_selftest(EngineState *st, unsigned long long *ctr, int grid,
                                    unsigned long long timeout_ns, cudaStream_t s);
// Bulking of one sim whose bricks start at global index bb.
cudaError_t launch_bulk_classify(const MediaDev &m, int nx, int ny, int nz, int mx, int my, int mz,
                                 double dt, double dx, long long bb, float *kscal, int *kslab_of_brick,
                                 int *n_kslabs, cudaStream_t s);
cudaError_t launch_bulk_fill(const MediaDev &m, int nx, int ny, int nz, int mx, int my, int mz,
                             double dt, double dx, long long bb, const int *kslab_of_brick, float *kslabs,
                             cudaStream_t s);
cudaError_t launch_iota_desc(int *a, int n, int first, cudaStream_t s);
// Between steps: fold the boxes released by the last step into the free stack.
cudaError_t launch_settle(const Engine &e, cudaStream_t s);
// Box bricks[0..n) (local ids; all n bricks when bricks == nullptr) of sim,
// zeroed, popped from the free stack.
cudaError_t launch_admit(const Engine &e, int sim, const long long *bricks, long long n, cudaStream_t s);
// Take every brick of sim out of the active set (boxes stay) / release its boxes.
cudaError_t launch_freeze(const Engine &e, int sim, long long words_begin, long long n_words, cudaStream_t s);
// Put every boxed brick of a paused sim back into the active set (its range
// is bricks [bb, bb + n) in words [words_begin, words_begin + n_words)).
cudaError_t launch_thaw(const Engine &e, int sim, long long words_begin, long long n_words, long long bb,
                        long long n, cudaStream_t s);
// Unboxed bricks of live sims within Chebyshev distance r (in bricks) of a
// boxed brick of the same sim, added to *count; scratch a/b hold one byte per
// brick of the brick tables.
cudaError_t launch_reach(const Engine &e, int r, unsigned char *a, unsigned char *b, unsigned long long *count,
                         cudaStream_t s);
cudaError_t launch_release(const Engine &e, int sim, long long bb, long long n, cudaStream_t s);
// Rebuild the active list `list_parity` from the bitmap (same grid as the step).
cudaError_t launch_compact(const Engine &e, int grid, int list_parity, cudaStream_t s);
// packed[i] = {phi^n, phi^{n-1}} of global brick gids[i] (boxed), into its box.
cudaError_t launch_scatter_field(const Engine &e, const float *packed, const long long *gids, long long n,
                                 int now_half, cudaStream_t s);
// manage = 0: no simulation runs the update procedure after this step (time
// stepping only; the active list is kept).
cudaError_t launch_step(const Engine &e, int grid, int parity, int manage, cudaStream_t s);
// Eq. 7 filtering after a launch whose update released bricks of LPF sims.
cudaError_t launch_lpf(const Engine &e, int grid, cudaStream_t s);
int lpf_grid_size(int device);
// Multiply-adds of the Eq. 7 filter per filtered brick: two time levels, each
// through the separable operator along x (L^2 rows of C outputs from L
// inputs), y (L C rows) and z (C^2 rows).
constexpr long long LPF_FMA_PER_BRICK =
    2LL * ((long long)LPF_L * LPF_L * LPF_C * LPF_L + (long long)LPF_L * LPF_C * LPF_C * LPF_L +
           (long long)LPF_C * LPF_C * LPF_C * LPF_L);
int step_grid_size(int device);
cudaError_t launch_read_window(const Engine &e, int sim, int now_half, int which, long long x0, long long y0,
                               long long z0, long long wx, long long wy, long long wz, float *out,
                               cudaStream_t s);
cudaError_t launch_energy(const Engine &e, int sim, int now_half, int list_parity, double *out,
                          cudaStream_t s);
// Active bricks of sim in the list: local ids (unsorted, count in *n_out) and in-domain nodes.
cudaError_t launch_active_bricks(const Engine &e, int sim, int list_parity, long long *ids_out,
                                 unsigned long long *n_out, unsigned long long *cells_out, cudaStream_t s);

// Read-only view of a simulation for entry points defined outside tcm_api.cu.
struct SimView {
    const Engine *E;
    int device;
    cudaStream_t stream;
    bool started;          // the simulation's initial state is on the device
    bool list_ok;          // the active list matches the current state
    long long step;
    int list_parity;
    int sim;
};

}  // namespace tcm

struct tcm_sim;
// Fills *v; false when sim is NULL.  refresh_list: if the simulation has
// started and its batch changed since the last step (admission, removal,
// freeze), rebuild the active list first (one compaction launch, no device
// allocation).  Defined in tcm_api.cu.
__attribute__((visibility("hidden"))) bool tcm_internal_view(const tcm_sim *sim, tcm::SimView *v,
                                                             bool refresh_list);
