/*
 * tcm_oracle.h -- CPU oracle for the Triggered Cells Method (Naeh, arXiv:1702.00216).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load
 * this library: only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no source, header, table or helper with the
 * CUDA library (paper_1702_00216_gb300/csrc, include/tcm.h).
 *
 * Two programs, each compiled for binary32 (suffix _f32) and binary64 (_f64):
 *
 *  1. Dense FDTD -- the plain definition: Eq. 3 applied to every node of an
 *     nx*ny*nz grid, zero (Dirichlet) ghost values outside the domain, two
 *     field arrays plus the coefficient k = (c*dt/dx)^2 (Introduction, Eq. 1-4).
 *
 *  2. Triggered Cells Method -- the algorithm in the paper's order: cells
 *     ("bricks") of bx*by*bz nodes, boxes (slots) allocated on triggering and
 *     reused after shut-down (Boxes, Fig. 1), Heterogenic Bulking of the media
 *     (Media), source insertion with manual activation (Simulation / Source
 *     insertion), the active-cell update procedure (Simulation / Updating active
 *     cells), boxes padded by their neighbours' boundaries (Time stepping) and
 *     the time-domain shut-down of Eq. 6.
 *
 * Conventions shared by both programs (each implements them independently):
 *  - Arrays are x fastest: index = (z*ny + y)*nx + x.
 *  - Eq. 3 is evaluated with one fixed grouping, every + - * rounded separately:
 *        s   = ((((xm + xp) + ym) + yp) + zm) + zp
 *        lap = s - 6*p
 *        q   = (2*p - pm) + k*lap
 *    then each source whose insertion window covers step n adds w[n - start];
 *    then a box in shut-down scales q by alpha (Eq. 6).
 *  - Step n turns (phi^n, phi^{n-1}) into (phi^{n+1}, phi^n).
 *  - Media rules: node (i,j,l) has c = background; then for each layer m in
 *    order, c = layer_c[m] where l >= layer_z[m]; then for each sphere s in
 *    order, c = sphere_c[s] where (i-x)^2+(j-y)^2+(l-z)^2 <= r^2 (FP64).
 *  - k = (c*dt/dx)^2 evaluated in FP64 as ((double)c*dt/dx) squared, then
 *    rounded to the program's type.
 *
 * Error returns are negative; 0 is success.
 */
#ifndef TCM_ORACLE_H
#define TCM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ESTATE = -3 };
enum { ORC_MEDIA_DENSE = 0, ORC_MEDIA_RULES = 1 };
enum { ORC_THR_ABSOLUTE = 0, ORC_THR_RELATIVE = 1 };

/* Number of OpenMP threads used by the per-node loops (1 = serial; results
 * do not depend on it).  Returns the number actually available. */
int orc_set_threads(int n);

/* ---- media ------------------------------------------------------------ */
/* Evaluate the media rules at every node of an nx*ny*nz grid -> c (float). */
void orc_rules_c(int64_t nx, int64_t ny, int64_t nz, float c_background,
                 int n_layers, const double *layer_z, const float *layer_c,
                 int n_spheres, const double *sphere_xyzr, const float *sphere_c,
                 float *c_out);

/* k = (c*dt/dx)^2 for n values (Eq. 3 coefficient). */
void orc_k_from_c_f32(const float *c, int64_t n, double dt, double dx, float *k_out);
void orc_k_from_c_f64(const float *c, int64_t n, double dt, double dx, double *k_out);

/* ---- dense FDTD (Eq. 3 on every node) ---------------------------------- */
/* Advance `steps` steps starting at step index `step0`.  On entry now = phi^step0,
 * prev = phi^(step0-1); on return they hold phi^(step0+steps), phi^(step0+steps-1).
 * Source s sits at flat node index src_idx[s], starts at step src_start[s] and
 * has src_len[s] samples at w + s*w_stride. */
int orc_dense_run_f32(int64_t nx, int64_t ny, int64_t nz, const float *k,
                      float *now, float *prev, int nsrc, const int64_t *src_idx,
                      const int64_t *src_start, const int64_t *src_len,
                      const float *w, int64_t w_stride, int64_t step0, int64_t steps);
int orc_dense_run_f64(int64_t nx, int64_t ny, int64_t nz, const double *k,
                      double *now, double *prev, int nsrc, const int64_t *src_idx,
                      const int64_t *src_start, const int64_t *src_len,
                      const double *w, int64_t w_stride, int64_t step0, int64_t steps);

/* Discrete energy of the leapfrog scheme between two consecutive fields
 * a = phi^{n+1}, b = phi^n:  E = sum_i (a_i-b_i)^2 / k_i + sum_i a_i (K b)_i,
 * (K b)_i = 6 b_i - sum of the six neighbours (zero outside).  It is constant
 * once all sources have stopped; it requires k_i > 0 everywhere. */
double orc_energy_f64(int64_t nx, int64_t ny, int64_t nz, const double *k,
                      const double *a, const double *b);
double orc_energy_f32(int64_t nx, int64_t ny, int64_t nz, const float *k,
                      const float *a, const float *b);

/* ---- 16-bit storage formats -------------------------------------------- */
/* Round a binary32 value to nearest (ties to even) in a narrower format and
 * return it as binary32 (exactly representable):
 *   bfloat16: 8 significant bits, binary32's exponent range (normal down to
 *             2^-126, subnormals in steps of 2^-133), overflow to +-inf;
 *   binary16: 11 significant bits, normal down to 2^-14, subnormals in steps
 *             of 2^-24, largest finite 65504, overflow to +-inf.
 * Written from the formats' definitions; zeros, infinities and NaN pass. */
float orc_round_bf16(float v);
float orc_round_f16(float v);

enum { ORC_STORAGE_F32 = 0, ORC_STORAGE_BF16 = 1, ORC_STORAGE_F16 = 2 };

/* ---- frequency-domain shut-down (Eq. 7) ---------------------------------- */
/* Radix-2 complex DFT in place (n a power of two; sign -1 forward, +1
 * inverse, unscaled). */
void orc_fft(double *re, double *im, int n, int sign);
/* Low-pass response at DFT index kappa of an M-point transform: 1 up to
 * `pass`, 0 from `stop` (fractions of the Nyquist frequency), raised cosine
 * between. */
double orc_lpf_response(int kappa, int M, double pass, double stop);
/* Phi~ = F^-1[F(Phi) LPF] (Eq. 7) on an L^3 region (x fastest), zero-padded
 * to M^3 (spatial oversampling), LPF = H(kx) H(ky) H(kz); in place. */
void orc_lpf_region(double *v, int L, int M, double pass, double stop);

/* ---- Triggered Cells Method ---------------------------------------------- */
typedef struct orc_tcm orc_tcm;

/* Create a simulation.  media_kind selects the dense c array (nx*ny*nz floats,
 * copied) or the rules.  thr_mode/tau: absolute threshold tau, or tau times the
 * domain's maximal |phi^{n+1}|.  decay_alpha/decay_steps: Eq. 6 shut-down
 * (decay_steps = 0 retires a quiet box at once).  max_slots caps the number of
 * boxes (<= 0: unlimited).  dense_mode = 1 boxes every cell and never retires.
 * Returns NULL on invalid arguments. */
orc_tcm *orc_tcm_create_f32(int64_t nx, int64_t ny, int64_t nz, int bx, int by, int bz,
                            int media_kind, const float *c_dense, float c_background,
                            int n_layers, const double *layer_z, const float *layer_c,
                            int n_spheres, const double *sphere_xyzr, const float *sphere_c,
                            double dx, double dt, int thr_mode, double tau,
                            double decay_alpha, int decay_steps, int64_t max_slots,
                            int dense_mode);
orc_tcm *orc_tcm_create_f64(int64_t nx, int64_t ny, int64_t nz, int bx, int by, int bz,
                            int media_kind, const float *c_dense, float c_background,
                            int n_layers, const double *layer_z, const float *layer_c,
                            int n_spheres, const double *sphere_xyzr, const float *sphere_c,
                            double dx, double dt, int thr_mode, double tau,
                            double decay_alpha, int decay_steps, int64_t max_slots,
                            int dense_mode);

/* Add a point source at node (x,y,z) whose samples w[0..len) are added at
 * steps step_index .. step_index+len-1 (Source insertion). */
int orc_tcm_add_source_f32(orc_tcm *t, int64_t x, int64_t y, int64_t z,
                           const float *w, int64_t len);
int orc_tcm_add_source_f64(orc_tcm *t, int64_t x, int64_t y, int64_t z,
                           const double *w, int64_t len);
/* Initial fields (dense nx*ny*nz arrays); only before the first step. */
int orc_tcm_set_field_f32(orc_tcm *t, const float *now, const float *prev);
int orc_tcm_set_field_f64(orc_tcm *t, const double *now, const double *prev);
/* Field storage precision (before the first step; default ORC_STORAGE_F32).
 * With BF16 or F16 every phi^{n+1} is rounded to the format when it is
 * written -- after Eq. 3, the source samples and the shut-down factor, all in
 * the program's type -- and the maxima, the trigger decisions and the domain
 * maximum are taken on the rounded value.  Initial fields are rounded the
 * same way at the first step.  F16 holds phi / s with s = 2^(e-8), where
 * 2^(e-1) <= m < 2^e and m is the largest |value| among the source samples
 * and initial fields at the first step (s = 1 when m = 0; e - 8 clamped to
 * [-100, 100]); BF16 and F32 use s = 1.  Only the _f32 program takes a
 * 16-bit storage (the _f64 one would round twice); it returns ORC_EINVAL.
 * A 16-bit storage also selects the velocity form (orc_tcm_set_velocity_form). */
int orc_tcm_set_storage_f32(orc_tcm *t, int storage);
/* Velocity form of the recursion (before the first step; on with any 16-bit
 * storage, optional with F32 and F64): each box holds phi^n and v^n = phi^n -
 * phi^{n-1} instead of phi^n and phi^{n-1}.  A step computes
 * v' = v + k lap (lap as in Eq. 3), v' += w for a source node,
 * phi^{n+1} = phi^n + v', and in shut-down phi^{n+1} *= alpha, v' = phi^{n+1} -
 * phi^n; phi^{n+1} and v' are then written in the storage format.  In exact
 * arithmetic it is Eq. 3; rounding a stored phi no longer acts on the
 * velocity.  Initial fields give v^0 = phi^0 - phi^{-1} (before rounding);
 * reading which = 1 returns phi^n - v^n; after an Eq. 7 filter v is set to the
 * difference of the filtered levels. */
int orc_tcm_set_velocity_form_f32(orc_tcm *t, int on);
int orc_tcm_set_velocity_form_f64(orc_tcm *t, int on);
/* Velocity form: initial phi^0 and v^0 directly (dense nx*ny*nz arrays),
 * and a window of v^n (zeros where no box is allocated). */
int orc_tcm_set_field_velocity_f32(orc_tcm *t, const float *now, const float *v);
int orc_tcm_set_field_velocity_f64(orc_tcm *t, const double *now, const double *v);
int orc_tcm_read_velocity_f32(const orc_tcm *t, int64_t x0, int64_t y0, int64_t z0,
                              int64_t wx, int64_t wy, int64_t wz, float *out);
int orc_tcm_read_velocity_f64(const orc_tcm *t, int64_t x0, int64_t y0, int64_t z0,
                              int64_t wx, int64_t wy, int64_t wz, double *out);
int orc_tcm_set_storage_f64(orc_tcm *t, int storage);
/* The scale s in use (1 before the first step). */
double orc_tcm_storage_scale_f32(const orc_tcm *t);
double orc_tcm_storage_scale_f64(const orc_tcm *t);
/* Schedule of the update procedure (before the first step; default 1, 6).
 * interval >= 1: the procedure runs after every interval-th step (after step
 * n when (n+1) % interval == 0; Eq. 5 gives interval = dx*L/(2 c dt) for
 * cells of L nodes).  Between runs the active cells, their shut-down counts
 * and the Eq. 6 factors stay as set.  A run covers steps n+1 .. n+interval:
 * a source cell fed at any of them is kept / boxed, and a cell in shut-down
 * has its count (in time steps) reduced by interval, released at <= 0.
 * neighbours = 6: a cell stays if its maximum or a boxed face neighbour's
 * touching face is above the level; faces above the level trigger the cell
 * across them.  neighbours = 26: a cell is triggered when it is boxed with
 * its maximum above the level, or a source feeds it during the steps the run
 * covers; a cell stays if it or any of its 26 neighbours is triggered; a
 * triggered cell boxes all 26 neighbours (steps 4 and 5 of the update,
 * Fig. 3: nearest and diagonal cells).  Before the first step the procedure
 * runs once on the initial state (level from max |phi^0|; 6 neighbours: the
 * cell across each face whose max |phi^0| is above it; 26: all neighbours of
 * a cell above it in max(|phi^0|,|phi^-1|) or fed by a source in steps
 * 0 .. interval-1), releasing nothing; with the 26-neighbour set, adding a
 * source boxes its cell's neighbourhood at once.  Returns ORC_EINVAL for
 * interval < 1 or another neighbour count, ORC_ESTATE after the first step. */
/* Frequency-domain shut-down (Eq. 7) instead of the time-domain decay:
 * at a run of the update procedure, a cell that is not kept is released at
 * once (Q), and every boxed cell that stays and has among its 26 neighbours a
 * cell of Q that held a non-zero value (removing an all-zero cell cuts
 * nothing) gets both time levels (phi^{n+1}, phi^n) replaced by the centre
 * cell of orc_lpf_region applied to the 3x3x3-cell block around it (cells of
 * Q, unboxed cells and nodes outside the domain read zero; region L = 3 cell
 * edges, padded to M = 64 per axis; results are rounded to the program's
 * type and storage, and nodes outside the domain stay zero).  All filtered
 * values come from the state before any is written.  Cells only, 8^3 bricks
 * assumed for L = 24.  pass/stop as in orc_lpf_response; 0 < pass < stop <= 1.
 * Before the first step. */
int orc_tcm_set_lpf_f32(orc_tcm *t, double pass, double stop);
int orc_tcm_set_lpf_f64(orc_tcm *t, double pass, double stop);
int orc_tcm_set_schedule_f32(orc_tcm *t, int interval, int neighbours);
int orc_tcm_set_schedule_f64(orc_tcm *t, int interval, int neighbours);
int orc_tcm_step_f32(orc_tcm *t, int64_t n);
int orc_tcm_step_f64(orc_tcm *t, int64_t n);
/* which = 0: phi^n, 1: phi^{n-1}; zeros where no box is allocated. */
int orc_tcm_read_field_f32(const orc_tcm *t, int which, int64_t x0, int64_t y0, int64_t z0,
                           int64_t wx, int64_t wy, int64_t wz, float *out);
int orc_tcm_read_field_f64(const orc_tcm *t, int which, int64_t x0, int64_t y0, int64_t z0,
                           int64_t wx, int64_t wy, int64_t wz, double *out);
/* Active (boxed) cells: count, in-domain node count, sorted ids. */
int64_t orc_tcm_active_count_f32(const orc_tcm *t, int64_t *nodes);
int64_t orc_tcm_active_count_f64(const orc_tcm *t, int64_t *nodes);
int64_t orc_tcm_active_bricks_f32(const orc_tcm *t, int64_t *ids, int64_t cap);
int64_t orc_tcm_active_bricks_f64(const orc_tcm *t, int64_t *ids, int64_t cap);
/* Cumulative node updates performed (sum over steps of boxed in-domain nodes). */
int64_t orc_tcm_updates_f32(const orc_tcm *t);
int64_t orc_tcm_updates_f64(const orc_tcm *t);
int64_t orc_tcm_step_index_f32(const orc_tcm *t);
int64_t orc_tcm_step_index_f64(const orc_tcm *t);
/* Sticky status: 0 or ORC_ENOMEM once a box could not be allocated. */
int orc_tcm_status_f32(const orc_tcm *t);
int orc_tcm_status_f64(const orc_tcm *t);
/* Heterogenic bulking of cell b: returns 1 homogeneous (k in *kscal), 2 bulked. */
int orc_tcm_brick_media_f32(orc_tcm *t, int64_t b, double *kscal);
int orc_tcm_brick_media_f64(orc_tcm *t, int64_t b, double *kscal);
void orc_tcm_destroy_f32(orc_tcm *t);
void orc_tcm_destroy_f64(orc_tcm *t);

#ifdef __cplusplus
}
#endif
#endif
