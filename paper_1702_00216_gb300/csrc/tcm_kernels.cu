// tcm_kernels.cu -- sm_103a kernels of the Triggered Cells Method
// (Naeh, arXiv:1702.00216).
//
// The hot path is one cooperative, persistent launch per time step (k_step):
//   P1  Eq. 3 on every active brick ("Time stepping"): a half-warp owns one
//       8x8x8 brick, each lane one float4 column marching in z; the one-node
//       halo comes from the six face neighbours' boxes (zero where a neighbour
//       is inactive or outside the domain), the x/y neighbours inside the
//       brick come through warp shuffles, so no shared-memory round trip.  The
//       epilogue inserts source samples, applies the Eq. 6 decay, stores
//       phi^{n+1} over phi^{n-1} (float4, coalesced) and reduces the cell
//       maximum, six face maxima and the domain maximum with shuffles.
//   --  device-wide barrier (bounded wait)
//   P2  "Updating active cells": each active brick decides keep / shut-down /
//       release from its own maximum and its neighbours' touching faces, and
//       claims the neighbours across faces above the trigger level
//       (atomicCAS on Cell2box, a box popped from the free stack).
//   --  device-wide barrier
//   P3  zero the claimed boxes, return released boxes to the free stack and
//       rebuild the active list from the brick bitmap (warp ballot/popc +
//       block prefix scan), in brick order, for the next launch.
// Arithmetic: binary32, every + - * an explicit round-to-nearest intrinsic
// (no FMA contraction), no flush-to-zero.
#include "tcm_internal.cuh"

namespace tcm {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long BARRIER_TIMEOUT_NS = 4000000000ull;  // 4 s

static_assert(XQ >= 2, "the lane layout needs at least two float4 columns per row");
static_assert(32 % TPB == 0, "bricks must tile a warp");

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Device-wide barrier for a cooperative launch.  The wait is bounded: after
// BARRIER_TIMEOUT_NS the block records ERR_TIMEOUT and returns false, and the
// caller leaves the kernel (the others then time out at their next barrier).
__device__ bool grid_barrier(EngineState *st)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire(&st->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&st->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            st_release(&st->bar_gen, gen + 1);
        } else {
            const unsigned long long t0 = globaltimer();
            while (ld_acquire(&st->bar_gen) == gen) {
                __nanosleep(128);
                if (globaltimer() - t0 > BARRIER_TIMEOUT_NS) {
                    atomicOr(&st->err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

__device__ __forceinline__ SlotMeta load_meta(const SlotMeta *p)
{
    const int4 v = __ldcg(reinterpret_cast<const int4 *>(p));
    SlotMeta m;
    m.brick = v.x;
    m.kslab = v.y;
    m.kscal = __int_as_float(v.z);
    m.flags = (unsigned)v.w;
    return m;
}

__device__ __forceinline__ void store_meta(SlotMeta *p, const SlotMeta &m)
{
    *reinterpret_cast<int4 *>(p) = make_int4(m.brick, m.kslab, __float_as_int(m.kscal), (int)m.flags);
}

// Eq. 3 at one node, fixed grouping, each operation rounded once.
__device__ __forceinline__ float eq3(float p, float pm, float k, float xm, float xp, float ym,
                                     float yp, float zm, float zp)
{
    const float s = __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)), __fadd_rn(zm, zp));
    const float lap = __fsub_rn(s, __fmul_rn(6.0f, p));
    return __fadd_rn(__fsub_rn(__fmul_rn(2.0f, p), pm), __fmul_rn(k, lap));
}

__device__ __forceinline__ float4 eq3v(float4 p, float4 pm, float4 k, float xm0, float xp3, float4 ym,
                                       float4 yp, float4 zm, float4 zp)
{
    float4 q;
    q.x = eq3(p.x, pm.x, k.x, xm0, p.y, ym.x, yp.x, zm.x, zp.x);
    q.y = eq3(p.y, pm.y, k.y, p.x, p.z, ym.y, yp.y, zm.y, zp.y);
    q.z = eq3(p.z, pm.z, k.z, p.y, p.w, ym.z, yp.z, zm.z, zp.z);
    q.w = eq3(p.w, pm.w, k.w, p.z, xp3, ym.w, yp.w, zm.w, zp.w);
    return q;
}

__device__ __forceinline__ float comp(const float4 &v, int j)
{
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

__device__ __forceinline__ void add_comp(float4 &v, int j, float w)
{
    if (j == 0) v.x = __fadd_rn(v.x, w);
    else if (j == 1) v.y = __fadd_rn(v.y, w);
    else if (j == 2) v.z = __fadd_rn(v.z, w);
    else v.w = __fadd_rn(v.w, w);
}

__device__ __forceinline__ float max4abs(const float4 &v)
{
    return fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
}

__device__ __forceinline__ float seg_max(float v)
{
#pragma unroll
    for (int o = TPB / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o, TPB));
    return v;
}

__device__ __forceinline__ const float4 *half4(const Engine &E, int slot, int half)
{
    return reinterpret_cast<const float4 *>(E.phi + ((size_t)slot * 2 + half) * BVOL);
}

// ---------------------------------------------------------------------------
// P1: one brick per TPB-lane segment.  Every lane of the warp calls this (with
// valid = false on a missing brick) so the shuffles see full warps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void p1_brick(const Engine &E, int slot, bool valid, int t,
                                         unsigned long long &cells)
{
    const int x4 = t % XQ;
    const int y = t / XQ;
    SlotMeta m;
    if (valid) {
        m = load_meta(E.meta + slot);
    } else {
        m.brick = 0;
        m.kslab = -1;
        m.kscal = 0.f;
        m.flags = 0u;
    }
    const int sim = (int)(m.flags >> 16);
    SimDev *S = E.sims + sim;
    const int mx = S->mx, my = S->my, mz = S->mz;
    const int nx = S->nx, ny = S->ny, nz = S->nz;
    const long long bb = S->brick_base;
    const long long step = __ldcg(&S->step);
    const int b = m.brick;
    const int cx = b % mx, cy = (b / mx) % my, cz = b / (mx * my);

    // Cell2box of the six face neighbours (lanes 0..5 look one up each).
    int nslot = -3;
    if (valid && t < 6) {
        const int ax = cx + (t == 0 ? -1 : (t == 1 ? 1 : 0));
        const int ay = cy + (t == 2 ? -1 : (t == 3 ? 1 : 0));
        const int az = cz + (t == 4 ? -1 : (t == 5 ? 1 : 0));
        if (ax >= 0 && ay >= 0 && az >= 0 && ax < mx && ay < my && az < mz)
            nslot = E.slot_of_brick[bb + ((long long)az * my + ay) * mx + ax];
    }
    const int s_xm = __shfl_sync(FULL, nslot, 0, TPB);
    const int s_xp = __shfl_sync(FULL, nslot, 1, TPB);
    const int s_ym = __shfl_sync(FULL, nslot, 2, TPB);
    const int s_yp = __shfl_sync(FULL, nslot, 3, TPB);
    const int s_zm = __shfl_sync(FULL, nslot, 4, TPB);
    const int s_zp = __shfl_sync(FULL, nslot, 5, TPB);

    const int nh = (int)(step & 1);
    float4 P[BZ], Q[BZ], K[BZ];
    if (valid) {
        const float4 *now4 = half4(E, slot, nh);
        const float4 *prv4 = half4(E, slot, nh ^ 1);
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            P[z] = __ldg(now4 + z * TPB + t);
            Q[z] = __ldcs(prv4 + z * TPB + t);
        }
        if (m.kslab >= 0) {
            const float4 *k4 = reinterpret_cast<const float4 *>(E.kslabs + (size_t)m.kslab * BVOL);
#pragma unroll
            for (int z = 0; z < BZ; ++z) K[z] = __ldg(k4 + z * TPB + t);
        } else {
#pragma unroll
            for (int z = 0; z < BZ; ++z) K[z] = make_float4(m.kscal, m.kscal, m.kscal, m.kscal);
        }
    } else {
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            P[z] = f4zero();
            Q[z] = f4zero();
            K[z] = f4zero();
        }
    }
    // Halo ("padding the box ... by the boundaries of its relevant neighbors").
    float4 Zm = f4zero(), Zp = f4zero();
    if (s_zm >= 0) Zm = __ldg(half4(E, s_zm, nh) + (BZ - 1) * TPB + t);
    if (s_zp >= 0) Zp = __ldg(half4(E, s_zp, nh) + t);
    const int ys = (y == 0) ? s_ym : ((y == BY - 1) ? s_yp : -1);
    const int yrow = (y == 0) ? BY - 1 : 0;
    const int xs = (x4 == 0) ? s_xm : ((x4 == XQ - 1) ? s_xp : -1);
    const int xcol = (x4 == 0) ? BX - 1 : 0;
    float4 Yh[BZ];
    float Xh[BZ];
    if (ys >= 0) {
        const float4 *yb = half4(E, ys, nh) + yrow * XQ + x4;
#pragma unroll
        for (int z = 0; z < BZ; ++z) Yh[z] = __ldg(yb + z * TPB);
    } else {
#pragma unroll
        for (int z = 0; z < BZ; ++z) Yh[z] = f4zero();
    }
    if (xs >= 0) {
        const float *xb = E.phi + ((size_t)xs * 2 + nh) * BVOL + y * BX + xcol;
#pragma unroll
        for (int z = 0; z < BZ; ++z) Xh[z] = __ldg(xb + z * BY * BX);
    } else {
#pragma unroll
        for (int z = 0; z < BZ; ++z) Xh[z] = 0.f;
    }

    // Eq. 3, plane by plane.
#pragma unroll
    for (int z = 0; z < BZ; ++z) {
        const float4 p = P[z];
        const float lw = __shfl_up_sync(FULL, p.w, 1, TPB);
        const float rx = __shfl_down_sync(FULL, p.x, 1, TPB);
        const float xm0 = (x4 == 0) ? Xh[z] : lw;
        const float xp3 = (x4 == XQ - 1) ? Xh[z] : rx;
        float4 ym, yp;
        ym.x = __shfl_up_sync(FULL, p.x, XQ, TPB);
        ym.y = __shfl_up_sync(FULL, p.y, XQ, TPB);
        ym.z = __shfl_up_sync(FULL, p.z, XQ, TPB);
        ym.w = __shfl_up_sync(FULL, p.w, XQ, TPB);
        yp.x = __shfl_down_sync(FULL, p.x, XQ, TPB);
        yp.y = __shfl_down_sync(FULL, p.y, XQ, TPB);
        yp.z = __shfl_down_sync(FULL, p.z, XQ, TPB);
        yp.w = __shfl_down_sync(FULL, p.w, XQ, TPB);
        if (y == 0) ym = Yh[z];
        if (y == BY - 1) yp = Yh[z];
        const float4 zm = (z > 0) ? P[z > 0 ? z - 1 : 0] : Zm;
        const float4 zp = (z < BZ - 1) ? P[z < BZ - 1 ? z + 1 : 0] : Zp;
        Q[z] = eq3v(p, Q[z], K[z], xm0, xp3, ym, yp, zm, zp);
    }

    // Source insertion in box coordinates.
    if (valid && (m.flags & FLAG_HAS_SRC)) {
        for (int s = S->src_begin; s < S->src_end; ++s) {
            const SrcDev sd = E.src[s];
            if (sd.brick != b) continue;
            const long long tt = step - sd.start;
            if (tt < 0 || tt >= sd.len) continue;
            const int lx = sd.local % BX, ly = (sd.local / BX) % BY, lz = sd.local / (BX * BY);
            if (ly != y || (lx >> 2) != x4) continue;
            const float w = E.wave[sd.w_off + tt];
#pragma unroll
            for (int z = 0; z < BZ; ++z)
                if (z == lz) add_comp(Q[z], lx & 3, w);
        }
    }
    // Time-domain shut-down (Eq. 6).
    if ((m.flags & SD_MASK) != 0u) {
        const float a = S->alpha;
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            Q[z].x = __fmul_rn(a, Q[z].x);
            Q[z].y = __fmul_rn(a, Q[z].y);
            Q[z].z = __fmul_rn(a, Q[z].z);
            Q[z].w = __fmul_rn(a, Q[z].w);
        }
    }
    // Nodes outside the domain stay zero.
    const int gx0 = cx * BX + 4 * x4, gy = cy * BY + y, gz0 = cz * BZ;
    if ((cx + 1) * BX > nx || (cy + 1) * BY > ny || (cz + 1) * BZ > nz) {
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            const bool rowin = gy < ny && gz0 + z < nz;
            if (!rowin || gx0 + 0 >= nx) Q[z].x = 0.f;
            if (!rowin || gx0 + 1 >= nx) Q[z].y = 0.f;
            if (!rowin || gx0 + 2 >= nx) Q[z].z = 0.f;
            if (!rowin || gx0 + 3 >= nx) Q[z].w = 0.f;
        }
    }
    if (valid) {
        float4 *prv4 = reinterpret_cast<float4 *>(E.phi + ((size_t)slot * 2 + (nh ^ 1)) * BVOL);
#pragma unroll
        for (int z = 0; z < BZ; ++z) prv4[z * TPB + t] = Q[z];
    }

    // Max_cell_val, face maxima, domain maximum.
    float mc = 0.f, qm = 0.f, f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f, f4 = 0.f, f5 = 0.f;
#pragma unroll
    for (int z = 0; z < BZ; ++z) {
        const float mq = max4abs(Q[z]);
        const float mp = max4abs(P[z]);
        qm = fmaxf(qm, mq);
        mc = fmaxf(mc, fmaxf(mq, mp));
        if (z == 0) f4 = mq;
        if (z == BZ - 1) f5 = mq;
        if (y == 0) f2 = fmaxf(f2, mq);
        if (y == BY - 1) f3 = fmaxf(f3, mq);
        if (x4 == 0) f0 = fmaxf(f0, fabsf(Q[z].x));
        if (x4 == XQ - 1) f1 = fmaxf(f1, fabsf(Q[z].w));
    }
    mc = seg_max(mc);
    qm = seg_max(qm);
    f0 = seg_max(f0);
    f1 = seg_max(f1);
    f2 = seg_max(f2);
    f3 = seg_max(f3);
    f4 = seg_max(f4);
    f5 = seg_max(f5);
    if (valid) {
        if (t < 6) E.nbr[(size_t)slot * 8 + t] = nslot;
        if (t == 0) {
            float4 *r = reinterpret_cast<float4 *>(E.rec + (size_t)slot * 8);
            r[0] = make_float4(f0, f1, f2, f3);
            r[1] = make_float4(f4, f5, mc, qm);
            unsigned *gp = &S->gmax[step & 1];
            const unsigned bits = __float_as_uint(qm);
            if (bits > __ldcg(gp)) atomicMax(gp, bits);
            const int ex = min(BX, nx - cx * BX), ey = min(BY, ny - cy * BY), ez = min(BZ, nz - cz * BZ);
            cells += (unsigned long long)(ex * ey * ez);
        }
    }
}

// ---------------------------------------------------------------------------
// P2 helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool brick_has_src(const Engine &E, const SimDev *S, int b)
{
    for (int s = S->src_begin; s < S->src_end; ++s)
        if (E.src[s].brick == b) return true;
    return false;
}

__device__ __forceinline__ bool forced_at(const Engine &E, const SimDev *S, int b, long long n)
{
    for (int s = S->src_begin; s < S->src_end; ++s) {
        const SrcDev &sd = E.src[s];
        if (sd.brick == b && n >= sd.start && n < sd.start + sd.len) return true;
    }
    return false;
}

// Trigger brick b_local of sim: box it unless it is already boxed or being
// boxed by another thread (Boxes: "Boxing new cells in vacant boxes").
__device__ void claim_brick(const Engine &E, int sim, SimDev *S, int b_local)
{
    const long long g = S->brick_base + b_local;
    if (atomicCAS(E.slot_of_brick + g, -1, -2) != -1) return;
    const int top = atomicSub(&E.st->free_top, 1) - 1;
    if (top < 0) {
        atomicExch(E.slot_of_brick + g, -1);
        atomicOr(&E.st->err, ERR_NOMEM);
        atomicOr(&S->poisoned, 1u);
        return;
    }
    const int ns = __ldcg(E.free_stack + top);
    SlotMeta m;
    m.brick = b_local;
    m.kslab = E.kslab_of_brick[g];
    m.kscal = E.kscal[g];
    m.flags = ((unsigned)sim << 16) | (brick_has_src(E, S, b_local) ? FLAG_HAS_SRC : 0u);
    store_meta(E.meta + ns, m);
    atomicOr(E.bitmap + (g >> 5), 1u << (unsigned)(g & 31));
    atomicAdd(E.blocktot + (int)((g >> 5) / E.words_per_block), 1);
    E.newslots[atomicAdd(&E.st->n_new, 1)] = ns;
    atomicExch(E.slot_of_brick + g, ns);
}

__device__ __forceinline__ int warp_incl_scan(int x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block scan of v; *total receives the block sum.
__device__ int block_excl_scan(int v, int *total)
{
    __shared__ int s_w[BLOCK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int inc = warp_incl_scan(v);
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int w = lane < BLOCK / 32 ? s_w[lane] : 0;
        w = warp_incl_scan(w);
        if (lane < BLOCK / 32) s_w[lane] = w;
    }
    __syncthreads();
    const int before = wid > 0 ? s_w[wid - 1] : 0;
    *total = s_w[BLOCK / 32 - 1];
    __syncthreads();
    return before + inc - v;
}

__device__ long long block_sum(long long v)
{
    __shared__ long long s_w[BLOCK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0) s_w[wid] = v;
    __syncthreads();
    long long r = 0;
#pragma unroll
    for (int i = 0; i < BLOCK / 32; ++i) r += s_w[i];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// The step kernel.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BLOCK, 2) k_step(Engine E)
{
    EngineState *st = E.st;
    const int cur = __ldcg(&st->list_parity);
    const int *L = cur ? E.list1 : E.list0;
    int *Lnext = cur ? E.list0 : E.list1;
    const int nact = __ldcg(&st->n_active[cur]);
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * BLOCK) >> 5;

    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // Boxes released last step were pushed above max(free_top, 0).
        const int ft = max(__ldcg(&st->free_top), 0) + __ldcg(&st->n_retired);
        st->free_top = ft;
        st->n_retired = 0;
        st->n_new = 0;
    }

    // ---- P1: time stepping of every active brick -------------------------
    {
        unsigned long long cells = 0;
        const int seg = lane / TPB;
        const int t = lane % TPB;
        for (int base = gwarp * BRICKS_PER_WARP; base < nact; base += nwarps * BRICKS_PER_WARP) {
            const int i = base + seg;
            const bool valid = i < nact;
            const int slot = valid ? __ldg(L + i) : 0;
            p1_brick(E, slot, valid, t, cells);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cells += __shfl_xor_sync(FULL, cells, o);
        if (lane == 0 && cells) atomicAdd(&st->updates, cells);
    }
    if (!grid_barrier(st)) return;

    // ---- P2: updating active cells ---------------------------------------
    {
        const int gtid = blockIdx.x * BLOCK + threadIdx.x;
        const int nthr = gridDim.x * BLOCK;
        for (int i = gtid; i < nact; i += nthr) {
            const int slot = __ldg(L + i);
            const SlotMeta m = load_meta(E.meta + slot);
            const int sim = (int)(m.flags >> 16);
            SimDev *S = E.sims + sim;
            if (S->dense) continue;
            const long long step = __ldcg(&S->step);
            const double G = (double)__uint_as_float(__ldcg(&S->gmax[step & 1]));
            const double thr = S->thr_mode == 1 ? S->tau * G : S->tau;
            const float4 r0 = __ldcg(reinterpret_cast<const float4 *>(E.rec + (size_t)slot * 8));
            const float4 r1 = __ldcg(reinterpret_cast<const float4 *>(E.rec + (size_t)slot * 8) + 1);
            const int4 n0 = __ldcg(reinterpret_cast<const int4 *>(E.nbr + (size_t)slot * 8));
            const int4 n1 = __ldcg(reinterpret_cast<const int4 *>(E.nbr + (size_t)slot * 8) + 1);
            const float fc[6] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y};
            const int ns[6] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y};
            bool hot = (double)r1.z > thr;
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (!hot && ns[f] >= 0) {
                    const float v = __ldcg(E.rec + (size_t)ns[f] * 8 + (f ^ 1));
                    if ((double)v > thr) hot = true;
                }
            }
            const int b = m.brick;
            if (!hot && (m.flags & FLAG_HAS_SRC) && forced_at(E, S, b, step + 1)) hot = true;
            unsigned sd = m.flags & SD_MASK;
            bool keep;
            if (hot) {
                sd = 0;
                keep = true;
            } else if (sd > 0) {
                sd -= 1;
                keep = sd > 0;
            } else if (S->decay_steps > 0) {
                sd = (unsigned)S->decay_steps;
                keep = true;
            } else {
                keep = false;
            }
            const long long g = S->brick_base + b;
            if (keep) {
                const unsigned nf = (m.flags & ~SD_MASK) | sd;
                if (nf != m.flags) E.meta[slot].flags = nf;
            } else {
                atomicExch(E.slot_of_brick + g, -1);
                atomicAnd(E.bitmap + (g >> 5), ~(1u << (unsigned)(g & 31)));
                atomicSub(E.blocktot + (int)((g >> 5) / E.words_per_block), 1);
                E.retired[atomicAdd(&st->n_retired, 1)] = slot;
            }
            // Trigger the neighbours across faces above the level (Fig. 3a).
            const int mx = S->mx, my = S->my;
            const int cx = b % mx, cy = (b / mx) % my, cz = b / (mx * my);
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (ns[f] == -1 && (double)fc[f] > thr) {
                    const int ax = cx + (f == 0 ? -1 : (f == 1 ? 1 : 0));
                    const int ay = cy + (f == 2 ? -1 : (f == 3 ? 1 : 0));
                    const int az = cz + (f == 4 ? -1 : (f == 5 ? 1 : 0));
                    claim_brick(E, sim, S, (az * my + ay) * mx + ax);
                }
            }
        }
        // Manual activation of source bricks still being fed at step n+1.
        if (blockIdx.x == 0) {
            for (int s = threadIdx.x; s < E.n_src; s += BLOCK) {
                const SrcDev sd = E.src[s];
                SimDev *S = E.sims + sd.sim;
                if (S->dense) continue;
                const long long n1 = __ldcg(&S->step) + 1;
                if (n1 >= sd.start && n1 < sd.start + sd.len) claim_brick(E, sd.sim, S, sd.brick);
            }
        }
    }
    if (!grid_barrier(st)) return;

    // ---- P3: box recycling and compaction of the active list -------------
    {
        const int gtid = blockIdx.x * BLOCK + threadIdx.x;
        const int nthr = gridDim.x * BLOCK;
        const int n_new = __ldcg(&st->n_new);
        for (int i = gwarp; i < n_new; i += nwarps) {
            float4 *p = reinterpret_cast<float4 *>(E.phi + (size_t)__ldcg(E.newslots + i) * 2 * BVOL);
            for (int e = lane; e < 2 * BVOL / 4; e += 32) p[e] = f4zero();
        }
        const int n_ret = __ldcg(&st->n_retired);
        const int base = max(__ldcg(&st->free_top), 0);
        for (int i = gtid; i < n_ret; i += nthr) E.free_stack[base + i] = __ldcg(E.retired + i);

        // Offset of this block's bitmap range = active bricks in earlier ranges.
        long long before = 0, all = 0;
        for (int j = threadIdx.x; j < (int)gridDim.x; j += BLOCK) {
            const int v = __ldcg(E.blocktot + j);
            all += v;
            if (j < (int)blockIdx.x) before += v;
        }
        before = block_sum(before);
        all = block_sum(all);
        const long long w0 = (long long)blockIdx.x * E.words_per_block;
        const long long w1 = min(w0 + E.words_per_block, E.n_words);
        int off = (int)before;
        for (long long wb = w0; wb < w1; wb += BLOCK) {
            const long long w = wb + threadIdx.x;
            unsigned bits = w < w1 ? __ldcg(E.bitmap + w) : 0u;
            int total;
            int pos = off + block_excl_scan(__popc(bits), &total);
            while (bits) {
                const int bit = __ffs(bits) - 1;
                bits &= bits - 1;
                if (pos < E.n_slots) Lnext[pos] = __ldcg(E.slot_of_brick + (w * 32 + bit));
                ++pos;
            }
            off += total;
        }
        if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) st->n_active[cur ^ 1] = (int)all;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            for (int s = 0; s < E.n_sims; ++s) {
                SimDev *S = E.sims + s;
                const long long n = S->step;
                S->gmax[(n + 1) & 1] = 0u;
                S->step = n + 1;
            }
            st->list_parity = cur ^ 1;
            st->launches += 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Heterogenic Bulking (create time)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float k_of_c(float c, double dt, double dx)
{
    const double r = (double)c * dt / dx;
    return (float)(r * r);
}

__device__ float media_c(const MediaDev &M, int nx, int ny, long long i, long long j, long long l)
{
    if (M.kind == MEDIA_DENSE) return M.c[(l * ny + j) * nx + i];
    float c = M.c_bg;
    for (int m = 0; m < M.n_layers; ++m)
        if ((double)l >= M.layer_z[m]) c = M.layer_c[m];
    for (int s = 0; s < M.n_spheres; ++s) {
        const double dx = (double)i - M.sph[4 * s + 0];
        const double dy = (double)j - M.sph[4 * s + 1];
        const double dz = (double)l - M.sph[4 * s + 2];
        const double r = M.sph[4 * s + 3];
        if (dx * dx + dy * dy + dz * dz <= r * r) c = M.sph_c[s];
    }
    return c;
}

// Nearest distance (as the rule computes it) from coordinate X to [lo, hi].
__device__ __forceinline__ double near_axis(double X, long long lo, long long hi)
{
    if (X <= (double)lo) return fabs((double)lo - X);
    if (X >= (double)hi) return fabs((double)hi - X);
    return fmin(fabs(floor(X) - X), fabs(ceil(X) - X));
}

// True when no rule boundary crosses the node box [x0,x1]x[y0,y1]x[z0,z1]:
// every node then has the same velocity.  The rule's expressions are
// monotone in each |coordinate - centre|, so the box extremes decide.
__device__ bool rules_uniform(const MediaDev &M, long long x0, long long x1, long long y0,
                              long long y1, long long z0, long long z1)
{
    for (int m = 0; m < M.n_layers; ++m)
        if (((double)z0 >= M.layer_z[m]) != ((double)z1 >= M.layer_z[m])) return false;
    for (int s = 0; s < M.n_spheres; ++s) {
        const double X = M.sph[4 * s + 0], Y = M.sph[4 * s + 1], Z = M.sph[4 * s + 2];
        const double r = M.sph[4 * s + 3];
        const double fx = fmax(fabs((double)x0 - X), fabs((double)x1 - X));
        const double fy = fmax(fabs((double)y0 - Y), fabs((double)y1 - Y));
        const double fz = fmax(fabs((double)z0 - Z), fabs((double)z1 - Z));
        const double far2 = fx * fx + fy * fy + fz * fz;
        const double ax = near_axis(X, x0, x1), ay = near_axis(Y, y0, y1), az = near_axis(Z, z0, z1);
        const double near2 = ax * ax + ay * ay + az * az;
        const double rr = r * r;
        if (!(far2 <= rr) && !(near2 > rr)) return false;
    }
    return true;
}

__global__ void k_bulk_classify(MediaDev M, int nx, int ny, int nz, int mx, int my, int mz, double dt,
                                double dx, float *kscal, int *kslab_of_brick, int *n_kslabs)
{
    const long long nb = (long long)mx * my * mz;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nb; g += nw) {
        const long long cx = g % mx, cy = (g / mx) % my, cz = g / ((long long)mx * my);
        const long long x0 = cx * BX, y0 = cy * BY, z0 = cz * BZ;
        const long long x1 = min(x0 + BX, (long long)nx) - 1, y1 = min(y0 + BY, (long long)ny) - 1,
                        z1 = min(z0 + BZ, (long long)nz) - 1;
        const float k0 = k_of_c(media_c(M, nx, ny, x0, y0, z0), dt, dx);
        bool uniform = M.kind == MEDIA_RULES && rules_uniform(M, x0, x1, y0, y1, z0, z1);
        bool diff = false;
        if (!uniform) {
            for (int e = lane; e < BVOL; e += 32) {
                const long long gx = x0 + e % BX, gy = y0 + (e / BX) % BY, gz = z0 + e / (BX * BY);
                if (gx > x1 || gy > y1 || gz > z1) continue;
                const float k = k_of_c(media_c(M, nx, ny, gx, gy, gz), dt, dx);
                if (__float_as_uint(k) != __float_as_uint(k0)) diff = true;
            }
            diff = __any_sync(FULL, diff);
        }
        if (lane == 0) {
            if (diff) {
                kslab_of_brick[g] = atomicAdd(n_kslabs, 1);
                kscal[g] = 0.f;
            } else {
                kslab_of_brick[g] = -1;
                kscal[g] = k0;
            }
        }
    }
}

__global__ void k_bulk_fill(MediaDev M, int nx, int ny, int nz, int mx, int my, int mz, double dt,
                            double dx, const int *kslab_of_brick, float *kslabs)
{
    const long long nb = (long long)mx * my * mz;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nb; g += nw) {
        const int ks = kslab_of_brick[g];
        if (ks < 0) continue;
        const long long cx = g % mx, cy = (g / mx) % my, cz = g / ((long long)mx * my);
        for (int e = lane; e < BVOL; e += 32) {
            const long long gx = cx * BX + e % BX, gy = cy * BY + (e / BX) % BY, gz = cz * BZ + e / (BX * BY);
            float k = 0.f;
            if (gx < nx && gy < ny && gz < nz) k = k_of_c(media_c(M, nx, ny, gx, gy, gz), dt, dx);
            kslabs[(size_t)ks * BVOL + e] = k;
        }
    }
}

// ---------------------------------------------------------------------------
// set-up, readback and diagnostics
// ---------------------------------------------------------------------------
__global__ void k_iota_desc(int *a, int n, int first)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = first - (int)i;
}

// Box the initial bricks: bricks[i] (or brick i when bricks == nullptr) gets
// box slot0 + i and list position slot0 + i.
__global__ void k_prime(Engine E, int sim, const long long *bricks, long long n, int slot0, int parity)
{
    SimDev *S = E.sims + sim;
    int *L = parity ? E.list1 : E.list0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int b = bricks ? (int)bricks[i] : (int)i;
        const int slot = slot0 + (int)i;
        const long long g = S->brick_base + b;
        E.slot_of_brick[g] = slot;
        SlotMeta m;
        m.brick = b;
        m.kslab = E.kslab_of_brick[g];
        m.kscal = E.kscal[g];
        m.flags = ((unsigned)sim << 16) | (brick_has_src(E, S, b) ? FLAG_HAS_SRC : 0u);
        store_meta(E.meta + slot, m);
        atomicOr(E.bitmap + (g >> 5), 1u << (unsigned)(g & 31));
        atomicAdd(E.blocktot + (int)((g >> 5) / E.words_per_block), 1);
        L[slot] = slot;
    }
}

__global__ void k_zero_slots(float *phi, int slot0, long long n)
{
    float4 *p = reinterpret_cast<float4 *>(phi + (size_t)slot0 * 2 * BVOL);
    const long long total = n * 2 * BVOL / 4;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        p[i] = f4zero();
}

// packed[i] = {now brick (BVOL), prev brick (BVOL)} for box slot0 + i.
__global__ void k_scatter_field(float *phi, const float *packed, long long n, int slot0, int now_half)
{
    const long long total = n * 2 * BVOL;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long brick = i / (2 * BVOL);
        const int r = (int)(i % (2 * BVOL));
        const int which = r / BVOL, e = r % BVOL;
        const int half = which == 0 ? now_half : (now_half ^ 1);
        phi[((size_t)(slot0 + brick) * 2 + half) * BVOL + e] = packed[i];
    }
}

__global__ void k_read_window(Engine E, int sim, int half, long long x0, long long y0, long long z0,
                              long long wx, long long wy, long long wz, float *out)
{
    const SimDev *S = E.sims + sim;
    const long long total = wx * wy * wz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long x = x0 + i % wx, y = y0 + (i / wx) % wy, z = z0 + i / (wx * wy);
        float v = 0.f;
        if (x >= 0 && y >= 0 && z >= 0 && x < S->nx && y < S->ny && z < S->nz) {
            const long long b = ((z / BZ) * S->my + (y / BY)) * S->mx + (x / BX);
            const int slot = E.slot_of_brick[S->brick_base + b];
            if (slot >= 0) {
                const int e = (int)(((z % BZ) * BY + (y % BY)) * BX + (x % BX));
                v = E.phi[((size_t)slot * 2 + half) * BVOL + e];
            }
        }
        out[i] = v;
    }
}

// phi^{n-1} at global node (x,y,z) of sim, zero outside or when inactive.
__device__ __forceinline__ double prev_at(const Engine &E, const SimDev *S, int prev_half, long long x,
                                          long long y, long long z)
{
    if (x < 0 || y < 0 || z < 0 || x >= S->nx || y >= S->ny || z >= S->nz) return 0.0;
    const long long b = ((z / BZ) * S->my + (y / BY)) * S->mx + (x / BX);
    const int slot = E.slot_of_brick[S->brick_base + b];
    if (slot < 0) return 0.0;
    return (double)E.phi[((size_t)slot * 2 + prev_half) * BVOL + ((z % BZ) * BY + (y % BY)) * BX + (x % BX)];
}

__global__ void k_energy(Engine E, int sim, int now_half, int parity, double *out)
{
    const SimDev *S = E.sims + sim;
    const int *L = parity ? E.list1 : E.list0;
    const long long n = (long long)E.st->n_active[parity] * BVOL;
    const int ph = now_half ^ 1;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int slot = L[i / BVOL];
        const int e = (int)(i % BVOL);
        const SlotMeta m = load_meta(E.meta + slot);
        if ((int)(m.flags >> 16) != sim) continue;
        const int b = m.brick;
        const long long x = (long long)(b % S->mx) * BX + e % BX;
        const long long y = (long long)((b / S->mx) % S->my) * BY + (e / BX) % BY;
        const long long z = (long long)(b / (S->mx * S->my)) * BZ + e / (BX * BY);
        if (x >= S->nx || y >= S->ny || z >= S->nz) continue;
        const double a = (double)E.phi[((size_t)slot * 2 + now_half) * BVOL + e];
        const double bb = (double)E.phi[((size_t)slot * 2 + ph) * BVOL + e];
        const double nb = prev_at(E, S, ph, x - 1, y, z) + prev_at(E, S, ph, x + 1, y, z) +
                          prev_at(E, S, ph, x, y - 1, z) + prev_at(E, S, ph, x, y + 1, z) +
                          prev_at(E, S, ph, x, y, z - 1) + prev_at(E, S, ph, x, y, z + 1);
        const double k = m.kslab >= 0 ? (double)E.kslabs[(size_t)m.kslab * BVOL + e] : (double)m.kscal;
        const double d = a - bb;
        acc += d * d / k + a * (6.0 * bb - nb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

__global__ void k_active_bricks(Engine E, int parity, long long *ids, unsigned long long *cells)
{
    const int *L = parity ? E.list1 : E.list0;
    const int n = E.st->n_active[parity];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SlotMeta m = load_meta(E.meta + L[i]);
        const SimDev *S = E.sims + (m.flags >> 16);
        const int b = m.brick;
        if (ids) ids[i] = b;
        const int cx = b % S->mx, cy = (b / S->mx) % S->my, cz = b / (S->mx * S->my);
        const int ex = min(BX, S->nx - cx * BX), ey = min(BY, S->ny - cy * BY), ez = min(BZ, S->nz - cz * BZ);
        if (cells) atomicAdd(cells, (unsigned long long)(ex * ey * ez));
    }
}

int grid_for(long long work, int block)
{
    long long g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 65535LL * 8) g = 65535LL * 8;
    return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_bulk_classify(const MediaDev &m, int nx, int ny, int nz, int mx, int my, int mz,
                                 double dt, double dx, float *kscal, int *kslab_of_brick,
                                 int *n_kslabs, cudaStream_t s)
{
    const long long nb = (long long)mx * my * mz;
    k_bulk_classify<<<grid_for(nb * 32, 256), 256, 0, s>>>(m, nx, ny, nz, mx, my, mz, dt, dx, kscal,
                                                           kslab_of_brick, n_kslabs);
    return cudaGetLastError();
}

cudaError_t launch_bulk_fill(const MediaDev &m, int nx, int ny, int nz, int mx, int my, int mz,
                             double dt, double dx, const int *kslab_of_brick, float *kslabs,
                             cudaStream_t s)
{
    const long long nb = (long long)mx * my * mz;
    k_bulk_fill<<<grid_for(nb * 32, 256), 256, 0, s>>>(m, nx, ny, nz, mx, my, mz, dt, dx,
                                                       kslab_of_brick, kslabs);
    return cudaGetLastError();
}

cudaError_t launch_iota_desc(int *a, int n, int first, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_iota_desc<<<grid_for(n, 256), 256, 0, s>>>(a, n, first);
    return cudaGetLastError();
}

cudaError_t launch_prime(const Engine &e, int sim, const long long *bricks, long long n, int slot0,
                         int list_parity, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_prime<<<grid_for(n, 256), 256, 0, s>>>(e, sim, bricks, n, slot0, list_parity);
    return cudaGetLastError();
}

cudaError_t launch_zero_slots(const Engine &e, int slot0, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_zero_slots<<<grid_for(n * 2 * BVOL / 4, 256), 256, 0, s>>>(e.phi, slot0, n);
    return cudaGetLastError();
}

cudaError_t launch_scatter_field(const Engine &e, const float *packed, long long n, int slot0,
                                 int now_half, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_scatter_field<<<grid_for(n * 2 * BVOL, 256), 256, 0, s>>>(e.phi, packed, n, slot0, now_half);
    return cudaGetLastError();
}

int step_grid_size(int device)
{
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step, BLOCK, 0) != cudaSuccess) return 0;
    return sms * per_sm;
}

cudaError_t launch_step(const Engine &e, int grid, cudaStream_t s)
{
    Engine copy = e;
    void *args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void *)k_step, dim3(grid), dim3(BLOCK), args, 0, s);
}

cudaError_t launch_read_window(const Engine &e, int sim, int half, long long x0, long long y0,
                               long long z0, long long wx, long long wy, long long wz, float *out,
                               cudaStream_t s)
{
    const long long n = wx * wy * wz;
    if (n <= 0) return cudaSuccess;
    k_read_window<<<grid_for(n, 256), 256, 0, s>>>(e, sim, half, x0, y0, z0, wx, wy, wz, out);
    return cudaGetLastError();
}

cudaError_t launch_energy(const Engine &e, int sim, int now_half, int list_parity, double *out,
                          cudaStream_t s)
{
    k_energy<<<1024, 256, 0, s>>>(e, sim, now_half, list_parity, out);
    return cudaGetLastError();
}

cudaError_t launch_active_bricks(const Engine &e, int list_parity, long long *ids_out,
                                 unsigned long long *cells_out, cudaStream_t s)
{
    k_active_bricks<<<256, 256, 0, s>>>(e, list_parity, ids_out, cells_out);
    return cudaGetLastError();
}

}  // namespace tcm
