// tcm_kernels.cu -- sm_103a kernels of the Triggered Cells Method
// (Naeh, arXiv:1702.00216).
//
// The hot path is one cooperative, persistent launch per time step (k_step):
//   P1  Eq. 3 on every active brick (Time stepping section): a half-warp owns one
//       8x8x8 brick, each lane one float4 column marching in z; the one-node
//       halo comes from the six face neighbours' boxes (zero where a neighbour
//       is inactive or outside the domain), the x/y neighbours inside the
//       brick come through warp shuffles, so no shared-memory round trip.  The
//       epilogue inserts source samples, applies the Eq. 6 decay, stores
//       phi^{n+1} over phi^{n-1} (float4, coalesced) and reduces the cell
//       maximum, six face maxima and the domain maximum with shuffles.
//   --  device-wide barrier (bounded wait)
//   P2  the update procedure (Simulation section, Fig. 3a): each active brick decides keep / shut-down /
//       release from its own maximum and its neighbours' touching faces, and
//       claims the neighbours across faces above the trigger level
//       (atomicCAS on Cell2box, a box popped from the free stack).
//   --  device-wide barrier
//   P3  zero the claimed boxes, return released boxes to the free stack and
//       rebuild the active list from the brick bitmap (warp ballot/popc +
//       block prefix scan), in brick order, for the next launch.
// Arithmetic: binary32, every + - * an explicit round-to-nearest intrinsic
// (no FMA contraction), no flush-to-zero.
#include <cmath>
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include "tcm_internal.cuh"

namespace cg = cooperative_groups;

namespace tcm {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long BARRIER_TIMEOUT_NS = 4000000000ull;  // 4 s

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Device-wide barrier for a cooperative launch: one arrival per block on a
// counter that only grows (the blocks of a launch arrive gridDim.x times per
// barrier, so the barrier ends when the counter reaches the next multiple of
// gridDim.x); thread 0 arrives with an acquire-release atomic after the
// block's __syncthreads and waits with acquire loads, then the block
// synchronises again.  The wait is bounded: after timeout_ns the block
// records ERR_TIMEOUT and returns false, and the caller leaves the kernel
// (the others then time out at their next barrier).
__device__ bool grid_barrier(EngineState *st, unsigned long long *ctr,
                             unsigned long long timeout_ns = BARRIER_TIMEOUT_NS)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned long long old;
        asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], 1;" : "=l"(old) : "l"(ctr) : "memory");
        const unsigned long long target = (old / gridDim.x + 1) * gridDim.x;
        unsigned long long cur;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(cur) : "l"(ctr) : "memory");
        if (cur < target) {
            const unsigned long long t0 = globaltimer();
            do {
                if (globaltimer() - t0 > timeout_ns) {
                    atomicOr(&st->err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(cur) : "l"(ctr) : "memory");
            } while (cur < target);
        }
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
    const float s = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(xm, xp), ym), yp), zm), zp);
    const float lap = __fsub_rn(s, __fmul_rn(6.0f, p));
    return __fadd_rn(__fsub_rn(__fmul_rn(2.0f, p), pm), __fmul_rn(k, lap));
}

// Velocity form (16-bit storages): v + k lap, the same lap as eq3.
__device__ __forceinline__ float vel3(float p, float v, float k, float xm, float xp, float ym, float yp, float zm,
                                      float zp)
{
    const float s = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(xm, xp), ym), yp), zm), zp);
    const float lap = __fsub_rn(s, __fmul_rn(6.0f, p));
    return __fadd_rn(v, __fmul_rn(k, lap));
}

__device__ __forceinline__ float4 vel3v(float4 p, float4 v, float4 k, float xm0, float xp3, float4 ym, float4 yp,
                                        float4 zm, float4 zp)
{
    float4 q;
    q.x = vel3(p.x, v.x, k.x, xm0, p.y, ym.x, yp.x, zm.x, zp.x);
    q.y = vel3(p.y, v.y, k.y, p.x, p.z, ym.y, yp.y, zm.y, zp.y);
    q.z = vel3(p.z, v.z, k.z, p.y, p.w, ym.z, yp.z, zm.z, zp.z);
    q.w = vel3(p.w, v.w, k.w, p.z, xp3, ym.w, yp.w, zm.w, zp.w);
    return q;
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


__device__ __forceinline__ WorkItem load_item(const WorkItem *L, int i)
{
    const int4 *p = reinterpret_cast<const int4 *>(L + i);
    const int4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    WorkItem w;
    w.slot = a.x;
    w.brick = a.y;
    w.kp = ((unsigned long long)(unsigned)a.w << 32) | (unsigned)a.z;
    w.flags = (unsigned)b.x;
    w.nb[0] = b.y;
    w.nb[1] = b.z;
    w.nb[2] = b.w;
    w.nb[3] = c.x;
    w.nb[4] = c.y;
    w.nb[5] = c.z;
    w.nh = c.w;
    return w;
}

// Vector access to 4 consecutive field elements (x fastest) in the storage
// format ST, as physical binary32 values.  Scaling by a power of two is exact.
template <int ST>
struct Fld;

template <>
struct Fld<ST_F32> {
    using T = float;
    static __device__ __forceinline__ float4 ld(const T *p, float) { return __ldg(reinterpret_cast<const float4 *>(p)); }
    static __device__ __forceinline__ float4 ld_stream(const T *p, float)
    {
        return __ldcs(reinterpret_cast<const float4 *>(p));
    }
    static __device__ __forceinline__ float ld1(const T *p, float) { return __ldg(p); }
    // Round q to the storage format: returns the stored value (physical) and
    // its bit pattern for st().
    using V = float4;
    static __device__ __forceinline__ float4 rnd(float4 q, float, float, V &v)
    {
        v = q;
        return q;
    }
    static __device__ __forceinline__ void st(T *p, V v) { __stcg(reinterpret_cast<float4 *>(p), v); }
};

__device__ __forceinline__ float4 scale4(float4 v, float s)
{
    return make_float4(v.x * s, v.y * s, v.z * s, v.w * s);
}

template <>
struct Fld<ST_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float4 cvt(uint2 u, float s)
    {
        return scale4(make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                                  __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u)),
                      s);
    }
    static __device__ __forceinline__ float4 ld(const T *p, float s)
    {
        return cvt(__ldg(reinterpret_cast<const uint2 *>(p)), s);
    }
    static __device__ __forceinline__ float4 ld_stream(const T *p, float s)
    {
        return cvt(__ldcs(reinterpret_cast<const uint2 *>(p)), s);
    }
    static __device__ __forceinline__ float ld1(const T *p, float s)
    {
        return __uint_as_float((unsigned)__ldg(reinterpret_cast<const unsigned short *>(p)) << 16) * s;
    }
    using V = uint2;
    static __device__ __forceinline__ float4 rnd(float4 q, float s, float inv_s, V &v)
    {
        const __nv_bfloat162 a = __floats2bfloat162_rn(q.x * inv_s, q.y * inv_s);
        const __nv_bfloat162 b = __floats2bfloat162_rn(q.z * inv_s, q.w * inv_s);
        v.x = *reinterpret_cast<const unsigned *>(&a);
        v.y = *reinterpret_cast<const unsigned *>(&b);
        return cvt(v, s);
    }
    static __device__ __forceinline__ void st(T *p, V v) { __stcg(reinterpret_cast<uint2 *>(p), v); }
};

template <>
struct Fld<ST_F16> {
    using T = __half;
    static __device__ __forceinline__ float4 cvt(uint2 u, float s)
    {
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
        return scale4(make_float4(a.x, a.y, b.x, b.y), s);
    }
    static __device__ __forceinline__ float4 ld(const T *p, float s)
    {
        return cvt(__ldg(reinterpret_cast<const uint2 *>(p)), s);
    }
    static __device__ __forceinline__ float4 ld_stream(const T *p, float s)
    {
        return cvt(__ldcs(reinterpret_cast<const uint2 *>(p)), s);
    }
    static __device__ __forceinline__ float ld1(const T *p, float s)
    {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p)))) * s;
    }
    using V = uint2;
    static __device__ __forceinline__ float4 rnd(float4 q, float s, float inv_s, V &v)
    {
        const __half2 a = __floats2half2_rn(q.x * inv_s, q.y * inv_s);
        const __half2 b = __floats2half2_rn(q.z * inv_s, q.w * inv_s);
        v.x = *reinterpret_cast<const unsigned *>(&a);
        v.y = *reinterpret_cast<const unsigned *>(&b);
        return cvt(v, s);
    }
    static __device__ __forceinline__ void st(T *p, V v) { __stcg(reinterpret_cast<uint2 *>(p), v); }
};

// Array `half` of a box: 0/1 the field halves, V_HALF the velocity (16-bit).
// MIX: a batch of mixed storages, whose boxes are E.slot_bytes apart.
template <int ST, bool MIX = false>
__device__ __forceinline__ typename Fld<ST>::T *half_ptr(const Engine &E, int slot, int half)
{
    using T = typename Fld<ST>::T;
    if constexpr (MIX) return reinterpret_cast<T *>(box_base(E, slot)) + (size_t)half * BVOL;
    return static_cast<T *>(E.phi) + (size_t)slot * slot_elems(ST) + (size_t)half * BVOL;
}

// Zero one box (every array of it) with the lanes of a warp.
__device__ __forceinline__ void zero_box(const Engine &E, int slot, int lane)
{
    const size_t bytes = (size_t)E.slot_bytes;
    const int n16 = (int)(bytes / 16);
    float4 *p = reinterpret_cast<float4 *>(static_cast<unsigned char *>(E.phi) + (size_t)slot * bytes);
    for (int e = lane; e < n16; e += 32) p[e] = f4zero();
}

// Merge a lane's running max |phi^{n+1}| into its sim's domain maximum.  The
// step being computed has phi^n in half nh, so its maximum lives in gmax[nh].
__device__ __forceinline__ void flush_gmax(const Engine &E, float gacc, int gsim, int nh)
{
    if (gsim >= 0 && gacc > 0.f) atomicMax(&E.sims[gsim].gmax[nh], __float_as_uint(gacc));
}

// Add a lane's node-update count to its sim's counter.
__device__ __forceinline__ void flush_updates(const Engine &E, unsigned long long &n, int gsim)
{
    if (gsim >= 0 && n) atomicAdd(&E.sims[gsim].updates, n);
    n = 0;
}

// Two 16-bit values of storage ST packed in a word (low half first): the
// larger of each half, and the halves as binary32.
template <int ST>
__device__ __forceinline__ unsigned hmax2u(unsigned a, unsigned b)
{
    if constexpr (ST == ST_BF16) {
        const __nv_bfloat162 r =
            __hmax2(*reinterpret_cast<const __nv_bfloat162 *>(&a), *reinterpret_cast<const __nv_bfloat162 *>(&b));
        return *reinterpret_cast<const unsigned *>(&r);
    } else {
        const __half2 r = __hmax2(*reinterpret_cast<const __half2 *>(&a), *reinterpret_cast<const __half2 *>(&b));
        return *reinterpret_cast<const unsigned *>(&r);
    }
}

template <int ST>
__device__ __forceinline__ float half_lo(unsigned u)
{
    if constexpr (ST == ST_BF16) return __uint_as_float(u << 16);
    else return __half2float(__ushort_as_half((unsigned short)(u & 0xffffu)));
}

template <int ST>
__device__ __forceinline__ float half_hi(unsigned u)
{
    if constexpr (ST == ST_BF16) return __uint_as_float(u & 0xffff0000u);
    else return __half2float(__ushort_as_half((unsigned short)(u >> 16)));
}

template <int ST>
__device__ __forceinline__ float max2h(unsigned u)
{
    return fmaxf(half_lo<ST>(u), half_hi<ST>(u));
}

// ---------------------------------------------------------------------------
// P1: Eq. 3 on one brick per TPB-lane segment, straight from global memory.
// Each lane owns one float4 column (x4, y) of all BZ planes: it issues every
// load of the brick up front (phi^n, phi^{n-1}, k, and the halo values it
// needs from the six neighbours' boxes), so a warp keeps two bricks' worth of
// 16-byte loads in flight; x/y neighbours inside the brick come through warp
// shuffles.  When the pair's second brick is the x+ neighbour of the first
// (consecutive bricks of a row), their touching columns are exchanged between
// lanes (lane ^ 17) instead of being loaded.  Every lane of the warp calls
// this (valid = false on a missing brick) so shuffles see full warps.
// ---------------------------------------------------------------------------
template <int ST, bool MIX = false>
__device__ __forceinline__ void p1_brick(const Engine &E, const WorkItem &w, bool valid, int t, int seg,
                                         bool share_xm, bool share_xp, int age_flip, unsigned stamp,
                                         unsigned long long &cells, unsigned long long &scells, float &gacc,
                                         int &gsim, int &gnh)
{
    const int x4 = t % XQ;
    const int y = t / XQ;
    valid = valid && TCM_SLOT_OK(E, w.slot);
    const int sim = valid ? (int)(w.flags >> 16) : 0;
    SimDev *S = E.sims + sim;
    const int mx = __ldg(&S->mx), my = __ldg(&S->my);
    const int nx = __ldg(&S->nx), ny = __ldg(&S->ny), nz = __ldg(&S->nz);
    const int nh = w.nh ^ age_flip;   // the list may be older than this step
    const int b = w.brick;
    const int cx = b % mx, cy = (b / mx) % my, cz = b / (mx * my);
    using F = Fld<ST>;
    // The plane loop works in stored units (phi / scale, scale a power of
    // two; 1 for binary32 and bfloat16): every + - * then rounds to the same
    // bits as on physical values, so the stored results are unchanged.  The
    // source samples enter scaled, and the maxima leave scaled back.
    const float sc = __ldg(&S->scale), isc = __ldg(&S->inv_scale);
    constexpr float U1 = 1.f;

    // binary32 columns in P, M, YH; with more than 8 warps per CTA (at most
    // 170 registers a thread) 16-bit columns stay as loaded (two registers
    // per plane instead of four) in PR, MR, YR and are converted where the
    // plane loop uses them, phi^n once per plane
    constexpr bool RAW = ST != ST_F32 && P1_WARPS > 8;   // only where registers are tight
    float4 P[BZ], M[BZ], K[BZ], YH[BZ];
    [[maybe_unused]] uint2 PR[BZ], MR[BZ], YR[BZ];
    float XH[BZ];
    float XH2[XQ == 1 ? BZ : 1];
    float4 Zm = f4zero(), Zp = f4zero();
    // y-edge lanes read the touching row of y- / y+, x-edge lanes the
    // touching column of x- / x+ (unless exchanged within the pair)
    int ys = !valid ? -1 : (y == 0 ? w.nb[2] : (y == BY - 1 ? w.nb[3] : -1));
    if (ys >= 0 && !TCM_SLOT_OK(E, ys)) ys = -1;
    // x-edge lanes: the column of x- (x4 == 0) or x+ (x4 == XQ-1); with one
    // float4 per row (XQ == 1) a lane is both, and xs2 is the x+ one
    int xs = !valid ? -1 : (x4 == 0 ? (share_xm ? -1 : w.nb[0]) : (x4 == XQ - 1 ? (share_xp ? -1 : w.nb[1]) : -1));
    int xs2 = (XQ == 1 && valid && !share_xp) ? w.nb[1] : -1;
    if (xs >= 0 && !TCM_SLOT_OK(E, xs)) xs = -1;
    if (xs2 >= 0 && !TCM_SLOT_OK(E, xs2)) xs2 = -1;
    if (valid) {
        const typename F::T *now = half_ptr<ST, MIX>(E, w.slot, nh);
        // phi^{n-1} in binary32; v^n in the velocity form (16-bit storages)
        const typename F::T *prv = half_ptr<ST, MIX>(E, w.slot, ST == ST_F32 ? (nh ^ 1) : V_HALF);
        if constexpr (RAW) {
#pragma unroll
            for (int z = 0; z < BZ; ++z) PR[z] = __ldg(reinterpret_cast<const uint2 *>(now + 4 * (z * TPB + t)));
#pragma unroll
            for (int z = 0; z < BZ; ++z) MR[z] = __ldcs(reinterpret_cast<const uint2 *>(prv + 4 * (z * TPB + t)));
        } else {
#pragma unroll
            for (int z = 0; z < BZ; ++z) P[z] = F::ld(now + 4 * (z * TPB + t), U1);
#pragma unroll
            for (int z = 0; z < BZ; ++z) M[z] = F::ld_stream(prv + 4 * (z * TPB + t), U1);
        }
        if (!(w.kp & KP_SCALAR)) {
            const float4 *k4 = reinterpret_cast<const float4 *>(w.kp);
#pragma unroll
            for (int z = 0; z < BZ; ++z) K[z] = __ldg(k4 + z * TPB + t);
        } else {
            const float ks = __uint_as_float((unsigned)w.kp);
#pragma unroll
            for (int z = 0; z < BZ; ++z) K[z] = make_float4(ks, ks, ks, ks);
        }
        if (w.nb[4] >= 0 && TCM_SLOT_OK(E, w.nb[4]))
            Zm = F::ld(half_ptr<ST, MIX>(E, w.nb[4], nh) + 4 * ((BZ - 1) * TPB + t), U1);
        if (w.nb[5] >= 0 && TCM_SLOT_OK(E, w.nb[5])) Zp = F::ld(half_ptr<ST, MIX>(E, w.nb[5], nh) + 4 * t, U1);
    } else {
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            P[z] = f4zero();
            M[z] = f4zero();
            K[z] = f4zero();
            if constexpr (RAW) PR[z] = MR[z] = make_uint2(0u, 0u);
        }
    }
    if (ys >= 0) {
        const typename F::T *yb = half_ptr<ST, MIX>(E, ys, nh) + 4 * ((y == 0 ? BY - 1 : 0) * XQ + x4);
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            if constexpr (RAW) YR[z] = __ldg(reinterpret_cast<const uint2 *>(yb + 4 * z * TPB));
            else YH[z] = F::ld(yb + 4 * z * TPB, U1);
        }
    } else {
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            YH[z] = f4zero();
            if constexpr (RAW) YR[z] = make_uint2(0u, 0u);
        }
    }
    if (xs >= 0) {
        const typename F::T *xb = half_ptr<ST, MIX>(E, xs, nh) + y * BX + (x4 == 0 ? BX - 1 : 0);
#pragma unroll
        for (int z = 0; z < BZ; ++z) XH[z] = F::ld1(xb + z * BY * BX, U1);
    } else {
#pragma unroll
        for (int z = 0; z < BZ; ++z) XH[z] = 0.f;
    }
    if constexpr (XQ == 1) {
        if (xs2 >= 0) {
            const typename F::T *xb = half_ptr<ST, MIX>(E, xs2, nh) + y * BX;
#pragma unroll
            for (int z = 0; z < BZ; ++z) XH2[z] = F::ld1(xb + z * BY * BX, U1);
        } else {
#pragma unroll
            for (int z = 0; z < BZ; ++z) XH2[z] = 0.f;
        }
    }

    const float alpha = __ldg(&S->alpha);
    const bool decay = (w.flags & SD_MASK) != 0u;
    const bool ragged = (cx + 1) * BX > nx || (cy + 1) * BY > ny || (cz + 1) * BZ > nz;
    const int gx0 = cx * BX + 4 * x4, gy = cy * BY + y, gz0 = cz * BZ;
    typename F::T *out = half_ptr<ST, MIX>(E, w.slot, nh ^ 1);
    typename F::T *vout = half_ptr<ST, MIX>(E, w.slot, V_HALF);   // used by 16-bit storages only
    const bool src = valid && (w.flags & FLAG_HAS_SRC);
    const long long step = src ? __ldcg(&S->step) : 0;
    const bool xrecv = (x4 == 0 && share_xm) || (x4 == XQ - 1 && share_xp);

    float mc = 0.f, qm = 0.f, f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f, f4 = 0.f, f5 = 0.f;
    [[maybe_unused]] unsigned qm2 = 0u, f02 = 0u, f12 = 0u, f42 = 0u, f52 = 0u;
    // 16-bit: phi^n of the plane below, this plane and the plane above
    [[maybe_unused]] float4 pprev = Zm, pcur = f4zero();
    if constexpr (RAW) pcur = F::cvt(PR[0], U1);
#pragma unroll
    for (int z = 0; z < BZ; ++z) {
        float4 p, zm, zp;
        if constexpr (RAW) {
            p = pcur;
            zm = pprev;
            zp = (z < BZ - 1) ? F::cvt(PR[z < BZ - 1 ? z + 1 : 0], U1) : Zp;
            pprev = pcur;
            pcur = zp;
        } else {
            p = P[z];
            zm = (z > 0) ? P[z > 0 ? z - 1 : 0] : Zm;
            zp = (z < BZ - 1) ? P[z < BZ - 1 ? z + 1 : 0] : Zp;
        }
        // x neighbours inside the brick through shuffles; the edge value from
        // the loaded face column or, within a pair, from lane ^ 17 (the x = 7
        // column of the first brick / the x = 0 column of the second)
        float xm0, xp3;
        if constexpr (XQ == 1) {
            // the whole row in one float4: x- from the x- brick (or the pair's
            // first brick), x+ from the x+ brick (or the pair's second)
            float recv = 0.f;
            if constexpr (BRICKS_PER_WARP >= 2) recv = __shfl_xor_sync(FULL, share_xp ? p.w : p.x, TPB);
            xm0 = share_xm ? recv : XH[z];
            xp3 = share_xp ? recv : XH2[z];
        } else if constexpr (XQ == 2) {
            // the two columns of a row trade their touching values in one
            // shuffle: x4 = 0 gets p.x of x4 = 1, x4 = 1 gets p.w of x4 = 0
            const float nbr = __shfl_xor_sync(FULL, x4 == 0 ? p.w : p.x, 1);
            float recv = 0.f;
            if constexpr (BRICKS_PER_WARP >= 2)
                recv = __shfl_xor_sync(FULL, (x4 == XQ - 1) ? p.w : p.x, TPB + XQ - 1);
            const float xe = xrecv ? recv : XH[z];
            xm0 = (x4 == 0) ? xe : nbr;
            xp3 = (x4 == 0) ? nbr : xe;
        } else {
            const float lw = __shfl_up_sync(FULL, p.w, 1, TPB);
            const float rx = __shfl_down_sync(FULL, p.x, 1, TPB);
            float recv = 0.f;
            if constexpr (BRICKS_PER_WARP >= 2)
                recv = __shfl_xor_sync(FULL, (x4 == XQ - 1) ? p.w : p.x, TPB + XQ - 1);
            const float xe = xrecv ? recv : XH[z];
            xm0 = (x4 == 0) ? xe : lw;
            xp3 = (x4 == XQ - 1) ? xe : rx;
        }
        // y neighbours inside the brick through shuffles
        float4 ym, yp;
        ym.x = __shfl_up_sync(FULL, p.x, XQ, TPB);
        ym.y = __shfl_up_sync(FULL, p.y, XQ, TPB);
        ym.z = __shfl_up_sync(FULL, p.z, XQ, TPB);
        ym.w = __shfl_up_sync(FULL, p.w, XQ, TPB);
        yp.x = __shfl_down_sync(FULL, p.x, XQ, TPB);
        yp.y = __shfl_down_sync(FULL, p.y, XQ, TPB);
        yp.z = __shfl_down_sync(FULL, p.z, XQ, TPB);
        yp.w = __shfl_down_sync(FULL, p.w, XQ, TPB);
        if constexpr (RAW) {
            if (y == 0) ym = F::cvt(YR[z], U1);
            if (y == BY - 1) yp = F::cvt(YR[z], U1);
        } else {
            if (y == 0) ym = YH[z];
            if (y == BY - 1) yp = YH[z];
        }
        // binary32: q = phi^{n+1} by Eq. 3.  Velocity form: vq = v + k lap
        // (+ source), then q = phi^n + vq.
        float4 q, vq;
        if constexpr (ST == ST_F32) q = eq3v(p, M[z], K[z], xm0, xp3, ym, yp, zm, zp);
        else vq = vel3v(p, RAW ? F::cvt(MR[z], U1) : M[z], K[z], xm0, xp3, ym, yp, zm, zp);
        float4 &acc = (ST == ST_F32) ? q : vq;
        if (src) {
            // Source insertion in box coordinates: every sample of this
            // plane, in source order.
            for (int s = S->src_begin; s < S->src_end; ++s) {
                const SrcDev sd = E.src[s];
                if (sd.brick != b) continue;
                const long long tt = step - sd.start;
                if (tt < 0 || tt >= sd.len) continue;
                const int lx = sd.local % BX, ly = (sd.local / BX) % BY, lz = sd.local / (BX * BY);
                if (lz != z || ly != y || (lx >> 2) != x4) continue;
                const float smp = E.wave[sd.w_off + tt];
                add_comp(acc, lx & 3, ST == ST_F32 ? smp : __fmul_rn(smp, isc));
            }
        }
        if constexpr (ST != ST_F32) {
            q.x = __fadd_rn(p.x, vq.x);
            q.y = __fadd_rn(p.y, vq.y);
            q.z = __fadd_rn(p.z, vq.z);
            q.w = __fadd_rn(p.w, vq.w);
        }
        if (decay) {
            q.x = __fmul_rn(alpha, q.x);
            q.y = __fmul_rn(alpha, q.y);
            q.z = __fmul_rn(alpha, q.z);
            q.w = __fmul_rn(alpha, q.w);
            if constexpr (ST != ST_F32) {
                vq.x = __fsub_rn(q.x, p.x);
                vq.y = __fsub_rn(q.y, p.y);
                vq.z = __fsub_rn(q.z, p.z);
                vq.w = __fsub_rn(q.w, p.w);
            }
        }
        if (ragged) {
            const bool rowin = gy < ny && gz0 + z < nz;
            if (!rowin || gx0 + 0 >= nx) q.x = 0.f;
            if (!rowin || gx0 + 1 >= nx) q.y = 0.f;
            if (!rowin || gx0 + 2 >= nx) q.z = 0.f;
            if (!rowin || gx0 + 3 >= nx) q.w = 0.f;
            if constexpr (ST != ST_F32) {
                if (!rowin || gx0 + 0 >= nx) vq.x = 0.f;
                if (!rowin || gx0 + 1 >= nx) vq.y = 0.f;
                if (!rowin || gx0 + 2 >= nx) vq.z = 0.f;
                if (!rowin || gx0 + 3 >= nx) vq.w = 0.f;
            }
        }
        // phi^{n+1} is what the storage holds: maxima and thresholds see the
        // stored (rounded) value.
        typename F::V qs;
        q = F::rnd(q, U1, U1, qs);
        if (valid) F::st(out + 4 * (z * TPB + t), qs);
        if constexpr (ST != ST_F32) {
            typename F::V vs;
            F::rnd(vq, U1, U1, vs);
            if (valid) F::st(vout + 4 * (z * TPB + t), vs);
        }
        // per lane: the column maximum (qm) and the maxima of its x = 4 x4 and
        // x = 4 x4 + 3 nodes (f0, f1) over the planes; the y faces are the
        // column maxima of the y-edge lanes, so they are taken after the loop
        if constexpr (ST == ST_F32) {
            const float mq = max4abs(q);
            qm = fmaxf(qm, mq);
            mc = fmaxf(mc, fmaxf(mq, max4abs(p)));
            if (z == 0) f4 = mq;
            if (z == BZ - 1) f5 = mq;
            f0 = fmaxf(f0, fabsf(q.x));
            f1 = fmaxf(f1, fabsf(q.w));
        } else {
            // 16-bit: the maxima of |phi^{n+1}| straight from the stored
            // bits, per 16-bit half (exact: the conversion is monotone)
            const unsigned a0 = qs.x & 0x7fff7fffu, a1 = qs.y & 0x7fff7fffu;
            const unsigned m2 = hmax2u<ST>(a0, a1);
            qm2 = hmax2u<ST>(qm2, m2);
            mc = fmaxf(mc, max4abs(p));
            if (z == 0) f42 = m2;
            if (z == BZ - 1) f52 = m2;
            f02 = hmax2u<ST>(f02, a0);   // low half: |phi| at x = 4 x4
            f12 = hmax2u<ST>(f12, a1);   // high half: at x = 4 x4 + 3
        }
    }
    if constexpr (ST != ST_F32) {
        qm = max2h<ST>(qm2);
        mc = __fmul_rn(fmaxf(mc, qm), sc);
        qm = __fmul_rn(qm, sc);
        f0 = __fmul_rn(half_lo<ST>(f02), sc);
        f1 = __fmul_rn(half_hi<ST>(f12), sc);
        f4 = __fmul_rn(max2h<ST>(f42), sc);
        f5 = __fmul_rn(max2h<ST>(f52), sc);
    }
    f2 = y == 0 ? qm : 0.f;
    f3 = y == BY - 1 ? qm : 0.f;
    f0 = x4 == 0 ? f0 : 0.f;
    f1 = x4 == XQ - 1 ? f1 : 0.f;
    mc = seg_max(mc);
    qm = seg_max(qm);
    f0 = seg_max(f0);
    f1 = seg_max(f1);
    f2 = seg_max(f2);
    f3 = seg_max(f3);
    f4 = seg_max(f4);
    f5 = seg_max(f5);
    if (valid && t == 0) {
        // rec[7]: the launch that wrote the record (a box claimed during an
        // update still holds its previous owner's record, from an older launch)
        float4 *r = reinterpret_cast<float4 *>(E.rec + (size_t)w.slot * 8);
        __stcg(r, make_float4(f0, f1, f2, f3));
        __stcg(r + 1, make_float4(f4, f5, mc, __uint_as_float(stamp)));
        // running domain maximum of this lane's sim, flushed when the sim
        // (or its step parity) changes
        if (sim != gsim || nh != gnh) {
            flush_gmax(E, gacc, gsim, gnh);
            flush_updates(E, scells, gsim);
            gsim = sim;
            gnh = nh;
            gacc = 0.f;
        }
        gacc = fmaxf(gacc, qm);
        const int ex = min(BX, nx - cx * BX), ey = min(BY, ny - cy * BY), ez = min(BZ, nz - cz * BZ);
        cells += (unsigned long long)(ex * ey * ez);
        scells += (unsigned long long)(ex * ey * ez);
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

// A source of this sim feeds brick b at some step of [n0, n1].
__device__ __forceinline__ bool forced_in(const Engine &E, const SimDev *S, int b, long long n0, long long n1)
{
    for (int s = S->src_begin; s < S->src_end; ++s) {
        const SrcDev &sd = E.src[s];
        if (sd.brick == b && n1 >= sd.start && n0 < sd.start + sd.len) return true;
    }
    return false;
}

// Warp-aggregated counter update: the converged lanes calling this together
// take consecutive values with one atomic; returns this lane's old value.
__device__ __forceinline__ int agg_add(int *ctr, int sign)
{
    cg::coalesced_group g = cg::coalesced_threads();
    int base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(ctr, sign * (int)g.size());
    base = g.shfl(base, 0);
    return base + sign * (int)g.thread_rank();
}

// Warp-aggregated reservation of n consecutive counter values per lane
// (lanes may ask for different n); returns this lane's first value.
__device__ __forceinline__ int agg_add_n(int *ctr, int n)
{
    cg::coalesced_group g = cg::coalesced_threads();
    const int incl = cg::inclusive_scan(g, n);
    int base = 0;
    if (g.thread_rank() == g.size() - 1) base = atomicAdd(ctr, incl);
    base = g.shfl(base, g.size() - 1);
    return base + incl - n;
}

// Trigger up to N bricks of one sim (update procedure step 8, Fig. 1): claim
// each with a CAS on Cell2box (-1 -> -2; another thread may be boxing it),
// pop one vacant box per claim won, then publish.  All a new box's record
// needs (the vacant box, coefficients, has-source bit from the shut-down
// word) loads in one round after the reservation, so a won claim costs three
// rounds of dependent accesses: the CAS, the reservation, those loads.  The
// shut-down word of an unboxed brick is written only by the thread that wins
// its claim.  Only claims that got a box take an entry of newslots (at most
// one per box on the free stack, so never more than n_slots in a step); a
// claim that finds the stack empty is undone and flags ERR_NOMEM.
template <int N>
__device__ void claim_bricks(const Engine &E, int sim, SimDev *S, const int *b_local, int n)
{
    static_assert(N <= 32, "one bit per candidate");
    const long long bb = S->brick_base;
    const int step = (int)__ldcg(&S->step);
    unsigned won = 0;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i < n && TCM_BRICK_OK(E, bb + b_local[i]) && atomicCAS(E.slot_of_brick + bb + b_local[i], -1, -2) == -1)
            won |= 1u << i;
    if (won == 0) return;
    const int nw = __popc(won);
    // vacant boxes free_stack[top - nw .. top - 1]; the first nv claims get one
    const int top = atomicSub(&E.st->free_top, nw);
    const int nv = min(max(top, 0), nw);
    const int nn = agg_add_n(&E.st->n_new, nv);
    int k = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (!(won >> i & 1u)) continue;
        const long long g = bb + b_local[i];
        if (k >= nv) {   // no vacant box left: undo the claim
            atomicExch(E.slot_of_brick + g, -1);
            atomicOr(&E.st->err, ERR_NOMEM);
            atomicOr(&S->poisoned, 1u);
            ++k;
            continue;
        }
        const int kslab = __ldg(E.kslab_of_brick + g);
        const float kscal = __ldg(E.kscal + g);
        const unsigned short sdw = __ldcg(E.sd_of_brick + g);
        const int ns = TCM_SLOT_OK(E, top - 1 - k) ? __ldcg(E.free_stack + (top - 1 - k)) : -1;
        if (!TCM_SLOT_OK(E, ns) || !TCM_SLOT_OK(E, nn + k)) {   // checked build: give the claim up
            atomicExch(E.slot_of_brick + g, -1);
            ++k;
            continue;
        }
        E.claim_step[ns] = step;
        SlotMeta m;
        m.brick = b_local[i];
        m.kslab = kslab;
        m.kscal = kscal;
        m.flags = ((unsigned)sim << 16) | (sdw & FLAG_HAS_SRC);
        store_meta(E.meta + ns, m);
        E.sd_of_brick[g] = (unsigned short)(sdw & FLAG_HAS_SRC);   // not shutting down
        atomicOr(E.bitmap + (g >> 5), 1u << (unsigned)(g & 31));
        atomicAdd(E.blocktot + (int)((g >> 5) / E.words_per_block), 1);
        E.newslots[nn + k] = ns;
        atomicExch(E.slot_of_brick + g, ns);
        ++k;
    }
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

// Block sums of two values at once (one pair of barriers).
__device__ void block_sum2(long long &a, long long &b)
{
    __shared__ long long s_a[BLOCK / 32], s_b[BLOCK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(FULL, a, o);
        b += __shfl_xor_sync(FULL, b, o);
    }
    if (lane == 0) {
        s_a[wid] = a;
        s_b[wid] = b;
    }
    __syncthreads();
    long long ra = 0, rb = 0;
#pragma unroll
    for (int i = 0; i < BLOCK / 32; ++i) {
        ra += s_a[i];
        rb += s_b[i];
    }
    __syncthreads();
    a = ra;
    b = rb;
}

// Per-thread copy of one sim's geometry for building work items.
struct ItemSim {
    int sim = -1;
    int mx = 1, my = 1, mz = 0;
    long long bb = 0, step = 0;
    unsigned long long kslabs = 0;
};

__device__ __forceinline__ void item_sim(const Engine &E, int si, ItemSim &c)
{
    if (si == c.sim) return;
    const SimDev *S = E.sims + si;
    c.sim = si;
    c.step = __ldcg(&S->step);
    c.mx = max(__ldg(&S->mx), 1);
    c.my = max(__ldg(&S->my), 1);
    c.mz = __ldg(&S->mz);
    c.bb = __ldg(&S->brick_base);
    c.kslabs = __ldg(reinterpret_cast<const unsigned long long *>(&S->kslabs));
}

// Brick g's local id b, its box and the boxes of its six face neighbours,
// addressed with the geometry of sim q.  Every address stays inside q's
// bricks even when g belongs to another sim (the caller then redoes it).
__device__ __forceinline__ void item_geom(const Engine &E, long long g, const ItemSim &q, int &b, int &slot,
                                          int (&nb)[6])
{
    b = (int)(g - q.bb);
    const int cx = b % q.mx, cy = (b / q.mx) % q.my, cz = b / (q.mx * q.my);
    // a brick outside its sim's grid (never listed) gets no box
    slot = (b >= 0 && cz < q.mz && TCM_BRICK_OK(E, g)) ? __ldcg(E.slot_of_brick + g) : -1;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const int ax = cx + (f == 0 ? -1 : (f == 1 ? 1 : 0));
        const int ay = cy + (f == 2 ? -1 : (f == 3 ? 1 : 0));
        const int az = cz + (f == 4 ? -1 : (f == 5 ? 1 : 0));
        nb[f] = (ax >= 0 && ay >= 0 && az >= 0 && ax < q.mx && ay < q.my && az < q.mz)
                    ? __ldcg(E.slot_of_brick + q.bb + ((long long)az * q.my + ay) * q.mx + ax)
                    : -3;
    }
}

// Work items of up to IB bricks g[0..n) (global ids) at once.  An item
// holds the brick's box, the boxes of its six face neighbours, its
// coefficient address (or scalar k), its sim and shut-down word, and the
// half that holds phi^n when the next launch steps it.  All loads of all
// the items are issued together: the neighbour boxes are addressed with the
// geometry of the sim cached in c (a block's sims change rarely), and an
// item whose sim turns out to be another is redone with its own.
constexpr int IB = 4;

__device__ __forceinline__ void build_items(const Engine &E, const long long (&g)[IB], int n, WorkItem *const (&out)[IB],
                                            int step_ahead, ItemSim &c)
{
    int si[IB], b[IB], slot[IB], kslab[IB], nb[IB][6];
    float kscal[IB];
    unsigned sd[IB];
    const ItemSim c0 = c;
#pragma unroll
    for (int k = 0; k < IB; ++k) {
        if (k >= n) continue;
        si[k] = (int)__ldg(E.sim_of_word + (g[k] >> 5));
        kslab[k] = __ldg(E.kslab_of_brick + g[k]);
        kscal[k] = __ldg(E.kscal + g[k]);
        sd[k] = __ldcg(E.sd_of_brick + g[k]);
        item_geom(E, g[k], c0, b[k], slot[k], nb[k]);
    }
    ItemSim ck[IB];
#pragma unroll
    for (int k = 0; k < IB; ++k) {
        if (k >= n) continue;
        ck[k] = c0;
        if (si[k] != c0.sim) {
            item_sim(E, si[k], c);
            ck[k] = c;
            item_geom(E, g[k], c, b[k], slot[k], nb[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < IB; ++k) {
        if (k >= n) continue;
        const ItemSim &q = ck[k];
        const unsigned long long kp = kslab[k] >= 0 ? q.kslabs + (size_t)kslab[k] * BVOL * sizeof(float)
                                                     : (KP_SCALAR | __float_as_uint(kscal[k]));
        const unsigned flags = ((unsigned)si[k] << 16) | sd[k];   // sd word carries the has-source bit
        // The item is processed by the next launch, which steps from phi^{n+1}.
        const int nh = (int)((q.step + step_ahead) & 1);
        int4 *p = reinterpret_cast<int4 *>(out[k]);
        p[0] = make_int4(slot[k], b[k], (int)(unsigned)kp, (int)(unsigned)(kp >> 32));
        p[1] = make_int4((int)flags, nb[k][0], nb[k][1], nb[k][2]);
        p[2] = make_int4(nb[k][3], nb[k][4], nb[k][5], nh);
    }
}

// Rebuild the active list from the bitmap in brick order.  Each block owns
// a range of bitmap words; its offset in the list is the sum of the
// per-range counts (blocktot, kept by the update procedure) of the blocks
// before it.  The brick ids of the range (popc + block scan) go to shared
// memory when they fit, else to the global listids, and the block then
// builds the items from there, IB per thread at a time.  The loads that
// depend on nothing (the range's first words, the counts, the range's first
// sim) are issued before the caller's own work, mid(), runs.
constexpr int SMEM_IDS = 4096;

template <class Mid>
__device__ void compact_list(const Engine &E, WorkItem *Lout, int *n_out, int step_ahead, Mid &&mid)
{
    __shared__ int s_ids[SMEM_IDS];
    const int G = (int)gridDim.x;
    const long long w0 = (long long)blockIdx.x * E.words_per_block;
    const long long w1 = min(w0 + E.words_per_block, E.n_words);
    const long long wf = w0 + threadIdx.x;
    const unsigned bits0 = wf < w1 ? __ldcg(E.bitmap + wf) : 0u;
    const int v0 = (int)threadIdx.x < G ? __ldcg(E.blocktot + threadIdx.x) : 0;
    const int mine = __ldcg(E.blocktot + blockIdx.x);
    const int s0 = w0 < w1 ? (int)__ldg(E.sim_of_word + w0) : -1;
    mid();
    ItemSim c;
    if (s0 >= 0) item_sim(E, s0, c);
    long long before = (int)threadIdx.x < (int)blockIdx.x ? v0 : 0, all = v0;
    for (int j = threadIdx.x + BLOCK; j < G; j += BLOCK) {
        const int v = __ldcg(E.blocktot + j);
        all += v;
        if (j < (int)blockIdx.x) before += v;
    }
    block_sum2(before, all);
    const bool local = mine <= SMEM_IDS;
    int *ids = local ? s_ids : E.listids + before;
    const int cap = local ? SMEM_IDS : (int)max(0ll, (long long)E.n_slots - before);
    int off = 0;
    for (long long wb = w0; wb < w1; wb += BLOCK) {
        const long long w = wb + threadIdx.x;
        unsigned bits = wb == w0 ? bits0 : (w < w1 ? __ldcg(E.bitmap + w) : 0u);
        int total;
        int pos = off + block_excl_scan(__popc(bits), &total);
        while (bits) {
            const int bit = __ffs(bits) - 1;
            bits &= bits - 1;
            if (pos < cap) ids[pos] = (int)(w * 32 + bit);
            ++pos;
        }
        off += total;
    }
    __syncthreads();
    const int n = min(off, cap);
    const int end = (int)min((long long)n, (long long)E.n_slots - before);
    for (int i = threadIdx.x; i < end; i += IB * BLOCK) {
        long long g[IB];
        WorkItem *o[IB];
        int m = 0;
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            const int ik = i + k * BLOCK;
            g[k] = ik < end ? (long long)ids[ik] : 0;
            o[k] = Lout + before + ik;
            m += ik < end ? 1 : 0;
        }
        build_items(E, g, m, o, step_ahead, c);
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *n_out = (int)all;
}

// Per-thread copy of one sim's step state (step counter, level): every
// item of the same sim reuses it instead of re-reading one shared address.
struct SimCache {
    int sim = -1;
    bool dense = false;
    bool manage = false;   // this sim runs the update procedure after this step
    bool lpf = false;
    int interval = 1;
    int neighbours = 6;
    long long step = 0;
    double thr = 0.0;
    // The level rounded down to binary32: for a binary32 value v,
    // (double)v > thr exactly when v > thr_f (no binary32 lies between them),
    // so the decisions stay in FP32 (the FP64 pipe is slow here).
    float thr_f = 0.f;
};

// nh: the half holding phi^n this step (= step parity), known from the item,
// so the domain maximum loads alongside the step counter.
__device__ __forceinline__ void sim_cache(const Engine &E, int sim, int nh, SimCache &c)
{
    if (sim == c.sim) return;
    const SimDev *S = E.sims + sim;
    c.sim = sim;
    c.dense = __ldg(&S->dense) != 0;
    c.step = __ldcg(&S->step);
    c.interval = __ldg(&S->interval);
    c.neighbours = __ldg(&S->neighbours);
    c.manage = (c.step + 1) % c.interval == 0;
    c.lpf = __ldg(&S->lpf) != 0;
    const double G = (double)__uint_as_float(__ldcg(&S->gmax[nh]));
    c.thr = __ldg(&S->thr_mode) == 1 ? __ldg(&S->tau) * G : __ldg(&S->tau);
    c.thr_f = __double2float_rd(c.thr);
}

// Record the shut-down count of a kept brick, or release its box.
__device__ __forceinline__ void keep_or_release(const Engine &E, const WorkItem &w, bool keep, unsigned sd,
                                                unsigned sd0, long long g, int slot)
{
    if (keep) {
        if (sd != sd0) E.sd_of_brick[g] = (unsigned short)((w.flags & FLAG_HAS_SRC) | sd);
    } else {
        if (!TCM_BRICK_OK(E, g)) return;
        if (sd0 != 0) E.sd_of_brick[g] = (unsigned short)(w.flags & FLAG_HAS_SRC);
        atomicExch(E.slot_of_brick + g, -1);
        atomicAnd(E.bitmap + (g >> 5), ~(1u << (unsigned)(g & 31)));
        atomicSub(E.blocktot + (int)((g >> 5) / E.words_per_block), 1);
        const int r = agg_add(&E.st->n_retired, 1);
        if (TCM_SLOT_OK(E, r)) E.retired[r] = slot;
    }
}

// The update procedure with the 26-neighbour set (steps 4-5, Fig. 3): a
// brick is triggered when its own maximum is above the level or a source
// feeds it during the steps the update covers; it stays when it or any of
// its 26 neighbours is triggered; a triggered brick boxes all 26 neighbours.
__device__ __noinline__ void p2_item26(const Engine &E, const WorkItem &w, bool above, bool nonzero, float thr,
                                       int interval, bool lpf, int sim, SimDev *S, unsigned stamp)
{
    const int b = w.brick;
    const int mx = __ldg(&S->mx), my = __ldg(&S->my), mz = __ldg(&S->mz);
    const int cx = b % mx, cy = (b / mx) % my, cz = b / (mx * my);
    const long long g0 = __ldg(&S->brick_base);
    const long long step = __ldcg(&S->step);
    const bool forced = (w.flags & FLAG_HAS_SRC) && forced_in(E, S, b, step + 1, step + interval);
    int nslot[26];
    int nid[26];
    int k = 0;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy && !dz) continue;
                const int ax = cx + dx, ay = cy + dy, az = cz + dz;
                const bool in = ax >= 0 && ay >= 0 && az >= 0 && ax < mx && ay < my && az < mz;
                nid[k] = in ? (az * my + ay) * mx + ax : -1;
                nslot[k] = in ? __ldcg(E.slot_of_brick + g0 + nid[k]) : -3;
                ++k;
            }
    bool hot = above || forced;
    if (!hot) {
        // a neighbour a source feeds during the steps this update covers
        const long long n0 = step + 1, n1 = n0 + interval - 1;
        for (int s = S->src_begin; s < S->src_end && !hot; ++s) {
            const SrcDev &sd = E.src[s];
            const int sx = sd.brick % mx, sy = (sd.brick / mx) % my, sz = sd.brick / (mx * my);
            if (abs(sx - cx) <= 1 && abs(sy - cy) <= 1 && abs(sz - cz) <= 1 && n1 >= sd.start &&
                n0 < sd.start + sd.len)
                hot = true;
        }
    }
    if (!hot) {
        // neighbours stepped in this launch: a neighbour claimed during this
        // update by another thread reads as boxed here, but its box still
        // holds its previous owner's record, stamped with an older launch
        float2 nm[26];
#pragma unroll
        for (int i = 0; i < 26; ++i)
            nm[i] = (nslot[i] >= 0 && TCM_SLOT_OK(E, nslot[i]))
                        ? __ldcg(reinterpret_cast<const float2 *>(E.rec + (size_t)nslot[i] * 8 + 6))
                        : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 26; ++i)
            if (nslot[i] >= 0 && __float_as_uint(nm[i].y) == stamp && nm[i].x > thr) hot = true;
    }
    unsigned sd = w.flags & SD_MASK;
    const unsigned sd0 = sd;
    bool keep;
    if (hot) {
        sd = 0;
        keep = true;
    } else if (lpf) {
        keep = false;
        if (nonzero) E.lpf_q[agg_add(&E.st->n_lpf_q, 1)] = g0 + b;
    } else if (sd > 0) {
        sd = sd > (unsigned)interval ? sd - (unsigned)interval : 0u;
        keep = sd > 0;
    } else if (__ldg(&S->decay_steps) > 0) {
        sd = (unsigned)__ldg(&S->decay_steps);
        keep = true;
    } else {
        keep = false;
    }
    keep_or_release(E, w, keep, sd, sd0, g0 + w.brick, w.slot);
    if (above || forced) {
        int nbs[26];
        int n = 0;
#pragma unroll
        for (int i = 0; i < 26; ++i)
            if (nslot[i] == -1) nbs[n++] = nid[i];
        if (n > 0) claim_bricks<26>(E, sim, S, nbs, n);
    }
}

// The update of one brick in general (6-neighbour set): `thr` its sim's
// level, `step`, `interval`, `lpf` its sim's schedule.  Out of line, so the
// unrolled call sites of the caller stay small.
__device__ __noinline__ void p2_item_general(const Engine &E, const WorkItem w, const float4 r0, const float4 r1,
                                             float thr, long long step, int interval, bool lpf)
{
    const int slot = w.slot;
    const int sim = (int)(w.flags >> 16);
    SimDev *S = E.sims + sim;
    const int b = w.brick;
    const float fc[6] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y};
    bool hot = r1.z > thr;
    if (!hot) {
        // the touching faces of the boxed neighbours (loads in parallel)
        float nf[6];
#pragma unroll
        for (int f = 0; f < 6; ++f)
            nf[f] = (w.nb[f] >= 0 && TCM_SLOT_OK(E, w.nb[f])) ? __ldcg(E.rec + (size_t)w.nb[f] * 8 + (f ^ 1)) : 0.f;
#pragma unroll
        for (int f = 0; f < 6; ++f)
            if (w.nb[f] >= 0 && nf[f] > thr) hot = true;
    }
    // a source feeds it during the steps this update covers
    if (!hot && (w.flags & FLAG_HAS_SRC) && forced_in(E, S, b, step + 1, step + interval)) hot = true;
    unsigned sd = w.flags & SD_MASK;
    const unsigned sd0 = sd;
    bool keep;
    if (hot) {
        sd = 0;
        keep = true;
    } else if (lpf) {
        keep = false;   // Eq. 7: released now, its neighbours filtered after the launch
        if (r1.z > 0.f) E.lpf_q[agg_add(&E.st->n_lpf_q, 1)] = __ldg(&S->brick_base) + b;
    } else if (sd > 0) {
        // the count is in time steps; `interval` of them passed
        sd = sd > (unsigned)interval ? sd - (unsigned)interval : 0u;
        keep = sd > 0;
    } else if (__ldg(&S->decay_steps) > 0) {
        sd = (unsigned)__ldg(&S->decay_steps);
        keep = true;
    } else {
        keep = false;
    }
    keep_or_release(E, w, keep, sd, sd0, __ldg(&S->brick_base) + b, slot);
    const int mx = __ldg(&S->mx), my = __ldg(&S->my);
    const int cx = b % mx, cy = (b / mx) % my, cz = b / (mx * my);
    int nbs[6];
    int n = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        if (w.nb[f] == -1 && fc[f] > thr) {
            const int ax = cx + (f == 0 ? -1 : (f == 1 ? 1 : 0));
            const int ay = cy + (f == 2 ? -1 : (f == 3 ? 1 : 0));
            const int az = cz + (f == 4 ? -1 : (f == 5 ? 1 : 0));
            nbs[n++] = (az * my + ay) * mx + ax;
        }
    }
    if (n > 0) claim_bricks<6>(E, sim, S, nbs, n);
}

// The update procedure (Simulation section, Fig. 3a) for one active brick (item w, its own maxima
// r0/r1): keep / shut down / release it, and trigger its neighbours across
// faces above the level (Fig. 3a).  Most bricks are above the level, not
// shutting down and have no face above it towards an unboxed neighbour:
// for them the update changes nothing, which is decided here without a
// memory access; the rest take the general path.
__device__ __forceinline__ void p2_item(const Engine &E, const WorkItem &w, const float4 &r0, const float4 &r1,
                                        int age_flip, unsigned stamp, SimCache &c)
{
    const int sim = (int)(w.flags >> 16);
    sim_cache(E, sim, w.nh ^ age_flip, c);
    if (c.dense || !c.manage) return;
    const float thr = c.thr_f;   // see SimCache
    if (c.neighbours == 26) {
        p2_item26(E, w, r1.z > thr, r1.z > 0.f, thr, c.interval, c.lpf, sim, E.sims + sim, stamp);
        return;
    }
    if (r1.z > thr && (w.flags & SD_MASK) == 0) {
        const float fc[6] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y};
        bool edge = false;
#pragma unroll
        for (int f = 0; f < 6; ++f) edge = edge || (w.nb[f] == -1 && fc[f] > thr);
        if (!edge) return;
    }
    p2_item_general(E, w, r0, r1, thr, c.step, c.interval, c.lpf);
}

// ---------------------------------------------------------------------------
// The step kernel.
// ---------------------------------------------------------------------------
// True in every thread of the last block to get here (block-uniform); the
// other blocks' writes before their arrival are visible to it.
__device__ bool last_block(EngineState *st)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const bool last = atomicAdd(&st->p3_done, 1u) == gridDim.x - 1;
        if (last) __threadfence();
        s_last = last;
    }
    __syncthreads();
    return s_last != 0;
}

// Advance every live sim's step (after all blocks have read it this launch);
// called by every thread of one block.
__device__ void advance_steps(const Engine &E)
{
    for (int s = threadIdx.x; s < E.n_sims; s += BLOCK) {
        SimDev *S = E.sims + s;
        if (!__ldcg(&S->live)) continue;
        const long long n = __ldcg(&S->step);
        S->gmax[(n + 1) & 1] = 0u;
        S->step = n + 1;
    }
}

// Ask L2 for the field arrays and per-node k of the brick this lane's
// segment steps next, one 128-byte line per lane and array, so that the
// stepping's loads of them find L2 instead of HBM; no registers or shared
// memory stay held.  Only bricks with per-node k (three arrays to read) are
// prefetched: measured, the prefetch pays for those and costs time on
// bricks with a scalar k.
template <int ST, bool MIX = false>
__device__ __forceinline__ void prefetch_brick(const Engine &E, const WorkItem &w, bool v, int t, int age_flip)
{
    if (!v || (w.kp & KP_SCALAR)) return;
    const int nh = w.nh ^ age_flip;
    constexpr int LINE = 128;
    constexpr int HB = BVOL * (int)sizeof(typename Fld<ST>::T);
    const char *a = reinterpret_cast<const char *>(half_ptr<ST, MIX>(E, w.slot, nh));
    const char *b = reinterpret_cast<const char *>(half_ptr<ST, MIX>(E, w.slot, ST == ST_F32 ? (nh ^ 1) : V_HALF));
    for (int o = t * LINE; o < HB; o += TPB * LINE) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a + o) : "memory");
        asm volatile("prefetch.global.L2 [%0];" ::"l"(b + o) : "memory");
    }
    const char *k = reinterpret_cast<const char *>(w.kp);
    for (int o = t * LINE; o < BVOL * (int)sizeof(float); o += TPB * LINE)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(k + o) : "memory");
}

// One pair of bricks of a warp (bricks 2j and 2j+1; one brick per warp for
// 16-wide bricks): when the second is the x+ neighbour of the first, their
// touching columns are exchanged instead of loaded.
template <int ST, bool MIX>
__device__ __forceinline__ void p1_pair(const Engine &E, const WorkItem &w, bool v, int t, int seg, int age_flip,
                                        unsigned stamp, unsigned long long &cells, unsigned long long &scells,
                                        float &gacc, int &gsim, int &gnh)
{
    bool pair_x = false;
    const bool first = (seg & 1) == 0;
    if constexpr (BRICKS_PER_WARP >= 2) {
        const int other_slot = __shfl_xor_sync(FULL, w.slot, TPB);
        const bool other_v = __shfl_xor_sync(FULL, (int)v, TPB) != 0;
        pair_x = v && other_v &&
                 (first ? (w.nb[1] >= 0 && w.nb[1] == other_slot) : (w.nb[0] >= 0 && w.nb[0] == other_slot));
    }
    p1_brick<ST, MIX>(E, w, v, t, seg, !first && pair_x, first && pair_x, age_flip, stamp, cells, scells, gacc,
                      gsim, gnh);
}

template <int ST>
__global__ void __launch_bounds__(BLOCK, 1) k_step(Engine E, int cur, int manage)
{
    EngineState *st = E.st;
    const int age_flip = __ldcg(&st->list_age) & 1;
    const unsigned stamp = (unsigned)__ldcg(&st->launches);   // this launch, in the maxima records
    const WorkItem *L = cur ? E.items1 : E.items0;
    WorkItem *Lnext = cur ? E.items0 : E.items1;
    const int nact = __ldcg(&st->n_active[cur]);
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * BLOCK) >> 5;

    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->t_start = globaltimer();
        // Boxes released last step were pushed above max(free_top, 0).
        const int ft = max(__ldcg(&st->free_top), 0) + __ldcg(&st->n_retired);
        st->free_top = ft;
        st->n_retired = 0;
        st->n_new = 0;
        st->n_lpf_q = 0;
        st->n_lpf_aff = 0;
    }

    // ---- P1: time stepping of every active brick -------------------------
    {
        unsigned long long cells = 0, scells = 0;
        float gacc = 0.f;
        int gsim = -1;
        int gnh = 0;
        const int seg = lane / TPB;
        const int t = lane % TPB;
        const int npairs = (nact + BRICKS_PER_WARP - 1) / BRICKS_PER_WARP;
        int pr = gwarp;
        int i = pr * BRICKS_PER_WARP + seg;
        bool v = pr < npairs && i < nact;
        WorkItem w = load_item(L, v ? i : 0);
        v = v && w.slot >= 0;
        int pn = pr + nwarps;
        int in = pn * BRICKS_PER_WARP + seg;
        bool vn = pn < npairs && in < nact;
        WorkItem wn = load_item(L, vn ? in : 0);
        vn = vn && wn.slot >= 0;
        while (pr < npairs) {
            // the item two pairs ahead, loaded while this pair is stepped;
            // the next pair's arrays fetched into L2 meanwhile
            const int pnn = pn + nwarps;
            const int inn = pnn * BRICKS_PER_WARP + seg;
            bool vnn = pnn < npairs && inn < nact;
            const WorkItem wnn = load_item(L, vnn ? inn : 0);
            vnn = vnn && wnn.slot >= 0;
            if constexpr (ST != ST_MIXED) {
                if (E.prefetch) prefetch_brick<ST>(E, wn, vn, t, age_flip);
                p1_pair<ST, false>(E, w, v, t, seg, age_flip, stamp, cells, scells, gacc, gsim, gnh);
            } else {
                // Simulations of different storages in one launch: the warp
                // steps the bricks of each storage present among its lanes in
                // turn (every lane takes part in every call, so the shuffles
                // see full warps).
                if (E.prefetch && vn) {
                    const int sn = __ldg(&E.sims[wn.flags >> 16].storage);
                    if (sn == ST_F32) prefetch_brick<ST_F32, true>(E, wn, true, t, age_flip);
                    else if (sn == ST_BF16) prefetch_brick<ST_BF16, true>(E, wn, true, t, age_flip);
                    else prefetch_brick<ST_F16, true>(E, wn, true, t, age_flip);
                }
                const int sw = v ? __ldg(&E.sims[w.flags >> 16].storage) : -1;
                if (__any_sync(FULL, sw == ST_F32))
                    p1_pair<ST_F32, true>(E, w, v && sw == ST_F32, t, seg, age_flip, stamp, cells, scells, gacc, gsim,
                                          gnh);
                if (__any_sync(FULL, sw == ST_BF16))
                    p1_pair<ST_BF16, true>(E, w, v && sw == ST_BF16, t, seg, age_flip, stamp, cells, scells, gacc,
                                           gsim, gnh);
                if (__any_sync(FULL, sw == ST_F16))
                    p1_pair<ST_F16, true>(E, w, v && sw == ST_F16, t, seg, age_flip, stamp, cells, scells, gacc,
                                          gsim, gnh);
            }
            pr = pn;
            w = wn;
            v = vn;
            pn = pnn;
            wn = wnn;
            vn = vnn;
        }
        flush_gmax(E, gacc, gsim, gnh);
        flush_updates(E, scells, gsim);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cells += __shfl_xor_sync(FULL, cells, o);
        if (lane == 0 && cells) atomicAdd(&st->updates, cells);
    }
    if (!manage) {
        // Time stepping only: the last block to finish advances the step and
        // the age of the (kept) active list.
        if (last_block(st)) {
            advance_steps(E);
            if (threadIdx.x == 0) {
                st->list_age += 1;
                st->launches += 1;
                st->p3_done = 0u;
                st->phase_ns[0] += globaltimer() - __ldcg(&st->t_start);
            }
        }
        return;
    }
    if (!grid_barrier(st, &st->bar_count)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->t_p1 = globaltimer();

    // ---- P2: the update procedure ---------------------------------------
    {
        const int gtid = blockIdx.x * BLOCK + threadIdx.x;
        const int nthr = gridDim.x * BLOCK;
        // Two items per thread at a time, so their loads overlap (measured
        // over the 512^3 run on one GPU: 1, 2, 3, 4, 5, 6 items took 14.5,
        // 14.0, 14.2, 14.4-14.6, 15.1, 15.5 ms for FP32; a thread's items
        // that take the general path run one after another).
        constexpr int U = 2;
        SimCache sc;
        for (int base = gtid; base < nact; base += U * nthr) {
            WorkItem w[U];
            float4 r0[U], r1[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = base + u * nthr;
                w[u] = load_item(L, i < nact ? i : 0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float4 *r = reinterpret_cast<const float4 *>(E.rec + (size_t)max(w[u].slot, 0) * 8);
                r0[u] = __ldcg(r);
                r1[u] = __ldcg(r + 1);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (base + u * nthr < nact && w[u].slot >= 0 && TCM_SLOT_OK(E, w[u].slot))
                    p2_item(E, w[u], r0[u], r1[u], age_flip, stamp, sc);
        }
        // (Source bricks need no activation here: every source starts at its
        // sim's first step, its brick is boxed when the sim starts, and the
        // update keeps it while samples remain.)
    }
    if (!grid_barrier(st, &st->bar_count)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->t_p2 = globaltimer();

    // ---- P3: box recycling and compaction of the active list -------------
    {
        const int gtid = blockIdx.x * BLOCK + threadIdx.x;
        const int nthr = gridDim.x * BLOCK;
        const int n_new = min(__ldcg(&st->n_new), E.n_slots);
        const int n_ret = __ldcg(&st->n_retired);
        const int base = max(__ldcg(&st->free_top), 0);
        compact_list(E, Lnext, &st->n_active[cur ^ 1], 1, [&] {
            // the boxes claimed by this update zeroed, the released ones
            // pushed on the free stack (the first loads of both together)
            const bool r = gtid < n_ret && TCM_SLOT_OK(E, base + gtid) && TCM_SLOT_OK(E, gtid);
            const int r0 = r ? __ldcg(E.retired + gtid) : 0;
            int ns = gwarp < n_new ? __ldcg(E.newslots + gwarp) : -1;
            for (int i = gwarp; i < n_new; i += nwarps) {
                if (TCM_SLOT_OK(E, ns)) zero_box(E, ns, lane);
                ns = i + nwarps < n_new ? __ldcg(E.newslots + i + nwarps) : -1;
            }
            if (r) E.free_stack[base + gtid] = r0;
            for (int i = gtid + nthr; i < n_ret; i += nthr)
                if (TCM_SLOT_OK(E, base + i) && TCM_SLOT_OK(E, i)) E.free_stack[base + i] = __ldcg(E.retired + i);
        });
        // The last block to finish advances the step: every block has read
        // the step counters by then.
        if (last_block(st)) {
            advance_steps(E);
            if (threadIdx.x == 0) {
                st->list_parity = cur ^ 1;
                st->list_age = 0;
                st->launches += 1;
                st->p3_done = 0u;
                const unsigned long long t3 = globaltimer();
                const unsigned long long t0 = __ldcg(&st->t_start), t1 = __ldcg(&st->t_p1),
                                         t2 = __ldcg(&st->t_p2);
                st->phase_ns[0] += t1 - t0;
                st->phase_ns[1] += t2 - t1;
                st->phase_ns[2] += t3 - t2;
            }
        }
    }
}

// Build active list `parity` from the bitmap (start of a simulation).
__global__ void __launch_bounds__(BLOCK, 1) k_compact(Engine E, int parity)
{
    compact_list(E, parity ? E.items1 : E.items0, &E.st->n_active[parity], 0, [] {});
    if (blockIdx.x == 0 && threadIdx.x == 0) E.st->list_age = 0;
}

// ---------------------------------------------------------------------------
// Heterogenic Bulking (create time)
// ---------------------------------------------------------------------------
// Eq. 3 coefficient (c dt / dx)^2: the product and the quotient in FP64,
// squared, rounded to binary32.  dts = dt / dx when dx is a power of two and
// dt / dx is at least 2^-100 (0 otherwise): then (c dt) / dx is an exact
// scaling of c dt that stays in the normal range for every binary32 c, and it
// equals c (dt / dx) rounded once -- the same bits with one FP64 product
// instead of a product and a division (FP64 is slow on this part).
__device__ __forceinline__ float k_of_c(float c, double dt, double dx, double dts)
{
    const double r = dts != 0.0 ? (double)c * dts : (double)c * dt / dx;
    return (float)(r * r);
}

// dt / dx for k_of_c when that shortcut is exact, else 0.
double exact_ratio(double dt, double dx)
{
    int e = 0;
    const double m = std::frexp(dx, &e);   // dx = m 2^e, m in [0.5, 1)
    if (m != 0.5 || e <= -1000 || e >= 1000) return 0.0;
    const double r = dt * std::ldexp(1.0, 1 - e);   // exact: a power-of-two scaling
    return (std::isfinite(r) && r >= std::ldexp(1.0, -100)) ? r : 0.0;
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

// Classification, 32 bricks per warp at a time, one per lane: each lane
// takes its brick's corner k and, for rule-described media, decides from
// the rules alone whether no boundary crosses the brick (the common case
// needs no node: one lane's FP64 work per brick).  The warp then scans the
// nodes of every brick that is left undecided, one brick at a time, 32 nodes
// per round; the first round that finds a k different from the corner's
// decides.  A brick with more than one k gets the next per-node array id.
__global__ void k_bulk_classify(MediaDev M, int nx, int ny, int nz, int mx, int my, int mz, double dt,
                                double dx, double dts, long long bb, float *kscal, int *kslab_of_brick,
                                int *n_kslabs)
{
    const long long nb = (long long)mx * my * mz;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; g0 < nb; g0 += nw * 32) {
        const long long g = g0 + lane;
        const bool mine = g < nb;
        int x0 = 0, y0 = 0, z0 = 0, x1 = 0, y1 = 0, z1 = 0;
        float k0 = 0.f;
        bool uniform = false;
        if (mine) {
            const long long cx = g % mx, cy = (g / mx) % my, cz = g / ((long long)mx * my);
            x0 = (int)(cx * BX);
            y0 = (int)(cy * BY);
            z0 = (int)(cz * BZ);
            x1 = min(x0 + BX, nx) - 1;
            y1 = min(y0 + BY, ny) - 1;
            z1 = min(z0 + BZ, nz) - 1;
            k0 = k_of_c(media_c(M, nx, ny, x0, y0, z0), dt, dx, dts);
            uniform = M.kind == MEDIA_RULES && rules_uniform(M, x0, x1, y0, y1, z0, z1);
        }
        bool mydiff = false;
        unsigned todo = __ballot_sync(FULL, mine && !uniform);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int bx0 = __shfl_sync(FULL, x0, src), by0 = __shfl_sync(FULL, y0, src);
            const int bz0 = __shfl_sync(FULL, z0, src), bx1 = __shfl_sync(FULL, x1, src);
            const int by1 = __shfl_sync(FULL, y1, src), bz1 = __shfl_sync(FULL, z1, src);
            const unsigned kb = __float_as_uint(__shfl_sync(FULL, k0, src));
            bool diff = false;
            for (int e0 = 0; e0 < BVOL && !diff; e0 += 32) {
                const int e = e0 + lane;
                const int gx = bx0 + e % BX, gy = by0 + (e / BX) % BY, gz = bz0 + e / (BX * BY);
                bool d = false;
                if (e < BVOL && gx <= bx1 && gy <= by1 && gz <= bz1)
                    d = __float_as_uint(k_of_c(media_c(M, nx, ny, gx, gy, gz), dt, dx, dts)) != kb;
                diff = __any_sync(FULL, d);
            }
            if (lane == src) mydiff = diff;
        }
        if (mine) {
            if (mydiff) {
                kslab_of_brick[bb + g] = atomicAdd(n_kslabs, 1);
                kscal[bb + g] = 0.f;
            } else {
                kslab_of_brick[bb + g] = -1;
                kscal[bb + g] = k0;
            }
        }
    }
}

// Per-node k of every brick that has an array: each warp reads the array
// ids of 32 bricks at once and fills the arrays of those that have one, a
// brick at a time, every c of a lane loaded before any k is computed.
__global__ void k_bulk_fill(MediaDev M, int nx, int ny, int nz, int mx, int my, int mz, double dt,
                            double dx, double dts, long long bb, const int *kslab_of_brick, float *kslabs)
{
    const long long nb = (long long)mx * my * mz;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; g0 < nb; g0 += nw * 32) {
        const long long gl = g0 + lane;
        const int ksl = gl < nb ? kslab_of_brick[bb + gl] : -1;
        unsigned todo = __ballot_sync(FULL, ksl >= 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int ks = __shfl_sync(FULL, ksl, src);
            const long long g = g0 + src;
            const long long cx = g % mx, cy = (g / mx) % my, cz = g / ((long long)mx * my);
            constexpr int PER = (BVOL + 31) / 32;
            float c[PER];
            unsigned in = 0u;   // bit j: node lane + 32 j lies in the grid
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int e = lane + 32 * j;
                const long long gx = cx * BX + e % BX, gy = cy * BY + (e / BX) % BY, gz = cz * BZ + e / (BX * BY);
                const bool ok = e < BVOL && gx < nx && gy < ny && gz < nz;
                c[j] = ok ? media_c(M, nx, ny, gx, gy, gz) : 0.f;
                in |= (ok ? 1u : 0u) << j;
            }
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int e = lane + 32 * j;
                if (e < BVOL) kslabs[(size_t)ks * BVOL + e] = (in >> j & 1u) ? k_of_c(c[j], dt, dx, dts) : 0.f;
            }
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

// Fold the boxes released by the last step into the free stack (the step
// kernel does the same at its start); leaves the counters consistent for
// admissions and releases between steps.
__global__ void k_settle(Engine E)
{
    EngineState *st = E.st;
    st->free_top = max(st->free_top, 0) + st->n_retired;
    st->n_retired = 0;
    st->n_new = 0;
}

// Box bricks[i] (or brick i) of sim: one warp per brick pops a vacant box,
// writes Cell2box / Box2cell and the active bit, and zeroes the box.
__global__ void k_admit(Engine E, int sim, const long long *bricks, long long n)
{
    SimDev *S = E.sims + sim;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const int b = bricks ? (int)bricks[i] : (int)i;
        const long long g = S->brick_base + b;
        int slot = -1;
        if (lane == 0) {
            const int idx = atomicSub(&E.st->free_top, 1) - 1;
            if (idx < 0) {
                atomicAdd(&E.st->free_top, 1);
                atomicOr(&E.st->err, ERR_NOMEM);
                atomicOr(&S->poisoned, 1u);
            } else if (TCM_SLOT_OK(E, idx) && TCM_BRICK_OK(E, g) && TCM_SLOT_OK(E, E.free_stack[idx])) {
                slot = E.free_stack[idx];
                E.slot_of_brick[g] = slot;
                E.claim_step[slot] = -1;
                SlotMeta m;
                m.brick = b;
                m.kslab = E.kslab_of_brick[g];
                m.kscal = E.kscal[g];
                m.flags = ((unsigned)sim << 16) | (brick_has_src(E, S, b) ? FLAG_HAS_SRC : 0u);
                store_meta(E.meta + slot, m);
                E.sd_of_brick[g] &= (unsigned short)FLAG_HAS_SRC;
                atomicOr(E.bitmap + (g >> 5), 1u << (unsigned)(g & 31));
                atomicAdd(E.blocktot + (int)((g >> 5) / E.words_per_block), 1);
            }
        }
        slot = __shfl_sync(FULL, slot, 0);
        if (slot < 0) continue;
        zero_box(E, slot, lane);
    }
}

// Take sim's bricks out of the active set; their boxes (and fields) stay.
__global__ void k_freeze(Engine E, int sim, long long w0, long long n_words)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_words; i += (long long)gridDim.x * blockDim.x) {
        const long long w = w0 + i;
        const int c = __popc(E.bitmap[w]);
        if (c) {
            E.bitmap[w] = 0u;
            atomicSub(E.blocktot + (int)(w / E.words_per_block), c);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) E.sims[sim].live = 0;
}

// Release every box of sim's bricks [bb, bb + n) back to the free stack.
__global__ void k_release(Engine E, int sim, long long bb, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long g = bb + i;
        const int slot = E.slot_of_brick[g];
        if (slot < 0) continue;
        const int idx = atomicAdd(&E.st->free_top, 1);
        if (!TCM_SLOT_OK(E, idx)) continue;
        E.free_stack[idx] = slot;
        E.slot_of_brick[g] = -1;
        E.sd_of_brick[g] = 0;
        const unsigned bit = 1u << (unsigned)(g & 31);
        if (atomicAnd(E.bitmap + (g >> 5), ~bit) & bit)
            atomicSub(E.blocktot + (int)((g >> 5) / E.words_per_block), 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) E.sims[sim].live = 0;
}

// Put a paused sim's boxed bricks back into the active set (the freeze that
// paused it cleared its bitmap words; its boxes, fields and shut-down counts
// stayed) and let it step again.
__global__ void k_thaw(Engine E, int sim, long long w0, long long n_words, long long bb, long long nb)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_words; i += (long long)gridDim.x * blockDim.x) {
        const long long w = w0 + i;
        unsigned bits = 0u;
        for (int j = 0; j < 32; ++j) {
            const long long g = w * 32 + j;
            if (g - bb < nb && E.slot_of_brick[g] >= 0) bits |= 1u << j;
        }
        E.bitmap[w] = bits;
        if (bits) atomicAdd(E.blocktot + (int)(w / E.words_per_block), __popc(bits));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) E.sims[sim].live = 1;
}

// Reach of the live sims' boxed sets: the bricks a sim can box within a few
// steps lie within Chebyshev distance r (in bricks) of a brick it has boxed
// now.  Separable dilation of the boxed set along x, y and z over the brick
// tables (one byte per brick); the z pass counts the unboxed bricks of the
// dilated set.  A brick g belongs to the sim that owns its bitmap word, if it
// lies inside that sim's range (ranges never overlap).
__device__ __forceinline__ const SimDev *reach_sim(const Engine &E, long long g, long long &b)
{
    const SimDev *S = E.sims + E.sim_of_word[g >> 5];
    b = g - S->brick_base;
    return (S->live && b >= 0 && b < S->n_bricks) ? S : nullptr;
}

__global__ void k_reach_x(Engine E, int r, unsigned char *out)
{
    const long long n = E.n_words * 32;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        long long b;
        const SimDev *S = reach_sim(E, g, b);
        unsigned char v = 0;
        if (S) {
            const int cx = (int)(b % S->mx);
            for (int d = max(-r, -cx); d <= r && cx + d < S->mx; ++d)
                if (__ldg(E.slot_of_brick + g + d) >= 0) v = 1;
        }
        out[g] = v;
    }
}

__global__ void k_reach_y(Engine E, int r, const unsigned char *in, unsigned char *out)
{
    const long long n = E.n_words * 32;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        long long b;
        const SimDev *S = reach_sim(E, g, b);
        unsigned char v = 0;
        if (S) {
            const int cy = (int)((b / S->mx) % S->my);
            for (int d = max(-r, -cy); d <= r && cy + d < S->my; ++d)
                if (in[g + (long long)d * S->mx]) v = 1;
        }
        out[g] = v;
    }
}

__global__ void k_reach_z(Engine E, int r, const unsigned char *in, unsigned long long *count)
{
    const long long n = E.n_words * 32;
    unsigned long long c = 0;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        long long b;
        const SimDev *S = reach_sim(E, g, b);
        if (!S || __ldg(E.slot_of_brick + g) >= 0) continue;
        const long long plane = (long long)S->mx * S->my;
        const int cz = (int)(b / plane);
        for (int d = max(-r, -cz); d <= r && cz + d < S->mz; ++d)
            if (in[g + (long long)d * plane]) {
                ++c;
                break;
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// packed[i] = {phi^n, phi^{n-1}} of boxed global brick gids[i].
__global__ void k_scatter_field(Engine E, const float *packed, const long long *gids, long long n, int now_half)
{
    const long long total = n * 2 * BVOL;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long bi = i / (2 * BVOL);
        const int r = (int)(i % (2 * BVOL));
        const int which = r / BVOL, e = r % BVOL;
        // the second array is phi^{-1} in binary32, v^0 in the velocity form
        const long long g = gids[bi];
        const SimDev *S = E.sims + E.sim_of_word[g >> 5];
        const int st = sim_storage(E, S);
        const int half = which == 0 ? now_half : (st == ST_F32 ? (now_half ^ 1) : V_HALF);
        const int slot = E.slot_of_brick[g];
        if (slot >= 0) store_phys(E, st, slot, half, e, packed[i], S->inv_scale);
    }
}

__global__ void k_read_window(Engine E, int sim, int now_half, int which, long long x0, long long y0, long long z0,
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
                const int st = sim_storage(E, S);
                v = which == 0 ? load_phys(E, st, slot, now_half, e, S->scale)
                               : load_prev_phys(E, st, slot, now_half, e, S->scale);
            }
        }
        out[i] = v;
    }
}

// phi^{n-1} at global node (x,y,z) of sim, zero outside or when inactive.
__device__ __forceinline__ double prev_at(const Engine &E, const SimDev *S, int now_half, long long x,
                                          long long y, long long z)
{
    if (x < 0 || y < 0 || z < 0 || x >= S->nx || y >= S->ny || z >= S->nz) return 0.0;
    const long long b = ((z / BZ) * S->my + (y / BY)) * S->mx + (x / BX);
    const int slot = E.slot_of_brick[S->brick_base + b];
    if (slot < 0) return 0.0;
    return (double)load_prev_phys(E, sim_storage(E, S), slot, now_half,
                                  (int)(((z % BZ) * BY + (y % BY)) * BX + (x % BX)), S->scale);
}

__global__ void k_energy(Engine E, int sim, int now_half, int parity, double *out)
{
    const SimDev *S = E.sims + sim;
    const WorkItem *L = parity ? E.items1 : E.items0;
    const long long n = (long long)E.st->n_active[parity] * BVOL;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int slot = L[i / BVOL].slot;
        const int e = (int)(i % BVOL);
        const SlotMeta m = load_meta(E.meta + slot);
        if ((int)(m.flags >> 16) != sim) continue;
        const int b = m.brick;
        const long long x = (long long)(b % S->mx) * BX + e % BX;
        const long long y = (long long)((b / S->mx) % S->my) * BY + (e / BX) % BY;
        const long long z = (long long)(b / (S->mx * S->my)) * BZ + e / (BX * BY);
        if (x >= S->nx || y >= S->ny || z >= S->nz) continue;
        const int st = sim_storage(E, S);
        const double a = (double)load_phys(E, st, slot, now_half, e, S->scale);
        const double bb = (double)load_prev_phys(E, st, slot, now_half, e, S->scale);
        const int nh = now_half;
        const double nb = prev_at(E, S, nh, x - 1, y, z) + prev_at(E, S, nh, x + 1, y, z) +
                          prev_at(E, S, nh, x, y - 1, z) + prev_at(E, S, nh, x, y + 1, z) +
                          prev_at(E, S, nh, x, y, z - 1) + prev_at(E, S, nh, x, y, z + 1);
        const double k = m.kslab >= 0 ? (double)S->kslabs[(size_t)m.kslab * BVOL + e] : (double)m.kscal;
        const double d = a - bb;
        acc += d * d / k + a * (6.0 * bb - nb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// Boxed bricks of sim (its active set; a frozen sim keeps the set it ended
// with): local ids (unsorted, count in *count) and in-domain nodes.
__global__ void k_active_bricks(Engine E, int sim, long long *ids, unsigned long long *count,
                                unsigned long long *cells)
{
    const SimDev *S = E.sims + sim;
    const long long bb = S->brick_base, nb = S->n_bricks;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x) {
        if (E.slot_of_brick[bb + b] < 0) continue;
        const unsigned long long k = atomicAdd(count, 1ull);
        if (ids) ids[k] = b;
        const int cx = (int)(b % S->mx), cy = (int)((b / S->mx) % S->my), cz = (int)(b / ((long long)S->mx * S->my));
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
                                 double dt, double dx, long long bb, float *kscal, int *kslab_of_brick,
                                 int *n_kslabs, cudaStream_t s)
{
    const long long nb = (long long)mx * my * mz;
    k_bulk_classify<<<grid_for(nb, 256), 256, 0, s>>>(m, nx, ny, nz, mx, my, mz, dt, dx, exact_ratio(dt, dx), bb,
                                                      kscal, kslab_of_brick, n_kslabs);
    return cudaGetLastError();
}

cudaError_t launch_bulk_fill(const MediaDev &m, int nx, int ny, int nz, int mx, int my, int mz,
                             double dt, double dx, long long bb, const int *kslab_of_brick, float *kslabs,
                             cudaStream_t s)
{
    const long long nb = (long long)mx * my * mz;
    k_bulk_fill<<<grid_for(nb, 256), 256, 0, s>>>(m, nx, ny, nz, mx, my, mz, dt, dx, exact_ratio(dt, dx), bb,
                                                  kslab_of_brick, kslabs);
    return cudaGetLastError();
}

cudaError_t launch_iota_desc(int *a, int n, int first, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_iota_desc<<<grid_for(n, 256), 256, 0, s>>>(a, n, first);
    return cudaGetLastError();
}

cudaError_t launch_settle(const Engine &e, cudaStream_t s)
{
    k_settle<<<1, 1, 0, s>>>(e);
    return cudaGetLastError();
}

cudaError_t launch_admit(const Engine &e, int sim, const long long *bricks, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_admit<<<grid_for(n * 32, 256), 256, 0, s>>>(e, sim, bricks, n);
    return cudaGetLastError();
}

cudaError_t launch_freeze(const Engine &e, int sim, long long words_begin, long long n_words, cudaStream_t s)
{
    k_freeze<<<grid_for(n_words, 256), 256, 0, s>>>(e, sim, words_begin, n_words);
    return cudaGetLastError();
}

cudaError_t launch_release(const Engine &e, int sim, long long bb, long long n, cudaStream_t s)
{
    k_release<<<grid_for(n, 256), 256, 0, s>>>(e, sim, bb, n);
    return cudaGetLastError();
}

cudaError_t launch_thaw(const Engine &e, int sim, long long words_begin, long long n_words, long long bb,
                        long long n, cudaStream_t s)
{
    k_thaw<<<grid_for(n_words, 256), 256, 0, s>>>(e, sim, words_begin, n_words, bb, n);
    return cudaGetLastError();
}

cudaError_t launch_reach(const Engine &e, int r, unsigned char *a, unsigned char *b, unsigned long long *count,
                         cudaStream_t s)
{
    const long long n = e.n_words * 32;
    const int g = grid_for(n, 256);
    k_reach_x<<<g, 256, 0, s>>>(e, r, a);
    k_reach_y<<<g, 256, 0, s>>>(e, r, a, b);
    k_reach_z<<<g, 256, 0, s>>>(e, r, b, count);
    return cudaGetLastError();
}

cudaError_t launch_compact(const Engine &e, int grid, int list_parity, cudaStream_t s)
{
    k_compact<<<grid, BLOCK, 0, s>>>(e, list_parity);
    return cudaGetLastError();
}

cudaError_t launch_scatter_field(const Engine &e, const float *packed, const long long *gids, long long n,
                                 int now_half, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_scatter_field<<<grid_for(n * 2 * BVOL, 256), 256, 0, s>>>(e, packed, gids, n, now_half);
    return cudaGetLastError();
}

int step_grid_size(int device)
{
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    int a = 0, b = 0, c = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_step<ST_F32>, BLOCK, 0) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step<ST_BF16>, BLOCK, 0) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_step<ST_F16>, BLOCK, 0) != cudaSuccess) return 0;
    int d = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, k_step<ST_MIXED>, BLOCK, 0) != cudaSuccess) return 0;
    per_sm = min(min(a, d), min(b, c));
    return sms * per_sm;
}

// ---------------------------------------------------------------------------
// Eq. 7 frequency-domain shut-down, after an update that released bricks
// holding values (lpf_q): (A) every boxed 26-neighbour of such a brick that
// was not claimed by this update is listed once; (B) for each listed brick
// and each of its two levels, the level over its 3x3x3-brick block
// (released, unboxed and outside bricks read zero) goes through the
// separable filter operator A (x, then y, then z; binary32 FMA, each output
// summed over the taps in increasing order) and the centre brick is kept in
// lpf_out; (C) the filtered values replace the bricks' halves (nodes outside
// the domain stay zero).  Every filtered value comes from the state before (C).
// ---------------------------------------------------------------------------
// Shared memory of one (brick, level) unit: R [L][L][L] the level over the
// block; T1 [L][L][C] after the x pass; T2 [L][C][C] after the y pass; Ax
// [C][LPF_LP] the operator's rows, padded so that the two row groups a warp
// reads sit in different banks; At [L][C] the operator transposed (four
// consecutive outputs per vector).
constexpr int LPF_LP = LPF_L + 4;
constexpr int LPF_BLOCK = 256;   // threads per CTA of the filter kernel (every build)
constexpr size_t LPF_SMEM = sizeof(float) * ((size_t)LPF_L * LPF_L * LPF_L + (size_t)LPF_L * LPF_L * LPF_C +
                                             (size_t)LPF_L * LPF_C * LPF_C + (size_t)LPF_C * LPF_LP +
                                             (size_t)LPF_L * LPF_C);

__device__ __forceinline__ long long lpf_neighbour(const SimDev *S, long long base, int b, int dx, int dy, int dz)
{
    const int mx = S->mx, my = S->my, mz = S->mz;
    const int ax = b % mx + dx, ay = (b / mx) % my + dy, az = b / (mx * my) + dz;
    if (ax < 0 || ay < 0 || az < 0 || ax >= mx || ay >= my || az >= mz) return -1;
    return base + ((long long)az * my + ay) * mx + ax;
}

// Four consecutive elements e..e+3 (e a multiple of 4) of box half (slot,
// half) as physical binary32 values, in one vector load.
__device__ __forceinline__ float4 load_phys4(const Engine &E, int st, int slot, int half, int e, float scale)
{
    const unsigned char *base = box_base(E, slot);
    const size_t i = (size_t)half * BVOL + e;
    if (st == ST_F32) return scale4(__ldcg(reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(base) + i)), scale);
    const uint2 u = __ldcg(reinterpret_cast<const uint2 *>(reinterpret_cast<const unsigned short *>(base) + i));
    if (st == ST_BF16) return Fld<ST_BF16>::cvt(u, scale);
    return Fld<ST_F16>::cvt(u, scale);
}

// acc + w.x v.x + w.y v.y + w.z v.z + w.w v.w, one FMA per term in that order
__device__ __forceinline__ float fma4(float4 w, float4 v, float acc)
{
    acc = __fmaf_rn(w.x, v.x, acc);
    acc = __fmaf_rn(w.y, v.y, acc);
    acc = __fmaf_rn(w.z, v.z, acc);
    return __fmaf_rn(w.w, v.w, acc);
}

// o[t] += w[t] * v (one tap j of four outputs i0+t, over four x)
__device__ __forceinline__ void outer4(float4 w, float4 v, float4 *o)
{
    const float wt[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        o[t].x = __fmaf_rn(wt[t], v.x, o[t].x);
        o[t].y = __fmaf_rn(wt[t], v.y, o[t].y);
        o[t].z = __fmaf_rn(wt[t], v.z, o[t].z);
        o[t].w = __fmaf_rn(wt[t], v.w, o[t].w);
    }
}

__global__ void __launch_bounds__(LPF_BLOCK, 2) k_lpf(Engine E)
{
    extern __shared__ __align__(16) unsigned char smem[];
    EngineState *st = E.st;
    const int nq = __ldcg(&st->n_lpf_q);
    if (nq == 0) return;   // the same value for every block: nobody waits
    const int gtid = blockIdx.x * LPF_BLOCK + threadIdx.x, nthr = gridDim.x * LPF_BLOCK;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->t_lpf = globaltimer();
    // (A) the affected bricks
    for (long long i = gtid; i < (long long)nq * 26; i += nthr) {
        const long long q = E.lpf_q[i / 26];
        const int k = (int)(i % 26);
        const int kk = k < 13 ? k : k + 1;   // skip the centre of the 3x3x3 block
        const SimDev *S = E.sims + E.sim_of_word[q >> 5];
        const long long base = S->brick_base;
        const long long g = lpf_neighbour(S, base, (int)(q - base), kk % 3 - 1, (kk / 3) % 3 - 1, kk / 9 - 1);
        if (g < 0) continue;
        const int slot = __ldcg(E.slot_of_brick + g);
        if (slot < 0) continue;
        if (__ldcg(E.claim_step + slot) == (int)(__ldcg(&S->step) - 1)) continue;   // claimed by this update
        if (atomicCAS(E.lpf_mark + slot, 0, 1) != 0) continue;
        const int idx = atomicAdd(&st->n_lpf_aff, 1);
        if (idx < E.lpf_cap) E.lpf_aff[idx] = g;
        else atomicOr(&st->err, ERR_NOMEM);
    }
    if (!grid_barrier(st, &st->bar_count_lpf)) return;
    const int naff = min(__ldcg(&st->n_lpf_aff), E.lpf_cap);
    // (B) one block per (affected brick, level)
    __shared__ int s_nbslot[27];   // boxes of the 3x3x3 block (-1: none)
    float *R = reinterpret_cast<float *>(smem);
    float *T1 = R + LPF_L * LPF_L * LPF_L;
    float *T2 = T1 + LPF_L * LPF_L * LPF_C;
    float *Ax = T2 + LPF_L * LPF_C * LPF_C;
    float *At = Ax + LPF_C * LPF_LP;
    static_assert(LPF_C % 4 == 0, "four outputs per thread");
    constexpr int C4 = LPF_C / 4, Q = BVOL / 4;
    for (int u = blockIdx.x; u < 2 * naff; u += gridDim.x) {
        const int c = u >> 1, h = u & 1;
        const long long g = E.lpf_aff[c];
        const SimDev *S = E.sims + E.sim_of_word[g >> 5];
        const long long base = S->brick_base;
        const int b = (int)(g - base);
        const float sc = S->scale;
        const int st = sim_storage(E, S);
        if (threadIdx.x < 27) {
            const int nb = threadIdx.x;
            const long long gn = lpf_neighbour(S, base, b, nb % 3 - 1, (nb / 3) % 3 - 1, nb / 9 - 1);
            s_nbslot[nb] = gn >= 0 ? __ldcg(E.slot_of_brick + gn) : -1;
        }
        for (int i = threadIdx.x; i < LPF_C * LPF_L; i += LPF_BLOCK) {
            const float a = S->lpf_a[i];
            Ax[(i / LPF_L) * LPF_LP + i % LPF_L] = a;
            At[(i % LPF_L) * LPF_C + i / LPF_L] = a;
        }
        __syncthreads();
        // the level over the block, four x-consecutive nodes per vector (a row
        // of a brick is x-contiguous in its box and in R)
#pragma unroll 4
        for (int e4 = threadIdx.x; e4 < 27 * Q; e4 += LPF_BLOCK) {
            const int nb = e4 / Q, loc = (e4 % Q) * 4;
            const int slot = s_nbslot[nb];
            const float4 v = slot >= 0 ? load_phys4(E, st, slot, h, loc, sc) : make_float4(0.f, 0.f, 0.f, 0.f);
            const int lx = loc % BX, ly = (loc / BX) % BY, lz = loc / (BX * BY);
            *reinterpret_cast<float4 *>(R + (((nb / 9) * LPF_C + lz) * LPF_L + ((nb / 3) % 3) * LPF_C + ly) * LPF_L +
                                        (nb % 3) * LPF_C + lx) = v;
        }
        __syncthreads();
        // Rows of R that lie in bricks of the block with no box are zero and
        // filter to +0 exactly: those rows (x pass) and z-slabs (y pass) are
        // skipped.  Each thread keeps four (x pass) or sixteen (y, z passes)
        // independent outputs in flight.
        auto row_live = [&](int dz, int dy) {
            const int k = (dz * 3 + dy) * 3;
            return s_nbslot[k] >= 0 || s_nbslot[k + 1] >= 0 || s_nbslot[k + 2] >= 0;
        };
        for (int e = threadIdx.x; e < LPF_L * LPF_L * C4; e += LPF_BLOCK) {   // along x
            const int i0 = (e % C4) * 4, zy = e / C4;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            if (row_live((zy / LPF_L) / LPF_C, (zy % LPF_L) / LPF_C)) {
                const float4 *row = reinterpret_cast<const float4 *>(R + zy * LPF_L);
                const float4 *w0 = reinterpret_cast<const float4 *>(Ax + (i0 + 0) * LPF_LP);
                const float4 *w1 = reinterpret_cast<const float4 *>(Ax + (i0 + 1) * LPF_LP);
                const float4 *w2 = reinterpret_cast<const float4 *>(Ax + (i0 + 2) * LPF_LP);
                const float4 *w3 = reinterpret_cast<const float4 *>(Ax + (i0 + 3) * LPF_LP);
#pragma unroll
                for (int q = 0; q < LPF_L / 4; ++q) {
                    const float4 v = row[q];
                    a0 = fma4(w0[q], v, a0);
                    a1 = fma4(w1[q], v, a1);
                    a2 = fma4(w2[q], v, a2);
                    a3 = fma4(w3[q], v, a3);
                }
            }
            *reinterpret_cast<float4 *>(T1 + zy * LPF_C + i0) = make_float4(a0, a1, a2, a3);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < LPF_L * C4 * C4; e += LPF_BLOCK) {   // along y
            const int x0 = (e % C4) * 4, i0 = ((e / C4) % C4) * 4, z = e / (C4 * C4);
            float4 o[4] = {};
            const int dz = z / LPF_C;
            if (row_live(dz, 0) || row_live(dz, 1) || row_live(dz, 2)) {
#pragma unroll 4
                for (int j = 0; j < LPF_L; ++j)
                    outer4(*reinterpret_cast<const float4 *>(At + j * LPF_C + i0),
                           *reinterpret_cast<const float4 *>(T1 + (z * LPF_L + j) * LPF_C + x0), o);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) *reinterpret_cast<float4 *>(T2 + (z * LPF_C + i0 + t) * LPF_C + x0) = o[t];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < LPF_C * C4 * C4; e += LPF_BLOCK) {   // along z
            const int x0 = (e % C4) * 4, i0 = ((e / C4) % C4) * 4, y = e / (C4 * C4);
            float4 o[4] = {};
#pragma unroll 4
            for (int j = 0; j < LPF_L; ++j)
                outer4(*reinterpret_cast<const float4 *>(At + j * LPF_C + i0),
                       *reinterpret_cast<const float4 *>(T2 + (j * LPF_C + y) * LPF_C + x0), o);
            float *out = E.lpf_out + (size_t)c * 2 * BVOL + h * BVOL;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                *reinterpret_cast<float4 *>(out + ((i0 + t) * LPF_C + y) * LPF_C + x0) = o[t];
        }
        __syncthreads();
    }
    if (!grid_barrier(st, &st->bar_count_lpf)) return;
    // (C) write back, one node (both levels) per thread; in the velocity
    // form v becomes the difference of the two stored filtered levels
    for (long long i = gtid; i < (long long)naff * BVOL; i += nthr) {
        const int c = (int)(i / BVOL), loc = (int)(i % BVOL);
        const long long g = E.lpf_aff[c];
        const SimDev *S = E.sims + E.sim_of_word[g >> 5];
        const int b = (int)(g - S->brick_base);
        const int slot = __ldcg(E.slot_of_brick + g);
        const int mx = S->mx, my = S->my;
        const int x = (b % mx) * BX + loc % BX, y = ((b / mx) % my) * BY + (loc / BX) % BY,
                  z = (b / (mx * my)) * BZ + loc / (BX * BY);
        const bool in = x < S->nx && y < S->ny && z < S->nz;
        const size_t o = (size_t)c * 2 * BVOL + loc;
        const int st = sim_storage(E, S);
        store_phys(E, st, slot, 0, loc, in ? E.lpf_out[o] : 0.f, S->inv_scale);
        store_phys(E, st, slot, 1, loc, in ? E.lpf_out[o + BVOL] : 0.f, S->inv_scale);
        if (st != ST_F32) {
            const int nh = (int)(__ldcg(&S->step) & 1);   // the half holding phi^{n+1}
            const float sn = load_phys(E, st, slot, nh, loc, S->scale), so = load_phys(E, st, slot, nh ^ 1, loc, S->scale);
            store_phys(E, st, slot, V_HALF, loc, __fsub_rn(sn, so), S->inv_scale);
        }
        if (loc == 0) E.lpf_mark[slot] = 0;
    }
    // the last block accounts the launch (time and filtered bricks)
    __shared__ int s_last_lpf;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last_lpf = atomicAdd(&st->lpf_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last_lpf && threadIdx.x == 0) {
        __threadfence();
        st->lpf_ns += globaltimer() - __ldcg(&st->t_lpf);
        st->lpf_bricks += (unsigned long long)naff;
        st->lpf_done = 0u;
    }
}

// Cooperative launch (every block resident at once, so the grid barriers
// are safe) through cudaLaunchKernelEx, which stream capture accepts.
// Self-test of the bounded barrier: every block arrives once at a counter
// the host has set to `start`.  start = 0: the barrier completes.  start = 1:
// the block that arrives last waits for a round no block completes and gives
// up after timeout_ns with ERR_TIMEOUT; every block returns.
__global__ void __launch_bounds__(BLOCK, 1) k_barrier_selftest(EngineState *st, unsigned long long *ctr,
                                                              unsigned long long timeout_ns)
{
    grid_barrier(st, ctr, timeout_ns);
}

cudaError_t launch_cooperative(const void *fn, int grid, int block, size_t smem, void **args, cudaStream_t s);

cudaError_t launch_barrier_selftest(EngineState *st, unsigned long long *ctr, int grid,
                                    unsigned long long timeout_ns, cudaStream_t s)
{
    void *args[] = {&st, &ctr, &timeout_ns};
    return launch_cooperative((const void *)k_barrier_selftest, grid, BLOCK, 0, args, s);
}

cudaError_t launch_cooperative(const void *fn, int grid, int block, size_t smem, void **args, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

int lpf_grid_size(int device)
{
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k_lpf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LPF_SMEM) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lpf, LPF_BLOCK, LPF_SMEM) != cudaSuccess) return 0;
    return sms * per_sm;
}

cudaError_t launch_lpf(const Engine &e, int grid, cudaStream_t s)
{
    Engine copy = e;
    void *args[] = {&copy};
    return launch_cooperative((const void *)k_lpf, grid, LPF_BLOCK, LPF_SMEM, args, s);
}

cudaError_t launch_step(const Engine &e, int grid, int parity, int manage, cudaStream_t s)
{
    Engine copy = e;
    int p = parity, m = manage;
    void *args[] = {&copy, &p, &m};
    const void *fn = e.storage == ST_BF16  ? (const void *)k_step<ST_BF16>
                     : e.storage == ST_F16   ? (const void *)k_step<ST_F16>
                     : e.storage == ST_MIXED ? (const void *)k_step<ST_MIXED>
                                             : (const void *)k_step<ST_F32>;
    return launch_cooperative(fn, grid, BLOCK, 0, args, s);
}

cudaError_t launch_read_window(const Engine &e, int sim, int now_half, int which, long long x0, long long y0,
                               long long z0, long long wx, long long wy, long long wz, float *out,
                               cudaStream_t s)
{
    const long long n = wx * wy * wz;
    if (n <= 0) return cudaSuccess;
    k_read_window<<<grid_for(n, 256), 256, 0, s>>>(e, sim, now_half, which, x0, y0, z0, wx, wy, wz, out);
    return cudaGetLastError();
}

cudaError_t launch_energy(const Engine &e, int sim, int now_half, int list_parity, double *out,
                          cudaStream_t s)
{
    k_energy<<<1024, 256, 0, s>>>(e, sim, now_half, list_parity, out);
    return cudaGetLastError();
}

cudaError_t launch_active_bricks(const Engine &e, int sim, int list_parity, long long *ids_out,
                                 unsigned long long *n_out, unsigned long long *cells_out, cudaStream_t s)
{
    (void)list_parity;
    k_active_bricks<<<1024, 256, 0, s>>>(e, sim, ids_out, n_out, cells_out);
    return cudaGetLastError();
}

}  // namespace tcm
