// tcm_noalloc.cu -- tcm_energy_noalloc: the discrete energy of a simulation
// computed without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc/cudaFree while a
// simulation runs -- code whose device memory is owned by another allocator
// with a fixed budget, and code on a latency-critical path that must not
// synchronise the device (cudaFree does).  tcm_energy allocates an
// accumulator on every call; this variant keeps its scratch in a file-scope
// __device__ array instead.
//
// Scratch: one FP64 partial sum per entry of the batch's active list (the
// active bricks of every simulation of the batch; a simulation made by
// tcm_create is a batch of one), NOALLOC_MAX_BRICKS of them (512 KiB),
// resident on every GPU that loads the library until the process exits.
// Entries of other simulations get a zero partial.  Every call overwrites the
// partials it reads, so nothing has to start at zero; calls whose kernels
// overlap on the GPU (two streams, two simulations) race on the array and
// must be serialised by the caller.
#include "../../include/tcm.h"
#include "tcm_internal.cuh"

namespace {

constexpr int NOALLOC_MAX_BRICKS = 65536;
constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr int FINAL_THREADS = 1024;

static __device__ __align__(256) double g_energy_partials[NOALLOC_MAX_BRICKS];

// Host-side device addresses of g_energy_partials, one per device (the name
// itself is only a host stand-in and must never be passed to a kernel).
double *g_partials_addr[NOALLOC_MAX_DEVICES] = {};

// phi^{n-1} at a global node of the sim, zero outside or when inactive.
__device__ __forceinline__ double prev_node(const tcm::Engine &E, const tcm::SimDev *S, int now_half,
                                            long long x, long long y, long long z)
{
    using namespace tcm;
    if (x < 0 || y < 0 || z < 0 || x >= S->nx || y >= S->ny || z >= S->nz) return 0.0;
    const long long b = ((z / BZ) * S->my + (y / BY)) * S->mx + (x / BX);
    const int slot = E.slot_of_brick[S->brick_base + b];
    if (slot < 0) return 0.0;
    return (double)load_prev_phys(E, sim_storage(E, S), slot, now_half,
                                  (int)(((z % BZ) * BY + (y % BY)) * BX + (x % BX)), S->scale);
}

// One warp per active brick: its energy contribution, reduced in a fixed
// order so the result does not depend on scheduling.
__global__ void k_energy_partials(tcm::Engine E, int sim, int now_half, int parity, int n, double *part)
{
    using namespace tcm;
    const int lane = threadIdx.x & 31;
    const WorkItem *L = parity ? E.items1 : E.items0;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int ph = now_half;   // prev_node derives phi^{n-1} from the half holding phi^n
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const int slot = L[i].slot;
        const int4 mv = *reinterpret_cast<const int4 *>(E.meta + slot);
        const int b = mv.x, kslab = mv.y;
        const double kscal = (double)__int_as_float(mv.z);
        const SimDev *S = E.sims + ((unsigned)mv.w >> 16);
        if ((int)((unsigned)mv.w >> 16) != sim) {
            if (lane == 0) part[i] = 0.0;
            continue;
        }
        const int st = sim_storage(E, S);
        const long long bx0 = (long long)(b % S->mx) * BX, by0 = (long long)((b / S->mx) % S->my) * BY,
                        bz0 = (long long)(b / (S->mx * S->my)) * BZ;
        double acc = 0.0;
        for (int e = lane; e < BVOL; e += 32) {
            const long long x = bx0 + e % BX, y = by0 + (e / BX) % BY, z = bz0 + e / (BX * BY);
            if (x >= S->nx || y >= S->ny || z >= S->nz) continue;
            const double a = (double)load_phys(E, st, slot, now_half, e, S->scale);
            const double bb = (double)load_prev_phys(E, st, slot, now_half, e, S->scale);
            const double nb = prev_node(E, S, ph, x - 1, y, z) + prev_node(E, S, ph, x + 1, y, z) +
                              prev_node(E, S, ph, x, y - 1, z) + prev_node(E, S, ph, x, y + 1, z) +
                              prev_node(E, S, ph, x, y, z - 1) + prev_node(E, S, ph, x, y, z + 1);
            const double k = kslab >= 0 ? (double)S->kslabs[(size_t)kslab * BVOL + e] : kscal;
            const double d = a - bb;
            acc += d * d / k + a * (6.0 * bb - nb);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) part[i] = acc;
    }
}

// One block sums the n partials in a fixed order and writes the total.
__global__ void k_energy_total(const double *part, int n, double *out)
{
    __shared__ double s[FINAL_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += FINAL_THREADS) acc += part[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = FINAL_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

}  // namespace

extern "C" tcm_status tcm_energy_noalloc(const tcm_sim *sim, double *device_out)
{
    tcm::SimView v;
    // A started simulation whose batch changed since the last step gets its
    // active list rebuilt first (a compaction launch, which allocates nothing).
    if (!device_out || !tcm_internal_view(sim, &v, true)) return TCM_EINVAL;
    if (!v.started) return TCM_ESTATE;
    if (!v.list_ok) return TCM_EDEVICE;
    if (v.device < 0 || v.device >= NOALLOC_MAX_DEVICES) return TCM_EINVAL;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return TCM_EDEVICE;
    if (prev != v.device && cudaSetDevice(v.device) != cudaSuccess) return TCM_EDEVICE;
    tcm_status st = TCM_OK;
    do {
        // Set-up, once per device, with that device current: the device
        // address of the scratch array.
        if (!g_partials_addr[v.device]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_energy_partials) != cudaSuccess || !p) {
                cudaGetLastError();
                st = TCM_EDEVICE;
                break;
            }
            g_partials_addr[v.device] = static_cast<double *>(p);
        }
        int n = 0;
        if (cudaMemcpyAsync(&n, &v.E->st->n_active[v.list_parity], sizeof(int), cudaMemcpyDeviceToHost,
                            v.stream) != cudaSuccess ||
            cudaStreamSynchronize(v.stream) != cudaSuccess) {
            st = TCM_EDEVICE;
            break;
        }
        if (n > NOALLOC_MAX_BRICKS) {  // a longer active list than the scratch holds
            st = TCM_EINVAL;
            break;
        }
        double *part = g_partials_addr[v.device];
        if (n > 0) {
            const int blocks = (n + 7) / 8;
            k_energy_partials<<<blocks, 256, 0, v.stream>>>(*v.E, v.sim, (int)(v.step & 1), v.list_parity, n, part);
        }
        k_energy_total<<<1, FINAL_THREADS, 0, v.stream>>>(part, n, device_out);
        if (cudaGetLastError() != cudaSuccess) st = TCM_EDEVICE;
    } while (0);
    if (prev >= 0 && prev != v.device) cudaSetDevice(prev);
    return st;
}
