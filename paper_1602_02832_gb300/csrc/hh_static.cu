// hh_force_static: the list force of hh_force for callers that cannot
// allocate device memory.  Its scratch (packed j records, tiles, work items,
// per-part partial sums, counters) lives in one file-scope __device__ array
// of fixed size instead of cudaMalloc'd buffers.  See include/hh.h.

#include <atomic>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "hh_internal.h"
#include "hh_kernels.cuh"

using namespace hh;

namespace {

constexpr int64_t kStaticMaxJ = 131072;    // j entries
constexpr int64_t kStaticMaxAct = 65536;   // active particles (and tiles)
constexpr int64_t kStaticMaxParts = 8192;  // (tile, list part) work items
constexpr int32_t kStaticPartLen = 2048;   // list entries per part
constexpr int kStaticTj = 256;             // staged chunk (both precisions)
constexpr int kMaxDevices = 64;

// byte layout of the scratch array (each region 256-byte aligned)
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffDs = 0;
constexpr size_t kOffCnt = kOffDs + align256(sizeof(DevScalars));
constexpr size_t kOffTiles = kOffCnt + align256(sizeof(int32_t) * kStaticMaxAct);
constexpr size_t kOffItems = kOffTiles + align256(sizeof(int4) * kStaticMaxAct);
constexpr size_t kOffParts = kOffItems + align256(sizeof(WorkItem) * kStaticMaxParts);
constexpr size_t kOffRec = kOffParts + align256(sizeof(RedF64) * kMaxTileI * kStaticMaxParts);
constexpr size_t kScratchBytes = kOffRec + align256(sizeof(RecF64) * kStaticMaxJ);
constexpr size_t kZeroBytes = kOffTiles;  // DevScalars and tile counters start at zero

static_assert(sizeof(RedMix) <= sizeof(RedF64) && sizeof(RecMix) <= sizeof(RecF64), "scratch sizing");

// The scratch itself.  In host code g_scratch is only a host-side stand-in
// for the symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSetup {
    std::once_flag once;
    int rc = HH_ECUDA;
    unsigned char *base = nullptr;
    int force_grid = 0, elem_grid = 0;
};
DeviceSetup g_setup[kMaxDevices];

void setup_device(int device, DeviceSetup &st)
{
    // called with `device` current
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || ptr == nullptr) {
        cudaGetLastError();
        st.rc = HH_ECUDA;
        return;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        st.rc = HH_ECUDA;
        return;
    }
    int per_f64 = 0, per_mix = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_f64, k_force<RecF64, kStaticTj, true>, kThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_mix, k_force<RecMix, kStaticTj, true>, kThreads, 0);
    const int per = per_f64 < per_mix ? per_f64 : per_mix;
    st.force_grid = prop.multiProcessorCount * (per > 0 ? per : 1);
    st.elem_grid = prop.multiProcessorCount * 4;
    st.base = static_cast<unsigned char *>(ptr);
    st.rc = HH_OK;
}

template <typename Rec>
__global__ void k_static_pack(Rec *rec, const double *x, const double *v, const double *m, int64_t n_j)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_j; e += (int64_t)gridDim.x * blockDim.x) {
        const double xp[3] = {x[e], x[n_j + e], x[2 * n_j + e]};
        const double vp[3] = {v[e], v[n_j + e], v[2 * n_j + e]};
        store_rec<Rec>(rec, e, xp, vp, m[e]);
    }
}

// Tiles = runs of consecutive active positions with the same list, cut at
// every 32nd position; one warp per 32 positions.  Every part of every tile
// becomes a work item.  Overflowing the fixed item capacity sets ds->err and
// writes nothing out of bounds.
__global__ void k_static_tiles(const int32_t *gid, int32_t n_act, int32_t n_groups, const int64_t *off,
                               int4 *tiles, WorkItem *items, DevScalars *ds)
{
    if (*(volatile int32_t *)&ds->err) return;  // inputs failed the checks
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = warp0; c * 32 < n_act; c += nwarps) {
        const int64_t k = c * 32 + lane;
        const bool in = k < n_act;
        const int32_t g = in ? gid[k] : -1;
        const bool bad = in && (g < 0 || g >= n_groups);
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) atomicExch(&ds->err, HH_EINVAL);
            continue;
        }
        const int32_t gprev = __shfl_up_sync(0xffffffffu, g, 1);
        const bool start = in && (lane == 0 || g != gprev);
        const uint32_t starts = __ballot_sync(0xffffffffu, start);
        const uint32_t valid = __ballot_sync(0xffffffffu, in);
        if (start) {
            // this tile spans [k, next start or end of valid lanes)
            const uint32_t later = starts & ~((2u << lane) - 1u);
            const int end_lane = later ? (__ffs(later) - 1) : (32 - __clz(valid));
            const int n_a = end_lane - lane;
            const int64_t len = off[g + 1] - off[g];
            const int n_parts = len > 0 ? (int)((len + kStaticPartLen - 1) / kStaticPartLen) : 1;
            const int t = atomicAdd(&ds->n_tiles, 1);
            const uint32_t base = atomicAdd(&ds->n_items, (uint32_t)n_parts);
            if ((int64_t)base + n_parts > kStaticMaxParts) {
                atomicExch(&ds->err, HH_ENOMEM);
            } else {
                const int4 td = make_int4((int)k, (int)k + n_a, g, (int)base);
                tiles[t] = td;
                const uint32_t mask = n_a == 32 ? 0xffffffffu : ((1u << n_a) - 1u);
                for (int q = 0; q < n_parts; q++) items[base + q] = make_item(t, q, mask, (int)base, td, off[g], off[g + 1], kStaticPartLen);
            }
        }
    }
}

// Caller-supplied device inputs are checked before the force kernel reads
// them: off[0] = 0 and non-decreasing, list and i indices inside [0, n_j).
__global__ void k_static_check(const int64_t *off, int32_t n_groups, const int32_t *idx, const int32_t *i_idx,
                               int32_t n_act, int64_t n_j, DevScalars *ds)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    if (tid == 0 && off[0] != 0) bad = true;
    for (int64_t g = tid; g < n_groups; g += nth)
        if (off[g + 1] < off[g]) bad = true;
    for (int64_t k = tid; k < n_act; k += nth)
        if (i_idx[k] < 0 || i_idx[k] >= n_j) bad = true;
    if (bad) atomicExch(&ds->err, HH_EINVAL);
}

__global__ void k_static_check_idx(const int64_t *off, int32_t n_groups, const int32_t *idx, int64_t n_j,
                                   DevScalars *ds)
{
    if (ds->err) return;  // off itself is not trusted after a failed check
    const int64_t L = off[n_groups];
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L; e += (int64_t)gridDim.x * blockDim.x)
        if (idx[e] < 0 || idx[e] >= n_j) bad = true;
    if (bad) atomicExch(&ds->err, HH_EINVAL);
}

__global__ void k_static_finish(DevScalars *ds)
{
    // the force kernel must see no items when tiling failed
    if (ds->err) ds->n_items = 0u;
    ds->part_len = kStaticPartLen;
}

// Restores the current device of the calling thread when it goes out of scope.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    DeviceGuard() { ok = cudaGetDevice(&prev) == cudaSuccess; }
    ~DeviceGuard()
    {
        if (ok) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" int hh_force_static(int device, int precision, double eps2, int64_t n_j, const double *xj,
                               const double *vj, const double *mj, int32_t n_groups, const int64_t *off,
                               const int32_t *idx, int32_t n_act, const int32_t *i_idx, const int32_t *gid,
                               double *acc, double *jerk, double *pot, void *stream)
{
    if (device < 0 || device >= kMaxDevices) return hh_set_global_error(HH_EINVAL, "hh_force_static: bad device");
    if (precision != HH_FP64 && precision != HH_MIXED)
        return hh_set_global_error(HH_EINVAL, "hh_force_static: precision must be HH_FP64 or HH_MIXED");
    if (!(eps2 >= 0.0)) return hh_set_global_error(HH_EINVAL, "hh_force_static: eps2 must be >= 0");
    if (n_j < 1 || n_j > kStaticMaxJ)
        return hh_set_global_error(HH_EINVAL, "hh_force_static: n_j must be in [1, 131072] (static scratch limit)");
    if (n_act < 0 || n_act > kStaticMaxAct)
        return hh_set_global_error(HH_EINVAL, "hh_force_static: n_act must be in [0, 65536] (static scratch limit)");
    if (n_groups < 1) return hh_set_global_error(HH_EINVAL, "hh_force_static: n_groups must be >= 1");
    if (!xj || !vj || !mj || !off || !idx || (n_act > 0 && (!i_idx || !gid || !acc || !jerk || !pot)))
        return hh_set_global_error(HH_EINVAL, "hh_force_static: NULL array");
    // the caller's current device is put back on every return
    DeviceGuard guard;
    if (!guard.ok) return hh_set_global_error(HH_ECUDA, "hh_force_static: cudaGetDevice failed");
    if (cudaSetDevice(device) != cudaSuccess) return hh_set_global_error(HH_ECUDA, "hh_force_static: cudaSetDevice failed");
    DeviceSetup &st = g_setup[device];
    std::call_once(st.once, [&] { setup_device(device, st); });
    if (st.rc != HH_OK) return hh_set_global_error(st.rc, "hh_force_static: scratch set-up (cudaGetSymbolAddress) failed");
    if (n_act == 0) return HH_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *base = st.base;
    DevScalars *ds = reinterpret_cast<DevScalars *>(base + kOffDs);
    if (cudaMemsetAsync(base, 0, kZeroBytes, s) != cudaSuccess)
        return hh_set_global_error(HH_ECUDA, "hh_force_static: clearing the scratch header failed");
    Lists L;
    L.off = off;
    L.idx = idx;
    L.tiles = reinterpret_cast<int4 *>(base + kOffTiles);
    L.items = reinterpret_cast<WorkItem *>(base + kOffItems);
    L.partials = base + kOffParts;
    L.tile_cnt = reinterpret_cast<int32_t *>(base + kOffCnt);
    L.i_map = i_idx;
    State S;
    std::memset(&S, 0, sizeof(S));
    S.acc1 = acc;
    S.jerk1 = jerk;
    S.pot1 = pot;
    S.cap_n = n_act;  // outputs are SoA [3][n_act], indexed by active position
    Params prm;
    std::memset(&prm, 0, sizeof(prm));
    prm.eps2 = eps2;
    StepCtl c{1, 0, 1, 0, 0.0};
    if (precision == HH_MIXED)
        k_static_pack<RecMix><<<st.elem_grid, 256, 0, s>>>(reinterpret_cast<RecMix *>(base + kOffRec), xj, vj, mj, n_j);
    else
        k_static_pack<RecF64><<<st.elem_grid, 256, 0, s>>>(reinterpret_cast<RecF64 *>(base + kOffRec), xj, vj, mj, n_j);
    k_static_check<<<st.elem_grid, 256, 0, s>>>(off, n_groups, idx, i_idx, n_act, n_j, ds);
    k_static_check_idx<<<st.elem_grid, 256, 0, s>>>(off, n_groups, idx, n_j, ds);
    k_static_tiles<<<st.elem_grid, 256, 0, s>>>(gid, n_act, n_groups, off, const_cast<int4 *>(L.tiles), L.items, ds);
    k_static_finish<<<1, 1, 0, s>>>(ds);
    if (precision == HH_MIXED)
        k_force<RecMix, kStaticTj, true><<<st.force_grid, kThreads, 0, s>>>(
            S, reinterpret_cast<const RecMix *>(base + kOffRec), L, ds, c, prm);
    else
        k_force<RecF64, kStaticTj, true><<<st.force_grid, kThreads, 0, s>>>(
            S, reinterpret_cast<const RecF64 *>(base + kOffRec), L, ds, c, prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hh_set_global_error(HH_ECUDA, cudaGetErrorString(e));
    int32_t err = 0;
    if (cudaMemcpyAsync(&err, &ds->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return hh_set_global_error(HH_ECUDA, "hh_force_static: kernel execution failed");
    if (err == HH_ENOMEM)
        return hh_set_global_error(HH_ENOMEM, "hh_force_static: more than 8192 (tile, list part) work items; "
                                              "split the active set into smaller calls");
    if (err) return hh_set_global_error(HH_EINVAL, "hh_force_static: bad input (off not starting at 0 or "
                                                   "decreasing, an index outside [0, n_j), or a list id outside "
                                                   "[0, n_groups))");
    return HH_OK;
}
