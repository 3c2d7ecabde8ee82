// Tree-loop step 1 on the device (Section 2): Morton octree, Barnes groups
// and interaction lists built from the synchronised particle state without
// leaving the GPU, then the particles reordered into Morton order and the
// node records written behind them.  The rules are those of the host builder
// (include/hh.h, hh_tree_build): root cube from the bounding box, 21-bit
// Morton keys, cells split while they hold more than `leaf` particles,
// pre-order cell numbering, groups = maximal cells with <= n_crit particles,
// the same opening walk.  Node moments are warp sums (the host sums in
// index order), so a node's centre of mass may differ in the last bits.
//
// CUB (shipped with the CUDA toolkit) provides the radix sort of the keys and
// the prefix sums; every other step is a kernel of this file.

#include <algorithm>
#include <cstring>
#include <functional>
#include <vector>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_segmented_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "hh_ctx.h"

using namespace hh;

namespace {

constexpr int kBits = 21;
constexpr int kMaxDepth = 21;

// ------------------------------------------------------------ small helpers
__device__ __forceinline__ unsigned long long order_bits(double v)  // monotone map double -> u64
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_order_bits(unsigned long long o)
{
    const unsigned long long b = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ uint64_t spread_bits(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ int digit_at(uint64_t key, int depth) { return int((key >> (3 * (kBits - 1 - depth))) & 7u); }

// Peano-Hilbert key of a cell of the 2^21 grid (Skilling 2004): the low bit
// fields are mapped level by level into each sub-cube's frame, Gray-coded,
// and the resulting transposed index is interleaved like a Morton key.
__device__ __forceinline__ uint64_t hilbert_key(uint32_t a0, uint32_t a1, uint32_t a2)
{
    uint32_t c[3] = {a0, a1, a2};
#pragma unroll 1
    for (uint32_t q = 1u << (kBits - 1); q > 1u; q >>= 1) {
        const uint32_t p = q - 1u;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const uint32_t t = (c[0] ^ c[i]) & p;
            if (c[i] & q) {
                c[0] ^= p;
            } else {
                c[0] ^= t;
                c[i] ^= t;
            }
        }
    }
    c[1] ^= c[0];
    c[2] ^= c[1];
    uint32_t flip = 0;
    for (uint32_t q = 1u << (kBits - 1); q > 1u; q >>= 1)
        if (c[2] & q) flip ^= q - 1u;
    return (spread_bits(c[0] ^ flip) << 2) | (spread_bits(c[1] ^ flip) << 1) | spread_bits(c[2] ^ flip);
}

struct Box {
    unsigned long long lo[3], hi[3];  // order bits
    int32_t bad;                      // a particle not at the tree time
};

// BFS level arrays: cells of one level are contiguous; the children of a cell
// are one contiguous block of the next level, in octant order (the blocks of
// different cells are placed in whatever order the reservations happen, which
// changes no pre-order number: those follow from the tree alone).
struct Cells {
    int32_t *begin, *end, *depth, *nchild, *first;  // first: BFS index of the first child
    int32_t *parent;                                 // BFS index of the parent (-1 root)
    int32_t *size;                                   // cells in the subtree
    int32_t *pre;                                    // pre-order number
};

// Sizes the build keeps on the device, so that no step waits for the host:
// level d holds cells [lvl_c0[d], lvl_c0[d] + lvl_n[d]).
struct GCounts {
    int32_t lvl_c0[kMaxDepth + 2];
    int32_t lvl_n[kMaxDepth + 2];
    int32_t ncells, overflow, bad, G, R, A, pad[2];
    int64_t L, n_tiles, total_parts;
    unsigned long long lmax;  // longest list
};

// Pre-order cell table used by the group and list kernels.
struct PCells {
    int32_t *begin, *end, *nchild, *parent;
    int32_t *size;   // cells in the subtree: the subtree of p is [p, p + size)
    int4 *pack;      // {begin, end, nchild, size}: what the list walk reads per cell
    float4 *cf;      // {centre of mass x, y, z, side} rounded to FP32 (screening)
    int32_t *child;  // [8 * n]
    double *side;
};

enum : int { kOpen = 0, kEmitParticles = 1, kEmitNode = 2 };

// The opening decision of cell c for group g (rules of hh_tree_build): the
// group's own cell and single particles go in as particles; a cell that does
// not contain the group goes in as a node when side < theta * (distance of its
// centre of mass to the group's box), else as particles when it is a leaf;
// everything else is opened.
//
// The distance test is screened in FP32 (FP64 throughput is low on this part).
// With X a bound on |coordinates|, rounding centre, box and side to FP32 and
// evaluating gaps, squares, sum, sqrtf and the product with theta in FP32
// moves side - theta * distance by less than
// 2^-21 (side + theta * distance) + 2^-21 theta X; the screen's margin is
// 2^-18 (side + theta * distance) + 2^-19 theta X.  Inside the margin the test
// is redone in FP64 with the roundings of the sequential builder (no
// contraction), so the decision is always the FP64 one.
struct GroupView {
    int32_t gc, gb, ge;
    double lo[3], hi[3];
    float3 lof, hif;
};

__device__ __forceinline__ int decide(const State &s, const PCells &P, int64_t n, double theta, float theta_f,
                                      float tol_abs, const GroupView &G, int32_t c, int4 &pk)
{
    // both records are loaded before any test, so that a walk step waits for
    // one memory round trip, not two (the tables are read-only here)
    pk = __ldg(&P.pack[c]);
    const float4 cf = __ldg(&P.cf[c]);
    if (c == G.gc) return kEmitParticles;
    if (pk.x <= G.gb && G.ge <= pk.y) return kOpen;
    if (pk.y - pk.x == 1) return kEmitParticles;
    const float gx = fmaxf(fmaxf(G.lof.x - cf.x, cf.x - G.hif.x), 0.f);
    const float gy = fmaxf(fmaxf(G.lof.y - cf.y, cf.y - G.hif.y), 0.f);
    const float gz = fmaxf(fmaxf(G.lof.z - cf.z, cf.z - G.hif.z), 0.f);
    const float rhs = theta_f * sqrtf(gx * gx + gy * gy + gz * gz);
    const float tol = 0x1p-18f * (cf.w + rhs) + tol_abs;
    bool accept;
    if (cf.w < rhs - tol) {
        accept = true;
    } else if (cf.w > rhs + tol) {
        accept = false;
    } else {
        double d2 = 0.0;
        for (int d = 0; d < 3; d++) {
            const double cm = s.x[d * s.cap_j + n + c];
            double gap = 0.0;
            if (cm < G.lo[d]) gap = __dsub_rn(G.lo[d], cm);
            else if (cm > G.hi[d]) gap = __dsub_rn(cm, G.hi[d]);
            d2 = __dadd_rn(d2, __dmul_rn(gap, gap));
        }
        accept = P.side[c] < __dmul_rn(theta, __dsqrt_rn(d2));
    }
    if (accept) return kEmitNode;
    return pk.z == 0 ? kEmitParticles : kOpen;
}

// Everything a rebuild kernel reads or writes for one simulation.  A kernel
// runs for one simulation (the record passed by value) or for many (an array
// in device memory, simulation = blockIdx.y): the same code either way.
// Scans are read relative to their first entry, so a simulation's slice of
// one scan over many simulations' arrays reads like its own scan.
struct RbSim {
    State st, alt;            // particle state and the buffer it is reordered into
    Cells C;
    PCells P;
    GCounts *gc;
    Box *box;
    double *root_side;
    float *xmax;
    uint64_t *key, *key2;     // particle keys, and sorted
    int32_t *idx, *perm;      // particle indices, and in key order
    uint64_t *ckey, *ckey2;   // cell keys (first particle, depth), and sorted
    int32_t *cval, *cval2;    // cell indices, and in key order
    double *mom;              // [13][cap_c] cell sums (BFS order)
    int32_t *flag3, *pos3;    // [3][ncells] selection flags and their exclusive scan
    int32_t *g_cell, *cut, *above;
    double *box_lo, *box_hi;  // [3][G] group boxes
    float4 *box_f;
    int64_t *ids, *ids2;
    int32_t *group_of;
    int64_t *off;             // [G + 1] list offsets
    int32_t *lidx;            // list entries
    int4 *tiles;
    int64_t *nt2, *tscan2;    // [tile counts | part counts], G + 1 each, and their scan
    int64_t *pair2, *pscan2;  // [particle | node entries per (group, cut cell)], pairs + 1 each, and their scan
    int32_t *top;             // [G][A] topmost unopened cell above the cut
    DevScalars *ds;           // the context's device sizes (set by k_finish)
    double t, theta;
    float theta_f;
    int64_t n, cap_c, pairs;
    int32_t cap_g, cap_cells, leaf, n_crit, order, tile_i, part_len, work_item, work_split;
    int32_t ncells, S, G, R, A;  // set by the host as they become known
};

#define RB_ARGS const RbSim one, const RbSim *many

// For many simulations a block first copies its record into shared memory:
// read from there (as from the constant bank for one), the record's fields
// can be fetched again where they are used instead of occupying registers.
template <bool kMany>
__device__ __forceinline__ const RbSim &rb_sim_of(const RbSim &one, const RbSim *many, unsigned char *sh)
{
    if (!kMany) return one;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(many + blockIdx.y);
    uint32_t *dst = reinterpret_cast<uint32_t *>(sh);
    for (int i = threadIdx.x; i < int(sizeof(RbSim) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    return *reinterpret_cast<const RbSim *>(sh);
}
#define RB_SIM                                                      \
    __shared__ __align__(16) unsigned char rb_rec_[sizeof(RbSim)]; \
    const RbSim &a = rb_sim_of<kMany>(one, many, rb_rec_)

template <bool kMany>
__global__ void k_box(RB_ARGS)
{
    RB_SIM;
    const State &s = a.st;
    const double t_tree = a.t;
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int d = 0; d < 3; d++) {
            const unsigned long long o = order_bits(s.x[d * s.cap_j + i]);
            lo[d] = o < lo[d] ? o : lo[d];
            hi[d] = o > hi[d] ? o : hi[d];
        }
        bad |= s.t[i] != t_tree;
    }
    // warp, then block reduction (blockDim.x = 256): one atomic per block and
    // bound, and none from a block that saw no particle
    __shared__ unsigned long long s_lo[8][3], s_hi[8][3];
    __shared__ int s_bad[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = 0; d < 3; d++) {
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo[d], off);
            const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi[d], off);
            lo[d] = l2 < lo[d] ? l2 : lo[d];
            hi[d] = h2 > hi[d] ? h2 : hi[d];
        }
        if (lane == 0) {
            s_lo[w][d] = lo[d];
            s_hi[w][d] = hi[d];
        }
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) s_bad[w] = any_bad;
    __syncthreads();
    if (threadIdx.x == 0) {
        int b = 0;
        for (int k = 0; k < int(blockDim.x >> 5); k++) {
            b |= s_bad[k];
            for (int d = 0; d < 3; d++) {
                lo[d] = s_lo[k][d] < lo[d] ? s_lo[k][d] : lo[d];
                hi[d] = s_hi[k][d] > hi[d] ? s_hi[k][d] : hi[d];
            }
        }
        if (lo[0] <= hi[0])
            for (int d = 0; d < 3; d++) {
                atomicMin(&a.box->lo[d], lo[d]);
                atomicMax(&a.box->hi[d], hi[d]);
            }
        if (b) atomicExch(&a.box->bad, 1);
    }
}

template <bool kMany>
__global__ void k_keys(RB_ARGS)
{
    RB_SIM;
    const State &s = a.st;
    const Box *b = a.box;
    double lo[3], side = 0.0;
    for (int d = 0; d < 3; d++) {
        lo[d] = from_order_bits(b->lo[d]);
        const double ext = from_order_bits(b->hi[d]) - lo[d];
        if (ext > side) side = ext;
    }
    if (side == 0.0) side = 1.0;
    const double scale = double(1u << kBits) / side;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.root_side = side;
        double xm = 0.0;  // bound on |coordinate| of every particle, node and group box
        for (int d = 0; d < 3; d++) xm = fmax(xm, fmax(fabs(lo[d]), fabs(from_order_bits(b->hi[d]))));
        *a.xmax = float(xm) * 1.0001f;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t u[3];
        for (int d = 0; d < 3; d++) {
            double f = floor((s.x[d * s.cap_j + i] - lo[d]) * scale);
            f = f < 0.0 ? 0.0 : f;
            f = f > double((1u << kBits) - 1u) ? double((1u << kBits) - 1u) : f;
            u[d] = uint32_t(f);
        }
        a.key[i] = a.order == HH_ORDER_HILBERT ? hilbert_key(u[0], u[1], u[2])
                                               : (spread_bits(u[0]) << 2) | (spread_bits(u[1]) << 1) | spread_bits(u[2]);
        a.idx[i] = int32_t(i);
    }
}

// one thread per simulation
template <bool kMany>
__global__ void k_root_init(RB_ARGS)
{
    RB_SIM;
    Box *b = a.box;
    GCounts *gc = a.gc;
    for (int d = 0; d < 3; d++) {  // empty bounding box
        b->lo[d] = ~0ull;
        b->hi[d] = 0ull;
    }
    b->bad = 0;
    a.C.begin[0] = 0;
    a.C.end[0] = int32_t(a.n);
    a.C.depth[0] = 0;
    a.C.parent[0] = -1;
    a.C.pre[0] = 0;
    for (int d = 0; d < kMaxDepth + 2; d++) gc->lvl_c0[d] = gc->lvl_n[d] = 0;
    gc->lvl_n[0] = 1;
    gc->ncells = gc->overflow = gc->bad = gc->G = gc->R = gc->A = 0;
    gc->lmax = 0ull;
}

// Splits the cells of level d that hold more than `leaf` particles (and are
// above the depth limit): the octant boundaries come from binary searches of
// the sorted keys, and each cell reserves its block of children in level d+1.
template <bool kMany>
__global__ void k_level(RB_ARGS, int d)
{
    RB_SIM;
    const Cells &C = a.C;
    const uint64_t *key = a.key2;
    GCounts *gc = a.gc;
    // after an overflow the level counts include blocks that were not written:
    // nothing below reads them, and the host reports HH_ENOMEM
    if (gc->overflow) return;
    const int32_t c0 = gc->lvl_c0[d], nc = gc->lvl_n[d], next0 = c0 + nc;
    if (blockIdx.x == 0 && threadIdx.x == 0) gc->lvl_c0[d + 1] = next0;
    // Eight lanes per cell: lane o finds where octant o ends (the first
    // index of the cell's sorted range whose digit at this depth exceeds o)
    // by its own binary search, so a large cell costs one search, not
    // eight in a row.  The digit is monotone over the range, so these ends
    // are the octant boundaries.
    const int lane = threadIdx.x & 31;
    const int64_t n_q = (int64_t)nc * 8;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;  // a multiple of 32: warps stay whole
    for (int64_t q0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; q0 < n_q; q0 += stride) {
        const int64_t q = q0 + lane;
        const bool valid = q < n_q;
        const int32_t c = c0 + (int32_t)(q >> 3);
        const int o = (int)(q & 7);
        int32_t b = 0, e = 0, hi = 0;
        bool split = false;
        if (valid) {
            b = C.begin[c];
            e = C.end[c];
            split = e - b > a.leaf && d < kMaxDepth;
            if (split) {
                int32_t l = b, h = e;
                while (l < h) {
                    const int32_t mid = (l + h) >> 1;
                    if (digit_at(key[mid], d) <= o) l = mid + 1;
                    else h = mid;
                }
                hi = l;
            }
        }
        int32_t ends[8];
#pragma unroll
        for (int k = 0; k < 8; k++) ends[k] = __shfl_sync(0xffffffffu, hi, (lane & ~7) | k);
        if (!valid || o != 0) continue;
        int32_t bound[9];
        int nch = 0;
        if (split) {
            int32_t lo = b;
            for (int k = 0; k < 8 && lo < e; k++) {
                if (ends[k] > lo) bound[nch++] = lo;
                lo = ends[k];
            }
            bound[nch] = e;
        }
        C.first[c] = next0;
        C.nchild[c] = 0;
        if (nch == 0) continue;
        const int32_t w = next0 + atomicAdd(&gc->lvl_n[d + 1], nch);
        if ((int64_t)w + nch > a.cap_cells) {
            atomicExch(&gc->overflow, 1);
            continue;
        }
        C.first[c] = w;
        C.nchild[c] = nch;
        for (int k = 0; k < nch; k++) {
            C.begin[w + k] = bound[k];
            C.end[w + k] = bound[k + 1];
            C.depth[w + k] = d + 1;
            C.parent[w + k] = c;
        }
    }
}

// After the levels 0..d: the cells made so far (complete when level d made
// no children, i.e. lvl_n[d + 1] == 0), and the synchronisation flag of the
// bounding-box pass.  One thread per simulation.
template <bool kMany>
__global__ void k_cells_done(RB_ARGS, int d)
{
    RB_SIM;
    a.gc->ncells = a.gc->lvl_c0[d + 1] + a.gc->lvl_n[d + 1];
    a.gc->bad = a.box->bad;
}

// Pre-order numbers and subtree sizes without a pass per level: the cells
// sorted by (first particle, depth) are in pre-order (children follow their
// parent in octant order, which is particle order, and a cell's descendants
// are the cells after it that start before it ends).  Key of a cell:
// begin << 5 | depth (depth <= kMaxDepth < 32).
template <bool kMany>
__global__ void k_cell_keys(RB_ARGS)
{
    RB_SIM;
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < a.ncells; c += gridDim.x * blockDim.x) {
        a.ckey[c] = (uint64_t(a.C.begin[c]) << 5) | uint64_t(a.C.depth[c]);
        a.cval[c] = c;
    }
}

// From the sorted keys and cells: pre[c] = its rank; size[c] = the cells from
// it to the first one that starts at or after its end.
template <bool kMany>
__global__ void k_pre_size(RB_ARGS)
{
    RB_SIM;
    const int32_t ncells = a.ncells;
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < ncells; p += gridDim.x * blockDim.x) {
        const int32_t c = a.cval2[p];
        a.C.pre[c] = p;
        const uint64_t lim = uint64_t(a.C.end[c]) << 5;
        int32_t lo = p + 1, hi = ncells;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (a.ckey2[mid] < lim) lo = mid + 1;
            else hi = mid;
        }
        a.C.size[c] = lo - p;
    }
}

template <bool kMany>
__global__ void k_to_preorder(RB_ARGS)
{
    RB_SIM;
    const Cells &C = a.C;
    const PCells &P = a.P;
    const double s0 = *a.root_side;
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < a.ncells; c += gridDim.x * blockDim.x) {
        const int32_t p = C.pre[c];
        P.begin[p] = C.begin[c];
        P.end[p] = C.end[c];
        P.nchild[p] = C.nchild[c];
        P.size[p] = C.size[c];
        P.pack[p] = make_int4(C.begin[c], C.end[c], C.nchild[c], C.size[c]);
        P.parent[p] = C.parent[c] >= 0 ? C.pre[C.parent[c]] : -1;
        double side = s0;
        for (int d = 0; d < C.depth[c]; d++) side *= 0.5;
        P.side[p] = side;
        for (int k = 0; k < C.nchild[c]; k++) P.child[8 * p + k] = C.pre[C.first[c] + k];
    }
}

// State of the reordered particles: alt[k] = st[perm[k]] (Morton order).
template <bool kMany>
__global__ void k_permute(RB_ARGS)
{
    RB_SIM;
    const State &src = a.st;
    const State &dst = a.alt;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a.perm[k];
        for (int d = 0; d < 3; d++) {
            dst.x[d * dst.cap_j + k] = src.x[d * src.cap_j + i];
            dst.v[d * dst.cap_j + k] = src.v[d * src.cap_j + i];
            dst.a[d * dst.cap_j + k] = src.a[d * src.cap_j + i];
            dst.jk[d * dst.cap_j + k] = src.jk[d * src.cap_j + i];
        }
        dst.m[k] = src.m[i];
        dst.t[k] = src.t[i];
        dst.dt[k] = src.dt[i];
        a.ids2[k] = a.ids[i];
    }
}

// Node records (pseudo-particles): mass and mass-weighted sums of x, v, a, jk
// of the members, bottom-up one tree level per launch: a leaf sums its
// particles, an inner cell the sums of its children.  mom is [13][cap] in BFS
// cell order.  (st is the reordered state.)
template <bool kMany>
__global__ void k_moments_level(RB_ARGS, int d)
{
    RB_SIM;
    const State &s = a.st;
    const Cells &C = a.C;
    const int64_t cap = a.cap_c;
    double *mom = a.mom;
    if (a.gc->overflow) return;
    const int32_t c0 = a.gc->lvl_c0[d], nc = a.gc->lvl_n[d];
    // one thread per (cell, moment): the 13 sums of a cell run side by side
    // (each in the same order as a single thread would take them), since a
    // warp's FP64 instruction costs the pipe the same however few lanes use it
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)nc * 13;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = c0 + (int32_t)(q / 13);
        const int w = (int)(q - (q / 13) * 13);
        double acc = 0.0;
        const int nch = C.nchild[c];
        if (nch == 0) {
            // w = 0: mass; 1 + 3k + dim: mass times x, v, a, jerk (k = 0..3)
            const double *f = w == 0 ? nullptr : (w < 4 ? s.x : w < 7 ? s.v : w < 10 ? s.a : s.jk) +
                                                     (int64_t)((w - 1) % 3) * s.cap_j;
            for (int32_t p = C.begin[c]; p < C.end[c]; p++) {
                const double mi = s.m[p];
                acc = w == 0 ? acc + mi : fma(mi, f[p], acc);
            }
        } else {
            const int32_t f = C.first[c];
            for (int k = 0; k < nch; k++) acc += mom[w * cap + f + k];
        }
        mom[w * cap + c] = acc;
    }
}

// j entry n + (pre-order number) of every cell: centre of mass and
// mass-weighted mean velocity, acceleration and jerk at the tree time.
template <bool kMany>
__global__ void k_node_records(RB_ARGS)
{
    RB_SIM;
    const State &s = a.st;
    const int64_t cap = a.cap_c;
    const double *mom = a.mom;
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < a.ncells; c += gridDim.x * blockDim.x) {
        const int32_t p = a.C.pre[c];
        const int64_t j = a.n + p;
        const double M = mom[c];
        s.m[j] = M;
        s.t[j] = a.t;
        double x[3];
        for (int d = 0; d < 3; d++) {
            x[d] = mom[(1 + d) * cap + c] / M;
            s.x[d * s.cap_j + j] = x[d];
            s.v[d * s.cap_j + j] = mom[(4 + d) * cap + c] / M;
            s.a[d * s.cap_j + j] = mom[(7 + d) * cap + c] / M;
            s.jk[d * s.cap_j + j] = mom[(10 + d) * cap + c] / M;
        }
        a.P.cf[p] = make_float4(float(x[0]), float(x[1]), float(x[2]), float(a.P.side[p]));
    }
}

// Bounding box of each group's particles ([3][G] lo and hi), one warp per group
// (none beyond cap_g groups: the host then reports the overflow).
template <bool kMany>
__global__ void k_group_box(RB_ARGS)
{
    RB_SIM;
    const State &s = a.st;
    const int32_t G = a.gc->G;
    if (G > a.cap_g) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = w0; g < G; g += nw) {
        const int32_t c = a.g_cell[g], b = a.P.begin[c], e = a.P.end[c];
        for (int d = 0; d < 3; d++) {
            double lo = s.x[d * s.cap_j + b], hi = lo;
            for (int32_t p = b + lane; p < e; p += 32) {
                const double u = s.x[d * s.cap_j + p];
                lo = u < lo ? u : lo;
                hi = u > hi ? u : hi;
            }
            for (int off = 16; off > 0; off >>= 1) {
                const double l2 = __shfl_xor_sync(0xffffffffu, lo, off), h2 = __shfl_xor_sync(0xffffffffu, hi, off);
                lo = l2 < lo ? l2 : lo;
                hi = h2 > hi ? h2 : hi;
            }
            if (lane == 0) {
                a.box_lo[d * G + g] = lo;
                a.box_hi[d * G + g] = hi;
            }
        }
        if (lane == 0) {
            a.box_f[2 * g] = make_float4(float(a.box_lo[g]), float(a.box_lo[G + g]), float(a.box_lo[2 * G + g]), 0.f);
            a.box_f[2 * g + 1] =
                make_float4(float(a.box_hi[g]), float(a.box_hi[G + g]), float(a.box_hi[2 * G + g]), 0.f);
        }
    }
}

// Groups (Barnes 1990): maximal cells with <= n_crit particles (or leaves).
// Cut through the tree: the maximal cells whose subtree holds <= S cells.
// They partition the cells at or below the cut; every cell above it is an
// ancestor of some cut cell.  The three selections at once: flags [groups |
// cut cells | cells above the cut], each ncells long, in pre-order,
// compacted by one exclusive scan (positions of the second and third
// selections are offset by the counts before them).
template <bool kMany>
__global__ void k_flags3(RB_ARGS)
{
    RB_SIM;
    const PCells &P = a.P;
    const int32_t ncells = a.ncells, S = a.S;
    int32_t *flag = a.flag3;
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        const int32_t cnt = P.end[c] - P.begin[c];
        const bool small = cnt <= a.n_crit || P.nchild[c] == 0;
        const int32_t par = P.parent[c];
        const bool parent_big = par < 0 || !((P.end[par] - P.begin[par]) <= a.n_crit || P.nchild[par] == 0);
        flag[c] = (small && parent_big) ? 1 : 0;                                         // group
        flag[ncells + c] = (P.size[c] <= S && (par < 0 || P.size[par] > S)) ? 1 : 0;     // cut cell
        flag[2 * ncells + c] = P.size[c] > S ? 1 : 0;                                    // above the cut
    }
}

// one thread per simulation
template <bool kMany>
__global__ void k_counts3(RB_ARGS)
{
    RB_SIM;
    const int32_t *pos = a.pos3, *flag = a.flag3;
    const int32_t ncells = a.ncells;
    a.gc->G = pos[ncells] - pos[0];
    a.gc->R = pos[2 * ncells] - pos[ncells];
    a.gc->A = pos[3 * ncells - 1] + flag[3 * ncells - 1] - pos[2 * ncells];
}

// groups (g_cell, group_of), cut cells and cells above the cut, in pre-order
// (group cells beyond cap_g are not stored: the host reports the overflow)
template <bool kMany>
__global__ void k_write3(RB_ARGS)
{
    RB_SIM;
    const int32_t *pos = a.pos3, *flag = a.flag3;
    const int32_t ncells = a.ncells;
    const int32_t g0 = pos[0], r0 = pos[ncells], a0 = pos[2 * ncells];
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        if (flag[c]) {
            const int32_t g = pos[c] - g0;
            if (g < a.cap_g) a.g_cell[g] = c;
            for (int32_t p = a.P.begin[c]; p < a.P.end[c]; p++) a.group_of[p] = g;
        }
        if (flag[ncells + c]) a.cut[pos[ncells + c] - r0] = c;
        if (flag[2 * ncells + c]) a.above[pos[2 * ncells + c] - a0] = c;
    }
}

// The group's cell, its particle range and its box (FP64 and FP32), as the
// list walk reads them.
__device__ __forceinline__ GroupView group_view(const RbSim &a, int32_t g)
{
    GroupView V;
    V.gc = a.g_cell[g];
    V.gb = a.P.begin[V.gc];
    V.ge = a.P.end[V.gc];
    for (int d = 0; d < 3; d++) {
        V.lo[d] = a.box_lo[d * a.G + g];
        V.hi[d] = a.box_hi[d * a.G + g];
    }
    const float4 l = a.box_f[2 * g], h = a.box_f[2 * g + 1];
    V.lof = make_float3(l.x, l.y, l.z);
    V.hif = make_float3(h.x, h.y, h.z);
    return V;
}

// the FP32 screen's absolute margin, 2^-19 theta X
__device__ __forceinline__ float walk_tol(const RbSim &a) { return 0x1p-19f * a.theta_f * *a.xmax; }


// For every (group g, cell above the cut a = above[i]): the topmost cell on
// the path root -> a that the walk of g does not open (-1: all opened).
// Cells above the cut are few; this replaces a walk up the tree per
// (group, cut cell) pair by one table lookup.
template <bool kMany>
__global__ void k_top_above(RB_ARGS)
{
    RB_SIM;
    const float tol = walk_tol(a);
    const int32_t A = a.A;
    const int64_t total = int64_t(a.G) * A;
    // neighbouring threads take neighbouring groups under the same cell: the
    // same path, similar decisions, coalesced group records
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = int32_t(t / a.G), g = int32_t(t - int64_t(i) * a.G);
        const int64_t q = int64_t(g) * A + i;
        const GroupView V = group_view(a, g);
        int32_t top = -1;
        int4 pk;
        for (int32_t c = a.above[i]; c >= 0; c = a.P.parent[c])
            if (decide(a.st, a.P, a.n, a.theta, a.theta_f, tol, V, c, pk) != kOpen) top = c;
        a.top[q] = top;
    }
}

// One thread per (group g, cut cell k).  The topmost cell on the path
// root -> cut[k] that the walk does not open comes from the table of the
// parent (above the cut) and the decision on cut[k] itself; if there is one,
// the leftmost cut cell below it emits it (once); otherwise the thread walks
// the subtree of cut[k] in pre-order, skipping every emitted cell's subtree.
// The list of a group is then the concatenation over k in pre-order:
// particles ascending, then nodes ascending, as in the sequential walk.
// Pass 0 counts into cnt_p/cnt_n[g * R + k] (and zeroes both arrays'
// terminal entries); pass 1 writes at the scanned offsets.  cnt_n follows
// cnt_p's terminal entry, so one exclusive scan covers both (each read
// relative to its first entry).
template <bool kMany, bool kWrite>
__global__ void k_lists_cut(RB_ARGS)
{
    RB_SIM;
    const float tol = walk_tol(a);
    const int32_t R = a.R, A = a.A;
    const int64_t total = int64_t(a.G) * R;
    const int64_t n = a.n;
    const int32_t *cut = a.cut, *above_pos = a.pos3 + 2 * int64_t(a.ncells);
    int64_t *cnt_p = a.pair2, *cnt_n = a.pair2 + a.pairs + 1;
    const int64_t *scan_p = a.pscan2, *scan_n = a.pscan2 + a.pairs + 1;
    if (!kWrite && blockIdx.x == 0 && threadIdx.x == 0) cnt_p[total] = cnt_n[total] = 0;
    const int64_t pb = kWrite ? scan_p[0] : 0, nb = kWrite ? scan_n[0] : 0;
    // neighbouring threads take neighbouring groups (in space too) under the
    // same cut cell: they walk the same subtree, mostly alike, and read the
    // same cells; the counts stay indexed by g * R + k
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = int32_t(t / a.G), g = int32_t(t - int64_t(k) * a.G);
        const int64_t q = int64_t(g) * R + k;
        const int32_t r = cut[k], par = a.P.parent[r];
        int32_t top = par >= 0 ? a.top[int64_t(g) * A + (above_pos[par] - above_pos[0])] : -1;
        if (top >= 0 && k > 0 && cut[k - 1] >= top) {  // emitted by an earlier cut cell
            if (!kWrite) cnt_p[q] = cnt_n[q] = 0;
            continue;
        }
        const GroupView V = group_view(a, g);
        int64_t wp = 0, wn = 0;
        if (kWrite) {
            wp = (scan_p[q] - pb) + (scan_n[int64_t(g) * R] - nb);
            wn = (scan_p[int64_t(g + 1) * R] - pb) + (scan_n[q] - nb);
        }
        int64_t np = 0, nn = 0;
        int4 pk;
        int top_dec;
        if (top >= 0) {
            top_dec = decide(a.st, a.P, n, a.theta, a.theta_f, tol, V, top, pk);
        } else {
            top_dec = decide(a.st, a.P, n, a.theta, a.theta_f, tol, V, r, pk);
            if (top_dec != kOpen) top = r;
        }
        if (top >= 0) {
            if (top_dec == kEmitNode) {
                if (kWrite) a.lidx[wn] = int32_t(n + top);
                nn = 1;
            } else {
                if (kWrite)
                    for (int32_t p = pk.x; p < pk.y; p++) a.lidx[wp++] = p;
                np = pk.y - pk.x;
            }
        } else {
            const int32_t end = r + pk.w;
            int32_t c = r + 1;
            while (c < end) {
                const int dec = decide(a.st, a.P, n, a.theta, a.theta_f, tol, V, c, pk);
                if (dec == kOpen) {
                    c++;
                    continue;
                }
                if (dec == kEmitNode) {
                    if (kWrite) a.lidx[wn++] = int32_t(n + c);
                    nn++;
                } else {
                    if (kWrite)
                        for (int32_t p = pk.x; p < pk.y; p++) a.lidx[wp++] = p;
                    np += pk.y - pk.x;
                }
                c += pk.w;
            }
        }
        if (!kWrite) {
            cnt_p[q] = np;
            cnt_n[q] = nn;
        }
    }
}

// off[g] = entries of all lists before group g (g = 0..G)
template <bool kMany>
__global__ void k_list_off(RB_ARGS)
{
    RB_SIM;
    const int32_t G = a.G, R = a.R;
    const int64_t *scan_p = a.pscan2, *scan_n = a.pscan2 + a.pairs + 1;
    const int64_t pb = scan_p[0], nb = scan_n[0];
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += gridDim.x * blockDim.x)
        a.off[g] = (scan_p[int64_t(g) * R] - pb) + (scan_n[int64_t(g) * R] - nb);
}

// tiles of <= tile_i particles per group and their list parts; the longest list
template <bool kMany>
__global__ void k_tile_counts(RB_ARGS)
{
    RB_SIM;
    const int32_t G = a.G;
    int64_t *ntile = a.nt2, *nparts = a.nt2 + G + 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) ntile[G] = nparts[G] = 0;  // terminal entries of the scan
    unsigned long long lmax = 0ull;
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const int32_t c = a.g_cell[g];
        const int64_t cnt = a.P.end[c] - a.P.begin[c];
        const int64_t nt = (cnt + a.tile_i - 1) / a.tile_i;
        const int64_t L = a.off[g + 1] - a.off[g];
        const int64_t parts = L > 0 ? (L + a.part_len - 1) / a.part_len : 1;
        ntile[g] = nt;
        nparts[g] = nt * parts;
        lmax = max(lmax, (unsigned long long)L);
    }
    if (lmax) atomicMax(&a.gc->lmax, lmax);
}

// list length and tile / work-item totals (one thread per simulation)
template <bool kMany>
__global__ void k_store_totals(RB_ARGS)
{
    RB_SIM;
    const int32_t G = a.G;
    const int64_t *tile_off = a.tscan2, *parts_off = a.tscan2 + G + 1;
    a.gc->L = a.off[G];
    a.gc->n_tiles = tile_off[G] - tile_off[0];
    a.gc->total_parts = parts_off[G] - parts_off[0];
}

template <bool kMany>
__global__ void k_tiles(RB_ARGS)
{
    RB_SIM;
    const int64_t t0 = a.tscan2[0];
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < a.G; g += gridDim.x * blockDim.x) {
        const int32_t c = a.g_cell[g];
        const int32_t b = a.P.begin[c], e = a.P.end[c];
        int64_t t = a.tscan2[g] - t0;
        for (int32_t p = b; p < e; p += a.tile_i) a.tiles[t++] = make_int4(p, min(p + a.tile_i, e), g, 0);
    }
}

// Closing step of a batched build: the context's sizes on the device and,
// for the mixed form, the base records of every j entry (particles in their
// new order, then the new nodes).
template <bool kMany>
__global__ void k_finish(RB_ARGS)
{
    RB_SIM;
    const GCounts *gc = a.gc;
    const int64_t nj = a.n + gc->ncells;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ds->n = a.n;
        a.ds->nj = nj;
        a.ds->n_tiles = int32_t(gc->n_tiles);
        a.ds->part_len = a.part_len;
        a.ds->work_item = a.work_item;
        a.ds->work_split = a.work_split;
    }
    if (a.st.base)
        for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nj; q += (int64_t)gridDim.x * blockDim.x)
            refresh_base(a.st, q);
}

template <typename K, typename V>
int cub_sort_pairs(void *&tmp, size_t &tmp_bytes, const K *kin, K *kout, const V *vin, V *vout, int64_t n, int bits,
                   cudaStream_t st)
{
    size_t need = 0;
    if (cub::DeviceRadixSort::SortPairs(nullptr, need, kin, kout, vin, vout, (int)n, 0, bits, st) != cudaSuccess ||
        need == 0)
        return HH_ECUDA;
    if (need > tmp_bytes) {
        if (tmp) cudaFree(tmp);
        tmp = nullptr;
        tmp_bytes = 0;
        if (cudaMalloc(&tmp, need) != cudaSuccess) return HH_ENOMEM;
        tmp_bytes = need;
    }
    return cub::DeviceRadixSort::SortPairs(tmp, need, kin, kout, vin, vout, (int)n, 0, bits, st) == cudaSuccess
               ? HH_OK
               : HH_ECUDA;
}

template <typename T>
int cub_exclusive_sum(void *&tmp, size_t &tmp_bytes, const T *in, T *out, int64_t n, cudaStream_t st)
{
    size_t need = 0;
    if (cub::DeviceScan::ExclusiveSum(nullptr, need, in, out, (int)n, st) != cudaSuccess || need == 0) return HH_ECUDA;
    if (need > tmp_bytes) {
        if (tmp) cudaFree(tmp);
        tmp = nullptr;
        tmp_bytes = 0;
        if (cudaMalloc(&tmp, need) != cudaSuccess) return HH_ENOMEM;
        tmp_bytes = need;
    }
    return cub::DeviceScan::ExclusiveSum(tmp, need, in, out, (int)n, st) == cudaSuccess ? HH_OK : HH_ECUDA;
}

}  // namespace

// Buffers of the device builder, owned by the context (allocated on first use).
struct GTreeBuf {
    int64_t cap_n = 0, cap_c = 0;
    uint64_t *key = nullptr, *key2 = nullptr;
    int32_t *idx = nullptr, *perm = nullptr;
    Box *box = nullptr;
    double *root_side = nullptr;
    float *xmax = nullptr;
    GCounts *gc = nullptr;      // device
    GCounts *gc_host = nullptr;  // pinned mirror
    float4 *box_f = nullptr;
    Cells C{};
    PCells P{};
    int32_t *flag3 = nullptr, *pos3 = nullptr;  // [3][cap_c] selection flags and their scan
    int32_t *g_cell = nullptr, *cut = nullptr, *above = nullptr;
    // [tile counts | part counts] and their one scan, each 2 (G + 1) long
    int64_t *ntile = nullptr, *tile_off = nullptr;
    double *mom = nullptr;                    // [13][cap_c] cell sums (BFS order)
    double *box_lo = nullptr, *box_hi = nullptr;  // [3][cap_g] group boxes
    State alt{};                 // second particle-state buffer for the reordering
    int64_t *ids = nullptr, *ids2 = nullptr;
    // (group, cut cell) counts and their scans, grown on demand
    int64_t *pair_buf = nullptr;
    int64_t pair_cap = 0;
    int32_t *top_buf = nullptr;  // [G][A] topmost unopened cell above the cut
    int64_t top_cap = 0;
    int depth = -1;              // depth of the last tree (-1: none yet)
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    std::vector<void *> all;
};

int64_t *hh_gtree_ids(GTreeBuf *g) { return g->ids; }

// Ordered on the context's stream: the copy lands before the next rebuild's
// reordering kernel reads the ids (a copy on the legacy stream would not be
// ordered with a non-blocking stream).
int hh_gtree_set_ids(GTreeBuf *g, const int64_t *ids, int64_t n, cudaStream_t st)
{
    if (cudaMemcpyAsync(g->ids, ids, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return HH_ECUDA;
    return HH_OK;
}

// The second state set is swapped with the context's at every rebuild, so it
// is freed through its current pointers (the context frees the other set).
void hh_gtree_free(GTreeBuf *g)
{
    if (!g) return;
    for (void *p : g->all)
        if (p) cudaFree(p);
    for (double *p : {g->alt.x, g->alt.v, g->alt.a, g->alt.jk, g->alt.m, g->alt.t, g->alt.dt})
        if (p) cudaFree(p);
    if (g->tmp) cudaFree(g->tmp);
    if (g->pair_buf) cudaFree(g->pair_buf);
    if (g->top_buf) cudaFree(g->top_buf);
    if (g->gc_host) cudaFreeHost(g->gc_host);
    delete g;
}

namespace {

int gfail(hh_ctx *ctx, int code, const char *m)
{
    ctx->err = m;
    return hh_set_global_error(code, m);
}

template <typename T>
bool galloc(GTreeBuf *g, T **p, size_t count, bool track = true)
{
    if (cudaMalloc((void **)p, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return false;
    }
    if (track) g->all.push_back(*p);
    return true;
}

GTreeBuf *gtree_alloc(hh_ctx *ctx)
{
    GTreeBuf *g = new GTreeBuf;
    const int64_t n = ctx->cap_n, cc = ctx->cap_j;  // cells <= cap_j - n, capped by cap_j
    g->cap_n = n;
    g->cap_c = cc;
    bool ok = galloc(g, &g->key, n) && galloc(g, &g->key2, n) && galloc(g, &g->idx, n) && galloc(g, &g->perm, n) &&
              galloc(g, &g->box, 1) && galloc(g, &g->root_side, 1) && galloc(g, &g->C.begin, cc) &&
              galloc(g, &g->C.end, cc) && galloc(g, &g->C.depth, cc) && galloc(g, &g->C.nchild, cc) &&
              galloc(g, &g->C.first, cc) && galloc(g, &g->C.parent, cc) && galloc(g, &g->C.size, cc) &&
              galloc(g, &g->C.pre, cc) && galloc(g, &g->P.begin, cc) && galloc(g, &g->P.end, cc) &&
              galloc(g, &g->P.nchild, cc) && galloc(g, &g->P.parent, cc) && galloc(g, &g->P.child, 8 * cc) &&
              galloc(g, &g->P.side, cc) && galloc(g, &g->P.size, cc) && galloc(g, &g->P.pack, cc) &&
              galloc(g, &g->P.cf, cc) && galloc(g, &g->xmax, 1) && galloc(g, &g->gc, 1) &&
              galloc(g, &g->box_f, 2 * ctx->cap_g) && galloc(g, &g->flag3, 3 * cc) && galloc(g, &g->pos3, 3 * cc) &&
              galloc(g, &g->g_cell, ctx->cap_g) && galloc(g, &g->cut, cc) && galloc(g, &g->above, cc) &&
              galloc(g, &g->mom, 13 * cc) && galloc(g, &g->box_lo, 3 * ctx->cap_g) &&
              galloc(g, &g->box_hi, 3 * ctx->cap_g) &&
              galloc(g, &g->ntile, 2 * (ctx->cap_g + 1)) && galloc(g, &g->tile_off, 2 * (ctx->cap_g + 1)) &&
              galloc(g, &g->ids, n) && galloc(g, &g->ids2, n);
    // the second state buffer mirrors the context's (same capacities)
    g->alt = ctx->st;
    g->alt.x = g->alt.v = g->alt.a = g->alt.jk = g->alt.m = g->alt.t = g->alt.dt = nullptr;
    ok = ok && galloc(g, &g->alt.x, 3 * ctx->cap_j, false) && galloc(g, &g->alt.v, 3 * ctx->cap_j, false) &&
         galloc(g, &g->alt.a, 3 * ctx->cap_j, false) && galloc(g, &g->alt.jk, 3 * ctx->cap_j, false) &&
         galloc(g, &g->alt.m, ctx->cap_j, false) && galloc(g, &g->alt.t, ctx->cap_j, false) &&
         galloc(g, &g->alt.dt, n, false);
    if (ok && cudaHostAlloc((void **)&g->gc_host, sizeof(GCounts), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        g->gc_host = nullptr;
        ok = false;
    }
    if (!ok) {
        hh_gtree_free(g);
        return nullptr;
    }
    return g;
}

int64_t gtree_bytes(const hh_ctx *ctx)
{
    const int64_t n = ctx->cap_n, cc = ctx->cap_j, G = ctx->cap_g + 1;
    return n * (8 * 2 + 4 * 2 + 8 * 2) + cc * (4 * 8 + 4 * 5 + 32 + 8 + 4 * 8 + 13 * 8 + 32) +
           G * (4 + 8 * 4 + 6 * 8 + 32) + ctx->cap_j * 8 * (12 + 2) + n * 8;
}

}  // namespace

namespace {

// The record of one simulation for the rebuild kernels, with the buffers of
// its context and of its device builder; sizes and scratch pointers are
// filled in as the build goes.
RbSim rb_sim(hh_ctx *ctx, GTreeBuf *g, double t)
{
    RbSim a{};
    a.st = ctx->st;
    a.alt = g->alt;
    a.C = g->C;
    a.P = g->P;
    a.gc = g->gc;
    a.box = g->box;
    a.root_side = g->root_side;
    a.xmax = g->xmax;
    a.key = g->key;
    a.key2 = g->key2;
    a.idx = g->idx;
    a.perm = g->perm;
    // the cell sort's keys and values live in the moment sums and the
    // selection arrays, not yet in use when the cells are sorted
    a.ckey = reinterpret_cast<uint64_t *>(g->mom);
    a.ckey2 = a.ckey + g->cap_c;
    a.cval = g->flag3;
    a.cval2 = g->pos3;
    a.mom = g->mom;
    a.flag3 = g->flag3;
    a.pos3 = g->pos3;
    a.g_cell = g->g_cell;
    a.cut = g->cut;
    a.above = g->above;
    a.box_lo = g->box_lo;
    a.box_hi = g->box_hi;
    a.box_f = g->box_f;
    a.ids = g->ids;
    a.ids2 = g->ids2;
    a.group_of = ctx->group_of;
    a.off = ctx->off;
    a.lidx = ctx->idx;
    a.tiles = ctx->tiles;
    a.nt2 = g->ntile;
    a.tscan2 = g->tile_off;
    a.pair2 = g->pair_buf;
    a.pscan2 = nullptr;
    a.top = g->top_buf;
    a.t = t;
    a.theta = ctx->cfg.theta;
    a.theta_f = float(ctx->cfg.theta);
    a.n = ctx->n;
    a.cap_c = g->cap_c;
    a.cap_g = ctx->cap_g;
    a.cap_cells = int32_t(std::min<int64_t>(ctx->cap_j - ctx->n, INT32_MAX));
    a.leaf = ctx->cfg.leaf;
    a.n_crit = ctx->cfg.n_crit;
    a.order = ctx->cfg.order;
    a.tile_i = ctx->tile_i;
    a.part_len = ctx->part_len;
    a.ds = ctx->ds;
    a.work_item = ctx->cfg.work_item;
    a.work_split = ctx->cfg.work_split;
    return a;
}

// After the reordering the context's state and the builder's second buffer
// trade places.
void swap_state(hh_ctx *ctx, GTreeBuf *g)
{
    std::swap(ctx->st.x, g->alt.x);
    std::swap(ctx->st.v, g->alt.v);
    std::swap(ctx->st.a, g->alt.a);
    std::swap(ctx->st.jk, g->alt.jk);
    std::swap(ctx->st.m, g->alt.m);
    std::swap(ctx->st.t, g->alt.t);
    std::swap(ctx->st.dt, g->alt.dt);
    std::swap(g->ids, g->ids2);
}

int gtree_prepare(hh_ctx *ctx)
{
    // A non-sticky error left pending by earlier runtime calls would make the
    // library calls below report failure; every call here is checked itself.
    cudaGetLastError();
    if (!ctx->gtree) {
        ctx->gtree = gtree_alloc(ctx);
        if (!ctx->gtree) return gfail(ctx, HH_ENOMEM, "hh_rebuild: device tree buffers do not fit");
        ctx->device_bytes += gtree_bytes(ctx);
        // particle ids live on the device from now on
        if (hh_gtree_set_ids(ctx->gtree, ctx->ids.data(), ctx->n, ctx->stream) != HH_OK)
            return gfail(ctx, HH_ECUDA, "hh_rebuild: id upload failed");
    }
    return HH_OK;
}

// Grows a device buffer to at least `need` elements (its contents are not kept).
template <typename T>
bool grow(T *&p, int64_t &cap, int64_t need)
{
    if (need <= cap) return true;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc((void **)&p, sizeof(T) * size_t(need)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cap = need;
    return true;
}

int grow_list(hh_ctx *ctx, int64_t L)
{
    if (L <= ctx->cap_list) return HH_OK;  // the list buffer grows by a quarter beyond the need
    const int64_t cap = L + L / 4 + 1024;
    int32_t *idx = nullptr;
    if (cudaMalloc(&idx, sizeof(int32_t) * cap) != cudaSuccess) {
        cudaGetLastError();
        return gfail(ctx, HH_ENOMEM, "hh_rebuild: lists do not fit in device memory");
    }
    cudaFree(ctx->idx);
    ctx->idx = idx;
    ctx->device_bytes += (cap - ctx->cap_list) * int64_t(sizeof(int32_t));
    ctx->cap_list = cap;
    return HH_OK;
}

// bits of a cell key: begin (< 2^b with 2^b > n) above 5 bits of depth
int cell_key_bits(int64_t n)
{
    int bits = 5;
    while (bits < 64 && (int64_t(1) << (bits - 5)) <= n) bits++;
    return bits;
}

}  // namespace

// Called by hh_rebuild when the context builds on the device.
int hh_rebuild_device(hh_ctx *ctx, double t)
{
    int rc = gtree_prepare(ctx);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->n;
    GTreeBuf *g = ctx->gtree;
    // element-wise kernels: a thread per particle at most (they stride over
    // cells, groups and particles alike), so a small tree launches few blocks
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(ctx->elem_grid, (n + 255) / 256)));
    int64_t launches = 0;
    RbSim a = rb_sim(ctx, g, t);
    // Sizes stay on the device (GCounts) and the host reads them three times:
    // after the cells, after groups and cut, and after the list counts.
    auto read_counts = [&]() {
        cudaMemcpyAsync(g->gc_host, g->gc, sizeof(GCounts), cudaMemcpyDeviceToHost, st);
        return cudaStreamSynchronize(st) == cudaSuccess;
    };
    // 1. bounding box, synchronisation check, keys, sort
    k_root_init<false><<<1, 1, 0, st>>>(a, nullptr);
    k_box<false><<<grid, 256, 0, st>>>(a, nullptr);
    k_keys<false><<<grid, 256, 0, st>>>(a, nullptr);
    launches += 3;
    {
        size_t need = 0;
        if (cub::DeviceRadixSort::SortPairs(nullptr, need, g->key, g->key2, g->idx, g->perm, (int)n, 0, 63, st) !=
                cudaSuccess ||
            need == 0)
            return gfail(ctx, HH_ECUDA, "hh_rebuild: key sort size query failed");
        if (need > g->tmp_bytes) {
            if (g->tmp) cudaFree(g->tmp);
            g->tmp = nullptr;
            if (cudaMalloc(&g->tmp, need) != cudaSuccess) return gfail(ctx, HH_ENOMEM, "hh_rebuild: sort buffer");
            g->tmp_bytes = need;
        }
        if (cub::DeviceRadixSort::SortPairs(g->tmp, need, g->key, g->key2, g->idx, g->perm, (int)n, 0, 63, st) !=
            cudaSuccess)
            return gfail(ctx, HH_ECUDA, "hh_rebuild: key sort failed");
    }
    // 2. cells level by level (BFS).  The levels run up to two below the last
    //    tree's depth (the tree changes little in one dt_tree); if the last of
    //    them still made children, the rest follow after the read of the counts.
    const int d_guess = g->depth < 0 ? kMaxDepth : std::min(kMaxDepth, g->depth + 2);
    for (int d = 0; d <= d_guess; d++) k_level<false><<<grid, 256, 0, st>>>(a, nullptr, d);
    k_cells_done<false><<<1, 1, 0, st>>>(a, nullptr, d_guess);
    launches += (d_guess + 1) + 1;
    if (!read_counts()) return gfail(ctx, HH_ECUDA, "hh_rebuild: tree build failed");
    if (!g->gc_host->overflow && g->gc_host->lvl_n[d_guess + 1] > 0) {
        for (int d = d_guess + 1; d <= kMaxDepth; d++) k_level<false><<<grid, 256, 0, st>>>(a, nullptr, d);
        k_cells_done<false><<<1, 1, 0, st>>>(a, nullptr, kMaxDepth);
        launches += (kMaxDepth - d_guess) + 1;
        if (!read_counts()) return gfail(ctx, HH_ECUDA, "hh_rebuild: tree build failed");
    }
    if (g->gc_host->bad) return gfail(ctx, HH_ESTATE, "hh_rebuild: particles are not synchronised at t");
    if (g->gc_host->overflow)
        return gfail(ctx, HH_ENOMEM, "hh_rebuild: tree exceeds nj_max (more cells than room for nodes)");
    const int32_t ncells = g->gc_host->ncells;
    a.ncells = ncells;
    a.S = std::max<int32_t>(32, ncells / 256);
    // the deepest level that holds cells: the moment loop runs from there
    int depth = 0;
    for (int d = 0; d <= kMaxDepth; d++)
        if (g->gc_host->lvl_n[d] > 0) depth = d;
    g->depth = depth;
    // pre-order numbers and subtree sizes from one sort of the cells by
    // (first particle, depth)
    k_cell_keys<false><<<grid, 256, 0, st>>>(a, nullptr);
    if ((rc = cub_sort_pairs(g->tmp, g->tmp_bytes, a.ckey, a.ckey2, a.cval, a.cval2, ncells, cell_key_bits(n), st)))
        return gfail(ctx, rc, "hh_rebuild: cell sort failed");
    k_pre_size<false><<<grid, 256, 0, st>>>(a, nullptr);
    k_to_preorder<false><<<grid, 256, 0, st>>>(a, nullptr);
    // 3. particles into Morton order (into the second buffer), then swap
    k_permute<false><<<grid, 256, 0, st>>>(a, nullptr);
    swap_state(ctx, g);
    a.st = ctx->st;
    a.alt = g->alt;
    a.ids = g->ids;
    a.ids2 = g->ids2;
    // 4. node records (bottom-up moments); groups, and (5.) the cut of
    //    subtrees of <= S cells and the cells above it: flags, one scan,
    //    counts and the three compacted tables; group boxes
    for (int d = depth; d >= 0; d--) k_moments_level<false><<<grid, 256, 0, st>>>(a, nullptr, d);
    k_node_records<false><<<grid, 256, 0, st>>>(a, nullptr);
    k_flags3<false><<<grid, 256, 0, st>>>(a, nullptr);
    if ((rc = cub_exclusive_sum(g->tmp, g->tmp_bytes, g->flag3, g->pos3, 3 * int64_t(ncells), st)))
        return gfail(ctx, rc, "hh_rebuild: scan failed");
    k_counts3<false><<<1, 1, 0, st>>>(a, nullptr);
    k_write3<false><<<grid, 256, 0, st>>>(a, nullptr);
    k_group_box<false><<<grid, 256, 0, st>>>(a, nullptr);
    launches += 6 + (depth + 1) + 6;
    if (!read_counts()) return gfail(ctx, HH_ECUDA, "hh_rebuild: group build failed");
    const int32_t G = g->gc_host->G, R = g->gc_host->R, A = g->gc_host->A;
    if (G > ctx->cap_g) return gfail(ctx, HH_ENOMEM, "hh_rebuild: more groups than groups_max");
    a.G = G;
    a.R = R;
    a.A = A;
    // then per-(group, cut cell) list counts, one scan, offsets, tiles, write
    if (!grow(g->top_buf, g->top_cap, std::max<int64_t>(1, int64_t(G) * A)))
        return gfail(ctx, HH_ENOMEM, "hh_rebuild: list walk table does not fit");
    a.top = g->top_buf;
    if (A > 0) {
        k_top_above<false><<<unsigned((int64_t(G) * A + 127) / 128), 128, 0, st>>>(a, nullptr);
        launches++;
    }
    const int64_t pairs = int64_t(G) * R;
    if (2 * (pairs + 1) >= int64_t(INT32_MAX))  // (one scan covers both count arrays)
        return gfail(ctx, HH_ENOMEM, "hh_rebuild: too many (group, subtree) pairs");
    if (!grow(g->pair_buf, g->pair_cap, 4 * (pairs + 1)))
        return gfail(ctx, HH_ENOMEM, "hh_rebuild: list count buffers do not fit");
    a.pairs = pairs;
    a.pair2 = g->pair_buf;
    a.pscan2 = g->pair_buf + 2 * (pairs + 1);
    const int64_t lgrid = std::min<int64_t>((pairs + 127) / 128, int64_t(1) << 30);
    k_lists_cut<false, false><<<unsigned(lgrid), 128, 0, st>>>(a, nullptr);
    if ((rc = cub_exclusive_sum(g->tmp, g->tmp_bytes, a.pair2, a.pscan2, 2 * (pairs + 1), st)))  // cnt_p, cnt_n at once
        return gfail(ctx, rc, "hh_rebuild: scan failed");
    k_list_off<false><<<grid, 256, 0, st>>>(a, nullptr);
    // 6. tiles and their work-item capacity (from the list lengths)
    k_tile_counts<false><<<grid, 256, 0, st>>>(a, nullptr);
    if ((rc = cub_exclusive_sum(g->tmp, g->tmp_bytes, g->ntile, g->tile_off, 2 * (int64_t(G) + 1), st)))
        return gfail(ctx, rc, "hh_rebuild: scan failed");
    k_store_totals<false><<<1, 1, 0, st>>>(a, nullptr);
    launches += 4;
    if (!read_counts()) return gfail(ctx, HH_ECUDA, "hh_rebuild: list count failed");
    const int64_t L = g->gc_host->L, n_tiles = g->gc_host->n_tiles, total_parts = g->gc_host->total_parts;
    if (n_tiles > ctx->cap_tiles) return gfail(ctx, HH_ENOMEM, "hh_rebuild: too many tiles");
    if ((rc = grow_list(ctx, L))) return rc;
    a.lidx = ctx->idx;
    k_lists_cut<false, true><<<unsigned(lgrid), 128, 0, st>>>(a, nullptr);
    k_tiles<false><<<grid, 256, 0, st>>>(a, nullptr);
    launches += 2;
    const cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return gfail(ctx, HH_ECUDA, cudaGetErrorString(ce));
    hh_count_launches(launches);  // kernels of this file; the radix sort and the scans are CUB's
    ctx->nj = n + ncells;
    ctx->n_groups = G;
    ctx->list_len = L;
    ctx->n_tiles = int32_t(n_tiles);
    ctx->ids_on_device = true;
    return hh_finish_device_rebuild(ctx, total_parts, int64_t(g->gc_host->lmax));
}

// ---------------------------------------------------------------- many at once
// Scratch of the batched rebuild: the simulations' records (one region per
// stage, so that a record is never rewritten while its copy to the device may
// be pending), their counts, the segment offsets of the sorts, and the arrays
// that the sorts and scans run over as one (each simulation a slice).
struct RbScratch {
    cudaStream_t stream = nullptr;
    RbSim *h_sims = nullptr, *d_sims = nullptr;  // [kStages][cap_sims]
    GCounts *h_gc = nullptr, *d_gc = nullptr;     // [cap_sims], by the simulation's slot
    int32_t *h_seg = nullptr, *d_seg = nullptr;   // [2][cap_sims + 1]: particles, cells
    int64_t cap_sims = 0;
    uint64_t *key = nullptr, *key2 = nullptr;
    int32_t *idx = nullptr, *perm = nullptr;
    int64_t cap_key = 0, cap_key2 = 0, cap_idx = 0, cap_perm = 0;
    uint64_t *ckey = nullptr, *ckey2 = nullptr;
    int32_t *cval = nullptr, *cval2 = nullptr;
    int64_t cap_ckey = 0, cap_ckey2 = 0, cap_cval = 0, cap_cval2 = 0;
    int32_t *flag3 = nullptr, *pos3 = nullptr;
    int64_t cap_flag3 = 0, cap_pos3 = 0;
    int64_t *pair2 = nullptr, *pscan2 = nullptr;
    int64_t cap_pair2 = 0, cap_pscan2 = 0;
    int32_t *top = nullptr;
    int64_t cap_top = 0;
    int64_t *nt2 = nullptr, *tscan2 = nullptr;
    int64_t cap_nt2 = 0, cap_tscan2 = 0;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
};

namespace {

constexpr int kStages = 6;  // the records of stages 0..5 (a stage per read of the counts, and the close)

void rb_free_sims(RbScratch *r)
{
    for (void *p : {(void *)r->d_sims, (void *)r->d_gc, (void *)r->d_seg})
        if (p) cudaFree(p);
    for (void *p : {(void *)r->h_sims, (void *)r->h_gc, (void *)r->h_seg})
        if (p) cudaFreeHost(p);
    r->d_sims = r->h_sims = nullptr;
    r->d_gc = r->h_gc = nullptr;
    r->d_seg = r->h_seg = nullptr;
    r->cap_sims = 0;
}

bool rb_reserve_sims(RbScratch *r, int64_t k)
{
    if (k <= r->cap_sims) return true;
    rb_free_sims(r);
    const int64_t cap = k + k / 2 + 8;
    if (cudaMalloc(&r->d_sims, sizeof(RbSim) * kStages * cap) != cudaSuccess ||
        cudaMalloc(&r->d_gc, sizeof(GCounts) * cap) != cudaSuccess ||
        cudaMalloc(&r->d_seg, sizeof(int32_t) * 2 * (cap + 1)) != cudaSuccess ||
        cudaHostAlloc((void **)&r->h_sims, sizeof(RbSim) * kStages * cap, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&r->h_gc, sizeof(GCounts) * cap, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&r->h_seg, sizeof(int32_t) * 2 * (cap + 1), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        rb_free_sims(r);
        return false;
    }
    r->cap_sims = cap;
    return true;
}

// grows a scratch array (a quarter beyond the need)
template <typename T>
bool rb_grow(T *&p, int64_t &cap, int64_t need)
{
    return need <= cap || grow(p, cap, need + need / 4 + 1024);
}

template <typename K, typename V>
int rb_seg_sort(RbScratch *r, const K *kin, K *kout, const V *vin, V *vout, int64_t n, int k, const int32_t *seg,
                int bits)
{
    size_t need = 0;
    if (cub::DeviceSegmentedRadixSort::SortPairs(nullptr, need, kin, kout, vin, vout, (int)n, k, seg, seg + 1, 0, bits,
                                                  r->stream) != cudaSuccess)
        return HH_ECUDA;
    if (need > r->tmp_bytes) {
        if (r->tmp) cudaFree(r->tmp);
        r->tmp = nullptr;
        r->tmp_bytes = 0;
        if (cudaMalloc(&r->tmp, need) != cudaSuccess) {
            cudaGetLastError();
            return HH_ENOMEM;
        }
        r->tmp_bytes = need;
    }
    return cub::DeviceSegmentedRadixSort::SortPairs(r->tmp, need, kin, kout, vin, vout, (int)n, k, seg, seg + 1, 0,
                                                     bits, r->stream) == cudaSuccess
               ? HH_OK
               : HH_ECUDA;
}

}  // namespace

RbScratch *hh_rb_scratch_create()
{
    RbScratch *r = new RbScratch;
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        return nullptr;
    }
    return r;
}

void hh_rb_scratch_free(RbScratch *r)
{
    if (!r) return;
    cudaStreamSynchronize(r->stream);
    rb_free_sims(r);
    for (void *p : {(void *)r->key, (void *)r->key2, (void *)r->idx, (void *)r->perm, (void *)r->ckey,
                    (void *)r->ckey2, (void *)r->cval, (void *)r->cval2, (void *)r->flag3, (void *)r->pos3,
                    (void *)r->pair2, (void *)r->pscan2, (void *)r->top, (void *)r->nt2, (void *)r->tscan2, r->tmp})
        if (p) cudaFree(p);
    cudaStreamDestroy(r->stream);
    delete r;
}

// Rebuilds k contexts on the device at once: every step of hh_rebuild_device
// runs as one launch over all of them (simulation = blockIdx.y), the key and
// cell sorts as segmented sorts and each scan as one scan over all
// simulations' arrays (a simulation reads its slice relative to its first
// entry).  Each context gets the tree, groups, lists and node records it
// would get alone.  rcs[s] receives context s's result; a context that fails
// leaves the build at that point and the others go on.
int hh_rebuild_device_many(hh_ctx *const *ctxs, const double *ts, int k, int *rcs, RbScratch *r)
{
    if (k < 1 || !r) return HH_EINVAL;
    cudaStream_t st = r->stream;
    if (!rb_reserve_sims(r, k)) return HH_ENOMEM;
    std::vector<int> act, slot;  // contexts still in the build, and their count slots
    for (int s = 0; s < k; s++) {
        rcs[s] = gtree_prepare(ctxs[s]);
        if (rcs[s] == HH_OK && cudaStreamSynchronize(ctxs[s]->stream) != cudaSuccess)
            rcs[s] = gfail(ctxs[s], HH_ECUDA, "hh_rebuild: context stream failed");
        if (rcs[s] == HH_OK) act.push_back(s);
    }
    if (act.empty()) return HH_OK;
    const int K0 = int(act.size());
    int stage = 0;
    auto H = [&](int q) -> RbSim & { return r->h_sims[stage * r->cap_sims + q]; };
    auto D = [&]() { return r->d_sims + stage * r->cap_sims; };
    auto upload = [&]() {
        return cudaMemcpyAsync(D(), &H(0), sizeof(RbSim) * act.size(), cudaMemcpyHostToDevice, st) == cudaSuccess;
    };
    auto read_counts = [&]() {
        return cudaMemcpyAsync(r->h_gc, r->d_gc, sizeof(GCounts) * K0, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
               cudaStreamSynchronize(st) == cudaSuccess;
    };
    auto cnt = [&](size_t q) -> const GCounts & { return r->h_gc[slot[q]]; };
    // the next stage's records: those of the contexts for which keep(q) holds
    auto next_stage = [&](const std::function<bool(size_t)> &keep) {
        size_t w = 0;
        RbSim *src = r->h_sims + stage * r->cap_sims, *dst = r->h_sims + (stage + 1) * r->cap_sims;
        for (size_t q = 0; q < act.size(); q++)
            if (keep(q)) {
                dst[w] = src[q];
                act[w] = act[q];
                slot[w++] = slot[q];
            }
        act.resize(w);
        slot.resize(w);
        stage++;
    };
    auto fail_all = [&](int code, const char *m) {
        for (int s : act) rcs[s] = gfail(ctxs[s], code, m);
        act.clear();
        return HH_OK;
    };
    // exclusive prefix of per-context sizes into segment offsets `which`
    auto segments = [&](int which, const std::function<int64_t(size_t)> &size, int64_t *total) {
        int32_t *h = r->h_seg + which * (r->cap_sims + 1);
        int64_t acc = 0;
        for (size_t q = 0; q < act.size(); q++) {
            h[q] = int32_t(acc);
            acc += size(q);
            if (acc >= int64_t(INT32_MAX)) return false;
        }
        h[act.size()] = int32_t(acc);
        *total = acc;
        return cudaMemcpyAsync(r->d_seg + which * (r->cap_sims + 1), h, sizeof(int32_t) * (act.size() + 1),
                               cudaMemcpyHostToDevice, st) == cudaSuccess;
    };
    // blocks per simulation of the element-wise kernels (they stride over
    // cells, groups and particles alike): a thread per particle of the
    // largest one, but no more than about twice the threads the SMs hold in
    // all, since a level or a moment pass has little work for most blocks
    int64_t launches = 0, gx = 1, max_n = 1;
    for (int s : act) {
        gx = std::max<int64_t>(gx, std::min<int64_t>(ctxs[s]->elem_grid, (ctxs[s]->n + 255) / 256));
        max_n = std::max<int64_t>(max_n, ctxs[s]->n);
    }
    const int64_t gx_full = gx;  // (the group boxes, a warp per group, take every block)
    gx = std::max<int64_t>(1, std::min<int64_t>(gx, 2 * int64_t(ctxs[act[0]]->elem_grid) / int64_t(act.size())));
    // 1. bounding boxes, keys, one segmented key sort, levels, counts
    int64_t tot = 0;
    if (!segments(0, [&](size_t q) { return ctxs[act[q]]->n; }, &tot))
        return fail_all(HH_ENOMEM, "hh_rebuild: batch too large");
    if (!rb_grow(r->key, r->cap_key, tot) || !rb_grow(r->key2, r->cap_key2, tot) || !rb_grow(r->idx, r->cap_idx, tot) ||
        !rb_grow(r->perm, r->cap_perm, tot))
        return fail_all(HH_ENOMEM, "hh_rebuild: batch key buffers do not fit");
    int d_guess = 0;
    for (size_t q = 0; q < act.size(); q++) {
        hh_ctx *ctx = ctxs[act[q]];
        GTreeBuf *g = ctx->gtree;
        RbSim &a = H(int(q));
        a = rb_sim(ctx, g, ts[act[q]]);
        const int64_t o = r->h_seg[q];
        a.gc = r->d_gc + q;
        a.key = r->key + o;
        a.key2 = r->key2 + o;
        a.idx = r->idx + o;
        a.perm = r->perm + o;
        slot.push_back(int(q));
        d_guess = std::max(d_guess, g->depth < 0 ? kMaxDepth : std::min(kMaxDepth, g->depth + 2));
    }
    if (!upload()) return fail_all(HH_ECUDA, "hh_rebuild: batch upload failed");
    const dim3 g1 = dim3(unsigned(gx), unsigned(K0)), one1(1, unsigned(K0));
    k_root_init<true><<<one1, 1, 0, st>>>(RbSim{}, D());
    k_box<true><<<g1, 256, 0, st>>>(RbSim{}, D());
    k_keys<true><<<g1, 256, 0, st>>>(RbSim{}, D());
    launches += 3;
    int rc = rb_seg_sort(r, r->key, r->key2, r->idx, r->perm, tot, K0, r->d_seg, 63);
    if (rc) return fail_all(rc, "hh_rebuild: batch key sort failed");
    for (int d = 0; d <= d_guess; d++) k_level<true><<<g1, 256, 0, st>>>(RbSim{}, D(), d);
    k_cells_done<true><<<one1, 1, 0, st>>>(RbSim{}, D(), d_guess);
    launches += (d_guess + 1) + 1;
    if (!read_counts()) return fail_all(HH_ECUDA, "hh_rebuild: tree build failed");
    bool deeper = false;
    for (size_t q = 0; q < act.size(); q++) deeper |= !cnt(q).overflow && cnt(q).lvl_n[d_guess + 1] > 0;
    if (deeper) {  // (a context that is complete gains empty levels)
        for (int d = d_guess + 1; d <= kMaxDepth; d++) k_level<true><<<g1, 256, 0, st>>>(RbSim{}, D(), d);
        k_cells_done<true><<<one1, 1, 0, st>>>(RbSim{}, D(), kMaxDepth);
        launches += (kMaxDepth - d_guess) + 1;
        if (!read_counts()) return fail_all(HH_ECUDA, "hh_rebuild: tree build failed");
    }
    next_stage([&](size_t q) {
        if (cnt(q).bad) {
            rcs[act[q]] = gfail(ctxs[act[q]], HH_ESTATE, "hh_rebuild: particles are not synchronised at t");
            return false;
        }
        if (cnt(q).overflow) {
            rcs[act[q]] =
                gfail(ctxs[act[q]], HH_ENOMEM, "hh_rebuild: tree exceeds nj_max (more cells than room for nodes)");
            return false;
        }
        return true;
    });
    if (act.empty()) return HH_OK;
    // 2. one segmented cell sort, pre-order, reordering, moments, node
    //    records, the three selections (one scan), group boxes
    int64_t tcells = 0;
    if (!segments(1, [&](size_t q) { return int64_t(cnt(q).ncells); }, &tcells))
        return fail_all(HH_ENOMEM, "hh_rebuild: batch too large");
    if (!rb_grow(r->ckey, r->cap_ckey, tcells) || !rb_grow(r->ckey2, r->cap_ckey2, tcells) ||
        !rb_grow(r->cval, r->cap_cval, tcells) || !rb_grow(r->cval2, r->cap_cval2, tcells) ||
        !rb_grow(r->flag3, r->cap_flag3, 3 * tcells) || !rb_grow(r->pos3, r->cap_pos3, 3 * tcells))
        return fail_all(HH_ENOMEM, "hh_rebuild: batch cell buffers do not fit");
    const int32_t *hs1 = r->h_seg + (r->cap_sims + 1);
    int depth = 0;
    for (size_t q = 0; q < act.size(); q++) {
        RbSim &a = H(int(q));
        GTreeBuf *g = ctxs[act[q]]->gtree;
        a.ncells = cnt(q).ncells;
        a.S = std::max<int32_t>(32, a.ncells / 256);
        int dq = 0;
        for (int d = 0; d <= kMaxDepth; d++)
            if (cnt(q).lvl_n[d] > 0) dq = d;
        g->depth = dq;
        depth = std::max(depth, dq);
        const int64_t o = hs1[q];
        a.ckey = r->ckey + o;
        a.ckey2 = r->ckey2 + o;
        a.cval = r->cval + o;
        a.cval2 = r->cval2 + o;
        a.flag3 = r->flag3 + 3 * o;
        a.pos3 = r->pos3 + 3 * o;
    }
    const int K2 = int(act.size());
    const dim3 g2 = dim3(unsigned(gx), unsigned(K2)), one2(1, unsigned(K2));
    if (!upload()) return fail_all(HH_ECUDA, "hh_rebuild: batch upload failed");
    k_cell_keys<true><<<g2, 256, 0, st>>>(RbSim{}, D());
    if ((rc = rb_seg_sort(r, r->ckey, r->ckey2, r->cval, r->cval2, tcells, K2, r->d_seg + (r->cap_sims + 1),
                          cell_key_bits(max_n))))
        return fail_all(rc, "hh_rebuild: batch cell sort failed");
    k_pre_size<true><<<g2, 256, 0, st>>>(RbSim{}, D());
    k_to_preorder<true><<<g2, 256, 0, st>>>(RbSim{}, D());
    k_permute<true><<<g2, 256, 0, st>>>(RbSim{}, D());
    next_stage([](size_t) { return true; });
    for (size_t q = 0; q < act.size(); q++) {  // the reordered state becomes the context's
        hh_ctx *ctx = ctxs[act[q]];
        GTreeBuf *g = ctx->gtree;
        swap_state(ctx, g);
        RbSim &a = H(int(q));
        a.st = ctx->st;
        a.alt = g->alt;
        a.ids = g->ids;
        a.ids2 = g->ids2;
    }
    if (!upload()) return fail_all(HH_ECUDA, "hh_rebuild: batch upload failed");
    for (int d = depth; d >= 0; d--) k_moments_level<true><<<g2, 256, 0, st>>>(RbSim{}, D(), d);
    k_node_records<true><<<g2, 256, 0, st>>>(RbSim{}, D());
    k_flags3<true><<<g2, 256, 0, st>>>(RbSim{}, D());
    if ((rc = cub_exclusive_sum(r->tmp, r->tmp_bytes, r->flag3, r->pos3, 3 * tcells, st)))
        return fail_all(rc, "hh_rebuild: batch scan failed");
    k_counts3<true><<<one2, 1, 0, st>>>(RbSim{}, D());
    k_write3<true><<<g2, 256, 0, st>>>(RbSim{}, D());
    k_group_box<true><<<dim3(unsigned(gx_full), unsigned(K2)), 256, 0, st>>>(RbSim{}, D());
    launches += 6 + (depth + 1) + 6;
    if (!read_counts()) return fail_all(HH_ECUDA, "hh_rebuild: group build failed");
    next_stage([&](size_t q) {
        if (cnt(q).G > ctxs[act[q]]->cap_g) {
            rcs[act[q]] = gfail(ctxs[act[q]], HH_ENOMEM, "hh_rebuild: more groups than groups_max");
            return false;
        }
        return true;
    });
    if (act.empty()) return HH_OK;
    // 3. per-(group, cut cell) list counts (one scan), offsets, tiles (one scan)
    int64_t t_top = 0, t_pair = 0, t_nt = 0, tgrid = 1, lgrid = 1;
    for (size_t q = 0; q < act.size(); q++) {
        RbSim &a = H(int(q));
        a.G = cnt(q).G;
        a.R = cnt(q).R;
        a.A = cnt(q).A;
        a.pairs = int64_t(a.G) * a.R;
        a.top = reinterpret_cast<int32_t *>(t_top);  // offsets for now
        a.pair2 = reinterpret_cast<int64_t *>(t_pair);
        a.nt2 = reinterpret_cast<int64_t *>(t_nt);
        t_top += std::max<int64_t>(1, int64_t(a.G) * a.A);
        t_pair += 2 * (a.pairs + 1);
        t_nt += 2 * (int64_t(a.G) + 1);
        tgrid = std::max<int64_t>(tgrid, (int64_t(a.G) * a.A + 127) / 128);
        lgrid = std::max<int64_t>(lgrid, (a.pairs + 127) / 128);
    }
    if (t_pair >= int64_t(INT32_MAX) || t_nt >= int64_t(INT32_MAX))  // (one CUB scan each)
        return fail_all(HH_ENOMEM, "hh_rebuild: too many (group, subtree) pairs in one batch");
    if (!rb_grow(r->top, r->cap_top, t_top) || !rb_grow(r->pair2, r->cap_pair2, t_pair) ||
        !rb_grow(r->pscan2, r->cap_pscan2, t_pair) || !rb_grow(r->nt2, r->cap_nt2, t_nt) ||
        !rb_grow(r->tscan2, r->cap_tscan2, t_nt))
        return fail_all(HH_ENOMEM, "hh_rebuild: batch list buffers do not fit");
    for (size_t q = 0; q < act.size(); q++) {
        RbSim &a = H(int(q));
        const int64_t o_top = reinterpret_cast<int64_t>(a.top), o_pair = reinterpret_cast<int64_t>(a.pair2),
                      o_nt = reinterpret_cast<int64_t>(a.nt2);
        a.top = r->top + o_top;
        a.pair2 = r->pair2 + o_pair;
        a.pscan2 = r->pscan2 + o_pair;
        a.nt2 = r->nt2 + o_nt;
        a.tscan2 = r->tscan2 + o_nt;
    }
    const int K3 = int(act.size());
    const dim3 g3 = dim3(unsigned(gx), unsigned(K3)), one3(1, unsigned(K3));
    const dim3 lg3(unsigned(std::min<int64_t>(lgrid, int64_t(1) << 30)), unsigned(K3));
    if (!upload()) return fail_all(HH_ECUDA, "hh_rebuild: batch upload failed");
    k_top_above<true><<<dim3(unsigned(std::min<int64_t>(tgrid, int64_t(1) << 30)), unsigned(K3)), 128, 0, st>>>(
        RbSim{}, D());
    k_lists_cut<true, false><<<lg3, 128, 0, st>>>(RbSim{}, D());
    if ((rc = cub_exclusive_sum(r->tmp, r->tmp_bytes, r->pair2, r->pscan2, t_pair, st)))
        return fail_all(rc, "hh_rebuild: batch scan failed");
    k_list_off<true><<<g3, 256, 0, st>>>(RbSim{}, D());
    k_tile_counts<true><<<g3, 256, 0, st>>>(RbSim{}, D());
    if ((rc = cub_exclusive_sum(r->tmp, r->tmp_bytes, r->nt2, r->tscan2, t_nt, st)))
        return fail_all(rc, "hh_rebuild: batch scan failed");
    k_store_totals<true><<<one3, 1, 0, st>>>(RbSim{}, D());
    launches += 5;
    if (!read_counts()) return fail_all(HH_ECUDA, "hh_rebuild: list count failed");
    next_stage([&](size_t q) {
        hh_ctx *ctx = ctxs[act[q]];
        if (cnt(q).n_tiles > ctx->cap_tiles) {
            rcs[act[q]] = gfail(ctx, HH_ENOMEM, "hh_rebuild: too many tiles");
            return false;
        }
        if ((rcs[act[q]] = grow_list(ctx, cnt(q).L)) != HH_OK) return false;
        return true;
    });
    if (act.empty()) return HH_OK;
    // 4. lists and tiles
    for (size_t q = 0; q < act.size(); q++) H(int(q)).lidx = ctxs[act[q]]->idx;
    const int K4 = int(act.size());
    const dim3 g4 = dim3(unsigned(gx), unsigned(K4));
    const dim3 lg4(unsigned(std::min<int64_t>(lgrid, int64_t(1) << 30)), unsigned(K4));
    if (!upload()) return fail_all(HH_ECUDA, "hh_rebuild: batch upload failed");
    k_lists_cut<true, true><<<lg4, 128, 0, st>>>(RbSim{}, D());
    k_tiles<true><<<g4, 256, 0, st>>>(RbSim{}, D());
    launches += 2;
    const cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail_all(HH_ECUDA, cudaGetErrorString(ce));
    // 5. per context on the host: work-item capacity and sizes; then one
    //    closing kernel over those that got them
    next_stage([&](size_t q) {
        hh_ctx *ctx = ctxs[act[q]];
        const GCounts &c = cnt(q);
        ctx->nj = ctx->n + c.ncells;
        ctx->n_groups = c.G;
        ctx->list_len = c.L;
        ctx->n_tiles = int32_t(c.n_tiles);
        ctx->ids_on_device = true;
        rcs[act[q]] = hh_finish_device_rebuild(ctx, c.total_parts, int64_t(c.lmax), true);
        return rcs[act[q]] == HH_OK;
    });
    if (!act.empty()) {
        int64_t fx = 1;
        for (int s : act) fx = std::max<int64_t>(fx, std::min<int64_t>(ctxs[s]->elem_grid, (ctxs[s]->nj + 255) / 256));
        if (!upload()) return fail_all(HH_ECUDA, "hh_rebuild: batch upload failed");
        k_finish<true><<<dim3(unsigned(fx), unsigned(act.size())), 256, 0, st>>>(RbSim{}, D());
        launches++;
    }
    hh_count_launches(launches);  // kernels of this file; the sorts and scans are CUB's
    const cudaError_t ce2 = cudaGetLastError();
    if (ce2 != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        for (int s : act) ctxs[s]->have_lists = false;
        return fail_all(HH_ECUDA, "hh_rebuild: batch build failed");
    }
    return HH_OK;
}
