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
#include <vector>

#include <cub/device/device_radix_sort.cuh>
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

// ------------------------------------------------------------ kernels
__global__ void k_box(const State s, int64_t n, double t_tree, Box *b)
{
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int d = 0; d < 3; d++) {
            const unsigned long long o = order_bits(s.x[d * s.cap_j + i]);
            lo[d] = o < lo[d] ? o : lo[d];
            hi[d] = o > hi[d] ? o : hi[d];
        }
        bad |= s.t[i] != t_tree;
    }
    for (int d = 0; d < 3; d++) {
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo[d], off);
            const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi[d], off);
            lo[d] = l2 < lo[d] ? l2 : lo[d];
            hi[d] = h2 > hi[d] ? h2 : hi[d];
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&b->lo[d], lo[d]);
            atomicMax(&b->hi[d], hi[d]);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(&b->bad, 1);
}

__global__ void k_keys(const State s, int64_t n, const Box *b, uint64_t *key, int32_t *idx, double *root_side,
                       float *xmax, int order)
{
    double lo[3], side = 0.0;
    for (int d = 0; d < 3; d++) {
        lo[d] = from_order_bits(b->lo[d]);
        const double ext = from_order_bits(b->hi[d]) - lo[d];
        if (ext > side) side = ext;
    }
    if (side == 0.0) side = 1.0;
    const double scale = double(1u << kBits) / side;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *root_side = side;
        double xm = 0.0;  // bound on |coordinate| of every particle, node and group box
        for (int d = 0; d < 3; d++) xm = fmax(xm, fmax(fabs(lo[d]), fabs(from_order_bits(b->hi[d]))));
        *xmax = float(xm) * 1.0001f;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t u[3];
        for (int d = 0; d < 3; d++) {
            double f = floor((s.x[d * s.cap_j + i] - lo[d]) * scale);
            f = f < 0.0 ? 0.0 : f;
            f = f > double((1u << kBits) - 1u) ? double((1u << kBits) - 1u) : f;
            u[d] = uint32_t(f);
        }
        key[i] = order == HH_ORDER_HILBERT ? hilbert_key(u[0], u[1], u[2])
                                           : (spread_bits(u[0]) << 2) | (spread_bits(u[1]) << 1) | spread_bits(u[2]);
        idx[i] = int32_t(i);
    }
}

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

__global__ void k_root_init(Cells C, int32_t n, GCounts *gc, Box *b)
{
    for (int d = 0; d < 3; d++) {  // empty bounding box
        b->lo[d] = ~0ull;
        b->hi[d] = 0ull;
    }
    b->bad = 0;
    C.begin[0] = 0;
    C.end[0] = n;
    C.depth[0] = 0;
    C.parent[0] = -1;
    C.pre[0] = 0;
    for (int d = 0; d < kMaxDepth + 2; d++) gc->lvl_c0[d] = gc->lvl_n[d] = 0;
    gc->lvl_n[0] = 1;
    gc->ncells = gc->overflow = gc->bad = gc->G = gc->R = gc->A = 0;
    gc->lmax = 0ull;
}

// Splits the cells of level d that hold more than `leaf` particles (and are
// above the depth limit): the octant boundaries come from binary searches of
// the sorted keys, and each cell reserves its block of children in level d+1.
__global__ void k_level(Cells C, const uint64_t *key, int d, int leaf, GCounts *gc, int32_t cap_cells)
{
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
            split = e - b > leaf && d < kMaxDepth;
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
        if ((int64_t)w + nch > cap_cells) {
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

// Pre-order numbers and subtree sizes without a pass per level: the cells
// sorted by (first particle, depth) are in pre-order (children follow their
// parent in octant order, which is particle order, and a cell's descendants
// are the cells after it that start before it ends).  Key of a cell:
// begin << 5 | depth (depth <= kMaxDepth < 32).
__global__ void k_cell_keys(Cells C, int32_t ncells, uint64_t *key, int32_t *val)
{
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        key[c] = (uint64_t(C.begin[c]) << 5) | uint64_t(C.depth[c]);
        val[c] = c;
    }
}

// From the sorted keys and cells: pre[c] = its rank; size[c] = the cells from
// it to the first one that starts at or after its end.
__global__ void k_pre_size(Cells C, int32_t ncells, const uint64_t *skey, const int32_t *sval)
{
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < ncells; p += gridDim.x * blockDim.x) {
        const int32_t c = sval[p];
        C.pre[c] = p;
        const uint64_t lim = uint64_t(C.end[c]) << 5;
        int32_t lo = p + 1, hi = ncells;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (skey[mid] < lim) lo = mid + 1;
            else hi = mid;
        }
        C.size[c] = lo - p;
    }
}

// cell count, and the synchronisation flag of the bounding-box pass
// After the levels 0..d: the cells made so far (complete when level d made
// no children, i.e. lvl_n[d + 1] == 0).
__global__ void k_cells_done(GCounts *gc, const Box *b, int d)
{
    gc->ncells = gc->lvl_c0[d + 1] + gc->lvl_n[d + 1];
    gc->bad = b->bad;
}

// Pre-order cell table used by the group and list kernels.
struct PCells {
    int32_t *begin, *end, *nchild, *parent;
    int32_t *size;   // cells in the subtree: the subtree of p is [p, p + size)
    int4 *pack;      // {begin, end, nchild, size}: what the list walk reads per cell
    float4 *cf;      // {centre of mass x, y, z, side} rounded to FP32 (screening)
    int32_t *child;  // [8 * n]
    double *side;
};

__global__ void k_to_preorder(Cells C, int32_t ncells, PCells P, const double *root_side)
{
    const double s0 = *root_side;
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
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

// State of the reordered particles: new[k] = old[perm[k]] (Morton order).
__global__ void k_permute(const State src, State dst, const int32_t *perm, int64_t n, const int64_t *ids_src,
                          int64_t *ids_dst)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm[k];
        for (int d = 0; d < 3; d++) {
            dst.x[d * dst.cap_j + k] = src.x[d * src.cap_j + i];
            dst.v[d * dst.cap_j + k] = src.v[d * src.cap_j + i];
            dst.a[d * dst.cap_j + k] = src.a[d * src.cap_j + i];
            dst.jk[d * dst.cap_j + k] = src.jk[d * src.cap_j + i];
        }
        dst.m[k] = src.m[i];
        dst.t[k] = src.t[i];
        dst.dt[k] = src.dt[i];
        ids_dst[k] = ids_src[i];
    }
}

// Node records (pseudo-particles): mass and mass-weighted sums of x, v, a, jk
// of the members, bottom-up one tree level per launch: a leaf sums its
// particles, an inner cell the sums of its children.  mom is [13][cap] in BFS
// cell order.
__global__ void k_moments_level(const State s, Cells C, const GCounts *gc, int d, int64_t cap, double *mom)
{
    if (gc->overflow) return;
    const int32_t c0 = gc->lvl_c0[d], nc = gc->lvl_n[d];
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
__global__ void k_node_records(State s, Cells C, PCells P, int32_t ncells, int64_t cap, const double *mom, int64_t n,
                               double t_tree)
{
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        const int32_t p = C.pre[c];
        const int64_t j = n + p;
        const double M = mom[c];
        s.m[j] = M;
        s.t[j] = t_tree;
        double x[3];
        for (int d = 0; d < 3; d++) {
            x[d] = mom[(1 + d) * cap + c] / M;
            s.x[d * s.cap_j + j] = x[d];
            s.v[d * s.cap_j + j] = mom[(4 + d) * cap + c] / M;
            s.a[d * s.cap_j + j] = mom[(7 + d) * cap + c] / M;
            s.jk[d * s.cap_j + j] = mom[(10 + d) * cap + c] / M;
        }
        P.cf[p] = make_float4(float(x[0]), float(x[1]), float(x[2]), float(P.side[p]));
    }
}

// Bounding box of each group's particles ([3][G] lo and hi), one warp per group
// (none beyond cap_g groups: the host then reports the overflow).
__global__ void k_group_box(const State s, PCells P, const GCounts *gc, int32_t cap_g, const int32_t *g_cell,
                            double *box_lo, double *box_hi, float4 *box_f)
{
    const int32_t G = gc->G;
    if (G > cap_g) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = w0; g < G; g += nw) {
        const int32_t c = g_cell[g], b = P.begin[c], e = P.end[c];
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
                box_lo[d * G + g] = lo;
                box_hi[d * G + g] = hi;
            }
        }
        if (lane == 0) {
            box_f[2 * g] = make_float4(float(box_lo[g]), float(box_lo[G + g]), float(box_lo[2 * G + g]), 0.f);
            box_f[2 * g + 1] = make_float4(float(box_hi[g]), float(box_hi[G + g]), float(box_hi[2 * G + g]), 0.f);
        }
    }
}

// Groups (Barnes 1990): maximal cells with <= n_crit particles (or leaves).
// Cut through the tree: the maximal cells whose subtree holds <= S cells.
// They partition the cells at or below the cut; every cell above it is an
// ancestor of some cut cell.  All three in pre-order (k_flags3 below).

// list length and tile / work-item totals, from the ends of their scans
// parts_scan: the second half of the one scan over [tile counts, part
// counts], so its values are offset by its first entry (the tile total)
__global__ void k_store_totals(GCounts *gc, const int64_t *off_end, const int64_t *tiles_end, const int64_t *parts_scan,
                               int32_t G)
{
    gc->L = *off_end;
    gc->n_tiles = *tiles_end;
    gc->total_parts = parts_scan[G] - parts_scan[0];
}

// The three cell selections at once: flags [groups | cut cells | cells above
// the cut], each ncells long, compacted by one exclusive scan (positions of
// the second and third selections are offset by the counts before them).
__global__ void k_flags3(PCells P, int32_t ncells, int n_crit, int32_t S, int32_t *flag)
{
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        const int32_t cnt = P.end[c] - P.begin[c];
        const bool small = cnt <= n_crit || P.nchild[c] == 0;
        const int32_t par = P.parent[c];
        const bool parent_big = par < 0 || !((P.end[par] - P.begin[par]) <= n_crit || P.nchild[par] == 0);
        flag[c] = (small && parent_big) ? 1 : 0;                                         // group (Barnes 1990)
        flag[ncells + c] = (P.size[c] <= S && (par < 0 || P.size[par] > S)) ? 1 : 0;     // cut cell
        flag[2 * ncells + c] = P.size[c] > S ? 1 : 0;                                    // above the cut
    }
}

__global__ void k_counts3(GCounts *gc, const int32_t *flag, const int32_t *pos, int32_t ncells)
{
    gc->G = pos[ncells];
    gc->R = pos[2 * ncells] - pos[ncells];
    gc->A = pos[3 * ncells - 1] + flag[3 * ncells - 1] - pos[2 * ncells];
}

// groups (g_cell, group_of), cut cells and cells above the cut, in pre-order
// (group cells beyond cap_g are not stored: the host reports the overflow)
__global__ void k_write3(PCells P, int32_t ncells, const int32_t *flag, const int32_t *pos, int32_t *g_cell,
                         int32_t cap_g, int32_t *group_of, int32_t *cut, int32_t *above)
{
    const int32_t r0 = pos[ncells], a0 = pos[2 * ncells];
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        if (flag[c]) {
            const int32_t g = pos[c];
            if (g < cap_g) g_cell[g] = c;
            for (int32_t p = P.begin[c]; p < P.end[c]; p++) group_of[p] = g;
        }
        if (flag[ncells + c]) cut[pos[ncells + c] - r0] = c;
        if (flag[2 * ncells + c]) above[pos[2 * ncells + c] - a0] = c;
    }
}

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
    pk = P.pack[c];
    if (c == G.gc) return kEmitParticles;
    if (pk.x <= G.gb && G.ge <= pk.y) return kOpen;
    if (pk.y - pk.x == 1) return kEmitParticles;
    const float4 cf = P.cf[c];
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

// What the list walk kernels read: the pre-order cells, the node records,
// the groups and their boxes, the opening angle and the FP32 screen's
// absolute margin (2^-19 theta X).
struct WalkArgs {
    State s;
    PCells P;
    int64_t n;
    int32_t G;
    const int32_t *g_cell;
    const double *box_lo, *box_hi;
    const float4 *box_f;
    double theta;
    float theta_f;
    const float *xmax;
};

__device__ __forceinline__ GroupView group_view(const WalkArgs &W, int32_t g)
{
    GroupView V;
    V.gc = W.g_cell[g];
    V.gb = W.P.begin[V.gc];
    V.ge = W.P.end[V.gc];
    for (int d = 0; d < 3; d++) {
        V.lo[d] = W.box_lo[d * W.G + g];
        V.hi[d] = W.box_hi[d * W.G + g];
    }
    const float4 l = W.box_f[2 * g], h = W.box_f[2 * g + 1];
    V.lof = make_float3(l.x, l.y, l.z);
    V.hif = make_float3(h.x, h.y, h.z);
    return V;
}

__device__ __forceinline__ float walk_tol(const WalkArgs &W) { return 0x1p-19f * W.theta_f * *W.xmax; }

// For every (group g, cell above the cut a = above[i]): the topmost cell on
// the path root -> a that the walk of g does not open (-1: all opened).
// Cells above the cut are few; this replaces a walk up the tree per
// (group, cut cell) pair by one table lookup.
__global__ void k_top_above(const WalkArgs W, const int32_t *above, int32_t A, int32_t *top_above)
{
    const float tol = walk_tol(W);
    const int64_t total = int64_t(W.G) * A;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = int32_t(q / A), i = int32_t(q - int64_t(g) * A);
        const GroupView V = group_view(W, g);
        int32_t top = -1;
        int4 pk;
        for (int32_t a = above[i]; a >= 0; a = W.P.parent[a])
            if (decide(W.s, W.P, W.n, W.theta, W.theta_f, tol, V, a, pk) != kOpen) top = a;
        top_above[q] = top;
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
// cnt_p's terminal entry, so one exclusive scan covers both: scan_n's values
// are then offset by scan_n[0], the particle total.
template <bool kWrite>
__global__ void k_lists_cut(const WalkArgs W, const int32_t *cut, int32_t R, const int32_t *above_pos,
                            const int32_t *top_above, int32_t A, int64_t *cnt_p, int64_t *cnt_n,
                            const int64_t *scan_p, const int64_t *scan_n, int32_t *idx)
{
    const float tol = walk_tol(W);
    const int64_t total = int64_t(W.G) * R;
    const int64_t n = W.n;
    if (!kWrite && blockIdx.x == 0 && threadIdx.x == 0) cnt_p[total] = cnt_n[total] = 0;
    const int64_t nb = kWrite ? scan_n[0] : 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = int32_t(q / R), k = int32_t(q - int64_t(g) * R);
        const int32_t r = cut[k], par = W.P.parent[r];
        int32_t top = par >= 0 ? top_above[int64_t(g) * A + (above_pos[par] - above_pos[0])] : -1;
        if (top >= 0 && k > 0 && cut[k - 1] >= top) {  // emitted by an earlier cut cell
            if (!kWrite) cnt_p[q] = cnt_n[q] = 0;
            continue;
        }
        const GroupView V = group_view(W, g);
        int64_t wp = 0, wn = 0;
        if (kWrite) {
            wp = scan_p[q] + (scan_n[int64_t(g) * R] - nb);
            wn = scan_p[int64_t(g + 1) * R] + (scan_n[q] - nb);
        }
        int64_t np = 0, nn = 0;
        int4 pk;
        int top_dec;
        if (top >= 0) {
            top_dec = decide(W.s, W.P, n, W.theta, W.theta_f, tol, V, top, pk);
        } else {
            top_dec = decide(W.s, W.P, n, W.theta, W.theta_f, tol, V, r, pk);
            if (top_dec != kOpen) top = r;
        }
        if (top >= 0) {
            if (top_dec == kEmitNode) {
                if (kWrite) idx[wn] = int32_t(n + top);
                nn = 1;
            } else {
                if (kWrite)
                    for (int32_t p = pk.x; p < pk.y; p++) idx[wp++] = p;
                np = pk.y - pk.x;
            }
        } else {
            const int32_t end = r + pk.w;
            int32_t c = r + 1;
            while (c < end) {
                const int dec = decide(W.s, W.P, n, W.theta, W.theta_f, tol, V, c, pk);
                if (dec == kOpen) {
                    c++;
                    continue;
                }
                if (dec == kEmitNode) {
                    if (kWrite) idx[wn++] = int32_t(n + c);
                    nn++;
                } else {
                    if (kWrite)
                        for (int32_t p = pk.x; p < pk.y; p++) idx[wp++] = p;
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

// off[g] = entries of all lists before group g (g = 0..G); scan_n is offset
// by scan_n[0] (one scan over both count arrays)
__global__ void k_list_off(int32_t G, int32_t R, const int64_t *scan_p, const int64_t *scan_n, int64_t *off)
{
    const int64_t nb = scan_n[0];
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += gridDim.x * blockDim.x)
        off[g] = scan_p[int64_t(g) * R] + (scan_n[int64_t(g) * R] - nb);
}

// tiles of <= tile_i particles per group, written at tile_off[g]
__global__ void k_tile_counts(const int32_t *g_cell, PCells P, int32_t G, int tile_i, const int64_t *off, int pj,
                              int64_t *ntile, int64_t *nparts, GCounts *gc)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) ntile[G] = nparts[G] = 0;  // terminal entries of the scan
    unsigned long long lmax = 0ull;
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const int32_t c = g_cell[g];
        const int64_t cnt = P.end[c] - P.begin[c];
        const int64_t nt = (cnt + tile_i - 1) / tile_i;
        const int64_t L = off[g + 1] - off[g];
        const int64_t parts = L > 0 ? (L + pj - 1) / pj : 1;
        ntile[g] = nt;
        nparts[g] = nt * parts;
        lmax = max(lmax, (unsigned long long)L);
    }
    if (lmax) atomicMax(&gc->lmax, lmax);
}

__global__ void k_tiles(const int32_t *g_cell, PCells P, int32_t G, int tile_i, const int64_t *tile_off, int4 *tiles)
{
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const int32_t c = g_cell[g];
        const int32_t b = P.begin[c], e = P.end[c];
        int64_t t = tile_off[g];
        for (int32_t p = b; p < e; p += tile_i) tiles[t++] = make_int4(p, min(p + tile_i, e), g, 0);
    }
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
              galloc(g, &g->P.cf, cc) && galloc(g, &g->xmax, 1) && galloc(g, &g->gc, 1) && galloc(g, &g->box_f, 2 * ctx->cap_g) && galloc(g, &g->flag3, 3 * cc) &&
              galloc(g, &g->pos3, 3 * cc) &&
              galloc(g, &g->g_cell, ctx->cap_g) && galloc(g, &g->cut, cc) && galloc(g, &g->above, cc) && galloc(g, &g->mom, 13 * cc) &&
              galloc(g, &g->box_lo, 3 * ctx->cap_g) && galloc(g, &g->box_hi, 3 * ctx->cap_g) &&
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
    return n * (8 * 2 + 4 * 2 + 8 * 2) + cc * (4 * 8 + 4 * 5 + 32 + 8 + 4 * 8 + 13 * 8 + 32) + G * (4 + 8 * 4 + 6 * 8 + 32) +
           ctx->cap_j * 8 * (12 + 2) + n * 8;
}


}  // namespace

// Called by hh_rebuild when the context builds on the device.
int hh_rebuild_device(hh_ctx *ctx, double t)
{
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->n;
    // A non-sticky error left pending by earlier runtime calls would make the
    // library calls below report failure; every call here is checked itself.
    cudaGetLastError();
    if (!ctx->gtree) {
        ctx->gtree = gtree_alloc(ctx);
        if (!ctx->gtree) return gfail(ctx, HH_ENOMEM, "hh_rebuild: device tree buffers do not fit");
        ctx->device_bytes += gtree_bytes(ctx);
        // particle ids live on the device from now on
        if (hh_gtree_set_ids(ctx->gtree, ctx->ids.data(), n, st) != HH_OK)
            return gfail(ctx, HH_ECUDA, "hh_rebuild: id upload failed");
    }
    GTreeBuf *g = ctx->gtree;
    const int grid = ctx->elem_grid;
    int64_t launches = 0;
    // Sizes stay on the device (GCounts) and the host reads them three times:
    // after the cells, after groups and cut, and after the list counts.
    auto read_counts = [&]() {
        cudaMemcpyAsync(g->gc_host, g->gc, sizeof(GCounts), cudaMemcpyDeviceToHost, st);
        return cudaStreamSynchronize(st) == cudaSuccess;
    };
    // 1. bounding box, synchronisation check, keys, sort
    k_root_init<<<1, 1, 0, st>>>(g->C, int32_t(n), g->gc, g->box);
    k_box<<<grid, 256, 0, st>>>(ctx->st, n, t, g->box);
    k_keys<<<grid, 256, 0, st>>>(ctx->st, n, g->box, g->key, g->idx, g->root_side, g->xmax, ctx->cfg.order);
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
    // 2. cells level by level (BFS), subtree sizes bottom-up, pre-order numbers top-down.
    //    The levels run up to two below the last tree's depth (the tree
    //    changes little in one dt_tree); if the last of them still made
    //    children, the rest follow after the read of the counts.
    const int64_t cap_cells = ctx->cap_j - n;
    const int32_t cap_c32 = int32_t(std::min<int64_t>(cap_cells, INT32_MAX));
    const int d_guess = g->depth < 0 ? kMaxDepth : std::min(kMaxDepth, g->depth + 2);
    for (int d = 0; d <= d_guess; d++) k_level<<<grid, 256, 0, st>>>(g->C, g->key2, d, ctx->cfg.leaf, g->gc, cap_c32);
    k_cells_done<<<1, 1, 0, st>>>(g->gc, g->box, d_guess);
    launches += (d_guess + 1) + 1;
    if (!read_counts()) return gfail(ctx, HH_ECUDA, "hh_rebuild: tree build failed");
    if (!g->gc_host->overflow && g->gc_host->lvl_n[d_guess + 1] > 0) {
        for (int d = d_guess + 1; d <= kMaxDepth; d++)
            k_level<<<grid, 256, 0, st>>>(g->C, g->key2, d, ctx->cfg.leaf, g->gc, cap_c32);
        k_cells_done<<<1, 1, 0, st>>>(g->gc, g->box, kMaxDepth);
        launches += (kMaxDepth - d_guess) + 1;
        if (!read_counts()) return gfail(ctx, HH_ECUDA, "hh_rebuild: tree build failed");
    }
    if (g->gc_host->bad) return gfail(ctx, HH_ESTATE, "hh_rebuild: particles are not synchronised at t");
    if (g->gc_host->overflow)
        return gfail(ctx, HH_ENOMEM, "hh_rebuild: tree exceeds nj_max (more cells than room for nodes)");
    const int32_t ncells = g->gc_host->ncells;
    // the deepest level that holds cells: the level loops below stop there
    // (a Plummer tree of 2^16 particles is 12-14 levels deep, the limit 21)
    int depth = 0;
    for (int d = 0; d <= kMaxDepth; d++)
        if (g->gc_host->lvl_n[d] > 0) depth = d;
    g->depth = depth;
    {
        // pre-order numbers and subtree sizes from one sort of the cells by
        // (first particle, depth); the moment sums and the selection arrays, not
        // yet in use, hold its keys and values
        uint64_t *ckey = reinterpret_cast<uint64_t *>(g->mom), *ckey2 = ckey + g->cap_c;
        int32_t *cval = g->flag3, *cval2 = g->pos3;
        int bits = 5;
        while (bits < 64 && (int64_t(1) << (bits - 5)) <= n) bits++;
        k_cell_keys<<<grid, 256, 0, st>>>(g->C, ncells, ckey, cval);
        int rs = cub_sort_pairs(g->tmp, g->tmp_bytes, ckey, ckey2, cval, cval2, ncells, bits, st);
        if (rs) return gfail(ctx, rs, "hh_rebuild: cell sort failed");
        k_pre_size<<<grid, 256, 0, st>>>(g->C, ncells, ckey2, cval2);
        launches += 2;
    }
    k_to_preorder<<<grid, 256, 0, st>>>(g->C, ncells, g->P, g->root_side);
    // 3. particles into Morton order (into the second buffer), then swap
    k_permute<<<grid, 256, 0, st>>>(ctx->st, g->alt, g->perm, n, g->ids, g->ids2);
    std::swap(ctx->st.x, g->alt.x);
    std::swap(ctx->st.v, g->alt.v);
    std::swap(ctx->st.a, g->alt.a);
    std::swap(ctx->st.jk, g->alt.jk);
    std::swap(ctx->st.m, g->alt.m);
    std::swap(ctx->st.t, g->alt.t);
    std::swap(ctx->st.dt, g->alt.dt);
    std::swap(g->ids, g->ids2);
    // 4. node records (bottom-up moments), groups and their boxes
    const int64_t cap_c = g->cap_c;
    for (int d = depth; d >= 0; d--) k_moments_level<<<grid, 256, 0, st>>>(ctx->st, g->C, g->gc, d, cap_c, g->mom);
    k_node_records<<<grid, 256, 0, st>>>(ctx->st, g->C, g->P, ncells, cap_c, g->mom, n, t);
    // 4b. groups, and (5.) the cut of subtrees of <= S cells and the cells
    //    above it: flags, one scan, counts and the three compacted tables
    const int32_t S = std::max<int32_t>(32, ncells / 256);
    k_flags3<<<grid, 256, 0, st>>>(g->P, ncells, ctx->cfg.n_crit, S, g->flag3);
    int rc = cub_exclusive_sum(g->tmp, g->tmp_bytes, g->flag3, g->pos3, 3 * int64_t(ncells), st);
    if (rc) return gfail(ctx, rc, "hh_rebuild: scan failed");
    k_counts3<<<1, 1, 0, st>>>(g->gc, g->flag3, g->pos3, ncells);
    k_write3<<<grid, 256, 0, st>>>(g->P, ncells, g->flag3, g->pos3, g->g_cell, ctx->cap_g, ctx->group_of, g->cut,
                                   g->above);
    k_group_box<<<grid, 256, 0, st>>>(ctx->st, g->P, g->gc, ctx->cap_g, g->g_cell, g->box_lo, g->box_hi, g->box_f);
    //    then per-(group, cut cell) list counts, scans, offsets, write
    launches += (depth + 1) + 7;
    if (!read_counts()) return gfail(ctx, HH_ECUDA, "hh_rebuild: group build failed");
    const int32_t G = g->gc_host->G, R = g->gc_host->R, A = g->gc_host->A;
    if (G > ctx->cap_g) return gfail(ctx, HH_ENOMEM, "hh_rebuild: more groups than groups_max");
    WalkArgs W;
    W.s = ctx->st;
    W.P = g->P;
    W.n = n;
    W.G = G;
    W.g_cell = g->g_cell;
    W.box_lo = g->box_lo;
    W.box_hi = g->box_hi;
    W.box_f = g->box_f;
    W.theta = ctx->cfg.theta;
    W.theta_f = float(ctx->cfg.theta);
    W.xmax = g->xmax;
    const int64_t top_n = std::max<int64_t>(1, int64_t(G) * A);
    if (top_n > g->top_cap) {
        if (g->top_buf) cudaFree(g->top_buf);
        g->top_buf = nullptr;
        g->top_cap = 0;
        if (cudaMalloc(&g->top_buf, sizeof(int32_t) * top_n) != cudaSuccess) {
            cudaGetLastError();
            return gfail(ctx, HH_ENOMEM, "hh_rebuild: list walk table does not fit");
        }
        g->top_cap = top_n;
    }
    if (A > 0) {
        k_top_above<<<unsigned((int64_t(G) * A + 127) / 128), 128, 0, st>>>(W, g->above, A, g->top_buf);
        launches++;
    }
    const int64_t pairs = int64_t(G) * R;
    if (2 * (pairs + 1) >= int64_t(INT32_MAX))  // (one scan covers both count arrays)
        return gfail(ctx, HH_ENOMEM, "hh_rebuild: too many (group, subtree) pairs");
    if (4 * (pairs + 1) > g->pair_cap) {
        if (g->pair_buf) cudaFree(g->pair_buf);
        g->pair_buf = nullptr;
        g->pair_cap = 0;
        if (cudaMalloc(&g->pair_buf, sizeof(int64_t) * 4 * (pairs + 1)) != cudaSuccess) {
            cudaGetLastError();
            return gfail(ctx, HH_ENOMEM, "hh_rebuild: list count buffers do not fit");
        }
        g->pair_cap = 4 * (pairs + 1);
    }
    int64_t *cnt_p = g->pair_buf, *cnt_n = cnt_p + pairs + 1, *scan_p = cnt_n + pairs + 1, *scan_n = scan_p + pairs + 1;
    const int64_t lgrid = std::min<int64_t>((pairs + 127) / 128, int64_t(1) << 30);
    k_lists_cut<false><<<unsigned(lgrid), 128, 0, st>>>(W, g->cut, R, g->pos3 + 2 * int64_t(ncells), g->top_buf, A, cnt_p, cnt_n, nullptr,
                                                        nullptr, nullptr);
    launches++;
    if ((rc = cub_exclusive_sum(g->tmp, g->tmp_bytes, cnt_p, scan_p, 2 * (pairs + 1), st)))  // cnt_p, cnt_n at once
        return gfail(ctx, rc, "hh_rebuild: scan failed");
    k_list_off<<<grid, 256, 0, st>>>(G, R, scan_p, scan_n, ctx->off);
    // 6. tiles and their work-item capacity (from the list lengths)
    int64_t *nparts = g->ntile + (G + 1), *parts_off = g->tile_off + (G + 1);
    k_tile_counts<<<grid, 256, 0, st>>>(g->g_cell, g->P, G, ctx->tile_i, ctx->off, ctx->part_len, g->ntile, nparts,
                                        g->gc);
    if ((rc = cub_exclusive_sum(g->tmp, g->tmp_bytes, g->ntile, g->tile_off, 2 * (int64_t(G) + 1), st)))
        return gfail(ctx, rc, "hh_rebuild: scan failed");
    k_store_totals<<<1, 1, 0, st>>>(g->gc, ctx->off + G, g->tile_off + G, parts_off, G);
    launches += 3;
    if (!read_counts()) return gfail(ctx, HH_ECUDA, "hh_rebuild: list count failed");
    const int64_t L = g->gc_host->L, n_tiles = g->gc_host->n_tiles, total_parts = g->gc_host->total_parts;
    if (n_tiles > ctx->cap_tiles) return gfail(ctx, HH_ENOMEM, "hh_rebuild: too many tiles");
    if (L > ctx->cap_list) {  // the list buffer grows (by a quarter beyond the need)
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
    }
    k_lists_cut<true><<<unsigned(lgrid), 128, 0, st>>>(W, g->cut, R, g->pos3 + 2 * int64_t(ncells), g->top_buf, A, nullptr, nullptr, scan_p,
                                                       scan_n, ctx->idx);
    k_tiles<<<grid, 256, 0, st>>>(g->g_cell, g->P, G, ctx->tile_i, g->tile_off, ctx->tiles);
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
