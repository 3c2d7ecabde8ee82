// Host tree and interaction-list builder (Section 2, tree-loop step 1).
//
// Builds, from particle positions at the tree time, a Morton-ordered octree,
// the particle groups of the modified tree algorithm (Barnes 1990: one list
// shared by a group of at most n_crit neighbouring particles) and one
// interaction list per group, plus the node records (mass-weighted position,
// velocity, acceleration and jerk of each cell's members) that the device
// predicts like particles.  The rules are stated in include/hh.h.
//
// Design: keys by magic-number bit interleaving, one std::sort of
// (key, index), cells split by binary search on the key digit of each level
// with an explicit stack, node moments in parallel over cells, and one list
// walk per group in parallel (OpenMP).  Arithmetic that decides membership
// (root cube, key scaling, centre of mass summed in Morton index order,
// group bounding box, distance test) is written so that it is exactly
// reproducible; the build compiles host code without FMA contraction.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "hh_internal.h"

namespace {

constexpr int kBits = 21;
constexpr uint32_t kMaxCoord = (1u << kBits) - 1u;
// below this many particles a build runs on the calling thread: small trees
// are built by several server threads at once, and a thread team per build
// costs more than it saves
constexpr int64_t kOmpMinN = 8192;

inline uint64_t spread_bits(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

inline int digit_at(uint64_t key, int depth) { return int((key >> (3 * (kBits - 1 - depth))) & 7u); }

// Peano-Hilbert key (Skilling 2004): from the top bit level down, the lower
// bits are mapped into the sub-cube's own frame (complement of the first
// coordinate's low bits where a coordinate's bit is set, else an exchange of
// low bits with the first coordinate), the coordinates are Gray-coded, and
// the transposed index is interleaved like a Morton key.
inline uint64_t hilbert_key(uint32_t c0, uint32_t c1, uint32_t c2)
{
    uint32_t c[3] = {c0, c1, c2};
    for (uint32_t q = 1u << (kBits - 1); q > 1u; q >>= 1) {
        const uint32_t p = q - 1u;
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

struct Cell {
    int32_t begin, end, depth, n_child;
    int32_t child[8];
    double side;
};

}  // namespace

struct hh_tree {
    int64_t n = 0;
    std::vector<int32_t> perm;
    std::vector<uint64_t> key;
    std::vector<Cell> cells;
    std::vector<double> cm, cx, cv, ca, cj;  // cx etc. AoS [cell][3]
    std::vector<int32_t> g_cell, g_begin, g_end, group_of;
    std::vector<int64_t> off;
    std::vector<int32_t> idx;
    // work buffers kept between rebuilds so that repeated builds reuse memory
    std::vector<std::pair<uint64_t, int32_t>> ki;
    std::vector<std::vector<int32_t>> lists;
};

namespace {

void build_cells(hh_tree &t, int leaf, double root_side)
{
    // explicit-stack pre-order construction
    struct Item {
        int32_t begin, end, depth, parent;
        double side;
    };
    std::vector<Item> stack;
    stack.push_back({0, int32_t(t.n), 0, -1, root_side});
    t.cells.reserve(size_t(t.n / 2 + 16));
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        int32_t id = int32_t(t.cells.size());
        Cell c;
        c.begin = it.begin;
        c.end = it.end;
        c.depth = it.depth;
        c.n_child = 0;
        c.side = it.side;
        t.cells.push_back(c);
        if (it.parent >= 0) {
            Cell &p = t.cells[it.parent];
            p.child[p.n_child++] = id;
        }
        if (it.end - it.begin <= leaf || it.depth >= kBits) continue;
        // children ranges by binary search on this level's octant digit;
        // pushed in reverse so that they pop in octant order (pre-order ids)
        Item kids[8];
        int nk = 0;
        int32_t b = it.begin;
        const uint64_t *k0 = t.key.data();
        for (int o = 0; o < 8 && b < it.end; o++) {
            const uint64_t *e = std::partition_point(k0 + b, k0 + it.end,
                                                     [&](uint64_t k) { return digit_at(k, it.depth) <= o; });
            int32_t ei = int32_t(e - k0);
            if (ei > b) kids[nk++] = {b, ei, it.depth + 1, id, it.side * 0.5};
            b = ei;
        }
        for (int q = nk - 1; q >= 0; q--) stack.push_back(kids[q]);
    }
}

void node_moments(hh_tree &t, const double *x, const double *v, const double *a, const double *jk,
                  const double *m)
{
    const int64_t n = t.n;
    const int32_t nc = int32_t(t.cells.size());
    t.cm.assign(nc, 0.0);
    t.cx.assign(3 * size_t(nc), 0.0);
    t.cv.assign(3 * size_t(nc), 0.0);
    t.ca.assign(3 * size_t(nc), 0.0);
    t.cj.assign(3 * size_t(nc), 0.0);
#pragma omp parallel for schedule(dynamic, 32) if (t.n >= kOmpMinN)
    for (int32_t c = 0; c < nc; c++) {
        double M = 0.0, sx[3] = {0, 0, 0}, sv[3] = {0, 0, 0}, sa[3] = {0, 0, 0}, sj[3] = {0, 0, 0};
        for (int32_t q = t.cells[c].begin; q < t.cells[c].end; q++) {
            const int64_t i = t.perm[q];
            const double mi = m[i];
            M += mi;
            for (int d = 0; d < 3; d++) {
                sx[d] += mi * x[d * n + i];
                sv[d] += mi * v[d * n + i];
                sa[d] += mi * a[d * n + i];
                sj[d] += mi * jk[d * n + i];
            }
        }
        t.cm[c] = M;
        for (int d = 0; d < 3; d++) {
            t.cx[3 * size_t(c) + d] = sx[d] / M;
            t.cv[3 * size_t(c) + d] = sv[d] / M;
            t.ca[3 * size_t(c) + d] = sa[d] / M;
            t.cj[3 * size_t(c) + d] = sj[d] / M;
        }
    }
}

void find_groups(hh_tree &t, int n_crit)
{
    std::vector<int32_t> stack{0};
    while (!stack.empty()) {
        int32_t c = stack.back();
        stack.pop_back();
        const Cell &cell = t.cells[c];
        if (cell.end - cell.begin <= n_crit || cell.n_child == 0) {
            t.g_cell.push_back(c);
            t.g_begin.push_back(cell.begin);
            t.g_end.push_back(cell.end);
            continue;
        }
        for (int q = cell.n_child - 1; q >= 0; q--) stack.push_back(cell.child[q]);
    }
    t.group_of.assign(size_t(t.n), 0);
    for (size_t g = 0; g < t.g_cell.size(); g++)
        for (int32_t q = t.g_begin[g]; q < t.g_end[g]; q++) t.group_of[q] = int32_t(g);
}

// The walk is pre-order with children in octant order, so particles (Morton
// indices) and nodes (n + pre-order cell number) each come out ascending:
// collecting them apart and concatenating gives the sorted list directly.
void group_list(const hh_tree &t, int32_t g, double theta, const double *x, std::vector<int32_t> &out,
                std::vector<int32_t> &stack, std::vector<int32_t> &nodes)
{
    const int64_t n = t.n;
    const int32_t gb = t.g_begin[g], ge = t.g_end[g], gc = t.g_cell[g];
    double lo[3], hi[3];
    {
        const int64_t i0 = t.perm[gb];
        for (int d = 0; d < 3; d++) lo[d] = hi[d] = x[d * n + i0];
        for (int32_t q = gb; q < ge; q++) {
            const int64_t i = t.perm[q];
            for (int d = 0; d < 3; d++) {
                const double u = x[d * n + i];
                if (u < lo[d]) lo[d] = u;
                if (u > hi[d]) hi[d] = u;
            }
        }
    }
    out.clear();
    nodes.clear();
    stack.clear();
    stack.push_back(0);
    while (!stack.empty()) {
        const int32_t c = stack.back();
        stack.pop_back();
        const Cell &cell = t.cells[c];
        if (c == gc) {
            for (int32_t q = cell.begin; q < cell.end; q++) out.push_back(q);
            continue;
        }
        const bool contains_group = cell.begin <= gb && ge <= cell.end;
        if (!contains_group) {
            if (cell.end - cell.begin == 1) {
                out.push_back(cell.begin);
                continue;
            }
            double d2 = 0.0;
            for (int d = 0; d < 3; d++) {
                const double cmd = t.cx[3 * size_t(c) + d];
                double gap = 0.0;
                if (cmd < lo[d]) gap = lo[d] - cmd;
                else if (cmd > hi[d]) gap = cmd - hi[d];
                d2 += gap * gap;
            }
            const double dist = std::sqrt(d2);
            if (cell.side < theta * dist) {
                nodes.push_back(int32_t(n + c));
                continue;
            }
            if (cell.n_child == 0) {
                for (int32_t q = cell.begin; q < cell.end; q++) out.push_back(q);
                continue;
            }
        }
        for (int q = cell.n_child - 1; q >= 0; q--) stack.push_back(cell.child[q]);
    }
    out.insert(out.end(), nodes.begin(), nodes.end());
}

}  // namespace

namespace {

int check_inputs(int64_t n, const double *x, const double *v, const double *a, const double *jk, const double *m,
                 int32_t leaf, int32_t n_crit, double theta, int32_t order)
{
    if (n < 1 || n > INT32_MAX / 2 || !x || !v || !a || !jk || !m || leaf < 1 || n_crit < 1 || !(theta >= 0.0) ||
        (order != HH_ORDER_MORTON && order != HH_ORDER_HILBERT))
        return hh_set_global_error(HH_EINVAL, "hh_tree_build: bad arguments");
    for (int64_t i = 0; i < 3 * n; i++)
        if (!std::isfinite(x[i]) || !std::isfinite(v[i]) || !std::isfinite(a[i]) || !std::isfinite(jk[i]))
            return hh_set_global_error(HH_EINVAL, "hh_tree_build: non-finite particle data");
    for (int64_t i = 0; i < n; i++)
        if (!(m[i] > 0.0) || !std::isfinite(m[i]))
            return hh_set_global_error(HH_EINVAL, "hh_tree_build: masses must be positive and finite");
    return HH_OK;
}

// Builds into t, reusing the capacity of its vectors.
int build_into(hh_tree *t, int64_t n, const double *x, const double *v, const double *a, const double *jk,
               const double *m, int32_t leaf, int32_t n_crit, double theta, int32_t order)
{
    try {
        t->n = n;
        t->cells.clear();
        t->g_cell.clear();
        t->g_begin.clear();
        t->g_end.clear();
        double lo[3], hi[3];
        for (int d = 0; d < 3; d++) {
            lo[d] = hi[d] = x[d * n];
            for (int64_t i = 1; i < n; i++) {
                const double u = x[d * n + i];
                lo[d] = u < lo[d] ? u : lo[d];
                hi[d] = u > hi[d] ? u : hi[d];
            }
        }
        double side = 0.0;
        for (int d = 0; d < 3; d++)
            if (hi[d] - lo[d] > side) side = hi[d] - lo[d];
        if (side == 0.0) side = 1.0;
        const double scale = double(1u << kBits) / side;
        auto &ki = t->ki;
        ki.resize(size_t(n));
#pragma omp parallel for schedule(static) if (n >= kOmpMinN)
        for (int64_t i = 0; i < n; i++) {
            uint32_t u[3];
            for (int d = 0; d < 3; d++) {
                double f = std::floor((x[d * n + i] - lo[d]) * scale);
                f = f < 0.0 ? 0.0 : f;
                f = f > double(kMaxCoord) ? double(kMaxCoord) : f;
                u[d] = uint32_t(f);
            }
            const uint64_t k = order == HH_ORDER_HILBERT
                                   ? hilbert_key(u[0], u[1], u[2])
                                   : (spread_bits(u[0]) << 2) | (spread_bits(u[1]) << 1) | spread_bits(u[2]);
            ki[size_t(i)] = {k, int32_t(i)};
        }
        std::sort(ki.begin(), ki.end());
        t->perm.resize(size_t(n));
        t->key.resize(size_t(n));
        for (int64_t q = 0; q < n; q++) {
            t->key[size_t(q)] = ki[size_t(q)].first;
            t->perm[size_t(q)] = ki[size_t(q)].second;
        }
        build_cells(*t, leaf, side);
        node_moments(*t, x, v, a, jk, m);
        find_groups(*t, n_crit);
        const int32_t G = int32_t(t->g_cell.size());
        auto &lists = t->lists;
        if (lists.size() < size_t(G)) lists.resize(size_t(G));
#pragma omp parallel if (n >= kOmpMinN)
        {
            std::vector<int32_t> stack, nodes;
#pragma omp for schedule(dynamic, 4)
            for (int32_t g = 0; g < G; g++) group_list(*t, g, theta, x, lists[size_t(g)], stack, nodes);
        }
        t->off.assign(size_t(G) + 1, 0);
        for (int32_t g = 0; g < G; g++) t->off[size_t(g) + 1] = t->off[size_t(g)] + int64_t(lists[size_t(g)].size());
        t->idx.resize(size_t(t->off[size_t(G)]));
#pragma omp parallel for schedule(static) if (n >= kOmpMinN)
        for (int32_t g = 0; g < G; g++)
            std::copy(lists[size_t(g)].begin(), lists[size_t(g)].end(), t->idx.begin() + t->off[size_t(g)]);
    } catch (const std::bad_alloc &) {
        return hh_set_global_error(HH_ENOMEM, "hh_tree_build: out of host memory");
    }
    return HH_OK;
}

}  // namespace

extern "C" int hh_tree_build(hh_tree **out, int64_t n, const double *x, const double *v, const double *a,
                             const double *jk, const double *m, int32_t leaf, int32_t n_crit, double theta)
{
    return hh_tree_build_ordered(out, n, x, v, a, jk, m, leaf, n_crit, theta, HH_ORDER_MORTON);
}

extern "C" int hh_tree_build_ordered(hh_tree **out, int64_t n, const double *x, const double *v, const double *a,
                                     const double *jk, const double *m, int32_t leaf, int32_t n_crit, double theta,
                                     int32_t order)
{
    if (!out) return hh_set_global_error(HH_EINVAL, "hh_tree_build: out is NULL");
    *out = nullptr;
    int rc = check_inputs(n, x, v, a, jk, m, leaf, n_crit, theta, order);
    if (rc) return rc;
    hh_tree *t = new (std::nothrow) hh_tree;
    if (!t) return hh_set_global_error(HH_ENOMEM, "hh_tree_build: out of host memory");
    rc = build_into(t, n, x, v, a, jk, m, leaf, n_crit, theta, order);
    if (rc) {
        delete t;
        return rc;
    }
    *out = t;
    return HH_OK;
}

// Internal: rebuild an existing tree object (or create one if *tp is NULL).
int hh_tree_rebuild(hh_tree **tp, int64_t n, const double *x, const double *v, const double *a, const double *jk,
                    const double *m, int32_t leaf, int32_t n_crit, double theta, int32_t order)
{
    int rc = check_inputs(n, x, v, a, jk, m, leaf, n_crit, theta, order);
    if (rc) return rc;
    if (!*tp) {
        *tp = new (std::nothrow) hh_tree;
        if (!*tp) return hh_set_global_error(HH_ENOMEM, "hh_tree_build: out of host memory");
    }
    return build_into(*tp, n, x, v, a, jk, m, leaf, n_crit, theta, order);
}

extern "C" int hh_tree_sizes(const hh_tree *t, int64_t *n_nodes, int32_t *n_groups, int64_t *list_len)
{
    if (!t) return hh_set_global_error(HH_EINVAL, "hh_tree_sizes: NULL tree");
    if (n_nodes) *n_nodes = int64_t(t->cells.size());
    if (n_groups) *n_groups = int32_t(t->g_cell.size());
    if (list_len) *list_len = int64_t(t->idx.size());
    return HH_OK;
}

extern "C" int hh_tree_export(const hh_tree *t, int32_t *perm, double *node_x, double *node_v, double *node_a,
                              double *node_jk, double *node_m, int64_t *off, int32_t *idx, int32_t *group_of)
{
    if (!t) return hh_set_global_error(HH_EINVAL, "hh_tree_export: NULL tree");
    const size_t nc = t->cells.size();
    if (perm) std::memcpy(perm, t->perm.data(), sizeof(int32_t) * size_t(t->n));
    auto soa = [&](const std::vector<double> &src, double *dst) {
        if (!dst) return;
        for (size_t c = 0; c < nc; c++)
            for (int d = 0; d < 3; d++) dst[d * nc + c] = src[3 * c + d];
    };
    soa(t->cx, node_x);
    soa(t->cv, node_v);
    soa(t->ca, node_a);
    soa(t->cj, node_jk);
    if (node_m) std::memcpy(node_m, t->cm.data(), sizeof(double) * nc);
    if (off) std::memcpy(off, t->off.data(), sizeof(int64_t) * t->off.size());
    if (idx && !t->idx.empty()) std::memcpy(idx, t->idx.data(), sizeof(int32_t) * t->idx.size());
    if (group_of) std::memcpy(group_of, t->group_of.data(), sizeof(int32_t) * size_t(t->n));
    return HH_OK;
}

extern "C" int hh_tree_free(hh_tree *t)
{
    delete t;
    return HH_OK;
}

// Internal (not in hh.h): read-only view of a built tree for the library's
// own rebuild path, which uploads straight from these arrays.
int hh_tree_view(const hh_tree *t, HhTreeView *v)
{
    if (!t || !v) return HH_EINVAL;
    v->n = t->n;
    v->n_nodes = int64_t(t->cells.size());
    v->n_groups = int32_t(t->g_cell.size());
    v->list_len = int64_t(t->idx.size());
    v->perm = t->perm.data();
    v->cm = t->cm.data();
    v->cx = t->cx.data();
    v->cv = t->cv.data();
    v->ca = t->ca.data();
    v->cj = t->cj.data();
    v->off = t->off.data();
    v->idx = t->idx.data();
    v->group_of = t->group_of.data();
    return HH_OK;
}
