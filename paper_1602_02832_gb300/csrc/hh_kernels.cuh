// Device code of the list-driven Hermite hot path (sm_103a).
//
// One block step (Section 2, tree-loop steps 2-7) is three kernels:
//   k_predict  every j entry (particles and tree nodes) to the block time
//              (GRAPE predictor; step 4), written as packed records;
//              and, with one ballot per static i tile, appends the work
//              items (tile, list part) of tiles with active particles
//              (t_i + dt_i == t_next, step 2);
//   k_force    CTAs pull work items from a queue and sum acc / jerk / pot
//              over the item's part of the group's list (steps 4a + 5);
//   k_correct  4th-order Hermite corrector + Aarseth block step (step 6),
//              and the min over t_i + dt_i that starts the next step.
// No kernel waits on another CTA; there are no spin loops.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace hh {

constexpr int kThreads = 128;  // threads per force CTA (4 warps)
constexpr int kMaxTileI = 32;  // particles per static i tile (one ballot)
constexpr int kFold = 16;     // FP32 terms per thread between compensated folds

// ---------------------------------------------------------------- scalars
struct DevScalars {
    unsigned long long tmin[2];  // min(t_i + dt_i) as positive-double bit patterns
    double t_end;                // loop bound of hh_advance
    int32_t done;                // set once the next block time exceeds t_end
    int32_t err;                 // device-detected error (HH_* code), 0 = none
    uint32_t work;               // force work-queue head
    uint32_t n_items;            // work items of this step
    int32_t part_len;            // shortest list part (a multiple of the staging chunk)
    int32_t work_item;           // target interactions per work item (0: every part is part_len long)
    int32_t work_split;          // > 0: work_item applies only to batched steps with this many active particles
    uint32_t slot_ctr;           // partial-sum slots handed out this step
    uint32_t slot_par[2];        // the same for the batched loop, by step parity
    int32_t n_act_last;          // active particles of the last corrected step
    int64_t n;                   // particles
    int64_t nj;                  // j entries
    int32_t n_tiles;             // static i tiles
    int32_t pad0;
    unsigned long long block_steps, particle_steps, interactions;
    unsigned long long list_steps;  // batched steps that predicted only their list parts' entries
    unsigned long long na_hist[32];  // active i tiles summed over block steps, by n_a - 1
    // block-step levels (level k <=> dt = 2^-k), kept by the batched loop
    int32_t lvl_cnt[32];          // particles per level
    unsigned long long t_cur_bits;  // latest block time (max t_i), positive-double bits
};

// Block-step control passed by value to every kernel of a step.
struct StepCtl {
    int32_t mode;       // 0: active = {t_i + dt_i == t_next}; 1: marked; 2: all particles
    int32_t slot_cur;   // tmin slot holding this step's time (mode 0)
    int32_t slot_next;  // tmin slot that receives the next step's time (mode 0)
    int32_t pad;
    double t_arg;       // step time for modes 1 and 2
};

// ---------------------------------------------------------------- records
// Predicted j record, plain form: (x, y, z, m), (vx, vy, vz, 0) in FP64.
struct __align__(32) RecF64 {
    double4 xm;
    double4 v;
};
// Predicted j record, mixed form: position as an unevaluated float pair
// x = hi + lo (|lo| <= ulp(hi)/2), velocity and mass in FP32.
struct __align__(16) RecMix {
    float4 hm;  // (x_hi, y_hi, z_hi, m)
    float4 lo;  // (x_lo, y_lo, z_lo, 0)
    float4 v;   // (vx, vy, vz, 0)
};

// Mixed form: per j entry, the FP32 quantities the predictor needs,
// refreshed whenever the entry's FP64 state changes (upload, correction):
// position as a float pair, velocity, a/2 and jerk/6.
struct __align__(16) BaseMix {
    float4 hm;  // (x_hi, y_hi, z_hi, m)
    float4 lo;  // (x_lo, y_lo, z_lo, 0)
    float4 v;   // (vx, vy, vz, 0)
    float4 a2;  // a / 2
    float4 j6;  // jerk / 6
};

struct State {
    double *x, *v, *a, *jk;  // [3][cap_j]
    BaseMix *base;           // [cap_j] mixed form only (else nullptr)
    double *m, *t;           // [cap_j]
    double *dt;              // [cap_n]
    double *acc1, *jerk1, *pot1;  // [3][cap_n], [cap_n]: last force results
    int32_t *mark;           // [cap_n]
    int64_t cap_j, cap_n;
};

// One work item: a part of one i tile's interaction list.  It carries the
// tile record and the group's list range, so a worker reads one record before
// it can load particles and list indices.
struct __align__(16) WorkItem {
    int32_t tile;      // static tile index
    int32_t part_sim;  // list part | simulation << 16
    uint32_t mask;     // active lanes of the tile
    int32_t slot;      // first partial-sum slot of the tile's parts (0 with one part)
    int32_t p_begin, p_end, group;  // the tile's particles and list group
    int32_t part_len;               // list entries per part of this tile (the last part may be shorter)
    int64_t gb, ge;    // the group's list [gb, ge) in idx
};

__device__ __forceinline__ WorkItem make_item(int tile, int part_sim, uint32_t mask, int slot, const int4 td, int64_t gb,
                                              int64_t ge, int part_len)
{
    WorkItem w;
    w.tile = tile;
    w.part_sim = part_sim;
    w.mask = mask;
    w.slot = slot;
    w.p_begin = td.x;
    w.p_end = td.y;
    w.group = td.z;
    w.part_len = part_len;
    w.gb = gb;
    w.ge = ge;
    return w;
}

struct Lists {
    const int64_t *off;
    const int32_t *idx;
    const int4 *tiles;  // static i tiles: (p_begin, p_end, group, first part slot)
    WorkItem *items;    // this step's work
    void *partials;     // per (tile part, i slot) sums of split lists [part slots][32]
    int32_t *tile_cnt;  // arrivals per tile (reset by the last arriver)
    const int32_t *i_map;  // optional: i slot position -> j index (kMapI kernels only)
};

struct Params {
    double eps2, eta, eta_s, dt_min, dt_max;
};

__device__ __forceinline__ double bits_to_time(unsigned long long b) { return __longlong_as_double((long long)b); }

// Time of this step; false if the step is a no-op (loop finished).
__device__ __forceinline__ bool step_time(const DevScalars *ds, const StepCtl &c, double *t)
{
    if (c.mode != 0) {
        *t = c.t_arg;
        return true;
    }
    if (*(volatile const int32_t *)&ds->done) return false;
    double tn = bits_to_time(*(volatile const unsigned long long *)&ds->tmin[c.slot_cur]);
    if (!(tn <= ds->t_end)) return false;
    *t = tn;
    return true;
}

__device__ __forceinline__ bool is_active(const State &s, const StepCtl &c, int64_t p, double tnow)
{
    if (c.mode == 0) return s.t[p] + s.dt[p] == tnow;
    if (c.mode == 1) return s.mark[p] != 0;
    return true;
}

// Largest power of two <= x for positive normal x: clear the mantissa.
__device__ __forceinline__ double pow2_floor(double x)
{
    return __longlong_as_double(__double_as_longlong(x) & (long long)0xFFF0000000000000ull);
}

// ------------------------------------------------------- tile selection
// Step 2 on the device: for each static i tile (<= 32 consecutive particles
// of one group) one warp ballots the tile's active particles; a tile with
// any active particle appends one work item per part of its group's list.
// Item order may vary between runs; results do not depend on it.
// Warp-collective: appends one work item per part of tile `tile`'s list.
// List entries per work item for a tile with n_a active particles: about
// `work` interactions per item (n_a x part length), never shorter than
// pj_min, a multiple of pj_min.  Items of equal cost keep the SMs evenly
// loaded; the length depends only on n_a, so results stay deterministic.
__device__ __forceinline__ int part_len_for(int n_a, int pj_min, int work)
{
    if (work <= 0) return pj_min;
    const int want = (work + n_a - 1) / n_a;
    const int k = (want + pj_min - 1) / pj_min;
    return (k < 1 ? 1 : k) * pj_min;
}

__device__ __forceinline__ int parts_of(int64_t len, int pj) { return len > 0 ? (int)((len + pj - 1) / pj) : 1; }

// Warp-collective: appends one work item per part of tile `tile`'s list;
// item = (tile, part | sim << 16, active mask, first partial-sum slot, part
// length).  `work` is the equal-cost target of this step (0: parts of pj_min).
__device__ __forceinline__ void append_tile_items(const Lists &L, int tile, const int4 td, uint32_t mask, int pj_min,
                                                  int work, uint32_t *n_items, uint32_t *slot_ctr, WorkItem *items,
                                                  int sim, unsigned long long *na_hist, uint32_t *max_chunks = nullptr)
{
    const int lane = threadIdx.x & 31;
    const int64_t gb = L.off[td.z], ge = L.off[td.z + 1];
    const int64_t len = ge - gb;
    const int pj = part_len_for(__popc(mask), pj_min, work);
    const int n_parts = parts_of(len, pj);
    int base = 0, slot = 0;
    if (lane == 0) {
        base = (int)atomicAdd(n_items, (uint32_t)n_parts);
        slot = n_parts > 1 ? (int)atomicAdd(slot_ctr, (uint32_t)n_parts) : 0;
        atomicAdd(&na_hist[__popc(mask) - 1], 1ull);
        // (with max_chunks: the longest part so far, in 32-entry chunks)
        if (max_chunks) atomicMax(max_chunks, (uint32_t)((min((int64_t)pj, len) + 31) / 32));
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    for (int q = lane; q < n_parts; q += 32) items[base + q] = make_item(tile, q | (sim << 16), mask, slot, td, gb, ge, pj);
}

__device__ __forceinline__ void select_tiles(const State &s, const Lists &L, DevScalars *ds, const StepCtl &c,
                                             double tnow)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int n_tiles = ds->n_tiles;
    // (this loop does not count a step's active particles first, so a
    // work_item limited to large steps, work_split > 0, is not used here)
    const int pj = ds->part_len, work = ds->work_split > 0 ? 0 : ds->work_item;
    for (int64_t tile = warp0; tile < n_tiles; tile += nwarps) {
        const int4 td = L.tiles[tile];
        const int64_t p = td.x + lane;
        const bool act = (p < td.y) && is_active(s, c, p, tnow);
        const uint32_t mask = __ballot_sync(0xffffffffu, act);
        if (mask == 0u) continue;
        append_tile_items(L, (int)tile, td, mask, pj, work, &ds->n_items, &ds->slot_ctr, L.items, 0, ds->na_hist);
    }
}

static __global__ void k_select(State s, Lists L, DevScalars *ds, StepCtl c)
{
    double tnow;
    if (!step_time(ds, c, &tnow)) return;
    select_tiles(s, L, ds, c, tnow);
}

// -------------------------------------------------------------- predictor
// x + v D + a D^2/2 + jk D^3/6 and v + a D + jk D^2/2, in Horner form.
// Taylor predictor of one component over D (Section 2, step 3).
__device__ __forceinline__ void predict_xv(double D, double x, double v, double a, double j, double &xp, double &vp)
{
    const double h = 0.5 * D, th = D * (1.0 / 3.0);
    xp = x + D * (v + h * (a + th * j));
    vp = v + D * (a + h * j);
}

__device__ __forceinline__ void predict_one(const State &s, int64_t e, double tnow, double xp[3], double vp[3])
{
    const double D = tnow - s.t[e];
#pragma unroll
    for (int d = 0; d < 3; d++)
        predict_xv(D, s.x[d * s.cap_j + e], s.v[d * s.cap_j + e], s.a[d * s.cap_j + e], s.jk[d * s.cap_j + e], xp[d],
                   vp[d]);
}

template <typename Rec>
__device__ __forceinline__ void store_rec(Rec *out, int64_t e, const double xp[3], const double vp[3], double m);

template <>
__device__ __forceinline__ void store_rec<RecF64>(RecF64 *out, int64_t e, const double xp[3], const double vp[3],
                                                 double m)
{
    RecF64 r;
    r.xm = make_double4(xp[0], xp[1], xp[2], m);
    r.v = make_double4(vp[0], vp[1], vp[2], 0.0);
    out[e] = r;
}

template <>
__device__ __forceinline__ void store_rec<RecMix>(RecMix *out, int64_t e, const double xp[3], const double vp[3],
                                                 double m)
{
    float hi[3], lo[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        hi[d] = __double2float_rn(xp[d]);
        lo[d] = __double2float_rn(xp[d] - (double)hi[d]);
    }
    RecMix r;
    r.hm = make_float4(hi[0], hi[1], hi[2], __double2float_rn(m));
    r.lo = make_float4(lo[0], lo[1], lo[2], 0.f);
    r.v = make_float4(__double2float_rn(vp[0]), __double2float_rn(vp[1]), __double2float_rn(vp[2]), 0.f);
    out[e] = r;
}

// FP32 copy of entry e's FP64 state for the mixed predictor, one component
// (d = 0, 1, 2) from the values x, v, a, jk of that component; the mass m goes
// with component 0.
__device__ __forceinline__ void refresh_base_values(const State &s, int64_t e, int d, double x, double v, double a,
                                                    double jk, double m)
{
    const float hi = __double2float_rn(x);
    const float lo = __double2float_rn(x - (double)hi);
    const float vf = __double2float_rn(v);
    const float a2 = 0.5f * __double2float_rn(a);
    const float j6 = __double2float_rn(jk) * (1.0f / 6.0f);
    float *b = reinterpret_cast<float *>(&s.base[e]);  // hm, lo, v, a2, j6: float4 each
    b[0 + d] = hi;
    b[4 + d] = lo;
    b[8 + d] = vf;
    b[12 + d] = a2;
    b[16 + d] = j6;
    if (d == 0) {
        b[3] = __double2float_rn(m);
        b[7] = b[11] = b[15] = b[19] = 0.f;
    }
}

// The same from the state arrays.
__device__ __forceinline__ void refresh_base_component(const State &s, int64_t e, int d)
{
    refresh_base_values(s, e, d, s.x[d * s.cap_j + e], s.v[d * s.cap_j + e], s.a[d * s.cap_j + e],
                        s.jk[d * s.cap_j + e], d == 0 ? s.m[e] : 0.0);
}

__device__ __forceinline__ void refresh_base(const State &s, int64_t e)
{
#pragma unroll
    for (int d = 0; d < 3; d++) refresh_base_component(s, e, d);
}

// Mixed predictor: the FP64 base position (as a float pair) plus an FP32
// increment D (v + D (a/2 + D jerk/6)), added with TwoSum; v + D (a + D jerk/2)
// in FP32.  D = t - t_e is exact in FP32 (a multiple of dt_min below dt_tree).
__device__ __forceinline__ RecMix mix_from_base(const BaseMix &b, float D)
{
    const float hx[3] = {b.hm.x, b.hm.y, b.hm.z}, lx[3] = {b.lo.x, b.lo.y, b.lo.z};
    const float vv[3] = {b.v.x, b.v.y, b.v.z}, aa[3] = {b.a2.x, b.a2.y, b.a2.z}, jj[3] = {b.j6.x, b.j6.y, b.j6.z};
    float ho[3], lo[3], vo[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float dx = D * fmaf(D, fmaf(D, jj[d], aa[d]), vv[d]);
        const float sum = __fadd_rn(hx[d], dx);
        const float bb = __fsub_rn(sum, hx[d]);
        const float err = __fadd_rn(__fsub_rn(hx[d], __fsub_rn(sum, bb)), __fsub_rn(dx, bb));
        ho[d] = sum;
        lo[d] = __fadd_rn(lx[d], err);
        vo[d] = fmaf(D, fmaf(D, 3.f * jj[d], 2.f * aa[d]), vv[d]);
    }
    RecMix r;
    r.hm = make_float4(ho[0], ho[1], ho[2], b.hm.w);
    r.lo = make_float4(lo[0], lo[1], lo[2], 0.f);
    r.v = make_float4(vo[0], vo[1], vo[2], 0.f);
    return r;
}

// Inputs of one entry's prediction, loaded ahead of its arithmetic so that a
// thread can keep several entries' loads in flight (pred_load, then
// pred_store: the same arithmetic as predict_one / mix_from_base).
template <typename Rec>
struct PredIn;
template <>
struct PredIn<RecF64> {
    double t, m, x[3], v[3], a[3], j[3];
};
template <>
struct PredIn<RecMix> {
    double t;
    BaseMix b;
};

template <typename Rec>
__device__ __forceinline__ void pred_load(const State &s, int64_t e, PredIn<Rec> &in);
template <>
__device__ __forceinline__ void pred_load<RecF64>(const State &s, int64_t e, PredIn<RecF64> &in)
{
    in.t = s.t[e];
    in.m = s.m[e];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        in.x[d] = s.x[d * s.cap_j + e];
        in.v[d] = s.v[d * s.cap_j + e];
        in.a[d] = s.a[d * s.cap_j + e];
        in.j[d] = s.jk[d * s.cap_j + e];
    }
}
template <>
__device__ __forceinline__ void pred_load<RecMix>(const State &s, int64_t e, PredIn<RecMix> &in)
{
    in.t = s.t[e];
    in.b = s.base[e];
}

template <typename Rec>
__device__ __forceinline__ void pred_store(const PredIn<Rec> &in, Rec *rec, int64_t e, double tnow);
template <>
__device__ __forceinline__ void pred_store<RecF64>(const PredIn<RecF64> &in, RecF64 *rec, int64_t e, double tnow)
{
    const double D = tnow - in.t;
    double xp[3], vp[3];
#pragma unroll
    for (int d = 0; d < 3; d++) predict_xv(D, in.x[d], in.v[d], in.a[d], in.j[d], xp[d], vp[d]);
    store_rec<RecF64>(rec, e, xp, vp, in.m);
}
template <>
__device__ __forceinline__ void pred_store<RecMix>(const PredIn<RecMix> &in, RecMix *rec, int64_t e, double tnow)
{
    rec[e] = mix_from_base(in.b, __double2float_rn(tnow - in.t));
}

// Predicted record of entry e at tnow, in the form's own arithmetic.
template <typename Rec>
__device__ __forceinline__ void predict_entry(const State &s, Rec *rec, int64_t e, double tnow)
{
    PredIn<Rec> in;
    pred_load<Rec>(s, e, in);
    pred_store<Rec>(in, rec, e, tnow);
}

template <typename Rec>
__global__ void k_predict(State s, Rec *rec, Lists L, DevScalars *ds, StepCtl c)
{
    double tnow;
    if (!step_time(ds, c, &tnow)) {
        if (c.mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) ds->done = 1;
        return;
    }
    if (c.mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        ds->tmin[c.slot_next] = 0x7FF0000000000000ull;  // +inf
        ds->work = 0u;
        ds->n_act_last = 0;
        ds->block_steps += 1ull;
    }

    const int64_t nj = ds->nj;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nj; e += (int64_t)gridDim.x * blockDim.x)
        predict_entry<Rec>(s, rec, e, tnow);
    if (c.mode == 0) select_tiles(s, L, ds, c, tnow);
}

// ------------------------------------------------------ pairwise kernels
// Plummer-softened pair term (Makino & Aarseth 1992): r = x_j - x_i,
// w = v_j - v_i, s = r^2 + eps^2; a += m r s^-3/2;
// jerk += m (w s^-3/2 - 3 (r.w) r s^-5/2); pot -= m s^-1/2.

struct AccF64 {
    double ax, ay, az, jx, jy, jz, p;
    __device__ void zero() { ax = ay = az = jx = jy = jz = p = 0.0; }
};

struct IF64 {
    double x, y, z, vx, vy, vz;
};

__device__ __forceinline__ void load_i(const RecF64 *rec, int64_t i, IF64 &o)
{
    const RecF64 r = rec[i];
    o.x = r.xm.x; o.y = r.xm.y; o.z = r.xm.z;
    o.vx = r.v.x; o.vy = r.v.y; o.vz = r.v.z;
}

__device__ __forceinline__ void interact(const IF64 &I, const RecF64 &J, bool self, double eps2, AccF64 &A)
{
    const double dx = J.xm.x - I.x, dy = J.xm.y - I.y, dz = J.xm.z - I.z;
    const double wx = J.v.x - I.vx, wy = J.v.y - I.vy, wz = J.v.z - I.vz;
    double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    r2 = self ? 1.0 : r2;
    const double mj = self ? 0.0 : J.xm.w;
    const double rw = fma(dx, wx, fma(dy, wy, dz * wz));
    const double rinv = rsqrt(r2);
    const double rinv2 = rinv * rinv;
    const double mr = mj * rinv;
    const double mr3 = mr * rinv2;
    const double al = 3.0 * rw * rinv2;
    A.p += mr;
    A.ax = fma(mr3, dx, A.ax);
    A.ay = fma(mr3, dy, A.ay);
    A.az = fma(mr3, dz, A.az);
    A.jx = fma(mr3, fma(-al, dx, wx), A.jx);
    A.jy = fma(mr3, fma(-al, dy, wy), A.jy);
    A.jz = fma(mr3, fma(-al, dz, wz), A.jz);
}

// Mixed: chunk partials in FP32, folded into (hi, lo) pairs after each
// staged chunk with Knuth's TwoSum, so that the running sum is carried to
// about 2^-48 relative while the inner loop stays plain FP32.
struct F2 {
    float h, l;
};

__device__ __forceinline__ void two_sum_into(F2 &acc, float b)
{
    const float s = __fadd_rn(acc.h, b);
    const float bb = __fsub_rn(s, acc.h);
    const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    acc.h = s;
    acc.l = __fadd_rn(acc.l, err);
}

// (h1, l1) + (h2, l2) with one TwoSum on the heads and a renormalising
// Fast2Sum (Dekker): deterministic for a fixed operand order.
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    F2 r;
    r.h = __fadd_rn(s, e);
    r.l = __fsub_rn(e, __fsub_rn(r.h, s));
    return r;
}

struct AccMix {
    float ax, ay, az, jx, jy, jz, p;  // current chunk
    F2 Ax, Ay, Az, Jx, Jy, Jz, P;     // running compensated sums
    __device__ void zero()
    {
        ax = ay = az = jx = jy = jz = p = 0.f;
        Ax = Ay = Az = Jx = Jy = Jz = P = F2{0.f, 0.f};
    }
    __device__ void fold()
    {
        two_sum_into(Ax, ax); two_sum_into(Ay, ay); two_sum_into(Az, az);
        two_sum_into(Jx, jx); two_sum_into(Jy, jy); two_sum_into(Jz, jz);
        two_sum_into(P, p);
        ax = ay = az = jx = jy = jz = p = 0.f;
    }
};

struct IMix {
    float xh, yh, zh, xl, yl, zl, vx, vy, vz;
};

__device__ __forceinline__ void load_i(const RecMix *rec, int64_t i, IMix &o)
{
    const RecMix r = rec[i];
    o.xh = r.hm.x; o.yh = r.hm.y; o.zh = r.hm.z;
    o.xl = r.lo.x; o.yl = r.lo.y; o.zl = r.lo.z;
    o.vx = r.v.x; o.vy = r.v.y; o.vz = r.v.z;
}

__device__ __forceinline__ void interact(const IMix &I, const RecMix &J, bool self, float eps2, AccMix &A)
{
    // i-j difference of the float pairs: (hi_j - hi_i) + (lo_j - lo_i)
    const float dx = __fadd_rn(__fsub_rn(J.hm.x, I.xh), __fsub_rn(J.lo.x, I.xl));
    const float dy = __fadd_rn(__fsub_rn(J.hm.y, I.yh), __fsub_rn(J.lo.y, I.yl));
    const float dz = __fadd_rn(__fsub_rn(J.hm.z, I.zh), __fsub_rn(J.lo.z, I.zl));
    const float wx = J.v.x - I.vx, wy = J.v.y - I.vy, wz = J.v.z - I.vz;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    r2 = self ? 1.f : r2;
    const float mj = self ? 0.f : J.hm.w;
    const float rw = fmaf(dx, wx, fmaf(dy, wy, dz * wz));
    // 1/sqrt: hardware estimate, then one Newton-Raphson step
    // y <- y + (y/2) h, h = 1 - r2 y^2, with the residual formed exactly
    // (r2 y = p + e by an FMA) so the step lands within ~1/2 ulp.
    const float y0 = rsqrtf(r2);
    const float pr = r2 * y0;
    const float er = fmaf(r2, y0, -pr);
    const float hres = fmaf(-er, y0, fmaf(-pr, y0, 1.f));
    const float rinv = fmaf(0.5f * y0, hres, y0);
    const float rinv2 = rinv * rinv;
    const float mr = mj * rinv;
    const float mr3 = mr * rinv2;
    const float al = 3.f * rw * rinv2;
    A.p += mr;
    A.ax = fmaf(mr3, dx, A.ax);
    A.ay = fmaf(mr3, dy, A.ay);
    A.az = fmaf(mr3, dz, A.az);
    A.jx = fmaf(mr3, fmaf(-al, dx, wx), A.jx);
    A.jy = fmaf(mr3, fmaf(-al, dy, wy), A.jy);
    A.jz = fmaf(mr3, fmaf(-al, dz, wz), A.jz);
}

// ---------------------------------------------- cross-slice reductions
__device__ __forceinline__ void acc_shfl_add(AccF64 &A, int off)
{
    A.ax += __shfl_xor_sync(0xffffffffu, A.ax, off);
    A.ay += __shfl_xor_sync(0xffffffffu, A.ay, off);
    A.az += __shfl_xor_sync(0xffffffffu, A.az, off);
    A.jx += __shfl_xor_sync(0xffffffffu, A.jx, off);
    A.jy += __shfl_xor_sync(0xffffffffu, A.jy, off);
    A.jz += __shfl_xor_sync(0xffffffffu, A.jz, off);
    A.p += __shfl_xor_sync(0xffffffffu, A.p, off);
}

__device__ __forceinline__ F2 f2_shfl(F2 a, int off)
{
    F2 b;
    b.h = __shfl_xor_sync(0xffffffffu, a.h, off);
    b.l = __shfl_xor_sync(0xffffffffu, a.l, off);
    // operand order by lane bit keeps both partners bitwise identical
    return ((threadIdx.x & off) == 0) ? f2_add(a, b) : f2_add(b, a);
}

__device__ __forceinline__ void acc_shfl_add(AccMix &A, int off)
{
    A.Ax = f2_shfl(A.Ax, off); A.Ay = f2_shfl(A.Ay, off); A.Az = f2_shfl(A.Az, off);
    A.Jx = f2_shfl(A.Jx, off); A.Jy = f2_shfl(A.Jy, off); A.Jz = f2_shfl(A.Jz, off);
    A.P = f2_shfl(A.P, off);
}

// Adds the partner's sums (lane + delta) into this lane's where `take`; every
// lane takes part in the shuffles.  The receiving lane's sums come first, so
// the order of every addition is fixed.
__device__ __forceinline__ double shfl_down_take(double x, int delta, bool take)
{
    const double o = __shfl_down_sync(0xffffffffu, x, delta);
    return take ? x + o : x;
}

__device__ __forceinline__ void acc_shfl_down_add(AccF64 &A, int delta, bool take)
{
    A.ax = shfl_down_take(A.ax, delta, take);
    A.ay = shfl_down_take(A.ay, delta, take);
    A.az = shfl_down_take(A.az, delta, take);
    A.jx = shfl_down_take(A.jx, delta, take);
    A.jy = shfl_down_take(A.jy, delta, take);
    A.jz = shfl_down_take(A.jz, delta, take);
    A.p = shfl_down_take(A.p, delta, take);
}

__device__ __forceinline__ F2 f2_shfl_down_take(F2 a, int delta, bool take)
{
    F2 o;
    o.h = __shfl_down_sync(0xffffffffu, a.h, delta);
    o.l = __shfl_down_sync(0xffffffffu, a.l, delta);
    return take ? f2_add(a, o) : a;
}

__device__ __forceinline__ void acc_shfl_down_add(AccMix &A, int delta, bool take)
{
    A.Ax = f2_shfl_down_take(A.Ax, delta, take);
    A.Ay = f2_shfl_down_take(A.Ay, delta, take);
    A.Az = f2_shfl_down_take(A.Az, delta, take);
    A.Jx = f2_shfl_down_take(A.Jx, delta, take);
    A.Jy = f2_shfl_down_take(A.Jy, delta, take);
    A.Jz = f2_shfl_down_take(A.Jz, delta, take);
    A.P = f2_shfl_down_take(A.P, delta, take);
}

struct RedF64 {
    double v[7];
};
struct RedMix {
    F2 v[7];
};

__device__ __forceinline__ void to_red(const AccF64 &A, RedF64 &r)
{
    r.v[0] = A.ax; r.v[1] = A.ay; r.v[2] = A.az; r.v[3] = A.jx; r.v[4] = A.jy; r.v[5] = A.jz; r.v[6] = A.p;
}
__device__ __forceinline__ void to_red(const AccMix &A, RedMix &r)
{
    r.v[0] = A.Ax; r.v[1] = A.Ay; r.v[2] = A.Az; r.v[3] = A.Jx; r.v[4] = A.Jy; r.v[5] = A.Jz; r.v[6] = A.P;
}
__device__ __forceinline__ double red_get(const RedF64 &r, int q) { return r.v[q]; }
__device__ __forceinline__ double red_get(const RedMix &r, int q) { return (double)r.v[q].h + (double)r.v[q].l; }
// partial sums written by other CTAs are read through L2 (bypassing L1)
// One component of a reduction record (double, or an FP32 pair).
__device__ __forceinline__ double shfl_down_e(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ F2 shfl_down_e(const F2 &v, int d)
{
    F2 r;
    r.h = __shfl_down_sync(0xffffffffu, v.h, d);
    r.l = __shfl_down_sync(0xffffffffu, v.l, d);
    return r;
}
__device__ __forceinline__ void comp_add(double &a, double b) { a += b; }
__device__ __forceinline__ void comp_add(F2 &a, const F2 &b) { a = f2_add(a, b); }
__device__ __forceinline__ double comp_get(double a) { return a; }
__device__ __forceinline__ double comp_get(const F2 &a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ double ld_comp_cg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ F2 ld_comp_cg(const F2 *p)
{
    F2 r;
    r.h = __ldcg(&p->h);
    r.l = __ldcg(&p->l);
    return r;
}

template <typename Rec>
struct Traits;
template <>
struct Traits<RecF64> {
    using I = IF64;
    using Acc = AccF64;
    using Red = RedF64;
    using Eps = double;
};
template <>
struct Traits<RecMix> {
    using I = IMix;
    using Acc = AccMix;
    using Red = RedMix;
    using Eps = float;
};

__device__ __forceinline__ void fold_chunk(AccF64 &) {}
__device__ __forceinline__ void fold_chunk(AccMix &A) { A.fold(); }

// ------------------------------------------------------------ list force
// One 128-thread group (4 warps) per work item = (tile, part of its group's
// list).  With n_a active particles in the tile each warp holds floor(32 /
// n_a) j slices of n_a lanes (lane = i slot + n_a * slice; leftover lanes
// idle), and the slices stride through each staged chunk of the part.
// Slices are summed in a fixed order (shuffles, then warps).  A list split
// into several parts leaves per-part sums in the partials buffer; the group
// that finishes a tile's last part (acquire-release arrival counter: no
// waiting) adds the parts in part order.  So each particle's result depends
// only on its list, its tile's active count and the part length, never on
// scheduling.
// Asynchronous global -> shared copies (16 B each) for chunk staging,
// cached in L1: the 16-byte pieces of one record, and the records of
// neighbouring list entries (consecutive particles of a leaf, sibling
// cells), share sectors, which L1 then serves instead of L2.  Measured on
// real tree lists (N = 65536, staging alone) at 1.0e11 records/s against
// 5.9e10 through L2 only.  The records are rewritten every block step, but
// always before a grid barrier or a kernel boundary that orders them before
// these (weak) reads, as for any plain load.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename Rec>
__device__ __forceinline__ void cp_async_rec(Rec *dst, const Rec *src)
{
    static_assert(sizeof(Rec) % 16 == 0, "records are whole 16-byte pieces");
#pragma unroll
    for (int q = 0; q < (int)(sizeof(Rec) / 16); q++)
        cp_async16(reinterpret_cast<char *>(dst) + 16 * q, reinterpret_cast<const char *>(src) + 16 * q);
}

// Staged list chunks per 128-thread group: one is summed while kStages - 1
// are in flight.  (Three stages measured no faster in the tree loop and up to
// 18% slower for short list parts: the deeper prologue adds latency to every
// part, and parts are only a few chunks long.)
constexpr int kStages = 2;

template <typename Rec, int TJ>
struct ForceSmem {
    Rec rec[kStages][TJ];  // ring of staged list chunks
    int32_t idx[kStages][TJ];
    typename Traits<Rec>::Red red[kThreads / 32][kMaxTileI];
    int item;
    int last;
    double tn[kThreads / 32];  // per-warp minimum of t + dt after the corrector
    int lv[kMaxTileI];         // new step level of each corrected particle, by active index
    double fin[kMaxTileI][7];  // the completed tile's new acc, jerk, pot by active index (for its corrector)
};

// GPU-scope acquire / release operations (PTX memory model): an
// acquire-release arrival on a counter sees every earlier arrival's writes and
// passes its own on, without full fences.
__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int *p, unsigned int v)
{
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_max_gpu(unsigned int *p, unsigned int v)
{
    asm volatile("red.release.gpu.global.max.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier over the 128 threads working on one item: the whole CTA
// (bar_id 0) or one of several 128-thread worker groups of a larger CTA
// (named barrier bar_id = 1 + group).
__device__ __forceinline__ void group_sync(int bar_id)
{
    if (bar_id == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(kThreads) : "memory");
}

// item = (tile, part | sim << 16, active mask, parts of the tile); tid is
// the thread's index in its 128-thread group.  Returns true (in every thread
// of the group) for the item that wrote the tile's final forces.
template <typename Rec, int TJ, bool kMapI>
__device__ __forceinline__ bool force_item(const State &s, const Rec *__restrict__ rec, const Lists &L,
                                           typename Traits<Rec>::Eps eps2, const WorkItem &it,
                                           ForceSmem<Rec, TJ> &sm, unsigned long long &n_int, const int tid,
                                           const int bar_id)
{
    using T = Traits<Rec>;
    using Red = typename T::Red;
    const int lane = tid & 31, warp = tid >> 5;
    Red *partials = reinterpret_cast<Red *>(L.partials);
    const int p0 = it.p_begin;
    const uint32_t mask = it.mask;
    const int n_a = __popc(mask);
    const int pj = it.part_len;
    const int part = it.part_sim & 0xFFFF, slot0 = it.slot;

    // Lane mapping: every warp holds K = floor(32 / n_a) j slices of n_a lanes
    // (lane = i slot + n_a * slice); the 32 - K n_a leftover lanes idle.  So no
    // lane is spent on a missing particle (rounding n_a up to a power of two
    // left up to half the lanes idle, and the FP64 pipe charges the whole warp).
    const int I = n_a;
    const int K = 32 / I;
    const int islot = lane % I, kslice = lane / I;
    const bool idle = kslice >= K;
    const int jslice = warp * K + kslice;
    const int S = (kThreads / 32) * K;
    const bool has_i = !idle;
    int64_t pi = -1;
    {
        uint32_t mm = mask;
        for (int q = 0; q < islot && mm; q++) mm &= mm - 1;
        if (has_i) pi = p0 + (__ffs(mm) - 1);
    }
    int64_t pload = has_i ? pi : p0 + (__ffs(mask) - 1);  // spare slots repeat a live one; dropped
    if constexpr (kMapI) {
        // slots are positions in a caller's active list; i is its j index
        pload = L.i_map[pload];
        if (has_i) pi = pload;
    }
    typename T::I Iv;
    load_i(rec, pload, Iv);
    typename T::Acc A;
    A.zero();

    const int64_t gb = it.gb, ge = it.ge;
    const int n_parts = parts_of(ge - gb, pj);
    const int64_t lb = gb + (int64_t)part * pj;
    const int64_t le = min(ge, lb + (int64_t)pj);
    const int64_t len = le - lb;
    if (tid == 0 && part == 0) n_int += (unsigned long long)n_a * (unsigned long long)(ge - gb - 1);
    // Chunks of TJ list entries are staged in a ring of kStages shared
    // buffers: while one is summed, cp.async fills the next kStages - 1; the
    // list indices of the chunk after those are already loading into
    // registers.  Every step commits one copy group (empty past the end), so
    // waiting for all but the newest kStages - 1 groups means chunk c landed.
    constexpr int EPT = TJ / kThreads;  // staged entries per thread and chunk
    const int n_chunks = (int)((len + TJ - 1) / TJ);
    int32_t nxt[EPT];
    auto load_idx = [&](int c) {
#pragma unroll
        for (int q = 0; q < EPT; q++) {
            const int64_t e = (int64_t)c * TJ + q * kThreads + tid;
            nxt[q] = (c < n_chunks && e < len) ? L.idx[lb + e] : -1;
        }
    };
    auto issue = [&](int c) {  // chunk c's records into buffer c % kStages, indices from nxt
        if (c < n_chunks) {
            const int b = c % kStages;
#pragma unroll
            for (int q = 0; q < EPT; q++) {
                const int e = q * kThreads + tid;
                sm.idx[b][e] = nxt[q];
                if (nxt[q] >= 0) cp_async_rec(&sm.rec[b][e], &rec[nxt[q]]);
            }
        }
        cp_async_commit();
    };
    if (n_chunks > 0) {
#pragma unroll
        for (int k = 0; k < kStages - 1; k++) {
            load_idx(k);
            issue(k);
        }
        load_idx(kStages - 1);
    }
    for (int c = 0; c < n_chunks; c++) {
        const int b = c % kStages;
        const int nc = (len - (int64_t)c * TJ < (int64_t)TJ) ? (int)(len - (int64_t)c * TJ) : TJ;
        issue(c + kStages - 1);  // into the buffer summed in step c - 1 (freed by its closing barrier)
        load_idx(c + kStages);
        cp_async_wait<kStages - 1>();
        group_sync(bar_id);
        // FP32 partials are folded into the compensated sums every
        // kFold terms per thread (short plain-FP32 runs keep the
        // partial-sum rounding below the per-term rounding).
        for (int e = idle ? nc : jslice; e < nc;) {
            const int e_end = min(nc, e + kFold * S);
            for (; e < e_end; e += S) {
                const int32_t j = sm.idx[b][e];
                interact(Iv, sm.rec[b][e], (int64_t)j == pi, eps2, A);
            }
            fold_chunk(A);
        }
        group_sync(bar_id);  // buffer b is refilled by the next step's issue
    }
    // Plain form: sum over the group's 4 K slices for each (i slot,
    // component): the partials go to shared memory, then P contiguous lanes of
    // one warp (P a power of two, P * 7 n_a <= 128) each add a contiguous run
    // of slices in order and a shuffle tree adds the P runs.  A fixed order,
    // with about 4 K / P + log2 P adds per thread, where a butterfly over the
    // lanes costs 7 adds per level for every lane (a warp instruction costs the
    // FP64 pipe the same with one lane active).  With P = 1 a thread may own
    // two outputs (7 n_a <= 224).  Mixed form (FP32 pair adds are cheap, the
    // extra barriers are not): a butterfly over the lanes when n_a is a power
    // of two, else a tree towards slice 0, then a sum over the four warps.
    constexpr bool kTreeTail = std::is_same<Rec, RecF64>::value;
    if (!kTreeTail) {
        if ((I & (I - 1)) == 0) {
            for (int off = I; off < 32; off <<= 1) acc_shfl_add(A, off);
        } else {
            for (int step = 1; step < K; step <<= 1)
                acc_shfl_down_add(A, step * I, !idle && (kslice & (2 * step - 1)) == 0 && kslice + step < K);
        }
    }
    if (kTreeTail ? !idle : lane < I) {
        Red rr;
        to_red(A, rr);
        sm.red[warp][lane] = rr;
    }
    group_sync(bar_id);
    using E = typename std::remove_reference<decltype(sm.red[0][0].v[0])>::type;
    const int n_out = 7 * n_a;
    const int n_sl = kTreeTail ? (kThreads / 32) * K : kThreads / 32;  // terms per output
    int P = 1;  // (mixed form: one thread per output, warps 0..3 in order)
    if (kTreeTail)
        while (P < 32 && 2 * P * n_out <= kThreads && 2 * P <= n_sl) P <<= 1;
    const int per = (n_sl + P - 1) / P;
    E r[2] = {E{}, E{}};
    bool has[2] = {false, false};
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int t = tid + u * kThreads;
        const int o = t / P, q = t - o * P;
        if ((u == 0 || P == 1) && o < n_out) {
            const int slot = o / 7, comp = o - 7 * slot;
            const int x1 = min(n_sl, (q + 1) * per);
            for (int x = q * per; x < x1; x++) {
                const int w = kTreeTail ? x / K : x, k = kTreeTail ? x - w * K : 0;
                const E v = sm.red[w][k * I + slot].v[comp];
                if (has[u]) comp_add(r[u], v);
                else {
                    r[u] = v;
                    has[u] = true;
                }
            }
        }
        if (u == 0)
            for (int off = P >> 1; off > 0; off >>= 1) {  // P is the same in every lane
                const E ov = shfl_down_e(r[0], off);
                const bool oh = __shfl_down_sync(0xffffffffu, (int)has[0], off) != 0;
                if (q < off && oh) {
                    if (has[0]) comp_add(r[0], ov);
                    else {
                        r[0] = ov;
                        has[0] = true;
                    }
                }
            }
    }
    // the sums, one per output, back into slot order: thread t then holds
    // output t (and t + 128) for the part merge below (already so when P = 1)
    if (P > 1) {
        group_sync(bar_id);
        E *outv = &sm.red[0][0].v[0];
        const int o = tid / P;
        if (o < n_out && tid - o * P == 0) outv[o] = r[0];
        group_sync(bar_id);
        if (tid < n_out) r[0] = outv[tid];
    }
    bool write_out = n_parts == 1;
    if (n_parts > 1) {
        // the group's partials are ordered before its arrival by the group
        // barrier and the arrival's release; the last arrival's acquire (and
        // the barrier after it) orders the other parts' partials before the sum
        Red *mine = partials + ((int64_t)slot0 + part) * kMaxTileI;
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int t = tid + u * kThreads, slot = t / 7, comp = t - 7 * (t / 7);
            if (t < n_out) mine[slot].v[comp] = r[u];
        }
        group_sync(bar_id);
        if (tid == 0) {
            const unsigned int old = atom_add_acq_rel_gpu(reinterpret_cast<unsigned int *>(&L.tile_cnt[it.tile]), 1u);
            sm.last = ((int)old == n_parts - 1);
        }
        group_sync(bar_id);
        write_out = sm.last;
        if (write_out) {
            const Red *base = partials + (int64_t)slot0 * kMaxTileI;
            // Parts are added in blocks of kMergeBlock consecutive parts (more
            // if the block sums would not fit the staging buffers, idle now):
            // (output, block) pairs over all the group's threads each add
            // their block's parts in part order, every load issued first;
            // then each output adds its block sums in block order.  The order
            // depends only on the number of parts, so results stay
            // deterministic; with at most kMergeBlock parts it is the plain
            // sequence p0 + p1 + p2 + ...  A long sequential chain of
            // dependent adds would otherwise dominate a small block step split
            // into many short parts.
            E *buf = reinterpret_cast<E *>(&sm.rec[0][0]);
            constexpr int kBuf = (int)(sizeof(sm.rec) / sizeof(E));
            constexpr int kMergeBlock = 8;
            int blk = kMergeBlock;
            while ((int64_t)n_out * ((n_parts + blk - 1) / blk) > kBuf) blk *= 2;
            const int n_blk = (n_parts + blk - 1) / blk;
            for (int x = tid; x < n_out * n_blk; x += kThreads) {
                const int b = x / n_out, o = x - b * n_out;
                const int q0 = b * blk, q1 = min(n_parts, q0 + blk);
                const Red *src = base + o / 7;
                const int comp = o - 7 * (o / 7);
                E vals[kMergeBlock];
#pragma unroll
                for (int k = 0; k < kMergeBlock; k++)
                    if (q0 + k < q1) vals[k] = ld_comp_cg(&src[(int64_t)(q0 + k) * kMaxTileI].v[comp]);
                E acc = vals[0];
#pragma unroll
                for (int k = 1; k < kMergeBlock; k++)
                    if (q0 + k < q1) comp_add(acc, vals[k]);
                for (int q = q0 + kMergeBlock; q < q1; q++)  // blocks longer than kMergeBlock
                    comp_add(acc, ld_comp_cg(&src[(int64_t)q * kMaxTileI].v[comp]));
                buf[x] = acc;
            }
            group_sync(bar_id);
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int t = tid + u * kThreads;
                if (t < n_out) {
                    r[u] = buf[t];
                    for (int b = 1; b < n_blk; b++) comp_add(r[u], buf[b * n_out + t]);
                }
            }
            if (tid == 0) L.tile_cnt[it.tile] = 0;
        }
    }
    if (write_out) {
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int t = tid + u * kThreads, slot = t / 7, comp = t - 7 * (t / 7);
            if (t < n_out) {
                uint32_t mm = mask;
                for (int q = 0; q < slot; q++) mm &= mm - 1;
                const int64_t p = p0 + (__ffs(mm) - 1);
                const double v = comp_get(r[u]);
                sm.fin[slot][comp] = v;
                if (comp < 3) s.acc1[comp * s.cap_n + p] = v;
                else if (comp < 6) s.jerk1[(comp - 3) * s.cap_n + p] = v;
                else s.pot1[p] = -v;
            }
        }
    }
    // callers put a barrier before the shared buffers are reused
    return write_out;
}

template <typename Rec, int TJ, bool kMapI = false>
__global__ void __launch_bounds__(kThreads, 6) k_force(State s, const Rec *__restrict__ rec, Lists L, DevScalars *ds,
                                                    StepCtl c, Params prm)
{
    double tnow;
    if (!step_time(ds, c, &tnow)) return;
    __shared__ ForceSmem<Rec, TJ> sm;
    const int n_items = (int)ds->n_items;
    const typename Traits<Rec>::Eps eps2 = (typename Traits<Rec>::Eps)prm.eps2;
    unsigned long long n_int = 0;
    for (;;) {
        if (threadIdx.x == 0) sm.item = (int)atomicAdd(&ds->work, 1u);
        __syncthreads();
        const int item = sm.item;
        if (item >= n_items) break;
        force_item<Rec, TJ, kMapI>(s, rec, L, eps2, L.items[item], sm, n_int, threadIdx.x, 0);
        // the next iteration's first barrier protects sm reuse
    }
    if (threadIdx.x == 0 && n_int) atomicAdd(&ds->interactions, n_int);
}

// -------------------------------------------------------------- corrector
__device__ __forceinline__ double norm3(double a, double b, double c) { return sqrt(a * a + b * b + c * c); }

// Largest power of two <= |x| for finite x, as frexp / ldexp give it (so 1/2
// for a zero, whose frexp exponent is 0), on the bits.
__device__ __forceinline__ long long pow2_floor_abs_bits(long long W)
{
    const long long b = W & 0x7FFFFFFFFFFFFFFFll;
    if (b == 0) return 0x3FE0000000000000ll;                          // 1/2
    if ((b >> 52) == 0) return 1ll << (63 - __clzll((unsigned long long)b));  // subnormal: its top bit
    return b & (long long)0xFFF0000000000000ull;
}

// fmod(t, 2^k) == 0 on t's bits: t finite and a multiple of 2^k (fmod of an
// infinity or a NaN is a NaN, so those are not).
__device__ __forceinline__ bool multiple_of_pow2(double t, int k)
{
    const long long b = __double_as_longlong(t) & 0x7FFFFFFFFFFFFFFFll;  // |t|
    if (b == 0) return true;
    const int ef = (int)(b >> 52);
    if (ef == 0x7ff) return false;
    const long long m = ef ? ((b & 0xFFFFFFFFFFFFFll) | (1ll << 52)) : b;  // |t| = m 2^(max(ef, 1) - 1075)
    return (ef ? ef : 1) - 1075 + (__ffsll(m) - 1) >= k;
}

// Block quantisation (McMillan 1986): the largest power of two <= want, at
// most double the old step, doubled only where t_new is a multiple of the
// new step, clamped to [dt_min, dt_max]; a NaN keeps the old step and an
// infinity asks to double.  (The largest power of two below |want| follows
// frexp, so a zero asks for 1/2.)  When dt_old is a normal power of two (as
// in the block-step loops) and dt_min, dt_max are positive normal values,
// every candidate is a positive power of two, IEEE order is the integer order
// of the bits and the multiple test is exact on t_new's bits: the path below
// then uses no FP64 instruction (the FP64 pipe is narrow); otherwise the same
// rule runs in FP64.
__device__ __forceinline__ double block_dt(double want, double dt_old, double t_new, double dt_min, double dt_max)
{
    const long long O = __double_as_longlong(dt_old), Mn = __double_as_longlong(dt_min),
                    Mx = __double_as_longlong(dt_max);
    const long long kNormLo = 0x0010000000000000ll, kTop = 0x7FE0000000000000ll;  // normal, doubling stays finite
    if (O >= kNormLo && O < kTop && (O & 0xFFFFFFFFFFFFFll) == 0 && Mn >= kNormLo && Mn < 0x7FF0000000000000ll && Mx >= kNormLo &&
        Mx < 0x7FF0000000000000ll) {
        const long long W = __double_as_longlong(want);
        const long long O2 = O + (1ll << 52);  // 2 dt_old
        long long Q;
        if ((W & 0x7FF0000000000000ll) == 0x7FF0000000000000ll) Q = (W & 0xFFFFFFFFFFFFFll) ? O : O2;  // NaN, inf
        else Q = pow2_floor_abs_bits(W);
        if (Q > O2) Q = O2;
        if (Q > O && !multiple_of_pow2(t_new, (int)((Q >> 52) & 0x7ff) - 1023)) Q = O;
        if (Q > Mx) Q = Mx;
        if (Q < Mn) Q = Mn;
        return __longlong_as_double(Q);
    }
    double q;
    if (isnan(want)) q = dt_old;
    else if (isinf(want)) q = 2.0 * dt_old;
    else {
        int e;
        frexp(want, &e);
        q = ldexp(1.0, e - 1);
    }
    if (q > 2.0 * dt_old) q = 2.0 * dt_old;
    if (q > dt_old && fmod(t_new, q) != 0.0) q = dt_old;
    if (q > dt_max) q = dt_max;
    if (q < dt_min) q = dt_min;
    return q;
}

__device__ __forceinline__ void atomic_min_time(unsigned long long *slot, double t)
{
    atomicMin(slot, (unsigned long long)__double_as_longlong(t));
}

// Hermite corrector (Makino & Aarseth 1992) for the active particles:
// a2 = (-6 (a0 - a1) - D (4 j0 + 2 j1)) / D^2, a3 = (12 (a0 - a1) + 6 D (j0 + j1)) / D^3,
// x1 = x_p + a2 D^4/24 + a3 D^5/120, v1 = v_p + a2 D^3/6 + a3 D^4/24;
// new step from Aarseth's criterion at the end of the step.
//
// The FP64 pipe is narrow on this GPU (a warp instruction issues in 64
// cycles per SM sub-partition), so the corrector avoids FP64 divisions and
// roots: D is the particle's power-of-two step, so 1/D^2 and 1/D^3 are exact
// powers of two, and the timestep criterion is screened in FP32.  The
// per-component arithmetic and the order of every sum are shared by the
// one-thread-per-particle and the three-lanes-per-particle correctors, so
// both give the same bits.

// Powers of D (a power of two) needed by the corrector, exact.
struct StepPowers {
    double D, iD2, iD3, D3, D4;
};

__device__ __forceinline__ StepPowers step_powers(double D)
{
    StepPowers P;
    P.D = D;
    const long long b = __double_as_longlong(D);
    if ((b & ((1ll << 52) - 1)) == 0 && b > 0) {
        const int e = (int)((b >> 52) & 0x7ff) - 1023;  // D = 2^e
        auto p2 = [](int k) { return __longlong_as_double((long long)(1023 + k) << 52); };
        P.iD2 = p2(-2 * e);
        P.iD3 = p2(-3 * e);
        P.D3 = p2(3 * e);
        P.D4 = p2(4 * e);
    } else {  // not reached from the block-step loops (D is a level step)
        const double iD = 1.0 / D;
        P.iD2 = iD * iD;
        P.iD3 = P.iD2 * iD;
        P.D3 = D * D * D;
        P.D4 = D * D * D * D;
    }
    return P;
}

// One Cartesian component: state (x, v, a0, j0) at t, new force (a1, j1) at
// t + D.  Returns the corrected x, v and the a^(2) at t + D and a^(3).
struct CorrComp {
    double x, v, a2e, a3;
};

__device__ __forceinline__ CorrComp correct_component(double x, double v, double a0, double j0, double a1, double j1,
                                                      const StepPowers &P)
{
    const double D = P.D;
    const double h = 0.5 * D, th = D * (1.0 / 3.0);
    const double xp = x + D * (v + h * (a0 + th * j0));
    const double vp = v + D * (a0 + h * j0);
    const double a2 = (-6.0 * (a0 - a1) - D * (4.0 * j0 + 2.0 * j1)) * P.iD2;
    const double a3 = (12.0 * (a0 - a1) + 6.0 * D * (j0 + j1)) * P.iD3;
    CorrComp c;
    c.x = xp + P.D4 * (a2 * (1.0 / 24.0) + a3 * D * (1.0 / 120.0));
    c.v = vp + P.D3 * (a2 * (1.0 / 6.0) + a3 * D * (1.0 / 24.0));
    c.a2e = a2 + a3 * D;
    c.a3 = a3;
    return c;
}

// |u|^2 from the components' squares, summed x, y, z with single roundings.
__device__ __forceinline__ double norm2_of(double sx, double sy, double sz) { return __dadd_rn(__dadd_rn(sx, sy), sz); }
__device__ __forceinline__ double sq(double u) { return __dmul_rn(u, u); }

// Aarseth's criterion dt^2 = eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2) from
// A = |a|^2, J = |j|^2, S = |a2|^2, T = |a3|^2.  Only the largest power of
// two below dt is used (block_dt), so it is screened in FP32, which keeps the
// narrow FP64 pipe free.
//
// The criterion is invariant under a change of time unit (J, S, T scale as
// c^-2, c^-4, c^-6 and dt as c) and under a common factor on A, J, S, T.  So
// the four norms are first normalised by exact powers of two taken from the
// exponents of A and J (A' in [1, 2), J' in [1, 8)), which brings the
// shortest steps' huge higher derivatives into FP32 range, and the power of
// two found for the normalised step is shifted back.  The screen works on
// w2 = dt'^2 itself: the power of two below dt' = sqrt(w2) is 2^floor(e / 2)
// for w2's exponent e, and its boundaries are w2's even powers of two.
// Error bound of the FP32 w2 against the exact value of the same normalised
// inputs: truncation to FP32 2^-23 per input (and eta), the square roots as
// y rsqrtf(y) (rsqrtf within 2 ulp), the quotient by __fdividef (within 2
// ulp), the sums of positive terms and the products: at most 24 * 2^-24 in
// all.  When w2 is at least 128 ulps (>= 2^-17 relative) from the even power
// of two on its side (the lower one for an even exponent, the upper one for
// an odd exponent), the exact value and the FP64 expression (within ~1e-15 of
// it) lie between the same two even powers of two, and the exact power of two
// below the FP64 value is returned.  Otherwise (near a boundary, zero or
// non-normal inputs, normalised values outside [2^-60, 2^61), eta outside
// [2^-30, 2^30], or products and steps near the FP64 range's ends, where the
// FP64 expression itself would lose range) the FP64 expression decides.
__device__ __forceinline__ int exp2_of(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023; }

// x * 2^m in FP32 for a positive normal double x, mantissa truncated; the
// caller keeps the exponent in FP32's normal range.
__device__ __forceinline__ float f32_scaled(double x, int m)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff) - 1023 + m;
    return __int_as_float(((e + 127) << 23) | (int)((b >> 29) & 0x7fffff));
}

__device__ __forceinline__ bool normal_pos(double x)
{
    const long long b = __double_as_longlong(x);
    return b >= 0x0010000000000000ll && b < 0x7ff0000000000000ll;
}

__device__ __forceinline__ double aarseth_want(double A, double J, double S, double T, double eta)
{
    if (normal_pos(A) && normal_pos(J) && normal_pos(S) && normal_pos(T) && eta >= 0x1p-30 && eta <= 0x1p30) {
        const int eA = exp2_of(A), eJ = exp2_of(J), eS = exp2_of(S), eT = exp2_of(T);
        const int k = (eJ - eA) >> 1;  // 2^2k ~ J / A: the time unit
        const int mA = -eA, mJ = -eA - 2 * k, mS = -eA - 4 * k, mT = -eA - 6 * k;
        const int xS = eS + mS, xT = eT + mT;
        // the FP64 expression of the original inputs stays finite and normal
        const bool fp64_ok = eA + eS > -1000 && eA + eS < 1000 && eJ + eT > -1000 && eJ + eT < 1000;
        if (fp64_ok && xS >= -60 && xS <= 60 && xT >= -60 && xT <= 60) {
            const float Af = f32_scaled(A, mA), Jf = f32_scaled(J, mJ), Sf = f32_scaled(S, mS), Tf = f32_scaled(T, mT);
            const float p1 = Af * Sf, p2 = Jf * Tf;
            const float num = p1 * rsqrtf(p1) + Jf, den = p2 * rsqrtf(p2) + Sf;
            const float w2 = f32_scaled(eta, 0) * __fdividef(num, den);
            const int wb = __float_as_int(w2);
            const int frac = wb & 0x7fffff, ex = (wb >> 23) & 0xff;
            const int e = ex - 127, odd = e & 1;
            const int e2 = (e >> 1) - k;  // dt = sqrt(w2) / 2^k: exponent of the power of two below dt
            if (ex > 0 && ex < 255 && (odd ? frac <= 0x7fffff - 128 : frac >= 128) && e2 > -400 && e2 < 400)
                return __longlong_as_double((long long)(e2 + 1023) << 52);
        }
    }
    return sqrt(eta * (sqrt(A * S) + J) / (sqrt(J * T) + S));
}

__device__ __forceinline__ void correct_particle(const State &s, int64_t p, double tnow, const Params &prm)
{
    const StepPowers P = step_powers(tnow - s.t[p]);
    double sa[3], sj[3], ss[3], st[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double a0 = s.a[d * s.cap_j + p], j0 = s.jk[d * s.cap_j + p];
        const double a1 = s.acc1[d * s.cap_n + p];
        const double j1 = s.jerk1[d * s.cap_n + p];
        const CorrComp c = correct_component(s.x[d * s.cap_j + p], s.v[d * s.cap_j + p], a0, j0, a1, j1, P);
        s.x[d * s.cap_j + p] = c.x;
        s.v[d * s.cap_j + p] = c.v;
        s.a[d * s.cap_j + p] = a1;
        s.jk[d * s.cap_j + p] = j1;
        sa[d] = sq(a1);
        sj[d] = sq(j1);
        ss[d] = sq(c.a2e);
        st[d] = sq(c.a3);
    }
    const double want = aarseth_want(norm2_of(sa[0], sa[1], sa[2]), norm2_of(sj[0], sj[1], sj[2]),
                                     norm2_of(ss[0], ss[1], ss[2]), norm2_of(st[0], st[1], st[2]), prm.eta);
    const double dtn = block_dt(want, s.dt[p], tnow, prm.dt_min, prm.dt_max);
    s.t[p] = tnow;
    s.dt[p] = dtn;
    if (s.base) refresh_base(s, p);
}

static __global__ void k_correct(State s, DevScalars *ds, StepCtl c, Params prm)
{
    double tnow;
    if (!step_time(ds, c, &tnow)) return;
    const int64_t n = ds->n;
    double my_min = __longlong_as_double(0x7FF0000000000000LL);
    int my_cnt = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const bool act = is_active(s, c, p, tnow);
        if (act) {
            if (c.mode == 1 && s.t[p] + s.dt[p] != tnow) {
                atomicExch(&ds->err, -1);  // HH_EINVAL: marked particle not due at t
                continue;
            }
            correct_particle(s, p, tnow, prm);
            my_cnt++;
        }
        const double tn = s.t[p] + s.dt[p];
        my_min = tn < my_min ? tn : my_min;
    }
    if (c.mode != 0) return;
    // block min, then one atomic per CTA
    for (int off = 16; off > 0; off >>= 1) {
        my_min = fmin(my_min, __shfl_xor_sync(0xffffffffu, my_min, off));
        my_cnt += __shfl_xor_sync(0xffffffffu, my_cnt, off);
    }
    __shared__ double s_min[32];
    __shared__ int s_cnt[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_min[warp] = my_min;
        s_cnt[warp] = my_cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mn = s_min[0];
        int cn = s_cnt[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            mn = fmin(mn, s_min[w]);
            cn += s_cnt[w];
        }
        atomic_min_time(&ds->tmin[c.slot_next], mn);
        if (blockIdx.x == 0) {  // the force kernel of this step has finished
            ds->n_items = 0u;
            ds->slot_ctr = 0u;
        }
        if (cn) {
            atomicAdd(&ds->n_act_last, cn);
            atomicAdd(&ds->particle_steps, (unsigned long long)cn);
        }
    }
}

// min over particles of t_i + dt_i into tmin[slot] (slot preset to +inf).
static __global__ void k_min_time(State s, DevScalars *ds, int slot)
{
    const int64_t n = ds->n;
    double my_min = __longlong_as_double(0x7FF0000000000000LL);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const double tn = s.t[p] + s.dt[p];
        my_min = tn < my_min ? tn : my_min;
    }
    for (int off = 16; off > 0; off >>= 1) my_min = fmin(my_min, __shfl_xor_sync(0xffffffffu, my_min, off));
    if ((threadIdx.x & 31) == 0) atomic_min_time(&ds->tmin[slot], my_min);
}

// Initial step from eta_s |a| / |jk|, quantised (reading: the paper is silent).
static __global__ void k_init_dt(State s, DevScalars *ds, Params prm)
{
    const int64_t n = ds->n;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const double na = norm3(s.a[p], s.a[s.cap_j + p], s.a[2 * s.cap_j + p]);
        const double nj = norm3(s.jk[p], s.jk[s.cap_j + p], s.jk[2 * s.cap_j + p]);
        double q;
        if (nj == 0.0) q = prm.dt_max;
        else {
            const double want = prm.eta_s * na / nj;
            q = (want > 0.0 && want < 1.0e300) ? pow2_floor(want) : prm.dt_max;
        }
        if (q > prm.dt_max) q = prm.dt_max;
        if (q < prm.dt_min) q = prm.dt_min;
        s.dt[p] = q;
    }
}

// a, jk of every particle <- last force results (initial forces).
static __global__ void k_adopt_forces(State s, DevScalars *ds)
{
    const int64_t n = ds->n;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            s.a[d * s.cap_j + p] = s.acc1[d * s.cap_n + p];
            s.jk[d * s.cap_j + p] = s.jerk1[d * s.cap_n + p];
        }
        if (s.base) refresh_base(s, p);
    }
}

static __global__ void k_refresh_base(State s, int64_t first, int64_t n)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        refresh_base(s, first + q);
}

static __global__ void k_set_marks(int32_t *mark, const int32_t *idx, int32_t n, int32_t value)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) mark[idx[q]] = value;
}

// out[3][n_act] (SoA) <- acc1 etc. at i_idx
static __global__ void k_gather_out(State s, const int32_t *idx, int32_t n_act, double *acc, double *jerk, double *pot)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_act; q += gridDim.x * blockDim.x) {
        const int64_t p = idx[q];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (acc) acc[(int64_t)d * n_act + q] = s.acc1[d * s.cap_n + p];
            if (jerk) jerk[(int64_t)d * n_act + q] = s.jerk1[d * s.cap_n + p];
        }
        if (pot) pot[q] = s.pot1[p];
    }
}

// Device-side input validation for *_dev uploads: finite values, m > 0.
static __global__ void k_check_j(const State s, int64_t first, int64_t n, DevScalars *ds)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = first + q;
        bool ok = s.m[e] > 0.0 && isfinite(s.m[e]) && isfinite(s.t[e]);
        for (int d = 0; d < 3; d++)
            ok = ok && isfinite(s.x[d * s.cap_j + e]) && isfinite(s.v[d * s.cap_j + e]) &&
                 isfinite(s.a[d * s.cap_j + e]) && isfinite(s.jk[d * s.cap_j + e]);
        if (!ok) atomicExch(&ds->err, -1);
    }
}

static __global__ void k_check_idx(const int32_t *idx, int32_t n, int64_t n_part, DevScalars *ds)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        if (idx[q] < 0 || idx[q] >= n_part) atomicExch(&ds->err, -1);
}

}  // namespace hh
