// Batched, persistent block-step loop: one cooperative launch
// advances many independent simulations, each by its own block steps (Section 2,
// tree-loop steps 2-7), until each reaches its stop time or the step budget.
//
// A "global step" gives every live simulation one block step, in two
// phases separated by grid barriers:
//   1. predict every j entry of every live simulation to its own block time
//      and append the work items of tiles with active particles (one shared
//      queue for all simulations);
//   2. CTAs pull (simulation, tile, list part) items and run the same
//      force_item body as the single-simulation kernel; the worker group
//      that completes a tile's forces corrects its particles at once and
//      lowers, per simulation, the min of t_i + dt_i that starts its next
//      block step.
// Per-step counters alternate between two copies by step parity, so the
// copy of the previous step is cleared while this step fills the other.
// Uneven active sets and list lengths of different simulations share one
// queue, so small block steps of many simulations fill the GPU together.
// Results of a simulation do not depend on what else is in the batch: its
// tiles, active masks and list parts are its own, and sums run in fixed order.
//
// A run is one captured CUDA graph (upload of the descriptors, the launch,
// read-back of the outputs), replayed with new descriptors each time.
//
// Grid barriers spin with an iteration limit; on expiry the kernel records
// HH_ETIMEOUT and every CTA returns.

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>

#include "hh_ctx.h"

using namespace hh;

namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;  // a barrier wait gives up after 2 s
constexpr long long kSpinLimit = 1ll << 28;            // iteration backstop for the same wait
constexpr int kGroups = 4;                   // 128-thread worker groups per CTA (one CTA per SM)
constexpr int kBlock = kThreads * kGroups;
constexpr int kSimCache = 256;               // simulations whose step data a CTA keeps in shared memory
constexpr int kSdCache = 32;                 // simulations whose descriptors a CTA keeps in shared memory

struct SimDesc {
    State st;
    const void *rec;
    Lists L;
    uint32_t *tile_lv;  // levels present in each tile
    DevScalars *ds;
    int64_t n, nj;
    int32_t n_tiles, pj, work, work_split, pj_small;
    int32_t lmax;  // longest group list
    int64_t lbar;  // mean list length per group (list entries / groups)
    Params prm;
    double t_end;
};

struct BatchScalars {
    unsigned int bar_count;  // grid-barrier arrivals; top bit: an error was raised
    int32_t err;
    uint32_t work[2];     // force queue head, by step parity
    uint32_t n_items[2];  // work items, by step parity
    uint32_t max_chunks[2];  // longest list part of a list-mode simulation in 32-entry chunks, by step parity
    int32_t steps_done;
};

// What changes from one run to the next, read by the kernel from device
// memory, so that the launch itself (captured once in a CUDA graph) keeps
// fixed arguments.
struct BatchHdr {
    int32_t n_sims;
    int32_t max_steps;
    WorkItem *items;  // work queue (grows with the simulations' list parts; at least kGroups x grid)
};

struct BatchDev {
    const BatchHdr *hdr;
    const SimDesc *sims;                   // [max_sims]
    const int64_t *jbase, *pbase, *tbase;  // prefix sums [n_sims + 1], each of capacity max_sims + 1
    BatchScalars *bs;
    unsigned long long *step_ns;  // [3 max_steps + 1] global timer at the start and after each phase
    double *t_next_out;           // [max_sims]
};

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier for a cooperative launch (all CTAs resident).  Arrivals
// count up monotonically within a launch (the host zeroes the counter), so
// an arrival's count tells which barrier it belongs to: barrier b is passed
// once the counter reaches (b + 1) x gridDim.x.  Each CTA's threads
// synchronise with its arriving thread first; the arrival is an
// acquire-release add, and the waiters poll the counter itself with acquire
// loads.  The adds form one release sequence, so a waiter that reads the
// final count has seen every CTA's writes, and the last arrival is released
// by its own add: no second write and no second round trip through L2.
//
// Errors travel in the counter's top bit: raise_error sets it, every waiter
// sees it with the count it polls, and an arrival after it sees it in the
// value its add returns.  (A CTA that passed a barrier before another CTA
// failed runs one more phase and stops at the next barrier.)  Waits give up
// after kWaitNs / kSpinLimit with HH_ETIMEOUT.  Returns false once an error
// is known.
constexpr unsigned int kGenErr = 0x80000000u;

__device__ __forceinline__ void raise_error(BatchScalars *bs, int code)
{
    atomicExch(&bs->err, code);
    atomicOr(&bs->bar_count, kGenErr);
}

__device__ __forceinline__ bool grid_sync(BatchScalars *bs)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int v = atom_add_acq_rel_gpu(&bs->bar_count, 1u);
        const unsigned int cnt = v & ~kGenErr;
        const unsigned int target = (cnt / gridDim.x + 1u) * gridDim.x;
        int ok = (v & kGenErr) ? 0 : 1;
        if (ok && cnt + 1u < target) {
            long long it = 0;
            const unsigned long long t0 = globaltimer_ns();
            for (;;) {
                const unsigned int g = ld_acquire_gpu(&bs->bar_count);
                if (g & kGenErr) {
                    ok = 0;
                    break;
                }
                if (g >= target) break;
                if ((++it & 15) == 0 && (it > kSpinLimit || globaltimer_ns() - t0 > kWaitNs)) {
                    raise_error(bs, HH_ETIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ int find_sim(const int64_t *base, int n_sims, int64_t g)
{
    int lo = 0, hi = n_sims;  // base[lo] <= g < base[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ double sim_time(const SimDesc &sd, int par)
{
    return __longlong_as_double((long long)__ldcg(&sd.ds->tmin[par]));
}

// Block-step levels: a step dt = 2^-k has level k.  Power-of-two steps that
// start on multiples of themselves (the block rule) make every particle of
// level k due at the same time, the first multiple of 2^-k after the latest
// block time; at block time t the due particles are exactly those with
// levels >= kmin(t), where 2^-kmin(t) is the largest power of two dividing t.
__device__ __forceinline__ int level_of(double dt)
{
    return 1023 - (int)((__double_as_longlong(dt) >> 52) & 0x7ff);
}

__device__ __forceinline__ bool is_level_step(double dt)
{
    const long long b = __double_as_longlong(dt);
    const int lv = 1023 - (int)((b >> 52) & 0x7ff);
    return (b & ((1ll << 52) - 1)) == 0 && b > 0 && lv >= 0 && lv <= 31;
}

__device__ __forceinline__ double pow2i(int k)  // 2^k for |k| < 1000
{
    return __longlong_as_double((long long)(1023 + k) << 52);
}

__device__ __forceinline__ int kmin_of(double t)  // t > 0
{
    const long long b = __double_as_longlong(t);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const long long mant = (b & ((1ll << 52) - 1)) | (1ll << 52);
    const int z = __ffsll(mant) - 1;
    const int k = 52 - z - e;
    return k < 0 ? 0 : k;
}

// Earliest due time after block time t of the occupied levels below kmin(t)
// (those particles are not corrected at t, so their due times stand).
// Warp-collective: lane k looks at level k, all lanes return the minimum.
__device__ __forceinline__ double due_below_warp(const int32_t *lvl_cnt, double t, int kmin)
{
    const int k = threadIdx.x & 31;
    double m = __longlong_as_double(0x7FF0000000000000LL);
    if (k < kmin && __ldcg(&lvl_cnt[k]) > 0) m = (floor(t * pow2i(k)) + 1.0) * pow2i(-k);
    for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
    return m;
}

// Step 6 for the due particles of one tile (mask over its lanes), three
// lanes per particle (one Cartesian component each), ten particles per warp
// and round (particles k_first + 10 r' ... of the active list, rounds k_step
// apart): a warp instruction costs the same on the FP64 pipe whether one lane
// or 32 are active, so this cuts the corrector's FP64 issue per small step
// about threefold.  Same arithmetic as correct_particle, component by
// component.  Returns (in every lane) the minimum of t + dt over the tile's
// corrected particles, updates the simulation's level histogram and leaves
// each corrected particle's new level in lv_out[its index among the active].
// The new forces come from fin[active index] (the force tail's copy in
// shared memory; the same values as acc1 / jerk1).
__device__ __forceinline__ double correct_tile_3lane(const SimDesc &sd, const int4 td, uint32_t mask, double tnow,
                                                     int lane, int k_first, int k_step, int *lv_out,
                                                     const double (*fin)[7])
{
    const unsigned full = 0xffffffffu;
    const State &s = sd.st;
    const int na = __popc(mask);
    const int q = lane / 3, d = lane - 3 * q, g = 3 * q;
    // next times are positive and finite: their minimum is the integer minimum
    // of the bit patterns (no FP64 instruction)
    unsigned long long tn_min = 0x7FF0000000000000ull;
    for (int base = k_first; base < na; base += k_step) {
        const int k = base + q;
        const bool on = lane < 30 && k < na;
        const int64_t p = on ? td.x + (__fns(mask, 0, k + 1)) : td.x;
        double sa = 0.0, sj = 0.0, ss = 0.0, st = 0.0, a1 = 0.0, j1 = 0.0, dt_old = 1.0;
        CorrComp c{};
        if (on) {
            dt_old = s.dt[p];
            const StepPowers P = step_powers(tnow - s.t[p]);
            const double a0 = s.a[d * s.cap_j + p], j0 = s.jk[d * s.cap_j + p];
            a1 = fin[k][d];
            j1 = fin[k][3 + d];
            c = correct_component(s.x[d * s.cap_j + p], s.v[d * s.cap_j + p], a0, j0, a1, j1, P);
            sa = sq(a1);
            sj = sq(j1);
            ss = sq(c.a2e);
            st = sq(c.a3);
        }
        // the particle's three lanes: g, g + 1, g + 2 (lanes 30, 31 are idle)
        const double A = norm2_of(__shfl_sync(full, sa, g), __shfl_sync(full, sa, g + 1), __shfl_sync(full, sa, g + 2));
        const double J = norm2_of(__shfl_sync(full, sj, g), __shfl_sync(full, sj, g + 1), __shfl_sync(full, sj, g + 2));
        const double S = norm2_of(__shfl_sync(full, ss, g), __shfl_sync(full, ss, g + 1), __shfl_sync(full, ss, g + 2));
        const double T = norm2_of(__shfl_sync(full, st, g), __shfl_sync(full, st, g + 1), __shfl_sync(full, st, g + 2));
        __syncwarp();  // every lane has read t and dt before any is rewritten
        if (on) {
            const double dtn = block_dt(aarseth_want(A, J, S, T, sd.prm.eta), dt_old, tnow, sd.prm.dt_min,
                                        sd.prm.dt_max);
            s.x[d * s.cap_j + p] = c.x;
            s.v[d * s.cap_j + p] = c.v;
            s.a[d * s.cap_j + p] = a1;
            s.jk[d * s.cap_j + p] = j1;
            if (s.base) refresh_base_values(s, p, d, c.x, c.v, a1, j1, d == 0 ? s.m[p] : 0.0);
            if (d == 0) {
                s.t[p] = tnow;
                s.dt[p] = dtn;
                const int lv_old = level_of(dt_old), lv_new = level_of(dtn);
                lv_out[k] = lv_new;
                if (lv_new != lv_old) {
                    atomicSub(&sd.ds->lvl_cnt[lv_old], 1);
                    atomicAdd(&sd.ds->lvl_cnt[lv_new & 31], 1);
                }
                tn_min = min(tn_min, (unsigned long long)__double_as_longlong(tnow + dtn));
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) tn_min = min(tn_min, __shfl_xor_sync(full, tn_min, off));
    return __longlong_as_double((long long)tn_min);
}

// Per-CTA copy of each simulation's block time for the current step
// (read once per phase instead of once per element).
struct StepCache {
    double t[kSimCache];
    double t_end[kSimCache];
    int due[kSimCache];                  // particles due at t (levels >= kmin(t)); -1: not counted
    unsigned char list_mode[kSimCache];  // predict only the entries of this step's list parts
    int any_list;                        // some simulation of the batch is in list mode this step
    int any_full;                        // some live simulation predicts every entry this step
};

// Due particles of a simulation at block time tnow: its level histogram's
// levels >= kmin(tnow) (nobody writes the histogram during phase 1, so
// every CTA counts alike).
__device__ __forceinline__ int due_count(const SimDesc &sd, double tnow)
{
    const int k0 = kmin_of(tnow);
    int due = 0;
#pragma unroll
    for (int k = 0; k < 32; k++) {
        const int c = __ldcg(&sd.ds->lvl_cnt[k]);
        due += k >= k0 ? c : 0;
    }
    return due;
}

// A small block step of a large simulation references few of its j entries:
// its due tiles' lists.  Then predicting those (in a phase after the tile
// selection) is cheaper than predicting every entry.  The choice compares the
// due particles times the mean list length with the number of j entries, and
// applies only to simulations whose every-entry pass costs more than the
// extra phase and grid barrier (a few microseconds): at least kListModeMinJ
// entries.  (Many small simulations together gain nothing from it: their
// every-entry passes are short and run side by side.)  It changes no result:
// a predicted record is the same whoever computes it.
constexpr int64_t kListModeMinJ = 1 << 18;

__device__ __forceinline__ bool list_mode_of(const SimDesc &sd, double tnow, int due)
{
    constexpr int64_t kDiv = 2;  // list entries counted with their repeats across a step's tiles
    if (sd.nj < kListModeMinJ || !(tnow <= sd.t_end) || !(tnow > 0.0)) return false;
    return (int64_t)due * sd.lbar * kDiv < sd.nj;
}

__device__ __forceinline__ void cache_times(StepCache &c, const SimDesc *sims, int n_sims, int par)
{
    if (threadIdx.x == 0) {
        c.any_list = 0;
        c.any_full = n_sims > kSimCache;  // (simulations beyond the cache predict every entry)
    }
    __syncthreads();
    int any = 0, full = 0;
    for (int s = threadIdx.x; s < n_sims && s < kSimCache; s += blockDim.x) {
        c.t[s] = __longlong_as_double((long long)__ldcg(&sims[s].ds->tmin[par]));
        c.t_end[s] = sims[s].t_end;
        // (counted here only where list mode may apply: the count is one
        // more round trip to L2 on the path of every step)
        const int due = sims[s].nj >= kListModeMinJ ? due_count(sims[s], c.t[s]) : -1;
        c.due[s] = due;
        const bool lm = due >= 0 && list_mode_of(sims[s], c.t[s], due);
        c.list_mode[s] = lm;
        any |= lm;
        full |= !lm && c.t[s] <= c.t_end[s];
    }
    if (any) c.any_list = 1;
    if (full) c.any_full = 1;
    __syncthreads();
}

// List mode of simulation s (simulations beyond the cache predict every entry).
__device__ __forceinline__ bool cached_list_mode(const StepCache &c, int s)
{
    return s < kSimCache && c.list_mode[s];
}

__device__ __forceinline__ double cached_time(const StepCache &c, const SimDesc *sims, int s, int par)
{
    return s < kSimCache ? c.t[s] : __longlong_as_double((long long)__ldcg(&sims[s].ds->tmin[par]));
}

// Running (simulation, min of t_i + dt_i, corrected count) of one thread;
// a change of simulation flushes the previous one with atomics.
struct MinCnt {
    int s;
    double m;
    int c;
};

__device__ __forceinline__ void mc_flush(const SimDesc *sims, const MinCnt &a, int slot)
{
    if (a.s < 0) return;
    atomicMin(&sims[a.s].ds->tmin[slot], (unsigned long long)__double_as_longlong(a.m));
    if (a.c) {
        atomicAdd(&sims[a.s].ds->particle_steps, (unsigned long long)a.c);
        atomicAdd(&sims[a.s].ds->n_act_last, a.c);
    }
}

__device__ __forceinline__ void mc_push(const SimDesc *sims, MinCnt &a, int s, double tn, int cnt, int slot)
{
    if (a.s != s) {
        mc_flush(sims, a, slot);
        a.s = s;
        a.m = tn;
        a.c = cnt;
    } else {
        a.m = fmin(a.m, tn);
        a.c += cnt;
    }
}

// CTA-wide combination of the threads' running values: one atomic per
// simulation run of consecutive warps (all warps of a CTA usually share one
// simulation, so a phase costs one atomic per CTA).
__device__ __forceinline__ void mc_block_flush(const SimDesc *sims, MinCnt a, int slot)
{
    __shared__ int w_s[kBlock / 32];
    __shared__ double w_m[kBlock / 32];
    __shared__ int w_c[kBlock / 32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int smax = __reduce_max_sync(full, a.s);
    const bool same = __all_sync(full, a.s < 0 || a.s == smax);
    if (!same) {
        mc_flush(sims, a, slot);
        if (lane == 0) w_s[warp] = -1;
    } else {
        double m = a.s < 0 ? __longlong_as_double(0x7FF0000000000000LL) : a.m;
        int c = a.s < 0 ? 0 : a.c;
        for (int off = 16; off > 0; off >>= 1) {
            m = fmin(m, __shfl_xor_sync(full, m, off));
            c += __shfl_xor_sync(full, c, off);
        }
        if (lane == 0) {
            w_s[warp] = smax;
            w_m[warp] = m;
            w_c[warp] = c;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        MinCnt acc{-1, 0.0, 0};
        for (int w = 0; w < kBlock / 32; w++) {
            if (w_s[w] < 0) continue;
            if (acc.s != w_s[w]) {
                mc_flush(sims, acc, slot);
                acc = MinCnt{w_s[w], w_m[w], w_c[w]};
            } else {
                acc.m = fmin(acc.m, w_m[w]);
                acc.c += w_c[w];
            }
        }
        mc_flush(sims, acc, slot);
    }
    __syncthreads();
}

template <typename Rec, int TJ>
__global__ void __launch_bounds__(kBlock, 1) k_batch(BatchDev B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ StepCache sc;
    __shared__ SimDesc sd_sm[kGroups];  // each worker group's current simulation (for its corrector)
    // Descriptors do not change during a launch: the first kSdCache live in
    // shared memory, so a worker reaches a simulation's arrays without an L2
    // round trip at the start of every item and every corrector.
    __shared__ SimDesc sd_all[kSdCache];
    __shared__ int64_t base_sm[3][kSdCache + 1];  // jbase, pbase, tbase of a batch of <= kSdCache simulations
    // each worker group's current and next work item (by item parity): kept
    // in shared memory instead of 12 registers live across the whole item
    __shared__ WorkItem it_sm[kGroups][2];
    static_assert(sizeof(SimDesc) % 8 == 0 && sizeof(SimDesc) / 8 <= kThreads - 64, "descriptor copy by 64 threads");
    const int tid = threadIdx.x;
    const int group = tid / kThreads, gt = tid - group * kThreads;
    ForceSmem<Rec, TJ> &sm = reinterpret_cast<ForceSmem<Rec, TJ> *>(smem_raw)[group];
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + tid;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int n_sims = B.hdr->n_sims, max_steps = B.hdr->max_steps;
    WorkItem *const items = B.hdr->items;
    const int64_t NJ = B.jbase[n_sims], NP = B.pbase[n_sims], NT = B.tbase[n_sims];
    for (int w = tid; w < min(n_sims, kSdCache) * (int)(sizeof(SimDesc) / 8); w += blockDim.x)
        reinterpret_cast<long long *>(sd_all)[w] = reinterpret_cast<const long long *>(B.sims)[w];
    const bool small_batch = n_sims <= kSdCache;
    if (small_batch)
        for (int w = tid; w < 3 * (n_sims + 1); w += blockDim.x) {
            const int a = w / (n_sims + 1), q = w - a * (n_sims + 1);
            base_sm[a][q] = (a == 0 ? B.jbase : a == 1 ? B.pbase : B.tbase)[q];
        }
    // (visible after the first grid barrier's block barrier, before any use below it)
    auto SD = [&](int s) -> const SimDesc & { return s < kSdCache ? sd_all[s] : B.sims[s]; };
    const int64_t *const JB = small_batch ? base_sm[0] : B.jbase;
    const int64_t *const PB = small_batch ? base_sm[1] : B.pbase;
    const int64_t *const TB = small_batch ? base_sm[2] : B.tbase;

    // phase 0: every simulation's first block time, latest time, level
    // histogram and tile level masks; the block rule is checked here
    if (blockIdx.x == 0)
        for (int s = tid; s < n_sims; s += blockDim.x) {
            DevScalars *ds = B.sims[s].ds;
            ds->tmin[0] = 0x7FF0000000000000ull;
            ds->tmin[1] = 0x7FF0000000000000ull;
            ds->t_cur_bits = 0ull;
            ds->slot_par[0] = ds->slot_par[1] = 0u;
            for (int k = 0; k < 32; k++) ds->lvl_cnt[k] = 0;
        }
    if (blockIdx.x == 0 && tid == 0) B.step_ns[0] = globaltimer_ns();
    if (!grid_sync(B.bs)) return;
    {
        MinCnt acc{-1, 0.0, 0};
        const int lane = tid & 31;
        for (int64_t g0 = gtid - lane; g0 < NP; g0 += nth) {  // warp-aligned so that lanes can aggregate
            const int64_t g = g0 + lane;
            const bool valid = g < NP;
            int s = -1, lv = -1;
            double t = 0.0, dt = 0.0;
            if (valid) {
                s = find_sim(PB, n_sims, g);
                const SimDesc &sd = SD(s);
                const int64_t p = g - PB[s];
                t = sd.st.t[p];
                dt = sd.st.dt[p];
                if (!is_level_step(dt) || !(t >= 0.0)) {
                    raise_error(B.bs, HH_EINVAL);
                } else {
                    lv = level_of(dt);
                    const double u = t * pow2i(lv);
                    if (u != floor(u)) raise_error(B.bs, HH_EINVAL);  // t_i not a multiple of dt_i
                }
                mc_push(B.sims, acc, s, t + dt, 0, 0);
            }
            // histogram and latest time: lanes of one simulation and level combine
            const unsigned grp = __match_any_sync(0xffffffffu, valid ? s * 64 + (lv & 63) : -1);
            const int leader = __ffs(grp) - 1;
            double tmax = t;
            for (unsigned m2 = grp; m2; m2 &= m2 - 1) tmax = fmax(tmax, __shfl_sync(grp, t, __ffs(m2) - 1));
            if (valid && lane == leader && lv >= 0) {
                DevScalars *ds = B.sims[s].ds;
                atomicAdd(&ds->lvl_cnt[lv], __popc(grp));
                atomicMax(&ds->t_cur_bits, (unsigned long long)__double_as_longlong(tmax));
            }
        }
        mc_block_flush(B.sims, acc, 0);
        const int64_t w0 = gtid >> 5, nw = nth >> 5;
        for (int64_t wt = w0; wt < NT; wt += nw) {
            const int s = find_sim(TB, n_sims, wt);  // warp-uniform
            const SimDesc &sd = SD(s);
            const int tile = (int)(wt - TB[s]);
            const int4 td = sd.L.tiles[tile];
            const int64_t p = td.x + lane;
            const uint32_t bit = (p < td.y) ? (1u << (level_of(sd.st.dt[p]) & 31)) : 0u;
            const uint32_t m = __reduce_or_sync(0xffffffffu, bit);
            if (lane == 0) sd.tile_lv[tile] = m;
        }
    }
    if (!grid_sync(B.bs)) return;
    if (blockIdx.x == 0)
        for (int s = tid; s < n_sims; s += blockDim.x) {
            const DevScalars *ds = B.sims[s].ds;
            const double tcur = __longlong_as_double((long long)__ldcg(&ds->t_cur_bits));
            if (!(sim_time(B.sims[s], 0) > tcur)) raise_error(B.bs, HH_EINVAL);  // an overdue particle
        }

    int step = 0;
    bool prev_full = true;  // the last step predicted every entry of some simulation
    for (; step < max_steps; step++) {
        const int par = step & 1;
        // ---- phase 1: select + predict
        // The inputs of this thread's first predicted entry (mixed form; the
        // plain form's FP64 inputs would not fit in registers, and its
        // predictor is bound by the FP64 pipe) do not depend on the block
        // time: their loads go out before the block times are read, unless
        // the last step predicted only list entries (then this one likely
        // does too, and the loads would be wasted).
        constexpr bool kEarly = std::is_same<Rec, RecMix>::value;
        constexpr bool kPlain = std::is_same<Rec, RecF64>::value;
        constexpr bool kExactChunks = std::is_same<Rec, RecMix>::value;
        PredIn<Rec> in0;
        const int s_p0 = gtid < NJ ? find_sim(JB, n_sims, gtid) : 0;
        const bool early = kEarly && prev_full && gtid < NJ;
        if (early) pred_load<Rec>(SD(s_p0).st, gtid - JB[s_p0], in0);
        cache_times(sc, B.sims, n_sims, par);
        prev_full = sc.any_full;
        // counters of the previous step (other parity) are free again
        if (blockIdx.x == 0 && tid == 0) {
            B.bs->work[par ^ 1] = 0u;
            B.bs->n_items[par ^ 1] = 0u;
            B.bs->max_chunks[par ^ 1] = 0u;
        }
        {
            // one warp per simulation, spread over the CTAs (a loop in one
            // CTA put a latency chain per 16 simulations on every step)
            const int wpb = (int)(blockDim.x >> 5);
            for (int s = (int)blockIdx.x * wpb + (tid >> 5); s < n_sims; s += (int)gridDim.x * wpb) {
                // the next block time starts from the due times of the levels
                // not corrected now; the corrector lowers it with the
                // corrected ones.  A finished simulation keeps its time.
                DevScalars *ds = B.sims[s].ds;
                const double tnow = cached_time(sc, B.sims, s, par);
                const bool live = tnow <= B.sims[s].t_end;
                const double below = due_below_warp(ds->lvl_cnt, tnow, kmin_of(tnow));
                if ((tid & 31) == 0) {
                    ds->tmin[par ^ 1] = live ? (unsigned long long)__double_as_longlong(below) : ds->tmin[par];
                    ds->n_act_last = 0;
                    ds->slot_par[par ^ 1] = 0u;
                    if (live) ds->block_steps += 1ull;
                    if (live && cached_list_mode(sc, s)) ds->list_steps += 1ull;
                }
            }
        }
        {
            // Tile selection: warp w takes tiles w + k W (W warps, k = 0,
            // 1, ...); its lanes read the level masks of 32 of them per round
            // trip, and the warp then builds the items of the due ones among
            // them, one tile at a time.  It runs before the prediction: the
            // few warps of a small step that find due tiles wait on chains of
            // loads and atomics while the others' predictions use the pipes.
            const int lane = tid & 31;
            const int64_t w0 = gtid >> 5, nw = nth >> 5;
            for (int64_t k0 = 0; w0 + k0 * nw < NT; k0 += 32) {
                const int64_t wt = w0 + (k0 + lane) * nw;
                int s_l = 0;
                bool due_l = false;
                if (wt < NT) {
                    s_l = find_sim(TB, n_sims, wt);
                    const SimDesc &sd = SD(s_l);
                    const double tnow = cached_time(sc, B.sims, s_l, par);
                    const uint32_t lv = sd.tile_lv[wt - TB[s_l]];
                    due_l = tnow <= sd.t_end && (lv >> kmin_of(tnow)) != 0u;  // a due level in this tile
                }
                for (uint32_t dmask = __ballot_sync(0xffffffffu, due_l); dmask; dmask &= dmask - 1) {
                    const int l = __ffs(dmask) - 1;
                    const int s = __shfl_sync(0xffffffffu, s_l, l);
                    const SimDesc &sd = SD(s);
                    const double tnow = cached_time(sc, B.sims, s, par);
                    const int tile = (int)(w0 + (k0 + l) * nw - TB[s]);
                    const int4 td = sd.L.tiles[tile];
                    const int64_t p = td.x + lane;
                    const bool act = (p < td.y) && (sd.st.t[p] + sd.st.dt[p] == tnow);
                    // equal-cost items in this step?  With work_split the
                    // simulation's due particles (levels >= kmin, from its
                    // level histogram, fixed during this phase) must reach
                    // work_split; below it the mixed form keeps parts of
                    // tile_j and the plain form takes equal-cost parts of
                    // kMedWork x tile_j interactions (an item's FP64 work
                    // bounds its time, so smaller items spread such a step
                    // over more SMs), and with tile_j_small, steps of at most
                    // kSmallDue due particles take parts of that length
                    int work = sd.work, pj = sd.pj;
                    if (sd.work_split > 0 || sd.pj_small > 0) {
                        int due;
                        if (s < kSimCache && sc.due[s] >= 0) {
                            due = sc.due[s];
                        } else {
                            const int cnt = __ldcg(&sd.ds->lvl_cnt[lane]);
                            due = __reduce_add_sync(0xffffffffu, lane >= kmin_of(tnow) ? cnt : 0);
                        }
                        if (sd.work_split > 0 && due < sd.work_split) {
                            work = kPlain ? kMedWork * sd.pj : 0;
                            if (kPlain) pj = 32;
                        }
                        if (sd.pj_small > 0 && due <= kSmallDue) {
                            work = 0;
                            pj = sd.pj_small;
                        }
                    }
                    const uint32_t mask = __ballot_sync(0xffffffffu, act);
                    if (mask)
                        append_tile_items(sd.L, tile, td, mask, pj, work, &B.bs->n_items[par], &sd.ds->slot_par[par],
                                          items, s, sd.ds->na_hist,
                                          kExactChunks && cached_list_mode(sc, s) ? &B.bs->max_chunks[par] : nullptr);
                }
            }
        }
        for (int64_t g = gtid; sc.any_full && g < NJ; g += nth) {
            const int s = g == gtid ? s_p0 : find_sim(JB, n_sims, g);
            const SimDesc &sd = SD(s);
            const double tnow = cached_time(sc, B.sims, s, par);
            if (!(tnow <= sd.t_end) || cached_list_mode(sc, s)) continue;
            if (early && g == gtid) pred_store<Rec>(in0, (Rec *)sd.rec, g - JB[s], tnow);
            else predict_entry<Rec>(sd.st, (Rec *)sd.rec, g - JB[s], tnow);
        }
        if (!grid_sync(B.bs)) return;
        if (sc.any_list) {
            // ---- phase 1b: list-mode simulations predict the entries of
            // this step's list parts.  A task is 32 consecutive entries of
            // one work item (lane = entry), up to the longest part, so the few
            // items of a small step spread over every SM.  The mixed form
            // tracks the step's longest part during the selection; the plain
            // form (whose registers that would spill) bounds it by the longest
            // part a list-mode simulation can have.  Entries shared by
            // several parts are predicted more than once, with the same
            // result.
            const uint32_t n_items = __ldcg(&B.bs->n_items[par]);
            int maxc = 1;
            if (kExactChunks) {
                maxc = max(1, (int)__ldcg(&B.bs->max_chunks[par]));
            } else {
                for (int s = 0; s < n_sims && s < kSimCache; s++)
                    if (cached_list_mode(sc, s)) {
                        // the longest part of any rule: tile_j, an equal-cost
                        // part of work_item or (below work_split) of kMedWork x
                        // tile_j interactions for one active particle
                        const SimDesc &sd = SD(s);
                        int plen = sd.pj;
                        if (sd.work > 0) plen = max(plen, part_len_for(1, sd.pj, sd.work));
                        if (kPlain && sd.work_split > 0) plen = max(plen, part_len_for(1, 32, kMedWork * sd.pj));
                        maxc = max(maxc, (min(plen, sd.lmax) + 31) / 32);
                    }
            }
            const int lane = tid & 31;
            const int64_t w0 = gtid >> 5, nw = nth >> 5;
            const int64_t n_tasks = (int64_t)n_items * maxc;
            for (int64_t task = w0; task < n_tasks; task += nw) {
                const int64_t i = task / maxc;
                const int c = (int)(task - i * maxc);
                const WorkItem &it = items[i];
                const int s = it.part_sim >> 16;
                if (!cached_list_mode(sc, s)) continue;  // warp-uniform
                const SimDesc &sd = SD(s);
                const int64_t lb = it.gb + (int64_t)(it.part_sim & 0xFFFF) * it.part_len;
                const int64_t le = min(it.ge, lb + (int64_t)it.part_len);
                const int64_t e = lb + 32 * (int64_t)c + lane;
                if (e < le) predict_entry<Rec>(sd.st, (Rec *)sd.rec, sd.L.idx[e], cached_time(sc, B.sims, s, par));
            }
            if (!grid_sync(B.bs)) return;
        }
        if (blockIdx.x == 0 && tid == 0) B.step_ns[3 * step + 1] = globaltimer_ns();

        // ---- phase 2: forces from the shared queue, one item per worker
        // group; the group that completes a tile corrects its particles
        // right away (step 6 needs only the particle's own new force)
        {
            const uint32_t n_items = __ldcg(&B.bs->n_items[par]);
            const int bar = 1 + group;
            const int gw = gt >> 5, glane = gt & 31;
            // The first item of every group is fixed, round-robin over the
            // SMs (item i -> SM i mod grid): the few items of a small step
            // land on different SMs instead of sharing one SM's FP64 pipe.
            // Later items come from the shared queue.
            // The queue holds at least n_static slots, so the first item is
            // read together with the count (and used only below it).
            const int n_static = (int)gridDim.x * kGroups;
            int item = group * (int)gridDim.x + (int)blockIdx.x;
            int ip = 0;  // parity of it_sm[group] holding the current item
            if (gt < 3)
                reinterpret_cast<int4 *>(&it_sm[group][0])[gt] = reinterpret_cast<const int4 *>(&items[item])[gt];
            group_sync(bar);
            for (;;) {
                if (item >= (int)n_items) break;
                const WorkItem &it = it_sm[group][ip];
                const int s = it.part_sim >> 16;
                const SimDesc &sd = SD(s);
                if (gt < 45) {
                    // the corrector's inputs (15 state arrays, <= 3 cache lines
                    // of each for the tile's <= 32 particles) into this SM's L1,
                    // in case this group completes the tile
                    const int arr = gt / 3, ln = gt - 3 * arr;
                    const State &st = sd.st;
                    const double *a = arr < 12 ? (arr < 3 ? st.x : arr < 6 ? st.v : arr < 9 ? st.a : st.jk) +
                                                     (int64_t)(arr % 3) * st.cap_j
                                               : (arr == 12 ? st.t : arr == 13 ? st.dt : st.m);
                    const int64_t q = min((int64_t)it.p_begin + 16 * ln, (int64_t)it.p_end - 1);
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(a + q));
                } else if (s >= kSdCache && gt >= 64 && gt < 64 + (int)(sizeof(SimDesc) / 8)) {
                    // and the simulation's descriptor into shared memory (the
                    // item's record staging through L1 may evict its lines)
                    reinterpret_cast<long long *>(&sd_sm[group])[gt - 64] =
                        reinterpret_cast<const long long *>(&B.sims[s])[gt - 64];
                }
                unsigned long long n_int = 0;
                const bool done = force_item<Rec, TJ, false>(sd.st, (const Rec *)sd.rec, sd.L,
                                                             (typename Traits<Rec>::Eps)sd.prm.eps2, it, sm, n_int,
                                                             gt, bar);
                if (gt == 0 && n_int) atomicAdd(&sd.ds->interactions, n_int);
                if (done) {
                    group_sync(bar);  // the tile's new forces are visible to the group
                    const SimDesc &sdc = s < kSdCache ? sd_all[s] : sd_sm[group];  // copied at the item's start
                    const double tnow = cached_time(sc, B.sims, s, par);
                    const int4 td = make_int4(it.p_begin, it.p_end, it.group, it.slot);
                    const uint32_t mask = it.mask;
                    // steps of the tile's particles that are not corrected now,
                    // loaded while the corrector runs
                    const int64_t pw = td.x + glane;
                    const double dt_keep = (gw == 0 && pw < td.y && !((mask >> glane) & 1u)) ? sdc.st.dt[pw] : 0.0;
                    const double tn =
                        correct_tile_3lane(sdc, td, mask, tnow, glane, 10 * gw, 10 * (kThreads / 32), sm.lv, sm.fin);
                    if (glane == 0) sm.tn[gw] = tn;
                    group_sync(bar);  // new levels and times are visible to the group
                    if (gw == 0) {
                        const bool corrected = (mask >> glane) & 1u;
                        const int lv = corrected ? sm.lv[__popc(mask & ((1u << glane) - 1u))] : level_of(dt_keep);
                        const uint32_t bit = (pw < td.y) ? (1u << (lv & 31)) : 0u;
                        const uint32_t lvm = __reduce_or_sync(0xffffffffu, bit);
                        if (glane == 0) {
                            double m = sm.tn[0];
                            for (int w = 1; w < kThreads / 32; w++)
                                if (__double_as_longlong(sm.tn[w]) < __double_as_longlong(m)) m = sm.tn[w];
                            const int c = __popc(mask);
                            sdc.tile_lv[it.tile] = lvm;
                            atomicMin(&sdc.ds->tmin[par ^ 1], (unsigned long long)__double_as_longlong(m));
                            atomicAdd(&sdc.ds->particle_steps, (unsigned long long)c);
                            atomicAdd(&sdc.ds->n_act_last, c);
                        }
                    }
                }
                // (with no more items than groups every item was a first item:
                // no queue round trip before the barrier)
                if (gt == 0) {
                    const int nx = (int)n_items <= n_static ? (int)n_items
                                                            : n_static + (int)atomicAdd(&B.bs->work[par], 1u);
                    sm.item = nx;
                    // the next item into the other slot (nobody reads it now)
                    if (nx < (int)n_items) {
                        const int4 *src = reinterpret_cast<const int4 *>(&items[nx]);
                        int4 *dst = reinterpret_cast<int4 *>(&it_sm[group][ip ^ 1]);
                        dst[0] = src[0];
                        dst[1] = src[1];
                        dst[2] = src[2];
                    }
                }
                group_sync(bar);  // also ends the use of the shared buffers by this item
                item = sm.item;   // rewritten only after the next item's group barriers
                ip ^= 1;
            }
        }
        if (!grid_sync(B.bs)) return;
        if (blockIdx.x == 0 && tid == 0) {
            const unsigned long long now = globaltimer_ns();
            B.step_ns[3 * step + 2] = now;
            B.step_ns[3 * step + 3] = now;  // the corrector ran inside the force phase
        }

        // any simulation still live for the next step?
        int live = 0;
        for (int s = tid; s < n_sims; s += blockDim.x) live |= sim_time(B.sims[s], par ^ 1) <= B.sims[s].t_end;
        if (!__syncthreads_or(live)) {
            step++;
            break;
        }
    }
    if (blockIdx.x == 0) {
        const int par = step & 1;
        for (int s = tid; s < n_sims; s += blockDim.x) B.t_next_out[s] = sim_time(B.sims[s], par);
        if (tid == 0) B.bs->steps_done = step;
    }
}

}  // namespace

// Host and device copies of one block holding everything a run uploads
// (header, simulation descriptors, prefix sums, zeroed scalars) followed by
// everything it reads back (scalars, next times, phase stamps), so that a run
// is one captured graph: one host-to-device copy, the cooperative launch and
// one device-to-host copy, all of fixed size.
struct BatchLayout {
    size_t hdr = 0, sims = 0, base = 0, bs = 0, tnext = 0, step_ns = 0, total = 0;
    size_t up_bytes() const { return bs + sizeof(BatchScalars); }
    size_t down_bytes() const { return total - bs; }
};

// A simulation admitted to a batch's resident set.
struct Resident {
    hh_ctx *ctx;
    double t_end;    // end of the run, a multiple of dt_tree
    double t_stop;   // next rebuild time (<= t_end)
    int64_t bytes;   // device bytes counted against the budget
    int state;       // 0 running, 1 finished (reached t_end), 2 failed rebuild
};

struct hh_batch {
    int device = 0;
    int precision = HH_FP64;
    int32_t max_sims = 0, max_steps = 0;
    int grid = 0;
    size_t smem = 0;
    cudaStream_t stream = nullptr;
    BatchLayout lay;
    unsigned char *d_blk = nullptr;  // device block
    unsigned char *h_blk = nullptr;  // pinned host mirror
    WorkItem *d_items = nullptr;
    int64_t cap_items = 0;
    cudaGraphExec_t graph = nullptr;  // upload, k_batch, read-back
    // resident set (hh_batch_admit / hh_batch_step / hh_batch_retire)
    int64_t budget = 0;               // device bytes of admitted contexts, 0 = no limit
    int64_t used = 0;
    int64_t launch_particles = 0;     // particles per launch, 0 = no limit
    size_t rr = 0;                    // round-robin start of the next launch
    std::vector<Resident> res;
    RbScratch *rb = nullptr;          // batched device rebuilds (made on first use)
    std::string err;
};

namespace {

int bfail(hh_batch *b, int code, const std::string &m)
{
    if (b) b->err = m;
    return hh_set_global_error(code, m.c_str());
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

BatchLayout batch_layout(int32_t max_sims, int32_t max_steps)
{
    BatchLayout L;
    L.hdr = 0;
    L.sims = align16(sizeof(BatchHdr));
    L.base = align16(L.sims + sizeof(SimDesc) * size_t(max_sims));
    L.bs = align16(L.base + sizeof(int64_t) * 3 * (size_t(max_sims) + 1));
    L.tnext = align16(L.bs + sizeof(BatchScalars));
    L.step_ns = align16(L.tnext + sizeof(double) * size_t(max_sims));
    L.total = L.step_ns + sizeof(unsigned long long) * (3 * size_t(max_steps) + 1);
    return L;
}

// Captures the run's graph on the batch stream (thread-local capture mode:
// other threads may use CUDA meanwhile).
int capture_graph(hh_batch *b)
{
    const BatchLayout &L = b->lay;
    unsigned char *d = b->d_blk;
    BatchDev B;
    B.hdr = reinterpret_cast<const BatchHdr *>(d + L.hdr);
    B.sims = reinterpret_cast<const SimDesc *>(d + L.sims);
    const int64_t *base = reinterpret_cast<const int64_t *>(d + L.base);
    B.jbase = base;
    B.pbase = base + (b->max_sims + 1);
    B.tbase = base + 2 * (size_t(b->max_sims) + 1);
    B.bs = reinterpret_cast<BatchScalars *>(d + L.bs);
    B.t_next_out = reinterpret_cast<double *>(d + L.tnext);
    B.step_ns = reinterpret_cast<unsigned long long *>(d + L.step_ns);
    void *args[] = {&B};
    const void *fn = b->precision == HH_MIXED ? (const void *)k_batch<RecMix, kTjMix>
                                              : (const void *)k_batch<RecF64, kTjF64>;
    cudaStream_t st = b->stream;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bfail(b, HH_ECUDA, "hh_batch_create: cannot begin graph capture");
    cudaError_t e = cudaMemcpyAsync(d, b->h_blk, L.up_bytes(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel(fn, dim3(b->grid), dim3(kBlock), args, b->smem, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_blk + L.bs, d + L.bs, L.down_bytes(), cudaMemcpyDeviceToHost, st);
    cudaGraph_t g = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(st, &g);
    if (e == cudaSuccess) e = e_end;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph = nullptr;
        return bfail(b, HH_ECUDA, std::string("hh_batch_create: graph capture: ") + cudaGetErrorString(e));
    }
    return HH_OK;
}

}  // namespace

extern "C" int hh_batch_create(hh_batch **out, int device, int precision, int32_t max_sims, int32_t max_steps)
{
    if (!out) return hh_set_global_error(HH_EINVAL, "hh_batch_create: out is NULL");
    *out = nullptr;
    if ((precision != HH_FP64 && precision != HH_MIXED) || max_sims < 1 || max_sims > 32767 || max_steps < 1 ||
        max_steps > (1 << 20))
        return hh_set_global_error(HH_EINVAL,
                                   "hh_batch_create: bad precision, max_sims (1..32767) or max_steps (1..2^20)");
    hh_batch *b = new (std::nothrow) hh_batch;
    if (!b) return hh_set_global_error(HH_ENOMEM, "hh_batch_create: out of host memory");
    b->device = device;
    b->precision = precision;
    b->max_sims = max_sims;
    b->max_steps = max_steps;
    auto bail = [&](int code, const char *m) {
        hh_batch_destroy(b);
        return hh_set_global_error(code, m);
    };
    if (cudaSetDevice(device) != cudaSuccess) return bail(HH_ECUDA, "hh_batch_create: cudaSetDevice failed");
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(HH_ECUDA, "hh_batch_create: stream creation failed");
    cudaDeviceProp prop;
    int coop = 0;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop)
        return bail(HH_ECUDA, "hh_batch_create: device lacks cooperative launch");
    int per = 0;
    if (precision == HH_MIXED) {
        b->smem = sizeof(ForceSmem<RecMix, kTjMix>) * kGroups;
        cudaFuncSetAttribute(k_batch<RecMix, kTjMix>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(b->smem));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<RecMix, kTjMix>, kBlock, b->smem);
    } else {
        b->smem = sizeof(ForceSmem<RecF64, kTjF64>) * kGroups;
        cudaFuncSetAttribute(k_batch<RecF64, kTjF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(b->smem));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<RecF64, kTjF64>, kBlock, b->smem);
    }
    if (per < 1) return bail(HH_ECUDA, "hh_batch_create: kernel does not fit on an SM");
    b->grid = prop.multiProcessorCount;  // one persistent CTA per SM
    b->lay = batch_layout(max_sims, max_steps);
    if (cudaMalloc(&b->d_blk, b->lay.total) != cudaSuccess ||
        cudaMallocHost(&b->h_blk, b->lay.total) != cudaSuccess) {
        cudaGetLastError();
        return bail(HH_ENOMEM, "hh_batch_create: allocation failed");
    }
    std::memset(b->h_blk, 0, b->lay.total);
    if (int rc = capture_graph(b)) {
        const std::string m = b->err;
        hh_batch_destroy(b);
        return hh_set_global_error(rc, m.c_str());
    }
    *out = b;
    return HH_OK;
}

extern "C" int hh_batch_set_ctas(hh_batch *b, int32_t n_ctas)
{
    if (!b) return hh_set_global_error(HH_EINVAL, "hh_batch_set_ctas: NULL batch");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, HH_ECUDA, "hh_batch_set_ctas: cudaSetDevice failed");
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
        return bfail(b, HH_ECUDA, "hh_batch_set_ctas: no SM count");
    const int32_t want = n_ctas > 0 ? n_ctas : sms + n_ctas;
    if (want < 1 || want > sms) return bfail(b, HH_EINVAL, "hh_batch_set_ctas: CTA count outside [1, SM count]");
    if (want == b->grid) return HH_OK;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, HH_ECUDA, "hh_batch_set_ctas: stream failed");
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->grid = want;
    return capture_graph(b);
}

extern "C" int hh_batch_destroy(hh_batch *b)
{
    if (!b) return HH_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->d_blk) cudaFree(b->d_blk);
    if (b->d_items) cudaFree(b->d_items);
    if (b->h_blk) cudaFreeHost(b->h_blk);
    if (b->rb) hh_rb_scratch_free(b->rb);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return HH_OK;
}

extern "C" int hh_batch_run(hh_batch *b, int32_t n, hh_ctx *const *ctxs, const double *t_end, int32_t max_steps,
                            int32_t *steps_out, double *t_next_out, double *step_us_out, double *phase_us_out)
{
    if (!b) return hh_set_global_error(HH_EINVAL, "hh_batch_run: NULL batch");
    if (n < 1 || n > b->max_sims || !ctxs || !t_end) return bfail(b, HH_EINVAL, "hh_batch_run: bad n or NULL arrays");
    if (max_steps < 1 || max_steps > b->max_steps) return bfail(b, HH_EINVAL, "hh_batch_run: max_steps out of range");
    if (!b->graph) return bfail(b, HH_ESTATE, "hh_batch_run: the batch has no captured launch (a failed re-capture)");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, HH_ECUDA, "hh_batch_run: cudaSetDevice failed");
    const BatchLayout &Ly = b->lay;
    SimDesc *sims = reinterpret_cast<SimDesc *>(b->h_blk + Ly.sims);
    int64_t *jb = reinterpret_cast<int64_t *>(b->h_blk + Ly.base);
    int64_t *pb = jb + (b->max_sims + 1), *tb = pb + (b->max_sims + 1);
    jb[0] = pb[0] = tb[0] = 0;
    int64_t items_needed = 0;
    for (int32_t s = 0; s < n; s++) {
        hh_ctx *c = ctxs[s];
        if (!c) return bfail(b, HH_EINVAL, "hh_batch_run: NULL context");
        if (c->device != b->device || c->cfg.precision != b->precision)
            return bfail(b, HH_EINVAL, "hh_batch_run: context device or precision differs from the batch");
        if (!c->have_lists || !c->have_dt) return bfail(b, HH_ESTATE, "hh_batch_run: a context lacks lists or steps");
        for (int32_t q = 0; q < s; q++)
            if (ctxs[q] == c) return bfail(b, HH_EINVAL, "hh_batch_run: a context appears twice");
        if (!(t_end[s] == t_end[s])) return bfail(b, HH_EINVAL, "hh_batch_run: NaN stop time");
        SimDesc &d = sims[s];
        std::memset(&d, 0, sizeof(d));
        d.st = c->st;
        d.rec = c->rec;
        d.L.off = c->off;
        d.L.idx = c->idx;
        d.L.tiles = c->tiles;
        d.L.items = nullptr;
        d.L.partials = c->partials;
        d.L.tile_cnt = c->tile_cnt;
        d.L.i_map = nullptr;
        d.tile_lv = c->tile_lv;
        d.ds = c->ds;
        d.n = c->n;
        d.nj = c->nj;
        d.n_tiles = c->n_tiles;
        d.pj = c->part_len;
        d.work = c->cfg.work_item;
        d.work_split = c->cfg.work_split;
        d.pj_small = c->cfg.tile_j_small;
        d.lmax = int32_t(std::min<int64_t>(c->list_max, INT32_MAX));
        d.lbar = c->n_groups > 0 ? std::max<int64_t>(1, c->list_len / c->n_groups) : 1;
        d.prm.eps2 = c->cfg.eps2;
        d.prm.eta = c->cfg.eta;
        d.prm.eta_s = c->cfg.eta_s;
        d.prm.dt_min = c->cfg.dt_min;
        d.prm.dt_max = c->cfg.dt_max;
        d.t_end = t_end[s];
        jb[s + 1] = jb[s] + c->nj;
        pb[s + 1] = pb[s] + c->n;
        tb[s + 1] = tb[s] + c->n_tiles;
        items_needed += std::max(c->total_parts, c->small_parts);
        // pending work of the context must be finished before the batch stream uses its memory
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bfail(b, HH_ECUDA, "hh_batch_run: context stream failed");
    }
    if (items_needed > INT32_MAX / 2) return bfail(b, HH_ENOMEM, "hh_batch_run: too many work items");
    // every worker group reads its first slot before it knows the count
    const int64_t min_items = int64_t(b->grid) * kGroups;
    if (items_needed > b->cap_items || b->cap_items < min_items) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        const int64_t cap = std::max(items_needed + items_needed / 4 + 64, min_items);
        if (cudaMalloc(&b->d_items, sizeof(WorkItem) * cap) != cudaSuccess) {
            cudaGetLastError();
            b->cap_items = 0;
            return bfail(b, HH_ENOMEM, "hh_batch_run: cannot allocate the work queue");
        }
        b->cap_items = cap;
    }
    BatchHdr *hdr = reinterpret_cast<BatchHdr *>(b->h_blk + Ly.hdr);
    hdr->n_sims = n;
    hdr->max_steps = max_steps;
    hdr->items = b->d_items;
    std::memset(b->h_blk + Ly.bs, 0, sizeof(BatchScalars));
    if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        return bfail(b, HH_ECUDA, std::string("hh_batch_run: launch: ") + cudaGetErrorString(e));
    }
    hh_count_launches(1);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess)
        return bfail(b, HH_ECUDA, "hh_batch_run: kernel execution failed");
    BatchScalars hbs;
    std::memcpy(&hbs, b->h_blk + Ly.bs, sizeof(hbs));
    if (hbs.err == HH_ETIMEOUT) return bfail(b, hbs.err, "hh_batch_run: grid barrier timed out");
    if (hbs.err)
        return bfail(b, hbs.err, "hh_batch_run: block-step state breaks the block rule (a step that is not a power "
                                 "of two in [2^-31, 1], a time not a multiple of its step, or an overdue particle)");
    for (int32_t s = 0; s < n; s++) {
        ctxs[s]->predicted = false;
        ctxs[s]->have_forces = true;
    }
    if (steps_out) *steps_out = hbs.steps_done;
    if (t_next_out) std::memcpy(t_next_out, b->h_blk + Ly.tnext, sizeof(double) * size_t(n));
    const unsigned long long *T = reinterpret_cast<const unsigned long long *>(b->h_blk + Ly.step_ns);
    for (int32_t q = 0; q < hbs.steps_done; q++) {
        const size_t k = 3 * size_t(q);
        if (step_us_out) step_us_out[q] = double(T[k + 3] - T[k]) * 1e-3;
        if (phase_us_out)
            for (int ph = 0; ph < 3; ph++) phase_us_out[3 * size_t(q) + ph] = double(T[k + ph + 1] - T[k + ph]) * 1e-3;
    }
    return HH_OK;
}

extern "C" const char *hh_batch_last_error(const hh_batch *b) { return b ? b->err.c_str() : hh_last_error(nullptr); }

// ---- resident set: admission by memory budget, continuous batching --------

extern "C" int hh_batch_set_budget(hh_batch *b, int64_t budget_bytes, int64_t launch_particles)
{
    if (!b) return hh_set_global_error(HH_EINVAL, "hh_batch_set_budget: NULL batch");
    if (budget_bytes < 0 || launch_particles < 0)
        return bfail(b, HH_EINVAL, "hh_batch_set_budget: negative budget or particle cap");
    b->budget = budget_bytes;
    b->launch_particles = launch_particles;
    return HH_OK;
}

extern "C" int hh_batch_admit(hh_batch *b, hh_ctx *ctx, double t_end)
{
    if (!b) return hh_set_global_error(HH_EINVAL, "hh_batch_admit: NULL batch");
    if (!ctx) return bfail(b, HH_EINVAL, "hh_batch_admit: NULL context");
    if (ctx->device != b->device || ctx->cfg.precision != b->precision)
        return bfail(b, HH_EINVAL, "hh_batch_admit: context device or precision differs from the batch");
    if (!ctx->have_lists || !ctx->have_dt)
        return bfail(b, HH_ESTATE, "hh_batch_admit: the context lacks lists or steps (call hh_run(ctx, t0, t0))");
    for (const Resident &r : b->res)
        if (r.ctx == ctx) return bfail(b, HH_EINVAL, "hh_batch_admit: context already admitted");
    const double dtt = ctx->cfg.dt_tree;
    const double k = t_end / dtt;
    if (!(t_end >= ctx->t_tree) || k != std::floor(k))
        return bfail(b, HH_EINVAL, "hh_batch_admit: t_end must be a multiple of dt_tree, not before the tree time");
    if (int32_t(b->res.size()) >= b->max_sims) return bfail(b, HH_ENOMEM, "hh_batch_admit: every slot is taken");
    const int64_t bytes = ctx->device_bytes;
    if (b->budget > 0 && b->used + bytes > b->budget)
        return bfail(b, HH_ENOMEM, "hh_batch_admit: the context's device memory does not fit the budget");
    Resident r;
    r.ctx = ctx;
    r.t_end = t_end;
    r.t_stop = std::min(ctx->t_tree + dtt, t_end);
    r.bytes = bytes;
    r.state = t_end > ctx->t_tree ? 0 : 1;  // nothing to run: finished at once
    b->res.push_back(r);
    b->used += bytes;
    return HH_OK;
}

extern "C" int hh_batch_retire(hh_batch *b, hh_ctx *ctx)
{
    if (!b) return hh_set_global_error(HH_EINVAL, "hh_batch_retire: NULL batch");
    for (size_t q = 0; q < b->res.size(); q++)
        if (b->res[q].ctx == ctx) {
            b->used -= b->res[q].bytes;
            b->res.erase(b->res.begin() + q);
            if (b->rr > q) b->rr--;
            return HH_OK;
        }
    return bfail(b, HH_EINVAL, "hh_batch_retire: context not resident");
}

extern "C" int hh_batch_resident(const hh_batch *b, int32_t *n_out, int32_t *running_out, int64_t *bytes_out)
{
    if (!b) return hh_set_global_error(HH_EINVAL, "hh_batch_resident: NULL batch");
    int32_t run = 0;
    for (const Resident &r : b->res) run += r.state == 0;
    if (n_out) *n_out = int32_t(b->res.size());
    if (running_out) *running_out = run;
    if (bytes_out) *bytes_out = b->used;
    return HH_OK;
}

extern "C" int hh_batch_rebuild(hh_batch *b, int32_t n, hh_ctx *const *ctxs, const double *t, int *rc_out)
{
    if (!b) return hh_set_global_error(HH_EINVAL, "hh_batch_rebuild: NULL batch");
    if (n < 1 || !ctxs || !t) return bfail(b, HH_EINVAL, "hh_batch_rebuild: bad n or NULL arrays");
    std::vector<hh_ctx *> sorted(ctxs, ctxs + n);
    std::sort(sorted.begin(), sorted.end(), std::less<hh_ctx *>());
    if (!sorted[0]) return bfail(b, HH_EINVAL, "hh_batch_rebuild: NULL context");
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
        return bfail(b, HH_EINVAL, "hh_batch_rebuild: a context appears twice");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, HH_ECUDA, "hh_batch_rebuild: cudaSetDevice failed");
    if (!b->rb && !(b->rb = hh_rb_scratch_create()))
        return bfail(b, HH_ECUDA, "hh_batch_rebuild: rebuild stream creation failed");
    std::vector<int> rcs(size_t(n), HH_OK);
    hh_rebuild_many(ctxs, t, int(n), rcs.data(), b->rb);
    int first = HH_OK;
    for (int32_t s = 0; s < n; s++) {
        if (rc_out) rc_out[s] = rcs[size_t(s)];
        if (first == HH_OK && rcs[size_t(s)] != HH_OK) {
            first = rcs[size_t(s)];
            b->err = std::string("hh_batch_rebuild: ") + hh_last_error(ctxs[s]);
        }
    }
    return first;
}

extern "C" int hh_batch_step(hh_batch *b, int32_t max_steps, int32_t *steps_out, int32_t *launched_out,
                             int32_t *n_done_out, hh_ctx **done_out, double *step_us_out, double *phase_us_out)
{
    if (!b) return hh_set_global_error(HH_EINVAL, "hh_batch_step: NULL batch");
    if (steps_out) *steps_out = 0;
    if (launched_out) *launched_out = 0;
    if (n_done_out) *n_done_out = 0;
    // this launch: running residents in round-robin order from b->rr, up to
    // the particle cap (at least one simulation per launch)
    const size_t R = b->res.size();
    std::vector<size_t> pick;
    int64_t parts = 0;
    for (size_t q = 0; q < R; q++) {
        const size_t i = (b->rr + q) % R;
        const Resident &r = b->res[i];
        if (r.state != 0) continue;
        if (b->launch_particles > 0 && !pick.empty() && parts + r.ctx->n > b->launch_particles) break;
        pick.push_back(i);
        parts += r.ctx->n;
    }
    int32_t nd = 0;
    if (!pick.empty()) {
        b->rr = (pick.back() + 1) % R;
        std::vector<hh_ctx *> ctxs(pick.size());
        std::vector<double> stop(pick.size()), tn(pick.size());
        for (size_t q = 0; q < pick.size(); q++) {
            ctxs[q] = b->res[pick[q]].ctx;
            stop[q] = b->res[pick[q]].t_stop;
        }
        int32_t steps = 0;
        int rc = hh_batch_run(b, int32_t(pick.size()), ctxs.data(), stop.data(), max_steps, &steps, tn.data(),
                              step_us_out, phase_us_out);
        if (rc) return rc;
        if (steps_out) *steps_out = steps;
        if (launched_out) *launched_out = int32_t(pick.size());
        // simulations past their stop time: finished, or rebuilt for the next
        // interval.  Device builders run as one batched build over all of
        // them; host builders concurrently, one host thread each.
        std::vector<size_t> rebuild, on_host;
        std::vector<hh_ctx *> dev;
        std::vector<double> tdev;
        for (size_t q = 0; q < pick.size(); q++) {
            Resident &r = b->res[pick[q]];
            if (!(tn[q] > r.t_stop)) continue;
            if (r.t_stop >= r.t_end) {
                r.state = 1;
                continue;
            }
            rebuild.push_back(pick[q]);
            if (r.ctx->rebuild_device) {
                dev.push_back(r.ctx);
                tdev.push_back(r.t_stop);
            } else {
                on_host.push_back(rebuild.size() - 1);
            }
        }
        std::vector<int> rcs(rebuild.size(), HH_OK);
        if (!dev.empty()) {
            std::vector<int> rd(dev.size(), HH_OK);
            const int rc = hh_batch_rebuild(b, int32_t(dev.size()), dev.data(), tdev.data(), rd.data());
            if (rc == HH_ECUDA && !b->rb) return rc;
            for (size_t q = 0, w = 0; q < rebuild.size(); q++)
                if (b->res[rebuild[q]].ctx->rebuild_device) rcs[q] = rd[w++];
        }
#pragma omp parallel for schedule(dynamic, 1) num_threads(int(std::min<size_t>(8, std::max<size_t>(1, on_host.size()))))
        for (int64_t q = 0; q < int64_t(on_host.size()); q++) {
            const size_t i = on_host[size_t(q)];
            Resident &r = b->res[rebuild[i]];
            rcs[i] = hh_rebuild(r.ctx, r.t_stop);
        }
        int first_rc = HH_OK;
        std::string first_msg;
        for (size_t q = 0; q < rebuild.size(); q++) {
            Resident &r = b->res[rebuild[q]];
            if (rcs[q] != HH_OK) {
                r.state = 2;
                if (first_rc == HH_OK) {
                    first_rc = rcs[q];
                    first_msg = std::string("hh_batch_step: rebuild failed: ") + hh_last_error(r.ctx);
                }
            } else {
                r.t_stop = std::min(r.t_stop + r.ctx->cfg.dt_tree, r.t_end);
            }
        }
        if (first_rc != HH_OK) {
            cudaSetDevice(b->device);
            return bfail(b, first_rc, first_msg);
        }
    }
    // every finished resident not yet reported is reported once
    for (Resident &r : b->res)
        if (r.state == 1) {
            if (done_out) done_out[nd] = r.ctx;
            nd++;
            r.state = 3;  // reported; stays resident until retired
        }
    if (n_done_out) *n_done_out = nd;
    return HH_OK;
}

namespace {

// Runs `rounds` grid barriers; CTA `skip` (if >= 0) never arrives, so the
// others' bounded waits must give up and report HH_ETIMEOUT.
__global__ void k_barrier_selftest(BatchScalars *bs, int rounds, int skip)
{
    if ((int)blockIdx.x == skip) return;
    for (int r = 0; r < rounds; r++)
        if (!grid_sync(bs)) return;
}

}  // namespace

extern "C" int hh_barrier_selftest(int device, int skip_cta, double *elapsed_s)
{
    if (cudaSetDevice(device) != cudaSuccess) return hh_set_global_error(HH_ECUDA, "hh_barrier_selftest: bad device");
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
        return hh_set_global_error(HH_ECUDA, "hh_barrier_selftest: device query failed");
    const int grid = prop.multiProcessorCount;
    if (skip_cta >= grid) return hh_set_global_error(HH_EINVAL, "hh_barrier_selftest: skip_cta >= number of CTAs");
    BatchScalars *bs = nullptr;
    if (cudaMalloc(&bs, sizeof(BatchScalars)) != cudaSuccess || cudaMemset(bs, 0, sizeof(BatchScalars)) != cudaSuccess) {
        cudaGetLastError();
        if (bs) cudaFree(bs);
        return hh_set_global_error(HH_ENOMEM, "hh_barrier_selftest: allocation failed");
    }
    int rounds = 64;
    void *args[] = {&bs, &rounds, &skip_cta};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(grid), dim3(kThreads), args, 0, 0);
    cudaEventRecord(e1);
    BatchScalars h;
    std::memset(&h, 0, sizeof(h));
    if (e == cudaSuccess) e = cudaMemcpy(&h, bs, sizeof(h), cudaMemcpyDeviceToHost);
    float ms = 0.f;
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(bs);
    if (elapsed_s) *elapsed_s = ms * 1e-3;
    if (e != cudaSuccess) return hh_set_global_error(HH_ECUDA, cudaGetErrorString(e));
    hh_count_launches(1);
    if (h.err) return hh_set_global_error(h.err, "hh_barrier_selftest: a grid barrier timed out");
    return HH_OK;
}

namespace {

__global__ void k_aarseth_selftest(int64_t n, const double *A, const double *J, const double *S, const double *T,
                                   double eta, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = aarseth_want(A[i], J[i], S[i], T[i], eta);
}

__global__ void k_block_dt_selftest(int64_t n, const double *want, const double *dt_old, const double *t_new,
                                    double dt_min, double dt_max, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = block_dt(want[i], dt_old[i], t_new[i], dt_min, dt_max);
}

}  // namespace

extern "C" int hh_selftest_block_dt(int device, int64_t n, const double *want, const double *dt_old,
                                    const double *t_new, double dt_min, double dt_max, double *out)
{
    if (n < 0 || (n > 0 && (!want || !dt_old || !t_new || !out)))
        return hh_set_global_error(HH_EINVAL, "hh_selftest_block_dt: bad n or NULL array");
    if (n == 0) return HH_OK;
    if (n > (int64_t(1) << 26)) return hh_set_global_error(HH_EINVAL, "hh_selftest_block_dt: n above 2^26");
    if (cudaSetDevice(device) != cudaSuccess) return hh_set_global_error(HH_ECUDA, "hh_selftest_block_dt: bad device");
    double *d = nullptr;
    const size_t bytes = sizeof(double) * size_t(n);
    if (cudaMalloc(&d, 4 * bytes) != cudaSuccess) {
        cudaGetLastError();
        return hh_set_global_error(HH_ENOMEM, "hh_selftest_block_dt: allocation failed");
    }
    cudaError_t e = cudaSuccess;
    const double *src[3] = {want, dt_old, t_new};
    for (int q = 0; q < 3 && e == cudaSuccess; q++) e = cudaMemcpy(d + q * n, src[q], bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int grid = int(std::min<int64_t>((n + 255) / 256, 4096));
        k_block_dt_selftest<<<grid, 256>>>(n, d, d + n, d + 2 * n, dt_min, dt_max, d + 3 * n);
        hh_count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d + 3 * n, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return hh_set_global_error(HH_ECUDA, cudaGetErrorString(e));
    return HH_OK;
}

extern "C" int hh_selftest_aarseth(int device, int64_t n, const double *A, const double *J, const double *S,
                                   const double *T, double eta, double *out)
{
    if (n < 0 || (n > 0 && (!A || !J || !S || !T || !out)))
        return hh_set_global_error(HH_EINVAL, "hh_selftest_aarseth: bad n or NULL array");
    if (n == 0) return HH_OK;
    if (n > (int64_t(1) << 26)) return hh_set_global_error(HH_EINVAL, "hh_selftest_aarseth: n above 2^26");
    if (cudaSetDevice(device) != cudaSuccess) return hh_set_global_error(HH_ECUDA, "hh_selftest_aarseth: bad device");
    double *d = nullptr;
    const size_t bytes = sizeof(double) * size_t(n);
    if (cudaMalloc(&d, 5 * bytes) != cudaSuccess) {
        cudaGetLastError();
        return hh_set_global_error(HH_ENOMEM, "hh_selftest_aarseth: allocation failed");
    }
    cudaError_t e = cudaSuccess;
    const double *src[4] = {A, J, S, T};
    for (int q = 0; q < 4 && e == cudaSuccess; q++) e = cudaMemcpy(d + q * n, src[q], bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int grid = int(std::min<int64_t>((n + 255) / 256, 4096));
        k_aarseth_selftest<<<grid, 256>>>(n, d, d + n, d + 2 * n, d + 3 * n, eta, d + 4 * n);
        hh_count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d + 4 * n, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return hh_set_global_error(HH_ECUDA, cudaGetErrorString(e));
    return HH_OK;
}
