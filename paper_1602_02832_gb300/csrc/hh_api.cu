// C ABI of libhh: context management, uploads, the explicit GRAPE-style calls
// (predict / force / correct), the device-resident block-step loop in CUDA
// graphs, and the library-side tree rebuild.  See include/hh.h.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "hh_ctx.h"

using namespace hh;

namespace {

thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};

constexpr int kGraphSteps = 32;  // block steps unrolled per graph (even)

}  // namespace

void hh_count_launches(int64_t n) { g_launches.fetch_add(n); }

int hh_set_global_error(int code, const char *msg)
{
    g_err = msg;
    return code;
}

namespace {

int fail(hh_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    g_err = msg;
    return code;
}

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(ctx, HH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

#define CKL()                                                                                          \
    do {                                                                                               \
        cudaError_t e_ = cudaGetLastError();                                                           \
        if (e_ != cudaSuccess) return fail(ctx, HH_ECUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
        g_launches.fetch_add(1);                                                                       \
    } while (0)

Params params_of(const hh_ctx *ctx)
{
    Params p;
    p.eps2 = ctx->cfg.eps2;
    p.eta = ctx->cfg.eta;
    p.eta_s = ctx->cfg.eta_s;
    p.dt_min = ctx->cfg.dt_min;
    p.dt_max = ctx->cfg.dt_max;
    return p;
}

Lists lists_of(const hh_ctx *ctx)
{
    Lists L;
    L.off = ctx->off;
    L.idx = ctx->idx;
    L.tiles = ctx->tiles;
    L.items = ctx->items;
    L.partials = ctx->partials;
    L.tile_cnt = ctx->tile_cnt;
    L.i_map = nullptr;
    return L;
}

bool is_pow2(double x)
{
    if (!(x > 0.0) || !std::isfinite(x)) return false;
    int e;
    return std::frexp(x, &e) == 0.5;
}

__global__ void k_set_sizes(DevScalars *ds, int64_t n, int64_t nj, int32_t n_tiles, int32_t part_len,
                            int32_t work_item, int32_t work_split)
{
    ds->n = n;
    ds->nj = nj;
    ds->n_tiles = n_tiles;
    ds->part_len = part_len;
    ds->work_item = work_item;
    ds->work_split = work_split;
}

__global__ void k_begin_loop(DevScalars *ds, double t_end)
{
    ds->t_end = t_end;
    ds->done = 0;
    ds->n_items = 0u;
    ds->slot_ctr = 0u;
    ds->work = 0u;
    ds->tmin[0] = 0x7FF0000000000000ull;
    ds->tmin[1] = 0x7FF0000000000000ull;
}

int launch_predict(hh_ctx *ctx, StepCtl c)
{
    if (ctx->cfg.precision == HH_MIXED)
        k_predict<RecMix><<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, (RecMix *)ctx->rec, lists_of(ctx),
                                                                   ctx->ds, c);
    else
        k_predict<RecF64><<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, (RecF64 *)ctx->rec, lists_of(ctx),
                                                                   ctx->ds, c);
    CKL();
    return HH_OK;
}

int launch_force(hh_ctx *ctx, StepCtl c)
{
    if (ctx->cfg.precision == HH_MIXED)
        k_force<RecMix, kTjMix><<<ctx->force_grid, kThreads, 0, ctx->stream>>>(
            ctx->st, (const RecMix *)ctx->rec, lists_of(ctx), ctx->ds, c, params_of(ctx));
    else
        k_force<RecF64, kTjF64><<<ctx->force_grid, kThreads, 0, ctx->stream>>>(
            ctx->st, (const RecF64 *)ctx->rec, lists_of(ctx), ctx->ds, c, params_of(ctx));
    CKL();
    return HH_OK;
}

int launch_correct(hh_ctx *ctx, StepCtl c)
{
    k_correct<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, ctx->ds, c, params_of(ctx));
    CKL();
    return HH_OK;
}

// explicit modes: reset the work queue, then select work items
int launch_select(hh_ctx *ctx, StepCtl c)
{
    CK(cudaMemsetAsync(&ctx->ds->work, 0, 2 * sizeof(uint32_t), ctx->stream));  // work, n_items
    CK(cudaMemsetAsync(&ctx->ds->slot_ctr, 0, sizeof(uint32_t), ctx->stream));
    k_select<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, lists_of(ctx), ctx->ds, c);
    CKL();
    return HH_OK;
}

int sync_and_check(hh_ctx *ctx)
{
    CK(cudaMemcpyAsync(ctx->h_ds, ctx->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->h_ds->err) {
        const int e = ctx->h_ds->err;
        int32_t zero = 0;
        CK(cudaMemcpyAsync(&ctx->ds->err, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return fail(ctx, e, "device-side validation failed (bad index, value or call order)");
    }
    return HH_OK;
}

// Particle ids follow the slots; after device rebuilds they live on the device.
int sync_ids_to_host(hh_ctx *ctx)
{
    if (!ctx->ids_on_device || !ctx->gtree) return HH_OK;
    CK(cudaMemcpyAsync(ctx->ids.data(), hh_gtree_ids(ctx->gtree), sizeof(int64_t) * ctx->n, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->ids_on_device = false;
    return HH_OK;
}

int check_ctx(hh_ctx *ctx)
{
    if (!ctx) return hh_set_global_error(HH_EINVAL, "NULL context");
    CK(cudaSetDevice(ctx->device));
    return HH_OK;
}

int validate_j_host(hh_ctx *ctx, int64_t n, const double *x, const double *v, const double *a, const double *jk,
                    const double *m, const double *t)
{
    for (int64_t q = 0; q < 3 * n; q++)
        if (!std::isfinite(x[q]) || !std::isfinite(v[q]) || !std::isfinite(a[q]) || !std::isfinite(jk[q]))
            return fail(ctx, HH_EINVAL, "hh_set_j: non-finite x/v/a/jk");
    for (int64_t q = 0; q < n; q++) {
        if (!(m[q] > 0.0) || !std::isfinite(m[q])) return fail(ctx, HH_EINVAL, "hh_set_j: masses must be > 0");
        if (!std::isfinite(t[q])) return fail(ctx, HH_EINVAL, "hh_set_j: non-finite time");
    }
    return HH_OK;
}

// copies a host or device SoA [3][n] block into [3][cap_j] at `first`
int put3(hh_ctx *ctx, double *dst, int64_t first, int64_t n, const double *src, cudaMemcpyKind kind)
{
    for (int d = 0; d < 3; d++)
        CK(cudaMemcpyAsync(dst + d * ctx->cap_j + first, src + d * n, sizeof(double) * n, kind, ctx->stream));
    return HH_OK;
}

int set_j_impl(hh_ctx *ctx, int64_t first, int64_t n, const double *x, const double *v, const double *a,
               const double *jk, const double *m, const double *t, cudaMemcpyKind kind)
{
    if (first < 0 || n < 0 || first + n > ctx->cap_j) return fail(ctx, HH_EINVAL, "hh_set_j: range exceeds nj_max");
    if (n == 0) return HH_OK;
    if (!x || !v || !a || !jk || !m || !t) return fail(ctx, HH_EINVAL, "hh_set_j: NULL array");
    int rc;
    if ((rc = put3(ctx, ctx->st.x, first, n, x, kind))) return rc;
    if ((rc = put3(ctx, ctx->st.v, first, n, v, kind))) return rc;
    if ((rc = put3(ctx, ctx->st.a, first, n, a, kind))) return rc;
    if ((rc = put3(ctx, ctx->st.jk, first, n, jk, kind))) return rc;
    CK(cudaMemcpyAsync(ctx->st.m + first, m, sizeof(double) * n, kind, ctx->stream));
    CK(cudaMemcpyAsync(ctx->st.t + first, t, sizeof(double) * n, kind, ctx->stream));
    if (kind == cudaMemcpyDeviceToDevice) {
        k_check_j<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, first, n, ctx->ds);
        CKL();
    }
    if (ctx->st.base) {
        k_refresh_base<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, first, n);
        CKL();
    }
    ctx->have_j = true;
    ctx->predicted = false;
    return sync_and_check(ctx);
}

int ensure_graph(hh_ctx *ctx)
{
    const int timed = ctx->timing ? 1 : 0;
    if (ctx->graph && ctx->graph_timed == timed) return HH_OK;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    if (timed && ctx->ev.empty()) {
        ctx->ev.resize(2 * kGraphSteps);
        for (auto &e : ctx->ev) CK(cudaEventCreate(&e));
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int rc = HH_OK;
    for (int s = 0; s < kGraphSteps && rc == HH_OK; s++) {
        StepCtl c{0, s & 1, (s & 1) ^ 1, 0, 0.0};
        rc = launch_predict(ctx, c);
        if (rc == HH_OK && timed) rc = cudaEventRecordWithFlags(ctx->ev[2 * s], ctx->stream, cudaEventRecordExternal) == cudaSuccess ? HH_OK : HH_ECUDA;
        if (rc == HH_OK) rc = launch_force(ctx, c);
        if (rc == HH_OK && timed) rc = cudaEventRecordWithFlags(ctx->ev[2 * s + 1], ctx->stream, cudaEventRecordExternal) == cudaSuccess ? HH_OK : HH_ECUDA;
        if (rc == HH_OK) rc = launch_correct(ctx, c);
    }
    cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
    // capture launches are not executions
    g_launches.fetch_sub(3 * kGraphSteps);
    if (rc != HH_OK) {
        if (g) cudaGraphDestroy(g);
        return fail(ctx, rc, "graph capture failed: " + ctx->err);
    }
    if (ce != cudaSuccess) return fail(ctx, HH_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fail(ctx, HH_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
    ctx->graph_timed = timed;
    return HH_OK;
}

int mark_upload(hh_ctx *ctx, int32_t n_act, const int32_t *i_idx, bool dev, int32_t **dev_idx)
{
    if (n_act < 0 || n_act > ctx->n) return fail(ctx, HH_EINVAL, "n_act out of range");
    if (n_act == 0) {
        *dev_idx = ctx->i_buf;
        return HH_OK;
    }
    if (!i_idx) return fail(ctx, HH_EINVAL, "NULL i_idx");
    if (!dev) {
        std::vector<uint8_t> seen(size_t(ctx->n), 0);
        for (int32_t q = 0; q < n_act; q++) {
            if (i_idx[q] < 0 || i_idx[q] >= ctx->n) return fail(ctx, HH_EINVAL, "i_idx out of [0, n_particles)");
            if (seen[size_t(i_idx[q])]++) return fail(ctx, HH_EINVAL, "i_idx has repeated particles");
        }
        std::memcpy(ctx->h_ibuf, i_idx, sizeof(int32_t) * n_act);
        CK(cudaMemcpyAsync(ctx->i_buf, ctx->h_ibuf, sizeof(int32_t) * n_act, cudaMemcpyHostToDevice, ctx->stream));
        *dev_idx = ctx->i_buf;
    } else {
        k_check_idx<<<ctx->elem_grid, 256, 0, ctx->stream>>>(i_idx, n_act, ctx->n, ctx->ds);
        CKL();
        int rc = sync_and_check(ctx);
        if (rc) return rc;
        *dev_idx = const_cast<int32_t *>(i_idx);
    }
    k_set_marks<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st.mark, *dev_idx, n_act, 1);
    CKL();
    return HH_OK;
}

int force_impl(hh_ctx *ctx, int32_t n_act, const int32_t *i_idx, bool dev, double *acc, double *jerk, double *pot)
{
    if (!ctx->have_lists || !ctx->predicted) return fail(ctx, HH_ESTATE, "hh_force: needs hh_set_lists and hh_predict");
    int32_t *didx = nullptr;
    int rc = mark_upload(ctx, n_act, i_idx, dev, &didx);
    if (rc) return rc;
    if (n_act > 0) {
        StepCtl c{1, 0, 1, 0, 0.0};
        if ((rc = launch_select(ctx, c))) return rc;
        if (ctx->timing) CK(cudaEventRecord(ctx->e0, ctx->stream));
        if ((rc = launch_force(ctx, c))) return rc;
        if (ctx->timing) CK(cudaEventRecord(ctx->e1, ctx->stream));
        double *oa = acc, *oj = jerk, *op = pot;
        if (!dev) {
            oa = acc ? ctx->out_buf : nullptr;
            oj = jerk ? ctx->out_buf + 3 * int64_t(n_act) : nullptr;
            op = pot ? ctx->out_buf + 6 * int64_t(n_act) : nullptr;
        }
        k_gather_out<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, didx, n_act, oa, oj, op);
        CKL();
        k_set_marks<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st.mark, didx, n_act, 0);
        CKL();
        if (!dev) {
            if (acc) CK(cudaMemcpyAsync(acc, oa, sizeof(double) * 3 * n_act, cudaMemcpyDeviceToHost, ctx->stream));
            if (jerk) CK(cudaMemcpyAsync(jerk, oj, sizeof(double) * 3 * n_act, cudaMemcpyDeviceToHost, ctx->stream));
            if (pot) CK(cudaMemcpyAsync(pot, op, sizeof(double) * n_act, cudaMemcpyDeviceToHost, ctx->stream));
        }
    }
    ctx->have_forces = true;
    if (!dev || ctx->timing) {
        rc = sync_and_check(ctx);
        if (rc) return rc;
    }
    if (ctx->timing && n_act > 0) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->e0, ctx->e1));
        ctx->force_ms += ms;
        ctx->force_launches += 1;
    }
    return HH_OK;
}

}  // namespace

extern "C" {

void hh_config_default(hh_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->eps2 = 1e-8;
    cfg->eta = 0.02;
    cfg->eta_s = 0.01;
    cfg->dt_min = std::ldexp(1.0, -30);
    cfg->dt_max = std::ldexp(1.0, -6);
    cfg->dt_tree = std::ldexp(1.0, -6);
    cfg->theta = 0.5;
    cfg->leaf = 8;
    cfg->n_crit = 64;
    cfg->precision = HH_FP64;
    cfg->tile_i = 32;
    cfg->tile_j = 0;
}

const char *hh_last_error(const hh_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int64_t hh_kernel_launches(void) { return g_launches.load(); }

int hh_destroy(hh_ctx *ctx)
{
    if (!ctx) return HH_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    for (auto e : ctx->ev) cudaEventDestroy(e);
    if (ctx->e0) cudaEventDestroy(ctx->e0);
    if (ctx->e1) cudaEventDestroy(ctx->e1);
    void *dev[] = {ctx->st.base, ctx->st.x, ctx->st.v, ctx->st.a, ctx->st.jk, ctx->st.m, ctx->st.t, ctx->st.dt, ctx->st.acc1,
                   ctx->st.jerk1, ctx->st.pot1, ctx->st.mark, ctx->rec, ctx->off, ctx->idx, ctx->group_of,
                   ctx->tiles, ctx->ds, ctx->i_buf, ctx->out_buf, ctx->items, ctx->partials, ctx->tile_cnt,
                   ctx->tile_lv};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (ctx->h_ds) cudaFreeHost(ctx->h_ds);
    if (ctx->h_buf) cudaFreeHost(ctx->h_buf);
    if (ctx->h_ibuf) cudaFreeHost(ctx->h_ibuf);
    if (ctx->h_jbuf) cudaFreeHost(ctx->h_jbuf);
    if (ctx->tree) hh_tree_free(ctx->tree);
    if (ctx->gtree) hh_gtree_free(ctx->gtree);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return HH_OK;
}

int hh_create(hh_ctx **out, int device, const hh_config *cfg, int64_t n_max, int64_t nj_max, int64_t list_max,
              int32_t groups_max)
{
    if (!out) return hh_set_global_error(HH_EINVAL, "hh_create: out is NULL");
    *out = nullptr;
    hh_config c;
    if (cfg) c = *cfg;
    else hh_config_default(&c);
    if (n_max < 1 || nj_max < n_max || list_max < 1 || groups_max < 1 || n_max > (int64_t)INT32_MAX / 2 ||
        nj_max > (int64_t)INT32_MAX / 2)
        return hh_set_global_error(HH_EINVAL, "hh_create: bad capacities");
    if (!(c.eps2 >= 0.0) || !(c.eta > 0.0) || !(c.eta_s > 0.0) || !is_pow2(c.dt_min) || !is_pow2(c.dt_max) ||
        c.dt_max < c.dt_min || !is_pow2(c.dt_tree) || c.dt_max > c.dt_tree || !(c.theta >= 0.0) || c.leaf < 1 ||
        c.n_crit < 1 || (c.precision != HH_FP64 && c.precision != HH_MIXED) ||
        (c.order != HH_ORDER_MORTON && c.order != HH_ORDER_HILBERT))
        return hh_set_global_error(HH_EINVAL, "hh_create: bad configuration (steps must be powers of two, "
                                              "dt_min <= dt_max <= dt_tree, eps2 >= 0, eta > 0, order 0 or 1)");
    if (c.tile_i == 0) c.tile_i = 32;
    if (c.tile_i < 1 || c.tile_i > kMaxTileI) return hh_set_global_error(HH_EINVAL, "hh_create: tile_i must be 1..32");
    const int chunk = c.precision == HH_MIXED ? kTjMix : kTjF64;
    if (c.tile_j == 0) c.tile_j = c.precision == HH_MIXED ? 512 : 256;
    if (c.work_item < 0) c.work_item = 0;
    if (c.work_split < 0) c.work_split = 0;
    if (c.tile_j_small != 0 && (c.tile_j_small < 32 || c.tile_j_small % 32 != 0 || c.tile_j_small > c.tile_j))
        return hh_set_global_error(HH_EINVAL, "hh_create: tile_j_small must be 0 or a multiple of 32 in [32, tile_j]");
    if (c.tile_j < chunk || c.tile_j % chunk != 0 || c.tile_j > (1 << 20))
        return hh_set_global_error(HH_EINVAL, "hh_create: tile_j (list part length) must be a multiple of 128 "
                                              "(HH_FP64) or 256 (HH_MIXED)");
    hh_ctx *ctx = new (std::nothrow) hh_ctx;
    if (!ctx) return hh_set_global_error(HH_ENOMEM, "hh_create: out of host memory");
    ctx->device = device;
    ctx->cfg = c;
    ctx->tile_i = c.tile_i;
    ctx->cap_n = n_max;
    ctx->cap_j = nj_max;
    ctx->cap_list = list_max;
    ctx->cap_g = groups_max;
    ctx->cap_tiles = n_max / c.tile_i + groups_max + 1;
    ctx->part_len = c.tile_j;
    ctx->cap_parts = ctx->cap_tiles + list_max / c.tile_j + 1;
    auto bail = [&](int code, const std::string &m) {
        std::string msg = "hh_create: " + m;
        hh_destroy(ctx);
        return hh_set_global_error(code, msg.c_str());
    };
    if (cudaSetDevice(device) != cudaSuccess) return bail(HH_ECUDA, "cudaSetDevice failed");
    if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(HH_ECUDA, "stream creation failed");
    ctx->stream = ctx->own_stream;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return bail(HH_ECUDA, "device query failed");
    ctx->n_sm = prop.multiProcessorCount;
    int per_sm = 0;
    if (c.precision == HH_MIXED)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force<RecMix, kTjMix>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force<RecF64, kTjF64>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    ctx->force_grid = ctx->n_sm * per_sm;
    ctx->elem_grid = ctx->n_sm * 8;
    const size_t rec_bytes = c.precision == HH_MIXED ? sizeof(RecMix) : sizeof(RecF64);
    struct A {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&ctx->st.x, sizeof(double) * 3 * nj_max},      {(void **)&ctx->st.v, sizeof(double) * 3 * nj_max},
        {(void **)&ctx->st.a, sizeof(double) * 3 * nj_max},      {(void **)&ctx->st.jk, sizeof(double) * 3 * nj_max},
        {(void **)&ctx->st.m, sizeof(double) * nj_max},          {(void **)&ctx->st.t, sizeof(double) * nj_max},
        {(void **)&ctx->st.dt, sizeof(double) * n_max},          {(void **)&ctx->st.acc1, sizeof(double) * 3 * n_max},
        {(void **)&ctx->st.jerk1, sizeof(double) * 3 * n_max},   {(void **)&ctx->st.pot1, sizeof(double) * n_max},
        {(void **)&ctx->st.mark, sizeof(int32_t) * n_max},       {(void **)&ctx->rec, rec_bytes * nj_max},
        {(void **)&ctx->off, sizeof(int64_t) * (groups_max + 1)}, {(void **)&ctx->idx, sizeof(int32_t) * list_max},
        {(void **)&ctx->group_of, sizeof(int32_t) * n_max},      {(void **)&ctx->tiles, sizeof(int4) * ctx->cap_tiles},
        {(void **)&ctx->ds, sizeof(DevScalars)},                 {(void **)&ctx->i_buf, sizeof(int32_t) * n_max},
        {(void **)&ctx->out_buf, sizeof(double) * 7 * n_max},
        {(void **)&ctx->tile_cnt, sizeof(int32_t) * ctx->cap_tiles},
        {(void **)&ctx->tile_lv, sizeof(uint32_t) * ctx->cap_tiles},
        {(void **)&ctx->st.base, c.precision == HH_MIXED ? sizeof(BaseMix) * nj_max : 0},
        {(void **)&ctx->items, sizeof(WorkItem) * ctx->cap_parts},
        {(void **)&ctx->partials, sizeof(RedF64) * kMaxTileI * ctx->cap_parts},
    };
    for (auto &al : allocs) {
        if (al.bytes == 0) {
            *al.p = nullptr;
            continue;
        }
        if (cudaMalloc(al.p, al.bytes) != cudaSuccess) {
            cudaGetLastError();
            return bail(HH_ENOMEM, "device allocation failed (capacities too large)");
        }
        ctx->device_bytes += int64_t(al.bytes);
    }
    ctx->st.cap_j = nj_max;
    ctx->st.cap_n = n_max;
    // the pinned staging of the host tree build (h_buf, h_jbuf) is allocated by
    // the first host rebuild: contexts that rebuild on the device never need it
    if (cudaHostAlloc((void **)&ctx->h_ds, sizeof(DevScalars), cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&ctx->h_ibuf, sizeof(int32_t) * n_max, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return bail(HH_ENOMEM, "pinned host allocation failed");
    }
    if (cudaMemsetAsync(ctx->ds, 0, sizeof(DevScalars), ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->st.mark, 0, sizeof(int32_t) * n_max, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->tile_cnt, 0, sizeof(int32_t) * ctx->cap_tiles, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->st.acc1, 0, sizeof(double) * 3 * n_max, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->st.jerk1, 0, sizeof(double) * 3 * n_max, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->st.dt, 0, sizeof(double) * n_max, ctx->stream) != cudaSuccess ||
        cudaEventCreate(&ctx->e0) != cudaSuccess || cudaEventCreate(&ctx->e1) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return bail(HH_ECUDA, "initialisation failed");
    *out = ctx;
    return HH_OK;
}

int hh_set_stream(hh_ctx *ctx, void *s)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->stream = s ? (cudaStream_t)s : ctx->own_stream;
    return HH_OK;
}

int hh_set_j(hh_ctx *ctx, int64_t first, int64_t n, const double *x, const double *v, const double *a,
             const double *jk, const double *m, const double *t)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (n > 0 && x && v && a && jk && m && t && (rc = validate_j_host(ctx, n, x, v, a, jk, m, t))) return rc;
    return set_j_impl(ctx, first, n, x, v, a, jk, m, t, cudaMemcpyHostToDevice);
}

int hh_set_j_dev(hh_ctx *ctx, int64_t first, int64_t n, const double *x, const double *v, const double *a,
                 const double *jk, const double *m, const double *t)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    return set_j_impl(ctx, first, n, x, v, a, jk, m, t, cudaMemcpyDeviceToDevice);
}

namespace {
int set_lists_core(hh_ctx *ctx, int64_t n_particles, int64_t n_j, int32_t n_groups, const int64_t *off,
                   const int32_t *idx, const int32_t *group_of, bool trusted);
}

int hh_set_lists(hh_ctx *ctx, int64_t n_particles, int64_t n_j, int32_t n_groups, const int64_t *off,
                 const int32_t *idx, const int32_t *group_of)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    return set_lists_core(ctx, n_particles, n_j, n_groups, off, idx, group_of, false);
}

}  // extern "C"

namespace {
// `trusted`: lists made by this library's own builder skip the per-entry
// index scan (they are valid by construction); everything else is checked.
// Work items and partial sums grow with the lists; kernels captured in the
// loop graph hold the old pointers, so the graph is rebuilt.
// Work items a block step of the batched loop can have beyond those of
// parts of tile_j: with tile_j_small, a step with at most kSmallDue due
// particles (at most kSmallDue tiles, each with the longest list, in parts
// of tile_j_small); in the plain form with work_split, a step with fewer due
// particles than work_split (as many tiles at most, in equal-cost parts of
// kMedWork x tile_j interactions, the shortest for a full tile).
int64_t small_parts_bound(const hh_ctx *ctx, int64_t n_tiles, int64_t lmax)
{
    int64_t b = 0;
    const int64_t pjs = ctx->cfg.tile_j_small;
    if (pjs > 0) b = std::min<int64_t>(n_tiles, kSmallDue) * std::max<int64_t>(1, (lmax + pjs - 1) / pjs);
    if (ctx->cfg.precision == HH_FP64 && ctx->cfg.work_split > 0) {
        const int64_t want = (int64_t(kMedWork) * ctx->part_len + ctx->tile_i - 1) / ctx->tile_i;
        const int64_t shortest = std::max<int64_t>(32, (want + 31) / 32 * 32);
        b = std::max(b, std::min<int64_t>(n_tiles, ctx->cfg.work_split) * std::max<int64_t>(1, (lmax + shortest - 1) /
                                                                                                  shortest));
    }
    return b;
}

int ensure_parts(hh_ctx *ctx, int64_t total_parts)
{
    if (total_parts <= ctx->cap_parts) return HH_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    const int64_t cap = total_parts + total_parts / 4 + 64;
    WorkItem *items = nullptr;
    void *partials = nullptr;
    if (cudaMalloc(&items, sizeof(WorkItem) * cap) != cudaSuccess ||
        cudaMalloc(&partials, sizeof(RedF64) * kMaxTileI * cap) != cudaSuccess) {
        cudaGetLastError();
        if (items) cudaFree(items);
        return fail(ctx, HH_ENOMEM, "cannot grow the work-item buffers");
    }
    cudaFree(ctx->items);
    cudaFree(ctx->partials);
    ctx->device_bytes += (cap - ctx->cap_parts) * int64_t(sizeof(WorkItem) + sizeof(RedF64) * kMaxTileI);
    ctx->items = items;
    ctx->partials = partials;
    ctx->cap_parts = cap;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return HH_OK;
}

int set_lists_core(hh_ctx *ctx, int64_t n_particles, int64_t n_j, int32_t n_groups, const int64_t *off,
                   const int32_t *idx, const int32_t *group_of, bool trusted)
{
    int rc = HH_OK;
    if (n_particles < 1 || n_particles > ctx->cap_n || n_j < n_particles || n_j > ctx->cap_j)
        return fail(ctx, HH_EINVAL, "hh_set_lists: n_particles / n_j out of capacity");
    if (n_groups < 1 || n_groups > ctx->cap_g || !off || !idx || !group_of)
        return fail(ctx, HH_EINVAL, "hh_set_lists: bad n_groups or NULL array");
    if (off[0] != 0) return fail(ctx, HH_EINVAL, "hh_set_lists: off[0] must be 0");
    for (int32_t g = 0; g < n_groups; g++)
        if (off[g + 1] < off[g]) return fail(ctx, HH_EINVAL, "hh_set_lists: off must be non-decreasing");
    const int64_t L = off[n_groups];
    if (L > ctx->cap_list) return fail(ctx, HH_ENOMEM, "hh_set_lists: list_max exceeded");
    if (!trusted)
        for (int64_t q = 0; q < L; q++)
            if (idx[q] < 0 || idx[q] >= n_j) return fail(ctx, HH_EINVAL, "hh_set_lists: list index outside [0, n_j)");
    // groups must be contiguous ascending particle ranges
    std::vector<int4> tiles;
    tiles.reserve(size_t(n_particles / ctx->tile_i + n_groups + 1));
    int64_t total_parts = 0;
    int64_t p = 0;
    int32_t prev = -1;
    while (p < n_particles) {
        const int32_t g = group_of[p];
        if (g < 0 || g >= n_groups || g <= prev) return fail(ctx, HH_EINVAL, "hh_set_lists: group_of must be ascending contiguous ranges");
        int64_t e = p;
        while (e < n_particles && group_of[e] == g) e++;
        const int64_t n_parts = std::max<int64_t>(1, (off[g + 1] - off[g] + ctx->part_len - 1) / ctx->part_len);
        for (int64_t b = p; b < e; b += ctx->tile_i) {
            tiles.push_back(make_int4(int(b), int(std::min<int64_t>(b + ctx->tile_i, e)), g, int(total_parts)));
            total_parts += n_parts;
        }
        prev = g;
        p = e;
    }
    if (int64_t(tiles.size()) > ctx->cap_tiles) return fail(ctx, HH_ENOMEM, "hh_set_lists: too many tiles");
    if (total_parts > INT32_MAX / 2) return fail(ctx, HH_ENOMEM, "hh_set_lists: too many list parts");
    int64_t lmax = 0;
    for (int32_t g = 0; g < n_groups; g++) lmax = std::max<int64_t>(lmax, off[g + 1] - off[g]);
    const int64_t small_parts = small_parts_bound(ctx, int64_t(tiles.size()), lmax);
    if (small_parts > INT32_MAX / 2) return fail(ctx, HH_ENOMEM, "hh_set_lists: too many short list parts");
    if ((rc = ensure_parts(ctx, std::max(total_parts, small_parts)))) return rc;
    CK(cudaMemcpyAsync(ctx->off, off, sizeof(int64_t) * (n_groups + 1), cudaMemcpyHostToDevice, ctx->stream));
    if (L) CK(cudaMemcpyAsync(ctx->idx, idx, sizeof(int32_t) * L, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->group_of, group_of, sizeof(int32_t) * n_particles, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, ctx->stream));
    k_set_sizes<<<1, 1, 0, ctx->stream>>>(ctx->ds, n_particles, n_j, int32_t(tiles.size()), ctx->part_len,
                                           ctx->cfg.work_item, ctx->cfg.work_split);
    CKL();
    CK(cudaStreamSynchronize(ctx->stream));  // host arrays may be freed after return
    ctx->n = n_particles;
    ctx->nj = n_j;
    ctx->n_groups = n_groups;
    ctx->list_len = L;
    ctx->list_max = lmax;
    ctx->n_tiles = int32_t(tiles.size());
    ctx->total_parts = total_parts;
    ctx->small_parts = small_parts;
    ctx->h_group_of.assign(group_of, group_of + n_particles);
    if (int64_t(ctx->ids.size()) != n_particles) {
        ctx->ids.resize(size_t(n_particles));
        for (int64_t q = 0; q < n_particles; q++) ctx->ids[size_t(q)] = q;
    }
    ctx->have_lists = true;
    ctx->predicted = false;
    return HH_OK;
}
}  // namespace

extern "C" {

int hh_set_dt(hh_ctx *ctx, const double *dt)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!ctx->have_lists) return fail(ctx, HH_ESTATE, "hh_set_dt: set lists first (fixes n_particles)");
    if (!dt) return fail(ctx, HH_EINVAL, "hh_set_dt: NULL");
    for (int64_t q = 0; q < ctx->n; q++)
        if (!is_pow2(dt[q])) return fail(ctx, HH_EINVAL, "hh_set_dt: steps must be positive powers of two");
    CK(cudaMemcpyAsync(ctx->st.dt, dt, sizeof(double) * ctx->n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->have_dt = true;
    return HH_OK;
}

int hh_init_dt(hh_ctx *ctx)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!ctx->have_lists) return fail(ctx, HH_ESTATE, "hh_init_dt: set lists first");
    k_init_dt<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, ctx->ds, params_of(ctx));
    CKL();
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->have_dt = true;
    return HH_OK;
}

int hh_predict(hh_ctx *ctx, double t)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!ctx->have_lists) return fail(ctx, HH_ESTATE, "hh_predict: needs hh_set_j and hh_set_lists");
    if (!std::isfinite(t)) return fail(ctx, HH_EINVAL, "hh_predict: non-finite t");
    StepCtl c{1, 0, 1, 0, t};
    if ((rc = launch_predict(ctx, c))) return rc;
    ctx->predicted = true;
    return HH_OK;
}

int hh_force(hh_ctx *ctx, int32_t n_act, const int32_t *i_idx, double *acc, double *jerk, double *pot)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    return force_impl(ctx, n_act, i_idx, false, acc, jerk, pot);
}

int hh_force_dev(hh_ctx *ctx, int32_t n_act, const int32_t *i_idx, double *acc, double *jerk, double *pot)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    return force_impl(ctx, n_act, i_idx, true, acc, jerk, pot);
}

int hh_correct(hh_ctx *ctx, double t, int32_t n_act, const int32_t *i_idx)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!ctx->have_forces || !ctx->have_dt) return fail(ctx, HH_ESTATE, "hh_correct: needs forces and steps");
    int32_t *didx = nullptr;
    if ((rc = mark_upload(ctx, n_act, i_idx, false, &didx))) return rc;
    if (n_act > 0) {
        StepCtl c{1, 0, 1, 0, t};
        if ((rc = launch_correct(ctx, c))) return rc;
        k_set_marks<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st.mark, didx, n_act, 0);
        CKL();
    }
    ctx->predicted = false;
    return sync_and_check(ctx);
}

int hh_init_forces(hh_ctx *ctx, double t)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!ctx->have_lists) return fail(ctx, HH_ESTATE, "hh_init_forces: needs j entries and lists");
    StepCtl cp{1, 0, 1, 0, t};
    if ((rc = launch_predict(ctx, cp))) return rc;
    StepCtl cf{2, 0, 1, 0, t};
    if ((rc = launch_select(ctx, cf))) return rc;
    if ((rc = launch_force(ctx, cf))) return rc;
    k_adopt_forces<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, ctx->ds);
    CKL();
    ctx->have_forces = true;
    ctx->predicted = true;
    return sync_and_check(ctx);
}

int hh_step(hh_ctx *ctx, double *t_next_out, int32_t *n_act_out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!ctx->have_lists || !ctx->have_dt) return fail(ctx, HH_ESTATE, "hh_step: needs lists and steps");
    k_begin_loop<<<1, 1, 0, ctx->stream>>>(ctx->ds, INFINITY);
    CKL();
    k_min_time<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, ctx->ds, 0);
    CKL();
    StepCtl c{0, 0, 1, 0, 0.0};
    if ((rc = launch_predict(ctx, c)) || (rc = launch_force(ctx, c)) || (rc = launch_correct(ctx, c))) return rc;
    if ((rc = sync_and_check(ctx))) return rc;
    if (t_next_out) std::memcpy(t_next_out, &ctx->h_ds->tmin[0], sizeof(double));
    if (n_act_out) *n_act_out = ctx->h_ds->n_act_last;
    ctx->predicted = true;
    ctx->have_forces = true;
    return HH_OK;
}

int hh_advance(hh_ctx *ctx, double t_end, int64_t *n_steps_out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!ctx->have_lists || !ctx->have_dt) return fail(ctx, HH_ESTATE, "hh_advance: needs lists and steps");
    if (!(t_end == t_end)) return fail(ctx, HH_EINVAL, "hh_advance: t_end is NaN");
    if ((rc = ensure_graph(ctx))) return rc;
    k_begin_loop<<<1, 1, 0, ctx->stream>>>(ctx->ds, t_end);
    CKL();
    k_min_time<<<ctx->elem_grid, 256, 0, ctx->stream>>>(ctx->st, ctx->ds, 0);
    CKL();
    if ((rc = sync_and_check(ctx))) return rc;
    const unsigned long long bs0 = ctx->h_ds->block_steps;
    unsigned long long bs_prev = bs0;
    for (int64_t replay = 0;; replay++) {
        CK(cudaGraphLaunch(ctx->graph, ctx->stream));
        g_launches.fetch_add(3 * kGraphSteps);
        if ((rc = sync_and_check(ctx))) return rc;
        const unsigned long long bs = ctx->h_ds->block_steps;
        if (ctx->timing) {
            const int ran = int(bs - bs_prev);
            for (int s = 0; s < ran && s < kGraphSteps; s++) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, ctx->ev[2 * s], ctx->ev[2 * s + 1]));
                ctx->force_ms += ms;
                ctx->force_launches += 1;
            }
        }
        bs_prev = bs;
        if (ctx->h_ds->done) break;
        if (replay > (int64_t(1) << 40)) return fail(ctx, HH_ETIMEOUT, "hh_advance: no progress");
    }
    if (n_steps_out) *n_steps_out = int64_t(bs_prev - bs0);
    ctx->predicted = false;
    return HH_OK;
}

int hh_get_state(hh_ctx *ctx, double *x, double *v, double *a, double *jk, double *t, double *dt)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (ctx->n < 1 || !ctx->have_j) return fail(ctx, HH_ESTATE, "hh_get_state: no particles loaded");
    const int64_t n = ctx->n;
    double *src[4] = {ctx->st.x, ctx->st.v, ctx->st.a, ctx->st.jk};
    double *dst[4] = {x, v, a, jk};
    for (int f = 0; f < 4; f++)
        if (dst[f])
            for (int d = 0; d < 3; d++)
                CK(cudaMemcpyAsync(dst[f] + d * n, src[f] + d * ctx->cap_j, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                   ctx->stream));
    if (t) CK(cudaMemcpyAsync(t, ctx->st.t, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (dt) CK(cudaMemcpyAsync(dt, ctx->st.dt, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return HH_OK;
}

int hh_get_ids(hh_ctx *ctx, int64_t *ids)
{
    if (!ctx || !ids) return hh_set_global_error(HH_EINVAL, "hh_get_ids: NULL");
    int rc = sync_ids_to_host(ctx);
    if (rc) return rc;
    std::copy(ctx->ids.begin(), ctx->ids.end(), ids);
    return HH_OK;
}

int hh_get_lists(hh_ctx *ctx, int32_t *n_groups, int64_t *list_len, int64_t *off, int32_t *idx, int32_t *group_of)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!ctx->have_lists) return fail(ctx, HH_ESTATE, "hh_get_lists: no lists");
    if (n_groups) *n_groups = ctx->n_groups;
    if (list_len) *list_len = ctx->list_len;
    if (off) CK(cudaMemcpyAsync(off, ctx->off, sizeof(int64_t) * (ctx->n_groups + 1), cudaMemcpyDeviceToHost, ctx->stream));
    if (idx && ctx->list_len)
        CK(cudaMemcpyAsync(idx, ctx->idx, sizeof(int32_t) * ctx->list_len, cudaMemcpyDeviceToHost, ctx->stream));
    if (group_of) CK(cudaMemcpyAsync(group_of, ctx->group_of, sizeof(int32_t) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return HH_OK;
}

int hh_get_j(hh_ctx *ctx, int64_t first, int64_t count, double *x, double *v, double *a, double *jk, double *m,
             double *t)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (first < 0 || count < 0 || first + count > ctx->nj) return fail(ctx, HH_EINVAL, "hh_get_j: range outside [0, n_j)");
    double *src[4] = {ctx->st.x, ctx->st.v, ctx->st.a, ctx->st.jk};
    double *dst[4] = {x, v, a, jk};
    for (int f = 0; f < 4; f++)
        if (dst[f])
            for (int d = 0; d < 3; d++)
                CK(cudaMemcpyAsync(dst[f] + d * count, src[f] + d * ctx->cap_j + first, sizeof(double) * count,
                                   cudaMemcpyDeviceToHost, ctx->stream));
    if (m) CK(cudaMemcpyAsync(m, ctx->st.m + first, sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->stream));
    if (t) CK(cudaMemcpyAsync(t, ctx->st.t + first, sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return HH_OK;
}

int64_t hh_n_particles(const hh_ctx *ctx) { return ctx ? ctx->n : -1; }
int64_t hh_ctx_device_bytes(const hh_ctx *ctx) { return ctx ? ctx->device_bytes : -1; }
int64_t hh_n_j(const hh_ctx *ctx) { return ctx ? ctx->nj : -1; }

int hh_get_counters(hh_ctx *ctx, hh_counters *out)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!out) return fail(ctx, HH_EINVAL, "hh_get_counters: NULL");
    if ((rc = sync_and_check(ctx))) return rc;
    out->block_steps = int64_t(ctx->h_ds->block_steps);
    out->particle_steps = int64_t(ctx->h_ds->particle_steps);
    out->interactions = int64_t(ctx->h_ds->interactions);
    out->rebuilds = ctx->rebuilds;
    out->tile_steps = 0;
    for (int k = 0; k < 32; k++) out->tile_steps += int64_t(ctx->h_ds->na_hist[k]);
    out->list_steps = int64_t(ctx->h_ds->list_steps);
    return HH_OK;
}

int hh_get_tile_histogram(hh_ctx *ctx, int64_t counts[32])
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!counts) return fail(ctx, HH_EINVAL, "hh_get_tile_histogram: NULL");
    if ((rc = sync_and_check(ctx))) return rc;
    for (int k = 0; k < 32; k++) counts[k] = int64_t(ctx->h_ds->na_hist[k]);
    return HH_OK;
}

int hh_reset_counters(hh_ctx *ctx)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    CK(cudaMemsetAsync(&ctx->ds->block_steps, 0, 4 * sizeof(unsigned long long), ctx->stream));
    CK(cudaMemsetAsync(ctx->ds->na_hist, 0, sizeof(ctx->ds->na_hist), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->rebuilds = 0;
    return HH_OK;
}

int hh_force_timing(hh_ctx *ctx, int enable, double *ms_out, int64_t *launches_out)
{
    if (!ctx) return hh_set_global_error(HH_EINVAL, "hh_force_timing: NULL");
    if (ms_out) *ms_out = ctx->force_ms;
    if (launches_out) *launches_out = ctx->force_launches;
    if (enable >= 0) {
        ctx->timing = enable != 0;
        ctx->force_ms = 0.0;
        ctx->force_launches = 0;
    }
    return HH_OK;
}

int hh_load_particles(hh_ctx *ctx, int64_t n, const double *x, const double *v, const double *m, double t)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (n < 2 || n > ctx->cap_n || !x || !v || !m) return fail(ctx, HH_EINVAL, "hh_load_particles: bad n or NULL");
    std::vector<double> zeros(3 * size_t(n), 0.0), tt(size_t(n), t);
    if ((rc = validate_j_host(ctx, n, x, v, zeros.data(), zeros.data(), m, tt.data()))) return rc;
    if ((rc = set_j_impl(ctx, 0, n, x, v, zeros.data(), zeros.data(), m, tt.data(), cudaMemcpyHostToDevice))) return rc;
    ctx->n = n;
    ctx->nj = n;
    ctx->ids.resize(size_t(n));
    for (int64_t q = 0; q < n; q++) ctx->ids[size_t(q)] = q;
    ctx->ids_on_device = false;
    ctx->have_lists = false;
    ctx->have_dt = false;
    return HH_OK;
}

}  // extern "C"


// Completes a device rebuild (hh_gtree.cu): work-item capacity, sizes,
// mixed-form base records; the state buffers were swapped, so the loop graph
// is rebuilt on the next hh_advance.
int hh_finish_device_rebuild(hh_ctx *ctx, int64_t total_parts, int64_t lmax, bool batched)
{
    cudaStream_t st = ctx->stream;
    const int64_t small_parts = small_parts_bound(ctx, ctx->n_tiles, lmax);
    if (small_parts > INT32_MAX / 2) return fail(ctx, HH_ENOMEM, "hh_rebuild: too many short list parts");
    ctx->list_max = lmax;
    int rc = ensure_parts(ctx, std::max(total_parts, small_parts));
    if (rc) return rc;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    if (!batched) {
        k_set_sizes<<<1, 1, 0, st>>>(ctx->ds, ctx->n, ctx->nj, ctx->n_tiles, ctx->part_len, ctx->cfg.work_item,
                                     ctx->cfg.work_split);
        CKL();
        if (ctx->st.base) {
            k_refresh_base<<<ctx->elem_grid, 256, 0, st>>>(ctx->st, 0, ctx->nj);
            CKL();
        }
        CK(cudaStreamSynchronize(st));
    }
    ctx->total_parts = total_parts;
    ctx->small_parts = small_parts;
    ctx->have_j = true;
    ctx->have_lists = true;
    ctx->predicted = false;
    ctx->rebuilds++;
    return HH_OK;
}

extern "C" {

int hh_set_rebuild_device(hh_ctx *ctx, int on_device)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    ctx->rebuild_device = on_device != 0;
    return HH_OK;
}

}  // extern "C"

namespace {
// Checks before a rebuild; for a device rebuild also brings the particle ids
// to the device builder.
int rebuild_begin(hh_ctx *ctx)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!ctx->have_j || ctx->n < 2) return fail(ctx, HH_ESTATE, "hh_rebuild: no particles loaded");
    // until this rebuild succeeds the lists are not valid (a failure part way
    // may have overwritten them); the state stays readable
    ctx->have_lists = false;
    if (ctx->rebuild_device && ctx->gtree && !ctx->ids_on_device &&
        hh_gtree_set_ids(ctx->gtree, ctx->ids.data(), ctx->n, ctx->stream) != HH_OK)
        return fail(ctx, HH_ECUDA, "hh_rebuild: id upload failed");
    return HH_OK;
}

int rebuild_impl(hh_ctx *ctx, double t)
{
    int rc = rebuild_begin(ctx);
    if (rc) return rc;
    if (ctx->rebuild_device) return hh_rebuild_device(ctx, t);
    if ((rc = sync_ids_to_host(ctx))) return rc;
    if (!ctx->h_buf &&
        (cudaHostAlloc((void **)&ctx->h_buf, sizeof(double) * 14 * ctx->cap_j, cudaHostAllocDefault) != cudaSuccess ||
         cudaHostAlloc((void **)&ctx->h_jbuf, sizeof(double) * 14 * ctx->cap_j, cudaHostAllocDefault) != cudaSuccess)) {
        cudaGetLastError();
        return fail(ctx, HH_ENOMEM, "hh_rebuild: pinned host staging does not fit");
    }
    const int64_t n = ctx->n;
    double *H = ctx->h_buf;  // pinned: x v a jk [3][n] each, then m, t, dt
    double *hx = H, *hv = H + 3 * n, *ha = H + 6 * n, *hj = H + 9 * n, *hm = H + 12 * n, *ht = H + 13 * n;
    double *src[4] = {ctx->st.x, ctx->st.v, ctx->st.a, ctx->st.jk};
    double *dst[4] = {hx, hv, ha, hj};
    for (int f = 0; f < 4; f++)
        for (int d = 0; d < 3; d++)
            CK(cudaMemcpyAsync(dst[f] + d * n, src[f] + d * ctx->cap_j, sizeof(double) * n, cudaMemcpyDeviceToHost,
                               ctx->stream));
    CK(cudaMemcpyAsync(hm, ctx->st.m, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ht, ctx->st.t, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<double> dtv(static_cast<size_t>(n));
    CK(cudaMemcpyAsync(dtv.data(), ctx->st.dt, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int64_t q = 0; q < n; q++)
        if (ht[q] != t) return fail(ctx, HH_ESTATE, "hh_rebuild: particles are not synchronised at t");
    if ((rc = hh_tree_rebuild(&ctx->tree, n, hx, hv, ha, hj, hm, ctx->cfg.leaf, ctx->cfg.n_crit, ctx->cfg.theta,
                              ctx->cfg.order)))
        return fail(ctx, rc, std::string("hh_rebuild: ") + g_err);
    HhTreeView V;
    hh_tree_view(ctx->tree, &V);
    const int64_t nn = V.n_nodes, nj = n + nn;
    if (nj > ctx->cap_j || V.list_len > ctx->cap_list || V.n_groups > ctx->cap_g)
        return fail(ctx, HH_ENOMEM, "hh_rebuild: tree exceeds nj_max / list_max / groups_max");
    double *J = ctx->h_jbuf;  // pinned: x v a jk [3][nj], m [nj], t [nj]
    double *Jx = J, *Jv = J + 3 * nj, *Ja = J + 6 * nj, *Jj = J + 9 * nj, *Jm = J + 12 * nj, *Jt = J + 13 * nj;
    std::vector<double> dt_new(static_cast<size_t>(n));
    std::vector<int64_t> ids_new(static_cast<size_t>(n));
#pragma omp parallel for schedule(static) if (n >= 8192)
    for (int64_t k = 0; k < n; k++) {
        const int64_t i = V.perm[k];
        for (int d = 0; d < 3; d++) {
            Jx[d * nj + k] = hx[d * n + i];
            Jv[d * nj + k] = hv[d * n + i];
            Ja[d * nj + k] = ha[d * n + i];
            Jj[d * nj + k] = hj[d * n + i];
        }
        Jm[k] = hm[i];
        Jt[k] = t;
        dt_new[size_t(k)] = dtv[size_t(i)];
        ids_new[size_t(k)] = ctx->ids[size_t(i)];
    }
#pragma omp parallel for schedule(static) if (n >= 8192)
    for (int64_t c = 0; c < nn; c++) {
        for (int d = 0; d < 3; d++) {
            Jx[d * nj + n + c] = V.cx[3 * c + d];
            Jv[d * nj + n + c] = V.cv[3 * c + d];
            Ja[d * nj + n + c] = V.ca[3 * c + d];
            Jj[d * nj + n + c] = V.cj[3 * c + d];
        }
        Jm[n + c] = V.cm[c];
        Jt[n + c] = t;
    }
    if ((rc = set_j_impl(ctx, 0, nj, Jx, Jv, Ja, Jj, Jm, Jt, cudaMemcpyHostToDevice))) return rc;
    ctx->ids = ids_new;
    if ((rc = set_lists_core(ctx, n, nj, V.n_groups, V.off, V.idx, V.group_of, true))) return rc;
    CK(cudaMemcpyAsync(ctx->st.dt, dt_new.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->rebuilds++;
    return HH_OK;
}
}  // namespace

extern "C" {

int hh_rebuild(hh_ctx *ctx, double t)
{
    const int rc = rebuild_impl(ctx, t);
    if (rc == HH_OK) ctx->t_tree = t;
    return rc;
}

}  // extern "C"

int hh_rebuild_many(hh_ctx *const *ctxs, const double *ts, int k, int *rcs, RbScratch *r)
{
    // device builders of at most kBatchRebuildMaxN particles build together
    // when there are two or more of them; the rest one by one (a large tree's
    // key sort is faster as one device-wide sort than as a segment sorted by
    // one CTA, and one context alone gains nothing from the batch)
    int small = 0;
    for (int s = 0; s < k; s++)
        small += ctxs[s] && ctxs[s]->rebuild_device && ctxs[s]->n <= kBatchRebuildMaxN;
    std::vector<hh_ctx *> dev;
    std::vector<double> tdev;
    std::vector<int> where;
    for (int s = 0; s < k; s++) {
        hh_ctx *ctx = ctxs[s];
        if (small >= 2 && ctx && ctx->rebuild_device && ctx->n <= kBatchRebuildMaxN) {
            rcs[s] = rebuild_begin(ctx);
            if (rcs[s] == HH_OK) {
                dev.push_back(ctx);
                tdev.push_back(ts[s]);
                where.push_back(s);
            }
        } else {
            rcs[s] = hh_rebuild(ctx, ts[s]);
        }
    }
    if (dev.empty()) return HH_OK;
    std::vector<int> rd(dev.size(), HH_OK);
    const int rc = hh_rebuild_device_many(dev.data(), tdev.data(), int(dev.size()), rd.data(), r);
    for (size_t q = 0; q < dev.size(); q++) {
        rcs[where[q]] = rc ? fail(dev[q], rc, "hh_rebuild: batched device rebuild failed") : rd[q];
        if (rcs[where[q]] == HH_OK) dev[q]->t_tree = tdev[q];
    }
    return HH_OK;
}

extern "C" {

int hh_run(hh_ctx *ctx, double t0, double t_end)
{
    int rc = check_ctx(ctx);
    if (rc) return rc;
    const double dtt = ctx->cfg.dt_tree;
    const double k0 = t0 / dtt, k1 = t_end / dtt;
    if (k0 != std::floor(k0) || k1 != std::floor(k1) || t_end < t0)
        return fail(ctx, HH_EINVAL, "hh_run: t0 and t_end must be multiples of dt_tree");
    if ((rc = hh_rebuild(ctx, t0))) return rc;
    if ((rc = hh_init_forces(ctx, t0))) return rc;
    if ((rc = hh_rebuild(ctx, t0))) return rc;  // node derivatives from the initial forces
    ctx->rebuilds--;                            // the t0 pair counts as one build
    if ((rc = hh_init_dt(ctx))) return rc;
    for (double tt = t0; tt < t_end;) {
        const double tn = tt + dtt;
        if ((rc = hh_advance(ctx, tn, nullptr))) return rc;
        if ((rc = hh_rebuild(ctx, tn))) return rc;
        tt = tn;
    }
    return HH_OK;
}

}  // extern "C"
