// The hh_ctx structure, shared by the CUDA translation units of libhh.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "hh_internal.h"
#include "hh_kernels.cuh"

constexpr int kTjF64 = 128;  // list entries staged per chunk, plain form
constexpr int kTjMix = 256;  // list entries staged per chunk, mixed form

// Adds n to the process-wide count of kernels launched by libhh.
void hh_count_launches(int64_t n);

struct GTreeBuf;  // device tree-builder buffers (hh_gtree.cu)
void hh_gtree_free(GTreeBuf *g);
int64_t *hh_gtree_ids(GTreeBuf *g);
int hh_gtree_set_ids(GTreeBuf *g, const int64_t *ids, int64_t n, cudaStream_t st);
struct hh_ctx;
int hh_rebuild_device(hh_ctx *ctx, double t);        // hh_gtree.cu
// Batched device rebuild of k contexts (hh_gtree.cu): rcs[s] gets context
// s's result; the scratch (and its stream) belongs to the caller.
struct RbScratch;
RbScratch *hh_rb_scratch_create();
void hh_rb_scratch_free(RbScratch *r);
int hh_rebuild_device_many(hh_ctx *const *ctxs, const double *ts, int k, int *rcs, RbScratch *r);
// Ends a device rebuild (hh_api.cu): work-item capacity, then the sizes on the
// device and the mixed form's base records on the context's stream,
// synchronised.  batched: the batched build's closing kernel (k_finish) sets
// the sizes and base records, and it synchronises.
int hh_finish_device_rebuild(hh_ctx *ctx, int64_t total_parts, int64_t lmax, bool batched = false);
// hh_rebuild for k contexts (hh_api.cu): device builders of at most
// kBatchRebuildMaxN particles are rebuilt together by hh_rebuild_device_many
// (when there are two or more), the others one by one.
constexpr int64_t kBatchRebuildMaxN = 32768;
int hh_rebuild_many(hh_ctx *const *ctxs, const double *ts, int k, int *rcs, RbScratch *r);
// Block steps of the batched loop with at most this many due particles use
// list parts of tile_j_small (when set).
constexpr int kSmallDue = 16;
// Block steps of the batched plain-form loop with fewer due particles than
// work_split (when set) use equal-cost list parts of kMedWork x tile_j
// interactions (32-entry granularity).
constexpr int kMedWork = 2;

struct hh_ctx {
    int device = 0;
    hh_config cfg{};
    cudaStream_t own_stream = nullptr, stream = nullptr;
    int64_t cap_n = 0, cap_j = 0, cap_list = 0;
    int32_t cap_g = 0;
    int64_t cap_tiles = 0;
    int64_t n = 0, nj = 0, list_len = 0;
    int64_t list_max = 0;  // longest group list
    int32_t n_groups = 0, n_tiles = 0, tile_i = 32;
    // device memory
    hh::State st{};
    void *rec = nullptr;
    int64_t *off = nullptr;
    int32_t *idx = nullptr, *group_of = nullptr;
    int4 *tiles = nullptr;
    hh::WorkItem *items = nullptr;  // [cap_parts]
    void *partials = nullptr;   // [cap_parts][32] partial sums (scratch)
    int32_t *tile_cnt = nullptr;  // [cap_tiles]
    uint32_t *tile_lv = nullptr;  // [cap_tiles] levels present in each tile (batched loop)
    int64_t cap_parts = 0;
    int64_t total_parts = 0;    // work items of a step with every tile active
    int64_t small_parts = 0;    // work items a step below work_split can have beyond parts of tile_j
    int64_t device_bytes = 0;   // device memory allocated for this context
    int32_t part_len = 512;
    hh::DevScalars *ds = nullptr;
    int32_t *i_buf = nullptr;  // [cap_n]
    double *out_buf = nullptr; // [7 * cap_n]
    // pinned host staging
    hh::DevScalars *h_ds = nullptr;
    double *h_buf = nullptr;   // [14 * cap_j]
    int32_t *h_ibuf = nullptr; // [cap_n]
    double *h_jbuf = nullptr;  // [14 * cap_j] staging of the rebuilt j entries
    hh_tree *tree = nullptr;   // host tree reused by hh_rebuild
    GTreeBuf *gtree = nullptr; // device tree builder (rebuild_device)
    bool rebuild_device = false;
    bool ids_on_device = false;  // particle ids kept by the device builder
    std::vector<int64_t> ids;  // slot -> particle id
    std::vector<int32_t> h_group_of;
    // grid shapes
    int n_sm = 0, force_grid = 0, elem_grid = 0;
    // loop graph
    cudaGraphExec_t graph = nullptr;
    int graph_timed = -1;
    std::vector<cudaEvent_t> ev;  // 2 per unrolled step when timed
    // timing
    bool timing = false;
    double force_ms = 0.0;
    int64_t force_launches = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // state flags
    bool have_j = false, have_lists = false, have_dt = false, predicted = false, have_forces = false;
    int64_t rebuilds = 0;
    double t_tree = 0.0;  // time of the last successful rebuild (the j entries' base time)
    std::string err;
};

