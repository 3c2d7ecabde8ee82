// Internal declarations shared by the libhh translation units.
#pragma once

#include <cstdint>
#include <string>

#include "../../include/hh.h"

// Sets the process-wide "last error" (used where there is no context) and
// returns code.
int hh_set_global_error(int code, const char *msg);

// Read-only view of a host tree (hh_tree.cpp); node arrays are AoS [n_nodes][3].
struct HhTreeView {
    int64_t n, n_nodes, list_len;
    int32_t n_groups;
    const int32_t *perm;
    const double *cm, *cx, *cv, *ca, *cj;
    const int64_t *off;
    const int32_t *idx;
    const int32_t *group_of;
};
int hh_tree_view(const hh_tree *t, HhTreeView *v);
int hh_tree_rebuild(hh_tree **tp, int64_t n, const double *x, const double *v, const double *a, const double *jk,
                    const double *m, int32_t leaf, int32_t n_crit, double theta, int32_t order);
