// grouped.cuh -- the lockstep batched closure of a batch's larger graphs (grouped.cu).
#pragma once

#include <vector>

#include "tgemm.cuh"

namespace apsp {

// Graphs of kGroupMinNb..kGroupMaxNb 128-vertex blocks (257..2048 vertices) are staged.
constexpr int kGroupMinNb = 3;
constexpr int kGroupMaxNb = 16;

struct StagePlan {
  int64_t G = 0;   // staged graphs
  int64_t R = 0;   // staged rows
  int64_t NP = 0;  // leading dimension of the staging matrix (the largest nb x 128)
  int ngroups = 0;
  GraphGroup groups[kMaxGroups] = {};
  std::vector<int> staged;  // graph indices in staged order (groups by decreasing nb)
  std::vector<int> sizes;   // their host sizes
  std::vector<int> rest;    // every other graph, largest first (for the persistent kernel)
};

// Plans the staging from the host copy of the sizes; false when no graph qualifies.
bool make_stage_plan(const int32_t *ns_host, int64_t count, StagePlan &pl);

// Workspace bytes of apsp_batched with the staged path (the 256-byte word block included).
size_t staged_workspace_bytes(const StagePlan &pl, int64_t count, int dtype);

// Enqueues the whole batched closure: the graphs of pl.rest through launch_rest (the
// persistent kernel, given a device order list of nq entries), the staged graphs in lockstep.
// ws: staged_workspace_bytes(pl, count, dtype) bytes, 256-byte aligned; its first two words
// (the persistent kernel's queue counters) are zeroed by the caller.  int32: inf_i > kCap16;
// float32: inf_f is the caller's sentinel.
int batched_staged(const StagePlan &pl, int *pool, const int64_t *offsets, const int32_t *ns, const int32_t *lds,
                   int64_t count, int dtype, int inf_i, float inf_f, void *ws,
                   int (*launch_rest)(void *ctx, const int *order, int64_t nq), void *ctx, cudaStream_t s);

}  // namespace apsp
