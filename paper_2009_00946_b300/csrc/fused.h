// Fused FP32 path: one persistent kernel runs a whole frame (RHS, warm
// restart, n_iter iterations of Alg. 2) with bounded grid barriers.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "setup.h"

namespace fewha {

template <typename T>
struct DevGeo;

// State vectors shared with the plain path (device pointers, FP32).
struct FusedBuffers {
    float *c, *r, *p, *q, *b, *bprev, *phi;
    const float *Jinv, *aD, *slopes;
    double* sc;
    int* errw;
};

struct FusedPlan;

// Build the fused plan (tiles, work lists, cluster shape); nullptr if the
// device cannot run it (err says why), in which case the plain path is used.
FusedPlan* fused_create(const HostSetup& hs, const DevGeo<float>& G, const FusedBuffers& fb, std::string& err);

// One plan over several independent instances (solved together in one
// launch; every instance has its own tables, state and scalars).
// max_tile_side > 0 bounds the sensor tiles (nodes per side).
// forced_C > 0 builds only that cluster size (the autotuner's candidates);
// forced_V >= 0 only that layer-phase form (0 row stripes, 1 level-stacked),
// else the level-stacked form wherever it fits.
FusedPlan* fused_create_multi(const std::vector<const HostSetup*>& hs, const std::vector<DevGeo<float>>& G,
                              const std::vector<FusedBuffers>& fb, int max_tile_side, std::string& err,
                              int forced_C, int forced_V = -1);
// Cluster size and layer-phase form of a plan.
int fused_cluster_size(const FusedPlan* plan);
int fused_layer_form(const FusedPlan* plan);
void fused_destroy(FusedPlan* plan);

// Enqueue one frame on `stream`: b = W P^T Gamma^T C^{-1} s; warm restart
// (or replacement r = b - M c, or cold start); n_iter iterations of Alg. 2.
// One frame (RHS, restart, n_iter iterations) in one launch.  slopes /
// layers_out (device, may be NULL; single-instance plans only): read the
// frame's slopes from there instead of the handle's buffer (they are copied
// into it as they are read), and also write the final layers there.
// done_host (device alias of a mapped pinned host word, may be NULL; single
// instance): set to (1 << 32) | error word by the launch once all of its
// results are visible to the host, so a host caller can wait on the word.
// doorbell (device alias of a mapped pinned host word, may be NULL; single
// instance): the launch does its set-up, then waits until the word equals
// doorbell_want (at most doorbell_ns ns; then TIMEOUT and no frame work).
int fused_solve(FusedPlan* plan, const float* slopes, int n_iter, int warm, int replace, long long budget,
                cudaStream_t stream, std::string& err, long long& launches, float* layers_out = nullptr,
                unsigned long long* done_host = nullptr, const unsigned* doorbell = nullptr,
                unsigned doorbell_want = 0, long long doorbell_ns = 0);
// After a kernel error the barrier counters may be left set: zero them first
// at the next launch.
void fused_mark_dirty(FusedPlan* plan);
// A captured single-instance frame launch (kernel node `node` of the graph
// `exec` was instantiated from) re-pointed at other slopes / layers buffers,
// in the executable graph and in the node: no re-capture, no instantiation.
// Returns 0, or -1 when the node is not a fused frame launch.
int fused_repoint_node(cudaGraphExec_t exec, cudaGraphNode_t node, const float* slopes, float* layers_out);

// Plan summary (cluster shape, grid, shared memory, work items).
int fused_describe(const FusedPlan* plan, char* buf, int len);
// Per-phase globaltimer trace of the following launches (arrival / departure
// of every CTA at every grid barrier).
void fused_set_trace(FusedPlan* plan, bool on);
int fused_get_trace(FusedPlan* plan, unsigned long long* out, int max_entries, int* slots, int* grid);
// Sub-phase marks of the last traced launch: [cta][per_cta] of (tag << 56 | ns).
int fused_get_fine_trace(FusedPlan* plan, unsigned long long* out, int max_entries, int* per_cta, int* grid);

}  // namespace fewha
