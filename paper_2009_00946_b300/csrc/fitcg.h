// Persistent FP32 mirror fit: the least-squares fit of Alg. 1 (reading R10,
// R17 for the LTAO / MOAO modes) by plain CG on its normal equations, n_fit
// steps warm-started from the previous solution, followed by the open- or
// closed-loop gain -- all in one cooperative launch.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "solver.h"

namespace fewha {

// Device buffers of one handle's fit (FP32).  v: [T][np1^2] pupil samples;
// x, r, p, p2, q: [NA]; acur, aprev: the mirror state the gain updates.
struct FitCgBuffers {
    float *v, *x, *r, *p, *p2, *q, *acur, *aprev;
    double* part;     // partial sums (fitcg_part_doubles of them)
    unsigned* bar;    // [2] barrier arrivals, exits (zero before the first launch)
    int* errw;        // error word (kErrTimeout on an expired barrier)
};

struct FitCgPlan;

// Plan for the handle's fit geometry (grid = one CTA per SM, cooperative):
// assembles the normal matrix A = sum_t P^DM_t^T P^DM_t + eps I from the
// host's mirror sample tables (CSR, FP32 values) and uploads it; nullptr if
// the device cannot co-schedule the kernel (err says why).
FitCgPlan* fitcg_create(const HostSetup& hs, const DevFit<float>& F, std::string& err);
// Non-zeros of the assembled normal matrix (for the plan summary).
long fitcg_nnz(const FitCgPlan* plan);
void fitcg_destroy(FitCgPlan* plan);
int fitcg_grid(const FitCgPlan* plan);
// Size of the partial-sum buffer the launch needs (doubles).
size_t fitcg_part_doubles(const FitCgPlan* plan);
// After a kernel error the barrier counters may be left set: zero them first
// at the next launch.
void fitcg_mark_dirty(FitCgPlan* plan);
// Enqueue the fit of the layers phi (device, FP32) and the gain on `stream`.
int fitcg_launch(FitCgPlan* plan, const DevFit<float>& F, const float* phi, const FitCgBuffers& b, int n_fit,
                 float gain, int closed, long long budget, cudaStream_t stream, std::string& err,
                 long long& launches);

}  // namespace fewha
