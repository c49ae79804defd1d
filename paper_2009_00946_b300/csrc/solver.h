// Device-side solver of one FEWHA instance: buffers, tables and the plain
// (one kernel per operator) path; the fused persistent path lives in fused.cu.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "setup.h"

namespace fewha {

constexpr int kRedBlocks = 296;    // fixed reduction grid (2 x 148 SMs): deterministic sums
constexpr int kRedThreads = 256;

// Error bits of the device error word.
constexpr int kErrInput = 1;
constexpr int kErrBreakdown = 2;
constexpr int kErrTimeout = 4;
constexpr int kErrLaunch = 8;      // the fused kernel found a launch shape it was not planned for

// Device geometry tables (pointers into one allocation), passed by value.
template <typename T>
struct DevGeo {
    int L, G, N, S, NW, NS, Jmax, nmax, nsmax;
    const int* lay_n;
    const int* lay_J;
    const int* lay_off;
    const int* wfs_n;
    const int* wfs_soff;
    const int* wfs_noff;
    const int* wfs_moff;
    const T* wfs_w;
    const unsigned char* mask;
    const int* tab_off;
    const int* cx;
    const int* cy;
    const T* tx;
    const T* ty;
    const int* gat_off;
    const int* jlo;
    const int* jhi;
    const int* ilo;
    const int* ihi;
    const T* Jinv;
    const T* aD;
    T h[6], g[6];
    int any_tt;                       // LGS tip-tilt filter on some sensor
    const int* wfs_tt;                // per sensor: 1 = filter its slope means
    const int* wfs_nact;              // per sensor: active subapertures
};

// Device fitting tables.
template <typename T>
struct DevFit {
    int L, M, T_, NA, np1;   // np1 = pupil nodes per side
    int moao;                // 1: mirror t enters direction t only
    T eps;
    const int* lay_n;
    const int* lay_off;
    const int* dm_n;
    const int* dm_off;
    const int* ftab_off;
    const int* fcx;
    const int* fcy;
    const T* ftx;
    const T* fty;
    const int* dtab_off;
    const int* dcx;
    const int* dcy;
    const T* dtx;
    const T* dty;
    const int* dgat_off;
    const int* djlo;
    const int* djhi;
    const int* dilo;
    const int* dihi;
    // L = M co-located mirrors: per mirror, its actuators on its layer's grid
    int colocated;
    const int* ctab_off;
    const int* ccx;
    const T* ctx;
    // closed loop: mirror m at the nodes of sensor g (G*M tables)
    const int* wdtab_off;
    const int* wdcx;
    const int* wdcy;
    const T* wdtx;
    const T* wdty;
};

struct FusedPlan;   // fused.cu

// Alg. 2 scalars kept on the device (FP64).
enum Scalar { kRho = 0, kMu, kRhoOld, kAlphaOld, kBeta, kAlphaK, kRR, kRRold, kNumScalars = 16 };

class SolverBase {
  public:
    virtual ~SolverBase() {}
    virtual int set_frame(const void* s, int on_device) = 0;
    virtual int solve(int n_iter, int warm) = 0;
    virtual int fit(double gain, int n_fit, void* out, int on_device) = 0;
    virtual int get_layers(void* out, int on_device) = 0;
    virtual int get_vector(int which, void* out, int on_device) = 0;
    virtual int get_state(void* c, void* b, void* r, int on_device) = 0;
    virtual int set_state(const void* c, const void* b, const void* r, int on_device, long count) = 0;
    virtual int apply_M(const void* x, void* y, int on_device) = 0;
    virtual int frame(const void* s, int n_iter, int warm, double gain, int n_fit, void* layers_out,
                      void* dm_out, int on_device) = 0;
    virtual int sync() = 0;
    virtual int describe(char* buf, int len) = 0;
    virtual int set_trace(int on) = 0;
    virtual int get_trace(unsigned long long* out, int max_entries, int* slots, int* grid) = 0;
    virtual int get_fine_trace(unsigned long long* out, int max_entries, int* per_cta, int* grid) = 0;
    virtual int set_cluster_size(int C) = 0;
    virtual int set_layer_transform(int form) = 0;
    virtual int get_frame_timing(double* out) = 0;
    virtual int autotune(int n_iter, int reps, char* report, int len) = 0;
    virtual int set_params(const double* cn2, double alpha, const double* w) = 0;
    virtual int solve_taped(const void* slopes, int n_iter, void* tape, void* layers_out) = 0;
    virtual int backward(const void* slopes, int n_iter, const void* tape, const void* layers_bar, double* g_gam,
                         double* g_alpha, double* g_w, void* g_slopes) = 0;
    virtual size_t tape_size(int n_iter) const = 0;
    virtual size_t tape_size_batch(int n_iter, int n_frames) const = 0;
    virtual int solve_taped_batch(int n_frames, const void* slopes, int n_iter, void* tape, void* layers_out) = 0;
    virtual int backward_batch(int n_frames, const void* slopes, int n_iter, const void* tape, const void* layers_bar,
                               double* g_gam, double* g_alpha, double* g_w, void* g_slopes) = 0;
    virtual int set_loop(int closed) = 0;
    virtual int set_host_transfer(int slopes_by_copy) = 0;
    virtual int frame_arm(const void* slopes, int n_iter, int warm, void* layers_out, double wait_s) = 0;
    virtual int frame_fire() = 0;
    virtual bool is_armed() const = 0;
    virtual int operator_dims(int op, long& n_in, long& n_out) = 0;
    virtual int apply_operator(int op, const void* x, void* y, int on_device) = 0;
    virtual int time_operator(int op, int reps, double* us) = 0;

    HostSetup hs;
    cudaStream_t stream = 0;
    int path = FEWHA_PATH_PLAIN;
    int k_rr = 10;
    long long barrier_budget = (1LL << 31);
    long long frame_count = 0;
    long long launches = 0;
    bool have_frame = false;
    bool fused_available = false;   // a fused plan exists for this geometry
    std::string fused_reason;       // else why not (set when the handle is created)
    std::string err;
};

SolverBase* make_solver(const HostSetup& hs, cudaStream_t stream, std::string& err, int& status);

// Many independent FP32 instances advanced together by one fused launch per
// group of instances (one group unless split) per frame: slopes and layers
// are concatenated in instance order.
class BatchBase {
  public:
    virtual ~BatchBase() {}
    virtual int frame(const void* slopes, int n_iter, int warm, void* layers_out, int on_device) = 0;
    virtual int sync() = 0;
    virtual int describe(char* buf, int len) = 0;
    virtual int get_state(int inst, void* c, void* b, void* r, int on_device) = 0;
    virtual int set_trace(int on) = 0;
    virtual int get_fine_trace(unsigned long long* out, int max_entries, int* per_cta, int* grid) = 0;
    virtual int autotune(int n_iter, int reps, char* report, int len) = 0;
    virtual int set_groups(const int* group, int count) = 0;

    std::vector<long> coeff_off, slope_off;   // count + 1 offsets
    int max_tile_side = 0, cluster_size = 0;  // as created: the plans of new groups follow them
    int max_launches = 0;                     // the autotuner's bound on launches per frame (0: none)
    cudaStream_t stream = 0;
    int k_rr = 10;
    long long barrier_budget = (1LL << 31);
    long long frame_count = 0;
    long long launches = 0;
    std::string err;
};

BatchBase* make_batch(const std::vector<HostSetup>& hss, cudaStream_t stream, int max_tile_side,
                      int cluster_size, std::string& err, int& status);

}  // namespace fewha
