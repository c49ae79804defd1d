// Fused FP32 FEWHA frame: one persistent cooperative kernel runs Alg. 1 up to
// the PCG and n_iter iterations of Alg. 2 (operator M of Eq. (fewha) applied
// matrix-free once per iteration), with FP64 reductions and scalars.
//
// Work decomposition (two kinds of phases, separated by grid barriers):
//   * layer phase: one thread-block cluster per layer; the layer's n x n array
//     is split into row stripes of R = n / C rows, one per CTA of the cluster,
//     kept in shared memory.  P^T (deterministic gather from the sensor
//     fields), the forward db3 DWT W, the Alg. 2 update, z = J^{-1} r and the
//     inverse DWT W^T run there; the column passes of the DWT read the other
//     stripes through distributed shared memory, one cluster barrier per level.
//   * sensor phase: one CTA per sensor tile: bilinear P of every layer (each
//     node's four cells per layer read in the L2), Gamma, C^{-1}, Gamma^T; the
//     data part of mu = (M z, z) = sum_g w_g |mask Gamma P W^T z|^2 is reduced
//     here, the regulariser part alpha (D z, z) in the layer phase.
// Per iteration: layer phase -> barrier -> sensor phase -> barrier.  Every sum
// is taken in a fixed order (per-item partials), so results are bit-identical
// from run to run.  The control flow never depends on data, so cluster
// barriers are always reached by every CTA; grid barriers spin with a clock
// budget and set the TIMEOUT bit when it runs out.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "debug.cuh"
#include "fused.h"
#include "solver.h"

namespace cg = cooperative_groups;

namespace fewha {

FEWHA_DBG_READER(dbg_read_fused)

constexpr int kFThreads = 512;
constexpr int kMaxC = 16;
constexpr int kMaxLayersFused = 64;
constexpr int kMaxWfsFused = 16;
constexpr int kFineCap = 4096;   // sub-phase marks per CTA per traced launch (a batch's CTAs take many items)
constexpr int kMaxKG = 4;        // P^T gather entries per layer row / column

// sensor phases: the RHS (weighted slopes), the data term of M on the
// current layers, and the data residual s - Gamma P phi of a residual
// replacement (weighted, then Gamma^T)
enum { kModeRhs = 0, kModeData = 1, kModeResid = 2 };
enum { kLpRhsStart = 0, kLpRhsRepl = 1, kLpReplStart = 2, kLpIter = 3 };

// One instance's device tables and state.
struct FInst {
    int L, G, N, NW;
    const int *lay_n, *lay_J, *lay_off;
    const int *wfs_n, *wfs_soff, *wfs_noff, *wfs_moff;
    const float* wfs_w;
    const unsigned char* mask;
    const int *tab_off, *cx, *cy;
    const float *tx, *ty;
    const int *gat_off, *jlo, *jhi, *ilo, *ihi;
    const float *Jinv, *aD;
    float *c, *r, *p, *q, *b, *bprev, *phi, *psi;
    const float* slopes;
    double* scal;          // [2 parities][2] = rho_old, alpha_old
    double* sc_out;        // final scalars for the host (kRho...)
    int w0, nw, l0, nl;    // ranges in the item lists
    // compact gather tables of P^T per (g, l): n x KG column entries (j, w)
    // then n x KG row entries (i, w); w as float bits, padding has w = 0
    const int2* gtab;
    const int* gtab_off;
    int KG;
    // CTA that computes part A of this instance's CG scalars during the
    // sensor phase and publishes it in preA[2 parities][6] (-1: the layer CTAs
    // compute it themselves)
    int preA_cta;
    double* preA;
    // the same CTA finishes the scalars at the start of the layer phase,
    // writes the instance's outputs, and publishes the FP64 alpha_k and
    // beta_k as four 64-bit words {32 bits of the double, tag k + 1} in
    // pubAB[2 parities][4] (alpha high, alpha low, beta high, beta low): a
    // word is read whole, so a layer CTA rebuilds both doubles exactly once
    // all four tags match, with no flag and no release / acquire round trip
    // (zeroed at launch start)
    unsigned long long* pubAB;
    // LGS tip-tilt filter (reading R15; level-stacked plans): per sensor the
    // flag, its active subapertures, its tiles [x, x + y) in the item list,
    // and the nodes where Gamma^T (mask 1_x) or Gamma^T (mask 1_y) is nonzero
    // (entries [x, x + y) of tt_nz: node in the sensor, the two values' bits)
    int tt_any;
    const int* tt;
    const int* nact;
    const int2* tt_tiles;
    const int2* tt_nzr;
    const int4* tt_nz;
};

struct WItem { int inst, g, i0, i1, j0, j1; };
struct PfChunk { const char* p; int bytes, pad; };   // <= 4 KB of data to bring into L2
struct LItem { int inst, l, stg, csh; };   // csh: offset of the layer shape's cascade tables

struct FParams {
    const FInst* inst;
    const WItem* witems;
    const LItem* litems;
    const int2* stg;       // Pt staging row ranges per (layer item, rank, sensor)
    float2* wpart;         // [n_witems] data part of mu, double-float (hi, lo)
    float4* tpart;         // [n_witems] tip-tilt filtered sensors: sums of the masked x and y slopes (df pairs)
    float4* lpart;         // [2][n_litems * C] (rho hi, lo, alpha D z.z hi, lo)
    // static work lists: sensor tiles of CTA b are wsched[wsched_off[b] ..
    // wsched_off[b+1]), layer items of cluster k lsched[lsched_off[k] ..)
    const int* wsched;
    const int* wsched_off;
    const int* lsched;
    const int* lsched_off;
    unsigned* bar;         // [0] grid-barrier arrivals, [1] exits (the last CTA out zeroes both),
                           // [2] the go of an armed frame passed on in device memory
    const float* slopes_in;   // single instance: read the frame's slopes here (and copy them to I.slopes)
    float* phi_out;           // single instance: also write the final layers here
    // single instance, may be NULL: a word in mapped pinned host memory that
    // the last CTA out sets to (1 << 32) | error word once every result of
    // the launch (host-mapped layers included) is visible to the host
    unsigned long long* done_host;
    // single instance, may be NULL: an armed frame (launched ahead of its
    // slopes) waits after its set-up until this mapped host word equals
    // doorbell_want, at most doorbell_ns nanoseconds (then TIMEOUT, no frame)
    const unsigned* doorbell;
    unsigned doorbell_want;
    long long doorbell_ns;
    int* errw;
    unsigned long long* trace;   // optional: [slot][cta][arrive, depart] globaltimer (ns)
    int trace_slots;
    unsigned long long* ftrace;  // optional: [cta][fcap] (tag << 56 | ns) marks inside the phases
    int fcap;
    long long budget;
    int n_inst, n_witems, n_litems;
    int grid;              // planned grid (the work lists have grid + 1 / grid / C + 1 offsets)
    int res_first, n_res;  // CTAs res_first + i publish part A of instance i's CG scalars
    // many instances (no reserved CTAs): duty[cta] = the instance whose CG
    // scalars that CTA computes once per iteration and publishes (part A after
    // its sensor tiles, part B first thing in the layer phase), or -1; NULL:
    // the reserved CTAs above, or every layer item computing its own
    const int* duty;
    int n_iter, warm, replace, out_layers;
    int C;
    int stripe_floats, stage_floats, tile_nodes, tile_subaps, tile_rows, tile_cols;
    int ltab_off, stab_off;   // dynamic shared memory (floats) of the layer / sensor tables
    int shared_tables;        // 1: the tables lie in the phases' common working area (rebuilt per phase)
    const PfChunk* pf;        // [grid][pf_per_cta] chunks each CTA prefetches into L2 at the start
    int pf_per_cta;
    int G_max, n_max;
    float h[6], g[6];
    // level-stacked layer phase (variant 1; see fused_cascade.cuh)
    const int* cshape;        // ownership tables, one block per layer shape (n, J)
    const int4* stg4;         // staging boxes per (layer item, rank, sensor): rows [x, y), columns [z, w)
    int v_z, v_t, v_u, v_r, v_c, v_tab;   // shared-memory offsets (floats)
    int v_rmax, v_smax;       // widest column stripe, most slots of a rank
    int v_tumax;              // own-map capacity (a multiple of 4)
    // resident iteration state (level-stacked plans whose clusters keep one
    // layer item for the launch): r, p, q, c, J^{-1}, alpha D of the owned
    // coefficients live in 6 arrays of v_sts floats at v_st from the first
    // layer phase of the frame on; c and r go back to global memory in the
    // last iteration (-1: the state is read and written in place)
    int v_st, v_sts;
};

// ---------------------------------------------------------------------------
// grid barrier with a clock budget
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Two 64-bit words, each read / written whole (relaxed, GPU scope).
__device__ __forceinline__ void st_relaxed_v2(unsigned long long* p, unsigned long long a, unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void ld_relaxed_v2(const unsigned long long* p, unsigned long long& a,
                                              unsigned long long& b) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void trace_mark(const FParams& P, int slot, int which) {
    if (P.trace && slot < P.trace_slots)
        P.trace[((size_t)slot * gridDim.x + blockIdx.x) * 2 + which] = global_ns();
}

// Sub-phase mark: thread 0 records (tag, time) in this CTA's row.  Callers
// synchronise the CTA first (only when tracing), so the mark closes the step.
__device__ int* fmark_counter() {
    __shared__ int cnt;
    return &cnt;
}

// Mark by thread 0 alone (no block barrier): for steps inside warp 0's work.
__device__ __forceinline__ void fmark0(const FParams& P, int tag) {
    if (!P.ftrace || threadIdx.x != 0) return;
    int* c = fmark_counter();
    if (*c < P.fcap)
        P.ftrace[(size_t)blockIdx.x * P.fcap + (*c)++] = ((unsigned long long)tag << 56) |
                                                         (global_ns() & 0x00FFFFFFFFFFFFFFull);
}

__device__ __forceinline__ void fmark(const FParams& P, int tag) {
    if (!P.ftrace) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        int* c = fmark_counter();
        if (*c < P.fcap)
            P.ftrace[(size_t)blockIdx.x * P.fcap + (*c)++] = ((unsigned long long)tag << 56) |
                                                             (global_ns() & 0x00FFFFFFFFFFFFFFull);
    }
}

// Arrive: one release reduction per CTA (cumulative over the CTA's writes,
// which the block barrier orders before it); wait: thread 0 polls with
// acquire loads and a short back-off (fewer polls on the counter's line leave
// the L2 slice free for the arrivals), bounded by the clock budget.  The
// acquire load that sees the last arrival orders everything after it, and the
// block barrier passes that on to the CTA's other threads.
__device__ void grid_barrier(const FParams& P, unsigned& target, int* s_abort, int& slot) {
    __syncthreads();
    if (threadIdx.x == 0) {
        trace_mark(P, slot, 0);
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(P.bar), "r"(1u) : "memory");
        if (!*s_abort) {
            long long t0 = clock64();
            while ((int)(ld_acquire_gpu(P.bar) - target) < 0) {
                if (clock64() - t0 > P.budget) {
                    atomicOr(P.errw, kErrTimeout);
                    *s_abort = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
        trace_mark(P, slot, 1);
    }
    ++slot;
    __syncthreads();
}

// 16-byte global -> shared copy that bypasses L1 (the source was written by
// other SMs in this launch); both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(float* smem_dst, const float* gsrc, int site = kDbgStgDst) {
    if (!FEWHA_IN_SMEM(smem_dst, 16, site)) return;
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
    if (!FEWHA_IN_SMEM(smem_dst, 4, kDbgTables)) return;
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
    if (!FEWHA_IN_SMEM(smem_dst, 8, kDbgTables)) return;
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}

// Dot-product partials without per-element FP64 work (FP64 runs at a small
// fraction of the FP32 rate on this part): a*b = p + e exactly (p = fl(a*b),
// e = fma(a, b, -p)), and the running sum is kept as an unevaluated pair
// hi + lo updated by TwoSum, so a thread's partial carries about 48 bits; the
// partials are combined in FP64.
// The _rn intrinsics keep the compiler from contracting these steps into FMAs,
// which would break the error-free transforms.
struct Acc2 {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float s = __fadd_rn(hi, x), bb = __fsub_rn(s, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
        hi = s;
    }
    // += a * b
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        add(p);
        lo = __fadd_rn(lo, fmaf(a, b, -p));
    }
    // += a * b * c  (a*b split exactly first)
    __device__ __forceinline__ void add_prod3(float a, float b, float c) {
        const float p = __fmul_rn(a, b), e = fmaf(a, b, -p);
        add_prod(p, c);
        lo = __fadd_rn(lo, __fmul_rn(e, c));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Double-float sums for the block reductions: the FP64 pipe of this part
// issues about two FMAs per clock per SM, so FP64 work done by every thread
// of a block at once (conversions, shuffle-adds) costs microseconds; pairs of
// floats combined by TwoSum keep about 44 bits and stay on the FP32 pipe.
// Only thread 0 forms the FP64 result.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (h, l) += (bh, bl), renormalised
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
    float s, e;
    two_sum(h, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(l, bl));
    h = __fadd_rn(s, e);
    l = __fsub_rn(e, __fsub_rn(h, s));
}

// Block sums of two accumulators as double-float pairs (hi, lo) of A and B
// (red: 32 float4 of shared memory); valid in thread 0.  Every thread must
// call it.
__device__ __forceinline__ float4 block_reduce2(const Acc2& A, const Acc2& B, float4* red) {
    float ah, al, bh, bl;
    two_sum(A.hi, A.lo, ah, al);
    two_sum(B.hi, B.lo, bh, bl);
    for (int o = 16; o > 0; o >>= 1) {
        const float x0 = __shfl_down_sync(0xffffffffu, ah, o), x1 = __shfl_down_sync(0xffffffffu, al, o);
        const float y0 = __shfl_down_sync(0xffffffffu, bh, o), y1 = __shfl_down_sync(0xffffffffu, bl, o);
        df_add(ah, al, x0, x1);
        df_add(bh, bl, y0, y1);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = make_float4(ah, al, bh, bl);
    __syncthreads();
    if (w == 0) {
        const float4 v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        ah = v.x;
        al = v.y;
        bh = v.z;
        bl = v.w;
        for (int o = 16; o > 0; o >>= 1) {
            const float x0 = __shfl_down_sync(0xffffffffu, ah, o), x1 = __shfl_down_sync(0xffffffffu, al, o);
            const float y0 = __shfl_down_sync(0xffffffffu, bh, o), y1 = __shfl_down_sync(0xffffffffu, bl, o);
            df_add(ah, al, x0, x1);
            df_add(bh, bl, y0, y1);
        }
    }
    return make_float4(ah, al, bh, bl);
}

// The CG scalars of iteration k, by warp 0 alone (no block barrier inside;
// the caller synchronises the block before sh[] is read).  Partials are
// summed in a fixed order as double-float pairs, so every CTA of an instance
// obtains bit-identical scalars.
//  part A needs only the previous layer phase: rho_k, the regulariser part of
//         mu_k, beta_k = rho_k / rho_{k-1} and t_k = rho_k^2 / (rho_{k-1}
//         alpha_{k-1}) (two divisions on two lanes at once);
//  part B adds the sensor part of mu_k (this iteration's sensor phase) and
//         forms alpha_k = rho_k / (mu_k - t_k).
struct ScalA {
    double rho, beta, t, aold;
    float mh, ml;   // regulariser part of mu, double-float
};

__device__ __forceinline__ void warp_df_sum(float& h, float& l) {
    // butterfly: df_add is commutative, so every lane ends with the same sum
    for (int o = 16; o > 0; o >>= 1) {
        const float a0 = __shfl_xor_sync(0xffffffffu, h, o), a1 = __shfl_xor_sync(0xffffffffu, l, o);
        df_add(h, l, a0, a1);
    }
}

__device__ __forceinline__ double df_to_double(float h, float l) {
    // lanes 0 / 1 convert one float each; every lane receives the sum
    const int lane = threadIdx.x & 31;
    const double d = (double)(lane == 0 ? h : l);
    return __shfl_sync(0xffffffffu, d + __shfl_down_sync(0xffffffffu, d, 1), 0);
}

__device__ void alg2_part_a(const FParams& P, const FInst& I, int k, ScalA& A) {
    const int lane = threadIdx.x & 31, C = P.C, par = k & 1;
    double rho_old = 1.0, aold = 1.0;
    if (k > 0) {   // issued first: independent of the partials
        const double* so = I.scal + ((k - 1) & 1) * 2;
        rho_old = __ldcg(so);
        aold = __ldcg(so + 1);
    }
    fmark0(P, 40);
    const float4* lp = P.lpart + (size_t)par * P.n_litems * C + (size_t)I.l0 * C;
    float rh = 0.f, rl = 0.f, mh = 0.f, ml = 0.f;
    // written by other CTAs in this launch: read through L2, never L1; up to
    // 8 entries per lane per round, all loads issued before the adds, then a
    // pairwise tree over them (depth 3) and one add into the running sums
    const int nlc = I.nl * C;
    for (int e0 = lane; e0 < nlc; e0 += 8 * 32) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = (e0 + 32 * u < nlc) ? __ldcg(lp + e0 + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int st = 1; st < 8; st <<= 1)
#pragma unroll
            for (int u = 0; u < 8; u += 2 * st) {
                df_add(v[u].x, v[u].y, v[u + st].x, v[u + st].y);
                df_add(v[u].z, v[u].w, v[u + st].z, v[u + st].w);
            }
        df_add(rh, rl, v[0].x, v[0].y);
        df_add(mh, ml, v[0].z, v[0].w);
    }
    warp_df_sum(rh, rl);
    warp_df_sum(mh, ml);
    fmark0(P, 41);
    const double rho = df_to_double(rh, rl);
    double beta = 0.0, t = 0.0;
    if (k > 0) {
        const double num = (lane == 1) ? rho * rho : rho;
        const double den = (lane == 1) ? rho_old * aold : rho_old;
        const double q = num / den;
        beta = __shfl_sync(0xffffffffu, q, 0);
        t = __shfl_sync(0xffffffffu, q, 1);
    }
    A.rho = rho;
    A.beta = beta;
    A.t = t;
    A.aold = (k > 0) ? aold : 0.0;
    A.mh = mh;
    A.ml = ml;
    fmark0(P, 42);
}

__device__ void alg2_part_b(const FParams& P, const FInst& I, int k, const ScalA& A, double* sh) {
    const int lane = threadIdx.x & 31;
    float wh = 0.f, wl = 0.f;
    for (int e0 = lane; e0 < I.nw; e0 += 8 * 32) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = (e0 + 32 * u < I.nw) ? __ldcg(P.wpart + I.w0 + e0 + 32 * u) : make_float2(0.f, 0.f);
#pragma unroll
        for (int st = 1; st < 8; st <<= 1)
#pragma unroll
            for (int u = 0; u < 8; u += 2 * st) df_add(v[u].x, v[u].y, v[u + st].x, v[u + st].y);
        df_add(wh, wl, v[0].x, v[0].y);
    }
    warp_df_sum(wh, wl);
    float mh = A.mh, ml = A.ml;
    df_add(mh, ml, wh, wl);
    double mu = df_to_double(mh, ml);
    if (I.tt_any) {
        // filtered sensors: s^T C^{-1} s = w (sum mask s^2 - (sum mask s)^2 / n_act)
        // per axis; the tiles summed the masked slopes, here the square terms go
        double corr = 0.0;
        for (int g = 0; g < I.G; ++g) {
            if (!I.tt[g]) continue;
            const int2 tr = I.tt_tiles[g];
            float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f;
            for (int e = lane; e < tr.y; e += 32) {
                const float4 v = __ldcg(P.tpart + tr.x + e);
                df_add(xh, xl, v.x, v.y);
                df_add(yh, yl, v.z, v.w);
            }
            warp_df_sum(xh, xl);
            warp_df_sum(yh, yl);
            const double Mx = df_to_double(xh, xl), My = df_to_double(yh, yl);
            corr += (double)I.wfs_w[g] * (Mx * Mx + My * My) / (double)I.nact[g];
        }
        mu -= corr;
    }
    const double denom = (k > 0) ? mu - A.t : mu;
    double a = A.rho / denom;
    double beta = A.beta;
    fmark0(P, 43);
    if (lane == 0) {
        const bool bad = !(denom > 0.0) || !isfinite(a) || !isfinite(beta);
        if (bad) {
            a = 0.0;
            beta = 0.0;
        }
        sh[0] = a;
        sh[1] = beta;
        sh[2] = A.rho;
        sh[3] = mu;
        sh[4] = bad ? 1.0 : 0.0;
        sh[5] = (a != 0.0) ? a : A.aold;
    }
}

// Static data of the work items a CTA is on, in shared memory: descriptors,
// interpolation and gather tables are (re)built only when the item changes,
// so a CTA that owns one sensor tile and one layer item for the whole launch
// reads them from global memory once.
struct CtaCache {
    int wkey, lkey, wtab;       // cached sensor item, layer item; interpolation tables built
    int ltkey;                  // layer item whose staging ranges and gather tables are built
    int ltx;                    // layer item whose gather tables are rewritten to staging offsets
    int lres, il_valid;         // the CTA has one layer item for the launch; IL holds it
    int pre_k;                  // iteration whose scalar part A is in pre (-1: none)
    double pre[6];              // rho, beta, t, alpha_{k-1}, mu part (as two floats)
    WItem W;
    LItem LI;
    int ns, w_noff, w_soff, w_moff;
    float w;
    int n, J, off;
    FInst IW, IL;
};

// Descriptors of sensor item `item` into the CTA cache (one thread).
__device__ __forceinline__ void sensor_desc(const FParams& P, int item, CtaCache* cc) {
    cc->W = P.witems[item];
    cc->IW = P.inst[cc->W.inst];
    const int gg = cc->W.g;
    cc->ns = cc->IW.wfs_n[gg];
    cc->w_noff = cc->IW.wfs_noff[gg];
    cc->w_soff = cc->IW.wfs_soff[gg];
    cc->w_moff = cc->IW.wfs_moff[gg];
    cc->w = cc->IW.wfs_w[gg];
    cc->wkey = item;
    cc->wtab = 0;
}

// Descriptors of layer item `li` into the CTA cache (one thread).
__device__ __forceinline__ void layer_desc(const FParams& P, int li, CtaCache* cc) {
    cc->LI = P.litems[li];
    cc->IL = P.inst[cc->LI.inst];
    const int ll = cc->LI.l;
    cc->n = cc->IL.lay_n[ll];
    cc->J = cc->IL.lay_J[ll];
    cc->off = cc->IL.lay_off[ll];
    cc->lkey = li;
    cc->il_valid = 1;
}

// Per-sensor staging ranges of the P^T gather, [sensor][8] ints.
__device__ int* sgi_buf() {
    __shared__ int sgi[8 * kMaxWfsFused];
    return sgi;
}

// Staging ranges (threads < G) and gather tables (cp.async by every thread)
// of the cached layer item for this rank.  The caller waits for the copies
// and synchronises the CTA before the tables or ranges are read.
__device__ void layer_tables(const FParams& P, int rank, const CtaCache* cc, float* sm) {
    const int tid = threadIdx.x, NT = blockDim.x;
    const LItem& LI = cc->LI;
    const FInst& I = cc->IL;
    const int n = cc->n, R = n / P.C, row0 = rank * R, G = I.G, L = I.L, l = LI.l, KG = I.KG;
    int* sgi = sgi_buf();
    if (tid < G) {
        // staged rows imin..imax-1 of sensor tid are one contiguous range of
        // the field array; it is copied from the 16-byte boundary below its
        // start, so its data begin (start & 3) floats into its staging slot
        auto range = [&](int g, int& a0, int& c4, int& s0) {
            const int2 r2 = P.stg[LI.stg + rank * G + g];
            const int np1 = I.wfs_n[g] + 1;
            s0 = I.wfs_noff[g] + r2.x * np1;
            const int e0 = I.wfs_noff[g] + r2.y * np1;
            a0 = s0 & ~3;
            c4 = (r2.y > r2.x) ? (e0 - a0 + 3) >> 2 : 0;
        };
        int so = 0, a0, c4, s0;
        for (int g = 0; g < tid; ++g) {
            range(g, a0, c4, s0);
            so += c4 << 2;
        }
        range(tid, a0, c4, s0);
        const int2 rg = P.stg[LI.stg + rank * G + tid];
        sgi[tid * 8 + 0] = rg.x;
        sgi[tid * 8 + 1] = rg.y;
        sgi[tid * 8 + 2] = so + (s0 - a0);
        sgi[tid * 8 + 3] = I.wfs_n[tid] + 1;
        sgi[tid * 8 + 4] = a0;
        sgi[tid * 8 + 5] = c4;
        sgi[tid * 8 + 6] = so;
    }
    // compact gather tables: columns for every sensor, rows of this stripe
    int2* xt = (int2*)(sm + P.ltab_off);        // [g][q][KG]  (j, w)
    int2* yt = xt + P.G_max * P.n_max * KG;     // [g][row][KG] (i, w)
    for (int e = tid; e < G * n * KG; e += NT) {
        const int g = e / (n * KG), r = e - g * n * KG;
        cp_async8(xt + e, I.gtab + I.gtab_off[g * L + l] + r);
    }
    for (int e = tid; e < G * R * KG; e += NT) {
        const int g = e / (R * KG), r = e - g * R * KG;
        cp_async8(yt + e, I.gtab + I.gtab_off[g * L + l] + n * KG + row0 * KG + r);
    }
}

// ---------------------------------------------------------------------------
// sensor phase: P, Gamma, C^{-1}, Gamma^T on one tile of nodes
// ---------------------------------------------------------------------------
__device__ void sensor_tile(const FParams& P, int item, float* sm, int mode, bool want_mu, double* red, CtaCache* cc,
                            int k) {
    const int tid = threadIdx.x, NT = blockDim.x;
    fmark(P, mode == kModeRhs ? 30 : 20);
    if (P.shared_tables && tid == 0) cc->lkey = cc->ltkey = cc->ltx = -1;   // this phase overwrites the layer tables
    if (cc->wkey != item) {
        __syncthreads();   // the previous item's data may still be in use
        if (tid == 0) sensor_desc(P, item, cc);
        __syncthreads();
    }
    const WItem& W = cc->W;
    const FInst& I = cc->IW;
    const int g = W.g, ns = cc->ns, np1 = ns + 1, L = I.L;
    // psi nodes [a_lo, a_hi] x [b_lo, b_hi]; subapertures [a_lo, sa_hi) x [b_lo, sb_hi)
    const int a_lo = max(W.i0 - 1, 0), a_hi = min(W.i1, ns);
    const int b_lo = max(W.j0 - 1, 0), b_hi = min(W.j1, ns);
    const int sa_hi = min(W.i1, ns), sb_hi = min(W.j1, ns);
    const int nsr = max(sa_hi - a_lo, 0), nsc = max(sb_hi - b_lo, 0);
    const int pr = a_hi - a_lo + 1, pc = b_hi - b_lo + 1;
    float* psi = sm;
    float* slx = psi + P.tile_nodes;
    float* sly = slx + P.tile_subaps;
    // per-tile interpolation tables: [l][row] (layer offset, weight bits),
    // [l][col] (column, weight bits) pairs, one 8-byte load each
    int2* rtab = (int2*)(sm + P.stab_off);
    int2* ctab = rtab + L * P.tile_rows;
    Acc2 mu, tmx, tmy;   // tmx, tmy: masked slope sums of a tip-tilt filtered sensor
    const bool ttg = I.tt_any && I.tt[g];
    const int ns2 = ns * ns;
    if (mode != kModeRhs) {
        // part A of the next layer phase's CG scalars
        if (want_mu && tid < 32 && cc->lres && cc->il_valid && cc->IL.preA_cta < 0) {
            ScalA A;
            alg2_part_a(P, cc->IL, k, A);
            if (tid == 0) {
                cc->pre[0] = A.rho;
                cc->pre[1] = A.beta;
                cc->pre[2] = A.t;
                cc->pre[3] = A.aold;
                cc->pre[4] = (double)A.mh;
                cc->pre[5] = (double)A.ml;
                cc->pre_k = k;
            }
        }
        cp_async_wait_all();   // copies issued at launch start for the first layer item
        if (!cc->wtab) {
            // interpolation tables of the tile: per layer and node row the
            // offset of the row's cells in the layer and the weight; per node
            // column the column and the weight
            for (int e = tid; e < L * (pr + pc); e += NT) {
                const int l = e / (pr + pc), k = e - l * (pr + pc);
                const int base = I.tab_off[g * L + l];
                if (k < pr)
                    rtab[l * P.tile_rows + k] =
                        make_int2(I.lay_off[l] + __ldg(I.cy + base + a_lo + k) * I.lay_n[l],
                                  __float_as_int(__ldg(I.ty + base + a_lo + k)));
                else
                    ctab[l * P.tile_cols + k - pr] = make_int2(__ldg(I.cx + base + b_lo + k - pr),
                                                               __float_as_int(__ldg(I.tx + base + b_lo + k - pr)));
            }
            if (tid == 0) cc->wtab = 1;
        }
        __syncthreads();
        fmark(P, 21);
        for (int e = tid; e < pr * pc; e += NT) {
            // the layers read in the L2 (written by other SMs in this launch:
            // not through L1), every node's four cells per layer
            const int ii = e / pc, jj = e - ii * pc;
            float acc = 0.f;
#pragma unroll 3
            for (int l = 0; l < L; ++l) {
                const int n = I.lay_n[l];
                const int2 rt = rtab[l * P.tile_rows + ii], ct = ctab[l * P.tile_cols + jj];
                const float ty = __int_as_float(rt.y), tx = __int_as_float(ct.y);
                if (!FEWHA_IN(rt.x + ct.x, I.N, n + 2, kDbgWinSrc)) continue;
                const float* f = I.phi + rt.x + ct.x;
                acc += (1.f - ty) * ((1.f - tx) * __ldcg(f) + tx * __ldcg(f + 1)) +
                       ty * ((1.f - tx) * __ldcg(f + n) + tx * __ldcg(f + n + 1));
            }
            psi[e] = acc;
        }
        __syncthreads();
        fmark(P, 22);
        const float w = cc->w;
        const float* Sm = I.slopes + cc->w_soff;   // the frame's slopes (residual mode)
        for (int e = tid; e < nsr * nsc; e += NT) {
            const int aa = e / nsc, bb = e - aa * nsc;
            const int a = a_lo + aa, b = b_lo + bb;
            if (!FEWHA_IN(a * ns + b, ns2, 1, kDbgSlopes)) continue;
            const float* pp = psi + aa * pc + bb;
            float sx = ((pp[1] - pp[0]) + (pp[pc + 1] - pp[pc])) / 2;
            float sy = ((pp[pc] - pp[0]) + (pp[pc + 1] - pp[1])) / 2;
            if (mode == kModeResid) {
                // measured minus modelled slopes: the residual of a replacement
                // frame without the cancellation of b - M c (b and M c agree to
                // a few per cent, their difference loses the digits)
                const float mx = __ldcg(Sm + a * ns + b), my = __ldcg(Sm + ns2 + a * ns + b);
                sx = (isfinite(mx) ? mx : 0.f) - sx;
                sy = (isfinite(my) ? my : 0.f) - sy;
            }
            const float wm = I.mask[cc->w_moff + a * ns + b] ? w : 0.f;
            slx[e] = wm * sx;
            sly[e] = wm * sy;
            if (want_mu && a >= W.i0 && b >= W.j0) {
                mu.add_prod3(wm, sx, sx);
                mu.add_prod3(wm, sy, sy);
            }
            if (ttg && wm != 0.f && a >= W.i0 && b >= W.j0) {
                tmx.add(sx);
                tmy.add(sy);
            }
        }
    } else {
        const float w = cc->w;
        const float* S = (P.slopes_in ? P.slopes_in : I.slopes) + cc->w_soff;
        float* Scopy = P.slopes_in ? const_cast<float*>(I.slopes) + cc->w_soff : nullptr;
        for (int e = tid; e < nsr * nsc; e += NT) {
            const int aa = e / nsc, bb = e - aa * nsc;
            const int a = a_lo + aa, b = b_lo + bb;
            if (!FEWHA_IN(a * ns + b, ns2, 1, kDbgSlopes)) continue;
            const bool on = I.mask[cc->w_moff + a * ns + b] != 0;
            const float vx = __ldcg(S + a * ns + b), vy = __ldcg(S + ns2 + a * ns + b);
            if (Scopy) {   // the handle keeps the frame's slopes (tiles may overlap: same values)
                Scopy[a * ns + b] = vx;
                Scopy[ns2 + a * ns + b] = vy;
            }
            const bool fx = isfinite(vx), fy = isfinite(vy);
            if (on && (!fx || !fy) && a >= W.i0 && b >= W.j0) atomicOr(P.errw, kErrInput);
            slx[e] = (on && fx) ? w * vx : 0.f;
            sly[e] = (on && fy) ? w * vy : 0.f;
            if (ttg && on && a >= W.i0 && b >= W.j0) {
                tmx.add(fx ? vx : 0.f);
                tmy.add(fy ? vy : 0.f);
            }
        }
    }
    __syncthreads();
    fmark(P, 23);
    const int ti = W.i1 - W.i0, tj = W.j1 - W.j0;
    float* out = I.psi + cc->w_noff;
    for (int e = tid; e < ti * tj; e += NT) {
        const int ii = e / tj, jj = e - ii * tj;
        const int i = W.i0 + ii, j = W.j0 + jj;
        float acc = 0.f;
        for (int a = i - 1; a <= i; ++a) {
            if (a < 0 || a >= ns) continue;
            for (int b = j - 1; b <= j; ++b) {
                if (b < 0 || b >= ns) continue;
                const int idx = (a - a_lo) * nsc + (b - b_lo);
                const float sx = slx[idx], sy = sly[idx];
                acc += (b == j - 1 ? sx : -sx) + (a == i - 1 ? sy : -sy);
            }
        }
        if (FEWHA_IN(cc->w_noff + i * np1 + j, I.NW, 1, kDbgGtOut)) out[i * np1 + j] = acc / 2;
    }
    if (want_mu) {
        const float4 s = block_reduce2(mu, Acc2(), (float4*)red);
        if (tid == 0) P.wpart[item] = make_float2(s.x, s.y);
    }
    if (ttg) {
        __syncthreads();   // red is reused
        const float4 s = block_reduce2(tmx, tmy, (float4*)red);
        if (tid == 0) P.tpart[item] = s;
    }
    __syncthreads();
    fmark(P, 24);
}

// ---------------------------------------------------------------------------
// distributed DWT on the cluster's row stripes
// ---------------------------------------------------------------------------
struct Stripe {
    int n, J, R, row0, ln, lR;
};

__device__ __forceinline__ void csync(cg::cluster_group& cl, bool multi) {
    if (multi) cl.sync();
    else __syncthreads();
}

// Z (own rows) <- W Z; P buffers alternate by level (remote reads in the
// column passes); one cluster barrier per level whose block spans CTAs.
// Sizes are powers of two: n = 2^ln, R = 2^lR, a level block m = 2^lm.
// Every pass handles up to kB outputs per thread per round and issues all of
// their loads (shared or distributed shared) before any store.
constexpr int kB = 4;

__device__ void fwd_dwt(const FParams& P, const Stripe& s, float* Z, float* P0, float* P1, float* const* rem0,
                        float* const* rem1, cg::cluster_group& cl) {
    const int tid = threadIdx.x, NT = blockDim.x, R = s.R, ln = s.ln, lR = s.lR;
    __syncthreads();
    for (int j = 1; j <= s.J; ++j) {
        const int lm = ln - (j - 1), m = 1 << lm, half = m >> 1, mask = m - 1;
        const bool multi = m > R;
        float* Pj = (j & 1) ? P0 : P1;
        float* const* rem = (j & 1) ? rem0 : rem1;
        const int nrows = max(0, min(m - s.row0, R));
        if (half >= 4) {
            // a thread makes 4 consecutive pairs of one row from 12 inputs
            // (three 16-byte loads; 2 k0 is a multiple of 8, the row of m a
            // multiple of 8 floats, so the wrap keeps them aligned)
            const int cnt4 = nrows << (lm - 3);
            for (int e = tid; e < cnt4; e += NT) {
                const int rr = e >> (lm - 3), k0 = (e & ((half >> 2) - 1)) << 2;
                const float* x = Z + (rr << ln);
                const float4 q0 = *reinterpret_cast<const float4*>(x + ((2 * k0) & mask));
                const float4 q1 = *reinterpret_cast<const float4*>(x + ((2 * k0 + 4) & mask));
                const float4 q2 = *reinterpret_cast<const float4*>(x + ((2 * k0 + 8) & mask));
                const float v[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
                float a[4], d[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = d[q] = 0.f;
#pragma unroll
                    for (int t = 0; t < 6; ++t) {
                        a[q] += P.h[t] * v[2 * q + t];
                        d[q] += P.g[t] * v[2 * q + t];
                    }
                }
                *reinterpret_cast<float4*>(Pj + (rr << ln) + k0) = make_float4(a[0], a[1], a[2], a[3]);
                *reinterpret_cast<float4*>(Pj + (rr << ln) + half + k0) = make_float4(d[0], d[1], d[2], d[3]);
            }
        }
        const int cnt_r = (half >= 4) ? 0 : nrows << (lm - 1);
        for (int e0 = tid; e0 < cnt_r; e0 += kB * NT) {
            float a[kB], d[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int e = e0 + u * NT;
                a[u] = d[u] = 0.f;
                if (e < cnt_r) {
                    const int rr = e >> (lm - 1), k = e & (half - 1);
                    const float* x = Z + (rr << ln);
#pragma unroll
                    for (int t = 0; t < 6; ++t) {
                        const float v = x[(2 * k + t) & mask];
                        a[u] += P.h[t] * v;
                        d[u] += P.g[t] * v;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int e = e0 + u * NT;
                if (e < cnt_r) {
                    const int rr = e >> (lm - 1), k = e & (half - 1);
                    Pj[(rr << ln) + k] = a[u];
                    Pj[(rr << ln) + half + k] = d[u];
                }
            }
        }
        csync(cl, multi);
        // column pass: a thread produces kR consecutive output rows of one
        // column from the 2 kR + 4 input rows they share (groups never
        // straddle the a/d boundary: half and row0 are multiples of kR)
        {
            const int kR = min(4, min(R, half)), lkR = 31 - __clz(kR);
            const int groups = nrows >> lkR, items = groups << lm;
            for (int e = tid; e < items; e += NT) {
                const int x = e & mask, grp = e >> lm;
                const int row = s.row0 + (grp << lkR);
                const bool lo = row < half;
                const int k0 = lo ? row : row - half;
                float f[6];   // h or g, selected per coefficient (no indexing of the parameters)
#pragma unroll
                for (int t = 0; t < 6; ++t) f[t] = lo ? P.h[t] : P.g[t];
                float v[12];
#pragma unroll
                for (int i = 0; i < 12; ++i) {
                    if (i < 2 * kR + 4) {
                        const int src = (2 * k0 + i) & mask;
                        v[i] = FEWHA_IN(src >> lR, P.C, 1, kDbgStripe) ? rem[src >> lR][((src & (R - 1)) << ln) + x] : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (u < kR) {
                        float acc = 0.f;
#pragma unroll
                        for (int t = 0; t < 6; ++t) acc += f[t] * v[2 * u + t];
                        Z[((row - s.row0 + u) << ln) + x] = acc;
                    }
                }
            }
        }
        const bool next_multi = (j < s.J) && (half > R);
        csync(cl, multi && !next_multi);
    }
}

// returns the buffer holding W^T Z (own rows); Z, Q0, Q1 read remotely.
__device__ float* inv_dwt(const FParams& P, const Stripe& s, float* Z, float* Pb, float* Q0, float* Q1,
                          float* const* remZ, float* const* remQ0, float* const* remQ1, cg::cluster_group& cl) {
    const int tid = threadIdx.x, NT = blockDim.x, n = s.n, R = s.R, ln = s.ln, lR = s.lR;
    csync(cl, (n >> (s.J - 1)) > R);
    float* out = Q1;
    for (int j = s.J; j >= 1; --j) {
        const int lm = ln - (j - 1), m = 1 << lm, half = m >> 1, mask = m - 1;
        float* const* remLL = (j == s.J) ? remZ : (((j + 1) & 1) ? remQ1 : remQ0);
        float* Qj = (j & 1) ? Q1 : Q0;
        const int nrows = max(0, min(m - s.row0, R));
        // column pass: output rows i0 .. i0 + kR - 1 (i0 even) of one column
        // need the a and d rows k0 - 2 .. k0 + kR/2 - 1 (k0 = i0 / 2); output
        // i0 + u takes taps t = e + 2 s (e = u & 1) from rows k0 + u/2 - s
        {
            const int kR = min(4, R), lkR = 31 - __clz(kR), hmask = half - 1;
            const int items = (nrows >> lkR) << lm;
            for (int e = tid; e < items; e += NT) {
                const int x = e & mask, i0 = s.row0 + ((e >> lm) << lkR), k0 = i0 >> 1;
                float* const* ra = (x < half) ? remLL : remZ;
                float va[4], vd[4];
#pragma unroll
                for (int mm = 0; mm < 4; ++mm) {
                    if (mm < (kR >> 1) + 2) {
                        const int k = (k0 - 2 + mm) & hmask, kd = half + k;
                        const bool okr = FEWHA_IN(kd >> lR, P.C, 1, kDbgStripe);
                        va[mm] = okr ? ra[k >> lR][((k & (R - 1)) << ln) + x] : 0.f;
                        vd[mm] = okr ? remZ[kd >> lR][((kd & (R - 1)) << ln) + x] : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (u < kR) {
                        const int ee = u & 1;
                        float acc = 0.f;
#pragma unroll
                        for (int sgrp = 0; sgrp < 3; ++sgrp) {
                            const int idx = (u >> 1) - sgrp + 2;
                            acc += P.h[ee + 2 * sgrp] * va[idx] + P.g[ee + 2 * sgrp] * vd[idx];
                        }
                        Pb[((i0 - s.row0 + u) << ln) + x] = acc;
                    }
                }
            }
        }
        __syncthreads();
        // row pass: entries 2kk and 2kk+1 of a row share the a and d entries
        // kk - s (s = 0..2, periodic) with taps 2s and 2s+1; one item makes both
        const int hmask2 = half - 1, cntp = nrows << (lm - 1);
        for (int e0 = tid; e0 < cntp; e0 += kB * NT) {
            float2 o[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int e = e0 + u * NT;
                o[u] = make_float2(0.f, 0.f);
                if (e < cntp) {
                    const float* pr = Pb + ((e >> (lm - 1)) << ln);
                    const int kk = e & hmask2;
#pragma unroll
                    for (int sg = 0; sg < 3; ++sg) {
                        const int k = (kk - sg) & hmask2;
                        const float av = pr[k], dv = pr[half + k];
                        o[u].x += P.h[2 * sg] * av + P.g[2 * sg] * dv;
                        o[u].y += P.h[2 * sg + 1] * av + P.g[2 * sg + 1] * dv;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int e = e0 + u * NT;
                if (e < cntp)
                    *reinterpret_cast<float2*>(Qj + ((e >> (lm - 1)) << ln) + 2 * (e & hmask2)) = o[u];
            }
        }
        out = Qj;
        if (j > 1) csync(cl, (m << 1) > R);
        else __syncthreads();
    }
    return out;
}

// ---------------------------------------------------------------------------
// layer phase
// ---------------------------------------------------------------------------
// P^T gather into the stripe rows: each thread keeps one layer column q and
// walks rows rr0, rr0 + rstep, ...; per sensor the column entries are read
// once for all its rows.  KGT = entries per gather row / column of the tables.
template <int KGT>
__device__ __forceinline__ void pt_gather(const int* sgi, const float* stg, const int2* xt, const int2* yt, float* Z,
                                          int G, int n, int R, int ln) {
    constexpr int kRows = 8;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int qpt = min(n, NT), rstep = NT / qpt;
    for (int qb = 0; qb < n; qb += qpt) {
        const int q = qb + tid % qpt, rr0 = tid / qpt;
        if (rr0 >= rstep) continue;
        for (int rb = rr0; rb < R; rb += rstep * kRows) {
            float acc[kRows];
#pragma unroll
            for (int u = 0; u < kRows; ++u) acc[u] = 0.f;
            for (int g = 0; g < G; ++g) {
                const int imin = sgi[g * 8], imax = sgi[g * 8 + 1];
                if (imax <= imin) continue;
                const int np1 = sgi[g * 8 + 3];
                const float* base = stg + sgi[g * 8 + 2] - imin * np1;
                int xj[KGT];
                float xw[KGT];
#pragma unroll
                for (int b = 0; b < KGT; ++b) {
                    const int2 xe = xt[(g * n + q) * KGT + b];
                    xj[b] = xe.x;
                    xw[b] = __int_as_float(xe.y);
                }
#pragma unroll
                for (int u = 0; u < kRows; ++u) {
                    const int rr = rb + u * rstep;
                    if (rr >= R) break;
                    const int2* yr = yt + (g * R + rr) * KGT;
#pragma unroll
                    for (int a = 0; a < KGT; ++a) {
                        const int2 ye = yr[a];
                        const float* row = base + max(ye.x, imin) * np1;
                        float racc = 0.f;
#pragma unroll
                        for (int b = 0; b < KGT; ++b)
                            if (FEWHA_IN_SMEM(row + xj[b], 4, kDbgPtRead)) racc += xw[b] * row[xj[b]];
                        acc[u] += __int_as_float(ye.y) * racc;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kRows; ++u) {
                const int rr = rb + u * rstep;
                if (rr < R) Z[(rr << ln) + q] = acc[u];
            }
        }
    }
}

// end_sync: the stripes may still be read by the other CTAs of the cluster,
// so a CTA waits for them before its shared memory is reused -- unless a grid
// barrier follows directly (it waits for every CTA).
__device__ void layer_phase(const FParams& P, int li, int mode, int k, float* sm, float* const (*rem)[kMaxC],
                            cg::cluster_group& cl, double* red, double* sh, CtaCache* cc, bool end_sync) {
    const int tid = threadIdx.x, NT = blockDim.x;
    fmark(P, 10);
    const bool fresh = cc->lkey != li;   // else the descriptors are cached
    if (P.shared_tables && tid == 0) cc->wtab = 0;   // this phase overwrites the interpolation tables
    if (fresh) {
        __syncthreads();   // the previous item's tables may still be in use
        if (tid == 0) layer_desc(P, li, cc);
        __syncthreads();
    }
    // staging ranges and gather tables: built at launch start for the first
    // item (next to the first sensor phase), here for any other
    const bool tabs = cc->ltkey != li;
    const FInst& I = cc->IL;
    const int C = P.C, rank = (int)cl.block_rank();
    const int n = cc->n, J = cc->J, off = cc->off;
    const int R = n / C, row0 = rank * R;
    const int G = I.G;
    const int SF = P.stripe_floats;
    const int* sgi = sgi_buf();
    float* Z = sm;
    float* B1 = sm + SF;
    float* B2 = sm + 2 * SF;
    float* B3 = sm + 3 * SF;
    float* stg = sm + 4 * SF;
    int2* xt = (int2*)(sm + P.ltab_off);                // [g][q][KG]  (j, w)
    int2* yt = xt + P.G_max * P.n_max * I.KG;           // [g][row][KG] (i, w)
    const int ln = 31 - __clz(n), lR = 31 - __clz(R), KG = I.KG;
    Stripe s{n, J, R, row0, ln, lR};

    // ---- P^T: gather of the sensor fields into the own rows ----
    {
        if (tabs) {
            layer_tables(P, rank, cc, sm);
            __syncthreads();   // the staging ranges
        }
        for (int g = 0; g < G; ++g) {
            const int c4 = sgi[g * 8 + 5];
            const float* src = I.psi + sgi[g * 8 + 4];
            float* dst = stg + sgi[g * 8 + 6];
            for (int e = tid; e < c4; e += NT)
                if (FEWHA_IN(sgi[g * 8 + 4] + (e << 2), I.NW + 8, 4, kDbgStgSrc))   // 8 floats of padding past NW
                    cp_async16(dst + (e << 2), src + (e << 2));
        }
        // the CG scalars of this iteration, while the copies are in flight
        // (part A from the sensor phase when that CTA computed it there)
        if (mode == kLpIter && tid < 32 && I.preA_cta < 0) {
            ScalA A;
            if (I.preA_cta >= 0) {   // published by the instance's reserved CTA before the grid barrier
                const double* pa = I.preA + (k & 1) * 6;
                A.rho = __ldcg(pa);
                A.beta = __ldcg(pa + 1);
                A.t = __ldcg(pa + 2);
                A.aold = __ldcg(pa + 3);
                A.mh = (float)__ldcg(pa + 4);   // exact: stored from floats
                A.ml = (float)__ldcg(pa + 5);
            } else if (cc->pre_k == k) {
                A.rho = cc->pre[0];
                A.beta = cc->pre[1];
                A.t = cc->pre[2];
                A.aold = cc->pre[3];
                A.mh = (float)cc->pre[4];   // exact: stored from floats
                A.ml = (float)cc->pre[5];
            } else {
                alg2_part_a(P, I, k, A);
            }
            alg2_part_b(P, I, k, A, sh);
        }
        cp_async_wait_all();   // the fields (and gather tables, if just issued)
        if (tabs && tid == 0) cc->ltkey = li;
        __syncthreads();
        fmark(P, 11);
        switch (KG) {   // the gather loops unrolled over the table's real width
            case 1: pt_gather<1>(sgi, stg, xt, yt, Z, G, n, R, ln); break;
            case 2: pt_gather<2>(sgi, stg, xt, yt, Z, G, n, R, ln); break;
            case 3: pt_gather<3>(sgi, stg, xt, yt, Z, G, n, R, ln); break;
            default: pt_gather<4>(sgi, stg, xt, yt, Z, G, n, R, ln); break;
        }
    }

    // ---- forward DWT ----
    // alpha_k, beta_k from the instance's reserved CTA: the first look is
    // issued here and lands while the transform runs
    const bool pub = (mode == kLpIter) && I.preA_cta >= 0;
    unsigned long long wa = 0ull, wa2 = 0ull, wb = 0ull, wb2 = 0ull;
    if (pub && tid == 0) {
        ld_relaxed_v2(I.pubAB + (k & 1) * 4, wa, wa2);
        ld_relaxed_v2(I.pubAB + (k & 1) * 4 + 2, wb, wb2);
    }
    fmark(P, 12);
    fwd_dwt(P, s, Z, B1, B2, rem[1], rem[2], cl);
    fmark(P, 13);

    // ---- elementwise (Alg. 1 restart / Alg. 2 update) ----
    const bool last = (mode == kLpIter) && (k + 1 >= P.n_iter);
    const bool make_z = (mode == kLpRhsStart) || (mode == kLpReplStart) || (mode == kLpIter && !last);
    Acc2 rho_p, dz_p;
    const long gbase = (long)off + (long)row0 * n;
    if (mode == kLpIter) {
        // the state does not depend on the scalars: its first batch is loaded
        // before the scalar reduction so the two latencies overlap
        constexpr int kE = 4;
        const int total = R * n;
        float vr[kE], vp[kE], vq[kE], vc[kE], vj[kE], va[kE];
        auto load = [&](int e0) {
#pragma unroll
            for (int u = 0; u < kE; ++u) {
                const int e = e0 + u * NT;
                if (e < total && FEWHA_IN(gbase + e, I.N, 1, kDbgCoef)) {
                    const long i = gbase + e;
                    vr[u] = I.r[i];
                    vp[u] = I.p[i];
                    vq[u] = I.q[i];
                    vc[u] = I.c[i];
                    vj[u] = __ldg(I.Jinv + i);
                    va[u] = __ldg(I.aD + i);
                }
            }
        };
        // sh[] holds the scalars (computed during the staging above) ...
        load(tid);
        if (pub) {
            // ... or the instance's reserved CTA publishes them (normally long
            // before this point); the wait is bounded by the barrier budget
            if (tid == 0) {
                const unsigned want = (unsigned)k + 1u;
                const long long t0 = clock64();
                bool ok = true;
                while ((unsigned)(wa >> 32) != want || (unsigned)(wa2 >> 32) != want ||
                       (unsigned)(wb >> 32) != want || (unsigned)(wb2 >> 32) != want) {
                    if (clock64() - t0 > P.budget) {
                        ok = false;
                        break;
                    }
                    __nanosleep(32);
                    ld_relaxed_v2(I.pubAB + (k & 1) * 4, wa, wa2);
                    ld_relaxed_v2(I.pubAB + (k & 1) * 4 + 2, wb, wb2);
                }
                sh[0] = ok ? __hiloint2double((int)(unsigned)wa, (int)(unsigned)wa2) : 0.0;
                sh[1] = ok ? __hiloint2double((int)(unsigned)wb, (int)(unsigned)wb2) : 0.0;
                if (!ok) atomicOr(P.errw, kErrTimeout);
            }
            __syncthreads();
        }
        fmark(P, 17);
        const double alpha = sh[0], beta = sh[1];
        if (!pub && tid == 0 && li == I.l0 && rank == 0) {
            double* sw = I.scal + (k & 1) * 2;
            sw[0] = sh[2];
            sw[1] = sh[5];
            if (sh[4] != 0.0) atomicOr(P.errw, kErrBreakdown);
            if (I.sc_out) {
                I.sc_out[kRho] = sh[2];
                I.sc_out[kMu] = sh[3];
                I.sc_out[kBeta] = beta;
                I.sc_out[kAlphaK] = alpha;
            }
        }
        const float fa = (float)alpha, fb = (float)beta;
        for (int e0 = tid; e0 < total; e0 += kE * NT) {
            if (e0 != tid) load(e0);
            {
                // the next batch's lines into the L2 while this one computes
                // (one lane per warp: a warp's 32 elements are one 128-byte line)
                const int en = e0 + kE * NT;
                if ((tid & 31) == 0 && en < total) {
#pragma unroll
                    for (int u = 0; u < kE; ++u) {
                        const int e = en + u * NT;
                        if (e < total) {
                            const long i = gbase + e;
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(I.r + i));
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(I.p + i));
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(I.q + i));
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(I.c + i));
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(I.Jinv + i));
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(I.aD + i));
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kE; ++u) {
                const int e = e0 + u * NT;
                if (e >= total) break;
                const long i = gbase + e;
                if (!FEWHA_IN(i, I.N, 1, kDbgCoef)) continue;
                const float z = vj[u] * vr[u];
                const float sv = Z[e] + va[u] * z;
                const float pv = (k == 0) ? z : z + fb * vp[u];
                const float qv = (k == 0) ? sv : sv + fb * vq[u];
                const float cv = vc[u] + fa * pv;
                const float rv = vr[u] - fa * qv;
                I.p[i] = pv;
                I.q[i] = qv;
                I.c[i] = cv;
                I.r[i] = rv;
                float zout;
                if (!last) {
                    zout = vj[u] * rv;
                    rho_p.add_prod(rv, zout);
                    dz_p.add_prod3(va[u], zout, zout);
                } else {
                    zout = cv;
                }
                Z[e] = zout;
            }
        }
    } else {
        // RHS, its replacement form and the restart: batches of kE elements
        // per thread, every load of a batch issued before its arithmetic
        constexpr int kE = 2;
        const int total = R * n;
        const bool need_ja = mode != kLpRhsRepl;
        const bool need_12 = mode != kLpRhsStart || P.warm;
        for (int e0 = tid; e0 < total; e0 += kE * NT) {
            float vj[kE], va[kE], v1[kE], v2[kE];
#pragma unroll
            for (int u = 0; u < kE; ++u) {
                const int e = e0 + u * NT;
                if (e < total && FEWHA_IN(gbase + e, I.N, 1, kDbgCoef)) {
                    const long i = gbase + e;
                    if (need_ja) {
                        vj[u] = __ldg(I.Jinv + i);
                        va[u] = __ldg(I.aD + i);
                    }
                    if (need_12) {
                        // RhsStart: bprev, r; RhsRepl: c; ReplStart: c, b
                        v1[u] = (mode == kLpRhsStart ? I.bprev : I.c)[i];
                        if (mode != kLpRhsRepl) v2[u] = (mode == kLpRhsStart ? I.r : I.b)[i];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kE; ++u) {
                const int e = e0 + u * NT;
                if (e >= total) break;
                const long i = gbase + e;
                if (!FEWHA_IN(i, I.N, 1, kDbgCoef)) continue;
                float zout = 0.f;
                if (mode == kLpRhsStart) {
                    const float bv = Z[e];
                    float rv;
                    if (!P.warm) {
                        rv = bv;
                        I.c[i] = 0.f;
                    } else {
                        rv = (bv - v1[u]) + v2[u];
                    }
                    I.b[i] = bv;
                    I.bprev[i] = bv;
                    I.r[i] = rv;
                    zout = vj[u] * rv;
                    rho_p.add_prod(rv, zout);
                    dz_p.add_prod3(va[u], zout, zout);
                } else if (mode == kLpRhsRepl) {
                    I.b[i] = Z[e];
                    zout = v1[u];
                } else if (mode == kLpReplStart) {
                    // r = b - M c = W P^T Gamma^T C^{-1} (s - Gamma P W^T c) - alpha D c
                    // (the data part arrives as the transformed slope residual)
                    const float cv = v1[u];
                    const float rv = (float)((double)Z[e] - (double)va[u] * (double)cv);
                    I.bprev[i] = v2[u];
                    I.r[i] = rv;
                    zout = vj[u] * rv;
                    rho_p.add_prod(rv, zout);
                    dz_p.add_prod3(va[u], zout, zout);
                }
                Z[e] = zout;
            }
        }
    }
    if (mode == kLpIter) fmark(P, 18);
    if (make_z) {
        const int par = (mode == kLpIter) ? ((k + 1) & 1) : 0;
        const float4 rd = block_reduce2(rho_p, dz_p, (float4*)red);
        if (tid == 0) P.lpart[(size_t)par * P.n_litems * C + (size_t)li * C + rank] = rd;
    }

    // ---- inverse DWT -> phi ----
    fmark(P, 14);
    const bool need_phi = make_z || mode == kLpRhsRepl || (last && P.out_layers);
    if (need_phi) {
        float* res = inv_dwt(P, s, Z, B3, B1, B2, rem[0], rem[1], rem[2], cl);
        fmark(P, 15);
        for (int e = tid; e < R * n; e += NT)
            if (FEWHA_IN(gbase + e, I.N, 1, kDbgPhiOut)) I.phi[gbase + e] = res[e];
        if (last && P.phi_out)
            for (int e = tid; e < R * n; e += NT)
                if (FEWHA_IN(gbase + e, I.N, 1, kDbgPhiOut)) P.phi_out[gbase + e] = res[e];
    }
    if (end_sync) cl.sync();
    fmark(P, 16);
}

#include "fused_cascade.cuh"

// ---------------------------------------------------------------------------
// L2 prefetch of the launch's static data and state
// ---------------------------------------------------------------------------
// With the L2 cold (other work between two frames) the first phases wait on
// DRAM for descriptors, tables and the CG state, one dependent round trip
// after another.  The plan lists every such array in chunks of at most 4 KB,
// dealt out to the CTAs; one warp of each CTA loads its chunk descriptors in a
// single round (one per lane) and requests their lines, so the transfers
// overlap the RHS phase instead of sitting on its critical path.
__device__ void prefetch_plan_data(const FParams& P) {
    const int lane = threadIdx.x & 31;
    const PfChunk* mine = P.pf + (size_t)blockIdx.x * P.pf_per_cta;
    for (int c0 = 0; c0 < P.pf_per_cta; c0 += 32) {
        PfChunk ch{nullptr, 0, 0};
        if (c0 + lane < P.pf_per_cta) ch = mine[c0 + lane];
        const int cnt = min(32, P.pf_per_cta - c0);
        for (int j = 0; j < cnt; ++j) {
            const char* p = (const char*)__shfl_sync(0xffffffffu, (unsigned long long)ch.p, j);
            const int bytes = __shfl_sync(0xffffffffu, ch.bytes, j);
            if ((lane << 7) < bytes) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + (lane << 7)));
        }
    }
}

// ---------------------------------------------------------------------------
// the frame kernel
// ---------------------------------------------------------------------------
// The cluster shape is compiled into each instance (one per cluster size), so
// it belongs to the kernel and not to the launch configuration.  V selects the
// layer phase: 0 row stripes (one cluster barrier per DWT level), 1 the
// level-stacked form (one exchange per transform, fused_cascade.cuh).
template <int CS, int V>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kFThreads, 1)
    k_fused_frame(const __grid_constant__ FParams P) {
    extern __shared__ __align__(16) float sm[];
    __shared__ float* rem[4][kMaxC];
    __shared__ __align__(16) double red[64];   // 32 float4 for the block reductions
    __shared__ double sh[8];
    __shared__ CtaCache cc;
    __shared__ int s_abort;
    __shared__ int s_go;
    cg::cluster_group cl = cg::this_cluster();
    const int C = P.C;
    // every shared-memory address below assumes the planned cluster shape
    if ((int)cl.num_blocks() != C || (int)gridDim.x != P.grid || (gridDim.x % C) != 0) {
        if (threadIdx.x == 0) atomicOr(P.errw, kErrLaunch);
        return;
    }
    const int cid = blockIdx.x / C;
    const int w_lo = P.wsched_off[blockIdx.x], w_hi = P.wsched_off[blockIdx.x + 1];
    const int l_lo = P.lsched_off[cid], l_hi = P.lsched_off[cid + 1];
    int slot = 0;
    if (threadIdx.x == 0) trace_mark(P, 0, 0);   // slot 0: start, and (below) set-up done / go seen
    ++slot;
    if (threadIdx.x < 4 * C) {
        const int b = threadIdx.x / C, r = threadIdx.x % C;
        if (V == 0) rem[b][r] = cl.map_shared_rank(sm + b * P.stripe_floats, r);
        else if (b < 2) rem[b][r] = cl.map_shared_rank(sm + (b == 0 ? P.v_r : P.v_u), r);   // Urow, Ucol
    }
    if (threadIdx.x == 0) {
        s_abort = 0;
        *fmark_counter() = 0;
        cc.wkey = cc.lkey = cc.ltkey = cc.ltx = -1;
        cc.wtab = 0;
        cc.lres = (l_hi - l_lo == 1) ? 1 : 0;
        cc.il_valid = 0;
        cc.pre_k = -1;
    }
    unsigned target = 0;
    const int res_inst = P.duty ? P.duty[blockIdx.x]
                                : ((int)blockIdx.x >= P.res_first && (int)blockIdx.x < P.res_first + P.n_res)
                                      ? (int)blockIdx.x - P.res_first : -1;
    // the published alpha / beta words restart at tag 0 with every launch
    // (read only after the first grid barrier)
    if (res_inst >= 0 && threadIdx.x < 8) P.inst[res_inst].pubAB[threadIdx.x] = 0ull;
    __syncthreads();
    if (P.pf && (int)threadIdx.x >= (int)blockDim.x - 32) prefetch_plan_data(P);   // the last warp
    // Descriptors of the CTA's first sensor and layer items, fetched side by
    // side (two dependent chains at once, not one at the top of each phase),
    // then the first layer item's staging ranges and gather tables, whose
    // copies land while the first sensor phase runs (separate shared memory)
    if (!P.shared_tables) {
        if (threadIdx.x == 0 && w_lo < w_hi) sensor_desc(P, P.wsched[w_lo], &cc);
        if (threadIdx.x == 32 && l_lo < l_hi) layer_desc(P, P.lsched[l_lo], &cc);
        __syncthreads();
        if (l_lo < l_hi) {
            if (V == 0) layer_tables(P, (int)cl.block_rank(), &cc, sm);
            else layer_tables_v1(P, (int)cl.block_rank(), &cc, sm);
            if (threadIdx.x == 0) cc.ltkey = cc.lkey;
        }
        __syncthreads();
    }

    // One loop over the phases of the frame, each phase function called from
    // a single site (one copy of its code, warm in the instruction caches and
    // the L2 from the first phase of its kind on).  Phases, a grid barrier
    // after every one but the last:
    //   0: Alg. 1 RHS, Gamma^T C^{-1} s per sensor tile
    //   1: P^T, W -> b; warm restart (or c -> phi for the replacement); z_0 -> phi
    //   [2, 3: replacement r = b - M c: the weighted slope residual
    //    Gamma^T C^{-1} (s - Gamma P phi_c), then the layer phase
    //    r = W P^T (...) - alpha D c]
    //   then per Alg. 2 iteration k: the data term (sensor tiles; the reserved
    //   CTA computes part A of the scalars), then the layer phase (the reserved
    //   CTA first publishes part B)
    const int base = P.replace ? 4 : 2, nph = base + 2 * P.n_iter;
    // an armed frame waits here for the host's go (its set-up above -- the L2
    // prefetch, descriptors, first tables -- done meanwhile); without it by the
    // deadline every phase is skipped and the frame reports TIMEOUT
    int nph_run = nph;
    if (P.doorbell) {
        // CTA 0 alone polls the host word (a read across the host link each
        // time) and passes the go on through a device word the others poll in
        // the L2: with every CTA polling the host the last ones saw the go
        // ~130 us after the first
        if (threadIdx.x == 0) {
            const unsigned long long t0 = global_ns();
            const unsigned* src = blockIdx.x == 0 ? P.doorbell : P.bar + 2;
            int go = 1;
            while ((blockIdx.x == 0 ? ld_acquire_sys(src) : ld_acquire_gpu(src)) != P.doorbell_want) {
                if ((long long)(global_ns() - t0) > P.doorbell_ns) {
                    go = 0;
                    break;
                }
                __nanosleep(64);
            }
            if (go && blockIdx.x == 0)
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(P.bar + 2), "r"(P.doorbell_want) : "memory");
            s_go = go;
            if (!go) atomicOr(P.errw, kErrTimeout);
        }
        __syncthreads();
        if (!s_go) nph_run = 0;
    }
    if (threadIdx.x == 0) trace_mark(P, 0, 1);
    for (int ph = 0; ph < nph_run; ++ph) {
        const bool it = ph >= base;
        const int k = it ? (ph - base) >> 1 : 0;
        const bool sensor_ph = it ? ((ph - base) & 1) == 0 : (ph & 1) == 0;
        if (sensor_ph) {
            const int smode = (ph == 0) ? kModeRhs : (!it && ph == 2) ? kModeResid : kModeData;
            for (int t = w_lo; t < w_hi; ++t) sensor_tile(P, P.wsched[t], sm, smode, it, red, &cc, k);
            if (it && res_inst >= 0 && threadIdx.x < 32) {
                // part A of instance res_inst's scalars for this iteration's layer phase
                const FInst& RI = P.inst[res_inst];
                ScalA A;
                alg2_part_a(P, RI, k, A);
                if (threadIdx.x == 0) {
                    double* pa = RI.preA + (k & 1) * 6;
                    pa[0] = A.rho;
                    pa[1] = A.beta;
                    pa[2] = A.t;
                    pa[3] = A.aold;
                    pa[4] = (double)A.mh;
                    pa[5] = (double)A.ml;
                }
            }
        } else {
            if (it && res_inst >= 0 && threadIdx.x < 32) {
                // part B of the reserved instance's scalars: publish, then flag
                const FInst& RI = P.inst[res_inst];
                const double* pa = RI.preA + (k & 1) * 6;
                ScalA A;
                A.rho = __ldcg(pa);
                A.beta = __ldcg(pa + 1);
                A.t = __ldcg(pa + 2);
                A.aold = __ldcg(pa + 3);
                A.mh = (float)__ldcg(pa + 4);
                A.ml = (float)__ldcg(pa + 5);
                alg2_part_b(P, RI, k, A, sh);
                __syncwarp();
                if (threadIdx.x == 0) {
                    // alpha_k, beta_k (FP64) for the layer CTAs first (tagged words) ...
                    const unsigned long long tag = (unsigned long long)(k + 1) << 32;
                    st_relaxed_v2(RI.pubAB + (k & 1) * 4, tag | (unsigned)__double2hiint(sh[0]),
                                  tag | (unsigned)__double2loint(sh[0]));
                    st_relaxed_v2(RI.pubAB + (k & 1) * 4 + 2, tag | (unsigned)__double2hiint(sh[1]),
                                  tag | (unsigned)__double2loint(sh[1]));
                    // ... then the instance's outputs (rho_k and the last
                    // nonzero alpha feed part A of the next iteration here)
                    double* sw = RI.scal + (k & 1) * 2;
                    sw[0] = sh[2];
                    sw[1] = sh[5];
                    if (sh[4] != 0.0) atomicOr(P.errw, kErrBreakdown);
                    if (RI.sc_out) {
                        RI.sc_out[kRho] = sh[2];
                        RI.sc_out[kMu] = sh[3];
                        RI.sc_out[kBeta] = sh[1];
                        RI.sc_out[kAlphaK] = sh[0];
                    }
                }
            }
            const int lmode = it ? kLpIter : (ph == 1 ? (P.replace ? kLpRhsRepl : kLpRhsStart) : kLpReplStart);
            const bool last_ph = it && k + 1 == P.n_iter;
            for (int t = l_lo; t < l_hi; ++t)
                if (V == 0) layer_phase(P, P.lsched[t], lmode, k, sm, rem, cl, red, sh, &cc, t + 1 < l_hi || last_ph);
                else layer_phase_v1(P, P.lsched[t], lmode, k, sm, rem, cl, red, sh, &cc, false);
        }
        if (ph + 1 < nph_run) grid_barrier(P, target, &s_abort, slot);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        trace_mark(P, slot, 0);
        trace_mark(P, slot, 1);
        // every CTA has passed its last barrier read: the last one out resets
        // the counters for the next launch on this stream
        if (P.done_host) __threadfence_system();   // this CTA's results, host-mapped ones too
        else __threadfence();
        if (atomicAdd(P.bar + 1, 1u) == gridDim.x - 1u) {
            P.bar[0] = 0u;
            P.bar[1] = 0u;
            if (P.done_host) {
                __threadfence_system();
                const unsigned e = (unsigned)atomicOr(P.errw, 0);
                *(volatile unsigned long long*)P.done_host = (1ull << 32) | e;
            } else {
                __threadfence();
            }
        }
    }
}

using FusedKernel = void (*)(FParams);

FusedKernel fused_kernel_for(int C, int V) {
    if (V == 1) {
        switch (C) {
            case 1: return k_fused_frame<1, 1>;
            case 2: return k_fused_frame<2, 1>;
            case 4: return k_fused_frame<4, 1>;
            case 8: return k_fused_frame<8, 1>;
            case 16: return k_fused_frame<16, 1>;
            default: return nullptr;
        }
    }
    switch (C) {
        case 1: return k_fused_frame<1, 0>;
        case 2: return k_fused_frame<2, 0>;
        case 4: return k_fused_frame<4, 0>;
        case 8: return k_fused_frame<8, 0>;
        case 16: return k_fused_frame<16, 0>;
        default: return nullptr;
    }
}

// ---------------------------------------------------------------------------
// host plan
// ---------------------------------------------------------------------------
struct FusedPlan {
    int C = 1, V = 0, nclusters = 0, grid = 0, smem = 0;
    bool cooperative = true;
    bool trace_on = false;
    unsigned long long* ftrace = nullptr;
    unsigned long long* trace = nullptr;
    int trace_slots = 0;
    int last_slots = 0;
    FParams P{};
    std::vector<void*> allocs;
    FInst* d_inst = nullptr;
    std::vector<FInst> inst;
    float* psi = nullptr;
    bool bar_dirty = true;   // the barrier counters must be zeroed before the next launch
};

namespace {

template <typename U>
bool dalloc(FusedPlan* pl, U*& p, size_t n, std::string& err) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(n, 1) * sizeof(U));
    if (e != cudaSuccess) {
        err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return false;
    }
    pl->allocs.push_back(v);
    p = (U*)v;
    return true;
}

template <typename U>
bool dupload(FusedPlan* pl, U*& p, const std::vector<U>& v, std::string& err) {
    if (!dalloc(pl, p, v.size(), err)) return false;
    if (v.empty()) return true;
    cudaError_t e = cudaMemcpy(p, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        err = std::string("cudaMemcpy: ") + cudaGetErrorString(e);
        return false;
    }
    return true;
}

// tiles of the (ns+1)^2 node grid: ty x tx tiles of near-equal size
void make_tiles(int inst, int g, int np1, int nty, int ntx, std::vector<WItem>& out) {
    for (int a = 0; a < nty; ++a)
        for (int b = 0; b < ntx; ++b) {
            WItem w;
            w.inst = inst;
            w.g = g;
            w.i0 = (int)((long)np1 * a / nty);
            w.i1 = (int)((long)np1 * (a + 1) / nty);
            w.j0 = (int)((long)np1 * b / ntx);
            w.j1 = (int)((long)np1 * (b + 1) / ntx);
            if (w.i1 > w.i0 && w.j1 > w.j0) out.push_back(w);
        }
}

}  // namespace

namespace {

// Per-instance host tables of the fused path: compact P^T gather tables.
struct InstPrep {
    int KG = 1, nmin = 1 << 30, nmax = 0;
    std::vector<int2> gtab;
    std::vector<int> gtab_off;
};

// For layer column q the sensor columns j with cell_j in {q-1, q} and their
// bilinear weights (1 - t if cell_j == q, t if cell_j == q-1), padded to KG
// entries (weight 0, index 0 for columns / -1 for rows); the same for rows.
bool prep_instance(const HostSetup& hs, InstPrep& ip, std::string& err) {
    if (hs.L > kMaxLayersFused || hs.G > kMaxWfsFused) {
        err = "too many layers or sensors for the fused path";
        return false;
    }
    for (auto& L : hs.lay) {
        ip.nmin = std::min(ip.nmin, L.n);
        ip.nmax = std::max(ip.nmax, L.n);
    }
    for (int g = 0; g < hs.G; ++g)
        for (int l = 0; l < hs.L; ++l) {
            const int gb = hs.gat_off[g * hs.L + l];
            for (int q = 0; q < hs.lay[l].n; ++q) {
                ip.KG = std::max(ip.KG, hs.jhi[gb + q] - hs.jlo[gb + q]);
                ip.KG = std::max(ip.KG, hs.ihi[gb + q] - hs.ilo[gb + q]);
            }
        }
    if (ip.KG > kMaxKG) {
        err = "sensor grid much finer than the layer grid (more than 4 sensor nodes per layer cell pair)";
        return false;
    }
    auto fbits = [](float f) {
        int i;
        std::memcpy(&i, &f, sizeof i);
        return i;
    };
    ip.gtab_off.assign((size_t)hs.G * hs.L, 0);
    for (int g = 0; g < hs.G; ++g)
        for (int l = 0; l < hs.L; ++l) {
            const int n = hs.lay[l].n, base = hs.tab_off[g * hs.L + l], gb = hs.gat_off[g * hs.L + l];
            ip.gtab_off[g * hs.L + l] = (int)ip.gtab.size();
            for (int axis = 0; axis < 2; ++axis) {
                const int* lo = axis ? hs.ilo.data() : hs.jlo.data();
                const int* hi = axis ? hs.ihi.data() : hs.jhi.data();
                const int* cell = axis ? hs.cy.data() : hs.cx.data();
                const double* t = axis ? hs.ty.data() : hs.tx.data();
                for (int q = 0; q < n; ++q) {
                    int cnt = 0;
                    for (int k = lo[gb + q]; k < hi[gb + q]; ++k, ++cnt) {
                        const float w = cell[base + k] == q ? (float)(1.0 - t[base + k]) : (float)t[base + k];
                        ip.gtab.push_back(make_int2(k, fbits(w)));
                    }
                    for (; cnt < ip.KG; ++cnt) ip.gtab.push_back(make_int2(axis ? -1 : 0, fbits(0.f)));
                }
            }
        }
    return true;
}

}  // namespace

// Longest-processing-time-first assignment: items in decreasing cost, each
// to the least-loaded worker so far (ties: lowest worker index).  With equal
// costs and no more items than workers this is the plain round-robin.
static void lpt_schedule(const std::vector<double>& cost, int workers, std::vector<int>& order,
                         std::vector<int>& off) {
    std::vector<int> idx(cost.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(workers, 0.0);
    std::vector<std::vector<int>> lists(workers);
    for (int it : idx) {
        int w = 0;
        for (int k = 1; k < workers; ++k)
            if (load[k] < load[w]) w = k;
        load[w] += cost[it];
        lists[w].push_back(it);
    }
    order.clear();
    off.assign(1, 0);
    for (auto& l : lists) {
        order.insert(order.end(), l.begin(), l.end());
        off.push_back((int)order.size());
    }
}

// Ownership tables of the level-stacked layer phase for layers of side n with
// J levels on clusters of C CTAs (layout in fused_cascade.cuh), appended to
// blob; returns the block's offset.  The T_U = 2n(1 - 2^-J) rows of the
// stacked column transform are dealt to the CTAs longest-processing-time
// first, a row costing n/2 (its share of the exchange and the cascade) plus
// twice its coefficients (the elementwise update); a CTA's rows are ordered
// by depth, deepest first, so the rows active at a level form a prefix.
struct CascStats { int smax = 0, ncoef_max = 0, tu_max = 0; };

static int build_casc_shape(int n, int J, int C, std::vector<int>& blob, CascStats& st) {
    struct Row { int u, j, isA, goff, ncoef; double cost; };
    std::vector<Row> rows;
    int base = 0;
    for (int j = 1; j <= J; ++j) {
        const int half = n >> j;
        for (int k = 0; k < half; ++k) {   // Lo_j rows: Hi_j (j < J), Lo_J and Hi_J (j = J)
            const bool A = j < J;
            rows.push_back(Row{base + k, j, A ? 1 : 0, k * n + (A ? half : 0), A ? half : 2 * half, 0.0});
        }
        for (int k = 0; k < half; ++k)     // Hi_j rows: Lo_j and Hi_j, Mallat row half + k
            rows.push_back(Row{base + half + k, j, 0, (half + k) * n, 2 * half, 0.0});
        base += 2 * half;
    }
    const int TU = base;
    std::vector<double> cost;
    for (auto& r : rows) cost.push_back(0.5 * n + 2.0 * r.ncoef);
    std::vector<int> order, off;
    lpt_schedule(cost, C, order, off);
    const int hdr = (5 + C + 3) & ~3;
    const int start = (int)blob.size();
    blob.resize(start + hdr, 0);
    blob[start + 0] = TU;
    blob[start + 1] = J;
    blob[start + 2] = n;
    blob[start + 3] = C;
    std::vector<int> own(TU, 0);
    for (int r = 0; r < C; ++r) {
        std::vector<Row> mine;
        for (int i = off[r]; i < off[r + 1]; ++i) mine.push_back(rows[order[i]]);
        std::sort(mine.begin(), mine.end(), [](const Row& a, const Row& b) { return a.j != b.j ? a.j > b.j : a.u < b.u; });
        const int rb = (int)blob.size();
        blob[start + 4 + r] = rb - start;
        blob.resize(rb + 20 + 4 * mine.size(), 0);
        int zoff = 0;
        std::vector<int> gidx;   // Mallat offset in the layer of every owned coefficient
        for (size_t s = 0; s < mine.size(); ++s) {
            const Row& w = mine[s];
            int* e = &blob[rb + 20 + 4 * s];
            e[0] = w.u;
            e[1] = w.j | (w.isA << 8);
            e[2] = w.goff;
            e[3] = zoff;
            own[w.u] = (r << 16) | (int)s;
            zoff += w.ncoef;
            for (int x = 0; x < w.ncoef; ++x) gidx.push_back(w.goff + x);
        }
        blob.insert(blob.end(), gidx.begin(), gidx.end());
        blob.resize((blob.size() + 3) & ~(size_t)3, 0);
        blob[rb + 0] = (int)mine.size();
        blob[rb + 1] = zoff;
        blob[rb + 2] = TU;
        blob[rb + 3] = J;
        for (int i = 1; i <= 16; ++i) {
            int c = 0;
            for (auto& w : mine) c += w.j >= i;
            blob[rb + 4 + i - 1] = c;
        }
        st.smax = std::max(st.smax, (int)mine.size());
        st.ncoef_max = std::max(st.ncoef_max, zoff);
    }
    blob[start + 4 + C] = (int)blob.size() - start;
    blob.insert(blob.end(), own.begin(), own.end());
    blob.resize((blob.size() + 3) & ~(size_t)3, 0);
    st.tu_max = std::max(st.tu_max, TU);
    return start;
}

FusedPlan* fused_create_multi(const std::vector<const HostSetup*>& hss, const std::vector<DevGeo<float>>& Gs,
                              const std::vector<FusedBuffers>& fbs, int max_tile_side, std::string& err,
                              int forced_C, int forced_V) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        err = "no device";
        return nullptr;
    }
    if (prop.major < 9) {
        err = "the fused path needs thread-block clusters (sm_90 or newer)";
        return nullptr;
    }
    const int ninst = (int)hss.size();
    if (ninst < 1 || (int)Gs.size() != ninst || (int)fbs.size() != ninst) {
        err = "no instances";
        return nullptr;
    }
    std::vector<InstPrep> preps(ninst);
    int nmin = 1 << 30, nmax = 0, KGmax = 1, Gmax = 0, Lmax = 0, Gtot = 0;
    for (int i = 0; i < ninst; ++i) {
        if (!prep_instance(*hss[i], preps[i], err)) return nullptr;
        nmin = std::min(nmin, preps[i].nmin);
        nmax = std::max(nmax, preps[i].nmax);
        KGmax = std::max(KGmax, preps[i].KG);
        Gmax = std::max(Gmax, hss[i]->G);
        Lmax = std::max(Lmax, hss[i]->L);
        Gtot += hss[i]->G;
    }
    const int sms = prop.multiProcessorCount;
    // dynamic shared memory available next to the kernel's static arrays
    size_t smem_cap = 0;
    {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fused_kernel_for(8, 0)) != cudaSuccess ||
            fa.sharedSizeBytes + 1024 >= (size_t)prop.sharedMemPerBlockOptin) {
            cudaGetLastError();
            err = "cannot query the fused kernel";
            return nullptr;
        }
        smem_cap = (size_t)prop.sharedMemPerBlockOptin - fa.sharedSizeBytes - 1024;
    }

    // cluster shape: clusters of 8 unless they leave layer items for a second
    // round of the layer phase and a smaller shape runs every item at once
    // (e.g. 35 layers: 15 clusters of 8 on this part, 37 of 4)
    std::vector<int> order = {8, 4, 16, 2, 1};
    if (forced_C == 0) {
        int items = 0;
        for (const HostSetup* h : hss) items += h->L;
        auto clusters_for = [&](int C) {
            const FusedKernel k = fused_kernel_for(C, 0);
            if (!k || 2 * C > nmin || (size_t)nmax * nmax / C * 4 * sizeof(float) > smem_cap) return 0;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3(C * 1024);
            q.blockDim = dim3(kFThreads);
            q.dynamicSmemBytes = std::min(smem_cap, (size_t)nmax * nmax / C * 4 * sizeof(float));
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k, &q) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            return std::min(n, sms / C);
        };
        if (items > clusters_for(8))
            for (int C : {4, 2})
                if (items <= clusters_for(C)) {
                    order.erase(std::find(order.begin(), order.end(), C));
                    order.insert(order.begin(), C);
                    break;
                }
    }
    // candidates: every cluster shape in order of preference, the level-stacked
    // layer phase (V = 1) before the row stripes (V = 0) for each
    std::vector<std::pair<int, int>> cand;
    for (int C : order)
        for (int V : {1, 0}) cand.push_back({C, V});
    FusedPlan* best = nullptr;
    for (auto [C, V] : cand) {
        if (forced_C > 0 && C != forced_C) continue;
        if (forced_V >= 0 && V != forced_V) continue;
        bool any_tt = false;
        for (const HostSetup* h : hss) any_tt = any_tt || h->any_tt;
        if (V == 0 && any_tt) {
            if (err.empty()) err = "the row-stripe layer phase does not model the LGS tip-tilt filter";
            continue;
        }
        if (V == 0) {
            if (2 * C > nmin) continue;   // stripes of at least 2 rows
            if ((size_t)nmax * nmax / C * 4 * sizeof(float) > smem_cap) continue;
        } else if (C > nmin || nmax / C > kFThreads) {
            continue;                     // column stripes of 1 .. 512 columns
        }
        auto* pl = new FusedPlan();
        pl->C = C;
        pl->V = V;
        // layer items (instance, layer) with the staged sensor rows (V = 0) or
        // boxes (V = 1) per rank, and for V = 1 the ownership tables per shape
        std::vector<LItem> litems;
        std::vector<int2> stg;
        std::vector<int4> stg4;
        std::vector<int> cshape;
        CascStats cst;
        std::vector<std::pair<std::pair<int, int>, int>> shape_off;
        std::vector<int> l0(ninst), nl(ninst);
        int stage_max = 0;
        for (int i = 0; i < ninst; ++i) {
            const HostSetup& hs = *hss[i];
            l0[i] = (int)litems.size();
            for (int l = 0; l < hs.L; ++l) {
                const int n = hs.lay[l].n, R = n / C;
                LItem li{i, l, V == 0 ? (int)stg.size() : (int)stg4.size(), 0};
                if (V == 1) {
                    const std::pair<int, int> key{n, hs.lay[l].J};
                    int o = -1;
                    for (auto& so : shape_off)
                        if (so.first == key) o = so.second;
                    if (o < 0) {
                        o = build_casc_shape(n, hs.lay[l].J, C, cshape, cst);
                        shape_off.push_back({key, o});
                    }
                    li.csh = o;
                }
                for (int rank = 0; rank < C; ++rank) {
                    int tot = 0;
                    for (int g = 0; g < hs.G; ++g) {
                        const int gb = hs.gat_off[g * hs.L + l];
                        if (V == 0) {
                            int lo = 1 << 30, hi = 0;
                            for (int p = rank * R; p < (rank + 1) * R; ++p) {
                                if (hs.ihi[gb + p] > hs.ilo[gb + p]) {
                                    lo = std::min(lo, hs.ilo[gb + p]);
                                    hi = std::max(hi, hs.ihi[gb + p]);
                                }
                            }
                            if (lo >= hi) lo = hi = 0;
                            stg.push_back(make_int2(lo, hi));
                            tot += (hi - lo) * (hs.wfs[g].n + 1) + 8;   // + 16-byte alignment slack
                        } else {
                            // every sensor row any layer row gathers from, the sensor
                            // columns of this rank's layer columns
                            int ilo = 1 << 30, ihi = 0, jlo = 1 << 30, jhi = 0;
                            for (int p = 0; p < n; ++p)
                                if (hs.ihi[gb + p] > hs.ilo[gb + p]) {
                                    ilo = std::min(ilo, hs.ilo[gb + p]);
                                    ihi = std::max(ihi, hs.ihi[gb + p]);
                                }
                            for (int q = rank * R; q < (rank + 1) * R; ++q)
                                if (hs.jhi[gb + q] > hs.jlo[gb + q]) {
                                    jlo = std::min(jlo, hs.jlo[gb + q]);
                                    jhi = std::max(jhi, hs.jhi[gb + q]);
                                }
                            if (ilo >= ihi || jlo >= jhi) ilo = ihi = jlo = jhi = 0;
                            stg4.push_back(make_int4(ilo, ihi, jlo, jhi));
                            const int W = (ihi > ilo && jhi > jlo) ? ((jhi - jlo + 6) & ~3) : 0;   // as the kernel
                            tot += (ihi - ilo) * W;
                        }
                    }
                    stage_max = std::max(stage_max, tot);
                }
                litems.push_back(li);
            }
            nl[i] = (int)litems.size() - l0[i];
        }
        const int stripe = nmax * nmax / C;
        const int Rmax = nmax / C;
        stage_max = (stage_max + 3) & ~3;
        auto r4 = [](size_t x) { return (x + 3) & ~(size_t)3; };
        size_t gtab_floats, layer_floats;
        size_t vz = 0, vt = 0, vu = 0, vr = 0, vc = 0;
        if (V == 0) {
            gtab_floats = 2 * (size_t)Gmax * nmax * KGmax + 2 * (size_t)Gmax * Rmax * KGmax;
            layer_floats = 4 * (size_t)stripe + stage_max;   // working set (gather tables apart)
        } else {
            // Z | T | Ucol (staged fields alias it) | Urow | Zc; tables: xt, yt, cascade tables
            vt = r4((size_t)nmax * Rmax);
            vu = vt + r4(std::max((size_t)cst.smax * (nmax / 2), (size_t)(nmax / 2) * Rmax));
            vr = vu + r4(std::max({(size_t)cst.tu_max * Rmax, (size_t)stage_max, (size_t)nmax * Rmax}));
            vc = vr + r4((size_t)cst.smax * nmax);
            layer_floats = vc + r4((size_t)cst.ncoef_max);
            gtab_floats = 2 * (size_t)Gmax * (Rmax + nmax) * KGmax +
                          r4(20 + 4 * (size_t)cst.smax + r4(cst.tu_max) + cst.ncoef_max);
        }

        // co-resident clusters: one 512-thread CTA per SM (register-limited),
        // so the answer does not depend on the shared memory below the cap;
        // the attribute is per function: allow the device maximum once
        const FusedKernel kern = fused_kernel_for(C, V);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap) != cudaSuccess ||
            (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
            cudaGetLastError();
            if (err.empty()) err = "the fused kernel's launch attributes were refused";
            delete pl;
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C * 1024);
        cfg.blockDim = dim3(kFThreads);
        cfg.dynamicSmemBytes = std::min(smem_cap, layer_floats * sizeof(float));
        cfg.numAttrs = 0;   // the cluster shape is compiled into the instance
        int ncl = 0;
        cudaError_t oe = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
        if (oe != cudaSuccess || ncl < 1) {
            cudaGetLastError();
            delete pl;
            continue;
        }
        pl->nclusters = std::max(1, std::min(ncl, std::max(1, sms / C)));
        pl->grid = pl->nclusters * C;

        // sensor tiles: near-square, about one round over the grid, and with
        // max_tile_side > 0 no side longer than that
        std::vector<WItem> witems;
        std::vector<int> w0(ninst), nw(ninst);
        std::vector<std::vector<int2>> tt_tiles(ninst);   // per instance, per sensor: its tiles
        // a few instances: the last CTAs of the grid compute part A of the CG
        // scalars (one per instance) instead of a sensor tile
        const int n_res = (ninst <= 4 && ninst * 8 <= pl->grid) ? ninst : 0;
        const int tile_ctas = pl->grid - n_res;
        // more instances: each gets a duty CTA among the working ones (one
        // instance per CTA, spread over the grid), so that its layer items
        // find the scalars published instead of each computing them again
        const bool use_duty = n_res == 0 && ninst > 1 && ninst <= pl->grid;
        auto duty_cta = [&](int i) { return (int)(((long)i * pl->grid) / ninst); };
        std::vector<int> duty;
        if (use_duty) {
            duty.assign(pl->grid, -1);
            for (int i = 0; i < ninst; ++i) duty[duty_cta(i)] = i;
        }
        const int per = std::max(1, tile_ctas / std::max(1, Gtot));
        for (int i = 0; i < ninst; ++i) {
            const HostSetup& hs = *hss[i];
            w0[i] = (int)witems.size();
            for (int g = 0; g < hs.G; ++g) {
                const int np1 = hs.wfs[g].n + 1;
                const int tmin = max_tile_side > 0 ? (np1 + max_tile_side - 1) / max_tile_side : 1;
                const int budget = std::max(per, tmin * tmin);
                int best_ty = tmin, best_tx = tmin;
                double best_cost = 1e30;
                for (int ty = tmin; ty <= std::min(budget, np1); ++ty)
                    for (int tx = tmin; tx <= std::min(budget / ty, np1); ++tx) {
                        const double h = std::ceil((double)np1 / ty) + 2, w = std::ceil((double)np1 / tx) + 2;
                        const double cost = h * w + 0.5 * (h + w);
                        if (cost < best_cost) {
                            best_cost = cost;
                            best_ty = ty;
                            best_tx = tx;
                        }
                    }
                const int t0 = (int)witems.size();
                make_tiles(i, g, np1, best_ty, best_tx, witems);
                tt_tiles[i].push_back(make_int2(t0, (int)witems.size() - t0));
            }
            nw[i] = (int)witems.size() - w0[i];
        }
        // a sensor tile's working set: its nodes' psi and its subapertures'
        // weighted slopes (P reads the layers in the L2 directly)
        int tile_nodes = 0, tile_sub = 0, tile_rows = 0, tile_cols = 0;
        for (auto& w : witems) {
            const int ns = hss[w.inst]->wfs[w.g].n;
            const int a_lo = std::max(w.i0 - 1, 0), a_hi = std::min(w.i1, ns);
            const int b_lo = std::max(w.j0 - 1, 0), b_hi = std::min(w.j1, ns);
            tile_rows = std::max(tile_rows, a_hi - a_lo + 1);
            tile_cols = std::max(tile_cols, b_hi - b_lo + 1);
            tile_nodes = std::max(tile_nodes, (a_hi - a_lo + 1) * (b_hi - b_lo + 1));
            tile_sub = std::max(tile_sub, (std::min(w.i1, ns) - a_lo) * (std::min(w.j1, ns) - b_lo));
        }
        tile_nodes = (tile_nodes + 3) & ~3;
        tile_sub = (tile_sub + 3) & ~3;
        const size_t sensor_floats = (size_t)tile_nodes + 2 * (size_t)tile_sub;
        const size_t stab_floats = 2 * (size_t)Lmax * (tile_rows + tile_cols);
        // [working set of either phase][layer gather tables][sensor tables]:
        // the tables persist across phases for a CTA that keeps its items
        const size_t work_floats = (std::max(layer_floats, sensor_floats) + 3) & ~(size_t)3;
        size_t smem = (work_floats + gtab_floats + stab_floats) * sizeof(float);
        bool shared_tables = false;
        if (smem > smem_cap) {
            // too big to keep the tables apart: each phase's tables follow its own
            // working set, and each phase invalidates the other's
            shared_tables = true;
            const size_t lw = (layer_floats + 3) & ~(size_t)3;
            smem = std::max(lw + gtab_floats, sensor_floats + stab_floats) * sizeof(float);
        }
        if (smem > smem_cap) {
            if (err.empty()) err = "the working sets and tables of the phases do not fit in shared memory";
            delete pl;
            continue;
        }
        pl->smem = (int)smem;

        // device data
        bool ok = true;
        for (int i = 0; i < ninst && ok; ++i) {
            const HostSetup& hs = *hss[i];
            const DevGeo<float>& G = Gs[i];
            const FusedBuffers& fb = fbs[i];
            FInst I{};
            I.L = hs.L;
            I.G = hs.G;
            I.N = (int)hs.N;
            I.NW = (int)hs.NW;
            I.lay_n = G.lay_n;
            I.lay_J = G.lay_J;
            I.lay_off = G.lay_off;
            I.wfs_n = G.wfs_n;
            I.wfs_soff = G.wfs_soff;
            I.wfs_noff = G.wfs_noff;
            I.wfs_moff = G.wfs_moff;
            I.wfs_w = G.wfs_w;
            I.mask = G.mask;
            I.tab_off = G.tab_off;
            I.cx = G.cx;
            I.cy = G.cy;
            I.tx = G.tx;
            I.ty = G.ty;
            I.gat_off = G.gat_off;
            I.jlo = G.jlo;
            I.jhi = G.jhi;
            I.ilo = G.ilo;
            I.ihi = G.ihi;
            I.Jinv = fb.Jinv;
            I.aD = fb.aD;
            I.c = fb.c;
            I.r = fb.r;
            I.p = fb.p;
            I.q = fb.q;
            I.b = fb.b;
            I.bprev = fb.bprev;
            I.phi = fb.phi;
            I.sc_out = fb.sc;
            I.slopes = fb.slopes;
            I.w0 = w0[i];
            I.nw = nw[i];
            I.l0 = l0[i];
            I.nl = nl[i];
            I.KG = preps[i].KG;
            int2* d_gtab = nullptr;
            int* d_gtab_off = nullptr;
            // sensor fields (+8 floats: aligned copies may read up to 3 past the end)
            I.preA_cta = (i < n_res) ? tile_ctas + i : use_duty ? duty_cta(i) : -1;
            I.preA = nullptr;
            I.pubAB = nullptr;
            // LGS tip-tilt filter: per sensor flag, active count, tile range, and
            // the node fields Gamma^T (mask 1_x), Gamma^T (mask 1_y) (exact halves)
            I.tt_any = hs.any_tt ? 1 : 0;
            I.tt = G.wfs_tt;
            I.nact = G.wfs_nact;
            int2* d_ttt = nullptr;
            int2* d_nzr = nullptr;
            int4* d_nz = nullptr;
            if (hs.any_tt) {
                std::vector<int4> nz;
                std::vector<int2> nzr(hs.G, make_int2(0, 0));
                for (int g = 0; g < hs.G; ++g) {
                    nzr[g].x = (int)nz.size();
                    if (!hs.wfs[g].tt) continue;
                    const int ns = hs.wfs[g].n, np1 = ns + 1;
                    for (int ii = 0; ii <= ns; ++ii)
                        for (int jj = 0; jj <= ns; ++jj) {
                            double ax = 0.0, ay = 0.0;
                            for (int a = ii - 1; a <= ii; ++a)
                                for (int b = jj - 1; b <= jj; ++b) {
                                    if (a < 0 || a >= ns || b < 0 || b >= ns) continue;
                                    if (!hs.mask[hs.wfs[g].moff + (long)a * ns + b]) continue;
                                    ax += (b == jj - 1) ? 0.5 : -0.5;
                                    ay += (a == ii - 1) ? 0.5 : -0.5;
                                }
                            if (ax != 0.0 || ay != 0.0) {
                                const float fx = (float)ax, fy = (float)ay;
                                int bx, by;
                                std::memcpy(&bx, &fx, 4);
                                std::memcpy(&by, &fy, 4);
                                nz.push_back(make_int4(ii * np1 + jj, bx, by, 0));
                            }
                        }
                    nzr[g].y = (int)nz.size() - nzr[g].x;
                }
                ok = ok && dupload(pl, d_nz, nz, err) && dupload(pl, d_nzr, nzr, err) &&
                     dupload(pl, d_ttt, tt_tiles[i], err);
            }
            I.tt_nz = d_nz;
            I.tt_nzr = d_nzr;
            I.tt_tiles = d_ttt;
            ok = ok && dalloc(pl, I.psi, hs.NW + 8, err) && dalloc(pl, I.scal, 4, err) && dalloc(pl, I.preA, 12, err) &&
                 dalloc(pl, I.pubAB, 8, err) &&
                 dupload(pl, d_gtab, preps[i].gtab, err) && dupload(pl, d_gtab_off, preps[i].gtab_off, err);
            I.gtab = d_gtab;
            I.gtab_off = d_gtab_off;
            if (ok) cudaMemset(I.scal, 0, 4 * sizeof(double));
            if (ok) cudaMemset(I.preA, 0, 12 * sizeof(double));
            if (i == 0) pl->psi = I.psi;
            pl->inst.push_back(I);
        }
        // work lists: a sensor tile costs its nodes times the layers sampled,
        // a layer item its nodes times (transform + update + one gather per sensor)
        std::vector<double> wcost, lcost;
        for (auto& w : witems) {
            const HostSetup& hs = *hss[w.inst];
            wcost.push_back((double)(w.i1 - w.i0 + 1) * (w.j1 - w.j0 + 1) * (hs.L + 2));
        }
        for (auto& li : litems) {
            const HostSetup& hs = *hss[li.inst];
            const double n = hs.lay[li.l].n;
            lcost.push_back(n * n * (6.0 + hs.G) + 4096.0 * hs.lay[li.l].J);
        }
        std::vector<int> wsched, wsched_off, lsched, lsched_off;
        lpt_schedule(wcost, tile_ctas, wsched, wsched_off);
        for (int r = 0; r < n_res; ++r) wsched_off.push_back(wsched_off.back());   // reserved: no tiles
        lpt_schedule(lcost, pl->nclusters, lsched, lsched_off);
        // resident state: one layer item per cluster and room in shared memory
        int st_off = -1, st_stride = 0;
        if (V == 1 && !shared_tables) {
            int most = 0;
            for (size_t k = 0; k + 1 < lsched_off.size(); ++k) most = std::max(most, lsched_off[k + 1] - lsched_off[k]);
            const size_t stride = (cst.ncoef_max + 3) & ~(size_t)3;
            const size_t with_st = (size_t)pl->smem + 6 * stride * sizeof(float);
            if (most <= 1 && with_st <= smem_cap) {
                st_off = pl->smem / (int)sizeof(float);
                st_stride = (int)stride;
                pl->smem = (int)with_st;
            }
        }
        int *dws = nullptr, *dwo = nullptr, *dls = nullptr, *dlo = nullptr;
        ok = ok && dupload(pl, dws, wsched, err) && dupload(pl, dwo, wsched_off, err) &&
             dupload(pl, dls, lsched, err) && dupload(pl, dlo, lsched_off, err);
        WItem* dw = nullptr;
        LItem* dl = nullptr;
        int2* ds = nullptr;
        int4* ds4 = nullptr;
        int* dcs = nullptr;
        float2* wp = nullptr;
        float4* tp = nullptr;
        float4* lp = nullptr;
        unsigned* bar = nullptr;
        ok = ok && dupload(pl, dw, witems, err) && dupload(pl, dl, litems, err) && dupload(pl, ds, stg, err) &&
             dupload(pl, ds4, stg4, err) && dupload(pl, dcs, cshape, err) &&
             dalloc(pl, wp, witems.size(), err) && dalloc(pl, tp, witems.size(), err) &&
             dalloc(pl, lp, 2 * litems.size() * C, err) &&
             dalloc(pl, bar, 3, err) && dupload(pl, pl->d_inst, pl->inst, err);
        if (!ok) {
            fused_destroy(pl);
            return nullptr;
        }
        FParams& P = pl->P;
        P.witems = dw;
        P.litems = dl;
        P.stg = ds;
        P.stg4 = ds4;
        P.cshape = dcs;
        P.wsched = dws;
        P.wsched_off = dwo;
        P.lsched = dls;
        P.lsched_off = dlo;
        P.grid = pl->grid;
        P.res_first = tile_ctas;
        P.n_res = n_res;
        P.duty = nullptr;
        if (use_duty) {
            int* dd = nullptr;
            if (!dupload(pl, dd, duty, err)) {
                fused_destroy(pl);
                return nullptr;
            }
            P.duty = dd;
        }
        P.wpart = wp;
        P.tpart = tp;
        P.lpart = lp;
        P.bar = bar;
        P.errw = fbs[0].errw;
        P.n_inst = ninst;
        P.n_witems = (int)witems.size();
        P.n_litems = (int)litems.size();
        P.C = C;
        P.stripe_floats = stripe;
        P.stage_floats = stage_max;
        P.tile_nodes = tile_nodes;
        P.tile_subaps = tile_sub;
        P.shared_tables = shared_tables ? 1 : 0;
        P.ltab_off = shared_tables ? (int)((layer_floats + 3) & ~(size_t)3) : (int)work_floats;
        P.stab_off = shared_tables ? (int)sensor_floats : (int)(work_floats + gtab_floats);
        P.tile_rows = tile_rows;
        P.tile_cols = tile_cols;
        P.G_max = Gmax;
        P.n_max = nmax;
        P.v_z = (int)vz;
        P.v_t = (int)vt;
        P.v_u = (int)vu;
        P.v_r = (int)vr;
        P.v_c = (int)vc;
        P.v_rmax = Rmax;
        P.v_smax = cst.smax;
        P.v_tumax = (int)r4(cst.tu_max);
        P.v_tab = P.ltab_off + (int)(2 * (size_t)Gmax * (Rmax + nmax) * KGmax);
        P.v_st = st_off;
        P.v_sts = st_stride;
        for (int i = 0; i < 6; ++i) {
            P.h[i] = (float)hss[0]->h[i];
            P.g[i] = (float)hss[0]->g[i];
        }
        P.inst = pl->d_inst;
        {
            // L2 prefetch list: descriptors first, then tables, then the state,
            // up to a quarter of the L2 (a large batch keeps only its head)
            std::vector<PfChunk> ranges;
            size_t pf_total = 0;
            const size_t pf_budget = 32u << 20;
            auto add = [&](const void* ptr, size_t bytes) {
                if (!ptr || !bytes || pf_total + bytes > pf_budget) return;
                pf_total += bytes;
                ranges.push_back(PfChunk{(const char*)ptr, (int)bytes, 0});
            };
            add(dw, witems.size() * sizeof(WItem));
            add(dl, litems.size() * sizeof(LItem));
            add(ds, stg.size() * sizeof(int2));
            add(ds4, stg4.size() * sizeof(int4));
            add(dcs, cshape.size() * sizeof(int));
            add(dws, wsched.size() * sizeof(int));
            add(dwo, wsched_off.size() * sizeof(int));
            add(dls, lsched.size() * sizeof(int));
            add(dlo, lsched_off.size() * sizeof(int));
            add(pl->d_inst, pl->inst.size() * sizeof(FInst));
            for (int i = 0; i < ninst; ++i) {
                const HostSetup& hs = *hss[i];
                const FInst& I = pl->inst[i];
                add(I.lay_n, hs.L * sizeof(int));
                add(I.lay_J, hs.L * sizeof(int));
                add(I.lay_off, hs.L * sizeof(int));
                add(I.wfs_n, hs.G * sizeof(int));
                add(I.wfs_soff, hs.G * sizeof(int));
                add(I.wfs_noff, hs.G * sizeof(int));
                add(I.wfs_moff, hs.G * sizeof(int));
                add(I.wfs_w, hs.G * sizeof(float));
                add(I.tab_off, hs.tab_off.size() * sizeof(int));
                add(I.gtab_off, preps[i].gtab_off.size() * sizeof(int));
            }
            for (int i = 0; i < ninst; ++i) {
                const HostSetup& hs = *hss[i];
                const FInst& I = pl->inst[i];
                add(I.mask, hs.mask.size());
                add(I.cy, hs.cy.size() * sizeof(int));
                add(I.ty, hs.ty.size() * sizeof(float));
                add(I.cx, hs.cx.size() * sizeof(int));
                add(I.tx, hs.tx.size() * sizeof(float));
                add(I.gtab, preps[i].gtab.size() * sizeof(int2));
            }
            for (int i = 0; i < ninst; ++i) {
                const FInst& I = pl->inst[i];
                const size_t nb = (size_t)I.N * sizeof(float);
                for (const float* a : {(const float*)I.b, (const float*)I.bprev, (const float*)I.r,
                                       (const float*)I.c, I.Jinv, I.aD, (const float*)I.p, (const float*)I.q})
                    add(a, nb);
            }
            // 4 KB chunks, dealt round-robin to the CTAs (a fixed number each)
            std::vector<PfChunk> chunks;
            for (const PfChunk& r : ranges)
                for (int o = 0; o < r.bytes; o += 4096) chunks.push_back(PfChunk{r.p + o, std::min(4096, r.bytes - o), 0});
            const int per = (int)((chunks.size() + pl->grid - 1) / pl->grid);
            std::vector<PfChunk> table((size_t)per * pl->grid, PfChunk{nullptr, 0, 0});
            for (size_t j = 0; j < chunks.size(); ++j)
                table[(j % pl->grid) * per + j / pl->grid] = chunks[j];
            PfChunk* dpf = nullptr;
            if (per > 0 && dupload(pl, dpf, table, err)) {
                P.pf = dpf;
                P.pf_per_cta = per;
            } else {
                P.pf = nullptr;
                P.pf_per_cta = 0;
            }
        }
        best = pl;
        break;
    }
    if (!best) {
        if (err.empty()) err = "no cluster shape fits this geometry";
        return nullptr;
    }
    return best;
}

FusedPlan* fused_create(const HostSetup& hs, const DevGeo<float>& G, const FusedBuffers& fb, std::string& err) {
    return fused_create_multi({&hs}, {G}, {fb}, 0, err, 0, -1);
}

int fused_describe(const FusedPlan* pl, char* buf, int len) {
    return snprintf(buf, len,
                    "fused: %d clusters x %d CTAs (grid %d, %d threads), smem %d B, %d sensor tiles, %d layer items, "
                    "cooperative %d, tables %s, layer transform %s",
                    pl->nclusters, pl->C, pl->grid, kFThreads, pl->smem, pl->P.n_witems, pl->P.n_litems,
                    pl->cooperative ? 1 : 0, pl->P.shared_tables ? "shared" : "kept",
                    pl->V ? "level-stacked" : "row stripes");
}

void fused_set_trace(FusedPlan* pl, bool on) { pl->trace_on = on; }

int fused_cluster_size(const FusedPlan* pl) { return pl->C; }

int fused_layer_form(const FusedPlan* pl) { return pl->V; }

int fused_get_trace(FusedPlan* pl, unsigned long long* out, int max_entries, int* slots, int* grid) {
    *slots = pl->trace ? pl->last_slots : 0;
    *grid = pl->grid;
    if (!pl->trace || !out) return 0;
    size_t n = std::min((size_t)max_entries, (size_t)pl->last_slots * pl->grid * 2);
    return cudaMemcpy(out, pl->trace, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : 1;
}

int fused_get_fine_trace(FusedPlan* pl, unsigned long long* out, int max_entries, int* per_cta, int* grid) {
    *per_cta = pl->ftrace ? kFineCap : 0;
    *grid = pl->grid;
    if (!pl->ftrace || !out) return 0;
    size_t n = std::min((size_t)max_entries, (size_t)kFineCap * pl->grid);
    return cudaMemcpy(out, pl->ftrace, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost) == cudaSuccess ? 0
                                                                                                            : 1;
}

void fused_destroy(FusedPlan* plan) {
    if (!plan) return;
    if (plan->trace) cudaFree(plan->trace);
    if (plan->ftrace) cudaFree(plan->ftrace);
    for (void* a : plan->allocs) cudaFree(a);
    delete plan;
}

void fused_mark_dirty(FusedPlan* pl) { pl->bar_dirty = true; }

int fused_repoint_node(cudaGraphExec_t exec, cudaGraphNode_t node, const float* slopes, float* layers_out) {
    cudaKernelNodeParams kp;
    if (cudaGraphKernelNodeGetParams(node, &kp) != cudaSuccess || !kp.kernelParams || !kp.kernelParams[0]) {
        cudaGetLastError();
        return -1;
    }
    bool ours = false;
    for (int C : {1, 2, 4, 8, 16})
        for (int V : {0, 1}) ours = ours || kp.func == (void*)fused_kernel_for(C, V);
    if (!ours) return -1;
    FParams P = *static_cast<const FParams*>(kp.kernelParams[0]);
    if (P.n_inst != 1) return -1;
    P.slopes_in = slopes;
    P.phi_out = layers_out;
    void* args[1] = {&P};
    kp.kernelParams = args;
    kp.extra = nullptr;
    if (cudaGraphExecKernelNodeSetParams(exec, node, &kp) != cudaSuccess ||
        cudaGraphKernelNodeSetParams(node, &kp) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return 0;
}

int fused_solve(FusedPlan* pl, const float* slopes, int n_iter, int warm, int replace, long long budget,
                cudaStream_t stream, std::string& err, long long& launches, float* layers_out,
                unsigned long long* done_host, const unsigned* doorbell, unsigned doorbell_want,
                long long doorbell_ns) {
    // a completed launch leaves the barrier counters at zero (the last CTA out
    // resets them); after a failed or first launch they are zeroed here
    cudaError_t e = cudaSuccess;
    if (pl->bar_dirty) {
        e = cudaMemsetAsync(pl->P.bar, 0, 3 * sizeof(unsigned), stream);
        if (e != cudaSuccess) {
            err = std::string("fused setup copy: ") + cudaGetErrorString(e);
            return FEWHA_ERR_CUDA;
        }
        pl->bar_dirty = false;
    }
    FParams P = pl->P;
    // single instance: the frame's slopes and layers may live in the caller's buffers
    P.slopes_in = (P.n_inst == 1) ? slopes : nullptr;
    P.phi_out = (P.n_inst == 1) ? layers_out : nullptr;
    P.done_host = (P.n_inst == 1) ? done_host : nullptr;
    P.doorbell = (P.n_inst == 1) ? doorbell : nullptr;
    P.doorbell_want = doorbell_want;
    P.doorbell_ns = doorbell_ns;
    P.trace = nullptr;
    P.trace_slots = 0;
    P.ftrace = nullptr;
    P.fcap = 0;
    if (pl->trace_on) {
        // start, RHS barrier, first layer-phase barrier, 2 n_iter - 1 iteration
        // barriers (+2 for the replacement), end
        const int need = 3 + 2 * n_iter + (replace ? 2 : 0);
        if (need > pl->trace_slots) {
            if (pl->trace) cudaFree(pl->trace);
            pl->trace = nullptr;
            pl->trace_slots = 0;
            if (cudaMalloc(&pl->trace, (size_t)need * pl->grid * 2 * sizeof(unsigned long long)) == cudaSuccess)
                pl->trace_slots = need;
        }
        P.trace = pl->trace;
        P.trace_slots = pl->trace_slots;
        pl->last_slots = need;
        if (!pl->ftrace && cudaMalloc(&pl->ftrace, (size_t)kFineCap * pl->grid * sizeof(unsigned long long)) !=
                               cudaSuccess)
            pl->ftrace = nullptr;
        if (pl->ftrace) {
            cudaMemsetAsync(pl->ftrace, 0, (size_t)kFineCap * pl->grid * sizeof(unsigned long long), stream);
            P.ftrace = pl->ftrace;
            P.fcap = kFineCap;
        }
    }
    P.n_iter = n_iter;
    P.warm = warm;
    P.replace = replace;
    P.out_layers = 1;
    P.budget = budget;
    const FusedKernel kern = fused_kernel_for(pl->C, pl->V);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(pl->grid);
    cfg.blockDim = dim3(kFThreads);
    cfg.dynamicSmemBytes = pl->smem;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pl->cooperative ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, kern, P);
    if (e != cudaSuccess && pl->cooperative) {
        // cooperative + cluster not accepted: the grid is sized from the
        // occupancy query, so every cluster is resident; barriers stay bounded
        cudaGetLastError();
        pl->cooperative = false;
        cfg.numAttrs = 0;
        e = cudaLaunchKernelEx(&cfg, kern, P);
    }
    if (e != cudaSuccess) {
        err = std::string("fused launch: ") + cudaGetErrorString(e);
        return FEWHA_ERR_LAUNCH;
    }
    launches += 1;
    return FEWHA_OK;
}

}  // namespace fewha
