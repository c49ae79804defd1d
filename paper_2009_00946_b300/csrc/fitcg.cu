// Persistent FP32 mirror fit (Alg. 1 fitting step; readings R10, R17).
//
//   min_a  sum_t |P^DM_t a - P^lay_t phi|^2 + eps |a|^2
//
// by plain CG on the normal equations A a = rhs, A = sum_t P^DM_t^T P^DM_t +
// eps I (MOAO: mirror t in direction t only), n_fit steps from the previous
// solution x, then the gain of Alg. 1 -- one cooperative launch instead of the
// ~7 + 7 n_fit small kernels of the plain path.
//
// A depends only on the geometry, so the plan assembles it once on the host:
// with bilinear mirrors, direction t couples actuator (m, p, q) to (m', p', q')
// through Y_t^{mm'}(p, p') X_t^{mm'}(q, q'), Y / X the products of the row /
// column interpolation weights summed over the pupil nodes; each factor has a
// few entries per row, so a row of A is assembled exactly from a few hundred
// products.  A CG step is then one sparse product and one update:
//
//   A  q = A (r + beta p), p' = r + beta p, (p', q)          B
//   C  alpha = (r, r) / (p', q); x += alpha p'; r -= alpha q; (r, r)   B
//
// (p and p' alternate, so phase A reads the old direction while it writes the
// new one), after the right-hand side:
//
//   1  v_t = P^lay_t phi at every pupil node of every direction       B
//   2  r = sum_t P^DM_t^T v_t - A x, p = r, (r, r)                    B
//
// B are bounded grid barriers; every CTA sums the same per-CTA partials in the
// same order, so all hold bit-identical CG scalars (deterministic result).
// The last step applies the gain in place of its barrier.
#include "debug.cuh"
#include "fitcg.h"

#include <algorithm>
#include <vector>

namespace fewha {

FEWHA_DBG_READER(dbg_read_fitcg)

namespace {

constexpr int kFitThreads = 512;

struct FitCgParams {
    DevFit<float> F;
    const float* phi;
    FitCgBuffers b;
    const int* row;    // CSR of A: [NA + 1]
    const int* col;
    const float* val;
    const int* prow;   // CSR of sum_t P^DM_t^T: [NA + 1], columns t np1^2 + node
    const int* pcol;
    const float* pval;
    int gp_log;        // P^T rows are reduced by groups of 2^gp_log lanes
    long long nnz, pnnz;   // entries of A and of sum_t P^DM_t^T
    long long budget;
    float gain;
    int closed, n_fit, gs_log;   // rows of A are reduced by groups of 2^gs_log lanes
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Arrive by a release reduction (the block barrier before it orders the CTA's
// writes), wait by polling with acquire loads, bounded by the clock budget; on
// expiry the timeout bit is set and the CTA stops waiting at later barriers.
__device__ void fit_barrier(const FitCgParams& P, unsigned& target, int* s_abort) {
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(P.b.bar), "r"(1u) : "memory");
        if (!*s_abort) {
            const long long t0 = clock64();
            while ((int)(ld_acquire(P.b.bar) - target) < 0) {
                if (clock64() - t0 > P.budget) {
                    atomicOr(P.b.errw, kErrTimeout);
                    *s_abort = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
    }
    __syncthreads();
}

// Per-CTA partial sums sit on their own 128-byte lines (kPartStride doubles
// apart): every CTA reads every partial after a barrier, and partials packed
// into a few lines made those reads queue on a few L2 slices.
constexpr int kPartStride = 16;

// Sums without per-thread FP64 (this part issues about two FP64 operations
// per clock per SM, so FP64 work in every thread costs microseconds): a
// thread's sum is an unevaluated pair hi + lo of floats kept by TwoSum and the
// exact FMA product error (~48 bits), pairs are combined the same way, and
// FP64 appears only in a CTA's final partial and in the grid sum.
struct Pair {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(hi, x), bb = __fsub_rn(t, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
        hi = t;
    }
    __device__ __forceinline__ void add_prod(float a, float b) {   // += a * b
        const float pr = __fmul_rn(a, b);
        add(pr);
        lo = __fadd_rn(lo, fmaf(a, b, -pr));
    }
    __device__ __forceinline__ void add_pair(float h, float l) {
        add(h);
        lo = __fadd_rn(lo, l);
    }
};

// This CTA's partial of a sum (fixed order: warps' shuffle trees, then warp 0
// over the warp totals) into slot s; only thread 0 converts to FP64.
__device__ void put_partial(const FitCgParams& P, int s, Pair v, float2* sh2) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_down_sync(0xffffffffu, v.hi, o), l = __shfl_down_sync(0xffffffffu, v.lo, o);
        v.add_pair(h, l);
    }
    if (lane == 0) sh2[w] = make_float2(v.hi, v.lo);
    __syncthreads();
    if (w == 0) {
        Pair t;
        if (lane < nw) {
            t.hi = sh2[lane].x;
            t.lo = sh2[lane].y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float h = __shfl_down_sync(0xffffffffu, t.hi, o), l = __shfl_down_sync(0xffffffffu, t.lo, o);
            t.add_pair(h, l);
        }
        if (lane == 0)
            reinterpret_cast<float2*>(P.b.part)[((size_t)s * gridDim.x + blockIdx.x) * kPartStride] =
                make_float2(t.hi, t.lo);
    }
    __syncthreads();
}

// Sum of slot s over the grid, the same value in every CTA (fixed order,
// read through L2: the partials were written by other SMs).
__device__ double sum_partials(const FitCgParams& P, int s, double* sh) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const float2* src = reinterpret_cast<const float2*>(P.b.part) + (size_t)s * gridDim.x * kPartStride;
        // all of a lane's loads in flight at once (grid <= 256), then its sum
        // as a float pair (no FP64 latency chain); one conversion at the end
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = lane + 32 * u;
            v[u] = i < (int)gridDim.x ? __ldcg(src + (size_t)i * kPartStride) : make_float2(0.f, 0.f);
        }
        Pair t;
#pragma unroll
        for (int u = 0; u < 8; ++u) t.add_pair(v[u].x, v[u].y);
        for (int o = 16; o > 0; o >>= 1) {
            const float h = __shfl_down_sync(0xffffffffu, t.hi, o), l = __shfl_down_sync(0xffffffffu, t.lo, o);
            t.add_pair(h, l);
        }
        if (lane == 0) sh[32] = (double)t.hi + (double)t.lo;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

// Layers per round of lay_sample: the table and layer loads of kFitLU layers
// are in flight together (a 35-layer sample is 5 rounds of two dependent
// loads, not 35 of three); the sum still runs over l in order.
constexpr int kFitLU = 8;
// direction-layer table offsets, layer sides and offsets staged in shared
// memory when T * L fits
constexpr int kFitTabMax = 2048;

// sum_l bilinear(phi_l) along direction t at pupil node (i, jx); toff, ln,
// loff: the direction-layer table offsets [T][L], layer sides and offsets
__device__ __forceinline__ float lay_sample(const DevFit<float>& F, const float* phi, const int* toff, const int* ln,
                                            const int* loff, int t, int i, int jx, long nphi) {
    float acc = 0.f;
    for (int l0 = 0; l0 < F.L; l0 += kFitLU) {
        int cy[kFitLU], cx[kFitLU], n[kFitLU], o[kFitLU];
        float ty[kFitLU], tx[kFitLU], v[kFitLU][4];
#pragma unroll
        for (int u = 0; u < kFitLU; ++u) {
            const int l = l0 + u;
            if (l < F.L) {
                const int base = toff[t * F.L + l];
                n[u] = ln[l];
                o[u] = loff[l];
                cy[u] = __ldg(F.fcy + base + i);
                cx[u] = __ldg(F.fcx + base + jx);
                ty[u] = __ldg(F.fty + base + i);
                tx[u] = __ldg(F.ftx + base + jx);
            }
        }
#pragma unroll
        for (int u = 0; u < kFitLU; ++u) {
            if (l0 + u < F.L) {
                if (!FEWHA_IN(o[u] + (long)cy[u] * n[u] + cx[u], nphi, n[u] + 2, kDbgFit)) {
                    cy[u] = cx[u] = 0;   // a valid node; its value is not used
                    ty[u] = tx[u] = 0.f;
                    o[u] = 0;
                    n[u] = 0;
                }
                const float* f = phi + o[u] + (long)cy[u] * n[u] + cx[u];
                v[u][0] = f[0];
                v[u][1] = f[1];
                v[u][2] = f[n[u]];
                v[u][3] = f[n[u] + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < kFitLU; ++u)
            if (l0 + u < F.L)
                acc += (1 - ty[u]) * ((1 - tx[u]) * v[u][0] + tx[u] * v[u][1]) +
                       ty[u] * ((1 - tx[u]) * v[u][2] + tx[u] * v[u][3]);
    }
    return acc;
}

// Entries of a row a lane takes per round of a sparse product: all their
// index, value and gathered loads are issued before the adds, so a row of up
// to kFitU * 32 entries (the 35-layer fit averages 183) costs two dependent
// L2 round trips.
constexpr int kFitU = 8;

// A lane's share of row i of a CSR matrix times x: entries sub, sub + gsz, ...
__device__ __forceinline__ float csr_dot(const int* row, const int* col, const float* val, const float* x, int i,
                                         int sub, int gsz, int nx) {
    float s = 0.f;
    const int j1 = row[i + 1];
    for (int j0 = row[i] + sub; j0 < j1; j0 += kFitU * gsz) {
        int c[kFitU];
        float a[kFitU], xv[kFitU];
#pragma unroll
        for (int u = 0; u < kFitU; ++u) {
            const int j = j0 + u * gsz;
            c[u] = j < j1 ? __ldg(col + j) : 0;
            a[u] = j < j1 ? __ldg(val + j) : 0.f;
            if (!FEWHA_IN(c[u], nx, 1, kDbgFit)) c[u] = 0;
        }
#pragma unroll
        for (int u = 0; u < kFitU; ++u) xv[u] = x[c[u]];
#pragma unroll
        for (int u = 0; u < kFitU; ++u) s += a[u] * xv[u];
    }
    return s;
}

// sum over a group of 2^lg lanes (fixed order), valid in the group's first lane
__device__ __forceinline__ float group_sum(float v, int lg) {
    for (int o = (1 << lg) >> 1; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kFitThreads, 1) k_fit_cg(const __grid_constant__ FitCgParams P) {
    __shared__ double sh[33];
    __shared__ float2 sh2[32];
    __shared__ float s_scal;   // alpha or beta, formed by thread 0
    __shared__ int s_abort;
    const DevFit<float>& F = P.F;
    const FitCgBuffers& B = P.b;
    const int nthr = gridDim.x * blockDim.x, gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, gwarp = gtid >> 5, nwarps = nthr >> 5;
    const int np1 = F.np1, nn = np1 * np1, Tn = F.T_ * nn, NA = F.NA;
    const int lg = P.gs_log, gsz = 1 << lg, sub = lane & (gsz - 1);
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    unsigned target = 0;

    double rr = 0.0;
    float beta = 0.f;
    if (P.n_fit > 0) {
        // the matrices of step 2 and the CG steps (static; evicted when other
        // work ran since the last frame) are requested into L2 first, so they
        // arrive while the layers are sampled: each CTA takes a share of the
        // 128-byte lines of each array
        {
            const char* arr[6] = {(const char*)P.col, (const char*)P.val, (const char*)P.pcol,
                                  (const char*)P.pval, (const char*)P.row, (const char*)P.prow};
            const long long bytes[6] = {P.nnz * 4, P.nnz * 4, P.pnnz * 4, P.pnnz * 4, (long long)(NA + 1) * 4,
                                        (long long)(NA + 1) * 4};
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const long long lines = (bytes[a] + 127) >> 7;
                for (long long q = gtid; q < lines; q += nthr)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(arr[a] + (q << 7)));
            }
        }
        // 1: the layers at every pupil node of every direction
        __shared__ int s_toff[kFitTabMax], s_ln[64], s_loff[64];
        const bool staged = F.T_ * F.L <= kFitTabMax && F.L <= 64;
        if (staged) {
            for (int e = threadIdx.x; e < F.T_ * F.L; e += blockDim.x) s_toff[e] = __ldg(F.ftab_off + e);
            for (int e = threadIdx.x; e < F.L; e += blockDim.x) {
                s_ln[e] = __ldg(F.lay_n + e);
                s_loff[e] = __ldg(F.lay_off + e);
            }
        }
        __syncthreads();
        const int* toff = staged ? s_toff : F.ftab_off;
        const int* lns = staged ? s_ln : F.lay_n;
        const int* loff = staged ? s_loff : F.lay_off;
        [[maybe_unused]] const long nphi = (long)loff[F.L - 1] + (long)lns[F.L - 1] * lns[F.L - 1];
        for (int e = gtid; e < Tn; e += nthr) {
            const int t = e / nn, idx = e - t * nn, i = idx / np1, jx = idx - i * np1;
            B.v[e] = lay_sample(F, P.phi, toff, lns, loff, t, i, jx, nphi);
        }
        fit_barrier(P, target, &s_abort);
        // 2: r = sum_t P^DM_t^T v_t - A x, p = r (groups of lanes per row, as in A)
        Pair acc;
        const int lp = P.gp_log, gpz = 1 << lp, subp = lane & (gpz - 1);
        for (int i0 = gwarp << (5 - lp); i0 < NA; i0 += nwarps << (5 - lp)) {
            const int i = i0 + (lane >> lp);
            float s = 0.f;
            if (i < NA) {
                s = csr_dot(P.prow, P.pcol, P.pval, B.v, i, subp, gpz, Tn);
                s -= csr_dot(P.row, P.col, P.val, B.x, i, subp, gpz, NA);
            }
            s = group_sum(s, lp);
            if (subp == 0 && i < NA) {
                B.r[i] = s;
                B.p[i] = s;
                acc.add_prod(s, s);
            }
        }
        put_partial(P, 0, acc, sh2);
        fit_barrier(P, target, &s_abort);
        rr = sum_partials(P, 0, sh);
    }
    float* pc = B.p;    // current direction
    float* pn = B.p2;   // next direction
    for (int k = 0; k < P.n_fit; ++k) {
        const bool last = k + 1 == P.n_fit;
        // A: p' = r + beta p, q = A p' (p' formed on the fly from the old p)
        const float fb = (float)beta;
        Pair pq_acc;
        // a warp takes 32 / 2^lg consecutive rows per pass (the trip count is the
        // same for the whole warp, so every shuffle has all its lanes).  Software
        // pipeline: the gathers of the current rows' first round are issued,
        // then the next rows' bounds and first round of entries are loaded
        // while those gathers are in flight
        const int stride = nwarps << (5 - lg);
        int nb = 0, ne = 0, nc[kFitU];
        float na[kFitU];
        auto first_round = [&](int i0x) {
            const int ix = i0x + (lane >> lg);
            nb = ne = 0;
            if (i0x < NA && ix < NA) {
                nb = __ldg(P.row + ix) + sub;
                ne = __ldg(P.row + ix + 1);
            }
#pragma unroll
            for (int u = 0; u < kFitU; ++u) {
                const int j = nb + u * gsz;
                nc[u] = j < ne ? __ldg(P.col + j) : 0;
                na[u] = j < ne ? __ldg(P.val + j) : 0.f;
                if (!FEWHA_IN(nc[u], NA, 1, kDbgFit)) nc[u] = 0;
            }
        };
        first_round(gwarp << (5 - lg));
        for (int i0 = gwarp << (5 - lg); i0 < NA; i0 += stride) {
            const int i = i0 + (lane >> lg);
            float s = 0.f;
            const int j0f = nb, j1 = ne;
            float a0[kFitU], rv0[kFitU], pv0[kFitU];
#pragma unroll
            for (int u = 0; u < kFitU; ++u) {   // index 0 (a valid entry, weight 0) past the row
                a0[u] = na[u];
                rv0[u] = B.r[nc[u]];
                pv0[u] = pc[nc[u]];
            }
            first_round(i0 + stride);
            if (i < NA) {
#pragma unroll
                for (int u = 0; u < kFitU; ++u) s += a0[u] * (rv0[u] + fb * pv0[u]);
                // rows longer than one round: the rest, round by round
                for (int j0 = j0f + kFitU * gsz; j0 < j1; j0 += kFitU * gsz) {
                    int c[kFitU];
                    float a[kFitU], rv[kFitU], pv[kFitU];
#pragma unroll
                    for (int u = 0; u < kFitU; ++u) {
                        const int j = j0 + u * gsz;
                        c[u] = j < j1 ? __ldg(P.col + j) : 0;
                        a[u] = j < j1 ? __ldg(P.val + j) : 0.f;
                        if (!FEWHA_IN(c[u], NA, 1, kDbgFit)) c[u] = 0;
                    }
#pragma unroll
                    for (int u = 0; u < kFitU; ++u) {
                        rv[u] = B.r[c[u]];
                        pv[u] = pc[c[u]];
                    }
#pragma unroll
                    for (int u = 0; u < kFitU; ++u) s += a[u] * (rv[u] + fb * pv[u]);
                }
            }
            s = group_sum(s, lg);
            if (sub == 0 && i < NA) {
                const float pi = B.r[i] + fb * pc[i];
                pn[i] = pi;
                B.q[i] = s;
                pq_acc.add_prod(pi, s);
            }
        }
        put_partial(P, 1, pq_acc, sh2);
        fit_barrier(P, target, &s_abort);
        const double pq = sum_partials(P, 1, sh);
        if (threadIdx.x == 0) s_scal = (pq > 0.0 && rr > 0.0) ? (float)(rr / pq) : 0.f;
        __syncthreads();
        const float alpha = s_scal;
        // C: the step (and on the last step the gain: the same thread owns x[a])
        Pair rr_acc;
        for (int a = gtid; a < NA; a += nthr) {
            const float xa = B.x[a] + alpha * pn[a];
            B.x[a] = xa;
            if (!last) {
                const float ra = B.r[a] - alpha * B.q[a];
                B.r[a] = ra;
                rr_acc.add_prod(ra, ra);
            } else {
                const float a0 = B.acur[a];
                B.acur[a] = P.closed ? a0 + P.gain * (xa - B.aprev[a]) : (1 - P.gain) * a0 + P.gain * xa;
                B.aprev[a] = a0;
            }
        }
        if (!last) {
            put_partial(P, 2, rr_acc, sh2);
            fit_barrier(P, target, &s_abort);
            const double rr_new = sum_partials(P, 2, sh);
            __syncthreads();   // every thread has read s_scal (alpha) above
            if (threadIdx.x == 0) s_scal = rr > 0.0 ? (float)(rr_new / rr) : 0.f;
            __syncthreads();
            beta = s_scal;
            rr = rr_new;
            float* t = pc;
            pc = pn;
            pn = t;
        }
    }
    if (P.n_fit == 0) {
        for (int a = gtid; a < NA; a += nthr) {
            const float a0 = B.acur[a], xa = B.x[a];
            B.acur[a] = P.closed ? a0 + P.gain * (xa - B.aprev[a]) : (1 - P.gain) * a0 + P.gain * xa;
            B.aprev[a] = a0;
        }
    }
    // the last CTA out zeroes the counters for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(B.bar + 1, 1u) == gridDim.x - 1u) {
            B.bar[0] = 0u;
            B.bar[1] = 0u;
            __threadfence();
        }
    }
}

// One factor of a direction's coupling: for every row index p of mirror m,
// the entries (p', sum over pupil nodes of w_m(node, p) w_m'(node, p')).
using Factor = std::vector<std::vector<std::pair<int, double>>>;

Factor make_factor(const int* cm, const double* tm, int na_m, const int* cn, const double* tn, int nodes) {
    Factor f(na_m);
    auto add = [&](int p, int q, double w) {
        for (auto& e : f[p])
            if (e.first == q) {
                e.second += w;
                return;
            }
        f[p].push_back({q, w});
    };
    for (int k = 0; k < nodes; ++k) {
        const double wm[2] = {1.0 - tm[k], tm[k]}, wn[2] = {1.0 - tn[k], tn[k]};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) add(cm[k] + a, cn[k] + b, wm[a] * wn[b]);
    }
    return f;
}

}  // namespace

struct FitCgPlan {
    int grid = 0, gs_log = 5, gp_log = 5;
    long nnz = 0, pnnz = 0;
    bool dirty = true;
    int* row = nullptr;
    int* col = nullptr;
    float* val = nullptr;
    int* prow = nullptr;
    int* pcol = nullptr;
    float* pval = nullptr;
};

FitCgPlan* fitcg_create(const HostSetup& hs, const DevFit<float>& F, std::string& err) {
    if (hs.M < 1 || hs.M > 8 || hs.T < 1 || hs.NA < 1 || hs.NA > (1L << 30)) {
        err = "no mirror fit to plan";
        return nullptr;
    }
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fit_cg, kFitThreads, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        err = "the device cannot co-schedule the fit kernel";
        return nullptr;
    }
    // the normal matrix: for every (t, m, m') the row and column factors
    const int M = hs.M, T = hs.T, nodes = hs.fit_n + 1;
    std::vector<Factor> Y((size_t)T * M * M), X((size_t)T * M * M);
    auto pair_ok = [&](int t, int m, int mp) { return !hs.moao || (m == t && mp == t); };
    for (int t = 0; t < T; ++t)
        for (int m = 0; m < M; ++m)
            for (int mp = 0; mp < M; ++mp) {
                if (!pair_ok(t, m, mp)) continue;
                const int bm = hs.dtab_off[t * M + m], bn = hs.dtab_off[t * M + mp];
                const size_t k = ((size_t)t * M + m) * M + mp;
                Y[k] = make_factor(hs.dcy.data() + bm, hs.dty.data() + bm, hs.dm[m].na, hs.dcy.data() + bn,
                                   hs.dty.data() + bn, nodes);
                X[k] = make_factor(hs.dcx.data() + bm, hs.dtx.data() + bm, hs.dm[m].na, hs.dcx.data() + bn,
                                   hs.dtx.data() + bn, nodes);
            }
    // sum_t P^DM_t^T: row k lists (t np1^2 + node, weight) of every pupil node
    // whose bilinear cell on mirror m touches actuator k (MOAO: t = m)
    std::vector<std::vector<std::pair<int, float>>> pt(hs.NA);
    for (int t = 0; t < T; ++t)
        for (int m = 0; m < M; ++m) {
            if (hs.moao && m != t) continue;
            const int b = hs.dtab_off[t * M + m], na = hs.dm[m].na;
            for (int i = 0; i < nodes; ++i)
                for (int j = 0; j < nodes; ++j) {
                    const double wy[2] = {1.0 - hs.dty[b + i], hs.dty[b + i]};
                    const double wx[2] = {1.0 - hs.dtx[b + j], hs.dtx[b + j]};
                    for (int a = 0; a < 2; ++a)
                        for (int c = 0; c < 2; ++c) {
                            const double w = wy[a] * wx[c];
                            if (w == 0.0) continue;
                            const long k = hs.dm[m].off + (long)(hs.dcy[b + i] + a) * na + hs.dcx[b + j] + c;
                            pt[k].push_back({t * nodes * nodes + i * nodes + j, (float)w});
                        }
                }
        }
    std::vector<int> prow(1, 0), pcol;
    std::vector<float> pval;
    for (auto& r : pt) {
        for (auto& e : r) {
            pcol.push_back(e.first);
            pval.push_back(e.second);
        }
        prow.push_back((int)pcol.size());
        std::vector<std::pair<int, float>>().swap(r);
    }
    std::vector<int> row(1, 0), col;
    std::vector<float> val;
    std::vector<double> buf(hs.NA, 0.0);
    std::vector<char> hit(hs.NA, 0);
    std::vector<int> touched;
    for (int m = 0; m < M; ++m) {
        const int na = hs.dm[m].na;
        for (int p = 0; p < na; ++p)
            for (int q = 0; q < na; ++q) {
                const long self = hs.dm[m].off + (long)p * na + q;
                touched.clear();
                for (int t = 0; t < T; ++t)
                    for (int mp = 0; mp < M; ++mp) {
                        if (!pair_ok(t, m, mp)) continue;
                        const size_t k = ((size_t)t * M + m) * M + mp;
                        const int nb = hs.dm[mp].na;
                        for (const auto& y : Y[k][p])
                            for (const auto& x : X[k][q]) {
                                const long c = hs.dm[mp].off + (long)y.first * nb + x.first;
                                if (!hit[c]) {
                                    hit[c] = 1;
                                    touched.push_back((int)c);
                                }
                                buf[c] += y.second * x.second;
                            }
                    }
                if (!hit[self]) {
                    hit[self] = 1;
                    touched.push_back((int)self);
                }
                buf[self] += hs.fit_eps;
                std::sort(touched.begin(), touched.end());
                for (int c : touched) {
                    col.push_back(c);
                    val.push_back((float)buf[c]);
                    buf[c] = 0.0;
                    hit[c] = 0;
                }
                row.push_back((int)col.size());
            }
    }
    auto* pl = new FitCgPlan();
    pl->grid = std::min(sms, 256);   // the partial sums are read 8 per lane
    pl->nnz = (long)col.size();
    pl->pnnz = (long)pcol.size();
    auto group_log = [&](double avg) { return avg > 48 ? 5 : avg > 24 ? 4 : avg > 12 ? 3 : 2; };
    pl->gs_log = group_log((double)pl->nnz / (double)hs.NA);
    pl->gp_log = group_log((double)pcol.size() / (double)hs.NA);
    auto up = [&](auto*& d, const auto& v) {
        using U = typename std::decay_t<decltype(v)>::value_type;
        if (cudaMalloc(&d, v.size() * sizeof(U)) != cudaSuccess) return false;
        return cudaMemcpy(d, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!up(pl->row, row) || !up(pl->col, col) || !up(pl->val, val) || !up(pl->prow, prow) ||
        !up(pl->pcol, pcol) || !up(pl->pval, pval)) {
        cudaGetLastError();
        err = "fit matrix upload";
        fitcg_destroy(pl);
        return nullptr;
    }
    (void)F;
    return pl;
}

void fitcg_destroy(FitCgPlan* pl) {
    if (!pl) return;
    cudaFree(pl->row);
    cudaFree(pl->col);
    cudaFree(pl->val);
    cudaFree(pl->prow);
    cudaFree(pl->pcol);
    cudaFree(pl->pval);
    delete pl;
}
long fitcg_nnz(const FitCgPlan* pl) { return pl ? pl->nnz : 0; }
int fitcg_grid(const FitCgPlan* pl) { return pl ? pl->grid : 0; }
size_t fitcg_part_doubles(const FitCgPlan* pl) { return pl ? 3 * (size_t)pl->grid * kPartStride : 0; }
void fitcg_mark_dirty(FitCgPlan* pl) {
    if (pl) pl->dirty = true;
}

int fitcg_launch(FitCgPlan* pl, const DevFit<float>& F, const float* phi, const FitCgBuffers& b, int n_fit,
                 float gain, int closed, long long budget, cudaStream_t stream, std::string& err,
                 long long& launches) {
    if (pl->dirty) {
        if (cudaMemsetAsync(b.bar, 0, 2 * sizeof(unsigned), stream) != cudaSuccess) {
            err = "fit barrier reset";
            return FEWHA_ERR_CUDA;
        }
        pl->dirty = false;
    }
    FitCgParams P{};
    P.F = F;
    P.phi = phi;
    P.b = b;
    P.row = pl->row;
    P.col = pl->col;
    P.val = pl->val;
    P.prow = pl->prow;
    P.pcol = pl->pcol;
    P.pval = pl->pval;
    P.gp_log = pl->gp_log;
    P.nnz = pl->nnz;
    P.pnnz = pl->pnnz;
    P.budget = budget;
    P.gain = gain;
    P.closed = closed;
    P.n_fit = n_fit;
    P.gs_log = pl->gs_log;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(pl->grid);
    cfg.blockDim = dim3(kFitThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_fit_cg, P);
    if (e != cudaSuccess) {
        err = std::string("fit launch: ") + cudaGetErrorString(e);
        return FEWHA_ERR_CUDA;
    }
    ++launches;
    return FEWHA_OK;
}

}  // namespace fewha
