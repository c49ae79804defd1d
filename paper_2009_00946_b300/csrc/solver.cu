// Plain FEWHA path: one simple kernel per operator (Sec. 3.2 matrix-free
// operators), templated on float / double, with FP64 reductions; plus the
// solver object that owns the device state of one instance.
#include <cuda.h>   // the types of the driver's stream write (taken through the runtime's entry-point query)
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <type_traits>

#include "debug.cuh"
#include "fitcg.h"
#include "fused.h"
#include "solver.h"

namespace fewha {

FEWHA_DBG_READER(dbg_read_solver)

#define FEWHA_CUDA(call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                      \
            return FEWHA_ERR_CUDA;                                                         \
        }                                                                                  \
    } while (0)

#define FEWHA_LAUNCHED()                                                                   \
    do {                                                                                   \
        ++launches;                                                                        \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess) {                                                           \
            err = std::string("kernel launch: ") + cudaGetErrorString(e_);                 \
            return FEWHA_ERR_CUDA;                                                         \
        }                                                                                  \
    } while (0)

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;   // valid in thread 0
}

// z = Jinv * r ; partial (r, z)
template <typename T>
__global__ void k_precond_dot(int N, const T* __restrict__ Jinv, const T* __restrict__ r, T* __restrict__ z,
                              double* __restrict__ part) {
    __shared__ double sh[32];
    const long fo = (long)blockIdx.z * N;   // frame blockIdx.z of a batch
    r += fo;
    z += fo;
    part += (size_t)blockIdx.z * gridDim.x;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        T zi = Jinv[i] * r[i];
        z[i] = zi;
        acc += (double)r[i] * (double)zi;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// s += aD * z ; partial (s, z)
template <typename T>
__global__ void k_reg_dot(int N, const T* __restrict__ aD, const T* __restrict__ z, T* __restrict__ s,
                          double* __restrict__ part) {
    __shared__ double sh[32];
    const long fo = (long)blockIdx.z * N;
    z += fo;
    s += fo;
    part += (size_t)blockIdx.z * gridDim.x;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        T si = s[i] + aD[i] * z[i];
        s[i] = si;
        acc += (double)si * (double)z[i];
    }
    double v = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// generic partial dot (a, b)
template <typename T>
__global__ void k_dot(int N, const T* __restrict__ a, const T* __restrict__ b, double* __restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    double v = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__device__ double sum_partials(const double* part, int n, double* sh) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    return block_sum(acc, sh);
}

// Alg. 2 scalar recurrence: beta = rho/rho_old, alpha = rho/(mu - rho beta/alpha_old).
__global__ void k_alg2_scalars(const double* part_rho, const double* part_mu, double* sc, int k, int* errw) {
    __shared__ double sh[32];
    part_rho += (size_t)blockIdx.x * kRedBlocks;   // one block per frame of a batch
    part_mu += (size_t)blockIdx.x * kRedBlocks;
    sc += (size_t)blockIdx.x * kNumScalars;
    double rho = sum_partials(part_rho, kRedBlocks, sh);
    __syncthreads();
    double mu = sum_partials(part_mu, kRedBlocks, sh);
    if (threadIdx.x == 0) {
        double beta = 0.0, denom = mu;
        if (k > 0) {
            beta = rho / sc[kRhoOld];
            denom = mu - rho * beta / sc[kAlphaOld];
        }
        double a = rho / denom;
        if (!(denom > 0.0) || !isfinite(a) || !isfinite(beta)) {
            atomicOr(errw, kErrBreakdown);
            a = 0.0;
            beta = 0.0;
        }
        sc[kRho] = rho;
        sc[kMu] = mu;
        sc[kBeta] = beta;
        sc[kAlphaK] = a;
        sc[kRhoOld] = rho;
        sc[kAlphaOld] = (a != 0.0) ? a : sc[kAlphaOld];
    }
}

// p = z + beta p ; q = s + beta q ; c += alpha p ; r -= alpha q
template <typename T>
__global__ void k_alg2_update(int N, const double* __restrict__ sc, int first, const T* __restrict__ z,
                              const T* __restrict__ s, T* __restrict__ p, T* __restrict__ q, T* __restrict__ c,
                              T* __restrict__ r) {
    const long fo = (long)blockIdx.z * N;
    sc += (size_t)blockIdx.z * kNumScalars;
    z += fo;
    s += fo;
    p += fo;
    q += fo;
    c += fo;
    r += fo;
    const T beta = (T)sc[kBeta], a = (T)sc[kAlphaK];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        T pi = first ? z[i] : z[i] + beta * p[i];
        T qi = first ? s[i] : s[i] + beta * q[i];
        p[i] = pi;
        q[i] = qi;
        c[i] += a * pi;
        r[i] -= a * qi;
    }
}

// ---------------------------------------------------------------------------
// periodic db3 DWT, one pass over the active LL block of every layer
// ---------------------------------------------------------------------------

// forward, rows: row y, output col c: a_c / d_{c-m/2} of x[y][(2k+t) mod m]
template <typename T>
__global__ void k_fwd_rows(DevGeo<T> G, int j, const T* __restrict__ src, T* __restrict__ dst) {
    int l = blockIdx.y;
    if (j > G.lay_J[l]) return;
    src += (long)blockIdx.z * G.N;   // frame blockIdx.z of a batch
    dst += (long)blockIdx.z * G.N;
    int n = G.lay_n[l], m = n >> (j - 1), half = m >> 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    int y = idx / m, c = idx - y * m;
    const T* s = src + G.lay_off[l] + (long)y * n;
    int k = c < half ? c : c - half;
    const T* f = c < half ? G.h : G.g;
    T acc = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) acc += f[t] * s[(2 * k + t) % m];
    dst[G.lay_off[l] + (long)y * n + c] = acc;
}

template <typename T>
__global__ void k_fwd_cols(DevGeo<T> G, int j, const T* __restrict__ src, T* __restrict__ dst) {
    int l = blockIdx.y;
    if (j > G.lay_J[l]) return;
    src += (long)blockIdx.z * G.N;   // frame blockIdx.z of a batch
    dst += (long)blockIdx.z * G.N;
    int n = G.lay_n[l], m = n >> (j - 1), half = m >> 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    int rr = idx / m, x = idx - rr * m;
    const T* s = src + G.lay_off[l] + x;
    int k = rr < half ? rr : rr - half;
    const T* f = rr < half ? G.h : G.g;
    T acc = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) acc += f[t] * s[(long)((2 * k + t) % m) * n];
    dst[G.lay_off[l] + (long)rr * n + x] = acc;
}

// inverse, columns: x[i] = sum over taps t with (i - t) mod m even of
// h_t a_k + g_t d_k, k = ((i - t) mod m) / 2
template <typename T>
__global__ void k_inv_cols(DevGeo<T> G, int j, const T* __restrict__ src, T* __restrict__ dst) {
    int l = blockIdx.y;
    if (j > G.lay_J[l]) return;
    src += (long)blockIdx.z * G.N;   // frame blockIdx.z of a batch
    dst += (long)blockIdx.z * G.N;
    int n = G.lay_n[l], m = n >> (j - 1), half = m >> 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    int i = idx / m, x = idx - i * m;
    const T* s = src + G.lay_off[l] + x;
    T acc = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        int r = ((i - t) % m + m) % m;
        if (r & 1) continue;
        int k = r >> 1;
        acc += G.h[t] * s[(long)k * n] + G.g[t] * s[(long)(half + k) * n];
    }
    dst[G.lay_off[l] + (long)i * n + x] = acc;
}

template <typename T>
__global__ void k_inv_rows(DevGeo<T> G, int j, const T* __restrict__ src, T* __restrict__ dst) {
    int l = blockIdx.y;
    if (j > G.lay_J[l]) return;
    src += (long)blockIdx.z * G.N;   // frame blockIdx.z of a batch
    dst += (long)blockIdx.z * G.N;
    int n = G.lay_n[l], m = n >> (j - 1), half = m >> 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    int y = idx / m, i = idx - y * m;
    const T* s = src + G.lay_off[l] + (long)y * n;
    T acc = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        int r = ((i - t) % m + m) % m;
        if (r & 1) continue;
        int k = r >> 1;
        acc += G.h[t] * s[k] + G.g[t] * s[half + k];
    }
    dst[G.lay_off[l] + (long)y * n + i] = acc;
}

// ---------------------------------------------------------------------------
// P, Gamma, C^{-1}, Gamma^T, P^T
// ---------------------------------------------------------------------------

// psi_g(i, j) = sum_l bilinear(phi_l) at the node's sample point (Sec. 2.1)
template <typename T>
__global__ void k_P(DevGeo<T> G, const T* __restrict__ phi, T* __restrict__ psi) {
    int g = blockIdx.y, ns = G.wfs_n[g], np1 = ns + 1;
    phi += (long)blockIdx.z * G.N;
    psi += (long)blockIdx.z * G.NW;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= np1 * np1) return;
    int i = idx / np1, jx = idx - i * np1;
    T acc = 0;
    for (int l = 0; l < G.L; ++l) {
        int base = G.tab_off[g * G.L + l], n = G.lay_n[l];
        int cy = G.cy[base + i], cx = G.cx[base + jx];
        T ty = G.ty[base + i], tx = G.tx[base + jx];
        const long fi = G.lay_off[l] + (long)cy * n + cx;
        if (!FEWHA_IN(fi, G.N, n + 2, kDbgPlainP)) continue;
        const T* f = phi + fi;
        acc += (1 - ty) * ((1 - tx) * f[0] + tx * f[1]) + ty * ((1 - tx) * f[n] + tx * f[n + 1]);
    }
    if (FEWHA_IN(G.wfs_noff[g] + idx, G.NW, 1, kDbgPlainP)) psi[G.wfs_noff[g] + idx] = acc;
}

// weighted slopes w_g mask (Gamma psi)  (C^{-1} Gamma, Sec. 2.1 / Sec. 2.2)
template <typename T>
__global__ void k_gamma_w(DevGeo<T> G, const T* __restrict__ psi, T* __restrict__ sl) {
    int g = blockIdx.y, ns = G.wfs_n[g], np1 = ns + 1;
    psi += (long)blockIdx.z * G.NW;
    sl += (long)blockIdx.z * G.S;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ns * ns) return;
    int a = idx / ns, b = idx - a * ns;
    if (!FEWHA_IN(G.wfs_noff[g] + (long)a * np1 + b, G.NW, np1 + 2, kDbgPlainGam) ||
        !FEWHA_IN(G.wfs_soff[g] + ns * ns + idx, G.S, 1, kDbgPlainGam))
        return;
    const T* p = psi + G.wfs_noff[g] + (long)a * np1 + b;
    T sx = ((p[1] - p[0]) + (p[np1 + 1] - p[np1])) / 2;
    T sy = ((p[np1] - p[0]) + (p[np1 + 1] - p[1])) / 2;
    T wm = G.mask[G.wfs_moff[g] + idx] ? G.wfs_w[g] : (T)0;
    sl[G.wfs_soff[g] + idx] = wm * sx;
    sl[G.wfs_soff[g] + ns * ns + idx] = wm * sy;
}

// weighted slope residual w mask (s - Gamma psi) of a residual replacement
// (measured minus modelled slopes; non-finite measured slopes count as 0, as
// in the right-hand side)
template <typename T>
__global__ void k_resid_w(DevGeo<T> G, const T* __restrict__ s, const T* __restrict__ psi, T* __restrict__ sl) {
    int g = blockIdx.y, ns = G.wfs_n[g], np1 = ns + 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ns * ns) return;
    int a = idx / ns, b = idx - a * ns;
    if (!FEWHA_IN(G.wfs_noff[g] + (long)a * np1 + b, G.NW, np1 + 2, kDbgPlainGam) ||
        !FEWHA_IN(G.wfs_soff[g] + ns * ns + idx, G.S, 1, kDbgPlainGam))
        return;
    const T* p = psi + G.wfs_noff[g] + (long)a * np1 + b;
    T sx = ((p[1] - p[0]) + (p[np1 + 1] - p[np1])) / 2;
    T sy = ((p[np1] - p[0]) + (p[np1 + 1] - p[1])) / 2;
    T mx = s[G.wfs_soff[g] + idx], my = s[G.wfs_soff[g] + ns * ns + idx];
    mx = isfinite((double)mx) ? mx : (T)0;
    my = isfinite((double)my) ? my : (T)0;
    T wm = G.mask[G.wfs_moff[g] + idx] ? G.wfs_w[g] : (T)0;
    sl[G.wfs_soff[g] + idx] = wm * (mx - sx);
    sl[G.wfs_soff[g] + ns * ns + idx] = wm * (my - sy);
}

// weighted measurement slopes for the right-hand side; non-finite active
// slopes raise the INPUT error bit, inactive ones are ignored
template <typename T>
__global__ void k_weight_meas(DevGeo<T> G, const T* __restrict__ s, T* __restrict__ sl, int* errw) {
    int g = blockIdx.y, ns = G.wfs_n[g];
    s += (long)blockIdx.z * G.S;
    sl += (long)blockIdx.z * G.S;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ns * ns) return;
    bool on = G.mask[G.wfs_moff[g] + idx] != 0;
    T vx = s[G.wfs_soff[g] + idx], vy = s[G.wfs_soff[g] + ns * ns + idx];
    if (on && (!isfinite((double)vx) || !isfinite((double)vy))) atomicOr(errw, kErrInput);
    T w = G.wfs_w[g];
    sl[G.wfs_soff[g] + idx] = on && isfinite((double)vx) ? w * vx : (T)0;
    sl[G.wfs_soff[g] + ns * ns + idx] = on && isfinite((double)vy) ? w * vy : (T)0;
}

// LGS tip-tilt filter: per filtered sensor (one block each) the sums of its
// weighted x and y slopes, reduced in a fixed order
template <typename T>
__global__ void k_tt_sums(DevGeo<T> G, const T* __restrict__ sl, double* __restrict__ sums) {
    __shared__ double sh[32];
    const int g = blockIdx.x;
    if (!G.wfs_tt[g]) return;
    const int ns = G.wfs_n[g], n2 = ns * ns;
    const T* S = sl + G.wfs_soff[g] + blockIdx.y * n2;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) acc += (double)S[i];
    const double v = block_sum(acc, sh);
    if (threadIdx.x == 0) sums[2 * g + blockIdx.y] = v;
}

// weighted slopes w mask s  ->  w mask (s - mean over active), per axis
template <typename T>
__global__ void k_tt_apply(DevGeo<T> G, const double* __restrict__ sums, T* __restrict__ sl) {
    const int g = blockIdx.y, ns = G.wfs_n[g];
    if (!G.wfs_tt[g]) return;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ns * ns || !G.mask[G.wfs_moff[g] + idx]) return;
    const double inv = 1.0 / G.wfs_nact[g];
    sl[G.wfs_soff[g] + idx] -= (T)(sums[2 * g] * inv);
    sl[G.wfs_soff[g] + ns * ns + idx] -= (T)(sums[2 * g + 1] * inv);
}

// psi'(i, j) = (Gamma^T sl)(i, j): gather of the <= 4 adjacent subapertures
template <typename T>
__global__ void k_gammaT(DevGeo<T> G, const T* __restrict__ sl, T* __restrict__ psi) {
    int g = blockIdx.y, ns = G.wfs_n[g], np1 = ns + 1;
    sl += (long)blockIdx.z * G.S;
    psi += (long)blockIdx.z * G.NW;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= np1 * np1) return;
    int i = idx / np1, jx = idx - i * np1;
    const T* SX = sl + G.wfs_soff[g];
    const T* SY = SX + ns * ns;
    T acc = 0;
    for (int a = i - 1; a <= i; ++a) {
        if (a < 0 || a >= ns) continue;
        for (int b = jx - 1; b <= jx; ++b) {
            if (b < 0 || b >= ns) continue;
            if (!FEWHA_IN(G.wfs_soff[g] + ns * ns + a * ns + b, G.S, 1, kDbgPlainGam)) continue;
            T sx = SX[a * ns + b], sy = SY[a * ns + b];
            acc += (b == jx - 1 ? sx : -sx) + (a == i - 1 ? sy : -sy);
        }
    }
    if (FEWHA_IN(G.wfs_noff[g] + idx, G.NW, 1, kDbgPlainGam)) psi[G.wfs_noff[g] + idx] = acc / 2;
}

// y_l(p, q) = sum_g (P_gl^T psi'_g)(p, q): deterministic gather over the
// sensor nodes whose sample point lies in one of the 4 cells around (p, q)
template <typename T>
__global__ void k_PT(DevGeo<T> G, const T* __restrict__ psi, T* __restrict__ y) {
    int l = blockIdx.y, n = G.lay_n[l];
    psi += (long)blockIdx.z * G.NW;
    y += (long)blockIdx.z * G.N;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int p = idx / n, q = idx - p * n;
    T acc = 0;
    for (int g = 0; g < G.G; ++g) {
        int base = G.tab_off[g * G.L + l], gb = G.gat_off[g * G.L + l];
        int i0 = G.ilo[gb + p], i1 = G.ihi[gb + p], j0 = G.jlo[gb + q], j1 = G.jhi[gb + q];
        int np1 = G.wfs_n[g] + 1;
        const T* P = psi + G.wfs_noff[g];
        for (int i = i0; i < i1; ++i) {
            T wy = (G.cy[base + i] == p) ? 1 - G.ty[base + i] : G.ty[base + i];
            T row = 0;
            for (int jx = j0; jx < j1; ++jx) {
                T wx = (G.cx[base + jx] == q) ? 1 - G.tx[base + jx] : G.tx[base + jx];
                if (FEWHA_IN(G.wfs_noff[g] + (long)i * np1 + jx, G.NW, 1, kDbgPlainPT)) row += wx * P[(long)i * np1 + jx];
            }
            acc += wy * row;
        }
    }
    if (FEWHA_IN(G.lay_off[l] + idx, G.N, 1, kDbgPlainPT)) y[G.lay_off[l] + idx] = acc;
}

// ---------------------------------------------------------------------------
// frame bookkeeping (Alg. 1)
// ---------------------------------------------------------------------------

// warm restart r = (b1 - b0) + r0 ; b0 = b1
template <typename T>
__global__ void k_warm(int N, const T* __restrict__ b, T* __restrict__ bprev, T* __restrict__ r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        T bi = b[i];
        r[i] = (bi - bprev[i]) + r[i];
        bprev[i] = bi;
    }
}

// residual replacement r = b1 - M c0 = d - alpha D c0 with d = W P^T Gamma^T
// C^{-1} (s - Gamma P W^T c0), the data residual formed in the slope domain
// (b1 and M c0 agree to a few per cent, so their difference would lose the
// digits of the working precision); the subtraction in FP64 ; b0 = b1
template <typename T>
__global__ void k_replace(int N, const T* __restrict__ b, const T* __restrict__ d, const T* __restrict__ aD,
                          const T* __restrict__ c, T* __restrict__ bprev, T* __restrict__ r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        r[i] = (T)((double)d[i] - (double)aD[i] * (double)c[i]);
        bprev[i] = b[i];
    }
}

// cold start c = 0, r = b1 ; b0 = b1
template <typename T>
__global__ void k_cold(int N, const T* __restrict__ b, T* __restrict__ bprev, T* __restrict__ r, T* __restrict__ c) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        T bi = b[i];
        r[i] = bi;
        bprev[i] = bi;
        c[i] = 0;
    }
}

// ---------------------------------------------------------------------------
// fitting: least squares over the fitting directions (NGS-type)
// ---------------------------------------------------------------------------

// v_t(node) = sum_l bilinear(phi_l) along direction t on the pupil grid
template <typename T>
__global__ void k_fit_lay(DevFit<T> F, const T* __restrict__ phi, T* __restrict__ v) {
    int t = blockIdx.y, np1 = F.np1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= np1 * np1) return;
    int i = idx / np1, jx = idx - i * np1;
    T acc = 0;
    for (int l = 0; l < F.L; ++l) {
        int base = F.ftab_off[t * F.L + l], n = F.lay_n[l];
        int cy = F.fcy[base + i], cx = F.fcx[base + jx];
        T ty = F.fty[base + i], tx = F.ftx[base + jx];
        const T* f = phi + F.lay_off[l] + (long)cy * n + cx;
        acc += (1 - ty) * ((1 - tx) * f[0] + tx * f[1]) + ty * ((1 - tx) * f[n] + tx * f[n + 1]);
    }
    v[(long)t * np1 * np1 + idx] = acc;
}

// v_t(node) = sum_m bilinear(a_m) along direction t (MOAO: m = t only)
template <typename T>
__global__ void k_fit_dm(DevFit<T> F, const T* __restrict__ a, T* __restrict__ v) {
    int t = blockIdx.y, np1 = F.np1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= np1 * np1) return;
    int i = idx / np1, jx = idx - i * np1;
    T acc = 0;
    for (int m = F.moao ? t : 0; m < (F.moao ? t + 1 : F.M); ++m) {
        int base = F.dtab_off[t * F.M + m], n = F.dm_n[m];
        int cy = F.dcy[base + i], cx = F.dcx[base + jx];
        T ty = F.dty[base + i], tx = F.dtx[base + jx];
        const T* f = a + F.dm_off[m] + (long)cy * n + cx;
        acc += (1 - ty) * ((1 - tx) * f[0] + tx * f[1]) + ty * ((1 - tx) * f[n] + tx * f[n + 1]);
    }
    v[(long)t * np1 * np1 + idx] = acc;
}

// out(actuator) = sum_t (P_DM_t^T v_t)(actuator) [+ eps * x(actuator)]
// (MOAO: t = m only)
template <typename T>
__global__ void k_fit_dmT(DevFit<T> F, const T* __restrict__ v, const T* __restrict__ x, T eps, T* __restrict__ out) {
    int m = blockIdx.y, n = F.dm_n[m];
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int p = idx / n, q = idx - p * n, np1 = F.np1;
    T acc = 0;
    for (int t = F.moao ? m : 0; t < (F.moao ? m + 1 : F.T_); ++t) {
        int base = F.dtab_off[t * F.M + m], gb = F.dgat_off[t * F.M + m];
        int i0 = F.dilo[gb + p], i1 = F.dihi[gb + p], j0 = F.djlo[gb + q], j1 = F.djhi[gb + q];
        const T* V = v + (long)t * np1 * np1;
        for (int i = i0; i < i1; ++i) {
            T wy = (F.dcy[base + i] == p) ? 1 - F.dty[base + i] : F.dty[base + i];
            T row = 0;
            for (int jx = j0; jx < j1; ++jx) {
                T wx = (F.dcx[base + jx] == q) ? 1 - F.dtx[base + jx] : F.dtx[base + jx];
                row += wx * V[(long)i * np1 + jx];
            }
            acc += wy * row;
        }
    }
    long o = F.dm_off[m] + idx;
    if (x) acc += eps * x[o];
    out[o] = acc;
}

// r = rhs - A x ; p = r
template <typename T>
__global__ void k_fit_init(int NA, const T* __restrict__ rhs, const T* __restrict__ Ax, T* __restrict__ r,
                           T* __restrict__ p) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NA; i += gridDim.x * blockDim.x) {
        T v = rhs[i] - Ax[i];
        r[i] = v;
        p[i] = v;
    }
}

// CG step: a = rr / pq (0 if pq <= 0 or rr == 0); x += a p ; r -= a q ; partial (r, r)
template <typename T>
__global__ void k_fit_step(int NA, const double* __restrict__ sc, T* __restrict__ x, T* __restrict__ r,
                           const T* __restrict__ p, const T* __restrict__ q, double* __restrict__ part) {
    __shared__ double sh[32];
    double rr = sc[kRR], pq = sc[kMu];
    T a = (pq > 0.0 && rr > 0.0) ? (T)(rr / pq) : (T)0;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NA; i += gridDim.x * blockDim.x) {
        x[i] += a * p[i];
        T ri = r[i] - a * q[i];
        r[i] = ri;
        acc += (double)ri * (double)ri;
    }
    double v = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// scalar helpers for the fit CG: which = 0 -> sc[kRR] = sum ; 1 -> sc[kMu] = sum ;
// 2 -> beta: sc[kBeta] = sum / sc[kRR], sc[kRR] = sum
__global__ void k_fit_scalar(const double* part, double* sc, int which) {
    __shared__ double sh[32];
    double s = sum_partials(part, kRedBlocks, sh);
    if (threadIdx.x == 0) {
        if (which == 0) sc[kRR] = s;
        else if (which == 1) sc[kMu] = s;
        else {
            double old = sc[kRR];
            sc[kBeta] = old > 0.0 ? s / old : 0.0;
            sc[kRR] = s;
        }
    }
}

template <typename T>
__global__ void k_fit_dir(int NA, const double* __restrict__ sc, const T* __restrict__ r, T* __restrict__ p) {
    T b = (T)sc[kBeta];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NA; i += gridDim.x * blockDim.x) p[i] = r[i] + b * p[i];
}

// a1 = (1 - g) a0 + g a~ ; a(-1) = a0 ; a0 = a1
template <typename T>
__global__ void k_gain(int NA, T gain, const T* __restrict__ afit, T* __restrict__ acur, T* __restrict__ aprev) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NA; i += gridDim.x * blockDim.x) {
        T a0 = acur[i];
        aprev[i] = a0;
        acur[i] = (1 - gain) * a0 + gain * afit[i];
    }
}

// co-located fit (L = M): actuator (ky, kx) of mirror m takes layer m's
// bilinear value at its position
template <typename T>
__global__ void k_fit_colocated(DevFit<T> F, const T* __restrict__ phi, T* __restrict__ a) {
    const int m = blockIdx.y, na = F.dm_n[m];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= na * na) return;
    const int ky = idx / na, kx = idx - ky * na, base = F.ctab_off[m], n = F.lay_n[m];
    const int cy = F.ccx[base + ky], cx = F.ccx[base + kx];
    const T ty = F.ctx[base + ky], tx = F.ctx[base + kx];
    const T* f = phi + F.lay_off[m] + (long)cy * n + cx;
    a[F.dm_off[m] + idx] = (1 - ty) * ((1 - tx) * f[0] + tx * f[1]) + ty * ((1 - tx) * f[n] + tx * f[n + 1]);
}

// closed-loop gain (Alg. 1): a1 = a0 + gain (a~ - a_{-1}); a_{-1} <- a0
template <typename T>
__global__ void k_gain_closed(int NA, T gain, const T* __restrict__ afit, T* __restrict__ acur,
                              T* __restrict__ aprev) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NA; i += gridDim.x * blockDim.x) {
        const T a0 = acur[i], am1 = aprev[i];
        aprev[i] = a0;
        acur[i] = a0 + gain * (afit[i] - am1);
    }
}

// psi_g = sum_m P_{g,m} a_m: the mirrors at the nodes of sensor g (Alg. 1, closed loop)
template <typename T>
__global__ void k_dm_wfs(DevGeo<T> G, DevFit<T> F, const T* __restrict__ a, T* __restrict__ psi) {
    const int g = blockIdx.y, np1 = G.wfs_n[g] + 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= np1 * np1) return;
    const int i = idx / np1, jx = idx - i * np1;
    T acc = 0;
    for (int m = 0; m < F.M; ++m) {
        const int base = F.wdtab_off[g * F.M + m], n = F.dm_n[m];
        const int cy = F.wdcy[base + i], cx = F.wdcx[base + jx];
        const T ty = F.wdty[base + i], tx = F.wdtx[base + jx];
        const T* f = a + F.dm_off[m] + (long)cy * n + cx;
        acc += (1 - ty) * ((1 - tx) * f[0] + tx * f[1]) + ty * ((1 - tx) * f[n] + tx * f[n + 1]);
    }
    psi[G.wfs_noff[g] + idx] = acc;
}

// s += Gamma psi on every subaperture: pseudo-open-loop slopes
template <typename T>
__global__ void k_add_gamma(DevGeo<T> G, const T* __restrict__ psi, T* __restrict__ s) {
    const int g = blockIdx.y, ns = G.wfs_n[g], np1 = ns + 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ns * ns) return;
    const int a = idx / ns, b = idx - a * ns;
    const T* p = psi + G.wfs_noff[g] + (long)a * np1 + b;
    const T sx = ((p[1] - p[0]) + (p[np1 + 1] - p[np1])) / 2;
    const T sy = ((p[np1] - p[0]) + (p[np1 + 1] - p[1])) / 2;
    s[G.wfs_soff[g] + idx] += sx;
    s[G.wfs_soff[g] + ns * ns + idx] += sy;
}

// ---------------------------------------------------------------------------
// solver object
// ---------------------------------------------------------------------------

template <typename T>
static void to_T(const std::vector<double>& v, std::vector<T>& o) {
    o.resize(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
}

#include "adjoint.cuh"

template <typename T>
class Solver : public SolverBase {
  public:
    DevGeo<T> G{};
    DevFit<T> F{};
    std::vector<void*> allocs;
    void* pinned_in = nullptr;    // staging for fewha_frame
    void* pinned_out = nullptr;
    void* pinned_dm = nullptr;
    T *slopes = nullptr, *c = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *s = nullptr;
    T *b = nullptr, *bprev = nullptr, *phi = nullptr, *tmp = nullptr, *y = nullptr, *wpsi = nullptr, *wpsi2 = nullptr,
      *wsl = nullptr, *Jinv = nullptr, *aD = nullptr, *Jd = nullptr, *ext = nullptr;
    T *afit = nullptr, *acur = nullptr, *aprev = nullptr, *fr = nullptr, *fp = nullptr, *fq = nullptr, *frhs = nullptr,
      *fv = nullptr;
    double *part = nullptr, *part2 = nullptr, *sc = nullptr, *ttsums = nullptr;
    int* errw = nullptr;
    int* errw_host = nullptr;
    // completion word of a host frame on the fused path (mapped pinned host
    // memory; the kernel sets it to (1 << 32) | error word when the frame's
    // results are visible, so the host waits on it instead of the stream)
    unsigned long long* done_host = nullptr;
    unsigned long long* done_dev = nullptr;
    // armed frames: a mapped pinned doorbell word the launched kernel waits on
    unsigned* bell_host = nullptr;
    unsigned* bell_dev = nullptr;
    unsigned bell_seq = 0;
    bool armed = false;
    double armed_wait_s = 0.0;
    const unsigned* ov_bell = nullptr;
    unsigned ov_bell_want = 0;
    long long ov_bell_ns = 0;
    // armed frames with host_slopes_copy: at the fire, the slopes go in by a
    // copy-engine transfer on a second stream and a stream write of the go
    // into a device word follows it (no SM work: the armed kernel holds them all)
    using WriteValue32 = CUresult (*)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);
    WriteValue32 write_value = nullptr;
    bool write_value_tried = false;
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t prior_done = nullptr;   // the handle's stream before the armed launch: the copy waits for it
    unsigned* go_dev = nullptr;
    bool armed_copy = false;
    const void* armed_src = nullptr;
    unsigned long long* ov_done = nullptr;
    FusedPlan* fused = nullptr;
    FitCgPlan* fitcg = nullptr;     // persistent FP32 fit (fused path)
    T* fu = nullptr;                // its second search direction [NA]
    double* fpart = nullptr;        // its partial sums [3][grid]
    unsigned* fbar = nullptr;       // its barrier counters
    FusedBuffers fbuf{};     // state the fused plans point to (FP32 only)
    // a device-pointer frame on the fused path: the kernel reads the caller's
    // slopes and writes the caller's layers directly (no copy nodes)
    const float* ov_slopes = nullptr;
    float* ov_layers = nullptr;
    bool closed = false;        // closed loop (Alg. 1): pseudo-open-loop slopes and closed-loop gain
    bool pol_pending = false;   // the frame's slopes still lack Gamma P_DM a_{-1}
    // graph cache
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraph_t gsrc[2] = {nullptr, nullptr};          // graph each exec was instantiated from
    cudaGraphNode_t gknode[2] = {nullptr, nullptr};    // its lone fused kernel node (direct frames)
    struct Key {
        int n_iter = -1, warm = -1, n_fit = -1, path = -1, k_rr = -1;
        double gain = -1;
        const void* sin = nullptr;
        void* lout = nullptr;
        void* dout = nullptr;
        bool same_work(const Key& o) const {   // all but the slopes / layers buffers
            return n_iter == o.n_iter && warm == o.warm && n_fit == o.n_fit && gain == o.gain && dout == o.dout &&
                   path == o.path && k_rr == o.k_rr && (lout == nullptr) == (o.lout == nullptr);
        }
        bool operator==(const Key& o) const { return same_work(o) && sin == o.sin && lout == o.lout; }
    } gkey[2];

    void drop_graph(int i) {
        if (gexec[i]) cudaGraphExecDestroy(gexec[i]);
        if (gsrc[i]) cudaGraphDestroy(gsrc[i]);
        gexec[i] = nullptr;
        gsrc[i] = nullptr;
        gknode[i] = nullptr;
    }

    ~Solver() override {
        if (armed) frame_fire();   // an armed frame still waiting: let it run rather than wait out its deadline
        if (aux_stream) {
            cudaStreamSynchronize(aux_stream);
            cudaStreamDestroy(aux_stream);
        }
        if (prior_done) cudaEventDestroy(prior_done);
        if (stream) cudaStreamSynchronize(stream);
        else cudaDeviceSynchronize();
        for (int i = 0; i < 2; ++i) drop_graph(i);
        if (fused) fused_destroy(fused);
        if (fitcg) fitcg_destroy(fitcg);
        for (void* a : allocs) cudaFree(a);
        if (pinned_in) cudaFreeHost(pinned_in);
        if (pinned_out) cudaFreeHost(pinned_out);
        if (pinned_dm) cudaFreeHost(pinned_dm);
        if (errw_host) cudaFreeHost(errw_host);
        if (done_host) cudaFreeHost(done_host);
        if (bell_host) cudaFreeHost(bell_host);
    }

    template <typename U>
    int alloc(U*& ptr, size_t count) {
        void* v = nullptr;
        FEWHA_CUDA(cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(U)));
        allocs.push_back(v);
        ptr = (U*)v;
        return FEWHA_OK;
    }
    template <typename U>
    int upload(U*& ptr, const std::vector<U>& v) {
        int st = alloc(ptr, v.size());
        if (st) return st;
        if (!v.empty()) FEWHA_CUDA(cudaMemcpy(ptr, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice));
        return FEWHA_OK;
    }
    template <typename U>
    int uploadT(U*& ptr, const std::vector<double>& v) {
        std::vector<U> t;
        to_T(v, t);
        return upload(ptr, t);
    }

#define TRY(x)                   \
    do {                         \
        int st_ = (x);           \
        if (st_) return st_;     \
    } while (0)

    int init() {
        const HostSetup& H = hs;
        std::vector<int> lay_n, lay_J, lay_off, wfs_n, wfs_soff, wfs_noff, wfs_moff;
        std::vector<double> wfs_w;
        int Jmax = 0, nmax = 0, nsmax = 0;
        for (auto& L : H.lay) {
            lay_n.push_back(L.n);
            lay_J.push_back(L.J);
            lay_off.push_back((int)L.off);
            Jmax = std::max(Jmax, L.J);
            nmax = std::max(nmax, L.n);
        }
        for (auto& w : H.wfs) {
            wfs_n.push_back(w.n);
            wfs_soff.push_back((int)w.soff);
            wfs_noff.push_back((int)w.noff);
            wfs_moff.push_back((int)w.moff);
            wfs_w.push_back(w.w);
            nsmax = std::max(nsmax, w.n);
        }
        G.L = H.L;
        G.G = H.G;
        G.N = (int)H.N;
        G.S = (int)H.S;
        G.NW = (int)H.NW;
        G.NS = (int)H.NS;
        G.Jmax = Jmax;
        G.nmax = nmax;
        G.nsmax = nsmax;
        for (int i = 0; i < 6; ++i) {
            G.h[i] = (T)H.h[i];
            G.g[i] = (T)H.g[i];
        }
        int *d_lay_n, *d_lay_J, *d_lay_off, *d_wfs_n, *d_wfs_soff, *d_wfs_noff, *d_wfs_moff;
        TRY(upload(d_lay_n, lay_n));
        TRY(upload(d_lay_J, lay_J));
        TRY(upload(d_lay_off, lay_off));
        TRY(upload(d_wfs_n, wfs_n));
        TRY(upload(d_wfs_soff, wfs_soff));
        TRY(upload(d_wfs_noff, wfs_noff));
        TRY(upload(d_wfs_moff, wfs_moff));
        G.lay_n = d_lay_n;
        G.lay_J = d_lay_J;
        G.lay_off = d_lay_off;
        G.wfs_n = d_wfs_n;
        G.wfs_soff = d_wfs_soff;
        G.wfs_noff = d_wfs_noff;
        G.wfs_moff = d_wfs_moff;
        T* d_w;
        TRY(uploadT(d_w, wfs_w));
        G.wfs_w = d_w;
        unsigned char* d_mask;
        TRY(upload(d_mask, H.mask));
        G.mask = d_mask;
        int *d_tab_off, *d_cx, *d_cy, *d_gat_off, *d_jlo, *d_jhi, *d_ilo, *d_ihi;
        T *d_tx, *d_ty;
        TRY(upload(d_tab_off, H.tab_off));
        TRY(upload(d_cx, H.cx));
        TRY(upload(d_cy, H.cy));
        TRY(uploadT(d_tx, H.tx));
        TRY(uploadT(d_ty, H.ty));
        TRY(upload(d_gat_off, H.gat_off));
        TRY(upload(d_jlo, H.jlo));
        TRY(upload(d_jhi, H.jhi));
        TRY(upload(d_ilo, H.ilo));
        TRY(upload(d_ihi, H.ihi));
        G.tab_off = d_tab_off;
        G.cx = d_cx;
        G.cy = d_cy;
        G.tx = d_tx;
        G.ty = d_ty;
        G.gat_off = d_gat_off;
        G.jlo = d_jlo;
        G.jhi = d_jhi;
        G.ilo = d_ilo;
        G.ihi = d_ihi;
        std::vector<double> jinv(H.N);
        for (long i = 0; i < H.N; ++i) jinv[i] = 1.0 / H.Jdiag[i];
        TRY(uploadT(Jinv, jinv));
        TRY(uploadT(aD, H.aD));
        TRY(uploadT(Jd, H.Jdiag));
        G.Jinv = Jinv;
        G.aD = aD;
        {
            std::vector<int> tt(H.G), nact(H.G);
            for (int g = 0; g < H.G; ++g) {
                tt[g] = H.wfs[g].tt ? 1 : 0;
                nact[g] = H.wfs[g].nact;
            }
            int *d_tt, *d_nact;
            TRY(upload(d_tt, tt));
            TRY(upload(d_nact, nact));
            G.wfs_tt = d_tt;
            G.wfs_nact = d_nact;
            G.any_tt = H.any_tt ? 1 : 0;
            TRY(alloc(ttsums, 2 * (size_t)H.G));
        }
        const size_t N = H.N;
        for (T** v : {&c, &r, &p, &q, &z, &s, &b, &bprev, &phi, &tmp, &y, &ext}) TRY(alloc(*v, N));
        TRY(alloc(slopes, H.S));
        TRY(alloc(wsl, H.S));
        TRY(alloc(wpsi, H.NW));
        TRY(alloc(wpsi2, H.NW));
        TRY(alloc(part, kRedBlocks));
        TRY(alloc(part2, kRedBlocks));
        TRY(alloc(sc, kNumScalars));
        TRY(alloc(errw, 1));
        FEWHA_CUDA(cudaMallocHost((void**)&errw_host, sizeof(int)));
        FEWHA_CUDA(cudaHostAlloc((void**)&done_host, sizeof(unsigned long long), cudaHostAllocMapped));
        *done_host = 0ull;
        FEWHA_CUDA(cudaHostGetDevicePointer((void**)&done_dev, done_host, 0));
        for (T* v : {c, r, p, q, z, s, b, bprev, phi, tmp, y, ext}) FEWHA_CUDA(cudaMemset(v, 0, N * sizeof(T)));
        FEWHA_CUDA(cudaMemset(slopes, 0, H.S * sizeof(T)));
        FEWHA_CUDA(cudaMemset(sc, 0, kNumScalars * sizeof(double)));
        FEWHA_CUDA(cudaMemset(errw, 0, sizeof(int)));
        if (H.M > 0) TRY(init_fit());
        FEWHA_CUDA(cudaDeviceSynchronize());
        return FEWHA_OK;
    }

    int init_fit() {
        const HostSetup& H = hs;
        F.L = H.L;
        F.M = H.M;
        F.T_ = H.T;
        F.moao = H.moao ? 1 : 0;
        F.NA = (int)H.NA;
        F.np1 = H.fit_n + 1;
        F.eps = (T)H.fit_eps;
        F.lay_n = G.lay_n;
        F.lay_off = G.lay_off;
        std::vector<int> dm_n, dm_off;
        for (auto& d : H.dm) {
            dm_n.push_back(d.na);
            dm_off.push_back((int)d.off);
        }
        int *d_dm_n, *d_dm_off, *a, *bb, *cc, *dd, *e, *f, *g1, *h1, *i1, *j1;
        T *tx1, *ty1, *tx2, *ty2;
        TRY(upload(d_dm_n, dm_n));
        TRY(upload(d_dm_off, dm_off));
        TRY(upload(a, H.ftab_off));
        TRY(upload(bb, H.fcx));
        TRY(upload(cc, H.fcy));
        TRY(uploadT(tx1, H.ftx));
        TRY(uploadT(ty1, H.fty));
        TRY(upload(dd, H.dtab_off));
        TRY(upload(e, H.dcx));
        TRY(upload(f, H.dcy));
        TRY(uploadT(tx2, H.dtx));
        TRY(uploadT(ty2, H.dty));
        TRY(upload(g1, H.dgat_off));
        TRY(upload(h1, H.djlo));
        TRY(upload(i1, H.djhi));
        TRY(upload(j1, H.dilo));
        int* k1;
        TRY(upload(k1, H.dihi));
        F.dm_n = d_dm_n;
        F.dm_off = d_dm_off;
        F.ftab_off = a;
        F.fcx = bb;
        F.fcy = cc;
        F.ftx = tx1;
        F.fty = ty1;
        F.dtab_off = dd;
        F.dcx = e;
        F.dcy = f;
        F.dtx = tx2;
        F.dty = ty2;
        F.dgat_off = g1;
        F.djlo = h1;
        F.djhi = i1;
        F.dilo = j1;
        F.dihi = k1;
        F.colocated = H.colocated ? 1 : 0;
        if (H.colocated) {
            int *c1, *c2;
            T* c3;
            TRY(upload(c1, H.ctab_off));
            TRY(upload(c2, H.ccx));
            TRY(uploadT(c3, H.ctx));
            F.ctab_off = c1;
            F.ccx = c2;
            F.ctx = c3;
        }
        if (H.closed_ok) {
            int *w1, *w2, *w3;
            T *w4, *w5;
            TRY(upload(w1, H.wdtab_off));
            TRY(upload(w2, H.wdcx));
            TRY(upload(w3, H.wdcy));
            TRY(uploadT(w4, H.wdtx));
            TRY(uploadT(w5, H.wdty));
            F.wdtab_off = w1;
            F.wdcx = w2;
            F.wdcy = w3;
            F.wdtx = w4;
            F.wdty = w5;
        }
        for (T** v : {&afit, &acur, &aprev, &fr, &fp, &fq, &frhs}) {
            TRY(alloc(*v, H.NA));
            FEWHA_CUDA(cudaMemset(*v, 0, H.NA * sizeof(T)));
        }
        TRY(alloc(fv, (size_t)H.T * F.np1 * F.np1));
        if constexpr (std::is_same<T, float>::value) {
            // the persistent fit of the fused path (none: the plain kernels)
            std::string ferr;
            if (!F.colocated && (fitcg = fitcg_create(H, F, ferr)) != nullptr) {
                TRY(alloc(fu, (size_t)H.NA));
                TRY(alloc(fpart, fitcg_part_doubles(fitcg)));
                TRY(alloc(fbar, 2));
                FEWHA_CUDA(cudaMemset(fbar, 0, 2 * sizeof(unsigned)));
            }
        }
        return FEWHA_OK;
    }

    // ---- building blocks (all enqueued on `stream`) ----
    // frames of the current launch sequence: 1, or the frame count of a batched
    // taped solve / reverse mode (every kernel of the operator chain takes
    // frame blockIdx.z, the frames' vectors contiguous)
    int nb = 1;
    dim3 grid_layers(int count) const { return dim3((count + 255) / 256, G.L, nb); }

    int inv_dwt(const T* src, T* dst) {   // dst = W^T src (dst != src)
        FEWHA_CUDA(cudaMemcpyAsync(dst, src, (size_t)G.N * nb * sizeof(T), cudaMemcpyDeviceToDevice, stream));
        for (int j = G.Jmax; j >= 1; --j) {
            int m = G.nmax >> (j - 1);
            k_inv_cols<T><<<grid_layers(m * m), 256, 0, stream>>>(G, j, dst, tmp);
            FEWHA_LAUNCHED();
            k_inv_rows<T><<<grid_layers(m * m), 256, 0, stream>>>(G, j, tmp, dst);
            FEWHA_LAUNCHED();
        }
        return FEWHA_OK;
    }

    int fwd_dwt(const T* src, T* dst) {   // dst = W src (dst != src)
        FEWHA_CUDA(cudaMemcpyAsync(dst, src, (size_t)G.N * nb * sizeof(T), cudaMemcpyDeviceToDevice, stream));
        for (int j = 1; j <= G.Jmax; ++j) {
            int m = G.nmax >> (j - 1);
            k_fwd_rows<T><<<grid_layers(m * m), 256, 0, stream>>>(G, j, dst, tmp);
            FEWHA_LAUNCHED();
            k_fwd_cols<T><<<grid_layers(m * m), 256, 0, stream>>>(G, j, tmp, dst);
            FEWHA_LAUNCHED();
        }
        return FEWHA_OK;
    }

    // LGS tip-tilt filter on weighted slopes (no-op without filtered sensors)
    int tt_filter(T* sl) {
        if (!G.any_tt) return FEWHA_OK;
        if (nb != 1) {
            err = "the LGS tip-tilt filter runs on single frames";
            return FEWHA_ERR_STATE;
        }
        k_tt_sums<T><<<dim3(G.G, 2), 256, 0, stream>>>(G, sl, ttsums);
        FEWHA_LAUNCHED();
        k_tt_apply<T><<<dim3((G.nsmax * G.nsmax + 255) / 256, G.G), 256, 0, stream>>>(G, ttsums, sl);
        FEWHA_LAUNCHED();
        return FEWHA_OK;
    }

    int backproject(const T* weighted_slopes, T* out) {   // out = W P^T Gamma^T sl
        int np1 = G.nsmax + 1;
        k_gammaT<T><<<dim3((np1 * np1 + 255) / 256, G.G, nb), 256, 0, stream>>>(G, weighted_slopes, wpsi2);
        FEWHA_LAUNCHED();
        k_PT<T><<<grid_layers(G.nmax * G.nmax), 256, 0, stream>>>(G, wpsi2, y);
        FEWHA_LAUNCHED();
        return fwd_dwt(y, out);
    }

    int data_term(const T* x, T* out) {   // out = W P^T Gamma^T C^{-1} Gamma P W^T x
        TRY(inv_dwt(x, phi));
        int np1 = G.nsmax + 1;
        k_P<T><<<dim3((np1 * np1 + 255) / 256, G.G, nb), 256, 0, stream>>>(G, phi, wpsi);
        FEWHA_LAUNCHED();
        k_gamma_w<T><<<dim3((G.nsmax * G.nsmax + 255) / 256, G.G, nb), 256, 0, stream>>>(G, wpsi, wsl);
        FEWHA_LAUNCHED();
        TRY(tt_filter(wsl));
        return backproject(wsl, out);
    }

    int rhs_and_restart(int warm) {
        k_weight_meas<T><<<dim3((G.nsmax * G.nsmax + 255) / 256, G.G), 256, 0, stream>>>(G, slopes, wsl, errw);
        FEWHA_LAUNCHED();
        TRY(tt_filter(wsl));
        TRY(backproject(wsl, b));
        if (!warm) {
            k_cold<T><<<kRedBlocks, kRedThreads, 0, stream>>>(G.N, b, bprev, r, c);
            FEWHA_LAUNCHED();
        } else if (k_rr > 0 && frame_count > 0 && frame_count % k_rr == 0) {
            TRY(inv_dwt(c, phi));
            const int np1 = G.nsmax + 1;
            k_P<T><<<dim3((np1 * np1 + 255) / 256, G.G), 256, 0, stream>>>(G, phi, wpsi);
            FEWHA_LAUNCHED();
            k_resid_w<T><<<dim3((G.nsmax * G.nsmax + 255) / 256, G.G), 256, 0, stream>>>(G, slopes, wpsi, wsl);
            FEWHA_LAUNCHED();
            TRY(tt_filter(wsl));
            TRY(backproject(wsl, ext));
            k_replace<T><<<kRedBlocks, kRedThreads, 0, stream>>>(G.N, b, ext, aD, c, bprev, r);
            FEWHA_LAUNCHED();
        } else {
            k_warm<T><<<kRedBlocks, kRedThreads, 0, stream>>>(G.N, b, bprev, r);
            FEWHA_LAUNCHED();
        }
        return FEWHA_OK;
    }

    int apply_M_dev(const T* x, T* out) {
        TRY(data_term(x, out));
        k_reg_dot<T><<<dim3(kRedBlocks, 1, nb), kRedThreads, 0, stream>>>(G.N, aD, x, out, part2);
        FEWHA_LAUNCHED();
        return FEWHA_OK;
    }

    int pcg_plain(int n_iter) {
        for (int k = 0; k < n_iter; ++k) {
            k_precond_dot<T><<<kRedBlocks, kRedThreads, 0, stream>>>(G.N, Jinv, r, z, part);
            FEWHA_LAUNCHED();
            TRY(data_term(z, s));
            k_reg_dot<T><<<kRedBlocks, kRedThreads, 0, stream>>>(G.N, aD, z, s, part2);
            FEWHA_LAUNCHED();
            k_alg2_scalars<<<1, 256, 0, stream>>>(part, part2, sc, k, errw);
            FEWHA_LAUNCHED();
            k_alg2_update<T><<<kRedBlocks, kRedThreads, 0, stream>>>(G.N, sc, k == 0, z, s, p, q, c, r);
            FEWHA_LAUNCHED();
        }
        return FEWHA_OK;
    }

    int fit_dev(double gain, int n_fit) {
        if (hs.M == 0) {
            err = "the geometry has no deformable mirrors";
            return FEWHA_ERR_STATE;
        }
        // phi = W^T c (the fused kernel has just written it)
        if (!(use_fused() && fused_layers_ready)) TRY(inv_dwt(c, phi));
        if (F.colocated) {
            int amax = 0;
            for (auto& d : hs.dm) amax = std::max(amax, d.na);
            k_fit_colocated<T><<<dim3((amax * amax + 255) / 256, F.M), 256, 0, stream>>>(F, phi, afit);
            FEWHA_LAUNCHED();
            return gain_enqueue(gain);
        }
        if constexpr (std::is_same<T, float>::value) {
            if (fitcg && use_fused()) {
                FitCgBuffers fb{fv, afit, fr, fp, fu, fq, acur, aprev, fpart, fbar, errw};
                return fitcg_launch(fitcg, F, phi, fb, n_fit, (float)gain, closed ? 1 : 0, barrier_budget, stream,
                                    err, launches);
            }
        }
        int np1 = F.np1;
        dim3 gdir((np1 * np1 + 255) / 256, F.T_);
        int amax = 0;
        for (auto& d : hs.dm) amax = std::max(amax, d.na);
        dim3 gact((amax * amax + 255) / 256, F.M);
        k_fit_lay<T><<<gdir, 256, 0, stream>>>(F, phi, fv);
        FEWHA_LAUNCHED();
        k_fit_dmT<T><<<gact, 256, 0, stream>>>(F, fv, nullptr, (T)0, frhs);
        FEWHA_LAUNCHED();
        // r = rhs - A x ; p = r ; rr = (r, r)
        k_fit_dm<T><<<gdir, 256, 0, stream>>>(F, afit, fv);
        FEWHA_LAUNCHED();
        k_fit_dmT<T><<<gact, 256, 0, stream>>>(F, fv, afit, F.eps, fq);
        FEWHA_LAUNCHED();
        k_fit_init<T><<<kRedBlocks, kRedThreads, 0, stream>>>(F.NA, frhs, fq, fr, fp);
        FEWHA_LAUNCHED();
        k_dot<T><<<kRedBlocks, kRedThreads, 0, stream>>>(F.NA, fr, fr, part);
        FEWHA_LAUNCHED();
        k_fit_scalar<<<1, 256, 0, stream>>>(part, sc, 0);
        FEWHA_LAUNCHED();
        for (int it = 0; it < n_fit; ++it) {
            k_fit_dm<T><<<gdir, 256, 0, stream>>>(F, fp, fv);
            FEWHA_LAUNCHED();
            k_fit_dmT<T><<<gact, 256, 0, stream>>>(F, fv, fp, F.eps, fq);
            FEWHA_LAUNCHED();
            k_dot<T><<<kRedBlocks, kRedThreads, 0, stream>>>(F.NA, fp, fq, part);
            FEWHA_LAUNCHED();
            k_fit_scalar<<<1, 256, 0, stream>>>(part, sc, 1);
            FEWHA_LAUNCHED();
            k_fit_step<T><<<kRedBlocks, kRedThreads, 0, stream>>>(F.NA, sc, afit, fr, fp, fq, part);
            FEWHA_LAUNCHED();
            k_fit_scalar<<<1, 256, 0, stream>>>(part, sc, 2);
            FEWHA_LAUNCHED();
            k_fit_dir<T><<<kRedBlocks, kRedThreads, 0, stream>>>(F.NA, sc, fr, fp);
            FEWHA_LAUNCHED();
        }
        return gain_enqueue(gain);
    }

    int gain_enqueue(double gain) {
        if (closed) k_gain_closed<T><<<kRedBlocks, kRedThreads, 0, stream>>>(F.NA, (T)gain, afit, acur, aprev);
        else k_gain<T><<<kRedBlocks, kRedThreads, 0, stream>>>(F.NA, (T)gain, afit, acur, aprev);
        FEWHA_LAUNCHED();
        return FEWHA_OK;
    }

    // ---- copies ----
    int copy_in(T* dst, const void* src, size_t count, int on_device) {
        if (!src) {
            err = "null input pointer";
            return FEWHA_ERR_ARG;
        }
        FEWHA_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T),
                                   on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream));
        if (!on_device) FEWHA_CUDA(cudaStreamSynchronize(stream));
        return FEWHA_OK;
    }
    int copy_out(void* dst, const T* src, size_t count, int on_device) {
        if (!dst) {
            err = "null output pointer";
            return FEWHA_ERR_ARG;
        }
        FEWHA_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T),
                                   on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
        if (!on_device) FEWHA_CUDA(cudaStreamSynchronize(stream));
        return FEWHA_OK;
    }

    // ---- SolverBase ----
    int set_frame(const void* sl, int on_device) override {
        TRY(copy_in(slopes, sl, hs.S, on_device));
        have_frame = true;
        pol_pending = true;
        return FEWHA_OK;
    }

    bool use_fused() const { return path == FEWHA_PATH_FUSED && fused != nullptr; }

    // closed loop: s += Gamma P_DM a_{-1}, once per frame (Alg. 1)
    int pol_enqueue() {
        if (!closed || !pol_pending) return FEWHA_OK;
        const int np1 = G.nsmax + 1;
        k_dm_wfs<T><<<dim3((np1 * np1 + 255) / 256, G.G), 256, 0, stream>>>(G, F, aprev, wpsi);
        FEWHA_LAUNCHED();
        k_add_gamma<T><<<dim3((G.nsmax * G.nsmax + 255) / 256, G.G), 256, 0, stream>>>(G, wpsi, slopes);
        FEWHA_LAUNCHED();
        pol_pending = false;
        return FEWHA_OK;
    }

    // host frames on the fused path: slopes by a copy-engine transfer (1) or
    // read by the kernel through the pinned buffer's mapping (0)
    bool host_slopes_copy = true;

    int set_host_transfer(int slopes_by_copy) override {
        host_slopes_copy = slopes_by_copy != 0;
        drop_graphs();
        return FEWHA_OK;
    }

    int set_loop(int c) override {
        if (c && hs.M == 0) {
            err = "the closed loop needs deformable mirrors";
            return FEWHA_ERR_STATE;
        }
        if (c && hs.moao) {
            err = "MOAO mirrors are not seen by the sensors: open loop only";
            return FEWHA_ERR_STATE;
        }
        if (c && !hs.closed_ok) {
            err = "a sensor sees beyond a mirror grid (mirrors are sized for the fitting directions)";
            return FEWHA_ERR_GEOMETRY;
        }
        closed = c != 0;
        drop_graphs();
        return FEWHA_OK;
    }

    int solve_enqueue(int n_iter, int warm) {
        TRY(pol_enqueue());
        if (use_fused()) {
            bool replace = warm && k_rr > 0 && frame_count > 0 && frame_count % k_rr == 0;
            int st = fused_solve(fused, ov_slopes, n_iter, warm, replace ? 1 : 0, barrier_budget, stream, err,
                                 launches, ov_layers, ov_done, ov_bell, ov_bell_want, ov_bell_ns);
            if (st) return st;
            fused_layers_ready = true;
        } else {
            TRY(rhs_and_restart(warm));
            TRY(pcg_plain(n_iter));
            fused_layers_ready = false;
        }
        frame_count += 1;
        return FEWHA_OK;
    }

    int solve(int n_iter, int warm) override {
        if (n_iter < 1 || n_iter > 100000) {
            err = "n_iter must be >= 1";
            return FEWHA_ERR_ARG;
        }
        if (!have_frame) {
            err = "fewha_solve before fewha_set_frame";
            return FEWHA_ERR_STATE;
        }
        return solve_enqueue(n_iter, warm);
    }

    int fit(double gain, int n_fit, void* out, int on_device) override {
        if (n_fit < 0 || !(gain >= 0.0 && gain <= 1.0)) {
            err = "gain must be in [0, 1] and n_fit >= 0";
            return FEWHA_ERR_ARG;
        }
        TRY(fit_dev(gain, n_fit));
        if (out) TRY(copy_out(out, acur, hs.NA, on_device));
        return FEWHA_OK;
    }

    int get_layers(void* out, int on_device) override {
        TRY(layers_enqueue());
        return copy_out(out, phi, hs.N, on_device);
    }

    int get_vector(int which, void* out, int on_device) override {
        const T* src = nullptr;
        switch (which) {
            case 0: src = c; break;
            case 1: src = r; break;
            case 2: src = b; break;
            case 3: src = Jd; break;
            case 4: src = aD; break;
            default: err = "unknown vector"; return FEWHA_ERR_ARG;
        }
        return copy_out(out, src, hs.N, on_device);
    }

    int get_state(void* oc, void* ob, void* orr, int on_device) override {
        if (oc) TRY(copy_out(oc, c, hs.N, on_device));
        if (ob) TRY(copy_out(ob, bprev, hs.N, on_device));
        if (orr) TRY(copy_out(orr, r, hs.N, on_device));
        return FEWHA_OK;
    }

    int set_state(const void* ic, const void* ib, const void* ir, int on_device, long count) override {
        if (!ic || !ib || !ir) {
            err = "set_state needs c, b and r";
            return FEWHA_ERR_ARG;
        }
        TRY(copy_in(c, ic, hs.N, on_device));
        TRY(copy_in(bprev, ib, hs.N, on_device));
        TRY(copy_in(r, ir, hs.N, on_device));
        frame_count = count;
        fused_layers_ready = false;
        return FEWHA_OK;
    }

    int apply_M(const void* x, void* yout, int on_device) override {
        fused_layers_ready = false;   // phi is scratch of the operator
        TRY(copy_in(z, x, hs.N, on_device));
        TRY(apply_M_dev(z, s));
        return copy_out(yout, s, hs.N, on_device);
    }

    // ---- single operators (plain kernels): W, W^T, P, P^T, Gamma, Gamma^T ----
    int operator_dims(int op, long& n_in, long& n_out) override {
        const long N = hs.N, NW = hs.NW, S = hs.S;
        switch (op) {
            case FEWHA_OP_W: case FEWHA_OP_WT: n_in = N; n_out = N; return FEWHA_OK;
            case FEWHA_OP_P: n_in = N; n_out = NW; return FEWHA_OK;
            case FEWHA_OP_PT: n_in = NW; n_out = N; return FEWHA_OK;
            case FEWHA_OP_GAMMA: n_in = NW; n_out = S; return FEWHA_OK;
            case FEWHA_OP_GAMMA_T: n_in = S; n_out = NW; return FEWHA_OK;
            default: err = "unknown operator"; return FEWHA_ERR_ARG;
        }
    }

    // input buffer of op, and the enqueue of op from it into its output buffer
    T* op_in(int op) {
        switch (op) {
            case FEWHA_OP_W: case FEWHA_OP_WT: return z;
            case FEWHA_OP_P: return y;
            case FEWHA_OP_PT: return wpsi2;
            case FEWHA_OP_GAMMA: return wpsi;
            default: return wsl;
        }
    }
    T* op_out(int op) {
        switch (op) {
            case FEWHA_OP_W: case FEWHA_OP_WT: return s;
            case FEWHA_OP_P: return wpsi;
            case FEWHA_OP_PT: return ext;
            case FEWHA_OP_GAMMA: return wsl;
            default: return wpsi2;
        }
    }
    int op_enqueue(int op) {
        const int np1 = G.nsmax + 1;
        const dim3 gn((np1 * np1 + 255) / 256, G.G), gs((G.nsmax * G.nsmax + 255) / 256, G.G);
        switch (op) {
            case FEWHA_OP_W: return fwd_dwt(z, s);
            case FEWHA_OP_WT: return inv_dwt(z, s);
            case FEWHA_OP_P:
                k_P<T><<<gn, 256, 0, stream>>>(G, y, wpsi);
                break;
            case FEWHA_OP_PT:
                k_PT<T><<<grid_layers(G.nmax * G.nmax), 256, 0, stream>>>(G, wpsi2, ext);
                break;
            case FEWHA_OP_GAMMA:
                FEWHA_CUDA(cudaMemsetAsync(wsl, 0, hs.S * sizeof(T), stream));
                k_add_gamma<T><<<gs, 256, 0, stream>>>(G, wpsi, wsl);
                break;
            default:
                k_gammaT<T><<<gn, 256, 0, stream>>>(G, wsl, wpsi2);
                break;
        }
        FEWHA_LAUNCHED();
        return FEWHA_OK;
    }

    int apply_operator(int op, const void* x, void* yout, int on_device) override {
        long nin = 0, nout = 0;
        TRY(operator_dims(op, nin, nout));
        fused_layers_ready = false;   // the operators' buffers are the plain path's scratch
        TRY(copy_in(op_in(op), x, nin, on_device));
        TRY(op_enqueue(op));
        return copy_out(yout, op_out(op), nout, on_device);
    }

    int time_operator(int op, int reps, double* us) override {
        long nin = 0, nout = 0;
        TRY(operator_dims(op, nin, nout));
        if (reps < 1 || !us) {
            err = "reps must be >= 1 and us not NULL";
            return FEWHA_ERR_ARG;
        }
        fused_layers_ready = false;
        FEWHA_CUDA(cudaMemsetAsync(op_in(op), 0, nin * sizeof(T), stream));
        TRY(op_enqueue(op));   // warm-up
        cudaEvent_t e0, e1;
        FEWHA_CUDA(cudaEventCreate(&e0));
        FEWHA_CUDA(cudaEventCreate(&e1));
        cudaEventRecord(e0, stream);
        for (int i = 0; i < reps; ++i) TRY(op_enqueue(op));
        cudaEventRecord(e1, stream);
        FEWHA_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *us = 1e3 * (double)ms / reps;
        return check_err();
    }

    int check_err() {
        FEWHA_CUDA(cudaMemcpyAsync(errw_host, errw, sizeof(int), cudaMemcpyDeviceToHost, stream));
        FEWHA_CUDA(cudaStreamSynchronize(stream));
        return decode_err(*errw_host);
    }

    // status of a device error word read back (the word is cleared if set)
    int decode_err(int e) {
        if (e) {
            if (fused) fused_mark_dirty(fused);
            fitcg_mark_dirty(fitcg);
            drop_graphs();   // captured frames would skip the counter reset the next launch needs
            FEWHA_CUDA(cudaMemsetAsync(errw, 0, sizeof(int), stream));
            FEWHA_CUDA(cudaStreamSynchronize(stream));
            if (e & kErrLaunch) {
                err = "the fused kernel was launched with a grid or cluster shape it was not planned for";
                return FEWHA_ERR_LAUNCH;
            }
            if (e & kErrTimeout) {
                err = "a grid barrier of the fused kernel expired";
                return FEWHA_ERR_TIMEOUT;
            }
            if (e & kErrInput) {
                err = "non-finite slopes in active subapertures";
                return FEWHA_ERR_INPUT;
            }
            if (e & kErrBreakdown) {
                err = "PCG breakdown (step denominator <= 0 or non-finite)";
                return FEWHA_ERR_BREAKDOWN;
            }
        }
        return FEWHA_OK;
    }

    int sync() override {
        FEWHA_CUDA(cudaStreamSynchronize(stream));
        return check_err();
    }

    int describe(char* buf, int len) override {
        if (!buf || len <= 0) {
            err = "null buffer";
            return FEWHA_ERR_ARG;
        }
        int k = snprintf(buf, len, "precision %s, path %s, N %ld, S %ld, A %ld; ", sizeof(T) == 8 ? "fp64" : "fp32",
                         use_fused() ? "fused" : "plain", hs.N, hs.S, hs.NA);
        if (fused && k >= 0 && k < len) fused_describe(fused, buf + k, len - k);
        const int used = (int)strnlen(buf, len);
        if (fitcg && use_fused() && used + 1 < len)
            snprintf(buf + used, len - used, "; fit: one launch, normal matrix %ld non-zeros", fitcg_nnz(fitcg));
        return FEWHA_OK;
    }

    int set_trace(int on) override {
        if (!fused) {
            err = "tracing is available on the fused path only";
            return FEWHA_ERR_STATE;
        }
        fused_set_trace(fused, on != 0);
        return FEWHA_OK;
    }

    int get_trace(unsigned long long* out, int max_entries, int* slots, int* grid) override {
        if (!fused) {
            err = "tracing is available on the fused path only";
            return FEWHA_ERR_STATE;
        }
        FEWHA_CUDA(cudaStreamSynchronize(stream));
        if (fused_get_trace(fused, out, max_entries, slots, grid)) {
            err = "trace copy failed";
            return FEWHA_ERR_CUDA;
        }
        return FEWHA_OK;
    }

    int get_fine_trace(unsigned long long* out, int max_entries, int* per_cta, int* grid) override {
        if (!fused) {
            err = "tracing is available on the fused path only";
            return FEWHA_ERR_STATE;
        }
        FEWHA_CUDA(cudaStreamSynchronize(stream));
        if (fused_get_fine_trace(fused, out, max_entries, per_cta, grid)) {
            err = "trace copy failed";
            return FEWHA_ERR_CUDA;
        }
        return FEWHA_OK;
    }

    // layer-phase form of the fused plan: -1 automatic, 0 row stripes, 1 level-stacked
    int layer_form = -1;

    // a fused plan with cluster size C (FP32 instances only)
    FusedPlan* make_plan(int C, std::string& e, int form = -2) {
        if constexpr (std::is_same<T, float>::value) {
            return fused_create_multi({&hs}, {G}, {fbuf}, 0, e, C, form == -2 ? layer_form : form);
        } else {
            e = "the fused path is FP32 only";
            return nullptr;
        }
    }

    // captured frame graphs hold the old plan's launch: drop them
    void drop_graphs() {
        for (int i = 0; i < 2; ++i) drop_graph(i);
    }

    int set_layer_transform(int form) override {
        if (sizeof(T) != 4) {
            err = "the fused path is FP32 only";
            return FEWHA_ERR_STATE;
        }
        std::string e;
        FusedPlan* pl = make_plan(fused ? fused_cluster_size(fused) : 0, e, form);
        if (!pl && fused) pl = make_plan(0, e, form);
        if (!pl) {
            err = "no fused plan with this layer transform: " + e;
            return FEWHA_ERR_ARG;
        }
        layer_form = form;
        FEWHA_CUDA(cudaStreamSynchronize(stream));
        if (fused) fused_destroy(fused);
        fused = pl;
        drop_graphs();
        return FEWHA_OK;
    }

    int set_cluster_size(int C) override {
        if (sizeof(T) != 4) {
            err = "the fused path is FP32 only";
            return FEWHA_ERR_STATE;
        }
        std::string e;
        FusedPlan* pl = make_plan(C, e);
        if (!pl) {
            err = "no fused plan with this cluster size: " + e;
            return FEWHA_ERR_ARG;
        }
        FEWHA_CUDA(cudaStreamSynchronize(stream));
        if (fused) fused_destroy(fused);
        fused = pl;
        drop_graphs();
        return FEWHA_OK;
    }

    // Time every feasible cluster shape on the current frame (warm start from
    // the current state, restored before each trial and at the end) and keep
    // the fastest plan.
    int autotune(int n_iter, int reps, char* report, int len) override {
        if (sizeof(T) != 4 || !fused) {
            err = "the autotuner needs the fused FP32 path";
            return FEWHA_ERR_STATE;
        }
        if (!have_frame) {
            err = "autotune needs a frame (fewha_set_frame) to time";
            return FEWHA_ERR_STATE;
        }
        if (n_iter < 1 || reps < 1) {
            err = "n_iter and reps must be >= 1";
            return FEWHA_ERR_ARG;
        }
        const size_t nb = (size_t)hs.N * sizeof(T);
        T* saved = nullptr;
        FEWHA_CUDA(cudaMalloc(&saved, 4 * nb));
        T* vec[4] = {c, r, b, bprev};
        for (int i = 0; i < 4; ++i)
            FEWHA_CUDA(cudaMemcpyAsync((char*)saved + i * nb, vec[i], nb, cudaMemcpyDeviceToDevice, stream));
        auto restore = [&]() {
            for (int i = 0; i < 4; ++i)
                cudaMemcpyAsync(vec[i], (char*)saved + i * nb, nb, cudaMemcpyDeviceToDevice, stream);
        };
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        auto time_plan = [&](FusedPlan* pl) -> float {
            std::vector<float> t;
            for (int rep = 0; rep < reps + 1; ++rep) {
                restore();
                cudaEventRecord(e0, stream);
                std::string e;
                long long dummy = 0;
                if (fused_solve(pl, nullptr, n_iter, 1, 0, barrier_budget, stream, e, dummy)) return -1.f;
                cudaEventRecord(e1, stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) t.push_back(ms);
            }
            if (check_err() != FEWHA_OK) return -1.f;
            std::sort(t.begin(), t.end());
            return t[t.size() / 2];
        };
        std::string rep_s;
        char buf[96];
        FusedPlan* best = fused;
        float best_t = time_plan(fused);
        const int C0 = fused_cluster_size(fused), V0 = fused_layer_form(fused);
        snprintf(buf, sizeof buf, "C=%d V=%d: %.1f us (current)", C0, V0, best_t * 1e3f);
        rep_s += buf;
        for (int C : {16, 8, 4, 2})
          for (int V : {1, 0}) {
            if (C == C0 && V == V0) continue;
            if (layer_form >= 0 && V != layer_form) continue;
            std::string e;
            FusedPlan* pl = make_plan(C, e, V);
            if (!pl || fused_cluster_size(pl) != C || fused_layer_form(pl) != V) {
                if (pl) fused_destroy(pl);
                continue;
            }
            const float t = time_plan(pl);
            snprintf(buf, sizeof buf, "; C=%d V=%d: %.1f us", C, V, t * 1e3f);
            rep_s += buf;
            if (t > 0.f && (best_t <= 0.f || t < best_t)) {
                if (best != fused) fused_destroy(best);
                best = pl;
                best_t = t;
            } else {
                fused_destroy(pl);
            }
        }
        restore();
        cudaStreamSynchronize(stream);
        cudaFree(saved);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (best != fused) {
            fused_destroy(fused);
            fused = best;
            drop_graphs();
        }
        snprintf(buf, sizeof buf, "; chosen C=%d V=%d", fused_cluster_size(fused), fused_layer_form(fused));
        rep_s += buf;
        if (report && len > 0) snprintf(report, len, "%s", rep_s.c_str());
        return FEWHA_OK;
    }

    // ---- differentiation: set_params, taped solve, reverse mode ----
    // Work of up to adj_cap frames differentiated together (one solve is a
    // batch of 1): forward iterates and adjoint vectors, their partials and
    // scalars, and frame-batched copies of the operator chain's scratch
    // (phi, wpsi, wpsi2, wsl, y, tmp, part, part2) that stand in for the
    // single-frame buffers while a batch runs.
    T *ac = nullptr, *ar = nullptr, *ap = nullptr, *aq = nullptr, *ab = nullptr;   // forward work
    T *cb = nullptr, *rb = nullptr, *pb = nullptr, *qb = nullptr, *sb = nullptr, *My = nullptr, *psiz = nullptr;
    T *bphi = nullptr, *bwpsi = nullptr, *bwpsi2 = nullptr, *bwsl = nullptr, *by = nullptr, *btmp = nullptr;
    double *tsc = nullptr, *asc = nullptr, *apart = nullptr, *alpart = nullptr, *awpart = nullptr, *gam = nullptr;
    double *bpart = nullptr, *bpart2 = nullptr;
    int adj_cap = 0;

    template <typename U>
    void release(U*& ptr) {
        if (!ptr) return;
        cudaFree(ptr);
        allocs.erase(std::remove(allocs.begin(), allocs.end(), (void*)ptr), allocs.end());
        ptr = nullptr;
    }

    int adj_init(int B) {
        if (!gam) {
            std::vector<double> g(hs.L);
            for (int l = 0; l < hs.L; ++l) g[l] = hs.lay[l].cn2;
            TRY(upload(gam, g));
        }
        if (adj_cap >= B) return FEWHA_OK;
        FEWHA_CUDA(cudaStreamSynchronize(stream));   // the smaller buffers may still be in use
        for (T** v : {&ac, &ar, &ap, &aq, &ab, &cb, &rb, &pb, &qb, &sb, &My, &psiz, &bphi, &bwpsi, &bwpsi2, &bwsl, &by,
                      &btmp})
            release(*v);
        for (double** v : {&tsc, &asc, &apart, &alpart, &awpart, &bpart, &bpart2}) release(*v);
        adj_cap = 0;
        const size_t N = (size_t)hs.N * B, NW = (size_t)hs.NW * B, S = (size_t)hs.S * B;
        for (T** v : {&ac, &ar, &ap, &aq, &ab, &cb, &rb, &pb, &qb, &sb, &My, &bphi, &by, &btmp}) TRY(alloc(*v, N));
        for (T** v : {&psiz, &bwpsi, &bwpsi2}) TRY(alloc(*v, NW));
        TRY(alloc(bwsl, S));
        TRY(alloc(tsc, (size_t)kNumScalars * B));
        TRY(alloc(asc, (size_t)8 * B));
        TRY(alloc(apart, (size_t)6 * kRedBlocks * B));
        TRY(alloc(alpart, (size_t)hs.L * kRedBlocks * B));
        TRY(alloc(awpart, (size_t)hs.G * kRedBlocks * B));
        TRY(alloc(bpart, (size_t)kRedBlocks * B));
        TRY(alloc(bpart2, (size_t)kRedBlocks * B));
        FEWHA_CUDA(cudaMemset(tsc, 0, (size_t)kNumScalars * B * sizeof(double)));
        adj_cap = B;
        return FEWHA_OK;
    }

    // The operator chain on B frames: the batch scratch swapped in, nb = B.
    struct FrameBatch {
        Solver* sv;
        T *phi, *wpsi, *wpsi2, *wsl, *y, *tmp;
        double *part, *part2;
        FrameBatch(Solver* s_, int B)
            : sv(s_), phi(s_->phi), wpsi(s_->wpsi), wpsi2(s_->wpsi2), wsl(s_->wsl), y(s_->y), tmp(s_->tmp),
              part(s_->part), part2(s_->part2) {
            sv->nb = B;
            sv->phi = sv->bphi;
            sv->wpsi = sv->bwpsi;
            sv->wpsi2 = sv->bwpsi2;
            sv->wsl = sv->bwsl;
            sv->y = sv->by;
            sv->tmp = sv->btmp;
            sv->part = sv->bpart;
            sv->part2 = sv->bpart2;
        }
        ~FrameBatch() {
            sv->nb = 1;
            sv->phi = phi;
            sv->wpsi = wpsi;
            sv->wpsi2 = wpsi2;
            sv->wsl = wsl;
            sv->y = y;
            sv->tmp = tmp;
            sv->part = part;
            sv->part2 = part2;
        }
    };

    size_t tape_size(int n_iter) const override { return tape_bytes(hs.N, n_iter, sizeof(T)); }
    size_t tape_size_batch(int n_iter, int B) const override { return tape_bytes(hs.N, n_iter, sizeof(T), B); }

    // New gamma_l, alpha, w_g for M and b; the Jacobi preconditioner keeps
    // the values of create (it is a constant of the differentiated solve).
    int set_params(const double* cn2, double alpha, const double* w) override {
        if (!cn2 || !w || !(alpha > 0) || !std::isfinite(alpha)) {
            err = "set_params needs cn2 and w arrays and a finite alpha > 0";
            return FEWHA_ERR_ARG;
        }
        for (int l = 0; l < hs.L; ++l)
            if (!(cn2[l] > 0) || !std::isfinite(cn2[l])) {
                err = "every Cn^2 fraction must be finite and > 0";
                return FEWHA_ERR_ARG;
            }
        for (int g = 0; g < hs.G; ++g)
            if (!(w[g] >= 0) || !std::isfinite(w[g])) {
                err = "every sensor weight must be finite and >= 0";
                return FEWHA_ERR_ARG;
            }
        hs.alpha = alpha;
        for (int l = 0; l < hs.L; ++l) {
            HostLayer& L = hs.lay[l];
            L.cn2 = cn2[l];
            for (long i = L.off; i < L.off + (long)L.n * L.n; ++i) {
                hs.Dreg[i] = reg_diag(hs.r0, L.cn2, L.delta, hs.level[i]);
                hs.aD[i] = alpha * hs.Dreg[i];
            }
        }
        std::vector<double> wv(hs.G);
        for (int g = 0; g < hs.G; ++g) wv[g] = hs.wfs[g].w = w[g];
        std::vector<T> t, tw;
        to_T(hs.aD, t);
        to_T(wv, tw);
        FEWHA_CUDA(cudaStreamSynchronize(stream));
        FEWHA_CUDA(cudaMemcpy(aD, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice));
        FEWHA_CUDA(cudaMemcpy((T*)G.wfs_w, tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice));
        if (gam) FEWHA_CUDA(cudaMemcpy(gam, cn2, hs.L * sizeof(double), cudaMemcpyHostToDevice));
        return FEWHA_OK;
    }

    // K steps of Alg. 2 from c = 0, r = b(slopes) for each of B frames
    // (slopes [B][S], layers [B][N]), every iterate on the tape (layout in
    // adjoint.cuh); the frames run together, each kernel of the chain taking
    // all of them.  The frame state (c, r, b of fewha_solve) is not touched.
    int solve_taped(const void* sl, int n_iter, void* tape, void* lout) override {
        return solve_taped_batch(1, sl, n_iter, tape, lout);
    }

    int solve_taped_batch(int B, const void* sl, int n_iter, void* tape, void* lout) override {
        if (G.any_tt) {
            err = "differentiation does not model the LGS tip-tilt filter";
            return FEWHA_ERR_STATE;
        }
        if (!sl || !tape || B < 1 || B > 65535 || n_iter < 1 || n_iter > 100000) {
            err = "solve_taped needs slopes, a tape, 1 <= frames <= 65535 and n_iter >= 1";
            return FEWHA_ERR_ARG;
        }
        TRY(adj_init(B));
        fused_layers_ready = false;   // phi is scratch of the operators below
        FrameBatch fb(this, B);
        const long N = hs.N;
        const size_t NB = (size_t)N * B;
        T* tv = (T*)tape;
        double* ts = (double*)((char*)tape + tape_vec_bytes(N, n_iter, sizeof(T), B));
        const dim3 red(kRedBlocks, 1, B);
        k_weight_meas<T><<<dim3((G.nsmax * G.nsmax + 255) / 256, G.G, B), 256, 0, stream>>>(G, (const T*)sl, wsl,
                                                                                            errw);
        FEWHA_LAUNCHED();
        TRY(backproject(wsl, ab));
        FEWHA_CUDA(cudaMemsetAsync(ac, 0, NB * sizeof(T), stream));
        FEWHA_CUDA(cudaMemcpyAsync(ar, ab, NB * sizeof(T), cudaMemcpyDeviceToDevice, stream));
        for (int k = 0; k < n_iter; ++k) {
            T* v = tv + (size_t)k * kTapeVecs * NB;
            T *rk = v + kTapeR * NB, *zk = v + kTapeZ * NB, *sk = v + kTapeS * NB;
            FEWHA_CUDA(cudaMemcpyAsync(rk, ar, NB * sizeof(T), cudaMemcpyDeviceToDevice, stream));
            k_precond_dot<T><<<red, kRedThreads, 0, stream>>>(N, Jinv, ar, zk, part);
            FEWHA_LAUNCHED();
            TRY(data_term(zk, sk));
            k_reg_dot<T><<<red, kRedThreads, 0, stream>>>(N, aD, zk, sk, part2);
            FEWHA_LAUNCHED();
            k_alg2_scalars<<<B, 256, 0, stream>>>(part, part2, tsc, k, errw);
            FEWHA_LAUNCHED();
            k_alg2_update<T><<<red, kRedThreads, 0, stream>>>(N, tsc, k == 0, zk, sk, ap, aq, ac, ar);
            FEWHA_LAUNCHED();
            FEWHA_CUDA(cudaMemcpyAsync(v + kTapeP * NB, ap, NB * sizeof(T), cudaMemcpyDeviceToDevice, stream));
            FEWHA_CUDA(cudaMemcpyAsync(v + kTapeQ * NB, aq, NB * sizeof(T), cudaMemcpyDeviceToDevice, stream));
            k_tape_scalars<<<B, 32, 0, stream>>>(tsc, ts, k);
            FEWHA_LAUNCHED();
        }
        if (lout) TRY(inv_dwt(ac, (T*)lout));
        return FEWHA_OK;
    }

    // Reverse mode of solve_taped for the layer cotangent layers_bar:
    // gradients with respect to gamma_l, alpha, w_g (device doubles,
    // overwritten) and the slopes (optional).
    int backward(const void* sl, int n_iter, const void* tape, const void* lbar, double* g_gam, double* g_alpha,
                 double* g_w, void* g_s) override {
        return backward_batch(1, sl, n_iter, tape, lbar, g_gam, g_alpha, g_w, g_s);
    }

    // The same for the B frames of solve_taped_batch: layers_bar [B][N]; per
    // frame gradients g_gam [B][L], g_alpha [B], g_w [B][G], g_s [B][S].
    int backward_batch(int B, const void* sl, int n_iter, const void* tape, const void* lbar, double* g_gam,
                       double* g_alpha, double* g_w, void* g_s) override {
        if (G.any_tt) {
            err = "differentiation does not model the LGS tip-tilt filter";
            return FEWHA_ERR_STATE;
        }
        if (!sl || !tape || !lbar || !g_gam || !g_alpha || !g_w || B < 1 || B > 65535 || n_iter < 1 ||
            n_iter > 100000) {
            err = "backward needs slopes, the tape, the layer cotangent, gradient outputs, 1 <= frames <= 65535 "
                  "and n_iter >= 1";
            return FEWHA_ERR_ARG;
        }
        TRY(adj_init(B));
        fused_layers_ready = false;
        FrameBatch fb(this, B);
        const long N = hs.N;
        const size_t NB = (size_t)N * B;
        const T* tv = (const T*)tape;
        const double* ts = (const double*)((const char*)tape + tape_vec_bytes(N, n_iter, sizeof(T), B));
        FEWHA_CUDA(cudaMemsetAsync(g_gam, 0, (size_t)B * hs.L * sizeof(double), stream));
        FEWHA_CUDA(cudaMemsetAsync(g_alpha, 0, (size_t)B * sizeof(double), stream));
        FEWHA_CUDA(cudaMemsetAsync(g_w, 0, (size_t)B * hs.G * sizeof(double), stream));
        FEWHA_CUDA(cudaMemsetAsync(asc, 0, (size_t)B * 8 * sizeof(double), stream));
        for (T* v : {rb, pb, qb}) FEWHA_CUDA(cudaMemsetAsync(v, 0, NB * sizeof(T), stream));
        TRY(fwd_dwt((const T*)lbar, cb));   // phi = W^T c  ->  c-bar = W phi-bar
        const int np1 = G.nsmax + 1;
        const dim3 gnodes((np1 * np1 + 255) / 256, G.G, B);
        const dim3 red(kRedBlocks, 1, B);
        for (int k = n_iter - 1; k >= 0; --k) {
            const T* v = tv + (size_t)k * kTapeVecs * NB;
            const T* vo = k > 0 ? tv + (size_t)(k - 1) * kTapeVecs * NB : nullptr;
            const T *rk = v + kTapeR * NB, *zk = v + kTapeZ * NB, *sk = v + kTapeS * NB;
            k_adj_dots<T><<<red, kRedThreads, 0, stream>>>(N, cb, rb, pb, qb, v + kTapeP * NB, v + kTapeQ * NB,
                                                           vo ? vo + kTapeP * NB : nullptr,
                                                           vo ? vo + kTapeQ * NB : nullptr, apart);
            FEWHA_LAUNCHED();
            k_adj_scalars<<<B, 256, 0, stream>>>(apart, ts, k, asc);
            FEWHA_LAUNCHED();
            k_adj_vec1<T><<<red, kRedThreads, 0, stream>>>(N, asc, cb, rb, pb, qb, zk, sb);
            FEWHA_LAUNCHED();
            TRY(apply_M_dev(sb, My));   // leaves P W^T sb in wpsi
            // sb^T (dM/dtheta) z_k: alpha D part per layer, C^{-1} part per sensor
            k_layer_dot<T><<<dim3(kRedBlocks, G.L, B), kRedThreads, 0, stream>>>(G, sb, aD, zk, alpart);
            FEWHA_LAUNCHED();
            TRY(inv_dwt(zk, phi));
            k_P<T><<<gnodes, 256, 0, stream>>>(G, phi, psiz);
            FEWHA_LAUNCHED();
            k_wfs_dot<T><<<dim3(kRedBlocks, G.G, B), kRedThreads, 0, stream>>>(G, psiz, wpsi, nullptr, awpart);
            FEWHA_LAUNCHED();
            k_adj_accum<<<B, 256, 0, stream>>>(alpart, G.L, awpart, G.G, gam, hs.alpha, g_gam, g_alpha, g_w);
            FEWHA_LAUNCHED();
            k_adj_vec2<T><<<red, kRedThreads, 0, stream>>>(N, asc, pb, qb, rb, zk, sk, rk, My, Jinv);
            FEWHA_LAUNCHED();
        }
        // b-bar = r-bar: b-bar^T (db/dw_g) and the slope gradient C^{-1} Gamma P W^T b-bar
        TRY(inv_dwt(rb, phi));
        k_P<T><<<gnodes, 256, 0, stream>>>(G, phi, psiz);
        FEWHA_LAUNCHED();
        k_wfs_dot<T><<<dim3(kRedBlocks, G.G, B), kRedThreads, 0, stream>>>(G, psiz, nullptr, (const T*)sl, awpart);
        FEWHA_LAUNCHED();
        k_adj_accum<<<B, 256, 0, stream>>>(nullptr, 0, awpart, G.G, gam, hs.alpha, g_gam, g_alpha, g_w);
        FEWHA_LAUNCHED();
        if (g_s) {
            k_gamma_w<T><<<dim3((G.nsmax * G.nsmax + 255) / 256, G.G, B), 256, 0, stream>>>(G, psiz, (T*)g_s);
            FEWHA_LAUNCHED();
        }
        return FEWHA_OK;
    }

    // host-side timing of the last fewha_frame (us): preparation (pointer
    // lookups, graph capture or re-pointing), the graph launch call, the wait
    // for the results, the whole call; then 1 if the kernel node was
    // re-pointed, 1 if the graph was captured
    double ftime[6] = {0, 0, 0, 0, 0, 0};

    int get_frame_timing(double* out) override {
        for (int i = 0; i < 6; ++i) out[i] = ftime[i];
        return FEWHA_OK;
    }

    int frame(const void* s_in, int n_iter, int warm, double gain, int n_fit, void* lout, void* dout,
              int on_device) override {
        using clk = std::chrono::steady_clock;
        const auto T0 = clk::now();
        auto T1 = T0, T2 = T0, T3 = T0;
        auto us = [](clk::time_point a, clk::time_point b) {
            return std::chrono::duration<double, std::micro>(b - a).count();
        };
        struct Stamp {   // fills ftime however the call returns
            double* f;
            clk::time_point t0;
            clk::time_point *t1, *t2, *t3;
            decltype(us)& u;
            ~Stamp() {
                const auto t4 = clk::now();
                f[0] = u(t0, *t1);
                f[1] = u(*t1, *t2);
                f[2] = u(*t2, *t3);
                f[3] = u(t0, t4);
            }
        } stamp{ftime, T0, &T1, &T2, &T3, us};
        ftime[4] = ftime[5] = 0.0;
        if (!s_in) {
            err = "null slopes";
            return FEWHA_ERR_ARG;
        }
        if (n_iter < 1) {
            err = "n_iter must be >= 1";
            return FEWHA_ERR_ARG;
        }
        if (dout && hs.M == 0) {
            err = "the geometry has no deformable mirrors";
            return FEWHA_ERR_STATE;
        }
        // pinned host pointers are captured directly, pageable ones are staged
        const void* sin = s_in;
        void* lo = lout;
        void* dm = dout;
        void* sin_map = on_device ? nullptr : host_dev_ptr(s_in);
        void* lo_map = (on_device || !lout) ? nullptr : host_dev_ptr(lout);
        bool stage_in = false, stage_l = false, stage_d = false;
        if (!on_device) {
            stage_in = !sin_map;
            stage_l = lout && !lo_map;
            stage_d = dout && !host_dev_ptr(dout);
            if (stage_in) {
                if (!pinned_in) FEWHA_CUDA(cudaMallocHost(&pinned_in, hs.S * sizeof(T)));
                std::memcpy(pinned_in, s_in, hs.S * sizeof(T));
                sin = pinned_in;
            }
            if (stage_l) {
                if (!pinned_out) FEWHA_CUDA(cudaMallocHost(&pinned_out, hs.N * sizeof(T)));
                lo = pinned_out;
            }
            if (stage_d) {
                if (!pinned_dm) FEWHA_CUDA(cudaMallocHost(&pinned_dm, std::max<long>(hs.NA, 1) * sizeof(T)));
                dm = pinned_dm;
            }
        }
        // pinned host slopes and layers on the fused path (open loop, no fit,
        // slopes brought in by the copy engine): the frame runs as an armed
        // frame fired at once, so the kernel is launched first and does its
        // set-up while the copy engine brings the slopes in, instead of
        // starting behind the copy
        if (!on_device && !dout && sin_map && lo_map && use_fused() && !closed && done_dev && host_slopes_copy) {
            T1 = clk::now();
            int st = frame_arm(s_in, n_iter, warm, lout, 2.0);
            T2 = T3 = clk::now();
            if (st) return st;
            st = frame_fire();
            T3 = clk::now();
            return st;
        }
        const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        // the fused kernel reads the slopes and writes the layers where they
        // are: device buffers, or pinned host buffers through their device
        // mapping (the transfers happen inside the kernel, no copy nodes) --
        // except host slopes under host_slopes_copy, which one copy-engine
        // transfer brings into the handle's slope buffer first: the kernel's
        // reads across the host link wait a round trip each, the copy streams
        const void* sin_dev = on_device ? sin : (stage_in ? host_dev_ptr(sin) : sin_map);
        void* lo_dev = !lo ? nullptr : on_device ? lo : (stage_l ? host_dev_ptr(lo) : lo_map);
        const bool direct = use_fused() && !closed && sin_dev && (!lo || lo_dev);
        const bool copy_in = direct && !on_device && host_slopes_copy;
        // a host frame that is the fused launch alone reports through the
        // completion word (no error-word copy node, no stream wait)
        const bool use_done = direct && !on_device && !dm && done_dev;
        bool replace = warm && k_rr > 0 && frame_count > 0 && frame_count % k_rr == 0;
        int slot = replace ? 1 : 0;
        Key key;
        key.n_iter = n_iter;
        key.warm = warm;
        key.n_fit = dout ? n_fit : -1;
        key.gain = dout ? gain : -1;
        key.sin = sin;
        key.lout = lo;
        key.dout = dm;
        key.path = path * 2 + (on_device ? 1 : 0);
        key.k_rr = k_rr;
        if (gexec[slot] && !(gkey[slot] == key) && gknode[slot] && direct && gkey[slot].same_work(key) &&
            fused_repoint_node(gexec[slot], gknode[slot], (const float*)sin_dev, (float*)lo_dev) == 0)
        {
            gkey[slot] = key;   // the same frame on other buffers: re-pointed in place
            ftime[4] = 1.0;
        }
        if (!gexec[slot] || !(gkey[slot] == key)) {
            if (stream == 0) {
                err = "fewha_frame needs a non-default stream (graph capture)";
                return FEWHA_ERR_STATE;
            }
            cudaGraph_t graph;
            long long fc = frame_count;
            FEWHA_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
            int st = FEWHA_OK;
            long long l0 = launches;
            do {
                if (!direct || copy_in) {
                    cudaError_t e = cudaMemcpyAsync(slopes, sin, hs.S * sizeof(T), kin, stream);
                    if (e != cudaSuccess) {
                        err = cudaGetErrorString(e);
                        st = FEWHA_ERR_CUDA;
                        break;
                    }
                }
                pol_pending = true;
                ov_slopes = (direct && !copy_in) ? (const float*)sin_dev : nullptr;
                ov_layers = (direct && lo) ? (float*)lo_dev : nullptr;
                ov_done = use_done ? done_dev : nullptr;
                st = solve_enqueue(n_iter, warm);
                ov_slopes = nullptr;
                ov_layers = nullptr;
                ov_done = nullptr;
                if (st) break;
                if (dm && (st = fit_dev(gain, n_fit))) break;
                if (lo && !direct && (st = layers_enqueue())) break;
                if (lo && !direct && cudaMemcpyAsync(lo, phi, hs.N * sizeof(T), kout, stream) != cudaSuccess) {
                    st = FEWHA_ERR_CUDA;
                    err = "copy of layers";
                    break;
                }
                // a host frame reads the device error word back with its results
                if (!on_device && !use_done &&
                    cudaMemcpyAsync(errw_host, errw, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess) {
                    st = FEWHA_ERR_CUDA;
                    err = "copy of the error word";
                    break;
                }
                if (dm && cudaMemcpyAsync(dm, acur, hs.NA * sizeof(T), kout, stream) != cudaSuccess) {
                    st = FEWHA_ERR_CUDA;
                    err = "copy of mirror commands";
                    break;
                }
            } while (0);
            graph = nullptr;
            cudaError_t ec = cudaStreamEndCapture(stream, &graph);
            frame_count = fc;              // the capture only recorded the work
            long long gl = launches - l0;
            launches = l0;
            if (st || ec != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                if (st) return st;
                err = std::string("graph capture: ") + cudaGetErrorString(ec);
                return FEWHA_ERR_CUDA;
            }
            drop_graph(slot);
            cudaError_t ei = cudaGraphInstantiate(&gexec[slot], graph, 0);
            if (ei != cudaSuccess) {
                cudaGraphDestroy(graph);
                err = std::string("graph instantiate: ") + cudaGetErrorString(ei);
                gexec[slot] = nullptr;
                return FEWHA_ERR_CUDA;
            }
            // a direct frame whose graph is the fused launch alone can later be
            // re-pointed at other buffers (kept: the graph and its node)
            gsrc[slot] = graph;
            size_t nn = 0;
            if (direct && cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn == 1) {
                cudaGraphNode_t nd;
                cudaGraphNodeType ty;
                if (cudaGraphGetNodes(graph, &nd, &nn) == cudaSuccess && cudaGraphNodeGetType(nd, &ty) == cudaSuccess &&
                    ty == cudaGraphNodeTypeKernel)
                    gknode[slot] = nd;
            }
            cudaGetLastError();
            gkey[slot] = key;
            graph_launch_count[slot] = gl;
            ftime[5] = 1.0;
        }
        if (use_done) {
            *(volatile unsigned long long*)done_host = 0ull;   // before the launch that sets it
            std::atomic_thread_fence(std::memory_order_seq_cst);
        }
        T1 = clk::now();
        FEWHA_CUDA(cudaGraphLaunch(gexec[slot], stream));
        T2 = T3 = clk::now();
        launches += graph_launch_count[slot];
        frame_count += 1;
        have_frame = true;
        if (on_device) return FEWHA_OK;
        if (use_done) {
            // the kernel's last CTA sets the word after every result is
            // visible here; a launch that never gets there is caught by the
            // stream wait after the deadline
            unsigned long long v = 0ull;
            const auto t0 = std::chrono::steady_clock::now();
            for (long it = 0;; ++it) {
                v = *(volatile unsigned long long*)done_host;
                if (v >> 32) {
                    T3 = clk::now();
                    break;
                }
                if ((it & 1023) == 1023 && std::chrono::steady_clock::now() - t0 > std::chrono::seconds(2)) break;
            }
            if (!(v >> 32)) {
                FEWHA_CUDA(cudaStreamSynchronize(stream));
                v = *(volatile unsigned long long*)done_host;
                if (!(v >> 32)) {
                    FEWHA_CUDA(cudaMemcpy(errw_host, errw, sizeof(int), cudaMemcpyDeviceToHost));
                    v = (unsigned)*errw_host;
                }
            }
            if (stage_l) std::memcpy(lout, pinned_out, hs.N * sizeof(T));
            return decode_err((int)(unsigned)(v & 0xffffffffull));
        }
        FEWHA_CUDA(cudaStreamSynchronize(stream));
        if (stage_l) std::memcpy(lout, pinned_out, hs.N * sizeof(T));
        if (stage_d) std::memcpy(dout, pinned_dm, hs.NA * sizeof(T));
        return decode_err(*errw_host);   // copied by the graph
    }

    // Armed host frame: the fused launch is issued now, does its set-up, and
    // waits (bounded) for frame_fire before it reads the pinned slopes, which
    // the caller fills in between; the kernel reads them and writes the
    // pinned layers through their device mapping, and frame_fire waits on the
    // completion word.  The launch latency is then off the slopes-to-layers path.
    int frame_arm(const void* s_in, int n_iter, int warm, void* lout, double wait_s) override {
        if (armed) {
            err = "a frame is already armed: fire it first";
            return FEWHA_ERR_STATE;
        }
        if (!s_in || !lout || n_iter < 1 || n_iter > 100000 || !(wait_s > 0.0 && wait_s <= 60.0)) {
            err = "frame_arm needs slopes, layers, n_iter >= 1 and 0 < wait_s <= 60";
            return FEWHA_ERR_ARG;
        }
        if (!use_fused() || closed || !done_dev) {
            err = "armed frames run on the fused path in open loop";
            return FEWHA_ERR_STATE;
        }
        void* sdev = host_dev_ptr(s_in);
        void* ldev = host_dev_ptr(lout);
        if (!sdev || !ldev) {
            err = "armed frames need pinned (device-mapped) host slopes and layers";
            return FEWHA_ERR_ARG;
        }
        if (!bell_host) {
            FEWHA_CUDA(cudaHostAlloc((void**)&bell_host, sizeof(unsigned), cudaHostAllocMapped));
            FEWHA_CUDA(cudaHostGetDevicePointer((void**)&bell_dev, bell_host, 0));
            *(volatile unsigned*)bell_host = 0u;
        }
        if (host_slopes_copy && !write_value_tried) {
            write_value_tried = true;
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &fn, 12000, cudaEnableDefault, &q) ==
                    cudaSuccess &&
                q == cudaDriverEntryPointSuccess && fn &&
                cudaStreamCreateWithFlags(&aux_stream, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&prior_done, cudaEventDisableTiming) == cudaSuccess &&
                alloc(go_dev, 1) == FEWHA_OK && cudaMemset(go_dev, 0, sizeof(unsigned)) == cudaSuccess)
                write_value = (WriteValue32)fn;
            cudaGetLastError();
        }
        armed_copy = host_slopes_copy && write_value && go_dev && aux_stream && prior_done;
        // the copy at the fire overwrites the handle's slope buffer: it waits
        // for the work enqueued before this frame (a device frame still
        // running copies its slopes into that buffer)
        if (armed_copy) FEWHA_CUDA(cudaEventRecord(prior_done, stream));
        bell_seq = (bell_seq + 1u) ? bell_seq + 1u : 1u;
        *(volatile unsigned long long*)done_host = 0ull;   // before the launch that sets it
        std::atomic_thread_fence(std::memory_order_seq_cst);
        pol_pending = true;
        ov_slopes = armed_copy ? nullptr : (const float*)sdev;   // copy mode: the handle's slope buffer
        ov_layers = (float*)ldev;
        ov_done = done_dev;
        ov_bell = armed_copy ? go_dev : bell_dev;
        ov_bell_want = bell_seq;
        armed_src = s_in;
        ov_bell_ns = (long long)(wait_s * 1e9);
        const int st = solve_enqueue(n_iter, warm);
        ov_slopes = nullptr;
        ov_layers = nullptr;
        ov_done = nullptr;
        ov_bell = nullptr;
        if (st) return st;
        have_frame = true;
        armed = true;
        armed_wait_s = wait_s;
        return FEWHA_OK;
    }

    bool is_armed() const override { return armed; }

    int frame_fire() override {
        using clk = std::chrono::steady_clock;
        if (!armed) {
            err = "no armed frame";
            return FEWHA_ERR_STATE;
        }
        armed = false;
        const auto t0 = clk::now();
        std::atomic_thread_fence(std::memory_order_seq_cst);   // the caller's slopes before the go
        bool rung = false;
        if (armed_copy) {
            // slopes in by the copy engine, then the go written behind them in stream order
            // (the stream write fences the copy's data before the word)
            if (cudaStreamWaitEvent(aux_stream, prior_done, 0) == cudaSuccess &&
                cudaMemcpyAsync(slopes, armed_src, hs.S * sizeof(T), cudaMemcpyHostToDevice, aux_stream) ==
                    cudaSuccess &&
                write_value((CUstream)aux_stream, (CUdeviceptr)go_dev, bell_seq, 0) == CUDA_SUCCESS)
                rung = true;
            cudaGetLastError();
        }
        if (!rung) {
            // host doorbell: the kernel polls it only in the mapped mode, so in the
            // copy mode a failed transfer leaves the frame to its deadline
            *(volatile unsigned*)bell_host = bell_seq;
        }
        unsigned long long v = 0ull;
        const auto limit = std::chrono::duration<double>(armed_wait_s + 2.0);
        for (long it = 0;; ++it) {
            v = *(volatile unsigned long long*)done_host;
            if (v >> 32) break;
            if ((it & 1023) == 1023 && clk::now() - t0 > limit) break;
        }
        ftime[2] = std::chrono::duration<double, std::micro>(clk::now() - t0).count();
        if (!(v >> 32)) {
            FEWHA_CUDA(cudaStreamSynchronize(stream));
            v = *(volatile unsigned long long*)done_host;
            if (!(v >> 32)) {
                FEWHA_CUDA(cudaMemcpy(errw_host, errw, sizeof(int), cudaMemcpyDeviceToHost));
                v = (unsigned)*errw_host;
            }
        }
        return decode_err((int)(unsigned)(v & 0xffffffffull));
    }

    // device alias of a pinned host pointer (nullptr for other memory)
    void* host_dev_ptr(const void* ptr) {
        if (!ptr) return nullptr;
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
    }

    // phi = W^T c for output (fused path: already produced by the frame kernel)
    int layers_enqueue() {
        if (use_fused() && fused_layers_ready) return FEWHA_OK;
        return inv_dwt(c, phi);
    }
    bool fused_layers_ready = false;

    long long graph_launch_count[2] = {0, 0};
};

SolverBase* make_solver(const HostSetup& hs, cudaStream_t stream, std::string& err, int& status) {
    SolverBase* out = nullptr;
    if (hs.prec == FEWHA_FP64) {
        auto* s = new Solver<double>();
        s->hs = hs;
        s->stream = stream;
        s->path = FEWHA_PATH_PLAIN;
        status = s->init();
        if (status) {
            err = s->err;
            delete s;
            return nullptr;
        }
        out = s;
    } else {
        auto* s = new Solver<float>();
        s->hs = hs;
        s->stream = stream;
        status = s->init();
        if (status) {
            err = s->err;
            delete s;
            return nullptr;
        }
        FusedBuffers fb;
        fb.c = s->c;
        fb.r = s->r;
        fb.p = s->p;
        fb.q = s->q;
        fb.b = s->b;
        fb.bprev = s->bprev;
        fb.phi = s->phi;
        fb.Jinv = s->Jinv;
        fb.aD = s->aD;
        fb.slopes = s->slopes;
        fb.sc = s->sc;
        fb.errw = s->errw;
        std::string ferr;
        s->fbuf = fb;
        s->fused = fused_create(hs, s->G, fb, ferr);
        s->path = s->fused ? FEWHA_PATH_FUSED : FEWHA_PATH_PLAIN;
        s->fused_available = s->fused != nullptr;
        s->fused_reason = ferr;
        out = s;
    }
    status = FEWHA_OK;
    return out;
}

// ---------------------------------------------------------------------------
// batch: independent FP32 instances, one fused launch per group of instances per frame
// ---------------------------------------------------------------------------

namespace {
bool host_pinned(const void* ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}
}  // namespace

class Batch : public BatchBase {
  public:
    std::vector<std::unique_ptr<Solver<float>>> inst;   // tables and state of each instance
    // The instances advance as one or more fused launches per frame, one after
    // another on the stream; a group of instances shares one plan.  One group
    // is the default; the autotuner may split the batch by layer size, so that
    // the small layers take the cluster shape and layer-phase form that suit
    // them while the large ones keep theirs.
    struct Group {
        std::vector<int> idx;   // instances, ascending
        FusedPlan* plan = nullptr;
    };
    std::vector<Group> groups;
    std::vector<const HostSetup*> hp;   // what a plan is built from (the autotuner rebuilds it)
    std::vector<DevGeo<float>> Gs;
    std::vector<FusedBuffers> fbs;
    float* s_all = nullptr;     // concatenated slopes (the instances read slices)
    float* phi_all = nullptr;   // concatenated layers (the instances write slices)
    float* pin_in = nullptr;    // staging for pageable host buffers
    float* pin_out = nullptr;

    long S_tot() const { return slope_off.back(); }
    long N_tot() const { return coeff_off.back(); }

    ~Batch() override {
        if (stream) cudaStreamSynchronize(stream);
        else cudaDeviceSynchronize();
        for (Group& g : groups) fused_destroy(g.plan);
        if (s_all) cudaFree(s_all);
        if (phi_all) cudaFree(phi_all);
        if (pin_in) cudaFreeHost(pin_in);
        if (pin_out) cudaFreeHost(pin_out);
    }

    // a plan over the instances idx (a sub-batch)
    FusedPlan* make_plan(const std::vector<int>& idx, int max_tile_side, int C, std::string& e) {
        std::vector<const HostSetup*> h;
        std::vector<DevGeo<float>> g;
        std::vector<FusedBuffers> f;
        for (int i : idx) {
            h.push_back(hp[i]);
            g.push_back(Gs[i]);
            f.push_back(fbs[i]);
        }
        return fused_create_multi(h, g, f, max_tile_side, e, C);
    }

    int set_trace(int on) override {
        if (groups.empty()) {
            err = "no fused plan";
            return FEWHA_ERR_STATE;
        }
        for (Group& g : groups) fused_set_trace(g.plan, on != 0);
        return FEWHA_OK;
    }

    // the launches' traces one after another: the CTAs of the first launch,
    // then those of the next (the timestamps are on one clock)
    int get_fine_trace(unsigned long long* out, int max_entries, int* per_cta, int* grid) override {
        if (groups.empty()) {
            err = "no fused plan";
            return FEWHA_ERR_STATE;
        }
        FEWHA_CUDA(cudaStreamSynchronize(stream));
        int tot = 0, pc = 0;
        for (Group& g : groups) {
            int p = 0, gr = 0;
            const long done = (long)pc * tot;
            unsigned long long* dst = (out && max_entries > done) ? out + done : nullptr;
            if (fused_get_fine_trace(g.plan, dst, dst ? (int)(max_entries - done) : 0, &p, &gr)) {
                err = "trace copy failed";
                return FEWHA_ERR_CUDA;
            }
            if (p == 0) {   // a launch without a trace buffer: no trace for the batch
                pc = 0;
                tot = 0;
                break;
            }
            pc = p;   // the same number of entries per CTA in every plan
            tot += gr;
        }
        *per_cta = pc;
        *grid = tot;
        return FEWHA_OK;
    }

    int frame(const void* sl, int n_iter, int warm, void* lout, int on_device) override {
        if (!sl) {
            err = "null slopes";
            return FEWHA_ERR_ARG;
        }
        if (n_iter < 1 || n_iter > 100000) {
            err = "n_iter must be >= 1";
            return FEWHA_ERR_ARG;
        }
        const size_t sb = (size_t)S_tot() * sizeof(float), nb = (size_t)N_tot() * sizeof(float);
        if (on_device) {
            FEWHA_CUDA(cudaMemcpyAsync(s_all, sl, sb, cudaMemcpyDeviceToDevice, stream));
        } else {
            const void* src = sl;
            if (!host_pinned(sl)) {
                std::memcpy(pin_in, sl, sb);   // the previous host frame has completed
                src = pin_in;
            }
            FEWHA_CUDA(cudaMemcpyAsync(s_all, src, sb, cudaMemcpyHostToDevice, stream));
        }
        const bool replace = warm && k_rr > 0 && frame_count > 0 && frame_count % k_rr == 0;
        int st = FEWHA_OK;
        for (Group& g : groups)
            if ((st = fused_solve(g.plan, nullptr, n_iter, warm, replace ? 1 : 0, barrier_budget, stream, err,
                                  launches)))
                return st;
        frame_count += 1;
        if (on_device) {
            if (lout) FEWHA_CUDA(cudaMemcpyAsync(lout, phi_all, nb, cudaMemcpyDeviceToDevice, stream));
            return FEWHA_OK;
        }
        void* dst = nullptr;
        if (lout) {
            dst = host_pinned(lout) ? lout : (void*)pin_out;
            FEWHA_CUDA(cudaMemcpyAsync(dst, phi_all, nb, cudaMemcpyDeviceToHost, stream));
        }
        st = sync();
        if (st) return st;
        if (lout && dst != lout) std::memcpy(lout, pin_out, nb);
        return FEWHA_OK;
    }

    int sync() override {
        FEWHA_CUDA(cudaStreamSynchronize(stream));
        int first = FEWHA_OK;
        for (Group& g : groups) {
            Solver<float>& s = *inst[g.idx[0]];   // a plan's error word is its first instance's
            const int st = s.check_err();
            if (st) {
                if (!first) {
                    first = st;
                    err = s.err;
                }
                fused_mark_dirty(g.plan);
            }
        }
        return first;
    }

    // Groupings of the instances by layer size (an instance's largest layer
    // side; groups are contiguous ranges of the sorted sides, one launch each)
    // and, per group, every cluster shape and sensor-tile bound that fit, timed
    // on the current slopes (n_iter warm-started iterations from the same state
    // per launch, CUDA events, median of reps).  A grouping costs the sum of
    // its groups' launches; the fastest is kept if it beats the current
    // launches timed the same way, and the instances' state is restored.
    int autotune(int n_iter, int reps, char* report, int len) override {
        if (n_iter < 1 || reps < 1 || !report || len <= 0) {
            err = "autotune needs n_iter >= 1, reps >= 1 and a report buffer";
            return FEWHA_ERR_ARG;
        }
        const long N = N_tot();
        float* saved = nullptr;
        if (cudaMalloc(&saved, 4 * (size_t)N * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            err = "autotune: no device memory for the saved state";
            return FEWHA_ERR_CUDA;
        }
        auto copy_state = [&](bool save) {
            for (size_t i = 0; i < inst.size(); ++i) {
                Solver<float>& s = *inst[i];
                const size_t n = (size_t)s.hs.N * sizeof(float);
                float* base = saved + coeff_off[i];
                float* vs[4] = {s.c, s.r, s.b, s.bprev};
                for (int v = 0; v < 4; ++v) {
                    float* slot = base + (size_t)v * N;
                    if (cudaMemcpyAsync(save ? slot : vs[v], save ? vs[v] : slot, n, cudaMemcpyDeviceToDevice,
                                        stream) != cudaSuccess)
                        return false;
                }
            }
            return true;
        };
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int st = FEWHA_OK;
        std::string rep;
        // median launch time of a plan over the instances whose first is lead
        auto time_plan = [&](FusedPlan* pl, int lead) -> float {
            std::vector<float> ts;
            long long dummy = 0;
            for (int r = 0; r <= reps && st == FEWHA_OK; ++r) {
                if (!copy_state(false)) st = FEWHA_ERR_CUDA;
                cudaEventRecord(e0, stream);
                if (st == FEWHA_OK) st = fused_solve(pl, nullptr, n_iter, 1, 0, barrier_budget, stream, err, dummy);
                cudaEventRecord(e1, stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) st = FEWHA_ERR_CUDA;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) ts.push_back(ms * 1e3f);   // the first launch warms up
            }
            if (st == FEWHA_OK && (st = inst[lead]->check_err()) != FEWHA_OK) err = inst[lead]->err;
            if (ts.empty()) return -1.f;
            std::sort(ts.begin(), ts.end());
            return ts[ts.size() / 2];
        };
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess || !copy_state(true)) {
            cudaGetLastError();
            st = FEWHA_ERR_CUDA;
            err = "autotune: events or state copy";
        }
        float cur_t = 0.f;
        for (Group& g : groups) {
            if (st != FEWHA_OK) break;
            const float t = time_plan(g.plan, g.idx[0]);
            cur_t = (t > 0.f && cur_t >= 0.f) ? cur_t + t : -1.f;
        }
        {
            char b[96];
            snprintf(b, sizeof b, "current: %.1f us in %d launch%s", cur_t, (int)groups.size(),
                     groups.size() == 1 ? "" : "es");
            rep = b;
        }
        // the sorted distinct sides; a range [a, b] of them is a group
        const int ni = (int)inst.size();
        std::vector<int> side(ni, 0);
        for (int i = 0; i < ni; ++i)
            for (int l = 0; l < inst[i]->hs.L; ++l) side[i] = std::max(side[i], inst[i]->hs.lay[l].n);
        std::vector<int> sides(side);
        std::sort(sides.begin(), sides.end());
        sides.erase(std::unique(sides.begin(), sides.end()), sides.end());
        const int k = (int)sides.size();
        struct Cand {
            std::vector<int> idx;
            FusedPlan* plan = nullptr;
            float t = -1.f;
            int C = 0, tile = 0;
        };
        std::vector<Cand> ranges((size_t)k * k);   // [a * k + b], filled on first use
        std::vector<char> tuned((size_t)k * k, 0);
        auto tune_range = [&](int a, int b) -> Cand& {
            Cand& c = ranges[(size_t)a * k + b];
            if (tuned[(size_t)a * k + b]) return c;
            tuned[(size_t)a * k + b] = 1;
            for (int i = 0; i < ni; ++i)
                if (side[i] >= sides[a] && side[i] <= sides[b]) c.idx.push_back(i);
            for (int C : {8, 4, 16, 2}) {
                for (int tile : {0, 64, 48, 32, 24, 16}) {
                    if (st != FEWHA_OK) break;
                    std::string e;
                    FusedPlan* pl = make_plan(c.idx, tile, C, e);
                    if (!pl) continue;
                    const float t = time_plan(pl, c.idx[0]);
                    if (t > 0.f && (c.t <= 0.f || t < c.t)) {
                        if (c.plan) fused_destroy(c.plan);
                        c.plan = pl;
                        c.t = t;
                        c.C = C;
                        c.tile = tile;
                    } else {
                        fused_destroy(pl);
                    }
                }
            }
            char b2[128];
            snprintf(b2, sizeof b2, "; sides %d-%d (%d instances): C=%d tile<=%d %.1f us", sides[a], sides[b],
                     (int)c.idx.size(), c.C, c.tile, c.t);
            rep += b2;
            return c;
        };
        // groupings: cuts between consecutive sides (all of them for up to
        // four sides, else one cut at most; fewer under a launch bound)
        int best_mask = -1;
        float best_t = -1.f;
        int max_cuts = k <= 4 ? k - 1 : 1;
        if (max_launches > 0) max_cuts = std::min(max_cuts, max_launches - 1);
        for (int mask = 0; k > 0 && mask < (1 << (k - 1)) && st == FEWHA_OK; ++mask) {
            if (__builtin_popcount(mask) > max_cuts) continue;
            float tot = 0.f;
            for (int a = 0, j = 0; j < k; ++j) {
                if (j < k - 1 && !(mask >> j & 1)) continue;
                const Cand& c = tune_range(a, j);
                tot = (c.t > 0.f && tot >= 0.f) ? tot + c.t : -1.f;
                a = j + 1;
            }
            if (tot > 0.f && (best_t <= 0.f || tot < best_t)) {
                best_t = tot;
                best_mask = mask;
            }
        }
        const bool cur_ok = max_launches <= 0 || (int)groups.size() <= max_launches;
        if (st == FEWHA_OK && best_mask >= 0 && (cur_t <= 0.f || best_t < cur_t || !cur_ok)) {
            for (Group& g : groups) fused_destroy(g.plan);
            groups.clear();
            for (int a = 0, j = 0; j < k; ++j) {
                if (j < k - 1 && !(best_mask >> j & 1)) continue;
                Cand& c = ranges[(size_t)a * k + j];
                groups.push_back(Group{c.idx, c.plan});
                c.plan = nullptr;   // owned by the group now
                a = j + 1;
            }
            char b[96];
            snprintf(b, sizeof b, "; chosen: %d launch%s, %.1f us", (int)groups.size(),
                     groups.size() == 1 ? "" : "es", best_t);
            rep += b;
        } else {
            rep += "; kept the current launches";
        }
        for (Cand& c : ranges)
            if (c.plan) fused_destroy(c.plan);
        if (!copy_state(false)) st = st ? st : FEWHA_ERR_CUDA;
        cudaStreamSynchronize(stream);
        cudaFree(saved);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        snprintf(report, len, "%s", rep.c_str());
        return st;
    }

    // group[i]: the launch of instance i (0 .. G - 1, every launch non-empty);
    // one plan per launch, built with the batch's tile bound and cluster
    // shape.  On any failure the current launches stay.
    int set_groups(const int* group, int count) override {
        const int ni = (int)inst.size();
        if (!group || count != ni) {
            err = "set_groups needs one launch index per instance";
            return FEWHA_ERR_ARG;
        }
        int G = 0;
        for (int i = 0; i < ni; ++i) {
            if (group[i] < 0 || group[i] >= ni) {
                err = "launch index out of range";
                return FEWHA_ERR_ARG;
            }
            G = std::max(G, group[i] + 1);
        }
        std::vector<Group> ng(G);
        for (int i = 0; i < ni; ++i) ng[group[i]].idx.push_back(i);
        for (Group& g : ng)
            if (g.idx.empty()) {
                err = "every launch index below the largest must have an instance";
                return FEWHA_ERR_ARG;
            }
        FEWHA_CUDA(cudaStreamSynchronize(stream));   // the current plans may be in flight
        for (size_t g = 0; g < ng.size(); ++g) {
            std::string e;
            ng[g].plan = make_plan(ng[g].idx, max_tile_side, cluster_size, e);
            if (!ng[g].plan) {
                for (Group& h : ng)
                    if (h.plan) fused_destroy(h.plan);
                err = "no fused plan for launch " + std::to_string(g) + ": " + e;
                return FEWHA_ERR_GEOMETRY;
            }
        }
        for (Group& g : groups) fused_destroy(g.plan);
        groups = std::move(ng);
        return FEWHA_OK;
    }

    int describe(char* buf, int len) override {
        if (!buf || len <= 0) {
            err = "null buffer";
            return FEWHA_ERR_ARG;
        }
        int k = snprintf(buf, len, "batch of %d fp32 instances, N %ld, S %ld, %d launch%s per frame", (int)inst.size(),
                         N_tot(), S_tot(), (int)groups.size(), groups.size() == 1 ? "" : "es");
        for (size_t g = 0; g < groups.size() && k >= 0 && k < len; ++g) {
            const int m = groups.size() == 1 ? snprintf(buf + k, len - k, "; ")
                                             : snprintf(buf + k, len - k, "; launch %d (%d instances): ", (int)g,
                                                        (int)groups[g].idx.size());
            if (m < 0) break;
            k += m;
            if (k >= len) break;
            const int f = fused_describe(groups[g].plan, buf + k, len - k);
            if (f < 0) break;
            k += f;
        }
        return FEWHA_OK;
    }

    int get_state(int i, void* c, void* b, void* r, int on_device) override {
        if (i < 0 || i >= (int)inst.size()) {
            err = "instance index out of range";
            return FEWHA_ERR_ARG;
        }
        const int st = inst[i]->get_state(c, b, r, on_device);
        if (st) err = inst[i]->err;
        return st;
    }
};

BatchBase* make_batch(const std::vector<HostSetup>& hss, cudaStream_t stream, int max_tile_side,
                      int cluster_size, std::string& err, int& status) {
    std::unique_ptr<Batch> B(new Batch());
    B->stream = stream;
    B->max_tile_side = max_tile_side;
    B->cluster_size = cluster_size;
    B->coeff_off.assign(1, 0);
    B->slope_off.assign(1, 0);
    for (size_t i = 0; i < hss.size(); ++i) {
        if (hss[i].any_tt) {
            err = "batched instances do not model the LGS tip-tilt filter";
            status = FEWHA_ERR_ARG;
            return nullptr;
        }
        if (hss[i].prec != FEWHA_FP32) {
            err = "batched instances are FP32 only";
            status = FEWHA_ERR_ARG;
            return nullptr;
        }
        std::unique_ptr<Solver<float>> s(new Solver<float>());
        s->hs = hss[i];
        s->stream = stream;
        s->path = FEWHA_PATH_PLAIN;
        status = s->init();
        if (status) {
            err = "instance " + std::to_string(i) + ": " + s->err;
            return nullptr;
        }
        B->coeff_off.push_back(B->coeff_off.back() + hss[i].N);
        B->slope_off.push_back(B->slope_off.back() + hss[i].S);
        B->inst.push_back(std::move(s));
    }
    const size_t sb = (size_t)B->S_tot() * sizeof(float), nb = (size_t)B->N_tot() * sizeof(float);
    if (cudaMalloc(&B->s_all, sb) != cudaSuccess || cudaMalloc(&B->phi_all, nb) != cudaSuccess ||
        cudaMallocHost(&B->pin_in, sb) != cudaSuccess || cudaMallocHost(&B->pin_out, nb) != cudaSuccess ||
        cudaMemset(B->s_all, 0, sb) != cudaSuccess) {
        cudaGetLastError();
        err = "device or pinned host allocation of the batch buffers failed";
        status = FEWHA_ERR_CUDA;
        return nullptr;
    }
    std::vector<const HostSetup*>& hp = B->hp;
    std::vector<DevGeo<float>>& Gs = B->Gs;
    std::vector<FusedBuffers>& fbs = B->fbs;
    for (size_t i = 0; i < B->inst.size(); ++i) {
        Solver<float>& s = *B->inst[i];
        FusedBuffers fb;
        fb.c = s.c;
        fb.r = s.r;
        fb.p = s.p;
        fb.q = s.q;
        fb.b = s.b;
        fb.bprev = s.bprev;
        fb.phi = B->phi_all + B->coeff_off[i];
        fb.Jinv = s.Jinv;
        fb.aD = s.aD;
        fb.slopes = B->s_all + B->slope_off[i];
        fb.sc = s.sc;
        fb.errw = s.errw;
        hp.push_back(&s.hs);
        Gs.push_back(s.G);
        fbs.push_back(fb);
    }
    Batch::Group all;
    for (int i = 0; i < (int)B->inst.size(); ++i) all.idx.push_back(i);
    all.plan = B->make_plan(all.idx, max_tile_side, cluster_size, err);
    if (all.plan) B->groups.push_back(all);
    if (!all.plan) {
        err = "no fused plan for this batch: " + err;
        status = FEWHA_ERR_GEOMETRY;
        return nullptr;
    }
    status = FEWHA_OK;
    return B.release();
}

}  // namespace fewha
