// Reverse mode through the fixed-iteration solve (K steps of Alg. 2 from a
// cold start, Alg. 1), for gradients of a loss on the layers with respect to
// the Cn^2 fractions gamma_l, the regularisation weight alpha and the sensor
// weights w_g, with the Jacobi preconditioner held fixed.  Included by
// solver.cu inside namespace fewha, after DevGeo, block_sum and the Alg. 2
// scalar slots.
#pragma once

// Tape of B differentiable solves run together (B = 1: one solve): per
// iteration k the vectors r_k (before the update), z_k = J^{-1} r_k,
// s_k = M z_k, p_k, q_k (after the update), each as B frames of N values
// ([k][vector][frame][N]), then per iteration and frame 8 doubles (rho, mu,
// beta, d, alpha, rho_{k-1}, alpha_{k-1}, unused), [k][frame][8].
enum TapeVec { kTapeR = 0, kTapeZ, kTapeS, kTapeP, kTapeQ, kTapeVecs };
enum TapeScalar { kTRho = 0, kTMu, kTBeta, kTD, kTAlpha, kTRhoOld, kTAlphaOld, kTapeScalars = 8 };

inline size_t tape_vec_bytes(long N, int n_iter, size_t elem, int B = 1) {
    const size_t b = (size_t)n_iter * kTapeVecs * (size_t)N * (size_t)B * elem;
    return (b + 255) & ~(size_t)255;
}
inline size_t tape_bytes(long N, int n_iter, size_t elem, int B = 1) {
    return tape_vec_bytes(N, n_iter, elem, B) + (size_t)n_iter * (size_t)B * kTapeScalars * sizeof(double);
}

// Record the scalars of iteration k (after k_alg2_scalars); one block per
// frame of the batch (gridDim.x frames).
__global__ void k_tape_scalars(const double* __restrict__ sc, double* __restrict__ ts, int k) {
    if (threadIdx.x != 0) return;
    const int f = blockIdx.x, B = gridDim.x;
    sc += (size_t)f * kNumScalars;
    double* t = ts + ((size_t)k * B + f) * kTapeScalars;
    const double rho = sc[kRho], mu = sc[kMu], beta = sc[kBeta], alpha = sc[kAlphaK];
    double rho_old = 0.0, alpha_old = 0.0, d = mu;
    if (k > 0) {
        rho_old = ts[((size_t)(k - 1) * B + f) * kTapeScalars + kTRho];
        alpha_old = ts[((size_t)(k - 1) * B + f) * kTapeScalars + kTAlpha];
        d = mu - rho * beta / alpha_old;
    }
    t[kTRho] = rho;
    t[kTMu] = mu;
    t[kTBeta] = beta;
    t[kTD] = d;
    t[kTAlpha] = alpha;
    t[kTRhoOld] = rho_old;
    t[kTAlphaOld] = alpha_old;
    t[7] = 0.0;
}

// Six partial dots of the reverse step k: (cb, p_k), (rb, q_k), (pb, p_{k-1}),
// (cb, p_{k-1}), (qb, q_{k-1}), (rb, q_{k-1}); the last four only for k > 0.
template <typename T>
__global__ void k_adj_dots(int N, const T* __restrict__ cb, const T* __restrict__ rb, const T* __restrict__ pb,
                           const T* __restrict__ qb, const T* __restrict__ pk, const T* __restrict__ qk,
                           const T* __restrict__ pold, const T* __restrict__ qold, double* __restrict__ part) {
    __shared__ double sh[32];
    const long fo = (long)blockIdx.z * N;   // frame blockIdx.z of a batch
    cb += fo;
    rb += fo;
    pb += fo;
    qb += fo;
    pk += fo;
    qk += fo;
    if (pold) {
        pold += fo;
        qold += fo;
    }
    part += (size_t)blockIdx.z * 6 * kRedBlocks;
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double c = cb[i], r = rb[i];
        a[0] += c * (double)pk[i];
        a[1] += r * (double)qk[i];
        if (pold) {
            const double po = pold[i], qo = qold[i];
            a[2] += (double)pb[i] * po;
            a[3] += c * po;
            a[4] += (double)qb[i] * qo;
            a[5] += r * qo;
        }
    }
    for (int j = 0; j < 6; ++j) {
        double v = block_sum(a[j], sh);
        if (threadIdx.x == 0) part[j * kRedBlocks + blockIdx.x] = v;
        __syncthreads();
    }
}

// Adjoint scalars of step k.  asc: [0] alpha_k, [1] beta_k, [2] mu-bar,
// [3] rho-bar, [4] alpha-bar carried to step k-1, [5] rho-bar carried to k-1.
__global__ void k_adj_scalars(const double* __restrict__ part, const double* __restrict__ ts, int k,
                              double* __restrict__ asc) {
    __shared__ double sh[32];
    const int f = blockIdx.x, B = gridDim.x;   // one block per frame
    part += (size_t)f * 6 * kRedBlocks;
    asc += (size_t)f * 8;
    double D[6];
    for (int j = 0; j < 6; ++j) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) acc += part[j * kRedBlocks + i];
        D[j] = block_sum(acc, sh);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double* t = ts + ((size_t)k * B + f) * kTapeScalars;
    const double rho = t[kTRho], beta = t[kTBeta], d = t[kTD], alpha = t[kTAlpha];
    const double alphab = asc[4] + D[0] - D[1];
    double betab = k > 0 ? (D[2] + alpha * D[3]) + (D[4] - alpha * D[5]) : 0.0;
    double rhob = asc[5] + alphab / d;
    const double db = -alphab * rho / (d * d);
    double alphab_prev = 0.0, rhob_prev = 0.0;
    if (k > 0) {
        const double ao = t[kTAlphaOld], ro = t[kTRhoOld];
        rhob -= db * beta / ao;
        betab -= db * rho / ao;
        alphab_prev = db * rho * beta / (ao * ao);
        rhob += betab / ro;
        rhob_prev = -betab * rho / (ro * ro);
    }
    asc[0] = alpha;
    asc[1] = beta;
    asc[2] = db;   // mu-bar = d-bar
    asc[3] = rhob;
    asc[4] = alphab_prev;
    asc[5] = rhob_prev;
}

// pb += alpha cb ; qb -= alpha rb ; sb = qb + mu-bar z_k
template <typename T>
__global__ void k_adj_vec1(int N, const double* __restrict__ asc, const T* __restrict__ cb, const T* __restrict__ rb,
                           T* __restrict__ pb, T* __restrict__ qb, const T* __restrict__ zk, T* __restrict__ sb) {
    const long fo = (long)blockIdx.z * N;
    asc += (size_t)blockIdx.z * 8;
    cb += fo;
    rb += fo;
    pb += fo;
    qb += fo;
    zk += fo;
    sb += fo;
    const T a = (T)asc[0], mub = (T)asc[2];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        pb[i] += a * cb[i];
        const T q = qb[i] - a * rb[i];
        qb[i] = q;
        sb[i] = q + mub * zk[i];
    }
}

// zb = pb + mu-bar s_k + rho-bar r_k + M sb ; rb += rho-bar z_k + J^{-1} zb ;
// pb = beta pb ; qb = beta qb
template <typename T>
__global__ void k_adj_vec2(int N, const double* __restrict__ asc, T* __restrict__ pb, T* __restrict__ qb,
                           T* __restrict__ rb, const T* __restrict__ zk, const T* __restrict__ sk,
                           const T* __restrict__ rk, const T* __restrict__ Msb, const T* __restrict__ Jinv) {
    const long fo = (long)blockIdx.z * N;
    asc += (size_t)blockIdx.z * 8;
    pb += fo;
    qb += fo;
    rb += fo;
    zk += fo;
    sk += fo;
    rk += fo;
    Msb += fo;
    const T beta = (T)asc[1], mub = (T)asc[2], rhob = (T)asc[3];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const T zb = pb[i] + mub * sk[i] + rhob * rk[i] + Msb[i];
        rb[i] += rhob * zk[i] + Jinv[i] * zb;
        pb[i] *= beta;
        qb[i] *= beta;
    }
}

// Per-layer partials of sum_i sb_i (alpha D)_i z_i: part[l * kRedBlocks + block]
template <typename T>
__global__ void k_layer_dot(DevGeo<T> G, const T* __restrict__ a, const T* __restrict__ w, const T* __restrict__ b,
                            double* __restrict__ part) {
    __shared__ double sh[32];
    const int l = blockIdx.y, n = G.lay_n[l], off = G.lay_off[l];
    a += (long)blockIdx.z * G.N;   // w (alpha D) is shared by the frames
    b += (long)blockIdx.z * G.N;
    part += (size_t)blockIdx.z * G.L * kRedBlocks;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * n; i += gridDim.x * blockDim.x)
        acc += (double)a[off + i] * (double)w[off + i] * (double)b[off + i];
    const double v = block_sum(acc, sh);
    if (threadIdx.x == 0) part[l * kRedBlocks + blockIdx.x] = v;
}

// Per-sensor partials of sum over active subapertures of (Gamma psiA).(Gamma
// psiB) (psiB != NULL) or of (Gamma psiA).s (measured slopes s, finite only).
template <typename T>
__global__ void k_wfs_dot(DevGeo<T> G, const T* __restrict__ psiA, const T* __restrict__ psiB,
                          const T* __restrict__ s, double* __restrict__ part) {
    __shared__ double sh[32];
    const int g = blockIdx.y, ns = G.wfs_n[g], np1 = ns + 1;
    psiA += (long)blockIdx.z * G.NW;
    if (psiB) psiB += (long)blockIdx.z * G.NW;
    else s += (long)blockIdx.z * G.S;
    part += (size_t)blockIdx.z * G.G * kRedBlocks;
    double acc = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ns * ns; idx += gridDim.x * blockDim.x) {
        if (!G.mask[G.wfs_moff[g] + idx]) continue;
        const int a = idx / ns, b = idx - a * ns;
        const T* p = psiA + G.wfs_noff[g] + (long)a * np1 + b;
        const double ax = ((p[1] - p[0]) + (p[np1 + 1] - p[np1])) / 2;
        const double ay = ((p[np1] - p[0]) + (p[np1 + 1] - p[1])) / 2;
        double bx, by;
        if (psiB) {
            const T* q = psiB + G.wfs_noff[g] + (long)a * np1 + b;
            bx = ((q[1] - q[0]) + (q[np1 + 1] - q[np1])) / 2;
            by = ((q[np1] - q[0]) + (q[np1 + 1] - q[1])) / 2;
        } else {
            bx = s[G.wfs_soff[g] + idx];
            by = s[G.wfs_soff[g] + ns * ns + idx];
            if (!isfinite(bx) || !isfinite(by)) continue;
        }
        acc += ax * bx + ay * by;
    }
    const double v = block_sum(acc, sh);
    if (threadIdx.x == 0) part[g * kRedBlocks + blockIdx.x] = v;
}

// Accumulate the contractions into the gradients (FP64, fixed order):
// layer sums S_l = sum sb (alpha D) z give dgamma_l -= S_l / gamma_l and
// dalpha += S_l / alpha; sensor sums give dw_g += sum.
__global__ void k_adj_accum(const double* __restrict__ lpart, int L, const double* __restrict__ wpart, int G,
                            const double* __restrict__ gam, double alpha, double* __restrict__ g_gam,
                            double* __restrict__ g_alpha, double* __restrict__ g_w) {
    __shared__ double sh[32];
    const int f = blockIdx.x;   // one block per frame: its own gradients
    if (lpart) lpart += (size_t)f * L * kRedBlocks;
    if (wpart) wpart += (size_t)f * G * kRedBlocks;
    g_gam += (size_t)f * L;
    g_alpha += f;
    g_w += (size_t)f * G;
    double alpha_acc = 0.0;
    for (int l = 0; l < L && lpart; ++l) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) acc += lpart[l * kRedBlocks + i];
        const double S = block_sum(acc, sh);
        __syncthreads();
        if (threadIdx.x == 0) {
            g_gam[l] -= S / gam[l];
            alpha_acc += S / alpha;
        }
    }
    for (int g = 0; g < G && wpart; ++g) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) acc += wpart[g * kRedBlocks + i];
        const double S = block_sum(acc, sh);
        __syncthreads();
        if (threadIdx.x == 0) g_w[g] += S;
    }
    if (threadIdx.x == 0 && lpart) *g_alpha += alpha_acc;
}
